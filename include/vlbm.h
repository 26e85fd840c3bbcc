/*
 * vlbm.h -- C ABI of the GB300-native vectorial lattice Boltzmann library
 * (fused collide-and-stream update of the MHD conserved variables, each on
 * its own small velocity set with a flux-carrying equilibrium).
 *
 * Paper passages implemented behind this interface (equations numbered in
 * the order the paper displays them):
 *   Eq. 2  fully local VLBM update: BGK collision, source injection, stream
 *   Eq. 3  first-order equilibrium f_eq_ki = w_i (Q_k + c_i . Phi_k / cs^2)
 *   Eq. 4  moments Q_k = sum_i f_ki
 *   Eq. 9  EOS p = (gamma - 1)(e_tot - rho|u|^2/2 - |B|^2/2)
 *   Eq. 12 ideal MHD state (rho, rho u, e_tot, B) and flux
 *   sec. 2.3 "Incompressible resistive MHD" with sec. 2.4 "Static
 *   boundaries" for the resistive channel model (D3Q19 flow lattice with a
 *   second-order equilibrium carrying the Maxwell stress, three D3Q7
 *   magnetic lattices with the Eq. 3 equilibrium, Guo body force, halfway
 *   bounce-back walls at y = 0 and ny-1, magnetic walls held at the
 *   equilibrium of the applied field).
 *   sec. 2.2.1 local moments evolution with sec. 2.3 "Evolution of the MHD
 *   equation system" for the dissipative model (viscous stress, eta(j)
 *   resistivity, gradients carried as lattices; VLBM_DISSIPATIVE).
 *
 * Conventions for every call
 *   - Lattice units: dx = dt = 1.  Fields are double precision, structure of
 *     arrays: Q[v * N + cell], cell = x + nx * (y + ny * z), x fastest,
 *     N = nx * ny * nz.  Ideal MHD has nvar = 8 fields (rho, rho u_x,
 *     rho u_y, rho u_z, e_tot, B_x, B_y, B_z); the resistive model has
 *     nvar = 7 (rho, m_x, m_y, m_z, B_x, B_y, B_z), where m includes the
 *     half-force shift of the Guo scheme; the Powell model adds D (nvar = 9)
 *     and the dissipative model G and W (nvar = 20 in 2-D, 26 in 3-D, see
 *     vlbm_model).
 *   - Velocity sets and direction order: D2Q5 (w0 = 1/3, w = 1/6,
 *     cs^2 = 1/3), D3Q7 (w0 = 1/4, w = 1/8, cs^2 = 1/4), D3Q19 (1/3, 1/18,
 *     1/36, cs^2 = 1/3).  Direction 0 is rest; 1 +x, 2 -x, 3 +y, 4 -y,
 *     5 +z, 6 -z; D3Q19 continues 7 (+1,+1,0) 8 (-1,-1,0) 9 (+1,-1,0)
 *     10 (-1,+1,0) 11 (+1,0,+1) 12 (-1,0,-1) 13 (+1,0,-1) 14 (-1,0,+1)
 *     15 (0,+1,+1) 16 (0,-1,-1) 17 (0,+1,-1) 18 (0,-1,+1).
 *   - Ownership: the caller owns every host and device array it passes and
 *     keeps it alive for the duration of the call; the library copies.
 *     The context owns all device memory it allocates (through the
 *     optional allocator hooks) and releases it in vlbm_destroy.
 *   - Streams: all device work of a context is enqueued on its stream
 *     (params.stream, or a stream the library creates when it is NULL).
 *     Calls that return host data synchronise that stream.  Device inputs
 *     must be complete before a call enqueues work that reads them, and
 *     device outputs are ready only after the context's stream reaches the
 *     call's work: order other streams against the context's stream (events
 *     or synchronisation) -- a stream created with cudaStreamNonBlocking does
 *     not wait for the legacy default stream.
 *   - Errors: every call returns a vlbm_status; vlbm_last_error() gives a
 *     one-line reason.  After VLBM_ERR_NONPHYSICAL or VLBM_ERR_TIMEOUT the
 *     context is sticky-failed (vlbm_step returns the error) until
 *     vlbm_init_fields or vlbm_load succeeds.  A NULL context or a
 *     non-positive size is VLBM_ERR_ARG.  No call aborts the process.
 */
#ifndef VLBM_H
#define VLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vlbm_ctx vlbm_ctx;

typedef enum {
    VLBM_OK = 0,
    VLBM_ERR_ARG = 1,          /* invalid argument or size */
    VLBM_ERR_UNSTABLE = 2,     /* tau <= 1/2, or max(|u| + c_f) >= cs at init */
    VLBM_ERR_OOM = 3,          /* device allocation failed */
    VLBM_ERR_CUDA = 4,         /* a CUDA runtime call failed */
    VLBM_ERR_NONPHYSICAL = 5,  /* NaN, rho <= 0 or p <= 0 seen by a kernel */
    VLBM_ERR_TIMEOUT = 6,      /* a bounded device wait expired */
    VLBM_ERR_STATE = 7,        /* call not valid in the context's state */
    VLBM_ERR_UNSUPPORTED = 8   /* combination of options not built */
} vlbm_status;

/* VLBM_IDEAL_POWELL: ideal MHD with Powell's source S = -(div B)(0, B, u.B, u)
 * (sec. 2.3, "Powell correction"), div B taken locally from a ninth lattice
 * that carries D, the trace of the gradient tensor of the local moments
 * evolution (sec. 2.2.1; flux D u - B, relaxation source -D / tau_m), as
 * div B = D / tau_m.  Nine fields: the eight of VLBM_IDEAL, then D.  Built
 * for F64 and F32 storage, single domains. */
/* VLBM_DISSIPATIVE: the full dissipative MHD system (sec. 2.3, "Evolution of
 * the MHD equation system" and "Incompressible resistive MHD") with the
 * gradients it needs evolved locally (sec. 2.2.1): besides the eight fields of
 * Eq. 12 the state carries G_ab ~ tau_m d_a B_b (flux G_ab u_c - delta_ac B_b)
 * and W_ab ~ tau_m d_a u_b (flux W_ab u_c - delta_ac u_b), a over the lattice
 * axes, b in {x, y, z}, both relaxed by the source -G / tau_m, -W / tau_m.
 * 2-D (D2Q5, 100 populations per cell), twenty fields: rho, rho u (3),
 * e_tot, B (3), then G_ab at 8 + 3a + b and W_ab at 14 + 3a + b, a in {x, y},
 * d_z = 0.  3-D (D3Q7, 182 populations per cell), twenty-six fields: G_ab at
 * 8 + 3a + b and W_ab at 17 + 3a + b, a in {x, y, z}.  The MHD fluxes add the
 * viscous stress rho nu (grad u + grad u^T), -eta grad B in the induction flux
 * and -u . tau_v + eta j x B in the energy flux (no heat flux), with
 * j = curl B and eta = eta0 (1 + |j|^2 / j_c^2) (j_c <= 0: eta = eta0);
 * params.powell adds Powell's source with div B = trace(G) / tau_m.  F64 and
 * F32 storage. */
typedef enum { VLBM_IDEAL = 0, VLBM_RESISTIVE = 1, VLBM_IDEAL_POWELL = 2, VLBM_DISSIPATIVE = 3 } vlbm_model;

/* Population storage.  F64: double storage and arithmetic.  F32: float
 * storage and arithmetic.  F16_DEV / BF16_DEV: populations stored as
 * half / bfloat16 shifted deviations (f_ki - w_i q_ref_k) / q_scale_k,
 * decoded to float for the arithmetic, except the gas pressure of cells
 * below params.p_theta and the moments read back (vlbm_moments,
 * vlbm_conservation), which decode the FP32 sum of a cell's deviations in
 * FP64. */
typedef enum { VLBM_F64 = 0, VLBM_F32 = 1, VLBM_F16_DEV = 2, VLBM_BF16_DEV = 3 } vlbm_storage;

typedef void *(*vlbm_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*vlbm_free_fn)(void *ptr, size_t bytes, void *stream, void *user);

typedef struct {
    int model;            /* vlbm_model */
    int dim;              /* 2 (D2Q5 lattices) or 3 (D3Q7); resistive: 3 */
    int nx, ny, nz;       /* cells per axis, nz = 1 when dim = 2 */
    int storage;          /* vlbm_storage */
    double gamma;         /* ideal: adiabatic index of the EOS (Eq. 9) */
    double tau[8];        /* BGK relaxation time per lattice (Eq. 2), > 1/2.
                             ideal, Powell, dissipative: one per MHD field;
                             resistive: tau[0] flow lattice, tau[1..3] magnetic */
    double source[8];     /* ideal: uniform direct-injection source S_k
                             (f* += w_i S_k); zero for the Eq. 12 system */
    double force[3];      /* resistive: body force per cell (Guo scheme) */
    double b_wall[3];     /* resistive: field held by the magnetic walls */
    int walls_y;          /* resistive: 1 = solid rows y = 0 and ny - 1 */
    int check_every;      /* read the device health flag back every this many
                             steps (0: only at vlbm_sync / vlbm_moments) */
    double q_ref[8];      /* deviation storage: reference state per lattice */
    double q_scale[8];    /* deviation storage: scale per lattice (0 -> 1) */
    void *stream;         /* cudaStream_t to enqueue on, or NULL */
    vlbm_alloc_fn alloc;  /* device allocator hook, or NULL for cudaMalloc */
    vlbm_free_fn dealloc; /* matching release hook */
    void *alloc_user;     /* passed back to the hooks */
    double tau_d;         /* Powell model: BGK relaxation time of the D lattice, > 1/2 */
    double tau_m;         /* Powell model: relaxation time of D in time steps (source
                             -D / tau_m; div B = D / tau_m), > 1/2; dissipative model:
                             relaxation time of G and W in time steps */
    double tau_g;         /* dissipative model: BGK relaxation time of the gradient
                             lattices (G, W: 12 in 2-D, 18 in 3-D), > 1/2; tau[0..7]
                             serve the eight MHD lattices */
    double nu;            /* dissipative model: kinematic viscosity (lattice units), >= 0 */
    double eta0;          /* dissipative model: resistivity at zero current, >= 0 */
    double j_c;           /* dissipative model: current scale of eta(j); <= 0: constant eta0 */
    int powell;           /* dissipative model: 1 adds Powell's source */
    double p_theta;       /* deviation storage (F16_DEV, BF16_DEV): a cell whose FP32 gas
                             pressure is below p_theta * e_tot (near vacuum, high Mach, low
                             beta: p is a small difference of large terms) recomputes p in
                             FP64 from the FP64 reference state q_ref + q_scale * (FP32 sum
                             of its stored deviations); >= 0, 0 disables */
} vlbm_params;

/* Fill *p with defaults: ideal MHD, dim 3, 64^3 cells, F32 storage,
 * gamma = 5/3, tau = 0.51 on every lattice (the paper's showcase value,
 * sec. 5 table), no source, no walls, check_every = 0, NULL hooks;
 * Powell model: tau_d = 0.51, tau_m = 1; dissipative model: tau_g = 0.51,
 * nu = eta0 = j_c = 0, no Powell source; p_theta = 0.01. */
void vlbm_default_params(vlbm_params *p);

/* Create a context for one domain: validates p (dims > 0, dim 2 => nz = 1,
 * tau > 1/2, gamma > 1, storage/model combination built), allocates the
 * single in-place population buffer (nvar lattices x q directions x N
 * cells in the storage type) and a few words of status memory. */
vlbm_status vlbm_create(const vlbm_params *p, vlbm_ctx **out);

/* Create one context holding `count` independent periodic 2-D ideal-MHD
 * domains (p[d] describes domain d; each may have its own size, gamma and
 * tau).  All domains advance together: one vlbm_step launch covers every
 * domain through a tile table.  Only F32 storage, dim 2, ideal model. */
vlbm_status vlbm_create_batch(const vlbm_params *p, int count, vlbm_ctx **out);

/* Set domain `domain` to f = f_eq(Q) (Eq. 3) from host fields Q
 * (nvar x N doubles, lattice units) and reset its step count to 0.
 * Returns VLBM_ERR_UNSTABLE when max(|u| + c_f) >= cs on some cell
 * (c_f^2 = (gamma p + |B|^2)/rho; the scheme's diffusion
 * (tau - 1/2)(cs^2 - a^2) would be negative), VLBM_ERR_NONPHYSICAL when
 * some cell has NaN, rho <= 0 or p <= 0 (this takes precedence).  Either
 * error leaves the populations written but the status word clear.
 * Synchronises the stream. */
vlbm_status vlbm_init_fields(vlbm_ctx *ctx, int domain, const double *Q_host);

/* As vlbm_init_fields from single-precision host fields (nvar x N floats):
 * the host link carries half the bytes (it bounds the host-field calls: about
 * 200 GB/s each way on a GB300), and the device widens each staged chunk to
 * double before the same init kernel, so the result equals vlbm_init_fields on
 * the fields rounded to float -- bit for bit the same populations wherever
 * the init arithmetic rounds its inputs to float first (ideal, Powell and
 * dissipative models with F32 storage).  The FP64 pressure check of 16-bit
 * storage sees the rounded fields.  F64 storage: VLBM_ERR_UNSUPPORTED (use
 * vlbm_init_fields).  No counterpart in the paper (host interface only). */
vlbm_status vlbm_init_fields_f32(vlbm_ctx *ctx, int domain, const float *Q_host);

/* As vlbm_init_fields, Q_dev a device pointer (nvar x N doubles). */
vlbm_status vlbm_init_fields_device(vlbm_ctx *ctx, int domain, const double *Q_dev);

/* Enqueue n >= 0 time steps of Eq. 2 on every domain: one fused
 * collide-and-stream kernel per step (in-place AA pattern), asynchronous.
 * Returns the sticky status from the last health flag read back (a NaN,
 * rho <= 0 or p <= 0 seen by a step kernel gives VLBM_ERR_NONPHYSICAL). */
vlbm_status vlbm_step(vlbm_ctx *ctx, int n);

/* Wait for the context's stream and return the health status. */
vlbm_status vlbm_sync(vlbm_ctx *ctx);

/* Zeroth moments Q_k = sum_i f_ki (Eq. 4) of domain `domain` at the
 * current step, nvar x N doubles into host memory (synchronises). */
vlbm_status vlbm_moments(vlbm_ctx *ctx, int domain, double *Q_host);

/* As vlbm_moments into single-precision host fields (nvar x N floats), half
 * the bytes over the host link; each staged chunk is narrowed on the device.
 * Lossless for F32 storage (its moments are FP32 sums); 16-bit storage: its
 * FP64-decoded moments rounded to float.  F64 storage: VLBM_ERR_UNSUPPORTED.
 * Synchronises.  No counterpart in the paper (host interface only). */
vlbm_status vlbm_moments_f32(vlbm_ctx *ctx, int domain, float *Q_host);

/* As vlbm_moments into a device buffer, enqueued on the stream only. */
vlbm_status vlbm_moments_device(vlbm_ctx *ctx, int domain, double *Q_dev);

/* Pre-collision populations f_ki(x) at the current step (after streaming)
 * for `ncells` cells listed in `cells` (linear indices, 0 <= cell < N),
 * into f_host[c * nvar_q + j] with j running over the context's lattices
 * in field order and directions in the order above (ideal: j = k*q + i;
 * resistive: 19 flow directions then 3 x 7 magnetic ones).  Decoded to
 * double.  Synchronises. */
vlbm_status vlbm_gather_populations(vlbm_ctx *ctx, int domain, const int64_t *cells,
                                    int ncells, double *f_host);

/* Domain sums of the conserved fields, sum_x Q_k(x), accumulated in
 * double precision from the stored populations (fixed reduction order:
 * repeated calls on the same state return identical values), into
 * sums[min(nvar, 8)] on the host (the Powell and dissipative models: the
 * eight MHD fields; D, G and W are not conserved fields).  Also refreshes the health status.
 * Synchronises. */
vlbm_status vlbm_conservation(vlbm_ctx *ctx, int domain, double *sums);

/* Domain sums of the eight ideal-MHD fields, like vlbm_conservation, for a
 * caller that owns the population buffer and may not allocate device memory
 * at all -- for example code embedded in a host application whose memory
 * manager owns every device allocation, or a latency-bound loop that must not
 * pay for (or synchronise on) cudaMalloc.  The paper has no counterpart: this
 * is a library-service entry point.
 *
 * Inputs: pop_dev, a device buffer in the library's population layout
 * (slot j = k * q + i of cell x at pop_dev + (j * stride + x) elements of the
 * storage type, q = 5 in 2-D and 7 in 3-D, x = x + nx * (y + ny * z),
 * periodic; a context's own buffer has stride = nx * ny * nz rounded up to a
 * multiple of 64 elements, so that every slot plane starts on a 128-byte
 * boundary), holding the state after a number of steps whose parity is
 * `parity` (the AA in-place pattern: at parity 0 slot (i, x) is f_i(x), at
 * parity 1 slot (opp i, x - c_i) is); storage as in vlbm_storage, with the
 * per-lattice q_ref and q_scale (8 host doubles each) required for the
 * deviation forms and ignored otherwise.  Output: sums_dev, 8 device doubles.
 * Work is enqueued on `stream` (a cudaStream_t, NULL for the default stream);
 * the call returns without synchronising.
 *
 * It allocates nothing: the per-CTA partial sums go to a fixed 256 KiB array
 * in the library's device image (present on every GPU that loads the library
 * until the process exits).  That bounds the domain to at most 2^28 =
 * 268,435,456 cells; larger domains are rejected with VLBM_ERR_ARG before any
 * device work.  The first call on each device looks up the array's device
 * address with that device current, so make that first call before capturing
 * any stream; the address is kept for the process, so after a cudaDeviceReset
 * of that device it is stale and the call must not be used again.  All calls share the one array; nothing in it has to start at
 * zero (every partial is written before it is read), but two calls whose work
 * overlaps on the GPU race on it -- serialise them (one stream, or events).
 * Errors: VLBM_ERR_ARG for NULL buffers, bad sizes or parity, missing
 * q_ref/q_scale; VLBM_ERR_CUDA if the look-up or a launch fails; the reason is
 * in vlbm_last_error(NULL). */
vlbm_status vlbm_conservation_noalloc(const void *pop_dev, int storage, int dim, int nx, int ny, int nz,
                                      int64_t stride, int parity, const double *q_ref, const double *q_scale,
                                      double *sums_dev, void *stream);

/* Checkpoint: raw populations, step count and parameters of every domain.
 * With buf == NULL, *bytes receives the size needed.  vlbm_load restores a
 * context created with identical parameters bit-exactly. */
vlbm_status vlbm_save(vlbm_ctx *ctx, void *buf, size_t *bytes);
vlbm_status vlbm_load(vlbm_ctx *ctx, const void *buf, size_t bytes);

/* Batched contexts: time each built tile configuration for `steps` steps on
 * the current state (state is restored afterwards) and keep the fastest;
 * *choice receives its index.  Single-domain contexts return VLBM_OK with
 * *choice = 0. */
vlbm_status vlbm_autotune(vlbm_ctx *ctx, int steps, int *choice);

/* ------------------------------------------------------------------------
 * Learned flux closure for coarse 3-D ideal-MHD runs (no counterpart in the
 * paper; the paper's fluxes are exact and local, this corrects the coarse
 * grid's discretisation error as learned from restricted fine runs).
 *
 * Network, per cell (3 x 3 x 3 periodic convolutions, BF16 weights and
 * activations, FP32 accumulation on the tensor cores):
 *   x = (Q - mu) / sigma (8 channels) -> tanh(conv 8 -> H) -> tanh(conv H -> H)
 *   -> conv H -> 24 = y;  dPhi[k][a] = out_scale[k] * y[3k + a],  H = 32.
 * The correction is added to the post-collision populations of the D3Q7
 * lattices: f*_{k,+a} += dPhi/2, f*_{k,-a} -= dPhi/2 (w_moving / cs^2 = 1/2),
 * leaving every zeroth moment unchanged: it adds dPhi to the flux carried by
 * the populations, so every domain sum is conserved exactly.
 * Flat parameter order: W1[H][8][27], b1[H], W2[H][H][27], b2[H], W3[24][H][27],
 * b3[24]; tap t = 9 (dz+1) + 3 (dy+1) + (dx+1), conv(x)[o] = b[o] +
 * sum_{c,t} W[o][c][t] x[c](p + e_t).
 * ------------------------------------------------------------------------ */
typedef struct vlbm_closure vlbm_closure;

typedef struct {
    int nx, ny, nz;           /* coarse grid the closure trains on (3-D, periodic) */
    double gamma;             /* EOS of the coarse solver used in training steps */
    double tau;               /* BGK relaxation time of the coarse solver */
    double mu[8], sigma[8];   /* feature normalisation per conserved field */
    double out_scale[8];      /* dPhi_k = out_scale_k * network output */
    double lr, beta1, beta2, eps;  /* Adam */
    void *stream;             /* cudaStream_t or NULL */
} vlbm_closure_params;

/* Allocate the network (FP32 master weights, Adam state, packed BF16
 * fragments, activation buffers for nx*ny*nz cells) and an internal coarse
 * context used by vlbm_closure_train_step.  Weights start at zero.
 * nx must be a multiple of 16 and nx*ny*nz at most 2^25 (VLBM_ERR_ARG). */
vlbm_status vlbm_closure_create(const vlbm_closure_params *p, vlbm_closure **out);
size_t vlbm_closure_num_params(const vlbm_closure *cl);
/* Copy count = vlbm_closure_num_params floats in the flat order above. */
vlbm_status vlbm_closure_set_weights(vlbm_closure *cl, const float *host, size_t count);
vlbm_status vlbm_closure_get_weights(vlbm_closure *cl, float *host, size_t count);

/* Network forward on device fields Q_dev (8 x N doubles, N = nx*ny*nz):
 * dphi_dev receives N x 24 floats (cell-major, dPhi[k][a] at 3k + a). */
vlbm_status vlbm_closure_forward(vlbm_closure *cl, const double *Q_dev, float *dphi_dev);

/* Gradient of sum(gy * y) over all cells with respect to every parameter, for
 * the network evaluated on Q_dev; gy_dev is N x 24 floats (dL/dy, before
 * out_scale).  grads_host receives vlbm_closure_num_params floats. */
vlbm_status vlbm_closure_backward(vlbm_closure *cl, const double *Q_dev, const float *gy_dev,
                                  float *grads_host);

/* One Adam step on the one-coarse-step loss
 *   L = sum_{k,x} ((Q1_k - Qt_k) / sigma_k)^2 / N,
 * Q1 = moments after one corrected lattice Boltzmann step from f_eq(Q0_dev).
 * Q0_dev, Qt_dev: 8 x N device doubles.  *loss receives L before the update. */
vlbm_status vlbm_closure_train_step(vlbm_closure *cl, const double *Q0_dev, const double *Qt_dev,
                                    double *loss);

/* One Adam step on the same loss along a coarse run: the network is applied
 * to the current state of `ctx` (a 3-D F32 ideal context on the closure's
 * grid, with its non-equilibrium populations), `ctx` advances one corrected
 * step, and Q1 is its new moments; Qt_dev is the target at that time.
 * Enqueued on the context's stream; synchronises it. */
vlbm_status vlbm_closure_train_step_ctx(vlbm_closure *cl, vlbm_ctx *ctx, const double *Qt_dev, double *loss);

/* The two halves of vlbm_closure_train_step_ctx, for data-parallel training
 * (one process per GPU, each on its own coarse runs, gradients averaged across
 * the processes between the halves; no counterpart in the paper, which trains
 * no network).  grad_step: the network on the context's state, one corrected
 * step of `ctx`, the loss against Qt_dev (*loss, host) and its gradient with
 * respect to every parameter into grads_dev (device, vlbm_closure_num_params
 * floats, flat order above); the weights are not changed.  Synchronises the
 * context's stream.  apply_grads: one Adam step with the gradient grads_dev
 * (device, complete before the call), then the weights are re-packed for the
 * tensor-core kernels; synchronises the closure's stream.  grad_step followed
 * by apply_grads of the same gradient equals vlbm_closure_train_step_ctx bit
 * for bit in the weights and the context's state (the gradient is summed in a
 * fixed order; the reported loss is summed with FP64 atomics, so its last
 * digits may differ between runs).  VLBM_ERR_ARG for NULL arguments or a context that is not a 3-D F32
 * ideal context on the closure's grid. */
vlbm_status vlbm_closure_grad_step_ctx(vlbm_closure *cl, vlbm_ctx *ctx, const double *Qt_dev, double *loss,
                                       float *grads_dev);
vlbm_status vlbm_closure_apply_grads(vlbm_closure *cl, const float *grads_dev);

/* Homogenised solid objects (sec. 2.4, "Homogenization", HLBM).  Attach
 * (solid_dev) or detach (NULL) per-cell solid fields to a single-domain
 * ideal-MHD context (VLBM_IDEAL, F32 or F64 storage, 2-D or 3-D, no closure):
 * solid_dev points to 7 x N floats on the device, structure of arrays,
 * solid_dev[v*N + cell] with v = 0 the porosity d in [0, 1] (1 fluid, 0 solid),
 * v = 1..3 the solid's velocity uB, v = 4..6 its field BB (lattice units),
 * N = nx*ny*nz, cell = x + nx*(y + ny*z).  Every following vlbm_step blends
 * u_hat = d u + (1 - d) uB and B_hat = d B + (1 - d) BB in the fused step and
 * relaxes towards the equilibrium of (rho, rho u_hat, e_hat, B_hat), with
 * e_hat = p/(gamma-1) + rho|u_hat|^2/2 + |B_hat|^2/2 from the cell's own gas
 * pressure p.  The caller owns the array: it must stay valid while attached.
 * A moving object may rewrite it between steps: the rewrite must wait until
 * the steps already enqueued have completed (they read the array when they
 * run; vlbm_sync, or an event on the context's stream), and it must be
 * complete before the next vlbm_step (the stream-ordering convention above).
 * VLBM_ERR_UNSUPPORTED for other models, storages, batches or with a closure
 * attached. */
vlbm_status vlbm_set_solid(vlbm_ctx *ctx, const float *solid_dev);

/* Porosity of the signed distance to a solid surface (sec. 2.4, positive in
 * the fluid): d = 0 for phi <= -eps_h/2, phi/eps_h + 1/2 inside the
 * transition, 1 for phi >= eps_h/2; n values, device pointers, enqueued on
 * `stream` (cudaStream_t or NULL).  eps_h > 0; VLBM_ERR_ARG otherwise. */
vlbm_status vlbm_porosity_from_distance(const float *phi_dev, int64_t n, double eps_h, float *d_dev,
                                        void *stream);

/* Static equilibrium boundaries (sec. 2.4, "Static boundaries").  Faces:
 * 0 x-, 1 x+, 2 y-, 3 y+, 4 z-, 5 z+ (2-D: 0..3).  Every face starts periodic.
 * kind VLBM_BC_EQUILIBRIUM opens the face: after each step, every cell on it
 * receives, in the one direction that enters the domain across the face, the
 * equilibrium f_eq_i (Eq. 3) of the boundary state Q_b, where Q_b,k is
 * values[k] if bit k of dirichlet_mask is set (Dirichlet) and otherwise the
 * moment Q_k of the cell one step along the discrete inward normal (Neumann,
 * "zero gradient"; at an edge or a corner the normal is the sum of the open
 * faces' normals, so the copied cell is never a boundary cell).  Populations
 * leaving across an open face are dropped.  values: 8 host doubles
 * (rho, rho u, e_tot, B), read during the call; NULL when the mask is 0.
 * Both faces of an axis must be open or both periodic when vlbm_step runs
 * (VLBM_ERR_ARG there otherwise); an open axis needs at least 3 cells.
 * Single ideal-MHD contexts with F32 or F64 storage, with or without
 * homogenised solids; VLBM_ERR_UNSUPPORTED for other models, storages,
 * batches or with a closure attached.  kind VLBM_BC_PERIODIC closes the face
 * again.  Each step with an open face launches one more (small) kernel. */
typedef enum { VLBM_BC_PERIODIC = 0, VLBM_BC_EQUILIBRIUM = 1 } vlbm_bc_kind;
vlbm_status vlbm_set_boundary(vlbm_ctx *ctx, int face, int kind, unsigned dirichlet_mask, const double *values);

/* Attach (cl) or detach (NULL) a closure to a 3-D ideal-MHD context with F32
 * storage and the closure's grid: every following vlbm_step evaluates the
 * network on the current state and applies the correction in the fused
 * step kernel. */
vlbm_status vlbm_set_closure(vlbm_ctx *ctx, vlbm_closure *cl);
void vlbm_closure_destroy(vlbm_closure *cl);

/* Conservative restriction: Qc[v][X] = mean of the factor^3 fine cells of
 * coarse cell X (fine grid nx x ny x nz, each divisible by factor), 8 fields
 * of device doubles, enqueued on `stream`. */
vlbm_status vlbm_restrict(const double *Qf_dev, int nx, int ny, int nz, int factor, double *Qc_dev,
                          void *stream);

/* ------------------------------------------------------------------------
 * Slab decomposition of one periodic domain (sec. 5: the paper ran its
 * 100-million-cell case on two GPUs; how it split the domain is not given,
 * this is the library's own decomposition).  A global domain, periodic along
 * its last axis a (z in 3-D, y in 2-D), is cut into P slabs of whole layers;
 * slab r (r = 0 .. P-1 in the order of the axis) is an ordinary context of
 * the slab's size with the global parameters (deviation storage: the same
 * q_ref and q_scale on every slab), initialised with its part of the global
 * fields and marked with vlbm_set_slab.  Its kernels wrap axis a inside the
 * slab; the streaming of Eq. 2 across a slab face is completed by moving, after
 * every step, the population slot planes that wrapped -- one "lo" message (the
 * slab's first layer, every slot whose direction has c_a = +1) and one "hi"
 * message (its last layer, every slot whose direction has c_a = -1).  Slots per
 * face: one per lattice for D2Q5/D3Q7 models (8 ideal, 9 Powell, 20
 * dissipative), 5 + 3 for the resistive model (the D3Q19 directions with
 * c_z = +-1 and the magnetic lattices' +-z slots; with walls, the rows next to
 * the walls keep their halfway bounce-back entries -- slots 15 and 17 at y = 1,
 * 16 and 18 at y = ny-2 -- out of the exchange, since they belong to their own
 * cell, and those message entries are left unwritten).  Every element moves
 * unchanged, so P slabs equal the single domain bit for bit.
 *
 * Routing after a step that leaves the slab's step count ODD (an even step
 * ran): slab r sends hi to slab r+1 and lo to slab r-1 (mod P), and unpacks the
 * hi it receives from r-1 and the lo from r+1.  After a step that leaves the
 * count EVEN: hi goes to r-1 and lo to r+1; r unpacks hi from r+1 and lo from
 * r-1.  Messages are [slot][cell of the face layer] in the storage type,
 * vlbm_halo_bytes each.  Conservation sums of the decomposed domain are the
 * sum of the slabs' vlbm_conservation (one all-reduce of 8 doubles across
 * processes).
 * ------------------------------------------------------------------------ */

/* Mark (on = 1) or unmark (on = 0) a context as one slab of a decomposed
 * domain; mark it at an even step count (after vlbm_init_fields).  A slab
 * steps one step at a time (vlbm_step with n <= 1; n > 1 is VLBM_ERR_STATE)
 * and after each step its halo exchange must be unpacked before anything
 * reads its state or steps it again: vlbm_moments*, vlbm_conservation,
 * vlbm_gather_populations, vlbm_save and vlbm_step return VLBM_ERR_STATE
 * until vlbm_halo_unpack (or vlbm_slabs_step, or a new init) completes it.
 * VLBM_ERR_UNSUPPORTED for batched contexts, with a closure attached, or with
 * an open face on the decomposed axis (faces on the other axes may be open). */
vlbm_status vlbm_set_slab(vlbm_ctx *ctx, int on);

/* Bytes of one face message (lo or hi) of this context: slots per face x cells
 * of one layer (nx * ny in 3-D, nx in 2-D) x bytes per stored population;
 * 0 for NULL or batched contexts. */
size_t vlbm_halo_bytes(const vlbm_ctx *ctx);

/* Copy the slab's face slot planes into the device buffers lo_dev and hi_dev
 * (vlbm_halo_bytes each, caller-owned), enqueued on the context's stream.  The
 * messages are complete when the stream reaches this work (send them from
 * that stream, or after an event on it).  VLBM_ERR_STATE if not a slab. */
vlbm_status vlbm_halo_pack(vlbm_ctx *ctx, void *lo_dev, void *hi_dev);

/* Write the received face messages (device buffers, vlbm_halo_bytes each,
 * complete before the context's stream reaches this work) into the slab's face
 * slot planes and mark the exchange done.  A slab with open faces (on the axes
 * the decomposition keeps whole) runs their equilibrium fill here rather than
 * after its step: the fill's Neumann moments of the first and last layers read
 * slots the exchange brings.  VLBM_ERR_STATE if not a slab. */
vlbm_status vlbm_halo_unpack(vlbm_ctx *ctx, const void *lo_dev, const void *hi_dev);

/* Advance P slabs of one decomposed domain that live in this process on one
 * device and share one stream (slabs[r] is slab r): n steps, each one step of
 * every slab followed by the exchange above (pack into a per-slab message
 * buffer the first call allocates through the context's hooks, then unpack
 * from the neighbours' buffers), 3 launches per slab per step; P = 1 is the
 * periodic domain itself and exchanges nothing.  All slabs must be slab
 * contexts of the same model, storage and face layer, at the same step
 * count, with no exchange pending (VLBM_ERR_ARG / VLBM_ERR_STATE otherwise).
 * Asynchronous; returns slab 0's sticky health status. */
vlbm_status vlbm_slabs_step(vlbm_ctx *const *slabs, int nslabs, int n);

/* Batched contexts: number of built tile shapes, and explicit selection of
 * one (0 <= shape < vlbm_tile_shapes; VLBM_ERR_ARG otherwise).  Single-domain
 * contexts have 0 shapes. */
int vlbm_tile_shapes(const vlbm_ctx *ctx);
vlbm_status vlbm_set_tile_shape(vlbm_ctx *ctx, int shape);

/* Failure-detection self-check (no counterpart in the paper).  The persistent
 * kernels wait on mbarriers with a bounded number of tries (each may suspend
 * the waiting thread for up to 20 us; 2^16 tries, about 1.3 s, in the step
 * kernels); when the tries run out a kernel raises the context's timeout flag,
 * lets its copies in flight land and returns instead of hanging.  This call
 * enqueues on the context's stream a one-thread kernel whose wait, by the same
 * bounded primitive, can never succeed (a barrier expecting two arrivals gets
 * one) and gives up after `tries` (1 .. 65536, VLBM_ERR_ARG otherwise): the next
 * vlbm_sync returns VLBM_ERR_TIMEOUT and the context stays failed until
 * vlbm_init_fields or vlbm_load succeeds, as after a real give-up.  Nothing
 * faults, traps or hangs; the kernel ends within about tries x 20 us. */
vlbm_status vlbm_check_bounded_wait(vlbm_ctx *ctx, int tries);

/* FP64 fused multiply-add rate of the current device's CUDA cores, in TFLOP/s
 * (2 flops per FMA), for placing the FP64 forms on their arithmetic roofline
 * (no counterpart in the paper: the FP64 pipe of a GB300 runs far below its
 * FP32 rate, and the FP64 step is bound by it).  One kernel of independent FMA
 * chains, `iters` FMAs per chain (1 .. 2^20; 4096 takes a few ms), timed with
 * CUDA events on `stream` (cudaStream_t or NULL); best of three timed launches
 * after one warm-up.  Synchronises that stream.  VLBM_ERR_ARG for bad
 * arguments, VLBM_ERR_CUDA if a launch fails. */
vlbm_status vlbm_measure_fp64_rate(int iters, void *stream, double *tflops);

/* Small queries. */
int vlbm_nvar(const vlbm_ctx *ctx);                  /* 8 ideal, 7 resistive, 9 Powell, 20 / 26 dissipative (2-D / 3-D) */
int vlbm_slots_per_cell(const vlbm_ctx *ctx);        /* populations per cell: 40 or 56 (ideal), 40 (D3Q19 +
                                                        3 x D3Q7), 45 or 63 (Powell), 100 or 182 (dissipative) */
int vlbm_num_domains(const vlbm_ctx *ctx);
int64_t vlbm_num_cells(const vlbm_ctx *ctx, int domain);
int64_t vlbm_step_count(const vlbm_ctx *ctx);
int64_t vlbm_launch_count(const vlbm_ctx *ctx);      /* kernels this ctx launched */
size_t vlbm_population_bytes(const vlbm_ctx *ctx);   /* device bytes of populations */
void *vlbm_stream(const vlbm_ctx *ctx);              /* the cudaStream_t in use */
const char *vlbm_last_error(const vlbm_ctx *ctx);
const char *vlbm_status_string(int status);

/* Release every device resource of the context (NULL is a no-op). */
void vlbm_destroy(vlbm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* VLBM_H */
