// vlbm_internal.cuh -- internal types of the GB300 VLBM library (not ABI).
//
// Population storage: one in-place buffer per context, structure of arrays.
// Slot (j, cell) of a domain lives at  base + j * stride + cell, where j runs
// over lattice-major (lattice k, direction i) pairs and stride is the cell
// count rounded up to a multiple of 64 elements, so that every slot plane
// starts on a 128-byte boundary for every storage type.
//
// AA in-place streaming (two kernels that alternate):
//   parity 0 ("even") step at cell x:  read slot (i, x), write the
//       post-collision value of direction i to slot (opp(i), x);
//   parity 1 ("odd") step at cell x:   read slot (opp(i), x - c_i), write
//       the post-collision value of direction i to slot (i, x + c_i).
// The set of slots a cell reads equals the set it writes, so one buffer
// suffices and no two threads touch the same slot.  The logical
// (pre-collision) population of the state is slot (i, x) at parity 0 and
// slot (opp(i), x - c_i) at parity 1.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>
#include <type_traits>
#include <vector>

#include "vlbm.h"

#include <nvtx3/nvToolsExt.h>

namespace vlbm {

constexpr int kMaxLat = 9;  // per-lattice tables of Domain: ideal 8, Powell 9 (resistive 4; the
                            // dissipative model's 12 gradient lattices share params.tau_g)
constexpr int kBlockX = 128;     // threads per CTA along x for the step kernels
constexpr int kReduceBlocks = 1216;  // 8 CTAs per SM on 152 SMs
constexpr int kReduceThreads = 256;

// Status bits written by kernels into the context's device flag word.
constexpr unsigned kFlagNonPhysical = 1u;  // NaN, rho <= 0 or p <= 0
constexpr unsigned kFlagUnstable = 2u;     // max(|u| + c_f) >= cs at init
constexpr unsigned kFlagTimeout = 4u;      // a bounded device wait gave up

// Direction i of the axis-aligned sets: 0 rest, 2a+1 = +e_a, 2a+2 = -e_a.
__host__ __device__ constexpr int opp_axis(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

// The per-cell arithmetic (ideal_cell.cuh) is host-and-device: the step
// kernels run it on the GPU, and the same source also compiles for the host,
// where a test checks it cell by cell without a GPU.  The two device-only
// operations it needs go through these helpers.
#define VLBM_HD __host__ __device__

// Raise status bits in the flag word (atomically on the device).
VLBM_HD __forceinline__ void raise_flag(unsigned *flags, unsigned bits)
{
#ifdef __CUDA_ARCH__
    atomicOr(flags, bits);
#else
    *flags |= bits;
#endif
}

// Load through the read-only data cache on the device.
template <class T> VLBM_HD __forceinline__ T ro_load(const T *p)
{
#ifdef __CUDA_ARCH__
    return __ldg(p);
#else
    return *p;
#endif
}

// Weights of the axis sets: D2Q5 (1/3, 1/6; cs^2 = 1/3), D3Q7 (1/4, 1/8;
// cs^2 = 1/4).  In both, w_moving / cs^2 = 1/2.
template <int D> struct AxisSet;
template <> struct AxisSet<2> {
    static constexpr int Q = 5;
    static constexpr double w0 = 1.0 / 3.0, w1 = 1.0 / 6.0, cs2 = 1.0 / 3.0;
};
template <> struct AxisSet<3> {
    static constexpr int Q = 7;
    static constexpr double w0 = 1.0 / 4.0, w1 = 1.0 / 8.0, cs2 = 1.0 / 4.0;
};

// Weights in the compute precision C that sum to one exactly.  D3Q7's 1/4 and
// 1/8 are exact in binary; for D2Q5, w0 = 1 - 4 w1 (exact: Sterbenz), and the
// relaxation products omega w0 = omega - 4 (omega w1) (also exact).  With
// rounded products instead, every cell would gain or lose the same fraction of
// Q_k per step -- a drift of about one or two ulps per step in the FP32 domain
// sums of the 2-D forms.
template <int D, class C> struct ExactWeights {
    static constexpr C w1 = C(AxisSet<D>::w1);
    static constexpr C w0 = D == 2 ? C(1) - C(4) * w1 : C(AxisSet<D>::w0);
};
template <int D, class C> VLBM_HD __forceinline__ void relax_weights(C om, C &ow0, C &ow1)
{
    ow1 = om * ExactWeights<D, C>::w1;
    ow0 = D == 2 ? om - C(4) * ow1 : om * ExactWeights<D, C>::w0;
}

// An opaque copy of a value: the compiler cannot reuse expressions computed
// from the original across it, so addresses built from the copy are
// recomputed where they are used instead of being held in registers.
__device__ __forceinline__ int64_t opaque(int64_t v)
{
    asm volatile("" : "+l"(v));
    return v;
}

// Storage codecs: deviation forms store (f - w_i ref_k) / scale_k.
template <class S> struct Codec;
template <> struct Codec<double> {
    static constexpr bool kDev = false;
    __device__ static __forceinline__ double load(const double *p) { return *p; }
    __device__ static __forceinline__ void store(double *p, double v) { *p = v; }
};
template <> struct Codec<float> {
    static constexpr bool kDev = false;
    __device__ static __forceinline__ float load(const float *p) { return *p; }
    __device__ static __forceinline__ void store(float *p, float v) { *p = v; }
};
template <> struct Codec<__half> {
    static constexpr bool kDev = true;
    __device__ static __forceinline__ float load(const __half *p) { return __half2float(*p); }
    __device__ static __forceinline__ void store(__half *p, float v) { *p = __float2half_rn(v); }
};
template <> struct Codec<__nv_bfloat16> {
    static constexpr bool kDev = true;
    __device__ static __forceinline__ float load(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    __device__ static __forceinline__ void store(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};

// Compute precision of a storage type: FP64 storage computes in FP64, the
// others in FP32 (as the step kernel does).  GB300 runs FP64 arithmetic far
// slower than FP32, so per-population FP64 work is kept out of the passes
// that read every population.
template <class S> struct ComputeOf {
    using T = float;
};
template <> struct ComputeOf<double> {
    using T = double;
};

// Per-domain description (host and device copies).
struct Domain {
    int nx, ny, nz;
    int64_t ncell;
    int64_t stride;        // elements between slot planes
    int64_t offset;        // element offset of the domain's block in the buffer
    double gamma;
    double tau[kMaxLat];
    double source[kMaxLat];
    double q_ref[kMaxLat];
    double q_scale[kMaxLat];
    double force[3];
    double b_wall[3];
    int walls_y;
    double tau_m;          // Powell model: relaxation time of D (steps)
};

// Slab decomposition: the slot planes of a slab's two faces that wrap in the
// odd step (k_slab.cu).  lo: first layer, directions with c_a = +1; hi: last
// layer, directions with c_a = -1 (a = z in 3-D, y in 2-D).
// A slot may keep one row of the face layer out of the exchange (-1: none):
// with walls, the rows next to a wall hold the halfway bounce-back of their own
// cell in some c_a != 0 slots, which never stream across a face.
constexpr int kMaxHaloSlots = 32;
struct HaloSlots {
    int n;                  // slots per face
    int lo[kMaxHaloSlots];
    int hi[kMaxHaloSlots];
    int lo_keep[kMaxHaloSlots];  // row y of the face layer that stays (3-D), or -1
    int hi_keep[kMaxHaloSlots];
};

}  // namespace vlbm

struct vlbm_ctx {
    vlbm_params params;                 // parameters of domain 0 (copied)
    int model = 0, dim = 3, q = 7, nlat = 8, nvar = 8;
    int storage = VLBM_F32;
    size_t elem = 4;                    // bytes per stored population
    int nslot = 56;                     // slots per cell (lattices x directions)
    std::vector<vlbm::Domain> dom;
    bool batched = false;

    void *pop = nullptr;                // population buffer
    size_t pop_bytes = 0;
    unsigned *d_flags = nullptr;        // device status word
    unsigned *h_flags = nullptr;        // pinned host mirror
    double *d_partials = nullptr;       // reduction scratch [kReduceBlocks x 8]
    double *d_sums = nullptr;           // reduction result [8]
    double *d_refscale = nullptr;       // q_ref[8] then q_scale[8] of domain 0 (deviation storage, FP64)
    double h_refscale[16] = {};         // host copy (the upload's source; kept alive with the context)
    double *d_q = nullptr;              // staging for host fields (lazily sized)
    size_t d_q_bytes = 0;
    double *h_stage = nullptr;          // pinned host staging
    size_t h_stage_bytes = 0;

    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t copy_stream = nullptr;  // host-field staging copies (overlap the chunk kernels)
    int bulk_ctas = 0;                   // persistent grid of the bulk-load step (0: not sized yet)
    cudaEvent_t ev_copy[2]{}, ev_kern[2]{};  // per staging buffer: last copy / last kernel done
    cudaEvent_t flag_event = nullptr;
    bool flag_pending = false;
    int64_t steps_since_check = 0;

    int64_t step = 0;                   // completed (enqueued) steps
    int64_t launches = 0;               // kernels launched by this context
    vlbm_status sticky = VLBM_OK;
    std::string err;

    std::map<int, cudaGraphExec_t> graphs;  // key: parity*1024 + length
    std::map<int, int64_t> graph_launches;  // kernels one replay of that graph launches

    // batched form
    std::vector<void *> tile_tables;    // per tile shape: device (domain, first cell) pairs
    std::vector<int> tile_counts;       // tiles per table
    std::vector<int> tile_grid;         // CTAs launched per table
    int tune_choice = 0;
    void *d_dom = nullptr;              // device copy of the domain table

    // learned flux closure applied in every step (not owned)
    struct vlbm_closure *closure = nullptr;
    const float *solid = nullptr;       // homogenised solids: [7][N] caller-owned fields, or null
    // static equilibrium boundaries, faces x-, x+, y-, y+, z-, z+
    int face_kind[6] = {0, 0, 0, 0, 0, 0};  // VLBM_BC_PERIODIC or VLBM_BC_EQUILIBRIUM
    unsigned face_mask[6] = {0, 0, 0, 0, 0, 0};  // bit k: Q_k Dirichlet (else Neumann)
    double face_vals[6][8] = {};             // Dirichlet values

    // slab of a decomposed domain (k_slab.cu): the face planes move between
    // slabs after every step; halo_pending: a step ran and its exchange has
    // not been unpacked yet
    bool slab = false;
    bool halo_pending = false;
    vlbm::HaloSlots halo{};
    void *halo_buf = nullptr;           // vlbm_slabs_step: this slab's packed lo then hi message

    // allocator
    std::vector<std::pair<void *, size_t>> owned;
};

namespace vlbm {

// A named range on the host timeline of profilers that read NVTX (header-only NVTX3: without
// an attached tool each push and pop is a test of one pointer).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// host helpers (vlbm_api.cu)
vlbm_status fail(vlbm_ctx *c, vlbm_status s, const std::string &msg);
vlbm_status cuda_check(vlbm_ctx *c, cudaError_t e, const char *what);

// launchers (k_ideal.cu)
vlbm_status ideal_init(vlbm_ctx *c, int d, const double *Q_dev);
vlbm_status ideal_init_range(vlbm_ctx *c, int d, const double *Q, int64_t c0, int64_t n, int64_t qstride);
vlbm_status ideal_moments_range(vlbm_ctx *c, int d, double *out, int64_t c0, int64_t n, int64_t ostride);
vlbm_status ideal_step(vlbm_ctx *c, int parity);
vlbm_status ideal_moments(vlbm_ctx *c, int d, double *Q_dev);
vlbm_status ideal_gather(vlbm_ctx *c, int d, const int64_t *cells_dev, int n, double *out_dev);
vlbm_status ideal_sums(vlbm_ctx *c, int d, double *sums_dev);

// launchers (k_resistive.cu)
vlbm_status resistive_init(vlbm_ctx *c, int d, const double *Q_dev);
vlbm_status resistive_init_range(vlbm_ctx *c, int d, const double *Q, int64_t c0, int64_t n, int64_t qstride);
vlbm_status resistive_moments_range(vlbm_ctx *c, int d, double *out, int64_t c0, int64_t n, int64_t ostride);
vlbm_status resistive_step(vlbm_ctx *c, int parity);
vlbm_status resistive_moments(vlbm_ctx *c, int d, double *Q_dev);
vlbm_status resistive_gather(vlbm_ctx *c, int d, const int64_t *cells_dev, int n, double *out_dev);
vlbm_status resistive_sums(vlbm_ctx *c, int d, double *sums_dev);

// launchers (k_diss.cu): dissipative model, 2-D, F32 / F64 storage
vlbm_status diss_step(vlbm_ctx *c, int parity);
vlbm_status diss_init_range(vlbm_ctx *c, const double *Q, int64_t c0, int64_t n, int64_t qstride);
vlbm_status diss_moments_range(vlbm_ctx *c, double *out, int64_t c0, int64_t n, int64_t ostride);
vlbm_status diss_gather(vlbm_ctx *c, const int64_t *cells_dev, int n, double *out_dev);

// launchers (k_batch.cu)
vlbm_status batch_prepare(vlbm_ctx *c);
vlbm_status batch_step(vlbm_ctx *c, int parity, int choice);
int batch_num_choices();

// learned closure (k_closure.cu / k_ideal.cu)
vlbm_status ideal_step_corrected(vlbm_ctx *c, int parity, const float *dphi);
// porosity of the signed distance (HLBM), elementwise
vlbm_status porosity_from_distance(const float *phi, int64_t n, double eps_h, float *d, cudaStream_t s);
bool any_open_face(const vlbm_ctx *c);
// failure-detection self-check: a bounded wait that must give up (k_ideal.cu)
vlbm_status wait_check(vlbm_ctx *c, uint32_t tries);
vlbm_status open_fill(vlbm_ctx *c, int parity);
// closure input features of a 3-D FP32 context straight from its populations:
// x[cell][k] = BF16((Q_k - mu_k) * inv_sigma_k), Q_k summed in FP32 as by ideal_moments
vlbm_status ideal_features(vlbm_ctx *c, const float *mu, const float *inv_sigma, __nv_bfloat16 *x);
vlbm_status closure_step(vlbm_ctx *c, int parity);
int closure_cells(const vlbm_closure *cl, int *nx, int *ny, int *nz);

// precision of staged host fields (k_convert.cu): nvar fields of n values each,
// field v at v * stride, enqueued on the context's stream
vlbm_status widen_fields(vlbm_ctx *c, const float *in, int nvar, int64_t n, int64_t stride, double *out);
vlbm_status narrow_fields(vlbm_ctx *c, const double *in, int nvar, int64_t n, int64_t stride, float *out);

// slab halo (k_slab.cu): the face slot list of the context's model, and one
// launch that packs (face planes -> lo, hi messages) or unpacks (the reverse)
HaloSlots halo_slots(const vlbm_ctx *c);
vlbm_status halo_copy(vlbm_ctx *c, void *lo, void *hi, bool pack);

// reduction of per-block partials into sums (k_ideal.cu)
vlbm_status finish_sums(vlbm_ctx *c, int nvar, double *sums_dev);

}  // namespace vlbm
