// k_diss.cu -- dissipative MHD with locally evolved gradients on D2Q5 (sm_103a).
//
// The full MHD system (sec. 2.3, "Evolution of the MHD equation system", with
// the local moments evolution of sec. 2.2.1) carries, besides the eight fields
// of Eq. 12, the gradient tensors that the dissipative fluxes need:
//   G_ab ~ tau_M d_a B_b   flux G_ab u_c - delta_ac B_b,   source -G_ab / tau_M
//   W_ab ~ tau_M d_a u_b   flux W_ab u_c - delta_ac u_b,   source -W_ab / tau_M
// with a in {x, y} (the lattice axes) and b in {x, y, z}.  Field order:
// Q[8 + 3a + b] = G_ab, Q[14 + 3a + b] = W_ab -- 20 lattices of D2Q5,
// 100 populations per cell.  With d_a B_b = G_ab / tau_M, d_a u_b = W_ab / tau_M
// and d_z = 0, the fluxes of the MHD fields are those of Eq. 12 plus
//   momentum   - tau_v,               tau_v = rho nu (grad u + grad u^T)
//   energy     - u . tau_v + eta j x B            (heat flux zero)
//   induction  - eta grad B
// with j = curl B and the current-dependent resistivity
// eta = eta0 (1 + |j|^2 / j_c^2) (sec. 2.3, "Incompressible resistive MHD";
// j_c <= 0 keeps eta = eta0).  Optional Powell source
// S = -(div B)(0, B, u.B, u) with div B = (G_xx + G_yy) / tau_M.
//
// 3-D (D3Q7): a in {x, y, z}, Q[8 + 3a + b] = G_ab, Q[17 + 3a + b] = W_ab --
// 26 lattices, 182 populations per cell, div B = (G_xx + G_yy + G_zz) / tau_M.
//
// One fused kernel per step as for ideal MHD (Eq. 2, AA in-place pattern,
// one cell per thread, x-contiguous slot planes): load the 100 populations,
// form the 20 moments, the fluxes and sources above, relax towards the
// first-order equilibrium of Eq. 3 with direct source injection, store.
// 2-D FP32 keeps the populations in registers between load and store; 2-D FP64
// (400 registers' worth) sums them on the way in and reads them again for the
// update -- the second read of a slot comes from the cache, and it is safe in
// place because a thread writes only slots it reads, each after reading it.
// The 3-D kernel (182 populations) relaxes the gradient lattices as it reads
// them and holds only the MHD lattices, forming each lattice's flux where it
// relaxes that lattice (see k_diss3_step).
#include "diss_cell.cuh"

namespace vlbm {
namespace {

// Linear indices of x + c_i (periodic), D2Q5 order.
__device__ __forceinline__ void diss_neighbours(int x, int y, int nx, int ny, int64_t cell, int64_t (&nb)[kDissQ])
{
    const int64_t plane = (int64_t)nx * ny;
    nb[0] = cell;
    nb[1] = (x + 1 < nx) ? cell + 1 : cell + 1 - nx;
    nb[2] = (x > 0) ? cell - 1 : cell - 1 + nx;
    nb[3] = (y + 1 < ny) ? cell + nx : cell + nx - plane;
    nb[4] = (y > 0) ? cell - nx : cell - nx + plane;
}

// The fused collide-and-stream step (Eq. 2): even parity reads slot (i, x) and
// sends direction i to slot (opp i, x); odd parity reads slot (opp i, x - c_i)
// and sends direction i to slot (i, x + c_i).  HOLD keeps the populations in
// registers between load and update, otherwise they are read twice.
template <class C, bool ODD, bool HOLD>
__global__ void __launch_bounds__(kBlockX) k_diss_step(const DissArgs<C> a)
{
    constexpr int Q = kDissQ;
    const int x = blockIdx.x * kBlockX + threadIdx.x;
    if (x >= a.nx) return;
    const int y = blockIdx.y;
    const int64_t cell = x + (int64_t)a.nx * y;
    int64_t nb[Q];
    diss_neighbours(x, y, a.nx, a.ny, cell, nb);
    C *pop = static_cast<C *>(a.pop);
    auto src = [&](int k, int i) -> C * {
        return pop + (int64_t)(k * Q + (ODD ? opp_axis(i) : i)) * a.stride + (ODD ? nb[opp_axis(i)] : cell);
    };
    auto dst = [&](int k, int i) -> C * {
        return pop + (int64_t)(k * Q + (ODD ? i : opp_axis(i))) * a.stride + (ODD ? nb[i] : cell);
    };

    C q[kDissLat];
    C f[HOLD ? kDissLat : 1][Q];
#pragma unroll
    for (int k = 0; k < kDissLat; ++k) {
        C s = C(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const C v = *src(k, i);
            if constexpr (HOLD) f[k][i] = v;
            s += v;
        }
        q[k] = s;
    }
    C phi[kDissLat][2], S[kDissLat];
    diss_flux_source<C>(q, a, phi, S, a.flags);

    // weights and relaxation products that sum to one (omega) exactly (vlbm_internal.cuh)
    constexpr C w0 = ExactWeights<2, C>::w0, w1 = ExactWeights<2, C>::w1;
#pragma unroll
    for (int k = 0; k < kDissLat; ++k) {
        C g[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) g[i] = HOLD ? f[HOLD ? k : 0][i] : *src(k, i);
        const C om = a.omega[k];
        const C omc = C(1) - om;
        C ow0, ow1;
        relax_weights<2, C>(om, ow0, ow1);
        const C A0 = ow0 * q[k] + w0 * S[k];
        const C A1 = ow1 * q[k] + w1 * S[k];
        const C hom = C(0.5) * om;  // omega * w_moving / cs^2
        const C bx = hom * phi[k][0], by = hom * phi[k][1];
        *dst(k, 0) = omc * g[0] + A0;
        *dst(k, 1) = omc * g[1] + A1 + bx;
        *dst(k, 2) = omc * g[2] + A1 - bx;
        *dst(k, 3) = omc * g[3] + A1 + by;
        *dst(k, 4) = omc * g[4] + A1 - by;
    }
}

// f = f_eq(Q) at parity 0 (Eq. 3 with the fluxes above) for cells c0 .. c0 + count;
// also checks positivity and the sub-characteristic condition
// max(|u| + c_f) < cs of the ideal part.
template <class C>
__global__ void k_diss_init(const DissArgs<C> a, double gamma, int64_t c0, int64_t count, int64_t qstride,
                            const double *__restrict__ Qin)
{
    constexpr int Q = kDissQ;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= count) return;
    const int64_t cell = c0 + t;
    C q[kDissLat];
#pragma unroll
    for (int k = 0; k < kDissLat; ++k) q[k] = (C)Qin[k * qstride + t];
    C phi[kDissLat][2], S[kDissLat];
    diss_flux_source<C>(q, a, phi, S, a.flags);
    {
        const C rho = q[0], ir = C(1) / rho;
        const C u2 = (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) * ir * ir;
        const C B2 = q[5] * q[5] + q[6] * q[6] + q[7] * q[7];
        const C p = a.gm1 * (q[4] - C(0.5) * rho * u2 - C(0.5) * B2);
        const C vsig = sqrt(u2) + sqrt(fmax((C(gamma) * p + B2) * ir, C(0)));
        if (!(vsig < (C)sqrt(AxisSet<2>::cs2))) atomicOr(a.flags, kFlagUnstable);
    }
    C *pop = static_cast<C *>(a.pop);
    constexpr C w0 = ExactWeights<2, C>::w0, w1 = ExactWeights<2, C>::w1;  // as in the step
    constexpr C h = C(AxisSet<2>::w1 / AxisSet<2>::cs2);
#pragma unroll
    for (int k = 0; k < kDissLat; ++k) {
        C *base = pop + (int64_t)(k * Q) * a.stride + cell;
        base[0] = w0 * q[k];
        base[a.stride] = w1 * q[k] + h * phi[k][0];
        base[2 * a.stride] = w1 * q[k] - h * phi[k][0];
        base[3 * a.stride] = w1 * q[k] + h * phi[k][1];
        base[4 * a.stride] = w1 * q[k] - h * phi[k][1];
    }
}

// Linear indices of x + c_i (periodic), D3Q7 order.
__device__ __forceinline__ void diss3_neighbours(int x, int y, int z, int nx, int ny, int nz, int64_t cell,
                                                 int64_t (&nb)[kDiss3Q])
{
    const int64_t plane = (int64_t)nx * ny, vol = plane * nz;
    nb[0] = cell;
    nb[1] = (x + 1 < nx) ? cell + 1 : cell + 1 - nx;
    nb[2] = (x > 0) ? cell - 1 : cell - 1 + nx;
    nb[3] = (y + 1 < ny) ? cell + nx : cell + nx - plane;
    nb[4] = (y > 0) ? cell - nx : cell - nx + plane;
    nb[5] = (z + 1 < nz) ? cell + plane : cell + plane - vol;
    nb[6] = (z > 0) ? cell - plane : cell - plane + vol;
}

// The 3-D fused step.  The fluxes of the 18 gradient lattices need only their
// own moment, u and B, so the step reads every population once:
//   A. the 8 MHD lattices into registers (56 values) and their moments -> u, B;
//   B. each gradient lattice: read its 7 populations, sum, flux G u_c - I B (or
//      W u_c - I u), source -G / tau_M, relax and store -- one read per slot;
//   C. with all 26 moments the derived state (viscous stress, grad B, eta(j),
//      Powell's div B), then the 8 MHD lattices relaxed from registers and stored.
// The step is bound by the bytes each SM keeps in flight: B's rounds of loads
// each wait for DRAM.  So FP32 (HOLD) stages them: every thread copies its own
// populations of the gradient lattices into its own column of shared memory
// with cp.async, kNs - 1 pairs of lattices ahead of the pair it relaxes (no
// registers held and no barrier: a thread reads back only what it copied).
// Measured at 256^3: 3.91 GLUPS against 3.63 with two lattices' loads issued
// together into registers (and 3.68 with every slot row of the CTA requested
// into L2 at its start; 3.37 with the MHD lattices staged too, at four CTAs per
// SM).  FP64 (HOLD false) keeps nothing in registers and reads the MHD lattices
// again in C (the FP64 pipe binds that form, not the memory traffic).
template <class C, bool ODD, bool HOLD>
__device__ __forceinline__ void diss3_step_body(const DissArgs<C> &a)
{
    constexpr int Q = kDiss3Q;
    const int x = blockIdx.x * kBlockX + threadIdx.x;
    if (x >= a.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const int64_t cell = x + (int64_t)a.nx * (y + (int64_t)a.ny * z);
    int64_t nb[Q];
    diss3_neighbours(x, y, z, a.nx, a.ny, a.nz, cell, nb);
    C *pop = static_cast<C *>(a.pop);
    auto src = [&](int k, int i) -> C * {
        return pop + (int64_t)(k * Q + (ODD ? opp_axis(i) : i)) * a.stride + (ODD ? nb[opp_axis(i)] : cell);
    };
    auto dst = [&](int k, int i) -> C * {
        return pop + (int64_t)(k * Q + (ODD ? i : opp_axis(i))) * a.stride + (ODD ? nb[i] : cell);
    };
    constexpr C w0 = ExactWeights<3, C>::w0, w1 = ExactWeights<3, C>::w1;
    // BGK with direct source injection for lattice k, populations g, moment qk
    auto relax = [&](int k, const C (&g)[Q], C qk, const C (&phi)[3], C S) {
        const C om = a.omega[k];
        const C omc = C(1) - om;
        C ow0, ow1;
        relax_weights<3, C>(om, ow0, ow1);
        const C A0 = ow0 * qk + w0 * S;
        const C A1 = ow1 * qk + w1 * S;
        const C hom = C(0.5) * om;  // omega * w_moving / cs^2
        const C bx = hom * phi[0], by = hom * phi[1], bz = hom * phi[2];
        *dst(k, 0) = omc * g[0] + A0;
        *dst(k, 1) = omc * g[1] + A1 + bx;
        *dst(k, 2) = omc * g[2] + A1 - bx;
        *dst(k, 3) = omc * g[3] + A1 + by;
        *dst(k, 4) = omc * g[4] + A1 - by;
        *dst(k, 5) = omc * g[5] + A1 + bz;
        *dst(k, 6) = omc * g[6] + A1 - bz;
    };

    // B's staging: pairs of gradient lattices, kNs stages of 14 populations per thread
    constexpr int GB = 2;
    constexpr int kNp = (kDiss3Lat - 8) / GB;
    constexpr int kNs = 4;
    __shared__ C stg[HOLD ? kNs : 1][HOLD ? GB * Q : 1][kBlockX];
    auto issue = [&](int p) {  // copies of pair p (none past the last), always one commit group
        if (p < kNp) {
            // lattice 8 + GB p, direction i: slot (8 + GB p) Q + i' at cell n_i', with i' = i
            // (even) or opp(i) (odd); one 64-bit base per lattice
            const C *lat = pop + (int64_t)(8 + GB * p) * Q * a.stride;
#pragma unroll
            for (int kk = 0; kk < GB; ++kk)
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const int j = ODD ? opp_axis(i) : i;
                    const C *g = lat + ((int64_t)(kk * Q + j) * a.stride + (ODD ? nb[j] : cell));
                    const uint32_t d =
                        (uint32_t)__cvta_generic_to_shared(&stg[p % kNs][kk * Q + i][threadIdx.x]);
                    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(g),
                                 "n"((int)sizeof(C))
                                 : "memory");
                }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    if constexpr (HOLD) {
#pragma unroll
        for (int p = 0; p < kNs - 1; ++p) issue(p);
    }

    // A: the MHD lattices
    C q[kDiss3Lat];
    C f8[HOLD ? 8 : 1][Q];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        C s = C(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const C v = *src(k, i);
            if constexpr (HOLD) f8[k][i] = v;
            s += v;
        }
        q[k] = s;
    }
    const C ir = C(1) / q[0];
    const C u[3] = {q[1] * ir, q[2] * ir, q[3] * ir};
    const C B[3] = {q[5], q[6], q[7]};

    // B: the gradient lattices G (8..16) and W (17..25), a pair at a time
#pragma unroll
    for (int p = 0; p < kNp; ++p) {
        const int k0 = 8 + GB * p;
        C g[GB][Q];
        if constexpr (HOLD) {
            issue(p + kNs - 1);
            // every group but the newest kNs - 1 complete: pairs 0..p have landed
            asm volatile("cp.async.wait_group %0;\n" ::"n"(kNs - 1) : "memory");
#pragma unroll
            for (int kk = 0; kk < GB; ++kk)
#pragma unroll
                for (int i = 0; i < Q; ++i) g[kk][i] = stg[p % kNs][kk * Q + i][threadIdx.x];
        } else {
#pragma unroll
            for (int kk = 0; kk < GB; ++kk)
#pragma unroll
                for (int i = 0; i < Q; ++i) g[kk][i] = *src(k0 + kk, i);
        }
#pragma unroll
        for (int kk = 0; kk < GB; ++kk) {
            const int k = k0 + kk;
            C s = C(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) s += g[kk][i];
            q[k] = s;
            const bool isG = k < 17;
            const int r = isG ? (k - 8) / 3 : (k - 17) / 3, b = isG ? (k - 8) % 3 : (k - 17) % 3;
            C phi[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) phi[c] = s * u[c] - (r == c ? (isG ? B[b] : u[b]) : C(0));
            relax(k, g[kk], s, phi, -s * a.inv_tau_m);
        }
    }

    // C: the derived state, then the MHD lattices
    const Diss3State<C> st = diss3_state<C>(q, a, a.flags);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        C phi[3];
        diss3_flux<C>(k, q, st, phi);
        const C S = diss3_source<C>(k, q, st, a.inv_tau_m);
        C g[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) g[i] = HOLD ? f8[HOLD ? k : 0][i] : *src(k, i);
        relax(k, g, q[k], phi, S);
    }
}

// Three CTAs of the FP32 form fit an SM at 168 registers and 28 KB of staging each
// (the FP64 form keeps the compiler's own register choice)
template <class C, bool ODD, bool HOLD>
__global__ void __launch_bounds__(kBlockX, HOLD ? 3 : 0) k_diss3_step(const DissArgs<C> a)
{
    diss3_step_body<C, ODD, HOLD>(a);
}

// 3-D f = f_eq(Q) at parity 0, and the positivity and sub-characteristic checks.
template <class C>
__global__ void k_diss3_init(const DissArgs<C> a, double gamma, int64_t c0, int64_t count, int64_t qstride,
                             const double *__restrict__ Qin)
{
    constexpr int Q = kDiss3Q;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= count) return;
    const int64_t cell = c0 + t;
    C q[kDiss3Lat];
#pragma unroll
    for (int k = 0; k < kDiss3Lat; ++k) q[k] = (C)Qin[k * qstride + t];
    const Diss3State<C> st = diss3_state<C>(q, a, a.flags);
    {
        const C rho = q[0], ir = C(1) / rho;
        const C u2 = (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) * ir * ir;
        const C B2 = q[5] * q[5] + q[6] * q[6] + q[7] * q[7];
        const C p = a.gm1 * (q[4] - C(0.5) * rho * u2 - C(0.5) * B2);
        const C vsig = sqrt(u2) + sqrt(fmax((C(gamma) * p + B2) * ir, C(0)));
        if (!(vsig < (C)sqrt(AxisSet<3>::cs2))) atomicOr(a.flags, kFlagUnstable);
    }
    C *pop = static_cast<C *>(a.pop);
    constexpr C w0 = ExactWeights<3, C>::w0, w1 = ExactWeights<3, C>::w1;
    constexpr C h = C(AxisSet<3>::w1 / AxisSet<3>::cs2);
#pragma unroll
    for (int k = 0; k < kDiss3Lat; ++k) {
        C phi[3];
        diss3_flux<C>(k, q, st, phi);
        C *base = pop + (int64_t)(k * Q) * a.stride + cell;
        base[0] = w0 * q[k];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            base[(2 * c + 1) * a.stride] = w1 * q[k] + h * phi[c];
            base[(2 * c + 2) * a.stride] = w1 * q[k] - h * phi[c];
        }
    }
}

struct DissRead {
    const void *pop;
    int nx, ny, nz;
    int64_t stride;
    int parity;
};

// Logical (pre-collision) population f_ki of a cell at the current parity.
template <class C>
__device__ __forceinline__ C diss_logical(const DissRead &a, int64_t cell, const int64_t (&nb)[kDissQ], int k, int i)
{
    const C *pop = static_cast<const C *>(a.pop);
    const int j = a.parity ? opp_axis(i) : i;
    const int64_t at = a.parity ? nb[opp_axis(i)] : cell;
    return pop[(int64_t)(k * kDissQ + j) * a.stride + at];
}

// 3-D: logical population f_ki and the moments and gather over D3Q7.
template <class C>
__device__ __forceinline__ C diss3_logical(const DissRead &a, int64_t cell, const int64_t (&nb)[kDiss3Q], int k,
                                           int i)
{
    const C *pop = static_cast<const C *>(a.pop);
    const int j = a.parity ? opp_axis(i) : i;
    const int64_t at = a.parity ? nb[opp_axis(i)] : cell;
    return pop[(int64_t)(k * kDiss3Q + j) * a.stride + at];
}

__device__ __forceinline__ void diss3_cell_nb(const DissRead &a, int64_t cell, int64_t (&nb)[kDiss3Q])
{
    const int x = (int)(cell % a.nx);
    const int64_t r = cell / a.nx;
    diss3_neighbours(x, (int)(r % a.ny), (int)(r / a.ny), a.nx, a.ny, a.nz, cell, nb);
}

template <class C>
__global__ void k_diss3_moments(const DissRead a, int64_t c0, int64_t count, int64_t ostride,
                                double *__restrict__ out)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= count) return;
    const int64_t cell = c0 + t;
    int64_t nb[kDiss3Q];
    diss3_cell_nb(a, cell, nb);
#pragma unroll
    for (int k = 0; k < kDiss3Lat; ++k) {
        C s = C(0);
#pragma unroll
        for (int i = 0; i < kDiss3Q; ++i) s += diss3_logical<C>(a, cell, nb, k, i);
        out[k * ostride + t] = (double)s;
    }
}

template <class C>
__global__ void k_diss3_gather(const DissRead a, const int64_t *__restrict__ cells, int n, double *__restrict__ out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int64_t cell = cells[t];
    int64_t nb[kDiss3Q];
    diss3_cell_nb(a, cell, nb);
#pragma unroll
    for (int k = 0; k < kDiss3Lat; ++k)
#pragma unroll
        for (int i = 0; i < kDiss3Q; ++i)
            out[(int64_t)t * kDiss3Lat * kDiss3Q + k * kDiss3Q + i] = (double)diss3_logical<C>(a, cell, nb, k, i);
}

// Q_k = sum_i f_ki (Eq. 4) for cells c0 .. c0 + count, summed in the storage precision.
template <class C>
__global__ void k_diss_moments(const DissRead a, int64_t c0, int64_t count, int64_t ostride, double *__restrict__ out)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= count) return;
    const int64_t cell = c0 + t;
    const int x = (int)(cell % a.nx), y = (int)(cell / a.nx);
    int64_t nb[kDissQ];
    diss_neighbours(x, y, a.nx, a.ny, cell, nb);
#pragma unroll
    for (int k = 0; k < kDissLat; ++k) {
        C s = C(0);
#pragma unroll
        for (int i = 0; i < kDissQ; ++i) s += diss_logical<C>(a, cell, nb, k, i);
        out[k * ostride + t] = (double)s;
    }
}

template <class C>
__global__ void k_diss_gather(const DissRead a, const int64_t *__restrict__ cells, int n, double *__restrict__ out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int64_t cell = cells[t];
    const int x = (int)(cell % a.nx), y = (int)(cell / a.nx);
    int64_t nb[kDissQ];
    diss_neighbours(x, y, a.nx, a.ny, cell, nb);
#pragma unroll
    for (int k = 0; k < kDissLat; ++k)
#pragma unroll
        for (int i = 0; i < kDissQ; ++i)
            out[(int64_t)t * kDissLat * kDissQ + k * kDissQ + i] = (double)diss_logical<C>(a, cell, nb, k, i);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

template <class C> DissArgs<C> make_diss_args(vlbm_ctx *c)
{
    const Domain &d = c->dom[0];
    const vlbm_params &p = c->params;
    DissArgs<C> a{};
    a.pop = c->pop;
    a.nx = d.nx;
    a.ny = d.ny;
    a.nz = d.nz;
    a.stride = d.stride;
    a.gm1 = C(d.gamma - 1.0);
    for (int k = 0; k < kDiss3Lat; ++k) a.omega[k] = C(1.0 / (k < 8 ? d.tau[k] : p.tau_g));
    a.nu = C(p.nu);
    a.eta0 = C(p.eta0);
    a.inv_jc2 = C(p.j_c > 0.0 ? 1.0 / (p.j_c * p.j_c) : 0.0);
    a.inv_tau_m = C(1.0 / d.tau_m);
    a.powell = p.powell ? 1 : 0;
    a.flags = c->d_flags;
    return a;
}

DissRead make_diss_read(vlbm_ctx *c)
{
    const Domain &d = c->dom[0];
    return DissRead{c->pop, d.nx, d.ny, d.nz, d.stride, (int)(c->step & 1)};
}

template <class C> vlbm_status step_t(vlbm_ctx *c, int parity)
{
    constexpr bool hold = sizeof(C) == 4;
    const Domain &d = c->dom[0];
    const DissArgs<C> a = make_diss_args<C>(c);
    const dim3 grid((unsigned)((d.nx + kBlockX - 1) / kBlockX), (unsigned)d.ny, (unsigned)d.nz);
    if (c->dim == 3) {
        if (parity)
            k_diss3_step<C, true, hold><<<grid, kBlockX, 0, c->stream>>>(a);
        else
            k_diss3_step<C, false, hold><<<grid, kBlockX, 0, c->stream>>>(a);
    } else if (parity) {
        k_diss_step<C, true, hold><<<grid, kBlockX, 0, c->stream>>>(a);
    } else {
        k_diss_step<C, false, hold><<<grid, kBlockX, 0, c->stream>>>(a);
    }
    c->launches++;
    return cuda_check(c, cudaGetLastError(), "dissipative step launch");
}

template <class C> vlbm_status init_t(vlbm_ctx *c, const double *Q, int64_t c0, int64_t n, int64_t qs)
{
    const int threads = 128;
    const unsigned blocks = (unsigned)((n + threads - 1) / threads);
    if (c->dim == 3)
        k_diss3_init<C><<<blocks, threads, 0, c->stream>>>(make_diss_args<C>(c), c->dom[0].gamma, c0, n, qs, Q);
    else
        k_diss_init<C><<<blocks, threads, 0, c->stream>>>(make_diss_args<C>(c), c->dom[0].gamma, c0, n, qs, Q);
    c->launches++;
    return cuda_check(c, cudaGetLastError(), "dissipative init launch");
}

template <class C> vlbm_status moments_t(vlbm_ctx *c, double *out, int64_t c0, int64_t n, int64_t os)
{
    const int threads = 256;
    const unsigned blocks = (unsigned)((n + threads - 1) / threads);
    if (c->dim == 3)
        k_diss3_moments<C><<<blocks, threads, 0, c->stream>>>(make_diss_read(c), c0, n, os, out);
    else
        k_diss_moments<C><<<blocks, threads, 0, c->stream>>>(make_diss_read(c), c0, n, os, out);
    c->launches++;
    return cuda_check(c, cudaGetLastError(), "dissipative moments launch");
}

template <class C> vlbm_status gather_t(vlbm_ctx *c, const int64_t *cells, int n, double *out)
{
    const int threads = 128;
    const unsigned blocks = (unsigned)((n + threads - 1) / threads);
    if (c->dim == 3)
        k_diss3_gather<C><<<blocks, threads, 0, c->stream>>>(make_diss_read(c), cells, n, out);
    else
        k_diss_gather<C><<<blocks, threads, 0, c->stream>>>(make_diss_read(c), cells, n, out);
    c->launches++;
    return cuda_check(c, cudaGetLastError(), "dissipative gather launch");
}

bool is_f64(const vlbm_ctx *c) { return c->storage == VLBM_F64; }

}  // namespace

vlbm_status diss_step(vlbm_ctx *c, int parity)
{
    return is_f64(c) ? step_t<double>(c, parity) : step_t<float>(c, parity);
}

vlbm_status diss_init_range(vlbm_ctx *c, const double *Q, int64_t c0, int64_t n, int64_t qstride)
{
    return is_f64(c) ? init_t<double>(c, Q, c0, n, qstride) : init_t<float>(c, Q, c0, n, qstride);
}

vlbm_status diss_moments_range(vlbm_ctx *c, double *out, int64_t c0, int64_t n, int64_t ostride)
{
    return is_f64(c) ? moments_t<double>(c, out, c0, n, ostride) : moments_t<float>(c, out, c0, n, ostride);
}

vlbm_status diss_gather(vlbm_ctx *c, const int64_t *cells_dev, int n, double *out_dev)
{
    return is_f64(c) ? gather_t<double>(c, cells_dev, n, out_dev) : gather_t<float>(c, cells_dev, n, out_dev);
}

}  // namespace vlbm
