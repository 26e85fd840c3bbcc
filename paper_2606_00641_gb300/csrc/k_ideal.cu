// k_ideal.cu -- ideal compressible MHD on D2Q5 / D3Q7 lattices (sm_103a).
//
// One fused kernel per time step performs Eq. 2 of the paper for every cell:
// it loads the cell's 8 x q populations (AA in-place pattern, see
// vlbm_internal.cuh), forms the moments Q_k (Eq. 4), the primitive state and
// gas pressure from the EOS (Eq. 9), the ideal MHD fluxes (Eq. 12), relaxes
// every population towards the first-order equilibrium of Eq. 3 (BGK), adds
// the direct-injection source w_i S_k, and stores the results so that the
// next step finds them streamed.
//
// The step is HBM-bound (8 q populations read and written once per cell;
// a few hundred flops per cell against 448 B at FP32/D3Q7), so the design
// goal is plain bandwidth: one cell per thread, coalesced x-contiguous slot
// planes, every load issued before any arithmetic, no shared memory, grid
// (ceil(nx/128), ny, nz).
#include <algorithm>

#include "ideal_cell.cuh"

namespace vlbm {
namespace {

template <class C> struct IdealArgs {
    void *pop;
    int nx, ny, nz;
    int64_t stride;
    C gm1;
    C omega[kMaxLat];
    C src0[kMaxLat];      // w_0 S_k       (deviation storage: / s_k)
    C src1[kMaxLat];      // w_moving S_k  (deviation storage: / s_k)
    C ref[kMaxLat];       // deviation storage: r_k
    C scale[kMaxLat];     //                    s_k
    C inv_scale[kMaxLat]; //                    1 / s_k
    unsigned *flags;
    const float *dphi;    // closure: per-cell flux correction [cell][24], or null
    C inv_tau_m;          // Powell model: 1 / tau_M (div B = D / tau_M)
    const float *solid;   // homogenised solids: [7][solid_n] d, uB, BB per cell, or null
    int64_t solid_n;
    const double *refscale;  // deviation storage: r_0..7, s_0..7 in FP64 (device; pressure recovery)
    C p_theta;               // deviation storage: FP64 pressure below p_theta * e_tot
};

// Linear indices of the cell's neighbours x + c_i (periodic), i in set order.
template <int D>
__device__ __forceinline__ void neighbours(int x, int y, int z, int nx, int ny, int nz, int64_t cell,
                                           int64_t *nb)
{
    const int64_t row = nx;
    const int64_t plane = (int64_t)nx * ny;
    nb[0] = cell;
    nb[1] = (x + 1 < nx) ? cell + 1 : cell + 1 - nx;
    nb[2] = (x > 0) ? cell - 1 : cell - 1 + nx;
    nb[3] = (y + 1 < ny) ? cell + row : cell + row - plane;
    nb[4] = (y > 0) ? cell - row : cell - row + plane;
    if (D == 3) {
        const int64_t vol = plane * nz;
        nb[5] = (z + 1 < nz) ? cell + plane : cell + plane - vol;
        nb[6] = (z > 0) ? cell - plane : cell - plane + vol;
    }
}


// The fused collide-and-stream step.  ODD selects the AA parity; CORR adds
// the learned flux correction dPhi[k][a] to the post-collision populations
// (f*_{k,+a} += dPhi/2, f*_{k,-a} -= dPhi/2: zero mass, first moment dPhi).
// NL = 9 is the Powell model (eight MHD lattices and the divergence lattice);
// HOM blends with homogenised solids (a.solid).
template <int D, class S, class C, bool ODD, bool CORR = false, int NL = 8, bool HOM = false>
__device__ __forceinline__ void ideal_step_body(const IdealArgs<C> &a)
{
    constexpr int Q = AxisSet<D>::Q;
    const int x = blockIdx.x * kBlockX + threadIdx.x;
    if (x >= a.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const int64_t cell = x + (int64_t)a.nx * (y + (int64_t)a.ny * z);
    int64_t nb[Q];
    neighbours<D>(x, y, z, a.nx, a.ny, a.nz, cell, nb);
    S *pop = static_cast<S *>(a.pop);

    // load: even parity reads slot (i, x); odd parity reads slot (opp i, x - c_i)
    C f[NL][Q];
#pragma unroll
    for (int k = 0; k < NL; ++k)
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int j = ODD ? opp_axis(i) : i;
            const int64_t at = ODD ? nb[opp_axis(i)] : cell;
            f[k][i] = Codec<S>::load(pop + (int64_t)(k * Q + j) * a.stride + at);
        }

    if constexpr (NL == 9) {
        powell_collide<D, C>(f, a.gm1, a.omega, a.src0, a.src1, a.inv_tau_m, a.flags);
    } else if constexpr (HOM) {
        const float *sp = a.solid + cell;
        const C d = C(__ldg(sp));
        const C uB[3] = {C(__ldg(sp + a.solid_n)), C(__ldg(sp + 2 * a.solid_n)), C(__ldg(sp + 3 * a.solid_n))};
        const C BB[3] = {C(__ldg(sp + 4 * a.solid_n)), C(__ldg(sp + 5 * a.solid_n)), C(__ldg(sp + 6 * a.solid_n))};
        ideal_collide_hom<D, C>(f, a.gm1, a.omega, a.src0, a.src1, a.flags, d, uB, BB);
    } else {
        // deviation storage collides on the stored deviations directly (ideal_cell.cuh)
        ideal_collide<D, C, Codec<S>::kDev>(f, a.gm1, a.omega, a.src0, a.src1, a.flags, a.ref, a.scale,
                                            a.inv_scale, a.refscale, a.p_theta);
    }
    if constexpr (CORR) {
        const float *dp = a.dphi + cell * 24;
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
            for (int ax = 0; ax < D; ++ax) {
                const C v = C(0.5f * dp[3 * k + ax]);
                f[k][2 * ax + 1] += v;
                f[k][2 * ax + 2] -= v;
            }
    }

    // store: even parity sends direction i to slot (opp i, x);
    //        odd parity sends direction i to slot (i, x + c_i)
#pragma unroll
    for (int k = 0; k < NL; ++k)
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int j = ODD ? i : opp_axis(i);
            const int64_t at = ODD ? nb[i] : cell;
            Codec<S>::store(pop + (int64_t)(k * Q + j) * a.stride + at, f[k][i]);
        }
}

template <int D, class S, class C, bool ODD, bool CORR = false, int NL = 8, bool HOM = false>
__global__ void __launch_bounds__(kBlockX) k_ideal_step(const IdealArgs<C> a)
{
    ideal_step_body<D, S, C, ODD, CORR, NL, HOM>(a);
}

// Deviation storage: the same step bounded to the occupancy of the plain 16-bit
// step (six CTAs per SM in 2-D, five in 3-D), so that the rare FP64
// pressure-recovery call does not lower it.
template <int D, class S, bool ODD>
__global__ void __launch_bounds__(kBlockX, D == 2 ? 6 : 5) k_ideal_step_dev(const IdealArgs<float> a)
{
    ideal_step_body<D, S, float, ODD>(a);
}

// The same step for 16-bit storage in 3-D with the loads done by the
// bulk-copy engine.  A tile is an x-row segment of 128 cells; the 56 slot
// plane rows its cells read (even parity: their own row; odd parity: the row
// of the upstream cell, one plane row over for the y and z directions and one
// element over for x) arrive in shared memory by one cp.async.bulk each, plus
// the single element beyond the tile edge that the x-moving slots of the odd
// parity need.  Persistent CTAs with two buffers: the rows of the next tile
// are in flight while the threads collide the current one from shared memory,
// so the bytes in flight per SM no longer depend on how many warps the
// registers allow -- the limit of the one-cell-per-thread kernel on 16-bit
// storage, whose 2-byte loads carry half the bytes of FP32 ones.  Each thread
// takes two x-adjacent cells (k_ideal_step_pairs below): the instruction issue
// of ~970 instructions per cell bound the one-cell-per-thread form of this
// kernel at 0.78 of the HBM roofline.  Measured slower at 512^3 and not
// adopted (one cell per thread): reading the staged populations twice instead
// of holding them (80 registers, six CTAs; 23.5 against 24.1 GLUPS), three
// buffers handed over by full/empty mbarriers instead of the CTA barrier per
// tile (18.8 GLUPS), and stores walked direction-major with a running pointer
// (23.53 against 23.67 GLUPS).  Needs nx % 8 == 0 (16-byte aligned rows).
constexpr int kBulkPad = 8;  // elements (16 bytes) before and after each staged row

// Bounded wait on phase `parity` of an mbarrier: up to `tries` tries, each of
// which may suspend the thread for up to 20 us (the default 2^16 tries: about
// 1.3 s); true once the phase has completed, false when the tries ran out.
constexpr uint32_t kWaitTries = 1u << 16;

__device__ __forceinline__ bool bounded_wait(uint32_t mbar, uint32_t parity, uint32_t tries = kWaitTries)
{
    uint32_t done = 0;
    for (uint32_t it = 0; it < tries && !done; ++it)
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(done)
                     : "r"(mbar), "r"(parity), "r"(20000u)
                     : "memory");
    return done != 0;
}

// The same wait, outcome ignored: on the way out of a CTA that gave up, for its
// copies in flight.
__device__ __forceinline__ void bulk_drain(uint32_t mbar, uint32_t parity) { (void)bounded_wait(mbar, parity); }

// Failure-detection self-check: one thread waits, with the bounded wait of the
// persistent step, for a phase that no thread completes (two arrivals expected,
// one made), gives up after `tries` and raises the timeout flag exactly as a
// stuck persistent kernel would.
__global__ void k_wait_check(unsigned *flags, uint32_t tries)
{
    __shared__ __align__(8) uint64_t bar;
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mb), "r"(2));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(mb) : "memory");
    if (!bounded_wait(mb, 0u, tries)) atomicOr(flags, kFlagTimeout);
}

// 16-bit pair access: two adjacent cells' values of one slot row as one 32-bit word.
template <class S> struct Pair;
template <> struct Pair<__half> {
    __device__ static __forceinline__ float2 load(const __half *p)
    {
        return __half22float2(*reinterpret_cast<const __half2 *>(p));
    }
    __device__ static __forceinline__ void store(__half *p, float lo, float hi)
    {
        *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(lo, hi);
    }
};
template <> struct Pair<__nv_bfloat16> {
    __device__ static __forceinline__ float2 load(const __nv_bfloat16 *p)
    {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
    }
    __device__ static __forceinline__ void store(__nv_bfloat16 *p, float lo, float hi)
    {
        *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(lo, hi);
    }
};

// The bulk-copy step with two x-adjacent cells per thread (64 threads per 128-cell
// tile).  A slot row's values of the pair are one 32-bit word in shared memory and
// in global memory (rows start on 16-byte boundaries and the pair on an even
// cell), so loads, conversions and stores come in pairs, and one address serves
// both cells; only the x-moving slots of the odd parity, shifted by one cell,
// stay 16-bit.  Needs nx % 8 == 0.
constexpr int kPairThreads = kBlockX / 2;

template <class S, bool ODD>
__global__ void __launch_bounds__(kPairThreads, 6) k_ideal_step_pairs(const IdealArgs<float> a)
{
    constexpr int Q = 7;
    constexpr int ROW = kBlockX + 2 * kBulkPad;
    __shared__ __align__(128) S sm[2][8 * Q][ROW];
    __shared__ __align__(8) uint64_t bar[2];
    const int tid = threadIdx.x;
    const int tiles_x = (a.nx + kBlockX - 1) / kBlockX;
    const int ntiles = tiles_x * a.ny * a.nz;
    const int64_t plane = (int64_t)a.nx * a.ny;
    S *pop = static_cast<S *>(a.pop);
    const uint32_t bar_s = (uint32_t)__cvta_generic_to_shared(bar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar_s), "r"(8 * Q));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar_s + 8u), "r"(8 * Q));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();

    struct Tile {
        int x0, y, z, tx;
        int64_t row, c0;
    };
    auto tile_of = [&](int t) {
        Tile T;
        T.x0 = (t % tiles_x) * kBlockX;
        const int r = t / tiles_x;
        T.y = r % a.ny;
        T.z = r / a.ny;
        T.tx = min(kBlockX, a.nx - T.x0);
        T.row = (int64_t)a.nx * T.y + plane * T.z;
        T.c0 = T.row + T.x0;
        return T;
    };
    // slot plane j = tid (threads 0 .. 55): arm the buffer's barrier and copy its row segment
    auto load_rows = [&](const Tile &T, int b) {
        if (tid >= 8 * Q) return;
        const int j = tid, jj = j % Q;
        int64_t src = T.c0;
        if (ODD) {
            const int i = opp_axis(jj);  // the direction that reads slot jj
            if (i == 3) src = T.y > 0 ? T.c0 - a.nx : T.c0 + (int64_t)(a.ny - 1) * a.nx;  // from y - 1
            else if (i == 4) src = T.y + 1 < a.ny ? T.c0 + a.nx : T.c0 - (int64_t)(a.ny - 1) * a.nx;
            else if (i == 5) src = T.z > 0 ? T.c0 - plane : T.c0 + (int64_t)(a.nz - 1) * plane;  // from z - 1
            else if (i == 6) src = T.z + 1 < a.nz ? T.c0 + plane : T.c0 - (int64_t)(a.nz - 1) * plane;
        }
        const uint32_t mb = bar_s + 8u * (uint32_t)b;
        const uint32_t bytes = (uint32_t)(T.tx * (int)sizeof(S));
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mb), "r"(bytes) : "memory");
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&sm[b][j][kBulkPad]);
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                     ::"r"(dst), "l"(pop + (int64_t)j * a.stride + src), "r"(bytes), "r"(mb)
                     : "memory");
    };
    // odd parity: +x reads slot 2 at x - 1, -x reads slot 1 at x + 1, one element beyond
    // each tile edge; threads 56 .. 63 stage two of the sixteen each
    const bool edge_thread = ODD && tid >= 8 * Q;
    const int eq0 = 2 * (tid - 8 * Q);
    auto edge_slot = [&](int eq) { return eq < 8 ? (eq & 7) * Q + 2 : (eq & 7) * Q + 1; };
    auto edge_load = [&](const Tile &T, int eq) -> S {
        const int xs = eq < 8 ? (T.x0 > 0 ? T.x0 - 1 : a.nx - 1) : (T.x0 + T.tx < a.nx ? T.x0 + T.tx : 0);
        return pop[(int64_t)edge_slot(eq) * a.stride + T.row + xs];
    };
    auto edge_store = [&](const Tile &T, int b, int eq, S v) {
        sm[b][edge_slot(eq)][eq < 8 ? kBulkPad - 1 : kBulkPad + T.tx] = v;
    };

    int t = blockIdx.x;
    Tile cur = tile_of(t);
    if (t < ntiles) {
        load_rows(cur, 0);
        if (edge_thread) {
            edge_store(cur, 0, eq0, edge_load(cur, eq0));
            edge_store(cur, 0, eq0 + 1, edge_load(cur, eq0 + 1));
        }
    }
    __syncthreads();
    bool ok = true;
    for (int i = 0; t < ntiles && ok; ++i, t += gridDim.x) {
        const int b = i & 1;
        const int tn = t + gridDim.x;
        const Tile nxt = tile_of(tn);
        S ev0{}, ev1{};
        if (tn < ntiles) {  // the next tile's rows travel while this one is collided
            load_rows(nxt, b ^ 1);
            if (edge_thread) {
                ev0 = edge_load(nxt, eq0);
                ev1 = edge_load(nxt, eq0 + 1);
            }
        }
        const bool done = bounded_wait(bar_s + 8u * (uint32_t)b, (uint32_t)((i >> 1) & 1));
        if (!__syncthreads_and((int)done)) {  // one outcome for the whole CTA
            if (tid == 0) atomicOr(a.flags, kFlagTimeout);
            // the CTA gives up: the row copies still in flight land first, within a bound
            if (tid < 8 * Q) {
                bulk_drain(bar_s + 8u * (uint32_t)b, (uint32_t)((i >> 1) & 1));
                if (tn < ntiles) bulk_drain(bar_s + 8u * (uint32_t)(b ^ 1), (uint32_t)(((i + 1) >> 1) & 1));
            }
            ok = false;
            break;
        }
        const int xl = 2 * tid;  // cells xl and xl + 1 of the tile
        if (xl < cur.tx) {
            float fa[8][Q], fb[8][Q];
#pragma unroll
            for (int k = 0; k < 8; ++k)
#pragma unroll
                for (int ii = 0; ii < Q; ++ii) {
                    const int jj = ODD ? opp_axis(ii) : ii;
                    const S *r = &sm[b][k * Q + jj][kBulkPad + xl];
                    if (ODD && (ii == 1 || ii == 2)) {  // shifted by one cell: 16-bit
                        const int sh = ii == 1 ? -1 : 1;
                        fa[k][ii] = Codec<S>::load(r + sh);
                        fb[k][ii] = Codec<S>::load(r + 1 + sh);
                    } else {
                        const float2 v = Pair<S>::load(r);
                        fa[k][ii] = v.x;
                        fb[k][ii] = v.y;
                    }
                }
            ideal_collide<3, float, true>(fa, a.gm1, a.omega, a.src0, a.src1, a.flags, a.ref, a.scale,
                                          a.inv_scale, a.refscale, a.p_theta);
            ideal_collide<3, float, true>(fb, a.gm1, a.omega, a.src0, a.src1, a.flags, a.ref, a.scale,
                                          a.inv_scale, a.refscale, a.p_theta);
            // store: even parity sends direction i to slot (opp i, x); odd parity to slot
            // (i, x + c_i), which keeps the pair together except along x
            const int xa = cur.x0 + xl;
            const int64_t ca = cur.c0 + xl;
            int64_t off[Q];  // x + c_i - x for the y and z directions (periodic), pair-aligned
            off[0] = 0;
            off[3] = cur.y + 1 < a.ny ? a.nx : -(int64_t)(a.ny - 1) * a.nx;
            off[4] = cur.y > 0 ? -(int64_t)a.nx : (int64_t)(a.ny - 1) * a.nx;
            off[5] = cur.z + 1 < a.nz ? plane : -(int64_t)(a.nz - 1) * plane;
            off[6] = cur.z > 0 ? -plane : (int64_t)(a.nz - 1) * plane;
            off[1] = off[2] = 0;
            const int64_t pa_plus = xa + 1 < a.nx ? ca + 1 : ca + 1 - a.nx;       // a + e_x
            const int64_t pb_plus = xa + 2 < a.nx ? ca + 2 : ca + 2 - a.nx;       // b + e_x
            const int64_t pa_minus = xa > 0 ? ca - 1 : ca - 1 + a.nx;             // a - e_x
#pragma unroll
            for (int k = 0; k < 8; ++k)
#pragma unroll
                for (int ii = 0; ii < Q; ++ii) {
                    const int j = ODD ? ii : opp_axis(ii);
                    S *row = pop + (int64_t)(k * Q + j) * a.stride;
                    if (ODD && ii == 1) {
                        Codec<S>::store(row + pa_plus, fa[k][ii]);
                        Codec<S>::store(row + pb_plus, fb[k][ii]);
                    } else if (ODD && ii == 2) {
                        Codec<S>::store(row + pa_minus, fa[k][ii]);
                        Codec<S>::store(row + ca, fb[k][ii]);  // b - e_x = a
                    } else {
                        Pair<S>::store(row + ca + (ODD ? off[ii] : 0), fa[k][ii], fb[k][ii]);
                    }
                }
        }
        if (edge_thread && tn < ntiles) {
            edge_store(nxt, b ^ 1, eq0, ev0);
            edge_store(nxt, b ^ 1, eq0 + 1, ev1);
        }
        __syncthreads();  // buffer b consumed before it is refilled; edge elements visible
        cur = nxt;
    }
}

// f = f_eq(Q) at parity 0 (Eq. 3 with the fluxes of Eq. 12), computed in the
// compute precision of the storage (FP64 only for FP64 storage; FP64 runs far
// slower than FP32 on GB300); also checks positivity and the
// sub-characteristic condition max(|u| + c_f) < cs of the scheme.
template <int D, class S> struct InitArgs {
    void *pop;
    int64_t stride;
    int64_t c0, count, qstride;
    double gamma;
    double ref[kMaxLat], scale[kMaxLat];
    unsigned *flags;
    double p_theta;  // deviation storage: p below p_theta * e_tot is taken in FP64, as in the step
};

template <int D, class S, int NL = 8>
__global__ void k_ideal_init(const InitArgs<D, S> a, const double *__restrict__ Qin)
{
    using R = typename ComputeOf<S>::T;
    constexpr int Q = AxisSet<D>::Q;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= a.count) return;
    const int64_t cell = a.c0 + t;
    R q[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) q[k] = (R)Qin[k * a.qstride + t];
    const R rho = q[0];
    const R inv_rho = R(1) / rho;
    const R u[3] = {q[1] * inv_rho, q[2] * inv_rho, q[3] * inv_rho};
    const R B[3] = {q[5], q[6], q[7]};
    const R B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    const R u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const R uB = u[0] * B[0] + u[1] * B[1] + u[2] * B[2];
    const R gamma = (R)a.gamma;
    R p = (gamma - R(1)) * (q[4] - R(0.5) * rho * u2 - R(0.5) * B2);
    if constexpr (Codec<S>::kDev) {
        if (a.p_theta > 0.0 && p < (R)a.p_theta * q[4]) {  // the step's FP64 recovery, from the FP64 fields
            double v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = Qin[k * a.qstride + t];
            p = (R)((a.gamma - 1.0) * (v[4] - 0.5 * (v[1] * v[1] + v[2] * v[2] + v[3] * v[3]) / v[0] -
                                       0.5 * (v[5] * v[5] + v[6] * v[6] + v[7] * v[7])));
        }
    }
    const R pt = p + R(0.5) * B2;
    if (!(rho > R(0)) || !(p > R(0))) atomicOr(a.flags, kFlagNonPhysical);
    const R vsig = sqrt(u2) + sqrt(fmax((gamma * p + B2) * inv_rho, R(0)));
    if (!(vsig < (R)sqrt(AxisSet<D>::cs2))) atomicOr(a.flags, kFlagUnstable);
    S *pop = static_cast<S *>(a.pop);
    constexpr double inv_cs2 = 1.0 / AxisSet<D>::cs2;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        R phi[D];
#pragma unroll
        for (int ax = 0; ax < D; ++ax) {
            if (k == 0) phi[ax] = q[1 + ax];
            else if (k <= 3) phi[ax] = rho * u[ax] * u[k - 1] - B[ax] * B[k - 1] + (ax == k - 1 ? pt : R(0));
            else if (k == 4) phi[ax] = (q[4] + pt) * u[ax] - B[ax] * uB;
            else phi[ax] = (ax == k - 5) ? R(0) : u[ax] * B[k - 5] - B[ax] * u[k - 5];
        }
        const R ref = (R)a.ref[k], inv_scale = (R)(1.0 / a.scale[k]);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const R w = i == 0 ? ExactWeights<D, R>::w0 : ExactWeights<D, R>::w1;
            R cphi = R(0);
            if (i > 0) cphi = ((i & 1) ? R(1) : R(-1)) * phi[(i - 1) / 2];
            const R feq = w * (q[k] + cphi * (R)inv_cs2);
            R v = feq;
            if (Codec<S>::kDev) v = (feq - w * ref) * inv_scale;
            Codec<S>::store(pop + (int64_t)(k * Q + i) * a.stride + cell, (decltype(Codec<S>::load(pop)))v);
        }
    }
    if constexpr (NL == 9) {  // Powell model: D lattice, flux D u - B (plain storage)
        const R Dv = (R)Qin[8 * a.qstride + t];
        R phi[D];
#pragma unroll
        for (int ax = 0; ax < D; ++ax) phi[ax] = Dv * u[ax] - B[ax];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const R w = i == 0 ? ExactWeights<D, R>::w0 : ExactWeights<D, R>::w1;
            R cphi = R(0);
            if (i > 0) cphi = ((i & 1) ? R(1) : R(-1)) * phi[(i - 1) / 2];
            Codec<S>::store(pop + (int64_t)(8 * Q + i) * a.stride + cell,
                            (decltype(Codec<S>::load(pop)))(w * (Dv + cphi * (R)inv_cs2)));
        }
    }
}

// Logical populations of one cell (parity-aware) decoded to double.
template <int D, class S> struct ReadArgs {
    const void *pop;
    int nx, ny, nz;
    int64_t stride;
    int parity;
    double ref[kMaxLat], scale[kMaxLat];
};


template <int D, class S>
__device__ __forceinline__ double logical(const ReadArgs<D, S> &a, int64_t cell, const int64_t *nb, int k,
                                          int i)
{
    constexpr int Q = AxisSet<D>::Q;
    const S *pop = static_cast<const S *>(a.pop);
    const int j = a.parity ? opp_axis(i) : i;
    const int64_t at = a.parity ? nb[opp_axis(i)] : cell;
    double v = (double)Codec<S>::load(pop + (int64_t)(k * Q + j) * a.stride + at);
    if (Codec<S>::kDev) v = v * a.scale[k] + (i == 0 ? AxisSet<D>::w0 : AxisSet<D>::w1) * a.ref[k];
    return v;
}

// Q_k of one cell: the sum of its populations (Eq. 3) in the compute precision;
// for deviation storage r_k + s_k sum_i g_ki (the weights sum to one), with the
// FP32 sum widened once and decoded in FP64 against the FP64 reference state.
template <int D, class S>
__device__ __forceinline__ double cell_moment(const ReadArgs<D, S> &a, int64_t cell, const int64_t *nb, int k)
{
    using R = typename ComputeOf<S>::T;
    constexpr int Q = AxisSet<D>::Q;
    const S *pop = static_cast<const S *>(a.pop);
    R s = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int j = a.parity ? opp_axis(i) : i;
        const int64_t at = a.parity ? nb[opp_axis(i)] : cell;
        s += (R)Codec<S>::load(pop + (int64_t)(k * Q + j) * a.stride + at);
    }
    if (Codec<S>::kDev) return fma((double)s, a.scale[k], a.ref[k]);
    return (double)s;
}

template <int D>
__device__ __forceinline__ void cell_xyz(int64_t cell, int nx, int ny, int &x, int &y, int &z)
{
    if (cell <= 0xFFFFFFFFll) {  // 32-bit division where the index fits
        const uint32_t c = (uint32_t)cell, r = c / (uint32_t)nx;
        x = (int)(c - r * (uint32_t)nx);
        y = (int)(r % (uint32_t)ny);
        z = (int)(r / (uint32_t)ny);
        return;
    }
    x = (int)(cell % nx);
    const int64_t r = cell / nx;
    y = (int)(r % ny);
    z = (int)(r / ny);
}

template <int D, class S, int NL = 8>
__global__ void k_ideal_moments(const ReadArgs<D, S> a, int64_t c0, int64_t count, int64_t ostride,
                                double *__restrict__ out)
{
    constexpr int Q = AxisSet<D>::Q;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= count) return;
    const int64_t cell = c0 + t;
    int x, y, z;
    cell_xyz<D>(cell, a.nx, a.ny, x, y, z);
    int64_t nb[Q];
    neighbours<D>(x, y, z, a.nx, a.ny, a.nz, cell, nb);
#pragma unroll
    for (int k = 0; k < NL; ++k) out[k * ostride + t] = (double)cell_moment<D, S>(a, cell, nb, k);
}

// Static equilibrium boundaries (sec. 2.4, "Static boundaries").  Faces
// x-, x+, y-, y+, z-, z+; both faces of an open axis are open.
struct OpenFaces {
    int open[3];          // axis open
    unsigned mask[6];     // bit k set: Q_k Dirichlet at vals[face][k]; clear: Neumann
    double vals[6][8];
    int64_t count[6];     // cells on the face (0 for a periodic face)
    double gm1;
};

// After a step, every cell on an open face receives, in the direction entering
// across that face, f_eq_i of the face's boundary state (Eq. 3): Q_k set
// (Dirichlet) or the moment of the cell one step along the discrete inward
// normal (Neumann; diagonal at edges and corners, so that cell is never on an
// open face).  The value goes to the slot this cell reads for that direction in
// the next step: (i, x) at even parity, (opp i, x - c_i) at odd parity, where
// periodic addressing puts x - c_i on the opposite face.  Only this cell reads
// that slot and no thread of the launch reads it, so the pass races neither
// with itself nor with the step.  One thread per (face, cell); blockIdx.y = face.
template <int D, class S>
__global__ void k_open_fill(const ReadArgs<D, S> a, const __grid_constant__ OpenFaces o, unsigned *flags)
{
    using R = typename ComputeOf<S>::T;
    constexpr int Q = AxisSet<D>::Q;
    const int face = blockIdx.y;
    const int ax = face >> 1;
    const bool high = face & 1;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= o.count[face]) return;
    // the cell: fixed on the face's axis, the other two from t (first in-face axis fastest)
    int x, y, z;
    if (ax == 0) {
        x = high ? a.nx - 1 : 0;
        y = (int)(t % a.ny);
        z = (int)(t / a.ny);
    } else if (ax == 1) {
        y = high ? a.ny - 1 : 0;
        x = (int)(t % a.nx);
        z = (int)(t / a.nx);
    } else {
        z = high ? a.nz - 1 : 0;
        x = (int)(t % a.nx);
        y = (int)(t / a.nx);
    }
    // discrete inward normal: every open face the cell lies on
    auto inward = [](int v, int nv, int open) { return !open ? 0 : (v == 0 ? 1 : (v == nv - 1 ? -1 : 0)); };
    const int xn = x + inward(x, a.nx, o.open[0]);
    const int yn = y + inward(y, a.ny, o.open[1]);
    const int zn = D == 3 ? z + inward(z, a.nz, o.open[2]) : z;
    const int64_t cell = x + (int64_t)a.nx * (y + (int64_t)a.ny * z);
    const int64_t ncell = xn + (int64_t)a.nx * (yn + (int64_t)a.ny * zn);
    int64_t nb[Q];
    neighbours<D>(xn, yn, zn, a.nx, a.ny, a.nz, ncell, nb);
    // a Dirichlet variable reads nothing: on an x face every population load of the
    // neighbour is a separate strided line, so skipping them is most of the pass's cost
    const unsigned mask = o.mask[face];
    R q[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) q[k] = ((mask >> k) & 1u) ? (R)o.vals[face][k] : cell_moment<D, S>(a, ncell, nb, k);

    // the flux of Eq. 12 along the face normal
    const R rho = q[0];
    const R ir = R(1) / rho;
    const R u[3] = {q[1] * ir, q[2] * ir, q[3] * ir};
    const R B[3] = {q[5], q[6], q[7]};
    const R B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    const R mu = q[1] * u[0] + q[2] * u[1] + q[3] * u[2];
    const R uB = u[0] * B[0] + u[1] * B[1] + u[2] * B[2];
    const R p = (R)o.gm1 * (q[4] - R(0.5) * mu - R(0.5) * B2);
    if (!(rho > R(0)) || !(p > R(0))) atomicOr(flags, kFlagNonPhysical);
    const R pt = p + R(0.5) * B2;
    // components along the face normal, selected without indexing by the runtime axis
    const R ma = ax == 0 ? q[1] : (ax == 1 ? q[2] : q[3]);
    const R ua = ax == 0 ? u[0] : (ax == 1 ? u[1] : u[2]);
    const R Ba = ax == 0 ? B[0] : (ax == 1 ? B[1] : B[2]);
    R phi[8];
    phi[0] = ma;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        phi[1 + b] = ma * u[b] - Ba * B[b] + (ax == b ? pt : R(0));
        phi[5 + b] = (ax == b) ? R(0) : ua * B[b] - Ba * u[b];
    }
    phi[4] = (q[4] + pt) * ua - Ba * uB;

    const int din = (face & 1) ? 2 * ax + 2 : 2 * ax + 1;  // +e_ax enters at the low face
    const R half = (face & 1) ? R(-AxisSet<D>::w1 / AxisSet<D>::cs2) : R(AxisSet<D>::w1 / AxisSet<D>::cs2);
    int j = din;
    int64_t at = cell;
    if (a.parity) {  // slot (opp i, x - c_i): x - c_i wraps to the opposite face
        j = opp_axis(din);
        const int64_t step = ax == 0 ? 1 : (ax == 1 ? (int64_t)a.nx : (int64_t)a.nx * a.ny);
        const int64_t span = ax == 0 ? (int64_t)a.nx : (ax == 1 ? (int64_t)a.ny : (int64_t)a.nz);
        at = high ? cell + step - span * step : cell - step + span * step;
    }
    S *pop = static_cast<S *>(const_cast<void *>(a.pop));
#pragma unroll
    for (int k = 0; k < 8; ++k)
        Codec<S>::store(pop + (int64_t)(k * Q + j) * a.stride + at, R(AxisSet<D>::w1) * q[k] + half * phi[k]);
}

// HLBM porosity of the signed distance phi (sec. 2.4): 0 in the solid, 1 in the
// fluid, phi / eps_h + 1/2 across the transition of width eps_h.
__global__ void k_porosity(const float *__restrict__ phi, int64_t n, float eps_h, float *__restrict__ d)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float v = phi[t];
    d[t] = v <= -0.5f * eps_h ? 0.f : (v >= 0.5f * eps_h ? 1.f : v / eps_h + 0.5f);
}

// Closure input features from the populations: the FP32 moments of
// k_ideal_moments, normalised and rounded to BF16, 16 bytes per cell.
struct FeatureNorm {
    float mu[8], inv_sigma[8];
};

template <int D, class S>
__global__ void k_ideal_features(const ReadArgs<D, S> a, int64_t count, const FeatureNorm fn,
                                 __nv_bfloat16 *__restrict__ x)
{
    constexpr int Q = AxisSet<D>::Q;
    const int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (cell >= count) return;
    int cx, cy, cz;
    cell_xyz<D>(cell, a.nx, a.ny, cx, cy, cz);
    int64_t nb[Q];
    neighbours<D>(cx, cy, cz, a.nx, a.ny, a.nz, cell, nb);
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
        v[k] = __float2bfloat16_rn(((float)cell_moment<D, S>(a, cell, nb, k) - fn.mu[k]) * fn.inv_sigma[k]);
    *reinterpret_cast<uint4 *>(x + cell * 8) = *reinterpret_cast<const uint4 *>(v);
}

template <int D, class S, int NL = 8>
__global__ void k_ideal_gather(const ReadArgs<D, S> a, const int64_t *__restrict__ cells, int n,
                               double *__restrict__ out)
{
    constexpr int Q = AxisSet<D>::Q;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int64_t cell = cells[t];
    int x, y, z;
    cell_xyz<D>(cell, a.nx, a.ny, x, y, z);
    int64_t nb[Q];
    neighbours<D>(x, y, z, a.nx, a.ny, a.nz, cell, nb);
#pragma unroll
    for (int k = 0; k < NL; ++k)
#pragma unroll
        for (int i = 0; i < Q; ++i) out[(int64_t)t * NL * Q + k * Q + i] = logical<D, S>(a, cell, nb, k, i);
}

// Domain sums of Q_k: each thread accumulates its cells in double, warps and
// the CTA reduce with shuffles and shared memory, one partial per CTA goes to
// the scratch array; k_finish_sums adds the partials in a fixed order.
template <int D, class S>
__global__ void __launch_bounds__(kReduceThreads) k_ideal_partials(const ReadArgs<D, S> a, int64_t ncell,
                                                                   double *__restrict__ partials)
{
    constexpr int Q = AxisSet<D>::Q;
    double acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = 0.0;
    for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < ncell;
         cell += (int64_t)gridDim.x * blockDim.x) {
        int x, y, z;
        cell_xyz<D>(cell, a.nx, a.ny, x, y, z);
        int64_t nb[Q];
        neighbours<D>(x, y, z, a.nx, a.ny, a.nz, cell, nb);
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] += (double)cell_moment<D, S>(a, cell, nb, k);
    }
    __shared__ double red[kReduceThreads / 32][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        double v = acc[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        double v = 0.0;
        for (int w = 0; w < kReduceThreads / 32; ++w) v += red[w][threadIdx.x];
        partials[(int64_t)blockIdx.x * 8 + threadIdx.x] = v;
    }
}

__global__ void k_finish_sums(const double *__restrict__ partials, int nblocks, int nvar,
                              double *__restrict__ sums)
{
    __shared__ double red[256];
    for (int k = 0; k < nvar; ++k) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partials[(int64_t)b * 8 + k];
        red[threadIdx.x] = v;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) sums[k] = red[0];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

template <class C> IdealArgs<C> make_step_args(vlbm_ctx *c)
{
    const Domain &d = c->dom[0];
    IdealArgs<C> a{};
    a.pop = c->pop;
    a.nx = d.nx;
    a.ny = d.ny;
    a.nz = d.nz;
    a.stride = d.stride;
    a.gm1 = C(d.gamma - 1.0);
    const double w0 = c->dim == 2 ? AxisSet<2>::w0 : AxisSet<3>::w0;
    const double w1 = c->dim == 2 ? AxisSet<2>::w1 : AxisSet<3>::w1;
    const bool dev = c->storage == VLBM_F16_DEV || c->storage == VLBM_BF16_DEV;
    for (int k = 0; k < kMaxLat; ++k) {
        const double s = dev ? d.q_scale[k] : 1.0;
        a.omega[k] = C(1.0 / d.tau[k]);
        a.src0[k] = C(w0 * d.source[k] / s);
        a.src1[k] = C(w1 * d.source[k] / s);
        a.ref[k] = C(dev ? d.q_ref[k] : 0.0);
        a.scale[k] = C(s);
        a.inv_scale[k] = C(1.0 / s);
    }
    a.flags = c->d_flags;
    a.inv_tau_m = C(1.0 / d.tau_m);
    a.solid = c->solid;
    a.solid_n = d.ncell;
    a.refscale = c->d_refscale;
    a.p_theta = C(dev ? c->params.p_theta : 0.0);
    return a;
}

template <int D, class S> ReadArgs<D, S> make_read_args(vlbm_ctx *c, int di)
{
    const Domain &d = c->dom[di];
    ReadArgs<D, S> a{};
    a.pop = static_cast<const char *>(c->pop) + d.offset * c->elem;
    a.nx = d.nx;
    a.ny = d.ny;
    a.nz = d.nz;
    a.stride = d.stride;
    a.parity = (int)(c->step & 1);
    for (int k = 0; k < kMaxLat; ++k) {
        a.ref[k] = d.q_ref[k];
        a.scale[k] = d.q_scale[k];
    }
    return a;
}

template <int D, class S, class C> vlbm_status step_t(vlbm_ctx *c, int parity)
{
    const Domain &d = c->dom[0];
    const IdealArgs<C> a = make_step_args<C>(c);
    const dim3 grid((unsigned)((d.nx + kBlockX - 1) / kBlockX), (unsigned)d.ny, (unsigned)d.nz);
    if constexpr (!Codec<S>::kDev) {
        if (c->solid) {  // homogenised solids
            if (parity)
                k_ideal_step<D, S, C, true, false, 8, true><<<grid, kBlockX, 0, c->stream>>>(a);
            else
                k_ideal_step<D, S, C, false, false, 8, true><<<grid, kBlockX, 0, c->stream>>>(a);
            c->launches++;
            return cuda_check(c, cudaGetLastError(), "homogenised step launch");
        }
        if (c->nlat == 9) {  // Powell model
            if (parity)
                k_ideal_step<D, S, C, true, false, 9><<<grid, kBlockX, 0, c->stream>>>(a);
            else
                k_ideal_step<D, S, C, false, false, 9><<<grid, kBlockX, 0, c->stream>>>(a);
            c->launches++;
            return cuda_check(c, cudaGetLastError(), "Powell step launch");
        }
    }
    if constexpr (D == 3 && Codec<S>::kDev) {
        if (d.nx % 8 == 0) {  // 16-byte aligned rows: bulk-copy loads, persistent CTAs
            if (c->bulk_ctas == 0) {  // every SM filled to the kernel's occupancy
                int dev = 0, sms = 1, per_sm = 1;
                cudaGetDevice(&dev);
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ideal_step_pairs<S, false>, kPairThreads, 0);
                c->bulk_ctas = std::max(1, sms) * std::max(1, per_sm);
            }
            const int ntiles = (int)grid.x * d.ny * d.nz;
            const unsigned g = (unsigned)std::min(ntiles, c->bulk_ctas);
            if (parity)
                k_ideal_step_pairs<S, true><<<g, kPairThreads, 0, c->stream>>>(a);
            else
                k_ideal_step_pairs<S, false><<<g, kPairThreads, 0, c->stream>>>(a);
            c->launches++;
            return cuda_check(c, cudaGetLastError(), "ideal step launch");
        }
    }
    if constexpr (Codec<S>::kDev) {
        if (parity)
            k_ideal_step_dev<D, S, true><<<grid, kBlockX, 0, c->stream>>>(a);
        else
            k_ideal_step_dev<D, S, false><<<grid, kBlockX, 0, c->stream>>>(a);
    } else {
        if (parity)
            k_ideal_step<D, S, C, true><<<grid, kBlockX, 0, c->stream>>>(a);
        else
            k_ideal_step<D, S, C, false><<<grid, kBlockX, 0, c->stream>>>(a);
    }
    c->launches++;
    return cuda_check(c, cudaGetLastError(), "ideal step launch");
}

template <int D, class S> vlbm_status init_t(vlbm_ctx *c, int di, const double *Q, int64_t c0, int64_t count,
                                             int64_t qstride)
{
    const Domain &d = c->dom[di];
    InitArgs<D, S> a{};
    a.pop = static_cast<char *>(c->pop) + d.offset * c->elem;
    a.stride = d.stride;
    a.c0 = c0;
    a.count = count;
    a.qstride = qstride;
    a.gamma = d.gamma;
    for (int k = 0; k < kMaxLat; ++k) {
        a.ref[k] = d.q_ref[k];
        a.scale[k] = d.q_scale[k];
    }
    a.flags = c->d_flags;
    a.p_theta = c->params.p_theta;
    const int threads = 256;
    const unsigned blocks = (unsigned)((count + threads - 1) / threads);
    if constexpr (!Codec<S>::kDev) {
        if (c->nlat == 9) {
            k_ideal_init<D, S, 9><<<blocks, threads, 0, c->stream>>>(a, Q);
            c->launches++;
            return cuda_check(c, cudaGetLastError(), "Powell init launch");
        }
    }
    k_ideal_init<D, S><<<blocks, threads, 0, c->stream>>>(a, Q);
    c->launches++;
    return cuda_check(c, cudaGetLastError(), "ideal init launch");
}

template <int D, class S> vlbm_status moments_t(vlbm_ctx *c, int di, double *out, int64_t c0, int64_t count,
                                                int64_t ostride)
{
    const int threads = 256;
    const unsigned blocks = (unsigned)((count + threads - 1) / threads);
    if (c->nlat == 9)
        k_ideal_moments<D, S, 9><<<blocks, threads, 0, c->stream>>>(make_read_args<D, S>(c, di), c0, count, ostride,
                                                                   out);
    else
        k_ideal_moments<D, S><<<blocks, threads, 0, c->stream>>>(make_read_args<D, S>(c, di), c0, count, ostride, out);
    c->launches++;
    return cuda_check(c, cudaGetLastError(), "ideal moments launch");
}

template <int D, class S> vlbm_status gather_t(vlbm_ctx *c, int di, const int64_t *cells, int n, double *out)
{
    const int threads = 128;
    const unsigned blocks = (unsigned)((n + threads - 1) / threads);
    if (c->nlat == 9)
        k_ideal_gather<D, S, 9><<<blocks, threads, 0, c->stream>>>(make_read_args<D, S>(c, di), cells, n, out);
    else
        k_ideal_gather<D, S><<<blocks, threads, 0, c->stream>>>(make_read_args<D, S>(c, di), cells, n, out);
    c->launches++;
    return cuda_check(c, cudaGetLastError(), "ideal gather launch");
}

template <int D, class S> vlbm_status sums_t(vlbm_ctx *c, int di, double *sums)
{
    k_ideal_partials<D, S><<<kReduceBlocks, kReduceThreads, 0, c->stream>>>(make_read_args<D, S>(c, di),
                                                                             c->dom[di].ncell, c->d_partials);
    c->launches++;
    vlbm_status s = cuda_check(c, cudaGetLastError(), "ideal partial sums launch");
    if (s != VLBM_OK) return s;
    return finish_sums(c, 8, sums);
}

template <int D, class S> vlbm_status open_fill_t(vlbm_ctx *c, int parity)
{
    ReadArgs<D, S> a = make_read_args<D, S>(c, 0);
    a.parity = parity;  // explicit: graph capture does not advance c->step
    OpenFaces o{};
    const Domain &d = c->dom[0];
    const int64_t n[3] = {d.nx, d.ny, d.nz};
    int64_t most = 0;
    for (int f = 0; f < 2 * D; ++f) {
        if (c->face_kind[f] != VLBM_BC_EQUILIBRIUM) continue;
        const int ax = f >> 1;
        o.open[ax] = 1;
        o.mask[f] = c->face_mask[f];
        for (int k = 0; k < 8; ++k) o.vals[f][k] = c->face_vals[f][k];
        o.count[f] = n[0] * n[1] * n[2] / n[ax];
        most = std::max(most, o.count[f]);
    }
    o.gm1 = d.gamma - 1.0;
    if (most == 0) return VLBM_OK;
    const int threads = 256;
    const dim3 grid((unsigned)((most + threads - 1) / threads), (unsigned)(2 * D));
    k_open_fill<D, S><<<grid, threads, 0, c->stream>>>(a, o, c->d_flags);
    c->launches++;
    return cuda_check(c, cudaGetLastError(), "boundary fill launch");
}

// dispatch on (dim, storage)
template <template <int, class> class F, class... A> vlbm_status dispatch(vlbm_ctx *c, A... args)
{
    const int D = c->dim;
    switch (c->storage) {
    case VLBM_F64: return D == 2 ? F<2, double>::run(c, args...) : F<3, double>::run(c, args...);
    case VLBM_F32: return D == 2 ? F<2, float>::run(c, args...) : F<3, float>::run(c, args...);
    case VLBM_F16_DEV: return D == 2 ? F<2, __half>::run(c, args...) : F<3, __half>::run(c, args...);
    case VLBM_BF16_DEV:
        return D == 2 ? F<2, __nv_bfloat16>::run(c, args...) : F<3, __nv_bfloat16>::run(c, args...);
    }
    return fail(c, VLBM_ERR_UNSUPPORTED, "unknown storage");
}

template <int D, class S> struct StepF {
    static vlbm_status run(vlbm_ctx *c, int parity)
    {
        if constexpr (std::is_same<S, double>::value) return step_t<D, S, double>(c, parity);
        else return step_t<D, S, float>(c, parity);
    }
};
template <int D, class S> struct InitF {
    static vlbm_status run(vlbm_ctx *c, int di, const double *Q, int64_t c0, int64_t n, int64_t qs)
    {
        return init_t<D, S>(c, di, Q, c0, n, qs);
    }
};
template <int D, class S> struct MomF {
    static vlbm_status run(vlbm_ctx *c, int di, double *out, int64_t c0, int64_t n, int64_t os)
    {
        return moments_t<D, S>(c, di, out, c0, n, os);
    }
};
template <int D, class S> struct GatherF {
    static vlbm_status run(vlbm_ctx *c, int di, const int64_t *cells, int n, double *out)
    {
        return gather_t<D, S>(c, di, cells, n, out);
    }
};
template <int D, class S> struct SumsF {
    static vlbm_status run(vlbm_ctx *c, int di, double *sums) { return sums_t<D, S>(c, di, sums); }
};
template <int D, class S> struct OpenF {
    static vlbm_status run(vlbm_ctx *c, int parity)
    {
        if constexpr (Codec<S>::kDev) return fail(c, VLBM_ERR_UNSUPPORTED, "open faces need F32 or F64 storage");
        else return open_fill_t<D, S>(c, parity);
    }
};

}  // namespace

vlbm_status finish_sums(vlbm_ctx *c, int nvar, double *sums_dev)
{
    k_finish_sums<<<1, 256, 0, c->stream>>>(c->d_partials, kReduceBlocks, nvar, sums_dev);
    c->launches++;
    return cuda_check(c, cudaGetLastError(), "finish sums launch");
}

vlbm_status ideal_step(vlbm_ctx *c, int parity) { return dispatch<StepF>(c, parity); }

vlbm_status ideal_step_corrected(vlbm_ctx *c, int parity, const float *dphi)
{
    if (c->dim != 3 || c->storage != VLBM_F32) return fail(c, VLBM_ERR_UNSUPPORTED, "closure needs 3-D F32 storage");
    const Domain &d = c->dom[0];
    IdealArgs<float> a = make_step_args<float>(c);
    a.dphi = dphi;
    const dim3 grid((unsigned)((d.nx + kBlockX - 1) / kBlockX), (unsigned)d.ny, (unsigned)d.nz);
    if (parity)
        k_ideal_step<3, float, float, true, true><<<grid, kBlockX, 0, c->stream>>>(a);
    else
        k_ideal_step<3, float, float, false, true><<<grid, kBlockX, 0, c->stream>>>(a);
    c->launches++;
    return cuda_check(c, cudaGetLastError(), "corrected step launch");
}

vlbm_status ideal_init_range(vlbm_ctx *c, int d, const double *Q, int64_t c0, int64_t n, int64_t qstride)
{
    return dispatch<InitF>(c, d, Q, c0, n, qstride);
}

vlbm_status ideal_moments_range(vlbm_ctx *c, int d, double *out, int64_t c0, int64_t n, int64_t ostride)
{
    return dispatch<MomF>(c, d, out, c0, n, ostride);
}

vlbm_status ideal_init(vlbm_ctx *c, int d, const double *Q_dev)
{
    const int64_t N = c->dom[d].ncell;
    return ideal_init_range(c, d, Q_dev, 0, N, N);
}

vlbm_status ideal_moments(vlbm_ctx *c, int d, double *Q_dev)
{
    const int64_t N = c->dom[d].ncell;
    return ideal_moments_range(c, d, Q_dev, 0, N, N);
}

vlbm_status ideal_gather(vlbm_ctx *c, int d, const int64_t *cells_dev, int n, double *out_dev)
{
    return dispatch<GatherF>(c, d, cells_dev, n, out_dev);
}

vlbm_status ideal_sums(vlbm_ctx *c, int d, double *sums_dev) { return dispatch<SumsF>(c, d, sums_dev); }

bool any_open_face(const vlbm_ctx *c)
{
    for (int f = 0; f < 6; ++f)
        if (c->face_kind[f] == VLBM_BC_EQUILIBRIUM) return true;
    return false;
}

vlbm_status open_fill(vlbm_ctx *c, int parity) { return dispatch<OpenF>(c, parity); }

vlbm_status wait_check(vlbm_ctx *c, uint32_t tries)
{
    k_wait_check<<<1, 1, 0, c->stream>>>(c->d_flags, tries);
    c->launches++;
    return cuda_check(c, cudaGetLastError(), "bounded-wait check launch");
}

vlbm_status porosity_from_distance(const float *phi, int64_t n, double eps_h, float *d, cudaStream_t s)
{
    const int threads = 256;
    k_porosity<<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(phi, n, (float)eps_h, d);
    return cuda_check(nullptr, cudaGetLastError(), "porosity launch");
}

vlbm_status ideal_features(vlbm_ctx *c, const float *mu, const float *inv_sigma, __nv_bfloat16 *x)
{
    if (c->batched || c->dim != 3 || c->storage != VLBM_F32)
        return fail(c, VLBM_ERR_ARG, "closure features need a 3-D FP32 context");
    FeatureNorm fn{};
    for (int k = 0; k < 8; ++k) {
        fn.mu[k] = mu[k];
        fn.inv_sigma[k] = inv_sigma[k];
    }
    const int64_t N = c->dom[0].ncell;
    const int threads = 256;
    k_ideal_features<3, float><<<(unsigned)((N + threads - 1) / threads), threads, 0, c->stream>>>(
        make_read_args<3, float>(c, 0), N, fn, x);
    c->launches++;
    return cuda_check(c, cudaGetLastError(), "closure features launch");
}

}  // namespace vlbm
