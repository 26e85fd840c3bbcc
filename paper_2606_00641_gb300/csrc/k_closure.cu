// k_closure.cu -- learned flux closure: BF16 tensor-core 3x3x3 convolutions
// (forward, backward-data, backward-weight), training step and application.
//
// The closure corrects the fluxes of a coarse ideal-MHD run (8 x D3Q7, FP32):
// a 3-layer periodic conv net maps the normalised conserved fields to
// dPhi[k][a], which the fused step kernel adds to the post-collision
// populations (f*_{k,+-a} +-= dPhi/2; see include/vlbm.h).
//
// Convolutions are implicit GEMMs on the tcgen05 tensor cores (BF16 operands
// in shared memory, FP32 accumulators in TMEM): k_conv_tc for the forward and
// data-gradient passes (halo tiles loaded with TMA, the three z-taps stacked
// along N), k_wgrad_tc for the weight and bias gradients (both operands read
// MN-major from the staged tiles, fixed-order partial sums).  Grids the
// tcgen05 tiles do not divide fall back to mma.sync.m16n8k16 kernels (M = 16
// cells per warp along an x-row, N = output channels, K = 27 taps x input
// channels in chunks of 16; weight gradient per (cell block, tap) with FP32
// atomics).  Activations are BF16, channel-blocked (planes of 8 channels, see
// blk()); weights are re-packed after every update into the tcgen05 and the
// mma.sync operand layouts.
#include <algorithm>
#include <cmath>
#include <cstring>

#include <cuda.h>

#include <mutex>

#include "vlbm_internal.cuh"

namespace vlbm {
namespace {

constexpr int kH = 32;          // hidden channels
constexpr int kOut = 24;        // 8 fields x 3 axes
constexpr int kConvThreads = 128;
constexpr int kWgradCells = 2048;  // cells per weight-gradient CTA

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(bf16 lo, bf16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// Periodic offsets of the 3 x 3 x 3 neighbourhood of a cell (x, y, z):
// neighbour(dx, dy, dz) = cell + ox[dx+1] + oy[dy+1] + oz[dz+1].
struct Nbr {
    int ox[3], oy[3], oz[3];
};

__device__ __forceinline__ Nbr nbr_of(int x, int y, int z, int nx, int ny, int nz)
{
    Nbr n;
    const int plane = nx * ny, vol = plane * nz;
    n.ox[0] = x > 0 ? -1 : nx - 1;
    n.ox[1] = 0;
    n.ox[2] = x + 1 < nx ? 1 : 1 - nx;
    n.oy[0] = y > 0 ? -nx : plane - nx;
    n.oy[1] = 0;
    n.oy[2] = y + 1 < ny ? nx : nx - plane;
    n.oz[0] = z > 0 ? -plane : vol - plane;
    n.oz[1] = 0;
    n.oz[2] = z + 1 < nz ? plane : plane - vol;
    return n;
}

__device__ __forceinline__ int tap_nbr(const Nbr &n, int cell, int t)
{
    return cell + n.ox[t % 3] + n.oy[(t / 3) % 3] + n.oz[t / 9];
}

__device__ __forceinline__ Nbr nbr_cell(int cell, int nx, int ny, int nz)
{
    const int x = cell % nx;
    const int r = cell / nx;
    return nbr_of(x, r % ny, r / ny, nx, ny, nz);
}

// ---------------------------------------------------------------------------
// implicit-GEMM convolution (forward and backward-data)
// ---------------------------------------------------------------------------

// Activations and their gradients are stored channel-blocked: channel c of
// cell p of an N-cell field at ((c / 8) N + p) 8 + c % 8, i.e. planes of
// 16-byte cell records, one plane per block of 8 channels (a field with 8
// channels is simply [cell][8]).  A halo row of a plane is contiguous, which
// lets TMA load the convolution halos in long rows.
__host__ __device__ __forceinline__ size_t blk(size_t cell, int c, size_t N)
{
    return ((size_t)(c >> 3) * N + cell) * 8 + (c & 7);
}

struct ConvEpilogue {
    const float *bias;     // per output channel, or null
    int tanh_act;          // apply tanh
    const bf16 *deriv;     // multiply by (1 - d^2), d = channel col of the cell (channel-blocked), or null
    const float *scale;    // per output channel, or null
    bf16 *out_bf;          // BF16 output, channel-blocked, or null
    float *out_f;          // FP32 output [cell][os], or null
    int os;
};

// tanh on the special-function unit (tanh.approx.f32, relative error below
// 2^-10.9); the activations it feeds are stored in BF16 (2^-8).
__device__ __forceinline__ float tanh_fast(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int CS, int NT>
__global__ void __launch_bounds__(kConvThreads) k_conv(const bf16 *__restrict__ act, int nx, int ny, int nz,
                                                       const uint2 *__restrict__ frag, const ConvEpilogue e)
{
    constexpr int NCHUNK = CS == 8 ? 14 : 54;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tg = lane & 3;
    const int N = nx * ny * nz;
    const int cell0 = (blockIdx.x * (kConvThreads / 32) + warp) * 16;
    if (cell0 >= N) return;  // nx % 16 == 0: a warp's 16 cells are one x-row segment
    const int cA = cell0 + g, cB = cell0 + g + 8;
    const Nbr nA = nbr_cell(cA, nx, ny, nz), nB = nbr_cell(cB, nx, ny, nz);
    const uint32_t *act32 = reinterpret_cast<const uint32_t *>(act);
    float acc[NT][4];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;

#pragma unroll 2
    for (int j = 0; j < NCHUNK; ++j) {
        uint32_t a0, a1, a2, a3;
        if (CS == 32) {
            // channels 16 h + 2 tg (+1) and 16 h + 8 + 2 tg (+1): planes 2 h and 2 h + 1
            const int t = j >> 1, h = j & 1;
            const size_t qA = tap_nbr(nA, cA, t), qB = tap_nbr(nB, cB, t);
            const uint32_t *p0 = act32 + (size_t)(2 * h) * N * 4, *p1 = p0 + (size_t)N * 4;
            a0 = p0[qA * 4 + tg];
            a2 = p1[qA * 4 + tg];
            a1 = p0[qB * 4 + tg];
            a3 = p1[qB * 4 + tg];
        } else {
            const int t0 = 2 * j, t1 = 2 * j + 1;
            a0 = act32[(size_t)tap_nbr(nA, cA, t0) * 4 + tg];
            a1 = act32[(size_t)tap_nbr(nB, cB, t0) * 4 + tg];
            if (t1 < 27) {
                a2 = act32[(size_t)tap_nbr(nA, cA, t1) * 4 + tg];
                a3 = act32[(size_t)tap_nbr(nB, cB, t1) * 4 + tg];
            } else {
                a2 = a3 = 0u;
            }
        }
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const uint2 b = __ldg(frag + ((size_t)j * NT + nt) * 32 + lane);
            mma_bf16(acc[nt], a0, a1, a2, a3, b.x, b.y);
        }
    }

#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        const int col = nt * 8 + 2 * tg;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int cell = half ? cB : cA;
            float v0 = acc[nt][2 * half], v1 = acc[nt][2 * half + 1];
            if (e.bias) {
                v0 += e.bias[col];
                v1 += e.bias[col + 1];
            }
            if (e.tanh_act) {
                v0 = tanh_fast(v0);
                v1 = tanh_fast(v1);
            }
            if (e.deriv) {
                const float d0 = __bfloat162float(e.deriv[blk(cell, col, N)]);
                const float d1 = __bfloat162float(e.deriv[blk(cell, col, N) + 1]);
                v0 *= 1.f - d0 * d0;
                v1 *= 1.f - d1 * d1;
            }
            if (e.scale) {
                v0 *= e.scale[col];
                v1 *= e.scale[col + 1];
            }
            if (e.out_bf) {
                __nv_bfloat162 o;
                o.x = __float2bfloat16_rn(v0);
                o.y = __float2bfloat16_rn(v1);
                *reinterpret_cast<__nv_bfloat162 *>(e.out_bf + blk(cell, col, N)) = o;
            } else {
                *reinterpret_cast<float2 *>(e.out_f + (size_t)cell * e.os + col) = make_float2(v0, v1);
            }
        }
    }
}

// Shared-memory variant: one CTA = 8 warps = a 16 x 8 (x, y) patch of cells
// at one z.  The patch and its one-cell halo (18 x 10 x 3 cells) are staged
// in shared memory with 16-byte copies; A fragments come from it by
// ldmatrix.x4 (16 cell rows x 8 channels per 8x8 matrix).  Channel rows are
// padded (CS = 32: 80 bytes) so the 8 rows of a matrix hit distinct banks.
constexpr int kTx = 16, kTy = 8;
constexpr int kHx = kTx + 2, kHy = kTy + 2, kHalo = kHx * kHy * 3;

__device__ __forceinline__ void ldmatrix_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

template <int CS, int NT>
__global__ void __launch_bounds__(kTx * kTy * 2) k_conv_smem(const bf16 *__restrict__ act, int nx, int ny, int nz,
                                                             const uint2 *__restrict__ frag, const ConvEpilogue e)
{
    constexpr int NCHUNK = CS == 8 ? 14 : 54;
    constexpr int ROW = CS == 8 ? 8 : 40;        // bf16 per staged cell (padded)
    constexpr int VEC = CS / 8;                  // 16-byte pieces per cell
    __shared__ __align__(16) bf16 tile[kHalo * ROW];
    const int x0 = blockIdx.x * kTx, y0 = blockIdx.y * kTy, z = blockIdx.z;
    const int plane = nx * ny;
    const size_t N = (size_t)plane * nz;
    // stage the halo box: (bx, by, bz) -> cell (x0-1+bx, y0-1+by, z-1+bz), periodic
    for (int idx = threadIdx.x; idx < kHalo * VEC; idx += blockDim.x) {
        const int piece = idx % VEC, c = idx / VEC;
        const int bx = c % kHx, by = (c / kHx) % kHy, bz = c / (kHx * kHy);
        int gx = x0 - 1 + bx, gy = y0 - 1 + by, gz = z - 1 + bz;
        gx += gx < 0 ? nx : (gx >= nx ? -nx : 0);
        gy += gy < 0 ? ny : (gy >= ny ? -ny : 0);
        gz += gz < 0 ? nz : (gz >= nz ? -nz : 0);
        const size_t cell = (size_t)gx + (size_t)nx * gy + (size_t)plane * gz;
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(act + blk(cell, piece * 8, N)));
        *reinterpret_cast<uint4 *>(tile + c * ROW + piece * 8) = v;
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;  // warp = row y0 + warp
    const int g = lane >> 2, tg = lane & 3;
    const int m = lane >> 3, rr = lane & 7;                      // ldmatrix: matrix m, row rr
    const uint32_t tile_s = (uint32_t)__cvta_generic_to_shared(tile);
    float acc[NT][4];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;

#pragma unroll 2
    for (int j = 0; j < NCHUNK; ++j) {
        int t, col;
        if (CS == 32) {
            t = j >> 1;
            col = (j & 1) * 16 + (m >> 1) * 8;  // matrices 2, 3 hold channels +8
        } else {
            t = 2 * j + (m >> 1);               // matrices 2, 3 hold the second tap
            col = 0;
        }
        const int tt = t < 27 ? t : 13;         // padding tap: any valid row, zeroed below
        const int dx = tt % 3 - 1, dy = (tt / 3) % 3 - 1, dz = tt / 9 - 1;
        const int r = (m & 1) * 8 + rr;         // cell row of the 16 within the warp
        const int c = (1 + dz) * (kHx * kHy) + (warp + 1 + dy) * kHx + (r + 1 + dx);
        uint32_t a0, a1, a2, a3;
        ldmatrix_x4(tile_s + (uint32_t)((c * ROW + col) * 2), a0, a1, a2, a3);
        if (CS == 8 && 2 * j + 1 >= 27) a2 = a3 = 0u;
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const uint2 b = __ldg(frag + ((size_t)j * NT + nt) * 32 + lane);
            mma_bf16(acc[nt], a0, a1, a2, a3, b.x, b.y);
        }
    }

    const int cA = (x0 + g) + nx * (y0 + warp) + plane * z, cB = cA + 8;
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        const int col = nt * 8 + 2 * tg;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int cell = half ? cB : cA;
            float v0 = acc[nt][2 * half], v1 = acc[nt][2 * half + 1];
            if (e.bias) {
                v0 += e.bias[col];
                v1 += e.bias[col + 1];
            }
            if (e.tanh_act) {
                v0 = tanh_fast(v0);
                v1 = tanh_fast(v1);
            }
            if (e.deriv) {
                const float d0 = __bfloat162float(e.deriv[blk(cell, col, N)]);
                const float d1 = __bfloat162float(e.deriv[blk(cell, col, N) + 1]);
                v0 *= 1.f - d0 * d0;
                v1 *= 1.f - d1 * d1;
            }
            if (e.scale) {
                v0 *= e.scale[col];
                v1 *= e.scale[col + 1];
            }
            if (e.out_bf) {
                __nv_bfloat162 o;
                o.x = __float2bfloat16_rn(v0);
                o.y = __float2bfloat16_rn(v1);
                *reinterpret_cast<__nv_bfloat162 *>(e.out_bf + blk(cell, col, N)) = o;
            } else {
                *reinterpret_cast<float2 *>(e.out_f + (size_t)cell * e.os + col) = make_float2(v0, v1);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// tcgen05 convolution (5th-generation tensor cores, accumulators in TMEM)
// ---------------------------------------------------------------------------
// Tile = 8 (x) x 16 (y) cells at one z = the M = 128 rows of one
// tcgen05.mma.cta_group::1.kind::f16 (BF16 in, FP32 accumulate), N = 32
// output channels (24-channel layers use zero weights for 24..31), K = 16 per
// instruction.  The halo box (10 x 18 x 3 cells) is staged as channel-block
// planes: plane cb holds channels 8cb..8cb+7 of every box cell (16 bytes per
// cell), so 8 x-consecutive cells form one 128-byte core matrix and each tap
// is only a start offset of the shared-memory descriptor: rows m = 8y + x,
// 8-row groups 160 bytes apart (SBO), K-adjacent core matrices one plane
// (Cin = 32) or one tap (Cin = 8) apart (LBO).  The weights of the layer sit
// in shared memory in the same canonical K-major layout.  Persistent CTAs:
// weights once, then one tile after another; one thread issues the MMAs,
// tcgen05.commit arrives on an mbarrier (bounded wait), and each warp reads
// its 32 TMEM lanes (= its 32 cells) with tcgen05.ld.
constexpr int kTcX = 8, kTcY = 16, kTcZ = 4;  // tile: kTcZ z-slices of 128 cells (one M block each)
constexpr int kTcHx = kTcX + 2, kTcHy = kTcY + 2, kTcHz = kTcZ + 2, kTcHalo = kTcHx * kTcHy * kTcHz;
constexpr int kTcPlane = kTcHalo * 16;    // bytes per channel-block plane
constexpr int kTcThreads = 480;           // warps 0-7 drain, 8-12 patch, 13 loads (TMA), 14 issues the MMAs
constexpr int kTcStage = 160;             // patching threads (warps 8-12)
constexpr int kTcBufs = 2;                // halo buffers
constexpr int kTcN = 96;                  // MMA N: 3 z-taps x 32 output channels
constexpr int kTcSetCols = 32 * (kTcZ + 4);  // one accumulator set: slices -2 .. kTcZ + 1
constexpr int kTcCols = 2 * kTcSetCols;   // two sets = all 512 TMEM columns
constexpr uint32_t kTcWaitLimit = 1u << 24;

// weight chunks of K = 16: (2-D tap, half of the 32 channels), or pairs of
// 2-D taps of the 8 channels; each chunk is 96 rows (dz, output channel) x 16
constexpr int tc_nchunk(int cs) { return cs == 8 ? 5 : 18; }

template <int CS>
constexpr int tc_smem_bytes()
{
    return tc_nchunk(CS) * kTcN * 32 + kTcBufs * (CS / 8) * kTcPlane;
}

// Bounded wait for the given phase of an mbarrier.  Each try_wait may park
// the warp for up to kTcSuspendNs (it resumes as soon as the phase completes),
// so waiting warps take no issue slots from the working ones.  Gives up after
// kTcWaitIters tries (about 1.3 s), or early once another role of the CTA has
// given up (*abort set); returns false then, and a give-up sets *abort itself.
constexpr uint32_t kTcSuspendNs = 20000;
constexpr uint32_t kTcWaitIters = 1u << 16;

__device__ __forceinline__ bool tc_wait(uint32_t mb, uint32_t phase, volatile int *abort)
{
    for (uint32_t it = 0; it < kTcWaitIters; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(done)
                     : "r"(mb), "r"(phase), "r"(kTcSuspendNs)
                     : "memory");
        if (done) return true;
        if (*abort) return false;
    }
    *abort = 1;
    return false;
}

// Bounded wait that ignores the abort flag: on the way out of a CTA that gave up,
// for the bulk copies it started to land before its shared memory is released.
__device__ __forceinline__ void tc_drain(uint32_t mb, uint32_t phase)
{
    for (uint32_t it = 0; it < kTcWaitIters; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(done)
                     : "r"(mb), "r"(phase), "r"(kTcSuspendNs)
                     : "memory");
        if (done) return;
    }
}

__device__ __forceinline__ void tc_arrive(uint32_t mb)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(mb) : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t mb)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mb)
                 : "memory");
}

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of the sm_100 family; no swizzle
    return d;
}

__device__ __forceinline__ void tc_mma(uint32_t dacc, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                 ::"r"(dacc), "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

// 3x3x3 convolution on the tcgen05 tensor cores.
// Tile = 8 (x) x 16 (y) x kTcZ (z) cells; each z-slice is one M = 128 block.
// The three z-taps are stacked along N: halo plane h (2-D tap (dx, dy),
// K-chunk j) times [W(dz=0) | W(dz=1) | W(dz=2)] (N = 96) contributes to the
// output slices h, h-1 and h-2 at once.  Slice s accumulates in the TMEM
// columns 32 (kTcZ + 1 - s) of a set, so the three 32-column blocks that one
// MMA writes are exactly those slices; the blocks of s = -2, -1, kTcZ,
// kTcZ + 1 collect products that belong to no slice of the tile and are
// never read.  One M128 x N96 x K16 MMA costs about as much as an N32 one,
// so this takes 3 (kTcZ + 2) / (3 kTcZ) of the instructions per cell of
// one-tap-per-MMA.  Every MMA accumulates: the drain clears the blocks it
// reads (and all of them at start).
// A operand: the halo, staged as 16-byte channel-block planes, so that a 2-D
// tap is an address offset (K-major, no swizzle).  B operand: the weights,
// resident in shared memory.  One persistent CTA per SM, three roles handing
// work over through mbarriers:
//   warp 13     loads the halo boxes into two buffers with TMA      (tma[b])
//   warps 8-12  patch the periodic images on the boundary (cp.async) (full[b])
//   warp 14     issues the MMAs of a tile into one of two TMEM sets  (empty[b], tfull[s])
//   warps 0-7   drain a finished set: warp w reads TMEM lanes 32 (w % 4)
//               of slices w / 4 and w / 4 + 2 (tanh derivative or bias,
//               tanh, scale; BF16 or FP32 store), then clears them    (tempty[s])
template <int CS>
__global__ void __launch_bounds__(kTcThreads, 1) k_conv_tc(const bf16 *__restrict__ act, int nx, int ny, int nz,
                                                           const bf16 *__restrict__ wtc, int cout_real,
                                                           const ConvEpilogue e, unsigned *err,
                                                           const __grid_constant__ CUtensorMap halo_map)
{
    constexpr int NCHUNK = tc_nchunk(CS);
    constexpr int NPLANE = CS / 8;
    constexpr int WBYTES = NCHUNK * kTcN * 32;
    constexpr int HBYTES = NPLANE * kTcPlane;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar[3 * kTcBufs + 4];  // full[2], empty[2], tfull[2], tempty[2], tma[2]
    __shared__ uint32_t tmem_base;
    __shared__ float s_bias[32], s_scale[32];
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = nx / kTcX, tiles_y = ny / kTcY, tiles_z = nz / kTcZ;
    const int ntiles = tiles_x * tiles_y * tiles_z;
    const int plane = nx * ny;
    const size_t N = (size_t)plane * nz;
    const int n_my = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const uint32_t bar_s = (uint32_t)__cvta_generic_to_shared(bar);
    auto full = [&](int b) { return bar_s + 8u * (uint32_t)b; };
    auto empty = [&](int b) { return bar_s + 8u * (uint32_t)(kTcBufs + b); };
    auto tfull = [&](int s2) { return bar_s + 8u * (uint32_t)(2 * kTcBufs + s2); };
    auto tempty = [&](int s2) { return bar_s + 8u * (uint32_t)(2 * kTcBufs + 2 + s2); };
    auto tma_bar = [&](int b) { return bar_s + 8u * (uint32_t)(2 * kTcBufs + 4 + b); };
    auto slice_col = [](int zz) { return (uint32_t)(32 * (kTcZ + 1 - zz)); };

    for (int i = tid; i < WBYTES / 16; i += kTcThreads)
        reinterpret_cast<uint4 *>(smem)[i] = __ldg(reinterpret_cast<const uint4 *>(wtc) + i);
    if (tid < 32) {  // absent bias / scale: 0 / 1, exact
        s_bias[tid] = e.bias && tid < cout_real ? e.bias[tid] : 0.f;
        s_scale[tid] = e.scale && tid < cout_real ? e.scale[tid] : 1.f;
    }
    if (warp == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&tmem_base);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(dst), "r"(kTcCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        s_abort = 0;
        for (int b = 0; b < kTcBufs; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(full(b)), "r"(kTcStage));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(empty(b)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tma_bar(b)));
        }
        for (int s2 = 0; s2 < 2; ++s2) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tfull(s2)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;\n" ::"r"(tempty(s2)));
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t sw_s = (uint32_t)__cvta_generic_to_shared(smem);
    const uint32_t sh_s = sw_s + WBYTES;
    volatile int *abort = &s_abort;
    uint32_t zero[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) zero[c] = 0u;
    auto tmem_clear = [&](uint32_t taddr) {
        asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                     "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n"
                     ::"r"(taddr), "r"(zero[0]), "r"(zero[1]), "r"(zero[2]), "r"(zero[3]), "r"(zero[4]),
                       "r"(zero[5]), "r"(zero[6]), "r"(zero[7]), "r"(zero[8]), "r"(zero[9]), "r"(zero[10]),
                       "r"(zero[11]), "r"(zero[12]), "r"(zero[13]), "r"(zero[14]), "r"(zero[15]), "r"(zero[16]),
                       "r"(zero[17]), "r"(zero[18]), "r"(zero[19]), "r"(zero[20]), "r"(zero[21]), "r"(zero[22]),
                       "r"(zero[23]), "r"(zero[24]), "r"(zero[25]), "r"(zero[26]), "r"(zero[27]), "r"(zero[28]),
                       "r"(zero[29]), "r"(zero[30]), "r"(zero[31])
                     : "memory");
    };
    if (warp < 8) {  // clear the blocks this warp drains, in both sets
        const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
        for (int s2 = 0; s2 < 2; ++s2)
            for (int p = 0; p < 2; ++p)
                tmem_clear(tmem + lanes + (uint32_t)(s2 * kTcSetCols) + slice_col((warp >> 2) + 2 * p));
        asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

    auto origin = [&](int i, int &x0, int &y0, int &z0) {
        const int tile = (int)blockIdx.x + i * (int)gridDim.x;
        x0 = (tile % tiles_x) * kTcX;
        y0 = ((tile / tiles_x) % tiles_y) * kTcY;
        z0 = (tile / (tiles_x * tiles_y)) * kTcZ;
    };

    if (warp == 13) {
        // ---- halo loads: one thread issues, a tile ahead of the MMAs as far as the buffers allow,
        // one bulk tensor copy per channel-block plane (box of 18 x 6 rows of 10 cells x 16 bytes,
        // contiguous in the channel-blocked field); coordinates outside the grid read as zeros
        if (lane == 0) {
            const uint64_t map_addr = reinterpret_cast<uint64_t>(&halo_map);
            bool ok = true;
            int issued = 0;  // tiles whose halo copies this thread started
            for (int i = 0; i < n_my && ok; ++i) {
                const int b = i % kTcBufs;
                if (i >= kTcBufs && !tc_wait(empty(b), (uint32_t)((i / kTcBufs - 1) & 1), abort)) {
                    ok = false;
                    break;
                }
                int x0, y0, z0;
                origin(i, x0, y0, z0);
                const uint32_t hb = sh_s + (uint32_t)(b * HBYTES);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(tma_bar(b)),
                             "r"((uint32_t)HBYTES)
                             : "memory");
                for (int cb = 0; cb < NPLANE; ++cb)
                    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                                 " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(hb + (uint32_t)(cb * kTcPlane)),
                                 "l"(map_addr), "r"(8 * (x0 - 1)), "r"(y0 - 1), "r"(z0 - 1), "r"(cb), "r"(tma_bar(b))
                                 : "memory");
                issued = i + 1;
            }
            if (!ok || *abort) {
                if (!ok) atomicOr(err, kFlagTimeout);
                // the CTA gives up: the last copies of each buffer land before it exits
                for (int j = issued > kTcBufs ? issued - kTcBufs : 0; j < issued; ++j)
                    tc_drain(tma_bar(j % kTcBufs), (uint32_t)((j / kTcBufs) & 1));
            }
        }
    } else if (warp >= 8 && warp < 13) {
        // ---- patching: once a tile's box has landed, tiles on the boundary get the periodic
        // images of the out-of-grid halo cells with cp.async; then every patching thread
        // hands the buffer to the MMA warp (full[b])
        const int ptid = tid - 256;
        bool ok = true;
        for (int i = 0; i < n_my && ok; ++i) {
            const int b = i % kTcBufs;
            if (!tc_wait(tma_bar(b), (uint32_t)((i / kTcBufs) & 1), abort)) {
                ok = false;
                break;
            }
            int x0, y0, z0;
            origin(i, x0, y0, z0);
            if (x0 == 0 || x0 + kTcX == nx || y0 == 0 || y0 + kTcY == ny || z0 == 0 || z0 + kTcZ == nz) {
                const uint32_t hb = sh_s + (uint32_t)(b * HBYTES);
                for (int idx = ptid; idx < kTcHalo * NPLANE; idx += kTcStage) {
                    const int cb = idx % NPLANE, c = idx / NPLANE;
                    const int bx = c % kTcHx, by = (c / kTcHx) % kTcHy, bz = c / (kTcHx * kTcHy);
                    int gx = x0 - 1 + bx, gy = y0 - 1 + by, gz = z0 - 1 + bz;
                    if (gx >= 0 && gx < nx && gy >= 0 && gy < ny && gz >= 0 && gz < nz) continue;
                    gx += gx < 0 ? nx : (gx >= nx ? -nx : 0);
                    gy += gy < 0 ? ny : (gy >= ny ? -ny : 0);
                    gz += gz < 0 ? nz : (gz >= nz ? -nz : 0);
                    const size_t cell = (size_t)gx + (size_t)nx * gy + (size_t)plane * gz;
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(hb + (uint32_t)(cb * kTcPlane + c * 16)),
                                 "l"(act + ((size_t)cb * N + cell) * 8)
                                 : "memory");
                }
                asm volatile("cp.async.commit_group;\n" ::: "memory");
                asm volatile("cp.async.wait_group 0;\n" ::: "memory");
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            tc_arrive(full(b));
        }
        if (!ok && ptid == 0) atomicOr(err, kFlagTimeout);
    } else if (warp == 14) {
        // ---- MMA issue (one thread)
        if (lane == 0) {
            const uint32_t idesc =
                (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) | ((128u >> 4) << 24);
            const uint64_t db0 = tc_desc(sw_s, 128, 256);
            bool ok = true;
            for (int i = 0; i < n_my && ok; ++i) {
                const int b = i % kTcBufs, sa = i & 1;
                if (!tc_wait(full(b), (uint32_t)((i / kTcBufs) & 1), abort)) ok = false;
                if (ok && i >= 2 && !tc_wait(tempty(sa), (uint32_t)(((i >> 1) - 1) & 1), abort)) ok = false;
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t hb = sh_s + (uint32_t)(b * HBYTES);
                for (int h = 0; h < kTcHz; ++h) {
                    const uint32_t dacc = tmem + (uint32_t)(sa * kTcSetCols) + slice_col(h);
                    const uint32_t pofs = (uint32_t)(h * kTcHy * kTcHx * 16);
                    if (CS == 32) {  // chunk 2 t2 + kc: 2-D tap t2, channel blocks 2 kc and 2 kc + 1
                        const uint64_t da0 = tc_desc(hb + pofs, kTcPlane, kTcHx * 16);
                        int j = 0;
                        for (int dy = 0; dy < 3; ++dy)
                            for (int dx = 0; dx < 3; ++dx) {
                                const uint32_t ofs = (uint32_t)((dy * kTcHx + dx) * 16);
#pragma unroll
                                for (int kc = 0; kc < 2; ++kc, ++j)
                                    tc_mma(dacc, da0 + ((ofs + (uint32_t)(kc * 2 * kTcPlane)) >> 4),
                                           db0 + (uint64_t)(j * (kTcN * 32 / 16)), idesc, 1u);
                            }
                    } else {         // chunk j: 2-D taps 2j and 2j + 1 of the single plane
                        for (int j = 0; j < NCHUNK; ++j) {
                            const int t0 = 2 * j, t1 = 2 * j + 1;
                            const int o0 = ((t0 / 3) * kTcHx + t0 % 3) * 16;
                            const uint32_t lbo = t1 < 9 ? (uint32_t)(((t1 / 3) * kTcHx + t1 % 3) * 16 - o0) : 0u;
                            tc_mma(dacc, tc_desc(hb + pofs + (uint32_t)o0, lbo, kTcHx * 16),
                                   db0 + (uint64_t)(j * (kTcN * 32 / 16)), idesc, 1u);  // tap 9: zero weights
                        }
                    }
                }
                tc_commit(empty(b));
                tc_commit(tfull(sa));
            }
            if (!ok) atomicOr(err, kFlagTimeout);
        }
    } else if (warp < 8) {
        // ---- drain
        const int q = warp & 3;
        const int m = q * 32 + lane;  // tile row = x + 8 y
        bool ok = true;
        for (int i = 0; i < n_my && ok; ++i) {
            const int sa = i & 1;
            // tcgen05.ld is warp-collective: the whole warp takes one outcome
            if (!__all_sync(0xffffffffu, tc_wait(tfull(sa), (uint32_t)((i >> 1) & 1), abort))) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            int x0, y0, z0;
            origin(i, x0, y0, z0);
#pragma unroll 1
            for (int p = 0; p < 2; ++p) {
                const int zz = (warp >> 2) + 2 * p;
                uint32_t r[32];
                const uint32_t taddr =
                    tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(sa * kTcSetCols) + slice_col(zz);
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
                             "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                               "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
                               "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
                               "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
                               "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
                               "=r"(r[31])
                             : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                tmem_clear(taddr);
                const size_t cell =
                    (size_t)(x0 + (m & 7)) + (size_t)nx * (y0 + (m >> 3)) + (size_t)plane * (z0 + zz);
                float v[32];
                if (e.deriv) {
#pragma unroll
                    for (int qd = 0; qd < 4; ++qd) {
                        const uint4 dv = __ldg(reinterpret_cast<const uint4 *>(e.deriv + ((size_t)qd * N + cell) * 8));
                        const bf16 *dh = reinterpret_cast<const bf16 *>(&dv);
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            const float d = __bfloat162float(dh[c]);
                            v[qd * 8 + c] = __uint_as_float(r[qd * 8 + c]) * (1.f - d * d);
                        }
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < 32; ++c) v[c] = __uint_as_float(r[c]);
                }
                if (e.tanh_act) {
#pragma unroll
                    for (int c = 0; c < 32; ++c) v[c] = tanh_fast(v[c] + s_bias[c]) * s_scale[c];
                } else {
#pragma unroll
                    for (int c = 0; c < 32; ++c) v[c] = (v[c] + s_bias[c]) * s_scale[c];
                }
                if (e.out_bf) {
                    __align__(16) bf16 o[32];
#pragma unroll
                    for (int c = 0; c < 32; ++c) o[c] = __float2bfloat16_rn(c < cout_real ? v[c] : 0.f);
#pragma unroll
                    for (int qd = 0; qd < 4; ++qd)
                        *reinterpret_cast<uint4 *>(e.out_bf + ((size_t)qd * N + cell) * 8) =
                            reinterpret_cast<const uint4 *>(o)[qd];
                } else {
                    float *dst = e.out_f + cell * e.os;
#pragma unroll
                    for (int c = 0; c < 32; c += 4)
                        if (c < cout_real)
                            *reinterpret_cast<float4 *>(dst + c) = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
                }
            }
            // both blocks read and cleared: hand the set back to the MMA warp
            asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) tc_arrive(tempty(sa));
        }
        if (!ok && lane == 0) atomicOr(err, kFlagTimeout);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTcCols));
    }
}

// Weights in the canonical K-major layout of k_conv_tc: chunk j, row
// n = 32 dz + o (o < 32; zero beyond the output channels), K-index k (< 16)
// at j*1536 + (n/8)*128 + (k/8)*64 + (n%8)*8 + k%8 (bf16 elements).  Chunk j
// holds 2-D tap j/2 and channels 16 (j%2) + k (32 input channels), or 2-D tap
// 2j + k/8 and channel k%8 (8 input channels; 2-D tap 9 is zero).  The
// transposed pack (data gradient) swaps the channel roles and mirrors the tap.
__global__ void k_pack_tc(const float *__restrict__ W, int cout, int cin, int CS, int transpose,
                          bf16 *__restrict__ out)
{
    const int nchunk = tc_nchunk(CS);
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nchunk * kTcN * 16) return;
    const int j = idx / (kTcN * 16), rem = idx % (kTcN * 16);
    const int g = rem / 128, kh = (rem / 64) % 2, r = (rem / 8) % 8, e8 = rem % 8;
    const int n = g * 8 + r, k = kh * 8 + e8;
    const int dz = n / 32, o = n % 32;
    int t2, c;
    if (CS == 32) {
        t2 = j >> 1;
        c = (j & 1) * 16 + k;
    } else {
        t2 = 2 * j + (k >= 8 ? 1 : 0);
        c = k & 7;
    }
    float w = 0.f;
    if (t2 < 9) {
        const int t = 9 * dz + t2;
        if (!transpose) {
            if (o < cout && c < cin) w = W[((size_t)o * cin + c) * 27 + t];
        } else {
            if (o < cin && c < cout) w = W[((size_t)c * cin + o) * 27 + (26 - t)];
        }
    }
    out[idx] = __float2bfloat16_rn(w);
}

// B-fragment packing.  Chunk j, n-tile nt, lane l (g = l/4, tg = l%4) holds
// b0 = B[2tg..2tg+1][n], b1 = B[2tg+8..2tg+9][n] with n = 8 nt + g, where
// B[k][n] is the weight of K-index k of chunk j for output channel n.
// Forward:   B[(t,c)][n] = W[n][c][t].
// Transpose (backward-data): B[(t,c)][n] = W[c][n][26 - t]  (input c = a
// forward output channel, output n = a forward input channel).
__global__ void k_pack(const float *__restrict__ W, int cout, int cin, int CS, int NT, int transpose,
                       uint2 *__restrict__ frag)
{
    const int nchunk = CS == 8 ? 14 : 54;
    const int total = nchunk * NT * 32;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int lane = idx & 31, nt = (idx >> 5) % NT, j = (idx >> 5) / NT;
    const int g = lane >> 2, tg = lane & 3;
    const int n = nt * 8 + g;
    float v[4];
    const int ks[4] = {2 * tg, 2 * tg + 1, 2 * tg + 8, 2 * tg + 9};
    for (int q = 0; q < 4; ++q) {
        const int k = ks[q];
        int t, c;
        if (CS == 32) {
            t = j >> 1;
            c = (j & 1) * 16 + k;
        } else {
            t = 2 * j + (k >= 8 ? 1 : 0);
            c = k & 7;
        }
        float w = 0.f;
        if (t < 27) {
            if (!transpose) {
                if (n < cout && c < cin) w = W[((size_t)n * cin + c) * 27 + t];
            } else {
                if (n < cin && c < cout) w = W[((size_t)c * cin + n) * 27 + (26 - t)];
            }
        }
        v[q] = w;
    }
    uint2 out;
    out.x = pack_bf16(__float2bfloat16_rn(v[0]), __float2bfloat16_rn(v[1]));
    out.y = pack_bf16(__float2bfloat16_rn(v[2]), __float2bfloat16_rn(v[3]));
    frag[idx] = out;
}

// ---------------------------------------------------------------------------
// weight gradient: gW[o][c][t] += sum_cells gz[cell][o] * a[cell + e_t][c]
// A = gz^T (M = 32 output channels, K = cells), B = shifted inputs (K = cells,
// N = input channels).  One CTA per (block of kWgradCells cells, tap t).
// ---------------------------------------------------------------------------
template <int CSIN>
__global__ void __launch_bounds__(kConvThreads) k_wgrad(const bf16 *__restrict__ gz, const bf16 *__restrict__ a,
                                                        int nx, int ny, int nz, int cout, int cin,
                                                        float *__restrict__ gW)
{
    constexpr int NTW = CSIN / 8;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tg = lane & 3;
    const int t = blockIdx.y;
    const int N = nx * ny * nz;
    const unsigned short *gz16 = reinterpret_cast<const unsigned short *>(gz);
    const unsigned short *a16 = reinterpret_cast<const unsigned short *>(a);
    float acc[2][NTW][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < NTW; ++nt) acc[mt][nt][0] = acc[mt][nt][1] = acc[mt][nt][2] = acc[mt][nt][3] = 0.f;

    const int per_warp = kWgradCells / (kConvThreads / 32);
    const int begin = blockIdx.x * kWgradCells + warp * per_warp;
    for (int c0 = begin; c0 < begin + per_warp && c0 < N; c0 += 16) {
        // this lane's four cells of the k-step and their tap neighbours
        int cells[4] = {c0 + 2 * tg, c0 + 2 * tg + 1, c0 + 2 * tg + 8, c0 + 2 * tg + 9};
        int nbs[4];
        bool ok[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            ok[q] = cells[q] < N;
            const int cc = ok[q] ? cells[q] : 0;
            nbs[q] = tap_nbr(nbr_cell(cc, nx, ny, nz), cc, t);
        }
        auto gzv = [&](int q, int o) -> uint32_t {
            return ok[q] ? (uint32_t)gz16[blk(cells[q], o, N)] : 0u;
        };
        auto av = [&](int q, int c) -> uint32_t { return ok[q] ? (uint32_t)a16[blk(nbs[q], c, N)] : 0u; };
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const int olo = mt * 16 + g, ohi = olo + 8;
            const uint32_t a0 = gzv(0, olo) | (gzv(1, olo) << 16);
            const uint32_t a1 = gzv(0, ohi) | (gzv(1, ohi) << 16);
            const uint32_t a2 = gzv(2, olo) | (gzv(3, olo) << 16);
            const uint32_t a3 = gzv(2, ohi) | (gzv(3, ohi) << 16);
#pragma unroll
            for (int nt = 0; nt < NTW; ++nt) {
                const int c = nt * 8 + g;
                const uint32_t b0 = av(0, c) | (av(1, c) << 16);
                const uint32_t b1 = av(2, c) | (av(3, c) << 16);
                mma_bf16(acc[mt][nt], a0, a1, a2, a3, b0, b1);
            }
        }
    }
    // reduce the four warps in shared memory, then one atomic add per weight
    __shared__ float red[kConvThreads / 32][32][CSIN];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < NTW; ++nt) {
            const int o = mt * 16 + g, c = nt * 8 + 2 * tg;
            red[warp][o][c] = acc[mt][nt][0];
            red[warp][o][c + 1] = acc[mt][nt][1];
            red[warp][o + 8][c] = acc[mt][nt][2];
            red[warp][o + 8][c + 1] = acc[mt][nt][3];
        }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 32 * CSIN; idx += blockDim.x) {
        const int o = idx / CSIN, c = idx % CSIN;
        if (o >= cout || c >= cin) continue;
        float s = 0.f;
        for (int w = 0; w < kConvThreads / 32; ++w) s += red[w][o][c];
        atomicAdd(gW + ((size_t)o * cin + c) * 27 + t, s);
    }
}

// Bias gradient, coalesced: each thread reads whole 16-byte channel blocks of a
// cell; one partial per CTA, summed by k_part_sum (fixed order).
__global__ void __launch_bounds__(256) k_bgrad_part(const bf16 *__restrict__ gz, int N, int cout,
                                                    float *__restrict__ part)
{
    __shared__ float red[256][9];
    const int cb = threadIdx.x & 3;
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int c = blockIdx.x * 64 + (threadIdx.x >> 2); c < N; c += gridDim.x * 64) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(gz + ((size_t)cb * N + c) * 8));
        const bf16 *h = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
        for (int e = 0; e < 8; ++e) s[e] += __bfloat162float(h[e]);
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) red[threadIdx.x][e] = s[e];
    __syncthreads();
    const int o = threadIdx.x;
    if (o < cout) {
        float t = 0.f;
        for (int r = 0; r < 64; ++r) t += red[r * 4 + (o >> 3)][o & 7];
        part[(size_t)blockIdx.x * cout + o] = t;
    }
}

// out[j] += sum over blocks b of part[b * count + j]: a CTA takes 32 outputs,
// warp w sums the blocks b = w mod 8, then the eight sums are added in order
// (a fixed order, so the result does not depend on scheduling)
__global__ void __launch_bounds__(256) k_part_sum(const float *__restrict__ part, int nblk, int count,
                                                  float *__restrict__ out)
{
    __shared__ float red[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int j = blockIdx.x * 32 + lane;
    float s = 0.f;
    if (j < count) {
#pragma unroll 4
        for (int b = w; b < nblk; b += 8) s += __ldg(part + (size_t)b * count + j);
    }
    red[w][lane] = s;
    __syncthreads();
    if (w == 0 && j < count) {
        float t = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) t += red[q][lane];
        out[j] += t;
    }
}

// Weight gradient on the tcgen05 tensor cores:
//   gW[o][c][t] = sum over cells p of gz[p][o] * a[p + e_t][c]
// is a GEMM whose reduction runs over the cells.  Both operands are read in
// their natural cell-major layout (channels contiguous), i.e. as MN-major
// operands, from planes staged in shared memory:
//   A (M = 128 rows) = 4 z-offsets x 4 slots x 8 channels.  Row z-offset h is
//     the tap dz = h (h = 3 is computed and discarded).  With 32 input channels
//     the slots are the 4 channel blocks and there is one accumulator per
//     (dy, dx); with 8 input channels the slots hold copies of the halo
//     shifted by dx = 0, 1, 2 (slot 3 discarded) and there is one accumulator
//     per dy.  A tap (dy, dx) is an address offset into the staged planes.
//   B (N = 32) = the output-channel gradients of the tile's cells.
// Tiles of 8 x 16 x kWgZ cells; persistent CTAs (one per SM: the two staging
// buffers take more than half of the shared memory) accumulate all their
// tiles in TMEM while the next tile is staged with cp.async (warps 0-7; warp
// 8 issues the MMAs).  While the MMAs run, warps 0-7 also sum the staged
// output gradients per channel: the bias gradient.  Each CTA writes one
// partial [cout][CIN][27] weight gradient followed by its [cout] bias
// gradient (the parameter order), summed in fixed order by k_part_sum.
constexpr int kWgZ = 2;
constexpr int kWgThreads = 288;  // warps 0-7 stage, warp 8 issues the MMAs, warps 0-2 drain
constexpr int kWgStage = 256;

template <int CIN>
struct WgLayout {
    static constexpr int PW = CIN == 32 ? 10 : 8;  // staged row width in cells
    static constexpr int S2D = 18 * PW * 16;       // bytes per (z plane, slot)
    static constexpr int ABYTES = (kWgZ + 3) * 4 * S2D;
    static constexpr int GBYTES = 4 * kWgZ * 128 * 16;
    static constexpr int BUF = ABYTES + GBYTES;
    static constexpr int NACC = CIN == 32 ? 9 : 3;
    static constexpr int COLS = CIN == 32 ? 512 : 128;  // TMEM columns (power of two >= 32 * NACC)
};

template <int CIN>
__global__ void __launch_bounds__(kWgThreads) k_wgrad_tc(const bf16 *__restrict__ gz, const bf16 *__restrict__ act,
                                                         int nx, int ny, int nz, int cout,
                                                         float *__restrict__ part, unsigned *err)
{
    using L = WgLayout<CIN>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = nx / 8, tiles_y = ny / 16, tiles_z = nz / kWgZ;
    const int ntiles = tiles_x * tiles_y * tiles_z;
    const int plane = nx * ny;
    const size_t Ncell = (size_t)plane * nz;
    const uint32_t s_base = (uint32_t)__cvta_generic_to_shared(smem);

    // slots that are never staged feed only discarded rows: clear them once
    for (int i = tid; i < 2 * L::BUF / 16; i += kWgThreads) reinterpret_cast<uint4 *>(smem)[i] = make_uint4(0, 0, 0, 0);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    if (warp == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&tmem_base);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(dst), "r"(L::COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;

    auto stage = [&](int tile, int b) {
        const int tx = tile % tiles_x, ty = (tile / tiles_x) % tiles_y, tz = tile / (tiles_x * tiles_y);
        const int x0 = tx * 8, y0 = ty * 16, z0 = tz * kWgZ;
        const uint32_t abase = s_base + (uint32_t)(b * L::BUF), gbase = abase + L::ABYTES;
        constexpr int NA = CIN == 32 ? (kWgZ + 2) * 4 * 18 * 10 : (kWgZ + 2) * 3 * 18 * 8;
        for (int idx = tid; idx < NA; idx += kWgStage) {
            int slot, bx, by, h, sx;
            if (CIN == 32) {  // slot = channel block; consecutive threads read one cell's 64 bytes
                slot = idx & 3;
                const int c = idx >> 2;
                bx = c % 10;
                by = (c / 10) % 18;
                h = c / 180;
                sx = bx;
            } else {          // slot = x shift
                bx = idx & 7;
                const int r = idx >> 3;
                by = r % 18;
                slot = (r / 18) % 3;
                h = r / 54;
                sx = bx + slot;
            }
            int gx = x0 - 1 + sx, gy = y0 - 1 + by, gzz = z0 - 1 + h;
            gx += gx < 0 ? nx : (gx >= nx ? -nx : 0);
            gy += gy < 0 ? ny : (gy >= ny ? -ny : 0);
            gzz += gzz < 0 ? nz : (gzz >= nz ? -nz : 0);
            const size_t cell = (size_t)gx + (size_t)nx * gy + (size_t)plane * gzz;
            const uint32_t dst = abase + (uint32_t)((((h * 4 + slot) * 18 + by) * L::PW + bx) * 16);
            const bf16 *src = act + ((size_t)(CIN == 32 ? slot : 0) * Ncell + cell) * 8;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
        }
        for (int idx = tid; idx < 4 * kWgZ * 128; idx += kWgStage) {
            const int cbo = idx & 3, c = idx >> 2;  // c = zz * 128 + y * 8 + x
            const size_t cell = (size_t)(x0 + (c & 7)) + (size_t)nx * (y0 + ((c >> 3) & 15)) +
                                (size_t)plane * (z0 + (c >> 7));
            const uint32_t dst = gbase + (uint32_t)((cbo * kWgZ * 128 + c) * 16);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(gz + ((size_t)cbo * Ncell + cell) * 8)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    // MN-major A and B (bits 15, 16), BF16 in, FP32 accumulate, M = 128, N = 32
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((32u >> 3) << 17) |
                           ((128u >> 4) << 24);
    uint32_t phase = 0;
    bool ok = true, first = true;
    int b = 0;
    float bsum = 0.f;  // bias gradient: channel lane, cells warp, warp + 8, ... of each tile
    if ((int)blockIdx.x < ntiles && warp < 8) stage(blockIdx.x, 0);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        if (tid == 8 * 32) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t abase = s_base + (uint32_t)(b * L::BUF), gbase = abase + L::ABYTES;
            for (int zz = 0; zz < kWgZ; ++zz)
                for (int ks = 0; ks < 8; ++ks) {  // two tile rows of 8 cells per K step
                    const uint64_t db = tc_desc(gbase + (uint32_t)(zz * 2048 + ks * 256), 128, kWgZ * 128 * 16);
                    const uint32_t acc = !(first && zz == 0 && ks == 0);
                    for (int j = 0; j < L::NACC; ++j) {
                        const int dy = CIN == 32 ? j / 3 : j, dx = CIN == 32 ? j % 3 : 0;
                        const uint32_t a_addr =
                            abase + (uint32_t)(zz * 4 * L::S2D + ((2 * ks + dy) * L::PW + dx) * 16);
                        const uint64_t da = tc_desc(a_addr, L::PW * 16, L::S2D);
                        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                                     ::"r"(tmem + (uint32_t)(32 * j)), "l"(da), "l"(db), "r"(idesc), "r"(acc));
                    }
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mb));
        }
        // stage the next tile into the other buffer while the tensor cores work
        const int next = tile + (int)gridDim.x;
        if (next < ntiles && warp < 8) stage(next, b ^ 1);
        if (warp < 8) {  // this tile's output gradients (channel lane) from the staged planes
            const unsigned char *g = smem + b * L::BUF + L::ABYTES + (lane >> 3) * (kWgZ * 128 * 16) + (lane & 7) * 2;
#pragma unroll 8
            for (int c = warp; c < kWgZ * 128; c += 8)
                bsum += __bfloat162float(*reinterpret_cast<const bf16 *>(g + c * 16));
        }
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        uint32_t done = 0;
        for (uint32_t it = 0; it < kTcWaitLimit && !done; ++it)
            asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                         "selp.u32 %0, 1, 0, p;\n\t}\n"
                         : "=r"(done)
                         : "r"(mb), "r"(phase));
        const int all_done = __syncthreads_and((int)done);
        phase ^= 1u;
        if (!all_done) {
            if (tid == 0) atomicOr(err, kFlagTimeout);
            ok = false;
        }
        first = false;
        b ^= 1;
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const size_t pstride = (size_t)cout * CIN * 27 + cout;
    {
        __shared__ float bred[8][32];
        if (warp < 8) bred[warp][lane] = bsum;
        __syncthreads();
        if (tid < cout) {
            float t = 0.f;
#pragma unroll
            for (int w = 0; w < 8; ++w) t += bred[w][tid];
            part[(size_t)blockIdx.x * pstride + (size_t)cout * CIN * 27 + tid] = t;
        }
    }
    if (ok && warp < 3) {  // warp h reads TMEM lanes of z-offset h = dz; warp 3 holds discarded rows
        float *dst = part + (size_t)blockIdx.x * pstride;
        for (int j = 0; j < L::NACC; ++j) {
            uint32_t r[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(32 * j);
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
                         "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
                           "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
                           "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
                           "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
                           "=r"(r[31])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            // row = (dz * 4 + slot) * 8 + e
            const int slot = lane >> 3;
            const int c = CIN == 32 ? lane : (lane & 7);
            const int t = CIN == 32 ? 9 * warp + j : 9 * warp + 3 * j + slot;
            if (CIN == 32 || slot < 3) {  // a CTA without tiles (never launched so) writes zeros
#pragma unroll
                for (int o = 0; o < 32; ++o)
                    if (o < cout) dst[((size_t)o * CIN + c) * 27 + t] = first ? 0.f : __uint_as_float(r[o]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(L::COLS));
    }
}

// ---------------------------------------------------------------------------
// elementwise pieces
// ---------------------------------------------------------------------------

struct Norm {
    float mu[8], inv_sigma[8];
};

__global__ void k_features(const double *__restrict__ Q, int N, const Norm n, bf16 *__restrict__ x)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    __align__(16) bf16 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __float2bfloat16_rn(((float)Q[(size_t)k * N + c] - n.mu[k]) * n.inv_sigma[k]);
    *reinterpret_cast<uint4 *>(x + (size_t)c * 8) = *reinterpret_cast<const uint4 *>(v);
}

struct LossArgs {
    float inv_sigma[8];
    float coef;  // 2 / N
};

// r = (Q1 - Qt)/sigma, loss += sum r^2 / N, gq = 2 r / (sigma N)
__global__ void __launch_bounds__(256) k_loss(const double *__restrict__ q1, const double *__restrict__ qt, int N,
                                              const LossArgs la, float *__restrict__ gq, double *__restrict__ loss)
{
    __shared__ double red[256];
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 8 * N; i += gridDim.x * blockDim.x) {
        const int k = i / N;
        const double r = (q1[i] - qt[i]) * la.inv_sigma[k];
        s += r * r;
        gq[i] = (float)(la.coef * r * la.inv_sigma[k]);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0] * 0.5 * la.coef);
}

// dL/dy[cell][3k+a] = out_scale_k * (gq_k(x + e_a) - gq_k(x - e_a)) / 2, zero for 24..31
__global__ void k_grad_out(const float *__restrict__ gq, int nx, int ny, int nz, const float *__restrict__ col_scale,
                           bf16 *__restrict__ gy)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = nx * ny * nz;
    if (c >= N) return;
    const Nbr n = nbr_cell(c, nx, ny, nz);
    const int plus[3] = {c + n.ox[2], c + n.oy[2], c + n.oz[2]};
    const int minus[3] = {c + n.ox[0], c + n.oy[0], c + n.oz[0]};
    __align__(16) bf16 v[32];
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a)
            v[3 * k + a] = __float2bfloat16_rn(col_scale[3 * k + a] * 0.5f *
                                               (gq[(size_t)k * N + plus[a]] - gq[(size_t)k * N + minus[a]]));
#pragma unroll
    for (int j = kOut; j < 32; ++j) v[j] = __float2bfloat16_rn(0.f);
#pragma unroll
    for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4 *>(gy + ((size_t)q * N + c) * 8) = reinterpret_cast<const uint4 *>(v)[q];
}

// dL/dy given as [N][24] floats -> BF16, 32 channels (zero padded), channel-blocked
__global__ void k_gy_from_f32(const float *__restrict__ src, int N, bf16 *__restrict__ gy)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    __align__(16) bf16 v[32];
    const float4 *s4 = reinterpret_cast<const float4 *>(src + (size_t)c * kOut);
#pragma unroll
    for (int q = 0; q < kOut / 4; ++q) {
        const float4 f = __ldg(s4 + q);
        v[4 * q] = __float2bfloat16_rn(f.x);
        v[4 * q + 1] = __float2bfloat16_rn(f.y);
        v[4 * q + 2] = __float2bfloat16_rn(f.z);
        v[4 * q + 3] = __float2bfloat16_rn(f.w);
    }
#pragma unroll
    for (int j = kOut; j < 32; ++j) v[j] = __float2bfloat16_rn(0.f);
#pragma unroll
    for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4 *>(gy + ((size_t)q * N + c) * 8) = reinterpret_cast<const uint4 *>(v)[q];
}

struct AdamArgs {
    float lr, b1, b2, eps, c1, c2;  // c1 = 1/(1 - b1^t), c2 = 1/(1 - b2^t)
};

__global__ void k_adam(float *__restrict__ th, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, int n, const AdamArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = a.b1 * m[i] + (1.f - a.b1) * gi;
    const float vi = a.b2 * v[i] + (1.f - a.b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    th[i] -= a.lr * (mi * a.c1) / (sqrtf(vi * a.c2) + a.eps);
}

__global__ void k_restrict(const double *__restrict__ qf, int nx, int ny, int nz, int f, double *__restrict__ qc)
{
    const int cx = nx / f, cy = ny / f, cz = nz / f;
    const int Nc = cx * cy * cz;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 8 * Nc) return;
    const int k = i / Nc, C = i % Nc;
    const int X = C % cx, Y = (C / cx) % cy, Z = C / (cx * cy);
    const int64_t Nf = (int64_t)nx * ny * nz;
    double s = 0.0;
    for (int dz = 0; dz < f; ++dz)
        for (int dy = 0; dy < f; ++dy)
            for (int dx = 0; dx < f; ++dx)
                s += qf[k * Nf + (X * f + dx) + (int64_t)nx * ((Y * f + dy) + (int64_t)ny * (Z * f + dz))];
    qc[i] = s / (double)(f * f * f);
}

}  // namespace
}  // namespace vlbm

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct vlbm_closure {
    vlbm_closure_params p{};
    int nx = 0, ny = 0, nz = 0, N = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t nparam = 0;
    size_t off_W[3]{}, off_b[3]{};
    float *theta = nullptr, *mom = nullptr, *vel = nullptr, *grad = nullptr;
    uint2 *frag_fwd[3]{}, *frag_bwd[3]{};
    vlbm::bf16 *wtc_fwd[3]{}, *wtc_bwd[3]{};  // weights in the tcgen05 layout
    unsigned *errflag = nullptr;             // bounded-wait failures of closure kernels
    unsigned *step_err = nullptr;            // where the running kernels report (errflag or a ctx flag)
    int sms = 1;                             // streaming multiprocessors of the device
    float *wpart = nullptr, *bpart = nullptr;  // per-CTA partial weight and bias gradients
    bool tc_maps = false;                    // halo tensor maps below are encoded
    CUtensorMap map_x{}, map_a1{}, map_a2{}, map_gy{}, map_gz{};  // TMA halo boxes of the conv inputs
    vlbm::bf16 *x = nullptr, *a1 = nullptr, *a2 = nullptr, *gy = nullptr, *gz = nullptr;
    float *dphi = nullptr, *gq = nullptr, *col_scale = nullptr;
    double *q = nullptr, *q1 = nullptr, *loss = nullptr;
    int64_t adam_t = 0;
    vlbm_ctx *inner = nullptr;
    std::vector<void *> owned;
};

namespace vlbm {

vlbm_status ideal_step_corrected(vlbm_ctx *c, int parity, const float *dphi);

namespace {

const int kCin[3] = {8, kH, kH};
const int kCout[3] = {kH, kH, kOut};
const int kCS[3] = {8, 32, 32};
const int kNT[3] = {4, 4, 3};

int nchunk(int cs) { return cs == 8 ? 14 : 54; }

vlbm_status cl_check(cudaError_t e, const char *what) { return cuda_check(nullptr, e, what); }

// After a synchronisation: a bounded device wait of a closure kernel gave up?
vlbm_status cl_flags(vlbm_closure *cl)
{
    unsigned h = 0;
    vlbm_status st = cl_check(cudaMemcpy(&h, cl->errflag, sizeof(unsigned), cudaMemcpyDeviceToHost),
                              "closure flag read-back");
    if (st == VLBM_OK && (h & kFlagTimeout))
        return fail(nullptr, VLBM_ERR_TIMEOUT, "a closure kernel's bounded wait for its tensor-core work expired");
    return st;
}

void *cl_alloc(vlbm_closure *cl, size_t bytes)
{
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    cl->owned.push_back(p);
    return p;
}

vlbm_status pack_all(vlbm_closure *cl, cudaStream_t s)
{
    for (int l = 0; l < 3; ++l) {
        const int ntc = tc_nchunk(kCS[l]) * kTcN * 16;
        k_pack_tc<<<(ntc + 255) / 256, 256, 0, s>>>(cl->theta + cl->off_W[l], kCout[l], kCin[l], kCS[l], 0,
                                                     cl->wtc_fwd[l]);
        if (l > 0) {
            const int nt = tc_nchunk(32) * kTcN * 16;
            k_pack_tc<<<(nt + 255) / 256, 256, 0, s>>>(cl->theta + cl->off_W[l], kCout[l], kCin[l], 32, 1,
                                                        cl->wtc_bwd[l]);
        }
        const int total = nchunk(kCS[l]) * kNT[l] * 32;
        k_pack<<<(total + 255) / 256, 256, 0, s>>>(cl->theta + cl->off_W[l], kCout[l], kCin[l], kCS[l], kNT[l], 0,
                                                    cl->frag_fwd[l]);
        if (l > 0) {  // transposed packs: input channels = forward outputs (stride 32), outputs = forward inputs
            const int tt = nchunk(32) * 4 * 32;
            k_pack<<<(tt + 255) / 256, 256, 0, s>>>(cl->theta + cl->off_W[l], kCout[l], kCin[l], 32, 4, 1,
                                                     cl->frag_bwd[l]);
        }
    }
    return cl_check(cudaGetLastError(), "closure weight packing");
}

// cuTensorMapEncodeTiled from the driver (no link against libcuda)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled_fn()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Halo box of k_conv_tc over a channel-blocked BF16 field with cs channels:
// dimensions (8 nx, ny, nz, cs/8 planes) with the 8 channels of a cell
// innermost, box (8 * 10, 18, kTcZ + 2, 1), so that one copy fills one
// channel-block plane with rows of 160 contiguous bytes.
vlbm_status encode_halo_map(CUtensorMap *m, const bf16 *base, int cs, int nx, int ny, int nz)
{
    EncodeTiledFn fn = encode_tiled_fn();
    if (!fn) return fail(nullptr, VLBM_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint64_t dims[4] = {(cuuint64_t)8 * nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)(cs / 8)};
    const cuuint64_t strides[3] = {(cuuint64_t)nx * 16, (cuuint64_t)nx * ny * 16, (cuuint64_t)nx * ny * nz * 16};
    const cuuint32_t box[4] = {8 * kTcHx, kTcHy, kTcHz, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16 *>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(nullptr, VLBM_ERR_CUDA, "halo tensor map encoding failed");
    return VLBM_OK;
}

// grids the tcgen05 kernels tile exactly
bool conv_tc_ok(const vlbm_closure *cl) { return cl->nx % kTcX == 0 && cl->ny % kTcY == 0 && cl->nz % kTcZ == 0; }
bool wgrad_tc_ok(const vlbm_closure *cl) { return cl->nx % 8 == 0 && cl->ny % 16 == 0 && cl->nz % kWgZ == 0; }

vlbm_status conv(vlbm_closure *cl, int layer, const bf16 *in, bool transpose, const ConvEpilogue &e, cudaStream_t s)
{
    if (conv_tc_ok(cl)) {
        // tcgen05 / TMEM tiles of 8 x 16 x 4 cells
        // persistent CTAs, one per SM (13 warps of up to 152 registers)
        const int ntiles = (cl->nx / kTcX) * (cl->ny / kTcY) * (cl->nz / kTcZ);
        const unsigned grid = (unsigned)std::min(ntiles, cl->sms);
        const int cout_real = transpose ? kCin[layer] : kCout[layer];
        const bf16 *w = transpose ? cl->wtc_bwd[layer] : cl->wtc_fwd[layer];
        const CUtensorMap *map = in == cl->x ? &cl->map_x
                                 : in == cl->a1 ? &cl->map_a1
                                 : in == cl->a2 ? &cl->map_a2
                                 : in == cl->gy ? &cl->map_gy
                                 : in == cl->gz ? &cl->map_gz
                                                : nullptr;
        if (!map || !cl->tc_maps) return fail(nullptr, VLBM_ERR_STATE, "closure convolution input has no halo map");
        if (!transpose && layer == 0)
            k_conv_tc<8><<<grid, kTcThreads, tc_smem_bytes<8>(), s>>>(in, cl->nx, cl->ny, cl->nz, w, cout_real, e,
                                                                     cl->step_err, *map);
        else
            k_conv_tc<32><<<grid, kTcThreads, tc_smem_bytes<32>(), s>>>(in, cl->nx, cl->ny, cl->nz, w, cout_real, e,
                                                                       cl->step_err, *map);
        return cl_check(cudaGetLastError(), "closure tcgen05 convolution launch");
    }
    if (cl->nx % kTx == 0 && cl->ny % kTy == 0) {
        // shared-memory staged tiles (16 x 8 cells per CTA)
        const dim3 grid((unsigned)(cl->nx / kTx), (unsigned)(cl->ny / kTy), (unsigned)cl->nz);
        const int threads = kTx * kTy * 2;
        if (!transpose) {
            if (layer == 0)
                k_conv_smem<8, 4><<<grid, threads, 0, s>>>(in, cl->nx, cl->ny, cl->nz, cl->frag_fwd[0], e);
            else if (layer == 1)
                k_conv_smem<32, 4><<<grid, threads, 0, s>>>(in, cl->nx, cl->ny, cl->nz, cl->frag_fwd[1], e);
            else
                k_conv_smem<32, 3><<<grid, threads, 0, s>>>(in, cl->nx, cl->ny, cl->nz, cl->frag_fwd[2], e);
        } else {
            k_conv_smem<32, 4><<<grid, threads, 0, s>>>(in, cl->nx, cl->ny, cl->nz, cl->frag_bwd[layer], e);
        }
        return cl_check(cudaGetLastError(), "closure convolution launch");
    }
    const int cells_per_cta = (kConvThreads / 32) * 16;
    const unsigned grid = (unsigned)((cl->N + cells_per_cta - 1) / cells_per_cta);
    if (!transpose) {
        if (layer == 0)
            k_conv<8, 4><<<grid, kConvThreads, 0, s>>>(in, cl->nx, cl->ny, cl->nz, cl->frag_fwd[0], e);
        else if (layer == 1)
            k_conv<32, 4><<<grid, kConvThreads, 0, s>>>(in, cl->nx, cl->ny, cl->nz, cl->frag_fwd[1], e);
        else
            k_conv<32, 3><<<grid, kConvThreads, 0, s>>>(in, cl->nx, cl->ny, cl->nz, cl->frag_fwd[2], e);
    } else {
        k_conv<32, 4><<<grid, kConvThreads, 0, s>>>(in, cl->nx, cl->ny, cl->nz, cl->frag_bwd[layer], e);
    }
    return cl_check(cudaGetLastError(), "closure convolution launch");
}

ConvEpilogue epi() { ConvEpilogue e{}; return e; }

// network forward from device fields Q (8 x N doubles) to dphi (N x 24 floats)
Norm feature_norm(const vlbm_closure *cl)
{
    Norm n{};
    for (int k = 0; k < 8; ++k) {
        n.mu[k] = (float)cl->p.mu[k];
        n.inv_sigma[k] = (float)(1.0 / cl->p.sigma[k]);
    }
    return n;
}

// the three convolutions from the features in cl->x to dphi
vlbm_status forward_convs(vlbm_closure *cl, float *dphi, cudaStream_t s)
{
    vlbm_status st = VLBM_OK;
    ConvEpilogue e = epi();
    e.bias = cl->theta + cl->off_b[0];
    e.tanh_act = 1;
    e.out_bf = cl->a1;
    e.os = 32;
    if (st == VLBM_OK) st = conv(cl, 0, cl->x, false, e, s);
    e.bias = cl->theta + cl->off_b[1];
    e.out_bf = cl->a2;
    if (st == VLBM_OK) st = conv(cl, 1, cl->a1, false, e, s);
    e = epi();
    e.bias = cl->theta + cl->off_b[2];
    e.scale = cl->col_scale;
    e.out_f = dphi;
    e.os = kOut;
    if (st == VLBM_OK) st = conv(cl, 2, cl->a2, false, e, s);
    return st;
}

vlbm_status forward(vlbm_closure *cl, const double *Q, float *dphi, cudaStream_t s)
{
    k_features<<<(cl->N + 255) / 256, 256, 0, s>>>(Q, cl->N, feature_norm(cl), cl->x);
    vlbm_status st = cl_check(cudaGetLastError(), "closure features launch");
    if (st == VLBM_OK) st = forward_convs(cl, dphi, s);
    return st;
}

// forward pass on the current state of a context: features straight from its populations
vlbm_status forward_ctx(vlbm_closure *cl, vlbm_ctx *c, float *dphi)
{
    const Norm n = feature_norm(cl);
    vlbm_status st = ideal_features(c, n.mu, n.inv_sigma, cl->x);
    if (st == VLBM_OK) st = forward_convs(cl, dphi, c->stream);
    return st;
}

// gradients of sum(gy * y) into cl->grad, given gy (BF16 [N][32]) and the
// activations of the last forward pass
vlbm_status backward(vlbm_closure *cl, cudaStream_t s)
{
    vlbm_status st = cl_check(cudaMemsetAsync(cl->grad, 0, cl->nparam * sizeof(float), s), "closure grad clear");
    const unsigned wgx = (unsigned)((cl->N + kWgradCells - 1) / kWgradCells);
    const bool tc = wgrad_tc_ok(cl);
    const int ntiles = (cl->nx / 8) * (cl->ny / 16) * (cl->nz / kWgZ);
    const unsigned wg_grid = (unsigned)std::min(ntiles, cl->sms), b_grid = (unsigned)(2 * cl->sms);
    auto wgrad = [&](int l, const bf16 *g, const bf16 *a) {
        float *gW = cl->grad + cl->off_W[l];
        if (tc) {  // tensor cores; per-CTA partials (weights, then bias) summed in a fixed order
            const int count = kCout[l] * kCin[l] * 27 + kCout[l];
            if (kCS[l] == 8)
                k_wgrad_tc<8><<<wg_grid, kWgThreads, 2 * WgLayout<8>::BUF, s>>>(g, a, cl->nx, cl->ny, cl->nz,
                                                                                kCout[l], cl->wpart, cl->step_err);
            else
                k_wgrad_tc<32><<<wg_grid, kWgThreads, 2 * WgLayout<32>::BUF, s>>>(g, a, cl->nx, cl->ny, cl->nz,
                                                                                  kCout[l], cl->wpart, cl->step_err);
            k_part_sum<<<(count + 31) / 32, 256, 0, s>>>(cl->wpart, (int)wg_grid, count, gW);  // b follows W
        } else {
            if (kCS[l] == 8)
                k_wgrad<8><<<dim3(wgx, 27), kConvThreads, 0, s>>>(g, a, cl->nx, cl->ny, cl->nz, kCout[l], kCin[l], gW);
            else
                k_wgrad<32><<<dim3(wgx, 27), kConvThreads, 0, s>>>(g, a, cl->nx, cl->ny, cl->nz, kCout[l], kCin[l], gW);
            k_bgrad_part<<<b_grid, 256, 0, s>>>(g, cl->N, kCout[l], cl->bpart);
            k_part_sum<<<1, 256, 0, s>>>(cl->bpart, (int)b_grid, kCout[l], cl->grad + cl->off_b[l]);
        }
        return cl_check(cudaGetLastError(), "closure weight gradient launch");
    };
    // layer 3: gy -> W3, b3; data gradient through tanh of layer 2 -> gz
    if (st == VLBM_OK) st = wgrad(2, cl->gy, cl->a2);
    ConvEpilogue e = epi();
    e.deriv = cl->a2;
    e.out_bf = cl->gz;
    e.os = 32;
    if (st == VLBM_OK) st = conv(cl, 2, cl->gy, true, e, s);
    // layer 2: gz -> W2, b2; data gradient through tanh of layer 1 -> gy (reused)
    if (st == VLBM_OK) st = wgrad(1, cl->gz, cl->a1);
    e.deriv = cl->a1;
    e.out_bf = cl->gy;
    if (st == VLBM_OK) st = conv(cl, 1, cl->gz, true, e, s);
    // layer 1
    if (st == VLBM_OK) st = wgrad(0, cl->gy, cl->x);
    return st;
}

}  // namespace
}  // namespace vlbm

using namespace vlbm;

extern "C" {

vlbm_status vlbm_closure_create(const vlbm_closure_params *p, vlbm_closure **out)
{
    if (!p || !out) return VLBM_ERR_ARG;
    *out = nullptr;
    if (p->nx < 16 || p->ny < 1 || p->nz < 1 || p->nx % 16 != 0)
        return fail(nullptr, VLBM_ERR_ARG, "closure grid: nx must be a multiple of 16");
    if ((int64_t)p->nx * p->ny * p->nz > (int64_t(1) << 25))
        return fail(nullptr, VLBM_ERR_ARG, "closure grid too large (at most 2^25 cells)");
    for (int k = 0; k < 8; ++k)
        if (!(p->sigma[k] > 0.0)) return fail(nullptr, VLBM_ERR_ARG, "closure sigma must be > 0");
    if (!(p->tau > 0.5) || !(p->gamma > 1.0)) return fail(nullptr, VLBM_ERR_ARG, "closure tau/gamma");
    vlbm_closure *cl = new vlbm_closure();
    cl->p = *p;
    cl->nx = p->nx;
    cl->ny = p->ny;
    cl->nz = p->nz;
    cl->N = p->nx * p->ny * p->nz;
    size_t off = 0;
    for (int l = 0; l < 3; ++l) {
        cl->off_W[l] = off;
        off += (size_t)kCout[l] * kCin[l] * 27;
        cl->off_b[l] = off;
        off += kCout[l];
    }
    cl->nparam = off;
    vlbm_status st = VLBM_OK;
    if (p->stream) {
        cl->stream = static_cast<cudaStream_t>(p->stream);
    } else {
        st = cl_check(cudaStreamCreateWithFlags(&cl->stream, cudaStreamNonBlocking), "closure stream");
        cl->own_stream = st == VLBM_OK;
    }
    const size_t N = cl->N;
    bool ok = st == VLBM_OK;
    auto A = [&](size_t bytes) -> void * {
        void *q = ok ? cl_alloc(cl, bytes) : nullptr;
        ok = ok && q;
        return q;
    };
    cl->theta = (float *)A(cl->nparam * 4);
    cl->mom = (float *)A(cl->nparam * 4);
    cl->vel = (float *)A(cl->nparam * 4);
    cl->grad = (float *)A(cl->nparam * 4);
    for (int l = 0; l < 3; ++l) {
        cl->frag_fwd[l] = (uint2 *)A((size_t)nchunk(kCS[l]) * kNT[l] * 32 * sizeof(uint2));
        cl->frag_bwd[l] = (uint2 *)A((size_t)nchunk(32) * 4 * 32 * sizeof(uint2));
        cl->wtc_fwd[l] = (bf16 *)A((size_t)tc_nchunk(kCS[l]) * kTcN * 16 * sizeof(bf16));
        cl->wtc_bwd[l] = (bf16 *)A((size_t)tc_nchunk(32) * kTcN * 16 * sizeof(bf16));
    }
    cl->errflag = (unsigned *)A(64);
    cl->step_err = cl->errflag;
    cl->x = (bf16 *)A(N * 8 * 2);
    cl->a1 = (bf16 *)A(N * 32 * 2);
    cl->a2 = (bf16 *)A(N * 32 * 2);
    cl->gy = (bf16 *)A(N * 32 * 2);
    cl->gz = (bf16 *)A(N * 32 * 2);
    cl->dphi = (float *)A(N * kOut * 4);
    cl->gq = (float *)A(N * 8 * 4);
    cl->q = (double *)A(N * 8 * 8);
    cl->q1 = (double *)A(N * 8 * 8);
    cl->loss = (double *)A(64);
    cl->col_scale = (float *)A(32 * 4);
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&cl->sms, cudaDevAttrMultiProcessorCount, dev);
        cl->sms = std::max(cl->sms, 1);
    }
    cl->wpart = (float *)A((size_t)cl->sms * (32 * 32 * 27 + 32) * 4);
    cl->bpart = (float *)A((size_t)2 * cl->sms * 32 * 4);
    if (!ok) {
        vlbm_closure_destroy(cl);
        return st != VLBM_OK ? st : fail(nullptr, VLBM_ERR_OOM, "closure allocation failed");
    }
    if (ok) {
        const int shm32 = tc_smem_bytes<32>(), shm8 = tc_smem_bytes<8>();
        st = cl_check(cudaFuncSetAttribute(k_conv_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, shm32),
                      "closure tcgen05 shared memory");
        if (st == VLBM_OK)
            st = cl_check(cudaFuncSetAttribute(k_conv_tc<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, shm8),
                          "closure tcgen05 shared memory");
        if (st == VLBM_OK)
            st = cl_check(cudaFuncSetAttribute(k_wgrad_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               2 * WgLayout<32>::BUF),
                          "closure tcgen05 shared memory");
        if (st == VLBM_OK)
            st = cl_check(cudaFuncSetAttribute(k_wgrad_tc<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               2 * WgLayout<8>::BUF),
                          "closure tcgen05 shared memory");
        if (st == VLBM_OK && conv_tc_ok(cl)) {
            st = encode_halo_map(&cl->map_x, cl->x, 8, cl->nx, cl->ny, cl->nz);
            if (st == VLBM_OK) st = encode_halo_map(&cl->map_a1, cl->a1, 32, cl->nx, cl->ny, cl->nz);
            if (st == VLBM_OK) st = encode_halo_map(&cl->map_a2, cl->a2, 32, cl->nx, cl->ny, cl->nz);
            if (st == VLBM_OK) st = encode_halo_map(&cl->map_gy, cl->gy, 32, cl->nx, cl->ny, cl->nz);
            if (st == VLBM_OK) st = encode_halo_map(&cl->map_gz, cl->gz, 32, cl->nx, cl->ny, cl->nz);
            cl->tc_maps = st == VLBM_OK;
        }
        if (st == VLBM_OK) st = cl_check(cudaMemsetAsync(cl->errflag, 0, 64, cl->stream), "closure flag clear");
        ok = st == VLBM_OK;
    }
    float cs[32] = {};
    for (int j = 0; j < kOut; ++j) cs[j] = (float)p->out_scale[j / 3];
    st = cl_check(cudaMemcpyAsync(cl->col_scale, cs, sizeof(cs), cudaMemcpyHostToDevice, cl->stream), "closure scale");
    for (float *b : {cl->theta, cl->mom, cl->vel, cl->grad})
        if (st == VLBM_OK) st = cl_check(cudaMemsetAsync(b, 0, cl->nparam * 4, cl->stream), "closure clear");
    if (st == VLBM_OK) st = pack_all(cl, cl->stream);
    if (st == VLBM_OK) {
        vlbm_params ip;
        vlbm_default_params(&ip);
        ip.dim = 3;
        ip.nx = p->nx;
        ip.ny = p->ny;
        ip.nz = p->nz;
        ip.storage = VLBM_F32;
        ip.gamma = p->gamma;
        for (int k = 0; k < 8; ++k) ip.tau[k] = p->tau;
        ip.stream = cl->stream;
        st = vlbm_create(&ip, &cl->inner);
    }
    if (st == VLBM_OK) st = cl_check(cudaStreamSynchronize(cl->stream), "closure create");
    if (st != VLBM_OK) {
        vlbm_closure_destroy(cl);
        return st;
    }
    *out = cl;
    return VLBM_OK;
}

size_t vlbm_closure_num_params(const vlbm_closure *cl) { return cl ? cl->nparam : 0; }

vlbm_status vlbm_closure_set_weights(vlbm_closure *cl, const float *host, size_t count)
{
    if (!cl || !host || count != cl->nparam) return VLBM_ERR_ARG;
    vlbm_status st = cl_check(cudaMemcpyAsync(cl->theta, host, count * 4, cudaMemcpyHostToDevice, cl->stream),
                              "closure weights upload");
    if (st == VLBM_OK) st = pack_all(cl, cl->stream);
    if (st == VLBM_OK) st = cl_check(cudaStreamSynchronize(cl->stream), "closure weights");
    return st;
}

vlbm_status vlbm_closure_get_weights(vlbm_closure *cl, float *host, size_t count)
{
    if (!cl || !host || count != cl->nparam) return VLBM_ERR_ARG;
    vlbm_status st = cl_check(cudaMemcpyAsync(host, cl->theta, count * 4, cudaMemcpyDeviceToHost, cl->stream),
                              "closure weights download");
    if (st == VLBM_OK) st = cl_check(cudaStreamSynchronize(cl->stream), "closure weights");
    return st;
}

vlbm_status vlbm_closure_forward(vlbm_closure *cl, const double *Q_dev, float *dphi_dev)
{
    vlbm::NvtxRange range("vlbm_closure_forward");
    if (!cl || !Q_dev || !dphi_dev) return VLBM_ERR_ARG;
    vlbm_status st = forward(cl, Q_dev, dphi_dev, cl->stream);
    if (st == VLBM_OK) st = cl_check(cudaStreamSynchronize(cl->stream), "closure forward");
    if (st == VLBM_OK) st = cl_flags(cl);
    return st;
}

vlbm_status vlbm_closure_backward(vlbm_closure *cl, const double *Q_dev, const float *gy_dev, float *grads_host)
{
    vlbm::NvtxRange range("vlbm_closure_backward");
    if (!cl || !Q_dev || !gy_dev || !grads_host) return VLBM_ERR_ARG;
    vlbm_status st = forward(cl, Q_dev, cl->dphi, cl->stream);
    if (st == VLBM_OK) {
        k_gy_from_f32<<<(cl->N + 255) / 256, 256, 0, cl->stream>>>(gy_dev, cl->N, cl->gy);
        st = cl_check(cudaGetLastError(), "closure gradient input");
    }
    if (st == VLBM_OK) st = backward(cl, cl->stream);
    if (st == VLBM_OK)
        st = cl_check(cudaMemcpyAsync(grads_host, cl->grad, cl->nparam * 4, cudaMemcpyDeviceToHost, cl->stream),
                      "closure gradient download");
    if (st == VLBM_OK) st = cl_check(cudaStreamSynchronize(cl->stream), "closure backward");
    if (st == VLBM_OK) st = cl_flags(cl);
    return st;
}

}  // extern "C"

namespace vlbm {
namespace {

// From Q1 (moments after a corrected step) and the target: loss and the
// gradient through the step (Q1 = Q_plain - delta . dPhi) and the network,
// left in cl->grad.
vlbm_status loss_backward(vlbm_closure *cl, const double *Qt_dev, cudaStream_t s)
{
    vlbm_status st = cl_check(cudaMemsetAsync(cl->loss, 0, sizeof(double), s), "closure loss clear");
    if (st == VLBM_OK) {
        LossArgs la{};
        for (int k = 0; k < 8; ++k) la.inv_sigma[k] = (float)(1.0 / cl->p.sigma[k]);
        la.coef = 2.0f / (float)cl->N;
        k_loss<<<1216, 256, 0, s>>>(cl->q1, Qt_dev, cl->N, la, cl->gq, cl->loss);
        k_grad_out<<<(cl->N + 255) / 256, 256, 0, s>>>(cl->gq, cl->nx, cl->ny, cl->nz, cl->col_scale, cl->gy);
        st = cl_check(cudaGetLastError(), "closure loss launch");
    }
    if (st == VLBM_OK) st = backward(cl, s);
    return st;
}

// The loss of the last loss_backward to the host, after the stream has finished.
vlbm_status loss_to_host(vlbm_closure *cl, double *loss, cudaStream_t s)
{
    double h = 0.0;
    vlbm_status st = cl_check(cudaMemcpyAsync(&h, cl->loss, sizeof(double), cudaMemcpyDeviceToHost, s), "loss");
    if (st == VLBM_OK) st = cl_check(cudaStreamSynchronize(s), "closure train step");
    if (st == VLBM_OK) st = cl_flags(cl);
    if (loss) *loss = h;
    return st;
}

// One Adam step from the gradient in cl->grad, and the re-packing of the weights.
vlbm_status adam_update(vlbm_closure *cl, cudaStream_t s)
{
    vlbm_status st = VLBM_OK;
    {
        cl->adam_t += 1;
        AdamArgs a{};
        a.lr = (float)cl->p.lr;
        a.b1 = (float)cl->p.beta1;
        a.b2 = (float)cl->p.beta2;
        a.eps = (float)cl->p.eps;
        a.c1 = (float)(1.0 / (1.0 - std::pow(cl->p.beta1, (double)cl->adam_t)));
        a.c2 = (float)(1.0 / (1.0 - std::pow(cl->p.beta2, (double)cl->adam_t)));
        const int n = (int)cl->nparam;
        k_adam<<<(n + 255) / 256, 256, 0, s>>>(cl->theta, cl->mom, cl->vel, cl->grad, n, a);
        st = cl_check(cudaGetLastError(), "closure adam launch");
    }
    if (st == VLBM_OK) st = pack_all(cl, s);
    return st;
}

// Loss, gradient, Adam step and re-packing (one training step).
vlbm_status loss_backward_update(vlbm_closure *cl, const double *Qt_dev, double *loss, cudaStream_t s)
{
    vlbm_status st = loss_backward(cl, Qt_dev, s);
    if (st == VLBM_OK) st = adam_update(cl, s);
    if (st == VLBM_OK) st = loss_to_host(cl, loss, s);
    return st;
}

// The forward half of a training step along a coarse run: the network on the
// context's state, one corrected step, the new moments into cl->q1.
vlbm_status advance_ctx(vlbm_closure *cl, vlbm_ctx *ctx)
{
    if (ctx->batched || ctx->model != VLBM_IDEAL || ctx->dim != 3 || ctx->storage != VLBM_F32 ||
        ctx->dom[0].nx != cl->nx || ctx->dom[0].ny != cl->ny || ctx->dom[0].nz != cl->nz)
        return fail(ctx, VLBM_ERR_ARG, "closure training context must be a 3-D F32 ideal context on the closure grid");
    vlbm_status st = forward_ctx(cl, ctx, cl->dphi);
    if (st == VLBM_OK) st = ideal_step_corrected(ctx, (int)(ctx->step & 1), cl->dphi);
    if (st == VLBM_OK) {
        ctx->step += 1;
        st = ideal_moments(ctx, 0, cl->q1);
    }
    return st;
}

}  // namespace
}  // namespace vlbm

extern "C" {

vlbm_status vlbm_closure_train_step(vlbm_closure *cl, const double *Q0_dev, const double *Qt_dev, double *loss)
{
    vlbm::NvtxRange range("vlbm_closure_train_step");
    if (!cl || !Q0_dev || !Qt_dev) return VLBM_ERR_ARG;
    cudaStream_t s = cl->stream;
    vlbm_ctx *in = cl->inner;
    // forward: network on Q0, then one corrected step from f_eq(Q0)
    vlbm_status st = forward(cl, Q0_dev, cl->dphi, s);
    in->step = 0;
    if (st == VLBM_OK) st = ideal_init_range(in, 0, Q0_dev, 0, cl->N, cl->N);
    if (st == VLBM_OK) st = ideal_step_corrected(in, 0, cl->dphi);
    if (st == VLBM_OK) {
        in->step = 1;
        st = ideal_moments(in, 0, cl->q1);
    }
    if (st != VLBM_OK) return st;
    return loss_backward_update(cl, Qt_dev, loss, s);
}

vlbm_status vlbm_closure_train_step_ctx(vlbm_closure *cl, vlbm_ctx *ctx, const double *Qt_dev, double *loss)
{
    vlbm::NvtxRange range("vlbm_closure_train_step_ctx");
    if (!cl || !ctx || !Qt_dev) return VLBM_ERR_ARG;
    vlbm_status st = advance_ctx(cl, ctx);
    if (st != VLBM_OK) return st;
    return loss_backward_update(cl, Qt_dev, loss, ctx->stream);
}

vlbm_status vlbm_closure_grad_step_ctx(vlbm_closure *cl, vlbm_ctx *ctx, const double *Qt_dev, double *loss,
                                       float *grads_dev)
{
    vlbm::NvtxRange range("vlbm_closure_grad_step_ctx");
    if (!cl || !ctx || !Qt_dev || !grads_dev) return VLBM_ERR_ARG;
    cudaStream_t s = ctx->stream;
    vlbm_status st = advance_ctx(cl, ctx);
    if (st == VLBM_OK) st = loss_backward(cl, Qt_dev, s);
    if (st == VLBM_OK)
        st = cl_check(cudaMemcpyAsync(grads_dev, cl->grad, cl->nparam * 4, cudaMemcpyDeviceToDevice, s),
                      "closure gradient copy");
    if (st == VLBM_OK) st = loss_to_host(cl, loss, s);
    return st;
}

vlbm_status vlbm_closure_apply_grads(vlbm_closure *cl, const float *grads_dev)
{
    vlbm::NvtxRange range("vlbm_closure_apply_grads");
    if (!cl || !grads_dev) return VLBM_ERR_ARG;
    cudaStream_t s = cl->stream;
    vlbm_status st = cl_check(cudaMemcpyAsync(cl->grad, grads_dev, cl->nparam * 4, cudaMemcpyDeviceToDevice, s),
                              "closure gradient copy");
    if (st == VLBM_OK) st = adam_update(cl, s);
    if (st == VLBM_OK) st = cl_check(cudaStreamSynchronize(s), "closure update");
    if (st == VLBM_OK) st = cl_flags(cl);
    return st;
}

vlbm_status vlbm_restrict(const double *Qf_dev, int nx, int ny, int nz, int factor, double *Qc_dev, void *stream)
{
    if (!Qf_dev || !Qc_dev || factor < 1 || nx % factor || ny % factor || nz % factor || nx < 1 || ny < 1 || nz < 1)
        return fail(nullptr, VLBM_ERR_ARG, "restrict: sizes must be divisible by the factor");
    const int64_t Nc = (int64_t)(nx / factor) * (ny / factor) * (nz / factor);
    if (8 * Nc >= (int64_t(1) << 31)) return fail(nullptr, VLBM_ERR_ARG, "restrict: coarse grid too large");
    k_restrict<<<(unsigned)((8 * Nc + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(Qf_dev, nx, ny, nz,
                                                                                               factor, Qc_dev);
    return cl_check(cudaGetLastError(), "restrict launch");
}

void vlbm_closure_destroy(vlbm_closure *cl)
{
    if (!cl) return;
    if (cl->stream) cudaStreamSynchronize(cl->stream);
    if (cl->inner) vlbm_destroy(cl->inner);
    for (void *q : cl->owned) cudaFree(q);
    if (cl->own_stream && cl->stream) cudaStreamDestroy(cl->stream);
    cudaGetLastError();
    delete cl;
}

}  // extern "C"

namespace vlbm {

// Used by the step loop of a context with an attached closure: the network
// runs on the context's current moments, then the corrected step kernel.
vlbm_status closure_step(vlbm_ctx *c, int parity)
{
    vlbm_closure *cl = c->closure;
    cl->step_err = c->d_flags;  // timeouts surface through the context's health word
    vlbm_status st = forward_ctx(cl, c, cl->dphi);
    cl->step_err = cl->errflag;
    c->launches += 3;  // three convolutions (features and the step count themselves)
    if (st == VLBM_OK) st = ideal_step_corrected(c, parity, cl->dphi);
    return st;
}

int closure_cells(const vlbm_closure *cl, int *nx, int *ny, int *nz)
{
    *nx = cl->nx;
    *ny = cl->ny;
    *nz = cl->nz;
    return cl->N;
}

}  // namespace vlbm
