// k_noalloc.cu -- domain sums of the ideal-MHD fields without any allocation.
//
// For callers that may not allocate device memory themselves (see
// vlbm_conservation_noalloc in include/vlbm.h).  The per-CTA partial sums
// live in a file-scope device array of fixed size instead of memory the
// library or the caller allocates.  The kernels are a variant of the context
// reduction in k_ideal.cu: one CTA per fixed block of cells (so the number of
// partials, and with it the scratch, is bounded by the cell count), then one
// CTA adds the partials in index order.
#include <mutex>

#include "vlbm_internal.cuh"

namespace vlbm {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaCellsPerThread = 256;
constexpr int64_t kNaCellsPerBlock = (int64_t)kNaThreads * kNaCellsPerThread;  // 65,536
constexpr int kNaMaxBlocks = 4096;
constexpr int64_t kNaMaxCells = kNaCellsPerBlock * kNaMaxBlocks;  // 268,435,456 = 2^28
constexpr int kNaMaxDevices = 64;

// 4096 CTAs x 8 fields x 8 bytes = 256 KiB on every device that loads the library.
static __device__ __align__(256) double g_na_partials[kNaMaxBlocks * 8];

std::mutex g_na_mutex;
void *g_na_scratch[kNaMaxDevices] = {};

template <class S> struct NaArgs {
    const S *pop;
    int nx, ny, nz;
    int64_t ncell, stride;
    int parity;
    double ref[8], scale[8];
};

// Linear indices of the upstream cells x - c_i (periodic) that the odd parity
// reads, i in set order; computed once per cell and shared by the eight fields.
template <int D>
__device__ __forceinline__ void na_upstream(int64_t cell, int x, int y, int z, int nx, int ny, int nz,
                                            int64_t *up)
{
    const int64_t row = nx, plane = (int64_t)nx * ny;
    up[0] = cell;
    up[1] = x > 0 ? cell - 1 : cell - 1 + nx;             // x - e_x
    up[2] = x + 1 < nx ? cell + 1 : cell + 1 - nx;        // x + e_x
    up[3] = y > 0 ? cell - row : cell - row + plane;      // x - e_y
    up[4] = y + 1 < ny ? cell + row : cell + row - plane;  // x + e_y
    if (D == 3) {
        const int64_t vol = plane * nz;
        up[5] = z > 0 ? cell - plane : cell - plane + vol;
        up[6] = z + 1 < nz ? cell + plane : cell + plane - vol;
    }
}

// Q_k of one cell, with the arithmetic of vlbm_conservation: the populations
// summed in the compute precision of the storage (FP64 only for FP64
// storage); deviation storage widens that sum once and decodes it in FP64,
// r_k + s_k sum_i g_ki.  At odd parity direction i is in slot opp(i) of the
// upstream cell up[i].
template <int D, class S>
__device__ __forceinline__ double na_moment(const NaArgs<S> &a, int64_t cell, const int64_t *up, int k)
{
    using R = typename ComputeOf<S>::T;
    constexpr int Q = AxisSet<D>::Q;
    R s = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int j = a.parity ? opp_axis(i) : i;
        const int64_t at = a.parity ? up[i] : cell;
        s += (R)Codec<S>::load(a.pop + (int64_t)(k * Q + j) * a.stride + at);
    }
    if (Codec<S>::kDev) return fma((double)s, a.scale[k], a.ref[k]);
    return (double)s;
}

template <int D, class S>
__global__ void __launch_bounds__(kNaThreads) k_na_partials(const NaArgs<S> a, double *__restrict__ partials)
{
    constexpr int Q = AxisSet<D>::Q;
    double acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = 0.0;
    const int64_t first = blockIdx.x * kNaCellsPerBlock;
    for (int r = 0; r < kNaCellsPerThread; ++r) {
        const int64_t cell = first + (int64_t)r * kNaThreads + threadIdx.x;
        if (cell >= a.ncell) break;
        const int x = (int)(cell % a.nx);
        const int64_t rest = cell / a.nx;
        const int y = (int)(rest % a.ny);
        const int z = (int)(rest / a.ny);
        int64_t up[Q];
        na_upstream<D>(cell, x, y, z, a.nx, a.ny, a.nz, up);
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] += (double)na_moment<D, S>(a, cell, up, k);
    }
    __shared__ double red[kNaThreads / 32][8];
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
        for (int w = 0; w < kNaThreads / 32; ++w) v += red[w][threadIdx.x];
        partials[(int64_t)blockIdx.x * 8 + threadIdx.x] = v;
    }
}

__global__ void __launch_bounds__(256) k_na_finish(const double *__restrict__ partials, int nblocks,
                                                   double *__restrict__ sums)
{
    __shared__ double red[256];
    for (int k = 0; k < 8; ++k) {
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

// Device address of the scratch array on the current device, looked up once
// per device with that device current (the host-side symbol is only a stand-in).
// The address belongs to the device's primary context: after cudaDeviceReset
// the module is loaded again and this cached address is stale.
vlbm_status na_scratch(double **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_check(nullptr, e, "no-allocation sums: cudaGetDevice");
    if (dev < 0 || dev >= kNaMaxDevices) return fail(nullptr, VLBM_ERR_ARG, "no-allocation sums: device index out of range");
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_scratch[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_partials);
        if (e != cudaSuccess || !p)
            return cuda_check(nullptr, e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                              "no-allocation sums: cudaGetSymbolAddress of the scratch array");
        g_na_scratch[dev] = p;
    }
    *out = static_cast<double *>(g_na_scratch[dev]);
    return VLBM_OK;
}

template <int D, class S>
vlbm_status na_run(const void *pop, int nx, int ny, int nz, int64_t stride, int parity, const double *q_ref,
                   const double *q_scale, double *sums, cudaStream_t stream, double *scratch)
{
    NaArgs<S> a{};
    a.pop = static_cast<const S *>(pop);
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.ncell = (int64_t)nx * ny * nz;
    a.stride = stride;
    a.parity = parity;
    for (int k = 0; k < 8; ++k) {
        a.ref[k] = q_ref ? q_ref[k] : 0.0;
        a.scale[k] = (q_scale && q_scale[k] > 0.0) ? q_scale[k] : 1.0;
    }
    const int nblocks = (int)((a.ncell + kNaCellsPerBlock - 1) / kNaCellsPerBlock);
    k_na_partials<D, S><<<nblocks, kNaThreads, 0, stream>>>(a, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(nullptr, e, "no-allocation sums: partials launch");
    k_na_finish<<<1, 256, 0, stream>>>(scratch, nblocks, sums);
    return cuda_check(nullptr, cudaGetLastError(), "no-allocation sums: finish launch");
}

}  // namespace
}  // namespace vlbm

extern "C" vlbm_status vlbm_conservation_noalloc(const void *pop_dev, int storage, int dim, int nx, int ny,
                                                 int nz, int64_t stride, int parity, const double *q_ref,
                                                 const double *q_scale, double *sums_dev, void *stream)
{
    using namespace vlbm;
    if (!pop_dev || !sums_dev) return fail(nullptr, VLBM_ERR_ARG, "no-allocation sums: NULL buffer");
    if (dim != 2 && dim != 3) return fail(nullptr, VLBM_ERR_ARG, "no-allocation sums: dim must be 2 or 3");
    if (nx < 1 || ny < 1 || nz < 1 || (dim == 2 && nz != 1))
        return fail(nullptr, VLBM_ERR_ARG, "no-allocation sums: bad grid size");
    if (parity != 0 && parity != 1) return fail(nullptr, VLBM_ERR_ARG, "no-allocation sums: parity must be 0 or 1");
    const int64_t ncell = (int64_t)nx * ny * nz;
    if (ncell > kNaMaxCells)
        return fail(nullptr, VLBM_ERR_ARG,
                    "no-allocation sums: the domain has more than 268435456 (2^28) cells, the most its "
                    "fixed 256 KiB scratch array can reduce");
    if (stride < ncell) return fail(nullptr, VLBM_ERR_ARG, "no-allocation sums: stride smaller than the cell count");
    const bool dev = storage == VLBM_F16_DEV || storage == VLBM_BF16_DEV;
    if (dev && (!q_ref || !q_scale))
        return fail(nullptr, VLBM_ERR_ARG, "no-allocation sums: deviation storage needs q_ref and q_scale");
    double *scratch = nullptr;
    vlbm_status s = na_scratch(&scratch);
    if (s != VLBM_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool d2 = dim == 2;
    switch (storage) {
    case VLBM_F64:
        return d2 ? na_run<2, double>(pop_dev, nx, ny, nz, stride, parity, q_ref, q_scale, sums_dev, st, scratch)
                  : na_run<3, double>(pop_dev, nx, ny, nz, stride, parity, q_ref, q_scale, sums_dev, st, scratch);
    case VLBM_F32:
        return d2 ? na_run<2, float>(pop_dev, nx, ny, nz, stride, parity, q_ref, q_scale, sums_dev, st, scratch)
                  : na_run<3, float>(pop_dev, nx, ny, nz, stride, parity, q_ref, q_scale, sums_dev, st, scratch);
    case VLBM_F16_DEV:
        return d2 ? na_run<2, __half>(pop_dev, nx, ny, nz, stride, parity, q_ref, q_scale, sums_dev, st, scratch)
                  : na_run<3, __half>(pop_dev, nx, ny, nz, stride, parity, q_ref, q_scale, sums_dev, st, scratch);
    case VLBM_BF16_DEV:
        return d2 ? na_run<2, __nv_bfloat16>(pop_dev, nx, ny, nz, stride, parity, q_ref, q_scale, sums_dev, st,
                                            scratch)
                  : na_run<3, __nv_bfloat16>(pop_dev, nx, ny, nz, stride, parity, q_ref, q_scale, sums_dev, st,
                                            scratch);
    }
    return fail(nullptr, VLBM_ERR_ARG, "no-allocation sums: unknown storage");
}
