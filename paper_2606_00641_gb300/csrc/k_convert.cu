// k_convert.cu -- precision of staged host fields (sm_103a).
//
// The single-precision host-field calls (vlbm_init_fields_f32,
// vlbm_moments_f32) move floats over the host link -- half the bytes of the
// double fields, and the host link (~200 GB/s) is what bounds those calls --
// and convert each staged chunk on the device: widen before the init kernel,
// narrow after the moments kernel.  Both are exact for values that are floats.
#include "vlbm_internal.cuh"

namespace vlbm {
namespace {

constexpr int kConvThreads = 256;

// in[v * stride + t] -> out[v * stride + t], t < n, v < nvar (blockIdx.y = v)
template <class A, class B>
__global__ void k_convert(const A *__restrict__ in, int64_t n, int64_t stride, B *__restrict__ out)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int64_t at = (int64_t)blockIdx.y * stride + t;
    out[at] = (B)in[at];
}

template <class A, class B>
vlbm_status convert(vlbm_ctx *c, const A *in, int nvar, int64_t n, int64_t stride, B *out, const char *what)
{
    if (n <= 0) return VLBM_OK;
    const dim3 grid((unsigned)((n + kConvThreads - 1) / kConvThreads), (unsigned)nvar);
    k_convert<A, B><<<grid, kConvThreads, 0, c->stream>>>(in, n, stride, out);
    c->launches++;
    return cuda_check(c, cudaGetLastError(), what);
}

}  // namespace

vlbm_status widen_fields(vlbm_ctx *c, const float *in, int nvar, int64_t n, int64_t stride, double *out)
{
    return convert(c, in, nvar, n, stride, out, "field widening launch");
}

vlbm_status narrow_fields(vlbm_ctx *c, const double *in, int nvar, int64_t n, int64_t stride, float *out)
{
    return convert(c, in, nvar, n, stride, out, "field narrowing launch");
}

}  // namespace vlbm
