// vlbm_api.cu -- the C ABI declared in include/vlbm.h.
//
// Host responsibilities only: validation, device memory, the stream, the
// step loop (kernels captured once into CUDA graphs of kGraphLen steps per
// AA parity and replayed), health-flag read-back, staging of host fields in
// bounded chunks, checkpoints.  Every arithmetic step of the method runs in
// the kernels of k_ideal.cu, k_resistive.cu, k_diss.cu and k_batch.cu.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "vlbm_internal.cuh"

using namespace vlbm;

namespace {

constexpr int kGraphLen = 32;                  // steps per captured graph
constexpr int64_t kStageCells = int64_t(1) << 22;  // cells per host-staging chunk
thread_local std::string g_err;                // errors raised before a ctx exists

size_t elem_size(int storage)
{
    switch (storage) {
    case VLBM_F64: return 8;
    case VLBM_F32: return 4;
    case VLBM_F16_DEV:
    case VLBM_BF16_DEV: return 2;
    }
    return 0;
}

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

void *dev_alloc(vlbm_ctx *c, size_t bytes)
{
    void *p = nullptr;
    if (bytes == 0) bytes = 256;
    if (c->params.alloc) {
        p = c->params.alloc(bytes, (void *)c->stream, c->params.alloc_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) c->owned.emplace_back(p, bytes);
    return p;
}

void dev_free_all(vlbm_ctx *c)
{
    for (auto &pr : c->owned) {
        if (c->params.dealloc)
            c->params.dealloc(pr.first, pr.second, (void *)c->stream, c->params.alloc_user);
        else if (!c->params.alloc)
            cudaFree(pr.first);
    }
    c->owned.clear();
}

vlbm_status validate(const vlbm_params *p, bool batch_member)
{
    if (!p) return VLBM_ERR_ARG;
    if (p->model != VLBM_IDEAL && p->model != VLBM_RESISTIVE && p->model != VLBM_IDEAL_POWELL &&
        p->model != VLBM_DISSIPATIVE) {
        g_err = "model must be VLBM_IDEAL, VLBM_RESISTIVE, VLBM_IDEAL_POWELL or VLBM_DISSIPATIVE";
        return VLBM_ERR_ARG;
    }
    if (p->dim != 2 && p->dim != 3) {
        g_err = "dim must be 2 or 3";
        return VLBM_ERR_ARG;
    }
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || (p->dim == 2 && p->nz != 1) || p->ny > 65535 ||
        p->nz > 65535) {
        g_err = "bad grid size (nx, ny, nz >= 1; ny, nz <= 65535; nz = 1 in 2-D)";
        return VLBM_ERR_ARG;
    }
    if (elem_size(p->storage) == 0) {
        g_err = "unknown storage";
        return VLBM_ERR_ARG;
    }
    const int nt = p->model == VLBM_RESISTIVE ? 4 : 8;
    for (int k = 0; k < nt; ++k)
        if (!(p->tau[k] > 0.5) || !(p->tau[k] < 1e6)) {
            g_err = "tau must be > 1/2 on every lattice";
            return VLBM_ERR_UNSTABLE;
        }
    if (p->model == VLBM_IDEAL_POWELL) {
        if (!(p->tau_d > 0.5) || !(p->tau_d < 1e6) || !(p->tau_m > 0.5) || !(p->tau_m < 1e12)) {
            g_err = "Powell model: tau_d and tau_m must be > 1/2";
            return VLBM_ERR_UNSTABLE;
        }
        if (p->storage != VLBM_F32 && p->storage != VLBM_F64) {
            g_err = "the Powell model is built for F32 and F64 storage";
            return VLBM_ERR_UNSUPPORTED;
        }
    }
    if (p->model == VLBM_DISSIPATIVE) {
        if (!(p->tau_g > 0.5) || !(p->tau_g < 1e6) || !(p->tau_m > 0.5) || !(p->tau_m < 1e12)) {
            g_err = "dissipative model: tau_g and tau_m must be > 1/2";
            return VLBM_ERR_UNSTABLE;
        }
        if (!(p->nu >= 0.0) || !(p->eta0 >= 0.0) || !std::isfinite(p->nu) || !std::isfinite(p->eta0) ||
            !std::isfinite(p->j_c)) {
            g_err = "dissipative model: nu and eta0 must be finite and >= 0, j_c finite";
            return VLBM_ERR_ARG;
        }
        if (p->storage != VLBM_F32 && p->storage != VLBM_F64) {
            g_err = "the dissipative model is built for F32 and F64 storage";
            return VLBM_ERR_UNSUPPORTED;
        }
    }
    if (p->model == VLBM_IDEAL || p->model == VLBM_IDEAL_POWELL || p->model == VLBM_DISSIPATIVE) {
        if (!(p->gamma > 1.0)) {
            g_err = "gamma must be > 1";
            return VLBM_ERR_ARG;
        }
        if ((p->storage == VLBM_F16_DEV || p->storage == VLBM_BF16_DEV) &&
            (!(p->p_theta >= 0.0) || !std::isfinite(p->p_theta))) {
            g_err = "p_theta must be finite and >= 0";
            return VLBM_ERR_ARG;
        }
        if (p->storage == VLBM_F16_DEV || p->storage == VLBM_BF16_DEV)
            for (int k = 0; k < 8; ++k)
                if (p->q_scale[k] < 0.0 || !(p->q_scale[k] < 1e300)) {
                    g_err = "q_scale must be >= 0 and finite";
                    return VLBM_ERR_ARG;
                }
    } else {
        if (p->dim != 3) {
            g_err = "the resistive model is 3-D";
            return VLBM_ERR_ARG;
        }
        if (p->storage != VLBM_F32) {
            g_err = "the resistive model is built for F32 storage";
            return VLBM_ERR_UNSUPPORTED;
        }
        if (p->walls_y && p->ny < 3) {
            g_err = "walls need ny >= 3";
            return VLBM_ERR_ARG;
        }
    }
    if (batch_member && (p->model != VLBM_IDEAL || p->dim != 2 || p->storage != VLBM_F32)) {
        g_err = "batched domains are 2-D ideal MHD with F32 storage";
        return VLBM_ERR_UNSUPPORTED;
    }
    return VLBM_OK;
}

Domain make_domain(const vlbm_params *p)
{
    Domain d{};
    d.nx = p->nx;
    d.ny = p->ny;
    d.nz = p->nz;
    d.ncell = (int64_t)p->nx * p->ny * p->nz;
    d.stride = round_up(d.ncell, 64);
    d.gamma = p->gamma;
    for (int k = 0; k < 8; ++k) {  // the public arrays hold 8 lattices
        d.tau[k] = p->tau[k] > 0.5 ? p->tau[k] : 1.0;
        d.source[k] = p->source[k];
        d.q_ref[k] = p->q_ref[k];
        d.q_scale[k] = p->q_scale[k] > 0.0 ? p->q_scale[k] : 1.0;
    }
    // ninth lattice (Powell model): D, no uniform source, no deviation storage
    d.tau[8] = p->tau_d > 0.5 ? p->tau_d : 1.0;
    d.source[8] = 0.0;
    d.q_ref[8] = 0.0;
    d.q_scale[8] = 1.0;
    d.tau_m = p->tau_m > 0.5 ? p->tau_m : 1.0;
    for (int a = 0; a < 3; ++a) {
        d.force[a] = p->force[a];
        d.b_wall[a] = p->b_wall[a];
    }
    d.walls_y = p->walls_y;
    return d;
}

vlbm_status apply_flags(vlbm_ctx *c, unsigned flags)
{
    if (flags & kFlagTimeout) {
        c->sticky = VLBM_ERR_TIMEOUT;
        c->err = "a bounded device wait expired";
    } else if (flags & kFlagNonPhysical) {
        c->sticky = VLBM_ERR_NONPHYSICAL;
        c->err = "a kernel saw NaN, rho <= 0 or p <= 0";
    }
    return c->sticky;
}

vlbm_status read_flags_sync(vlbm_ctx *c, unsigned *out)
{
    vlbm_status s = cuda_check(c, cudaMemcpyAsync(c->h_flags, c->d_flags, sizeof(unsigned),
                                                  cudaMemcpyDeviceToHost, c->stream),
                               "flag read-back");
    if (s != VLBM_OK) return s;
    s = cuda_check(c, cudaStreamSynchronize(c->stream), "stream synchronise");
    if (s != VLBM_OK) return s;
    *out = *c->h_flags;
    c->flag_pending = false;
    return VLBM_OK;
}

void poll_flags(vlbm_ctx *c)
{
    if (c->flag_pending && cudaEventQuery(c->flag_event) == cudaSuccess) {
        c->flag_pending = false;
        apply_flags(c, *c->h_flags);
    }
    cudaGetLastError();  // cudaErrorNotReady from the query is not an error
}

vlbm_status launch_step(vlbm_ctx *c, int parity)
{
    if (c->batched) return batch_step(c, parity, c->tune_choice);
    if (c->model == VLBM_RESISTIVE) return resistive_step(c, parity);
    if (c->model == VLBM_DISSIPATIVE) return diss_step(c, parity);
    if (c->closure) return closure_step(c, parity);
    vlbm_status s = ideal_step(c, parity);
    // for the next step's reads; a slab fills after its halo exchange (vlbm_halo_unpack), since
    // the Neumann moments of its first and last layers read slots the exchange brings
    if (s == VLBM_OK && any_open_face(c) && !c->slab) s = open_fill(c, parity ^ 1);
    return s;
}

vlbm_status init_range(vlbm_ctx *c, int d, const double *Q, int64_t c0, int64_t n, int64_t qs)
{
    if (c->model == VLBM_RESISTIVE) return resistive_init_range(c, d, Q, c0, n, qs);
    if (c->model == VLBM_DISSIPATIVE) return diss_init_range(c, Q, c0, n, qs);
    return ideal_init_range(c, d, Q, c0, n, qs);
}

vlbm_status moments_range(vlbm_ctx *c, int d, double *out, int64_t c0, int64_t n, int64_t os)
{
    if (c->model == VLBM_RESISTIVE) return resistive_moments_range(c, d, out, c0, n, os);
    if (c->model == VLBM_DISSIPATIVE) return diss_moments_range(c, out, c0, n, os);
    return ideal_moments_range(c, d, out, c0, n, os);
}

vlbm_status ensure_stage(vlbm_ctx *c, size_t bytes)
{
    if (c->d_q_bytes >= bytes) return VLBM_OK;
    // staging grows monotonically; the old block stays owned until destroy
    void *p = dev_alloc(c, bytes);
    if (!p) return fail(c, VLBM_ERR_OOM, "staging allocation failed");
    c->d_q = static_cast<double *>(p);
    c->d_q_bytes = bytes;
    return VLBM_OK;
}

// Host fields move through two device chunk buffers: the copies of one chunk
// run on an internal stream while the context's stream runs the kernel of
// the other chunk; events order the two streams per buffer.
static vlbm_status ensure_copy_stream(vlbm_ctx *c)
{
    if (c->copy_stream) return VLBM_OK;
    cudaStream_t s = nullptr;
    vlbm_status st = cuda_check(c, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "copy stream");
    for (int b = 0; b < 2 && st == VLBM_OK; ++b) {
        st = cuda_check(c, cudaEventCreateWithFlags(&c->ev_copy[b], cudaEventDisableTiming), "copy event");
        if (st == VLBM_OK)
            st = cuda_check(c, cudaEventCreateWithFlags(&c->ev_kern[b], cudaEventDisableTiming), "copy event");
    }
    if (st == VLBM_OK) c->copy_stream = s;
    else if (s) cudaStreamDestroy(s);
    return st;
}

void drop_graphs(vlbm_ctx *c)
{
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
    c->graph_launches.clear();
}

cudaGraphExec_t get_graph(vlbm_ctx *c, int parity, int len, int64_t *launches)
{
    const int key = parity * 1024 + len;
    auto it = c->graphs.find(key);
    if (it != c->graphs.end()) {
        *launches = c->graph_launches[key];
        return it->second;
    }
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    const int64_t before = c->launches;
    bool ok = true;
    for (int s = 0; s < len && ok; ++s) ok = launch_step(c, (parity + s) & 1) == VLBM_OK;
    const int64_t captured = c->launches - before;
    c->launches = before;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (!ok || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return nullptr;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    c->graphs[key] = exec;
    c->graph_launches[key] = captured;
    *launches = captured;
    return exec;
}

vlbm_status create_common(const vlbm_params *p, int count, vlbm_ctx **out)
{
    if (!out || !p || count < 1) return VLBM_ERR_ARG;
    *out = nullptr;
    for (int d = 0; d < count; ++d) {
        vlbm_status s = validate(&p[d], count > 1);
        if (s != VLBM_OK) return s;
    }
    vlbm_ctx *c = new vlbm_ctx();
    c->params = p[0];
    c->model = p[0].model;
    c->dim = p[0].dim;
    c->storage = p[0].storage;
    c->elem = elem_size(c->storage);
    c->batched = count > 1;
    if (c->model == VLBM_IDEAL || c->model == VLBM_IDEAL_POWELL) {
        c->q = c->dim == 2 ? 5 : 7;
        c->nlat = c->model == VLBM_IDEAL_POWELL ? 9 : 8;
        c->nvar = c->nlat;
        c->nslot = c->nlat * c->q;
    } else if (c->model == VLBM_DISSIPATIVE) {
        c->q = c->dim == 2 ? 5 : 7;
        c->nlat = 8 + 6 * c->dim;  // 20 in 2-D, 26 in 3-D
        c->nvar = c->nlat;
        c->nslot = c->nlat * c->q;
    } else {
        c->q = 19;
        c->nlat = 4;
        c->nvar = 7;
        c->nslot = 19 + 3 * 7;
    }
    int64_t total = 0;
    for (int d = 0; d < count; ++d) {
        Domain dm = make_domain(&p[d]);
        dm.offset = total;
        total += (int64_t)c->nslot * dm.stride;
        c->dom.push_back(dm);
    }
    vlbm_status s = VLBM_OK;
    if (p[0].stream) {
        c->stream = static_cast<cudaStream_t>(p[0].stream);
    } else {
        s = cuda_check(c, cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking), "stream create");
        c->own_stream = s == VLBM_OK;
    }
    if (s == VLBM_OK) s = cuda_check(c, cudaEventCreateWithFlags(&c->flag_event, cudaEventDisableTiming),
                                     "event create");
    if (s == VLBM_OK) s = cuda_check(c, cudaMallocHost(&c->h_flags, 64), "pinned flag word");
    if (s == VLBM_OK) {
        c->pop_bytes = (size_t)total * c->elem;
        c->pop = dev_alloc(c, c->pop_bytes);
        const size_t partial_bytes = (size_t)kReduceBlocks * 8 * sizeof(double);
        void *status = dev_alloc(c, 256 + partial_bytes + 16 * sizeof(double));
        if (!c->pop || !status) {
            s = fail(c, VLBM_ERR_OOM, "device allocation failed");
        } else {
            c->d_flags = static_cast<unsigned *>(status);
            c->d_sums = reinterpret_cast<double *>(static_cast<char *>(status) + 128);
            c->d_partials = reinterpret_cast<double *>(static_cast<char *>(status) + 256);
            c->d_refscale = reinterpret_cast<double *>(static_cast<char *>(status) + 256 + partial_bytes);
            for (int k = 0; k < 8; ++k) {
                c->h_refscale[k] = c->dom[0].q_ref[k];
                c->h_refscale[8 + k] = c->dom[0].q_scale[k];
            }
            s = cuda_check(c, cudaMemsetAsync(c->d_flags, 0, 128, c->stream), "flag clear");
            if (s == VLBM_OK)
                s = cuda_check(c, cudaMemcpyAsync(c->d_refscale, c->h_refscale, sizeof(c->h_refscale),
                                                  cudaMemcpyHostToDevice, c->stream),
                               "reference state upload");
        }
    }
    if (s == VLBM_OK && c->batched) s = batch_prepare(c);
    if (s == VLBM_OK) s = cuda_check(c, cudaStreamSynchronize(c->stream), "create synchronise");
    if (s != VLBM_OK) {
        g_err = c->err;
        vlbm_destroy(c);
        return s;
    }
    *out = c;
    return VLBM_OK;
}

}  // namespace

namespace vlbm {

vlbm_status fail(vlbm_ctx *c, vlbm_status s, const std::string &msg)
{
    if (c) c->err = msg;
    else g_err = msg;
    return s;
}

vlbm_status cuda_check(vlbm_ctx *c, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return VLBM_OK;
    return fail(c, e == cudaErrorMemoryAllocation ? VLBM_ERR_OOM : VLBM_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace vlbm

extern "C" {

void vlbm_default_params(vlbm_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->model = VLBM_IDEAL;
    p->dim = 3;
    p->nx = p->ny = p->nz = 64;
    p->storage = VLBM_F32;
    p->gamma = 5.0 / 3.0;
    for (int k = 0; k < 8; ++k) {
        p->tau[k] = 0.51;
        p->q_scale[k] = 1.0;
    }
    p->tau_d = 0.51;
    p->tau_m = 1.0;
    p->tau_g = 0.51;
    p->p_theta = 0.01;
}

vlbm_status vlbm_create(const vlbm_params *p, vlbm_ctx **out) { return create_common(p, 1, out); }

vlbm_status vlbm_create_batch(const vlbm_params *p, int count, vlbm_ctx **out)
{
    if (count < 1) return VLBM_ERR_ARG;
    return create_common(p, count, out);
}

static vlbm_status finish_init(vlbm_ctx *c)
{
    unsigned flags = 0;
    vlbm_status s = read_flags_sync(c, &flags);
    if (s != VLBM_OK) return s;
    // a NaN or non-positive state is reported as such even though it also
    // fails the signal-speed test
    if (flags & kFlagNonPhysical) {
        cudaMemsetAsync(c->d_flags, 0, sizeof(unsigned), c->stream);
        return fail(c, VLBM_ERR_NONPHYSICAL, "initial fields have NaN, rho <= 0 or p <= 0");
    }
    if (flags & kFlagUnstable) {
        cudaMemsetAsync(c->d_flags, 0, sizeof(unsigned), c->stream);
        return fail(c, VLBM_ERR_UNSTABLE, "max(|u| + c_f) >= cs: the scheme's diffusion would be negative");
    }
    c->sticky = VLBM_OK;
    return VLBM_OK;
}

static vlbm_status begin_init(vlbm_ctx *c, int domain)
{
    if (domain < 0 || domain >= (int)c->dom.size()) return fail(c, VLBM_ERR_ARG, "bad domain index");
    if (c->batched && (c->step & 1)) return fail(c, VLBM_ERR_STATE, "batched init needs an even step count");
    if (c->flag_pending) cudaEventSynchronize(c->flag_event);
    c->flag_pending = false;
    c->step = 0;
    c->steps_since_check = 0;
    c->halo_pending = false;  // parity 0: every population is in its own slab
    return cuda_check(c, cudaMemsetAsync(c->d_flags, 0, sizeof(unsigned), c->stream), "flag clear");
}

// Host fields (double, or float with f32) through the two staging chunks.  The
// float form copies half the bytes over the host link and widens each chunk to
// double on the device before the init kernel, whose arithmetic is unchanged.
static vlbm_status init_from_host(vlbm_ctx *c, int domain, const void *Q_host, bool f32)
{
    vlbm_status s = begin_init(c, domain);
    if (s != VLBM_OK) return s;
    const int64_t N = c->dom[domain].ncell;
    const int64_t chunk = std::min<int64_t>(N, kStageCells);
    const size_t half = (size_t)c->nvar * chunk;  // values per staging buffer
    s = ensure_stage(c, 2 * half * sizeof(double) + (f32 ? 2 * half * sizeof(float) : 0));
    if (s == VLBM_OK) s = ensure_copy_stream(c);
    // both buffers free once the work already queued on the context's stream is done
    for (int b = 0; b < 2 && s == VLBM_OK; ++b) s = cuda_check(c, cudaEventRecord(c->ev_kern[b], c->stream), "event");
    float *fstage = reinterpret_cast<float *>(c->d_q + 2 * half);
    const size_t vbytes = f32 ? sizeof(float) : sizeof(double);
    int i = 0;
    for (int64_t c0 = 0; s == VLBM_OK && c0 < N; c0 += chunk, ++i) {
        const int b = i & 1;
        double *buf = c->d_q + b * half;
        char *land = f32 ? reinterpret_cast<char *>(fstage + b * half) : reinterpret_cast<char *>(buf);
        const int64_t n = std::min<int64_t>(chunk, N - c0);
        s = cuda_check(c, cudaStreamWaitEvent(c->copy_stream, c->ev_kern[b], 0), "stream order");
        for (int v = 0; v < c->nvar && s == VLBM_OK; ++v)
            s = cuda_check(c, cudaMemcpyAsync(land + v * chunk * vbytes,
                                              static_cast<const char *>(Q_host) + (v * N + c0) * vbytes, n * vbytes,
                                              cudaMemcpyHostToDevice, c->copy_stream),
                           "field upload");
        if (s == VLBM_OK) s = cuda_check(c, cudaEventRecord(c->ev_copy[b], c->copy_stream), "event");
        if (s == VLBM_OK) s = cuda_check(c, cudaStreamWaitEvent(c->stream, c->ev_copy[b], 0), "stream order");
        if (s == VLBM_OK && f32) s = widen_fields(c, fstage + b * half, c->nvar, n, chunk, buf);
        if (s == VLBM_OK) s = init_range(c, domain, buf, c0, n, chunk);
        if (s == VLBM_OK) s = cuda_check(c, cudaEventRecord(c->ev_kern[b], c->stream), "event");
    }
    if (s != VLBM_OK) return s;
    return finish_init(c);
}

vlbm_status vlbm_init_fields(vlbm_ctx *c, int domain, const double *Q_host)
{
    vlbm::NvtxRange range("vlbm_init_fields");
    if (!c || !Q_host) return VLBM_ERR_ARG;
    return init_from_host(c, domain, Q_host, false);
}

vlbm_status vlbm_init_fields_f32(vlbm_ctx *c, int domain, const float *Q_host)
{
    vlbm::NvtxRange range("vlbm_init_fields_f32");
    if (!c || !Q_host) return VLBM_ERR_ARG;
    if (c->storage == VLBM_F64) return fail(c, VLBM_ERR_UNSUPPORTED, "single-precision fields need FP32 or 16-bit storage");
    return init_from_host(c, domain, Q_host, true);
}

vlbm_status vlbm_init_fields_device(vlbm_ctx *c, int domain, const double *Q_dev)
{
    vlbm::NvtxRange range("vlbm_init_fields_device");
    if (!c || !Q_dev) return VLBM_ERR_ARG;
    vlbm_status s = begin_init(c, domain);
    if (s != VLBM_OK) return s;
    const int64_t N = c->dom[domain].ncell;
    s = init_range(c, domain, Q_dev, 0, N, N);
    if (s != VLBM_OK) return s;
    return finish_init(c);
}

// After n steps were enqueued: read the health flag back asynchronously every
// params.check_every steps.
static void schedule_check(vlbm_ctx *c, int n)
{
    c->steps_since_check += n;
    const int every = c->params.check_every;
    if (every > 0 && c->steps_since_check >= every && !c->flag_pending) {
        c->steps_since_check = 0;
        if (cudaMemcpyAsync(c->h_flags, c->d_flags, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream) ==
                cudaSuccess &&
            cudaEventRecord(c->flag_event, c->stream) == cudaSuccess)
            c->flag_pending = true;
        cudaGetLastError();
    }
}

// A slab whose last step has not had its halo exchanged holds populations that
// belong to its neighbours: nothing may read its state yet.
static vlbm_status slab_ready(vlbm_ctx *c)
{
    if (c->slab && c->halo_pending)
        return fail(c, VLBM_ERR_STATE, "slab: the last step's halo exchange has not been unpacked");
    return VLBM_OK;
}

vlbm_status vlbm_step(vlbm_ctx *c, int n)
{
    vlbm::NvtxRange range("vlbm_step");
    if (!c || n < 0) return VLBM_ERR_ARG;
    poll_flags(c);
    if (c->sticky != VLBM_OK) return c->sticky;
    if (c->slab) {
        if (n > 1) return fail(c, VLBM_ERR_STATE, "slab: one step at a time, each followed by its halo exchange");
        vlbm_status s = slab_ready(c);
        if (s != VLBM_OK) return s;
    }
    for (int a = 0; a < 3; ++a)
        if ((c->face_kind[2 * a] == VLBM_BC_EQUILIBRIUM) != (c->face_kind[2 * a + 1] == VLBM_BC_EQUILIBRIUM))
            return fail(c, VLBM_ERR_ARG, "one face of an axis is open and the other periodic");
    const bool graphs = c->stream != nullptr && c->stream != cudaStreamLegacy &&
                        c->stream != cudaStreamPerThread;
    int left = n;
    while (left > 0) {
        if (graphs && left >= kGraphLen) {
            int64_t in_graph = 0;
            cudaGraphExec_t g = get_graph(c, (int)(c->step & 1), kGraphLen, &in_graph);
            if (g) {
                vlbm_status s = cuda_check(c, cudaGraphLaunch(g, c->stream), "graph launch");
                if (s != VLBM_OK) return s;
                c->step += kGraphLen;
                c->launches += in_graph;
                left -= kGraphLen;
                continue;
            }
        }
        vlbm_status s = launch_step(c, (int)(c->step & 1));
        if (s != VLBM_OK) return s;
        c->step += 1;
        left -= 1;
        if (c->slab) c->halo_pending = true;
    }
    schedule_check(c, n);
    return c->sticky;
}

vlbm_status vlbm_sync(vlbm_ctx *c)
{
    vlbm::NvtxRange range("vlbm_sync");
    if (!c) return VLBM_ERR_ARG;
    unsigned flags = 0;
    vlbm_status s = read_flags_sync(c, &flags);
    if (s != VLBM_OK) return s;
    return apply_flags(c, flags);
}

// Moments to host fields (double, or float with f32) through the staging chunks;
// the float form narrows each chunk on the device and copies half the bytes.
static vlbm_status moments_to_host(vlbm_ctx *c, int domain, void *Q_host, bool f32)
{
    if (domain < 0 || domain >= (int)c->dom.size()) return fail(c, VLBM_ERR_ARG, "bad domain index");
    if (slab_ready(c) != VLBM_OK) return VLBM_ERR_STATE;
    const int64_t N = c->dom[domain].ncell;
    const int64_t chunk = std::min<int64_t>(N, kStageCells);
    const size_t half = (size_t)c->nvar * chunk;  // values per staging buffer
    vlbm_status s = ensure_stage(c, 2 * half * sizeof(double) + (f32 ? 2 * half * sizeof(float) : 0));
    if (s == VLBM_OK) s = ensure_copy_stream(c);
    for (int b = 0; b < 2 && s == VLBM_OK; ++b)  // no download pending on either buffer
        s = cuda_check(c, cudaEventRecord(c->ev_copy[b], c->copy_stream), "event");
    float *fstage = reinterpret_cast<float *>(c->d_q + 2 * half);
    const size_t vbytes = f32 ? sizeof(float) : sizeof(double);
    int i = 0;
    for (int64_t c0 = 0; s == VLBM_OK && c0 < N; c0 += chunk, ++i) {
        const int b = i & 1;
        double *buf = c->d_q + b * half;
        char *land = f32 ? reinterpret_cast<char *>(fstage + b * half) : reinterpret_cast<char *>(buf);
        const int64_t n = std::min<int64_t>(chunk, N - c0);
        s = cuda_check(c, cudaStreamWaitEvent(c->stream, c->ev_copy[b], 0), "stream order");
        if (s == VLBM_OK) s = moments_range(c, domain, buf, c0, n, chunk);
        if (s == VLBM_OK && f32) s = narrow_fields(c, buf, c->nvar, n, chunk, fstage + b * half);
        if (s == VLBM_OK) s = cuda_check(c, cudaEventRecord(c->ev_kern[b], c->stream), "event");
        if (s == VLBM_OK) s = cuda_check(c, cudaStreamWaitEvent(c->copy_stream, c->ev_kern[b], 0), "stream order");
        for (int v = 0; v < c->nvar && s == VLBM_OK; ++v)
            s = cuda_check(c, cudaMemcpyAsync(static_cast<char *>(Q_host) + (v * N + c0) * vbytes,
                                              land + v * chunk * vbytes, n * vbytes, cudaMemcpyDeviceToHost,
                                              c->copy_stream),
                           "field download");
        if (s == VLBM_OK) s = cuda_check(c, cudaEventRecord(c->ev_copy[b], c->copy_stream), "event");
    }
    if (s != VLBM_OK) return s;
    s = cuda_check(c, cudaStreamSynchronize(c->copy_stream), "moments synchronise");
    if (s != VLBM_OK) return s;
    return cuda_check(c, cudaStreamSynchronize(c->stream), "moments synchronise");
}

vlbm_status vlbm_moments(vlbm_ctx *c, int domain, double *Q_host)
{
    vlbm::NvtxRange range("vlbm_moments");
    if (!c || !Q_host) return VLBM_ERR_ARG;
    return moments_to_host(c, domain, Q_host, false);
}

vlbm_status vlbm_moments_f32(vlbm_ctx *c, int domain, float *Q_host)
{
    vlbm::NvtxRange range("vlbm_moments_f32");
    if (!c || !Q_host) return VLBM_ERR_ARG;
    if (c->storage == VLBM_F64) return fail(c, VLBM_ERR_UNSUPPORTED, "single-precision fields need FP32 or 16-bit storage");
    return moments_to_host(c, domain, Q_host, true);
}

vlbm_status vlbm_moments_device(vlbm_ctx *c, int domain, double *Q_dev)
{
    vlbm::NvtxRange range("vlbm_moments_device");
    if (!c || !Q_dev) return VLBM_ERR_ARG;
    if (domain < 0 || domain >= (int)c->dom.size()) return fail(c, VLBM_ERR_ARG, "bad domain index");
    if (slab_ready(c) != VLBM_OK) return VLBM_ERR_STATE;
    const int64_t N = c->dom[domain].ncell;
    return moments_range(c, domain, Q_dev, 0, N, N);
}

vlbm_status vlbm_gather_populations(vlbm_ctx *c, int domain, const int64_t *cells, int ncells, double *f_host)
{
    if (!c || !cells || !f_host || ncells < 1) return VLBM_ERR_ARG;
    if (domain < 0 || domain >= (int)c->dom.size()) return fail(c, VLBM_ERR_ARG, "bad domain index");
    if (slab_ready(c) != VLBM_OK) return VLBM_ERR_STATE;
    const int64_t N = c->dom[domain].ncell;
    for (int t = 0; t < ncells; ++t)
        if (cells[t] < 0 || cells[t] >= N) return fail(c, VLBM_ERR_ARG, "cell index out of range");
    const size_t need = (size_t)ncells * (1 + c->nslot) * sizeof(double);
    vlbm_status s = ensure_stage(c, need);
    if (s != VLBM_OK) return s;
    int64_t *d_cells = reinterpret_cast<int64_t *>(c->d_q);
    double *d_out = c->d_q + ncells;
    s = cuda_check(c, cudaMemcpyAsync(d_cells, cells, ncells * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream),
                   "cell upload");
    if (s == VLBM_OK)
        s = c->model == VLBM_RESISTIVE     ? resistive_gather(c, domain, d_cells, ncells, d_out)
            : c->model == VLBM_DISSIPATIVE ? diss_gather(c, d_cells, ncells, d_out)
                                           : ideal_gather(c, domain, d_cells, ncells, d_out);
    if (s == VLBM_OK)
        s = cuda_check(c, cudaMemcpyAsync(f_host, d_out, (size_t)ncells * c->nslot * sizeof(double),
                                          cudaMemcpyDeviceToHost, c->stream),
                       "population download");
    if (s != VLBM_OK) return s;
    return cuda_check(c, cudaStreamSynchronize(c->stream), "gather synchronise");
}

vlbm_status vlbm_conservation(vlbm_ctx *c, int domain, double *sums)
{
    vlbm::NvtxRange range("vlbm_conservation");
    if (!c || !sums) return VLBM_ERR_ARG;
    if (domain < 0 || domain >= (int)c->dom.size()) return fail(c, VLBM_ERR_ARG, "bad domain index");
    if (slab_ready(c) != VLBM_OK) return VLBM_ERR_STATE;
    vlbm_status s = c->model == VLBM_RESISTIVE ? resistive_sums(c, domain, c->d_sums)
                                               : ideal_sums(c, domain, c->d_sums);
    if (s == VLBM_OK)
        s = cuda_check(c, cudaMemcpyAsync(sums, c->d_sums, std::min(c->nvar, 8) * sizeof(double), cudaMemcpyDeviceToHost,
                                          c->stream),
                       "sums download");
    if (s != VLBM_OK) return s;
    unsigned flags = 0;
    s = read_flags_sync(c, &flags);
    if (s != VLBM_OK) return s;
    apply_flags(c, flags);
    return VLBM_OK;
}

struct SaveHeader {
    uint64_t magic;
    int32_t model, dim, storage, ndomains;
    int64_t step;
    uint64_t pop_bytes;
};
static const uint64_t kMagic = 0x564c424d53415645ull;  // "VLBMSAVE"

vlbm_status vlbm_save(vlbm_ctx *c, void *buf, size_t *bytes)
{
    vlbm::NvtxRange range("vlbm_save");
    if (!c || !bytes) return VLBM_ERR_ARG;
    const size_t need = sizeof(SaveHeader) + c->pop_bytes;
    if (!buf) {
        *bytes = need;
        return VLBM_OK;
    }
    if (*bytes < need) return fail(c, VLBM_ERR_ARG, "checkpoint buffer too small");
    if (slab_ready(c) != VLBM_OK) return VLBM_ERR_STATE;
    SaveHeader h{kMagic, c->model, c->dim, c->storage, (int32_t)c->dom.size(), c->step, c->pop_bytes};
    std::memcpy(buf, &h, sizeof(h));
    vlbm_status s = cuda_check(c, cudaMemcpyAsync(static_cast<char *>(buf) + sizeof(h), c->pop, c->pop_bytes,
                                                  cudaMemcpyDeviceToHost, c->stream),
                               "checkpoint download");
    if (s != VLBM_OK) return s;
    *bytes = need;
    return cuda_check(c, cudaStreamSynchronize(c->stream), "checkpoint synchronise");
}

vlbm_status vlbm_load(vlbm_ctx *c, const void *buf, size_t bytes)
{
    vlbm::NvtxRange range("vlbm_load");
    if (!c || !buf || bytes < sizeof(SaveHeader)) return VLBM_ERR_ARG;
    SaveHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (h.magic != kMagic || h.model != c->model || h.dim != c->dim || h.storage != c->storage ||
        h.ndomains != (int32_t)c->dom.size() || h.pop_bytes != c->pop_bytes ||
        bytes < sizeof(h) + c->pop_bytes)
        return fail(c, VLBM_ERR_ARG, "checkpoint does not match this context");
    vlbm_status s = cuda_check(c, cudaMemcpyAsync(c->pop, static_cast<const char *>(buf) + sizeof(h),
                                                  c->pop_bytes, cudaMemcpyHostToDevice, c->stream),
                               "checkpoint upload");
    if (s == VLBM_OK) s = cuda_check(c, cudaMemsetAsync(c->d_flags, 0, sizeof(unsigned), c->stream), "flag clear");
    if (s == VLBM_OK) s = cuda_check(c, cudaStreamSynchronize(c->stream), "load synchronise");
    if (s != VLBM_OK) return s;
    c->step = h.step;
    c->sticky = VLBM_OK;
    c->flag_pending = false;
    c->halo_pending = false;  // checkpoints are taken with the exchange complete
    return VLBM_OK;
}

vlbm_status vlbm_autotune(vlbm_ctx *c, int steps, int *choice)
{
    vlbm::NvtxRange range("vlbm_autotune");
    if (!c || !choice || steps < 0) return VLBM_ERR_ARG;
    *choice = 0;
    if (!c->batched) return VLBM_OK;
    // save state, time every choice, restore
    size_t bytes = c->pop_bytes;
    std::vector<char> keep(bytes);
    vlbm_status s = cuda_check(c, cudaMemcpyAsync(keep.data(), c->pop, bytes, cudaMemcpyDeviceToHost, c->stream),
                               "autotune save");
    if (s == VLBM_OK) s = cuda_check(c, cudaStreamSynchronize(c->stream), "autotune synchronise");
    if (s != VLBM_OK) return s;
    const int64_t step0 = c->step;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int best_choice = 0;
    const int nchoice = batch_num_choices();
    for (int ch = 0; ch < nchoice && s == VLBM_OK; ++ch) {
        for (int w = 0; w < 2 && s == VLBM_OK; ++w) s = batch_step(c, (int)((step0 + w) & 1), ch);
        cudaEventRecord(e0, c->stream);
        for (int t = 0; t < steps && s == VLBM_OK; ++t) s = batch_step(c, (int)((step0 + 2 + t) & 1), ch);
        cudaEventRecord(e1, c->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_choice = ch;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s == VLBM_OK)
        s = cuda_check(c, cudaMemcpyAsync(c->pop, keep.data(), bytes, cudaMemcpyHostToDevice, c->stream),
                       "autotune restore");
    if (s == VLBM_OK) s = cuda_check(c, cudaStreamSynchronize(c->stream), "autotune synchronise");
    if (s != VLBM_OK) return s;
    c->step = step0;
    if (best_choice != c->tune_choice) drop_graphs(c);
    c->tune_choice = best_choice;
    *choice = best_choice;
    return VLBM_OK;
}

vlbm_status vlbm_set_closure(vlbm_ctx *c, vlbm_closure *cl)
{
    if (!c) return VLBM_ERR_ARG;
    if (cl) {
        int nx, ny, nz;
        closure_cells(cl, &nx, &ny, &nz);
        if (c->batched || c->model != VLBM_IDEAL || c->dim != 3 || c->storage != VLBM_F32)
            return fail(c, VLBM_ERR_UNSUPPORTED, "the closure applies to single 3-D ideal-MHD F32 contexts");
        if (c->dom[0].nx != nx || c->dom[0].ny != ny || c->dom[0].nz != nz)
            return fail(c, VLBM_ERR_ARG, "closure grid differs from the context grid");
        if (c->solid) return fail(c, VLBM_ERR_UNSUPPORTED, "a closure and homogenised solids do not combine");
        if (any_open_face(c)) return fail(c, VLBM_ERR_UNSUPPORTED, "a closure and open faces do not combine");
        if (c->slab) return fail(c, VLBM_ERR_UNSUPPORTED, "a closure and a slab context do not combine");
    }
    drop_graphs(c);
    c->closure = cl;
    return VLBM_OK;
}

vlbm_status vlbm_set_solid(vlbm_ctx *c, const float *solid_dev)
{
    if (!c) return VLBM_ERR_ARG;
    if (solid_dev) {
        if (c->batched || c->model != VLBM_IDEAL || (c->storage != VLBM_F32 && c->storage != VLBM_F64))
            return fail(c, VLBM_ERR_UNSUPPORTED,
                        "homogenised solids apply to single ideal-MHD contexts with F32 or F64 storage");
        if (c->closure) return fail(c, VLBM_ERR_UNSUPPORTED, "a closure and homogenised solids do not combine");
    }
    drop_graphs(c);  // captured steps hold the previous pointer
    c->solid = solid_dev;
    return VLBM_OK;
}

vlbm_status vlbm_set_boundary(vlbm_ctx *c, int face, int kind, unsigned dirichlet_mask, const double *values)
{
    if (!c) return VLBM_ERR_ARG;
    if (face < 0 || face >= 2 * c->dim) return fail(c, VLBM_ERR_ARG, "no such face");
    if (kind != VLBM_BC_PERIODIC && kind != VLBM_BC_EQUILIBRIUM) return fail(c, VLBM_ERR_ARG, "no such boundary kind");
    if (kind == VLBM_BC_EQUILIBRIUM) {
        if (c->batched || c->model != VLBM_IDEAL || (c->storage != VLBM_F32 && c->storage != VLBM_F64))
            return fail(c, VLBM_ERR_UNSUPPORTED,
                        "open faces apply to single ideal-MHD contexts with F32 or F64 storage");
        if (c->closure) return fail(c, VLBM_ERR_UNSUPPORTED, "a closure and open faces do not combine");
        if (c->slab && face / 2 == c->dim - 1)
            return fail(c, VLBM_ERR_UNSUPPORTED, "a slab's decomposed axis joins its neighbours: it cannot be open");
        const int64_t extent[3] = {c->dom[0].nx, c->dom[0].ny, c->dom[0].nz};
        if (extent[face / 2] < 3) return fail(c, VLBM_ERR_ARG, "an open axis needs at least 3 cells");
        if ((dirichlet_mask & ~0xFFu) != 0) return fail(c, VLBM_ERR_ARG, "Dirichlet mask has bits beyond the 8 fields");
        if (dirichlet_mask != 0 && !values) return fail(c, VLBM_ERR_ARG, "Dirichlet values missing");
        for (int k = 0; k < 8; ++k)
            if (((dirichlet_mask >> k) & 1u) && !std::isfinite(values[k]))
                return fail(c, VLBM_ERR_ARG, "Dirichlet value not finite");
    }
    drop_graphs(c);  // captured steps hold the previous faces
    c->face_kind[face] = kind;
    c->face_mask[face] = kind == VLBM_BC_EQUILIBRIUM ? dirichlet_mask : 0u;
    for (int k = 0; k < 8; ++k)
        c->face_vals[face][k] = (kind == VLBM_BC_EQUILIBRIUM && ((dirichlet_mask >> k) & 1u)) ? values[k] : 0.0;
    return VLBM_OK;
}

vlbm_status vlbm_porosity_from_distance(const float *phi_dev, int64_t n, double eps_h, float *d_dev, void *stream)
{
    if (!phi_dev || !d_dev || n < 0 || !(eps_h > 0.0)) return fail(nullptr, VLBM_ERR_ARG, "porosity: bad arguments");
    if (n == 0) return VLBM_OK;
    return porosity_from_distance(phi_dev, n, eps_h, d_dev, static_cast<cudaStream_t>(stream));
}

vlbm_status vlbm_check_bounded_wait(vlbm_ctx *c, int tries)
{
    if (!c) return VLBM_ERR_ARG;
    if (tries < 1 || tries > 65536) return fail(c, VLBM_ERR_ARG, "tries must be in 1 .. 65536");
    return wait_check(c, (uint32_t)tries);
}

vlbm_status vlbm_set_slab(vlbm_ctx *c, int on)
{
    if (!c) return VLBM_ERR_ARG;
    if (!on) {
        if (c->halo_pending) return fail(c, VLBM_ERR_STATE, "slab: unpack the last exchange first");
        c->slab = false;
        return VLBM_OK;
    }
    if (c->batched) return fail(c, VLBM_ERR_UNSUPPORTED, "batched contexts are not slabs");
    if (c->closure) return fail(c, VLBM_ERR_UNSUPPORTED, "a closure and a slab context do not combine");
    const int a = c->dim - 1;
    if (c->face_kind[2 * a] == VLBM_BC_EQUILIBRIUM || c->face_kind[2 * a + 1] == VLBM_BC_EQUILIBRIUM)
        return fail(c, VLBM_ERR_UNSUPPORTED, "a slab's decomposed axis joins its neighbours: it cannot be open");
    if (c->step & 1) return fail(c, VLBM_ERR_STATE, "slab: mark the context at an even step count");
    c->halo = halo_slots(c);
    c->slab = true;
    c->halo_pending = false;
    return VLBM_OK;
}

size_t vlbm_halo_bytes(const vlbm_ctx *c)
{
    if (!c || c->batched) return 0;
    const HaloSlots h = halo_slots(c);
    const Domain &d = c->dom[0];
    const int64_t layer = c->dim == 3 ? (int64_t)d.nx * d.ny : (int64_t)d.nx;
    return (size_t)h.n * (size_t)layer * c->elem;
}

vlbm_status vlbm_halo_pack(vlbm_ctx *c, void *lo_dev, void *hi_dev)
{
    vlbm::NvtxRange range("vlbm_halo_pack");
    if (!c || !lo_dev || !hi_dev) return VLBM_ERR_ARG;
    if (!c->slab) return fail(c, VLBM_ERR_STATE, "halo pack: not a slab context (vlbm_set_slab)");
    return halo_copy(c, lo_dev, hi_dev, true);
}

vlbm_status vlbm_halo_unpack(vlbm_ctx *c, const void *lo_dev, const void *hi_dev)
{
    vlbm::NvtxRange range("vlbm_halo_unpack");
    if (!c || !lo_dev || !hi_dev) return VLBM_ERR_ARG;
    if (!c->slab) return fail(c, VLBM_ERR_STATE, "halo unpack: not a slab context (vlbm_set_slab)");
    vlbm_status s = halo_copy(c, const_cast<void *>(lo_dev), const_cast<void *>(hi_dev), false);
    // open faces (on the axes the decomposition keeps whole) are filled once the slots their
    // Neumann moments read have arrived
    if (s == VLBM_OK && any_open_face(c)) s = open_fill(c, (int)(c->step & 1));
    if (s == VLBM_OK) c->halo_pending = false;
    return s;
}

vlbm_status vlbm_slabs_step(vlbm_ctx *const *slabs, int nslabs, int n)
{
    vlbm::NvtxRange range("vlbm_slabs_step");
    if (!slabs || nslabs < 1 || n < 0) return fail(nullptr, VLBM_ERR_ARG, "slabs step: bad arguments");
    vlbm_ctx *c0 = slabs[0];
    for (int r = 0; r < nslabs; ++r) {
        vlbm_ctx *c = slabs[r];
        if (!c) return fail(nullptr, VLBM_ERR_ARG, "slabs step: NULL context");
        for (int q = 0; q < r; ++q)
            if (slabs[q] == c) return fail(nullptr, VLBM_ERR_ARG, "slabs step: a context appears twice");
        if (!c->slab) return fail(c, VLBM_ERR_STATE, "slabs step: not a slab context (vlbm_set_slab)");
        if (c->model != c0->model || c->dim != c0->dim || c->storage != c0->storage || c->nlat != c0->nlat ||
            c->dom[0].nx != c0->dom[0].nx || (c->dim == 3 && c->dom[0].ny != c0->dom[0].ny))
            return fail(nullptr, VLBM_ERR_ARG, "slabs step: the slabs' models, storage or face layers differ");
        if (c->stream != c0->stream)
            return fail(nullptr, VLBM_ERR_ARG, "slabs step: the slabs must share one stream");
        if (c->step != c0->step) return fail(nullptr, VLBM_ERR_STATE, "slabs step: the slabs' step counts differ");
        vlbm_status s = slab_ready(c);
        if (s != VLBM_OK) return s;
        poll_flags(c);
        if (c->sticky != VLBM_OK) return c->sticky;
    }
    const size_t face = vlbm_halo_bytes(c0);
    if (nslabs > 1)
        for (int r = 0; r < nslabs; ++r)
            if (!slabs[r]->halo_buf) {
                slabs[r]->halo_buf = dev_alloc(slabs[r], 2 * face);
                if (!slabs[r]->halo_buf) return fail(slabs[r], VLBM_ERR_OOM, "slabs step: halo buffer allocation");
            }
    auto lo_of = [&](int r) { return static_cast<char *>(slabs[r]->halo_buf); };
    auto hi_of = [&](int r) { return static_cast<char *>(slabs[r]->halo_buf) + face; };
    for (int t = 0; t < n; ++t) {
        for (int r = 0; r < nslabs; ++r) {
            vlbm_ctx *c = slabs[r];
            vlbm_status s = launch_step(c, (int)(c->step & 1));
            if (s != VLBM_OK) return s;
            c->step += 1;
        }
        if (nslabs == 1) {  // one slab is the whole periodic domain: its wrap is the neighbour
            if (any_open_face(c0)) {
                vlbm_status s = open_fill(c0, (int)(c0->step & 1));
                if (s != VLBM_OK) return s;
            }
            continue;
        }
        for (int r = 0; r < nslabs; ++r) {
            vlbm_status s = halo_copy(slabs[r], lo_of(r), hi_of(r), true);
            if (s != VLBM_OK) return s;
        }
        // one stream: every pack is complete before the first unpack reads it
        const bool after_even = (c0->step & 1) != 0;
        for (int r = 0; r < nslabs; ++r) {
            const int below = (r + nslabs - 1) % nslabs, above = (r + 1) % nslabs;
            // after an even step a slab takes its lower neighbour's hi and its upper
            // neighbour's lo planes; after an odd step the upper's hi and the lower's lo
            const int hi_src = after_even ? below : above;
            const int lo_src = after_even ? above : below;
            vlbm_status s = halo_copy(slabs[r], lo_of(lo_src), hi_of(hi_src), false);
            if (s == VLBM_OK && any_open_face(slabs[r])) s = open_fill(slabs[r], (int)(slabs[r]->step & 1));
            if (s != VLBM_OK) return s;
        }
    }
    for (int r = 0; r < nslabs; ++r) schedule_check(slabs[r], n);
    return c0->sticky;
}

int vlbm_tile_shapes(const vlbm_ctx *c) { return (c && c->batched) ? batch_num_choices() : 0; }

vlbm_status vlbm_set_tile_shape(vlbm_ctx *c, int shape)
{
    if (!c) return VLBM_ERR_ARG;
    if (!c->batched || shape < 0 || shape >= batch_num_choices())
        return fail(c, VLBM_ERR_ARG, "no such tile shape");
    if (shape != c->tune_choice) drop_graphs(c);
    c->tune_choice = shape;
    return VLBM_OK;
}

int vlbm_nvar(const vlbm_ctx *c) { return c ? c->nvar : 0; }
int vlbm_slots_per_cell(const vlbm_ctx *c) { return c ? c->nslot : 0; }
int vlbm_num_domains(const vlbm_ctx *c) { return c ? (int)c->dom.size() : 0; }
int64_t vlbm_num_cells(const vlbm_ctx *c, int d)
{
    return (c && d >= 0 && d < (int)c->dom.size()) ? c->dom[d].ncell : 0;
}
int64_t vlbm_step_count(const vlbm_ctx *c) { return c ? c->step : 0; }
int64_t vlbm_launch_count(const vlbm_ctx *c) { return c ? c->launches : 0; }
size_t vlbm_population_bytes(const vlbm_ctx *c) { return c ? c->pop_bytes : 0; }
void *vlbm_stream(const vlbm_ctx *c) { return c ? (void *)c->stream : nullptr; }
const char *vlbm_last_error(const vlbm_ctx *c) { return c ? c->err.c_str() : g_err.c_str(); }

const char *vlbm_status_string(int s)
{
    switch (s) {
    case VLBM_OK: return "VLBM_OK";
    case VLBM_ERR_ARG: return "VLBM_ERR_ARG";
    case VLBM_ERR_UNSTABLE: return "VLBM_ERR_UNSTABLE";
    case VLBM_ERR_OOM: return "VLBM_ERR_OOM";
    case VLBM_ERR_CUDA: return "VLBM_ERR_CUDA";
    case VLBM_ERR_NONPHYSICAL: return "VLBM_ERR_NONPHYSICAL";
    case VLBM_ERR_TIMEOUT: return "VLBM_ERR_TIMEOUT";
    case VLBM_ERR_STATE: return "VLBM_ERR_STATE";
    case VLBM_ERR_UNSUPPORTED: return "VLBM_ERR_UNSUPPORTED";
    }
    return "unknown status";
}

void vlbm_destroy(vlbm_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    dev_free_all(c);
    if (c->h_flags) cudaFreeHost(c->h_flags);
    if (c->flag_event) cudaEventDestroy(c->flag_event);
    if (c->copy_stream) {
        cudaStreamSynchronize(c->copy_stream);
        cudaStreamDestroy(c->copy_stream);
    }
    for (int b = 0; b < 2; ++b) {
        if (c->ev_copy[b]) cudaEventDestroy(c->ev_copy[b]);
        if (c->ev_kern[b]) cudaEventDestroy(c->ev_kern[b]);
    }
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    cudaGetLastError();
    delete c;
}

}  // extern "C"
