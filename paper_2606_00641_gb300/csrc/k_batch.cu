// k_batch.cu -- many independent periodic 2-D ideal-MHD domains (D2Q5, F32)
// advanced by ONE kernel launch per time step.
//
// Every domain keeps its own block of the population buffer (AA in-place
// layout of vlbm_internal.cuh) and its own gamma and tau.  A tile table
// lists (domain, first cell) pairs; a CTA updates TX x R consecutive cells of
// one domain per tile.  The per-cell arithmetic is the same Eq. 2/3/4/9/12
// collision as the single-domain kernel (ideal_cell.cuh).  All domains share
// the step parity, so one launch per step keeps the AA pattern consistent.
//
// Tile shapes ("choices") differ in CTA width, cells per thread and whether
// the grid is persistent (a multiple of the SM count looping over tiles) or
// one CTA per tile; vlbm_autotune times them on the live batch.
#include <algorithm>

#include "ideal_cell.cuh"

namespace vlbm {
namespace {

struct BatchDomain {
    int nx, ny;
    int64_t ncell;
    int64_t offset;     // element offset of the domain's population block
    int64_t stride;
    float gm1;
    float omega[8];
    float src0[8], src1[8];
};

struct Choice {
    int tx, rows, persistent;
};
constexpr Choice kChoices[] = {{128, 1, 1}, {128, 1, 0}, {256, 1, 1}, {128, 2, 1}, {64, 4, 1}};
constexpr int kNumChoices = sizeof(kChoices) / sizeof(kChoices[0]);

template <bool ODD, int TX, int R>
__global__ void __launch_bounds__(TX, 640 / TX) k_batch_step(const int2 *__restrict__ tiles, int ntiles,
                                                   const BatchDomain *__restrict__ doms, float *pop,
                                                   unsigned *flags)
{
    constexpr int D = 2, Q = 5;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int2 tile = tiles[t];
        const BatchDomain *dm = doms + tile.x;
        // the domain's parameters, read once per tile into registers
        const int nx = __ldg(&dm->nx), ny = __ldg(&dm->ny);
        const int64_t ncell = __ldg(&dm->ncell);
        const int64_t stride = __ldg(&dm->stride);
        float *base = pop + __ldg(&dm->offset);
        const float gm1 = __ldg(&dm->gm1);
        float omega[8], src0[8], src1[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            omega[k] = __ldg(&dm->omega[k]);
            src0[k] = __ldg(&dm->src0[k]);
            src1[k] = __ldg(&dm->src1[k]);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int c32 = tile.y + r * TX + (int)threadIdx.x;  // per-domain cells < 2^31
            if (c32 >= ncell) continue;
            const int64_t cell = c32;
            const int y = c32 / nx;
            const int x = c32 - y * nx;
            const int64_t plane = (int64_t)nx * ny;
            int64_t nb[Q];
            nb[0] = cell;
            nb[1] = (x + 1 < nx) ? cell + 1 : cell + 1 - nx;
            nb[2] = (x > 0) ? cell - 1 : cell - 1 + nx;
            nb[3] = (y + 1 < ny) ? cell + nx : cell + nx - plane;
            nb[4] = (y > 0) ? cell - nx : cell - nx + plane;
            float f[8][Q];
#pragma unroll
            for (int k = 0; k < 8; ++k)
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const int j = ODD ? opp_axis(i) : i;
                    const int64_t at = ODD ? nb[opp_axis(i)] : cell;
                    f[k][i] = base[(int64_t)(k * Q + j) * stride + at];
                }
            ideal_collide<D, float>(f, gm1, omega, src0, src1, flags);
            // the stride is per-domain (not a kernel parameter): recompute the
            // store addresses rather than hold 40 offsets across the collision
            const int64_t sst = opaque(stride);
#pragma unroll
            for (int k = 0; k < 8; ++k)
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const int j = ODD ? i : opp_axis(i);
                    const int64_t at = ODD ? nb[i] : cell;
                    base[(int64_t)(k * Q + j) * sst + at] = f[k][i];
                }
        }
    }
}

template <int TX, int R> const void *kernel_for(bool odd)
{
    return odd ? (const void *)k_batch_step<true, TX, R> : (const void *)k_batch_step<false, TX, R>;
}

const void *kernel_of(int choice, bool odd)
{
    switch (choice) {
    case 0:
    case 1: return kernel_for<128, 1>(odd);
    case 2: return kernel_for<256, 1>(odd);
    case 3: return kernel_for<128, 2>(odd);
    default: return kernel_for<64, 4>(odd);
    }
}

}  // namespace

int batch_num_choices() { return kNumChoices; }

vlbm_status batch_prepare(vlbm_ctx *c)
{
    const int nd = (int)c->dom.size();
    std::vector<BatchDomain> bd(nd);
    for (int d = 0; d < nd; ++d) {
        const Domain &dm = c->dom[d];
        BatchDomain &b = bd[d];
        b.nx = dm.nx;
        b.ny = dm.ny;
        b.ncell = dm.ncell;
        b.offset = dm.offset;
        b.stride = dm.stride;
        b.gm1 = (float)(dm.gamma - 1.0);
        for (int k = 0; k < 8; ++k) {
            b.omega[k] = (float)(1.0 / dm.tau[k]);
            b.src0[k] = (float)(AxisSet<2>::w0 * dm.source[k]);
            b.src1[k] = (float)(AxisSet<2>::w1 * dm.source[k]);
        }
    }
    // tile tables for every choice, domains in decreasing size so that the
    // largest ones are scheduled first and small ones fill the tail
    std::vector<int> order(nd);
    for (int d = 0; d < nd; ++d) order[d] = d;
    std::sort(order.begin(), order.end(),
              [&](int a, int b) { return c->dom[a].ncell != c->dom[b].ncell ? c->dom[a].ncell > c->dom[b].ncell : a < b; });
    std::vector<std::vector<int2>> tables(kNumChoices);
    size_t table_bytes = 0;
    for (int ch = 0; ch < kNumChoices; ++ch) {
        const int64_t per = (int64_t)kChoices[ch].tx * kChoices[ch].rows;
        for (int d : order)
            for (int64_t c0 = 0; c0 < c->dom[d].ncell; c0 += per) {
                if (c0 > INT32_MAX) return fail(c, VLBM_ERR_ARG, "batched domain too large");
                tables[ch].push_back(make_int2(d, (int)c0));
            }
        table_bytes += tables[ch].size() * sizeof(int2);
    }
    const size_t dom_bytes = nd * sizeof(BatchDomain);
    void *blk = nullptr;
    if (c->params.alloc) {
        blk = c->params.alloc(dom_bytes + table_bytes + 256, (void *)c->stream, c->params.alloc_user);
    } else if (cudaMalloc(&blk, dom_bytes + table_bytes + 256) != cudaSuccess) {
        cudaGetLastError();
        blk = nullptr;
    }
    if (!blk) return fail(c, VLBM_ERR_OOM, "tile table allocation failed");
    c->owned.emplace_back(blk, dom_bytes + table_bytes + 256);
    char *p = static_cast<char *>(blk);
    c->d_dom = p;
    vlbm_status s = cuda_check(c, cudaMemcpyAsync(p, bd.data(), dom_bytes, cudaMemcpyHostToDevice, c->stream),
                               "domain table upload");
    size_t off = (dom_bytes + 15) / 16 * 16;
    c->tile_tables.clear();
    c->tile_counts.clear();
    for (int ch = 0; ch < kNumChoices && s == VLBM_OK; ++ch) {
        c->tile_tables.push_back(p + off);
        c->tile_counts.push_back((int)tables[ch].size());
        s = cuda_check(c, cudaMemcpyAsync(p + off, tables[ch].data(), tables[ch].size() * sizeof(int2),
                                          cudaMemcpyHostToDevice, c->stream),
                       "tile table upload");
        off += tables[ch].size() * sizeof(int2);
    }
    if (s != VLBM_OK) return s;
    // persistent grid sizes from the occupancy of each kernel
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    c->tile_grid.clear();
    for (int ch = 0; ch < kNumChoices; ++ch) {
        int per_sm = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel_of(ch, false), kChoices[ch].tx, 0);
        const int ntile = c->tile_counts[ch];
        int grid = kChoices[ch].persistent ? std::max(1, sms * std::max(per_sm, 1)) : ntile;
        c->tile_grid.push_back(std::min(grid, ntile));
    }
    return cuda_check(c, cudaGetLastError(), "batch prepare");
}

vlbm_status batch_step(vlbm_ctx *c, int parity, int choice)
{
    if (choice < 0 || choice >= kNumChoices) choice = 0;
    const int2 *tiles = static_cast<const int2 *>(c->tile_tables[choice]);
    int ntiles = c->tile_counts[choice];
    const BatchDomain *doms = static_cast<const BatchDomain *>(c->d_dom);
    float *pop = static_cast<float *>(c->pop);
    unsigned *flags = c->d_flags;
    void *args[] = {(void *)&tiles, (void *)&ntiles, (void *)&doms, (void *)&pop, (void *)&flags};
    const cudaError_t e = cudaLaunchKernel(kernel_of(choice, parity != 0), dim3(c->tile_grid[choice]),
                                           dim3(kChoices[choice].tx), args, 0, c->stream);
    c->launches++;
    return cuda_check(c, e, "batched step launch");
}

}  // namespace vlbm
