// k_slab.cu -- slab decomposition of one periodic domain: the population
// halo of a slab's two faces.
//
// A global domain, periodic along its last axis a (z in 3-D, y in 2-D), is cut
// into slabs of whole layers; each slab is an ordinary context whose kernels
// wrap axis a inside the slab.  With the AA pattern (vlbm_internal.cuh) the
// populations that wrap are exactly these slot planes:
//   lo face (the slab's first layer): the slots of the directions with
//     c_a = +1 -- at odd parity the last layer's cells read and write them;
//   hi face (the slab's last layer):  the slots of the directions with
//     c_a = -1 -- at odd parity the first layer's cells read and write them.
// In the decomposed domain those planes belong to the neighbouring slabs, so
// after every step they move between slabs (the host routes them, see
// vlbm_halo_pack in include/vlbm.h): after an even step each slab's planes are
// replaced by its lower neighbour's hi planes and its upper neighbour's lo
// planes (the values its boundary cells read in the odd step), after an odd
// step by its upper neighbour's hi planes and its lower neighbour's lo planes
// (the values the neighbours' boundary cells wrote there for it).  Every
// element moves unchanged, so a decomposed run equals the single domain bit
// for bit.
//
// The kernel below copies those planes between the population buffer and a
// contiguous message per face, [slot list index][cell of the face layer];
// one launch covers both faces.  HBM-bound and small: 2 x (slots per face) x
// (cells per layer) elements each way.
#include "vlbm_internal.cuh"

namespace vlbm {
namespace {

template <class E>
__global__ void k_halo_copy(E *__restrict__ pop, int64_t stride, int64_t layer, int64_t hi_first, int nx,
                            const __grid_constant__ HaloSlots hs, E *__restrict__ lo, E *__restrict__ hi,
                            int pack)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= layer) return;
    const int s = blockIdx.y;
    const bool high = blockIdx.z != 0;
    const int keep = high ? hs.hi_keep[s] : hs.lo_keep[s];
    if (keep >= 0 && t / nx == keep) return;  // a wall-adjacent row's own bounce-back slot
    const int slot = high ? hs.hi[s] : hs.lo[s];
    E *plane = pop + (int64_t)slot * stride + (high ? hi_first : 0);
    E *msg = (high ? hi : lo) + (int64_t)s * layer;
    if (pack) msg[t] = plane[t];
    else plane[t] = msg[t];
}

template <class E> vlbm_status launch(vlbm_ctx *c, void *lo, void *hi, bool pack)
{
    const Domain &d = c->dom[0];
    const int64_t layer = c->dim == 3 ? (int64_t)d.nx * d.ny : (int64_t)d.nx;
    const int64_t nlayers = c->dim == 3 ? d.nz : d.ny;
    const int threads = 256;
    const dim3 grid((unsigned)((layer + threads - 1) / threads), (unsigned)c->halo.n, 2u);
    k_halo_copy<E><<<grid, threads, 0, c->stream>>>(static_cast<E *>(c->pop), d.stride, layer,
                                                    (nlayers - 1) * layer, d.nx, c->halo, static_cast<E *>(lo),
                                                    static_cast<E *>(hi), pack ? 1 : 0);
    c->launches++;
    return cuda_check(c, cudaGetLastError(), pack ? "halo pack launch" : "halo unpack launch");
}

}  // namespace

HaloSlots halo_slots(const vlbm_ctx *c)
{
    HaloSlots h{};
    for (int s = 0; s < kMaxHaloSlots; ++s) h.lo_keep[s] = h.hi_keep[s] = -1;
    if (c->model == VLBM_RESISTIVE) {
        // D3Q19 directions with c_z = +1 and -1 (ABI order), then the magnetic
        // lattices' +z / -z slots
        const int up[5] = {5, 11, 14, 15, 18}, dn[5] = {6, 12, 13, 16, 17};
        for (int s = 0; s < 5; ++s) {
            h.lo[s] = up[s];
            h.hi[s] = dn[s];
        }
        if (c->dom[0].walls_y) {
            // Halfway bounce-back in AA form keeps, in the row next to each wall, the
            // cell's own populations in the slots of the directions that point into
            // and out of the wall (y = 1: 15 (0,1,1) and 17 (0,1,-1); y = ny-2: 16
            // (0,-1,-1) and 18 (0,-1,1)); nothing streams into those entries from
            // another cell (the source would be the wall row), so they stay put.
            const int ny = c->dom[0].ny;
            h.lo_keep[3] = 1;       // lo[3] = 15
            h.lo_keep[4] = ny - 2;  // lo[4] = 18
            h.hi_keep[3] = ny - 2;  // hi[3] = 16
            h.hi_keep[4] = 1;       // hi[4] = 17
        }
        for (int b = 0; b < 3; ++b) {
            h.lo[5 + b] = 19 + 7 * b + 5;
            h.hi[5 + b] = 19 + 7 * b + 6;
        }
        h.n = 8;
        return h;
    }
    const int a = c->dim - 1;  // slab axis: z in 3-D, y in 2-D
    for (int k = 0; k < c->nlat; ++k) {
        h.lo[k] = k * c->q + 2 * a + 1;  // +e_a
        h.hi[k] = k * c->q + 2 * a + 2;  // -e_a
    }
    h.n = c->nlat;
    return h;
}

vlbm_status halo_copy(vlbm_ctx *c, void *lo, void *hi, bool pack)
{
    switch (c->elem) {
    case 8: return launch<unsigned long long>(c, lo, hi, pack);
    case 4: return launch<unsigned>(c, lo, hi, pack);
    case 2: return launch<unsigned short>(c, lo, hi, pack);
    }
    return fail(c, VLBM_ERR_UNSUPPORTED, "halo: unknown element size");
}

}  // namespace vlbm
