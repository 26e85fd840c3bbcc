// k_resistive.cu -- resistive incompressible MHD channel: D3Q19 flow lattice
// plus three D3Q7 magnetic lattices, FP32, one fused kernel per step.
//
// Model (sec. 2.3 "Incompressible resistive MHD", read with a standard
// second-order flow equilibrium; sec. 2.4 "Static boundaries"):
//   rho = sum f_i,  m = sum f_i c_i + F/2,  u = m / rho,  B_b = sum_i g_bi
//   f_eq_i = w_i [rho + c_i.m/cs2 + (c_i c_i - cs2 I):(rho u u + |B|^2/2 I - B B)/(2 cs2^2)]
//   f*_i   = f_i + omega_f (f_eq_i - f_i)
//            + (1 - omega_f/2) w_i [(c_i - u)/cs2 + (c_i.u) c_i/cs2^2] . F    (Guo)
//   g_eq_bi = w_i (B_b + c_i . Phi_b / cs2_7),  Phi_{b,a} = u_a B_b - B_a u_b  (Eq. 3, 12)
//   g*_bi  = g_bi + omega_m (g_eq_bi - g_bi)
// Walls (rows y = 0 and ny - 1 when walls_y): halfway bounce-back for f;
// wall cells emit g*_bi = w_i b_wall_b (equilibrium of the applied field at
// rest) for the magnetic lattices.
//
// Slots: flow directions j = 0..18, then magnetic lattice b direction i at
// j = 19 + 7 b + i.  AA in-place pattern as in vlbm_internal.cuh; with walls,
// a flow population whose source (odd parity read) or destination (odd
// parity write) is a wall cell is taken from / put into the cell's own slot
// of the same direction -- the halfway bounce-back in AA form.
#include "vlbm_internal.cuh"

namespace vlbm {
namespace {

constexpr int kQf = 19;
constexpr int kSlots = 19 + 21;

// D3Q19 velocities in the ABI order; opposite of i is opp_axis(i).
__constant__ signed char c19[kQf][3] = {
    {0, 0, 0},   {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},   {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1},
    {-1, 0, 1},  {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

__host__ __device__ constexpr int cx19(int i)
{
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
           : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1
                                                                  : 0;
}
__host__ __device__ constexpr int cy19(int i)
{
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
           : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1
                                                                 : 0;
}
__host__ __device__ constexpr int cz19(int i)
{
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
           : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1
                                                                   : 0;
}
__host__ __device__ constexpr float w19(int i) { return i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f); }

struct Args {
    float *pop;
    int nx, ny, nz;
    int64_t stride;
    float omega_f, omega_m;
    float F[3];
    float guo;             // 1 - omega_f / 2
    float bw[3];           // wall field
    int walls_y;
    unsigned *flags;
};

// Offsets of x + c (periodic) from x along each axis, for c = -1, 0, +1.
struct Offsets {
    int64_t ox[3], oy[3], oz[3];
};

__device__ __forceinline__ Offsets offsets(int x, int y, int z, int nx, int ny, int nz)
{
    Offsets o;
    const int64_t row = nx, plane = (int64_t)nx * ny, vol = plane * nz;
    o.ox[0] = x > 0 ? -1 : nx - 1;
    o.ox[1] = 0;
    o.ox[2] = x + 1 < nx ? 1 : 1 - nx;
    o.oy[0] = y > 0 ? -row : plane - row;
    o.oy[1] = 0;
    o.oy[2] = y + 1 < ny ? row : row - plane;
    o.oz[0] = z > 0 ? -plane : vol - plane;
    o.oz[1] = 0;
    o.oz[2] = z + 1 < nz ? plane : plane - vol;
    return o;
}

__device__ __forceinline__ int64_t nbr(const Offsets &o, int64_t cell, int cx, int cy, int cz)
{
    return cell + o.ox[cx + 1] + o.oy[cy + 1] + o.oz[cz + 1];
}

__device__ __forceinline__ bool wall_row(int y, int ny, int walls) { return walls && (y == 0 || y == ny - 1); }

template <bool ODD>
__global__ void __launch_bounds__(kBlockX, 5) k_res_step(const Args a)
{
    const int x = blockIdx.x * kBlockX + threadIdx.x;
    if (x >= a.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const int64_t cell = x + (int64_t)a.nx * (y + (int64_t)a.ny * z);
    const Offsets o = offsets(x, y, z, a.nx, a.ny, a.nz);
    float *pop = a.pop;
    const int64_t S = a.stride;

    if (wall_row(y, a.ny, a.walls_y)) {
        // magnetic wall: emit the equilibrium of b_wall at rest
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int i = 0; i < 7; ++i) {
                const float v = (i == 0 ? 0.25f : 0.125f) * a.bw[b];
                const int j = ODD ? i : opp_axis(i);
                const int64_t at = ODD ? nbr(o, cell, cx19(i), cy19(i), cz19(i)) : cell;
                pop[(int64_t)(19 + 7 * b + j) * S + at] = v;
            }
        return;
    }
    const bool wall_lo = a.walls_y && y == 1;            // y - 1 is a wall row
    const bool wall_hi = a.walls_y && y == a.ny - 2;     // y + 1 is a wall row

    // ---- load ----
    float f[kQf], g[3][7];
#pragma unroll
    for (int i = 0; i < kQf; ++i) {
        int64_t at;
        int j;
        if (!ODD) {
            j = i;
            at = cell;
        } else {
            // source x - c_i; a wall source means the population bounced back
            const bool from_wall = (cy19(i) > 0 && wall_lo) || (cy19(i) < 0 && wall_hi);
            j = from_wall ? i : opp_axis(i);
            at = from_wall ? cell : nbr(o, cell, -cx19(i), -cy19(i), -cz19(i));
        }
        f[i] = pop[(int64_t)j * S + at];
    }
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int i = 0; i < 7; ++i) {
            const int j = ODD ? opp_axis(i) : i;
            const int64_t at = ODD ? nbr(o, cell, -cx19(i), -cy19(i), -cz19(i)) : cell;
            g[b][i] = pop[(int64_t)(19 + 7 * b + j) * S + at];
        }

    // ---- moments ----
    float rho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < kQf; ++i) {
        rho += f[i];
        if (cx19(i)) jx += cx19(i) * f[i];
        if (cy19(i)) jy += cy19(i) * f[i];
        if (cz19(i)) jz += cz19(i) * f[i];
    }
    const float m[3] = {jx + 0.5f * a.F[0], jy + 0.5f * a.F[1], jz + 0.5f * a.F[2]};
    const float ir = 1.0f / rho;
    const float u[3] = {m[0] * ir, m[1] * ir, m[2] * ir};
    float B[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        float s = g[b][0];
#pragma unroll
        for (int i = 1; i < 7; ++i) s += g[b][i];
        B[b] = s;
    }
    if (!(rho > 0.f)) atomicOr(a.flags, kFlagNonPhysical);
    const float B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    const float u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const float uF = u[0] * a.F[0] + u[1] * a.F[1] + u[2] * a.F[2];

    // ---- flow collision (cs2 = 1/3) ----
    const float om = a.omega_f, omc = 1.f - om;
#pragma unroll
    for (int i = 0; i < kQf; ++i) {
        const float cu = cx19(i) * u[0] + cy19(i) * u[1] + cz19(i) * u[2];
        const float cm = cx19(i) * m[0] + cy19(i) * m[1] + cz19(i) * m[2];
        const float cB = cx19(i) * B[0] + cy19(i) * B[1] + cz19(i) * B[2];
        const float cF = cx19(i) * a.F[0] + cy19(i) * a.F[1] + cz19(i) * a.F[2];
        const float c2 = float(cx19(i) * cx19(i) + cy19(i) * cy19(i) + cz19(i) * cz19(i));
        // (c c - cs2 I) : (rho u u + B^2/2 I - B B)
        const float second = rho * (cu * cu - u2 * (1.f / 3.f)) + 0.5f * B2 * (c2 - 1.f) - (cB * cB - B2 * (1.f / 3.f));
        const float feq = w19(i) * (rho + 3.f * cm + 4.5f * second);
        const float force = a.guo * w19(i) * (3.f * (cF - uF) + 9.f * cu * cF);
        f[i] = omc * f[i] + om * feq + force;
    }
    // ---- magnetic collision (D3Q7, cs2 = 1/4, w_moving/cs2 = 1/2) ----
    const float omm = a.omega_m, ommc = 1.f - omm;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const float A0 = omm * 0.25f * B[b];
        const float A1 = omm * 0.125f * B[b];
        g[b][0] = ommc * g[b][0] + A0;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const float phi = (ax == b) ? 0.f : u[ax] * B[b] - B[ax] * u[b];
            const float bv = 0.5f * omm * phi;
            g[b][2 * ax + 1] = ommc * g[b][2 * ax + 1] + A1 + bv;
            g[b][2 * ax + 2] = ommc * g[b][2 * ax + 2] + A1 - bv;
        }
    }

    // ---- store ---- (addresses recomputed from an opaque stride, not held)
    const int64_t Ss = opaque(S);
#pragma unroll
    for (int i = 0; i < kQf; ++i) {
        int64_t at;
        int j;
        if (!ODD) {
            j = opp_axis(i);
            at = cell;
        } else {
            // destination x + c_i; a wall destination bounces back into the own slot
            const bool to_wall = (cy19(i) > 0 && wall_hi) || (cy19(i) < 0 && wall_lo);
            j = to_wall ? opp_axis(i) : i;
            at = to_wall ? cell : nbr(o, cell, cx19(i), cy19(i), cz19(i));
        }
        pop[(int64_t)j * Ss + at] = f[i];
    }
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int i = 0; i < 7; ++i) {
            const int j = ODD ? i : opp_axis(i);
            const int64_t at = ODD ? nbr(o, cell, cx19(i), cy19(i), cz19(i)) : cell;
            pop[(int64_t)(19 + 7 * b + j) * Ss + at] = g[b][i];
        }
}

// f = f_eq(rho, m - F/2, B), g = g_eq(B, u = m/rho) at parity 0, in double.
struct InitArgs {
    float *pop;
    int64_t stride, c0, count, qstride;
    double F[3];
};

__global__ void k_res_init(const InitArgs a, const double *__restrict__ Qin)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= a.count) return;
    const int64_t cell = a.c0 + t;
    const double rho = Qin[t];
    double m[3], j[3], B[3], u[3];
    for (int ax = 0; ax < 3; ++ax) {
        m[ax] = Qin[(1 + ax) * a.qstride + t];
        B[ax] = Qin[(4 + ax) * a.qstride + t];
        j[ax] = m[ax] - 0.5 * a.F[ax];
        u[ax] = m[ax] / rho;
    }
    const double v[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
    const double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const double B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    for (int i = 0; i < kQf; ++i) {
        const double cv = c19[i][0] * v[0] + c19[i][1] * v[1] + c19[i][2] * v[2];
        const double cj = c19[i][0] * j[0] + c19[i][1] * j[1] + c19[i][2] * j[2];
        const double cB = c19[i][0] * B[0] + c19[i][1] * B[1] + c19[i][2] * B[2];
        const double c2 = c19[i][0] * c19[i][0] + c19[i][1] * c19[i][1] + c19[i][2] * c19[i][2];
        const double second = rho * (cv * cv - v2 / 3.0) + 0.5 * B2 * (c2 - 1.0) - (cB * cB - B2 / 3.0);
        const double w = i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
        a.pop[(int64_t)i * a.stride + cell] = (float)(w * (rho + 3.0 * cj + 4.5 * second));
    }
    for (int b = 0; b < 3; ++b)
        for (int i = 0; i < 7; ++i) {
            double cphi = 0.0;
            if (i > 0) {
                const int ax = (i - 1) / 2;
                const double s = (i & 1) ? 1.0 : -1.0;
                cphi = (ax == b) ? 0.0 : s * (u[ax] * B[b] - B[ax] * u[b]);
            }
            const double w = i == 0 ? 0.25 : 0.125;
            a.pop[(int64_t)(19 + 7 * b + i) * a.stride + cell] = (float)(w * (B[b] + 4.0 * cphi));
        }
}

struct ReadArgs {
    const float *pop;
    int nx, ny, nz;
    int64_t stride;
    int parity;
    int walls_y;
    double F[3], bw[3];
};

__device__ __forceinline__ void cell_xyz(int64_t cell, int nx, int ny, int &x, int &y, int &z)
{
    x = (int)(cell % nx);
    const int64_t r = cell / nx;
    y = (int)(r % ny);
    z = (int)(r / ny);
}

// logical pre-collision population of slot j (0..39) at a fluid cell
__device__ double res_logical(const ReadArgs &a, int64_t cell, int x, int y, int z, int jslot)
{
    const Offsets o = offsets(x, y, z, a.nx, a.ny, a.nz);
    const bool wall_lo = a.walls_y && y == 1, wall_hi = a.walls_y && y == a.ny - 2;
    if (jslot < kQf) {
        const int i = jslot;
        if (!a.parity) return a.pop[(int64_t)i * a.stride + cell];
        const bool from_wall = (cy19(i) > 0 && wall_lo) || (cy19(i) < 0 && wall_hi);
        if (from_wall) return a.pop[(int64_t)i * a.stride + cell];
        return a.pop[(int64_t)opp_axis(i) * a.stride + nbr(o, cell, -cx19(i), -cy19(i), -cz19(i))];
    }
    const int b = (jslot - kQf) / 7, i = (jslot - kQf) % 7;
    if (!a.parity) return a.pop[(int64_t)(19 + 7 * b + i) * a.stride + cell];
    return a.pop[(int64_t)(19 + 7 * b + opp_axis(i)) * a.stride + nbr(o, cell, -cx19(i), -cy19(i), -cz19(i))];
}

__device__ void res_cell_moments(const ReadArgs &a, int64_t cell, double *q)
{
    int x, y, z;
    cell_xyz(cell, a.nx, a.ny, x, y, z);
    if (wall_row(y, a.ny, a.walls_y)) {
        q[0] = 1.0;
        for (int ax = 0; ax < 3; ++ax) {
            q[1 + ax] = 0.0;
            q[4 + ax] = a.bw[ax];
        }
        return;
    }
    double rho = 0, m[3] = {0, 0, 0}, B[3] = {0, 0, 0};
    for (int i = 0; i < kQf; ++i) {
        const double v = res_logical(a, cell, x, y, z, i);
        rho += v;
        m[0] += c19[i][0] * v;
        m[1] += c19[i][1] * v;
        m[2] += c19[i][2] * v;
    }
    for (int b = 0; b < 3; ++b)
        for (int i = 0; i < 7; ++i) B[b] += res_logical(a, cell, x, y, z, kQf + 7 * b + i);
    q[0] = rho;
    for (int ax = 0; ax < 3; ++ax) {
        q[1 + ax] = m[ax] + 0.5 * a.F[ax];
        q[4 + ax] = B[ax];
    }
}

__global__ void k_res_moments(const ReadArgs a, int64_t c0, int64_t count, int64_t ostride, double *__restrict__ out)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= count) return;
    double q[7];
    res_cell_moments(a, c0 + t, q);
    for (int v = 0; v < 7; ++v) out[v * ostride + t] = q[v];
}

__global__ void k_res_gather(const ReadArgs a, const int64_t *__restrict__ cells, int n, double *__restrict__ out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int64_t cell = cells[t];
    int x, y, z;
    cell_xyz(cell, a.nx, a.ny, x, y, z);
    for (int j = 0; j < kSlots; ++j) out[(int64_t)t * kSlots + j] = res_logical(a, cell, x, y, z, j);
}

__global__ void __launch_bounds__(kReduceThreads) k_res_partials(const ReadArgs a, int64_t ncell,
                                                                 double *__restrict__ partials)
{
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < ncell;
         cell += (int64_t)gridDim.x * blockDim.x) {
        double q[7];
        res_cell_moments(a, cell, q);
        for (int v = 0; v < 7; ++v) acc[v] += q[v];
    }
    __shared__ double red[kReduceThreads / 32][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int v = 0; v < 7; ++v) {
        double s = acc[v];
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (lane == 0) red[warp][v] = s;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        double s = 0.0;
        if (threadIdx.x < 7)
            for (int w = 0; w < kReduceThreads / 32; ++w) s += red[w][threadIdx.x];
        partials[(int64_t)blockIdx.x * 8 + threadIdx.x] = s;
    }
}

Args make_args(vlbm_ctx *c)
{
    const Domain &d = c->dom[0];
    Args a{};
    a.pop = static_cast<float *>(c->pop);
    a.nx = d.nx;
    a.ny = d.ny;
    a.nz = d.nz;
    a.stride = d.stride;
    a.omega_f = (float)(1.0 / d.tau[0]);
    a.omega_m = (float)(1.0 / d.tau[1]);
    for (int ax = 0; ax < 3; ++ax) {
        a.F[ax] = (float)d.force[ax];
        a.bw[ax] = (float)d.b_wall[ax];
    }
    a.guo = (float)(1.0 - 0.5 / d.tau[0]);
    a.walls_y = d.walls_y;
    a.flags = c->d_flags;
    return a;
}

ReadArgs make_read(vlbm_ctx *c, int di)
{
    const Domain &d = c->dom[di];
    ReadArgs a{};
    a.pop = static_cast<const float *>(c->pop) + d.offset;
    a.nx = d.nx;
    a.ny = d.ny;
    a.nz = d.nz;
    a.stride = d.stride;
    a.parity = (int)(c->step & 1);
    a.walls_y = d.walls_y;
    for (int ax = 0; ax < 3; ++ax) {
        a.F[ax] = d.force[ax];
        a.bw[ax] = d.b_wall[ax];
    }
    return a;
}

}  // namespace

vlbm_status resistive_step(vlbm_ctx *c, int parity)
{
    const Domain &d = c->dom[0];
    const Args a = make_args(c);
    const dim3 grid((unsigned)((d.nx + kBlockX - 1) / kBlockX), (unsigned)d.ny, (unsigned)d.nz);
    if (parity)
        k_res_step<true><<<grid, kBlockX, 0, c->stream>>>(a);
    else
        k_res_step<false><<<grid, kBlockX, 0, c->stream>>>(a);
    c->launches++;
    return cuda_check(c, cudaGetLastError(), "resistive step launch");
}

vlbm_status resistive_init_range(vlbm_ctx *c, int di, const double *Q, int64_t c0, int64_t n, int64_t qstride)
{
    const Domain &d = c->dom[di];
    InitArgs a{};
    a.pop = static_cast<float *>(c->pop) + d.offset;
    a.stride = d.stride;
    a.c0 = c0;
    a.count = n;
    a.qstride = qstride;
    for (int ax = 0; ax < 3; ++ax) a.F[ax] = d.force[ax];
    k_res_init<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(a, Q);
    c->launches++;
    return cuda_check(c, cudaGetLastError(), "resistive init launch");
}

vlbm_status resistive_init(vlbm_ctx *c, int d, const double *Q_dev)
{
    const int64_t N = c->dom[d].ncell;
    return resistive_init_range(c, d, Q_dev, 0, N, N);
}

vlbm_status resistive_moments_range(vlbm_ctx *c, int di, double *out, int64_t c0, int64_t n, int64_t ostride)
{
    k_res_moments<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(make_read(c, di), c0, n, ostride, out);
    c->launches++;
    return cuda_check(c, cudaGetLastError(), "resistive moments launch");
}

vlbm_status resistive_moments(vlbm_ctx *c, int d, double *Q_dev)
{
    const int64_t N = c->dom[d].ncell;
    return resistive_moments_range(c, d, Q_dev, 0, N, N);
}

vlbm_status resistive_gather(vlbm_ctx *c, int di, const int64_t *cells_dev, int n, double *out_dev)
{
    k_res_gather<<<(unsigned)((n + 127) / 128), 128, 0, c->stream>>>(make_read(c, di), cells_dev, n, out_dev);
    c->launches++;
    return cuda_check(c, cudaGetLastError(), "resistive gather launch");
}

vlbm_status resistive_sums(vlbm_ctx *c, int di, double *sums_dev)
{
    k_res_partials<<<kReduceBlocks, kReduceThreads, 0, c->stream>>>(make_read(c, di), c->dom[di].ncell,
                                                                    c->d_partials);
    c->launches++;
    vlbm_status s = cuda_check(c, cudaGetLastError(), "resistive partial sums launch");
    if (s != VLBM_OK) return s;
    return finish_sums(c, 7, sums_dev);
}

}  // namespace vlbm
