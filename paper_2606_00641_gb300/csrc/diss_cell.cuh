// diss_cell.cuh -- per-cell fluxes and sources of the dissipative MHD system
// with locally evolved gradients (host and device).
//
// 2-D (D2Q5), state q[20]: the eight fields of Eq. 12, then G_ab ~ tau_M d_a B_b
// at 8 + 3a + b and W_ab ~ tau_M d_a u_b at 14 + 3a + b (a in {x, y}, b in
// {x, y, z}).  3-D (D3Q7), state q[26]: G_ab at 8 + 3a + b and W_ab at
// 17 + 3a + b with a, b in {x, y, z}.  The step kernels (k_diss.cu) relax
// towards the first-order equilibrium of these fluxes; the same source
// compiles for the host, where a test checks it state by state.
#pragma once

#include "vlbm_internal.cuh"

namespace vlbm {

constexpr int kDissLat = 20;
constexpr int kDissQ = 5;
constexpr int kDiss3Lat = 26;  // 3-D: 8 + 9 (G) + 9 (W) lattices of D3Q7
constexpr int kDiss3Q = 7;

template <class C> struct DissArgs {
    void *pop;
    int nx, ny, nz;
    int64_t stride;
    C gm1;
    C omega[kDiss3Lat];  // 2-D uses the first 20
    C nu, eta0, inv_jc2, inv_tau_m;
    int powell;
    unsigned *flags;
};

// Fluxes phi[k][c] along the two lattice axes and sources S[k] of one state.
template <class C>
VLBM_HD __forceinline__ void diss_flux_source(const C (&q)[kDissLat], const DissArgs<C> &a, C (&phi)[kDissLat][2],
                                              C (&S)[kDissLat], unsigned *flags)
{
    const C rho = q[0];
    const C ir = C(1) / rho;
    const C m[3] = {q[1], q[2], q[3]};
    const C u[3] = {m[0] * ir, m[1] * ir, m[2] * ir};
    const C E = q[4];
    const C B[3] = {q[5], q[6], q[7]};
    const C B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    const C mu = m[0] * u[0] + m[1] * u[1] + m[2] * u[2];
    const C uB = u[0] * B[0] + u[1] * B[1] + u[2] * B[2];
    const C p = a.gm1 * (E - C(0.5) * mu - C(0.5) * B2);  // Eq. 9
    const C pt = p + C(0.5) * B2;
    if (!(rho > C(0)) || !(p > C(0))) raise_flag(flags, kFlagNonPhysical);

    // gradients from the evolved tensors (rows a = x, y; the z row is zero in 2-D)
    C dB[2][3], du[2][3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            dB[r][b] = q[8 + 3 * r + b] * a.inv_tau_m;
            du[r][b] = q[14 + 3 * r + b] * a.inv_tau_m;
        }
    // viscous stress rows c = x, y: rho nu (d_c u_b + d_b u_c), d_z = 0
    const C rn = rho * a.nu;
    C vs[2][3];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b) vs[c][b] = rn * (du[c][b] + (b < 2 ? du[b][c] : C(0)));
    // current j = curl B (d_z = 0) and the resistivity eta(j)
    const C j[3] = {dB[1][2], -dB[0][2], dB[0][1] - dB[1][0]};
    const C jj = j[0] * j[0] + j[1] * j[1] + j[2] * j[2];
    const C eta = a.eta0 * (C(1) + jj * a.inv_jc2);
    const C jxB[2] = {j[1] * B[2] - j[2] * B[1], j[2] * B[0] - j[0] * B[2]};
    const C Ept = E + pt;

#pragma unroll
    for (int c = 0; c < 2; ++c) {
        phi[0][c] = m[c];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            phi[1 + b][c] = m[c] * u[b] - B[c] * B[b] + (b == c ? pt : C(0)) - vs[c][b];
            // u_c B_b - B_c u_b vanishes for b = c; written as zero so that no
            // fused multiply-add leaves a rounding residue there
            phi[5 + b][c] = (b == c ? C(0) : u[c] * B[b] - B[c] * u[b]) - eta * dB[c][b];
        }
        phi[4][c] = Ept * u[c] - B[c] * uB - (u[0] * vs[c][0] + u[1] * vs[c][1] + u[2] * vs[c][2]) + eta * jxB[c];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                phi[8 + 3 * r + b][c] = q[8 + 3 * r + b] * u[c] - (r == c ? B[b] : C(0));
                phi[14 + 3 * r + b][c] = q[14 + 3 * r + b] * u[c] - (r == c ? u[b] : C(0));
            }
    }

#pragma unroll
    for (int k = 0; k < 8; ++k) S[k] = C(0);
#pragma unroll
    for (int k = 8; k < kDissLat; ++k) S[k] = -q[k] * a.inv_tau_m;
    if (a.powell) {
        const C ndiv = -(q[8] + q[12]) * a.inv_tau_m;  // -(G_xx + G_yy) / tau_M
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            S[1 + b] = ndiv * B[b];
            S[5 + b] = ndiv * u[b];
        }
        S[4] = ndiv * uB;
    }
}

// ---------------------------------------------------------------------------
// 3-D: the quantities every one of the 26 fluxes is built from, so that the
// step kernel can form lattice k's flux when it relaxes lattice k instead of
// holding all 78 flux components.
// ---------------------------------------------------------------------------
template <class C> struct Diss3State {
    C m[3], u[3], B[3];
    C pt, Ept, uB;
    C vs[3][3];   // viscous stress rho nu (d_c u_b + d_b u_c)
    C dB[3][3];   // d_a B_b = G_ab / tau_M
    C eta;        // eta0 (1 + |j|^2 / j_c^2)
    C jxB[3];     // (curl B) x B
    C ndiv;       // Powell: -(div B) = -(G_xx + G_yy + G_zz) / tau_M; 0 without
};

template <class C>
VLBM_HD __forceinline__ Diss3State<C> diss3_state(const C (&q)[kDiss3Lat], const DissArgs<C> &a, unsigned *flags)
{
    Diss3State<C> s;
    const C rho = q[0];
    const C ir = C(1) / rho;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        s.m[b] = q[1 + b];
        s.u[b] = q[1 + b] * ir;
        s.B[b] = q[5 + b];
    }
    const C E = q[4];
    const C B2 = s.B[0] * s.B[0] + s.B[1] * s.B[1] + s.B[2] * s.B[2];
    const C mu = s.m[0] * s.u[0] + s.m[1] * s.u[1] + s.m[2] * s.u[2];
    s.uB = s.u[0] * s.B[0] + s.u[1] * s.B[1] + s.u[2] * s.B[2];
    const C p = a.gm1 * (E - C(0.5) * mu - C(0.5) * B2);  // Eq. 9
    s.pt = p + C(0.5) * B2;
    s.Ept = E + s.pt;
    if (!(rho > C(0)) || !(p > C(0))) raise_flag(flags, kFlagNonPhysical);
    C du[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            s.dB[r][b] = q[8 + 3 * r + b] * a.inv_tau_m;
            du[r][b] = q[17 + 3 * r + b] * a.inv_tau_m;
        }
    const C rn = rho * a.nu;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b) s.vs[c][b] = rn * (du[c][b] + du[b][c]);
    const C j[3] = {s.dB[1][2] - s.dB[2][1], s.dB[2][0] - s.dB[0][2], s.dB[0][1] - s.dB[1][0]};
    const C jj = j[0] * j[0] + j[1] * j[1] + j[2] * j[2];
    s.eta = a.eta0 * (C(1) + jj * a.inv_jc2);
    s.jxB[0] = j[1] * s.B[2] - j[2] * s.B[1];
    s.jxB[1] = j[2] * s.B[0] - j[0] * s.B[2];
    s.jxB[2] = j[0] * s.B[1] - j[1] * s.B[0];
    s.ndiv = a.powell ? -(q[8] + q[12] + q[16]) * a.inv_tau_m : C(0);
    return s;
}

// Flux of lattice k along x, y, z (the full system of sec. 2.3 with the
// gradients of sec. 2.2.1; k is a compile-time constant after unrolling).
template <class C>
VLBM_HD __forceinline__ void diss3_flux(int k, const C (&q)[kDiss3Lat], const Diss3State<C> &s, C (&phi)[3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        C v;
        if (k == 0) {
            v = s.m[c];
        } else if (k <= 3) {
            const int b = k - 1;
            v = s.m[c] * s.u[b] - s.B[c] * s.B[b] + (b == c ? s.pt : C(0)) - s.vs[c][b];
        } else if (k == 4) {
            v = s.Ept * s.u[c] - s.B[c] * s.uB - (s.u[0] * s.vs[0][c] + s.u[1] * s.vs[1][c] + s.u[2] * s.vs[2][c]) +
                s.eta * s.jxB[c];
        } else if (k <= 7) {
            const int b = k - 5;
            // u_c B_b - B_c u_b vanishes for b = c; written as zero so that no
            // fused multiply-add leaves a rounding residue there
            v = (b == c ? C(0) : s.u[c] * s.B[b] - s.B[c] * s.u[b]) - s.eta * s.dB[c][b];
        } else if (k < 17) {
            const int r = (k - 8) / 3, b = (k - 8) % 3;
            v = q[k] * s.u[c] - (r == c ? s.B[b] : C(0));
        } else {
            const int r = (k - 17) / 3, b = (k - 17) % 3;
            v = q[k] * s.u[c] - (r == c ? s.u[b] : C(0));
        }
        phi[c] = v;
    }
}

// Source of lattice k: relaxation -G/tau_M, -W/tau_M of the gradient lattices,
// Powell's -(div B)(0, B, u.B, u) on the MHD lattices (zero without it).
template <class C>
VLBM_HD __forceinline__ C diss3_source(int k, const C (&q)[kDiss3Lat], const Diss3State<C> &s, C inv_tau_m)
{
    if (k >= 8) return -q[k] * inv_tau_m;
    if (k == 0) return C(0);
    if (k <= 3) return s.ndiv * s.B[k - 1];
    if (k == 4) return s.ndiv * s.uB;
    return s.ndiv * s.u[k - 5];
}

}  // namespace vlbm
