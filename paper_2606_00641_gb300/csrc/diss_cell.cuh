// diss_cell.cuh -- per-cell fluxes and sources of the dissipative MHD system
// with locally evolved gradients on D2Q5 (host and device).
//
// State q[20]: the eight fields of Eq. 12, then G_ab ~ tau_M d_a B_b at
// 8 + 3a + b and W_ab ~ tau_M d_a u_b at 14 + 3a + b (a in {x, y}, b in
// {x, y, z}).  The step kernel (k_diss.cu) relaxes towards the first-order
// equilibrium of these fluxes; the same source compiles for the host, where a
// test checks it state by state.
#pragma once

#include "vlbm_internal.cuh"

namespace vlbm {

constexpr int kDissLat = 20;
constexpr int kDissQ = 5;

template <class C> struct DissArgs {
    void *pop;
    int nx, ny;
    int64_t stride;
    C gm1;
    C omega[kDissLat];
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

}  // namespace vlbm
