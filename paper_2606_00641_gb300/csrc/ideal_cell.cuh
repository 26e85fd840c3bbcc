// ideal_cell.cuh -- per-cell arithmetic of the ideal-MHD VLBM step (host and device).
//
// Given the 8 x q pre-collision populations of one cell, computes
//   moments          Q_k = sum_i f_ki                                (Eq. 4)
//   EOS              p = (gamma - 1)(e_tot - rho|u|^2/2 - |B|^2/2)    (Eq. 9)
//   fluxes           Phi_k of ideal MHD along the lattice axes       (Eq. 12)
//   BGK + source     f*_ki = f_ki + omega_k (f_eq_ki - f_ki) + w_i S_k
//                    with f_eq_ki = w_i (Q_k + c_i . Phi_k / cs^2)  (Eq. 2, 3)
// in place.  Directions: 0 rest, 2a+1 = +e_a, 2a+2 = -e_a; w_moving/cs^2 = 1/2.
#pragma once

#include "vlbm_internal.cuh"

namespace vlbm {

// Gas pressure of Eq. 9 in FP64 from the FP32 sums G_k of a cell's stored
// deviations: Q_k = r_k + s_k G_k, refscale = r_0..7 then s_0..7 (device).
static VLBM_HD __noinline__ double pressure_fp64(float G0, float G1, float G2, float G3, float G4, float G5, float G6,
                                            float G7, const double *__restrict__ refscale, double gm1)
{
    const float G[8] = {G0, G1, G2, G3, G4, G5, G6, G7};
    double q[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) q[k] = fma((double)G[k], ro_load(refscale + 8 + k), ro_load(refscale + k));
    const double kin = (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / q[0];
    const double mag = q[5] * q[5] + q[6] * q[6] + q[7] * q[7];
    return gm1 * (q[4] - 0.5 * kin - 0.5 * mag);
}

//
// Deviation storage (DEV): the values in f are the stored deviations
// g_ki = (f_ki - w_i r_k) / s_k.  Because sum_i w_i = 1 the moment is
// Q_k = r_k + s_k sum_i g_ki, and the BGK update is affine in f, so it runs on
// g directly: g*_ki = (1 - omega) g_ki + omega w_i G_k + w_i S_k / s_k
// +- omega Phi_k,a / (2 s_k) with G_k = sum_i g_ki -- no per-population decode
// or encode.  The caller passes src0/src1 already divided by s_k.
//
// Selective FP64 pressure recovery (deviation storage): where the FP32 gas
// pressure is below p_theta * e_tot -- near vacuum, high Mach or low beta, where
// p = (gamma - 1)(e_tot - rho|u|^2/2 - |B|^2/2) is a small difference of large
// terms -- the cell recomputes p in FP64 from the FP64 reference state,
// Q_k = r_k + s_k G_k (G_k, the FP32 sum of the stored deviations, is exact to
// its own rounding; refscale holds r_0..7 then s_0..7 in global memory, read
// only inside the rare branch so that they occupy no registers elsewhere).
// Everything else stays FP32.
// Fluxes phi[k][a] of one cell from its moment sums G_k (deviation storage:
// Q_k = r_k + s_k G_k), with the positivity check.
template <int D, class C, bool DEV>
VLBM_HD __forceinline__ void ideal_flux_of_sums(const C (&G)[8], const C gm1, unsigned *flags, const C *ref,
                                                const C *scale, const double *refscale, const C p_theta,
                                                C (&phi)[8][D])
{
    C q[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) q[k] = DEV ? ref[k] + scale[k] * G[k] : G[k];
    const C rho = q[0];
    const C ir = C(1) / rho;
    const C m[3] = {q[1], q[2], q[3]};
    const C u[3] = {m[0] * ir, m[1] * ir, m[2] * ir};
    const C E = q[4];
    const C B[3] = {q[5], q[6], q[7]};
    const C B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    const C mu = m[0] * u[0] + m[1] * u[1] + m[2] * u[2];
    const C uB = u[0] * B[0] + u[1] * B[1] + u[2] * B[2];
    C p = gm1 * (E - C(0.5) * mu - C(0.5) * B2);
    if constexpr (DEV) {
        if (p_theta > C(0) && p < p_theta * E)  // FP64 pressure recovery (a call: no registers held elsewhere)
            p = (C)pressure_fp64(G[0], G[1], G[2], G[3], G[4], G[5], G[6], G[7], refscale, (double)gm1);
    }
    const C pt = p + C(0.5) * B2;
    if (!(rho > C(0)) || !(p > C(0))) raise_flag(flags, kFlagNonPhysical);
    const C Ept = E + pt;
#pragma unroll
    for (int ax = 0; ax < D; ++ax) {
        phi[0][ax] = m[ax];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            phi[1 + b][ax] = m[ax] * u[b] - B[ax] * B[b] + (ax == b ? pt : C(0));
            phi[5 + b][ax] = (ax == b) ? C(0) : u[ax] * B[b] - B[ax] * u[b];
        }
        phi[4][ax] = Ept * u[ax] - B[ax] * uB;
    }
}

// BGK relaxation with source of lattice k's populations fk in place, given
// its sum G_k and flux phi_k.
template <int D, class C, bool DEV>
VLBM_HD __forceinline__ void ideal_relax_lattice(C (&fk)[AxisSet<D>::Q], const int k, const C Gk,
                                                 const C (&phik)[D], const C *omega, const C *src0,
                                                 const C *src1, const C *inv_scale)
{
    const C om = omega[k];
    const C omc = C(1) - om;
    C ow0, ow1;
    relax_weights<D, C>(om, ow0, ow1);
    const C A0 = ow0 * Gk + src0[k];
    const C A1 = ow1 * Gk + src1[k];
    const C hom = DEV ? C(0.5) * om * inv_scale[k] : C(0.5) * om;  // omega * w_moving / cs^2 (/ s_k)
    fk[0] = omc * fk[0] + A0;
#pragma unroll
    for (int ax = 0; ax < D; ++ax) {
        const C bv = hom * phik[ax];
        fk[2 * ax + 1] = omc * fk[2 * ax + 1] + A1 + bv;
        fk[2 * ax + 2] = omc * fk[2 * ax + 2] + A1 - bv;
    }
}

template <int D, class C, bool DEV = false>
VLBM_HD __forceinline__ void ideal_collide(C (&f)[8][AxisSet<D>::Q], const C gm1, const C *omega,
                                           const C *src0, const C *src1, unsigned *flags,
                                           const C *ref = nullptr, const C *scale = nullptr,
                                           const C *inv_scale = nullptr, const double *refscale = nullptr,
                                           const C p_theta = C(0))
{
    constexpr int Q = AxisSet<D>::Q;
    C G[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        C s = f[k][0];
#pragma unroll
        for (int i = 1; i < Q; ++i) s += f[k][i];
        G[k] = s;
    }
    C phi[8][D];
    ideal_flux_of_sums<D, C, DEV>(G, gm1, flags, ref, scale, refscale, p_theta, phi);
#pragma unroll
    for (int k = 0; k < 8; ++k) ideal_relax_lattice<D, C, DEV>(f[k], k, G[k], phi[k], omega, src0, src1, inv_scale);
}

// Homogenised solids (sec. 2.4, "Homogenization"): the equilibrium and the
// fluxes take the blended velocity and field u_hat = d u + (1 - d) uB,
// B_hat = d B + (1 - d) BB at the cell's own density and gas pressure, i.e. the
// state Q_hat = (rho, rho u_hat, p/(gamma-1) + rho|u_hat|^2/2 + |B_hat|^2/2,
// B_hat); BGK towards f_eq(Q_hat) plus the uniform source.  Plain storage.
template <int D, class C>
VLBM_HD __forceinline__ void ideal_collide_hom(C (&f)[8][AxisSet<D>::Q], const C gm1, const C *omega,
                                               const C *src0, const C *src1, unsigned *flags, const C d,
                                               const C (&uB)[3], const C (&BB)[3])
{
    constexpr int Q = AxisSet<D>::Q;
    C q[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        C s = f[k][0];
#pragma unroll
        for (int i = 1; i < Q; ++i) s += f[k][i];
        q[k] = s;
    }
    const C rho = q[0];
    const C ir = C(1) / rho;
    const C u[3] = {q[1] * ir, q[2] * ir, q[3] * ir};
    const C B[3] = {q[5], q[6], q[7]};
    const C B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    const C mu = q[1] * u[0] + q[2] * u[1] + q[3] * u[2];
    const C p = gm1 * (q[4] - C(0.5) * mu - C(0.5) * B2);
    if (!(rho > C(0)) || !(p > C(0))) raise_flag(flags, kFlagNonPhysical);
    // blended state
    const C dc = C(1) - d;
    C uh[3], Bh[3], mh[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        uh[a] = d * u[a] + dc * uB[a];
        Bh[a] = d * B[a] + dc * BB[a];
        mh[a] = rho * uh[a];
    }
    const C Bh2 = Bh[0] * Bh[0] + Bh[1] * Bh[1] + Bh[2] * Bh[2];
    const C muh = mh[0] * uh[0] + mh[1] * uh[1] + mh[2] * uh[2];
    const C Eh = p / gm1 + C(0.5) * muh + C(0.5) * Bh2;
    const C pt = p + C(0.5) * Bh2;
    const C uBh = uh[0] * Bh[0] + uh[1] * Bh[1] + uh[2] * Bh[2];
    const C qh[8] = {rho, mh[0], mh[1], mh[2], Eh, Bh[0], Bh[1], Bh[2]};

    C phi[8][D];
#pragma unroll
    for (int ax = 0; ax < D; ++ax) {
        phi[0][ax] = mh[ax];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            phi[1 + b][ax] = mh[ax] * uh[b] - Bh[ax] * Bh[b] + (ax == b ? pt : C(0));
            phi[5 + b][ax] = (ax == b) ? C(0) : uh[ax] * Bh[b] - Bh[ax] * uh[b];
        }
        phi[4][ax] = (Eh + pt) * uh[ax] - Bh[ax] * uBh;
    }

#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const C om = omega[k];
        const C omc = C(1) - om;
        C ow0, ow1;
        relax_weights<D, C>(om, ow0, ow1);
        const C A0 = ow0 * qh[k] + src0[k];
        const C A1 = ow1 * qh[k] + src1[k];
        const C hom = C(0.5) * om;  // omega * w_moving / cs^2
        f[k][0] = omc * f[k][0] + A0;
#pragma unroll
        for (int ax = 0; ax < D; ++ax) {
            const C bv = hom * phi[k][ax];
            f[k][2 * ax + 1] = omc * f[k][2 * ax + 1] + A1 + bv;
            f[k][2 * ax + 2] = omc * f[k][2 * ax + 2] + A1 - bv;
        }
    }
}

// Ideal MHD with Powell's source (sec. 2.3, "Powell correction") on nine
// lattices: the eight of ideal_collide plus D, the trace of the gradient
// tensor of the local moments evolution (sec. 2.2.1), with flux D u - B.
// div B = D / tau_M; the source S = -(div B)(0, B, u.B, u) for the eight MHD
// lattices and -D / tau_M for D is injected directly, f* += w_i S_k, on top
// of the uniform source src0/src1.  Plain storage only (no deviations).
template <int D, class C>
VLBM_HD __forceinline__ void powell_collide(C (&f)[9][AxisSet<D>::Q], const C gm1, const C *omega,
                                            const C *src0, const C *src1, const C inv_tau_m, unsigned *flags)
{
    constexpr int Q = AxisSet<D>::Q;
    C q[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        C s = f[k][0];
#pragma unroll
        for (int i = 1; i < Q; ++i) s += f[k][i];
        q[k] = s;
    }
    const C rho = q[0];
    const C ir = C(1) / rho;
    const C m[3] = {q[1], q[2], q[3]};
    const C u[3] = {m[0] * ir, m[1] * ir, m[2] * ir};
    const C E = q[4];
    const C B[3] = {q[5], q[6], q[7]};
    const C Dv = q[8];
    const C B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    const C mu = m[0] * u[0] + m[1] * u[1] + m[2] * u[2];
    const C uB = u[0] * B[0] + u[1] * B[1] + u[2] * B[2];
    const C p = gm1 * (E - C(0.5) * mu - C(0.5) * B2);
    const C pt = p + C(0.5) * B2;
    if (!(rho > C(0)) || !(p > C(0))) raise_flag(flags, kFlagNonPhysical);
    const C Ept = E + pt;

    C phi[9][D];
#pragma unroll
    for (int ax = 0; ax < D; ++ax) {
        phi[0][ax] = m[ax];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            phi[1 + b][ax] = m[ax] * u[b] - B[ax] * B[b] + (ax == b ? pt : C(0));
            phi[5 + b][ax] = (ax == b) ? C(0) : u[ax] * B[b] - B[ax] * u[b];
        }
        phi[4][ax] = Ept * u[ax] - B[ax] * uB;
        phi[8][ax] = Dv * u[ax] - B[ax];
    }
    // state-dependent source: S_k = -div B * (0, B, u.B, u), S_D = -D / tau_M = -div B
    const C ndiv = -Dv * inv_tau_m;
    C S[9];
    S[0] = C(0);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        S[1 + b] = ndiv * B[b];
        S[5 + b] = ndiv * u[b];
    }
    S[4] = ndiv * uB;
    S[8] = ndiv;

    constexpr C w0 = ExactWeights<D, C>::w0, w1 = ExactWeights<D, C>::w1;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const C om = omega[k];
        const C omc = C(1) - om;
        C ow0, ow1;
        relax_weights<D, C>(om, ow0, ow1);
        const C A0 = ow0 * q[k] + src0[k] + w0 * S[k];
        const C A1 = ow1 * q[k] + src1[k] + w1 * S[k];
        const C hom = C(0.5) * om;  // omega * w_moving / cs^2
        f[k][0] = omc * f[k][0] + A0;
#pragma unroll
        for (int ax = 0; ax < D; ++ax) {
            const C bv = hom * phi[k][ax];
            f[k][2 * ax + 1] = omc * f[k][2 * ax + 1] + A1 + bv;
            f[k][2 * ax + 2] = omc * f[k][2 * ax + 2] + A1 - bv;
        }
    }
}

}  // namespace vlbm
