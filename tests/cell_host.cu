// cell_host.cu -- host build of the step kernels' per-cell arithmetic
// (ideal_cell.cuh: moments, Eq. 4; pressure, Eq. 9; fluxes, Eq. 12; BGK with
// direct source injection, Eq. 2 and 3; the Powell, homogenised-solid and
// deviation-storage forms; diss_cell.cuh: the fluxes and sources of the
// dissipative system, sec. 2.2.1 and 2.3), so that CPU tests can compare it
// cell by cell with the oracle.  Test infrastructure only: nothing in the
// library calls it, and the library has no CPU path.
//
// The collision entries take one cell's populations f[k * q + i] (k lattice,
// i direction 0 rest, 2a+1 = +e_a, 2a+2 = -e_a; q = 5 in 2-D, 7 in 3-D) and
// collide them in place with the kernels' own inputs: omega_k = 1 / tau_k,
// src0_k = w_0 S_k, src1_k = w_moving S_k (deviation storage: both divided by
// the scale s_k); they return 0, or -1 for a dimension other than 2 or 3.
// The dissipative entries take one state and return its fluxes and sources.
// Status bits a cell raises are OR-ed into *flags.
#include "diss_cell.cuh"
#include "ideal_cell.cuh"

using namespace vlbm;

namespace {

template <int D, class C> struct Cell {
    static constexpr int Q = AxisSet<D>::Q;
    template <int NL> static void get(const C *f, C (&c)[NL][Q])
    {
        for (int k = 0; k < NL; ++k)
            for (int i = 0; i < Q; ++i) c[k][i] = f[k * Q + i];
    }
    template <int NL> static void put(const C (&c)[NL][Q], C *f)
    {
        for (int k = 0; k < NL; ++k)
            for (int i = 0; i < Q; ++i) f[k * Q + i] = c[k][i];
    }
};

template <int D, class C>
void ideal(C gm1, const C *omega, const C *src0, const C *src1, C *f, unsigned *flags)
{
    C c[8][AxisSet<D>::Q];
    Cell<D, C>::get(f, c);
    ideal_collide<D, C, false>(c, gm1, omega, src0, src1, flags);
    Cell<D, C>::put(c, f);
}

template <int D>
void ideal_dev(float gm1, const float *omega, const float *src0, const float *src1, const float *ref,
               const float *scale, const float *inv_scale, const double *refscale, float p_theta, float *g,
               unsigned *flags)
{
    float c[8][AxisSet<D>::Q];
    Cell<D, float>::get(g, c);
    ideal_collide<D, float, true>(c, gm1, omega, src0, src1, flags, ref, scale, inv_scale, refscale, p_theta);
    Cell<D, float>::put(c, g);
}

template <int D, class C>
void powell(C gm1, const C *omega, const C *src0, const C *src1, C inv_tau_m, C *f, unsigned *flags)
{
    C c[9][AxisSet<D>::Q];
    Cell<D, C>::get(f, c);
    powell_collide<D, C>(c, gm1, omega, src0, src1, inv_tau_m, flags);
    Cell<D, C>::put(c, f);
}

template <int D, class C>
void hom(C gm1, const C *omega, const C *src0, const C *src1, C d, const C *uB, const C *BB, C *f, unsigned *flags)
{
    C c[8][AxisSet<D>::Q];
    Cell<D, C>::get(f, c);
    const C u[3] = {uB[0], uB[1], uB[2]};
    const C b[3] = {BB[0], BB[1], BB[2]};
    ideal_collide_hom<D, C>(c, gm1, omega, src0, src1, flags, d, u, b);
    Cell<D, C>::put(c, f);
}

template <class C>
void diss(const C *q, C gm1, C nu, C eta0, C inv_jc2, C inv_tau_m, int powell, C *phi, C *S, unsigned *flags)
{
    DissArgs<C> a{};
    a.gm1 = gm1;
    a.nu = nu;
    a.eta0 = eta0;
    a.inv_jc2 = inv_jc2;
    a.inv_tau_m = inv_tau_m;
    a.powell = powell;
    C qq[kDissLat], ph[kDissLat][2], s[kDissLat];
    for (int k = 0; k < kDissLat; ++k) qq[k] = q[k];
    diss_flux_source<C>(qq, a, ph, s, flags);
    for (int k = 0; k < kDissLat; ++k) {
        phi[2 * k] = ph[k][0];
        phi[2 * k + 1] = ph[k][1];
        S[k] = s[k];
    }
}

template <class C>
void diss3(const C *q, C gm1, C nu, C eta0, C inv_jc2, C inv_tau_m, int powell, C *phi, C *S, unsigned *flags)
{
    DissArgs<C> a{};
    a.gm1 = gm1;
    a.nu = nu;
    a.eta0 = eta0;
    a.inv_jc2 = inv_jc2;
    a.inv_tau_m = inv_tau_m;
    a.powell = powell;
    C qq[kDiss3Lat];
    for (int k = 0; k < kDiss3Lat; ++k) qq[k] = q[k];
    const Diss3State<C> st = diss3_state<C>(qq, a, flags);
    for (int k = 0; k < kDiss3Lat; ++k) {
        C ph[3];
        diss3_flux<C>(k, qq, st, ph);
        for (int c = 0; c < 3; ++c) phi[3 * k + c] = ph[c];
        S[k] = diss3_source<C>(k, qq, st, inv_tau_m);
    }
}

}  // namespace

#define HC_DIM(dim, call2, call3) \
    do {                          \
        if ((dim) == 2) {         \
            call2;                \
        } else if ((dim) == 3) {  \
            call3;                \
        } else {                  \
            return -1;            \
        }                         \
        return 0;                 \
    } while (0)

extern "C" {

// Plain storage, FP64 (the FP64 kernels) and FP32 (the FP32 kernels).
int hc_ideal_f64(int dim, double gm1, const double *omega, const double *src0, const double *src1, double *f,
                 unsigned *flags)
{
    HC_DIM(dim, (ideal<2, double>(gm1, omega, src0, src1, f, flags)),
           (ideal<3, double>(gm1, omega, src0, src1, f, flags)));
}

int hc_ideal_f32(int dim, float gm1, const float *omega, const float *src0, const float *src1, float *f,
                 unsigned *flags)
{
    HC_DIM(dim, (ideal<2, float>(gm1, omega, src0, src1, f, flags)),
           (ideal<3, float>(gm1, omega, src0, src1, f, flags)));
}

// Deviation storage: g holds (f - w_i r_k) / s_k in FP32 (as decoded from
// FP16/BF16); refscale = r_0..7 then s_0..7 in FP64 for the pressure recovery.
int hc_ideal_dev(int dim, float gm1, const float *omega, const float *src0, const float *src1, const float *ref,
                 const float *scale, const float *inv_scale, const double *refscale, float p_theta, float *g,
                 unsigned *flags)
{
    HC_DIM(dim, (ideal_dev<2>(gm1, omega, src0, src1, ref, scale, inv_scale, refscale, p_theta, g, flags)),
           (ideal_dev<3>(gm1, omega, src0, src1, ref, scale, inv_scale, refscale, p_theta, g, flags)));
}

// Powell form: nine lattices, the ninth the divergence lattice D.
int hc_powell_f64(int dim, double gm1, const double *omega, const double *src0, const double *src1,
                  double inv_tau_m, double *f, unsigned *flags)
{
    HC_DIM(dim, (powell<2, double>(gm1, omega, src0, src1, inv_tau_m, f, flags)),
           (powell<3, double>(gm1, omega, src0, src1, inv_tau_m, f, flags)));
}

int hc_powell_f32(int dim, float gm1, const float *omega, const float *src0, const float *src1, float inv_tau_m,
                  float *f, unsigned *flags)
{
    HC_DIM(dim, (powell<2, float>(gm1, omega, src0, src1, inv_tau_m, f, flags)),
           (powell<3, float>(gm1, omega, src0, src1, inv_tau_m, f, flags)));
}

// Homogenised solid: porosity d, solid velocity uB[3] and field BB[3].
int hc_hom_f64(int dim, double gm1, const double *omega, const double *src0, const double *src1, double d,
               const double *uB, const double *BB, double *f, unsigned *flags)
{
    HC_DIM(dim, (hom<2, double>(gm1, omega, src0, src1, d, uB, BB, f, flags)),
           (hom<3, double>(gm1, omega, src0, src1, d, uB, BB, f, flags)));
}

int hc_hom_f32(int dim, float gm1, const float *omega, const float *src0, const float *src1, float d,
               const float *uB, const float *BB, float *f, unsigned *flags)
{
    HC_DIM(dim, (hom<2, float>(gm1, omega, src0, src1, d, uB, BB, f, flags)),
           (hom<3, float>(gm1, omega, src0, src1, d, uB, BB, f, flags)));
}

// Dissipative system (2-D): fluxes phi[2 k + c] along x, y and sources S[k] of
// one state q[20]; inv_jc2 = 1 / j_c^2 (0: constant eta), powell 0 or 1.
int hc_diss_f64(const double *q, double gm1, double nu, double eta0, double inv_jc2, double inv_tau_m, int powell,
                double *phi, double *S, unsigned *flags)
{
    diss<double>(q, gm1, nu, eta0, inv_jc2, inv_tau_m, powell, phi, S, flags);
    return 0;
}

int hc_diss_f32(const float *q, float gm1, float nu, float eta0, float inv_jc2, float inv_tau_m, int powell,
                float *phi, float *S, unsigned *flags)
{
    diss<float>(q, gm1, nu, eta0, inv_jc2, inv_tau_m, powell, phi, S, flags);
    return 0;
}

// Dissipative system (3-D): fluxes phi[3 k + c] along x, y, z and sources S[k]
// of one state q[26].
int hc_diss3_f64(const double *q, double gm1, double nu, double eta0, double inv_jc2, double inv_tau_m, int powell,
                 double *phi, double *S, unsigned *flags)
{
    diss3<double>(q, gm1, nu, eta0, inv_jc2, inv_tau_m, powell, phi, S, flags);
    return 0;
}

int hc_diss3_f32(const float *q, float gm1, float nu, float eta0, float inv_jc2, float inv_tau_m, int powell,
                 float *phi, float *S, unsigned *flags)
{
    diss3<float>(q, gm1, nu, eta0, inv_jc2, inv_tau_m, powell, phi, S, flags);
    return 0;
}

}  // extern "C"
