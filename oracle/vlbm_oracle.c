/*
 * vlbm_oracle.c -- plain, slow, FP64 CPU oracle of the vectorial lattice
 * Boltzmann method (VLBM) for magnetohydrodynamics.
 *
 * TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark load this library.
 * It shares no code, header, table or helper with the CUDA path.
 *
 * Equation numbers follow the order in which the paper displays them:
 *   Eq. 1  generic conservation law  dQ/dt + div Phi = S          (sec. 2.1)
 *   Eq. 2  fully local VLBM update (collision + source + stream)   (sec. 2.2)
 *   Eq. 3  first-order, flux-carrying equilibrium                  (sec. 2.2)
 *   Eq. 4  moments  Q_k = sum_i f_ki,  Phi_k = sum_i f_ki c_i      (sec. 2.2)
 *   Eq. 5  D = (tau - 1/2) c_s^2 dt                                (sec. 2.2)
 *   Eq. 9  ideal-gas EOS with magnetic energy                      (sec. 2.3)
 *   Eq. 12 ideal MHD state vector and flux                         (sec. 2.3)
 *   Powell source  S = -(div B)(0, B, u.B, u)          (sec. 2.3, "Powell correction")
 *   homogenised solids: blended u, B and the porosity of the signed distance
 *                                                      (sec. 2.4, "Homogenization")
 *   equilibrium Dirichlet / Neumann open boundaries    (sec. 2.4, "Static boundaries")
 *   dissipative MHD: viscous stress, eta(j) resistivity, gradients evolved
 *   as lattices                                        (sec. 2.2.1, 2.3; 2-D and 3-D)
 *   local gradient evolution  dG/dt + div Phi_G = -G/tau_R          (sec. 2.2.1)
 *
 * Readings where the paper is silent:
 *   - lattice weights: D2Q5 w0=1/3, w=1/6, cs2=1/3;  D3Q7 w0=1/4, w=1/8,
 *     cs2=1/4;  D3Q19 1/3, 1/18, 1/36, cs2=1/3 (the paper's lattice table is
 *     not printed);
 *   - "Strang splitting": every lattice takes its flux from the step-start
 *     state Q of the same cell; the source is injected in the same collision;
 *   - BGK collision and direct source injection  f* += w_i S_k  (sec. 3:
 *     BGK collisions with the source injected directly);
 *   - the resistive incompressible model (D3Q19 flow lattice with a
 *     second-order equilibrium carrying the Maxwell stress, Guo body force,
 *     three D3Q7 magnetic lattices with the Eq. 3 equilibrium and the
 *     induction flux of Eq. 12, halfway bounce-back walls in y, magnetic
 *     walls held at the equilibrium of the applied field) is the workload's
 *     reading of sec. 2.3 "Incompressible resistive MHD" with sec. 2.4
 *     "Static boundaries".
 *
 * Everything is written for clarity: plain loops, two population arrays,
 * push streaming, no blocking, no fusion.  Compile with -ffp-contract=off.
 *
 * Layout of every population array: f[(k*q + i)*N + cell],
 * cell = x + nx*(y + ny*z).  Direction order: 0 rest; 1 +x, 2 -x, 3 +y,
 * 4 -y, 5 +z, 6 -z; D3Q19 adds 7 (+1,+1,0) 8 (-1,-1,0) 9 (+1,-1,0)
 * 10 (-1,+1,0) 11 (+1,0,+1) 12 (-1,0,-1) 13 (+1,0,-1) 14 (-1,0,+1)
 * 15 (0,+1,+1) 16 (0,-1,-1) 17 (0,+1,-1) 18 (0,-1,+1).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_QMAX 19
#define ORC_NVAR_IDEAL 8

typedef struct {
    int q;
    int c[ORC_QMAX][3];
    double w[ORC_QMAX];
    double cs2;
    int opp[ORC_QMAX];
} orc_lattice;

static void set_dir(orc_lattice *L, int i, int cx, int cy, int cz, double w)
{
    L->c[i][0] = cx;
    L->c[i][1] = cy;
    L->c[i][2] = cz;
    L->w[i] = w;
}

/* Velocity sets (sec. 2.2, "Lattice independence"; weights are a reading). */
static int build_lattice(int q, orc_lattice *L)
{
    memset(L, 0, sizeof(*L));
    L->q = q;
    if (q == 5) {
        L->cs2 = 1.0 / 3.0;
        set_dir(L, 0, 0, 0, 0, 1.0 / 3.0);
        set_dir(L, 1, 1, 0, 0, 1.0 / 6.0);
        set_dir(L, 2, -1, 0, 0, 1.0 / 6.0);
        set_dir(L, 3, 0, 1, 0, 1.0 / 6.0);
        set_dir(L, 4, 0, -1, 0, 1.0 / 6.0);
    } else if (q == 7) {
        L->cs2 = 1.0 / 4.0;
        set_dir(L, 0, 0, 0, 0, 1.0 / 4.0);
        set_dir(L, 1, 1, 0, 0, 1.0 / 8.0);
        set_dir(L, 2, -1, 0, 0, 1.0 / 8.0);
        set_dir(L, 3, 0, 1, 0, 1.0 / 8.0);
        set_dir(L, 4, 0, -1, 0, 1.0 / 8.0);
        set_dir(L, 5, 0, 0, 1, 1.0 / 8.0);
        set_dir(L, 6, 0, 0, -1, 1.0 / 8.0);
    } else if (q == 19) {
        L->cs2 = 1.0 / 3.0;
        set_dir(L, 0, 0, 0, 0, 1.0 / 3.0);
        set_dir(L, 1, 1, 0, 0, 1.0 / 18.0);
        set_dir(L, 2, -1, 0, 0, 1.0 / 18.0);
        set_dir(L, 3, 0, 1, 0, 1.0 / 18.0);
        set_dir(L, 4, 0, -1, 0, 1.0 / 18.0);
        set_dir(L, 5, 0, 0, 1, 1.0 / 18.0);
        set_dir(L, 6, 0, 0, -1, 1.0 / 18.0);
        set_dir(L, 7, 1, 1, 0, 1.0 / 36.0);
        set_dir(L, 8, -1, -1, 0, 1.0 / 36.0);
        set_dir(L, 9, 1, -1, 0, 1.0 / 36.0);
        set_dir(L, 10, -1, 1, 0, 1.0 / 36.0);
        set_dir(L, 11, 1, 0, 1, 1.0 / 36.0);
        set_dir(L, 12, -1, 0, -1, 1.0 / 36.0);
        set_dir(L, 13, 1, 0, -1, 1.0 / 36.0);
        set_dir(L, 14, -1, 0, 1, 1.0 / 36.0);
        set_dir(L, 15, 0, 1, 1, 1.0 / 36.0);
        set_dir(L, 16, 0, -1, -1, 1.0 / 36.0);
        set_dir(L, 17, 0, 1, -1, 1.0 / 36.0);
        set_dir(L, 18, 0, -1, 1, 1.0 / 36.0);
    } else {
        return -1;
    }
    /* opposite direction found by search, not by a formula */
    for (int i = 0; i < q; ++i) {
        L->opp[i] = -1;
        for (int j = 0; j < q; ++j)
            if (L->c[j][0] == -L->c[i][0] && L->c[j][1] == -L->c[i][1] &&
                L->c[j][2] == -L->c[i][2])
                L->opp[i] = j;
    }
    return 0;
}

/* Periodic neighbour of cell (x,y,z) along velocity c. */
static long neighbour(int x, int y, int z, const int *c, int nx, int ny, int nz)
{
    int xn = (x + c[0] + nx) % nx;
    int yn = (y + c[1] + ny) % ny;
    int zn = (z + c[2] + nz) % nz;
    return (long)xn + (long)nx * ((long)yn + (long)ny * (long)zn);
}

static int check_dims(int dim, int nx, int ny, int nz)
{
    if (nx < 1 || ny < 1 || nz < 1) return -1;
    if (dim == 2 && nz != 1) return -1;
    if (dim != 2 && dim != 3) return -1;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Ideal compressible MHD (Eq. 12 with the EOS of Eq. 9)               */
/* ------------------------------------------------------------------ */

/*
 * Flux tensor of ideal MHD, Eq. 12.  Q = (rho, rho u_x, rho u_y, rho u_z,
 * e_tot, B_x, B_y, B_z).  phi[3*k + a] is the flux of Q_k along axis a:
 *   rho:     rho u_a
 *   rho u_b: rho u_a u_b + p_tot delta_ab - B_a B_b
 *   e_tot:   (e_tot + p_tot) u_a - B_a (u . B)
 *   B_b:     u_a B_b - B_a u_b
 * with p from the EOS (Eq. 9) and p_tot = p + |B|^2/2 (sec. 2.3).
 */
void orc_ideal_flux(double gamma, const double *Q, double *phi)
{
    double rho = Q[0];
    double u[3] = {Q[1] / rho, Q[2] / rho, Q[3] / rho};
    double e = Q[4];
    double B[3] = {Q[5], Q[6], Q[7]};
    double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    double uB = u[0] * B[0] + u[1] * B[1] + u[2] * B[2];
    double p = (gamma - 1.0) * (e - 0.5 * rho * u2 - 0.5 * B2); /* Eq. 9 */
    double ptot = p + 0.5 * B2;
    for (int a = 0; a < 3; ++a) {
        phi[3 * 0 + a] = rho * u[a];
        for (int b = 0; b < 3; ++b) {
            double delta = (a == b) ? 1.0 : 0.0;
            phi[3 * (1 + b) + a] = rho * u[a] * u[b] + ptot * delta - B[a] * B[b];
            phi[3 * (5 + b) + a] = u[a] * B[b] - B[a] * u[b];
        }
        phi[3 * 4 + a] = (e + ptot) * u[a] - B[a] * uB;
    }
}

/* Gas pressure from the EOS, Eq. 9 (used by tests for health checks). */
double orc_ideal_pressure(double gamma, const double *Q)
{
    double rho = Q[0];
    double m2 = Q[1] * Q[1] + Q[2] * Q[2] + Q[3] * Q[3];
    double B2 = Q[5] * Q[5] + Q[6] * Q[6] + Q[7] * Q[7];
    return (gamma - 1.0) * (Q[4] - 0.5 * m2 / rho - 0.5 * B2);
}

/* First-order equilibrium, Eq. 3:  f_eq_ki = w_i (Q_k + c_i . Phi_k / cs^2). */
static void ideal_feq(const orc_lattice *L, double gamma, const double *Q,
                      double feq[ORC_NVAR_IDEAL][ORC_QMAX])
{
    double phi[3 * ORC_NVAR_IDEAL];
    orc_ideal_flux(gamma, Q, phi);
    for (int k = 0; k < ORC_NVAR_IDEAL; ++k)
        for (int i = 0; i < L->q; ++i) {
            double cphi = 0.0;
            for (int a = 0; a < 3; ++a) cphi += L->c[i][a] * phi[3 * k + a];
            feq[k][i] = L->w[i] * (Q[k] + cphi / L->cs2);
        }
}

/*
 * Collision of one cell (Eq. 2 without the streaming): BGK relaxation towards
 * the Eq. 3 equilibrium built from the cell's own moments (Eq. 4), plus
 * direct injection of a source  w_i S_k.  fin/fout hold 8*q values, index
 * k*q + i.  src may be NULL (S = 0, the ideal system of Eq. 12).
 */
static void ideal_collide(const orc_lattice *L, double gamma, const double *tau,
                          const double *src, const double *fin, double *fout)
{
    double Q[ORC_NVAR_IDEAL];
    double feq[ORC_NVAR_IDEAL][ORC_QMAX];
    for (int k = 0; k < ORC_NVAR_IDEAL; ++k) {
        Q[k] = 0.0;
        for (int i = 0; i < L->q; ++i) Q[k] += fin[k * L->q + i]; /* Eq. 4 */
    }
    ideal_feq(L, gamma, Q, feq);
    for (int k = 0; k < ORC_NVAR_IDEAL; ++k)
        for (int i = 0; i < L->q; ++i) {
            double f = fin[k * L->q + i];
            double out = f + (feq[k][i] - f) / tau[k];
            if (src) out += L->w[i] * src[k];
            fout[k * L->q + i] = out;
        }
}

static int ideal_lattice(int dim, orc_lattice *L)
{
    return build_lattice(dim == 2 ? 5 : 7, L);
}

/* Lattice table export (for tests of the quadrature conditions). */
int orc_lattice_info(int q, int *c, double *w, double *cs2, int *opp)
{
    orc_lattice L;
    if (build_lattice(q, &L)) return -1;
    for (int i = 0; i < q; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = L.c[i][a];
        w[i] = L.w[i];
        opp[i] = L.opp[i];
    }
    *cs2 = L.cs2;
    return 0;
}

/* Single-cell collision, exported for sampled parity checks. */
int orc_ideal_collide_cell(int dim, double gamma, const double *tau, const double *src,
                           const double *fin, double *fout)
{
    orc_lattice L;
    if (dim != 2 && dim != 3) return -1;
    ideal_lattice(dim, &L);
    ideal_collide(&L, gamma, tau, src, fin, fout);
    return 0;
}

/* Initial populations: f = f_eq(Q0) (zero non-equilibrium part). */
int orc_ideal_init(int dim, int nx, int ny, int nz, double gamma, const double *Q0, double *f)
{
    orc_lattice L;
    if (check_dims(dim, nx, ny, nz)) return -1;
    ideal_lattice(dim, &L);
    long N = (long)nx * ny * nz;
    for (long cell = 0; cell < N; ++cell) {
        double Q[ORC_NVAR_IDEAL];
        double feq[ORC_NVAR_IDEAL][ORC_QMAX];
        for (int k = 0; k < ORC_NVAR_IDEAL; ++k) Q[k] = Q0[k * N + cell];
        ideal_feq(&L, gamma, Q, feq);
        for (int k = 0; k < ORC_NVAR_IDEAL; ++k)
            for (int i = 0; i < L.q; ++i) f[(long)(k * L.q + i) * N + cell] = feq[k][i];
    }
    return 0;
}

/*
 * One time step, Eq. 2: every cell collides, then each post-collision
 * population moves to x + c_i (periodic).  fin and fout must not alias.
 */
int orc_ideal_step(int dim, int nx, int ny, int nz, double gamma, const double *tau,
                   const double *src, const double *fin, double *fout, int nthreads)
{
    orc_lattice L;
    if (check_dims(dim, nx, ny, nz)) return -1;
    ideal_lattice(dim, &L);
    const long N = (long)nx * ny * nz;
    const int q = L.q;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (long cell = 0; cell < N; ++cell) {
        int x = (int)(cell % nx);
        int y = (int)((cell / nx) % ny);
        int z = (int)(cell / ((long)nx * ny));
        double fc[ORC_NVAR_IDEAL * ORC_QMAX];
        double fs[ORC_NVAR_IDEAL * ORC_QMAX];
        for (int k = 0; k < ORC_NVAR_IDEAL; ++k)
            for (int i = 0; i < q; ++i) fc[k * q + i] = fin[(long)(k * q + i) * N + cell];
        ideal_collide(&L, gamma, tau, src, fc, fs);
        for (int i = 0; i < q; ++i) {
            long dst = neighbour(x, y, z, L.c[i], nx, ny, nz);
            for (int k = 0; k < ORC_NVAR_IDEAL; ++k)
                fout[(long)(k * q + i) * N + dst] = fs[k * q + i];
        }
    }
    return 0;
}

/* Zeroth moments Q_k = sum_i f_ki (Eq. 4). */
int orc_ideal_moments(int dim, int nx, int ny, int nz, const double *f, double *Q)
{
    orc_lattice L;
    if (check_dims(dim, nx, ny, nz)) return -1;
    ideal_lattice(dim, &L);
    long N = (long)nx * ny * nz;
    for (int k = 0; k < ORC_NVAR_IDEAL; ++k)
        for (long cell = 0; cell < N; ++cell) {
            double s = 0.0;
            for (int i = 0; i < L.q; ++i) s += f[(long)(k * L.q + i) * N + cell];
            Q[k * N + cell] = s;
        }
    return 0;
}

/* Whole run: init from Q0, nsteps steps, moments into Qout. */
int orc_ideal_run(int dim, int nx, int ny, int nz, double gamma, const double *tau,
                  const double *src, const double *Q0, int nsteps, double *Qout, int nthreads)
{
    if (check_dims(dim, nx, ny, nz) || nsteps < 0) return -1;
    int q = dim == 2 ? 5 : 7;
    long N = (long)nx * ny * nz;
    double *a = (double *)malloc(sizeof(double) * ORC_NVAR_IDEAL * q * N);
    double *b = (double *)malloc(sizeof(double) * ORC_NVAR_IDEAL * q * N);
    if (!a || !b) {
        free(a);
        free(b);
        return -2;
    }
    orc_ideal_init(dim, nx, ny, nz, gamma, Q0, a);
    for (int s = 0; s < nsteps; ++s) {
        orc_ideal_step(dim, nx, ny, nz, gamma, tau, src, a, b, nthreads);
        double *t = a;
        a = b;
        b = t;
    }
    orc_ideal_moments(dim, nx, ny, nz, a, Qout);
    free(a);
    free(b);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Ideal MHD with the Powell correction and a local divergence of B     */
/* ------------------------------------------------------------------ */
/*
 * Sec. 2.3 "Powell correction": the source  S = -(div B) (0, B, u.B, u)  is
 * injected into the lattices of rho, rho u, e_tot and B.  div B comes from
 * the local moments evolution of sec. 2.2.1: the gradient tensor G of B is
 * carried with the flux Phi_G = G (x) u - I (x) B and the relaxation source
 * -G / tau_M (sec. 2.3 "Evolution of the MHD equation system"), so that
 * G ~ tau_M grad B.  The correction needs only the trace of G; a ninth lattice
 * carries it: D = tr G, with the trace of that flux, Phi_D = D u - B, and the
 * source -D / tau_M; then div B = D / tau_M.  (Reading, listed in the design
 * notes: one trace lattice instead of the full tensor, tau_M in time steps.)
 * State Q = (rho, rho u_x, rho u_y, rho u_z, e_tot, B_x, B_y, B_z, D).
 */
#define ORC_NVAR_POWELL 9

/* Flux of the nine fields along the three axes: Eq. 12 for the first eight,
 * Phi_D,a = D u_a - B_a for the ninth.  phi[3*k + a]. */
void orc_powell_flux(double gamma, const double *Q, double *phi)
{
    orc_ideal_flux(gamma, Q, phi);
    double rho = Q[0];
    for (int a = 0; a < 3; ++a) phi[3 * 8 + a] = Q[8] * (Q[1 + a] / rho) - Q[5 + a];
}

/* Source of the nine fields at one state: Powell's term with
 * div B = D / tau_M for the first eight, -D / tau_M for the ninth. */
void orc_powell_source(double tau_m, const double *Q, double *S)
{
    double rho = Q[0];
    double u[3] = {Q[1] / rho, Q[2] / rho, Q[3] / rho};
    double B[3] = {Q[5], Q[6], Q[7]};
    double divB = Q[8] / tau_m;
    double uB = u[0] * B[0] + u[1] * B[1] + u[2] * B[2];
    S[0] = 0.0;
    for (int b = 0; b < 3; ++b) {
        S[1 + b] = -divB * B[b];
        S[5 + b] = -divB * u[b];
    }
    S[4] = -divB * uB;
    S[8] = -Q[8] / tau_m;
}

static void powell_feq(const orc_lattice *L, double gamma, const double *Q,
                       double feq[ORC_NVAR_POWELL][ORC_QMAX])
{
    double phi[3 * ORC_NVAR_POWELL];
    orc_powell_flux(gamma, Q, phi);
    for (int k = 0; k < ORC_NVAR_POWELL; ++k)
        for (int i = 0; i < L->q; ++i) {
            double cphi = 0.0;
            for (int a = 0; a < 3; ++a) cphi += L->c[i][a] * phi[3 * k + a];
            double moving = cphi / L->cs2;
            feq[k][i] = L->w[i] * (Q[k] + moving); /* Eq. 3 */
        }
}

/* Collision of one cell: BGK towards Eq. 3 and direct injection of the
 * state-dependent source plus an optional uniform source src[9]. */
static void powell_collide(const orc_lattice *L, double gamma, const double *tau, double tau_m,
                           const double *src, const double *fin, double *fout)
{
    double Q[ORC_NVAR_POWELL];
    double feq[ORC_NVAR_POWELL][ORC_QMAX];
    double S[ORC_NVAR_POWELL];
    for (int k = 0; k < ORC_NVAR_POWELL; ++k) {
        Q[k] = 0.0;
        for (int i = 0; i < L->q; ++i) Q[k] += fin[k * L->q + i]; /* Eq. 4 */
    }
    powell_feq(L, gamma, Q, feq);
    orc_powell_source(tau_m, Q, S);
    for (int k = 0; k < ORC_NVAR_POWELL; ++k)
        for (int i = 0; i < L->q; ++i) {
            double f = fin[k * L->q + i];
            double sk = S[k] + (src ? src[k] : 0.0);
            fout[k * L->q + i] = f + (feq[k][i] - f) / tau[k] + L->w[i] * sk;
        }
}

int orc_powell_collide_cell(int dim, double gamma, const double *tau, double tau_m, const double *src,
                            const double *fin, double *fout)
{
    orc_lattice L;
    if (dim != 2 && dim != 3) return -1;
    ideal_lattice(dim, &L);
    powell_collide(&L, gamma, tau, tau_m, src, fin, fout);
    return 0;
}

int orc_powell_init(int dim, int nx, int ny, int nz, double gamma, const double *Q0, double *f)
{
    orc_lattice L;
    if (check_dims(dim, nx, ny, nz)) return -1;
    ideal_lattice(dim, &L);
    long N = (long)nx * ny * nz;
    for (long cell = 0; cell < N; ++cell) {
        double Q[ORC_NVAR_POWELL];
        double feq[ORC_NVAR_POWELL][ORC_QMAX];
        for (int k = 0; k < ORC_NVAR_POWELL; ++k) Q[k] = Q0[k * N + cell];
        powell_feq(&L, gamma, Q, feq);
        for (int k = 0; k < ORC_NVAR_POWELL; ++k)
            for (int i = 0; i < L.q; ++i) f[(long)(k * L.q + i) * N + cell] = feq[k][i];
    }
    return 0;
}

int orc_powell_step(int dim, int nx, int ny, int nz, double gamma, const double *tau, double tau_m,
                    const double *src, const double *fin, double *fout, int nthreads)
{
    orc_lattice L;
    if (check_dims(dim, nx, ny, nz) || !(tau_m > 0.0)) return -1;
    ideal_lattice(dim, &L);
    const long N = (long)nx * ny * nz;
    const int q = L.q;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (long cell = 0; cell < N; ++cell) {
        int x = (int)(cell % nx);
        int y = (int)((cell / nx) % ny);
        int z = (int)(cell / ((long)nx * ny));
        double fc[ORC_NVAR_POWELL * ORC_QMAX];
        double fs[ORC_NVAR_POWELL * ORC_QMAX];
        for (int k = 0; k < ORC_NVAR_POWELL; ++k)
            for (int i = 0; i < q; ++i) fc[k * q + i] = fin[(long)(k * q + i) * N + cell];
        powell_collide(&L, gamma, tau, tau_m, src, fc, fs);
        for (int i = 0; i < q; ++i) {
            long to = neighbour(x, y, z, L.c[i], nx, ny, nz); /* push along c_i */
            for (int k = 0; k < ORC_NVAR_POWELL; ++k)
                fout[(long)(k * q + i) * N + to] = fs[k * q + i];
        }
    }
    return 0;
}

int orc_powell_moments(int dim, int nx, int ny, int nz, const double *f, double *Q)
{
    orc_lattice L;
    if (check_dims(dim, nx, ny, nz)) return -1;
    ideal_lattice(dim, &L);
    long N = (long)nx * ny * nz;
    for (int k = 0; k < ORC_NVAR_POWELL; ++k)
        for (long cell = 0; cell < N; ++cell) {
            double s = 0.0;
            for (int i = 0; i < L.q; ++i) s += f[(long)(k * L.q + i) * N + cell];
            Q[k * N + cell] = s;
        }
    return 0;
}

int orc_powell_run(int dim, int nx, int ny, int nz, double gamma, const double *tau, double tau_m,
                   const double *src, const double *Q0, int nsteps, double *Qout, int nthreads)
{
    if (check_dims(dim, nx, ny, nz) || nsteps < 0 || !(tau_m > 0.0)) return -1;
    int q = dim == 2 ? 5 : 7;
    long N = (long)nx * ny * nz;
    double *a = (double *)malloc(sizeof(double) * ORC_NVAR_POWELL * q * N);
    double *b = (double *)malloc(sizeof(double) * ORC_NVAR_POWELL * q * N);
    if (!a || !b) {
        free(a);
        free(b);
        return -2;
    }
    orc_powell_init(dim, nx, ny, nz, gamma, Q0, a);
    for (int s = 0; s < nsteps; ++s) {
        orc_powell_step(dim, nx, ny, nz, gamma, tau, tau_m, src, a, b, nthreads);
        double *t = a;
        a = b;
        b = t;
    }
    orc_powell_moments(dim, nx, ny, nz, a, Qout);
    free(a);
    free(b);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Homogenised solid objects (HLBM) in ideal MHD                        */
/* ------------------------------------------------------------------ */
/*
 * Sec. 2.4 "Homogenization": a solid object is represented by the porosity
 * d(x) in [0, 1] (1 fluid, 0 solid), its velocity uB(x) and field BB(x).
 * The equilibrium and the fluxes use the convex blends
 *   u_hat = d u + (1 - d) uB,   B_hat = d B + (1 - d) BB
 * instead of u and B.  Reading (the paper does not say which state it keeps):
 * rho and the gas pressure p are the cell's own, and the blended state is
 *   Q_hat = (rho, rho u_hat, p/(gamma-1) + rho|u_hat|^2/2 + |B_hat|^2/2, B_hat);
 * the BGK collision relaxes towards f_eq(Q_hat) (Eq. 3 with the fluxes of
 * Eq. 12 at Q_hat).  Porosity from the signed distance phi to the surface
 * (positive in the fluid) with the transition width eps_h:
 *   d = 0 for phi <= -eps_h/2, phi/eps_h + 1/2 inside, 1 for phi >= eps_h/2.
 * Solid fields per cell, solid[(v)*N + cell], v = 0 d, 1..3 uB, 4..6 BB.
 */
double orc_hlbm_porosity(double phi, double eps_h)
{
    if (phi <= -0.5 * eps_h) return 0.0;
    if (phi >= 0.5 * eps_h) return 1.0;
    return phi / eps_h + 0.5;
}

void orc_hlbm_target(double gamma, const double *Q, double d, const double *uB, const double *BB,
                     double *Qhat)
{
    double rho = Q[0];
    double u[3] = {Q[1] / rho, Q[2] / rho, Q[3] / rho};
    double B[3] = {Q[5], Q[6], Q[7]};
    double p = orc_ideal_pressure(gamma, Q); /* Eq. 9 with the cell's own state */
    double uh[3], Bh[3], uh2 = 0.0, Bh2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        uh[a] = d * u[a] + (1.0 - d) * uB[a];
        Bh[a] = d * B[a] + (1.0 - d) * BB[a];
        uh2 += uh[a] * uh[a];
        Bh2 += Bh[a] * Bh[a];
    }
    Qhat[0] = rho;
    for (int a = 0; a < 3; ++a) {
        Qhat[1 + a] = rho * uh[a];
        Qhat[5 + a] = Bh[a];
    }
    Qhat[4] = p / (gamma - 1.0) + 0.5 * rho * uh2 + 0.5 * Bh2;
}

static void hlbm_collide(const orc_lattice *L, double gamma, const double *tau, const double *src, double d,
                         const double *uB, const double *BB, const double *fin, double *fout)
{
    double Q[ORC_NVAR_IDEAL], Qhat[ORC_NVAR_IDEAL];
    double feq[ORC_NVAR_IDEAL][ORC_QMAX];
    for (int k = 0; k < ORC_NVAR_IDEAL; ++k) {
        Q[k] = 0.0;
        for (int i = 0; i < L->q; ++i) Q[k] += fin[k * L->q + i]; /* Eq. 4 */
    }
    orc_hlbm_target(gamma, Q, d, uB, BB, Qhat);
    ideal_feq(L, gamma, Qhat, feq);
    for (int k = 0; k < ORC_NVAR_IDEAL; ++k)
        for (int i = 0; i < L->q; ++i) {
            double f = fin[k * L->q + i];
            double relaxed = f - (f - feq[k][i]) / tau[k];
            fout[k * L->q + i] = relaxed + (src ? L->w[i] * src[k] : 0.0);
        }
}

int orc_hlbm_step(int dim, int nx, int ny, int nz, double gamma, const double *tau, const double *src,
                  const double *solid, const double *fin, double *fout, int nthreads)
{
    orc_lattice L;
    if (check_dims(dim, nx, ny, nz)) return -1;
    ideal_lattice(dim, &L);
    const long N = (long)nx * ny * nz;
    const int q = L.q;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (long cell = 0; cell < N; ++cell) {
        int x = (int)(cell % nx);
        int y = (int)((cell / nx) % ny);
        int z = (int)(cell / ((long)nx * ny));
        double fc[ORC_NVAR_IDEAL * ORC_QMAX];
        double fs[ORC_NVAR_IDEAL * ORC_QMAX];
        double uB[3], BB[3];
        for (int a = 0; a < 3; ++a) {
            uB[a] = solid[(long)(1 + a) * N + cell];
            BB[a] = solid[(long)(4 + a) * N + cell];
        }
        for (int k = 0; k < ORC_NVAR_IDEAL; ++k)
            for (int i = 0; i < q; ++i) fc[k * q + i] = fin[(long)(k * q + i) * N + cell];
        hlbm_collide(&L, gamma, tau, src, solid[cell], uB, BB, fc, fs);
        for (int i = 0; i < q; ++i) {
            long target = neighbour(x, y, z, L.c[i], nx, ny, nz); /* streaming along c_i */
            for (int k = 0; k < ORC_NVAR_IDEAL; ++k)
                fout[(long)(k * q + i) * N + target] = fs[k * q + i];
        }
    }
    return 0;
}

int orc_hlbm_run(int dim, int nx, int ny, int nz, double gamma, const double *tau, const double *src,
                 const double *solid, const double *Q0, int nsteps, double *Qout, int nthreads)
{
    if (check_dims(dim, nx, ny, nz) || nsteps < 0) return -1;
    int q = dim == 2 ? 5 : 7;
    long N = (long)nx * ny * nz;
    double *a = (double *)malloc(sizeof(double) * ORC_NVAR_IDEAL * q * N);
    double *b = (double *)malloc(sizeof(double) * ORC_NVAR_IDEAL * q * N);
    if (!a || !b) {
        free(a);
        free(b);
        return -2;
    }
    orc_ideal_init(dim, nx, ny, nz, gamma, Q0, a);
    for (int s = 0; s < nsteps; ++s) {
        orc_hlbm_step(dim, nx, ny, nz, gamma, tau, src, solid, a, b, nthreads);
        double *t = a;
        a = b;
        b = t;
    }
    orc_ideal_moments(dim, nx, ny, nz, a, Qout);
    free(a);
    free(b);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Dissipative MHD with locally evolved gradients (sec. 2.2.1, 2.3), 2-D */
/* ------------------------------------------------------------------ */
/*
 * The state of the full MHD system ("Evolution of the MHD equation system")
 * carries, besides the eight fields of Eq. 12, the gradient tensors of the
 * local moments evolution: G_ab ~ tau_M d_a B_b with flux G_ab u_c - delta_ac B_b
 * and source -G_ab / tau_M, and the same construction for the velocity,
 * W_ab ~ tau_M d_a u_b with flux W_ab u_c - delta_ac u_b, from which the
 * viscous stress is built.  a runs over the lattice axes (x, y on D2Q5; x, y, z
 * on D3Q7) and b over x, y, z: Q[8 + 3a + b] = G_ab, Q[8 + 3 dim + 3a + b] = W_ab,
 * 8 + 6 dim lattices (20 in 2-D, 26 in 3-D).
 *
 * Fluxes (the full system of sec. 2.3), with d_a B_b = G_ab / tau_M,
 * d_a u_b = W_ab / tau_M and d_z = 0 in 2-D:
 *   momentum  rho u u + p_tot I - B B - tau_v,   tau_v = rho nu (grad u + grad u^T)
 *   energy    (e + p_tot) u - B (u.B) - u.tau_v + eta j x B   (heat flux zero)
 *   induction u B - B u - eta grad B
 * with j = curl B and eta = eta0 (1 + |j|^2 / j_c^2) (j_c <= 0: eta = eta0).
 * Optional Powell source with div B = (sum_a G_aa) / tau_M.
 */
#define ORC_NVAR_DISS 20   /* 2-D */
#define ORC_NVAR_DISS_MAX 26 /* 3-D */

static int diss_nvar(int dim) { return 8 + 6 * dim; }

static void diss_gradients(int dim, const double *Q, double tau_m, double dB[3][3], double du[3][3])
{
    const int w0 = 8 + 3 * dim;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            dB[a][b] = a < dim ? Q[8 + 3 * a + b] / tau_m : 0.0;
            du[a][b] = a < dim ? Q[w0 + 3 * a + b] / tau_m : 0.0;
        }
}

/* phi[3*k + c]: flux of Q_k along axis c (c = 2 unused in 2-D). */
void orc_diss_flux_d(int dim, double gamma, double nu, double eta0, double j_c, double tau_m, const double *Q,
                     double *phi)
{
    const int w0 = 8 + 3 * dim;
    double rho = Q[0];
    double u[3] = {Q[1] / rho, Q[2] / rho, Q[3] / rho};
    double e = Q[4];
    double B[3] = {Q[5], Q[6], Q[7]};
    double B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double uB = u[0] * B[0] + u[1] * B[1] + u[2] * B[2];
    double p = (gamma - 1.0) * (e - 0.5 * rho * uu - 0.5 * B2); /* Eq. 9 */
    double ptot = 0.5 * B2 + p; /* gas plus magnetic pressure */
    double dB[3][3], du[3][3];
    diss_gradients(dim, Q, tau_m, dB, du);
    double visc[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) visc[a][b] = rho * nu * (du[a][b] + du[b][a]);
    double j[3] = {dB[1][2] - dB[2][1], dB[2][0] - dB[0][2], dB[0][1] - dB[1][0]}; /* curl B */
    double j2 = j[0] * j[0] + j[1] * j[1] + j[2] * j[2];
    double eta = eta0 * (1.0 + (j_c > 0.0 ? j2 / (j_c * j_c) : 0.0));
    double jxB[3] = {j[1] * B[2] - j[2] * B[1], j[2] * B[0] - j[0] * B[2], j[0] * B[1] - j[1] * B[0]};
    for (int c = 0; c < 3; ++c) {
        phi[3 * 0 + c] = rho * u[c];
        double u_visc = 0.0;
        for (int b = 0; b < 3; ++b) {
            phi[3 * (1 + b) + c] = rho * u[c] * u[b] + (b == c ? ptot : 0.0) - B[c] * B[b] - visc[c][b];
            phi[3 * (5 + b) + c] = u[c] * B[b] - B[c] * u[b] - eta * dB[c][b];
            u_visc += u[b] * visc[b][c];
        }
        phi[3 * 4 + c] = (e + ptot) * u[c] - B[c] * uB - u_visc + eta * jxB[c];
        for (int a = 0; a < dim; ++a)
            for (int b = 0; b < 3; ++b) {
                phi[3 * (8 + 3 * a + b) + c] = Q[8 + 3 * a + b] * u[c] - (a == c ? B[b] : 0.0);
                phi[3 * (w0 + 3 * a + b) + c] = Q[w0 + 3 * a + b] * u[c] - (a == c ? u[b] : 0.0);
            }
    }
}

void orc_diss_flux(double gamma, double nu, double eta0, double j_c, double tau_m, const double *Q, double *phi)
{
    orc_diss_flux_d(2, gamma, nu, eta0, j_c, tau_m, Q, phi);
}

/* Sources: relaxation -G/tau_M and -W/tau_M; with powell != 0 also
 * S = -(div B)(0, B, u.B, u) on the eight MHD lattices (sec. 2.3). */
void orc_diss_source_d(int dim, double tau_m, int powell, const double *Q, double *S)
{
    const int nvar = diss_nvar(dim);
    for (int k = 0; k < nvar; ++k) S[k] = 0.0;
    for (int k = 8; k < nvar; ++k) S[k] = -Q[k] / tau_m;
    if (powell) {
        double rho = Q[0];
        double u[3] = {Q[1] / rho, Q[2] / rho, Q[3] / rho};
        double trace = 0.0;
        for (int a = 0; a < dim; ++a) trace += Q[8 + 4 * a]; /* G_aa */
        double minus_div = -trace / tau_m;
        double u_dot_B = u[0] * Q[5] + u[1] * Q[6] + u[2] * Q[7];
        for (int b = 0; b < 3; ++b) {
            S[1 + b] = minus_div * Q[5 + b];
            S[5 + b] = minus_div * u[b];
        }
        S[4] = minus_div * u_dot_B;
    }
}

void orc_diss_source(double tau_m, int powell, const double *Q, double *S)
{
    orc_diss_source_d(2, tau_m, powell, Q, S);
}

static void diss_feq(int dim, const orc_lattice *L, double gamma, double nu, double eta0, double j_c, double tau_m,
                     const double *Q, double feq[ORC_NVAR_DISS_MAX][ORC_QMAX])
{
    double phi[3 * ORC_NVAR_DISS_MAX];
    orc_diss_flux_d(dim, gamma, nu, eta0, j_c, tau_m, Q, phi);
    for (int k = 0; k < diss_nvar(dim); ++k)
        for (int i = 0; i < L->q; ++i) {
            double flux_c = 0.0;
            for (int a = 0; a < 3; ++a) flux_c += L->c[i][a] * phi[3 * k + a];
            feq[k][i] = L->w[i] * (Q[k] + flux_c / L->cs2); /* Eq. 3 */
        }
}

/* tau[nvar]: BGK time per lattice.  Collision with direct source injection. */
static void diss_collide(int dim, const orc_lattice *L, double gamma, const double *tau, double nu, double eta0,
                         double j_c, double tau_m, int powell, const double *fin, double *fout)
{
    const int nvar = diss_nvar(dim);
    double Q[ORC_NVAR_DISS_MAX], S[ORC_NVAR_DISS_MAX];
    double feq[ORC_NVAR_DISS_MAX][ORC_QMAX];
    for (int k = 0; k < nvar; ++k) {
        Q[k] = 0.0;
        for (int i = 0; i < L->q; ++i) Q[k] += fin[k * L->q + i]; /* Eq. 4 */
    }
    diss_feq(dim, L, gamma, nu, eta0, j_c, tau_m, Q, feq);
    orc_diss_source_d(dim, tau_m, powell, Q, S);
    for (int k = 0; k < nvar; ++k)
        for (int i = 0; i < L->q; ++i) {
            double fk = fin[k * L->q + i];
            fout[k * L->q + i] = fk + (feq[k][i] - fk) / tau[k] + L->w[i] * S[k];
        }
}

int orc_diss_init_d(int dim, int nx, int ny, int nz, double gamma, double nu, double eta0, double j_c,
                    double tau_m, const double *Q0, double *f)
{
    orc_lattice L;
    if (check_dims(dim, nx, ny, nz)) return -1;
    build_lattice(dim == 2 ? 5 : 7, &L);
    const int nvar = diss_nvar(dim);
    long N = (long)nx * ny * nz;
    for (long cell = 0; cell < N; ++cell) {
        double Q[ORC_NVAR_DISS_MAX];
        double feq[ORC_NVAR_DISS_MAX][ORC_QMAX];
        for (int k = 0; k < nvar; ++k) Q[k] = Q0[k * N + cell];
        diss_feq(dim, &L, gamma, nu, eta0, j_c, tau_m, Q, feq);
        for (int k = 0; k < nvar; ++k)
            for (int i = 0; i < L.q; ++i) f[(long)(k * L.q + i) * N + cell] = feq[k][i];
    }
    return 0;
}

int orc_diss_init(int nx, int ny, double gamma, double nu, double eta0, double j_c, double tau_m,
                  const double *Q0, double *f)
{
    return orc_diss_init_d(2, nx, ny, 1, gamma, nu, eta0, j_c, tau_m, Q0, f);
}

int orc_diss_step_d(int dim, int nx, int ny, int nz, double gamma, const double *tau, double nu, double eta0,
                    double j_c, double tau_m, int powell, const double *fin, double *fout, int nthreads)
{
    orc_lattice L;
    if (check_dims(dim, nx, ny, nz)) return -1;
    build_lattice(dim == 2 ? 5 : 7, &L);
    const int nvar = diss_nvar(dim);
    const long N = (long)nx * ny * nz;
    const int q = L.q;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (long cell = 0; cell < N; ++cell) {
        int x = (int)(cell % nx);
        int y = (int)((cell / nx) % ny);
        int z = (int)(cell / ((long)nx * ny));
        double fc[ORC_NVAR_DISS_MAX * ORC_QMAX];
        double fs[ORC_NVAR_DISS_MAX * ORC_QMAX];
        for (int k = 0; k < nvar; ++k)
            for (int i = 0; i < q; ++i) fc[k * q + i] = fin[(long)(k * q + i) * N + cell];
        diss_collide(dim, &L, gamma, tau, nu, eta0, j_c, tau_m, powell, fc, fs);
        for (int i = 0; i < q; ++i) {
            long moved = neighbour(x, y, z, L.c[i], nx, ny, nz);
            for (int k = 0; k < nvar; ++k)
                fout[(long)(k * q + i) * N + moved] = fs[k * q + i];
        }
    }
    return 0;
}

int orc_diss_step(int nx, int ny, double gamma, const double *tau, double nu, double eta0, double j_c,
                  double tau_m, int powell, const double *fin, double *fout, int nthreads)
{
    return orc_diss_step_d(2, nx, ny, 1, gamma, tau, nu, eta0, j_c, tau_m, powell, fin, fout, nthreads);
}

int orc_diss_moments_d(int dim, int nx, int ny, int nz, const double *f, double *Q)
{
    if (check_dims(dim, nx, ny, nz)) return -1;
    const int q = dim == 2 ? 5 : 7;
    long N = (long)nx * ny * nz;
    for (int k = 0; k < diss_nvar(dim); ++k)
        for (long cell = 0; cell < N; ++cell) {
            double s = 0.0;
            for (int i = 0; i < q; ++i) s += f[(long)(k * q + i) * N + cell];
            Q[k * N + cell] = s;
        }
    return 0;
}

int orc_diss_moments(int nx, int ny, const double *f, double *Q)
{
    return orc_diss_moments_d(2, nx, ny, 1, f, Q);
}

int orc_diss_run_d(int dim, int nx, int ny, int nz, double gamma, const double *tau, double nu, double eta0,
                   double j_c, double tau_m, int powell, const double *Q0, int nsteps, double *Qout, int nthreads)
{
    if (check_dims(dim, nx, ny, nz) || nsteps < 0) return -1;
    const int q = dim == 2 ? 5 : 7;
    long N = (long)nx * ny * nz;
    size_t len = (size_t)diss_nvar(dim) * q * N;
    double *a = (double *)malloc(sizeof(double) * len);
    double *b = (double *)malloc(sizeof(double) * len);
    if (!a || !b) {
        free(a);
        free(b);
        return -2;
    }
    orc_diss_init_d(dim, nx, ny, nz, gamma, nu, eta0, j_c, tau_m, Q0, a);
    for (int s = 0; s < nsteps; ++s) {
        orc_diss_step_d(dim, nx, ny, nz, gamma, tau, nu, eta0, j_c, tau_m, powell, a, b, nthreads);
        double *t = a;
        a = b;
        b = t;
    }
    orc_diss_moments_d(dim, nx, ny, nz, a, Qout);
    free(a);
    free(b);
    return 0;
}

int orc_diss_run(int nx, int ny, double gamma, const double *tau, double nu, double eta0, double j_c,
                 double tau_m, int powell, const double *Q0, int nsteps, double *Qout, int nthreads)
{
    return orc_diss_run_d(2, nx, ny, 1, gamma, tau, nu, eta0, j_c, tau_m, powell, Q0, nsteps, Qout, nthreads);
}

/* ------------------------------------------------------------------ */
/* Static equilibrium boundaries (sec. 2.4, "Static boundaries")         */
/* ------------------------------------------------------------------ */
/*
 * An axis is periodic or open.  On an open face every state variable is
 * Dirichlet (a set value) or Neumann (the value of the next cell along the
 * boundary's discrete normal); the equilibrium of that boundary state is
 * assigned to the lattice direction that enters the domain across the face.
 *
 * Faces: 0 x-, 1 x+, 2 y-, 3 y+, 4 z-, 5 z+.  open[a] = 1 makes both faces of
 * axis a open.  For face F, bit k of mask[F] set means Q_k = vals[8*F + k];
 * clear means Q_k is copied.  The discrete normal of a cell is the sum of the
 * inward normals of all open faces it lies on (at an edge or a corner it
 * points diagonally inwards), so the copied cell is never on an open face
 * when every open axis has at least three cells.
 *
 * solid (or NULL): homogenised solids [7][N] as in orc_hlbm_step.
 * One step: every cell collides; each post-collision population moves to
 * x + c_i, and one whose destination lies beyond an open face leaves the
 * domain; then every cell on an open face receives, in the direction that
 * enters across that face, f_eq_i of the face's boundary state, built from
 * the streamed (next pre-collision) state of its normal neighbour.
 */
static int on_face(int face, int x, int y, int z, int nx, int ny, int nz)
{
    switch (face) {
    case 0: return x == 0;
    case 1: return x == nx - 1;
    case 2: return y == 0;
    case 3: return y == ny - 1;
    case 4: return z == 0;
    default: return z == nz - 1;
    }
}

int orc_open_step(int dim, int nx, int ny, int nz, double gamma, const double *tau, const double *src,
                  const double *solid, const int *open, const unsigned *mask, const double *vals,
                  const double *fin, double *fout, int nthreads)
{
    orc_lattice L;
    if (check_dims(dim, nx, ny, nz)) return -1;
    const int size[3] = {nx, ny, nz};
    for (int a = 0; a < dim; ++a)
        if (open[a] && size[a] < 3) return -1;
    if (dim == 2 && open[2]) return -1;
    ideal_lattice(dim, &L);
    const long N = (long)nx * ny * nz;
    const int q = L.q;
    if (nthreads < 1) nthreads = 1;
    /* collide and stream; populations leaving across an open face are dropped */
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (long cell = 0; cell < N; ++cell) {
        int x = (int)(cell % nx);
        int y = (int)((cell / nx) % ny);
        int z = (int)(cell / ((long)nx * ny));
        int pos[3] = {x, y, z};
        double fc[ORC_NVAR_IDEAL * ORC_QMAX];
        double fs[ORC_NVAR_IDEAL * ORC_QMAX];
        for (int k = 0; k < ORC_NVAR_IDEAL; ++k)
            for (int i = 0; i < q; ++i) fc[k * q + i] = fin[(long)(k * q + i) * N + cell];
        if (solid) { /* homogenised solids in the domain (sec. 2.4, "Homogenization") */
            double uB[3], BB[3];
            for (int a = 0; a < 3; ++a) {
                uB[a] = solid[(long)(1 + a) * N + cell];
                BB[a] = solid[(long)(4 + a) * N + cell];
            }
            hlbm_collide(&L, gamma, tau, src, solid[cell], uB, BB, fc, fs);
        } else {
            ideal_collide(&L, gamma, tau, src, fc, fs);
        }
        for (int i = 0; i < q; ++i) {
            int leaves = 0;
            for (int a = 0; a < 3; ++a) {
                int to = pos[a] + L.c[i][a];
                if (open[a] && (to < 0 || to >= size[a])) leaves = 1;
            }
            if (leaves) continue;
            long arrive = neighbour(x, y, z, L.c[i], nx, ny, nz);
            for (int k = 0; k < ORC_NVAR_IDEAL; ++k)
                fout[(long)(k * q + i) * N + arrive] = fs[k * q + i];
        }
    }
    /* the directions entering across open faces get the boundary equilibrium */
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (long cell = 0; cell < N; ++cell) {
        int x = (int)(cell % nx);
        int y = (int)((cell / nx) % ny);
        int z = (int)(cell / ((long)nx * ny));
        int normal[3] = {0, 0, 0};
        int any = 0;
        for (int face = 0; face < 2 * dim; ++face) {
            int a = face / 2;
            if (!open[a] || !on_face(face, x, y, z, nx, ny, nz)) continue;
            normal[a] += (face % 2 == 0) ? 1 : -1; /* inward */
            any = 1;
        }
        if (!any) continue;
        long nb = (long)(x + normal[0]) + (long)nx * ((long)(y + normal[1]) + (long)ny * (long)(z + normal[2]));
        double Qn[ORC_NVAR_IDEAL];
        for (int k = 0; k < ORC_NVAR_IDEAL; ++k) {
            Qn[k] = 0.0;
            for (int i = 0; i < q; ++i) Qn[k] += fout[(long)(k * q + i) * N + nb]; /* Eq. 4 */
        }
        for (int face = 0; face < 2 * dim; ++face) {
            int a = face / 2;
            if (!open[a] || !on_face(face, x, y, z, nx, ny, nz)) continue;
            int inward[3] = {0, 0, 0};
            inward[a] = (face % 2 == 0) ? 1 : -1;
            int din = -1;
            for (int i = 0; i < q; ++i)
                if (L.c[i][0] == inward[0] && L.c[i][1] == inward[1] && L.c[i][2] == inward[2]) din = i;
            double Qb[ORC_NVAR_IDEAL];
            double feq[ORC_NVAR_IDEAL][ORC_QMAX];
            for (int k = 0; k < ORC_NVAR_IDEAL; ++k)
                Qb[k] = ((mask[face] >> k) & 1u) ? vals[ORC_NVAR_IDEAL * face + k] : Qn[k];
            ideal_feq(&L, gamma, Qb, feq); /* Eq. 3 */
            for (int k = 0; k < ORC_NVAR_IDEAL; ++k) fout[(long)(k * q + din) * N + cell] = feq[k][din];
        }
    }
    return 0;
}

int orc_open_run(int dim, int nx, int ny, int nz, double gamma, const double *tau, const double *src,
                 const double *solid, const int *open, const unsigned *mask, const double *vals,
                 const double *Q0, int nsteps, double *Qout, int nthreads)
{
    if (check_dims(dim, nx, ny, nz) || nsteps < 0) return -1;
    int q = dim == 2 ? 5 : 7;
    long N = (long)nx * ny * nz;
    double *a = (double *)malloc(sizeof(double) * ORC_NVAR_IDEAL * q * N);
    double *b = (double *)malloc(sizeof(double) * ORC_NVAR_IDEAL * q * N);
    if (!a || !b) {
        free(a);
        free(b);
        return -2;
    }
    orc_ideal_init(dim, nx, ny, nz, gamma, Q0, a);
    int rc = 0;
    for (int s = 0; s < nsteps && rc == 0; ++s) {
        rc = orc_open_step(dim, nx, ny, nz, gamma, tau, src, solid, open, mask, vals, a, b, nthreads);
        double *t = a;
        a = b;
        b = t;
    }
    if (rc == 0) orc_ideal_moments(dim, nx, ny, nz, a, Qout);
    free(a);
    free(b);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Resistive incompressible MHD: D3Q19 flow + three D3Q7 B lattices     */
/* ------------------------------------------------------------------ */
/*
 * State (7 fields): rho, m_x, m_y, m_z (physical momentum, including the
 * half-force shift of the Guo scheme), B_x, B_y, B_z.
 *
 * Flow lattice (D3Q19, BGK):
 *   rho = sum f_i,  m = sum f_i c_i + F/2,  u = m/rho,
 *   Pi  = rho u u + |B|^2/2 I - B B          (momentum flux of sec. 2.3
 *                                             with the Maxwell stress),
 *   f_eq_i = w_i [rho + c_i.m/cs2 + (c_i c_i - cs2 I):Pi/(2 cs2^2)],
 *   f*_i = f_i - (f_i - f_eq_i)/tau_f
 *          + (1 - 1/(2 tau_f)) w_i [(c_i - u)/cs2 + (c_i.u) c_i/cs2^2].F
 * Magnetic lattices (D3Q7, BGK, Eq. 3 with the induction flux of Eq. 12):
 *   B_b = sum_i g_bi,  Phi_{b,a} = u_a B_b - B_a u_b,
 *   g_eq_bi = w_i (B_b + c_i.Phi_b/cs2),  g*_bi = g_bi - (g_bi - g_eq_bi)/tau_m.
 * Walls (walls_y != 0): rows y = 0 and y = ny-1 are solid.  Flow: halfway
 * bounce-back, a population leaving fluid cell x towards a wall returns to x
 * in the opposite direction.  B: wall cells emit the equilibrium of the
 * applied field at rest, g_bi = w_i b_wall_b (equilibrium Dirichlet of
 * sec. 2.4, "Static boundaries").
 */
#define ORC_NVAR_RES 7

static int is_wall(int y, int ny, int walls_y)
{
    return walls_y && (y == 0 || y == ny - 1);
}

static void res_flow_feq(const orc_lattice *L, double rho, const double *m, const double *B,
                         double *feq)
{
    double u[3] = {m[0] / rho, m[1] / rho, m[2] / rho};
    double B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    double Pi[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            Pi[a][b] = rho * u[a] * u[b] + (a == b ? 0.5 * B2 : 0.0) - B[a] * B[b];
    for (int i = 0; i < L->q; ++i) {
        double cm = 0.0, second = 0.0;
        for (int a = 0; a < 3; ++a) cm += L->c[i][a] * m[a];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                second += (L->c[i][a] * L->c[i][b] - (a == b ? L->cs2 : 0.0)) * Pi[a][b];
        feq[i] = L->w[i] * (rho + cm / L->cs2 + second / (2.0 * L->cs2 * L->cs2));
    }
}

static void res_mag_feq(const orc_lattice *L7, const double *u, const double *B, double feq[3][7])
{
    for (int b = 0; b < 3; ++b) {
        double phi[3];
        for (int a = 0; a < 3; ++a) phi[a] = u[a] * B[b] - B[a] * u[b];
        for (int i = 0; i < L7->q; ++i) {
            double cphi = 0.0;
            for (int a = 0; a < 3; ++a) cphi += L7->c[i][a] * phi[a];
            feq[b][i] = L7->w[i] * (B[b] + cphi / L7->cs2);
        }
    }
}

/* Collision of one fluid cell of the resistive model (see the model block
 * above): moments, equilibria, BGK and the Guo force term. */
static void res_collide(const orc_lattice *L19, const orc_lattice *L7, double tau_f, double tau_m,
                        const double *force, const double *fl, double gl[3][7], double *fs,
                        double gs[3][7])
{
    double rho = 0.0, m[3] = {0, 0, 0}, B[3] = {0, 0, 0}, u[3];
    for (int i = 0; i < 19; ++i) {
        rho += fl[i];
        for (int a = 0; a < 3; ++a) m[a] += fl[i] * L19->c[i][a];
    }
    for (int a = 0; a < 3; ++a) {
        m[a] += 0.5 * force[a];
        u[a] = m[a] / rho;
    }
    for (int b = 0; b < 3; ++b)
        for (int i = 0; i < 7; ++i) B[b] += gl[b][i];
    double feq[ORC_QMAX], geq[3][7];
    res_flow_feq(L19, rho, m, B, feq);
    res_mag_feq(L7, u, B, geq);
    for (int i = 0; i < 19; ++i) {
        double cu = 0.0, cF = 0.0, cuF = 0.0;
        for (int a = 0; a < 3; ++a) {
            cu += L19->c[i][a] * u[a];
            cF += L19->c[i][a] * force[a];
            cuF += u[a] * force[a];
        }
        double guo = (1.0 - 0.5 / tau_f) * L19->w[i] *
                     ((cF - cuF) / L19->cs2 + cu * cF / (L19->cs2 * L19->cs2));
        fs[i] = fl[i] - (fl[i] - feq[i]) / tau_f + guo;
    }
    for (int b = 0; b < 3; ++b)
        for (int i = 0; i < 7; ++i) gs[b][i] = gl[b][i] - (gl[b][i] - geq[b][i]) / tau_m;
}

/* Single fluid-cell collision, exported for sampled parity checks:
 * fin = 19 flow then 21 magnetic populations, fout likewise. */
int orc_resistive_collide_cell(double tau_f, double tau_m, const double *force, const double *fin,
                               double *fout)
{
    orc_lattice L19, L7;
    build_lattice(19, &L19);
    build_lattice(7, &L7);
    double gl[3][7], gs[3][7];
    for (int b = 0; b < 3; ++b)
        for (int i = 0; i < 7; ++i) gl[b][i] = fin[19 + 7 * b + i];
    res_collide(&L19, &L7, tau_f, tau_m, force, fin, gl, fout, gs);
    for (int b = 0; b < 3; ++b)
        for (int i = 0; i < 7; ++i) fout[19 + 7 * b + i] = gs[b][i];
    return 0;
}

/* Initial populations from the state: flow f = f_eq(rho, m - F/2, B), so
 * that the momentum moment (sum f c + F/2) returns m; B lattices g = g_eq. */
int orc_resistive_init(int nx, int ny, int nz, const double *Qr, const double *force,
                       double *f, double *g)
{
    orc_lattice L19, L7;
    if (check_dims(3, nx, ny, nz)) return -1;
    build_lattice(19, &L19);
    build_lattice(7, &L7);
    long N = (long)nx * ny * nz;
    for (long cell = 0; cell < N; ++cell) {
        double rho = Qr[0 * N + cell];
        double m[3], j[3], B[3], u[3];
        for (int a = 0; a < 3; ++a) {
            m[a] = Qr[(1 + a) * N + cell];
            B[a] = Qr[(4 + a) * N + cell];
            j[a] = m[a] - 0.5 * force[a];
            u[a] = m[a] / rho;
        }
        double feq[ORC_QMAX], geq[3][7];
        res_flow_feq(&L19, rho, j, B, feq);
        res_mag_feq(&L7, u, B, geq);
        for (int i = 0; i < 19; ++i) f[(long)i * N + cell] = feq[i];
        for (int b = 0; b < 3; ++b)
            for (int i = 0; i < 7; ++i) g[(long)(b * 7 + i) * N + cell] = geq[b][i];
    }
    return 0;
}

int orc_resistive_step(int nx, int ny, int nz, double tau_f, double tau_m, const double *force,
                       const double *b_wall, int walls_y, const double *fin, const double *gin,
                       double *fout, double *gout, int nthreads)
{
    orc_lattice L19, L7;
    if (check_dims(3, nx, ny, nz)) return -1;
    if (walls_y && ny < 3) return -1;
    build_lattice(19, &L19);
    build_lattice(7, &L7);
    const long N = (long)nx * ny * nz;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (long cell = 0; cell < N; ++cell) {
        int x = (int)(cell % nx);
        int y = (int)((cell / nx) % ny);
        int z = (int)(cell / ((long)nx * ny));
        if (is_wall(y, ny, walls_y)) {
            /* magnetic wall: emit g_eq(B = b_wall, u = 0) = w_i b_wall */
            for (int i = 0; i < 7; ++i) {
                long dst = neighbour(x, y, z, L7.c[i], nx, ny, nz);
                for (int b = 0; b < 3; ++b) gout[(long)(b * 7 + i) * N + dst] = L7.w[i] * b_wall[b];
            }
            continue;
        }
        double fl[ORC_QMAX], gl[3][7], fs[ORC_QMAX], gs[3][7];
        for (int i = 0; i < 19; ++i) fl[i] = fin[(long)i * N + cell];
        for (int b = 0; b < 3; ++b)
            for (int i = 0; i < 7; ++i) gl[b][i] = gin[(long)(b * 7 + i) * N + cell];
        res_collide(&L19, &L7, tau_f, tau_m, force, fl, gl, fs, gs);
        for (int i = 0; i < 19; ++i) {
            long dst = neighbour(x, y, z, L19.c[i], nx, ny, nz);
            int dy = (y + L19.c[i][1] + ny) % ny;
            if (is_wall(dy, ny, walls_y))
                fout[(long)L19.opp[i] * N + cell] = fs[i]; /* halfway bounce-back */
            else
                fout[(long)i * N + dst] = fs[i];
        }
        for (int i = 0; i < 7; ++i) {
            long dst = neighbour(x, y, z, L7.c[i], nx, ny, nz);
            for (int b = 0; b < 3; ++b) gout[(long)(b * 7 + i) * N + dst] = gs[b][i];
        }
    }
    return 0;
}

/* Moments of the resistive state; wall cells report (1, 0, 0, 0, b_wall). */
int orc_resistive_moments(int nx, int ny, int nz, const double *force, const double *b_wall,
                          int walls_y, const double *f, const double *g, double *Qr)
{
    orc_lattice L19, L7;
    if (check_dims(3, nx, ny, nz)) return -1;
    build_lattice(19, &L19);
    build_lattice(7, &L7);
    long N = (long)nx * ny * nz;
    for (long cell = 0; cell < N; ++cell) {
        int y = (int)((cell / nx) % ny);
        if (is_wall(y, ny, walls_y)) {
            Qr[0 * N + cell] = 1.0;
            for (int a = 0; a < 3; ++a) {
                Qr[(1 + a) * N + cell] = 0.0;
                Qr[(4 + a) * N + cell] = b_wall[a];
            }
            continue;
        }
        double rho = 0.0, m[3] = {0, 0, 0};
        for (int i = 0; i < 19; ++i) {
            double v = f[(long)i * N + cell];
            rho += v;
            for (int a = 0; a < 3; ++a) m[a] += v * L19.c[i][a];
        }
        Qr[0 * N + cell] = rho;
        for (int a = 0; a < 3; ++a) Qr[(1 + a) * N + cell] = m[a] + 0.5 * force[a];
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int i = 0; i < 7; ++i) s += g[(long)(b * 7 + i) * N + cell];
            Qr[(4 + b) * N + cell] = s;
        }
    }
    return 0;
}

int orc_resistive_run(int nx, int ny, int nz, double tau_f, double tau_m, const double *force,
                      const double *b_wall, int walls_y, const double *Q0, int nsteps,
                      double *Qout, int nthreads)
{
    if (check_dims(3, nx, ny, nz) || nsteps < 0) return -1;
    long N = (long)nx * ny * nz;
    double *fa = (double *)malloc(sizeof(double) * 19 * N);
    double *fb = (double *)malloc(sizeof(double) * 19 * N);
    double *ga = (double *)malloc(sizeof(double) * 21 * N);
    double *gb = (double *)malloc(sizeof(double) * 21 * N);
    if (!fa || !fb || !ga || !gb) {
        free(fa);
        free(fb);
        free(ga);
        free(gb);
        return -2;
    }
    orc_resistive_init(nx, ny, nz, Q0, force, fa, ga);
    /* wall slots that no step writes keep their initial values */
    memcpy(fb, fa, sizeof(double) * 19 * N);
    memcpy(gb, ga, sizeof(double) * 21 * N);
    int rc = 0;
    for (int s = 0; s < nsteps && rc == 0; ++s) {
        rc = orc_resistive_step(nx, ny, nz, tau_f, tau_m, force, b_wall, walls_y, fa, ga, fb, gb,
                                nthreads);
        double *t = fa;
        fa = fb;
        fb = t;
        t = ga;
        ga = gb;
        gb = t;
    }
    if (rc == 0) orc_resistive_moments(nx, ny, nz, force, b_wall, walls_y, fa, ga, Qout);
    free(fa);
    free(fb);
    free(ga);
    free(gb);
    return rc;
}
