/* A plain C user of the library: no Python and no PyTorch in the process.
 *
 * 2-D ideal MHD (eight fields, D2Q5), 64 x 48 periodic cells, FP64 storage:
 * a uniform state with a small density wave, 50 steps through vlbm_step, and
 * two checks the scheme fixes exactly -- every domain sum is conserved (to
 * FP64 round-off), and a uniform state is a fixed point.  Prints one line
 * starting "c-abi ok" and exits 0 when both hold; exits 1 otherwise.
 *
 * Built by the tests with the system C compiler against include/vlbm.h and
 * the in-tree libvlbm.so. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "vlbm.h"

enum { NX = 64, NY = 48, STEPS = 50 };

static int fail(const char *what, vlbm_status s, vlbm_ctx *ctx)
{
    fprintf(stderr, "%s: %s (%s)\n", what, vlbm_status_string(s), ctx ? vlbm_last_error(ctx) : "");
    return 1;
}

/* Q[8][NY][NX]: rho, rho u, e_tot, B with p = 0.1 and gamma = 5/3 */
static void fields(double *Q, double amp)
{
    const double gamma = 5.0 / 3.0, p = 0.1;
    const double u[3] = {0.01, 0.005, 0.0}, B[3] = {0.02, 0.01, 0.005};
    const double pi = 3.14159265358979323846;
    const long N = (long)NX * NY;
    for (int y = 0; y < NY; ++y)
        for (int x = 0; x < NX; ++x) {
            const long c = x + (long)NX * y;
            const double rho = 1.0 + amp * sin(2.0 * pi * x / NX) * cos(2.0 * pi * y / NY);
            double u2 = 0.0, B2 = 0.0;
            Q[c] = rho;
            for (int a = 0; a < 3; ++a) {
                Q[(1 + a) * N + c] = rho * u[a];
                Q[(5 + a) * N + c] = B[a];
                u2 += u[a] * u[a];
                B2 += B[a] * B[a];
            }
            Q[4 * N + c] = p / (gamma - 1.0) + 0.5 * rho * u2 + 0.5 * B2;
        }
}

static int run(double amp, double *Q, double *out, double s0[8], double s1[8])
{
    vlbm_params p;
    vlbm_default_params(&p);
    p.model = VLBM_IDEAL;
    p.dim = 2;
    p.nx = NX;
    p.ny = NY;
    p.nz = 1;
    p.storage = VLBM_F64;
    p.gamma = 5.0 / 3.0;
    for (int k = 0; k < 8; ++k) p.tau[k] = 0.6;
    vlbm_ctx *ctx = NULL;
    vlbm_status s = vlbm_create(&p, &ctx);
    if (s != VLBM_OK) return fail("vlbm_create", s, ctx);
    fields(Q, amp);
    if ((s = vlbm_init_fields(ctx, 0, Q)) != VLBM_OK) return fail("vlbm_init_fields", s, ctx);
    if ((s = vlbm_conservation(ctx, 0, s0)) != VLBM_OK) return fail("vlbm_conservation", s, ctx);
    if ((s = vlbm_step(ctx, STEPS)) != VLBM_OK) return fail("vlbm_step", s, ctx);
    if ((s = vlbm_sync(ctx)) != VLBM_OK) return fail("vlbm_sync", s, ctx);
    if ((s = vlbm_conservation(ctx, 0, s1)) != VLBM_OK) return fail("vlbm_conservation", s, ctx);
    if ((s = vlbm_moments(ctx, 0, out)) != VLBM_OK) return fail("vlbm_moments", s, ctx);
    vlbm_destroy(ctx);
    return 0;
}

int main(void)
{
    const long N = (long)NX * NY;
    double *Q = malloc(sizeof(double) * 8 * N), *out = malloc(sizeof(double) * 8 * N);
    double s0[8], s1[8];
    if (!Q || !out) return 1;

    /* a density wave: every domain sum stays put (collision keeps each cell's moments,
       streaming permutes populations on the periodic grid) */
    if (run(0.01, Q, out, s0, s1)) return 1;
    double worst = 0.0;
    for (int k = 0; k < 8; ++k) {
        double mag = 0.0;
        for (long c = 0; c < N; ++c) mag += fabs(Q[k * N + c]);
        const double rel = mag > 0.0 ? fabs(s1[k] - s0[k]) / mag : fabs(s1[k] - s0[k]);
        if (!(rel <= 1e-12)) {
            fprintf(stderr, "field %d: sum moved by %g of sum |Q|\n", k, rel);
            return 1;
        }
        if (rel > worst) worst = rel;
    }
    for (long i = 0; i < 8 * N; ++i)
        if (!isfinite(out[i])) {
            fprintf(stderr, "non-finite moment at %ld\n", i);
            return 1;
        }

    /* a uniform state: a fixed point of the update */
    if (run(0.0, Q, out, s0, s1)) return 1;
    double drift = 0.0;
    for (long i = 0; i < 8 * N; ++i) {  /* relative, with a floor for the zero fields (rho u_z) */
        const double d = fabs(out[i] - Q[i]) / fmax(fabs(Q[i]), 1e-3);
        if (d > drift) drift = d;
    }
    if (!(drift <= 1e-13)) {
        fprintf(stderr, "uniform state drifted by %g\n", drift);
        return 1;
    }
    printf("c-abi ok: %d steps, worst sum drift %.2e, uniform drift %.2e\n", STEPS, worst, drift);
    free(Q);
    free(out);
    return 0;
}
