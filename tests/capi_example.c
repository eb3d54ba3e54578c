/*
 * A plain C99 user of the C-ABI (include/nb.h), built and run by the tests:
 * the softened_general worked example of tests/golden/pair_worked_examples.txt
 * (m_i = 10, m_j = 5, r = (0,4,0), v = (0,2,1), a = (1,1,0), eps = 3) through
 * nb_init / nb_set_state / nb_predict / nb_evaluate, its energy through
 * nb_energy (E_kin = 12.5 and E_pot = -10 in closed form), then, in a fresh
 * context started from the library's own forces, an integration to t = 1/4
 * with nb_run_until.
 *
 * Usage: capi_example PRECISION   (0 FP64, 1 mixed, 3 EX)
 * Prints "key value..." lines; exits 1 with the library's message on error.
 */
#include <stdio.h>
#include <stdlib.h>

#include "nb.h"

static int check(nb_status st, const nb_ctx *ctx, const char *what)
{
    if (st == NB_OK)
        return 0;
    fprintf(stderr, "%s failed (%d): %s\n", what, (int)st, nb_last_error(ctx));
    return 1;
}

static void print3(const char *key, const double *v)
{
    printf("%s %.17g %.17g %.17g\n", key, v[0], v[1], v[2]);
}

int main(int argc, char **argv)
{
    const double m[2] = {10.0, 5.0};
    const double x[6] = {0, 0, 0, 0, 4, 0};
    const double v[6] = {0, 0, 0, 0, 2, 1};
    const double a[6] = {0, 0, 0, 1, 1, 0};
    const double zero[6] = {0, 0, 0, 0, 0, 0};
    const double t[2] = {0, 0};
    const double dt[2] = {0.125, 0.125};
    const int32_t active[2] = {0, 1};
    double acc[6], jerk[6], snap[6], ekin, epot, tt[2];
    int64_t steps = 0;
    nb_config cfg;
    nb_ctx *ctx = NULL;
    int bad;

    nb_config_default(&cfg);
    cfg.precision = (nb_precision)(argc > 1 ? atoi(argv[1]) : 0);
    cfg.start_forces = 0;
    if (check(nb_init(&ctx, 2, m, x, v, 3.0, &cfg), NULL, "nb_init"))
        return 1;
    bad = check(nb_set_state(ctx, x, v, a, zero, zero, zero, t, dt), ctx, "nb_set_state") ||
          check(nb_predict(ctx, 0.0), ctx, "nb_predict") ||
          check(nb_evaluate(ctx, active, 2, 0, acc, jerk, snap, 0), ctx, "nb_evaluate") ||
          check(nb_energy(ctx, &ekin, &epot), ctx, "nb_energy");
    if (!bad) {
        print3("acc", acc);
        print3("jerk", jerk);
        print3("snap", snap);
        print3("acc_j", acc + 3);
        printf("ekin %.17g\nepot %.17g\n", ekin, epot);
    }
    nb_free(ctx);
    ctx = NULL;
    if (bad)
        return 1;

    /* a fresh context with the library's own start-up forces, integrated */
    cfg.start_forces = 1;
    if (check(nb_init(&ctx, 2, m, x, v, 3.0, &cfg), NULL, "nb_init"))
        return 1;
    bad = check(nb_run_until(ctx, 0.25, &steps, 0, NULL, NULL), ctx, "nb_run_until") ||
          check(nb_get_state(ctx, NULL, NULL, NULL, NULL, NULL, NULL, tt, NULL), ctx,
                "nb_get_state");
    if (!bad)
        printf("steps %lld\nt %.17g %.17g\n", (long long)steps, tt[0], tt[1]);
    nb_free(ctx);
    return bad;
}
