/*
 * masw_client.c -- a plain C11 client of libmasw (no Python, no C++), used by
 * the tests to show that the C ABI of include/masw.h stands on its own.
 *
 * Two layered models on host buffers go through masw_model_batch_create,
 * masw_dispersion (Algorithm 1), masw_misfit (Algorithm 2, least squares),
 * masw_dispersion_leaky and masw_model_batch_destroy. Output, one record per
 * line: "idx <item> <grid index> <status>", "leaky <item> <grid index>
 * <status>", "misfit <model> <value>". Exit status 0 on success, 1 with the
 * library's message on stderr otherwise.
 */
#include <stdio.h>

#include "masw.h"

static int check(int rc, const char* what) {
    if (rc != MASW_OK) fprintf(stderr, "%s: %s\n", what, masw_strerror(rc));
    return rc != MASW_OK;
}

int main(void) {
    /* model 0: 2 layers over a half-space; model 1: 1 layer over a half-space */
    const int32_t n_layers[2] = {2, 1};
    const double h[3] = {2.0, 4.0, 3.0};
    const double alpha[5] = {400.0, 600.0, 800.0, 450.0, 900.0};
    const double beta[5] = {180.0, 260.0, 380.0, 200.0, 420.0};
    const double rho[5] = {1850.0, 1900.0, 2000.0, 1800.0, 2000.0};
    const int32_t n_lambda[2] = {3, 2};
    const double lambda[5] = {2.0, 10.0, 40.0, 5.0, 25.0};
    const masw_models_desc md = {2, n_layers, h, alpha, beta, rho, n_lambda, lambda, MASW_HOST};
    const masw_grid grid = {50.0, 0.5, 1500};
    masw_batch* batch = NULL;
    if (check(masw_model_batch_create(&md, &grid, NULL, &batch), "create")) return 1;

    double ct[5], ct_l[5], misfit[2];
    int32_t idx[5], status[5], idx_l[5], status_l[5];
    int bad = check(masw_dispersion(batch, ct, idx, status, MASW_HOST), "dispersion");
    if (!bad) {
        double ce[5];
        for (int i = 0; i < 5; ++i) ce[i] = ct[i] + 1.0; /* an observed curve 1 m/s above */
        bad = check(masw_misfit(batch, ce, MASW_MISFIT_LSQ, 2.0, misfit), "misfit");
    }
    if (!bad) bad = check(masw_dispersion_leaky(batch, ct_l, idx_l, status_l, MASW_HOST), "leaky");
    if (!bad) {
        for (int i = 0; i < 5; ++i) printf("idx %d %d %d\n", i, (int)idx[i], (int)status[i]);
        for (int i = 0; i < 5; ++i) printf("leaky %d %d %d\n", i, (int)idx_l[i], (int)status_l[i]);
        for (int m = 0; m < 2; ++m) printf("misfit %d %.17g\n", m, misfit[m]);
    }
    if (check(masw_model_batch_destroy(batch), "destroy")) bad = 1;
    return bad;
}
