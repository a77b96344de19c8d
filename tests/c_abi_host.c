/* A plain C99 client of include/admm.h: it compiles against the header,
 * links libadmm.so and makes the calls that need no GPU (defaults, status
 * strings, argument checks).  Exit status 0 when every check holds. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "admm.h"

#define CHECK(c)                                                   \
    do {                                                           \
        if (!(c)) {                                                \
            fprintf(stderr, "check failed line %d: %s\n", __LINE__, #c); \
            return 1;                                              \
        }                                                          \
    } while (0)

int main(void)
{
    admm_params p;
    memset(&p, 0xff, sizeof p);
    admm_default_params(&p);
    CHECK(p.max_iter == 5000 && p.check_every == 10);
    CHECK(p.rho[0] == 1.0 && p.rho[3] == 1.0 && p.r_tol == 1e-6 && fabs(p.tau - 1.1) < 1e-15);
    CHECK(p.precision == ADMM_FP64 && p.xmin_mode == ADMM_XMIN_EXACT && p.sweep == ADMM_GAUSS_SEIDEL);
    CHECK(p.adapt_start == 0 && p.reserved[0] == 0 && p.reserved[1] == 0);

    admm_handle *h = NULL;
    CHECK(admm_create(NULL, &p, &h) == ADMM_EINVAL && h == NULL);
    CHECK(strlen(admm_last_error()) > 0);
    CHECK(admm_solve(NULL, NULL, NULL, NULL) == ADMM_EINVAL);
    CHECK(admm_destroy(NULL) == ADMM_OK);

    admm_server_config sc;
    admm_server_default_config(&sc);
    CHECK(sc.tick_iters == 10 && sc.max_active == 4096 && sc.batch.warps_per_cta == 8);
    admm_server *s = NULL;
    p.precision = ADMM_FP64;
    CHECK(admm_server_create(&p, &sc, &s) == ADMM_EUNSUPPORTED && s == NULL);
    CHECK(admm_batch_destroy(NULL) == ADMM_OK && admm_server_destroy(NULL) == ADMM_OK);

    for (int st = ADMM_OK; st <= ADMM_ECANCELLED; ++st)
        CHECK(admm_status_string((admm_status)st) != NULL && strlen(admm_status_string((admm_status)st)) > 0);
    CHECK(sizeof(admm_problem) == 16 + 10 * sizeof(void *) + 8);
    printf("c client ok\n");
    return 0;
}
