/* A plain C99 client of include/dirac.h: the header compiles as C, the
 * library links, and the calls that need no GPU behave as documented. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "dirac.h"

static int failures = 0;

static void check(int ok, const char* what) {
    if (!ok) {
        printf("FAIL %s\n", what);
        ++failures;
    }
}

int main(void) {
    /* status strings and the thread's last error */
    check(strcmp(dirac_status_string(DIRAC_OK), "ok") == 0, "status string of DIRAC_OK");
    check(dirac_last_error() != NULL, "last error is a string");

    /* argument validation before any device work */
    dirac_ctx* ctx = NULL;
    check(dirac_create(&ctx, 0, 8, 0.1, 0.1, 1.0, 137.036, 2, DIRAC_PERIODIC, DIRAC_FP64, 4, NULL)
              == DIRAC_EINVAL, "nx = 0 rejected");
    check(dirac_create(&ctx, 8, 8, 0.1, 0.1, 1.0, 137.036, 3, DIRAC_PERIODIC, DIRAC_FP64, 4, NULL)
              == DIRAC_EINVAL, "stencil order 3 rejected");
    check(dirac_create(&ctx, 8, 8, 0.1, 0.1, 1.0, 137.036, 2, DIRAC_PERIODIC, DIRAC_FP64,
                       DIRAC_KRYLOV_MAX + 1, NULL) == DIRAC_EINVAL, "m_max above the limit rejected");
    check(dirac_lanczos_step(NULL, NULL, 1e-4, 4, 0.0, NULL) == DIRAC_EINVAL, "null context");
    check(dirac_set_step_mode(NULL, DIRAC_STEP_AUTO) == DIRAC_EINVAL, "null context (step mode)");
    check(dirac_state_bytes(NULL) == 0, "state size of no context");
    dirac_destroy(NULL);

    /* closed-form helpers (host only) */
    const double a = dirac_pulse_sin2_mean(0.25, 2e-4, 50.0, 0.05, 1.0);
    check(isfinite(a) && a > 0.0, "pulse step mean");
    check(dirac_pulse_sin2_mean(2.0, 2e-4, 50.0, 0.05, 1.0) == 0.0, "pulse is zero after it ends");
    double W[6];
    check(dirac_pulse_sine_basis_means(2, 0.1, 3, 1.0, W) == DIRAC_OK, "sine basis means");
    /* the step mean of sin(pi t) over [0, 0.1] is (1 - cos(0.1 pi)) / (0.1 pi) */
    const double pi = 3.14159265358979323846;
    check(fabs(W[0] - (1.0 - cos(0.1 * pi)) / (0.1 * pi)) < 1e-14, "first basis mean in closed form");
    check(dirac_kernel_launches(NULL) == 0, "no launches without a context");

    printf("%s (%d failures)\n", failures ? "abi_check FAILED" : "abi_check ok", failures);
    return failures ? 1 : 0;
}
