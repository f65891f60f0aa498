/* A plain C99 client that propagates through include/dirac.h with device
 * memory from the CUDA runtime: a Gaussian packet, ten FP64 steps in a
 * static field, then the norm (the step is unitary: Sec. 4) and the
 * diagnostics are checked. */
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "dirac.h"

int main(void) {
    const int nx = 64, ny = 48, m = 10, steps = 10;
    const double dx = 0.1, dt = 1e-4;
    const size_t n = (size_t)nx * ny;
    double* h = (double*)malloc(n * 4 * sizeof(double));
    double norm0 = 0.0;
    for (int l = 0; l < ny; ++l)
        for (int j = 0; j < nx; ++j) {
            const double x = (j - nx / 2) * dx, y = (l - ny / 2) * dx;
            const double g = exp(-(x * x + y * y) / 2.0);
            double* s = h + 4 * ((size_t)l * nx + j);
            s[0] = g * cos(3.0 * x); s[1] = g * sin(3.0 * x);   /* upper: e^{i 3 x} */
            s[2] = 0.01 * g;         s[3] = 0.0;                /* a small lower part */
            norm0 += s[0] * s[0] + s[1] * s[1] + s[2] * s[2] + s[3] * s[3];
        }
    void* d = NULL;
    if (cudaMalloc(&d, n * 4 * sizeof(double)) != cudaSuccess) { printf("cudaMalloc failed\n"); return 2; }
    cudaMemcpy(d, h, n * 4 * sizeof(double), cudaMemcpyHostToDevice);

    dirac_ctx* ctx = NULL;
    int bad = 0;
    dirac_status s = dirac_create(&ctx, nx, ny, dx, dx, 1.0, 137.036, 2, DIRAC_PERIODIC, DIRAC_FP64, m, NULL);
    if (s != DIRAC_OK) { printf("create: %s\n", dirac_last_error()); return 3; }
    s = dirac_set_fields(ctx, NULL, 2.0, -1.0, 0.0);
    if (s != DIRAC_OK) { printf("set_fields: %s\n", dirac_last_error()); return 4; }
    dirac_step_info info;
    s = dirac_lanczos_steps(ctx, d, steps, dt, m, 0.0, NULL, &info);
    if (s != DIRAC_OK) { printf("steps: %s\n", dirac_last_error()); return 5; }
    cudaMemcpy(h, d, n * 4 * sizeof(double), cudaMemcpyDeviceToHost);
    double norm1 = 0.0;
    for (size_t i = 0; i < 4 * n; ++i) norm1 += h[i] * h[i];
    const double drift = fabs(sqrt(norm1) - sqrt(norm0)) / sqrt(norm0);
    if (!(drift < 1e-12)) { printf("norm drift %g\n", drift); bad = 1; }
    if (info.k_used != m) { printf("k_used %d\n", info.k_used); bad = 1; }
    if (!(info.err_est >= 0.0 && info.err_est < 1e-12 * info.norm)) { printf("err_est %g\n", info.err_est); bad = 1; }
    if (!isfinite(info.energy)) { printf("energy not finite\n"); bad = 1; }
    if (dirac_kernel_launches(ctx) <= 0) { printf("no kernel launches counted\n"); bad = 1; }
    dirac_destroy(ctx);
    cudaFree(d);
    free(h);
    printf("%s: norm drift %.3e, k_used %d, energy %.6f, err_est %.3e\n",
           bad ? "propagate_check FAILED" : "propagate_check ok", drift, info.k_used, info.energy, info.err_est);
    return bad;
}
