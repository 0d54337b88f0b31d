/* A plain C program on the library's C ABI (no Python, no PyTorch): sets up
 * the ring of Section 4 with degree p and nel elements per direction, solves
 * K~ u = f for the forcing of Eq. (exact-solution) with FD-preconditioned
 * BiCGStab through host buffers, and prints the iteration count, the residual
 * and the relative H1 error.  Usage: solve_ring [p] [nel] [rtol]. */
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>

#include "mfwq.h"

#define CHECK(call)                                                                    \
    do {                                                                               \
        int st_ = (call);                                                              \
        if (st_ != MFWQ_OK) {                                                          \
            fprintf(stderr, "%s failed: %s (%s)\n", #call, mfwq_status_string(st_),    \
                    mfwq_last_error());                                                \
            return 2;                                                                  \
        }                                                                              \
    } while (0)

int main(int argc, char** argv) {
    const int p = argc > 1 ? atoi(argv[1]) : 3;
    const int nel = argc > 2 ? atoi(argv[2]) : 16;
    const double rtol = argc > 3 ? atof(argv[3]) : 1e-10;
    const int nk = nel + 2 * p + 1;
    double* knots = (double*)malloc(sizeof(double) * nk);
    for (int i = 0; i < nk; ++i) {
        const int k = i - p;  /* p+1 zeros, k/nel for k = 1..nel-1, p+1 ones */
        knots[i] = k <= 0 ? 0.0 : (k >= nel ? 1.0 : (double)k / nel);
    }
    mfwq_setup_desc d = {{p, p, p}, {nk, nk, nk}, {knots, knots, knots}, 0, MFWQ_FD_TF32, NULL};
    mfwq_handle h = NULL;
    CHECK(mfwq_setup(&d, &h));
    int n[3], nq[3];
    CHECK(mfwq_sizes(h, n, nq));
    const size_t N = (size_t)n[0] * n[1] * n[2], Nq = (size_t)nq[0] * nq[1] * nq[2];
    double *C = NULL, *f = NULL;
    if (cudaMalloc((void**)&C, sizeof(double) * 6 * Nq) != cudaSuccess ||
        cudaMalloc((void**)&f, sizeof(double) * N) != cudaSuccess) {
        fprintf(stderr, "cudaMalloc failed\n");
        return 2;
    }
    CHECK(mfwq_eval_coeff(h, MFWQ_GEOM_RING, NULL, 0, 0.0, C));
    CHECK(mfwq_set_coeff(h, C));
    CHECK(mfwq_load_vector(h, MFWQ_GEOM_RING, MFWQ_FORCING_RING_EXACT, f));
    CHECK(mfwq_sync(h));
    double* fh = (double*)malloc(sizeof(double) * N);
    double* uh = (double*)malloc(sizeof(double) * N);
    cudaMemcpy(fh, f, sizeof(double) * N, cudaMemcpyDeviceToHost);
    mfwq_solve_opts o = {.rtol = rtol, .maxit = 1000, .res_hist = NULL};
    mfwq_solve_info info;
    const int st = mfwq_solve_host(h, fh, uh, &o, &info);
    if (st != MFWQ_OK) {
        fprintf(stderr, "solve: %s\n", mfwq_status_string(st));
        return 1;
    }
    cudaMemcpy(f, uh, sizeof(double) * N, cudaMemcpyHostToDevice); /* u back on the device */
    double err = 0.0;
    CHECK(mfwq_h1_error(h, MFWQ_GEOM_RING, MFWQ_EXACT_RING, f, &err));
    printf("n %d %d %d iterations %d rel_residual %.6e h1_error %.15e\n", n[0], n[1], n[2], info.iterations,
           info.rel_residual, err);
    mfwq_destroy(h);
    cudaFree(C);
    cudaFree(f);
    free(fh);
    free(uh);
    free(knots);
    return 0;
}
