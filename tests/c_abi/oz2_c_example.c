/*
 * A plain C client of liboz2.so: device buffers from the CUDA runtime, the
 * emulated DGEMM through the C ABI only (no Python, no torch).
 *
 * Integer-valued inputs with entries in [-5, 5] make A' = 2^mu A exact, and
 * for N <= 5 every step of Algorithm 3 is exact (s_l2 = P2 = 0), so C must
 * equal the exact product bit for bit (computed here in 64-bit integers).
 * The second call uses the bound rule (tau = 1e-15) through oz2_gemm_ex with
 * a caller workspace on a stream of its own; there the CRT sums may round
 * once P > 2^53, so the check is the normwise target: |C - AB| <=
 * 4 tau max_ij (|A||B|)_ij (the rule keeps the N-dependent part of the
 * Theorem 2 bound below tau times a lower bound of that maximum; the factor
 * leaves room for the N-independent rounding terms).  The third call,
 * oz2_gemm_host, takes the host arrays themselves (malloc'd, pageable) and
 * must give the exact product at N = 5 again.  Exit status 0 on success, a
 * distinct nonzero code per failed check.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "oz2.h"

#define CHECK_CUDA(x)                                                   \
    do {                                                                \
        if ((x) != cudaSuccess) {                                       \
            fprintf(stderr, "CUDA error at line %d\n", __LINE__);       \
            return 2;                                                   \
        }                                                               \
    } while (0)

/* max_ij |C_ij - (AB)_ij| and max_ij (|A||B|)_ij, both in exact integers */
static void errors(int m, int n, int k, const double *A, const double *B, const double *C, double *err,
                   double *absprod)
{
    *err = 0;
    *absprod = 0;
    for (int i = 0; i < m; i++)
        for (int j = 0; j < n; j++) {
            int64_t s = 0, a = 0;
            for (int h = 0; h < k; h++) {
                int64_t x = (int64_t)A[i * k + h], y = (int64_t)B[h * n + j];
                s += x * y;
                a += llabs(x * y);
            }
            double e = fabs(C[i * n + j] - (double)s);
            if (e > *err) *err = e;
            if ((double)a > *absprod) *absprod = (double)a;
        }
}

static int check_exact(int m, int n, int k, const double *A, const double *B, const double *C)
{
    for (int i = 0; i < m; i++)
        for (int j = 0; j < n; j++) {
            int64_t s = 0;
            for (int h = 0; h < k; h++) s += (int64_t)A[i * k + h] * (int64_t)B[h * n + j];
            if ((double)s != C[i * n + j]) {
                fprintf(stderr, "mismatch at (%d, %d): %.17g vs %lld\n", i, j, C[i * n + j], (long long)s);
                return 1;
            }
        }
    return 0;
}

int main(void)
{
    const int m = 193, n = 131, k = 517;
    double *A = malloc(sizeof(double) * m * k), *B = malloc(sizeof(double) * k * n);
    double *C = malloc(sizeof(double) * m * n);
    if (!A || !B || !C) return 2;
    for (int i = 0; i < m; i++)
        for (int h = 0; h < k; h++) A[i * k + h] = (double)((i * 7 + h * 3) % 11 - 5);
    for (int h = 0; h < k; h++)
        for (int j = 0; j < n; j++) B[h * n + j] = (double)((h * 5 + j * 2) % 11 - 5);

    double *dA, *dB, *dC;
    CHECK_CUDA(cudaMalloc((void **)&dA, sizeof(double) * m * k));
    CHECK_CUDA(cudaMalloc((void **)&dB, sizeof(double) * k * n));
    CHECK_CUDA(cudaMalloc((void **)&dC, sizeof(double) * m * n));
    CHECK_CUDA(cudaMemcpy(dA, A, sizeof(double) * m * k, cudaMemcpyHostToDevice));
    CHECK_CUDA(cudaMemcpy(dB, B, sizeof(double) * k * n, cudaMemcpyHostToDevice));

    printf("liboz2 version %d\n", oz2_version());
    /* argument errors come back before anything is enqueued */
    if (oz2_gemm(0, n, k, dA, k, dB, n, dC, n, 5, OZ2_ACCURATE) != OZ2_EINVAL) return 3;

    /* fixed N = 5: exact */
    int rc = oz2_gemm(m, n, k, dA, k, dB, n, dC, n, 5, OZ2_ACCURATE);
    if (rc == OZ2_OK) rc = oz2_sync(NULL);
    if (rc != OZ2_OK) { fprintf(stderr, "oz2_gemm: %s\n", oz2_status_str(rc)); return 4; }
    CHECK_CUDA(cudaMemcpy(C, dC, sizeof(double) * m * n, cudaMemcpyDeviceToHost));
    if (check_exact(m, n, k, A, B, C)) return 5;

    /* bound rule with a caller workspace on a stream of our own */
    cudaStream_t st;
    CHECK_CUDA(cudaStreamCreate(&st));
    const size_t bytes = oz2_workspace_size(m, n, k, 20, OZ2_ACCURATE, 0);
    void *ws;
    int *dN, N = 0;
    CHECK_CUDA(cudaMalloc(&ws, bytes));
    CHECK_CUDA(cudaMalloc((void **)&dN, sizeof(int)));
    oz2_opts o = {0};
    o.stream = st;
    o.workspace = ws;
    o.workspace_bytes = bytes;
    o.target = 1e-15;
    o.nmax = 20;
    o.n_out = dN;
    rc = oz2_gemm_ex(m, n, k, dA, k, dB, n, dC, n, 0, OZ2_ACCURATE, &o);
    if (rc == OZ2_OK) rc = oz2_sync(st);
    if (rc != OZ2_OK) { fprintf(stderr, "oz2_gemm_ex: %s\n", oz2_status_str(rc)); return 6; }
    CHECK_CUDA(cudaMemcpy(&N, dN, sizeof(int), cudaMemcpyDeviceToHost));
    CHECK_CUDA(cudaMemcpy(C, dC, sizeof(double) * m * n, cudaMemcpyDeviceToHost));
    if (N < 2 || N > 20) return 7;
    double err, absprod;
    errors(m, n, k, A, B, C, &err, &absprod);
    if (!(err <= 4e-15 * absprod)) {
        fprintf(stderr, "bound rule: error %.3g above %.3g\n", err, 4e-15 * absprod);
        return 8;
    }

    /* host arrays: the library uploads A and B, runs the emulation and downloads C */
    const size_t hbytes = oz2_host_workspace_size(m, n, k, 5, OZ2_ACCURATE, 0);
    void *hws;
    CHECK_CUDA(cudaMalloc(&hws, hbytes));
    for (int i = 0; i < m * n; i++) C[i] = -1.0;
    oz2_opts h = {0};
    h.stream = st;
    h.workspace = hws;
    h.workspace_bytes = hbytes;
    if (oz2_gemm_host(m, n, k, A, k, B, n, C, n, 5, OZ2_ACCURATE, NULL) != OZ2_OK) return 9;   /* managed buffer */
    if (oz2_sync(NULL) != OZ2_OK || check_exact(m, n, k, A, B, C)) return 10;
    for (int i = 0; i < m * n; i++) C[i] = -1.0;
    h.workspace_bytes = hbytes - 256;
    if (oz2_gemm_host(m, n, k, A, k, B, n, C, n, 5, OZ2_ACCURATE, &h) != OZ2_ENOMEM) return 11;
    h.workspace_bytes = hbytes;
    rc = oz2_gemm_host(m, n, k, A, k, B, n, C, n, 5, OZ2_ACCURATE, &h);
    if (rc == OZ2_OK) rc = oz2_sync(st);
    if (rc != OZ2_OK) { fprintf(stderr, "oz2_gemm_host: %s\n", oz2_status_str(rc)); return 12; }
    if (check_exact(m, n, k, A, B, C)) return 13;

    printf("ok: %dx%dx%d exact at N = 5 (device and host arrays); N = %d by the bound rule, max error %.3g\n",
           m, n, k, N, err);
    cudaFree(hws);
    cudaFree(ws);
    cudaFree(dN);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dC);
    cudaStreamDestroy(st);
    free(A);
    free(B);
    free(C);
    return 0;
}
