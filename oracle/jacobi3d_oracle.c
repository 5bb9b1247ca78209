/*
 * FP64 CPU oracle for the iterated 7-point Jacobi stencil in 3-D.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * definition that the CUDA library's 3-D path is checked against.  Only the
 * tests, the smoke check and the benchmark's CPU-baseline leg may build, load
 * or call it; the library itself never does, and this file shares no code,
 * header, constant or helper with the CUDA sources.
 *
 * What it computes.  The paper's Jacobi benchmark (Sec. 6.1) is a 5-point
 * stencil on a 2-D domain with constant boundary conditions, iterated T times
 * in a ping-pong state loop (Fig. 1 gives the same loop in 1-D).  This is the
 * same method one dimension up: a 7-point stencil on a D x R x C box whose
 * one-cell outer shell is fixed, iterated T times between two copies of the
 * array (Appendix A's state-transition semantics: one timestep finishes
 * before the next starts).
 *
 *   A = G0, B = G0                          (shell identical in both)
 *   for t = 1..T:
 *     for 1 <= z <= D-2, 1 <= i <= R-2, 1 <= j <= C-2:
 *       B[z][i][j] = (1/7) * (A[z][i][j] + (((A[z][i-1][j] + A[z][i+1][j])
 *                                           + (A[z][i][j-1] + A[z][i][j+1]))
 *                                           + (A[z-1][i][j] + A[z+1][i][j])))
 *     swap(A, B)
 *   result = A (full box, shell included)
 *
 * Readings of points the paper leaves open (each is listed in the design
 * notes of the repository):
 *   - coefficients: 1/7 on all seven points (the 3-D counterpart of 0.2 on
 *     the five points of the 2-D reading: positive weights summing to one),
 *     as the double nearest to 1/7, i.e. the value of 1.0 / 7.0;
 *   - boundary: whatever the input holds on the shell (planes z = 0, D-1,
 *     rows i = 0, R-1, columns j = 0, C-1), never written;
 *   - summation order: c + (((n + s) + (w + e)) + (u + d)) with n, s the
 *     rows i-1, i+1, w, e the columns j-1, j+1 and u, d the planes z-1, z+1;
 *     IEEE double, round to nearest, no contraction (-ffp-contract=off).
 *     Reflecting any axis, or transposing rows and columns, commutes with a
 *     step bit for bit;
 *   - boxes with fewer than 3 cells along an axis have no interior: the
 *     result is a copy; T = 0 is a copy.
 *
 * Plane-parallel OpenMP is optional (nth threads; 0 = the OpenMP default);
 * every output point is computed by the same expression whatever the thread
 * count, so results are bitwise independent of it.
 */
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)

static const double ONE_SEVENTH = 1.0 / 7.0;

/* One timestep: B(interior) <- stencil(A).  B's shell is not touched. */
static void oracle3d_step(const double *A, double *B, long D, long R, long C, int nth)
{
    const long P = R * C; /* plane stride */
    long z;
#pragma omp parallel for num_threads(nth) schedule(static) if (nth > 1)
    for (z = 1; z < D - 1; ++z) {
        long i;
        for (i = 1; i < R - 1; ++i) {
            const double *row = A + z * P + i * C;
            double *dst = B + z * P + i * C;
            long j;
            for (j = 1; j < C - 1; ++j) {
                double centre = row[j];
                double ns = row[j - C] + row[j + C];
                double we = row[j - 1] + row[j + 1];
                double ud = row[j - P] + row[j + P];
                double sum = centre + ((ns + we) + ud);
                dst[j] = ONE_SEVENTH * sum;
            }
        }
    }
}

int oracle_jacobi3d(const double *in, double *out, long D, long R, long C, long T, int nth)
{
    double *A, *B, *tmp;
    long t;
    size_t n;
    if (D < 0 || R < 0 || C < 0 || T < 0 || (D * R * C > 0 && (!in || !out)))
        return ORACLE_EINVAL;
    n = (size_t)D * (size_t)R * (size_t)C;
    if (n == 0)
        return ORACLE_OK;
    if (nth < 1) {
#ifdef _OPENMP
        nth = omp_get_max_threads();
#else
        nth = 1;
#endif
    }
    if (D < 3 || R < 3 || C < 3 || T == 0) {
        if (out != in)
            memmove(out, in, n * sizeof(double));
        return ORACLE_OK;
    }
    A = (double *)malloc(n * sizeof(double));
    B = (double *)malloc(n * sizeof(double));
    if (!A || !B) {
        free(A);
        free(B);
        return ORACLE_ENOMEM;
    }
    memcpy(A, in, n * sizeof(double));
    memcpy(B, in, n * sizeof(double));
    for (t = 1; t <= T; ++t) {
        oracle3d_step(A, B, D, R, C, nth);
        tmp = A;
        A = B;
        B = tmp;
    }
    memcpy(out, A, n * sizeof(double));
    free(A);
    free(B);
    return ORACLE_OK;
}
