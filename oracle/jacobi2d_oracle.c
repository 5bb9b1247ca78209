/*
 * FP64 CPU oracle for the iterated 5-point Jacobi-2D stencil.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * definition that the CUDA library is checked against.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may build, load or call it;
 * the library itself never does, and this file shares no code, header,
 * constant or helper with the CUDA sources.
 *
 * What it computes (paper: Sec. 6.1 "Fundamental Computational Kernels",
 * Jacobi stencil: a 5-point stencil applied repeatedly for T iterations on a
 * 2-D domain with constant boundary conditions; Fig. 1 shows the same
 * pattern in 1-D as a state loop over a map that ping-pongs between two
 * copies of the array; Appendix A gives the state-transition semantics, under
 * which one timestep finishes before the next starts):
 *
 *   A = G0, B = G0                          (boundary ring identical in both)
 *   for t = 1..T:
 *     for 1 <= i <= R-2, 1 <= j <= C-2:
 *       B[i][j] = 0.2 * (A[i][j] + ((A[i-1][j] + A[i+1][j])
 *                                  + (A[i][j-1] + A[i][j+1])))
 *     swap(A, B)
 *   result = A (full grid, boundary ring included)
 *
 * Readings of points the paper leaves open (each is listed in the design
 * notes of the repository):
 *   - coefficients: 0.2 on all five points (the paper only says "5-point");
 *   - boundary: whatever the input holds in row 0, row R-1, column 0 and
 *     column C-1, never written (the paper's zero boundary is the special
 *     case of a zero ring);
 *   - summation order: c + ((n + s) + (w + e)), then times 0.2, all in IEEE
 *     double with round-to-nearest and no contraction (compile with
 *     -ffp-contract=off).  Addition is commutative, so transposing or
 *     reflecting the grid commutes with a step bit for bit;
 *   - grids with fewer than 3 rows or columns have no interior: the result is
 *     a copy; T = 0 is a copy.
 *
 * Tolerance mode (the data-dependent state transition of Sec. 3 "State"):
 *   r_t = sqrt( sum over the interior of (A_t - A_{t-1})^2 )   in FP64,
 *   summed along each row in column order, then over rows in row order.
 *   rel_t = r_t / r_1 (r_1 = norm of the first step's update, which equals
 *   0.2 x the norm of the initial discrete-Laplace residual); rel_t = 0 when
 *   r_1 = 0.  The loop stops at the first t that is a multiple of
 *   check_stride with rel_t <= tol, or at t = T_cap.  The reported residual
 *   is rel at the final step.
 *
 * Row-parallel OpenMP is optional.  Every output point is computed by
 * exactly the same expression whatever the thread count, and residual sums
 * are formed per row and then added in row order, so results are bitwise
 * independent of the number of threads.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)

/* One timestep: B(interior) <- stencil(A).  B's boundary ring is not touched. */
static void oracle_step(const double *A, double *B, long R, long C, int nth)
{
    long i;
#pragma omp parallel for num_threads(nth) schedule(static) if (nth > 1)
    for (i = 1; i < R - 1; ++i) {
        const double *north = A + (i - 1) * C;
        const double *row = A + i * C;
        const double *south = A + (i + 1) * C;
        double *dst = B + i * C;
        long j;
        for (j = 1; j < C - 1; ++j) {
            double centre = row[j];
            double ns = north[j] + south[j];
            double we = row[j - 1] + row[j + 1];
            double sum = centre + (ns + we);
            dst[j] = 0.2 * sum;
        }
    }
}

/* sum over the interior of (X - Y)^2: per-row sums, then rows in order. */
static double oracle_sqdiff(const double *X, const double *Y, long R, long C,
                            double *rowsum, int nth)
{
    long i;
    double total = 0.0;
#pragma omp parallel for num_threads(nth) schedule(static) if (nth > 1)
    for (i = 1; i < R - 1; ++i) {
        double acc = 0.0;
        long j;
        for (j = 1; j < C - 1; ++j) {
            double d = X[i * C + j] - Y[i * C + j];
            acc += d * d;
        }
        rowsum[i] = acc;
    }
    for (i = 1; i < R - 1; ++i)
        total += rowsum[i];
    return total;
}

static int oracle_threads(int nth)
{
    if (nth > 0)
        return nth;
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int oracle_num_threads(int nth) { return oracle_threads(nth); }

/*
 * Plain mode: out <- the grid after T timesteps.  in and out are host arrays
 * of R*C doubles, row-major, contiguous.  in == out is allowed.
 */
int oracle_jacobi2d(const double *in, double *out, long R, long C, long T,
                    int nth)
{
    double *A, *B, *tmp;
    long t;
    size_t n;
    if (R < 0 || C < 0 || T < 0 || (R * C > 0 && (!in || !out)))
        return ORACLE_EINVAL;
    n = (size_t)R * (size_t)C;
    if (n == 0)
        return ORACLE_OK;
    nth = oracle_threads(nth);
    if (R < 3 || C < 3 || T == 0) {
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
        oracle_step(A, B, R, C, nth);
        tmp = A;
        A = B;
        B = tmp;
    }
    memcpy(out, A, n * sizeof(double));
    free(A);
    free(B);
    return ORACLE_OK;
}

/*
 * Tolerance mode (see the header comment).  Outputs: out (grid at the final
 * step), *steps_done, *rel_res (rel at the final step), *r_first (r_1).
 * check_stride >= 1; tol >= 0 (tol == 0 runs exactly T_cap steps but still
 * reports the residual).
 */
int oracle_jacobi2d_tol(const double *in, double *out, long R, long C,
                        long T_cap, double tol, long check_stride, int nth,
                        long *steps_done, double *rel_res, double *r_first)
{
    double *A, *B, *tmp, *rowsum;
    double r1 = 0.0, rt = 0.0, rel = 0.0;
    long t, done;
    size_t n;
    if (R < 0 || C < 0 || T_cap < 0 || check_stride < 1 || !(tol >= 0.0) ||
        !steps_done || !rel_res || !r_first || (R * C > 0 && (!in || !out)))
        return ORACLE_EINVAL;
    n = (size_t)R * (size_t)C;
    *steps_done = 0;
    *rel_res = 0.0;
    *r_first = 0.0;
    if (n == 0)
        return ORACLE_OK;
    nth = oracle_threads(nth);
    if (R < 3 || C < 3 || T_cap == 0) {
        if (out != in)
            memmove(out, in, n * sizeof(double));
        *steps_done = (R < 3 || C < 3) ? T_cap : 0;
        return ORACLE_OK;
    }
    A = (double *)malloc(n * sizeof(double));
    B = (double *)malloc(n * sizeof(double));
    rowsum = (double *)calloc((size_t)R, sizeof(double));
    if (!A || !B || !rowsum) {
        free(A);
        free(B);
        free(rowsum);
        return ORACLE_ENOMEM;
    }
    memcpy(A, in, n * sizeof(double));
    memcpy(B, in, n * sizeof(double));
    done = T_cap;
    for (t = 1; t <= T_cap; ++t) {
        int is_check = (t % check_stride) == 0;
        oracle_step(A, B, R, C, nth);
        /* B now holds A_t and A holds A_{t-1}. */
        if (t == 1 || is_check || t == T_cap) {
            rt = sqrt(oracle_sqdiff(B, A, R, C, rowsum, nth));
            if (t == 1)
                r1 = rt;
            rel = (r1 > 0.0) ? rt / r1 : 0.0;
        }
        tmp = A;
        A = B;
        B = tmp;
        if (is_check && tol > 0.0 && rel <= tol) {
            done = t;
            break;
        }
    }
    memcpy(out, A, n * sizeof(double));
    *steps_done = done;
    *rel_res = rel;
    *r_first = r1;
    free(A);
    free(B);
    free(rowsum);
    return ORACLE_OK;
}

/*
 * The 1-D Laplace program of the paper's Fig. 1: a float64[2, N] array A is
 * ping-ponged for T steps,
 *
 *   for t in 0..T-1:  for 1 <= i <= N-2:
 *       A[(t+1) % 2][i] = A[t % 2][i-1]*1 + A[t % 2][i]*(-2) + A[t % 2][i+1]*1
 *
 * (the memlet A[t%2, i-1:i+2] times [1, -2, 1], summed left to right).  The
 * end cells A[r][0] and A[r][N-1] of each row r are never written, so a step
 * reading row r sees row r's initial ends.  A (2*N doubles, row-major) is
 * updated in place exactly as the program leaves it.
 */
int oracle_laplace1d(double *A, long N, long T)
{
    long t, i;
    if (N < 0 || T < 0 || (N > 0 && !A))
        return ORACLE_EINVAL;
    for (t = 0; t < T; ++t) {
        const double *src = A + (t % 2) * N;
        double *dst = A + ((t + 1) % 2) * N;
        for (i = 1; i < N - 1; ++i)
            dst[i] = (src[i - 1] * 1.0 + src[i] * -2.0) + src[i + 1] * 1.0;
    }
    return ORACLE_OK;
}
