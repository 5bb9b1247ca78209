/*
 * FP64 CPU oracle for red-black successive over-relaxation (SOR) on the 2-D
 * 5-point Laplace problem: the in-place, ordered counterpart of the Jacobi
 * stencil.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * definition that the CUDA library's SOR path is checked against.  Only the
 * tests, the smoke check and the benchmark's CPU-baseline leg may build, load
 * or call it; the library itself never does, and this file shares no code,
 * header, constant or helper with the CUDA sources.
 *
 * What it computes.  The paper's Jacobi benchmark (Sec. 6.1) updates every
 * interior point from the previous timestep's values (two copies of the
 * array, Fig. 1).  A Gauss-Seidel / SOR sweep instead updates the array in
 * place, so a point sees the neighbours already updated in the same sweep.
 * With the red-black order -- first every interior point with i + j even
 * ("red"), then every one with i + j odd ("black") -- the points of one colour
 * only read points of the other colour, so each half-sweep is one map whose
 * instances are independent (the paper's Map scope), and the order inside a
 * colour does not change the result.
 *
 *   for t = 1..T:
 *     for colour in (red: (i + j) % 2 == 0, black: (i + j) % 2 == 1):
 *       for 1 <= i <= R-2, 1 <= j <= C-2 of that colour:
 *         q = (A[i-1][j] + A[i+1][j]) + (A[i][j-1] + A[i][j+1])
 *         A[i][j] = (1 - omega) * A[i][j] + (omega / 4) * q
 *   result = A (full grid, boundary ring included)
 *
 * Readings (listed in the design notes of the repository):
 *   - omega is the relaxation factor (omega = 1: Gauss-Seidel; 0 < omega < 2
 *     converges for this problem); the two coefficients are the doubles
 *     (1 - omega) and (0.25 * omega), evaluated once;
 *   - summation order as written: q = (n + s) + (w + e) (n, s: rows i-1,
 *     i+1; w, e: columns j-1, j+1), then (1 - omega) * c + (0.25 omega) * q,
 *     IEEE double, no contraction;
 *   - boundary: the outer ring holds its input values, never written;
 *   - grids with fewer than 3 rows or columns, or T = 0: a copy.
 */
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)

/* One half-sweep over the interior points of one colour, in place
 * (a = 1 - omega, b = omega / 4). */
static void sor_colour(double *A, long R, long C, int colour, double a, double b)
{
    long i, j;
    for (i = 1; i < R - 1; ++i) {
        double *row = A + i * C;
        const double *north = row - C;
        const double *south = row + C;
        /* first column of this colour in row i */
        j = 1 + ((i + 1 + colour) & 1);
        for (; j < C - 1; j += 2) {
            double q = (north[j] + south[j]) + (row[j - 1] + row[j + 1]);
            row[j] = a * row[j] + b * q;
        }
    }
}

/*
 * out <- the grid after T red-black SOR iterations with relaxation omega.  in and
 * out are host arrays of R*C doubles, row-major, contiguous; in == out is
 * allowed.
 */
int oracle_sor2d(const double *in, double *out, long R, long C, long T, double omega)
{
    long t;
    size_t n;
    double a, b;
    if (R < 0 || C < 0 || T < 0 || (R * C > 0 && (!in || !out)))
        return ORACLE_EINVAL;
    n = (size_t)R * (size_t)C;
    if (n == 0)
        return ORACLE_OK;
    if (out != in)
        memmove(out, in, n * sizeof(double));
    if (R < 3 || C < 3 || T == 0)
        return ORACLE_OK;
    a = 1.0 - omega;
    b = 0.25 * omega;
    for (t = 1; t <= T; ++t) {
        sor_colour(out, R, C, 0, a, b);
        sor_colour(out, R, C, 1, a, b);
    }
    return ORACLE_OK;
}
