/* Plain Parlett-Reid Pfaffian of a dense antisymmetric matrix (FP64).
 *
 * Test infrastructure: part of the CPU oracle, never linked into the product.
 *
 * The Pfaffian is the square root of the determinant of an antisymmetric
 * matrix with its sign fixed by Pf(J) = 1 for J = [[0,1],[-1,0]] blocks
 * (Sec. 3.2 uses it for tr(rho1 rho2) and Sec. 5 for N_nm).  Algorithm:
 * skew-symmetric Gaussian elimination with symmetric partial pivoting
 * (Parlett & Reid 1970): at step k the largest entry below the diagonal in
 * column k is swapped into row k+1 (each swap flips the sign), A[k][k+1]
 * multiplies the result, and the trailing block gets the rank-2 update that
 * zeroes column/row k.  Only the strictly lower triangle is read or written.
 * The result is returned as log|Pf| plus a unit phase so that large lattices
 * do not overflow.  Input is overwritten.
 */
#include <complex.h>
#include <math.h>
#include <stddef.h>

#define IDX(i, j) ((size_t)(i) * (size_t)n + (size_t)(j))

int oracle_pfaffian_z(int n, double complex *A, double *logabs, double complex *phase) {
    *logabs = 0.0;
    *phase = 1.0;
    if (n % 2) { *logabs = -INFINITY; *phase = 0.0; return 1; }
    for (int k = 0; k < n - 1; k += 2) {
        int p = k + 1;
        double best = cabs(A[IDX(k + 1, k)]);
        for (int i = k + 2; i < n; ++i) {
            double v = cabs(A[IDX(i, k)]);
            if (v > best) { best = v; p = i; }
        }
        if (p != k + 1) {
            int q = k + 1;
            for (int j = 0; j < q; ++j) { double complex t = A[IDX(q, j)]; A[IDX(q, j)] = A[IDX(p, j)]; A[IDX(p, j)] = t; }
            for (int i = p + 1; i < n; ++i) { double complex t = A[IDX(i, q)]; A[IDX(i, q)] = A[IDX(i, p)]; A[IDX(i, p)] = t; }
            for (int m = q + 1; m < p; ++m) { double complex t = A[IDX(m, q)]; A[IDX(m, q)] = -A[IDX(p, m)]; A[IDX(p, m)] = -t; }
            A[IDX(p, q)] = -A[IDX(p, q)];
            *phase = -*phase;
        }
        double complex piv = A[IDX(k + 1, k)];          /* = -A[k][k+1] */
        if (cabs(piv) == 0.0) { *logabs = -INFINITY; *phase = 0.0; return 1; }
        double complex akk1 = -piv;                      /* A[k][k+1] */
        *logabs += log(cabs(akk1));
        *phase *= akk1 / cabs(akk1);
        for (int i = k + 2; i < n; ++i) {
            double complex ti = A[IDX(i, k)] / piv;      /* tau_i = A[k][i] / A[k][k+1] */
            double complex ci = A[IDX(i, k + 1)];
            for (int j = k + 2; j < i; ++j) {
                double complex tj = A[IDX(j, k)] / piv;
                A[IDX(i, j)] += ti * A[IDX(j, k + 1)] - ci * tj;
            }
        }
    }
    return 0;
}

int oracle_pfaffian_d(int n, double *A, double *logabs, double *sign) {
    *logabs = 0.0;
    *sign = 1.0;
    if (n % 2) { *logabs = -INFINITY; *sign = 0.0; return 1; }
    for (int k = 0; k < n - 1; k += 2) {
        int p = k + 1;
        double best = fabs(A[IDX(k + 1, k)]);
        for (int i = k + 2; i < n; ++i) {
            double v = fabs(A[IDX(i, k)]);
            if (v > best) { best = v; p = i; }
        }
        if (p != k + 1) {
            int q = k + 1;
            for (int j = 0; j < q; ++j) { double t = A[IDX(q, j)]; A[IDX(q, j)] = A[IDX(p, j)]; A[IDX(p, j)] = t; }
            for (int i = p + 1; i < n; ++i) { double t = A[IDX(i, q)]; A[IDX(i, q)] = A[IDX(i, p)]; A[IDX(i, p)] = t; }
            for (int m = q + 1; m < p; ++m) { double t = A[IDX(m, q)]; A[IDX(m, q)] = -A[IDX(p, m)]; A[IDX(p, m)] = -t; }
            A[IDX(p, q)] = -A[IDX(p, q)];
            *sign = -*sign;
        }
        double piv = A[IDX(k + 1, k)];
        if (piv == 0.0) { *logabs = -INFINITY; *sign = 0.0; return 1; }
        double akk1 = -piv;
        *logabs += log(fabs(akk1));
        if (akk1 < 0) *sign = -*sign;
        for (int i = k + 2; i < n; ++i) {
            double ti = A[IDX(i, k)] / piv;
            double ci = A[IDX(i, k + 1)];
            for (int j = k + 2; j < i; ++j) {
                double tj = A[IDX(j, k)] / piv;
                A[IDX(i, j)] += ti * A[IDX(j, k + 1)] - ci * tj;
            }
        }
    }
    return 0;
}
