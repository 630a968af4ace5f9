/*
 * Oracle: cyclic Jacobi eigenvalue method for a dense symmetric matrix (FP64).
 *
 * TEST INFRASTRUCTURE ONLY: used by the CPU oracle of adaptive BDDC to solve
 * the pairwise face eigenproblems (Section 3 of the paper, eq. (eig-matrix))
 * after their reduction to standard symmetric form.  The CUDA library does
 * not use this file.
 *
 * Method (textbook cyclic-by-row Jacobi): sweep over all pairs p < q and
 * annihilate a_pq with the rotation that diagonalises the 2x2 block
 * [a_pp a_pq; a_pq a_qq]:  theta = (a_qq - a_pp) / (2 a_pq),
 * t = sign(theta) / (|theta| + sqrt(1 + theta^2)), c = 1/sqrt(1+t^2), s = t c.
 * Sweeps stop once the off-diagonal Frobenius norm falls below
 * tol * ||A||_F.  Rotations are accumulated in V (row-major, columns are the
 * eigenvectors).  A is overwritten; its diagonal holds the eigenvalues.
 */
#include <math.h>
#include <string.h>

static double off_norm(const double *a, int n) {
    double s = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (i != j) s += a[i * n + j] * a[i * n + j];
    return sqrt(s);
}

/* returns the number of sweeps, or -1 if max_sweeps was reached */
int oracle_jacobi_eig(int n, double *a, double *v, double tol, int max_sweeps) {
    memset(v, 0, sizeof(double) * (size_t)n * n);
    for (int i = 0; i < n; ++i) v[i * n + i] = 1.0;
    double fro = 0.0;
    for (int i = 0; i < n * n; ++i) fro += a[i] * a[i];
    fro = sqrt(fro);
    if (fro == 0.0) return 0;
    for (int sweep = 1; sweep <= max_sweeps; ++sweep) {
        if (off_norm(a, n) <= tol * fro) return sweep - 1;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double apq = a[p * n + q];
                if (apq == 0.0) continue;
                double app = a[p * n + p], aqq = a[q * n + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                /* A <- J^T A J with J the rotation in the (p, q) plane */
                for (int k = 0; k < n; ++k) {
                    double akp = a[k * n + p], akq = a[k * n + q];
                    a[k * n + p] = c * akp - s * akq;
                    a[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = a[p * n + k], aqk = a[q * n + k];
                    a[p * n + k] = c * apk - s * aqk;
                    a[q * n + k] = s * apk + c * aqk;
                }
                a[p * n + q] = a[q * n + p] = 0.0;
                for (int k = 0; k < n; ++k) {
                    double vkp = v[k * n + p], vkq = v[k * n + q];
                    v[k * n + p] = c * vkp - s * vkq;
                    v[k * n + q] = s * vkp + c * vkq;
                }
            }
        }
    }
    return off_norm(a, n) <= tol * fro ? max_sweeps : -1;
}
