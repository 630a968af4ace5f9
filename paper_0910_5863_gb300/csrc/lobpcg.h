// Batched LOBPCG for the large face-pair eigenproblems (lobpcg.cu).
//
// The face kernel (eig.cu) reduces every pair problem to a dense symmetric
// standard problem C y = lambda y of order n and factors it by Householder
// reduction in one CTA; for large n that single-CTA reduction is the critical
// path of the adapt phase.  Large faces instead run the locally optimal block
// preconditioned conjugate gradient method (Knyazev), which the paper names
// for the pair problems (Section 3), on C: a block of k Ritz vectors X, their
// residuals R and the previous search directions P span the trial space; the
// block products C R run as batched FP64 GEMMs over all large faces at once,
// and the Rayleigh-Ritz step is FP64 (Gram matrices, then cyclic Jacobi in one
// CTA per face).  The count of eigenvalues above the selection threshold is
// then certified without a tridiagonal Sturm sequence: with the selected Ritz
// pairs (theta_l, x_l) and a shift sigma just above the largest rejected Ritz
// value, the matrix  sigma I - C + sum_l theta_l x_l x_l^T  is positive
// definite exactly when C has no eigenvalue >= sigma outside span{x_l}, which
// a Cholesky factorization decides.  A face whose iteration does not converge,
// whose block is too small or whose certificate fails is solved by the dense
// kernel instead.
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"

namespace bddc {

constexpr int kLobMaxK = 32;   // largest block (trial space 3k <= 96)

struct LobDesc {
    const double *C;   // n x n symmetric (both triangles), ld ldc
    int n, ldc;
    int k;             // block size
    double *S[2];      // two n x 3k trial-space buffers [X | P | R], ld lds (alternate per iteration)
    double *AS[2];     // C times the same columns
    int lds;
    double *G;         // 2 (3k)^2: the Gram matrices S^T C S (first) and S^T S (second), ld 3k
    double *coef;      // 3k x 2k, ld 3k: [X coefficients | P coefficients]
    double *theta;     // k Ritz values (descending)
    double *scratch;   // 4 (3k)^2 doubles
    double *rnorm;     // k residual norms |C x_j - theta_j x_j| / |x_j| of the last test
    int *state;        // [0] done, [1] iterations, [2] status (0 running, 1 converged, 2 failed)
};

// x = deterministic pseudo-random start block (a counter-based hash), R = P = 0,
// theta = 0; state cleared.  cur: buffer index that holds X.
void launch_lob_init(const LobDesc *d, int nd, int cur, cudaStream_t s);
// C <- (C + C^T) / 2 in place; items: (descriptor, 64-column block)
void launch_lob_symmetrize(const LobDesc *d, const int2 *items, int nitems, cudaStream_t s);
// theta = the Rayleigh quotients of X, R = AX - X diag(theta) (the residual block), the
// convergence test (tau: selection threshold; fixed_k > 0: the fixed_k largest are
// selected; rtol: residual against the Ritz value), and the columns of R and P (with
// C P's) scaled to unit norm.  Faces already done are skipped, unless final: then every
// face's theta and residuals are recomputed (after a fresh C X) and a face whose
// residuals no longer pass is marked failed.
void launch_lob_prep(const LobDesc *d, int nd, int cur, double tau, int fixed_k, double rtol, int final_check,
                     cudaStream_t s);
// Rayleigh-Ritz on span[X P R]: coefficients of the new X and P, new theta.
void launch_lob_rr(const LobDesc *d, int nd, cudaStream_t s);

// Certificate matrix (lower triangle): M = sigma I - C + sum_{l < nsel} theta_l x_l x_l^T / |x_l|^2,
// sigma = theta_nsel + sigma_rel |theta_nsel| just above the largest rejected Ritz value,
// written at M (ld ldm).  items: (descriptor, 64-column block).
struct LobCertDesc {
    const double *C;
    int n, ldc;
    const double *X;   // n x k Ritz vectors, ld ldx
    int ldx, k;
    const double *theta;
    const int *nsel;   // selected count (device; clamped to [0, k - 1])
    double *M;
    int ldm;
    double sigma_rel;
};
void launch_lob_cert(const LobCertDesc *d, const int2 *items, int nitems, cudaStream_t s);

// Selection and outputs of one converged face: counts[0] = nsel, [2] = values in lam,
// [3] = ties, [4] = overflow (nsel above cap), the eigenvalues (descending) into lam and
// the selected Ritz vectors into vec (vector l at vec + l n).
struct LobOutDesc {
    const double *X;   // n x k, ld ldx
    int n, ldx, k;
    const double *theta;
    double *lam;
    double *vec;
    int *counts;
    int cap;           // most eigenpairs kept
    int *state;
};
void launch_lob_select(const LobOutDesc *d, int nd, double tau, int fixed_k, cudaStream_t s);

}  // namespace bddc
