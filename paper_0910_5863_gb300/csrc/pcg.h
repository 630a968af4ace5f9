// Interface operators of the reduced problem and the persistent PCG (pcg.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "common.cuh"

namespace bddc {

// Everything the operator S = sum R_i^T S_i R_i and the BDDC preconditioner
// M r = sum R_i^T D_i (P_i D_i R_i r + Phi_i R_ci u_c), S_C u_c = sum R_ci^T Phi_i^T D_i R_i r
// need, packed per substructure.  P~ = D P D and Phi~ = D Phi are stored
// with the weights folded in.
// One entry (substructure s, local interface position k) of an interface dof, with
// everything the assembly of z = sum (z_i + Phi~_i u_c,i) needs in one record.
struct ZEntry {
    int64_t pe;          // packed local index (offset of s + k)
    const double *phi;   // Phi~_s + k: entry m at phi[m * ld]
    const int *rc;       // R_c of s: global coarse index of local coarse dof m
    int ld, nc;
};

struct IfaceOps {
    int nsub, nG, nC;
    int maxGi;               // largest nGi
    const int *nGi;          // (nsub) interface size
    const int *ldS;          // (nsub) leading dimension of S_i and P~_i
    const int64_t *off;      // (nsub) offset of the substructure's packed local vector
    const int *RG;           // (sum nGi) global interface index of each local interface dof
    double *const *S;        // (nsub) S_i, full symmetric column-major
    double *const *P;        // (nsub) P~_i, full symmetric column-major
    double *const *Phi;      // (nsub) Phi~_i, nGi x nci column-major (ld = ldS)
    const int *nci;          // (nsub) local coarse count
    const int64_t *offc;     // (nsub) offset of the local coarse vector
    const int *Rc;           // (sum nci) global coarse index of each local coarse dof
    const double *SCinv;     // nC x nC inverse coarse matrix (full)
    const int *gptr;         // (nG+1) local entries of each interface dof
    const int64_t *gent;     // packed local index of each entry
    const int *gsub;         // substructure of each entry
    const ZEntry *zent;      // the entries again, as assembly records
    const int *cptr;         // (nC+1)
    const int64_t *cent;     // packed local coarse index of each entry
    const int2 *rowblk;      // (sub, first row) GEMV work items, 64 rows each, grouped by bin
    int nrowblk;
    const int *binptr;       // (nbins + 1) items of each bin: block b takes bins b, b + grid, ...
    int nbins;               // bins of near-equal cost (longest item first onto the lightest bin)
    int stream_mats;         // S_i and P~_i exceed L2: read them with the evict-first policy
    const int2 *cdot;        // (sub, first coarse column) items, 16 columns each
    int ncdot;
};

struct PcgBuffers {
    double *x, *r, *z, *p0, *p1, *q;  // nG
    double *zl, *yl;                  // sum nGi
    double *cl;                       // sum nci
    double *uc;                       // nC
    double *partial;                  // 2 x 2048: two sets of per-block partial sums
    double *alpha, *beta;             // maxit
    int *iters, *converged;
    double *relres;
};

enum PcgMode { PCG_SOLVE = 0, PCG_APPLY_M = 1, PCG_APPLY_S = 2 };

// Launches the persistent cooperative kernel.  Returns the cudaError of the launch.
cudaError_t launch_pcg(const IfaceOps &ops, const PcgBuffers &buf, int mode, double tol, int maxit,
                       DevStatus *st, double timeout_s, cudaStream_t s, int *nblocks_out);

// One cooperative launch (a block per SM) through the bounded grid barrier of the PCG kernel,
// told to wait for `extra` more blocks than exist (0: a normal barrier).  *passed counts the
// blocks that got through; a timeout is recorded in st.
cudaError_t launch_barrier_selftest(DevStatus *st, int extra, double timeout_s, int *passed, cudaStream_t s);

// Weights: delta(k) = diag_i(k) / sum over the substructures sharing the dof.
void launch_weights(const IfaceOps &ops, const double *diag_packed, double *total, double *delta_packed,
                    cudaStream_t s);
// Deterministic assembly of a packed local interface vector: out[x] = sum over entries.
void launch_iface_assemble(const IfaceOps &ops, const double *packed, double *out, cudaStream_t s);
// out[0] = ||g - q||^2, out[1] = ||g||^2 (one block, fixed summation order).
void launch_residual_norms2(const double *g, const double *q, int n, double *out, cudaStream_t s);

}  // namespace bddc
