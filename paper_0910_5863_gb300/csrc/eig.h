// Batched symmetric eigen-solver for the face-pair problems (eig.cu).
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"

namespace bddc {

constexpr int kEigCap = 48;   // most eigenpairs above tau kept per face

struct EigDesc {
    double *C;            // n x n symmetric standard-form matrix (destroyed)
    int n, ld;
    const double *W1;     // n x n, face row l = (W1 y_l) restricted to face_pos
    int ldw;
    const int *face_pos;  // positions of the face dofs among the n rows
    int nface;
    double *lam;          // out: eigenvalues, descending (selected + largest rejected), kEigCap + 1
    double *vec;          // scratch: kEigCap x n eigenvectors of C
    double *work;         // scratch: 64 n + 16
    double *rows;         // out: face rows, row l at rows[l * nface + f] (orthonormal)
    int *counts;          // out: [0] selected, [1] kept, [2] values in lam, [3] ties, [4] overflow
};

// nmax: largest n of the batch; when the matrix and work arrays do not fit in
// 200 KB of shared memory the matrix is reduced in place and work (64 n + 16
// doubles) is used from global memory.
void launch_face_eig_n(const EigDesc *descs, int npairs, int nmax, double tau, double drop_rel, DevStatus *st,
                       cudaStream_t s);

// Deflated pair matrix M3 (see adapt phase): adds sigma*c_blk*N0 N0^T to the
// (w2,w2), (b,w2) and (b,b) blocks with c = 4, 2, 1; sigma = max diag(S^).
struct DeflateDesc {
    const double *Shat;   // 2ns x 2ns Schur complement (lower), ld_s
    int ld_s;
    double *M3;           // 3ns x 3ns, ld_m
    int ld_m;
    const double *N0;     // ns x nnull (col-major, ld ns)
    int ns, nnull;
};
void launch_deflate(const DeflateDesc *d, int npairs, cudaStream_t s);

// Pair weights d_i = a_i / (a_i + a_j), d_j = a_j / (a_i + a_j) over s.
struct PairWeightDesc {
    const double *diag_i, *diag_j;   // packed diag(A) of the two substructures' interface dofs
    const int *pos_i, *pos_j;        // interface positions of the s dofs
    double *di, *dj;                 // out (ns)
    int ns;
};
void launch_pair_weights(const PairWeightDesc *d, int npairs, cudaStream_t s);

}  // namespace bddc
