// Batched symmetric eigen-solver for the face-pair problems (eig.cu).
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"

namespace bddc {

constexpr int kEigCap = 48;   // eigenpairs formed per face in the first pass (a face with more is redone)

struct EigDesc {
    double *C;            // n x n symmetric standard-form matrix (destroyed)
    int n, ld;
    const double *W1;     // n x n, face row l = (W1 y_l) restricted to face_pos
    int ldw;
    const int *face_pos;  // positions of the face dofs among the n rows
    int nface;
    double *lam;          // out: eigenvalues, descending (selected + largest rejected), cap + 1
    double *vec;          // scratch: cap x n eigenvectors of C
    double *work;         // scratch: 64 n + 16
    double *rows;         // out: face rows, row l at rows[l * nface + f] (orthonormal)
    int *counts;          // out: [0] selected, [1] kept, [2] values in lam, [3] ties, [4] overflow:
                          // the selected count when it exceeds cap (then only cap are formed), else 0
    int cap;              // most eigenpairs formed (lam, vec and rows are sized by it)
    int given;            // 1: lam, vec and counts [0], [2], [3], [4] are supplied (the batched
                          // LOBPCG, lobpcg.h); only the face rows are formed (C is not read).
                          // 2: the Householder reduction is supplied (launch_tridiag_multi):
                          // reflectors in C, dd / ee / bet in work; steps 2-4 run.
                          // 3: as 1 with the face rows supplied too (launch_face_vec): the
                          // clusters are orthonormalised and the rows reduced
};

// Householder tridiagonalisation of large face matrices by several CTAs per face
// (tridiag.cu): the face's G CTAs share every reduction step, with a bounded barrier of
// the face's CTAs between the matrix-vector product and the rank-2 update.  One
// cooperative launch; items = (descriptor, rank g < G) per CTA.  Leaves C and work as
// the face kernel's step 1 does (EigDesc::given = 2).  bar: 2 zeroed counters per face.
struct TridiagDesc {
    double *A;            // n x n, ld lda, both triangles (overwritten)
    int n, lda;
    double *work;         // the face's EigDesc::work
    int G;                // CTAs of this face
    unsigned *bar;
};
cudaError_t launch_tridiag_multi(const TridiagDesc *descs, const int2 *items, int nitems, int nmax, int use_ff,
                                 DevStatus *st, double timeout_s, cudaStream_t s);
// CTAs of launch_tridiag_multi that can be co-resident (one cooperative launch at most)
int tridiag_multi_capacity(int nmax);

// The eigenpairs and face rows of faces whose Householder reduction launch_tridiag_multi
// supplied (given == 2), G CTAs per face (items = (descriptor, g)); scr[descriptor]: G x 8 x 6 n
// doubles of scratch.  launch_face_eig_n with given = 3 then finishes them.
void launch_face_vec(const EigDesc *descs, const int2 *items, int nitems, int G, int nmax, double tau, int fixed_k,
                     double *const *scr, cudaStream_t s);
constexpr int kFaceVecCTAs = 7;   // CTAs per face: 7 x 8 warps cover 49 eigenvalues, one each
constexpr int kFaceVecWarps = 8;  // warps per CTA of launch_face_vec (its scratch is per warp)

// nmax: largest n of the batch; when the matrix and work arrays do not fit in
// 200 KB of shared memory the matrix is reduced in place and work (64 n + 16
// doubles) is used from global memory.
// use_ff: the Householder reduction runs in double-float on the FP32 pipe (mixed modes)
// fixed_k > 0: select the fixed_k largest eigenvalues of every face instead of lambda > tau
void launch_face_eig_n(const EigDesc *descs, int npairs, int nmax, double tau, double drop_rel, int use_ff,
                       int fixed_k, DevStatus *st, cudaStream_t s);

// Kept adaptive edge rows (Section 3: every row d split into a face row and one row
// per edge), in the per-edge form: on each edge, one orthonormal basis of the span of the
// edge parts of every face pair's selected rows, a constraint on all substructures of
// the edge.  Two launches:
//   launch_edge_parts: one CTA per face pair, after launch_face_eig_n on the same W1
//     and eigenvectors.  d_l = W1 y_l over the pair's s dofs (side i), l < selected.
//     For every edge of the pair (a segment of s positions) row l of the pair's slot
//     gets the edge part of d_l normalised, or zeros when that part is negligible,
//     |d_l|_edge| <= drop_rel * sqrt(2) |d_l| (the whole row has d_i and -d_i), or
//     l >= selected.  A slot is kEigCap rows x the segment's length, row-major.
//   launch_edge_globs: one CTA per edge, over the slots of all pairs on it (stacked,
//     nrows = slots x kEigCap): Gram-Schmidt with row pivoting, rows whose pivot falls
//     below drop_rel of the first dropped (the caller passes 1e-6: the pairs' rows on
//     one edge overlap in exact arithmetic).
constexpr int kMaxEdgeSlots = 8;   // face pairs per edge
struct EdgePartDesc {
    const double *W1;     // ns x n, ld ldw (the face kernel's W1)
    int ldw, ns, n;
    const double *vec;    // the face kernel's eigenvectors: y_l at vec + l * n
    const int *counts;    // the face kernel's counts: [0] = selected rows
    const int *seg_ptr;   // (nseg + 1) offsets into seg_pos
    const int *seg_pos;   // s positions (< ns) of every edge's dofs, in global dof order
    int nseg;
    double *const *slot;  // (nseg) the segment's slot: kEigCap x len, row-major
};
struct EdgeGlobDesc {
    double *R;            // nrows x len, row-major: the stacked slots (destroyed)
    int nrows, len;       // nrows <= kMaxEdgeSlots * kEigCap
    double *rowsT;        // out: kept row l, dof k at rowsT[k * len + l] (ld len)
    int *kept;            // out: rows kept
};
void launch_edge_parts(const EdgePartDesc *d, int npairs, double drop_rel, cudaStream_t s);
void launch_edge_globs(const EdgeGlobDesc *d, int nedges, double drop_rel, cudaStream_t s);

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

// Initial constraints of a pair (averages over globs inside s): the pair problem
// is restricted to jumps z with R z = 0, R the indicator rows of the groups
// (one glob and one component each).  z = G u with G's columns e_a (a in no
// group) and e_q - e_lead (q a non-leading member of a group); the leader
// (first member) of every group is dropped, so u has nsp = ns - ngroups entries.
//   compress: M3c = [[Mww, ., .], [G^T Mbw, G^T Mbb G, .], [0, I_nsp, 0]] from the
//             full M3 (lower blocks as built by the adapt phase)
//   expand:   Xg = G X' with X' = M3c[ns+nsp : ns+2nsp, ns : ns+nsp] after the
//             partial Cholesky of M3c (ns + nsp columns)
//   project:  W1 <- P W1, P the orthogonal projector onto null(R): the group
//             mean is removed from every column of W1 within each group
struct PiDesc {
    const double *M3;     // 3ns x 3ns, ld3
    int ld3;
    double *M3c;          // (ns + 2nsp)^2, ldc
    int ldc;
    double *Xg;           // ns x nsp, ldg
    int ldg;
    double *W1;           // ns x nsp, ldw
    int ldw;
    const int *newidx;    // (ns) index in u, -1 for a leader
    const int *lead;      // (ns) leader of the member's group, -1 for leaders and non-members
    const int *grp;       // (ns) group of the position, -1 if none
    const int *keep;      // (nsp) position of every u entry
    const int *gptr;      // (ngroups + 1)
    const int *gidx;      // members, leader first
    int ns, nsp, ngroups;
};
void launch_pi_compress(const PiDesc *d, int npairs, int nmax, cudaStream_t s);
void launch_pi_expand(const PiDesc *d, int npairs, int nmax, cudaStream_t s);
void launch_pi_project(const PiDesc *d, int npairs, cudaStream_t s);

// Pair weights d_i = a_i / (a_i + a_j), d_j = a_j / (a_i + a_j) over s.
struct PairWeightDesc {
    const double *diag_i, *diag_j;   // packed diag(A) of the two substructures' interface dofs
    const int *pos_i, *pos_j;        // interface positions of the s dofs
    double *di, *dj;                 // out (ns)
    int ns;
};
void launch_pair_weights(const PairWeightDesc *d, int npairs, cudaStream_t s);

}  // namespace bddc
