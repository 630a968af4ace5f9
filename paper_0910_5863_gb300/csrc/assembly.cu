// Q1 (trilinear hexahedron) element matrices and their subassembly into the
// dense local matrices A_i of the substructures (Section 2 of the paper: A_i
// is the subassembly of the element matrices of Omega_i only).
//
// Element matrices use 2x2x2 Gauss quadrature on the trilinear map:
//   diffusion:  K_ab = k_e sum_q w_q det J_q grad N_a . grad N_b
//   elasticity: K_ab^{ij} = sum_q w_q det J_q [lambda dN_a/dx_i dN_b/dx_j
//               + mu (dN_a/dx_j dN_b/dx_i + delta_ij grad N_a . grad N_b)]
// Elements are coloured so that no two elements of a colour share a node;
// one launch per colour adds every element block without atomics, so the
// result is deterministic.
#include "common.cuh"
#include "assembly.h"

namespace bddc {

__device__ __forceinline__ void ref_grad(int a, const double xi[3], double g[3]) {
    double s0 = (a & 1) ? 1.0 : -1.0, s1 = ((a >> 1) & 1) ? 1.0 : -1.0, s2 = ((a >> 2) & 1) ? 1.0 : -1.0;
    double f0 = 1.0 + s0 * xi[0], f1 = 1.0 + s1 * xi[1], f2 = 1.0 + s2 * xi[2];
    g[0] = 0.125 * s0 * f1 * f2;
    g[1] = 0.125 * f0 * s1 * f2;
    g[2] = 0.125 * f0 * f1 * s2;
}

// one thread per element: physical shape-function gradients and weights
__global__ void element_geometry_kernel(const double *xyz, const int64_t *elems, int64_t ne, double *grads,
                                        double *wdet) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    double xe[8][3];
    for (int a = 0; a < 8; ++a) {
        int64_t nd = elems[e * 8 + a];
        for (int d = 0; d < 3; ++d) xe[a][d] = xyz[nd * 3 + d];
    }
    const double gp = 0.57735026918962576451;  // 1/sqrt(3)
    for (int q = 0; q < 8; ++q) {
        double xi[3] = {(q & 1) ? gp : -gp, ((q >> 1) & 1) ? gp : -gp, ((q >> 2) & 1) ? gp : -gp};
        double gr[8][3];
        double J[3][3] = {};
        for (int a = 0; a < 8; ++a) {
            ref_grad(a, xi, gr[a]);
            for (int d = 0; d < 3; ++d)
                for (int k = 0; k < 3; ++k) J[d][k] += xe[a][d] * gr[a][k];
        }
        double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                     J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        double inv[3][3];
        inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
        inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
        inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
        inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
        inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
        inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
        inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
        inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
        inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
        // dN/dx_d = sum_k dN/dxi_k dxi_k/dx_d, dxi/dx = J^{-1}
        for (int a = 0; a < 8; ++a)
            for (int d = 0; d < 3; ++d) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k) s += gr[a][k] * inv[k][d];
                grads[((e * 8 + q) * 8 + a) * 3 + d] = s;
            }
        wdet[e * 8 + q] = det;  // Gauss weights are 1
    }
}

// one thread per (element of the colour, a, b): adds the element block K_ab
// into the substructure's dense matrix at the positions of nodes a and b.
__global__ void element_scatter_kernel(const AssemblyArgs args, const int32_t *color_elems, int ncolor_elems) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)ncolor_elems * 64) return;
    int64_t e = color_elems[t >> 6];
    int a = (t >> 3) & 7, b = t & 7;
    int pa = args.elem_pos[e * 8 + a], pb = args.elem_pos[e * 8 + b];
    if (pa < 0 || pb < 0) return;
    int s = args.elem_sub[e];
    double *A = args.A[s];
    int ld = args.ld[s];
    const double *G = args.grads + e * 8 * 8 * 3;
    const double *W = args.wdet + e * 8;
    double coef = args.coef[e];
    if (args.ncomp == 1) {
        double v = 0.0;
        for (int q = 0; q < 8; ++q) {
            const double *ga = G + (q * 8 + a) * 3, *gb = G + (q * 8 + b) * 3;
            v += W[q] * (ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2]);
        }
        A[(size_t)pb * ld + pa] += coef * v;
    } else {
        double nu = args.nu;
        double lam = coef * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
        double mu = coef / (2.0 * (1.0 + nu));
        double K[3][3] = {};
        for (int q = 0; q < 8; ++q) {
            const double *ga = G + (q * 8 + a) * 3, *gb = G + (q * 8 + b) * 3;
            double dot = ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    K[i][j] += W[q] * (lam * ga[i] * gb[j] + mu * (ga[j] * gb[i] + (i == j ? dot : 0.0)));
        }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) A[(size_t)(pb + j) * ld + pa + i] += K[i][j];
    }
}

// Algebraic input: one thread per (merged) CSR entry of every substructure
// writes its value at the precomputed dense offset (column-major, the local
// ordering [interior; interface]).  sub_start (ns + 1) splits the entries by
// substructure; entries are unique per destination, so plain stores suffice.
__global__ void csr_scatter_kernel(double *const *A, const int64_t *sub_start, int ns, const int64_t *off,
                                   const double *val, int64_t nnz) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nnz) return;
    int lo = 0, hi = ns - 1;  // largest s with sub_start[s] <= t
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (sub_start[mid] <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    A[lo][off[t]] = val[t];
}

void launch_csr_scatter(double *const *A, const int64_t *sub_start, int ns, const int64_t *off, const double *val,
                        int64_t nnz, cudaStream_t s) {
    if (nnz > 0 && ns > 0)
        csr_scatter_kernel<<<(unsigned)((nnz + 255) / 256), 256, 0, s>>>(A, sub_start, ns, off, val, nnz);
}

void launch_element_geometry(const double *xyz, const int64_t *elems, int64_t ne, double *grads, double *wdet,
                             cudaStream_t s) {
    if (ne > 0) element_geometry_kernel<<<(unsigned)((ne + 127) / 128), 128, 0, s>>>(xyz, elems, ne, grads, wdet);
}

void launch_element_scatter(const AssemblyArgs &args, const int32_t *color_elems, int n, cudaStream_t s) {
    if (n > 0) {
        int64_t threads = (int64_t)n * 64;
        element_scatter_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(args, color_elems, n);
    }
}

}  // namespace bddc
