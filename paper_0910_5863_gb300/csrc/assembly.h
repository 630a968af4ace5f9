// Launchers of the Q1 assembly kernels (assembly.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace bddc {

struct AssemblyArgs {
    const double *grads;      // (ne, 8 gauss, 8 nodes, 3) physical gradients
    const double *wdet;       // (ne, 8) quadrature weight * det J
    const double *coef;       // (ne)
    const int32_t *elem_sub;  // (ne)
    const int32_t *elem_pos;  // (ne, 8) dense position of the node's first dof, -1 = Dirichlet
    double *const *A;         // per-substructure dense matrix (device array of pointers)
    const int *ld;            // per-substructure leading dimension
    double nu;
    int ncomp;
};

void launch_element_geometry(const double *xyz, const int64_t *elems, int64_t ne, double *grads, double *wdet,
                             cudaStream_t s);
void launch_element_scatter(const AssemblyArgs &args, const int32_t *color_elems, int n, cudaStream_t s);
void launch_csr_scatter(double *const *A, const int64_t *sub_start, int ns, const int64_t *off, const double *val,
                        int64_t nnz, cudaStream_t s);

}  // namespace bddc
