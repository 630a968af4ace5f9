// Schur complement of one dense matrix for callers that cannot allocate
// device memory (no cudaMalloc / cudaFree / allocating library routine on
// this path).  Such callers include code that runs under an external memory
// budget, custom allocators that own the whole device, or plug-in hosts that
// forbid allocation after start-up.  The call reuses the partial Cholesky
// kernels of the library; its scratch -- the working copy of the matrix, the
// batched-kernel work lists and the device status word -- lives in the
// file-scope array below, which every GPU that loads the library holds until
// the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/bddc.h"
#include "common.cuh"
#include "dense.h"

namespace {

constexpr int kMaxN = 1024;                                   // largest n accepted
constexpr size_t kMatBytes = (size_t)kMaxN * kMaxN * sizeof(double);
constexpr size_t kListBytes = 512 * 1024;                     // descriptor + work items
constexpr size_t kScratchBytes = kMatBytes + kListBytes + 256;

// The shared scratch.  In host code this name is only a stand-in symbol;
// its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_bddc_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

void set_msg(char *msg, int cap, const char *text) {
    if (msg && cap > 0) {
        std::strncpy(msg, text, (size_t)cap - 1);
        msg[cap - 1] = '\0';
    }
}

// One-time set-up per device (with that device current): the device address of the scratch.
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_bddc_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

// Work lists of the partial Cholesky of one matrix, written in place: block k
// writes the panel items and the lower-triangle update tiles of step k.
__device__ __host__ inline int panel_count(int n, int n_int, int k) {
    int kb = k * bddc::kPanelNB, nb = n_int - kb < bddc::kPanelNB ? n_int - kb : bddc::kPanelNB;
    int below = n - kb - nb;
    int np = (below + bddc::kPanelRows - 1) / bddc::kPanelRows;
    return np > 1 ? np : 1;
}
__device__ __host__ inline int update_count(int n, int n_int, int k) {
    int kb = k * bddc::kPanelNB, nb = n_int - kb < bddc::kPanelNB ? n_int - kb : bddc::kPanelNB;
    int below = n - kb - nb;
    int nt = (below + bddc::kTile - 1) / bddc::kTile;
    return nt * (nt + 1) / 2 + 1;  // + the copy of the factored diagonal block
}

__global__ void static_init_kernel(double *W, int n, int ld, int n_int, int steps, bddc::PcholDesc<double> *desc,
                                   DevStatus *st, int2 *pit, int4 *uit, double *diag) {
    const int k = blockIdx.x;
    if (k == 0 && threadIdx.x == 0) {
        *desc = bddc::PcholDesc<double>{W, n, ld, n_int, 0, diag};
        st->code = st->item = st->pos = 0;
        st->arrive = st->gen = 0;
    }
    if (k >= steps) return;
    int po = 0, uo = 0;
    for (int j = 0; j < k; ++j) {
        po += panel_count(n, n_int, j);
        uo += update_count(n, n_int, j);
    }
    const int np = panel_count(n, n_int, k);
    for (int r = threadIdx.x; r < np; r += blockDim.x) pit[po + r] = make_int2(0, r);
    const int kb = k * bddc::kPanelNB, nb = min(bddc::kPanelNB, n_int - kb), below = n - kb - nb;
    (void)below;
    const int nt = (below + bddc::kTile - 1) / bddc::kTile;
    for (int e = threadIdx.x; e < nt * (nt + 1) / 2; e += blockDim.x) {
        int ti = 0;
        while ((ti + 1) * (ti + 2) / 2 <= e) ++ti;
        int tj = e - ti * (ti + 1) / 2;
        uit[uo + e] = make_int4(0, ti, tj, 0);
    }
    if (threadIdx.x == 0) uit[uo + nt * (nt + 1) / 2] = make_int4(0, -1, -1, 0);
}

// S[p, q] = W[m + max(p, q), m + min(p, q)] (lower triangle of the trailing block)
__global__ void static_extract_kernel(const double *W, int ldw, int m, int ns, double *S, int lds) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)ns * ns;
         e += (int64_t)gridDim.x * blockDim.x) {
        int p = (int)(e % ns), q = (int)(e / ns);
        int a = p > q ? p : q, b = p > q ? q : p;
        S[(size_t)q * lds + p] = W[(size_t)(m + b) * ldw + m + a];
    }
}

}  // namespace

extern "C" bddc_status bddc_schur_dense_static(int n, int n_int, const double *A, int lda, double *S, int lds,
                                               void *stream, char *msg, int msg_cap) {
    using namespace bddc;
    set_msg(msg, msg_cap, "");
    if (n <= 0 || n_int < 0 || n_int >= n || !A || !S || lda < n || lds < n - n_int) {
        set_msg(msg, msg_cap, "bddc_schur_dense_static: invalid sizes or null pointer");
        return BDDC_EINVAL;
    }
    if (n > kMaxN) {
        char buf[160];
        std::snprintf(buf, sizeof(buf), "bddc_schur_dense_static: n = %d exceeds the static scratch limit %d", n,
                      kMaxN);
        set_msg(msg, msg_cap, buf);
        return BDDC_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    void *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) {
        set_msg(msg, msg_cap, cudaGetErrorString(e));
        return BDDC_ECUDA;
    }
    const int ld = (n + 7) / 8 * 8;
    unsigned char *p = static_cast<unsigned char *>(base);
    double *W = reinterpret_cast<double *>(p);
    unsigned char *lists = p + kMatBytes;
    DevStatus *st = reinterpret_cast<DevStatus *>(lists);
    PcholDesc<double> *desc = reinterpret_cast<PcholDesc<double> *>(lists + 256);
    double *diag = reinterpret_cast<double *>(lists + kListBytes - kPanelNB * kPanelNB * sizeof(double));
    // work lists of the batched partial Cholesky (a batch of one matrix), built on the device
    const int steps = (n_int + kPanelNB - 1) / kPanelNB;
    size_t npit = 0, nuit = 0;
    for (int k = 0; k < steps; ++k) {
        npit += panel_count(n, n_int, k);
        nuit += update_count(n, n_int, k);
    }
    const size_t pit_off = 512, uit_off = pit_off + (npit * sizeof(int2) + 255) / 256 * 256;
    if (uit_off + nuit * sizeof(int4) > kListBytes - kPanelNB * kPanelNB * sizeof(double)) {
        set_msg(msg, msg_cap, "bddc_schur_dense_static: work lists exceed the static scratch");
        return BDDC_EINVAL;
    }
    int2 *d_pit = reinterpret_cast<int2 *>(lists + pit_off);
    int4 *d_uit = reinterpret_cast<int4 *>(lists + uit_off);
    static_init_kernel<<<steps > 0 ? steps : 1, 256, 0, s>>>(W, n, ld, n_int, steps, desc, st, d_pit, d_uit, diag);
    e = cudaMemcpy2DAsync(W, (size_t)ld * sizeof(double), A, (size_t)lda * sizeof(double), (size_t)n * sizeof(double),
                          n, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
        set_msg(msg, msg_cap, cudaGetErrorString(e));
        return BDDC_ECUDA;
    }
    int po = 0, uo = 0;
    for (int k = 0; k < steps; ++k) {
        const int np = panel_count(n, n_int, k), nu = update_count(n, n_int, k);
        launch_pchol_panel<double>(desc, d_pit + po, np, k * kPanelNB, st, s);
        launch_pchol_update<double>(desc, d_uit + uo, nu, k * kPanelNB, s);
        po += np;
        uo += nu;
    }
    const int ns = n - n_int;
    static_extract_kernel<<<std::max(1, std::min(1024, (ns * ns + 255) / 256)), 256, 0, s>>>(W, ld, n_int, ns, S,
                                                                                            lds);
    DevStatus hs;
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
        set_msg(msg, msg_cap, cudaGetErrorString(e));
        return BDDC_ECUDA;
    }
    if (hs.code == BDDC_DEV_ERR_NOTSPD) {
        set_msg(msg, msg_cap, "bddc_schur_dense_static: interior block not positive definite");
        return BDDC_ENOTSPD;
    }
    return BDDC_OK;
}
