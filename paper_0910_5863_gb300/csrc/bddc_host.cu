// Host orchestration and C ABI of the adaptive BDDC library.
//
// Phases (the hot path of the method, all numeric work in CUDA kernels):
//   bddc_set_mesh_q1  classification of the interface into faces, edges and
//                     corners (Section 2), index maps, device buffers;
//   bddc_setup        Q1 assembly of A_i, batched partial Cholesky giving
//                     S_i = A_GG - A_GI A_II^{-1} A_IG (Section 2), weights,
//                     local saddle + coarse operators of the preconditioner;
//   bddc_adapt        pair condensations, the face eigenproblems and the new
//                     face constraints (Section 3, Algorithm 3.1);
//   bddc_solve        condensed right-hand side, PCG (Lemma 2.1
//                     preconditioner), interior recovery.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <iterator>
#include <map>
#include <exception>
#include <memory>
#include <thread>
#include <numeric>
#include <set>
#include <string>
#include <vector>
#include <type_traits>

#include "../../include/bddc.h"
#include "assembly.h"
#include "common.cuh"
#include "dense.h"
#include "eig.h"
#include "ff.cuh"
#include "host_util.h"
#include "tc_gemm.h"
#include "mixed.h"
#include "lobpcg.h"
#include "ozaki.h"
#include "pcg.h"
#include "schedule.h"

using namespace bddc;

namespace {

struct SubData {
    std::vector<int64_t> nodes;   // local nodes (sorted), Dirichlet included
    std::vector<int64_t> gI, gG;  // global dofs of interior / interface (sorted)
    int nI = 0, nG = 0, n = 0, ld = 0, ldS = 0;
    std::vector<int> RG;          // interface index of each interface position
    std::vector<int> cpos, rpos;  // corner / remaining interface positions
    std::vector<int> corner_coarse;  // global coarse index of each corner dof (cpos order)
    bool floating = false;
    // constraint rows (averages and adaptive) over interface positions
    int na = 0;
    std::vector<int> row_coarse;  // global coarse index of each row
    // device
    double *A = nullptr, *S = nullptr, *P = nullptr, *Phi = nullptr, *Cb = nullptr;
    int capA = 0;                 // row capacity of Cb
    size_t offI = 0;              // offset in packed interior vectors
};

struct FacePair {
    int i, j;
    std::vector<int64_t> s_g;        // shared non-corner dofs (sorted)
    std::vector<int> pos_i, pos_j;   // their interface positions in i and j
    std::vector<int> face_idx;       // indices into s of the face dofs
    std::vector<int> ci_pos, cj_pos; // shared corner dofs (interface positions)
    bool floating = false;
    int nnull = 0;
    std::vector<double> N0;          // ns x nnull
    // results of the last adapt
    std::vector<double> lam;
    int nsel = 0, nkept = 0, ties = 0;
};

struct GlobRows {               // one glob with constraint rows (c . w equal for all sharing subs)
    std::vector<int> subs;
    std::vector<int64_t> gdofs;
    int nrows = 0;
    std::vector<double> rows;   // host rows (row-major nrows x gdofs) for averages
    int face = -1;              // >= 0: adaptive rows of that face (device buffer)
    int edge = -1;              // >= 0: kept adaptive edge rows, bddc_handle::edge_rows[edge]
    int coarse0 = 0;            // first global coarse index
};

struct PhaseTimer {
    cudaEvent_t a = nullptr, b = nullptr;
};

struct LobStats {   // batched LOBPCG of the last adapt: large faces, most iterations, dense fallbacks
    int faces = 0, iters = 0, fallback = 0;
};

}  // namespace

struct bddc_handle {
    bddc_options opt;
    cudaStream_t stream = nullptr;
    std::string err;
    int64_t launches = 0;
    Arena ar;
    DevStatus *dst = nullptr;
    // mesh
    int ncomp = 1;
    int64_t nn = 0, ne = 0;
    int nsub = 0;
    double nu = 0.0;
    std::vector<double> xyz, coef;
    std::vector<int64_t> elems;
    std::vector<int32_t> esub;
    std::vector<uint8_t> dirich;
    bool have_mesh = false, have_setup = false;
    // algebraic input (bddc_set_problem): per-substructure CSR, host copies
    bool csr_mode = false;
    std::vector<std::vector<int64_t>> csr_l2g, csr_rowptr;
    std::vector<std::vector<int32_t>> csr_col;
    std::vector<std::vector<double>> csr_val;
    // corners given by bddc_set_corners (used instead of the rule when set)
    bool user_corners = false;
    std::vector<int64_t> corner_list;
    std::vector<char> sub_floating;  // substructure without Dirichlet support
    int64_t csr_nnz = 0;             // merged CSR entries uploaded for the dense fill
    // numbering / classification
    std::vector<int64_t> node_first;
    int64_t nfree = 0;
    std::vector<int> node_set;              // set id per node
    std::vector<std::vector<int>> sets;     // set id -> sorted substructures
    std::vector<int64_t> corners;
    std::vector<char> is_corner;
    int n_augmented = 0;  // face nodes promoted to corners (Assumptions 1 and 2)
    std::vector<int32_t> epos;   // mesh input: local dof position of each element's 8 nodes (-1: Dirichlet)
    bool mesh_uploaded = false;  // xyz, elems, coef, esub of this mesh are in the arena
    // device-resident mesh arrays of the running bddc_set_mesh_q1 call (copied device to device)
    const double *in_xyz = nullptr, *in_coef = nullptr;
    const int64_t *in_elems = nullptr;
    const int32_t *in_esub = nullptr;
    int n_edges = 0;
    std::vector<std::pair<std::vector<int>, std::vector<int64_t>>> edge_globs;  // (subs, nodes)
    std::vector<FacePair> faces;
    std::vector<SubData> subs;
    int nG = 0;
    std::vector<int64_t> iface_gdof;
    std::vector<int> gptr, gsub;
    std::vector<int64_t> gent;
    std::vector<int64_t> offG;               // packed offset per sub
    int64_t sumG = 0, sumI = 0;
    std::vector<std::vector<int32_t>> colors;
    int avg_flags = 0;
    std::vector<GlobRows> globs;
    int nC = 0, n_corner_dofs = 0;
    // preconditioner / PCG
    IfaceOps ops{};
    PcgBuffers pb{};
    std::vector<double> alpha, beta;
    int last_iters = 0;
    double setup_ms = 0.0, adapt_ms = 0.0;
    // adapt results
    double omega = 0.0;
    LobStats lob_stats;   // the last adapt's batched LOBPCG (large faces)
    std::vector<double *> face_rows_dev;
    int face_row_ld = 0;
    // kept adaptive edge rows (Section 3's split rows; off unless bddc_set_edge_rows)
    struct EdgeRows {
        int edge_glob;           // index into edge_globs
        const double *rowsT;     // column-major over the edge's dofs (ascending), ld = ld
        int ld;                  // the edge's dofs
        int nrows;
    };
    bool keep_edge_rows = false;
    std::vector<EdgeRows> edge_rows;
    int n_edge_rows = 0, n_edges_with_rows = 0;   // kept by the last adapt
    bool coarse_dirty = true;   // coarse operators are (re)built before the next solve
    bool assembled = false;     // dense local matrices hold the assembled A_i
    bool coarse_fp32 = false;   // the current coarse operators used the FP32 local saddle
    bool interior_fp32 = false; // the current S_i came from the mixed interior elimination
    int interior_fallbacks = 0; // mixed mode: FP32 interior elimination rejected, redone in FP64
    int coarse_fallbacks = 0;   // mixed modes: local saddle rejected, rebuilt in FP64
    bool fp64_class_forced = false;  // mixed mode fallback: FP64-class factorizations in FP64
    float m1_min_pivot = 0.f;
    bool factored = false;      // FP64 mode: A_i factored in place
    int mixed_iters = 0;        // refinement steps the interior elimination needed (mixed mode)
    double mixed_relres = 0.0;  // largest relative residual of the refined A_II X = A_IG
    // kernel timers (bddc_set_kernel_timing): event pairs around the launches of a few
    // kernels, on the handle's stream; the work of every launch is counted on the host
    static constexpr int kKClasses = 9;
    bool ktiming = false;
    std::vector<cudaEvent_t> kev;
    size_t kev_used = 0;
    struct KPending {
        int cls;
        size_t ev;
    };
    std::vector<KPending> kpend;
    double kt_ms[kKClasses] = {}, kt_work[kKClasses] = {};
    int64_t kt_n[kKClasses] = {};
    // phase timing: events [2k, 2k+1] bracket phase k
    static constexpr int kPhases = 9;
    cudaEvent_t ev[2 * kPhases] = {};
    bool ev_used[kPhases] = {};
    bool nvtx_open = false;     // a phase's NVTX range is open on this thread
    double phase_ms[kPhases] = {};
    double phase_flop[kPhases] = {};
};

namespace {

void fail_check(bddc_handle *h, const char *where) {
    DevStatus hs;
    BDDC_CUDA(cudaMemcpyAsync(&hs, h->dst, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->stream));
    BDDC_CUDA(cudaStreamSynchronize(h->stream));
    if (hs.code == BDDC_DEV_ERR_NOTSPD) {
        static const char *names[] = {"?", "interior A_II", "local saddle", "local saddle (FP32)", "local saddle stage 2",
                                      "coarse matrix", "face condensation", "pair corner elimination",
                                      "pair deflated jump system", "interior A_II (FP32)"};
        const int tag = hs.item / 100000, m = hs.item % 100000;
        throw Error{BDDC_ENOTSPD, std::string(where) + ": non-positive pivot in " + names[tag >= 0 && tag < 10 ? tag : 0] +
                                      " matrix " + std::to_string(m) + " near column " + std::to_string(hs.pos)};
    }
    if (hs.code == BDDC_DEV_ERR_TIMEOUT) throw Error{BDDC_ETIMEOUT, std::string(where) + ": device wait timed out"};
    if (hs.code != 0) throw Error{BDDC_ECUDA, std::string(where) + ": device error " + std::to_string(hs.code)};
}

// Device phases, in the order of bddc_get_phase_times.  Each is also an NVTX range around the host
// code that issues it, so a profiler can select a phase's kernels (e.g. ncu --nvtx --nvtx-include
// "pcg/"); without a profiler attached the NVTX calls do nothing.  A range left open by an error
// inside a phase is closed when the next phase begins.
const char *const kPhaseNames[bddc_handle::kPhases] = {
    "assembly", "interior_elimination", "coarse_setup", "pair_condensation", "face_eigen",
    "analysis_host", "condensed_rhs", "pcg", "recovery"};

void phase_begin(bddc_handle *h, int k) {
    BDDC_CUDA(cudaEventRecord(h->ev[2 * k], h->stream));
    h->ev_used[k] = true;
    if (h->nvtx_open) nvtxRangePop();
    nvtxRangePushA(kPhaseNames[k]);
    h->nvtx_open = true;
}
void phase_end(bddc_handle *h, int k) {
    if (h->nvtx_open) nvtxRangePop();
    h->nvtx_open = false;
    BDDC_CUDA(cudaEventRecord(h->ev[2 * k + 1], h->stream));
}
void phase_collect(bddc_handle *h, int k0, int k1) {
    for (int k = k0; k <= k1; ++k) {
        if (!h->ev_used[k]) continue;
        float ms = 0.f;
        BDDC_CUDA(cudaEventSynchronize(h->ev[2 * k + 1]));
        BDDC_CUDA(cudaEventElapsedTime(&ms, h->ev[2 * k], h->ev[2 * k + 1]));
        h->phase_ms[k] = ms;
    }
}

void reset_status(bddc_handle *h) { BDDC_CUDA(cudaMemsetAsync(h->dst, 0, sizeof(DevStatus), h->stream)); }

void check_launch(bddc_handle *h) {
    h->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Error{BDDC_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e)};
}

// ---- kernel timers: classes of bddc_get_kernel_times --------------------------
enum KClass {
    KT_PCHOL_FF = 0, KT_PCHOL_F64 = 1, KT_PCHOL_F32 = 2, KT_TC_GEMM = 3, KT_PCG = 4, KT_FACE_RED = 5, KT_OZAKI = 6,
    KT_OZ_SPLIT = 7, KT_PANEL = 8
};

void kt_collect(bddc_handle *h) {
    for (const auto &p : h->kpend) {
        float ms = 0.f;
        BDDC_CUDA(cudaEventSynchronize(h->kev[p.ev + 1]));
        BDDC_CUDA(cudaEventElapsedTime(&ms, h->kev[p.ev], h->kev[p.ev + 1]));
        h->kt_ms[p.cls] += ms;
    }
    h->kpend.clear();
    h->kev_used = 0;
}

// records the start event of a timed launch; returns its index (or -1 when timing is off)
long kt_begin(bddc_handle *h) {
    if (!h->ktiming) return -1;
    if (h->kev_used + 2 > 4096) kt_collect(h);
    while (h->kev.size() < h->kev_used + 2) {
        cudaEvent_t e;
        BDDC_CUDA(cudaEventCreate(&e));
        h->kev.push_back(e);
    }
    const size_t i = h->kev_used;
    h->kev_used += 2;
    BDDC_CUDA(cudaEventRecord(h->kev[i], h->stream));
    return (long)i;
}

void kt_end(bddc_handle *h, long tok, int cls, double work) {
    if (tok < 0) return;
    BDDC_CUDA(cudaEventRecord(h->kev[tok + 1], h->stream));
    h->kpend.push_back({cls, (size_t)tok});
    h->kt_work[cls] += work;
    h->kt_n[cls] += 1;
}

// ---- batched partial Cholesky ------------------------------------------------
// batch tags reported with a failed pivot
// (a batch name may carry a '#' suffix that keeps its buffers apart, e.g. "E1#2")
int pchol_tag(const std::string &name_in) {
    static const char *names[] = {"", "AII", "M1", "M1f", "M2", "MC", "E1", "E2", "E3", "F"};
    const std::string name = name_in.substr(0, name_in.find('#'));
    for (int k = 1; k < 10; ++k)
        if (name == names[k]) return k;
    return 0;
}

template <typename T>
void run_pchol(bddc_handle *h, const std::vector<PcholDesc<T>> &descs_in, const std::string &tag) {
    if (descs_in.empty()) return;
    std::vector<PcholDesc<T>> descs(descs_in);
    T *scratch = static_cast<T *>(h->ar.get("pc_diag_" + tag, descs.size() * kPanelNB * kPanelNB * sizeof(T)));
    for (size_t k = 0; k < descs.size(); ++k) {
        descs[k].tag = pchol_tag(tag);
        descs[k].diag = scratch + k * kPanelNB * kPanelNB;
    }
    int nsteps = 0;
    for (auto &d : descs) nsteps = std::max(nsteps, (d.nstop + kPanelNB - 1) / kPanelNB);
    std::vector<int2> pitems;
    std::vector<int4> uitems;
    std::vector<int> poff(nsteps + 1, 0), uoff(nsteps + 1, 0);
    for (int s = 0; s < nsteps; ++s) {
        int kb = s * kPanelNB;
        poff[s] = (int)pitems.size();
        uoff[s] = (int)uitems.size();
        for (int m = 0; m < (int)descs.size(); ++m) {
            const auto &d = descs[m];
            if (kb >= d.nstop) continue;
            int nb = std::min(kPanelNB, d.nstop - kb);
            int below = d.n - kb - nb;
            // rows [z0, z1) are identity rows that this step leaves untouched (PcholDesc::id0)
            const int z0 = d.id0 > 0 ? d.id0 + std::max(0, kb + nb - d.idc) : d.n;
            const int z1 = d.id0 > 0 ? std::min(d.n, d.id0 + d.nstop - d.idc) : d.n;
            auto idle = [&](int r0, int r1) { return r0 >= z0 && std::min(r1, d.n) <= z1; };
            int np = std::max(1, (below + kPanelRows - 1) / kPanelRows);
            for (int r = 0; r < np; ++r) {
                const int r0 = kb + nb + r * kPanelRows;
                if (r > 0 && idle(r0, r0 + kPanelRows)) continue;
                pitems.push_back(make_int2(m, r));
            }
            uitems.push_back(make_int4(m, -1, -1, 0));  // copy of the factored diagonal block
            int tn = d.n - kb - nb;
            int nt = (tn + kTile - 1) / kTile;
            int ct = nt;   // column tiles: all, or those left of d.ncol
            if (d.ncol > 0) {
                const int cw = std::min(d.ncol, d.n) - kb - nb;
                ct = cw > 0 ? (cw + kTile - 1) / kTile : 0;
            }
            for (int ti = 0; ti < nt; ++ti) {
                const int i0 = kb + nb + ti * kTile;
                if (idle(i0, i0 + kTile)) continue;
                for (int tj = 0; tj <= ti && tj < ct; ++tj) {
                    const int j0 = kb + nb + tj * kTile;
                    if (idle(j0, j0 + kTile)) continue;
                    uitems.push_back(make_int4(m, ti, tj, 0));
                }
            }
        }
    }
    poff[nsteps] = (int)pitems.size();
    uoff[nsteps] = (int)uitems.size();
    auto *dd = h->ar.upload("pc_desc_" + tag, descs, h->stream);
    auto *dp = h->ar.upload("pc_pit_" + tag, pitems, h->stream);
    auto *du = h->ar.upload("pc_uit_" + tag, uitems, h->stream);
    const int cls = std::is_same<T, ff>::value ? KT_PCHOL_FF : (std::is_same<T, double>::value ? KT_PCHOL_F64 : KT_PCHOL_F32);
    for (int s = 0; s < nsteps; ++s) {
        int kb = s * kPanelNB;
        const long tokp = kt_begin(h);
        launch_pchol_panel<T>(dd, dp + poff[s], poff[s + 1] - poff[s], kb, h->dst, h->stream);
        check_launch(h);
        kt_end(h, tokp, KT_PANEL, 0.0);
        double work = 0.0;   // the trailing update's multiply-adds x 2 (lower triangle of diagonal tiles)
        if (h->ktiming)
            for (int u = uoff[s]; u < uoff[s + 1]; ++u) {
                const int4 w = uitems[u];
                if (w.y < 0) continue;
                const auto &d = descs[w.x];
                const int nb = std::min(kPanelNB, d.nstop - kb), t0 = kb + nb;
                const int cend = d.ncol > 0 ? std::min(d.ncol, d.n) : d.n;
                const double r = std::min(kTile, d.n - (t0 + w.y * kTile));
                const double c = std::min(kTile, cend - (t0 + w.z * kTile));
                work += 2.0 * nb * (w.y == w.z ? r * (r + 1) / 2 : r * c);
            }
        const long tok = kt_begin(h);
        launch_pchol_update<T>(dd, du + uoff[s], uoff[s + 1] - uoff[s], kb, h->stream);
        check_launch(h);
        kt_end(h, tok, cls, work);
    }
}

// Double-float partial Cholesky in block columns of kOzK = 128, every block column in
// five launches: (1) the w x w diagonal block factored in shared memory, with the inverse
// of its factor (one CTA per matrix); (2) the rows below and that inverse split into bf16
// digit planes; (3) those rows times the inverse's transpose on the tensor cores, which is
// the block column of the factor, L21 = A21 L11^-T; (4) L21 split; (5) the trailing block
// updated on the tensor cores, C -= L21 L21^T (ozaki.h).  Rows of an identity block that
// are still zero in the block column (PcholDesc::id0) take no part in (3) and (5): their
// tiles are skipped (zero rows of A21 give zero rows of L21).
void run_pchol_oz(bddc_handle *h, const std::vector<PcholDesc<ff>> &descs, const std::string &tag) {
    constexpr int W = kOzK;
    int nJ = 0;
    for (const auto &d : descs) nJ = std::max(nJ, (d.nstop + W - 1) / W);
    for (int jb = 0; jb < nJ; ++jb) {
        const int J = jb * W;
        const std::string t = tag + "_oz" + std::to_string(jb);
        std::vector<OzDiagDesc> dg;
        std::vector<OzSplitDesc> sd1, sd2;
        std::vector<OzSyrkDesc> gd, yd;
        std::vector<int2> si1, si2;
        std::vector<int4> gi, yi;
        size_t nsl = 0, nex = 0, ndg = 0;
        for (const auto &d : descs) {
            if (J >= d.nstop) continue;
            const int w = std::min(W, d.nstop - J), rows = d.n - J - w;
            ++ndg;
            if (rows > 0) {
                nsl += (size_t)oz_rows_pad(rows) * kOzSlices * W;
                nex += rows;
            }
        }
        ff *linv = h->ar.get_t<ff>("oz_linv_" + tag, std::max<size_t>(ndg, 1) * W * W);
        const size_t lsl = (size_t)oz_rows_pad(W) * kOzSlices * W;   // digit planes of one inverse
        uint16_t *slices = h->ar.get_t<uint16_t>("oz_sl_" + tag, std::max<size_t>(nsl, 8));
        uint16_t *lslices = h->ar.get_t<uint16_t>("oz_lsl_" + tag, std::max<size_t>(ndg, 1) * lsl);
        int *rexp = h->ar.get_t<int>("oz_ex_" + tag, std::max<size_t>(nex, 1));
        int *lrexp = h->ar.get_t<int>("oz_lex_" + tag, std::max<size_t>(ndg, 1) * W);
        size_t osl = 0, oex = 0;
        double work = 0.0, gwork = 0.0;
        for (const auto &d : descs) {
            if (J >= d.nstop) continue;
            const int w = std::min(W, d.nstop - J), rows = d.n - J - w;
            const size_t ld = (size_t)d.ld;
            const int q = (int)dg.size();
            ff *Li = linv + (size_t)q * W * W;
            dg.push_back(OzDiagDesc{d.A + (size_t)J * ld + J, d.ld, w, Li, d.tag, d.fail});
            if (rows <= 0) continue;
            const int k1 = (int)sd1.size();
            ff *A21 = d.A + (size_t)J * ld + J + w;
            // (2): A21 and the inverse; (4): L21 again into the same planes, after (3) consumed them
            sd1.push_back(OzSplitDesc{A21, d.ld, rows, w, slices + osl, rexp + oex});
            for (int g = 0; g < (oz_rows_pad(rows) + 255) / 256; ++g) si1.push_back(make_int2(k1, g));
            const int k1b = (int)sd1.size();
            sd1.push_back(OzSplitDesc{Li, W, w, w, lslices + (size_t)q * lsl, lrexp + (size_t)q * W});
            si1.push_back(make_int2(k1b, 0));
            const int k2 = (int)sd2.size();
            sd2.push_back(OzSplitDesc{A21, d.ld, rows, w, slices + osl, rexp + oex});
            for (int g = 0; g < (oz_rows_pad(rows) + 255) / 256; ++g) si2.push_back(make_int2(k2, g));
            const int kg = (int)gd.size();
            gd.push_back(OzSyrkDesc{A21, d.ld, rows, slices + osl, rexp + oex, lslices + (size_t)q * lsl,
                                    lrexp + (size_t)q * W, w, 1});
            const int ky = (int)yd.size();
            yd.push_back(OzSyrkDesc{d.A + (size_t)(J + w) * ld + J + w, d.ld, rows, slices + osl, rexp + oex,
                                    slices + osl, rexp + oex, rows, 0});
            osl += (size_t)oz_rows_pad(rows) * kOzSlices * W;
            oex += rows;
            // identity rows still zero in this block column (row id0 + q with idc + q >= J + w):
            // view rows [z0, z1) of the trailing block, whose origin is row J + w
            int z0 = rows, z1 = rows;
            if (d.id0 > 0) {
                z0 = std::max(0, std::max(d.id0 - J - w, d.id0 - d.idc));
                z1 = std::min(rows, d.id0 + d.nstop - d.idc - J - w);
                if (z0 >= z1) z0 = z1 = rows;
            }
            auto idle = [&](int a, int b) { return a >= z0 && std::min(b, rows) <= z1; };
            for (int a = 0; a * kOzTileM < rows; ++a) {
                if (idle(a * kOzTileM, (a + 1) * kOzTileM)) continue;
                const double r = std::min(kOzTileM, rows - a * kOzTileM);
                for (int c = 0; c * kOzTileN < w; ++c) {
                    gi.push_back(make_int4(kg, a, c, 0));
                    gwork += 2.0 * w * r * std::min(kOzTileN, w - c * kOzTileN);
                }
                for (int c = 0; c * kOzTileN < rows && c * kOzTileN <= a * kOzTileM + kOzTileM - 1; ++c) {
                    if (idle(c * kOzTileN, (c + 1) * kOzTileN)) continue;
                    yi.push_back(make_int4(ky, a, c, 0));
                    work += 2.0 * w * r * std::min(kOzTileN, rows - c * kOzTileN);
                }
            }
        }
        auto *ddg = h->ar.upload("oz_dg_" + t, dg, h->stream);
        const long tokd = kt_begin(h);
        launch_oz_diag(ddg, (int)dg.size(), h->dst, h->stream);
        check_launch(h);
        kt_end(h, tokd, KT_PANEL, 0.0);
        if (sd1.empty()) continue;
        auto split = [&](const std::vector<OzSplitDesc> &v, const std::vector<int2> &it, const std::string &nm) {
            auto *dd = h->ar.upload("oz_sd" + nm + "_" + t, v, h->stream);
            auto *di = h->ar.upload("oz_si" + nm + "_" + t, it, h->stream);
            const long tok = kt_begin(h);
            launch_oz_split(dd, di, (int)it.size(), h->stream);
            check_launch(h);
            kt_end(h, tok, KT_OZ_SPLIT, 0.0);
        };
        auto products = [&](const std::vector<OzSyrkDesc> &v, const std::vector<int4> &it, const std::string &nm,
                            double wk) {
            if (it.empty()) return;
            auto *dd = h->ar.upload("oz_yd" + nm + "_" + t, v, h->stream);
            auto *di = h->ar.upload("oz_yi" + nm + "_" + t, it, h->stream);
            const long tok = kt_begin(h);
            launch_oz_syrk(dd, di, (int)it.size(), h->dst, h->opt.timeout_s, h->stream);
            check_launch(h);
            kt_end(h, tok, KT_OZAKI, wk);
        };
        split(sd1, si1, "1");
        products(gd, gi, "g", gwork);
        split(sd2, si2, "2");
        products(yd, yi, "y", work);
    }
}

// Partial Cholesky of FP64 matrices in the FP64-class arithmetic of the precision
// mode: FP64 in BDDC_FP64; in the mixed modes double-float (the lower triangles are
// converted in place before and after, the upper triangles are not touched), with the
// trailing updates on the tensor cores (run_pchol_oz) unless mixed_updates selects the
// FP32 pipe.
void run_pchol_fp64class(bddc_handle *h, const std::vector<PcholDesc<double>> &descs, const std::string &tag) {
    if (descs.empty()) return;
    if (h->opt.precision == BDDC_FP64 || h->fp64_class_forced) {
        run_pchol<double>(h, descs, tag);
        return;
    }
    std::vector<int2> items;
    for (int m = 0; m < (int)descs.size(); ++m)
        for (int j = 0; j < descs[m].n; j += kConvertCols) items.push_back(make_int2(m, j));
    auto *dd = h->ar.upload("ffc_desc_" + tag, descs, h->stream);
    auto *di = h->ar.upload("ffc_it_" + tag, items, h->stream);
    launch_ff_convert(dd, di, (int)items.size(), 1, h->stream);
    check_launch(h);
    std::vector<PcholDesc<ff>> fd;
    for (const auto &d : descs)
        fd.push_back(PcholDesc<ff>{reinterpret_cast<ff *>(d.A), d.n, d.ld, d.nstop, d.tag, nullptr, d.ncol, d.id0,
                                   d.idc, d.fail});
    if (h->opt.mixed_updates == 0)
        run_pchol_oz(h, fd, tag);
    else
        run_pchol<ff>(h, fd, tag);
    launch_ff_convert(dd, di, (int)items.size(), 0, h->stream);
    check_launch(h);
}

void run_gathers(bddc_handle *h, const std::vector<GatherOp> &ops, const std::string &tag) {
    if (ops.empty()) return;
    std::vector<int2> items;
    for (int k = 0; k < (int)ops.size(); ++k)
        for (int q = 0; q < (ops[k].nc + 7) / 8; ++q) items.push_back(make_int2(k, q));
    auto *d_ops = h->ar.upload("g_ops_" + tag, ops, h->stream);
    auto *d_items = h->ar.upload("g_it_" + tag, items, h->stream);
    launch_gather(d_ops, d_items, (int)items.size(), h->stream);
    check_launch(h);
}

void run_diag(bddc_handle *h, const std::vector<DiagOp> &ops, const std::string &tag) {
    if (ops.empty()) return;
    auto *d = h->ar.upload("d_ops_" + tag, ops, h->stream);
    launch_diag_set(d, (int)ops.size(), h->stream);
    check_launch(h);
}

void run_gemm(bddc_handle *h, const std::vector<GemmDesc> &descs, const std::string &tag, bool use_ff = false) {
    if (descs.empty()) return;
    std::vector<int4> items;
    for (int k = 0; k < (int)descs.size(); ++k)
        for (int a = 0; a < (descs[k].m + kTile - 1) / kTile; ++a)
            for (int b = 0; b < (descs[k].n + kTile - 1) / kTile; ++b) items.push_back(make_int4(k, a, b, 0));
    auto *dd = h->ar.upload("gm_desc_" + tag, descs, h->stream);
    auto *di = h->ar.upload("gm_it_" + tag, items, h->stream);
    launch_gemm(dd, di, (int)items.size(), use_ff ? 1 : 0, h->stream);
    check_launch(h);
}

void run_gemv(bddc_handle *h, const std::vector<GemmDesc> &descs, const std::string &tag) {
    if (descs.empty()) return;
    std::vector<int2> items;
    for (int k = 0; k < (int)descs.size(); ++k) {
        const int rows = descs[k].transA ? 8 : 32;
        for (int r = 0; r < (descs[k].m + rows - 1) / rows; ++r) items.push_back(make_int2(k, r));
    }
    auto *dd = h->ar.upload("gv_desc_" + tag, descs, h->stream);
    auto *di = h->ar.upload("gv_it_" + tag, items, h->stream);
    launch_gemv(dd, di, (int)items.size(), h->stream);
    check_launch(h);
}

// Batched 3xTF32 tensor-core GEMMs (tc_gemm.cu): items are the 128 x 128 output tiles
// (with lower_only, the tiles on or below the diagonal of a square C).
std::vector<int4> tc_items(const std::vector<TcGemm> &jobs, bool lower_only = false) {
    std::vector<int4> items;
    for (int k = 0; k < (int)jobs.size(); ++k) {
        const auto &g = jobs[k];
        if (g.M <= 0 || g.N <= 0 || g.K <= 0) continue;
        const auto aligned = [](const void *p, int ld, int f64) {
            return ((uintptr_t)p % 16 == 0) && ((size_t)ld * (f64 ? 8 : 4)) % 16 == 0;
        };
        BDDC_REQUIRE(!g.a_f64 && !g.b_f64, BDDC_EINVAL, "tensor-core GEMM operands must be FP32");
        BDDC_REQUIRE(aligned(g.A, g.lda, g.a_f64) && aligned(g.B, g.ldb, g.b_f64), BDDC_EINVAL,
                     "tensor-core GEMM operand rows must be 16-byte aligned");
        for (int a = 0; a < (g.M + kTcM - 1) / kTcM; ++a)
            for (int b = 0; b < (g.N + kTcN - 1) / kTcN; ++b)
                if (!lower_only || b * kTcN <= a * kTcM + kTcM - 1) items.push_back(make_int4(k, a, b, 0));
    }
    return items;
}

void run_tc_gemm(bddc_handle *h, const std::vector<TcGemm> &jobs, const std::string &tag, bool lower_only = false) {
    std::vector<int4> items = tc_items(jobs, lower_only);
    if (items.empty()) return;
    auto *dj = h->ar.upload("tcj_" + tag, jobs, h->stream);
    auto *di = h->ar.upload("tci_" + tag, items, h->stream);
    double work = 0.0;   // effective multiply-adds x 2 (each executed as three TF32 products)
    for (const auto &g : jobs)
        if (g.M > 0 && g.N > 0 && g.K > 0) work += 2.0 * g.M * g.N * g.K * (lower_only ? 0.5 : 1.0);
    const long tok = kt_begin(h);
    launch_tc_gemm(dj, di, (int)items.size(), h->dst, h->opt.timeout_s, h->stream);
    check_launch(h);
    kt_end(h, tok, KT_TC_GEMM, work);
}

// FP32 partial Cholesky, left-looking in block columns of 128 with the long
// updates on the tensor cores (3xTF32, tc_gemm.cu).  For every block column J:
//   1. A[J:n, J:J+w] -= L[J:n, 0:J] L[J:J+w, 0:J]^T   (tensor cores, K = J),
//   2. the block column is factored by the right-looking panel kernels with
//      their updates confined to its w columns,
//   3. its L is copied, transposed, into the strict upper triangle, so that
//      row r of L is contiguous there (the K-major operand layout of step 1).
// After the last block column the trailing block is updated once,
// A[nstop:n, nstop:n] -= L21 L21^T (lower tiles only).  The strict upper
// triangle is overwritten: it must not hold anything the caller needs.
void run_pchol_tc(bddc_handle *h, const std::vector<PcholDesc<float>> &descs, const std::string &tag) {
    constexpr int W = 128;
    int nJ = 0;
    for (const auto &d : descs) nJ = std::max(nJ, (d.nstop + W - 1) / W);
    for (int jb = 0; jb < nJ; ++jb) {
        const int J = jb * W;
        const std::string t = tag + "_" + std::to_string(jb);
        std::vector<TcGemm> upd;
        std::vector<PcholDesc<float>> pv;
        std::vector<TransposeOp> tr;
        std::vector<int4> titems;
        for (const auto &d : descs) {
            if (J >= d.nstop) continue;
            const int w = std::min(W, d.nstop - J);
            float *F = d.A;
            const size_t ld = (size_t)d.ld;
            if (J > 0)
                upd.push_back(TcGemm{F + J * ld, F + J * ld, F + J * ld + J, nullptr, nullptr, d.ld, d.ld, d.ld,
                                     d.n - J, w, J, 0, 0, -1.0, 1});
            PcholDesc<float> v{F + J * ld + J, d.n - J, d.ld, w, 0, nullptr, w};
            pv.push_back(v);
            if (J + w < d.n) {   // upper (J + p, J + w + q) <- lower (J + w + q, J + p)
                const int k = (int)tr.size(), nc = d.n - J - w;
                tr.push_back(TransposeOp{F, d.ld, J, J + w, w, nc});
                for (int a = 0; a < (w + 31) / 32; ++a)
                    for (int b = 0; b < (nc + 31) / 32; ++b) titems.push_back(make_int4(k, a, b, 0));
            }
        }
        run_tc_gemm(h, upd, t);
        run_pchol<float>(h, pv, tag);
        if (!titems.empty()) {
            auto *dto = h->ar.upload("tr_o_" + t, tr, h->stream);
            auto *dti = h->ar.upload("tr_i_" + t, titems, h->stream);
            launch_transpose_block(dto, dti, (int)titems.size(), h->stream);
            check_launch(h);
        }
    }
    std::vector<TcGemm> trail;
    for (const auto &d : descs) {
        if (d.nstop <= 0 || d.nstop >= d.n) continue;
        float *F = d.A;
        const size_t ld = (size_t)d.ld, k = (size_t)d.nstop;
        trail.push_back(TcGemm{F + k * ld, F + k * ld, F + k * ld + k, nullptr, nullptr, d.ld, d.ld, d.ld,
                               d.n - d.nstop, d.n - d.nstop, d.nstop, 0, 0, -1.0, 1});
    }
    run_tc_gemm(h, trail, tag + "_trail", true);
}

void zero(bddc_handle *h, double *p, size_t n) {
    launch_zero(p, n, h->stream);
    check_launch(h);
}

// buffers to clear with a single launch
struct ZeroList {
    std::vector<double *> p;
    std::vector<int64_t> n;
    void add(double *ptr, size_t count) {
        p.push_back(ptr);
        n.push_back((int64_t)count);
    }
};

void zero_all(bddc_handle *h, const ZeroList &z, const std::string &tag) {
    if (z.p.empty()) return;
    std::vector<int2> items;
    for (int k = 0; k < (int)z.p.size(); ++k)
        for (int64_t c = 0; c < (z.n[k] + 8191) / 8192; ++c) items.push_back(make_int2(k, (int)c));
    auto *dp = h->ar.upload("z_p_" + tag, z.p, h->stream);
    auto *dn = h->ar.upload("z_n_" + tag, z.n, h->stream);
    auto *di = h->ar.upload("z_i_" + tag, items, h->stream);
    launch_zero_many(dp, dn, di, (int)items.size(), h->stream);
    check_launch(h);
}

GatherOp gop(const double *src, int ld_src, double *dst, int ld_dst, int nr, int nc) {
    GatherOp o;
    memset(&o, 0, sizeof(o));
    o.src = src;
    o.ld_src = ld_src;
    o.dst = dst;
    o.ld_dst = ld_dst;
    o.nr = nr;
    o.nc = nc;
    o.scale = 1.0;
    return o;
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

// ---- classification ------------------------------------------------------
const int HEX_EDGES[12][2] = {{0, 1}, {2, 3}, {4, 5}, {6, 7}, {0, 2}, {1, 3},
                              {4, 6}, {5, 7}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};

// Corner augmentation (Assumptions 1 and 2: the corners shared by a face pair with a
// floating member must fix its rigid modes).  Face pairs are visited in increasing
// (i, j); while the shared corners fix fewer than 1 (scalar) or 3 (elasticity: three
// non-collinear points) modes, the face node farthest from the shared corners (the
// largest smallest squared distance; ties within 1e-12 relative go to the lowest node
// id; the lowest node id when there are no shared corners) becomes a corner.  A node
// promoted for (i, j) belongs to that face only, so the faces do not interact.
using FaceList = std::vector<std::pair<std::pair<int, int>, std::vector<int64_t>>>;

int corner_fixed_modes(const bddc_handle *h, const std::vector<int64_t> &cn, int need) {
    if (cn.empty()) return 0;
    if (need == 1) return 1;
    const double *x0 = &h->xyz[cn[0] * 3];
    int best = 1;
    for (size_t a = 1; a < cn.size(); ++a) {
        const double *xa = &h->xyz[cn[a] * 3];
        double d1[3] = {xa[0] - x0[0], xa[1] - x0[1], xa[2] - x0[2]};
        double n1 = std::sqrt(d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2]);
        if (n1 > 0) best = 2;
        for (size_t b = a + 1; b < cn.size(); ++b) {
            const double *xb = &h->xyz[cn[b] * 3];
            double d2[3] = {xb[0] - x0[0], xb[1] - x0[1], xb[2] - x0[2]};
            double cr[3] = {d1[1] * d2[2] - d1[2] * d2[1], d1[2] * d2[0] - d1[0] * d2[2],
                            d1[0] * d2[1] - d1[1] * d2[0]};
            double n2 = std::sqrt(d2[0] * d2[0] + d2[1] * d2[1] + d2[2] * d2[2]);
            if (std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]) > 1e-8 * n1 * n2) return 3;
        }
    }
    return best;
}

void augment_corners(bddc_handle *h, FaceList &face_list) {
    const int ns = h->nsub, need = (h->ncomp == 1) ? 1 : 3;
    std::vector<std::vector<int64_t>> sub_corners(ns);
    for (int64_t v : h->corners)
        for (int sb : h->sets[h->node_set[v]]) sub_corners[sb].push_back(v);
    h->n_augmented = 0;
    for (auto &fl : face_list) {
        const int i = fl.first.first, j = fl.first.second;
        if (!h->sub_floating[i] && !h->sub_floating[j]) continue;
        std::vector<int64_t> shared;
        std::set_intersection(sub_corners[i].begin(), sub_corners[i].end(), sub_corners[j].begin(),
                              sub_corners[j].end(), std::back_inserter(shared));
        auto &face = fl.second;
        while (!face.empty() && corner_fixed_modes(h, shared, need) < need) {
            size_t pick = 0;
            if (!shared.empty()) {
                std::vector<double> dmin(face.size());
                double best = -1.0;
                for (size_t q = 0; q < face.size(); ++q) {
                    const double *x = &h->xyz[face[q] * 3];
                    double m = INFINITY;
                    for (int64_t v : shared) {
                        const double *y = &h->xyz[v * 3];
                        double dx = x[0] - y[0], dy = x[1] - y[1], dz = x[2] - y[2];
                        m = std::min(m, dx * dx + dy * dy + dz * dz);
                    }
                    dmin[q] = m;
                    best = std::max(best, m);
                }
                while (dmin[pick] < best * (1 - 1e-12)) ++pick;
            }
            const int64_t v = face[pick];
            face.erase(face.begin() + pick);
            shared.push_back(v);
            h->is_corner[v] = 1;
            h->corners.push_back(v);
            h->n_augmented++;
        }
    }
    if (h->n_augmented) {
        std::sort(h->corners.begin(), h->corners.end());
        face_list.erase(std::remove_if(face_list.begin(), face_list.end(),
                                       [](const FaceList::value_type &f) { return f.second.empty(); }),
                        face_list.end());
    }
}

// Floating substructures (no Dirichlet support).  Mesh input: no element of the
// substructure touches a Dirichlet node.  Algebraic input: A_i annihilates every
// rigid mode r (the constant for ncomp = 1; three translations and three
// rotations e_a x x for ncomp = 3) to 1e-8 relative: max |A_i r| <= 1e-8 max_k
// sum_l |A_i,kl| |r_l|.
void mark_floating(bddc_handle *h) {
    const int ns = h->nsub, c = h->ncomp;
    h->sub_floating.assign(ns, 1);
    if (!h->csr_mode) {
        for (int64_t e = 0; e < h->ne; ++e)
            for (int a = 0; a < 8; ++a)
                if (h->dirich[h->elems[e * 8 + a]]) h->sub_floating[h->esub[e]] = 0;
        return;
    }
    const int nmodes = (c == 1) ? 1 : 6;
    for (int s = 0; s < ns; ++s) {
        const auto &l2g = h->csr_l2g[s];
        const auto &rp = h->csr_rowptr[s];
        const auto &cl = h->csr_col[s];
        const auto &vl = h->csr_val[s];
        const size_t n = l2g.size();
        std::vector<double> r(n);
        for (int m = 0; m < nmodes && h->sub_floating[s]; ++m) {
            for (size_t k = 0; k < n; ++k) {
                const int64_t g = l2g[k];
                const int comp = (int)(g % c);
                if (m < 3 || c == 1) {
                    r[k] = (c == 1 || comp == m) ? 1.0 : 0.0;
                } else {
                    // (e_a x x)_comp for a = m - 3
                    const double *x = &h->xyz[(g / c) * 3];
                    const int a = m - 3, b1 = (a + 1) % 3, b2 = (a + 2) % 3;
                    r[k] = comp == b1 ? -x[b2] : (comp == b2 ? x[b1] : 0.0);
                }
            }
            double worst = 0.0, scale = 0.0;
            for (size_t k = 0; k < n; ++k) {
                double y = 0.0, a = 0.0;
                for (int64_t q = rp[k]; q < rp[k + 1]; ++q) {
                    y += vl[q] * r[cl[q]];
                    a += std::fabs(vl[q]) * std::fabs(r[cl[q]]);
                }
                worst = std::max(worst, std::fabs(y));
                scale = std::max(scale, a);
            }
            if (worst > 1e-8 * scale) h->sub_floating[s] = 0;
        }
    }
}

std::vector<int32_t> element_positions(bddc_handle *h);

// Greedy element colouring for the race-free scatter of element matrices: an element
// takes the lowest colour not used by an element sharing one of its nodes.
void colour_elements(const bddc_handle *h, std::vector<std::vector<int32_t>> &colors) {
    colors.clear();
    std::vector<uint64_t> node_mask(h->nn, 0);
    for (int64_t e = 0; e < h->ne; ++e) {
        uint64_t used = 0;
        for (int a = 0; a < 8; ++a) used |= node_mask[h->elems[e * 8 + a]];
        int col = 0;
        while (col < 64 && (used >> col) & 1ull) ++col;
        BDDC_REQUIRE(col < 64, BDDC_EINVAL, "element colouring needs more than 64 colours");
        for (int a = 0; a < 8; ++a) node_mask[h->elems[e * 8 + a]] |= (1ull << col);
        if ((int)colors.size() <= col) colors.resize(col + 1);
        colors[col].push_back((int32_t)e);
    }
}

// A helper thread of the mesh analysis: joined when the scope ends (also on an
// exception), its own exception kept for rethrow() on the calling thread.
struct HostTask {
    std::thread t;
    std::exception_ptr err;
    template <typename F>
    void start(F f) {
        t = std::thread([this, f]() {
            try {
                f();
            } catch (...) {
                err = std::current_exception();
            }
        });
    }
    void join() {
        if (t.joinable()) t.join();
    }
    void rethrow() {
        join();
        if (err) std::rethrow_exception(err);
    }
    ~HostTask() { join(); }
};

void classify(bddc_handle *h) {
    const auto tc0 = std::chrono::steady_clock::now();
    const int64_t nn = h->nn, ne = h->ne;
    const int c = h->ncomp;
    // mesh input: the element colouring needs only the elements; it runs beside the rest
    std::vector<std::vector<int32_t>> colors;
    HostTask colour_task, epos_task;
    if (!h->csr_mode) colour_task.start([h, &colors]() { colour_elements(h, colors); });
    // free dofs
    h->node_first.assign(nn, -1);
    int64_t nf = 0;
    for (int64_t v = 0; v < nn; ++v)
        if (!h->dirich[v]) {
            h->node_first[v] = nf;
            nf += c;
        }
    h->nfree = nf;
    // node -> sorted set of substructures (flat, at most kMaxSet per node)
    constexpr int kMaxSet = 16;
    struct NodeSubs {
        int cnt;
        int s[kMaxSet];
    };
    std::unique_ptr<NodeSubs[]> nsv_buf(new NodeSubs[nn]);   // only the counts are initialised
    NodeSubs *nsv = nsv_buf.get();
    for (int64_t v = 0; v < nn; ++v) nsv[v].cnt = 0;
    auto add_sub = [&](int64_t v, int sb) {
        NodeSubs &x = nsv[v];
        for (int k = 0; k < x.cnt; ++k)
            if (x.s[k] == sb) return;
        BDDC_REQUIRE(x.cnt < kMaxSet, BDDC_EINVAL, "a node lies in more than 16 substructures");
        x.s[x.cnt++] = sb;
    };
    if (h->csr_mode) {
        for (int sb = 0; sb < h->nsub; ++sb)
            for (int64_t g : h->csr_l2g[sb]) add_sub(g / c, sb);
    } else {
        for (int64_t e = 0; e < ne; ++e)
            for (int a = 0; a < 8; ++a) add_sub(h->elems[e * 8 + a], h->esub[e]);
    }
    for (int64_t v = 0; v < nn; ++v) std::sort(nsv[v].s, nsv[v].s + nsv[v].cnt);
    // set ids: {s} -> s for the one-substructure sets; interface sets are sorted by key
    h->sets.clear();
    for (int sb = 0; sb < h->nsub; ++sb) h->sets.push_back({sb});
    std::vector<int> set_count(h->nsub, 0);
    h->node_set.assign(nn, -1);
    struct Key {
        int cnt;
        int s[kMaxSet];
        int64_t node;
    };
    std::vector<Key> keys;
    for (int64_t v = 0; v < nn; ++v) {
        const NodeSubs &x = nsv[v];
        BDDC_REQUIRE(x.cnt >= 1, BDDC_EINVAL, "a node belongs to no substructure");
        if (x.cnt == 1) {
            h->node_set[v] = x.s[0];
            set_count[x.s[0]]++;
            continue;
        }
        Key k;
        k.cnt = x.cnt;
        for (int q = 0; q < kMaxSet; ++q) k.s[q] = q < x.cnt ? x.s[q] : -1;
        k.node = v;
        keys.push_back(k);
    }
    auto key_less = [](const Key &a, const Key &b) {
        if (a.cnt != b.cnt) return a.cnt < b.cnt;
        for (int q = 0; q < a.cnt; ++q)
            if (a.s[q] != b.s[q]) return a.s[q] < b.s[q];
        return a.node < b.node;
    };
    auto key_same = [](const Key &a, const Key &b) {
        if (a.cnt != b.cnt) return false;
        for (int q = 0; q < a.cnt; ++q)
            if (a.s[q] != b.s[q]) return false;
        return true;
    };
    std::sort(keys.begin(), keys.end(), key_less);
    for (size_t q = 0; q < keys.size(); ++q) {
        if (q == 0 || !key_same(keys[q], keys[q - 1])) {
            h->sets.emplace_back(keys[q].s, keys[q].s + keys[q].cnt);
            set_count.push_back(0);
        }
        h->node_set[keys[q].node] = (int)h->sets.size() - 1;
        set_count.back()++;
    }
    // element-edge neighbours of nodes in edge sets (set size >= 3)
    std::vector<int> eidx(nn, -1);
    int n_edge_nodes = 0;
    for (int64_t v = 0; v < nn; ++v)
        if (nsv[v].cnt >= 3) eidx[v] = n_edge_nodes++;
    std::vector<std::vector<int64_t>> nb(n_edge_nodes);
    if (h->csr_mode) {
        // neighbours = nodes coupled to the node in some A_i
        for (int sb = 0; sb < h->nsub; ++sb) {
            const auto &l2g = h->csr_l2g[sb];
            const auto &rp = h->csr_rowptr[sb];
            const auto &cl = h->csr_col[sb];
            for (size_t r = 0; r < l2g.size(); ++r) {
                const int64_t u = l2g[r] / c;
                if (eidx[u] < 0) continue;
                for (int64_t q = rp[r]; q < rp[r + 1]; ++q) {
                    const int64_t v = l2g[cl[q]] / c;
                    if (v != u) nb[eidx[u]].push_back(v);
                }
            }
        }
    } else {
        for (int64_t e = 0; e < ne; ++e)
            for (auto &ed : HEX_EDGES) {
                int64_t a = h->elems[e * 8 + ed[0]], b = h->elems[e * 8 + ed[1]];
                if (eidx[a] >= 0) nb[eidx[a]].push_back(b);
                if (eidx[b] >= 0) nb[eidx[b]].push_back(a);
            }
    }
    auto is_superset = [&](int big, int small) {
        const auto &B = h->sets[big], &S = h->sets[small];
        if (B.size() <= S.size()) return false;
        return std::includes(B.begin(), B.end(), S.begin(), S.end());
    };
    h->is_corner.assign(nn, 0);
    if (h->user_corners) {
        for (int64_t v : h->corner_list) {
            BDDC_REQUIRE(v >= 0 && v < nn, BDDC_EINVAL, "corner node id out of range");
            BDDC_REQUIRE(h->sets[h->node_set[v]].size() >= 2 && !h->dirich[v], BDDC_EINVAL,
                         "corner node " + std::to_string(v) + " is not an interface node");
            h->is_corner[v] = 1;
        }
    }
    for (int64_t v = 0; v < nn && !h->user_corners; ++v) {
        int sid = h->node_set[v];
        if (h->sets[sid].size() < 3) continue;
        if (set_count[sid] == 1) {
            h->is_corner[v] = 1;
            continue;
        }
        auto &L = nb[eidx[v]];
        std::sort(L.begin(), L.end());
        L.erase(std::unique(L.begin(), L.end()), L.end());
        int same = 0;
        bool sup = false;
        for (int64_t m : L) {
            int ms = h->node_set[m];
            if (ms == sid) same++;
            if (is_superset(ms, sid)) sup = true;
        }
        if (same <= 1 && !sup) h->is_corner[v] = 1;
    }
    h->corners.clear();
    for (int64_t v = 0; v < nn; ++v) {
        if (h->is_corner[v] && h->dirich[v]) h->is_corner[v] = 0;
        if (h->is_corner[v]) h->corners.push_back(v);
    }
    // globs: interface nodes grouped by set (the key sort keeps each set contiguous, ascending node ids)
    h->edge_globs.clear();
    FaceList face_list;
    for (size_t q = 0; q < keys.size();) {
        const int sid = h->node_set[keys[q].node];
        size_t q1 = q;
        std::vector<int64_t> nodes;
        while (q1 < keys.size() && h->node_set[keys[q1].node] == sid) {
            int64_t v = keys[q1++].node;
            if (!h->dirich[v] && !h->is_corner[v]) nodes.push_back(v);
        }
        q = q1;
        const auto &S = h->sets[sid];
        if (nodes.empty()) continue;
        if (S.size() == 2)
            face_list.push_back({{S[0], S[1]}, nodes});
        else
            h->edge_globs.push_back({S, nodes});
    }
    std::sort(face_list.begin(), face_list.end());
    h->n_edges = (int)h->edge_globs.size();
    mark_floating(h);
    h->n_augmented = 0;
    if (!h->user_corners) augment_corners(h, face_list);

    // substructures
    const int ns = h->nsub;
    h->subs.assign(ns, SubData());
    // local nodes of every substructure, ascending (each node appended to the substructures of its set)
    std::vector<std::vector<int64_t>> snodes(ns);
    {
        std::vector<int64_t> cnt(ns, 0);
        for (int64_t v = 0; v < nn; ++v)
            for (int q = 0; q < nsv[v].cnt; ++q) cnt[nsv[v].s[q]]++;
        for (int sb = 0; sb < ns; ++sb) snodes[sb].reserve(cnt[sb]);
        for (int64_t v = 0; v < nn; ++v)
            for (int q = 0; q < nsv[v].cnt; ++q) snodes[nsv[v].s[q]].push_back(v);
    }
    const auto tc_sub = std::chrono::steady_clock::now();
    std::vector<char> is_iface_node(nn, 0);
    for (int64_t v = 0; v < nn; ++v) is_iface_node[v] = h->sets[h->node_set[v]].size() >= 2 && !h->dirich[v];
    for (int s = 0; s < ns; ++s) {
        auto &sd = h->subs[s];
        auto &L = snodes[s];
        sd.nodes = L;
        bool touches_dirichlet = false;
        for (int64_t v : L) {
            if (h->dirich[v]) {
                touches_dirichlet = true;
                continue;
            }
            for (int k = 0; k < c; ++k) (is_iface_node[v] ? sd.gG : sd.gI).push_back(h->node_first[v] + k);
        }
        (void)touches_dirichlet;
        sd.floating = h->sub_floating[s] != 0;
        sd.nI = (int)sd.gI.size();
        sd.nG = (int)sd.gG.size();
        sd.n = sd.nI + sd.nG;
        sd.ld = round_up(std::max(sd.n, 1), 8);
        sd.ldS = round_up(std::max(sd.nG, 1), 8);
    }
    // interface numbering (ascending global dof) and gather maps
    std::vector<int> gidx(h->nfree, -1);
    for (auto &sd : h->subs)
        for (int64_t g : sd.gG) gidx[g] = 0;
    h->iface_gdof.clear();
    for (int64_t g = 0; g < h->nfree; ++g)
        if (gidx[g] == 0) {
            gidx[g] = (int)h->iface_gdof.size();
            h->iface_gdof.push_back(g);
        }
    h->nG = (int)h->iface_gdof.size();
    h->offG.assign(ns, 0);
    int64_t off = 0, offI = 0;
    h->gptr.assign(h->nG + 1, 0);
    for (int s = 0; s < ns; ++s) {
        auto &sd = h->subs[s];
        h->offG[s] = off;
        sd.offI = offI;
        sd.RG.resize(sd.nG);
        for (int k = 0; k < sd.nG; ++k) {
            sd.RG[k] = gidx[sd.gG[k]];
            h->gptr[sd.RG[k] + 1]++;
        }
        off += sd.nG;
        offI += sd.nI;
        sd.cpos.clear();
        sd.rpos.clear();
    }
    h->sumG = off;
    h->sumI = offI;
    // node of each free dof
    std::vector<int64_t> dof_node(h->nfree);
    for (int64_t v = 0; v < nn; ++v)
        if (h->node_first[v] >= 0)
            for (int k = 0; k < c; ++k) dof_node[h->node_first[v] + k] = v;
    for (auto &sd : h->subs) {
        for (int k = 0; k < sd.nG; ++k) (h->is_corner[dof_node[sd.gG[k]]] ? sd.cpos : sd.rpos).push_back(k);
    }
    for (int x = 0; x < h->nG; ++x) h->gptr[x + 1] += h->gptr[x];
    h->gent.assign(h->gptr[h->nG], 0);
    h->gsub.assign(h->gptr[h->nG], 0);
    {
        std::vector<int> fill(h->gptr.begin(), h->gptr.end() - 1);
        for (int s = 0; s < ns; ++s) {
            auto &sd = h->subs[s];
            for (int k = 0; k < sd.nG; ++k) {
                int slot = fill[sd.RG[k]]++;
                h->gent[slot] = h->offG[s] + k;
                h->gsub[slot] = s;
            }
        }
    }
    // corner dofs: global coarse indices 0..n_corner_dofs-1 in global dof order
    std::vector<int64_t> cdofs;
    for (int64_t v : h->corners)
        for (int k = 0; k < c; ++k) cdofs.push_back(h->node_first[v] + k);
    h->n_corner_dofs = (int)cdofs.size();
    std::vector<int> cidx(h->nfree, -1);
    for (int k = 0; k < (int)cdofs.size(); ++k) cidx[cdofs[k]] = k;
    for (auto &sd : h->subs) {
        sd.corner_coarse.clear();
        for (int p : sd.cpos) sd.corner_coarse.push_back(cidx[sd.gG[p]]);
    }
    // Assumption 1: every floating substructure needs corners that fix its rigid modes
    auto rank_corners = [&](const std::vector<int64_t> &cn) {
        // number of independent rigid modes fixed: 1 (scalar) or affine rank test (elasticity)
        if (cn.empty()) return 0;
        if (c == 1) return 1;
        // elasticity: need 3 non-collinear points
        const double *x0 = &h->xyz[cn[0] * 3];
        int best = 1;
        for (size_t a = 1; a < cn.size(); ++a) {
            const double *xa = &h->xyz[cn[a] * 3];
            double d1[3] = {xa[0] - x0[0], xa[1] - x0[1], xa[2] - x0[2]};
            if (d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2] > 0) best = std::max(best, 2);
            for (size_t b = a + 1; b < cn.size(); ++b) {
                const double *xb = &h->xyz[cn[b] * 3];
                double d2[3] = {xb[0] - x0[0], xb[1] - x0[1], xb[2] - x0[2]};
                double cr[3] = {d1[1] * d2[2] - d1[2] * d2[1], d1[2] * d2[0] - d1[0] * d2[2], d1[0] * d2[1] - d1[1] * d2[0]};
                double n1 = std::sqrt(d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2]);
                double n2 = std::sqrt(d2[0] * d2[0] + d2[1] * d2[1] + d2[2] * d2[2]);
                if (std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]) > 1e-8 * n1 * n2) return 3;
            }
        }
        return best;
    };
    for (int s = 0; s < ns; ++s) {
        auto &sd = h->subs[s];
        if (!sd.floating) continue;
        std::vector<int64_t> cn;
        for (size_t k = 0; k < sd.cpos.size(); k += c) cn.push_back(dof_node[sd.gG[sd.cpos[k]]]);
        int need = (c == 1) ? 1 : 3;
        if (rank_corners(cn) < need)
            throw Error{BDDC_EASSUMPTION, "Assumption 1: floating substructure " + std::to_string(s) +
                                              " has too few corners to fix its rigid body modes"};
    }
    const auto tc_faces = std::chrono::steady_clock::now();
    // element positions read the substructure dof lists, which are final now; the face
    // pairs below only read them as well
    if (!h->csr_mode) epos_task.start([h]() { h->epos = element_positions(h); });
    // face pairs: independent of each other, built by a few host threads (each with its own
    // scratch); the failure reported is the first face's in face order, as a serial loop would
    const size_t nfl = face_list.size();
    h->faces.assign(nfl, FacePair());
    std::vector<std::string> face_err(nfl);
    auto build_faces = [&](size_t t0, size_t tstep) {
        std::vector<int> pj(h->nfree, -1);   // position of a dof in sj's interface list
        // per set: the face (index + 1) it was last tested for, and whether it holds both substructures
        std::vector<int> set_stamp(h->sets.size(), 0);
        std::vector<char> set_both(h->sets.size(), 0);
        for (size_t q = t0; q < nfl; q += tstep) {
            const auto &fl = face_list[q];
            const int face_no = (int)q + 1;
            FacePair fp;
            fp.i = fl.first.first;
            fp.j = fl.first.second;
            auto &si = h->subs[fp.i], &sj = h->subs[fp.j];
            for (int k = 0; k < sj.nG; ++k) pj[sj.gG[k]] = k;
            std::vector<int64_t> cn;
            for (int k = 0; k < si.nG; ++k) {
                int64_t g = si.gG[k];
                int64_t v = dof_node[g];
                const int sid = h->node_set[v];
                if (set_stamp[sid] != face_no) {
                    const auto &S = h->sets[sid];
                    set_stamp[sid] = face_no;
                    set_both[sid] = std::binary_search(S.begin(), S.end(), fp.i) && std::binary_search(S.begin(), S.end(), fp.j);
                }
                if (!set_both[sid]) continue;
                if (h->is_corner[v]) {
                    fp.ci_pos.push_back(k);
                    fp.cj_pos.push_back(pj[g]);
                    if (g % c == 0 || c == 1) cn.push_back(v);
                    continue;
                }
                fp.s_g.push_back(g);
                fp.pos_i.push_back(k);
            }
            // s sorted by global dof (si.gG is sorted so s_g is too)
            for (size_t k = 0; k < fp.s_g.size(); ++k) {
                int64_t g = fp.s_g[k];
                fp.pos_j.push_back(pj[g]);
                const auto &S = h->sets[h->node_set[dof_node[g]]];
                if (S.size() == 2) fp.face_idx.push_back((int)k);
            }
            fp.floating = si.floating && sj.floating;
            const int nsd = (int)fp.s_g.size();
            for (int k = 0; k < sj.nG; ++k) pj[sj.gG[k]] = -1;
            if (si.floating || sj.floating) {
                // with one floating member the pair matrix is singular unless the shared corners fix its rigid modes
                int need = (c == 1) ? 1 : 3;
                std::vector<int64_t> cnu;
                for (size_t k = 0; k < fp.ci_pos.size(); k += c) cnu.push_back(dof_node[si.gG[fp.ci_pos[k]]]);
                if (rank_corners(cnu) < need) {
                    face_err[q] = "Assumption 2: corners shared by substructures " + std::to_string(fp.i) + " and " +
                                  std::to_string(fp.j) + " do not fix relative rigid motions";
                    continue;
                }
            }
            if (fp.floating) {
                // null space of S^ on s: rigid modes, identical on both sides; N0 orthonormal with N = [N0; N0]
                int nr = (c == 1) ? 1 : 6;
                std::vector<double> R((size_t)nsd * nr, 0.0);
                for (int k = 0; k < nsd; ++k) {
                    int64_t g = fp.s_g[k];
                    int comp = (int)(g % c);
                    const double *x = &h->xyz[dof_node[g] * 3];
                    if (c == 1) {
                        R[k] = 1.0;
                    } else {
                        R[(size_t)comp * nsd + k] = 1.0;  // translations
                        // rotations omega x x: e_a x x, component comp
                        double rot[3][3] = {{0, -x[2], x[1]}, {x[2], 0, -x[0]}, {-x[1], x[0], 0}};
                        // omega = e_a: (e_a x x)_comp = rot[comp][a]... (e_a x x) = -x x e_a
                        for (int a = 0; a < 3; ++a) R[(size_t)(3 + a) * nsd + k] = -rot[comp][a];
                    }
                }
                // modified Gram-Schmidt, then scale by 1/sqrt(2)
                int kept = 0;
                std::vector<double> Q;
                for (int a = 0; a < nr; ++a) {
                    std::vector<double> v(R.begin() + (size_t)a * nsd, R.begin() + (size_t)(a + 1) * nsd);
                    for (int b = 0; b < kept; ++b) {
                        double d = 0;
                        for (int k = 0; k < nsd; ++k) d += v[k] * Q[(size_t)b * nsd + k];
                        for (int k = 0; k < nsd; ++k) v[k] -= d * Q[(size_t)b * nsd + k];
                    }
                    double nrm = 0;
                    for (double t : v) nrm += t * t;
                    nrm = std::sqrt(nrm);
                    if (nrm < 1e-10) continue;
                    for (double &t : v) t /= nrm;
                    Q.insert(Q.end(), v.begin(), v.end());
                    kept++;
                }
                for (double &t : Q) t /= std::sqrt(2.0);
                fp.N0 = Q;
                fp.nnull = kept;
            }
            h->faces[q] = std::move(fp);
        }
    };
    {
        const unsigned hw = std::thread::hardware_concurrency();
        const size_t nthr = std::max<size_t>(1, std::min<size_t>({8, hw > 0 ? (size_t)hw : 1, (nfl + 15) / 16}));
        std::vector<HostTask> tasks(nthr - 1);
        for (size_t t = 1; t < nthr; ++t) tasks[t - 1].start([&build_faces, t, nthr]() { build_faces(t, nthr); });
        std::exception_ptr err0;
        try {
            build_faces(0, nthr);
        } catch (...) {
            err0 = std::current_exception();
        }
        for (auto &t : tasks) t.rethrow();
        if (err0) std::rethrow_exception(err0);
        for (size_t q = 0; q < nfl; ++q)
            if (!face_err[q].empty()) throw Error{BDDC_EASSUMPTION, face_err[q]};
    }
    const auto tc_color = std::chrono::steady_clock::now();
    colour_task.rethrow();
    epos_task.rethrow();
    if (!h->csr_mode) h->colors = std::move(colors);
    if (getenv("BDDC_DEBUG_TIMING")) {
        auto ms = [](auto x, auto y) { return std::chrono::duration<double, std::milli>(y - x).count(); };
        const auto tc_end = std::chrono::steady_clock::now();
        fprintf(stderr, "classify: sets+globs %.3f subs+maps %.3f faces %.3f colours %.3f ms\n", ms(tc0, tc_sub),
                ms(tc_sub, tc_faces), ms(tc_faces, tc_color), ms(tc_color, tc_end));
    }
}

// positions of each node's first dof in the dense local ordering [interior; interface]
std::vector<int32_t> element_positions(bddc_handle *h) {
    std::vector<int32_t> pos(h->ne * 8, -1);
    std::vector<std::vector<int32_t>> sub_elems(h->nsub);
    for (int64_t e = 0; e < h->ne; ++e) sub_elems[h->esub[e]].push_back((int32_t)e);
    std::vector<int> lp(h->nfree, -1);
    for (int s = 0; s < h->nsub; ++s) {
        auto &sd = h->subs[s];
        for (int k = 0; k < sd.nI; k += h->ncomp) lp[sd.gI[k]] = k;
        for (int k = 0; k < sd.nG; k += h->ncomp) lp[sd.gG[k]] = sd.nI + k;
        for (int32_t e : sub_elems[s])
            for (int a = 0; a < 8; ++a) {
                int64_t v = h->elems[(int64_t)e * 8 + a];
                if (h->node_first[v] >= 0) pos[(int64_t)e * 8 + a] = lp[h->node_first[v]];
            }
        for (int k = 0; k < sd.nI; k += h->ncomp) lp[sd.gI[k]] = -1;
        for (int k = 0; k < sd.nG; k += h->ncomp) lp[sd.gG[k]] = -1;
    }
    return pos;
}

void build_average_globs(bddc_handle *h) {
    h->globs.clear();
    const int c = h->ncomp;
    auto add = [&](const std::vector<int> &subs, const std::vector<int64_t> &nodes) {
        GlobRows g;
        g.subs = subs;
        for (int64_t v : nodes)
            for (int k = 0; k < c; ++k) g.gdofs.push_back(h->node_first[v] + k);
        g.nrows = c;
        g.rows.assign((size_t)c * g.gdofs.size(), 0.0);
        for (int comp = 0; comp < c; ++comp)
            for (size_t k = comp; k < g.gdofs.size(); k += c) g.rows[(size_t)comp * g.gdofs.size() + k] = 1.0;
        h->globs.push_back(g);
    };
    if (h->avg_flags & BDDC_AVG_EDGE)
        for (auto &eg : h->edge_globs) add(eg.first, eg.second);
    if (h->avg_flags & BDDC_AVG_FACE)
        for (auto &fp : h->faces) {
            std::set<int64_t> ns;
            for (int k : fp.face_idx) ns.insert(fp.s_g[k] - fp.s_g[k] % c);
            GlobRows g;
            g.subs = {fp.i, fp.j};
            for (int64_t g0 : ns)
                for (int k = 0; k < c; ++k) g.gdofs.push_back(g0 + k);
            g.nrows = c;
            g.rows.assign((size_t)c * g.gdofs.size(), 0.0);
            for (int comp = 0; comp < c; ++comp)
                for (size_t k = comp; k < g.gdofs.size(); k += c) g.rows[(size_t)comp * g.gdofs.size() + k] = 1.0;
            h->globs.push_back(g);
        }
}

// Lays out the constraint rows of every substructure, numbers the coarse
// dofs and fills the constraint buffers (averages from the host, adaptive
// rows copied on the device from the face row buffers).
void layout_constraints(bddc_handle *h) {
    const int ns = h->nsub;
    int nC = h->n_corner_dofs;
    std::vector<std::vector<std::pair<int, int>>> sub_rows(ns);  // (glob, row)
    for (int gi = 0; gi < (int)h->globs.size(); ++gi) {
        auto &g = h->globs[gi];
        g.coarse0 = nC;
        nC += g.nrows;
        for (int s : g.subs)
            for (int r = 0; r < g.nrows; ++r) sub_rows[s].push_back({gi, r});
    }
    h->nC = nC;
    std::vector<GatherOp> ops;
    std::vector<int> pos(h->nfree, -1);
    for (int s = 0; s < ns; ++s) {
        auto &sd = h->subs[s];
        sd.na = (int)sub_rows[s].size();
        sd.capA = std::max(1, sd.na);
        sd.Cb = h->ar.get_t<double>("Cb_" + std::to_string(s), (size_t)sd.capA * sd.nG);
        std::vector<double> host((size_t)sd.capA * sd.nG, 0.0);
        for (int k = 0; k < sd.nG; ++k) pos[sd.gG[k]] = k;
        sd.row_coarse.clear();
        for (int m = 0; m < sd.na; ++m) {
            auto &g = h->globs[sub_rows[s][m].first];
            int r = sub_rows[s][m].second;
            sd.row_coarse.push_back(g.coarse0 + r);
            if (g.face >= 0 || g.edge >= 0) continue;
            for (size_t k = 0; k < g.gdofs.size(); ++k)
                host[(size_t)pos[g.gdofs[k]] * sd.capA + m] = g.rows[(size_t)r * g.gdofs.size() + k];
        }
        BDDC_CUDA(cudaMemcpyAsync(sd.Cb, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        // adaptive rows: one gather per (sub, face glob): Cb[m0 + l, facepos] = rows[l, f]
        for (int m = 0; m < sd.na;) {
            auto &g = h->globs[sub_rows[s][m].first];
            if (g.face < 0 && g.edge < 0) {
                ++m;
                continue;
            }
            if (g.edge >= 0) {
                // kept edge rows: Cb[m + l, k] = rowsT(l, cmap[k]), ld = the edge's dofs
                const auto &er = h->edge_rows[g.edge];
                std::vector<int> cmap(sd.nG, -1);
                for (size_t t = 0; t < g.gdofs.size(); ++t) {
                    const int k = pos[g.gdofs[t]];
                    BDDC_REQUIRE(k >= 0, BDDC_EINVAL, "internal: an edge dof outside a substructure of the edge");
                    cmap[k] = (int)t;
                }
                int *dcm = h->ar.upload("ecmap_" + std::to_string(s) + "_" + std::to_string(g.edge), cmap, h->stream);
                GatherOp o = gop(er.rowsT, er.ld, sd.Cb, sd.capA, g.nrows, sd.nG);
                o.dst_row_off = m;
                o.cmap = dcm;
                ops.push_back(o);
                m += g.nrows;
                continue;
            }
            auto &fp = h->faces[g.face];
            int nf = (int)fp.face_idx.size();
            // column map over interface positions: face index or -1
            std::vector<int> cmap(sd.nG, -1);
            for (int f = 0; f < nf; ++f) {
                int k = fp.face_idx[f];
                cmap[(s == fp.i) ? fp.pos_i[k] : fp.pos_j[k]] = f;
            }
            int *dcm = h->ar.upload("cmap_" + std::to_string(s) + "_" + std::to_string(g.face), cmap, h->stream);
            // face rows stored column-major (l, f) with ld = nrows: Cb[m + l, k] = rows(l, cmap[k])
            GatherOp o = gop(h->face_rows_dev[g.face], g.nrows, sd.Cb, sd.capA, g.nrows, sd.nG);
            o.dst_row_off = m;
            o.cmap = dcm;
            ops.push_back(o);
            m += g.nrows;
        }
        for (int k = 0; k < sd.nG; ++k) pos[sd.gG[k]] = -1;
    }
    run_gathers(h, ops, "cons");
}

// Builds the local saddle operators (P~_i, Phi~_i, S_C,i), the coarse matrix
// and its inverse for the current constraints (Remark 5.1: all constraints
// primal).  Two partial Cholesky passes on augmented matrices per substructure:
//   M1 = [S_rr . . .; I 0 . .; C_r 0 0 .; S_cr 0 0 0], stop n_r:
//        trailing = -[[S_rr^-1, Z_a, Z_c]; [Z_a^T, G, H]; [Z_c^T, H^T, J]]
//   M2 = [G . . .; Z_a K . .; H^T Z_c^T J .; I 0 0 0], stop n_a:
//        trailing = [[P_rr, -Phi_rc, -Phi_ra]; [., J - H^T G^-1 H, -H^T G^-1]; [., ., -G^-1]]
// with K = S_rr^-1, Z = K [S_rc, C_r^T], G = C_r K C_r^T, H = C_r K S_rc, J = S_cr K S_rc.
// Thrown by the mixed local saddle factorization when FP32 is not accurate enough.
struct Fp32Breakdown {};

void coarse_setup(bddc_handle *h, bool allow_fp32) {
    const int ns = h->nsub;
    const bool mixed = h->opt.precision == BDDC_MIXED_FP32_SADDLE && allow_fp32;
    layout_constraints(h);
    // mixed: M1 in FP32 with the symmetric equilibration d = diag(S)^-1/2 of the remaining dofs
    double *eqS = nullptr, *dr = nullptr, *s2 = nullptr;
    std::vector<int64_t> off_r(ns, 0), off_s2(ns, 0);
    if (mixed) {
        std::vector<MixedSub> ms(ns);
        std::vector<int64_t> idx_r, idx_s2;
        eqS = h->ar.get_t<double>("eqS", h->sumG + 1);
        for (int s = 0; s < ns; ++s) {
            auto &sd = h->subs[s];
            ms[s] = MixedSub{sd.S, sd.nG, 0, sd.ldS, eqS + h->offG[s], nullptr, nullptr, nullptr, 0};
            off_r[s] = (int64_t)idx_r.size();
            for (int p : sd.rpos) idx_r.push_back(h->offG[s] + p);
            off_s2[s] = (int64_t)idx_s2.size();
            for (int k = 0; k < sd.na; ++k) idx_s2.push_back(h->sumG);  // the constant 1
            for (int p : sd.rpos) idx_s2.push_back(h->offG[s] + p);
            for (size_t k = 0; k < sd.cpos.size(); ++k) idx_s2.push_back(h->sumG);
        }
        auto *dms = h->ar.upload("ms_S", ms, h->stream);
        launch_equilibrate(dms, ns, h->stream);
        check_launch(h);
        const double one = 1.0;
        BDDC_CUDA(cudaMemcpyAsync(eqS + h->sumG, &one, sizeof(double), cudaMemcpyHostToDevice, h->stream));
        dr = h->ar.get_t<double>("dr", idx_r.size() + 1);
        s2 = h->ar.get_t<double>("s2", idx_s2.size() + 1);
        auto *di = h->ar.upload("idx_r", idx_r, h->stream);
        auto *d2i = h->ar.upload("idx_s2", idx_s2, h->stream);
        launch_gatherv(dr, di, eqS, (int64_t)idx_r.size(), h->stream);
        check_launch(h);
        launch_gatherv(s2, d2i, eqS, (int64_t)idx_s2.size(), h->stream);
        check_launch(h);
        BDDC_CUDA(cudaStreamSynchronize(h->stream));  // 'one' lives on the host stack
    }
    std::vector<PcholDesc<double>> d1, d2;
    std::vector<PcholDesc<float>> d1f;
    std::vector<GatherOp> g1, g2, g3;
    std::vector<DiagOp> id1, id2;
    std::vector<double *> M1(ns), M2(ns), SCi(ns);
    std::vector<int> N1(ns), N2(ns), ld1(ns), ld2(ns);
    // map arrays uploaded per sub
    ZeroList zl;
    for (int s = 0; s < ns; ++s) {
        auto &sd = h->subs[s];
        const int nr = (int)sd.rpos.size(), nc = (int)sd.cpos.size(), na = sd.na;
        N1[s] = 2 * nr + na + nc;
        ld1[s] = round_up(std::max(N1[s], 1), 8);
        N2[s] = na + nr + nc + na;
        ld2[s] = round_up(std::max(N2[s], 1), 8);
        M1[s] = h->ar.get_t<double>("M1_" + std::to_string(s), (size_t)ld1[s] * N1[s]);
        M2[s] = h->ar.get_t<double>("M2_" + std::to_string(s), (size_t)ld2[s] * std::max(N2[s], 1));
        // in mixed mode M1 holds floats (ld1 is a multiple of 8, so half the doubles cover it)
        zl.add(M1[s], mixed ? (size_t)ld1[s] * N1[s] / 2 : (size_t)ld1[s] * N1[s]);
        zl.add(M2[s], (size_t)ld2[s] * std::max(N2[s], 1));
        int *drpos = h->ar.upload("rpos_" + std::to_string(s), sd.rpos, h->stream);
        int *dcpos = h->ar.upload("cpos_" + std::to_string(s), sd.cpos, h->stream);
        // M1 blocks (mixed: FP32, columns of the remaining dofs scaled by d)
        const double *dsc = mixed ? dr + off_r[s] : nullptr;
        GatherOp o = gop(sd.S, sd.ldS, M1[s], ld1[s], nr, nr);
        o.rmap = drpos;
        o.cmap = drpos;
        o.dst_lower = 1;
        o.rscale = dsc;
        o.cscale = dsc;
        o.dst_f32 = mixed;
        g1.push_back(o);
        if (na > 0) {
            o = gop(sd.Cb, sd.capA, M1[s], ld1[s], na, nr);
            o.cmap = drpos;
            o.dst_row_off = 2 * nr;
            o.cscale = dsc;
            o.dst_f32 = mixed;
            g1.push_back(o);
        }
        if (nc > 0) {
            o = gop(sd.S, sd.ldS, M1[s], ld1[s], nc, nr);
            o.rmap = dcpos;
            o.cmap = drpos;
            o.dst_row_off = 2 * nr + na;
            o.cscale = dsc;
            o.dst_f32 = mixed;
            g1.push_back(o);
        }
        DiagOp dop{M1[s], ld1[s], nr, 0, nr, 1.0, mixed ? 1 : 0, 0};
        id1.push_back(dop);
        if (mixed)
            d1f.push_back(PcholDesc<float>{reinterpret_cast<float *>(M1[s]), N1[s], ld1[s], nr, 0, nullptr, 0, nr});
        else
            d1.push_back(PcholDesc<double>{M1[s], N1[s], ld1[s], nr, 0, nullptr, 0, nr});
    }
    zero_all(h, zl, "M12");
    run_gathers(h, g1, "M1");
    run_diag(h, id1, "M1");
    if (mixed) {
        // the equilibrated S_rr has a unit diagonal: a pivot below 1e-5 means a condition
        // number FP32 cannot carry; the coarse operators are then rebuilt in FP64
        static const unsigned inf_bits = 0x7f800000u;
        BDDC_CUDA(cudaMemcpyAsync(&h->dst->minpiv, &inf_bits, sizeof(unsigned), cudaMemcpyHostToDevice, h->stream));
        run_pchol<float>(h, d1f, "M1f");
        DevStatus hs;
        BDDC_CUDA(cudaMemcpyAsync(&hs, h->dst, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->stream));
        BDDC_CUDA(cudaStreamSynchronize(h->stream));
        float minpiv;
        memcpy(&minpiv, &hs.minpiv, sizeof(float));
        h->m1_min_pivot = minpiv;
        if (hs.code == BDDC_DEV_ERR_NOTSPD || !(minpiv >= 1e-5f)) throw Fp32Breakdown{};
    } else {
        run_pchol_fp64class(h, d1, "M1");
    }
    for (int s = 0; s < ns; ++s) {
        auto &sd = h->subs[s];
        const int nr = (int)sd.rpos.size(), nc = (int)sd.cpos.size(), na = sd.na;
        // M2[0:K, 0:K] = -M1(perm, perm), perm = (a, id, c) in M1 coordinates
        std::vector<int> perm;
        for (int k = 0; k < na; ++k) perm.push_back(2 * nr + k);
        for (int k = 0; k < nr; ++k) perm.push_back(nr + k);
        for (int k = 0; k < nc; ++k) perm.push_back(2 * nr + na + k);
        int K = (int)perm.size();
        int *dperm = h->ar.upload("perm2_" + std::to_string(s), perm, h->stream);
        if (K > 0) {
            GatherOp o = gop(M1[s], ld1[s], M2[s], ld2[s], K, K);
            o.rmap = dperm;
            o.cmap = dperm;
            o.src_sym = 1;
            o.dst_lower = 1;
            o.scale = -1.0;
            if (mixed) {  // undo the equilibration on the (id) block: K = D K_s D, Z = D (K_s D C^T) ...
                o.src_f32 = 1;
                o.rscale = s2 + off_s2[s];
                o.cscale = s2 + off_s2[s];
            }
            g2.push_back(o);
        }
        if (na > 0) id2.push_back(DiagOp{M2[s], ld2[s], K, 0, na, 1.0});
        d2.push_back(PcholDesc<double>{M2[s], N2[s], ld2[s], na, 0});
    }
    run_gathers(h, g2, "M2");
    run_diag(h, id2, "M2");
    run_pchol_fp64class(h, d2, "M2");
    if (mixed) {  // G = C_r S_rr^-1 C_r^T from the FP32 stage must factor
        DevStatus hs;
        BDDC_CUDA(cudaMemcpyAsync(&hs, h->dst, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->stream));
        BDDC_CUDA(cudaStreamSynchronize(h->stream));
        if (hs.code == BDDC_DEV_ERR_NOTSPD) throw Fp32Breakdown{};
    }
    // extraction of P~, Phi~, S_C,i
    std::vector<CoarseAsmDesc> cad;
    std::vector<int> Rc_all;
    std::vector<int64_t> offc(ns);
    int64_t oc = 0;
    for (int s = 0; s < ns; ++s) {
        auto &sd = h->subs[s];
        offc[s] = oc;
        oc += (int)sd.cpos.size() + sd.na;
    }
    for (int s = 0; s < ns; ++s) {
        auto &sd = h->subs[s];
        const int nr = (int)sd.rpos.size(), nc = (int)sd.cpos.size(), na = sd.na, nG = sd.nG;
        const int nci = nc + na;
        double *dl = h->ar.get_t<double>("delta", h->sumG) + h->offG[s];
        // row map over interface positions into T2 (offset na): r_k -> na + k, corners -> -1
        std::vector<int> rm(nG, -1);
        for (int k = 0; k < nr; ++k) rm[sd.rpos[k]] = na + k;
        int *drm = h->ar.upload("rmP_" + std::to_string(s), rm, h->stream);
        GatherOp o = gop(M2[s], ld2[s], sd.P, sd.ldS, nG, nG);
        o.rmap = drm;
        o.cmap = drm;
        o.src_sym = 1;
        o.rscale = dl;
        o.cscale = dl;
        g3.push_back(o);
        // Phi~: columns corners then averages
        std::vector<int> cm(nci);
        for (int m = 0; m < nc; ++m) cm[m] = na + nr + m;
        for (int m = 0; m < na; ++m) cm[nc + m] = na + nr + nc + m;
        int *dcm = h->ar.upload("cmPhi_" + std::to_string(s), cm, h->stream);
        if (nci > 0) {
            o = gop(M2[s], ld2[s], sd.Phi, sd.ldS, nG, nci);
            o.rmap = drm;
            o.cmap = dcm;
            o.src_sym = 1;
            o.scale = -1.0;
            o.rscale = dl;
            g3.push_back(o);
        }
        // identity on the corner rows (accumulate): Phi[cpos[m], m] += delta
        std::vector<int> cr(nG, -1);
        for (int m = 0; m < nc; ++m) cr[sd.cpos[m]] = m;
        int *dcr = h->ar.upload("crPhi_" + std::to_string(s), cr, h->stream);
        // S_C,i = -T2(cm, cm) + [S_cc 0; 0 0]
        double *sci = h->ar.get_t<double>("SCi_" + std::to_string(s), (size_t)std::max(nci, 1) * std::max(nci, 1));
        SCi[s] = sci;
        if (nci > 0) {
            o = gop(M2[s], ld2[s], sci, nci, nci, nci);
            o.rmap = dcm;
            o.cmap = dcm;
            o.src_sym = 1;
            o.scale = -1.0;
            g3.push_back(o);
        }
        std::vector<int> Rc;
        for (int m = 0; m < nc; ++m) Rc.push_back(sd.corner_coarse[m]);
        for (int m = 0; m < na; ++m) Rc.push_back(sd.row_coarse[m]);
        Rc_all.insert(Rc_all.end(), Rc.begin(), Rc.end());
        (void)dcr;
    }
    run_gathers(h, g3, "ext");
    std::vector<GatherOp> g4;
    for (int s = 0; s < ns; ++s) {
        auto &sd = h->subs[s];
        const int nc = (int)sd.cpos.size(), nci = nc + sd.na, nG = sd.nG;
        double *dl = h->ar.get_t<double>("delta", h->sumG) + h->offG[s];
        if (nc > 0) {
            int *dcr = h->ar.get_t<int>("crPhi_" + std::to_string(s), nG);
            GatherOp o = gop(nullptr, 0, sd.Phi, sd.ldS, nG, nc);
            o.rmap = dcr;
            o.rscale = dl;
            o.accumulate = 1;
            g4.push_back(o);
            int *dcpos = h->ar.get_t<int>("cpos_" + std::to_string(s), nc);
            o = gop(sd.S, sd.ldS, SCi[s], nci, nc, nc);
            o.rmap = dcpos;
            o.cmap = dcpos;
            o.accumulate = 1;
            g4.push_back(o);
        }
    }
    run_gathers(h, g4, "ext2");
    int *dRc = h->ar.upload("Rc", Rc_all, h->stream);
    for (int s = 0; s < ns; ++s) {
        auto &sd = h->subs[s];
        int nci = (int)sd.cpos.size() + sd.na;
        cad.push_back(CoarseAsmDesc{SCi[s], dRc + offc[s], nci, std::max(nci, 1)});
    }
    const int nC = h->nC;
    BDDC_REQUIRE(nC > 0, BDDC_EASSUMPTION, "no coarse degrees of freedom");
    BDDC_REQUIRE(nC <= 12000, BDDC_EINVAL, "coarse problem larger than 12000 dofs");
    double *SC = h->ar.get_t<double>("SC", (size_t)nC * nC);
    int ldm = round_up(2 * nC, 8);
    double *MC = h->ar.get_t<double>("MC", (size_t)ldm * 2 * nC);
    {
        ZeroList zc;
        zc.add(SC, (size_t)nC * nC);
        zc.add(MC, (size_t)ldm * 2 * nC);
        zero_all(h, zc, "SC");
    }
    auto *dcad = h->ar.upload("cad", cad, h->stream);
    launch_coarse_assemble(dcad, ns, SC, nC, h->stream);
    check_launch(h);
    // inverse by partial Cholesky of [[S_C, .]; [I, 0]], in the FP64-class arithmetic of the
    // precision mode (double-float with tensor-core updates in the mixed modes)
    std::vector<GatherOp> g5{gop(SC, nC, MC, ldm, nC, nC)};
    g5[0].dst_lower = 1;
    run_gathers(h, g5, "MC");
    run_diag(h, {DiagOp{MC, ldm, nC, 0, nC, 1.0}}, "MC");
    run_pchol_fp64class(h, {PcholDesc<double>{MC, 2 * nC, ldm, nC, 0, nullptr, 0, nC}}, "MC");
    double *SCinv = h->ar.get_t<double>("SCinv", (size_t)nC * nC);
    GatherOp o = gop(MC, ldm, SCinv, nC, nC, nC);
    o.src_row_off = nC;
    o.src_col_off = nC;
    o.src_sym = 1;
    o.scale = -1.0;
    run_gathers(h, {o}, "SCinv");
    fail_check(h, "coarse setup");
    // interface operator descriptors
    std::vector<int> nci_v(ns);
    std::vector<int2> cdot;
    for (int s = 0; s < ns; ++s) {
        nci_v[s] = (int)h->subs[s].cpos.size() + h->subs[s].na;
        for (int m = 0; m < nci_v[s]; m += 16) cdot.push_back(make_int2(s, m));
    }
    h->ops.nci = h->ar.upload("nci", nci_v, h->stream);
    h->ops.offc = h->ar.upload("offc", offc, h->stream);
    h->ops.Rc = dRc;
    h->ops.SCinv = SCinv;
    h->ops.nC = nC;
    // coarse gather map
    std::vector<std::vector<int64_t>> cl(nC);
    for (int s = 0; s < ns; ++s)
        for (int m = 0; m < nci_v[s]; ++m) cl[Rc_all[offc[s] + m]].push_back(offc[s] + m);
    std::vector<int> cptr(nC + 1, 0);
    std::vector<int64_t> cent;
    for (int k = 0; k < nC; ++k) {
        cent.insert(cent.end(), cl[k].begin(), cl[k].end());
        cptr[k + 1] = (int)cent.size();
    }
    h->ops.cptr = h->ar.upload("cptr", cptr, h->stream);
    h->ops.cent = h->ar.upload("cent", cent, h->stream);
    h->ops.cdot = h->ar.upload("cdot", cdot, h->stream);
    h->ops.ncdot = (int)cdot.size();
    {   // assembly records of the interface entries
        std::vector<ZEntry> ze(h->gent.size());
        for (size_t e = 0; e < h->gent.size(); ++e) {
            const int s = h->gsub[e];
            const auto &sd = h->subs[s];
            const int k = (int)(h->gent[e] - h->offG[s]);
            ze[e] = ZEntry{h->gent[e], sd.Phi + k, dRc + offc[s], sd.ldS, nci_v[s]};
        }
        h->ops.zent = h->ar.upload("zent", ze, h->stream);
    }
    h->pb.cl = h->ar.get_t<double>("cl", std::max<int64_t>(oc, 1));
    h->pb.uc = h->ar.get_t<double>("uc", nC);
}

void alloc_solver_buffers(bddc_handle *h) {
    const int ns = h->nsub;
    std::vector<double *> S(ns), P(ns), Phi(ns);
    for (int s = 0; s < ns; ++s) {
        auto &sd = h->subs[s];
        sd.A = h->ar.get_t<double>("A_" + std::to_string(s), (size_t)sd.ld * std::max(sd.n, 1));
        sd.S = h->ar.get_t<double>("S_" + std::to_string(s), (size_t)sd.ldS * std::max(sd.nG, 1));
        sd.P = h->ar.get_t<double>("P_" + std::to_string(s), (size_t)sd.ldS * std::max(sd.nG, 1));
        S[s] = sd.S;
        P[s] = sd.P;
    }
    h->ops.nsub = ns;
    h->ops.nG = h->nG;
    h->ops.maxGi = 0;
    for (auto &sd : h->subs) h->ops.maxGi = std::max(h->ops.maxGi, sd.nG);
    std::vector<int> nGi(ns), ldS(ns), RG;
    std::vector<int2> rb;
    for (int s = 0; s < ns; ++s) {
        nGi[s] = h->subs[s].nG;
        ldS[s] = h->subs[s].ldS;
        RG.insert(RG.end(), h->subs[s].RG.begin(), h->subs[s].RG.end());
        for (int r = 0; r < nGi[s]; r += 64) rb.push_back(make_int2(s, r));
    }
    {   // S_i and P~_i together larger than about 3/4 of L2 (126 MB): stream them
        size_t bytes = 0;
        for (int s = 0; s < ns; ++s) bytes += 2 * sizeof(double) * (size_t)ldS[s] * nGi[s];
        h->ops.stream_mats = bytes > ((size_t)96 << 20) ? 1 : 0;
    }
    h->ops.nGi = h->ar.upload("nGi", nGi, h->stream);
    h->ops.ldS = h->ar.upload("ldS", ldS, h->stream);
    h->ops.off = h->ar.upload("offG", h->offG, h->stream);
    h->ops.RG = h->ar.upload("RG", RG, h->stream);
    h->ops.S = h->ar.upload("Sptr", S, h->stream);
    h->ops.P = h->ar.upload("Pptr", P, h->stream);
    h->ops.gptr = h->ar.upload("gptr", h->gptr, h->stream);
    h->ops.gent = h->ar.upload("gent", h->gent, h->stream);
    h->ops.gsub = h->ar.upload("gsub", h->gsub, h->stream);
    {   // The PCG kernel runs one block per SM; one bin of row blocks per SM.  An item
        // costs about its substructure's column count (the warps' multiply-adds issue per
        // column whatever the rows left in a ragged last block); binned by cost, the
        // blocks' shares between grid barriers differ by ~2%, where handing the items out
        // in turn left ~10%.  A bin keeps the (substructure, row) order, so a block stages
        // each v_i once per bin.
        int dev = 0, nsm = 0;
        BDDC_CUDA(cudaGetDevice(&dev));
        BDDC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        std::vector<int2> rbs;
        std::vector<int> bp;
        bin_by_cost(rb, [&](const int2 &w) { return (int64_t)nGi[w.x]; }, std::max(nsm, 1), rbs, bp);
        h->ops.rowblk = h->ar.upload("rowblk", rbs, h->stream);
        h->ops.nrowblk = (int)rbs.size();
        h->ops.binptr = h->ar.upload("binptr", bp, h->stream);
        h->ops.nbins = std::max(nsm, 1);
    }
    const int nG = std::max(h->nG, 1);
    h->pb.x = h->ar.get_t<double>("x", nG);
    h->pb.r = h->ar.get_t<double>("r", nG);
    h->pb.z = h->ar.get_t<double>("z", nG);
    h->pb.p0 = h->ar.get_t<double>("p0", nG);
    h->pb.p1 = h->ar.get_t<double>("p1", nG);
    h->pb.q = h->ar.get_t<double>("q", nG);
    h->pb.zl = h->ar.get_t<double>("zl", std::max<int64_t>(h->sumG, 1));
    h->pb.yl = h->ar.get_t<double>("yl", std::max<int64_t>(h->sumG, 1));
    h->pb.partial = h->ar.get_t<double>("partial", 4096);
    int maxit = std::max(h->opt.maxit, 1);
    h->pb.alpha = h->ar.get_t<double>("alpha", maxit);
    h->pb.beta = h->ar.get_t<double>("beta", maxit);
    h->pb.iters = h->ar.get_t<int>("iters", 4);
    h->pb.converged = h->pb.iters + 1;
    h->pb.relres = h->ar.get_t<double>("relres", 1);
}

void set_phi_pointers(bddc_handle *h) {
    const int ns = h->nsub;
    std::vector<double *> Phi(ns);
    for (int s = 0; s < ns; ++s) {
        auto &sd = h->subs[s];
        int nci = (int)sd.cpos.size() + sd.na;
        sd.Phi = h->ar.get_t<double>("Phi_" + std::to_string(s), (size_t)sd.ldS * std::max(nci, 1));
        Phi[s] = sd.Phi;
    }
    h->ops.Phi = h->ar.upload("Phiptr", Phi, h->stream);
}

// ---- mixed precision: FP32 factorization, FP64 refinement ---------------------
constexpr int kEllPerComp = 32;  // ELL width per component (27-point stencil + slack)

struct RefineJob {  // A_II X = B for one substructure, X starts at zero
    int s;
    const double *B;
    int ldb;
    double *X;
    int ldx;
    double *R;
    int ldr;
    int ncol;
};

void run_ell(bddc_handle *h, const std::vector<EllProduct> &ps, const std::string &tag) {
    if (ps.empty()) return;
    const int update = ps[0].update ? 1 : 0;
    std::vector<int4> items;
    for (int k = 0; k < (int)ps.size(); ++k) {
        BDDC_REQUIRE((ps[k].update != 0) == (update != 0) && (!update || ps[k].r0 == 0), BDDC_EINVAL,
                     "internal: mixed ELL product kinds");
        for (int rb = 0; rb < (ps[k].m + 255) / 256; ++rb)
            for (int c0 = 0; c0 < ps[k].ncol; c0 += 8) items.push_back(make_int4(k, rb, c0, 0));
    }
    auto *dp = h->ar.upload("ell_p_" + tag, ps, h->stream);
    auto *di = h->ar.upload("ell_i_" + tag, items, h->stream);
    launch_ell_product(dp, di, (int)items.size(), update, h->stream);
    check_launch(h);
}

EllProduct ell_of(bddc_handle *h, int s) {
    auto &sd = h->subs[s];
    const std::string t = std::to_string(s);
    const int W = kEllPerComp * h->ncomp;
    EllProduct p;
    memset(&p, 0, sizeof(p));
    p.ell_cnt = h->ar.get_t<int>("ellc_" + t, sd.n);
    p.ell_col = h->ar.get_t<int>("ellj_" + t, (size_t)sd.n * W);
    p.ell_val = h->ar.get_t<double>("ellv_" + t, (size_t)sd.n * W);
    p.ell_w = W;
    p.ell_n = sd.n;
    p.ell_valf = h->ar.get_t<double>("ellvf_" + t, (size_t)sd.n * W);
    return p;
}

// Refinement for A_II X = B from X = 0: the first correction is X = D K_s D B, then
// R = B - A_II X (FP64) and X += D K_s D R.  With check, stops at the first residual
// whose relative norm is below tol for every job (R then holds that residual);
// without, stops after exactly `corrections` corrections.  Returns the corrections made.
//
// Jobs with several columns (the interior elimination, X = A_II^-1 A_IG) use the
// tensor cores for the correction dX = D K_s D R (FP32 copy of R in, FP32 dX out).
// The first residual R = B - A_II X is formed in FP64; the later ones are updated,
// R <- R - A_II dX, with the product in double-float: its error is relative to the
// small correction, so the updated R tracks B - A_II X to FP64 accuracy while the
// FP64 pipe (~2 multiply-adds per clock and SM on this GPU) only adds dX into X.
// Single-column jobs (right-hand sides) form every residual in FP64.
int refine(bddc_handle *h, const std::vector<RefineJob> &jobs, int corrections, int max_corr, double tol, bool check,
           const std::string &tag) {
    if (jobs.empty()) return 0;
    const bool multi = jobs[0].ncol > 1;
    for (const auto &j : jobs) BDDC_REQUIRE((j.ncol > 1) == multi, BDDC_EINVAL, "refine: mixed job kinds");
    std::vector<EllProduct> ps, pu;
    std::vector<MixedUpdate> us, us0;
    std::vector<TcGemm> tg;
    std::vector<GatherOp> gB, gX;   // float(B) into the FP32 residual copy; X += dX after the first correction
    std::vector<int2> vitems;
    int max_nI = 0;
    ZeroList zx;
    for (int k = 0; k < (int)jobs.size(); ++k) {
        const auto &j = jobs[k];
        auto &sd = h->subs[j.s];
        const std::string t = std::to_string(j.s);
        EllProduct p = ell_of(h, j.s);
        p.r0 = 0;
        p.m = sd.nI;
        p.ncol = j.ncol;
        p.X = j.X;
        p.ldx = j.ldx;
        p.B = j.B;
        p.ldb = j.ldb;
        p.out = j.R;
        p.ldo = j.ldr;
        float *Rf = multi ? h->ar.get_t<float>("Rf_" + tag + t, (size_t)j.ldr * j.ncol) : nullptr;
        p.outf = Rf;
        ps.push_back(p);
        const int ldk = round_up(std::max(sd.nI, 1), 8);
        const float *K = reinterpret_cast<const float *>(h->ar.get("Kinv_" + t, (size_t)ldk * sd.nI * 4 + 16));
        const double *eq = h->ar.get_t<double>("eq_" + t, sd.n);
        const float *eqf = h->ar.get_t<float>("eqf_" + t, sd.n);
        if (!multi) {
            us.push_back(MixedUpdate{K, ldk, eq, j.R, j.ldr, j.X, j.ldx, sd.nI, j.ncol});
            us0.push_back(MixedUpdate{K, ldk, eq, j.B, j.ldb, j.X, j.ldx, sd.nI, j.ncol});
            for (int a = 0; a < (sd.nI + 31) / 32; ++a) vitems.push_back(make_int2(k, a));
            max_nI = std::max(max_nI, sd.nI);
        } else {
            // dX[r, c] = d[r] sum_k K_s[r, k] d[k] R[k, c]: rows of the symmetric K_s are its columns
            float *dX = h->ar.get_t<float>("dX_" + tag + t, (size_t)j.ldx * j.ncol);
            TcGemm g{K, Rf, dX, eq, eqf, ldk, j.ldr, j.ldx, sd.nI, j.ncol, sd.nI, 0, 0, 1.0};
            g.c_f32 = 1;
            g.store = 1;
            tg.push_back(g);
            GatherOp o = gop(j.B, j.ldb, reinterpret_cast<double *>(Rf), j.ldr, sd.nI, j.ncol);
            o.dst_f32 = 1;
            gB.push_back(o);
            o = gop(reinterpret_cast<const double *>(dX), j.ldx, j.X, j.ldx, sd.nI, j.ncol);
            o.src_f32 = 1;
            gX.push_back(o);   // X = dX (X starts at zero)
            EllProduct q = p;
            q.B = j.R;         // R <- R - A dX in place
            q.ldb = j.ldr;
            q.update = 1;
            q.dXf = dX;
            q.Xu = j.X;
            pu.push_back(q);
        }
        zx.add(j.X, (size_t)j.ldx * j.ncol);
    }
    zero_all(h, zx, "X_" + tag);
    auto *dus = h->ar.upload("mu_" + tag, us, h->stream);
    auto *dus0 = h->ar.upload("mu0_" + tag, us0, h->stream);
    auto *dvi = h->ar.upload("mvi_" + tag, vitems, h->stream);
    const std::vector<int4> titems = tc_items(tg);
    auto *dtg = h->ar.upload("mtg_" + tag, tg, h->stream);
    auto *dti = h->ar.upload("mti_" + tag, titems, h->stream);
    run_gathers(h, gB, "Bf_" + tag);
    auto correction = [&](const MixedUpdate *d) {
        if (multi) {
            launch_tc_gemm(dtg, dti, (int)titems.size(), h->dst, h->opt.timeout_s, h->stream);
        } else {
            BDDC_CUDA(launch_mixed_update_vec(d, dvi, (int)vitems.size(), max_nI, h->stream));
        }
        check_launch(h);
    };
    auto *dps = h->ar.upload("mps_" + tag, ps, h->stream);
    double *norms = h->ar.get_t<double>("rnorm_" + tag, 2 * jobs.size());
    std::vector<double> hn(2 * jobs.size());
    std::vector<int> col_off(jobs.size() + 1, 0);
    for (size_t k = 0; k < jobs.size(); ++k) col_off[k + 1] = col_off[k] + jobs[k].ncol;
    int *dcol_off = h->ar.upload("rn_off_" + tag, col_off, h->stream);
    double *colsums = h->ar.get_t<double>("rn_cols_" + tag, 2 * (size_t)std::max(col_off.back(), 1));
    correction(dus0);
    if (multi) run_gathers(h, gX, "dX0_" + tag);
    int done = 1;
    bool first_check = true;
    int max_ncol = 0;
    for (const auto &j : jobs) max_ncol = std::max(max_ncol, j.ncol);
    for (;;) {
        if (!check && done >= corrections) break;
        if (multi && done > 1)
            run_ell(h, pu, tag + "u");   // R -= A dX, X += dX
        else
            run_ell(h, ps, tag);         // R = B - A X (FP64)
        if (check) {
            launch_residual_norms(dps, (int)ps.size(), max_ncol, colsums, dcol_off, norms, first_check ? 1 : 0,
                                  h->stream);
            first_check = false;
            check_launch(h);
            BDDC_CUDA(cudaMemcpyAsync(hn.data(), norms, hn.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
            BDDC_CUDA(cudaStreamSynchronize(h->stream));
            double worst = 0.0;
            for (size_t k = 0; k < jobs.size(); ++k)
                worst = std::max(worst, std::sqrt(hn[2 * k] / std::max(hn[2 * k + 1], 1e-300)));
            h->mixed_relres = worst;
            if (worst <= tol && done >= corrections) break;
            BDDC_REQUIRE(done < max_corr, BDDC_ENOCONV,
                         "mixed-precision refinement of the interior solves did not converge (relative residual " +
                             std::to_string(worst) + "); use BDDC_FP64");
        }
        correction(dus);
        ++done;
    }
    if (multi && done > 1 && !check) run_ell(h, pu, tag + "u");   // fold the last correction into X
    return done;
}

// Interior elimination in mixed precision (see mixed.cu): FP32 explicit inverse of the
// equilibrated A_II, FP64-refined X = A_II^-1 A_IG, S_i = A_GG - A_GI X in FP64.
void interior_mixed(bddc_handle *h) {
    const int ns = h->nsub, W = kEllPerComp * h->ncomp;
    std::vector<MixedSub> ms(ns);
    std::vector<int2> eitems;
    ZeroList zl;
    std::vector<GatherOp> gF, gK;
    std::vector<DiagOp> dI;
    std::vector<PcholDesc<float>> pd;
    std::vector<RefineJob> jobs;
    for (int s = 0; s < ns; ++s) {
        auto &sd = h->subs[s];
        const int n = sd.n, nI = sd.nI, nG = sd.nG;
        const std::string t = std::to_string(s);
        double *eq = h->ar.get_t<double>("eq_" + t, n);
        float *eqf = h->ar.get_t<float>("eqf_" + t, n);
        EllProduct e = ell_of(h, s);
        ms[s] = MixedSub{sd.A, n, nI, sd.ld, eq, const_cast<int *>(e.ell_cnt), const_cast<int *>(e.ell_col),
                         const_cast<double *>(e.ell_val), W, eqf, const_cast<double *>(e.ell_valf)};
        for (int r = 0; r < n; ++r) eitems.push_back(make_int2(s, r));
        if (nI == 0) continue;
        const int ldF = round_up(2 * nI, 8);
        double *F = static_cast<double *>(h->ar.get("F_" + t, (size_t)ldF * 2 * nI * sizeof(float) + 16));
        zl.add(F, (size_t)ldF * nI);
        GatherOp o = gop(sd.A, sd.ld, F, ldF, nI, nI);
        o.dst_lower = 1;
        o.rscale = eq;
        o.cscale = eq;
        o.dst_f32 = 1;
        gF.push_back(o);
        dI.push_back(DiagOp{F, ldF, nI, 0, nI, 1.0, 1, 0});
        pd.push_back(PcholDesc<float>{reinterpret_cast<float *>(F), 2 * nI, ldF, nI, 0});
        const int ldk = round_up(nI, 8);
        double *K = static_cast<double *>(h->ar.get("Kinv_" + t, (size_t)ldk * nI * sizeof(float) + 16));
        GatherOp k = gop(F, ldF, K, ldk, nI, nI);
        k.src_row_off = nI;
        k.src_col_off = nI;
        k.src_sym = 1;
        k.src_f32 = 1;
        k.dst_f32 = 1;
        k.scale = -1.0;
        gK.push_back(k);
        const int ldx = round_up(nI, 8);
        double *X = h->ar.get_t<double>("X_" + t, (size_t)ldx * std::max(nG, 1));
        double *R = h->ar.get_t<double>("R_" + t, (size_t)ldx * std::max(nG, 1));
        jobs.push_back(RefineJob{s, sd.A + (size_t)nI * sd.ld, sd.ld, X, ldx, R, ldx, nG});
    }
    auto *dms = h->ar.upload("ms_A", ms, h->stream);
    launch_equilibrate(dms, ns, h->stream);
    check_launch(h);
    auto *dei = h->ar.upload("ell_items", eitems, h->stream);
    launch_ell_build(dms, dei, (int)eitems.size(), h->dst, h->stream);
    check_launch(h);
    zero_all(h, zl, "F");
    run_gathers(h, gF, "F");
    run_diag(h, dI, "F");
    run_pchol_tc(h, pd, "F");
    run_gathers(h, gK, "Kinv");
    fail_check(h, "mixed interior factorization");
    // refine until ||A_IG - A_II X|| <= refine_tol ||A_IG||; the energy form below squares that error
    h->mixed_iters = refine(h, jobs, 1, 12, h->opt.refine_tol, true, "X");
    // S_i = A_GG - A_GI X - X^T R  (R = A_IG - A_II X, the residual of the accepted X)
    std::vector<EllProduct> ps;
    for (const auto &j : jobs) {
        auto &sd = h->subs[j.s];
        EllProduct p = ell_of(h, j.s);
        p.r0 = sd.nI;
        p.m = sd.nG;
        p.ncol = sd.nG;
        p.X = j.X;
        p.ldx = j.ldx;
        p.B = sd.A + (size_t)sd.nI * sd.ld + sd.nI;
        p.ldb = sd.ld;
        p.out = sd.S;
        p.ldo = sd.ldS;
        ps.push_back(p);
    }
    run_ell(h, ps, "S");
    // S[a, b] -= sum_k X[k, a] R[k, b]  (3xTF32 tensor-core products; the term is second order)
    // (FP32 copies of X and of R, the residual of the accepted X written by the refinement)
    std::vector<TcGemm> gc;
    std::vector<GatherOp> gx;
    for (const auto &j : jobs) {
        auto &sd = h->subs[j.s];
        float *Xf = h->ar.get_t<float>("Xf_" + std::to_string(j.s), (size_t)j.ldx * j.ncol);
        const float *Rf = h->ar.get_t<float>("Rf_X" + std::to_string(j.s), (size_t)j.ldr * j.ncol);
        GatherOp o = gop(j.X, j.ldx, reinterpret_cast<double *>(Xf), j.ldx, sd.nI, j.ncol);
        o.dst_f32 = 1;
        gx.push_back(o);
        gc.push_back(TcGemm{Xf, Rf, sd.S, nullptr, nullptr, j.ldx, j.ldr, sd.ldS, sd.nG, sd.nG, sd.nI, 0, 0, -1.0});
    }
    run_gathers(h, gx, "Xf");
    run_tc_gemm(h, gc, "gc");
    launch_symmetrize(h->ops.S, h->ops.nGi, h->ops.ldS, ns, h->stream);
    check_launch(h);
}

// ---- phases --------------------------------------------------------------
void count_coarse(bddc_handle *h) {
    int nC = h->n_corner_dofs;
    for (auto &g : h->globs) nC += g.nrows;
    h->nC = nC;
}

// builds the coarse operators for the current constraints if they changed
void ensure_coarse(bddc_handle *h) {
    if (!h->coarse_dirty) return;
    phase_begin(h, 2);
    h->coarse_fp32 = false;
    if (h->opt.precision == BDDC_MIXED_FP32_SADDLE) {
        try {
            coarse_setup(h, true);
            h->coarse_fp32 = true;
        } catch (const Fp32Breakdown &) {
            reset_status(h);
            h->coarse_fallbacks++;
            coarse_setup(h, false);
        }
    } else if (h->opt.precision == BDDC_MIXED) {
        // the local saddle runs in double-float; a coarse matrix that does not factor
        // in that precision is rebuilt with FP64 local saddles
        try {
            coarse_setup(h, false);
        } catch (const Error &e) {
            if (e.status != BDDC_ENOTSPD) throw;
            reset_status(h);
            h->coarse_fallbacks++;
            h->fp64_class_forced = true;
            try {
                coarse_setup(h, false);
            } catch (const Error &e2) {
                h->fp64_class_forced = false;
                throw Error{e2.status, e2.msg + " (after an FP64 rebuild of the local saddle operators)"};
            }
            h->fp64_class_forced = false;
        }
    } else {
        coarse_setup(h, false);
    }
    phase_end(h, 2);
    phase_collect(h, 2, 2);
    h->coarse_dirty = false;
}

void do_setup(bddc_handle *h) {
    const int ns = h->nsub;
    reset_status(h);
    phase_begin(h, 0);
    std::vector<double *> Aptr(ns);
    std::vector<int> lds(ns);
    ZeroList zl;
    for (int s = 0; s < ns; ++s) {
        auto &sd = h->subs[s];
        zl.add(sd.A, (size_t)sd.ld * sd.n);
        Aptr[s] = sd.A;
        lds[s] = sd.ld;
    }
    zero_all(h, zl, "A");
    if (h->csr_mode) {
        // algebraic input: the CSR entries of every A_i into the dense local matrices
        launch_csr_scatter(h->ar.upload("Aptr", Aptr, h->stream), h->ar.get_t<int64_t>("csr_start", ns + 1), ns,
                           h->ar.get_t<int64_t>("csr_off", std::max<int64_t>(h->csr_nnz, 1)),
                           h->ar.get_t<double>("csr_val", std::max<int64_t>(h->csr_nnz, 1)), h->csr_nnz, h->stream);
        check_launch(h);
    } else {
        // element geometry and assembly
        double *grads = h->ar.get_t<double>("grads", (size_t)h->ne * 8 * 8 * 3);
        double *wdet = h->ar.get_t<double>("wdet", (size_t)h->ne * 8);
        const double *dxyz = h->ar.get_t<double>("xyz", h->nn * 3);
        const int64_t *delems = h->ar.get_t<int64_t>("elems", h->ne * 8);
        launch_element_geometry(dxyz, delems, h->ne, grads, wdet, h->stream);
        check_launch(h);
        AssemblyArgs aa;
        aa.grads = grads;
        aa.wdet = wdet;
        aa.coef = h->ar.get_t<double>("coef", h->ne);
        aa.elem_sub = h->ar.get_t<int32_t>("esub", h->ne);
        aa.elem_pos = h->ar.get_t<int32_t>("epos", h->ne * 8);
        aa.A = h->ar.upload("Aptr", Aptr, h->stream);
        aa.ld = h->ar.upload("Ald", lds, h->stream);
        aa.nu = h->nu;
        aa.ncomp = h->ncomp;
        for (size_t col = 0; col < h->colors.size(); ++col) {
            const int32_t *ce = h->ar.get_t<int32_t>("color_" + std::to_string(col), h->colors[col].size());
            launch_element_scatter(aa, ce, (int)h->colors[col].size(), h->stream);
            check_launch(h);
        }
    }
    // weights: diag of the interface block (before elimination of interiors)
    double *diag = h->ar.get_t<double>("diag", std::max<int64_t>(h->sumG, 1));
    std::vector<GatherOp> gd;
    for (int s = 0; s < ns; ++s) {
        auto &sd = h->subs[s];
        if (sd.nG == 0) continue;
        // a 1 x nG gather with column stride ld + 1 walks the diagonal of the interface block
        gd.push_back(gop(sd.A + (size_t)sd.nI * sd.ld + sd.nI, sd.ld + 1, diag + h->offG[s], 1, 1, sd.nG));
    }
    run_gathers(h, gd, "diag");
    double *total = h->ar.get_t<double>("wtotal", std::max(h->nG, 1));
    double *delta = h->ar.get_t<double>("delta", std::max<int64_t>(h->sumG, 1));
    launch_weights(h->ops, diag, total, delta, h->stream);
    check_launch(h);
    phase_end(h, 0);
    h->assembled = true;
    phase_begin(h, 1);
    // interior elimination: partial Cholesky of every A_i with nstop = n_I
    double fl = 0.0;
    for (auto &sd : h->subs)
        fl += (double)sd.nI * sd.nI * sd.nI / 3.0 + (double)sd.nI * sd.nI * sd.nG + (double)sd.nI * sd.nG * sd.nG;
    h->phase_flop[1] = fl;
    h->interior_fp32 = false;
    bool fp64_interior = h->opt.precision == BDDC_FP64;
    if (!fp64_interior) {
        try {
            interior_mixed(h);
            h->interior_fp32 = true;
        } catch (const Error &e) {
            // FP32 factorization or refinement failed: the interior elimination is redone in FP64
            if (e.status != BDDC_ENOCONV && e.status != BDDC_ENOTSPD) throw;
            reset_status(h);
            h->interior_fallbacks++;
            fp64_interior = true;
        }
    }
    h->factored = fp64_interior;
    if (fp64_interior) {
        std::vector<PcholDesc<double>> d;
        for (int s = 0; s < ns; ++s)
            d.push_back(PcholDesc<double>{h->subs[s].A, h->subs[s].n, h->subs[s].ld, h->subs[s].nI, 0});
        run_pchol<double>(h, d, "AII");
        // S_i full from the trailing lower block
        std::vector<GatherOp> gs;
        for (int s = 0; s < ns; ++s) {
            auto &sd = h->subs[s];
            GatherOp o = gop(sd.A, sd.ld, sd.S, sd.ldS, sd.nG, sd.nG);
            o.src_row_off = sd.nI;
            o.src_col_off = sd.nI;
            o.src_sym = 1;
            gs.push_back(o);
        }
        run_gathers(h, gs, "S");
    }
    phase_end(h, 1);
    fail_check(h, "interior factorization");
    build_average_globs(h);
    // coarse numbering needs the glob list; Phi buffers depend on the row counts
    for (int s = 0; s < ns; ++s) h->subs[s].na = 0;
    {
        // count rows per sub to size Phi before coarse_setup lays them out
        std::vector<int> na(ns, 0);
        for (auto &g : h->globs)
            for (int s : g.subs) na[s] += g.nrows;
        for (int s = 0; s < ns; ++s) h->subs[s].na = na[s];
        set_phi_pointers(h);
    }
    count_coarse(h);
    h->coarse_dirty = true;
    h->face_rows_dev.assign(h->faces.size(), nullptr);
    phase_collect(h, 0, 1);
}

}  // namespace

// ===========================================================================
// adapt
namespace {

// Face eigenproblems C y = lambda y (eig.h).  Faces of order <= opt.eig_large_n go to the dense
// kernel (Householder + Sturm counts, one CTA each).  Larger faces, whose one-CTA reduction
// would set the length of the phase, run the batched LOBPCG of lobpcg.h: k = 16, then 32
// for faces whose block held no rejected Ritz value, each converged face checked by the
// Cholesky certificate of its count; a face that does not converge or whose certificate
// fails is solved by the dense kernel.  The face rows of the LOBPCG faces are then formed
// by the face kernel from the supplied eigenpairs.
constexpr int kTriMultiN = 200;

void run_face_eigs(bddc_handle *h, const std::vector<EigDesc> &eds, double tau, int fixed_k, LobStats *stats) {
    const int use_ff = h->opt.precision != BDDC_FP64 ? 1 : 0;
    std::vector<EigDesc> small, big;
    const int large_n = h->opt.eig_large_n;
    // LOBPCG needs a trial space [X P R] narrower than the problem: n > 3 x 16
    for (const auto &e : eds) (large_n >= 0 && e.n > large_n && e.n > 48 && fixed_k + 1 < kLobMaxK
                                   ? big : small).push_back(e);
    auto dense1 = [&](const std::vector<EigDesc> &v, const std::string &tag, int ff) {
        if (v.empty()) return;
        int nmax = 0;
        for (const auto &e : v) nmax = std::max(nmax, e.n);
        auto *d = h->ar.upload("eigdesc_" + tag, v, h->stream);
        double work = 0.0;   // the Householder reduction, 4/3 n^3 flop per face it reduces
        for (const auto &e : v)
            if (e.given == 0) work += 4.0 / 3.0 * (double)e.n * e.n * e.n;
        const long tok = kt_begin(h);
        launch_face_eig_n(d, (int)v.size(), nmax, tau, h->opt.drop_rel, ff, fixed_k, h->dst, h->stream);
        check_launch(h);
        kt_end(h, tok, KT_FACE_RED, work);
    };
    // the dense kernel; faces above kTriMultiN get their Householder reduction from
    // several CTAs each (tridiag.cu), then the kernel's remaining steps
    auto dense = [&](const std::vector<EigDesc> &v, const std::string &tag, int ff) {
        std::vector<EigDesc> one, multi;
        for (const auto &e : v) (e.n > kTriMultiN ? multi : one).push_back(e);
        dense1(one, tag, ff);
        if (multi.empty()) return;
        std::stable_sort(multi.begin(), multi.end(), [](const EigDesc &a, const EigDesc &b) { return a.n > b.n; });
        int nmax = multi.front().n;
        const int cap = tridiag_multi_capacity(nmax);
        BDDC_REQUIRE(cap >= 2, BDDC_ECUDA, "no co-resident CTAs for the face reduction");
        unsigned *bar = h->ar.get_t<unsigned>("tri_bar_" + tag, 2 * multi.size());
        // CTAs per face in proportion to its reduction work (n^3), so that the largest faces,
        // whose n - 2 dependent steps are the launch's critical path, get the most: all faces in
        // one cooperative launch when 2 CTAs each fit, at most 64 for one face
        std::vector<int> Gf(multi.size(), 2);
        if (2 * multi.size() <= (size_t)cap) {
            double w3 = 0.0;
            for (const auto &e : multi) w3 += (double)e.n * e.n * e.n;
            const int spare = cap - 2 * (int)multi.size();
            for (size_t q = 0; q < multi.size(); ++q) {
                const double n = multi[q].n;
                Gf[q] = 2 + (int)std::floor(spare * (n * n * n) / w3);
                Gf[q] = std::min(Gf[q], std::min(64, std::max(2, (multi[q].n + 15) / 16)));
            }
        }
        size_t pos = 0;
        int wave = 0;
        while (pos < multi.size()) {   // waves of faces whose CTAs fit co-resident
            std::vector<TridiagDesc> td;
            std::vector<int2> items;
            int used = 0;
            for (; pos < multi.size(); ++pos) {
                const EigDesc &e = multi[pos];
                const int G = std::min(Gf[pos], cap);
                if (used + G > cap) break;
                for (int g = 0; g < G; ++g) items.push_back(make_int2((int)td.size(), g));
                td.push_back(TridiagDesc{e.C, e.n, e.ld, e.work, G, bar + 2 * pos});
                used += G;
            }
            const std::string ws = tag + "_" + std::to_string(wave++);
            BDDC_CUDA(cudaMemsetAsync(bar, 0, sizeof(unsigned) * 2 * multi.size(), h->stream));
            auto *dtd = h->ar.upload("tri_desc_" + ws, td, h->stream);
            auto *dti = h->ar.upload("tri_it_" + ws, items, h->stream);
            double work = 0.0;
            for (const auto &t : td) work += 4.0 / 3.0 * (double)t.n * t.n * t.n;
            const long tok = kt_begin(h);
            cudaError_t err = launch_tridiag_multi(dtd, dti, (int)items.size(), nmax, ff, h->dst, h->opt.timeout_s,
                                                   h->stream);
            BDDC_REQUIRE(err == cudaSuccess, BDDC_ECUDA, std::string("face reduction launch: ") + cudaGetErrorString(err));
            h->launches++;
            kt_end(h, tok, KT_FACE_RED, work);
        }
        // eigenpairs and face rows of these faces, several CTAs each; the face kernel finishes them
        for (auto &e : multi) e.given = 2;
        {
            const int G = kFaceVecCTAs;
            std::vector<int2> vit;
            std::vector<size_t> off(multi.size() + 1, 0);
            for (size_t q = 0; q < multi.size(); ++q) {
                off[q + 1] = off[q] + (size_t)G * kFaceVecWarps * 6 * multi[q].n;
                for (int g = 0; g < G; ++g) vit.push_back(make_int2((int)q, g));
            }
            double *scr_all = h->ar.get_t<double>("fvscr_" + tag, std::max<size_t>(off.back(), 1));
            std::vector<double *> scr(multi.size());
            for (size_t q = 0; q < multi.size(); ++q) scr[q] = scr_all + off[q];
            auto *dvd = h->ar.upload("fvdesc_" + tag, multi, h->stream);
            auto *dvi = h->ar.upload("fvit_" + tag, vit, h->stream);
            auto *dvs = h->ar.upload("fvscrp_" + tag, scr, h->stream);
            const long tok = kt_begin(h);
            launch_face_vec(dvd, dvi, (int)vit.size(), G, nmax, tau, fixed_k, dvs, h->stream);
            check_launch(h);
            kt_end(h, tok, KT_FACE_RED, 0.0);
        }
        for (auto &e : multi) e.given = 3;
        dense1(multi, tag + "_tri", 0);
    };
    dense(small, "small", use_ff);
    if (stats) *stats = LobStats{(int)big.size(), 0, 0};
    if (big.empty()) return;
    // batched FP64 GEMMs with the descriptors and tile items uploaded once
    struct GemmBatch {
        GemmDesc *d = nullptr;
        int4 *it = nullptr;
        int n = 0;
    };
    auto prep_gemm = [&](const std::vector<GemmDesc> &g, const std::string &tag) {
        GemmBatch b;
        std::vector<int4> items;
        for (int q = 0; q < (int)g.size(); ++q)
            for (int a = 0; a < (g[q].m + kTile - 1) / kTile; ++a)
                for (int c = 0; c < (g[q].n + kTile - 1) / kTile; ++c) items.push_back(make_int4(q, a, c, 0));
        b.d = h->ar.upload("lobg_" + tag, g, h->stream);
        b.it = h->ar.upload("lobi_" + tag, items, h->stream);
        b.n = (int)items.size();
        return b;
    };
    auto gemm = [&](const GemmBatch &b) {
        launch_gemm(b.d, b.it, b.n, 0, h->stream);
        check_launch(h);
    };
    std::vector<int> todo(big.size());
    std::iota(todo.begin(), todo.end(), 0);
    std::vector<char> solved(big.size(), 0);
    std::vector<int> fallback;
    for (int pass = 0; pass < 2 && !todo.empty(); ++pass) {
        const int k = pass == 0 ? 16 : kLobMaxK, m = 3 * k;
        const int nb = (int)todo.size();
        const std::string ps = std::to_string(pass);
        std::vector<size_t> off(nb + 1, 0);
        std::vector<int> lds(nb);
        for (int b = 0; b < nb; ++b) {
            const int n = big[todo[b]].n;
            lds[b] = round_up(n, 8);
            off[b + 1] = off[b] + 4 * (size_t)lds[b] * m + 6 * (size_t)m * m + 2 * (size_t)k * m + 2 * k;
        }
        double *pool = h->ar.get_t<double>("lob_pool" + ps, off[nb]);
        int *ipool = h->ar.get_t<int>("lob_ipool" + ps, (size_t)nb * 4 + 1);
        std::vector<LobDesc> ld(nb);
        std::vector<GemmDesc> gar[2], ggram[2], gupd[2], gax[2];
        for (int b = 0; b < nb; ++b) {
            const EigDesc &e = big[todo[b]];
            const int n = e.n;
            double *p = pool + off[b];
            LobDesc &d = ld[b];
            d.C = e.C;
            d.n = n;
            d.ldc = e.ld;
            d.k = k;
            d.lds = lds[b];
            for (int c = 0; c < 2; ++c) {
                d.S[c] = p;
                p += (size_t)lds[b] * m;
                d.AS[c] = p;
                p += (size_t)lds[b] * m;
            }
            d.G = p;
            p += 2 * (size_t)m * m;
            d.coef = p;
            p += 2 * (size_t)k * m;
            d.theta = p;
            p += k;
            d.rnorm = p;
            p += k;
            d.scratch = p;
            d.state = ipool + 4 * b;
            for (int c = 0; c < 2; ++c) {
                const size_t r0 = (size_t)2 * k * d.lds;
                gar[c].push_back(GemmDesc{e.C, d.S[c] + r0, d.AS[c] + r0, e.ld, d.lds, d.lds, n, k, n, 0, 0, 1.0, 0.0});
                ggram[c].push_back(GemmDesc{d.S[c], d.AS[c], d.G, d.lds, d.lds, m, m, m, n, 1, 0, 1.0, 0.0});
                ggram[c].push_back(GemmDesc{d.S[c], d.S[c], d.G + (size_t)m * m, d.lds, d.lds, m, m, m, n, 1, 0, 1.0, 0.0});
                gupd[c].push_back(GemmDesc{d.S[c], d.coef, d.S[1 - c], d.lds, m, d.lds, n, 2 * k, m, 0, 0, 1.0, 0.0});
                // C P by the same combination; C X is recomputed from X every iteration (below),
                // so rounding in the combined products never enters the residual test
                gupd[c].push_back(GemmDesc{d.AS[c], d.coef + (size_t)k * m, d.AS[1 - c] + (size_t)k * d.lds, d.lds, m,
                                           d.lds, n, k, m, 0, 0, 1.0, 0.0});
                gax[c].push_back(GemmDesc{e.C, d.S[c], d.AS[c], e.ld, d.lds, d.lds, n, k, n, 0, 0, 1.0, 0.0});
            }
        }
        auto *dl = h->ar.upload("lob_desc" + ps, ld, h->stream);
        GemmBatch b_ar[2], b_gram[2], b_upd[2], b_ax[2];
        for (int c = 0; c < 2; ++c) {
            const std::string cs = ps + "_" + std::to_string(c);
            b_ar[c] = prep_gemm(gar[c], "ar" + cs);
            b_gram[c] = prep_gemm(ggram[c], "gram" + cs);
            b_upd[c] = prep_gemm(gupd[c], "upd" + cs);
            b_ax[c] = prep_gemm(gax[c], "ax" + cs);
        }
        if (pass == 0) {
            std::vector<int2> sym;
            for (int b = 0; b < nb; ++b)
                for (int c = 0; c < (ld[b].n + 63) / 64; ++c) sym.push_back(make_int2(b, c));
            auto *dsy = h->ar.upload("lob_sym", sym, h->stream);
            launch_lob_symmetrize(dl, dsy, (int)sym.size(), h->stream);
            check_launch(h);
        }
        launch_lob_init(dl, nb, 0, h->stream);
        check_launch(h);
        int cur = 0, it = 0;
        std::vector<int> st((size_t)nb * 4);
        for (; it < h->opt.eig_maxit; ++it) {
            gemm(b_ax[cur]);
            launch_lob_prep(dl, nb, cur, tau, fixed_k, h->opt.eig_tol, 0, h->stream);
            check_launch(h);
            gemm(b_ar[cur]);
            gemm(b_gram[cur]);
            launch_lob_rr(dl, nb, h->stream);
            check_launch(h);
            gemm(b_upd[cur]);
            cur ^= 1;
            if (it % 4 == 3) {
                BDDC_CUDA(cudaMemcpyAsync(st.data(), ipool, st.size() * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
                BDDC_CUDA(cudaStreamSynchronize(h->stream));
                bool all = true;
                for (int b = 0; b < nb; ++b) all = all && st[4 * b] != 0;
                if (all) break;
            }
        }
        // fresh C X, the final residual test, the outputs and the certificate
        gemm(b_ax[cur]);
        launch_lob_prep(dl, nb, cur, tau, fixed_k, h->opt.eig_tol, 1, h->stream);
        check_launch(h);
        std::vector<LobOutDesc> od(nb);
        std::vector<LobCertDesc> cd(nb);
        std::vector<int2> citems;
        std::vector<PcholDesc<double>> chol(nb);
        int *fails = h->ar.get_t<int>("lob_fail" + ps, nb);
        BDDC_CUDA(cudaMemsetAsync(fails, 0, sizeof(int) * nb, h->stream));
        for (int b = 0; b < nb; ++b) {
            const EigDesc &e = big[todo[b]];
            const int n = e.n, ldm = round_up(n, 8);
            od[b] = LobOutDesc{ld[b].S[cur], n, ld[b].lds, k, ld[b].theta, e.lam, e.vec, e.counts, e.cap, ld[b].state};
            double *M = h->ar.get_t<double>("lob_cert" + ps + "_" + std::to_string(b), (size_t)ldm * n);
            cd[b] = LobCertDesc{e.C, n, e.ld, ld[b].S[cur], ld[b].lds, k, ld[b].theta, e.counts, M, ldm, 1e-6};
            for (int c = 0; c < (n + 63) / 64; ++c) citems.push_back(make_int2(b, c));
            chol[b] = PcholDesc<double>{M, n, ldm, n, 0, nullptr, 0, 0, 0, fails + b};
        }
        auto *dod = h->ar.upload("lob_out" + ps, od, h->stream);
        launch_lob_select(dod, nb, tau, fixed_k, h->stream);
        check_launch(h);
        auto *dcd = h->ar.upload("lob_certd" + ps, cd, h->stream);
        auto *dci = h->ar.upload("lob_certi" + ps, citems, h->stream);
        launch_lob_cert(dcd, dci, (int)citems.size(), h->stream);
        check_launch(h);
        run_pchol<double>(h, chol, "F#lob" + ps);
        std::vector<int> fl(nb);
        BDDC_CUDA(cudaMemcpyAsync(st.data(), ipool, st.size() * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        BDDC_CUDA(cudaMemcpyAsync(fl.data(), fails, sizeof(int) * nb, cudaMemcpyDeviceToHost, h->stream));
        BDDC_CUDA(cudaStreamSynchronize(h->stream));
        std::vector<int> next;
        for (int b = 0; b < nb; ++b) {
            if (stats) stats->iters = std::max(stats->iters, st[4 * b + 1]);
            if (st[4 * b + 2] == 1 && fl[b] == 0)
                solved[todo[b]] = 1;
            else if (st[4 * b + 2] == 2 && pass == 0 && big[todo[b]].n > 3 * kLobMaxK)
                next.push_back(todo[b]);   // block too small: again with the larger block
            else
                fallback.push_back(todo[b]);
        }
        todo = next;
    }
    for (int b : todo) fallback.push_back(b);
    std::vector<EigDesc> given, dense_big;
    for (size_t b = 0; b < big.size(); ++b) {
        if (solved[b]) {
            EigDesc e = big[b];
            e.given = 1;
            given.push_back(e);
        }
    }
    for (int b : fallback) dense_big.push_back(big[b]);
    if (stats) stats->fallback = (int)dense_big.size();
    dense(dense_big, "fallback", use_ff);
    dense(given, "given", 0);
}

void do_adapt(bddc_handle *h, double tau, bddc_adapt_info *info, int fixed_k = 0) {
    const int nf = (int)h->faces.size();
    reset_status(h);
    // the pair problems use the initial constraints only; drop rows of an earlier adapt
    h->globs.erase(std::remove_if(h->globs.begin(), h->globs.end(),
                                  [](const GlobRows &g) { return g.face >= 0 || g.edge >= 0; }),
                   h->globs.end());
    h->edge_rows.clear();
    h->n_edge_rows = h->n_edges_with_rows = 0;
    if (nf == 0) {
        if (info) *info = bddc_adapt_info{};
        return;
    }
    for (auto &fp : h->faces) {
        fp.lam.clear();
        fp.nsel = fp.nkept = fp.ties = 0;
    }
    phase_begin(h, 3);
    // E1: per (sub, face) Schur complement of S_i onto t = [s (s order); shared corners],
    // by nested condensation.  The faces of every substructure are split into a binary
    // tree; a tree node holds the Schur complement of S_i onto the union R of its faces'
    // target sets, formed from its parent's by eliminating the parent's dofs outside R
    // (a gather + a partial Cholesky).  By the quotient property of Schur complements a
    // leaf's matrix is the Schur complement of S_i onto its target, as a direct
    // elimination would give it; with halving sets the tree costs ~0.8 n^3 flop per
    // substructure where one elimination per face costs ~n^3/3 each.
    std::vector<PcholDesc<double>> dE1, dE2, dE3;
    std::vector<GatherOp> gE1, gE2, gE3, gQ;
    std::vector<DiagOp> idE3;
    struct PairBufs {
        double *T[2];
        int nT[2], ldT[2], no[2];
        double *Y;
        int nY, ldY;
        double *M3;
        int ldM3;
        double *Q, *W1, *C;
        int ns, nc;
        // initial constraints on s (averages): the problem in u with z = G u
        int nsp = 0, pi = -1;   // order of the reduced problem; index into pis (-1: none)
        double *M3c = nullptr, *Xg = nullptr;
        int ldM3c = 0, ldXg = 0;
    };
    std::vector<PairBufs> pbufs(nf);
    int nmax = 0;
    // algorithmic FP64 flops of the condensations: partial Cholesky of n with nstop = m
    // (m^3/3 + m^2 (n - m) + m (n - m)^2), for the E1 matrices here and E2, E3 below
    auto pchol_flop = [](double n, double m) { return m * m * m / 3.0 + m * m * (n - m) + m * (n - m) * (n - m); };
    double cflop = 0.0;
    struct CondNode {
        int sub = 0, parent = -1, leaf = -1, depth = 0;
        std::vector<int> R;          // retained interface positions, in the node's matrix order
        const double *base = nullptr;
        int ld = 0, off = 0, n = 0;  // matrix (lower triangle) at base[off + a + (off + b) ld], a, b < |R|
    };
    std::vector<CondNode> cn;
    std::vector<std::vector<int>> leaf_t(2 * nf);   // leaf (2 f + side): target [s (s order); corners]
    std::vector<std::vector<int>> sub_leaves(h->nsub);
    for (int f = 0; f < nf; ++f) {
        auto &fp = h->faces[f];
        pbufs[f].ns = (int)fp.s_g.size();
        pbufs[f].nc = (int)fp.ci_pos.size();
        nmax = std::max(nmax, pbufs[f].ns);
        for (int side = 0; side < 2; ++side) {
            const auto &spos = side ? fp.pos_j : fp.pos_i;
            const auto &cpos = side ? fp.cj_pos : fp.ci_pos;
            auto &t = leaf_t[2 * f + side];
            t.assign(spos.begin(), spos.end());
            t.insert(t.end(), cpos.begin(), cpos.end());
            sub_leaves[side ? fp.j : fp.i].push_back(2 * f + side);
        }
    }
    int max_depth = 0;
    for (int s = 0; s < h->nsub; ++s) {
        auto &leaves = sub_leaves[s];
        if (leaves.empty()) continue;
        // leaves ordered by the mean interface position of their targets (interface
        // positions follow the global dof order, so nearby faces stay together)
        std::vector<double> key(2 * nf, 0.0);
        for (int l : leaves) {
            double m = 0.0;
            for (int p : leaf_t[l]) m += p;
            key[l] = m / std::max<size_t>(1, leaf_t[l].size());
        }
        std::stable_sort(leaves.begin(), leaves.end(), [&](int a, int b) { return key[a] < key[b]; });
        // recursive split into halves of about equal target size
        struct Range { int lo, hi, parent, depth; };
        std::vector<Range> todo{{0, (int)leaves.size(), -1, 0}};
        std::vector<std::pair<int, std::pair<int, int>>> made;   // node -> leaf range
        while (!todo.empty()) {
            Range r = todo.back();
            todo.pop_back();
            CondNode nd;
            nd.sub = s;
            nd.parent = r.parent;
            nd.depth = r.depth;
            max_depth = std::max(max_depth, r.depth);
            const int id = (int)cn.size();
            if (r.hi - r.lo == 1) {
                nd.leaf = leaves[r.lo];
                nd.R = leaf_t[nd.leaf];
            } else {
                std::vector<char> in(h->subs[s].nG, 0);
                size_t tot = 0;
                for (int k = r.lo; k < r.hi; ++k) tot += leaf_t[leaves[k]].size();
                for (int k = r.lo; k < r.hi; ++k)
                    for (int p : leaf_t[leaves[k]]) in[p] = 1;
                for (int p = 0; p < h->subs[s].nG; ++p)
                    if (in[p]) nd.R.push_back(p);
                size_t acc = 0;
                int mid = r.lo + 1;
                for (int k = r.lo; k < r.hi - 1; ++k) {
                    acc += leaf_t[leaves[k]].size();
                    mid = k + 1;
                    if (2 * acc >= tot) break;
                }
                todo.push_back({r.lo, mid, id, r.depth + 1});
                todo.push_back({mid, r.hi, id, r.depth + 1});
            }
            cn.push_back(std::move(nd));
        }
    }
    // level by level: every node's matrix from its parent's (the roots from S_i)
    for (int d = 0; d <= max_depth; ++d) {
        std::vector<GatherOp> g;
        std::vector<PcholDesc<double>> dd;
        for (int v = 0; v < (int)cn.size(); ++v) {
            auto &nd = cn[v];
            if (nd.depth != d) continue;
            const auto &sd = h->subs[nd.sub];
            std::vector<int> perm;           // parent-local indices: [eliminated; R in node order]
            const double *src;
            int ld_src, off_src, n_par;
            if (nd.parent < 0) {
                src = sd.S;
                ld_src = sd.ldS;
                off_src = 0;
                n_par = sd.nG;
                if (nd.leaf < 0 && (int)nd.R.size() == sd.nG) {   // all of S_i retained: the root is S_i
                    nd.base = sd.S;
                    nd.ld = sd.ldS;
                    nd.off = 0;
                    nd.n = sd.nG;
                    continue;
                }
                std::vector<char> in(sd.nG, 0);
                for (int p : nd.R) in[p] = 1;
                for (int p = 0; p < sd.nG; ++p)
                    if (!in[p]) perm.push_back(p);
                perm.insert(perm.end(), nd.R.begin(), nd.R.end());
            } else {
                const auto &pn = cn[nd.parent];
                src = pn.base;
                ld_src = pn.ld;
                off_src = pn.off;
                n_par = (int)pn.R.size();
                std::vector<int> loc(sd.nG, -1);
                for (int k = 0; k < n_par; ++k) loc[pn.R[k]] = k;
                std::vector<char> in(n_par, 0);
                for (int p : nd.R) in[loc[p]] = 1;
                for (int k = 0; k < n_par; ++k)
                    if (!in[k]) perm.push_back(k);
                for (int p : nd.R) perm.push_back(loc[p]);
            }
            const int n = n_par, no = n - (int)nd.R.size();
            nd.ld = round_up(std::max(n, 1), 8);
            nd.n = n;
            nd.off = no;
            double *buf = h->ar.get_t<double>("E1n_" + std::to_string(v), (size_t)nd.ld * std::max(n, 1));
            nd.base = buf;
            int *dp = h->ar.upload("E1p_" + std::to_string(v), perm, h->stream);
            GatherOp o = gop(src, ld_src, buf, nd.ld, n, n);
            o.rmap = dp;
            o.cmap = dp;
            o.src_row_off = off_src;
            o.src_col_off = off_src;
            o.src_sym = 1;
            o.dst_lower = 1;
            g.push_back(o);
            if (no > 0) {
                dd.push_back(PcholDesc<double>{buf, n, nd.ld, no, 0});
                cflop += pchol_flop(n, no);
            }
        }
        run_gathers(h, g, "E1#" + std::to_string(d));
        run_pchol_fp64class(h, dd, "E1#" + std::to_string(d));
    }
    for (const auto &nd : cn) {
        if (nd.leaf < 0) continue;
        auto &B = pbufs[nd.leaf / 2];
        const int side = nd.leaf % 2;
        B.T[side] = const_cast<double *>(nd.base);
        B.nT[side] = nd.n;
        B.ldT[side] = nd.ld;
        B.no[side] = nd.off;
    }
    // E2: pair matrix [C; s_i; s_j], eliminate C -> S^ (2 ns)
    ZeroList zy;
    for (int f = 0; f < nf; ++f) {
        auto &B = pbufs[f];
        const int ns = B.ns, nc = B.nc;
        B.nY = nc + 2 * ns;
        B.ldY = round_up(std::max(B.nY, 1), 8);
        B.Y = h->ar.get_t<double>("E2_" + std::to_string(f), (size_t)B.ldY * std::max(B.nY, 1));
        zy.add(B.Y, (size_t)B.ldY * std::max(B.nY, 1));
        for (int side = 0; side < 2; ++side) {
            const int o0 = B.no[side];  // trailing offset: [s (ns); C (nc)]
            // C block (accumulate both sides)
            if (nc > 0) {
                GatherOp o = gop(B.T[side], B.ldT[side], B.Y, B.ldY, nc, nc);
                o.src_row_off = o0 + ns;
                o.src_col_off = o0 + ns;
                o.src_sym = 1;
                o.dst_lower = 1;
                o.accumulate = 1;
                (side ? gE3 : gE2).push_back(o);  // two passes to avoid write conflicts
                o = gop(B.T[side], B.ldT[side], B.Y, B.ldY, ns, nc);
                o.src_row_off = o0;
                o.src_col_off = o0 + ns;
                o.src_sym = 1;
                o.dst_row_off = nc + side * ns;
                gE2.push_back(o);
            }
            GatherOp o = gop(B.T[side], B.ldT[side], B.Y, B.ldY, ns, ns);
            o.src_row_off = o0;
            o.src_col_off = o0;
            o.src_sym = 1;
            o.dst_row_off = nc + side * ns;
            o.dst_col_off = nc + side * ns;
            o.dst_lower = 1;
            gE2.push_back(o);
        }
        dE2.push_back(PcholDesc<double>{B.Y, B.nY, B.ldY, nc, 0});
    }
    zero_all(h, zy, "E2");
    run_gathers(h, gE2, "E2a");
    run_gathers(h, gE3, "E2b");
    gE3.clear();
    run_pchol_fp64class(h, dE2, "E2");
    for (auto &dd : dE2) cflop += pchol_flop(dd.n, dd.nstop);
    // E3: M3 = [[Mww, ., .], [Mbw, Mbb, .], [0, I, 0]] from S^ blocks, + deflation, eliminate 2 ns
    // (pairs with initial constraints: compressed to the jumps that satisfy them first)
    std::vector<PiDesc> pis;
    int pi_nmax = 0;
    std::vector<DeflateDesc> defl;
    std::vector<PairWeightDesc> pw;
    ZeroList zm;
    for (int f = 0; f < nf; ++f) {
        auto &fp = h->faces[f];
        auto &B = pbufs[f];
        const int ns = B.ns, nc = B.nc;
        int n3 = 3 * ns;
        B.ldM3 = round_up(std::max(n3, 1), 8);
        B.M3 = h->ar.get_t<double>("M3_" + std::to_string(f), (size_t)B.ldM3 * std::max(n3, 1));
        zm.add(B.M3, (size_t)B.ldM3 * std::max(n3, 1));
        if (ns == 0) continue;
        // S^ blocks live in Y at offset nc: S11 at (nc, nc), S21 at (nc+ns, nc), S22 at (nc+ns, nc+ns)
        auto blk = [&](int bi, int bj, int dro, int dco, double scale, int lower, std::vector<GatherOp> &dst) {
            GatherOp o = gop(B.Y, B.ldY, B.M3, B.ldM3, ns, ns);
            o.src_row_off = nc + bi * ns;
            o.src_col_off = nc + bj * ns;
            o.src_sym = 1;
            o.dst_row_off = dro;
            o.dst_col_off = dco;
            o.scale = scale;
            o.dst_lower = lower;
            o.accumulate = 1;
            dst.push_back(o);
        };
        // (w2,w2) = S11 + S12 + S21 + S22 ; (b,w2) = S11 + S12 ; (b,b) = S11
        // each pass writes every target once so passes can run in parallel over pairs
        blk(0, 0, 0, 0, 1.0, 1, gE3);
        blk(0, 0, ns, 0, 1.0, 0, gE3);
        blk(0, 0, ns, ns, 1.0, 1, gE3);
        blk(0, 1, 0, 0, 1.0, 1, gQ);
        blk(0, 1, ns, 0, 1.0, 0, gQ);
        idE3.push_back(DiagOp{B.M3, B.ldM3, 2 * ns, ns, ns, 1.0});
        if (fp.nnull > 0) {
            double *N0 = h->ar.upload("N0_" + std::to_string(f), fp.N0, h->stream);
            defl.push_back(DeflateDesc{B.Y + (size_t)nc * B.ldY + nc, B.ldY, B.M3, B.ldM3, N0, ns, fp.nnull});
        }
        // initial constraints (averages over globs inside s shared by i and j): groups of s positions
        std::vector<std::vector<int>> groups;
        for (auto &g : h->globs) {
            if (g.face >= 0) continue;
            if (std::find(g.subs.begin(), g.subs.end(), fp.i) == g.subs.end() ||
                std::find(g.subs.begin(), g.subs.end(), fp.j) == g.subs.end())
                continue;
            std::vector<int> pos(g.gdofs.size());
            bool inside = true;
            for (size_t k = 0; k < g.gdofs.size() && inside; ++k) {
                auto it = std::lower_bound(fp.s_g.begin(), fp.s_g.end(), g.gdofs[k]);
                inside = it != fp.s_g.end() && *it == g.gdofs[k];
                if (inside) pos[k] = (int)(it - fp.s_g.begin());
            }
            if (!inside) continue;
            for (int comp = 0; comp < h->ncomp; ++comp) {
                std::vector<int> mem;
                for (size_t k = comp; k < pos.size(); k += h->ncomp) mem.push_back(pos[k]);
                if (!mem.empty()) groups.push_back(mem);
            }
        }
        if (groups.empty()) {
            dE3.push_back(PcholDesc<double>{B.M3, n3, B.ldM3, 2 * ns, 0, nullptr, 0, 2 * ns, ns});
        } else {
            std::vector<int> newidx(ns, 0), lead(ns, -1), grp(ns, -1), keep, gptr{0}, gidx;
            for (size_t g = 0; g < groups.size(); ++g) {
                for (size_t q = 0; q < groups[g].size(); ++q) {
                    const int a = groups[g][q];
                    grp[a] = (int)g;
                    if (q == 0)
                        newidx[a] = -1;
                    else
                        lead[a] = groups[g][0];
                    gidx.push_back(a);
                }
                gptr.push_back((int)gidx.size());
            }
            for (int a = 0; a < ns; ++a)
                if (newidx[a] >= 0) {
                    newidx[a] = (int)keep.size();
                    keep.push_back(a);
                }
            const std::string fs = std::to_string(f);
            B.nsp = (int)keep.size();
            const int nc3 = ns + 2 * B.nsp;
            B.ldM3c = round_up(std::max(nc3, 1), 8);
            B.M3c = h->ar.get_t<double>("M3c_" + fs, (size_t)B.ldM3c * std::max(nc3, 1));
            B.ldXg = round_up(ns, 8);
            B.Xg = h->ar.get_t<double>("Xg_" + fs, (size_t)B.ldXg * std::max(B.nsp, 1));
            PiDesc pd{};
            pd.M3 = B.M3;
            pd.ld3 = B.ldM3;
            pd.M3c = B.M3c;
            pd.ldc = B.ldM3c;
            pd.Xg = B.Xg;
            pd.ldg = B.ldXg;
            pd.newidx = h->ar.upload("pin_" + fs, newidx, h->stream);
            pd.lead = h->ar.upload("pil_" + fs, lead, h->stream);
            pd.grp = h->ar.upload("pig_" + fs, grp, h->stream);
            pd.keep = h->ar.upload("pik_" + fs, keep, h->stream);
            pd.gptr = h->ar.upload("pip_" + fs, gptr, h->stream);
            pd.gidx = h->ar.upload("pii_" + fs, gidx, h->stream);
            pd.ns = ns;
            pd.nsp = B.nsp;
            pd.ngroups = (int)groups.size();
            B.pi = (int)pis.size();
            pis.push_back(pd);
            pi_nmax = std::max(pi_nmax, ns);
            if (B.nsp > 0) dE3.push_back(PcholDesc<double>{B.M3c, nc3, B.ldM3c, ns + B.nsp, 0});
        }
        // pair weights for Q
        double *di = h->ar.get_t<double>("pwi_" + std::to_string(f), ns);
        double *dj = h->ar.get_t<double>("pwj_" + std::to_string(f), ns);
        int *pi = h->ar.upload("ppi_" + std::to_string(f), fp.pos_i, h->stream);
        int *pj = h->ar.upload("ppj_" + std::to_string(f), fp.pos_j, h->stream);
        double *diag = h->ar.get_t<double>("diag", h->sumG);
        pw.push_back(PairWeightDesc{diag + h->offG[fp.i], diag + h->offG[fp.j], pi, pj, di, dj, ns});
    }
    zero_all(h, zm, "E3");
    run_gathers(h, gE3, "E3a");
    run_gathers(h, gQ, "E3b");
    // pass 3: S21 into (w2,w2) and S22 into (w2,w2)
    {
        std::vector<GatherOp> g;
        for (int f = 0; f < nf; ++f) {
            auto &B = pbufs[f];
            const int ns = B.ns, nc = B.nc;
            if (ns == 0) continue;
            GatherOp o = gop(B.Y, B.ldY, B.M3, B.ldM3, ns, ns);
            o.src_row_off = nc + ns;
            o.src_col_off = nc;
            o.src_sym = 1;
            o.dst_lower = 1;
            o.accumulate = 1;
            g.push_back(o);
        }
        run_gathers(h, g, "E3c");
        g.clear();
        for (int f = 0; f < nf; ++f) {
            auto &B = pbufs[f];
            const int ns = B.ns, nc = B.nc;
            if (ns == 0) continue;
            GatherOp o = gop(B.Y, B.ldY, B.M3, B.ldM3, ns, ns);
            o.src_row_off = nc + ns;
            o.src_col_off = nc + ns;
            o.src_sym = 1;
            o.dst_lower = 1;
            o.accumulate = 1;
            g.push_back(o);
        }
        run_gathers(h, g, "E3d");
    }
    run_diag(h, idE3, "E3");
    if (!defl.empty()) {
        auto *dd = h->ar.upload("defl", defl, h->stream);
        launch_deflate(dd, (int)defl.size(), h->stream);
        check_launch(h);
    }
    PiDesc *dpis = nullptr;
    if (!pis.empty()) {
        // every PiDesc needs its W1 pointer, set below; upload after that, compress needs only M3/M3c
        dpis = h->ar.upload("pidesc", pis, h->stream);
        launch_pi_compress(dpis, (int)pis.size(), pi_nmax, h->stream);
        check_launch(h);
    }
    run_pchol_fp64class(h, dE3, "E3");
    for (auto &dd : dE3) cflop += pchol_flop(dd.n, dd.nstop);
    h->phase_flop[3] = cflop;
    {
        auto *dpw = h->ar.upload("pw", pw, h->stream);
        launch_pair_weights(dpw, (int)pw.size(), h->stream);
        check_launch(h);
    }
    phase_end(h, 3);
    phase_begin(h, 4);
    // Q = Dj S_i,ss Dj + Di S_j,ss Di ; W1 = Q X ; C = X^T W1 with X = R^-T at M3[2ns:3ns, ns:2ns]
    std::vector<GatherOp> gq1, gq2;
    std::vector<GemmDesc> gm1, gm2;
    std::vector<EigDesc> eds;
    std::vector<int> eig_face;
    for (int f = 0; f < nf; ++f) {
        auto &fp = h->faces[f];
        auto &B = pbufs[f];
        const int ns = B.ns;
        if (ns == 0) continue;
        if (B.pi >= 0 && B.nsp == 0) continue;  // the initial constraints fix every jump on s
        int ldq = round_up(ns, 8);
        B.Q = h->ar.get_t<double>("Q_" + std::to_string(f), (size_t)ldq * ns);
        B.W1 = h->ar.get_t<double>("W1_" + std::to_string(f), (size_t)ldq * ns);
        B.C = h->ar.get_t<double>("C_" + std::to_string(f), (size_t)ldq * ns);
        double *di = h->ar.get_t<double>("pwi_" + std::to_string(f), ns);
        double *dj = h->ar.get_t<double>("pwj_" + std::to_string(f), ns);
        int *pi = h->ar.get_t<int>("ppi_" + std::to_string(f), ns);
        int *pj = h->ar.get_t<int>("ppj_" + std::to_string(f), ns);
        GatherOp o = gop(h->subs[fp.i].S, h->subs[fp.i].ldS, B.Q, ldq, ns, ns);
        o.rmap = pi;
        o.cmap = pi;
        o.rscale = dj;
        o.cscale = dj;
        gq1.push_back(o);
        o = gop(h->subs[fp.j].S, h->subs[fp.j].ldS, B.Q, ldq, ns, ns);
        o.rmap = pj;
        o.cmap = pj;
        o.rscale = di;
        o.cscale = di;
        o.accumulate = 1;
        gq2.push_back(o);
        // order of the eigenproblem: ns, or nsp with initial constraints (X -> Xg = G X')
        const int ne = B.pi >= 0 ? B.nsp : ns;
        const double *X = B.pi >= 0 ? B.Xg : B.M3 + (size_t)ns * B.ldM3 + 2 * ns;
        const int ldx = B.pi >= 0 ? B.ldXg : B.ldM3;
        if (B.pi >= 0) {
            pis[B.pi].W1 = B.W1;
            pis[B.pi].ldw = ldq;
        }
        GemmDesc g1{B.Q, X, B.W1, ldq, ldx, ldq, ns, ne, ns, 0, 0, 1.0, 0.0};
        GemmDesc g2{X, B.W1, B.C, ldx, ldq, ldq, ne, ne, ns, 1, 0, 1.0, 0.0};
        gm1.push_back(g1);
        gm2.push_back(g2);
        int nface = (int)fp.face_idx.size();
        int *fpos = h->ar.upload("fpos_" + std::to_string(f), fp.face_idx, h->stream);
        EigDesc e{};
        e.C = B.C;
        e.n = ne;
        e.ld = ldq;
        e.W1 = B.W1;
        e.ldw = ldq;
        e.face_pos = fpos;
        e.nface = nface;
        e.lam = h->ar.get_t<double>("lam_all", (size_t)nf * (kEigCap + 1)) + (size_t)f * (kEigCap + 1);
        e.vec = h->ar.get_t<double>("vec_" + std::to_string(f), (size_t)kEigCap * ns);
        e.work = h->ar.get_t<double>("ework_" + std::to_string(f), (size_t)64 * ns + 16);
        e.rows = h->ar.get_t<double>("frows_" + std::to_string(f), (size_t)kEigCap * std::max(nface, 1));
        e.counts = h->ar.get_t<int>("fcnt_all", (size_t)nf * 8) + (size_t)f * 8;
        e.cap = kEigCap;
        eds.push_back(e);
        eig_face.push_back(f);
    }
    run_gathers(h, gq1, "Q1");
    run_gathers(h, gq2, "Q2");
    if (!pis.empty()) {
        // Xg = G X' for the constrained pairs (W1 pointers now set)
        dpis = h->ar.upload("pidesc", pis, h->stream);
        launch_pi_expand(dpis, (int)pis.size(), pi_nmax, h->stream);
        check_launch(h);
    }
    const bool ff_mode = h->opt.precision != BDDC_FP64;   // FP64-class products in double-float
    run_gemm(h, gm1, "W1", ff_mode);
    if (!pis.empty()) {
        // W1 <- P W1 (the face rows become P L P w); C = Xg^T W1 is unchanged by P
        launch_pi_project(dpis, (int)pis.size(), h->stream);
        check_launch(h);
    }
    run_gemm(h, gm2, "C", ff_mode);
    run_face_eigs(h, eds, tau, fixed_k, &h->lob_stats);
    {   // faces with more than kEigCap eigenvalues above tau: their matrix C formed again (the
        // first pass reduced it in place) and the dense path run once more with room for all
        std::vector<int> cnt0((size_t)nf * 8, 0);
        BDDC_CUDA(cudaMemcpyAsync(cnt0.data(), h->ar.get_t<int>("fcnt_all", (size_t)nf * 8), cnt0.size() * sizeof(int),
                                  cudaMemcpyDeviceToHost, h->stream));
        BDDC_CUDA(cudaStreamSynchronize(h->stream));
        std::vector<EigDesc> redo;
        std::vector<GemmDesc> gredo;
        for (size_t k = 0; k < eds.size(); ++k) {
            const int f = eig_face[k], over = cnt0[(size_t)f * 8 + 4];
            if (over <= 0) continue;
            EigDesc &e = eds[k];
            const int ns = pbufs[f].ns;
            e.cap = over;
            e.lam = h->ar.get_t<double>("lamx_" + std::to_string(f), (size_t)over + 1);
            e.vec = h->ar.get_t<double>("vec_" + std::to_string(f), (size_t)over * ns);
            e.rows = h->ar.get_t<double>("frows_" + std::to_string(f), (size_t)over * std::max(e.nface, 1));
            redo.push_back(e);
            gredo.push_back(gm2[k]);
        }
        if (!redo.empty()) {
            BDDC_REQUIRE(!h->keep_edge_rows, BDDC_EINVAL,
                         "kept edge rows allow at most 48 selected eigenvectors per face");
            run_gemm(h, gredo, "Cx", ff_mode);
            const int keep = h->opt.eig_large_n;
            h->opt.eig_large_n = -1;   // the dense path forms every selected pair
            run_face_eigs(h, redo, tau, fixed_k, nullptr);
            h->opt.eig_large_n = keep;
        }
    }
    // kept edge rows (Section 3: d split into a face row and one row per edge), per edge:
    // the edge parts of the same rows d from every face pair on the edge, stacked in the
    // edge's slots (pairs in face order), then one orthonormal basis per edge
    std::vector<int> eglob_ids, eglob_len; // edge globs with slots (ascending), their dofs
    int *ekept_dev = nullptr;
    if (h->keep_edge_rows && !eds.empty()) {
        std::vector<int> dof_edge(h->nfree, -1);
        for (size_t k = 0; k < h->edge_globs.size(); ++k)
            for (int64_t v : h->edge_globs[k].second)
                if (h->node_first[v] >= 0)
                    for (int comp = 0; comp < h->ncomp; ++comp) dof_edge[h->node_first[v] + comp] = (int)k;
        struct PairSegs {
            size_t k;                                  // index into eds
            std::vector<int> ptr, pos, eglob;
        };
        std::vector<PairSegs> ps;
        std::map<int, int> nslot;                      // edge glob -> slots (face pairs on it)
        std::map<int, int> elen;                       // edge glob -> dofs
        for (size_t k = 0; k < eds.size(); ++k) {
            const auto &fp = h->faces[eig_face[k]];
            const int ns = (int)fp.s_g.size();
            std::vector<char> on_face(ns, 0);
            for (int q : fp.face_idx) on_face[q] = 1;
            std::map<int, std::vector<int>> by_edge;   // edge glob -> s positions, ascending
            for (int q = 0; q < ns; ++q) {
                if (on_face[q]) continue;
                const int eg = dof_edge[fp.s_g[q]];
                BDDC_REQUIRE(eg >= 0, BDDC_EINVAL, "internal: a shared dof on no face and no edge");
                by_edge[eg].push_back(q);
            }
            if (by_edge.empty()) continue;
            PairSegs P;
            P.k = k;
            P.ptr.push_back(0);
            for (auto &kv : by_edge) {
                P.pos.insert(P.pos.end(), kv.second.begin(), kv.second.end());
                P.ptr.push_back((int)P.pos.size());
                P.eglob.push_back(kv.first);
                const int len = (int)kv.second.size();
                BDDC_REQUIRE(!elen.count(kv.first) || elen[kv.first] == len, BDDC_EINVAL,
                             "internal: an edge seen with different lengths by two face pairs");
                elen[kv.first] = len;
                ++nslot[kv.first];
            }
            ps.push_back(std::move(P));
        }
        if (!ps.empty()) {
            std::map<int, double *> stack;
            std::map<int, int> next_slot;
            std::vector<EdgeGlobDesc> egd;
            ekept_dev = h->ar.get_t<int>("ekept_all", nslot.size());
            for (auto &kv : nslot) {
                const int eg = kv.first, len = elen[eg];
                BDDC_REQUIRE(kv.second <= kMaxEdgeSlots, BDDC_EINVAL,
                             "an edge shared by more than 8 face pairs (kept edge rows)");
                const std::string tag = std::to_string(eg);
                stack[eg] = h->ar.get_t<double>("estack_" + tag, (size_t)kv.second * kEigCap * len);
                next_slot[eg] = 0;
                EdgeGlobDesc g{};
                g.R = stack[eg];
                g.nrows = kv.second * kEigCap;
                g.len = len;
                g.rowsT = h->ar.get_t<double>("erowsT_" + tag, (size_t)len * len);
                g.kept = ekept_dev + egd.size();
                egd.push_back(g);
                eglob_ids.push_back(eg);
                eglob_len.push_back(len);
            }
            std::vector<EdgePartDesc> epd;
            for (auto &P : ps) {
                const auto &ed = eds[P.k];
                const std::string tag = std::to_string(eig_face[P.k]);
                std::vector<double *> slots;
                for (size_t e = 0; e < P.eglob.size(); ++e) {
                    const int eg = P.eglob[e];
                    slots.push_back(stack[eg] + (size_t)(next_slot[eg]++) * kEigCap * elen[eg]);
                }
                EdgePartDesc d{};
                d.W1 = ed.W1;
                d.ldw = ed.ldw;
                d.ns = (int)h->faces[eig_face[P.k]].s_g.size();
                d.n = ed.n;
                d.vec = ed.vec;
                d.counts = ed.counts;
                d.seg_ptr = h->ar.upload("eseg_ptr_" + tag, P.ptr, h->stream);
                d.seg_pos = h->ar.upload("eseg_pos_" + tag, P.pos, h->stream);
                d.nseg = (int)P.eglob.size();
                d.slot = h->ar.upload("eslot_" + tag, slots, h->stream);
                epd.push_back(d);
            }
            auto *dp = h->ar.upload("edgepartdesc", epd, h->stream);
            launch_edge_parts(dp, (int)epd.size(), h->opt.drop_rel, h->stream);
            check_launch(h);
            auto *dg = h->ar.upload("edgeglobdesc", egd, h->stream);
            // the rows of the pairs on one edge overlap in exact arithmetic.  The FP64 path keeps
            // the rank rule of the face rows (drop_rel).  The mixed modes' eigenvectors carry
            // rounding directions of ~1e-8 relative (double-float reduction), which that rule
            // would keep as rows; they keep pivots above 1e-6 of the first only
            const double edge_drop = h->opt.precision == BDDC_FP64 || h->fp64_class_forced
                                         ? h->opt.drop_rel : std::max(h->opt.drop_rel, 1e-6);
            launch_edge_globs(dg, (int)egd.size(), edge_drop, h->stream);
            check_launch(h);
        }
    }
    phase_end(h, 4);
    fail_check(h, "adapt");
    // results back to the host
    int n_added = 0, n_ties = 0;
    double omega = 0.0;
    h->face_rows_dev.assign(nf, nullptr);
    std::vector<int> cnt_all((size_t)nf * 8, 0);
    std::vector<double> lam_all((size_t)nf * (kEigCap + 1), 0.0);
    std::vector<int> ekept(eglob_ids.size(), 0);
    if (!eds.empty()) {
        BDDC_CUDA(cudaMemcpyAsync(cnt_all.data(), h->ar.get_t<int>("fcnt_all", (size_t)nf * 8), cnt_all.size() * sizeof(int),
                                  cudaMemcpyDeviceToHost, h->stream));
        BDDC_CUDA(cudaMemcpyAsync(lam_all.data(), h->ar.get_t<double>("lam_all", (size_t)nf * (kEigCap + 1)),
                                  lam_all.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        if (ekept_dev)
            BDDC_CUDA(cudaMemcpyAsync(ekept.data(), ekept_dev, ekept.size() * sizeof(int), cudaMemcpyDeviceToHost,
                                      h->stream));
        BDDC_CUDA(cudaStreamSynchronize(h->stream));
    }
    for (size_t k = 0; k < eds.size(); ++k) {
        int f = eig_face[k];
        auto &fp = h->faces[f];
        const int *cnt = &cnt_all[(size_t)f * 8];
        std::vector<double> lam;
        if (eds[k].cap > kEigCap) {   // a face redone with a larger capacity
            lam.resize(cnt[2]);
            if (cnt[2] > 0)
                BDDC_CUDA(cudaMemcpy(lam.data(), eds[k].lam, cnt[2] * sizeof(double), cudaMemcpyDeviceToHost));
        } else {
            lam.assign(lam_all.begin() + (size_t)f * (kEigCap + 1), lam_all.begin() + (size_t)(f + 1) * (kEigCap + 1));
            lam.resize(cnt[2]);
        }
        fp.nsel = cnt[0];
        fp.nkept = cnt[1];
        fp.ties = cnt[3];
        fp.lam = lam;
        if (!lam.empty()) omega = std::max(omega, lam[0]);
        n_added += fp.nkept;
        n_ties += fp.ties;
        BDDC_REQUIRE(cnt[4] == 0, BDDC_ECUDA, "internal: a face's eigenpairs exceed its capacity");
        h->face_rows_dev[f] = eds[k].rows;
        if (fp.nkept > 0) {
            GlobRows g;
            g.subs = {fp.i, fp.j};
            for (int idx : fp.face_idx) g.gdofs.push_back(fp.s_g[idx]);
            g.nrows = fp.nkept;
            g.face = f;
            h->globs.push_back(g);
        }
    }
    // kept edge rows: one glob constraint per edge, on all substructures of the edge
    for (size_t q = 0; q < eglob_ids.size(); ++q) {
        if (ekept[q] <= 0) continue;
        const int eg = eglob_ids[q];
        const auto &E = h->edge_globs[eg];
        GlobRows g;
        g.subs = E.first;
        for (int64_t v : E.second)
            if (h->node_first[v] >= 0)
                for (int comp = 0; comp < h->ncomp; ++comp) g.gdofs.push_back(h->node_first[v] + comp);
        BDDC_REQUIRE((int)g.gdofs.size() == eglob_len[q] && ekept[q] <= eglob_len[q], BDDC_EINVAL,
                     "internal: an edge's rows do not match its dofs");
        g.nrows = ekept[q];
        g.edge = (int)h->edge_rows.size();
        h->edge_rows.push_back({eg, h->ar.get_t<double>("erowsT_" + std::to_string(eg), g.gdofs.size() * g.gdofs.size()),
                                (int)g.gdofs.size(), ekept[q]});
        h->n_edge_rows += ekept[q];
        ++h->n_edges_with_rows;
        h->globs.push_back(g);
    }
    h->omega = omega;
    // rows are stored row-major (l * nf + f); the constraint gather reads src(l, cmap[k]) = src[cmap[k] * ld + l]
    // which needs the transpose: rows[f * kEigCap + l].  Transpose on the device via a gather.
    {
        std::vector<GatherOp> gt;
        for (size_t k = 0; k < eds.size(); ++k) {
            int f = eig_face[k];
            auto &fp = h->faces[f];
            if (fp.nkept == 0) continue;
            int nface = (int)fp.face_idx.size();
            double *T = h->ar.get_t<double>("frowsT_" + std::to_string(f), (size_t)nface * fp.nkept);
            // T(l, f) = rows[l * nface + f]: read with ld_src = 1 and row map l -> l * nface
            GatherOp o = gop(eds[k].rows, 1, T, fp.nkept, fp.nkept, nface);
            std::vector<int> rm(fp.nkept);
            for (int l = 0; l < fp.nkept; ++l) rm[l] = l * nface;
            int *drm = h->ar.upload("frT_rm_" + std::to_string(f), rm, h->stream);
            o.rmap = drm;
            gt.push_back(o);
            h->face_rows_dev[f] = T;
        }
        run_gathers(h, gt, "frT");
    }
    // rebuild the preconditioner with the new constraints
    {
        const int ns = h->nsub;
        std::vector<int> na(ns, 0);
        for (auto &g : h->globs)
            for (int s : g.subs) na[s] += g.nrows;
        for (int s = 0; s < ns; ++s) h->subs[s].na = na[s];
        set_phi_pointers(h);
    }
    count_coarse(h);
    h->coarse_dirty = true;
    phase_collect(h, 3, 4);
    if (info) {
        info->n_faces = nf;
        info->n_added = n_added;
        info->n_ties = n_ties;
        info->omega = omega;
        info->n_lobpcg = h->lob_stats.faces;
        info->lobpcg_iters = h->lob_stats.iters;
        info->n_dense_fallback = h->lob_stats.fallback;
    }
}

// ===========================================================================
void do_solve(bddc_handle *h, const double *f, double *u, int mem, bddc_solve_info *info) {
    const int ns = h->nsub;
    reset_status(h);
    ensure_coarse(h);
    double *df = h->ar.get_t<double>("f", std::max<int64_t>(h->nfree, 1));
    phase_begin(h, 6);
    if (mem == BDDC_MEM_DEVICE)
        BDDC_CUDA(cudaMemcpyAsync(df, f, h->nfree * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    else
        BDDC_CUDA(cudaMemcpyAsync(df, f, h->nfree * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    double *yI = h->ar.get_t<double>("yI", std::max<int64_t>(h->sumI, 1));
    double *gl = h->ar.get_t<double>("gl", std::max<int64_t>(h->sumG, 1));
    const int64_t *gIall = h->ar.get_t<int64_t>("gIall", std::max<int64_t>(h->sumI, 1));
    const int64_t *gGall = h->ar.get_t<int64_t>("gGall", std::max<int64_t>(h->sumG, 1));
    launch_gatherv(yI, gIall, df, h->sumI, h->stream);
    check_launch(h);
    (void)gGall;
    const bool mixed = h->interior_fp32;
    // mixed: y = A_II^{-1} f_I by refinement (yI keeps f_I), g_i = -A_GI y (sparse)
    double *yx = h->ar.get_t<double>("yIx", std::max<int64_t>(h->sumI, 1));
    double *yr = h->ar.get_t<double>("yIr", std::max<int64_t>(h->sumI, 1));
    std::vector<TrsvDesc<double>> tv;
    std::vector<GemmDesc> gm;
    std::vector<RefineJob> rj;
    std::vector<EllProduct> gp;
    for (int s = 0; s < ns; ++s) {
        auto &sd = h->subs[s];
        if (sd.nI == 0) continue;
        if (mixed) {
            rj.push_back(RefineJob{s, yI + sd.offI, sd.nI, yx + sd.offI, sd.nI, yr + sd.offI, sd.nI, 1});
            EllProduct p = ell_of(h, s);
            p.r0 = sd.nI;
            p.m = sd.nG;
            p.ncol = 1;
            p.X = yx + sd.offI;
            p.ldx = sd.nI;
            p.B = nullptr;
            p.ldb = 1;
            p.out = gl + h->offG[s];
            p.ldo = std::max(sd.nG, 1);
            gp.push_back(p);
            continue;
        }
        tv.push_back(TrsvDesc<double>{sd.A, yI + sd.offI, sd.nI, sd.ld});
        // g_i = -L21 y = -A_GI A_II^{-1} f_I  (f_G is added once after assembly)
        gm.push_back(GemmDesc{sd.A + sd.nI, yI + sd.offI, gl + h->offG[s], sd.ld, std::max(sd.nI, 1), std::max(sd.nG, 1),
                              sd.nG, 1, sd.nI, 0, 0, -1.0, 0.0});
    }
    auto *dtv = h->ar.upload("trsv", tv, h->stream);
    zero(h, gl, h->sumG);
    if (mixed) {
        refine(h, rj, 2 * h->mixed_iters + 1, 64, 0.0, false, "y");
        run_ell(h, gp, "g");
    } else {
        launch_trsv<double>(dtv, (int)tv.size(), 0, h->stream);
        check_launch(h);
        run_gemv(h, gm, "cond");
    }
    launch_iface_assemble(h->ops, gl, h->pb.r, h->stream);
    check_launch(h);
    // g = f_G - sum_i R_i^T A_GI A_II^{-1} f_I
    launch_gatherv_add(h->pb.r, h->ar.get_t<int64_t>("ifgdof", std::max(h->nG, 1)), df, h->nG, h->stream);
    check_launch(h);
    phase_end(h, 6);
    phase_begin(h, 7);
    // the condensed right-hand side g, kept for the true residual after PCG
    double *gsave = h->ar.get_t<double>("g_save", std::max(h->nG, 1));
    double *nrm2 = h->ar.get_t<double>("relres_nrm2", 2);
    BDDC_CUDA(cudaMemcpyAsync(gsave, h->pb.r, h->nG * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    int nblocks = 0;
    const long tok_pcg = kt_begin(h);
    cudaError_t e = launch_pcg(h->ops, h->pb, PCG_SOLVE, h->opt.tol, h->opt.maxit, h->dst, h->opt.timeout_s,
                               h->stream, &nblocks);
    BDDC_REQUIRE(e == cudaSuccess, BDDC_ECUDA, std::string("PCG launch: ") + cudaGetErrorString(e));
    h->launches++;
    kt_end(h, tok_pcg, KT_PCG, 0.0);
    // true residual ||g - S u_G|| / ||g||: one more application of the local S_i
    BDDC_CUDA(cudaMemcpyAsync(h->pb.z, h->pb.x, h->nG * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    e = launch_pcg(h->ops, h->pb, PCG_APPLY_S, h->opt.tol, h->opt.maxit, h->dst, h->opt.timeout_s, h->stream,
                   &nblocks);
    BDDC_REQUIRE(e == cudaSuccess, BDDC_ECUDA, std::string("residual launch: ") + cudaGetErrorString(e));
    h->launches++;
    launch_residual_norms2(gsave, h->pb.q, h->nG, nrm2, h->stream);
    check_launch(h);
    phase_end(h, 7);
    phase_begin(h, 8);
    // recovery: t = y - L21^T u_G ; u_I = L11^-T t
    double *ug = h->ar.get_t<double>("ugl", std::max<int64_t>(h->sumG, 1));
    const int64_t *RGall = h->ar.get_t<int64_t>("RG64", std::max<int64_t>(h->sumG, 1));
    launch_gatherv(ug, RGall, h->pb.x, h->sumG, h->stream);
    check_launch(h);
    std::vector<GemmDesc> gr;
    for (int s = 0; s < ns; ++s) {
        auto &sd = h->subs[s];
        if (sd.nI == 0 || sd.nG == 0) continue;
        if (mixed)  // b = f_I - A_IG u_G (dense FP64 block of the unfactored A_i), in yI
            gr.push_back(GemmDesc{sd.A + (size_t)sd.nI * sd.ld, ug + h->offG[s], yI + sd.offI, sd.ld, std::max(sd.nG, 1),
                                  std::max(sd.nI, 1), sd.nI, 1, sd.nG, 0, 0, -1.0, 1.0});
        else
            gr.push_back(GemmDesc{sd.A + sd.nI, ug + h->offG[s], yI + sd.offI, sd.ld, std::max(sd.nG, 1),
                                  std::max(sd.nI, 1), sd.nI, 1, sd.nG, 1, 0, -1.0, 1.0});
    }
    run_gemv(h, gr, "rec");
    double *uI = yI;
    if (mixed) {
        refine(h, rj, 2 * h->mixed_iters + 1, 64, 0.0, false, "u");  // u_I = A_II^{-1} b, in yIx
        uI = yx;
    } else {
        launch_trsv<double>(dtv, (int)tv.size(), 1, h->stream);
        check_launch(h);
    }
    double *du = h->ar.get_t<double>("u", std::max<int64_t>(h->nfree, 1));
    launch_scatter(du, gIall, uI, h->sumI, h->stream);
    check_launch(h);
    const int64_t *ifg = h->ar.get_t<int64_t>("ifgdof", std::max(h->nG, 1));
    launch_scatter(du, ifg, h->pb.x, h->nG, h->stream);
    check_launch(h);
    phase_end(h, 8);
    if (mem == BDDC_MEM_DEVICE)
        BDDC_CUDA(cudaMemcpyAsync(u, du, h->nfree * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    else
        BDDC_CUDA(cudaMemcpyAsync(u, du, h->nfree * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    int it[2];
    double rr, tr[2];
    BDDC_CUDA(cudaMemcpyAsync(it, h->pb.iters, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    BDDC_CUDA(cudaMemcpyAsync(&rr, h->pb.relres, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    BDDC_CUDA(cudaMemcpyAsync(tr, h->ar.get_t<double>("relres_nrm2", 2), 2 * sizeof(double), cudaMemcpyDeviceToHost,
                              h->stream));
    BDDC_CUDA(cudaStreamSynchronize(h->stream));
    fail_check(h, "solve");
    // A non-finite load makes the condensed right-hand side non-finite: PCG then stops at once
    // (p^T S p is not positive), and the residual ratios would read 0.  Report it as a bad argument.
    if (!std::isfinite(tr[1]))
        throw Error{BDDC_EINVAL, "the load vector has non-finite entries (condensed right-hand side norm " +
                                     std::to_string(tr[1]) + ")"};
    phase_collect(h, 6, 8);
    h->last_iters = it[0];
    h->alpha.assign(it[0], 0.0);
    h->beta.assign(std::max(it[0] - 1, 0), 0.0);
    if (it[0] > 0) BDDC_CUDA(cudaMemcpy(h->alpha.data(), h->pb.alpha, it[0] * sizeof(double), cudaMemcpyDeviceToHost));
    if (it[0] > 1) BDDC_CUDA(cudaMemcpy(h->beta.data(), h->pb.beta, (it[0] - 1) * sizeof(double), cudaMemcpyDeviceToHost));
    if (info) {
        info->iters = it[0];
        info->converged = it[1];
        info->relres = tr[1] > 0.0 ? std::sqrt(tr[0] / tr[1]) : 0.0;
        info->relres_recurrence = rr;
        double lmin = 1, lmax = 1;
        bddc_condition_estimate(h, &lmin, &lmax);
        info->kappa = lmax / lmin;
        info->setup_ms = h->phase_ms[0] + h->phase_ms[1] + h->phase_ms[2] + h->phase_ms[3] + h->phase_ms[4] +
                         h->phase_ms[5];
        info->solve_ms = h->phase_ms[6] + h->phase_ms[7] + h->phase_ms[8];
        info->interior_fp32 = h->interior_fp32 ? 1 : 0;
        info->coarse_fp32 = h->coarse_fp32 ? 1 : 0;
        info->refine_steps = h->interior_fp32 ? h->mixed_iters : 0;
        info->refine_relres = h->interior_fp32 ? h->mixed_relres : 0.0;
    }
    if (!it[1]) throw Error{BDDC_ENOCONV, "PCG did not reach the tolerance within maxit"};
}

}  // namespace

// ===========================================================================
// C ABI
extern "C" {

void bddc_default_options(bddc_options *opt) {
    if (!opt) return;
    opt->precision = BDDC_FP64;
    opt->tol = 1e-8;
    opt->maxit = 1000;
    opt->drop_rel = 1e-10;
    opt->timeout_s = 10.0;
    opt->stream = nullptr;
    opt->dev_alloc = nullptr;
    opt->dev_free = nullptr;
    opt->alloc_ctx = nullptr;
    opt->refine_tol = 1e-8;
    opt->eig_large_n = -1;
    opt->eig_tol = 1e-8;
    opt->eig_maxit = 240;
    opt->mixed_updates = 0;
}

const char *bddc_status_str(bddc_status s) {
    switch (s) {
        case BDDC_OK: return "ok";
        case BDDC_EINVAL: return "invalid argument";
        case BDDC_ENOMEM: return "out of memory";
        case BDDC_ENOTSPD: return "matrix not positive definite";
        case BDDC_EASSUMPTION: return "too few corners (Assumption 1 or 2)";
        case BDDC_ENOCONV: return "PCG did not converge";
        case BDDC_ETIMEOUT: return "device wait timed out";
        case BDDC_ECUDA: return "CUDA error";
        case BDDC_ESTATE: return "call out of order";
    }
    return "unknown status";
}

const char *bddc_last_error(const bddc_handle *h) { return h ? h->err.c_str() : "null handle"; }

#define BDDC_TRY(h, ...)                                    \
    try {                                                   \
        __VA_ARGS__;                                        \
        (h)->err.clear();                                   \
        return BDDC_OK;                                     \
    } catch (const Error &e_) {                             \
        (h)->err = e_.msg;                                  \
        return (bddc_status)e_.status;                      \
    } catch (const std::exception &e_) {                    \
        (h)->err = e_.what();                               \
        return BDDC_EINVAL;                                 \
    }

bddc_status bddc_create(const bddc_options *opt, bddc_handle **out) {
    if (!out) return BDDC_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return BDDC_ECUDA;
    bddc_handle *h = new (std::nothrow) bddc_handle();
    if (!h) return BDDC_ENOMEM;
    if (opt)
        h->opt = *opt;
    else
        bddc_default_options(&h->opt);
    h->stream = (cudaStream_t)h->opt.stream;
    if ((h->opt.dev_alloc == nullptr) != (h->opt.dev_free == nullptr)) {
        delete h;
        return BDDC_EINVAL;
    }
    h->ar.set_allocator(h->opt.dev_alloc, h->opt.dev_free, h->opt.alloc_ctx, h->stream);
    try {
        h->dst = h->ar.get_t<DevStatus>("status", 1);
    } catch (const Error &) {
        delete h;
        return BDDC_ENOMEM;
    }
    if (cudaMemsetAsync(h->dst, 0, sizeof(DevStatus), h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
        delete h;
        return BDDC_ECUDA;
    }
    for (auto &e : h->ev) {
        if (cudaEventCreate(&e) != cudaSuccess) {
            delete h;
            return BDDC_ECUDA;
        }
    }
    *out = h;
    return BDDC_OK;
}

void bddc_destroy(bddc_handle *h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    h->ar.release();
    for (auto &e : h->ev)
        if (e) cudaEventDestroy(e);
    for (auto &e : h->kev) cudaEventDestroy(e);
    delete h;
}

// Classification, index maps, device copies of the input and solver buffers;
// shared by bddc_set_mesh_q1, bddc_set_problem, bddc_set_corners and
// bddc_select_corners.  Constraints are reset to corners only.
void analyze(bddc_handle *h, std::chrono::steady_clock::time_point t_host0) {
    h->have_mesh = h->have_setup = false;
    h->assembled = h->factored = false;
    h->coarse_dirty = true;
    if (h->xyz.size() < (size_t)h->nn * 3) h->xyz.assign((size_t)h->nn * 3, 0.0);
    classify(h);
    const auto t_class = std::chrono::steady_clock::now();
    for (auto &sd : h->subs) BDDC_REQUIRE(sd.n > 0, BDDC_EINVAL, "substructure without free dofs");
    h->avg_flags = 0;
    if (h->csr_mode) {
        // merged CSR entries with their dense offsets (column-major, [interior; interface])
        const int ns = h->nsub;
        std::vector<int64_t> start(ns + 1, 0), off;
        std::vector<double> val;
        std::vector<int32_t> lp(h->nfree, -1);
        std::vector<std::pair<int64_t, double>> ent;
        for (int s = 0; s < ns; ++s) {
            const auto &sd = h->subs[s];
            for (int k = 0; k < sd.nI; ++k) lp[sd.gI[k]] = k;
            for (int k = 0; k < sd.nG; ++k) lp[sd.gG[k]] = sd.nI + k;
            const auto &l2g = h->csr_l2g[s];
            const auto &rp = h->csr_rowptr[s];
            const auto &cl = h->csr_col[s];
            const auto &vl = h->csr_val[s];
            ent.clear();
            ent.reserve(vl.size());
            for (size_t r = 0; r < l2g.size(); ++r) {
                const int64_t pr = lp[l2g[r]];
                BDDC_REQUIRE(pr >= 0, BDDC_EINVAL, "internal: CSR row outside the substructure's dofs");
                for (int64_t q = rp[r]; q < rp[r + 1]; ++q) {
                    const int64_t pc = lp[l2g[cl[q]]];
                    BDDC_REQUIRE(pc >= 0, BDDC_EINVAL, "internal: CSR column outside the substructure's dofs");
                    ent.push_back({pc * sd.ld + pr, vl[q]});
                }
            }
            std::sort(ent.begin(), ent.end(),
                      [](const std::pair<int64_t, double> &x, const std::pair<int64_t, double> &y) { return x.first < y.first; });
            for (size_t q = 0; q < ent.size(); ++q) {
                if (q > 0 && ent[q].first == ent[q - 1].first)
                    val.back() += ent[q].second;
                else {
                    off.push_back(ent[q].first);
                    val.push_back(ent[q].second);
                }
            }
            start[s + 1] = (int64_t)off.size();
            for (int k = 0; k < sd.nI; ++k) lp[sd.gI[k]] = -1;
            for (int k = 0; k < sd.nG; ++k) lp[sd.gG[k]] = -1;
        }
        h->csr_nnz = (int64_t)off.size();
        h->ar.upload("csr_start", start, h->stream);
        h->ar.upload("csr_off", off, h->stream);
        h->ar.upload("csr_val", val, h->stream);
    } else {
        if (!h->mesh_uploaded) {
            if (h->in_xyz) {   // device-resident input: device-to-device copies, no host round trip
                auto d2d = [&](const std::string &name, const void *src, size_t bytes) {
                    BDDC_CUDA(cudaMemcpyAsync(h->ar.get(name, bytes), src, bytes, cudaMemcpyDeviceToDevice, h->stream));
                };
                d2d("xyz", h->in_xyz, (size_t)h->nn * 3 * sizeof(double));
                d2d("elems", h->in_elems, (size_t)h->ne * 8 * sizeof(int64_t));
                d2d("coef", h->in_coef, (size_t)h->ne * sizeof(double));
                d2d("esub", h->in_esub, (size_t)h->ne * sizeof(int32_t));
            } else {
                h->ar.upload("xyz", h->xyz, h->stream);
                h->ar.upload("elems", h->elems, h->stream);
                h->ar.upload("coef", h->coef, h->stream);
                h->ar.upload("esub", h->esub, h->stream);
            }
            h->mesh_uploaded = true;
        }
        h->ar.upload("epos", h->epos, h->stream);
        for (size_t col = 0; col < h->colors.size(); ++col)
            h->ar.upload("color_" + std::to_string(col), h->colors[col], h->stream);
    }
    std::vector<int64_t> gIall, gGall, RG64;
    for (auto &sd : h->subs) {
        gIall.insert(gIall.end(), sd.gI.begin(), sd.gI.end());
        gGall.insert(gGall.end(), sd.gG.begin(), sd.gG.end());
        for (int x : sd.RG) RG64.push_back(x);
    }
    h->ar.upload("gIall", gIall, h->stream);
    h->ar.upload("gGall", gGall, h->stream);
    h->ar.upload("RG64", RG64, h->stream);
    h->ar.upload("ifgdof", h->iface_gdof, h->stream);
    const auto t_up = std::chrono::steady_clock::now();
    alloc_solver_buffers(h);
    BDDC_CUDA(cudaStreamSynchronize(h->stream));
    const auto t_end = std::chrono::steady_clock::now();
    h->phase_ms[5] = std::chrono::duration<double, std::milli>(t_end - t_host0).count();
    if (getenv("BDDC_DEBUG_TIMING")) {
        auto ms = [](auto a, auto b) { return std::chrono::duration<double, std::milli>(b - a).count(); };
        fprintf(stderr, "analysis: input+classify %.3f uploads %.3f buffers %.3f ms\n", ms(t_host0, t_class),
                ms(t_class, t_up), ms(t_up, t_end));
    }
    h->have_mesh = true;
}

bddc_status bddc_set_mesh_q1(bddc_handle *h, int ncomp, int64_t nn, const double *xyz, int64_t ne,
                             const int64_t *elems, const double *coef, double nu, const int32_t *elem_sub,
                             int32_t nsub, const uint8_t *dirichlet, int mem) {
    if (!h) return BDDC_EINVAL;
    BDDC_TRY(h, {
        BDDC_REQUIRE(ncomp == 1 || ncomp == 3, BDDC_EINVAL, "ncomp must be 1 or 3");
        BDDC_REQUIRE(nn > 0 && ne > 0 && nsub > 0, BDDC_EINVAL, "empty mesh");
        BDDC_REQUIRE(xyz && elems && coef && elem_sub && dirichlet, BDDC_EINVAL, "null array");
        const auto t_host0 = std::chrono::steady_clock::now();
        h->have_mesh = h->have_setup = false;
        h->assembled = h->factored = false;
        h->ncomp = ncomp;
        h->nn = nn;
        h->ne = ne;
        h->nsub = nsub;
        h->nu = nu;
        h->xyz.resize(nn * 3);
        h->elems.resize(ne * 8);
        h->esub.resize(ne);
        h->dirich.resize(nn);
        auto cp = [&](void *dst, const void *src, size_t bytes) {
            BDDC_CUDA(cudaMemcpy(dst, src, bytes, mem == BDDC_MEM_DEVICE ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
        };
        cp(h->xyz.data(), xyz, nn * 3 * sizeof(double));
        cp(h->elems.data(), elems, ne * 8 * sizeof(int64_t));
        cp(h->esub.data(), elem_sub, ne * sizeof(int32_t));
        cp(h->dirich.data(), dirichlet, nn);
        // the coefficients are only needed on the device; device-resident arrays are
        // copied device to device by the analysis (the pointers are valid during this call)
        h->mesh_uploaded = false;
        if (mem == BDDC_MEM_DEVICE) {
            h->coef.clear();
            h->in_xyz = xyz;
            h->in_elems = elems;
            h->in_coef = coef;
            h->in_esub = elem_sub;
        } else {
            h->coef.assign(coef, coef + ne);
            h->in_xyz = h->in_coef = nullptr;
            h->in_elems = nullptr;
            h->in_esub = nullptr;
        }
        struct InputReset {
            bddc_handle *h;
            ~InputReset() {
                h->in_xyz = h->in_coef = nullptr;
                h->in_elems = nullptr;
                h->in_esub = nullptr;
            }
        } input_reset{h};
        for (int64_t k = 0; k < ne * 8; ++k)
            BDDC_REQUIRE(h->elems[k] >= 0 && h->elems[k] < nn, BDDC_EINVAL, "element node id out of range");
        for (int64_t e = 0; e < ne; ++e)
            BDDC_REQUIRE(h->esub[e] >= 0 && h->esub[e] < nsub, BDDC_EINVAL, "substructure id out of range");
        h->csr_mode = false;
        h->user_corners = false;
        h->corner_list.clear();
        h->csr_l2g.clear();
        h->csr_rowptr.clear();
        h->csr_col.clear();
        h->csr_val.clear();
        analyze(h, t_host0);
    });
}

bddc_status bddc_classify_q1(int ncomp, int64_t nn, const double *xyz, int64_t ne, const int64_t *elems,
                             const int32_t *elem_sub, int32_t nsub, const uint8_t *dirichlet, int64_t *n_free,
                             int64_t *n_interface, int *n_corners, int *n_edges, int *n_faces, int *n_augmented,
                             int64_t *corners, int corners_cap) {
    if (ncomp != 1 && ncomp != 3) return BDDC_EINVAL;
    if (nn <= 0 || ne <= 0 || nsub <= 0 || !xyz || !elems || !elem_sub || !dirichlet) return BDDC_EINVAL;
    if (corners_cap > 0 && !corners) return BDDC_EINVAL;
    try {
        // a handle that never touches the device: only the host mesh fields are set
        std::unique_ptr<bddc_handle> hp(new bddc_handle());
        bddc_handle *h = hp.get();
        h->ncomp = ncomp;
        h->nn = nn;
        h->ne = ne;
        h->nsub = nsub;
        h->xyz.assign(xyz, xyz + nn * 3);
        h->elems.assign(elems, elems + ne * 8);
        h->esub.assign(elem_sub, elem_sub + ne);
        h->dirich.assign(dirichlet, dirichlet + nn);
        for (int64_t k = 0; k < ne * 8; ++k)
            if (h->elems[k] < 0 || h->elems[k] >= nn) return BDDC_EINVAL;
        for (int64_t e = 0; e < ne; ++e)
            if (h->esub[e] < 0 || h->esub[e] >= nsub) return BDDC_EINVAL;
        h->csr_mode = false;
        h->user_corners = false;
        classify(h);
        for (auto &sd : h->subs)
            if (sd.n <= 0) return BDDC_EINVAL;
        if (n_free) *n_free = h->nfree;
        if (n_interface) *n_interface = h->nG;
        if (n_corners) *n_corners = (int)h->corners.size();
        if (n_edges) *n_edges = h->n_edges;
        if (n_faces) *n_faces = (int)h->faces.size();
        if (n_augmented) *n_augmented = h->n_augmented;
        for (int k = 0; k < corners_cap && k < (int)h->corners.size(); ++k) corners[k] = h->corners[k];
    } catch (const Error &e) {
        return (bddc_status)e.status;
    } catch (const std::bad_alloc &) {
        return BDDC_ENOMEM;
    }
    return BDDC_OK;
}

bddc_status bddc_set_problem(bddc_handle *h, int64_t n_global, int ncomp, int32_t n_sub, const bddc_subdomain *subs,
                             const double *node_xyz, int mem) {
    if (!h) return BDDC_EINVAL;
    BDDC_TRY(h, {
        BDDC_REQUIRE(ncomp == 1 || ncomp == 3, BDDC_EINVAL, "ncomp must be 1 or 3");
        BDDC_REQUIRE(n_global > 0 && n_sub > 0 && subs, BDDC_EINVAL, "empty problem");
        BDDC_REQUIRE(n_global % ncomp == 0, BDDC_EINVAL, "n_global must be a multiple of ncomp");
        BDDC_REQUIRE(ncomp == 1 || node_xyz, BDDC_EINVAL, "node_xyz is required for ncomp = 3 (rigid body modes)");
        const auto t_host0 = std::chrono::steady_clock::now();
        const int64_t nn = n_global / ncomp;
        auto cp = [&](void *dst, const void *src, size_t bytes) {
            if (bytes == 0) return;
            BDDC_REQUIRE(src, BDDC_EINVAL, "null array");
            BDDC_CUDA(cudaMemcpy(dst, src, bytes, mem == BDDC_MEM_DEVICE ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
        };
        std::vector<std::vector<int64_t>> l2g(n_sub), rowptr(n_sub);
        std::vector<std::vector<int32_t>> col(n_sub);
        std::vector<std::vector<double>> val(n_sub);
        std::vector<int32_t> owner(nn, -1);
        for (int s = 0; s < n_sub; ++s) {
            const bddc_subdomain &d = subs[s];
            BDDC_REQUIRE(d.n_local > 0, BDDC_EINVAL, "substructure " + std::to_string(s) + " has no dofs");
            const int n = d.n_local;
            l2g[s].resize(n);
            rowptr[s].resize(n + 1);
            cp(l2g[s].data(), d.l2g, n * sizeof(int64_t));
            cp(rowptr[s].data(), d.rowptr, (n + 1) * sizeof(int64_t));
            const int64_t nnz = rowptr[s][n];
            BDDC_REQUIRE(rowptr[s][0] == 0 && nnz >= 0, BDDC_EINVAL, "bad rowptr of substructure " + std::to_string(s));
            for (int r = 0; r < n; ++r)
                BDDC_REQUIRE(rowptr[s][r + 1] >= rowptr[s][r], BDDC_EINVAL, "rowptr not monotone");
            col[s].resize(nnz);
            val[s].resize(nnz);
            cp(col[s].data(), d.col, nnz * sizeof(int32_t));
            cp(val[s].data(), d.val, nnz * sizeof(double));
            for (int32_t q : col[s]) BDDC_REQUIRE(q >= 0 && q < n, BDDC_EINVAL, "column index out of range");
            // every node of the substructure complete, each global dof once
            std::vector<int64_t> sorted = l2g[s];
            std::sort(sorted.begin(), sorted.end());
            for (size_t k = 0; k < sorted.size(); ++k) {
                BDDC_REQUIRE(sorted[k] >= 0 && sorted[k] < n_global, BDDC_EINVAL, "l2g entry out of range");
                BDDC_REQUIRE(k == 0 || sorted[k] != sorted[k - 1], BDDC_EINVAL, "l2g repeats a global dof");
            }
            BDDC_REQUIRE(sorted.size() % ncomp == 0, BDDC_EINVAL, "a node is split between substructures");
            for (size_t k = 0; k < sorted.size(); k += ncomp)
                BDDC_REQUIRE(sorted[k] % ncomp == 0 && sorted[k + ncomp - 1] == sorted[k] + ncomp - 1, BDDC_EINVAL,
                             "substructure " + std::to_string(s) + " holds only some dofs of a node");
        }
        h->csr_mode = true;
        h->user_corners = false;
        h->corner_list.clear();
        h->ncomp = ncomp;
        h->nn = nn;
        h->ne = 0;
        h->nsub = n_sub;
        h->nu = 0.0;
        h->elems.clear();
        h->coef.clear();
        h->esub.clear();
        h->dirich.assign(nn, 0);
        h->xyz.assign((size_t)nn * 3, 0.0);
        if (node_xyz) cp(h->xyz.data(), node_xyz, (size_t)nn * 3 * sizeof(double));
        h->csr_l2g = std::move(l2g);
        h->csr_rowptr = std::move(rowptr);
        h->csr_col = std::move(col);
        h->csr_val = std::move(val);
        analyze(h, t_host0);
    });
}

bddc_status bddc_set_corners(bddc_handle *h, int64_t n, const int64_t *nodes) {
    if (!h) return BDDC_EINVAL;
    BDDC_TRY(h, {
        BDDC_REQUIRE(h->have_mesh, BDDC_ESTATE, "set_corners before set_problem / set_mesh_q1");
        BDDC_REQUIRE(n >= 0 && (n == 0 || nodes), BDDC_EINVAL, "null corner list");
        const auto t_host0 = std::chrono::steady_clock::now();
        std::vector<int64_t> list(nodes, nodes + n);
        std::sort(list.begin(), list.end());
        list.erase(std::unique(list.begin(), list.end()), list.end());
        for (int64_t v : list) BDDC_REQUIRE(v >= 0 && v < h->nn, BDDC_EINVAL, "corner node id out of range");
        h->user_corners = true;
        h->corner_list = list;
        analyze(h, t_host0);
    });
}

bddc_status bddc_select_corners(bddc_handle *h, int64_t *n_out) {
    if (!h) return BDDC_EINVAL;
    BDDC_TRY(h, {
        BDDC_REQUIRE(h->have_mesh, BDDC_ESTATE, "select_corners before set_problem / set_mesh_q1");
        const auto t_host0 = std::chrono::steady_clock::now();
        h->user_corners = false;
        h->corner_list.clear();
        analyze(h, t_host0);
        if (n_out) *n_out = (int64_t)h->corners.size();
    });
}

bddc_status bddc_set_averages(bddc_handle *h, int flags) {
    if (!h) return BDDC_EINVAL;
    BDDC_TRY(h, {
        BDDC_REQUIRE(h->have_mesh, BDDC_ESTATE, "no mesh");
        h->avg_flags = flags & (BDDC_AVG_EDGE | BDDC_AVG_FACE);
        h->have_setup = false;
    });
}

bddc_status bddc_setup(bddc_handle *h) {
    if (!h) return BDDC_EINVAL;
    BDDC_TRY(h, {
        BDDC_REQUIRE(h->have_mesh, BDDC_ESTATE, "no mesh");
        h->have_setup = false;
        do_setup(h);
        BDDC_CUDA(cudaStreamSynchronize(h->stream));
        h->have_setup = true;
    });
}

bddc_status bddc_adapt(bddc_handle *h, double tau, bddc_adapt_info *info) {
    if (!h) return BDDC_EINVAL;
    BDDC_TRY(h, {
        BDDC_REQUIRE(h->have_setup, BDDC_ESTATE, "adapt before setup");
        BDDC_REQUIRE(tau > 0, BDDC_EINVAL, "tau must be positive");
        do_adapt(h, tau, info);
        BDDC_CUDA(cudaStreamSynchronize(h->stream));
    });
}

bddc_status bddc_adapt_fixed(bddc_handle *h, int n_per_face, bddc_adapt_info *info) {
    if (!h) return BDDC_EINVAL;
    BDDC_TRY(h, {
        BDDC_REQUIRE(h->have_setup, BDDC_ESTATE, "adapt before setup");
        BDDC_REQUIRE(n_per_face >= 1 && n_per_face <= 48, BDDC_EINVAL, "n_per_face must be in 1..48");
        do_adapt(h, 1.0, info, n_per_face);
        BDDC_CUDA(cudaStreamSynchronize(h->stream));
    });
}

bddc_status bddc_set_edge_rows(bddc_handle *h, int keep) {
    if (!h) return BDDC_EINVAL;
    BDDC_TRY(h, {
        BDDC_REQUIRE(keep == 0 || keep == 1, BDDC_EINVAL, "keep must be 0 or 1");
        h->keep_edge_rows = keep != 0;
    });
}

bddc_status bddc_get_edge_rows(const bddc_handle *h, int *n_rows, int *n_edges) {
    if (!h) return BDDC_EINVAL;
    if (n_rows) *n_rows = h->n_edge_rows;
    if (n_edges) *n_edges = h->n_edges_with_rows;
    return BDDC_OK;
}

bddc_status bddc_solve(bddc_handle *h, const double *f, double *u, int mem, bddc_solve_info *info) {
    if (!h) return BDDC_EINVAL;
    BDDC_TRY(h, {
        BDDC_REQUIRE(h->have_setup, BDDC_ESTATE, "solve before setup");
        BDDC_REQUIRE(f && u, BDDC_EINVAL, "null vector");
        do_solve(h, f, u, mem, info);
    });
}

bddc_status bddc_condition_estimate(const bddc_handle *h, double *lmin, double *lmax) {
    if (!h || !lmin || !lmax) return BDDC_EINVAL;
    const int k = (int)h->alpha.size();
    if (k == 0) {
        *lmin = *lmax = 1.0;
        return BDDC_OK;
    }
    // Lanczos tridiagonal from the PCG coefficients; eigenvalues by bisection (Sturm counts)
    std::vector<double> d(k), e(k, 0.0);
    for (int j = 0; j < k; ++j) {
        d[j] = 1.0 / h->alpha[j] + (j > 0 ? h->beta[j - 1] / h->alpha[j - 1] : 0.0);
        if (j + 1 < k) e[j] = std::sqrt(h->beta[j]) / h->alpha[j];
    }
    double lo = 1e300, hi = -1e300;
    for (int j = 0; j < k; ++j) {
        double r = (j > 0 ? std::fabs(e[j - 1]) : 0.0) + std::fabs(e[j]);
        lo = std::min(lo, d[j] - r);
        hi = std::max(hi, d[j] + r);
    }
    auto less = [&](double x) {
        int c = 0;
        double q = d[0] - x;
        if (std::fabs(q) < 1e-300) q = -1e-300;
        if (q < 0) ++c;
        for (int j = 1; j < k; ++j) {
            q = d[j] - x - e[j - 1] * e[j - 1] / q;
            if (std::fabs(q) < 1e-300) q = -1e-300;
            if (q < 0) ++c;
        }
        return c;
    };
    auto kth = [&](int idx) {
        double a = lo - 1, b = hi + 1;
        for (int it = 0; it < 200; ++it) {
            double m = 0.5 * (a + b);
            if (less(m) > idx)
                b = m;
            else
                a = m;
        }
        return 0.5 * (a + b);
    };
    *lmin = kth(0);
    *lmax = kth(k - 1);
    return BDDC_OK;
}

bddc_status bddc_get_sizes(const bddc_handle *h, int64_t *n_free, int64_t *n_interface, int *n_corners, int *n_edges,
                           int *n_faces, int *n_coarse) {
    if (!h || !h->have_mesh) return BDDC_ESTATE;
    if (n_free) *n_free = h->nfree;
    if (n_interface) *n_interface = h->nG;
    if (n_corners) *n_corners = (int)h->corners.size();
    if (n_edges) *n_edges = h->n_edges;
    if (n_faces) *n_faces = (int)h->faces.size();
    if (n_coarse) *n_coarse = h->nC;
    return BDDC_OK;
}

bddc_status bddc_get_corners(const bddc_handle *h, int64_t *nodes, int cap, int *n) {
    if (!h || !h->have_mesh) return BDDC_ESTATE;
    if (n) *n = (int)h->corners.size();
    for (int k = 0; k < (int)h->corners.size() && k < cap; ++k) nodes[k] = h->corners[k];
    return BDDC_OK;
}

bddc_status bddc_get_face_eigs(const bddc_handle *h, int f, int32_t *i, int32_t *j, double *lam, int cap, int *n_lam,
                               int *n_selected, int *n_kept) {
    if (!h || !h->have_mesh) return BDDC_ESTATE;
    if (f < 0 || f >= (int)h->faces.size()) return BDDC_EINVAL;
    const auto &fp = h->faces[f];
    if (i) *i = fp.i;
    if (j) *j = fp.j;
    if (n_lam) *n_lam = (int)fp.lam.size();
    if (n_selected) *n_selected = fp.nsel;
    if (n_kept) *n_kept = fp.nkept;
    for (int k = 0; k < (int)fp.lam.size() && k < cap; ++k) lam[k] = fp.lam[k];
    return BDDC_OK;
}

bddc_status bddc_barrier_selftest(bddc_handle *h, int extra, double timeout_s, int *n_passed) {
    if (!h) return BDDC_ESTATE;
    if (!(timeout_s > 0.0 && timeout_s <= 60.0)) return BDDC_EINVAL;
    try {
        reset_status(h);
        int *passed = h->ar.get_t<int>("selftest_passed", 1);
        BDDC_CUDA(cudaMemsetAsync(passed, 0, sizeof(int), h->stream));
        BDDC_CUDA(launch_barrier_selftest(h->dst, extra, timeout_s, passed, h->stream));
        h->launches++;
        int hp = 0;
        DevStatus hs;
        BDDC_CUDA(cudaMemcpyAsync(&hp, passed, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        BDDC_CUDA(cudaMemcpyAsync(&hs, h->dst, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->stream));
        BDDC_CUDA(cudaStreamSynchronize(h->stream));
        if (n_passed) *n_passed = hp;
        reset_status(h);
        BDDC_CUDA(cudaStreamSynchronize(h->stream));
        if (hs.code == BDDC_DEV_ERR_TIMEOUT) {
            h->err = "barrier self-test: the bounded wait gave up after " + std::to_string(timeout_s) + " s";
            return BDDC_ETIMEOUT;
        }
        if (hs.code != 0) return BDDC_ECUDA;
    } catch (const Error &e) {
        h->err = e.msg;
        return (bddc_status)e.status;
    }
    return BDDC_OK;
}

bddc_status bddc_get_face_rows(const bddc_handle *h, int f, int64_t *gdofs, double *rows, int cap_rows,
                               int cap_dofs, int *n_rows, int *n_dofs) {
    if (!h || !h->have_mesh) return BDDC_ESTATE;
    if (f < 0 || f >= (int)h->faces.size()) return BDDC_EINVAL;
    const auto &fp = h->faces[f];
    const int nd = (int)fp.face_idx.size();
    const int nr = (f < (int)h->face_rows_dev.size() && h->face_rows_dev[f]) ? fp.nkept : 0;
    if (n_rows) *n_rows = nr;
    if (n_dofs) *n_dofs = nd;
    if (!gdofs || !rows || cap_rows < nr || cap_dofs < nd) return BDDC_OK;
    try {
        for (int k = 0; k < nd; ++k) gdofs[k] = fp.s_g[fp.face_idx[k]];
        if (nr == 0) return BDDC_OK;
        std::vector<double> T((size_t)nr * nd);   // column-major nr x nd on the device
        BDDC_CUDA(cudaMemcpyAsync(T.data(), h->face_rows_dev[f], T.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                  h->stream));
        BDDC_CUDA(cudaStreamSynchronize(h->stream));
        for (int l = 0; l < nr; ++l)
            for (int k = 0; k < nd; ++k) rows[(size_t)l * nd + k] = T[(size_t)k * nr + l];
    } catch (const Error &e) {
        const_cast<bddc_handle *>(h)->err = e.msg;
        return (bddc_status)e.status;
    }
    return BDDC_OK;
}

bddc_status bddc_get_interface_dofs(const bddc_handle *h, int s, int64_t *gdofs, int cap, int *n) {
    if (!h || !h->have_mesh) return BDDC_ESTATE;
    if (s < 0 || s >= h->nsub) return BDDC_EINVAL;
    const auto &sd = h->subs[s];
    if (n) *n = sd.nG;
    for (int k = 0; k < sd.nG && k < cap; ++k) gdofs[k] = sd.gG[k];
    return BDDC_OK;
}

bddc_status bddc_get_local_matrix(const bddc_handle *h, int s, double *A, int ld, int mem) {
    if (!h || !h->assembled) return BDDC_ESTATE;
    if (h->opt.precision == BDDC_FP64 && h->factored) return BDDC_ESTATE;
    if (s < 0 || s >= h->nsub || ld < h->subs[s].n) return BDDC_EINVAL;
    const auto &sd = h->subs[s];
    cudaError_t e = cudaMemcpy2D(A, (size_t)ld * sizeof(double), sd.A, (size_t)sd.ld * sizeof(double),
                                 (size_t)sd.n * sizeof(double), sd.n,
                                 mem == BDDC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? BDDC_OK : BDDC_ECUDA;
}

bddc_status bddc_get_schur(const bddc_handle *h, int s, double *S, int ld, int mem) {
    if (!h || !h->have_setup) return BDDC_ESTATE;
    if (s < 0 || s >= h->nsub || ld < h->subs[s].nG) return BDDC_EINVAL;
    const auto &sd = h->subs[s];
    cudaError_t e = cudaMemcpy2D(S, (size_t)ld * sizeof(double), sd.S, (size_t)sd.ldS * sizeof(double),
                                 (size_t)sd.nG * sizeof(double), sd.nG,
                                 mem == BDDC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? BDDC_OK : BDDC_ECUDA;
}

static bddc_status apply_op(bddc_handle *h, const double *in, double *out, int mem, int mode) {
    if (!h) return BDDC_EINVAL;
    BDDC_TRY(h, {
        BDDC_REQUIRE(h->have_setup, BDDC_ESTATE, "apply before setup");
        reset_status(h);
        ensure_coarse(h);
        auto kind = mem == BDDC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        double *dst_in = mode == PCG_APPLY_M ? h->pb.r : h->pb.z;
        BDDC_CUDA(cudaMemcpyAsync(dst_in, in, h->nG * sizeof(double), kind, h->stream));
        int nb = 0;
        cudaError_t e = launch_pcg(h->ops, h->pb, mode, h->opt.tol, h->opt.maxit, h->dst, h->opt.timeout_s, h->stream, &nb);
        BDDC_REQUIRE(e == cudaSuccess, BDDC_ECUDA, std::string("apply launch: ") + cudaGetErrorString(e));
        h->launches++;
        double *src_out = mode == PCG_APPLY_M ? h->pb.z : h->pb.q;
        auto kind2 = mem == BDDC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        BDDC_CUDA(cudaMemcpyAsync(out, src_out, h->nG * sizeof(double), kind2, h->stream));
        BDDC_CUDA(cudaStreamSynchronize(h->stream));
        fail_check(h, "apply");
    });
}

bddc_status bddc_apply_preconditioner(bddc_handle *h, const double *r, double *z, int mem) {
    return apply_op(h, r, z, mem, PCG_APPLY_M);
}

bddc_status bddc_apply_schur(bddc_handle *h, const double *x, double *y, int mem) {
    return apply_op(h, x, y, mem, PCG_APPLY_S);
}

int64_t bddc_launch_count(const bddc_handle *h) { return h ? h->launches : 0; }

bddc_status bddc_set_kernel_timing(bddc_handle *h, int on) {
    if (!h || (on != 0 && on != 1)) return BDDC_EINVAL;
    BDDC_TRY(h, {
        kt_collect(h);
        h->ktiming = on != 0;
        for (int k = 0; k < bddc_handle::kKClasses; ++k) {
            h->kt_ms[k] = h->kt_work[k] = 0.0;
            h->kt_n[k] = 0;
        }
    });
}

bddc_status bddc_get_kernel_times(bddc_handle *h, double *ms, double *work, int64_t *launches, int cap, int *n) {
    if (!h) return BDDC_EINVAL;
    BDDC_TRY(h, {
        kt_collect(h);
        if (n) *n = bddc_handle::kKClasses;
        for (int k = 0; k < bddc_handle::kKClasses && k < cap; ++k) {
            if (ms) ms[k] = h->kt_ms[k];
            if (work) work[k] = h->kt_work[k];
            if (launches) launches[k] = h->kt_n[k];
        }
    });
}

bddc_status bddc_get_phase_times(const bddc_handle *h, double *ms, double *flop, int cap, int *n) {
    if (!h) return BDDC_EINVAL;
    if (n) *n = bddc_handle::kPhases;
    for (int k = 0; k < bddc_handle::kPhases && k < cap; ++k) {
        if (ms) ms[k] = h->phase_ms[k];
        if (flop) flop[k] = h->phase_flop[k];
    }
    return BDDC_OK;
}

}  // extern "C"
