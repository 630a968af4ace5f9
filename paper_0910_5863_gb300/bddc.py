"""Python binding of the C ABI in include/bddc.h (argument marshalling only).

Every numeric step runs in the CUDA library libbddc.so; this module converts
numpy arrays / torch tensors to pointers and status codes to exceptions.  It
fails loudly when the library has not been built (``python -m
paper_0910_5863_gb300.build``): there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbddc.so")

MEM_HOST, MEM_DEVICE = 0, 1
FP64, MIXED, MIXED_FP32_SADDLE = 0, 1, 2
AVG_EDGE, AVG_FACE = 1, 2
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ENOTSPD", 4: "EASSUMPTION", 5: "ENOCONV", 6: "ETIMEOUT",
          7: "ECUDA", 8: "ESTATE"}

EXPORTS = ["bddc_default_options", "bddc_create", "bddc_destroy", "bddc_set_mesh_q1", "bddc_set_averages",
           "bddc_setup", "bddc_adapt", "bddc_solve", "bddc_condition_estimate", "bddc_get_sizes",
           "bddc_get_corners", "bddc_get_face_eigs", "bddc_get_interface_dofs", "bddc_get_schur",
           "bddc_apply_preconditioner", "bddc_apply_schur", "bddc_launch_count", "bddc_status_str",
           "bddc_last_error", "bddc_get_phase_times", "bddc_get_local_matrix", "bddc_set_problem",
           "bddc_set_corners", "bddc_select_corners", "bddc_get_face_rows", "bddc_barrier_selftest",
           "bddc_classify_q1", "bddc_adapt_fixed", "bddc_set_edge_rows", "bddc_get_edge_rows",
           "bddc_set_kernel_timing", "bddc_get_kernel_times"]
PHASES = ["assembly", "interior_elimination", "coarse_setup", "pair_condensation", "face_eigen",
          "analysis_host", "condensed_rhs", "pcg", "recovery"]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("tol", C.c_double), ("maxit", C.c_int), ("drop_rel", C.c_double),
                ("timeout_s", C.c_double), ("stream", C.c_void_p), ("dev_alloc", C.c_void_p),
                ("dev_free", C.c_void_p), ("alloc_ctx", C.c_void_p), ("refine_tol", C.c_double),
                ("eig_large_n", C.c_int), ("eig_tol", C.c_double), ("eig_maxit", C.c_int),
                ("mixed_updates", C.c_int)]


class Subdomain(C.Structure):
    _fields_ = [("n_local", C.c_int32), ("l2g", C.c_void_p), ("rowptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p)]


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class AdaptInfo(C.Structure):
    _fields_ = [("n_faces", C.c_int), ("n_added", C.c_int), ("n_ties", C.c_int), ("omega", C.c_double),
                ("n_lobpcg", C.c_int), ("lobpcg_iters", C.c_int), ("n_dense_fallback", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("converged", C.c_int), ("relres", C.c_double), ("kappa", C.c_double),
                ("setup_ms", C.c_double), ("solve_ms", C.c_double), ("interior_fp32", C.c_int),
                ("coarse_fp32", C.c_int), ("refine_steps", C.c_int), ("refine_relres", C.c_double),
                ("relres_recurrence", C.c_double)]


def _adapt_dict(info):
    return {"n_faces": info.n_faces, "n_added": info.n_added, "n_ties": info.n_ties, "omega": info.omega,
            "n_lobpcg": info.n_lobpcg, "lobpcg_iters": info.lobpcg_iters, "n_dense_fallback": info.n_dense_fallback}


class BddcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Loads libbddc.so; raises if it is missing (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} missing (run paper_0910_5863_gb300.build.build())")
    lib = C.CDLL(path)
    vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double
    sig = {
        "bddc_default_options": (None, [vp]),
        "bddc_create": (i32, [vp, vp]),
        "bddc_destroy": (None, [vp]),
        "bddc_set_mesh_q1": (i32, [vp, i32, i64, vp, i64, vp, vp, dbl, vp, C.c_int32, vp, i32]),
        "bddc_set_averages": (i32, [vp, i32]),
        "bddc_setup": (i32, [vp]),
        "bddc_adapt": (i32, [vp, dbl, vp]),
        "bddc_solve": (i32, [vp, vp, vp, i32, vp]),
        "bddc_condition_estimate": (i32, [vp, vp, vp]),
        "bddc_get_sizes": (i32, [vp, vp, vp, vp, vp, vp, vp]),
        "bddc_get_corners": (i32, [vp, vp, i32, vp]),
        "bddc_get_face_eigs": (i32, [vp, i32, vp, vp, vp, i32, vp, vp, vp]),
        "bddc_get_interface_dofs": (i32, [vp, i32, vp, i32, vp]),
        "bddc_get_schur": (i32, [vp, i32, vp, i32, i32]),
        "bddc_apply_preconditioner": (i32, [vp, vp, vp, i32]),
        "bddc_apply_schur": (i32, [vp, vp, vp, i32]),
        "bddc_launch_count": (i64, [vp]),
        "bddc_status_str": (C.c_char_p, [i32]),
        "bddc_last_error": (C.c_char_p, [vp]),
        "bddc_get_phase_times": (i32, [vp, vp, vp, i32, vp]),
        "bddc_set_kernel_timing": (i32, [vp, i32]),
        "bddc_get_kernel_times": (i32, [vp, vp, vp, vp, i32, vp]),
        "bddc_get_local_matrix": (i32, [vp, i32, vp, i32, i32]),
        "bddc_set_problem": (i32, [vp, i64, i32, C.c_int32, vp, vp, i32]),
        "bddc_set_corners": (i32, [vp, i64, vp]),
        "bddc_select_corners": (i32, [vp, vp]),
        "bddc_get_face_rows": (i32, [vp, i32, vp, vp, i32, i32, vp, vp]),
        "bddc_barrier_selftest": (i32, [vp, i32, dbl, vp]),
        "bddc_adapt_fixed": (i32, [vp, i32, vp]),
        "bddc_set_edge_rows": (i32, [vp, i32]),
        "bddc_get_edge_rows": (i32, [vp, vp, vp]),
        "bddc_classify_q1": (i32, [i32, i64, vp, i64, vp, vp, C.c_int32, vp, vp, vp, vp, vp, vp, vp, vp, i32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _torch_allocator(stream):
    """ctypes callbacks that take device memory from PyTorch's caching allocator."""
    import torch
    dev = torch.cuda.current_device()
    sid = int(stream) if stream else torch.cuda.current_stream(dev).cuda_stream

    def alloc(nbytes, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, sid)
        except Exception:
            return None

    def free(ptr, nbytes, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    return _ALLOC_FN(alloc), _FREE_FN(free)


def _ptr(a):
    """(pointer, mem) of a C-contiguous numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data, MEM_HOST
    import torch
    assert isinstance(a, torch.Tensor) and a.is_contiguous()
    return a.data_ptr(), (MEM_DEVICE if a.is_cuda else MEM_HOST)


class Solver:
    """One handle of the library (one GPU, one stream)."""

    def __init__(self, precision=FP64, tol=1e-8, maxit=1000, drop_rel=1e-10, timeout_s=10.0, stream=None,
                 allocator=None, refine_tol=None, eig_large_n=None, eig_tol=None, eig_maxit=None,
                 mixed_updates=None):
        """allocator: None (the library's cudaMalloc) or "torch" (device memory from
        PyTorch's caching allocator on the handle's stream).  eig_large_n / eig_tol /
        eig_maxit: the batched LOBPCG of the pair problems (bddc_options); None = default."""
        self.lib = load()
        opt = Options()
        self.lib.bddc_default_options(C.byref(opt))
        opt.precision = precision
        self.precision = precision
        opt.tol = tol
        opt.maxit = maxit
        opt.drop_rel = drop_rel
        opt.timeout_s = timeout_s
        opt.stream = stream
        if refine_tol is not None:
            opt.refine_tol = refine_tol
        if eig_large_n is not None:
            opt.eig_large_n = int(eig_large_n)
        if eig_tol is not None:
            opt.eig_tol = float(eig_tol)
        if eig_maxit is not None:
            opt.eig_maxit = int(eig_maxit)
        if mixed_updates is not None:
            opt.mixed_updates = int(mixed_updates)
        self._callbacks = None
        if allocator == "torch":
            self._callbacks = _torch_allocator(stream)
            opt.dev_alloc = C.cast(self._callbacks[0], C.c_void_p)
            opt.dev_free = C.cast(self._callbacks[1], C.c_void_p)
        elif allocator is not None:
            raise ValueError("allocator must be None or 'torch'")
        h = C.c_void_p()
        st = self.lib.bddc_create(C.byref(opt), C.byref(h))
        if st != 0:
            raise BddcError(st, "bddc_create failed")
        self.h = h
        self.nfree = 0

    def close(self):
        if getattr(self, "h", None):
            self.lib.bddc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != 0:
            raise BddcError(st, self.lib.bddc_last_error(self.h).decode())

    # -- problem ------------------------------------------------------------
    def set_mesh(self, ncomp, xyz, elems, coef, nu, elem_sub, nsub, dirichlet):
        """Arrays: numpy (host) or torch CUDA tensors (device), all in the same memory."""
        arrs = [xyz, elems, coef, elem_sub, dirichlet]
        ptrs = [_ptr(a) for a in arrs]
        mem = ptrs[0][1]
        assert all(p[1] == mem for p in ptrs), "all mesh arrays must live in the same memory"
        nn = xyz.shape[0]
        ne = elems.shape[0]
        self._check(self.lib.bddc_set_mesh_q1(self.h, ncomp, nn, ptrs[0][0], ne, ptrs[1][0], ptrs[2][0], float(nu),
                                              ptrs[3][0], int(nsub), ptrs[4][0], mem))
        self.nfree = self.sizes()["n_free"]
        self.nsub = int(nsub)

    def set_problem(self, n_global, ncomp, subs, node_xyz=None):
        """Algebraic problem: subs = [(l2g, A_i)] with l2g (n_local,) global dof ids
        and A_i a scipy.sparse matrix (any format) or a (rowptr, col, val) triple over
        local dofs; node_xyz (n_global // ncomp, 3) or None.  Host memory."""
        keep, desc = [], (Subdomain * len(subs))()
        for k, (l2g, A) in enumerate(subs):
            if isinstance(A, tuple):
                rowptr, col, val = A
            else:
                A = A.tocsr()
                rowptr, col, val = A.indptr, A.indices, A.data
            arrs = (np.ascontiguousarray(l2g, dtype=np.int64), np.ascontiguousarray(rowptr, dtype=np.int64),
                    np.ascontiguousarray(col, dtype=np.int32), np.ascontiguousarray(val, dtype=np.float64))
            keep.append(arrs)
            desc[k] = Subdomain(arrs[0].size, arrs[0].ctypes.data, arrs[1].ctypes.data, arrs[2].ctypes.data,
                                arrs[3].ctypes.data)
        xyz = None if node_xyz is None else np.ascontiguousarray(node_xyz, dtype=np.float64)
        self._check(self.lib.bddc_set_problem(self.h, int(n_global), int(ncomp), len(subs), desc,
                                              None if xyz is None else xyz.ctypes.data, MEM_HOST))
        self.nfree = self.sizes()["n_free"]
        self.nsub = len(subs)

    def set_corners(self, nodes):
        a = np.ascontiguousarray(nodes, dtype=np.int64)
        self._check(self.lib.bddc_set_corners(self.h, a.size, a.ctypes.data))

    def select_corners(self):
        n = C.c_int64()
        self._check(self.lib.bddc_select_corners(self.h, C.byref(n)))
        return n.value

    def set_mesh_problem(self, prob):
        """Host arrays of a paper_0910_5863_gb300.problems.Problem."""
        self.set_mesh(prob.ncomp, np.ascontiguousarray(prob.xyz, dtype=np.float64),
                      np.ascontiguousarray(prob.elems, dtype=np.int64),
                      np.ascontiguousarray(prob.coef, dtype=np.float64), prob.nu,
                      np.ascontiguousarray(prob.elem_sub, dtype=np.int32), prob.nsub,
                      np.ascontiguousarray(prob.dirichlet, dtype=np.uint8))

    def set_averages(self, edge=False, face=False):
        self._check(self.lib.bddc_set_averages(self.h, (AVG_EDGE if edge else 0) | (AVG_FACE if face else 0)))

    def setup(self):
        self._check(self.lib.bddc_setup(self.h))

    def adapt(self, tau):
        info = AdaptInfo()
        self._check(self.lib.bddc_adapt(self.h, float(tau), C.byref(info)))
        return _adapt_dict(info)

    def adapt_fixed(self, n_per_face):
        """The n_per_face dominant eigenvector constraints on every face (Section 7, "3eigv")."""
        info = AdaptInfo()
        self._check(self.lib.bddc_adapt_fixed(self.h, int(n_per_face), C.byref(info)))
        return _adapt_dict(info)

    def set_edge_rows(self, keep=True):
        """Later adapt calls also keep the edge parts of the rows d (Section 3), one
        orthonormal basis per edge on all substructures of the edge."""
        self._check(self.lib.bddc_set_edge_rows(self.h, 1 if keep else 0))

    def edge_rows(self):
        """(edge rows kept by the last adapt, edges that got rows)."""
        n, e = C.c_int(), C.c_int()
        self._check(self.lib.bddc_get_edge_rows(self.h, C.byref(n), C.byref(e)))
        return n.value, e.value

    def solve(self, f, u=None, check=True):
        """f: global free-dof load vector (numpy or torch CUDA).  Returns (u, info)."""
        if u is None:
            if isinstance(f, np.ndarray):
                u = np.zeros_like(f)
            else:
                import torch
                u = torch.zeros_like(f)
        pf, mem = _ptr(f)
        pu, mem2 = _ptr(u)
        assert mem == mem2
        info = SolveInfo()
        st = self.lib.bddc_solve(self.h, pf, pu, mem, C.byref(info))
        out = {"iters": info.iters, "converged": bool(info.converged), "relres": info.relres, "kappa": info.kappa,
               "interior_fp32": bool(info.interior_fp32), "coarse_fp32": bool(info.coarse_fp32),
               "refine_steps": info.refine_steps, "refine_relres": info.refine_relres,
               "relres_recurrence": info.relres_recurrence}
        if check or st not in (0, 5):
            self._check(st)
        out["status"] = STATUS.get(st, st)
        return u, out

    def condition_estimate(self):
        lo, hi = C.c_double(), C.c_double()
        self._check(self.lib.bddc_condition_estimate(self.h, C.byref(lo), C.byref(hi)))
        return lo.value, hi.value

    # -- inspection --------------------------------------------------------
    def sizes(self):
        nf, ni = C.c_int64(), C.c_int64()
        nc, ne, nfa, nco = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        self._check(self.lib.bddc_get_sizes(self.h, C.byref(nf), C.byref(ni), C.byref(nc), C.byref(ne), C.byref(nfa),
                                            C.byref(nco)))
        return {"n_free": nf.value, "n_interface": ni.value, "n_corners": nc.value, "n_edges": ne.value,
                "n_faces": nfa.value, "n_coarse": nco.value}

    def corners(self):
        n = C.c_int()
        self._check(self.lib.bddc_get_corners(self.h, None, 0, C.byref(n)))
        out = np.zeros(n.value, dtype=np.int64)
        self._check(self.lib.bddc_get_corners(self.h, out.ctypes.data, n.value, C.byref(n)))
        return out

    def face_eigs(self, f):
        i, j = C.c_int32(), C.c_int32()
        nl, ns, nk = C.c_int(), C.c_int(), C.c_int()
        buf = np.zeros(64)
        self._check(self.lib.bddc_get_face_eigs(self.h, f, C.byref(i), C.byref(j), buf.ctypes.data, 64, C.byref(nl),
                                                C.byref(ns), C.byref(nk)))
        return {"pair": (i.value, j.value), "lam": buf[: nl.value].copy(), "selected": ns.value, "kept": nk.value}

    def barrier_selftest(self, extra, timeout_s):
        """(status, blocks that passed) of the bounded-barrier self-test (no exception)."""
        n = C.c_int()
        st = self.lib.bddc_barrier_selftest(self.h, int(extra), float(timeout_s), C.byref(n))
        return STATUS.get(st, st), n.value

    def face_rows(self, f):
        """(global face dofs, kept adaptive rows n_rows x n_dofs) of face f."""
        nr, nd = C.c_int(), C.c_int()
        self._check(self.lib.bddc_get_face_rows(self.h, f, None, None, 0, 0, C.byref(nr), C.byref(nd)))
        gd = np.zeros(nd.value, dtype=np.int64)
        rows = np.zeros((nr.value, nd.value))
        self._check(self.lib.bddc_get_face_rows(self.h, f, gd.ctypes.data, rows.ctypes.data, nr.value, nd.value,
                                                C.byref(nr), C.byref(nd)))
        return gd, rows

    def interface_dofs(self, s):
        n = C.c_int()
        self._check(self.lib.bddc_get_interface_dofs(self.h, s, None, 0, C.byref(n)))
        out = np.zeros(n.value, dtype=np.int64)
        self._check(self.lib.bddc_get_interface_dofs(self.h, s, out.ctypes.data, n.value, C.byref(n)))
        return out

    def schur(self, s):
        n = self.interface_dofs(s).size
        S = np.zeros((n, n))
        self._check(self.lib.bddc_get_schur(self.h, s, S.ctypes.data, n, MEM_HOST))
        return S.T.copy()   # column-major -> row-major (symmetric anyway)

    def local_matrix(self, s, n):
        """Assembled A_s (n x n, [interior; interface]); mixed mode, after setup."""
        A = np.zeros((n, n))
        self._check(self.lib.bddc_get_local_matrix(self.h, s, A.ctypes.data, n, MEM_HOST))
        return A.T.copy()

    def apply_preconditioner(self, r):
        r = np.ascontiguousarray(r, dtype=np.float64)
        z = np.zeros_like(r)
        self._check(self.lib.bddc_apply_preconditioner(self.h, r.ctypes.data, z.ctypes.data, MEM_HOST))
        return z

    def apply_schur(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros_like(x)
        self._check(self.lib.bddc_apply_schur(self.h, x.ctypes.data, y.ctypes.data, MEM_HOST))
        return y

    KERNEL_CLASSES = ["pchol_update_ff", "pchol_update_fp64", "pchol_update_fp32", "tc_gemm_3xtf32", "pcg_kernel",
                      "face_reduction", "oz_syrk_bf16", "oz_split", "pchol_panel"]

    def set_kernel_timing(self, on=True):
        self._check(self.lib.bddc_set_kernel_timing(self.h, 1 if on else 0))

    def kernel_times(self):
        """{class: (ms, algorithmic flop, launches)} since set_kernel_timing(True)."""
        ms = np.zeros(16)
        wk = np.zeros(16)
        nl = np.zeros(16, dtype=np.int64)
        n = C.c_int()
        self._check(self.lib.bddc_get_kernel_times(self.h, ms.ctypes.data, wk.ctypes.data, nl.ctypes.data, 16,
                                                   C.byref(n)))
        return {self.KERNEL_CLASSES[k]: (ms[k], wk[k], int(nl[k])) for k in range(n.value)}

    def phase_times(self):
        """{phase: (ms, algorithmic flop)} of the last setup / adapt / solve."""
        ms = np.zeros(16)
        fl = np.zeros(16)
        n = C.c_int()
        self._check(self.lib.bddc_get_phase_times(self.h, ms.ctypes.data, fl.ctypes.data, 16, C.byref(n)))
        return {PHASES[k]: (ms[k], fl[k]) for k in range(n.value)}

    def launch_count(self):
        return int(self.lib.bddc_launch_count(self.h))


def classify_mesh(prob):
    """Host-only mesh analysis of a paper_0910_5863_gb300.problems.Problem (no GPU):
    dict with n_free, n_interface, n_corners, n_edges, n_faces, n_augmented, corners."""
    lib = load()
    xyz = np.ascontiguousarray(prob.xyz, dtype=np.float64)
    el = np.ascontiguousarray(prob.elems, dtype=np.int64)
    sub = np.ascontiguousarray(prob.elem_sub, dtype=np.int32)
    dr = np.ascontiguousarray(prob.dirichlet, dtype=np.uint8)
    nf, ni = C.c_int64(), C.c_int64()
    nc, ne, nfa, na = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    cap = xyz.shape[0]
    corners = np.zeros(cap, dtype=np.int64)
    st = lib.bddc_classify_q1(prob.ncomp, xyz.shape[0], xyz.ctypes.data, el.shape[0], el.ctypes.data,
                              sub.ctypes.data, prob.nsub, dr.ctypes.data, C.byref(nf), C.byref(ni), C.byref(nc),
                              C.byref(ne), C.byref(nfa), C.byref(na), corners.ctypes.data, cap)
    if st != 0:
        raise BddcError(st, lib.bddc_status_str(st).decode())
    return {"n_free": nf.value, "n_interface": ni.value, "n_corners": nc.value, "n_edges": ne.value,
            "n_faces": nfa.value, "n_augmented": na.value, "corners": corners[: nc.value].copy()}


def free_load_vector(prob):
    """Global free-dof load vector of a Problem (node-major over non-Dirichlet nodes)."""
    return np.ascontiguousarray(prob.load[~prob.dirichlet].reshape(-1), dtype=np.float64)
