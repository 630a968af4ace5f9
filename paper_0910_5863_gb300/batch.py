"""Throughput over many independent problems on one GPU.

Each worker thread owns one library handle and one CUDA stream and takes the
next problem from a shared counter: set the mesh (device-resident arrays),
setup, adapt (Algorithm 3.1 of the paper), solve.  The handles keep their
device buffers between problems, and the library releases the Python GIL
inside every call (ctypes), so the workers' launches interleave on the GPU
and its SMs are shared by several problems at a time.  This is argument
marshalling and scheduling only: every step runs in the CUDA library.

The adaptive constraint count of each face is decided on the host between the
adapt and coarse phases, so a problem's launch sequence is data dependent and
is not captured as one static CUDA graph; concurrent streams are what fill the
GPU with independent problems instead.
"""
from __future__ import annotations

import threading
import time

import numpy as np

from . import bddc as B


def upload(problems, device):
    """Device copies of every problem's mesh arrays and load vector (inputs resident in HBM)."""
    import torch
    out = []
    for p in problems:
        out.append((torch.from_numpy(np.ascontiguousarray(p.xyz)).to(device),
                    torch.from_numpy(np.ascontiguousarray(p.elems, dtype=np.int64)).to(device),
                    torch.from_numpy(np.ascontiguousarray(p.coef)).to(device),
                    torch.from_numpy(np.ascontiguousarray(p.elem_sub, dtype=np.int32)).to(device),
                    torch.from_numpy(np.ascontiguousarray(p.dirichlet, dtype=np.uint8)).to(device),
                    torch.from_numpy(B.free_load_vector(p)).to(device)))
    return out


class Pool:
    """Worker handles (one CUDA stream each).  Keeping a pool across runs keeps the
    handles' device buffers, so later runs allocate nothing."""

    def __init__(self, precision, workers=8, tol=1e-8, device=None):
        import torch
        self.device = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.streams = [torch.cuda.Stream(self.device) for _ in range(max(1, workers))]
        self.solvers = [B.Solver(precision=precision, tol=tol, stream=st.cuda_stream) for st in self.streams]


def run(problems, arrays, pool, tau=10.0, keep_solutions=False):
    """Solves every problem once on the pool's handles.  Returns (wall seconds,
    per-problem records): each record has the problem's host-side latency
    (set_mesh to solution, stream synchronised), its iterations, condition
    estimate, added constraints and, with keep_solutions, the solution as a
    device tensor."""
    import torch
    n = len(problems)
    records = [None] * n
    nxt = [0]
    lock = threading.Lock()
    errors = []

    def worker(stream, solver):
        try:
            torch.cuda.set_device(pool.device)
            while True:
                with lock:
                    i = nxt[0]
                    nxt[0] += 1
                if i >= n:
                    break
                p = problems[i]
                xyz, el, coef, sub, dirich, f = arrays[i]
                with torch.cuda.stream(stream):
                    u = torch.zeros_like(f)
                t0 = time.perf_counter()
                solver.set_mesh(p.ncomp, xyz, el, coef, p.nu, sub, p.nsub, dirich)
                solver.setup()
                ad = solver.adapt(tau)
                _, info = solver.solve(f, u)
                stream.synchronize()
                t1 = time.perf_counter()
                records[i] = {"latency_s": t1 - t0, "iters": info["iters"], "kappa": info["kappa"],
                              "n_added": ad["n_added"], "converged": info["converged"],
                              "u": u if keep_solutions else None}
        except Exception as e:   # reported to the caller after the join
            errors.append(e)

    torch.cuda.synchronize(pool.device)
    t0 = time.perf_counter()
    threads = [threading.Thread(target=worker, args=(st, sv)) for st, sv in zip(pool.streams, pool.solvers)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    torch.cuda.synchronize(pool.device)
    wall = time.perf_counter() - t0
    if errors:
        raise errors[0]
    return wall, records
