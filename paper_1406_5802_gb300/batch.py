"""Batched randomized-GENP solves of uneven size: packing, longest-first ordering, the autotuner that picks
the persistent kernel's tile shape and CTA count, and CUDA-graph capture of the single launch.

All arithmetic runs in ``rmge_solve_batched`` (librmge); this module only lays out device buffers,
measures candidate launch configurations, and replays the captured launch.
"""
from __future__ import annotations

import ctypes as C
import json
import os

import numpy as np
import torch

from . import rmge

# (config id, threads, tile) of the compiled persistent-kernel variants
CONFIGS = {0: (256, 32), 1: (256, 64), 2: (1024, 64)}
TUNE_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "batch_tune.json")


def _lib():
    return rmge._cuda_lib()


def pack_layout(sizes):
    """Packing of uneven systems: element offsets of A_i (n_i x n_i, back to back) and of b_i, x_i, and the
    processing order (decreasing n, ties in index order), as the persistent kernel's queue takes them."""
    sizes = np.asarray(sizes, dtype=np.int32)
    if sizes.ndim != 1 or sizes.size == 0 or sizes.min() < 1:
        raise ValueError("sizes must be a non-empty list of positive orders")
    sq = sizes.astype(np.int64) ** 2
    offA = np.zeros(sizes.size, np.int64)
    offv = np.zeros(sizes.size, np.int64)
    offA[1:] = np.cumsum(sq)[:-1]
    offv[1:] = np.cumsum(sizes.astype(np.int64))[:-1]
    order = np.argsort(-sizes, kind="stable").astype(np.int32)  # longest first
    return offA, offv, order


class BatchedSolver:
    """Holds one packed batch (A_i, b_i) on the device and solves it with one persistent launch."""

    def __init__(self, As, bs, seed: int, max_sweeps: int = 10, be_tol: float = 1e-13, device="cuda"):
        sizes = np.array([a.shape[0] for a in As], dtype=np.int32)
        offA, offv, _ = pack_layout(sizes)
        A_h = torch.empty(int((sizes.astype(np.int64) ** 2).sum()), dtype=torch.float64)
        b_h = torch.empty(int(sizes.sum()), dtype=torch.float64)
        for i, (a, b) in enumerate(zip(As, bs)):
            n = sizes[i]
            A_h[offA[i]:offA[i] + n * n] = torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).reshape(-1)
            b_h[offv[i]:offv[i] + n] = torch.as_tensor(np.ascontiguousarray(b, dtype=np.float64)).reshape(-1)
        self._init_packed(sizes, offA, offv, A_h.to(device), b_h.to(device), seed, max_sweeps, be_tol)

    @classmethod
    def synthetic(cls, sizes, seed: int, leading_scale: float = 1e-10, **kw):
        """The uneven-batch workload drawn on the device: A_i i.i.d. N(0,1) with A_i[0,0] scaled by
        leading_scale, b_i i.i.d. N(0,1) (torch's generator, seeded)."""
        self = cls.__new__(cls)
        sizes = np.asarray(sizes, dtype=np.int32)
        g = torch.Generator(device="cuda")
        g.manual_seed(int(seed))
        offA, offv, _ = pack_layout(sizes)
        A = torch.randn(int((sizes.astype(np.int64) ** 2).sum()), generator=g, dtype=torch.float64, device="cuda")
        A[torch.as_tensor(offA, device="cuda")] *= leading_scale
        b = torch.randn(int(sizes.sum()), generator=g, dtype=torch.float64, device="cuda")
        self._init_packed(sizes, offA, offv, A, b, seed, **kw)
        return self

    def _init_packed(self, sizes, offA, offv, A, b, seed, max_sweeps=10, be_tol=1e-13):
        device = A.device
        self.count = len(sizes)
        self.nmax = int(sizes.max())
        self.sizes, self.offA, self.offv = sizes, offA, offv
        order = pack_layout(sizes)[2]
        self.d_n = torch.as_tensor(sizes).to(device)
        self.d_offA = torch.as_tensor(offA).to(device)
        self.d_offv = torch.as_tensor(offv).to(device)
        self.d_order = torch.as_tensor(order).to(device)
        self.A, self.b = A, b
        self.x = torch.empty_like(b)
        self.info = torch.empty(self.count, dtype=torch.int32, device=device)
        self.berr = torch.empty(self.count, dtype=torch.float64, device=device)
        self.sweeps = torch.empty(self.count, dtype=torch.int32, device=device)
        self.seed, self.max_sweeps, self.be_tol = int(seed), int(max_sweeps), float(be_tol)
        self.config, self.ctas = 1, torch.cuda.get_device_properties(device).multi_processor_count
        self.ws = None
        self.graph = None

    def flops(self) -> float:
        """Algorithmic flops of one pass: per system A G (2n^3 - n^2) and GENP (2n^3/3 - n^2/2 - n/6)."""
        n = self.sizes.astype(np.float64)
        return float(np.sum((2 * n**3 - n**2) + (2 * n**3 / 3 - n**2 / 2 - n / 6)))

    def _ensure_ws(self, ctas):
        need = int(_lib().rmge_batched_workspace_size(self.nmax, ctas))
        if need == 0:
            raise ValueError("invalid batched workspace request")
        if self.ws is None or self.ws.numel() < need:
            self.ws = torch.empty(need, dtype=torch.uint8, device=self.A.device)

    def launch(self, config=None, ctas=None, opts=None):
        """One launch of rmge_solve_batched (rmge_solve_batched_ex with opts, an rmge.Options); returns the
        call's return value (its outcome when opts.sync is set)."""
        config = self.config if config is None else config
        ctas = self.ctas if ctas is None else ctas
        self._ensure_ws(ctas)
        p = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
        args = (self.count, p(self.d_n), p(self.d_offA), p(self.d_offv), p(self.d_order), p(self.A), p(self.b),
                p(self.x), p(self.info), p(self.berr), p(self.sweeps), self.seed, self.max_sweeps, self.be_tol,
                self.nmax, int(config), int(ctas))
        tail = (p(self.ws), self.ws.numel(), C.c_void_p(torch.cuda.current_stream().cuda_stream))
        if opts is None:
            st = _lib().rmge_solve_batched(*args, *tail)
            rmge._check("rmge_solve_batched", st)
            return st
        st = _lib().rmge_solve_batched_ex(*args, C.byref(opts), *tail)
        return rmge._check_ex("rmge_solve_batched_ex", st, opts)

    def tune(self, reps: int = 2, use_cache: bool = True):
        """Time every compiled variant at 1..3 persistent CTAs per SM on this batch; keep the fastest.
        Results are cached per (device, size histogram)."""
        sms = torch.cuda.get_device_properties(self.A.device).multi_processor_count
        key = f"{torch.cuda.get_device_name(self.A.device)}|{self.count}|{self.nmax}|{int(self.sizes.sum())}"
        cache = {}
        if use_cache and os.path.exists(TUNE_FILE):
            try:
                cache = json.load(open(TUNE_FILE))
            except Exception:
                cache = {}
        if key in cache:
            self.config, self.ctas = cache[key]["config"], cache[key]["ctas"]
            return cache[key]
        results = []
        for cfg, (threads, _) in CONFIGS.items():
            for per_sm in (1, 2, 3):
                if threads * per_sm > 2048:
                    continue
                ctas = sms * per_sm
                self.launch(cfg, ctas)  # warm
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    self.launch(cfg, ctas)
                e1.record()
                torch.cuda.synchronize()
                results.append((e0.elapsed_time(e1) / reps, cfg, ctas))
        ms, cfg, ctas = min(results)
        self.config, self.ctas = cfg, ctas
        entry = {"config": cfg, "ctas": ctas, "ms": ms, "candidates": [[m, c, k] for m, c, k in results]}
        cache[key] = entry
        try:
            os.makedirs(os.path.dirname(TUNE_FILE), exist_ok=True)
            json.dump(cache, open(TUNE_FILE, "w"), indent=1)
        except OSError:
            pass
        return entry

    def capture(self):
        """Capture the chosen launch in a CUDA graph (one memset + one persistent kernel)."""
        self._ensure_ws(self.ctas)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.launch()  # warm-up outside capture
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.launch()
        return self.graph

    def run(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self.launch()

    def system(self, i: int):
        """(A_i, b_i) of system i: views of the packed device arrays (A_i row-major, n_i x n_i)."""
        n = int(self.sizes[i])
        return self.A[self.offA[i]:self.offA[i] + n * n].view(n, n), self.b[self.offv[i]:self.offv[i] + n]

    def solution(self, i: int) -> torch.Tensor:
        n = int(self.sizes[i])
        return self.x[self.offv[i]:self.offv[i] + n]
