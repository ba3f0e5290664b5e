"""Many independent instances at once: uneven (m_i, n_i) problems, or one A under a
sequence of interior-point-style column scalings A diag(d_j).

Each instance has its own handle in the asynchronous mode (opts.async: no host
synchronization inside precondition) on one of several CUDA streams, so independent
instances run concurrently on the GPU: a small instance's pivoted QR occupies one 16-SM
cluster and its products a fraction of the SMs, leaving the rest to the others. One step --
every instance's precondition and null_project -- can be captured once into a CUDA graph and
replayed with one host call, which removes the host's per-launch cost from the loop. Every
kernel is librtproj's; conditions found on the device stay latched per handle
(``statuses()``).
"""
from __future__ import annotations

import ctypes

import torch

from . import Projector, _dev_ptr, _check, load_library

__all__ = ["Batch"]


class Batch:
    """Instances (A_i) with right-hand sides B_i (k_i x n_i rows), sketch sizes l_i."""

    def __init__(self, As, ks, ls, streams: int = 8, mode: str = "mixed", **opts):
        if not (len(As) == len(ks) == len(ls)):
            raise ValueError("one k and one l per instance")
        dev = As[0].device
        self.device = dev
        self.streams = [torch.cuda.Stream(dev) for _ in range(max(1, streams))]
        self.P = []
        for i, (A, k, l) in enumerate(zip(As, ks, ls)):
            s = self.streams[i % len(self.streams)]
            self.P.append(Projector(A, l_max=int(l), k_max=int(k), mode=mode, stream=s, async_=1, **opts))
        self.ls = [int(l) for l in ls]
        self.graph = None

    def step(self, Bs, seeds, Zs):
        """Enqueues precondition(seed_i, l_i) and Z_i = null_project(B_i) for every instance
        (no host synchronization); the caller's current stream waits for all of them."""
        lib = load_library()
        cur = torch.cuda.current_stream(self.device)
        for s in self.streams:
            s.wait_stream(cur)
        for P, B, seed, Z, l in zip(self.P, Bs, seeds, Zs, self.ls):
            with torch.cuda.device(self.device):
                _check(lib.rtproj_precondition(P._h, ctypes.c_uint64(int(seed)), l), "rtproj_precondition")
                _check(lib.rtproj_null_project(P._h, _dev_ptr(B), B.stride(0), B.shape[0], _dev_ptr(Z), Z.stride(0)),
                       "rtproj_null_project")
        for s in self.streams:
            cur.wait_stream(s)

    def capture(self, Bs, seeds, Zs):
        """Records one step into a CUDA graph (the inputs' and outputs' memory is fixed)."""
        self.step(Bs, seeds, Zs)                      # warm-up outside the capture
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.step(Bs, seeds, Zs)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def statuses(self):
        return [P.info()["status"] for P in self.P]

    def close(self):
        for P in self.P:
            P.close()
