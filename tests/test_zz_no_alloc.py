"""rtproj_sketch_noalloc: the float64 sketch without any caller-provided scratch.

Callers whose device memory is owned by a pool or a fixed budget (so that a cudaMalloc
would fail or fragment it), or that cannot afford cudaMalloc's implicit synchronization,
use this entry point: its split-K scratch is a fixed 32 MiB array inside the library.
The test calls it twice in a row through the C ABI (the second call reuses the array
the first one filled) and checks each result against the oracle's A G (G from
oracle.philox) and against rtproj_sketch, the entry point that takes its scratch from a
workspace, within the sketch test's tolerance."""
import ctypes

import numpy as np
import pytest

import workloads
from oracle import philox
from tests.gpu_common import EPS, rt_module, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def _noalloc(rt):
    lib = rt.load_library()
    fn = lib.rtproj_sketch_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64,
                   ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    return fn


def test_noalloc_sketch_matches_workspace_sketch_on_two_calls():
    torch = torch_cuda()
    rt = rt_module()
    fn = _noalloc(rt)
    stream = torch.cuda.current_stream()
    for (m, n, l, seed) in [(64, 2048, 256, 101), (37, 1000, 41, 202)]:
        A = workloads.haar_spectrum_matrix(m, n, 1e-6, seed)
        At = to_dev(torch, A)
        with rt.Projector(At, l_max=l, k_max=1, mode="fp64", omega="uniform") as P:
            ref = P.sketch(seed=seed, l=l).cpu().numpy()
        G = philox.omega(seed, n, l, "uniform")
        S = torch.full((m, l), float("nan"), dtype=torch.float64, device="cuda")
        code = fn(ctypes.c_void_p(At.data_ptr()), m, n, n, seed, l, 0, ctypes.c_void_p(S.data_ptr()), l,
                  ctypes.c_void_p(stream.cuda_stream))
        assert code == 0
        torch.cuda.synchronize()
        scale = np.abs(A).sum(axis=1)[:, None]     # |G| <= 1: bounds (|A| |G|)_ij
        got = S.cpu().numpy()
        assert np.all(np.abs(got - A @ G) <= 4 * n * EPS * scale)
        assert np.all(np.abs(got - ref) <= 4 * n * EPS * scale)


def test_noalloc_sketch_rejects_sizes_beyond_its_scratch():
    torch = torch_cuda()
    rt = rt_module()
    fn = _noalloc(rt)
    m, n, l = 2048, 4096, 4096                 # one 2048 x 4096 slab exceeds the 4 Mi-entry array
    A = torch.zeros((m, n), dtype=torch.float64, device="cuda")
    S = torch.zeros((m, l), dtype=torch.float64, device="cuda")
    code = fn(ctypes.c_void_p(A.data_ptr()), m, n, n, 1, l, 0, ctypes.c_void_p(S.data_ptr()), l,
              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 7                           # RTPROJ_ENOMEM
