"""The bench's roofline arithmetic (CPU): digit-pair counts of the sliced products and the
apply's algorithmic bytes, against hand counts; the pipelined steps' memory cap."""
import ctypes
import types

import bench
import workloads


def test_digit_pairs_hand_counts():
    # pairs (p, q), p < sa, q < sb, p + q < terms
    assert bench.digit_pairs(7, 7, 7) == 28          # 1 + 2 + ... + 7
    assert bench.digit_pairs(9, 9, 9) == 45
    assert bench.digit_pairs(4, 4, 4) == 10
    assert bench.digit_pairs(1, 5, 5) == 5           # one plane of G against five of A
    assert bench.digit_pairs(2, 5, 5) == 9           # two Gaussian planes: 5 + 4
    assert bench.digit_pairs(3, 3, 1) == 1


def test_apply_bytes_of_the_headline_workload():
    """A read as float64 twice per apply plus twice per refinement pass, B read and Z
    written (16 n k bytes), h written (8 m k): 1,141,112,832 bytes at 512 x 65536, k 64, one
    pass."""
    w = workloads.WORKLOADS["dense_512x65536"]
    opts = types.SimpleNamespace(apply_slices=7, resid_slices=9)
    pk = {"hbm_gbs": 1000.0, "bf16_tflops": 1000.0, "_source": "test"}
    e = bench.apply_roofline(w, opts, 64, 1.0, 1, pk)
    assert e["bytes_per_call"] == 4 * 512 * 65536 * 8 + 65536 * 64 * 16 + 512 * 64 * 8 == 1141112832
    assert abs(e["achieved"] - 1141.112832) < 1e-9 and abs(e["frac"] - 1.141112832) < 1e-12


def test_apply_ceiling_of_the_headline_workload():
    """Digit pairs per call: c = A b and s - A^* dh at 7 digits (28 each), b - A^* h and
    r = A s at 9 (45 each), plus the two m x m products per pass at 7; at the measured peaks
    the pairs' tensor floor (0.366 ms) is above the bytes' HBM floor (0.168 ms)."""
    w = workloads.WORKLOADS["dense_512x65536"]
    opts = types.SimpleNamespace(apply_slices=7, resid_slices=9)
    pk = {"hbm_gbs": 6780.7, "bf16_tflops": 1947.8, "bf16_tflops_sustained": 1724.9, "_source": "test"}
    e = bench.apply_roofline(w, opts, 64, 1.0, 1, pk)
    flops = 2.0 * 512 * 65536 * 64 * (28 + 45 + 45 + 28) + 2 * 2 * 2.0 * 512 * 512 * 64 * 28
    t_pairs, t_bytes = flops / 1724.9e12, 1141112832 / 6780.7e9
    assert abs(e["frac_ceiling"] - t_bytes / t_pairs) < 1e-12
    assert 0.45 < e["frac_ceiling"] < 0.47


def test_qr_flop_count():
    w = workloads.WORKLOADS["dense_512x65536"]
    o = types.SimpleNamespace(sketch_slices=5, gram_slices=7, gram2_slices=4, apply_slices=7, resid_slices=9,
                              refine_passes=1, qr_form=0)
    work = bench.phase_work("mixed", w, o)
    flops, bound, kernel = work["qr"]
    assert flops == 2.0 * 516 * 512 ** 2 - 2.0 * 512 ** 3 / 3.0 and kernel == "qr_persistent_ff_kernel"


def test_pipeline_depth_is_capped_by_free_memory():
    """--pipeline handles, as many as fit in a third of the free device memory."""
    per = 2 << 30                                               # one handle's workspace

    class Lib:
        @staticmethod
        def rtproj_workspace_bytes(m, n, l, k, opts):
            return per

    rt = types.SimpleNamespace(load_library=lambda: Lib)
    P = types.SimpleNamespace(opts=ctypes.c_int(0))             # stands in for the handle's rtproj_opts
    w = workloads.WORKLOADS["dense_512x65536"]

    def depth(pipeline, free):
        torch = types.SimpleNamespace(cuda=types.SimpleNamespace(mem_get_info=lambda dev: (free, 2 * free)))
        return bench.pipeline_depth(torch, rt, types.SimpleNamespace(pipeline=pipeline), w, {}, P, None)

    assert depth(6, 270 << 30) == 6                             # the headline size on a GB300
    assert depth(6, 12 * per) == 4                              # a third of the room: four handles
    assert depth(6, per) == 1                                   # never fewer than one
    assert depth(1, 270 << 30) == 1
