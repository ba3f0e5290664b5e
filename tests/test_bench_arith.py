"""The bench's roofline arithmetic (CPU): digit-pair counts of the sliced products and the
apply's algorithmic bytes, against hand counts."""
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


def test_qr_flop_count():
    w = workloads.WORKLOADS["dense_512x65536"]
    o = types.SimpleNamespace(sketch_slices=5, gram_slices=7, gram2_slices=4, apply_slices=7, resid_slices=9,
                              refine_passes=1, qr_form=0)
    work = bench.phase_work("mixed", w, o)
    flops, bound, kernel = work["qr"]
    assert flops == 2.0 * 516 * 512 ** 2 - 2.0 * 512 ** 3 / 3.0 and kernel == "qr_persistent_ff_kernel"
