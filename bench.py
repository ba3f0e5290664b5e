"""Benchmark: null-space projections per second on one GB300, mixed vs float64 form.

One step = the whole hot path on one batch: rtproj_precondition(seed, l) -- the sketch
S = A G with G generated on the device, the pivoted QR of S^*, the Gram matrix and its
Cholesky factor -- followed by rtproj_null_project on k right-hand sides (with the
refinement pass in the mixed form). value = k * steps / (device time of the timed
steps), all ranks together; each rank runs an independent replica (one GPU each).

Workload (synthetic, seeded): A = U diag(sigma) V^T, 512 x 65536 float64, U and V Haar,
sigma log-spaced over [1e-10, 1]; G standard normal (Box-Muller on Philox4x32-10), l = m + 4 = 516;
k = 64 right-hand sides with N(0,1) entries. A (268 MB) is larger than L2 (129 MB).
The line also carries the plain float64 form measured on the same workload (the
comparison the metric names) and the accuracy of both against the exact oracle.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}
# GB300 FP64 pipe: 152 SMs x 2 DFMA/clk/SM x 2 flop at the 2070 MHz maximum SM clock.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2070e6 / 1e12

METRIC = "null-space projections/s & % roofline, mixed vs FP64 form at <=1e-10 rel err"

# Options a workload's precision needs beyond the defaults: at kappa = 1e12 the sketch takes
# six digits (its error, 2^-48 relative, must stay below sigma_min / sigma_max = 1e-12), the
# rank test's threshold sits below 1/kappa, the refinement residuals take ten digits
# (2^-80 kappa ~ 1e-12) and the refinement runs to a tolerance.
WORKLOAD_OPTS = {"dense_2048x262144": dict(sketch_slices=6, resid_slices=10, refine_passes=4, refine_tol=1e-11,
                                           rank_tol=1e-14)}
# Workloads whose Haar factor is formed on the device (its host QR takes minutes).
DEVICE_GENERATED = {"dense_2048x262144"}


def workload_key(w):
    return next((k for k, v in workloads.WORKLOADS.items() if v.name == w.name), None)


def apply_roofline(w, opts, k, ms_call, passes, pk):
    """The apply (null_project on k right-hand sides) against the HBM roof, on the method's
    own bytes: A read as float64 once for c = A b and once for b - A^* h, twice more per
    refinement pass (r = A s and s - A^* dh), plus B read and Z written and the m x k
    solution; next to it, the tensor pipe's share for the digit-pair products the exact
    slicing performs (the emulation's work, labelled as such), and the float64-equivalent
    flop rate against the FP64 pipe."""
    m, n = w.m, w.n
    ap, rs = opts.apply_slices, opts.resid_slices
    bytes_alg = (2 + 2 * passes) * m * n * 8 + n * k * 16 + m * k * 8
    t = ms_call * 1e-3
    hbm = bytes_alg / t / 1e9
    pairs = digit_pairs(ap, ap, ap) + digit_pairs(rs, rs, rs) + passes * (digit_pairs(rs, rs, rs) + digit_pairs(ap, ap, ap))
    tensor_flops = 2.0 * m * n * k * pairs + (1 + passes) * 2 * 2.0 * m * m * k * digit_pairs(ap, ap, ap)
    tpeak = float(pk.get("bf16_tflops_sustained") or pk["bf16_tflops"])
    fp64_equiv = 4.0 * m * n * k * (1 + passes)
    # the HBM fraction of a call that took the longer of its two floors: the method's bytes
    # at the HBM peak, the digit pairs at the tensor peak
    t_bytes = bytes_alg / (float(pk["hbm_gbs"]) * 1e9)
    t_pairs = tensor_flops / (tpeak * 1e12)
    return {
        "bound": "hbm", "achieved": hbm, "peak": float(pk["hbm_gbs"]), "unit": "GB/s", "frac": hbm / float(pk["hbm_gbs"]),
        "frac_ceiling": t_bytes / max(t_bytes, t_pairs),
        "frac_ceiling_note": "HBM fraction at the larger of the bytes' HBM floor and the digit pairs' tensor floor",
        "bytes_per_call": bytes_alg, "ms_per_call": ms_call, "peak_source": f"{pk['_source']} hbm_gbs",
        "tensor_digit_pairs": {"achieved": tensor_flops / t / 1e12, "peak": tpeak, "unit": "TFLOP/s",
                               "frac": tensor_flops / t / 1e12 / tpeak,
                               "note": "bf16 tensor flops of the digit-pair products of the exact slicing "
                                       "(the emulation's work, not the method's float64 flops)"},
        "fp64_equivalent": {"achieved": fp64_equiv / t / 1e12, "fp64_pipe_peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                            "note": "4 m n k (1 + passes) float64 flops of the same products per call"},
    }


def peaks():
    if os.path.exists(MEASURED_PEAKS):
        with open(MEASURED_PEAKS) as f:
            p = json.load(f)
        p["_source"] = "measured"
        return p
    p = dict(FALLBACK_PEAKS)
    p["_source"] = "fallback"
    return p


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def setup_dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """Largest value of x over the ranks (the slowest replica sets the job time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, k: int, steps: int, ms_max: float) -> float:
    """Whole-job projections/s: every rank projects k right-hand sides per step on its own
    replica, and the job takes as long as the slowest rank."""
    return world * k * steps / (ms_max * 1e-3)


def cpu_oracle_step(A, B):
    from oracle import reference
    t0 = time.perf_counter()
    reference.project(A, B)
    return time.perf_counter() - t0


def cpu_cores() -> int:
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n and n[0]:
            return int(n[0])
    except Exception:
        pass
    return os.cpu_count() or 1


def cpu_baseline(A, B, budget_s: float = 12.0):
    """The oracle's Householder-QR definition (oracle.reference.project) on the same A and
    all k right-hand sides, repeated until ~budget_s of CPU work."""
    times = []
    t_end = time.perf_counter() + budget_s
    while time.perf_counter() < t_end or not times:
        times.append(cpu_oracle_step(A, B))
        if len(times) >= 20:
            break
    t = statistics.median(times)
    return {"value": B.shape[0] / t, "unit": "projections/s", "cores": cpu_cores(), "kind": "oracle",
            "sample": f"oracle.reference.project (Householder QR of A^T + apply) on the full {A.shape[0]}x{A.shape[1]} "
                      f"A and all {B.shape[0]} RHS, median of {len(times)} runs"}


def run_reference(args, w, world, rank):
    if rank != 0:
        return 0
    A = w.matrix()
    B = w.rhs()
    for _ in range(args.warmup):
        cpu_oracle_step(A, B)
    ts = [cpu_oracle_step(A, B) for _ in range(args.steps)]
    total = sum(ts)
    value = w.k * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "projections/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "m": w.m, "n": w.n, "k": w.k, "l": w.l, "kappa": 1.0 / w.sigma_min,
                   "l2": "inputs larger than L2"},
        "cpu_baseline": {"value": value, "unit": "projections/s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": "oracle.reference.project on the full workload per step"},
        "e2e": {"value": value, "unit": "projections/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def time_steps(torch, P, Bt, seed, l, steps, stream):
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for i in range(steps):
        P.precondition(seed + i, l)
        P.null_project(Bt, out=Zbuf_of(P, Bt))
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1)


def pipeline_depth(torch, rt, args, w, wopts, P, dev):
    """Handles for the pipelined steps: --pipeline, as many as fit in a third of the free
    device memory (each handle holds its own digit planes of A and its own buffers)."""
    if args.pipeline <= 1:
        return 1
    import ctypes
    o = P.opts
    per = int(rt.load_library().rtproj_workspace_bytes(w.m, w.n, w.l, w.k, ctypes.byref(o)))
    free = torch.cuda.mem_get_info(dev)[0]
    return max(1, min(args.pipeline, free // 3 // max(per, 1)))


def time_steps_pipelined(torch, Ps, Bt, seed, l, steps, stream, Zs):
    """The same steps on len(Ps) handles bound to the same A, each on its own stream and in
    the asynchronous mode: step i runs on handle i mod len(Ps), so a step's apply (tensor
    cores) overlaps the next step's precondition, whose pivoted QR and Cholesky are bound by
    the latency of their sequential steps and leave the SMs' pipes mostly idle."""
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for P in Ps:
        P.stream.wait_stream(stream)
    for i in range(steps):
        P = Ps[i % len(Ps)]
        # issued with the handle's stream current, so that the binding adds no wait on
        # another stream: consecutive steps are ordered only through their own handle
        with torch.cuda.stream(P.stream):
            P.precondition(seed + i, l)
            P.null_project(Bt, out=Zs[i % len(Ps)])
    for P in Ps:
        stream.wait_stream(P.stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1)


_ZBUF = {}


def Zbuf_of(P, Bt):
    key = id(P)
    if key not in _ZBUF:
        import torch
        _ZBUF[key] = torch.empty_like(Bt)
    return _ZBUF[key]


def digit_pairs(sa, sb, terms):
    """Digit pairs (p, q) with p < sa, q < sb, p + q < terms multiplied by the sliced GEMM."""
    return sum(1 for p in range(sa) for q in range(sb) if p + q < terms)


def phase_work(mode, w, o):
    """Algorithmic work per step of each timed phase: (flops, unit, bound, kernel).

    float64 form: float64 flops of each product. Mixed form: bf16 tensor flops of the
    digit-pair products the Ozaki scheme performs (2 M N K per pair), since that is the
    work the tensor pipe must do; QR and factor phases stay float64 (FP64 pipe)."""
    m, n, l, k = w.m, w.n, w.l, w.k
    qr = 2.0 * l * m * m - 2.0 * m ** 3 / 3.0
    if mode == "fp64":
        return {
            "sketch": (2.0 * m * n * l, "alu", "gemm64_kernel"),
            "gram": (2.0 * m * m * n + m * m * n, "alu", "gemm64_kernel"),
            "apply_a": (2.0 * m * n * k, "alu", "gemm64_kernel"),
            "apply_at": (2.0 * m * n * k, "alu", "gemm64_kernel"),
            "qr": (qr, "alu", "qr_persistent_kernel"),
        }
    sk, g1, g2, ap, rs = o.sketch_slices, o.gram_slices, o.gram2_slices, o.apply_slices, o.resid_slices
    passes = o.refine_passes
    return {
        "sketch": (2.0 * m * n * l * digit_pairs(1, sk, sk), "tensor", "sliced_gemm2_kernel"),
        "gram": (2.0 * m * m * n * digit_pairs(g1, g1, g1) + 2.0 * m * m * n * digit_pairs(g2, g2, g2) * 0.5,
                 "tensor", "sliced_gemm2_kernel"),
        "apply_a": (2.0 * m * n * k * (digit_pairs(ap, ap, ap) + passes * digit_pairs(rs, rs, rs)), "tensor",
                    "sliced_gemm2_kernel"),
        "apply_at": (2.0 * m * n * k * (digit_pairs(rs, rs, rs) + passes * digit_pairs(ap, ap, ap)), "tensor",
                     "sliced_gemm2_kernel"),
        # float-float on the FP32 pipe; counted as the float64 work it replaces, against the
        # FP64 pipe (the kernel is bound by the latency of its m sequential grid exchanges)
        "qr": (qr, "alu", "qr_persistent_ff_kernel" if getattr(o, "qr_form", 0) == 0 else "qr_persistent_kernel"),
    }


# DRAM bytes (read + write) per launch of a kernel, from one ncu capture of
# `bench.py --steps 1 --warmup 3 --no-e2e --no-cpu-baseline --no-accuracy --no-fp64-form`
# on the 512 x 65536 workload; to be replaced by None whenever that kernel changes.
PROFILED_TRAFFIC = {("dense_512x65536", "qr_persistent_kernel"): 2160128 + 217600,
                    ("dense_512x65536", "qr_persistent_ff_kernel"): 2189568 + 289024}


def roofline_entry(mode, phase_ms, phase_cnt, steps, w, pk, opts):
    """Per-phase achieved rate against its peak, and the entry for the dominant phase."""
    work = phase_work(mode, w, opts)
    tensor_peak = float(pk.get("bf16_tflops_sustained") or pk["bf16_tflops"])
    phases = {}
    for ph, (flops, bound, kernel) in work.items():
        ms = phase_ms.get(ph, 0.0)
        if ms <= 0:
            continue
        achieved = flops * steps / (ms * 1e-3) / 1e12
        peak = tensor_peak if bound == "tensor" else FP64_PEAK_TFLOPS
        phases[ph] = {"bound": bound, "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                      "frac": achieved / peak, "ms_per_step": ms / steps}
    dom = max(phases, key=lambda p: phases[p]["ms_per_step"])
    e = dict(phases[dom])
    e.pop("ms_per_step")
    e["phase"] = dom
    key = next((k for k in workloads.WORKLOADS if workloads.WORKLOADS[k].name == w.name), None)
    e["traffic"] = PROFILED_TRAFFIC.get((key, e["kernel"])) if w.l == workloads.WORKLOADS.get(key, w).l else None
    e["peak_source"] = (f"{pk['_source']} bf16_tflops_sustained" if e["bound"] == "tensor"
                        else "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (FP64 pipe)")
    return e, phases


def run_ours(args, w, world, rank, local):
    import torch
    import paper_0912_1135_gb300 as rt
    from oracle import exact, metrics

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pk = peaks()
    key = workload_key(w)
    wopts = dict(WORKLOAD_OPTS.get(key, {})) if args.mode == "mixed" else {}
    for kv in args.opt or []:                 # --opt name=value: an rtproj_opts field
        name, val = kv.split("=", 1)
        wopts[name] = float(val) if name.endswith("_tol") else int(val)
    A = w.matrix(device=dev) if key in DEVICE_GENERATED else w.matrix()
    B = w.rhs()
    At = torch.from_numpy(A).to(dev)
    Bt = torch.from_numpy(B).to(dev)
    stream = torch.cuda.current_stream(dev)
    seed0 = w.seed_omega
    out = {}

    P = rt.Projector(At, l_max=w.l, k_max=w.k, mode=args.mode, timing=1, **wopts)
    for i in range(args.warmup):
        P.precondition(seed0 + i, w.l)
        P.null_project(Bt, out=Zbuf_of(P, Bt))
    torch.cuda.synchronize()
    P.timings()
    pipe = []
    depth = pipeline_depth(torch, rt, args, w, wopts, P, dev)
    if depth > 1:
        pipe = [rt.Projector(At, l_max=w.l, k_max=w.k, mode=args.mode, stream=torch.cuda.Stream(dev), async_=1,
                             **wopts) for _ in range(depth)]
        Zs = [torch.empty_like(Bt) for _ in pipe]
        time_steps_pipelined(torch, pipe, Bt, seed0, w.l, args.warmup, stream, Zs)
    launches0 = rt.launch_count()
    sampler = ClockSampler(local)
    sampler.start()
    barrier(world)
    if pipe:
        ms = time_steps_pipelined(torch, pipe, Bt, seed0 + 1000, w.l, args.steps, stream, Zs)
    else:
        ms = time_steps(torch, P, Bt, seed0 + 1000, w.l, args.steps, stream)
    barrier(world)
    clocks = sampler.stop()
    launches = rt.launch_count() - launches0
    if pipe:
        bad = sum(1 for Q in pipe if Q.info()["status"] != 0)
        if bad:
            raise RuntimeError(f"{bad} pipelined handles latched a nonzero status")
        Zbuf_of(P, Bt).copy_(Zs[(args.steps - 1) % len(pipe)])
        for Q in pipe:
            Q.close()
        # the per-phase breakdown comes from the same steps run one after another
        time_steps(torch, P, Bt, seed0 + 1000, w.l, args.steps, stream)
    tim = P.timings()
    ms_max = max_over_ranks(ms, world)
    value = job_throughput(world, w.k, args.steps, ms_max)
    phase_ms = {p: v[0] for p, v in tim.items()}
    phase_cnt = {p: v[1] for p, v in tim.items()}

    # accuracy of the timed configuration: sampled RHS against the exact oracle
    Z = Zbuf_of(P, Bt).cpu().numpy()
    info = P.info()
    acc = {"library_resid_rel": info["resid_rel"], "refine_passes": info["passes"]}
    if key in DEVICE_GENERATED:
        # beyond the exact oracle's reach: ||A z|| in double-double on sampled RHS
        nb = np.linalg.norm(B, axis=1)
        acc["normalised_residual_sampled"] = float(max(exact.exact_residual(A, Z[j:j + 1])[0] / nb[j] for j in (0, w.k - 1)))
    else:
        acc["normalised_residual_max"] = metrics.normalised_residual(A, Z, B, normA=1.0)
        if not args.no_accuracy and rank == 0:
            Zx, _, _ = exact.exact_project(A, B[:1])
            acc["z_rel_err_vs_exact_oracle"] = metrics.max_rel_err(Z[:1], Zx)
            acc["sample"] = "RHS 0 against oracle.exact (double-double refinement)"
    P.close()

    line = {
        "metric": METRIC, "value": value, "unit": "projections/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.mode == "fp64" else "bf16-slices/f64",
        "data": "synthetic",
        "config": {"workload": w.name, "mode": args.mode, "m": w.m, "n": w.n, "k": w.k, "l": w.l,
                   "kappa": 1.0 / w.sigma_min, "omega": "gaussian (Box-Muller on Philox4x32-10, 2^-12 grid)",
                   "step": "precondition(seed, l) + null_project(k RHS)",
                   "pipeline": (f"up to {depth} consecutive steps in flight, each on its own handle and stream: "
                                "their latency-bound QRs and Cholesky factorizations share the SMs, and so do their "
                                "tensor-core products") if depth > 1 else "one handle, steps in order",
                   "l2": f"inputs larger than L2 (A is {A.nbytes / 1e6:.0f} MB float64)",
                   "parallelism": f"replicas x{world}", "options": wopts},
        "phase_ms_per_step": {p: phase_ms[p] / args.steps for p in phase_ms if phase_cnt[p]},
        "accuracy": acc,
        "clocks": clocks,
        "gpu_launches": int(launches),
    }
    rl, rl_phases = roofline_entry(args.mode, phase_ms, phase_cnt, args.steps, w, pk, P.opts)
    line["roofline"] = rl
    line["roofline_phases"] = rl_phases

    with rt.Projector(At, l_max=w.l, k_max=w.k, mode=args.mode, **wopts) as P2:
        line["split"] = split_times(torch, P2, Bt, w, args, stream)
        if args.mode == "mixed":
            passes = P2.info()["passes"]
            ap = apply_roofline(w, P2.opts, w.k, line["split"]["null_project_ms"], passes, pk)
            ap["projections_per_s"] = line["split"]["projection_only"]["value"]
            line["apply"] = ap
        if key in DEVICE_GENERATED:
            line["per_k"] = per_k_times(torch, P2, Bt, w, pk, A, B)
    if key in DEVICE_GENERATED and not args.no_accuracy and rank == 0:
        line["paper_family"] = paper_family_errors(torch, rt, w, args, wopts, dev)
    if args.mode == "mixed" and not args.no_fp64_form:
        line["fp64_form"] = fp64_form(torch, rt, A, B, At, Bt, w, args, rank)
    if not args.no_e2e:
        line["e2e"] = e2e(torch, rt, A, B, w, args, dev, wopts)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(A, B)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def per_k_times(torch, P, Bt, w, pk, A, B):
    """null_project at k = 1, 16 and the workload's k with one preconditioner: device time
    per call (median of 10 after 2 warm-up calls), projections/s, the apply's HBM roofline
    and ||A z|| in double-double on the first right-hand side."""
    from oracle import exact
    out = {}
    stream = torch.cuda.current_stream(Bt.device)
    for k in sorted({1, 16, w.k}):
        Bk = Bt[:k]
        Zk = torch.empty_like(Bk)
        for _ in range(2):
            P.null_project(Bk, out=Zk)
        times = []
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            P.null_project(Bk, out=Zk)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = statistics.median(times)
        info = P.info()
        z0 = Zk[:1].cpu().numpy()
        r = float(exact.exact_residual(A, z0)[0] / np.linalg.norm(B[0]))
        out[str(k)] = {"ms_per_call": ms, "projections_per_s": k / (ms * 1e-3), "refine_passes": info["passes"],
                       "normalised_residual_rhs0": r,
                       "roofline": apply_roofline(w, P.opts, k, ms, info["passes"], pk)}
    return out


def paper_family_errors(torch, rt, w, args, wopts, dev):
    """Z against the closed form of the paper's own family (Eqs. 20-21) at the workload's
    size and kappa, for 16 right-hand sides, at k = 1, 16 and the workload's k."""
    from oracle import closed_form, metrics
    A, Bb, pu, pv = w.paper_family(return_parts=True)
    B = w.rhs()
    Zc, _, _ = closed_form.project(Bb, pu, pv, B[:16])
    out = {}
    with rt.Projector(torch.from_numpy(A).to(dev), l_max=w.l, k_max=w.k, mode=args.mode, **wopts) as P:
        del A
        P.precondition(w.seed_omega, w.l)
        Bt = torch.from_numpy(B).to(dev)
        for k in sorted({1, 16, w.k}):
            Z = P.null_project(Bt[:k]).cpu().numpy()
            kk = min(k, 16)
            out[str(k)] = metrics.max_rel_err(Z[:kk], Zc[:kk])
    return {"z_rel_err_vs_closed_form": out, "matrix": "U [B|...|B] V of Eqs. 20-21, same m, n, kappa"}


def split_times(torch, P, Bt, w, args, stream):
    """The two halves of a step timed apart, as the paper's t_pre and t_pro: preconditioning
    alone, then null_project calls that reuse one preconditioner (projections/s of the apply
    path with the preconditioner amortised)."""
    calls = max(args.steps, 10)
    P.precondition(w.seed_omega, w.l)
    P.null_project(Bt, out=Zbuf_of(P, Bt))
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(stream)
    for i in range(calls):
        P.precondition(w.seed_omega + 3000 + i, w.l)
    ev[1].record(stream)
    ev[2].record(stream)
    for _ in range(calls):
        P.null_project(Bt, out=Zbuf_of(P, Bt))
    ev[3].record(stream)
    torch.cuda.synchronize()
    pre = ev[0].elapsed_time(ev[1]) / calls
    pro = ev[2].elapsed_time(ev[3]) / calls
    return {"precondition_ms": pre, "null_project_ms": pro,
            "projection_only": {"value": w.k / (pro * 1e-3), "unit": "projections/s", "calls": calls,
                                "note": "null_project on k RHS with the preconditioner reused (t_pro analogue)"}}


def fp64_form(torch, rt, A, B, At, Bt, w, args, rank):
    """The plain float64 GPU form on the same workload: a few steps, device-timed, and
    its error on RHS 0 against the exact oracle."""
    from oracle import exact, metrics
    steps = 3
    P = rt.Projector(At, l_max=w.l, k_max=w.k, mode="fp64")
    try:
        P.precondition(w.seed_omega, w.l)
    except rt.RtprojError as e:
        P.close()
        return {"error": str(e)}
    P.null_project(Bt, out=Zbuf_of(P, Bt))
    stream = torch.cuda.current_stream(At.device)
    ms = time_steps(torch, P, Bt, w.seed_omega + 2000, w.l, steps, stream)
    out = {"value": w.k * steps / (ms * 1e-3), "unit": "projections/s", "ms_per_step": ms / steps, "steps": steps}
    if not args.no_accuracy and rank == 0:
        Z = Zbuf_of(P, Bt).cpu().numpy()
        if workload_key(w) in DEVICE_GENERATED:
            out["normalised_residual_rhs0"] = float(exact.exact_residual(A, Z[:1])[0] / np.linalg.norm(B[0]))
        else:
            Zx, _, _ = exact.exact_project(A, B[:1])
            out["z_rel_err_vs_exact_oracle"] = metrics.max_rel_err(Z[:1], Zx)
            out["normalised_residual_max"] = metrics.normalised_residual(A, Z, B, normA=1.0)
    P.close()
    return out


def e2e(torch, rt, A, B, w, args, dev, wopts):
    """Same metric through the public API from pinned host buffers. Every step copies its A
    and B host-to-device, creates a Projector (A is sliced at create), preconditions,
    projects and copies Z device-to-host, all inside the timed region. As a serving loop
    would, the next step's host-to-device copies run on a second stream while the current
    step computes (two device buffers for A and B), and each step's device-to-host copy of
    Z runs on a third stream while the next step computes. The handles run in the
    asynchronous mode (no host synchronization inside create or precondition); every
    handle's latched status is read after the timed region."""
    Ah = torch.from_numpy(A).pin_memory()
    Bh = torch.from_numpy(B).pin_memory()
    npipe = max(1, min(args.pipeline, 4))               # steps in flight, one compute stream each
    Zh = [torch.empty(B.shape, dtype=torch.float64).pin_memory() for _ in range(npipe)]
    # every step's handle stays alive until the end: as many steps as fit in half the free
    # memory besides the device copies of A and B
    import ctypes
    o = rt.make_opts(args.mode, **wopts)
    per = int(rt.load_library().rtproj_workspace_bytes(w.m, w.n, w.l, w.k, ctypes.byref(o)))
    room = torch.cuda.mem_get_info(dev)[0] // 2 - npipe * (A.nbytes + B.nbytes)
    steps = max(1, min(args.steps, 15, room // max(per, 1) - 1))
    comp = torch.cuda.current_stream(dev)
    comps = [torch.cuda.Stream(dev) for _ in range(npipe)]
    copy = torch.cuda.Stream(dev)
    d2h = torch.cuda.Stream(dev)
    Ad = [torch.empty(A.shape, dtype=torch.float64, device=dev) for _ in range(npipe)]
    Bd = [torch.empty(B.shape, dtype=torch.float64, device=dev) for _ in range(npipe)]
    copied = [torch.cuda.Event() for _ in range(npipe)]
    freed = [torch.cuda.Event() for _ in range(npipe)]
    for ev in freed:
        ev.record(comp)

    def issue_copy(i):
        s = i % npipe
        with torch.cuda.stream(copy):
            copy.wait_event(freed[s])          # the buffers' previous step is done with them
            Ad[s].copy_(Ah, non_blocking=True)
            Bd[s].copy_(Bh, non_blocking=True)
            copied[s].record(copy)

    handles = []

    def run(i):
        s = i % npipe
        cs = comps[s]
        with torch.cuda.stream(cs):
            cs.wait_event(copied[s])
            P = rt.Projector(Ad[s], l_max=w.l, k_max=w.k, mode=args.mode, stream=cs, async_=1, **wopts)
            P.precondition(w.seed_omega + i, w.l)
            Z = P.null_project(Bd[s])
            handles.append(P)
            freed[s].record(cs)
        d2h.wait_event(freed[s])
        with torch.cuda.stream(d2h):
            Zh[s].copy_(Z, non_blocking=True)
        Z.record_stream(d2h)                   # Z stays allocated until its copy is done

    issue_copy(0)
    run(0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    issue_copy(1)
    for i in range(1, steps + 1):
        if i + 1 <= steps:
            issue_copy(i + 1)
        run(i)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    bad = sum(1 for P in handles if P.info()["status"] != 0)
    for P in handles:
        P.close()
    return {"value": w.k * steps / wall, "unit": "projections/s", "h2d_bytes_per_step": int(A.nbytes + B.nbytes),
            "d2h_bytes_per_step": int(B.nbytes), "steps": steps, "handles_with_nonzero_status": bad,
            "pipelining": f"consecutive steps compute on {npipe} rotating streams; the next step's H2D "
                          "copies and the previous step's D2H copy overlap the compute (two more streams); "
                          "asynchronous handles"}


def _family_errors(torch, rt, dev, m, n, l, kappa, mode, nb=100, seed=5, **kw):
    """delta/kappa and epsilon/kappa of Section 5 (max over nb random unit b) on the paper's
    family, with ||A z|| accumulated in double-double through the family's structure; also
    the device times of precondition and of the projection of the nb vectors."""
    from oracle import closed_form
    A, Bb, pu, pv = workloads.paper_test_matrix(m, n, kappa, seed, return_parts=True)
    B = workloads.rhs(nb, n, seed + 1)
    B /= np.linalg.norm(B, axis=1, keepdims=True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    with rt.Projector(torch.from_numpy(A).to(dev), l_max=l, k_max=nb, mode=mode, **kw) as P:
        del A
        Bt = torch.from_numpy(B).to(dev)
        P.precondition(seed + 2, l)
        P.null_project(Bt)
        stream = torch.cuda.current_stream(dev)
        ev[0].record(stream)
        P.precondition(seed + 2, l)
        ev[1].record(stream)
        ev[2].record(stream)
        Z = P.null_project(Bt)
        ev[3].record(stream)
        torch.cuda.synchronize()
        ZZ = P.null_project(Z.clone()).cpu().numpy()
        Z = Z.cpu().numpy()
    delta = float(np.max(np.linalg.norm(closed_form.apply_A(Bb, pu, pv, Z), axis=1)))
    eps = float(np.max(np.linalg.norm(Z - ZZ, axis=1)))
    return {"delta_over_kappa": delta / kappa, "epsilon_over_kappa": eps / kappa,
            "precondition_ms": ev[0].elapsed_time(ev[1]), "project_ms": ev[2].elapsed_time(ev[3])}


def study_accuracy(args):
    """Section 5, Tables 2 and 4 (the randomized method's columns) on the GPU: the rows that
    fit one GB300 at the paper's sizes, and the kappa sweep at m = 1000, n = 100000 (the
    paper's sweep is m = 4000, n = 10^6), in both arithmetic forms, next to the values the
    paper prints for its float64 CPU runs."""
    import torch
    import paper_0912_1135_gb300 as rt
    golden = json.load(open(os.path.join(ROOT, "tests", "golden", "section5_randomized_errors.json")))
    printed = {(r["m"], r["n"], r["l"], r["kappa"]): r for r in golden["table2"]}
    printed4 = {r["kappa"]: r for r in golden["table4"]}
    dev = torch.device("cuda", 0)
    rows = [(40, 10 ** 6, 44, 1e8), (400, 10 ** 6, 404, 1e8), (1000, 3000, 1004, 1e8), (1000, 30000, 1004, 1e8),
            (1000, 300000, 1004, 1e8)] + [(1000, 100000, 1004, k) for k in (1e4, 1e6, 1e8, 1e10, 1e12)]
    out = []
    for (m, n, l, kappa) in rows:
        row = {"m": m, "n": n, "l": l, "kappa": kappa}
        mixed_kw = dict(WORKLOAD_OPTS["dense_2048x262144"]) if kappa > 1e10 else dict(refine_passes=4,
                                                                                          refine_tol=1e-12)
        for form, kw in (("mixed", mixed_kw), ("fp64", {})):
            try:
                row[form] = _family_errors(torch, rt, dev, m, n, l, kappa, form, **kw)
            except rt.RtprojError as e:
                row[form] = {"error": str(e)}
        ref = printed.get((m, n, l, kappa)) or (printed4.get(kappa) if n == 100000 else None)
        if ref:
            row["paper"] = {"delta_over_kappa": ref["delta_over_kappa"], "epsilon_over_kappa": ref["epsilon_over_kappa"],
                            "row": f"{ref['m']} x {ref['n']}, l = {ref['l']}"}
        out.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    print(json.dumps({"study": "section5_accuracy", "omega": "gaussian", "rhs": "100 random unit b per row",
                      "rows": out}), flush=True)
    return 0


def study_variates(args):
    """Variates and sketch sizes (Section 5's remarks on the choice of G; Table 1's l rows):
    for each distribution of G and l in {m, m + 4, 2m, 4m} on the headline workload, the
    device time of precondition, kappa(P^{-1} A) from the GPU's R and Pi, the library's
    estimate, and the mixed form's error on RHS 0 against the exact oracle."""
    import scipy.linalg as sla
    import torch
    import paper_0912_1135_gb300 as rt
    from oracle import exact, metrics
    w = workloads.WORKLOADS["dense_512x65536"]
    A = w.matrix()
    B = w.rhs()
    Zx, _, _ = exact.exact_project(A, B[:1])
    dev = torch.device("cuda", 0)
    At = torch.from_numpy(A).to(dev)
    Bt = torch.from_numpy(B).to(dev)
    out = []
    for dist in ("gaussian", "uniform", "rademacher"):
        for l in (w.m, w.m + 4, 2 * w.m, 4 * w.m):
            with rt.Projector(At, l_max=l, k_max=w.k, omega=dist) as P:
                times, refused = [], []
                for i in range(6):                   # seed 0 untimed; a refused seed is recorded
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    try:
                        P.precondition(w.seed_omega + i, l)
                    except rt.RtprojError as e:
                        refused.append({"seed": w.seed_omega + i, "status": str(e)})
                        continue
                    e1.record()
                    torch.cuda.synchronize()
                    if i:
                        times.append(e0.elapsed_time(e1))
                ok_seed = next((w.seed_omega + i for i in range(6)
                                if all(r["seed"] != w.seed_omega + i for r in refused)), None)
                if ok_seed is None or not times:
                    out.append({"omega": dist, "l": l, "refused_seeds": refused})
                    print(json.dumps(out[-1]), file=sys.stderr, flush=True)
                    continue
                P.precondition(ok_seed, l)
                Z = P.null_project(Bt).cpu().numpy()
                info = P.info()
                R, perm, _ = P.export_state()
            W = sla.solve_triangular(R.T, A[perm], lower=True)
            s = np.linalg.svd(W, compute_uv=False)
            row = {"omega": dist, "l": l, "precondition_ms": statistics.median(times), "kappa_PinvA": float(s[0] / s[-1]),
                   "kappa_pre_estimate": info["kappa_pre"], "z_rel_err_rhs0": metrics.max_rel_err(Z[:1], Zx),
                   "refused_seeds": refused}
            out.append(row)
            print(json.dumps(row), file=sys.stderr, flush=True)
    print(json.dumps({"study": "variates_and_sketch_size", "workload": w.name, "rows": out}), flush=True)
    return 0


def study_batch(args):
    """Batching (the interior-point and many-instance configuration):
    (a) 500 independent float32 instances, m = round(exp U(ln 16, ln 512)),
        n = round(m exp U(ln 4, ln 64)) rounded up to a multiple of 16, sigma over [1e-4, 1],
        l = 2m + 32, 32 right-hand sides each, seeds 1000 + i: one step (every instance's
        precondition and null_project) timed eagerly on 8 streams and as one CUDA-graph replay;
    (b) A 1024 x 32768 (sigma over [1e-8, 1]) under 64 scalings A diag(d_j), d_j log-uniform
        over [1e-6, 1e6] (seed 400 + j), 32 right-hand sides each: set_scaling, precondition and
        null_project per scaling, timed over the sequence; the library's residual report and
        kappa estimates per scaling."""
    import torch
    import paper_0912_1135_gb300 as rt
    from paper_0912_1135_gb300.batch import Batch
    dev = torch.device("cuda", 0)
    out = {"study": "batching"}
    # (a) uneven instances
    rng = np.random.default_rng(999)
    count = int(os.environ.get("RTPROJ_BATCH_COUNT", "500"))
    sizes = []
    for i in range(count):
        m = int(round(np.exp(rng.uniform(np.log(16), np.log(512)))))
        n = int(round(m * np.exp(rng.uniform(np.log(4), np.log(64)))))
        n = max(2 * m + 32, (n + 15) // 16 * 16)
        sizes.append((m, n))
    k = 32
    As = [torch.from_numpy(workloads.haar_spectrum_matrix(m, n, 1e-4, 1000 + i, dtype=np.float32)).to(dev)
          for i, (m, n) in enumerate(sizes)]
    Bs = [torch.from_numpy(workloads.rhs(k, n, 5000 + i, dtype=np.float32)).to(dev) for i, (m, n) in enumerate(sizes)]
    Zs = [torch.empty_like(B) for B in Bs]
    bt = Batch(As, [k] * count, [2 * m + 32 for m, _ in sizes], streams=8)
    seeds = [7000 + i for i in range(count)]
    bt.step(Bs, seeds, Zs)
    torch.cuda.synchronize()
    reps = 3
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    for _ in range(reps):
        bt.step(Bs, seeds, Zs)
    ev[1].record()
    torch.cuda.synchronize()
    eager_ms = ev[0].elapsed_time(ev[1]) / reps
    t0 = time.perf_counter()
    bt.capture(Bs, seeds, Zs)
    capture_s = time.perf_counter() - t0
    bt.replay()
    torch.cuda.synchronize()
    ev[0].record()
    for _ in range(reps):
        bt.replay()
    ev[1].record()
    torch.cuda.synchronize()
    graph_ms = ev[0].elapsed_time(ev[1]) / reps
    st = bt.statuses()
    bt.close()
    mn = np.array([m * n for m, n in sizes], dtype=np.float64)
    out["instances"] = {"count": count, "k": k, "mean_mn": float(mn.mean()), "total_A_bytes_f32": float(4 * mn.sum()),
                        "eager_ms_per_step": eager_ms, "graph_ms_per_step": graph_ms, "graph_capture_s": capture_s,
                        "instances_per_s": count / (graph_ms * 1e-3), "projections_per_s": count * k / (graph_ms * 1e-3),
                        "nonzero_status": int(sum(1 for s in st if s != 0))}
    del As, Bs, Zs
    torch.cuda.empty_cache()
    # (b) interior-point scalings
    m, n, kk, J = 1024, 32768, 32, 64
    l = 2 * m + 32
    A = workloads.haar_spectrum_matrix(m, n, 1e-8, 4, device=dev)
    At = torch.from_numpy(A).to(dev)
    B = torch.from_numpy(workloads.rhs(kk, n, 24)).to(dev)
    Z = torch.empty_like(B)
    ds = [torch.from_numpy(10.0 ** np.random.default_rng(400 + j).uniform(-6, 6, n)).to(dev) for j in range(J)]
    per = []
    with rt.Projector(At, l_max=l, k_max=kk, scalable=1, refine_passes=3, refine_tol=1e-12) as P:
        P.set_scaling(ds[0])
        P.precondition(400, l)
        P.null_project(B, out=Z)
        torch.cuda.synchronize()
        ev[0].record()
        for j in range(J):
            P.set_scaling(ds[j])
            P.precondition(400 + j, l)
            P.null_project(B, out=Z)
            if j < 4 or j == J - 1:
                inf = P.info()
                per.append({"j": j, "status": inf["status"], "kappa_R": inf["kappa_R"], "kappa_pre": inf["kappa_pre"],
                            "resid_rel": inf["resid_rel"], "dh_rel": inf["dh_rel"], "passes": inf["passes"]})
        ev[1].record()
        torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1])
    out["scalings"] = {"m": m, "n": n, "k": kk, "l": l, "count": J, "ms_total": ms, "scalings_per_s": J / (ms * 1e-3),
                       "projections_per_s": J * kk / (ms * 1e-3), "sampled_reports": per,
                       "note": "each scaling: A diag(d_j) formed and sliced, preconditioned, 32 RHS projected; the "
                               "sampled reports synchronize"}
    print(json.dumps(out), flush=True)
    return 0


def _sparse_row(torch, rt, dev, m, n, l, kappa, low_rank, nb=100, seed=5, refine=(8, 1e-15)):
    """One row of Section 5's tables with the sparse operator form: the test matrix of
    Eq. 21 in compressed sparse row form (plus the rank-10 term of Eq. 22 when low_rank),
    precondition and projection device-timed (one vector, and nb vectors at once), and
    delta/kappa, epsilon/kappa over nb random unit b (||A z|| through the family's
    structure in double-double, the low-rank part in float64)."""
    from oracle import closed_form
    rp, ci, v, b, pu, pv = workloads.paper_test_csr(m, n, kappa, seed)
    U = V = None
    if low_rank:
        U, V = workloads.paper_low_rank(m, n, seed + 3)
    B = workloads.rhs(nb, n, seed + 1)
    B /= np.linalg.norm(B, axis=1, keepdims=True)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    out = {"m": m, "n": n, "l": l, "kappa": kappa, "nnz": int(len(v)), "low_rank": 10 if low_rank else 0}
    with rt.SparseProjector(t(rp), t(ci), t(v), n, U=t(U) if low_rank else None, V=t(V) if low_rank else None,
                            l_max=l, k_max=nb, refine_passes=refine[0], refine_tol=refine[1], timing=1) as P:
        Bt = t(B)
        P.precondition(seed + 2, l)
        P.null_project(Bt[:1])
        P.timings()
        P.precondition(seed + 2, l)
        out["precondition_phases_ms"] = {k: round(v[0], 3) for k, v in P.timings().items() if v[1]}
        stream = torch.cuda.current_stream(dev)
        ev[0].record(stream)
        P.precondition(seed + 2, l)
        ev[1].record(stream)
        ev[2].record(stream)
        P.null_project(Bt[:1])
        ev[3].record(stream)
        ev[4].record(stream)
        Z = P.null_project(Bt)
        ev[5].record(stream)
        torch.cuda.synchronize()
        inf = P.info()
        ZZ = P.null_project(Z.clone()).cpu().numpy()
        Z = Z.cpu().numpy()
    AZ = closed_form.apply_A(b, pu, pv, Z)
    if low_rank:
        AZ = AZ + (U @ (V @ Z.T)).T
    delta = float(np.max(np.linalg.norm(AZ, axis=1)))
    eps = float(np.max(np.linalg.norm(Z - ZZ, axis=1)))
    out.update({"t_pre_s": ev[0].elapsed_time(ev[1]) * 1e-3, "t_pro_s": ev[2].elapsed_time(ev[3]) * 1e-3,
                "t_pro_per_vector_batched_s": ev[4].elapsed_time(ev[5]) * 1e-3 / nb,
                "delta_over_kappa": delta / kappa, "epsilon_over_kappa": eps / kappa,
                "passes": inf["passes"], "kappa_pre": inf["kappa_pre"], "status": inf["status"]})
    if not low_rank:
        Zc, _, _ = closed_form.project(b, pu, pv, B)
        out["z_err_vs_closed_form"] = float(np.max(np.linalg.norm(Z - Zc, axis=1)))
    return out


def study_sparse(args):
    """Section 5, Tables 1-2 and 5-6, in the paper's own setting: A applied as a sparse
    operator (five nonzeros per column), and its sum with a rank-10 term, at the paper's
    sizes, next to the paper's printed timings (one 2009 CPU core) and errors."""
    import torch
    import paper_0912_1135_gb300 as rt
    gd = os.path.join(ROOT, "tests", "golden")
    tim = json.load(open(os.path.join(gd, "section5_timings.json")))
    err = json.load(open(os.path.join(gd, "section5_randomized_errors.json")))
    key = lambda r: (r["m"], r["n"], r["l"], r["kappa"])
    t1 = {key(r): r for r in tim["table1"]}
    t2 = {key(r): r for r in err["table2"]}
    t5 = {key(r): r for r in tim["table5"]}
    t6 = {key(r): r for r in tim["table6"]}
    dev = torch.device("cuda", 0)
    rows = []
    only = None
    if args.sparse_row:
        mm, nn, ll, kk = args.sparse_row.split(",")
        only = (int(mm), int(nn), int(ll), float(kk))
    for low_rank, tt, te in ((False, t1, t2), (True, t5, t6)):
        for k in tt:
            if only is not None and k != only:
                continue
            m, n, l, kappa = k
            try:
                r = _sparse_row(torch, rt, dev, m, n, l, kappa, low_rank)
            except rt.RtprojError as e:
                r = {"m": m, "n": n, "l": l, "kappa": kappa, "low_rank": 10 if low_rank else 0, "error": str(e)}
            r["paper"] = {"t_pre_s": tt[k]["t_pre"], "t_pro_s": tt[k]["t_pro"],
                          "delta_over_kappa": te[k]["delta_over_kappa"], "epsilon_over_kappa": te[k]["epsilon_over_kappa"]}
            rows.append(r)
            print(json.dumps(r), file=sys.stderr, flush=True)
            torch.cuda.empty_cache()
    print(json.dumps({"study": "section5_sparse_operator", "omega": "gaussian", "rhs": "100 random unit b per row",
                      "rows": rows}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--workload", default="dense_512x65536", choices=sorted(workloads.WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-fp64-form", action="store_true", help="skip the float64-form comparison")
    ap.add_argument("--l", type=int, default=None, help="sketch size (default: the workload's)")
    ap.add_argument("--pipeline", type=int, default=6,
                    help="handles (and streams) the timed steps rotate over; > 1 overlaps consecutive steps")
    ap.add_argument("--opt", action="append", default=None,
                    help="an rtproj_opts field for the timed handles, name=value (repeatable)")
    ap.add_argument("--sparse-row", default=None,
                    help="with --study sparse: only the rows m,n,l,kappa of Tables 1 and 5 (e.g. 1000,300000,1004,1e8)")
    ap.add_argument("--study", choices=["accuracy", "variates", "batch", "sparse"], default=None,
                    help="run a study (Section 5 accuracy; variates and sketch sizes) instead of the bench")
    args = ap.parse_args()
    if args.study:
        import __graft_entry__
        __graft_entry__.build()
        return {"accuracy": study_accuracy, "variates": study_variates, "batch": study_batch,
                "sparse": study_sparse}[args.study](args)
    if args.warmup < 3:
        args.warmup = 3
    w = workloads.WORKLOADS[args.workload]
    if args.l is not None:
        import dataclasses
        w = dataclasses.replace(w, l=args.l)
    world, rank, local = setup_dist() if args.impl == "ours" else (
        int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")))
    if args.impl == "reference":
        return run_reference(args, w, world, rank)
    if rank == 0:
        import __graft_entry__
        __graft_entry__.build()
    barrier(world)
    return run_ours(args, w, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
