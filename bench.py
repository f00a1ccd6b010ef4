#!/usr/bin/env python
"""Benchmark: FMM solve throughput (particles/s) on the uniform 1M workload.

Workload: N = 1,048,576 points uniform in the unit cube, charges U[-1,1],
p = 10, theta = 0.4, ncrit = 64, depth <= 10 (synthetic, SplitMix64 seed 1002).
A step is one whole solve (box, keys, sort, tree, traversal, P2M/M2M, M2L,
L2L/L2P, P2P, combine) from device-resident inputs to device-resident outputs.
The inputs (16 MB) fit in L2, so a 512 MB buffer is written between timed steps
to flush it; each step is bracketed by CUDA events on the solve's stream.

Also reported:
  e2e          the same solve through fmm_laplace3d_host (pinned host buffers,
               host->device and device->host copies inside the timed region)
  roofline     the dominant kernel against the measured/derived peak
  cpu_baseline the whole FP64 oracle FMM on the same workload on the host
               cores (measured, one run), the single-core time of the 4,096-point
               uniform case, and the sampled FP64 direct sum
  clocks       nvidia-smi SM clock samples during the timed region
  configs      the other workloads, GPU only: Plummer 4M at p = 6/8/12 in each
               M2L precision (time and error against the FP64 direct sum per p),
               512 batched systems (tuned schedule, one call, one graph replay,
               one call per system) and Plummer 16M (learned vs plain selection
               at the measured-best N_crit, and the plain FP32 FMM)
  peaks        SM count from the device, the derived FP32 peak, and TF32 / FP64
               dense GEMM rates measured with cuBLAS in this process

--impl reference times the oracle (the reference arm of this project): each
step is the whole oracle pipeline (keys, sort, tree, traversal, upward pass)
plus the evaluation of every 8th leaf (every 8th system for a batch), and the
line reports the particles evaluated per second of those steps as measured.
Multi-GPU (torchrun): every rank solves its own replica (the single system is
not sharded), the reported value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

P2P_FLOPS = 23          # counted flops per P2P interaction (FMA = 2)
FP32_LANES = 128        # FP32 lanes per SM (4 partitions x 32)
REF_STRIDE = 8          # the reference arm evaluates every 8th leaf / system per step


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="uniform1m")
    ap.add_argument("--precision", default="tf32x3", choices=["fp32", "tf32x3", "bf16x3"])
    ap.add_argument("--no-modes", action="store_true", help="skip timing the other M2L precisions")
    ap.add_argument("--p", type=int, default=None, help="override the workload's expansion order")
    ap.add_argument("--ncrit", type=int, default=None, help="override the workload's ncrit")
    ap.add_argument("--select", default="plain", choices=["plain", "autotune", "learned"],
                    help="interaction-type selection of MAC-accepted pairs (hybrid FMM)")
    ap.add_argument("--no-select-modes", action="store_true",
                    help="skip timing the other selection modes")
    ap.add_argument("--train-steps", type=int, default=3000)
    ap.add_argument("--tune-ncrit", action="store_true",
                    help="pick ncrit and the M2L work-unit size with the measured autotuner before timing")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="skip timing the captured plan (graph replay)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other workloads (Plummer 4M per p, batched 512, Plummer 16M)")
    return ap.parse_args()


def workload(name, p=None, ncrit=None):
    """(parameters, xyz, q, offsets) -- offsets is None for a single system."""
    from paper_1108_5815_gb300 import inputs
    w = dict(inputs.WORKLOADS[name])
    if p is not None:
        w["p"] = p
    if ncrit is not None:
        w["ncrit"] = ncrit
    if w["kind"] == "batched":
        x, q, off = inputs.batched_systems(w["nsys"], w["seed"])
        w["n"] = int(off[-1])
        return w, x, q, off
    x, q = inputs.make(w["kind"], w["n"], w["seed"])
    return w, x, q, None


def config_of(w, args):
    if w["kind"] == "batched":
        desc = (f"{args.workload}: {w['nsys']} independent systems, N_i log-uniform in [1e3, 1e5] "
                f"(total {w['n']}), half uniform cube / half Plummer, q~U[-1,1]")
    else:
        desc = f"{args.workload}: N={w['n']} {w['kind']}, " + ("q=1/N" if w["kind"] == "plummer" else "q~U[-1,1]")
    return {"workload": desc, "N": w["n"], "p": w["p"], "theta": w["theta"], "ncrit": w["ncrit"],
            "max_depth": w["max_depth"], "m2l": args.precision, "select": args.select,
            "l2_policy": "512 MB buffer written between timed steps"}


# ------------------------------------------------------------------ oracle timing

def oracle_full(x, q, w):
    """The whole FP64 oracle FMM on the workload (all targets), timed once on all
    host cores.  Returns (particles_per_s, seconds, description)."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    f = O.Fmm(x, q, w["p"], w["theta"], w["ncrit"], max_depth=w["max_depth"])
    f.evaluate()
    t = time.perf_counter() - t0
    return w["n"] / t, t, (f"the whole oracle FMM on the full workload ({w['n']} particles: keys, sort, "
                           f"tree, traversal, P2M/M2M, M2L, L2L, L2P, P2P over all {f.ncells} cells), one run")


def oracle_full_batched(x, q, off, w):
    """The oracle FMM on every system of a batch, one after another."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    for sy in range(len(off) - 1):
        a, b = off[sy], off[sy + 1]
        O.Fmm(x[a:b], q[a:b], w["p"], w["theta"], w["ncrit"], max_depth=w["max_depth"]).evaluate()
    t = time.perf_counter() - t0
    return int(off[-1]) / t, t, f"the oracle FMM on all {len(off) - 1} systems ({int(off[-1])} particles), one run"


def oracle_single_core_config1():
    """Single-core time of the oracle FMM on the 4,096-point uniform case (p = 4,
    theta = 0.5, ncrit = 64): median of three runs."""
    from oracle import oracle as O
    from paper_1108_5815_gb300 import inputs
    w = inputs.WORKLOADS["uniform4k"]
    x, q = inputs.make(w["kind"], w["n"], w["seed"])
    nt = O.num_threads()
    O.set_num_threads(1)
    try:
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            O.Fmm(x, q, w["p"], w["theta"], w["ncrit"], max_depth=w["max_depth"]).evaluate()
            ts.append(time.perf_counter() - t0)
    finally:
        O.set_num_threads(nt)
    return statistics.median(ts)


def oracle_step(x, q, w, k, stride=REF_STRIDE):
    """One step of the reference arm: the oracle's keys, sort, tree, traversal and
    upward pass over the whole workload, then the far/near evaluation of the
    leaves k, k+stride, ... (a different slice each step).  Returns (particles
    evaluated, seconds)."""
    import numpy as np
    from oracle import oracle as O
    t0 = time.perf_counter()
    f = O.Fmm(x, q, w["p"], w["theta"], w["ncrit"], max_depth=w["max_depth"])
    f.upward()
    c = f.cells()
    leaves = np.flatnonzero(c["nchild"] == 0)
    pos, _, _ = f.evaluate_leaves(leaves[k % stride::stride])
    return len(pos), time.perf_counter() - t0


def oracle_step_batched(x, q, off, w, k, stride=REF_STRIDE):
    """One step of the reference arm for a batch: the whole oracle FMM of systems
    k, k+stride, ... Returns (particles evaluated, seconds)."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    done = 0
    for sy in range(k % stride, len(off) - 1, stride):
        a, b = off[sy], off[sy + 1]
        O.Fmm(x[a:b], q[a:b], w["p"], w["theta"], w["ncrit"], max_depth=w["max_depth"]).evaluate()
        done += int(b - a)
    return done, time.perf_counter() - t0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    w, x, q, off = workload(args.workload, args.p, args.ncrit)
    if off is None:
        step = lambda k: oracle_step(x, q, w, k)
        desc = (f"each step: the oracle's keys, sort, tree, traversal and upward pass over the whole "
                f"workload, then M2L/L2L/L2P/P2P for the particles of every {REF_STRIDE}th leaf (a "
                f"different slice each step); value = particles evaluated / measured seconds")
    else:
        step = lambda k: oracle_step_batched(x, q, off, w, k)
        desc = (f"each step: the whole oracle FMM of every {REF_STRIDE}th system (a different slice each "
                f"step); value = particles evaluated / measured seconds")
    for k in range(args.warmup):
        step(k)
    done, secs = 0, 0.0
    for k in range(args.steps):
        n_k, t_k = step(args.warmup + k)
        done += n_k
        secs += t_k
    value = done / secs
    line = {"impl": "reference", "metric": "FMM particles/s", "value": value,
            "unit": "particles/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(w, args),
            "cpu_baseline": {"value": value, "unit": "particles/s", "cores": O.num_threads(),
                             "kind": "oracle", "sample": desc, "measured": True,
                             "particles_per_step": done / args.steps},
            "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def direct_reference(x, q, nsample=512, seed=77, off=None):
    """FP64 direct sums (oracle) on nsample seeded targets (for a batch: 128 targets
    in each of 4 systems, each against its own system).  Returns (targets, phi*,
    grad*, seconds)."""
    from oracle import oracle as O
    from paper_1108_5815_gb300 import inputs
    import numpy as np
    t0 = time.perf_counter()
    if off is None:
        t = inputs.sample_indices(len(q), nsample, seed)
        pd, gd = O.direct(x, q, targets=t)
    else:
        nsys = len(off) - 1
        ts, pds, gds = [], [], []
        for sy in (0, nsys // 3, 2 * nsys // 3, nsys - 1):
            a, b = int(off[sy]), int(off[sy + 1])
            tt = inputs.sample_indices(b - a, 128, seed + sy)
            p_, g_ = O.direct(x[a:b], q[a:b], targets=tt)
            ts.append(a + tt)
            pds.append(p_)
            gds.append(g_)
        t, pd, gd = np.concatenate(ts), np.concatenate(pds), np.concatenate(gds)
    return t, pd, gd, time.perf_counter() - t0


def compare(ref, phi, grad):
    """Relative L2 and worst-particle errors of phi/grad (numpy, caller order) at
    the reference's targets."""
    import numpy as np
    t, pd, gd, _ = ref
    got_p, got_g = np.asarray(phi, np.float64)[t], np.asarray(grad, np.float64)[t]
    return {"rel_l2_phi": float(np.linalg.norm(got_p - pd) / np.linalg.norm(pd)),
            "rel_l2_grad": float(np.linalg.norm(got_g - gd) / np.linalg.norm(gd)),
            "max_err_phi_rel_max": float(np.abs(got_p - pd).max() / np.abs(pd).max()),
            "max_err_grad_rel_max": float(np.linalg.norm(got_g - gd, axis=1).max()
                                          / np.linalg.norm(gd, axis=1).max()),
            "reference": "FP64 direct sum (oracle)", "targets": int(len(t))}


def accuracy(x, q, phi, grad, nsample=512, seed=77, off=None):
    """compare() against a fresh direct_reference()."""
    return compare(direct_reference(x, q, nsample, seed, off), phi, grad)


# ------------------------------------------------------------------ peaks and rooflines

def measured_peaks():
    """(HBM GB/s, BF16 dense TF/s, label): MEASURED_PEAKS.json when present, else
    the fallback figures of one earlier GB300 measurement."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "of measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, 1900.0, "of fallback"


def sm_max_mhz():
    """Maximum SM clock: MEASURED_PEAKS.json, else nvidia-smi, else the GB300 figure."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"]), "MEASURED_PEAKS.json"
    except (OSError, KeyError, ValueError):
        pass
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=20).stdout.split()
        return float(out[0]), "nvidia-smi"
    except (OSError, IndexError, ValueError, subprocess.SubprocessError):
        return 2070.0, "GB300 maximum SM clock"


def gemm_tflops(torch, dev, dtype, n, reps, tf32=False):
    """Best-of-reps rate of one dense n x n x n cuBLAS GEMM (2 n^3 flop), CUDA events."""
    old = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = tf32
    try:
        g = torch.Generator(device=dev)
        g.manual_seed(5)
        a = torch.randn(n, n, device=dev, dtype=dtype, generator=g)
        b = torch.randn(n, n, device=dev, dtype=dtype, generator=g)
        c = a @ b
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        del a, b, c
        return 2.0 * n ** 3 / (best * 1e-3) / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old


def device_peaks(torch, dev):
    """Peaks for the rooflines: the SM count from the device, the FP32 peak derived
    from it (SMs x 128 lanes x 2 flop x maximum SM clock), HBM and BF16 from
    MEASURED_PEAKS.json, and TF32 / FP64 dense GEMM rates measured here with
    cuBLAS (TF32: fp32 matmul with TF32 allowed, 8192^3; FP64: 4096^3)."""
    props = torch.cuda.get_device_properties(dev)
    sms = int(props.multi_processor_count)
    mhz, mhz_src = sm_max_mhz()
    hbm, bf16, label = measured_peaks()
    return {"sms": sms, "sm_max_mhz": mhz, "sm_max_mhz_source": mhz_src,
            "fp32_derived_tflops": sms * FP32_LANES * 2 * mhz * 1e6 / 1e12,
            "hbm_gbs": hbm, "bf16_tflops": bf16, "hbm_bf16_label": label,
            "tf32_tflops": gemm_tflops(torch, dev, torch.float32, 8192, 10, tf32=True),
            "fp64_tflops": gemm_tflops(torch, dev, torch.float64, 4096, 3),
            "what": "sms: cudaDevAttrMultiProcessorCount; tf32/fp64: cuBLAS dense GEMM measured in this "
                    "process (best of 10 / 3, CUDA events); hbm/bf16: MEASURED_PEAKS.json"}


def captured_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu capture record,
    or None when the kernel's source changed since the capture."""
    import hashlib
    rec_path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(rec_path))[kernel]
        src = open(os.path.join(ROOT, rec["source"]), "rb").read()
    except (OSError, KeyError, ValueError):
        return None
    if hashlib.sha256(src).hexdigest() != rec["source_sha256"]:
        return None
    return rec["dram_bytes_per_launch"]


def m2l_tc_kernel(p):
    """The tensor-core M2L kernel the library runs at order p: A in tensor
    memory while the padded expansion length (p+1)^2 -> multiple of 32 is at
    most 128, A in shared memory above that."""
    return "k_m2l_tc_ta" if -(-(p + 1) ** 2 // 32) * 32 <= 128 else "k_m2l_tc"


def hot_kernel_rooflines(st, ms_p2p, ms_m2l, p, precision, pk):
    """P2P against the FP32 pipe (derived peak) and M2L against its own pipe.

    P2P work: interactions x 23 flop.  M2L work: M2L pairs x 2 (p+1)^4 flop, the
    useful flops of the dense translation (the 3-way split, padding to 128 and
    empty rows of a tile are not counted)."""
    fp32_peak = pk["fp32_derived_tflops"]
    out = []
    p2p_tf = st["n_p2p_interactions"] * P2P_FLOPS / (ms_p2p * 1e-3) / 1e12
    out.append({"kernel": "k_p2p", "bound": "alu", "achieved": p2p_tf, "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": p2p_tf / fp32_peak, "traffic": captured_traffic("k_p2p"),
                "ms": ms_p2p,
                "peak_source": (f"derived: {pk['sms']} SMs (device query) x {FP32_LANES} FP32 lanes x 2 flop x "
                                f"{pk['sm_max_mhz']:.0f} MHz ({pk['sm_max_mhz_source']})"),
                "work": f"{st['n_p2p_interactions']} interactions x {P2P_FLOPS} flop"})
    P2 = (p + 1) ** 2
    m2l_tf = st["n_m2l_pairs"] * 2 * P2 * P2 / (ms_m2l * 1e-3) / 1e12
    if precision == "fp32":
        kern, bound, peak, src = "k_m2l_simt", "alu", fp32_peak, "derived FP32 peak (as for P2P)"
    elif precision == "tf32x3":
        kern, bound, peak = f"{m2l_tc_kernel(p)}<tf32x3>", "tensor", pk["tf32_tflops"]
        src = "TF32 dense: cuBLAS fp32 GEMM with TF32, 8192^3, measured in this process"
    else:
        kern, bound, peak = f"{m2l_tc_kernel(p)}<bf16x3>", "tensor", pk["bf16_tflops"]
        src = f"BF16 dense {pk['hbm_bf16_label']} (MEASURED_PEAKS.json)"
    out.append({"kernel": kern, "bound": bound, "achieved": m2l_tf, "peak": peak,
                "unit": "TFLOP/s", "frac": m2l_tf / peak, "traffic": captured_traffic(kern),
                "ms": ms_m2l, "peak_source": src,
                "work": f"{st['n_m2l_pairs']} M2L pairs x 2 (p+1)^4 = {2 * P2 * P2} flop"})
    return out


def tree_roofline(n, ms_tree, pk):
    """The tree build (box, keys, radix sort, permute, level splits) against HBM.

    Algorithmic bytes per particle: 16 read (x, y, z, q) + 16 permuted write +
    12 key/index write, plus 24 per 8-bit radix pass (8 passes over 63-bit keys).
    The phase time includes every launch of the phase; it is a phase, not one kernel."""
    hbm, label = pk["hbm_gbs"], pk["hbm_bf16_label"]
    bytes_ = n * (16 + 16 + 12 + 24 * 8)
    gbs = bytes_ / (ms_tree * 1e-3) / 1e9
    return {"kernel": "tree build phase", "phase": True, "bound": "hbm", "achieved": gbs, "peak": hbm,
            "unit": "GB/s", "frac": gbs / hbm, "traffic": None, "ms": ms_tree,
            "peak_source": f"STREAM-style copy {label}",
            "work": f"{n} particles x 236 B (16 read + 16 permuted write + 12 key/index + 8 radix passes x 24)"}


def solve_roofline_fraction(rooflines, ms_solve):
    """Sum over the measured steps of (algorithmic work / that step's peak) over the
    solve time: the share of the solve the hardware bounds alone would need."""
    terms = {}
    for r in rooflines:
        terms[r["kernel"]] = r["ms"] * r["frac"]  # work / peak, in ms
    return {"value": sum(terms.values()) / ms_solve, "bound_ms": terms, "solve_ms": ms_solve}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    def __init__(self, index):
        self.proc = None
        self.path = None
        self.index = index

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        # nvidia-smi takes a while to start: wait (up to 5 s) for its first sample, so
        # that the samples after it fall inside the timed region that follows
        self.skip = 0
        if self.proc is not None:
            t0 = time.time()
            while time.time() - t0 < 5.0 and self.proc.poll() is None:
                with open(self.path) as f:
                    n = sum(1 for line in f if line.strip())
                if n:
                    self.skip = n
                    break
                time.sleep(0.01)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if getattr(self, "fh", None):
            self.fh.close()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                rows.append(parts)
        os.unlink(self.path)
        if len(rows) > self.skip:
            rows = rows[self.skip:]  # the samples taken before the timed region started
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[4 + i]
                          and "Not" not in r[4 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------------ the other workloads

def _time_gpu(torch, stream, flush, fn, steps, warm=2):
    """Median device time (ms) of fn() over `steps` calls after `warm` untimed
    ones, L2 flushed before each, CUDA events on the solve's stream."""
    for _ in range(warm):
        fn()
    ms = []
    for k in range(steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return statistics.median(ms)


def run_configs(torch, dev, stream, flush, cost_model, args):
    """The benchmark's other configurations on the GPU (no CPU oracle runs but the
    sampled FP64 direct sums that judge accuracy):

    * plummer4m: N = 4,194,304 Plummer points, q = 1/N, theta 0.4, ncrit 64, at
      p = 6, 8, 12 in each M2L precision (FP32, TF32x3, BF16x3): time and error
      against the FP64 direct sum per p;
    * batched512: 512 systems (N_i log-uniform in [1e3, 1e5], half uniform, half
      Plummer), p = 8, theta 0.5: schedule (N_crit, M2L work-unit size) from the
      measured autotuner, then one batched call (TF32x3 and FP32), one replay of
      the captured graph, and one call per system;
    * plummer16m: N = 16,777,216 Plummer points, p = 10, theta 0.4: N_crit from the
      measured autotuner (plain selection) and from the learned cost model; plain
      and learned selection with TF32x3 M2L, and the plain FP32 FMM."""
    from paper_1108_5815_gb300 import fmm, inputs
    out = {}
    t_all = time.perf_counter()
    tm = lambda fn, k=3: _time_gpu(torch, stream, flush, fn, k)

    # ---- mixed precision per p
    w = inputs.WORKLOADS["plummer4m"]
    x, q = inputs.make(w["kind"], w["n"], w["seed"])
    n = w["n"]
    xd, qd = torch.from_numpy(x).to(dev), torch.from_numpy(q).to(dev)
    phi, grad = torch.empty(n, device=dev), torch.empty(n, 3, device=dev)
    ref = direct_reference(x, q)
    per_p = {}
    for p in (6, 8, 12):
        rec = {}
        for prec in ("fp32", "tf32x3", "bf16x3"):
            m = tm(lambda: fmm.laplace3d(xd, qd, p, w["theta"], w["ncrit"], max_depth=w["max_depth"],
                                         precision=prec, out=(phi, grad)))
            rec[prec] = {"ms": m, "value": n / (m / 1e3),
                         "accuracy": compare(ref, phi.cpu().numpy(), grad.cpu().numpy())}
        rec["speedup_vs_fp32"] = {k: rec["fp32"]["ms"] / rec[k]["ms"] for k in ("tf32x3", "bf16x3")}
        per_p[str(p)] = rec
    out["plummer4m"] = {"workload": f"N={n} Plummer (a=1, r<=20), q=1/N, theta={w['theta']}, "
                                    f"ncrit={w['ncrit']}", "per_p": per_p}
    del xd, qd, phi, grad

    # ---- batched systems
    w = inputs.WORKLOADS["batched512"]
    x, q, off = inputs.batched_systems(w["nsys"], w["seed"])
    n = int(off[-1])
    xd, qd = torch.from_numpy(x).to(dev), torch.from_numpy(q).to(dev)
    phi, grad = torch.empty(n, device=dev), torch.empty(n, 3, device=dev)
    ref = direct_reference(x, q, off=off)
    bn, bu, table = fmm.tune_schedule(xd, qd, w["p"], w["theta"], offsets=off, ncrit_candidates=(32, 64, 128, 256),
                                      unit_candidates=(0, 32, 128), max_depth=w["max_depth"], precision="tf32x3")
    kb = dict(max_depth=w["max_depth"], m2l_unit_blocks=bu)
    rec = {"schedule": {"ncrit": bn, "m2l_unit_blocks": bu,
                        "candidates_ms": {f"ncrit={a},unit={b}": v for (a, b), v in table.items()}}}
    for prec in ("fp32", "tf32x3"):
        m = tm(lambda: fmm.laplace3d_batched(xd, qd, off, w["p"], w["theta"], bn, precision=prec,
                                             out=(phi, grad), **kb))
        rec["batched_" + prec] = {"ms": m, "value": n / (m / 1e3),
                                  "accuracy": compare(ref, phi.cpu().numpy(), grad.cpu().numpy())}
    plan = fmm.Plan(xd, qd, w["p"], w["theta"], bn, offsets=off, precision="tf32x3", headroom=1.25, **kb)
    gphi, ggrad = torch.empty_like(phi), torch.empty_like(grad)
    m = tm(lambda: plan.execute(xd, qd, out=(gphi, ggrad)))
    valid = plan.check() == 0
    info = plan.info()
    plan.close()
    fmm.laplace3d_batched(xd, qd, off, w["p"], w["theta"], bn, precision="tf32x3", out=(phi, grad), **kb)
    torch.cuda.synchronize()
    rec["graph_replay_tf32x3"] = {"ms": m, "value": n / (m / 1e3), "valid": valid,
                                  "equal_to_batched_call": bool(torch.equal(gphi, phi) and torch.equal(ggrad, grad)),
                                  "graph_kernels": info["graph_kernels"]}

    def loop():
        for sy in range(len(off) - 1):
            a_, b_ = int(off[sy]), int(off[sy + 1])
            fmm.laplace3d(xd[a_:b_], qd[a_:b_], w["p"], w["theta"], bn, precision="tf32x3",
                          out=(phi[a_:b_], grad[a_:b_]), **kb)
    m = _time_gpu(torch, stream, flush, loop, 2, warm=1)
    rec["one_call_per_system_tf32x3"] = {"ms": m, "value": n / (m / 1e3)}
    rec["speedup_batched_vs_per_system"] = m / rec["batched_tf32x3"]["ms"]
    rec["speedup_batched_tf32x3_vs_batched_fp32"] = rec["batched_fp32"]["ms"] / rec["batched_tf32x3"]["ms"]
    out["batched512"] = dict(workload=f"{len(off) - 1} systems, {n} particles, N_i log-uniform in [1e3, 1e5], "
                                      f"half uniform / half Plummer, p={w['p']}, theta={w['theta']}", **rec)
    del xd, qd, phi, grad, gphi, ggrad

    # ---- learned cost model at scale
    w = inputs.WORKLOADS["plummer16m"]
    x, q = inputs.make(w["kind"], w["n"], w["seed"])
    n = w["n"]
    xd, qd = torch.from_numpy(x).to(dev), torch.from_numpy(q).to(dev)
    phi, grad = torch.empty(n, device=dev), torch.empty(n, 3, device=dev)
    ref = direct_reference(x, q)
    cands = (64, 128, 256)
    bn, _, table = fmm.tune_schedule(xd, qd, w["p"], w["theta"], ncrit_candidates=cands, unit_candidates=(0,),
                                     max_depth=w["max_depth"], precision="tf32x3")
    if cost_model is None:
        cost_model = fmm.cost_model_train(precision="tf32x3", p_lo=3, p_hi=12, steps=args.train_steps, seed=1)
    nb, pred = fmm.cost_model_pick_ncrit(xd, qd, w["p"], w["theta"], cands, max_depth=w["max_depth"],
                                         precision="tf32x3", select="learned")
    rec = {"ncrit_measured_best": bn, "ncrit_tuner_ms": {str(a): v for (a, _), v in table.items()},
           "ncrit_network_pick": nb, "ncrit_network_predicted_ms": {str(k): v for k, v in pred.items()}}
    variants = [("plain_fp32", "fp32", "plain", bn), ("plain_tf32x3", "tf32x3", "plain", bn),
                ("learned_tf32x3", "tf32x3", "learned", bn)]
    if nb != bn:
        variants.append(("learned_tf32x3_network_ncrit", "tf32x3", "learned", nb))
    for name, prec, sel, nc in variants:
        m = tm(lambda: fmm.laplace3d(xd, qd, w["p"], w["theta"], nc, max_depth=w["max_depth"], precision=prec,
                                     select=sel, out=(phi, grad)))
        rec[name] = {"ms": m, "value": n / (m / 1e3), "ncrit": nc,
                     "accuracy": compare(ref, phi.cpu().numpy(), grad.cpu().numpy())}
    rec["speedup_learned_tf32x3_vs_plain_fp32"] = rec["plain_fp32"]["ms"] / rec["learned_tf32x3"]["ms"]
    rec["speedup_learned_vs_plain_tf32x3"] = rec["plain_tf32x3"]["ms"] / rec["learned_tf32x3"]["ms"]
    out["plummer16m"] = dict(workload=f"N={n} Plummer, q=1/N, p={w['p']}, theta={w['theta']}", **rec)
    del xd, qd, phi, grad
    out["seconds"] = time.perf_counter() - t_all
    return out


# ------------------------------------------------------------------ main arm

def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1108_5815_gb300 import build, fmm

    from paper_1108_5815_gb300 import replicas
    rank, world, local = replicas.rank_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    build.build()

    w, x, q, off = workload(args.workload, args.p, args.ncrit)
    n = w["n"]
    xd = torch.from_numpy(x).to(dev)
    qd = torch.from_numpy(q).to(dev)
    phi = torch.empty(n, device=dev)
    grad = torch.empty(n, 3, device=dev)
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device=dev)  # 512 MB > L2
    kw = dict(max_depth=w["max_depth"], precision=args.precision, select=args.select)
    # the learned cost model is trained before timing (samples generated by the
    # method's own kernels on artificial data, then GPU training); its tables are
    # measured and cached by the warm-up solves, as the pre-timed tables are
    cost_model = None
    if args.select == "learned" or (not args.no_select_modes and rank == 0):
        cost_model = fmm.cost_model_train(precision=args.precision, p_lo=3, p_hi=12,
                                          steps=args.train_steps, seed=1)

    def solve(stats=False, **over):
        k2 = dict(kw, **over)
        if off is None:
            return fmm.laplace3d(xd, qd, w["p"], w["theta"], w["ncrit"], stats=stats,
                                 out=(phi, grad), **k2)
        return fmm.laplace3d_batched(xd, qd, off, w["p"], w["theta"], w["ncrit"], stats=stats,
                                     out=(phi, grad), **k2)

    ncrit_tuning = None
    if args.tune_ncrit:
        # the measured autotuner picks N_crit and the M2L work-unit size together
        ncs, ucs = (32, 64, 128, 256, 512), (0, 8, 32, 128)
        bn, bu, table = fmm.tune_schedule(xd, qd, w["p"], w["theta"], offsets=off, ncrit_candidates=ncs,
                                          unit_candidates=ucs, **kw)
        ncrit_tuning = {"candidates_ms": {f"ncrit={a},unit={b}": v for (a, b), v in table.items()},
                        "best_ncrit": bn, "best_m2l_unit_blocks": bu, "workload_ncrit": w["ncrit"]}
        if cost_model is not None and off is None:
            # the network's pick from the candidates' interaction lists, judged by the measurement
            nb, pred = fmm.cost_model_pick_ncrit(xd, qd, w["p"], w["theta"], ncs, **kw)
            ncrit_tuning["network"] = {"pick": nb, "predicted_ms": pred,
                                       "measured_ms_of_pick": min(v for (a, _), v in table.items() if a == nb),
                                       "measured_best_ms": min(table.values())}
        w["ncrit"] = bn
        kw["m2l_unit_blocks"] = bu

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    st_list = []
    with ClockSampler(local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))
            starts[k].record(stream)
            solve()
            ends[k].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    # the same solve with its statistics (phase events, pair and interaction
    # counts; the count of P2P interactions is one more kernel), outside the
    # timed loop
    for k in range(args.steps):
        flush.fill_(float(k))
        st_list.append(solve(stats=True)[2])
    torch.cuda.synchronize()
    # the timed solve replays the plan the library captured from the warm-up
    # calls (fmm_options.replay); the same solve without it, for comparison
    plain_ms = []
    for k in range(args.steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        solve(replay=False)
        b.record(stream)
        b.synchronize()
        plain_ms.append(a.elapsed_time(b))
    plain = {"ms_per_step": statistics.mean(plain_ms), "value": n / (statistics.mean(plain_ms) / 1e3),
             "what": "the same solve with fmm_options.replay = 0: every call launches its kernels from the "
                     "host, with read-backs of the sizes between phases"}
    # each rank solved its own replica: job time = slowest rank, work = all ranks
    total_ms, _, value = replicas.aggregate(sum(step_ms), n * args.steps, device=dev)
    ms_per_step = total_ms / args.steps
    clocks = clk.summary()

    # In the solve the far-field chain takes SMs as P2P's blocks retire, so the
    # events of a phase span whatever ran beside it.  The rooflines and phase times
    # come from a second timed loop of the same solve with the far-field chain held
    # until P2P has finished (fmm_options.serialize_phases), each phase then alone.
    ser_list = []
    for _ in range(2):
        solve(serialize_phases=True)
    for k in range(args.steps):
        flush.fill_(float(k))
        ser_list.append(solve(stats=True, serialize_phases=True)[2])
    torch.cuda.synchronize()
    phases_overlapped = {k: round(statistics.mean(s[k] for s in st_list), 4)
                         for k in ("ms_tree", "ms_traverse", "ms_upward", "ms_m2l", "ms_downward", "ms_p2p",
                                   "ms_total")}

    # rooflines of the two hot kernels, from the library's event timing of each phase
    st0 = st_list[-1]
    ms_p2p = statistics.mean(s["ms_p2p"] for s in ser_list)
    ms_m2l = statistics.mean(s["ms_m2l"] for s in ser_list)
    pk = device_peaks(torch, dev)
    rooflines = hot_kernel_rooflines(st0, ms_p2p, ms_m2l, w["p"], args.precision, pk)
    # the FP32 pipe's measured ceilings beside the derived peak (context for the P2P line)
    ceil = fmm.measure_fp32()
    p2p_line = rooflines[0]
    body_tf = ceil["body_interactions_per_s"] * P2P_FLOPS / 1e12
    p2p_line["peak_measured_ffma_stream"] = ceil["ffma_tflops"]
    p2p_line["frac_of_measured_ffma_stream"] = p2p_line["achieved"] / ceil["ffma_tflops"]
    p2p_line["ceilings"] = {
        "ffma_stream_tflops": ceil["ffma_tflops"],
        "ffma_stream_frac_of_derived_peak": ceil["ffma_tflops"] / p2p_line["peak"],
        "p2p_body_tflops": body_tf,
        "p2p_body_frac_of_derived_peak": body_tf / p2p_line["peak"],
        "kernel_frac_of_body": p2p_line["achieved"] / body_tf,
        "what": "FP32x2 FMA chains alone (the measured FP32 rate), and the P2P interaction code on staged "
                "sources with no list walk (fmm_measure_fp32), timed live beside the solve"}
    for r in rooflines:
        r["timing"] = ("CUDA events around the kernel on its stream, mean of a second timed loop of "
                       f"{args.steps} solves with the far-field chain held until P2P ends "
                       "(fmm_options.serialize_phases = 1)")
    roof = max(rooflines, key=lambda r: r["ms"])  # the dominant kernel
    rooflines.append(tree_roofline(n, statistics.mean(s["ms_tree"] for s in ser_list), pk))
    solve_frac = solve_roofline_fraction(rooflines, ms_per_step)
    phases = {k: round(statistics.mean(s[k] for s in ser_list), 4)
              for k in ("ms_tree", "ms_traverse", "ms_upward", "ms_m2l", "ms_downward", "ms_p2p",
                        "ms_total")}

    # end to end through the host-pointer entry point
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(x).pin_memory().numpy()
        qh = torch.from_numpy(q).pin_memory().numpy()
        ph = torch.empty(n, dtype=torch.float32).pin_memory().numpy()
        gh = torch.empty(n, 3, dtype=torch.float32).pin_memory().numpy()
        sp = stream.cuda_stream
        xdt, qdt = torch.empty_like(xd), torch.empty_like(qd)

        def host_solve():
            if off is None:   # the C-ABI entry point with host buffers
                fmm.laplace3d_host(xh, qh, w["p"], w["theta"], w["ncrit"], out=(ph, gh), stream=sp, **kw)
                return
            # batched: pinned host -> device, the batched call, device -> pinned host
            xdt.copy_(torch.from_numpy(xh), non_blocking=True)
            qdt.copy_(torch.from_numpy(qh), non_blocking=True)
            pr, gr = fmm.laplace3d_batched(xdt, qdt, off, w["p"], w["theta"], w["ncrit"], **kw)
            torch.from_numpy(ph).copy_(pr, non_blocking=True)
            torch.from_numpy(gh).copy_(gr, non_blocking=True)
            torch.cuda.synchronize()

        for _ in range(2):
            host_solve()
        t_e2e = 0.0
        for k in range(args.steps):
            flush.fill_(float(k))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            host_solve()
            t_e2e += time.perf_counter() - t0
        e2e_ms, _, e2e_value = replicas.aggregate(1e3 * t_e2e / args.steps, n, device=dev)
        e2e = {"value": e2e_value, "unit": "particles/s",
               "h2d_bytes_per_step": int(x.nbytes + q.nbytes),
               "d2h_bytes_per_step": int(ph.nbytes + gh.nbytes), "ms_per_step": e2e_ms}

    # accuracy of this very solve against the FP64 direct sum on sampled targets
    acc = ref = None
    if rank == 0:
        ref = direct_reference(x, q, off=off)
        acc = compare(ref, phi.cpu().numpy(), grad.cpu().numpy())

    # the other M2L precisions, timed the same way (value and accuracy)
    modes = {}
    if rank == 0 and not args.no_modes:
        for prec in ("fp32", "tf32x3", "bf16x3"):
            if prec == args.precision:
                continue
            for _ in range(2):
                solve(precision=prec)
            ms = []
            for k in range(args.steps):
                flush.fill_(float(k))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                solve(precision=prec)
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
            m = statistics.mean(ms)
            modes[prec] = {"value": n / (m / 1e3), "ms_per_step": m,
                           "accuracy": compare(ref, phi.cpu().numpy(), grad.cpu().numpy())}

    # the other selection modes (plain FMM, pre-timed, learned, and the treecode: cell-particle
    # for every accepted pair), timed the same way
    select_modes = {}
    if rank == 0 and not args.no_select_modes:
        for sel in ("plain", "autotune", "learned", "treecode"):
            if sel == args.select:
                continue
            # the treecode is orders of magnitude slower on large workloads: fewer steps
            nst = min(args.steps, 3) if sel == "treecode" else args.steps
            for _ in range(1 if sel == "treecode" else 2):
                solve(select=sel)
            # timed as the main loop (no statistics, so repeated calls replay their plan);
            # the pair counts come from one more call with statistics
            ms = []
            for k in range(nst):
                flush.fill_(float(k))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                solve(select=sel)
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
            sts = [solve(stats=True, select=sel)[2]]
            m = statistics.mean(ms)
            select_modes[sel] = {"value": n / (m / 1e3), "ms_per_step": m,
                                 "n_m2l_pairs": sts[-1]["n_m2l_pairs"],
                                 "n_m2p_pairs": sts[-1]["n_m2p_pairs"],
                                 "n_p2p_pairs": sts[-1]["n_p2p_pairs"],
                                 "n_p2p_interactions": sts[-1]["n_p2p_interactions"],
                                 "accuracy": compare(ref, phi.cpu().numpy(), grad.cpu().numpy())}

    # the same solve captured once into a CUDA graph (fmm_plan_create) and
    # replayed: one graph launch per step, no host read-back, inputs copied into
    # the plan and results out of it inside the timed region
    graph = None
    if rank == 0 and not args.no_graph:
        plan = fmm.Plan(xd, qd, w["p"], w["theta"], w["ncrit"], offsets=off, headroom=1.25, **kw)
        gphi = torch.empty_like(phi)
        ggrad = torch.empty_like(grad)
        for _ in range(2):
            plan.execute(xd, qd, out=(gphi, ggrad))
        ms = []
        for k in range(args.steps):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plan.execute(xd, qd, out=(gphi, ggrad))
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        status = plan.check()
        solve(replay=False)  # the plain solve, for the bit-for-bit comparison
        torch.cuda.synchronize()
        info = plan.info()
        m = statistics.mean(ms)
        graph = {"value": n / (m / 1e3), "ms_per_step": m, "valid": status == 0,
                 "equal_to_plain_solve": bool(torch.equal(gphi, phi) and torch.equal(ggrad, grad)),
                 "graph_kernels": info["graph_kernels"], "graph_nodes": info["graph_nodes"],
                 "levels": info["levels"], "operators": info["operators"],
                 "what": "fmm_plan_execute: the solve captured once into one CUDA graph, replayed with one "
                         "graph launch per step (device-side sizes, capacities 1.25x the first solve)"}
        plan.close()

    # a batch against solving its systems one call at a time
    loop = None
    if rank == 0 and off is not None:
        def solve_loop():
            for sy in range(len(off) - 1):
                a_, b_ = int(off[sy]), int(off[sy + 1])
                fmm.laplace3d(xd[a_:b_], qd[a_:b_], w["p"], w["theta"], w["ncrit"],
                              out=(phi[a_:b_], grad[a_:b_]), **kw)
        solve_loop()
        ms = []
        for k in range(max(1, args.steps // 2)):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            solve_loop()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        m = statistics.mean(ms)
        loop = {"value": n / (m / 1e3), "ms_per_step": m, "speedup_of_batch": m / ms_per_step,
                "what": "one fmm_laplace3d call per system, same workload"}

    configs = None
    if rank == 0 and world == 1 and not args.no_configs:
        configs = run_configs(torch, dev, stream, flush, cost_model, args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        v, secs, desc = oracle_full(x, q, w) if off is None else oracle_full_batched(x, q, off, w)
        cpu = {"value": v, "unit": "particles/s", "cores": O.num_threads(), "kind": "oracle",
               "sample": desc, "measured": True, "seconds": secs,
               "single_core_config1_s": oracle_single_core_config1(),
               "single_core_config1": "oracle FMM, N=4096 uniform cube, p=4, theta=0.5, ncrit=64, 1 thread, "
                                      "median of 3",
               "direct_sum_sample_s": ref[3] if ref is not None else None,
               "direct_sum_sample": f"FP64 direct sum on {len(ref[0]) if ref is not None else 0} sampled "
                                    f"targets against all {n} sources"}

    if rank == 0:
        line = {"metric": "FMM particles/s", "value": value, "unit": "particles/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_of(w, args), "roofline": roof, "rooflines": rooflines,
                "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": (args.steps * graph["graph_kernels"] if graph is not None
                                 else int(sum(s["n_launches"] for s in st_list))),
                "solve_path": ("fmm_laplace3d_ex with fmm_options.replay = 1 (the default): from the third "
                               "call of one key on, each call replays the plan captured after the second -- "
                               "every step of the solve in one graph launch, results bit-identical to the "
                               "plain solve (graph_replay.equal_to_plain_solve)"),
                "plain_solve": plain,
                "accuracy": acc, "m2l_modes": modes, "select_modes": select_modes,
                "cost_model": cost_model, "ncrit_tuning": ncrit_tuning, "per_system_loop": loop,
                "graph_replay": graph, "solve_roofline_fraction": solve_frac, "peaks": pk,
                "configs": configs,
                "clocks": clocks, "phases_ms": phases, "phases_ms_overlapped": phases_overlapped,
                "phases_what": ("phases_ms: each phase alone (far-field chain held until P2P ends); "
                                "phases_ms_overlapped: the timed solve, where P2P and the far-field "
                                "phases share the GPU and their event times overlap"),
                "counts": {k: st0[k] for k in ("ncells", "nleaves", "depth", "n_p2p_pairs",
                                               "n_p2p_interactions", "n_m2l_pairs",
                                               "n_offset_classes", "n_m2l_blocks", "n_m2p_pairs")}}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
