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
  cpu_baseline the FP64 oracle on the host cores on a bounded sample
  clocks       nvidia-smi SM clock samples during the timed region

--impl reference times the oracle (the reference arm of this project).
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
SMS = 152
FP32_LANES = 128
SM_MAX_MHZ = 2070.0


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

def oracle_sample(x, q, w, leaf_stride=128):
    """Oracle FMM on the full workload with the far/near evaluation restricted to
    every `leaf_stride`-th leaf; the evaluation time is scaled to all leaves.
    Returns (particles_per_s, seconds, description)."""
    import numpy as np
    from oracle import oracle as O
    t0 = time.perf_counter()
    f = O.Fmm(x, q, w["p"], w["theta"], w["ncrit"], max_depth=w["max_depth"])
    f.upward()
    t1 = time.perf_counter()
    c = f.cells()
    leaves = np.flatnonzero(c["nchild"] == 0)
    pick = leaves[::leaf_stride]
    f.evaluate_leaves(pick)
    t2 = time.perf_counter()
    t_total = (t1 - t0) + (t2 - t1) * (len(leaves) / len(pick))
    desc = (f"oracle FMM on the full workload (keys, sort, tree, traversal, P2M/M2M over all "
            f"{f.ncells} cells), M2L/L2L/L2P/P2P on {len(pick)} of {len(leaves)} leaves, "
            f"evaluation time scaled by {len(leaves) / len(pick):.1f}")
    return w["n"] / t_total, t2 - t0, desc


def oracle_sample_batched(x, q, off, w, stride=32):
    """Oracle FMM on every `stride`-th system, its time scaled to all systems."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    done = 0
    picked = list(range(0, len(off) - 1, stride))
    for sy in picked:
        a, b = off[sy], off[sy + 1]
        O.Fmm(x[a:b], q[a:b], w["p"], w["theta"], w["ncrit"], max_depth=w["max_depth"]).evaluate()
        done += b - a
    t = time.perf_counter() - t0
    desc = (f"oracle FMM on {len(picked)} of {len(off) - 1} systems ({done} particles), "
            f"rate applied to all {int(off[-1])} particles")
    return done / t, t, desc


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    w, x, q, off = workload(args.workload, args.p, args.ncrit)
    sample = (lambda: oracle_sample(x, q, w)) if off is None else (lambda: oracle_sample_batched(x, q, off, w))
    for _ in range(args.warmup):
        sample()
    vals = []
    wall = 0.0
    desc = ""
    for _ in range(args.steps):
        v, t, desc = sample()
        vals.append(v)
        wall += t
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": "FMM particles/s", "value": value,
            "unit": "particles/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * w["n"] / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(w, args),
            "cpu_baseline": {"value": value, "unit": "particles/s", "cores": O.num_threads(),
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def accuracy(x, q, phi, grad, nsample=512, seed=77, off=None):
    """Relative L2 error of phi and grad against the FP64 direct sum (oracle) on
    nsample seeded targets (for a batch: 128 targets in each of 4 systems, each
    against its own system)."""
    from oracle import oracle as O
    from paper_1108_5815_gb300 import inputs
    import numpy as np
    if off is None:
        t = inputs.sample_indices(len(q), nsample, seed)
        pd, gd = O.direct(x, q, targets=t)
        got_p, got_g = phi[t], grad[t]
    else:
        nsys = len(off) - 1
        pds, gds, gps, ggs = [], [], [], []
        for sy in (0, nsys // 3, 2 * nsys // 3, nsys - 1):
            a, b = int(off[sy]), int(off[sy + 1])
            t = inputs.sample_indices(b - a, 128, seed + sy)
            p_, g_ = O.direct(x[a:b], q[a:b], targets=t)
            pds.append(p_)
            gds.append(g_)
            gps.append(phi[a + t])
            ggs.append(grad[a + t])
        pd, gd, got_p, got_g = np.concatenate(pds), np.concatenate(gds), np.concatenate(gps), np.concatenate(ggs)
        nsample = len(pd)
    e_phi = float(np.linalg.norm(got_p - pd) / np.linalg.norm(pd))
    e_grad = float(np.linalg.norm(got_g - gd) / np.linalg.norm(gd))
    return {"rel_l2_phi": e_phi, "rel_l2_grad": e_grad, "reference": "FP64 direct sum (oracle)",
            "targets": int(nsample)}


# ------------------------------------------------------------------ rooflines

def measured_peaks():
    """(HBM GB/s, BF16 dense TF/s, label): MEASURED_PEAKS.json when present, else
    the fallback figures of one earlier GB300 measurement."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "of measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, 1900.0, "of fallback"


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


def hot_kernel_rooflines(st, ms_p2p, ms_m2l, p, precision):
    """P2P against the FP32 pipe (derived peak) and M2L against its own pipe.

    P2P work: interactions x 23 flop.  M2L work: M2L pairs x 2 (p+1)^4 flop, the
    useful flops of the dense translation (the 3-way split, padding to 128 and
    empty rows of a tile are not counted)."""
    _, bf16_tf, label = measured_peaks()
    fp32_peak = SMS * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
    out = []
    p2p_tf = st["n_p2p_interactions"] * P2P_FLOPS / (ms_p2p * 1e-3) / 1e12
    out.append({"kernel": "k_p2p", "bound": "alu", "achieved": p2p_tf, "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": p2p_tf / fp32_peak, "traffic": captured_traffic("k_p2p"),
                "ms": ms_p2p, "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                "work": f"{st['n_p2p_interactions']} interactions x {P2P_FLOPS} flop"})
    P2 = (p + 1) ** 2
    m2l_tf = st["n_m2l_pairs"] * 2 * P2 * P2 / (ms_m2l * 1e-3) / 1e12
    if precision == "fp32":
        kern, bound, peak, src = "k_m2l_simt", "alu", fp32_peak, "derived FP32 peak (as for P2P)"
    elif precision == "tf32x3":
        kern, bound, peak = "k_m2l_tc<tf32x3>", "tensor", bf16_tf * 1.1 / 2.25
        src = f"TF32 = BF16 dense {label} x nominal ratio 1.1/2.25"
    else:
        kern, bound, peak, src = "k_m2l_tc<bf16x3>", "tensor", bf16_tf, f"BF16 dense {label}"
    out.append({"kernel": kern, "bound": bound, "achieved": m2l_tf, "peak": peak,
                "unit": "TFLOP/s", "frac": m2l_tf / peak, "traffic": captured_traffic(kern),
                "ms": ms_m2l, "peak_source": src,
                "work": f"{st['n_m2l_pairs']} M2L pairs x 2 (p+1)^4 = {2 * P2 * P2} flop"})
    return out


def tree_roofline(n, ms_tree):
    """The tree build (box, keys, radix sort, permute, level splits) against HBM.

    Algorithmic bytes per particle: 16 read (x, y, z, q) + 16 permuted write +
    12 key/index write, plus 24 per 8-bit radix pass (8 passes over 63-bit keys).
    The phase time includes every launch of the phase; it is a phase, not one kernel."""
    hbm, _, label = measured_peaks()
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
            st_list.append(solve(stats=True)[2])
            ends[k].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    # each rank solved its own replica: job time = slowest rank, work = all ranks
    total_ms, _, value = replicas.aggregate(sum(step_ms), n * args.steps, device=dev)
    ms_per_step = total_ms / args.steps
    clocks = clk.summary()

    # rooflines of the two hot kernels, from the library's event timing of each phase
    st0 = st_list[-1]
    ms_p2p = statistics.mean(s["ms_p2p"] for s in st_list)
    ms_m2l = statistics.mean(s["ms_m2l"] for s in st_list)
    rooflines = hot_kernel_rooflines(st0, ms_p2p, ms_m2l, w["p"], args.precision)
    # the FP32 pipe's measured ceilings beside the derived peak (context for the P2P line)
    ceil = fmm.measure_fp32()
    p2p_line = rooflines[0]
    body_tf = ceil["body_interactions_per_s"] * P2P_FLOPS / 1e12
    p2p_line["ceilings"] = {
        "ffma_stream_tflops": ceil["ffma_tflops"],
        "ffma_stream_frac_of_derived_peak": ceil["ffma_tflops"] / p2p_line["peak"],
        "p2p_body_tflops": body_tf,
        "p2p_body_frac_of_derived_peak": body_tf / p2p_line["peak"],
        "kernel_frac_of_body": p2p_line["achieved"] / body_tf,
        "what": "FP32x2 FMA chains alone, and the P2P interaction code on staged sources with no list walk "
                "(fmm_measure_fp32), timed live beside the solve"}
    roof = max(rooflines, key=lambda r: r["ms"])  # the dominant kernel
    rooflines.append(tree_roofline(n, statistics.mean(s["ms_tree"] for s in st_list)))
    solve_frac = solve_roofline_fraction(rooflines, ms_per_step)
    phases = {k: round(statistics.mean(s[k] for s in st_list), 4)
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
    acc = None
    if rank == 0:
        acc = accuracy(x, q, phi.cpu().numpy(), grad.cpu().numpy(), off=off)

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
                           "accuracy": accuracy(x, q, phi.cpu().numpy(), grad.cpu().numpy(), off=off)}

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
            ms, sts = [], []
            for k in range(nst):
                flush.fill_(float(k))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                sts.append(solve(stats=True, select=sel)[2])
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
            m = statistics.mean(ms)
            select_modes[sel] = {"value": n / (m / 1e3), "ms_per_step": m,
                                 "n_m2l_pairs": sts[-1]["n_m2l_pairs"],
                                 "n_m2p_pairs": sts[-1]["n_m2p_pairs"],
                                 "n_p2p_pairs": sts[-1]["n_p2p_pairs"],
                                 "n_p2p_interactions": sts[-1]["n_p2p_interactions"],
                                 "accuracy": accuracy(x, q, phi.cpu().numpy(), grad.cpu().numpy(), off=off)}

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
        solve()
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

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        v, _, desc = oracle_sample(x, q, w) if off is None else oracle_sample_batched(x, q, off, w)
        cpu = {"value": v, "unit": "particles/s", "cores": O.num_threads(), "kind": "oracle",
               "sample": desc}

    if rank == 0:
        line = {"metric": "FMM particles/s", "value": value, "unit": "particles/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_of(w, args), "roofline": roof, "rooflines": rooflines,
                "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(sum(s["n_launches"] for s in st_list)),
                "accuracy": acc, "m2l_modes": modes, "select_modes": select_modes,
                "cost_model": cost_model, "ncrit_tuning": ncrit_tuning, "per_system_loop": loop,
                "graph_replay": graph, "solve_roofline_fraction": solve_frac,
                "clocks": clocks, "phases_ms": phases,
                "counts": {k: st0[k] for k in ("ncells", "nleaves", "depth", "n_p2p_pairs",
                                               "n_p2p_interactions", "n_m2l_pairs",
                                               "n_offset_classes", "n_m2l_blocks", "n_m2p_pairs")}}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
