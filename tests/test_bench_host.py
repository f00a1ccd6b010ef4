"""Host logic of bench.py that needs no GPU: the reference arm's line reports the
steps it ran and a per-step time that fits the wall clock around it, and the
accuracy record's worst-particle figures."""
import contextlib
import io
import json
import time
import types

import numpy as np

import bench


def test_reference_line_matches_what_ran():
    args = types.SimpleNamespace(workload="uniform4k", p=None, ncrit=None, steps=3, warmup=1, gpus=1,
                                 precision="tf32x3", select="plain")
    buf = io.StringIO()
    t0 = time.perf_counter()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(args)
    wall = time.perf_counter() - t0
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 3 and line["warmup"] == 1
    # the timed steps fit inside the wall clock of the whole run
    assert line["ms_per_step"] * line["steps"] <= 1e3 * wall
    cb = line["cpu_baseline"]
    assert cb["measured"] and cb["kind"] == "oracle" and cb["cores"] >= 1
    # value = particles evaluated per measured second of the timed steps
    assert abs(line["value"] - cb["particles_per_step"] / (line["ms_per_step"] * 1e-3)) <= 1e-6 * line["value"]
    assert 0 < cb["particles_per_step"] < 4096


def test_compare_reports_relative_and_worst_errors():
    t = np.array([0, 2, 3])
    pd = np.array([1.0, -2.0, 4.0])
    gd = np.array([[1.0, 0, 0], [0, 2.0, 0], [0, 0, -3.0]])
    phi = np.zeros(5)
    grad = np.zeros((5, 3))
    phi[t] = pd
    grad[t] = gd
    phi[3] += 0.04            # worst phi error 0.04 of max |phi*| = 4
    grad[2, 1] += 0.3         # worst grad error 0.3 of max |grad*| = 3
    r = bench.compare((t, pd, gd, 0.0), phi, grad)
    assert abs(r["max_err_phi_rel_max"] - 0.01) < 1e-12
    assert abs(r["max_err_grad_rel_max"] - 0.1) < 1e-12
    assert abs(r["rel_l2_phi"] - 0.04 / np.sqrt(21.0)) < 1e-12
    assert r["targets"] == 3
