"""Host-side logic of bench.py, on the CPU: the per-vertex byte model behind
the roofline figures, the synthetic workloads' shapes, and the reference
arm's JSON line (the oracle, run here on the host cores), including the
ranks other than 0 exiting without work."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_bytes_per_vertex_model():
    # AAR / AP: the scan reads s_k and a_k and writes x_k per block; the update
    # reads w, s_k, x_k and writes s_k
    b3 = bench.kernel_bytes_per_vertex(3, "aar")
    assert b3["prox"] == 36 and b3["update"] == 40 and b3["check_extra"] == 4
    b2 = bench.kernel_bytes_per_vertex(2, "ap")
    assert b2["prox"] == 24 and b2["update"] == 28
    # BCD: one block per launch
    bb = bench.kernel_bytes_per_vertex(3, "bcd")
    assert bb["prox"] == 12 and bb["update"] == 16 and bb["eval"] == 20
    bf = bench.kernel_bytes_per_vertex(2, "fista")
    assert bf["prox"] == 24 and bf["update"] == 28 and bf["eval"] == 16


def test_workload_shapes():
    dims, probs = bench.batch_problems(512, bench.WORKLOADS["batch512"]["seed"])
    assert len(dims) == 512 and len(probs) == 512
    H = np.array([d[0] for d in dims])
    W = np.array([d[1] for d in dims])
    assert H.min() >= 64 and H.max() <= 1024 and W.min() >= 64 and W.max() <= 768
    w, a = probs[7]
    assert w.shape == tuple(dims[7]) and a[0].shape == (dims[7][0] - 1, dims[7][1])
    assert a[1].shape == (dims[7][0], dims[7][1] - 1)
    w, a = bench.make_problem("volume256")
    assert w.shape == (256, 256, 256) and len(a) == 3 and w.dtype == np.int32
    assert a[0].shape == (255, 256, 256) and a[2].shape == (256, 256, 255)
    w, a = bench.make_problem("seg1024c8")
    assert w.shape == (1024, 1024) and len(a) == 4 and a[2].shape == (1023, 1023)
    # every config's convolution list: the 18 layers of a 4-level, 32-channel U-Net
    assert len(bench.UNET_CONVS) == 18 and bench.UNET_CONVS[0] == (0, 16, 32) and bench.UNET_CONVS[-1] == (0, 32, 16)


def run_bench(args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True, text=True,
                         cwd=ROOT, env=e, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return [json.loads(l) for l in out.stdout.splitlines() if l.startswith("{")]


def test_reference_arm_line():
    lines = run_bench(["--impl", "reference", "--workload", "seg1024", "--steps", "2", "--warmup", "1"])
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["metric"] == "Mvertex-iter/s" and d["unit"] == "Mvertex-iter/s"
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1 and d["value"] > 0
    assert d["config"]["workload"] == "seg1024"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_no_work():
    lines = run_bench(["--impl", "reference", "--workload", "seg1024", "--steps", "1", "--warmup", "0"],
                      env={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert lines == []
