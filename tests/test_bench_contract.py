"""The benchmark's output contract, on CPU.

* The reference arm (the FP64 oracle) prints one JSON line with the
  contract's keys, its cpu_baseline describing the run, and an e2e block of
  its own value with no host-device bytes.
* roofline_fp32: nominal 5 N log2 N flop per FFT over every symbol of every
  antenna, against the FMA peak measured in the same run, or (marked
  nominal) SMs x 128 lanes x 2 flop x clock when there is none.
* roofline.traffic: the committed capture's bytes scaled by frames while the
  kernel source hash and workload match, None otherwise.
* --sweep: the antenna x FFT-length grid of the scale workload (CP = N/8)
  and the paper's own (N, CP) shapes.
"""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402
from synth.frames import sweep_config  # noqa: E402


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    assert d["metric"] == "antenna*subcarrier samples/s" and d["unit"] == "samples/s"
    assert d["higher_is_better"] is True and d["value"] > 0
    assert "workload" in d["config"]
    # the GPU arm's workload, not the size of the sample
    assert d["config"]["frames"] == synth.config_by_name("scale").F
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_fp32_roofline_arithmetic():
    cfg = synth.config_by_name("scale")
    r = bench.fp32_roofline(cfg, 1000, 2.0, {"sm_max_mhz": 2000.0}, sms=100)
    flops = 1000 * cfg.M * cfg.S * 5 * cfg.N * 10          # log2(1024) = 10
    assert r["flop_per_frame"] == pytest.approx(flops / 1000)
    assert r["achieved"] == pytest.approx(flops / 2e-3 / 1e12)
    assert r["peak"] == pytest.approx(100 * 128 * 2 * 2000e6 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["peak_source"] == "nominal"
    # with a measured FMA peak the roofline uses it
    fma = {"tflops": 70.0, "launch": "x", "clocks": {"sm_mhz": 1900.0}}
    m = bench.fp32_roofline(cfg, 1000, 2.0, {"sm_max_mhz": 2000.0}, fma=fma, sms=100)
    assert m["peak"] == 70.0 and m["peak_source"] == "measured"
    assert m["frac"] == pytest.approx(m["achieved"] / 70.0)


def test_traffic_follows_the_source_hash(monkeypatch):
    cfg = synth.config_by_name("scale")
    with open(bench.TRAFFIC_FILE) as fh:
        recs = json.load(fh)
    recs = recs if isinstance(recs, list) else [recs]
    rec = next(r for r in recs if r["workload"] == "scale")
    monkeypatch.setattr(bench, "kernel_hash", lambda kernel: rec["kernel_sha"])
    assert bench.ncu_traffic(cfg, 1000) == pytest.approx(rec["dram_bytes_per_frame"] * 1000)
    assert bench.ncu_traffic(synth.config_by_name("tiny"), 1000) is None   # other workload
    monkeypatch.setattr(bench, "kernel_hash", lambda kernel: "0" * 16)
    assert bench.ncu_traffic(cfg, 1000) is None                           # kernel changed


def test_sweep_shapes_cover_the_grid():
    shapes = bench.sweep_shapes()
    grid = {(c.M, c.N, c.cp) for c in shapes[:-2]}
    assert grid == {(M, N, N // 8) for M in (8, 16, 32, 64, 128) for N in (64, 256, 512, 1024, 2048)}
    assert [(c.M, c.N, c.cp) for c in shapes[-2:]] == [(16, 64, 16), (16, 1024, 72)]
    scale = synth.CONFIGS["scale"]
    for c in shapes:
        assert (c.S, c.Q, c.fmt, c.pilot_idx) == (scale.S, scale.Q, scale.fmt, scale.pilot_idx)


@pytest.mark.parametrize("M,N,fmt,kernel", [
    (64, 1024, "sc16", "twin_kernel"), (8, 1024, "sc16", "twin_kernel"),
    (32, 512, "sc16", "twin_kernel"), (31, 512, "sc16", "warp_kernel"),
    (128, 256, "sc16", "twin_kernel"), (127, 256, "sc16", "warp_kernel"),
    (128, 128, "sc16", "warp_kernel"), (128, 64, "sc16", "warp_kernel"),
    (8, 2048, "sc16", "twinpair_kernel"), (64, 1024, "fc32", "warp_kernel"),
    (64, 2048, "fc32", "frame_kernel")])
def test_fused_kernel_name_follows_the_plan(monkeypatch, M, N, fmt, kernel):
    """The kernel the benchmark names (and whose traffic entry it reads) is the
    one the plan picks: two symbols per step from sc16 rows at N = 1024 and
    2048, at N = 512 from 32 antennas and at N = 256 from 128; one symbol per
    step otherwise; LSAS_FUSED_KERNEL=warp keeps one symbol per step."""
    monkeypatch.delenv("LSAS_FUSED_KERNEL", raising=False)
    cfg = sweep_config(M, N).replace(fmt=fmt)
    assert bench.fused_kernel_name(cfg).split(" ")[0] == kernel
    monkeypatch.setenv("LSAS_FUSED_KERNEL", "warp")
    one = {"twin_kernel": "warp_kernel", "twinpair_kernel": "pair_kernel"}.get(kernel, kernel)
    assert bench.fused_kernel_name(cfg).split(" ")[0] == one


def test_kernel_hashes_cover_their_includes():
    """Each fused kernel's source hash (which decides whether a committed ncu
    traffic figure still describes the kernel) covers the file that defines
    the kernel and every local header it includes, directly or not."""
    import re
    csrc = bench.CSRC

    def text(name):
        with open(os.path.join(csrc, name)) as fh:
            return fh.read()

    def includes(name):
        return re.findall(r'^#include "([^"]+)"', text(name), re.M)

    for kernel, files in bench.KERNEL_SRC.items():
        defining = [f for f in os.listdir(csrc) if f.endswith((".cuh", ".cu"))
                    and re.search(r"__global__.*\b%s\(" % kernel, text(f))]
        assert len(defining) == 1, (kernel, defining)
        closure, todo = set(), [defining[0]]
        while todo:
            f = todo.pop()
            if f not in closure:
                closure.add(f)
                todo.extend(includes(f))
        assert set(files) == closure, (kernel, sorted(files), sorted(closure))
