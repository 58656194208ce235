"""Call timing of a plan (lsas_plan_set_profile / lsas_plan_profile).

With profiling on, each call of a device entry point is timed by CUDA events
on its stream: the counts match the calls made, every time is positive, the
fused receiver's total agrees with CUDA events taken around the same calls
by the test (within 5 % plus 50 us), a read clears the totals, a buffer that
is too small is refused without losing them, and with profiling off nothing
is recorded.  The host-buffer call is timed on the host clock.
"""

import ctypes as C

import numpy as np
import pytest

import synth
from synth.frames import sweep_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available()
    import paper_1901_07499_gb300.lsas as lsas
    return lsas


def test_profile_counts_and_times(L):
    import torch
    cfg = sweep_config(32, 1024)
    F = 16
    b = synth.generate(cfg, frame_ids=range(F))
    plan = L.Plan(cfg.M, cfg.N, cfg.cp, cfg.S, cfg.pilot_idx, cfg.Q, fmt=cfg.fmt, max_frames=F,
                  pilot=b.pilot)
    x = torch.from_numpy(np.ascontiguousarray(b.frames)).cuda()
    H, bits, _ = plan.run_frame(x)                   # warm up, not recorded
    plan.sync()
    assert plan.profile() == {}
    plan.set_profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(5):
        plan.run_frame(x, H, bits)
    e1.record()
    plan.estimate(x, H)
    plan.demodulate(x, H, bits)
    plan.run_frame_split(x, 4, H, bits)
    xh = x.cpu().pin_memory()
    Hh = torch.empty(H.shape, dtype=H.dtype).pin_memory()
    bh = torch.empty(bits.shape, dtype=bits.dtype).pin_memory()
    plan.run_frame_host(xh, Hh, bh)
    plan.sync()
    # a buffer that is too small: refused, totals kept
    need = C.c_size_t()
    tiny = C.create_string_buffer(8)
    assert L.lsas_plan_profile(plan.handle, tiny, 8, C.byref(need)) == L.LSAS_ERR_CAPACITY
    assert need.value > 8
    prof = plan.profile()
    assert prof["lsas_run_frame"]["calls"] == 5
    assert prof["lsas_estimate"]["calls"] == 1 and prof["lsas_demodulate"]["calls"] == 1
    assert prof["lsas_run_frame_split_static"]["calls"] == 1
    assert prof["lsas_run_frame_host"]["calls"] == 1
    assert all(v["ms"] > 0 for v in prof.values())
    ref = e0.elapsed_time(e1)
    assert abs(prof["lsas_run_frame"]["ms"] - ref) <= 0.05 * ref + 0.05, (prof, ref)
    assert plan.profile() == {}                      # the read cleared them
    plan.set_profile(False)
    plan.run_frame(x, H, bits)
    plan.sync()
    assert plan.profile() == {}
