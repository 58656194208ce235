"""Failure detection on the GPU without a fault: the fused kernel's bounded
wait on a staging copy runs out (lsas_plan_set_fault(1): block 0 waits for
16 bytes that no copy delivers), in each fused kernel: the per-warp kernel
(N = 1024), the warp-pair kernel (N = 2048 from sc16 rows) and the
warp-specialised one (N = 2048 from fc32 rows).  The call finishes,
lsas_plan_sync returns LSAS_ERR_TIMEOUT (and clears it), the other frames of
the same launch are still right, and the same plan then runs normally and
meets the oracle bars.
"""

import dataclasses
import time

import numpy as np
import pytest

import synth
from synth.frames import sweep_config
from tests.parity_util import check_frame_outputs, oracle_run

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,fmt", [(1024, "sc16"), (2048, "sc16"), (2048, "fc32")])
def test_bounded_wait_runs_out_and_recovers(N, fmt):
    import torch
    import paper_1901_07499_gb300.lsas as L
    cfg = sweep_config(16, N).replace(fmt=fmt)
    b = synth.generate(cfg, frame_ids=range(3))
    plan = L.Plan(cfg.M, cfg.N, cfg.cp, cfg.S, cfg.pilot_idx, cfg.Q, fmt=cfg.fmt, max_frames=4,
                  pilot=b.pilot)
    x = torch.from_numpy(np.ascontiguousarray(b.frames)).cuda()
    ref = oracle_run(cfg, b)
    assert L.lsas_plan_set_fault(plan.handle, 2) == L.LSAS_ERR_INVALID_ARG
    assert L.lsas_plan_set_fault(plan.handle, 1) == L.LSAS_OK
    t0 = time.time()
    H, bits, eq = plan.run_frame(x, want_eq=True)
    assert plan.sync_status() == L.LSAS_ERR_TIMEOUT
    assert time.time() - t0 < 30.0
    assert plan.sync_status() == L.LSAS_OK            # read clears it
    # frames 1 and 2 ran in other blocks and are unaffected
    sub = dataclasses.replace(ref, **{f.name: (getattr(ref, f.name)[1:]
                                               if getattr(ref, f.name) is not None else None)
                                       for f in dataclasses.fields(ref)})
    check_frame_outputs(cfg, sub, H.cpu().numpy()[1:], bits.cpu().numpy()[1:], eq.cpu().numpy()[1:])
    assert L.lsas_plan_set_fault(plan.handle, 0) == L.LSAS_OK
    H, bits, eq = plan.run_frame(x, want_eq=True)
    plan.sync()
    check_frame_outputs(cfg, ref, H.cpu().numpy(), bits.cpu().numpy(), eq.cpu().numpy())
