"""GPU parity of the antenna split: lsas_mrc_partial per shard of antennas,
then lsas_mrc_combine over the shards (the distributed receiver of Sec. IV,
run as G logical shards on one GPU and reduced in fixed shard order).

Checked against
* the FP64 oracle's per-shard partial sums P = sum conj(H) Y, E = sum |H|^2
  (per frame and shard, max error / rms <= 1e-4),
* the oracle receiver (H, z, bits) at the bars of the whole path,
* the unsharded GPU run: H bit-identical (an antenna's transform does not
  depend on its neighbours), bits identical wherever the oracle is sure,
* the combine step alone on the oracle's partials, including subcarriers
  with no energy in any shard (z = 0, LSAS_ERR_DEVICE latched),
for even and uneven splits, one-antenna shards, ragged antenna chunks, FFT
lengths 64 .. 2048, plus determinism and argument errors.
"""

import numpy as np
import pytest

import oracle
import synth
from synth.frames import sweep_config
from tests.parity_util import (MARGIN, TOL_REL, check_frame_outputs, oracle_run,
                               rel_err, to_torch_frames, unpack)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available()
    import paper_1901_07499_gb300.lsas as lsas
    return lsas


def make_plan(L, cfg, max_frames=1024):
    return L.Plan(cfg.M, cfg.N, cfg.cp, cfg.S, cfg.pilot_idx, cfg.Q, fmt=cfg.fmt,
                  max_frames=max_frames, pilot=synth.frames.pilot_sequence(cfg))


def even_bounds(M, G):
    sizes = [M // G + (1 if g < M % G else 0) for g in range(G)]
    ends = np.cumsum(sizes)
    return [(int(e - s), int(e)) for s, e in zip(sizes, ends)]


def run_split(L, plan, x, bounds, want_eq=True):
    import torch
    F = x.shape[0]
    H = torch.full((F, plan.M, plan.N), float("nan"), dtype=torch.complex64, device=x.device)
    P, E = plan.empty_partials(F, len(bounds), device=x.device)
    for g, (a, c) in enumerate(bounds):
        plan.mrc_partial(x, a, c - a, H, P[g], E[g])
    bits, eq = plan.mrc_combine(P, E, want_eq=want_eq)
    return H, P, E, bits, eq


def oracle_partials(cfg, ref, bounds):
    ds = oracle.data_symbols(cfg.S, cfg.pilot_idx)
    F = ref.H.shape[0]
    P = np.empty((len(bounds), F, cfg.D, cfg.N), np.complex128)
    E = np.empty((len(bounds), F, cfg.N))
    for g, (a, c) in enumerate(bounds):
        for f in range(F):
            P[g, f], E[g, f] = oracle.mrc_partial(ref.H[f, a:c], ref.Y[f, a:c][:, ds])
    return P, E


def check_split(L, cfg, bounds, F=2):
    b = synth.generate(cfg, frame_ids=range(F))
    plan = make_plan(L, cfg)
    x = to_torch_frames(b)
    H, P, E, bits, eq = run_split(L, plan, x, bounds)
    plan.sync()
    ref = oracle_run(cfg, b, keep_Y=True)
    Po, Eo = oracle_partials(cfg, ref, bounds)
    eP = rel_err(P.cpu().numpy(), Po, axes=(2, 3))
    eE = rel_err(E.cpu().numpy(), Eo, axes=(2,))
    assert eP.max() <= TOL_REL, f"partial P rel err {eP.max():.3g}"
    assert eE.max() <= TOL_REL, f"partial E rel err {eE.max():.3g}"
    stats = check_frame_outputs(cfg, ref, H.cpu().numpy(), bits.cpu().numpy(),
                                eq.cpu().numpy())
    # against the unsharded fused path on the same frames
    H1, bits1, _ = plan.run_frame(x)
    plan.sync()
    assert np.array_equal(H.cpu().numpy().view(np.uint32), H1.cpu().numpy().view(np.uint32))
    q = int(round(np.log2(cfg.Q)))
    g1 = unpack(bits1.cpu().numpy(), cfg.D, cfg.N, q)
    g2 = unpack(bits.cpu().numpy(), cfg.D, cfg.N, q)
    sure = ref.margin >= MARGIN
    assert not np.any(np.any(g1 != g2, axis=-1) & sure)
    stats.update(P=float(eP.max()), E=float(eE.max()))
    return stats


@pytest.mark.parametrize("G", [1, 2, 4, 8])
def test_tiny_even_splits(L, G):
    cfg = synth.CONFIGS["tiny"]
    check_split(L, cfg, even_bounds(cfg.M, G), F=4)


def test_scale_uneven_split(L):
    cfg = synth.CONFIGS["scale"]
    check_split(L, cfg, [(0, 20), (20, 37), (37, 64)], F=2)


@pytest.mark.parametrize("M,N,G", [(5, 64, 5), (13, 256, 3), (33, 512, 2), (7, 2048, 3),
                                   (40, 1024, 6)])
def test_split_grid(L, M, N, G):
    check_split(L, sweep_config(M, N).replace(M=M), even_bounds(M, G), F=2)


def test_precision_config_split(L):
    cfg = synth.CONFIGS["precision"]
    check_split(L, cfg, even_bounds(cfg.M, 4), F=1)


def test_shard_writes_only_its_rows(L):
    cfg = sweep_config(16, 256)
    b = synth.generate(cfg, frame_ids=range(2))
    plan = make_plan(L, cfg)
    x = to_torch_frames(b)
    H, P, E, _, _ = run_split(L, plan, x, [(5, 11)])
    plan.sync()
    h = H.cpu().numpy()
    assert np.all(np.isnan(h[:, :5])) and np.all(np.isnan(h[:, 11:]))
    assert np.all(np.isfinite(h[:, 5:11]))


def test_combine_alone_on_oracle_partials_and_zero_energy(L):
    import torch
    cfg = sweep_config(12, 512)
    b = synth.generate(cfg, frame_ids=range(3))
    ref = oracle_run(cfg, b, keep_Y=True)
    bounds = even_bounds(cfg.M, 3)
    Po, Eo = oracle_partials(cfg, ref, bounds)
    Eo[:, 1, 77] = 0.0          # no shard has energy at frame 1, bin 77
    Eo[0, 2, 5] = 0.0           # one shard empty, the others not: fine
    plan = make_plan(L, cfg)
    P = torch.from_numpy(Po.astype(np.complex64)).cuda()
    E = torch.from_numpy(Eo.astype(np.float32)).cuda()
    bits, eq = plan.mrc_combine(P, E, want_eq=True)
    assert plan.sync_status() == L.LSAS_ERR_DEVICE
    assert plan.sync_status() == L.LSAS_OK
    # the oracle's combiner on the float32-rounded inputs the kernel saw
    P32 = Po.astype(np.complex64).astype(np.complex128)
    E32 = Eo.astype(np.float32).astype(np.float64)
    z = eq.cpu().numpy()
    got = unpack(bits.cpu().numpy(), cfg.D, cfg.N, cfg.q)
    for f in range(3):
        zo, _, bad = oracle.mrc_combine(list(P32[:, f]), list(E32[:, f]))
        assert bad == (f == 1)
        assert rel_err(z[f], zo, axes=(0, 1)) <= 1e-6
        bo, margin = oracle.demap(zo, cfg.Q)
        assert not np.any(np.any(got[f] != bo, axis=-1) & (margin >= MARGIN))
    assert np.all(z[1, :, 77] == 0)
    zero_bits, _ = oracle.demap(np.zeros(1, complex), cfg.Q)
    assert np.all(got[1, :, 77] == zero_bits[0])


def test_split_is_deterministic(L):
    cfg = sweep_config(32, 1024)
    b = synth.generate(cfg, frame_ids=range(3))
    plan = make_plan(L, cfg)
    x = to_torch_frames(b)
    bounds = even_bounds(cfg.M, 4)
    r1 = [t.cpu().numpy() for t in run_split(L, plan, x, bounds)]
    r2 = [t.cpu().numpy() for t in run_split(L, plan, x, bounds)]
    plan.sync()
    for a, c in zip(r1, r2):
        assert np.array_equal(a.view(np.uint8), c.view(np.uint8))


def test_split_argument_errors(L):
    import torch
    cfg = sweep_config(8, 256)
    plan = make_plan(L, cfg, max_frames=4)
    x = torch.zeros((5, 8, cfg.T, 2), dtype=torch.int16, device="cuda")
    H = plan.empty_H(5)
    P, E = plan.empty_partials(5, 2)
    bits = plan.empty_bits(5)
    s = torch.cuda.current_stream().cuda_stream
    h = plan.handle
    ok, bad, cap = L.LSAS_OK, L.LSAS_ERR_INVALID_ARG, L.LSAS_ERR_CAPACITY
    part = lambda n, a, c, Pp=P.data_ptr(): L.lsas_mrc_partial(
        h, x.data_ptr(), n, a, c, H.data_ptr(), Pp, E.data_ptr(), s)
    assert part(2, 0, 8) == ok
    assert part(2, -1, 4) == bad
    assert part(2, 0, 0) == bad
    assert part(2, 5, 4) == bad
    assert part(2, 0, 9) == bad
    assert part(2, 0, 4, None) == bad
    assert part(5, 0, 4) == cap
    comb = lambda n, G, Pp=P.data_ptr(): L.lsas_mrc_combine(
        h, Pp, E.data_ptr(), G, n, bits.data_ptr(), None, s)
    assert comb(2, 2) == ok
    assert comb(0, 2) == ok
    assert comb(2, 0) == bad
    assert comb(2, 257) == bad
    assert comb(2, 2, P.data_ptr() + 4) == bad      # not 16-byte aligned
    assert comb(5, 2) == cap
    assert L.lsas_mrc_combine(h, P.data_ptr(), E.data_ptr(), 2, 2, None, None, s) == bad
    # the all-zero input has no channel energy anywhere: the combine flagged it
    assert plan.sync_status() == L.LSAS_ERR_DEVICE
    assert plan.sync_status() == L.LSAS_OK
