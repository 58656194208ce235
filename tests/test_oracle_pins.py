"""Pins of the FP64 oracle to facts the method and the mathematics fix.

No test here compares the oracle with itself.  Each check is chosen so that a
plausible slip in the oracle (wrong DFT sign or scale, an off-by-one CP window,
a missing conjugate in LS or MRC, the wrong MRC normaliser, a transposed
operand, a wrong Gray label or tie rule, bit order) fails at least one of them:

* FFT: textbook worked example (golden), numpy's FFT as an independent library
  routine, brute-force summation on tiny N, Parseval, impulse and tone.
* CP removal: index-encoded samples.
* LS: noiseless single-tap and multi-tap channels against the closed-form
  frequency response; a complex (non +-1) pilot, where a missing conjugate
  shows; pilot at a symbol other than the first.
* MRC: M = 1 equals per-subcarrier division; permutation and scale invariance;
  identical antennas; noiseless recovery of the transmitted symbols.  The
  antenna split: shard partials recover the symbols of a noiseless channel,
  reduce to division for one antenna, match the whole array for any partition
  and flag only bins with no energy in any shard.
* Demap: brute-force nearest constellation point, Gray adjacency, golden Gray
  table, round trip through the transmitter's independent mapper, tie rule.
* Statistics: LS error variance = sigma^2, and QPSK MRC bit-error rate against
  the closed form for M-branch Rayleigh diversity.
* Packet detection: the PN chips form an m-sequence (two-valued periodic
  autocorrelation), the metric equals numpy's correlation, a noiseless
  single-tap capture peaks at the true delay with the closed-form height, and
  a multipath capture peaks on one of the channel's paths.  fftshift moves a
  tone by half the band.
"""

import cmath
import math
import os

import numpy as np
import pytest

import oracle
import synth
from synth.frames import FrameConfig

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- FFT ----

def test_dft_textbook_example():
    rows = np.array(_golden_rows("dft4.txt"), dtype=np.float64)
    x = rows[:, 1] + 1j * rows[:, 2]
    want = rows[:, 3] + 1j * rows[:, 4]
    assert np.allclose(oracle.dft(x), want, atol=1e-14)


@pytest.mark.parametrize("N", [64, 128, 256, 512, 1024, 2048])
def test_dft_matches_numpy_fft(N):
    rng = np.random.default_rng(N)
    x = rng.standard_normal((3, N)) + 1j * rng.standard_normal((3, N))
    want = np.fft.fft(x, axis=-1) / np.sqrt(N)
    got = oracle.dft(x)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.sqrt(np.mean(np.abs(want) ** 2))


@pytest.mark.parametrize("N", [1, 2, 4, 8, 16])
def test_dft_brute_force_small(N):
    rng = np.random.default_rng(100 + N)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    brute = []
    for k in range(N):
        acc = 0j
        for n in range(N):
            acc += x[n] * cmath.exp(-2j * math.pi * k * n / N)
        brute.append(acc / math.sqrt(N))
    assert np.allclose(oracle.dft(x), brute, atol=1e-13)


def test_dft_parseval_impulse_tone():
    N = 256
    rng = np.random.default_rng(7)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    Y = oracle.dft(x)
    assert abs(np.sum(np.abs(x) ** 2) - np.sum(np.abs(Y) ** 2)) < 1e-9
    # impulse at n0 -> exp(-2j pi k n0 / N) / sqrt(N)
    n0 = 5
    imp = np.zeros(N, complex); imp[n0] = 1
    k = np.arange(N)
    assert np.allclose(oracle.dft(imp), np.exp(-2j * np.pi * k * n0 / N) / 16, atol=1e-14)
    # tone exp(+2j pi k0 n / N) -> sqrt(N) at +k0 only (sign convention)
    k0 = 37
    tone = np.exp(2j * np.pi * k0 * np.arange(N) / N)
    Yt = oracle.dft(tone)
    assert abs(Yt[k0] - 16) < 1e-12
    Yt[k0] = 0
    assert np.max(np.abs(Yt)) < 1e-12


# ---------------------------------------------------------- CP removal ----

def test_strip_cp_positions():
    N, cp, S, M = 8, 3, 4, 2
    y = np.arange(M * S * (N + cp)).reshape(M, S * (N + cp)).astype(complex)
    r = oracle.strip_cp(y, N, cp, S)
    for m in range(M):
        for s in range(S):
            base = m * S * (N + cp) + s * (N + cp) + cp
            assert np.array_equal(r[m, s].real, np.arange(base, base + N))


# ------------------------------------------------------------------ LS ----

def _closed_form_H(taps, N):
    """H[k] = sum_l h_l exp(-2j pi k l / N) by direct summation over taps."""
    k = np.arange(N)
    return sum(taps[..., l, None] * np.exp(-2j * np.pi * k * l / N)
               for l in range(taps.shape[-1]))


def _run(cfg, batch, H_given=None):
    return oracle.receive(batch.frames, cfg.N, cfg.cp, cfg.S, cfg.pilot_idx,
                          cfg.Q, batch.pilot, H_given=H_given)


@pytest.mark.parametrize("pilot_idx", [0, 3])
def test_noiseless_single_tap_exact(pilot_idx):
    cfg = FrameConfig(M=3, N=64, cp=16, S=6, Q=16, pilot_idx=pilot_idx,
                      snr_db=None, fmt="fc32", F=2)
    h0 = 0.8 - 0.45j
    b = synth.generate(cfg, taps=np.array([h0]))
    res = _run(cfg, b)
    # fc32 input carries float32 rounding of the received samples
    assert np.max(np.abs(res.H - h0)) < 1e-5
    ds = oracle.data_symbols(cfg.S, cfg.pilot_idx)
    assert np.max(np.abs(res.z - b.X[:, ds, :])) < 1e-5
    assert np.array_equal(res.bits, b.bits)


def test_noiseless_multitap_closed_form():
    cfg = FrameConfig(M=4, N=128, cp=16, S=3, Q=4, taps=9, decay_db=1.0,
                      snr_db=None, fmt="fc32", F=3)
    b = synth.generate(cfg)
    res = _run(cfg, b)
    Ht = _closed_form_H(b.taps, cfg.N)              # [F][M][N]
    rms = np.sqrt(np.mean(np.abs(Ht) ** 2))
    assert np.max(np.abs(res.H - Ht)) < 1e-5 * rms
    assert np.array_equal(res.bits, b.bits)


def test_ls_complex_pilot_needs_conjugate():
    cfg = FrameConfig(M=2, N=64, cp=8, S=3, Q=4, taps=3, snr_db=None,
                      fmt="fc32", F=2)
    rng = np.random.default_rng(3)
    pilot = (rng.standard_normal(64) + 1j * rng.standard_normal(64)) * 1.3
    b = synth.generate(cfg, pilot=pilot)
    res = _run(cfg, b)
    Ht = _closed_form_H(b.taps, cfg.N)
    assert np.max(np.abs(res.H - Ht)) < 1e-4 * np.sqrt(np.mean(np.abs(Ht) ** 2))


def test_sc16_scaling_and_gain():
    cfg = synth.CONFIGS["scale"].replace(M=8, N=256, cp=32, F=2,
                                         snr_db=None)
    b = synth.generate(cfg)
    y = b.as_complex()
    rms = np.sqrt(np.mean(np.abs(y[0]) ** 2))
    assert abs(rms - 2048) < 1.0
    assert b.frames.dtype == np.int16 and np.max(np.abs(b.frames)) <= 32767
    res = _run(cfg, b)
    # H is in int16 count units: g * (true frequency response), up to the
    # rounding of the samples to integers (|error| <= 0.5 per component)
    Ht = _closed_form_H(b.taps, cfg.N) * b.gain[:, None, None]
    assert np.sqrt(np.mean(np.abs(res.H - Ht) ** 2)) < 1.0


# ----------------------------------------------------------------- MRC ----

def test_mrc_single_antenna_is_division():
    rng = np.random.default_rng(11)
    H = rng.standard_normal((1, 32)) + 1j * rng.standard_normal((1, 32))
    Y = rng.standard_normal((1, 5, 32)) + 1j * rng.standard_normal((1, 5, 32))
    z, E, bad = oracle.mrc(H, Y)
    assert not bad
    assert np.allclose(z, Y[0] / H[0], rtol=1e-13)


def test_mrc_invariances():
    rng = np.random.default_rng(12)
    H = rng.standard_normal((6, 16)) + 1j * rng.standard_normal((6, 16))
    Y = rng.standard_normal((6, 4, 16)) + 1j * rng.standard_normal((6, 4, 16))
    z, E, _ = oracle.mrc(H, Y)
    p = rng.permutation(6)
    zp, _, _ = oracle.mrc(H[p], Y[p])
    assert np.allclose(z, zp, rtol=1e-13)
    c = 3.7 - 1.2j          # y -> c y scales both H and Y by c
    zc, Ec, _ = oracle.mrc(c * H, c * Y)
    assert np.allclose(z, zc, rtol=1e-12)
    assert np.allclose(Ec, abs(c) ** 2 * E, rtol=1e-12)
    # M copies of one antenna combine to that antenna alone
    zr, _, _ = oracle.mrc(np.repeat(H[:1], 5, 0), np.repeat(Y[:1], 5, 0))
    z1, _, _ = oracle.mrc(H[:1], Y[:1])
    assert np.allclose(zr, z1, rtol=1e-13)
    # the weights are the conjugate channel: an antenna with Y = H x gives x
    x = rng.standard_normal(16) + 1j * rng.standard_normal(16)
    zx, _, _ = oracle.mrc(H, H[:, None, :] * x)
    assert np.allclose(zx[0], x, rtol=1e-12)


def test_mrc_zero_energy_flag():
    H = np.zeros((2, 8), complex)
    H[:, 1:] = 1.0
    Y = np.ones((2, 3, 8), complex)
    z, E, bad = oracle.mrc(H, Y)
    assert bad and np.all(z[:, 0] == 0) and np.allclose(z[:, 1:], 1.0)


def _partition(M, rng):
    cuts = sorted(rng.choice(np.arange(1, M), size=min(3, M - 1), replace=False))
    return list(zip([0] + cuts, cuts + [M]))


def test_mrc_antenna_split_recovers_symbols_and_divides():
    rng = np.random.default_rng(14)
    M, D, N = 7, 3, 16
    H = rng.standard_normal((M, N)) + 1j * rng.standard_normal((M, N))
    x = rng.standard_normal((D, N)) + 1j * rng.standard_normal((D, N))
    Y = H[:, None, :] * x                        # noiseless: every antenna sees H x
    for bounds in ([(m, m + 1) for m in range(M)], _partition(M, rng)):
        parts = [oracle.mrc_partial(H[a:b], Y[a:b]) for a, b in bounds]
        z, E, bad = oracle.mrc_combine([P for P, _ in parts], [e for _, e in parts])
        assert not bad
        assert np.allclose(z, x, rtol=1e-12)     # conj(H) weights undo the channel
        assert np.allclose(E, np.sum(H.real ** 2 + H.imag ** 2, axis=0), rtol=1e-13)
    # one antenna in one shard: the combiner is the per-subcarrier division
    Yn = rng.standard_normal((1, D, N)) + 1j * rng.standard_normal((1, D, N))
    P, e = oracle.mrc_partial(H[:1], Yn)
    z1, _, _ = oracle.mrc_combine([P], [e])
    assert np.allclose(z1, Yn[0] / H[0], rtol=1e-13)


def test_mrc_antenna_split_matches_whole_array_and_flags():
    rng = np.random.default_rng(15)
    M, D, N = 9, 4, 32
    H = rng.standard_normal((M, N)) + 1j * rng.standard_normal((M, N))
    Y = rng.standard_normal((M, D, N)) + 1j * rng.standard_normal((M, D, N))
    zf, Ef, _ = oracle.mrc(H, Y)
    for _ in range(3):
        parts = [oracle.mrc_partial(H[a:b], Y[a:b]) for a, b in _partition(M, rng)]
        z, E, bad = oracle.mrc_combine([P for P, _ in parts], [e for _, e in parts])
        assert not bad and np.allclose(z, zf, rtol=1e-12) and np.allclose(E, Ef, rtol=1e-13)
    # a shard with no energy at a bin is fine while another shard has some
    H0 = H.copy()
    H0[:4, 5] = 0
    H0[:, 7] = 0
    parts = [oracle.mrc_partial(H0[a:b], Y[a:b]) for a, b in ((0, 4), (4, M))]
    z, E, bad = oracle.mrc_combine([P for P, _ in parts], [e for _, e in parts])
    assert bad and np.all(z[:, 7] == 0) and E[7] == 0
    assert np.allclose(z[:, 5], np.sum(np.conj(H0[4:, 5])[:, None] * Y[4:, :, 5], axis=0)
                       / np.sum(np.abs(H0[4:, 5]) ** 2), rtol=1e-12)


# ------------------------------------------------- packet detection ----

def test_pn_sequence_is_an_m_sequence():
    p = synth.pn_sequence()
    assert p.shape == (255,) and set(np.unique(p)) == {-1.0, 1.0}
    assert p.sum() == -1.0                      # 128 ones and 127 zeros
    ac = np.array([np.dot(p, np.roll(p, k)) for k in range(255)])
    assert ac[0] == 255 and np.all(ac[1:] == -1)   # two-valued autocorrelation


def test_pn_metric_matches_library_correlation():
    rng = np.random.default_rng(21)
    y = rng.standard_normal((3, 400)) + 1j * rng.standard_normal((3, 400))
    pn = synth.pn_sequence()
    W = 400 - 255 + 1
    want = sum(np.abs(np.correlate(y[m], pn, "valid")) ** 2 for m in range(3))
    assert np.allclose(oracle.pn_metric(y, pn, W), want, rtol=1e-12)


def test_pn_sync_noiseless_single_tap_closed_form():
    cfg = FrameConfig(M=4, N=64, cp=16, S=3, Q=4, taps=1, snr_db=None, fmt="fc32")
    c = synth.generate_capture(cfg, frame_ids=range(3), max_delay=200)
    pn = synth.pn_sequence()
    for i in range(3):
        y = oracle.to_complex(c.captures[i])
        off, metric = oracle.pn_sync(y, pn, c.max_delay)
        assert off == c.delay[i]
        h = c.taps[i][:, 0].astype(np.complex64).astype(np.complex128)
        assert np.isclose(metric[off], 255.0 ** 2 * np.sum(np.abs(h) ** 2), rtol=1e-5)


def test_pn_sync_multipath_lands_on_a_path():
    cfg = FrameConfig(M=8, N=256, cp=32, S=3, Q=16, taps=6, decay_db=2.0, snr_db=15.0, fmt="sc16")
    c = synth.generate_capture(cfg, frame_ids=range(6), max_delay=300)
    for i in range(6):
        off, _ = oracle.pn_sync(oracle.to_complex(c.captures[i]), c.pn, c.max_delay)
        assert c.delay[i] <= off < c.delay[i] + cfg.taps


def test_fftshift_moves_a_tone_half_a_band():
    N = 64
    for k0 in (0, 5, 40):
        x = np.exp(2j * np.pi * k0 * np.arange(N) / N)
        Xs = oracle.fftshift_rows(oracle.dft(x))
        assert np.argmax(np.abs(Xs)) == (k0 + N // 2) % N
    r = np.arange(12).reshape(2, 6)
    assert np.array_equal(oracle.fftshift_rows(r), np.roll(r, 3, axis=-1))


# --------------------------------------------------------------- demap ----

def test_gray_golden_table():
    rows = np.array(_golden_rows("gray4.txt"), dtype=np.int64)
    got = oracle.gray_bits(rows[:, 0], 2)
    assert np.array_equal(got, rows[:, 1:])


@pytest.mark.parametrize("Q", [2, 4, 16, 64, 256])
def test_demap_round_trip_and_brute_force(Q):
    q = int(math.log2(Q))
    rng = np.random.default_rng(Q)
    bits = rng.integers(0, 2, size=(4000, q), dtype=np.uint8)
    sym = synth.qam_map(bits, Q)
    assert abs(np.mean(np.abs(sym) ** 2) - 1.0) < 0.05
    got, margin = oracle.demap(sym, Q)
    assert np.array_equal(got, bits)
    # brute force: nearest of all Q points, for noisy points away from ties
    all_bits = np.array([[(i >> (q - 1 - j)) & 1 for j in range(q)]
                         for i in range(Q)], dtype=np.uint8)
    pts = synth.qam_map(all_bits, Q)
    if Q == 2:
        pts = pts.real
    z = sym + 0.3 * (rng.standard_normal(4000) + 1j * rng.standard_normal(4000)) / math.sqrt(Q)
    zz = z.real if Q == 2 else z
    nearest = np.argmin(np.abs(zz[:, None] - pts[None, :]), axis=1)
    dec, m = oracle.demap(z, Q)
    away = m > 1e-9
    assert np.array_equal(dec[away], all_bits[nearest][away])


@pytest.mark.parametrize("Q", [4, 16, 64])
def test_gray_adjacency(Q):
    L, A, w, _ = oracle.qam_axis(Q)
    lv = np.arange(L)
    g = oracle.gray_bits(lv, w)
    assert np.all(np.sum(g[1:] != g[:-1], axis=1) == 1)


def test_tie_goes_to_upper_level_and_margin():
    Q = 16
    L, A, w, _ = oracle.qam_axis(Q)
    th = oracle.thresholds(Q)
    assert np.allclose(th, [-2 * A, 0.0, 2 * A])
    lvl, dist = oracle.slice_axis(np.array([0.0, -2 * A, 2 * A, 0.5 * A, -5.0]), Q)
    assert list(lvl) == [2, 1, 3, 2, 0]
    assert np.allclose(dist, [0, 0, 0, 0.5 * A, 5.0 - 2 * A])
    # a float32 decision on the float32 copy of a value just above a boundary
    v = np.nextafter(np.float32(2 * A), np.float32(0))
    l32, _ = oracle.slice_axis(np.array([v], np.float32), Q, np.float32)
    assert l32[0] == 2


def test_pack_bits_golden():
    rows = _golden_rows("pack_msb.txt")
    bits = np.array(rows[0], dtype=np.uint8)[None, :]
    want = bytes(int(h, 16) for h in rows[1])
    assert oracle.pack_bits(bits).tobytes() == want


# ----------------------------------------------------------- statistics ----

@pytest.mark.slow
def test_ls_error_variance_equals_sigma2():
    snr = 10.0
    cfg = FrameConfig(M=16, N=256, cp=32, S=2, Q=4, taps=6, decay_db=2.0,
                      snr_db=snr, fmt="fc32", F=30, seed=99)
    b = synth.generate(cfg)
    res = _run(cfg, b)
    err = res.H - _closed_form_H(b.taps, cfg.N)
    n = err.size                                   # 122880 samples
    mse = np.mean(np.abs(err) ** 2)
    s2 = 10 ** (-snr / 10)
    # |err|^2 / sigma^2 is Exp(1): standard error of the mean is 1/sqrt(n)
    assert abs(mse / s2 - 1.0) < 4.0 / math.sqrt(n)


def _mrc_ber_closed_form(M, gamma):
    mu = math.sqrt(gamma / (1.0 + gamma))
    return ((1 - mu) / 2) ** M * sum(math.comb(M - 1 + k, k) * ((1 + mu) / 2) ** k
                                     for k in range(M))


@pytest.mark.slow
@pytest.mark.parametrize("M", [1, 2, 4])
def test_qpsk_mrc_diversity_ber(M):
    # genie channel, iid Rayleigh per (frame, subcarrier, antenna), QPSK
    rng = np.random.default_rng(500 + M)
    n = 400000
    sigma2 = 0.5
    gamma = 1.0 / (2.0 * sigma2)                   # per-branch Eb/N0
    bits = rng.integers(0, 2, size=(n, 2), dtype=np.uint8)
    x = synth.qam_map(bits, 4)
    H = (rng.standard_normal((M, n)) + 1j * rng.standard_normal((M, n))) / math.sqrt(2)
    w = (rng.standard_normal((M, n)) + 1j * rng.standard_normal((M, n))) * math.sqrt(sigma2 / 2)
    Y = (H * x + w)[:, None, :]
    z, _, _ = oracle.mrc(H, Y)
    dec, _ = oracle.demap(z[0], 4)
    ber = np.mean(dec != bits)
    p = _mrc_ber_closed_form(M, gamma)
    se = math.sqrt(p * (1 - p) / (2 * n))
    assert abs(ber - p) < 5 * se + 1e-4 * p, (ber, p)
