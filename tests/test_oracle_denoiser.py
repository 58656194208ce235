"""Pins of the FP64 denoiser reference (oracle/denoiser.py).

* conv equals numpy's correlation of the zero-padded row (the definition, by
  an independent library routine), channel by channel.
* prepare: every row of x0 has unit mean power and rms is the row's norm
  over sqrt(N); the refinement is scale-equivariant per row (c H -> c out
  for real c > 0, any weights).
* With every weight zero the residual network is the identity.
* The backward pass equals central finite differences of the forward pass
  (sampled parameters, tiny rows), and the MSE gradient likewise.
* Adam's first step from a zero state moves each parameter by
  lr * g / (|g| + eps).
* The LS-domain pairs have unit expected channel power and LS error
  variance sigma^2.
* bf16_round: exact bfloat16 values stay, ties go to the even significand,
  and the relative error never exceeds 2^-8; the activation hook is applied
  exactly once to each of the three ReLU outputs (with zero biases, doubling
  every activation scales the network's residual by 2^3).
"""

import numpy as np

from oracle import denoiser as dn
import synth


def test_conv_is_padded_correlation():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 17))
    W = rng.standard_normal((4, 3, 5))
    b = rng.standard_normal(4)
    out = dn.conv(x, W, b)
    for r in range(2):
        for o in range(4):
            want = b[o] + sum(np.correlate(np.pad(x[r, c], 2), W[o, c], "valid") for c in range(3))
            assert np.allclose(out[r, o], want, rtol=1e-12, atol=1e-12)


def test_prepare_normalises_each_row_to_unit_power():
    # rows of very different scale: each row of x0 has mean |x0|^2 = 1 and
    # rms is that row's root-mean-square magnitude (the norm divided by
    # sqrt(N), computed independently of the definition)
    rng = np.random.default_rng(11)
    scales = np.array([1e-3, 1.0, 37.0, 2e4])
    H = (rng.standard_normal((4, 48)) + 1j * rng.standard_normal((4, 48))) * scales[:, None]
    x0, rms = dn.prepare(H)
    assert x0.shape == (4, 2, 48)
    assert np.allclose(np.mean(x0[:, 0] ** 2 + x0[:, 1] ** 2, axis=-1), 1.0, rtol=0, atol=1e-12)
    assert np.allclose(rms, np.linalg.norm(H, axis=-1) / np.sqrt(48), rtol=1e-13)
    assert np.allclose(x0[:, 0] * rms[:, None], H.real, rtol=1e-13)
    assert np.allclose(x0[:, 1] * rms[:, None], H.imag, rtol=1e-13)


def test_refinement_is_scale_equivariant():
    # the network sees each row normalised by its own rms, so scaling a row
    # by a real c > 0 scales the refined row by c, for any weights (random
    # biases included, so the map is far from linear)
    rng = np.random.default_rng(12)
    params = dn.init_params(5) * 2.0
    params += 0.05 * rng.standard_normal(params.size)
    H = rng.standard_normal((3, 40)) + 1j * rng.standard_normal((3, 40))
    base = dn.apply(params, H)
    assert not np.allclose(base, H)             # the weights do something
    for c in (1e-3, 0.5, 7.0, 3e3):
        assert np.allclose(dn.apply(params, c * H), c * base, rtol=1e-11, atol=1e-11 * c)
    # per row: scaling one row leaves the others unchanged
    H2 = H.copy()
    H2[1] *= 9.0
    out2 = dn.apply(params, H2)
    assert np.allclose(out2[0], base[0], rtol=1e-12) and np.allclose(out2[2], base[2], rtol=1e-12)
    assert np.allclose(out2[1], 9.0 * base[1], rtol=1e-11)


def test_zero_weights_are_identity():
    rng = np.random.default_rng(2)
    H = rng.standard_normal((3, 32)) + 1j * rng.standard_normal((3, 32))
    assert np.allclose(dn.apply(np.zeros(dn.n_params()), H), H, rtol=1e-13)
    assert dn.n_params() == 10978


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(3)
    params = dn.init_params(7) * 3.0
    x0 = rng.standard_normal((2, 2, 12))
    t = rng.standard_normal((2, 2, 12))

    def loss(p):
        y, _ = dn.forward(p, x0)
        return dn.mse(y, t)[0]

    y, cache = dn.forward(params, x0)
    _, dy = dn.mse(y, t)
    g = dn.backward(params, cache, dy)
    idx = rng.choice(params.size, 300, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(params)
        e[i] = h
        fd = (loss(params + e) - loss(params - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_mse_gradient_and_adam_first_step():
    rng = np.random.default_rng(4)
    y, t = rng.standard_normal(50), rng.standard_normal(50)
    L, d = dn.mse(y, t)
    e = np.zeros(50)
    e[7] = 1e-7
    assert np.isclose((dn.mse(y + e, t)[0] - dn.mse(y - e, t)[0]) / 2e-7, d[7], rtol=1e-6)
    p, g = rng.standard_normal(20), rng.standard_normal(20)
    p1, m, v = dn.adam(p, g, np.zeros(20), np.zeros(20), 1, lr=0.01, eps=1e-8)
    assert np.allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_ls_pairs_statistics():
    H, Hls, snr = synth.ls_pairs(400, 256, snr_db_range=(10.0, 10.0), seed=5)
    assert abs(np.mean(np.abs(H) ** 2) - 1.0) < 0.1
    err = np.mean(np.abs(Hls - H) ** 2)
    assert abs(err - 0.1) < 0.005          # sigma^2 = 10^-1


def test_bf16_round_values_and_bound():
    u = 2.0 ** -7                     # bf16 spacing in [1, 2)
    got = dn.bf16_round(np.array([1.0, 1 + u / 2, 1 + 1.5 * u, 1 + 0.49 * u, -3.0, 0.0, 2.0 ** -130]))
    assert list(got[:6]) == [1.0, 1.0, 1 + 2 * u, 1.0, -3.0, 0.0]
    assert got[6] == 2.0 ** -130      # a bfloat16 subnormal: kept, not flushed
    x = np.random.default_rng(9).standard_normal(100_000) * 10.0 ** np.random.default_rng(10).uniform(-3, 3, 100_000)
    r = dn.bf16_round(x)
    assert np.max(np.abs(r - x) / np.abs(x)) <= 2.0 ** -8 * (1 + 1e-6)   # half the spacing 2^-7
    assert np.array_equal(dn.bf16_round(r), r)


def test_activation_hook_applied_once_per_relu():
    rng = np.random.default_rng(11)
    p = dn.init_params(5) * 3.0
    W1, b1, W2, b2, W3, b3, W4, b4 = dn.unpack(p)
    assert not b1.any() and not b4.any()          # init has zero biases
    x0 = rng.standard_normal((2, 2, 40))
    y, _ = dn.forward(p, x0)
    y2, _ = dn.forward(p, x0, act=lambda v: 2.0 * v)
    assert np.allclose(y2 - x0, 8.0 * (y - x0), rtol=1e-12, atol=1e-12)
    yb, _ = dn.forward(p, x0, act=dn.bf16_round)
    assert 0 < np.max(np.abs(yb - y)) < 0.05 * np.max(np.abs(y - x0))
