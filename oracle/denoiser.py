"""FP64 reference of the learned LS-channel denoiser (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may import this module; it shares no code with the CUDA library.

The denoiser refines the LS estimate of Sec. II-C, one antenna row of N
subcarriers at a time (the paper's LS is the fallback and the yardstick):

  rms  = sqrt(mean_k |H_LS[k]|^2)                     per row
  x0   = [Re H_LS / rms, Im H_LS / rms]               2 channels x N
  a1 = conv(x0; W1, b1), r1 = relu(a1)                2 -> 32
  a2 = conv(r1; W2, b2), r2 = relu(a2)                32 -> 32
  a3 = conv(r2; W3, b3), r3 = relu(a3)                32 -> 32
  a4 = conv(r3; W4, b4)                               32 -> 2
  y  = x0 + a4,  H = (y[0] + j y[1]) * rms            residual, denormalised
  conv(x; W, b)[o][p] = b[o] + sum_c sum_{k<5} W[o][c][k] x[c][p + k - 2]
  (zero outside 0 <= p < N).

Training minimises the mean squared error between y and the true channel
normalised by the same rms, with Adam.  Parameters are one flat vector in
the order W1, b1, W2, b2, W3, b3, W4, b4.
"""

from __future__ import annotations

import numpy as np

K = 5
SHAPES = [(32, 2, K), (32,), (32, 32, K), (32,), (32, 32, K), (32,), (2, 32, K), (2,)]


def n_params() -> int:
    return int(sum(np.prod(s) for s in SHAPES))


def unpack(params: np.ndarray):
    out, o = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(np.asarray(params[o:o + n], np.float64).reshape(s))
        o += n
    return out


def init_params(seed: int = 0) -> np.ndarray:
    """He-style initial weights, zero biases, a small last layer (the network
    starts close to the identity through the residual)."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, s in enumerate(SHAPES):
        if len(s) == 1:
            parts.append(np.zeros(s))
        else:
            fan_in = s[1] * s[2]
            scale = np.sqrt(2.0 / fan_in) * (0.1 if i == 6 else 1.0)
            parts.append(rng.standard_normal(s) * scale)
    return np.concatenate([p.reshape(-1) for p in parts])


def conv(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x [R][Cin][N] -> [R][Cout][N] (the definition above)."""
    R, Cin, N = x.shape
    xp = np.zeros((R, Cin, N + K - 1))
    xp[:, :, 2:2 + N] = x
    out = np.zeros((R, W.shape[0], N))
    for k in range(K):
        out += np.einsum("oc,rcn->ron", W[:, :, k], xp[:, :, k:k + N])
    return out + b[None, :, None]


def prepare(H: np.ndarray):
    """H [R][N] complex -> (x0 [R][2][N], rms [R])."""
    H = np.asarray(H, np.complex128)
    rms = np.sqrt(np.mean(np.abs(H) ** 2, axis=-1))
    x0 = np.stack([H.real, H.imag], axis=1) / rms[:, None, None]
    return x0, rms


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (8 significant bits, ties to even) by way
    of float32, as a kernel rounds its float32 sums: the float32 bit pattern
    plus 0x7FFF plus the lowest kept bit, truncated to the upper 16 bits."""
    b = np.asarray(x, np.float64).astype(np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(params: np.ndarray, x0: np.ndarray, act=None):
    """Network output y and the pre-activations.  ``act`` (optional) is
    applied to every ReLU output before the next layer reads it: the
    tensor-core inference path stores its activations as bfloat16, which
    ``act=bf16_round`` reproduces."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(params)
    f = (lambda v: v) if act is None else act
    a1 = conv(x0, W1, b1)
    a2 = conv(f(np.maximum(a1, 0)), W2, b2)
    a3 = conv(f(np.maximum(a2, 0)), W3, b3)
    a4 = conv(f(np.maximum(a3, 0)), W4, b4)
    return x0 + a4, (x0, a1, a2, a3)


def conv_backward(dout: np.ndarray, x: np.ndarray, W: np.ndarray):
    """Gradients of conv: (d input, d W, d b)."""
    R, Cin, N = x.shape
    xp = np.zeros((R, Cin, N + K - 1))
    xp[:, :, 2:2 + N] = x
    dW = np.zeros_like(W)
    dxp = np.zeros_like(xp)
    for k in range(K):
        dW[:, :, k] = np.einsum("ron,rcn->oc", dout, xp[:, :, k:k + N])
        dxp[:, :, k:k + N] += np.einsum("oc,ron->rcn", W[:, :, k], dout)
    return dxp[:, :, 2:2 + N], dW, dout.sum(axis=(0, 2))


def backward(params: np.ndarray, cache, dy: np.ndarray) -> np.ndarray:
    """dL/dparams from dL/dy (the residual passes dy to x0, which has no
    parameters)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(params)
    x0, a1, a2, a3 = cache
    d3, gW4, gb4 = conv_backward(dy, np.maximum(a3, 0), W4)
    d3 = d3 * (a3 > 0)
    d2, gW3, gb3 = conv_backward(d3, np.maximum(a2, 0), W3)
    d2 = d2 * (a2 > 0)
    d1, gW2, gb2 = conv_backward(d2, np.maximum(a1, 0), W2)
    d1 = d1 * (a1 > 0)
    _, gW1, gb1 = conv_backward(d1, x0, W1)
    return np.concatenate([g.reshape(-1) for g in (gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4)])


def mse(y: np.ndarray, t: np.ndarray):
    """(loss, dL/dy) of the mean squared error over all elements."""
    d = y - t
    return float(np.mean(d ** 2)), 2.0 * d / d.size


def adam(params, grad, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (bias-corrected), step counted from 1."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad ** 2
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def apply(params: np.ndarray, H: np.ndarray, act=None) -> np.ndarray:
    """Denoised channel rows H [R][N] complex (``act`` as in forward)."""
    x0, rms = prepare(H)
    y, _ = forward(params, x0, act)
    return (y[:, 0] + 1j * y[:, 1]) * rms[:, None]
