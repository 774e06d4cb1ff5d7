"""Pins of the FP64 MLP reference used to check the learned-flux kernels.

* SiLU closed form on a 1-1-1 network; a zero-weight network outputs its bias.
* Permuting hidden units (rows of W_l, b_l, columns of W_{l+1}) leaves the
  output unchanged: catches transposed or mis-indexed weight matrices.
* Backpropagation equals central finite differences of the forward pass.
"""
import math

import numpy as np

import oracle as O

DIMS = [14, 128, 128, 128, 7]


def _layers(dims, p):
    out, off = [], 0
    for l in range(len(dims) - 1):
        nin, nout = dims[l], dims[l + 1]
        W = p[off:off + nout * nin].reshape(nout, nin); off += nout * nin
        b = p[off:off + nout]; off += nout
        out.append((W, b))
    return out


def _pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers])


def test_silu_closed_form_and_zero_network():
    y = O.mlp_forward([1, 1, 1], np.array([1.0, 0.0, 1.0, 0.0]), np.array([[1.0], [-2.0]]))
    assert y[0, 0] == math.fsum([1.0 / (1.0 + math.exp(-1.0))])
    assert abs(y[1, 0] - (-2.0 / (1.0 + math.exp(2.0)))) < 1e-16
    rng = np.random.default_rng(0)
    p = np.zeros(O.mlp_param_count(DIMS))
    p[-7:] = rng.normal(size=7)
    x = rng.normal(size=(5, 14))
    np.testing.assert_array_equal(O.mlp_forward(DIMS, p, x), np.tile(p[-7:], (5, 1)))


def test_hidden_permutation_invariance():
    rng = np.random.default_rng(1)
    dims = [14, 32, 24, 7]
    p = rng.normal(size=O.mlp_param_count(dims)) * 0.3
    x = rng.normal(size=(9, 14))
    y0 = O.mlp_forward(dims, p, x)
    L = _layers(dims, p)
    perm1 = rng.permutation(32)
    perm2 = rng.permutation(24)
    (W1, b1), (W2, b2), (W3, b3) = L
    q = _pack([(W1[perm1], b1[perm1]), (W2[perm2][:, perm1], b2[perm2]), (W3[:, perm2], b3)])
    np.testing.assert_allclose(O.mlp_forward(dims, q, x), y0, rtol=1e-13, atol=1e-14)
    # permuting one side only is NOT invariant (the pin is sensitive)
    q2 = _pack([(W1[perm1], b1[perm1]), (W2, b2), (W3, b3)])
    assert np.max(np.abs(O.mlp_forward(dims, q2, x) - y0)) > 1e-3


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(2)
    dims = [14, 16, 12, 7]
    p = rng.normal(size=O.mlp_param_count(dims)) * 0.4
    x = rng.normal(size=(6, 14))
    t = rng.normal(size=(6, 7))
    loss, g = O.mlp_grad(dims, p, x, t)
    idx = rng.choice(p.size, 60, replace=False)
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h; pm[i] -= h
        lp = 0.5 * np.mean(np.sum((O.mlp_forward(dims, pp, x) - t) ** 2, axis=1))
        lm = 0.5 * np.mean(np.sum((O.mlp_forward(dims, pm, x) - t) ** 2, axis=1))
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    assert loss == 0.5 * np.mean(np.sum((O.mlp_forward(dims, p, x) - t) ** 2, axis=1)) or \
        abs(loss - 0.5 * np.mean(np.sum((O.mlp_forward(dims, p, x) - t) ** 2, axis=1))) < 1e-14
