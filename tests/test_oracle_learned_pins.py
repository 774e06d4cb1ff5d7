"""Pins of the oracle's learned face flux (oracle/learned.c).

The paper has no learned flux (it solves every face with the Riemann
solvers of Sec. 2.4); the oracle writes out this build's definition:
features, network output y, F = F_E + k J y, the acceptance checks and the
HLLD fallback.  Each pin below ties a part of that definition to something
outside it:

* a zero network gives the HLLE flux (orc_hlle, written independently in
  its branch-free form) on every face: the correction term is wired in and
  F_E is HLLE;
* equal left and right states give the physical flux (HLLD of equal
  states), whatever the network: J vanishes, so the flux is consistent;
* a network whose output leaves the HLL bracket is rejected and the face
  takes HLLD bit for bit;
* with the bracket opened (tau huge) a network that empties the density, or
  the pressure, of an implied HLL-fan state is rejected the same way, while
  y = 0 is kept: the positivity checks look at the right states;
* the training target composed back through the flux gives HLLD: the sign
  and scaling of the correction match the target's definition;
* ideal MHD has no intrinsic scale: rescaling density by a and speeds by b
  (p by a b^2, B by sqrt(a) b) leaves the features and y unchanged and
  rescales every flux by its dimension -- a wrong exponent in a feature or
  flux scale breaks it.
"""
import numpy as np
import pytest

import oracle as O
from paper_2608_14048_gb300 import inputs as I

G = 5.0 / 3.0
DIMS = list(I.MLP_DIMS)
N_PARAM = sum(DIMS[l + 1] * DIMS[l] + DIMS[l + 1] for l in range(4))


def _const_net(y):
    """A network whose output is y whatever its input (last layer W = 0)."""
    p = I.mlp_init_params(3, bias_scale=0.1).astype(np.float64)
    o = N_PARAM - (7 * 128 + 7)
    p[o:o + 7 * 128] = 0.0
    p[o + 7 * 128:] = y
    return p


def _faces(n=400, seed=1, mhd=True):
    return I.face_states(n, seed, mhd=mhd, gamma=G)


def _hlle(wl, wr, bn):
    out = np.zeros((len(bn), 7))
    for f in range(len(bn)):
        O.lib().orc_hlle(G, O._dp(np.ascontiguousarray(wl[f])), O._dp(np.ascontiguousarray(wr[f])),
                         float(bn[f]), O._dp(out[f]))
    return out


def _hlld(wl, wr, bn):
    out = np.zeros((len(bn), 7))
    for f in range(len(bn)):
        O.lib().orc_hlld(G, O._dp(np.ascontiguousarray(wl[f])), O._dp(np.ascontiguousarray(wr[f])),
                         float(bn[f]), O._dp(out[f]))
    return out


def _fscale(wl, wr, bn):
    """Per face and component, the larger of the two sides' flux sizes."""
    k = np.array([O.learned_features(G, wl[f], wr[f], bn[f])[1] for f in range(len(bn))])
    return k


@pytest.mark.parametrize("mhd", [True, False])
def test_zero_network_is_hlle(mhd):
    wl, wr, bn = _faces(mhd=mhd)
    F, acc = O.learned_flux(G, wl, wr, bn, np.zeros(N_PARAM), tau=0.25, mhd=mhd)
    ref = _hlle(wl, wr, bn)
    k = _fscale(wl, wr, bn)
    # the HLL fan state of HLLE is positive for these speed bounds, so the
    # zero correction is accepted on every face
    assert acc.all()
    assert np.max(np.abs(F - ref) / k) < 1e-13


def test_equal_states_give_the_physical_flux():
    wl, _, bn = _faces(seed=2)
    p = I.mlp_init_params(5, bias_scale=0.3).astype(np.float64)
    F, acc, rec = O.learned_flux(G, wl, wl, bn, p, tau=0.25, info=True)
    assert acc.all()
    assert np.all(rec[:, 7] == 0.0)                     # J = 0
    assert np.any(np.abs(rec[:, 17:24]) > 0.1)          # the network does output something
    ref = _hlld(wl, wl, bn)                             # HLLD(U, U) = the physical flux
    assert np.max(np.abs(F - ref) / _fscale(wl, wl, bn)) < 1e-14


def test_output_outside_the_bracket_falls_back_to_hlld_exactly():
    wl, wr, bn = _faces(seed=3)
    _, _, rec = O.learned_flux(G, wl, wr, bn, np.zeros(N_PARAM), info=True)
    big = rec[:, 7] > 1e-2                              # faces with a real jump
    wl, wr, bn = wl[big], wr[big], bn[big]
    for q in range(7):
        y = np.zeros(7)
        y[q] = 50.0
        F, acc = O.learned_flux(G, wl, wr, bn, _const_net(y), tau=0.25)
        # 50 k_q J exceeds tau (S_R - S_L) |dU_q| + 0.02 k_q wherever J > 1e-3
        assert not acc.any(), q
        assert np.array_equal(F, _hlld(wl, wr, bn))


@pytest.mark.parametrize("q,what", [(0, "density"), (4, "pressure")])
def test_positivity_of_the_fan_states_rejects(q, what):
    wl, wr, bn = _faces(seed=4)
    _, _, rec = O.learned_flux(G, wl, wr, bn, np.zeros(N_PARAM), info=True)
    sel = rec[:, 7] > 1e-2
    wl, wr, bn = wl[sel], wr[sel], bn[sel]
    # the bracket is opened, so only the positivity test can reject
    F0, acc0 = O.learned_flux(G, wl, wr, bn, _const_net(np.zeros(7)), tau=1e12)
    assert acc0.all()
    # a mass (energy) flux far below F_E empties the fan state behind the
    # right-going wave (S_R > 0), one far above it the state behind the
    # left-going wave (S_L < 0): every subsonic face rejects both, a
    # supersonic face (one outer wave only) at least one of them
    acc = {}
    for sign in (-1.0, 1.0):
        y = np.zeros(7)
        y[q] = sign * 1e3
        F, acc[sign] = O.learned_flux(G, wl, wr, bn, _const_net(y), tau=1e12)
        r = ~acc[sign]
        assert np.array_equal(F[r], _hlld(wl[r], wr[r], bn[r]))
    assert not (acc[-1.0] & acc[1.0]).any(), what
    assert acc[-1.0].sum() + acc[1.0].sum() < 0.2 * len(bn), what


def test_target_composed_back_gives_hlld():
    wl, wr, bn = _faces(n=60, seed=6)
    for f in range(len(bn)):
        y = O.learned_target(G, wl[f], wr[f], bn[f])
        F, acc = O.learned_flux(G, wl[f:f + 1], wr[f:f + 1], bn[f:f + 1], _const_net(y), tau=1e12)
        ref = _hlld(wl[f:f + 1], wr[f:f + 1], bn[f:f + 1])
        k = _fscale(wl[f:f + 1], wr[f:f + 1], bn[f:f + 1])
        if acc[0]:
            assert np.max(np.abs(F - ref) / k) < 1e-12, f
        else:
            # HLLD's own fan state failing the positivity test: the fallback
            # is HLLD itself
            assert np.array_equal(F, ref)


@pytest.mark.parametrize("a,b", [(4.0, 1.0), (1.0, 3.0), (0.05, 0.2)])
def test_scale_invariance(a, b):
    wl, wr, bn = _faces(n=200, seed=7)
    p = I.mlp_init_params(8, bias_scale=0.05).astype(np.float64)
    F, acc, rec = O.learned_flux(G, wl, wr, bn, p, info=True)
    s = np.array([a, b, b, b, a * b * b, np.sqrt(a) * b, np.sqrt(a) * b])
    F2, acc2, rec2 = O.learned_flux(G, wl * s, wr * s, bn * np.sqrt(a) * b, p, info=True)
    dim = np.array([a * b, a * b * b, a * b * b, a * b * b, a * b ** 3,
                    np.sqrt(a) * b * b, np.sqrt(a) * b * b])
    k = _fscale(wl, wr, bn)
    assert np.array_equal(acc, acc2)
    assert np.max(np.abs(rec2[:, 17:24] - rec[:, 17:24])) < 1e-12   # same network output
    assert np.max(np.abs(F2 / dim - F) / k) < 1e-12
    assert 0 < acc.sum() < len(acc)            # both decisions occur on these faces
