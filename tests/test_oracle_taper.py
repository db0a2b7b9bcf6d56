"""Pins of the oracle's optional lubrication taper (the differentiable cutoff
used by the adjoint; not in the paper).  With taper width w the lubrication
of a listed pair at gap d is scaled by a factor s that must (i) be exactly 1
for d <= (1 - w) delta_ij, (ii) fall continuously to 0 at the cutoff
d = delta_ij, (iii) have zero slope at both ends (C1 joins), (iv) be 1/2 at
the middle of the band (the smoothstep is antisymmetric about it) and (v)
decrease monotonically across the band; contact forces are untouched."""
import numpy as np
import pytest

import oracle

W = 0.2


def _pair(d, w, ai=1.0, aj=1.4, mode=0):
    box = np.array([40.0, 40.0, 40.0])
    p = oracle.make_params(box, lub_taper=w, lub_cutoff_mode=mode, delta_lub=0.1)
    n = np.array([0.48, 0.6, 0.64])
    n /= np.linalg.norm(n)
    xi = np.array([20.0, 20.0, 20.0])
    xj = xi + (ai + aj + d) * n
    ui = np.array([0.3, -0.2, 0.1])
    uj = np.array([-0.1, 0.25, 0.05])
    wi = np.array([0.2, 0.1, -0.3])
    wj = np.array([-0.05, 0.3, 0.2])
    fl, Fi, Fj, Ti, Tj, S, xn = oracle.pair_eval(p, 0.0, xi, xj, ui, uj, wi, wj, ai, aj)
    return fl, np.concatenate([Fi, Fj, Ti, Tj, S.ravel()])


def _delta_ij(ai=1.0, aj=1.4, mode=0):
    return 0.1 * (ai + aj) / 2 if mode == 0 else 0.1


def _ratio(d, mode=0):
    fl0, v0 = _pair(d, 0.0, mode=mode)
    fl1, v1 = _pair(d, W, mode=mode)
    assert fl0 == fl1 == 1
    k = np.argmax(np.abs(v0))
    # every component scales by the same factor
    np.testing.assert_allclose(v1, (v1[k] / v0[k]) * v0, rtol=1e-12, atol=1e-14 * np.abs(v0).max())
    return v1[k] / v0[k]


@pytest.mark.parametrize("mode", [0, 1])
def test_full_strength_below_band_and_zero_at_cutoff(mode):
    dl = _delta_ij(mode=mode)
    for f in (0.0, 0.3, 0.79999):
        assert _ratio(f * dl, mode) == 1.0
    assert abs(_ratio(dl * (1 - 1e-9), mode)) < 1e-15


def test_c1_joins_midpoint_and_monotone():
    dl = _delta_ij()
    lo, hi = (1 - W) * dl, dl
    h = 1e-5 * dl
    # slope of s with respect to d at both ends of the band vanishes (in
    # units of the band width; it is 1.5 at the middle)
    band = hi - lo
    assert abs((_ratio(lo + h) - 1.0) / h) * band < 1e-3
    assert abs(_ratio(hi - h) / h) * band < 1e-3
    assert abs((_ratio(lo + 0.5 * band + h) - _ratio(lo + 0.5 * band - h)) / (2 * h)) * band == \
        pytest.approx(1.5, rel=1e-6)
    assert _ratio(0.5 * (lo + hi)) == pytest.approx(0.5, abs=1e-12)
    ds = np.linspace(lo, hi, 41)[1:-1]
    r = np.array([_ratio(d) for d in ds])
    assert np.all(np.diff(r) < 0) and r.max() < 1 and r.min() > 0
    # antisymmetry about the middle of the band
    np.testing.assert_allclose(r + r[::-1], 1.0, atol=1e-12)


def test_contact_is_not_tapered():
    fl0, v0 = _pair(-0.01, 0.0)
    fl1, v1 = _pair(-0.01, W)
    assert fl0 & 2 and fl1 & 2
    np.testing.assert_array_equal(v0, v1)
