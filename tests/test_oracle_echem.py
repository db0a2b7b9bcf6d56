"""Pins of the oracle's electro-chemical forces (Eq. 6-7, Fig. 3): checks
against what the mathematics fixes, not a retyped formula.

- The force derives from a closed-form pair potential U(d): its component
  along n (on i, towards j) is dU/dd, so integrated over the surface distance
  it must reproduce the potential difference of
  U_R = F_ER (abar/a0) lambda_D exp(-d/lambda_D) (repulsion) and
  U_A = (A abar / (12 eps)) atan(d/eps) (regularised van der Waals).
- The repulsion decays by e over one Debye length; at a fixed gap both terms
  scale with the harmonic radius abar = 2 a_i a_j/(a_i + a_j) as Eq. 6-7 state.
- Both terms are flat for overlapping pairs and continuous at contact; they
  vanish at and beyond 20 lambda_D and 4 a0 and not just below.
- A pair at rest beyond the lubrication range feels only the central force:
  equal and opposite, no torques, stresslet r (x) F with the sign of a
  tension for attraction and of a compression for repulsion.
- The brute-force list extends to the electro-chemical range."""
import math

import numpy as np
import pytest

import oracle

N = np.array([0.6, -0.48, 0.64])   # unit vector


def _p(**kw):
    base = dict(f_er=2.0, lambda_d=0.05, hamaker=0.0, vdw_eps=0.01)
    base.update(kw)
    return oracle.make_params([40.0, 40.0, 40.0], **base)


def _fn(p, d, ai, aj):
    return float(oracle.echem(p, d, ai, aj, N) @ N)


def _quad(f, a, b, m=20001):
    x = np.linspace(a, b, m)
    y = np.array([f(t) for t in x])
    return float(np.sum((y[1:] + y[:-1]) * np.diff(x)) * 0.5)


@pytest.mark.parametrize("ai,aj", [(1.0, 1.0), (1.0, 1.4), (2.5, 0.7)])
def test_repulsion_is_minus_gradient_of_its_potential(ai, aj):
    p = _p()
    abar = 2 * ai * aj / (ai + aj)
    lam = p.lambda_d
    U = lambda d: p.f_er * (abar / p.a0) * lam * math.exp(-d / lam)
    d1, d2 = 0.01, 0.7
    work = _quad(lambda d: _fn(p, d, ai, aj), d1, d2)
    assert work == pytest.approx(U(d2) - U(d1), rel=1e-6)


@pytest.mark.parametrize("ai,aj", [(1.0, 1.0), (1.0, 1.4)])
def test_attraction_is_minus_gradient_of_its_potential(ai, aj):
    p = _p(f_er=0.0, hamaker=0.3, vdw_eps=0.02)
    abar = 2 * ai * aj / (ai + aj)
    eps = p.vdw_eps * abar
    U = lambda d: (p.hamaker * abar / (12 * eps)) * math.atan(d / eps)
    d1, d2 = 0.0, 1.5
    work = _quad(lambda d: _fn(p, d, ai, aj), d1, d2, m=200001)
    assert work == pytest.approx(U(d2) - U(d1), rel=1e-6)


def test_debye_decay_and_harmonic_radius_scaling():
    p = _p()
    lam = p.lambda_d
    for d in (0.0, 0.1, 0.37):
        assert _fn(p, d + lam, 1.0, 1.4) / _fn(p, d, 1.0, 1.4) == pytest.approx(math.exp(-1.0), rel=1e-12)
    # abar(1, 1) = 1, abar(2, 2) = 2, abar(1, 3) = 1.5
    assert _fn(p, 0.2, 2.0, 2.0) / _fn(p, 0.2, 1.0, 1.0) == pytest.approx(2.0, rel=1e-12)
    assert _fn(p, 0.2, 1.0, 3.0) / _fn(p, 0.2, 1.0, 1.0) == pytest.approx(1.5, rel=1e-12)
    pa = _p(f_er=0.0, hamaker=0.5)
    # far from contact (d >> eps) the van der Waals term goes as abar / d^2
    assert _fn(pa, 1.0, 2.0, 2.0) / _fn(pa, 1.0, 1.0, 1.0) == pytest.approx(2.0, rel=1e-3)
    assert _fn(pa, 2.0, 1.0, 1.0) / _fn(pa, 1.0, 1.0, 1.0) == pytest.approx(0.25, rel=1e-3)


def test_contact_values_cutoffs_and_symmetry():
    p = _p(hamaker=0.3)
    ai, aj = 1.0, 1.4
    f0 = _fn(p, 0.0, ai, aj)
    for d in (-1e-12, -0.01, -0.3):
        assert _fn(p, d, ai, aj) == pytest.approx(f0, rel=1e-9)
    assert _fn(p, 1e-9, ai, aj) == pytest.approx(f0, rel=1e-6)
    assert _fn(p, 0.3, ai, aj) == _fn(p, 0.3, aj, ai)
    # repulsion only up to 20 lambda_D = 1.0, attraction up to 4 a0 = 4.0
    pr = _p()
    assert _fn(pr, 1.0 - 1e-9, ai, aj) < 0.0 and _fn(pr, 1.0, ai, aj) == 0.0
    pa = _p(f_er=0.0, hamaker=0.3)
    assert _fn(pa, 4.0 - 1e-9, ai, aj) > 0.0 and _fn(pa, 4.0, ai, aj) == 0.0
    assert oracle.echem_range(pr) == pytest.approx(1.0) and oracle.echem_range(pa) == 4.0
    assert oracle.echem_range(_p(f_er=0.0)) == 0.0


@pytest.mark.parametrize("hamaker,f_er,sign", [(0.3, 0.0, 1.0), (0.0, 2.0, -1.0)])
def test_pair_beyond_lubrication_feels_only_the_central_force(hamaker, f_er, sign):
    p = _p(f_er=f_er, hamaker=hamaker, lambda_d=0.1)
    ai, aj = 1.0, 1.4
    d = 0.5                                   # beyond delta_lub (0.06), inside both ranges
    xi = np.array([10.0, 10.0, 10.0])
    xj = xi + (ai + aj + d) * N
    z = np.zeros(3)
    u = np.array([p.shear_rate * xi[1], 0.0, 0.0])
    uj = np.array([p.shear_rate * xj[1], 0.0, 0.0])
    w = np.array([0.0, 0.0, -0.5 * p.shear_rate])
    fl, Fi, Fj, Ti, Tj, S, xn = oracle.pair_eval(p, 0.0, xi, xj, u, uj, w, w, ai, aj)
    assert fl & 1 and not fl & 2
    np.testing.assert_allclose(Fi + Fj, 0.0, atol=1e-14)
    assert np.all(Ti == 0.0) and np.all(Tj == 0.0)
    Fe = oracle.echem(p, d, ai, aj, N)
    np.testing.assert_allclose(Fi, Fe, rtol=1e-13)
    assert sign * (Fi @ N) > 0.0               # attraction pulls i toward j
    r = xj - xi
    np.testing.assert_allclose(S, np.outer(r, Fi), rtol=1e-12, atol=1e-15)
    assert sign * (N @ S @ N) > 0.0            # tension for attraction, compression for repulsion


def test_list_extends_to_the_electrochemical_range():
    ai, aj = 1.0, 1.4
    for ham, rng in ((0.3, 4.0), (0.0, 0.06)):
        p = _p(f_er=0.0, hamaker=ham)
        for d, want in ((rng - 1e-6, 1), (rng + 1e-6, 0)):
            x = np.array([[10.0, 10.0 + ai + aj + d], [10.0, 10.0], [10.0, 10.0]])
            pairs = oracle.pairs_bruteforce(x, np.array([ai, aj]), np.array([0, 1]), p, 0.0)
            assert len(pairs) == want, (ham, d)
