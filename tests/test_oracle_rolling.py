"""Pins of the oracle's rolling resistance (App. B, Eq. B1) against what the
mechanics fixes, not against its own formula.

- A periodic row of touching spheres of alternating radii a1, a2 (normal
  forces balanced, no fluid, no sliding spring) spinning about z: the
  rolling springs make the relative spin w1 - w2 oscillate at
  Omega_r = abar sqrt(2 k_r (1/I1 + 1/I2)), abar = 2 a1 a2 / (a1 + a2),
  while I1 w1 + I2 w2 stays constant (the torques of a contact are equal and
  opposite).  A wrong reduced radius, a sign that drives instead of resists,
  or torques that do not cancel all break it.
- The Coulomb limit: |k_r xi_r| never exceeds mu |F_nor| and reaches it when
  the spring is overloaded; torques are tangential and opposite.
- The rolling spring exerts no force and no stresslet; a rigid co-rotation
  (w_i = w_j) loads no rolling spring; the stretch does not depend on which
  particle of the pair is i.
"""
import math

import numpy as np
import pytest

import oracle


def _inertia(a, rho=1.0):
    return 0.4 * (4.0 / 3.0 * math.pi * rho * a ** 3) * a * a


def _ring(a1, a2, kr, dt, steps, N=8, delta=0.02):
    s = a1 + a2 - delta
    L = [N * s, 12.0, 12.0]
    x = np.zeros((3, N))
    x[0] = (np.arange(N) + 0.5) * s
    x[1] = 6.0
    x[2] = 6.0
    a = np.array([a1 if k % 2 == 0 else a2 for k in range(N)])
    p = oracle.make_params(L, kn=1e4, kt=0.0, gamma_n=0.0, mu=1e3, eta0=0.0,
                           shear_rate=0.0, dt=dt, k_r=kr)
    u = np.zeros((3, N))
    w = np.zeros((3, N))
    w[2] = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)
    sysm = oracle.System(p, x, a, u=u, w=w)
    sysm.init_accel()
    out = []
    for _ in range(steps):
        sysm.step(1)
        out.append(sysm.get_state()["w"][2, :2].copy())
    return np.array(out), sysm


@pytest.mark.parametrize("a1,a2", [(1.0, 1.0), (1.0, 1.5)])
def test_rolling_springs_make_the_relative_spin_oscillate(a1, a2):
    kr, dt = 50.0, 1e-3
    W, sysm = _ring(a1, a2, kr, dt, 3000)
    I1, I2 = _inertia(a1), _inertia(a2)
    abar = 2 * a1 * a2 / (a1 + a2)
    om = abar * math.sqrt(2 * kr * (1 / I1 + 1 / I2))
    t = np.arange(1, W.shape[0] + 1) * dt
    # closed form of the continuous dynamics; the scheme's phase error at
    # Omega_r dt ~ 0.01 over ~5 periods stays below 1e-3 of the amplitude 2
    np.testing.assert_allclose(W[:, 0] - W[:, 1], 2.0 * np.cos(om * t), atol=1e-3)
    np.testing.assert_allclose(I1 * W[:, 0] + I2 * W[:, 1], I1 - I2, atol=1e-12)
    # every contact carries a rolling stretch
    keys, xi, xr = sysm.get_history(rolling=True)
    assert len(keys) == 8 and np.abs(xr).max() > 0


def test_coulomb_limit_of_the_rolling_spring():
    rng = np.random.default_rng(3)
    p = oracle.make_params([20.0] * 3, kn=1e4, gamma_n=5.0, mu=0.4, dt=1e-3, k_r=300.0)
    hit = 0
    for _ in range(200):
        ai, aj = rng.uniform(0.5, 2.0, size=2)
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        r = (ai + aj) * (1 - rng.uniform(0.001, 0.02)) * n
        ui, uj, wi, wj = (rng.normal(size=3) for _ in range(4))
        xo = rng.normal(size=3) * rng.choice([1e-4, 1.0])
        Ti, Tj, xr = oracle.rolling(p, r, ai, aj, ui, uj, wi, wj, xo)
        d = np.linalg.norm(r) - (ai + aj)
        fnor = p.kn * d * n + p.gamma_n * n * np.dot(n, uj - ui)
        abar = 2 * ai * aj / (ai + aj)
        lim = abar * p.mu * np.linalg.norm(fnor)
        assert np.linalg.norm(Ti) <= lim * (1 + 1e-12)
        assert abs(np.dot(xr, n)) <= 1e-12 * (1 + np.linalg.norm(xr))
        assert abs(np.dot(Ti, n)) <= 1e-12 * (1 + np.linalg.norm(Ti))
        np.testing.assert_array_equal(Tj, -Ti)
        hit += np.linalg.norm(Ti) > lim * (1 - 1e-12)
    assert hit > 50          # the overloaded springs sit exactly on the limit


def test_rolling_exerts_no_force_and_ignores_co_rotation():
    rng = np.random.default_rng(5)
    box = [30.0] * 3
    base = dict(kn=1e4, mu=0.5, dt=1e-3, shear_rate=0.7)
    p0 = oracle.make_params(box, **base)
    p1 = oracle.make_params(box, k_r=800.0, **base)
    for _ in range(30):
        ai, aj = rng.uniform(0.7, 1.6, size=2)
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        xi = np.array([10.0, 12.0, 9.0])
        xj = xi + (ai + aj) * (1 - 0.01) * n
        ui, uj, wi, wj = (rng.normal(size=3) for _ in range(4))
        xo = rng.normal(size=3) * 1e-3
        ro = rng.normal(size=3) * 1e-3
        a = oracle.pair_eval(p0, 0.0, xi, xj, ui, uj, wi, wj, ai, aj, xo)
        b = oracle.pair_eval(p1, 0.0, xi, xj, ui, uj, wi, wj, ai, aj, xo, ro)
        assert a[0] == b[0] == 3
        for k in (1, 2, 5, 6):            # F_i, F_j, S, sliding stretch
            np.testing.assert_array_equal(a[k], b[k])
        assert np.abs(b[3] - a[3]).max() > 0
        # the rolling torques cancel
        np.testing.assert_allclose((b[3] - a[3]) + (b[4] - a[4]), 0.0, atol=1e-12)
        # swapping i and j: the same rolling stretch, the torques exchanged
        c0 = oracle.pair_eval(p0, 0.0, xj, xi, uj, ui, wj, wi, aj, ai, -xo)
        c = oracle.pair_eval(p1, 0.0, xj, xi, uj, ui, wj, wi, aj, ai, -xo, ro)
        np.testing.assert_allclose(c[7], b[7], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(c[3] - c0[3], b[4] - a[4], rtol=1e-9, atol=1e-12)
        # rigid co-rotation: a fresh rolling spring stays unloaded
        d = oracle.pair_eval(p1, 0.0, xi, xj, ui, uj, wi, wi, ai, aj, xo, (0, 0, 0))
        np.testing.assert_allclose(d[7], 0.0, atol=1e-15)


def test_rolling_stretch_lives_with_the_contact():
    """Two spheres pushed together, held, then pulled apart and back: the
    rolling stretch appears with the contact, is dropped with it, and starts
    again from zero (one step of u_r dt) on the next contact."""
    L = 20.0
    p = oracle.make_params([L] * 3, kn=1e4, mu=0.8, eta0=0.0, shear_rate=0.0, dt=1e-3, k_r=200.0)
    a = [1.0, 1.0]
    def run(gap, steps, xr_seed=None):
        x = np.array([[8.0, 8.0 + 2.0 + gap], [10.0, 10.0], [10.0, 10.0]])
        u = np.zeros((3, 2))
        w = np.zeros((3, 2))
        w[2] = [3.0, -1.0]
        s = oracle.System(p, x, a, u=u, w=w)
        s.init_accel()
        if xr_seed is not None:
            keys, xi = np.array([1], dtype=np.int64), np.zeros((1, 3))
            s.set_history(keys, xi, xr_seed)
        s.step(steps)
        return s
    s = run(-0.01, 5)
    keys, xi, xr = s.get_history(rolling=True)
    assert list(keys) == [1] and np.abs(xr).max() > 0
    # separated pair: no entry, whatever stretch it carried before
    s = run(+0.05, 1, xr_seed=np.array([[0.0, 0.3, 0.0]]))
    keys, xi, xr = s.get_history(rolling=True)
    assert len(keys) == 0
    # a fresh contact starts from zero: one step adds abar (n x (w_i - w_j)) dt
    s = run(-0.01, 1)
    keys, xi, xr = s.get_history(rolling=True)
    wrel = 4.0                                     # w_i - w_j about z, at the half step
    assert abs(np.linalg.norm(xr[0]) - 1.0 * wrel * p.dt) < 1e-2 * wrel * p.dt
