"""Pins of the oracle's wavy shear flow (Eq. 17) with the Faxen term of the
Stokes drag (Eq. A1), against what the flow and the mechanics fix.

- Faxen's first law is the mean of the ambient flow over the sphere's
  surface; for U_inf,x = gdot y + U sin(k y) that mean is
  gdot y + U sin(k y) sin(k a)/(k a), which the truncated law
  (1 + a^2/6 Laplacian) matches up to U (k a)^4 / 120.  A free sphere's drag
  vanishes there (a wrong factor or sign of the Laplacian leaves
  U (k a)^2 / 6), and a free sphere relaxes to that velocity and to the spin
  -1/2 dU_inf,x/dy of the local vorticity (central differences of Eq. 17).
- A pair in the wavy flow equals a pair in a simple shear whose rate is the
  mean of the two centres' local rates, with the same velocities relative to
  the flow: exactly for a pair at one height (contact included), and for
  the lubrication of a pair at two heights.
- The particles' stresslets take the local strain: a sphere on a crest of
  the wave adds the stress of a simple shear at the crest's rate; spheres
  evenly spread over a period add that of the mean rate.
- The wave is L_y-periodic, so a sphere crossing y = L_y keeps its velocity
  relative to the flow and its drag.
- No wave (U = 0 or n = 0) is the simple shear, bit for bit.
"""
import math

import numpy as np
import pytest

import oracle


def _ux(gd, U, k, y):
    """Eq. 17, x component."""
    return gd * y + U * math.sin(k * y)


def _surface_mean_ux(gd, U, k, y, a, nq=24):
    """Mean of U_inf,x over the sphere of radius a centred at height y
    (Gauss-Legendre in cos(theta); the flow depends on y only)."""
    mu, wq = np.polynomial.legendre.leggauss(nq)
    return 0.5 * sum(w * _ux(gd, U, k, y + a * m) for m, w in zip(mu, wq))


def _rate_fd(gd, U, k, y, h=1e-5):
    return (_ux(gd, U, k, y + h) - _ux(gd, U, k, y - h)) / (2 * h)


def _one(p, x, a, u, w):
    s = oracle.System(p, np.array(x, float).reshape(3, 1), [a],
                      u=np.array(u, float).reshape(3, 1), w=np.array(w, float).reshape(3, 1))
    F, T, S = s.forces()
    return F[:, 0], T[:, 0], S


@pytest.mark.parametrize("y,a", [(3.1, 1.0), (11.7, 1.4), (17.0, 0.6)])
def test_faxen_drag_vanishes_at_the_surface_mean_velocity(y, a):
    L, gd, U, nw, eta0 = 24.0, 0.8, 5.0, 1, 1.3
    k = 2 * math.pi * nw / L
    p = oracle.make_params([L] * 3, shear_rate=gd, eta0=eta0, wave_amp=U, wave_n=nw)
    us = _surface_mean_ux(gd, U, k, y, a)
    wz = -0.5 * _rate_fd(gd, U, k, y)
    F, T, _ = _one(p, [5.0, y, 7.0], a, [us, 0, 0], [0, 0, wz])
    scale = 6 * math.pi * eta0 * a * U
    assert abs(F[0]) <= scale * (k * a) ** 4 / 100
    assert abs(F[1]) == 0 and abs(F[2]) == 0
    assert np.abs(T).max() <= 8 * math.pi * eta0 * a ** 3 * 1e-8 * (1 + U * k)
    # the drag at the centre's flow velocity is the Faxen term itself
    F0, _, _ = _one(p, [5.0, y, 7.0], a, [_ux(gd, U, k, y), 0, 0], [0, 0, wz])
    want = -scale * (k * a) ** 2 / 6 * math.sin(k * y)
    assert F0[0] == pytest.approx(want, rel=(k * a) ** 2 / 10)
    assert abs(F0[0]) > 1e-3 * scale


def test_free_sphere_relaxes_to_the_faxen_velocity_and_local_spin():
    L, gd, U, nw = 30.0, 0.5, 4.0, 2
    k = 2 * math.pi * nw / L
    a, y = 1.2, 9.3
    p = oracle.make_params([L] * 3, shear_rate=gd, eta0=1.0, rho=1.0, dt=5e-3,
                           wave_amp=U, wave_n=nw)
    s = oracle.System(p, np.array([[4.0], [y], [6.0]]), [a], u=np.zeros((3, 1)),
                      w=np.zeros((3, 1)))
    s.init_accel()
    s.step(3000)          # ~50 translational relaxation times
    st = s.get_state()
    assert st["x"][1, 0] == y
    assert st["u"][0, 0] == pytest.approx(_surface_mean_ux(gd, U, k, y, a),
                                          abs=U * (k * a) ** 4 / 100)
    assert st["w"][2, 0] == pytest.approx(-0.5 * _rate_fd(gd, U, k, y), rel=1e-8)


def _shifted(p_wave, gd_mean, y, u, w):
    """Velocities of the same motion relative to the flow in a simple shear
    of rate gd_mean."""
    V = u[0] - oracle.flow_ux(p_wave, y)
    Wz = w[2] + 0.5 * oracle.flow_rate(p_wave, y)
    return [V + gd_mean * y, u[1], u[2]], [w[0], w[1], Wz - 0.5 * gd_mean]


@pytest.mark.parametrize("case", ["same_height_contact", "two_heights_lubrication"])
def test_pair_equals_a_simple_shear_pair_at_the_mean_rate(case):
    rng = np.random.default_rng(11)
    L, gd, U, nw = 26.0, 1.1, 6.0, 1
    box = [L] * 3
    pw = oracle.make_params(box, shear_rate=gd, wave_amp=U, wave_n=nw, mu=0.6,
                            delta_lub=0.2, dt=1e-3)
    ai, aj = 1.0, 1.7
    xi = np.array([8.0, 10.4, 12.0])
    if case == "same_height_contact":
        n = np.array([0.6, 0.0, 0.8])
        gap = -0.01
    else:
        n = np.array([0.3, 0.8, -0.52])
        n /= np.linalg.norm(n)
        gap = 0.04
    xj = xi + (ai + aj + gap) * n
    ui, uj, wi, wj = (rng.normal(size=3) for _ in range(4))
    xo = np.array([1e-3, -2e-3, 5e-4])
    xo -= n * np.dot(n, xo)
    got = oracle.pair_eval(pw, 0.0, xi, xj, ui, uj, wi, wj, ai, aj, xo)
    gm = 0.5 * (oracle.flow_rate(pw, xi[1]) + oracle.flow_rate(pw, xj[1]))
    ps = oracle.make_params(box, shear_rate=gm, mu=0.6, delta_lub=0.2, dt=1e-3,
                            gamma_n=pw.gamma_n)
    ui2, wi2 = _shifted(pw, gm, xi[1], ui, wi)
    uj2, wj2 = _shifted(pw, gm, xj[1], uj, wj)
    want = oracle.pair_eval(ps, 0.0, xi, xj, ui2, uj2, wi2, wj2, ai, aj, xo)
    assert got[0] == want[0] == (3 if gap < 0 else 1)
    for q in range(1, 7):
        np.testing.assert_allclose(got[q], want[q], rtol=1e-11, atol=1e-11 * np.abs(want[q]).max())
    # the local rates at the two heights really differ in the second case
    if case == "two_heights_lubrication":
        assert abs(oracle.flow_rate(pw, xi[1]) - oracle.flow_rate(pw, xj[1])) > 0.1


def test_particle_stresslets_take_the_local_strain():
    L, gd, U, nw, eta0, a = 40.0, 0.7, 3.0, 2, 1.2, 1.0
    k = 2 * math.pi * nw / L
    pw = oracle.make_params([L] * 3, shear_rate=gd, eta0=eta0, wave_amp=U, wave_n=nw)
    # a crest of the rate: k y = 2 pi
    y = L / nw
    _, _, Sw = _one(pw, [10.0, y, 10.0], a, [oracle.flow_ux(pw, y), 0, 0],
                    [0, 0, -0.5 * oracle.flow_rate(pw, y)])
    gc = gd + U * k
    ps = oracle.make_params([L] * 3, shear_rate=gc, eta0=eta0)
    _, _, Ss = _one(ps, [10.0, y, 10.0], a, [gc * y, 0, 0], [0, 0, -0.5 * gc])
    assert Sw[0, 1] - eta0 * gd == pytest.approx(Ss[0, 1] - eta0 * gc, rel=1e-12)
    # eight dilute spheres evenly over one period: the wave averages out
    m = 8
    ys = (np.arange(m) + 0.25) * (L / nw) / m
    x = np.stack([np.linspace(3, 35, m), ys, np.full(m, 20.0)])
    s = oracle.System(pw, x, np.full(m, a))
    _, _, S8 = s.forces()
    p0 = oracle.make_params([L] * 3, shear_rate=gd, eta0=eta0)
    s0 = oracle.System(p0, x, np.full(m, a))
    _, _, S0 = s0.forces()
    assert S8[0, 1] == pytest.approx(S0[0, 1], rel=1e-13)


@pytest.mark.parametrize("vy", [+4.0, -4.0])
def test_crossing_y_boundary_keeps_the_relative_velocity(vy):
    L, gd, U, nw = 20.0, 0.9, 3.0, 1
    p = oracle.make_params([L] * 3, shear_rate=gd, wave_amp=U, wave_n=nw, dt=1e-3,
                           eta0=1.0, rho=50.0)
    y0 = L - 0.01 if vy > 0 else 0.01
    u0 = oracle.faxen_ux(p, y0, 1.0)
    s = oracle.System(p, np.array([[5.0], [y0], [5.0]]), [1.0],
                      u=np.array([[u0], [vy], [0.0]]), w=np.zeros((3, 1)))
    s.init_accel()
    rel = []
    for _ in range(6):
        s.step(1)
        st = s.get_state()
        rel.append(st["u"][0, 0] - oracle.faxen_ux(p, st["x"][1, 0], 1.0))
    assert s.get_images()[0] == (1 if vy > 0 else -1)
    # smooth through the wrap: the relative velocity changes by O(dt) per step
    assert np.abs(np.diff(rel)).max() < 1e-2


def test_no_wave_is_the_simple_shear_bit_for_bit():
    rng = np.random.default_rng(2)
    L = 14.0
    pts = []
    while len(pts) < 40:
        q = rng.uniform(0, L, size=3)
        if all(np.linalg.norm(q - r) > 2.05 for r in pts):
            pts.append(q)
    x = np.array(pts).T
    a = np.ones(40)
    res = []
    for kw in (dict(), dict(wave_amp=5.0, wave_n=0), dict(wave_amp=0.0, wave_n=3)):
        p = oracle.make_params([L] * 3, shear_rate=2.0, dt=2e-3, delta_lub=0.3, **kw)
        s = oracle.System(p, x, a)
        s.init_accel()
        s.step(20)
        st = s.get_state()
        res.append(np.concatenate([st[q].ravel() for q in ("x", "u", "w")]))
    np.testing.assert_array_equal(res[0], res[1])
    np.testing.assert_array_equal(res[0], res[2])
