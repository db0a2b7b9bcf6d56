"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every expected value comes from
a closed form, a textbook limit (tests/golden), an explicit-image brute force
written differently from the oracle's minimum-image arithmetic, or an
invariant that a dropped term, a wrong sign or a transposed block breaks.
"""
import json
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def unit(v):
    v = np.asarray(v, dtype=float)
    return v / np.linalg.norm(v)


# --------------------------------------------------------------------------
# Neighbour set (Sec. II A, fixed-radius near neighbours; Eq. 16 images)
# --------------------------------------------------------------------------

def _explicit_image_pairs(x, a, ids, box, off, delta, mode=0, a0=1.0):
    """Pairs by enumerating explicit periodic / Lees-Edwards images."""
    n = a.shape[0]
    Lx, Ly, Lz = box
    out = []
    for i in range(n):
        for j in range(i + 1, n):
            best = np.inf
            for ky in (-1, 0, 1):
                for kx in (-2, -1, 0, 1, 2):
                    for kz in (-1, 0, 1):
                        xj = x[0, j] + kx * Lx + ky * off
                        yj = x[1, j] + ky * Ly
                        zj = x[2, j] + kz * Lz
                        d2 = (xj - x[0, i]) ** 2 + (yj - x[1, i]) ** 2 + (zj - x[2, i]) ** 2
                        best = min(best, d2)
            dij = delta * a0 if mode == 1 else delta * (a[i] + a[j]) / 2
            if best < (a[i] + a[j] + dij) ** 2:
                out.append((min(ids[i], ids[j]), max(ids[i], ids[j])))
    return np.array(sorted(out), dtype=np.int64).reshape(-1, 2)


def test_pairs_hand_placed(orc):
    box = [20.0, 20.0, 20.0]
    p = orc.make_params(box, shear_rate=1.0, dt=0.01)
    nstep = 137
    off = orc.le_offset(p, nstep)
    assert off == pytest.approx(math.fmod(1.0 * 20.0 * nstep * 0.01, 20.0))
    pts = [
        (5.0, 5.0, 5.0),          # 0
        (7.04, 5.0, 5.0),         # 1: 2.04 from 0, inside 2.05
        (5.0, 7.06, 5.0),         # 2: 2.06 from 0, outside
        (0.5, 10.0, 10.0),        # 3
        (19.0, 10.0, 10.0),       # 4: 1.5 from 3 through x wrap
        (12.0, 12.0, 0.4),        # 5
        (12.0, 12.0, 19.1),       # 6: 1.3 from 5 through z wrap
        (3.0, 19.5, 15.0),        # 7: near the top
        (math.fmod(3.3 - off + 40.0, 20.0), 0.5, 15.0),  # 8: image above at x+off
        (3.3, 0.5, 15.0),         # 9: no offset compensation -> not a pair of 7
    ]
    x = np.array(pts).T.copy()
    a = np.ones(len(pts))
    ids = np.arange(len(pts), dtype=np.int32)
    got = orc.pairs_bruteforce(x, a, ids, p, off)
    exp = {(0, 1), (3, 4), (5, 6), (7, 8)}
    # 8 and 9 are both near y=0.5 with x differing by off; they pair only if close
    d89 = abs(((x[0, 8] - x[0, 9]) + 10.0) % 20.0 - 10.0)
    if d89 < 2.05:
        exp.add((8, 9))
    assert {tuple(r) for r in got.tolist()} == exp


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_pairs_match_explicit_images(orc, seed, mode):
    rng = np.random.default_rng(seed)
    n = 70
    box = np.array([13.0, 11.0, 12.0])
    x = rng.uniform(0, 1, size=(3, n)) * box[:, None]
    a = rng.choice([1.0, 1.4], size=n)
    ids = rng.permutation(n).astype(np.int32)
    p = orc.make_params(box, shear_rate=0.7, dt=0.013, delta_lub=0.3, lub_cutoff_mode=mode)
    off = orc.le_offset(p, 1000 + seed * 77)
    assert 0.0 <= off < box[0]
    got = orc.pairs_bruteforce(x, a, ids, p, off)
    exp = _explicit_image_pairs(x, a, ids, box, off, 0.3, mode)
    assert len(exp) > 10
    np.testing.assert_array_equal(got, exp)
    # every row query agrees with the pair set
    for k in range(0, n, 7):
        nb = orc.neighbours_of(x, a, ids, p, off, k)
        want = sorted([hi if lo == ids[k] else lo for lo, hi in exp.tolist() if ids[k] in (lo, hi)])
        assert nb.tolist() == want


# --------------------------------------------------------------------------
# Contact: Eq. 4 (spring-dashpot) and Eq. 5 (tangential spring, Coulomb cap)
# --------------------------------------------------------------------------

def test_head_on_collision_restitution(orc):
    """Two spheres, no fluid: damped-oscillator contact, exact restitution."""
    kn, gn, a = 1e4, 20.0, 1.0
    box = [40.0, 40.0, 40.0]
    p = orc.make_params(box, kn=kn, gamma_n=gn, mu=0.0, eta0=0.0, shear_rate=0.0, dt=2e-5)
    v0 = 1.0
    x = np.array([[19.0 - 1e-3, 21.0 + 1e-3], [20.0, 20.0], [20.0, 20.0]])
    u = np.array([[0.5 * v0, -0.5 * v0], [0.0, 0.0], [0.0, 0.0]])
    s = orc.System(p, x, [a, a], u=u, w=np.zeros((3, 2)))
    s.init_accel()
    m = 4.0 / 3.0 * math.pi * a ** 3
    ms = m / 2.0
    t_contact = None
    in_contact = False
    for k in range(20000):
        s.step(1)
        st = s.get_state()
        gap = st["x"][0, 1] - st["x"][0, 0] - 2 * a
        if gap < 0 and not in_contact:
            in_contact, t0 = True, k
        if in_contact and gap >= 0:
            t_contact = (k - t0) * p.dt
            break
    assert t_contact is not None
    vout = st["u"][0, 1] - st["u"][0, 0]
    zeta = gn / (2.0 * math.sqrt(kn * ms))
    wd = math.sqrt(kn / ms) * math.sqrt(1 - zeta ** 2)
    e = math.exp(-zeta * math.pi / math.sqrt(1 - zeta ** 2))
    assert vout / v0 == pytest.approx(e, rel=2e-3)
    assert t_contact == pytest.approx(math.pi / wd, rel=2e-3)


def test_tangential_spring_loads_then_slides(orc):
    """Constant sliding: xi grows as u_t t, then stays at mu|F_nor|/k_t."""
    kn, kt, mu, dt = 1e4, 5e3, 0.5, 1e-3
    p = orc.make_params([50] * 3, kn=kn, kt=kt, gamma_n=3.0, mu=mu, dt=dt)
    ai, aj, ov, v = 1.0, 1.4, 0.01, 0.2
    n = np.array([0.0, 1.0, 0.0])
    r = n * (ai + aj - ov)
    ui, uj = np.zeros(3), np.array([v, 0.0, 0.0])
    cap = mu * kn * ov / kt
    xi = np.zeros(3)
    for k in range(1, 200):
        F, Ti, Tj, xi = orc.contact(p, r, ai, aj, ui, uj, np.zeros(3), np.zeros(3), xi)
        want = min(k * v * dt, cap)
        assert xi[0] == pytest.approx(want, rel=1e-12)
        assert abs(xi[1]) < 1e-15 and abs(xi[2]) < 1e-15
        # normal: k_n d n with d = -ov pushes i away from j (-y)
        assert F[1] == pytest.approx(-kn * ov, rel=1e-12)
        # friction drags i along with j's motion (+x)
        assert F[0] == pytest.approx(kt * want, rel=1e-12)
        # lever arms: force +f x at i's contact point (+a_i y), -f x at j's (-a_j y)
        lever_i = np.cross(ai * n, np.array([F[0], 0, 0]))
        lever_j = np.cross(-aj * n, np.array([-F[0], 0, 0]))
        np.testing.assert_allclose(Ti, lever_i, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(Tj, lever_j, rtol=1e-12, atol=1e-14)
    assert xi[0] == pytest.approx(cap, rel=1e-12)


def test_rolling_contact_has_no_slip(orc):
    """Contact points moving together (rolling without slip): u_t = 0."""
    p = orc.make_params([50] * 3, mu=1.0)
    rng = np.random.default_rng(4)
    for _ in range(20):
        ai, aj = rng.uniform(0.5, 3, size=2)
        n = unit(rng.normal(size=3))
        r = n * (ai + aj - 1e-3)
        wi, wj = rng.normal(size=3), rng.normal(size=3)
        c = rng.normal(size=3)             # common contact-point velocity
        ui = c - np.cross(wi, ai * n)      # u_i + w_i x (a_i n) = c
        uj = c - np.cross(wj, -aj * n)     # u_j + w_j x (-a_j n) = c
        F, Ti, Tj, xi = orc.contact(p, r, ai, aj, ui, uj, wi, wj, np.zeros(3))
        assert np.linalg.norm(xi) < 1e-14
        assert np.linalg.norm(Ti) < 1e-10


def test_old_stretch_is_projected_on_tangent_plane(orc):
    p = orc.make_params([50] * 3, mu=10.0)
    n = unit([1.0, 2.0, -0.5])
    r = n * 1.99
    old = np.array([1e-4, -2e-4, 3e-4])
    F, Ti, Tj, xi = orc.contact(p, r, 1.0, 1.0, np.zeros(3), np.zeros(3), np.zeros(3),
                                np.zeros(3), old)
    np.testing.assert_allclose(xi, old - n * (n @ old), rtol=1e-12, atol=1e-18)


# --------------------------------------------------------------------------
# Lubrication: App. A (Eq. A2, A3, A6, A7) with the 6 pi eta0 prefactor
# --------------------------------------------------------------------------

def _lub(orc, p, r, ai, aj, ui, uj, wi, wj, xi=(0.0, 0.0, 0.0)):
    """Lubrication from absolute velocities at absolute position xi, xi + r."""
    gd = p.shear_rate
    Om = np.array([0.0, 0.0, -0.5 * gd])
    xi = np.asarray(xi, float)
    xj = xi + r
    Vi = np.asarray(ui) - np.array([gd * xi[1], 0, 0])
    Vj = np.asarray(uj) - np.array([gd * xj[1], 0, 0])
    return orc.lubrication(p, r, ai, aj, Vi, Vj, np.asarray(wi) - Om, np.asarray(wj) - Om)


@pytest.mark.parametrize("alpha", [1.0, 1.4, 3.0, 10.0])
def test_squeeze_force_matches_reynolds(orc, alpha):
    """Normal approach: F h -> 6 pi eta a_eff^2 V, a_eff = a_i a_j/(a_i + a_j)."""
    ai, aj = 1.0, alpha
    p = orc.make_params([100] * 3, shear_rate=0.0, lub_eps=0.0, eta0=1.3)
    n = unit([0.3, -1.0, 0.2])
    aeff = ai * aj / (ai + aj)
    for h in (1e-3, 1e-4, 1e-5):
        r = n * (ai + aj + h)
        V = 0.7
        Fi, Fj, Ti, Tj = _lub(orc, p, r, ai, aj, V * n, np.zeros(3), np.zeros(3), np.zeros(3))
        want = 6 * math.pi * 1.3 * aeff ** 2 * V / h
        # the gap is |r| - (a_i + a_j): rounding of |r| limits the relative accuracy
        assert -(Fi @ n) == pytest.approx(want, rel=max(1e-12, 1e-14 * (ai + aj) / h))
        np.testing.assert_allclose(Fi + Fj, 0.0, atol=1e-9 * want)
    # the regulariser: F = 6 pi eta a_eff^2 V / (h + eps (a_i + a_j)/2)
    p2 = orc.make_params([100] * 3, shear_rate=0.0, lub_eps=1e-3)
    h = 2e-3
    Fi, *_ = _lub(orc, p2, n * (ai + aj + h), ai, aj, n, np.zeros(3), np.zeros(3), np.zeros(3))
    assert -(Fi @ n) == pytest.approx(6 * math.pi * aeff ** 2 / (h + 1e-3 * (ai + aj) / 2), rel=1e-12)


def test_sphere_wall_limit_matches_textbook(orc):
    """alpha -> infinity reproduces the sphere-wall asymptotics (golden)."""
    g = json.load(open(os.path.join(GOLDEN, "sphere_wall_limits.json")))
    ai, aj = 1.0, 1e7
    p = orc.make_params([1e9] * 3, shear_rate=0.0, lub_eps=0.0)
    n = np.array([0.0, 1.0, 0.0])
    h = 1e-3
    r = n * (ai + aj + h)
    dstar = 2 * h / (ai + aj)
    logf = math.log(1.0 / dstar)
    k = 6 * math.pi
    z = np.zeros(3)
    Fi, _, Ti, _ = _lub(orc, p, r, ai, aj, np.array([0, 1.0, 0]), z, z, z)
    assert -Fi[1] * h / k == pytest.approx(g["normal_Fh_over_6pi_eta_a2_V"], rel=1e-5)
    Fi, _, Ti, _ = _lub(orc, p, r, ai, aj, np.array([1.0, 0, 0]), z, z, z)
    assert -Fi[0] / (k * logf) == pytest.approx(g["tangential_translation_log_coefficient"], rel=1e-5)
    Fi, _, Ti, _ = _lub(orc, p, r, ai, aj, z, z, np.array([0, 0, 1.0]), z)
    assert abs(Fi[0]) / (k * logf) == pytest.approx(g["rotation_coupling_log_coefficient"], rel=1e-5)
    assert -Ti[2] / (8 * math.pi * logf) == pytest.approx(g["rotation_torque_log_coefficient_8pi"], rel=1e-5)
    # sign: a sphere spinning next to a wall is pushed opposite to its
    # surface velocity in the gap (surface moves along w x (a n))
    surf = np.cross(np.array([0, 0, 1.0]), ai * n)
    assert Fi @ surf < 0


@pytest.mark.parametrize("seed", range(4))
def test_rigid_motion_of_pair_is_free(orc, seed):
    """No lubrication for rigid-body translation/rotation of the pair."""
    rng = np.random.default_rng(seed)
    p = orc.make_params([100] * 3, shear_rate=0.0)
    for _ in range(10):
        ai, aj = rng.uniform(0.5, 10, size=2)
        n = unit(rng.normal(size=3))
        h = 1e-10
        xi = rng.uniform(10, 20, size=3)
        r = n * (ai + aj + h)
        xj = xi + r
        scale = np.linalg.norm(_lub(orc, p, r, ai, aj, n, np.zeros(3), np.zeros(3), np.zeros(3))[0])
        U = rng.normal(size=3)
        out = _lub(orc, p, r, ai, aj, U, U, np.zeros(3), np.zeros(3), xi)
        assert max(np.linalg.norm(v) for v in out) < 1e-12 * scale
        W = rng.normal(size=3)
        c = xi + ai * n
        out = _lub(orc, p, r, ai, aj, np.cross(W, xi - c), np.cross(W, xj - c), W, W, xi)
        assert max(np.linalg.norm(v) for v in out) < 1e-8 * scale


@pytest.mark.parametrize("seed", range(4))
def test_particles_at_rest_in_shear_feel_no_lubrication(orc, seed):
    """u = 0, w = 0 in simple shear: no relative surface motion in the gap, so
    the strain terms R'(E) cancel the U_inf / Omega_inf terms (forces and
    torques), which pins X^G, Y^G, Y^H and n_perp against the A, B, C blocks."""
    rng = np.random.default_rng(100 + seed)
    p = orc.make_params([100] * 3, shear_rate=1.7)
    for _ in range(10):
        ai, aj = rng.uniform(0.5, 10, size=2)
        n = unit(rng.normal(size=3))
        xi = rng.uniform(10, 20, size=3)
        r = n * (ai + aj + 1e-10)
        scale = np.linalg.norm(_lub(orc, p, r, ai, aj, n, np.zeros(3), np.zeros(3),
                                    np.array([0, 0, -0.85]), xi)[0])
        out = _lub(orc, p, r, ai, aj, np.zeros(3), np.zeros(3), np.zeros(3), np.zeros(3), xi)
        assert max(np.linalg.norm(v) for v in out) < 1e-8 * scale


def test_lubrication_antisymmetric_swap_and_dissipative(orc):
    rng = np.random.default_rng(7)
    p = orc.make_params([100] * 3, shear_rate=0.0)
    pe = orc.make_params([100] * 3, shear_rate=1.0)
    for _ in range(300):
        ai, aj = rng.uniform(1, 10, size=2)
        n = unit(rng.normal(size=3))
        ds = rng.uniform(-0.01, 0.05)
        r = n * (ai + aj) * (1 + ds / 2)
        V = rng.normal(size=(4, 3))
        Fi, Fj, Ti, Tj = orc.lubrication(p, r, ai, aj, *V)
        s = np.linalg.norm(Fi)
        np.testing.assert_allclose(Fi + Fj, 0.0, atol=1e-12 * s)
        # dissipation: resistance is positive semi-definite
        P = Fi @ V[0] + Fj @ V[1] + Ti @ V[2] + Tj @ V[3]
        assert P <= 1e-12 * s * np.abs(V).max()
        # relabelling i <-> j gives the same physical forces (incl. strain terms)
        for pp in (p, pe):
            a1 = orc.lubrication(pp, r, ai, aj, *V)
            b1 = orc.lubrication(pp, -r, aj, ai, V[1], V[0], V[3], V[2])
            sc = max(np.linalg.norm(v) for v in a1)
            for u_, v_ in zip(a1, (b1[1], b1[0], b1[3], b1[2])):
                np.testing.assert_allclose(u_, v_, atol=1e-11 * sc)


def _lub_resistance(orc, p, r, ai, aj):
    """The 12x12 matrix R with (F_i, F_j, T_i, T_j) = -R (U_i, U_j, W_i, W_j)
    at rest in a quiescent fluid, column by column from unit motions."""
    R = np.zeros((12, 12))
    for k in range(12):
        V = np.zeros(12)
        V[k] = 1.0
        out = orc.lubrication(p, r, ai, aj, V[0:3], V[3:6], V[6:9], V[9:12])
        R[:, k] = -np.concatenate(out)
    return R


@pytest.mark.parametrize("ratio", [1.0, 1.4, 3.0, 10.0, 0.37])
def test_lubrication_resistance_is_reciprocal(orc, ratio):
    """Lorentz reciprocal theorem: the resistance matrix of the pair (forces
    and torques on both spheres against both spheres' velocities and
    angular velocities) is symmetric, and positive semi-definite.  Symmetry
    ties each cross coefficient of App. A between i and j (X^A, Y^A, Y^B,
    Y^C) at size ratio alpha to the same formula at 1/alpha, so a wrong power
    of alpha, a dropped term, a sign or an exchanged argument in one of them
    breaks it at the intermediate ratios where the paper prints no value."""
    rng = np.random.default_rng(int(ratio * 100))
    p = orc.make_params([100] * 3, shear_rate=0.0)
    for _ in range(6):
        ai = rng.uniform(0.5, 3.0)
        aj = ratio * ai
        n = unit(rng.normal(size=3))
        ds = rng.uniform(1e-4, 0.04)          # normalised gap inside the cutoff
        r = n * (ai + aj) * (1 + ds / 2)
        R = _lub_resistance(orc, p, r, ai, aj)
        scale = np.abs(R).max()
        np.testing.assert_allclose(R, R.T, rtol=0, atol=1e-12 * scale)
        assert np.linalg.eigvalsh(0.5 * (R + R.T)).min() >= -1e-12 * scale


def test_overlap_clamps_gap(orc):
    p = orc.make_params([100] * 3, shear_rate=0.0)
    n = unit([1, 1, 0])
    F0 = orc.lubrication(p, n * 2.0, 1.0, 1.0, n, np.zeros(3), np.zeros(3), np.zeros(3))[0]
    F1 = orc.lubrication(p, n * 1.99, 1.0, 1.0, n, np.zeros(3), np.zeros(3), np.zeros(3))[0]
    np.testing.assert_allclose(F0, F1, rtol=1e-14)
    assert -(F0 @ n) == pytest.approx(6 * math.pi * 0.25 / 1e-3, rel=1e-12)


# --------------------------------------------------------------------------
# One-body terms, Verlet (Eq. 15), Lees-Edwards (Eq. 16), stress (Eq. 8, 9)
# --------------------------------------------------------------------------

def test_stokes_relaxation_discrete_closed_form(orc):
    """Isolated sphere under drag alpha = -k v (k = 6 pi eta a / m for
    translation, 8 pi eta a^3 / I for rotation).  Eq. 15 evaluates alpha at
    u^{n+1/2}, so the half-step velocity decays by (1 - k dt) per step and
    v_N = v_0 (1 - k dt/2)^2 (1 - k dt)^(N-1) exactly; the spin relaxes to
    Omega_inf = -gdot/2 z."""
    a, eta, rho, dt, gd = 1.3, 0.9, 2.0, 1e-3, 1.5
    p = orc.make_params([30] * 3, eta0=eta, rho=rho, dt=dt, shear_rate=gd)
    x = np.array([[10.0], [12.0], [14.0]])
    v0, w0 = 0.8, np.array([0.3, -0.2, 0.5])
    u = np.array([[gd * 12.0], [0.0], [v0]])
    w = (np.array([0, 0, -gd / 2]) + w0).reshape(3, 1)
    s = orc.System(p, x, [a], u=u, w=w)
    s.init_accel()
    m = 4 / 3 * math.pi * rho * a ** 3
    kt = 6 * math.pi * eta * a / m
    kr = 8 * math.pi * eta * a ** 3 / (0.4 * m * a * a)
    nst = 300
    s.step(nst)
    st = s.get_state()
    decay = lambda k: (1 - k * dt / 2) ** 2 * (1 - k * dt) ** (nst - 1)
    assert st["u"][2, 0] == pytest.approx(v0 * decay(kt), rel=1e-12)
    assert st["u"][0, 0] == pytest.approx(gd * 12.0, rel=1e-14)
    want_w = np.array([0, 0, -gd / 2]) + w0 * decay(kr)
    np.testing.assert_allclose(st["w"][:, 0], want_w, rtol=1e-12)


def test_lees_edwards_crossing_keeps_the_affine_frame(orc):
    """A particle crossing y = L_y re-enters at the bottom shifted by -off in x
    with u_x reduced by gdot L_y: its velocity relative to U_inf is unchanged."""
    L, gd, dt = 20.0, 2.0, 1e-3
    p = orc.make_params([L] * 3, shear_rate=gd, dt=dt, eta0=1e-9)
    y0, vy = L - 0.0005, 1.0
    x = np.array([[5.0], [y0], [5.0]])
    u = np.array([[gd * y0 + 0.1], [vy], [0.0]])
    s = orc.System(p, x, [1.0], u=u, w=np.array([[0.0], [0.0], [-gd / 2]]), nstep=500)
    s.init_accel()
    s.step(1)
    st = s.get_state()
    off = orc.le_offset(p, 501)
    ynew = y0 + dt * vy
    assert st["x"][1, 0] == pytest.approx(ynew - L, abs=1e-12)
    want_x = (5.0 + dt * (gd * y0 + 0.1) - off) % L
    assert st["x"][0, 0] == pytest.approx(want_x, abs=1e-12)
    # u_x relative to U_inf at the new height, identical to an unwrapped move
    assert st["u"][0, 0] - gd * st["x"][1, 0] == pytest.approx(0.1 - gd * dt * vy, abs=1e-9)


def test_pair_across_lees_edwards_boundary_matches_interior_pair(orc):
    """The same relative configuration and relative motion gives the same pair
    forces whether it straddles y = L_y (image shifted by off, moving at
    gdot L_y) or sits in the middle of the box."""
    L, gd = 20.0, 1.3
    p = orc.make_params([L] * 3, shear_rate=gd, mu=0.7)
    nstep = 1234
    off = orc.le_offset(p, nstep)
    rng = np.random.default_rng(11)
    ai, aj = 1.0, 1.4
    n = unit([0.4, 1.0, -0.3])
    r = n * (ai + aj - 0.003)
    vi, vj = rng.normal(size=3), rng.normal(size=3)     # fluctuation velocities
    wi, wj = rng.normal(size=3), rng.normal(size=3)
    xo = np.array([0.7, 0.0, 0.0])
    # interior
    xi = np.array([7.0, 9.0, 5.0])
    xj = xi + r
    Ui = vi + np.array([gd * xi[1], 0, 0])
    Uj = vj + np.array([gd * xj[1], 0, 0])
    A = orc.pair_eval(p, off, xi, xj, Ui, Uj, wi, wj, ai, aj, xo)
    # straddling: i near the top, j's stored copy at the bottom
    xi2 = np.array([7.0, L - 0.5, 5.0])
    xj_img = xi2 + r                                   # above the box
    xj2 = np.array([(xj_img[0] - off) % L, xj_img[1] - L, xj_img[2]])
    Ui2 = vi + np.array([gd * xi2[1], 0, 0])
    Uj2 = vj + np.array([gd * xj2[1], 0, 0])           # stored (primary-box) velocity
    B = orc.pair_eval(p, off, xi2, xj2, Ui2, Uj2, wi, wj, ai, aj, xo)
    assert A[0] == B[0] == 3
    for u_, v_ in zip(A[1:], B[1:]):
        np.testing.assert_allclose(u_, v_, rtol=1e-9, atol=1e-9 * np.abs(A[1]).max())


def _dense(n, phi, seed):
    from paper_2108_01013_gb300 import synth
    return synth.small(n, phi, seed)


def test_relabelling_and_history_orientation(orc):
    """Permuting the array order and the ids leaves a frictional trajectory
    unchanged (per particle), which pins the lo->hi history orientation."""
    g = _dense(150, 0.50, 3)
    box = g["box"]
    p = orc.make_params(box, mu=0.8, dt=1e-4, shear_rate=50.0)
    n = g["a"].shape[0]
    s1 = orc.System(p, g["x"], g["a"], ids=np.arange(n, dtype=np.int32))
    perm = np.random.default_rng(5).permutation(n)
    ids2 = (n - 1 - np.arange(n)).astype(np.int32)          # reversed ids
    s2 = orc.System(p, g["x"][:, perm], g["a"][perm], ids=ids2[perm])
    for s in (s1, s2):
        s.init_accel()
        s.step(60)
    assert s1.ncontacts > 5
    st1, st2 = s1.get_state(), s2.get_state()
    np.testing.assert_allclose(st2["x"], st1["x"][:, perm], rtol=0, atol=1e-10)
    np.testing.assert_allclose(st2["w"], st1["w"][:, perm], rtol=0, atol=1e-9 * np.abs(st1["w"]).max())
    k1, x1 = s1.get_history()
    k2, x2 = s2.get_history()
    # same contacts (ids mapped), stretch flips sign when lo/hi swap
    m1 = {}
    for k, v in zip(k1.tolist(), x1):
        m1[(k >> 32, k & 0xFFFFFFFF)] = v
    assert len(k1) == len(k2)
    for k, v in zip(k2.tolist(), x2):
        lo2, hi2 = k >> 32, k & 0xFFFFFFFF
        # map back to labelling 1
        a1, b1 = n - 1 - lo2, n - 1 - hi2
        key1 = (min(a1, b1), max(a1, b1))
        np.testing.assert_allclose(-v, m1[key1], atol=1e-12)


def test_net_pair_force_vanishes(orc):
    g = _dense(300, 0.52, 8)
    p = orc.make_params(g["box"], mu=0.5, shear_rate=1.0, eta0=1.0)
    s = orc.System(p, g["x"], g["a"])
    F, T, S = s.forces()
    # subtract drag (u = U_inf, w = Omega_inf initially, so drag is zero)
    tot = F.sum(axis=1)
    assert np.abs(tot).max() < 1e-9 * np.abs(F).max()
    assert s.npairs > 300


def test_einstein_viscosity(orc):
    g = json.load(open(os.path.join(GOLDEN, "einstein.json")))
    L, a = 40.0, 2.0
    p = orc.make_params([L] * 3, shear_rate=0.6, eta0=1.7)
    s = orc.System(p, np.array([[3.0], [4.0], [5.0]]), [a])
    F, T, S = s.forces()
    phi = 4 / 3 * math.pi * a ** 3 / L ** 3
    assert S[0, 1] / (1.7 * 0.6) == pytest.approx(1 + g["coefficient"] * phi, rel=1e-13)
    np.testing.assert_allclose(S, S.T)
    assert abs(S[0, 0]) < 1e-15 and abs(S[2, 2]) < 1e-15


@pytest.mark.parametrize("sign", [+1, -1])
def test_contact_stresslet_signs(orc, sign):
    """A repulsive contact along the compressional axis (1,-1)/sqrt2 raises the
    shear stress; along the extensional axis it lowers it; pressure > 0."""
    L = 30.0
    p = orc.make_params([L] * 3, shear_rate=0.0, eta0=0.0, mu=0.0)
    n = unit([1.0, -sign, 0.0])
    ov = 0.01
    xi = np.array([10.0, 10.0, 10.0])
    xj = xi + n * (2.0 - ov)
    s = orc.System(p, np.stack([xi, xj], axis=1), [1.0, 1.0])
    F, T, S = s.forces()
    want = 1e4 * ov * (2.0 - ov) / 2 / L ** 3
    assert S[0, 1] == pytest.approx(sign * want, rel=1e-12)
    assert -np.trace(S) / 3 > 0


def test_sampled_forces_are_rows_of_the_full_evaluation(orc):
    g = _dense(400, 0.52, 9)
    p = orc.make_params(g["box"], mu=0.6, shear_rate=10.0)
    s = orc.System(p, g["x"], g["a"])
    s.init_accel()
    s.step(20)                       # build up a contact history
    F, T, _ = s.forces()
    idx = np.array([0, 5, 17, 99, 250, 399])
    Fs, Ts = s.forces_sampled(idx)
    np.testing.assert_allclose(Fs, F[:, idx], rtol=1e-12, atol=1e-12 * np.abs(F).max())
    np.testing.assert_allclose(Ts, T[:, idx], rtol=1e-12, atol=1e-12 * np.abs(T).max())
