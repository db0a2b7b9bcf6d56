"""GPU path (libdss via the C ABI) against the CPU FP64 oracle.

Neighbour sets must be equal bit for bit (as sorted (lo id, hi id) pairs);
FP64 forces and torques within 1e-10 of each particle's own (the per-particle
bound of tests/parity.py), every stress component and reported quantity
within 1e-10 of its own value; the 1000-step FP64 trajectory of the
1000-particle configuration within 1e-10 per particle.
"""
import numpy as np
import pytest

from parity import (FP64_TOL, KAPPA_FP64, MIXED_TOL, KAPPA_MIXED, check_forces, check_per_particle,
                    check_stress, periodic_diff)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import oracle
    import paper_2108_01013_gb300 as dss
    from paper_2108_01013_gb300 import synth
    oracle.build()
    dss.build()
    synth.build()
    return dict(oracle=oracle, dss=dss, synth=synth, torch=torch)


def _params(env, box, **kw):
    return env["dss"].default_params(box, **kw), env["oracle"].make_params(box, **kw)


CASES = [
    # n, phi, seed, nstep (Lees-Edwards offset), cutoff mode, delta
    (300, 0.45, 1, 0, 0, 0.05),
    (777, 0.55, 2, 12345, 0, 0.05),
    (1000, 0.50, 3, 987654, 0, 0.05),
    (1501, 0.52, 4, 31, 1, 0.08),
    (2048, 0.40, 5, 4567, 0, 0.25),
]


@pytest.mark.parametrize("n,phi,seed,nstep,mode,delta", CASES)
def test_neighbour_pairs_bit_exact(env, n, phi, seed, nstep, mode, delta):
    g = env["synth"].small(n, phi, seed)
    box = g["box"]
    p, po = _params(env, box, lub_cutoff_mode=mode, delta_lub=delta, shear_rate=1.3, dt=1e-3)
    s = env["dss"].Suspension(g["x"], g["a"], box, p, ids=g["ids"], nstep=nstep,
                              alpha_lin=np.zeros((3, n)), alpha_ang=np.zeros((3, n)))
    s.neighbour_build()
    got = s.pairs()
    off = env["oracle"].le_offset(po, nstep)
    want = env["oracle"].pairs_bruteforce(g["x"], g["a"], g["ids"], po, off)
    assert len(want) > n // 2
    np.testing.assert_array_equal(got, want)
    c = s.counters()
    assert c["npairs"] == len(want)
    s.close()


def test_neighbour_pairs_polydisperse_and_boundary_layer(env):
    """Radii log-uniform in [1, 3], many particles at the Lees-Edwards
    boundary, offsets across one full period of the shift."""
    rng = np.random.default_rng(9)
    synth = env["synth"]
    spec = synth.Spec("poly", 1200, 0.45, radii="loguniform", a_min=1.0, a_max=3.0, seed=21)
    g = synth.generate(spec)
    box = g["box"]
    x = g["x"].copy()
    # push a third of the particles into the top and bottom layers
    k = rng.choice(g["a"].shape[0], size=400, replace=False)
    x[1, k[:200]] = rng.uniform(0, 2.0, size=200)
    x[1, k[200:]] = box[1] - rng.uniform(1e-9, 2.0, size=200)
    p, po = _params(env, box, shear_rate=0.9, dt=1e-2)
    for nstep in (0, 7, 333, 1001, 5555):
        s = env["dss"].Suspension(x, g["a"], box, p, ids=g["ids"], nstep=nstep,
                                  alpha_lin=np.zeros_like(x), alpha_ang=np.zeros_like(x))
        s.neighbour_build()
        off = env["oracle"].le_offset(po, nstep)
        want = env["oracle"].pairs_bruteforce(x, g["a"], g["ids"], po, off)
        np.testing.assert_array_equal(s.pairs(), want)
        s.close()


def test_neighbour_pairs_near_cutoff(env):
    """Pairs placed within a few ulps of the cutoff on both sides."""
    rng = np.random.default_rng(4)
    box = np.array([30.0, 30.0, 30.0])
    pts, rad = [], []
    for t in range(60):
        c = rng.uniform(3, 27, size=3)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        ai, aj = (1.0, 1.4) if t % 2 else (1.4, 1.4)
        s = (ai + aj) * (1 + 0.05 / 2)
        r = s * (1 + rng.choice([-1, 1]) * rng.uniform(0, 4e-16))
        pts += [c, c + r * u]
        rad += [ai, aj]
    x = np.array(pts).T.copy()
    x = np.mod(x, box[:, None])
    a = np.array(rad)
    n = a.shape[0]
    ids = np.arange(n, dtype=np.int32)
    p, po = _params(env, box, shear_rate=0.0)
    s = env["dss"].Suspension(x, a, box, p, ids=ids, alpha_lin=np.zeros_like(x),
                              alpha_ang=np.zeros_like(x))
    s.neighbour_build()
    want = env["oracle"].pairs_bruteforce(x, a, ids, po, 0.0)
    np.testing.assert_array_equal(s.pairs(), want)
    s.close()


@pytest.mark.parametrize("seed,nstep,mu", [(1, 0, 0.5), (2, 4321, 1.0)])
def test_forces_and_stress_fp64(env, seed, nstep, mu):
    g = env["synth"].small(1000, 0.50, seed)
    box = g["box"]
    p, po = _params(env, box, mu=mu)
    rng = np.random.default_rng(seed)
    n = g["a"].shape[0]
    u = np.zeros((3, n))
    u[0] = 1.0 * g["x"][1]
    u += 0.3 * rng.normal(size=(3, n))
    w = 0.3 * rng.normal(size=(3, n))
    s = env["dss"].Suspension(g["x"], g["a"], box, p, ids=g["ids"], u=u, w=w, nstep=nstep,
                              alpha_lin=np.zeros((3, n)), alpha_ang=np.zeros((3, n)))
    F, T = s.forces()
    S = s.stress()
    o = env["oracle"].System(po, g["x"], g["a"], ids=g["ids"], u=u, w=w, nstep=nstep)
    Fo, To, So = o.forces()
    Fa, Ta = o.force_scale()
    assert o.ncontacts > 10
    check_forces(F.cpu().numpy(), Fo, Fa, FP64_TOL, KAPPA_FP64, "force")
    check_forces(T.cpu().numpy(), To, Ta, FP64_TOL, KAPPA_FP64, "torque")
    check_stress(S, So, FP64_TOL)
    c = s.counters()
    assert c["npairs"] == o.npairs and c["ncontacts"] == o.ncontacts
    s.close()


@pytest.mark.parametrize("precision,tol,kappa,mode", [("fp64", FP64_TOL, KAPPA_FP64, 0),
                                                      ("mixed", MIXED_TOL, KAPPA_MIXED, 0),
                                                      ("fp64", FP64_TOL, KAPPA_FP64, 1)])
def test_forces_with_lubrication_taper(env, precision, tol, kappa, mode):
    """The differentiable cutoff (lubrication scaled down over the last 30% of
    the range) against the oracle, with a wide range so that many pairs sit in
    the band."""
    g = env["synth"].small(1200, 0.50, 7)
    box = g["box"]
    kw = dict(mu=0.5, lub_taper=0.3, delta_lub=0.3, lub_cutoff_mode=mode)
    p = env["dss"].default_params(box, precision=precision, **kw)
    po = env["oracle"].make_params(box, **kw)
    rng = np.random.default_rng(3)
    n = g["a"].shape[0]
    u = 0.3 * rng.normal(size=(3, n))
    w = 0.3 * rng.normal(size=(3, n))
    s = env["dss"].Suspension(g["x"], g["a"], box, p, ids=g["ids"], u=u, w=w,
                              alpha_lin=np.zeros((3, n)), alpha_ang=np.zeros((3, n)))
    F, T = s.forces()
    o = env["oracle"].System(po, g["x"], g["a"], ids=g["ids"], u=u, w=w)
    Fo, To, So = o.forces()
    Fa, Ta = o.force_scale()
    check_forces(F.cpu().numpy(), Fo, Fa, tol, kappa, "force")
    check_forces(T.cpu().numpy(), To, Ta, tol, kappa, "torque")
    check_stress(s.stress(), So, tol)
    # the taper changes the answer: the untapered oracle differs
    po0 = env["oracle"].make_params(box, **dict(kw, lub_taper=0.0))
    Fu = env["oracle"].System(po0, g["x"], g["a"], ids=g["ids"], u=u, w=w).forces()[0]
    assert np.linalg.norm(Fu - Fo) > 1e-3 * np.linalg.norm(Fo)
    s.close()


def test_forces_with_carried_history(env):
    """History handed over from the oracle gives the same tangential forces."""
    g = env["synth"].small(800, 0.52, 7)
    box = g["box"]
    p, po = _params(env, box, mu=0.7, shear_rate=20.0)
    o = env["oracle"].System(po, g["x"], g["a"], ids=g["ids"])
    o.init_accel()
    o.step(40)
    st = o.get_state()
    keys, xi = o.get_history()
    assert len(keys) > 20 and np.abs(xi).max() > 0
    s = env["dss"].Suspension(st["x"], g["a"], box, p, ids=g["ids"], u=st["u"], w=st["w"],
                              alpha_lin=st["al"], alpha_ang=st["aw"], nstep=o.nstep)
    s.set_history(keys, xi)
    k2, x2 = s.history()
    np.testing.assert_array_equal(k2, keys)
    np.testing.assert_array_equal(x2, xi)
    F, T = s.forces()
    Fo, To, So = o.forces()
    Fa, Ta = o.force_scale()
    check_forces(F.cpu().numpy(), Fo, Fa, FP64_TOL, KAPPA_FP64, "force")
    check_forces(T.cpu().numpy(), To, Ta, FP64_TOL, KAPPA_FP64, "torque")
    check_stress(s.stress(), So, FP64_TOL)
    s.close()


def test_trajectory_fp64_c1(env):
    """The 1000-particle FP64 configuration over its full 1000 steps on both
    sides (Eq. 15-16).  In FP64 mode the predictor, the corrector, the drag
    and the accelerations round every product and sum on their own as the
    oracle does, so the two trajectories differ only through the order of
    the force sums; every 100 steps each particle's position is within
    1e-10 a_min, its velocity and angular velocity within 1e-10 of their own,
    every stress component within 1e-10.  The divergence is recorded per
    chunk and must grow by less than a factor 1e3 over the run (measured on
    GB300: ~1e-14 of the velocities after 50 steps, ~4e-13 after 1000)."""
    synth = env["synth"]
    g = synth.generate(synth.SPECS["c1"])
    box = g["box"]
    p, po = _params(env, box, mu=0.5)
    s = env["dss"].Suspension(g["x"], g["a"], box, p, ids=g["ids"])
    o = env["oracle"].System(po, g["x"], g["a"], ids=g["ids"])
    o.init_accel()
    st0 = s.state()
    so = o.get_state()
    check_per_particle(st0["al"].cpu().numpy(), so["al"], FP64_TOL, what="alpha^0")
    growth = []
    for chunk in range(10):
        s.step(100)
        o.step(100)
        st = {k: v.cpu().numpy() for k, v in s.state().items()}
        so = o.get_state()
        dx = periodic_diff(st["x"], so["x"], box).max()
        assert dx < 1e-10 * g["a"].min(), (chunk, dx)
        ru = check_per_particle(st["u"], so["u"], FP64_TOL, what="u after %d steps" % (100 * chunk + 100))
        rw = check_per_particle(st["w"], so["w"], FP64_TOL, what="w after %d steps" % (100 * chunk + 100))
        check_stress(s.stress(), o.get_forces()[2], FP64_TOL)
        growth.append(max(ru, rw, dx))
    assert max(growth) < 1e3 * max(growth[0], 1e-16), growth
    k1, x1 = s.history()
    k2, x2 = o.get_history()
    np.testing.assert_array_equal(k1, k2)
    assert np.abs(x1 - x2).max() < FP64_TOL * max(np.abs(x2).max(), 1e-12)
    assert s.counters()["steps_done"] == 1000
    s.close()


def test_deterministic_bitwise(env):
    g = env["synth"].small(1500, 0.52, 12)
    box = g["box"]
    p, _ = _params(env, box, mu=0.5, shear_rate=5.0)
    out = []
    for rep in range(2):
        s = env["dss"].Suspension(g["x"], g["a"], box, p, ids=g["ids"])
        s.step(50)
        st = s.state()
        out.append((st["x"].cpu().numpy(), st["u"].cpu().numpy(), st["w"].cpu().numpy(), s.stress()))
        s.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_error_reporting(env):
    dss = env["dss"]
    g = env["synth"].small(500, 0.5, 3)
    box = g["box"]
    p = dss.default_params(box, capacity_M=1)
    with pytest.raises(dss.DssError) as e:
        s = dss.Suspension(g["x"], g["a"], box, p, ids=g["ids"])
    assert e.value.code == -3
    small = np.array([6.0, 6.0, 6.0])
    with pytest.raises(dss.DssError) as e:
        dss.Suspension(np.full((3, 4), 1.0) + np.arange(4), np.ones(4), small, dss.default_params())
    assert e.value.code == -2
    x = g["x"].copy()
    x[0, 5] = box[0] + 1.0
    with pytest.raises(dss.DssError) as e:
        dss.Suspension(x, g["a"], box, dss.default_params(box))
    assert e.value.code == -1
    ids = g["ids"].copy()
    ids[3] = ids[4]
    with pytest.raises(dss.DssError) as e:
        dss.Suspension(g["x"], g["a"], box, dss.default_params(box), ids=ids)
    assert e.value.code == -1


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_load_state_keeps_history(env, precision):
    """dss_load_state (the per-step upload of a caller that keeps its own
    state) with the same values must leave the trajectory unchanged, bit for
    bit: the contact history is then found through the id map rather than
    the sort permutation."""
    g = env["synth"].small(1500, 0.54, 8)
    box = g["box"]
    p = env["dss"].default_params(box, mu=1.0, shear_rate=3.0, precision=precision)
    a = env["dss"].Suspension(g["x"], g["a"], box, p, ids=g["ids"])
    b = env["dss"].Suspension(g["x"], g["a"], box, p, ids=g["ids"])
    a.step(20)
    b.step(20)
    st = a.state()
    a.load_state(st["x"], st["u"], st["w"], st["al"], st["aw"])
    a.step(15)
    b.step(15)
    assert a.counters()["ncontacts"] > 50
    sa, sb = a.state(), b.state()
    for k in sa:
        assert env["torch"].equal(sa[k], sb[k]), k
    ka, xa = a.history()
    kb, xb = b.history()
    assert np.array_equal(ka, kb) and np.array_equal(xa, xb)
    a.close()
    b.close()
