"""The wavy shear flow of Eq. 17 (Faxen drag of Eq. A1, local Omega_inf and
E_inf) and the rolling resistance of App. B on the GPU, against the FP64
oracle: default velocities, forces, torques and stress with a carried
sliding and rolling history (FP64 within 1e-10, mixed precision within
1e-5), FP64 trajectories with the committed history, batched instances whose
boxes give each its own wave number, the history and checkpoint round trips
of the rolling stretch, and the Table 5 workload (2^16 particles, a2/a1 = 3)
on sampled particles in the configurations the benchmark times."""
import numpy as np
import pytest

from fullsize_cases import contact_history, partners, sample, velocities
from parity import FP64_TOL, KAPPA_FP64, check_forces, check_per_particle, check_stress, kappa_for

pytestmark = pytest.mark.gpu

BASE = dict(mu=0.7, shear_rate=2.0, dt=1e-4, kn=1e4, kt=1e4 * 2.0 / 7.0, delta_lub=0.25,
            lub_cutoff_mode=1, f_er=5.0, lambda_d=0.05)
MODELS = {
    "wave": dict(wave_amp=8.0, wave_n=1),
    "rolling": dict(k_r=500.0),
    "both": dict(wave_amp=-6.0, wave_n=2, k_r=300.0),
}


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
    g = synth.small(3000, 0.50, 31, a_large=3.0, frac_large=0.03)
    return dict(oracle=oracle, dss=dss, synth=synth, g=g)


def _stirred(g, seed):
    rng = np.random.default_rng(seed)
    n = g["a"].shape[0]
    u = 0.5 * rng.normal(size=(3, n))
    u[0] += 2.0 * g["x"][1]
    w = 2.0 * rng.normal(size=(3, n))
    return u, w


def _kw(model, **extra):
    kw = dict(BASE)
    kw.update(MODELS[model])
    kw.update(extra)
    return kw


def test_default_velocities_follow_the_wave(env):
    g, dss, oracle = env["g"], env["dss"], env["oracle"]
    kw = _kw("both")
    o = oracle.System(oracle.make_params(g["box"], **kw), g["x"], g["a"], ids=g["ids"])
    s = dss.Suspension(g["x"], g["a"], g["box"], dss.default_params(g["box"], **kw), ids=g["ids"])
    so, st = o.get_state(), s.state()
    np.testing.assert_allclose(st["u"].cpu().numpy(), so["u"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(st["w"].cpu().numpy(), so["w"], rtol=0, atol=1e-13)
    assert np.ptp(so["w"][2]) > 1.0          # the local spin varies across the box
    s.close()


@pytest.mark.parametrize("model", ["wave", "rolling", "both"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_forces_and_stress_with_sliding_and_rolling_history(env, model, precision, tol):
    g, dss, oracle = env["g"], env["dss"], env["oracle"]
    box = g["box"]
    kw = _kw(model)
    po = oracle.make_params(box, **kw)
    u, w = _stirred(g, 5)
    o = oracle.System(po, g["x"], g["a"], ids=g["ids"], u=u, w=w)
    o.init_accel()
    o.step(12)
    st = o.get_state()
    keys, xi, xr = o.get_history(rolling=True)
    assert len(keys) > 100
    if kw.get("k_r", 0.0) > 0:
        assert np.abs(xr).max() > 0
        # overloaded rolling springs as well (the Coulomb limit acts)
        rng = np.random.default_rng(9)
        xr = xr + 0.03 * rng.normal(size=xr.shape)
    o.set_history(keys, xi, xr)
    p = dss.default_params(box, precision=precision, **kw)
    s = dss.Suspension(st["x"], g["a"], box, p, ids=g["ids"], u=st["u"], w=st["w"],
                       alpha_lin=st["al"], alpha_ang=st["aw"], nstep=o.nstep)
    s.set_history(keys, xi, xr)
    F, T = s.forces()
    Fo, To, So = o.forces()
    Fa, Ta = o.force_scale()
    check_forces(F.cpu().numpy(), Fo, Fa, tol, kappa_for(tol), "force")
    check_forces(T.cpu().numpy(), To, Ta, tol, kappa_for(tol), "torque")
    check_stress(s.stress(), So, tol)
    s.close()


@pytest.mark.parametrize("model", ["wave", "both"])
def test_trajectory_fp64(env, model):
    g, dss, oracle = env["g"], env["dss"], env["oracle"]
    box = g["box"]
    kw = _kw(model)
    u, w = _stirred(g, 6)
    po = oracle.make_params(box, **kw)
    o = oracle.System(po, g["x"], g["a"], ids=g["ids"], u=u, w=w)
    o.init_accel()
    s = dss.Suspension(g["x"], g["a"], box, dss.default_params(box, **kw), ids=g["ids"], u=u, w=w)
    for _ in range(2):
        o.step(20)
        s.step(20)
        st, so = s.state(), o.get_state()
        d = np.abs(st["x"].cpu().numpy() - so["x"])
        d = np.minimum(d, box[:, None] - d)
        assert d.max() < 1e-10
        check_per_particle(st["u"].cpu().numpy(), so["u"], FP64_TOL, what="u")
        check_per_particle(st["w"].cpu().numpy(), so["w"], FP64_TOL, what="w")
        check_stress(s.stress(), o.get_forces()[2], FP64_TOL)
        k1, x1, r1 = s.history(rolling=True)
        k2, x2, r2 = o.get_history(rolling=True)
        np.testing.assert_array_equal(k1, k2)
        check_per_particle(x1.T, x2.T, FP64_TOL, floor=0.1, what="stretch")
        if kw.get("k_r", 0.0) > 0:
            check_per_particle(r1.T, r2.T, FP64_TOL, floor=0.1, what="rolling stretch")
            assert np.abs(r2).max() > 0
        else:
            assert not np.any(r1)
    s.close()


def test_rolling_history_and_checkpoint_round_trip(env):
    g, dss, oracle = env["g"], env["dss"], env["oracle"]
    box = g["box"]
    kw = _kw("both")
    u, w = _stirred(g, 7)
    p = dss.default_params(box, **kw)
    s = dss.Suspension(g["x"], g["a"], box, p, ids=g["ids"], u=u, w=w)
    s.step(10)
    keys, xi, xr = s.history(rolling=True)
    assert np.abs(xr).max() > 0
    # replacing the history with itself changes nothing
    s.set_history(keys, xi, xr)
    k2, x2, r2 = s.history(rolling=True)
    np.testing.assert_array_equal(k2, keys)
    np.testing.assert_array_equal(x2, xi)
    np.testing.assert_array_equal(r2, xr)
    ck = s.save()
    s.step(15)
    a = s.state()
    ha = s.history(rolling=True)
    s.load(ck)
    s.step(15)
    b = s.state()
    hb = s.history(rolling=True)
    for q in ("x", "u", "w"):
        np.testing.assert_array_equal(a[q].cpu().numpy(), b[q].cpu().numpy())
    for q in range(3):
        np.testing.assert_array_equal(ha[q], hb[q])
    # a plain history drops the rolling stretch
    s.set_history(keys, xi)
    assert not np.any(s.history(rolling=True)[2])
    s.close()


def test_batched_instances_take_their_own_wave_number(env):
    dss, oracle, synth = env["dss"], env["oracle"], env["synth"]
    members = [(synth.small(900, 0.45, 41, a_large=2.0, frac_large=0.1), 1.5),
               (synth.small(1500, 0.52, 42, a_large=2.0, frac_large=0.1), 0.6)]
    kw = _kw("both")
    kw.pop("shear_rate")
    xs, us, ws, keys_all, xi_all, xr_all, Fo, To, Fa_all, Ta_all = [], [], [], [], [], [], [], [], [], []
    off = 0
    for g, gd in members:
        po = oracle.make_params(g["box"], shear_rate=gd, **kw)
        u, w = _stirred(g, 8)
        o = oracle.System(po, g["x"], g["a"], ids=g["ids"], u=u, w=w)
        o.init_accel()
        o.step(8)
        st = o.get_state()
        k, xi, xr = o.get_history(rolling=True)
        F, T, _ = o.forces()
        fa, ta = o.force_scale()
        Fa_all.append(fa)
        Ta_all.append(ta)
        lo, hi = k >> 32, k & 0xffffffff
        keys_all.append(((lo + off) << 32) | (hi + off))
        xi_all.append(xi)
        xr_all.append(xr)
        xs.append(st)
        Fo.append(F)
        To.append(T)
        off += g["a"].shape[0]
    assert all(np.abs(r).max() > 0 for r in xr_all)
    cat = lambda q: np.concatenate([s[q] for s in xs], axis=1)
    a = np.concatenate([g["a"] for g, _ in members])
    ids = np.concatenate([g["ids"] for g, _ in members[:1]] +
                         [members[1][0]["ids"] + members[0][0]["a"].shape[0]]).astype(np.int32)
    p = dss.default_params(**kw)
    b = dss.Batch(cat("x"), a, [g["a"].shape[0] for g, _ in members], [g["box"] for g, _ in members],
                  [gd for _, gd in members], p, ids=ids, u=cat("u"), w=cat("w"),
                  alpha_lin=cat("al"), alpha_ang=cat("aw"), nstep=8)
    b.set_history(np.concatenate(keys_all), np.concatenate(xi_all), np.concatenate(xr_all))
    F, T = b.forces()
    F, T = F.cpu().numpy(), T.cpu().numpy()
    n0 = members[0][0]["a"].shape[0]
    for q, (f, t, fa, ta) in enumerate(zip(Fo, To, Fa_all, Ta_all)):
        sl = slice(0, n0) if q == 0 else slice(n0, None)
        check_forces(F[:, sl], f, fa, FP64_TOL, KAPPA_FP64, "force %d" % q)
        check_forces(T[:, sl], t, ta, FP64_TOL, KAPPA_FP64, "torque %d" % q)
    b.close()


@pytest.fixture(scope="module")
def table5(env):
    oracle, synth = env["oracle"], env["synth"]
    spec = synth.SPECS["c6"]
    g = synth.generate(spec)
    box = g["box"]
    kw = dict(mu=spec.mu, kn=spec.kn, shear_rate=spec.shear_rate, dt=spec.dt, **spec.extra)
    kw_r = dict(kw, k_r=0.05 * spec.kn)
    po = oracle.make_params(box, **kw_r)
    u, w = velocities(g["x"], g["a"], spec.shear_rate, seed=61)
    idx = sample(g["a"], m=120, seed=6)
    nstep = 3_333_333
    off = oracle.le_offset(po, nstep)
    keys, xi = contact_history(oracle, po, off, g["x"], g["a"], g["ids"], u, w, idx, seed=61)
    xr = 2e-4 * np.random.default_rng(62).normal(size=xi.shape)
    out = dict(g=g, kw=kw, kw_r=kw_r, u=u, w=w, idx=idx, nstep=nstep, keys=keys, xi=xi, xr=xr)
    for name, k in (("plain", kw), ("rolling", kw_r)):
        o = oracle.System(oracle.make_params(box, **k), g["x"], g["a"], ids=g["ids"], u=u, w=w, nstep=nstep)
        o.set_history(keys, xi, xr)
        out[name] = o.forces_sampled(idx, scale=True)
    out["want"] = {int(k): oracle.neighbours_of(g["x"], g["a"], g["ids"], po, off, int(k)) for k in idx}
    return out


@pytest.mark.parametrize("rolling", [False, True])
@pytest.mark.parametrize("precision,tol", [("mixed", 1e-5), ("fp64", 1e-10)])
def test_table5_sampled_neighbours_and_forces(env, table5, rolling, precision, tol):
    dss = env["dss"]
    c = table5
    g, idx = c["g"], c["idx"]
    n = g["a"].shape[0]
    p = dss.default_params(g["box"], precision=precision, **(c["kw_r"] if rolling else c["kw"]))
    s = dss.Suspension(g["x"], g["a"], g["box"], p, ids=g["ids"], u=c["u"], w=c["w"], nstep=c["nstep"],
                       alpha_lin=np.zeros((3, n)), alpha_ang=np.zeros((3, n)))
    s.neighbour_build()
    pairs = s.pairs()
    for k in idx:
        np.testing.assert_array_equal(partners(pairs, int(g["ids"][k])), c["want"][int(k)])
    assert len(c["keys"]) > 100
    s.set_history(c["keys"], c["xi"], c["xr"])
    F, T = s.forces()
    F, T = F.cpu().numpy(), T.cpu().numpy()
    Fo, To, Fa, Ta = c["rolling" if rolling else "plain"]
    check_forces(F[:, idx], Fo, Fa, tol, kappa_for(tol), "force")
    check_forces(T[:, idx], To, Ta, tol, kappa_for(tol), "torque")
    s.close()
