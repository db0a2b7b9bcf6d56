"""Analysis pass on the GPU (§8(f) item 3) against the oracle: Lees-Edwards
image counts (exact), the shear-wise dispersion D_y and velocity
autocorrelation C_v of Eq. 18-19 over an FP64 trajectory, the clusters of
contacting particles (Fig. 10-11; exact labels) for the oracle's own contact
set, and the rheological quantities derived from the bulk stress (last
evaluation and running mean)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import oracle
    from oracle import analysis
    import paper_2108_01013_gb300 as dss
    from paper_2108_01013_gb300 import synth
    oracle.build()
    dss.build()
    synth.build()
    return dict(oracle=oracle, an=analysis, dss=dss, synth=synth)


def _stirred(g, seed, vy=20.0):
    rng = np.random.default_rng(seed)
    n = g["a"].shape[0]
    u = np.zeros((3, n))
    u[0] = g["x"][1]
    u[1] = vy * rng.normal(size=n)
    w = np.zeros((3, n))
    w[2] = -0.5
    return u, w


def test_images_and_dispersion_match_oracle(env):
    g = env["synth"].small(900, 0.45, 41)
    box = g["box"]
    n = g["a"].shape[0]
    u, w = _stirred(g, 3, vy=16.0)
    kw = dict(mu=0.5, shear_rate=1.0, dt=1e-3)
    po = env["oracle"].make_params(box, **kw)
    o = env["oracle"].System(po, g["x"], g["a"], ids=g["ids"], u=u, w=w)
    o.init_accel()
    p = env["dss"].default_params(box, **kw)
    s = env["dss"].Suspension(g["x"], g["a"], box, p, ids=g["ids"], u=u, w=w)
    s.dispersion_mark()
    y0, v0 = g["x"][1].copy(), u[1].copy()
    for chunk in range(2):
        o.step(40)
        s.step(40)
        st = o.get_state()
        iy = o.get_images()
        np.testing.assert_array_equal(s.images(), iy)
        y = st["x"][1] + iy * box[1]
        want = env["an"].dispersion(y, y0, st["u"][1], v0, o.nstep * kw["dt"], kw["shear_rate"])
        got = s.dispersion()[0]
        assert got[2] == pytest.approx(o.nstep * kw["dt"], rel=1e-12)
        # the two FP64 trajectories agree to ~1e-9 in velocity (summation
        # orders differ), which bounds these ratios of sums
        assert got[0] == pytest.approx(want[0], rel=1e-7)
        assert got[1] == pytest.approx(want[1], rel=1e-7, abs=1e-12)
    assert np.abs(iy).sum() > 10              # the trajectory did cross y = 0 and y = L_y
    s.close()


@pytest.mark.parametrize("mu,phi,seed", [(0.7, 0.55, 5), (0.3, 0.50, 6)])
def test_contact_clusters_match_oracle(env, mu, phi, seed):
    g = env["synth"].small(1500, phi, seed)
    box = g["box"]
    n = g["a"].shape[0]
    kw = dict(mu=mu, shear_rate=5.0)
    po = env["oracle"].make_params(box, **kw)
    o = env["oracle"].System(po, g["x"], g["a"], ids=g["ids"])
    o.init_accel()
    o.step(15)
    st = o.get_state()
    keys, xi = o.get_history()
    assert len(keys) > 100
    label_o, k_o = env["an"].contact_clusters(n, keys)
    p = env["dss"].default_params(box, **kw)
    s = env["dss"].Suspension(st["x"], g["a"], box, p, ids=g["ids"], u=st["u"], w=st["w"],
                              alpha_lin=st["al"], alpha_ang=st["aw"], nstep=o.nstep)
    # before any history: every particle is its own cluster
    lab0, k0 = s.contact_clusters()
    assert k0 == n and np.array_equal(lab0, np.arange(n))
    s.set_history(keys, xi)
    label, k = s.contact_clusters()
    assert k == k_o
    np.testing.assert_array_equal(label, label_o)
    assert env["an"].cluster_sizes(label).max() > 3
    s.close()


def test_rheology_matches_oracle(env):
    g = env["synth"].small(1200, 0.52, 8)
    box = g["box"]
    kw = dict(mu=0.6, shear_rate=2.0, eta0=1.3)
    po = env["oracle"].make_params(box, **kw)
    o = env["oracle"].System(po, g["x"], g["a"], ids=g["ids"])
    o.init_accel()
    o.step(5)
    st = o.get_state()
    keys, xi = o.get_history()
    p = env["dss"].default_params(box, **kw)
    s = env["dss"].Suspension(st["x"], g["a"], box, p, ids=g["ids"], u=st["u"], w=st["w"],
                              alpha_lin=st["al"], alpha_ang=st["aw"], nstep=o.nstep)
    s.set_history(keys, xi)
    s.forces()
    _, _, So = o.forces()
    want = env["an"].rheology(So, kw["shear_rate"], kw["eta0"])
    got = s.rheology(mean=False)[0]
    names = ["sigma", "N1", "N2", "Pi", "eta_r", "eta_n"]
    scale = np.abs(So).max()
    for q, nm in enumerate(names):
        tol = 1e-10 * (scale if nm in ("sigma", "N1", "N2", "Pi") else scale / (kw["eta0"] * kw["shear_rate"]))
        assert abs(got[q] - want[nm]) <= tol, nm
    # running mean over the committed steps (the mean restarts with the state)
    means = []
    for _ in range(6):
        o.step(1)
        means.append(o.get_forces()[2])
    s.step(6)
    got = s.rheology(mean=True)[0]
    want = env["an"].rheology(np.mean(means, axis=0), kw["shear_rate"], kw["eta0"])
    for q, nm in enumerate(names):
        assert got[q] == pytest.approx(want[nm], rel=1e-8, abs=1e-10 * scale), nm
    s.close()


def test_phi_profile_matches_oracle(env):
    """The local volume fraction along y by size class (Sec. III B, Fig. 12)
    of the committed state after 30 FP64 steps (particles crossing y = 0
    and y = L_y included), single instance and a two-instance batch, against
    the oracle's slab integrals of the same state, per slab within 1e-12;
    reproducible bit for bit."""
    an, dss = env["an"], env["dss"]
    g = env["synth"].small(2000, 0.52, 43)
    box = g["box"]
    p = dss.default_params(box, mu=0.5, shear_rate=3.0)
    u, w = _stirred(g, 8)
    s = dss.Suspension(g["x"], g["a"], box, p, ids=g["ids"], u=u, w=w)
    s.step(30)
    y = s.state()["x"].cpu().numpy()[1]
    for nb in (1, 7, 40):
        got = s.phi_profile(nb, a_split=1.2)
        want = an.phi_profile(y, g["a"], box, nb, a_split=1.2)
        np.testing.assert_allclose(got[0], want, rtol=1e-12, atol=1e-14)
        assert np.array_equal(got, s.phi_profile(nb, a_split=1.2))
    s.close()
    # two instances, each its own box
    ms = [env["synth"].small(700, 0.45, 44), env["synth"].small(900, 0.55, 45)]
    x = np.concatenate([m["x"] for m in ms], axis=1)
    a = np.concatenate([m["a"] for m in ms])
    b = dss.Batch(x, a, [700, 900], [m["box"] for m in ms], [1.0, 2.0], dss.default_params(mu=0.5))
    got = b.phi_profile(12, a_split=1.2)
    for k, m in enumerate(ms):
        want = an.phi_profile(m["x"][1], m["a"], m["box"], 12, a_split=1.2)
        np.testing.assert_allclose(got[k], want, rtol=1e-12, atol=1e-14)
    b.close()
