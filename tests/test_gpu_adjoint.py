"""Reverse-mode gradients of a rollout (dss_adjoint) against the FP64 adjoint
oracle (plain PyTorch autograd over the oracle's model), against central
finite differences of the GPU forward, and for independence of the
checkpoint interval (the replayed segments repeat the forward bit for bit).
Gradients with respect to the initial state are compared per particle, the
parameter gradients one by one (tests/parity.py)."""
import numpy as np
import pytest

from parity import check_per_particle, check_scalars

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import oracle
    from oracle import adjoint as oadj
    import paper_2108_01013_gb300 as dss
    from paper_2108_01013_gb300 import synth
    oracle.build()
    dss.build()
    synth.build()
    return dict(oracle=oracle, oadj=oadj, dss=dss, synth=synth, torch=torch)


def _case(env, taper, n=260, seed=61):
    g = env["synth"].small(n, 0.52, seed)
    rng = np.random.default_rng(5)
    u0 = np.zeros((3, n))
    u0[0] = 5.0 * g["x"][1]
    u0 += 0.5 * rng.normal(size=(3, n))
    w0 = 0.5 * rng.normal(size=(3, n))
    kw = dict(shear_rate=5.0, dt=1e-4, lub_taper=taper)
    th = dict(kn=1e4, kt=6e3, gamma_n=0.5, mu=0.4, delta_lub=0.2 if taper else 0.05)
    return g, u0, w0, kw, th


def _weights(T, gd):
    W = np.zeros((T, 9))
    W[:, 1] = 1.0 / (T * gd)
    W[:, 3] = 0.25 / (T * gd)
    W[:, 0] = 0.1 / T
    return W


def _gpu(env, g, u0, w0, kw, th, T, W, precision="fp64", ckpt=5, nstep0=3):
    p = env["dss"].default_params(g["box"], precision=precision, **th, **kw)
    s = env["dss"].Suspension(g["x"], g["a"], g["box"], p, ids=g["ids"], u=u0, w=w0, nstep=nstep0)
    r = s.adjoint(T, W, ckpt_every=ckpt)
    st = s.state()
    s.close()
    return r, st


@pytest.mark.parametrize("taper", [0.0, 0.3])
def test_adjoint_matches_oracle_fp64(env, taper):
    g, u0, w0, kw, th = _case(env, taper)
    T = 12
    W = _weights(T, kw["shear_rate"])
    o = env["oadj"].gradients(g["box"], g["x"], g["a"], u0, w0, T, W, **th, **kw, nstep0=3)
    r, st = _gpu(env, g, u0, w0, kw, th, T, W)
    assert r["J"] == pytest.approx(o["J"], rel=1e-11)
    check_scalars(r["params"], o["params"], 1e-8, floor=1e-6, what="dJ/dtheta")
    for k in range(5):
        assert r["params"][k] == pytest.approx(o["params"][k], rel=1e-7, abs=1e-12 * abs(o["J"]))
    check_per_particle(r["x0"], o["x0"], 1e-8, what="dJ/dx0")
    check_per_particle(r["u0"], o["u0"], 1e-8, what="dJ/du0")
    check_per_particle(r["w0"], o["w0"], 1e-8, what="dJ/dw0")
    assert np.abs(r["alpha0"]).max() == 0.0
    # the handle ends after the rollout
    box = g["box"]
    d = np.abs(st["x"].cpu().numpy() - o["final"]["x"])
    d = np.minimum(d, box[:, None] - d)
    assert d.max() < 1e-12


def test_adjoint_independent_of_checkpoint_interval(env):
    g, u0, w0, kw, th = _case(env, 0.3)
    T = 12
    W = _weights(T, kw["shear_rate"])
    a, _ = _gpu(env, g, u0, w0, kw, th, T, W, ckpt=12)
    b, _ = _gpu(env, g, u0, w0, kw, th, T, W, ckpt=5)
    c, _ = _gpu(env, g, u0, w0, kw, th, T, W, ckpt=1)
    for k in ("params", "x0", "u0", "w0"):
        assert np.array_equal(a[k], b[k]) and np.array_equal(a[k], c[k]), k
    assert a["J"] == b["J"] == c["J"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adjoint_recovers_pair_capacity_growth(env, precision):
    """A rollout whose first step overflows the pair buffers (allocated for
    one pair per particle, no enumeration before the rollout): the forward
    segment is redone from its device checkpoint after the buffers grow, and
    the objective, the gradients and the final state equal those of a handle
    that never overflowed."""
    g, u0, w0, kw, th = _case(env, 0.3)
    n = g["a"].shape[0]
    T = 9
    W = _weights(T, kw["shear_rate"])
    dss = env["dss"]
    out = []
    for pc in (1, 0):
        p = dss.default_params(g["box"], precision=precision, pair_capacity=pc, **th, **kw)
        s = dss.Suspension(g["x"], g["a"], g["box"], p, ids=g["ids"], u=u0, w=w0, nstep=3,
                           alpha_lin=np.zeros((3, n)), alpha_ang=np.zeros((3, n)))
        b0 = s.device_bytes()
        r = s.adjoint(T, W, ckpt_every=4, initial_forces=False)
        grew = s.device_bytes() > b0
        st = s.state()
        c = s.counters()
        s.close()
        out.append((r, st, grew, c))
    (ra, sa, grew_a, ca), (rb, sb, _, cb) = out
    assert grew_a
    assert ca["steps_done"] == cb["steps_done"] == T
    assert ra["J"] == rb["J"]
    for k in ("params", "x0", "u0", "w0", "alpha0", "beta0"):
        assert np.array_equal(ra[k], rb[k]), k
    for k in sa:
        assert env["torch"].equal(sa[k], sb[k]), k


def test_adjoint_mixed_precision_vs_oracle(env):
    g, u0, w0, kw, th = _case(env, 0.3)
    T = 12
    W = _weights(T, kw["shear_rate"])
    o = env["oadj"].gradients(g["box"], g["x"], g["a"], u0, w0, T, W, **th, **kw, nstep0=3)
    r, _ = _gpu(env, g, u0, w0, kw, th, T, W, precision="mixed")
    assert r["J"] == pytest.approx(o["J"], rel=1e-6)
    for k in range(5):
        assert r["params"][k] == pytest.approx(o["params"][k], rel=1e-4, abs=1e-9 * abs(o["J"]))
    check_per_particle(r["x0"], o["x0"], 1e-4, floor=0.1, what="dJ/dx0 (mixed)")


def test_adjoint_with_echem_matches_oracle(env):
    """The electro-chemical forces of Eq. 6-7 (repulsion below 20 lambda_D,
    attraction below 4 a0) in the differentiated rollout: FP64 gradients
    equal the FP64 autograd oracle."""
    g = env["synth"].small(1400, 0.52, 62)
    n = g["a"].shape[0]
    rng = np.random.default_rng(6)
    u0 = np.zeros((3, n))
    u0[0] = 5.0 * g["x"][1]
    u0 += 0.5 * rng.normal(size=(3, n))
    w0 = 0.5 * rng.normal(size=(3, n))
    kw = dict(shear_rate=5.0, dt=1e-4, lub_taper=0.3, f_er=30.0, lambda_d=0.05, hamaker=0.01,
              vdw_eps=0.05)
    th = dict(kn=1e4, kt=6e3, gamma_n=0.5, mu=0.4, delta_lub=0.2)
    T = 10
    W = _weights(T, kw["shear_rate"])
    o = env["oadj"].gradients(g["box"], g["x"], g["a"], u0, w0, T, W, **th, **kw, nstep0=3)
    r, _ = _gpu(env, g, u0, w0, kw, th, T, W)
    assert r["J"] == pytest.approx(o["J"], rel=1e-11)
    check_scalars(r["params"], o["params"], 1e-8, floor=1e-6, what="dJ/dtheta")
    check_per_particle(r["x0"], o["x0"], 1e-8, what="dJ/dx0")
    check_per_particle(r["u0"], o["u0"], 1e-8, what="dJ/du0")
    check_per_particle(r["w0"], o["w0"], 1e-8, what="dJ/dw0")


@pytest.mark.parametrize("ext", [dict(wave_amp=4.0, wave_n=1), dict(k_r=1e3),
                                 dict(wave_amp=4.0, wave_n=1, k_r=1e3)],
                         ids=["wave", "rolling", "wave_rolling"])
def test_adjoint_wave_and_rolling_match_oracle(env, ext):
    """The wavy shear flow of Eq. 17 (ambient flow, pair strain, Faxen drag
    and local stresslets depending on y) and rolling resistance (App. B, the
    rolling stretch carried between steps) in the differentiated rollout:
    FP64 gradients equal the FP64 autograd oracle."""
    g, u0, w0, kw, th = _case(env, 0.3)
    kw = dict(kw, **ext)
    T = 12
    W = _weights(T, kw["shear_rate"])
    o = env["oadj"].gradients(g["box"], g["x"], g["a"], u0, w0, T, W, **th, **kw, nstep0=3)
    r, st = _gpu(env, g, u0, w0, kw, th, T, W)
    assert r["J"] == pytest.approx(o["J"], rel=1e-11)
    check_scalars(r["params"], o["params"], 1e-8, floor=1e-6, what="dJ/dtheta")
    check_per_particle(r["x0"], o["x0"], 1e-8, what="dJ/dx0")
    check_per_particle(r["u0"], o["u0"], 1e-8, what="dJ/du0")
    check_per_particle(r["w0"], o["w0"], 1e-8, what="dJ/dw0")
    box = g["box"]
    d = np.abs(st["x"].cpu().numpy() - o["final"]["x"])
    d = np.minimum(d, box[:, None] - d)
    assert d.max() < 1e-12


def test_adjoint_cutoff_mode_1_matches_oracle(env):
    """The lubrication range delta_lub a0 (cutoff mode 1) with the taper:
    its parameter derivative goes through a0 instead of the mean radius."""
    g, u0, w0, kw, th = _case(env, 0.3)
    kw = dict(kw, lub_cutoff_mode=1)
    th = dict(th, delta_lub=0.3)
    T = 10
    W = _weights(T, kw["shear_rate"])
    o = env["oadj"].gradients(g["box"], g["x"], g["a"], u0, w0, T, W, **th, **kw, nstep0=3)
    r, _ = _gpu(env, g, u0, w0, kw, th, T, W)
    assert r["J"] == pytest.approx(o["J"], rel=1e-11)
    check_scalars(r["params"], o["params"], 1e-8, floor=1e-6, what="dJ/dtheta")
    check_per_particle(r["x0"], o["x0"], 1e-8, what="dJ/dx0")
    check_per_particle(r["u0"], o["u0"], 1e-8, what="dJ/du0")
    check_per_particle(r["w0"], o["w0"], 1e-8, what="dJ/dw0")


def test_adjoint_wave_rolling_mixed_vs_oracle(env):
    """Mixed-precision forward (FP64 reverse) with the wave and rolling."""
    g, u0, w0, kw, th = _case(env, 0.3)
    kw = dict(kw, wave_amp=4.0, wave_n=1, k_r=1e3)
    T = 12
    W = _weights(T, kw["shear_rate"])
    o = env["oadj"].gradients(g["box"], g["x"], g["a"], u0, w0, T, W, **th, **kw, nstep0=3)
    r, _ = _gpu(env, g, u0, w0, kw, th, T, W, precision="mixed")
    assert r["J"] == pytest.approx(o["J"], rel=1e-6)
    for k in range(5):
        assert r["params"][k] == pytest.approx(o["params"][k], rel=1e-4, abs=1e-9 * abs(o["J"]))
    check_per_particle(r["x0"], o["x0"], 1e-4, floor=0.1, what="dJ/dx0 (mixed)")


def test_autograd_function_and_tied_parameters(env):
    torch = env["torch"]
    dss = env["dss"]
    g, u0, w0, kw, th = _case(env, 0.3)
    T = 8
    W = dss.viscosity_weights(T, shear_rate=kw["shear_rate"])
    x0 = torch.tensor(g["x"], requires_grad=True)
    kn = torch.tensor(th["kn"], dtype=torch.float64, requires_grad=True)
    mu = torch.tensor(th["mu"], dtype=torch.float64, requires_grad=True)
    # k_t = k_n / 2 tied: the total derivative flows through both slots
    theta = torch.stack([kn, 0.5 * kn, torch.tensor(th["gamma_n"], dtype=torch.float64), mu,
                         torch.tensor(th["delta_lub"], dtype=torch.float64)])
    J = dss.rollout_stress(x0, theta, g["a"], g["box"], u0, w0, T, W, ckpt_every=4, **kw)
    J.backward()
    th2 = dict(th, kt=0.5 * th["kn"])
    o = env["oadj"].gradients(g["box"], g["x"], g["a"], u0, w0, T, W, **th2, **kw)
    assert J.item() == pytest.approx(o["J"], rel=1e-11)
    assert float(kn.grad) == pytest.approx(o["params"][0] + 0.5 * o["params"][1], rel=1e-7)
    assert float(mu.grad) == pytest.approx(o["params"][3], rel=1e-7)
    check_per_particle(x0.grad.numpy(), o["x0"], 1e-8, what="dJ/dx0")


def test_adjoint_20k_rollout_vs_central_differences(env):
    """The differentiable-rollout workload: 20,000 bidisperse spheres at
    volume fraction 0.54, mu = 0.5, 200 steps with a checkpoint every 20;
    time-averaged relative viscosity.  FP64 gradients against central
    differences of the GPU forward (FP64) for mu, k_n and delta_lub (taper on),
    and along random directions of the initial positions."""
    dss = env["dss"]
    synth = env["synth"]
    g = synth.generate(synth.SPECS["c5"])
    box = g["box"]
    T = 200
    kw = dict(shear_rate=1.0, dt=1e-4, lub_taper=0.2)
    th = dict(kn=1e4, kt=5e3, gamma_n=1e-3, mu=0.5, delta_lub=0.1)
    W = dss.viscosity_weights(T, shear_rate=1.0)
    n = g["a"].shape[0]
    u0 = np.zeros((3, n))
    u0[0] = g["x"][1]
    w0 = np.zeros((3, n))
    w0[2] = -0.5

    def make(th_, x=None):
        p = dss.default_params(box, precision="fp64", **th_, **kw)
        return dss.Suspension(g["x"] if x is None else x, g["a"], box, p, ids=g["ids"], u=u0, w=w0)

    s = make(th)
    r = s.adjoint(T, W, ckpt_every=20)
    s.close()

    def J(th_, x=None):
        s2 = make(th_, x)
        v = s2.rollout_objective(T, W)
        s2.close()
        return v

    for k, name, rel in ((3, "mu", 1e-3), (0, "kn", 1e-3), (4, "delta_lub", 1e-3)):
        h = rel * th[name]
        fd = (J(dict(th, **{name: th[name] + h})) - J(dict(th, **{name: th[name] - h}))) / (2 * h)
        assert r["params"][k] == pytest.approx(fd, rel=1e-4, abs=1e-6 * abs(fd) + 1e-12), name
    # initial positions: directions that move 20 particles.  A perturbed
    # trajectory can cross a cell boundary a step earlier or later, which
    # reorders force sums; the dense packing amplifies those last-bit changes
    # over 200 steps into FD noise.  The noise is estimated from the spread of
    # the difference quotient over two steps and allowed for on top of 1e-4.
    for seed in (3, 4):
        rng = np.random.default_rng(seed)
        v = np.zeros((3, n))
        idx = rng.choice(n, 20, replace=False)
        v[:, idx] = rng.normal(size=(3, 20))
        fds = []
        for h in (1e-7, 2e-7):
            fds.append((J(th, np.mod(g["x"] + h * v, box[:, None]))
                        - J(th, np.mod(g["x"] - h * v, box[:, None]))) / (2 * h))
        noise = abs(fds[0] - fds[1])
        ad = float((r["x0"] * v).sum())
        assert noise < 1e-2 * abs(fds[0])
        assert abs(ad - fds[0]) <= 1e-4 * abs(fds[0]) + 2.0 * noise


def test_adjoint_20k_rollout_mixed_vs_central_differences(env):
    """The differentiable-rollout workload in the precision the benchmark
    runs it in: 20,000 spheres, 200 steps, checkpoint every 20, FP32 pair
    forces with FP64 state (the reverse sweep in FP64 on the taped mixed
    forward).  (1) Its parameter gradients and directional derivatives along
    the initial positions equal the FP64 adjoint's of the same rollout (which
    test_adjoint_20k_rollout_vs_central_differences pins to central
    differences) within 1e-4.  (2) Against central differences of the mixed
    forward itself, at the largest step (1e-3 .. 1e-5 of the parameter) whose
    two sides have the same event set (pairs and contacts of every step):
    within 1e-4 plus the spread of the difference quotient over two steps
    (the FP32 rounding of the forward)."""
    dss = env["dss"]
    synth = env["synth"]
    g = synth.generate(synth.SPECS["c5"])
    box = g["box"]
    T = 200
    kw = dict(shear_rate=1.0, dt=1e-4, lub_taper=0.2)
    th = dict(kn=1e4, kt=5e3, gamma_n=1e-3, mu=0.5, delta_lub=0.1)
    W = dss.viscosity_weights(T, shear_rate=1.0)
    n = g["a"].shape[0]
    u0 = np.zeros((3, n))
    u0[0] = g["x"][1]
    w0 = np.zeros((3, n))
    w0[2] = -0.5

    def make(th_, precision="mixed"):
        p = dss.default_params(box, precision=precision, **th_, **kw)
        return dss.Suspension(g["x"], g["a"], box, p, ids=g["ids"], u=u0, w=w0)

    grads = {}
    for prec in ("mixed", "fp64"):
        s = make(th, prec)
        grads[prec] = s.adjoint(T, W, ckpt_every=20)
        s.close()
    rm, rf = grads["mixed"], grads["fp64"]
    for k, name in ((3, "mu"), (0, "kn"), (4, "delta_lub")):
        assert rm["params"][k] == pytest.approx(rf["params"][k], rel=1e-4), name
    rng = np.random.default_rng(7)
    for _ in range(2):
        v = rng.normal(size=(3, n))
        assert float((rm["x0"] * v).sum()) == pytest.approx(float((rf["x0"] * v).sum()), rel=1e-4)

    def J(th_):
        s2 = make(th_)
        val, events = 0.0, []
        for k in range(T):
            s2.step(1)
            val += float((W[k] * s2.stress().reshape(9)).sum())
            c = s2.counters()
            events.append((c["npairs"], c["ncontacts"]))
        s2.close()
        return val, events

    _, ev0 = J(th)
    checked = 0
    for k, name in ((3, "mu"), (0, "kn"), (4, "delta_lub")):
        for rel in (1e-3, 1e-4, 1e-5):
            fds, same = [], True
            for hh in (rel, 2 * rel):
                h = hh * th[name]
                jp, evp = J(dict(th, **{name: th[name] + h}))
                jm, evm = J(dict(th, **{name: th[name] - h}))
                same = same and evp == ev0 and evm == ev0
                fds.append((jp - jm) / (2 * h))
            if not same:
                continue
            noise = abs(fds[0] - fds[1])
            assert abs(rm["params"][k] - fds[0]) <= 1e-4 * abs(fds[0]) + 2.0 * noise, (name, rel, rm["params"][k], fds)
            checked += 1
            break
    assert checked >= 1
