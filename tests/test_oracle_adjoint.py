"""Pins of the adjoint oracle (oracle/adjoint.py): its forward rollout must
repeat oracle.c step for step, and its reverse-mode gradient must match
central finite differences of oracle.c, with the event set (pair set,
contacts, Coulomb slips) checked unchanged between the two sides of each
difference.  One case adds the electro-chemical forces of Eq. 6-7 (the
list then reaches their range and lubrication keeps its own), one the wavy
shear flow of Eq. 17 with rolling resistance (App. B).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import adjoint
from paper_2108_01013_gb300 import synth


ECHEM = dict(f_er=30.0, lambda_d=0.05, hamaker=0.01, vdw_eps=0.05)
WAVE_ROLL = dict(wave_amp=4.0, wave_n=1, k_r=1e3)
EXTRA = tuple(ECHEM) + tuple(WAVE_ROLL)


def _case(taper, echem=False):
    g = synth.small(260, 0.52, 61)
    n = g["a"].shape[0]
    rng = np.random.default_rng(5)
    u0 = np.zeros((3, n))
    u0[0] = 5.0 * g["x"][1]
    u0 += 0.5 * rng.normal(size=(3, n))
    w0 = 0.5 * rng.normal(size=(3, n))
    kw = dict(shear_rate=5.0, dt=1e-4, lub_taper=taper, nstep0=3)
    if echem == "wave_roll":
        kw.update(WAVE_ROLL)
    elif echem:
        kw.update(ECHEM)
    th = dict(kn=1e4, kt=6e3, gamma_n=0.5, mu=0.4, delta_lub=0.2 if taper else 0.05)
    return g, u0, w0, kw, th


def _c_oracle(g, u0, w0, kw, th, nsteps, weights, x0=None):
    p = oracle.make_params(g["box"], kn=th["kn"], kt=th["kt"], gamma_n=th["gamma_n"], mu=th["mu"],
                           delta_lub=th["delta_lub"], shear_rate=kw["shear_rate"], dt=kw["dt"],
                           lub_taper=kw["lub_taper"], **{k: kw[k] for k in EXTRA if k in kw})
    o = oracle.System(p, g["x"] if x0 is None else x0, g["a"], u=u0, w=w0, nstep=kw["nstep0"])
    o.init_accel()
    J, sig, ev = 0.0, [], []
    for k in range(nsteps):
        o.step(1)
        s = o.get_forces()[2].reshape(9)
        sig.append(s)
        ev.append((o.npairs, o.ncontacts))
        J += float((weights[k] * s).sum())
    return J, np.array(sig), ev, o


def _weights(nsteps, gd):
    W = np.zeros((nsteps, 9))
    W[:, 1] = 1.0 / (nsteps * gd)          # time-averaged relative viscosity (eta0 = 1)
    W[:, 3] = 0.25 / (nsteps * gd)
    W[:, 0] = 0.1 / nsteps                 # and a normal-stress term
    return W


@pytest.mark.parametrize("taper,echem", [(0.0, False), (0.3, False), (0.3, True), (0.3, "wave_roll")])
def test_torch_rollout_repeats_c_oracle(taper, echem):
    g, u0, w0, kw, th = _case(taper, echem)
    T = 15
    W = _weights(T, kw["shear_rate"])
    r = adjoint.gradients(g["box"], g["x"], g["a"], u0, w0, T, W, **th, **kw)
    J, sig, ev, o = _c_oracle(g, u0, w0, kw, th, T, W)
    st = o.get_state()
    box = g["box"]
    d = np.abs(r["final"]["x"] - st["x"])
    d = np.minimum(d, box[:, None] - d)
    assert d.max() < 1e-12
    for k in ("u", "w", "al", "aw"):
        np.testing.assert_allclose(r["final"][k], st[k], rtol=1e-9, atol=1e-10 * np.abs(st[k]).max())
    np.testing.assert_allclose(r["sigma"], sig, rtol=1e-9, atol=1e-11 * np.abs(sig).max())
    assert r["J"] == pytest.approx(J, rel=1e-10)
    assert [e[:2] for e in r["events"][1:]] == ev
    assert sum(e[1] for e in ev) > 50 and sum(e[2] for e in r["events"]) > 0   # contacts and slips


def _fd(g, u0, w0, kw, th, T, W, key, h, x0=None, du=None, dw=None):
    out = []
    for sgn in (1.0, -1.0):
        t2 = dict(th)
        x2, u2, w2 = g["x"], u0, w0
        if key in t2:
            t2[key] = th[key] + sgn * h
        if x0 is not None:
            x2 = g["x"] + sgn * h * x0
        if du is not None:
            u2 = u0 + sgn * h * du
        if dw is not None:
            w2 = w0 + sgn * h * dw
        J, _, ev, _ = _c_oracle(g, u2, w2, kw, t2, T, W, x0=x2)
        tk = {k: v for k, v in t2.items()}
        r = adjoint.Model(g["box"], g["a"], **kw)
        th_t = {k: torch.tensor(v, dtype=torch.float64) for k, v in
                (("kn", tk["kn"]), ("kt", tk["kt"]), ("gn", tk["gamma_n"]), ("mu", tk["mu"]),
                 ("delta", tk["delta_lub"]))}
        with torch.no_grad():
            _, _, evt, _ = r.rollout(torch.tensor(x2), torch.tensor(u2), torch.tensor(w2), th_t, T, None)
        out.append((J, evt))
    (Jp, ep), (Jm, em) = out
    assert ep == em, "event set changed across the difference"
    return (Jp - Jm) / (2 * h)


@pytest.mark.parametrize("taper,echem", [(0.0, False), (0.3, False), (0.3, True), (0.3, "wave_roll")])
def test_gradient_matches_central_differences(taper, echem):
    g, u0, w0, kw, th = _case(taper, echem)
    T = 12
    W = _weights(T, kw["shear_rate"])
    r = adjoint.gradients(g["box"], g["x"], g["a"], u0, w0, T, W, **th, **kw)
    names = ["kn", "kt", "gamma_n", "mu", "delta_lub"]
    for k, name in enumerate(names):
        if name == "delta_lub" and taper == 0.0:
            assert r["params"][k] == 0.0        # hard cutoff: no pathwise dependence
            continue
        # the largest relative step that leaves the event set unchanged
        for rel in (1e-4, 3e-5, 1e-5, 3e-6):
            try:
                fd = _fd(g, u0, w0, kw, th, T, W, name, rel * th[name])
                break
            except AssertionError:
                continue
        else:
            pytest.fail("no step keeps the event set: " + name)
        assert r["params"][k] == pytest.approx(fd, rel=2e-5, abs=1e-9 * abs(r["J"])), name
    rng = np.random.default_rng(9)
    for _ in range(2):
        # the packing holds contacts within ~1e-7 of touching: take the
        # largest step that leaves the event set unchanged
        v = rng.normal(size=g["x"].shape)
        for h in (1e-7, 3e-8, 1e-8, 3e-9):
            try:
                fd = _fd(g, u0, w0, kw, th, T, W, "x", h, x0=v)
                break
            except AssertionError:
                continue
        else:
            pytest.fail("no step keeps the event set")
        assert float((r["x0"] * v).sum()) == pytest.approx(fd, rel=2e-5)
    v = rng.normal(size=g["x"].shape)
    fd = _fd(g, u0, w0, kw, th, T, W, "u", 1e-5, du=v)
    assert float((r["u0"] * v).sum()) == pytest.approx(fd, rel=2e-5)
    fd = _fd(g, u0, w0, kw, th, T, W, "w", 1e-5, dw=v)
    assert float((r["w0"] * v).sum()) == pytest.approx(fd, rel=2e-5)
