"""Mixed-precision mode (FP32 pair arithmetic; FP64 positions, gaps,
Lees-Edwards offset, tangential stretch and stress accumulation) against the
FP64 oracle: forces, torques and stress within 1e-5 relative (normwise over
the particles) from the same state, and per-step accelerations within 1e-5."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-5


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
    return dict(oracle=oracle, dss=dss, synth=synth)


def relerr(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def _state_with_history(env, n, phi, seed, gdot, mu, steps):
    g = env["synth"].small(n, phi, seed)
    po = env["oracle"].make_params(g["box"], mu=mu, shear_rate=gdot)
    o = env["oracle"].System(po, g["x"], g["a"], ids=g["ids"])
    o.init_accel()
    o.step(steps)
    return g, po, o


@pytest.mark.parametrize("n,phi,seed,gdot,mu", [(1000, 0.50, 1, 1.0, 0.5), (2000, 0.55, 2, 30.0, 1.0)])
def test_mixed_forces_and_stress(env, n, phi, seed, gdot, mu):
    g, po, o = _state_with_history(env, n, phi, seed, gdot, mu, 30)
    st = o.get_state()
    keys, xi = o.get_history()
    p = env["dss"].default_params(g["box"], mu=mu, shear_rate=gdot, precision="mixed")
    s = env["dss"].Suspension(st["x"], g["a"], g["box"], p, ids=g["ids"], u=st["u"], w=st["w"],
                              alpha_lin=st["al"], alpha_ang=st["aw"], nstep=o.nstep)
    s.set_history(keys, xi)
    F, T = s.forces()
    Fo, To, So = o.forces()
    assert o.ncontacts > 20
    assert relerr(F.cpu().numpy(), Fo) < MIXED_TOL
    assert relerr(T.cpu().numpy(), To) < MIXED_TOL
    assert relerr(s.stress(), So) < MIXED_TOL
    s.close()


def test_mixed_one_step_accelerations(env):
    g, po, o = _state_with_history(env, 1500, 0.52, 5, 10.0, 1.0, 25)
    st = o.get_state()
    keys, xi = o.get_history()
    p = env["dss"].default_params(g["box"], mu=1.0, shear_rate=10.0, precision="mixed")
    s = env["dss"].Suspension(st["x"], g["a"], g["box"], p, ids=g["ids"], u=st["u"], w=st["w"],
                              alpha_lin=st["al"], alpha_ang=st["aw"], nstep=o.nstep)
    s.set_history(keys, xi)
    s.step(1)
    o.step(1)
    sg = s.state()
    so = o.get_state()
    assert relerr(sg["al"].cpu().numpy(), so["al"]) < MIXED_TOL
    assert relerr(sg["aw"].cpu().numpy(), so["aw"]) < MIXED_TOL
    assert relerr(sg["u"].cpu().numpy() - st["u"], so["u"] - st["u"]) < MIXED_TOL
    assert relerr(s.stress(), o.get_forces()[2]) < MIXED_TOL
    k1, x1 = s.history()
    k2, x2 = o.get_history()
    np.testing.assert_array_equal(k1, k2)
    assert relerr(x1, x2) < MIXED_TOL
    s.close()


def test_mixed_trajectory_stays_close(env):
    """100 steps of the 1000-particle configuration: the mixed trajectory
    stays within 1e-6 of the FP64 oracle in position (relative to a radius)."""
    synth = env["synth"]
    g = synth.generate(synth.SPECS["c1"])
    box = g["box"]
    p = env["dss"].default_params(box, mu=0.5, precision="mixed")
    po = env["oracle"].make_params(box, mu=0.5)
    s = env["dss"].Suspension(g["x"], g["a"], box, p, ids=g["ids"])
    o = env["oracle"].System(po, g["x"], g["a"], ids=g["ids"])
    o.init_accel()
    s.step(100)
    o.step(100)
    x = s.state()["x"].cpu().numpy()
    d = np.abs(x - o.get_state()["x"])
    d = np.minimum(d, box[:, None] - d)
    assert d.max() < 1e-6
    assert relerr(s.stress(), o.get_forces()[2]) < 1e-4
    s.close()
