"""Size-class cell lists (cell_mode 1; Sec. II A: cells smaller than
2 a_max, larger stencils for larger particles) on polydisperse packings:
pair sets bit-exact against brute force (Lees-Edwards offsets, both cutoff
modes, several cell edges), forces and stress against the FP64 oracle with
contact history, and trajectories equal to the one-list mode within
rounding."""
import numpy as np
import pytest

from parity import FP64_TOL, check_forces, check_per_particle, check_stress, kappa_for

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
    g = synth.small(3000, 0.50, 81, radii="loguniform", a_min=1.0, a_max=6.0, max_iter=300)
    return dict(oracle=oracle, dss=dss, synth=synth, torch=torch, g=g)


@pytest.mark.parametrize("cell_size,nstep,mode,delta", [(0.0, 0, 0, 0.05), (0.0, 7777, 0, 0.05),
                                                        (2.2, 123, 0, 0.05), (5.0, 31, 0, 0.2),
                                                        (0.0, 999, 1, 0.1), (4.0, 4321, 1, 0.3)])
def test_class_pairs_bit_exact(env, cell_size, nstep, mode, delta):
    g = env["g"]
    box = g["box"]
    n = g["a"].shape[0]
    kw = dict(lub_cutoff_mode=mode, delta_lub=delta, shear_rate=2.7, dt=1e-3)
    p = env["dss"].default_params(box, cell_mode=1, cell_size=cell_size, **kw)
    s = env["dss"].Suspension(g["x"], g["a"], box, p, ids=g["ids"], nstep=nstep,
                              alpha_lin=np.zeros((3, n)), alpha_ang=np.zeros((3, n)))
    s.neighbour_build()
    got = s.pairs()
    po = env["oracle"].make_params(box, **kw)
    want = env["oracle"].pairs_bruteforce(g["x"], g["a"], g["ids"], po, env["oracle"].le_offset(po, nstep))
    assert len(want) > n // 2
    np.testing.assert_array_equal(got, want)
    c = s.counters()
    assert c["npairs"] == len(want)
    assert c["ncell"][0] > 12          # cells well below 2 a_max + delta
    s.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_class_forces_with_history_vs_oracle(env, precision, tol):
    g = env["g"]
    box = g["box"]
    kw = dict(mu=1.0, shear_rate=4.0)
    po = env["oracle"].make_params(box, **kw)
    o = env["oracle"].System(po, g["x"], g["a"], ids=g["ids"])
    o.init_accel()
    o.step(15)
    st = o.get_state()
    keys, xi = o.get_history()
    p = env["dss"].default_params(box, precision=precision, cell_mode=1, **kw)
    s = env["dss"].Suspension(st["x"], g["a"], box, p, ids=g["ids"], u=st["u"], w=st["w"],
                              alpha_lin=st["al"], alpha_ang=st["aw"], nstep=o.nstep)
    s.set_history(keys, xi)
    F, T = s.forces()
    Fo, To, So = o.forces()
    Fa, Ta = o.force_scale()
    assert o.ncontacts > 100
    check_forces(F.cpu().numpy(), Fo, Fa, tol, kappa_for(tol), "force")
    check_forces(T.cpu().numpy(), To, Ta, tol, kappa_for(tol), "torque")
    check_stress(s.stress(), So, tol)
    s.step(3)
    o.step(3)
    d = np.abs(s.state()["x"].cpu().numpy() - o.get_state()["x"])
    d = np.minimum(d, box[:, None] - d)
    assert d.max() < (1e-12 if precision == "fp64" else 1e-8)
    k1, x1 = s.history()
    k2, x2 = o.get_history()
    np.testing.assert_array_equal(k1, k2)
    s.close()


def test_class_mode_matches_one_list_mode(env):
    g = env["g"]
    box = g["box"]
    runs = []
    for mode in (0, 1):
        p = env["dss"].default_params(box, cell_mode=mode, mu=0.5, shear_rate=3.0)
        s = env["dss"].Suspension(g["x"], g["a"], box, p, ids=g["ids"])
        s.step(30)
        runs.append((s.state()["x"].cpu().numpy(), s.stress(), s.history()))
        s.close()
    d = np.abs(runs[0][0] - runs[1][0])
    d = np.minimum(d, box[:, None] - d)
    assert d.max() < 1e-11
    check_stress(runs[1][1], runs[0][1], FP64_TOL)
    np.testing.assert_array_equal(runs[0][2][0], runs[1][2][0])
