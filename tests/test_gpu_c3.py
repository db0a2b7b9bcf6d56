"""The 1,000,000-particle polydisperse workload (radii log-uniform in [1, 10],
volume fraction 0.50, mu = 0.5; list capacity M = 728 from the shell bound),
in the launch configuration the benchmark uses.  The oracle cannot do the
full O(N^2) problem, so it checks sampled outputs it computes one by one: the
complete neighbour set of sampled particles (bit-exact; the largest and the
smallest particles are always sampled) and the force and torque on them, at
the initial state and after steps with contact history, in FP64 and mixed
precision, with one cell list and with size classes."""
import numpy as np
import pytest

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
    g = synth.generate(synth.SPECS["c3"])
    return dict(oracle=oracle, dss=dss, synth=synth, g=g)


def _sample(g, m=48, seed=0):
    a = g["a"]
    order = np.argsort(a)
    rng = np.random.default_rng(seed)
    pick = np.concatenate([order[-8:], order[:8], rng.choice(a.shape[0], m - 16, replace=False)])
    return np.unique(pick)


def relerr(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


@pytest.mark.parametrize("precision,tol,cell_mode", [("fp64", 1e-10, 0), ("mixed", 1e-5, 0),
                                                    ("fp64", 1e-10, 1), ("mixed", 1e-5, 1)])
def test_c3_sampled_neighbours_and_forces(env, precision, tol, cell_mode):
    g, dss, oracle = env["g"], env["dss"], env["oracle"]
    box = g["box"]
    p = dss.default_params(box, precision=precision, mu=0.5, cell_mode=cell_mode)
    s = dss.Suspension(g["x"], g["a"], box, p, ids=g["ids"])
    assert s.counters()["M"] == 728
    s.step(5)
    st = {k: v.cpu().numpy() for k, v in s.state().items()}
    nstep = s.counters()["nstep"]
    keys, xi = s.history()
    assert len(keys) > 100_000
    # neighbour sets at the current state
    s.neighbour_build()
    pairs = s.pairs()
    po = oracle.make_params(box, mu=0.5)
    off = oracle.le_offset(po, nstep)
    idx = _sample(g)
    for k in idx:
        want = oracle.neighbours_of(st["x"], g["a"], g["ids"], po, off, int(k))
        got = np.sort(np.concatenate([pairs[pairs[:, 0] == k, 1], pairs[pairs[:, 1] == k, 0]]))
        np.testing.assert_array_equal(got, want)
    # forces and torques on the sample, with the carried history
    F, T = s.forces()
    F, T = F.cpu().numpy(), T.cpu().numpy()
    o = oracle.System(po, st["x"], g["a"], ids=g["ids"], u=st["u"], w=st["w"], nstep=nstep)
    o.set_history(keys, xi)
    Fo, To = o.forces_sampled(idx)
    assert relerr(F[:, idx], Fo) < tol
    assert relerr(T[:, idx], To) < tol
    big = idx[np.argsort(g["a"][idx])[-8:]]
    j = np.searchsorted(idx, big)
    assert relerr(F[:, big], Fo[:, j]) < tol
    s.close()
