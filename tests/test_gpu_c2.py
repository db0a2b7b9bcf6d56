"""The 100,000-particle bidisperse workload of the headline benchmark (radius
ratio 1 : 1.4, equal numbers, volume fraction 0.55, mu = 1.0), in the launch
configuration the benchmark times (mixed precision; FP64 as well).  The
oracle checks sampled outputs it computes one by one, on inputs made without
the CUDA path (the seeded packing, seeded velocities, a seeded stretch on the
contacts the oracle finds around the sample): the complete neighbour set of
200 sampled particles, bit-exact, at two Lees-Edwards offsets, and the force
and torque on each of them with that contact history (per particle,
tests/parity.py)."""
import numpy as np
import pytest

from fullsize_cases import contact_history, partners, sample, velocities
from parity import check_forces, check_stress, kappa_for

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
    spec = synth.SPECS["c2"]
    g = synth.generate(spec)
    box = g["box"]
    kw = dict(mu=spec.mu, kn=spec.kn, shear_rate=spec.shear_rate, dt=spec.dt)
    po = oracle.make_params(box, **kw)
    u, w = velocities(g["x"], g["a"], spec.shear_rate, seed=21)
    idx = sample(g["a"], m=200, seed=2)
    cases = {}
    for nstep in (0, 7_654_321):
        off = oracle.le_offset(po, nstep)
        keys, xi = contact_history(oracle, po, off, g["x"], g["a"], g["ids"], u, w, idx, seed=nstep % 89)
        o = oracle.System(po, g["x"], g["a"], ids=g["ids"], u=u, w=w, nstep=nstep)
        o.set_history(keys, xi)
        Fo, To, Fa, Ta = o.forces_sampled(idx, scale=True)
        want = {int(k): oracle.neighbours_of(g["x"], g["a"], g["ids"], po, off, int(k)) for k in idx}
        cases[nstep] = dict(keys=keys, xi=xi, Fo=Fo, To=To, Fa=Fa, Ta=Ta, want=want)
    return dict(oracle=oracle, po=po, dss=dss, g=g, kw=kw, u=u, w=w, idx=idx, cases=cases)


@pytest.mark.parametrize("precision,tol", [("mixed", 1e-5), ("fp64", 1e-10)])
def test_c2_sampled_neighbours_and_forces(env, precision, tol):
    g, dss = env["g"], env["dss"]
    box, idx = g["box"], env["idx"]
    n = g["a"].shape[0]
    p = dss.default_params(box, precision=precision, **env["kw"])
    for nstep, c in env["cases"].items():
        s = dss.Suspension(g["x"], g["a"], box, p, ids=g["ids"], u=env["u"], w=env["w"], nstep=nstep,
                           alpha_lin=np.zeros((3, n)), alpha_ang=np.zeros((3, n)))
        s.neighbour_build()
        pairs = s.pairs()
        assert len(pairs) > 200_000
        for k in idx:
            np.testing.assert_array_equal(partners(pairs, int(g["ids"][k])), c["want"][int(k)])
        assert len(c["keys"]) > 300
        s.set_history(c["keys"], c["xi"])
        F, T = s.forces()
        F, T = F.cpu().numpy(), T.cpu().numpy()
        check_forces(F[:, idx], c["Fo"], c["Fa"], tol, kappa_for(tol), "force")
        check_forces(T[:, idx], c["To"], c["Ta"], tol, kappa_for(tol), "torque")
        s.close()


@pytest.mark.parametrize("precision,tol", [("mixed", 1e-5), ("fp64", 1e-10)])
def test_c2_every_particle_and_the_stress(env, precision, tol):
    """All 100,000 particles and the bulk stress of Eq. 8 against the oracle's
    full evaluation (its cell-list search, checked equal to the brute force
    in tests/test_oracle_cells.py), with the seeded history of the second
    Lees-Edwards offset."""
    g, dss, oracle = env["g"], env["dss"], env["oracle"]
    box = g["box"]
    n = g["a"].shape[0]
    nstep = 7_654_321
    c = env["cases"][nstep]
    o = oracle.System(env["po"], g["x"], g["a"], ids=g["ids"], u=env["u"], w=env["w"], nstep=nstep,
                      cells=True)
    o.set_history(c["keys"], c["xi"])
    Fo, To, So = o.forces()
    Fa, Ta = o.force_scale()
    p = dss.default_params(box, precision=precision, **env["kw"])
    s = dss.Suspension(g["x"], g["a"], box, p, ids=g["ids"], u=env["u"], w=env["w"], nstep=nstep,
                       alpha_lin=np.zeros((3, n)), alpha_ang=np.zeros((3, n)))
    s.set_history(c["keys"], c["xi"])
    F, T = s.forces()
    check_forces(F.cpu().numpy(), Fo, Fa, tol, kappa_for(tol), "force")
    check_forces(T.cpu().numpy(), To, Ta, tol, kappa_for(tol), "torque")
    check_stress(s.stress(), So, tol)
    assert s.counters()["npairs"] == o.npairs
    s.close()
