"""Neighbour search over crowded cells (Sec. II A with cells of edge
2 a_max + delta holding many small particles): the enumeration must give the
brute-force pair set bit for bit over cells of ~6 and ~56 particles (several
hundred candidates per half stencil), with pairs across the Lees-Edwards
layer, and forces built on those rows.
"""
import numpy as np
import pytest

from parity import FP64_TOL, KAPPA_FP64, MIXED_TOL, KAPPA_MIXED, check_forces, check_stress

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
    return dict(oracle=oracle, dss=dss, synth=synth)


@pytest.fixture(scope="module")
def poly(env):
    """20k spheres, radii log-uniform in [1, 6]: ~5.5 per cell."""
    spec = env["synth"].Spec("crowded_poly", 20000, 0.50, radii="loguniform", a_min=1.0, a_max=6.0, seed=31)
    return env["synth"].generate(spec)


@pytest.fixture(scope="module")
def dilute_giants(env):
    """30k spheres, 1% of radius 10 among radius 1: ~56 per cell, several
    hundred candidates per half stencil."""
    spec = env["synth"].Spec("crowded_giants", 30000, 0.30, a_small=1.0, a_large=10.0, frac_large=0.01,
                             seed=32)
    return env["synth"].generate(spec)


def _crowded(s, n):
    c = s.counters()
    cells = int(np.prod(c["ncell"]))
    assert n >= 4 * cells, (n, c["ncell"])
    return c


@pytest.mark.parametrize("which", ["poly", "dilute_giants"])
def test_crowded_pairs_bit_exact(env, which, request):
    g = request.getfixturevalue(which)
    n = g["a"].shape[0]
    box = g["box"]
    x = g["x"].copy()
    # a layer of particles at y = 0 and y = L_y for the shifted image rows
    rng = np.random.default_rng(5)
    k = rng.choice(n, size=n // 20, replace=False)
    x[1, k[: len(k) // 2]] = rng.uniform(0, 1.5, size=len(k) // 2)
    x[1, k[len(k) // 2:]] = box[1] - rng.uniform(1e-9, 1.5, size=len(k) - len(k) // 2)
    dss, orc = env["dss"], env["oracle"]
    p = dss.default_params(box, shear_rate=0.9, dt=1e-2)
    po = orc.make_params(box, shear_rate=0.9, dt=1e-2)
    for nstep in (0, 333, 4321):
        s = dss.Suspension(x, g["a"], box, p, ids=g["ids"], nstep=nstep,
                           alpha_lin=np.zeros_like(x), alpha_ang=np.zeros_like(x))
        s.neighbour_build()
        c = _crowded(s, n)
        o = orc.System(po, x, g["a"], ids=g["ids"], nstep=nstep)
        want = o.pairs_cell()
        assert want is not None and len(want) > n // 20
        got = s.pairs()
        np.testing.assert_array_equal(got, want)
        assert c["npairs"] == len(want)
        s.close()


@pytest.mark.parametrize("precision,tol,kappa", [("fp64", FP64_TOL, KAPPA_FP64), ("mixed", MIXED_TOL, KAPPA_MIXED)])
def test_crowded_forces_vs_oracle(env, poly, precision, tol, kappa):
    """Forces and torques of every particle on rows from the crowded-cell
    search (per-particle bound of tests/parity.py)."""
    g = poly
    n = g["a"].shape[0]
    box = g["box"]
    rng = np.random.default_rng(8)
    u = np.zeros((3, n))
    u[0] = 0.7 * g["x"][1]
    u += 0.05 * rng.normal(size=(3, n))
    w = 0.05 * rng.normal(size=(3, n))
    w[2] -= 0.35
    dss, orc = env["dss"], env["oracle"]
    p = dss.default_params(box, precision=precision, mu=0.5, shear_rate=0.7, dt=1e-4)
    po = orc.make_params(box, mu=0.5, shear_rate=0.7, dt=1e-4)
    s = dss.Suspension(g["x"], g["a"], box, p, ids=g["ids"], u=u, w=w, nstep=777,
                       alpha_lin=np.zeros((3, n)), alpha_ang=np.zeros((3, n)))
    F, T = s.forces()
    S = s.stress()
    _crowded(s, n)
    o = orc.System(po, g["x"], g["a"], ids=g["ids"], u=u, w=w, nstep=777, cells=True)
    Fo, To, So = o.forces()
    Fa, Ta = o.force_scale()
    assert o.ncontacts > 100
    check_forces(F.cpu().numpy(), Fo, Fa, tol, kappa, "crowded %s force" % precision)
    check_forces(T.cpu().numpy(), To, Ta, tol, kappa, "crowded %s torque" % precision)
    check_stress(S, So, tol)
    c = s.counters()
    assert c["npairs"] == o.npairs and c["ncontacts"] == o.ncontacts
    s.close()
