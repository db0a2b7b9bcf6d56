"""The oracle's cell-list neighbour search (Sec. II A: counting sort into cells
of edge >= the largest pair range, symmetric half stencil, the shifted x cells
across the Lees-Edwards boundary) against its brute-force definition, and the
per-particle scale of the force sums (the sum of the magnitudes of the
terms).  CPU only."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def synth():
    from paper_2108_01013_gb300 import synth
    synth.build()
    return synth


@pytest.mark.parametrize("n,phi,seed,kw", [
    (2000, 0.50, 1, {}),
    (3000, 0.45, 2, dict(lub_cutoff_mode=1, delta_lub=0.2)),
    (1500, 0.50, 3, dict(f_er=1.0, lambda_d=0.05, hamaker=1e-4)),
    (20000, 0.54, 5, {}),
])
def test_cell_pairs_equal_brute_force(orc, synth, n, phi, seed, kw):
    g = synth.small(n, phi, seed)
    po = orc.make_params(g["box"], mu=0.5, shear_rate=1.3, dt=1e-3, **kw)
    for nstep in (0, 777, 123456):
        o = orc.System(po, g["x"], g["a"], ids=g["ids"], nstep=nstep)
        got = o.pairs_cell()
        assert got is not None
        want = orc.pairs_bruteforce(g["x"], g["a"], g["ids"], po, orc.le_offset(po, nstep))
        assert len(want) > n // 2
        np.testing.assert_array_equal(got, want)


def test_cell_pairs_polydisperse_boundary_layer(orc, synth):
    """Radii log-uniform in [1, 3], a third of the particles pushed into the
    layers at y = 0 and y = L_y, offsets across a full period of the shift."""
    rng = np.random.default_rng(9)
    spec = synth.Spec("poly", 1500, 0.45, radii="loguniform", a_min=1.0, a_max=3.0, seed=21)
    g = synth.generate(spec)
    box = g["box"]
    x = g["x"].copy()
    k = rng.choice(g["a"].shape[0], size=500, replace=False)
    x[1, k[:250]] = rng.uniform(0, 2.0, size=250)
    x[1, k[250:]] = box[1] - rng.uniform(1e-9, 2.0, size=250)
    po = orc.make_params(box, shear_rate=0.9, dt=1e-2)
    for nstep in range(0, 12000, 997):
        o = orc.System(po, x, g["a"], ids=g["ids"], nstep=nstep)
        want = orc.pairs_bruteforce(x, g["a"], g["ids"], po, orc.le_offset(po, nstep))
        np.testing.assert_array_equal(o.pairs_cell(), want)


def test_cell_pairs_near_cutoff(orc):
    """Pairs within a few ulps of the cutoff on both sides."""
    rng = np.random.default_rng(4)
    box = np.array([30.0, 30.0, 30.0])
    pts, rad = [], []
    for t in range(60):
        c = rng.uniform(3, 27, size=3)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        ai, aj = (1.0, 1.4) if t % 2 else (1.4, 1.4)
        s = (ai + aj) * (1 + 0.05 / 2)
        r = s * (1 + rng.choice([-1, 1]) * rng.uniform(0, 4e-16))
        pts += [c, c + r * u]
        rad += [ai, aj]
    x = np.mod(np.array(pts).T.copy(), box[:, None])
    a = np.array(rad)
    ids = np.arange(a.shape[0], dtype=np.int32)
    po = orc.make_params(box, shear_rate=0.0)
    o = orc.System(po, x, a, ids=ids)
    np.testing.assert_array_equal(o.pairs_cell(), orc.pairs_bruteforce(x, a, ids, po, 0.0))


def test_cell_search_gives_the_same_trajectory(orc, synth):
    """Same pair set in the same order: forces, stress, history and a
    40-step trajectory bit for bit."""
    g = synth.small(3000, 0.52, 5)
    po = orc.make_params(g["box"], mu=0.5, shear_rate=3.0)
    a = orc.System(po, g["x"], g["a"], ids=g["ids"])
    b = orc.System(po, g["x"], g["a"], ids=g["ids"], cells=True)
    a.init_accel()
    b.init_accel()
    a.step(40)
    b.step(40)
    sa, sb = a.get_state(), b.get_state()
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k
    for u, v in zip(a.get_forces(), b.get_forces()):
        assert np.array_equal(u, v)
    for u, v in zip(a.get_history(), b.get_history()):
        assert np.array_equal(u, v)
    assert a.ncontacts > 50 and a.npairs == b.npairs


def test_cell_search_falls_back_on_small_boxes(orc, synth):
    """A box with fewer than 3 cells per axis has no cell list (pairs_cell is
    None) and the cell mode evaluates by brute force."""
    g = synth.small(60, 0.45, 7)
    po = orc.make_params(g["box"], mu=0.5)
    o = orc.System(po, g["x"], g["a"], ids=g["ids"], cells=True)
    assert o.pairs_cell() is None
    F, T, S = o.forces()
    b = orc.System(po, g["x"], g["a"], ids=g["ids"])
    F2, T2, S2 = b.forces()
    assert np.array_equal(F, F2) and np.array_equal(S, S2)


def test_force_scale_is_the_sum_of_the_term_magnitudes(orc):
    """The per-particle scale of the force sums: an isolated sphere, the
    drag alone; two overlapping spheres at rest without shear, the contact
    spring alone (no velocity, no strain: every lubrication sub-term is
    zero); two equal spheres 0.002 apart moving together along their line
    of centres, lubrication sub-terms that cancel (no net pair force) but
    count in the scale; any system, at least the magnitude of the sum."""
    box = np.array([40.0, 40.0, 40.0])
    po = orc.make_params(box, mu=0.5, shear_rate=0.0)
    x = np.array([[10.0, 12.3, 30.0], [20.0, 20.0, 5.0], [20.0, 20.0, 20.0]])
    a = np.array([1.0, 1.4, 1.2])
    zero = np.zeros((3, 3))
    o = orc.System(po, x, a, u=zero, w=zero)
    F, T, _ = o.forces()
    Fa, Ta = o.force_scale()
    assert Fa[2] == 0.0 and Ta[2] == 0.0
    # overlap 0.1: spring force kn * 0.1 on each, nothing else
    for k in (0, 1):
        assert np.linalg.norm(F[:, k]) == pytest.approx(1e4 * 0.1, rel=1e-12)
        assert Fa[k] == pytest.approx(np.linalg.norm(F[:, k]), rel=1e-12)
    # a moving sphere alone: its drag
    u = np.zeros((3, 3))
    u[:, 2] = [0.3, -0.1, 0.2]
    o = orc.System(po, x, a, u=u, w=zero)
    F, T, _ = o.forces()
    Fa, _ = o.force_scale()
    assert Fa[2] == pytest.approx(np.linalg.norm(F[:, 2]), rel=1e-15)
    assert Fa[2] == pytest.approx(6 * np.pi * 1.2 * np.linalg.norm(u[:, 2]), rel=1e-12)
    # two equal spheres 0.002 apart moving together along x: squeeze terms cancel
    x2 = np.array([[10.0, 12.002], [20.0, 20.0], [20.0, 20.0]])
    a2 = np.array([1.0, 1.0])
    u2 = np.array([[0.5, 0.5], [0.0, 0.0], [0.0, 0.0]])
    o = orc.System(po, x2, a2, u=u2, w=np.zeros((3, 2)))
    F, T, _ = o.forces()
    Fa, _ = o.force_scale()
    drag = 6 * np.pi * 1.0 * 0.5
    for k in (0, 1):
        pair = F[:, k] + np.array([drag, 0.0, 0.0])
        assert np.linalg.norm(pair) < 1e-9 * Fa[k]
        assert Fa[k] - drag > 100.0 * drag
    # a packing: never below the magnitude of the sum
    from paper_2108_01013_gb300 import synth
    g = synth.small(800, 0.52, 3)
    po = orc.make_params(g["box"], mu=0.5, shear_rate=2.0)
    o = orc.System(po, g["x"], g["a"], ids=g["ids"])
    o.init_accel()
    o.step(5)
    F, T, _ = o.forces()
    Fa, Ta = o.force_scale()
    assert np.all(Fa >= np.linalg.norm(F, axis=0) * (1 - 1e-15))
    assert np.all(Ta >= np.linalg.norm(T, axis=0) * (1 - 1e-15))
