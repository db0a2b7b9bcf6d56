"""Pins of the oracle's analysis pass (oracle/analysis.py and the image
count of oracle.c): checks against what the definitions and the physics fix.

- Rheology (Sec. II, after Eq. 9): a dilute sphere in shear gives the
  Einstein viscosity eta_r = 1 + 5 phi / 2 (golden coefficient) with no
  normal-stress differences and no pressure; a single repulsive contact
  along the compressional axis (1, -1, 0)/sqrt 2 has S = -c n (x) n, so
  N1 = 0, N2 = -sigma and Pi = 2 sigma / 3 (a transposed or shifted index
  breaks one of them).
- Clusters of contacting particles (Fig. 10-11): hand-built graphs with known
  components, and random graphs against scipy's connected components.
- Dispersion (Eq. 18-19): ballistic motion y = y0 + v t gives
  D_y = <v^2> t / (2 a0^2 gdot); unchanged velocities give C_v = 1, reversed
  ones -1; the image count keeps the unwrapped y continuous when a particle
  crosses y = L_y in either direction."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import analysis

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_rheology_of_a_dilute_sphere_is_einstein():
    g = json.load(open(os.path.join(GOLDEN, "einstein.json")))
    L, a, gd, eta0 = 40.0, 2.0, 0.6, 1.7
    p = oracle.make_params([L] * 3, shear_rate=gd, eta0=eta0)
    s = oracle.System(p, np.array([[3.0], [4.0], [5.0]]), [a])
    _, _, S = s.forces()
    r = analysis.rheology(S, gd, eta0)
    phi = 4 / 3 * math.pi * a ** 3 / L ** 3
    assert r["eta_r"] == pytest.approx(1 + g["coefficient"] * phi, rel=1e-13)
    assert abs(r["N1"]) < 1e-15 and abs(r["N2"]) < 1e-15 and abs(r["Pi"]) < 1e-15
    assert r["eta_n"] == pytest.approx(r["Pi"] / (eta0 * gd))


def test_rheology_of_a_compressional_contact():
    L = 30.0
    p = oracle.make_params([L] * 3, shear_rate=0.0, eta0=0.0, mu=0.0)
    n = np.array([1.0, -1.0, 0.0]) / math.sqrt(2.0)
    xi = np.array([10.0, 10.0, 10.0])
    xj = xi + n * (2.0 - 0.01)
    s = oracle.System(p, np.stack([xi, xj], axis=1), [1.0, 1.0])
    _, _, S = s.forces()
    r = analysis.rheology(S, 1.0, 1.0)
    assert r["sigma"] > 0
    assert abs(r["N1"]) <= 1e-12 * r["sigma"]
    assert r["N2"] == pytest.approx(-r["sigma"], rel=1e-12)
    assert r["Pi"] == pytest.approx(2.0 * r["sigma"] / 3.0, rel=1e-12)


def _keys(edges):
    return np.array([(min(a, b) << 32) | max(a, b) for a, b in edges], dtype=np.int64)


def test_clusters_of_hand_built_graphs():
    label, k = analysis.contact_clusters(7, _keys([(0, 3), (3, 5), (1, 2)]))
    np.testing.assert_array_equal(label, [0, 1, 1, 0, 4, 0, 6])
    assert k == 4
    np.testing.assert_array_equal(analysis.cluster_sizes(label), [3, 2, 1, 1])
    # a ring closed by its last edge, and a chain listed from its far end
    label, k = analysis.contact_clusters(6, _keys([(4, 5), (3, 4), (2, 3), (1, 2), (1, 5)]))
    np.testing.assert_array_equal(label, [0, 1, 1, 1, 1, 1])
    assert k == 2
    label, k = analysis.contact_clusters(3, _keys([]))
    np.testing.assert_array_equal(label, [0, 1, 2])
    assert k == 3


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_clusters_match_scipy_connected_components(seed):
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    from scipy.sparse import coo_matrix
    rng = np.random.default_rng(seed)
    n = 500
    e = rng.integers(0, n, size=(380, 2))
    e = e[e[:, 0] != e[:, 1]]
    label, k = analysis.contact_clusters(n, _keys(e.tolist()))
    m = coo_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(n, n))
    kk, lab = csgraph.connected_components(m, directed=False)
    assert k == kk
    # same partition, labelled by the smallest member
    mins = {}
    for i, c in enumerate(lab):
        mins.setdefault(c, i)
    np.testing.assert_array_equal(label, [mins[c] for c in lab])


def test_dispersion_closed_forms():
    rng = np.random.default_rng(7)
    v = rng.normal(size=1000)
    y0 = rng.uniform(0, 10, size=1000)
    t, a0, gd = 2.5, 2.0, 3.0
    dy, cv = analysis.dispersion(y0 + v * t, y0, v, v, t, gd, a0)
    assert dy == pytest.approx(np.mean(v ** 2) * t / (2 * a0 * a0 * gd), rel=1e-12)
    assert cv == pytest.approx(1.0, rel=1e-14)
    _, cv = analysis.dispersion(y0, y0, -v, v, t, gd, a0)
    assert cv == pytest.approx(-1.0, rel=1e-14)


@pytest.mark.parametrize("vy", [+3.0, -3.0])
def test_image_count_keeps_the_unwrapped_y_continuous(vy):
    L = 20.0
    p = oracle.make_params([L] * 3, shear_rate=0.5, eta0=0.0, dt=1e-2)
    y0 = 19.9 if vy > 0 else 0.1
    x = np.array([[5.0], [y0], [5.0]])
    s = oracle.System(p, x, [1.0], u=np.array([[0.0], [vy], [0.0]]), w=np.zeros((3, 1)))
    s.step(10)
    st = s.get_state()
    iy = s.get_images()
    assert iy[0] == (1 if vy > 0 else -1)
    assert st["x"][1, 0] + iy[0] * L == pytest.approx(y0 + 10 * 1e-2 * vy, abs=1e-12)


# ---- local volume fraction along y by size class (Sec. III B, Fig. 12)

def test_phi_profile_pins():
    import math
    from scipy.integrate import quad
    from oracle import analysis as an
    box = np.array([20.0, 16.0, 12.0])
    nb = 8
    w = box[1] / nb
    slab = box[0] * box[2] * w
    # one sphere in the middle of slab 3, radius below half a slab: all of it there
    p = an.phi_profile([3.5 * w], [0.7], box, nb, a_split=1.0)
    want = np.zeros((2, nb))
    want[0, 3] = 4.0 / 3.0 * math.pi * 0.7 ** 3 / slab
    np.testing.assert_allclose(p, want, rtol=1e-14, atol=0)
    # centred on the plane between slabs 4 and 5 (class 1): half in each
    p = an.phi_profile([5 * w], [1.3], box, nb, a_split=1.0)
    half = 0.5 * 4.0 / 3.0 * math.pi * 1.3 ** 3 / slab
    assert p[1, 4] == pytest.approx(half, rel=1e-13) and p[1, 5] == pytest.approx(half, rel=1e-13)
    assert p[0].sum() == 0.0 and np.count_nonzero(p[1]) == 2
    # a sphere across y = 0: its parts in the first and the last slab, each
    # the quadrature of its cross-sections over the part
    a, yc = 1.5, 0.4
    p = an.phi_profile([yc], [a], box, nb, a_split=2.0)
    disk = lambda t: math.pi * (a * a - t * t)
    top = quad(disk, -a, -yc)[0]          # below y = 0, seen from y = L_y
    bottom = quad(disk, -yc, a)[0]
    assert p[0, 0] * slab == pytest.approx(bottom, rel=1e-12)
    assert p[0, -1] * slab == pytest.approx(top, rel=1e-12)
    # a packing: each slab against the quadrature of every sphere's
    # cross-sections, and the mean over slabs is the class volume fraction
    rng = np.random.default_rng(3)
    y = rng.uniform(0, box[1], size=40)
    r = rng.uniform(0.5, 2.5, size=40)
    p = an.phi_profile(y, r, box, nb, a_split=1.5)
    q = np.zeros((2, nb))
    for yy, aa in zip(y, r):
        for img in (-1, 0, 1):
            for b in range(nb):
                lo, hi = max(b * w - (yy + img * box[1]), -aa), min((b + 1) * w - (yy + img * box[1]), aa)
                if hi > lo:
                    q[int(aa > 1.5), b] += quad(lambda t: math.pi * (aa * aa - t * t), lo, hi)[0]
    np.testing.assert_allclose(p * slab, q, rtol=1e-11, atol=1e-12)
    V = box.prod()
    for c in (0, 1):
        sel = (r > 1.5) if c else (r <= 1.5)
        assert p[c].mean() == pytest.approx(np.sum(4.0 / 3.0 * math.pi * r[sel] ** 3) / V, rel=1e-13)
