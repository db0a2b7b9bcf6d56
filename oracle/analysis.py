"""CPU oracle of the analysis pass (TEST INFRASTRUCTURE ONLY; only tests/
may import it): the rheological quantities derived from the bulk stress
(Sec. II, after Eq. 9), the clusters of contacting particles (Sec. III A,
Fig. 10-11), the shear-wise dispersion of Eq. 18-19 and the local volume
fraction along y by size class (Sec. III B, Fig. 12).  Plain Python and
numpy, written from the definitions; pinned in tests/test_oracle_analysis.py.
"""
from __future__ import annotations

import numpy as np


def rheology(sigma, shear_rate: float, eta0: float = 1.0) -> dict:
    """sigma = S_12, N1 = S_11 - S_22, N2 = S_22 - S_33, Pi = -tr(S)/3,
    eta_r = sigma / (eta0 gdot), eta_n = Pi / (eta0 gdot) of a 3x3 bulk stress
    (indices 1, 2, 3 = flow x, gradient y, vorticity z)."""
    S = np.asarray(sigma, dtype=np.float64).reshape(3, 3)
    s12 = S[0, 1]
    pi = -(S[0, 0] + S[1, 1] + S[2, 2]) / 3.0
    return dict(sigma=s12, N1=S[0, 0] - S[1, 1], N2=S[1, 1] - S[2, 2], Pi=pi,
                eta_r=s12 / (eta0 * shear_rate), eta_n=pi / (eta0 * shear_rate))


def contact_clusters(n: int, keys) -> tuple[np.ndarray, int]:
    """Connected components of the graph on ids 0..n-1 whose edges are the
    contacting pairs (keys lo << 32 | hi).  Returns (label, count): label[id]
    is the smallest id of its cluster; a particle with no contact is a
    cluster of one."""
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            x = parent[x]
        return x

    for k in np.asarray(keys, dtype=np.int64).tolist():
        a, b = k >> 32, k & 0xFFFFFFFF
        ra, rb = find(a), find(b)
        if ra != rb:
            # keep the smaller id as the root: the root is the smallest id
            parent[max(ra, rb)] = min(ra, rb)
    label = np.array([find(i) for i in range(n)], dtype=np.int64)
    return label, int(np.sum(label == np.arange(n)))


def cluster_sizes(label) -> np.ndarray:
    """Sizes of the clusters, in increasing order of their labels."""
    _, counts = np.unique(np.asarray(label), return_counts=True)
    return counts


def dispersion(y, y0, v, v0, dt_elapsed: float, shear_rate: float, a0: float = 1.0) -> tuple[float, float]:
    """Eq. 18: D_y = <(y(t) - y(t0))^2> / (2 (t - t0)) / (a0^2 gdot), with y
    the unwrapped shear-wise (gradient) position; Eq. 19: C_v = <v'(t) v'(t0)>
    / <v'(t)^2> with v' the shear-wise velocity fluctuation.  Averages over
    the given particles."""
    y, y0, v, v0 = (np.asarray(t, dtype=np.float64) for t in (y, y0, v, v0))
    msd = np.mean((y - y0) ** 2)
    dy = msd / (2.0 * dt_elapsed) / (a0 * a0 * shear_rate) if dt_elapsed > 0 else 0.0
    cv = np.mean(v * v0) / np.mean(v * v)
    return float(dy), float(cv)


def phi_profile(y, a, box, nbins: int, a_split: float) -> np.ndarray:
    """Local volume fraction along y (Sec. III B, Fig. 12): (2, nbins), the
    volume of the spheres of class 0 (a <= a_split) and class 1 (a > a_split)
    inside each of nbins equal slabs of the periodic box, over the slab's
    volume.  A sphere of radius a centred at yc holds, between the planes
    y0 < y1, the integral of its cross-sections pi (a^2 - t^2) over
    t in [max(y0 - yc, -a), min(y1 - yc, a)]; its images at yc -+ L_y count
    the same way."""
    y = np.asarray(y, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    Lx, Ly, Lz = (float(v) for v in box)
    w = Ly / nbins
    out = np.zeros((2, nbins))
    for yy, aa in zip(y.tolist(), a.tolist()):
        c = 1 if aa > a_split else 0
        for img in (-1, 0, 1):
            yc = yy + img * Ly
            for b in range(nbins):
                y0, y1 = b * w, (Ly if b == nbins - 1 else (b + 1) * w)
                t0, t1 = max(y0 - yc, -aa), min(y1 - yc, aa)
                if t1 > t0:
                    out[c, b] += np.pi * (aa * aa * (t1 - t0) - (t1 ** 3 - t0 ** 3) / 3.0)
    return out / (Lx * Lz * w)
