"""Element-wise parity checks of the CUDA path against the oracle.

Every check is per particle (or per component), never through one norm over
all particles, so a particle whose force is small next to the others cannot
hide a large relative error.

Forces and torques: for each particle i (a column of a (3, n) array)

    |g_i - w_i| <= tol * max(|w_i|, kappa * A_i)

with w the oracle's vector and A_i the sum of the magnitudes of the terms
that make it up (per pair the contact force, each sub-term of the
lubrication resistance of Eq. A2-A3, the electro-chemical force; and the
drag: ``oracle.System.force_scale``).  Where the terms do not cancel,
|w_i| ~ A_i and the bound is tol relative to the particle's own force.
Where they nearly cancel (a pair in contact whose spring balances the
lubrication strain term, two spheres moving together), the rounding of any
evaluation of the terms (FP32 pair arithmetic in mixed precision: each term
good to ~1e-7 of itself) is bounded by A_i, not by |w_i|, and the bound
becomes tol * kappa * A_i.  kappa is stated beside each tolerance below.

Other per-particle vectors (velocities, accelerations, gradients) use the
same form with a floor of a stated fraction of the median magnitude in place
of kappa * A_i.

Stress: each of the nine components within tol of max(|S_q|, floor * |S|),
and each reported quantity (sigma_xy, N1 = S_xx - S_yy, N2 = S_yy - S_zz,
Pi = -tr S / 3) within tol of its own value (same floor; 1e-3 in FP64, 1e-2
in mixed precision).
"""
import numpy as np

FP64_TOL = 1e-10
MIXED_TOL = 1e-5
# kappa of the force bound: FP64 rounding is ~1e-16 of each term, so the own
# force bounds every particle whose terms cancel to less than 1e6 of
# themselves; FP32 terms carry ~1e-7 of themselves, so where the terms cancel
# by more than a factor 10 the error scales with their magnitudes
KAPPA_FP64 = 1e-3
KAPPA_MIXED = 0.1
# stress: components and reported quantities relative to their own value, or
# to this fraction of |S| where they nearly vanish (N2 = S_yy - S_zz or an
# off-diagonal component can be ~1e-2 |S|); the mixed pair stresslets carry
# ~1e-7 |S| each, so the floor there is 1e-2 |S|
STRESS_FLOOR = 1e-3
STRESS_FLOOR_MIXED = 1e-2


def check_vectors(got, want, tol, scale, what="vector"):
    """|got_i - want_i| <= tol * max(|want_i|, scale_i) for every column i
    ((3, n) arrays; scale: (n,) or a scalar).  Returns the largest ratio."""
    g, w = np.asarray(got, dtype=np.float64), np.asarray(want, dtype=np.float64)
    assert g.shape == w.shape, (g.shape, w.shape)
    d = np.linalg.norm(g - w, axis=0)
    m = np.linalg.norm(w, axis=0)
    s = np.maximum(m, np.broadcast_to(np.asarray(scale, dtype=np.float64), m.shape))
    s = np.maximum(s, 1e-300)
    r = d / s
    k = int(np.argmax(r))
    assert np.all(np.isfinite(g)), "%s: non-finite values" % what
    assert r[k] <= tol, ("%s: particle %d off by %.3e of max(|w|, scale) (|w| = %.3e, scale = %.3e, "
                         "|d| = %.3e; tolerance %.1e)" % (what, k, r[k], m[k], s[k], d[k], tol))
    return float(r[k])


def check_forces(got, want, absum, tol, kappa, what="force"):
    """Per-particle force (or torque) bound of this module's docstring.  A
    particle with no terms at all (alone and moving with the flow: its
    oracle force is exactly zero) is held to 1e-6 of the median scale."""
    A = np.asarray(absum, dtype=np.float64)
    floor = 1e-6 * float(np.median(A)) if A.size else 0.0
    return check_vectors(got, want, tol, np.maximum(kappa * A, floor), what)


def check_per_particle(got, want, tol, floor=1e-3, what="vector"):
    """Per-particle bound with a floor of ``floor`` times the median magnitude."""
    w = np.asarray(want, dtype=np.float64)
    med = float(np.median(np.linalg.norm(w, axis=0)))
    return check_vectors(got, want, tol, floor * med, what)


def stress_quantities(S):
    S = np.asarray(S, dtype=np.float64).reshape(3, 3)
    return {"sigma_xy": S[0, 1], "N1": S[0, 0] - S[1, 1], "N2": S[1, 1] - S[2, 2],
            "Pi": -np.trace(S) / 3.0}


def check_stress(got, want, tol, floor=None, what="stress"):
    """Every component and every reported quantity within tol of its own
    value (or of floor * |S| where that is larger; by default the floor of
    the precision the tolerance belongs to)."""
    if floor is None:
        floor = STRESS_FLOOR if tol <= FP64_TOL * 10 else STRESS_FLOOR_MIXED
    g = np.asarray(got, dtype=np.float64).reshape(3, 3)
    w = np.asarray(want, dtype=np.float64).reshape(3, 3)
    assert np.all(np.isfinite(g)), "%s: non-finite" % what
    fl = floor * np.linalg.norm(w)
    worst = 0.0
    for q in range(9):
        r = abs(g.flat[q] - w.flat[q]) / max(abs(w.flat[q]), fl, 1e-300)
        assert r <= tol, "%s: component %d off by %.3e (tolerance %.1e)" % (what, q, r, tol)
        worst = max(worst, r)
    qg, qw = stress_quantities(g), stress_quantities(w)
    for k in qw:
        r = abs(qg[k] - qw[k]) / max(abs(qw[k]), fl, 1e-300)
        assert r <= tol, "%s: %s off by %.3e (tolerance %.1e)" % (what, k, r, tol)
        worst = max(worst, r)
    return worst


def check_scalars(got, want, tol, floor=0.0, what="values"):
    """Element by element: |g_k - w_k| <= tol * max(|w_k|, floor * max|w|)."""
    g = np.asarray(got, dtype=np.float64).ravel()
    w = np.asarray(want, dtype=np.float64).ravel()
    assert g.shape == w.shape
    s = np.maximum(np.abs(w), max(floor * float(np.abs(w).max(initial=0.0)), 1e-300))
    r = np.abs(g - w) / s
    k = int(np.argmax(r)) if r.size else 0
    assert r.size == 0 or r[k] <= tol, "%s: entry %d off by %.3e (tolerance %.1e)" % (what, k, r[k], tol)
    return float(r[k]) if r.size else 0.0


def periodic_diff(x, y, box):
    d = np.abs(np.asarray(x) - np.asarray(y))
    return np.minimum(d, np.asarray(box)[:, None] - d)


def kappa_for(tol):
    """kappa of the force bound for a tolerance (FP64 or mixed precision)."""
    return KAPPA_FP64 if tol <= FP64_TOL * 10 else KAPPA_MIXED
