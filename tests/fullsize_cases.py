"""Inputs for the sampled parity checks at the benchmark sizes, made without
the CUDA path: the seeded packing, seeded velocities, and a seeded contact
history on the contacts the oracle itself finds around the sampled
particles."""
import numpy as np


def sample(a, m=48, seed=0):
    """The 8 largest, the 8 smallest and m - 16 random particles (indices)."""
    order = np.argsort(a)
    rng = np.random.default_rng(seed)
    pick = np.concatenate([order[-8:], order[:8], rng.choice(a.shape[0], m - 16, replace=False)])
    return np.unique(pick)


def velocities(x, a, shear_rate, seed):
    """Ambient shear plus noise on the translational and rotational velocities."""
    rng = np.random.default_rng(seed)
    n = a.shape[0]
    u = 0.3 * shear_rate * rng.normal(size=(3, n)) * a
    u[0] += shear_rate * x[1]
    w = 0.3 * shear_rate * rng.normal(size=(3, n))
    w[2] -= 0.5 * shear_rate
    return u, w


def contact_history(oracle, po, off, x, a, ids, u, w, idx, seed, scale=3e-4):
    """Pair keys (lo id << 32 | hi id) of every contact of the sampled
    particles, as the oracle decides it (Eq. 4: overlap), each with a seeded
    tangential stretch (some below, some above the Coulomb limit)."""
    pos = np.empty(ids.max() + 1, dtype=np.int64)
    pos[ids] = np.arange(ids.shape[0])
    keys = set()
    for k in idx:
        k = int(k)
        for jid in oracle.neighbours_of(x, a, ids, po, off, k):
            j = int(pos[jid])
            fl = oracle.pair_eval(po, off, x[:, k], x[:, j], u[:, k], u[:, j], w[:, k], w[:, j],
                                  a[k], a[j])[0]
            if fl & 2:
                lo, hi = sorted((int(ids[k]), int(ids[j])))
                keys.add((lo << 32) | hi)
    keys = np.array(sorted(keys), dtype=np.int64)
    rng = np.random.default_rng(seed)
    xi = scale * rng.normal(size=(keys.shape[0], 3))
    return keys, xi


def partners(pairs, k):
    """Sorted partner ids of id k in a (lo, hi) pair list."""
    return np.sort(np.concatenate([pairs[pairs[:, 0] == k, 1], pairs[pairs[:, 1] == k, 0]]))
