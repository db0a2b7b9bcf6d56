"""Seeded synthetic suspensions (inputs only; none of the model's arithmetic).

The paper starts its runs from packings made with third-party packing
software (Sec. III).  That software and its outputs are not available, so
every configuration here is generated from a seed:

1. radii: bidisperse by number (``frac_large`` of the particles get
   ``a_large``), or log-uniform in ``[a_min, a_max]``; the array order is a
   seeded random permutation, so memory order carries no spatial or size
   structure;
2. box: cubic, edge chosen so that the solid volume fraction equals ``phi``;
3. positions: random sequential insertion, largest first, ``tries`` attempts
   per particle; particles that do not fit are dropped at random positions;
4. Jacobi overlap-removal sweeps until the largest overlap is below
   ``tol * a_min`` or ``max_iter`` sweeps have run;
5. ids are the array indices (already in random spatial order).

Velocities are not drawn: the solver starts from the ambient flow.

Random numbers come from a counter-based splitmix64 stream (same values on
any machine), the sweeps accumulate in a fixed order, so a (config, seed)
pair always gives the same bytes.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from ctypes import POINTER, c_double, c_int, c_int64, c_uint64
from dataclasses import dataclass, field, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth_relax.c")
_OUT = os.path.join(_HERE, "_build", "libsynth.so")


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if (not force and os.path.exists(_OUT)
            and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC)):
        return _OUT
    tmp = _OUT + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:],
                              stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(base)
    os.replace(tmp, _OUT)
    return _OUT


_lib = None


def _clib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = POINTER(c_double)
        _lib.synth_insert.restype = c_int64
        _lib.synth_insert.argtypes = [c_int64, dp, dp, c_uint64, c_int, dp]
        _lib.synth_relax.restype = c_int
        _lib.synth_relax.argtypes = [c_int64, dp, dp, dp, c_int, c_double, c_double, dp]
    return _lib


_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, stream: int, count: int) -> np.ndarray:
    """``count`` uniform doubles in [0,1) from counter-based splitmix64."""
    k = np.arange(count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        base = np.uint64(seed) * np.uint64(0x9E3779B97F4A7C15) + np.uint64(stream) * np.uint64(0x632BE59BD9B4E019)
        z = _mix64(base + (k + np.uint64(1)) * np.uint64(0xD1B54A32D192ED03))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass(frozen=True)
class Spec:
    """A synthetic suspension and the model parameters it is run with."""
    name: str
    n: int
    phi: float
    radii: str = "bidisperse"       # or "loguniform"
    a_small: float = 1.0
    a_large: float = 1.4
    frac_large: float = 0.5
    a_min: float = 1.0
    a_max: float = 10.0
    mu: float = 0.5
    kn: float = 1e4
    shear_rate: float = 1.0
    dt: float = 1e-4
    steps: int = 1000
    seed: int = 1
    tries: int = 30
    max_iter: int = 2000
    tol: float = 1e-3
    extra: dict = field(default_factory=dict)


# The workloads the solver is exercised on (sizes, radii, volume fractions,
# friction and step counts of the benchmark configurations).
SPECS = {
    "c1": Spec("c1_fp64_bidisperse_1k", 1000, 0.50, mu=0.5, steps=1000, seed=1),
    "c2": Spec("c2_mixed_bidisperse_100k", 100_000, 0.55, mu=1.0, steps=10_000, seed=2),
    "c3": Spec("c3_polydisperse_1m", 1_000_000, 0.50, radii="loguniform", mu=0.5,
               steps=1000, seed=3, max_iter=20),
    "c5": Spec("c5_rollout_20k", 20_000, 0.54, mu=0.5, steps=200, seed=5),
    # Table 5 (case YW): 2^16 particles, radius ratio a2/a1 = 3 with the large
    # spheres holding a quarter of the small ones' volume (V2/V1 = 0.25),
    # phi = 0.5; k_n = 4e5 eta0 a0 gdot, k_t/k_n = 2/7, gamma_n gdot/k_n = 1e-7,
    # St = rho a0^2 gdot/eta0 = 1e-3, mu = 1, delta_lub = 0.25 a0,
    # lambda_D = 0.02 a0, F^R/F^A = 19 at contact with the repulsion at
    # gdot/gdot_0 = 1 (F_ER = eta0 a0^2 gdot), the wave U = 20 gdot a0 with
    # n = 1; time step gamma_n/k_n (Sec. II A).
    "c6": Spec("c6_wavy_bidisperse_65k", 65_536, 0.50, a_small=1.0, a_large=3.0,
               frac_large=(0.25 / 27.0) / (1.0 + 0.25 / 27.0), mu=1.0, kn=4e5, dt=1e-7,
               steps=1000, seed=6,
               extra=dict(kt=4e5 * 2.0 / 7.0, rho=1e-3, eta0=1.0, delta_lub=0.25,
                          lub_cutoff_mode=1, f_er=1.0, lambda_d=0.02,
                          hamaker=12.0 * 1e-4 / 19.0, vdw_eps=0.01, wave_amp=20.0, wave_n=1)),
}


def radii(spec: Spec) -> np.ndarray:
    n = spec.n
    if spec.radii == "bidisperse":
        nl = int(round(spec.frac_large * n))
        a = np.full(n, spec.a_small)
        a[:nl] = spec.a_large
    elif spec.radii == "loguniform":
        u = uniform(spec.seed, 1, n)
        a = spec.a_min * np.exp(u * math.log(spec.a_max / spec.a_min))
    else:
        raise ValueError(spec.radii)
    # seeded random permutation of the array order
    perm = np.argsort(uniform(spec.seed, 2, n), kind="stable")
    return np.ascontiguousarray(a[perm])


def box_edge(a: np.ndarray, phi: float) -> float:
    vs = float(np.sum(4.0 / 3.0 * math.pi * a ** 3))
    return (vs / phi) ** (1.0 / 3.0)


def generate(spec: Spec, relax: bool = True):
    """Returns dict(x=(3,n) f64, a=(n,) f64, ids=(n,) i32, box=(3,) f64, info)."""
    a = radii(spec)
    n = a.shape[0]
    L = box_edge(a, spec.phi)
    box = np.array([L, L, L], dtype=np.float64)
    order = np.argsort(-a, kind="stable")          # largest first
    a_sorted = np.ascontiguousarray(a[order])
    xs = np.zeros((3, n), dtype=np.float64)
    lib = _clib()
    dp = POINTER(c_double)
    placed = lib.synth_insert(n, a_sorted.ctypes.data_as(dp), box.ctypes.data_as(dp),
                              spec.seed, spec.tries, xs.ctypes.data_as(dp))
    x = np.zeros((3, n), dtype=np.float64)
    x[:, order] = xs
    x = np.ascontiguousarray(x)
    mo = c_double(0.0)
    sweeps = 0
    if relax:
        sweeps = lib.synth_relax(n, x.ctypes.data_as(dp), a.ctypes.data_as(dp),
                                 box.ctypes.data_as(dp), spec.max_iter,
                                 spec.tol * float(a.min()), 0.8, ctypes.byref(mo))
    ids = np.arange(n, dtype=np.int32)
    return dict(x=x, a=a, ids=ids, box=box,
                info=dict(inserted=int(placed), sweeps=int(sweeps), max_overlap=float(mo.value)))


@dataclass(frozen=True)
class BatchSpec:
    """K independent bidisperse suspensions of a flow-curve sweep: particle
    count uniform in ``n_range``, volume fraction uniform in ``phi_range`` and
    shear rate log-uniform in ``gdot_range``, each drawn per instance."""
    name: str
    K: int
    n_range: tuple = (500, 20_000)
    phi_range: tuple = (0.40, 0.58)
    gdot_range: tuple = (1e-2, 1e2)
    mu: float = 0.5
    kn: float = 1e4
    dt: float = 1e-4
    steps: int = 5000
    seed: int = 4
    max_iter: int = 60


BATCH_SPECS = {
    "c4": BatchSpec("c4_batched_256_flow_curve", 256),
}


def batch_members(spec: BatchSpec):
    """[(Spec, shear rate)] of the instances (seeded draws, no packing yet)."""
    un = uniform(spec.seed, 10, spec.K)
    up = uniform(spec.seed, 11, spec.K)
    ug = uniform(spec.seed, 12, spec.K)
    n0, n1 = spec.n_range
    out = []
    for k in range(spec.K):
        n = n0 + min(int(un[k] * (n1 - n0 + 1)), n1 - n0)
        phi = spec.phi_range[0] + up[k] * (spec.phi_range[1] - spec.phi_range[0])
        g0, g1 = math.log(spec.gdot_range[0]), math.log(spec.gdot_range[1])
        gdot = math.exp(g0 + ug[k] * (g1 - g0))
        s = Spec("%s_%d" % (spec.name, k), n, phi, mu=spec.mu, kn=spec.kn, shear_rate=gdot, dt=spec.dt,
                 steps=spec.steps, seed=spec.seed * 100_003 + k, max_iter=spec.max_iter)
        out.append((s, gdot))
    return out


def _generate_member(spec: Spec):
    os.environ["OMP_NUM_THREADS"] = "1"     # one core per worker process
    build()
    return generate(spec)


def generate_batch(spec: BatchSpec, workers: int = 0) -> dict:
    """Packs every instance (in ``workers`` spawned processes; 0: one per
    core, up to 16) and concatenates them instance-major.  Returns dict(x
    (3, N), a (N), ids (N, instance k holds its own index range), n (K),
    boxes (K, 3), shear_rates (K), phi (K))."""
    members = batch_members(spec)
    build()
    if workers == 0:
        workers = min(16, os.cpu_count() or 1)
    if workers > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            gs = pool.map(_generate_member, [m[0] for m in members], chunksize=1)
    else:
        gs = [generate(m[0]) for m in members]
    n = np.array([g["a"].shape[0] for g in gs], dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(n)])
    return dict(x=np.ascontiguousarray(np.concatenate([g["x"] for g in gs], axis=1)),
                a=np.ascontiguousarray(np.concatenate([g["a"] for g in gs])),
                ids=np.concatenate([g["ids"] + off[k] for k, g in enumerate(gs)]).astype(np.int32),
                n=n, boxes=np.array([g["box"] for g in gs]),
                shear_rates=np.array([m[1] for m in members]),
                phi=np.array([m[0].phi for m in members]))


def small(n: int, phi: float, seed: int, **kw) -> dict:
    """A small bidisperse (1 : 1.4) packing for tests."""
    return generate(replace(Spec("small", n, phi, seed=seed), **kw))
