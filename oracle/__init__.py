"""CPU FP64 oracle for the dense-suspension time step (arXiv:2108.01013).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow definition that
the CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code
with the CUDA path and never imports the product package.

The arithmetic lives in ``oracle.c`` (plain C, FP64, compiled with FMA
contraction disabled so that the neighbour predicate is evaluated exactly as
written); this module only marshals arguments through ctypes.

Parity status of each function (see the pins in ``tests/test_oracle_*.py``):
  pairs_bruteforce / neighbours_of  pinned (brute-force definition, hand
                                    placed geometry, Lees-Edwards images)
  contact                           pinned (head-on spring-dashpot closed
                                    form, Coulomb-capped tangential loading)
  analysis (rheology, clusters,     pinned in tests/test_oracle_analysis.py
    dispersion, image count)        (Einstein viscosity, compressional
                                    contact, hand-built and scipy graphs,
                                    ballistic dispersion, wrap continuity)
  echem / echem_range               pinned (integrates to the closed-form
                                    potentials of Eq. 6-7, Debye decay,
                                    harmonic-radius scaling, flat and
                                    continuous at contact, exact ranges,
                                    central and balanced in pair_eval)
  lubrication                       pinned by physics invariants (Reynolds
                                    squeeze law for equal spheres, zero
                                    force/torque for rigid motion of the pair
                                    and for particles at rest in a linear
                                    flow, antisymmetry, dissipation >= 0,
                                    a symmetric resistance matrix by the
                                    reciprocal theorem).
                                    The absolute values of the log-order
                                    coefficients for unequal radii beyond
                                    these invariants are parity unpinned.
  flow_ux / flow_rate / faxen_ux,    pinned in tests/test_oracle_wavy.py (Faxen
    the wavy flow of Eq. 17         drag = surface mean of the flow up to
                                    (ka)^4, relaxation to it and to the local
                                    spin, pairs equal simple-shear pairs at
                                    the mean rate, local stresslets, wrap
                                    continuity, no wave = simple shear)
  rolling (App. B)                  pinned in tests/test_oracle_rolling.py
                                    (oscillation of the relative spin of a
                                    row of spheres at the closed-form
                                    frequency with its angular momentum
                                    conserved, Coulomb limit, no force, no
                                    stresslet, orientation independence)
  System.step / forces / stress     pinned (Stokes relaxation closed form,
                                    Lees-Edwards wrap invariants, momentum
                                    balance, stress sign checks)
  System(cells=True), pairs_cell    the cell list with the half stencil of
                                    Sec. II A: pinned to the brute force
                                    (equal pair sets up to 20k particles,
                                    Lees-Edwards layers, polydisperse radii,
                                    near-cutoff pairs; bit-identical forces,
                                    stress and trajectories)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from ctypes import POINTER, c_double, c_int, c_int32, c_int64, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``_build/liboracle.so`` (gcc, FP64, no FMA;
    OpenMP over the host cores where the compiler offers it)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if (not force and os.path.exists(_OUT)
            and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC)):
        return _OUT
    tmp = _OUT + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.check_call(cmd[:1] + ["-fopenmp"] + cmd[1:], stdout=subprocess.DEVNULL,
                              stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(cmd)
    os.replace(tmp, _OUT)
    return _OUT


class Params(ctypes.Structure):
    """Mirror of ``orc_params`` in oracle.c."""
    _fields_ = [("kn", c_double), ("kt", c_double), ("gamma_n", c_double),
                ("mu", c_double), ("eta0", c_double), ("rho", c_double),
                ("delta_lub", c_double), ("lub_eps", c_double), ("a0", c_double),
                ("lub_cutoff_mode", c_int32), ("pad_", c_int32),
                ("shear_rate", c_double), ("dt", c_double), ("L", c_double * 3),
                ("lub_taper", c_double), ("f_er", c_double), ("lambda_d", c_double),
                ("hamaker", c_double), ("vdw_eps", c_double),
                ("wave_amp", c_double), ("k_r", c_double), ("wave_n", c_int32),
                ("pad2_", c_int32)]


def make_params(box, kn=1e4, kt=None, gamma_n=None, mu=0.5, eta0=1.0, rho=1.0,
                delta_lub=0.05, lub_eps=1e-3, a0=1.0, lub_cutoff_mode=0,
                shear_rate=1.0, dt=1e-4, lub_taper=0.0, f_er=0.0, lambda_d=0.05,
                hamaker=0.0, vdw_eps=0.01, wave_amp=0.0, wave_n=0, k_r=0.0) -> Params:
    """Oracle parameters; kt defaults to kn/2 and gamma_n to 1e-7 kn/gdot.
    wave_amp, wave_n: the wavy shear flow of Eq. 17; k_r: the rolling spring
    of App. B (0: off)."""
    if kt is None:
        kt = 0.5 * kn
    if gamma_n is None:
        gamma_n = 1e-7 * kn / shear_rate if shear_rate != 0 else 0.0
    p = Params()
    p.kn, p.kt, p.gamma_n, p.mu = kn, kt, gamma_n, mu
    p.eta0, p.rho, p.delta_lub, p.lub_eps, p.a0 = eta0, rho, delta_lub, lub_eps, a0
    p.lub_cutoff_mode = lub_cutoff_mode
    p.shear_rate, p.dt = shear_rate, dt
    p.lub_taper = lub_taper
    p.f_er, p.lambda_d, p.hamaker, p.vdw_eps = f_er, lambda_d, hamaker, vdw_eps
    p.wave_amp, p.wave_n, p.k_r = wave_amp, int(wave_n), k_r
    for k in range(3):
        p.L[k] = float(box[k])
    return p


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        dp = POINTER(c_double)
        i64p = POINTER(c_int64)
        i32p = POINTER(c_int32)
        pp = POINTER(Params)
        L.orc_le_offset.restype = c_double
        L.orc_le_offset.argtypes = [pp, c_int64]
        L.orc_pairs_bruteforce.restype = c_int64
        L.orc_pairs_bruteforce.argtypes = [c_int64, dp, dp, i32p, pp, c_double, i64p, c_int64]
        L.orc_neighbours_of.restype = c_int64
        L.orc_neighbours_of.argtypes = [c_int64, dp, dp, i32p, pp, c_double, c_int64, i64p, c_int64]
        L.orc_contact.restype = None
        L.orc_contact.argtypes = [pp, dp, c_double, c_double] + [dp] * 5 + [dp] * 4
        L.orc_lubrication.restype = None
        L.orc_lubrication.argtypes = [pp, dp, c_double, c_double] + [dp] * 4 + [dp] * 4
        L.orc_lubrication_rate.restype = None
        L.orc_lubrication_rate.argtypes = [pp, c_double, dp, c_double, c_double] + [dp] * 8
        L.orc_rolling.restype = None
        L.orc_rolling.argtypes = [pp, dp, c_double, c_double] + [dp] * 5 + [dp] * 3
        for nm in ("orc_flow_ux", "orc_flow_rate"):
            getattr(L, nm).restype = c_double
            getattr(L, nm).argtypes = [pp, c_double]
        L.orc_faxen_ux.restype = c_double
        L.orc_faxen_ux.argtypes = [pp, c_double, c_double]
        L.orc_pair_eval_full.restype = c_int
        L.orc_pair_eval_full.argtypes = ([pp, c_double] + [dp] * 6 + [c_double, c_double, dp, dp]
                                         + [dp] * 7)
        L.orc_set_history_r.restype = None
        L.orc_set_history_r.argtypes = [c_void_p, c_int64, i64p, dp, dp]
        L.orc_get_history_r.restype = c_int64
        L.orc_get_history_r.argtypes = [c_void_p, c_int64, i64p, dp, dp]
        L.orc_echem.restype = None
        L.orc_echem.argtypes = [pp, c_double, c_double, c_double, dp, dp]
        L.orc_echem_range.restype = c_double
        L.orc_echem_range.argtypes = [pp]
        L.orc_pair_eval.restype = c_int
        L.orc_pair_eval.argtypes = [pp, c_double] + [dp] * 6 + [c_double, c_double, dp] + [dp] * 6
        L.orc_create.restype = c_void_p
        L.orc_create.argtypes = [c_int64, pp]
        L.orc_destroy.restype = None
        L.orc_destroy.argtypes = [c_void_p]
        L.orc_set_state.restype = None
        L.orc_set_state.argtypes = [c_void_p, dp, dp, i32p, dp, dp, dp, dp, c_int64]
        L.orc_set_history.restype = None
        L.orc_set_history.argtypes = [c_void_p, c_int64, i64p, dp]
        L.orc_get_history.restype = c_int64
        L.orc_get_history.argtypes = [c_void_p, c_int64, i64p, dp]
        L.orc_forces.restype = None
        L.orc_forces.argtypes = [c_void_p, c_int]
        L.orc_init_accel.restype = None
        L.orc_init_accel.argtypes = [c_void_p]
        L.orc_step.restype = None
        L.orc_step.argtypes = [c_void_p, c_int64]
        L.orc_get_state.restype = None
        L.orc_get_state.argtypes = [c_void_p, dp, dp, dp, dp, dp]
        L.orc_get_forces.restype = None
        L.orc_get_forces.argtypes = [c_void_p, dp, dp, dp]
        L.orc_get_images.restype = None
        L.orc_get_images.argtypes = [c_void_p, i64p]
        L.orc_forces_sampled.restype = None
        L.orc_forces_sampled.argtypes = [c_void_p, i64p, c_int64, dp, dp, dp, dp]
        L.orc_set_cells.restype = None
        L.orc_set_cells.argtypes = [c_void_p, c_int]
        L.orc_pairs_cell.restype = c_int64
        L.orc_pairs_cell.argtypes = [c_void_p, i64p, c_int64]
        L.orc_get_force_scale.restype = None
        L.orc_get_force_scale.argtypes = [c_void_p, dp, dp]
        for nm in ("orc_get_nstep", "orc_get_npairs", "orc_get_ncontacts"):
            getattr(L, nm).restype = c_int64
            getattr(L, nm).argtypes = [c_void_p]
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t=c_double):
    return a.ctypes.data_as(POINTER(t))


def _opt(a):
    return None if a is None else _ptr(a)


def le_offset(p: Params, nstep: int) -> float:
    return lib().orc_le_offset(ctypes.byref(p), int(nstep))


def pairs_bruteforce(x, a, ids, p: Params, off: float) -> np.ndarray:
    """All (lo id, hi id) pairs within range, sorted; x is SoA (3, n)."""
    x = _d(x)
    a = _d(a)
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    n = a.shape[0]
    cnt = lib().orc_pairs_bruteforce(n, _ptr(x), _ptr(a), _ptr(ids, c_int32),
                                     ctypes.byref(p), off, None, 0)
    out = np.zeros((max(cnt, 1), 2), dtype=np.int64)
    lib().orc_pairs_bruteforce(n, _ptr(x), _ptr(a), _ptr(ids, c_int32),
                               ctypes.byref(p), off, _ptr(out, c_int64), cnt)
    return out[:cnt]


def neighbours_of(x, a, ids, p: Params, off: float, k: int) -> np.ndarray:
    """Sorted ids of all particles within range of array index k."""
    x = _d(x)
    a = _d(a)
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    n = a.shape[0]
    cap = 4096
    out = np.zeros(cap, dtype=np.int64)
    cnt = lib().orc_neighbours_of(n, _ptr(x), _ptr(a), _ptr(ids, c_int32),
                                  ctypes.byref(p), off, int(k), _ptr(out, c_int64), cap)
    assert cnt <= cap
    return np.sort(out[:cnt])


def contact(p: Params, r, ai, aj, ui, uj, wi, wj, xi_old):
    """Eq. 4-5 contact on i from j: returns (F_i, T_i, T_j, xi_new)."""
    args = [_d(v) for v in (r, ui, uj, wi, wj, xi_old)]
    outs = [np.zeros(3) for _ in range(4)]
    lib().orc_contact(ctypes.byref(p), _ptr(args[0]), float(ai), float(aj),
                      *[_ptr(v) for v in args[1:]], *[_ptr(o) for o in outs])
    return tuple(outs)


def lubrication(p: Params, r, ai, aj, Vi, Vj, Wi, Wj, rate=None):
    """App. A lubrication: returns (F_i, F_j, T_i, T_j); the strain is that of
    a shear of rate ``rate`` along x (default: gdot)."""
    args = [_d(v) for v in (Vi, Vj, Wi, Wj)]
    outs = [np.zeros(3) for _ in range(4)]
    if rate is None:
        lib().orc_lubrication(ctypes.byref(p), _ptr(_d(r)), float(ai), float(aj),
                              *[_ptr(v) for v in args], *[_ptr(o) for o in outs])
    else:
        lib().orc_lubrication_rate(ctypes.byref(p), float(rate), _ptr(_d(r)), float(ai),
                                   float(aj), *[_ptr(v) for v in args], *[_ptr(o) for o in outs])
    return tuple(outs)


def rolling(p: Params, r, ai, aj, ui, uj, wi, wj, xr_old=(0, 0, 0)):
    """App. B rolling resistance of a contact: returns (T_i, T_j, xr_new)."""
    args = [_d(v) for v in (r, ui, uj, wi, wj, xr_old)]
    outs = [np.zeros(3) for _ in range(3)]
    lib().orc_rolling(ctypes.byref(p), _ptr(args[0]), float(ai), float(aj),
                      *[_ptr(v) for v in args[1:]], *[_ptr(o) for o in outs])
    return tuple(outs)


def flow_ux(p: Params, y):
    """U_inf,x at height y (Eq. 17)."""
    return lib().orc_flow_ux(ctypes.byref(p), float(y))


def flow_rate(p: Params, y):
    """Local shear rate dU_inf,x/dy at height y."""
    return lib().orc_flow_rate(ctypes.byref(p), float(y))


def faxen_ux(p: Params, y, a):
    """(1 + a^2/6 Laplacian) U_inf,x at height y (the Faxen velocity of Eq. A1)."""
    return lib().orc_faxen_ux(ctypes.byref(p), float(y), float(a))


def echem(p: Params, d, ai, aj, n):
    """Eq. 6-7 electro-chemical force on i from j at surface distance d along n."""
    F = np.zeros(3)
    lib().orc_echem(ctypes.byref(p), float(d), float(ai), float(aj), _ptr(_d(n)), _ptr(F))
    return F


def echem_range(p: Params) -> float:
    """Surface distance below which the electro-chemical forces act (0: off)."""
    return lib().orc_echem_range(ctypes.byref(p))


def pair_eval(p: Params, off, xi, xj, ui, uj, wi, wj, ai, aj, xi_old=(0, 0, 0),
              xr_old=None):
    """Whole pair from absolute state: (flags, F_i, F_j, T_i, T_j, S(3x3), xi_new),
    plus xr_new (the rolling stretch) at the end when xr_old is given."""
    ins = [_d(v) for v in (xi, xj, ui, uj, wi, wj)]
    xo = _d(xi_old)
    Fi, Fj, Ti, Tj, xn, rn = (np.zeros(3) for _ in range(6))
    S = np.zeros(9)
    if xr_old is None:
        fl = lib().orc_pair_eval(ctypes.byref(p), float(off), *[_ptr(v) for v in ins],
                                 float(ai), float(aj), _ptr(xo), _ptr(Fi), _ptr(Fj),
                                 _ptr(Ti), _ptr(Tj), _ptr(S), _ptr(xn))
        return fl, Fi, Fj, Ti, Tj, S.reshape(3, 3), xn
    ro = _d(xr_old)
    fl = lib().orc_pair_eval_full(ctypes.byref(p), float(off), *[_ptr(v) for v in ins],
                                  float(ai), float(aj), _ptr(xo), _ptr(ro), _ptr(Fi), _ptr(Fj),
                                  _ptr(Ti), _ptr(Tj), _ptr(S), _ptr(xn), _ptr(rn))
    return fl, Fi, Fj, Ti, Tj, S.reshape(3, 3), xn, rn


class System:
    """Oracle simulation: state + contact history, brute-force pairs."""

    def __init__(self, p: Params, x, a, ids=None, u=None, w=None, al=None, aw=None,
                 nstep: int = 0, cells: bool = False):
        a = _d(a)
        self.n = a.shape[0]
        self.p = p
        self._h = lib().orc_create(self.n, ctypes.byref(p))
        if ids is None:
            ids = np.arange(self.n, dtype=np.int32)
        self.ids = np.ascontiguousarray(ids, dtype=np.int32)
        self.a = a
        bufs = [None if v is None else _d(v).reshape(3, self.n) for v in (u, w, al, aw)]
        self._keep = bufs
        lib().orc_set_state(self._h, _ptr(_d(x).reshape(3, self.n)), _ptr(a),
                            _ptr(self.ids, c_int32), *[_opt(b) for b in bufs], int(nstep))
        self.set_cells(cells)

    def set_cells(self, cells: bool):
        """Neighbour search by the cell list with the half stencil (True) or
        the brute force (False, the default); the same pair set in the same
        order, hence the same numbers."""
        lib().orc_set_cells(self._h, 1 if cells else 0)

    def pairs_cell(self) -> np.ndarray:
        """(lo id, hi id) pairs of the current state found by the cell list,
        sorted (compare ``pairs_bruteforce``); None when the box holds too few
        cells for it."""
        cnt = lib().orc_pairs_cell(self._h, None, 0)
        if cnt < 0:
            return None
        out = np.zeros((max(cnt, 1), 2), dtype=np.int64)
        lib().orc_pairs_cell(self._h, _ptr(out, c_int64), cnt)
        return out[:cnt]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def init_accel(self):
        lib().orc_init_accel(self._h)

    def forces(self, commit: bool = False):
        lib().orc_forces(self._h, 1 if commit else 0)
        return self.get_forces()

    def forces_sampled(self, idx, scale: bool = False):
        """Force and torque (3, m) on the listed particles (array indices);
        with scale=True also the sums of the magnitudes of their terms (m)."""
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        m = idx.shape[0]
        F, T = np.zeros((3, m)), np.zeros((3, m))
        Fa, Ta = np.zeros(m), np.zeros(m)
        lib().orc_forces_sampled(self._h, _ptr(idx, c_int64), m, _ptr(F), _ptr(T), _ptr(Fa), _ptr(Ta))
        if scale:
            return F, T, Fa, Ta
        return F, T

    def step(self, nsteps: int = 1):
        lib().orc_step(self._h, int(nsteps))

    def get_state(self):
        n = self.n
        x, u, w, al, aw = (np.zeros((3, n)) for _ in range(5))
        lib().orc_get_state(self._h, _ptr(x), _ptr(u), _ptr(w), _ptr(al), _ptr(aw))
        return dict(x=x, u=u, w=w, al=al, aw=aw)

    def get_forces(self):
        n = self.n
        F, T = np.zeros((3, n)), np.zeros((3, n))
        s = np.zeros(9)
        lib().orc_get_forces(self._h, _ptr(F), _ptr(T), _ptr(s))
        return F, T, s.reshape(3, 3)

    def force_scale(self):
        """Per particle, the sums of the magnitudes of the terms of the force
        and of the torque of the last evaluation (pair terms and drag), (n,)
        each: the scale of the rounding error of any summation of them."""
        Fa, Ta = np.zeros(self.n), np.zeros(self.n)
        lib().orc_get_force_scale(self._h, _ptr(Fa), _ptr(Ta))
        return Fa, Ta

    def get_images(self):
        """Lees-Edwards image count along y of each particle since set_state
        (the unwrapped gradient coordinate is y + images * L_y)."""
        iy = np.zeros(self.n, dtype=np.int64)
        lib().orc_get_images(self._h, _ptr(iy, c_int64))
        return iy

    def set_history(self, keys, xi, xr=None):
        """Contact history: sorted keys lo_id << 32 | hi_id, sliding stretch
        (lo -> hi) and, optionally, the rolling stretch of each contact."""
        keys = np.ascontiguousarray(keys, dtype=np.int64)
        xi = _d(xi).reshape(-1, 3)
        xr = None if xr is None else _d(xr).reshape(-1, 3)
        lib().orc_set_history_r(self._h, keys.shape[0], _ptr(keys, c_int64), _ptr(xi), _opt(xr))

    def get_history(self, rolling: bool = False):
        """(keys, xi), or (keys, xi, xr) with the rolling stretch."""
        k = lib().orc_get_history(self._h, 0, None, None)
        keys = np.zeros(max(k, 1), dtype=np.int64)
        xi = np.zeros((max(k, 1), 3))
        xr = np.zeros((max(k, 1), 3))
        lib().orc_get_history_r(self._h, k, _ptr(keys, c_int64), _ptr(xi), _ptr(xr))
        if rolling:
            return keys[:k], xi[:k], xr[:k]
        return keys[:k], xi[:k]

    @property
    def nstep(self):
        return lib().orc_get_nstep(self._h)

    @property
    def npairs(self):
        return lib().orc_get_npairs(self._h)

    @property
    def ncontacts(self):
        return lib().orc_get_ncontacts(self._h)
