"""Python face of libdss: a ``Suspension`` handle over the C ABI.

Argument marshalling only: every step of the time step runs in the CUDA
kernels of libdss.so.  PyTorch provides device memory and the CUDA stream.
Arrays may be torch tensors (CPU or CUDA) or numpy arrays; vector quantities
have shape (3, n) (SoA), per-particle outputs are in id order.
"""
from __future__ import annotations

import ctypes
from ctypes import byref, c_double, c_int64, c_void_p

import numpy as np

from . import _native as nat


def default_params(box=None, *, kn=1e4, kt=None, gamma_n=None, mu=0.5, eta0=1.0, rho=1.0,
                   delta_lub=0.05, lub_eps=1e-3, a0=1.0, lub_cutoff_mode=0, precision="fp64",
                   shear_rate=1.0, dt=1e-4, cell_size=0.0, capacity_M=0, pair_capacity=0,
                   lub_taper=0.0, cell_mode=0, f_er=0.0, lambda_d=0.05, hamaker=0.0, vdw_eps=0.01,
                   wave_amp=0.0, wave_n=0, k_r=0.0):
    """Model parameters; kt defaults to kn/2 and gamma_n to 1e-7 kn / gdot.
    wave_amp, wave_n: the wavy shear flow of Eq. 17; k_r: the rolling spring of
    App. B (0: off)."""
    p = nat.Params()
    p.kn = kn
    p.kt = 0.5 * kn if kt is None else kt
    if gamma_n is None:
        gamma_n = 1e-7 * kn / shear_rate if shear_rate != 0 else 0.0
    p.gamma_n = gamma_n
    p.mu, p.eta0, p.rho = mu, eta0, rho
    p.delta_lub, p.lub_eps, p.a0 = delta_lub, lub_eps, a0
    p.lub_cutoff_mode = lub_cutoff_mode
    p.precision = {"fp64": nat.FP64, "mixed": nat.MIXED}[precision] if isinstance(precision, str) else precision
    p.shear_rate, p.dt = shear_rate, dt
    p.cell_size, p.capacity_M, p.pair_capacity = cell_size, capacity_M, pair_capacity
    p.lub_taper = lub_taper
    p.cell_mode = cell_mode
    p.f_er, p.lambda_d, p.hamaker, p.vdw_eps = f_er, lambda_d, hamaker, vdw_eps
    p.wave_amp, p.wave_n, p.k_r = wave_amp, int(wave_n), k_r
    return p


class _Arg:
    """Holds a contiguous buffer alive and exposes its address."""

    def __init__(self, v, dtype):
        import torch
        if v is None:
            self.obj, self.ptr = None, None
            return
        if isinstance(v, torch.Tensor):
            tdt = {np.float64: torch.float64, np.int32: torch.int32, np.int64: torch.int64}[dtype]
            if v.dtype == tdt and v.is_contiguous():
                self.obj, self.ptr = v, v.data_ptr()   # as it is (the common case)
                return
            t = v.detach()
            if t.dtype != tdt:
                t = t.to(tdt)
            t = t.contiguous()
            self.obj, self.ptr = t, t.data_ptr()
        else:
            a = np.ascontiguousarray(v, dtype=dtype)
            self.obj, self.ptr = a, a.ctypes.data


def capacity_estimate(a_min: float, a_max: float, a0: float = 1.0) -> int:
    """Half-list capacity M from the shell estimate (host only)."""
    return int(nat.load().dss_capacity_estimate(a_min, a_max, a0))


class Suspension:
    """N spheres in a Lees-Edwards sheared periodic box on one GPU."""

    def __init__(self, x, a, box, params=None, *, ids=None, u=None, w=None, alpha_lin=None,
                 alpha_ang=None, nstep=0, stream=None, **kw):
        import torch
        self.lib = nat.load()
        self.n = int(np.asarray(a).shape[0] if not isinstance(a, torch.Tensor) else a.shape[0])
        self.box = np.asarray(box, dtype=np.float64).copy()
        self.params = params if params is not None else default_params(self.box, **kw)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self._h = c_void_p()
        boxc = (c_double * 3)(*self.box.tolist())
        nat.check(self.lib.dss_create(byref(self._h), byref(self.params), self.n, boxc,
                                      c_void_p(stream.cuda_stream)), "dss_create")
        self.set_state(x, a, ids=ids, u=u, w=w, alpha_lin=alpha_lin, alpha_ang=alpha_ang, nstep=nstep)

    # -- state -------------------------------------------------------------
    def set_state(self, x, a, *, ids=None, u=None, w=None, alpha_lin=None, alpha_ang=None, nstep=0):
        args = [_Arg(x, np.float64), _Arg(a, np.float64), _Arg(ids, np.int32), _Arg(u, np.float64),
                _Arg(w, np.float64), _Arg(alpha_lin, np.float64), _Arg(alpha_ang, np.float64)]
        nat.check(self.lib.dss_set_state(self._h, *[c_void_p(g.ptr) for g in args], int(nstep)),
                  "dss_set_state")

    def load_state(self, x, u, w, alpha_lin, alpha_ang):
        """Per-step upload of the dynamic state (id order); keeps history."""
        args = [_Arg(v, np.float64) for v in (x, u, w, alpha_lin, alpha_ang)]
        self._keep = args
        nat.check(self.lib.dss_load_state(self._h, *[c_void_p(g.ptr) for g in args]),
                  "dss_load_state")

    def get_state_into(self, x, u, w, alpha_lin, alpha_ang):
        """Copies the state into caller buffers (torch tensors, any device)."""
        nat.check(self.lib.dss_get_state(self._h, *[c_void_p(t.data_ptr()) for t in
                                                    (x, u, w, alpha_lin, alpha_ang)]),
                  "dss_get_state")

    def step_io(self, state_in, nsteps: int, state_out=None, sigma=None):
        """Upload (x, u, w, alpha_lin, alpha_ang) (id order), advance nsteps,
        read the state after them into state_out (five buffers or None) and
        the last stress into sigma (9 doubles or None), with one
        synchronisation (dss_step_io).  Buffers are contiguous float64 torch
        tensors on any device, or numpy arrays (outputs are written in
        place, so they must be float64 and contiguous already)."""
        ins = [_Arg(v, np.float64) for v in state_in]
        outs = [_Arg(v, np.float64) for v in state_out] if state_out is not None else None
        sg = _Arg(sigma, np.float64) if sigma is not None else None
        pin = (c_void_p * 5)(*[g.ptr for g in ins])
        pout = (c_void_p * 5)(*[g.ptr for g in outs]) if outs is not None else None
        nat.check(self.lib.dss_step_io(self._h, pin, int(nsteps), pout, c_void_p(sg.ptr) if sg else None),
                  "dss_step_io")

    def set_profiling(self, on: bool = True):
        nat.check(self.lib.dss_set_profiling(self._h, 1 if on else 0), "dss_set_profiling")

    def last_step_ms(self) -> float:
        """GPU time of the last step() call (events around the graph launches)."""
        ms = c_double(0.0)
        nat.check(self.lib.dss_last_step_ms(self._h, byref(ms)), "dss_last_step_ms")
        return ms.value

    def profile(self):
        """{kernel name: summed ms} and the number of profiled steps."""
        ms = (c_double * nat.PROF_KERNELS)()
        cnt = c_int64(0)
        nat.check(self.lib.dss_get_profile(self._h, ms, byref(cnt)), "dss_get_profile")
        names = [self.lib.dss_profile_name(k).decode() for k in range(nat.PROF_KERNELS)]
        return dict(zip(names, list(ms))), cnt.value

    def state(self, device="cuda"):
        """Current x, u, w, alpha_lin, alpha_ang as (3, n) float64 tensors (id order)."""
        import torch
        out = {k: torch.empty((3, self.n), dtype=torch.float64, device=device)
               for k in ("x", "u", "w", "al", "aw")}
        nat.check(self.lib.dss_get_state(self._h, *[c_void_p(out[k].data_ptr())
                                                    for k in ("x", "u", "w", "al", "aw")]),
                  "dss_get_state")
        return out

    # -- the time step and its phases ---------------------------------------
    def step(self, nsteps: int = 1):
        nat.check(self.lib.dss_step(self._h, int(nsteps)), "dss_step")

    def neighbour_build(self):
        nat.check(self.lib.dss_neighbour_build(self._h), "dss_neighbour_build")

    def pairs(self) -> np.ndarray:
        """(lo id, hi id) pairs of the last build, sorted."""
        cnt = c_int64(0)
        nat.check(self.lib.dss_get_pairs(self._h, None, 0, byref(cnt)), "dss_get_pairs")
        out = np.zeros((max(cnt.value, 1), 2), dtype=np.int64)
        nat.check(self.lib.dss_get_pairs(self._h, c_void_p(out.ctypes.data), cnt.value, byref(cnt)),
                  "dss_get_pairs")
        return out[:cnt.value]

    def forces(self, device="cuda"):
        """Total force and torque (pairs + drag) at the current state, (3, n) each."""
        import torch
        F = torch.empty((3, self.n), dtype=torch.float64, device=device)
        T = torch.empty((3, self.n), dtype=torch.float64, device=device)
        nat.check(self.lib.dss_force_eval(self._h, c_void_p(F.data_ptr()), c_void_p(T.data_ptr())),
                  "dss_force_eval")
        return F, T

    def stress(self) -> np.ndarray:
        s = (c_double * 9)()
        nat.check(self.lib.dss_stress(self._h, s), "dss_stress")
        return np.array(list(s)).reshape(3, 3)

    def counters(self) -> dict:
        c = nat.Counters()
        nat.check(self.lib.dss_get_counters(self._h, byref(c)), "dss_get_counters")
        return dict(steps_done=c.steps_done, nstep=c.nstep, npairs=c.npairs, ncontacts=c.ncontacts,
                    max_row=c.max_row, band_checks=c.band_checks, M=c.M, ncell=tuple(c.ncell))

    def history(self, rolling: bool = False):
        """Committed contact history sorted by key: (keys, xi), or (keys, xi, xr)
        with the rolling stretch of App. B."""
        cnt = c_int64(0)
        nat.check(self.lib.dss_get_history(self._h, None, None, 0, byref(cnt)), "dss_get_history")
        k = cnt.value
        keys = np.zeros(max(k, 1), dtype=np.int64)
        xi = np.zeros((max(k, 1), 3))
        xr = np.zeros((max(k, 1), 3))
        nat.check(self.lib.dss_get_history_rolling(self._h, c_void_p(keys.ctypes.data),
                                                   c_void_p(xi.ctypes.data), c_void_p(xr.ctypes.data),
                                                   k, byref(cnt)), "dss_get_history_rolling")
        if rolling:
            return keys[:k], xi[:k], xr[:k]
        return keys[:k], xi[:k]

    # ---- analysis pass (dss_rheology, dss_get_images, dss_dispersion*,
    # dss_contact_clusters); per instance rows for a batch
    def _instances(self) -> int:
        return int(self.lib.dss_batch_size(self._h))

    def rheology(self, mean: bool = True) -> np.ndarray:
        """(K, 6): sigma, N1, N2, Pi, eta_r, eta_n per instance."""
        out = np.zeros((self._instances(), 6))
        nat.check(self.lib.dss_rheology(self._h, 1 if mean else 0, c_void_p(out.ctypes.data)), "dss_rheology")
        return out

    def images(self) -> np.ndarray:
        """Lees-Edwards image count along y of each id since the state was set."""
        iy = np.zeros(self.n, dtype=np.int32)
        nat.check(self.lib.dss_get_images(self._h, c_void_p(iy.ctypes.data)), "dss_get_images")
        return iy

    def dispersion_mark(self):
        nat.check(self.lib.dss_dispersion_mark(self._h), "dss_dispersion_mark")

    def dispersion(self) -> np.ndarray:
        """(K, 3): D_y, C_v, t - t0 per instance (Eq. 18-19)."""
        out = np.zeros((self._instances(), 3))
        nat.check(self.lib.dss_dispersion(self._h, c_void_p(out.ctypes.data)), "dss_dispersion")
        return out

    def contact_clusters(self):
        """(label by id: smallest id of its cluster, number of clusters)."""
        label = np.zeros(self.n, dtype=np.int32)
        cnt = c_int64(0)
        nat.check(self.lib.dss_contact_clusters(self._h, c_void_p(label.ctypes.data), byref(cnt)),
                  "dss_contact_clusters")
        return label, int(cnt.value)

    def phi_profile(self, nbins: int, a_split: float) -> np.ndarray:
        """(K, 2, nbins): local volume fraction along y in nbins slabs of the
        particles with radius <= a_split (class 0) and > a_split (class 1)."""
        out = np.zeros((self._instances(), 2, int(nbins)))
        nat.check(self.lib.dss_phi_profile(self._h, int(nbins), float(a_split), c_void_p(out.ctypes.data)),
                  "dss_phi_profile")
        return out

    def set_history(self, keys, xi, xr=None):
        """Replace the contact history (keys lo_id << 32 | hi_id, sliding stretch
        lo -> hi, optional rolling stretch)."""
        keys = np.ascontiguousarray(keys, dtype=np.int64)
        xi = np.ascontiguousarray(xi, dtype=np.float64).reshape(-1, 3)
        if xr is None:
            nat.check(self.lib.dss_set_history(self._h, keys.shape[0], c_void_p(keys.ctypes.data),
                                               c_void_p(xi.ctypes.data)), "dss_set_history")
            return
        xr = np.ascontiguousarray(xr, dtype=np.float64).reshape(-1, 3)
        nat.check(self.lib.dss_set_history_rolling(self._h, keys.shape[0], c_void_p(keys.ctypes.data),
                                                   c_void_p(xi.ctypes.data), c_void_p(xr.ctypes.data)),
                  "dss_set_history_rolling")

    def save(self) -> bytes:
        """Checkpoint of the dynamic state, history, step count and stress sums."""
        ln = ctypes.c_size_t(0)
        nat.check(self.lib.dss_save(self._h, None, byref(ln)), "dss_save")
        buf = ctypes.create_string_buffer(ln.value)
        nat.check(self.lib.dss_save(self._h, buf, byref(ln)), "dss_save")
        return buf.raw[:ln.value]

    def load(self, ckpt: bytes):
        """Resume from a checkpoint of a handle with the same configuration."""
        buf = ctypes.create_string_buffer(bytes(ckpt), len(ckpt))
        nat.check(self.lib.dss_load(self._h, buf, len(ckpt)), "dss_load")

    def autotune(self, trial_steps: int = 20, factors=None):
        """Time candidate cell edges (factors of the smallest admissible one),
        keep the fastest, restore the state.  Returns (cell edge, {factor: ms/step})."""
        f = np.ascontiguousarray(factors if factors is not None else [1.0, 1.1, 1.25, 1.5], dtype=np.float64)
        ms = np.zeros(f.shape[0])
        cs = c_double(0.0)
        dp = ctypes.POINTER(c_double)
        nat.check(self.lib.dss_autotune(self._h, int(trial_steps), f.shape[0], f.ctypes.data_as(dp),
                                        ms.ctypes.data_as(dp), byref(cs)), "dss_autotune")
        return cs.value, dict(zip(f.tolist(), ms.tolist()))

    def autotune_kernels(self, trial_steps: int = 20):
        """Time the kernel shapes (pair-kernel blocks per SM 3 or 4; the
        enumeration's candidate loop 1: plain, 4: screened with four loads
        ahead), keep the fastest, restore the state.  Returns
        ((blocks, loop), {(blocks, loop): ms/step})."""
        ms = np.zeros(4)
        ch = np.zeros(2, dtype=np.int32)
        dp = ctypes.POINTER(c_double)
        nat.check(self.lib.dss_autotune_kernels(self._h, int(trial_steps), ms.ctypes.data_as(dp),
                                                ch.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))),
                  "dss_autotune_kernels")
        keys = [(3, 1), (3, 4), (4, 1), (4, 4)]
        return (int(ch[0]), int(ch[1])), dict(zip(keys, ms.tolist()))

    def adjoint(self, nsteps: int, weights, *, ckpt_every: int = 20, initial_forces: bool = True):
        """Reverse-mode gradient of J = sum_n sum_q weights[n, q] sigma^{n+1}_q
        over nsteps steps from the current state (the handle ends after them).
        Returns dict(J, params (k_n, k_t, gamma_n, mu, delta_lub), x0, u0, w0,
        alpha0, beta0) with (3, n) arrays in id order."""
        W = np.ascontiguousarray(weights, dtype=np.float64).reshape(int(nsteps), 9)
        J = c_double(0.0)
        gp = np.zeros(5)
        outs = [np.zeros((3, self.n)) for _ in range(5)]
        dp = ctypes.POINTER(c_double)
        nat.check(self.lib.dss_adjoint(self._h, int(nsteps), int(ckpt_every), c_void_p(W.ctypes.data),
                                       1 if initial_forces else 0, byref(J), gp.ctypes.data_as(dp),
                                       *[c_void_p(o.ctypes.data) for o in outs]), "dss_adjoint")
        return dict(J=J.value, params=gp, x0=outs[0], u0=outs[1], w0=outs[2], alpha0=outs[3],
                    beta0=outs[4])

    def rollout_objective(self, nsteps: int, weights) -> float:
        """J of nsteps steps from the current state (forward only)."""
        W = np.asarray(weights, dtype=np.float64).reshape(int(nsteps), 9)
        J = 0.0
        for k in range(int(nsteps)):
            self.step(1)
            J += float((W[k] * self.stress().reshape(9)).sum())
        return J

    def device_bytes(self) -> int:
        return int(self.lib.dss_device_bytes(self._h))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self.lib.dss_destroy(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch(Suspension):
    """K independent suspensions advanced together in one handle.

    ``n`` lists the particle counts, ``boxes`` the (K, 3) box edges and
    ``shear_rates`` the K shear rates; ``gamma_n`` (K) defaults to
    1e-7 kn / gdot per instance.  x (3, sum n), a and the optional per-particle
    arrays are concatenated instance-major; ``ids`` (optional) permutes each
    instance's own index range.  Every ``Suspension`` method applies to the
    concatenated system; ``batch_stress`` returns every instance's stress.
    """

    def __init__(self, x, a, n, boxes, shear_rates, params=None, *, gamma_n=None, ids=None, u=None,
                 w=None, alpha_lin=None, alpha_ang=None, nstep=0, stream=None, **kw):
        import torch
        self.lib = nat.load()
        self.sizes = np.asarray(n, dtype=np.int64).copy()
        self.K = int(self.sizes.shape[0])
        self.n = int(self.sizes.sum())
        self.boxes = np.ascontiguousarray(boxes, dtype=np.float64).reshape(self.K, 3).copy()
        self.box = self.boxes[0]
        self.shear_rates = np.ascontiguousarray(shear_rates, dtype=np.float64).reshape(self.K).copy()
        self.params = params if params is not None else default_params(**kw)
        if gamma_n is None:
            kn = self.params.kn
            gamma_n = np.array([1e-7 * kn / g if g != 0 else 0.0 for g in self.shear_rates])
        self.gamma_n = np.ascontiguousarray(gamma_n, dtype=np.float64).reshape(self.K).copy()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self._h = c_void_p()
        dp = ctypes.POINTER(c_double)
        nat.check(self.lib.dss_batch_create(
            byref(self._h), byref(self.params), self.K,
            self.sizes.ctypes.data_as(ctypes.POINTER(c_int64)), self.boxes.ctypes.data_as(dp),
            self.shear_rates.ctypes.data_as(dp), self.gamma_n.ctypes.data_as(dp),
            c_void_p(stream.cuda_stream)), "dss_batch_create")
        self.set_state(x, a, ids=ids, u=u, w=w, alpha_lin=alpha_lin, alpha_ang=alpha_ang, nstep=nstep)

    def batch_stress(self, reset: bool = False):
        """(sigma, sigma_mean, steps): (K, 3, 3) stress of the last force
        evaluation, its mean over the steps since set_state / the last reset,
        and the number of those steps."""
        s = np.zeros((self.K, 9))
        m = np.zeros((self.K, 9))
        cnt = c_int64(0)
        nat.check(self.lib.dss_batch_stress(self._h, c_void_p(s.ctypes.data), c_void_p(m.ctypes.data),
                                            byref(cnt), 1 if reset else 0), "dss_batch_stress")
        return s.reshape(self.K, 3, 3), m.reshape(self.K, 3, 3), cnt.value
