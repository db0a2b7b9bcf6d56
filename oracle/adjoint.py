"""Reverse-mode derivatives of a rollout, CPU FP64 (oracle of the adjoint).

TEST INFRASTRUCTURE ONLY.  Only ``tests/`` may import this module.  It shares
no code with the CUDA path.

The rollout is restated with plain PyTorch CPU float64 tensor operations,
following oracle.c step for step: the brute-force pair set (taken from the C
oracle; it is discrete and carries no derivative), the stick-and-slide
contact of Eq. 4-5, the lubrication blocks of Eq. A2/A3 with the g functions
of Eq. A7 (6 pi eta0 prefactor) and the optional taper of the cutoff, the
optional electro-chemical forces of Eq. 6-7 (central, with their stresslet),
the optional wavy shear flow of Eq. 17 (velocities relative to the local
flow, the strain of the mean local rate, the Faxen drag, local stresslets)
and rolling resistance of App. B (a rolling stretch carried with the
contact, torques only), the Stokes drag of Eq. A1, the modified
velocity-Verlet step of Eq. 15 in the
Lees-Edwards box of Eq. 16, and the bulk stress of Eq. 8.  The objective is a
weighted sum of the stress over the steps,

    J = sum_{n=1..T} sum_q W[n-1, q] sigma^n_q      (sigma row major 3x3),

so W[n-1] = e_xy / (T eta0 gdot) gives the time-averaged relative viscosity.
Derivatives come from torch.autograd (a library primitive).  Branch decisions
(pair set, contact, Coulomb slips of both springs, gap clamp, taper ends,
box wraps) are taken
on the values and held fixed, so these are the derivatives of the branch
taken (pathwise derivatives).

Parity status: the forward rollout is pinned to oracle.c (same trajectory and
stress series); the gradient is pinned to central finite differences of
oracle.c with the event set checked unchanged (tests/test_oracle_adjoint.py).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import make_params, pairs_bruteforce

TD = torch.float64


def _gfun(name, al, ai, aj):
    """g coefficients of Eq. A7 (lengths only), numpy, per pair."""
    s = ai + aj
    if name == "XA_ii":
        return 2.0 * ai * al * al / (1.0 + al) ** 3
    if name == "XA_ij":
        return -2.0 * s * al * al / (1.0 + al) ** 4
    if name == "YA_ii":
        return 4.0 * ai / 15.0 * al * (2.0 + al + 2.0 * al * al) / (1.0 + al) ** 3
    if name == "YA_ij":
        return -4.0 * s / 15.0 * al * (2.0 + al + 2.0 * al * al) / (1.0 + al) ** 4
    if name == "YB_ii":
        return -2.0 * ai * ai / 15.0 * al * (4.0 + al) / (1.0 + al) ** 2
    if name == "YB_ij":
        return 2.0 * s ** 2 / 15.0 * al * (4.0 + al) / (1.0 + al) ** 4
    if name == "YC_ii":
        return 8.0 * ai ** 3 / 15.0 * al / (1.0 + al)
    if name == "YC_ij":
        return 2.0 * s ** 3 / 15.0 * al * al / (1.0 + al) ** 4
    if name == "XG_ii":
        return 2.0 * ai * ai * al * al / (1.0 + al) ** 3
    if name == "XG_ij":
        return -2.0 * s ** 2 * al * al / (1.0 + al) ** 5
    if name == "YG_ii":
        return ai * ai / 15.0 * al * (4.0 - al + 7.0 * al * al) / (1.0 + al) ** 3
    if name == "YG_ij":
        return -s ** 2 / 15.0 * al * (4.0 - al + 7.0 * al * al) / (1.0 + al) ** 5
    if name == "YH_ii":
        return 2.0 * ai ** 3 / 15.0 * al * (2.0 - al) / (1.0 + al) ** 2
    if name == "YH_ij":
        return s ** 3 / 15.0 * al * al * (1.0 + 7.0 * al) / (1.0 + al) ** 5
    raise KeyError(name)


def _coefficients(ai, aj):
    """Radius-only factors of every block (the X or Y factor is applied
    later): the ii, jj, ij, ji entries of Eq. A7 for each pair."""
    al = aj / ai
    ial = 1.0 / al
    c = {}
    for blk, jjf, jif in (("XA", al, 1.0), ("YA", al, 1.0), ("YB", -al * al, -1.0),
                          ("YC", al ** 3, 1.0), ("XG", -al * al, -1.0), ("YG", -al * al, -1.0),
                          ("YH", al ** 3, 1.0)):
        c[blk + "_ii"] = _gfun(blk + "_ii", al, ai, aj)
        c[blk + "_jj"] = jjf * _gfun(blk + "_ii", ial, ai, aj)
        c[blk + "_ij"] = _gfun(blk + "_ij", al, ai, aj)
        c[blk + "_ji"] = jif * _gfun(blk + "_ij", ial, ai, aj)
    return {k: torch.as_tensor(v, dtype=TD) for k, v in c.items()}


def _dot(a, b):
    return (a * b).sum(-1, keepdim=True)


def _cross(a, b):
    return torch.stack([a[:, 1] * b[:, 2] - a[:, 2] * b[:, 1],
                        a[:, 2] * b[:, 0] - a[:, 0] * b[:, 2],
                        a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0]], dim=1)


class Model:
    """Fixed settings of a differentiable rollout (everything except the
    differentiated inputs)."""

    def __init__(self, box, a, *, eta0=1.0, rho=1.0, lub_eps=1e-3, a0=1.0, lub_cutoff_mode=0,
                 shear_rate=1.0, dt=1e-4, lub_taper=0.0, nstep0=0, f_er=0.0, lambda_d=0.05,
                 hamaker=0.0, vdw_eps=0.01, wave_amp=0.0, wave_n=0, k_r=0.0):
        self.box = np.asarray(box, dtype=np.float64)
        self.a = np.asarray(a, dtype=np.float64)
        self.n = self.a.shape[0]
        self.eta0, self.rho, self.eps, self.a0 = eta0, rho, lub_eps, a0
        self.mode, self.gdot, self.dt, self.taper = lub_cutoff_mode, shear_rate, dt, lub_taper
        self.nstep0 = nstep0
        # electro-chemical forces, Eq. 6-7 (constants, not differentiated)
        self.f_er, self.lambda_d, self.hamaker, self.vdw_eps = f_er, lambda_d, hamaker, vdw_eps
        # the wavy shear flow of Eq. 17 and the rolling spring of App. B
        self.wave_amp, self.wave_n, self.k_r = wave_amp, int(wave_n), k_r
        self.wk = 2.0 * math.pi * float(wave_n) / float(self.box[1])
        at = torch.as_tensor(self.a, dtype=TD)
        self.at = at
        self.mass = 4.0 / 3.0 * math.pi * rho * at ** 3
        self.inertia = 0.4 * self.mass * at ** 2
        self.k6 = 6.0 * math.pi * eta0
        self.k8 = 8.0 * math.pi * eta0

    # U_inf,x, the local rate dU_inf,x/dy and the Faxen velocity of Eq. A1
    # (1 + a^2/6 Laplacian) U_inf,x at heights y (Eq. 17)
    def ux_inf(self, y):
        return self.gdot * y + self.wave_amp * torch.sin(self.wk * y)

    def rate(self, y):
        return self.gdot + self.wave_amp * self.wk * torch.cos(self.wk * y)

    def faxen_ux(self, y, a):
        return self.gdot * y + self.wave_amp * (1.0 - a * a * self.wk * self.wk / 6.0) * torch.sin(self.wk * y)

    def offset(self, nstep):
        t = float(nstep) * self.dt
        return math.fmod(self.gdot * self.box[1] * t, self.box[0])

    # -- one force evaluation ------------------------------------------------
    def forces(self, x, u, w, th, hist, nstep):
        """Forces, torques, stress and the new history at time nstep*dt.
        x, u, w: (3, n) tensors; th: dict of scalar tensors kn, kt, gn, mu,
        delta; hist: (keys ndarray sorted, xi (k, 3) tensor in lo -> hi
        orientation, xr (k, 3) tensor: the rolling stretch).  Returns F, T
        (3, n), sigma (9,), new hist, counts."""
        n, L, gd = self.n, self.box, self.gdot
        off = self.offset(nstep)
        p = make_params(L, kn=th["kn"].item(), kt=th["kt"].item(), gamma_n=th["gn"].item(),
                        mu=th["mu"].item(), eta0=self.eta0, rho=self.rho,
                        delta_lub=th["delta"].item(), lub_eps=self.eps, a0=self.a0,
                        lub_cutoff_mode=self.mode, shear_rate=gd, dt=self.dt, lub_taper=self.taper,
                        f_er=self.f_er, lambda_d=self.lambda_d, hamaker=self.hamaker, vdw_eps=self.vdw_eps,
                        wave_amp=self.wave_amp, wave_n=self.wave_n, k_r=self.k_r)
        xn = x.detach().numpy()
        pr = pairs_bruteforce(xn, self.a, np.arange(n, dtype=np.int32), p, off)
        i = torch.as_tensor(pr[:, 0])
        j = torch.as_tensor(pr[:, 1])
        P = pr.shape[0]
        # minimum image, Eq. 16 (shifts decided on the values)
        dx = x[0, j] - x[0, i]
        dy = x[1, j] - x[1, i]
        dz = x[2, j] - x[2, i]
        dyv = dy.detach().numpy()
        sy = np.where(dyv > 0.5 * L[1], -1, np.where(dyv < -0.5 * L[1], 1, 0))
        syt = torch.as_tensor(sy, dtype=TD)
        dy = dy + syt * L[1]
        dx = dx + syt * off
        dx = dx - L[0] * torch.as_tensor(np.rint(dx.detach().numpy() / L[0]), dtype=TD)
        dz = dz - L[2] * torch.as_tensor(np.rint(dz.detach().numpy() / L[2]), dtype=TD)
        r = torch.stack([dx, dy, dz], dim=1)
        ai = torch.as_tensor(self.a[pr[:, 0]], dtype=TD)
        aj = torch.as_tensor(self.a[pr[:, 1]], dtype=TD)
        S = ai + aj
        dist = torch.sqrt((r * r).sum(1))
        nv = r / dist[:, None]
        d = dist - S
        ui, uj = u[:, i].T, u[:, j].T
        wi, wj = w[:, i].T, w[:, j].T
        ujm = uj + torch.stack([syt * gd * L[1], torch.zeros_like(syt), torch.zeros_like(syt)], 1)
        yjm = x[1, j] + syt * L[1]
        # ---- contact, Eq. 4-5
        cmask = (d.detach() < 0.0)
        keys = (pr[:, 0].astype(np.int64) << 32) | pr[:, 1].astype(np.int64)
        hk, hxi, hxr = hist
        xo = torch.zeros((P, 3), dtype=TD)
        ro = torch.zeros((P, 3), dtype=TD)
        if len(hk):
            pos = np.searchsorted(hk, keys)
            pos = np.minimum(pos, len(hk) - 1)
            found = (hk[pos] == keys) if len(hk) else np.zeros(P, bool)
            if found.any():
                idx = torch.as_tensor(np.nonzero(found)[0])
                xo = xo.index_copy(0, idx, hxi[torch.as_tensor(pos[found])])
                ro = ro.index_copy(0, idx, hxr[torch.as_tensor(pos[found])])
        du = ujm - ui
        un = _dot(nv, du) * nv
        Fnor = th["kn"] * d[:, None] * nv + th["gn"] * un
        aw = ai[:, None] * wi + aj[:, None] * wj
        rel = du - _cross(aw, nv)
        ut = rel - _dot(nv, rel) * nv
        xp = xo - _dot(nv, xo) * nv
        xs = xp + ut * self.dt
        cap = th["mu"] * torch.sqrt((Fnor * Fnor).sum(1)) / th["kt"]
        xm = torch.sqrt((xs * xs).sum(1))
        slip = (xm.detach() > cap.detach()) & cmask
        scale = torch.where(slip, cap / torch.where(slip, xm, torch.ones_like(xm)), torch.ones_like(xm))
        xs = xs * scale[:, None]
        Ftan = th["kt"] * xs
        cm = cmask.to(TD)[:, None]
        Fc = (Fnor + Ftan) * cm
        nxf = _cross(nv, Ftan)
        Tci = ai[:, None] * nxf * cm
        Tcj = aj[:, None] * nxf * cm
        xinew = xs * cm
        # ---- rolling resistance, App. B: Eq. 5 on u_r = abar n x (w_i - w_j)
        # with k_r, under the sliding contact's Coulomb limit; torques only
        rslip = np.zeros(P, bool)
        xrnew = torch.zeros((P, 3), dtype=TD)
        if self.k_r > 0.0:
            abar_r = (2.0 * ai * aj / S)[:, None]
            xrp = ro - _dot(nv, ro) * nv
            xrs = xrp + (abar_r * _cross(nv, wi - wj)) * self.dt
            capr = th["mu"] * torch.sqrt((Fnor * Fnor).sum(1)) / self.k_r
            xrm = torch.sqrt((xrs * xrs).sum(1))
            rs = (xrm.detach() > capr.detach()) & cmask
            rscale = torch.where(rs, capr / torch.where(rs, xrm, torch.ones_like(xrm)), torch.ones_like(xrm))
            xrs = xrs * rscale[:, None]
            Tr = abar_r * _cross(nv, self.k_r * xrs) * cm
            Tci = Tci + Tr
            Tcj = Tcj - Tr
            xrnew = xrs * cm
            rslip = rs.numpy()
        # ---- lubrication, App. A (block form of Eq. A2/A3)
        ds = 2.0 * d / S
        ds = torch.where(ds.detach() < 0.0, torch.zeros_like(ds), ds)
        X = 1.0 / (ds + self.eps)
        Y = torch.log(1.0 / (ds + self.eps))
        c = _coefficients(ai.numpy(), aj.numpy())
        XY = {"XA": X, "YA": Y, "YB": Y, "YC": Y, "XG": X, "YG": Y, "YH": Y}
        cc = {k: (XY[k[:2]] * v)[:, None] for k, v in c.items()}
        # velocities relative to the flow at each centre (Eq. 17), the
        # strain of the mean of the two centres' local rates
        zP = torch.zeros(P, dtype=TD)
        Vi = ui - torch.stack([self.ux_inf(x[1, i]), zP, zP], 1)
        Vj = ujm - torch.stack([self.ux_inf(yjm), zP, zP], 1)
        rate_i, rate_j = self.rate(x[1, i]), self.rate(yjm)
        Wi = wi + torch.stack([zP, zP, 0.5 * rate_i], 1)
        Wj = wj + torch.stack([zP, zP, 0.5 * rate_j], 1)
        gp = (0.5 * (rate_i + rate_j))[:, None]

        def N(v):
            return _dot(nv, v) * nv

        def T(v):
            return v - _dot(nv, v) * nv

        nxWi, nxWj = _cross(nv, Wi), _cross(nv, Wj)
        nxVi, nxVj = _cross(nv, Vi), _cross(nv, Vj)
        E = torch.zeros((3, 3), dtype=TD)
        E[0, 1] = E[1, 0] = 0.5 * gd
        # E_inf of the pair: E_xy = E_yx = gp/2 (traceless, symmetric)
        En = 0.5 * gp * torch.stack([nv[:, 1], nv[:, 0], torch.zeros_like(nv[:, 0])], 1)
        Enn = _dot(nv, En)
        Pq = Enn
        Qn = 2.0 * En - 2.0 * Enn * nv
        nperp = _cross(nv, 2.0 * En)
        fi = (cc["XA_ii"] * N(Vi) + cc["YA_ii"] * T(Vi) + cc["XA_ij"] * N(Vj) + cc["YA_ij"] * T(Vj)
              + cc["YB_ii"] * nxWi + cc["YB_ji"] * nxWj)
        fj = (cc["XA_ji"] * N(Vi) + cc["YA_ji"] * T(Vi) + cc["XA_jj"] * N(Vj) + cc["YA_jj"] * T(Vj)
              + cc["YB_ij"] * nxWi + cc["YB_jj"] * nxWj)
        ti = -cc["YB_ii"] * nxVi - cc["YB_ij"] * nxVj + cc["YC_ii"] * T(Wi) + cc["YC_ij"] * T(Wj)
        tj = -cc["YB_ji"] * nxVi - cc["YB_jj"] * nxVj + cc["YC_ji"] * T(Wi) + cc["YC_jj"] * T(Wj)
        gi = (cc["XG_ii"] * Pq * nv + cc["YG_ii"] * Qn) + (cc["XG_ji"] * Pq * nv + cc["YG_ji"] * Qn)
        gj = (cc["XG_ij"] * Pq * nv + cc["YG_ij"] * Qn) + (cc["XG_jj"] * Pq * nv + cc["YG_jj"] * Qn)
        hi = cc["YH_ii"] * nperp + cc["YH_ji"] * nperp
        hj = cc["YH_ij"] * nperp + cc["YH_jj"] * nperp
        k = self.k6
        Fli, Flj = -k * fi + k * gi, -k * fj + k * gj
        Tli, Tlj = -k * ti + k * hi, -k * tj + k * hj
        if self.taper > 0.0:
            dl = th["delta"] * self.a0 if self.mode == 1 else th["delta"] * 0.5 * S
            t = (dl - d) / (self.taper * dl)
            tv = t.detach()
            s = torch.where(tv >= 1.0, torch.ones_like(t),
                            torch.where(tv <= 0.0, torch.zeros_like(t), t * t * (3.0 - 2.0 * t)))
            Fli, Flj, Tli, Tlj = (s[:, None] * v for v in (Fli, Flj, Tli, Tlj))
        # lubrication only within its own cutoff (the listing test with the
        # lubrication range; the list may reach further for Eq. 6-7)
        dlub = th["delta"].item() * self.a0 if self.mode == 1 else th["delta"].item() * S.numpy() * 0.5
        r2v = ((dx * dx).detach().numpy() + (dy * dy).detach().numpy()) + (dz * dz).detach().numpy()
        lub_on = r2v < (S.numpy() + dlub) ** 2
        lm = torch.as_tensor(lub_on.astype(np.float64), dtype=TD)[:, None]
        Fli, Flj, Tli, Tlj = (lm * v for v in (Fli, Flj, Tli, Tlj))
        # electro-chemical forces, Eq. 6-7: central, stresslet r (x) F like contact
        if self.f_er > 0.0 or self.hamaker > 0.0:
            abar = 2.0 * ai * aj / S
            dv = d.detach()
            mE = torch.zeros_like(d)
            if self.f_er > 0.0:
                rep_ = torch.where(dv >= 0.0, torch.exp(-d / self.lambda_d), torch.ones_like(d))
                mE = mE - torch.where(dv < 20.0 * self.lambda_d, self.f_er * (abar / self.a0) * rep_,
                                      torch.zeros_like(d))
            if self.hamaker > 0.0:
                eps = self.vdw_eps * abar
                dp = torch.where(dv >= 0.0, d, torch.zeros_like(d))
                mE = mE + torch.where(dv < 4.0 * self.a0, self.hamaker * abar / (12.0 * (dp * dp + eps * eps)),
                                      torch.zeros_like(d))
            Fc = Fc + mE[:, None] * nv
        Fi = Fc + Fli
        Fj = -Fc + Flj
        Ti = Tci + Tli
        Tj = Tcj + Tlj
        F = torch.zeros((n, 3), dtype=TD).index_add(0, i, Fi).index_add(0, j, Fj)
        Tq = torch.zeros((n, 3), dtype=TD).index_add(0, i, Ti).index_add(0, j, Tj)
        # Stokes drag, Eq. A1 (Faxen velocity and local Omega_inf at the centre)
        V = torch.stack([u[0] - self.faxen_ux(x[1], self.at), u[1], u[2]], 1)
        F = F - self.k6 * self.at[:, None] * V
        zn = torch.zeros(n, dtype=TD)
        Wp = w.T + torch.stack([zn, zn, 0.5 * self.rate(x[1])], 1)
        Tq = Tq - self.k8 * (self.at ** 3)[:, None] * Wp
        # stress, Eq. 8 and 9
        Sp = (r[:, :, None] * Fc[:, None, :] + 0.5 * (r[:, :, None] * Fli[:, None, :]
                                                     + Fli[:, :, None] * r[:, None, :])).sum(0)
        Vol = float(L[0] * L[1] * L[2])
        # single-particle stresslets 20/3 pi eta0 a^3 E_inf(x_i); the fluid
        # term with the box mean of E_inf
        ein = 20.0 / 3.0 * math.pi * self.eta0 * (self.at ** 3 * 0.5 * self.rate(x[1])).sum()
        Sein = torch.zeros((3, 3), dtype=TD)
        Sein = Sein.index_put((torch.tensor([0, 1]), torch.tensor([1, 0])), ein.expand(2))
        sigma = (2.0 * self.eta0 * E + (Sein + Sp) / Vol).reshape(9)
        # new history: the pairs in contact, sorted by key (ids are indices, lo = i)
        cm_np = cmask.numpy()
        nk = keys[cm_np]
        order = np.argsort(nk, kind="stable")
        sel = torch.as_tensor(np.nonzero(cm_np)[0][order])
        new_hist = (nk[order], xinew[sel], xrnew[sel])
        # event signature: pair count, contact count, slip count, and the
        # identities of the contacts, slips and pairs in the taper band
        band = np.zeros(P, bool)
        if self.taper > 0.0:
            dlv = (th["delta"].item() * (self.a0 if self.mode == 1 else 0.5 * S.numpy()))
            band = (d.detach().numpy() > (1.0 - self.taper) * dlv)
        sl = slip.numpy()
        ev = (P, int(cm_np.sum()), int(sl.sum()), hash(keys[cm_np].tobytes()),
              hash(keys[sl].tobytes()), hash(keys[band].tobytes()), hash(keys.tobytes()),
              hash(keys[lub_on].tobytes()), hash(keys[rslip].tobytes()))
        return F.T, Tq.T, sigma, new_hist, ev

    # -- the rollout -----------------------------------------------------------
    def rollout(self, x0, u0, w0, th, nsteps, weights=None):
        """J and the stress series of nsteps steps from (x0, u0, w0) with the
        initial accelerations from one force evaluation (empty history).
        Returns (J, sigma list, event counts per step, final state dict)."""
        dt, L, gd = self.dt, self.box, self.gdot
        nstep = self.nstep0
        F, Tq, _, _, ev0 = self.forces(x0, u0, w0, th, (np.zeros(0, np.int64), None, None), nstep)
        al = F / self.mass
        aw = Tq / self.inertia
        x, u, w = x0, u0, w0
        hist = (np.zeros(0, np.int64), None, None)
        J = torch.zeros((), dtype=TD)
        sig, events = [], [ev0]
        for k in range(nsteps):
            nstep += 1
            off = self.offset(nstep)
            x = x + dt * u + 0.5 * dt * dt * al
            u = u + 0.5 * dt * al
            w = w + 0.5 * dt * aw
            # Lees-Edwards wrap, Eq. 16 (decisions on the values)
            xv = x.detach().numpy()
            up = xv[1] >= L[1]
            dn = xv[1] < 0.0
            cross = np.where(up, -1.0, np.where(dn, 1.0, 0.0))
            ct = torch.as_tensor(cross, dtype=TD)
            ny = x[1] + ct * L[1]
            nx = x[0] + ct * off
            # x into [0, L_x), z into [0, L_z): fmod then the corrections
            nxv = nx.detach().numpy()
            q = np.fmod(nxv, L[0]) - nxv
            q = q + np.where(nxv + q < 0.0, L[0], 0.0)
            q = q - np.where(nxv + q >= L[0], L[0], 0.0)
            nx = nx + torch.as_tensor(q, dtype=TD)
            nz = x[2]
            zv = nz.detach().numpy()
            nz = nz + torch.as_tensor(np.where(zv >= L[2], -L[2], np.where(zv < 0.0, L[2], 0.0)), dtype=TD)
            x = torch.stack([nx, ny, nz])
            u = torch.stack([u[0] + ct * gd * L[1], u[1], u[2]])
            F, Tq, s, hist, ev = self.forces(x, u, w, th, hist, nstep)
            al = F / self.mass
            aw = Tq / self.inertia
            u = u + 0.5 * dt * al
            w = w + 0.5 * dt * aw
            sig.append(s)
            events.append(ev)
            if weights is not None:
                J = J + (torch.as_tensor(weights[k], dtype=TD) * s).sum()
        return J, sig, events, dict(x=x, u=u, w=w, al=al, aw=aw)


def gradients(box, x0, a, u0, w0, nsteps, weights, *, kn=1e4, kt=None, gamma_n=None, mu=0.5,
              delta_lub=0.05, **kw):
    """J and dJ/d{x0, u0, w0, kn, kt, gamma_n, mu, delta_lub} (pathwise)."""
    gd = kw.get("shear_rate", 1.0)
    kt = 0.5 * kn if kt is None else kt
    gamma_n = 1e-7 * kn / gd if gamma_n is None else gamma_n
    m = Model(box, a, **kw)
    xs = torch.tensor(np.asarray(x0, dtype=np.float64), requires_grad=True)
    us = torch.tensor(np.asarray(u0, dtype=np.float64), requires_grad=True)
    ws = torch.tensor(np.asarray(w0, dtype=np.float64), requires_grad=True)
    th = {k: torch.tensor(float(v), dtype=TD, requires_grad=True)
          for k, v in (("kn", kn), ("kt", kt), ("gn", gamma_n), ("mu", mu), ("delta", delta_lub))}
    J, sig, events, fin = m.rollout(xs, us, ws, th, nsteps, weights)
    gx, gu, gw, *gp = torch.autograd.grad(J, [xs, us, ws] + [th[k] for k in ("kn", "kt", "gn", "mu", "delta")],
                                          allow_unused=True)
    gp = [0.0 if g is None else float(g) for g in gp]
    return dict(J=J.item(), x0=gx.numpy(), u0=gu.numpy(), w0=gw.numpy(),
                params=np.array(gp), sigma=np.array([s.detach().numpy() for s in sig]),
                events=events, final={k: v.detach().numpy() for k, v in fin.items()})
