// Reverse sweep of a rollout (the adjoint of the time step of Eq. 15-16 with
// the pair model of Eq. 4-5 and App. A and the stress of Eq. 8).
//
// The objective is J = sum_n sum_q W[n][q] sigma^n_q over the steps of the
// rollout.  dss_adjoint (host side in dss_api.cu) replays each checkpointed
// segment forward, recording per step a tape (the sorted state at the force
// evaluation, the pair list, the stretch carried into each pair and where it
// came from), then walks the segment backwards:
//
//   k_adj_pre      per particle: cotangents of force and torque from the
//                  adjoint accelerations (and the corrector u^{n+1} = u^{n+1/2}
//                  + dt/2 alpha^{n+1}), the Stokes-drag part of the VJP;
//   k_adj_pairs    per pair: the vector-Jacobian product of the pair model
//                  with respect to its 25 inputs (r, y_i, y_j, u_i, u_j, w_i,
//                  w_j, the carried stretch, k_n, k_t, gamma_n, mu, delta_lub;
//                  with rolling resistance also the carried rolling stretch),
//                  the reverse of the pair model of dss_pair_model.cuh written
//                  out by hand (pair_vjp) and contracted with the cotangents;
//                  the stretch adjoints are routed to the pair of the previous
//                  step they came from;
//   k_adj_gather   per particle: own-row and partner contributions summed in
//                  a fixed order (owner rows in list order, partner records by
//                  increasing pair index), so gradients are bitwise
//                  reproducible;
//   k_adj_predict  per particle: the predictor of Eq. 15a-b backwards.
//
// With the wavy shear flow of Eq. 17 the ambient velocity and spin, the
// pair's strain rate, the Faxen drag and the local single-particle
// stresslets depend on y; with rolling resistance (App. B) the rolling
// stretch is carried and differentiated like the sliding one.  Branch
// decisions (pair set, contact, Coulomb slips, gap clamp, taper ends, box
// wraps) are those of the forward step and are held fixed.
#include <algorithm>
#include <climits>
#include <cstring>

#include "dss_internal.cuh"
#include "dss_pair_model.cuh"

namespace {
constexpr int kThreads = 128;
constexpr int kAdjThreads = 128;
constexpr int kNin = 28;          // pair-model inputs differentiated

struct PairIn {
  double r[3];
  double yi, yj;
  double ui[3], uj[3], wi[3], wj[3], xo[3], ro[3];
  double ai, aj;
  int sy;
};

struct PairCot {
  double F[3], Ti[3], Tj[3], xi[3], xr[3];
  double Ws[9];      // stress weights / volume
};

// The vector-Jacobian product of one pair, written out by hand: one forward sweep
// through the pair model of dss_pair_model.cuh (Eq. 4-5, App. A, Eq. 6-7,
// App. B, Eq. 17) keeping its intermediates, then one backward sweep that
// applies the chain rule operation by operation in reverse order.  Branches
// (contact, Coulomb slips, gap clamp, taper ends, the electro-chemical and
// lubrication ranges) are those of the values.  About three forward
// evaluations of work (forward-mode derivative passes over the 28 inputs
// took thirty, on GB300's narrow FP64 pipe).
using V3d = Vec3<double>;
__device__ __forceinline__ V3d operator-(const V3d& a) { return mk3<double>(-a.x, -a.y, -a.z); }
__device__ __forceinline__ V3d operator*(const V3d& a, double s) { return mk3<double>(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ void acc3(V3d& a, const V3d& b) { a = a + b; }
// d/dn and d/dv of c . tang(n, v) = c . (v - (n.v) n)
__device__ __forceinline__ void tang_rev(const V3d& n, const V3d& v, const V3d& cb, V3d& nb, V3d& vb) {
  const double nc = dot(n, cb), nv = dot(n, v);
  acc3(vb, cb - n * nc);
  acc3(nb, -(cb * nv + v * nc));
}
// d/da and d/db of c . (a x b)
__device__ __forceinline__ void cross_rev(const V3d& a, const V3d& b, const V3d& cb, V3d& ab, V3d& bb) {
  acc3(ab, cross(b, cb));
  acc3(bb, cross(cb, a));
}
// a Coulomb rescale x = (cap / |x0|) x0 when |x0| > cap: adjoints of x0 and cap
__device__ __forceinline__ void cap_rev(const V3d& x0, double cap, bool slip, const V3d& xb, V3d& x0b,
                                        double& capb) {
  if (!slip) {
    acc3(x0b, xb);
    return;
  }
  const double xm = ::sqrt(dot(x0, x0)), f = cap / xm, xx = dot(xb, x0);
  acc3(x0b, xb * f - x0 * (cap * xx / (xm * xm * xm)));
  capb += xx / xm;
}

__device__ __noinline__ void pair_vjp(const Geo& g, const InstGeo& I, const PairIn& in, const PairCot& c,
                                      double* out) {
  const V3d zero = mk3<double>(0.0, 0.0, 0.0);
  const double ai = in.ai, aj = in.aj, S = ai + aj;
  const double gd = I.gdot, kn = g.kn, kt = g.kt, gn = I.gn, mu = g.mu, delta = g.delta;
  // ---- forward sweep
  const V3d r = mk3<double>(in.r[0], in.r[1], in.r[2]);
  const double rr = ::sqrt(dot(r, r));
  const double ir = 1.0 / rr;
  const V3d n = r * ir;
  const double d = rr - S;
  const V3d ui = mk3<double>(in.ui[0], in.ui[1], in.ui[2]), uj = mk3<double>(in.uj[0], in.uj[1], in.uj[2]);
  const V3d wi = mk3<double>(in.wi[0], in.wi[1], in.wi[2]), wj = mk3<double>(in.wj[0], in.wj[1], in.wj[2]);
  V3d Vi = mk3<double>(ui.x - gd * in.yi, ui.y, ui.z), Vj = mk3<double>(uj.x - gd * in.yj, uj.y, uj.z);
  V3d Wi = mk3<double>(wi.x, wi.y, wi.z + 0.5 * gd), Wj = mk3<double>(wj.x, wj.y, wj.z + 0.5 * gd);
  double rate = gd, si = 0.0, sj = 0.0, ci = 0.0, cj = 0.0;
  const double U = g.wave_amp, kw = I.wave_k;
  if (g.wave) {
    sincos(kw * in.yi, &si, &ci);
    sincos(kw * in.yj, &sj, &cj);
    Vi.x -= U * si;
    Vj.x -= U * sj;
    Wi.z += 0.5 * U * kw * ci;
    Wj.z += 0.5 * U * kw * cj;
    rate += 0.5 * U * kw * (ci + cj);
  }
  const V3d du = mk3<double>(uj.x + in.sy * gd * I.L[1] - ui.x, uj.y - ui.y, uj.z - ui.z);
  const V3d xo = mk3<double>(in.xo[0], in.xo[1], in.xo[2]), ro = mk3<double>(in.ro[0], in.ro[1], in.ro[2]);
  // contact
  const bool contact = d < 0.0;
  double fn = 0.0, cap = 0.0, capr = 0.0;
  bool slip = false, rslip = false;
  V3d aw = zero, rel = zero, xs0 = zero, xs = zero, Ft = zero, Fc = zero, nxf = zero, wr = zero, xr0 = zero,
      xr = zero;
  const double abar = 2.0 * ai * aj / (ai + aj);
  const bool rolling = contact && g.k_r > 0.0;
  if (contact) {
    fn = kn * d + gn * dot(n, du);
    aw = wi * ai + wj * aj;
    rel = du - cross(aw, n);
    xs0 = tang(n, xo) + g.dt * tang(n, rel);
    cap = mu * fabs(fn) / kt;
    const double xm = ::sqrt(dot(xs0, xs0));
    slip = xm > cap;
    xs = slip ? xs0 * (cap / xm) : xs0;
    Ft = xs * kt;
    Fc = n * fn + Ft;
    nxf = cross(n, Ft);
    if (rolling) {
      wr = wi - wj;
      xr0 = tang(n, ro) + cross(n, wr) * (g.dt * abar);
      capr = mu * fabs(fn) / g.k_r;
      const double xrm = ::sqrt(dot(xr0, xr0));
      rslip = xrm > capr;
      xr = rslip ? xr0 * (capr / xrm) : xr0;
    }
  }
  // electro-chemical forces and the lubrication range
  bool lub_on = true;
  double m = 0.0, mp = 0.0;   // m(d) and dm/dd
  if (g.de > 0.0) {
    if (g.f_er > 0.0 && d < 20.0 * g.lambda_d) {
      const double A = g.f_er * (abar / g.a0);
      if (d >= 0.0) {
        const double ex = ::exp(-d / g.lambda_d);
        m -= A * ex;
        mp += A * ex / g.lambda_d;
      } else {
        m -= A;
      }
    }
    if (g.hamaker > 0.0 && d < 4.0 * g.a0) {
      const double eps = g.vdw_eps * abar, dp = d >= 0.0 ? d : 0.0;
      const double den = 12.0 * (dp * dp + eps * eps);
      m += (g.hamaker * abar) / den;
      if (d >= 0.0) mp -= (g.hamaker * abar) * 24.0 * dp / (den * den);
    }
    Fc = Fc + n * m;
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(r.x, r.x), __dmul_rn(r.y, r.y)), __dmul_rn(r.z, r.z));
    const double dl = g.mode == 1 ? __dmul_rn(delta, g.a0) : __dmul_rn(__dmul_rn(delta, S), 0.5);
    const double sl = __dadd_rn(S, dl);
    lub_on = r2 < __dmul_rn(sl, sl);
  }
  // lubrication
  const double A = ai, B = aj, AB = A * B;
  const double iS = 1.0 / S, iS2 = iS * iS, iS3 = iS2 * iS;
  const double cxa = 2.0 * AB * AB * iS3;
  const double cya = (4.0 / 15.0) * AB * (2.0 * A * A + AB + 2.0 * B * B) * iS3;
  const double cybi = -(2.0 / 15.0) * A * AB * (4.0 * A + B) * iS2;
  const double cybj = -(2.0 / 15.0) * AB * B * (A + 4.0 * B) * iS2;
  const double cyci = (8.0 / 15.0) * A * A * AB * iS;
  const double cycj = (8.0 / 15.0) * AB * B * B * iS;
  const double cycx = (2.0 / 15.0) * AB * AB * iS;
  const double cxg = 2.0 * AB * AB * iS2;
  const double cyg = (1.0 / 15.0) * AB * (4.0 - 6.0 * AB * iS2);
  const double cyhi = iS2 * ((2.0 / 15.0) * A * A * AB * (2.0 * A - B) + (1.0 / 15.0) * AB * AB * (7.0 * A + B));
  const double cyhj = iS2 * ((1.0 / 15.0) * AB * AB * (A + 7.0 * B) + (2.0 / 15.0) * AB * B * B * (2.0 * B - A));
  double X = 0.0, Y = 0.0, dd = 1.0, sw = 1.0, tt = 2.0, dl = 0.0;
  bool clamped = false, tapered = false;
  V3d dV = zero, twoEn = zero, Qn = zero, nperp = zero, tWi = zero, tWj = zero, ndV = zero;
  V3d Fl0 = zero, Tli0 = zero, Tlj0 = zero;
  double nV = 0.0, P = 0.0;
  if (lub_on) {
    double ds = 2.0 * d / S;
    clamped = !(ds >= 0.0);
    if (clamped) ds = 0.0;
    dd = ds + g.eps;
    X = 1.0 / dd;
    Y = -::log(dd);
    dV = Vi - Vj;
    nV = dot(n, dV);
    const V3d fr = n * (X * cxa * nV) + tang(n, dV) * (Y * cya) + cross(n, Wi) * (Y * cybi) +
                   cross(n, Wj) * (Y * cybj);
    twoEn = mk3<double>(rate * n.y, rate * n.x, 0.0);
    P = rate * n.x * n.y;
    Qn = twoEn - n * (2.0 * P);
    nperp = cross(n, twoEn);
    const V3d fe = n * (X * cxg * P) + Qn * (Y * cyg);
    Fl0 = (fe - fr) * g.k6;
    ndV = cross(n, dV);
    tWi = tang(n, Wi);
    tWj = tang(n, Wj);
    Tli0 = (ndV * (Y * cybi) - (tWi * (Y * cyci) + tWj * (Y * cycx)) + nperp * (Y * cyhi)) * g.k6;
    Tlj0 = (ndV * (Y * cybj) - (tWi * (Y * cycx) + tWj * (Y * cycj)) + nperp * (Y * cyhj)) * g.k6;
    if (g.taper > 0.0) {
      dl = g.mode == 1 ? delta * g.a0 : delta * (0.5 * S);
      tt = (dl - d) / (g.taper * dl);
      if (tt < 1.0) {
        tapered = true;
        sw = tt > 0.0 ? tt * tt * (3.0 - 2.0 * tt) : 0.0;
      }
    }
  }
  const V3d Fl = Fl0 * sw;
  // ---- backward sweep
  const V3d cF = mk3<double>(c.F[0], c.F[1], c.F[2]);
  const V3d cTi = mk3<double>(c.Ti[0], c.Ti[1], c.Ti[2]), cTj = mk3<double>(c.Tj[0], c.Tj[1], c.Tj[2]);
  // stress of Eq. 9, weighted: sum_ab W_ab (r_a Fc_b + (r_a Fl_b + r_b Fl_a) / 2)
  const double* W = c.Ws;
  const V3d Wr = mk3<double>(W[0] * r.x + W[1] * r.y + W[2] * r.z, W[3] * r.x + W[4] * r.y + W[5] * r.z,
                             W[6] * r.x + W[7] * r.y + W[8] * r.z);
  const V3d WTr = mk3<double>(W[0] * r.x + W[3] * r.y + W[6] * r.z, W[1] * r.x + W[4] * r.y + W[7] * r.z,
                              W[2] * r.x + W[5] * r.y + W[8] * r.z);
  const V3d WFc = mk3<double>(W[0] * Fc.x + W[1] * Fc.y + W[2] * Fc.z, W[3] * Fc.x + W[4] * Fc.y + W[5] * Fc.z,
                              W[6] * Fc.x + W[7] * Fc.y + W[8] * Fc.z);
  const V3d WFl = mk3<double>(W[0] * Fl.x + W[1] * Fl.y + W[2] * Fl.z, W[3] * Fl.x + W[4] * Fl.y + W[5] * Fl.z,
                              W[6] * Fl.x + W[7] * Fl.y + W[8] * Fl.z);
  const V3d WTFl = mk3<double>(W[0] * Fl.x + W[3] * Fl.y + W[6] * Fl.z, W[1] * Fl.x + W[4] * Fl.y + W[7] * Fl.z,
                               W[2] * Fl.x + W[5] * Fl.y + W[8] * Fl.z);
  V3d rb = WFc + (WFl + WTFl) * 0.5;
  const V3d Fcb = cF + WTr;
  const V3d Flb = cF + (WTr + Wr) * 0.5;
  V3d nb = zero, Vib = zero, Vjb = zero, Wib = zero, Wjb = zero, dub = zero, wib = zero, wjb = zero;
  V3d xob = zero, rob = zero;
  double db = 0.0, rateb = 0.0, knb = 0.0, ktb = 0.0, gnb = 0.0, mub = 0.0, deltab = 0.0;
  // lubrication
  if (lub_on) {
    V3d Fl0b = Flb * sw, Tli0b = cTi * sw, Tlj0b = cTj * sw;
    if (tapered && tt > 0.0) {
      const double swb = dot(Flb, Fl0) + dot(cTi, Tli0) + dot(cTj, Tlj0);
      const double ttb = swb * 6.0 * tt * (1.0 - tt);
      // tt = (dl - d) / (w dl)
      db += -ttb / (g.taper * dl);
      const double dlb = ttb * d / (g.taper * dl * dl);
      deltab += dlb * (g.mode == 1 ? g.a0 : 0.5 * S);
    }
    const V3d feb = Fl0b * g.k6, frb = Fl0b * (-g.k6);
    const V3d Ab = Tli0b * g.k6, Bb = Tlj0b * g.k6;
    // torques
    double Yb = 0.0, Xb = 0.0;
    Yb += dot(Ab, ndV) * cybi + dot(Bb, ndV) * cybj;
    const V3d ndVb = Ab * (Y * cybi) + Bb * (Y * cybj);
    Yb += -dot(Ab, tWi) * cyci - dot(Bb, tWj) * cycj - (dot(Ab, tWj) + dot(Bb, tWi)) * cycx;
    const V3d tWib = -(Ab * (Y * cyci) + Bb * (Y * cycx));
    const V3d tWjb = -(Ab * (Y * cycx) + Bb * (Y * cycj));
    Yb += dot(Ab, nperp) * cyhi + dot(Bb, nperp) * cyhj;
    V3d nperpb = Ab * (Y * cyhi) + Bb * (Y * cyhj);
    // fe = (X cxg P) n + (Y cyg) Qn
    double Pb = 0.0;
    Xb += dot(feb, n) * cxg * P;
    Pb += dot(feb, n) * X * cxg;
    acc3(nb, feb * (X * cxg * P));
    Yb += dot(feb, Qn) * cyg;
    const V3d Qnb = feb * (Y * cyg);
    // Qn = twoEn - 2 P n
    V3d twoEnb = Qnb;
    Pb += -2.0 * dot(Qnb, n);
    acc3(nb, Qnb * (-2.0 * P));
    // nperp = n x twoEn
    cross_rev(n, twoEn, nperpb, nb, twoEnb);
    // P = rate n_x n_y; twoEn = rate (n_y, n_x, 0)
    rateb += Pb * n.x * n.y + twoEnb.x * n.y + twoEnb.y * n.x;
    nb.x += Pb * rate * n.y + rate * twoEnb.y;
    nb.y += Pb * rate * n.x + rate * twoEnb.x;
    // tang(n, Wi), tang(n, Wj); ndV = n x dV
    tang_rev(n, Wi, tWib, nb, Wib);
    tang_rev(n, Wj, tWjb, nb, Wjb);
    V3d dVb = zero;
    cross_rev(n, dV, ndVb, nb, dVb);
    // fr = (X cxa nV) n + (Y cya) tang(n, dV) + (Y cybi) n x Wi + (Y cybj) n x Wj
    double nVb = 0.0;
    Xb += dot(frb, n) * cxa * nV;
    nVb += dot(frb, n) * X * cxa;
    acc3(nb, frb * (X * cxa * nV));
    Yb += dot(frb, tang(n, dV)) * cya;
    tang_rev(n, dV, frb * (Y * cya), nb, dVb);
    Yb += dot(frb, cross(n, Wi)) * cybi + dot(frb, cross(n, Wj)) * cybj;
    cross_rev(n, Wi, frb * (Y * cybi), nb, Wib);
    cross_rev(n, Wj, frb * (Y * cybj), nb, Wjb);
    // nV = n . dV; dV = Vi - Vj
    acc3(nb, dV * nVb);
    acc3(dVb, n * nVb);
    acc3(Vib, dVb);
    acc3(Vjb, -dVb);
    // X = 1 / dd, Y = -log dd, dd = ds + eps, ds = 2 d / S unless clamped
    const double ddb = -Xb * X * X - Yb / dd;
    if (!clamped) db += ddb * 2.0 / S;
  }
  // electro-chemical central force m(d) n
  if (g.de > 0.0) {
    const double mb = dot(Fcb, n);
    acc3(nb, Fcb * m);
    db += mb * mp;
  }
  // contact
  if (contact) {
    V3d nxfb = cTi * ai + cTj * aj;
    double fnb = dot(Fcb, n);
    acc3(nb, Fcb * fn);
    V3d Ftb = Fcb;
    if (rolling) {
      // Tr = abar k_r (n x xr), added to T_i and taken from T_j
      const V3d Trb = cTi - cTj;
      V3d qb = zero;   // adjoint of q = abar k_r xr
      cross_rev(n, xr * (abar * g.k_r), Trb, nb, qb);
      const V3d xrb = mk3<double>(c.xr[0], c.xr[1], c.xr[2]) + qb * (abar * g.k_r);
      V3d xr0b = zero;
      double caprb = 0.0;
      cap_rev(xr0, capr, rslip, xrb, xr0b, caprb);
      mub += caprb * fabs(fn) / g.k_r;
      fnb += caprb * mu * (fn >= 0.0 ? 1.0 : -1.0) / g.k_r;
      // xr0 = tang(n, ro) + (dt abar) n x wr
      tang_rev(n, ro, xr0b, nb, rob);
      V3d wrb = zero;
      cross_rev(n, wr, xr0b * (g.dt * abar), nb, wrb);
      acc3(wib, wrb);
      acc3(wjb, -wrb);
    }
    // nxf = n x Ft
    cross_rev(n, Ft, nxfb, nb, Ftb);
    // Ft = kt xs
    ktb += dot(Ftb, xs);
    const V3d xsb = Ftb * kt + mk3<double>(c.xi[0], c.xi[1], c.xi[2]);
    V3d xs0b = zero;
    double capb = 0.0;
    cap_rev(xs0, cap, slip, xsb, xs0b, capb);
    // cap = mu |fn| / kt
    mub += capb * fabs(fn) / kt;
    fnb += capb * mu * (fn >= 0.0 ? 1.0 : -1.0) / kt;
    ktb += -capb * mu * fabs(fn) / (kt * kt);
    // xs0 = tang(n, xo) + dt tang(n, rel)
    tang_rev(n, xo, xs0b, nb, xob);
    V3d relb = zero;
    tang_rev(n, rel, xs0b * g.dt, nb, relb);
    // rel = du - aw x n, aw = ai wi + aj wj
    acc3(dub, relb);
    V3d awb = zero;
    cross_rev(aw, n, -relb, awb, nb);
    acc3(wib, awb * ai);
    acc3(wjb, awb * aj);
    // fn = kn d + gn n.du
    knb += fnb * d;
    db += fnb * kn;
    gnb += fnb * dot(n, du);
    acc3(nb, du * (fnb * gn));
    acc3(dub, n * (fnb * gn));
  }
  // geometry: n = r / |r|, d = |r| - S
  acc3(rb, nb * ir - n * (dot(nb, n) * ir) + n * db);
  // inputs
  double yib = -gd * Vib.x, yjb = -gd * Vjb.x;
  if (g.wave) {
    yib += -U * kw * ci * Vib.x - 0.5 * U * kw * kw * si * (Wib.z + rateb);
    yjb += -U * kw * cj * Vjb.x - 0.5 * U * kw * kw * sj * (Wjb.z + rateb);
  }
  const V3d uib = Vib - dub, ujb = Vjb + dub;
  const V3d wiab = Wib + wib, wjab = Wjb + wjb;
  out[0] = rb.x; out[1] = rb.y; out[2] = rb.z;
  out[3] = yib; out[4] = yjb;
  out[5] = uib.x; out[6] = uib.y; out[7] = uib.z;
  out[8] = ujb.x; out[9] = ujb.y; out[10] = ujb.z;
  out[11] = wiab.x; out[12] = wiab.y; out[13] = wiab.z;
  out[14] = wjab.x; out[15] = wjab.y; out[16] = wjab.z;
  out[17] = xob.x; out[18] = xob.y; out[19] = xob.z;
  out[20] = knb; out[21] = ktb; out[22] = gnb; out[23] = mub; out[24] = deltab;
  out[25] = rob.x; out[26] = rob.y; out[27] = rob.z;
}

// ---------------------------------------------------------------- tape
// Per owner: the pair's owner / partner, and the stretch carried in from the
// history list (contact pairs whose key was in contact at the previous step).
__global__ void __launch_bounds__(kThreads)
k_adj_tape_pairs(Geo g, const InstGeo* __restrict__ ig, const StepGeo* __restrict__ sgk, StateBuf s,
                 ListBuf W, ListBuf H, int empty_history, AdjTape t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = g.n;
  if (i >= n) return;
  const InstGeo& I = ig[0];
  const double off = sgk[0].off;
  const int cnt = W.count[i];
  const int p0 = W.start[i];
  const double xi = s.x[i], yi = s.x[n + i], zi = s.x[2 * n + i], ai = s.a[i];
  const int idi = s.id[i];
  for (int k = 0; k < cnt; ++k) {
    const int p = p0 + k;
    const int j = W.list[(int64_t)i * g.Ms + k];
    t.op[p] = i;
    t.pj[p] = j;
    double dx, dy, dz;
    int sy;
    min_image(I, off, xi, yi, zi, s.x[j], s.x[n + j], s.x[2 * n + j], dx, dy, dz, sy);
    const double rr = exact_dist(dx, dy, dz);
    int pold = -1;
    double xo[3] = {0.0, 0.0, 0.0}, ro[3] = {0.0, 0.0, 0.0};
    if (!empty_history && __dsub_rn(rr, __dadd_rn(ai, s.a[j])) < 0.0) {
      const int idj = s.id[j];
      const int oi = H.slot_of_id[idi], oj = H.slot_of_id[idj];
      int q = -1;
      for (int m = 0; m < H.count[oi]; ++m)
        if (H.list[(int64_t)oi * g.Ms + m] == oj) { q = H.start[oi] + m; break; }
      if (q < 0)
        for (int m = 0; m < H.count[oj]; ++m)
          if (H.list[(int64_t)oj * g.Ms + m] == oi) { q = H.start[oj] + m; break; }
      const Xi4 hv = q >= 0 ? H.xi[q] : Xi4{0.0, 0.0, 0.0, 0.0};
      if (xi_flag(hv)) {
        const double sgn = idi < idj ? 1.0 : -1.0;
        double c[3];
        xi_components(hv, g.precision == DSS_MIXED, c);
        pold = q;
        xo[0] = sgn * c[0];
        xo[1] = sgn * c[1];
        xo[2] = sgn * c[2];
        if (t.xro) xi_components(H.xr[q], g.precision == DSS_MIXED, ro);   // orientation-free
      }
    }
    t.pold[p] = pold;
    t.xo[p] = xo[0];
    t.xo[g.pcap + p] = xo[1];
    t.xo[2 * g.pcap + p] = xo[2];
    if (t.xro) {
      t.xro[p] = ro[0];
      t.xro[g.pcap + p] = ro[1];
      t.xro[2 * g.pcap + p] = ro[2];
    }
  }
}

// ---------------------------------------------------------------- reverse
__global__ void __launch_bounds__(kThreads)
k_adj_pre(Geo g, const InstGeo* __restrict__ ig, AdjTape t, const double* __restrict__ a_by_id,
          double* __restrict__ xb, double* __restrict__ ub, double* __restrict__ wb,
          const double* __restrict__ ab, const double* __restrict__ bb, double* __restrict__ Fb,
          double* __restrict__ Tb, int* __restrict__ bw_n, int initial, const double* __restrict__ Wn,
          double inv_vol) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = g.n;
  if (s >= n) return;
  const int id = t.id[s];
  const double a = a_by_id[id];
  const double m = 4.0 / 3.0 * DSS_PI * g.rho * a * a * a;
  const double Iner = 0.4 * m * a * a;
  const double hdt = 0.5 * g.dt;
  const double gd = ig[0].gdot;
  double F[3], T[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double at = initial ? ab[c * n + id] : ab[c * n + id] + hdt * ub[c * n + id];
    const double bt = initial ? bb[c * n + id] : bb[c * n + id] + hdt * wb[c * n + id];
    F[c] = at / m;
    T[c] = bt / Iner;
    Fb[c * n + s] = F[c];
    Tb[c * n + s] = T[c];
  }
  // Stokes drag (Eq. A1): F = -6 pi eta0 a (u - gdot y e_x), T = -8 pi eta0 a^3 (w - Omega_inf)
  const double kd = g.k6 * a, kr = g.k8 * a * a * a;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    ub[c * n + id] -= kd * F[c];
    wb[c * n + id] -= kr * T[c];
  }
  if (g.wave) {
    // Eq. 17: dF_x/dy through the Faxen-corrected U_inf,x, dT_z/dy through
    // Omega_inf,z, and the local single-particle stresslets (xy, yx) of the
    // weighted stress
    const InstGeo& I = ig[0];
    const double k = I.wave_k, U = g.wave_amp, y = t.x[n + s];
    double sn, cs;
    sincos(k * y, &sn, &cs);
    double yb = kd * (gd + U * (1.0 - a * a * I.faxen_c) * k * cs) * F[0];
    yb += kr * 0.5 * U * k * k * sn * T[2];
    if (Wn) yb -= (Wn[1] + Wn[3]) * inv_vol * (10.0 / 3.0) * DSS_PI * g.eta0 * a * a * a * U * k * k * sn;
    xb[n + id] += yb;
  } else {
    xb[n + id] += kd * gd * F[0];
  }
  bw_n[s] = 0;
}

__global__ void __launch_bounds__(kAdjThreads)
k_adj_pairs(Geo g, const InstGeo* __restrict__ ig, AdjTape t, const double* __restrict__ a_by_id, int P,
            const double* __restrict__ Fb, const double* __restrict__ Tb,
            const double* __restrict__ xib_cur, double* __restrict__ xib_prev,
            const double* __restrict__ xrb_cur, double* __restrict__ xrb_prev,
            const double* __restrict__ Wn, double inv_vol, double* __restrict__ pout,
            int* __restrict__ bw_n, int* __restrict__ bw_p, double* __restrict__ thb_part,
            DevStatus* st) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = g.n;
  double th[5] = {0, 0, 0, 0, 0};
  if (p < P) {
    const InstGeo& I = ig[0];
    const int i = t.op[p], j = t.pj[p];
    PairIn in;
    int sy;
    min_image(I, t.sg->off, t.x[i], t.x[n + i], t.x[2 * n + i], t.x[j], t.x[n + j], t.x[2 * n + j],
              in.r[0], in.r[1], in.r[2], sy);
    in.sy = sy;
    in.yi = t.x[n + i];
    in.yj = t.x[n + j];
    const int idi = t.id[i], idj = t.id[j];
    in.ai = a_by_id[idi];
    in.aj = a_by_id[idj];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      in.ui[c] = t.u[c * n + i];
      in.uj[c] = t.u[c * n + j];
      in.wi[c] = t.w[c * n + i];
      in.wj[c] = t.w[c * n + j];
      in.xo[c] = t.xo[c * g.pcap + p];
      in.ro[c] = t.xro ? t.xro[c * g.pcap + p] : 0.0;
    }
    PairCot cot;
    const double sgn = idi < idj ? 1.0 : -1.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      cot.F[c] = Fb[c * n + i] - Fb[c * n + j];
      cot.Ti[c] = Tb[c * n + i];
      cot.Tj[c] = Tb[c * n + j];
      cot.xi[c] = sgn * xib_cur[c * g.pcap + p];   // stored lo -> hi, model i -> j
      cot.xr[c] = xrb_cur ? xrb_cur[c * g.pcap + p] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) cot.Ws[q] = Wn ? Wn[q] * inv_vol : 0.0;
    double out[kNin];
#pragma unroll
    for (int k = 0; k < kNin; ++k) out[k] = 0.0;
    pair_vjp(g, I, in, cot, out);
    double* po = pout + (int64_t)p * 18;
    // i side: x = -r_bar + y_i, u_i, w_i; j side: x = +r_bar + y_j, u_j, w_j
    po[0] = -out[0]; po[1] = -out[1] + out[3]; po[2] = -out[2];
    po[3] = out[5]; po[4] = out[6]; po[5] = out[7];
    po[6] = out[11]; po[7] = out[12]; po[8] = out[13];
    po[9] = out[0]; po[10] = out[1] + out[4]; po[11] = out[2];
    po[12] = out[8]; po[13] = out[9]; po[14] = out[10];
    po[15] = out[14]; po[16] = out[15]; po[17] = out[16];
    const int q = t.pold[p];
    if (q >= 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) xib_prev[c * g.pcap + q] = sgn * out[17 + c];
      if (xrb_prev)
#pragma unroll
        for (int c = 0; c < 3; ++c) xrb_prev[c * g.pcap + q] = out[25 + c];
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) th[c] = out[20 + c];
    const int slot = atomicAdd(&bw_n[j], 1);
    if (slot < g.M) bw_p[(int64_t)j * g.M + slot] = p;
    else set_err(st, DSS_ERR_CAPACITY);
  }
  // parameter adjoints: fixed-order block reduction
  __shared__ double red[kAdjThreads / 32][5];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    double v = th[c];
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    if (lane == 0) red[wid][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    double v = 0.0;
    for (int w = 0; w < kAdjThreads / 32; ++w) v += red[w][threadIdx.x];
    thb_part[blockIdx.x * 5 + threadIdx.x] = v;
  }
}

__global__ void __launch_bounds__(kThreads)
k_adj_gather(Geo g, AdjTape t, const double* __restrict__ pout, const int* __restrict__ bw_n,
             const int* __restrict__ bw_p, double* __restrict__ xb, double* __restrict__ ub,
             double* __restrict__ wb) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = g.n;
  if (s >= n) return;
  double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int p = t.start[s]; p < t.start[s + 1]; ++p) {
    const double* po = pout + (int64_t)p * 18;
#pragma unroll
    for (int c = 0; c < 9; ++c) v[c] += po[c];
  }
  int cnt = bw_n[s];
  cnt = cnt < g.M ? cnt : g.M;
  const int* row = bw_p + (int64_t)s * g.M;
  int prev = -1;
  for (int k = 0; k < cnt; ++k) {
    int best = INT_MAX;
    for (int q = 0; q < cnt; ++q) {
      const int pq = row[q];
      if (pq > prev && pq < best) best = pq;
    }
    const double* po = pout + (int64_t)best * 18 + 9;
#pragma unroll
    for (int c = 0; c < 9; ++c) v[c] += po[c];
    prev = best;
  }
  const int id = t.id[s];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    xb[c * n + id] += v[c];
    ub[c * n + id] += v[3 + c];
    wb[c * n + id] += v[6 + c];
  }
}

// Eq. 15a-b backwards: x^{n+1} = x^n + dt u^n + dt^2/2 alpha^n,
// u^{n+1/2} = u^n + dt/2 alpha^n, w^{n+1/2} = w^n + dt/2 beta^n.
__global__ void __launch_bounds__(kThreads)
k_adj_predict(int n3, double dt, const double* __restrict__ xb, double* __restrict__ ub,
              double* __restrict__ wb, double* __restrict__ ab, double* __restrict__ bb) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n3) return;
  const double hdt = 0.5 * dt, hdt2 = 0.5 * dt * dt;
  const double x = xb[k], u = ub[k];
  ab[k] = hdt * u + hdt2 * x;
  ub[k] = u + dt * x;
  bb[k] = hdt * wb[k];
}

// The five parameter adjoints of one step from the pair blocks' partials:
// warp c sums parameter c, its lanes striding over the blocks, then a fixed
// butterfly (the order depends on the block count alone).
__global__ void k_adj_theta(const double* __restrict__ part, int nblocks, double* __restrict__ thb) {
  const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (c >= 5) return;
  double v = 0.0;
  for (int b = lane; b < nblocks; b += 32) v += part[b * 5 + c];
  for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
  if (lane == 0) thb[c] += v;
}

__global__ void k_adj_accum_J(const double* __restrict__ sigma, const double* __restrict__ W,
                              double* __restrict__ J) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double v = 0.0;
  for (int q = 0; q < 9; ++q) v += W[q] * sigma[q];
  *J += v;
}

template <typename T>
int adj_dalloc(dss_handle* h, T** p, size_t count) {
  size_t b = sizeof(T) * (count > 0 ? count : 1);
  if (cudaMalloc((void**)p, b) != cudaSuccess) return DSS_ERR_CUDA;
  h->bytes += (int64_t)b;
  return DSS_OK;
}
}  // namespace

void adj_free(dss_handle* h) {
  AdjBuf* A = h->adj;
  if (!A) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (int k = 0; k < A->slots; ++k) {
    AdjTape& t = A->tape[k];
    cudaFree(t.x); cudaFree(t.u); cudaFree(t.w); cudaFree(t.id); cudaFree(t.start);
    cudaFree(t.op); cudaFree(t.pj); cudaFree(t.pold); cudaFree(t.xo); cudaFree(t.xro); cudaFree(t.sg);
  }
  delete[] A->tape;
  if (A->P_host) cudaFreeHost(A->P_host);
  cudaFree(A->xb); cudaFree(A->ub); cudaFree(A->wb); cudaFree(A->ab); cudaFree(A->bb);
  cudaFree(A->Fb); cudaFree(A->Tb); cudaFree(A->pout); cudaFree(A->bw_n); cudaFree(A->bw_p);
  cudaFree(A->xib[0]); cudaFree(A->xib[1]); cudaFree(A->xrb[0]); cudaFree(A->xrb[1]);
  cudaFree(A->thb_part); cudaFree(A->thb); cudaFree(A->J);
  cudaFree(A->W);
  delete A;
  h->adj = nullptr;
}

// Tapes for `slots` steps and the adjoint state, sized for the handle's
// current pair capacity.
int adj_alloc(dss_handle* h, int slots, int64_t nsteps) {
  if (h->adj && (h->adj->slots < slots || h->adj->pcap != h->pcap || h->adj->W_steps < nsteps))
    adj_free(h);
  if (h->adj) return DSS_OK;
  AdjBuf* A = new AdjBuf();
  memset((void*)A, 0, sizeof(AdjBuf));
  h->adj = A;
  A->slots = slots;
  A->pcap = h->pcap;
  A->W_steps = nsteps;
  A->tape = new AdjTape[slots];
  memset((void*)A->tape, 0, sizeof(AdjTape) * slots);
  const size_t n = (size_t)h->n, pc = (size_t)h->pcap;
  int r;
  for (int k = 0; k < slots; ++k) {
    AdjTape& t = A->tape[k];
    if ((r = adj_dalloc(h, &t.x, 3 * n)) || (r = adj_dalloc(h, &t.u, 3 * n)) ||
        (r = adj_dalloc(h, &t.w, 3 * n)) || (r = adj_dalloc(h, &t.id, n)) ||
        (r = adj_dalloc(h, &t.start, n + 1)) || (r = adj_dalloc(h, &t.op, pc)) ||
        (r = adj_dalloc(h, &t.pj, pc)) || (r = adj_dalloc(h, &t.pold, pc)) ||
        (r = adj_dalloc(h, &t.xo, 3 * pc)) || (r = adj_dalloc(h, &t.sg, 1)))
      return r;
    if (h->g.k_r > 0.0 && (r = adj_dalloc(h, &t.xro, 3 * pc))) return r;
  }
  if (cudaMallocHost((void**)&A->P_host, sizeof(int) * slots) != cudaSuccess) return DSS_ERR_CUDA;
  const int pb = (int)((pc + kAdjThreads - 1) / kAdjThreads);
  if ((r = adj_dalloc(h, &A->xb, 3 * n)) || (r = adj_dalloc(h, &A->ub, 3 * n)) ||
      (r = adj_dalloc(h, &A->wb, 3 * n)) || (r = adj_dalloc(h, &A->ab, 3 * n)) ||
      (r = adj_dalloc(h, &A->bb, 3 * n)) || (r = adj_dalloc(h, &A->Fb, 3 * n)) ||
      (r = adj_dalloc(h, &A->Tb, 3 * n)) || (r = adj_dalloc(h, &A->pout, 18 * pc)) ||
      (r = adj_dalloc(h, &A->bw_n, n)) || (r = adj_dalloc(h, &A->bw_p, n * (size_t)h->g.M)) ||
      (r = adj_dalloc(h, &A->xib[0], 3 * pc)) || (r = adj_dalloc(h, &A->xib[1], 3 * pc)) ||
      (r = adj_dalloc(h, &A->thb_part, 5 * (size_t)std::max(pb, 1))) || (r = adj_dalloc(h, &A->thb, 5)) ||
      (r = adj_dalloc(h, &A->J, 1)) || (r = adj_dalloc(h, &A->W, 9 * (size_t)std::max<int64_t>(nsteps, 1))))
    return r;
  if (h->g.k_r > 0.0 &&
      ((r = adj_dalloc(h, &A->xrb[0], 3 * pc)) || (r = adj_dalloc(h, &A->xrb[1], 3 * pc))))
    return r;
  return DSS_OK;
}

int adj_upload_weights(dss_handle* h, const double* W, int64_t nsteps) {
  if (cudaMemcpyAsync(h->adj->W, W, sizeof(double) * 9 * nsteps, cudaMemcpyDefault, h->stream) !=
      cudaSuccess)
    return DSS_ERR_CUDA;
  return DSS_OK;
}

void adj_zero(dss_handle* h) {
  AdjBuf* A = h->adj;
  const size_t b3 = sizeof(double) * 3 * (size_t)h->n;
  cudaMemsetAsync(A->xb, 0, b3, h->stream);
  cudaMemsetAsync(A->ub, 0, b3, h->stream);
  cudaMemsetAsync(A->wb, 0, b3, h->stream);
  cudaMemsetAsync(A->ab, 0, b3, h->stream);
  cudaMemsetAsync(A->bb, 0, b3, h->stream);
  cudaMemsetAsync(A->xib[0], 0, sizeof(double) * 3 * A->pcap, h->stream);
  cudaMemsetAsync(A->xib[1], 0, sizeof(double) * 3 * A->pcap, h->stream);
  for (int k = 0; k < 2; ++k)
    if (A->xrb[k]) cudaMemsetAsync(A->xrb[k], 0, sizeof(double) * 3 * A->pcap, h->stream);
  cudaMemsetAsync(A->thb, 0, sizeof(double) * 5, h->stream);
  cudaMemsetAsync(A->J, 0, sizeof(double), h->stream);
  A->cur = 0;
}

void adj_accum_J(dss_handle* h, int64_t step) {
  k_adj_accum_J<<<1, 32, 0, h->stream>>>(h->sigma, h->adj->W + 9 * step, h->adj->J);
}

// Records the tape of the force evaluation about to run on state buffer
// stbuf with pair list `list` (history from hist_list unless empty).
void adj_tape(dss_handle* h, int slot, int stbuf, int list, int hist_list, bool empty_history) {
  AdjBuf* A = h->adj;
  AdjTape& t = A->tape[slot];
  const StateBuf& s = h->st[stbuf];
  const size_t n = (size_t)h->n;
  cudaMemcpyAsync(t.x, s.x, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, h->stream);
  cudaMemcpyAsync(t.u, s.u, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, h->stream);
  cudaMemcpyAsync(t.w, s.w, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, h->stream);
  cudaMemcpyAsync(t.id, s.id, sizeof(int) * n, cudaMemcpyDeviceToDevice, h->stream);
  cudaMemcpyAsync(t.start, h->lb[list].start, sizeof(int) * (n + 1), cudaMemcpyDeviceToDevice, h->stream);
  cudaMemcpyAsync(t.sg, h->sg, sizeof(StepGeo), cudaMemcpyDeviceToDevice, h->stream);
  cudaMemcpyAsync(&A->P_host[slot], h->lb[list].start + n, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  k_adj_tape_pairs<<<(int)((n + kThreads - 1) / kThreads), kThreads, 0, h->stream>>>(
      h->g, h->ig, h->sg, s, h->lb[list], h->lb[hist_list], empty_history ? 1 : 0, t);
}

// Reverse of one step (initial: the force evaluation that set the initial
// accelerations) from its tape.  `step` indexes the stress weights (the
// step's stress sigma^{step+1}); ignored for the initial evaluation.  The
// stream must have been synchronised since the tape was recorded (its pair
// count is read on the host).
void adj_reverse(dss_handle* h, int slot, int64_t step, bool initial) {
  AdjBuf* A = h->adj;
  AdjTape& t = A->tape[slot];
  const int n = (int)h->n;
  const int P = A->P_host[slot];
  const int nb = (n + kThreads - 1) / kThreads;
  const InstGeo& I = h->ig_host[0];
  const double vol = I.L[0] * I.L[1] * I.L[2];
  double* xib_cur = A->xib[A->cur];
  double* xib_prev = A->xib[1 - A->cur];
  double* xrb_cur = A->xrb[A->cur];
  double* xrb_prev = A->xrb[1 - A->cur];
  cudaMemsetAsync(xib_prev, 0, sizeof(double) * 3 * A->pcap, h->stream);
  if (xrb_prev) cudaMemsetAsync(xrb_prev, 0, sizeof(double) * 3 * A->pcap, h->stream);
  const double* Wn = initial ? nullptr : A->W + 9 * step;
  k_adj_pre<<<nb, kThreads, 0, h->stream>>>(h->g, h->ig, t, h->a_by_id, A->xb, A->ub, A->wb, A->ab, A->bb,
                                            A->Fb, A->Tb, A->bw_n, initial ? 1 : 0, Wn, 1.0 / vol);
  const int pb = std::max((P + kAdjThreads - 1) / kAdjThreads, 1);
  k_adj_pairs<<<pb, kAdjThreads, 0, h->stream>>>(
      h->g, h->ig, t, h->a_by_id, P, A->Fb, A->Tb, xib_cur, xib_prev, xrb_cur, xrb_prev, Wn,
      1.0 / vol, A->pout, A->bw_n, A->bw_p, A->thb_part, h->status);
  k_adj_theta<<<1, 160, 0, h->stream>>>(A->thb_part, pb, A->thb);
  k_adj_gather<<<nb, kThreads, 0, h->stream>>>(h->g, t, A->pout, A->bw_n, A->bw_p, A->xb, A->ub, A->wb);
  if (initial) {
    // alpha^0, beta^0 are consumed by the initial evaluation
    cudaMemsetAsync(A->ab, 0, sizeof(double) * 3 * n, h->stream);
    cudaMemsetAsync(A->bb, 0, sizeof(double) * 3 * n, h->stream);
  } else {
    k_adj_predict<<<(3 * n + kThreads - 1) / kThreads, kThreads, 0, h->stream>>>(3 * n, h->g.dt, A->xb, A->ub,
                                                                                 A->wb, A->ab, A->bb);
  }
  A->cur = 1 - A->cur;
}
