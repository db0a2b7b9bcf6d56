// Pair forces and their deterministic symmetric accumulation.
//
// k_pairs<MIXED, MINB, EXT>: a warp takes 32 consecutive owners and deals out their
//   listed pairs (owner-sorted) 32 at a time.  Per pair: lubrication of
//   App. A (Eq. A2, A3 with the coefficients of Eq. A6, A7 and the
//   6 pi eta0 prefactor), stick-and-slide contact of Eq. 4-5 with the
//   tangential stretch carried from the previous step's rows, and the pair
//   stresslet of Eq. 9.  The owner's share is summed by a warp-segmented
//   reduction (lanes holding the same owner are contiguous) into a per-warp
//   shared-memory accumulator and written once per owner; the partner's share
//   (-F and its torque) is appended to the partner's fixed-capacity row
//   together with the owner's index.  No float is ever accumulated with an
//   atomic.
// k_pairs_pb<MIXED, MINB, EXT> (one instance): the same per pair, with the
//   pairs in owner order dealt out 32 to a warp over the resident blocks
//   (every lane busy whatever the row lengths); owners whose pairs cross a
//   warp boundary leave head / tail partial sums the gather adds in order.
// k_gather<MIXED, EXT>: one thread per particle: its own sum plus the partner
//   records of its row taken in increasing owner index (a fixed order, so the
//   result is bitwise reproducible; rows of 9 to 24 FP32 records and longer
//   FP64 rows are summed by the whole warp, ranks counted and placed, then a
//   fixed reduction; longer FP32 rows by their own thread in 64-bit fixed
//   point, whose sum does not depend on the order), Stokes drag (Eq. A1) and
//   the corrector
//   of Eq. 15d.  K leading blocks reduce each instance's bulk stress of
//   Eq. 8 from the pair blocks' partials; the last block of the gather to
//   finish adds them to the running sums and commits the step.
#include <climits>

#include "dss_internal.cuh"
#include "dss_pair_model.cuh"

namespace {
constexpr int kPairThreads = 256;
constexpr int kWarps = kPairThreads / 32;
constexpr int kThreads = 128;
constexpr int kSlot = 8;   // partner-row slot: F (3), T (3), owner index, pad

// Position of `target` in a row (rows are in stencil visiting order and
// start on 16-byte boundaries, so four entries come per load); -1 if absent.
__device__ __forceinline__ int row_find(const int* row, int cnt, int target) {
  const int4* r4 = reinterpret_cast<const int4*>(row);
  for (int k = 0; k < cnt; k += 4) {
    const int4 v = r4[k >> 2];
    if (v.x == target) return k;
    if (k + 1 < cnt && v.y == target) return k + 1;
    if (k + 2 < cnt && v.z == target) return k + 2;
    if (k + 3 < cnt && v.w == target) return k + 3;
  }
  return -1;
}

// Where the particles of the current sorted order sit in the rows of the
// committed history: perm (the sort's new -> previous index) when the sort's
// source was in the history's row order, else the history's id -> row map.
struct HistRef {
  const int* perm;
  int idorder;
};

// Where pair (i, j) sat in the committed history: the rows of the previous
// step's list are searched for it (the owner's row first: ownership in the
// half stencil rarely changes between steps).  The probe takes one round of
// loads after the sorted-order map: the owner row's length, offset and first
// four entries (rows hold at least four entries and start on 16-byte
// boundaries, so the first int4 is always in bounds).
struct HistProbe {
  int oi, oj, cnt, st;
  int4 r;
};

__device__ __forceinline__ HistProbe hist_probe(const Geo& g, const ListBuf& H, const HistRef& hr, int i, int j,
                                                int idi, int idj) {
  HistProbe p;
  p.oi = hr.idorder ? H.slot_of_id[idi] : hr.perm[i];
  p.oj = hr.idorder ? H.slot_of_id[idj] : hr.perm[j];
  p.cnt = H.count[p.oi];
  p.st = H.start[p.oi];
  p.r = *reinterpret_cast<const int4*>(H.list + (int64_t)p.oi * g.Ms);
  return p;
}

// Slot of the pair in the committed list's pair arrays, -1 if it was not
// listed.
__device__ __forceinline__ int64_t hist_slot(const Geo& g, const ListBuf& H, const HistProbe& p) {
  int k = -1;
  if (p.cnt > 0 && p.r.x == p.oj) k = 0;
  else if (p.cnt > 1 && p.r.y == p.oj) k = 1;
  else if (p.cnt > 2 && p.r.z == p.oj) k = 2;
  else if (p.cnt > 3 && p.r.w == p.oj) k = 3;
  else if (p.cnt > 4) {
    k = row_find(H.list + (int64_t)p.oi * g.Ms + 4, p.cnt - 4, p.oj);
    if (k >= 0) k += 4;
  }
  if (k >= 0) return (int64_t)p.st + k;
  k = row_find(H.list + (int64_t)p.oj * g.Ms, H.count[p.oj], p.oi);
  return k >= 0 ? (int64_t)H.start[p.oj] + k : -1;
}

// Tangential stretch of pair (i, j) (ids idi, idj) at the last committed
// step, in the lo -> hi orientation, and (when k_r > 0) its rolling stretch;
// zero when the pair was not in contact.
template <bool EXT>
__device__ __forceinline__ void history_lookup(const Geo& g, const ListBuf& H, const HistRef& hr, int i,
                                               int j, int idi, int idj, double xo[3], double ro[3]) {
  xo[0] = xo[1] = xo[2] = 0.0;
  ro[0] = ro[1] = ro[2] = 0.0;
  const int64_t pold = hist_slot(g, H, hist_probe(g, H, hr, i, j, idi, idj));
  if (pold >= 0) {
    const Xi4 v = H.xi[pold];
    if (xi_flag(v)) {
      xo[0] = v.x;
      xo[1] = v.y;
      xo[2] = v.z;
      if (EXT && g.k_r > 0.0) {
        const Xi4 vr = H.xr[pold];
        ro[0] = vr.x;
        ro[1] = vr.y;
        ro[2] = vr.z;
      }
    }
  }
}

using V3 = Vec3<double>;
__device__ __forceinline__ V3 v3(double a, double b, double c) { return V3{a, b, c}; }

struct F3 {
  float x, y, z;
};
__device__ __forceinline__ F3 f3(float a, float b, float c) { return F3{a, b, c}; }
__device__ __forceinline__ F3 operator+(F3 a, F3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ F3 operator-(F3 a, F3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ F3 operator*(float s, F3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dotf(F3 a, F3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ F3 crossf(F3 a, F3 b) {
  return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ F3 tangf(F3 n, F3 v) { return v - dotf(n, v) * n; }


// Result of one pair in the arithmetic precision R, with its stretch
// records as they are stored.
template <typename R>
struct PairRes {
  R F[3], Ti[3], Tj[3], Fc[3], Fl[3], r[3];
  Xi4 xrec, rrec;
  int contact;
};

// FP64 pair from the state (exact FP64 throughout).  EXT: the wave of
// Eq. 17 or rolling resistance may be on (compiled out otherwise).
template <bool EXT>
__device__ __forceinline__ PairRes<double> pair_eval_fp64(const Geo& g, const InstGeo& I, const StateBuf& s,
                                                         const ListBuf& H, const HistRef& hr, double off,
                                                         int i, int j) {
  const int n = g.n;
  const double xi = s.x[i], yi = s.x[n + i], zi = s.x[2 * n + i];
  const double xj = s.x[j], yj = s.x[n + j], zj = s.x[2 * n + j];
  double dx, dy, dz;
  int sy;
  min_image(I, off, xi, yi, zi, xj, yj, zj, dx, dy, dz, sy);
  const V3 r = v3(dx, dy, dz);
  const double ai = s.a[i], aj = s.a[j];
  const V3 ui = v3(s.u[i], s.u[n + i], s.u[2 * n + i]);
  const V3 uj = v3(s.u[j], s.u[n + j], s.u[2 * n + j]);
  const V3 wi = v3(s.w[i], s.w[n + i], s.w[2 * n + i]);
  const V3 wj = v3(s.w[j], s.w[n + j], s.w[2 * n + j]);
  const int idi = s.id[i], idj = s.id[j];
  const double sgn = idi < idj ? 1.0 : -1.0;
  double xo[3] = {0.0, 0.0, 0.0}, ro[3] = {0.0, 0.0, 0.0};
  const double rr = exact_dist(dx, dy, dz);
  if (__dsub_rn(rr, __dadd_rn(ai, aj)) < 0.0) {
    history_lookup<EXT>(g, H, hr, i, j, idi, idj, xo, ro);
    xo[0] *= sgn; xo[1] *= sgn; xo[2] *= sgn;
  }
  const double Om = -0.5 * I.gdot;
  V3 Vi = v3(ui.x - I.gdot * yi, ui.y, ui.z);
  V3 Vj = v3(uj.x - I.gdot * yj, uj.y, uj.z);
  V3 Wi = v3(wi.x, wi.y, wi.z - Om);
  V3 Wj = v3(wj.x, wj.y, wj.z - Om);
  double rate = I.gdot;
  if (EXT && g.wave) {
    // the wave of Eq. 17 at each centre: V and W relative to the local flow,
    // the pair's strain from the mean of the two local rates
    const double2 qi = s.wv[i], qj = s.wv[j];
    Vi.x -= qi.x;
    Vj.x -= qj.x;
    Wi.z += 0.5 * qi.y;
    Wj.z += 0.5 * qj.y;
    rate = I.gdot + 0.5 * (qi.y + qj.y);
  }
  const V3 du = v3(uj.x + sy * I.gdot * I.L[1] - ui.x, uj.y - ui.y, uj.z - ui.z);
  const PairParams<double> pp{g.kn, g.kt, I.gn, g.mu, g.delta};
  const PairModelOut<double> o = pair_model<double, EXT>(g, I, pp, r, rr, ai, aj, Vi, Vj, Wi, Wj, du, wi, wj,
                                                    v3(xo[0], xo[1], xo[2]), v3(ro[0], ro[1], ro[2]), rate);
  PairRes<double> q;
  q.F[0] = o.F.x; q.F[1] = o.F.y; q.F[2] = o.F.z;
  q.Ti[0] = o.Ti.x; q.Ti[1] = o.Ti.y; q.Ti[2] = o.Ti.z;
  q.Tj[0] = o.Tj.x; q.Tj[1] = o.Tj.y; q.Tj[2] = o.Tj.z;
  q.Fc[0] = o.Fc.x; q.Fc[1] = o.Fc.y; q.Fc[2] = o.Fc.z;
  q.Fl[0] = o.Fl.x; q.Fl[1] = o.Fl.y; q.Fl[2] = o.Fl.z;
  q.r[0] = dx; q.r[1] = dy; q.r[2] = dz;
  q.xrec = Xi4{sgn * o.xi.x, sgn * o.xi.y, sgn * o.xi.z, o.contact ? 1.0 : 0.0};
  q.rrec = Xi4{o.xr.x, o.xr.y, o.xr.z, 0.0};
  q.contact = o.contact;
  return q;
}

// Mixed precision.  The separation and the gap numerator r^2 - S^2 are taken
// in FP64 from the FP64 positions (the lubrication coefficients diverge as
// 1/(d* + eps), so the gap needs far more than FP32's 7 digits); the gap is
// then d = (r^2 - S^2)/(r + S) with the division in FP32.  The tangential
// stretch is carried and updated as a double-float (~48 bits); the rest of
// the pair arithmetic is FP32, on velocities taken relative to the ambient
// flow.
template <bool EXT>
__device__ __forceinline__ PairRes<float> pair_eval_mixed(const Geo& g, const InstGeo& I, const StateBuf& s,
                                                         const ListBuf& H, const HistRef& hr,
                                                         const StepGeo& sg,
                                                         const float4* __restrict__ posf, int i, int j) {
  const float gd = I.gdot_f;
  const float k6 = g.f.k6;
  // double-float separation from cell-local hi/lo words and the cell offset
  // (listed pairs are at most `reach` cells apart along y and z; a pair whose
  // rows differ by more crosses y = L_y, its image shifted by +-off along x)
  const float4 pi = posf[i], pj = posf[j], li = s.posl[i], lj = s.posl[j];
  const int ci = s.cellc[i], cj = s.cellc[j];
  // the ids and the probe of the committed rows go out with the state loads
  // (their latency hides behind the geometry; the probe is used by contacts)
  const int idi = s.id[i], idj = s.id[j];
  const HistProbe pr = hist_probe(g, H, hr, i, j, idi, idj);
  const int nx = I.nc[0], ny = I.nc[1], nz = I.nc[2];
  const int R = g.reach;
  int wy = ((cj >> 10) & 1023) - ((ci >> 10) & 1023);
  const int le = wy < -R ? 1 : (wy > R ? -1 : 0);
  wy += le * ny;
  int wx = (cj & 1023) - (ci & 1023) + le * sg.fsh;
  wx %= nx;
  if (wx < 0) wx += nx;
  // the image row spans x offsets -R-1..R (above) or -R..R+1 (below)
  if (le == -1 ? 2 * wx > nx : 2 * wx >= nx) wx -= nx;
  int wz = (cj >> 20) - (ci >> 20);
  if (wz > R) wz -= nz; else if (wz < -R) wz += nz;
  FF cx = cell_shift(wx, I.csf[0], I.cs_lo[0]);
  if (le == 1) cx = ff_add(cx, FF{sg.offr_hi, sg.offr_lo});
  else if (le == -1) cx = ff_add(cx, FF{-sg.offr_hi, -sg.offr_lo});
  const FF dxf = ff_add(two_sum(pj.x, -pi.x), ff_add(cx, FF{lj.x - li.x, 0.f}));
  const FF dyf = ff_add(two_sum(pj.y, -pi.y),
                        ff_add(cell_shift(wy, I.csf[1], I.cs_lo[1]), FF{lj.y - li.y, 0.f}));
  const FF dzf = ff_add(two_sum(pj.z, -pi.z),
                        ff_add(cell_shift(wz, I.csf[2], I.cs_lo[2]), FF{lj.z - li.z, 0.f}));
  const FF Sff = ff_add(FF{pi.w, li.w}, FF{pj.w, lj.w});
  const FF r2ff = ff_add(ff_add(ff_sqr(dxf), ff_sqr(dyf)), ff_sqr(dzf));
  const FF numff = ff_add(r2ff, ff_neg(ff_sqr(Sff)));          // r^2 - S^2, ~44 bits
  const float num = numff.hi + numff.lo;
  const float r2 = r2ff.hi + r2ff.lo;
  const float ir = rsqrtf(r2);
  const float rr = r2 * ir;
  const float S = Sff.hi + Sff.lo;
  const float d = __fdividef(num, rr + S);
  const F3 r = f3(dxf.hi + dxf.lo, dyf.hi + dyf.lo, dzf.hi + dzf.lo);
  const F3 nn = ir * r;
  const float4 vi4 = s.vf[i], vj4 = s.vf[j], wi4 = s.wf[i], wj4 = s.wf[j];
  const F3 Vi = f3(vi4.x, vi4.y, vi4.z), Vj = f3(vj4.x, vj4.y, vj4.z);
  const F3 Wi = f3(wi4.x, wi4.y, wi4.z), Wj = f3(wj4.x, wj4.y, wj4.z);
  const float Ai = pi.w + li.w, Bj = pj.w + lj.w;
  PairRes<float> q;
  // ---- contact, Eq. 4-5: the flag here, the forces after the lubrication
  F3 Fc = f3(0, 0, 0), nxf = f3(0, 0, 0), Tr = f3(0, 0, 0);
  q.xrec = Xi4{0.0, 0.0, 0.0, 0.0};
  q.rrec = Xi4{0.0, 0.0, 0.0, 0.0};
  // The contact flag is a decision, taken as in FP64: the double-float gap
  // numerator (~44 bits) decides it unless it lies within 1e-9 S^2 of zero
  // (spheres touching to the last bits, which relaxed packings produce);
  // there the FP64 state decides with the operations of the plain FP64
  // evaluation.
  if (fabsf(num) > 1e-9f * S * S) {
    q.contact = num < 0.0f;
  } else {
    const int n = g.n;
    double ex, ey, ez;
    int sy;
    min_image(I, sg.off, s.x[i], s.x[n + i], s.x[2 * n + i], s.x[j], s.x[n + j], s.x[2 * n + j], ex, ey, ez, sy);
    q.contact = __dsub_rn(exact_dist(ex, ey, ez), __dadd_rn(s.a[i], s.a[j])) < 0.0;
  }
  Xi4 xrec{0.0, 0.0, 0.0, 0.0}, rrec{0.0, 0.0, 0.0, 0.0};
  if (q.contact) {
    const int64_t pold = hist_slot(g, H, pr);
    if (pold >= 0) {
      xrec = H.xi[pold];
      if (EXT && g.k_r > 0.0) rrec = H.xr[pold];
    }
  }
  // ---- contact forces and the stretch update (the stretch carried as a
  // double-float)
  if (q.contact) {
    const float sg = idi < idj ? 1.0f : -1.0f;   // stored (lo -> hi) vs i -> j orientation
    if (!xi_flag(xrec)) xrec = rrec = Xi4{0.0, 0.0, 0.0, 0.0};
    const FF xo[3] = {word_ff(xrec.x), word_ff(xrec.y), word_ff(xrec.z)};
    // u_j(image) - u_i = (V_j - V_i) + gdot dy x (+ the wave's U_inf,x
    // difference); absolute w = W + Omega_inf (local with the wave)
    F3 du = (Vj - Vi) + f3(gd * r.y, 0.f, 0.f);
    F3 wi = f3(Wi.x, Wi.y, Wi.z - 0.5f * gd), wj = f3(Wj.x, Wj.y, Wj.z - 0.5f * gd);
    if (EXT && g.wave) {
      du.x += wj4.w - wi4.w;
      wi.z -= 0.5f * vi4.w;
      wj.z -= 0.5f * vj4.w;
    }
    const float fn = g.f.kn * d + I.gn_f * dotf(nn, du);
    const F3 ut = tangf(nn, du - crossf(Ai * wi + Bj * wj, nn));
    // stretch (stored orientation) as a double-float: xi + delta, with the
    // small change delta = -n (n.xi) + s u_t dt (projection onto the new
    // tangent plane and the increment) formed in FP32 from the high words
    const F3 xf = f3(xo[0].hi, xo[1].hi, xo[2].hi);
    const float pn = dotf(nn, xf);
    const float sdt = sg * g.f.dt;
    const F3 dxs = f3(sdt * ut.x - pn * nn.x, sdt * ut.y - pn * nn.y, sdt * ut.z - pn * nn.z);
    FF xs0 = ff_add_f(xo[0], dxs.x), xs1 = ff_add_f(xo[1], dxs.y), xs2 = ff_add_f(xo[2], dxs.z);
    // the FP32 copy for the force (within an ulp of the double-float's value)
    F3 xsf = xf + dxs;
    const float cap = g.f.mu_kt * fabsf(fn);
    const float xm2 = dotf(xsf, xsf);
    if (xm2 > cap * cap) {
      const float fs = cap * rsqrtf(xm2);
      xs0 = ff_mul_f(xs0, fs);
      xs1 = ff_mul_f(xs1, fs);
      xs2 = ff_mul_f(xs2, fs);
      xsf = fs * xsf;
    }
    const F3 Ft = (sg * g.f.kt) * xsf;
    Fc = fn * nn + Ft;
    nxf = crossf(nn, Ft);
    q.xrec = Xi4{ff_word(xs0), ff_word(xs1), ff_word(xs2), ff_word(FF{1.0f, 0.0f})};
    if (EXT && g.k_r > 0.0) {
      // rolling resistance, App. B: the rolling stretch (orientation-free)
      // carried as a double-float with its FP32 increment, like the sliding
      // one
      const FF ro[3] = {word_ff(rrec.x), word_ff(rrec.y), word_ff(rrec.z)};
      const float abar = 2.0f * Ai * Bj / (Ai + Bj);
      const F3 rf = f3(ro[0].hi, ro[1].hi, ro[2].hi);
      const float rn = dotf(nn, rf);
      const F3 ur = (abar * g.f.dt) * crossf(nn, wi - wj);
      const F3 dr = f3(ur.x - rn * nn.x, ur.y - rn * nn.y, ur.z - rn * nn.z);
      FF r0 = ff_add_f(ro[0], dr.x), r1 = ff_add_f(ro[1], dr.y), r2 = ff_add_f(ro[2], dr.z);
      F3 xrf = rf + dr;
      const float capr = g.f.mu_kr * fabsf(fn);
      const float xrm2 = dotf(xrf, xrf);
      if (xrm2 > capr * capr) {
        const float fs = capr * rsqrtf(xrm2);
        r0 = ff_mul_f(r0, fs);
        r1 = ff_mul_f(r1, fs);
        r2 = ff_mul_f(r2, fs);
        xrf = fs * xrf;
      }
      Tr = abar * crossf(nn, g.f.k_r * xrf);
      q.rrec = Xi4{ff_word(r0), ff_word(r1), ff_word(r2), 0.0};
    }
  }
  // ---- electro-chemical forces, Eq. 6-7 (FP32; central, stresslet r (x) F).
  // The range decisions (lubrication cutoff, 20 lambda_D, 4 a0) are taken on
  // the FP32 gap unless it lies within 1e-5 of a threshold; there the FP64
  // state decides, in the operations of the neighbour test.
  bool lub_on = true;
  float m = 0.0f;
  if (g.de > 0.0) {
    const float dl = g.mode == 1 ? g.f.delta_a0 : g.f.delta * 0.5f * S;
    const float tol = 1e-5f * (S + dl);
    const bool rep = g.f.f_er > 0.0f, att = g.f.hamaker12 > 0.0f;
    bool in_r = d < g.f.range_r, in_a = d < g.f.range_a;
    lub_on = d < dl;
    if (fabsf(d - dl) < tol || (rep && fabsf(d - g.f.range_r) < tol) || (att && fabsf(d - g.f.range_a) < tol)) {
      const int n = g.n;
      double ex, ey, ez;
      int sy;
      min_image(I, sg.off, s.x[i], s.x[n + i], s.x[2 * n + i], s.x[j], s.x[n + j], s.x[2 * n + j], ex, ey, ez, sy);
      const double ai = s.a[i], aj = s.a[j];
      const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
      const double sl = __dadd_rn(__dadd_rn(ai, aj), lub_delta(g, ai, aj));
      lub_on = r2 < __dmul_rn(sl, sl);
      const double d64 = sqrt(r2) - (ai + aj);
      in_r = d64 < 20.0 * g.lambda_d;
      in_a = d64 < 4.0 * g.a0;
    }
    const float abar = 2.0f * Ai * Bj / (Ai + Bj);
    if (rep && in_r) m -= g.f.f_er * abar * (d >= 0.0f ? __expf(-d * g.f.inv_lambda) : 1.0f);
    if (att && in_a) {
      const float eps = g.f.vdw_eps * abar, dp = fmaxf(d, 0.0f);
      m += __fdividef(g.f.hamaker12 * abar, fmaf(dp, dp, eps * eps));
    }
  }
  // ---- lubrication, App. A (FP32), for the pairs within its range (every
  // listed pair unless electro-chemical forces widen the list; a warp whose
  // pairs are all beyond it skips the block)
  F3 Fl = f3(0.0f, 0.0f, 0.0f), Tli = Fl, Tlj = Fl;
  if (lub_on) {
    const float iS = __fdividef(1.0f, S), iS2 = iS * iS, iS3 = iS2 * iS;
    float ds = 2.0f * d * iS;
    ds = ds > 0.0f ? ds : 0.0f;
    const float dd = ds + g.f.eps;
    const float X = __fdividef(1.0f, dd);
    const float Y = -__logf(dd);
    const float A = Ai, B = Bj, AB = A * B;
    const float xa = X * 2.0f * AB * AB * iS3;
    const float ya = Y * (4.0f / 15.0f) * AB * (2.0f * A * A + AB + 2.0f * B * B) * iS3;
    const float ybi = -Y * (2.0f / 15.0f) * A * AB * (4.0f * A + B) * iS2;
    const float ybj = -Y * (2.0f / 15.0f) * AB * B * (A + 4.0f * B) * iS2;
    const float yci = Y * (8.0f / 15.0f) * A * A * AB * iS;
    const float ycj = Y * (8.0f / 15.0f) * AB * B * B * iS;
    const float ycx = Y * (2.0f / 15.0f) * AB * AB * iS;
    const float xg = X * 2.0f * AB * AB * iS2;
    const float yg = Y * (1.0f / 15.0f) * AB * (4.0f - 6.0f * AB * iS2);
    const float yhi = Y * iS2 * ((2.0f / 15.0f) * A * A * AB * (2.0f * A - B) + (1.0f / 15.0f) * AB * AB * (7.0f * A + B));
    const float yhj = Y * iS2 * ((1.0f / 15.0f) * AB * AB * (A + 7.0f * B) + (2.0f / 15.0f) * AB * B * B * (2.0f * B - A));
    const F3 dV = Vi - Vj;
    const float nV = dotf(nn, dV);
    const F3 fr = (xa * nV) * nn + ya * tangf(nn, dV) + ybi * crossf(nn, Wi) + ybj * crossf(nn, Wj);
    // strain of the shear rate acting on the pair (the wave of Eq. 17: the
    // mean of the two centres' local rates)
    const float rate = (EXT && g.wave) ? gd + 0.5f * (vi4.w + vj4.w) : gd;
    const F3 twoEn = f3(rate * nn.y, rate * nn.x, 0.0f);
    const float Pn = rate * nn.x * nn.y;
    const F3 Qn = twoEn - (2.0f * Pn) * nn;
    const F3 nperp = crossf(nn, twoEn);
    Fl = k6 * (((xg * Pn) * nn + yg * Qn) - fr);
    const F3 ndV = crossf(nn, dV);
    Tli = k6 * (ybi * ndV - (yci * tangf(nn, Wi) + ycx * tangf(nn, Wj)) + yhi * nperp);
    Tlj = k6 * (ybj * ndV - (ycx * tangf(nn, Wi) + ycj * tangf(nn, Wj)) + yhj * nperp);
    if (g.f.taper > 0.0f) {
      // differentiable cutoff: smoothstep over the last fraction w of the range
      const float dl = g.mode == 1 ? g.f.delta_a0 : g.f.delta * 0.5f * S;
      const float t = (dl - d) / (g.f.taper * dl);
      if (t < 1.0f) {
        const float s = t > 0.0f ? t * t * (3.0f - 2.0f * t) : 0.0f;
        Fl = s * Fl;
        Tli = s * Tli;
        Tlj = s * Tlj;
      }
    }
  }
  if (g.de > 0.0) Fc = Fc + m * nn;
  const F3 F = Fc + Fl;
  F3 Ti = Ai * nxf + Tli;
  F3 Tj = Bj * nxf + Tlj;
  if (EXT && g.k_r > 0.0) {
    Ti = Ti + Tr;
    Tj = Tj - Tr;
  }
  q.F[0] = F.x; q.F[1] = F.y; q.F[2] = F.z;
  q.Ti[0] = Ti.x; q.Ti[1] = Ti.y; q.Ti[2] = Ti.z;
  q.Tj[0] = Tj.x; q.Tj[1] = Tj.y; q.Tj[2] = Tj.z;
  q.Fc[0] = Fc.x; q.Fc[1] = Fc.y; q.Fc[2] = Fc.z;
  q.Fl[0] = Fl.x; q.Fl[1] = Fl.y; q.Fl[2] = Fl.z;
  q.r[0] = r.x; q.r[1] = r.y; q.r[2] = r.z;
  return q;
}

template <typename R>
__device__ __forceinline__ R owner_bits(int o);
template <>
__device__ __forceinline__ float owner_bits<float>(int o) { return __int_as_float(o); }
template <>
__device__ __forceinline__ double owner_bits<double>(int o) { return __longlong_as_double((long long)o); }
__device__ __forceinline__ int bits_owner(float v) { return __float_as_int(v); }
__device__ __forceinline__ int bits_owner(double v) { return (int)__double_as_longlong(v); }

__device__ __forceinline__ void load_record(const float* b, float* v) {
  const float4 p = reinterpret_cast<const float4*>(b)[0], q = reinterpret_cast<const float4*>(b)[1];
  v[0] = p.x; v[1] = p.y; v[2] = p.z; v[3] = p.w; v[4] = q.x; v[5] = q.y; v[6] = q.z; v[7] = q.w;
}
__device__ __forceinline__ void load_record(const double* b, double* v) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double2 p = reinterpret_cast<const double2*>(b)[k];
    v[2 * k] = p.x;
    v[2 * k + 1] = p.y;
  }
}

// A partner record (8 values, 32 B in FP32 / 64 B in FP64, slot-aligned) in
// wide stores.
__device__ __forceinline__ void store_record(float* b, float a0, float a1, float a2, float a3, float a4,
                                             float a5, float a6) {
  reinterpret_cast<float4*>(b)[0] = make_float4(a0, a1, a2, a3);
  reinterpret_cast<float4*>(b)[1] = make_float4(a4, a5, a6, 0.f);
}
__device__ __forceinline__ void store_record(double* b, double a0, double a1, double a2, double a3,
                                             double a4, double a5, double a6) {
  reinterpret_cast<double2*>(b)[0] = make_double2(a0, a1);
  reinterpret_cast<double2*>(b)[1] = make_double2(a2, a3);
  reinterpret_cast<double2*>(b)[2] = make_double2(a4, a5);
  reinterpret_cast<double2*>(b)[3] = make_double2(a6, 0.0);
}

// Per pair after its evaluation: the partner's share (-F and its torque)
// written to slot `slot` of the partner's row (taken by the caller with an
// atomic on the row's count) with the owner's index, the stretch records,
// the contact count and the stresslet of Eq. 9 (S^C = r (x) F^C,
// S^L = sym(r (x) F^L), F on the owner) added to the thread's sum.
template <typename R, bool EXT>
__device__ __forceinline__ void pair_commit(const Geo& g, const PairRes<R>& q, int i, int j, int p, ListBuf& W,
                                            int slot, R* __restrict__ bw, DevStatus* st, R Sx[9],
                                            int& ncont) {
  if (slot < g.M) {
    R* b = bw + ((int64_t)j * g.M + slot) * kSlot;
    store_record(b, -q.F[0], -q.F[1], -q.F[2], q.Tj[0], q.Tj[1], q.Tj[2], owner_bits<R>(i));
  } else {
    set_err(st, DSS_ERR_CAPACITY);
  }
  W.xi[p] = q.xrec;
  if (EXT && g.k_r > 0.0) W.xr[p] = q.rrec;
  ncont += q.contact;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b2 = 0; b2 < 3; ++b2)
      Sx[3 * a + b2] += q.r[a] * q.Fc[b2] + R(0.5) * (q.r[a] * q.Fl[b2] + q.r[b2] * q.Fl[a]);
}

// Number of values per warp-boundary slot of the pair-balanced kernel: force
// and torque (6), and with per-owner stresslets (batched instances) the
// owner's stresslet sum (9 more).
template <bool PERS>
__host__ __device__ constexpr int pb_slot() { return PERS ? 15 : 6; }

// Warp-segmented inclusive scan of the six force/torque sums over lanes with
// the same owner (seg; lanes of one owner are contiguous).
template <typename R, int NV = 6>
__device__ __forceinline__ void owner_scan(int lane, int seg, R v[NV]) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int so = __shfl_up_sync(0xffffffffu, seg, d);
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      const R u = __shfl_up_sync(0xffffffffu, v[c], d);
      if (lane >= d && so == seg) v[c] += u;
    }
  }
}

// The block's stresslet partials (fixed tree over lanes, warps and blocks):
// x0 the thread's sums for the instance of the block's first owner, x1 for
// the next instance (zero unless `second`), e0/e1 the single-particle wave
// stresslets the thread adds to them.  FP64 throughout in FP64.  In mixed
// precision the thread sums (one to a few pairs each) are FP32, the lanes and
// warps of the block are summed with compensation (Knuth's TwoSum on every
// addition, ~48 significant bits: an FP64 butterfly on every lane costs ~90
// additions per thread on GB300's narrow FP64 pipe, +40% on this kernel),
// and the block's sum is converted to FP64 once; every sum beyond the block
// is FP64.
template <bool MIXED, bool EXT>
__device__ __forceinline__ void stress_partials(
    const typename std::conditional<MIXED, float, double>::type* x0,
    const typename std::conditional<MIXED, float, double>::type* x1, bool second, double e0, double e1,
    int ncont, double* __restrict__ spart, DevStatus* st) {
  using R = typename std::conditional<MIXED, float, double>::type;
  __shared__ double red[MIXED ? 1 : kWarps][18];
  __shared__ float redh[MIXED ? kWarps : 1][18], redl[MIXED ? kWarps : 1][18];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // the second instance slot holds anything only where a lane of the warp
  // met a second instance (in its pairs, or as the owner of a wave stresslet)
  const int nq = __any_sync(0xffffffffu, second || e1 != 0.0) ? 18 : 9;
#pragma unroll
  for (int q = 0; q < 18; ++q) {
    if (q >= nq) {
      if (lane == 0) {
        if constexpr (MIXED) {
          redh[wid][q] = 0.0f;
          redl[wid][q] = 0.0f;
        } else {
          red[wid][q] = 0.0;
        }
      }
      continue;
    }
    const R x = q < 9 ? x0[q] : (second ? x1[q - 9] : R(0));
    const double e = (q == 1 || q == 3) ? e0 : ((q == 10 || q == 12) ? e1 : 0.0);
    if constexpr (MIXED) {
      FF v{x, 0.0f};
      if (EXT && e != 0.0) {
        v = two_sum(x, (float)e);
        v.lo += (float)(e - (double)(float)e);
      }
      for (int dlt = 16; dlt > 0; dlt >>= 1) {
        const float h2 = __shfl_down_sync(0xffffffffu, v.hi, dlt);
        const float l2 = __shfl_down_sync(0xffffffffu, v.lo, dlt);
        const FF t = two_sum(v.hi, h2);
        v.hi = t.hi;
        v.lo = (v.lo + l2) + t.lo;
      }
      if (lane == 0) {
        redh[wid][q] = v.hi;
        redl[wid][q] = v.lo;
      }
    } else {
      double v = (double)x + e;
      for (int dlt = 16; dlt > 0; dlt >>= 1) v += __shfl_down_sync(0xffffffffu, v, dlt);
      if (lane == 0) red[wid][q] = v;
    }
  }
  int c = ncont;
  for (int dlt = 16; dlt > 0; dlt >>= 1) c += __shfl_down_sync(0xffffffffu, c, dlt);
  if (lane == 0 && c) atomicAdd(&st->w[ST_NCONT], c);
  __syncthreads();
  if (threadIdx.x < 18) {
    if constexpr (MIXED) {
      const int q = threadIdx.x;
      FF v{redh[0][q], redl[0][q]};
      for (int w = 1; w < kWarps; ++w) {
        const FF t = two_sum(v.hi, redh[w][q]);
        v.hi = t.hi;
        v.lo = (v.lo + redl[w][q]) + t.lo;
      }
      spart[blockIdx.x * 18 + q] = (double)v.hi + (double)v.lo;
    } else {
      double v = 0.0;
      for (int w = 0; w < kWarps; ++w) v += red[w][threadIdx.x];
      spart[blockIdx.x * 18 + threadIdx.x] = v;
    }
  }
}

// MINB: resident blocks per SM the register budget is cut for (a grid that
// fills more than three blocks per SM gains from the fourth; smaller grids
// run faster with the larger budget).
template <bool MIXED, int MINB, bool EXT>
__global__ void __launch_bounds__(kPairThreads, MINB)
k_pairs(Geo g, const InstGeo* __restrict__ ig, const StepGeo* __restrict__ sgk, StateBuf s, ListBuf W,
        ListBuf H, const float4* __restrict__ posf, void* __restrict__ own_v, int* __restrict__ bw_count,
        void* __restrict__ bw_v, double* __restrict__ spart, DevStatus* st,
        const int* __restrict__ perm) {
  using R = typename std::conditional<MIXED, float, double>::type;
  if (dev_err(st)) return;
  R* __restrict__ own = static_cast<R*>(own_v);
  R* __restrict__ bw = static_cast<R*>(bw_v);
  const int n = g.n;
  const int P = W.start[n];
  const HistRef hr{perm, *((volatile const int*)&st->w[ST_IDORDER])};
  if (P > g.pcap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st->w[ST_NPAIRS] = P;
      set_err(st, DSS_ERR_CAPACITY);
    }
    return;
  }
  __shared__ R acc[kWarps][32][6];
  // The block's owners span at most two instances (an instance has at least
  // as many particles as a block has threads), and a lane meets its pairs in
  // increasing owner order, so its instance changes at most once: the
  // stresslet sum of the first instance is parked in shared memory then.
  __shared__ R park[kPairThreads][9];
  const int inst0 = s.inst[min((int)(blockIdx.x * blockDim.x), n - 1)];
  int cur_inst = inst0;
  R Sx[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  int ncont = 0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
#pragma unroll
  for (int c = 0; c < 6; ++c) acc[wid][lane][c] = R(0);
  __syncwarp();
  for (int w0 = gw * 32; w0 < n; w0 += nw * 32) {
    const int il = w0 + lane;
    const int cnt = il < n ? W.count[il] : 0;
    int incl = cnt;
    for (int d = 1; d < 32; d <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += t;
    }
    const int excl = incl - cnt;
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int base = W.start[w0];
    for (int t0 = 0; t0 < total; t0 += 32) {
      const int t = t0 + lane;
      int Lw = 0;
      for (int step = 16; step >= 1; step >>= 1) {
        const int e = __shfl_sync(0xffffffffu, excl, Lw + step);
        if (e <= t) Lw += step;
      }
      const int kk = t - __shfl_sync(0xffffffffu, excl, Lw);
      const bool valid = t < total;
      R v[6] = {0, 0, 0, 0, 0, 0};
      int seg = valid ? Lw : 32 + lane;      // owner lane, unique sentinel when idle
      if (valid) {
        const int i = w0 + Lw;
        const int p = base + t;
        const int j = W.list[(int64_t)i * g.Ms + kk];
        const int inst = s.inst[i];
        const InstGeo& I = ig[inst];
        const StepGeo sg = sgk[inst];
        PairRes<R> q;
        if constexpr (MIXED) q = pair_eval_mixed<EXT>(g, I, s, H, hr, sg, posf, i, j);
        else q = pair_eval_fp64<EXT>(g, I, s, H, hr, sg.off, i, j);
        v[0] = q.F[0]; v[1] = q.F[1]; v[2] = q.F[2];
        v[3] = q.Ti[0]; v[4] = q.Ti[1]; v[5] = q.Ti[2];
        if (inst != cur_inst) {
#pragma unroll
          for (int c = 0; c < 9; ++c) {
            park[threadIdx.x][c] = Sx[c];
            Sx[c] = R(0);
          }
          cur_inst = inst;
        }
        pair_commit<R, EXT>(g, q, i, j, p, W, atomicAdd(&bw_count[j], 1), bw, st, Sx, ncont);
      }
      owner_scan<R>(lane, seg, v);
      const int nxt = __shfl_down_sync(0xffffffffu, seg, 1);
      if (valid && (lane == 31 || nxt != seg)) {
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[wid][Lw][c] += v[c];
      }
      __syncwarp();
    }
    // one write per owner, then clear for the next group
    if (il < n) {
#pragma unroll
      for (int c = 0; c < 6; ++c) own[(int64_t)c * n + il] = acc[wid][lane][c];
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[wid][lane][c] = R(0);
    __syncwarp();
  }
  const bool moved = cur_inst != inst0;
  // With the wave of Eq. 17 the single-particle stresslets 20/3 pi eta0 a^3
  // E_inf(x) carry a local part, (10/3) pi eta0 a^3 U k cos(k y) on xy and
  // yx: one owner per thread (the grid covers each owner once), added to its
  // instance's slot.
  double ew0 = 0.0, ew1 = 0.0;
  if (EXT && g.wave) {
    const int il0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (il0 < n) {
      const double a = s.a[il0];
      const double e = (10.0 / 3.0) * DSS_PI * g.eta0 * a * a * a * s.wv[il0].y;
      if (s.inst[il0] == inst0) ew0 = e; else ew1 = e;
    }
  }
  R x0[9], x1[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    x0[c] = moved ? park[threadIdx.x][c] : Sx[c];
    x1[c] = moved ? Sx[c] : R(0);
  }
  stress_partials<MIXED, EXT>(x0, x1, moved, ew0, ew1, ncont, spart, st);
}

// Pair-balanced pair kernel.  The listed pairs in owner order (the compact
// arrays pown, pj written with the row offsets by the enumeration) are dealt
// out 32 to a warp over a grid of resident blocks, so every lane holds a pair
// whatever the row lengths.  An owner's pairs are contiguous: the
// warp-segmented scan sums each owner's share; an owner whose pairs lie in
// one warp is written once (own), one whose pairs cross a warp boundary
// leaves its part in the warp's head slot (continued from the previous warp)
// or tail slot (continuing into the next), which the gather adds in warp
// order.  Deterministic: the sums' order depends on the pair order alone.
// One instance (PERS = false): each thread sums the stresslets of its pairs
// and the blocks reduce them (stress_partials).  Batched instances (PERS):
// the stresslet of Eq. 9 rides along in the owner scan, so that each owner's
// stresslet sum is written with its force (own_s, or the boundary slots) and
// the gather's instance blocks add them up over the instance's particles.
template <bool MIXED, int MINB, bool EXT, bool PERS>
__global__ void __launch_bounds__(kPairThreads, MINB)
k_pairs_pb(Geo g, const InstGeo* __restrict__ ig, const StepGeo* __restrict__ sgk, StateBuf s, ListBuf W,
           ListBuf H, const float4* __restrict__ posf, void* __restrict__ own_v, void* __restrict__ own_s_v,
           void* __restrict__ carry_v, int* __restrict__ bw_count, void* __restrict__ bw_v,
           double* __restrict__ spart, DevStatus* st, const int* __restrict__ perm) {
  using R = typename std::conditional<MIXED, float, double>::type;
  constexpr int NV = pb_slot<PERS>();
  if (dev_err(st)) return;
  R* __restrict__ own = static_cast<R*>(own_v);
  R* __restrict__ own_s = static_cast<R*>(own_s_v);
  R* __restrict__ carry = static_cast<R*>(carry_v);
  R* __restrict__ bw = static_cast<R*>(bw_v);
  const int n = g.n;
  const int P = W.start[n];
  const HistRef hr{perm, *((volatile const int*)&st->w[ST_IDORDER])};
  if (P > g.pcap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st->w[ST_NPAIRS] = P;
      set_err(st, DSS_ERR_CAPACITY);
    }
    return;
  }
  R Sx[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  int ncont = 0;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int npw = (P + 31) >> 5;
  for (int pw = gw; pw < npw; pw += nw) {
    const int p = pw * 32 + lane;
    const bool valid = p < P;
    const int i = valid ? W.pown[p] : -1;
    const int j = valid ? W.pj[p] : 0;
    // the partner-record slot, taken first (its latency hides behind the pair)
    const int slot = valid ? atomicAdd(&bw_count[j], 1) : 0;
    // lane 0: does its owner continue from the previous warp?  lane 31: into
    // the next?
    const int before = (lane == 0 && valid && p > 0) ? W.pown[p - 1] : -1;
    const int after = (lane == 31 && p + 1 < P) ? W.pown[p + 1] : -1;
    R v[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) v[c] = R(0);
    const int seg = valid ? i : -2 - lane;   // owner, unique sentinel when idle
    if (valid) {
      const int inst = PERS ? s.inst[i] : 0;
      const InstGeo& I = ig[inst];
      const StepGeo sg = sgk[inst];
      PairRes<R> q;
      if constexpr (MIXED) q = pair_eval_mixed<EXT>(g, I, s, H, hr, sg, posf, i, j);
      else q = pair_eval_fp64<EXT>(g, I, s, H, hr, sg.off, i, j);
      v[0] = q.F[0]; v[1] = q.F[1]; v[2] = q.F[2];
      v[3] = q.Ti[0]; v[4] = q.Ti[1]; v[5] = q.Ti[2];
      if constexpr (PERS) {
        R Sp[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        pair_commit<R, EXT>(g, q, i, j, p, W, slot, bw, st, Sp, ncont);
#pragma unroll
        for (int c = 0; c < 9; ++c) v[6 + c] = Sp[c];
      } else {
        pair_commit<R, EXT>(g, q, i, j, p, W, slot, bw, st, Sx, ncont);
      }
    }
    owner_scan<R, NV>(lane, seg, v);
    const int nxt = __shfl_down_sync(0xffffffffu, seg, 1);
    const int head = __shfl_sync(0xffffffffu, (before >= 0 && before == seg) ? seg : -1, 0);
    if (valid && (lane == 31 || nxt != seg)) {
      R* dst = nullptr;
      if (seg == head) dst = carry + (int64_t)pw * 2 * NV;                // continued from before
      else if (after == seg) dst = carry + (int64_t)pw * 2 * NV + NV;     // continues after (lane 31)
      if (dst) {
#pragma unroll
        for (int c = 0; c < NV; ++c) dst[c] = v[c];
      } else {
#pragma unroll
        for (int c = 0; c < 6; ++c) own[(int64_t)c * n + i] = v[c];
        if constexpr (PERS) {
#pragma unroll
          for (int c = 0; c < 9; ++c) own_s[(int64_t)c * n + i] = v[6 + c];
        }
      }
    }
  }
  if constexpr (PERS) {
    const int c = __reduce_add_sync(0xffffffffu, ncont);
    if (lane == 0 && c) atomicAdd(&st->w[ST_NCONT], c);
  } else {
    // the wave's single-particle stresslets (see k_pairs), particles strided
    // over the grid's threads
    double ew0 = 0.0;
    if (EXT && g.wave) {
      for (int il = blockIdx.x * blockDim.x + threadIdx.x; il < n; il += gridDim.x * blockDim.x) {
        const double a = s.a[il];
        ew0 += (10.0 / 3.0) * DSS_PI * g.eta0 * a * a * a * s.wv[il].y;
      }
    }
    stress_partials<MIXED, EXT>(Sx, Sx, false, ew0, 0.0, ncont, spart, st);
  }
}

// Bulk stress (Eq. 8) of one instance from the pair blocks' partials, by one
// block of the gather (fixed strided assignment and fixed tree).  Pair block b
// holds the sums of the instance containing its first owner (slot 0) and of
// the next instance (slot 1).
// With the pair-balanced kernel (one instance, pb_blocks > 0) every block's
// first slot belongs to the instance.
__device__ void inst_stress(const Geo& g, const InstGeo& I, const double* __restrict__ spart,
                            double* __restrict__ sigma, int pb_blocks) {
  __shared__ double red[kThreads / 32][9];
  double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  const int b0 = pb_blocks ? 0 : I.p_begin / kPairThreads;
  const int b1 = pb_blocks ? pb_blocks - 1 : (I.p_end - 1) / kPairThreads;
  for (int b = b0 + threadIdx.x; b <= b1; b += blockDim.x) {
    const double* p = spart + b * 18 + (pb_blocks || b * kPairThreads >= I.p_begin ? 0 : 9);
#pragma unroll
    for (int q = 0; q < 9; ++q) v[q] += p[q];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    for (int d = 16; d > 0; d >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], d);
    if (lane == 0) red[wid][q] = v[q];
  }
  __syncthreads();
  if (threadIdx.x < 9) {
    const int q = threadIdx.x;
    double S = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) S += red[w][q];
    // E_inf: only xy and yx are non-zero (gdot/2)
    const double E = (q == 1 || q == 3) ? 0.5 * I.gdot : 0.0;
    const double V = I.L[0] * I.L[1] * I.L[2];
    const double ein = 20.0 / 3.0 * DSS_PI * g.eta0 * I.sumA3;
    sigma[q] = 2.0 * g.eta0 * E + (ein * E + S) / V;
  }
}

// Bulk stress (Eq. 8) of batched instances from their owners' stresslet sums
// (the pair-balanced kernel with per-owner stresslets): kOsParts blocks per
// instance, each summing a slice of its particles in a fixed strided order
// and tree: per particle its own-row sum, or the tail slot of its first
// warp plus the head slots of the next ones (as the forces), and with the
// wave of Eq. 17 its local single-particle stresslet.  The gather's instance
// blocks add the slices (inst_stress_parts).
constexpr int kOsParts = 16;

template <bool MIXED, bool EXT>
__global__ void __launch_bounds__(kPairThreads)
k_owner_stress(Geo g, const InstGeo* __restrict__ ig, StateBuf s, const void* __restrict__ own_s_v,
               const void* __restrict__ carry_v, const int* __restrict__ start, double* __restrict__ spart,
               DevStatus* st) {
  using R = typename std::conditional<MIXED, float, double>::type;
  if (dev_err(st)) return;
  const R* __restrict__ own_s = static_cast<const R*>(own_s_v);
  const R* __restrict__ carry = static_cast<const R*>(carry_v);
  constexpr int64_t cs = 2 * 15;
  const int n = g.n;
  const int k = blockIdx.x / kOsParts, part = blockIdx.x % kOsParts;
  const InstGeo& I = ig[k];
  const int chunk = (I.p_end - I.p_begin + kOsParts - 1) / kOsParts;
  const int j0 = I.p_begin + part * chunk, j1 = min(I.p_end, j0 + chunk);
  // each thread sums its particles' owner sums in the pair arithmetic's
  // precision (a few each), then the block's lanes and warps as in the pair
  // kernel (compensated in mixed precision), one FP64 value per block
  R v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  double ew = 0.0;
  for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
    const int s0 = start[j], s1 = start[j + 1];
    if (s1 > s0) {
      const int w0 = s0 >> 5, w1 = (s1 - 1) >> 5;
      if (w0 == w1) {
#pragma unroll
        for (int q = 0; q < 9; ++q) v[q] += own_s[(int64_t)q * n + j];
      } else {
#pragma unroll
        for (int q = 0; q < 9; ++q) v[q] += carry[w0 * cs + 15 + 6 + q];
        for (int w = w0 + 1; w <= w1; ++w)
#pragma unroll
          for (int q = 0; q < 9; ++q) v[q] += carry[w * cs + 6 + q];
      }
    }
    if (EXT && g.wave) {
      const double a = s.a[j];
      ew += (10.0 / 3.0) * DSS_PI * g.eta0 * a * a * a * s.wv[j].y;
    }
  }
  stress_partials<MIXED, EXT>(v, v, false, ew, 0.0, 0, spart, st);
}

// The instance's stress from its kOsParts slices (by one block of the gather).
__device__ void inst_stress_parts(const Geo& g, const InstGeo& I, const double* __restrict__ parts,
                                  double* __restrict__ sigma) {
  if (threadIdx.x < 9) {
    const int q = threadIdx.x;
    double S = 0.0;
    for (int p = 0; p < kOsParts; ++p) S += parts[p * 18 + q];
    const double E = (q == 1 || q == 3) ? 0.5 * I.gdot : 0.0;
    const double V = I.L[0] * I.L[1] * I.L[2];
    const double ein = 20.0 / 3.0 * DSS_PI * g.eta0 * I.sumA3;
    sigma[q] = 2.0 * g.eta0 * E + (ein * E + S) / V;
  }
}

// Step commit, by the last block of the gather to finish.
__device__ void commit_step(const Geo& g, DevStatus* st, const int* __restrict__ start, int step) {
  if (dev_err(st)) return;
  st->w[ST_NPAIRS] = start[g.n];
  if (step) {
    st->w[ST_IDORDER] = 0;   // the new history rows follow the committed order
    st->w[ST_STEPS] += 1;
    int64_t ns = dev_nstep(st) + 1;
    st->w[ST_NSTEP_LO] = (int)(uint32_t)(ns & 0xffffffffll);
    st->w[ST_NSTEP_HI] = (int)(ns >> 32);
  }
}

// Sums one particle's partner records in increasing owner index.  Owners are
// distinct within a row; the rank of each record is counted in registers
// for rows of up to 8 records, otherwise by repeated minimum search.
template <typename R>
__device__ __forceinline__ void sum_records(const R* __restrict__ row, int cnt, R* F, R* T) {
  if (cnt <= 8) {
    int ow[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) ow[q] = q < cnt ? bits_owner(row[q * kSlot + 6]) : INT_MAX;
    int rk[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      int r0 = 0;
#pragma unroll
      for (int r = 0; r < 8; ++r) r0 += (ow[r] < ow[q]) || (ow[r] == ow[q] && r < q);
      rk[q] = r0;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      if (t < cnt) {
        int sel = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) sel = rk[q] == t ? q : sel;
        R b[8];
        load_record(row + sel * kSlot, b);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          F[c] += b[c];
          T[c] += b[3 + c];
        }
      }
    }
    return;
  }
}

constexpr int kHeavyWin = 256;   // ranks placed per pass of a heavy row
constexpr int kRankedMax = 24;   // FP32 rows up to this length are summed in owner order

// FP32 value as a fixed-point integer in units of 2^(e - 126 - bits), e the
// largest biased exponent of its row: the 24-bit significand shifted left by
// bits - 24 - (e - e_v) (at most bits - 24), or right with the low bits
// dropped.  Zero and denormals give 0.  Integer operations only, so the
// value is the same on every path.
__device__ __forceinline__ long long fx_of(float v, int e, int bits) {
  const int u = __float_as_int(v);
  const int ev = (u >> 23) & 0xff;
  if (ev == 0) return 0;
  long long m = (long long)((u & 0x7fffff) | 0x800000);
  const int sh = bits - 24 - (e - ev);
  m = sh >= 0 ? (m << sh) : (sh > -25 ? (m >> -sh) : 0);
  return u < 0 ? -m : m;
}

// A row of more than 8 FP32 records (mixed precision), summed by its own
// thread in 64-bit fixed point.  Per component the largest exponent e of the
// row fixes the unit 2^(e - 126 - bits), bits = 62 - ceil(log2(cc + 1)), so
// that every record is an integer below 2^bits and the row's sum stays below
// 2^62 (a first pass finds e, a second adds; four records in flight per
// thread).  Integer addition is
// associative: the total is a function of the set of records alone, whatever
// their order in the row, so no ranking and no help from the other lanes is
// needed.  It is exact up to the dropped bits below 2^-(bits - 24) of each
// record relative to the row's largest (more accurate than an FP32 running
// sum).  A non-finite record makes the total NaN.
__device__ __forceinline__ void row_sum_fixed(const float* __restrict__ row, int cc, float tot[6]) {
  int e[6] = {0, 0, 0, 0, 0, 0};
  bool bad = false;
  int k = 0;
  for (; k + 4 <= cc; k += 4) {
    float b[4][8];
#pragma unroll
    for (int t = 0; t < 4; ++t) load_record(row + (k + t) * kSlot, b[t]);
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const int ev = (__float_as_int(b[t][c]) >> 23) & 0xff;
        e[c] = max(e[c], ev);
        bad |= ev == 0xff;
      }
  }
  for (; k < cc; ++k) {
    float b[8];
    load_record(row + k * kSlot, b);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const int ev = (__float_as_int(b[c]) >> 23) & 0xff;
      e[c] = max(e[c], ev);
      bad |= ev == 0xff;
    }
  }
  const int bits = 62 - (32 - __clz(cc));
  long long acc[6] = {0, 0, 0, 0, 0, 0};
  k = 0;
  for (; k + 4 <= cc; k += 4) {
    float b[4][8];
#pragma unroll
    for (int t = 0; t < 4; ++t) load_record(row + (k + t) * kSlot, b[t]);
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int c = 0; c < 6; ++c) acc[c] += fx_of(b[t][c], e[c], bits);
  }
  for (; k < cc; ++k) {
    float b[8];
    load_record(row + k * kSlot, b);
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[c] += fx_of(b[c], e[c], bits);
  }
#pragma unroll
  for (int c = 0; c < 6; ++c)
    tot[c] = bad ? __int_as_float(0x7fc00000) : (float)ldexp((double)acc[c], e[c] - 126 - bits);
}

// A row of more than 8 records, summed by the whole warp: each record's rank
// in owner order is counted (the lanes read the owner words together), the
// ranks are placed in a per-warp table, and the records are added in rank
// order, lane k taking ranks k, k + 32, ..., then a fixed butterfly.  The
// result is a function of the set of records alone.  Every lane returns the
// total.
template <typename R>
__device__ __forceinline__ void warp_sum_row(const R* __restrict__ row, int cc, int* slots, R tot[6]) {
  const int lane = threadIdx.x & 31;
  R part[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
  for (int base = 0; base < cc; base += kHeavyWin) {
    for (int q = lane; q < cc; q += 32) {
      const int oq = bits_owner(row[q * kSlot + 6]);
      int rk = 0;
      for (int r = 0; r < cc; ++r) {
        const int o = bits_owner(row[r * kSlot + 6]);
        rk += (o < oq) || (o == oq && r < q);
      }
      if (rk >= base && rk < base + kHeavyWin) slots[rk - base] = q;
    }
    __syncwarp();
    const int we = min(cc - base, kHeavyWin);
    for (int k = lane; k < we; k += 32) {
      R b[8];
      load_record(row + slots[k] * kSlot, b);
#pragma unroll
      for (int c = 0; c < 6; ++c) part[c] += b[c];
    }
    __syncwarp();
  }
#pragma unroll
  for (int c = 0; c < 6; ++c) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) part[c] += __shfl_xor_sync(0xffffffffu, part[c], d);
    tot[c] = part[c];
  }
}

// Total force and torque on particle j (its own pair sum, its partner
// records, Stokes drag), then the accelerations and, in a step, the velocity
// half-kick of Eq. 15d.  Returns true when the sums are not finite (the
// error is then set).  Every load that does not depend on the partner rows
// is issued first.
template <bool MIXED, bool EXT>
__device__ __forceinline__ bool gather_one(const Geo& g, const InstGeo* __restrict__ ig, const StateBuf& s,
                                           const void* __restrict__ own_v,
                                           const int* __restrict__ bw_count, const void* __restrict__ bw_v,
                                           double* __restrict__ Fout, double* __restrict__ Tout,
                                           DevStatus* st, int mode, int j0, int* slots,
                                           const void* __restrict__ carry_v, int cnv,
                                           const int* __restrict__ start) {
  using R = typename std::conditional<MIXED, float, double>::type;
  const R* __restrict__ own = static_cast<const R*>(own_v);
  const R* __restrict__ carry = static_cast<const R*>(carry_v);
  const R* __restrict__ bw = static_cast<const R*>(bw_v);
  const int n = g.n;
  // every lane of the warp takes part in the long FP64 rows below; lanes
  // past the last particle work on particle 0 and write nothing
  const bool valid = j0 < n;
  const int j = valid ? j0 : 0;
  int cnt = valid ? __ldg(bw_count + j) : 0;
  R F[3], T[3];
  if (carry) {
    // pair-balanced sums: none (no owned pair), the owner's single write, or
    // the tail slot of its first warp plus the head slots of the next ones
    const int s0 = __ldg(start + j), s1 = __ldg(start + j + 1);
    const int w0 = s0 >> 5, w1 = (s1 - 1) >> 5;
#pragma unroll
    for (int c = 0; c < 3; ++c) F[c] = T[c] = R(0);
    if (s1 > s0 && w0 == w1) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        F[c] = own[(int64_t)c * n + j];
        T[c] = own[(int64_t)(3 + c) * n + j];
      }
    } else if (s1 > s0) {
      const int64_t cs = 2 * cnv;   // head slot, tail slot
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        F[c] = carry[w0 * cs + cnv + c];
        T[c] = carry[w0 * cs + cnv + 3 + c];
      }
      for (int w = w0 + 1; w <= w1; ++w) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          F[c] += carry[w * cs + c];
          T[c] += carry[w * cs + 3 + c];
        }
      }
    }
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      F[c] = own[(int64_t)c * n + j];
      T[c] = own[(int64_t)(3 + c) * n + j];
    }
  }
  const double a = __ldg(s.a + j);
  const int id = __ldg(s.id + j);
  const bool stepm = mode == G_STEP;
  const double* __restrict__ su = s.u;
  const double* __restrict__ sw = s.w;
  double u[3] = {0.0, 0.0, 0.0}, w[3] = {0.0, 0.0, 0.0};
  float4 v4 = make_float4(0.f, 0.f, 0.f, 0.f), w4 = v4;
  double yj = 0.0, gd = 0.0, fx = 0.0;
  double2 wq = make_double2(0.0, 0.0);
  if constexpr (MIXED) {
    v4 = __ldg(s.vf + j);
    w4 = __ldg(s.wf + j);
  } else {
    yj = __ldg(s.x + n + j);
    gd = __ldg(&ig[__ldg(s.inst + j)].gdot);
  }
  if (EXT && g.wave) {
    fx = __ldg(&ig[__ldg(s.inst + j)].faxen_c);
    if constexpr (!MIXED) wq = s.wv[j];
  }
  if (!MIXED || stepm) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      u[c] = su[c * n + j];
      w[c] = sw[c * n + j];
    }
  }
  cnt = cnt < g.M ? cnt : g.M;
  if (cnt <= 8) {
    sum_records<R>(bw + (int64_t)j * g.M * kSlot, cnt, F, T);
  } else if constexpr (MIXED) {
    if (cnt > kRankedMax) {
      // long FP32 rows: each thread its own, in fixed point
      float tot[6];
      row_sum_fixed(bw + (int64_t)j * g.M * kSlot, cnt, tot);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        F[c] += tot[c];
        T[c] += tot[3 + c];
      }
    }
  }
  {
    // rows of 9..kRankedMax FP32 records, and every longer FP64 row: the
    // whole warp, one row after another, in owner order
    unsigned heavy = __ballot_sync(0xffffffffu, cnt > 8 && (!MIXED || cnt <= kRankedMax));
    while (heavy) {
      const int src = __ffs(heavy) - 1;
      heavy &= heavy - 1u;
      const int jj = __shfl_sync(0xffffffffu, j, src), cc = __shfl_sync(0xffffffffu, cnt, src);
      R tot[6];
      warp_sum_row<R>(bw + (int64_t)jj * g.M * kSlot, cc, slots, tot);
      if ((int)(threadIdx.x & 31) == src) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          F[c] += tot[c];
          T[c] += tot[3 + c];
        }
      }
    }
  }
  if (!valid) return false;
  if constexpr (MIXED) {
    // Stokes drag on the FP32 velocities relative to the ambient flow (with
    // the wave of Eq. 17, relative to the Faxen velocity of Eq. A1:
    // u - (1 + a^2/6 Laplacian) U_inf = (u - U_inf) + a^2 k^2/6 U sin(k y))
    const float af = (float)a;
    const float kd = -g.f.k6 * af, kr = -g.f.k8 * af * af * af;
    const float vx = (EXT && g.wave) ? v4.x + (float)(a * a * fx) * w4.w : v4.x;
    F[0] += kd * vx; F[1] += kd * v4.y; F[2] += kd * v4.z;
    T[0] += kr * w4.x; T[1] += kr * w4.y; T[2] += kr * w4.z;
  } else {
    // FP64: each product and sum rounded on its own (no contraction), in the
    // order of the plain evaluation -6 pi eta0 a (u - U_inf)
    const double kd = __dmul_rn(-g.k6, a);
    const double kr = __dmul_rn(__dmul_rn(__dmul_rn(-g.k8, a), a), a);
    double vx, wz;
    if (EXT && g.wave) {
      // Faxen velocity (1 + a^2/6 Laplacian) U_inf,x and local Omega_inf
      vx = u[0] - gd * yj - (1.0 - a * a * fx) * wq.x;
      wz = w[2] + 0.5 * (gd + wq.y);
    } else {
      vx = __dsub_rn(u[0], __dmul_rn(gd, yj));
      wz = __dadd_rn(w[2], __dmul_rn(0.5, gd));
    }
    F[0] = __dadd_rn(F[0], __dmul_rn(kd, vx));
    F[1] = __dadd_rn(F[1], __dmul_rn(kd, u[1]));
    F[2] = __dadd_rn(F[2], __dmul_rn(kd, u[2]));
    T[0] = __dadd_rn(T[0], __dmul_rn(kr, w[0]));
    T[1] = __dadd_rn(T[1], __dmul_rn(kr, w[1]));
    T[2] = __dadd_rn(T[2], __dmul_rn(kr, wz));
  }
  bool bad = false;
  if (!(isfinite(F[0]) && isfinite(F[1]) && isfinite(F[2]) && isfinite(T[0]) && isfinite(T[1]) &&
        isfinite(T[2]))) {
    set_err(st, DSS_ERR_NONFINITE);
    bad = true;
  }
  if (mode == G_EVAL) {
    if (Fout) { Fout[id] = F[0]; Fout[n + id] = F[1]; Fout[2 * n + id] = F[2]; }
    if (Tout) { Tout[id] = T[0]; Tout[n + id] = T[1]; Tout[2 * n + id] = T[2]; }
    return bad;
  }
  // accelerations: m = 4/3 pi rho a^3, I = 2/5 m a^2
  R al[3], aw[3];
  if constexpr (MIXED) {
    const float af = (float)a;
    const float imr = 1.0f / (g.f.mass_c * af * af * af);
    const float iIr = imr * (2.5f / (af * af));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      al[c] = F[c] * imr;
      aw[c] = T[c] * iIr;
    }
  } else {
    // FP64: F/m and T/I as IEEE divisions, m and I formed left to right
    const double m = __dmul_rn(__dmul_rn(__dmul_rn(__dmul_rn(4.0 / 3.0 * DSS_PI, g.rho), a), a), a);
    const double I = __dmul_rn(__dmul_rn(__dmul_rn(0.4, m), a), a);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      al[c] = __ddiv_rn(F[c], m);
      aw[c] = __ddiv_rn(T[c], I);
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    s.al[c * n + j] = al[c];
    s.aw[c * n + j] = aw[c];
  }
  if (stepm) {
    // Eq. 15d from u^{n+1/2}: u^{n+1} = u^{n+1/2} + dt/2 alpha^{n+1} (FP64
    // mode: product and sum rounded separately)
    const double hdt = g.hdt;
    if constexpr (MIXED) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        s.u[c * n + j] = __fma_rn(hdt, (double)al[c], u[c]);
        s.w[c * n + j] = __fma_rn(hdt, (double)aw[c], w[c]);
      }
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        s.u[c * n + j] = __dadd_rn(u[c], __dmul_rn(hdt, (double)al[c]));
        s.w[c * n + j] = __dadd_rn(w[c], __dmul_rn(hdt, (double)aw[c]));
      }
    }
  }
  return bad;
}

// Blocks 0..K-1 reduce the bulk stress of instance k (scheduled first, off
// the particles' critical path); the blocks after them take one particle per
// thread.  At most 80 registers, so that six blocks fit on an SM and a
// 100k-particle grid runs in one wave.  The last block to finish commits the step; only the writes that
// block reads (the stresses, an error code) are fenced before the count.
template <bool MIXED, bool EXT>
__global__ void __launch_bounds__(kThreads, 6)
k_gather(Geo g, const InstGeo* __restrict__ ig, StateBuf s, const void* __restrict__ own_v,
         const int* __restrict__ bw_count, const void* __restrict__ bw_v, double* __restrict__ Fout,
         double* __restrict__ Tout, DevStatus* st, int mode, const double* __restrict__ spart,
         double* sigma, double* sigma_sum, const int* __restrict__ start, unsigned int* done_blocks,
         const void* __restrict__ carry_v, int pb_blocks, const void* __restrict__ own_s_v) {
  // An error set before this kernel (an earlier kernel of the step, or an
  // earlier step of the same dss_step call, whose successors still replay)
  // means this step is void: touch no state, since the buffer this step
  // would write can be the committed one.  Every block still reaches the
  // counter below.
  __shared__ int s_err0;
  __shared__ int s_slot[kThreads / 32][kHeavyWin];
  if (threadIdx.x == 0) s_err0 = dev_err(st);
  __syncthreads();
  bool fence = false;
  if (!s_err0) {
    if (blockIdx.x < (unsigned)g.K) {
      if (own_s_v)
        inst_stress_parts(g, ig[blockIdx.x], spart + (int64_t)blockIdx.x * kOsParts * 18,
                          sigma + 9 * blockIdx.x);
      else
        inst_stress(g, ig[blockIdx.x], spart, sigma + 9 * blockIdx.x, pb_blocks);
      fence = threadIdx.x < 9;
    } else {
      const int j = (int)(blockIdx.x - g.K) * blockDim.x + threadIdx.x;
      fence = gather_one<MIXED, EXT>(g, ig, s, own_v, bw_count, bw_v, Fout, Tout, st, mode, j,
                                s_slot[threadIdx.x >> 5], carry_v, own_s_v ? 15 : 6, start);
    }
  }
  __shared__ bool last;
  if (fence) __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(done_blocks, 1u) == gridDim.x - 1;
  __syncthreads();
  if (last) {
    __threadfence();
    __shared__ int s_err;
    if (threadIdx.x == 0) s_err = dev_err(st);
    __syncthreads();
    // a committed step adds every instance's stress to the running sums
    if (!s_err && mode == G_STEP)
      for (int t = threadIdx.x; t < 9 * g.K; t += blockDim.x) sigma_sum[t] += __ldcg(sigma + t);
    if (threadIdx.x == 0) commit_step(g, st, start, mode == G_STEP ? 1 : 0);
    if (threadIdx.x == 0) *done_blocks = 0u;
  }
}

// Pairs of a list as (lo id, hi id) in owner order (for dss_get_pairs).
__global__ void k_pairs_out(Geo g, ListBuf W, long long* __restrict__ out) {
  const int n = g.n;
  const int P = W.start[n];
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (W.start[mid] <= p) lo = mid; else hi = mid;
    }
    const int j = W.list[(int64_t)lo * g.Ms + (p - W.start[lo])];
    const int a = W.id_of_slot[lo], b = W.id_of_slot[j];
    out[2 * (int64_t)p] = a < b ? a : b;
    out[2 * (int64_t)p + 1] = a < b ? b : a;
  }
}
}  // namespace

// One warp per 32 owners: ceil(n / kPairThreads) blocks cover every owner
// once (the pair kernel also strides when given fewer).
int pair_grid_blocks(const dss_handle* h) {
  int64_t need = (h->n + kPairThreads - 1) / kPairThreads;
  return (int)(need > 0 ? need : 1);
}

// The pair-balanced kernel's grid: the blocks its
// register budget keeps resident on every SM (3 of 256 threads in mixed
// precision, 2 in FP64), their warps striding over the warps of pairs.
int pair_pb_blocks(const dss_handle* h) {
  return h->sms * (h->g.precision == DSS_MIXED ? 3 : 2);
}

int bw_slot_values() { return kSlot; }

namespace {
// The pair and gather kernels of one configuration (EXT: the wave of Eq. 17
// or rolling resistance is on; the plain kernels carry none of its code).
template <bool EXT>
void launch_forces_t(dss_handle* h, int stbuf, int work_list, int hist_list, int adv, int mode,
                     double* F_out, double* T_out) {
  (void)adv;
  const int n = (int)h->n;
  const int pb = pair_grid_blocks(h);
  const bool mixed = h->g.precision == DSS_MIXED;
  prof_mark(h, 5);
  // pairs dealt out 32 to a warp over the resident blocks (batched
  // instances: with per-owner stresslets)
  const bool pbal = h->pb_blocks > 0 && h->compact_ok[work_list];
  const bool pers = h->g.K > 1;
  const bool big = h->tune_pairs_minb ? h->tune_pairs_minb == 4 : pb > 3 * h->sms;
  // the balanced grid: the resident blocks of its register budget (mixed
  // precision: 3 per SM, or, for one instance, 4 when the kernel autotuner
  // chose the smaller budget)
  const bool pb4 = pbal && mixed && !pers && h->tune_pairs_minb == 4;
  const int pbg = pb4 ? 4 * h->sms : h->pb_blocks;
#define DSS_PB_ARGS                                                                                     \
  h->g, h->ig, h->sg, h->st[stbuf], h->lb[work_list], h->lb[hist_list], h->posf, h->own, h->own_s,    \
      h->carry, h->bw_count, h->bw_rec, h->spart, h->status, h->perm
  if (pb4)
    k_pairs_pb<true, 4, EXT, false><<<pbg, kPairThreads, 0, h->stream>>>(DSS_PB_ARGS);
  else if (pbal && mixed && pers)
    k_pairs_pb<true, 3, EXT, true><<<pbg, kPairThreads, 0, h->stream>>>(DSS_PB_ARGS);
  else if (pbal && mixed)
    k_pairs_pb<true, 3, EXT, false><<<pbg, kPairThreads, 0, h->stream>>>(DSS_PB_ARGS);
  else if (pbal && pers)
    k_pairs_pb<false, 2, EXT, true><<<pbg, kPairThreads, 0, h->stream>>>(DSS_PB_ARGS);
  else if (pbal)
    k_pairs_pb<false, 2, EXT, false><<<pbg, kPairThreads, 0, h->stream>>>(DSS_PB_ARGS);
#undef DSS_PB_ARGS
  else if (mixed && big)
    k_pairs<true, 4, EXT><<<pb, kPairThreads, 0, h->stream>>>(
        h->g, h->ig, h->sg, h->st[stbuf], h->lb[work_list], h->lb[hist_list], h->posf, h->own, h->bw_count,
        h->bw_rec, h->spart, h->status, h->perm);
  else if (mixed)
    k_pairs<true, 3, EXT><<<pb, kPairThreads, 0, h->stream>>>(
        h->g, h->ig, h->sg, h->st[stbuf], h->lb[work_list], h->lb[hist_list], h->posf, h->own, h->bw_count,
        h->bw_rec, h->spart, h->status, h->perm);
  else
    k_pairs<false, 2, EXT><<<pb, kPairThreads, 0, h->stream>>>(
        h->g, h->ig, h->sg, h->st[stbuf], h->lb[work_list], h->lb[hist_list], h->posf, h->own, h->bw_count,
        h->bw_rec, h->spart, h->status, h->perm);
  prof_mark(h, 6);
  const int gb = (n + kThreads - 1) / kThreads + h->g.K;
  const void* carry = pbal ? h->carry : nullptr;
  const int pbb = pbal ? pbg : 0;
  const void* own_s = pbal && pers ? h->own_s : nullptr;
  if (own_s) {
    if (mixed)
      k_owner_stress<true, EXT><<<h->g.K * kOsParts, kPairThreads, 0, h->stream>>>(
          h->g, h->ig, h->st[stbuf], own_s, carry, h->lb[work_list].start, h->spart, h->status);
    else
      k_owner_stress<false, EXT><<<h->g.K * kOsParts, kPairThreads, 0, h->stream>>>(
          h->g, h->ig, h->st[stbuf], own_s, carry, h->lb[work_list].start, h->spart, h->status);
  }
  if (mixed)
    k_gather<true, EXT><<<gb, kThreads, 0, h->stream>>>(h->g, h->ig, h->st[stbuf], h->own, h->bw_count,
                                                        h->bw_rec, F_out, T_out, h->status, mode, h->spart,
                                                        h->sigma, h->sigma_sum, h->lb[work_list].start,
                                                        h->done_blocks, carry, pbb, own_s);
  else
    k_gather<false, EXT><<<gb, kThreads, 0, h->stream>>>(h->g, h->ig, h->st[stbuf], h->own, h->bw_count,
                                                         h->bw_rec, F_out, T_out, h->status, mode, h->spart,
                                                         h->sigma, h->sigma_sum, h->lb[work_list].start,
                                                         h->done_blocks, carry, pbb, own_s);
  prof_mark(h, 7);
}
}  // namespace

void launch_forces(dss_handle* h, int stbuf, int work_list, int hist_list, int adv, int mode,
                   double* F_out, double* T_out) {
  if (h->g.wave || h->g.k_r > 0.0)
    launch_forces_t<true>(h, stbuf, work_list, hist_list, adv, mode, F_out, T_out);
  else
    launch_forces_t<false>(h, stbuf, work_list, hist_list, adv, mode, F_out, T_out);
}

void launch_pairs_out(dss_handle* h, int list, long long* out) {
  k_pairs_out<<<pair_grid_blocks(h), kPairThreads, 0, h->stream>>>(h->g, h->lb[list], out);
}
