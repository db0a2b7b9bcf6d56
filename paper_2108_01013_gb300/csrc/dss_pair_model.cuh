// The pair model of one listed pair (FP64 arithmetic), written over a scalar
// type T (the FP64 force pass; the adjoint's hand-written reverse in
// dss_adjoint.cu follows its operations one by one).  Branches (contact,
// Coulomb slip, gap clamp, taper ends) are taken on the values.
//
// Contact: Eq. 4-5 (linear spring-dashpot normal force, tangential spring
// with the stretch carried between steps, Coulomb rescale of the stretch).
// Lubrication: App. A (Eq. A2, A3 with the coefficient functions of Eq. A6,
// A7 and the 6 pi eta0 prefactor) in the simple shear of Sec. II; with a
// taper width w > 0 the lubrication force and torques are scaled by
// s = t^2 (3 - 2t), t = clamp((delta_ij - d) / (w delta_ij), 0, 1) (an
// extension that makes the cutoff differentiable; w = 0 is the hard cutoff).
#pragma once

#include "dss_internal.cuh"

// ---------------------------------------------------------------- scalars
__device__ __forceinline__ double val(double x) { return x; }

template <typename T>
__device__ __forceinline__ T cst(double c);
template <>
__device__ __forceinline__ double cst<double>(double c) { return c; }

// ---------------------------------------------------------------- vectors
template <typename T>
struct Vec3 {
  T x, y, z;
};
template <typename T>
__device__ __forceinline__ Vec3<T> mk3(T a, T b, T c) { return Vec3<T>{a, b, c}; }
template <typename T>
__device__ __forceinline__ Vec3<T> operator+(const Vec3<T>& a, const Vec3<T>& b) {
  return mk3<T>(a.x + b.x, a.y + b.y, a.z + b.z);
}
template <typename T>
__device__ __forceinline__ Vec3<T> operator-(const Vec3<T>& a, const Vec3<T>& b) {
  return mk3<T>(a.x - b.x, a.y - b.y, a.z - b.z);
}
template <typename T, typename S>
__device__ __forceinline__ Vec3<T> operator*(const S& s, const Vec3<T>& a) {
  return mk3<T>(s * a.x, s * a.y, s * a.z);
}
template <typename T>
__device__ __forceinline__ T dot(const Vec3<T>& a, const Vec3<T>& b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}
template <typename T>
__device__ __forceinline__ Vec3<T> cross(const Vec3<T>& a, const Vec3<T>& b) {
  return mk3<T>(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
template <typename T>
__device__ __forceinline__ Vec3<T> tang(const Vec3<T>& n, const Vec3<T>& v) {
  return v - dot(n, v) * n;
}

// The model parameters a pair depends on (differentiable in the adjoint).
template <typename T>
struct PairParams {
  T kn, kt, gn, mu, delta;
};

// Outputs: force on i (F = Fc + Fl), torques on i and j, the parts of the
// force whose stresslet is r (x) F (contact and electro-chemical, Fc) and
// sym(r (x) F) (lubrication, Fl), the new stretch (i -> j orientation) and
// the new rolling stretch (App. B; orientation-free).
template <typename T>
struct PairModelOut {
  Vec3<T> F, Ti, Tj, Fc, Fl, xi, xr;
  int contact;
};

// r = x_j(image) - x_i, rr = |r|; Vi, Vj velocities relative to U_inf at each
// centre; Wi, Wj angular velocities relative to Omega_inf at each centre;
// du = u_j(image) - u_i (absolute); wi, wj absolute angular velocities; xo
// stretch (i -> j); ro rolling stretch (used when k_r > 0); rate the shear
// rate whose strain acts on the pair's lubrication (gdot, or in the wave of
// Eq. 17 the mean of the two centres' local rates).
template <typename T, bool EXT = false>
__device__ __forceinline__ PairModelOut<T> pair_model(const Geo& g, const InstGeo& I,
                                                      const PairParams<T>& q, Vec3<T> r, T rr,
                                                      double ai, double aj, Vec3<T> Vi, Vec3<T> Vj,
                                                      Vec3<T> Wi, Vec3<T> Wj, Vec3<T> du, Vec3<T> wi,
                                                      Vec3<T> wj, Vec3<T> xo, Vec3<T> ro, T rate) {
  (void)I;
  PairModelOut<T> o;
  const T zero = cst<T>(0.0);
  const T ir = 1.0 / rr;
  const Vec3<T> n = ir * r;
  const double S = ai + aj;
  const T d = rr - S;
  // ---- contact, Eq. 4-5
  o.Fc = mk3<T>(zero, zero, zero);
  Vec3<T> Tci = o.Fc, Tcj = o.Fc;
  o.xi = o.Fc;
  o.xr = o.Fc;
  o.contact = 0;
  if (val(d) < 0.0) {
    o.contact = 1;
    const T fn = q.kn * d + q.gn * dot(n, du);
    const Vec3<T> rel = du - cross(ai * wi + aj * wj, n);
    const Vec3<T> ut = tang(n, rel);
    Vec3<T> xs = tang(n, xo) + g.dt * ut;
    const T cap = q.mu * fabs(fn) / q.kt;
    const T xm = sqrt(dot(xs, xs));
    if (val(xm) > val(cap)) xs = (cap / xm) * xs;
    const Vec3<T> Ft = q.kt * xs;
    o.Fc = fn * n + Ft;
    const Vec3<T> nxf = cross(n, Ft);
    Tci = ai * nxf;
    Tcj = aj * nxf;
    o.xi = xs;
    // rolling resistance, App. B: the procedure of Eq. 5 on the rolling
    // velocity abar (n x w_i - n x w_j) with k_r; torques only
    if (EXT && g.k_r > 0.0) {
      const double abar = 2.0 * ai * aj / (ai + aj);
      Vec3<T> xr = tang(n, ro) + g.dt * (abar * cross(n, wi - wj));
      const T capr = q.mu * fabs(fn) / g.k_r;
      const T xrm = sqrt(dot(xr, xr));
      if (val(xrm) > val(capr)) xr = (capr / xrm) * xr;
      const Vec3<T> Tr = abar * cross(n, g.k_r * xr);
      Tci = Tci + Tr;
      Tcj = Tcj - Tr;
      o.xr = xr;
    }
  }
  // ---- electro-chemical forces, Eq. 6-7 (central; stresslet r (x) F like contact)
  bool lub_on = true;
  if (g.de > 0.0) {
    const double abar = 2.0 * ai * aj / (ai + aj);
    T m = zero;
    if (g.f_er > 0.0 && val(d) < 20.0 * g.lambda_d)
      m = m - (g.f_er * (abar / g.a0)) * (val(d) >= 0.0 ? exp(-d / g.lambda_d) : cst<T>(1.0));
    if (g.hamaker > 0.0 && val(d) < 4.0 * g.a0) {
      const double eps = g.vdw_eps * abar;
      const T dp = val(d) >= 0.0 ? d : zero;
      m = m + (g.hamaker * abar) / (12.0 * (dp * dp + eps * eps));
    }
    o.Fc = o.Fc + m * n;
    // lubrication only within its own cutoff: the listing predicate with the
    // lubrication range, in the same operations as the neighbour test
    const double rx = val(r.x), ry = val(r.y), rz = val(r.z);
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(rx, rx), __dmul_rn(ry, ry)), __dmul_rn(rz, rz));
    const double dl = g.mode == 1 ? __dmul_rn(val(q.delta), g.a0)
                                  : __dmul_rn(__dmul_rn(val(q.delta), __dadd_rn(ai, aj)), 0.5);
    const double sl = __dadd_rn(__dadd_rn(ai, aj), dl);
    lub_on = r2 < __dmul_rn(sl, sl);
  }
  // ---- lubrication, App. A, for the pairs within its range (every listed
  // pair unless electro-chemical forces widen the list)
  Vec3<T> Fl = mk3<T>(zero, zero, zero), Tli = Fl, Tlj = Fl;
  if (lub_on) {
    T ds = 2.0 * d / S;
    // the clamp's branch: overlapping pairs only (a pair exactly touching keeps
    // the gap's derivative, the branch its values share with d > 0)
    if (!(val(ds) >= 0.0)) ds = zero;
    const T dd = ds + g.eps;
    const T X = 1.0 / dd;
    const T Y = -log(dd);
    const double A = ai, B = aj, AB = A * B;
    const double iS = 1.0 / S, iS2 = iS * iS, iS3 = iS2 * iS;
    const T xa = X * (2.0 * AB * AB * iS3);
    const T ya = Y * ((4.0 / 15.0) * AB * (2.0 * A * A + AB + 2.0 * B * B) * iS3);
    const T ybi = -Y * ((2.0 / 15.0) * A * AB * (4.0 * A + B) * iS2);
    const T ybj = -Y * ((2.0 / 15.0) * AB * B * (A + 4.0 * B) * iS2);
    const T yci = Y * ((8.0 / 15.0) * A * A * AB * iS);
    const T ycj = Y * ((8.0 / 15.0) * AB * B * B * iS);
    const T ycx = Y * ((2.0 / 15.0) * AB * AB * iS);
    const T xg = X * (2.0 * AB * AB * iS2);
    const T yg = Y * ((1.0 / 15.0) * AB * (4.0 - 6.0 * AB * iS2));
    const T yhi = Y * (iS2 * ((2.0 / 15.0) * A * A * AB * (2.0 * A - B) + (1.0 / 15.0) * AB * AB * (7.0 * A + B)));
    const T yhj = Y * (iS2 * ((1.0 / 15.0) * AB * AB * (A + 7.0 * B) + (2.0 / 15.0) * AB * B * B * (2.0 * B - A)));
    const Vec3<T> dV = Vi - Vj;
    const T nV = dot(n, dV);
    const Vec3<T> fr = (xa * nV) * n + ya * tang(n, dV) + ybi * cross(n, Wi) + ybj * cross(n, Wj);
    // shear along x of rate `rate`: 2 E n = rate (n_y, n_x, 0), P = rate n_x n_y,
    // Q.n = 2 E n - 2 P n
    const Vec3<T> twoEn = mk3<T>(rate * n.y, rate * n.x, zero);
    const T P = rate * n.x * n.y;
    const Vec3<T> Qn = twoEn - (2.0 * P) * n;
    const Vec3<T> nperp = cross(n, twoEn);
    const Vec3<T> fe = (xg * P) * n + yg * Qn;
    Fl = g.k6 * (fe - fr);
    const Vec3<T> ndV = cross(n, dV);
    Tli = g.k6 * (ybi * ndV - (yci * tang(n, Wi) + ycx * tang(n, Wj)) + yhi * nperp);
    Tlj = g.k6 * (ybj * ndV - (ycx * tang(n, Wi) + ycj * tang(n, Wj)) + yhj * nperp);
    if (g.taper > 0.0) {
      const T dl = g.mode == 1 ? q.delta * g.a0 : q.delta * (0.5 * S);
      const T t = (dl - d) / (g.taper * dl);
      if (val(t) < 1.0) {
        const T s = val(t) > 0.0 ? t * t * (3.0 - 2.0 * t) : zero;
        Fl = s * Fl;
        Tli = s * Tli;
        Tlj = s * Tlj;
      }
    }
  }
  o.Fl = Fl;
  o.F = o.Fc + Fl;
  o.Ti = Tci + Tli;
  o.Tj = Tcj + Tlj;
  return o;
}
