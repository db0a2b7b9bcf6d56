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
//                  built from forward-mode derivative blocks of the shared
//                  pair model (dss_pair_model.cuh) contracted with the
//                  cotangents; the stretch adjoints are routed to the pair of
//                  the previous step they came from;
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
constexpr int kNin = 28;          // pair-model inputs differentiated (25 without rolling springs)
constexpr int kDualK = 5;         // derivative directions per forward-mode pass

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

template <int K>
__device__ __forceinline__ Dual<K> seed(double v, int idx, int base) {
  Dual<K> d = dual_const<K>(v);
  const int k = idx - base;
#pragma unroll
  for (int q = 0; q < K; ++q)
    if (q == k) d.d[q] = 1.0;
  return d;
}

// One forward-mode pass over inputs [base, base + K): writes the input
// adjoints of those inputs (the contraction of the outputs' derivatives with
// the cotangents).
template <int K>
__device__ __noinline__ void vjp_pass(const Geo& g, const InstGeo& I, const PairIn& in,
                                      const PairCot& c, int base, double* out) {
  using D = Dual<K>;
  const Vec3<D> r = mk3<D>(seed<K>(in.r[0], 0, base), seed<K>(in.r[1], 1, base), seed<K>(in.r[2], 2, base));
  const D yi = seed<K>(in.yi, 3, base), yj = seed<K>(in.yj, 4, base);
  const Vec3<D> ui = mk3<D>(seed<K>(in.ui[0], 5, base), seed<K>(in.ui[1], 6, base), seed<K>(in.ui[2], 7, base));
  const Vec3<D> uj = mk3<D>(seed<K>(in.uj[0], 8, base), seed<K>(in.uj[1], 9, base), seed<K>(in.uj[2], 10, base));
  const Vec3<D> wi = mk3<D>(seed<K>(in.wi[0], 11, base), seed<K>(in.wi[1], 12, base), seed<K>(in.wi[2], 13, base));
  const Vec3<D> wj = mk3<D>(seed<K>(in.wj[0], 14, base), seed<K>(in.wj[1], 15, base), seed<K>(in.wj[2], 16, base));
  const Vec3<D> xo = mk3<D>(seed<K>(in.xo[0], 17, base), seed<K>(in.xo[1], 18, base), seed<K>(in.xo[2], 19, base));
  const Vec3<D> ro = mk3<D>(seed<K>(in.ro[0], 25, base), seed<K>(in.ro[1], 26, base), seed<K>(in.ro[2], 27, base));
  PairParams<D> q;
  q.kn = seed<K>(g.kn, 20, base);
  q.kt = seed<K>(g.kt, 21, base);
  q.gn = seed<K>(I.gn, 22, base);
  q.mu = seed<K>(g.mu, 23, base);
  q.delta = seed<K>(g.delta, 24, base);
  const D rr = sqrt(dot(r, r));
  const double Om = -0.5 * I.gdot;
  Vec3<D> Vi = mk3<D>(ui.x - I.gdot * yi, ui.y, ui.z);
  Vec3<D> Vj = mk3<D>(uj.x - I.gdot * yj, uj.y, uj.z);
  Vec3<D> Wi = mk3<D>(wi.x, wi.y, wi.z - Om);
  Vec3<D> Wj = mk3<D>(wj.x, wj.y, wj.z - Om);
  D rate = cst<D>(I.gdot);
  if (g.wave) {
    // Eq. 17 at each centre: U sin(k y) in U_inf,x, (U k cos(k y))/2 in -Omega_inf,z,
    // the strain of the mean of the two local rates
    const D ci = cos(I.wave_k * yi), cj = cos(I.wave_k * yj);
    Vi.x = Vi.x - g.wave_amp * sin(I.wave_k * yi);
    Vj.x = Vj.x - g.wave_amp * sin(I.wave_k * yj);
    Wi.z = Wi.z + (0.5 * g.wave_amp * I.wave_k) * ci;
    Wj.z = Wj.z + (0.5 * g.wave_amp * I.wave_k) * cj;
    rate = rate + (0.5 * g.wave_amp * I.wave_k) * (ci + cj);
  }
  const Vec3<D> du = mk3<D>(uj.x + in.sy * I.gdot * I.L[1] - ui.x, uj.y - ui.y, uj.z - ui.z);
  const PairModelOut<D> o =
      pair_model<D, true>(g, I, q, r, rr, in.ai, in.aj, Vi, Vj, Wi, Wj, du, wi, wj, xo, ro, rate);
  D v = c.F[0] * o.F.x + c.F[1] * o.F.y + c.F[2] * o.F.z;
  v = v + c.Ti[0] * o.Ti.x + c.Ti[1] * o.Ti.y + c.Ti[2] * o.Ti.z;
  v = v + c.Tj[0] * o.Tj.x + c.Tj[1] * o.Tj.y + c.Tj[2] * o.Tj.z;
  v = v + c.xi[0] * o.xi.x + c.xi[1] * o.xi.y + c.xi[2] * o.xi.z;
  if (g.k_r > 0.0) v = v + c.xr[0] * o.xr.x + c.xr[1] * o.xr.y + c.xr[2] * o.xr.z;
  // Eq. 9: S = r (x) F^C + sym(r (x) F^L), weighted
  const D rv[3] = {r.x, r.y, r.z};
  const D fc[3] = {o.Fc.x, o.Fc.y, o.Fc.z};
  const D fl[3] = {o.Fl.x, o.Fl.y, o.Fl.z};
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const double wab = c.Ws[3 * a + b];
      if (wab != 0.0) v = v + wab * (rv[a] * fc[b] + 0.5 * (rv[a] * fl[b] + rv[b] * fl[a]));
    }
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (base + k < kNin) out[base + k] = v.d[k];
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

template <int K>
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
    const int nin = g.k_r > 0.0 ? kNin : 25;
    for (int base = 0; base < nin; base += K) vjp_pass<K>(g, I, in, cot, base, out);
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

__global__ void k_adj_theta(const double* __restrict__ part, int nblocks, double* __restrict__ thb) {
  const int c = threadIdx.x;
  if (c >= 5) return;
  double v = 0.0;
  for (int b = 0; b < nblocks; ++b) v += part[b * 5 + c];
  thb[c] += v;
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
  k_adj_pairs<kDualK><<<pb, kAdjThreads, 0, h->stream>>>(
      h->g, h->ig, t, h->a_by_id, P, A->Fb, A->Tb, xib_cur, xib_prev, xrb_cur, xrb_prev, Wn,
      1.0 / vol, A->pout, A->bw_n, A->bw_p, A->thb_part, h->status);
  k_adj_theta<<<1, 32, 0, h->stream>>>(A->thb_part, pb, A->thb);
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
