// Pair forces and their deterministic accumulation.
//
// k_pairs: one thread per listed pair (owner-sorted order).  Lubrication of
//   App. A (Eq. A2, A3 with the coefficients of Eq. A6, A7 and the
//   6 pi eta0 prefactor), stick-and-slide contact of Eq. 4-5 with the
//   tangential stretch carried from the previous step's sorted rows, and the
//   pair stresslet of Eq. 9, reduced per block in a fixed order.  The
//   per-pair records (force on the owner, torques on owner and partner) go
//   to memory; nothing is accumulated with atomics.
// k_gather: one thread per particle.  Sums its own records (its row, in
//   order) and the records where it is the partner (found by the mirrored
//   backward half-stencil, in increasing owner order: the transposed index),
//   adds Stokes drag (Eq. A1) and applies the corrector of Eq. 15d.
// k_finalize: bulk stress of Eq. 8 from the block partials, step counters.
#include "dss_internal.cuh"

namespace {
constexpr int kPairThreads = 256;
constexpr int kThreads = 128;

// Binary search of `target` in a sorted row; -1 when absent.
__device__ __forceinline__ int row_find(const int* row, int cnt, int target) {
  int lo = 0, hi = cnt - 1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    int v = row[mid];
    if (v == target) return mid;
    if (v < target) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

// Tangential stretch of pair (idi, idj) at the last committed step, in the
// lo -> hi orientation; zero when the pair was not in contact then.
__device__ __forceinline__ void history_lookup(const Geo& g, const ListBuf& H, int idi, int idj,
                                               double xo[3]) {
  xo[0] = xo[1] = xo[2] = 0.0;
  const int oi = H.slot_of_id[idi], oj = H.slot_of_id[idj];
  int64_t pold = -1;
  int k = row_find(H.list + (int64_t)oi * g.M, H.count[oi], oj);
  if (k >= 0) {
    pold = (int64_t)H.start[oi] + k;
  } else {
    k = row_find(H.list + (int64_t)oj * g.M, H.count[oj], oi);
    if (k >= 0) pold = (int64_t)H.start[oj] + k;
  }
  if (pold >= 0 && H.cflag[pold]) {
    xo[0] = H.xi[pold];
    xo[1] = H.xi[g.pcap + pold];
    xo[2] = H.xi[2 * g.pcap + pold];
  }
}

struct V3 {
  double x, y, z;
};
__device__ __forceinline__ V3 v3(double a, double b, double c) { return V3{a, b, c}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ V3 operator*(double s, V3 a) { return v3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
  return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ V3 tang(V3 n, V3 v) { return v - dot(n, v) * n; }

// FP64 pair physics.  r = x_j(image) - x_i, n = r/|r|, d = |r| - (a_i+a_j).
// Vi, Vj: velocities relative to U_inf at each centre; Wi, Wj: relative to
// Omega_inf.  du: u_j(image) - u_i (absolute).  xo: stretch in i->j
// orientation.  Outputs: force on i, torques on i and j, new stretch.
struct PairOut {
  V3 F, Ti, Tj, Fc, Fl, xi;
  int contact;
};

__device__ __forceinline__ PairOut pair_fp64(const Geo& g, V3 r, double rr, double ai, double aj,
                                             V3 Vi, V3 Vj, V3 Wi, V3 Wj, V3 du, V3 wi, V3 wj,
                                             const double xo[3]) {
  PairOut o;
  const double ir = 1.0 / rr;
  const V3 n = ir * r;
  const double S = ai + aj;
  const double d = rr - S;
  // ---- contact, Eq. 4-5
  o.Fc = v3(0, 0, 0);
  V3 Tci = v3(0, 0, 0), Tcj = v3(0, 0, 0);
  o.xi = v3(0, 0, 0);
  o.contact = 0;
  if (d < 0.0) {
    o.contact = 1;
    const double fn = g.kn * d + g.gn * dot(n, du);
    const V3 rel = du - cross(ai * wi + aj * wj, n);
    const V3 ut = tang(n, rel);
    V3 xs = tang(n, v3(xo[0], xo[1], xo[2])) + g.dt * ut;
    const double cap = g.mu * fabs(fn) / g.kt;
    const double xm = sqrt(dot(xs, xs));
    if (xm > cap) xs = (cap / xm) * xs;
    const V3 Ft = g.kt * xs;
    o.Fc = fn * n + Ft;
    const V3 nxf = cross(n, Ft);
    Tci = ai * nxf;
    Tcj = aj * nxf;
    o.xi = xs;
  }
  // ---- lubrication, App. A
  double ds = 2.0 * d / S;
  ds = ds > 0.0 ? ds : 0.0;
  const double dd = ds + g.eps;
  const double X = 1.0 / dd;
  const double Y = -log(dd);
  const double A = ai, B = aj, AB = A * B;
  const double iS = 1.0 / S, iS2 = iS * iS, iS3 = iS2 * iS;
  const double xa = X * 2.0 * AB * AB * iS3;
  const double ya = Y * (4.0 / 15.0) * AB * (2.0 * A * A + AB + 2.0 * B * B) * iS3;
  const double ybi = -Y * (2.0 / 15.0) * A * AB * (4.0 * A + B) * iS2;
  const double ybj = -Y * (2.0 / 15.0) * AB * B * (A + 4.0 * B) * iS2;
  const double yci = Y * (8.0 / 15.0) * A * A * AB * iS;
  const double ycj = Y * (8.0 / 15.0) * AB * B * B * iS;
  const double ycx = Y * (2.0 / 15.0) * AB * AB * iS;
  const double xg = X * 2.0 * AB * AB * iS2;
  const double yg = Y * (1.0 / 15.0) * AB * (4.0 - 6.0 * AB * iS2);
  const double yhi = Y * iS2 * ((2.0 / 15.0) * A * A * AB * (2.0 * A - B) + (1.0 / 15.0) * AB * AB * (7.0 * A + B));
  const double yhj = Y * iS2 * ((1.0 / 15.0) * AB * AB * (A + 7.0 * B) + (2.0 / 15.0) * AB * B * B * (2.0 * B - A));
  const V3 dV = Vi - Vj;
  const double nV = dot(n, dV);
  const V3 fr = (xa * nV) * n + ya * tang(n, dV) + ybi * cross(n, Wi) + ybj * cross(n, Wj);
  // simple shear: 2 E n = gdot (n_y, n_x, 0), P = gdot n_x n_y, Q.n = 2 E n - 2 P n
  const V3 twoEn = v3(g.gdot * n.y, g.gdot * n.x, 0.0);
  const double P = g.gdot * n.x * n.y;
  const V3 Qn = twoEn - (2.0 * P) * n;
  const V3 nperp = cross(n, twoEn);
  const V3 fe = (xg * P) * n + yg * Qn;
  const V3 Fl = g.k6 * (fe - fr);
  const V3 ndV = cross(n, dV);
  const V3 Tli = g.k6 * (ybi * ndV - (yci * tang(n, Wi) + ycx * tang(n, Wj)) + yhi * nperp);
  const V3 Tlj = g.k6 * (ybj * ndV - (ycx * tang(n, Wi) + ycj * tang(n, Wj)) + yhj * nperp);
  o.Fl = Fl;
  o.F = o.Fc + Fl;
  o.Ti = Tci + Tli;
  o.Tj = Tcj + Tlj;
  return o;
}

__global__ void __launch_bounds__(kPairThreads)
k_pairs(Geo g, StateBuf s, ListBuf W, ListBuf H, double* __restrict__ rec,
        double* __restrict__ spart, DevStatus* st, int adv) {
  if (dev_err(st)) return;
  const int n = g.n;
  const int P = W.start[n];
  if (P > g.pcap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st->w[ST_NPAIRS] = P;
      set_err(st, DSS_ERR_CAPACITY);
    }
    return;
  }
  const double off = le_offset(g, dev_nstep(st) + adv);
  const double Om = -0.5 * g.gdot;
  double Sx[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  int ncont = 0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (W.start[mid] <= p) lo = mid; else hi = mid;
    }
    const int i = lo;
    const int j = W.list[(int64_t)i * g.M + (p - W.start[i])];
    const double xi = s.x[i], yi = s.x[n + i], zi = s.x[2 * n + i];
    const double xj = s.x[j], yj = s.x[n + j], zj = s.x[2 * n + j];
    double dx, dy, dz;
    int sy;
    min_image(g, off, xi, yi, zi, xj, yj, zj, dx, dy, dz, sy);
    const V3 r = v3(dx, dy, dz);
    const double ai = s.a[i], aj = s.a[j];
    const V3 ui = v3(s.u[i], s.u[n + i], s.u[2 * n + i]);
    const V3 uj = v3(s.u[j], s.u[n + j], s.u[2 * n + j]);
    const V3 wi = v3(s.w[i], s.w[n + i], s.w[2 * n + i]);
    const V3 wj = v3(s.w[j], s.w[n + j], s.w[2 * n + j]);
    const int idi = s.id[i], idj = s.id[j];
    const double sgn = idi < idj ? 1.0 : -1.0;
    double xo[3] = {0.0, 0.0, 0.0};
    // the gap decides contact; look the history up only for contacts
    const double rr = sqrt(dot(r, r));
    if (rr - (ai + aj) < 0.0) {
      history_lookup(g, H, idi, idj, xo);
      xo[0] *= sgn; xo[1] *= sgn; xo[2] *= sgn;
    }
    const V3 Vi = v3(ui.x - g.gdot * yi, ui.y, ui.z);
    const V3 Vj = v3(uj.x - g.gdot * yj, uj.y, uj.z);
    const V3 Wi = v3(wi.x, wi.y, wi.z - Om);
    const V3 Wj = v3(wj.x, wj.y, wj.z - Om);
    const V3 du = v3(uj.x + sy * g.gdot * g.L[1] - ui.x, uj.y - ui.y, uj.z - ui.z);
    const PairOut o = pair_fp64(g, r, rr, ai, aj, Vi, Vj, Wi, Wj, du, wi, wj, xo);
    rec[p] = o.F.x;
    rec[g.pcap + p] = o.F.y;
    rec[2 * g.pcap + p] = o.F.z;
    rec[3 * g.pcap + p] = o.Ti.x;
    rec[4 * g.pcap + p] = o.Ti.y;
    rec[5 * g.pcap + p] = o.Ti.z;
    rec[6 * g.pcap + p] = o.Tj.x;
    rec[7 * g.pcap + p] = o.Tj.y;
    rec[8 * g.pcap + p] = o.Tj.z;
    W.xi[p] = sgn * o.xi.x;
    W.xi[g.pcap + p] = sgn * o.xi.y;
    W.xi[2 * g.pcap + p] = sgn * o.xi.z;
    W.cflag[p] = (unsigned char)o.contact;
    ncont += o.contact;
    // Eq. 9: S^C = r (x) F^C, S^L = sym(r (x) F^L), F on the owner
    const double rv[3] = {r.x, r.y, r.z};
    const double fc[3] = {o.Fc.x, o.Fc.y, o.Fc.z};
    const double fl[3] = {o.Fl.x, o.Fl.y, o.Fl.z};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) Sx[3 * a + b] += rv[a] * fc[b] + 0.5 * (rv[a] * fl[b] + rv[b] * fl[a]);
  }
  // deterministic block reduction of the stresslet (fixed tree)
  __shared__ double red[kPairThreads / 32][9];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    double v = Sx[q];
    for (int dlt = 16; dlt > 0; dlt >>= 1) v += __shfl_down_sync(0xffffffffu, v, dlt);
    if (lane == 0) red[wid][q] = v;
  }
  int c = ncont;
  for (int dlt = 16; dlt > 0; dlt >>= 1) c += __shfl_down_sync(0xffffffffu, c, dlt);
  if (lane == 0 && c) atomicAdd(&st->w[ST_NCONT], c);
  __syncthreads();
  if (threadIdx.x < 9) {
    double v = 0.0;
    for (int w = 0; w < kPairThreads / 32; ++w) v += red[w][threadIdx.x];
    spart[blockIdx.x * 9 + threadIdx.x] = v;
  }
}

__global__ void __launch_bounds__(kThreads)
k_gather(Geo g, StateBuf s, ListBuf W, const float4* __restrict__ posf,
         const int* __restrict__ cellid, const int* __restrict__ cell_start,
         const double* __restrict__ rec, double* __restrict__ Fout, double* __restrict__ Tout,
         DevStatus* st, int adv, int mode) {
  if (dev_err(st)) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = g.n;
  if (j >= n) return;
  const int64_t pc = g.pcap;
  V3 F = v3(0, 0, 0), T = v3(0, 0, 0);
  // own rows: the particle is the owner
  const int p0 = W.start[j], p1 = W.start[j + 1];
  for (int p = p0; p < p1; ++p) {
    F = F + v3(rec[p], rec[pc + p], rec[2 * pc + p]);
    T = T + v3(rec[3 * pc + p], rec[4 * pc + p], rec[5 * pc + p]);
  }
  // transposed records: owners found by the backward half-stencil
  const double off = le_offset(g, dev_nstep(st) + adv);
  const int fsh = le_shift_cells(g, off);
  const int c = cellid[j];
  const int cx = c % g.nc[0], cy = (c / g.nc[0]) % g.nc[1], cz = c / (g.nc[0] * g.nc[1]);
  StencilCell sc[17];
  const int ns = backward_cells(g, cx, cy, cz, fsh, sc);
  const float4 pj = posf[j];
  const double xj = s.x[j], yj = s.x[n + j], zj = s.x[2 * n + j], aj = s.a[j];
  for (int q = 0; q < ns; ++q) {
    const StencilCell cur = sc[q];
    const int ob = cell_start[cur.cell];
    const int oe = cur.le == 2 ? j : cell_start[cur.cell + 1];
    // separation seen from the owner: partner cell displaced by -(ox,oy,oz)
    const float cxo = (float)((-cur.ox) * g.cs[0] + (cur.le == 1 ? off : 0.0));
    const float cyo = (float)((-cur.oy) * g.cs[1]);
    const float czo = (float)((-cur.oz) * g.cs[2]);
    for (int o = ob; o < oe; ++o) {
      const float4 po = posf[o];
      const float sf = po.w + pj.w + pair_delta_f(g, po.w, pj.w);
      int dec = prefilter(g, po, pj, cxo, cyo, czo, sf);
      if (dec < 0)
        dec = exact_is_pair(g, off, s.x[o], s.x[n + o], s.x[2 * n + o], s.a[o], xj, yj, zj, aj) ? 1 : 0;
      if (!dec) continue;
      const int k = row_find(W.list + (int64_t)o * g.M, W.count[o], j);
      if (k < 0) {
        set_err(st, DSS_ERR_INTERNAL);
        continue;
      }
      const int64_t p = (int64_t)W.start[o] + k;
      F = F - v3(rec[p], rec[pc + p], rec[2 * pc + p]);
      T = T + v3(rec[6 * pc + p], rec[7 * pc + p], rec[8 * pc + p]);
    }
  }
  // Stokes drag, Eq. A1 (no Faxen term in simple shear)
  const double a = aj;
  const V3 u = v3(s.u[j], s.u[n + j], s.u[2 * n + j]);
  const V3 w = v3(s.w[j], s.w[n + j], s.w[2 * n + j]);
  F = F + (-g.k6 * a) * v3(u.x - g.gdot * yj, u.y, u.z);
  T = T + (-g.k8 * a * a * a) * v3(w.x, w.y, w.z + 0.5 * g.gdot);
  if (!(isfinite(F.x) && isfinite(F.y) && isfinite(F.z) && isfinite(T.x) && isfinite(T.y) &&
        isfinite(T.z)))
    set_err(st, DSS_ERR_NONFINITE);
  const int id = s.id[j];
  if (mode == G_EVAL) {
    if (Fout) { Fout[id] = F.x; Fout[n + id] = F.y; Fout[2 * n + id] = F.z; }
    if (Tout) { Tout[id] = T.x; Tout[n + id] = T.y; Tout[2 * n + id] = T.z; }
    return;
  }
  // accelerations: m = 4/3 pi rho a^3, I = 2/5 m a^2
  const double m = 4.0 / 3.0 * DSS_PI * g.rho * a * a * a;
  const double I = 0.4 * m * a * a;
  const V3 al = v3(F.x / m, F.y / m, F.z / m);
  const V3 aw = v3(T.x / I, T.y / I, T.z / I);
  s.al[j] = al.x; s.al[n + j] = al.y; s.al[2 * n + j] = al.z;
  s.aw[j] = aw.x; s.aw[n + j] = aw.y; s.aw[2 * n + j] = aw.z;
  if (mode == G_STEP) {
    // Eq. 15d from u^{n+1/2}: u^{n+1} = u^{n+1/2} + dt/2 alpha^{n+1}
    const double hdt = __dmul_rn(0.5, g.dt);
    s.u[j] = __dadd_rn(u.x, __dmul_rn(hdt, al.x));
    s.u[n + j] = __dadd_rn(u.y, __dmul_rn(hdt, al.y));
    s.u[2 * n + j] = __dadd_rn(u.z, __dmul_rn(hdt, al.z));
    s.w[j] = __dadd_rn(w.x, __dmul_rn(hdt, aw.x));
    s.w[n + j] = __dadd_rn(w.y, __dmul_rn(hdt, aw.y));
    s.w[2 * n + j] = __dadd_rn(w.z, __dmul_rn(hdt, aw.z));
  }
}

// Bulk stress (Eq. 8) and counters.  One block, fixed reduction order.
__global__ void k_finalize(Geo g, const double* __restrict__ spart, int nblocks, double* sigma,
                           DevStatus* st, const int* __restrict__ start, int step) {
  __shared__ double red[256][9];
  double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
    for (int q = 0; q < 9; ++q) v[q] += spart[b * 9 + q];
#pragma unroll
  for (int q = 0; q < 9; ++q) red[threadIdx.x][q] = v[q];
  __syncthreads();
  for (int s2 = blockDim.x / 2; s2 > 0; s2 >>= 1) {
    if (threadIdx.x < s2)
#pragma unroll
      for (int q = 0; q < 9; ++q) red[threadIdx.x][q] += red[threadIdx.x + s2][q];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int err = dev_err(st);
    if (!err) {
      // E_inf: only xy and yx are non-zero (gdot/2)
      const double Exy = 0.5 * g.gdot;
      const double V = g.L[0] * g.L[1] * g.L[2];
      const double ein = 20.0 / 3.0 * DSS_PI * g.eta0 * g.sumA3;
      for (int q = 0; q < 9; ++q) {
        const double E = (q == 1 || q == 3) ? Exy : 0.0;
        sigma[q] = 2.0 * g.eta0 * E + (ein * E + red[0][q]) / V;
      }
      st->w[ST_NPAIRS] = start[g.n];
      if (step) {
        st->w[ST_STEPS] += 1;
        int64_t ns = dev_nstep(st) + 1;
        st->w[ST_NSTEP_LO] = (int)(uint32_t)(ns & 0xffffffffll);
        st->w[ST_NSTEP_HI] = (int)(ns >> 32);
      }
    }
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
    const int j = W.list[(int64_t)lo * g.M + (p - W.start[lo])];
    const int a = W.id_of_slot[lo], b = W.id_of_slot[j];
    out[2 * (int64_t)p] = a < b ? a : b;
    out[2 * (int64_t)p + 1] = a < b ? b : a;
  }
}
}  // namespace

int pair_grid_blocks(const dss_handle* h) {
  int64_t need = (h->pcap + kPairThreads - 1) / kPairThreads;
  int64_t cap = 152 * 8;
  return (int)(need < cap ? (need > 0 ? need : 1) : cap);
}

void launch_forces(dss_handle* h, int stbuf, int work_list, int hist_list, int adv, int mode,
                   double* F_out, double* T_out) {
  const int n = (int)h->n;
  const int pb = pair_grid_blocks(h);
  prof_mark(h, 7);
  k_pairs<<<pb, kPairThreads, 0, h->stream>>>(h->g, h->st[stbuf], h->lb[work_list], h->lb[hist_list],
                                              h->rec, h->spart, h->status, adv);
  prof_mark(h, 8);
  k_gather<<<(n + kThreads - 1) / kThreads, kThreads, 0, h->stream>>>(
      h->g, h->st[stbuf], h->lb[work_list], h->posf, h->cellid, h->cell_start, h->rec, F_out, T_out,
      h->status, adv, mode);
  prof_mark(h, 9);
  k_finalize<<<1, 256, 0, h->stream>>>(h->g, h->spart, pb, h->sigma, h->status,
                                       h->lb[work_list].start, mode == G_STEP ? 1 : 0);
  prof_mark(h, 10);
}

void launch_pairs_out(dss_handle* h, int list, long long* out) {
  k_pairs_out<<<pair_grid_blocks(h), kPairThreads, 0, h->stream>>>(h->g, h->lb[list], out);
}
