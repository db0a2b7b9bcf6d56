// Counting sort of the particles into cells (Sec. II A; the paper follows
// Hoetzlein's counting sort), redone every step with no Verlet skin:
//   1. predictor + Lees-Edwards wrap (Eq. 15a-b, 16) fused with the cell key
//      and a warp-aggregated histogram (one atomic per distinct key per warp);
//   2. exclusive scan of the histogram (single-pass decoupled look-back);
//   3. scatter to the cell's slot range;
//   4. deterministic in-cell order (by id) and the gather of the state into
//      the new sorted order; the predicted position and velocity are stored by
//      step 1 (SoA, source order) and gathered, not recomputed.
#include "dss_internal.cuh"

namespace {

constexpr int kThreads = 256;

// Predictor of Eq. 15a-b and the wrap of Eq. 16 for one particle; computed
// once per step and stored for the gather.  In FP64 mode each product and
// sum is rounded separately (the trajectory then differs from a plain FP64
// evaluation only through the order of the force sums); in mixed precision
// as fused multiply-adds (GB300's narrow FP64 pipe bounds this kernel).
// Returns the y crossing (-1 out through the top, +1 bottom).
// Comparisons for the wrap on the IEEE bit patterns (integer instructions
// instead of GB300's narrow FP64 pipe).  For L > 0 and any finite v the
// signed 64-bit order of the patterns is the order of the values on the
// non-negative side, and every negative v sorts below; -0.0 is not below 0.
__device__ __forceinline__ bool ge_pos(double v, double L) {
  return __double_as_longlong(v) >= __double_as_longlong(L);
}
__device__ __forceinline__ bool lt_zero(double v) {
  const long long b = __double_as_longlong(v);
  return b < 0 && b != (long long)0x8000000000000000ull;
}

struct Pred {
  double x, y, z, ux, uy, uz;
  int cross;
};

// Lees-Edwards wrap of Eq. 16 and the periodic wraps along x and z, for a
// particle that left the box (out of line: see f32_rn_slow).
__device__ __noinline__ Pred wrap_out(const Geo& g, const InstGeo& I, const DevStatus* st, int adv, Pred r) {
  double x = r.x, y = r.y, z = r.z, ux = r.ux;
  // leaving through y >= L_y re-enters at the bottom shifted by -off along
  // x with u_x - gdot L_y, and vice versa
  const double Ly = I.L[1];
  if (ge_pos(y, Ly)) {
    y = __dsub_rn(y, Ly);
    x = __dsub_rn(x, le_offset(g, I, dev_nstep(st) + adv));
    r.cross = -1;
  } else if (lt_zero(y)) {
    y = __dadd_rn(y, Ly);
    x = __dadd_rn(x, le_offset(g, I, dev_nstep(st) + adv));
    r.cross = 1;
    if (ge_pos(y, Ly)) y = 0.0;
  }
  // x back into [0, L_x): two conditional shifts give the same bits as
  // fmod followed by the two corrections, for |x| < 2 L_x
  const double Lx = I.L[0];
  if (lt_zero(x)) x = __dadd_rn(x, Lx); else if (ge_pos(x, Lx)) x = __dsub_rn(x, Lx);
  if (lt_zero(x)) x = __dadd_rn(x, Lx); else if (ge_pos(x, Lx)) x = __dsub_rn(x, Lx);
  if (ge_pos(z, I.L[2])) {
    z = __dsub_rn(z, I.L[2]);
  } else if (lt_zero(z)) {
    z = __dadd_rn(z, I.L[2]);
    if (ge_pos(z, I.L[2])) z = 0.0;
  }
  if (r.cross != 0)
    ux = __dadd_rn(ux, __dmul_rn(__dmul_rn((double)r.cross, I.gdot), Ly));
  r.x = x; r.y = y; r.z = z; r.ux = ux;
  return r;
}

__device__ __forceinline__ Pred predict_one(const Geo& g, const InstGeo& I, const DevStatus* st,
                                            int adv, const StateBuf& s, int i, bool predict) {
  const int n = g.n;
  Pred r;
  double x = s.x[i], y = s.x[n + i], z = s.x[2 * n + i];
  double ux = s.u[i], uy = s.u[n + i], uz = s.u[2 * n + i];
  r.cross = 0;
  if (predict) {
    const double dt = g.dt;
    const double hdt2 = g.hdt2;
    const double hdt = g.hdt;
    double ax = s.al[i], ay = s.al[n + i], az = s.al[2 * n + i];
    if (g.precision == DSS_FP64) {
      // FP64 mode: every product and sum rounded on its own, in the order
      // x + dt u + (dt/2 dt) alpha of Eq. 15a (no contraction)
      x = __dadd_rn(__dadd_rn(x, __dmul_rn(dt, ux)), __dmul_rn(hdt2, ax));
      y = __dadd_rn(__dadd_rn(y, __dmul_rn(dt, uy)), __dmul_rn(hdt2, ay));
      z = __dadd_rn(__dadd_rn(z, __dmul_rn(dt, uz)), __dmul_rn(hdt2, az));
      ux = __dadd_rn(ux, __dmul_rn(hdt, ax));
      uy = __dadd_rn(uy, __dmul_rn(hdt, ay));
      uz = __dadd_rn(uz, __dmul_rn(hdt, az));
    } else {
      x = __fma_rn(hdt2, ax, __fma_rn(dt, ux, x));
      y = __fma_rn(hdt2, ay, __fma_rn(dt, uy, y));
      z = __fma_rn(hdt2, az, __fma_rn(dt, uz, z));
      ux = __fma_rn(hdt, ax, ux);
      uy = __fma_rn(hdt, ay, uy);
      uz = __fma_rn(hdt, az, uz);
    }
  }
  r.x = x; r.y = y; r.z = z;
  r.ux = ux; r.uy = uy; r.uz = uz;
  // inside the box (nearly every particle): nothing to wrap
  if (predict && (ge_pos(y, I.L[1]) || lt_zero(y) || ge_pos(x, I.L[0]) || lt_zero(x) || ge_pos(z, I.L[2]) ||
                  lt_zero(z)))
    r = wrap_out(g, I, st, adv, r);
  return r;
}

// Cell coordinate floor(x / cs) along one axis, clamped to the grid (the
// FP64 product's floor, mostly decided in FP32: floor_mul).
__device__ __forceinline__ int cell_coord_fast(double v, double inv, float invf, int nc) {
  const int k = floor_mul(v, inv, invf);
  return k < 0 ? 0 : (k >= nc ? nc - 1 : k);
}

// Bin of a particle: its instance's bins, its size class's layer, its cell.
__device__ __forceinline__ int cell_key(const InstGeo& I, int cls, double x, double y, double z) {
  int cx = cell_coord_fast(x, I.inv_cs[0], I.inv_csf[0], I.nc[0]);
  int cy = cell_coord_fast(y, I.inv_cs[1], I.inv_csf[1], I.nc[1]);
  int cz = cell_coord_fast(z, I.inv_cs[2], I.inv_csf[2], I.nc[2]);
  return I.cell_base + cls * I.ncell_layer + (cz * I.nc[1] + cy) * I.nc[0] + cx;
}

// 1. key + warp-aggregated histogram
__global__ void __launch_bounds__(kThreads)
k_key_hist(Geo g, const InstGeo* __restrict__ ig, StepGeo* __restrict__ sg, StateBuf s,
           int* __restrict__ key, int* __restrict__ offs, int* __restrict__ cell_count,
           DevStatus* st, bool predict, unsigned long long* scan_status, int* scan_ticket,
           int scan_tiles, double* __restrict__ pred, signed char* __restrict__ xc) {
  if (dev_err(st)) return;
  // reset the look-back state of both scans of this operation (spread over
  // the grid), the counters, and set every instance's Lees-Edwards geometry
  // for its time
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 2 * scan_tiles; t += gridDim.x * blockDim.x)
    scan_status[t] = 0ull;
  if (blockIdx.x == 0) {
    if (threadIdx.x < 2) scan_ticket[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
      st->w[ST_MAXROW] = 0;
      st->w[ST_BAND] = 0;
      st->w[ST_NCONT] = 0;
    }
    for (int k = threadIdx.x; k < g.K; k += blockDim.x) {
      const InstGeo& I = ig[k];
      const double off = le_offset(g, I, dev_nstep(st) + (predict ? 1 : 0));
      const int fsh = le_shift_cells(I, off);
      const double offr = off - fsh * I.cs[0];
      StepGeo q;
      q.off = off;
      q.fsh = fsh;
      q.offr_hi = (float)offr;
      q.offr_lo = (float)(offr - (double)q.offr_hi);
      sg[k] = q;
    }
  }
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  const InstGeo& I = ig[s.inst[i]];
  Pred p = predict_one(g, I, st, predict ? 1 : 0, s, i, predict);
  if (predict) {
    const int n = g.n;
    pred[i] = p.x;
    pred[n + i] = p.y;
    pred[2 * n + i] = p.z;
    pred[3 * n + i] = p.ux;
    pred[4 * n + i] = p.uy;
    pred[5 * n + i] = p.uz;
    xc[i] = (signed char)p.cross;
  }
  int k = cell_key(I, s.cls[i], p.x, p.y, p.z);
  unsigned act = __activemask();
  unsigned peers = __match_any_sync(act, k);
  int lane = threadIdx.x & 31;
  int leader = __ffs(peers) - 1;
  int rank = __popc(peers & ((1u << lane) - 1u));
  int base = 0;
  if (lane == leader) base = atomicAdd(&cell_count[k], __popc(peers));
  base = __shfl_sync(peers, base, leader);
  key[i] = k;
  offs[i] = base + rank;
}

// 3. scatter to the cell slot range (order inside a cell not yet fixed)
__global__ void __launch_bounds__(kThreads)
k_scatter(int n, const int* __restrict__ key, const int* __restrict__ offs,
          const int* __restrict__ cell_start, int* __restrict__ tmp, const DevStatus* st) {
  if (dev_err(st)) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  tmp[cell_start[key[i]] + offs[i]] = i;
}

// 4. order inside each cell by id (so the sorted order, and with it every
// summation order downstream, is a function of positions and ids alone) and
// state gather (WAVE: the wave of Eq. 17 is on, compiled out otherwise)
template <bool WAVE>
__global__ void __launch_bounds__(kThreads)
k_rank_gather(Geo g, const InstGeo* __restrict__ ig, const StepGeo* __restrict__ sgk, StateBuf src,
              StateBuf dst, const int* __restrict__ key, const int* __restrict__ cell_start,
              const int* __restrict__ tmp, int* __restrict__ perm, int* __restrict__ cellid,
              float4* __restrict__ posf, DevStatus* st, bool predict,
              const double* __restrict__ pred, const signed char* __restrict__ xc) {
  if (dev_err(st)) return;
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = g.n;
  if (s >= n) return;
  int o = tmp[s];
  int k = key[o];
  int c0 = cell_start[k], c1 = cell_start[k + 1];
  const int id = src.id[o];
  int rank = 0;
  for (int q = c0; q < c1; ++q) rank += (src.id[tmp[q]] < id);
  int f = c0 + rank;
  perm[f] = o;
  cellid[f] = k;
  const int inst = src.inst[o];
  const InstGeo& I = ig[inst];
  Pred p;
  if (predict) {
    p.x = pred[o]; p.y = pred[n + o]; p.z = pred[2 * n + o];
    p.ux = pred[3 * n + o]; p.uy = pred[4 * n + o]; p.uz = pred[5 * n + o];
  } else {
    p.x = src.x[o]; p.y = src.x[n + o]; p.z = src.x[2 * n + o];
    p.ux = src.u[o]; p.uy = src.u[n + o]; p.uz = src.u[2 * n + o];
  }
  dst.x[f] = p.x; dst.x[n + f] = p.y; dst.x[2 * n + f] = p.z;
  dst.u[f] = p.ux; dst.u[n + f] = p.uy; dst.u[2 * n + f] = p.uz;
  double wv3[3];
  if (predict) {
    const double hdt = g.hdt;
    if (g.precision == DSS_FP64)
      for (int c = 0; c < 3; ++c)
        wv3[c] = __dadd_rn(src.w[c * n + o], __dmul_rn(hdt, src.aw[c * n + o]));
    else
      for (int c = 0; c < 3; ++c)
        wv3[c] = __fma_rn(hdt, src.aw[c * n + o], src.w[c * n + o]);
  } else {
    for (int c = 0; c < 3; ++c) {
      wv3[c] = src.w[c * n + o];
      dst.al[c * n + f] = src.al[c * n + o];
      dst.aw[c * n + f] = src.aw[c * n + o];
    }
  }
  for (int c = 0; c < 3; ++c) dst.w[c * n + f] = wv3[c];
  const double w0 = wv3[0], w1 = wv3[1], w2 = wv3[2];
  const double a = src.a[o];
  dst.a[f] = a;
  dst.id[f] = id;
  dst.inst[f] = inst;
  dst.cls[f] = src.cls[o];
  // image count: leaving through the top is one image up
  dst.iy[f] = src.iy[o] - (predict ? (int)xc[o] : 0);
  if (WAVE) {
    // the wave of Eq. 17 at the centre, once per evaluation: its part of
    // U_inf,x and of the local rate dU_inf,x/dy
    double sn, cs;
    sincos(I.wave_k * p.y, &sn, &cs);
    const double ws = g.wave_amp * sn, wc = g.wave_amp * I.wave_k * cs;
    dst.wv[f] = make_double2(ws, wc);
    if (g.precision == DSS_MIXED) {
      dst.vf[f] = make_float4(f32_rn(p.ux - I.gdot * p.y - ws), f32_rn(p.uy), f32_rn(p.uz), f32_rn(wc));
      dst.wf[f] = make_float4(f32_rn(w0), f32_rn(w1), f32_rn(w2 + 0.5 * (I.gdot + wc)), f32_rn(ws));
    }
  } else if (g.precision == DSS_MIXED) {
    // FP32 copies relative to the ambient flow for the FP32 pair arithmetic:
    // u - U_inf(x) and w - Omega_inf are O(gdot a), free of O(gdot L) terms
    dst.vf[f] = make_float4(f32_rn(p.ux - I.gdot * p.y), f32_rn(p.uy), f32_rn(p.uz), 0.f);
    dst.wf[f] = make_float4(f32_rn(w0), f32_rn(w1), f32_rn(w2 + 0.5 * I.gdot), 0.f);
  }
  // cell-local position (FP32 for the enumeration prefilter; in mixed
  // precision also the low words, for double-float pair geometry)
  const int kl = (k - I.cell_base) % I.ncell_layer;
  int cx = kl % I.nc[0];
  int cy = (kl / I.nc[0]) % I.nc[1];
  int cz = kl / (I.nc[0] * I.nc[1]);
  const double lx = __fma_rn(-f64_of_nonneg(cx), I.cs[0], p.x),
               ly = __fma_rn(-f64_of_nonneg(cy), I.cs[1], p.y),
               lz = __fma_rn(-f64_of_nonneg(cz), I.cs[2], p.z);
  // the FP32 words and (mixed precision) the low words of the double-float
  // pair geometry
  float4 pf, pl;
  f32_split(lx, pf.x, pl.x);
  f32_split(ly, pf.y, pl.y);
  f32_split(lz, pf.z, pl.z);
  f32_split(a, pf.w, pl.w);
  posf[f] = pf;
  if (g.precision == DSS_MIXED) {
    dst.posl[f] = pl;
    dst.cellc[f] = cx | (cy << 10) | (cz << 20);
  }
  (void)sgk;
}

}  // namespace

// Single-pass exclusive scan with decoupled look-back.  Tiles are taken in
// launch order through an atomic ticket, so every predecessor a tile waits
// on is already running; each wait is bounded and reports DSS_ERR_TIMEOUT.
namespace {
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__host__ __device__ constexpr int scan_pad(int q) { return q + (q >> 5); }   // no bank conflicts

// A tile is loaded and stored coalesced through shared memory; each thread
// scans 8 consecutive items of it.  The input is cleared as soon as it is
// read when zero_in is set (the histogram of the next operation).
__global__ void __launch_bounds__(kScanThreads)
k_scan(const int* __restrict__ in, int* __restrict__ out, int count,
       unsigned long long* status, int* ticket, DevStatus* st, int zero_in) {
  __shared__ int s_tile, s_err, s_prefix, s_agg;
  __shared__ int s_warp[kScanThreads / 32];
  __shared__ int s_v[scan_pad(kScanTile)];
  if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1);
  if (threadIdx.x == 32) s_err = dev_err(st);
  __syncthreads();
  if (s_err) return;
  const int tile = s_tile;
  const int base = tile * kScanTile;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int q = k * kScanThreads + threadIdx.x;
    const int idx = base + q;
    int x = 0;
    if (idx < count) {
      x = in[idx];
      if (zero_in) const_cast<int*>(in)[idx] = 0;
    }
    s_v[scan_pad(q)] = x;
  }
  __syncthreads();
  int v[kScanItems];
  int local = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = s_v[scan_pad(threadIdx.x * kScanItems + k)];
    local += v[k];
  }
  // block exclusive scan of the per-thread sums
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = local;
  for (int d = 1; d < 32; d <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += t;
  }
  if (lane == 31) s_warp[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const int w = lane < kScanThreads / 32 ? s_warp[lane] : 0;
    int wi = w;
    for (int d = 1; d < 32; d <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= d) wi += t;
    }
    if (lane < kScanThreads / 32) s_warp[lane] = wi - w;   // exclusive warp offsets
    if (lane == kScanThreads / 32 - 1) s_agg = wi;
  }
  __syncthreads();
  // tile prefix by look-back (warp 0) while every thread stores its
  // tile-local exclusive values
  if (wid == 0) {
    const int agg = s_agg;
    const int prefix = lookback_warp(status, tile, agg, st);
    if (lane == 0) {
      s_prefix = prefix;
      if (base + kScanTile >= count) out[count] = prefix + agg;   // total
    }
  }
  int run = incl - local + s_warp[wid];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    s_v[scan_pad(threadIdx.x * kScanItems + k)] = run;
    run += v[k];
  }
  __syncthreads();
  const int pre = s_prefix;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int q = k * kScanThreads + threadIdx.x;
    const int idx = base + q;
    if (idx < count) out[idx] = s_v[scan_pad(q)] + pre;
  }
}
}  // namespace

int scan_tiles_for(int count) { return (count + kScanTile - 1) / kScanTile; }

void launch_scan(dss_handle* h, const int* in, int* out, int count, int which, bool zero_in) {
  int tiles = scan_tiles_for(count);
  if (tiles < 1) tiles = 1;
  k_scan<<<tiles, kScanThreads, 0, h->stream>>>(in, out, count,
                                                 h->scan_status + which * h->scan_tiles_max,
                                                 h->scan_ticket + which, h->status, zero_in ? 1 : 0);
}

void launch_sort(dss_handle* h, bool predict, int src, int dst) {
  const int n = (int)h->n;
  const int blocks = (n + kThreads - 1) / kThreads;
  prof_mark(h, 0);
  k_key_hist<<<blocks, kThreads, 0, h->stream>>>(h->g, h->ig, h->sg, h->st[src], h->key, h->offs,
                                                 h->cell_count, h->status, predict, h->scan_status,
                                                 h->scan_ticket, h->scan_tiles_max, h->pred, h->xc);
  prof_mark(h, 1);
  launch_scan(h, h->cell_count, h->cell_start, h->g.ncell, 0, true);
  prof_mark(h, 2);
  k_scatter<<<blocks, kThreads, 0, h->stream>>>(n, h->key, h->offs, h->cell_start, h->tmp, h->status);
  prof_mark(h, 3);
  if (h->g.wave)
    k_rank_gather<true><<<blocks, kThreads, 0, h->stream>>>(h->g, h->ig, h->sg, h->st[src], h->st[dst], h->key,
                                                            h->cell_start, h->tmp, h->perm, h->cellid,
                                                            h->posf, h->status, predict, h->pred, h->xc);
  else
    k_rank_gather<false><<<blocks, kThreads, 0, h->stream>>>(h->g, h->ig, h->sg, h->st[src], h->st[dst], h->key,
                                                             h->cell_start, h->tmp, h->perm, h->cellid,
                                                             h->posf, h->status, predict, h->pred, h->xc);
}

// Self-test of the integer-operation conversions (f32_rn, f32_split, f64_of,
// floor_mul, f64_of_nonneg) over caller-chosen inputs.
namespace {
__global__ void k_selftest_conversions(const double* __restrict__ v, int64_t n, double inv, float invf,
                                       float* __restrict__ hi, float* __restrict__ shi,
                                       float* __restrict__ slo, double* __restrict__ back,
                                       int* __restrict__ fl, const int* __restrict__ ci,
                                       double* __restrict__ cd) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const double x = v[k];
    const float h = f32_rn(x);
    hi[k] = h;
    f32_split(x, shi[k], slo[k]);
    back[k] = f64_of(h);
    fl[k] = floor_mul(x, inv, invf);
    cd[k] = f64_of_nonneg(ci[k]);
  }
}
}  // namespace

extern "C" int dss_selftest_conversions(const double* v, int64_t n, double inv, float* hi, float* split_hi,
                                        float* split_lo, double* back, int32_t* floor_out,
                                        const int32_t* ints, double* ints_out, void* cuda_stream) {
  if (n < 0 || (n > 0 && (!v || !hi || !split_hi || !split_lo || !back || !floor_out || !ints || !ints_out)))
    return DSS_ERR_ARG;
  if (n == 0) return DSS_OK;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  k_selftest_conversions<<<(int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, s>>>(
      v, n, inv, (float)inv, hi, split_hi, split_lo, back, floor_out, ints, ints_out);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return DSS_ERR_CUDA;
  return DSS_OK;
}
