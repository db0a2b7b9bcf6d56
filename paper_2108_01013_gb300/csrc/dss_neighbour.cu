// Symmetric (half-stencil) fixed-radius near-neighbour enumeration
// (Sec. II A, Fig. 5): each pair is found exactly once, by its owner, and
// written into the owner's fixed-capacity row (capacity M, the shell
// estimate of Sec. II A), in a fixed visiting order.
//
// The decision uses an FP32 conservative prefilter on cell-local coordinates;
// candidates within the rounding band of the cutoff are decided by the exact
// FP64 predicate, so the pair set is the FP64 brute-force set bit for bit.
//
// The exclusive scan of the row lengths (the pair offsets of each owner) is
// fused into the same kernel with a single-pass decoupled look-back over
// warps (32 owners each) of blocks taken in launch order.
#include "dss_internal.cuh"

namespace {
constexpr int kThreads = 128;

// Per-owner state of the enumeration; everything the candidate loop reads is
// held in registers.
struct EnumCtx {
  const float4* __restrict__ posf;
  float4 pi;
  float sc, sa;     // cutoff of pair (i, j): s = a_j sc + sa (a_i + a_j + delta)
  float sa2;        // with electro-chemical forces the cutoff is max(s, a_j + sa2)
  float m2;         // r^2 margin of the FP32 decision
  float lc, la;     // lubrication cutoff of pair (i, j): a_j lc + la (row order only)
  float hx, hy, hz; // half box: a separation beyond it is decided exactly
  bool img;         // the stencil reaches past half the box along some axis
  int M;
  int cnt;
  int nnear;        // SPLIT rows: pairs within the lubrication range, at the row's front
  int band;
  int* row;
  // exact FP64 decision
  const Geo* g;
  const InstGeo* I;
  const StateBuf* s;
  double off;
  int i;
};

__device__ __forceinline__ void enum_init(EnumCtx& e, const Geo& g, const InstGeo& I, const StateBuf& s,
                                          const float4* __restrict__ posf, int i, double off, int* row,
                                          int reach) {
  e.posf = posf;
  e.pi = posf[i];
  // delta of Sec. II A: a fixed multiple of a0 (mode 1) or of the mean
  // radius (mode 0); the FP32 cutoff is within a few ulp of the exact one,
  // far inside the margin
  if (g.mode == 1) {
    e.sc = 1.0f;
    e.sa = e.pi.w + (float)(g.delta * g.a0 > g.de ? g.delta * g.a0 : g.de);
  } else {
    e.sc = 1.0f + 0.5f * (float)g.delta;
    e.sa = e.pi.w * e.sc;
  }
  // the electro-chemical range (a surface distance): a_i + a_j + de
  e.sa2 = e.pi.w + (float)g.de;
  if (g.mode == 1) {
    e.lc = 1.0f;
    e.la = e.pi.w + (float)(g.delta * g.a0);
  } else {
    e.lc = 1.0f + 0.5f * (float)g.delta;
    e.la = e.pi.w * e.lc;
  }
  e.nnear = 0;
  e.m2 = I.r2_margin;
  e.hx = I.halfLf[0];
  e.hy = I.halfLf[1];
  e.hz = I.halfLf[2];
  // a stencil cell is at most reach+1 cells away along y and z and, across
  // y = L_y, reach+2 along x: separations stay below half the box when the
  // box is wider than twice that (plus one cell of slack)
  e.img = I.nc[0] < 2 * reach + 5 || I.nc[1] < 2 * reach + 3 || I.nc[2] < 2 * reach + 3;
  e.M = g.M;
  e.cnt = 0;
  e.band = 0;
  e.row = row;
  e.g = &g;
  e.I = &I;
  e.s = &s;
  e.off = off;
  e.i = i;
}

// One candidate j of owner i (positions relative to the candidate cell's
// origin): FP32 decision on cell-local coordinates, certainly a pair,
// certainly not, or (within the margin of the cutoff, or past half the box)
// the exact FP64 predicate; a pair is appended to the row.  SPLIT (pairs
// listed beyond the lubrication range, i.e. with electro-chemical forces):
// pairs within the lubrication range by an FP32 test go to the row's front
// in visiting order, the others to its back from the end; the row is closed
// up afterwards (close_row).  Only the order within the row changes.
// r^2 - s^2 of a candidate in FP32 on cell-local coordinates (s: the
// pair's cutoff), the one value every decision starts from.
template <bool ECH>
__device__ __forceinline__ float cand_t(const EnumCtx& e, float4 pj, float px, float py, float pz, float& dx,
                                       float& dy, float& dz) {
  dx = pj.x - px;
  dy = pj.y - py;
  dz = pj.z - pz;
  float sv = fmaf(pj.w, e.sc, e.sa);
  if (ECH) sv = fmaxf(sv, pj.w + e.sa2);
  return fmaf(-sv, sv, fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
}

template <bool ECH, bool SPLIT>
__device__ __forceinline__ void take_candidate(EnumCtx& e, float4 pj, int j, float px, float py, float pz) {
  float dx, dy, dz;
  const float t = cand_t<ECH>(e, pj, px, py, pz, dx, dy, dz);
  // nearly every candidate lies beyond the cutoff by more than the margin:
  // one test and out (the half-box image test only on boxes narrower than
  // the stencil)
  if (t > e.m2 && !e.img) return;
  int dec;
  if (e.img && (fabsf(dx) > e.hx || fabsf(dy) > e.hy || fabsf(dz) > e.hz))
    dec = -1;
  else
    dec = t < -e.m2 ? 1 : (t > e.m2 ? 0 : -1);
  if (dec < 0) {
    ++e.band;
    const StateBuf& s = *e.s;
    const int n = e.g->n, i = e.i;
    dec = exact_is_pair(*e.g, *e.I, e.off, s.x[i], s.x[n + i], s.x[2 * n + i], s.a[i], s.x[j],
                        s.x[n + j], s.x[2 * n + j], s.a[j]) ? 1 : 0;
  }
  if (dec) {
    if (SPLIT) {
      const float sl = fmaf(pj.w, e.lc, e.la);
      const bool near = fmaf(dz, dz, fmaf(dy, dy, dx * dx)) < sl * sl;
      if (e.cnt < e.M) e.row[near ? e.nnear : e.M - 1 - (e.cnt - e.nnear)] = j;
      e.nnear += near;
    } else {
      if (e.cnt < e.M) e.row[e.cnt] = j;
    }
    ++e.cnt;
  }
}

// SPLIT rows: the far block [M - nf, M) moves down to follow the near block
// (ascending, each entry read before any write reaches it: the source index
// exceeds the destination by the gap).  Overflowing rows are left as they
// are (the step is not committed).
__device__ __forceinline__ void close_row(EnumCtx& e) {
  if (e.cnt > e.M) return;
  const int nf = e.cnt - e.nnear;
  const int gap = e.M - e.cnt;
  if (nf > 0 && gap > 0)
    for (int k = 0; k < nf; ++k) e.row[e.nnear + k] = e.row[e.nnear + gap + k];
}

// SCREEN: the candidates of a range go 32 at a time through a screen first:
// the one-test rejection alone, unrolled with four loads ahead and no branch
// in the body, leaves a bit per candidate that may be a pair (about one in a
// hundred on the polydisperse packings); those take the full decision
// afterwards in ascending order, so the row is the one the plain loop
// writes.  It pays on cells of three or more particles (1M log-uniform
// [1, 10]: 247 -> 212 us; Table 5, radius ratio 3: 59 -> 47 us); on the
// sparse 100k grid (1.7 per cell) the plain loop is faster (28.7 against
// 30.7 us).
template <bool ECH, bool SPLIT>
__device__ __forceinline__ void scan_screened(EnumCtx& e, int jb, int je, float px, float py, float pz) {
  for (int base = jb; base < je; base += 32) {
    const int cnt = min(32, je - base);
    const float4* __restrict__ q = e.posf + base;
    unsigned m = 0u;
#pragma unroll 4
    for (int k = 0; k < cnt; ++k) {
      float dx, dy, dz;
      const float t = cand_t<ECH>(e, __ldg(q + k), px, py, pz, dx, dy, dz);
      m |= (t > e.m2 ? 0u : 1u) << k;
    }
    while (m) {
      const int k = __ffs(m) - 1;
      m &= m - 1u;
      take_candidate<ECH, SPLIT>(e, __ldg(q + k), base + k, px, py, pz);
    }
  }
}

// Visits the candidates [jb, je) of one stencil cell (origin displaced by
// (cxo, cyo, czo) from the owner's cell) in order, plainly or (SCREEN) through
// the screen; boxes narrower than the stencil, where every candidate takes
// the image test, always take the plain loop.  Both make the same decisions
// in the same order, so the rows are identical.
template <bool ECH, bool SCREEN, bool SPLIT = false>
__device__ __forceinline__ void scan_range(EnumCtx& e, int jb, int je, float cxo, float cyo, float czo) {
  const float px = e.pi.x - cxo, py = e.pi.y - cyo, pz = e.pi.z - czo;
  if (SCREEN && !e.img) {
    scan_screened<ECH, SPLIT>(e, jb, je, px, py, pz);
    return;
  }
  for (int j = jb; j < je; ++j) take_candidate<ECH, SPLIT>(e, __ldg(e.posf + j), j, px, py, pz);
}

// Row lengths, counters and the fused exclusive scan of the row lengths:
// each warp is one scan tile (32 owners) with its own decoupled look-back,
// so no warp waits for the others of its block.
__device__ __forceinline__ void finish_rows(const Geo& g, const StateBuf& s, ListBuf& L,
                                            int* __restrict__ bw_count, unsigned long long* scan_status,
                                            DevStatus* st, const EnumCtx& e, int i, int wtile) {
  const int n = g.n;
  const int lane = threadIdx.x & 31;
  const int v = i < n ? (e.cnt < g.M ? e.cnt : g.M) : 0;
  if (i < n) {
    L.count[i] = v;
    if (e.cnt > g.M) set_err(st, DSS_ERR_CAPACITY);
    bw_count[i] = 0;
    const int id = s.id[i];
    L.slot_of_id[id] = i;
    L.id_of_slot[i] = id;
  }
  int m = i < n ? e.cnt : 0, b = i < n ? e.band : 0;
  int incl = v;
  for (int d = 1; d < 32; d <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += t;
  }
  for (int d = 16; d > 0; d >>= 1) {
    m = max(m, __shfl_xor_sync(0xffffffffu, m, d));
    b += __shfl_xor_sync(0xffffffffu, b, d);
  }
  if (lane == 0) {
    atomicMax(&st->w[ST_MAXROW], m);
    if (b) atomicAdd(&st->w[ST_BAND], b);
  }
  const int agg = __shfl_sync(0xffffffffu, incl, 31);
  const int prefix = lookback_warp(scan_status, wtile, agg, st);
  if (i < n) L.start[i] = prefix + incl - v;
  if (lane == 0 && (wtile + 1) * 32 >= n) L.start[n] = prefix + agg;
  // one instance: the row, compacted at its offset with its owner (the pair
  // order of the pair-balanced force kernel; the thread reads back its own
  // row writes)
  if (L.pown && i < n) {
    const int64_t s0 = prefix + incl - v;
    for (int k = 0; k < v && s0 + k < g.pcap; ++k) {
      L.pj[s0 + k] = e.row[k];
      L.pown[s0 + k] = i;
    }
  }
}

template <bool ECH, bool SCREEN, bool SPLIT>
__global__ void __launch_bounds__(kThreads, 8)
k_enumerate(Geo g, const InstGeo* __restrict__ ig, const StepGeo* __restrict__ sgk, StateBuf s,
            const float4* __restrict__ posf, const int* __restrict__ cellid,
            const int* __restrict__ cell_start, ListBuf L, int* __restrict__ bw_count,
            unsigned long long* scan_status, int* scan_ticket, DevStatus* st, int adv) {
  if (dev_err(st)) return;
  __shared__ int s_tile;
  if (threadIdx.x == 0) s_tile = atomicAdd(scan_ticket, 1);
  __syncthreads();
  const int tile = s_tile;
  const int i = tile * kThreads + threadIdx.x;
  const int n = g.n;
  EnumCtx e;
  e.cnt = 0;
  e.band = 0;
  if (i < n) {
    const int inst = s.inst[i];
    const InstGeo& I = ig[inst];
    const StepGeo sg = sgk[inst];
    enum_init(e, g, I, s, posf, i, sg.off, L.list + (int64_t)i * g.Ms, 1);
    const int fsh = sg.fsh;
    const float offr = sg.offr_hi;
    const int nx = I.nc[0], ny = I.nc[1], nz = I.nc[2];
    const int cb = I.cell_base;
    const int c = cellid[i] - cb;
    const int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
    // neighbouring cell coordinates by conditional wraps (no integer
    // division in the stencil walk; every offset below stays within one box)
    const int xm = cx == 0 ? nx - 1 : cx - 1, xp = cx + 1 == nx ? 0 : cx + 1;
    const int zm = cz == 0 ? nz - 1 : cz - 1, zp = cz + 1 == nz ? 0 : cz + 1;
    // own cell (partners after i) and the cell x+1
    scan_range<ECH, SCREEN, SPLIT>(e, i + 1, cell_start[cb + c + 1], 0.f, 0.f, 0.f);
    {
      const int q = cb + (cz * ny + cy) * nx + xp;
      scan_range<ECH, SCREEN, SPLIT>(e, cell_start[q], cell_start[q + 1], I.csf[0], 0.f, 0.f);
    }
    // layer y, z+1: three x cells
    {
      const int row = cb + (zp * ny + cy) * nx;
      scan_range<ECH, SCREEN, SPLIT>(e, cell_start[row + xm], cell_start[row + xm + 1], -I.csf[0], 0.f, I.csf[2]);
      scan_range<ECH, SCREEN, SPLIT>(e, cell_start[row + cx], cell_start[row + cx + 1], 0.f, 0.f, I.csf[2]);
      scan_range<ECH, SCREEN, SPLIT>(e, cell_start[row + xp], cell_start[row + xp + 1], I.csf[0], 0.f, I.csf[2]);
    }
    // layer y+1: 3x3 cells, or across y = L_y the 4 x cells covering the
    // image range shifted by the Lees-Edwards offset
    const bool le = cy == ny - 1;
    const int qy = le ? 0 : cy + 1;
    const int x0 = le ? -2 - fsh : -1, x1 = le ? 1 - fsh : 1;
    const int xs = le ? wrapi(cx + x0, nx) : xm;   // x cell of the first offset
    for (int oz = -1; oz <= 1; ++oz) {
      const int qz = oz < 0 ? zm : (oz > 0 ? zp : cz);
      int qx = xs;
      for (int ox = x0; ox <= x1; ++ox, qx = qx + 1 == nx ? 0 : qx + 1) {
        const int q = cb + (qz * ny + qy) * nx + qx;
        float cxo, cyo, czo;
        stencil_shift(I, ox, 1, oz, le ? 1 : 0, fsh, offr, cxo, cyo, czo);
        scan_range<ECH, SCREEN, SPLIT>(e, cell_start[q], cell_start[q + 1], cxo, cyo, czo);
      }
    }
  }
  if (SPLIT && i < n) close_row(e);
  finish_rows(g, s, L, bw_count, scan_status, st, e, i, tile * (kThreads / 32) + (threadIdx.x >> 5));
}

// Size classes (Sec. II A: cells smaller than 2 a_max, a larger stencil for
// the larger particles).  Owner i of class c takes the partners of its own
// class from the half stencil of reach R = rtab[c][c] (own bin after i; the
// rest of the own row in +x; the rows z+1..z+R of its y layer; the layers
// y+1..y+R), and the partners of every smaller class c2 from the full stencil
// of reach rtab[c][c2] in that class's layer of bins: each pair is found
// once, by its larger member (or by the half stencil within a class).  Rows
// crossing y = L_y (either way) cover the x range shifted by the
// Lees-Edwards offset.
template <bool ECH>
__global__ void __launch_bounds__(kThreads, 8)
k_enumerate_classes(Geo g, const InstGeo* __restrict__ ig, const StepGeo* __restrict__ sgk, StateBuf s,
                    const float4* __restrict__ posf, const int* __restrict__ cellid,
                    const int* __restrict__ cell_start, ListBuf L, int* __restrict__ bw_count,
                    unsigned long long* scan_status, int* scan_ticket, DevStatus* st) {
  if (dev_err(st)) return;
  __shared__ int s_tile;
  if (threadIdx.x == 0) s_tile = atomicAdd(scan_ticket, 1);
  __syncthreads();
  const int tile = s_tile;
  const int i = tile * kThreads + threadIdx.x;
  const int n = g.n;
  EnumCtx e;
  e.cnt = 0;
  e.band = 0;
  if (i < n) {
    const int inst = s.inst[i];
    const InstGeo& I = ig[inst];
    const StepGeo sg = sgk[inst];
    enum_init(e, g, I, s, posf, i, sg.off, L.list + (int64_t)i * g.Ms, g.reach);
    const int fsh = sg.fsh;
    const float offr = sg.offr_hi;
    const int nx = I.nc[0], ny = I.nc[1], nz = I.nc[2];
    const int layer = I.ncell_layer;
    const int cls = s.cls[i];
    const int c = (cellid[i] - I.cell_base) % layer;
    const int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
    // own bin, partners after i
    scan_range<ECH, false>(e, i + 1, cell_start[cellid[i] + 1], 0.f, 0.f, 0.f);
    for (int c2 = cls; c2 >= 0; --c2) {
      const int R = g.rtab[cls][c2];
      const bool half = c2 == cls;
      const int lb = I.cell_base + c2 * layer;
      for (int oy = half ? 0 : -R; oy <= R; ++oy) {
        const int yy = cy + oy;
        const int le = yy >= ny ? 1 : (yy < 0 ? -1 : 0);
        const int qy = le == 1 ? yy - ny : (le == -1 ? yy + ny : yy);
        for (int oz = (half && oy == 0) ? 0 : -R; oz <= R; ++oz) {
          const int qz = wrapi(cz + oz, nz);
          int xa, xb;
          if (half && oy == 0 && oz == 0) {
            xa = 1;
            xb = R;
          } else if (le == 1) {
            xa = -R - 1 - fsh;
            xb = R - fsh;
          } else if (le == -1) {
            xa = -R + fsh;
            xb = R + 1 + fsh;
          } else {
            xa = -R;
            xb = R;
          }
          // the row's cells are adjacent bins (split where x wraps): one
          // candidate range per piece, most of them empty on small cells
          const int rowq = lb + (qz * ny + qy) * nx;
          int ox = xa;
          while (ox <= xb) {
            const int x0 = wrapi(cx + ox, nx);
            const int m = min(xb - ox + 1, nx - x0);
            const int q0 = rowq + x0;
            const int lo = cell_start[q0], hi = cell_start[q0 + m];
            if (lo < hi) {
              int k = 0, kend = cell_start[q0 + 1];
              float cxo, cyo, czo;
              stencil_shift(I, ox, oy, oz, le, fsh, offr, cxo, cyo, czo);
              for (int j = lo; j < hi; ++j) {
                if (j >= kend) {
                  do {
                    ++k;
                    kend = cell_start[q0 + k + 1];
                  } while (j >= kend);
                  stencil_shift(I, ox + k, oy, oz, le, fsh, offr, cxo, cyo, czo);
                }
                scan_range<ECH, false>(e, j, j + 1, cxo, cyo, czo);
              }
            }
            ox += m;
          }
        }
      }
    }
  }
  finish_rows(g, s, L, bw_count, scan_status, st, e, i, tile * (kThreads / 32) + (threadIdx.x >> 5));
}
}  // namespace

int enum_tiles_for(int n) { return (n + kThreads - 1) / kThreads; }
int enum_scan_tiles_for(int n) { return enum_tiles_for(n) * (kThreads / 32); }

void launch_enumerate(dss_handle* h, int stbuf, int dst_list, int adv) {
  const int n = (int)h->n;
  ListBuf& L = h->lb[dst_list];
  prof_mark(h, 4);
  // the pair-mean lubrication cutoff and the electro-chemical range combine
  // by a maximum, which only that case needs in the candidate test
  const bool ech = h->g.de > 0.0 && h->g.mode == 0;
  auto kc = ech ? k_enumerate_classes<true> : k_enumerate_classes<false>;
  // cells holding many particles (long ranges, large radius ratios)
  const bool crowded = h->tune_enum_unr ? h->tune_enum_unr == 4 : h->n >= 8 * (int64_t)h->g.ncell;
  // with electro-chemical forces over crowded cells (long ranges) most
  // listed pairs lie beyond the lubrication range: rows put the others
  // first, so that the pair kernel's warps meet runs of pairs without
  // lubrication (short rows gain less than the reordering costs)
  const bool split = h->g.de > 0.0 && crowded;
  // cells of three or more particles on average (the 1M log-uniform
  // packing: 7.5; Table 5: 24) take the screened candidate loop; under two
  // per cell (the 100k packing: 1.7) the plain loop is faster
  const bool screen = crowded || (!h->tune_enum_unr && h->n >= 3 * (int64_t)h->g.ncell);
  auto k1 = ech ? (split ? k_enumerate<true, true, true> : k_enumerate<true, false, false>)
                : split  ? k_enumerate<false, true, true>
                : screen ? k_enumerate<false, true, false>
                         : k_enumerate<false, false, false>;
  if (h->g.nclass > 1)
    kc<<<enum_tiles_for(n), kThreads, 0, h->stream>>>(
        h->g, h->ig, h->sg, h->st[stbuf], h->posf, h->cellid, h->cell_start, L, h->bw_count,
        h->scan_status + h->scan_tiles_max, h->scan_ticket + 1, h->status);
  else
    k1<<<enum_tiles_for(n), kThreads, 0, h->stream>>>(
        h->g, h->ig, h->sg, h->st[stbuf], h->posf, h->cellid, h->cell_start, L, h->bw_count,
        h->scan_status + h->scan_tiles_max, h->scan_ticket + 1, h->status, adv);
  h->last_list = dst_list;
  h->compact_ok[dst_list] = L.pown != nullptr;
}
