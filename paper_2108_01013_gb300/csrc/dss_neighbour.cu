// Symmetric (half-stencil) fixed-radius near-neighbour enumeration
// (Sec. II A, Fig. 6): each pair is found exactly once, by its owner, and
// written into the owner's fixed-capacity row (capacity M, the shell
// estimate of Sec. II A).  Rows come out sorted by partner index because the
// stencil cells are visited in increasing cell id and every cell is a
// contiguous, increasing range of the sorted order.
//
// The decision uses an FP32 conservative prefilter on cell-local coordinates;
// candidates within the rounding band of the cutoff are decided by the exact
// FP64 predicate, so the pair set is the FP64 brute-force set bit for bit.
#include "dss_internal.cuh"

namespace {
constexpr int kThreads = 128;

__global__ void __launch_bounds__(kThreads)
k_enumerate(Geo g, StateBuf s, const float4* __restrict__ posf, const int* __restrict__ cellid,
            const int* __restrict__ cell_start, ListBuf L, DevStatus* st, int adv) {
  int* __restrict__ count = L.count;
  int* __restrict__ list = L.list;
  if (dev_err(st)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = g.n;
  int cnt = 0, band = 0;
  if (i < n) {
    const double off = le_offset(g, dev_nstep(st) + adv);
    const int fsh = le_shift_cells(g, off);
    const int c = cellid[i];
    const int cx = c % g.nc[0], cy = (c / g.nc[0]) % g.nc[1], cz = c / (g.nc[0] * g.nc[1]);
    StencilCell sc[17];
    const int ns = forward_cells(g, cx, cy, cz, fsh, sc);
    const float4 pi = posf[i];
    const double ai = s.a[i];
    int* row = list + (int64_t)i * g.M;
    for (int q = 0; q < ns; ++q) {
      const StencilCell cur = sc[q];
      const int jb = cur.le == 2 ? i + 1 : cell_start[cur.cell];
      const int je = cell_start[cur.cell + 1];
      const float cxo = (float)(cur.ox * g.cs[0] + (cur.le == 1 ? off : 0.0));
      const float cyo = (float)(cur.oy * g.cs[1]);
      const float czo = (float)(cur.oz * g.cs[2]);
      for (int j = jb; j < je; ++j) {
        const float4 pj = posf[j];
        const float sf = pi.w + pj.w + pair_delta_f(g, pi.w, pj.w);
        int dec = prefilter(g, pi, pj, cxo, cyo, czo, sf);
        if (dec < 0) {
          ++band;
          dec = exact_is_pair(g, off, s.x[i], s.x[n + i], s.x[2 * n + i], ai, s.x[j], s.x[n + j],
                              s.x[2 * n + j], s.a[j]) ? 1 : 0;
        }
        if (dec) {
          if (cnt < g.M) row[cnt] = j;
          ++cnt;
        }
      }
    }
    count[i] = cnt < g.M ? cnt : g.M;
    if (cnt > g.M) set_err(st, DSS_ERR_CAPACITY);
    // id <-> row maps of this list's index space (history lookups, output)
    const int id = s.id[i];
    L.slot_of_id[id] = i;
    L.id_of_slot[i] = id;
  }
  // warp-aggregated counters
  int m = cnt;
  for (int d = 16; d > 0; d >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, d));
  int b = band;
  for (int d = 16; d > 0; d >>= 1) b += __shfl_xor_sync(0xffffffffu, b, d);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&st->w[ST_MAXROW], m);
    if (b) atomicAdd(&st->w[ST_BAND], b);
  }
}

__global__ void k_reset_counters(DevStatus* st) {
  st->w[ST_MAXROW] = 0;
  st->w[ST_BAND] = 0;
  st->w[ST_NCONT] = 0;
}
}  // namespace

void launch_enumerate(dss_handle* h, int stbuf, int dst_list, int adv) {
  const int n = (int)h->n;
  ListBuf& L = h->lb[dst_list];
  prof_mark(h, 4);
  k_reset_counters<<<1, 1, 0, h->stream>>>(h->status);
  prof_mark(h, 5);
  k_enumerate<<<(n + kThreads - 1) / kThreads, kThreads, 0, h->stream>>>(
      h->g, h->st[stbuf], h->posf, h->cellid, h->cell_start, L, h->status, adv);
  h->last_list = dst_list;
  prof_mark(h, 6);
  launch_scan(h, L.count, L.start, n, 1, false);
}
