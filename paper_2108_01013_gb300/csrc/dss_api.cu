// Host side of the C ABI declared in include/dss.h: validation, buffer
// management, the per-step launch sequence and its CUDA-graph capture.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "dss_internal.cuh"

namespace {

#define CK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) return DSS_ERR_CUDA; \
  } while (0)

template <typename T>
int dalloc(dss_handle* h, T** p, size_t count) {
  size_t b = sizeof(T) * (count > 0 ? count : 1);
  if (cudaMalloc((void**)p, b) != cudaSuccess) return DSS_ERR_CUDA;
  h->bytes += (int64_t)b;
  return DSS_OK;
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

void free_buffers(dss_handle* h) {
  for (int b = 0; b < 2; ++b) {
    StateBuf& s = h->st[b];
    dfree(s.x); dfree(s.u); dfree(s.w); dfree(s.al); dfree(s.aw); dfree(s.a); dfree(s.id); dfree(s.inst);
    dfree(s.cls);
    dfree(s.iy);
    dfree(s.vf); dfree(s.wf); dfree(s.posl); dfree(s.cellc); dfree(s.wv);
    memset(&s, 0, sizeof(s));
    ListBuf& L = h->lb[b];
    dfree(L.count); dfree(L.list); dfree(L.start); dfree(L.xi); dfree(L.xr); dfree(L.slot_of_id);
    dfree(L.id_of_slot); dfree(L.pown); dfree(L.pj);
    memset(&L, 0, sizeof(L));
  }
  dfree(h->posf); dfree(h->cellid); dfree(h->perm); dfree(h->key); dfree(h->offs); dfree(h->pred);
  h->pred = nullptr;
  dfree(h->xc); dfree(h->mark);
  h->xc = nullptr; h->mark = nullptr; h->marked = false;
  dfree(h->cell_count); dfree(h->cell_start); dfree(h->tmp); dfree(h->spart);
  dfree(h->own); dfree(h->bw_count); dfree(h->bw_rec); dfree(h->carry); dfree(h->own_s);
  h->own = nullptr; h->bw_count = nullptr; h->bw_rec = nullptr; h->carry = nullptr; h->own_s = nullptr;
  h->pb_blocks = 0;
  h->compact_ok[0] = h->compact_ok[1] = false;
  dfree(h->io3); dfree(h->io3b); dfree(h->io_id); dfree(h->stage);
  h->stage = nullptr; dfree(h->scan_status); dfree(h->scan_ticket);
  dfree(h->sigma);
  dfree(h->sigma_sum);
  dfree(h->a_by_id);
  dfree(h->inst_map);
  dfree(h->cls_map);
  h->cls_map = nullptr;
  dfree(h->ig);
  dfree(h->sg);
  h->sigma_sum = nullptr;
  h->inst_map = nullptr;
  h->ig = nullptr;
  h->sg = nullptr;
  dfree(h->done_blocks);
  h->done_blocks = nullptr;
  h->sigma = nullptr;
  h->a_by_id = nullptr;
  h->posf = nullptr; h->cellid = nullptr; h->perm = nullptr; h->key = nullptr; h->offs = nullptr;
  h->cell_count = nullptr; h->cell_start = nullptr; h->tmp = nullptr;
  h->spart = nullptr; h->io3 = nullptr; h->io3b = nullptr; h->io_id = nullptr; h->scan_status = nullptr;
  h->scan_ticket = nullptr;
  h->bytes = 0;
  h->sized = false;
}

void drop_graphs(dss_handle* h) {
  for (int k = 0; k < 4; ++k) {
    if (h->graph_ok[k]) cudaGraphExecDestroy(h->step_graph[k]);
    h->graph_ok[k] = false;
    if (h->multi_ok[k]) cudaGraphExecDestroy(h->multi_graph[k]);
    h->multi_ok[k] = false;
  }
}

// Pair-capacity dependent buffers: per-pair records, stretch, contact flags,
// stress partials.  keep_hist copies the committed history's pair arrays.
int alloc_pair_buffers(dss_handle* h, int64_t pcap, bool keep_hist) {
  const int64_t old = h->pcap;
  int r;
  for (int b = 0; b < 2; ++b) {
    ListBuf& L = h->lb[b];
    Xi4 *xi = nullptr, *xr = nullptr;
    if ((r = dalloc(h, &xi, (size_t)pcap))) return r;
    if (h->g.k_r > 0.0 && (r = dalloc(h, &xr, (size_t)pcap))) {
      dfree(xi);
      return r;
    }
    if (keep_hist && b == h->hist && L.xi && old > 0) {
      CK(cudaMemcpyAsync(xi, L.xi, sizeof(Xi4) * old, cudaMemcpyDeviceToDevice, h->stream));
      if (xr && L.xr) CK(cudaMemcpyAsync(xr, L.xr, sizeof(Xi4) * old, cudaMemcpyDeviceToDevice, h->stream));
      CK(cudaStreamSynchronize(h->stream));
    }
    dfree(L.xi);
    dfree(L.xr);
    L.xi = xi;
    L.xr = xr;
    // the compact owner / partner arrays of the pair-balanced pair kernel
    // (rewritten by every enumeration of the list)
    {
      int *pown = nullptr, *pj = nullptr;
      if ((r = dalloc(h, &pown, (size_t)pcap))) return r;
      if ((r = dalloc(h, &pj, (size_t)pcap))) {
        dfree(pown);
        return r;
      }
      dfree(L.pown);
      dfree(L.pj);
      L.pown = pown;
      L.pj = pj;
    }
  }
  h->pcap = pcap;
  h->g.pcap = pcap;
  {
    const size_t rb = h->p.precision == DSS_MIXED ? sizeof(float) : sizeof(double);
    const size_t per = h->K > 1 ? 30 : 12;   // two boundary slots per warp of pairs
    char* carry = nullptr;
    if ((r = dalloc(h, &carry, per * rb * (size_t)((pcap + 31) / 32)))) return r;
    dfree(h->carry);
    h->carry = carry;
    h->pb_blocks = pair_pb_blocks(h);
  }
  h->compact_ok[0] = h->compact_ok[1] = false;
  double* sp = nullptr;
  // (the balanced grid holds at most 4 blocks per SM; batched instances keep
  // 16 stress slices each)
  const int pb = std::max(std::max(pair_grid_blocks(h), h->K == 1 ? 4 * h->sms : 0), 16 * h->K);
  if ((r = dalloc(h, &sp, 18 * (size_t)pb))) return r;
  dfree(h->spart);
  h->spart = sp;
  h->spart_blocks = pb;
  drop_graphs(h);
  return DSS_OK;
}

int alloc_buffers(dss_handle* h) {
  const size_t n = (size_t)h->n;
  int r;
  for (int b = 0; b < 2; ++b) {
    StateBuf& s = h->st[b];
    if ((r = dalloc(h, &s.x, 3 * n)) || (r = dalloc(h, &s.u, 3 * n)) || (r = dalloc(h, &s.w, 3 * n)) ||
        (r = dalloc(h, &s.al, 3 * n)) || (r = dalloc(h, &s.aw, 3 * n)) || (r = dalloc(h, &s.a, n)) ||
        (r = dalloc(h, &s.id, n)) || (r = dalloc(h, &s.inst, n)) || (r = dalloc(h, &s.cls, n)) ||
        (r = dalloc(h, &s.iy, n)))
      return r;
    if (h->p.precision == DSS_MIXED &&
        ((r = dalloc(h, &s.vf, n)) || (r = dalloc(h, &s.wf, n)) || (r = dalloc(h, &s.posl, n)) ||
         (r = dalloc(h, &s.cellc, n))))
      return r;
    if (h->g.wave && (r = dalloc(h, &s.wv, n))) return r;
    ListBuf& L = h->lb[b];
    if ((r = dalloc(h, &L.count, n)) || (r = dalloc(h, &L.list, n * (size_t)h->g.Ms)) ||
        (r = dalloc(h, &L.start, n + 1)) || (r = dalloc(h, &L.slot_of_id, n)) ||
        (r = dalloc(h, &L.id_of_slot, n)))
      return r;
  }
  if ((r = dalloc(h, &h->posf, n)) || (r = dalloc(h, &h->cellid, n)) || (r = dalloc(h, &h->perm, n)) ||
      (r = dalloc(h, &h->pred, 6 * n)) || (r = dalloc(h, &h->xc, n)) ||
      (r = dalloc(h, &h->key, n)) || (r = dalloc(h, &h->offs, n)) ||
      (r = dalloc(h, &h->cell_count, (size_t)h->g.ncell)) ||
      (r = dalloc(h, &h->cell_start, (size_t)h->g.ncell + 1)) || (r = dalloc(h, &h->tmp, n)) ||
      (r = dalloc(h, &h->io3, 3 * n)) || (r = dalloc(h, &h->io3b, 3 * n)) ||
      (r = dalloc(h, &h->stage, 15 * n)) ||
      (r = dalloc(h, &h->io_id, n)) || (r = dalloc(h, &h->sigma, 9 * (size_t)h->K)) ||
      (r = dalloc(h, &h->sigma_sum, 9 * (size_t)h->K)) || (r = dalloc(h, &h->a_by_id, n)) ||
      (r = dalloc(h, &h->inst_map, n)) || (r = dalloc(h, &h->cls_map, n)) ||
      (r = dalloc(h, &h->ig, (size_t)h->K)) ||
      (r = dalloc(h, &h->sg, (size_t)h->K)) || (r = dalloc(h, &h->done_blocks, 1)))
    return r;
  CK(cudaMemsetAsync(h->sigma, 0, 9 * sizeof(double) * h->K, h->stream));
  CK(cudaMemsetAsync(h->sigma_sum, 0, 9 * sizeof(double) * h->K, h->stream));
  CK(cudaMemsetAsync(h->done_blocks, 0, sizeof(unsigned int), h->stream));
  {
    const size_t rb = h->p.precision == DSS_MIXED ? sizeof(float) : sizeof(double);
    char* own = nullptr;
    char* bwr = nullptr;
    if ((r = dalloc(h, &own, 6 * n * rb)) || (r = dalloc(h, &h->bw_count, n)) ||
        (r = dalloc(h, &bwr, n * (size_t)h->g.M * bw_slot_values() * rb)))
      return r;
    h->own = own;
    h->bw_rec = bwr;
    if (h->K > 1) {
      char* own_s = nullptr;
      if ((r = dalloc(h, &own_s, 9 * n * rb))) return r;
      h->own_s = own_s;
    }
  }
  int tiles = std::max(scan_tiles_for(h->g.ncell), enum_scan_tiles_for((int)n));
  h->scan_tiles_max = std::max(tiles, 1);
  if ((r = dalloc(h, &h->scan_status, 2 * (size_t)h->scan_tiles_max)) ||
      (r = dalloc(h, &h->scan_ticket, 2)))
    return r;
  CK(cudaMemsetAsync(h->cell_count, 0, sizeof(int) * h->g.ncell, h->stream));
  h->pcap = 0;
  int per = h->p.pair_capacity > 0 ? h->p.pair_capacity : 16;
  if ((r = alloc_pair_buffers(h, std::max<int64_t>((int64_t)n * per, 1024), false))) return r;
  h->sized = true;
  return DSS_OK;
}

// Orders the library's stream after everything queued on the caller's stream.
int enter(dss_handle* h) {
  if (!h->own_stream) return DSS_OK;
  CK(cudaEventRecord(h->ev_enter, h->user_stream));
  CK(cudaStreamWaitEvent(h->stream, h->ev_enter, 0));
  return DSS_OK;
}

#define ENTER(h)            \
  do {                      \
    int e__ = enter(h);     \
    if (e__) return e__;    \
  } while (0)

int sync_status(dss_handle* h) {
  CK(cudaMemcpyAsync(h->status_host, h->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return DSS_OK;
}

int clear_err(dss_handle* h) {
  CK(cudaMemsetAsync(&h->status->w[ST_ERR], 0, sizeof(int), h->stream));
  return DSS_OK;
}

// The committed state (sorted order) into id order, all five vectors in one
// pass: dst[k] is device-accessible (device memory, mapped pinned host memory)
// or the staging area; a null dst[k] is skipped.
struct Dst5 {
  double* d[5];
};
__global__ void k_state_out(int n, StateBuf s, Dst5 dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k = s.id[i];
  const double* src[5] = {s.x, s.u, s.w, s.al, s.aw};
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    double* d = dst.d[q];
    if (!d) continue;
    d[k] = src[q][i];
    d[n + k] = src[q][n + i];
    d[2 * n + k] = src[q][2 * n + i];
  }
}

// Coalesced copy of up to five 3n-vectors (staging -> device-accessible views).
__global__ void k_copy5(int64_t m, Dst5 src, Dst5 dst) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int q = 0; q < 5; ++q)
      if (dst.d[q]) dst.d[q][t] = src.d[q][t];
}

// dss_load_state in one pass: the five vectors from device-accessible views,
// radii and instances in id order, ids = indices.
struct Src5 {
  const double* d[5];
};
__global__ void k_state_in(int n, Src5 src, StateBuf s, const double* __restrict__ a_by_id,
                           const int* __restrict__ inst_map, const unsigned char* __restrict__ cls_map) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double* dst[5] = {s.x, s.u, s.w, s.al, s.aw};
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    dst[q][i] = src.d[q][i];
    dst[q][n + i] = src.d[q][n + i];
    dst[q][2 * n + i] = src.d[q][2 * n + i];
  }
  s.a[i] = a_by_id[i];
  s.inst[i] = inst_map[i];
  s.cls[i] = cls_map[i];
  s.iy[i] = 0;
  s.id[i] = i;
}

// Address through which a kernel may access a caller's buffer: device and
// managed memory as is, pinned host memory through its mapped device
// pointer; nullptr for pageable host memory (copy engines only).
const void* device_view(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (at.type == cudaMemoryTypeDevice) return p;
  if ((at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeManaged) && at.devicePointer)
    return at.devicePointer;
  return nullptr;
}

// Tile 1 of a look-back whose tile 0 never publishes: the wait must give up.
__global__ void k_selftest_wait(unsigned long long* status, DevStatus* st) {
  lookback_warp(status, 1, 0, st);
}

__global__ void k_set_nstep(DevStatus* st, long long nstep) {
  st->w[ST_IDORDER] = 0;
  st->w[ST_NSTEP_LO] = (int)(unsigned)(nstep & 0xffffffffll);
  st->w[ST_NSTEP_HI] = (int)(nstep >> 32);
  st->w[ST_STEPS] = 0;
  st->w[ST_ERR] = 0;
}

__global__ void k_iota(int n, int* __restrict__ v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = i;
}

__global__ void k_default_vel(Geo g, int n, const double* __restrict__ x, const InstGeo* __restrict__ ig,
                              const int* __restrict__ inst, double* __restrict__ u,
                              double* __restrict__ w, bool du, bool dw) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const InstGeo& I = ig[inst[i]];
  const double gdot = I.gdot;
  const double y = x[n + i];
  if (g.wave) {
    // U_inf and Omega_inf of the wave of Eq. 17 at the centre
    double sn, cs;
    sincos(I.wave_k * y, &sn, &cs);
    if (du) { u[i] = gdot * y + g.wave_amp * sn; u[n + i] = 0.0; u[2 * n + i] = 0.0; }
    if (dw) { w[i] = 0.0; w[n + i] = 0.0; w[2 * n + i] = -0.5 * (gdot + g.wave_amp * I.wave_k * cs); }
    return;
  }
  if (du) { u[i] = gdot * y; u[n + i] = 0.0; u[2 * n + i] = 0.0; }
  if (dw) { w[i] = 0.0; w[n + i] = 0.0; w[2 * n + i] = -0.5 * gdot; }
}

// Attach the stretch of a given history (sorted keys) to a freshly built list
// (and the rolling stretch, xr, when the list keeps one; NULL: zero).
__global__ void k_attach_history(Geo g, StateBuf s, ListBuf L, const long long* __restrict__ keys,
                                 const double* __restrict__ xi, const double* __restrict__ xr, int k) {
  const int n = g.n;
  const int P = (int)min((int64_t)L.start[n], g.pcap);   // the host grew pcap to the list first
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (L.start[mid] <= p) lo = mid; else hi = mid;
    }
    const int j = L.list[(int64_t)lo * g.Ms + (p - L.start[lo])];
    const long long a = s.id[lo], b = s.id[j];
    const long long key = a < b ? (a << 32) | b : (b << 32) | a;
    int l = 0, r = k - 1, f = -1;
    while (l <= r) {
      int m = (l + r) >> 1;
      if (keys[m] == key) { f = m; break; }
      if (keys[m] < key) l = m + 1; else r = m - 1;
    }
    const bool mixed = g.precision == DSS_MIXED;
    Xi4 v{0.0, 0.0, 0.0, 0.0}, vr{0.0, 0.0, 0.0, 0.0};
    if (f >= 0) {
      v = xi_record(xi[3 * (int64_t)f], xi[3 * (int64_t)f + 1], xi[3 * (int64_t)f + 2], true, mixed);
      if (xr) {
        vr = xi_record(xr[3 * (int64_t)f], xr[3 * (int64_t)f + 1], xr[3 * (int64_t)f + 2], true, mixed);
        vr.w = 0.0;   // the rolling record carries no flag
      }
    }
    L.xi[p] = v;
    if (L.xr) L.xr[p] = vr;
  }
}

__global__ void k_history_out(Geo g, ListBuf L, long long* __restrict__ keys,
                              double* __restrict__ xi, double* __restrict__ xr, int* __restrict__ counter,
                              int cap) {
  const int n = g.n;
  const int P = (int)min((int64_t)L.start[n], g.pcap);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    const Xi4 v = L.xi[p];
    if (!xi_flag(v)) continue;
    int lo = 0, hi = n;
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (L.start[mid] <= p) lo = mid; else hi = mid;
    }
    const int j = L.list[(int64_t)lo * g.Ms + (p - L.start[lo])];
    const long long a = L.id_of_slot[lo], b = L.id_of_slot[j];
    int q = atomicAdd(counter, 1);
    if (q < cap) {
      keys[q] = a < b ? (a << 32) | b : (b << 32) | a;
      const bool mixed = g.precision == DSS_MIXED;
      double c[3];
      xi_components(v, mixed, c);
      xi[3 * (int64_t)q] = c[0];
      xi[3 * (int64_t)q + 1] = c[1];
      xi[3 * (int64_t)q + 2] = c[2];
      xi_components(L.xr ? L.xr[p] : Xi4{0.0, 0.0, 0.0, 0.0}, mixed, c);
      xr[3 * (int64_t)q] = c[0];
      xr[3 * (int64_t)q + 1] = c[1];
      xr[3 * (int64_t)q + 2] = c[2];
    }
  }
}

// The operation sequences.  stbuf/list indices follow the handle's
// committed (cur, hist) pair; "w" is the scratch side.
void seq_sort_enum(dss_handle* h, bool predict, int adv) {
  const int w = 1 - h->cur;
  launch_sort(h, predict, h->cur, w);
  launch_enumerate(h, w, 1 - h->hist, adv);
}

void seq_step(dss_handle* h) {
  const int w = 1 - h->cur;
  seq_sort_enum(h, true, 1);
  launch_forces(h, w, 1 - h->hist, h->hist, 1, G_STEP, nullptr, nullptr);
}

int capture_step(dss_handle* h, int key) {
  cudaGraph_t graph;
  CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  h->capturing = true;
  seq_step(h);
  h->capturing = false;
  cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
  if (e != cudaSuccess) return DSS_ERR_CUDA;
  e = cudaGraphInstantiate(&h->step_graph[key], graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return DSS_ERR_CUDA;
  h->graph_ok[key] = true;
  return DSS_OK;
}

// DSS_MULTI_STEPS steps in one graph, starting with the buffers in the
// roles (cur, hist) of key; each step's kernels skip after an earlier
// failure exactly as in separate launches.
int capture_multi(dss_handle* h, int key) {
  const int cur0 = h->cur, hist0 = h->hist;
  h->cur = key >> 1;
  h->hist = key & 1;
  cudaGraph_t graph;
  CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  h->capturing = true;
  for (int k = 0; k < DSS_MULTI_STEPS; ++k) {
    seq_step(h);
    h->cur = 1 - h->cur;
    h->hist = 1 - h->hist;
  }
  h->capturing = false;
  h->cur = cur0;
  h->hist = hist0;
  cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
  if (e != cudaSuccess) return DSS_ERR_CUDA;
  e = cudaGraphInstantiate(&h->multi_graph[key], graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return DSS_ERR_CUDA;
  h->multi_ok[key] = true;
  return DSS_OK;
}

int accumulate_profile(dss_handle* h) {
  CK(cudaStreamSynchronize(h->stream));
  for (int k = 0; k < DSS_PROF_KERNELS; ++k) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->prof_ev[k], h->prof_ev[k + 1]));
    h->prof_ms[k] += ms;
  }
  h->prof_count += 1;
  return DSS_OK;
}

int status_error(dss_handle* h) {
  int e = h->status_host->w[ST_ERR];
  return e ? e : DSS_OK;
}

// Outside a step (where the pair kernel reports an overflow and the step is
// replayed), a list just built may hold more pairs than the pair buffers fit:
// grow them before anything writes per-pair data.  Waits for the list and
// returns the status of the kernels before it.
int ensure_pair_capacity(dss_handle* h, int list) {
  int r = sync_status(h);
  if (r) return r;
  if ((r = status_error(h))) { clear_err(h); return r; }
  int P = 0;
  CK(cudaMemcpyAsync(&P, h->lb[list].start + h->n, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (P > h->pcap) return alloc_pair_buffers(h, (int64_t)(P * 1.25) + 1024, true);
  return DSS_OK;
}


// Cell grid of every instance (Sec. II A: cells of edge >= the largest
// interaction range, 2 a_max + delta_max); cells are numbered instance-major.
// Interaction range beyond contact of the largest pair a particle of radius a
// can own (partners no larger than itself).
double dmax_of(const dss_params& p, double a) {
  const double dl = p.lub_cutoff_mode == 1 ? p.delta_lub * p.a0 : p.delta_lub * a;
  const double de = echem_range(&p);
  return de > dl ? de : dl;
}

// Size class of a particle of radius a on cells of edge cs: the particle's own
// pairs reach at most (class + 1) cells.  Rounded up by a relative 1e-9 so
// that rounding never shortens a reach.
int class_of(const dss_params& p, double a, double cs) {
  const double need = (2.0 * a + dmax_of(p, a)) * (1.0 + 1e-9) / cs;
  int c = (int)std::ceil(need) - 1;
  return c < 0 ? 0 : c;
}

// Cell grid of every instance (Sec. II A).  Mode 0: cells of edge >= the
// largest interaction range, 2 a_max + delta_max, one cell list, the 27-cell
// (half: 14-cell) stencil.  Mode 1 (highly polydisperse suspensions): smaller
// cells, particles binned by size class; a class-c particle searches its own
// class in the half stencil of reach rtab[c][c] and each smaller class in the
// full stencil of reach rtab[c][c2].  Bins are numbered instance-major, then
// class, then cell.
int geometry(dss_handle* h) {
  Geo& g = h->g;
  const dss_params& p = h->p;
  double range = 2.0 * h->a_max + dmax_of(p, h->a_max);
  double cmin = range * (1.0 + 1e-9) + 1e-12;
  double cs = cmin;
  int C = 1;
  if (p.cell_mode == 1) {
    const double rmin = (2.0 * h->a_min + dmax_of(p, h->a_min)) * (1.0 + 1e-9) + 1e-12;
    cs = p.cell_size > 0.0 ? p.cell_size : std::max(rmin, cmin / 4.0);
    if (cs < rmin) return DSS_ERR_ARG;
    C = class_of(p, h->a_max, cs) + 1;
    if (C > 8) return DSS_ERR_ARG;
  } else if (p.cell_size > 0.0) {
    if (p.cell_size < cmin) return DSS_ERR_ARG;
    cs = p.cell_size;
  }
  // reach table from the largest radius of each class
  double A[8];
  const double de = echem_range(&p);
  for (int c = 0; c < C; ++c) {
    // the largest radius a with 2 a + dmax(a) <= (c + 1) cs / (1 + 1e-9)
    const double X = (c + 1) * cs / (1.0 + 1e-9);
    A[c] = p.lub_cutoff_mode == 1 ? (X - std::max(p.delta_lub * p.a0, de)) * 0.5
                                  : std::min(X / (2.0 + p.delta_lub), (X - de) * 0.5);
  }
  if (C == 1) A[0] = h->a_max;
  int reach = 1;
  memset(g.rtab, 0, sizeof(g.rtab));
  for (int c = 0; c < C; ++c)
    for (int c2 = 0; c2 <= c; ++c2) {
      const double dpair = std::max(de, p.lub_cutoff_mode == 1 ? p.delta_lub * p.a0
                                                                 : p.delta_lub * 0.5 * (A[c] + A[c2]));
      // A[] already carries the 1e-9 margin of class_of: the ranges of the
      // class pair stay below (A + A2 + dpair), so no further margin
      int R = (int)std::ceil((A[c] + A[c2] + dpair) / cs);
      if (c2 == c) R = std::min(R, c + 1);
      if (C == 1) R = 1;
      if (R < 1) R = 1;
      g.rtab[c][c2] = (unsigned char)R;
      reach = std::max(reach, R);
    }
  g.nclass = C;
  g.reach = reach;
  int64_t cells = 0, pos = 0;
  for (int k = 0; k < h->K; ++k) {
    InstGeo& I = h->ig_host[k];
    const double* L = h->inst_box + 3 * k;
    for (int d = 0; d < 3; ++d) {
      I.L[d] = L[d];
      I.halfL[d] = 0.5 * L[d];
      I.nc[d] = (int)std::floor(L[d] / cs);
      if (I.nc[d] < 1) I.nc[d] = 1;
      I.cs[d] = L[d] / I.nc[d];
      I.inv_cs[d] = 1.0 / I.cs[d];
      I.halfLf[d] = (float)(0.5 * L[d]) * (1.0f - 1e-5f);
      I.csf[d] = (float)I.cs[d];
      I.cs_lo[d] = (float)(I.cs[d] - (double)I.csf[d]);
      I.invL[d] = 1.0 / L[d];
    }
    // the stencil may not meet itself across the periodic box
    if (I.nc[0] < 2 * reach + 2 || I.nc[1] < 2 * reach + 1 || I.nc[2] < 2 * reach + 1) return DSS_ERR_BOX;
    if (I.nc[0] > 1023 || I.nc[1] > 1023 || I.nc[2] > 1023) return DSS_ERR_ARG;   // packed coords
    const int64_t nck = (int64_t)I.nc[0] * I.nc[1] * I.nc[2];
    if (cells + C * nck > (int64_t)2000000000) return DSS_ERR_ARG;
    I.cell_base = (int)cells;
    I.ncell_layer = (int)nck;
    I.ncell = (int)(C * nck);
    cells += C * nck;
    const double csmax = std::max(I.cs[0], std::max(I.cs[1], I.cs[2]));
    I.r2_margin = (float)(1e-4 * csmax * csmax);
    for (int d = 0; d < 3; ++d) I.inv_csf[d] = (float)I.inv_cs[d];
    I.p_begin = (int)pos;
    pos += h->inst_n[k];
    I.p_end = (int)pos;
    I.gdot = h->inst_gdot[k];
    I.gn = h->inst_gn[k];
    I.gdot_f = (float)I.gdot;
    I.gn_f = (float)I.gn;
    // the wave of Eq. 17 spans wave_n periods of this instance's L_y
    I.wave_k = g.wave ? 2.0 * DSS_PI * (double)p.wave_n / I.L[1] : 0.0;
    I.faxen_c = I.wave_k * I.wave_k / 6.0;
  }
  g.ncell = (int)cells;
  h->cell_edge = cs;
  int M = p.capacity_M > 0 ? p.capacity_M : dss_capacity_estimate(h->a_min, h->a_max, p.a0);
  if (p.capacity_M <= 0 && de > 0.0) {
    // with electro-chemical forces pairs reach beyond the 2 a0 shell of
    // Sec. II A: the shell then spans every partner within the range
    const double outer = h->a_max + std::max(2.0 * p.a0, 2.0 * h->a_min + de);
    const double v = (outer * outer * outer - h->a_max * h->a_max * h->a_max) /
                     (h->a_min * h->a_min * h->a_min);
    M = v < 2e9 ? std::max(M, (int)std::ceil(v)) : -1;
  }
  if (M <= 0) return DSS_ERR_ARG;
  g.M = M;
  g.Ms = (M + 3) & ~3;   // row stride: rows start on 16-byte boundaries
  return DSS_OK;
}

bool valid_params(const dss_params* p) {
  return (p->kn >= 0) && (p->kt > 0) && (p->gamma_n >= 0) && (p->mu >= 0) && (p->eta0 >= 0) &&
         (p->rho > 0) && (p->delta_lub >= 0) && (p->lub_eps > 0) && (p->a0 > 0) && (p->dt > 0) &&
         std::isfinite(p->shear_rate) && (p->lub_cutoff_mode == 0 || p->lub_cutoff_mode == 1) &&
         (p->precision == DSS_FP64 || p->precision == DSS_MIXED) &&
         (p->lub_taper >= 0.0 && p->lub_taper < 1.0) && (p->cell_mode == 0 || p->cell_mode == 1) &&
         (p->f_er >= 0.0 && std::isfinite(p->f_er)) && (p->hamaker >= 0.0 && std::isfinite(p->hamaker)) &&
         (!(p->f_er > 0.0) || (p->lambda_d > 0.0 && std::isfinite(p->lambda_d))) &&
         (!(p->hamaker > 0.0) || (p->vdw_eps > 0.0 && std::isfinite(p->vdw_eps))) &&
         std::isfinite(p->wave_amp) && (p->wave_n >= 0) && (p->k_r >= 0.0 && std::isfinite(p->k_r));
}

// Common constructor: K instances of n[k] particles in boxes box[3k..3k+2]
// with shear rates gdot[k] and normal dashpots gn[k].
int create_handle(dss_handle** out, const dss_params* p, int K, const int64_t* n, const double* box,
                  const double* gdot, const double* gn, void* cuda_stream) {
  dss_handle* h = new dss_handle();
  memset((void*)h, 0, sizeof(dss_handle));
  h->p = *p;
  h->K = K;
  h->ig_host = new InstGeo[K];
  memset((void*)h->ig_host, 0, sizeof(InstGeo) * K);
  h->inst_box = new double[3 * K];
  h->inst_gdot = new double[K];
  h->inst_gn = new double[K];
  h->inst_n = new int64_t[K];
  int64_t total = 0;
  for (int k = 0; k < K; ++k) {
    for (int d = 0; d < 3; ++d) h->inst_box[3 * k + d] = box[3 * k + d];
    h->inst_gdot[k] = gdot[k];
    h->inst_gn[k] = gn[k];
    h->inst_n[k] = n[k];
    total += n[k];
  }
  h->n = total;
  h->user_stream = (cudaStream_t)cuda_stream;
  if (cudaGetDevice(&h->device) != cudaSuccess) { dss_destroy(h); return DSS_ERR_CUDA; }
  if (cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess || h->sms < 1)
    h->sms = 1;
  // work runs on the caller's stream; for the legacy default stream (NULL),
  // where graph capture is not allowed, on a stream of our own ordered after it
  if (cuda_stream) {
    h->stream = (cudaStream_t)cuda_stream;
    h->own_stream = false;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      dss_destroy(h);
      return DSS_ERR_CUDA;
    }
    h->own_stream = true;
  }
  if (cudaEventCreateWithFlags(&h->ev_enter, cudaEventDisableTiming) != cudaSuccess) {
    dss_destroy(h);
    return DSS_ERR_CUDA;
  }
  if (cudaMalloc((void**)&h->status, sizeof(DevStatus)) != cudaSuccess) {
    dss_destroy(h);
    return DSS_ERR_CUDA;
  }
  if (cudaMallocHost((void**)&h->status_host, sizeof(DevStatus)) != cudaSuccess) {
    dss_destroy(h);
    return DSS_ERR_CUDA;
  }
  cudaMemsetAsync(h->status, 0, sizeof(DevStatus), h->stream);
  Geo& g = h->g;
  g.n = (int)total;
  g.K = K;
  g.kn = p->kn; g.kt = p->kt; g.mu = p->mu;
  g.eta0 = p->eta0; g.rho = p->rho;
  g.delta = p->delta_lub; g.eps = p->lub_eps; g.a0 = p->a0;
  g.mode = p->lub_cutoff_mode; g.precision = p->precision;
  g.dt = p->dt;
  g.hdt = 0.5 * p->dt;
  g.hdt2 = g.hdt * p->dt;
  g.k6 = 6.0 * DSS_PI * p->eta0;
  g.k8 = 8.0 * DSS_PI * p->eta0;
  g.f.kn = (float)p->kn;
  g.f.kt = (float)p->kt;
  g.f.mu_kt = (float)(p->mu / p->kt);
  g.f.dt = (float)p->dt;
  g.f.eps = (float)p->lub_eps;
  g.f.k6 = (float)g.k6;
  g.f.k8 = (float)g.k8;
  g.f.mass_c = (float)(4.0 / 3.0 * DSS_PI * p->rho);
  g.taper = p->lub_taper;
  g.f.taper = (float)p->lub_taper;
  g.f.delta = (float)p->delta_lub;
  g.f.delta_a0 = (float)(p->delta_lub * p->a0);
  g.f_er = p->f_er;
  g.lambda_d = p->lambda_d;
  g.hamaker = p->hamaker;
  g.vdw_eps = p->vdw_eps;
  g.de = echem_range(p);
  g.f.f_er = (float)(p->f_er / p->a0);   // F_ER / a0
  g.f.inv_lambda = p->f_er > 0.0 ? (float)(1.0 / p->lambda_d) : 0.0f;
  g.f.range_r = (float)(20.0 * p->lambda_d);
  g.f.hamaker12 = (float)(p->hamaker / 12.0);
  g.f.vdw_eps = (float)p->vdw_eps;
  g.f.range_a = (float)(4.0 * p->a0);
  g.wave = (p->wave_amp != 0.0 && p->wave_n > 0) ? 1 : 0;
  g.wave_amp = g.wave ? p->wave_amp : 0.0;
  g.k_r = p->k_r;
  g.f.k_r = (float)p->k_r;
  g.f.mu_kr = p->k_r > 0.0 ? (float)(p->mu / p->k_r) : 0.0f;
  *out = h;
  return DSS_OK;
}

}  // namespace

// Surface-distance range of the electro-chemical forces (Fig. 3): 20 lambda_D
// for the repulsion, 4 a0 for the attraction, the larger of the active ones;
// 0 when both are off.
double echem_range(const dss_params* p) {
  double r = 0.0;
  if (p->f_er > 0.0 && 20.0 * p->lambda_d > r) r = 20.0 * p->lambda_d;
  if (p->hamaker > 0.0 && 4.0 * p->a0 > r) r = 4.0 * p->a0;
  return r;
}

void prof_mark(dss_handle* h, int k) {
  if (!h->profiling) return;
  if (h->capturing)
    cudaEventRecordWithFlags(h->prof_ev[k], h->stream, cudaEventRecordExternal);
  else
    cudaEventRecord(h->prof_ev[k], h->stream);
}

// Runs the body of an entry point so that no C++ exception crosses the C ABI:
// a failed host allocation returns DSS_ERR_NOMEM, anything else
// DSS_ERR_INTERNAL.
template <class F>
static int guard(F&& body) {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    return DSS_ERR_NOMEM;
  } catch (...) {
    return DSS_ERR_INTERNAL;
  }
}

extern "C" {

int32_t dss_capacity_estimate(double a_min, double a_max, double a0) {
  if (!(a_min > 0.0) || !(a_max >= a_min) || !(a0 > 0.0)) return -1;
  double outer = a_max + 2.0 * a0;
  double shell = outer * outer * outer - a_max * a_max * a_max;
  double v = shell / (a_min * a_min * a_min);
  double c = std::ceil(v - 1e-9 * v);
  if (c < 1.0) c = 1.0;
  if (c > 1e8) return -1;
  return (int32_t)c;
}

const char* dss_strerror(int code) {
  switch (code) {
    case DSS_OK: return "ok";
    case DSS_ERR_ARG: return "invalid argument";
    case DSS_ERR_BOX: return "box too small for the cell grid (need >= 4 cells along x, >= 3 along y, z)";
    case DSS_ERR_CAPACITY: return "neighbour-list capacity exceeded";
    case DSS_ERR_NONFINITE: return "non-finite force or state";
    case DSS_ERR_UNSTABLE: return "time step above the stability estimate";
    case DSS_ERR_CUDA: return "CUDA runtime error";
    case DSS_ERR_TIMEOUT: return "bounded device wait gave up";
    case DSS_ERR_STATE: return "call out of order (no state loaded)";
    case DSS_ERR_INTERNAL: return "internal consistency check failed";
    case DSS_ERR_NOMEM: return "host memory allocation failed";
    case DSS_ERR_SCRATCH_LIMIT:
      return "problem too large for the fixed scratch array of dss_pairs_noalloc "
             "(needs n + 3*cells + 17 <= DSS_NOALLOC_SCRATCH_INTS words)";
    default: return "unknown error";
  }
}

int dss_create(dss_handle** out, const dss_params* p, int64_t n, const double box[3],
               void* cuda_stream) {
  return guard([&]() -> int {
    if (!out || !p || !box || n < 2 || n > (int64_t)1 << 30) return DSS_ERR_ARG;
    *out = nullptr;
    for (int d = 0; d < 3; ++d)
      if (!(box[d] > 0.0) || !std::isfinite(box[d])) return DSS_ERR_ARG;
    if (!valid_params(p)) return DSS_ERR_ARG;
    const double gd = p->shear_rate, gn = p->gamma_n;
    return create_handle(out, p, 1, &n, box, &gd, &gn, cuda_stream);
  });
}

int dss_batch_create(dss_handle** out, const dss_params* p, int32_t K, const int64_t* n,
                     const double* box, const double* shear_rate, const double* gamma_n,
                     void* cuda_stream) {
  return guard([&]() -> int {
    if (!out || !p || !n || !box || !shear_rate || K < 1 || K > (1 << 20)) return DSS_ERR_ARG;
    *out = nullptr;
    if (!valid_params(p)) return DSS_ERR_ARG;
    int64_t total = 0;
    for (int k = 0; k < K; ++k) {
      // a pair block (256 owners) spans at most two instances
      if (n[k] < (K > 1 ? DSS_BATCH_MIN_N : 2)) return DSS_ERR_ARG;
      total += n[k];
      if (total > (int64_t)1 << 30) return DSS_ERR_ARG;
      for (int d = 0; d < 3; ++d)
        if (!(box[3 * k + d] > 0.0) || !std::isfinite(box[3 * k + d])) return DSS_ERR_ARG;
      if (!std::isfinite(shear_rate[k])) return DSS_ERR_ARG;
      if (gamma_n && !(gamma_n[k] >= 0.0 && std::isfinite(gamma_n[k]))) return DSS_ERR_ARG;
    }
    std::vector<double> gn(K);
    for (int k = 0; k < K; ++k) gn[k] = gamma_n ? gamma_n[k] : p->gamma_n;
    return create_handle(out, p, K, n, box, shear_rate, gn.data(), cuda_stream);
  });
}

int dss_set_state(dss_handle* h, const double* x, const double* a, const int32_t* ids,
                  const double* u, const double* w, const double* alpha_lin,
                  const double* alpha_ang, int64_t nstep) {
  return guard([&]() -> int {
    if (!h || !x || !a || nstep < 0) return DSS_ERR_ARG;
    if ((alpha_lin == nullptr) != (alpha_ang == nullptr)) return DSS_ERR_ARG;
    ENTER(h);
    const int64_t n = h->n;
    // host-side validation of radii, positions and ids
    std::vector<double> ha(n), hx(3 * n);
    CK(cudaMemcpy(ha.data(), a, sizeof(double) * n, cudaMemcpyDefault));
    CK(cudaMemcpy(hx.data(), x, sizeof(double) * 3 * n, cudaMemcpyDefault));
    double amin = INFINITY, amax = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      if (!(ha[i] > 0.0) || !std::isfinite(ha[i])) return DSS_ERR_ARG;
      amin = std::min(amin, ha[i]);
      amax = std::max(amax, ha[i]);
    }
    // instance of each index (instance-major); positions inside their box
    std::vector<int32_t> imap(n);
    std::vector<int64_t> ibeg(h->K + 1, 0);
    for (int k = 0; k < h->K; ++k) {
      ibeg[k + 1] = ibeg[k] + h->inst_n[k];
      for (int64_t i = ibeg[k]; i < ibeg[k + 1]; ++i) imap[i] = k;
    }
    for (int d = 0; d < 3; ++d)
      for (int64_t i = 0; i < n; ++i) {
        double v = hx[d * n + i];
        if (!(v >= 0.0 && v < h->inst_box[3 * imap[i] + d])) return DSS_ERR_ARG;
      }
    std::vector<int32_t> hid(n);
    if (ids) {
      // ids of instance k are a permutation of its own index range
      CK(cudaMemcpy(hid.data(), ids, sizeof(int32_t) * n, cudaMemcpyDefault));
      std::vector<char> seen(n, 0);
      for (int64_t i = 0; i < n; ++i) {
        if (hid[i] < 0 || hid[i] >= n || seen[hid[i]] || imap[hid[i]] != imap[i]) return DSS_ERR_ARG;
        seen[hid[i]] = 1;
      }
    } else {
      for (int64_t i = 0; i < n; ++i) hid[i] = (int32_t)i;
    }
    if (!h->sized || amax > h->a_max || amin < h->a_min) {
      if (h->sized) free_buffers(h);
      drop_graphs(h);
      h->a_min = amin;
      h->a_max = amax;
      int r = geometry(h);
      if (r) return r;
      r = alloc_buffers(h);
      if (r) { free_buffers(h); return r; }
    }
    for (int k = 0; k < h->K; ++k) {
      double s3 = 0.0;
      for (int64_t i = ibeg[k]; i < ibeg[k + 1]; ++i) s3 += ha[i] * ha[i] * ha[i];
      h->ig_host[k].sumA3 = s3;
    }
    drop_graphs(h);
    h->cur = 0;
    h->hist = 0;
    h->mean_steps = 0;
    StateBuf& s = h->st[0];
    CK(cudaMemcpyAsync(h->ig, h->ig_host, sizeof(InstGeo) * h->K, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->inst_map, imap.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(s.inst, h->inst_map, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, h->stream));
    {
      // size classes (all 0 with one cell list), by index and by id
      std::vector<unsigned char> cu(n), cid(n);
      for (int64_t i = 0; i < n; ++i) {
        int c = h->g.nclass > 1 ? class_of(h->p, ha[i], h->cell_edge) : 0;
        if (c > h->g.nclass - 1) c = h->g.nclass - 1;
        cu[i] = (unsigned char)c;
        cid[hid[i]] = (unsigned char)c;
      }
      CK(cudaMemcpyAsync(s.cls, cu.data(), n, cudaMemcpyHostToDevice, h->stream));
      CK(cudaMemcpyAsync(h->cls_map, cid.data(), n, cudaMemcpyHostToDevice, h->stream));
      CK(cudaStreamSynchronize(h->stream));
    }
    CK(cudaMemsetAsync(h->sigma_sum, 0, 9 * sizeof(double) * h->K, h->stream));
    CK(cudaMemcpyAsync(s.x, hx.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(s.a, ha.data(), sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(s.id, hid.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemsetAsync(s.iy, 0, sizeof(int) * n, h->stream));
    h->marked = false;
    {
      std::vector<double> aid(n);
      for (int64_t i = 0; i < n; ++i) aid[hid[i]] = ha[i];
      CK(cudaMemcpyAsync(h->a_by_id, aid.data(), sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
      CK(cudaStreamSynchronize(h->stream));
    }
    if (u) CK(cudaMemcpyAsync(s.u, u, sizeof(double) * 3 * n, cudaMemcpyDefault, h->stream));
    if (w) CK(cudaMemcpyAsync(s.w, w, sizeof(double) * 3 * n, cudaMemcpyDefault, h->stream));
    const int nb = (int)((n + 255) / 256);
    if (!u || !w) k_default_vel<<<nb, 256, 0, h->stream>>>(h->g, (int)n, s.x, h->ig, s.inst, s.u, s.w, !u, !w);
    if (alpha_lin) {
      CK(cudaMemcpyAsync(s.al, alpha_lin, sizeof(double) * 3 * n, cudaMemcpyDefault, h->stream));
      CK(cudaMemcpyAsync(s.aw, alpha_ang, sizeof(double) * 3 * n, cudaMemcpyDefault, h->stream));
    }
    // empty history: no rows, identity id map
    for (int b = 0; b < 2; ++b) {
      CK(cudaMemsetAsync(h->lb[b].count, 0, sizeof(int) * n, h->stream));
      CK(cudaMemsetAsync(h->lb[b].start, 0, sizeof(int) * (n + 1), h->stream));
      k_iota<<<nb, 256, 0, h->stream>>>((int)n, h->lb[b].slot_of_id);
      k_iota<<<nb, 256, 0, h->stream>>>((int)n, h->lb[b].id_of_slot);
    }
    k_set_nstep<<<1, 1, 0, h->stream>>>(h->status, (long long)nstep);
    CK(cudaGetLastError());
    h->have_state = true;
    h->host_steps_done = 0;
    if (alpha_lin) {
      int r0 = sync_status(h);
      if (r0) return r0;
    }
    if (!alpha_lin) {
      // alpha^0 from one force evaluation at the initial state (empty history)
      seq_sort_enum(h, false, 0);
      h->cur = 1 - h->cur;
      int rc = ensure_pair_capacity(h, 1 - h->hist);
      if (rc) return rc;
      launch_forces(h, h->cur, 1 - h->hist, h->hist, 0, G_ACCEL, nullptr, nullptr);
      CK(cudaGetLastError());
      int r = sync_status(h);
      if (r) return r;
      if ((r = status_error(h))) { clear_err(h); return r; }
    }
    return DSS_OK;
  });
}

// The committed state out in id order (any of out[0..4] may be null):
// enqueued on the stream, not synchronised.
int get_state_enqueue(dss_handle* h, double* const out[5]) {
  const int n = (int)h->n;
  const StateBuf& s = h->st[h->cur];
  // device outputs are written in place by the scatter; host outputs go
  // through the staging area, then out by a coalesced copy kernel (mapped
  // pinned memory) or the copy engine (pageable memory)
  Dst5 direct, staged, views;
  for (int k = 0; k < 5; ++k) {
    direct.d[k] = staged.d[k] = views.d[k] = nullptr;
    if (!out[k]) continue;
    cudaPointerAttributes at;
    const bool is_dev = cudaPointerGetAttributes(&at, out[k]) == cudaSuccess && at.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    if (is_dev) {
      direct.d[k] = out[k];
    } else {
      staged.d[k] = h->stage + (size_t)k * 3 * n;
      views.d[k] = static_cast<double*>(const_cast<void*>(device_view(out[k])));
    }
  }
  Dst5 all = direct;
  for (int k = 0; k < 5; ++k)
    if (staged.d[k]) all.d[k] = staged.d[k];
  k_state_out<<<(n + 255) / 256, 256, 0, h->stream>>>(n, s, all);
  Dst5 src_c, dst_c;
  bool any_view = false;
  for (int k = 0; k < 5; ++k) {
    src_c.d[k] = dst_c.d[k] = nullptr;
    if (!staged.d[k]) continue;
    if (views.d[k]) {
      src_c.d[k] = staged.d[k];
      dst_c.d[k] = views.d[k];
      any_view = true;
    } else {
      CK(cudaMemcpyAsync(out[k], staged.d[k], sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, h->stream));
    }
  }
  if (any_view) k_copy5<<<std::min((3 * n + 255) / 256, 8 * h->sms), 256, 0, h->stream>>>(3 * (int64_t)n, src_c, dst_c);
  CK(cudaGetLastError());
  return DSS_OK;
}

int dss_get_state(dss_handle* h, double* x, double* u, double* w, double* alpha_lin,
                  double* alpha_ang) {
  return guard([&]() -> int {
    if (!h) return DSS_ERR_ARG;
    if (!h->have_state) return DSS_ERR_STATE;
    ENTER(h);
    double* const out[5] = {x, u, w, alpha_lin, alpha_ang};
    int r = get_state_enqueue(h, out);
    if (r) return r;
    CK(cudaStreamSynchronize(h->stream));
    return DSS_OK;
  });
}

int dss_neighbour_build(dss_handle* h) {
  if (!h) return DSS_ERR_ARG;
  if (!h->have_state) return DSS_ERR_STATE;
  ENTER(h);
  seq_sort_enum(h, false, 0);
  h->cur = 1 - h->cur;
  CK(cudaGetLastError());
  int r = sync_status(h);
  if (r) return r;
  if ((r = status_error(h))) { clear_err(h); return r; }
  return DSS_OK;
}

int dss_get_pairs(dss_handle* h, int64_t* lohi, int64_t cap, int64_t* count) {
  return guard([&]() -> int {
    if (!h || !count || cap < 0 || (cap > 0 && !lohi)) return DSS_ERR_ARG;
    if (!h->have_state) return DSS_ERR_STATE;
    ENTER(h);
    const int list = h->last_list;
    int P = 0;
    CK(cudaMemcpyAsync(&P, h->lb[list].start + h->n, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *count = P;
    if (P == 0 || cap == 0) return DSS_OK;
    // scratch: the partner-row buffer (n*M slots of >= 32 bytes >= 16 bytes per pair)
    long long* dev = (long long*)h->bw_rec;
    launch_pairs_out(h, list, dev);
    std::vector<long long> hp(2 * (size_t)P);
    CK(cudaMemcpyAsync(hp.data(), dev, sizeof(long long) * 2 * P, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    std::vector<std::pair<long long, long long>> v(P);
    for (int p = 0; p < P; ++p) v[p] = {hp[2 * p], hp[2 * p + 1]};
    std::sort(v.begin(), v.end());
    int64_t m = std::min<int64_t>(cap, P);
    for (int64_t p = 0; p < m; ++p) {
      lohi[2 * p] = v[p].first;
      lohi[2 * p + 1] = v[p].second;
    }
    return DSS_OK;
  });
}

int dss_force_eval(dss_handle* h, double* F, double* T) {
  if (!h) return DSS_ERR_ARG;
  if (!h->have_state) return DSS_ERR_STATE;
  ENTER(h);
  const int n = (int)h->n;
  seq_sort_enum(h, false, 0);
  h->cur = 1 - h->cur;
  int rc = ensure_pair_capacity(h, 1 - h->hist);
  if (rc) return rc;
  launch_forces(h, h->cur, 1 - h->hist, h->hist, 0, G_EVAL, F ? h->io3 : nullptr,
                T ? h->io3b : nullptr);
  CK(cudaGetLastError());
  if (F) CK(cudaMemcpyAsync(F, h->io3, sizeof(double) * 3 * n, cudaMemcpyDefault, h->stream));
  if (T) CK(cudaMemcpyAsync(T, h->io3b, sizeof(double) * 3 * n, cudaMemcpyDefault, h->stream));
  int r = sync_status(h);
  if (r) return r;
  if ((r = status_error(h))) { clear_err(h); return r; }
  return DSS_OK;
}

// The step graphs of `remaining` steps from the committed (cur, hist)
// state, enqueued (graphs captured first where missing), between the two
// step events.  StepRun keeps what the commit needs after the synchronisation.
struct StepRun {
  int steps0, cur0, hist0;
};

int step_launch(dss_handle* h, int64_t remaining, StepRun& run) {
  int r;
  if (!h->step_ev[0]) {
    CK(cudaEventCreate(&h->step_ev[0]));
    CK(cudaEventCreate(&h->step_ev[1]));
  }
  // the host mirror holds the counter of the last synchronisation; only
  // dss_step and dss_set_state change it, and both end synchronised
  run.steps0 = h->status_host->w[ST_STEPS];
  run.cur0 = h->cur;
  run.hist0 = h->hist;
  int c = run.cur0, hs = run.hist0;
  for (int64_t k = 0; k < remaining; ++k) {
    if (!h->graph_ok[c * 2 + hs]) {
      h->cur = c;
      h->hist = hs;
      r = capture_step(h, c * 2 + hs);
      if (r) return r;
    }
    c = 1 - c;
    hs = 1 - hs;
  }
  c = run.cur0;
  hs = run.hist0;
  // runs of DSS_MULTI_STEPS steps go out as one graph launch (not while
  // profiling, which times each step's kernels)
  const int64_t multi = h->profiling ? 0 : remaining / DSS_MULTI_STEPS;
  if (multi > 0 && !h->multi_ok[c * 2 + hs]) {
    r = capture_multi(h, c * 2 + hs);
    if (r) return r;
  }
  CK(cudaEventRecord(h->step_ev[0], h->stream));
  for (int64_t k = 0; k < multi; ++k) CK(cudaGraphLaunch(h->multi_graph[c * 2 + hs], h->stream));
  for (int64_t k = multi * DSS_MULTI_STEPS; k < remaining; ++k) {
    const int key = c * 2 + hs;
    CK(cudaGraphLaunch(h->step_graph[key], h->stream));
    if (h->profiling) {
      r = accumulate_profile(h);
      if (r) return r;
    }
    c = 1 - c;
    hs = 1 - hs;
  }
  CK(cudaEventRecord(h->step_ev[1], h->stream));
  return DSS_OK;
}

// After the synchronisation (the status mirror current): the steps the
// device committed, the buffer roles after them, the step time; returns the
// device error (0 when none).
int step_commit(dss_handle* h, const StepRun& run, int64_t& done) {
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, h->step_ev[0], h->step_ev[1]));
  h->last_step_ms += ms;
  done = h->status_host->w[ST_STEPS] - run.steps0;
  h->cur = (done & 1) ? 1 - run.cur0 : run.cur0;
  h->hist = (done & 1) ? 1 - run.hist0 : run.hist0;
  h->host_steps_done += done;
  h->mean_steps += done;
  if (done > 0) h->last_list = h->hist;
  return status_error(h);
}

// dss_step's loop from the committed state; the caller holds the handle.
int step_run(dss_handle* h, int64_t nsteps) {
  int64_t remaining = nsteps;
  int retries = 0;
  while (remaining > 0) {
    StepRun run;
    int r = step_launch(h, remaining, run);
    if (r) return r;
    r = sync_status(h);
    if (r) return r;
    int64_t done = 0;
    const int err = step_commit(h, run, done);
    remaining -= done;
    if (!err) break;
    clear_err(h);
    // a pair-capacity overflow is recovered by growing the pair buffers
    const int P = h->status_host->w[ST_NPAIRS];
    if (err == DSS_ERR_CAPACITY && P > h->pcap && retries < 4) {
      ++retries;
      r = alloc_pair_buffers(h, (int64_t)(P * 1.25) + 1024, true);
      if (r) return r;
      continue;
    }
    return err;
  }
  return DSS_OK;
}

int dss_step(dss_handle* h, int64_t nsteps) {
  return guard([&]() -> int {
    if (!h || nsteps < 0) return DSS_ERR_ARG;
    if (!h->have_state) return DSS_ERR_STATE;
    ENTER(h);
    h->last_step_ms = 0.0;
    return step_run(h, nsteps);
  });
}

int load_state_enqueue(dss_handle* h, const double* const in[5]);

int dss_step_io(dss_handle* h, const double* const in[5], int64_t nsteps, double* const out[5],
                double sigma[9]) {
  return guard([&]() -> int {
    if (!h || !in || nsteps < 0) return DSS_ERR_ARG;
    for (int k = 0; k < 5; ++k)
      if (!in[k]) return DSS_ERR_ARG;
    if (!h->have_state) return DSS_ERR_STATE;
    ENTER(h);
    h->last_step_ms = 0.0;
    int r = load_state_enqueue(h, in);
    if (r) return r;
    double* const none[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    double* const* dst = out ? out : none;
    StepRun run;
    int64_t done = 0;
    if (nsteps > 0) {
      r = step_launch(h, nsteps, run);
      if (r) return r;
    }
    // the state after the steps, as the buffer roles will be once they are
    // all committed, and the stress: enqueued behind the step graphs (the
    // commit below sets the roles from what the device did)
    if (nsteps > 0) h->cur = (nsteps & 1) ? 1 - run.cur0 : run.cur0;
    r = get_state_enqueue(h, dst);
    if (r) return r;
    if (sigma) CK(cudaMemcpyAsync(sigma, h->sigma, 9 * sizeof(double), cudaMemcpyDefault, h->stream));
    r = sync_status(h);
    if (r) return r;
    if (nsteps == 0) return DSS_OK;
    const int err = step_commit(h, run, done);
    if (!err && done == nsteps) return DSS_OK;
    // a step did not commit (what was copied out is not the final state):
    // finish as dss_step would, then read the state and the stress again
    if (err) {
      clear_err(h);
      const int P = h->status_host->w[ST_NPAIRS];
      if (err != DSS_ERR_CAPACITY || P <= h->pcap) return err;
      r = alloc_pair_buffers(h, (int64_t)(P * 1.25) + 1024, true);
      if (r) return r;
    }
    r = step_run(h, nsteps - done);
    if (r) return r;
    r = get_state_enqueue(h, dst);
    if (r) return r;
    if (sigma) CK(cudaMemcpyAsync(sigma, h->sigma, 9 * sizeof(double), cudaMemcpyDefault, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return DSS_OK;
  });
}

int dss_stress(dss_handle* h, double sigma[9]) {
  if (!h || !sigma) return DSS_ERR_ARG;
  if (!h->have_state) return DSS_ERR_STATE;
  ENTER(h);
  CK(cudaMemcpyAsync(sigma, h->sigma, 9 * sizeof(double), cudaMemcpyDefault, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return DSS_OK;
}

int dss_batch_stress(dss_handle* h, double* sigma, double* sigma_mean, int64_t* steps, int reset) {
  return guard([&]() -> int {
    if (!h) return DSS_ERR_ARG;
    if (!h->have_state) return DSS_ERR_STATE;
    ENTER(h);
    const size_t b = 9 * sizeof(double) * h->K;
    if (sigma) CK(cudaMemcpyAsync(sigma, h->sigma, b, cudaMemcpyDefault, h->stream));
    if (sigma_mean) {
      std::vector<double> sum(9 * (size_t)h->K);
      CK(cudaMemcpyAsync(sum.data(), h->sigma_sum, b, cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      const double c = h->mean_steps > 0 ? 1.0 / (double)h->mean_steps : 0.0;
      for (auto& v : sum) v *= c;
      CK(cudaMemcpyAsync(sigma_mean, sum.data(), b, cudaMemcpyDefault, h->stream));
    }
    if (steps) *steps = h->mean_steps;
    if (reset) {
      CK(cudaMemsetAsync(h->sigma_sum, 0, b, h->stream));
      h->mean_steps = 0;
    }
    CK(cudaStreamSynchronize(h->stream));
    return DSS_OK;
  });
}

int32_t dss_batch_size(const dss_handle* h) { return h ? h->K : 0; }

int dss_rheology(dss_handle* h, int mean, double* out) {
  return guard([&]() -> int {
    if (!h || !out) return DSS_ERR_ARG;
    if (!h->have_state) return DSS_ERR_STATE;
    const int K = h->K;
    std::vector<double> S(9 * (size_t)K), r(6 * (size_t)K);
    int rc = mean ? dss_batch_stress(h, nullptr, S.data(), nullptr, 0) : dss_batch_stress(h, S.data(), nullptr, nullptr, 0);
    if (rc) return rc;
    for (int k = 0; k < K; ++k) {
      const double* s = &S[9 * (size_t)k];
      const double g = h->p.eta0 * h->inst_gdot[k];
      if (!(g != 0.0)) return DSS_ERR_ARG;
      const double pi = -(s[0] + s[4] + s[8]) / 3.0;
      double* o = &r[6 * (size_t)k];
      o[0] = s[1];
      o[1] = s[0] - s[4];
      o[2] = s[4] - s[8];
      o[3] = pi;
      o[4] = s[1] / g;
      o[5] = pi / g;
    }
    CK(cudaMemcpy(out, r.data(), sizeof(double) * r.size(), cudaMemcpyDefault));
    return DSS_OK;
  });
}

int dss_get_images(dss_handle* h, int32_t* iy) {
  if (!h || !iy) return DSS_ERR_ARG;
  if (!h->have_state) return DSS_ERR_STATE;
  ENTER(h);
  launch_images_out(h, h->io_id);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(iy, h->io_id, sizeof(int32_t) * h->n, cudaMemcpyDefault, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return DSS_OK;
}

int dss_dispersion_mark(dss_handle* h) {
  if (!h) return DSS_ERR_ARG;
  if (!h->have_state) return DSS_ERR_STATE;
  ENTER(h);
  if (!h->mark) {
    int r = dalloc(h, &h->mark, 2 * (size_t)h->n);
    if (r) return r;
  }
  launch_mark(h);
  CK(cudaGetLastError());
  int r = sync_status(h);
  if (r) return r;
  h->mark_nstep = (int64_t)(uint32_t)h->status_host->w[ST_NSTEP_LO] |
                  ((int64_t)h->status_host->w[ST_NSTEP_HI] << 32);
  h->marked = true;
  return DSS_OK;
}

int dss_phi_profile(dss_handle* h, int32_t nbins, double a_split, double* out) {
  return guard([&]() -> int {
    if (!h || !out || nbins < 1 || nbins > (1 << 20) || !std::isfinite(a_split)) return DSS_ERR_ARG;
    if (!h->have_state) return DSS_ERR_STATE;
    ENTER(h);
    const int K = h->K;
    // per instance: the integer unit 2^-62 of its solid volume, so that no
    // slab sum can overflow
    std::vector<double> unit(K);
    for (int k = 0; k < K; ++k) {
      const double vol = 4.0 / 3.0 * DSS_PI * h->ig_host[k].sumA3;
      unit[k] = std::ldexp(vol > 0.0 ? vol : 1.0, -62);
    }
    const size_t nacc = (size_t)K * 2 * nbins;
    double* du = nullptr;
    unsigned long long* acc = nullptr;
    CK(cudaMalloc((void**)&du, sizeof(double) * K));
    if (cudaMalloc((void**)&acc, sizeof(unsigned long long) * nacc) != cudaSuccess) {
      cudaFree(du);
      return DSS_ERR_CUDA;
    }
    std::vector<unsigned long long> hacc(nacc);
    cudaError_t e = cudaMemcpyAsync(du, unit.data(), sizeof(double) * K, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * nacc, h->stream);
    if (e == cudaSuccess) {
      launch_phi_profile(h, nbins, a_split, du, acc);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hacc.data(), acc, sizeof(unsigned long long) * nacc, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(du);
    cudaFree(acc);
    if (e != cudaSuccess) return DSS_ERR_CUDA;
    std::vector<double> r(nacc);
    for (int k = 0; k < K; ++k) {
      const double* L = h->inst_box + 3 * k;
      const double slab = L[0] * L[2] * (L[1] / nbins);
      for (int q = 0; q < 2 * nbins; ++q)
        r[(size_t)k * 2 * nbins + q] = (double)hacc[(size_t)k * 2 * nbins + q] * unit[k] / slab;
    }
    CK(cudaMemcpy(out, r.data(), sizeof(double) * nacc, cudaMemcpyDefault));
    return DSS_OK;
  });
}

int dss_dispersion(dss_handle* h, double* out) {
  return guard([&]() -> int {
    if (!h || !out) return DSS_ERR_ARG;
    if (!h->have_state || !h->marked || !h->mark) return DSS_ERR_STATE;
    ENTER(h);
    const int K = h->K;
    launch_dispersion(h, h->io3);
    CK(cudaGetLastError());
    std::vector<double> sums(3 * (size_t)K), r(3 * (size_t)K);
    CK(cudaMemcpyAsync(sums.data(), h->io3, sizeof(double) * sums.size(), cudaMemcpyDeviceToHost, h->stream));
    int rc = sync_status(h);
    if (rc) return rc;
    const int64_t ns = (int64_t)(uint32_t)h->status_host->w[ST_NSTEP_LO] |
                       ((int64_t)h->status_host->w[ST_NSTEP_HI] << 32);
    const double t = (double)(ns - h->mark_nstep) * h->p.dt;
    for (int k = 0; k < K; ++k) {
      const double nk = (double)h->inst_n[k];
      const double g = h->inst_gdot[k] * h->p.a0 * h->p.a0;
      r[3 * k] = t > 0.0 && g != 0.0 ? sums[3 * k] / nk / (2.0 * t) / g : 0.0;
      r[3 * k + 1] = sums[3 * k + 2] != 0.0 ? sums[3 * k + 1] / sums[3 * k + 2] : 0.0;
      r[3 * k + 2] = t;
    }
    CK(cudaMemcpy(out, r.data(), sizeof(double) * r.size(), cudaMemcpyDefault));
    return DSS_OK;
  });
}

int dss_contact_clusters(dss_handle* h, int32_t* label, int64_t* nclusters) {
  return guard([&]() -> int {
    if (!h || !nclusters) return DSS_ERR_ARG;
    if (!h->have_state) return DSS_ERR_STATE;
    ENTER(h);
    // scratch, free between steps: the sort's key, offset and slot arrays hold
    // the parents, the smallest ids and the labels; the id staging array the
    // count
    int* count = h->io_id;
    launch_clusters(h, h->key, h->offs, count, h->tmp);
    CK(cudaGetLastError());
    int c = 0;
    CK(cudaMemcpyAsync(&c, count, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    int r = sync_status(h);
    if (r) return r;
    if ((r = status_error(h))) { clear_err(h); return r; }
    if (label) {
      CK(cudaMemcpy(label, h->tmp, sizeof(int32_t) * h->n, cudaMemcpyDefault));
    }
    *nclusters = c;
    return DSS_OK;
  });
}

int dss_get_counters(dss_handle* h, dss_counters* c) {
  if (!h || !c) return DSS_ERR_ARG;
  int r = sync_status(h);
  if (r) return r;
  const DevStatus& s = *h->status_host;
  memset(c, 0, sizeof(*c));
  c->steps_done = h->host_steps_done;
  c->nstep = (int64_t)(uint32_t)s.w[ST_NSTEP_LO] | ((int64_t)s.w[ST_NSTEP_HI] << 32);
  int P = 0;
  CK(cudaMemcpy(&P, h->lb[h->last_list].start + h->n, sizeof(int), cudaMemcpyDeviceToHost));
  c->npairs = P;
  c->ncontacts = s.w[ST_NCONT];
  c->max_row = s.w[ST_MAXROW];
  c->band_checks = s.w[ST_BAND];
  c->M = h->g.M;
  for (int d = 0; d < 3; ++d) c->ncell[d] = h->ig_host[0].nc[d];
  return DSS_OK;
}

int dss_set_history_rolling(dss_handle* h, int64_t k, const int64_t* keys, const double* xi,
                            const double* xr) {
  return guard([&]() -> int {
    if (!h || k < 0 || (k > 0 && (!keys || !xi))) return DSS_ERR_ARG;
    if (!h->have_state) return DSS_ERR_STATE;
    ENTER(h);
    std::vector<std::pair<int64_t, int64_t>> order(k);
    std::vector<int64_t> hk(k);
    std::vector<double> hx(3 * k), hr(3 * k, 0.0);
    if (k) {
      CK(cudaMemcpy(hk.data(), keys, sizeof(int64_t) * k, cudaMemcpyDefault));
      CK(cudaMemcpy(hx.data(), xi, sizeof(double) * 3 * k, cudaMemcpyDefault));
      if (xr) CK(cudaMemcpy(hr.data(), xr, sizeof(double) * 3 * k, cudaMemcpyDefault));
    }
    for (int64_t q = 0; q < k; ++q) order[q] = {hk[q], q};
    std::sort(order.begin(), order.end());
    const size_t m = (size_t)std::max<int64_t>(k, 1);
    std::vector<long long> sk(m);
    std::vector<double> sx(6 * m, 0.0);   // sliding then rolling stretch
    for (int64_t q = 0; q < k; ++q) {
      sk[q] = order[q].first;
      for (int c = 0; c < 3; ++c) {
        sx[3 * q + c] = hx[3 * order[q].second + c];
        sx[3 * m + 3 * q + c] = hr[3 * order[q].second + c];
      }
    }
    long long* dk = nullptr;
    double* dx = nullptr;
    CK(cudaMalloc((void**)&dk, sizeof(long long) * sk.size()));
    CK(cudaMalloc((void**)&dx, sizeof(double) * sx.size()));
    CK(cudaMemcpy(dk, sk.data(), sizeof(long long) * sk.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dx, sx.data(), sizeof(double) * sx.size(), cudaMemcpyHostToDevice));
    // neighbour build at the current state, attach the stretch, commit as history
    seq_sort_enum(h, false, 0);
    h->cur = 1 - h->cur;
    const int L = 1 - h->hist;
    {
      const int rc = ensure_pair_capacity(h, L);
      if (rc) { cudaFree(dk); cudaFree(dx); return rc; }
    }
    k_attach_history<<<pair_grid_blocks(h), 256, 0, h->stream>>>(h->g, h->st[h->cur], h->lb[L], dk, dx,
                                                                   dx + 3 * m, (int)k);
    CK(cudaGetLastError());
    int r = sync_status(h);
    cudaFree(dk);
    cudaFree(dx);
    if (r) return r;
    if ((r = status_error(h))) { clear_err(h); return r; }
    h->hist = L;
    // the new history's rows follow the committed (sorted) order
    CK(cudaMemsetAsync(&h->status->w[ST_IDORDER], 0, sizeof(int), h->stream));
    return DSS_OK;
  });
}

int dss_set_history(dss_handle* h, int64_t k, const int64_t* keys, const double* xi) {
  return dss_set_history_rolling(h, k, keys, xi, nullptr);
}

int dss_get_history_rolling(dss_handle* h, int64_t* keys, double* xi, double* xr, int64_t cap,
                            int64_t* count) {
  return guard([&]() -> int {
    if (!h || !count || cap < 0 || (cap > 0 && (!keys || !xi))) return DSS_ERR_ARG;
    if (!h->have_state) return DSS_ERR_STATE;
    ENTER(h);
    int P = 0;
    CK(cudaMemcpy(&P, h->lb[h->hist].start + h->n, sizeof(int), cudaMemcpyDeviceToHost));
    long long* dk = nullptr;
    double* dx = nullptr;
    int* cnt = nullptr;
    size_t m = std::max(P, 1);
    CK(cudaMalloc((void**)&dk, sizeof(long long) * m));
    CK(cudaMalloc((void**)&dx, sizeof(double) * 6 * m));
    CK(cudaMalloc((void**)&cnt, sizeof(int)));
    CK(cudaMemsetAsync(cnt, 0, sizeof(int), h->stream));
    k_history_out<<<pair_grid_blocks(h), 256, 0, h->stream>>>(h->g, h->lb[h->hist], dk, dx, dx + 3 * m, cnt,
                                                                (int)m);
    int K = 0;
    CK(cudaMemcpyAsync(&K, cnt, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    std::vector<long long> hk(std::max(K, 1));
    std::vector<double> hx(3 * (size_t)std::max(K, 1)), hr(3 * (size_t)std::max(K, 1));
    CK(cudaMemcpy(hk.data(), dk, sizeof(long long) * K, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hx.data(), dx, sizeof(double) * 3 * K, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hr.data(), dx + 3 * m, sizeof(double) * 3 * K, cudaMemcpyDeviceToHost));
    cudaFree(dk); cudaFree(dx); cudaFree(cnt);
    std::vector<std::pair<long long, int>> order(K);
    for (int q = 0; q < K; ++q) order[q] = {hk[q], q};
    std::sort(order.begin(), order.end());
    *count = K;
    int64_t mm = std::min<int64_t>(cap, K);
    for (int64_t q = 0; q < mm; ++q) {
      keys[q] = order[q].first;
      for (int c = 0; c < 3; ++c) {
        xi[3 * q + c] = hx[3 * order[q].second + c];
        if (xr) xr[3 * q + c] = hr[3 * order[q].second + c];
      }
    }
    return DSS_OK;
  });
}

int dss_get_history(dss_handle* h, int64_t* keys, double* xi, int64_t cap, int64_t* count) {
  return dss_get_history_rolling(h, keys, xi, nullptr, cap, count);
}

// The five state vectors in (id order) into the committed buffer: enqueued,
// not synchronised.
int load_state_enqueue(dss_handle* h, const double* const in[5]) {
    const size_t b = sizeof(double) * 3 * (size_t)h->n;
    StateBuf& s = h->st[h->cur];
    // device and mapped pinned host buffers are read by one kernel; pageable
    // host buffers go through the staging area with the copy engine first
    Src5 src;
    for (int k = 0; k < 5; ++k) {
      src.d[k] = static_cast<const double*>(device_view(in[k]));
      if (!src.d[k]) {
        double* st = h->stage + (size_t)k * 3 * h->n;
        CK(cudaMemcpyAsync(st, in[k], b, cudaMemcpyHostToDevice, h->stream));
        src.d[k] = st;
      }
    }
    k_state_in<<<(int)((h->n + 255) / 256), 256, 0, h->stream>>>((int)h->n, src, s, h->a_by_id, h->inst_map,
                                                                 h->cls_map);
    // the committed state is now in id order, not in the history's row order
    CK(cudaMemsetAsync(&h->status->w[ST_IDORDER], 1, sizeof(int), h->stream));
    CK(cudaGetLastError());
    return DSS_OK;
}

int dss_load_state(dss_handle* h, const double* x, const double* u, const double* w,
                   const double* alpha_lin, const double* alpha_ang) {
  return guard([&]() -> int {
    if (!h || !x || !u || !w || !alpha_lin || !alpha_ang) return DSS_ERR_ARG;
    if (!h->have_state) return DSS_ERR_STATE;
    ENTER(h);
    const double* const in[5] = {x, u, w, alpha_lin, alpha_ang};
    return load_state_enqueue(h, in);
  });
}

int dss_set_profiling(dss_handle* h, int on) {
  if (!h) return DSS_ERR_ARG;
  if (on && !h->prof_ev[0]) {
    for (int k = 0; k <= DSS_PROF_KERNELS; ++k) CK(cudaEventCreate(&h->prof_ev[k]));
  }
  h->profiling = on != 0;
  for (int k = 0; k < DSS_PROF_KERNELS; ++k) h->prof_ms[k] = 0.0;
  h->prof_count = 0;
  drop_graphs(h);
  return DSS_OK;
}

int dss_get_profile(dss_handle* h, double* ms, int64_t* steps) {
  if (!h || !ms || !steps) return DSS_ERR_ARG;
  for (int k = 0; k < DSS_PROF_KERNELS; ++k) ms[k] = h->prof_ms[k];
  *steps = h->prof_count;
  return DSS_OK;
}

const char* dss_profile_name(int k) {
  static const char* names[DSS_PROF_KERNELS] = {"k_key_hist", "k_scan_cells", "k_scatter",
                                                  "k_rank_gather", "k_enumerate", "k_pairs",
                                                  "k_gather"};
  return (k >= 0 && k < DSS_PROF_KERNELS) ? names[k] : "";
}

int dss_last_step_ms(dss_handle* h, double* ms) {
  if (!h || !ms) return DSS_ERR_ARG;
  *ms = h->last_step_ms;
  return DSS_OK;
}

// ------------------------------------------------------------------------
// Checkpoint / resume.  Layout (host byte order):
//   CkptHeader, then x, u, w, alpha_lin, alpha_ang (3n doubles each, id
//   order), a (n doubles, id order), history keys (nhist int64), stretch
//   (3*nhist doubles), with rolling resistance (k_r > 0) the rolling stretch
//   (3*nhist doubles), sigma and sigma_sum (9K doubles each).
// The sorted order inside the library is a function of positions and ids
// alone, so a run resumed from a checkpoint repeats the uninterrupted run bit
// for bit.
// ------------------------------------------------------------------------
namespace {
struct CkptHeader {
  char magic[8];
  uint32_t version;
  int32_t K;
  int64_t n;
  int64_t nstep;
  int64_t nhist;
  int64_t mean_steps;
  uint64_t config;
};
constexpr char kMagic[8] = {'D', 'S', 'S', 'C', 'K', 'P', 'T', '1'};

uint64_t fnv1a(uint64_t hsh, const void* p, size_t len) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < len; ++i) {
    hsh ^= b[i];
    hsh *= 1099511628211ull;
  }
  return hsh;
}

// Fingerprint of what a checkpoint must agree with: instance layout, boxes,
// shear rates, dashpots and the model constants.
uint64_t config_hash(const dss_handle* h) {
  uint64_t v = 1469598103934665603ull;
  v = fnv1a(v, &h->K, sizeof(h->K));
  v = fnv1a(v, h->inst_n, sizeof(int64_t) * h->K);
  v = fnv1a(v, h->inst_box, sizeof(double) * 3 * h->K);
  v = fnv1a(v, h->inst_gdot, sizeof(double) * h->K);
  v = fnv1a(v, h->inst_gn, sizeof(double) * h->K);
  const dss_params& p = h->p;
  const double c[10] = {p.kn, p.kt, p.mu, p.eta0, p.rho, p.delta_lub, p.lub_eps, p.a0, p.dt, p.lub_taper};
  v = fnv1a(v, c, sizeof(c));
  const int32_t m[2] = {p.lub_cutoff_mode, p.precision};
  v = fnv1a(v, m, sizeof(m));
  if (echem_range(&p) > 0.0) {
    const double e[4] = {p.f_er, p.lambda_d, p.hamaker, p.vdw_eps};
    v = fnv1a(v, e, sizeof(e));
  }
  if (h->g.wave) {
    const double wv[2] = {p.wave_amp, (double)p.wave_n};
    v = fnv1a(v, wv, sizeof(wv));
  }
  if (p.k_r > 0.0) v = fnv1a(v, &p.k_r, sizeof(p.k_r));
  return v;
}

size_t ckpt_bytes(int64_t n, int64_t nhist, int K, bool rolling) {
  return sizeof(CkptHeader) + sizeof(double) * 16 * (size_t)n +
         (sizeof(int64_t) + (rolling ? 6 : 3) * sizeof(double)) * nhist + sizeof(double) * 18 * (size_t)K;
}

// Forces the next dss_set_state to rebuild the cell grid and buffers.
void unsize(dss_handle* h) {
  if (h->stream) cudaStreamSynchronize(h->stream);
  drop_graphs(h);
  if (h->sized) free_buffers(h);
  h->sized = false;
  h->have_state = false;
}
}  // namespace

int dss_save(dss_handle* h, void* buf, size_t* len) {
  return guard([&]() -> int {
    if (!h || !len) return DSS_ERR_ARG;
    if (!h->have_state) return DSS_ERR_STATE;
    int64_t nh = 0;
    int r = dss_get_history(h, nullptr, nullptr, 0, &nh);
    if (r) return r;
    const int64_t n = h->n;
    const bool rolling = h->g.k_r > 0.0;
    const size_t need = ckpt_bytes(n, nh, h->K, rolling);
    if (!buf) {
      *len = need;
      return DSS_OK;
    }
    if (*len < need) {
      *len = need;
      return DSS_ERR_ARG;
    }
    CkptHeader hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.magic, kMagic, 8);
    hd.version = 1;
    hd.K = h->K;
    hd.n = n;
    hd.nhist = nh;
    hd.mean_steps = h->mean_steps;
    hd.config = config_hash(h);
    char* out = static_cast<char*>(buf);
    double* x = reinterpret_cast<double*>(out + sizeof(CkptHeader));
    double* a = x + 15 * n;
    int64_t* keys = reinterpret_cast<int64_t*>(a + n);
    double* xi = reinterpret_cast<double*>(keys + nh);
    double* xr = xi + 3 * nh;
    double* sig = xr + (rolling ? 3 * nh : 0);
    std::vector<double> st(15 * (size_t)n);
    if ((r = dss_get_state(h, st.data(), st.data() + 3 * n, st.data() + 6 * n, st.data() + 9 * n,
                           st.data() + 12 * n)))
      return r;
    memcpy(x, st.data(), sizeof(double) * 15 * n);
    int64_t nh2 = 0;
    if (nh > 0 && (r = dss_get_history_rolling(h, keys, xi, rolling ? xr : nullptr, nh, &nh2))) return r;
    if (nh2 != nh && nh > 0) return DSS_ERR_INTERNAL;
    CK(cudaMemcpyAsync(a, h->a_by_id, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(sig, h->sigma, sizeof(double) * 9 * h->K, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(sig + 9 * h->K, h->sigma_sum, sizeof(double) * 9 * h->K, cudaMemcpyDeviceToHost,
                       h->stream));
    if ((r = sync_status(h))) return r;
    hd.nstep = (int64_t)(uint32_t)h->status_host->w[ST_NSTEP_LO] |
               ((int64_t)h->status_host->w[ST_NSTEP_HI] << 32);
    memcpy(out, &hd, sizeof(hd));
    *len = need;
    return DSS_OK;
  });
}

int dss_load(dss_handle* h, const void* buf, size_t len) {
  return guard([&]() -> int {
    if (!h || !buf || len < sizeof(CkptHeader)) return DSS_ERR_ARG;
    CkptHeader hd;
    memcpy(&hd, buf, sizeof(hd));
    if (memcmp(hd.magic, kMagic, 8) != 0 || hd.version != 1 || hd.K != h->K || hd.n != h->n ||
        hd.nhist < 0 || hd.nstep < 0 || hd.mean_steps < 0 || hd.config != config_hash(h))
      return DSS_ERR_ARG;
    const int64_t n = hd.n, nh = hd.nhist;
    const bool rolling = h->g.k_r > 0.0;
    // the history entries must fit in what the buffer holds beyond the fixed
    // part (checked before any size arithmetic on nhist, which could overflow)
    const size_t fixed = ckpt_bytes(n, 0, h->K, rolling);
    const size_t per_entry = sizeof(int64_t) + (rolling ? 6 : 3) * sizeof(double);
    if (len < fixed || (uint64_t)nh > (len - fixed) / per_entry) return DSS_ERR_ARG;
    // copies keep the arrays aligned whatever the caller's buffer alignment
    const char* in = static_cast<const char*>(buf) + sizeof(CkptHeader);
    std::vector<double> st(16 * (size_t)n);
    memcpy(st.data(), in, sizeof(double) * 16 * n);
    in += sizeof(double) * 16 * n;
    std::vector<int64_t> keys(std::max<int64_t>(nh, 1));
    std::vector<double> xi(3 * (size_t)std::max<int64_t>(nh, 1));
    memcpy(keys.data(), in, sizeof(int64_t) * nh);
    in += sizeof(int64_t) * nh;
    memcpy(xi.data(), in, sizeof(double) * 3 * nh);
    in += sizeof(double) * 3 * nh;
    std::vector<double> xr(3 * (size_t)std::max<int64_t>(nh, 1), 0.0);
    if (rolling) {
      memcpy(xr.data(), in, sizeof(double) * 3 * nh);
      in += sizeof(double) * 3 * nh;
    }
    std::vector<double> sig(18 * (size_t)h->K);
    memcpy(sig.data(), in, sizeof(double) * 18 * h->K);
    const double* x = st.data();
    int r = dss_set_state(h, x, x + 15 * n, nullptr, x + 3 * n, x + 6 * n, x + 9 * n, x + 12 * n, hd.nstep);
    if (r) return r;
    if ((r = dss_set_history_rolling(h, nh, keys.data(), xi.data(), rolling ? xr.data() : nullptr))) return r;
    CK(cudaMemcpyAsync(h->sigma, sig.data(), sizeof(double) * 9 * h->K, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->sigma_sum, sig.data() + 9 * h->K, sizeof(double) * 9 * h->K,
                       cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->mean_steps = hd.mean_steps;
    return DSS_OK;
  });
}

int dss_autotune(dss_handle* h, int32_t trial_steps, int32_t ncand, const double* factors,
                 double* ms_per_step, double* cell_size) {
  return guard([&]() -> int {
    static const double kDefault[4] = {1.0, 1.1, 1.25, 1.5};
    if (!h || trial_steps < 1 || ncand < 0 || ncand > 16 || (ncand > 0 && !factors)) return DSS_ERR_ARG;
    if (!h->have_state) return DSS_ERR_STATE;
    if (ncand == 0) {
      ncand = 4;
      factors = kDefault;
    }
    for (int c = 0; c < ncand; ++c)
      if (!(factors[c] >= 1.0) || !std::isfinite(factors[c])) return DSS_ERR_ARG;
    size_t len = 0;
    int r = dss_save(h, nullptr, &len);
    if (r) return r;
    std::vector<char> ck(len);
    if ((r = dss_save(h, ck.data(), &len))) return r;
    const dss_params& p = h->p;
    const double dmax = dmax_of(p, h->a_max);
    const double cmin = (2.0 * h->a_max + dmax) * (1.0 + 1e-9) + 1e-12;
    const double base = p.cell_size > 0.0 ? p.cell_size : cmin;
    const bool prof_was = h->profiling;
    h->profiling = false;
    double best = INFINITY, best_cs = base;
    for (int c = 0; c < ncand; ++c) {
      const double cs = factors[c] * cmin;
      double ms = INFINITY;
      h->p.cell_size = cs;
      unsize(h);
      r = dss_load(h, ck.data(), len);
      if (r == DSS_OK) {
        r = dss_step(h, 2);   // captures the step graphs
        double t = 0.0;
        if (r == DSS_OK) r = dss_step(h, trial_steps);
        if (r == DSS_OK && dss_last_step_ms(h, &t) == DSS_OK) ms = t / trial_steps;
      }
      if (r != DSS_OK && r != DSS_ERR_BOX && r != DSS_ERR_ARG) {
        h->p.cell_size = base;
        unsize(h);
        dss_load(h, ck.data(), len);
        h->profiling = prof_was;
        return r;
      }
      if (ms_per_step) ms_per_step[c] = ms;
      if (ms < best) {
        best = ms;
        best_cs = cs;
      }
    }
    // keep the fastest grid and return to the saved state
    h->p.cell_size = best < INFINITY ? best_cs : base;
    unsize(h);
    r = dss_load(h, ck.data(), len);
    h->profiling = prof_was;
    if (r) return r;
    if (cell_size) *cell_size = h->p.cell_size;
    return best < INFINITY ? DSS_OK : DSS_ERR_BOX;
  });
}

int dss_autotune_kernels(dss_handle* h, int32_t trial_steps, double* ms_per_step, int32_t* choice) {
  return guard([&]() -> int {
    if (!h || trial_steps < 1) return DSS_ERR_ARG;
    if (!h->have_state) return DSS_ERR_STATE;
    size_t len = 0;
    int r = dss_save(h, nullptr, &len);
    if (r) return r;
    std::vector<char> ck(len);
    if ((r = dss_save(h, ck.data(), &len))) return r;
    const bool prof_was = h->profiling;
    h->profiling = false;
    static const int kMinb[2] = {3, 4}, kUnr[2] = {1, 4};
    double best = INFINITY;
    int bm = 0, bu = 0;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        h->tune_pairs_minb = kMinb[a];
        h->tune_enum_unr = kUnr[b];
        drop_graphs(h);
        double ms = INFINITY;
        r = dss_load(h, ck.data(), len);
        if (r == DSS_OK) r = dss_step(h, 2);
        double t = 0.0;
        if (r == DSS_OK) r = dss_step(h, trial_steps);
        if (r == DSS_OK && dss_last_step_ms(h, &t) == DSS_OK) ms = t / trial_steps;
        if (r != DSS_OK) {
          h->tune_pairs_minb = h->tune_enum_unr = 0;
          drop_graphs(h);
          dss_load(h, ck.data(), len);
          h->profiling = prof_was;
          return r;
        }
        if (ms_per_step) ms_per_step[2 * a + b] = ms;
        if (ms < best) {
          best = ms;
          bm = kMinb[a];
          bu = kUnr[b];
        }
      }
    h->tune_pairs_minb = bm;
    h->tune_enum_unr = bu;
    drop_graphs(h);
    r = dss_load(h, ck.data(), len);
    h->profiling = prof_was;
    if (r) return r;
    if (choice) {
      choice[0] = bm;
      choice[1] = bu;
    }
    return DSS_OK;
  });
}

// ------------------------------------------------------------------------
// Adjoint of a rollout: forward with a checkpoint every ckpt_every steps,
// then per segment (last first) a taped replay and the reverse sweep.
// ------------------------------------------------------------------------
// Device checkpoint of the committed state for the adjoint's replays: the
// buffers a step reads (the committed state, the history list with its
// stretch records, the status words with the step counters, the stresses),
// copied as they are, so that a replayed segment repeats the forward bit for
// bit without a round trip through host memory.
}  // extern "C"
namespace {
struct DevSnap {
  char* mem = nullptr;
  size_t bytes = 0;
  int cur = 0, hist = 0;
  int64_t P = 0;
  int64_t mean_steps = 0, host_steps_done = 0;
};

// The copies of one snapshot as (device buffer, bytes) pairs, in a fixed order.
template <typename F>
void snap_fields(dss_handle* h, int cur, int hist, int64_t P, F&& f) {
  const size_t n = (size_t)h->n, d3 = sizeof(double) * 3 * n;
  StateBuf& s = h->st[cur];
  ListBuf& L = h->lb[hist];
  f((void*)s.x, d3); f((void*)s.u, d3); f((void*)s.w, d3); f((void*)s.al, d3); f((void*)s.aw, d3);
  f((void*)s.a, sizeof(double) * n);
  f((void*)s.id, sizeof(int) * n);
  f((void*)s.inst, sizeof(int) * n);
  f((void*)s.cls, n);
  f((void*)s.iy, sizeof(int) * n);
  f((void*)L.count, sizeof(int) * n);
  f((void*)L.list, sizeof(int) * n * (size_t)h->g.Ms);
  f((void*)L.start, sizeof(int) * (n + 1));
  f((void*)L.slot_of_id, sizeof(int) * n);
  f((void*)L.id_of_slot, sizeof(int) * n);
  f((void*)L.xi, sizeof(Xi4) * (size_t)P);
  if (L.xr) f((void*)L.xr, sizeof(Xi4) * (size_t)P);
  f((void*)h->status, sizeof(DevStatus));
  f((void*)h->sigma, sizeof(double) * 9 * (size_t)h->K);
  f((void*)h->sigma_sum, sizeof(double) * 9 * (size_t)h->K);
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

int snap_take(dss_handle* h, DevSnap& sn) {
  int Pd = 0;
  CK(cudaMemcpyAsync(&Pd, h->lb[h->hist].start + h->n, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  const int64_t P = std::min<int64_t>(std::max(Pd, 0), h->pcap);
  size_t need = 0;
  snap_fields(h, h->cur, h->hist, P, [&](void*, size_t b) { need += align256(b); });
  if (need > sn.bytes) {
    if (sn.mem) cudaFree(sn.mem);
    sn.mem = nullptr;
    sn.bytes = 0;
    if (cudaMalloc((void**)&sn.mem, need) != cudaSuccess) {
      cudaGetLastError();
      return DSS_ERR_CUDA;
    }
    sn.bytes = need;
  }
  size_t off = 0;
  snap_fields(h, h->cur, h->hist, P, [&](void* p, size_t b) {
    cudaMemcpyAsync(sn.mem + off, p, b, cudaMemcpyDeviceToDevice, h->stream);
    off += align256(b);
  });
  sn.cur = h->cur;
  sn.hist = h->hist;
  sn.P = P;
  sn.mean_steps = h->mean_steps;
  sn.host_steps_done = h->host_steps_done;
  CK(cudaGetLastError());
  return DSS_OK;
}

int snap_restore(dss_handle* h, const DevSnap& sn) {
  h->cur = sn.cur;
  h->hist = sn.hist;
  h->mean_steps = sn.mean_steps;
  h->host_steps_done = sn.host_steps_done;
  h->last_list = sn.hist;
  size_t off = 0;
  snap_fields(h, sn.cur, sn.hist, sn.P, [&](void* p, size_t b) {
    cudaMemcpyAsync(p, sn.mem + off, b, cudaMemcpyDeviceToDevice, h->stream);
    off += align256(b);
  });
  CK(cudaGetLastError());
  return sync_status(h);   // the host mirror of the restored status words
}
}  // namespace
extern "C" {

int dss_adjoint(dss_handle* h, int64_t nsteps, int32_t ckpt_every, const double* weights,
                int32_t initial_forces, double* J, double* dJ_dparams, double* dJ_dx0,
                double* dJ_du0, double* dJ_dw0, double* dJ_dalpha0, double* dJ_dbeta0) {
  return guard([&]() -> int {
    if (!h || nsteps < 1 || ckpt_every < 1 || !weights) return DSS_ERR_ARG;
    // single instance (the simple shear or the wave of Eq. 17, with or
    // without rolling springs)
    if (h->K != 1) return DSS_ERR_ARG;
    if (!h->have_state) return DSS_ERR_STATE;
    ENTER(h);
    const int64_t nseg = (nsteps + ckpt_every - 1) / ckpt_every;
    int r;
    // device checkpoints, freed on every exit
    std::vector<DevSnap> ck((size_t)nseg);
    DevSnap ck_end;
    struct Free {
      std::vector<DevSnap>& a;
      DevSnap& b;
      ~Free() {
        for (auto& q : a)
          if (q.mem) cudaFree(q.mem);
        if (b.mem) cudaFree(b.mem);
      }
    } free_snaps{ck, ck_end};
    std::vector<double> Wh(9 * (size_t)nsteps);
    CK(cudaMemcpy(Wh.data(), weights, sizeof(double) * 9 * nsteps, cudaMemcpyDefault));
    const bool from_forces = initial_forces != 0;
    const int slots = (int)std::min<int64_t>(ckpt_every, nsteps);
    if ((r = adj_alloc(h, slots, nsteps))) return r;
    if ((r = adj_upload_weights(h, Wh.data(), nsteps))) return r;
    adj_zero(h);
    // ---- forward, with checkpoints and the objective (J summed on the
    // device after every step; one synchronisation per segment)
    double Jacc = 0.0;
    for (int64_t s = 0; s < nseg; ++s) {
      if ((r = snap_take(h, ck[(size_t)s]))) return r;
      const int64_t k1 = std::min<int64_t>(ckpt_every, nsteps - s * ckpt_every);
      const int steps0 = h->status_host->w[ST_STEPS];
      for (int64_t k = 0; k < k1; ++k) {
        StepRun run;
        if ((r = step_launch(h, 1, run))) return r;
        // the roles once the step commits (checked below)
        h->cur = 1 - run.cur0;
        h->hist = 1 - run.hist0;
        adj_accum_J(h, s * ckpt_every + k);
      }
      if ((r = sync_status(h))) return r;
      const int done = h->status_host->w[ST_STEPS] - steps0;
      int err = status_error(h);
      if (err || done != k1) {
        // a step did not commit (e.g. the pair capacity grew): the segment
        // again from its checkpoint, one synchronised step at a time
        if (err) clear_err(h);
        if ((r = snap_restore(h, ck[(size_t)s]))) return r;
        const int P = h->status_host->w[ST_NPAIRS];
        if (err == DSS_ERR_CAPACITY && P > h->pcap &&
            (r = alloc_pair_buffers(h, (int64_t)(P * 1.25) + 1024, true)))
          return r;
        // J back to its value at the segment's start: the sum so far
        CK(cudaMemcpy(h->adj->J, &Jacc, sizeof(double), cudaMemcpyHostToDevice));
        for (int64_t k = 0; k < k1; ++k) {
          if ((r = step_run(h, 1))) return r;
          adj_accum_J(h, s * ckpt_every + k);
        }
        if ((r = sync_status(h))) return r;
      } else {
        h->host_steps_done += done;
        h->mean_steps += done;
        h->last_list = h->hist;
      }
      CK(cudaMemcpy(&Jacc, h->adj->J, sizeof(double), cudaMemcpyDeviceToHost));
    }
    if ((r = snap_take(h, ck_end))) return r;
    // ---- reverse (the pair buffers may have grown during the forward)
    if ((r = adj_alloc(h, slots, nsteps))) return r;
    if ((r = adj_upload_weights(h, Wh.data(), nsteps))) return r;
    adj_zero(h);
    for (int64_t s = nseg - 1; s >= 0; --s) {
      if ((r = snap_restore(h, ck[(size_t)s]))) return r;
      const int64_t k1 = std::min<int64_t>(ckpt_every, nsteps - s * ckpt_every);
      // taped replay (the same kernels as dss_step, without the graph)
      for (int64_t k = 0; k < k1; ++k) {
        const int w = 1 - h->cur;
        launch_sort(h, true, h->cur, w);
        launch_enumerate(h, w, 1 - h->hist, 1);
        adj_tape(h, (int)k, w, 1 - h->hist, h->hist, false);
        launch_forces(h, w, 1 - h->hist, h->hist, 1, G_STEP, nullptr, nullptr);
        h->cur = w;
        h->hist = 1 - h->hist;
        h->last_list = h->hist;
      }
      CK(cudaGetLastError());
      if ((r = sync_status(h))) return r;
      if ((r = status_error(h))) { clear_err(h); return r; }
      for (int64_t k = k1 - 1; k >= 0; --k) adj_reverse(h, (int)k, s * ckpt_every + k, false);
      CK(cudaGetLastError());
    }
    if (from_forces) {
      // alpha^0 came from a force evaluation at the initial state with an
      // empty history: its reverse adds the dependence through alpha^0
      if ((r = snap_restore(h, ck[0]))) return r;
      // its pairs, listed again as that evaluation listed them (a sort
      // without the predictor, the enumeration) over the committed state
      const int w = 1 - h->cur;
      launch_sort(h, false, h->cur, w);
      launch_enumerate(h, w, 1 - h->hist, 0);
      adj_tape(h, 0, w, 1 - h->hist, h->hist, true);
      CK(cudaStreamSynchronize(h->stream));   // the tape's pair count is read on the host
      adj_reverse(h, 0, 0, true);
    }
    CK(cudaGetLastError());
    if ((r = sync_status(h))) return r;
    if ((r = status_error(h))) { clear_err(h); return r; }
    // outputs, then back to the state after the rollout
    AdjBuf* A = h->adj;
    const size_t b3 = sizeof(double) * 3 * (size_t)h->n;
    if (dJ_dx0) CK(cudaMemcpyAsync(dJ_dx0, A->xb, b3, cudaMemcpyDefault, h->stream));
    if (dJ_du0) CK(cudaMemcpyAsync(dJ_du0, A->ub, b3, cudaMemcpyDefault, h->stream));
    if (dJ_dw0) CK(cudaMemcpyAsync(dJ_dw0, A->wb, b3, cudaMemcpyDefault, h->stream));
    if (dJ_dalpha0) CK(cudaMemcpyAsync(dJ_dalpha0, A->ab, b3, cudaMemcpyDefault, h->stream));
    if (dJ_dbeta0) CK(cudaMemcpyAsync(dJ_dbeta0, A->bb, b3, cudaMemcpyDefault, h->stream));
    if (dJ_dparams) CK(cudaMemcpyAsync(dJ_dparams, A->thb, 5 * sizeof(double), cudaMemcpyDefault, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (J) *J = Jacc;
    return snap_restore(h, ck_end);
  });
}

int dss_selftest_bounded_wait(void* cuda_stream) {
  cudaStream_t s = (cudaStream_t)cuda_stream;
  unsigned long long* status = nullptr;
  DevStatus* st = nullptr;
  if (cudaMalloc((void**)&status, 2 * sizeof(unsigned long long)) != cudaSuccess) return DSS_ERR_CUDA;
  if (cudaMalloc((void**)&st, sizeof(DevStatus)) != cudaSuccess) {
    cudaFree(status);
    return DSS_ERR_CUDA;
  }
  DevStatus host;
  int r = DSS_OK;
  if (cudaMemsetAsync(status, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess ||
      cudaMemsetAsync(st, 0, sizeof(DevStatus), s) != cudaSuccess) {
    r = DSS_ERR_CUDA;
  } else {
    k_selftest_wait<<<1, 32, 0, s>>>(status, st);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&host, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      r = DSS_ERR_CUDA;
    else
      r = host.w[ST_ERR];
  }
  cudaFree(status);
  cudaFree(st);
  return r;
}

int64_t dss_device_bytes(const dss_handle* h) { return h ? h->bytes : 0; }

void dss_destroy(dss_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  adj_free(h);
  drop_graphs(h);
  free_buffers(h);
  if (h->status) cudaFree(h->status);
  if (h->status_host) cudaFreeHost(h->status_host);
  if (h->ev_enter) cudaEventDestroy(h->ev_enter);
  for (int k = 0; k <= DSS_PROF_KERNELS; ++k)
    if (h->prof_ev[k]) cudaEventDestroy(h->prof_ev[k]);
  for (int k = 0; k < 2; ++k)
    if (h->step_ev[k]) cudaEventDestroy(h->step_ev[k]);
  if (h->stream && h->own_stream) cudaStreamDestroy(h->stream);
  delete[] h->ig_host;
  delete[] h->inst_box;
  delete[] h->inst_gdot;
  delete[] h->inst_gn;
  delete[] h->inst_n;
  delete h;
}

}  // extern "C"
