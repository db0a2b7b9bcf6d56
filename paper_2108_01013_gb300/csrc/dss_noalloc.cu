// Neighbour-pair search that allocates no device memory.
//
// Some callers cannot allocate GPU memory at all: code that runs inside a
// host application which owns every device allocation (a plugin, a solver
// embedded in another framework's memory pool), or a process whose memory is
// fully reserved up front.  dss_pairs_noalloc gives them the same pair set
// as dss_neighbour_build + dss_get_pairs with no cudaMalloc/cudaFree and no
// allocating library call: its only working memory is the fixed array
// g_noalloc_scratch below, which every GPU that loads this library holds
// until the process exits.
//
// The search is a plain cell list: count particles per cell, scan, fill,
// then every particle visits the 27 surrounding cells (the rows reached
// through y = L_y shifted by the Lees-Edwards offset) and keeps partners with
// a larger array index, deciding with the same exact FP64 predicate as the
// main path.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "dss_internal.cuh"

namespace {

constexpr int kHeader = 16;   // [0..1] pair counter (64 bit), [2] error flag

static __device__ __align__(256) int g_noalloc_scratch[DSS_NOALLOC_SCRATCH_INTS];

struct NoAllocGrid {
  double L[3], cs[3], inv_cs[3], halfL[3];
  int nc[3];
  int ncell;
};

__global__ void k_na_clear(int* s, int words) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < words; i += gridDim.x * blockDim.x) s[i] = 0;
}

__device__ __forceinline__ int na_cell(const NoAllocGrid& q, double x, double y, double z) {
  int cx = cell_coord(x, q.inv_cs[0], q.nc[0]);
  int cy = cell_coord(y, q.inv_cs[1], q.nc[1]);
  int cz = cell_coord(z, q.inv_cs[2], q.nc[2]);
  return (cz * q.nc[1] + cy) * q.nc[0] + cx;
}

__global__ void k_na_count(NoAllocGrid q, int n, const double* __restrict__ x,
                           const double* __restrict__ a, double a_max, int* s, int* cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (!(a[i] <= a_max) || !(a[i] > 0.0)) atomicExch(&s[2], 1);
  atomicAdd(&cnt[na_cell(q, x[i], x[n + i], x[2 * n + i])], 1);
}

// exclusive scan of the cell counts by one block (sizes here are modest)
__global__ void k_na_scan(int ncell, const int* __restrict__ cnt, int* __restrict__ start) {
  __shared__ int warp_sums[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int base = 0; base < ncell; base += blockDim.x) {
    int i = base + threadIdx.x;
    int v = i < ncell ? cnt[i] : 0;
    int incl = v;
    for (int d = 1; d < 32; d <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += t;
    }
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      int w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
      int wi = w;
      for (int d = 1; d < 32; d <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, wi, d);
        if (lane >= d) wi += t;
      }
      if (lane < (int)(blockDim.x >> 5)) warp_sums[lane] = wi - w;
    }
    __syncthreads();
    if (i < ncell) start[i] = carry + warp_sums[wid] + incl - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += warp_sums[wid] + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) start[ncell] = carry;
}

__global__ void k_na_fill(NoAllocGrid q, int n, const double* __restrict__ x,
                          const int* __restrict__ start, int* cursor, int* __restrict__ order) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = na_cell(q, x[i], x[n + i], x[2 * n + i]);
  order[start[c] + atomicAdd(&cursor[c], 1)] = i;
}

__global__ void k_na_pairs(NoAllocGrid q, Geo g, InstGeo I, int n, const double* __restrict__ x,
                           const double* __restrict__ a, const int* __restrict__ ids, double off,
                           const int* __restrict__ start, const int* __restrict__ order, int* s,
                           long long* __restrict__ out, long long cap) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double xi = x[i], yi = x[n + i], zi = x[2 * n + i], ai = a[i];
  const int c = na_cell(q, xi, yi, zi);
  const int cx = c % q.nc[0], cy = (c / q.nc[0]) % q.nc[1], cz = c / (q.nc[0] * q.nc[1]);
  const int fsh = (int)floor(off * q.inv_cs[0]);
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(s);
  for (int oy = -1; oy <= 1; ++oy) {
    const int ry = cy + oy;
    int x0 = -1, x1 = 1;
    if (ry >= q.nc[1]) { x0 = -2 - fsh; x1 = 1 - fsh; }   // image above, shifted by +off
    if (ry < 0) { x0 = -1 + fsh; x1 = 2 + fsh; }          // image below, shifted by -off
    const int qy = wrapi(ry, q.nc[1]);
    for (int oz = -1; oz <= 1; ++oz) {
      const int qz = wrapi(cz + oz, q.nc[2]);
      for (int ox = x0; ox <= x1; ++ox) {
        const int qc = (qz * q.nc[1] + qy) * q.nc[0] + wrapi(cx + ox, q.nc[0]);
        for (int t = start[qc]; t < start[qc + 1]; ++t) {
          const int j = order[t];
          if (j <= i) continue;
          if (!exact_is_pair(g, I, off, xi, yi, zi, ai, x[j], x[n + j], x[2 * n + j], a[j])) continue;
          const unsigned long long k = atomicAdd(counter, 1ull);
          if ((long long)k < cap) {
            const long long u = ids ? ids[i] : i, v = ids ? ids[j] : j;
            out[2 * k] = u < v ? u : v;
            out[2 * k + 1] = u < v ? v : u;
          }
        }
      }
    }
  }
}

// Device address of the scratch array, looked up once per device.
std::mutex g_na_mutex;
void* g_na_ptr[128];
bool g_na_ready[128];

int noalloc_scratch(int** ptr) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return DSS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ready[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DSS_ERR_CUDA;
    g_na_ptr[dev] = p;
    g_na_ready[dev] = true;
  }
  *ptr = static_cast<int*>(g_na_ptr[dev]);
  return DSS_OK;
}

}  // namespace

extern "C" int dss_pairs_noalloc(const double* x, const double* a, const int32_t* ids, int64_t n,
                                 const double box[3], const dss_params* p, double a_max,
                                 int64_t nstep, int64_t* pairs, int64_t cap, int64_t* count,
                                 void* cuda_stream) {
  if (!x || !a || !box || !p || !count || n < 2 || n > (1 << 30) || cap < 0 || (cap > 0 && !pairs) ||
      !(a_max > 0.0) || nstep < 0 || (p->lub_cutoff_mode != 0 && p->lub_cutoff_mode != 1))
    return DSS_ERR_ARG;
  // cell grid: edge >= the largest interaction range, as in the main path
  const double dl = p->lub_cutoff_mode == 1 ? p->delta_lub * p->a0 : p->delta_lub * a_max;
  const double de = echem_range(p);
  const double dmax = de > dl ? de : dl;
  const double cmin = (2.0 * a_max + dmax) * (1.0 + 1e-9) + 1e-12;
  NoAllocGrid q;
  for (int d = 0; d < 3; ++d) {
    if (!(box[d] > 0.0)) return DSS_ERR_ARG;
    q.L[d] = box[d];
    q.halfL[d] = 0.5 * box[d];
    q.nc[d] = (int)std::floor(box[d] / cmin);
    if (q.nc[d] < 1) q.nc[d] = 1;
    q.cs[d] = box[d] / q.nc[d];
    q.inv_cs[d] = 1.0 / q.cs[d];
  }
  if (q.nc[0] < 4 || q.nc[1] < 3 || q.nc[2] < 3) return DSS_ERR_BOX;
  const double cells = (double)q.nc[0] * q.nc[1] * q.nc[2];
  // scratch: header, counts, starts (+1), cursors, order
  if ((double)kHeader + 3.0 * cells + 1.0 + (double)n > (double)DSS_NOALLOC_SCRATCH_INTS)
    return DSS_ERR_SCRATCH_LIMIT;
  q.ncell = (int)cells;
  int* s = nullptr;
  int r = noalloc_scratch(&s);
  if (r) return r;
  int* cnt = s + kHeader;
  int* start = cnt + q.ncell;
  int* cursor = start + q.ncell + 1;
  int* order = cursor + q.ncell;
  Geo g;
  memset(&g, 0, sizeof(g));
  InstGeo I;
  memset(&I, 0, sizeof(I));
  for (int d = 0; d < 3; ++d) {
    I.L[d] = box[d];
    I.halfL[d] = 0.5 * box[d];
    I.invL[d] = 1.0 / box[d];
  }
  g.delta = p->delta_lub;
  g.a0 = p->a0;
  g.mode = p->lub_cutoff_mode;
  g.de = de;
  I.gdot = p->shear_rate;
  g.dt = p->dt;
  // Lees-Edwards offset at time nstep*dt, with the same operations as the main path
  const double t = (double)nstep * p->dt;
  const double off = std::fmod(p->shear_rate * box[1] * t, box[0]);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int words = kHeader + 3 * q.ncell + 1;
  const int nb = (int)((n + 255) / 256);
  // the array keeps the previous call's contents: clear header, counts, cursors
  k_na_clear<<<std::min(1024, (words + 255) / 256), 256, 0, st>>>(s, words);
  k_na_count<<<nb, 256, 0, st>>>(q, (int)n, x, a, a_max, s, cnt);
  k_na_scan<<<1, 1024, 0, st>>>(q.ncell, cnt, start);
  k_na_fill<<<nb, 256, 0, st>>>(q, (int)n, x, start, cursor, order);
  k_na_pairs<<<nb, 256, 0, st>>>(q, g, I, (int)n, x, a, ids, off, start, order, s,
                                 reinterpret_cast<long long*>(pairs), (long long)cap);
  if (cudaGetLastError() != cudaSuccess) return DSS_ERR_CUDA;
  int head[4] = {0, 0, 0, 0};
  if (cudaMemcpyAsync(head, s, sizeof(head), cudaMemcpyDeviceToHost, st) != cudaSuccess) return DSS_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return DSS_ERR_CUDA;
  if (head[2]) return DSS_ERR_ARG;   // a radius above a_max or not positive
  long long total = 0;
  memcpy(&total, head, sizeof(total));
  *count = total;
  return DSS_OK;
}
