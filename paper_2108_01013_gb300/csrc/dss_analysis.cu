// Analysis pass over the committed state (not part of the time step):
//   - the Lees-Edwards image count along y of each particle (the step keeps it
//     with the state), from which the shear-wise dispersion of Eq. 18 and the
//     velocity autocorrelation of Eq. 19 are reduced per instance, in a fixed
//     order, against a marked reference time;
//   - the clusters of contacting particles (Sec. III A, Fig. 10-11): the
//     connected components of the graph whose edges are the pairs in contact
//     at the last committed step, by a lock-free union-find (a root is only
//     ever linked below a smaller root, so every parent chain decreases and
//     every walk ends), labelled by the smallest id of each cluster, which
//     makes the result unique;
//   - the local volume fraction along the shear-wise direction y by size
//     class (Sec. III B, Fig. 12): the volume of each sphere inside each of
//     nbins slabs of the box (the exact integral of its cross-sections,
//     periodic in y), summed per instance, class and slab as 64-bit integers
//     in a unit of 2^-62 of the instance's solid volume (integer sums do not
//     depend on their order, so the profile is reproducible bit for bit).
#include <climits>

#include "dss_internal.cuh"

namespace {
constexpr int kThreads = 256;

// Image count of each particle, by id.
__global__ void k_images_out(int n, StateBuf s, int* __restrict__ out) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f < n) out[s.id[f]] = s.iy[f];
}

// Reference of the dispersion: unwrapped y and v_y of each id.
__global__ void k_mark(int n, const InstGeo* __restrict__ ig, StateBuf s, double* __restrict__ mark) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n) return;
  const int id = s.id[f];
  mark[id] = s.x[n + f] + (double)s.iy[f] * ig[s.inst[f]].L[1];
  mark[n + id] = s.u[n + f];
}

// One block per instance: sum over its particles (sorted range) of
// (y - y0)^2, v v0 and v^2, strided then a fixed tree.  The shear-wise
// velocity fluctuation is u_y (the imposed flow has no y component).
__global__ void __launch_bounds__(kThreads)
k_dispersion(int n, const InstGeo* __restrict__ ig, StateBuf s, const double* __restrict__ mark,
             double* __restrict__ sums) {
  const InstGeo& I = ig[blockIdx.x];
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (int f = I.p_begin + threadIdx.x; f < I.p_end; f += blockDim.x) {
    const int id = s.id[f];
    const double dy = s.x[n + f] + (double)s.iy[f] * I.L[1] - mark[id];
    const double v = s.u[n + f];
    a0 += dy * dy;
    a1 += v * mark[n + id];
    a2 += v * v;
  }
  __shared__ double red[3][kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int d = 16; d > 0; d >>= 1) {
    a0 += __shfl_down_sync(0xffffffffu, a0, d);
    a1 += __shfl_down_sync(0xffffffffu, a1, d);
    a2 += __shfl_down_sync(0xffffffffu, a2, d);
  }
  if (lane == 0) {
    red[0][wid] = a0;
    red[1][wid] = a1;
    red[2][wid] = a2;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double v = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) v += red[threadIdx.x][w];
    sums[3 * blockIdx.x + threadIdx.x] = v;
  }
}

// ---------------------------------------------------------------- clusters
__device__ __forceinline__ int ld(const int* p) { return *((volatile const int*)p); }

// Root of x, halving the path on the way (a grandparent is always an
// ancestor, so the racing writes only shorten chains).  Parent indices
// strictly decrease along a chain, so the walk ends.
__device__ __forceinline__ int cc_find(int* parent, int x) {
  while (true) {
    const int p = ld(parent + x);
    if (p == x) return x;
    const int gp = ld(parent + p);
    if (gp != p) parent[x] = gp;
    x = gp;
  }
}

__global__ void k_cc_init(int n, int* __restrict__ parent, int* __restrict__ minid) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    parent[i] = i;
    minid[i] = INT_MAX;
  }
}

// One thread per owner row of the committed list: every pair whose stretch
// record carries the contact flag joins its two particles.  A root is linked
// below the other, smaller root by a compare-and-swap that fails only if it
// was linked meanwhile; the retries are bounded (an error flag instead of a
// spin).
__global__ void k_cc_link(Geo g, ListBuf H, int* parent, DevStatus* st) {
  const int n = g.n;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = H.count[i];
  const int p0 = H.start[i];
  for (int k = 0; k < c; ++k) {
    if (p0 + k >= g.pcap) break;
    if (!xi_flag(H.xi[p0 + k])) continue;
    int a = i, b = H.list[(int64_t)i * g.Ms + k];
    bool done = false;
    for (int it = 0; it < (1 << 20) && !done; ++it) {
      a = cc_find(parent, a);
      b = cc_find(parent, b);
      if (a == b) {
        done = true;
      } else {
        if (a < b) { const int t = a; a = b; b = t; }
        done = atomicCAS(parent + a, a, b) == a;
      }
    }
    if (!done) set_err(st, DSS_ERR_INTERNAL);
  }
}

// Roots, the smallest id of each cluster, and the count of clusters.
__global__ void k_cc_root(int n, ListBuf H, int* parent, int* __restrict__ minid, int* __restrict__ count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int r = cc_find(parent, i);
  parent[i] = r;
  atomicMin(minid + r, H.id_of_slot[i]);
  if (r == i) atomicAdd(count, 1);
}

__global__ void k_cc_label(int n, ListBuf H, const int* __restrict__ parent, const int* __restrict__ minid,
                           int* __restrict__ label) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) label[H.id_of_slot[i]] = minid[parent[i]];
}
// ------------------------------------------------------------ phi(y)
// Volume of the sphere of radius a centred at yc between the planes y0 < y1:
// the integral of the cross-section pi (a^2 - t^2) over t = y - yc clipped
// to [-a, a].
__device__ __forceinline__ double slab_volume(double a, double yc, double y0, double y1) {
  const double t0 = fmax(y0 - yc, -a), t1 = fmin(y1 - yc, a);
  if (t1 <= t0) return 0.0;
  return DSS_PI * (a * a * (t1 - t0) - (t1 * t1 * t1 - t0 * t0 * t0) / 3.0);
}

// One thread per particle: its volume in every slab it reaches (its images
// across y = 0 and y = L_y included), class 1 when a > a_split.
__global__ void k_phi_profile(int n, const InstGeo* __restrict__ ig, StateBuf s, int nbins, double a_split,
                              const double* __restrict__ unit, unsigned long long* __restrict__ acc) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n) return;
  const int inst = s.inst[f];
  const InstGeo& I = ig[inst];
  const double y = s.x[n + f], a = s.a[f], Ly = I.L[1], w = Ly / nbins, u = unit[inst];
  unsigned long long* row = acc + ((size_t)inst * 2 + (a > a_split ? 1 : 0)) * nbins;
  for (int img = -1; img <= 1; ++img) {
    const double yc = y + img * Ly;
    if (yc + a <= 0.0 || yc - a >= Ly) continue;
    const int b0 = max(0, (int)floor((yc - a) / w)), b1 = min(nbins - 1, (int)floor((yc + a) / w));
    for (int b = b0; b <= b1; ++b) {
      const double v = slab_volume(a, yc, b * w, b == nbins - 1 ? Ly : (b + 1) * w);
      if (v > 0.0) atomicAdd(row + b, (unsigned long long)llrint(v / u));
    }
  }
}
}  // namespace

void launch_phi_profile(dss_handle* h, int nbins, double a_split, const double* unit, unsigned long long* acc) {
  const int n = (int)h->n;
  k_phi_profile<<<(n + kThreads - 1) / kThreads, kThreads, 0, h->stream>>>(n, h->ig, h->st[h->cur], nbins,
                                                                            a_split, unit, acc);
}

void launch_images_out(dss_handle* h, int* out) {
  const int n = (int)h->n;
  k_images_out<<<(n + kThreads - 1) / kThreads, kThreads, 0, h->stream>>>(n, h->st[h->cur], out);
}

void launch_mark(dss_handle* h) {
  const int n = (int)h->n;
  k_mark<<<(n + kThreads - 1) / kThreads, kThreads, 0, h->stream>>>(n, h->ig, h->st[h->cur], h->mark);
}

void launch_dispersion(dss_handle* h, double* sums) {
  k_dispersion<<<h->K, kThreads, 0, h->stream>>>((int)h->n, h->ig, h->st[h->cur], h->mark, sums);
}

// The committed list's index space (its rows, id map and stretch records);
// parent and minid are n-int scratch, count one int, label n ints by id.
void launch_clusters(dss_handle* h, int* parent, int* minid, int* count, int* label) {
  const int n = (int)h->n;
  const int nb = (n + kThreads - 1) / kThreads;
  const ListBuf& H = h->lb[h->hist];
  k_cc_init<<<nb, kThreads, 0, h->stream>>>(n, parent, minid);
  cudaMemsetAsync(count, 0, sizeof(int), h->stream);
  k_cc_link<<<nb, kThreads, 0, h->stream>>>(h->g, H, parent, h->status);
  k_cc_root<<<nb, kThreads, 0, h->stream>>>(n, H, parent, minid, count);
  k_cc_label<<<nb, kThreads, 0, h->stream>>>(n, H, parent, minid, label);
}
