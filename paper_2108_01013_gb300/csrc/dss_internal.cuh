// Internal definitions shared by the libdss CUDA translation units.
// Geometry, cell stencils and the exact neighbour predicate live here so that
// every kernel evaluates them with the same instruction sequence.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dss.h"

#define DSS_PI 3.14159265358979323846
#define DSS_PROF_KERNELS 7
#define DSS_MULTI_STEPS 8

// Device status word layout (int32 slots in DevStatus::w).
enum {
  ST_ERR = 0,        // first error code seen (0 = none); later kernels early-exit
  ST_MAXROW = 1,     // largest half-list row of the last enumeration
  ST_NPAIRS = 2,     // pairs of the last enumeration
  ST_NCONT = 3,      // contacts of the last force pass
  ST_BAND = 4,       // exact-predicate fallbacks of the last enumeration
  ST_STEPS = 5,      // committed steps (low 32 bits)
  ST_NSTEP_LO = 6,   // time step counter (64 bit, lo/hi)
  ST_NSTEP_HI = 7,
  ST_BADPOS = 8,     // set_state: positions outside the box
  ST_IDORDER = 9,    // 1 after dss_load_state: the committed state is not in the history's row order
  ST_WORDS = 16
};

// Lees-Edwards geometry of one instance at the time the current operation
// evaluates at, written once per operation by the first kernel (k_key_hist):
// off = fsh * cs_x + offr, offr = offr_hi + offr_lo in [0, cs_x).
struct StepGeo {
  double off;
  int fsh;
  float offr_hi, offr_lo;
};

struct DevStatus {
  int w[ST_WORDS];
};

// Model constants shared by every instance, by value.
struct Geo {
  int n;              // particles of all instances
  int K;              // instances
  int ncell;          // cell bins of all instances (classes x cells)
  int nclass;         // particle size classes (1: one cell list, cells >= 2 a_max + delta)
  int reach;          // largest stencil reach in cells of any class pair
  unsigned char rtab[8][8];   // rtab[c][c2], c2 <= c: reach of class c searching class c2
  int M;              // half-list capacity per particle
  int Ms;             // row stride of the half lists (M rounded up to 4)
  int64_t pcap;       // pair capacity
  double kn, kt, mu;
  double eta0, rho;
  double delta, eps, a0;
  int mode;           // cutoff mode
  int precision;
  double dt;
  double hdt, hdt2;   // dt/2 and (dt/2) dt, each rounded once
  double k6;          // 6 pi eta0
  double k8;          // 8 pi eta0
  double taper;       // lubrication taper width w (0: hard cutoff)
  double f_er, lambda_d, hamaker, vdw_eps;   // electro-chemical forces (Eq. 6-7)
  double de;          // their range as a surface distance (0: off)
  int wave;           // the wavy shear flow of Eq. 17 is on (wave_amp != 0, wave_n > 0)
  double wave_amp;    // its amplitude U (wave number per instance: InstGeo::wave_k)
  double k_r;         // rolling spring stiffness of App. B (0: off)
  struct {             // FP32 copies of the model constants (mixed precision)
    float kn, kt, mu_kt, dt, eps, k6, k8, mass_c;
    float taper, delta, delta_a0;
    float f_er, inv_lambda, range_r, hamaker12, vdw_eps, range_a;   // f_er: F_ER / a0
    float k_r, mu_kr;  // rolling: k_r, mu / k_r
  } f;
};

// One instance (an independent suspension): its box, cell grid, shear rate
// and dashpot; read by each thread from a small device table.  Its particles
// occupy sorted positions [p_begin, p_end) (cell ids are instance-major) and
// ids [p_begin, p_end).
struct InstGeo {
  double L[3], halfL[3], invL[3];
  double cs[3], inv_cs[3];      // cell edge per axis
  float csf[3], cs_lo[3];       // double-float cell edges
  float inv_csf[3];             // FP32 inverse cell edges (the cell test's fast path)
  float halfLf[3];
  float r2_margin;              // FP32 prefilter margin on r^2 (absolute)
  int nc[3];
  int cell_base, ncell;        // first bin and bins (= classes x ncell_layer)
  int ncell_layer;             // cells of one class layer (nc[0] nc[1] nc[2])
  int p_begin, p_end;
  double gdot, gn;              // shear rate, normal dashpot
  float gdot_f, gn_f;
  double sumA3;                 // sum of a^3 (Einstein stresslet of Eq. 9)
  double wave_k;                // 2 pi n / L_y of the wave of Eq. 17 (0: no wave)
  double faxen_c;               // wave_k^2 / 6: the Faxen factor is 1 - a^2 faxen_c
};

// ------------------------------------------------------------------------
// Small device helpers
// ------------------------------------------------------------------------
__device__ __forceinline__ int dev_err(const DevStatus* s) {
  return *((volatile const int*)&s->w[ST_ERR]);
}
__device__ __forceinline__ void set_err(DevStatus* s, int code) {
  atomicCAS(&s->w[ST_ERR], 0, code);
}
__device__ __forceinline__ int64_t dev_nstep(const DevStatus* s) {
  const volatile int* w = (const volatile int*)s->w;
  return (int64_t)(uint32_t)w[ST_NSTEP_LO] | ((int64_t)w[ST_NSTEP_HI] << 32);
}

// Lees-Edwards offset at step count nstep: fmod(gdot * L_y * (nstep dt), L_x),
// with the product taken in that order and no fused operations.
__device__ __forceinline__ double le_offset(const Geo& g, const InstGeo& I, int64_t nstep) {
  double t = __dmul_rn((double)nstep, g.dt);
  return fmod(__dmul_rn(__dmul_rn(I.gdot, I.L[1]), t), I.L[0]);
}

// Interaction range beyond contact for the pair.
__device__ __forceinline__ double lub_delta(const Geo& g, double ai, double aj) {
  if (g.mode == 1) return __dmul_rn(g.delta, g.a0);
  return __dmul_rn(__dmul_rn(g.delta, __dadd_rn(ai, aj)), 0.5);
}

// Listing range of a pair: the larger of the lubrication cutoff and the
// electro-chemical range.
__device__ __forceinline__ double pair_delta(const Geo& g, double ai, double aj) {
  const double dl = lub_delta(g, ai, aj);
  return g.de > dl ? g.de : dl;
}

// Minimum-image separation r = x_j - x_i under Lees-Edwards conditions,
// spelled out operation by operation (no contraction) so that the neighbour
// decision is the same bit pattern on every path.  sy: image shift in y
// (-1: image one box below, +1: above).
__device__ __forceinline__ void min_image(const InstGeo& g, double off, double xi, double yi,
                                          double zi, double xj, double yj, double zj,
                                          double& dx, double& dy, double& dz, int& sy) {
  dx = __dsub_rn(xj, xi);
  dy = __dsub_rn(yj, yi);
  dz = __dsub_rn(zj, zi);
  sy = 0;
  if (dy > g.halfL[1]) {
    dy = __dsub_rn(dy, g.L[1]);
    dx = __dsub_rn(dx, off);
    sy = -1;
  } else if (dy < -g.halfL[1]) {
    dy = __dadd_rn(dy, g.L[1]);
    dx = __dadd_rn(dx, off);
    sy = 1;
  }
  // image count rint(dx / L) taken as rint(dx * (1/L)): the two differ only
  // when dx is within rounding of +-L/2, where both images lie at least
  // L/2 >= 1.5 cells away, beyond any pair's cutoff, so no decision changes
  dx = __dsub_rn(dx, __dmul_rn(g.L[0], rint(__dmul_rn(dx, g.invL[0]))));
  dz = __dsub_rn(dz, __dmul_rn(g.L[2], rint(__dmul_rn(dz, g.invL[2]))));
}

// Centre distance |r| with the operations of the plain FP64 evaluation
// ((dx dx + dy dy) + dz dz, then the square root): the contact decision
// d = |r| - (a_i + a_j) < 0 of Eq. 4 is then the same bit for bit.
__device__ __forceinline__ double exact_dist(double dx, double dy, double dz) {
  return sqrt(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
}

// Exact neighbour predicate: r^2 < (a_i + a_j + delta_ij)^2, strict.
__device__ __forceinline__ bool exact_is_pair(const Geo& g, const InstGeo& I, double off, double xi,
                                              double yi, double zi, double ai, double xj,
                                              double yj, double zj, double aj) {
  double dx, dy, dz;
  int sy;
  min_image(I, off, xi, yi, zi, xj, yj, zj, dx, dy, dz, sy);
  double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  double s = __dadd_rn(__dadd_rn(ai, aj), pair_delta(g, ai, aj));
  return r2 < __dmul_rn(s, s);
}

__device__ __forceinline__ int cell_coord(double v, double inv, int nc) {
  int k = __double2int_rd(v * inv);   // floor, one conversion
  return k < 0 ? 0 : (k >= nc ? nc - 1 : k);
}

// ------------------------------------------------------------------------
// Conversions by integer operations on the IEEE-754 bit patterns.  GB300's
// FP64 pipe (two lanes per SM per clock) runs the FP64 conversions too; in
// the sort's kernels they outnumbered the arithmetic.  Each function returns
// exactly what the named hardware conversion returns (round to nearest,
// ties to even) and hands the cases outside its range (zero, subnormal,
// infinite, NaN, out of the float range) to that conversion, called out of
// line: a branch the compiler turns into predicated instructions still
// issues them to the FP64 pipe.
// ------------------------------------------------------------------------
static __device__ __noinline__ float f32_rn_slow(double v) { return __double2float_rn(v); }
static __device__ __noinline__ double f64_of_slow(float f) { return (double)f; }
static __device__ __noinline__ double f64_of_int_slow(int c) { return (double)c; }
static __device__ __noinline__ float2 f32_split_slow(double v) {
  const float hi = __double2float_rn(v);
  return make_float2(hi, __double2float_rn(v - (double)hi));
}
static __device__ __noinline__ int floor_mul_slow(double v, double inv) { return __double2int_rd(v * inv); }

// double -> float, as __double2float_rn.  A double of biased exponent e in
// [897, 1150] is a normal float after rounding: the top 23 fraction bits are
// kept, the 29 below decide the rounding, and a carry out of the fraction
// moves into the exponent field (up to infinity), as IEEE rounding does.
__device__ __forceinline__ float f32_rn(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned long long a = b & 0x7FFFFFFFFFFFFFFFull;
  const unsigned e = (unsigned)(a >> 52);
  if (e - 897u > 1150u - 897u) return f32_rn_slow(v);
  unsigned t = (unsigned)((a >> 29) - (896ull << 23));
  const unsigned rem = (unsigned)a & 0x1FFFFFFFu;
  t += (rem > 0x10000000u) | ((rem == 0x10000000u) & t);
  return __uint_as_float(t | ((unsigned)(b >> 32) & 0x80000000u));
}

// float -> double (exact), as (double)f.
__device__ __forceinline__ double f64_of(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned a = u & 0x7FFFFFFFu;
  if (a - 0x00800000u >= 0x7F000000u) return f64_of_slow(f);
  return __longlong_as_double((long long)((((unsigned long long)a + (896ull << 23)) << 29) |
                                          ((unsigned long long)(u & 0x80000000u) << 32)));
}

// Non-negative int -> double (exact), as (double)c.
__device__ __forceinline__ double f64_of_nonneg(int c) {
  if (c <= 0) return f64_of_int_slow(c);
  const int e = 31 - __clz(c);   // c in [2^e, 2^(e+1))
  const unsigned long long m = ((unsigned long long)c << (52 - e)) & 0xFFFFFFFFFFFFFull;
  return __longlong_as_double((long long)(((unsigned long long)(e + 1023) << 52) | m));
}

// The double-float split of v: hi = RN_f32(v), lo = RN_f32(v - hi), as
// hi = __double2float_rn(v); lo = __double2float_rn(v - (double)hi).  With
// v = M 2^(e-1075) (M the 53-bit significand), v - hi is exactly
// (rem - up 2^29) 2^(e-1075) with rem the 29 discarded bits and up the
// rounding carry; its float is the integer's float (round to nearest) scaled
// by a power of two, exact while the result is a normal float (e >= 949).
// Below 2^126 (e <= 1149) hi cannot round up to infinity.
__device__ __forceinline__ void f32_split(double v, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned long long a = b & 0x7FFFFFFFFFFFFFFFull;
  const unsigned e = (unsigned)(a >> 52);
  if (e - 949u > 1149u - 949u) {
    const float2 q = f32_split_slow(v);
    hi = q.x;
    lo = q.y;
    return;
  }
  unsigned t = (unsigned)((a >> 29) - (896ull << 23));
  const unsigned rem = (unsigned)a & 0x1FFFFFFFu;
  const unsigned up = (rem > 0x10000000u) | ((rem == 0x10000000u) & t);
  t += up;
  const bool neg = (b >> 63) != 0;
  hi = __uint_as_float(t | (neg ? 0x80000000u : 0u));
  const int r = (int)rem - (int)(up << 29);
  lo = __int2float_rn(neg ? -r : r) * __uint_as_float((e - 948u) << 23);
}

// floor(RN_d(v inv)) as __double2int_rd(v * inv), for |v inv| < 2^22: the
// FP32 product is within 2^-21 |product| of the FP64 one, so away from an
// integer by more than that their floors agree; closer, the FP64 product
// decides.
__device__ __forceinline__ int floor_mul(double v, double inv, float invf) {
  const float pf = f32_rn(v) * invf;
  const float k = floorf(pf);
  const float tol = fabsf(pf) * 4.76837158203125e-7f;   // 2^-21
  if (pf - k > tol && (k + 1.0f) - pf > tol && fabsf(pf) < 4194304.0f) return (int)k;
  return floor_mul_slow(v, inv);
}

__device__ __forceinline__ int wrapi(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// Shift (in cells) of the Lees-Edwards row: floor(off / cs_x).
__device__ __forceinline__ int le_shift_cells(const InstGeo& g, double off) {
  return (int)floor(off * g.inv_cs[0]);
}

// FP32 conservative prefilter.  Positions are stored relative to their cell
// origin in FP32 (|error| <= 2^-24 cs).  For a candidate in a stencil cell
// with displacement (ox, oy, oz) the separation is
//   d = (xl_j - xl_i) + (o * cs [+ off for a Lees-Edwards image])
// up to a bounded rounding error; the decision is:
//   1: certainly a pair, 0: certainly not, -1: decide with exact_is_pair.
__device__ __forceinline__ int prefilter(const InstGeo& g, float4 pi, float4 pj, float cxo, float cyo,
                                         float czo, float s) {
  float dx = (pj.x - pi.x) + cxo;
  float dy = (pj.y - pi.y) + cyo;
  float dz = (pj.z - pi.z) + czo;
  if (fabsf(dx) > g.halfLf[0] || fabsf(dy) > g.halfLf[1] || fabsf(dz) > g.halfLf[2]) return -1;
  float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
  float s2 = s * s;
  if (r2 < s2 - g.r2_margin) return 1;
  if (r2 > s2 + g.r2_margin) return 0;
  return -1;
}

// FP32 displacement of a stencil cell's origin (cells ox, oy, oz away; for a
// Lees-Edwards image plus the offset off = fsh*cs_x + offr, offr in [0, cs_x)),
// computed without any FP64 instruction.
__device__ __forceinline__ void stencil_shift(const InstGeo& g, int ox, int oy, int oz, int le,
                                              int fsh, float offr, float& cx, float& cy,
                                              float& cz) {
  // le = 1: image one box above (shifted by +off), -1: one box below (-off)
  cx = le == 1 ? (float)(ox + fsh) * g.csf[0] + offr
               : (le == -1 ? (float)(ox - fsh) * g.csf[0] - offr : (float)ox * g.csf[0]);
  cy = (float)oy * g.csf[1];
  cz = (float)oz * g.csf[2];
}

__device__ __forceinline__ float pair_delta_f(const Geo& g, float ai, float aj) {
  if (g.mode == 1) return (float)(g.delta * g.a0);
  return (float)g.delta * (ai + aj) * 0.5f;
}

// ------------------------------------------------------------------------
// Decoupled look-back for single-pass scans (tiles taken in launch order
// through an atomic ticket, so every predecessor is already running).  One
// warp publishes the tile's aggregate, then polls 32 predecessors per round:
// it sums the aggregates up to the nearest predecessor holding an inclusive
// prefix.  Every wait is bounded; on give-up it reports DSS_ERR_TIMEOUT.
// Called by all 32 lanes of one warp; returns the exclusive prefix.
// ------------------------------------------------------------------------
constexpr unsigned long long kLbAgg = 1ull << 32;
constexpr unsigned long long kLbPre = 2ull << 32;
constexpr unsigned long long kWaitLimitNs = 500000000ull;   // a device wait gives up after 0.5 s

// Global nanosecond timer (the %globaltimer special register).
__device__ __forceinline__ unsigned long long dev_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int lookback_warp(unsigned long long* status, int tile, int agg,
                                             DevStatus* st) {
  const int lane = threadIdx.x & 31;
  if (tile == 0) {
    if (lane == 0) atomicExch(&status[0], kLbPre | (unsigned)agg);
    return 0;
  }
  if (lane == 0) atomicExch(&status[tile], kLbAgg | (unsigned)agg);
  int prefix = 0;
  int t = tile - 1;
  const unsigned long long t0 = dev_ns();
  long long spins = 0;
  while (true) {
    const int idx = t - lane;                 // lane 0: nearest predecessor
    const unsigned long long w = idx >= 0 ? atomicAdd(&status[idx], 0ull) : 0ull;
    const unsigned f = (unsigned)(w >> 32);
    const unsigned not_ready = __ballot_sync(0xffffffffu, f == 0u);
    const unsigned pre = __ballot_sync(0xffffffffu, f == 2u);
    const int p = pre ? __ffs(pre) - 1 : 32;
    const unsigned need = p == 32 ? 0xffffffffu : (p == 31 ? 0xffffffffu : ((2u << p) - 1u));
    if (not_ready & need) {
      // bounded: a predecessor that never publishes (an earlier failure)
      // ends the wait with DSS_ERR_TIMEOUT instead of a hang
      ++spins;
      const bool late = (spins & 63) == 0 && dev_ns() - t0 > kWaitLimitNs;
      if (__any_sync(0xffffffffu, late) || spins > (1ll << 24)) {
        if (lane == 0) set_err(st, DSS_ERR_TIMEOUT);
        break;
      }
      __nanosleep(20);
      continue;
    }
    int v = (lane <= p && idx >= 0) ? (int)(unsigned)(w & 0xffffffffull) : 0;
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    prefix += v;
    if (p < 32) break;
    t -= 32;
  }
  if (lane == 0) atomicExch(&status[tile], kLbPre | (unsigned)(prefix + agg));
  return prefix;
}

// ------------------------------------------------------------------------
// Double-float arithmetic (a value is hi + lo, |lo| <= ulp(hi)/2): error-free
// transformations of Knuth (TwoSum) and Dekker (TwoProduct, with FMA), used
// where the mixed-precision path needs more than FP32's 24 bits without
// touching GB300's narrow FP64 pipe.
// ------------------------------------------------------------------------
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return FF{s, e};
}
__device__ __forceinline__ FF fast_two_sum(float a, float b) {   // |a| >= |b|
  const float s = a + b;
  return FF{s, b - (s - a)};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  FF s = two_sum(a.hi, b.hi);
  const FF t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ FF ff_neg(FF a) { return FF{-a.hi, -a.lo}; }
// a + b for an FP32 increment b (TwoSum on the high words; the stretch
// changes sign, so no magnitude order is assumed)
__device__ __forceinline__ FF ff_add_f(FF a, float b) {
  const FF s = two_sum(a.hi, b);
  return two_sum(s.hi, s.lo + a.lo);
}
// a b for an FP32 factor b (Dekker's TwoProduct on the high word)
__device__ __forceinline__ FF ff_mul_f(FF a, float b) {
  const float p = a.hi * b;
  return fast_two_sum(p, fmaf(a.hi, b, -p) + a.lo * b);
}
// w whole cells of edge (cs_hi + cs_lo) as a double-float: the product of
// the FP32 words is made exact with Dekker's TwoProduct (w cs_hi needs more
// than 24 bits once |w| >= 3: a pair several cells apart, or across the
// Lees-Edwards layer).
__device__ __forceinline__ FF cell_shift(int w, float cs_hi, float cs_lo) {
  const float wf = (float)w;
  const float p = wf * cs_hi;
  return FF{p, fmaf(wf, cs_hi, -p) + wf * cs_lo};
}
__device__ __forceinline__ FF ff_sqr(FF a) {
  const float p = a.hi * a.hi;
  const float e = fmaf(a.hi, a.hi, -p);
  return fast_two_sum(p, e + 2.0f * a.hi * a.lo);
}

// ------------------------------------------------------------------------
// Host-side handle
// ------------------------------------------------------------------------
struct StateBuf {
  double* x;    // 3n positions
  double* u;    // 3n velocity (u^{n+1/2} after the sort of a step)
  double* w;    // 3n angular velocity
  double* al;   // 3n linear acceleration
  double* aw;   // 3n angular acceleration
  double* a;    // n radius
  int* id;      // n persistent id
  int* inst;    // n instance index
  unsigned char* cls;  // n size class (stencil reach), see Geo::rtab
  int* iy;      // n Lees-Edwards image count along y since the state was set (unwrapped y = y + iy L_y)
  float4* vf;   // n, mixed precision: FP32 velocity relative to U_inf (xyz); with the wave
                //    of Eq. 17, w = U k cos(k y) (the wave's part of the local rate)
  float4* wf;   // n, mixed precision: FP32 angular velocity relative to Omega_inf (xyz); with
                //    the wave, w = U sin(k y) (the wave's part of U_inf,x)
  double2* wv;  // n, wave of Eq. 17 on: (U sin(k y), U k cos(k y)) at the centre
  float4* posl; // n, mixed precision: low words of the cell-local position and radius
  int* cellc;   // n, mixed precision: cell coordinates packed cx | cy << 10 | cz << 20
};

// Tangential stretch of one listed pair and its contact flag (one 32-byte
// load or store).  FP64 precision: the components x, y, z and w = 1 when the
// pair was in contact, else 0.  Mixed precision: each component as a
// double-float, two FP32 words (hi, lo) in place of the double, and the flag
// as FP32 1 in the first word of w: words {x.hi, x.lo, y.hi, y.lo, z.hi,
// z.lo, flag, 0}, so the stretch is carried with ~48 significant bits and
// updated without GB300's narrow FP64 pipe.  Either way the record is all
// zero bits when the pair was not in contact (xi_flag).
struct __align__(32) Xi4 {
  double x, y, z, w;
};

__device__ __forceinline__ bool xi_flag(const Xi4& v) { return __double_as_longlong(v.w) != 0; }
// double-float <-> the 8 bytes of one component (first word hi, second lo)
__device__ __forceinline__ double ff_word(FF v) {
  return __hiloint2double(__float_as_int(v.lo), __float_as_int(v.hi));
}
__device__ __forceinline__ FF word_ff(double d) {
  return FF{__int_as_float(__double2loint(d)), __int_as_float(__double2hiint(d))};
}
// FP64 components of a record (either layout)
__device__ __forceinline__ void xi_components(const Xi4& v, bool mixed, double o[3]) {
  if (mixed) {
    const FF a = word_ff(v.x), b = word_ff(v.y), c = word_ff(v.z);
    o[0] = (double)a.hi + (double)a.lo;
    o[1] = (double)b.hi + (double)b.lo;
    o[2] = (double)c.hi + (double)c.lo;
  } else {
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
  }
}
// a record from FP64 components (either layout; the double-float split is
// exact to ~2^-48)
__device__ __forceinline__ Xi4 xi_record(double x, double y, double z, bool contact, bool mixed) {
  if (!contact) return Xi4{0.0, 0.0, 0.0, 0.0};
  if (!mixed) return Xi4{x, y, z, 1.0};
  const float xh = (float)x, yh = (float)y, zh = (float)z;
  return Xi4{ff_word(FF{xh, (float)(x - (double)xh)}), ff_word(FF{yh, (float)(y - (double)yh)}),
             ff_word(FF{zh, (float)(z - (double)zh)}), ff_word(FF{1.0f, 0.0f})};
}

struct ListBuf {
  int* count;       // n half-list row lengths
  int* list;        // n*M partner sorted indices
  int* start;       // n+1 row offsets into the pair arrays (exclusive scan of count)
  Xi4* xi;          // pcap: tangential stretch (lo->hi orientation) per pair slot; w = 1
                    // when the pair was in contact (d < 0), else 0
  Xi4* xr;          // pcap when k_r > 0: rolling stretch (App. B) per pair slot (w unused)
  int* slot_of_id;  // n: sorted index of each id in this list's index space
  int* id_of_slot;  // n: id of each sorted index of this list
  int* pown;        // pcap: owner of each pair, in pair order (pair-balanced kernel)
  int* pj;          // pcap: partner of each pair (the rows, compacted)
};

// Buffers of the adjoint (reverse sweep over a rollout): per-step tapes of
// the replayed forward and the adjoint state.  Owned by the handle.
struct AdjTape {
  double* x;        // 3n sorted positions at the step's force evaluation
  double* u;        // 3n velocities u^{n+1/2} (or u^n for the initial evaluation)
  double* w;        // 3n angular velocities
  int* id;          // n ids of the sorted order
  int* start;       // n+1 CSR row offsets of the step's pairs
  int* op;          // pcap owner (sorted index) of each pair
  int* pj;          // pcap partner (sorted index)
  int* pold;        // pcap index of the pair in the previous step's list, -1 if none
  double* xo;       // 3*pcap stretch carried in (i -> j orientation), 0 if none
  double* xro;      // 3*pcap rolling stretch carried in (k_r > 0; else null)
  StepGeo* sg;      // Lees-Edwards geometry of the step (instance 0)
};

struct AdjBuf {
  int slots;
  int64_t pcap;
  AdjTape* tape;         // [slots] (host array of device pointers)
  int* P_host;           // [slots] pairs per taped step (pinned)
  double *xb, *ub, *wb, *ab, *bb;   // 3n adjoint state, id order
  double* Fb;            // 3n force cotangent, sorted order of the step
  double* Tb;            // 3n torque cotangent
  double* pout;          // 18*pcap per-pair input adjoints (i side 9, j side 9)
  int* bw_n;             // n partner records per particle
  int* bw_p;             // n*M pair indices of the partner records
  double* xib[2];        // 3*pcap stretch adjoints of the current / previous step's pairs
  double* xrb[2];        // 3*pcap rolling-stretch adjoints (k_r > 0; else null)
  double* thb_part;      // 5 per pair block
  double* thb;           // 5: kn, kt, gamma_n, mu, delta_lub
  double* J;             // objective
  double* W;             // [nsteps][9] stress weights
  int64_t W_steps;
  int cur;               // which xib is the current step's
};

struct dss_handle {
  dss_params p;
  int64_t n;                 // particles of all instances
  int K;                     // instances
  InstGeo* ig_host;          // K (host)
  InstGeo* ig;               // K (device)
  StepGeo* sg;               // K (device): Lees-Edwards geometry of the current operation
  double* inst_box;          // 3K (host) box edges
  double* inst_gdot;         // K (host) shear rates
  double* inst_gn;           // K (host) dashpots
  int64_t* inst_n;           // K (host) particle counts
  cudaStream_t stream;       // stream all work is issued on
  cudaStream_t user_stream;  // the caller's stream (NULL: legacy default stream)
  bool own_stream;           // stream created by the library (caller passed NULL)
  cudaEvent_t ev_enter;
  // per-kernel timing of captured steps (dss_set_profiling)
  bool profiling;
  bool capturing;
  cudaEvent_t prof_ev[DSS_PROF_KERNELS + 1];
  cudaEvent_t step_ev[2];    // around the graph launches of one dss_step call
  double last_step_ms;
  double prof_ms[DSS_PROF_KERNELS];
  int64_t prof_count;
  double* a_by_id;           // n radii in id order (dss_load_state)
  int device;
  int sms;                   // streaming multiprocessors of the device
  bool have_state;
  bool sized;
  double a_min, a_max;
  double cell_edge;          // cell edge the grid was built for
  Geo g;
  // state: cur holds the committed state; the other buffer is scratch
  StateBuf st[2];
  int cur;
  // sorted-order extras of the last sort (belong to st[cur] after a sort)
  float4* posf;      // n: cell-local FP32 position + radius
  int* cellid;       // n
  int* perm;         // n: new sorted index -> previous index
  double* pred;      // 6n: predicted position and velocity of a step, source order
  signed char* xc;   // n: the step's y crossing of each particle (source order): -1 out through
                     // the top, +1 through the bottom
  double* mark;      // 2n (analysis): unwrapped y and v_y of each id at the marked time
  int64_t mark_nstep;
  bool marked;
  // counting sort scratch
  int* key;          // n
  int* offs;         // n
  int* cell_count;   // ncell
  int* cell_start;   // ncell+1
  int* tmp;          // n
  // lists: hist = committed (history source), work = being built
  ListBuf lb[2];
  int hist;
  // force accumulation of the last force pass (FP32 in mixed precision)
  void* own;         // 6n: force and torque summed over each particle's own row
  void* carry;       // per warp of 32 pairs, the sums of the owners whose pairs continue
                     // from the previous warp and into the next: force and torque (6 + 6;
                     // batched instances also the stresslet, 15 + 15)
  void* own_s;       // batched instances: 9n, each owner's stresslet sum (Eq. 9)
  int pb_blocks;     // blocks of the pair-balanced pair kernel (0: owner rows)
  bool compact_ok[2];  // the list's compact pair arrays were written by its last enumeration
                       // (false after the pair buffers are reallocated)
  int* bw_count;     // n: records appended to each particle's partner row
  void* bw_rec;      // n*M slots of 8 values: partner force (3), torque (3), owner index
  int64_t pcap;
  // stress
  double* spart;     // 18 per pair block: stresslet sums for the block's first instance and the next
  int spart_blocks;
  double* sigma;     // 9K: stress of each instance at the last force pass
  double* sigma_sum; // 9K: sum over committed steps since the last reset
  int64_t mean_steps;         // steps summed in sigma_sum
  int* inst_map;     // n: instance of each index in instance-major (id) order
  unsigned char* cls_map;   // n: size class of each id
  unsigned int* done_blocks;  // last-block counter of the gather (reset by that block)
  // scans
  unsigned long long* scan_status;  // tile status words (2 scans)
  int* scan_ticket;                 // 2 tickets
  int scan_tiles_max;
  // status
  DevStatus* status;
  DevStatus* status_host;           // pinned mirror
  // user-order io scratch
  double* io3;       // 3n
  double* io3b;      // 3n
  double* stage;     // 15n: staging of the five state vectors for host transfers
  int* io_id;        // n
  int last_list;     // list written by the last enumeration
  // graphs: one per (cur, hist) combination
  cudaGraphExec_t step_graph[4];
  bool graph_ok[4];
  // DSS_MULTI_STEPS consecutive steps in one graph (an even count: the
  // buffers are back in their roles after it), one per (cur, hist) start
  cudaGraphExec_t multi_graph[4];
  bool multi_ok[4];
  // kernel shapes chosen by dss_autotune_kernels (0: the built-in rule):
  // resident pair blocks per SM the register budget is cut for (3 or 4), and
  // candidates loaded ahead in the enumeration's loop (1 or 4)
  int tune_pairs_minb;
  int tune_enum_unr;
  int64_t bytes;
  int64_t host_steps_done;
  AdjBuf* adj;               // adjoint buffers (allocated by dss_adjoint)
};

// Kernel launchers (defined in the .cu files).  adv = 1 inside a time step
// (positions are at time (nstep+1) dt), 0 for an evaluation at the current
// time.
void launch_sort(dss_handle* h, bool predict, int src, int dst);
void launch_enumerate(dss_handle* h, int stbuf, int dst_list, int adv);
enum GatherMode { G_STEP = 0, G_EVAL = 1, G_ACCEL = 2 };
void launch_forces(dss_handle* h, int stbuf, int work_list, int hist_list, int adv, int mode,
                   double* F_out, double* T_out);
void launch_pairs_out(dss_handle* h, int list, long long* out);
void launch_images_out(dss_handle* h, int* out);
void launch_mark(dss_handle* h);
void launch_dispersion(dss_handle* h, double* sums);
void launch_clusters(dss_handle* h, int* parent, int* minid, int* count, int* label);
void launch_phi_profile(dss_handle* h, int nbins, double a_split, const double* unit, unsigned long long* acc);
int pair_grid_blocks(const dss_handle* h);
int pair_pb_blocks(const dss_handle* h);
void launch_scan(dss_handle* h, const int* in, int* out, int count, int which, bool zero_in);
int scan_tiles_for(int count);
int enum_tiles_for(int n);
double echem_range(const dss_params* p);
int enum_scan_tiles_for(int n);
int bw_slot_values();
// Marks the start of kernel k of a step when profiling (event record node
// when the step is being captured).
void prof_mark(dss_handle* h, int k);

// Adjoint (dss_adjoint.cu).
int adj_alloc(dss_handle* h, int slots, int64_t nsteps);
void adj_free(dss_handle* h);
int adj_upload_weights(dss_handle* h, const double* W, int64_t nsteps);
void adj_zero(dss_handle* h);
void adj_accum_J(dss_handle* h, int64_t step);
void adj_tape(dss_handle* h, int slot, int stbuf, int list, int hist_list, bool empty_history);
void adj_reverse(dss_handle* h, int slot, int64_t step, bool initial);
