/*
 * Plain CPU FP64 oracle for the per-timestep path of the dense-suspension
 * solver of Monti, Rathee, Shen & Rosti, "A fast and efficient tool to study
 * the rheology of dense suspensions" (arXiv:2108.01013).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * definition that the CUDA path is checked against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product path never calls it and shares no code, header, table or constant
 * with it.
 *
 * Conventions (Sec. II): flow along x, gradient along y, vorticity along z;
 * U_inf = (gdot*y, 0, 0), E_inf_xy = E_inf_yx = gdot/2, Omega_inf =
 * (0, 0, -gdot/2); in the wavy shear flow of Eq. 17 U_inf,x gains
 * U sin(2 pi n y / L_y) and E_inf, Omega_inf follow the local rate
 * dU_inf,x/dy.  Arrays are SoA: v[0*n+i], v[1*n+i], v[2*n+i].
 * Neighbour pairs come from an O(N^2) brute-force scan (the plain definition
 * of the fixed-radius near-neighbour set) or, on request, from a cell list
 * with the paper's half stencil (Sec. II A) that is checked to give the same
 * set; either set is sorted by (i, j) and evaluated in that order, so both
 * give the same numbers bit for bit.  Pairs are evaluated on all host cores
 * (OpenMP, each pair on its own) and summed in the set's order.
 *
 * Readings of the paper that this file takes (each one is listed in the
 * design notes of the repository):
 *  - lubrication prefactor 6*pi*eta0 on every block of App. A (the g
 *    coefficients carry only lengths);
 *  - lubrication acts on every listed pair; a pair is listed when its centre
 *    distance r obeys r^2 < (a_i + a_j + delta_ij)^2 with
 *    delta_ij = delta_lub*(a_i+a_j)/2 (mode 0, i.e. d* < delta_lub) or
 *    delta_ij = delta_lub*a0 (mode 1);
 *  - X and Y use max(d*,0)+eps (no sign flip when particles overlap);
 *  - the omega-omega blocks of Eq. A2 use the tangential projector T, the
 *    torque-velocity blocks are the transposes of the force-rotation blocks;
 *  - g^{Y^H_ji}(alpha) = g^{Y^H_ij}(1/alpha);
 *  - n_perp = n x [(E+E^T) n] (the factor that makes the torque on two
 *    particles at rest in a linear flow vanish at contact);
 *  - Lees-Edwards velocity jump of gdot*L_y on a y wrap (Eq. 16);
 *  - tangential spring: xi <- T.xi_old + u_t dt, then the Coulomb rescale of
 *    Eq. 5 with |F_nor| including the dashpot; history lives while d < 0,
 *    stored for the (lower id -> higher id) orientation;
 *  - u^{n+1} = u^{n+1/2} + dt/2 alpha^{n+1}, algebraically Eq. 15d, so that a
 *    Lees-Edwards velocity jump applied to u^{n+1/2} carries over;
 *  - each pair's stresslet is counted once in Eq. 8;
 *  - wavy flow (Eq. 17): n a whole number (the wave is L_y-periodic); the
 *    Stokes drag takes the Faxen velocity (1 + a^2/6 Laplacian) U_inf and
 *    the local Omega_inf at the centre (Eq. A1: no Laplacian on rotation);
 *    lubrication takes V and W at each centre and the strain of the mean of
 *    the two centres' local rates; the single-particle stresslet takes
 *    E_inf at the centre (no Laplacian), the fluid term 2 eta0 E_inf the box
 *    mean gdot; default velocities are U_inf and Omega_inf at the centre;
 *  - rolling resistance (App. B): u_r = abar (n x w_i - n x w_j), the
 *    Coulomb limit mu |F_nor| / k_r with the sliding contact's mu and normal
 *    force, torques only (no force, no stresslet), the stretch lives with
 *    the contact like the sliding one;
 *  - optional lubrication taper (an extension for differentiation, not in
 *    the paper): with w = lub_taper > 0 the lubrication force, torques and
 *    stresslet of a listed pair are scaled by s = t^2 (3 - 2t),
 *    t = clamp((delta_ij - d) / (w delta_ij), 0, 1), so that they fall to
 *    zero continuously at the cutoff; w = 0 is the hard cutoff.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct orc_params {
  double kn, kt, gamma_n, mu;   /* Eq. 4: spring, tangential spring, dashpot, Coulomb */
  double eta0, rho;             /* fluid viscosity, particle density */
  double delta_lub, lub_eps;    /* lubrication cutoff, regulariser eps of Eq. A6 */
  double a0;                    /* reference radius (mode-1 cutoff) */
  int32_t lub_cutoff_mode;      /* 0: d* < delta_lub, 1: d < delta_lub*a0 */
  int32_t pad_;
  double shear_rate, dt;        /* gdot, time step */
  double L[3];                  /* box edges */
  double lub_taper;             /* w of the lubrication taper; 0: hard cutoff */
  double f_er, lambda_d;        /* Eq. 6 (repulsion): magnitude F_ER, Debye length */
  double hamaker, vdw_eps;      /* Eq. 7 (attraction): Hamaker constant A, eps / abar */
  double wave_amp;              /* Eq. 17: amplitude U of the wavy part of U_inf; 0: simple shear */
  double k_r;                   /* App. B: rolling spring stiffness; 0: no rolling resistance */
  int32_t wave_n;               /* Eq. 17: number n of periods of the wave along L_y */
  int32_t pad2_;
} orc_params;

typedef struct orc_sys {
  orc_params p;
  int64_t n;
  double *x, *u, *w, *al, *aw;  /* position, velocity, angular velocity, accelerations */
  double *a;                    /* radius */
  int32_t *id;                  /* persistent id */
  double *F, *T;                /* total force/torque of the last evaluation */
  double *Fa, *Ta;              /* sums of the magnitudes of the terms of F and T (per pair the
                                   contact, each lubrication sub-term, the electro-chemical and
                                   rolling terms; the drag): the scale of the rounding error of
                                   any evaluation that forms these terms and sums them */
  double sigma[9];              /* bulk stress of the last evaluation, row major */
  int64_t nstep;                /* time t = nstep*dt */
  int64_t hk, hcap;             /* contact history: sorted keys lo<<32|hi */
  int64_t *hkey;
  int64_t *iy;                  /* Lees-Edwards image count along y (unwrapped y = y + iy L_y) */
  double *hxi;                  /* [hk][3], orientation lo -> hi */
  double *hxr;                  /* [hk][3], rolling stretch (the same in both orientations) */
  int64_t npairs_last, ncontacts_last;
  int cells;                    /* neighbour search: 0 brute force, 1 cell list (same pair set) */
} orc_sys;

/* ------------------------------------------------------------------------ */
/* Geometry: Lees-Edwards offset and minimum image                           */
/* ------------------------------------------------------------------------ */

/* Eq. 16: the image boxes above/below are displaced along x by
 * gdot*L_y*t, taken modulo L_x and computed from the integer step count. */
double orc_le_offset(const orc_params *p, int64_t nstep) {
  double t = (double)nstep * p->dt;
  return fmod(p->shear_rate * p->L[1] * t, p->L[0]);
}

/* Minimum-image separation r = x_j - x_i under Lees-Edwards conditions.
 * sy = -1 when the image of j sits one box below (y_j - L_y, x_j - off),
 * +1 when it sits one box above, 0 otherwise. */
static void min_image(const orc_params *p, double off, const double xi[3],
                      const double xj[3], double r[3], int *sy) {
  double dx = xj[0] - xi[0];
  double dy = xj[1] - xi[1];
  double dz = xj[2] - xi[2];
  int s = 0;
  if (dy > 0.5 * p->L[1]) {
    dy = dy - p->L[1];
    dx = dx - off;
    s = -1;
  } else if (dy < -0.5 * p->L[1]) {
    dy = dy + p->L[1];
    dx = dx + off;
    s = 1;
  }
  dx = dx - p->L[0] * rint(dx / p->L[0]);
  dz = dz - p->L[2] * rint(dz / p->L[2]);
  r[0] = dx; r[1] = dy; r[2] = dz;
  *sy = s;
}

/* The lubrication cutoff delta_lub of Sec. II (Fig. 1) expressed as a
 * surface distance for the pair. */
static double lub_delta(const orc_params *p, double ai, double aj) {
  if (p->lub_cutoff_mode == 1) return p->delta_lub * p->a0;
  return p->delta_lub * (ai + aj) * 0.5;
}

/* Range of the electro-chemical forces (Fig. 3): the repulsion acts below a
 * surface distance of 20 lambda_D, the attraction below 4 a0; 0 when both
 * are off. */
double orc_echem_range(const orc_params *p) {
  double r = 0.0;
  if (p->f_er > 0.0 && 20.0 * p->lambda_d > r) r = 20.0 * p->lambda_d;
  if (p->hamaker > 0.0 && 4.0 * p->a0 > r) r = 4.0 * p->a0;
  return r;
}

/* Interaction range beyond contact: the larger of the lubrication cutoff and
 * the electro-chemical range. */
static double pair_delta(const orc_params *p, double ai, double aj) {
  double dl = lub_delta(p, ai, aj), de = orc_echem_range(p);
  return de > dl ? de : dl;
}

/* Neighbour predicate: r^2 < (a_i + a_j + delta_ij)^2 (strict). */
static int is_pair(const orc_params *p, const double r[3], double ai, double aj) {
  double r2 = (r[0] * r[0] + r[1] * r[1]) + r[2] * r[2];
  double s = (ai + aj) + pair_delta(p, ai, aj);
  return r2 < s * s;
}

/* Lubrication acts on a listed pair iff it is within the lubrication cutoff
 * (the same strict test with the lubrication range alone). */
static int in_lub_range(const orc_params *p, const double r[3], double ai, double aj) {
  double r2 = (r[0] * r[0] + r[1] * r[1]) + r[2] * r[2];
  double s = (ai + aj) + lub_delta(p, ai, aj);
  return r2 < s * s;
}

static int cmp_i64pair(const void *A, const void *B) {
  const int64_t *a = (const int64_t *)A, *b = (const int64_t *)B;
  if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1;
  if (a[1] != b[1]) return a[1] < b[1] ? -1 : 1;
  return 0;
}

/* Brute-force fixed-radius near-neighbour set: every unordered pair whose
 * minimum-image distance passes the predicate.  Written out as (lo id, hi id)
 * sorted lexicographically.  Returns the number of pairs; at most cap are
 * written. */
int64_t orc_pairs_bruteforce(int64_t n, const double *x, const double *a,
                             const int32_t *id, const orc_params *p,
                             double off, int64_t *out, int64_t cap) {
  int64_t cnt = 0, alloc = 1024;
  int64_t *buf = (int64_t *)malloc(sizeof(int64_t) * 2 * alloc);
  for (int64_t i = 0; i < n; ++i) {
    double xi[3] = {x[i], x[n + i], x[2 * n + i]};
    for (int64_t j = i + 1; j < n; ++j) {
      double xj[3] = {x[j], x[n + j], x[2 * n + j]};
      double r[3];
      int sy;
      min_image(p, off, xi, xj, r, &sy);
      if (!is_pair(p, r, a[i], a[j])) continue;
      if (cnt == alloc) {
        alloc *= 2;
        buf = (int64_t *)realloc(buf, sizeof(int64_t) * 2 * alloc);
      }
      int64_t lo = id[i] < id[j] ? id[i] : id[j];
      int64_t hi = id[i] < id[j] ? id[j] : id[i];
      buf[2 * cnt] = lo;
      buf[2 * cnt + 1] = hi;
      ++cnt;
    }
  }
  qsort(buf, (size_t)cnt, sizeof(int64_t) * 2, cmp_i64pair);
  int64_t m = cnt < cap ? cnt : cap;
  if (out && m > 0) memcpy(out, buf, sizeof(int64_t) * 2 * (size_t)m);
  free(buf);
  return cnt;
}

/* Neighbours of a single particle k (by array index), brute force over all
 * others; used to check sampled rows at sizes where the full O(N^2) scan is
 * too slow.  Writes partner ids (unsorted order of the scan). */
int64_t orc_neighbours_of(int64_t n, const double *x, const double *a,
                          const int32_t *id, const orc_params *p, double off,
                          int64_t k, int64_t *out, int64_t cap) {
  int64_t cnt = 0;
  double xk[3] = {x[k], x[n + k], x[2 * n + k]};
  for (int64_t j = 0; j < n; ++j) {
    if (j == k) continue;
    double xj[3] = {x[j], x[n + j], x[2 * n + j]};
    double r[3];
    int sy;
    min_image(p, off, xk, xj, r, &sy);
    if (!is_pair(p, r, a[k], a[j])) continue;
    if (cnt < cap) out[cnt] = id[j];
    ++cnt;
  }
  return cnt;
}

/* ------------------------------------------------------------------------ */
/* Small vector helpers                                                      */
/* ------------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
/* T.v = v - n (n.v) */
static void tproj(const double n[3], const double v[3], double o[3]) {
  double s = dot3(n, v);
  o[0] = v[0] - n[0] * s; o[1] = v[1] - n[1] * s; o[2] = v[2] - n[2] * s;
}
/* N.v = n (n.v) */
static void nproj(const double n[3], const double v[3], double o[3]) {
  double s = dot3(n, v);
  o[0] = n[0] * s; o[1] = n[1] * s; o[2] = n[2] * s;
}

/* A shear along x with local rate g = dU_x/dy: E_inf (3x3, row major) with
 * E_xy = E_yx = g/2 and Omega_inf = curl(U_inf)/2 = (0, 0, -g/2). */
static void ambient_rate(double g, double E[9], double Om[3]) {
  memset(E, 0, 9 * sizeof(double));
  E[0 * 3 + 1] = 0.5 * g;
  E[1 * 3 + 0] = 0.5 * g;
  Om[0] = 0.0; Om[1] = 0.0; Om[2] = -0.5 * g;
}

/* Ambient simple shear of Sec. II (the box mean of the flow of Eq. 17). */
static void ambient(const orc_params *p, double E[9], double Om[3]) {
  ambient_rate(p->shear_rate, E, Om);
}

/* ------------------------------------------------------------------------ */
/* Wavy shear flow, Eq. 17: U_inf = (gdot y + U sin(k y), 0, 0) with         */
/* k = 2 pi n / L_y (n = 0 or U = 0: the simple shear).  The wave is         */
/* L_y-periodic, so the Lees-Edwards velocity jump stays gdot L_y.           */
/* ------------------------------------------------------------------------ */
static double wave_k(const orc_params *p) { return 2.0 * M_PI * (double)p->wave_n / p->L[1]; }

/* U_inf,x at height y. */
double orc_flow_ux(const orc_params *p, double y) {
  return p->shear_rate * y + p->wave_amp * sin(wave_k(p) * y);
}

/* Local shear rate dU_inf,x/dy at height y (E_xy = rate/2, Omega_z = -rate/2). */
double orc_flow_rate(const orc_params *p, double y) {
  double k = wave_k(p);
  return p->shear_rate + p->wave_amp * k * cos(k * y);
}

/* The Faxen velocity of Eq. A1: (1 + a^2/6 Laplacian) U_inf,x at height y
 * for a sphere of radius a; the Laplacian of sin(k y) is -k^2 sin(k y). */
double orc_faxen_ux(const orc_params *p, double y, double a) {
  double k = wave_k(p);
  return p->shear_rate * y + p->wave_amp * (1.0 - a * a * k * k / 6.0) * sin(k * y);
}

/* ------------------------------------------------------------------------ */
/* Contact: stick-and-slide model, Eq. 4 and Eq. 5                            */
/* ------------------------------------------------------------------------ */

/* Contact force on i from j, torques on i and j, and the updated tangential
 * stretch.  r = x_j - x_i (image), uj is the image velocity of j.  xi_old is
 * the stretch in the i -> j orientation (zero at the start of a contact). */
void orc_contact(const orc_params *p, const double r[3], double ai, double aj,
                 const double ui[3], const double uj[3], const double wi[3],
                 const double wj[3], const double xi_old[3], double Fi[3],
                 double Ti[3], double Tj[3], double xi_new[3]) {
  double dist = sqrt(dot3(r, r));
  double n[3] = {r[0] / dist, r[1] / dist, r[2] / dist};
  double d = dist - (ai + aj);
  double du[3] = {uj[0] - ui[0], uj[1] - ui[1], uj[2] - ui[2]};
  /* normal: F_nor = k_n d n + gamma_n (n n).(u_j - u_i) */
  double un[3];
  nproj(n, du, un);
  double Fnor[3];
  for (int c = 0; c < 3; ++c) Fnor[c] = p->kn * d * n[c] + p->gamma_n * un[c];
  /* tangential velocity of the contact point: T.(u_j - u_i - (a_i w_i + a_j w_j) x n) */
  double aw[3] = {ai * wi[0] + aj * wj[0], ai * wi[1] + aj * wj[1], ai * wi[2] + aj * wj[2]};
  double awxn[3];
  cross3(aw, n, awxn);
  double rel[3] = {du[0] - awxn[0], du[1] - awxn[1], du[2] - awxn[2]};
  double ut[3];
  tproj(n, rel, ut);
  /* stretch: project the old stretch on the current tangent plane, integrate */
  double xp[3];
  tproj(n, xi_old, xp);
  double xs[3] = {xp[0] + ut[0] * p->dt, xp[1] + ut[1] * p->dt, xp[2] + ut[2] * p->dt};
  /* Coulomb limit |k_t xi| <= mu |F_nor| */
  double cap = p->mu * sqrt(dot3(Fnor, Fnor)) / p->kt;
  double xm = sqrt(dot3(xs, xs));
  if (xm > cap) {
    double f = cap / xm;
    xs[0] *= f; xs[1] *= f; xs[2] *= f;
  }
  double Ftan[3] = {p->kt * xs[0], p->kt * xs[1], p->kt * xs[2]};
  for (int c = 0; c < 3; ++c) Fi[c] = Fnor[c] + Ftan[c];
  /* T_ij = a_i n x F_tan, T_ji = (a_j/a_i) T_ij */
  double nxf[3];
  cross3(n, Ftan, nxf);
  for (int c = 0; c < 3; ++c) {
    Ti[c] = ai * nxf[c];
    Tj[c] = (aj / ai) * Ti[c];
    xi_new[c] = xs[c];
  }
}

/* Rolling resistance, App. B (Eq. B1), after Luding: a rolling spring of
 * stiffness k_r whose stretch integrates the rolling velocity
 * u_r = abar (n x w_i - n x w_j), abar = 2 a_i a_j / (a_i + a_j), by the
 * procedure of Eq. 5 with u_r and k_r in place of u_t and k_t: the old
 * stretch projected on the current tangent plane plus u_r dt, rescaled so
 * that |k_r xi_r| <= mu |F_nor| (the Coulomb coefficient and the normal
 * force, dashpot included, of the sliding contact).  The pseudo-force
 * k_r xi_r acts through torques only: T_i = abar n x (k_r xi_r), T_j = -T_i.
 * u_r, and with it xi_r, is unchanged when i and j swap (n and w_i - w_j
 * both change sign). */
void orc_rolling(const orc_params *p, const double r[3], double ai, double aj,
                 const double ui[3], const double uj[3], const double wi[3],
                 const double wj[3], const double xr_old[3], double Ti[3], double Tj[3],
                 double xr_new[3]) {
  double dist = sqrt(dot3(r, r));
  double n[3] = {r[0] / dist, r[1] / dist, r[2] / dist};
  double d = dist - (ai + aj);
  double abar = 2.0 * ai * aj / (ai + aj);
  double du[3] = {uj[0] - ui[0], uj[1] - ui[1], uj[2] - ui[2]};
  double un[3];
  nproj(n, du, un);
  double Fnor[3];
  for (int c = 0; c < 3; ++c) Fnor[c] = p->kn * d * n[c] + p->gamma_n * un[c];
  double dw[3] = {wi[0] - wj[0], wi[1] - wj[1], wi[2] - wj[2]};
  double nxdw[3];
  cross3(n, dw, nxdw);
  double xp[3];
  tproj(n, xr_old, xp);
  double xs[3];
  for (int c = 0; c < 3; ++c) xs[c] = xp[c] + abar * nxdw[c] * p->dt;
  double cap = p->mu * sqrt(dot3(Fnor, Fnor)) / p->k_r;
  double xm = sqrt(dot3(xs, xs));
  if (xm > cap) {
    double f = cap / xm;
    xs[0] *= f; xs[1] *= f; xs[2] *= f;
  }
  double Fr[3] = {p->k_r * xs[0], p->k_r * xs[1], p->k_r * xs[2]};
  double nxf[3];
  cross3(n, Fr, nxf);
  for (int c = 0; c < 3; ++c) {
    Ti[c] = abar * nxf[c];
    Tj[c] = -Ti[c];
    xr_new[c] = xs[c];
  }
}

/* ------------------------------------------------------------------------ */
/* Lubrication: App. A, Eq. A2, A3 and the g coefficients of Eq. A7          */
/* alpha = a_j/a_i.  The jj and ji entries are obtained from the ii and ij   */
/* formulas evaluated at 1/alpha, with a_i and a_j left as they are, exactly */
/* as the relations of Eq. A7 are written.                                   */
/* ------------------------------------------------------------------------ */
static double gXA_ii(double al, double ai, double aj) { (void)aj; return 2.0 * ai * al * al / pow(1.0 + al, 3); }
static double gXA_ij(double al, double ai, double aj) { return -2.0 * (ai + aj) * al * al / pow(1.0 + al, 4); }
static double gYA_ii(double al, double ai, double aj) { (void)aj; return 4.0 * ai / 15.0 * al * (2.0 + al + 2.0 * al * al) / pow(1.0 + al, 3); }
static double gYA_ij(double al, double ai, double aj) { return -4.0 * (ai + aj) / 15.0 * al * (2.0 + al + 2.0 * al * al) / pow(1.0 + al, 4); }
static double gYB_ii(double al, double ai, double aj) { (void)aj; return -2.0 * ai * ai / 15.0 * al * (4.0 + al) / pow(1.0 + al, 2); }
static double gYB_ij(double al, double ai, double aj) { return 2.0 * pow(ai + aj, 2) / 15.0 * al * (4.0 + al) / pow(1.0 + al, 4); }
static double gYC_ii(double al, double ai, double aj) { (void)aj; return 8.0 * pow(ai, 3) / 15.0 * al / (1.0 + al); }
static double gYC_ij(double al, double ai, double aj) { return 2.0 * pow(ai + aj, 3) / 15.0 * al * al / pow(1.0 + al, 4); }
static double gXG_ii(double al, double ai, double aj) { (void)aj; return 2.0 * ai * ai * al * al / pow(1.0 + al, 3); }
static double gXG_ij(double al, double ai, double aj) { return -2.0 * pow(ai + aj, 2) * al * al / pow(1.0 + al, 5); }
static double gYG_ii(double al, double ai, double aj) { (void)aj; return ai * ai / 15.0 * al * (4.0 - al + 7.0 * al * al) / pow(1.0 + al, 3); }
static double gYG_ij(double al, double ai, double aj) { return -pow(ai + aj, 2) / 15.0 * al * (4.0 - al + 7.0 * al * al) / pow(1.0 + al, 5); }
static double gYH_ii(double al, double ai, double aj) { (void)aj; return 2.0 * pow(ai, 3) / 15.0 * al * (2.0 - al) / pow(1.0 + al, 2); }
static double gYH_ij(double al, double ai, double aj) { return pow(ai + aj, 3) / 15.0 * al * al * (1.0 + 7.0 * al) / pow(1.0 + al, 5); }

/* The full set of scalar resistances for one pair (Eq. A6, A7). */
typedef struct lub_coef {
  double XA_ii, XA_ij, XA_ji, XA_jj;
  double YA_ii, YA_ij, YA_ji, YA_jj;
  double YB_ii, YB_ij, YB_ji, YB_jj;
  double YC_ii, YC_ij, YC_ji, YC_jj;
  double XG_ii, XG_ij, XG_ji, XG_jj;
  double YG_ii, YG_ij, YG_ji, YG_jj;
  double YH_ii, YH_ij, YH_ji, YH_jj;
} lub_coef;

static void lub_coefficients(const orc_params *p, double d, double ai, double aj, lub_coef *c) {
  double ds = 2.0 * d / (ai + aj);      /* normalised gap d* */
  if (ds < 0.0) ds = 0.0;               /* overlap: stay at the contact value */
  double X = 1.0 / (ds + p->lub_eps);
  double Y = log(1.0 / (ds + p->lub_eps));
  double al = aj / ai, ial = 1.0 / al;
  c->XA_ii = X * gXA_ii(al, ai, aj);
  c->XA_jj = X * al * gXA_ii(ial, ai, aj);
  c->XA_ij = X * gXA_ij(al, ai, aj);
  c->XA_ji = X * gXA_ij(ial, ai, aj);
  c->YA_ii = Y * gYA_ii(al, ai, aj);
  c->YA_jj = Y * al * gYA_ii(ial, ai, aj);
  c->YA_ij = Y * gYA_ij(al, ai, aj);
  c->YA_ji = Y * gYA_ij(ial, ai, aj);
  c->YB_ii = Y * gYB_ii(al, ai, aj);
  c->YB_jj = Y * (-al * al) * gYB_ii(ial, ai, aj);
  c->YB_ij = Y * gYB_ij(al, ai, aj);
  c->YB_ji = Y * (-gYB_ij(ial, ai, aj));
  c->YC_ii = Y * gYC_ii(al, ai, aj);
  c->YC_jj = Y * al * al * al * gYC_ii(ial, ai, aj);
  c->YC_ij = Y * gYC_ij(al, ai, aj);
  c->YC_ji = Y * gYC_ij(ial, ai, aj);
  c->XG_ii = X * gXG_ii(al, ai, aj);
  c->XG_jj = X * (-al * al) * gXG_ii(ial, ai, aj);
  c->XG_ij = X * gXG_ij(al, ai, aj);
  c->XG_ji = X * (-gXG_ij(ial, ai, aj));
  c->YG_ii = Y * gYG_ii(al, ai, aj);
  c->YG_jj = Y * (-al * al) * gYG_ii(ial, ai, aj);
  c->YG_ij = Y * gYG_ij(al, ai, aj);
  c->YG_ji = Y * (-gYG_ij(ial, ai, aj));
  c->YH_ii = Y * gYH_ii(al, ai, aj);
  c->YH_jj = Y * al * al * al * gYH_ii(ial, ai, aj);
  c->YH_ij = Y * gYH_ij(al, ai, aj);
  c->YH_ji = Y * gYH_ij(ial, ai, aj);
}

/* Lubrication forces and torques on i and j (Eq. 3 without the Stokes part):
 *   (F_i,F_j,T_i,T_j) = -6 pi eta0 R_Lub.(V_i,V_j,W_i,W_j) + 6 pi eta0 R'_Lub.(n,n,n_perp,n_perp)
 * with V = u - U_inf(x), W = omega - Omega_inf (particle-by-particle),
 * r = x_j - x_i and the strain E_inf of a shear of local rate `rate` along x.
 * Each block of Eq. A2/A3 is applied as written. */
/* mag (may be NULL): the sums of the magnitudes of the sub-terms of F_i,
 * F_j, T_i, T_j (each coefficient times its projected velocity, angular
 * velocity or strain vector), the scale of the rounding of any evaluation
 * that forms the sub-terms separately; a diagnostic for the parity checks
 * that does not change the result. */
static void lubrication_core(const orc_params *p, double rate, const double r[3], double ai,
                             double aj, const double Vi[3], const double Vj[3],
                             const double Wi[3], const double Wj[3], double Fi[3], double Fj[3],
                             double Ti[3], double Tj[3], double mag[4]) {
  double dist = sqrt(dot3(r, r));
  double n[3] = {r[0] / dist, r[1] / dist, r[2] / dist};
  double d = dist - (ai + aj);
  lub_coef c;
  lub_coefficients(p, d, ai, aj, &c);
  double E[9], Om[3];
  ambient_rate(rate, E, Om);
  (void)Om;
  /* projections of each velocity */
  double NVi[3], TVi[3], NVj[3], TVj[3], TWi[3], TWj[3], nxVi[3], nxVj[3], nxWi[3], nxWj[3];
  nproj(n, Vi, NVi); tproj(n, Vi, TVi);
  nproj(n, Vj, NVj); tproj(n, Vj, TVj);
  tproj(n, Wi, TWi); tproj(n, Wj, TWj);
  cross3(n, Vi, nxVi); cross3(n, Vj, nxVj);
  cross3(n, Wi, nxWi); cross3(n, Wj, nxWj);
  /* strain operators: P = E:nn - Tr(E)/3, Q.n = 2 E.n - 2 (E:nn) n,
   * n_perp = n x [(E + E^T).n] */
  double En[3] = {E[0] * n[0] + E[1] * n[1] + E[2] * n[2],
                  E[3] * n[0] + E[4] * n[1] + E[5] * n[2],
                  E[6] * n[0] + E[7] * n[1] + E[8] * n[2]};
  double EnT[3] = {E[0] * n[0] + E[3] * n[1] + E[6] * n[2],
                   E[1] * n[0] + E[4] * n[1] + E[7] * n[2],
                   E[2] * n[0] + E[5] * n[1] + E[8] * n[2]};
  double Enn = dot3(n, En);
  double trE = E[0] + E[4] + E[8];
  double P = Enn - trE / 3.0;
  double Qn[3] = {2.0 * En[0] - 2.0 * Enn * n[0], 2.0 * En[1] - 2.0 * Enn * n[1],
                  2.0 * En[2] - 2.0 * Enn * n[2]};
  double sE[3] = {En[0] + EnT[0], En[1] + EnT[1], En[2] + EnT[2]};
  double nperp[3];
  cross3(n, sE, nperp);
  double k = 6.0 * M_PI * p->eta0;
  for (int q = 0; q < 3; ++q) {
    /* row F_i: [XA_ii N + YA_ii T, XA_ij N + YA_ij T, YB_ii nx, YB_ji nx] */
    double fi = c.XA_ii * NVi[q] + c.YA_ii * TVi[q] + c.XA_ij * NVj[q] + c.YA_ij * TVj[q] +
                c.YB_ii * nxWi[q] + c.YB_ji * nxWj[q];
    /* row F_j: [XA_ji N + YA_ji T, XA_jj N + YA_jj T, YB_ij nx, YB_jj nx] */
    double fj = c.XA_ji * NVi[q] + c.YA_ji * TVi[q] + c.XA_jj * NVj[q] + c.YA_jj * TVj[q] +
                c.YB_ij * nxWi[q] + c.YB_jj * nxWj[q];
    /* row T_i: [-YB_ii nx, -YB_ij nx, YC_ii T, YC_ij T] */
    double ti = -c.YB_ii * nxVi[q] - c.YB_ij * nxVj[q] + c.YC_ii * TWi[q] + c.YC_ij * TWj[q];
    /* row T_j: [-YB_ji nx, -YB_jj nx, YC_ji T, YC_jj T] */
    double tj = -c.YB_ji * nxVi[q] - c.YB_jj * nxVj[q] + c.YC_ji * TWi[q] + c.YC_jj * TWj[q];
    /* strain terms, Eq. A3: columns act on (n, n) for forces, (n_perp, n_perp) for torques */
    double gi = (c.XG_ii * P * n[q] + c.YG_ii * Qn[q]) + (c.XG_ji * P * n[q] + c.YG_ji * Qn[q]);
    double gj = (c.XG_ij * P * n[q] + c.YG_ij * Qn[q]) + (c.XG_jj * P * n[q] + c.YG_jj * Qn[q]);
    double hi = c.YH_ii * nperp[q] + c.YH_ji * nperp[q];
    double hj = c.YH_ij * nperp[q] + c.YH_jj * nperp[q];
    Fi[q] = -k * fi + k * gi;
    Fj[q] = -k * fj + k * gj;
    Ti[q] = -k * ti + k * hi;
    Tj[q] = -k * tj + k * hj;
  }
  if (mag) {
    double nNVi = sqrt(dot3(NVi, NVi)), nTVi = sqrt(dot3(TVi, TVi)), nNVj = sqrt(dot3(NVj, NVj));
    double nTVj = sqrt(dot3(TVj, TVj)), nWi = sqrt(dot3(nxWi, nxWi)), nWj = sqrt(dot3(nxWj, nxWj));
    double nVi = sqrt(dot3(nxVi, nxVi)), nVj = sqrt(dot3(nxVj, nxVj));
    double nTWi = sqrt(dot3(TWi, TWi)), nTWj = sqrt(dot3(TWj, TWj));
    double nQ = sqrt(dot3(Qn, Qn)), nP = fabs(P), nH = sqrt(dot3(nperp, nperp));
    mag[0] = k * (fabs(c.XA_ii) * nNVi + fabs(c.YA_ii) * nTVi + fabs(c.XA_ij) * nNVj +
                  fabs(c.YA_ij) * nTVj + fabs(c.YB_ii) * nWi + fabs(c.YB_ji) * nWj +
                  (fabs(c.XG_ii) + fabs(c.XG_ji)) * nP + (fabs(c.YG_ii) + fabs(c.YG_ji)) * nQ);
    mag[1] = k * (fabs(c.XA_ji) * nNVi + fabs(c.YA_ji) * nTVi + fabs(c.XA_jj) * nNVj +
                  fabs(c.YA_jj) * nTVj + fabs(c.YB_ij) * nWi + fabs(c.YB_jj) * nWj +
                  (fabs(c.XG_ij) + fabs(c.XG_jj)) * nP + (fabs(c.YG_ij) + fabs(c.YG_jj)) * nQ);
    mag[2] = k * (fabs(c.YB_ii) * nVi + fabs(c.YB_ij) * nVj + fabs(c.YC_ii) * nTWi +
                  fabs(c.YC_ij) * nTWj + (fabs(c.YH_ii) + fabs(c.YH_ji)) * nH);
    mag[3] = k * (fabs(c.YB_ji) * nVi + fabs(c.YB_jj) * nVj + fabs(c.YC_ji) * nTWi +
                  fabs(c.YC_jj) * nTWj + (fabs(c.YH_ij) + fabs(c.YH_jj)) * nH);
  }
}

void orc_lubrication_rate(const orc_params *p, double rate, const double r[3], double ai,
                          double aj, const double Vi[3], const double Vj[3],
                          const double Wi[3], const double Wj[3], double Fi[3], double Fj[3],
                          double Ti[3], double Tj[3]) {
  lubrication_core(p, rate, r, ai, aj, Vi, Vj, Wi, Wj, Fi, Fj, Ti, Tj, NULL);
}

/* The same in the simple shear of rate gdot. */
void orc_lubrication(const orc_params *p, const double r[3], double ai, double aj,
                     const double Vi[3], const double Vj[3], const double Wi[3],
                     const double Wj[3], double Fi[3], double Fj[3], double Ti[3],
                     double Tj[3]) {
  orc_lubrication_rate(p, p->shear_rate, r, ai, aj, Vi, Vj, Wi, Wj, Fi, Fj, Ti, Tj);
}

/* Lubrication taper factor of a listed pair at gap d (1 for w = 0). */
static double lub_taper_factor(const orc_params *p, double d, double ai, double aj) {
  if (!(p->lub_taper > 0.0)) return 1.0;
  double dl = lub_delta(p, ai, aj);
  double t = (dl - d) / (p->lub_taper * dl);
  if (t >= 1.0) return 1.0;
  if (t <= 0.0) return 0.0;
  return t * t * (3.0 - 2.0 * t);
}

/* Electro-chemical force on i from j at surface distance d, along the unit
 * vector n from i to j (Eq. 6-7): the double-layer repulsion
 * -F_ER (abar/a0) exp(-d/lambda_D) n (its contact value for d < 0), acting
 * below d = 20 lambda_D, plus the van der Waals attraction
 * A abar / (12 (d^2 + eps^2)) n (its contact value for d < 0), acting below
 * d = 4 a0, with abar = 2 a_i a_j / (a_i + a_j) and eps = vdw_eps abar.  The
 * force on j is the opposite. */
void orc_echem(const orc_params *p, double d, double ai, double aj, const double n[3], double F[3]) {
  double abar = 2.0 * ai * aj / (ai + aj);
  double m = 0.0;
  if (p->f_er > 0.0 && d < 20.0 * p->lambda_d) {
    double e = d >= 0.0 ? exp(-d / p->lambda_d) : 1.0;
    m -= p->f_er * (abar / p->a0) * e;
  }
  if (p->hamaker > 0.0 && d < 4.0 * p->a0) {
    double eps = p->vdw_eps * abar;
    double dd = d >= 0.0 ? d : 0.0;
    m += p->hamaker * abar / (12.0 * (dd * dd + eps * eps));
  }
  for (int q = 0; q < 3; ++q) F[q] = m * n[q];
}

/* ------------------------------------------------------------------------ */
/* One pair, everything: contact (if overlapping) + lubrication + stresslet  */
/* ------------------------------------------------------------------------ */

/* Evaluates pair (i, j) from absolute state.  Returns bit 0 set when the
 * pair is listed (within the interaction range), bit 1 when in contact.
 * xi_old/xi_new (sliding stretch) are in the i -> j orientation; xr_old and
 * xr_new (rolling stretch, App. B) do not depend on it and may be NULL when
 * k_r = 0.  S is the pair stresslet S^C + S^L + S^E of Eq. 9 (row major).
 * Outputs are zero for unlisted pairs.
 * In the wavy flow of Eq. 17, V = u - U_inf and W = w - Omega_inf are taken
 * at each centre and the strain acting on the pair is that of the mean of
 * the two centres' local shear rates. */
static int pair_eval_core(const orc_params *p, double off, const double xi[3], const double xj[3],
                          const double ui[3], const double uj[3], const double wi[3],
                          const double wj[3], double ai, double aj, const double xi_old[3],
                          const double xr_old[3], double Fi[3], double Fj[3], double Ti[3],
                          double Tj[3], double S[9], double xi_new[3], double xr_new[3],
                          double mag[4]) {
  double r[3];
  int sy;
  memset(Fi, 0, 3 * sizeof(double)); memset(Fj, 0, 3 * sizeof(double));
  memset(Ti, 0, 3 * sizeof(double)); memset(Tj, 0, 3 * sizeof(double));
  memset(S, 0, 9 * sizeof(double)); memset(xi_new, 0, 3 * sizeof(double));
  if (xr_new) memset(xr_new, 0, 3 * sizeof(double));
  min_image(p, off, xi, xj, r, &sy);
  if (!is_pair(p, r, ai, aj)) return 0;
  int flags = 1;
  /* image of j: shifted by sy boxes along y, moving with sy*gdot*L_y along x */
  double ujm[3] = {uj[0] + sy * p->shear_rate * p->L[1], uj[1], uj[2]};
  double yjm = xj[1] + sy * p->L[1];
  double dist = sqrt(dot3(r, r));
  double d = dist - (ai + aj);
  double Fc[3] = {0, 0, 0}, Tci[3] = {0, 0, 0}, Tcj[3] = {0, 0, 0};
  double Tri[3] = {0, 0, 0}, Trj[3] = {0, 0, 0};
  if (d < 0.0) {
    flags |= 2;
    orc_contact(p, r, ai, aj, ui, ujm, wi, wj, xi_old, Fc, Tci, Tcj, xi_new);
    if (p->k_r > 0.0) {
      double zero[3] = {0, 0, 0}, xr_tmp[3];
      orc_rolling(p, r, ai, aj, ui, ujm, wi, wj, xr_old ? xr_old : zero, Tri, Trj,
                  xr_new ? xr_new : xr_tmp);
    }
  }
  /* velocities relative to the ambient flow at each centre */
  double rate_i = orc_flow_rate(p, xi[1]), rate_j = orc_flow_rate(p, yjm);
  double Vi[3] = {ui[0] - orc_flow_ux(p, xi[1]), ui[1], ui[2]};
  double Vj[3] = {ujm[0] - orc_flow_ux(p, yjm), ujm[1], ujm[2]};
  double Wi[3] = {wi[0], wi[1], wi[2] + 0.5 * rate_i};
  double Wj[3] = {wj[0], wj[1], wj[2] + 0.5 * rate_j};
  double Fli[3] = {0, 0, 0}, Flj[3] = {0, 0, 0}, Tli[3] = {0, 0, 0}, Tlj[3] = {0, 0, 0};
  double lm[4] = {0, 0, 0, 0};
  if (in_lub_range(p, r, ai, aj)) {
    lubrication_core(p, 0.5 * (rate_i + rate_j), r, ai, aj, Vi, Vj, Wi, Wj, Fli, Flj, Tli, Tlj,
                     mag ? lm : NULL);
    double tap = lub_taper_factor(p, d, ai, aj);
    for (int q = 0; q < 3; ++q) {
      Fli[q] *= tap; Flj[q] *= tap; Tli[q] *= tap; Tlj[q] *= tap;
    }
    for (int q = 0; q < 4; ++q) lm[q] *= tap;
  }
  /* electro-chemical force (Eq. 6-7), central */
  double Fe[3] = {0, 0, 0};
  if (orc_echem_range(p) > 0.0) {
    double n[3] = {r[0] / dist, r[1] / dist, r[2] / dist};
    orc_echem(p, d, ai, aj, n, Fe);
  }
  for (int q = 0; q < 3; ++q) {
    Fi[q] = Fc[q] + Fli[q] + Fe[q];
    Fj[q] = -Fc[q] + Flj[q] - Fe[q];
    Ti[q] = Tci[q] + Tli[q] + Tri[q];
    Tj[q] = Tcj[q] + Tlj[q] + Trj[q];
  }
  /* Eq. 9: S^C = r (x) F^C_ij, S^L = sym(r (x) F^L_ij), S^E = r (x) F^E_ij,
   * r = x_j - x_i (the rolling pseudo-force exerts no force: no stresslet) */
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      S[3 * a + b] = r[a] * Fc[b] + 0.5 * (r[a] * Fli[b] + r[b] * Fli[a]) + r[a] * Fe[b];
  if (mag) {
    /* each physical term on its own: contact, lubrication sub-terms,
     * electro-chemical, rolling */
    double c = sqrt(dot3(Fc, Fc)), e = sqrt(dot3(Fe, Fe));
    mag[0] = c + lm[0] + e;
    mag[1] = c + lm[1] + e;
    mag[2] = sqrt(dot3(Tci, Tci)) + lm[2] + sqrt(dot3(Tri, Tri));
    mag[3] = sqrt(dot3(Tcj, Tcj)) + lm[3] + sqrt(dot3(Trj, Trj));
  }
  return flags;
}

int orc_pair_eval_full(const orc_params *p, double off, const double xi[3], const double xj[3],
                       const double ui[3], const double uj[3], const double wi[3],
                       const double wj[3], double ai, double aj, const double xi_old[3],
                       const double xr_old[3], double Fi[3], double Fj[3], double Ti[3],
                       double Tj[3], double S[9], double xi_new[3], double xr_new[3]) {
  return pair_eval_core(p, off, xi, xj, ui, uj, wi, wj, ai, aj, xi_old, xr_old, Fi, Fj, Ti, Tj, S,
                        xi_new, xr_new, NULL);
}

/* The pair without rolling history (a new rolling spring when k_r > 0). */
int orc_pair_eval(const orc_params *p, double off, const double xi[3], const double xj[3],
                  const double ui[3], const double uj[3], const double wi[3],
                  const double wj[3], double ai, double aj, const double xi_old[3],
                  double Fi[3], double Fj[3], double Ti[3], double Tj[3], double S[9],
                  double xi_new[3]) {
  return orc_pair_eval_full(p, off, xi, xj, ui, uj, wi, wj, ai, aj, xi_old, NULL, Fi, Fj, Ti,
                            Tj, S, xi_new, NULL);
}

/* ------------------------------------------------------------------------ */
/* System: state, history, force evaluation, time step                       */
/* ------------------------------------------------------------------------ */

orc_sys *orc_create(int64_t n, const orc_params *p) {
  orc_sys *s = (orc_sys *)calloc(1, sizeof(orc_sys));
  s->p = *p;
  s->n = n;
  size_t v3 = sizeof(double) * 3 * (size_t)(n > 0 ? n : 1);
  s->x = (double *)calloc(1, v3); s->u = (double *)calloc(1, v3);
  s->w = (double *)calloc(1, v3); s->al = (double *)calloc(1, v3);
  s->aw = (double *)calloc(1, v3); s->F = (double *)calloc(1, v3);
  s->T = (double *)calloc(1, v3);
  s->Fa = (double *)calloc(1, v3 / 3);
  s->Ta = (double *)calloc(1, v3 / 3);
  s->a = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  s->id = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
  s->hcap = 16;
  s->hkey = (int64_t *)malloc(sizeof(int64_t) * (size_t)s->hcap);
  s->hxi = (double *)malloc(sizeof(double) * 3 * (size_t)s->hcap);
  s->hxr = (double *)calloc(3 * (size_t)s->hcap, sizeof(double));
  s->iy = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  return s;
}

void orc_destroy(orc_sys *s) {
  if (!s) return;
  free(s->x); free(s->u); free(s->w); free(s->al); free(s->aw);
  free(s->F); free(s->T); free(s->Fa); free(s->Ta); free(s->a); free(s->id); free(s->hkey); free(s->hxi); free(s->hxr); free(s->iy);
  free(s);
}

/* Copies state in.  Any of u, w, al, aw may be NULL: u defaults to
 * U_inf(x), w to Omega_inf(x), al/aw to zero. */
void orc_set_state(orc_sys *s, const double *x, const double *a, const int32_t *id,
                   const double *u, const double *w, const double *al,
                   const double *aw, int64_t nstep) {
  int64_t n = s->n;
  memcpy(s->x, x, sizeof(double) * 3 * (size_t)n);
  memcpy(s->a, a, sizeof(double) * (size_t)n);
  memcpy(s->id, id, sizeof(int32_t) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    for (int c = 0; c < 3; ++c) {
      s->u[c * n + i] = u ? u[c * n + i] : (c == 0 ? orc_flow_ux(&s->p, x[n + i]) : 0.0);
      s->w[c * n + i] = w ? w[c * n + i] : (c == 2 ? -0.5 * orc_flow_rate(&s->p, x[n + i]) : 0.0);
      s->al[c * n + i] = al ? al[c * n + i] : 0.0;
      s->aw[c * n + i] = aw ? aw[c * n + i] : 0.0;
    }
  }
  s->nstep = nstep;
  s->hk = 0;
  memset(s->iy, 0, sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
}

static void hist_reserve(orc_sys *s, int64_t k) {
  if (k > s->hcap) {
    s->hcap = k;
    s->hkey = (int64_t *)realloc(s->hkey, sizeof(int64_t) * (size_t)k);
    s->hxi = (double *)realloc(s->hxi, sizeof(double) * 3 * (size_t)k);
    s->hxr = (double *)realloc(s->hxr, sizeof(double) * 3 * (size_t)k);
  }
}

/* Contact history as (key, xi, xr) arrays sorted by key = lo_id << 32 |
 * hi_id: the sliding stretch (lo -> hi orientation) and the rolling stretch
 * of each contact; xr may be NULL (zero rolling stretch). */
void orc_set_history_r(orc_sys *s, int64_t k, const int64_t *key, const double *xi,
                       const double *xr) {
  hist_reserve(s, k);
  memcpy(s->hkey, key, sizeof(int64_t) * (size_t)k);
  memcpy(s->hxi, xi, sizeof(double) * 3 * (size_t)k);
  if (xr) memcpy(s->hxr, xr, sizeof(double) * 3 * (size_t)k);
  else memset(s->hxr, 0, sizeof(double) * 3 * (size_t)k);
  s->hk = k;
}

void orc_set_history(orc_sys *s, int64_t k, const int64_t *key, const double *xi) {
  orc_set_history_r(s, k, key, xi, NULL);
}

int64_t orc_get_history_r(const orc_sys *s, int64_t cap, int64_t *key, double *xi, double *xr) {
  int64_t m = s->hk < cap ? s->hk : cap;
  if (m > 0) {
    memcpy(key, s->hkey, sizeof(int64_t) * (size_t)m);
    memcpy(xi, s->hxi, sizeof(double) * 3 * (size_t)m);
    if (xr) memcpy(xr, s->hxr, sizeof(double) * 3 * (size_t)m);
  }
  return s->hk;
}

int64_t orc_get_history(const orc_sys *s, int64_t cap, int64_t *key, double *xi) {
  return orc_get_history_r(s, cap, key, xi, NULL);
}

static int64_t hist_find(const orc_sys *s, int64_t key) {
  int64_t lo = 0, hi = s->hk - 1;
  while (lo <= hi) {
    int64_t mid = (lo + hi) / 2;
    if (s->hkey[mid] == key) return mid;
    if (s->hkey[mid] < key) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

typedef struct hrec { int64_t key; double xi[3], xr[3]; } hrec;
static int cmp_hrec(const void *A, const void *B) {
  const hrec *a = (const hrec *)A, *b = (const hrec *)B;
  return a->key < b->key ? -1 : (a->key > b->key ? 1 : 0);
}

/* Stokes drag of Eq. A1 on particle k with the Faxen term:
 * F = -6 pi eta0 a (u - (1 + a^2/6 Laplacian) U_inf), T = -8 pi eta0 a^3
 * (w - Omega_inf), both at the centre (the Laplacian vanishes in the simple
 * shear). */
static void stokes_drag(const orc_sys *s, int64_t k, double f[3], double t[3]) {
  const orc_params *p = &s->p;
  int64_t n = s->n;
  double a = s->a[k], y = s->x[n + k];
  double V[3] = {s->u[k] - orc_faxen_ux(p, y, a), s->u[n + k], s->u[2 * n + k]};
  double W[3] = {s->w[k], s->w[n + k], s->w[2 * n + k] + 0.5 * orc_flow_rate(p, y)};
  for (int c = 0; c < 3; ++c) {
    f[c] = -6.0 * M_PI * p->eta0 * a * V[c];
    t[c] = -8.0 * M_PI * p->eta0 * a * a * a * W[c];
  }
}

/* ------------------------------------------------------------------------ */
/* Pair sets of the current state: (i, j) array indices with i < j, sorted   */
/* by (i, j).  The brute force is the definition; the cell list (Sec. II A:  */
/* a counting sort into cells of edge >= the largest pair range, then the    */
/* symmetric half stencil) finds the same set, and since the set is then     */
/* sorted the same way, the evaluation below is the same arithmetic in the   */
/* same order either way.                                                    */
/* ------------------------------------------------------------------------ */

/* Brute force: every i < j, in that order. */
static int64_t pairs_brute(const orc_sys *s, double off, int64_t **out) {
  const orc_params *p = &s->p;
  int64_t n = s->n;
  int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  /* two passes over the rows (count, then fill), each row on its own */
  for (int pass = 0; pass < 2; ++pass) {
    int64_t *pr = pass ? *out : NULL;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
      double xi[3] = {s->x[i], s->x[n + i], s->x[2 * n + i]};
      int64_t k = pass ? cnt[i] : 0;
      for (int64_t j = i + 1; j < n; ++j) {
        double xj[3] = {s->x[j], s->x[n + j], s->x[2 * n + j]};
        double r[3];
        int sy;
        min_image(p, off, xi, xj, r, &sy);
        if (!is_pair(p, r, s->a[i], s->a[j])) continue;
        if (pass) {
          pr[2 * k] = i;
          pr[2 * k + 1] = j;
        }
        ++k;
      }
      if (!pass) cnt[i + 1] = k;
    }
    if (!pass) {
      for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
      *out = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)(cnt[n] > 0 ? cnt[n] : 1));
    }
  }
  int64_t P = cnt[n];
  free(cnt);
  return P;
}

/* Cell list with the half stencil.  Cells: nc = floor(L / (range (1 + 1e-9)))
 * per axis, range = 2 a_max + the largest delta_ij, so that a pair's cells
 * differ by at most one along each axis.  Particle i of cell (cx, cy, cz)
 * looks at the particles after it in its own cell, the cell x+1, the three
 * cells x-1..x+1 of the row z+1, and the layer y+1: its nine cells, or, when
 * y+1 wraps through y = L_y, the four x cells cx - s - 2 .. cx - s + 1
 * (s = floor(off / cs_x)) of rows z-1..z+1, which hold every particle whose
 * Lees-Edwards image (x + off) can lie within range.  Each unordered pair of
 * cells is visited from one side only, so each pair is found once.  Needs at
 * least 4 cells along x and 3 along y and z; returns -1 otherwise. */
static int64_t pairs_cell(const orc_sys *s, double off, int64_t **out) {
  const orc_params *p = &s->p;
  int64_t n = s->n;
  double amax = 0.0;
  for (int64_t i = 0; i < n; ++i) amax = s->a[i] > amax ? s->a[i] : amax;
  double range = 2.0 * amax + pair_delta(p, amax, amax);
  int nc[3];
  double cs[3];
  for (int d = 0; d < 3; ++d) {
    nc[d] = (int)floor(p->L[d] / (range * (1.0 + 1e-9)));
    if (nc[d] < (d == 0 ? 4 : 3)) return -1;
    cs[d] = p->L[d] / nc[d];
  }
  int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
  int32_t *cell = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int64_t *cstart = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
  int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  /* counting sort (stable: increasing index within a cell) */
  for (int64_t i = 0; i < n; ++i) {
    int c[3];
    for (int d = 0; d < 3; ++d) {
      c[d] = (int)floor(s->x[d * n + i] / cs[d]);
      if (c[d] < 0) c[d] = 0;
      if (c[d] >= nc[d]) c[d] = nc[d] - 1;
    }
    cell[i] = (int32_t)((c[2] * nc[1] + c[1]) * nc[0] + c[0]);
    cstart[cell[i] + 1] += 1;
  }
  for (int64_t c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
  {
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
    memcpy(fill, cstart, sizeof(int64_t) * (size_t)ncell);
    for (int64_t i = 0; i < n; ++i) order[fill[cell[i]]++] = i;
    free(fill);
  }
  int fsh = (int)floor(off / cs[0]);
  /* pairs grouped by their lower index: count, offsets, fill, sort each group */
  int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  int64_t *pos = NULL;
  for (int pass = 0; pass < 2; ++pass) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
      int ci = cell[i];
      int cx = ci % nc[0], cy = (ci / nc[0]) % nc[1], cz = ci / (nc[0] * nc[1]);
      double xi[3] = {s->x[i], s->x[n + i], s->x[2 * n + i]};
      /* the stencil: up to 1 + 1 + 3 + 12 cells */
      int64_t cells[17];
      int nq = 0;
      cells[nq++] = ci;
      cells[nq++] = (cz * nc[1] + cy) * nc[0] + (cx + 1) % nc[0];
      for (int ox = -1; ox <= 1; ++ox)
        cells[nq++] = (((cz + 1) % nc[2]) * nc[1] + cy) * nc[0] + (cx + ox + nc[0]) % nc[0];
      int wrap = cy + 1 == nc[1];
      int qy = wrap ? 0 : cy + 1;
      int x0 = wrap ? -2 - fsh : -1, x1 = wrap ? 1 - fsh : 1;
      for (int oz = -1; oz <= 1; ++oz)
        for (int ox = x0; ox <= x1; ++ox) {
          int qx = ((cx + ox) % nc[0] + nc[0]) % nc[0];
          cells[nq++] = (((cz + oz + nc[2]) % nc[2]) * nc[1] + qy) * nc[0] + qx;
        }
      for (int q = 0; q < nq; ++q) {
        int64_t b = cstart[cells[q]], e = cstart[cells[q] + 1];
        for (int64_t t = b; t < e; ++t) {
          int64_t j = order[t];
          if (q == 0 && j <= i) continue;   /* own cell: partners after i */
          double xj[3] = {s->x[j], s->x[n + j], s->x[2 * n + j]};
          double r[3];
          int sy;
          min_image(p, off, xi, xj, r, &sy);
          if (!is_pair(p, r, s->a[i], s->a[j])) continue;
          int64_t lo = i < j ? i : j, hi = i < j ? j : i;
          if (!pass) {
#pragma omp atomic
            cnt[lo + 1] += 1;
          } else {
            int64_t k;
#pragma omp atomic capture
            k = pos[lo]++;
            (*out)[2 * k] = lo;
            (*out)[2 * k + 1] = hi;
          }
        }
      }
    }
    if (!pass) {
      for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
      *out = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)(cnt[n] > 0 ? cnt[n] : 1));
      pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
      memcpy(pos, cnt, sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    }
  }
  /* each group in increasing partner index (insertion sort: groups are short) */
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < n; ++i) {
    int64_t *g = *out + 2 * cnt[i];
    int64_t m = cnt[i + 1] - cnt[i];
    for (int64_t k = 1; k < m; ++k) {
      int64_t v = g[2 * k + 1], t = k;
      while (t > 0 && g[2 * (t - 1) + 1] > v) {
        g[2 * t + 1] = g[2 * (t - 1) + 1];
        --t;
      }
      g[2 * t + 1] = v;
    }
  }
  int64_t P = cnt[n];
  free(cell); free(cstart); free(order); free(cnt); free(pos);
  return P;
}

/* Pair set of the current state by the system's neighbour mode (0: brute
 * force, 1: cell list; the brute force also when the box holds too few
 * cells). */
static int64_t pairs_of(const orc_sys *s, double off, int64_t **out) {
  if (s->cells) {
    int64_t P = pairs_cell(s, off, out);
    if (P >= 0) return P;
  }
  return pairs_brute(s, off, out);
}

/* Neighbour search mode of a system: 0 brute force (the default), 1 cell
 * list.  Both give the same pair set in the same order. */
void orc_set_cells(orc_sys *s, int cells) { s->cells = cells ? 1 : 0; }

/* The pair set of the current state found by the cell list, as (lo id, hi
 * id) sorted lexicographically (compare orc_pairs_bruteforce).  Returns the
 * number of pairs (at most cap written), -1 when the box holds too few
 * cells. */
int64_t orc_pairs_cell(orc_sys *s, int64_t *out, int64_t cap) {
  int64_t *pr = NULL;
  int64_t P = pairs_cell(s, orc_le_offset(&s->p, s->nstep), &pr);
  if (P < 0) return -1;
  for (int64_t k = 0; k < P; ++k) {
    int64_t a = s->id[pr[2 * k]], b = s->id[pr[2 * k + 1]];
    pr[2 * k] = a < b ? a : b;
    pr[2 * k + 1] = a < b ? b : a;
  }
  qsort(pr, (size_t)P, sizeof(int64_t) * 2, cmp_i64pair);
  int64_t m = P < cap ? P : cap;
  if (out && m > 0) memcpy(out, pr, sizeof(int64_t) * 2 * (size_t)m);
  free(pr);
  return P;
}

/* One pair's results, kept until they are summed in pair order. */
typedef struct pres {
  double Fi[3], Fj[3], Ti[3], Tj[3], S[9], xn[3], rn[3], mag[4];
  int fl;
} pres;

/* Force evaluation at the current state (x, u, w) and time nstep*dt:
 * all pair interactions (from the pair set, in its order), Stokes drag
 * (Eq. A1), per-particle totals F and T, the bulk stress of Eq. 8, and, when
 * commit != 0, the new contact history.  The pairs are evaluated in parallel
 * (each on its own) and summed one after another in the set's order, so the
 * result does not depend on the number of threads. */
void orc_forces(orc_sys *s, int commit) {
  const orc_params *p = &s->p;
  int64_t n = s->n;
  double off = orc_le_offset(p, s->nstep);
  double E[9], Om[3];
  ambient(p, E, Om);
  memset(s->F, 0, sizeof(double) * 3 * (size_t)n);
  memset(s->T, 0, sizeof(double) * 3 * (size_t)n);
  memset(s->Fa, 0, sizeof(double) * (size_t)n);
  memset(s->Ta, 0, sizeof(double) * (size_t)n);
  int64_t *pr = NULL;
  int64_t P = pairs_of(s, off, &pr);
  pres *res = (pres *)malloc(sizeof(pres) * (size_t)(P > 0 ? P : 1));
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t k = 0; k < P; ++k) {
    int64_t i = pr[2 * k], j = pr[2 * k + 1];
    double xi[3] = {s->x[i], s->x[n + i], s->x[2 * n + i]};
    double ui[3] = {s->u[i], s->u[n + i], s->u[2 * n + i]};
    double wi[3] = {s->w[i], s->w[n + i], s->w[2 * n + i]};
    double xj[3] = {s->x[j], s->x[n + j], s->x[2 * n + j]};
    double uj[3] = {s->u[j], s->u[n + j], s->u[2 * n + j]};
    double wj[3] = {s->w[j], s->w[n + j], s->w[2 * n + j]};
    int64_t lo = s->id[i] < s->id[j] ? s->id[i] : s->id[j];
    int64_t hi = s->id[i] < s->id[j] ? s->id[j] : s->id[i];
    double sgn = s->id[i] < s->id[j] ? 1.0 : -1.0;   /* i->j vs lo->hi */
    double xo[3] = {0, 0, 0}, ro[3] = {0, 0, 0};
    int64_t h = hist_find(s, (lo << 32) | hi);
    if (h >= 0)
      for (int c = 0; c < 3; ++c) {
        xo[c] = sgn * s->hxi[3 * h + c];
        ro[c] = s->hxr[3 * h + c];
      }
    pres *q = &res[k];
    q->fl = pair_eval_core(p, off, xi, xj, ui, uj, wi, wj, s->a[i], s->a[j], xo, ro, q->Fi, q->Fj,
                           q->Ti, q->Tj, q->S, q->xn, q->rn, q->mag);
  }
  double Spair[9] = {0};
  int64_t hn = 0, hc = 64;
  hrec *hnew = (hrec *)malloc(sizeof(hrec) * (size_t)hc);
  int64_t ncont = 0;
  for (int64_t k = 0; k < P; ++k) {
    int64_t i = pr[2 * k], j = pr[2 * k + 1];
    const pres *q = &res[k];
    for (int c = 0; c < 3; ++c) {
      s->F[c * n + i] += q->Fi[c]; s->F[c * n + j] += q->Fj[c];
      s->T[c * n + i] += q->Ti[c]; s->T[c * n + j] += q->Tj[c];
    }
    s->Fa[i] += q->mag[0]; s->Fa[j] += q->mag[1];
    s->Ta[i] += q->mag[2]; s->Ta[j] += q->mag[3];
    for (int c = 0; c < 9; ++c) Spair[c] += q->S[c];
    if (q->fl & 2) {
      ++ncont;
      if (hn == hc) { hc *= 2; hnew = (hrec *)realloc(hnew, sizeof(hrec) * (size_t)hc); }
      int64_t lo = s->id[i] < s->id[j] ? s->id[i] : s->id[j];
      int64_t hi = s->id[i] < s->id[j] ? s->id[j] : s->id[i];
      double sgn = s->id[i] < s->id[j] ? 1.0 : -1.0;
      hnew[hn].key = (lo << 32) | hi;
      for (int c = 0; c < 3; ++c) {
        hnew[hn].xi[c] = sgn * q->xn[c];
        hnew[hn].xr[c] = q->rn[c];
      }
      ++hn;
    }
  }
  free(res);
  free(pr);
  /* Stokes drag, Eq. A1, and the single-particle stresslets
   * S^S_i = 20/3 pi eta0 a_i^3 E_inf(x_i) (E_inf at the centre, no Laplacian) */
  double Sein[9] = {0};
  for (int64_t i = 0; i < n; ++i) {
    double f[3], t[3];
    stokes_drag(s, i, f, t);
    for (int c = 0; c < 3; ++c) {
      s->F[c * n + i] += f[c];
      s->T[c * n + i] += t[c];
    }
    s->Fa[i] += sqrt(dot3(f, f));
    s->Ta[i] += sqrt(dot3(t, t));
    double a = s->a[i], Ei[9], Oi[3];
    ambient_rate(orc_flow_rate(p, s->x[n + i]), Ei, Oi);
    for (int q = 0; q < 9; ++q) Sein[q] += 20.0 / 3.0 * M_PI * p->eta0 * a * a * a * Ei[q];
  }
  /* Eq. 8; the fluid's own term with the box mean of E_inf (the wave of
   * Eq. 17 averages to zero over L_y) */
  double V = p->L[0] * p->L[1] * p->L[2];
  for (int q = 0; q < 9; ++q) s->sigma[q] = 2.0 * p->eta0 * E[q] + (Sein[q] + Spair[q]) / V;
  s->npairs_last = P;
  s->ncontacts_last = ncont;
  if (commit) {
    qsort(hnew, (size_t)hn, sizeof(hrec), cmp_hrec);
    hist_reserve(s, hn);
    for (int64_t h = 0; h < hn; ++h) {
      s->hkey[h] = hnew[h].key;
      for (int c = 0; c < 3; ++c) {
        s->hxi[3 * h + c] = hnew[h].xi[c];
        s->hxr[3 * h + c] = hnew[h].xr[c];
      }
    }
    s->hk = hn;
  }
  free(hnew);
}

/* Force and torque on the m particles listed in idx (array indices), brute
 * force over all others plus Stokes drag, at the current state, time and
 * history: the rows of orc_forces for those particles.  Used to time the
 * oracle on systems where the full O(N^2) evaluation takes minutes. */
void orc_forces_sampled(orc_sys *s, const int64_t *idx, int64_t m, double *F, double *T,
                        double *Fa, double *Ta) {
  const orc_params *p = &s->p;
  int64_t n = s->n;
  double off = orc_le_offset(p, s->nstep);
  for (int64_t q = 0; q < m; ++q) {
    int64_t k = idx[q];
    double f[3] = {0, 0, 0}, t[3] = {0, 0, 0}, fa = 0.0, ta = 0.0;
    for (int64_t o = 0; o < n; ++o) {
      if (o == k) continue;
      int64_t i = k < o ? k : o, j = k < o ? o : k;   /* same orientation as orc_forces */
      double xi[3] = {s->x[i], s->x[n + i], s->x[2 * n + i]};
      double xj[3] = {s->x[j], s->x[n + j], s->x[2 * n + j]};
      double r[3];
      int sy;
      min_image(p, off, xi, xj, r, &sy);
      if (!is_pair(p, r, s->a[i], s->a[j])) continue;
      double ui[3] = {s->u[i], s->u[n + i], s->u[2 * n + i]};
      double uj[3] = {s->u[j], s->u[n + j], s->u[2 * n + j]};
      double wi[3] = {s->w[i], s->w[n + i], s->w[2 * n + i]};
      double wj[3] = {s->w[j], s->w[n + j], s->w[2 * n + j]};
      int64_t lo = s->id[i] < s->id[j] ? s->id[i] : s->id[j];
      int64_t hi = s->id[i] < s->id[j] ? s->id[j] : s->id[i];
      double sgn = s->id[i] < s->id[j] ? 1.0 : -1.0;
      double xo[3] = {0, 0, 0}, ro[3] = {0, 0, 0};
      int64_t h = hist_find(s, (lo << 32) | hi);
      if (h >= 0)
        for (int c = 0; c < 3; ++c) {
          xo[c] = sgn * s->hxi[3 * h + c];
          ro[c] = s->hxr[3 * h + c];
        }
      double Fi[3], Fj[3], Ti[3], Tj[3], S[9], xn[3], rn[3];
      double mag[4];
      pair_eval_core(p, off, xi, xj, ui, uj, wi, wj, s->a[i], s->a[j], xo, ro, Fi, Fj, Ti, Tj, S,
                     xn, rn, mag);
      for (int c = 0; c < 3; ++c) {
        f[c] += (k == i) ? Fi[c] : Fj[c];
        t[c] += (k == i) ? Ti[c] : Tj[c];
      }
      fa += (k == i) ? mag[0] : mag[1];
      ta += (k == i) ? mag[2] : mag[3];
    }
    double fd[3], td[3];
    stokes_drag(s, k, fd, td);
    for (int c = 0; c < 3; ++c) {
      f[c] += fd[c];
      t[c] += td[c];
      F[c * m + q] = f[c];
      T[c * m + q] = t[c];
    }
    if (Fa) Fa[q] = fa + sqrt(dot3(fd, fd));
    if (Ta) Ta[q] = ta + sqrt(dot3(td, td));
  }
}

/* Accelerations from the last force evaluation: alpha = F/m, T/I with
 * m = 4/3 pi rho a^3 and I = 2/5 m a^2 (spheres, Eq. 1). */
static void accelerations(orc_sys *s) {
  int64_t n = s->n;
  for (int64_t i = 0; i < n; ++i) {
    double a = s->a[i];
    double m = 4.0 / 3.0 * M_PI * s->p.rho * a * a * a;
    double I = 0.4 * m * a * a;
    for (int c = 0; c < 3; ++c) {
      s->al[c * n + i] = s->F[c * n + i] / m;
      s->aw[c * n + i] = s->T[c * n + i] / I;
    }
  }
}

/* Initial accelerations from one force evaluation at the initial state,
 * with an empty contact history that stays empty afterwards. */
void orc_init_accel(orc_sys *s) {
  s->hk = 0;
  orc_forces(s, 0);
  accelerations(s);
}

/* Lees-Edwards wrap of one particle (Eq. 16).  Returns the y-crossing:
 * -1 when it left through y >= L_y, +1 through y < 0, 0 otherwise. */
static int le_wrap(const orc_params *p, double off, double *x, double *y, double *z) {
  int cross = 0;
  double Ly = p->L[1];
  if (*y >= Ly) {
    *y = *y - Ly;
    *x = *x - off;
    cross = -1;
  } else if (*y < 0.0) {
    *y = *y + Ly;
    *x = *x + off;
    cross = 1;
    if (*y >= Ly) *y = 0.0;   /* y + L_y rounded up to L_y */
  }
  *x = fmod(*x, p->L[0]);
  if (*x < 0.0) *x = *x + p->L[0];
  if (*x >= p->L[0]) *x = *x - p->L[0];
  if (*z >= p->L[2]) *z = *z - p->L[2];
  else if (*z < 0.0) {
    *z = *z + p->L[2];
    if (*z >= p->L[2]) *z = 0.0;
  }
  return cross;
}

/* Modified velocity-Verlet step(s), Eq. 15, in the Lees-Edwards box, Eq. 16. */
void orc_step(orc_sys *s, int64_t nsteps) {
  const orc_params *p = &s->p;
  int64_t n = s->n;
  double dt = p->dt;
  for (int64_t k = 0; k < nsteps; ++k) {
    s->nstep += 1;
    double off = orc_le_offset(p, s->nstep);
    for (int64_t i = 0; i < n; ++i) {
      double *X = &s->x[i], *Y = &s->x[n + i], *Z = &s->x[2 * n + i];
      /* Eq. 15a, 15b */
      *X = *X + dt * s->u[i] + 0.5 * dt * dt * s->al[i];
      *Y = *Y + dt * s->u[n + i] + 0.5 * dt * dt * s->al[n + i];
      *Z = *Z + dt * s->u[2 * n + i] + 0.5 * dt * dt * s->al[2 * n + i];
      for (int c = 0; c < 3; ++c) {
        s->u[c * n + i] = s->u[c * n + i] + 0.5 * dt * s->al[c * n + i];
        s->w[c * n + i] = s->w[c * n + i] + 0.5 * dt * s->aw[c * n + i];
      }
      int cr = le_wrap(p, off, X, Y, Z);
      s->u[i] = s->u[i] + cr * p->shear_rate * p->L[1];
      s->iy[i] -= cr;   /* left through the top: one image up */
    }
    /* Eq. 15c at (x^{n+1}, u^{n+1/2}) */
    orc_forces(s, 1);
    accelerations(s);
    /* Eq. 15d */
    for (int64_t i = 0; i < n; ++i)
      for (int c = 0; c < 3; ++c) {
        s->u[c * n + i] = s->u[c * n + i] + 0.5 * dt * s->al[c * n + i];
        s->w[c * n + i] = s->w[c * n + i] + 0.5 * dt * s->aw[c * n + i];
      }
  }
}

/* Accessors for the ctypes wrapper. */
void orc_get_images(const orc_sys *s, int64_t *iy) {
  memcpy(iy, s->iy, sizeof(int64_t) * (size_t)s->n);
}

void orc_get_state(const orc_sys *s, double *x, double *u, double *w, double *al, double *aw) {
  size_t b = sizeof(double) * 3 * (size_t)s->n;
  if (x) memcpy(x, s->x, b);
  if (u) memcpy(u, s->u, b);
  if (w) memcpy(w, s->w, b);
  if (al) memcpy(al, s->al, b);
  if (aw) memcpy(aw, s->aw, b);
}
/* Per particle, the sum of the magnitudes of the terms of its force and its
 * torque in the last evaluation (per pair: contact, each lubrication
 * sub-term of Eq. A2-A3, electro-chemical, rolling; and the drag): the
 * rounding error of an evaluation that forms these terms in a given
 * precision and sums them is bounded in proportion to it, so parity checks
 * scale by it where the terms cancel. */
void orc_get_force_scale(const orc_sys *s, double *Fa, double *Ta) {
  memcpy(Fa, s->Fa, sizeof(double) * (size_t)s->n);
  memcpy(Ta, s->Ta, sizeof(double) * (size_t)s->n);
}

void orc_get_forces(const orc_sys *s, double *F, double *T, double sigma[9]) {
  size_t b = sizeof(double) * 3 * (size_t)s->n;
  if (F) memcpy(F, s->F, b);
  if (T) memcpy(T, s->T, b);
  if (sigma) memcpy(sigma, s->sigma, 9 * sizeof(double));
}
int64_t orc_get_nstep(const orc_sys *s) { return s->nstep; }
int64_t orc_get_npairs(const orc_sys *s) { return s->npairs_last; }
int64_t orc_get_ncontacts(const orc_sys *s) { return s->ncontacts_last; }
