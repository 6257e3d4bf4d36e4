/*
 * gic_oracle.c -- plain, slow, single-threaded FP64 oracle for the per-substep
 * granule-grid coupling of the Granule-In-Cell method (Tang et al., "The
 * Granule-In-Cell Method for Simulating Sand-Water Mixtures", TOG 2025).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header or constant with the
 * CUDA library; it has its own parameter structs and reads the canonical
 * input encoding itself.
 *
 * Everything is FP64 and uses ABSOLUTE positions.  Granules are kept in their
 * original order; the cell sort is a separate function (or_sort) used only to
 * check the GPU's sort, because ordering does not change what the substep
 * computes.
 *
 * One substep follows Algorithm 2 (SandSubstep) of the paper, in its order:
 *   CalCoupling   -> or_g2p        (Sec. 3.3 Eqs. 5a-5c, Sec. 5.2)
 *   TransferCoupling -> or_p2g     (Sec. 5.2 "Exchange Momentum"; alpha_s of Sec. 5.1)
 *   CollisionHandling -> or_contact (Sec. 3.1 contact law, Eq. k_n)
 *   MoveParticle  -> or_integrate  (Sec. 5.2 Eq. "sand kine", symplectic Euler Sec. 4)
 * The contact force only feeds MoveParticle, and the exchange force needs the
 * granule's acceleration (virtual-mass term), so or_run evaluates contact and
 * coupling first, integrates, then transfers; the values are identical to the
 * paper's ordering because none of these steps reads another's output except
 * MoveParticle and the transfer.
 *
 * Readings taken where the paper is silent or ambiguous (listed in full in the
 * design notes of the repository):
 *  - drag prefactor: F_d = c_drag * pi r^2 rho_f |dv| dv (c_drag = 0.22 default,
 *    i.e. one half of the drag coefficient 0.44 of Sec. 6 "Parameters");
 *  - normal force: linear spring k_n * overlap plus a dashpot -c_n v_n with
 *    c_n = 2 zeta sqrt(k_n m_eff), not clamped at zero;
 *  - tangential force: f_t = -k_t v_t with k_t = kt_over_cn * c_n, capped at
 *    mu |F_n| (Sec. 3.1: tan(phi) = mu), memoryless;
 *  - polydisperse radii generalise 2r to r_i + r_j;
 *  - interpolation kernel N: trilinear tent on the MAC samples; a point beyond
 *    the first/last sample takes the end sample's value (G2P), and P2G puts
 *    the whole weight on that end sample (the transpose);
 *  - grad p on an x-face i is (p_i - p_{i-1}) / dx, boundary faces copy the
 *    adjacent interior face;
 *  - dv_f/dt = g - grad p / rho_f (the F_s / (rho alpha_f) term of Eq.
 *    momentum4 is unknown during the sand step and dropped);
 *  - exchange force per granule f = F_p + F_d + m_a (a_f - a_s), scattered at
 *    the substep's starting position, scaled by -dt'/dt;
 *  - walls: the six box planes, infinite mass, at rest, same contact law;
 *  - a granule that would leave the box is put back on the boundary it
 *    crossed (and flagged); its velocity is kept.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

/* status bits reported by the oracle */
#define OR_OUT_OF_DOMAIN 1u
#define OR_COINCIDENT 2u
#define OR_NONFINITE 4u

typedef struct {
  int nx, ny, nz; /* MAC cells per axis */
  int k;          /* contact cells per MAC cell and axis: h_c = dx / k */
  double dx;
  double ox, oy, oz; /* domain origin; the domain is [o, o + n dx] */
} or_grid;

typedef struct {
  double rho_s, rho_f, k_n, zeta, kt_over_cn, mu, c_drag;
  double gx, gy, gz;
  double dt;       /* sand substep dt' */
  double dt_fluid; /* fluid step dt (exchange scale dt'/dt) */
  int virtual_mass, walls;
  /* concentration-gradient / capillary pair force (Sec. 5.4); sigma = 0: off */
  double sigma;         /* surface tension coefficient */
  double bridge_frac;   /* liquid-bridge volume V* as a fraction of the granule volume */
  double moisture;      /* water ratio r_i held by every granule */
  double moisture_peak; /* where Gamma peaks (the maximum absorption ratio), in [1/4, 3/4] */
} or_params;

/* ------------------------------------------------------------------------ */
/* canonical input encoding                                                 */
/* ------------------------------------------------------------------------ */

/* x = origin + (cell + q / 2^30) * h_c */
void or_decode(const or_grid* G, int64_t n, const int32_t* cell, const uint32_t* q, double* x) {
  double hc = G->dx / G->k;
  double o[3] = {G->ox, G->oy, G->oz};
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a)
      x[3 * i + a] = o[a] + ((double)cell[3 * i + a] + (double)q[3 * i + a] / 1073741824.0) * hc;
}

/* ------------------------------------------------------------------------ */
/* Morton cell sort (the neighbour search the method needs, Sec. 3.1:       */
/* contacts only between granules closer than 2r)                           */
/* ------------------------------------------------------------------------ */

/* contact cell of each granule: floor((x - o) / h_c), clamped into the grid */
void or_cells(const or_grid* G, int64_t n, const double* x, int32_t* c) {
  double hc = G->dx / G->k;
  double o[3] = {G->ox, G->oy, G->oz};
  int nc[3] = {G->nx * G->k, G->ny * G->k, G->nz * G->k};
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) {
      double f = floor((x[3 * i + a] - o[a]) / hc);
      int ci = !(f >= 0.0) ? 0 : (f > nc[a] - 1 ? nc[a] - 1 : (int)f); /* NaN -> 0 */
      c[3 * i + a] = ci;
    }
}

/* Morton key: bit b of x goes to bit 3b, of y to 3b+1, of z to 3b+2 */
uint64_t or_morton(uint32_t ix, uint32_t iy, uint32_t iz) {
  uint64_t key = 0;
  for (int b = 0; b < 21; ++b) {
    key |= (uint64_t)((ix >> b) & 1u) << (3 * b);
    key |= (uint64_t)((iy >> b) & 1u) << (3 * b + 1);
    key |= (uint64_t)((iz >> b) & 1u) << (3 * b + 2);
  }
  return key;
}

typedef struct {
  uint64_t key;
  int64_t idx;
} or_keyidx;

static int cmp_keyidx(const void* a, const void* b) {
  const or_keyidx* x = (const or_keyidx*)a;
  const or_keyidx* y = (const or_keyidx*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
  return 0;
}

/* Stable sort of the granules by the Morton key of their contact cell.
 * perm[k] = index (in the input order) of the k-th granule after sorting;
 * ties keep input order.  keys[k] = key of that granule. */
void or_sort(int64_t n, const int32_t* c, int64_t* perm, uint64_t* keys) {
  or_keyidx* t = (or_keyidx*)malloc(sizeof(or_keyidx) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) {
    t[i].key = or_morton((uint32_t)c[3 * i], (uint32_t)c[3 * i + 1], (uint32_t)c[3 * i + 2]);
    t[i].idx = i;
  }
  qsort(t, (size_t)n, sizeof(or_keyidx), cmp_keyidx);
  for (int64_t i = 0; i < n; ++i) {
    perm[i] = t[i].idx;
    keys[i] = t[i].key;
  }
  free(t);
}

/* Run-length table of the sorted keys: one row (key, start, count) per
 * occupied cell, in key order.  Returns the number of occupied cells. */
int64_t or_cell_table(int64_t n, const uint64_t* keys, uint64_t* cell_key, int64_t* start, int64_t* count) {
  int64_t m = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (i == 0 || keys[i] != keys[i - 1]) {
      cell_key[m] = keys[i];
      start[m] = i;
      count[m] = 0;
      ++m;
    }
    count[m - 1] += 1;
  }
  return m;
}

/* ------------------------------------------------------------------------ */
/* DEM contact (Sec. 3.1, Eq. k_n, with the dashpot / tangential readings)  */
/* ------------------------------------------------------------------------ */

static double granule_volume(double r) { return 4.0 / 3.0 * OR_PI * r * r * r; }

/* Force on granule i from partner j.  xij = x_i - x_j, vij = v_i - v_j.
 * mj <= 0 marks a wall (infinite mass).  Returns 1 if in contact, 0 if not,
 * -1 for coincident centres (skipped). */
static int pair_force(const or_params* P, const double xij[3], const double vij[3], double ri, double rj,
                      double mi, double mj, double F[3]) {
  double d2 = xij[0] * xij[0] + xij[1] * xij[1] + xij[2] * xij[2];
  double R = ri + rj;
  if (!(d2 < R * R)) return 0;
  double d = sqrt(d2);
  if (d == 0.0) return -1;
  double n[3] = {xij[0] / d, xij[1] / d, xij[2] / d};
  double overlap = R - d;
  double meff = mj > 0.0 ? mi * mj / (mi + mj) : mi;
  double cn = 2.0 * P->zeta * sqrt(P->k_n * meff);
  double vn = vij[0] * n[0] + vij[1] * n[1] + vij[2] * n[2];
  double Fn = P->k_n * overlap - cn * vn; /* signed normal magnitude */
  double vt[3] = {vij[0] - vn * n[0], vij[1] - vn * n[1], vij[2] - vn * n[2]};
  double kt = P->kt_over_cn * cn;
  double ft[3] = {-kt * vt[0], -kt * vt[1], -kt * vt[2]};
  double ftn = sqrt(ft[0] * ft[0] + ft[1] * ft[1] + ft[2] * ft[2]);
  double cap = P->mu * fabs(Fn);
  double s = 1.0; /* F_t = min(|f_t|, cap) * f_t / |f_t| */
  if (ftn > cap) s = cap / ftn;
  for (int a = 0; a < 3; ++a) F[a] = Fn * n[a] + s * ft[a];
  return 1;
}

/* ------------------------------------------------------------------------ */
/* Concentration-gradient force in its capillary form (Sec. 5.4)            */
/* ------------------------------------------------------------------------ */

/* Gamma(sr): the moisture factor, zero for a dry (sr = 0) and a saturated
 * (sr >= 1) neighbourhood, largest (1) at the maximum absorption ratio.  The
 * paper fits it with a Bezier curve without giving its points; reading:
 * the quadratic Bezier curve in the (sr, Gamma) plane through (0, 0) and
 * (1, 0) with middle control point (2 peak - 1/2, 2), whose top, at its
 * parameter t = 1/2, is (peak, 1).  Along it sr(t) = 2 c t (1 - t) + t^2
 * (c = 2 peak - 1/2, increasing in t for c in [0, 1]) and Gamma = 4 t (1 - t);
 * t(sr) is the root in [0, 1] of (1 - 2c) t^2 + 2 c t - sr = 0. */
double or_gamma(double sr, double peak) {
  if (!(sr > 0.0) || !(sr < 1.0)) return 0.0;
  double c = 2.0 * peak - 0.5;
  double t = sr / (c + sqrt(c * c + (1.0 - 2.0 * c) * sr));
  return 4.0 * t * (1.0 - t);
}

/* dGamma/dsr along the same curve (0 outside (0, 1)). */
static double gamma_slope(double sr, double peak) {
  if (!(sr > 0.0) || !(sr < 1.0)) return 0.0;
  double c = 2.0 * peak - 0.5;
  double t = sr / (c + sqrt(c * c + (1.0 - 2.0 * c) * sr));
  return 4.0 * (1.0 - 2.0 * t) / (2.0 * (1.0 - 2.0 * c) * t + 2.0 * c);
}

/* The moisture ratio of Sec. 5.4, sr_i = r_i + alpha_f,i / (1 - alpha_f,i):
 * the water held by the granule plus the free water around it, per unit of
 * sand; +inf where there is no sand (alpha_f = 1). */
double or_moisture_ratio(double moisture, double af) { return af < 1.0 ? moisture + af / (1.0 - af) : INFINITY; }

/* F^st of the liquid bridge at separation s > 0 (Sec. 5.4 with cos theta =
 * 1): 2 pi sigma R (1 - (1 + 2 V* / (pi R s^2))^(-1/2)), the derivative
 * dE/ds of the bridge energy E(s) = -2 pi sigma R (-s + sqrt(s^2 + 2 V* /
 * (pi R))); it tends to 2 pi sigma R as s -> 0 and to 0 as V* -> 0. */
double or_bridge_force(double sigma, double R, double Vs, double s) {
  return 2.0 * OR_PI * sigma * R * (1.0 - 1.0 / sqrt(1.0 + 2.0 * Vs / (OR_PI * R * s * s)));
}

/* dF^st/ds (< 0). */
static double bridge_slope(double sigma, double R, double Vs, double s) {
  double b = 2.0 * Vs / (OR_PI * R);
  double q = 1.0 + b / (s * s);
  return -2.0 * OR_PI * sigma * R * b / (s * s * s) / (q * sqrt(q));
}

/* Rupture distance (Willett et al., cited in Sec. 5.4):
 * d_r = R (v^(1/3) + 0.1 v^(2/3)) with v = V* / R^3.  The paper prints it
 * without the radius; reading: the dimensionless form of the cited formula
 * (distances and volume in units of the radius), the only one of consistent
 * units; for the paper's sizes the two differ by 0.75%. */
double or_rupture(double R, double Vs) {
  double v = Vs / (R * R * R);
  return R * (cbrt(v) + 0.1 * cbrt(v * v));
}

/* Pair constants of the bridge between radii ri and rj: R = 2 ri rj / (ri + rj)
 * (the paper's r for equal spheres), V* = bridge_frac (V_i + V_j) / 2. */
static void bridge_pair(const or_params* P, double ri, double rj, double* R, double* Vs) {
  *R = 2.0 * ri * rj / (ri + rj);
  *Vs = P->bridge_frac * 0.5 * (granule_volume(ri) + granule_volume(rj));
}

/* Capillary force on granule i from j (xij = x_i - x_j), Sec. 5.4:
 * F = -Gamma((sr_i + sr_j) / 2) F^st(s) xij / |xij| for 0 < s < d_r, with
 * s = |xij| - r_i - r_j; granules in contact (s <= 0) feel the contact law
 * instead.  Returns 1 if the force applies. */
static int capillary_force(const or_params* P, const double xij[3], double ri, double rj, double sri, double srj,
                           double F[3]) {
  double d = sqrt(xij[0] * xij[0] + xij[1] * xij[1] + xij[2] * xij[2]);
  double s = d - (ri + rj);
  double R, Vs;
  bridge_pair(P, ri, rj, &R, &Vs);
  if (!(s > 0.0) || !(s < or_rupture(R, Vs))) return 0;
  double f = -or_gamma(0.5 * (sri + srj), P->moisture_peak) * or_bridge_force(P->sigma, R, Vs, s);
  for (int a = 0; a < 3; ++a) F[a] = f * xij[a] / d;
  return 1;
}

/* The largest d_r over the radii present (R and V* grow with the radii). */
static double capillary_reach(const or_params* P, int64_t n, const double* r) {
  if (!(P->sigma > 0.0)) return 0.0;
  double rmax = 0.0;
  for (int64_t i = 0; i < n; ++i) rmax = r[i] > rmax ? r[i] : rmax;
  if (!(rmax > 0.0)) return 0.0;
  return or_rupture(rmax, P->bridge_frac * granule_volume(rmax));
}

/* wall contacts of one granule: the six planes of the box */
static void wall_forces(const or_grid* G, const or_params* P, const double* x, const double* v, double r, double m,
                        double F[3], uint32_t* status) {
  double lo[3] = {G->ox, G->oy, G->oz};
  int nn[3] = {G->nx, G->ny, G->nz};
  for (int a = 0; a < 3; ++a) {
    double hi = lo[a] + nn[a] * G->dx;
    for (int side = 0; side < 2; ++side) {
      double gap = side == 0 ? x[a] - lo[a] : hi - x[a];
      if (gap >= r) continue;
      if (gap <= 0.0) {
        *status |= OR_OUT_OF_DOMAIN;
        continue;
      }
      double xij[3] = {0, 0, 0};
      xij[a] = side == 0 ? gap : -gap;
      double f[3];
      pair_force(P, xij, v, r, 0.0, m, 0.0, f);
      for (int b = 0; b < 3; ++b) F[b] += f[b];
    }
  }
}

/* uniform bins of width >= 2 r_max over the granules' bounding box, for the
 * oracle's own neighbour search (granules outside the box, or NaN, clamp to
 * an edge bin: still correct, only slower) */
typedef struct {
  int nb[3];
  double w[3], lo[3];
  int64_t *head, *next; /* linked lists, ascending index within a bin */
} or_bins;

static void bin_of(const or_bins* B, const double* xi, int bi[3]) {
  for (int a = 0; a < 3; ++a) {
    double f = floor((xi[a] - B->lo[a]) / B->w[a]);
    bi[a] = !(f >= 0.0) ? 0 : (f >= B->nb[a] - 1 ? B->nb[a] - 1 : (int)f); /* NaN -> bin 0 */
  }
}

static void bins_build(or_bins* B, const or_grid* G, int64_t n, const double* x, const double* r, double reach) {
  double rmax = 0;
  for (int64_t i = 0; i < n; ++i) rmax = r[i] > rmax ? r[i] : rmax;
  double hb = 2.0 * rmax + reach; /* every pair that interacts lies in adjacent bins */
  if (!(hb > 0)) hb = G->dx;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) {
      double t = x[3 * i + a];
      if (t < lo[a]) lo[a] = t; /* false for NaN */
      if (t > hi[a]) hi[a] = t;
    }
  int64_t tot = 1;
  for (int a = 0; a < 3; ++a) {
    if (!(hi[a] >= lo[a]) || !isfinite(hi[a] - lo[a])) { /* no finite coordinate */
      lo[a] = 0.0;
      hi[a] = 0.0;
    }
    double ext = hi[a] - lo[a];
    B->nb[a] = ext > hb ? (int)fmin(floor(ext / hb), 2048.0) : 1; /* bin width ext / nb >= 2 r_max */
    tot *= B->nb[a];
  }
  while (tot > 16 * n + 4096) { /* sparse clouds: coarser bins, still >= 2 r_max */
    tot = 1;
    for (int a = 0; a < 3; ++a) {
      B->nb[a] = B->nb[a] > 1 ? B->nb[a] / 2 : 1;
      tot *= B->nb[a];
    }
  }
  for (int a = 0; a < 3; ++a) {
    B->lo[a] = lo[a];
    B->w[a] = B->nb[a] > 1 ? (hi[a] - lo[a]) / B->nb[a] : INFINITY;
  }
  B->head = (int64_t*)malloc(sizeof(int64_t) * (size_t)tot);
  B->next = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t b = 0; b < tot; ++b) B->head[b] = -1;
  /* insert in descending order so each list is ascending */
  for (int64_t i = n - 1; i >= 0; --i) {
    int bi[3];
    bin_of(B, x + 3 * i, bi);
    int64_t lin = bi[0] + (int64_t)B->nb[0] * (bi[1] + (int64_t)B->nb[1] * bi[2]);
    B->next[i] = B->head[lin];
    B->head[lin] = i;
  }
}

static void bins_free(or_bins* B) {
  free(B->head);
  free(B->next);
}

/* Enumerate the contact pairs i < j (d_ij < r_i + r_j).  brute != 0: O(N^2)
 * double loop; else the binned search.  Writes up to max_pairs pairs and
 * returns the total count. */
int64_t or_contact_pairs(const or_grid* G, int64_t n, const double* x, const double* r, int brute, int64_t max_pairs,
                         int64_t* pairs) {
  int64_t m = 0;
  if (brute) {
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = i + 1; j < n; ++j) {
        double d2 = 0;
        for (int a = 0; a < 3; ++a) {
          double t = x[3 * i + a] - x[3 * j + a];
          d2 += t * t;
        }
        double R = r[i] + r[j];
        if (d2 < R * R) {
          if (m < max_pairs) {
            pairs[2 * m] = i;
            pairs[2 * m + 1] = j;
          }
          ++m;
        }
      }
    return m;
  }
  or_bins B;
  bins_build(&B, G, n, x, r, 0.0);
  for (int64_t i = 0; i < n; ++i) {
    int bi[3];
    bin_of(&B, x + 3 * i, bi);
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          int b[3] = {bi[0] + dx, bi[1] + dy, bi[2] + dz};
          if (b[0] < 0 || b[1] < 0 || b[2] < 0 || b[0] >= B.nb[0] || b[1] >= B.nb[1] || b[2] >= B.nb[2]) continue;
          int64_t lin = b[0] + (int64_t)B.nb[0] * (b[1] + (int64_t)B.nb[1] * b[2]);
          for (int64_t j = B.head[lin]; j >= 0; j = B.next[j]) {
            if (j <= i) continue;
            double d2 = 0;
            for (int a = 0; a < 3; ++a) {
              double t = x[3 * i + a] - x[3 * j + a];
              d2 += t * t;
            }
            double R = r[i] + r[j];
            if (d2 < R * R) {
              if (m < max_pairs) {
                pairs[2 * m] = i;
                pairs[2 * m + 1] = j;
              }
              ++m;
            }
          }
        }
  }
  bins_free(&B);
  return m;
}

/* Force on granule i from partner j: the contact law while they overlap,
 * else (with sigma > 0) the capillary force within the rupture distance. */
static void pair_total(const or_params* P, const double* x, const double* v, const double* r, const double* sr,
                       int64_t i, int64_t j, double mi, double Fi[3], uint32_t* status) {
  double xij[3], vij[3], f[3];
  for (int a = 0; a < 3; ++a) {
    xij[a] = x[3 * i + a] - x[3 * j + a];
    vij[a] = v[3 * i + a] - v[3 * j + a];
  }
  int c = pair_force(P, xij, vij, r[i], r[j], mi, P->rho_s * granule_volume(r[j]), f);
  if (c < 0) *status |= OR_COINCIDENT;
  if (c == 0 && sr) c = capillary_force(P, xij, r[i], r[j], sr[i], sr[j], f);
  if (c > 0)
    for (int a = 0; a < 3; ++a) Fi[a] += f[a];
}

static void moisture_ratios(const or_grid* G, const or_params* P, int64_t n, const double* x, const double* af,
                            double* sr, double* gsr);

/* Force on every granule from its partners: the contact law over all
 * partners with d < r_i + r_j and, with sigma > 0, the capillary force
 * (af: the cell-centred fluid fraction field, interpolated at each granule
 * as G2P does), plus the walls.  brute != 0 uses the O(N^2) loop. */
void or_contact(const or_grid* G, const or_params* P, int64_t n, const double* x, const double* v, const double* r,
                const double* af, int brute, double* F, uint32_t* status) {
  or_bins B;
  double* sr = NULL;
  if (P->sigma > 0.0) {
    sr = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    moisture_ratios(G, P, n, x, af, sr, NULL);
  }
  if (!brute) bins_build(&B, G, n, x, r, capillary_reach(P, n, r));
  for (int64_t i = 0; i < n; ++i) {
    double Fi[3] = {0, 0, 0};
    double mi = P->rho_s * granule_volume(r[i]);
    const double* xi = x + 3 * i;
    const double* vi = v + 3 * i;
    if (brute) {
      for (int64_t j = 0; j < n; ++j)
        if (j != i) pair_total(P, x, v, r, sr, i, j, mi, Fi, status);
    } else {
      int bi[3];
      bin_of(&B, xi, bi);
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            int b[3] = {bi[0] + dx, bi[1] + dy, bi[2] + dz};
            if (b[0] < 0 || b[1] < 0 || b[2] < 0 || b[0] >= B.nb[0] || b[1] >= B.nb[1] || b[2] >= B.nb[2]) continue;
            int64_t lin = b[0] + (int64_t)B.nb[0] * (b[1] + (int64_t)B.nb[1] * b[2]);
            for (int64_t j = B.head[lin]; j >= 0; j = B.next[j])
              if (j != i) pair_total(P, x, v, r, sr, i, j, mi, Fi, status);
          }
    }
    if (P->walls) wall_forces(G, P, xi, vi, r[i], mi, Fi, status);
    for (int a = 0; a < 3; ++a) F[3 * i + a] = Fi[a];
  }
  if (!brute) bins_free(&B);
  free(sr);
}

/* ------------------------------------------------------------------------ */
/* interpolation kernel N (trilinear tent on MAC samples), Sec. 5.1 / 5.2   */
/* ------------------------------------------------------------------------ */

/* One axis: samples at (k + s) dx, k = 0..ns-1.  Lower sample i0 and the
 * weight t of sample i0+1 (1 - t on i0).  A point beyond the first or last
 * sample is clamped onto it. */
static void axis_stencil(double xg, double s, int ns, int* i0, double* t) {
  double f = xg - s;
  if (!(f > 0.0)) { /* also NaN */
    *i0 = 0;
    *t = 0.0;
    return;
  }
  if (f >= (double)(ns - 1)) {
    *i0 = ns - 2;
    *t = 1.0;
    return;
  }
  double fl = floor(f);
  *i0 = (int)fl;
  *t = f - fl;
}

/* A sampled MAC field: ns samples per axis, sample offsets s (in cells). */
typedef struct {
  int ns[3];
  double s[3];
} or_layout;

static or_layout layout_of(const or_grid* G, int comp) {
  /* comp 0,1,2: u, v, w faces; 3: cell centres */
  or_layout L;
  int n[3] = {G->nx, G->ny, G->nz};
  for (int a = 0; a < 3; ++a) {
    L.ns[a] = n[a] + (a == comp ? 1 : 0);
    L.s[a] = a == comp ? 0.0 : 0.5;
  }
  return L;
}

/* sample index (x fastest) */
static int64_t sidx(const or_layout* L, int i, int j, int k) {
  return i + (int64_t)L->ns[0] * (j + (int64_t)L->ns[1] * k);
}

/* weights of the 8 stencil samples of point x for layout L */
typedef struct {
  int i0[3];
  double t[3];
} or_stencil;

static or_stencil stencil_at(const or_grid* G, const or_layout* L, const double* x) {
  or_stencil S;
  double o[3] = {G->ox, G->oy, G->oz};
  for (int a = 0; a < 3; ++a) axis_stencil((x[a] - o[a]) / G->dx, L->s[a], L->ns[a], &S.i0[a], &S.t[a]);
  return S;
}

static double corner_weight(const or_stencil* S, int a, int b, int c) {
  double wx = a ? S->t[0] : 1.0 - S->t[0];
  double wy = b ? S->t[1] : 1.0 - S->t[1];
  double wz = c ? S->t[2] : 1.0 - S->t[2];
  return wx * wy * wz;
}

/* Pressure gradient component `comp` on its face sample (i,j,k): (p_i - p_{i-1}) / dx
 * along `comp`; boundary faces take the adjacent interior face's value. */
static double grad_p_face(const or_grid* G, const double* p, int comp, int i, int j, int k) {
  int idx[3] = {i, j, k};
  int n[3] = {G->nx, G->ny, G->nz};
  int c = idx[comp];
  if (c < 1) c = 1;
  if (c > n[comp] - 1) c = n[comp] - 1;
  int hi[3] = {idx[0], idx[1], idx[2]};
  int lo[3] = {idx[0], idx[1], idx[2]};
  hi[comp] = c;
  lo[comp] = c - 1;
  int64_t ih = hi[0] + (int64_t)G->nx * (hi[1] + (int64_t)G->ny * hi[2]);
  int64_t il = lo[0] + (int64_t)G->nx * (lo[1] + (int64_t)G->ny * lo[2]);
  return (p[ih] - p[il]) / G->dx;
}

/* interpolate a plain sampled field */
static double interp(const or_grid* G, const or_layout* L, const double* f, const double* x) {
  or_stencil S = stencil_at(G, L, x);
  double acc = 0.0;
  for (int c = 0; c < 2; ++c)
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a)
        acc += corner_weight(&S, a, b, c) * f[sidx(L, S.i0[0] + a, S.i0[1] + b, S.i0[2] + c)];
  return acc;
}

/* interpolate grad p component comp (sampled on comp-faces) */
static double interp_grad_p(const or_grid* G, const double* p, int comp, const double* x) {
  or_layout L = layout_of(G, comp);
  or_stencil S = stencil_at(G, &L, x);
  double acc = 0.0;
  for (int c = 0; c < 2; ++c)
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a)
        acc += corner_weight(&S, a, b, c) * grad_p_face(G, p, comp, S.i0[0] + a, S.i0[1] + b, S.i0[2] + c);
  return acc;
}

/* Public helper for tests: interpolate field `comp` (0..2 faces, 3 centres)
 * at m points. */
void or_interp(const or_grid* G, int comp, const double* f, int64_t m, const double* x, double* out) {
  or_layout L = layout_of(G, comp);
  for (int64_t i = 0; i < m; ++i) out[i] = interp(G, &L, f, x + 3 * i);
}

void or_interp_grad_p(const or_grid* G, const double* p, int64_t m, const double* x, double* out /*3m*/) {
  for (int64_t i = 0; i < m; ++i)
    for (int a = 0; a < 3; ++a) out[3 * i + a] = interp_grad_p(G, p, a, x + 3 * i);
}

/* ------------------------------------------------------------------------ */
/* CalCoupling: G2P of fluid velocity, grad p and alpha_f (Sec. 3.3, 5.2)   */
/* ------------------------------------------------------------------------ */

/* F_fl = F_d + F_p,  F_p = -(4/3) pi r^3 grad p (Eq. gradient-force),
 * F_d = c_drag pi r^2 rho_f |u_f - v| (u_f - v) (Eq. 5b with the drag reading),
 * a_f = dv_f/dt = g - grad p / rho_f (Eq. momentum4 without the F_s term),
 * alpha_f_p = alpha_f interpolated at the granule. */
static double interp_grad_layout(const or_grid* G, const or_layout* L, const double* f, int gp_comp, const double* p,
                                 const double* x, double grad[3]);

/* sr_i = r_i + alpha_f,i / (1 - alpha_f,i) at every granule (Sec. 5.4) from the
 * cell-centred fluid fraction interpolated as G2P does, and (gsr, 3n, may be
 * NULL) its gradient w.r.t. the granule's position: d sr / d alpha =
 * 1 / (1 - alpha)^2 times the gradient of the interpolated alpha_f (zero
 * along an axis where the point is clamped onto an end sample). */
static void moisture_ratios(const or_grid* G, const or_params* P, int64_t n, const double* x, const double* af,
                            double* sr, double* gsr) {
  or_layout Lc = layout_of(G, 3);
  for (int64_t i = 0; i < n; ++i) {
    double g[3];
    double a = interp_grad_layout(G, &Lc, af, -1, NULL, x + 3 * i, g);
    sr[i] = or_moisture_ratio(P->moisture, a);
    if (gsr) {
      double k = a < 1.0 ? 1.0 / ((1.0 - a) * (1.0 - a)) : 0.0;
      for (int c = 0; c < 3; ++c) gsr[3 * i + c] = k * g[c];
    }
  }
}

void or_g2p(const or_grid* G, const or_params* P, int64_t n, const double* x, const double* v, const double* r,
            const double* u, const double* vf, const double* wf, const double* p, const double* af, double* F_fl,
            double* a_f, double* alpha_f_p) {
  or_layout Lu = layout_of(G, 0), Lv = layout_of(G, 1), Lw = layout_of(G, 2), Lc = layout_of(G, 3);
  double g[3] = {P->gx, P->gy, P->gz};
  for (int64_t i = 0; i < n; ++i) {
    const double* xi = x + 3 * i;
    double uf[3] = {interp(G, &Lu, u, xi), interp(G, &Lv, vf, xi), interp(G, &Lw, wf, xi)};
    double gp[3];
    for (int a = 0; a < 3; ++a) gp[a] = interp_grad_p(G, p, a, xi);
    double V = granule_volume(r[i]);
    double dv[3] = {uf[0] - v[3 * i], uf[1] - v[3 * i + 1], uf[2] - v[3 * i + 2]};
    double sp = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    double cd = P->c_drag * OR_PI * r[i] * r[i] * P->rho_f * sp;
    for (int a = 0; a < 3; ++a) {
      F_fl[3 * i + a] = cd * dv[a] - V * gp[a];
      a_f[3 * i + a] = P->rho_f > 0.0 ? g[a] - gp[a] / P->rho_f : g[a];
    }
    alpha_f_p[i] = interp(G, &Lc, af, xi);
  }
}

/* ------------------------------------------------------------------------ */
/* MoveParticle: virtual-mass symplectic Euler (Sec. 5.2 Eq. sand kine)     */
/* ------------------------------------------------------------------------ */

/* (m + m_a) a = m_a a_f + F_c + F_fl + m g,  m_a = (2/3) pi r^3 rho_f;
 * v' = v + dt a;  x' = x + dt v';  exchange force f = F_fl + m_a (a_f - a).
 * A granule whose new position leaves the box is put back on the boundary
 * it crossed, per axis: onto the lower plane itself, or onto the largest
 * position below the upper plane that the canonical encoding holds (h_c
 * 2^-30 inside), and flagged; its velocity is kept.  (The paper has no
 * rule for this; positions live in the grid's cells, so none lies outside.) */
void or_integrate(const or_grid* G, const or_params* P, int64_t n, const double* x, const double* v, const double* r,
                  const double* F_c, const double* F_fl, const double* a_f, double* x_new, double* v_new, double* f_ex,
                  uint32_t* status) {
  double g[3] = {P->gx, P->gy, P->gz};
  double lo[3] = {G->ox, G->oy, G->oz};
  double hi[3] = {G->ox + G->nx * G->dx, G->oy + G->ny * G->dx, G->oz + G->nz * G->dx};
  for (int64_t i = 0; i < n; ++i) {
    double V = granule_volume(r[i]);
    double m = P->rho_s * V;
    double ma = P->virtual_mass ? 0.5 * P->rho_f * V : 0.0;
    for (int a = 0; a < 3; ++a) {
      double acc = (F_c[3 * i + a] + F_fl[3 * i + a] + m * g[a] + ma * a_f[3 * i + a]) / (m + ma);
      double vn = v[3 * i + a] + P->dt * acc;
      double xn = x[3 * i + a] + P->dt * vn;
      if (!isfinite(vn) || !isfinite(xn)) *status |= OR_NONFINITE;
      if (xn < lo[a]) {
        xn = lo[a];
        *status |= OR_OUT_OF_DOMAIN;
      } else if (xn >= hi[a]) {
        xn = hi[a] - G->dx / G->k / 1073741824.0;
        *status |= OR_OUT_OF_DOMAIN;
      }
      v_new[3 * i + a] = vn;
      x_new[3 * i + a] = xn;
      f_ex[3 * i + a] = F_fl[3 * i + a] + ma * (a_f[3 * i + a] - acc);
    }
  }
}

/* ------------------------------------------------------------------------ */
/* TransferCoupling: P2G (Sec. 5.1 alpha_s, Sec. 5.2 exchange momentum)     */
/* ------------------------------------------------------------------------ */

/* alpha_s(c) = (1/dx^3) sum_i V_i N(x_new_i - x_c)       (written, cell centres)
 * F_s(face) += -(dt'/dt) sum_i f_i N(x_old_i - x_face)   (accumulated, MAC faces)
 * sums[0] = sum_c alpha_s(c) dx^3,  sums[1] = sum_i V_i */
void or_p2g(const or_grid* G, const or_params* P, int64_t n, const double* x_old, const double* x_new, const double* r,
            const double* f_ex, double* alpha_s, double* Fs_u, double* Fs_v, double* Fs_w, double* sums) {
  or_layout Lc = layout_of(G, 3);
  int64_t ncell = (int64_t)G->nx * G->ny * G->nz;
  double dx3 = G->dx * G->dx * G->dx;
  for (int64_t c = 0; c < ncell; ++c) alpha_s[c] = 0.0;
  double* Fs[3] = {Fs_u, Fs_v, Fs_w};
  double scale = -P->dt / P->dt_fluid;
  double sumV = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double V = granule_volume(r[i]);
    sumV += V;
    or_stencil S = stencil_at(G, &Lc, x_new + 3 * i);
    for (int c = 0; c < 2; ++c)
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a)
          alpha_s[sidx(&Lc, S.i0[0] + a, S.i0[1] + b, S.i0[2] + c)] += V / dx3 * corner_weight(&S, a, b, c);
    for (int comp = 0; comp < 3; ++comp) {
      or_layout L = layout_of(G, comp);
      or_stencil T = stencil_at(G, &L, x_old + 3 * i);
      for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b)
          for (int a = 0; a < 2; ++a)
            Fs[comp][sidx(&L, T.i0[0] + a, T.i0[1] + b, T.i0[2] + c)] +=
                scale * f_ex[3 * i + comp] * corner_weight(&T, a, b, c);
    }
  }
  double tot = 0.0;
  for (int64_t c = 0; c < ncell; ++c) tot += alpha_s[c] * dx3;
  sums[0] = tot;
  sums[1] = sumV;
}

/* ------------------------------------------------------------------------ */
/* SandSubstep loop (Algorithm 2), K substeps, state updated in place       */
/* ------------------------------------------------------------------------ */

typedef struct {
  const double *u, *vf, *wf, *p, *af;
} or_fluid;

/* One substep.  Scratch arrays of 3n doubles: F_c, F_fl, a_f, f_ex, x_new,
 * v_new; n doubles alpha_f_p. */
static void substep(const or_grid* G, const or_params* P, const or_fluid* Fd, int64_t n, double* x, double* v,
                    const double* r, double* alpha_s, double* Fs_u, double* Fs_v, double* Fs_w, double* sums,
                    int brute, double* scratch, uint32_t* status) {
  double* F_c = scratch;
  double* F_fl = F_c + 3 * n;
  double* a_f = F_fl + 3 * n;
  double* f_ex = a_f + 3 * n;
  double* x_new = f_ex + 3 * n;
  double* v_new = x_new + 3 * n;
  double* afp = v_new + 3 * n;
  or_g2p(G, P, n, x, v, r, Fd->u, Fd->vf, Fd->wf, Fd->p, Fd->af, F_fl, a_f, afp);
  or_contact(G, P, n, x, v, r, Fd->af, brute, F_c, status);
  or_integrate(G, P, n, x, v, r, F_c, F_fl, a_f, x_new, v_new, f_ex, status);
  or_p2g(G, P, n, x, x_new, r, f_ex, alpha_s, Fs_u, Fs_v, Fs_w, sums);
  memcpy(x, x_new, sizeof(double) * 3 * (size_t)n);
  memcpy(v, v_new, sizeof(double) * 3 * (size_t)n);
}

/* K substeps.  x, v (3n) updated in place; alpha_s is the last substep's;
 * F_s accumulates over all K substeps (caller zeroes it); sums = last
 * substep's conservation sums. */
void or_run(const or_grid* G, const or_params* P, int64_t n, int K, double* x, double* v, const double* r,
            const double* u, const double* vf, const double* wf, const double* p, const double* af, double* alpha_s,
            double* Fs_u, double* Fs_v, double* Fs_w, double* sums, int brute, uint32_t* status) {
  or_fluid Fd = {u, vf, wf, p, af};
  double* scratch = (double*)malloc(sizeof(double) * (size_t)(19 * (n > 0 ? n : 1)));
  for (int s = 0; s < K; ++s) substep(G, P, &Fd, n, x, v, r, alpha_s, Fs_u, Fs_v, Fs_w, sums, brute, scratch, status);
  free(scratch);
}

/* ======================================================================== */
/* ADJOINT (hand-derived, explicit Jacobians)                               */
/*                                                                          */
/* The paper has no gradients; these are the exact derivatives of the       */
/* forward functions above, written out as 3x3 Jacobians (not as a replay   */
/* of the forward code), so the CUDA reverse-mode kernels are checked       */
/* against an independent derivation.  Non-smooth points (contact onset,    */
/* the Coulomb switch, clamped interpolation) take the one-sided branch the */
/* forward takes.                                                           */
/* ======================================================================== */

typedef struct {
  double m[3][3];
} or_m3;

static void m3_zero(or_m3* A) { memset(A, 0, sizeof(*A)); }
/* y += A^T x */
static void m3_tmul_add(const or_m3* A, const double x[3], double y[3]) {
  for (int b = 0; b < 3; ++b)
    for (int a = 0; a < 3; ++a) y[b] += A->m[a][b] * x[a];
}

/* Jacobians of the pair force F(x, v) of pair_force w.r.t. x = x_i - x_j and
 * v = v_i - v_j, and dF/dmu.  Returns 0 if the pair is not in contact. */
static int pair_force_jac(const or_params* P, const double x[3], const double v[3], double ri, double rj, double mi,
                          double mj, or_m3* Jx, or_m3* Jv, double dmu[3], int* slip_out) {
  double d2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
  double R = ri + rj;
  if (!(d2 < R * R)) return 0;
  double d = sqrt(d2);
  if (d == 0.0) return 0;
  double n[3] = {x[0] / d, x[1] / d, x[2] / d};
  double meff = mj > 0.0 ? mi * mj / (mi + mj) : mi;
  double cn = 2.0 * P->zeta * sqrt(P->k_n * meff);
  double kt = P->kt_over_cn * cn;
  double vn = v[0] * n[0] + v[1] * n[1] + v[2] * n[2];
  double Fn = P->k_n * (R - d) - cn * vn;
  double vt[3] = {v[0] - vn * n[0], v[1] - vn * n[1], v[2] - vn * n[2]};
  double vtn = sqrt(vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2]);
  int slip = kt * vtn > P->mu * fabs(Fn);
  /* projector Pn = I - n n^T */
  double Pn[3][3], dndx[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      Pn[a][b] = (a == b ? 1.0 : 0.0) - n[a] * n[b];
      dndx[a][b] = Pn[a][b] / d;
    }
  /* d vn / dx = v^T dn/dx,  d vn / dv = n^T */
  double dvn_dx[3];
  for (int b = 0; b < 3; ++b) dvn_dx[b] = v[0] * dndx[0][b] + v[1] * dndx[1][b] + v[2] * dndx[2][b];
  /* d Fn / dx = -k_n n^T - cn dvn/dx,  d Fn / dv = -cn n^T */
  double dFn_dx[3], dFn_dv[3];
  for (int b = 0; b < 3; ++b) {
    dFn_dx[b] = -P->k_n * n[b] - cn * dvn_dx[b];
    dFn_dv[b] = -cn * n[b];
  }
  /* d vt / dx = -n dvn/dx - vn dn/dx,  d vt / dv = Pn */
  double dvt_dx[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) dvt_dx[a][b] = -n[a] * dvn_dx[b] - vn * dndx[a][b];
  m3_zero(Jx);
  m3_zero(Jv);
  /* normal part Fn n */
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      Jx->m[a][b] += n[a] * dFn_dx[b] + Fn * dndx[a][b];
      Jv->m[a][b] += n[a] * dFn_dv[b];
    }
  dmu[0] = dmu[1] = dmu[2] = 0.0;
  if (!slip) {
    /* F_t = -kt vt */
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        Jx->m[a][b] += -kt * dvt_dx[a][b];
        Jv->m[a][b] += -kt * Pn[a][b];
      }
  } else {
    /* F_t = -mu |Fn| u, u = vt / |vt| */
    double u[3] = {vt[0] / vtn, vt[1] / vtn, vt[2] / vtn};
    double sg = Fn > 0 ? 1.0 : (Fn < 0 ? -1.0 : 0.0);
    double A = P->mu * fabs(Fn);
    double Q[3][3]; /* du/dvt = (I - u u^T) / |vt| */
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) Q[a][b] = ((a == b ? 1.0 : 0.0) - u[a] * u[b]) / vtn;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double qx = 0, qv = 0;
        for (int c = 0; c < 3; ++c) {
          qx += Q[a][c] * dvt_dx[c][b];
          qv += Q[a][c] * Pn[c][b];
        }
        Jx->m[a][b] += -P->mu * sg * u[a] * dFn_dx[b] - A * qx;
        Jv->m[a][b] += -P->mu * sg * u[a] * dFn_dv[b] - A * qv;
      }
    for (int a = 0; a < 3; ++a) dmu[a] = -fabs(Fn) * u[a];
  }
  if (slip_out) *slip_out = slip;
  return 1;
}

/* Jacobians of the capillary force of capillary_force: Jx = dF/dxij and
 * dsr = dF/d(sr_mean), sr_mean = (sr_i + sr_j) / 2.  F = -Gamma F^st n gives
 * dF/dx = -Gamma (dF^st/ds n n^T + F^st / d (I - n n^T)) and
 * dF/dsr_mean = -Gamma' F^st n.  Returns 0 outside 0 < s < d_r. */
static int capillary_jac(const or_params* P, const double x[3], double ri, double rj, double sri, double srj,
                         or_m3* Jx, double dsr[3]) {
  double d = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  double s = d - (ri + rj);
  double R, Vs;
  bridge_pair(P, ri, rj, &R, &Vs);
  if (!(s > 0.0) || !(s < or_rupture(R, Vs))) return 0;
  double n[3] = {x[0] / d, x[1] / d, x[2] / d};
  double srm = 0.5 * (sri + srj);
  double g = or_gamma(srm, P->moisture_peak);
  double gp = gamma_slope(srm, P->moisture_peak);
  double Fs = or_bridge_force(P->sigma, R, Vs, s);
  double Fp = bridge_slope(P->sigma, R, Vs, s);
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b)
      Jx->m[a][b] = -g * (Fp * n[a] * n[b] + Fs / d * ((a == b ? 1.0 : 0.0) - n[a] * n[b]));
    dsr[a] = -gp * Fs * n[a];
  }
  return 1;
}

/* contact adjoint: gx_i += sum_j Jx_ij^T (l_i - l_j), gv_i likewise,
 * g_mu += sum_i l_i . dF_i/dmu.  Walls: partner gradient zero.  With the
 * capillary force (sigma > 0, af = the cell-centred fluid fraction) the pair
 * force also depends on x_i through sr_i(x_i): gx_i += (1/2) ((l_i - l_j) .
 * dF/dsr_mean) dsr_i/dx_i; the gather form holds because F_ji = -F_ij as
 * functions of both positions. */
void or_contact_adj(const or_grid* G, const or_params* P, int64_t n, const double* x, const double* v,
                    const double* r, const double* af, const double* gF, int brute, double* gx, double* gv,
                    double* g_mu) {
  or_bins B;
  double *sr = NULL, *gsr = NULL;
  if (P->sigma > 0.0) {
    sr = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    gsr = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    moisture_ratios(G, P, n, x, af, sr, gsr);
  }
  if (!brute) bins_build(&B, G, n, x, r, capillary_reach(P, n, r));
  double gm = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double mi = P->rho_s * granule_volume(r[i]);
    const double* li = gF + 3 * i;
    /* candidate partners: every j (brute) or the 27 bins around i */
    int64_t* cand = NULL;
    int64_t nc = 0;
    if (brute) {
      cand = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
      for (int64_t j = 0; j < n; ++j) cand[nc++] = j;
    } else {
      int bi[3];
      bin_of(&B, x + 3 * i, bi);
      int64_t cap = 64;
      cand = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            int b[3] = {bi[0] + dx, bi[1] + dy, bi[2] + dz};
            if (b[0] < 0 || b[1] < 0 || b[2] < 0 || b[0] >= B.nb[0] || b[1] >= B.nb[1] || b[2] >= B.nb[2]) continue;
            int64_t lin = b[0] + (int64_t)B.nb[0] * (b[1] + (int64_t)B.nb[1] * b[2]);
            for (int64_t j = B.head[lin]; j >= 0; j = B.next[j]) {
              if (nc == cap) {
                cap *= 2;
                cand = (int64_t*)realloc(cand, sizeof(int64_t) * (size_t)cap);
              }
              cand[nc++] = j;
            }
          }
    }
    for (int64_t c = 0; c < nc; ++c) {
      int64_t j = cand[c];
      if (j == i) continue;
      double xij[3], vij[3], lam[3], dmu[3];
      for (int a = 0; a < 3; ++a) {
        xij[a] = x[3 * i + a] - x[3 * j + a];
        vij[a] = v[3 * i + a] - v[3 * j + a];
        lam[a] = li[a] - gF[3 * j + a];
      }
      or_m3 Jx, Jv;
      if (!pair_force_jac(P, xij, vij, r[i], r[j], mi, P->rho_s * granule_volume(r[j]), &Jx, &Jv, dmu, NULL)) {
        double dsr[3];
        if (sr && isfinite(sr[i]) && isfinite(sr[j]) && capillary_jac(P, xij, r[i], r[j], sr[i], sr[j], &Jx, dsr)) {
          m3_tmul_add(&Jx, lam, gx + 3 * i);
          double w = 0.5 * (lam[0] * dsr[0] + lam[1] * dsr[1] + lam[2] * dsr[2]);
          for (int a = 0; a < 3; ++a) gx[3 * i + a] += w * gsr[3 * i + a];
        }
        continue;
      }
      m3_tmul_add(&Jx, lam, gx + 3 * i);
      m3_tmul_add(&Jv, lam, gv + 3 * i);
      gm += li[0] * dmu[0] + li[1] * dmu[1] + li[2] * dmu[2];
    }
    free(cand);
    if (P->walls) {
      double lo[3] = {G->ox, G->oy, G->oz};
      int nn[3] = {G->nx, G->ny, G->nz};
      for (int a = 0; a < 3; ++a) {
        double hi = lo[a] + nn[a] * G->dx;
        for (int side = 0; side < 2; ++side) {
          double gap = side == 0 ? x[3 * i + a] - lo[a] : hi - x[3 * i + a];
          if (gap >= r[i] || gap <= 0.0) continue;
          double xw[3] = {0, 0, 0}, dmu[3];
          xw[a] = side == 0 ? gap : -gap;
          or_m3 Jx, Jv;
          if (!pair_force_jac(P, xw, v + 3 * i, r[i], 0.0, mi, 0.0, &Jx, &Jv, dmu, NULL)) continue;
          /* x_w = +-(x_i - wall): d x_w / d x_i = I on this axis only, 0 on the others */
          double tmp[3] = {0, 0, 0};
          m3_tmul_add(&Jx, li, tmp);
          gx[3 * i + a] += tmp[a];
          m3_tmul_add(&Jv, li, gv + 3 * i);
          gm += li[0] * dmu[0] + li[1] * dmu[1] + li[2] * dmu[2];
        }
      }
    }
  }
  *g_mu += gm;
  if (!brute) bins_free(&B);
  free(sr);
  free(gsr);
}

/* value and x-gradient of the interpolation of a sampled field */
static double interp_grad_layout(const or_grid* G, const or_layout* L, const double* f, int gp_comp, const double* p,
                                 const double* x, double grad[3]) {
  double o[3] = {G->ox, G->oy, G->oz};
  or_stencil S;
  int clamped[3];
  for (int a = 0; a < 3; ++a) {
    double xg = (x[a] - o[a]) / G->dx;
    double fpos = xg - L->s[a];
    clamped[a] = !(fpos > 0.0) || fpos >= (double)(L->ns[a] - 1);
    axis_stencil(xg, L->s[a], L->ns[a], &S.i0[a], &S.t[a]);
  }
  double val = 0.0, g[3] = {0, 0, 0};
  for (int c = 0; c < 2; ++c)
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        double fv = gp_comp >= 0 ? grad_p_face(G, p, gp_comp, S.i0[0] + a, S.i0[1] + b, S.i0[2] + c)
                                 : f[sidx(L, S.i0[0] + a, S.i0[1] + b, S.i0[2] + c)];
        double wx = a ? S.t[0] : 1.0 - S.t[0];
        double wy = b ? S.t[1] : 1.0 - S.t[1];
        double wz = c ? S.t[2] : 1.0 - S.t[2];
        val += wx * wy * wz * fv;
        g[0] += (a ? 1.0 : -1.0) * wy * wz * fv;
        g[1] += wx * (b ? 1.0 : -1.0) * wz * fv;
        g[2] += wx * wy * (c ? 1.0 : -1.0) * fv;
      }
  for (int a = 0; a < 3; ++a) grad[a] = clamped[a] ? 0.0 : g[a] / G->dx;
  return val;
}

/* G2P adjoint.  gx, gv accumulated; g_cdrag accumulated. galpha may be NULL. */
void or_g2p_adj(const or_grid* G, const or_params* P, int64_t n, const double* x, const double* v, const double* r,
                const double* u, const double* vf, const double* wf, const double* p, const double* af,
                const double* gFfl, const double* gaf, const double* galpha, double* gx, double* gv,
                double* g_cdrag) {
  const double* uvw[3] = {u, vf, wf};
  double gc = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const double* xi = x + 3 * i;
    double uf[3], Du[3][3], H[3][3];
    for (int comp = 0; comp < 3; ++comp) {
      or_layout L = layout_of(G, comp);
      uf[comp] = interp_grad_layout(G, &L, uvw[comp], -1, NULL, xi, Du[comp]);
      interp_grad_layout(G, &L, NULL, comp, p, xi, H[comp]);
    }
    double V = granule_volume(r[i]);
    double k = P->c_drag * OR_PI * r[i] * r[i] * P->rho_f;
    double dv[3] = {uf[0] - v[3 * i], uf[1] - v[3 * i + 1], uf[2] - v[3 * i + 2]};
    double sp = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    double D[3][3]; /* d F_d / d dv = k (|dv| I + dv dv^T / |dv|) */
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) D[a][b] = sp > 0 ? k * ((a == b ? sp : 0.0) + dv[a] * dv[b] / sp) : 0.0;
    const double* lF = gFfl + 3 * i;
    const double* la = gaf + 3 * i;
    /* dF_fl/dx = D Du - V H ; da_f/dx = -H / rho_f ; dF_fl/dv = -D */
    for (int b = 0; b < 3; ++b) {
      double s = 0.0, t = 0.0;
      for (int a = 0; a < 3; ++a) {
        double DDu = 0.0;
        for (int c = 0; c < 3; ++c) DDu += D[a][c] * Du[c][b];
        s += lF[a] * (DDu - V * H[a][b]);
        if (P->rho_f > 0) s += la[a] * (-H[a][b] / P->rho_f);
        t += lF[a] * (-D[a][b]);
      }
      gx[3 * i + b] += s;
      gv[3 * i + b] += t;
    }
    if (galpha) {
      or_layout Lc = layout_of(G, 3);
      double ga[3];
      interp_grad_layout(G, &Lc, af, -1, NULL, xi, ga);
      for (int b = 0; b < 3; ++b) gx[3 * i + b] += galpha[i] * ga[b];
    }
    /* dF_d / dc_drag = pi r^2 rho_f |dv| dv */
    double q = OR_PI * r[i] * r[i] * P->rho_f * sp;
    gc += q * (dv[0] * lF[0] + dv[1] * lF[1] + dv[2] * lF[2]);
  }
  *g_cdrag += gc;
}

/* integrate adjoint: writes gx, gv, gFc, gFfl, gaf from gx_new, gv_new, gfex (may be NULL) */
void or_integrate_adj(const or_grid* G, const or_params* P, int64_t n, const double* r, const double* gx_new,
                      const double* gv_new, const double* gfex, double* gx, double* gv, double* gFc, double* gFfl,
                      double* gaf) {
  (void)G;
  double dt = P->dt;
  for (int64_t i = 0; i < n; ++i) {
    double V = granule_volume(r[i]);
    double m = P->rho_s * V;
    double ma = P->virtual_mass ? 0.5 * P->rho_f * V : 0.0;
    double M = m + ma;
    for (int a = 0; a < 3; ++a) {
      double gX = gx_new[3 * i + a], gV = gv_new[3 * i + a], gf = gfex ? gfex[3 * i + a] : 0.0;
      /* x' = x + dt v + dt^2 a, v' = v + dt a, f = F_fl + ma (a_f - a) */
      double through_a = dt * dt / M * gX + dt / M * gV; /* d(x', v')/dF . g for F in {F_c, F_fl} */
      gx[3 * i + a] = gX;
      gv[3 * i + a] = dt * gX + gV;
      gFc[3 * i + a] = through_a - ma / M * gf;
      gFfl[3 * i + a] = through_a + (1.0 - ma / M) * gf;
      gaf[3 * i + a] = ma * through_a + ma * m / M * gf;
    }
  }
}

/* P2G adjoint: gx_old, gx_new accumulated; gfex written.  g_alpha and gFs
 * (all three) may be NULL. */
void or_p2g_adj(const or_grid* G, const or_params* P, int64_t n, const double* x_old, const double* x_new,
                const double* r, const double* f_ex, const double* g_alpha, const double* gFs_u, const double* gFs_v,
                const double* gFs_w, double* gx_old, double* gx_new, double* gfex) {
  const double* gF[3] = {gFs_u, gFs_v, gFs_w};
  double dx3 = G->dx * G->dx * G->dx;
  double scale = -P->dt / P->dt_fluid;
  for (int64_t i = 0; i < n; ++i) {
    if (g_alpha) {
      or_layout Lc = layout_of(G, 3);
      double g[3];
      interp_grad_layout(G, &Lc, g_alpha, -1, NULL, x_new + 3 * i, g);
      double s = granule_volume(r[i]) / dx3;
      for (int a = 0; a < 3; ++a) gx_new[3 * i + a] += s * g[a];
    }
    for (int comp = 0; comp < 3; ++comp) {
      if (!gF[comp]) {
        gfex[3 * i + comp] = 0.0;
        continue;
      }
      or_layout L = layout_of(G, comp);
      double g[3];
      double val = interp_grad_layout(G, &L, gF[comp], -1, NULL, x_old + 3 * i, g);
      gfex[3 * i + comp] = scale * val;
      for (int a = 0; a < 3; ++a) gx_old[3 * i + a] += scale * f_ex[3 * i + comp] * g[a];
    }
  }
}

/* Contact signature of one state: number of contacts, number slipping and
 * an order-free hash of (i, j, slip) -- used to tell whether a finite-
 * difference pair of runs saw the same contact set. */
static void contact_signature(const or_grid* G, const or_params* P, int64_t n, const double* x, const double* v,
                              const double* r, const double* af, uint64_t sig[3]) {
  int64_t m = 0, ms = 0;
  uint64_t h = 0;
  double* sr = NULL;
  if (P->sigma > 0.0) { /* capillary pairs (0 < s < d_r) count as a third kind of pair */
    sr = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    moisture_ratios(G, P, n, x, af, sr, NULL);
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j) {
      double xij[3], vij[3], dmu[3];
      for (int a = 0; a < 3; ++a) {
        xij[a] = x[3 * i + a] - x[3 * j + a];
        vij[a] = v[3 * i + a] - v[3 * j + a];
      }
      or_m3 Jx, Jv;
      int slip = 0;
      if (!pair_force_jac(P, xij, vij, r[i], r[j], P->rho_s * granule_volume(r[i]),
                          P->rho_s * granule_volume(r[j]), &Jx, &Jv, dmu, &slip)) {
        if (!sr || !capillary_jac(P, xij, r[i], r[j], sr[i], sr[j], &Jx, dmu)) continue;
        slip = 2;
      }
      ++m;
      ms += slip;
      uint64_t k = (uint64_t)i * 0x9E3779B97F4A7C15ull ^ ((uint64_t)j + 0x632BE59BD9B4E019ull) * 0xBF58476D1CE4E5B9ull;
      k ^= (uint64_t)slip * 0x94D049BB133111EBull;
      h += k * 0xD6E8FEB86659FD93ull;
    }
  free(sr);
  sig[0] += (uint64_t)m;
  sig[1] += (uint64_t)ms;
  sig[2] = sig[2] * 31u + h;
}

/* K substeps forward (storing every state) and the reverse pass.
 *   gxK, gvK: dL/dx_K, dL/dv_K (3n each, v may be NULL)
 *   out: g_x0, g_v0 (3n), g_c = dL/dc_drag, g_mu = dL/dmu.
 *   sig (3 uint64, may be NULL): contact signature summed over the window
 *   (O(N^2) per substep: small problems only).
 * x, v are left at the final state. */
void or_run_adjoint(const or_grid* G, const or_params* P, int64_t n, int K, double* x, double* v, const double* r,
                    const double* u, const double* vf, const double* wf, const double* p, const double* af,
                    const double* gxK, const double* gvK, double* g_x0, double* g_v0, double* g_c, double* g_mu,
                    uint64_t* sig, int brute, uint32_t* status) {
  size_t n3 = 3 * (size_t)(n > 0 ? n : 1);
  double* xs = (double*)malloc(sizeof(double) * n3 * (size_t)(K + 1));
  double* vs = (double*)malloc(sizeof(double) * n3 * (size_t)(K + 1));
  double* Fc = (double*)malloc(sizeof(double) * n3);
  double* Ffl = (double*)malloc(sizeof(double) * n3);
  double* a_f = (double*)malloc(sizeof(double) * n3);
  double* fex = (double*)malloc(sizeof(double) * n3);
  double* afp = (double*)malloc(sizeof(double) * (n3 / 3));
  memcpy(xs, x, sizeof(double) * 3 * n);
  memcpy(vs, v, sizeof(double) * 3 * n);
  if (sig) sig[0] = sig[1] = sig[2] = 0;
  for (int s = 0; s < K; ++s) {
    double* xc = xs + n3 * s;
    double* vc = vs + n3 * s;
    if (sig) contact_signature(G, P, n, xc, vc, r, af, sig);
    or_g2p(G, P, n, xc, vc, r, u, vf, wf, p, af, Ffl, a_f, afp);
    or_contact(G, P, n, xc, vc, r, af, brute, Fc, status);
    or_integrate(G, P, n, xc, vc, r, Fc, Ffl, a_f, xs + n3 * (s + 1), vs + n3 * (s + 1), fex, status);
  }
  memcpy(x, xs + n3 * K, sizeof(double) * 3 * n);
  memcpy(v, vs + n3 * K, sizeof(double) * 3 * n);
  double* gX = (double*)malloc(sizeof(double) * n3);
  double* gV = (double*)malloc(sizeof(double) * n3);
  double* gXp = (double*)malloc(sizeof(double) * n3);
  double* gVp = (double*)malloc(sizeof(double) * n3);
  double* gFc = (double*)malloc(sizeof(double) * n3);
  double* gFfl = (double*)malloc(sizeof(double) * n3);
  double* gaf = (double*)malloc(sizeof(double) * n3);
  for (size_t k = 0; k < 3 * (size_t)n; ++k) {
    gXp[k] = gxK ? gxK[k] : 0.0;
    gVp[k] = gvK ? gvK[k] : 0.0;
  }
  *g_c = 0.0;
  *g_mu = 0.0;
  for (int s = K - 1; s >= 0; --s) {
    double* xc = xs + n3 * s;
    double* vc = vs + n3 * s;
    or_integrate_adj(G, P, n, r, gXp, gVp, NULL, gX, gV, gFc, gFfl, gaf);
    or_g2p_adj(G, P, n, xc, vc, r, u, vf, wf, p, af, gFfl, gaf, NULL, gX, gV, g_c);
    or_contact_adj(G, P, n, xc, vc, r, af, gFc, brute, gX, gV, g_mu);
    memcpy(gXp, gX, sizeof(double) * 3 * n);
    memcpy(gVp, gV, sizeof(double) * 3 * n);
  }
  memcpy(g_x0, gXp, sizeof(double) * 3 * n);
  memcpy(g_v0, gVp, sizeof(double) * 3 * n);
  free(xs); free(vs); free(Fc); free(Ffl); free(a_f); free(fex); free(afp);
  free(gX); free(gV); free(gXp); free(gVp); free(gFc); free(gFfl); free(gaf);
}
