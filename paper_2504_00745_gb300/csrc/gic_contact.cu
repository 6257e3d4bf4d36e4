// gic_contact.cu -- a2: DEM contact forces and their adjoint.
//
// Gather form: one thread per granule of the sorted state walks the 27
// contact cells around its own (h_c >= 2 r_max), reads each partner's
// position / velocity and sums the pair forces on itself.  No atomics.  The
// adjoint uses the antisymmetry F_ji = -F_ij, so it is a gather as well:
// dL/dx_i = sum_j (dF_ij/dx_ij)^T (lambda_i - lambda_j).
//
// Contact law (Sec. 3.1, Eq. k_n), polydisperse and with the readings of this
// library: n = x_ij / d, overlap = r_i + r_j - d,
//   F_n = (k_n overlap - c_n v_n) n,   c_n = 2 zeta sqrt(k_n m_eff),
//   f_t = -k_t v_t,  k_t = kt_over_cn c_n,   F_t = min(|f_t|, mu |F_n|) f_t/|f_t|.
// Walls are partners of infinite mass at rest (m_eff = m_i).
#include "gic_internal.cuh"

namespace gic {

template <typename T>
__device__ __forceinline__ T granule_mass(const DParams<T>& P, T r) {
  return P.rho_s * (T(4.0 / 3.0 * kPi) * r * r * r);
}

// Pair force on i (x = x_i - x_j, v = v_i - v_j) at distance d with
// overlap = r_i + r_j - d > 0.  Returns false for coincident centres.
template <typename T>
__device__ __forceinline__ bool pair_force(const DParams<T>& P, T x0, T x1, T x2, T d, T overlap, T v0, T v1, T v2,
                                           T meff, T& F0, T& F1, T& F2) {
  if (d == T(0)) return false;
  T inv_d = T(1) / d;
  T n0 = x0 * inv_d, n1 = x1 * inv_d, n2 = x2 * inv_d;
  T cn = T(2) * P.zeta * sqrt(P.k_n * meff);
  T vn = v0 * n0 + v1 * n1 + v2 * n2;
  T Fn = P.k_n * overlap - cn * vn;
  T t0 = v0 - vn * n0, t1 = v1 - vn * n1, t2 = v2 - vn * n2;
  T kt = P.kt_over_cn * cn;
  T ftn = kt * sqrt(t0 * t0 + t1 * t1 + t2 * t2);
  T cap = P.mu * fabs(Fn);
  T s = ftn > cap ? cap / ftn : T(1);
  T a = s * kt;
  F0 = Fn * n0 - a * t0;
  F1 = Fn * n1 - a * t1;
  F2 = Fn * n2 - a * t2;
  return true;
}

// Reverse mode of pair_force for upstream l (gradient of the pair force):
// adds d<l, F>/dx to gx and d<l, F>/dv to gv; returns d<lm, F>/dmu for the
// second upstream lm (the granule's own gradient).
template <typename T>
__device__ __forceinline__ T pair_force_adj(const DParams<T>& P, T x0, T x1, T x2, T d, T overlap, T v0, T v1, T v2,
                                            T meff, T l0, T l1, T l2, T lm0, T lm1, T lm2, T& gx0, T& gx1, T& gx2,
                                            T& gv0, T& gv1, T& gv2) {
  if (d == T(0)) return T(0);
  T inv_d = T(1) / d;
  T n0 = x0 * inv_d, n1 = x1 * inv_d, n2 = x2 * inv_d;
  T cn = T(2) * P.zeta * sqrt(P.k_n * meff);
  T vn = v0 * n0 + v1 * n1 + v2 * n2;
  T Fn = P.k_n * overlap - cn * vn;
  T t0 = v0 - vn * n0, t1 = v1 - vn * n1, t2 = v2 - vn * n2;
  T kt = P.kt_over_cn * cn;
  T vtn = sqrt(t0 * t0 + t1 * t1 + t2 * t2);
  T ftn = kt * vtn;
  T cap = P.mu * fabs(Fn);
  bool slip = ftn > cap;
  // F = Fn n + F_t
  T gFn = l0 * n0 + l1 * n1 + l2 * n2;
  T gn0 = Fn * l0, gn1 = Fn * l1, gn2 = Fn * l2;
  T gt0, gt1, gt2;
  T gmu = T(0);
  if (slip) {
    // F_t = -A u, A = mu |Fn|, u = v_t / |v_t|
    T inv_vt = T(1) / vtn;
    T u0 = t0 * inv_vt, u1 = t1 * inv_vt, u2 = t2 * inv_vt;
    T A = cap;
    T gA = -(l0 * u0 + l1 * u1 + l2 * u2);
    T sgn = Fn > T(0) ? T(1) : (Fn < T(0) ? T(-1) : T(0));
    gFn += gA * P.mu * sgn;
    gmu = -(lm0 * u0 + lm1 * u1 + lm2 * u2) * fabs(Fn);
    T gu0 = -A * l0, gu1 = -A * l1, gu2 = -A * l2;
    T gudu = gu0 * u0 + gu1 * u1 + gu2 * u2;
    gt0 = (gu0 - gudu * u0) * inv_vt;
    gt1 = (gu1 - gudu * u1) * inv_vt;
    gt2 = (gu2 - gudu * u2) * inv_vt;
  } else {
    gt0 = -kt * l0;
    gt1 = -kt * l1;
    gt2 = -kt * l2;
  }
  // v_t = v - vn n
  gv0 += gt0;
  gv1 += gt1;
  gv2 += gt2;
  T gvn = -(gt0 * n0 + gt1 * n1 + gt2 * n2);
  gn0 -= vn * gt0;
  gn1 -= vn * gt1;
  gn2 -= vn * gt2;
  // Fn = k_n (R - d) - cn vn
  T gd = -P.k_n * gFn;
  gvn -= cn * gFn;
  // vn = v . n
  gv0 += gvn * n0;
  gv1 += gvn * n1;
  gv2 += gvn * n2;
  gn0 += gvn * v0;
  gn1 += gvn * v1;
  gn2 += gvn * v2;
  // n = x / d, d = |x|
  T gnn = gn0 * n0 + gn1 * n1 + gn2 * n2;
  gx0 += (gn0 - gnn * n0) * inv_d + gd * n0;
  gx1 += (gn1 - gnn * n1) * inv_d + gd * n1;
  gx2 += (gn2 - gnn * n2) * inv_d + gd * n2;
  return gmu;
}

// Contact geometry of a candidate pair: x_ij (metres), distance d and overlap
// r_i + r_j - d.  Returns false if the pair does not overlap.
template <typename T>
struct PairGeom {
  T x0, x1, x2, d, overlap;
};

// FP32 path.  The separation is an exact integer vector D in 2^-30 h_c units.
// A float pre-test with a small margin rejects most candidates; survivors get
// the overlap to ~1e-7 of itself (not of d): R = (r_i + r_j) 2^30 / h_c as a
// float pair (TwoSum / TwoProd), |D|^2 exact in 64-bit integers, d = sqrt with
// one exact-residual correction, and R - d taken hi-to-hi (exact) plus the
// low parts.  Plain FP32 would lose the overlap to cancellation (d ~ 100x
// overlap in dense packings).
// Exact part for a candidate that passed a pre-test (D = integer separation).
__device__ __forceinline__ bool pair_geom_exact(const DGrid& G, int Dx, int Dy, int Dz, float ri, float rj,
                                                PairGeom<float>& g) {
  // R (2^-30 h_c units) as hi + lo
  float Rh = ri + rj;
  float bb = Rh - ri;
  float Rl = (ri - (Rh - bb)) + (rj - bb);  // TwoSum error
  float Ph = Rh * G.s_hi;
  float Pl = fmaf(Rh, G.s_hi, -Ph) + fmaf(Rh, G.s_lo, Rl * G.s_hi);
  // exact |D|^2 and a corrected square root
  unsigned long long d2 = (unsigned long long)((long long)Dx * Dx) + (unsigned long long)((long long)Dy * Dy) +
                          (unsigned long long)((long long)Dz * Dz);
  float dh = sqrtf(__ull2float_rn(d2));
  float ov;
  if (dh >= 8388608.0f) {  // dh is an integer: the residual d2 - dh^2 is exact
    unsigned long long di = (unsigned long long)dh;
    long long res = (long long)(d2 - di * di);
    float c = (float)res / (2.0f * dh);
    ov = (Ph - dh) + (Pl - c);
    dh += c;
  } else {  // deep overlap (d < h_c / 128): relative precision is ample
    ov = (Ph - dh) + Pl;
  }
  if (!(ov > 0.0f)) return false;
  g.x0 = (float)Dx * G.unit_f;
  g.x1 = (float)Dy * G.unit_f;
  g.x2 = (float)Dz * G.unit_f;
  g.d = dh * G.unit_f;
  g.overlap = ov * G.unit_f;
  return true;
}

__device__ __forceinline__ void int_sep(const uint4& pi, const uint4& pj, int ox, int oy, int oz, int& Dx, int& Dy,
                                        int& Dz) {
  Dx = (int)pi.x - (int)pj.x - ox * (int)kFracOne;
  Dy = (int)pi.y - (int)pj.y - oy * (int)kFracOne;
  Dz = (int)pi.z - (int)pj.z - oz * (int)kFracOne;
}

__device__ __forceinline__ bool pair_geom(const DGrid& G, const uint4& pi, const uint4& pj, int ox, int oy, int oz,
                                          float ri, float rj, PairGeom<float>& g) {
  int Dx, Dy, Dz;
  int_sep(pi, pj, ox, oy, oz, Dx, Dy, Dz);
  float fx = (float)Dx, fy = (float)Dy, fz = (float)Dz;
  float d2f = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
  float Rs = ri + rj;
  if (!(d2f < Rs * Rs * G.s2_margin)) return false;
  return pair_geom_exact(G, Dx, Dy, Dz, ri, rj, g);
}

__device__ __forceinline__ bool pair_geom(const DGrid& G, const d4& pi, const d4& pj, int ox, int oy, int oz,
                                          double ri, double rj, PairGeom<double>& g) {
  double x0, x1, x2;
  rel_ij(G, pi, pj, ox, oy, oz, x0, x1, x2);
  double d2 = x0 * x0 + x1 * x1 + x2 * x2;
  double R = ri + rj;
  if (!(d2 < R * R)) return false;
  g.x0 = x0;
  g.x1 = x1;
  g.x2 = x2;
  g.d = sqrt(d2);
  g.overlap = R - g.d;
  return true;
}

// Wall geometry: the granule's gap to the lower (side 0) or upper wall of
// axis a when it sits in the first / last contact cell.  FP32: the gap is the
// exact integer q (or 2^30 - q) and the overlap r 2^30/h_c - gap is formed
// from the float pair of r 2^30 / h_c.
__device__ __forceinline__ bool wall_geom(const DGrid& G, const uint4& p, int a, int side, float r, float& gap,
                                          float& overlap) {
  uint32_t q = pcomp(p, a);
  long long gq = side == 0 ? (long long)q : (long long)kFracOne - (long long)q;
  float Ph = r * G.s_hi;
  float Pl = fmaf(r, G.s_hi, -Ph) + r * G.s_lo;
  float ov;
  if (Ph >= 16777216.0f)
    ov = (float)((long long)Ph - gq) + Pl;  // Ph is an integer here
  else
    ov = (Ph - (float)gq) + Pl;
  if (!(ov > 0.0f)) return false;
  gap = (float)gq * G.unit_f;
  overlap = ov * G.unit_f;
  return true;
}
__device__ __forceinline__ bool wall_geom(const DGrid& G, const d4& p, int a, int side, double r, double& gap,
                                          double& overlap) {
  gap = side == 0 ? gap_lo(G, p, a) : gap_hi(G, p, a);
  if (!(gap < r)) return false;
  overlap = r - gap;
  return true;
}

template <typename T>
__device__ __forceinline__ void load_cell_coords(int32_t c, int& x, int& y, int& z) {
  x = cell_x(c);
  y = cell_y(c);
  z = cell_z(c);
}

// Visit every granule j != i in the 27 contact cells around (cx, cy, cz).
template <typename F>
__device__ __forceinline__ void for_each_partner(const DGrid& G, const uint4* __restrict__ table, uint32_t epoch,
                                                 int64_t i, int cx, int cy, int cz, F&& f) {
  for (int oz = -1; oz <= 1; ++oz) {
    int z = cz + oz;
    if (z < 0 || z >= G.nc[2]) continue;
    for (int oy = -1; oy <= 1; ++oy) {
      int y = cy + oy;
      if (y < 0 || y >= G.nc[1]) continue;
      for (int ox = -1; ox <= 1; ++ox) {
        int x = cx + ox;
        if (x < 0 || x >= G.nc[0]) continue;
        uint4 e = __ldg(&table[table_index(G, x, y, z)]);
        if (e.z != epoch) continue;
        for (uint32_t j = e.x; j < e.x + e.y; ++j) {
          if ((int64_t)j == i) continue;
          f((int64_t)j, ox, oy, oz);
        }
      }
    }
  }
}

// Visit every occupied contact cell of the 27 around (cx, cy, cz):
// f(start, count, ox, oy, oz).
template <typename F>
__device__ __forceinline__ void for_each_cell(const DGrid& G, const uint4* __restrict__ table, uint32_t epoch, int cx,
                                              int cy, int cz, F&& f) {
  for (int oz = -1; oz <= 1; ++oz) {
    int z = cz + oz;
    if (z < 0 || z >= G.nc[2]) continue;
    for (int oy = -1; oy <= 1; ++oy) {
      int y = cy + oy;
      if (y < 0 || y >= G.nc[1]) continue;
      for (int ox = -1; ox <= 1; ++ox) {
        int x = cx + ox;
        if (x < 0 || x >= G.nc[0]) continue;
        uint4 e = __ldg(&table[table_index(G, x, y, z)]);
        if (e.z != epoch) continue;
        f(e.x, e.y, ox, oy, oz);
      }
    }
  }
}

// FP32 candidate loop on the float copy of the positions: per candidate only
// float adds / FMAs and one compare; the exact integer geometry runs for
// candidates within 1e-5 of contact.  f(j, ox, oy, oz, geometry).
template <typename F>
__device__ __forceinline__ void for_each_contact_f(const DGrid& G, const uint4* __restrict__ table, uint32_t epoch,
                                                   int64_t i, int cx, int cy, int cz, const float4& fi,
                                                   const uint4& pi, float ri, const float4* __restrict__ posf,
                                                   const uint4* __restrict__ pos, F&& f) {
  const float rci = ri * G.inv_hc_f;
  const float m2 = 1.0f + 1e-5f;
  for_each_cell(G, table, epoch, cx, cy, cz, [&](uint32_t start, uint32_t cnt, int ox, int oy, int oz) {
    float ax = (float)ox - fi.x, ay = (float)oy - fi.y, az = (float)oz - fi.z;
    for (uint32_t j = start; j < start + cnt; ++j) {
      if ((int64_t)j == i) continue;
      float4 fj = __ldg(&posf[j]);
      float rx = ax + fj.x, ry = ay + fj.y, rz = az + fj.z;
      float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
      float Rc = fmaf(fj.w, G.inv_hc_f, rci);
      if (!(d2 < Rc * Rc * m2)) continue;
      uint4 pj = __ldg(&pos[j]);
      int Dx, Dy, Dz;
      int_sep(pi, pj, ox, oy, oz, Dx, Dy, Dz);
      PairGeom<float> g;
      if (!pair_geom_exact(G, Dx, Dy, Dz, ri, fj.w, g)) continue;
      f((int64_t)j, g);
    }
  });
}

// Every partner j of granule i in contact (overlap > 0), with its geometry:
// f(j, g).  FP32 with a float position copy uses the float pre-test loop.
template <typename T, typename F>
__device__ __forceinline__ void for_each_contact(const DGrid& G, const uint4* __restrict__ table, uint32_t epoch,
                                                 int64_t i, int cx, int cy, int cz, const pos_t<T>& pi, T ri,
                                                 const pos_t<T>* __restrict__ pos, const float4* __restrict__ posf,
                                                 F&& f) {
  if constexpr (sizeof(T) == 4) {
    if (posf) {
      for_each_contact_f(G, table, epoch, i, cx, cy, cz, __ldg(&posf[i]), pi, ri, posf, pos, f);
      return;
    }
  }
  for_each_partner(G, table, epoch, i, cx, cy, cz, [&](int64_t j, int ox, int oy, int oz) {
    pos_t<T> pj = ldg(&pos[j]);
    PairGeom<T> g;
    if (pair_geom(G, pi, pj, ox, oy, oz, ri, radius_of(pj), g)) f(j, g);
  });
}

template <typename T>
__global__ void __launch_bounds__(128) k_contact(DGrid G, DParams<T> P, int64_t n, const int32_t* __restrict__ cell,
                                                  const pos_t<T>* __restrict__ pos, const float4* __restrict__ posf,
                                                  const vec_t<T>* __restrict__ vel, const uint4* __restrict__ table,
                                                  vec_t<T>* __restrict__ F, uint32_t* status) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t ci = cell[i];
  int cx, cy, cz;
  load_cell_coords<T>(ci, cx, cy, cz);
  pos_t<T> pi = pos[i];
  vec_t<T> vi = vel[i];
  T ri = radius_of(pi);
  T mi = granule_mass(P, ri);
  uint32_t epoch = __ldg(&table[0].x);
  if (T(2) * ri > (T)G.hc) raise_status(status, GIC_STATUS_RADIUS);
  T F0 = 0, F1 = 0, F2 = 0;
  bool coincident = false;
  for_each_contact<T>(G, table, epoch, i, cx, cy, cz, pi, ri, pos, posf, [&](int64_t j, const PairGeom<T>& g) {
    vec_t<T> vj = ldg(&vel[j]);
    T mj = granule_mass(P, radius_of(ldg(&pos[j])));
    T f0, f1, f2;
    if (pair_force(P, g.x0, g.x1, g.x2, g.d, g.overlap, vi.x - vj.x, vi.y - vj.y, vi.z - vj.z, mi * mj / (mi + mj), f0,
                   f1, f2)) {
      F0 += f0;
      F1 += f1;
      F2 += f2;
    } else {
      coincident = true;
    }
  });
  if (P.walls) {
    const int c3[3] = {cx, cy, cz};
    for (int a = 0; a < 3; ++a) {
      for (int side = 0; side < 2; ++side) {
        if (side == 0 ? c3[a] != 0 : c3[a] != G.nc[a] - 1) continue;
        T gap, ov;
        if (!wall_geom(G, pi, a, side, ri, gap, ov)) continue;
        T x[3] = {0, 0, 0};
        x[a] = side == 0 ? gap : -gap;
        T f0, f1, f2;
        if (pair_force(P, x[0], x[1], x[2], gap, ov, vi.x, vi.y, vi.z, mi, f0, f1, f2)) {
          F0 += f0;
          F1 += f1;
          F2 += f2;
        } else {
          raise_status(status, GIC_STATUS_OUT_OF_DOMAIN);
        }
      }
    }
  }
  if (coincident) raise_status(status, GIC_STATUS_COINCIDENT);
  if (!isfinite(F0) || !isfinite(F1) || !isfinite(F2)) raise_status(status, GIC_STATUS_NONFINITE);
  F[i] = make_vec<T>(F0, F1, F2);
}

// ----------------------------------------------------------------- staged FP32 contact
//
// One CTA = 128 consecutive granules of the Morton-sorted state: a compact
// blob of contact cells.  The CTA stages the cell-table entries of the
// blob's bounding box (+1 cell halo) and the float positions of every
// granule in those cells in shared memory, then each thread walks its 27
// neighbour cells there.  A CTA whose box or granule count exceeds the
// shared-memory budget (a Morton range that jumps across the domain) takes
// the global-memory path instead; the results are identical.

constexpr int kTileThreads = 128;
constexpr int kTileMaxCells = 512;
constexpr int kTileMaxGranules = 1152;

__device__ __forceinline__ void add_pair_force(const DParams<float>& P, const PairGeom<float>& g, const float4& vi,
                                               const float4& vj, float mi, float mj, float& F0, float& F1, float& F2,
                                               bool& coincident) {
  float f0, f1, f2;
  if (pair_force(P, g.x0, g.x1, g.x2, g.d, g.overlap, vi.x - vj.x, vi.y - vj.y, vi.z - vj.z, mi * mj / (mi + mj), f0,
                 f1, f2)) {
    F0 += f0;
    F1 += f1;
    F2 += f2;
  } else {
    coincident = true;
  }
}

__global__ void __launch_bounds__(kTileThreads) k_contact_tile(DGrid G, DParams<float> P, int64_t n,
                                                               const int32_t* __restrict__ cell,
                                                               const uint4* __restrict__ pos,
                                                               const float4* __restrict__ posf,
                                                               const float4* __restrict__ vel,
                                                               const uint4* __restrict__ table,
                                                               float4* __restrict__ F, uint32_t* status) {
  __shared__ int s_lo[3], s_hi[3];
  __shared__ uint32_t s_start[kTileMaxCells];
  __shared__ uint32_t s_cnt[kTileMaxCells];
  __shared__ uint32_t s_off[kTileMaxCells + 1];
  __shared__ float4 s_pf[kTileMaxGranules];
  __shared__ uint32_t s_wsum[kTileThreads / 32];
  __shared__ int s_mode;  // 0: staged, 1: global fallback

  const int64_t i = blockIdx.x * (int64_t)kTileThreads + threadIdx.x;
  const bool valid = i < n;
  const uint32_t epoch = __ldg(&table[0].x);
  int cx = 0, cy = 0, cz = 0;
  if (threadIdx.x < 3) {
    s_lo[threadIdx.x] = 1 << 30;
    s_hi[threadIdx.x] = -1;
  }
  __syncthreads();
  if (valid) {
    int32_t ci = cell[i];
    cx = cell_x(ci);
    cy = cell_y(ci);
    cz = cell_z(ci);
    atomicMin(&s_lo[0], cx);
    atomicMin(&s_lo[1], cy);
    atomicMin(&s_lo[2], cz);
    atomicMax(&s_hi[0], cx);
    atomicMax(&s_hi[1], cy);
    atomicMax(&s_hi[2], cz);
  }
  __syncthreads();
  // bounding box with a one-cell halo, clipped to the grid
  const int bx0 = max(s_lo[0] - 1, 0), by0 = max(s_lo[1] - 1, 0), bz0 = max(s_lo[2] - 1, 0);
  const int bx = min(s_hi[0] + 1, G.nc[0] - 1) - bx0 + 1;
  const int by = min(s_hi[1] + 1, G.nc[1] - 1) - by0 + 1;
  const int bz = min(s_hi[2] + 1, G.nc[2] - 1) - bz0 + 1;
  const int ncell = bx * by * bz;
  if (threadIdx.x == 0) s_mode = (ncell > kTileMaxCells || s_hi[0] < 0) ? 1 : 0;
  __syncthreads();
  if (s_mode == 0) {
    // stage the table entries of the box
    // box index -> coordinates with float reciprocals (exact for these small integers)
    const float ibx = 1.0f / (float)bx, ibxy = 1.0f / (float)(bx * by);
    for (int b = threadIdx.x; b < ncell; b += kTileThreads) {
      int z = (int)(((float)b + 0.5f) * ibxy);
      int rem = b - z * bx * by;
      int y = (int)(((float)rem + 0.5f) * ibx);
      int x = bx0 + rem - y * bx;
      y += by0;
      z += bz0;
      uint4 e = __ldg(&table[table_index(G, x, y, z)]);
      bool ok = e.z == epoch;
      s_start[b] = ok ? e.x : 0u;
      s_cnt[b] = ok ? e.y : 0u;
    }
    __syncthreads();
    // exclusive scan of the counts (ncell <= 512: 4 per thread)
    {
      const int per = (kTileMaxCells + kTileThreads - 1) / kTileThreads;
      uint32_t loc[per];
      uint32_t sum = 0;
#pragma unroll
      for (int k = 0; k < per; ++k) {
        int b = threadIdx.x * per + k;
        loc[k] = b < ncell ? s_cnt[b] : 0u;
        sum += loc[k];
      }
      uint32_t incl = sum;
      for (int off = 1; off < 32; off <<= 1) {
        uint32_t o = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane_id() >= off) incl += o;
      }
      if (lane_id() == 31) s_wsum[threadIdx.x >> 5] = incl;
      __syncthreads();
      uint32_t base = 0;
      for (int w = 0; w < (threadIdx.x >> 5); ++w) base += s_wsum[w];
      uint32_t run = base + incl - sum;
#pragma unroll
      for (int k = 0; k < per; ++k) {
        int b = threadIdx.x * per + k;
        if (b < kTileMaxCells) s_off[b] = run;
        run += loc[k];
      }
      if (threadIdx.x == kTileThreads - 1) s_off[kTileMaxCells] = run;
    }
    __syncthreads();
    const uint32_t total = s_off[kTileMaxCells];
    if (total > (uint32_t)kTileMaxGranules) {
      if (threadIdx.x == 0) s_mode = 1;
    } else {
      // stage the float positions: slot t belongs to cell b with s_off[b] <= t < s_off[b + 1]
      for (uint32_t t = threadIdx.x; t < total; t += kTileThreads) {
        int lo = 0, hi = ncell - 1;  // last b with s_off[b] <= t
        while (lo < hi) {
          int mid = (lo + hi + 1) >> 1;
          if (s_off[mid] <= t) lo = mid;
          else hi = mid - 1;
        }
        // position in units of contact cells relative to the box corner: the three
        // cells of an x-row are consecutive slots, and no cell offset is needed
        float4 p = __ldg(&posf[s_start[lo] + (t - s_off[lo])]);
        int lz = (int)(((float)lo + 0.5f) * ibxy);
        int rem = lo - lz * bx * by;
        int ly = (int)(((float)rem + 0.5f) * ibx);
        int lx = rem - ly * bx;
        s_pf[t] = make_float4((float)lx + p.x, (float)ly + p.y, (float)lz + p.z, p.w);
      }
    }
    __syncthreads();
  }
  if (!valid) return;
  const uint4 pi = pos[i];
  const float4 vi = vel[i];
  const float ri = __uint_as_float(pi.w);
  const float mi = granule_mass(P, ri);
  if (2.0f * ri > G.hc_f) raise_status(status, GIC_STATUS_RADIUS);
  float F0 = 0.f, F1 = 0.f, F2 = 0.f;
  bool coincident = false;
  if (s_mode == 0) {
    const int lx = cx - bx0, ly = cy - by0, lz = cz - bz0;
    const float4 fi0 = __ldg(&posf[i]);
    const float xi = (float)lx + fi0.x, yi = (float)ly + fi0.y, zi = (float)lz + fi0.z;
    const float rci = ri * G.inv_hc_f;
    // box coordinates reach 2^6 cells: their float rounding (< 1e-5 cell) stays inside this margin
    const float m2 = 1.0f + 1e-4f;
    const int xa = max(lx - 1, 0), xb = min(lx + 1, bx - 1);
    // own slot (excluded): own cell's first slot + rank inside the cell
    const int bown = lx + bx * (ly + by * lz);
    const uint32_t tself = s_off[bown] + (uint32_t)(i - (int64_t)s_start[bown]);
    for (int oz = -1; oz <= 1; ++oz) {
      int z = lz + oz;
      if (z < 0 || z >= bz) continue;
      for (int oy = -1; oy <= 1; ++oy) {
        int y = ly + oy;
        if (y < 0 || y >= by) continue;
        int row = bx * (y + by * z);
        uint32_t t0 = s_off[row + xa], t1 = s_off[row + xb + 1];
        for (uint32_t t = t0; t < t1; ++t) {
          float4 fj = s_pf[t];
          float rx = fj.x - xi, ry = fj.y - yi, rz = fj.z - zi;
          float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
          float Rc = fmaf(fj.w, G.inv_hc_f, rci);
          if (!(d2 < Rc * Rc * m2) || t == tself) continue;
          // contact candidate: locate j and its cell offset, then the exact geometry
          int bj = row + xa;
          while (s_off[bj + 1] <= t) ++bj;
          uint32_t j = s_start[bj] + (t - s_off[bj]);
          int ox = (bj - row) - lx;
          uint4 pj = __ldg(&pos[j]);
          int Dx, Dy, Dz;
          int_sep(pi, pj, ox, oy, oz, Dx, Dy, Dz);
          PairGeom<float> g;
          if (!pair_geom_exact(G, Dx, Dy, Dz, ri, fj.w, g)) continue;
          add_pair_force(P, g, vi, __ldg(&vel[j]), mi, granule_mass(P, fj.w), F0, F1, F2, coincident);
        }
      }
    }
  } else {
    for_each_contact<float>(G, table, epoch, i, cx, cy, cz, pi, ri, pos, posf, [&](int64_t j, const PairGeom<float>& g) {
      add_pair_force(P, g, vi, __ldg(&vel[j]), mi, granule_mass(P, radius_of(__ldg(&pos[j]))), F0, F1, F2, coincident);
    });
  }
  if (P.walls) {
    const int c3[3] = {cx, cy, cz};
    for (int a = 0; a < 3; ++a) {
      for (int side = 0; side < 2; ++side) {
        if (side == 0 ? c3[a] != 0 : c3[a] != G.nc[a] - 1) continue;
        float gap, ov;
        if (!wall_geom(G, pi, a, side, ri, gap, ov)) continue;
        float x[3] = {0, 0, 0};
        x[a] = side == 0 ? gap : -gap;
        float f0, f1, f2;
        if (pair_force(P, x[0], x[1], x[2], gap, ov, vi.x, vi.y, vi.z, mi, f0, f1, f2)) {
          F0 += f0;
          F1 += f1;
          F2 += f2;
        } else {
          raise_status(status, GIC_STATUS_OUT_OF_DOMAIN);
        }
      }
    }
  }
  if (coincident) raise_status(status, GIC_STATUS_COINCIDENT);
  if (!isfinite(F0) || !isfinite(F1) || !isfinite(F2)) raise_status(status, GIC_STATUS_NONFINITE);
  F[i] = make_float4(F0, F1, F2, 0.f);
}

template <typename T>
__global__ void __launch_bounds__(128) k_contact_adj(DGrid G, DParams<T> P, int64_t n, const int32_t* __restrict__ cell,
                                                      const pos_t<T>* __restrict__ pos,
                                                      const float4* __restrict__ posf,
                                                      const vec_t<T>* __restrict__ vel, const uint4* __restrict__ table,
                                                      const vec_t<T>* __restrict__ gF, vec_t<T>* __restrict__ gpos,
                                                      vec_t<T>* __restrict__ gvel, double* __restrict__ g_mu) {
  __shared__ double s_red[32];
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double my_gmu = 0.0;
  if (i < n) {
    int32_t ci = cell[i];
    int cx, cy, cz;
    load_cell_coords<T>(ci, cx, cy, cz);
    pos_t<T> pi = pos[i];
    vec_t<T> vi = vel[i];
    vec_t<T> li = gF[i];
    T ri = radius_of(pi);
    T mi = granule_mass(P, ri);
    uint32_t epoch = __ldg(&table[0].x);
    T gx0 = 0, gx1 = 0, gx2 = 0, gv0 = 0, gv1 = 0, gv2 = 0, gm = 0;
    for_each_contact<T>(G, table, epoch, i, cx, cy, cz, pi, ri, pos, posf, [&](int64_t j, const PairGeom<T>& g) {
      vec_t<T> vj = ldg(&vel[j]);
      vec_t<T> lj = ldg(&gF[j]);
      T mj = granule_mass(P, radius_of(ldg(&pos[j])));
      gm += pair_force_adj(P, g.x0, g.x1, g.x2, g.d, g.overlap, vi.x - vj.x, vi.y - vj.y, vi.z - vj.z,
                           mi * mj / (mi + mj), li.x - lj.x, li.y - lj.y, li.z - lj.z, li.x, li.y, li.z, gx0, gx1, gx2,
                           gv0, gv1, gv2);
    });
    if (P.walls) {
      const int c3[3] = {cx, cy, cz};
      for (int a = 0; a < 3; ++a) {
        for (int side = 0; side < 2; ++side) {
          if (side == 0 ? c3[a] != 0 : c3[a] != G.nc[a] - 1) continue;
          T gap, ov;
          if (!wall_geom(G, pi, a, side, ri, gap, ov)) continue;
          T x[3] = {0, 0, 0};
          x[a] = side == 0 ? gap : -gap;
          // the wall vector depends on x_i only through its axis-a component
          T w[3] = {0, 0, 0};
          gm += pair_force_adj(P, x[0], x[1], x[2], gap, ov, vi.x, vi.y, vi.z, mi, li.x, li.y, li.z, li.x, li.y, li.z,
                               w[0], w[1], w[2], gv0, gv1, gv2);
          if (a == 0) gx0 += w[0];
          else if (a == 1) gx1 += w[1];
          else gx2 += w[2];
        }
      }
    }
    vec_t<T> a = gpos[i];
    vec_t<T> b = gvel[i];
    gpos[i] = make_vec<T>(a.x + gx0, a.y + gx1, a.z + gx2);
    gvel[i] = make_vec<T>(b.x + gv0, b.y + gv1, b.z + gv2);
    my_gmu = (double)gm;
  }
  if (g_mu) {
    double s = block_sum(my_gmu, s_red);
    if (threadIdx.x == 0) atomicAdd(g_mu, s);
  }
}

// Diagnostic: number of partners per granule and the pair list by id.
template <typename T>
__global__ void k_contact_pairs(DGrid G, int64_t n, const int32_t* __restrict__ cell, const pos_t<T>* __restrict__ pos,
                                const float4* __restrict__ posf, const int32_t* __restrict__ id, const uint4* __restrict__ table,
                                int32_t* __restrict__ counts, int32_t* __restrict__ pairs, int64_t max_pairs,
                                unsigned long long* __restrict__ n_pairs) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int cx, cy, cz;
  load_cell_coords<T>(cell[i], cx, cy, cz);
  pos_t<T> pi = pos[i];
  T ri = radius_of(pi);
  int32_t idi = id ? id[i] : (int32_t)i;
  uint32_t epoch = __ldg(&table[0].x);
  int cnt = 0;
  for_each_contact<T>(G, table, epoch, i, cx, cy, cz, pi, ri, pos, posf, [&](int64_t j, const PairGeom<T>&) {
    ++cnt;
    int32_t idj = id ? id[j] : (int32_t)j;
    if (pairs && idi < idj) {
      unsigned long long slot = atomicAdd(n_pairs, 1ull);
      if ((int64_t)slot < max_pairs) {
        pairs[2 * slot] = idi;
        pairs[2 * slot + 1] = idj;
      }
    }
  });
  if (counts) counts[i] = cnt;
}

// ----------------------------------------------------------------- Verlet lists
//
// A build gives every granule a slot (its sorted index then); row s of
// `list` holds the slots of the granules that were within r_i + r_j + skin of
// slot s.  While every granule has moved less than skin / 2 since then, every
// pair now in contact is in the rows, so walking them gives exactly
// gic_contact's pairs.  Between builds the sorted order changes little, so
// rows, reference positions and partners are read almost in order.

enum : int { kNbRebuild = 0, kNbSticky = 1, kNbCounter = 2, kNbOverflow = 3, kNbBuilds = 4, kNbWords = 8 };

struct NbDev {
  int cap;
  int32_t* list;
  int32_t* count;
  int32_t* ref_cell;
  void* ref_pos;
  int32_t* slot;  // by id
  int32_t* cur;   // by slot
  int32_t* at;    // by sorted index
  uint32_t* flags;
};

// displacement since the last build beyond skin / 2 (lim2 = (skin / 2)^2 in
// the units of each precision's position record)
__device__ __forceinline__ bool moved_far(const DGrid&, int32_t c, const uint4& p, int32_t cr, const uint4& pr,
                                          float lim2) {
  // 32-bit pieces: the offset difference is exact, the cell part a multiple of 2^30
  float dx = fmaf((float)(cell_x(c) - cell_x(cr)), 0x1p30f, (float)((int)p.x - (int)pr.x));
  float dy = fmaf((float)(cell_y(c) - cell_y(cr)), 0x1p30f, (float)((int)p.y - (int)pr.y));
  float dz = fmaf((float)(cell_z(c) - cell_z(cr)), 0x1p30f, (float)((int)p.z - (int)pr.z));
  return fmaf(dx, dx, fmaf(dy, dy, dz * dz)) > lim2;
}
__device__ __forceinline__ bool moved_far(const DGrid& G, int32_t c, const d4& p, int32_t cr, const d4& pr,
                                          double lim2) {
  double dx = (double)(cell_x(c) - cell_x(cr)) * G.hc + (p.x - pr.x);
  double dy = (double)(cell_y(c) - cell_y(cr)) * G.hc + (p.y - pr.y);
  double dz = (double)(cell_z(c) - cell_z(cr)) * G.hc + (p.z - pr.z);
  return dx * dx + dy * dy + dz * dz > lim2;
}

template <typename T>
__global__ void __launch_bounds__(256) k_verlet_check(DGrid G, int64_t n, const int32_t* __restrict__ cell,
                                                       const pos_t<T>* __restrict__ pos,
                                                       const int32_t* __restrict__ id, NbDev nb, T lim2) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  bool far = false;
  if (i < n && !nb.flags[kNbSticky]) {  // after a reset the slots are not set yet
    int32_t k = id[i];
    int32_t s = (k >= 0 && (int64_t)k < n) ? nb.slot[k] : -1;
    if (s >= 0 && (int64_t)s < n) {
      nb.cur[s] = (int32_t)i;
      nb.at[i] = s;
      far = moved_far(G, cell[i], pos[i], nb.ref_cell[s], reinterpret_cast<const pos_t<T>*>(nb.ref_pos)[s], lim2);
    } else {
      far = true;  // ids outside 0..n-1: rebuild (the build path does not need them)
    }
  }
  if (__any_sync(0xffffffffu, far) && lane_id() == 0) atomicOr(&nb.flags[kNbRebuild], 1u);
}

template <typename T>
__device__ __forceinline__ void add_force(const DParams<T>& P, const PairGeom<T>& g, const vec_t<T>& vi,
                                          const vec_t<T>& vj, T mi, T mj, T& F0, T& F1, T& F2, bool& coincident) {
  T f0, f1, f2;
  if (pair_force(P, g.x0, g.x1, g.x2, g.d, g.overlap, vi.x - vj.x, vi.y - vj.y, vi.z - vj.z, mi * mj / (mi + mj), f0,
                 f1, f2)) {
    F0 += f0;
    F1 += f1;
    F2 += f2;
  } else {
    coincident = true;
  }
}

// FP32 candidate j (cell offset o from i): whether it is within R + skin
// (list test, a superset with a float margin), and its contact geometry.
__device__ __forceinline__ void verlet_pair(const DGrid& G, const uint4& pi, float ri, bool has_f, const float4& fi,
                                            const float4& fj, const uint4* __restrict__ pos, int64_t j, int ox,
                                            int oy, int oz, float skin, bool& near, bool& touch,
                                            PairGeom<float>& g) {
  uint4 pj;
  float rj;
  float d2, Rs, Rc;
  if (has_f) {  // float positions in contact cells
    rj = fj.w;
    float rx = (float)ox + fj.x - fi.x, ry = (float)oy + fj.y - fi.y, rz = (float)oz + fj.z - fi.z;
    d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
    Rc = (ri + rj) * G.inv_hc_f;
    Rs = (ri + rj + skin) * G.inv_hc_f;
    near = d2 < Rs * Rs * (1.0f + 1e-4f);
    touch = d2 < Rc * Rc * (1.0f + 1e-4f);
    if (!touch) return;
    pj = __ldg(&pos[j]);
  } else {  // the exact integer separation, float pre-test
    pj = __ldg(&pos[j]);
    rj = radius_of(pj);
    int Dx, Dy, Dz;
    int_sep(pi, pj, ox, oy, oz, Dx, Dy, Dz);
    float fx = (float)Dx, fy = (float)Dy, fz = (float)Dz;
    d2 = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
    Rc = ri + rj;
    Rs = ri + rj + skin;
    near = d2 < Rs * Rs * G.s2_margin;
    touch = d2 < Rc * Rc * G.s2_margin;
    if (!touch) return;
  }
  int Dx, Dy, Dz;
  int_sep(pi, pj, ox, oy, oz, Dx, Dy, Dz);
  touch = pair_geom_exact(G, Dx, Dy, Dz, ri, rj, g);
}

__device__ __forceinline__ void verlet_pair(const DGrid& G, const d4& pi, double ri, bool, const float4&,
                                            const float4&, const d4* __restrict__ pos, int64_t j, int ox, int oy, int oz,
                                            double skin, bool& near, bool& touch, PairGeom<double>& g) {
  d4 pj = ldg(&pos[j]);
  double x0, x1, x2;
  rel_ij(G, pi, pj, ox, oy, oz, x0, x1, x2);
  double d2 = x0 * x0 + x1 * x1 + x2 * x2;
  double R = ri + pj.w;
  near = d2 < (R + skin) * (R + skin);
  touch = d2 < R * R;
  if (!touch) return;
  g.x0 = x0;
  g.x1 = x1;
  g.x2 = x2;
  g.d = sqrt(d2);
  g.overlap = R - g.d;
}

// Wall forces of granule i (cell coordinates c3) added to F.
template <typename T>
__device__ __forceinline__ void add_walls(const DGrid& G, const DParams<T>& P, const pos_t<T>& pi, T ri, T mi,
                                          const vec_t<T>& vi, int cx, int cy, int cz, T& F0, T& F1, T& F2,
                                          uint32_t* status) {
  const int c3[3] = {cx, cy, cz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      if (side == 0 ? c3[a] != 0 : c3[a] != G.nc[a] - 1) continue;
      T gap, ov;
      if (!wall_geom(G, pi, a, side, ri, gap, ov)) continue;
      T x[3] = {0, 0, 0};
      x[a] = side == 0 ? gap : -gap;
      T f0, f1, f2;
      if (pair_force(P, x[0], x[1], x[2], gap, ov, vi.x, vi.y, vi.z, mi, f0, f1, f2)) {
        F0 += f0;
        F1 += f1;
        F2 += f2;
      } else {
        raise_status(status, GIC_STATUS_OUT_OF_DOMAIN);
      }
    }
  }
}

// kBuild = true: runs only when this call rebuilds -- walks the 27 cells,
// writes every row (slot = sorted index) and the forces.  kBuild = false:
// runs only when it does not -- walks the rows; its last CTA then clears the
// per-call words.  The two are launched back to back; the idle one exits.
template <typename T, bool kBuild>
__global__ void __launch_bounds__(kBuild ? 128 : 256, kBuild ? 1 : 4) k_contact_verlet(
    DGrid G, DParams<T> P, int64_t n, const int32_t* __restrict__ cell, const pos_t<T>* __restrict__ pos,
    const float4* __restrict__ posf, const vec_t<T>* __restrict__ vel, const int32_t* __restrict__ id,
    const uint4* __restrict__ table, NbDev nb, T skin, vec_t<T>* __restrict__ F, uint32_t* status) {
  const bool rebuild = (nb.flags[kNbRebuild] | nb.flags[kNbSticky]) != 0u;  // uniform over the launch
  if (kBuild && !rebuild) return;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (kBuild == rebuild && i < n) {
    const int32_t ci = cell[i];
    const int cx = cell_x(ci), cy = cell_y(ci), cz = cell_z(ci);
    const pos_t<T> pi = pos[i];
    const vec_t<T> vi = vel[i];
    const T ri = radius_of(pi);
    const T mi = granule_mass(P, ri);
    if (T(2) * ri > (T)G.hc) raise_status(status, GIC_STATUS_RADIUS);
    const bool has_f = sizeof(T) == 4 && posf != nullptr;
    const float4 fi = has_f ? __ldg(&posf[i]) : make_float4(0.f, 0.f, 0.f, 0.f);
    T F0 = 0, F1 = 0, F2 = 0;
    bool coincident = false;
    if constexpr (kBuild) {
      int32_t* row = nb.list + i * nb.cap;
      const uint32_t epoch = __ldg(&table[0].x);
      int cnt = 0;
      bool over = false;
      for_each_partner(G, table, epoch, i, cx, cy, cz, [&](int64_t j, int ox, int oy, int oz) {
        const float4 fj = has_f ? __ldg(&posf[j]) : fi;
        bool near, touch;
        PairGeom<T> g;
        verlet_pair(G, pi, ri, has_f, fi, fj, pos, j, ox, oy, oz, skin, near, touch, g);
        if (near) {
          if (cnt < nb.cap)
            row[cnt++] = (int32_t)j;
          else
            over = true;
        }
        if (touch) add_force(P, g, vi, ldg(&vel[j]), mi, granule_mass(P, radius_of(ldg(&pos[j]))), F0, F1, F2,
                             coincident);
      });
      nb.count[i] = cnt;
      nb.ref_cell[i] = ci;
      reinterpret_cast<pos_t<T>*>(nb.ref_pos)[i] = pi;
      const int32_t idi = id[i];
      if (idi >= 0 && (int64_t)idi < n) nb.slot[idi] = (int32_t)i;
      if (over) atomicOr(&nb.flags[kNbOverflow], 1u);
    } else {
      const int32_t s = nb.at[i];
      const int32_t* row = nb.list + (int64_t)s * nb.cap;
      const int cnt = nb.count[s];
      // four partners at a time: their index, cell and float-position loads overlap
      for (int k = 0; k < cnt; k += 4) {
        int64_t jj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) jj[u] = k + u < cnt ? (int64_t)nb.cur[row[k + u]] : -1;
        int32_t cj[4];
        float4 fj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          cj[u] = jj[u] >= 0 ? __ldg(&cell[jj[u]]) : ci;
          fj[u] = (has_f && jj[u] >= 0) ? __ldg(&posf[jj[u]]) : fi;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (jj[u] < 0) continue;
          const int ox = cell_x(cj[u]) - cx, oy = cell_y(cj[u]) - cy, oz = cell_z(cj[u]) - cz;
          // partners two or more cells apart are farther than h_c >= 2 r_max
          if (ox < -1 || ox > 1 || oy < -1 || oy > 1 || oz < -1 || oz > 1) continue;
          bool near, touch;
          PairGeom<T> g;
          verlet_pair(G, pi, ri, has_f, fi, fj[u], pos, jj[u], ox, oy, oz, T(0), near, touch, g);
          if (touch)
            add_force(P, g, vi, ldg(&vel[jj[u]]), mi, granule_mass(P, radius_of(ldg(&pos[jj[u]]))), F0, F1, F2,
                      coincident);
        }
      }
    }
    if (P.walls) add_walls(G, P, pi, ri, mi, vi, cx, cy, cz, F0, F1, F2, status);
    if (coincident) raise_status(status, GIC_STATUS_COINCIDENT);
    if (!isfinite(F0) || !isfinite(F1) || !isfinite(F2)) raise_status(status, GIC_STATUS_NONFINITE);
    F[i] = make_vec<T>(F0, F1, F2);
  }
  if constexpr (!kBuild) {
    // the last CTA to finish clears the per-call words for the next call
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      if (atomicAdd(&nb.flags[kNbCounter], 1u) == gridDim.x - 1) {
        __threadfence();
        if (rebuild) {
          nb.flags[kNbSticky] = atomicExch(&nb.flags[kNbOverflow], 0u) ? 2u : 0u;
          nb.flags[kNbBuilds] += 1u;
        }
        nb.flags[kNbRebuild] = 0u;
        nb.flags[kNbCounter] = 0u;
        __threadfence();
      }
    }
  }
}

__global__ void k_neighbors_reset(uint32_t* flags) {
  if (threadIdx.x < kNbWords) flags[threadIdx.x] = threadIdx.x == kNbSticky ? 1u : 0u;
}

static int check_table(const void* t) {
  if (!t) return set_error(GIC_ERR_INVALID, "cell_table is NULL");
  if ((uintptr_t)t % 16) return set_error(GIC_ERR_ALIGN, "cell_table must be 16-byte aligned");
  return GIC_OK;
}

}  // namespace gic

using namespace gic;

extern "C" int gic_contact(const GicGrid* grid, const GicParams* params, const GicGranules* s, const void* table,
                           void* F_c, gic_stream_t stream) {
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if ((rc = check_granules(s, "gic_contact"))) return rc;
  if ((rc = check_table(table))) return rc;
  if (s->n == 0) return GIC_OK;
  if (!F_c) return set_error(GIC_ERR_INVALID, "gic_contact: F_c is NULL");
  if ((rc = check_vecs(s->precision, "gic_contact", {F_c}))) return rc;
  const int threads = 128;
  if (s->precision == GIC_FP32) {
    DParams<float> P;
    if ((rc = make_params(params, &P))) return rc;
    if (s->posf)
      k_contact_tile<<<grid_blocks(s->n, kTileThreads), kTileThreads, 0, stream>>>(
          G, P, s->n, s->cell, (const uint4*)s->pos, (const float4*)s->posf, (const float4*)s->vel,
          (const uint4*)table, (float4*)F_c, status_word());
    else
      k_contact<float><<<grid_blocks(s->n, threads), threads, 0, stream>>>(
          G, P, s->n, s->cell, (const uint4*)s->pos, nullptr, (const float4*)s->vel, (const uint4*)table,
          (float4*)F_c, status_word());
  } else {
    DParams<double> P;
    if ((rc = make_params(params, &P))) return rc;
    k_contact<double><<<grid_blocks(s->n, threads), threads, 0, stream>>>(
        G, P, s->n, s->cell, (const d4*)s->pos, nullptr, (const d4*)s->vel, (const uint4*)table, (d4*)F_c,
        status_word());
  }
  count_launches(1);
  GIC_CHECK_LAUNCH("gic_contact");
  return GIC_OK;
}

extern "C" int gic_contact_adj(const GicGrid* grid, const GicParams* params, const GicGranules* s, const void* table,
                               const void* gF_c, void* g_pos, void* g_vel, double* g_mu, gic_stream_t stream) {
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if ((rc = check_granules(s, "gic_contact_adj"))) return rc;
  if ((rc = check_table(table))) return rc;
  if (s->n == 0) return GIC_OK;
  if (!gF_c || !g_pos || !g_vel) return set_error(GIC_ERR_INVALID, "gic_contact_adj: null gradient array");
  if ((rc = check_vecs(s->precision, "gic_contact_adj", {gF_c, g_pos, g_vel}))) return rc;
  const int threads = 128;
  if (s->precision == GIC_FP32) {
    DParams<float> P;
    if ((rc = make_params(params, &P))) return rc;
    k_contact_adj<float><<<grid_blocks(s->n, threads), threads, 0, stream>>>(
        G, P, s->n, s->cell, (const uint4*)s->pos, (const float4*)s->posf, (const float4*)s->vel, (const uint4*)table,
        (const float4*)gF_c, (float4*)g_pos, (float4*)g_vel, g_mu);
  } else {
    DParams<double> P;
    if ((rc = make_params(params, &P))) return rc;
    k_contact_adj<double><<<grid_blocks(s->n, threads), threads, 0, stream>>>(
        G, P, s->n, s->cell, (const d4*)s->pos, nullptr, (const d4*)s->vel, (const uint4*)table, (const d4*)gF_c,
        (d4*)g_pos, (d4*)g_vel, g_mu);
  }
  count_launches(1);
  GIC_CHECK_LAUNCH("gic_contact_adj");
  return GIC_OK;
}

extern "C" int gic_contact_pairs(const GicGrid* grid, const GicGranules* s, const void* table, int32_t* counts,
                                 int32_t* pairs, int64_t max_pairs, int64_t* n_pairs, gic_stream_t stream) {
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if ((rc = check_granules(s, "gic_contact_pairs"))) return rc;
  if ((rc = check_table(table))) return rc;
  if (s->n == 0) return GIC_OK;
  if (pairs && !n_pairs) return set_error(GIC_ERR_INVALID, "gic_contact_pairs: n_pairs is NULL");
  if (s->precision == GIC_FP32)
    k_contact_pairs<float><<<grid_blocks(s->n, 128), 128, 0, stream>>>(G, s->n, s->cell, (const uint4*)s->pos,
                                                                        (const float4*)s->posf, s->id,
                                                                        (const uint4*)table, counts, pairs, max_pairs,
                                                                        (unsigned long long*)n_pairs);
  else
    k_contact_pairs<double><<<grid_blocks(s->n, 128), 128, 0, stream>>>(G, s->n, s->cell, (const d4*)s->pos, nullptr,
                                                                         s->id,
                                                                         (const uint4*)table, counts, pairs,
                                                                         max_pairs, (unsigned long long*)n_pairs);
  count_launches(1);
  GIC_CHECK_LAUNCH("gic_contact_pairs");
  return GIC_OK;
}

static int check_neighbors(const GicNeighbors* nb, const GicGranules* s, const char* what) {
  if (!nb) return set_error(GIC_ERR_INVALID, "%s: neighbours struct is NULL", what);
  if (!nb->list || !nb->count || !nb->ref_cell || !nb->ref_pos || !nb->slot || !nb->cur || !nb->at || !nb->flags)
    return set_error(GIC_ERR_INVALID, "%s: a neighbour array is NULL", what);
  if (nb->cap < 1) return set_error(GIC_ERR_INVALID, "%s: cap must be >= 1", what);
  if (!(nb->skin >= 0.0)) return set_error(GIC_ERR_INVALID, "%s: skin must be >= 0", what);
  if (s && nb->n != s->n) return set_error(GIC_ERR_INVALID, "%s: neighbour lists are for %lld granules, got %lld",
                                           what, (long long)nb->n, (long long)s->n);
  if (s && (uintptr_t)nb->ref_pos % (s->precision == GIC_FP32 ? 16 : 32))
    return set_error(GIC_ERR_ALIGN, "%s: ref_pos misaligned", what);
  return GIC_OK;
}

extern "C" int gic_contact_verlet(const GicGrid* grid, const GicParams* params, const GicGranules* s,
                                  const void* table, const GicNeighbors* nb, void* F_c, gic_stream_t stream) {
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if ((rc = check_granules(s, "gic_contact_verlet", true))) return rc;
  if ((rc = check_table(table))) return rc;
  if ((rc = check_neighbors(nb, s, "gic_contact_verlet"))) return rc;
  if (s->n == 0) return GIC_OK;
  if (!F_c) return set_error(GIC_ERR_INVALID, "gic_contact_verlet: F_c is NULL");
  if ((rc = check_vecs(s->precision, "gic_contact_verlet", {F_c}))) return rc;
  NbDev d{nb->cap, nb->list, nb->count, nb->ref_cell, nb->ref_pos, nb->slot, nb->cur, nb->at, nb->flags};
  const double half = 0.5 * nb->skin;
  if (s->precision == GIC_FP32) {
    DParams<float> P;
    if ((rc = make_params(params, &P))) return rc;
    const double lim = half * G.inv_unit;  // skin / 2 in 2^-30 h_c units
    k_verlet_check<float><<<grid_blocks(s->n, 256), 256, 0, stream>>>(G, s->n, s->cell, (const uint4*)s->pos, s->id, d,
                                                                      (float)(lim * lim));
    k_contact_verlet<float, true><<<grid_blocks(s->n, 128), 128, 0, stream>>>(
        G, P, s->n, s->cell, (const uint4*)s->pos, (const float4*)s->posf, (const float4*)s->vel, s->id,
        (const uint4*)table, d, (float)nb->skin, (float4*)F_c, status_word());
    k_contact_verlet<float, false><<<grid_blocks(s->n, 256), 256, 0, stream>>>(
        G, P, s->n, s->cell, (const uint4*)s->pos, (const float4*)s->posf, (const float4*)s->vel, s->id,
        (const uint4*)table, d, (float)nb->skin, (float4*)F_c, status_word());
  } else {
    DParams<double> P;
    if ((rc = make_params(params, &P))) return rc;
    k_verlet_check<double><<<grid_blocks(s->n, 256), 256, 0, stream>>>(G, s->n, s->cell, (const d4*)s->pos, s->id, d,
                                                                       half * half);
    k_contact_verlet<double, true><<<grid_blocks(s->n, 128), 128, 0, stream>>>(
        G, P, s->n, s->cell, (const d4*)s->pos, nullptr, (const d4*)s->vel, s->id, (const uint4*)table, d, nb->skin,
        (d4*)F_c, status_word());
    k_contact_verlet<double, false><<<grid_blocks(s->n, 256), 256, 0, stream>>>(
        G, P, s->n, s->cell, (const d4*)s->pos, nullptr, (const d4*)s->vel, s->id, (const uint4*)table, d, nb->skin,
        (d4*)F_c, status_word());
  }
  count_launches(3);
  GIC_CHECK_LAUNCH("gic_contact_verlet");
  return GIC_OK;
}

extern "C" int gic_neighbors_reset(const GicNeighbors* nb, gic_stream_t stream) {
  int rc = check_neighbors(nb, nullptr, "gic_neighbors_reset");
  if (rc) return rc;
  k_neighbors_reset<<<1, 32, 0, stream>>>(nb->flags);
  count_launches(1);
  GIC_CHECK_LAUNCH("gic_neighbors_reset");
  return GIC_OK;
}
