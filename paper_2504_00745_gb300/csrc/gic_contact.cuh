// gic_contact.cuh -- device side of a2 (contact): the pair law (Sec. 3.1,
// Eq. k_n, polydisperse form, with the library's readings), contact
// geometry in both precisions, the 27-cell walks and the Verlet-list walk.
// Shared by the contact kernels and the fused substep.
#pragma once

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
  // gq <= 2^30; 32-bit conversions where the values fit (the 64-bit ones run on the FP64 pipe)
  if (Ph >= 2147483648.0f)
    ov = (float)((long long)Ph - gq) + Pl;
  else if (Ph >= 16777216.0f)
    ov = (float)((int)Ph - (int)gq) + Pl;  // Ph is an integer here
  else
    ov = (Ph - (float)(int)gq) + Pl;
  if (!(ov > 0.0f)) return false;
  gap = (float)(int)gq * G.unit_f;
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
// candidates within kPosfTol of contact.  f(j, ox, oy, oz, geometry).
template <typename F>
__device__ __forceinline__ void for_each_contact_f(const DGrid& G, const uint4* __restrict__ table, uint32_t epoch,
                                                   int64_t i, int cx, int cy, int cz, const float4& fi,
                                                   const uint4& pi, float ri, const float4* __restrict__ posf,
                                                   const uint4* __restrict__ pos, F&& f) {
  const float rci = fmaf(ri, G.inv_hc_f, kPosfTol);
  for_each_cell(G, table, epoch, cx, cy, cz, [&](uint32_t start, uint32_t cnt, int ox, int oy, int oz) {
    for (uint32_t j = start; j < start + cnt; ++j) {
      if ((int64_t)j == i) continue;
      float4 fj = __ldg(&posf[j]);
      float rx = fj.x - fi.x, ry = fj.y - fi.y, rz = fj.z - fi.z;
      float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
      float Rc = fmaf(fj.w, G.inv_hc_f, rci);
      if (!(d2 < Rc * Rc)) continue;
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

// ----------------------------------------------------------------- Verlet lists
//
// A build gives every granule a slot (its sorted index then); row s of
// `list` holds the slots of the granules that were within r_i + r_j + skin of
// slot s.  While every granule has moved less than skin / 2 since then, every
// pair now in contact is in the rows, so walking them gives exactly
// gic_contact's pairs.  Between builds the sorted order changes little, so
// rows, reference positions and partners are read almost in order.  When the
// state is still in the order of the build (gic_step keeps it so between
// builds) slots are indices, and the walk skips the slot maps (ident).
//
// Flag words: kNbRebuild -- this call rebuilds (set by the displacement
// check before the call, or by gic_step's decision); kNbSticky -- bit 0 a
// rebuild was requested, bit 1 a row overflowed at the last build (rebuild
// every call); kNbCounter -- CTAs done; kNbOverflow -- overflow during this
// build; kNbBuilds -- builds so far; kNbNext -- a granule written by a
// k_substep is beyond skin / 2 of its reference (gic_step's next call
// rebuilds; gic_step consumes the word).

enum : int {
  kNbRebuild = 0,
  kNbSticky = 1,
  kNbCounter = 2,
  kNbOverflow = 3,
  kNbBuilds = 4,
  kNbNext = 5,
  kNbWords = 8
};

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
  int ident;      // the state is in the order of the last build: slot = index
  float lim2_f;   // (skin / 2)^2 in (2^-30 h_c)^2, FP32 positions
  double lim2_d;  // (skin / 2)^2 in m^2, FP64 positions
  int64_t n;      // granules (debug builds check partner indices against it)
  uint32_t* dbg;  // debug builds: the status word the index checks flag
};

__device__ __forceinline__ float nb_lim2(const NbDev& nb, float) { return nb.lim2_f; }
__device__ __forceinline__ double nb_lim2(const NbDev& nb, double) { return nb.lim2_d; }

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
  if (has_f) {  // float positions in contact-cell units
    rj = fj.w;
    float rx = fj.x - fi.x, ry = fj.y - fi.y, rz = fj.z - fi.z;
    d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
    Rc = fmaf(ri + rj, G.inv_hc_f, kPosfTol);
    Rs = fmaf(ri + rj + skin, G.inv_hc_f, kPosfTol);
    near = d2 < Rs * Rs;
    touch = d2 < Rc * Rc;
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

// FP32 wall forces out of line: granule i's force with the walls of the set
// bits of `ends` (bit 2a + side: the granule's cell is that end cell of axis
// a) added in the order of add_walls, so the sums are the same bits.  Only
// the few granules in an end cell make the call; the grid and contact
// constants come as scalars.
struct WallSum {
  float F0, F1, F2;
  bool ok;
};
static __device__ __noinline__ WallSum walls_f32(float s_hi, float s_lo, float unit_f, float k_n, float zeta,
                                                 float kt_over_cn, float mu, uint4 pi, float ri, float mi, float4 vi,
                                                 unsigned ends, float F0, float F1, float F2) {
  DGrid G{};  // only the constants the wall law reads are set
  G.s_hi = s_hi;
  G.s_lo = s_lo;
  G.unit_f = unit_f;
  DParams<float> P{};
  P.k_n = k_n;
  P.zeta = zeta;
  P.kt_over_cn = kt_over_cn;
  P.mu = mu;
  WallSum R{F0, F1, F2, true};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      if (!(ends >> (2 * a + side) & 1u)) continue;
      float gap, ov;
      if (!wall_geom(G, pi, a, side, ri, gap, ov)) continue;
      float x[3] = {0.f, 0.f, 0.f};
      x[a] = side == 0 ? gap : -gap;
      float f0, f1, f2;
      if (pair_force(P, x[0], x[1], x[2], gap, ov, vi.x, vi.y, vi.z, mi, f0, f1, f2)) {
        R.F0 += f0;
        R.F1 += f1;
        R.F2 += f2;
      } else {
        R.ok = false;
      }
    }
  }
  return R;
}

__device__ __forceinline__ void add_walls_f32(const DGrid& G, const DParams<float>& P, const uint4& pi, float ri,
                                              float mi, const float4& vi, int cx, int cy, int cz, float& F0, float& F1,
                                              float& F2, uint32_t* status) {
  const unsigned ends = (unsigned)(cx == 0) | (unsigned)(cx == G.nc[0] - 1) << 1 | (unsigned)(cy == 0) << 2 |
                        (unsigned)(cy == G.nc[1] - 1) << 3 | (unsigned)(cz == 0) << 4 |
                        (unsigned)(cz == G.nc[2] - 1) << 5;
  if (!ends) return;
  const WallSum R = walls_f32(G.s_hi, G.s_lo, G.unit_f, P.k_n, P.zeta, P.kt_over_cn, P.mu, pi, ri, mi, vi, ends, F0,
                              F1, F2);
  F0 = R.F0;
  F1 = R.F1;
  F2 = R.F2;
  if (!R.ok) raise_status(status, GIC_STATUS_OUT_OF_DOMAIN);
}

// The walls' part of the contact adjoint of granule i (upstream l = its own
// force gradient): adds to gx, gv and returns the mu part.  A wall vector
// depends on x_i only through its axis-a component.
template <typename T>
__device__ __forceinline__ T add_walls_adj(const DGrid& G, const DParams<T>& P, const pos_t<T>& pi, T ri, T mi,
                                           const vec_t<T>& vi, int cx, int cy, int cz, T l0, T l1, T l2, T& gx0,
                                           T& gx1, T& gx2, T& gv0, T& gv1, T& gv2) {
  const int c3[3] = {cx, cy, cz};
  T gm = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      if (side == 0 ? c3[a] != 0 : c3[a] != G.nc[a] - 1) continue;
      T gap, ov;
      if (!wall_geom(G, pi, a, side, ri, gap, ov)) continue;
      T x[3] = {0, 0, 0};
      x[a] = side == 0 ? gap : -gap;
      T w[3] = {0, 0, 0};
      gm += pair_force_adj(P, x[0], x[1], x[2], gap, ov, vi.x, vi.y, vi.z, mi, l0, l1, l2, l0, l1, l2, w[0], w[1],
                           w[2], gv0, gv1, gv2);
      if (a == 0) gx0 += w[0];
      else if (a == 1) gx1 += w[1];
      else gx2 += w[2];
    }
  }
  return gm;
}

// Host side of a Verlet call up to the list walk: argument checks, the
// displacement check and (launch_build) the build launch, after which F_c
// holds the build's forces when it ran.  Fills the device view of the lists.
int verlet_prelude(const DGrid& G, const GicParams* params, const GicGranules* s, const void* table,
                   const GicNeighbors* nb, void* F_c, cudaStream_t stream, const char* what, NbDev* out,
                   bool launch_build);
// The device view of the lists (ident: the state is in the build's order);
// verlet_view also checks the arguments, and launches nothing.
NbDev nb_dev(const DGrid& G, const GicNeighbors* nb, bool ident);
int verlet_view(const DGrid& G, const GicGranules* s, const void* table, const GicNeighbors* nb, const char* what,
                bool ident, NbDev* out);
// The displacement check alone (maps the state's ids to slots, sets the
// rebuild word); with copy_to, it also copies the state into copy_to in the
// same order and writes the identity into perm.
int verlet_check(const DGrid& G, const GicGranules* s, const void* table, const GicNeighbors* nb,
                 cudaStream_t stream, const char* what, NbDev* out, GicGranules* copy_to, int32_t* perm);

// The staged list build of gic_step's rebuilding substep (FP32 path with
// float copies): rows and reference entries of the sorted state, no forces;
// records the build unless a row overflowed (see gic_contact.cu).
int launch_build_tile(const DGrid& G, const GicGranules* sorted, const void* table, const NbDev& d, double skin,
                      cudaStream_t stream);

// The list build of granule i: walks the 27 cells with the pre-test radius
// r_i + r_j + skin, writes row i (slot = sorted index) and its reference
// entries, and hands every partner in contact to f(j, g).
template <typename T, typename F>
__device__ __forceinline__ void verlet_build_row(const DGrid& G, const NbDev& nb, const uint4* __restrict__ table,
                                                 int64_t n, int64_t i, int cx, int cy, int cz, int32_t ci,
                                                 const pos_t<T>& pi, T ri, bool has_f, const float4& fi, T skin,
                                                 const int32_t* __restrict__ id, const pos_t<T>* __restrict__ pos,
                                                 const float4* __restrict__ posf, F&& f) {
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
    if (touch) f(j, g);
  });
  nb.count[i] = cnt;
  nb.at[i] = (int32_t)i;  // after a build, slot = sorted index
  nb.cur[i] = (int32_t)i;
  nb.ref_cell[i] = ci;
  reinterpret_cast<pos_t<T>*>(nb.ref_pos)[i] = pi;
  const int32_t idi = id[i];
  if (idi >= 0 && (int64_t)idi < n) nb.slot[idi] = (int32_t)i;
  if (over) atomicOr(&nb.flags[kNbOverflow], 1u);
}

// The list build of granule i and its contact forces, walls excluded.
template <typename T>
__device__ __forceinline__ void verlet_build_granule(const DGrid& G, const DParams<T>& P, const NbDev& nb,
                                                     const uint4* __restrict__ table, int64_t n, int64_t i,
                                                     int cx, int cy, int cz, int32_t ci, const pos_t<T>& pi, T ri,
                                                     T mi, const vec_t<T>& vi, bool has_f, const float4& fi, T skin,
                                                     const int32_t* __restrict__ id, const pos_t<T>* __restrict__ pos,
                                                     const float4* __restrict__ posf,
                                                     const vec_t<T>* __restrict__ vel, T& F0, T& F1, T& F2,
                                                     bool& coincident) {
  verlet_build_row<T>(G, nb, table, n, i, cx, cy, cz, ci, pi, ri, has_f, fi, skin, id, pos, posf,
                      [&](int64_t j, const PairGeom<T>& g) {
                        add_force(P, g, vi, ldg(&vel[j]), mi, granule_mass(P, radius_of(ldg(&pos[j]))), F0, F1, F2,
                                  coincident);
                      });
}

// Called by every thread of the last launch of a Verlet call: the last CTA
// to finish clears the per-call words (after a build: records an overflow
// as the sticky bit and counts the build).
__device__ __forceinline__ void verlet_call_done(const NbDev& nb, bool rebuild) {
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

// Every partner j of granule i in its Verlet row (slot at[i]) that is in
// contact, with the geometry: f(j, g).  Four partners at a time, so that
// their index, cell and float-position loads overlap.
template <typename T, typename F>
__device__ __forceinline__ void for_each_list_contact(const DGrid& G, const NbDev& nb, int64_t i, int cx, int cy,
                                                      int cz, int32_t ci, const pos_t<T>& pi, T ri, bool has_f,
                                                      const float4& fi, const int32_t* __restrict__ cell,
                                                      const pos_t<T>* __restrict__ pos,
                                                      const float4* __restrict__ posf, F&& f) {
  const int32_t s = nb.ident ? (int32_t)i : nb.at[i];
  const int32_t* row = nb.list + (int64_t)s * nb.cap;
  int cnt = nb.count[s];
  if (!GIC_DBG_OK(nb.dbg, cnt >= 0 && cnt <= nb.cap)) cnt = 0;
  for (int k = 0; k < cnt; k += 4) {
    int64_t jj[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      jj[u] = k + u < cnt ? (int64_t)(nb.ident ? row[k + u] : nb.cur[row[k + u]]) : -1;
      if (jj[u] >= 0 && !GIC_DBG_OK(nb.dbg, jj[u] < nb.n)) jj[u] = -1;
    }
    if (has_f) {  // FP32: the float pre-test needs no partner cell; load it for the pairs that pass
      float4 fj[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) fj[u] = jj[u] >= 0 ? __ldg(&posf[jj[u]]) : fi;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (jj[u] < 0) continue;
        const float rx = fj[u].x - fi.x, ry = fj[u].y - fi.y, rz = fj[u].z - fi.z;
        const float Rc = fmaf((float)ri + fj[u].w, G.inv_hc_f, kPosfTol);
        if (!(fmaf(rx, rx, fmaf(ry, ry, rz * rz)) < Rc * Rc)) continue;
        const int32_t cj = __ldg(&cell[jj[u]]);
        const int ox = cell_x(cj) - cx, oy = cell_y(cj) - cy, oz = cell_z(cj) - cz;
        if (ox < -1 || ox > 1 || oy < -1 || oy > 1 || oz < -1 || oz > 1) continue;
        bool near, touch;
        PairGeom<T> g;
        verlet_pair(G, pi, ri, true, fi, fj[u], pos, jj[u], ox, oy, oz, T(0), near, touch, g);
        if (touch) f(jj[u], g);
      }
      continue;
    }
    int32_t cj[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) cj[u] = jj[u] >= 0 ? __ldg(&cell[jj[u]]) : ci;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (jj[u] < 0) continue;
      const int ox = cell_x(cj[u]) - cx, oy = cell_y(cj[u]) - cy, oz = cell_z(cj[u]) - cz;
      // partners two or more cells apart are farther than h_c >= 2 r_max
      if (ox < -1 || ox > 1 || oy < -1 || oy > 1 || oz < -1 || oz > 1) continue;
      bool near, touch;
      PairGeom<T> g;
      verlet_pair(G, pi, ri, false, fi, fi, pos, jj[u], ox, oy, oz, T(0), near, touch, g);
      if (touch) f(jj[u], g);
    }
  }
}

// Forces of the partners in granule i's Verlet row (the list walk of
// gic_contact_verlet).
template <typename T>
__device__ __forceinline__ void verlet_list_force(const DGrid& G, const DParams<T>& P, const NbDev& nb, int64_t i,
                                                  int cx, int cy, int cz, int32_t ci, const pos_t<T>& pi, T ri, T mi,
                                                  const vec_t<T>& vi, bool has_f, const float4& fi,
                                                  const int32_t* __restrict__ cell, const pos_t<T>* __restrict__ pos,
                                                  const float4* __restrict__ posf, const vec_t<T>* __restrict__ vel,
                                                  T& F0, T& F1, T& F2, bool& coincident) {
  for_each_list_contact<T>(G, nb, i, cx, cy, cz, ci, pi, ri, has_f, fi, cell, pos, posf,
                           [&](int64_t j, const PairGeom<T>& g) {
                             add_force(P, g, vi, ldg(&vel[j]), mi, granule_mass(P, radius_of(ldg(&pos[j]))), F0, F1,
                                       F2, coincident);
                           });
}

}  // namespace gic
