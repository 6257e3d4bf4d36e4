// gic_capillary.cuh -- the concentration-gradient force of Sec. 5.4 in its
// capillary (liquid-bridge) form, evaluated inside the fused substep's pair
// loop, and its adjoint.  Between granules i and j whose surfaces are
// 0 < s < d_r apart:
//   F_ij = -Gamma((sr_i + sr_j) / 2) F^st(s) (x_i - x_j) / |x_i - x_j|,
//   F^st(s) = 2 pi sigma R (1 - (1 + 2 V* / (pi R s^2))^(-1/2))   (cos theta = 1),
//   d_r = R (v^(1/3) + 0.1 v^(2/3)), v = V* / R^3,
//   sr_i = r + alpha_f,i / (1 - alpha_f,i)  (alpha_f interpolated at the granule),
// with the library's readings: R = 2 r_i r_j / (r_i + r_j) (the paper's r for
// equal spheres), V* = bridge_frac (V_i + V_j) / 2, and Gamma the quadratic
// Bezier curve through (0, 0), (2 peak - 1/2, 2), (1, 0) in the (sr, Gamma)
// plane (zero outside 0 < sr < 1).  Pairs in contact (s <= 0) feel the
// contact law only.
#pragma once

#include "gic_contact.cuh"
#include "gic_grid.cuh"

namespace gic {

// Gamma(sr) and, if slope != nullptr, dGamma/dsr: along the curve sr(t) =
// 2 c t (1 - t) + t^2, Gamma(t) = 4 t (1 - t), t the root in [0, 1] (the
// rationalised form has no cancellation, also for c = 1/2).
template <typename T>
__device__ __forceinline__ T cap_gamma(T sr, T c, T* slope) {
  if (!(sr > T(0)) || !(sr < T(1))) {
    if (slope) *slope = T(0);
    return T(0);
  }
  const T t = sr / (c + sqrt(c * c + (T(1) - T(2) * c) * sr));
  if (slope) *slope = T(4) * (T(1) - T(2) * t) / (T(2) * (T(1) - T(2) * c) * t + T(2) * c);
  return T(4) * t * (T(1) - t);
}

template <typename T>
struct Bridge {
  T R, Vs, dr;
};

template <typename T>
__device__ __forceinline__ Bridge<T> bridge_of(const DParams<T>& P, T ri, T rj) {
  Bridge<T> b;
  b.R = T(2) * ri * rj / (ri + rj);
  b.Vs = P.frac * T(2.0 * kPi / 3.0) * (ri * ri * ri + rj * rj * rj);
  const T v = b.Vs / (b.R * b.R * b.R);
  const T c = cbrt(v);
  b.dr = b.R * (c + T(0.1) * c * c);
  return b;
}

// F^st(s) of a bridge (> 0), as 2 pi sigma R y / (sqrt(1+y) (sqrt(1+y) + 1)),
// y = 2 V* / (pi R s^2) (the same value, without cancellation for small y);
// slope: dF^st/ds.
template <typename T>
__device__ __forceinline__ T bridge_force(const DParams<T>& P, const Bridge<T>& b, T s, T* slope) {
  const T bb = T(2) * b.Vs / (T(kPi) * b.R);
  const T y = bb / (s * s);
  const T q = T(1) + y;
  const T sq = sqrt(q);
  const T k = T(2.0 * kPi) * P.sigma * b.R;
  if (slope) *slope = -k * bb / (s * s * s) / (q * sq);
  return k * y / (sq * (sq + T(1)));
}

// sr of a granule (cell c, position p) from the cell-centred fluid fraction,
// interpolated as G2P does; with gsr != nullptr also d sr / d x (1 / (1 -
// alpha)^2 times the interpolation's gradient, zero along clamped axes).
// +inf where alpha_f >= 1.
template <typename T>
__device__ __forceinline__ T moisture_ratio_at(const DGrid& G, const DParams<T>& P, const T* __restrict__ af,
                                               int32_t c, const pos_t<T>& p, T* gsr) {
  int m[3];
  T t[3];
  granule_mac<T>(G, c, p, m, t);
  const Stencil3<T> S = make_stencil<T>(G, m, t, 3);
  FieldLoad<T> L;
  L.f = af;
  L.nsx = G.nx;
  L.nsy = G.ny;
  L.nsz = G.nz;
  L.dbg = G.dbg;
  T g[3];
  const T a = interp<T>(S, L, grid_inv_dx<T>(G), gsr ? g : nullptr);
  if (!(a < T(1))) {
    if (gsr) gsr[0] = gsr[1] = gsr[2] = T(0);
    return T(INFINITY);
  }
  if (gsr) {
    const T k = T(1) / ((T(1) - a) * (T(1) - a));
    gsr[0] = k * g[0];
    gsr[1] = k * g[1];
    gsr[2] = k * g[2];
  }
  return P.moist + a / (T(1) - a);
}

// Signed pair geometry: x_ij, d and overlap = r_i + r_j - d (< 0 for a gap).
// FP32: from the exact integer separation as in pair_geom_exact.  Coincident
// centres give d = 0 (the contact law then skips the pair and flags it).
__device__ __forceinline__ bool pair_geom_signed(const DGrid& G, int Dx, int Dy, int Dz, float ri, float rj,
                                                 PairGeom<float>& g) {
  float Rh = ri + rj;
  float bb = Rh - ri;
  float Rl = (ri - (Rh - bb)) + (rj - bb);
  float Ph = Rh * G.s_hi;
  float Pl = fmaf(Rh, G.s_hi, -Ph) + fmaf(Rh, G.s_lo, Rl * G.s_hi);
  unsigned long long d2 = (unsigned long long)((long long)Dx * Dx) + (unsigned long long)((long long)Dy * Dy) +
                          (unsigned long long)((long long)Dz * Dz);
  if (d2 == 0ull) {
    g.x0 = g.x1 = g.x2 = g.d = 0.f;
    g.overlap = (ri + rj);
    return true;
  }
  float dh = sqrtf(__ull2float_rn(d2));
  float ov;
  if (dh >= 8388608.0f) {
    unsigned long long di = (unsigned long long)dh;
    long long res = (long long)(d2 - di * di);
    float c = (float)res / (2.0f * dh);
    ov = (Ph - dh) + (Pl - c);
    dh += c;
  } else {
    ov = (Ph - dh) + Pl;
  }
  g.x0 = (float)Dx * G.unit_f;
  g.x1 = (float)Dy * G.unit_f;
  g.x2 = (float)Dz * G.unit_f;
  g.d = dh * G.unit_f;
  g.overlap = ov * G.unit_f;
  return true;
}

// Granule j (position pj, cell offset o from i) within r_i + r_j + reach:
// its signed geometry (FP32 from the exact integer separation).
__device__ __forceinline__ bool pair_within(const DGrid& G, const uint4& pi, const uint4& pj, int ox, int oy, int oz,
                                            float ri, float rj, float reach, PairGeom<float>& g) {
  int Dx, Dy, Dz;
  int_sep(pi, pj, ox, oy, oz, Dx, Dy, Dz);
  const float fx = (float)Dx, fy = (float)Dy, fz = (float)Dz;
  const float Rs = ri + rj + reach;
  if (!(fmaf(fx, fx, fmaf(fy, fy, fz * fz)) < Rs * Rs * G.s2_margin)) return false;
  return pair_geom_signed(G, Dx, Dy, Dz, ri, rj, g);
}
__device__ __forceinline__ bool pair_within(const DGrid& G, const d4& pi, const d4& pj, int ox, int oy, int oz,
                                            double ri, double rj, double reach, PairGeom<double>& g) {
  double x0, x1, x2;
  rel_ij(G, pi, pj, ox, oy, oz, x0, x1, x2);
  const double d2 = x0 * x0 + x1 * x1 + x2 * x2;
  const double Rs = ri + rj + reach;
  if (!(d2 < Rs * Rs)) return false;
  g.x0 = x0;
  g.x1 = x1;
  g.x2 = x2;
  g.d = sqrt(d2);
  g.overlap = ri + rj - g.d;
  return true;
}

// Every partner j in granule i's Verlet row within r_i + r_j + kappa (r_i +
// r_j) (contacts and bridge candidates), in row order: f(j, cj, pj, g) with
// the signed geometry.
template <typename T, typename F>
__device__ __forceinline__ void for_each_list_near(const DGrid& G, const DParams<T>& P, const NbDev& nb, int64_t i,
                                                   int cx, int cy, int cz, const pos_t<T>& pi, T ri, bool has_f,
                                                   const float4& fi, const int32_t* __restrict__ cell,
                                                   const pos_t<T>* __restrict__ pos,
                                                   const float4* __restrict__ posf, F&& f) {
  const int32_t s = nb.ident ? (int32_t)i : nb.at[i];
  const int32_t* row = nb.list + (int64_t)s * nb.cap;
  int cnt = nb.count[s];
  if (!GIC_DBG_OK(nb.dbg, cnt >= 0 && cnt <= nb.cap)) cnt = 0;
  const T grow = T(1) + P.kappa;
  for (int k = 0; k < cnt; ++k) {
    const int64_t j = nb.ident ? row[k] : nb.cur[row[k]];
    if (!GIC_DBG_OK(nb.dbg, j >= 0 && j < nb.n)) continue;
    T rj;
    if constexpr (sizeof(T) == 4) {
      if (has_f) {  // float pre-test on the copies, widened by the bridge reach
        const float4 fj = __ldg(&posf[j]);
        const float rx = fj.x - fi.x, ry = fj.y - fi.y, rz = fj.z - fi.z;
        const float Rc = fmaf(((float)ri + fj.w) * (float)grow, G.inv_hc_f, kPosfTol);
        if (!(fmaf(rx, rx, fmaf(ry, ry, rz * rz)) < Rc * Rc)) continue;
      }
    }
    const int32_t cj = __ldg(&cell[j]);
    const int ox = cell_x(cj) - cx, oy = cell_y(cj) - cy, oz = cell_z(cj) - cz;
    if (ox < -1 || ox > 1 || oy < -1 || oy > 1 || oz < -1 || oz > 1) continue;
    const pos_t<T> pj = ldg(&pos[j]);
    rj = radius_of(pj);
    PairGeom<T> g;
    if (!pair_within(G, pi, pj, ox, oy, oz, ri, rj, P.kappa * (ri + rj), g)) continue;
    f(j, cj, pj, g);
  }
}

// The list build of granule i with the bridge reach: walks the 27 cells,
// keeps in row i every granule within r_i + r_j + skin + kappa (r_i + r_j),
// and hands every one within r_i + r_j + kappa (r_i + r_j) to f(j, cj, pj, g).
template <typename T, typename F>
__device__ __forceinline__ void verlet_build_row_near(const DGrid& G, const DParams<T>& P, const NbDev& nb,
                                                      const uint4* __restrict__ table, int64_t n, int64_t i, int cx,
                                                      int cy, int cz, int32_t ci, const pos_t<T>& pi, T ri, T skin,
                                                      const int32_t* __restrict__ id,
                                                      const pos_t<T>* __restrict__ pos, F&& f) {
  int32_t* row = nb.list + i * nb.cap;
  const uint32_t epoch = __ldg(&table[0].x);
  int cnt = 0;
  bool over = false;
  for_each_partner(G, table, epoch, i, cx, cy, cz, [&](int64_t j, int ox, int oy, int oz) {
    const pos_t<T> pj = ldg(&pos[j]);
    const T rj = radius_of(pj);
    const T reach = P.kappa * (ri + rj);
    PairGeom<T> g;
    if (!pair_within(G, pi, pj, ox, oy, oz, ri, rj, reach + skin, g)) return;
    if (cnt < nb.cap)
      row[cnt++] = (int32_t)j;
    else
      over = true;
    if (g.overlap > -reach) f(j, pack_cell(cx + ox, cy + oy, cz + oz), pj, g);
  });
  nb.count[i] = cnt;
  nb.at[i] = (int32_t)i;
  nb.cur[i] = (int32_t)i;
  nb.ref_cell[i] = ci;
  reinterpret_cast<pos_t<T>*>(nb.ref_pos)[i] = pi;
  const int32_t idi = id[i];
  if (idi >= 0 && (int64_t)idi < n) nb.slot[idi] = (int32_t)i;
  if (over) atomicOr(&nb.flags[kNbOverflow], 1u);
}

// Bridge force on i from j (geometry g with a gap) added to F: zero unless
// 0 < s < d_r.
template <typename T>
__device__ __forceinline__ void add_bridge(const DParams<T>& P, const PairGeom<T>& g, T ri, T rj, T sri, T srj, T& F0,
                                           T& F1, T& F2) {
  const T s = -g.overlap;
  const Bridge<T> b = bridge_of(P, ri, rj);
  if (!(s > T(0)) || !(s < b.dr)) return;
  const T gam = cap_gamma(T(0.5) * (sri + srj), P.cpk, (T*)nullptr);
  if (gam == T(0)) return;
  const T f = -gam * bridge_force(P, b, s, (T*)nullptr) / g.d;
  F0 += f * g.x0;
  F1 += f * g.x1;
  F2 += f * g.x2;
}

// Adjoint of add_bridge for l = lambda_i - lambda_j: adds (dF/dx_ij)^T l to
// gx and returns l . dF/dsr_mean (the caller adds half of it times
// d sr_i / d x_i).  F = -Gamma F^st n: dF/dx = -Gamma (F^st' n n^T + F^st / d
// (I - n n^T)), dF/dsr_mean = -Gamma' F^st n.
template <typename T>
__device__ __forceinline__ T add_bridge_adj(const DParams<T>& P, const PairGeom<T>& g, T ri, T rj, T sri, T srj,
                                            T l0, T l1, T l2, T& gx0, T& gx1, T& gx2) {
  const T s = -g.overlap;
  const Bridge<T> b = bridge_of(P, ri, rj);
  if (!(s > T(0)) || !(s < b.dr)) return T(0);
  T gs;
  const T gam = cap_gamma(T(0.5) * (sri + srj), P.cpk, &gs);
  T fp;
  const T fs = bridge_force(P, b, s, &fp);
  const T inv_d = T(1) / g.d;
  const T n0 = g.x0 * inv_d, n1 = g.x1 * inv_d, n2 = g.x2 * inv_d;
  const T ln = l0 * n0 + l1 * n1 + l2 * n2;
  const T a = fs * inv_d;
  gx0 += -gam * (fp * ln * n0 + a * (l0 - ln * n0));
  gx1 += -gam * (fp * ln * n1 + a * (l1 - ln * n1));
  gx2 += -gam * (fp * ln * n2 + a * (l2 - ln * n2));
  return -gs * fs * ln;
}

}  // namespace gic
