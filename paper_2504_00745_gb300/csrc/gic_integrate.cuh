// gic_integrate.cuh -- device side of a4 (virtual-mass symplectic Euler,
// Sec. 5.2 Eq. sand kine; Alg. 2 MoveParticle), shared by the integrate
// kernel and the fused substep.
#pragma once

#include "gic_internal.cuh"

namespace gic {

template <typename T>
struct Masses {
  T m, ma;
};

template <typename T>
__device__ __forceinline__ Masses<T> masses(const DParams<T>& P, T r) {
  T V = T(4.0 / 3.0 * kPi) * r * r * r;
  Masses<T> M;
  M.m = P.rho_s * V;
  M.ma = P.vm ? T(0.5) * P.rho_f * V : T(0);
  return M;
}

__device__ __forceinline__ void advance_axis(const DGrid& G, float dt, float v, uint32_t q, int c, int nc,
                                             uint32_t& q_out, int& c_out, uint32_t& flags) {
  float inc_f = dt * v * G.inv_unit_f;
  // clamp far beyond one cell so the integer conversion is defined
  inc_f = fminf(fmaxf(inc_f, -0x1p40f), 0x1p40f);
  // the same rounding either way; the 64-bit conversion runs on the FP64
  // pipe, so it is kept for moves of a cell or more (flagged as fast)
  long long inc = fabsf(inc_f) < 0x1p30f ? (long long)__float2int_rn(inc_f) : __float2ll_rn(inc_f);
  long long s = (long long)q + inc;
  long long shift = s >> kFracBits;  // floor division by 2^30
  q_out = (uint32_t)(s & (long long)kFracMask);
  long long cn = (long long)c + shift;
  if (shift > 1 || shift < -1) flags |= GIC_STATUS_FAST;
  if (cn < 0) {
    cn = 0;
    q_out = 0;
    flags |= GIC_STATUS_OUT_OF_DOMAIN;
  } else if (cn > nc - 1) {
    cn = nc - 1;
    q_out = kFracMask;
    flags |= GIC_STATUS_OUT_OF_DOMAIN;
  }
  c_out = (int)cn;
}

__device__ __forceinline__ void advance_axis(const DGrid& G, double dt, double v, double o, int c, int nc,
                                             double& o_out, int& c_out, uint32_t& flags) {
  double x = o + dt * v;
  double sh = floor(x * G.inv_hc);
  if (!(fabs(sh) < 1e9)) sh = x > 0 ? 1e9 : -1e9;
  long long shift = (long long)sh;
  x -= sh * G.hc;
  // guard against rounding just outside [0, h_c)
  if (x < 0.0) x = 0.0;
  if (x >= G.hc) x = nextafter(G.hc, 0.0);
  if (shift > 1 || shift < -1) flags |= GIC_STATUS_FAST;
  long long cn = (long long)c + shift;
  if (cn < 0) {
    cn = 0;
    x = 0.0;
    flags |= GIC_STATUS_OUT_OF_DOMAIN;
  } else if (cn > nc - 1) {
    cn = nc - 1;
    x = nextafter(G.hc, 0.0);
    flags |= GIC_STATUS_OUT_OF_DOMAIN;
  }
  o_out = x;
  c_out = (int)cn;
}

// One granule: new cell / position record / velocity and the exchange force
// f_ex = F_fl + m_a (a_f - a) from the forces on it; status bits in flags.
template <typename T>
__device__ __forceinline__ void integrate_granule(const DGrid& G, const DParams<T>& P, int32_t c, const pos_t<T>& p,
                                                  const vec_t<T>& v, T fc0, T fc1, T fc2, T ff0, T ff1, T ff2,
                                                  T fa0, T fa1, T fa2, int32_t& c_out, pos_t<T>& p_out,
                                                  vec_t<T>& v_out, T& fe0, T& fe1, T& fe2, uint32_t& flags) {
  Masses<T> M = masses(P, radius_of(p));
  T inv = T(1) / (M.m + M.ma);
  T a0 = (fc0 + ff0 + M.m * P.g[0] + M.ma * fa0) * inv;
  T a1 = (fc1 + ff1 + M.m * P.g[1] + M.ma * fa1) * inv;
  T a2 = (fc2 + ff2 + M.m * P.g[2] + M.ma * fa2) * inv;
  T v0 = v.x + P.dt * a0, v1 = v.y + P.dt * a1, v2 = v.z + P.dt * a2;
  if (!isfinite(v0) || !isfinite(v1) || !isfinite(v2)) flags |= GIC_STATUS_NONFINITE;
  int c3[3] = {cell_x(c), cell_y(c), cell_z(c)};
  int cn[3];
  p_out = p;
  advance_axis(G, P.dt, v0, p.x, c3[0], G.nc[0], p_out.x, cn[0], flags);
  advance_axis(G, P.dt, v1, p.y, c3[1], G.nc[1], p_out.y, cn[1], flags);
  advance_axis(G, P.dt, v2, p.z, c3[2], G.nc[2], p_out.z, cn[2], flags);
  c_out = pack_cell(cn[0], cn[1], cn[2]);
  v_out = make_vec<T>(v0, v1, v2);
  fe0 = ff0 + M.ma * (fa0 - a0);
  fe1 = ff1 + M.ma * (fa1 - a1);
  fe2 = ff2 + M.ma * (fa2 - a2);
}

// Adjoint of integrate_granule: from the gradients gx, gv, gf of (x', v',
// f_ex) of a granule of radius r to those of v (gvt; x's is gx itself), F_c,
// F_fl and a_f.  x' = x + dt v', v' = v + dt a, a = (F_c + F_fl + m g +
// m_a a_f) / (m + m_a), f_ex = F_fl + m_a (a_f - a).
template <typename T>
struct IntegrateAdj {
  T gvt[3], gFc[3], gFfl[3], gaf[3];
};

template <typename T>
__device__ __forceinline__ IntegrateAdj<T> integrate_adj_granule(const DParams<T>& P, T r, const vec_t<T>& gx,
                                                                 const vec_t<T>& gv, const vec_t<T>& gf) {
  const Masses<T> M = masses(P, r);
  const T inv = T(1) / (M.m + M.ma);
  IntegrateAdj<T> o;
  const T x[3] = {gx.x, gx.y, gx.z}, v[3] = {gv.x, gv.y, gv.z}, f[3] = {gf.x, gf.y, gf.z};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    o.gvt[a] = v[a] + P.dt * x[a];
    const T ga = P.dt * o.gvt[a] - M.ma * f[a];  // a enters v' (dt) and f_ex (-m_a)
    o.gFc[a] = ga * inv;
    o.gFfl[a] = ga * inv + f[a];
    o.gaf[a] = M.ma * (ga * inv + f[a]);
  }
  return o;
}

}  // namespace gic
