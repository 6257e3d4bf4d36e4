// gic_interp.cuh -- trilinear (tent-kernel) G2P / P2G stencils on the MAC grid.
#pragma once

#include "gic_internal.cuh"

namespace gic {

// Stencil with the axes on which the point was clamped onto an end sample
// (no derivative along those).
template <typename T>
struct Stencil3 {
  int i0[3];
  T w[3];
  bool clamped[3];
  int ns[3];
};

template <typename T>
__device__ __forceinline__ Stencil3<T> make_stencil(const DGrid& G, const int m[3], const T t[3], int comp) {
  Stencil3<T> S;
  const int n[3] = {G.nx, G.ny, G.nz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    bool face = (a == comp);
    int ns = n[a] + (face ? 1 : 0);
    int i0;
    T w;
    bool cl = false;
    if (face) {
      i0 = m[a];
      w = t[a];
    } else if (t[a] >= T(0.5)) {
      i0 = m[a];
      w = t[a] - T(0.5);
    } else {
      i0 = m[a] - 1;
      w = t[a] + T(0.5);
    }
    if (i0 < 0) {
      i0 = 0;
      w = T(0);
      cl = true;
    } else if (i0 > ns - 2) {
      i0 = ns - 2;
      w = T(1);
      cl = true;
    }
    S.i0[a] = i0;
    S.w[a] = w;
    S.clamped[a] = cl;
    S.ns[a] = ns;
  }
  return S;
}

template <typename T>
__device__ __forceinline__ int64_t base_index(const Stencil3<T>& S) {
  return sample_index(S.ns[0], S.ns[1], S.i0[0], S.i0[1], S.i0[2]);
}

// MAC cell and in-cell fraction of a granule on each axis
template <typename T, typename P>
__device__ __forceinline__ void granule_mac(const DGrid& G, int32_t cell, const P& pos, int m[3], T t[3]) {
  int c3[3] = {cell_x(cell), cell_y(cell), cell_z(cell)};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    m[a] = mac_of(G, c3[a]);
    t[a] = (T)mac_frac(G, c3[a], m[a], pcomp(pos, a));
  }
}

// FP64 fraction (exact from the fixed-point state) for the alpha_s path
template <typename P>
__device__ __forceinline__ void granule_mac_fp64(const DGrid& G, int32_t cell, const P& pos, int m[3], double t[3]) {
  int c3[3] = {cell_x(cell), cell_y(cell), cell_z(cell)};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    m[a] = mac_of(G, c3[a]);
    t[a] = mac_frac_fp64(G, c3[a], m[a], pcomp(pos, a));
  }
}

// Interpolate with loader f(i, j, k); optionally the gradient w.r.t. the
// point (per metre).
template <typename T, typename Load>
__device__ __forceinline__ T interp(const Stencil3<T>& S, Load load, T inv_dx, T* grad) {
  T acc = 0, g0 = 0, g1 = 0, g2 = 0;
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        T f = load(S.i0[0] + a, S.i0[1] + b, S.i0[2] + c);
        T wx = a ? S.w[0] : T(1) - S.w[0];
        T wy = b ? S.w[1] : T(1) - S.w[1];
        T wz = c ? S.w[2] : T(1) - S.w[2];
        acc += wx * wy * wz * f;
        if (grad) {
          g0 += (a ? T(1) : T(-1)) * wy * wz * f;
          g1 += wx * (b ? T(1) : T(-1)) * wz * f;
          g2 += wx * wy * (c ? T(1) : T(-1)) * f;
        }
      }
  if (grad) {
    grad[0] = S.clamped[0] ? T(0) : g0 * inv_dx;
    grad[1] = S.clamped[1] ? T(0) : g1 * inv_dx;
    grad[2] = S.clamped[2] ? T(0) : g2 * inv_dx;
  }
  return acc;
}

// Plain sampled field loader
template <typename T>
struct FieldLoad {
  const T* __restrict__ f;
  int nsx, nsy, nsz;
  uint32_t* dbg;
  __device__ __forceinline__ T operator()(int i, int j, int k) const {
    if (!GIC_DBG_OK(dbg, i >= 0 && i < nsx && j >= 0 && j < nsy && k >= 0 && k < nsz)) return T(0);
    return __ldg(&f[sample_index(nsx, nsy, i, j, k)]);
  }
};

// Face-difference pressure gradient on the faces normal to `comp`:
// (p_c - p_{c-1}) / dx, boundary faces copy the adjacent interior face.
template <typename T>
struct GradPLoad {
  const T* __restrict__ p;
  int nx, ny, nz, comp;
  T inv_dx;
  uint32_t* dbg;
  __device__ __forceinline__ T operator()(int i, int j, int k) const {
    int idx[3] = {i, j, k};
    const int n[3] = {nx, ny, nz};
    int c = idx[comp];
    c = c < 1 ? 1 : (c > n[comp] - 1 ? n[comp] - 1 : c);
    idx[comp] = c;
    if (!GIC_DBG_OK(dbg, idx[0] >= 0 && idx[0] < nx && idx[1] >= 0 && idx[1] < ny && idx[2] >= 0 && idx[2] < nz))
      return T(0);
    T hi = __ldg(&p[sample_index(nx, ny, idx[0], idx[1], idx[2])]);
    idx[comp] = c - 1;
    T lo = __ldg(&p[sample_index(nx, ny, idx[0], idx[1], idx[2])]);
    return (hi - lo) * inv_dx;
  }
};

}  // namespace gic
