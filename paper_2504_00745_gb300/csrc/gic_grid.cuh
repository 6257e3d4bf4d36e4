// gic_grid.cuh -- device side of a3 (G2P coupling) and a5 (P2G), shared by
// the grid kernels and the fused substep.
#pragma once

#include <climits>

#include "gic_interp.cuh"

namespace gic {

template <typename T>
struct Fields {
  const T* u;
  const T* v;
  const T* w;
  const T* p;
  const T* af;
};

template <typename T>
__device__ __forceinline__ FieldLoad<T> face_loader(const DGrid& G, const T* f, int comp) {
  FieldLoad<T> L;
  L.f = f;
  L.nsx = G.nx + (comp == 0);
  L.nsy = G.ny + (comp == 1);
  L.nsz = G.nz + (comp == 2);
  L.dbg = G.dbg;
  return L;
}

template <typename T>
__device__ __forceinline__ GradPLoad<T> gradp_loader(const DGrid& G, const T* p, int comp) {
  GradPLoad<T> L;
  L.p = p;
  L.nx = G.nx;
  L.ny = G.ny;
  L.nz = G.nz;
  L.comp = comp;
  L.inv_dx = grid_inv_dx<T>(G);
  L.dbg = G.dbg;
  return L;
}

// G2P coupling of one granule at (cell, p) with velocity v (Sec. 3.3 Eqs. 5a,
// 5b; Sec. 5.2 Eq. momentum4): F_fl = c_drag pi r^2 rho_f |u_f - v| (u_f - v)
// - V grad p and a_f = g - grad p / rho_f.  Returns |u_f - v|.  face(comp)
// and gradp(comp) give the samplers of the face velocities and of the face
// pressure gradients (global memory or a staged tile: the same values).
template <typename T, typename Face, typename GradP>
__device__ __forceinline__ T g2p_granule_with(const DGrid& G, const DParams<T>& P, int32_t cell, const pos_t<T>& pi,
                                              const vec_t<T>& vi, Face face, GradP gradp, T F[3], T a[3]) {
  int m[3];
  T t[3];
  granule_mac<T>(G, cell, pi, m, t);
  T uf[3], gp[3];
  T inv_dx = grid_inv_dx<T>(G);
#pragma unroll
  for (int comp = 0; comp < 3; ++comp) {
    Stencil3<T> S = make_stencil<T>(G, m, t, comp);
    uf[comp] = interp<T>(S, face(comp), inv_dx, nullptr);
    gp[comp] = interp<T>(S, gradp(comp), inv_dx, nullptr);
  }
  T r = radius_of(pi);
  T V = T(4.0 / 3.0 * kPi) * r * r * r;
  T d0 = uf[0] - vi.x, d1 = uf[1] - vi.y, d2 = uf[2] - vi.z;
  T sp = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
  T cd = P.c_drag * T(kPi) * r * r * P.rho_f * sp;
  F[0] = cd * d0 - V * gp[0];
  F[1] = cd * d1 - V * gp[1];
  F[2] = cd * d2 - V * gp[2];
  if (P.rho_f > T(0)) {
    a[0] = P.g[0] - gp[0] * P.inv_rho_f;
    a[1] = P.g[1] - gp[1] * P.inv_rho_f;
    a[2] = P.g[2] - gp[2] * P.inv_rho_f;
  } else {
    a[0] = P.g[0];
    a[1] = P.g[1];
    a[2] = P.g[2];
  }
  return sp;
}

template <typename T>
__device__ __forceinline__ T g2p_granule(const DGrid& G, const DParams<T>& P, const Fields<T>& Fd, int32_t cell,
                                         const pos_t<T>& pi, const vec_t<T>& vi, T F[3], T a[3]) {
  const T* uvw[3] = {Fd.u, Fd.v, Fd.w};
  return g2p_granule_with<T>(
      G, P, cell, pi, vi, [&](int comp) { return face_loader<T>(G, uvw[comp], comp); },
      [&](int comp) { return gradp_loader<T>(G, Fd.p, comp); }, F, a);
}

// Adjoint of g2p_granule for upstream gradients l (of F_fl) and la (of
// a_f): adds their gradient w.r.t. the position to gx, writes in gdv the one
// w.r.t. the slip u_f - v (so the velocity's is -gdv) and returns the c_drag
// gradient.  m, t: the granule's MAC cell and offsets, for further stencils.
template <typename T>
__device__ __forceinline__ T g2p_adj_granule(const DGrid& G, const DParams<T>& P, const Fields<T>& Fd, int32_t cell,
                                             const pos_t<T>& pi, const vec_t<T>& vi, const T l[3], const T la[3],
                                             T gx[3], T gdv[3], int m[3], T t[3]) {
  granule_mac<T>(G, cell, pi, m, t);
  const T* uvw[3] = {Fd.u, Fd.v, Fd.w};
  T uf[3], gu[3][3], ggp[3][3];
  const T inv_dx = grid_inv_dx<T>(G);
#pragma unroll
  for (int comp = 0; comp < 3; ++comp) {
    Stencil3<T> S = make_stencil<T>(G, m, t, comp);
    uf[comp] = interp<T>(S, face_loader<T>(G, uvw[comp], comp), inv_dx, gu[comp]);
    interp<T>(S, gradp_loader<T>(G, Fd.p, comp), inv_dx, ggp[comp]);
  }
  const T r = radius_of(pi);
  const T V = T(4.0 / 3.0 * kPi) * r * r * r;
  const T dv[3] = {uf[0] - vi.x, uf[1] - vi.y, uf[2] - vi.z};
  const T sp = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
  const T k = P.c_drag * T(kPi) * r * r * P.rho_f;
  const T dvl = dv[0] * l[0] + dv[1] * l[1] + dv[2] * l[2];
  // d/d dv of k |dv| dv . l = k (|dv| l + (dv . l) dv / |dv|)
#pragma unroll
  for (int a = 0; a < 3; ++a) gdv[a] = sp > T(0) ? k * (sp * l[a] + dvl * dv[a] / sp) : T(0);
#pragma unroll
  for (int comp = 0; comp < 3; ++comp) {
    const T ggrad = -V * l[comp] - P.inv_rho_f * la[comp];  // upstream of grad p component
#pragma unroll
    for (int b = 0; b < 3; ++b) gx[b] += gdv[comp] * gu[comp][b] + ggrad * ggp[comp][b];
  }
  return T(kPi) * r * r * P.rho_f * sp * dvl;
}

// ---- FP32 path: exact fixed-point volume fraction ----
//
// alpha_s is accumulated as a 64-bit integer in units of 2^-53: per granule
// the volume fraction S = V / dx^3 is rounded once to 2^-53; the per-axis
// tent weights come from the 30-bit fixed-point position as 31-bit integers
// (exact when the contact cell is the MAC cell), S times their product is
// formed to 2^-62 and each corner's deposit truncated to 2^-53, and the eighth
// corner takes the rest, so every granule deposits exactly S; integer atomics
// make the sum independent of the order of arrival -- bitwise reproducible.
// k_alpha_finish turns the integers into doubles in place.

constexpr uint32_t kW1 = 1u << 31;  // weight 1.0

// Centred-stencil weights of one axis from the contact coordinate c and the
// fixed-point offset q: lower sample i0 and integer weights (w0, w1), w0 + w1 = 2^31.
__device__ __forceinline__ void fixed_axis(const DGrid& G, int c, uint32_t q, int n, int& i0, uint32_t& w1) {
  int m = mac_of(G, c);
  unsigned long long N = ((unsigned long long)(c - m * G.k) << kFracBits) | q;  // offset in 2^-30 h_c
  // P = round(N * 2 / k): the offset inside the MAC cell in units of 2^-31 dx
  unsigned long long P;
  if (G.k == 1)
    P = N << 1;
  else if (G.k == 2)
    P = N;
  else
    P = (__umul64hi(N << 2, G.kinv64) + 1ull) >> 1;
  uint32_t p = (uint32_t)P;  // < 2^31
  if (p >= (1u << 30)) {
    i0 = m;
    w1 = p - (1u << 30);
  } else {
    i0 = m - 1;
    w1 = p + (1u << 30);
  }
  if (i0 < 0) {
    i0 = 0;
    w1 = 0;
  } else if (i0 > n - 2) {
    i0 = n - 2;
    w1 = kW1;
  }
}

// An integer-valued float (|v| >= 2^23) as int64, exactly, with integer ops.
__device__ __forceinline__ long long float_int_to_ll(float v) {
  uint32_t b = __float_as_uint(v);
  int e = (int)((b >> 23) & 0xffu) - 127 - 23;
  long long m = (long long)((b & 0x7fffffu) | 0x800000u);
  long long r = e >= 0 ? (m << e) : (m >> (-e));
  return (b >> 31) ? -r : r;
}

// S = V / dx^3 in 2^-53 units for radius r, rounded, in FP32 double-float
// arithmetic (r^3 exact to ~2^-46, the constant as a float pair): the FP64
// pipe of this GPU is 1/64 of the FP32 rate.
__device__ __forceinline__ unsigned long long volume_fixed(const DGrid& G, float r) {
  float r2h = r * r;
  float r2l = fmaf(r, r, -r2h);
  float r3h = r2h * r;
  float r3l = fmaf(r2h, r, -r3h) + r2l * r;
  float sh = r3h * G.vol_fx_hi;
  float sl = fmaf(r3h, G.vol_fx_hi, -sh) + fmaf(r3h, G.vol_fx_lo, r3l * G.vol_fx_hi);
  long long a = fabsf(sh) >= 8388608.0f ? float_int_to_ll(sh) : (long long)__float2ll_rn(sh);
  return (unsigned long long)(a + __float2ll_rn(sl));
}

// floor(x w / 2^31) for x < 2^63, w <= 2^31, with two 32x32->64 products.
__device__ __forceinline__ unsigned long long mul31(unsigned long long x, uint32_t w) {
  unsigned long long hi = (unsigned long long)(uint32_t)(x >> 32) * w;
  unsigned long long lo = (unsigned long long)(uint32_t)x * w;
  return (hi << 1) + (lo >> 31);
}

// FP32-path alpha_s deposits of one granule at its new position: the base
// sample i0 and the eight integer deposits (2^-53 units) summing to S exactly.
// S is carried in 2^-62 units through the three per-axis weight products
// (each truncated once), so a deposit is within ~2^-53 of S w_x w_y w_z; the
// eighth corner takes S minus the other seven.
__device__ __forceinline__ void alpha_deposits(const DGrid& G, int32_t cn, uint4 pn, int i0[3], long long v[8],
                                               unsigned long long& S) {
  S = volume_fixed(G, __uint_as_float(pn.w));
  int c3[3] = {cell_x(cn), cell_y(cn), cell_z(cn)};
  const int nn[3] = {G.nx, G.ny, G.nz};
  uint32_t w1[3], w0[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    fixed_axis(G, c3[a], pcomp(pn, a), nn[a], i0[a], w1[a]);
    w0[a] = kW1 - w1[a];
  }
  const unsigned long long S9 = S << 9;  // < 2^63
  unsigned long long sx[2], sxy[4];
  sx[0] = mul31(S9, w0[0]);
  sx[1] = mul31(S9, w1[0]);
#pragma unroll
  for (int k = 0; k < 4; ++k) sxy[k] = mul31(sx[k & 1], (k & 2) ? w1[1] : w0[1]);
  long long sum7 = 0;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    v[k] = (long long)(mul31(sxy[k & 3], (k & 4) ? w1[2] : w0[2]) >> 9);
    sum7 += v[k];
  }
  v[7] = (long long)S - sum7;
}

// FP32 path of P2G.  One CTA takes its consecutive granules (512 in the P2G
// kernel, 256 in the fused substep) of the Morton-sorted state, which occupy
// a compact block of MAC cells.  When the
// samples they may touch fit a kP2GTile-entry box, every deposit goes to
// shared-memory copies of alpha_s and the three F_s grids over that box,
// held as 32-bit integer limbs (32-bit shared integer atomics run at full
// rate even when lanes collide, unlike float or 64-bit ones), and the box's
// non-zero entries then go to global memory with one atomic each; otherwise
// every deposit is a global atomic.
//   alpha_s: a deposit (< 2^54 units of 2^-53) is split into three 18-bit
//   limbs, so up to 2^14 deposits per entry add without overflow -- exact.
//   F_s: a deposit d is rounded to a multiple of u = M 2^-b, M the CTA's
//   largest |exch f_ex| component and b = 30 - ceil(log2(CTA threads)), so
//   |q| = |d / u| <= 2^b and the at most one deposit per granule and entry
//   sum to |sum q| <= 2^30 in one 32-bit integer: exact, and the only
//   rounding besides the float product d is the grid u (2^-22 M for 256
//   threads, finer than the float sum it replaces).
// alpha_s stays 64-bit fixed point (exact, order-independent) until
// k_alpha_finish_f32.
constexpr int kP2GTile = 1024;

// Shared-memory copies of alpha_s and the three F_s grids over one CTA's box.
struct P2GShared {
  uint32_t a[3][kP2GTile];
  int32_t f[3][kP2GTile];
  int lo[3], hi[3];
  unsigned M;
};

// One thread's contribution to its CTA's box and fixed-point scale.
struct P2GExtent {
  int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
  float M = 0.f;
  // a stencil's base is the MAC cell m or m - 1 on each axis, and it reaches one sample further
  __device__ __forceinline__ void add_cell(const DGrid& G, int32_t c) {
    const int c3[3] = {cell_x(c), cell_y(c), cell_z(c)};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      int m = mac_of(G, c3[a]);
      lo[a] = min(lo[a], m - 1);
      hi[a] = max(hi[a], m + 1);
    }
  }
  __device__ __forceinline__ void add_force(const float fc[3]) {
    float m = fmaxf(fabsf(fc[0]), fmaxf(fabsf(fc[1]), fabsf(fc[2])));
    M = fmaxf(M, m <= 3.0e38f ? m : INFINITY);  // NaN or inf: no fixed-point grid for this CTA
  }
};

struct P2GBox {
  bool tile, ftile;     // deposits go to the shared box (alpha_s; F_s)
  bool do_a, do_f;      // alpha_s / F_s requested
  int b[3], ex, sy, sz, vol;
  float unit, inv_unit;  // F_s fixed-point unit M 2^-b and its inverse
};

__device__ __forceinline__ void p2g_box_init(P2GShared& sh) {
  if (threadIdx.x < 3) {
    sh.lo[threadIdx.x] = INT_MAX;
    sh.hi[threadIdx.x] = INT_MIN;
  }
  if (threadIdx.x == 0) sh.M = 0u;
}

// CTA-wide: reduce the extents, decide the tile and zero it.  Every thread
// of the CTA must call it (it synchronises the CTA).
__device__ __forceinline__ P2GBox p2g_box(P2GShared& sh, const P2GExtent& ext, bool do_a, bool do_f) {
  __syncthreads();
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int l = __reduce_min_sync(0xffffffffu, ext.lo[a]);
    int h = __reduce_max_sync(0xffffffffu, ext.hi[a]);
    if (lane_id() == 0) {
      atomicMin(&sh.lo[a], l);
      atomicMax(&sh.hi[a], h);
    }
  }
  if (do_f) {  // non-negative floats order like their bit patterns
    unsigned mb = __reduce_max_sync(0xffffffffu, __float_as_uint(ext.M));
    if (lane_id() == 0) atomicMax(&sh.M, mb);
  }
  __syncthreads();
  P2GBox B;
  B.do_a = do_a;
  B.do_f = do_f;
  B.b[0] = max(sh.lo[0], 0);
  B.b[1] = max(sh.lo[1], 0);
  B.b[2] = max(sh.lo[2], 0);
  const int ex = sh.hi[0] - B.b[0] + 1, ey = sh.hi[1] - B.b[1] + 1, ez = sh.hi[2] - B.b[2] + 1;
  // a CTA without granules has lo > hi
  B.tile = ex > 0 && ey > 0 && ez > 0 && (int64_t)ex * ey * ez <= kP2GTile;
  const float Mc = __uint_as_float(sh.M);
  B.ftile = B.tile && do_f && Mc >= 1e-30f && Mc <= 3.0e38f;
  const int bits = 30 - (32 - __clz((int)blockDim.x - 1));  // 22 for 256 threads, 21 for 512
  B.unit = ldexpf(Mc, -bits);
  B.inv_unit = B.ftile ? ldexpf(1.0f, bits) / Mc : 0.f;
  B.vol = B.tile ? ex * ey * ez : 0;
  B.ex = ex;
  B.sy = ex;
  B.sz = ex * ey;
  for (int e = threadIdx.x; e < B.vol; e += blockDim.x) {
    if (do_a) sh.a[0][e] = sh.a[1][e] = sh.a[2][e] = 0u;
    if (B.ftile) {
#pragma unroll
      for (int c = 0; c < 3; ++c) sh.f[c][e] = 0;
    }
  }
  if (B.tile) __syncthreads();
  return B;
}

__device__ __forceinline__ void p2g_add_alpha(P2GShared& sh, const P2GBox& B, const DGrid& G,
                                              unsigned long long* acc, const int ia[3], const long long va[8]) {
  if (B.tile) {
    const int e0 = (ia[0] - B.b[0]) + B.sy * (ia[1] - B.b[1]) + B.sz * (ia[2] - B.b[2]);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int e = e0 + (k & 1) + ((k >> 1) & 1) * B.sy + (k >> 2) * B.sz;
      const unsigned long long v = (unsigned long long)va[k];
      atomicAdd(&sh.a[0][e], (uint32_t)(v & 0x3ffffull));
      atomicAdd(&sh.a[1][e], (uint32_t)((v >> 18) & 0x3ffffull));
      atomicAdd(&sh.a[2][e], (uint32_t)(v >> 36));
    }
  } else {
    unsigned long long* g0 = acc + sample_index(G.nx, G.ny, ia[0], ia[1], ia[2]);
    const int64_t gy = G.nx, gz = (int64_t)G.nx * G.ny;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (va[k]) atomicAdd(g0 + (k & 1) + ((k >> 1) & 1) * gy + (k >> 2) * gz, (unsigned long long)va[k]);
  }
}

// F_s deposit of one granule on face grid comp: the eight stencil weights
// times fc (= exch f_ex component).
__device__ __forceinline__ void p2g_add_face(P2GShared& sh, const P2GBox& B, const DGrid& G, float* Fs, int comp,
                                             const Stencil3<float>& St, float fc) {
  const float wx = St.w[0], wy = St.w[1], wz = St.w[2];
  const float fx0 = (1.f - wx) * fc, fx1 = wx * fc;
  const float wyz[4] = {(1.f - wy) * (1.f - wz), wy * (1.f - wz), (1.f - wy) * wz, wy * wz};
  if (B.ftile) {
    const int e0 = (St.i0[0] - B.b[0]) + B.sy * (St.i0[1] - B.b[1]) + B.sz * (St.i0[2] - B.b[2]);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int q = __float2int_rn(((k & 1) ? fx1 : fx0) * wyz[k >> 1] * B.inv_unit);
      const int e = e0 + (k & 1) + ((k >> 1) & 1) * B.sy + (k >> 2) * B.sz;
      atomicAdd(&sh.f[comp][e], q);
    }
  } else {
    const int nsx = G.nx + (comp == 0), nsy = G.ny + (comp == 1);
    float* g0 = Fs + sample_index(nsx, nsy, St.i0[0], St.i0[1], St.i0[2]);
    const int64_t gy = nsx, gz = (int64_t)nsx * nsy;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float d = ((k & 1) ? fx1 : fx0) * wyz[k >> 1];
      if (d != 0.f) atomicAdd(g0 + (k & 1) + ((k >> 1) & 1) * gy + (k >> 2) * gz, d);
    }
  }
}

// CTA-wide: the box's non-zero entries to global memory (one atomic each).
__device__ __forceinline__ void p2g_flush(P2GShared& sh, const P2GBox& B, const DGrid& G, unsigned long long* acc,
                                          float* const Fs[3], int threads) {
  if (!B.tile) return;
  __syncthreads();
  // e = lx + ex (ly + ey lz); (e + 1/2) / d stays >= 1/(2 d) away from an
  // integer, far beyond the float error for e, d <= 1024
  const float rx = 1.f / (float)B.ex, rxy = 1.f / (float)B.sz;
  for (int e = threadIdx.x; e < B.vol; e += threads) {
    int lz = (int)(((float)e + 0.5f) * rxy);
    int r = e - lz * B.sz;
    int ly = (int)(((float)r + 0.5f) * rx);
    int lx = r - ly * B.ex;
    int gx = B.b[0] + lx, gy = B.b[1] + ly, gz = B.b[2] + lz;
    if (B.do_a) {
      unsigned long long a = (unsigned long long)sh.a[0][e] + ((unsigned long long)sh.a[1][e] << 18) +
                             ((unsigned long long)sh.a[2][e] << 36);
      if (a) atomicAdd(&acc[sample_index(G.nx, G.ny, gx, gy, gz)], a);
    }
    if (B.ftile) {
#pragma unroll
      for (int comp = 0; comp < 3; ++comp) {
        const int q = sh.f[comp][e];
        if (q) atomicAdd(&Fs[comp][sample_index(G.nx + (comp == 0), G.ny + (comp == 1), gx, gy, gz)],
                         (float)q * B.unit);
      }
    }
  }
}

// Exact integer total of sum_i S_i (S_i = V_i / dx^3 in 2^-53 units, the
// amount every granule deposits) while the scatter runs: a 128-bit unsigned
// integer held in the 16 bytes of sums[0..1] (low word in sums[1], high word
// in sums[0]); a warp adds its total (< 2^59) to the low word and carries into
// the high word when the low word wraps, so the sum is exact and independent
// of the order of the atomics.  k_alpha_total_f32 turns it into sum_i V_i.
__device__ __forceinline__ void p2g_sums(double* sums, long long v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if (lane_id() == 0 && v != 0) {
    const unsigned long long add = (unsigned long long)v;
    const unsigned long long old = atomicAdd((unsigned long long*)&sums[1], add);
    if (old + add < old) atomicAdd((unsigned long long*)&sums[0], 1ull);
  }
}

// ---- FP32 fused substep: one CTA tile for G2P staging and P2G ----
//
// The CTA's granules (consecutive in Morton order) have MAC cells m; every
// sample their G2P and F_s stencils touch has indices m - 1 .. m + 1 per
// axis.  At the start of the substep the CTA reduces that box, stages the
// face velocities and the face pressure gradients of its samples in shared
// memory (each computed as the global-memory samplers compute it, so G2P
// gives the same bits) and zeroes its F_s (and alpha_s) accumulators; F_s is
// then scattered into the same box (fixed point as in the P2G kernel), and
// alpha_s, at the new positions, into it where the stencil fits.  A box
// beyond kSubTile entries falls back to global memory.
constexpr int kSubTile = 960;  // 46 KB of static shared memory
constexpr int kSubWarps = 8;  // CTA of 256 threads

struct SubTile {
  float u[kSubTile], v[kSubTile], w[kSubTile];
  float gp[3][kSubTile];
  int32_t f[3][kSubTile];
  uint32_t a[3][kSubTile];
  int wlo[3][kSubWarps], whi[3][kSubWarps];
  unsigned wM[kSubWarps];
};

struct SubBox {
  bool tile;
  int b[3], ex, ey, ez, sy, sz, vol;
  __device__ __forceinline__ int index(int i, int j, int k) const {
    return (i - b[0]) + sy * (j - b[1]) + sz * (k - b[2]);
  }
  __device__ __forceinline__ bool holds(int i, int j, int k) const {  // the 2x2x2 stencil based at (i, j, k)
    return i >= b[0] && j >= b[1] && k >= b[2] && i + 1 < b[0] + ex && j + 1 < b[1] + ey && k + 1 < b[2] + ez;
  }
};

// Sampler of a staged field: the same values as the global sampler.
struct TileLoad {
  const float* s;
  SubBox B;
  uint32_t* dbg;
  __device__ __forceinline__ float operator()(int i, int j, int k) const {
    const int e = B.index(i, j, k);
    if (!GIC_DBG_OK(dbg, e >= 0 && e < B.vol)) return 0.f;
    return s[e];
  }
};

// CTA-wide (every thread calls it): the box of the granules' MAC cells, the
// staged fields and the zeroed accumulators.  valid: this thread has a
// granule in contact cell c.
__device__ __forceinline__ SubBox sub_tile_begin(SubTile& sh, const DGrid& G, const Fields<float>& Fd, bool valid,
                                                 int32_t c, bool do_a, bool do_f) {
  const int warp = threadIdx.x >> 5;
  const int c3[3] = {cell_x(c), cell_y(c), cell_z(c)};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int m = valid ? mac_of(G, c3[a]) : 0;
    const int l = __reduce_min_sync(0xffffffffu, valid ? m : INT_MAX);
    const int h = __reduce_max_sync(0xffffffffu, valid ? m : INT_MIN);
    if (lane_id() == 0) {
      sh.wlo[a][warp] = l;
      sh.whi[a][warp] = h;
    }
  }
  __syncthreads();
  int lo[3], hi[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = INT_MAX;
    hi[a] = INT_MIN;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      lo[a] = min(lo[a], sh.wlo[a][w]);
      hi[a] = max(hi[a], sh.whi[a][w]);
    }
  }
  SubBox B;
  const bool any = lo[0] <= hi[0];  // a CTA without granules has lo > hi
  B.b[0] = any ? max(lo[0] - 1, 0) : 0;
  B.b[1] = any ? max(lo[1] - 1, 0) : 0;
  B.b[2] = any ? max(lo[2] - 1, 0) : 0;
  B.ex = any ? hi[0] + 1 - B.b[0] + 1 : 1;
  B.ey = any ? hi[1] + 1 - B.b[1] + 1 : 1;
  B.ez = any ? hi[2] + 1 - B.b[2] + 1 : 1;
  B.tile = any && (int64_t)B.ex * B.ey * B.ez <= kSubTile;
  B.sy = B.ex;
  B.sz = B.ex * B.ey;
  B.vol = B.tile ? B.ex * B.ey * B.ez : 0;
  const float rx = 1.f / (float)B.ex, rxy = 1.f / (float)max(B.sz, 1);
  for (int e = threadIdx.x; e < B.vol; e += blockDim.x) {
    // e = lx + ex (ly + ey lz); (e + 1/2) / d stays >= 1/(2 d) from an integer
    const int lz = (int)(((float)e + 0.5f) * rxy);
    const int r = e - lz * B.sz;
    const int ly = (int)(((float)r + 0.5f) * rx);
    const int lx = r - ly * B.ex;
    const int i = B.b[0] + lx, j = B.b[1] + ly, k = B.b[2] + lz;
    const bool cx = i < G.nx, cy = j < G.ny, cz = k < G.nz;  // a cell-centred index
    const bool fx = i <= G.nx, fy = j <= G.ny, fz = k <= G.nz;  // a face index
    sh.u[e] = (fx && cy && cz) ? face_loader<float>(G, Fd.u, 0)(i, j, k) : 0.f;
    sh.v[e] = (cx && fy && cz) ? face_loader<float>(G, Fd.v, 1)(i, j, k) : 0.f;
    sh.w[e] = (cx && cy && fz) ? face_loader<float>(G, Fd.w, 2)(i, j, k) : 0.f;
    sh.gp[0][e] = (fx && cy && cz) ? gradp_loader<float>(G, Fd.p, 0)(i, j, k) : 0.f;
    sh.gp[1][e] = (cx && fy && cz) ? gradp_loader<float>(G, Fd.p, 1)(i, j, k) : 0.f;
    sh.gp[2][e] = (cx && cy && fz) ? gradp_loader<float>(G, Fd.p, 2)(i, j, k) : 0.f;
    if (do_f) sh.f[0][e] = sh.f[1][e] = sh.f[2][e] = 0;
    if (do_a) sh.a[0][e] = sh.a[1][e] = sh.a[2][e] = 0u;
  }
  __syncthreads();
  return B;
}

// G2P of one granule from global memory, out of line: the path of a CTA whose
// box exceeds the tile, kept out of the fused kernel's instruction stream.
struct G2POut {
  float F[3], a[3], sp;
};
static __device__ __noinline__ G2POut g2p_global_f32(const DGrid G, const DParams<float> P, const Fields<float> Fd,
                                                     int32_t c, uint4 pi, float4 vi) {
  G2POut o;
  o.sp = g2p_granule<float>(G, P, Fd, c, pi, vi, o.F, o.a);
  return o;
}

// G2P of one granule from the staged tile (B.tile) or global memory.
__device__ __forceinline__ float sub_g2p(const SubTile& sh, const SubBox& B, const DGrid& G, const DParams<float>& P,
                                         const Fields<float>& Fd, int32_t c, const uint4& pi, const float4& vi,
                                         float F[3], float a[3]) {
  if (!B.tile) {
    const G2POut o = g2p_global_f32(G, P, Fd, c, pi, vi);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      F[d] = o.F[d];
      a[d] = o.a[d];
    }
    return o.sp;
  }
  const float* uvw[3] = {sh.u, sh.v, sh.w};
  return g2p_granule_with<float>(
      G, P, c, pi, vi, [&](int comp) { return TileLoad{uvw[comp], B, G.dbg}; },
      [&](int comp) { return TileLoad{sh.gp[comp], B, G.dbg}; }, F, a);
}

// CTA-wide: the F_s fixed-point unit from the largest |exch f_ex| component
// of the CTA (M); returns 2^b / M (0 if F_s cannot use the tile).
__device__ __forceinline__ float sub_fs_scale(SubTile& sh, const SubBox& B, float Mthread, float& unit) {
  const int warp = threadIdx.x >> 5;
  const unsigned mb = __reduce_max_sync(0xffffffffu, __float_as_uint(Mthread));  // non-negative floats
  if (lane_id() == 0) sh.wM[warp] = mb;
  __syncthreads();
  unsigned M = 0u;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) M = max(M, sh.wM[w]);
  const float Mc = __uint_as_float(M);
  const int bits = 30 - (32 - __clz((int)blockDim.x - 1));  // 22 for 256 threads
  const bool ok = B.tile && Mc >= 1e-30f && Mc <= 3.0e38f;
  unit = ldexpf(Mc, -bits);
  return ok ? ldexpf(1.0f, bits) / Mc : 0.f;
}

// F_s deposit of one granule on face grid comp (its stencil lies in the box
// whenever the tile is used; inv_unit = 0: global atomics).
// F_s deposit of one granule on face grid comp straight to global memory
// (float atomics).
__device__ __forceinline__ void add_face_global(const DGrid& G, float* Fs, int comp, const Stencil3<float>& St,
                                                float fc) {
  const float wx = St.w[0], wy = St.w[1], wz = St.w[2];
  const float fx0 = (1.f - wx) * fc, fx1 = wx * fc;
  const float wyz[4] = {(1.f - wy) * (1.f - wz), wy * (1.f - wz), (1.f - wy) * wz, wy * wz};
  const int nsx = G.nx + (comp == 0), nsy = G.ny + (comp == 1);
  float* g0 = Fs + sample_index(nsx, nsy, St.i0[0], St.i0[1], St.i0[2]);
  const int64_t gy = nsx, gz = (int64_t)nsx * nsy;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float d = ((k & 1) ? fx1 : fx0) * wyz[k >> 1];
    if (d != 0.f) atomicAdd(g0 + (k & 1) + ((k >> 1) & 1) * gy + (k >> 2) * gz, d);
  }
}

__device__ __forceinline__ void sub_add_face(SubTile& sh, const SubBox& B, const DGrid& G, float* Fs, int comp,
                                             const Stencil3<float>& St, float fc, float inv_unit) {
  if (inv_unit == 0.f) {
    add_face_global(G, Fs, comp, St, fc);
    return;
  }
  const float wx = St.w[0], wy = St.w[1], wz = St.w[2];
  const float fx0 = (1.f - wx) * fc, fx1 = wx * fc;
  const float wyz[4] = {(1.f - wy) * (1.f - wz), wy * (1.f - wz), (1.f - wy) * wz, wy * wz};
  const int e0 = B.index(St.i0[0], St.i0[1], St.i0[2]);
  if (!GIC_DBG_OK(G.dbg, e0 >= 0 && e0 + 1 + B.sy + B.sz < B.vol)) return;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int q = __float2int_rn(((k & 1) ? fx1 : fx0) * wyz[k >> 1] * inv_unit);
    atomicAdd(&sh.f[comp][e0 + (k & 1) + ((k >> 1) & 1) * B.sy + (k >> 2) * B.sz], q);
  }
}

// F_s deposits of one granule straight to global memory, out of line: in a
// call without alpha_s, the path of a CTA whose F_s cannot use the tile.
static __device__ __noinline__ void fs_deposit_global(const DGrid G, float* Fs_u, float* Fs_v, float* Fs_w, int32_t c,
                                                      uint4 pi, float fc0, float fc1, float fc2) {
  int m[3];
  float t[3];
  granule_mac<float>(G, c, pi, m, t);
  add_face_global(G, Fs_u, 0, make_stencil<float>(G, m, t, 0), fc0);
  add_face_global(G, Fs_v, 1, make_stencil<float>(G, m, t, 1), fc1);
  add_face_global(G, Fs_w, 2, make_stencil<float>(G, m, t, 2), fc2);
}

// F_s deposits spread over the lanes.  Consecutive sorted granules share
// stencil samples, and a shared-memory atomic takes one pass per lane on the
// same address, so granule g's deposits are made by lane g / W of warp g % W
// (W warps): the lanes of a warp then hold granules W apart, mostly in other
// cells.  Each thread first parks its granule's inputs (packed MAC cell,
// in-cell fractions, exchange force) in the alpha_s limbs' space, which a
// call without alpha_s leaves unused; a CTA barrier separates the two sides.
// The tile receives the same integer deposits as from the granules' own
// threads.
constexpr int kSpreadWords = 7;
constexpr int kSpreadStride = 256 + 8;  // 256 granules, bank-skewed
static_assert(kSpreadWords * kSpreadStride <= 3 * kSubTile, "spread inputs exceed the alpha_s limbs");
__device__ __forceinline__ int spread_slot(int g) { return g + (g >> 5); }

__device__ __forceinline__ void spread_put(SubTile& sh, bool valid, const int m[3], const float t[3],
                                           const float fc[3]) {
  float* s = reinterpret_cast<float*>(&sh.a[0][0]);
  const int k = spread_slot(threadIdx.x);
  s[k] = __int_as_float(valid ? (m[0] | (m[1] << 10) | (m[2] << 20)) : -1);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    s[(1 + a) * kSpreadStride + k] = t[a];
    s[(4 + a) * kSpreadStride + k] = fc[a];
  }
}

__device__ __forceinline__ void spread_deposit(SubTile& sh, const SubBox& B, const DGrid& G, float* const Fs[3],
                                               float inv_unit) {
  const int W = blockDim.x >> 5;
  const int g = lane_id() * W + (threadIdx.x >> 5);
  const float* s = reinterpret_cast<const float*>(&sh.a[0][0]);
  const int k = spread_slot(g);
  const int pm = __float_as_int(s[k]);
  if (pm < 0) return;
  const int m[3] = {pm & 1023, (pm >> 10) & 1023, pm >> 20};
  const float t[3] = {s[kSpreadStride + k], s[2 * kSpreadStride + k], s[3 * kSpreadStride + k]};
#pragma unroll
  for (int comp = 0; comp < 3; ++comp)
    sub_add_face(sh, B, G, Fs[comp], comp, make_stencil<float>(G, m, t, comp), s[(4 + comp) * kSpreadStride + k],
                 inv_unit);
}

// alpha_s deposits of one granule at its new position: into the tile when
// its stencil lies in the box, else straight to global memory (both exact).
__device__ __forceinline__ void sub_add_alpha(SubTile& sh, const SubBox& B, const DGrid& G, unsigned long long* acc,
                                              const int ia[3], const long long va[8]) {
  if (B.tile && B.holds(ia[0], ia[1], ia[2])) {
    const int e0 = B.index(ia[0], ia[1], ia[2]);
    if (!GIC_DBG_OK(G.dbg, e0 >= 0 && e0 + 1 + B.sy + B.sz < B.vol)) return;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int e = e0 + (k & 1) + ((k >> 1) & 1) * B.sy + (k >> 2) * B.sz;
      const unsigned long long v = (unsigned long long)va[k];
      atomicAdd(&sh.a[0][e], (uint32_t)(v & 0x3ffffull));
      atomicAdd(&sh.a[1][e], (uint32_t)((v >> 18) & 0x3ffffull));
      atomicAdd(&sh.a[2][e], (uint32_t)(v >> 36));
    }
  } else {
    unsigned long long* g0 = acc + sample_index(G.nx, G.ny, ia[0], ia[1], ia[2]);
    const int64_t gy = G.nx, gz = (int64_t)G.nx * G.ny;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (va[k]) atomicAdd(g0 + (k & 1) + ((k >> 1) & 1) * gy + (k >> 2) * gz, (unsigned long long)va[k]);
  }
}

// CTA-wide: the tile's non-zero entries to global memory (one atomic each).
__device__ __forceinline__ void sub_tile_flush(SubTile& sh, const SubBox& B, const DGrid& G, unsigned long long* acc,
                                               float* const Fs[3], bool do_a, bool fs_tile, float unit) {
  if (!B.tile || (!do_a && !fs_tile)) return;
  __syncthreads();
  const float rx = 1.f / (float)B.ex, rxy = 1.f / (float)B.sz;
  for (int e = threadIdx.x; e < B.vol; e += blockDim.x) {
    const int lz = (int)(((float)e + 0.5f) * rxy);
    const int r = e - lz * B.sz;
    const int ly = (int)(((float)r + 0.5f) * rx);
    const int lx = r - ly * B.ex;
    const int gx = B.b[0] + lx, gy = B.b[1] + ly, gz = B.b[2] + lz;
    if (do_a) {  // non-zero only at samples of alpha_s
      const unsigned long long a = (unsigned long long)sh.a[0][e] + ((unsigned long long)sh.a[1][e] << 18) +
                                   ((unsigned long long)sh.a[2][e] << 36);
      if (a) atomicAdd(&acc[sample_index(G.nx, G.ny, gx, gy, gz)], a);
    }
    if (fs_tile) {
#pragma unroll
      for (int comp = 0; comp < 3; ++comp) {  // non-zero only at samples of that face grid
        const int q = sh.f[comp][e];
        if (q) atomicAdd(&Fs[comp][sample_index(G.nx + (comp == 0), G.ny + (comp == 1), gx, gy, gz)],
                         (float)q * unit);
      }
    }
  }
}

template <typename T>
inline Fields<T> fields(const void* u, const void* v, const void* w, const void* p, const void* af) {
  Fields<T> F;
  F.u = (const T*)u;
  F.v = (const T*)v;
  F.w = (const T*)w;
  F.p = (const T*)p;
  F.af = (const T*)af;
  return F;
}

// scratch (optional): 32 bytes of 16-byte aligned global memory the caller
// lends for the exact totals; with it the totals come out of the conversion
// pass (one read of the grid), without it from a separate cluster pass.
int alpha_begin(double* alpha_s, int64_t ncell, double* sums2, cudaStream_t stream, void* scratch = nullptr);
// one-time per-device set-up of the exact totals' kernel (call before any capture)
int alpha_prepare();
int alpha_end(const DGrid& G, int32_t precision, double* alpha_s, int64_t ncell, double* sums2, cudaStream_t stream,
              void* scratch = nullptr);

}  // namespace gic
