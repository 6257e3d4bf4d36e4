// gic_grid.cu -- a3 G2P coupling (drag, pressure gradient, fluid acceleration,
// fluid fraction) and a5 P2G (volume fraction, exchange momentum), with
// adjoints.  One thread per granule; granules arrive Morton-sorted, so the
// lanes of a warp read and write the same few MAC cells.
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
  L.inv_dx = (T)G.inv_dx;
  return L;
}

// ------------------------------------------------------------------ G2P

// F_fl = c_drag pi r^2 rho_f |u_f - v| (u_f - v) - V grad p   (Sec. 3.3 Eqs. 5a, 5b)
// a_f  = g - grad p / rho_f                                   (Sec. 5.2 Eq. momentum4)
template <typename T>
__global__ void __launch_bounds__(256, 4) k_g2p(DGrid G, DParams<T> P, int64_t n, const int32_t* __restrict__ cell,
                                              const pos_t<T>* __restrict__ pos, const vec_t<T>* __restrict__ vel,
                                              Fields<T> Fd, vec_t<T>* __restrict__ F_fl, vec_t<T>* __restrict__ a_f,
                                              T* __restrict__ afp, uint32_t* status) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  pos_t<T> pi = pos[i];
  vec_t<T> vi = vel[i];
  int m[3];
  T t[3];
  granule_mac<T>(G, cell[i], pi, m, t);
  const T* uvw[3] = {Fd.u, Fd.v, Fd.w};
  T uf[3], gp[3];
  T inv_dx = (T)G.inv_dx;
#pragma unroll
  for (int comp = 0; comp < 3; ++comp) {
    Stencil3<T> S = make_stencil<T>(G, m, t, comp);
    uf[comp] = interp<T>(S, face_loader<T>(G, uvw[comp], comp), inv_dx, nullptr);
    gp[comp] = interp<T>(S, gradp_loader<T>(G, Fd.p, comp), inv_dx, nullptr);
  }
  T r = radius_of(pi);
  T V = T(4.0 / 3.0 * kPi) * r * r * r;
  T d0 = uf[0] - vi.x, d1 = uf[1] - vi.y, d2 = uf[2] - vi.z;
  T sp = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
  T cd = P.c_drag * T(kPi) * r * r * P.rho_f * sp;
  F_fl[i] = make_vec<T>(cd * d0 - V * gp[0], cd * d1 - V * gp[1], cd * d2 - V * gp[2]);
  if (P.rho_f > T(0))
    a_f[i] = make_vec<T>(P.g[0] - gp[0] * P.inv_rho_f, P.g[1] - gp[1] * P.inv_rho_f, P.g[2] - gp[2] * P.inv_rho_f);
  else
    a_f[i] = make_vec<T>(P.g[0], P.g[1], P.g[2]);
  if (afp) {
    Stencil3<T> S = make_stencil<T>(G, m, t, 3);
    FieldLoad<T> L;
    L.f = Fd.af;
    L.nsx = G.nx;
    L.nsy = G.ny;
    afp[i] = interp<T>(S, L, inv_dx, nullptr);
  }
  if (!isfinite(sp)) raise_status(status, GIC_STATUS_NONFINITE);
}

template <typename T>
__global__ void __launch_bounds__(256) k_g2p_adj(DGrid G, DParams<T> P, int64_t n, const int32_t* __restrict__ cell,
                                                  const pos_t<T>* __restrict__ pos, const vec_t<T>* __restrict__ vel,
                                                  Fields<T> Fd, const vec_t<T>* __restrict__ gF,
                                                  const vec_t<T>* __restrict__ ga, const T* __restrict__ galpha,
                                                  vec_t<T>* __restrict__ gpos, vec_t<T>* __restrict__ gvel,
                                                  double* __restrict__ g_cdrag) {
  __shared__ double s_red[32];
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double my_gc = 0.0;
  if (i < n) {
    pos_t<T> pi = pos[i];
    vec_t<T> vi = vel[i];
    int m[3];
    T t[3];
    granule_mac<T>(G, cell[i], pi, m, t);
    const T* uvw[3] = {Fd.u, Fd.v, Fd.w};
    T uf[3], gu[3][3], gp[3], ggp[3][3];
    T inv_dx = (T)G.inv_dx;
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      Stencil3<T> S = make_stencil<T>(G, m, t, comp);
      uf[comp] = interp<T>(S, face_loader<T>(G, uvw[comp], comp), inv_dx, gu[comp]);
      gp[comp] = interp<T>(S, gradp_loader<T>(G, Fd.p, comp), inv_dx, ggp[comp]);
    }
    T r = radius_of(pi);
    T V = T(4.0 / 3.0 * kPi) * r * r * r;
    T dv[3] = {uf[0] - vi.x, uf[1] - vi.y, uf[2] - vi.z};
    T sp = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    T k = P.c_drag * T(kPi) * r * r * P.rho_f;
    vec_t<T> lF = gF[i];
    vec_t<T> la = ga[i];
    T l[3] = {lF.x, lF.y, lF.z};
    T lam_a[3] = {la.x, la.y, la.z};
    T dvl = dv[0] * l[0] + dv[1] * l[1] + dv[2] * l[2];
    // d/d dv of k |dv| dv . l = k (|dv| l + (dv . l) dv / |dv|)
    T gdv[3];
    for (int a = 0; a < 3; ++a) gdv[a] = sp > T(0) ? k * (sp * l[a] + dvl * dv[a] / sp) : T(0);
    T gx[3] = {0, 0, 0};
    for (int comp = 0; comp < 3; ++comp) {
      T ggrad = -V * l[comp] - P.inv_rho_f * lam_a[comp];  // upstream of grad p component
      for (int b = 0; b < 3; ++b) gx[b] += gdv[comp] * gu[comp][b] + ggrad * ggp[comp][b];
    }
    if (galpha) {
      Stencil3<T> S = make_stencil<T>(G, m, t, 3);
      FieldLoad<T> L;
      L.f = Fd.af;
      L.nsx = G.nx;
      L.nsy = G.ny;
      T gal[3];
      interp<T>(S, L, inv_dx, gal);
      T la_ = galpha[i];
      for (int b = 0; b < 3; ++b) gx[b] += la_ * gal[b];
    }
    vec_t<T> a = gpos[i];
    vec_t<T> bb = gvel[i];
    gpos[i] = make_vec<T>(a.x + gx[0], a.y + gx[1], a.z + gx[2]);
    gvel[i] = make_vec<T>(bb.x - gdv[0], bb.y - gdv[1], bb.z - gdv[2]);
    my_gc = (double)(T(kPi) * r * r * P.rho_f * sp * dvl);
  }
  if (g_cdrag) {
    double s = block_sum(my_gc, s_red);
    if (threadIdx.x == 0) atomicAdd(g_cdrag, s);
  }
}

// ------------------------------------------------------------------ P2G

__global__ void k_zero(double* __restrict__ a, int64_t m, double* __restrict__ sums) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < m; i += stride) a[i] = 0.0;
  if (sums && blockIdx.x == 0 && threadIdx.x < 2) sums[threadIdx.x] = 0.0;
}

__global__ void k_alpha_sum(const double* __restrict__ a, int64_t m, double dx3, double* __restrict__ sums) {
  __shared__ double s_red[32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    acc += a[i];
  double s = block_sum(acc, s_red);
  if (threadIdx.x == 0) atomicAdd(&sums[0], s * dx3);
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

// FP64 path: alpha_s(c) = sum_i V_i N(x'_i - x_c) / dx^3 at the new positions, FP64
// weights and FP64 atomics;
// F_s(face) += exch * f_ex_i N(x_i - x_face) at the old positions, with a
// warp-segmented pre-sum over lanes that share the stencil's base sample.
template <typename T>
__global__ void __launch_bounds__(256) k_p2g(DGrid G, DParams<T> P, int64_t n, const int32_t* __restrict__ cell_old,
                                              const pos_t<T>* __restrict__ pos_old,
                                              const int32_t* __restrict__ cell_new,
                                              const pos_t<T>* __restrict__ pos_new, const vec_t<T>* __restrict__ fex,
                                              double* __restrict__ alpha, T* __restrict__ Fs_u, T* __restrict__ Fs_v,
                                              T* __restrict__ Fs_w, double* __restrict__ sums) {
  __shared__ double s_red[32];
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  bool valid = i < n;
  double Vi = 0.0;
  if (valid && alpha) {
    pos_t<T> pn = pos_new[i];
    double r = (double)radius_of(pn);
    Vi = 4.0 / 3.0 * kPi * r * r * r;
    int m[3];
    double t[3];
    granule_mac_fp64(G, cell_new[i], pn, m, t);
    Stencil3<double> S = make_stencil<double>(G, m, t, 3);
    double s = Vi * G.inv_dx * G.inv_dx * G.inv_dx;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        double wyz = (b ? S.w[1] : 1.0 - S.w[1]) * (c ? S.w[2] : 1.0 - S.w[2]) * s;
        int64_t row = sample_index(G.nx, G.ny, S.i0[0], S.i0[1] + b, S.i0[2] + c);
        atomicAdd(&alpha[row], (1.0 - S.w[0]) * wyz);
        atomicAdd(&alpha[row + 1], S.w[0] * wyz);
      }
  }
  bool do_fs = Fs_u != nullptr;  // uniform over the launch
  if (do_fs) {
    int m[3] = {0, 0, 0};
    T t[3] = {0, 0, 0};
    vec_t<T> f = make_vec<T>(0, 0, 0);
    if (valid) {
      granule_mac<T>(G, cell_old[i], pos_old[i], m, t);
      f = fex[i];
    }
    T* Fs[3] = {Fs_u, Fs_v, Fs_w};
    T fv[3] = {P.exch * f.x, P.exch * f.y, P.exch * f.z};
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      Stencil3<T> S = make_stencil<T>(G, m, t, comp);
      unsigned key = valid ? (unsigned)base_index(S) : 0xffffffffu - (unsigned)lane_id();
      int end = run_end(key);
      bool head = run_head(key);
      T val[8];
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int a = 0; a < 2; ++a) {
            T w = (a ? S.w[0] : T(1) - S.w[0]) * (b ? S.w[1] : T(1) - S.w[1]) * (c ? S.w[2] : T(1) - S.w[2]);
            val[a + 2 * b + 4 * c] = seg_sum(valid ? w * fv[comp] : T(0), end);
          }
      if (valid && head) {
        int nsx = S.ns[0], nsy = S.ns[1];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int b = 0; b < 2; ++b) {
            int64_t row = sample_index(nsx, nsy, S.i0[0], S.i0[1] + b, S.i0[2] + c);
            atomicAdd(&Fs[comp][row], val[2 * b + 4 * c]);
            atomicAdd(&Fs[comp][row + 1], val[1 + 2 * b + 4 * c]);
          }
      }
    }
  }
  if (sums) {
    double s = block_sum(Vi, s_red);
    if (threadIdx.x == 0) atomicAdd(&sums[1], s);
  }
}

// ---- FP32 path scatter ----
//
// v * 2^e2 rounded to double with integer operations only (the FP64 pipe is
// the slowest unit of this GPU)
__device__ __forceinline__ double i64_scaled_to_double(long long v, int e2) {
  if (v == 0) return 0.0;
  unsigned long long sign = v < 0 ? (1ull << 63) : 0ull;
  unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  int msb = 63 - __clzll(a);
  unsigned long long m;
  if (msb > 52) {
    int sh = msb - 52;
    unsigned long long rem = a & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    m = a >> sh;
    if (rem > half || (rem == half && (m & 1ull))) {
      ++m;
      if (m == (1ull << 53)) {
        m >>= 1;
        ++msb;
      }
    }
  } else {
    m = a << (52 - msb);
  }
  unsigned long long e = (unsigned long long)(msb + e2 + 1023);
  return __longlong_as_double((long long)(sign | (e << 52) | (m & ((1ull << 52) - 1ull))));
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

// FP32 path of P2G.  One CTA takes 512 consecutive granules of the
// Morton-sorted state, which occupy a compact block of MAC cells.  When the
// samples they may touch fit a kP2GTile-entry box, every deposit goes to
// shared-memory copies of alpha_s and the three F_s grids over that box,
// held as 32-bit integer limbs (32-bit shared integer atomics run at full
// rate even when lanes collide, unlike float or 64-bit ones), and the box's
// non-zero entries then go to global memory with one atomic each; otherwise
// every deposit is a global atomic.
//   alpha_s: a deposit (< 2^54 units of 2^-53) is split into three 18-bit
//   limbs, so up to 2^14 deposits per entry add without overflow -- exact.
//   F_s: a deposit d is rounded to a multiple of u = M 2^-30, M the CTA's
//   largest |exch f_ex| component, and q = d / u (|q| <= 2^30) is split into
//   a signed high and an unsigned low 15-bit limb; the limb sums are exact,
//   so the only rounding besides the float product d is the 2^-30 M grid.
// alpha_s stays 64-bit fixed point (exact, order-independent) until
// k_alpha_finish_f32.
constexpr int kP2GThreads = 512;
constexpr int kP2GTile = 1024;

__global__ void __launch_bounds__(kP2GThreads, 2) k_p2g_f32(DGrid G, DParams<float> P, int64_t n,
                                                           const int32_t* __restrict__ cell_old,
                                                           const uint4* __restrict__ pos_old,
                                                           const int32_t* __restrict__ cell_new,
                                                           const uint4* __restrict__ pos_new,
                                                           const float4* __restrict__ fex,
                                                           double* __restrict__ alpha, float* __restrict__ Fs_u,
                                                           float* __restrict__ Fs_v, float* __restrict__ Fs_w,
                                                           double* __restrict__ sums) {
  __shared__ uint32_t s_a[3][kP2GTile];
  __shared__ int32_t s_fh[3][kP2GTile];
  __shared__ uint32_t s_fl[3][kP2GTile];
  __shared__ int s_lo[3], s_hi[3];
  __shared__ unsigned s_M;
  const int64_t i = blockIdx.x * (int64_t)kP2GThreads + threadIdx.x;
  const bool valid = i < n;
  const bool do_a = alpha != nullptr, do_f = Fs_u != nullptr;  // uniform over the launch
  if (threadIdx.x < 3) {
    s_lo[threadIdx.x] = INT_MAX;
    s_hi[threadIdx.x] = INT_MIN;
  }
  if (threadIdx.x == 0) s_M = 0u;

  // box of every sample this CTA may touch: a stencil's base is the MAC cell
  // m or m - 1 on each axis, and it reaches one sample further
  int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
  int32_t cn = 0, co = 0;
  float fc[3] = {0.f, 0.f, 0.f};
  float M = 0.f;
  if (valid) {
    if (do_a) cn = cell_new[i];
    if (do_f) {
      co = cell_old[i];
      float4 f = fex[i];
      fc[0] = P.exch * f.x;
      fc[1] = P.exch * f.y;
      fc[2] = P.exch * f.z;
      M = fmaxf(fabsf(fc[0]), fmaxf(fabsf(fc[1]), fabsf(fc[2])));
      if (!(M <= 3.0e38f)) M = INFINITY;  // NaN or inf: no fixed-point grid for this CTA
    }
    int32_t cs[2] = {do_a ? cn : co, do_f ? co : cn};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      int c3[3] = {cell_x(cs[h]), cell_y(cs[h]), cell_z(cs[h])};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        int m = mac_of(G, c3[a]);
        lo[a] = min(lo[a], m - 1);
        hi[a] = max(hi[a], m + 1);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int l = __reduce_min_sync(0xffffffffu, lo[a]);
    int h = __reduce_max_sync(0xffffffffu, hi[a]);
    if (lane_id() == 0) {
      atomicMin(&s_lo[a], l);
      atomicMax(&s_hi[a], h);
    }
  }
  if (do_f) {  // non-negative floats order like their bit patterns
    unsigned mb = __reduce_max_sync(0xffffffffu, __float_as_uint(M));
    if (lane_id() == 0) atomicMax(&s_M, mb);
  }
  __syncthreads();
  const int bx = max(s_lo[0], 0), by = max(s_lo[1], 0), bz = max(s_lo[2], 0);
  const int ex = s_hi[0] - bx + 1, ey = s_hi[1] - by + 1, ez = s_hi[2] - bz + 1;
  // every CTA holds at least one granule, so the box is not empty
  const bool tile = (int64_t)ex * ey * ez <= kP2GTile;
  const float Mc = __uint_as_float(s_M);
  const bool ftile = tile && Mc >= 1e-30f && Mc <= 3.0e38f;  // F_s through the fixed-point tile
  const float unit = Mc * 0x1p-30f, inv_unit = ftile ? 0x1p30f / Mc : 0.f;
  const int vol = tile ? ex * ey * ez : 0;
  const int sy = ex, sz = ex * ey;
  for (int e = threadIdx.x; e < vol; e += kP2GThreads) {
    if (do_a) s_a[0][e] = s_a[1][e] = s_a[2][e] = 0u;
    if (ftile) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        s_fh[c][e] = 0;
        s_fl[c][e] = 0u;
      }
    }
  }
  if (tile) __syncthreads();

  unsigned long long S = 0;
  if (valid && do_a) {
    int ia[3];
    long long va[8];
    alpha_deposits(G, cn, pos_new[i], ia, va, S);
    if (tile) {
      const int e0 = (ia[0] - bx) + sy * (ia[1] - by) + sz * (ia[2] - bz);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int e = e0 + (k & 1) + ((k >> 1) & 1) * sy + (k >> 2) * sz;
        const unsigned long long v = (unsigned long long)va[k];
        atomicAdd(&s_a[0][e], (uint32_t)(v & 0x3ffffull));
        atomicAdd(&s_a[1][e], (uint32_t)((v >> 18) & 0x3ffffull));
        atomicAdd(&s_a[2][e], (uint32_t)(v >> 36));
      }
    } else {
      unsigned long long* g0 = (unsigned long long*)alpha + sample_index(G.nx, G.ny, ia[0], ia[1], ia[2]);
      const int64_t gy = G.nx, gz = (int64_t)G.nx * G.ny;
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (va[k]) atomicAdd(g0 + (k & 1) + ((k >> 1) & 1) * gy + (k >> 2) * gz, (unsigned long long)va[k]);
    }
  }
  if (valid && do_f) {
    int m[3];
    float t[3];
    granule_mac<float>(G, co, pos_old[i], m, t);
    float* Fs[3] = {Fs_u, Fs_v, Fs_w};
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      Stencil3<float> St = make_stencil<float>(G, m, t, comp);
      const float wx = St.w[0], wy = St.w[1], wz = St.w[2];
      const float fx0 = (1.f - wx) * fc[comp], fx1 = wx * fc[comp];
      const float wyz[4] = {(1.f - wy) * (1.f - wz), wy * (1.f - wz), (1.f - wy) * wz, wy * wz};
      if (ftile) {
        const int e0 = (St.i0[0] - bx) + sy * (St.i0[1] - by) + sz * (St.i0[2] - bz);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int q = __float2int_rn(((k & 1) ? fx1 : fx0) * wyz[k >> 1] * inv_unit);
          const int e = e0 + (k & 1) + ((k >> 1) & 1) * sy + (k >> 2) * sz;
          atomicAdd(&s_fh[comp][e], q >> 15);
          atomicAdd(&s_fl[comp][e], (uint32_t)(q & 0x7fff));
        }
      } else {
        const int nsx = G.nx + (comp == 0), nsy = G.ny + (comp == 1);
        float* g0 = Fs[comp] + sample_index(nsx, nsy, St.i0[0], St.i0[1], St.i0[2]);
        const int64_t gy = nsx, gz = (int64_t)nsx * nsy;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float d = ((k & 1) ? fx1 : fx0) * wyz[k >> 1];
          if (d != 0.f) atomicAdd(g0 + (k & 1) + ((k >> 1) & 1) * gy + (k >> 2) * gz, d);
        }
      }
    }
  }

  if (tile) {  // the box's non-zero entries to global memory
    __syncthreads();
    unsigned long long* acc = (unsigned long long*)alpha;
    float* Fs[3] = {Fs_u, Fs_v, Fs_w};
    // e = lx + ex (ly + ey lz); (e + 1/2) / d stays >= 1/(2 d) away from an
    // integer, far beyond the float error for e, d <= 1024
    const float rx = 1.f / (float)ex, rxy = 1.f / (float)sz;
    for (int e = threadIdx.x; e < vol; e += kP2GThreads) {
      int lz = (int)(((float)e + 0.5f) * rxy);
      int r = e - lz * sz;
      int ly = (int)(((float)r + 0.5f) * rx);
      int lx = r - ly * ex;
      int gx = bx + lx, gy = by + ly, gz = bz + lz;
      if (do_a) {
        unsigned long long a = (unsigned long long)s_a[0][e] + ((unsigned long long)s_a[1][e] << 18) +
                               ((unsigned long long)s_a[2][e] << 36);
        if (a) atomicAdd(&acc[sample_index(G.nx, G.ny, gx, gy, gz)], a);
      }
      if (ftile) {
#pragma unroll
        for (int comp = 0; comp < 3; ++comp) {
          long long q = (long long)s_fh[comp][e] * (1ll << 15) + (long long)s_fl[comp][e];
          if (q) atomicAdd(&Fs[comp][sample_index(G.nx + (comp == 0), G.ny + (comp == 1), gx, gy, gz)],
                           (float)q * unit);
        }
      }
    }
  }

  if (sums) {  // exact integer warp totals of sum_i V_i / dx^3; every granule deposits exactly S
    long long v = (long long)S;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane_id() == 0 && v != 0) {
      atomicAdd((unsigned long long*)&sums[0], (unsigned long long)v);
      atomicAdd((unsigned long long*)&sums[1], (unsigned long long)v);
    }
  }
}

// In place: 64-bit fixed-point alpha_s -> double; sums[0] and sums[1] (integer
// totals of the deposits and of V_i / dx^3) -> sum_c alpha_s dx^3, sum_i V_i.
__global__ void k_alpha_finish_f32(double* __restrict__ a, int64_t m, double dx3, double* __restrict__ sums) {
  long long* ai = reinterpret_cast<long long*>(a);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = i64_scaled_to_double(ai[i], -53);
  if (sums && blockIdx.x == 0 && threadIdx.x == 0) {  // both sums were accumulated as 2^-53 integers
    long long tot = *reinterpret_cast<long long*>(&sums[0]);
    long long vol = *reinterpret_cast<long long*>(&sums[1]);
    sums[0] = i64_scaled_to_double(tot, -53) * dx3;
    sums[1] = i64_scaled_to_double(vol, -53) * dx3;
  }
}

// Adjoint of P2G: G2P-shaped gathers of the grid gradients.
template <typename T>
__global__ void __launch_bounds__(256) k_p2g_adj(DGrid G, DParams<T> P, int64_t n,
                                                  const int32_t* __restrict__ cell_old,
                                                  const pos_t<T>* __restrict__ pos_old,
                                                  const int32_t* __restrict__ cell_new,
                                                  const pos_t<T>* __restrict__ pos_new,
                                                  const vec_t<T>* __restrict__ fex, const double* __restrict__ galpha,
                                                  const T* __restrict__ gu, const T* __restrict__ gv,
                                                  const T* __restrict__ gw, vec_t<T>* __restrict__ gpos_old,
                                                  vec_t<T>* __restrict__ gpos_new, vec_t<T>* __restrict__ gfex) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  T inv_dx = (T)G.inv_dx;
  if (galpha && gpos_new) {
    pos_t<T> pn = pos_new[i];
    double r = (double)radius_of(pn);
    double s = 4.0 / 3.0 * kPi * r * r * r * G.inv_dx * G.inv_dx * G.inv_dx;
    int m[3];
    double t[3];
    granule_mac_fp64(G, cell_new[i], pn, m, t);
    Stencil3<double> S = make_stencil<double>(G, m, t, 3);
    FieldLoad<double> L;
    L.f = galpha;
    L.nsx = G.nx;
    L.nsy = G.ny;
    double g[3];
    interp<double>(S, L, G.inv_dx, g);
    vec_t<T> a = gpos_new[i];
    gpos_new[i] = make_vec<T>(a.x + (T)(s * g[0]), a.y + (T)(s * g[1]), a.z + (T)(s * g[2]));
  }
  const T* gF[3] = {gu, gv, gw};
  vec_t<T> f = fex[i];
  T fv[3] = {f.x, f.y, f.z};
  T gf[3] = {0, 0, 0}, gx[3] = {0, 0, 0};
  int m[3];
  T t[3];
  granule_mac<T>(G, cell_old[i], pos_old[i], m, t);
#pragma unroll
  for (int comp = 0; comp < 3; ++comp) {
    if (!gF[comp]) continue;
    Stencil3<T> S = make_stencil<T>(G, m, t, comp);
    T g[3];
    T val = interp<T>(S, face_loader<T>(G, gF[comp], comp), inv_dx, g);
    gf[comp] = P.exch * val;
    for (int b = 0; b < 3; ++b) gx[b] += P.exch * fv[comp] * g[b];
  }
  if (gfex) gfex[i] = make_vec<T>(gf[0], gf[1], gf[2]);
  if (gpos_old) {
    vec_t<T> a = gpos_old[i];
    gpos_old[i] = make_vec<T>(a.x + gx[0], a.y + gx[1], a.z + gx[2]);
  }
}

template <typename T>
static Fields<T> fields(const void* u, const void* v, const void* w, const void* p, const void* af) {
  Fields<T> F;
  F.u = (const T*)u;
  F.v = (const T*)v;
  F.w = (const T*)w;
  F.p = (const T*)p;
  F.af = (const T*)af;
  return F;
}

}  // namespace gic

using namespace gic;

extern "C" int gic_g2p_couple(const GicGrid* grid, const GicParams* params, const GicGranules* s, const void* u,
                              const void* v, const void* w, const void* p, const void* alpha_f, void* F_fl, void* a_f,
                              void* alpha_f_p, gic_stream_t stream) {
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if ((rc = check_granules(s, "gic_g2p_couple"))) return rc;
  if (s->n == 0) return GIC_OK;
  if (!u || !v || !w || !p || !F_fl || !a_f) return set_error(GIC_ERR_INVALID, "gic_g2p_couple: null array");
  if (alpha_f_p && !alpha_f) return set_error(GIC_ERR_INVALID, "gic_g2p_couple: alpha_f_p needs alpha_f");
  if ((rc = check_vecs(s->precision, "gic_g2p_couple", {F_fl, a_f}))) return rc;
  if (s->precision == GIC_FP32) {
    DParams<float> P;
    if ((rc = make_params(params, &P))) return rc;
    k_g2p<float><<<grid_blocks(s->n, 256), 256, 0, stream>>>(G, P, s->n, s->cell, (const uint4*)s->pos,
                                                              (const float4*)s->vel, fields<float>(u, v, w, p, alpha_f),
                                                              (float4*)F_fl, (float4*)a_f, (float*)alpha_f_p,
                                                              status_word());
  } else {
    DParams<double> P;
    if ((rc = make_params(params, &P))) return rc;
    k_g2p<double><<<grid_blocks(s->n, 256), 256, 0, stream>>>(
        G, P, s->n, s->cell, (const d4*)s->pos, (const d4*)s->vel, fields<double>(u, v, w, p, alpha_f), (d4*)F_fl,
        (d4*)a_f, (double*)alpha_f_p, status_word());
  }
  count_launches(1);
  GIC_CHECK_LAUNCH("gic_g2p_couple");
  return GIC_OK;
}

extern "C" int gic_g2p_couple_adj(const GicGrid* grid, const GicParams* params, const GicGranules* s, const void* u,
                                  const void* v, const void* w, const void* p, const void* alpha_f, const void* gF_fl,
                                  const void* ga_f, const void* galpha_f_p, void* g_pos, void* g_vel,
                                  double* g_cdrag, gic_stream_t stream) {
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if ((rc = check_granules(s, "gic_g2p_couple_adj"))) return rc;
  if (s->n == 0) return GIC_OK;
  if (!u || !v || !w || !p || !gF_fl || !ga_f || !g_pos || !g_vel)
    return set_error(GIC_ERR_INVALID, "gic_g2p_couple_adj: null array");
  if (galpha_f_p && !alpha_f) return set_error(GIC_ERR_INVALID, "gic_g2p_couple_adj: galpha_f_p needs alpha_f");
  if ((rc = check_vecs(s->precision, "gic_g2p_couple_adj", {gF_fl, ga_f, g_pos, g_vel}))) return rc;
  if (s->precision == GIC_FP32) {
    DParams<float> P;
    if ((rc = make_params(params, &P))) return rc;
    k_g2p_adj<float><<<grid_blocks(s->n, 256), 256, 0, stream>>>(
        G, P, s->n, s->cell, (const uint4*)s->pos, (const float4*)s->vel, fields<float>(u, v, w, p, alpha_f),
        (const float4*)gF_fl, (const float4*)ga_f, (const float*)galpha_f_p, (float4*)g_pos, (float4*)g_vel,
        g_cdrag);
  } else {
    DParams<double> P;
    if ((rc = make_params(params, &P))) return rc;
    k_g2p_adj<double><<<grid_blocks(s->n, 256), 256, 0, stream>>>(
        G, P, s->n, s->cell, (const d4*)s->pos, (const d4*)s->vel, fields<double>(u, v, w, p, alpha_f),
        (const d4*)gF_fl, (const d4*)ga_f, (const double*)galpha_f_p, (d4*)g_pos, (d4*)g_vel, g_cdrag);
  }
  count_launches(1);
  GIC_CHECK_LAUNCH("gic_g2p_couple_adj");
  return GIC_OK;
}

extern "C" int gic_p2g(const GicGrid* grid, const GicParams* params, const GicGranules* old_, const GicGranules* new_,
                       const void* f_ex, double* alpha_s, void* Fs_u, void* Fs_v, void* Fs_w, double* sums2,
                       gic_stream_t stream) {
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if ((rc = check_granules(old_, "gic_p2g old"))) return rc;
  if ((rc = check_granules(new_, "gic_p2g new"))) return rc;
  if (old_->n != new_->n || old_->precision != new_->precision)
    return set_error(GIC_ERR_INVALID, "gic_p2g: old/new differ in size or precision");
  bool fs = Fs_u || Fs_v || Fs_w;
  if (fs && !(Fs_u && Fs_v && Fs_w)) return set_error(GIC_ERR_INVALID, "gic_p2g: give all three F_s arrays or none");
  if (fs && !f_ex && old_->n > 0) return set_error(GIC_ERR_INVALID, "gic_p2g: F_s needs f_ex");
  if (sums2 && !alpha_s) return set_error(GIC_ERR_INVALID, "gic_p2g: sums2 needs alpha_s");
  if ((rc = check_vecs(old_->precision, "gic_p2g", {f_ex}))) return rc;
  int64_t n = old_->n;
  int64_t ncell = (int64_t)G.nx * G.ny * G.nz;
  int launches = 0;
  if (alpha_s) {
    k_zero<<<1184, 256, 0, stream>>>(alpha_s, ncell, sums2);
    ++launches;
  }
  if (n > 0 && (alpha_s || fs)) {
    if (old_->precision == GIC_FP32) {
      DParams<float> P;
      if ((rc = make_params(params, &P))) return rc;
      k_p2g_f32<<<grid_blocks(n, kP2GThreads), kP2GThreads, 0, stream>>>(
          G, P, n, old_->cell, (const uint4*)old_->pos, new_->cell, (const uint4*)new_->pos, (const float4*)f_ex,
          alpha_s, (float*)Fs_u, (float*)Fs_v, (float*)Fs_w, sums2);
    } else {
      DParams<double> P;
      if ((rc = make_params(params, &P))) return rc;
      k_p2g<double><<<grid_blocks(n, 256), 256, 0, stream>>>(
          G, P, n, old_->cell, (const d4*)old_->pos, new_->cell, (const d4*)new_->pos, (const d4*)f_ex, alpha_s,
          (double*)Fs_u, (double*)Fs_v, (double*)Fs_w, sums2);
    }
    ++launches;
  }
  if (alpha_s && old_->precision == GIC_FP32) {
    // the FP32 path accumulated 64-bit fixed point: convert in place
    k_alpha_finish_f32<<<1184, 256, 0, stream>>>(alpha_s, ncell, G.dx * G.dx * G.dx, sums2);
    ++launches;
  } else if (sums2) {
    k_alpha_sum<<<592, 256, 0, stream>>>(alpha_s, ncell, G.dx * G.dx * G.dx, sums2);
    ++launches;
  }
  count_launches(launches);
  GIC_CHECK_LAUNCH("gic_p2g");
  return GIC_OK;
}

extern "C" int gic_p2g_adj(const GicGrid* grid, const GicParams* params, const GicGranules* old_,
                           const GicGranules* new_, const void* f_ex, const double* g_alpha_s, const void* gFs_u,
                           const void* gFs_v, const void* gFs_w, void* g_pos_old, void* g_pos_new, void* g_f_ex,
                           gic_stream_t stream) {
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if ((rc = check_granules(old_, "gic_p2g_adj old"))) return rc;
  if ((rc = check_granules(new_, "gic_p2g_adj new"))) return rc;
  if (old_->n != new_->n || old_->precision != new_->precision)
    return set_error(GIC_ERR_INVALID, "gic_p2g_adj: old/new differ in size or precision");
  int64_t n = old_->n;
  if (n == 0) return GIC_OK;
  if (!f_ex) return set_error(GIC_ERR_INVALID, "gic_p2g_adj: f_ex is NULL");
  if ((rc = check_vecs(old_->precision, "gic_p2g_adj", {f_ex, g_pos_old, g_pos_new, g_f_ex}))) return rc;
  if (old_->precision == GIC_FP32) {
    DParams<float> P;
    if ((rc = make_params(params, &P))) return rc;
    k_p2g_adj<float><<<grid_blocks(n, 256), 256, 0, stream>>>(
        G, P, n, old_->cell, (const uint4*)old_->pos, new_->cell, (const uint4*)new_->pos, (const float4*)f_ex,
        g_alpha_s, (const float*)gFs_u, (const float*)gFs_v, (const float*)gFs_w, (float4*)g_pos_old,
        (float4*)g_pos_new, (float4*)g_f_ex);
  } else {
    DParams<double> P;
    if ((rc = make_params(params, &P))) return rc;
    k_p2g_adj<double><<<grid_blocks(n, 256), 256, 0, stream>>>(
        G, P, n, old_->cell, (const d4*)old_->pos, new_->cell, (const d4*)new_->pos, (const d4*)f_ex, g_alpha_s,
        (const double*)gFs_u, (const double*)gFs_v, (const double*)gFs_w, (d4*)g_pos_old, (d4*)g_pos_new,
        (d4*)g_f_ex);
  }
  count_launches(1);
  GIC_CHECK_LAUNCH("gic_p2g_adj");
  return GIC_OK;
}
