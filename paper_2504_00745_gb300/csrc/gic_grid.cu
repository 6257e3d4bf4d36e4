// gic_grid.cu -- a3 G2P coupling (drag, pressure gradient, fluid acceleration,
// fluid fraction) and a5 P2G (volume fraction, exchange momentum), with
// adjoints.  One thread per granule; granules arrive Morton-sorted, so the
// lanes of a warp read and write the same few MAC cells.
#include <mutex>

#include "gic_grid.cuh"

namespace gic {

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
  int32_t ci = cell[i];
  T F[3], a[3];
  T sp = g2p_granule(G, P, Fd, ci, pi, vel[i], F, a);
  F_fl[i] = make_vec<T>(F[0], F[1], F[2]);
  a_f[i] = make_vec<T>(a[0], a[1], a[2]);
  if (afp) {
    int m[3];
    T t[3];
    granule_mac<T>(G, ci, pi, m, t);
    Stencil3<T> S = make_stencil<T>(G, m, t, 3);
    FieldLoad<T> L;
    L.f = Fd.af;
    L.nsx = G.nx;
    L.nsy = G.ny;
    L.nsz = G.nz;
    L.dbg = G.dbg;
    afp[i] = interp<T>(S, L, (T)G.inv_dx, nullptr);
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
    const pos_t<T> pi = pos[i];
    const vec_t<T> vi = vel[i];
    const vec_t<T> lF = gF[i];
    const vec_t<T> la = ga[i];
    const T l[3] = {lF.x, lF.y, lF.z};
    const T lam_a[3] = {la.x, la.y, la.z};
    int m[3];
    T t[3], gx[3] = {0, 0, 0}, gdv[3];
    const T gc = g2p_adj_granule<T>(G, P, Fd, cell[i], pi, vi, l, lam_a, gx, gdv, m, t);
    const T inv_dx = (T)G.inv_dx;
    if (galpha) {
      Stencil3<T> S = make_stencil<T>(G, m, t, 3);
      FieldLoad<T> L;
      L.f = Fd.af;
      L.nsx = G.nx;
      L.nsy = G.ny;
      L.nsz = G.nz;
      L.dbg = G.dbg;
      T gal[3];
      interp<T>(S, L, inv_dx, gal);
      T la_ = galpha[i];
      for (int b = 0; b < 3; ++b) gx[b] += la_ * gal[b];
    }
    vec_t<T> a = gpos[i];
    vec_t<T> bb = gvel[i];
    gpos[i] = make_vec<T>(a.x + gx[0], a.y + gx[1], a.z + gx[2]);
    gvel[i] = make_vec<T>(bb.x - gdv[0], bb.y - gdv[1], bb.z - gdv[2]);
    my_gc = (double)gc;
  }
  if (g_cdrag) {
    double s = block_sum(my_gc, s_red);
    if (threadIdx.x == 0) atomicAdd(g_cdrag, s);
  }
}

// ------------------------------------------------------------------ P2G

__global__ void k_zero(double* __restrict__ a, int64_t m, double* __restrict__ sums,
                       unsigned long long* __restrict__ scratch) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < m; i += stride) a[i] = 0.0;
  if (sums && blockIdx.x == 0 && threadIdx.x < 2) sums[threadIdx.x] = 0.0;
  if (scratch && blockIdx.x == 0 && threadIdx.x < 4) scratch[threadIdx.x] = 0ull;
}

__global__ void k_alpha_sum(const double* __restrict__ a, int64_t m, double dx3, double* __restrict__ sums) {
  __shared__ double s_red[32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    acc += a[i];
  double s = block_sum(acc, s_red);
  if (threadIdx.x == 0) atomicAdd(&sums[0], s * dx3);
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

constexpr int kP2GThreads = 512;

__global__ void __launch_bounds__(kP2GThreads, 2) k_p2g_f32(DGrid G, DParams<float> P, int64_t n,
                                                           const int32_t* __restrict__ cell_old,
                                                           const uint4* __restrict__ pos_old,
                                                           const int32_t* __restrict__ cell_new,
                                                           const uint4* __restrict__ pos_new,
                                                           const float4* __restrict__ fex,
                                                           double* __restrict__ alpha, float* __restrict__ Fs_u,
                                                           float* __restrict__ Fs_v, float* __restrict__ Fs_w,
                                                           double* __restrict__ sums) {
  __shared__ P2GShared sh;
  const int64_t i = blockIdx.x * (int64_t)kP2GThreads + threadIdx.x;
  const bool valid = i < n;
  const bool do_a = alpha != nullptr, do_f = Fs_u != nullptr;  // uniform over the launch
  p2g_box_init(sh);
  P2GExtent ext;
  int32_t cn = 0, co = 0;
  float fc[3] = {0.f, 0.f, 0.f};
  if (valid) {
    if (do_a) {
      cn = cell_new[i];
      ext.add_cell(G, cn);
    }
    if (do_f) {
      co = cell_old[i];
      ext.add_cell(G, co);
      float4 f = fex[i];
      fc[0] = P.exch * f.x;
      fc[1] = P.exch * f.y;
      fc[2] = P.exch * f.z;
      ext.add_force(fc);
    }
  }
  const P2GBox B = p2g_box(sh, ext, do_a, do_f);
  float* Fs[3] = {Fs_u, Fs_v, Fs_w};
  unsigned long long S = 0;
  if (valid && do_a) {
    int ia[3];
    long long va[8];
    alpha_deposits(G, cn, pos_new[i], ia, va, S);
    p2g_add_alpha(sh, B, G, (unsigned long long*)alpha, ia, va);
  }
  if (valid && do_f) {
    int m[3];
    float t[3];
    granule_mac<float>(G, co, pos_old[i], m, t);
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) p2g_add_face(sh, B, G, Fs[comp], comp, make_stencil<float>(G, m, t, comp),
                                                      fc[comp]);
  }
  p2g_flush(sh, B, G, (unsigned long long*)alpha, Fs, kP2GThreads);
  if (sums) p2g_sums(sums, (long long)S);
}

// In place: 64-bit fixed-point alpha_s -> double.
__global__ void k_alpha_finish_f32(double* __restrict__ a, int64_t m) {
  long long* ai = reinterpret_cast<long long*>(a);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = i64_scaled_to_double(ai[i], -53);
}

// ---- FP32 path: exact conservation totals ----
//
// Both totals are unsigned 128-bit integers in 2^-53 units: sum_i S_i, added
// by the scatter into the 16 bytes of sums[0..1] (p2g_sums), and sum_c
// alpha_s(c), formed here from the cells' integers before they are
// converted.  Every granule deposits exactly S_i, so the two are equal; each
// is rounded once to a double and multiplied by dx^3.  The cell total is one
// cluster of kTotalCtas CTAs: every thread sums its cells in 128 bits, a CTA
// reduces its threads', and CTA 0 reads the other CTAs' partial totals
// from their shared memory (distributed shared memory of the cluster), so
// no global scratch word is needed and the result does not depend on timing.
struct U128 {
  unsigned long long lo, hi;
};
__device__ __forceinline__ void add128(U128& a, unsigned long long lo, unsigned long long hi) {
  const unsigned long long l = a.lo + lo;
  a.hi += hi + (l < a.lo ? 1ull : 0ull);
  a.lo = l;
}

// v * 2^e2 rounded to the nearest double (ties to even), v an unsigned 128-bit integer.
__device__ __forceinline__ double u128_scaled_to_double(U128 v, int e2) {
  if (v.hi == 0 && v.lo < (1ull << 63)) return i64_scaled_to_double((long long)v.lo, e2);
  const int msb = v.hi ? 127 - __clzll(v.hi) : 63;
  const int sh = msb - 52;  // 11 .. 75 low bits are dropped
  unsigned long long m;     // v >> sh: 53 bits
  bool above, tie;          // the dropped bits against half a unit of m
  if (sh < 64) {
    m = (v.hi << (64 - sh)) | (v.lo >> sh);
    const unsigned long long rem = v.lo & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    above = rem > half;
    tie = rem == half;
  } else if (sh == 64) {
    m = v.hi;
    above = v.lo > (1ull << 63);
    tie = v.lo == (1ull << 63);
  } else {
    m = v.hi >> (sh - 64);
    const unsigned long long rh = v.hi & ((1ull << (sh - 64)) - 1ull), half = 1ull << (sh - 65);
    above = rh > half || (rh == half && v.lo != 0);
    tie = rh == half && v.lo == 0;
  }
  int e = msb;
  if (above || (tie && (m & 1ull))) {
    ++m;
    if (m == (1ull << 53)) {
      m >>= 1;
      ++e;
    }
  }
  const unsigned long long be = (unsigned long long)(e + e2 + 1023);
  return __longlong_as_double((long long)((be << 52) | (m & ((1ull << 52) - 1ull))));
}

constexpr int kTotalCtas = 16;  // one cluster of 16 CTAs (a non-portable size, enabled per device)
constexpr int kTotalThreads = 1024;
constexpr int kTotalUnroll = 4;  // 16-byte loads in flight per thread and pass

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// 64-bit load from the shared memory of CTA `rank` of the cluster, at the
// address that `p` has in this CTA's shared memory
__device__ __forceinline__ unsigned long long ld_cluster_u64(const void* p, unsigned rank) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  unsigned ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  unsigned long long v;
  asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(ra) : "memory");
  return v;
}

__global__ void __launch_bounds__(kTotalThreads)
    k_alpha_total_f32(const unsigned long long* __restrict__ a, int64_t m, int vec, double dx3,
                      double* __restrict__ sums) {
  __shared__ unsigned long long s_lo[kTotalThreads / 32], s_hi[kTotalThreads / 32];
  __shared__ unsigned long long part[2];
  U128 t{0ull, 0ull};
  const int64_t tid = blockIdx.x * (int64_t)kTotalThreads + threadIdx.x;
  const int64_t S = (int64_t)kTotalCtas * kTotalThreads;
  if (vec) {  // pairs of cells as 16-byte loads, kTotalUnroll of them in flight
    const ulonglong2* a2 = reinterpret_cast<const ulonglong2*>(a);
    const int64_t m2 = m >> 1;
    for (int64_t p = tid; p < m2; p += kTotalUnroll * S) {
      ulonglong2 v[kTotalUnroll];
#pragma unroll
      for (int u = 0; u < kTotalUnroll; ++u) v[u] = p + u * S < m2 ? __ldg(&a2[p + u * S]) : make_ulonglong2(0ull, 0ull);
#pragma unroll
      for (int u = 0; u < kTotalUnroll; ++u) {
        add128(t, v[u].x, 0ull);
        add128(t, v[u].y, 0ull);
      }
    }
    if ((m & 1) && tid == 0) add128(t, __ldg(&a[m - 1]), 0ull);
  } else {
    for (int64_t i = tid; i < m; i += S) add128(t, __ldg(&a[i]), 0ull);
  }
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long lo = __shfl_down_sync(0xffffffffu, t.lo, off);
    const unsigned long long hi = __shfl_down_sync(0xffffffffu, t.hi, off);
    add128(t, lo, hi);
  }
  if (lane_id() == 0) {
    s_lo[threadIdx.x >> 5] = t.lo;
    s_hi[threadIdx.x >> 5] = t.hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    U128 c{0ull, 0ull};
    for (int w = 0; w < kTotalThreads / 32; ++w) add128(c, s_lo[w], s_hi[w]);
    part[0] = c.lo;
    part[1] = c.hi;
  }
  cluster_sync();  // every CTA's partial total is in its shared memory
  if (cluster_rank() == 0 && threadIdx.x == 0) {
    U128 cells{0ull, 0ull};
    for (unsigned r = 0; r < kTotalCtas; ++r) add128(cells, ld_cluster_u64(&part[0], r), ld_cluster_u64(&part[1], r));
    const U128 grains{*reinterpret_cast<const unsigned long long*>(&sums[1]),
                      *reinterpret_cast<const unsigned long long*>(&sums[0])};
    sums[0] = u128_scaled_to_double(cells, -53) * dx3;
    sums[1] = u128_scaled_to_double(grains, -53) * dx3;
  }
  cluster_sync();  // no CTA leaves while CTA 0 may still read its shared memory
}

// The same totals in the in-place conversion pass, when the caller lends 32
// bytes of global scratch (zeroed with the grid): every CTA adds its cells'
// 128-bit sum into the scratch with two 64-bit atomics (the low word's carry
// read from its old value), and the CTA that takes the last ticket rounds
// both totals.  The sum is an integer, so neither the CTAs' order nor the
// timing changes it, and the cells are read once instead of twice.
constexpr int kFinishThreads = 256;
__global__ void __launch_bounds__(kFinishThreads)
    k_alpha_finish_total_f32(double* __restrict__ a, int64_t m, int vec, double dx3, double* __restrict__ sums,
                             unsigned long long* __restrict__ scratch) {
  __shared__ unsigned long long s_lo[kFinishThreads / 32], s_hi[kFinishThreads / 32];
  U128 t{0ull, 0ull};
  const int64_t tid = blockIdx.x * (int64_t)kFinishThreads + threadIdx.x;
  const int64_t S = (int64_t)gridDim.x * kFinishThreads;
  long long* ai = reinterpret_cast<long long*>(a);
  if (vec) {  // pairs of cells, 16-byte loads and stores
    longlong2* a2 = reinterpret_cast<longlong2*>(a);
    const int64_t m2 = m >> 1;
    for (int64_t p = tid; p < m2; p += S) {
      const longlong2 v = a2[p];
      add128(t, (unsigned long long)v.x, 0ull);
      add128(t, (unsigned long long)v.y, 0ull);
      reinterpret_cast<double2*>(a)[p] = make_double2(i64_scaled_to_double(v.x, -53), i64_scaled_to_double(v.y, -53));
    }
    if ((m & 1) && tid == 0) {
      const long long v = ai[m - 1];
      add128(t, (unsigned long long)v, 0ull);
      a[m - 1] = i64_scaled_to_double(v, -53);
    }
  } else {
    for (int64_t i = tid; i < m; i += S) {
      const long long v = ai[i];
      add128(t, (unsigned long long)v, 0ull);
      a[i] = i64_scaled_to_double(v, -53);
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long lo = __shfl_down_sync(0xffffffffu, t.lo, off);
    const unsigned long long hi = __shfl_down_sync(0xffffffffu, t.hi, off);
    add128(t, lo, hi);
  }
  if (lane_id() == 0) {
    s_lo[threadIdx.x >> 5] = t.lo;
    s_hi[threadIdx.x >> 5] = t.hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    U128 c{0ull, 0ull};
    for (int w = 0; w < kFinishThreads / 32; ++w) add128(c, s_lo[w], s_hi[w]);
    const unsigned long long old = atomicAdd(&scratch[0], c.lo);
    atomicAdd(&scratch[1], c.hi + (old + c.lo < old ? 1ull : 0ull));
    __threadfence();
    if (atomicAdd(&scratch[2], 1ull) == (unsigned long long)gridDim.x - 1ull) {  // the last CTA
      __threadfence();
      const U128 cells{atomicAdd(&scratch[0], 0ull), atomicAdd(&scratch[1], 0ull)};
      const U128 grains{*reinterpret_cast<const unsigned long long*>(&sums[1]),
                        *reinterpret_cast<const unsigned long long*>(&sums[0])};
      sums[0] = u128_scaled_to_double(cells, -53) * dx3;
      sums[1] = u128_scaled_to_double(grains, -53) * dx3;
    }
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
    L.nsz = G.nz;
    L.dbg = G.dbg;
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

// The cluster size of k_alpha_total_f32 is beyond the portable 8: allowed
// once per device, before any capture.
int alpha_prepare() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return set_error(GIC_ERR_CUDA, "no current device");
  std::lock_guard<std::mutex> lk(mu);
  if (!done[dev]) {
    const cudaError_t e = cudaFuncSetAttribute(k_alpha_total_f32, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return set_error(GIC_ERR_CUDA, "alpha_s totals: %s", cudaGetErrorString(e));
    done[dev] = true;
  }
  return GIC_OK;
}

static int launch_alpha_total(double* alpha_s, int64_t ncell, double dx3, double* sums2, cudaStream_t stream) {
  int rc = alpha_prepare();
  if (rc) return rc;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kTotalCtas, 1, 1);
  cfg.blockDim = dim3(kTotalThreads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kTotalCtas;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const int vec = ((uintptr_t)alpha_s % 16 == 0) ? 1 : 0;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_alpha_total_f32, (const unsigned long long*)alpha_s, ncell, vec,
                                           dx3, sums2);
  if (e != cudaSuccess) return set_error(GIC_ERR_CUDA, "alpha_s totals: %s", cudaGetErrorString(e));
  return GIC_OK;
}

// alpha_s accumulation around a P2G pass: zero the grid (and sums) before,
// then convert (FP32 fixed point -> double) or sum (FP64) after.
int alpha_begin(double* alpha_s, int64_t ncell, double* sums2, cudaStream_t stream, void* scratch) {
  k_zero<<<1184, 256, 0, stream>>>(alpha_s, ncell, sums2, sums2 ? (unsigned long long*)scratch : nullptr);
  count_launches(1);
  return GIC_OK;
}

int alpha_end(const DGrid& G, int32_t precision, double* alpha_s, int64_t ncell, double* sums2, cudaStream_t stream,
              void* scratch) {
  if (precision == GIC_FP32) {
    if (sums2 && scratch) {  // the totals inside the conversion pass
      k_alpha_finish_total_f32<<<1184, kFinishThreads, 0, stream>>>(
          alpha_s, ncell, ((uintptr_t)alpha_s % 16 == 0) ? 1 : 0, G.dx * G.dx * G.dx, sums2,
          (unsigned long long*)scratch);
      count_launches(1);
      return GIC_OK;
    }
    if (sums2) {
      if (int rc = launch_alpha_total(alpha_s, ncell, G.dx * G.dx * G.dx, sums2, stream)) return rc;
      count_launches(1);
    }
    k_alpha_finish_f32<<<1184, 256, 0, stream>>>(alpha_s, ncell);
    count_launches(1);
  } else if (sums2) {
    k_alpha_sum<<<592, 256, 0, stream>>>(alpha_s, ncell, G.dx * G.dx * G.dx, sums2);
    count_launches(1);
  }
  return GIC_OK;
}

}  // namespace gic

using namespace gic;

extern "C" int gic_g2p_couple(const GicGrid* grid, const GicParams* params, const GicGranules* s, const void* u,
                              const void* v, const void* w, const void* p, const void* alpha_f, void* F_fl, void* a_f,
                              void* alpha_f_p, gic_stream_t stream) {
  GIC_RANGE("gic_g2p_couple");
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
  GIC_RANGE("gic_g2p_couple_adj");
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
  GIC_RANGE("gic_p2g");
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
    k_zero<<<1184, 256, 0, stream>>>(alpha_s, ncell, sums2, nullptr);
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
    if (sums2) {
      if (int rc = launch_alpha_total(alpha_s, ncell, G.dx * G.dx * G.dx, sums2, stream)) return rc;
      ++launches;
    }
    k_alpha_finish_f32<<<1184, 256, 0, stream>>>(alpha_s, ncell);
    ++launches;
  } else if (sums2) {
    k_alpha_sum<<<592, 256, 0, stream>>>(alpha_s, ncell, G.dx * G.dx * G.dx, sums2);
    ++launches;
  }
  count_launches(launches);
  GIC_CHECK_LAUNCH("gic_p2g");
  return GIC_OK;
}

extern "C" int gic_p2g_alpha_atomic64(const GicGrid* grid, const GicGranules* state, double* alpha_s,
                                      gic_stream_t stream) {
  GIC_RANGE("gic_p2g_alpha_atomic64");
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if ((rc = check_granules(state, "gic_p2g_alpha_atomic64"))) return rc;
  if (state->precision != GIC_FP32)
    return set_error(GIC_ERR_INVALID, "gic_p2g_alpha_atomic64: the state must be of the FP32 path");
  if (!alpha_s) return set_error(GIC_ERR_INVALID, "gic_p2g_alpha_atomic64: alpha_s is NULL");
  const int64_t ncell = (int64_t)G.nx * G.ny * G.nz;
  k_zero<<<1184, 256, 0, stream>>>(alpha_s, ncell, nullptr, nullptr);
  int launches = 1;
  if (state->n > 0) {
    DParams<float> P{};
    k_p2g<float><<<grid_blocks(state->n, 256), 256, 0, stream>>>(G, P, state->n, state->cell,
                                                                 (const uint4*)state->pos, state->cell,
                                                                 (const uint4*)state->pos, nullptr, alpha_s, nullptr,
                                                                 nullptr, nullptr, nullptr);
    ++launches;
  }
  count_launches(launches);
  GIC_CHECK_LAUNCH("gic_p2g_alpha_atomic64");
  return GIC_OK;
}

extern "C" int gic_p2g_adj(const GicGrid* grid, const GicParams* params, const GicGranules* old_,
                           const GicGranules* new_, const void* f_ex, const double* g_alpha_s, const void* gFs_u,
                           const void* gFs_v, const void* gFs_w, void* g_pos_old, void* g_pos_new, void* g_f_ex,
                           gic_stream_t stream) {
  GIC_RANGE("gic_p2g_adj");
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
