// gic_internal.cuh -- device/host helpers shared by the library's translation
// units (not installed; the public interface is include/gic.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <initializer_list>
#include <cmath>

#include <nvtx3/nvToolsExt.h>

#include "gic.h"

namespace gic {

// A named range around an entry point for timeline tools (NVTX; costs a
// function-pointer test when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define GIC_RANGE(name) ::gic::NvtxRange gic_nvtx_range_(name)

// ----------------------------------------------------------------- constants

constexpr int kFracBits = 30;                    // fixed-point offset bits (FP32 path)
constexpr uint32_t kFracOne = 1u << kFracBits;
constexpr uint32_t kFracMask = kFracOne - 1u;
constexpr int kCellBits = 10;                    // packed cell: cx | cy << 10 | cz << 20
constexpr int kMaxCellsPerAxis = 1 << kCellBits;
constexpr double kPi = 3.14159265358979323846;

struct alignas(32) d4 {
  double x, y, z, w;
};

// ----------------------------------------------------------------- host side

// error reporting (thread-local text) and launch accounting
int set_error(int code, const char* fmt, ...);
void count_launches(int64_t k);
void set_capturing(bool on);
int wait_stream(cudaStream_t stream, int64_t timeout_ms, const char* what);
uint32_t* status_word();  // device address of the sticky status word (current device)

#define GIC_CHECK_LAUNCH(what)                                                                           \
  do {                                                                                                   \
    cudaError_t e_ = cudaGetLastError();                                                                 \
    if (e_ != cudaSuccess) return ::gic::set_error(GIC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e_)); \
  } while (0)

// Derived grid constants, passed to kernels by value.
struct DGrid {
  int nx, ny, nz, k;
  int nc[3];       // contact cells per axis
  uint32_t kmul;   // floor(c / k) == (c * kmul) >> 20 for c < 1024
  double dx, hc, inv_dx, inv_hc;
  double origin[3];
  double unit, inv_unit;  // h_c 2^-30 and its inverse
  double inv_k_frac;      // 1 / (k 2^30)
  float dx_f, hc_f, inv_dx_f, inv_hc_f, unit_f, inv_unit_f, inv_k_f;
  float s_hi, s_lo;  // 2^30 / h_c as an unevaluated float pair (hi + lo)
  float s2_margin;   // s_hi^2 (1 + 4e-6): contact pre-test threshold factor
  unsigned long long kinv64;  // ceil(2^64 / k) for k > 1 (fixed-point division by k), 0 for k = 1
  double vol_fx;              // (4/3) pi / dx^3 * 2^53: granule volume fraction in 2^-53 units per r^3
  float vol_fx_hi, vol_fx_lo;  // the same as an unevaluated float pair
  uint32_t* dbg;               // debug builds: the status word the index checks flag (null otherwise)
};

// The grid's h_c and 1 / dx in each precision: the FP32 path reads the float
// copies (a double-to-float conversion runs on the FP64 pipe, a small
// fraction of the FP32 rate on this GPU).
template <typename T>
__device__ __forceinline__ T grid_inv_dx(const DGrid& G) {
  if constexpr (sizeof(T) == 4) return G.inv_dx_f;
  else return G.inv_dx;
}
template <typename T>
__device__ __forceinline__ T grid_hc(const DGrid& G) {
  if constexpr (sizeof(T) == 4) return G.hc_f;
  else return G.hc;
}

// Debug builds (compiled with GIC_DEBUG): device-side checks that an index
// lies inside its array.  A failed check sets GIC_STATUS_DEBUG_INDEX in the
// status word and the caller skips the access -- no trap, no assert.
// Release builds compile the checks away.
__device__ __forceinline__ bool dbg_fail(uint32_t* dbg) {
  if (dbg) atomicOr(dbg, (uint32_t)GIC_STATUS_DEBUG_INDEX);
  return false;
}
#ifdef GIC_DEBUG
#define GIC_DBG_OK(dbg, cond) ((cond) ? true : ::gic::dbg_fail(dbg))
#else
#define GIC_DBG_OK(dbg, cond) true
#endif

template <typename T>
struct DParams {
  T rho_s, rho_f, k_n, zeta, kt_over_cn, mu, c_drag;
  T g[3];
  T dt;
  T exch;     // -dt' / dt (exchange scale)
  T inv_rho_f;
  int vm, walls;
  // capillary pair force (Sec. 5.4); cap = 0: off
  int cap;
  T sigma, frac, moist;
  T cpk;    // 2 moisture_peak - 1/2: the middle control point of Gamma's Bezier curve
  T kappa;  // d_r of a pair <= kappa (r_i + r_j) for radii within a factor 16: the search reach
};

int make_grid(const GicGrid* g, DGrid* out);
template <typename T>
int make_params(const GicParams* p, DParams<T>* out);
int check_granules(const GicGranules* s, const char* what, bool need_id = false);
// gic_sort gated by two device words (see gic_sort.cu)
int sort_gated(const GicGrid* grid, const GicGranules* in, GicGranules* out, int32_t* perm, void* cell_table, void* ws,
               size_t ws_bytes, const uint32_t* gate, cudaStream_t stream);
// per-granule vectors are real[4n]: 16-byte (FP32) / 32-byte (FP64) aligned
int check_vecs(int32_t precision, const char* what, std::initializer_list<const void*> ptrs);

inline unsigned grid_blocks(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// ----------------------------------------------------------------- device side

__device__ __forceinline__ int cell_x(int32_t c) { return c & (kMaxCellsPerAxis - 1); }
__device__ __forceinline__ int cell_y(int32_t c) { return (c >> kCellBits) & (kMaxCellsPerAxis - 1); }
__device__ __forceinline__ int cell_z(int32_t c) { return (c >> (2 * kCellBits)) & (kMaxCellsPerAxis - 1); }
__device__ __forceinline__ int32_t pack_cell(int x, int y, int z) {
  return x | (y << kCellBits) | (z << (2 * kCellBits));
}

// The float position copy of an FP32 granule (posf): its position in
// contact-cell units, c + q / 2^30 per axis, and its radius (metres).  The
// coordinates are below 1024, so each is off by at most 2^-14 cell and a
// distance between two copies by less than 2.2e-4 cell: the float pre-tests
// widen the contact radius by kPosfTol cell and leave the decision to the
// exact integer geometry.
constexpr float kPosfTol = 1.0f / 2048.0f;
__device__ __forceinline__ float4 posf_of(int32_t c, const uint4& p) {
  return make_float4((float)cell_x(c) + (float)p.x * 0x1p-30f, (float)cell_y(c) + (float)p.y * 0x1p-30f,
                     (float)cell_z(c) + (float)p.z * 0x1p-30f, __uint_as_float(p.w));
}
__device__ __forceinline__ int64_t table_index(const DGrid& G, int x, int y, int z) {
  return 1 + x + (int64_t)G.nc[0] * (y + (int64_t)G.nc[1] * z);
}

// 10-bit value -> bits at positions 0, 3, 6, ...
__host__ __device__ __forceinline__ uint32_t spread3(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}
__device__ __forceinline__ uint32_t morton_of_cell(int32_t c) {
  return spread3((uint32_t)cell_x(c)) | (spread3((uint32_t)cell_y(c)) << 1) | (spread3((uint32_t)cell_z(c)) << 2);
}

__device__ __forceinline__ void raise_status(uint32_t* status, uint32_t bits) {
  if (status) atomicOr(status, bits);
}

// vector type of each precision
template <typename T>
struct Vec;
template <>
struct Vec<float> {
  using type = float4;
};
template <>
struct Vec<double> {
  using type = d4;
};
template <typename T>
using vec_t = typename Vec<T>::type;

template <typename T>
__device__ __forceinline__ vec_t<T> make_vec(T x, T y, T z) {
  vec_t<T> v;
  v.x = x;
  v.y = y;
  v.z = z;
  v.w = T(0);
  return v;
}

// position storage of each precision
template <typename T>
struct Pos;
template <>
struct Pos<float> {
  using type = uint4;  // {qx, qy, qz, bits(r)}
};
template <>
struct Pos<double> {
  using type = d4;  // {ox, oy, oz, r}
};
template <typename T>
using pos_t = typename Pos<T>::type;

// read-only cached loads of state elements
__device__ __forceinline__ uint4 ldg(const uint4* p) { return __ldg(p); }
__device__ __forceinline__ float4 ldg(const float4* p) { return __ldg(p); }
__device__ __forceinline__ d4 ldg(const d4* p) {
  double2 a = __ldg(reinterpret_cast<const double2*>(p));
  double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  d4 r;
  r.x = a.x;
  r.y = a.y;
  r.z = b.x;
  r.w = b.y;
  return r;
}

// Prefetch of the line holding p into L2 (no register is tied up until the
// value is loaded).
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

__device__ __forceinline__ float radius_of(const uint4& p) { return __uint_as_float(p.w); }
__device__ __forceinline__ double radius_of(const d4& p) { return p.w; }

__device__ __forceinline__ uint32_t pcomp(const uint4& p, int a) { return a == 0 ? p.x : (a == 1 ? p.y : p.z); }
__device__ __forceinline__ double pcomp(const d4& p, int a) { return a == 0 ? p.x : (a == 1 ? p.y : p.z); }

template <typename T>
__device__ __forceinline__ T vcomp(const vec_t<T>& v, int a) {
  return a == 0 ? v.x : (a == 1 ? v.y : v.z);
}

// x_i - x_j for granule j sitting in the contact cell offset (ox, oy, oz) from
// granule i's cell; metres.
__device__ __forceinline__ void rel_ij(const DGrid& G, const uint4& pi, const uint4& pj, int ox, int oy, int oz,
                                       float& rx, float& ry, float& rz) {
  // exact integer difference in 2^-30 h_c units, |.| < 2^31
  int dxq = (int)pi.x - (int)pj.x - ox * (int)kFracOne;
  int dyq = (int)pi.y - (int)pj.y - oy * (int)kFracOne;
  int dzq = (int)pi.z - (int)pj.z - oz * (int)kFracOne;
  rx = (float)dxq * G.unit_f;
  ry = (float)dyq * G.unit_f;
  rz = (float)dzq * G.unit_f;
}
__device__ __forceinline__ void rel_ij(const DGrid& G, const d4& pi, const d4& pj, int ox, int oy, int oz, double& rx,
                                       double& ry, double& rz) {
  rx = (pi.x - pj.x) - ox * G.hc;
  ry = (pi.y - pj.y) - oy * G.hc;
  rz = (pi.z - pj.z) - oz * G.hc;
}

// distance to the lower wall of axis a for a granule in contact cell c == 0,
// and to the upper wall for c == nc - 1 (metres)
__device__ __forceinline__ float gap_lo(const DGrid& G, const uint4& p, int a) { return (float)pcomp(p, a) * G.unit_f; }
__device__ __forceinline__ float gap_hi(const DGrid& G, const uint4& p, int a) {
  return (float)(kFracOne - pcomp(p, a)) * G.unit_f;
}
__device__ __forceinline__ double gap_lo(const DGrid& G, const d4& p, int a) { return pcomp(p, a); }
__device__ __forceinline__ double gap_hi(const DGrid& G, const d4& p, int a) { return G.hc - pcomp(p, a); }

// MAC cell m and fraction t in [0, 1) of the position along one axis, from the
// contact coordinate c and the in-cell offset.
__device__ __forceinline__ int mac_of(const DGrid& G, int c) { return (int)(((uint32_t)c * G.kmul) >> 20); }

__device__ __forceinline__ float mac_frac(const DGrid& G, int c, int m, uint32_t q) {
  int sub = c - m * G.k;
  return ((float)sub + (float)q * 0x1p-30f) * G.inv_k_f;
}
__device__ __forceinline__ double mac_frac(const DGrid& G, int c, int m, double o) {
  int sub = c - m * G.k;
  return ((double)sub * G.hc + o) * G.inv_dx;
}
// FP64 fraction from the fixed-point state (used where the volume fraction is
// accumulated in FP64): exact integer numerator, one rounding.
__device__ __forceinline__ double mac_frac_fp64(const DGrid& G, int c, int m, uint32_t q) {
  uint64_t sub = (uint64_t)(c - m * G.k);
  return (double)((sub << kFracBits) | q) * G.inv_k_frac;
}
__device__ __forceinline__ double mac_frac_fp64(const DGrid& G, int c, int m, double o) { return mac_frac(G, c, m, o); }

// Tent-kernel stencil along one axis.  Samples sit at (i + s) dx, i = 0..ns-1,
// with s = 0 (the axis normal to a face) or 1/2 (cell centres).  The point is
// at m + t (grid units).  Returns the lower sample i0 and the weight w of
// sample i0 + 1; points beyond the end samples clamp onto them (G2P), which
// is also the folding rule of the scatter (P2G).
template <typename T>
__device__ __forceinline__ void stencil_axis(int m, T t, bool face, int ns, int& i0, T& w) {
  if (face) {
    i0 = m;
    w = t;
  } else if (t >= T(0.5)) {
    i0 = m;
    w = t - T(0.5);
  } else {
    i0 = m - 1;
    w = t + T(0.5);
  }
  if (i0 < 0) {
    i0 = 0;
    w = T(0);
  } else if (i0 > ns - 2) {
    i0 = ns - 2;
    w = T(1);
  }
}

template <typename T>
struct Stencil {
  int i0[3];
  T w[3];
};

// stencil of MAC component comp (0,1,2: faces normal to x,y,z; 3: centres)
template <typename T>
__device__ __forceinline__ Stencil<T> stencil_of(const DGrid& G, const int m[3], const T t[3], int comp) {
  Stencil<T> S;
  const int n[3] = {G.nx, G.ny, G.nz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    bool face = (a == comp);
    stencil_axis<T>(m[a], t[a], face, n[a] + (face ? 1 : 0), S.i0[a], S.w[a]);
  }
  return S;
}

__device__ __forceinline__ int64_t sample_index(int nsx, int nsy, int i, int j, int k) {
  return i + (int64_t)nsx * (j + (int64_t)nsy * k);
}

// ----------------------------------------------------------------- warp helpers

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Last lane of the run of equal keys that starts at or before this lane
// (runs are maximal sequences of consecutive lanes with the same key).
__device__ __forceinline__ int run_end(unsigned key) {
  const unsigned full = 0xffffffffu;
  int lane = lane_id();
  unsigned prev = __shfl_up_sync(full, key, 1);
  bool head = (lane == 0) || (prev != key);
  unsigned heads = __ballot_sync(full, head);
  unsigned after = lane == 31 ? 0u : (heads & ~((2u << lane) - 1u));
  return after ? (__ffs(after) - 2) : 31;
}
__device__ __forceinline__ bool run_head(unsigned key) {
  unsigned prev = __shfl_up_sync(0xffffffffu, key, 1);
  return lane_id() == 0 || prev != key;
}

// Sum of v over lanes [lane, end] (segmented suffix sum; exact for the head).
__device__ __forceinline__ float seg_sum(float v, int end) {
  int lane = lane_id();
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    float o = __shfl_down_sync(0xffffffffu, v, off);
    if (lane + off <= end) v += o;
  }
  return v;
}
__device__ __forceinline__ double seg_sum(double v, int end) {
  int lane = lane_id();
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    double o = __shfl_down_sync(0xffffffffu, v, off);
    if (lane + off <= end) v += o;
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* smem /* >= 32 */) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  int w = threadIdx.x >> 5;
  if (lane_id() == 0) smem[w] = v;
  __syncthreads();
  T r = T(0);
  if (threadIdx.x < 32) {
    int nw = (blockDim.x + 31) >> 5;
    r = threadIdx.x < nw ? smem[threadIdx.x] : T(0);
    for (int off = 16; off > 0; off >>= 1) r += __shfl_down_sync(0xffffffffu, r, off);
  }
  __syncthreads();
  return r;  // valid in thread 0
}

// Block sums of two values in one pass (one barrier); the results are valid
// in thread 0, and smem (>= 64 doubles) is free again after the next barrier.
__device__ __forceinline__ void block_sum2(double& a, double& b, double* smem) {
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, off);
    b += __shfl_down_sync(0xffffffffu, b, off);
  }
  const int w = threadIdx.x >> 5;
  if (lane_id() == 0) {
    smem[w] = a;
    smem[32 + w] = b;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int nw = (blockDim.x + 31) >> 5;
    a = threadIdx.x < nw ? smem[threadIdx.x] : 0.0;
    b = threadIdx.x < nw ? smem[32 + threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, off);
      b += __shfl_down_sync(0xffffffffu, b, off);
    }
  }
}

}  // namespace gic
