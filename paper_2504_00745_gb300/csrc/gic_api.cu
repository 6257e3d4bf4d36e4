// gic_api.cu -- library housekeeping: status word, errors, sizes, state
// conversion (pack / unpack) and the status query.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <thread>

#include "gic_internal.cuh"

namespace gic {

// Sticky status word, one per device that loads the library.
__device__ uint32_t g_status_word;

namespace {
thread_local char t_last_error[512] = "";
std::atomic<int64_t> g_launches{0};
std::mutex g_status_mu;
uint32_t* g_status_ptr[64] = {nullptr};
}  // namespace

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(t_last_error, sizeof(t_last_error), fmt, ap);
  va_end(ap);
  return code;
}

// Launches made while a graph is being captured are not executions: the
// graph launches count their kernels themselves.
thread_local bool g_capturing = false;
void count_launches(int64_t k) {
  if (!g_capturing) g_launches.fetch_add(k, std::memory_order_relaxed);
}
void set_capturing(bool on) { g_capturing = on; }

// Poll the stream against a deadline instead of blocking forever.
int wait_stream(cudaStream_t stream, int64_t timeout_ms, const char* what) {
  auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t q = cudaStreamQuery(stream);
    if (q == cudaSuccess) return GIC_OK;
    if (q != cudaErrorNotReady) return set_error(GIC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(q));
    auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
    if (ms > timeout_ms) return set_error(GIC_ERR_TIMEOUT, "%s: stream still busy after %lld ms", what, (long long)ms);
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

uint32_t* status_word() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_status_mu);
  if (!g_status_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_status_word) != cudaSuccess) return nullptr;
    g_status_ptr[dev] = (uint32_t*)p;
  }
  return g_status_ptr[dev];
}

int make_grid(const GicGrid* g, DGrid* G) {
  if (!g) return set_error(GIC_ERR_INVALID, "grid is NULL");
  if (g->nx < 2 || g->ny < 2 || g->nz < 2) return set_error(GIC_ERR_INVALID, "grid needs at least 2 cells per axis");
  if (g->k_contact < 1) return set_error(GIC_ERR_INVALID, "k_contact must be >= 1");
  if (!(g->dx > 0.0) || !std::isfinite(g->dx)) return set_error(GIC_ERR_INVALID, "dx must be positive");
  int64_t nc[3] = {(int64_t)g->nx * g->k_contact, (int64_t)g->ny * g->k_contact, (int64_t)g->nz * g->k_contact};
  for (int a = 0; a < 3; ++a)
    if (nc[a] > kMaxCellsPerAxis)
      return set_error(GIC_ERR_INVALID, "contact grid axis %d has %lld cells; at most %d are supported", a,
                       (long long)nc[a], kMaxCellsPerAxis);
  G->nx = g->nx;
  G->ny = g->ny;
  G->nz = g->nz;
  G->k = g->k_contact;
#ifdef GIC_DEBUG
  G->dbg = status_word();
#else
  G->dbg = nullptr;
#endif
  for (int a = 0; a < 3; ++a) G->nc[a] = (int)nc[a];
  G->kmul = (uint32_t)(((1u << 20) + (uint32_t)g->k_contact - 1) / (uint32_t)g->k_contact);
  G->dx = g->dx;
  G->hc = g->dx / g->k_contact;
  G->inv_dx = 1.0 / g->dx;
  G->inv_hc = 1.0 / G->hc;
  for (int a = 0; a < 3; ++a) G->origin[a] = g->origin[a];
  G->unit = G->hc / (double)kFracOne;
  G->inv_unit = (double)kFracOne / G->hc;
  G->inv_k_frac = 1.0 / ((double)g->k_contact * (double)kFracOne);
  G->dx_f = (float)G->dx;
  G->hc_f = (float)G->hc;
  G->inv_dx_f = (float)G->inv_dx;
  G->inv_hc_f = (float)G->inv_hc;
  G->unit_f = (float)G->unit;
  G->inv_unit_f = (float)G->inv_unit;
  G->inv_k_f = (float)(1.0 / g->k_contact);
  G->s_hi = (float)G->inv_unit;
  G->s_lo = (float)(G->inv_unit - (double)G->s_hi);
  G->s2_margin = (float)((double)G->s_hi * (double)G->s_hi * (1.0 + 4e-6));
  if (g->k_contact == 1) {
    G->kinv64 = 0;
  } else {
    // ceil(2^64 / k) = floor((2^64 - 1) / k) + 1 for k not a power of two, exact otherwise
    unsigned long long k = (unsigned long long)g->k_contact;
    unsigned long long q = ~0ull / k;
    G->kinv64 = q + 1;
  }
  G->vol_fx = 4.0 / 3.0 * kPi / (g->dx * g->dx * g->dx) * 9007199254740992.0;  // * 2^53
  G->vol_fx_hi = (float)G->vol_fx;
  G->vol_fx_lo = (float)(G->vol_fx - (double)G->vol_fx_hi);
  return GIC_OK;
}

template <typename T>
int make_params(const GicParams* p, DParams<T>* P) {
  if (!p) return set_error(GIC_ERR_INVALID, "params is NULL");
  if (!(p->rho_s > 0.0)) return set_error(GIC_ERR_INVALID, "rho_s must be positive");
  if (!(p->rho_f >= 0.0)) return set_error(GIC_ERR_INVALID, "rho_f must be >= 0");
  if (!(p->dt_sub > 0.0) || !(p->dt_fluid > 0.0)) return set_error(GIC_ERR_INVALID, "time steps must be positive");
  P->rho_s = (T)p->rho_s;
  P->rho_f = (T)p->rho_f;
  P->k_n = (T)p->k_n;
  P->zeta = (T)p->zeta;
  P->kt_over_cn = (T)p->kt_over_cn;
  P->mu = (T)p->mu_fric;
  P->c_drag = (T)p->c_drag;
  for (int a = 0; a < 3; ++a) P->g[a] = (T)p->g[a];
  P->dt = (T)p->dt_sub;
  P->exch = (T)(-p->dt_sub / p->dt_fluid);
  P->inv_rho_f = p->rho_f > 0.0 ? (T)(1.0 / p->rho_f) : T(0);
  P->vm = p->virtual_mass ? 1 : 0;
  P->walls = p->walls ? 1 : 0;
  P->cap = 0;
  P->sigma = P->frac = P->moist = P->cpk = P->kappa = T(0);
  if (p->sigma != 0.0) {
    if (!(p->sigma > 0.0)) return set_error(GIC_ERR_INVALID, "sigma must be >= 0");
    if (!(p->bridge_frac > 0.0) || !(p->bridge_frac < 1.0))
      return set_error(GIC_ERR_INVALID, "bridge_frac must lie in (0, 1)");
    if (!(p->moisture >= 0.0)) return set_error(GIC_ERR_INVALID, "moisture must be >= 0");
    if (!(p->moisture_peak >= 0.25 && p->moisture_peak <= 0.75))
      return set_error(GIC_ERR_INVALID, "moisture_peak must lie in [0.25, 0.75]");
    P->cap = 1;
    P->sigma = (T)p->sigma;
    P->frac = (T)p->bridge_frac;
    P->moist = (T)p->moisture;
    P->cpk = (T)(2.0 * p->moisture_peak - 0.5);
    // the largest d_r / (r_i + r_j) over radius ratios rho = r_j / r_i in [1/16, 1]:
    // R = 2 rho / (1 + rho), V* = frac (2 pi / 3) (1 + rho^3), v = V* / R^3,
    // d_r = R (v^(1/3) + 0.1 v^(2/3))  (radii in units of r_i)
    double k = 0.0;
    for (int t = 0; t <= 4096; ++t) {
      const double rho = 1.0 / 16.0 + (1.0 - 1.0 / 16.0) * t / 4096.0;
      const double R = 2.0 * rho / (1.0 + rho);
      const double v = p->bridge_frac * (2.0 * kPi / 3.0) * (1.0 + rho * rho * rho) / (R * R * R);
      const double c = std::cbrt(v);
      k = std::max(k, R * (c + 0.1 * c * c) / (1.0 + rho));
    }
    P->kappa = (T)(1.01 * k);
  }
  return GIC_OK;
}
template int make_params<float>(const GicParams*, DParams<float>*);
template int make_params<double>(const GicParams*, DParams<double>*);

int check_granules(const GicGranules* s, const char* what, bool need_id) {
  if (!s) return set_error(GIC_ERR_INVALID, "%s: granules is NULL", what);
  if (s->n < 0 || s->n > (int64_t)INT32_MAX) return set_error(GIC_ERR_INVALID, "%s: bad granule count", what);
  if (s->precision != GIC_FP32 && s->precision != GIC_FP64)
    return set_error(GIC_ERR_INVALID, "%s: precision must be GIC_FP32 or GIC_FP64", what);
  if (s->n == 0) return GIC_OK;
  if (!s->cell || !s->pos || !s->vel) return set_error(GIC_ERR_INVALID, "%s: null state array", what);
  if (need_id && !s->id) return set_error(GIC_ERR_INVALID, "%s: id array required", what);
  size_t al = s->precision == GIC_FP32 ? 16 : 32;
  if (((uintptr_t)s->pos % al) || ((uintptr_t)s->vel % al))
    return set_error(GIC_ERR_ALIGN, "%s: pos/vel must be %zu-byte aligned", what, al);
  if ((uintptr_t)s->posf % 16) return set_error(GIC_ERR_ALIGN, "%s: posf must be 16-byte aligned", what);
  return GIC_OK;
}

int check_vecs(int32_t precision, const char* what, std::initializer_list<const void*> ptrs) {
  size_t al = precision == GIC_FP32 ? 16 : 32;
  for (const void* p : ptrs)
    if (p && ((uintptr_t)p % al)) return set_error(GIC_ERR_ALIGN, "%s: vector arrays must be %zu-byte aligned", what, al);
  return GIC_OK;
}

// ----------------------------------------------------------------- kernels

template <typename T>
__global__ void k_pack(DGrid G, int64_t n, const int32_t* __restrict__ cxyz, const uint32_t* __restrict__ q,
                       const float* __restrict__ r, const float* __restrict__ v, int32_t* __restrict__ cell,
                       pos_t<T>* __restrict__ pos, vec_t<T>* __restrict__ vel, int32_t* __restrict__ id,
                       uint32_t* status) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c[3];
  uint32_t f[3];
  bool bad = false;
  for (int a = 0; a < 3; ++a) {
    c[a] = cxyz[3 * i + a];
    f[a] = q[3 * i + a];
    if (c[a] < 0 || c[a] >= G.nc[a] || f[a] >= kFracOne) bad = true;
    c[a] = min(max(c[a], 0), G.nc[a] - 1);
    f[a] = min(f[a], kFracMask);
  }
  if (bad) raise_status(status, GIC_STATUS_BAD_CELL);
  cell[i] = pack_cell(c[0], c[1], c[2]);
  if constexpr (sizeof(T) == 4) {
    pos[i] = make_uint4(f[0], f[1], f[2], __float_as_uint(r[i]));
  } else {
    d4 p;
    p.x = (double)f[0] * G.unit;
    p.y = (double)f[1] * G.unit;
    p.z = (double)f[2] * G.unit;
    p.w = (double)r[i];
    pos[i] = p;
  }
  vel[i] = make_vec<T>((T)v[3 * i], (T)v[3 * i + 1], (T)v[3 * i + 2]);
  if (id) id[i] = (int32_t)i;
}

template <typename T>
__global__ void k_unpack(DGrid G, int64_t n, const int32_t* __restrict__ cell, const pos_t<T>* __restrict__ pos,
                         const vec_t<T>* __restrict__ vel, const int32_t* __restrict__ id, double* __restrict__ x,
                         double* __restrict__ v) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t c = cell[i];
  int cc[3] = {cell_x(c), cell_y(c), cell_z(c)};
  pos_t<T> p = pos[i];
  vec_t<T> vv = vel[i];
  int64_t slot = id ? (int64_t)id[i] : i;
  for (int a = 0; a < 3; ++a) {
    double off;
    if constexpr (sizeof(T) == 4)
      off = (double)pcomp(p, a) * G.unit;
    else
      off = pcomp(p, a);
    if (x) x[3 * slot + a] = G.origin[a] + ((double)cc[a] * G.hc + off);
    if (v) v[3 * slot + a] = (double)vcomp<T>(vv, a);
  }
}

template <typename T>
__global__ void k_unpack_adj(int64_t n, const int32_t* __restrict__ id, const double* __restrict__ gx,
                             const double* __restrict__ gv, vec_t<T>* __restrict__ gpos, vec_t<T>* __restrict__ gvel) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t s = id ? (int64_t)id[i] : i;
  if (gpos) gpos[i] = gx ? make_vec<T>((T)gx[3 * s], (T)gx[3 * s + 1], (T)gx[3 * s + 2]) : make_vec<T>(0, 0, 0);
  if (gvel) gvel[i] = gv ? make_vec<T>((T)gv[3 * s], (T)gv[3 * s + 1], (T)gv[3 * s + 2]) : make_vec<T>(0, 0, 0);
}

}  // namespace gic

using namespace gic;

extern "C" {

const char* gic_last_error(void) { return t_last_error; }

int64_t gic_launch_count(void) { return g_launches.load(); }

const char* gic_version(void) { return "gic-gb300 0.1 (sm_103a)"; }

int gic_cell_table_size(const GicGrid* grid, size_t* bytes) {
  GIC_RANGE("gic_cell_table_size");
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if (!bytes) return set_error(GIC_ERR_INVALID, "bytes is NULL");
  *bytes = 16 * (1 + (size_t)G.nc[0] * G.nc[1] * G.nc[2]);
  return GIC_OK;
}

int gic_pack(const GicGrid* grid, int64_t n, const int32_t* cell_xyz, const uint32_t* q, const float* r, const float* v,
             GicGranules* out, gic_stream_t stream) {
  GIC_RANGE("gic_pack");
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if ((rc = check_granules(out, "gic_pack"))) return rc;
  if (out->n != n) return set_error(GIC_ERR_INVALID, "gic_pack: out->n != n");
  if (n == 0) return GIC_OK;
  if (!cell_xyz || !q || !r || !v) return set_error(GIC_ERR_INVALID, "gic_pack: null input");
  uint32_t* st = status_word();
  if (out->precision == GIC_FP32)
    k_pack<float><<<grid_blocks(n, 256), 256, 0, stream>>>(G, n, cell_xyz, q, r, v, out->cell, (uint4*)out->pos,
                                                            (float4*)out->vel, out->id, st);
  else
    k_pack<double><<<grid_blocks(n, 256), 256, 0, stream>>>(G, n, cell_xyz, q, r, v, out->cell, (d4*)out->pos,
                                                             (d4*)out->vel, out->id, st);
  count_launches(1);
  GIC_CHECK_LAUNCH("gic_pack");
  return GIC_OK;
}

int gic_unpack(const GicGrid* grid, const GicGranules* in, double* x, double* v, gic_stream_t stream) {
  GIC_RANGE("gic_unpack");
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if ((rc = check_granules(in, "gic_unpack"))) return rc;
  if (in->n == 0) return GIC_OK;
  if (!x && !v) return set_error(GIC_ERR_INVALID, "gic_unpack: nothing to write");
  if (in->precision == GIC_FP32)
    k_unpack<float><<<grid_blocks(in->n, 256), 256, 0, stream>>>(G, in->n, in->cell, (const uint4*)in->pos,
                                                                  (const float4*)in->vel, in->id, x, v);
  else
    k_unpack<double><<<grid_blocks(in->n, 256), 256, 0, stream>>>(G, in->n, in->cell, (const d4*)in->pos,
                                                                   (const d4*)in->vel, in->id, x, v);
  count_launches(1);
  GIC_CHECK_LAUNCH("gic_unpack");
  return GIC_OK;
}

int gic_unpack_adj(const GicGrid* grid, const GicGranules* in, const double* gx, const double* gv, void* g_pos,
                   void* g_vel, gic_stream_t stream) {
  GIC_RANGE("gic_unpack_adj");
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if ((rc = check_granules(in, "gic_unpack_adj"))) return rc;
  if (in->n == 0) return GIC_OK;
  if ((rc = check_vecs(in->precision, "gic_unpack_adj", {g_pos, g_vel}))) return rc;
  if (in->precision == GIC_FP32)
    k_unpack_adj<float><<<grid_blocks(in->n, 256), 256, 0, stream>>>(in->n, in->id, gx, gv, (float4*)g_pos,
                                                                      (float4*)g_vel);
  else
    k_unpack_adj<double><<<grid_blocks(in->n, 256), 256, 0, stream>>>(in->n, in->id, gx, gv, (d4*)g_pos, (d4*)g_vel);
  count_launches(1);
  GIC_CHECK_LAUNCH("gic_unpack_adj");
  return GIC_OK;
}

int gic_check_status(uint32_t* flags, int32_t clear, int32_t timeout_ms, gic_stream_t stream) {
  GIC_RANGE("gic_check_status");
  if (!flags) return set_error(GIC_ERR_INVALID, "flags is NULL");
  uint32_t* st = status_word();
  if (!st) return set_error(GIC_ERR_CUDA, "status word unavailable");
  int rc = wait_stream((cudaStream_t)stream, timeout_ms > 0 ? timeout_ms : 60000, "gic_check_status");
  if (rc) return rc;
  uint32_t h = 0;
  cudaError_t e = cudaMemcpy(&h, st, sizeof(uint32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return set_error(GIC_ERR_CUDA, "gic_check_status: %s", cudaGetErrorString(e));
  if (clear) {
    e = cudaMemset(st, 0, sizeof(uint32_t));
    if (e != cudaSuccess) return set_error(GIC_ERR_CUDA, "gic_check_status: %s", cudaGetErrorString(e));
  }
  *flags = h;
  return GIC_OK;
}

}  // extern "C"
