// gic_window.cu -- K substeps of Alg. 2 (SandSubstep) driven from the host:
// sort -> contact -> G2P couple -> integrate -> P2G, K times, on device
// buffers (gic_window_forward) or on host buffers with the copies included
// (gic_window_forward_host).  All scratch comes from the caller's workspace.
#include <string.h>

#include "gic_internal.cuh"

namespace gic {

constexpr int kWindowNbCap = 64;  // Verlet partners per granule in the window's lists

struct WindowLayout {
  size_t sort_ws, off_sort, state_bytes, off_state_b, off_perm, off_fc, off_ffl, off_af, off_fex, off_nb, total;
  // host variant only: device copies of inputs and outputs
  size_t off_cxyz, off_q, off_r, off_v, off_fields, off_alpha, off_fs, off_sums, off_x, off_vout, off_state_a,
      off_table, host_total;
  size_t n_fields_u, n_fields_v, n_fields_w, n_cells;
};

static size_t al(size_t v) { return (v + 255) & ~(size_t)255; }

static int window_layout(const GicGrid* grid, int64_t n, int32_t precision, WindowLayout* L) {
  size_t ws = 0;
  int rc = gic_workspace_size(grid, n, precision, &ws);
  if (rc) return rc;
  size_t real = precision == GIC_FP32 ? 4 : 8;
  size_t nn = (size_t)(n > 0 ? n : 1);
  size_t vec = al(4 * real * nn);
  size_t off = 0;
  L->sort_ws = al(ws);
  L->off_sort = off;
  off += L->sort_ws;
  // three states: the sorted one and the two that gic_step alternates between; each cell, pos, vel, id (+ float
  // positions, FP32)
  L->state_bytes = al(4 * nn) + vec + vec + al(4 * nn) + (precision == GIC_FP32 ? al(16 * nn) : 0);
  L->off_state_b = off;
  off += 3 * L->state_bytes;
  L->off_perm = off;
  off += al(4 * nn);
  L->off_fc = off;
  off += vec;
  L->off_ffl = off;
  off += vec;
  L->off_af = off;
  off += vec;
  L->off_fex = off;
  off += vec;
  L->off_nb = off;  // Verlet lists: list, count, ref_cell, ref_pos, slot, cur, at, flags
  off += al(4 * nn * kWindowNbCap) + 5 * al(4 * nn) + al(4 * real * nn) + al(32);
  L->total = off;
  // host variant
  const GicGrid& g = *grid;
  L->n_fields_u = (size_t)(g.nx + 1) * g.ny * g.nz;
  L->n_fields_v = (size_t)g.nx * (g.ny + 1) * g.nz;
  L->n_fields_w = (size_t)g.nx * g.ny * (g.nz + 1);
  L->n_cells = (size_t)g.nx * g.ny * g.nz;
  size_t table = 0;
  if ((rc = gic_cell_table_size(grid, &table))) return rc;
  L->off_cxyz = off;
  off += al(12 * nn);
  L->off_q = off;
  off += al(12 * nn);
  L->off_r = off;
  off += al(4 * nn);
  L->off_v = off;
  off += al(12 * nn);
  L->off_fields = off;
  off += al(real * L->n_fields_u) + al(real * L->n_fields_v) + al(real * L->n_fields_w) + 2 * al(real * L->n_cells);
  L->off_alpha = off;
  off += al(8 * L->n_cells);
  L->off_fs = off;
  off += al(real * L->n_fields_u) + al(real * L->n_fields_v) + al(real * L->n_fields_w);
  L->off_sums = off;
  off += 256;
  L->off_x = off;
  off += al(24 * nn);
  L->off_vout = off;
  off += al(24 * nn);
  L->off_state_a = off;
  off += al(4 * nn) + vec + vec + al(4 * nn);
  L->off_table = off;
  off += al(table);
  L->host_total = off;
  return GIC_OK;
}

// The window's Verlet lists in the workspace.
static GicNeighbors window_lists(const GicGrid* grid, char* base, const WindowLayout& L, int64_t n,
                                 int32_t precision) {
  GicNeighbors nb;
  size_t nn = (size_t)n;
  size_t real = precision == GIC_FP32 ? 4 : 8;
  char* q = base + L.off_nb;
  nb.n = n;
  nb.cap = kWindowNbCap;
  nb.skin = 0.025 * grid->dx / grid->k_contact;
  nb.list = (int32_t*)q;
  q += al(4 * nn * kWindowNbCap);
  nb.count = (int32_t*)q;
  q += al(4 * nn);
  nb.ref_cell = (int32_t*)q;
  q += al(4 * nn);
  nb.ref_pos = q;
  q += al(4 * real * nn);
  nb.slot = (int32_t*)q;
  q += al(4 * nn);
  nb.cur = (int32_t*)q;
  q += al(4 * nn);
  nb.at = (int32_t*)q;
  q += al(4 * nn);
  nb.flags = (uint32_t*)q;
  return nb;
}

static GicGranules state_at(char* base, int64_t n, int32_t precision) {
  size_t real = precision == GIC_FP32 ? 4 : 8;
  size_t nn = (size_t)(n > 0 ? n : 1);
  size_t vec = al(4 * real * nn);
  GicGranules s;
  s.n = n;
  s.cell = (int32_t*)base;
  s.pos = base + al(4 * nn);
  s.vel = base + al(4 * nn) + vec;
  s.id = (int32_t*)(base + al(4 * nn) + 2 * vec);
  s.precision = precision;
  s.posf = nullptr;
  return s;
}

// The window's three states in the workspace: S[0] sorted, S[1] and S[2]
// the states gic_step alternates between.
static void window_states(char* base, const WindowLayout& L, int64_t n, int32_t precision, bool with_id,
                          GicGranules S[3]) {
  for (int k = 0; k < 3; ++k) {
    S[k] = state_at(base + L.off_state_b + k * L.state_bytes, n, precision);
    if (!with_id) S[k].id = nullptr;
    if (precision == GIC_FP32) {
      size_t nn = (size_t)(n > 0 ? n : 1);
      S[k].posf = (float*)(base + L.off_state_b + k * L.state_bytes + al(4 * nn) + 2 * al(16 * nn) + al(4 * nn));
    }
  }
}

// A second stream and the two events that fork it from and join it to the
// caller's stream, released on every return.
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  int open(const char* what) {
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return set_error(GIC_ERR_CUDA, "%s: side stream set-up failed", what);
    }
    return GIC_OK;
  }
  ~SideStream() {
    if (join) cudaEventDestroy(join);
    if (fork) cudaEventDestroy(fork);
    if (s) cudaStreamDestroy(s);  // returns at once; the stream's work still completes
  }
};

// The window of gic_window_forward_host with the first substep's sort and
// list build done before the fluid fields are needed: A is sorted into S[0],
// the rows of S[0] are built on the staged neighbourhood (FP32, contact law
// alone), the stream waits for `fields`, and the K gic_step calls start from
// S[0] with the lists already current (a build that overflows leaves the
// rebuild flag set, and the first call rebuilds as usual).  The same kernels
// in the same order as gic_window_forward: the same results.
static int window_prebuilt(const GicGrid* grid, const GicParams* params, const WindowLayout& L, char* base,
                           const GicGranules* A, int32_t K, cudaEvent_t fields, const void* u, const void* v,
                           const void* w, const void* p, const void* alpha_f, double* alpha_s, void* Fs_u,
                           void* Fs_v, void* Fs_w, double* sums2, void* table, cudaStream_t st,
                           const GicGranules** result) {
  int rc;
  GicGranules S[3];
  window_states(base, L, A->n, A->precision, true, S);
  int32_t* perm = (int32_t*)(base + L.off_perm);
  GicNeighbors nb = window_lists(grid, base, L, A->n, A->precision);
  const gic_stream_t stream = (gic_stream_t)st;
  if ((rc = gic_neighbors_reset(&nb, stream))) return rc;
  if ((rc = gic_sort(grid, A, &S[0], perm, table, base + L.off_sort, L.sort_ws, stream))) return rc;
  if ((rc = gic_neighbors_build(grid, &S[0], table, &nb, stream))) return rc;
  if (cudaStreamWaitEvent(st, fields, 0) != cudaSuccess)
    return set_error(GIC_ERR_CUDA, "gic_window_forward_host: stream wait failed");
  const GicGranules* cur = &S[0];
  for (int s = 0; s < K; ++s) {
    const bool last = s == K - 1;
    GicGranules* nxt = cur == &S[1] ? &S[2] : &S[1];
    GicGranules* srt = cur == &S[0] ? &S[2] : &S[0];  // shares no array with cur or nxt
    if ((rc = gic_step(grid, params, cur, nxt, srt, perm, table, base + L.off_sort, L.sort_ws, &nb, u, v, w, p,
                       alpha_f, last ? alpha_s : nullptr, Fs_u, Fs_v, Fs_w, last ? sums2 : nullptr, stream)))
      return rc;
    cur = nxt;
  }
  *result = cur;
  return GIC_OK;
}

}  // namespace gic

using namespace gic;

extern "C" int gic_window_workspace_size(const GicGrid* grid, int64_t n, int32_t precision, size_t* bytes) {
  GIC_RANGE("gic_window_workspace_size");
  if (!bytes) return set_error(GIC_ERR_INVALID, "bytes is NULL");
  WindowLayout L;
  int rc = window_layout(grid, n, precision, &L);
  if (rc) return rc;
  *bytes = L.total;
  return GIC_OK;
}

extern "C" int gic_window_host_workspace_size(const GicGrid* grid, int64_t n, int32_t precision, size_t* bytes) {
  GIC_RANGE("gic_window_host_workspace_size");
  if (!bytes) return set_error(GIC_ERR_INVALID, "bytes is NULL");
  WindowLayout L;
  int rc = window_layout(grid, n, precision, &L);
  if (rc) return rc;
  *bytes = L.host_total;
  return GIC_OK;
}

extern "C" int gic_window_forward(const GicGrid* grid, const GicParams* params, GicGranules* state, int32_t K,
                                  const void* u, const void* v, const void* w, const void* p, const void* alpha_f,
                                  double* alpha_s, void* Fs_u, void* Fs_v, void* Fs_w, double* sums2,
                                  void* cell_table, void* ws, size_t ws_bytes, gic_stream_t stream) {
  GIC_RANGE("gic_window_forward");
  int rc = check_granules(state, "gic_window_forward");
  if (rc) return rc;
  if (K < 0) return set_error(GIC_ERR_INVALID, "gic_window_forward: K < 0");
  WindowLayout L;
  if ((rc = window_layout(grid, state->n, state->precision, &L))) return rc;
  if (!ws || ws_bytes < L.total)
    return set_error(GIC_ERR_WORKSPACE, "gic_window_forward: workspace of %zu bytes needed, %zu given", L.total,
                     ws_bytes);
  if ((uintptr_t)ws % 256) return set_error(GIC_ERR_ALIGN, "gic_window_forward: workspace must be 256-byte aligned");
  char* base = (char*)ws;
  GicGranules S[3];  // S[0] sorted, S[1] and S[2] the states gic_step alternates between
  window_states(base, L, state->n, state->precision, state->id != nullptr, S);
  GicGranules& B = S[0];
  int32_t* perm = (int32_t*)(base + L.off_perm);
  void* Fc = base + L.off_fc;
  void* Ffl = base + L.off_ffl;
  void* af = base + L.off_af;
  void* fex = base + L.off_fex;
  // Verlet lists (skin 0.05 h_c / 2, at least 0.05 r_max since h_c >= 2 r_max) when the state carries ids
  GicNeighbors nb;
  const bool verlet = state->id != nullptr && state->n > 0;
  if (verlet) {
    nb = window_lists(grid, base, L, state->n, state->precision);
    if ((rc = gic_neighbors_reset(&nb, stream))) return rc;
  }
  // alpha_s once, at the final positions (Alg. 1 CalTargetFraction); F_s every substep (Alg. 2)
  const GicGranules* cur = state;  // the lists were just reset: the first gic_step sorts `state`
  for (int s = 0; s < K; ++s) {
    bool last = s == K - 1;
    if (verlet) {  // sort only on list rebuilds, the rest of the substep fused
      GicGranules* nxt = cur == &S[1] ? &S[2] : &S[1];
      if ((rc = gic_step(grid, params, cur, nxt, &B, perm, cell_table, base + L.off_sort, L.sort_ws, &nb, u, v, w, p,
                         alpha_f, last ? alpha_s : nullptr, Fs_u, Fs_v, Fs_w, last ? sums2 : nullptr, stream)))
        return rc;
      cur = nxt;
      continue;
    }
    if ((rc = gic_sort(grid, state, &B, perm, cell_table, base + L.off_sort, L.sort_ws, stream))) return rc;
    if ((rc = gic_contact(grid, params, &B, cell_table, Fc, stream))) return rc;
    if ((rc = gic_g2p_couple(grid, params, &B, u, v, w, p, alpha_f, Ffl, af, nullptr, stream))) return rc;
    if ((rc = gic_integrate(grid, params, &B, Fc, Ffl, af, state, fex, stream))) return rc;
    if ((rc = gic_p2g(grid, params, &B, state, fex, last ? alpha_s : nullptr, Fs_u, Fs_v, Fs_w,
                      last ? sums2 : nullptr, stream)))
      return rc;
  }
  if (cur != state) {  // the result back into the caller's state
    const size_t n = (size_t)state->n, real = state->precision == GIC_FP32 ? 4 : 8;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(state->cell, cur->cell, 4 * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(state->pos, cur->pos, 4 * real * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(state->vel, cur->vel, 4 * real * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(state->id, cur->id, 4 * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return set_error(GIC_ERR_CUDA, "gic_window_forward: copy of the result failed");
    if (state->posf && cur->posf &&
        cudaMemcpyAsync(state->posf, cur->posf, 16 * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return set_error(GIC_ERR_CUDA, "gic_window_forward: copy of the result failed");
  }
  return GIC_OK;
}

extern "C" int gic_window_forward_host(const GicGrid* grid, const GicParams* params, int64_t n, int32_t precision,
                                       const int32_t* cell_xyz, const uint32_t* q, const float* r, const float* v,
                                       const void* u_f, const void* v_f, const void* w_f, const void* p_f,
                                       const void* alpha_f, int32_t K, double* x_out, double* v_out,
                                       double* alpha_s, void* Fs_u, void* Fs_v, void* Fs_w, double* sums2, void* ws,
                                       size_t ws_bytes, gic_stream_t stream) {
  GIC_RANGE("gic_window_forward_host");
  if (n < 0) return set_error(GIC_ERR_INVALID, "gic_window_forward_host: n < 0");
  if (precision != GIC_FP32 && precision != GIC_FP64) return set_error(GIC_ERR_INVALID, "bad precision");
  WindowLayout L;
  int rc = window_layout(grid, n, precision, &L);
  if (rc) return rc;
  if (!ws || ws_bytes < L.host_total)
    return set_error(GIC_ERR_WORKSPACE, "gic_window_forward_host: workspace of %zu bytes needed, %zu given",
                     L.host_total, ws_bytes);
  if ((uintptr_t)ws % 256) return set_error(GIC_ERR_ALIGN, "workspace must be 256-byte aligned");
  if (n > 0 && (!cell_xyz || !q || !r || !v)) return set_error(GIC_ERR_INVALID, "null granule input");
  if (!u_f || !v_f || !w_f || !p_f || !alpha_f) return set_error(GIC_ERR_INVALID, "null fluid field");
  cudaStream_t st = (cudaStream_t)stream;
  char* base = (char*)ws;
  size_t real = precision == GIC_FP32 ? 4 : 8;
  char* fu = base + L.off_fields;
  char* fv = fu + al(real * L.n_fields_u);
  char* fw = fv + al(real * L.n_fields_v);
  char* fp = fw + al(real * L.n_fields_w);
  char* fa = fp + al(real * L.n_cells);
  char* su = base + L.off_fs;
  char* sv = su + al(real * L.n_fields_u);
  char* sw = sv + al(real * L.n_fields_v);
  double* d_alpha = (double*)(base + L.off_alpha);
  double* d_sums = (double*)(base + L.off_sums);
  double* d_x = (double*)(base + L.off_x);
  double* d_v = (double*)(base + L.off_vout);
  void* table = base + L.off_table;
  size_t table_bytes = 0;
  gic_cell_table_size(grid, &table_bytes);
  GicGranules A = state_at(base + L.off_state_a, n, precision);
#define GIC_CU(call)                                                                               \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return set_error(GIC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)
  // FP32 with the contact law alone: the granules go first, and their sort and
  // list build run while the fluid fields are copied on a second stream (the
  // first substep waits for them); otherwise everything in stream order
  const bool overlap = precision == GIC_FP32 && n > 0 && K > 0 && params && params->sigma == 0.0;
  SideStream side;
  if (overlap && (rc = side.open("gic_window_forward_host"))) return rc;
  cudaStream_t sf = overlap ? side.s : st;  // the fields' stream
  // inputs: host -> device (one copy per array)
  if (n > 0) {
    GIC_CU(cudaMemcpyAsync(base + L.off_cxyz, cell_xyz, 12 * (size_t)n, cudaMemcpyHostToDevice, st));
    GIC_CU(cudaMemcpyAsync(base + L.off_q, q, 12 * (size_t)n, cudaMemcpyHostToDevice, st));
    GIC_CU(cudaMemcpyAsync(base + L.off_r, r, 4 * (size_t)n, cudaMemcpyHostToDevice, st));
    GIC_CU(cudaMemcpyAsync(base + L.off_v, v, 12 * (size_t)n, cudaMemcpyHostToDevice, st));
  }
  if (overlap) {  // the fields' stream starts after everything on st so far (earlier calls included)
    GIC_CU(cudaEventRecord(side.fork, st));
    GIC_CU(cudaStreamWaitEvent(sf, side.fork, 0));
  }
  GIC_CU(cudaMemcpyAsync(fu, u_f, real * L.n_fields_u, cudaMemcpyHostToDevice, sf));
  GIC_CU(cudaMemcpyAsync(fv, v_f, real * L.n_fields_v, cudaMemcpyHostToDevice, sf));
  GIC_CU(cudaMemcpyAsync(fw, w_f, real * L.n_fields_w, cudaMemcpyHostToDevice, sf));
  GIC_CU(cudaMemcpyAsync(fp, p_f, real * L.n_cells, cudaMemcpyHostToDevice, sf));
  GIC_CU(cudaMemcpyAsync(fa, alpha_f, real * L.n_cells, cudaMemcpyHostToDevice, sf));
  GIC_CU(cudaMemsetAsync(su, 0, real * L.n_fields_u, sf));
  GIC_CU(cudaMemsetAsync(sv, 0, real * L.n_fields_v, sf));
  GIC_CU(cudaMemsetAsync(sw, 0, real * L.n_fields_w, sf));
  if (overlap) GIC_CU(cudaEventRecord(side.join, sf));
  GIC_CU(cudaMemsetAsync(table, 0, table_bytes, st));
  if ((rc = gic_pack(grid, n, (const int32_t*)(base + L.off_cxyz), (const uint32_t*)(base + L.off_q),
                     (const float*)(base + L.off_r), (const float*)(base + L.off_v), &A, stream)))
    return rc;
  const GicGranules* result = &A;
  if (overlap) {
    if ((rc = window_prebuilt(grid, params, L, base, &A, K, side.join, fu, fv, fw, fp, fa, d_alpha, su, sv, sw,
                              d_sums, table, st, &result)))
      return rc;
  } else if ((rc = gic_window_forward(grid, params, &A, K, fu, fv, fw, fp, fa, d_alpha, su, sv, sw, d_sums, table,
                                      base + L.off_sort, L.total, stream))) {
    return rc;
  }
  if ((rc = gic_unpack(grid, result, d_x, d_v, stream))) return rc;
  // outputs: device -> host
  if (n > 0) {
    if (x_out) GIC_CU(cudaMemcpyAsync(x_out, d_x, 24 * (size_t)n, cudaMemcpyDeviceToHost, st));
    if (v_out) GIC_CU(cudaMemcpyAsync(v_out, d_v, 24 * (size_t)n, cudaMemcpyDeviceToHost, st));
  }
  if (alpha_s) GIC_CU(cudaMemcpyAsync(alpha_s, d_alpha, 8 * L.n_cells, cudaMemcpyDeviceToHost, st));
  if (Fs_u) GIC_CU(cudaMemcpyAsync(Fs_u, su, real * L.n_fields_u, cudaMemcpyDeviceToHost, st));
  if (Fs_v) GIC_CU(cudaMemcpyAsync(Fs_v, sv, real * L.n_fields_v, cudaMemcpyDeviceToHost, st));
  if (Fs_w) GIC_CU(cudaMemcpyAsync(Fs_w, sw, real * L.n_fields_w, cudaMemcpyDeviceToHost, st));
  if (sums2) GIC_CU(cudaMemcpyAsync(sums2, d_sums, 16, cudaMemcpyDeviceToHost, st));
#undef GIC_CU
  return wait_stream(st, 600000, "gic_window_forward_host");
}
