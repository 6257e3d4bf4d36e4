// gic_sort.cu -- a1: stable Morton sort of granules by contact cell.
//
// LSD radix sort over the Morton key of the packed contact cell, 8-bit digits,
// reduce-then-scan per pass (upsweep histograms, per-digit scan over tiles,
// downsweep ranking + scatter).  No kernel waits on another block, so nothing
// can spin.  The first pass computes keys from the cells on the fly; the last
// pass scatters the whole granule state (cell, pos, vel, id) together with the
// permutation, so there is no separate gather pass.  A final kernel writes the
// epoch-tagged cell table {start, count, epoch} of the occupied cells.
//
// Stability: inside a tile each warp ranks 4 consecutive chunks of 32 keys in
// order, warps own consecutive sub-ranges and tiles are offset by the counts
// of earlier tiles, so equal keys keep their input order in every pass.

#include "gic_internal.cuh"

namespace gic {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kChunksPerWarp = 4;
constexpr int kTile = kSortThreads * kChunksPerWarp;  // 1024 keys per CTA
constexpr int kRadix = 256;
// upsweep / downsweep CTAs loop over tiles; a gated sort uses at most this
// many CTAs, so that a launch that exits at once costs a short wave
constexpr int kMaxSortCtas = 304;

struct SortLayout {
  int64_t n;
  int tiles;
  int passes;
  size_t off_keys_a, off_vals_a, off_keys_b, off_vals_b, off_counts, off_totals, total;
};

static int key_bits(const DGrid& G) {
  int m = G.nc[0];
  if (G.nc[1] > m) m = G.nc[1];
  if (G.nc[2] > m) m = G.nc[2];
  int b = 0;
  while ((1 << b) < m) ++b;
  if (b < 1) b = 1;
  return 3 * b;
}

static size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

static SortLayout sort_layout(const DGrid& G, int64_t n) {
  SortLayout L;
  L.n = n;
  L.tiles = (int)((n + kTile - 1) / kTile);
  if (L.tiles < 1) L.tiles = 1;
  L.passes = (key_bits(G) + 7) / 8;
  size_t a = align_up(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
  size_t off = 0;
  L.off_keys_a = off;
  off += a;
  L.off_vals_a = off;
  off += a;
  L.off_keys_b = off;
  off += a;
  L.off_vals_b = off;
  off += a;
  L.off_counts = off;
  off += align_up(sizeof(uint32_t) * (size_t)kRadix * L.tiles);
  L.off_totals = off;
  off += align_up(sizeof(uint32_t) * kRadix);
  L.total = off;
  return L;
}

__device__ __forceinline__ uint32_t digit_of(uint32_t key, int shift) { return (key >> shift) & (kRadix - 1); }

// A gated sort runs only when gate[0] | gate[1] != 0 (a Verlet-list rebuild in
// this call); otherwise every kernel exits at once (the caller has copied the
// state in its current order; the cell table keeps the last sort's entries).
// gate == NULL: always sort.
__device__ __forceinline__ bool sort_skipped(const uint32_t* gate) { return gate && (gate[0] | gate[1]) == 0u; }

// Per-tile digit histogram.  counts[d * tiles + tile].
template <bool kFirst>
__global__ void __launch_bounds__(kSortThreads) k_upsweep(int64_t n, int shift, const int32_t* __restrict__ cell,
                                                          const uint32_t* __restrict__ keys,
                                                          uint32_t* __restrict__ counts, int tiles,
                                                          const uint32_t* gate) {
  if (sort_skipped(gate)) return;
  __shared__ uint32_t s_hist[kRadix];
  int warp = threadIdx.x >> 5, lane = lane_id();
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    s_hist[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)tile * kTile + warp * (32 * kChunksPerWarp);
#pragma unroll
    for (int c = 0; c < kChunksPerWarp; ++c) {
      int64_t idx = base + c * 32 + lane;
      bool valid = idx < n;
      uint32_t key = 0;
      if (valid) key = kFirst ? morton_of_cell(cell[idx]) : keys[idx];
      uint32_t d = valid ? digit_of(key, shift) : 0xffffffffu;
      unsigned peers = __match_any_sync(0xffffffffu, d);
      if (valid && (peers & lanemask_lt()) == 0) atomicAdd(&s_hist[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * tiles + tile] = s_hist[threadIdx.x];
  }
}

// Exclusive scan over tiles for one digit per CTA; totals[d] = count of digit d.
// CTA 0 of the first pass also advances the cell-table epoch.
__global__ void __launch_bounds__(kSortThreads) k_scan_tiles(uint32_t* __restrict__ counts, int tiles,
                                                             uint32_t* __restrict__ totals, uint4* table_head,
                                                             const uint32_t* gate) {
  if (sort_skipped(gate)) return;
  __shared__ uint32_t s_warp[kSortWarps];
  __shared__ uint32_t s_carry;
  int d = blockIdx.x;
  uint32_t* row = counts + (int64_t)d * tiles;
  if (threadIdx.x == 0) s_carry = 0;
  if (table_head && d == 0 && threadIdx.x == 0) {
    uint32_t e = table_head->x + 1u;
    table_head->x = e == 0u ? 1u : e;
  }
  __syncthreads();
  int lane = lane_id(), warp = threadIdx.x >> 5;
  for (int base = 0; base < tiles; base += kSortThreads) {
    int t = base + threadIdx.x;
    uint32_t v = t < tiles ? row[t] : 0u;
    uint32_t incl = v;
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t o = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += o;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    uint32_t wsum = 0;
    for (int w = 0; w < warp; ++w) wsum += s_warp[w];
    uint32_t excl = s_carry + wsum + incl - v;
    if (t < tiles) row[t] = excl;
    __syncthreads();
    if (threadIdx.x == kSortThreads - 1) s_carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) totals[d] = s_carry;
}

struct ScatterState {
  const int32_t* in_cell;
  const void* in_pos;
  const void* in_vel;
  const int32_t* in_id;
  int32_t* out_cell;
  void* out_pos;
  void* out_vel;
  int32_t* out_id;
  int32_t* perm;
  float4* out_posf;  // FP32 path: float copy of the sorted positions, or NULL
};

// Rank every key of the tile stably and scatter.  Not-last passes write
// (key, value); the last pass writes the sorted key, the permutation and the
// permuted state.
template <bool kFirst, bool kLast, typename T>
__global__ void __launch_bounds__(kSortThreads) k_downsweep(int64_t n, int shift, const uint32_t* __restrict__ keys_in,
                                                            const uint32_t* __restrict__ vals_in,
                                                            uint32_t* __restrict__ keys_out,
                                                            uint32_t* __restrict__ vals_out,
                                                            const uint32_t* __restrict__ counts,
                                                            const uint32_t* __restrict__ totals, int tiles,
                                                            ScatterState S, const uint32_t* gate) {
  if (sort_skipped(gate)) return;
  __shared__ uint32_t s_warp_hist[kSortWarps][kRadix];
  __shared__ uint32_t s_base[kRadix];
  __shared__ uint32_t s_scan[kSortWarps];
  int warp = threadIdx.x >> 5, lane = lane_id();
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
  __syncthreads();  // the previous tile's reads of the shared arrays are done
  for (int w = 0; w < kSortWarps; ++w) s_warp_hist[w][threadIdx.x] = 0;
  // digit base = (exclusive scan of totals)[d] + (scanned count of earlier tiles)[d]
  {
    uint32_t t = totals[threadIdx.x];
    uint32_t incl = t;
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t o = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += o;
    }
    if (lane == 31) s_scan[warp] = incl;
    __syncthreads();
    uint32_t wsum = 0;
    for (int w = 0; w < warp; ++w) wsum += s_scan[w];
    s_base[threadIdx.x] = wsum + incl - t + counts[(int64_t)threadIdx.x * tiles + tile];
  }
  __syncthreads();

  uint32_t r_key[kChunksPerWarp], r_val[kChunksPerWarp], r_rank[kChunksPerWarp];
  int64_t base = (int64_t)tile * kTile + warp * (32 * kChunksPerWarp);
#pragma unroll
  for (int c = 0; c < kChunksPerWarp; ++c) {
    int64_t idx = base + c * 32 + lane;
    bool valid = idx < n;
    uint32_t key = 0, val = 0;
    if (valid) {
      if (kFirst) {
        key = morton_of_cell(S.in_cell[idx]);
        val = (uint32_t)idx;
      } else {
        key = keys_in[idx];
        val = vals_in[idx];
      }
    }
    uint32_t d = valid ? digit_of(key, shift) : 0xffffffffu;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    unsigned before = peers & lanemask_lt();
    uint32_t prior = valid ? s_warp_hist[warp][d] : 0u;
    __syncwarp();
    if (valid && before == 0) s_warp_hist[warp][d] = prior + (uint32_t)__popc(peers);
    __syncwarp();
    r_key[c] = key;
    r_val[c] = val;
    r_rank[c] = valid ? prior + (uint32_t)__popc(before) : 0xffffffffu;
  }
  __syncthreads();
  // exclusive scan over warps, per digit
  {
    uint32_t run = 0;
    for (int w = 0; w < kSortWarps; ++w) {
      uint32_t t = s_warp_hist[w][threadIdx.x];
      s_warp_hist[w][threadIdx.x] = run;
      run += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < kChunksPerWarp; ++c) {
    if (r_rank[c] == 0xffffffffu) continue;
    uint32_t d = digit_of(r_key[c], shift);
    uint32_t pos = s_base[d] + s_warp_hist[warp][d] + r_rank[c];
    keys_out[pos] = r_key[c];
    if (!kLast)
      vals_out[pos] = r_val[c];
    else
      S.perm[pos] = (int32_t)r_val[c];
  }
  }
}

// Gather the state into sorted order (out[k] = in[perm[k]]: perm is close to
// the identity because the input is the previous substep's sorted order, so
// the reads are nearly coalesced) and write the cell table entry
// {start, count, epoch, 0} of every occupied cell at 1 + its linear index.
template <typename T>
__global__ void __launch_bounds__(256) k_permute_table(DGrid G, int64_t n, const uint32_t* __restrict__ keys,
                                                       int32_t* __restrict__ perm, ScatterState S,
                                                       uint4* __restrict__ table, uint32_t* status,
                                                       const uint32_t* gate) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  if (sort_skipped(gate)) return;  // the caller copied the state in its current order
  int32_t src = perm[k];
  int32_t c = S.in_cell[src];
  pos_t<T> p = ((const pos_t<T>*)S.in_pos)[src];
  S.out_cell[k] = c;
  ((pos_t<T>*)S.out_pos)[k] = p;
  ((vec_t<T>*)S.out_vel)[k] = ((const vec_t<T>*)S.in_vel)[src];
  if (S.out_id) S.out_id[k] = S.in_id ? S.in_id[src] : src;
  if constexpr (sizeof(T) == 4) {
    if (S.out_posf)
      S.out_posf[k] = posf_of(c, p);
  }
  uint32_t key = keys[k];
  if (k > 0 && keys[k - 1] == key) return;
  int64_t e = k + 1;
  while (e < n && keys[e] == key) ++e;
  int x = cell_x(c), y = cell_y(c), z = cell_z(c);
  if (x >= G.nc[0] || y >= G.nc[1] || z >= G.nc[2]) {
    raise_status(status, GIC_STATUS_BAD_CELL);
    return;
  }
  uint32_t epoch = table[0].x;
  table[table_index(G, x, y, z)] = make_uint4((uint32_t)k, (uint32_t)(e - k), epoch, 0u);
}

template <typename T>
static int launch_sort(const DGrid& G, const GicGranules* in, GicGranules* out, int32_t* perm, uint4* table,
                       char* ws, const SortLayout& L, cudaStream_t st, const uint32_t* gate = nullptr) {
  int64_t n = in->n;
  uint32_t* keys_a = (uint32_t*)(ws + L.off_keys_a);
  uint32_t* vals_a = (uint32_t*)(ws + L.off_vals_a);
  uint32_t* keys_b = (uint32_t*)(ws + L.off_keys_b);
  uint32_t* vals_b = (uint32_t*)(ws + L.off_vals_b);
  uint32_t* counts = (uint32_t*)(ws + L.off_counts);
  uint32_t* totals = (uint32_t*)(ws + L.off_totals);
  ScatterState S{in->cell, in->pos,  in->vel, in->id, out->cell,
                 out->pos, out->vel, out->id, perm, sizeof(T) == 4 ? (float4*)out->posf : nullptr};
  const uint32_t* kin = nullptr;
  const uint32_t* vin = nullptr;
  uint32_t* kout = keys_a;
  uint32_t* vout = vals_a;
  int launches = 0;
  const int grid_ctas = (gate && L.tiles > kMaxSortCtas) ? kMaxSortCtas : L.tiles;
  for (int p = 0; p < L.passes; ++p) {
    int shift = 8 * p;
    bool first = p == 0, last = p == L.passes - 1;
    if (first)
      k_upsweep<true><<<grid_ctas, kSortThreads, 0, st>>>(n, shift, in->cell, nullptr, counts, L.tiles, gate);
    else
      k_upsweep<false><<<grid_ctas, kSortThreads, 0, st>>>(n, shift, nullptr, kin, counts, L.tiles, gate);
    k_scan_tiles<<<kRadix, kSortThreads, 0, st>>>(counts, L.tiles, totals, first ? table : nullptr, gate);
    if (first && last)
      k_downsweep<true, true, T><<<grid_ctas, kSortThreads, 0, st>>>(n, shift, kin, vin, kout, vout, counts, totals,
                                                                    L.tiles, S, gate);
    else if (first)
      k_downsweep<true, false, T><<<grid_ctas, kSortThreads, 0, st>>>(n, shift, kin, vin, kout, vout, counts, totals,
                                                                     L.tiles, S, gate);
    else if (last)
      k_downsweep<false, true, T><<<grid_ctas, kSortThreads, 0, st>>>(n, shift, kin, vin, kout, vout, counts, totals,
                                                                     L.tiles, S, gate);
    else
      k_downsweep<false, false, T><<<grid_ctas, kSortThreads, 0, st>>>(n, shift, kin, vin, kout, vout, counts, totals,
                                                                      L.tiles, S, gate);
    launches += 3;
    kin = kout;
    vin = vout;
    kout = (kout == keys_a) ? keys_b : keys_a;
    vout = (vout == vals_a) ? vals_b : vals_a;
  }
  // kin now holds the sorted keys
  k_permute_table<T><<<grid_blocks(n, 256), 256, 0, st>>>(G, n, kin, perm, S, table, status_word(), gate);
  launches += 1;
  count_launches(launches);
  GIC_CHECK_LAUNCH("gic_sort");
  return GIC_OK;
}

}  // namespace gic

using namespace gic;

extern "C" int gic_workspace_size(const GicGrid* grid, int64_t n, int32_t precision, size_t* bytes) {
  GIC_RANGE("gic_workspace_size");
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if (!bytes) return set_error(GIC_ERR_INVALID, "bytes is NULL");
  if (n < 0) return set_error(GIC_ERR_INVALID, "n < 0");
  if (precision != GIC_FP32 && precision != GIC_FP64) return set_error(GIC_ERR_INVALID, "bad precision");
  *bytes = sort_layout(G, n).total;
  return GIC_OK;
}

extern "C" int gic_sort(const GicGrid* grid, const GicGranules* in, GicGranules* out, int32_t* perm, void* cell_table,
                        void* ws, size_t ws_bytes, gic_stream_t stream) {
  GIC_RANGE("gic_sort");
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if ((rc = check_granules(in, "gic_sort in"))) return rc;
  if ((rc = check_granules(out, "gic_sort out"))) return rc;
  if (in->n != out->n || in->precision != out->precision)
    return set_error(GIC_ERR_INVALID, "gic_sort: in/out size or precision differ");
  if (!cell_table) return set_error(GIC_ERR_INVALID, "gic_sort: cell_table is NULL");
  if ((uintptr_t)cell_table % 16) return set_error(GIC_ERR_ALIGN, "gic_sort: cell_table must be 16-byte aligned");
  int64_t n = in->n;
  if (n == 0) return GIC_OK;
  if (!perm) return set_error(GIC_ERR_INVALID, "gic_sort: perm is NULL");
  if (in->cell == out->cell || in->pos == out->pos || in->vel == out->vel)
    return set_error(GIC_ERR_INVALID, "gic_sort: in and out must not alias");
  SortLayout L = sort_layout(G, n);
  if (!ws || ws_bytes < L.total)
    return set_error(GIC_ERR_WORKSPACE, "gic_sort: workspace of %zu bytes needed, %zu given", L.total, ws_bytes);
  if ((uintptr_t)ws % 256) return set_error(GIC_ERR_ALIGN, "gic_sort: workspace must be 256-byte aligned");
  if (in->precision == GIC_FP32)
    return launch_sort<float>(G, in, out, perm, (uint4*)cell_table, (char*)ws, L, (cudaStream_t)stream);
  return launch_sort<double>(G, in, out, perm, (uint4*)cell_table, (char*)ws, L, (cudaStream_t)stream);
}

namespace gic {

int sort_gated(const GicGrid* grid, const GicGranules* in, GicGranules* out, int32_t* perm, void* cell_table, void* ws,
               size_t ws_bytes, const uint32_t* gate, cudaStream_t stream) {
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if ((rc = check_granules(in, "gic_step state"))) return rc;
  if ((rc = check_granules(out, "gic_step sorted"))) return rc;
  if (in->n != out->n || in->precision != out->precision)
    return set_error(GIC_ERR_INVALID, "gic_step: state/sorted size or precision differ");
  if (!cell_table) return set_error(GIC_ERR_INVALID, "gic_step: cell_table is NULL");
  if ((uintptr_t)cell_table % 16) return set_error(GIC_ERR_ALIGN, "gic_step: cell_table must be 16-byte aligned");
  int64_t n = in->n;
  if (n == 0) return GIC_OK;
  if (!perm) return set_error(GIC_ERR_INVALID, "gic_step: perm is NULL");
  if (in->cell == out->cell || in->pos == out->pos || in->vel == out->vel)
    return set_error(GIC_ERR_INVALID, "gic_step: state and sorted must not alias");
  SortLayout L = sort_layout(G, n);
  if (!ws || ws_bytes < L.total)
    return set_error(GIC_ERR_WORKSPACE, "gic_step: workspace of %zu bytes needed, %zu given", L.total, ws_bytes);
  if ((uintptr_t)ws % 256) return set_error(GIC_ERR_ALIGN, "gic_step: workspace must be 256-byte aligned");
  if (in->precision == GIC_FP32)
    return launch_sort<float>(G, in, out, perm, (uint4*)cell_table, (char*)ws, L, stream, gate);
  return launch_sort<double>(G, in, out, perm, (uint4*)cell_table, (char*)ws, L, stream, gate);
}

}  // namespace gic

// ----------------------------------------------------------------- adjoint

namespace gic {
template <typename T>
__global__ void k_sort_adj(int64_t n, const int32_t* __restrict__ perm, const vec_t<T>* __restrict__ gpo,
                           const vec_t<T>* __restrict__ gvo, vec_t<T>* __restrict__ gpi, vec_t<T>* __restrict__ gvi) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  int32_t s = perm[k];
  if (gpi) gpi[s] = gpo[k];
  if (gvi) gvi[s] = gvo[k];
}
}  // namespace gic

extern "C" int gic_sort_adj(int64_t n, int32_t precision, const int32_t* perm, const void* g_pos_out,
                            const void* g_vel_out, void* g_pos_in, void* g_vel_in, gic_stream_t stream) {
  GIC_RANGE("gic_sort_adj");
  if (n < 0) return set_error(GIC_ERR_INVALID, "gic_sort_adj: n < 0");
  if (n == 0) return GIC_OK;
  if (!perm) return set_error(GIC_ERR_INVALID, "gic_sort_adj: perm is NULL");
  if ((g_pos_in && !g_pos_out) || (g_vel_in && !g_vel_out))
    return set_error(GIC_ERR_INVALID, "gic_sort_adj: missing upstream gradient");
  if (precision == GIC_FP32 || precision == GIC_FP64) {
    int rc = check_vecs(precision, "gic_sort_adj", {g_pos_out, g_vel_out, g_pos_in, g_vel_in});
    if (rc) return rc;
  }
  if (precision == GIC_FP32)
    k_sort_adj<float><<<grid_blocks(n, 256), 256, 0, stream>>>(n, perm, (const float4*)g_pos_out,
                                                                (const float4*)g_vel_out, (float4*)g_pos_in,
                                                                (float4*)g_vel_in);
  else if (precision == GIC_FP64)
    k_sort_adj<double><<<grid_blocks(n, 256), 256, 0, stream>>>(n, perm, (const d4*)g_pos_out, (const d4*)g_vel_out,
                                                                 (d4*)g_pos_in, (d4*)g_vel_in);
  else
    return set_error(GIC_ERR_INVALID, "gic_sort_adj: bad precision");
  count_launches(1);
  GIC_CHECK_LAUNCH("gic_sort_adj");
  return GIC_OK;
}

// ----------------------------------------------------------------- sort without a caller workspace
//
// For callers that cannot allocate device memory themselves -- code running
// where a cudaMalloc would be unsafe or unavailable, such as inside a host
// callback, a signal-free real-time loop, or a host that hands the library
// only pre-registered buffers -- this variant takes its radix-sort scratch
// from a fixed array compiled into the library instead of a workspace
// argument.  The array exists once per device that loads the library and
// lives until the process exits.

namespace gic {

// Largest granule count the static scratch holds.
constexpr int64_t kStaticSortMaxN = 1 << 18;  // 262,144 granules
constexpr int kStaticSortTiles = (int)((kStaticSortMaxN + kTile - 1) / kTile);
// keys and values ping-pong (4 x n x 4 B) + per-tile digit counts + digit totals
constexpr size_t kStaticSortBytes =
    4 * ((sizeof(uint32_t) * kStaticSortMaxN + 255) & ~(size_t)255) +
    ((sizeof(uint32_t) * (size_t)kRadix * kStaticSortTiles + 255) & ~(size_t)255) +
    ((sizeof(uint32_t) * kRadix + 255) & ~(size_t)255);

static __device__ __align__(256) unsigned char g_static_sort_scratch[kStaticSortBytes];

// Device address of the static scratch on the current device (host code may
// not use the symbol's name as an address).  It is looked up on every call
// rather than cached: a cudaDeviceReset in the same process reloads the
// module, after which a cached address would point at freed memory.  The
// lookup allocates nothing; the first one on a device loads the module
// (lazy loading), which is why that first call must precede any stream
// capture.
static int static_scratch(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_sort_scratch);
  if (e != cudaSuccess || !p)
    return set_error(GIC_ERR_CUDA, "gic_sort_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
  *out = p;
  return GIC_OK;
}

}  // namespace gic

extern "C" int64_t gic_sort_static_max_n(void) { return gic::kStaticSortMaxN; }

extern "C" int gic_sort_static(const GicGrid* grid, const GicGranules* in, GicGranules* out, int32_t* perm,
                               void* cell_table, gic_stream_t stream) {
  GIC_RANGE("gic_sort_static");
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if ((rc = check_granules(in, "gic_sort_static in"))) return rc;
  if ((rc = check_granules(out, "gic_sort_static out"))) return rc;
  if (in->n != out->n || in->precision != out->precision)
    return set_error(GIC_ERR_INVALID, "gic_sort_static: in/out size or precision differ");
  if (in->n > kStaticSortMaxN)
    return set_error(GIC_ERR_INVALID, "gic_sort_static: %lld granules exceed the static scratch limit of %lld",
                     (long long)in->n, (long long)kStaticSortMaxN);
  if (!cell_table) return set_error(GIC_ERR_INVALID, "gic_sort_static: cell_table is NULL");
  if ((uintptr_t)cell_table % 16) return set_error(GIC_ERR_ALIGN, "gic_sort_static: cell_table must be 16-byte aligned");
  int64_t n = in->n;
  if (n == 0) return GIC_OK;
  if (!perm) return set_error(GIC_ERR_INVALID, "gic_sort_static: perm is NULL");
  if (in->cell == out->cell || in->pos == out->pos || in->vel == out->vel)
    return set_error(GIC_ERR_INVALID, "gic_sort_static: in and out must not alias");
  void* scratch = nullptr;
  if ((rc = static_scratch(&scratch))) return rc;
  // Every pass writes the scratch regions it later reads (all tile counts in
  // the upsweep, keys and values in the downsweep), so the previous call's
  // contents need no clearing.
  SortLayout L = sort_layout(G, n);
  if (L.total > kStaticSortBytes) return set_error(GIC_ERR_INVALID, "gic_sort_static: scratch layout too large");
  if (in->precision == GIC_FP32)
    return launch_sort<float>(G, in, out, perm, (uint4*)cell_table, (char*)scratch, L, (cudaStream_t)stream);
  return launch_sort<double>(G, in, out, perm, (uint4*)cell_table, (char*)scratch, L, (cudaStream_t)stream);
}
