// gic_contact.cu -- a2: DEM contact forces and their adjoint.
//
// Gather form: one thread per granule of the sorted state walks the 27
// contact cells around its own (h_c >= 2 r_max), reads each partner's
// position / velocity and sums the pair forces on itself.  No atomics.  The
// adjoint uses the antisymmetry F_ji = -F_ij, so it is a gather as well:
// dL/dx_i = sum_j (dF_ij/dx_ij)^T (lambda_i - lambda_j).
//
// Contact law (Sec. 3.1, Eq. k_n), polydisperse and with the readings of this
// library: n = x_ij / d, overlap = r_i + r_j - d,
//   F_n = (k_n overlap - c_n v_n) n,   c_n = 2 zeta sqrt(k_n m_eff),
//   f_t = -k_t v_t,  k_t = kt_over_cn c_n,   F_t = min(|f_t|, mu |F_n|) f_t/|f_t|.
// Walls are partners of infinite mass at rest (m_eff = m_i).
#include "gic_contact.cuh"

namespace gic {

template <typename T>
__global__ void __launch_bounds__(128) k_contact(DGrid G, DParams<T> P, int64_t n, const int32_t* __restrict__ cell,
                                                  const pos_t<T>* __restrict__ pos, const float4* __restrict__ posf,
                                                  const vec_t<T>* __restrict__ vel, const uint4* __restrict__ table,
                                                  vec_t<T>* __restrict__ F, uint32_t* status) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t ci = cell[i];
  int cx, cy, cz;
  load_cell_coords<T>(ci, cx, cy, cz);
  pos_t<T> pi = pos[i];
  vec_t<T> vi = vel[i];
  T ri = radius_of(pi);
  T mi = granule_mass(P, ri);
  uint32_t epoch = __ldg(&table[0].x);
  if (T(2) * ri > (T)G.hc) raise_status(status, GIC_STATUS_RADIUS);
  T F0 = 0, F1 = 0, F2 = 0;
  bool coincident = false;
  for_each_contact<T>(G, table, epoch, i, cx, cy, cz, pi, ri, pos, posf, [&](int64_t j, const PairGeom<T>& g) {
    vec_t<T> vj = ldg(&vel[j]);
    T mj = granule_mass(P, radius_of(ldg(&pos[j])));
    T f0, f1, f2;
    if (pair_force(P, g.x0, g.x1, g.x2, g.d, g.overlap, vi.x - vj.x, vi.y - vj.y, vi.z - vj.z, mi * mj / (mi + mj), f0,
                   f1, f2)) {
      F0 += f0;
      F1 += f1;
      F2 += f2;
    } else {
      coincident = true;
    }
  });
  if (P.walls) {
    const int c3[3] = {cx, cy, cz};
    for (int a = 0; a < 3; ++a) {
      for (int side = 0; side < 2; ++side) {
        if (side == 0 ? c3[a] != 0 : c3[a] != G.nc[a] - 1) continue;
        T gap, ov;
        if (!wall_geom(G, pi, a, side, ri, gap, ov)) continue;
        T x[3] = {0, 0, 0};
        x[a] = side == 0 ? gap : -gap;
        T f0, f1, f2;
        if (pair_force(P, x[0], x[1], x[2], gap, ov, vi.x, vi.y, vi.z, mi, f0, f1, f2)) {
          F0 += f0;
          F1 += f1;
          F2 += f2;
        } else {
          raise_status(status, GIC_STATUS_OUT_OF_DOMAIN);
        }
      }
    }
  }
  if (coincident) raise_status(status, GIC_STATUS_COINCIDENT);
  if (!isfinite(F0) || !isfinite(F1) || !isfinite(F2)) raise_status(status, GIC_STATUS_NONFINITE);
  F[i] = make_vec<T>(F0, F1, F2);
}

// ----------------------------------------------------------------- staged FP32 contact
//
// One CTA = 128 consecutive granules of the Morton-sorted state: a compact
// blob of contact cells.  The CTA stages the cell-table entries of the
// blob's bounding box (+1 cell halo) and the float positions of every
// granule in those cells in shared memory, then each thread walks its 27
// neighbour cells there.  A CTA whose box or granule count exceeds the
// shared-memory budget (a Morton range that jumps across the domain) takes
// the global-memory path instead; the results are identical.

constexpr int kTileThreads = 128;
constexpr int kTileMaxCells = 512;
constexpr int kTileMaxGranules = 1152;

__device__ __forceinline__ void add_pair_force(const DParams<float>& P, const PairGeom<float>& g, const float4& vi,
                                               const float4& vj, float mi, float mj, float& F0, float& F1, float& F2,
                                               bool& coincident) {
  float f0, f1, f2;
  if (pair_force(P, g.x0, g.x1, g.x2, g.d, g.overlap, vi.x - vj.x, vi.y - vj.y, vi.z - vj.z, mi * mj / (mi + mj), f0,
                 f1, f2)) {
    F0 += f0;
    F1 += f1;
    F2 += f2;
  } else {
    coincident = true;
  }
}

// The CTA's staged neighbourhood in shared memory.
struct TileShared {
  int lo[3], hi[3];
  uint32_t start[kTileMaxCells];
  uint32_t cnt[kTileMaxCells];
  uint32_t off[kTileMaxCells + 1];
  float4 pf[kTileMaxGranules];
  uint32_t wsum[kTileThreads / 32];
  int mode;             // 0: staged, 1: global fallback
  unsigned rmax_bits;   // the largest staged radius (float bits)
};

struct TileBox {
  int bx0, by0, bz0, bx, by, bz;
};

// CTA-wide (every thread calls it): the bounding box of the CTA's contact
// cells with a one-cell halo, clipped to the grid; its table entries (start,
// count of this epoch), their exclusive scan and the float positions of every
// granule in the box, relative to the box corner.  sh.mode = 1 when the box or
// its granules exceed the tile.  valid / ci: this thread's granule and cell.
__device__ __forceinline__ TileBox tile_stage(TileShared& sh, const DGrid& G, const uint4* __restrict__ table,
                                              uint32_t epoch, const float4* __restrict__ posf, bool valid,
                                              int32_t ci) {
  if (threadIdx.x < 3) {
    sh.lo[threadIdx.x] = 1 << 30;
    sh.hi[threadIdx.x] = -1;
  }
  if (threadIdx.x == 0) sh.rmax_bits = 0u;
  __syncthreads();
  if (valid) {
    atomicMin(&sh.lo[0], cell_x(ci));
    atomicMin(&sh.lo[1], cell_y(ci));
    atomicMin(&sh.lo[2], cell_z(ci));
    atomicMax(&sh.hi[0], cell_x(ci));
    atomicMax(&sh.hi[1], cell_y(ci));
    atomicMax(&sh.hi[2], cell_z(ci));
  }
  __syncthreads();
  TileBox T;
  T.bx0 = max(sh.lo[0] - 1, 0);
  T.by0 = max(sh.lo[1] - 1, 0);
  T.bz0 = max(sh.lo[2] - 1, 0);
  T.bx = min(sh.hi[0] + 1, G.nc[0] - 1) - T.bx0 + 1;
  T.by = min(sh.hi[1] + 1, G.nc[1] - 1) - T.by0 + 1;
  T.bz = min(sh.hi[2] + 1, G.nc[2] - 1) - T.bz0 + 1;
  const int ncell = T.bx * T.by * T.bz;
  if (threadIdx.x == 0) sh.mode = (ncell > kTileMaxCells || sh.hi[0] < 0) ? 1 : 0;
  __syncthreads();
  if (sh.mode == 0) {
    // stage the table entries of the box
    // box index -> coordinates with float reciprocals (exact for these small integers)
    const float ibx = 1.0f / (float)T.bx, ibxy = 1.0f / (float)(T.bx * T.by);
    constexpr int kU = 4;  // loads in flight per thread
    for (int b0 = threadIdx.x; b0 < ncell; b0 += kU * kTileThreads) {
      uint4 e[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int b = b0 + u * kTileThreads;
        if (b >= ncell) break;
        int z = (int)(((float)b + 0.5f) * ibxy);
        int rem = b - z * T.bx * T.by;
        int y = (int)(((float)rem + 0.5f) * ibx);
        int x = T.bx0 + rem - y * T.bx;
        y += T.by0;
        z += T.bz0;
        e[u] = __ldg(&table[table_index(G, x, y, z)]);
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int b = b0 + u * kTileThreads;
        if (b >= ncell) break;
        const bool ok = e[u].z == epoch;
        sh.start[b] = ok ? e[u].x : 0u;
        sh.cnt[b] = ok ? e[u].y : 0u;
      }
    }
    __syncthreads();
    // exclusive scan of the counts (ncell <= 512: 4 per thread)
    {
      const int per = (kTileMaxCells + kTileThreads - 1) / kTileThreads;
      uint32_t loc[per];
      uint32_t sum = 0;
#pragma unroll
      for (int k = 0; k < per; ++k) {
        int b = threadIdx.x * per + k;
        loc[k] = b < ncell ? sh.cnt[b] : 0u;
        sum += loc[k];
      }
      uint32_t incl = sum;
      for (int off = 1; off < 32; off <<= 1) {
        uint32_t o = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane_id() >= off) incl += o;
      }
      if (lane_id() == 31) sh.wsum[threadIdx.x >> 5] = incl;
      __syncthreads();
      uint32_t base = 0;
      for (int w = 0; w < (threadIdx.x >> 5); ++w) base += sh.wsum[w];
      uint32_t run = base + incl - sum;
#pragma unroll
      for (int k = 0; k < per; ++k) {
        int b = threadIdx.x * per + k;
        if (b < kTileMaxCells) sh.off[b] = run;
        run += loc[k];
      }
      if (threadIdx.x == kTileThreads - 1) sh.off[kTileMaxCells] = run;
    }
    __syncthreads();
    const uint32_t total = sh.off[kTileMaxCells];
    if (total > (uint32_t)kTileMaxGranules) {
      if (threadIdx.x == 0) sh.mode = 1;
    } else {
      // stage the float positions: slot t belongs to cell b with off[b] <= t < off[b + 1]
      float rmax = 0.f;
      for (uint32_t t0 = threadIdx.x; t0 < total; t0 += kU * kTileThreads) {
        float4 pv[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const uint32_t t = t0 + u * kTileThreads;
          if (t >= total) break;
          int lo = 0, hi = ncell - 1;  // last b with off[b] <= t
          while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (sh.off[mid] <= t) lo = mid;
            else hi = mid - 1;
          }
          pv[u] = __ldg(&posf[sh.start[lo] + (t - sh.off[lo])]);
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const uint32_t t = t0 + u * kTileThreads;
          if (t >= total) break;
          // position in units of contact cells relative to the box corner (exact
          // differences of the absolute copies): the three cells of an x-row are
          // consecutive slots, and no cell offset is needed
          const float4 p = pv[u];
          sh.pf[t] = make_float4(p.x - (float)T.bx0, p.y - (float)T.by0, p.z - (float)T.bz0, p.w);
          rmax = fmaxf(rmax, p.w);
        }
      }
      const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(rmax));  // radii >= 0
      if (lane_id() == 0) atomicMax(&sh.rmax_bits, m);
    }
    __syncthreads();
  }
  return T;
}

__global__ void __launch_bounds__(kTileThreads) k_contact_tile(DGrid G, DParams<float> P, int64_t n,
                                                               const int32_t* __restrict__ cell,
                                                               const uint4* __restrict__ pos,
                                                               const float4* __restrict__ posf,
                                                               const float4* __restrict__ vel,
                                                               const uint4* __restrict__ table,
                                                               float4* __restrict__ F, uint32_t* status) {
  __shared__ TileShared sh;
  const int64_t i = blockIdx.x * (int64_t)kTileThreads + threadIdx.x;
  const bool valid = i < n;
  const uint32_t epoch = __ldg(&table[0].x);
  const int32_t ci = valid ? cell[i] : 0;
  const int cx = cell_x(ci), cy = cell_y(ci), cz = cell_z(ci);
  const TileBox T = tile_stage(sh, G, table, epoch, posf, valid, ci);
  const int bx0 = T.bx0, by0 = T.by0, bz0 = T.bz0, bx = T.bx, by = T.by, bz = T.bz;
  uint32_t* const s_start = sh.start;
  uint32_t* const s_off = sh.off;
  const float4* const s_pf = sh.pf;
  const int s_mode = sh.mode;
  if (!valid) return;
  const uint4 pi = pos[i];
  const float4 vi = vel[i];
  const float ri = __uint_as_float(pi.w);
  const float mi = granule_mass(P, ri);
  if (2.0f * ri > G.hc_f) raise_status(status, GIC_STATUS_RADIUS);
  float F0 = 0.f, F1 = 0.f, F2 = 0.f;
  bool coincident = false;
  if (s_mode == 0) {
    const int lx = cx - bx0, ly = cy - by0, lz = cz - bz0;
    const float4 fi0 = __ldg(&posf[i]);
    const float xi = fi0.x - (float)bx0, yi = fi0.y - (float)by0, zi = fi0.z - (float)bz0;
    const float rci = fmaf(ri, G.inv_hc_f, kPosfTol);
    const int xa = max(lx - 1, 0), xb = min(lx + 1, bx - 1);
    // own slot (excluded): own cell's first slot + rank inside the cell
    const int bown = lx + bx * (ly + by * lz);
    const uint32_t tself = s_off[bown] + (uint32_t)(i - (int64_t)s_start[bown]);
    for (int oz = -1; oz <= 1; ++oz) {
      int z = lz + oz;
      if (z < 0 || z >= bz) continue;
      for (int oy = -1; oy <= 1; ++oy) {
        int y = ly + oy;
        if (y < 0 || y >= by) continue;
        int row = bx * (y + by * z);
        uint32_t t0 = s_off[row + xa], t1 = s_off[row + xb + 1];
        for (uint32_t t = t0; t < t1; ++t) {
          float4 fj = s_pf[t];
          float rx = fj.x - xi, ry = fj.y - yi, rz = fj.z - zi;
          float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
          float Rc = fmaf(fj.w, G.inv_hc_f, rci);
          if (!(d2 < Rc * Rc) || t == tself) continue;
          // contact candidate: locate j and its cell offset, then the exact geometry
          int bj = row + xa;
          while (s_off[bj + 1] <= t) ++bj;
          uint32_t j = s_start[bj] + (t - s_off[bj]);
          int ox = (bj - row) - lx;
          uint4 pj = __ldg(&pos[j]);
          int Dx, Dy, Dz;
          int_sep(pi, pj, ox, oy, oz, Dx, Dy, Dz);
          PairGeom<float> g;
          if (!pair_geom_exact(G, Dx, Dy, Dz, ri, fj.w, g)) continue;
          add_pair_force(P, g, vi, __ldg(&vel[j]), mi, granule_mass(P, fj.w), F0, F1, F2, coincident);
        }
      }
    }
  } else {
    for_each_contact<float>(G, table, epoch, i, cx, cy, cz, pi, ri, pos, posf, [&](int64_t j, const PairGeom<float>& g) {
      add_pair_force(P, g, vi, __ldg(&vel[j]), mi, granule_mass(P, radius_of(__ldg(&pos[j]))), F0, F1, F2, coincident);
    });
  }
  if (P.walls) {
    const int c3[3] = {cx, cy, cz};
    for (int a = 0; a < 3; ++a) {
      for (int side = 0; side < 2; ++side) {
        if (side == 0 ? c3[a] != 0 : c3[a] != G.nc[a] - 1) continue;
        float gap, ov;
        if (!wall_geom(G, pi, a, side, ri, gap, ov)) continue;
        float x[3] = {0, 0, 0};
        x[a] = side == 0 ? gap : -gap;
        float f0, f1, f2;
        if (pair_force(P, x[0], x[1], x[2], gap, ov, vi.x, vi.y, vi.z, mi, f0, f1, f2)) {
          F0 += f0;
          F1 += f1;
          F2 += f2;
        } else {
          raise_status(status, GIC_STATUS_OUT_OF_DOMAIN);
        }
      }
    }
  }
  if (coincident) raise_status(status, GIC_STATUS_COINCIDENT);
  if (!isfinite(F0) || !isfinite(F1) || !isfinite(F2)) raise_status(status, GIC_STATUS_NONFINITE);
  F[i] = make_float4(F0, F1, F2, 0.f);
}

// The list build of gic_step's rebuilding substep (FP32 path with float
// copies, contact law only), on the staged neighbourhood: every granule's row
// -- the partners within r_i + r_j + skin by the float pre-test of
// verlet_pair, in the order of the 27-cell walk, slot = sorted index -- and its
// reference entries; no forces (the substep then walks the fresh rows, so the
// forces and their order are those of a build inside the substep).  The last
// CTA records the build; if a row overflowed it leaves the rebuild word set,
// and the substep's own 27-cell walk takes over as before.
__global__ void __launch_bounds__(kTileThreads) k_verlet_build_tile(DGrid G, int64_t n, const int32_t* __restrict__ cell,
                                                                    const uint4* __restrict__ pos,
                                                                    const float4* __restrict__ posf,
                                                                    const int32_t* __restrict__ id,
                                                                    const uint4* __restrict__ table, NbDev nb,
                                                                    float skin) {
  __shared__ TileShared sh;
  const bool rebuild = (nb.flags[kNbRebuild] | nb.flags[kNbSticky]) != 0u;  // uniform over the launch
  const int64_t i = blockIdx.x * (int64_t)kTileThreads + threadIdx.x;
  const bool valid = i < n;
  const uint32_t epoch = __ldg(&table[0].x);
  const int32_t ci = valid ? cell[i] : 0;
  const int cx = cell_x(ci), cy = cell_y(ci), cz = cell_z(ci);
  const TileBox T = tile_stage(sh, G, table, epoch, posf, valid, ci);
  if (valid && rebuild) {
    const uint4 pi = pos[i];
    const float ri = __uint_as_float(pi.w);
    const float4 fi = __ldg(&posf[i]);
    int32_t* row = nb.list + i * nb.cap;
    int cnt = 0;
    bool over = false;
    auto keep = [&](int64_t j) {
      if (cnt < nb.cap)
        row[cnt++] = (int32_t)j;
      else
        over = true;
    };
    if (sh.mode == 0) {
      const int lx = cx - T.bx0, ly = cy - T.by0, lz = cz - T.bz0;
      const float xi = fi.x - (float)T.bx0, yi = fi.y - (float)T.by0, zi = fi.z - (float)T.bz0;
      const int bown = lx + T.bx * (ly + T.by * lz);
      const uint32_t tself = sh.off[bown] + (uint32_t)(i - (int64_t)sh.start[bown]);
      // Cells farther than the largest pre-test radius of any staged partner
      // (plus a margin past the float rounding of d2) hold no partner: whole
      // rows (oy, oz) and the end cells of a row are skipped.  A staged copy
      // lies in its closed cell, so its distance is at least the cell's.
      const float Rmax = fmaf(ri + __uint_as_float(sh.rmax_bits) + skin, G.inv_hc_f, kPosfTol) + 1e-3f;
      const float R2 = Rmax * Rmax;
      const float dxl = xi - (float)lx, dxh = (float)(lx + 1) - xi;  // to the own cell's x faces
      for (int oz = -1; oz <= 1; ++oz) {
        const int z = lz + oz;
        if (z < 0 || z >= T.bz) continue;
        const float dz = oz < 0 ? zi - (float)lz : (oz > 0 ? (float)(lz + 1) - zi : 0.f);
        for (int oy = -1; oy <= 1; ++oy) {
          const int y = ly + oy;
          if (y < 0 || y >= T.by) continue;
          const float dy = oy < 0 ? yi - (float)ly : (oy > 0 ? (float)(ly + 1) - yi : 0.f);
          const float dyz = fmaf(dy, dy, dz * dz);
          if (dyz >= R2) continue;
          const int xa = (lx > 0 && fmaf(dxl, dxl, dyz) < R2) ? lx - 1 : lx;
          const int xb = (lx + 1 < T.bx && fmaf(dxh, dxh, dyz) < R2) ? lx + 1 : lx;
          const int rb = T.bx * (y + T.by * z);
          const uint32_t t0 = sh.off[rb + xa], t1 = sh.off[rb + xb + 1];
          for (uint32_t t = t0; t < t1; ++t) {
            if (t == tself) continue;
            const float4 fj = sh.pf[t];
            const float rx = fj.x - xi, ry = fj.y - yi, rz = fj.z - zi;
            const float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
            const float Rs = fmaf(ri + fj.w + skin, G.inv_hc_f, kPosfTol);
            if (d2 < Rs * Rs) {
              int bj = rb + xa;
              while (sh.off[bj + 1] <= t) ++bj;  // the cell of slot t (cells of the row in x order)
              keep((int64_t)sh.start[bj] + (t - sh.off[bj]));
            }
          }
        }
      }
    } else {
      for_each_partner(G, table, epoch, i, cx, cy, cz, [&](int64_t j, int, int, int) {
        const float4 fj = __ldg(&posf[j]);
        const float rx = fj.x - fi.x, ry = fj.y - fi.y, rz = fj.z - fi.z;
        const float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
        const float Rs = fmaf(ri + fj.w + skin, G.inv_hc_f, kPosfTol);
        if (d2 < Rs * Rs) keep(j);
      });
    }
    nb.count[i] = cnt;
    nb.at[i] = (int32_t)i;
    nb.cur[i] = (int32_t)i;
    nb.ref_cell[i] = ci;
    reinterpret_cast<uint4*>(nb.ref_pos)[i] = pi;
    const int32_t idi = id[i];
    if (idi >= 0 && (int64_t)idi < n) nb.slot[idi] = (int32_t)i;
    if (over) atomicOr(&nb.flags[kNbOverflow], 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&nb.flags[kNbCounter], 1u) == gridDim.x - 1) {
      __threadfence();
      if (rebuild && atomicExch(&nb.flags[kNbOverflow], 0u) == 0u) {  // a complete build: the substep walks it
        nb.flags[kNbSticky] = 0u;
        nb.flags[kNbRebuild] = 0u;
        nb.flags[kNbBuilds] += 1u;
      }
      nb.flags[kNbCounter] = 0u;
      __threadfence();
    }
  }
}

int launch_build_tile(const DGrid& G, const GicGranules* sorted, const void* table, const NbDev& d, double skin,
                      cudaStream_t stream) {
  if (sorted->n == 0) return GIC_OK;
  k_verlet_build_tile<<<grid_blocks(sorted->n, kTileThreads), kTileThreads, 0, stream>>>(
      G, sorted->n, sorted->cell, (const uint4*)sorted->pos, (const float4*)sorted->posf, sorted->id,
      (const uint4*)table, d, (float)skin);
  return GIC_OK;
}

// kList: walk the Verlet rows (nb) instead of the 27 cells; the last CTA
// then clears the per-call Verlet words.
template <typename T, bool kList>
__global__ void __launch_bounds__(128) k_contact_adj(DGrid G, DParams<T> P, int64_t n, const int32_t* __restrict__ cell,
                                                      const pos_t<T>* __restrict__ pos,
                                                      const float4* __restrict__ posf,
                                                      const vec_t<T>* __restrict__ vel, const uint4* __restrict__ table,
                                                      const vec_t<T>* __restrict__ gF, vec_t<T>* __restrict__ gpos,
                                                      vec_t<T>* __restrict__ gvel, double* __restrict__ g_mu,
                                                      NbDev nb) {
  bool rebuilt = false;
  if constexpr (kList) rebuilt = (nb.flags[kNbRebuild] | nb.flags[kNbSticky]) != 0u;
  __shared__ double s_red[32];
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double my_gmu = 0.0;
  if (i < n) {
    int32_t ci = cell[i];
    int cx, cy, cz;
    load_cell_coords<T>(ci, cx, cy, cz);
    pos_t<T> pi = pos[i];
    vec_t<T> vi = vel[i];
    vec_t<T> li = gF[i];
    T ri = radius_of(pi);
    T mi = granule_mass(P, ri);
    T gx0 = 0, gx1 = 0, gx2 = 0, gv0 = 0, gv1 = 0, gv2 = 0, gm = 0;
    auto pair = [&](int64_t j, const PairGeom<T>& g) {
      vec_t<T> vj = ldg(&vel[j]);
      vec_t<T> lj = ldg(&gF[j]);
      T mj = granule_mass(P, radius_of(ldg(&pos[j])));
      gm += pair_force_adj(P, g.x0, g.x1, g.x2, g.d, g.overlap, vi.x - vj.x, vi.y - vj.y, vi.z - vj.z,
                           mi * mj / (mi + mj), li.x - lj.x, li.y - lj.y, li.z - lj.z, li.x, li.y, li.z, gx0, gx1, gx2,
                           gv0, gv1, gv2);
    };
    if constexpr (kList) {
      const bool has_f = sizeof(T) == 4 && posf != nullptr;
      const float4 fi = has_f ? __ldg(&posf[i]) : make_float4(0.f, 0.f, 0.f, 0.f);
      for_each_list_contact<T>(G, nb, i, cx, cy, cz, ci, pi, ri, has_f, fi, cell, pos, posf, pair);
    } else {
      uint32_t epoch = __ldg(&table[0].x);
      for_each_contact<T>(G, table, epoch, i, cx, cy, cz, pi, ri, pos, posf, pair);
    }
    if (P.walls)
      gm += add_walls_adj(G, P, pi, ri, mi, vi, cx, cy, cz, li.x, li.y, li.z, gx0, gx1, gx2, gv0, gv1, gv2);
    vec_t<T> a = gpos[i];
    vec_t<T> b = gvel[i];
    gpos[i] = make_vec<T>(a.x + gx0, a.y + gx1, a.z + gx2);
    gvel[i] = make_vec<T>(b.x + gv0, b.y + gv1, b.z + gv2);
    my_gmu = (double)gm;
  }
  if (g_mu) {
    double s = block_sum(my_gmu, s_red);
    if (threadIdx.x == 0) atomicAdd(g_mu, s);
  }
  if constexpr (kList) verlet_call_done(nb, rebuilt);
}

// Diagnostic: number of partners per granule and the pair list by id.
template <typename T>
__global__ void k_contact_pairs(DGrid G, int64_t n, const int32_t* __restrict__ cell, const pos_t<T>* __restrict__ pos,
                                const float4* __restrict__ posf, const int32_t* __restrict__ id, const uint4* __restrict__ table,
                                int32_t* __restrict__ counts, int32_t* __restrict__ pairs, int64_t max_pairs,
                                unsigned long long* __restrict__ n_pairs) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int cx, cy, cz;
  load_cell_coords<T>(cell[i], cx, cy, cz);
  pos_t<T> pi = pos[i];
  T ri = radius_of(pi);
  int32_t idi = id ? id[i] : (int32_t)i;
  uint32_t epoch = __ldg(&table[0].x);
  int cnt = 0;
  for_each_contact<T>(G, table, epoch, i, cx, cy, cz, pi, ri, pos, posf, [&](int64_t j, const PairGeom<T>&) {
    ++cnt;
    int32_t idj = id ? id[j] : (int32_t)j;
    if (pairs && idi < idj) {
      unsigned long long slot = atomicAdd(n_pairs, 1ull);
      if ((int64_t)slot < max_pairs) {
        pairs[2 * slot] = idi;
        pairs[2 * slot + 1] = idj;
      }
    }
  });
  if (counts) counts[i] = cnt;
}

// Optional copy of the checked state into a second state (same order), for a
// caller whose sort may be skipped: cell, position record, velocity, id, the
// FP32 float positions and an identity permutation.
template <typename T>
struct StateCopy {
  const vec_t<T>* vel;
  int32_t* cell_out;
  pos_t<T>* pos_out;
  vec_t<T>* vel_out;
  int32_t* id_out;
  float4* posf_out;
  int32_t* perm_out;
};

template <typename T>
__global__ void __launch_bounds__(256) k_verlet_check(DGrid G, int64_t n, const int32_t* __restrict__ cell,
                                                       const pos_t<T>* __restrict__ pos,
                                                       const int32_t* __restrict__ id, NbDev nb, T lim2,
                                                       StateCopy<T> cp) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  bool far = false;
  if (i < n) {
    const int32_t c = cell[i];
    const pos_t<T> p = pos[i];
    const int32_t k = id[i];
    if (!nb.flags[kNbSticky]) {  // after a reset the slots are not set yet
      int32_t s = (k >= 0 && (int64_t)k < n) ? nb.slot[k] : -1;
      if (s >= 0 && (int64_t)s < n) {
        nb.cur[s] = (int32_t)i;
        nb.at[i] = s;
        far = moved_far(G, c, p, nb.ref_cell[s], reinterpret_cast<const pos_t<T>*>(nb.ref_pos)[s], lim2);
      } else {
        far = true;  // ids outside 0..n-1: rebuild (the build path does not need them)
      }
    }
    if (cp.cell_out) {
      cp.cell_out[i] = c;
      cp.pos_out[i] = p;
      cp.vel_out[i] = cp.vel[i];
      cp.id_out[i] = k;
      cp.perm_out[i] = (int32_t)i;
      if constexpr (sizeof(T) == 4) {
        if (cp.posf_out)
          cp.posf_out[i] = posf_of(c, p);
      }
    }
  }
  if (__any_sync(0xffffffffu, far) && lane_id() == 0) atomicOr(&nb.flags[kNbRebuild], 1u);
}

// kBuild = true: runs only when this call rebuilds -- walks the 27 cells,
// writes every row (slot = sorted index) and the forces.  kBuild = false:
// runs only when it does not -- walks the rows; its last CTA then clears the
// per-call words.  The two are launched back to back; the idle one exits.
template <typename T, bool kBuild>
__global__ void __launch_bounds__(kBuild ? 128 : 256, kBuild ? 1 : 4) k_contact_verlet(
    DGrid G, DParams<T> P, int64_t n, const int32_t* __restrict__ cell, const pos_t<T>* __restrict__ pos,
    const float4* __restrict__ posf, const vec_t<T>* __restrict__ vel, const int32_t* __restrict__ id,
    const uint4* __restrict__ table, NbDev nb, T skin, vec_t<T>* __restrict__ F, uint32_t* status) {
  const bool rebuild = (nb.flags[kNbRebuild] | nb.flags[kNbSticky]) != 0u;  // uniform over the launch
  if (kBuild && !rebuild) return;
  // the build runs on a capped grid (grid-stride), so that its idle launch on
  // the substeps that keep their lists is one short wave; the list walk has
  // one thread per granule
  const int64_t stride = kBuild ? (int64_t)gridDim.x * blockDim.x : n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; kBuild == rebuild && i < n; i += stride) {
    const int32_t ci = cell[i];
    const int cx = cell_x(ci), cy = cell_y(ci), cz = cell_z(ci);
    const pos_t<T> pi = pos[i];
    const vec_t<T> vi = vel[i];
    const T ri = radius_of(pi);
    const T mi = granule_mass(P, ri);
    if (T(2) * ri > (T)G.hc) raise_status(status, GIC_STATUS_RADIUS);
    const bool has_f = sizeof(T) == 4 && posf != nullptr;
    const float4 fi = has_f ? __ldg(&posf[i]) : make_float4(0.f, 0.f, 0.f, 0.f);
    T F0 = 0, F1 = 0, F2 = 0;
    bool coincident = false;
    if constexpr (kBuild) {
      verlet_build_granule(G, P, nb, table, n, i, cx, cy, cz, ci, pi, ri, mi, vi, has_f, fi, skin, id, pos, posf, vel,
                           F0, F1, F2, coincident);
    } else {
      verlet_list_force(G, P, nb, i, cx, cy, cz, ci, pi, ri, mi, vi, has_f, fi, cell, pos, posf, vel, F0, F1, F2,
                        coincident);
    }
    if (P.walls) add_walls(G, P, pi, ri, mi, vi, cx, cy, cz, F0, F1, F2, status);
    if (coincident) raise_status(status, GIC_STATUS_COINCIDENT);
    if (!isfinite(F0) || !isfinite(F1) || !isfinite(F2)) raise_status(status, GIC_STATUS_NONFINITE);
    F[i] = make_vec<T>(F0, F1, F2);
  }
  if constexpr (!kBuild) verlet_call_done(nb, rebuild);
}

__global__ void k_neighbors_reset(uint32_t* flags) {
  if (threadIdx.x < kNbWords) flags[threadIdx.x] = threadIdx.x == kNbSticky ? 1u : 0u;
}

static int check_table(const void* t) {
  if (!t) return set_error(GIC_ERR_INVALID, "cell_table is NULL");
  if ((uintptr_t)t % 16) return set_error(GIC_ERR_ALIGN, "cell_table must be 16-byte aligned");
  return GIC_OK;
}

}  // namespace gic

using namespace gic;

// The separate contact entry points evaluate the contact law only: the
// capillary bridges (sigma > 0) need the fluid fraction at both granules,
// which only the fused entry points receive.
static int reject_capillary(const GicParams* params, const char* what) {
  if (params && params->sigma != 0.0)
    return set_error(GIC_ERR_INVALID,
                     "%s: the capillary force (sigma > 0) is evaluated by gic_step / gic_substep only", what);
  return GIC_OK;
}

extern "C" int gic_contact(const GicGrid* grid, const GicParams* params, const GicGranules* s, const void* table,
                           void* F_c, gic_stream_t stream) {
  GIC_RANGE("gic_contact");
  if (int rc0 = reject_capillary(params, "gic_contact")) return rc0;
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if ((rc = check_granules(s, "gic_contact"))) return rc;
  if ((rc = check_table(table))) return rc;
  if (s->n == 0) return GIC_OK;
  if (!F_c) return set_error(GIC_ERR_INVALID, "gic_contact: F_c is NULL");
  if ((rc = check_vecs(s->precision, "gic_contact", {F_c}))) return rc;
  const int threads = 128;
  if (s->precision == GIC_FP32) {
    DParams<float> P;
    if ((rc = make_params(params, &P))) return rc;
    if (s->posf)
      k_contact_tile<<<grid_blocks(s->n, kTileThreads), kTileThreads, 0, stream>>>(
          G, P, s->n, s->cell, (const uint4*)s->pos, (const float4*)s->posf, (const float4*)s->vel,
          (const uint4*)table, (float4*)F_c, status_word());
    else
      k_contact<float><<<grid_blocks(s->n, threads), threads, 0, stream>>>(
          G, P, s->n, s->cell, (const uint4*)s->pos, nullptr, (const float4*)s->vel, (const uint4*)table,
          (float4*)F_c, status_word());
  } else {
    DParams<double> P;
    if ((rc = make_params(params, &P))) return rc;
    k_contact<double><<<grid_blocks(s->n, threads), threads, 0, stream>>>(
        G, P, s->n, s->cell, (const d4*)s->pos, nullptr, (const d4*)s->vel, (const uint4*)table, (d4*)F_c,
        status_word());
  }
  count_launches(1);
  GIC_CHECK_LAUNCH("gic_contact");
  return GIC_OK;
}

extern "C" int gic_contact_adj(const GicGrid* grid, const GicParams* params, const GicGranules* s, const void* table,
                               const void* gF_c, void* g_pos, void* g_vel, double* g_mu, gic_stream_t stream) {
  GIC_RANGE("gic_contact_adj");
  if (int rc0 = reject_capillary(params, "gic_contact_adj")) return rc0;
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if ((rc = check_granules(s, "gic_contact_adj"))) return rc;
  if ((rc = check_table(table))) return rc;
  if (s->n == 0) return GIC_OK;
  if (!gF_c || !g_pos || !g_vel) return set_error(GIC_ERR_INVALID, "gic_contact_adj: null gradient array");
  if ((rc = check_vecs(s->precision, "gic_contact_adj", {gF_c, g_pos, g_vel}))) return rc;
  const int threads = 128;
  if (s->precision == GIC_FP32) {
    DParams<float> P;
    if ((rc = make_params(params, &P))) return rc;
    k_contact_adj<float, false><<<grid_blocks(s->n, threads), threads, 0, stream>>>(
        G, P, s->n, s->cell, (const uint4*)s->pos, (const float4*)s->posf, (const float4*)s->vel, (const uint4*)table,
        (const float4*)gF_c, (float4*)g_pos, (float4*)g_vel, g_mu, NbDev{});
  } else {
    DParams<double> P;
    if ((rc = make_params(params, &P))) return rc;
    k_contact_adj<double, false><<<grid_blocks(s->n, threads), threads, 0, stream>>>(
        G, P, s->n, s->cell, (const d4*)s->pos, nullptr, (const d4*)s->vel, (const uint4*)table, (const d4*)gF_c,
        (d4*)g_pos, (d4*)g_vel, g_mu, NbDev{});
  }
  count_launches(1);
  GIC_CHECK_LAUNCH("gic_contact_adj");
  return GIC_OK;
}

extern "C" int gic_contact_pairs(const GicGrid* grid, const GicGranules* s, const void* table, int32_t* counts,
                                 int32_t* pairs, int64_t max_pairs, int64_t* n_pairs, gic_stream_t stream) {
  GIC_RANGE("gic_contact_pairs");
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if ((rc = check_granules(s, "gic_contact_pairs"))) return rc;
  if ((rc = check_table(table))) return rc;
  if (s->n == 0) return GIC_OK;
  if (pairs && !n_pairs) return set_error(GIC_ERR_INVALID, "gic_contact_pairs: n_pairs is NULL");
  if (s->precision == GIC_FP32)
    k_contact_pairs<float><<<grid_blocks(s->n, 128), 128, 0, stream>>>(G, s->n, s->cell, (const uint4*)s->pos,
                                                                        (const float4*)s->posf, s->id,
                                                                        (const uint4*)table, counts, pairs, max_pairs,
                                                                        (unsigned long long*)n_pairs);
  else
    k_contact_pairs<double><<<grid_blocks(s->n, 128), 128, 0, stream>>>(G, s->n, s->cell, (const d4*)s->pos, nullptr,
                                                                         s->id,
                                                                         (const uint4*)table, counts, pairs,
                                                                         max_pairs, (unsigned long long*)n_pairs);
  count_launches(1);
  GIC_CHECK_LAUNCH("gic_contact_pairs");
  return GIC_OK;
}

static int check_neighbors(const GicNeighbors* nb, const GicGranules* s, const char* what) {
  if (!nb) return set_error(GIC_ERR_INVALID, "%s: neighbours struct is NULL", what);
  if (!nb->list || !nb->count || !nb->ref_cell || !nb->ref_pos || !nb->slot || !nb->cur || !nb->at || !nb->flags)
    return set_error(GIC_ERR_INVALID, "%s: a neighbour array is NULL", what);
  if (nb->cap < 1) return set_error(GIC_ERR_INVALID, "%s: cap must be >= 1", what);
  if (!(nb->skin >= 0.0)) return set_error(GIC_ERR_INVALID, "%s: skin must be >= 0", what);
  if (s && nb->n != s->n) return set_error(GIC_ERR_INVALID, "%s: neighbour lists are for %lld granules, got %lld",
                                           what, (long long)nb->n, (long long)s->n);
  if (s && (uintptr_t)nb->ref_pos % (s->precision == GIC_FP32 ? 16 : 32))
    return set_error(GIC_ERR_ALIGN, "%s: ref_pos misaligned", what);
  return GIC_OK;
}

namespace gic {

// Grid of the list build: at most 2048 CTAs of 128 (grid-stride beyond).
static unsigned build_blocks(int64_t n) {
  unsigned b = grid_blocks(n, 128);
  return b < 2048u ? b : 2048u;
}

NbDev nb_dev(const DGrid& G, const GicNeighbors* nb, bool ident) {
  const double half = 0.5 * nb->skin;
  const double lim = half * G.inv_unit;  // skin / 2 in 2^-30 h_c units
  return NbDev{nb->cap, nb->list, nb->count, nb->ref_cell, nb->ref_pos, nb->slot, nb->cur, nb->at, nb->flags,
               ident ? 1 : 0, (float)(lim * lim), half * half, nb->n, G.dbg};
}

int verlet_view(const DGrid& G, const GicGranules* s, const void* table, const GicNeighbors* nb, const char* what,
                bool ident, NbDev* out) {
  int rc;
  if ((rc = check_table(table))) return rc;
  if ((rc = check_neighbors(nb, s, what))) return rc;
  *out = nb_dev(G, nb, ident);
  return GIC_OK;
}

int verlet_check(const DGrid& G, const GicGranules* s, const void* table, const GicNeighbors* nb,
                 cudaStream_t stream, const char* what, NbDev* out, GicGranules* copy_to, int32_t* perm) {
  int rc;
  if ((rc = check_table(table))) return rc;
  if ((rc = check_neighbors(nb, s, what))) return rc;
  const NbDev d = nb_dev(G, nb, false);
  *out = d;
  if (s->n == 0) return GIC_OK;
  if (copy_to && (!perm || !copy_to->id)) return set_error(GIC_ERR_INVALID, "%s: copy needs ids and perm", what);
  const double half = 0.5 * nb->skin;
  if (s->precision == GIC_FP32) {
    const double lim = half * G.inv_unit;  // skin / 2 in 2^-30 h_c units
    StateCopy<float> cp{};
    if (copy_to)
      cp = StateCopy<float>{(const float4*)s->vel, copy_to->cell, (uint4*)copy_to->pos, (float4*)copy_to->vel,
                            copy_to->id, (float4*)copy_to->posf, perm};
    k_verlet_check<float><<<grid_blocks(s->n, 256), 256, 0, stream>>>(G, s->n, s->cell, (const uint4*)s->pos, s->id, d,
                                                                      (float)(lim * lim), cp);
  } else {
    StateCopy<double> cp{};
    if (copy_to)
      cp = StateCopy<double>{(const d4*)s->vel, copy_to->cell, (d4*)copy_to->pos, (d4*)copy_to->vel, copy_to->id,
                             nullptr, perm};
    k_verlet_check<double><<<grid_blocks(s->n, 256), 256, 0, stream>>>(G, s->n, s->cell, (const d4*)s->pos, s->id, d,
                                                                       half * half, cp);
  }
  count_launches(1);
  return GIC_OK;
}

int verlet_prelude(const DGrid& G, const GicParams* params, const GicGranules* s, const void* table,
                   const GicNeighbors* nb, void* F_c, cudaStream_t stream, const char* what, NbDev* out,
                   bool launch_build) {
  int rc;
  if (launch_build && !F_c) return set_error(GIC_ERR_INVALID, "%s: F_c is NULL", what);
  if ((rc = check_vecs(s->precision, what, {F_c}))) return rc;
  if ((rc = verlet_check(G, s, table, nb, stream, what, out, nullptr, nullptr))) return rc;
  if (s->n == 0 || !launch_build) return GIC_OK;
  const NbDev d = *out;
  if (s->precision == GIC_FP32) {
    DParams<float> P;
    if ((rc = make_params(params, &P))) return rc;
    k_contact_verlet<float, true><<<build_blocks(s->n), 128, 0, stream>>>(
        G, P, s->n, s->cell, (const uint4*)s->pos, (const float4*)s->posf, (const float4*)s->vel, s->id,
        (const uint4*)table, d, (float)nb->skin, (float4*)F_c, status_word());
  } else {
    DParams<double> P;
    if ((rc = make_params(params, &P))) return rc;
    k_contact_verlet<double, true><<<build_blocks(s->n), 128, 0, stream>>>(
        G, P, s->n, s->cell, (const d4*)s->pos, nullptr, (const d4*)s->vel, s->id, (const uint4*)table, d, nb->skin,
        (d4*)F_c, status_word());
  }
  count_launches(1);
  return GIC_OK;
}

}  // namespace gic

extern "C" int gic_contact_verlet(const GicGrid* grid, const GicParams* params, const GicGranules* s,
                                  const void* table, const GicNeighbors* nb, void* F_c, gic_stream_t stream) {
  GIC_RANGE("gic_contact_verlet");
  if (int rc0 = reject_capillary(params, "gic_contact_verlet")) return rc0;
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if ((rc = check_granules(s, "gic_contact_verlet", true))) return rc;
  NbDev d;
  if ((rc = verlet_prelude(G, params, s, table, nb, F_c, stream, "gic_contact_verlet", &d, true))) return rc;
  if (s->n == 0) return GIC_OK;
  if (s->precision == GIC_FP32) {
    DParams<float> P;
    make_params(params, &P);
    k_contact_verlet<float, false><<<grid_blocks(s->n, 256), 256, 0, stream>>>(
        G, P, s->n, s->cell, (const uint4*)s->pos, (const float4*)s->posf, (const float4*)s->vel, s->id,
        (const uint4*)table, d, (float)nb->skin, (float4*)F_c, status_word());
  } else {
    DParams<double> P;
    make_params(params, &P);
    k_contact_verlet<double, false><<<grid_blocks(s->n, 256), 256, 0, stream>>>(
        G, P, s->n, s->cell, (const d4*)s->pos, nullptr, (const d4*)s->vel, s->id, (const uint4*)table, d, nb->skin,
        (d4*)F_c, status_word());
  }
  count_launches(1);
  GIC_CHECK_LAUNCH("gic_contact_verlet");
  return GIC_OK;
}

extern "C" int gic_neighbors_reset(const GicNeighbors* nb, gic_stream_t stream) {
  GIC_RANGE("gic_neighbors_reset");
  int rc = check_neighbors(nb, nullptr, "gic_neighbors_reset");
  if (rc) return rc;
  k_neighbors_reset<<<1, 32, 0, stream>>>(nb->flags);
  count_launches(1);
  GIC_CHECK_LAUNCH("gic_neighbors_reset");
  return GIC_OK;
}

namespace gic {
// A rebuild request (the sticky word's bit 0): the build kernel reads it and
// clears it after a complete build; after an overflow it stays, and the next
// call on these lists rebuilds.
__global__ void k_request_build(uint32_t* flags) { flags[kNbSticky] |= 1u; }
}  // namespace gic

extern "C" int gic_neighbors_build(const GicGrid* grid, const GicGranules* sorted, const void* cell_table,
                                   const GicNeighbors* nb, gic_stream_t stream) {
  GIC_RANGE("gic_neighbors_build");
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if ((rc = check_granules(sorted, "gic_neighbors_build", true))) return rc;
  if (sorted->precision != GIC_FP32 || !sorted->posf)
    return set_error(GIC_ERR_INVALID, "gic_neighbors_build: the staged build needs an FP32 state with posf");
  NbDev d;
  if ((rc = verlet_view(G, sorted, cell_table, nb, "gic_neighbors_build", true, &d))) return rc;
  if (sorted->n == 0) return GIC_OK;
  k_request_build<<<1, 1, 0, (cudaStream_t)stream>>>(nb->flags);
  if ((rc = launch_build_tile(G, sorted, cell_table, d, nb->skin, (cudaStream_t)stream))) return rc;
  count_launches(2);
  GIC_CHECK_LAUNCH("gic_neighbors_build");
  return GIC_OK;
}

extern "C" int gic_contact_verlet_adj(const GicGrid* grid, const GicParams* params, const GicGranules* s,
                                      const void* table, const GicNeighbors* nb, void* F_c, const void* gF_c,
                                      void* g_pos, void* g_vel, double* g_mu, gic_stream_t stream) {
  GIC_RANGE("gic_contact_verlet_adj");
  if (int rc0 = reject_capillary(params, "gic_contact_verlet_adj")) return rc0;
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if ((rc = check_granules(s, "gic_contact_verlet_adj", true))) return rc;
  if (s->n > 0 && (!gF_c || !g_pos || !g_vel))
    return set_error(GIC_ERR_INVALID, "gic_contact_verlet_adj: null gradient array");
  if ((rc = check_vecs(s->precision, "gic_contact_verlet_adj", {gF_c, g_pos, g_vel}))) return rc;
  NbDev d;
  if ((rc = verlet_prelude(G, params, s, table, nb, F_c, stream, "gic_contact_verlet_adj", &d, true))) return rc;
  if (s->n == 0) return GIC_OK;
  const int threads = 128;
  if (s->precision == GIC_FP32) {
    DParams<float> P;
    make_params(params, &P);
    k_contact_adj<float, true><<<grid_blocks(s->n, threads), threads, 0, stream>>>(
        G, P, s->n, s->cell, (const uint4*)s->pos, (const float4*)s->posf, (const float4*)s->vel, (const uint4*)table,
        (const float4*)gF_c, (float4*)g_pos, (float4*)g_vel, g_mu, d);
  } else {
    DParams<double> P;
    make_params(params, &P);
    k_contact_adj<double, true><<<grid_blocks(s->n, threads), threads, 0, stream>>>(
        G, P, s->n, s->cell, (const d4*)s->pos, nullptr, (const d4*)s->vel, (const uint4*)table, (const d4*)gF_c,
        (d4*)g_pos, (d4*)g_vel, g_mu, d);
  }
  count_launches(1);
  GIC_CHECK_LAUNCH("gic_contact_verlet_adj");
  return GIC_OK;
}
