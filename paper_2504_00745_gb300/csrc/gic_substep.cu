// gic_substep.cu -- one SandSubstep (Alg. 2) after the sort, fused into one
// pass over the sorted state: contact forces from the Verlet lists (or, on a
// substep that rebuilds them, from the 27-cell walk that builds them), the G2P coupling
// (Sec. 3.3), the virtual-mass integration (Sec. 5.2) into the next state,
// and the P2G scatter of F_s at the old positions and, when asked, of
// alpha_s at the new ones.  The per-granule force arrays of the separate
// entry points (F_c, F_fl, a_f, f_ex) never leave registers.
#include <string.h>

#include <mutex>
#include <type_traits>

#include "gic_capillary.cuh"
#include "gic_contact.cuh"
#include "gic_grid.cuh"
#include "gic_integrate.cuh"

namespace gic {

constexpr int kSubstepThreads = 256;
static_assert(kSubstepThreads == 32 * kSubWarps && kSubstepThreads + kSubstepThreads / 32 <= kSpreadStride,
              "the shared tile's warp arrays and the spread deposits are sized for CTAs of 256 threads");

// kKeep: the kernel of gic_step's list-keeping branch without the capillary
// force (its lists are valid by the branch's condition, so it carries neither
// the build nor the bridge code: a smaller instruction footprint); otherwise
// the general kernel, which reads from the list flags whether it rebuilds.
// kNoAlpha: a call without alpha_s (the kernel then carries none of its code).
template <typename T, bool kKeep, bool kNoAlpha = false>
__global__ void __launch_bounds__(kSubstepThreads, sizeof(T) == 4 ? 4 : 2) k_substep(
    DGrid G, DParams<T> P, int64_t n, const int32_t* __restrict__ cell, const pos_t<T>* __restrict__ pos,
    const float4* __restrict__ posf, const vec_t<T>* __restrict__ vel, const int32_t* __restrict__ id, NbDev nb,
    const uint4* __restrict__ table, T skin, Fields<T> Fd, int32_t* __restrict__ cell_out, pos_t<T>* __restrict__ pos_out,
    vec_t<T>* __restrict__ vel_out, int32_t* __restrict__ id_out, float4* __restrict__ posf_out,
    vec_t<T>* __restrict__ fex_out, double* __restrict__ alpha, T* __restrict__ Fs_u, T* __restrict__ Fs_v,
    T* __restrict__ Fs_w, double* __restrict__ sums, uint32_t* status) {
  __shared__ std::conditional_t<sizeof(T) == 4, SubTile, int> sh;  // FP32 path only
  const bool rebuild = !kKeep && (nb.flags[kNbRebuild] | nb.flags[kNbSticky]) != 0u;  // uniform over the launch
  const bool do_a = !kNoAlpha && alpha != nullptr, do_f = Fs_u != nullptr;
  const int64_t i = blockIdx.x * (int64_t)kSubstepThreads + threadIdx.x;
  const bool valid = i < n;
  const int32_t ci = valid ? cell[i] : 0;
  // the granule's own records, prefetched into L2 before the CTA's tile
  // barriers (the loads themselves come after them; no register is held)
  if (valid) {
    prefetch_l2(&pos[i]);
    prefetch_l2(&vel[i]);
    if (posf) prefetch_l2(&posf[i]);
    if (!rebuild) {
      const int32_t sl = nb.ident ? (int32_t)i : nb.at[i];
      prefetch_l2(&nb.count[sl]);  // (not the row: a whole line for a few entries)
      prefetch_l2(&nb.ref_cell[sl]);
      prefetch_l2(reinterpret_cast<const pos_t<T>*>(nb.ref_pos) + sl);
    }
  }
  // FP32: the CTA's tile (fields staged for G2P, F_s / alpha_s accumulators)
  SubBox B{};
  if constexpr (sizeof(T) == 4) B = sub_tile_begin(sh, G, Fd, valid, ci, do_a, do_f);

  int32_t co = 0;
  pos_t<T> pi{}, po{};
  T fe[3] = {T(0), T(0), T(0)};
  bool far = false;
  if (valid) {
    pi = pos[i];
    const vec_t<T> vi = vel[i];
    const T ri = radius_of(pi);
    const T mi = granule_mass(P, ri);
    uint32_t flags = 0;
    if (T(2) * ri > grid_hc<T>(G)) flags |= GIC_STATUS_RADIUS;
    // a2: contact
    T F0 = 0, F1 = 0, F2 = 0;
    bool coincident = false;
    {
      const int cx = cell_x(ci), cy = cell_y(ci), cz = cell_z(ci);
      const bool has_f = sizeof(T) == 4 && posf != nullptr;
      const float4 fi = has_f ? __ldg(&posf[i]) : make_float4(0.f, 0.f, 0.f, 0.f);
      if (!kKeep && P.cap) {  // with the capillary bridges (Sec. 5.4): contacts and bridge candidates
        const T sri = moisture_ratio_at(G, P, Fd.af, ci, pi, (T*)nullptr);
        auto near = [&](int64_t j, int32_t cj, const pos_t<T>& pj, const PairGeom<T>& g) {
          if (g.overlap > T(0))
            add_force(P, g, vi, ldg(&vel[j]), mi, granule_mass(P, radius_of(pj)), F0, F1, F2, coincident);
          else
            add_bridge(P, g, ri, radius_of(pj), sri, moisture_ratio_at(G, P, Fd.af, cj, pj, (T*)nullptr), F0, F1,
                       F2);
        };
        if (rebuild)
          verlet_build_row_near<T>(G, P, nb, table, n, i, cx, cy, cz, ci, pi, ri, skin, id, pos, near);
        else
          for_each_list_near<T>(G, P, nb, i, cx, cy, cz, pi, ri, has_f, fi, cell, pos, posf, near);
      } else if (rebuild) {  // this substep rebuilds the lists: walk the 27 cells
        verlet_build_granule(G, P, nb, table, n, i, cx, cy, cz, ci, pi, ri, mi, vi, has_f, fi, skin, id, pos, posf,
                             vel, F0, F1, F2, coincident);
      } else {
        verlet_list_force(G, P, nb, i, cx, cy, cz, ci, pi, ri, mi, vi, has_f, fi, cell, pos, posf, vel, F0, F1, F2,
                          coincident);
      }
      if (P.walls) {
        if constexpr (sizeof(T) == 4)
          add_walls_f32(G, P, pi, ri, mi, vi, cx, cy, cz, F0, F1, F2, status);
        else
          add_walls(G, P, pi, ri, mi, vi, cx, cy, cz, F0, F1, F2, status);
      }
      if (coincident) flags |= GIC_STATUS_COINCIDENT;
      if (!isfinite(F0) || !isfinite(F1) || !isfinite(F2)) flags |= GIC_STATUS_NONFINITE;
    }
    // a3: G2P coupling
    T Ffl[3], af[3];
    T sp;
    if constexpr (sizeof(T) == 4)
      sp = sub_g2p(sh, B, G, P, Fd, ci, pi, vi, Ffl, af);
    else
      sp = g2p_granule(G, P, Fd, ci, pi, vi, Ffl, af);
    if (!isfinite(sp)) flags |= GIC_STATUS_NONFINITE;
    // a4: integrate into the next state
    vec_t<T> vo;
    integrate_granule(G, P, ci, pi, vi, F0, F1, F2, Ffl[0], Ffl[1], Ffl[2], af[0], af[1], af[2], co, po, vo, fe[0],
                      fe[1], fe[2], flags);
    if (flags) raise_status(status, flags);
    cell_out[i] = co;
    pos_out[i] = po;
    vel_out[i] = vo;
    if (id_out && id) id_out[i] = id[i];
    if constexpr (sizeof(T) == 4) {
      if (posf_out)
        posf_out[i] = posf_of(co, po);
    }
    if (fex_out) fex_out[i] = make_vec<T>(fe[0], fe[1], fe[2]);
    // the next call's displacement test, on the positions just written
    // (after a build this call's positions are the reference)
    if (rebuild) {
      far = moved_far(G, co, po, ci, pi, nb_lim2(nb, T(0)));
    } else {
      const int32_t sl = nb.ident ? (int32_t)i : nb.at[i];
      far = moved_far(G, co, po, nb.ref_cell[sl], reinterpret_cast<const pos_t<T>*>(nb.ref_pos)[sl],
                      nb_lim2(nb, T(0)));
    }
  }
  if (__any_sync(0xffffffffu, far) && lane_id() == 0) atomicOr(&nb.flags[kNbNext], 1u);

  // a5: P2G
  if constexpr (sizeof(T) == 4) {
    const float fc[3] = {P.exch * fe[0], P.exch * fe[1], P.exch * fe[2]};
    float unit = 0.f, inv_unit = 0.f;
    const bool spread = do_f && !do_a && B.tile;  // uniform over the CTA
    if (do_f) {  // the CTA's fixed-point unit
      float Mt = 0.f;
      if (valid) {
        const float m = fmaxf(fabsf(fc[0]), fmaxf(fabsf(fc[1]), fabsf(fc[2])));
        Mt = m <= 3.0e38f ? m : INFINITY;  // NaN or inf: no fixed point for this CTA
      }
      if (spread) {  // park the deposit's inputs before the barrier in sub_fs_scale
        int m[3] = {0, 0, 0};
        float t[3] = {0.f, 0.f, 0.f};
        if (valid) granule_mac<float>(G, ci, pi, m, t);
        spread_put(sh, valid, m, t, fc);
      }
      inv_unit = sub_fs_scale(sh, B, Mt, unit);
    }
    float* Fs[3] = {Fs_u, Fs_v, Fs_w};
    unsigned long long S = 0;
    if (valid && do_a) {
      int ia[3];
      long long va[8];
      alpha_deposits(G, co, po, ia, va, S);
      sub_add_alpha(sh, B, G, (unsigned long long*)alpha, ia, va);
    }
    if (spread && inv_unit != 0.f) {
      spread_deposit(sh, B, G, Fs, inv_unit);
    } else if (kNoAlpha && valid && do_f) {  // inv_unit == 0 here: no tile for F_s
      fs_deposit_global(G, Fs_u, Fs_v, Fs_w, ci, pi, fc[0], fc[1], fc[2]);
    } else if (valid && do_f) {
      int m[3];
      float t[3];
      granule_mac<float>(G, ci, pi, m, t);
#pragma unroll
      for (int comp = 0; comp < 3; ++comp)
        sub_add_face(sh, B, G, Fs[comp], comp, make_stencil<float>(G, m, t, comp), fc[comp], inv_unit);
    }
    sub_tile_flush(sh, B, G, (unsigned long long*)alpha, Fs, do_a, inv_unit != 0.f, unit);
    if (sums) p2g_sums(sums, (long long)S);
  } else {
    // FP64: straight double atomics (alpha_s from V / dx^3 and the tent
    // weights at the new position, F_s at the old one)
    __shared__ double s_red[32];
    double Vi = 0.0;
    if (valid && do_a) {
      double r = (double)radius_of(po);
      Vi = 4.0 / 3.0 * kPi * r * r * r;
      int m[3];
      double t[3];
      granule_mac_fp64(G, co, po, m, t);
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
    if (valid && do_f) {
      int m[3];
      T t[3];
      granule_mac<T>(G, ci, pi, m, t);
      T* Fs[3] = {Fs_u, Fs_v, Fs_w};
#pragma unroll
      for (int comp = 0; comp < 3; ++comp) {
        Stencil3<T> St = make_stencil<T>(G, m, t, comp);
        const T fv = P.exch * fe[comp];
        const int nsx = St.ns[0], nsy = St.ns[1];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int b = 0; b < 2; ++b) {
            T wyz = (b ? St.w[1] : T(1) - St.w[1]) * (c ? St.w[2] : T(1) - St.w[2]) * fv;
            int64_t row = sample_index(nsx, nsy, St.i0[0], St.i0[1] + b, St.i0[2] + c);
            atomicAdd(&Fs[comp][row], (T(1) - St.w[0]) * wyz);
            atomicAdd(&Fs[comp][row + 1], St.w[0] * wyz);
          }
      }
    }
    if (sums) {
      double s = block_sum(Vi, s_red);
      if (threadIdx.x == 0) atomicAdd(&sums[1], s);
    }
  }
  verlet_call_done(nb, rebuild);
}

constexpr int kSubstepAdjThreads = 128;

// Adjoint of k_substep's granule outputs (next position, velocity, f_ex) for
// one granule of the sorted state: the integration's adjoint gives the
// granule's own F_c, F_fl and a_f gradients, the G2P adjoint adds its
// position and velocity parts, and the contact adjoint walks the granule's
// Verlet row (or the 27 cells, writing the row, on a substep that rebuilds
// it), forming each partner's F_c gradient from the partner's upstream
// gradients.  Writes the result through perm (the sort's scatter).
template <typename T>
__global__ void __launch_bounds__(kSubstepAdjThreads, sizeof(T) == 4 ? 6 : 3) k_substep_adj(
    DGrid G, DParams<T> P, int64_t n, const int32_t* __restrict__ cell, const pos_t<T>* __restrict__ pos,
    const float4* __restrict__ posf, const vec_t<T>* __restrict__ vel, const int32_t* __restrict__ id, NbDev nb,
    const uint4* __restrict__ table, T skin, Fields<T> Fd, const vec_t<T>* __restrict__ gxo,
    const vec_t<T>* __restrict__ gvo, const vec_t<T>* __restrict__ gfe, const int32_t* __restrict__ perm,
    vec_t<T>* __restrict__ gxi, vec_t<T>* __restrict__ gvi, double* __restrict__ g_cdrag,
    double* __restrict__ g_mu) {
  __shared__ double s_red[64];
  const bool rebuild = (nb.flags[kNbRebuild] | nb.flags[kNbSticky]) != 0u;  // uniform over the launch
  const int64_t i = blockIdx.x * (int64_t)kSubstepAdjThreads + threadIdx.x;
  T my_gc = T(0), my_gmu = T(0);
  if (i < n) {
    const int32_t ci = cell[i];
    const pos_t<T> pi = pos[i];
    const vec_t<T> vi = vel[i];
    const T ri = radius_of(pi);
    const T mi = granule_mass(P, ri);
    const vec_t<T> zero = make_vec<T>(0, 0, 0);
    // a4: x' = x + dt v', v' = v + dt a
    const vec_t<T> gxi_ = gxo[i];
    const IntegrateAdj<T> o = integrate_adj_granule(P, ri, gxi_, gvo[i], gfe ? gfe[i] : zero);
    T gx[3] = {gxi_.x, gxi_.y, gxi_.z};
    T gv[3] = {o.gvt[0], o.gvt[1], o.gvt[2]};
    // a3: F_fl and a_f at the granule
    {
      int m[3];
      T t[3], gdv[3];
      my_gc = g2p_adj_granule<T>(G, P, Fd, ci, pi, vi, o.gFfl, o.gaf, gx, gdv, m, t);
#pragma unroll
      for (int a = 0; a < 3; ++a) gv[a] -= gdv[a];
    }
    // a2: contact pairs (F_ji = -F_ij) and walls
    const T l0 = o.gFc[0], l1 = o.gFc[1], l2 = o.gFc[2];
    T gm = T(0);
    auto pair = [&](int64_t j, const PairGeom<T>& g) {
      const vec_t<T> vj = ldg(&vel[j]);
      const T rj = radius_of(ldg(&pos[j]));
      const IntegrateAdj<T> oj =
          integrate_adj_granule(P, rj, ldg(&gxo[j]), ldg(&gvo[j]), gfe ? ldg(&gfe[j]) : zero);
      const T mj = granule_mass(P, rj);
      gm += pair_force_adj(P, g.x0, g.x1, g.x2, g.d, g.overlap, vi.x - vj.x, vi.y - vj.y, vi.z - vj.z,
                           mi * mj / (mi + mj), l0 - oj.gFc[0], l1 - oj.gFc[1], l2 - oj.gFc[2], l0, l1, l2, gx[0],
                           gx[1], gx[2], gv[0], gv[1], gv[2]);
    };
    const int cx = cell_x(ci), cy = cell_y(ci), cz = cell_z(ci);
    const bool has_f = sizeof(T) == 4 && posf != nullptr;
    const float4 fi = has_f ? __ldg(&posf[i]) : make_float4(0.f, 0.f, 0.f, 0.f);
    if (P.cap) {  // contacts and capillary bridges; a bridge also depends on x_i through sr_i
      T gsr[3];
      const T sri = moisture_ratio_at(G, P, Fd.af, ci, pi, gsr);
      T wsr = T(0);  // sum over bridges of (lambda_i - lambda_j) . dF/d sr_mean
      auto near = [&](int64_t j, int32_t cj, const pos_t<T>& pj, const PairGeom<T>& g) {
        if (g.overlap > T(0)) {
          pair(j, g);
          return;
        }
        const T rj = radius_of(pj);
        const IntegrateAdj<T> oj =
            integrate_adj_granule(P, rj, ldg(&gxo[j]), ldg(&gvo[j]), gfe ? ldg(&gfe[j]) : zero);
        wsr += add_bridge_adj(P, g, ri, rj, sri, moisture_ratio_at(G, P, Fd.af, cj, pj, (T*)nullptr),
                              l0 - oj.gFc[0], l1 - oj.gFc[1], l2 - oj.gFc[2], gx[0], gx[1], gx[2]);
      };
      if (rebuild)
        verlet_build_row_near<T>(G, P, nb, table, n, i, cx, cy, cz, ci, pi, ri, skin, id, pos, near);
      else
        for_each_list_near<T>(G, P, nb, i, cx, cy, cz, pi, ri, has_f, fi, cell, pos, posf, near);
#pragma unroll
      for (int a = 0; a < 3; ++a) gx[a] += T(0.5) * wsr * gsr[a];
    } else if (rebuild) {
      verlet_build_row<T>(G, nb, table, n, i, cx, cy, cz, ci, pi, ri, has_f, fi, skin, id, pos, posf, pair);
    } else {
      for_each_list_contact<T>(G, nb, i, cx, cy, cz, ci, pi, ri, has_f, fi, cell, pos, posf, pair);
    }
    if (P.walls)
      gm += add_walls_adj(G, P, pi, ri, mi, vi, cx, cy, cz, l0, l1, l2, gx[0], gx[1], gx[2], gv[0], gv[1], gv[2]);
    my_gmu = gm;
    const int64_t out = perm ? (int64_t)perm[i] : i;
    gxi[out] = make_vec<T>(gx[0], gx[1], gx[2]);
    gvi[out] = make_vec<T>(gv[0], gv[1], gv[2]);
  }
  if (g_cdrag || g_mu) {
    if constexpr (sizeof(T) == 4) {
      // FP32 path: the warp sums in FP32 (the terms are FP32 values), then the
      // CTA's warps in FP64: the FP64 pipe of this GPU runs at 1/64 of the
      // FP32 rate, and a per-thread FP64 shuffle tree cost as much as the
      // rest of the kernel's arithmetic
      float a = my_gc, b = my_gmu;
      for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        b += __shfl_down_sync(0xffffffffu, b, off);
      }
      const int w = threadIdx.x >> 5;
      if (lane_id() == 0) {
        s_red[w] = (double)a;
        s_red[32 + w] = (double)b;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double ga = 0.0, gb = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
          ga += s_red[k];
          gb += s_red[32 + k];
        }
        if (g_cdrag) atomicAdd(g_cdrag, ga);
        if (g_mu) atomicAdd(g_mu, gb);
      }
    } else {
      block_sum2(my_gc, my_gmu, s_red);
      if (threadIdx.x == 0) {
        if (g_cdrag) atomicAdd(g_cdrag, my_gc);
        if (g_mu) atomicAdd(g_mu, my_gmu);
      }
    }
  }
  verlet_call_done(nb, rebuild);  // its barrier also frees s_red
}

}  // namespace gic

using namespace gic;

namespace gic {

// [zero alpha_s] -> k_substep (sorted -> next) -> [alpha_s out]; counts its
// launches into *launches.
static int substep_launch(const DGrid& G, const GicParams* params, const GicGranules* s, const void* cell_table,
                          const GicNeighbors* nb, const NbDev& d, const void* u, const void* v, const void* w,
                          const void* p, const void* alpha_f, GicGranules* next, void* f_ex, double* alpha_s,
                          void* Fs_u, void* Fs_v, void* Fs_w, double* sums2, cudaStream_t stream, int* launches,
                          bool keep = false, void* scratch = nullptr) {
  int rc;
  const int64_t ncell = (int64_t)G.nx * G.ny * G.nz;
  if (alpha_s) {
    alpha_begin(alpha_s, ncell, sums2, stream, scratch);
    ++*launches;
  }
  if (s->n > 0) {
    const unsigned blocks = grid_blocks(s->n, kSubstepThreads);
    if (s->precision == GIC_FP32) {
      DParams<float> P;
      if ((rc = make_params(params, &P))) return rc;
      auto kern = !(keep && !P.cap) ? k_substep<float, false>
                  : alpha_s             ? k_substep<float, true>
                                        : k_substep<float, true, true>;
      kern<<<blocks, kSubstepThreads, 0, stream>>>(
          G, P, s->n, s->cell, (const uint4*)s->pos, (const float4*)s->posf, (const float4*)s->vel, s->id, d,
          (const uint4*)cell_table, (float)nb->skin, fields<float>(u, v, w, p, alpha_f), next->cell,
          (uint4*)next->pos, (float4*)next->vel, next->id, (float4*)next->posf, (float4*)f_ex, alpha_s,
          (float*)Fs_u, (float*)Fs_v, (float*)Fs_w, sums2, status_word());
    } else {
      DParams<double> P;
      if ((rc = make_params(params, &P))) return rc;
      auto kern = keep && !P.cap ? k_substep<double, true> : k_substep<double, false>;
      kern<<<blocks, kSubstepThreads, 0, stream>>>(
          G, P, s->n, s->cell, (const d4*)s->pos, nullptr, (const d4*)s->vel, s->id, d, (const uint4*)cell_table,
          nb->skin, fields<double>(u, v, w, p, alpha_f), next->cell, (d4*)next->pos, (d4*)next->vel, next->id,
          nullptr, (d4*)f_ex, alpha_s, (double*)Fs_u, (double*)Fs_v, (double*)Fs_w, sums2, status_word());
    }
    count_launches(1);
    ++*launches;
  }
  if (alpha_s) {
    alpha_end(G, s->precision, alpha_s, ncell, sums2, stream, scratch);
    ++*launches;
  }
  return GIC_OK;
}

}  // namespace gic

extern "C" int gic_substep(const GicGrid* grid, const GicParams* params, const GicGranules* sorted,
                           const void* cell_table, const GicNeighbors* nb, const void* u, const void* v,
                           const void* w, const void* p, const void* alpha_f, GicGranules* next, void* f_ex,
                           double* alpha_s, void* Fs_u, void* Fs_v, void* Fs_w, double* sums2,
                           gic_stream_t stream) {
  GIC_RANGE("gic_substep");
  {  // parameters first, before any device work
    DParams<double> chk;
    if (int rc0 = make_params(params, &chk)) return rc0;
  }
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  const GicGranules* s = sorted;
  if ((rc = check_granules(s, "gic_substep sorted", true))) return rc;
  if ((rc = check_granules(next, "gic_substep next"))) return rc;
  if (next->n != s->n || next->precision != s->precision)
    return set_error(GIC_ERR_INVALID, "gic_substep: sorted/next differ in size or precision");
  if (!u || !v || !w || !p || !alpha_f) return set_error(GIC_ERR_INVALID, "gic_substep: null fluid field");
  bool fs = Fs_u || Fs_v || Fs_w;
  if (fs && !(Fs_u && Fs_v && Fs_w)) return set_error(GIC_ERR_INVALID, "gic_substep: give all three F_s arrays or none");
  if (sums2 && !alpha_s) return set_error(GIC_ERR_INVALID, "gic_substep: sums2 needs alpha_s");
  if ((rc = check_vecs(s->precision, "gic_substep", {f_ex}))) return rc;
  NbDev d;
  if ((rc = verlet_prelude(G, params, s, cell_table, nb, nullptr, stream, "gic_substep", &d, false))) return rc;
  int launches = 0;
  if ((rc = substep_launch(G, params, s, cell_table, nb, d, u, v, w, p, alpha_f, next, f_ex, alpha_s, Fs_u, Fs_v, Fs_w,
                           sums2, (cudaStream_t)stream, &launches)))
    return rc;
  GIC_CHECK_LAUNCH("gic_substep");
  return GIC_OK;
}

namespace gic {

// gic_step's decision: this call rebuilds the lists (and sorts) when the
// previous call's k_substep left a granule beyond skin / 2 of its reference,
// or a rebuild was requested.  Sets the two branches' conditionals.
__global__ void k_step_decide(uint32_t* flags, cudaGraphConditionalHandle rebuild, cudaGraphConditionalHandle keep) {
  const unsigned r = (flags[kNbNext] | flags[kNbSticky]) != 0u ? 1u : 0u;
  flags[kNbRebuild] = r;
  flags[kNbNext] = 0u;
  cudaGraphSetConditional(rebuild, r);
  cudaGraphSetConditional(keep, 1u - r);
}

// Everything a gic_step graph depends on; a call with the same bytes reuses
// the instantiated graph.
struct StepKey {
  GicGrid grid;
  GicParams params;
  GicGranules state, next, sorted;
  GicNeighbors nb;
  const void* ptr[13];
  size_t ws_bytes;
};

struct StepGraph {
  bool used = false;
  uint64_t last = 0;
  StepKey key;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int launches = 0;  // kernels every launch runs (the sort's are not counted)
};

constexpr int kStepGraphs = 8;
static StepGraph g_step_graphs[kStepGraphs];
static uint64_t g_step_clock = 0;
static std::mutex g_step_mu;

static bool same_key(const StepKey& a, const StepKey& b) { return memcmp(&a, &b, sizeof(StepKey)) == 0; }

static void store_key(StepKey& k, const GicGrid* grid, const GicParams* params, const GicGranules* state,
                      const GicGranules* next, const GicGranules* sorted, const GicNeighbors* nb,
                      const void* const ptr[13], size_t ws_bytes) {
  memset(&k, 0, sizeof(k));  // padding bytes take part in the comparison
  memcpy(&k.grid, grid, sizeof(GicGrid));
  memcpy(&k.params, params, sizeof(GicParams));
  memcpy(&k.state, state, sizeof(GicGranules));
  memcpy(&k.next, next, sizeof(GicGranules));
  memcpy(&k.sorted, sorted, sizeof(GicGranules));
  memcpy(&k.nb, nb, sizeof(GicNeighbors));
  for (int i = 0; i < 13; ++i) k.ptr[i] = ptr[i];
  k.ws_bytes = ws_bytes;
}

// Adds an IF node on `dep` with handle h and captures fill(stream) into its body.
template <typename Fill>
static int add_branch(cudaGraph_t g, cudaGraphNode_t dep, cudaGraphConditionalHandle h, cudaStream_t cs, Fill&& fill) {
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeIf;
  cp.conditional.size = 1;
  cudaGraphNode_t cond;
  if (cudaGraphAddNode(&cond, g, &dep, nullptr, 1, &cp) != cudaSuccess)
    return set_error(GIC_ERR_CUDA, "gic_step: conditional node failed");
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  cudaGraph_t got = nullptr;
  if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
    return set_error(GIC_ERR_CUDA, "gic_step: graph capture failed");
  int rc = fill(cs);
  if (cudaStreamEndCapture(cs, &got) != cudaSuccess && rc == GIC_OK)
    rc = set_error(GIC_ERR_CUDA, "gic_step: graph capture failed");
  return rc;
}

// Builds the graph of one gic_step configuration:
//   decide -> IF rebuild: sort (state -> sorted) -> [zero alpha] -> k_substep (sorted -> next) -> [alpha out]
//          -> IF keep:    [zero alpha] -> k_substep (state -> next) -> [alpha out]
static int build_step_graph(StepGraph& sg, const DGrid& G, const GicGrid* grid, const GicParams* params,
                            const GicGranules* state, GicGranules* next, GicGranules* sorted, int32_t* perm,
                            void* cell_table, void* ws, size_t ws_bytes, const GicNeighbors* nb, const NbDev& d,
                            const void* u, const void* v, const void* w, const void* p, const void* alpha_f,
                            double* alpha_s, void* Fs_u, void* Fs_v, void* Fs_w, double* sums2) {
  int rc = GIC_OK;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  cudaStream_t cs = nullptr;
  cudaGraph_t got = nullptr;
  cudaGraphConditionalHandle h_rebuild, h_keep;
  int launches = 0;
  status_word();  // resolve the device address before capturing
  if ((rc = alpha_prepare())) return rc;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return set_error(GIC_ERR_CUDA, "gic_step: cudaGraphCreate failed");
  if (cudaGraphConditionalHandleCreate(&h_rebuild, g, 0, cudaGraphCondAssignDefault) != cudaSuccess ||
      cudaGraphConditionalHandleCreate(&h_keep, g, 0, cudaGraphCondAssignDefault) != cudaSuccess ||
      cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    return set_error(GIC_ERR_CUDA, "gic_step: graph setup failed");
  }
  set_capturing(true);
  do {
    // 1. the decision
    if (cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      rc = set_error(GIC_ERR_CUDA, "gic_step: graph capture failed");
      break;
    }
    k_step_decide<<<1, 1, 0, cs>>>(nb->flags, h_rebuild, h_keep);
    if (cudaStreamEndCapture(cs, &got) != cudaSuccess) {
      rc = set_error(GIC_ERR_CUDA, "gic_step: graph capture failed");
      break;
    }
    launches += 1;
    size_t nn = 0;
    cudaGraphNode_t decide = nullptr;
    if (cudaGraphGetNodes(g, nullptr, &nn) != cudaSuccess || nn != 1 || cudaGraphGetNodes(g, &decide, &nn) != cudaSuccess) {
      rc = set_error(GIC_ERR_CUDA, "gic_step: unexpected graph");
      break;
    }
    // 2. the branch that rebuilds: sort, then the substep from the sorted state (its launches not counted)
    int uncounted = 0;
    rc = add_branch(g, decide, h_rebuild, cs, [&](cudaStream_t st) {
      int r = sort_gated(grid, state, sorted, perm, cell_table, ws, ws_bytes, nullptr, st);
      // FP32 with float copies and the contact law alone: the rows are built on
      // the staged neighbourhood first, and the substep walks them
      if (r == GIC_OK && state->precision == GIC_FP32 && sorted->posf && params->sigma == 0.0)
        r = launch_build_tile(G, sorted, cell_table, d, nb->skin, st);
      if (r == GIC_OK)
        r = substep_launch(G, params, sorted, cell_table, nb, d, u, v, w, p, alpha_f, next, nullptr, alpha_s, Fs_u,
                           Fs_v, Fs_w, sums2, st, &uncounted, false, ws);
      return r;
    });
    if (rc) break;
    // 3. the branch that keeps the lists: the substep straight from the state
    rc = add_branch(g, decide, h_keep, cs, [&](cudaStream_t st) {
      return substep_launch(G, params, state, cell_table, nb, d, u, v, w, p, alpha_f, next, nullptr, alpha_s, Fs_u,
                            Fs_v, Fs_w, sums2, st, &launches, true, ws);
    });
    if (rc) break;
    if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
      rc = set_error(GIC_ERR_CUDA, "gic_step: graph instantiation failed");
      break;
    }
  } while (false);
  set_capturing(false);
  cudaStreamDestroy(cs);
  if (rc) {
    cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  sg.graph = g;
  sg.exec = ex;
  sg.launches = launches;
  return GIC_OK;
}

}  // namespace gic

static bool share_array(const GicGranules* a, const GicGranules* b) {
  return a->cell == b->cell || a->pos == b->pos || a->vel == b->vel || a->id == b->id ||
         (a->posf && a->posf == b->posf);
}

extern "C" int gic_step(const GicGrid* grid, const GicParams* params, const GicGranules* state, GicGranules* next,
                        GicGranules* sorted, int32_t* perm, void* cell_table, void* ws, size_t ws_bytes,
                        const GicNeighbors* nb, const void* u, const void* v, const void* w, const void* p,
                        const void* alpha_f, double* alpha_s, void* Fs_u, void* Fs_v, void* Fs_w, double* sums2,
                        gic_stream_t stream) {
  GIC_RANGE("gic_step");
  {  // parameters first, before any device work
    DParams<double> chk;
    if (int rc0 = make_params(params, &chk)) return rc0;
  }
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if (!params) return set_error(GIC_ERR_INVALID, "gic_step: params is NULL");
  if ((rc = check_granules(state, "gic_step state", true))) return rc;
  if ((rc = check_granules(next, "gic_step next", true))) return rc;
  if ((rc = check_granules(sorted, "gic_step sorted", true))) return rc;
  if (next->n != state->n || next->precision != state->precision || sorted->n != state->n ||
      sorted->precision != state->precision)
    return set_error(GIC_ERR_INVALID, "gic_step: state/next/sorted size or precision differ");
  if (share_array(state, next) || share_array(state, sorted) || share_array(next, sorted))
    return set_error(GIC_ERR_INVALID, "gic_step: state, next and sorted must not share arrays");
  if (state->n > 0 && !perm) return set_error(GIC_ERR_INVALID, "gic_step: perm is NULL");
  if (!u || !v || !w || !p || !alpha_f) return set_error(GIC_ERR_INVALID, "gic_step: null fluid field");
  bool fs = Fs_u || Fs_v || Fs_w;
  if (fs && !(Fs_u && Fs_v && Fs_w)) return set_error(GIC_ERR_INVALID, "gic_step: give all three F_s arrays or none");
  if (sums2 && !alpha_s) return set_error(GIC_ERR_INVALID, "gic_step: sums2 needs alpha_s");
  if (!nb) return set_error(GIC_ERR_INVALID, "gic_step: neighbours struct is NULL");
  NbDev d;
  if ((rc = verlet_view(G, state, cell_table, nb, "gic_step", true, &d))) return rc;
  if (state->n == 0) return GIC_OK;
  {  // arguments of the sort, checked before they are baked into a graph
    size_t need = 0;
    if ((rc = gic_workspace_size(grid, state->n, state->precision, &need))) return rc;
    if (!ws || ws_bytes < need)
      return set_error(GIC_ERR_WORKSPACE, "gic_step: workspace of %zu bytes needed, %zu given", need, ws_bytes);
    if ((uintptr_t)ws % 256) return set_error(GIC_ERR_ALIGN, "gic_step: workspace must be 256-byte aligned");
  }
  const void* ptr[13] = {perm, cell_table, ws, u, v, w, p, alpha_f, alpha_s, Fs_u, Fs_v, Fs_w, sums2};
  StepKey key;
  store_key(key, grid, params, state, next, sorted, nb, ptr, ws_bytes);
  std::lock_guard<std::mutex> lock(g_step_mu);
  StepGraph* hit = nullptr;
  for (auto& sg : g_step_graphs)
    if (sg.used && same_key(sg.key, key)) hit = &sg;
  if (!hit) {
    StepGraph* slot = &g_step_graphs[0];
    for (auto& sg : g_step_graphs) {
      if (!sg.used) {
        slot = &sg;
        break;
      }
      if (sg.last < slot->last) slot = &sg;
    }
    if (slot->used) {
      cudaGraphExecDestroy(slot->exec);
      cudaGraphDestroy(slot->graph);
      slot->used = false;
    }
    if ((rc = build_step_graph(*slot, G, grid, params, state, next, sorted, perm, cell_table, ws, ws_bytes, nb, d, u,
                               v, w, p, alpha_f, alpha_s, Fs_u, Fs_v, Fs_w, sums2)))
      return rc;
    memcpy(&slot->key, &key, sizeof(StepKey));
    slot->used = true;
    hit = slot;
  }
  hit->last = ++g_step_clock;
  cudaError_t e = cudaGraphLaunch(hit->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return set_error(GIC_ERR_CUDA, "gic_step: cudaGraphLaunch: %s", cudaGetErrorString(e));
  count_launches(hit->launches);
  return GIC_OK;
}

extern "C" int gic_substep_adj(const GicGrid* grid, const GicParams* params, const GicGranules* sorted,
                               const int32_t* perm, const void* cell_table, const GicNeighbors* nb, const void* u,
                               const void* v, const void* w, const void* p, const void* alpha_f,
                               const void* g_pos_out, const void* g_vel_out, const void* g_f_ex, void* g_pos_in,
                               void* g_vel_in, double* g_cdrag, double* g_mu, gic_stream_t stream) {
  GIC_RANGE("gic_substep_adj");
  {  // parameters first, before any device work
    DParams<double> chk;
    if (int rc0 = make_params(params, &chk)) return rc0;
  }
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  const GicGranules* s = sorted;
  if ((rc = check_granules(s, "gic_substep_adj sorted", true))) return rc;
  if (!u || !v || !w || !p || !alpha_f) return set_error(GIC_ERR_INVALID, "gic_substep_adj: null fluid field");
  if (!g_pos_out || !g_vel_out || !g_pos_in || !g_vel_in)
    return set_error(GIC_ERR_INVALID, "gic_substep_adj: null gradient array");
  if ((rc = check_vecs(s->precision, "gic_substep_adj", {g_pos_out, g_vel_out, g_f_ex, g_pos_in, g_vel_in})))
    return rc;
  // partners read the upstream gradients while others are written
  const void* ins[3] = {g_pos_out, g_vel_out, g_f_ex};
  for (const void* q : ins)
    if (q && (q == g_pos_in || q == g_vel_in))
      return set_error(GIC_ERR_INVALID, "gic_substep_adj: an output aliases an input gradient");
  if (g_pos_in == g_vel_in) return set_error(GIC_ERR_INVALID, "gic_substep_adj: g_pos_in aliases g_vel_in");
  NbDev d;
  if ((rc = verlet_prelude(G, params, s, cell_table, nb, nullptr, stream, "gic_substep_adj", &d, false))) return rc;
  if (s->n == 0) return GIC_OK;
  const unsigned blocks = grid_blocks(s->n, kSubstepAdjThreads);
  if (s->precision == GIC_FP32) {
    DParams<float> P;
    if ((rc = make_params(params, &P))) return rc;
    k_substep_adj<float><<<blocks, kSubstepAdjThreads, 0, stream>>>(
        G, P, s->n, s->cell, (const uint4*)s->pos, (const float4*)s->posf, (const float4*)s->vel, s->id, d,
        (const uint4*)cell_table, (float)nb->skin, fields<float>(u, v, w, p, alpha_f), (const float4*)g_pos_out,
        (const float4*)g_vel_out, (const float4*)g_f_ex, perm, (float4*)g_pos_in, (float4*)g_vel_in, g_cdrag, g_mu);
  } else {
    DParams<double> P;
    if ((rc = make_params(params, &P))) return rc;
    k_substep_adj<double><<<blocks, kSubstepAdjThreads, 0, stream>>>(
        G, P, s->n, s->cell, (const d4*)s->pos, nullptr, (const d4*)s->vel, s->id, d, (const uint4*)cell_table,
        nb->skin, fields<double>(u, v, w, p, alpha_f), (const d4*)g_pos_out, (const d4*)g_vel_out,
        (const d4*)g_f_ex, perm, (d4*)g_pos_in, (d4*)g_vel_in, g_cdrag, g_mu);
  }
  count_launches(1);
  GIC_CHECK_LAUNCH("gic_substep_adj");
  return GIC_OK;
}
