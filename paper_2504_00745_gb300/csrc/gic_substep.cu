// gic_substep.cu -- one SandSubstep (Alg. 2) after the sort, fused into one
// pass over the sorted state: contact forces from the Verlet lists (or, on a
// substep that rebuilds them, from the 27-cell walk that builds them), the G2P coupling
// (Sec. 3.3), the virtual-mass integration (Sec. 5.2) into the next state,
// and the P2G scatter of F_s at the old positions and, when asked, of
// alpha_s at the new ones.  The per-granule force arrays of the separate
// entry points (F_c, F_fl, a_f, f_ex) never leave registers.
#include "gic_contact.cuh"
#include "gic_grid.cuh"
#include "gic_integrate.cuh"

namespace gic {

constexpr int kSubstepThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kSubstepThreads, sizeof(T) == 4 ? 4 : 2) k_substep(
    DGrid G, DParams<T> P, int64_t n, const int32_t* __restrict__ cell, const pos_t<T>* __restrict__ pos,
    const float4* __restrict__ posf, const vec_t<T>* __restrict__ vel, const int32_t* __restrict__ id, NbDev nb,
    const uint4* __restrict__ table, T skin, Fields<T> Fd, int32_t* __restrict__ cell_out, pos_t<T>* __restrict__ pos_out,
    vec_t<T>* __restrict__ vel_out, int32_t* __restrict__ id_out, vec_t<T>* __restrict__ fex_out,
    double* __restrict__ alpha, T* __restrict__ Fs_u, T* __restrict__ Fs_v, T* __restrict__ Fs_w,
    double* __restrict__ sums, uint32_t* status) {
  __shared__ P2GShared sh;  // FP32 path only
  const bool rebuild = (nb.flags[kNbRebuild] | nb.flags[kNbSticky]) != 0u;  // uniform over the launch
  const bool do_a = alpha != nullptr, do_f = Fs_u != nullptr;
  const int64_t i = blockIdx.x * (int64_t)kSubstepThreads + threadIdx.x;
  const bool valid = i < n;
  if constexpr (sizeof(T) == 4) p2g_box_init(sh);

  int32_t ci = 0, co = 0;
  pos_t<T> pi{}, po{};
  T fe[3] = {T(0), T(0), T(0)};
  if (valid) {
    ci = cell[i];
    pi = pos[i];
    const vec_t<T> vi = vel[i];
    const T ri = radius_of(pi);
    const T mi = granule_mass(P, ri);
    uint32_t flags = 0;
    if (T(2) * ri > (T)G.hc) flags |= GIC_STATUS_RADIUS;
    // a2: contact
    T F0 = 0, F1 = 0, F2 = 0;
    bool coincident = false;
    {
      const int cx = cell_x(ci), cy = cell_y(ci), cz = cell_z(ci);
      const bool has_f = sizeof(T) == 4 && posf != nullptr;
      const float4 fi = has_f ? __ldg(&posf[i]) : make_float4(0.f, 0.f, 0.f, 0.f);
      if (rebuild)  // this substep rebuilds the lists: walk the 27 cells
        verlet_build_granule(G, P, nb, table, n, i, cx, cy, cz, ci, pi, ri, mi, vi, has_f, fi, skin, id, pos, posf,
                             vel, F0, F1, F2, coincident);
      else
        verlet_list_force(G, P, nb, i, cx, cy, cz, ci, pi, ri, mi, vi, has_f, fi, cell, pos, posf, vel, F0, F1, F2,
                          coincident);
      if (P.walls) add_walls(G, P, pi, ri, mi, vi, cx, cy, cz, F0, F1, F2, status);
      if (coincident) flags |= GIC_STATUS_COINCIDENT;
      if (!isfinite(F0) || !isfinite(F1) || !isfinite(F2)) flags |= GIC_STATUS_NONFINITE;
    }
    // a3: G2P coupling
    T Ffl[3], af[3];
    const T sp = g2p_granule(G, P, Fd, ci, pi, vi, Ffl, af);
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
    if (fex_out) fex_out[i] = make_vec<T>(fe[0], fe[1], fe[2]);
  }

  // a5: P2G
  if constexpr (sizeof(T) == 4) {
    P2GExtent ext;
    float fc[3] = {P.exch * fe[0], P.exch * fe[1], P.exch * fe[2]};
    if (valid) {
      if (do_a) ext.add_cell(G, co);
      if (do_f) {
        ext.add_cell(G, ci);
        ext.add_force(fc);
      }
    }
    const P2GBox B = p2g_box(sh, ext, do_a, do_f);
    float* Fs[3] = {Fs_u, Fs_v, Fs_w};
    unsigned long long S = 0;
    if (valid && do_a) {
      int ia[3];
      long long va[8];
      alpha_deposits(G, co, po, ia, va, S);
      p2g_add_alpha(sh, B, G, (unsigned long long*)alpha, ia, va);
    }
    if (valid && do_f) {
      int m[3];
      float t[3];
      granule_mac<float>(G, ci, pi, m, t);
#pragma unroll
      for (int comp = 0; comp < 3; ++comp)
        p2g_add_face(sh, B, G, Fs[comp], comp, make_stencil<float>(G, m, t, comp), fc[comp]);
    }
    p2g_flush(sh, B, G, (unsigned long long*)alpha, Fs, kSubstepThreads);
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

}  // namespace gic

using namespace gic;

extern "C" int gic_substep(const GicGrid* grid, const GicParams* params, const GicGranules* sorted,
                           const void* cell_table, const GicNeighbors* nb, const void* u, const void* v,
                           const void* w, const void* p, const void* alpha_f, GicGranules* next, void* f_ex, double* alpha_s, void* Fs_u, void* Fs_v, void* Fs_w, double* sums2,
                           gic_stream_t stream) {
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
  const int64_t ncell = (int64_t)G.nx * G.ny * G.nz;
  if (alpha_s) alpha_begin(alpha_s, ncell, sums2, stream);
  if (s->n > 0) {
    const unsigned blocks = grid_blocks(s->n, kSubstepThreads);
    if (s->precision == GIC_FP32) {
      DParams<float> P;
      if ((rc = make_params(params, &P))) return rc;
      k_substep<float><<<blocks, kSubstepThreads, 0, stream>>>(
          G, P, s->n, s->cell, (const uint4*)s->pos, (const float4*)s->posf, (const float4*)s->vel, s->id, d,
          (const uint4*)cell_table, (float)nb->skin, fields<float>(u, v, w, p, alpha_f), next->cell, (uint4*)next->pos, (float4*)next->vel,
          next->id, (float4*)f_ex, alpha_s, (float*)Fs_u, (float*)Fs_v, (float*)Fs_w, sums2, status_word());
    } else {
      DParams<double> P;
      if ((rc = make_params(params, &P))) return rc;
      k_substep<double><<<blocks, kSubstepThreads, 0, stream>>>(
          G, P, s->n, s->cell, (const d4*)s->pos, nullptr, (const d4*)s->vel, s->id, d, (const uint4*)cell_table,
          nb->skin, fields<double>(u, v, w, p, alpha_f), next->cell, (d4*)next->pos, (d4*)next->vel, next->id, (d4*)f_ex,
          alpha_s, (double*)Fs_u, (double*)Fs_v, (double*)Fs_w, sums2, status_word());
    }
    count_launches(1);
  }
  if (alpha_s) alpha_end(G, s->precision, alpha_s, ncell, sums2, stream);
  GIC_CHECK_LAUNCH("gic_substep");
  return GIC_OK;
}

extern "C" int gic_step(const GicGrid* grid, const GicParams* params, GicGranules* state, GicGranules* sorted,
                        int32_t* perm, void* cell_table, void* ws, size_t ws_bytes, const GicNeighbors* nb,
                        const void* u, const void* v, const void* w, const void* p, const void* alpha_f,
                        double* alpha_s, void* Fs_u, void* Fs_v, void* Fs_w, double* sums2, gic_stream_t stream) {
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if ((rc = check_granules(state, "gic_step state", true))) return rc;
  if ((rc = check_granules(sorted, "gic_step sorted", true))) return rc;
  if (sorted->n != state->n || sorted->precision != state->precision)
    return set_error(GIC_ERR_INVALID, "gic_step: state/sorted size or precision differ");
  if (state->cell == sorted->cell || state->pos == sorted->pos || state->vel == sorted->vel ||
      state->id == sorted->id)
    return set_error(GIC_ERR_INVALID, "gic_step: state and sorted must not alias");
  if (state->n > 0 && !perm) return set_error(GIC_ERR_INVALID, "gic_step: perm is NULL");
  // 1. displacements of the current state against the lists (sets the rebuild
  //    word), and the state copied into `sorted` in its current order
  NbDev d;
  if ((rc = verlet_check(G, state, cell_table, nb, stream, "gic_step", &d, sorted, perm))) return rc;
  // 2. the sort over that copy, only when the lists are rebuilt
  if ((rc = sort_gated(grid, state, sorted, perm, cell_table, ws, ws_bytes, nb->flags, stream))) return rc;
  // 3. the fused rest of the substep, sorted -> state
  const GicGranules* s = sorted;
  if (!u || !v || !w || !p || !alpha_f) return set_error(GIC_ERR_INVALID, "gic_step: null fluid field");
  bool fs = Fs_u || Fs_v || Fs_w;
  if (fs && !(Fs_u && Fs_v && Fs_w)) return set_error(GIC_ERR_INVALID, "gic_step: give all three F_s arrays or none");
  if (sums2 && !alpha_s) return set_error(GIC_ERR_INVALID, "gic_step: sums2 needs alpha_s");
  const int64_t ncell = (int64_t)G.nx * G.ny * G.nz;
  if (alpha_s) alpha_begin(alpha_s, ncell, sums2, stream);
  if (s->n > 0) {
    const unsigned blocks = grid_blocks(s->n, kSubstepThreads);
    if (s->precision == GIC_FP32) {
      DParams<float> P;
      if ((rc = make_params(params, &P))) return rc;
      k_substep<float><<<blocks, kSubstepThreads, 0, stream>>>(
          G, P, s->n, s->cell, (const uint4*)s->pos, (const float4*)s->posf, (const float4*)s->vel, s->id, d,
          (const uint4*)cell_table, (float)nb->skin, fields<float>(u, v, w, p, alpha_f), state->cell,
          (uint4*)state->pos, (float4*)state->vel, state->id, nullptr, alpha_s, (float*)Fs_u, (float*)Fs_v,
          (float*)Fs_w, sums2, status_word());
    } else {
      DParams<double> P;
      if ((rc = make_params(params, &P))) return rc;
      k_substep<double><<<blocks, kSubstepThreads, 0, stream>>>(
          G, P, s->n, s->cell, (const d4*)s->pos, nullptr, (const d4*)s->vel, s->id, d, (const uint4*)cell_table,
          nb->skin, fields<double>(u, v, w, p, alpha_f), state->cell, (d4*)state->pos, (d4*)state->vel, state->id,
          nullptr, alpha_s, (double*)Fs_u, (double*)Fs_v, (double*)Fs_w, sums2, status_word());
    }
    count_launches(1);
  }
  if (alpha_s) alpha_end(G, s->precision, alpha_s, ncell, sums2, stream);
  GIC_CHECK_LAUNCH("gic_step");
  return GIC_OK;
}
