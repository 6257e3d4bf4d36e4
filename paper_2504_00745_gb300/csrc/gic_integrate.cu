// gic_integrate.cu -- a4: virtual-mass symplectic Euler (Sec. 5.2 Eq. sand
// kine; Alg. 2 MoveParticle) and its adjoint.
//
//   (m + m_a) a = F_c + F_fl + m g + m_a a_f,   m_a = (2/3) pi r^3 rho_f
//   v' = v + dt' a,   x' = x + dt' v',   f_ex = F_fl + m_a (a_f - a)
//
// FP32 path: the position increment dt' v' is rounded to the 2^-30 h_c
// fixed-point lattice of the cell offset and added in integer arithmetic, so
// positions carry no floating-point drift; a carry or borrow moves the granule
// to the neighbouring contact cell.  FP64 path: offsets are doubles re-binned
// into [0, h_c).
#include "gic_integrate.cuh"

namespace gic {

template <typename T>
__global__ void __launch_bounds__(256) k_integrate(DGrid G, DParams<T> P, int64_t n, const int32_t* __restrict__ cell,
                                                    const pos_t<T>* __restrict__ pos,
                                                    const vec_t<T>* __restrict__ vel,
                                                    const vec_t<T>* __restrict__ Fc, const vec_t<T>* __restrict__ Ffl,
                                                    const vec_t<T>* __restrict__ af, int32_t* __restrict__ cell_out,
                                                    pos_t<T>* __restrict__ pos_out, vec_t<T>* __restrict__ vel_out,
                                                    vec_t<T>* __restrict__ fex, const int32_t* id_in, int32_t* id_out,
                                                    uint32_t* status) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  vec_t<T> fc = Fc[i], ff = Ffl[i], fa = af[i];
  int32_t co;
  pos_t<T> po;
  vec_t<T> vo;
  T e0, e1, e2;
  uint32_t flags = 0;
  integrate_granule(G, P, cell[i], pos[i], vel[i], fc.x, fc.y, fc.z, ff.x, ff.y, ff.z, fa.x, fa.y, fa.z, co, po, vo,
                    e0, e1, e2, flags);
  if (flags) raise_status(status, flags);
  cell_out[i] = co;
  pos_out[i] = po;
  vel_out[i] = vo;
  if (fex) fex[i] = make_vec<T>(e0, e1, e2);
  if (id_out && id_in && id_out != id_in) id_out[i] = id_in[i];
}

// From the gradients of (x', v', f_ex) to those of (x, v, F_c, F_fl, a_f).
template <typename T>
__global__ void __launch_bounds__(256) k_integrate_adj(DParams<T> P, int64_t n, const pos_t<T>* __restrict__ pos,
                                                        const vec_t<T>* __restrict__ gxo,
                                                        const vec_t<T>* __restrict__ gvo,
                                                        const vec_t<T>* __restrict__ gfe, vec_t<T>* __restrict__ gxi,
                                                        vec_t<T>* __restrict__ gvi, vec_t<T>* __restrict__ gFc,
                                                        vec_t<T>* __restrict__ gFfl, vec_t<T>* __restrict__ gaf) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const vec_t<T> gx = gxo[i];
  const IntegrateAdj<T> o =
      integrate_adj_granule(P, radius_of(pos[i]), gx, gvo[i], gfe ? gfe[i] : make_vec<T>(0, 0, 0));
  gxi[i] = gx;
  gvi[i] = make_vec<T>(o.gvt[0], o.gvt[1], o.gvt[2]);
  gFc[i] = make_vec<T>(o.gFc[0], o.gFc[1], o.gFc[2]);
  gFfl[i] = make_vec<T>(o.gFfl[0], o.gFfl[1], o.gFfl[2]);
  gaf[i] = make_vec<T>(o.gaf[0], o.gaf[1], o.gaf[2]);
}

}  // namespace gic

using namespace gic;

extern "C" int gic_integrate(const GicGrid* grid, const GicParams* params, const GicGranules* in, const void* F_c,
                             const void* F_fl, const void* a_f, GicGranules* out, void* f_ex, gic_stream_t stream) {
  GIC_RANGE("gic_integrate");
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if ((rc = check_granules(in, "gic_integrate in"))) return rc;
  if ((rc = check_granules(out, "gic_integrate out"))) return rc;
  if (in->n != out->n || in->precision != out->precision)
    return set_error(GIC_ERR_INVALID, "gic_integrate: in/out differ in size or precision");
  int64_t n = in->n;
  if (n == 0) return GIC_OK;
  if (!F_c || !F_fl || !a_f) return set_error(GIC_ERR_INVALID, "gic_integrate: null force array");
  if ((rc = check_vecs(in->precision, "gic_integrate", {F_c, F_fl, a_f, f_ex}))) return rc;
  if (in->precision == GIC_FP32) {
    DParams<float> P;
    if ((rc = make_params(params, &P))) return rc;
    k_integrate<float><<<grid_blocks(n, 256), 256, 0, stream>>>(
        G, P, n, in->cell, (const uint4*)in->pos, (const float4*)in->vel, (const float4*)F_c, (const float4*)F_fl,
        (const float4*)a_f, out->cell, (uint4*)out->pos, (float4*)out->vel, (float4*)f_ex, in->id, out->id,
        status_word());
  } else {
    DParams<double> P;
    if ((rc = make_params(params, &P))) return rc;
    k_integrate<double><<<grid_blocks(n, 256), 256, 0, stream>>>(
        G, P, n, in->cell, (const d4*)in->pos, (const d4*)in->vel, (const d4*)F_c, (const d4*)F_fl, (const d4*)a_f,
        out->cell, (d4*)out->pos, (d4*)out->vel, (d4*)f_ex, in->id, out->id, status_word());
  }
  count_launches(1);
  GIC_CHECK_LAUNCH("gic_integrate");
  return GIC_OK;
}

extern "C" int gic_integrate_adj(const GicGrid* grid, const GicParams* params, const GicGranules* in,
                                 const void* g_pos_out, const void* g_vel_out, const void* g_f_ex, void* g_pos_in,
                                 void* g_vel_in, void* gF_c, void* gF_fl, void* ga_f, gic_stream_t stream) {
  GIC_RANGE("gic_integrate_adj");
  DGrid G;
  int rc = make_grid(grid, &G);
  if (rc) return rc;
  if ((rc = check_granules(in, "gic_integrate_adj"))) return rc;
  int64_t n = in->n;
  if (n == 0) return GIC_OK;
  if (!g_pos_out || !g_vel_out || !g_pos_in || !g_vel_in || !gF_c || !gF_fl || !ga_f)
    return set_error(GIC_ERR_INVALID, "gic_integrate_adj: null array");
  if ((rc = check_vecs(in->precision, "gic_integrate_adj", {g_pos_out, g_vel_out, g_f_ex, g_pos_in, g_vel_in, gF_c, gF_fl, ga_f})))
    return rc;
  if (in->precision == GIC_FP32) {
    DParams<float> P;
    if ((rc = make_params(params, &P))) return rc;
    k_integrate_adj<float><<<grid_blocks(n, 256), 256, 0, stream>>>(
        P, n, (const uint4*)in->pos, (const float4*)g_pos_out, (const float4*)g_vel_out, (const float4*)g_f_ex,
        (float4*)g_pos_in, (float4*)g_vel_in, (float4*)gF_c, (float4*)gF_fl, (float4*)ga_f);
  } else {
    DParams<double> P;
    if ((rc = make_params(params, &P))) return rc;
    k_integrate_adj<double><<<grid_blocks(n, 256), 256, 0, stream>>>(
        P, n, (const d4*)in->pos, (const d4*)g_pos_out, (const d4*)g_vel_out, (const d4*)g_f_ex, (d4*)g_pos_in,
        (d4*)g_vel_in, (d4*)gF_c, (d4*)gF_fl, (d4*)ga_f);
  }
  count_launches(1);
  GIC_CHECK_LAUNCH("gic_integrate_adj");
  return GIC_OK;
}
