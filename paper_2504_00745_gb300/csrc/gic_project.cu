// gic_project.cu -- the velocity and density projections that consume
// alpha_s (Sec. 5.1: Eqs. discret momentum, backward Euler, bring2, ppe1 a/b
// and position change; the limits stated after Eq. position change; the face
// weight beta_j of the appendix on the Push-Out boundary condition).
//
// Both systems are A p = b with (A p)_c = sum over the cell's faces of
// beta_f (p_c - p_nb): beta_f the mean alpha_f' of the two cells, the inner
// cell's alpha_f' on an open side (p_nb = 0 beyond), no term on a solid side.
// A is symmetric positive definite (an open side is required).
//
// GB300's FP64 rate is a small fraction of its FP32 rate, and an all-FP32 CG
// stalls at a relative residual of order eps_32 * cond(A) (~1e-3 on a 128^3
// box with one open side).  So the solve is mixed-precision iterative
// refinement: the solution p and each residual b - A p are FP64 (one FP64
// stencil pass per refinement step), and each correction A e = r comes from
// an FP32 Jacobi-preconditioned conjugate-gradient run to a modest reduction.
// A CG iteration is two kernels: the new direction fused with y = A d
// (z-marching tiles), then the vector updates; 16 iterations run as one CUDA
// graph between host reads of the stop flag.
// Reductions are deterministic: every block writes a partial sum, and the
// block that finishes last (an atomic ticket, no waiting) adds the partials
// in index order and writes the scalar that the next kernels read.
#include <math.h>
#include <string.h>

#include <vector>

#include "gic_internal.cuh"

namespace gic {

constexpr int kProjThreads = 256;

struct PGrid {
  int nx, ny, nz;
  int64_t n;        // cells (< 2^31: cell indices are 32-bit)
  int64_t nxy;      // nx * ny
  int open[6];      // -x, +x, -y, +y, -z, +z
};

__device__ __forceinline__ void cell_ijk(const PGrid& g, int64_t c, int& i, int& j, int& k) {
  const unsigned cu = (unsigned)c, nxy = (unsigned)g.nxy, nx = (unsigned)g.nx;
  const unsigned kk = cu / nxy;
  const unsigned r = cu - kk * nxy;
  const unsigned jj = r / nx;
  k = (int)kk;
  j = (int)jj;
  i = (int)(r - jj * nx);
}

// Device scalars of the solver (in the workspace).
struct ProjRed {
  double dy;       // d . A d
  double rz[2];    // r . M^-1 r of the current and the next CG iterate
  double rr;       // r . r of the FP32 iterate
  double rr64, bb; // ||b - A p||^2 (FP64) and ||b||^2
  double rr_stop;  // the CG run stops when r . r <= rr_stop
  unsigned ticket; // blocks done with the current kernel
  int done, iters; // stop flag and iteration count of the CG run
};

// Every block calls it once with its partials (valid in thread 0); the
// block that arrives last sums all partials in index order into out[]
// (NV values, component-major partials P[v * gridDim.x + block]) and resets
// the ticket.  Returns true in that block (all threads).
template <int NV>
__device__ __forceinline__ bool reduce_last(const double (&v)[NV], double* __restrict__ P, ProjRed* red,
                                            double* const (&out)[NV]) {
  __shared__ bool last;
  __shared__ double smem[32];
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) P[q * gridDim.x + blockIdx.x] = v[q];
    __threadfence();
    last = atomicAdd(&red->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double s = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) s += __ldcg(&P[q * gridDim.x + b]);
    s = block_sum(s, smem);
    if (threadIdx.x == 0) *out[q] = s;
  }
  if (threadIdx.x == 0) red->ticket = 0u;
  return true;
}

// Visits the six faces of cell (i, j, k): f(neighbour index or -1, face
// kind) with kind 0 = interior face, 1 = open side, 2 = solid side.
template <typename F>
__device__ __forceinline__ void for_faces(const PGrid& g, int i, int j, int k, int64_t c, F f) {
  const int idx[3] = {i, j, k};
  const int n[3] = {g.nx, g.ny, g.nz};
  const int64_t stride[3] = {1, g.nx, g.nxy};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (idx[a] > 0)
      f(c - stride[a], 0);
    else
      f((int64_t)-1, g.open[2 * a] ? 1 : 2);
    if (idx[a] < n[a] - 1)
      f(c + stride[a], 0);
    else
      f((int64_t)-1, g.open[2 * a + 1] ? 1 : 2);
  }
}

// A flag read once per block (uniform over the block's threads).
__device__ __forceinline__ bool block_flag(const int* flag) {
  __shared__ int f;
  if (threadIdx.x == 0) f = *(volatile const int*)flag;
  __syncthreads();
  const bool r = f != 0;
  __syncthreads();
  return r;
}

// Compensated FP32 sum (Kahan): the CG's per-thread dot-product partials stay
// off the FP64 pipe, whose rate on GB300 is a small fraction of FP32's.
struct KahanF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

// alpha_f' = 1 - min(alpha_s, alpha_s_max); a NaN alpha_s stays NaN (and is reported)
__device__ __forceinline__ double target_fraction(double alpha_s, double amax) {
  return 1.0 - (alpha_s > amax ? amax : alpha_s);
}

// alpha_f' as float (the FP32 operator of the corrections; the FP64 residual
// forms it from alpha_s itself).
__global__ void __launch_bounds__(kProjThreads) k_proj_prep(PGrid g, const double* __restrict__ alpha_s, double amax,
                                                            float* __restrict__ ap32) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.n; c += (int64_t)gridDim.x * blockDim.x)
    ap32[c] = (float)target_fraction(alpha_s[c], amax);
}

// The inverse Jacobi diagonal of the FP32 operator (the preconditioner).
__global__ void __launch_bounds__(kProjThreads) k_proj_diag(PGrid g, unsigned open, const float* __restrict__ ap32,
                                                            float* __restrict__ invd) {
  const unsigned n = (unsigned)g.n, nx = (unsigned)g.nx, ny = (unsigned)g.ny, nz = (unsigned)g.nz;
  const unsigned nxy = nx * ny;
  for (unsigned c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    const unsigned k = c / nxy, rem = c - k * nxy, j = rem / nx, i = rem - j * nx;
    const float ac = ap32[c];
    float diag = 0.f;
    auto side = [&](bool inside, unsigned nb, unsigned bit) {
      if (inside)
        diag += 0.5f * (ac + ap32[nb]);
      else if (open & bit)
        diag += ac;
    };
    side(i > 0, c - 1, 1u);
    side(i + 1 < nx, c + 1, 2u);
    side(j > 0, c - nx, 4u);
    side(j + 1 < ny, c + nx, 8u);
    side(k > 0, c - nxy, 16u);
    side(k + 1 < nz, c + nxy, 32u);
    invd[c] = diag > 0.f ? 1.f / diag : 0.f;
  }
}

struct ProjScales {
  double vel;       // rho h / dt: b1 = vel * (sum of beta v over low faces - over high faces)
  double den;       // -rho h^2 / dt^2: b2 = den * alpha' (1 - clamp(ratio))
  double rmin, rmax, amax;
};

// FP64 residual r = b - A p of system `which` (1: velocity, 2: density);
// starts the FP32 correction run: r32 = r, d = M^-1 r, e = 0.  Scalars:
// ||r||^2 (FP64), ||b||^2 and r32 . M^-1 r32 (the CG's first rho).
__global__ void __launch_bounds__(kProjThreads) k_proj_residual(
    PGrid g, int which, ProjScales S, const double* __restrict__ alpha_s, const float* __restrict__ alpha_star,
    const float* __restrict__ u, const float* __restrict__ v, const float* __restrict__ w,
    const double* __restrict__ p, const float* __restrict__ invd, float* __restrict__ r32, float* __restrict__ d32,
    float* __restrict__ e32, double inner_tol2, double* __restrict__ P, ProjRed* red, uint32_t* status) {
  __shared__ double smem[64];
  double rr = 0.0, bb = 0.0;
  KahanF rzk;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.n; c += (int64_t)gridDim.x * blockDim.x) {
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    const double ac = target_fraction(alpha_s[c], S.amax);
    const double pc = p[c];
    double Ap = 0.0;
    for_faces(g, i, j, k, c, [&](int64_t nb, int kind) {
      if (kind == 0)
        Ap += 0.5 * (ac + target_fraction(alpha_s[nb], S.amax)) * (pc - p[nb]);
      else if (kind == 1)
        Ap += ac * pc;
    });
    double b;
    if (which == 1) {
      // b1 = (rho h / dt) (sum over low faces - sum over high faces) of beta v*
      const int64_t nxf = g.nx + 1, nyf = g.ny + 1;
      const int64_t fu = i + nxf * (j + (int64_t)g.ny * k);
      const int64_t fv = i + (int64_t)g.nx * (j + nyf * k);
      const int64_t fw = c;  // w: i + nx (j + ny k) on z-face k
      const double vlo[3] = {u[fu], v[fv], w[fw]};
      const double vhi[3] = {u[fu + 1], v[fv + g.nx], w[fw + g.nxy]};
      const int idx[3] = {i, j, k};
      const int nn[3] = {g.nx, g.ny, g.nz};
      const int64_t stride[3] = {1, g.nx, g.nxy};
      double flux = 0.0;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        double blo, bhi;
        if (idx[a] > 0)
          blo = 0.5 * (ac + target_fraction(alpha_s[c - stride[a]], S.amax));
        else
          blo = g.open[2 * a] ? ac : 0.0;
        if (idx[a] < nn[a] - 1)
          bhi = 0.5 * (ac + target_fraction(alpha_s[c + stride[a]], S.amax));
        else
          bhi = g.open[2 * a + 1] ? ac : 0.0;
        flux += blo * vlo[a] - bhi * vhi[a];
      }
      b = S.vel * flux;
    } else {
      const double q = (double)alpha_star[c] / ac;
      const double ratio = q < S.rmin ? S.rmin : (q > S.rmax ? S.rmax : q);  // NaN stays NaN
      b = S.den * ac * (1.0 - ratio);
    }
    const double r = b - Ap;
    if (!isfinite(r)) raise_status(status, GIC_STATUS_NONFINITE);
    const float rf = (float)r;
    const float df = invd[c] * rf;
    r32[c] = rf;
    d32[c] = df;
    e32[c] = 0.f;
    rr += r * r;
    bb += b * b;
    rzk.add(rf * df);
  }
  block_sum2(rr, bb, smem);
  __syncthreads();
  const double rz = block_sum((double)rzk.s, smem);
  const double vals[3] = {rr, bb, rz};
  double* const outs[3] = {&red->rr64, &red->bb, &red->rz[0]};
  if (reduce_last<3>(vals, P, red, outs) && threadIdx.x == 0) {  // arm the CG run on this residual
    red->rr_stop = inner_tol2 * red->rr64;
    red->done = 0;
    red->iters = 0;
  }
}

// CG step 1 (with the previous step's new direction): d_new = M^-1 r +
// beta d_old (beta = 0 on a run's first iteration), y = A d_new (FP32
// operator) and d_new . y into red->dy.  d_old and d_new are different
// buffers: neighbouring tiles read d_old while this one writes d_new.
// A CTA covers a kTX x kTY column tile and marches over lz planes in z: its
// threads keep the column's d_new and alpha_f' at k-1, k, k+1 in registers
// and the plane's values at the tile's four sides in shared memory.
constexpr int kTX = 32, kTY = 8;  // kTX * kTY = kProjThreads
static_assert(kTX * kTY == kProjThreads, "tile shape");

__global__ void __launch_bounds__(kProjThreads) k_cg_dir_apply(PGrid g, unsigned open, int lz, int tiles_x,
                                                               int tiles_y, int cur, const float* __restrict__ ap32,
                                                               const float* __restrict__ r,
                                                               const float* __restrict__ invd,
                                                               const float* __restrict__ d_old,
                                                               float* __restrict__ d_new, float* __restrict__ y,
                                                               double* __restrict__ P, ProjRed* red) {
  __shared__ float s_d[kTY + 2][kTX + 2];
  __shared__ float s_a[kTY + 2][kTX + 2];
  __shared__ double smem[32];
  if (block_flag(&red->done)) return;
  const float be = red->iters == 0 ? 0.f : (float)(red->rz[cur] / red->rz[cur ^ 1]);
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int b = blockIdx.x;
  const int bx = b % tiles_x, bt = b / tiles_x, by = bt % tiles_y, bz = bt / tiles_y;
  const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
  const int x0 = bx * kTX, y0 = by * kTY;
  const int i = x0 + tx, j = y0 + ty;
  const int z0 = bz * lz, z1 = min(z0 + lz, nz);
  const bool act = i < nx && j < ny;
  auto at = [&](int ii, int jj, int kk) -> unsigned {
    return (unsigned)ii + (unsigned)nx * ((unsigned)jj + (unsigned)ny * (unsigned)kk);
  };
  auto dn = [&](unsigned c) -> float { return fmaf(be, d_old[c], invd[c] * r[c]); };
  // this thread's entry of the tile's side ring (80 entries; corners are not needed)
  int ri = -1, rj = -1, sx = 0, sy = 0;
  {
    const int q = threadIdx.x;
    if (q < kTX) {
      ri = x0 + q, rj = y0 - 1, sx = q + 1, sy = 0;
    } else if (q < 2 * kTX) {
      ri = x0 + q - kTX, rj = y0 + kTY, sx = q - kTX + 1, sy = kTY + 1;
    } else if (q < 2 * kTX + kTY) {
      ri = x0 - 1, rj = y0 + q - 2 * kTX, sx = 0, sy = q - 2 * kTX + 1;
    } else if (q < 2 * kTX + 2 * kTY) {
      ri = x0 + kTX, rj = y0 + q - 2 * kTX - kTY, sx = kTX + 1, sy = q - 2 * kTX - kTY + 1;
    }
  }
  const bool ring = ri >= 0 && ri < nx && rj >= 0 && rj < ny;
  float dm = 0.f, dc = 0.f, dp = 0.f, am = 0.f, ac = 0.f, apl = 0.f;
  if (act) {
    if (z0 > 0) {
      const unsigned c = at(i, j, z0 - 1);
      dm = dn(c);
      am = ap32[c];
    }
    const unsigned c = at(i, j, z0);
    dc = dn(c);
    ac = ap32[c];
  }
  KahanF dyk;
  for (int k = z0; k < z1; ++k) {
    s_d[ty + 1][tx + 1] = dc;
    s_a[ty + 1][tx + 1] = ac;
    if (sx | sy) {  // a ring thread
      float rd = 0.f, ra = 0.f;
      if (ring) {
        const unsigned c = at(ri, rj, k);
        rd = dn(c);
        ra = ap32[c];
      }
      s_d[sy][sx] = rd;
      s_a[sy][sx] = ra;
    }
    __syncthreads();
    if (act) {
      if (k + 1 < nz) {
        const unsigned c = at(i, j, k + 1);
        dp = dn(c);
        apl = ap32[c];
      }
      float acc = 0.f;
      if (i > 0)
        acc += 0.5f * (ac + s_a[ty + 1][tx]) * (dc - s_d[ty + 1][tx]);
      else if (open & 1u)
        acc += ac * dc;
      if (i + 1 < nx)
        acc += 0.5f * (ac + s_a[ty + 1][tx + 2]) * (dc - s_d[ty + 1][tx + 2]);
      else if (open & 2u)
        acc += ac * dc;
      if (j > 0)
        acc += 0.5f * (ac + s_a[ty][tx + 1]) * (dc - s_d[ty][tx + 1]);
      else if (open & 4u)
        acc += ac * dc;
      if (j + 1 < ny)
        acc += 0.5f * (ac + s_a[ty + 2][tx + 1]) * (dc - s_d[ty + 2][tx + 1]);
      else if (open & 8u)
        acc += ac * dc;
      if (k > 0)
        acc += 0.5f * (ac + am) * (dc - dm);
      else if (open & 16u)
        acc += ac * dc;
      if (k + 1 < nz)
        acc += 0.5f * (ac + apl) * (dc - dp);
      else if (open & 32u)
        acc += ac * dc;
      const unsigned c = at(i, j, k);
      d_new[c] = dc;
      y[c] = acc;
      dyk.add(dc * acc);
    }
    __syncthreads();
    dm = dc;
    dc = dp;
    am = ac;
    ac = apl;
  }
  const double dy = block_sum((double)dyk.s, smem);
  const double vals[1] = {dy};
  double* const outs[1] = {&red->dy};
  reduce_last<1>(vals, P, red, outs);
}

// CG step 2: alpha = rho / (d . y); e += alpha d; r -= alpha y; the new rho
// = r . M^-1 r and r . r (four cells per thread and step, float4).  The last
// block counts the iteration and sets the stop flag when r . r <= rr_stop.
__global__ void __launch_bounds__(kProjThreads) k_cg_update(PGrid g, int cur, const float* __restrict__ d,
                                                            const float* __restrict__ y, const float* __restrict__ invd,
                                                            float* __restrict__ e, float* __restrict__ r,
                                                            double* __restrict__ P, ProjRed* red) {
  __shared__ double smem[64];
  if (block_flag(&red->done)) return;
  const double dy = red->dy, rz = red->rz[cur];  // the same values in every block
  if (!(dy > 0.0) || !isfinite(rz)) {  // d = 0 (r = 0: converged) or breakdown: stop this run
    if (blockIdx.x == 0 && threadIdx.x == 0) red->done = 1;
    return;
  }
  const float al = (float)(rz / dy);
  KahanF rzk, rrk;
  const unsigned n = (unsigned)g.n, n4 = n / 4u;
  const unsigned t0 = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  for (unsigned q = t0; q < n4; q += stride) {  // arrays are 256-byte aligned
    const float4 dq = reinterpret_cast<const float4*>(d)[q];
    const float4 yq = reinterpret_cast<const float4*>(y)[q];
    const float4 iq = reinterpret_cast<const float4*>(invd)[q];
    float4 eq = reinterpret_cast<const float4*>(e)[q];
    float4 rq = reinterpret_cast<const float4*>(r)[q];
    eq.x = fmaf(al, dq.x, eq.x);
    eq.y = fmaf(al, dq.y, eq.y);
    eq.z = fmaf(al, dq.z, eq.z);
    eq.w = fmaf(al, dq.w, eq.w);
    rq.x = fmaf(-al, yq.x, rq.x);
    rq.y = fmaf(-al, yq.y, rq.y);
    rq.z = fmaf(-al, yq.z, rq.z);
    rq.w = fmaf(-al, yq.w, rq.w);
    reinterpret_cast<float4*>(e)[q] = eq;
    reinterpret_cast<float4*>(r)[q] = rq;
    rzk.add(rq.x * (iq.x * rq.x) + rq.y * (iq.y * rq.y) + rq.z * (iq.z * rq.z) + rq.w * (iq.w * rq.w));
    rrk.add(rq.x * rq.x + rq.y * rq.y + rq.z * rq.z + rq.w * rq.w);
  }
  for (unsigned c = 4u * n4 + t0; c < n; c += stride) {
    const float dc = d[c];
    e[c] = fmaf(al, dc, e[c]);
    const float rc = fmaf(-al, y[c], r[c]);
    r[c] = rc;
    rzk.add(rc * (invd[c] * rc));
    rrk.add(rc * rc);
  }
  double rz_new = (double)rzk.s, rr = (double)rrk.s;
  block_sum2(rz_new, rr, smem);
  const double vals[2] = {rz_new, rr};
  double* const outs[2] = {&red->rz[cur ^ 1], &red->rr};
  if (reduce_last<2>(vals, P, red, outs) && threadIdx.x == 0) {
    red->iters += 1;
    if (!(red->rr > red->rr_stop)) red->done = 1;  // also stops on NaN
  }
}

// p += e (the FP32 correction into the FP64 solution).
__global__ void __launch_bounds__(kProjThreads) k_proj_add(int64_t n, double* __restrict__ p,
                                                           const float* __restrict__ e) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
    p[c] += (double)e[c];
}

// Face outputs: v' = v* - (dt/rho) grad p1 and dx = clamp(-(dt^2/rho) grad p2, -h, h);
// zero on solid sides' faces.  Faces of the three grids in one index range.
__global__ void __launch_bounds__(kProjThreads) k_proj_faces(
    PGrid g, double h, double dt_rho, double dt2_rho, const double* __restrict__ p1, const double* __restrict__ p2,
    const float* __restrict__ u, const float* __restrict__ v, const float* __restrict__ w, float* __restrict__ uo,
    float* __restrict__ vo, float* __restrict__ wo, float* __restrict__ dxu, float* __restrict__ dxv,
    float* __restrict__ dxw) {
  const int64_t nu = (int64_t)(g.nx + 1) * g.ny * g.nz, nv = (int64_t)g.nx * (g.ny + 1) * g.nz,
                nw = (int64_t)g.nx * g.ny * (g.nz + 1);
  const double inv_h = 1.0 / h;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nu + nv + nw;
       q += (int64_t)gridDim.x * blockDim.x) {
    int a;
    int64_t f;
    if (q < nu) {
      a = 0;
      f = q;
    } else if (q < nu + nv) {
      a = 1;
      f = q - nu;
    } else {
      a = 2;
      f = q - nu - nv;
    }
    // face (i, j, k) on grid a: x fastest with n_a + 1 samples along a
    int ns[3] = {g.nx, g.ny, g.nz};
    ns[a] += 1;
    const int64_t sxy = (int64_t)ns[0] * ns[1];
    const int k = (int)(f / sxy);
    const int64_t rem = f - (int64_t)k * sxy;
    const int j = (int)(rem / ns[0]);
    const int i = (int)(rem - (int64_t)j * ns[0]);
    const int idx[3] = {i, j, k};
    const int m = a == 0 ? g.nx : (a == 1 ? g.ny : g.nz);
    const int64_t stride = a == 0 ? 1 : (a == 1 ? g.nx : g.nxy);
    // the cell on the high side has index idx (if idx[a] < m), the low side idx - e_a (if idx[a] > 0)
    const int64_t cR = i + (int64_t)g.nx * (j + (int64_t)g.ny * k);  // valid when idx[a] < m
    const bool lo_in = idx[a] > 0, hi_in = idx[a] < m;
    const bool solid = (!lo_in && !g.open[2 * a]) || (!hi_in && !g.open[2 * a + 1]);
    float vo_ = 0.f, dx_ = 0.f;
    if (!solid) {
      const int64_t cL = cR - stride;
      const double pR1 = hi_in ? p1[cR] : 0.0, pL1 = lo_in ? p1[cL] : 0.0;
      const double pR2 = hi_in ? p2[cR] : 0.0, pL2 = lo_in ? p2[cL] : 0.0;
      const float* vin = a == 0 ? u : (a == 1 ? v : w);
      vo_ = (float)((double)vin[f] - dt_rho * (pR1 - pL1) * inv_h);
      const double dxf = -dt2_rho * (pR2 - pL2) * inv_h;
      dx_ = (float)(dxf < -h ? -h : (dxf > h ? h : dxf));
    }
    if (uo) (a == 0 ? uo : (a == 1 ? vo : wo))[f] = vo_;
    if (dxu) (a == 0 ? dxu : (a == 1 ? dxv : dxw))[f] = dx_;
  }
}

// ---- host side ----

struct ProjWs {
  float *ap32, *invd, *r, *d[2], *y, *e;  // d: the CG direction, double-buffered
  double* P;    // 3 * max(blocks) partial sums
  ProjRed* red;
};

// Tiles and z-planes per CTA of k_cg_dir_apply: lz halves from 64 until the
// grid has at least 6 CTAs per SM.
struct TileGrid {
  int tiles_x, tiles_y, lz, blocks;
};
static TileGrid tile_grid(const PGrid& g) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  TileGrid t;
  t.tiles_x = (g.nx + kTX - 1) / kTX;
  t.tiles_y = (g.ny + kTY - 1) / kTY;
  t.lz = 64;
  for (;;) {
    const int64_t b = (int64_t)t.tiles_x * t.tiles_y * ((g.nz + t.lz - 1) / t.lz);
    if (b >= 6 * (int64_t)(sms > 0 ? sms : 152) || t.lz <= 4) break;
    t.lz /= 2;
  }
  t.blocks = (int)((int64_t)t.tiles_x * t.tiles_y * ((g.nz + t.lz - 1) / t.lz));
  return t;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

static int proj_blocks(int64_t n) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (n + kProjThreads - 1) / kProjThreads;
  const int64_t cap = 8 * (int64_t)(sms > 0 ? sms : 152);
  return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

// Workspace for n cells and nblk blocks (laid out by the same walk that
// measures it).
static size_t proj_layout(int64_t n, int nblk, char* base, ProjWs* W) {
  // nblk: the most CTAs any kernel with partial sums launches
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += align256(bytes);
    return p;
  };
  ProjWs w;
  w.ap32 = (float*)take(4 * (size_t)n);
  w.invd = (float*)take(4 * (size_t)n);
  w.r = (float*)take(4 * (size_t)n);
  w.d[0] = (float*)take(4 * (size_t)n);
  w.d[1] = (float*)take(4 * (size_t)n);
  w.y = (float*)take(4 * (size_t)n);
  w.e = (float*)take(4 * (size_t)n);
  w.P = (double*)take(3 * 8 * (size_t)nblk);
  w.red = (ProjRed*)take(sizeof(ProjRed));
  if (W) *W = w;
  return off;
}

static int proj_grid(const GicGrid* grid, PGrid* g) {
  if (!grid) return set_error(GIC_ERR_INVALID, "gic_project: grid is NULL");
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return set_error(GIC_ERR_INVALID, "gic_project: empty grid");
  if (!(grid->dx > 0.0) || !isfinite(grid->dx)) return set_error(GIC_ERR_INVALID, "gic_project: dx must be positive");
  g->nx = grid->nx;
  g->ny = grid->ny;
  g->nz = grid->nz;
  g->nxy = (int64_t)grid->nx * grid->ny;
  g->n = g->nxy * grid->nz;
  if (g->n >= ((int64_t)1 << 31)) return set_error(GIC_ERR_INVALID, "gic_project: 2^31 cells or more");
  return GIC_OK;
}

// The solver's scalars, read to the host.
static int read_red(const ProjRed* dev, ProjRed* host, cudaStream_t st) {
  if (cudaMemcpyAsync(host, dev, sizeof(ProjRed), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return set_error(GIC_ERR_CUDA, "gic_project: reading the solver's scalars failed");
  return wait_stream(st, 60000, "gic_project");
}

}  // namespace gic

using namespace gic;

extern "C" int gic_project_workspace_size(const GicGrid* grid, size_t* bytes) {
  PGrid g;
  int rc = proj_grid(grid, &g);
  if (rc) return rc;
  if (!bytes) return set_error(GIC_ERR_INVALID, "gic_project_workspace_size: bytes is NULL");
  const TileGrid tg = tile_grid(g);
  const int nb = proj_blocks(g.n);
  *bytes = proj_layout(g.n, nb > tg.blocks ? nb : tg.blocks, nullptr, nullptr);
  return GIC_OK;
}

extern "C" int gic_project(const GicGrid* grid, const GicProjParams* P, const double* alpha_s, const float* alpha_star,
                           const float* u, const float* v, const float* w, double* p1, double* p2, float* u_out,
                           float* v_out, float* w_out, float* dx_u, float* dx_v, float* dx_w, void* ws,
                           size_t ws_bytes, GicProjInfo* info, gic_stream_t stream_) {
  PGrid g;
  int rc = proj_grid(grid, &g);
  if (rc) return rc;
  if (!P) return set_error(GIC_ERR_INVALID, "gic_project: params is NULL");
  if (!(P->dt > 0.0) || !(P->rho_f > 0.0)) return set_error(GIC_ERR_INVALID, "gic_project: dt and rho_f must be positive");
  if (!(P->alpha_s_max > 0.0 && P->alpha_s_max < 1.0))
    return set_error(GIC_ERR_INVALID, "gic_project: alpha_s_max must lie in (0, 1)");
  if (!(P->ratio_min > 0.0 && P->ratio_min <= 1.0 && P->ratio_max >= 1.0 && isfinite(P->ratio_max)))
    return set_error(GIC_ERR_INVALID, "gic_project: need 0 < ratio_min <= 1 <= ratio_max");
  if (!(P->tol > 0.0) || !(P->inner_tol > 0.0 && P->inner_tol < 1.0))
    return set_error(GIC_ERR_INVALID, "gic_project: tol must be positive and inner_tol in (0, 1)");
  if (P->max_outer < 1 || P->max_inner < 1)
    return set_error(GIC_ERR_INVALID, "gic_project: max_outer and max_inner must be >= 1");
  bool any_open = false;
  for (int s = 0; s < 6; ++s) {
    if (P->open[s] != 0 && P->open[s] != 1) return set_error(GIC_ERR_INVALID, "gic_project: open[%d] must be 0 or 1", s);
    any_open |= P->open[s] == 1;
  }
  if (!any_open) return set_error(GIC_ERR_INVALID, "gic_project: at least one side must be open (p = 0 beyond it)");
  if (!alpha_s || !alpha_star || !u || !v || !w || !p1 || !p2)
    return set_error(GIC_ERR_INVALID, "gic_project: null input or pressure array");
  const bool vel_out = u_out || v_out || w_out, disp_out = dx_u || dx_v || dx_w;
  if (vel_out && !(u_out && v_out && w_out))
    return set_error(GIC_ERR_INVALID, "gic_project: give all three projected velocity arrays or none");
  if (disp_out && !(dx_u && dx_v && dx_w))
    return set_error(GIC_ERR_INVALID, "gic_project: give all three displacement arrays or none");
  unsigned open_bits = 0u;
  for (int s = 0; s < 6; ++s) {
    g.open[s] = P->open[s];
    if (P->open[s]) open_bits |= 1u << s;
  }
  const int nblk = proj_blocks(g.n);
  const TileGrid tg = tile_grid(g);
  const int pblk = nblk > tg.blocks ? nblk : tg.blocks;  // partial-sum slots
  const size_t need = proj_layout(g.n, pblk, nullptr, nullptr);
  if (!ws || ws_bytes < need)
    return set_error(GIC_ERR_WORKSPACE, "gic_project: workspace of %zu bytes needed, %zu given", need, ws_bytes);
  if ((uintptr_t)ws % 256) return set_error(GIC_ERR_ALIGN, "gic_project: workspace must be 256-byte aligned");
  cudaStream_t st = (cudaStream_t)stream_;
  ProjWs W;
  proj_layout(g.n, pblk, (char*)ws, &W);
  uint32_t* status = status_word();
  const double h = grid->dx;
  ProjScales S;
  S.vel = P->rho_f * h / P->dt;
  S.den = -P->rho_f * h * h / (P->dt * P->dt);
  S.rmin = P->ratio_min;
  S.rmax = P->ratio_max;
  S.amax = P->alpha_s_max;
  GicProjInfo inf;
  memset(&inf, 0, sizeof(inf));
  ProjRed hr;
  int64_t launches = 0;
  int rc2 = GIC_OK;

  if (cudaMemsetAsync(W.red, 0, sizeof(ProjRed), st) != cudaSuccess)
    return set_error(GIC_ERR_CUDA, "gic_project: clearing the solver's scalars failed");
  // one CG iteration; all arguments but the parity are fixed for the call
  auto cg_iteration = [&](int cur, cudaStream_t s_) {
    k_cg_dir_apply<<<tg.blocks, kProjThreads, 0, s_>>>(g, open_bits, tg.lz, tg.tiles_x, tg.tiles_y, cur, W.ap32,
                                                       W.r, W.invd, W.d[cur], W.d[cur ^ 1], W.y, W.P, W.red);
    k_cg_update<<<nblk, kProjThreads, 0, s_>>>(g, cur, W.d[cur ^ 1], W.y, W.invd, W.e, W.r, W.P, W.red);
  };
  // kChunk iterations as one CUDA graph (kChunk even: the parities repeat),
  // built when the first CG run needs it
  constexpr int kChunk = 16;
  cudaGraphExec_t chunk = nullptr;
  auto build_chunk = [&]() -> int {
    cudaStream_t cs = nullptr;
    cudaGraph_t gr = nullptr;
    bool ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      for (int q = 0; q < kChunk; ++q) cg_iteration(q & 1, cs);
      ok = cudaStreamEndCapture(cs, &gr) == cudaSuccess && gr != nullptr;
    }
    ok = ok && cudaGraphInstantiate(&chunk, gr, 0) == cudaSuccess;
    if (gr) cudaGraphDestroy(gr);
    if (cs) cudaStreamDestroy(cs);
    if (!ok) {
      cudaGetLastError();
      if (chunk) cudaGraphExecDestroy(chunk);
      chunk = nullptr;
      return set_error(GIC_ERR_CUDA, "gic_project: building the CG graph failed");
    }
    return GIC_OK;
  };
  k_proj_prep<<<nblk, kProjThreads, 0, st>>>(g, alpha_s, P->alpha_s_max, W.ap32);
  k_proj_diag<<<nblk, kProjThreads, 0, st>>>(g, open_bits, W.ap32, W.invd);
  launches += 2;
  for (int which = 1; which <= 2 && rc2 == GIC_OK; ++which) {
    double* p = which == 1 ? p1 : p2;
    const int sys = which - 1;
    if (cudaMemsetAsync(p, 0, sizeof(double) * g.n, st) != cudaSuccess) {
      rc2 = set_error(GIC_ERR_CUDA, "gic_project: clearing p failed");
      break;
    }
    for (int outer = 0;; ++outer) {
      k_proj_residual<<<nblk, kProjThreads, 0, st>>>(g, which, S, alpha_s, alpha_star, u, v, w, p, W.invd, W.r, W.d[0],
                                                     W.e, P->inner_tol * P->inner_tol, W.P, W.red, status);
      ++launches;
      if ((rc2 = read_red(W.red, &hr, st))) break;
      if (!isfinite(hr.rr64) || !isfinite(hr.bb)) {
        rc2 = set_error(GIC_ERR_INVALID, "gic_project: non-finite residual (check alpha_s, alpha_star and v*)");
        break;
      }
      inf.outer[sys] = outer;
      inf.rel_residual[sys] = hr.bb > 0.0 ? sqrt(hr.rr64 / hr.bb) : 0.0;
      if (hr.bb == 0.0 || hr.rr64 <= P->tol * P->tol * hr.bb) {
        inf.converged[sys] = 1;
        break;
      }
      if (outer >= P->max_outer) break;
      // FP32 CG on A e = r to a reduction of inner_tol (of the FP32 copy's r . r):
      // graph launches of kChunk iterations, the stop flag read after each
      int it = 0;
      for (;;) {
        if (P->max_inner - it >= kChunk) {
          if (!chunk && (rc2 = build_chunk())) break;
          if (cudaGraphLaunch(chunk, st) != cudaSuccess) {
            rc2 = set_error(GIC_ERR_CUDA, "gic_project: graph launch failed");
            break;
          }
          it += kChunk;
          launches += 2 * kChunk;
        } else {
          for (; it < P->max_inner; ++it) {
            cg_iteration(it & 1, st);
            launches += 2;
          }
        }
        cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) {
          rc2 = set_error(GIC_ERR_CUDA, "gic_project: %s", cudaGetErrorString(le));
          break;
        }
        if ((rc2 = read_red(W.red, &hr, st))) break;
        if (hr.done || it >= P->max_inner) break;
      }
      if (rc2) break;
      inf.inner[sys] += hr.iters;
      k_proj_add<<<nblk, kProjThreads, 0, st>>>(g.n, p, W.e);
      ++launches;
    }
  }
  if (rc2 == GIC_OK && (vel_out || disp_out)) {
    const int64_t nf = (int64_t)(g.nx + 1) * g.ny * g.nz + (int64_t)g.nx * (g.ny + 1) * g.nz +
                       (int64_t)g.nx * g.ny * (g.nz + 1);
    const int fb = (int)((nf + kProjThreads - 1) / kProjThreads < 4096 ? (nf + kProjThreads - 1) / kProjThreads : 4096);
    k_proj_faces<<<fb, kProjThreads, 0, st>>>(g, h, P->dt / P->rho_f, P->dt * P->dt / P->rho_f, p1, p2, u, v, w,
                                              u_out, v_out, w_out, dx_u, dx_v, dx_w);
    ++launches;
  }
  if (chunk) cudaGraphExecDestroy(chunk);
  count_launches(launches);
  if (rc2) return rc2;
  GIC_CHECK_LAUNCH("gic_project");
  if (info) *info = inf;
  return GIC_OK;
}
