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
// an FP32 conjugate-gradient run, preconditioned by a geometric multigrid
// V-cycle, to a modest reduction.  The CG iterations run as CUDA graphs of a
// few iterations between host reads of the stop flag.
// Reductions are deterministic: every block writes a partial sum, and the
// block that finishes last (an atomic ticket, no waiting) adds the partials
// in index order and writes the scalar that the next kernels read.
#include <math.h>
#include <string.h>

#include "gic_internal.cuh"

namespace gic {

constexpr int kProjThreads = 256;

struct PGrid {
  int nx, ny, nz;
  int64_t n;        // cells (< 2^30: cell and face indices are 32-bit)
  int64_t nxy;      // nx * ny
  int open[6];      // -x, +x, -y, +y, -z, +z
};

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

struct ProjScales {
  double vel;       // rho h / dt: b1 = vel * (sum of beta v over low faces - over high faces)
  double den;       // -rho h^2 / dt^2: b2 = den * alpha' (1 - clamp(ratio))
  double rmin, rmax, amax;
};

// FP64 face weights of the operator (computed once per call, so that each
// residual pass spends its FP64 work on the stencil itself): the mean
// alpha_f' of the two cells, the inner cell's on an open side, 0 on a solid
// side.  Face arrays as the velocity components, x fastest.
__global__ void __launch_bounds__(kProjThreads) k_proj_faces64(PGrid g, unsigned open, const double* __restrict__ alpha_s,
                                                               double amax, double* __restrict__ fx,
                                                               double* __restrict__ fy, double* __restrict__ fz) {
  const unsigned nx = g.nx, ny = g.ny, nz = g.nz;
  const unsigned nu = (nx + 1) * ny * nz, nv = nx * (ny + 1) * nz, nw = nx * ny * (nz + 1);
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < nu + nv + nw; q += gridDim.x * blockDim.x) {
    unsigned a, f;
    if (q < nu) {
      a = 0, f = q;
    } else if (q < nu + nv) {
      a = 1, f = q - nu;
    } else {
      a = 2, f = q - nu - nv;
    }
    const unsigned sx = nx + (a == 0), sy = ny + (a == 1);
    const unsigned k = f / (sx * sy), rem = f - k * sx * sy, j = rem / sx, i = rem - j * sx;
    const unsigned pos = a == 0 ? i : (a == 1 ? j : k);
    const unsigned m = a == 0 ? nx : (a == 1 ? ny : nz);
    const unsigned stride = a == 0 ? 1u : (a == 1 ? nx : nx * ny);
    // the cell above the face (valid when pos < m) and the one below (pos > 0)
    const unsigned c_hi = i + nx * (j + ny * k), c_lo = c_hi - stride;
    double wgt;
    if (pos > 0 && pos < m)
      wgt = 0.5 * (target_fraction(alpha_s[c_hi], amax) + target_fraction(alpha_s[c_lo], amax));
    else if (pos == 0)
      wgt = (open >> (2 * a)) & 1u ? target_fraction(alpha_s[c_hi], amax) : 0.0;
    else
      wgt = (open >> (2 * a + 1)) & 1u ? target_fraction(alpha_s[c_lo], amax) : 0.0;
    (a == 0 ? fx : (a == 1 ? fy : fz))[f] = wgt;
  }
}

// FP64 residual r = b - A p of system `which` (1: velocity, 2: density);
// starts the FP32 correction run: r32 = r, e = 0, and arms its stop test.
// Scalars: ||r||^2 (FP64) and ||b||^2.
__global__ void __launch_bounds__(kProjThreads) k_proj_residual(
    PGrid g, int which, ProjScales S, const double* __restrict__ alpha_s, const float* __restrict__ alpha_star,
    const float* __restrict__ u, const float* __restrict__ v, const float* __restrict__ w,
    const double* __restrict__ fx, const double* __restrict__ fy, const double* __restrict__ fz,
    const double* __restrict__ p, float* __restrict__ r32, float* __restrict__ e32, double inner_tol2,
    double* __restrict__ P, ProjRed* red, uint32_t* status) {
  __shared__ double smem[64];
  double rr = 0.0, bb = 0.0;
  const unsigned n = (unsigned)g.n, nx = g.nx, ny = g.ny, nz = g.nz, nxy = nx * ny;
  for (unsigned c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    const unsigned k = c / nxy, rem = c - k * nxy, j = rem / nx, i = rem - j * nx;
    const unsigned fu = i + (nx + 1) * (j + ny * k), fv = i + nx * (j + (ny + 1) * k);
    // the six face weights: low and high x, y, z (0 on solid sides)
    const double w0 = fx[fu], w1 = fx[fu + 1], w2 = fy[fv], w3 = fy[fv + nx], w4 = fz[c], w5 = fz[c + nxy];
    const double pc = p[c];
    // (A p)_c as differences (a neighbour beyond an open side is 0)
    double Ap = 0.0;
    Ap = fma(w0, i > 0 ? pc - p[c - 1] : pc, Ap);
    Ap = fma(w1, i + 1 < nx ? pc - p[c + 1] : pc, Ap);
    Ap = fma(w2, j > 0 ? pc - p[c - nx] : pc, Ap);
    Ap = fma(w3, j + 1 < ny ? pc - p[c + nx] : pc, Ap);
    Ap = fma(w4, k > 0 ? pc - p[c - nxy] : pc, Ap);
    Ap = fma(w5, k + 1 < nz ? pc - p[c + nxy] : pc, Ap);
    double b;
    if (which == 1) {
      // b1 = (rho h / dt) (sum over low faces - sum over high faces) of beta v*
      const double flux = (w0 * (double)u[fu] - w1 * (double)u[fu + 1]) + (w2 * (double)v[fv] - w3 * (double)v[fv + nx]) +
                          (w4 * (double)w[c] - w5 * (double)w[c + nxy]);
      b = S.vel * flux;
    } else {
      const double ac = target_fraction(alpha_s[c], S.amax);
      const double q = (double)alpha_star[c] / ac;
      const double ratio = q < S.rmin ? S.rmin : (q > S.rmax ? S.rmax : q);  // NaN stays NaN
      b = S.den * ac * (1.0 - ratio);
    }
    const double r = b - Ap;
    if (!isfinite(r)) raise_status(status, GIC_STATUS_NONFINITE);
    r32[c] = (float)r;
    e32[c] = 0.f;
    rr += r * r;
    bb += b * b;
  }
  block_sum2(rr, bb, smem);
  const double vals[2] = {rr, bb};
  double* const outs[2] = {&red->rr64, &red->bb};
  if (reduce_last<2>(vals, P, red, outs) && threadIdx.x == 0) {  // arm the CG run on this residual
    red->rr_stop = inner_tol2 * red->rr64;
    red->done = 0;
    red->iters = 0;
  }
}

// ---- multigrid preconditioner (FP32) ----
//
// A level is the operator (A x)_c = sum over c's faces of beta_f (x_c -
// x_nb) on an nx ny nz cell grid, with x_nb = 0 beyond the boundary: open
// sides carry their weight, solid sides weight 0, so every level is the same
// kind of operator.  Level 0 has the face weights of the projection; level
// l + 1 halves each axis (ceil), a coarse cell covering up to 2 x 2 x 2 fine
// cells, and its face weights are the sums of the fine face weights across
// each coarse face: the Galerkin product R A P with P the piecewise-constant
// interpolation and R = P^T.  The V-cycle smooths with red-black Gauss-Seidel
// (red then black before the coarse correction, black then red after it, so
// the preconditioner is symmetric), restricts the residual by summing the
// children, adds kMgOmega times the interpolated coarse correction (the
// constant interpolation under-corrects; 1.6 keeps the preconditioner
// positive definite and halves the CG iterations against 1.0), and runs the
// small levels, down to the coarsest (every axis <= 4 cells, solved by a
// palindromic sequence of Gauss-Seidel sweeps), in one CTA.
constexpr float kMgOmega = 1.6f;
constexpr int kMgCoarsePairs = 8;  // (black, red) sweep pairs after the first red sweep on the coarsest level
constexpr int kMgMaxLevels = 16;

struct MgLevel {
  int nx, ny, nz;
  float *bx, *by, *bz;  // face weights: (nx+1) ny nz, nx (ny+1) nz, nx ny (nz+1)
  float* invd;          // 1 / (sum of the cell's six face weights)
  float *x, *b;         // correction and right-hand side
};

__device__ __forceinline__ bool stopped(const ProjRed* red) { return *(volatile const int*)&red->done != 0; }

__device__ __forceinline__ void level_ijk(const MgLevel& L, unsigned c, unsigned& i, unsigned& j, unsigned& k) {
  const unsigned nx = (unsigned)L.nx, nxy = nx * (unsigned)L.ny;
  k = c / nxy;
  const unsigned r = c - k * nxy;
  j = r / nx;
  i = r - j * nx;
}

// sum over the cell's interior faces of beta_f x_nb, and the sum of all six
// face weights
__device__ __forceinline__ void level_gather(const MgLevel& L, unsigned c, unsigned i, unsigned j, unsigned k,
                                             const float* __restrict__ x, float& s, float& diag) {
  const unsigned nx = (unsigned)L.nx, ny = (unsigned)L.ny, nz = (unsigned)L.nz, nxy = nx * ny;
  const unsigned fx = i + (nx + 1) * (j + ny * k);
  const unsigned fy = i + nx * (j + (ny + 1) * k);
  const float wxl = L.bx[fx], wxh = L.bx[fx + 1];
  const float wyl = L.by[fy], wyh = L.by[fy + nx];
  const float wzl = L.bz[c], wzh = L.bz[c + nxy];
  diag = ((wxl + wxh) + (wyl + wyh)) + (wzl + wzh);
  float t = 0.f;
  if (i > 0) t = fmaf(wxl, x[c - 1], t);
  if (i + 1 < nx) t = fmaf(wxh, x[c + 1], t);
  if (j > 0) t = fmaf(wyl, x[c - nx], t);
  if (j + 1 < ny) t = fmaf(wyh, x[c + nx], t);
  if (k > 0) t = fmaf(wzl, x[c - nxy], t);
  if (k + 1 < nz) t = fmaf(wzh, x[c + nxy], t);
  s = t;
}

__device__ __forceinline__ float level_diag(const MgLevel& L, unsigned c, unsigned i, unsigned j, unsigned k) {
  const unsigned nx = (unsigned)L.nx, ny = (unsigned)L.ny, nxy = nx * ny;
  const unsigned fx = i + (nx + 1) * (j + ny * k);
  const unsigned fy = i + nx * (j + (ny + 1) * k);
  return ((L.bx[fx] + L.bx[fx + 1]) + (L.by[fy] + L.by[fy + nx])) + (L.bz[c] + L.bz[c + nxy]);
}

// Level-0 face weights from alpha_f' (float): the mean of the two cells, the
// inner cell's value on an open side, 0 on a solid side.
__global__ void __launch_bounds__(kProjThreads) k_mg_faces0(MgLevel L, unsigned open, const float* __restrict__ ap) {
  const unsigned nx = L.nx, ny = L.ny, nz = L.nz;
  const unsigned nu = (nx + 1) * ny * nz, nv = nx * (ny + 1) * nz, nw = nx * ny * (nz + 1);
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < nu + nv + nw; q += gridDim.x * blockDim.x) {
    unsigned a, f;
    if (q < nu) {
      a = 0, f = q;
    } else if (q < nu + nv) {
      a = 1, f = q - nu;
    } else {
      a = 2, f = q - nu - nv;
    }
    const unsigned sx = nx + (a == 0), sy = ny + (a == 1);
    const unsigned k = f / (sx * sy), rem = f - k * sx * sy, j = rem / sx, i = rem - j * sx;
    const unsigned pos = a == 0 ? i : (a == 1 ? j : k);
    const unsigned m = a == 0 ? nx : (a == 1 ? ny : nz);
    const unsigned stride = a == 0 ? 1u : (a == 1 ? nx : nx * ny);
    // the cell above the face (valid when pos < m) and the one below (pos > 0)
    const unsigned c_hi = i + nx * (j + ny * k), c_lo = c_hi - stride;
    float wgt;
    if (pos > 0 && pos < m)
      wgt = 0.5f * (ap[c_hi] + ap[c_lo]);
    else if (pos == 0)
      wgt = (open >> (2 * a)) & 1u ? ap[c_hi] : 0.f;
    else
      wgt = (open >> (2 * a + 1)) & 1u ? ap[c_lo] : 0.f;
    (a == 0 ? L.bx : (a == 1 ? L.by : L.bz))[f] = wgt;
  }
}

// Coarse face weights: the sum of the fine face weights across each coarse face.
__global__ void __launch_bounds__(kProjThreads) k_mg_coarsen(MgLevel F, MgLevel C) {
  const unsigned cx = C.nx, cy = C.ny, cz = C.nz;
  const unsigned nu = (cx + 1) * cy * cz, nv = cx * (cy + 1) * cz, nw = cx * cy * (cz + 1);
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < nu + nv + nw; q += gridDim.x * blockDim.x) {
    unsigned a, f;
    if (q < nu) {
      a = 0, f = q;
    } else if (q < nu + nv) {
      a = 1, f = q - nu;
    } else {
      a = 2, f = q - nu - nv;
    }
    const unsigned sx = cx + (a == 0), sy = cy + (a == 1);
    const unsigned K = f / (sx * sy), rem = f - K * sx * sy, J = rem / sx, I = rem - J * sx;
    const unsigned fnx = F.nx, fny = F.ny, fnz = F.nz;
    // the fine face position along axis a, and the 2 x 2 footprint on the other two axes
    unsigned lo[3] = {2 * I, 2 * J, 2 * K}, hi[3], lim[3] = {fnx, fny, fnz};
    for (int b = 0; b < 3; ++b) hi[b] = min(lo[b] + 2, lim[b]);
    lo[a] = min(lo[a], lim[a]);
    hi[a] = lo[a] + 1;
    const float* src = a == 0 ? F.bx : (a == 1 ? F.by : F.bz);
    const unsigned fsx = fnx + (a == 0), fsy = fny + (a == 1);
    float s = 0.f;
    for (unsigned k = lo[2]; k < hi[2]; ++k)
      for (unsigned j = lo[1]; j < hi[1]; ++j)
        for (unsigned i = lo[0]; i < hi[0]; ++i) s += src[i + fsx * (j + fsy * k)];
    (a == 0 ? C.bx : (a == 1 ? C.by : C.bz))[f] = s;
  }
}

__global__ void __launch_bounds__(kProjThreads) k_mg_diag(MgLevel L) {
  const unsigned n = (unsigned)L.nx * L.ny * L.nz;
  for (unsigned c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    unsigned i, j, k;
    level_ijk(L, c, i, j, k);
    const float diag = level_diag(L, c, i, j, k);
    L.invd[c] = diag > 0.f ? 1.f / diag : 0.f;
  }
}

// The V-cycle's passes over the cells t0, t0 + stride, ... of a level: the
// kernels below run them grid-wide, k_mg_tail within one CTA.

// One Gauss-Seidel half sweep: the cells with (i + j + k) % 2 == color get
// x_c = (b_c + sum beta_f x_nb) / diag_c.  init: x is taken as 0 (the other
// color is written 0).
__device__ __forceinline__ void mg_smooth_range(const MgLevel& L, unsigned color, int init, unsigned t0,
                                                unsigned stride) {
  const unsigned n = (unsigned)L.nx * L.ny * L.nz;
  for (unsigned c = t0; c < n; c += stride) {
    unsigned i, j, k;
    level_ijk(L, c, i, j, k);
    if (((i + j + k) & 1u) != color) {
      if (init) L.x[c] = 0.f;
      continue;
    }
    float s = 0.f, diag;
    if (!init) level_gather(L, c, i, j, k, L.x, s, diag);
    L.x[c] = L.invd[c] * (L.b[c] + s);
  }
}

// Coarse right-hand side: the sum of the children's residuals b - A x.
__device__ __forceinline__ void mg_restrict_range(const MgLevel& F, const MgLevel& C, unsigned t0, unsigned stride) {
  const unsigned n = (unsigned)C.nx * C.ny * C.nz;
  const unsigned fnx = F.nx, fny = F.ny, fnz = F.nz;
  for (unsigned q = t0; q < n; q += stride) {
    unsigned I, J, K;
    level_ijk(C, q, I, J, K);
    float acc = 0.f;
    for (unsigned k = 2 * K; k < min(2 * K + 2, fnz); ++k)
      for (unsigned j = 2 * J; j < min(2 * J + 2, fny); ++j)
        for (unsigned i = 2 * I; i < min(2 * I + 2, fnx); ++i) {
          const unsigned c = i + fnx * (j + fny * k);
          float s, diag;
          level_gather(F, c, i, j, k, F.x, s, diag);
          acc += F.b[c] - (diag * F.x[c] - s);
        }
    C.b[q] = acc;
  }
}

// x_fine += kMgOmega x_coarse(parent)
__device__ __forceinline__ void mg_prolong_range(const MgLevel& C, const MgLevel& F, unsigned t0, unsigned stride) {
  const unsigned n = (unsigned)F.nx * F.ny * F.nz;
  for (unsigned c = t0; c < n; c += stride) {
    unsigned i, j, k;
    level_ijk(F, c, i, j, k);
    F.x[c] = fmaf(kMgOmega, C.x[(i >> 1) + (unsigned)C.nx * ((j >> 1) + (unsigned)C.ny * (k >> 1))], F.x[c]);
  }
}

__global__ void __launch_bounds__(kProjThreads) k_mg_smooth(MgLevel L, unsigned color, int init,
                                                            const ProjRed* red) {
  if (stopped(red)) return;
  mg_smooth_range(L, color, init, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

__global__ void __launch_bounds__(kProjThreads) k_mg_restrict(MgLevel F, MgLevel C, const ProjRed* red) {
  if (stopped(red)) return;
  mg_restrict_range(F, C, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

__global__ void __launch_bounds__(kProjThreads) k_mg_prolong(MgLevel C, MgLevel F, const ProjRed* red) {
  if (stopped(red)) return;
  mg_prolong_range(C, F, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// The levels from `first` (at most kMgTailCells cells) down to the coarsest
// in one CTA, with a barrier between passes (their launches would cost more
// than their work): the same passes as the grid-wide V-cycle, and on the
// coarsest level (every axis <= 4 cells) red from x = 0, then kMgCoarsePairs
// (black, red) sweep pairs.  Same-color cells do not touch, so a half sweep
// reads only values no thread of the pass writes.
constexpr int kMgTailThreads = 1024;
constexpr int kMgTailCells = 4096;
struct MgLevels {
  MgLevel l[kMgMaxLevels];
};

__global__ void __launch_bounds__(kMgTailThreads) k_mg_tail(MgLevels Ls, int first, int top, const ProjRed* red) {
  if (stopped(red)) return;
  const unsigned t0 = threadIdx.x, st = blockDim.x;
  for (int l = first; l < top; ++l) {
    mg_smooth_range(Ls.l[l], 0u, 1, t0, st);
    __syncthreads();
    mg_smooth_range(Ls.l[l], 1u, 0, t0, st);
    __syncthreads();
    mg_restrict_range(Ls.l[l], Ls.l[l + 1], t0, st);
    __syncthreads();
  }
  mg_smooth_range(Ls.l[top], 0u, 1, t0, st);
  __syncthreads();
  for (int p = 0; p < kMgCoarsePairs; ++p) {
    mg_smooth_range(Ls.l[top], 1u, 0, t0, st);
    __syncthreads();
    mg_smooth_range(Ls.l[top], 0u, 0, t0, st);
    __syncthreads();
  }
  for (int l = top - 1; l >= first; --l) {
    mg_prolong_range(Ls.l[l + 1], Ls.l[l], t0, st);
    __syncthreads();
    mg_smooth_range(Ls.l[l], 1u, 0, t0, st);
    __syncthreads();
    mg_smooth_range(Ls.l[l], 0u, 0, t0, st);
    __syncthreads();
  }
}

// ---- conjugate gradients on A e = r with the multigrid preconditioner ----

// rho = r . z (z = M^-1 r from the V-cycle) into red->rz[cur].
__global__ void __launch_bounds__(kProjThreads) k_cg_dot(int64_t n64, int cur, const float* __restrict__ r,
                                                         const float* __restrict__ z, double* __restrict__ P,
                                                         ProjRed* red) {
  __shared__ double smem[32];
  if (stopped(red)) return;
  const unsigned n = (unsigned)n64;
  KahanF k;
  for (unsigned c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) k.add(r[c] * z[c]);
  const double rz = block_sum((double)k.s, smem);
  const double vals[1] = {rz};
  double* const outs[1] = {&red->rz[cur]};
  reduce_last<1>(vals, P, red, outs);
}

// d_new = z + beta d_old (beta = rho / rho_prev; 0 on a run's first
// iteration), y = A d_new and d_new . y into red->dy.  d_old and d_new are
// different buffers: neighbours' d_new is formed from their z and d_old.
__global__ void __launch_bounds__(kProjThreads) k_cg_dir_apply(MgLevel L, int cur, const float* __restrict__ z,
                                                               const float* __restrict__ d_old,
                                                               float* __restrict__ d_new, float* __restrict__ y,
                                                               double* __restrict__ P, ProjRed* red) {
  __shared__ double smem[32];
  if (stopped(red)) return;
  // beta in FP32 (a double divide per thread would occupy GB300's slow FP64 pipe)
  const float be = red->iters == 0 ? 0.f : (float)red->rz[cur] / (float)red->rz[cur ^ 1];
  const unsigned nx = L.nx, ny = L.ny, nz = L.nz, nxy = nx * ny, n = nxy * nz;
  KahanF dyk;
  for (unsigned c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    unsigned i, j, k;
    level_ijk(L, c, i, j, k);
    // beta = 0 takes z alone (the old direction is not read into the sum)
    auto dn = [&](unsigned q) { return be != 0.f ? fmaf(be, d_old[q], z[q]) : z[q]; };
    const float dc = dn(c);
    const unsigned fx = i + (nx + 1) * (j + ny * k);
    const unsigned fy = i + nx * (j + (ny + 1) * k);
    const float wxl = L.bx[fx], wxh = L.bx[fx + 1], wyl = L.by[fy], wyh = L.by[fy + nx], wzl = L.bz[c],
                wzh = L.bz[c + nxy];
    float acc = (((wxl + wxh) + (wyl + wyh)) + (wzl + wzh)) * dc;
    if (i > 0) acc = fmaf(-wxl, dn(c - 1), acc);
    if (i + 1 < nx) acc = fmaf(-wxh, dn(c + 1), acc);
    if (j > 0) acc = fmaf(-wyl, dn(c - nx), acc);
    if (j + 1 < ny) acc = fmaf(-wyh, dn(c + nx), acc);
    if (k > 0) acc = fmaf(-wzl, dn(c - nxy), acc);
    if (k + 1 < nz) acc = fmaf(-wzh, dn(c + nxy), acc);
    d_new[c] = dc;
    y[c] = acc;
    dyk.add(dc * acc);
  }
  const double dy = block_sum((double)dyk.s, smem);
  const double vals[1] = {dy};
  double* const outs[1] = {&red->dy};
  reduce_last<1>(vals, P, red, outs);
}

// alpha = rho / (d . y); e += alpha d; r -= alpha y (float4); r . r into
// red->rr.  The last block counts the iteration and sets the stop flag when
// r . r <= rr_stop (or on a breakdown).
__global__ void __launch_bounds__(kProjThreads) k_cg_update(int64_t n64, int cur, const float* __restrict__ d,
                                                            const float* __restrict__ y, float* __restrict__ e,
                                                            float* __restrict__ r, double* __restrict__ P,
                                                            ProjRed* red) {
  __shared__ double smem[32];
  if (stopped(red)) return;
  const double dy = red->dy, rz = red->rz[cur];  // the same values in every block
  if (!(dy > 0.0) || !isfinite(rz)) {  // d = 0 (r = 0: converged) or breakdown: stop this run
    if (blockIdx.x == 0 && threadIdx.x == 0) red->done = 1;
    return;
  }
  const float al = (float)rz / (float)dy;  // FP32, as beta
  KahanF rrk;
  const unsigned n = (unsigned)n64, n4 = n / 4u;
  const unsigned t0 = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  for (unsigned q = t0; q < n4; q += stride) {  // arrays are 256-byte aligned
    const float4 dq = reinterpret_cast<const float4*>(d)[q];
    const float4 yq = reinterpret_cast<const float4*>(y)[q];
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
    rrk.add(rq.x * rq.x + rq.y * rq.y + rq.z * rq.z + rq.w * rq.w);
  }
  for (unsigned c = 4u * n4 + t0; c < n; c += stride) {
    e[c] = fmaf(al, d[c], e[c]);
    const float rc = fmaf(-al, y[c], r[c]);
    r[c] = rc;
    rrk.add(rc * rc);
  }
  const double rr = block_sum((double)rrk.s, smem);
  const double vals[1] = {rr};
  double* const outs[1] = {&red->rr};
  if (reduce_last<1>(vals, P, red, outs) && threadIdx.x == 0) {
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
  double *fx, *fy, *fz;                // FP64 face weights (the residual's operator)
  float *ap32, *r, *z, *d[2], *y, *e;  // d: the CG direction, double-buffered
  double* P;                           // 2 * nblk partial sums
  ProjRed* red;
  MgLevel lev[kMgMaxLevels];
  int levels;
};

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

static int proj_blocks(int64_t n) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (n + kProjThreads - 1) / kProjThreads;
  const int64_t cap = 8 * (int64_t)(sms > 0 ? sms : 152);
  return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

// Workspace of the call (laid out by the same walk that measures it): the
// FP32 CG vectors, the partial sums, the scalars and the multigrid levels
// (halving each axis until every axis has at most 4 cells).
static size_t proj_layout(const PGrid& g, int nblk, char* base, ProjWs* W) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += align256(bytes);
    return p;
  };
  const size_t n = (size_t)g.n;
  ProjWs w;
  w.fx = (double*)take(8 * (size_t)(g.nx + 1) * g.ny * g.nz);
  w.fy = (double*)take(8 * (size_t)g.nx * (g.ny + 1) * g.nz);
  w.fz = (double*)take(8 * (size_t)g.nx * g.ny * (g.nz + 1));
  w.ap32 = (float*)take(4 * n);
  w.r = (float*)take(4 * n);
  w.z = (float*)take(4 * n);
  w.d[0] = (float*)take(4 * n);
  w.d[1] = (float*)take(4 * n);
  w.y = (float*)take(4 * n);
  w.e = (float*)take(4 * n);
  w.P = (double*)take(2 * 8 * (size_t)nblk);
  w.red = (ProjRed*)take(sizeof(ProjRed));
  int nx = g.nx, ny = g.ny, nz = g.nz;
  w.levels = 0;
  for (;;) {
    MgLevel& L = w.lev[w.levels];
    L.nx = nx, L.ny = ny, L.nz = nz;
    const size_t nl = (size_t)nx * ny * nz;
    L.bx = (float*)take(4 * (size_t)(nx + 1) * ny * nz);
    L.by = (float*)take(4 * (size_t)nx * (ny + 1) * nz);
    L.bz = (float*)take(4 * (size_t)nx * ny * (nz + 1));
    L.invd = (float*)take(4 * nl);
    if (w.levels == 0) {
      L.x = w.z;
      L.b = w.r;
    } else {
      L.x = (float*)take(4 * nl);
      L.b = (float*)take(4 * nl);
    }
    ++w.levels;
    if ((nx <= 4 && ny <= 4 && nz <= 4) || w.levels == kMgMaxLevels) break;
    nx = (nx + 1) / 2, ny = (ny + 1) / 2, nz = (nz + 1) / 2;
  }
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
  if (g->n >= ((int64_t)1 << 30)) return set_error(GIC_ERR_INVALID, "gic_project: 2^30 cells or more");
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
  GIC_RANGE("gic_project_workspace_size");
  PGrid g;
  int rc = proj_grid(grid, &g);
  if (rc) return rc;
  if (!bytes) return set_error(GIC_ERR_INVALID, "gic_project_workspace_size: bytes is NULL");
  *bytes = proj_layout(g, proj_blocks(g.n), nullptr, nullptr);
  return GIC_OK;
}

extern "C" int gic_project(const GicGrid* grid, const GicProjParams* P, const double* alpha_s, const float* alpha_star,
                           const float* u, const float* v, const float* w, double* p1, double* p2, float* u_out,
                           float* v_out, float* w_out, float* dx_u, float* dx_v, float* dx_w, void* ws,
                           size_t ws_bytes, GicProjInfo* info, gic_stream_t stream_) {
  GIC_RANGE("gic_project");
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
  const size_t need = proj_layout(g, nblk, nullptr, nullptr);
  if (!ws || ws_bytes < need)
    return set_error(GIC_ERR_WORKSPACE, "gic_project: workspace of %zu bytes needed, %zu given", need, ws_bytes);
  if ((uintptr_t)ws % 256) return set_error(GIC_ERR_ALIGN, "gic_project: workspace must be 256-byte aligned");
  cudaStream_t st = (cudaStream_t)stream_;
  ProjWs W;
  proj_layout(g, nblk, (char*)ws, &W);
  if (W.levels == kMgMaxLevels && !(W.lev[kMgMaxLevels - 1].nx <= 4 && W.lev[kMgMaxLevels - 1].ny <= 4 &&
                                    W.lev[kMgMaxLevels - 1].nz <= 4))
    return set_error(GIC_ERR_INVALID, "gic_project: grid too large for the multigrid hierarchy");
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
  auto lblocks = [&](const MgLevel& L) { return proj_blocks((int64_t)L.nx * L.ny * L.nz); };
  auto fblocks = [&](const MgLevel& L) {
    return proj_blocks((int64_t)(L.nx + 1) * L.ny * L.nz + (int64_t)L.nx * (L.ny + 1) * L.nz +
                       (int64_t)L.nx * L.ny * (L.nz + 1));
  };

  if (cudaMemsetAsync(W.red, 0, sizeof(ProjRed), st) != cudaSuccess ||
      cudaMemsetAsync(W.d[0], 0, sizeof(float) * g.n, st) != cudaSuccess ||
      cudaMemsetAsync(W.d[1], 0, sizeof(float) * g.n, st) != cudaSuccess)
    return set_error(GIC_ERR_CUDA, "gic_project: clearing the workspace failed");
  // the operator's face weights on every level
  k_proj_faces64<<<fblocks(W.lev[0]), kProjThreads, 0, st>>>(g, open_bits, alpha_s, P->alpha_s_max, W.fx, W.fy, W.fz);
  k_proj_prep<<<nblk, kProjThreads, 0, st>>>(g, alpha_s, P->alpha_s_max, W.ap32);
  k_mg_faces0<<<fblocks(W.lev[0]), kProjThreads, 0, st>>>(W.lev[0], open_bits, W.ap32);
  k_mg_diag<<<lblocks(W.lev[0]), kProjThreads, 0, st>>>(W.lev[0]);
  launches += 4;
  for (int l = 1; l < W.levels; ++l) {
    k_mg_coarsen<<<fblocks(W.lev[l]), kProjThreads, 0, st>>>(W.lev[l - 1], W.lev[l]);
    k_mg_diag<<<lblocks(W.lev[l]), kProjThreads, 0, st>>>(W.lev[l]);
    launches += 2;
  }
  // the levels from `first` on run in one CTA (k_mg_tail)
  MgLevels levels;
  for (int l = 0; l < W.levels; ++l) levels.l[l] = W.lev[l];
  int first = 0;
  while (first < W.levels - 1 && (int64_t)W.lev[first].nx * W.lev[first].ny * W.lev[first].nz > kMgTailCells) ++first;
  // one preconditioned CG iteration: z = V-cycle(r), rho = r . z, the new
  // direction with y = A d, the updates; all arguments but the parity are
  // fixed for the call
  int per_iter = 0;
  auto cg_iteration = [&](int cur, cudaStream_t s_) {
    const int top = W.levels - 1;
    for (int l = 0; l < first; ++l) {
      k_mg_smooth<<<lblocks(W.lev[l]), kProjThreads, 0, s_>>>(W.lev[l], 0u, 1, W.red);
      k_mg_smooth<<<lblocks(W.lev[l]), kProjThreads, 0, s_>>>(W.lev[l], 1u, 0, W.red);
      k_mg_restrict<<<lblocks(W.lev[l + 1]), kProjThreads, 0, s_>>>(W.lev[l], W.lev[l + 1], W.red);
    }
    k_mg_tail<<<1, kMgTailThreads, 0, s_>>>(levels, first, top, W.red);
    for (int l = first - 1; l >= 0; --l) {
      k_mg_prolong<<<lblocks(W.lev[l]), kProjThreads, 0, s_>>>(W.lev[l + 1], W.lev[l], W.red);
      k_mg_smooth<<<lblocks(W.lev[l]), kProjThreads, 0, s_>>>(W.lev[l], 1u, 0, W.red);
      k_mg_smooth<<<lblocks(W.lev[l]), kProjThreads, 0, s_>>>(W.lev[l], 0u, 0, W.red);
    }
    k_cg_dot<<<nblk, kProjThreads, 0, s_>>>(g.n, cur, W.r, W.z, W.P, W.red);
    k_cg_dir_apply<<<nblk, kProjThreads, 0, s_>>>(W.lev[0], cur, W.z, W.d[cur ^ 1], W.d[cur], W.y, W.P, W.red);
    k_cg_update<<<nblk, kProjThreads, 0, s_>>>(g.n, cur, W.d[cur], W.y, W.e, W.r, W.P, W.red);
    per_iter = 6 * first + 4;
  };
  // kChunk iterations as one CUDA graph (kChunk even: the parities repeat),
  // built when the first CG run needs it
  constexpr int kChunk = 4;
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

  for (int which = 1; which <= 2 && rc2 == GIC_OK; ++which) {
    double* p = which == 1 ? p1 : p2;
    const int sys = which - 1;
    if (cudaMemsetAsync(p, 0, sizeof(double) * g.n, st) != cudaSuccess) {
      rc2 = set_error(GIC_ERR_CUDA, "gic_project: clearing p failed");
      break;
    }
    for (int outer = 0;; ++outer) {
      k_proj_residual<<<nblk, kProjThreads, 0, st>>>(g, which, S, alpha_s, alpha_star, u, v, w, W.fx, W.fy, W.fz, p,
                                                     W.r, W.e, P->inner_tol * P->inner_tol, W.P, W.red, status);
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
      // the FP32 preconditioned CG on A e = r to a reduction of inner_tol (of
      // the FP32 copy's r . r): graph launches of kChunk iterations, the stop
      // flag read after each
      int it = 0;
      for (;;) {
        if (P->max_inner - it >= kChunk) {
          if (!chunk && (rc2 = build_chunk())) break;
          if (cudaGraphLaunch(chunk, st) != cudaSuccess) {
            rc2 = set_error(GIC_ERR_CUDA, "gic_project: graph launch failed");
            break;
          }
          it += kChunk;
          launches += (int64_t)per_iter * kChunk;
        } else {
          for (; it < P->max_inner; ++it) {
            cg_iteration(it & 1, st);
            launches += per_iter;
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
