/*
 * gic.h -- C ABI of the GB300 (sm_103a) granule-grid coupling library.
 *
 * The library implements, as CUDA kernels, the per-substep granule-grid
 * coupling of the Granule-In-Cell (GIC) method (Tang, Zhu, Ni, Chen, "The
 * Granule-In-Cell Method for Simulating Sand-Water Mixtures", ACM TOG 44(6),
 * 2025): Algorithm 2 (SandSubstep), with the capillary form of the
 * concentration-gradient force (Sec. 5.4) in the fused entry points, plus a
 * Morton cell sort for the contact neighbour search and a hand-written
 * adjoint of every step.
 *
 * One substep is
 *   gic_sort        contact-cell Morton sort + cell table   (neighbour search for Sec. 3.1)
 *   gic_contact     DEM contact forces                       (Sec. 3.1, contact law Eq. k_n)
 *   gic_g2p_couple  drag, buoyancy, fluid acceleration       (Sec. 3.3 Eqs. 5a-5c, Sec. 5.2)
 *   gic_integrate   virtual-mass symplectic Euler            (Sec. 5.2 Eq. sand kine; Alg. 2 MoveParticle)
 *   gic_p2g         alpha_s and exchange momentum to the MAC grid (Sec. 5.1 alpha_s; Sec. 5.2 Exchange Momentum)
 * and, once per fluid step, gic_project consumes alpha_s: the velocity and
 * density projections of Sec. 5.1 (Eqs. ppe1 a/b).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Memory.  Every array argument is a DEVICE pointer owned by the caller
 * (except the *_host entry points, which say so).  The library allocates no
 * device memory: scratch space comes from a caller-provided workspace whose
 * size gic_workspace_size reports.
 * Streams.  Every call enqueues work on `stream` (a cudaStream_t; NULL is the
 * legacy default stream) and returns without synchronising, except where
 * stated.
 * Errors.  Return GIC_OK (0) or a negative GIC_ERR_* code for argument errors
 * detected on the host (null pointer, bad size, misalignment, workspace too
 * small) and for CUDA launch errors; gic_last_error() describes the last one.
 * Conditions met inside a kernel (granule left the domain, coincident centres,
 * non-finite value, radius too large for the contact grid) set bits of a sticky device status word
 * read by gic_check_status().  No kernel traps, asserts or spins.
 *
 * Granule state (GicGranules), structure of arrays, n granules:
 *   cell  int32[n]   contact-cell coordinates packed as cx | cy << 10 | cz << 20
 *                    (at most 1024 contact cells per axis)
 *   pos   GIC_FP32: uint32[4 n] = {qx, qy, qz, bits of float r}: the offset in
 *                    the contact cell as a 30-bit fixed-point fraction,
 *                    x = origin + (c + q / 2^30) h_c, 16-byte aligned;
 *         GIC_FP64: double[4 n] = {ox, oy, oz, r}, offset in metres in
 *                    [0, h_c), 32-byte aligned
 *   vel   float[4 n] / double[4 n] = {vx, vy, vz, 0}
 *   id    int32[n] or NULL: original granule id, carried along by gic_sort
 *   posf  float[4 n] or NULL (FP32 path only): the positions again as float,
 *         in contact-cell units {cx + qx/2^30, cy + qy/2^30, cz + qz/2^30, r}.
 *         Derived data: gic_sort writes it (into out->posf), gic_step and
 *         gic_substep into the next state, and the contact calls read it for
 *         their float pre-test (with a tolerance of 2^-11 cell; the exact
 *         integer geometry decides); leave it NULL anywhere else.  16-byte
 *         aligned.
 * Per-granule vectors (forces, accelerations, gradients) are real[4 n] with
 * the 4th lane unused (real = float for GIC_FP32, double for GIC_FP64).
 * Grid fields are real arrays on the MAC grid, x fastest:
 *   u (nx+1) ny nz on x-faces, v nx (ny+1) nz, w nx ny (nz+1), p and alpha_f at
 *   cell centres nx ny nz.  alpha_s is ALWAYS double (FP64 accumulation).
 * The contact grid subdivides each MAC cell into k_contact^3 cells of side
 * h_c = dx / k_contact, which must be at least 2 r_max.
 */
#ifndef GIC_H_
#define GIC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* gic_stream_t; /* == cudaStream_t */

enum { GIC_FP32 = 0, GIC_FP64 = 1 };

enum {
  GIC_OK = 0,
  GIC_ERR_INVALID = -1,   /* bad argument (null pointer, size, grid) */
  GIC_ERR_CUDA = -2,      /* a CUDA call failed */
  GIC_ERR_WORKSPACE = -3, /* workspace missing or too small */
  GIC_ERR_ALIGN = -4,     /* pointer not aligned as documented */
  GIC_ERR_TIMEOUT = -5    /* host wait exceeded its deadline */
};

/* sticky device status bits */
enum {
  GIC_STATUS_OUT_OF_DOMAIN = 1u, /* a granule left the box; it was clamped to the boundary */
  GIC_STATUS_COINCIDENT = 2u,    /* a pair at distance 0 was skipped */
  GIC_STATUS_NONFINITE = 4u,     /* a non-finite velocity or force appeared */
  GIC_STATUS_RADIUS = 8u,        /* a radius exceeds h_c / 2: contacts beyond the 27 cells are missed */
  GIC_STATUS_BAD_CELL = 16u,     /* an input cell id lay outside the contact grid */
  GIC_STATUS_FAST = 32u,         /* a granule moved more than one contact cell in a substep */
  GIC_STATUS_DEBUG_INDEX = 64u   /* a library built with GIC_DEBUG found an index out of its array; the access
                                    was skipped (release builds never set it) */
};

typedef struct GicGrid {
  int32_t nx, ny, nz; /* MAC cells per axis, each >= 2 */
  int32_t k_contact;  /* contact cells per MAC cell and axis, >= 1 */
  double dx;          /* MAC cell size */
  double origin[3];   /* lower corner of the box [origin, origin + n dx] */
} GicGrid;

typedef struct GicParams {
  double rho_s, rho_f;   /* granule and fluid density */
  double k_n;            /* normal stiffness (Sec. 3.1) */
  double zeta;           /* normal damping ratio: c_n = 2 zeta sqrt(k_n m_eff) */
  double kt_over_cn;     /* tangential coefficient k_t = kt_over_cn * c_n */
  double mu_fric;        /* Coulomb coefficient tan(phi) (Sec. 3.1) */
  double c_drag;         /* F_d = c_drag pi r^2 rho_f |dv| dv (Sec. 3.3 Eq. 5b) */
  double g[3];           /* gravity */
  double dt_sub;         /* sand substep dt' */
  double dt_fluid;       /* fluid step dt; the exchange force is scaled by dt'/dt */
  int32_t virtual_mass;  /* 1: added mass (2/3) pi r^3 rho_f (Sec. 5.2 Eq. sand kine) */
  int32_t walls;         /* 1: the six box planes are contact partners */
  /* Concentration-gradient force in its capillary form (Sec. 5.4), between
   * granules 0 < s < d_r apart: F_ij = -Gamma((sr_i + sr_j) / 2) F^st(s)
   * (x_i - x_j) / |x_i - x_j|, sr_i = moisture + alpha_f,i / (1 - alpha_f,i)
   * with alpha_f,i the fluid fraction interpolated at the granule.
   * sigma = 0 leaves it out.  Only the fused entry points (gic_step,
   * gic_substep, gic_substep_adj) evaluate it; the separate contact entry
   * points return GIC_ERR_INVALID when sigma > 0. */
  double sigma;          /* surface tension coefficient (>= 0) */
  double bridge_frac;    /* liquid-bridge volume V* as a fraction of the mean volume of the pair (> 0) */
  double moisture;       /* water ratio r_i held by every granule (>= 0) */
  double moisture_peak;  /* moisture ratio where Gamma peaks (the maximum absorption ratio), in [1/4, 3/4] */
} GicParams;

typedef struct GicGranules {
  int64_t n;
  int32_t* cell;
  void* pos;
  void* vel;
  int32_t* id;
  int32_t precision; /* GIC_FP32 or GIC_FP64 */
  float* posf;       /* optional, GIC_FP32 only: float[4 n] {fx, fy, fz, r}, fx = cx + qx / 2^30 (see above) */
} GicGranules;

/* ------------------------------------------------------------------ sizes */

/* Bytes of workspace gic_sort (and gic_window_forward) need for n granules. */
int gic_workspace_size(const GicGrid* grid, int64_t n, int32_t precision, size_t* bytes);

/* Bytes of the cell table: 16 * (1 + number of contact cells).  The caller
 * zero-fills it once; gic_sort tags every entry it writes with an epoch kept
 * in the table's first entry, so the table is never cleared again (after
 * 2^32 - 1 sorts the caller must zero it once more). */
int gic_cell_table_size(const GicGrid* grid, size_t* bytes);

/* ------------------------------------------------------------ conversion */

/* Build a state from the canonical encoding: cell_xyz int32[3n], q uint32[3n]
 * (30-bit fractions), r float[n], v float[3n] (device pointers).  Writes
 * out->cell, out->pos, out->vel and, if out->id != NULL, id = 0..n-1. */
int gic_pack(const GicGrid* grid, int64_t n, const int32_t* cell_xyz, const uint32_t* q, const float* r,
             const float* v, GicGranules* out, gic_stream_t stream);

/* Absolute FP64 positions and velocities (double[3n] each).  With in->id set,
 * granule k is written to slot id[k] (original order); else to slot k. */
int gic_unpack(const GicGrid* grid, const GicGranules* in, double* x, double* v, gic_stream_t stream);

/* Adjoint of gic_unpack: gradients w.r.t. the absolute positions/velocities
 * (double[3n], original order when in->id is set) gathered into the state's
 * order as real[4n] position / velocity gradients (written, not added). */
int gic_unpack_adj(const GicGrid* grid, const GicGranules* in, const double* gx, const double* gv, void* g_pos,
                   void* g_vel, gic_stream_t stream);

/* ------------------------------------------------------------ forward */

/* a1: stable Morton sort of the granules by contact cell (ties keep input
 * order), permutation of the state into out, and the cell table.
 *   perm[k] = input index of the k-th sorted granule (int32[n]).
 *   cell_table: see gic_cell_table_size.  in and out must not alias.
 * The neighbour search itself is not described by the paper; Sec. 3.1 only
 * states that granules interact when closer than 2 r. */
int gic_sort(const GicGrid* grid, const GicGranules* in, GicGranules* out, int32_t* perm, void* cell_table, void* ws,
             size_t ws_bytes, gic_stream_t stream);

/* gic_sort without a workspace argument, for callers that cannot allocate
 * device memory (for example code that runs inside a host callback or a
 * real-time loop where cudaMalloc must not be called, or a host that can only
 * pass buffers registered in advance).  The paper has no counterpart: this is
 * an interface convenience of the library.
 *   Same arguments, results and errors as gic_sort, minus ws / ws_bytes.  The
 *   radix-sort scratch is a static array of about 4.3 MB compiled into the
 *   library: it holds at most gic_sort_static_max_n() granules (262,144);
 *   larger n returns GIC_ERR_INVALID without launching anything.
 *   The array exists once per device that loads the library, until exit.
 *   Every call looks up the array's device address on the current device
 *   (no allocation; a cudaDeviceReset in between is harmless); the first
 *   call on a device also loads the library's kernels there, so make that
 *   first call before any stream capture.  Every call on a device uses the same
 *   array: calls that can run at the same time on the GPU (different streams
 *   without ordering) race and must be serialised by the caller.  The array
 *   keeps the last call's contents; nothing in it has to start at zero.
 *   Allocates nothing (no cudaMalloc, no allocating library routine). */
int gic_sort_static(const GicGrid* grid, const GicGranules* in, GicGranules* out, int32_t* perm, void* cell_table,
                    gic_stream_t stream);

/* Largest n gic_sort_static accepts. */
int64_t gic_sort_static_max_n(void);

/* a2: contact force on every granule of a SORTED state (the output of
 * gic_sort with the same cell table): linear spring k_n (r_i + r_j - d) plus
 * dashpot -c_n v_n along the normal, tangential -k_t v_t capped at
 * mu |F_n| (Sec. 3.1, Eq. k_n, polydisperse form), and the six walls when
 * params->walls.  F_c real[4n], written. */
int gic_contact(const GicGrid* grid, const GicParams* params, const GicGranules* sorted, const void* cell_table,
                void* F_c, gic_stream_t stream);

/* a2 with Verlet neighbour lists: the same forces as gic_contact (identical
 * contact pairs, the pair sums in another order), found through a list of
 * the partners each granule had within r_i + r_j + skin when the list was
 * built.  The paper walks the cell list every substep (Sec. 3.1); a list stays
 * exact while no granule has moved more than skin / 2 since it was built,
 * because a pair can then have closed by at most skin.
 *   A build numbers the granules by their sorted index at that moment (their
 *   slot) and stores each slot's partners as slots, so list rows and the
 *   reference positions are read in nearly sorted order between builds;
 *   granule ids map to slots.  Each call first maps the current sorted
 *   indices to slots and checks every displacement from the last build; if
 *   one exceeds skin / 2, or a rebuild was requested, this call walks the 27
 *   cells as gic_contact does and rebuilds every list while it sums the
 *   forces; otherwise it walks the lists only.  sorted must carry ids
 *   (0..n-1, each once).  Three launches, no host sync.
 *   A list that would exceed cap entries makes every later call rebuild
 *   (forces stay exact, the saving is lost) until gic_neighbors_reset with a
 *   larger cap; flags[1] bit 1 reports it.
 * Ownership: all arrays are device memory owned by the caller, sized for
 * n granules; gic_neighbors_reset must run once before the first use (and
 * whenever the granule set or radii change).  Errors: GIC_ERR_INVALID for a
 * null array, n mismatch, cap < 1 or a negative skin; GIC_ERR_ALIGN when
 * ref_pos is not 16-byte (FP32) / 32-byte (FP64) aligned. */
typedef struct GicNeighbors {
  int64_t n;         /* granules; ids run 0..n-1 */
  int32_t cap;       /* list slots per granule */
  double skin;       /* metres, >= 0 */
  int32_t* list;     /* [n * cap] partner slots of each slot (row = slot) */
  int32_t* count;    /* [n] entries used in each row */
  int32_t* ref_cell; /* [n] contact cell of each slot at the last build */
  void* ref_pos;     /* [n] position record (uint4 FP32, double4 FP64) of each slot at the last build */
  int32_t* slot;     /* [n] slot of each granule id (written by a build) */
  int32_t* cur;      /* [n] current sorted index of each slot (written by every call) */
  int32_t* at;       /* [n] slot of each current sorted index (written by every call) */
  uint32_t* flags;   /* [8]: [0] rebuild in this call, [1] bit 0 rebuild requested, bit 1 a list overflowed at the
                      * last build, [2] CTA counter, [3] overflow during a build, [4] builds performed, [5] a
                      * granule written by the last substep kernel is beyond skin / 2 (read by gic_step) */
} GicNeighbors;

int gic_contact_verlet(const GicGrid* grid, const GicParams* params, const GicGranules* sorted,
                       const void* cell_table, const GicNeighbors* nb, void* F_c, gic_stream_t stream);

/* gic_contact_adj through the Verlet lists nb: the same gradients (the pair
 * sums in another order).  The lists are checked, and rebuilt when needed,
 * exactly as by gic_contact_verlet (the build's forces go to the scratch
 * F_c, real[4n]).  Accumulates into g_pos, g_vel and *g_mu. */
int gic_contact_verlet_adj(const GicGrid* grid, const GicParams* params, const GicGranules* sorted,
                           const void* cell_table, const GicNeighbors* nb, void* F_c, const void* gF_c, void* g_pos,
                           void* g_vel, double* g_mu, gic_stream_t stream);

/* One substep after the sort, fused (Alg. 2 body): contact through the
 * Verlet lists nb (exactly gic_contact_verlet's forces; on a substep that
 * rebuilds the lists the 27-cell walk that builds them gives the forces),
 * the G2P coupling (gic_g2p_couple), the integration (gic_integrate) from
 * `sorted` into `next`, and the P2G scatter (gic_p2g with old = sorted,
 * new = next), in one pass that keeps the per-granule forces in registers.
 * The paper runs these as the steps of one substep (Alg. 2); fusing them is
 * this library's.
 *   sorted: the output of gic_sort (ids required); next: written (cell, pos,
 *   vel, id).  f_ex: real[4n] or NULL, written.  alpha_s (or NULL), F_s (all
 *   three or none) and sums2 as for gic_p2g: alpha_s and sums2 are written,
 *   F_s accumulates.  Fluid fields as for gic_g2p_couple.  Errors as for the
 *   calls it fuses (sorted and next must match in size and precision).  Two
 *   to four launches, no host sync. */
int gic_substep(const GicGrid* grid, const GicParams* params, const GicGranules* sorted, const void* cell_table,
                const GicNeighbors* nb, const void* u, const void* v, const void* w, const void* p,
                const void* alpha_f, GicGranules* next, void* f_ex, double* alpha_s, void* Fs_u, void* Fs_v,
                void* Fs_w, double* sums2, gic_stream_t stream);

/* One whole substep (Alg. 2 body with the sort in front) on a state kept
 * with Verlet lists, from `state` into `next` (state is not written).
 * When the lists are rebuilt in this call, `state` is first sorted into
 * `sorted` (perm, cell table as gic_sort) and the substep runs from there,
 * building the lists; otherwise the substep runs from `state` itself and
 * `next` keeps its order (the last sort's Morton order).  The rebuild is
 * decided on the device: the previous gic_step on these lists tests every
 * granule it writes against skin / 2 of its reference position, and
 * gic_neighbors_reset forces one.  So, between calls on the same lists,
 * `state` must be the previous call's `next`, unchanged; after anything else
 * (a new state, another entry point on these lists) call gic_neighbors_reset.
 * The caller swaps state and next between calls.
 *   FP32: `next` receives float positions (posf, if set) for the next
 *   call's contact pre-tests, read from `state` (if set) when no sort runs.
 *   The call runs as a CUDA graph: a one-thread decision kernel sets the
 *   conditionals of two branches (sort + substep, or substep alone), so a
 *   substep without a rebuild launches only the decision and the substep
 *   kernel and nothing waits on the host.  The first call with a given
 *   configuration (every argument's value, the params and the structs'
 *   contents) builds and instantiates the graph; up to eight configurations
 *   stay cached (least recently used replaced).  The graph bakes in the
 *   pointers: buffers must stay allocated while calls with them may come.
 *   Arguments as for gic_sort and gic_substep (state, next and sorted must
 *   carry ids and share no array); errors as for those calls, plus
 *   GIC_ERR_CUDA if a graph cannot be built.  With sums2 the first 32 bytes
 *   of ws also hold the exact alpha_s totals while the call runs. */
int gic_step(const GicGrid* grid, const GicParams* params, const GicGranules* state, GicGranules* next,
             GicGranules* sorted, int32_t* perm, void* cell_table, void* ws, size_t ws_bytes, const GicNeighbors* nb,
             const void* u, const void* v, const void* w, const void* p, const void* alpha_f, double* alpha_s,
             void* Fs_u, void* Fs_v, void* Fs_w, double* sums2, gic_stream_t stream);

/* Request a rebuild at the next gic_contact_verlet and clear the counters
 * (flags = {0, 1, 0, 0, 0, ...}). */
int gic_neighbors_reset(const GicNeighbors* nb, gic_stream_t stream);

/* Build the Verlet lists of a sorted state without computing forces (the
 * neighbour search of Sec. 3.1, stored as the lists above): every slot gets
 * the partners within r_i + r_j + skin, in the order a rebuilding
 * gic_contact_verlet / gic_substep / gic_step would store them, from a
 * per-CTA staged neighbourhood (the cell-table box and the float positions of
 * every granule in it, in shared memory).  `sorted` and `cell_table` are the
 * output of gic_sort (FP32 with posf and ids); slots are its sorted indices,
 * so gic_step may start from `sorted` with these lists.  The build is recorded
 * (flags[4] += 1, rebuild request cleared) unless a row would exceed cap, in
 * which case the request stays set and the next call rebuilds.  One or two
 * launches, no host sync.  Errors: GIC_ERR_INVALID for FP64, a missing posf
 * or id array, or sizes that differ. */
int gic_neighbors_build(const GicGrid* grid, const GicGranules* sorted, const void* cell_table,
                        const GicNeighbors* nb, gic_stream_t stream);

/* a3: trilinear G2P of u, v, w, grad p (face differences of p) and alpha_f:
 *   F_fl = c_drag pi r^2 rho_f |u_f - v| (u_f - v) - (4/3) pi r^3 grad p
 *   a_f  = g - grad p / rho_f   (dv_f/dt of Sec. 5.2 Eq. momentum4 without the
 *          F_s term, which the sand step cannot know; a_f = g if rho_f = 0)
 *   alpha_f_p = alpha_f at the granule.
 * Fields u, v, w, p, alpha_f are real; F_fl, a_f real[4n]; alpha_f_p real[n]
 * (may be NULL).  All written. */
int gic_g2p_couple(const GicGrid* grid, const GicParams* params, const GicGranules* granules, const void* u,
                   const void* v, const void* w, const void* p, const void* alpha_f, void* F_fl, void* a_f,
                   void* alpha_f_p, gic_stream_t stream);

/* a4: (m + m_a) a = F_c + F_fl + m g + m_a a_f;  v' = v + dt' a;
 * x' = x + dt' v' (Sec. 5.2 Eq. sand kine, symplectic Euler of Sec. 4);
 * exchange force f_ex = F_fl + m_a (a_f - a) (every force the fluid exerts on
 * the granule, Sec. 5.2).  out may alias in (element-wise); out->id receives
 * in->id when both are set.  Granules that
 * would leave the box are clamped onto its boundary and flagged
 * GIC_STATUS_OUT_OF_DOMAIN. */
int gic_integrate(const GicGrid* grid, const GicParams* params, const GicGranules* in, const void* F_c,
                  const void* F_fl, const void* a_f, GicGranules* out, void* f_ex, gic_stream_t stream);

/* a5: P2G with the trilinear tent (weights beyond the first/last sample fold
 * onto it, so every granule deposits weight 1):
 *   alpha_s(c) = sum_i V_i N(x'_i - x_c) / dx^3  at the NEW positions (Sec. 5.1;
 *                Alg. 1 computes the target fraction from x^{t+dt}); WRITTEN,
 *                accumulated in FP64.  May be NULL to skip.
 *   F_s(face) += -(dt'/dt) sum_i f_ex_i N(x_i - x_face) at the OLD positions
 *                (Sec. 5.2 Exchange Momentum); ACCUMULATED (the caller zeroes
 *                them once per fluid step).  May be NULL to skip.
 *   sums2[0] = sum_c alpha_s(c) dx^3, sums2[1] = sum_i V_i (FP64; written; may
 *                be NULL; needs alpha_s).
 * old_ and new_ are the input and output of gic_integrate (same order). */
int gic_p2g(const GicGrid* grid, const GicParams* params, const GicGranules* old_, const GicGranules* new_,
            const void* f_ex, double* alpha_s, void* Fs_u, void* Fs_v, void* Fs_w, double* sums2,
            gic_stream_t stream);

/* ------------------------------------------------------------ adjoints */
/* Gradients w.r.t. positions are w.r.t. ABSOLUTE positions (metres).
 * "accumulates" = adds into the output arrays. */

/* Adjoint of the permutation of gic_sort: g_in[perm[k]] = g_out[k] (written)
 * for real[4n] position and velocity gradients. */
int gic_sort_adj(int64_t n, int32_t precision, const int32_t* perm, const void* g_pos_out, const void* g_vel_out,
                 void* g_pos_in, void* g_vel_in, gic_stream_t stream);

/* Adjoint of gic_contact for upstream gF_c (real[4n]): accumulates
 * sum_j (dF_ij/dx_ij)^T (gF_i - gF_j) into g_pos and the velocity analogue
 * into g_vel (gather form, using F_ji = -F_ij), and adds
 * sum_i gF_i . dF_i/dmu into *g_mu (double, device). */
int gic_contact_adj(const GicGrid* grid, const GicParams* params, const GicGranules* sorted, const void* cell_table,
                    const void* gF_c, void* g_pos, void* g_vel, double* g_mu, gic_stream_t stream);

/* Adjoint of gic_g2p_couple for upstream gF_fl, ga_f (real[4n]) and
 * galpha_f_p (real[n] or NULL): accumulates into g_pos, g_vel and adds
 * sum_i gF_fl_i . dF_fl_i/dc_drag into *g_cdrag (double, device). */
int gic_g2p_couple_adj(const GicGrid* grid, const GicParams* params, const GicGranules* granules, const void* u,
                       const void* v, const void* w, const void* p, const void* alpha_f, const void* gF_fl,
                       const void* ga_f, const void* galpha_f_p, void* g_pos, void* g_vel, double* g_cdrag,
                       gic_stream_t stream);

/* Adjoint of gic_integrate: from gradients of the new state (g_pos_out,
 * g_vel_out) and of f_ex (g_f_ex, may be NULL) writes the gradients of the
 * old state (g_pos_in, g_vel_in) and of F_c, F_fl, a_f (all real[4n]). */
int gic_integrate_adj(const GicGrid* grid, const GicParams* params, const GicGranules* in, const void* g_pos_out,
                      const void* g_vel_out, const void* g_f_ex, void* g_pos_in, void* g_vel_in, void* gF_c,
                      void* gF_fl, void* ga_f, gic_stream_t stream);

/* Adjoint of gic_substep's granule outputs, fused into one pass over the
 * sorted state: from the gradients of the next state (g_pos_out, g_vel_out,
 * in the sorted order) and of f_ex (g_f_ex, may be NULL) to those of the
 * sorted state's positions and velocities, i.e. gic_integrate_adj,
 * gic_g2p_couple_adj and gic_contact_verlet_adj in one kernel, each
 * partner's F_c gradient formed again from its own upstream gradients.
 * With perm (gic_sort's, or the identity gic_step writes when it does not
 * sort) the results go to g_pos_in[perm[k]], g_vel_in[perm[k]] (the
 * gic_sort_adj scatter, i.e. the order before the sort); with perm NULL to
 * index k.  g_pos_in, g_vel_in (real[4n]) are WRITTEN; *g_cdrag and *g_mu
 * (double, device) are accumulated.  The lists are checked, and rebuilt in
 * the same kernel when needed, as by gic_substep (a rebuild needs the cell
 * table of `sorted`).  The grid outputs (alpha_s, F_s) have their own
 * adjoint, gic_p2g_adj, whose g_f_ex and position gradients the caller
 * adds in.  One to two launches, no host sync. */
int gic_substep_adj(const GicGrid* grid, const GicParams* params, const GicGranules* sorted, const int32_t* perm,
                    const void* cell_table, const GicNeighbors* nb, const void* u, const void* v, const void* w,
                    const void* p, const void* alpha_f, const void* g_pos_out, const void* g_vel_out,
                    const void* g_f_ex, void* g_pos_in, void* g_vel_in, double* g_cdrag, double* g_mu,
                    gic_stream_t stream);

/* Adjoint of gic_p2g for upstream grid gradients g_alpha_s (double, or NULL)
 * and gFs_u/v/w (real, or NULL): accumulates into g_pos_old, g_pos_new and
 * writes g_f_ex (real[4n]). */
int gic_p2g_adj(const GicGrid* grid, const GicParams* params, const GicGranules* old_, const GicGranules* new_,
                const void* f_ex, const double* g_alpha_s, const void* gFs_u, const void* gFs_v, const void* gFs_w,
                void* g_pos_old, void* g_pos_new, void* g_f_ex, gic_stream_t stream);

/* ------------------------------------------------------------ windows */

/* Bytes of workspace gic_window_forward needs (sort scratch, the sorted
 * state and the two states gic_step alternates between, the permutation,
 * the per-granule force arrays and the Verlet lists). */
int gic_window_workspace_size(const GicGrid* grid, int64_t n, int32_t precision, size_t* bytes);

/* K substeps of Alg. 2 (SandSubstep): per substep gic_step (Verlet lists
 * with skin 0.025 h_c and 64 partners per granule, kept in the workspace; the
 * sort runs on list rebuilds) when state->id is set, else gic_sort,
 * gic_contact, gic_g2p_couple, gic_integrate and gic_p2g.  `state` is
 * updated in place and ends in the order of the last sort (state->id, if
 * set, maps it back).
 * alpha_s (may be NULL) is computed once, at the final positions (Alg. 1
 * CalTargetFraction); F_s (all three or none) accumulates over the K
 * substeps; sums2 (may be NULL) goes with alpha_s.
 * cell_table as for gic_sort; ws of gic_window_workspace_size bytes,
 * 256-byte aligned.  Asynchronous on `stream`. */
int gic_window_forward(const GicGrid* grid, const GicParams* params, GicGranules* state, int32_t K, const void* u,
                       const void* v, const void* w, const void* p, const void* alpha_f, double* alpha_s, void* Fs_u,
                       void* Fs_v, void* Fs_w, double* sums2, void* cell_table, void* ws, size_t ws_bytes,
                       gic_stream_t stream);

/* Bytes of DEVICE workspace gic_window_forward_host needs: everything in
 * gic_window_workspace_size plus device copies of its inputs and outputs and
 * a cell table. */
int gic_window_host_workspace_size(const GicGrid* grid, int64_t n, int32_t precision, size_t* bytes);

/* The same K-substep window on HOST buffers: copies the canonical inputs
 * (cell_xyz int32[3n], q uint32[3n], r float[n], v float[3n]) and the fluid
 * fields (real, host) to the device, runs gic_window_forward, and copies back
 * the final positions / velocities (double[3n] each, original order),
 * alpha_s (double), F_s (real, accumulated from zero) and sums2 (any output
 * may be NULL).  Host buffers should be pinned for asynchronous copies.
 * FP32 with sigma = 0: the fluid fields are copied on a second stream of the
 * library's own (created and released by the call, joined to `stream` with
 * events) while the granules are sorted and the first substep's lists built.
 * Blocks until the results are on the host (deadline 10 minutes, then
 * GIC_ERR_TIMEOUT). */
int gic_window_forward_host(const GicGrid* grid, const GicParams* params, int64_t n, int32_t precision,
                            const int32_t* cell_xyz, const uint32_t* q, const float* r, const float* v,
                            const void* u, const void* v_f, const void* w, const void* p, const void* alpha_f,
                            int32_t K, double* x_out, double* v_out, double* alpha_s, void* Fs_u, void* Fs_v,
                            void* Fs_w, double* sums2, void* ws, size_t ws_bytes, gic_stream_t stream);

/* ------------------------------------------------------------ projection */

/* The consumer of alpha_s: the velocity and density projections of the
 * fluid step (Sec. 5.1: Eqs. discret momentum, backward Euler, bring2 and
 * ppe1 a/b; Eq. position change; the limits stated after it; the face weight
 * beta_j of the appendix on the Push-Out boundary condition).  On the MAC
 * grid of `grid` (only nx, ny, nz >= 1 and dx are used):
 *   alpha_f' = 1 - min(alpha_s, alpha_s_max)                    target fluid fraction
 *   (dt/rho_f)   div(alpha_f' grad p1) = div(alpha_f' v*)       velocity projection
 *   (dt^2/rho_f) div(alpha_f' grad p2) = alpha_f' (1 - clamp(alpha_f* / alpha_f', ratio_min, ratio_max))
 *   v'  = v* - (dt/rho_f) grad p1                               projected face velocities
 *   dx  = clamp(-(dt^2/rho_f) grad p2, -h, h)                   face displacements of the fluid
 * grad = face difference / h, div = net face flux / h.  The weight of the
 * face between two cells is the mean of their alpha_f'; an open side is a
 * fluid-air interface with p = 0 in the cell beyond and face weight the
 * inner cell's alpha_f'; a solid side is a wall at rest (no flux, v' = 0 and
 * dx = 0 on its faces).  At least one side must be open.  The equations are
 * solved multiplied by alpha_f' (a symmetric positive definite system) by
 * mixed-precision iterative refinement: FP64 residuals and solution, FP32
 * conjugate gradients preconditioned by a geometric multigrid V-cycle
 * (Galerkin face weights, red-black Gauss-Seidel) for each correction.
 * Grids of 2^30 cells or more are rejected. */
typedef struct GicProjParams {
  double dt;                   /* fluid step (s) */
  double rho_f;                /* fluid density rho_0 */
  double alpha_s_max;          /* densest-packing limit of alpha_s (0.740 in 3D), in (0, 1) */
  double ratio_min, ratio_max; /* limits of alpha_f* / alpha_f' (0.5, 1.5), 0 < min <= 1 <= max */
  double tol;                  /* stop when ||b - A p||_2 <= tol ||b||_2 (FP64), > 0 */
  double inner_tol;            /* FP32 CG reduction per refinement step (1e-3), in (0, 1) */
  int32_t max_outer;           /* refinement steps per solve, >= 1 */
  int32_t max_inner;           /* CG iterations per refinement step, >= 1 */
  int32_t open[6];             /* sides -x, +x, -y, +y, -z, +z: 1 open (p = 0 beyond), 0 solid wall */
} GicProjParams;

typedef struct GicProjInfo {
  int32_t outer[2];            /* refinement steps of the p1 and p2 solves */
  int32_t inner[2];            /* FP32 CG iterations, summed over the steps */
  int32_t converged[2];        /* 1 if ||b - A p|| <= tol ||b|| was reached */
  double rel_residual[2];      /* final ||b - A p||_2 / ||b||_2 (0 when b = 0) */
} GicProjInfo;

/* Bytes of workspace gic_project needs for this grid. */
int gic_project_workspace_size(const GicGrid* grid, size_t* bytes);

/* Both projections (see above).  Cell fields nx ny nz, x fastest: alpha_s
 * (double, e.g. gic_p2g's output), alpha_star = alpha_f* (float, the fluid
 * fraction before the projection, > 0 where it matters).  Face fields as for
 * the fluid velocity (float): u, v, w = v* in; u_out, v_out, w_out = v' and
 * dx_u, dx_v, dx_w = the displacements out (each triple all or none; the
 * values on solid sides' faces are written 0).  p1, p2 (double, nx ny nz)
 * are written with the two pressures.  ws: gic_project_workspace_size
 * bytes, 256-byte aligned.  info (host, may be NULL) receives the solver's
 * counts.  The call BLOCKS: after each refinement step it reads the residual
 * on the host (waits on `stream` with a 60 s deadline per wait, then
 * GIC_ERR_TIMEOUT).  A solve that reaches max_outer without tol returns
 * GIC_OK with converged = 0; a non-finite residual returns GIC_ERR_INVALID.
 * Errors: GIC_ERR_INVALID (null pointer, bad parameter, no open side),
 * GIC_ERR_WORKSPACE, GIC_ERR_ALIGN, GIC_ERR_CUDA, GIC_ERR_TIMEOUT. */
int gic_project(const GicGrid* grid, const GicProjParams* params, const double* alpha_s, const float* alpha_star,
                const float* u, const float* v, const float* w, double* p1, double* p2, float* u_out, float* v_out,
                float* w_out, float* dx_u, float* dx_v, float* dx_w, void* ws, size_t ws_bytes, GicProjInfo* info,
                gic_stream_t stream);

/* ------------------------------------------------------------ diagnostics */

/* Contact pairs of a sorted state with id set: counts[k] = number of partners
 * of sorted granule k (int32[n]); if pairs != NULL also writes up to max_pairs
 * pairs (id_a < id_b) as int32[2 max_pairs] in unspecified order and the
 * total number into *n_pairs (int64, device; the caller zeroes it). */
int gic_contact_pairs(const GicGrid* grid, const GicGranules* sorted, const void* cell_table, int32_t* counts,
                      int32_t* pairs, int64_t max_pairs, int64_t* n_pairs, gic_stream_t stream);

/* Copy the sticky status word to *flags (host) after synchronising the
 * stream; clear it if clear != 0.  The wait polls with a deadline of
 * timeout_ms (<= 0: 60 s) and returns GIC_ERR_TIMEOUT if it passes. */
int gic_check_status(uint32_t* flags, int32_t clear, int32_t timeout_ms, gic_stream_t stream);

/* Text of the last host-side error on this thread. */
const char* gic_last_error(void);

/* Number of kernels this process has launched through the library. */
int64_t gic_launch_count(void);

/* Library version string. */
const char* gic_version(void);

/* ------------------------------------------------------------ measurement aids
 * (no counterpart in the paper: they exist to measure the path's costs) */

/* FMA rate probe: `blocks` CTAs of 256 threads each run 8 independent FMA
 * chains of `iters` steps in FP32 (precision GIC_FP32) or FP64 and store one
 * value per thread into sink (device, blocks * 256 elements of that
 * precision, 8-byte aligned).  *fmas (host, may be NULL) receives the number
 * of FMAs the launch performs, so that timing the call on `stream` gives the
 * GPU's FMA rate.  GIC_ERR_INVALID for an unknown precision, blocks or iters
 * < 1 or a null sink; GIC_ERR_ALIGN for a misaligned sink. */
int gic_probe_fma(int32_t precision, int32_t blocks, int32_t iters, void* sink, int64_t* fmas, gic_stream_t stream);

/* alpha_s of an FP32-path state (as gic_p2g computes it at the new
 * positions, Sec. 5.1) accumulated with plain FP64 atomics instead of the
 * exact 64-bit fixed point: FP64 tent weights from the fixed-point
 * positions, order-dependent at the 1e-16 level.  It exists to measure what
 * the exact accumulation costs; alpha_s (double[nx ny nz], device) is
 * written.  GIC_ERR_INVALID for an FP64 state or a null alpha_s. */
int gic_p2g_alpha_atomic64(const GicGrid* grid, const GicGranules* state, double* alpha_s, gic_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* GIC_H_ */
