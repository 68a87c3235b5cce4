/*
 * icon.h -- C ABI of the GB300 dynamical-core library (sm_103a).
 *
 * The library advances the nonhydrostatic atmospheric dynamical core of an
 * ICON-style model on the icosahedral-triangular C grid (paper: Sec. "Current
 * State of the Art" -- nonhydrostatic formulation on an icosahedral-triangular
 * C grid with a terrain-following height coordinate; Table 2 -- 90 levels,
 * normal velocity on edges counted as 1.5 variables per cell; Sec. "Separation
 * of Concerns" -- index lookups on triangles and on the dual hexagons and 12
 * pentagons; Sec. "Innovations Realized" -- data stay resident on the GPU for
 * the whole run). The paper gives no equations; the discretisation implemented
 * here is stated operator by operator in the comments of the CUDA sources and
 * restated, independently, by the FP64 oracle used in the tests.
 *
 * Conventions (all entry points):
 *   - Every function except the *_free functions and icon_last_error returns an
 *     icon_status. On error, out-pointers are left untouched, a message is
 *     available from icon_last_error() (thread-local), and no handle leaks.
 *   - Handles are opaque and owned by the caller; free them with the matching
 *     *_free function (NULL is accepted). The library never frees caller memory.
 *   - Device memory comes from the allocator registered with icon_set_allocator
 *     (the Python binding registers PyTorch's caching allocator) or from
 *     cudaMalloc when none is registered. Work is issued on the stream bound by
 *     icon_set_stream (default: the legacy default stream).
 *   - Pointers named host_* are host memory (pageable or pinned); pointers named
 *     dev_* are device memory; no other pointer argument is a device pointer.
 *   - Sizes are element counts unless named *bytes.
 *   - Entry points are not reentrant on the same handle; distinct handles may be
 *     used from distinct threads.
 */
#ifndef ICON_GB300_H
#define ICON_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct icon_grid icon_grid;
typedef struct icon_state icon_state;
typedef struct icon_ensemble icon_ensemble;

typedef enum {
  ICON_OK = 0,
  ICON_EINVAL = 1,      /* bad argument (NULL handle, size mismatch, unsupported grid) */
  ICON_ENOMEM = 2,      /* the allocator returned NULL; nothing was leaked            */
  ICON_ECUDA = 3,       /* a CUDA runtime call failed (message has the CUDA error)    */
  ICON_ETIMEOUT = 4,    /* a bounded in-kernel wait ran out (persistent ensemble)     */
  ICON_ENONFINITE = 5,  /* a NaN or Inf appeared in the prognostic state              */
  ICON_EINDEX = 6       /* an internal index check failed (grid construction)         */
} icon_status;

typedef enum { ICON_FP64 = 0, ICON_MIXED = 1 } icon_precision;

typedef enum {
  ICON_CASE_REST = 0,    /* isothermal 250 K atmosphere at rest                          */
  ICON_CASE_SBR = 1,     /* solid-body rotation 20 m/s in gradient balance, 250 K        */
  ICON_CASE_JET = 2,     /* balanced 35 m/s midlatitude jet + 1 m/s bump at 20E 40N      */
  ICON_CASE_MEMBER = 3   /* case 2 with a seeded bump amplitude and position per member  */
} icon_case;

/* Integer connectivity tables (int32, row-major, entity-major). */
typedef enum {
  ICON_T_C2V = 0,   /* [Nc][3] corner vertices of each cell, counter-clockwise          */
  ICON_T_C2E = 1,   /* [Nc][3] edges; slot s joins corner s to corner (s+1)%3            */
  ICON_T_E2C = 2,   /* [Ne][2] (c1, c2); c1 is the lower cell id; normal points c1->c2  */
  ICON_T_E2V = 3,   /* [Ne][2] (v1, v2), counter-clockwise in c1; tangent points v1->v2 */
  ICON_T_V2E = 4,   /* [Nv][6] edges around each vertex, CCW from the lowest edge id    */
  ICON_T_V2C = 5,   /* [Nv][6] cell between v2e[j] and v2e[j+1]; pentagons repeat [0]   */
  ICON_T_VDEG = 6,  /* [Nv]    5 or 6                                                   */
  ICON_T_E2VT = 7,  /* [Ne][5] own edge, two other edges of c1, two other edges of c2   */
  ICON_T_E2Q = 8,   /* [Ne][4] v1, v2, vertex of c1 opposite e, vertex of c2 opposite e */
  ICON_T_C2C = 9    /* [Nc][3] cell across edge slot s (tracer transport; built on demand) */
} icon_table_int;

/* FP64 geometry tables (unit vectors are on the unit sphere; lengths in m, areas in m^2). */
typedef enum {
  ICON_G_XC = 16,   /* [Nc][3] cell circumcentres                                      */
  ICON_G_XE = 17,   /* [Ne][3] edge midpoints                                          */
  ICON_G_XV = 18,   /* [Nv][3] vertices                                                */
  ICON_G_NE = 19,   /* [Ne][3] edge normals                                            */
  ICON_G_TE = 20,   /* [Ne][3] edge tangents                                           */
  ICON_G_LE = 21,   /* [Ne] primal edge length                                         */
  ICON_G_DE = 22,   /* [Ne] dual edge length (distance of the two cell centres)        */
  ICON_G_AC = 23,   /* [Nc] cell area                                                  */
  ICON_G_AV = 24,   /* [Nv] dual cell area                                             */
  ICON_G_FE = 25,   /* [Ne] Coriolis parameter at edges                                */
  ICON_G_VTW = 26,  /* [Ne][5] tangential-velocity weights, order of ICON_T_E2VT       */
  ICON_G_KINW = 27, /* [Nc][3] kinetic-energy weights, order of ICON_T_C2E             */
  ICON_G_LSQW = 28, /* [Nv][6][3] least-squares vertex-velocity weights                */
  ICON_G_L34 = 29,  /* [Ne] distance of the two opposite quad vertices                 */
  ICON_G_SCE = 30,  /* [Nc][3] outward sign of each cell edge (+1 if c is c1)          */
  ICON_G_SVE = 31,  /* [Nv][6] circulation sign (-1 if v is v1, +1 if v2, 0 padding)   */
  ICON_G_LSQC = 32, /* [Nc][3][3] least-squares gradient weights (3-vectors, tracers)  */
  ICON_G_ROFF = 33  /* [Ne][2][3] R (x_e - x_c1), R (x_e - x_c2) (tracers)             */
} icon_table_geom;

/* Fields (copied out as FP64, row-major [entity][level], unpadded). */
typedef enum {
  ICON_F_VN = 0,       /* [Ne][N]   edge-normal velocity, m/s                        */
  ICON_F_W = 1,        /* [Nc][N+1] vertical velocity at half levels (0 = lid), m/s  */
  ICON_F_RHO = 2,      /* [Nc][N]   density, kg/m^3                                  */
  ICON_F_THETA_V = 3,  /* [Nc][N]   virtual potential temperature, K                 */
  ICON_F_EXNER = 4,    /* [Nc][N]   Exner pressure                                   */
  ICON_F_MFLX = 5,     /* [Ne][N]   step-mean horizontal mass flux, kg/m^2/s         */
  ICON_F_WFLX = 6      /* [Nc][N+1] step-mean vertical mass flux, kg/m^2/s           */
} icon_field;

/* Optional overrides for icon_state_init_ex. Negative / zero values select the default. */
typedef struct {
  double noise_K;    /* theta_v noise amplitude, K (<0: case default: 0.01 K for case 1, else 0) */
  double top_m;      /* model top, m (<=0: 75 km for N >= 60, else 30 km)                        */
  double stretch_s;  /* level stretching s (<=0: 5.5 for N >= 60, else 2)                        */
  double damp_m;     /* base of the Rayleigh damping layer, m (<=0: 45 km / 20 km)               */
  int precision;     /* icon_precision                                                           */
  int member;        /* ensemble member index for ICON_CASE_MEMBER                               */
  /* Topography (terrain-following levels, both precisions). A Gaussian mountain
   * hs = topo_height_m exp(-(r / topo_radius_m)^2), r the great-circle distance to 90E 30N,
   * under SLEVE-type levels z = zeta + hs b(zeta), b = sinh((z_top - zeta)/4 km) /
   * sinh(z_top/4 km): the lowest level follows the ground, the lid stays flat. The step then
   * takes the horizontal pressure gradient at constant height (metric correction on the
   * Exner perturbation from exp(-g z/(cpd 250 K))), the contravariant vertical velocity
   * w - (vn dz/dn + vt dz/dt) in vertical advection and vertical fluxes (zero at the ground:
   * w there is the terrain-following value), and thickness-weighted horizontal fluxes;
   * ICON_F_MFLX is then rho_e vn dz_e (kg/m/s per layer) and ICON_F_WFLX contravariant. The
   * paper's vertical coordinate is ICON's terrain-following hybrid height coordinate
   * (Sec. "Current State of the Art"). 0 = flat ground (default); 0 < topo_height_m <= 2000
   * and topo_radius_m >= 1e4, else ICON_EINVAL. Tracers of a state with topography are
   * transported with these fluxes on its own levels; such states join no ensemble. A
   * mixed-precision state with topography forms the metric terms in FP32 with its other
   * stencils and runs the lean column with each cell's own spacings and the contravariant
   * vertical velocity (or, if asked, the recomputing column; no stored-factor form). */
  double topo_height_m;
  double topo_radius_m;
} icon_case_params;

/* ---------------------------------------------------------------- allocator, stream */

/* Register device allocation callbacks (both non-NULL) or restore cudaMalloc/cudaFree
 * (both NULL). alloc(bytes, ctx) returns a device pointer aligned to >= 256 bytes or
 * NULL; dealloc(ptr, ctx) releases it. Handles created before the call keep the
 * allocator they were created with. Returns ICON_EINVAL if exactly one is NULL. */
int icon_set_allocator(void* (*alloc)(size_t bytes, void* ctx),
                       void (*dealloc)(void* ptr, void* ctx), void* ctx);

/* Bind the cudaStream_t (passed as void*) on which subsequent calls from this
 * thread enqueue work; NULL selects the legacy default stream. */
int icon_set_stream(void* cuda_stream);

/* Message of the last failing call on this thread ("" if none). Never NULL. */
const char* icon_last_error(void);

/* ---------------------------------------------------------------- grid */

/* Build the icosahedral grid R{root}B{bisections} with nlev full levels
 * (grid family: Sec. "Current State of the Art"; sizes: Table 2, where R2B8 has
 * 0.05e8 cells and R2B11 3.36e8). root must be 2 (RnBk = k+1 bisections of the
 * icosahedron), 0 <= bisections <= 10, 1 <= nlev <= 256 (nlev >= 2 for the
 * dycore). Cell ids follow the hierarchical (Morton) bisection order; vertex and
 * edge ids ascend with (lowest incident cell id, slot in that cell). Builds on the
 * GPU and returns after the build has completed. */
int icon_grid_build(int root, int bisections, int nlev, icon_grid** out);

/* Entity counts: Nc = 20*4^L, Ne = 30*4^L, Nv = 10*4^L + 2 with L = bisections+1. */
int icon_grid_counts(const icon_grid* grid, int64_t* nc, int64_t* ne, int64_t* nv);

/* Copy one table (ids above) to host memory; bytes must equal the table size
 * (int32 for ICON_T_*, double for ICON_G_*), else ICON_EINVAL. Synchronous. */
int icon_grid_copy_table(const icon_grid* grid, int table_id, void* host_dst, size_t bytes);

void icon_grid_free(icon_grid* grid);

/* ---------------------------------------------------------------- state */

/* Create a state on `grid` with the analytic initial condition `case_id`
 * (icon_case), FP64 precision and default parameters. seed selects the theta_v
 * noise and, for ICON_CASE_MEMBER, the member's bump (SplitMix64 draws). The
 * state borrows the grid, which must outlive it.
 *
 * What it computes: the paper's runs start from reanalysis and spun-up states on the
 * R2B8/R2B11 grids with 90 levels (Sec. "How Performance Was Measured", Table 2), which
 * are not available; this call stands in for them with analytic balanced states. The
 * prognostic set is the nonhydrostatic one of Sec. "Current State of the Art": edge-normal
 * velocity vn, vertical velocity w at half levels, density rho, virtual potential
 * temperature theta_v and Exner pressure pi. Readings (the paper prints none of them):
 * theta_v from the analytic case; pi analytic at the lowest full level and integrated
 * upward in discrete hydrostatic balance pi_{k-1} = pi_k - g dzh_k/(cpd theta_ic,k);
 * rho = p0 pi^(cvd/Rd)/(Rd theta_v); vn = u.n_e at edge midpoints; w = 0. Noise
 * theta_v += a(2U - 1), U from SplitMix64 draw (cell*N + k), pi held fixed. Layout and
 * precision: the state lives in device memory only (FP64 [entity][ld] rows; a mixed
 * state keeps vn in FP32 and rho, theta_v, pi, w level-major). Errors: ICON_EINVAL for a
 * NULL grid or out, an unknown case or nlev < 2; ICON_ENOMEM if the state does not fit. */
int icon_state_init(const icon_grid* grid, uint64_t seed, int case_id, icon_state** out);

/* As icon_state_init with explicit parameters (params may be NULL).
 * A mixed-precision state runs the lean column (FP32 rows and factors, FP64 hydrostatic
 * base, substitution and updates; 6 level-major scratch fields per cell) unless the
 * environment variable ICON_MIXED_COLUMN names another form when the state is created:
 * "stored" (the parts of the column system the two stages share, 17 level-major FP64
 * fields per cell, stored by the predictor when they take at most a quarter of the device
 * memory; flat levels only) or "recompute" (both stages form them; also selected by
 * ICON_MIXED_RECOMPUTE=1). The forms agree within the mixed-precision bounds. */
int icon_state_init_ex(const icon_grid* grid, uint64_t seed, int case_id,
                       const icon_case_params* params, icon_state** out);

/* Advance the state by one dycore step of length dt seconds: nsubsteps
 * predictor-corrector substeps of dt/nsubsteps (each with the vertically
 * implicit w/Exner column solve) followed by one Smagorinsky diffusion step
 * with dt. The step-mean mass fluxes (ICON_F_MFLX, ICON_F_WFLX) are recomputed;
 * the state's tracers, if any, are then transported with them, and the options set
 * with icon_state_set_option apply. The first call for a given (dt, nsubsteps)
 * records a CUDA graph of the step (again after an option or tracers are added);
 * later calls replay it. In the graph of a mixed-precision step on flat levels of a grid
 * of at least 327,680 cells (R2B6), each stage's edge diagnostics and cell kinetic energy
 * run on a second branch beside the previous stage's column (same kernels on the same inputs, so the results are the same;
 * the environment variable ICON_STEP_OVERLAP=0 at the first recording keeps one branch).
 * Waits for completion and returns ICON_ENONFINITE if a non-finite value was produced.
 * dt > 0, 1 <= nsubsteps <= 64.
 *
 * What it computes: the time step of the nonhydrostatic dynamical core on the
 * icosahedral-triangular C grid (Sec. "Current State of the Art"; the dycore is the
 * dominant, memory-bound part of the atmosphere, Sec. "Separation of Concerns"), with
 * the operators the paper names only by their stencils (triangles, dual hexagons and
 * pentagons). The discretisation is this library's reading, since the paper prints
 * none: edge-normal gradient, cell divergence, vertex curl, Perot tangential velocity,
 * kinetic-energy and vorticity-flux advection of vn, advection of w; per substep a
 * predictor (tendencies at S^n, horizontally explicit vn update, column solve) and a
 * corrector (averaged tendencies, pressure gradient at the predicted state, column
 * solve); the column is a tridiagonal system in w at the interior half levels with
 * off-centring beta = 0.65, Exner from the state equation linearised about S^n, rho,
 * Theta = rho theta_v updated in flux form, Rayleigh damping of w near the lid; after
 * the substeps a Smagorinsky diffusion of vn and theta_v. */
int icon_dycore_step(icon_state* state, double dt, int nsubsteps);

/* As icon_dycore_step without waiting: enqueues the step on the bound stream and
 * returns ICON_OK; the non-finite check is reported by icon_state_status(). */
int icon_dycore_step_async(icon_state* state, double dt, int nsubsteps);

/* Wait for the state's work and return ICON_ENONFINITE if any step since the last
 * call produced a non-finite value (the flag is then cleared), else ICON_OK. */
int icon_state_status(icon_state* state);

/* Total air mass  sum_c A_c sum_k dz_ck rho_ck  in kg, FP64, deterministic
 * (fixed summation order, bit-identical between calls on the same device). dz_ck is
 * the layer thickness of cell c (the flat levels' dz_k on flat ground, each column's
 * own thickness on terrain-following levels). The air mass is the conserved quantity
 * of the flux-form continuity equation of the step; the paper's model is run for the
 * full Earth system, whose atmosphere must conserve it (Sec. "Overview of the
 * Problem"); the FP64 sum is the precision the paper's model computes in. Errors:
 * ICON_EINVAL for a NULL argument; ICON_ECUDA if a launch fails. */
int icon_global_mass(const icon_state* state, double* out);

/* As icon_global_mass without waiting: enqueues the reduction and an asynchronous
 * copy of the result into host_out (8 bytes; pinned host memory for a truly
 * asynchronous copy). The value is valid after the bound stream has been
 * synchronised. */
int icon_global_mass_async(const icon_state* state, double* host_out);

/* Global air mass of a caller-owned density array, with no device allocation.
 *
 * The paper has no counterpart to this entry point. It exists for callers that
 * cannot allocate device memory when they need the integral: a component
 * embedded in a host model whose device memory belongs to that model's pool
 * allocator, or a latency-bound loop that forbids allocations after start-up.
 *
 * dev_rho is DEVICE memory holding the density of every cell of `grid`, row c at
 * dev_rho + c*ld, levels 0..N-1 used (ld >= N). dev_dz gives the layer thickness
 * in m: NULL takes the grid's flat levels (dz_k, the same for every cell), which is
 * right for a state on flat ground; a state on terrain-following levels needs its
 * own per-cell thicknesses dz_ck, passed as DEVICE memory in the same [Nc][ld]
 * layout as dev_rho (both pointers are only read). The result, in kg, is written to
 * *host_out; the call waits for it. With the thicknesses of the state it is the
 * integral icon_global_mass computes, summed per block of 1024 cells in a fixed
 * order (deterministic; it may differ from icon_global_mass in the last bits
 * because the grouping of the sum differs).
 *
 * Scratch: the partial sums live in one fixed array inside the library
 * (16384 partials, 128 KiB), which every GPU that loads the library holds until
 * the process exits. Hence at most 16,777,216 cells (R2B8 fits, R2B9 does not);
 * larger grids, ld < N, NULL dev_rho or host_out, a grid built on another device
 * than the current one, dev_rho or dev_dz not device memory of the current device,
 * or more than 64 devices give ICON_EINVAL with a message (the pointer check is a
 * cudaPointerGetAttributes query, which allocates nothing). Nothing is allocated
 * and no allocating library routine is called. The first call on a device looks
 * up the array's device address (with that device current); make that first call
 * before any stream capture. Every call on a device shares the array and
 * overwrites it (each call rewrites every partial it reads), so calls that overlap
 * on the GPU, for instance from two host threads or on two streams, race and must
 * be serialised by the caller. */
int icon_global_mass_noalloc(const icon_grid* grid, const double* dev_rho, const double* dev_dz, int ld,
                             double* host_out);

/* Copy a field (icon_field) to host memory as FP64, [entity][level] unpadded;
 * count must equal the field's element count. Synchronous. Pinned (page-locked) host
 * memory of a field stored in entity rows is written directly by the packing kernel over
 * the CPU-GPU link; other host memory goes through a device staging buffer and one copy. */
int icon_state_copy_field(const icon_state* state, int field_id, double* host_dst, size_t count);

/* Overwrite a prognostic field (ICON_F_VN .. ICON_F_EXNER) from FP64 host memory
 * in the same layout (rounded to FP32 where the state stores FP32). w at the lid
 * and the ground must be 0. Synchronous with respect to host_src. Pinned host memory
 * of a field stored in entity rows is read directly by the unpacking kernel. */
int icon_state_set_field(icon_state* state, int field_id, const double* host_src, size_t count);

/* Number of kernel launches in the recorded graph of one step with the given
 * (dt, nsubsteps) (records it if needed; no work is enqueued). */
int icon_state_step_kernels(icon_state* state, double dt, int nsubsteps, int* out);

/* Run one step eagerly (not from the graph) with a CUDA event pair around every
 * kernel launch and add each launch's duration (ms) to ms_per_kind[kind] and 1 to
 * launches_per_kind[kind] (host arrays of ICON_KIND_COUNT entries, accumulated,
 * not cleared). The state advances exactly as with icon_dycore_step. Waits. */
int icon_dycore_step_profile(icon_state* state, double dt, int nsubsteps, double* ms_per_kind,
                             int* launches_per_kind);

/* Self-test of internal device helpers that replace hardware operations: the
 * FP32 <-> FP64 conversions done on the integer pipe are compared bit for bit with
 * the hardware conversions on n random inputs each (finite normals up to the largest
 * binary32 exponent, zeros, exact halfway cases), checked outside the binary32 normal
 * range against their documented mapping (signed zero below, signed infinity above,
 * NaN included; binary32 subnormals to a signed zero), and the Newton-Raphson FP64
 * reciprocal of the column solves is
 * compared with the IEEE division on n random operands (within 1 ulp for 1/x,
 * 2 ulps for a * (1/x)). *failures receives the number of mismatches (0 expected).
 * Allocates 4 bytes with cudaMalloc (not the registered allocator). Waits. */
int icon_selftest(long long n, unsigned* failures);

/* Measured FP64 instruction throughput of the current device, instructions per second
 * (a fused multiply-add counts as one), for FP64 fused multiply-adds and for FP64 adds:
 * 16 blocks of 256 threads per SM, eight independent dependency chains per thread, best
 * of five timed launches (CUDA events on the bound stream). This is the peak the FP64-bound
 * kernels of the step are measured against (no counterpart in the paper). Allocates 8
 * bytes with cudaMalloc (not the registered allocator). Waits. */
int icon_probe_fp64_rate(double* fma_per_s, double* add_per_s);

/* Name of kernel kind i (0 <= i < ICON_KIND_COUNT), or NULL. Mixed-precision
 * stencil kinds: 10 vertex, 11 edge diagnostics, 12 cell kinetic energy,
 * 13 edge tendency, 15 column-input gather, 16 diffusion vertex/divergence;
 * 20 tracer transport, 21 divergence damping, 22 background diffusion (options),
 * 23 terrain metrics (states with topography), 24 and 25 the lean mixed column and
 * its input gather (the default column of mixed states on flat levels). */
const char* icon_kernel_kind_name(int kind);
#define ICON_KIND_COUNT 26

/* Storage precision of the state (icon_precision). */
int icon_state_precision(const icon_state* state, int* out);

void icon_state_free(icon_state* state);

/* ---------------------------------------------------------------- options */

/* Option ids of icon_state_set_option. */
enum {
  /* Fourth-order divergence damping of the corrector's vn^{n+1} before its fluxes are
   * formed: vn -= c4 Abar^2 grad(div(grad(div vn))), Abar = 4 pi R^2 / Nc, with the
   * step's own divergence and gradient operators (ICON damps its corrector's divergence
   * this way; the paper prints none). value = c4 in [0, 0.05]; 0 turns it off. Default
   * 0.0025 (ICON's default fourth-order coefficient): without it the triangular grid's
   * divergence noise grows at the pentagons under the jet and the R2B6/90 benchmark state
   * goes non-finite after about 23 simulated hours. Both precisions, the persistent
   * ensemble and the decomposed domain. */
  ICON_OPT_DIVDAMP4 = 1,
  /* Fourth-order background diffusion of vn in the diffusion step, once per step:
   * vn -= c Abar^2 L(L(vn)) with the step's vector Laplacian L (an ICON option; the paper
   * prints none). value = c in [0, 0.01]; 0 (the default) turns it off. Both precisions;
   * not in the persistent ensemble. */
  ICON_OPT_DIFF4 = 2,
  /* Upwind theta_v in the heat fluxes (value 1; 0, the default, is the centred mean):
   * the flux through an edge carries theta_v of the cell the flow comes from, in both
   * stages; the pressure gradient keeps the centred value (an ICON option, first order
   * here; the paper prints none). Both precisions; not in the persistent ensemble. */
  ICON_OPT_UPWIND_THETA = 3
};

/* Set an option of a state; the next step records a new graph. ICON_EINVAL for an
 * unknown option or a value outside its range. */
int icon_state_set_option(icon_state* state, int option, double value);

/* ---------------------------------------------------------------- tracers */

/* Give the state ntracers (1..8) mixing-ratio tracers, FP64 in both precisions,
 * initially 0; once per state. From then on every icon_dycore_step also transports
 * them after the dycore substeps and the diffusion with that step's substep-averaged
 * FP64 mass fluxes (ICON_F_MFLX, ICON_F_WFLX): flux form, second order (least-squares
 * cell gradients, upwind edge and half-level values at the half-step departure point),
 * consistent with the continuity equation of the step (a uniform tracer stays uniform,
 * tracer mass is conserved), no limiter. The atmosphere of the paper's model carries
 * tracers (Sec. "Overview of the Problem"); the scheme is this library's reading. Builds
 * the grid's tracer tables on first use and allocates 6 (FP64) or 8 (mixed) cell fields
 * and one edge field of scratch plus the tracers; ICON_ENOMEM if they do not fit.
 * States with tracers cannot join an ensemble. */
int icon_state_add_tracers(icon_state* state, int ntracers);
int icon_state_tracers(const icon_state* state, int* ntracers);

/* Copy tracer t (0 <= t < ntracers) from / to host memory: count must be Nc*N doubles
 * laid out [cell][level] (level 0 at the top), else ICON_EINVAL. Synchronous. */
int icon_state_set_tracer(icon_state* state, int t, const double* host_src, size_t count);
int icon_state_copy_tracer(const icon_state* state, int t, double* host_dst, size_t count);

/* ---------------------------------------------------------------- domain decomposition */

/* Horizontal domain decomposition of the FP64 step with halo exchanges (the paper runs
 * the atmosphere decomposed over many GPUs and exchanges subdomain halos point to point
 * after its stencil phases, Sec. "Exploiting the Earth System's Complexity to Flexibly
 * Utilize System Parallelism"). Part p of P owns the contiguous range [p Nc/P, (p+1) Nc/P)
 * of the Morton cell order, the edges whose first (lower-id) cell it owns and the
 * vertices whose lowest incident cell it owns; its local grid adds every cell within
 * halo_rings vertex rings of its own cells, with their edges and vertices. Local order:
 * owned entities first, then halo entities, each ascending in global id. */
typedef struct icon_domain icon_domain;

/* Host-only plan of one part from the global connectivity (ICON_T_C2E, ICON_T_E2C,
 * ICON_T_C2V, ICON_T_V2C, ICON_T_VDEG tables in host memory, as icon_grid_copy_table
 * writes them). host_counts[6] receives the owned cells, edges, vertices and the local
 * cells, edges, vertices. If host_local is not NULL it receives the local-to-global ids
 * (local cells, then edges, then vertices; sum of the local counts entries), and
 * host_owner / host_owner_index (same length, may be NULL) the owning part of each local
 * entity and its index in that part's local order. 1 <= nparts <= Nc, 0 <= part < nparts,
 * 0 <= halo_rings <= 16, else ICON_EINVAL. Allocates nothing on the device. */
int icon_partition_plan(int64_t nc, int64_t ne, int64_t nv, const int32_t* host_c2e, const int32_t* host_e2c,
                        const int32_t* host_c2v, const int32_t* host_v2c, const int32_t* host_vdeg, int nparts,
                        int part, int halo_rings, int64_t* host_counts, int32_t* host_local, int32_t* host_owner,
                        int32_t* host_owner_index);

/* Decompose an FP64 state on flat levels without tracers, background diffusion or upwind
 * theta (its divergence damping is kept, with the global grid's mean cell area) into
 * nparts parts (1..64) with halo_rings (3..16) vertex rings of halo, on the current device: each part
 * gets its local grid (connectivity remapped, geometry gathered) and a state holding its
 * local rows of the global state's fields. The global state is only read; the domain
 * keeps a pointer to its grid, which must outlive it. ICON_EINVAL for other states. */
int icon_domain_create(const icon_state* global_state, int nparts, int halo_rings, icon_domain** out);

/* One dycore step of every part (the kernels of icon_dycore_step on the local grids),
 * with the halo rows of the stage outputs (vn; w, rho, theta_v, Exner) copied from their
 * owners after each predictor and corrector stage and of vn, theta_v, Exner after the
 * diffusion. The owned rows equal the single-domain step's bit for bit. Eager launches on
 * the bound stream; waits; ICON_ENONFINITE as icon_dycore_step. */
int icon_domain_step(icon_domain* domain, double dt, int nsubsteps);

/* Air mass: each part's owned cells summed in a fixed order, the parts' sums added in
 * part order (the scalar all-reduce of a distributed run). */
int icon_domain_global_mass(icon_domain* domain, double* host_out);

/* A field of the decomposed state in the global layout of icon_state_copy_field, from
 * the owners' rows. Synchronous. */
int icon_domain_copy_field(icon_domain* domain, int field_id, double* host_dst, size_t count);

/* host_counts[6]: owned cells, edges, vertices and local cells, edges, vertices of a part. */
int icon_domain_part_counts(const icon_domain* domain, int part, int64_t* host_counts);

void icon_domain_free(icon_domain* domain);

/* ---------------------------------------------------------------- ensemble */

/* Tile of a kernel kind (the kind numbers of icon_kernel_kind_name) of a mixed-precision
 * state. Stencil kinds (10, 11, 12, 13, 15, 16): lanes per entity (32 = one entity per
 * warp, 16 = two, 8 = four) and threads per block (64, 128, 256 or 512). The lean column
 * (24): its launch shape, lanes = the unroll factor of its two sweeps and block = the
 * resident 128-thread blocks per SM its registers are held to, one of (2, 9), (2, 10),
 * (2, 8), (2, 12), (2, 6); a tuned shape applies to the predictor's column, the
 * corrector's keeps (2, 9) unless a shape is forced. The autotuner picks them on the
 * first step (timing every candidate on the state's data, in the order of the step;
 * cached per grid size, level count and GPU,
 * and in the file named by the environment variable ICON_TUNE_CACHE if set). set_tiling
 * forces a tile (lanes 0 restores automatic choice; ICON_EINVAL for any other value
 * outside these sets); results do not depend on the tile. */
int icon_state_tiling(const icon_state* state, int kind, int* lanes, int* block);
int icon_state_set_tiling(icon_state* state, int kind, int lanes, int block);

/* Group 1 <= n <= 64 distinct mixed-precision states (grids of any size, one
 * level count <= 96) for batched stepping (the paper runs ensemble members,
 * Sec. "Implications"). The ensemble borrows the states, which must outlive it. */
int icon_ensemble_create(icon_state* const* members, int n, icon_ensemble** out);

/* Advance every member by nsteps dycore steps (member i with dt_per_member[i],
 * host array of n doubles, all with nsubsteps substeps) in ONE persistent
 * cooperative launch per step for all members: every phase of the step is a work
 * list over (member, entity) separated by a bounded grid barrier. The launch is
 * recorded in a CUDA graph per (dt_per_member, nsubsteps). Waits; returns
 * ICON_ETIMEOUT if a barrier wait ran out (the kernel then returns early and the
 * members' states are not valid), ICON_ENONFINITE as icon_dycore_step. */
int icon_ensemble_step(icon_ensemble* ens, const double* dt_per_member, int nsubsteps, int nsteps);

/* Ensemble options: ICON_ENS_SPIN_LIMIT = spins (about 0.1 us each) before a grid
 * barrier wait gives up (default 2^24); ICON_ENS_TEST_SKIP_BARRIER = 1 makes block
 * 0 skip its first barrier arrival so that the others' waits run out (fault test). */
#define ICON_ENS_SPIN_LIMIT 1
#define ICON_ENS_TEST_SKIP_BARRIER 2
int icon_ensemble_set_option(icon_ensemble* ens, int option, long long value);

/* Phases of the persistent ensemble step, in the order they run (each a work list over
 * all members ended by a grid barrier; the damping phases only when a member damps,
 * the corrector-update phase only with stored column factors). */
#define ICON_ENS_PH_ZERO 0          /* zero the step-mean fluxes */
#define ICON_ENS_PH_VERTEX 1        /* vertex curl and w at vertices */
#define ICON_ENS_PH_EDGE_DIAG 2     /* tangential velocity */
#define ICON_ENS_PH_CELL_KE 3       /* cell kinetic energy */
#define ICON_ENS_PH_EDGE_TEND 4     /* vn tendency and update, edge fluxes */
#define ICON_ENS_PH_DD_DIV 5        /* divergence damping: cell divergence */
#define ICON_ENS_PH_DD_LAP 6        /* divergence damping: its Laplacian */
#define ICON_ENS_PH_DD_EDGE 7       /* divergence damping: edge update (not in the lean form) */
#define ICON_ENS_PH_GATHER 8        /* column inputs gathered from the edges */
#define ICON_ENS_PH_COLUMN 9        /* vertically implicit column solve */
#define ICON_ENS_PH_CORR_UPDATE 10  /* corrector update with stored factors */
#define ICON_ENS_PH_DIFF_VERTEX 11  /* diffusion: vertex and cell terms */
#define ICON_ENS_PH_DIFF_EDGE 12    /* diffusion: edge update */
#define ICON_ENS_PH_DIFF_THETA 13   /* diffusion: theta_v and Exner */
#define ICON_ENS_PHASE_COUNT 14

/* Advance every member by ONE step as icon_ensemble_step does, launched outside the
 * graph with a phase timer: block 0 of the persistent kernel reads the GPU's global
 * timer as it leaves each grid barrier. Adds each phase's wall time (ms, from the
 * previous barrier to the one that closes it; the last phase up to the kernel's end
 * measured with CUDA events) to ms_per_phase[kind] and 1 per barrier to
 * count_per_phase[kind] (host arrays of ICON_ENS_PHASE_COUNT entries, accumulated, not
 * cleared). Waits; errors as icon_ensemble_step. */
int icon_ensemble_step_profile(icon_ensemble* ens, const double* dt_per_member, int nsubsteps, double* ms_per_phase,
                               int* count_per_phase);

/* Name of ensemble phase i (0 <= i < ICON_ENS_PHASE_COUNT), or NULL. */
const char* icon_ensemble_phase_name(int phase);

void icon_ensemble_free(icon_ensemble* ens);

#ifdef __cplusplus
}
#endif
#endif /* ICON_GB300_H */
