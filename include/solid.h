/*
 * solid.h -- C-ABI of the GB300 solidification / macro-segregation time step.
 *
 * One time step of the operator-splitting, fully decoupled, matrix-based
 * scheme (Algorithm 1, Sec. 4 of Feng, Chen, Yu & Sun, arXiv 2303.10783):
 *   1 intermediate velocity u* from the semi-implicit momentum equation (Eq. 3.3)
 *   2 pressure-correction Poisson equation (Eq. 3.4)
 *   3 velocity projection (Eq. 3.5)
 *   4 solute transport by the matrix-based technique (Eq. 3.6-3.10)
 *   5 liquidus from the new mixture concentration (Eq. 3.14)
 *   6 intermediate temperature T* (first energy split step, Eq. 3.12)
 *   7 latent-heat correction and liquid fraction from the quadratic lever
 *     relation (Eq. 3.13, 3.15-3.17)
 *   8 liquid and solid concentrations (Eq. 3.18-3.19)
 * on a uniform staggered (MAC) grid (Sec. 3, Eq. 3.20-3.25) with 5/7-point
 * DIA systems (Sec. 4, Eq. 4.1-4.4). Every step runs in the library's own
 * CUDA kernels on the case's stream; there is no CPU fallback.
 *
 * Conventions
 *   - Cell arrays hold nx*ny*nz doubles, x fastest, then y, then z.
 *     Face arrays: u has (nx+1)*ny*nz entries (x-faces), v nx*(ny+1)*nz,
 *     w nx*ny*(nz+1); faces 0 and n along their own axis are walls.
 *     2D cases have nz = 1 and no w.
 *   - The vertical axis is y in 2D and z in 3D; gravity points along minus it.
 *   - All walls are rigid and impermeable to flow and solute. Each wall is
 *     no-slip or free-slip for the tangential velocity, and thermally
 *     adiabatic, Robin-cooled (heat flux U (T - T_ext), U = 1/(1/h + dx/(2k)))
 *     or held at a temperature that changes linearly in time (see ss_bc).
 *   - Device memory: the caller allocates one workspace of ss_workspace_bytes()
 *     bytes (any device allocator, e.g. torch) and keeps it alive until
 *     ss_destroy(); the library carves every field, DIA plane and solver
 *     vector out of it and calls no cudaMalloc for case state. Host-side
 *     case bookkeeping is malloc'd by the library.
 *   - Streams: every device operation of a case is enqueued on the stream
 *     given to ss_create_case (a cudaStream_t passed as void*; NULL = legacy
 *     default stream). Calls that return data to the host synchronise that
 *     stream; copies into device buffers stay stream-ordered.
 *   - Errors: every call returns an ss_status and never exits or traps.
 *     ss_last_error() gives a message for the calling thread. Solver
 *     outcomes are sticky on the device: a solve that reaches its iteration
 *     cap keeps its last iterate and records SS_ENOTCONV; a non-finite
 *     residual records SS_ENAN; ss_get_stats() / ss_sync() report and clear
 *     them.
 */
#ifndef SOLID_H
#define SOLID_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ss_case ss_case;

typedef enum {
  SS_OK = 0,
  SS_EINVAL = 1,    /* bad argument (NULL pointer, bad size, bad enum) */
  SS_ENOMEM = 2,    /* workspace too small */
  SS_ENOTCONV = 3,  /* a linear solve hit its iteration cap */
  SS_ENAN = 4,      /* a non-finite value appeared in a solve */
  SS_ECUDA = 5,     /* a CUDA runtime call failed (message in ss_last_error) */
  SS_ESTATE = 6,    /* call not allowed in the current state */
  SS_ETIMEOUT = 7   /* a device-side wait gave up (kernel returned early) */
} ss_status;

enum { SS_FP64 = 0, SS_MIXED = 1 };                  /* ss_grid.precision */
enum { SS_PRECOND_MG = 0, SS_PRECOND_JACOBI = 1, SS_PRECOND_DCT = 2 };   /* ss_grid.precond_p */
enum { SS_ADIABATIC = 0, SS_ROBIN = 1, SS_DIRICHLET = 2 };  /* ss_bc.thermal */
enum { SS_NOSLIP = 0, SS_FREESLIP = 1 };             /* ss_bc.flow */
enum { SS_XM = 0, SS_XP = 1, SS_YM = 2, SS_YP = 3, SS_ZM = 4, SS_ZP = 5 };  /* walls */

/* Field identifiers: bit i of a mask selects field i; pointer arrays passed
 * to ss_get_fields / ss_set_fields are indexed by these ids (SS_NFIELDS long). */
enum { SS_U = 0, SS_V = 1, SS_W = 2, SS_P = 3, SS_T = 4, SS_C = 5, SS_GL = 6, SS_CL = 7, SS_CS = 8,
       SS_NFIELDS = 9 };

/* Linear systems of one step, for the stage-level entry points. */
enum { SS_SYS_U = 0, SS_SYS_V = 1, SS_SYS_W = 2, SS_SYS_P = 3, SS_SYS_C = 4, SS_SYS_T = 5, SS_NSYS = 6 };

/* Grid, time step and solver controls. */
typedef struct {
  int dim;                   /* 2 or 3 */
  int nx, ny, nz;            /* cells per axis (nz is forced to 1 in 2D); each >= 1 */
  double lx, ly, lz;         /* domain extents [m] (lz ignored in 2D) */
  double dt;                 /* time step [s] */
  int precision;             /* SS_FP64, or SS_MIXED: FP32 inner Krylov iterations
                                inside FP64 iterative refinement */
  double tol_p;              /* relative 2-norm residual tolerance, pressure solve */
  double tol_t;              /* same for the transport solves (u, v, w, C, T) */
  int max_it_p, max_it_t;    /* iteration caps (>= 1) */
  int precond_p;             /* pressure solver (Eq. 3.4): SS_PRECOND_MG, CG preconditioned by a
                                geometric-multigrid V-cycle; SS_PRECOND_JACOBI, Jacobi-
                                preconditioned CG; SS_PRECOND_DCT, FP64 iterative refinement
                                around the exact inverse of the operator by cosine transforms
                                along x (and y in 3D) and tridiagonal solves along the last
                                axis, in FP32 (SS_MIXED) or FP64 */
} ss_grid;

/* Alloy and model data (Table 1 style). C is the mass fraction of the
 * solute-rich species in wt%. */
typedef struct {
  double Tm;        /* melting point at C = 0 [K] (Eq. 2.20) */
  double m;         /* liquidus slope [K/wt%] (< 0) */
  double kp;        /* partition coefficient, 0 < kp < 1 */
  double C0;        /* nominal concentration; Boussinesq reference C_ref [wt%] */
  double rho;       /* density [kg/m^3] */
  double k;         /* thermal conductivity [W/mK] */
  double cp;        /* specific heat [J/kgK] */
  double L;         /* latent heat [J/kg] */
  double mu;        /* liquid viscosity [Pa s] */
  double Dl;        /* liquid solute diffusivity [m^2/s] (Eq. 3.7) */
  double betaT;     /* thermal expansion [1/K] (Eq. 2.9) */
  double betaC;     /* solutal expansion [1/wt%] (Eq. 2.9) */
  double K0;        /* Carman-Kozeny prefactor [m^2]: K = K0 g^3/(1-g)^2 (Eq. 2.8) */
  double Ce;        /* eutectic concentration [wt%]; <= 0 disables the eutectic branch */
  double gravity;   /* [m/s^2] */
  double darcy_eps; /* K^{-1} = (1-g)^2 / (K0 (g^3 + darcy_eps)) */
  double Tref;      /* Boussinesq reference temperature [K] (Eq. 2.9) */
} ss_alloy;

/* Condition of one wall. All walls are impermeable (normal velocity 0).
 * Thermal: SS_ADIABATIC; SS_ROBIN, flux h (T - Text) through a film of
 * coefficient h in series with half a cell (Sec. 5, Example 1); SS_DIRICHLET,
 * wall temperature Text + dTdt * t at time t, reached over half a cell (Sec. 5,
 * Example 2 cools the bottom this way). The energy step of the step that
 * ends at time t takes the wall value at t. Flow: SS_NOSLIP (tangential
 * velocity 0 at the wall) or SS_FREESLIP (no tangential stress). */
typedef struct {
  int thermal;      /* SS_ADIABATIC, SS_ROBIN or SS_DIRICHLET */
  double h;         /* heat transfer coefficient [W/m^2K] (> 0 for Robin) */
  double Text;      /* external (Robin) or initial wall (Dirichlet) temperature [K] */
  double dTdt;      /* wall temperature rate [K/s] (Dirichlet only) */
  int flow;         /* SS_NOSLIP or SS_FREESLIP */
} ss_bc;

/* Per-step diagnostics of the most recent step (or stage call). */
typedef struct {
  long long steps;          /* steps completed since creation */
  int iters[SS_NSYS];       /* iterations of each solve (inner iterations in SS_MIXED) */
  int refinements[SS_NSYS]; /* FP64 refinement sweeps (SS_MIXED), else 0 */
  double relres[SS_NSYS];   /* final relative residual of each solve (FP64 residual) */
  int status;               /* sticky ss_status of the solves since the last read */
  int jacobi[SS_NSYS];      /* Jacobi sweeps of each transport solve (see ss_solve);
                               `iters` then counts the BiCGSTAB iterations only */
} ss_stats;

/* Stage timing: when profiling is on, the step driver records a CUDA event
 * pair on the case's stream around every stage; ss_get_profile returns the
 * accumulated device time per stage (ms) and the number of library kernels
 * launched per stage since the previous ss_get_profile call (launch counts
 * are kept whether or not profiling is on). With SS_PRECOND_DCT the pressure
 * solve of a step ends with the projection (Eq. 3.5): its time and launch
 * count under the pressure solve, and the projection stage stays at 0. */
enum { SS_PROF_ASSEMBLE = 0,   /* + SS_SYS_*: assembly of that system */
       SS_PROF_SOLVE = 6,      /* + SS_SYS_*: its solve */
       SS_PROF_PROJECT = 12, SS_PROF_LEVER = 13,
       SS_PROF_PRESOLVE_T = 14, /* the transform pre-solve of a mixed T* solve */
       SS_NPROF = 15 };
typedef struct {
  double ms[SS_NPROF];
  long long launches[SS_NPROF];
  long long kernels;        /* total library kernel launches */
  long long iters[SS_NSYS]; /* Krylov iterations summed over the solves of each system
                               (refinement sweeps for the transform pressure solver) */
  long long presolve_sweeps;/* sweeps of the T* transform pre-solve */
  long long jacobi[SS_NSYS];/* Jacobi sweeps summed over the solves of each system */
} ss_profile;

/* Bytes of device workspace a case of this grid needs (256-byte aligned
 * start required). Returns SS_EINVAL for a bad grid. */
ss_status ss_workspace_bytes(const ss_grid* grid, size_t* bytes);

/* Create a case on the current CUDA device. `workspace` is a device pointer
 * of at least ss_workspace_bytes() bytes, owned by the caller and kept alive
 * until ss_destroy(). The fields start at u = p = 0 and no alloy; call
 * ss_set_alloy before stepping. */
ss_status ss_create_case(const ss_grid* grid, void* workspace, size_t workspace_bytes, void* stream,
                         ss_case** out);

/* Set the alloy and model data; resets T = Tref, C = C0, u = p = 0 and the
 * liquid fraction to its equilibrium value (Eq. 3.15). Walls default to
 * adiabatic. Allowed before the first step only (SS_ESTATE afterwards). */
ss_status ss_set_alloy(ss_case* c, const ss_alloy* alloy);

/* Set the thermal and flow condition of wall `face` (SS_XM..SS_ZP). Allowed
 * at any time between steps. SS_EINVAL for an unknown condition, a Robin h
 * that is not > 0, or a non-finite wall temperature or rate. */
ss_status ss_set_boundary(ss_case* c, int face, const ss_bc* bc);

/* Enqueue n time steps (Algorithm 1) on the case's stream and return without
 * waiting. Launch failures return SS_ECUDA; solver outcomes are sticky (see
 * ss_sync / ss_get_stats). */
ss_status ss_step(ss_case* c, int n);

/* Same as ss_step, but the launches of one step are captured once into a
 * CUDA graph on the case's stream and the graph is replayed n times (fewer
 * host launch calls; for small cases stepped side by side on many streams).
 * The capture happens on the first call and again after any ss_set_alloy /
 * ss_set_boundary. The stream must not be the legacy default stream
 * (SS_EINVAL). Stage profiling is not recorded for graph steps; launch
 * counts are. */
ss_status ss_step_graph(ss_case* c, int n);

/* Wait for the case's stream; return and clear the sticky solver status. */
ss_status ss_sync(ss_case* c);

/* Copy the fields selected by `mask` into caller-owned buffers dst[id]
 * (device pointers if dst_is_device, else host). Host copies synchronise the
 * case's stream before returning; device copies are only enqueued on it
 * (stream-ordered, like ss_step), so work on another stream that reads dst
 * must first wait for the case's stream. */
ss_status ss_get_fields(ss_case* c, unsigned mask, void* const* dst, int dst_is_device);

/* Overwrite the fields selected by `mask` from src[id] (restart, or seeded
 * initial noise). Other fields are left as they are. In a mixed-precision
 * case with the multigrid or the cosine-transform pressure solver, each
 * step's pressure correction
 * (Eq. 3.4) starts from the previous step's correction; this call clears
 * that warm start, so the next step depends on the case's state alone and a
 * restarted case gives the same fields as a new case from the same state.
 * It clears the stored T* increment of the T* initial guess for the same
 * reason. */
ss_status ss_set_fields(ss_case* c, unsigned mask, const void* const* src, int src_is_device);

/* Recompute g_l, C_l and C_s from the current T and C in equilibrium: g_l = 1
 * at or above the liquidus, else Eq. 3.15 clamped to [0, 1]; C_l by
 * Eq. 3.18 (capped at C_e), C_s = kp C_l (Eq. 3.19). */
ss_status ss_equilibrate(ss_case* c);

/* Cap the blocks of every cooperative solver launch of this case at
 * max_blocks (0: no cap; the device's co-resident limit applies). Cases
 * stepped side by side on their own streams then share the GPU: a small case
 * whose solves are bound by synchronisation keeps few SMs busy for long, so
 * fewer blocks per case let more cases run at once. The block count sets the
 * order of the solvers' reductions: fields are deterministic for a given cap
 * and differ at rounding level between caps. A launch that solves the
 * momentum components together takes at least one block per component.
 * Drops a captured step graph. SS_EINVAL for max_blocks < 0. */
ss_status ss_set_block_cap(ss_case* c, int max_blocks);

/* Where the FP32 cosine transforms of the mixed path's pressure solve and
 * T* pre-solve form their products (SS_PRECOND_DCT; no effect otherwise):
 * SS_TC_AUTO (default): the tcgen05 tensor cores (three TF32 products per
 * step, see ss_tc_selftest) for the transforms along y of 3D slabs that fit
 * (n_y <= 128, n_z <= 256) and, on grids of at least 2^30 multiply-adds per
 * transform along x (n_x^2 n_y n_z), for those along x too, else the FP32
 * pipes; SS_TC_ON: the tensor cores for every transform they can take;
 * SS_TC_OFF: the FP32 pipes only. Results agree at rounding level. Takes
 * effect for the case's later launches (a packed batch keeps what its cases
 * had when it was created); drops a captured step graph. SS_EINVAL for
 * another mode. */
enum { SS_TC_AUTO = 0, SS_TC_ON = 1, SS_TC_OFF = 2 };
ss_status ss_set_tensor_cores(ss_case* c, int mode);

/* The FP64 -> FP32 rounding (to nearest, ties to even) that forms the FP32
 * plane copies, applied to n device values src -> dst in order on `stream`
 * (a cudaStream_t; NULL: the legacy default stream). For checking that
 * rounding against a reference conversion. SS_EINVAL for n < 0 or NULL
 * pointers with n > 0. */
ss_status ss_convert_f64_to_f32(const double* src, float* dst, long long n, void* stream);

/* Simulated time of the fields (0 at creation; each step adds dt, in the
 * lever stage that closes it). ss_set_time is stream-ordered; ss_get_time
 * synchronises the stream. Restarting from saved fields sets both. */
ss_status ss_set_time(ss_case* c, double t);
ss_status ss_get_time(ss_case* c, double* t);

/* Diagnostics of the last step; synchronises; clears the sticky status. */
ss_status ss_get_stats(ss_case* c, ss_stats* out);

/* Turn per-stage event timing on (1) or off (0). */
ss_status ss_set_profiling(ss_case* c, int on);

/* Accumulated stage times and launch counts since the previous call
 * (synchronises the stream, then resets the accumulators). */
ss_status ss_get_profile(ss_case* c, ss_profile* out);

/* Destroy the case (synchronises its stream). The workspace is the caller's. */
ss_status ss_destroy(ss_case* c);

/* Message of the last failing call on this thread ("" if none). */
const char* ss_last_error(void);

/* ---- Stage-level entry points: each runs one stage of Algorithm 1 on the
 * case's current fields, exactly as ss_step does, for stage-by-stage checks.
 *
 * ss_assemble(c, sys): build the DIA system `sys` from the current fields
 *   SS_SYS_U/V/W: momentum predictor rows (Eq. 3.3) from u^n, p^n, T^n, C_l^n, g_l^n;
 *   SS_SYS_P: pressure-correction right-hand side -(rho/dt) div u* (Eq. 3.4),
 *             mean removed, with u* the last solved momentum components;
 *   SS_SYS_C: solute system (Eq. 3.10) advected by the current u;
 *   SS_SYS_T: T* system (Eq. 3.12) advected by the current u; T is replaced
 *             by the solve's initial guess: T^n + (T* - T^{n-1}) of the
 *             previous step when that step ran its T* assembly and lever
 *             stage, else T^n unchanged.
 * ss_solve(c, sys): solve the assembled system (initial guess: the current
 *   field for U/V/W/C/T; for P the previous pressure correction in a
 *   mixed-precision case with the multigrid or cosine-transform solver, 0 in
 *   a new case, after ss_set_fields and on the other paths) into the system's
 *   solution vector;
 *   U/V/W/C use Jacobi sweeps x += D^-1 (b - A x) while each reduces the
 *   residual at least 20-fold, and BiCGSTAB after a sweep that does not:
 *   SS_FP64 sweeps in FP64 before its BiCGSTAB; SS_MIXED sweeps in FP32 as
 *   the inner solve of each FP64 refinement sweep;
 *   returns the solve's outcome.
 * ss_get_system(c, sys, dst, dst_is_device): copy planes and vectors of the
 *   system into dst[0..8] = P, W, E, S, N, B, T (DIA planes, Eq. 4.1), b
 *   (right-hand side), x (solution); NULL entries are skipped. SS_SYS_P has
 *   no planes (matrix-free constant Laplacian): only b and x.
 * ss_get_system_f32(c, sys, dst, dst_is_device): SS_MIXED cases only
 *   (SS_ESTATE otherwise; SS_EINVAL for SS_SYS_P): copy the FP32 planes the
 *   inner solves use into dst[0..7] = P, W, E, S, N, B, T, inverse diagonal
 *   (n floats each); NULL entries are skipped. Each plane entry is its FP64
 *   entry rounded to nearest, ties to even; the inverse diagonal is the FP32
 *   reciprocal of the FP32 P.
 * ss_assemble_forward(c, sys): validation mode of ss_assemble (Sec. 4,
 *   forward method, Eq. 4.5-4.7): the row equations are written from their
 *   fluxes and wall ghosts and the DIA planes and right-hand side recovered by
 *   residual probing with 3-colour trial vectors. It writes the same buffers
 *   as ss_assemble (ss_get_system then returns them; a following ss_solve
 *   uses them) and should agree with it to rounding. It evaluates each row's
 *   equation 8 times (about 30x the time of ss_assemble: 3 ms against
 *   0.1 ms per system at 1.2 M rows). SS_EINVAL for SS_SYS_P (no planes) or
 *   an unknown system.
 * ss_project(c): Eq. 3.5 with the solved u* and p'; p += p'.
 * ss_lever(c): Eq. 3.13-3.19 treating the current T field as T*, the
 *   current g_l as g_l^n and the current C as C^{n+1}; it closes a step and
 *   so advances the case's time by dt.
 * ss_assemble(c, SS_SYS_T) takes the wall temperatures at the case's time + dt. */
ss_status ss_assemble(ss_case* c, int sys);
ss_status ss_solve(ss_case* c, int sys);
ss_status ss_get_system(ss_case* c, int sys, void* const* dst, int dst_is_device);
ss_status ss_get_system_f32(ss_case* c, int sys, void* const* dst, int dst_is_device);
ss_status ss_assemble_forward(ss_case* c, int sys);
ss_status ss_project(ss_case* c);
ss_status ss_lever(ss_case* c);

/* ---- Packed batches of cases.
 *
 * The paper steps one case at a time; a packed batch steps many independent
 * cases (each a case created as above, with its own workspace and fields)
 * with one launch per stage of Algorithm 1 for all of them: the assembly and
 * pointwise stages (Eq. 3.3 and 3.4 right-hand sides, Eq. 3.10, Eq. 3.12,
 * Eq. 3.13-3.19) process a packed list of (case, row tile) items, and each
 * solve (Eq. 3.3, 3.4, 3.10, 3.12) is one cooperative launch in which every
 * case is solved by its own team of blocks, so uneven cases run side by side
 * without a launch per case; the pressure solve ends with the projection
 * (Eq. 3.5), and the T* solve starts, where ss_step's does, with the
 * transform pre-solve. Ten launches per batch step; on a non-default stream
 * they are captured once into a CUDA graph and replayed.
 * A member's fields agree with the same case stepped alone to rounding (the
 * reductions of a team of k blocks are ordered like a launch of k blocks);
 * the batch is deterministic for a given schedule.
 *
 * ss_batch_workspace_bytes(cases, n, bytes): device bytes the batch's tables
 *   need (descriptions of the n cases, solver arguments, team and tile tables).
 *   Every case must be SS_MIXED with the SS_PRECOND_DCT pressure solver and
 *   have its alloy set; a case may appear once (SS_EINVAL / SS_ESTATE else).
 * ss_batch_create(cases, n, workspace, bytes, stream, out): the batch over
 *   the n cases, its tables in `workspace` (device, 256-byte aligned, owned by
 *   the caller, alive until ss_batch_destroy), launched on `stream`. It waits
 *   for the cases' own streams once. While the batch steps them, the cases
 *   must not be used on their own streams; after ss_batch_sync they can be
 *   read (ss_get_fields, ss_get_stats) and stepped alone again. SS_EINVAL when
 *   the cases need more teams than one launch keeps resident (one block per
 *   case at least). The schedule starts at gamma = 1, tile_rows = 4096.
 * ss_batch_set_schedule(b, gamma, tile_rows): team sizes in proportion to
 *   cells^gamma (gamma in [0, 2]; at least one block, at most one per 512
 *   cells, all teams together the resident limit) and rows per tile of the
 *   packed stages (256 .. 2^24). Drops the captured graph. Changing it changes
 *   the reduction order of the solves, hence the fields at rounding level.
 * ss_batch_get_teams(b, blocks): blocks[q] = team size of case q.
 * ss_batch_step(b, n): enqueue n batch steps and return.
 * ss_batch_sync(b, launches): wait for the batch's stream, then read and
 *   clear every case's sticky solver status; returns the worst one.
 *   *launches (if not NULL) = library kernels launched by the batch so far.
 * ss_batch_destroy(b): wait for the stream and free the host side; the
 *   workspace and the cases are the caller's. */
typedef struct ss_batch ss_batch;
ss_status ss_batch_workspace_bytes(ss_case* const* cases, int n, size_t* bytes);
ss_status ss_batch_create(ss_case* const* cases, int n, void* workspace, size_t workspace_bytes, void* stream,
                          ss_batch** out);
ss_status ss_batch_set_schedule(ss_batch* b, double gamma, int tile_rows);
ss_status ss_batch_get_teams(ss_batch* b, int* blocks);
ss_status ss_batch_step(ss_batch* b, int n);
ss_status ss_batch_sync(ss_batch* b, long long* launches);
ss_status ss_batch_destroy(ss_batch* b);

/* ---- Device-side waits.
 *
 * Every wait inside a kernel of a case (the barriers of the cooperative
 * solvers) polls a bounded number of times; a wait that runs out sets a
 * sticky error, every block of the launch returns, and the next ss_sync /
 * ss_get_stats reports SS_ETIMEOUT (and clears it). The context stays
 * usable.
 *
 * ss_set_wait_limit(c, polls): polls per wait before giving up, for the
 *   case's later launches (stream-ordered); 0 restores the default (about a
 *   second). SS_EINVAL outside [0, 2^24].
 * ss_wait_selftest(c): enqueue one block that waits at a barrier no other
 *   block ever reaches, so the wait runs out after the case's limit; the
 *   next ss_sync then returns SS_ETIMEOUT. It exercises the timeout path
 *   without a fault or a hang; call ss_sync before stepping again (the
 *   sticky error would otherwise stop the next solves). */
ss_status ss_set_wait_limit(ss_case* c, long long polls);
ss_status ss_wait_selftest(ss_case* c);

/* ---- Tensor-core GEMM self-test.
 *
 * The cosine transforms of the FP32 transform solvers (SS_PRECOND_DCT in
 * SS_MIXED, and the T* pre-solve) are dense products; their tiles run on the
 * tcgen05 tensor cores as three TF32 products per K step (hi*hi + hi*lo +
 * lo*hi of a TF32 split of each FP32 operand), accumulated in FP32.
 * ss_tc_selftest(c, a, b, d, n, k, transposed) enqueues one block that forms
 * d = a b^T by that path on the case's stream: a is 128 x k, b is n x k and
 * d is 128 x n, FP32 device pointers, row-major; with transposed != 0, a and
 * b are stored transposed (k x 128 and k x n, row-major), the layout of the
 * inverse transform's operands. n a multiple of 16 in [16, 256] and
 * 1 <= k <= 4096, else SS_EINVAL. A wait that runs out sets the case's
 * sticky timeout (reported by the next ss_sync). */
ss_status ss_tc_selftest(ss_case* c, const float* a, const float* b, float* d, int n, int k, int transposed);

/* ---- Pressure-correction solve that allocates nothing.
 *
 * The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory: an application whose memory manager owns
 * the whole GPU and rejects allocations it did not make, a loop with a hard
 * latency budget where a cudaMalloc (which may synchronise the device) is
 * not acceptable, or a plugin that is handed only a stream and device
 * pointers. It solves A p = b - mean(b) for the zero-mean p, where A is the
 * negated 7-point (5-point in 2D) Laplacian on cells with zero-flux walls,
 * on an nx*ny*nz cell grid (x fastest; nz ignored when dim == 2) with
 * spacings hx, hy, hz, by the same Jacobi-preconditioned CG as ss_solve on
 * the pressure system with SS_PRECOND_JACOBI, and writes p to x.
 *
 *   b, x      device pointers to nx*ny*nz doubles (b is not modified; the
 *             caller owns both)
 *   tol       relative 2-norm residual tolerance (> 0); max_it >= 1
 *   iters, relres  optional host outputs; when either is non-NULL the call
 *             waits for the solve and returns its outcome (SS_ENOTCONV when
 *             max_it was reached); when both are NULL it returns after
 *             enqueueing on `stream` (a cudaStream_t, NULL = default stream).
 *
 * Its scratch is a fixed file-scope device array of about 4.3 MB (solver
 * vectors for at most 131072 cells, reduction partials, status block):
 * every GPU on which the library's device code is loaded holds it until the
 * process exits. Larger grids are rejected with SS_EINVAL and a message in
 * ss_last_error(). The array is shared by all calls and keeps the last
 * call's contents (each call clears what must start at zero), so calls that
 * overlap on the GPU -- on different streams or from different threads --
 * race and must not be issued. The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current
 * and caches it; devices with an index of 64 or more are refused
 * (SS_ECUDA, invalid device). Make that first call before any stream
 * capture. When iters and relres are both NULL the call only enqueues the
 * work: it then reports no solver outcome at all (no iteration cap, no
 * non-finite residual, no barrier timeout), because that outcome lives in the
 * shared array and the next call clears it. A call made while its stream is
 * being captured must pass iters = relres = NULL (the other form copies the
 * outcome back and waits for the stream). No cudaMalloc, cudaFree or
 * allocating library routine is called. */
ss_status ss_poisson_solve_noalloc(int dim, int nx, int ny, int nz, double hx, double hy, double hz,
                                   const double* b, double* x, double tol, int max_it, int* iters,
                                   double* relres, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SOLID_H */
