// C-ABI of libsolid: case lifetime, workspace layout, the Algorithm 1 step
// driver and field I/O. See include/solid.h for the contract of each call.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "solid_internal.cuh"

using namespace solid;


namespace {

thread_local char g_err[512] = "";

ss_status fail(ss_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return s;
}

#define CUDA_TRY(expr)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess) return fail(SS_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

__global__ void k_fill(double* x, double v, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = v;
}

__global__ void k_set_spin_limit(DevStatus* st, long long polls) { st->spin_limit = polls; }

// One block waits at a barrier of a two-block team whose other member is
// never launched: nothing ever completes the count, so the wait runs until
// the case's poll limit, then sets the sticky barrier error and returns.
__global__ void k_wait_selftest(DevStatus* st) {
  unsigned int epoch = 0;
  const Team t{0, 2, &st->selftest_counter, nullptr};
  team_barrier(st, t, epoch);
}

// Workspace planner: the same walk computes the size and the pointers.
struct Planner {
  char* base;
  size_t off;
  long long guard;
  explicit Planner(char* b, long long g) : base(b), off(0), guard(g) {}
  template <typename T>
  T* vec(long long n) {
    const size_t bytes = (size_t)(n + 2 * guard) * sizeof(T);
    T* p = base ? reinterpret_cast<T*>(base + off) + guard : nullptr;
    off += (bytes + 255) & ~(size_t)255;
    return p;
  }
  template <typename T>
  T* raw(size_t bytes) {
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += (bytes + 255) & ~(size_t)255;
    return p;
  }
};

}  // namespace

namespace solid {
// Lets other translation units set the message ss_last_error() returns.
void set_error_message(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}
}  // namespace solid

struct ss_case {
  ss_grid g;
  Params pr;
  cudaStream_t stream;
  char* ws;
  size_t ws_bytes;
  double *u, *v, *w, *p, *T, *C, *gl, *Cl, *Cs, *Kinv, *Ag;
  double *ustar[3], *pc, *pb;
  double* Tinc;              // T* - T^n of the last step (initial guess of the next T* solve), or 0
  int tinc_pending;          // the last T* assembly left -T^n in Tinc for the lever stage
  Sys sys[SS_NSYS];
  MGPlan mg;
  DctPlan dct;
  Scratch sc[kMaxTeams];   // Krylov scratch per team of a joint solve (set 0 for every other solve)
  DevStatus* st;
  int alloy_set;
  long long steps;
  ss_bc bc[6];
  long long n_face[3], n_cell;
  // stage profiling
  int profiling;
  std::vector<cudaEvent_t>* pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>>* pending;
  long long launches[SS_NPROF];
  // captured step graph
  cudaGraphExec_t graph;
  long long graph_kernels;   // library kernels per captured step
  int block_cap;             // > 0: blocks per cooperative solver launch at most (ss_set_block_cap)
  int cinv_n;                // cells of an exactly solved coarsest level (0: none)
  double cinv_host[kExactCoarse * kExactCoarse];   // its pseudo-inverse, row-major
  float cinv_host32[kExactCoarse * kExactCoarse];  // the same in FP32 (mixed cases)
};

namespace {

bool grid_ok(const ss_grid* g, char* why, size_t len) {
  if (!g) { snprintf(why, len, "grid is NULL"); return false; }
  if (g->dim != 2 && g->dim != 3) { snprintf(why, len, "dim must be 2 or 3 (got %d)", g->dim); return false; }
  const int nz = g->dim == 3 ? g->nz : 1;
  if (g->nx < 1 || g->ny < 1 || nz < 1) { snprintf(why, len, "cell counts must be >= 1"); return false; }
  const double cells = (double)(g->nx + 1) * (g->ny + 1) * (nz + 1);
  if (cells > 1.5e9) { snprintf(why, len, "grid too large for 32-bit row indices"); return false; }
  if (!(g->lx > 0) || !(g->ly > 0) || (g->dim == 3 && !(g->lz > 0))) { snprintf(why, len, "extents must be > 0"); return false; }
  if (!(g->dt > 0)) { snprintf(why, len, "dt must be > 0"); return false; }
  if (g->precision != SS_FP64 && g->precision != SS_MIXED) { snprintf(why, len, "unknown precision %d", g->precision); return false; }
  if (!(g->tol_p > 0) || !(g->tol_t > 0)) { snprintf(why, len, "tolerances must be > 0"); return false; }
  if (g->max_it_p < 1 || g->max_it_t < 1) { snprintf(why, len, "iteration caps must be >= 1"); return false; }
  if (g->precond_p != SS_PRECOND_MG && g->precond_p != SS_PRECOND_JACOBI && g->precond_p != SS_PRECOND_DCT) {
    snprintf(why, len, "unknown pressure preconditioner %d", g->precond_p);
    return false;
  }
  return true;
}

void fill_params(ss_case* c, const ss_alloy* al);

void plan(ss_case* c, Planner& pl) {
  const long long nx = c->g.nx, ny = c->g.ny, nz = c->g.dim == 3 ? c->g.nz : 1;
  c->n_cell = nx * ny * nz;
  c->n_face[0] = (nx + 1) * ny * nz;
  c->n_face[1] = nx * (ny + 1) * nz;
  c->n_face[2] = nx * ny * (nz + 1);
  const long long nmax = std::max(std::max(c->n_face[0], c->n_face[1]), std::max(c->n_face[2], c->n_cell));
  c->st = pl.raw<DevStatus>(sizeof(DevStatus));
  c->u = pl.vec<double>(c->n_face[0]);
  c->v = pl.vec<double>(c->n_face[1]);
  c->w = pl.vec<double>(c->n_face[2]);
  c->p = pl.vec<double>(c->n_cell);
  c->T = pl.vec<double>(c->n_cell);
  c->C = pl.vec<double>(c->n_cell);
  c->gl = pl.vec<double>(c->n_cell);
  c->Cl = pl.vec<double>(c->n_cell);
  c->Cs = pl.vec<double>(c->n_cell);
  c->Kinv = pl.vec<double>(c->n_cell);
  c->Ag = pl.vec<double>(c->n_cell);
  for (int a = 0; a < 3; ++a) c->ustar[a] = pl.vec<double>(c->n_face[a]);
  c->pc = pl.vec<double>(c->n_cell);
  c->pb = pl.vec<double>(c->n_cell);
  c->Tinc = pl.vec<double>(c->n_cell);
  // DIA planes: one set per momentum component, so that u*, v*, w* can be
  // solved together (one launch, one team of blocks each); the C and T
  // systems reuse the u* set, each assembled right before its solve (Sec. 4
  // term-wise assembly per step)
  const bool mixed = c->g.precision == SS_MIXED;
  Planes<double> a[3];
  Planes<float> af[3];
  double* b[3];
  const int ncomp = c->g.dim;
  for (int q = 0; q < 3; ++q) {
    if (q >= ncomp) {   // no w* system in 2D: alias the first set
      a[q] = a[0]; af[q] = af[0]; b[q] = b[0];
      continue;
    }
    a[q].P = pl.vec<double>(nmax); a[q].W = pl.vec<double>(nmax); a[q].E = pl.vec<double>(nmax);
    a[q].S = pl.vec<double>(nmax); a[q].N = pl.vec<double>(nmax);
    a[q].B = pl.vec<double>(nmax); a[q].T_ = pl.vec<double>(nmax); a[q].idiag = pl.vec<double>(nmax);
    b[q] = pl.vec<double>(nmax);
    af[q] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    if (mixed) {
      af[q].P = pl.vec<float>(nmax); af[q].W = pl.vec<float>(nmax); af[q].E = pl.vec<float>(nmax);
      af[q].S = pl.vec<float>(nmax); af[q].N = pl.vec<float>(nmax);
      af[q].B = pl.vec<float>(nmax); af[q].T_ = pl.vec<float>(nmax); af[q].idiag = pl.vec<float>(nmax);
    }
  }
  const int mdims[3][3] = {{(int)nx + 1, (int)ny, (int)nz}, {(int)nx, (int)ny + 1, (int)nz}, {(int)nx, (int)ny, (int)nz + 1}};
  for (int s = 0; s < SS_NSYS; ++s) {
    Sys& S = c->sys[s];
    const int set = (s <= SS_SYS_W) ? s : 0;
    S.a = a[set];
    S.af = af[set];
    S.b = b[set];
    if (s <= SS_SYS_W) {
      S.d = {mdims[s][0], mdims[s][1], mdims[s][2], c->n_face[s], make_fastdiv(mdims[s][0]), make_fastdiv(mdims[s][1])};
      S.x = c->ustar[s];
    } else {
      S.d = {(int)nx, (int)ny, (int)nz, c->n_cell, make_fastdiv((unsigned)nx), make_fastdiv((unsigned)ny)};
      S.x = (s == SS_SYS_C) ? c->C : (s == SS_SYS_T) ? c->T : c->pc;
    }
  }
  c->sys[SS_SYS_P].b = c->pb;
  if (c->g.precond_p == SS_PRECOND_MG) {
    fill_params(c, nullptr);
    plan_multigrid(c->pr, c->mg, c->g.precision == SS_MIXED);
    for (int l = 0; l < c->mg.nl; ++l) {
      const long long nl = (long long)c->mg.n[l][0] * c->mg.n[l][1] * c->mg.n[l][2];
      for (int q = 0; q < 4; ++q)
        c->mg.vec[l][q] = c->mg.fp32 ? (void*)pl.vec<float>(nl) : (void*)pl.vec<double>(nl);
    }
    // a small coarsest level is solved exactly: its pseudo-inverse, formed on
    // the host here and copied into the workspace when the case is created
    c->cinv_n = coarse_pseudo_inverse(c->mg, c->g.dim, c->cinv_host);
    if (c->cinv_n > 0)
      c->mg.cinv = pl.raw<char>((size_t)c->cinv_n * c->cinv_n * (c->mg.fp32 ? sizeof(float) : sizeof(double)));
  }
  if (c->g.precond_p == SS_PRECOND_DCT) {
    fill_params(c, nullptr);
    plan_dct(c->pr, c->dct, mixed);
    const size_t esz = mixed ? sizeof(float) : sizeof(double);
    c->dct.T1 = mixed ? (void*)pl.vec<float>(c->n_cell) : (void*)pl.vec<double>(c->n_cell);
    c->dct.T2 = mixed ? (void*)pl.vec<float>(c->n_cell) : (void*)pl.vec<double>(c->n_cell);
    c->dct.tables = pl.raw<char>(dct_table_elems(c->dct) * esz);
    c->dct.img = mixed ? pl.raw<char>(dct_image_bytes(c->dct)) : nullptr;
    const size_t tb = dct_thomas_bytes(c->dct);
    c->dct.thomas = tb ? pl.raw<char>(tb) : nullptr;
  }
  // Krylov scratch: set 0 serves every solve (multigrid included); sets 1, 2
  // serve the v* and w* teams of the joint momentum solve, with only the
  // vectors a transport solve uses (the mixed solve's FP64 refinement
  // residual and FP32 inner vectors, or the FP64 solve's seven vectors).
  for (int t = 0; t < kMaxTeams; ++t) {
    Scratch& sc = c->sc[t];
    const bool used = (t == 0) || (t < ncomp);
    const int nv = !used ? 0 : (t == 0) ? 8 : (mixed ? 1 : 7);
    for (int q = 0; q < 8; ++q) sc.v[q] = (q < nv) ? pl.vec<double>(nmax) : nullptr;
    for (int q = 0; q < 9; ++q) sc.f[q] = (used && mixed) ? pl.vec<float>(nmax) : nullptr;
    sc.max_blocks = max_cooperative_blocks();
    sc.partial = used ? pl.raw<double>((size_t)kMaxRedSlots * sc.max_blocks * sizeof(double)) : nullptr;
  }
}

// Guard band (elements) in front of and behind every vector: at least one
// x-y plane of any system so that the 7-point stencil reads in bounds, and a
// multiple of 64 elements so that every vector starts on a 256-byte boundary
// (element 0 of a warp's access then begins a cache line).
long long guard_of(const ss_grid* g) {
  const long long plane = (long long)(g->nx + 1) * (g->ny + 1) + 1;
  return (plane + 63) / 64 * 64;
}

void fill_params(ss_case* c, const ss_alloy* al) {
  Params& pr = c->pr;
  pr.dim = c->g.dim;
  pr.nx = c->g.nx;
  pr.ny = c->g.ny;
  pr.nz = c->g.dim == 3 ? c->g.nz : 1;
  pr.vert = c->g.dim == 2 ? 1 : 2;
  pr.fnx = make_fastdiv((unsigned)pr.nx);
  pr.fny = make_fastdiv((unsigned)pr.ny);
  pr.hx = c->g.lx / c->g.nx;
  pr.hy = c->g.ly / c->g.ny;
  pr.hz = c->g.dim == 3 ? c->g.lz / c->g.nz : 1.0;
  pr.dt = c->g.dt;
  if (al) {
    pr.Tm = al->Tm; pr.m = al->m; pr.kp = al->kp; pr.C0 = al->C0; pr.rho = al->rho; pr.k = al->k;
    pr.cp = al->cp; pr.L = al->L; pr.mu = al->mu; pr.Dl = al->Dl; pr.betaT = al->betaT; pr.betaC = al->betaC;
    pr.K0 = al->K0; pr.Ce = al->Ce; pr.gravity = al->gravity; pr.eps = al->darcy_eps; pr.Tref = al->Tref;
    pr.has_eutectic = al->Ce > 0.0;
  }
  const double h[3] = {pr.hx, pr.hy, pr.hz};
  for (int a = 0; a < 3; ++a) {
    pr.ih[a] = 1.0 / h[a];
    pr.ih2[a] = pr.ih[a] * pr.ih[a];
  }
  pr.idt = 1.0 / pr.dt;
  if (c->alloy_set || al) {
    pr.nu = pr.mu / pr.rho;
    pr.irho = 1.0 / pr.rho;
    pr.alphaT = pr.k / (pr.rho * pr.cp);
    pr.rhs_scale = -pr.rho / pr.dt;
    pr.proj_k = pr.dt / pr.rho;
    pr.cpL = pr.cp / pr.L;
    pr.Lcp = pr.L / pr.cp;
    pr.half_nu = 0.5 * pr.nu;
    pr.lev_a = 1.0 - pr.kp;
    pr.lev_cpLa = pr.cpL * pr.lev_a;
    pr.lev_aTm = pr.lev_a * pr.Tm;
    pr.lev_4a = 4.0 * pr.lev_a;
    pr.lev_2a = 2.0 * pr.lev_a;
    pr.lev_inv2a = 1.0 / pr.lev_2a;
    pr.Te = pr.Tm + pr.m * pr.Ce;
    for (int a = 0; a < 3; ++a) {
      pr.hh[a] = 0.5 * pr.ih[a];
      pr.nu_ih2[a] = pr.nu * pr.ih2[a];
      pr.two_nu_ih2[a] = 2.0 * pr.nu_ih2[a];
      pr.ih_irho[a] = pr.ih[a] * pr.irho;
      pr.alpha_ih2[a] = pr.alphaT * pr.ih2[a];
      pr.half_Dl_ih2[a] = 0.5 * pr.Dl * pr.ih2[a];
    }
  }
  for (int a = 0; a < 3; ++a) {
    pr.df_hh[a] = df_const(pr.hh[a]);
    pr.df_ih[a] = df_const(pr.ih[a]);
    pr.df_nu_ih2[a] = df_const(pr.nu_ih2[a]);
    pr.df_two_nu_ih2[a] = df_const(pr.two_nu_ih2[a]);
    pr.df_alpha_ih2[a] = df_const(pr.alpha_ih2[a]);
    pr.df_half_Dl_ih2[a] = df_const(pr.half_Dl_ih2[a]);
  }
  pr.df_idt = df_const(pr.idt);
  pr.df_half_nu = df_const(pr.half_nu);
  pr.wall_mask = 0;
  for (int q = 0; q < 6; ++q) {
    const int axis = q / 2;
    const ss_bc& bc = c->bc[q];
    pr.wall_coef[q] = 0.0;
    pr.wall_T0[q] = 0.0;
    pr.wall_rate[q] = 0.0;
    pr.slip[q] = bc.flow == SS_FREESLIP;
    if (axis >= pr.dim || !c->alloy_set) continue;
    if (bc.thermal == SS_ROBIN) {            // film h_c in series with half a cell
      const double U = 1.0 / (1.0 / bc.h + h[axis] / (2.0 * pr.k));
      pr.wall_coef[q] = U / (pr.rho * pr.cp * h[axis]);
      pr.wall_T0[q] = bc.Text;
    } else if (bc.thermal == SS_DIRICHLET) { // wall temperature over half a cell
      pr.wall_coef[q] = pr.k / (0.5 * h[axis]) / (pr.rho * pr.cp * h[axis]);
      pr.wall_T0[q] = bc.Text;
      pr.wall_rate[q] = bc.dTdt;
    }
    if (pr.wall_coef[q] != 0.0) pr.wall_mask |= 1 << q;
    pr.df_wall_coef[q] = df_const(pr.wall_coef[q]);
  }
}

ss_status check_case(ss_case* c) {
  if (!c) return fail(SS_EINVAL, "case is NULL");
  return SS_OK;
}

double* field_ptr(ss_case* c, int id) {
  switch (id) {
    case SS_U: return c->u;
    case SS_V: return c->v;
    case SS_W: return c->w;
    case SS_P: return c->p;
    case SS_T: return c->T;
    case SS_C: return c->C;
    case SS_GL: return c->gl;
    case SS_CL: return c->Cl;
    case SS_CS: return c->Cs;
  }
  return nullptr;
}

long long field_len(ss_case* c, int id) {
  if (id <= SS_W) return c->n_face[id];
  return c->n_cell;
}

const double* const* vel_of(ss_case* c, const double* out[3]) {
  out[0] = c->u; out[1] = c->v; out[2] = c->w;
  return out;
}

cudaEvent_t take_event(ss_case* c) {
  if (!c->pool->empty()) {
    cudaEvent_t e = c->pool->back();
    c->pool->pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// RAII timer around one stage: records an event pair when profiling is on
// and counts the kernels the stage launches.
struct StageTimer {
  ss_case* c;
  int id;
  cudaEvent_t a;
  StageTimer(ss_case* c_, int id_, int kernels) : c(c_), id(id_), a(nullptr) {
    c->launches[id] += kernels;
    if (c->profiling) {
      a = take_event(c);
      cudaEventRecord(a, c->stream);
    }
  }
  ~StageTimer() {
    if (a) {
      cudaEvent_t b = take_event(c);
      cudaEventRecord(b, c->stream);
      c->pending->push_back({id, {a, b}});
    }
  }
};

ss_status stage_assemble(ss_case* c, int sys) {
  StageTimer tm(c, SS_PROF_ASSEMBLE + (sys >= 0 && sys < SS_NSYS ? sys : 0), 1);
  const double* vel[3];
  vel_of(c, vel);
  cudaError_t e;
  switch (sys) {
    case SS_SYS_U:
    case SS_SYS_V:
    case SS_SYS_W:
      e = launch_assemble_momentum(sys, c->pr, c->sys[sys], vel, c->ustar[sys], c->p, c->T, c->Cl, c->Kinv, c->stream);
      break;
    case SS_SYS_P: {
      const double* us[3] = {c->ustar[0], c->ustar[1], c->ustar[2]};
      e = launch_poisson_rhs(c->pr, us, c->pb, c->stream);
      break;
    }
    case SS_SYS_C: e = launch_assemble_solute(c->pr, c->sys[sys], vel, c->gl, c->C, c->Ag, c->stream); break;
    case SS_SYS_T:
      // the solve starts from T^n + (T* - T^{n-1}) of the previous step; a
      // second assembly before the lever stage starts from T^n
      e = launch_assemble_temperature(c->pr, c->sys[sys], vel, &c->st->time, c->T, c->Tinc, !c->tinc_pending,
                                      c->stream);
      c->tinc_pending = 1;
      break;
    default: return fail(SS_EINVAL, "unknown system %d", sys);
  }
  if (e != cudaSuccess) return fail(SS_ECUDA, "assembly of system %d: %s", sys, cudaGetErrorString(e));
  return SS_OK;
}

// Relative tolerance of each FP32 inner solve of the mixed path (the outer
// FP64 refinement still stops on tol_p / tol_t). Measured at 128x96x96 with
// tol_p = 1e-10, tol_t = 1e-12: the MG-PCG reaches 1e-10 in two refinements
// of 3e-6 (14 inner iterations against 19 for three of 1e-5); the
// diffusion-dominated T* system needs fewer BiCGSTAB iterations with 1e-4
// per inner solve (18 against 24, still two refinements), while the
// momentum systems need a third refinement with 1e-4 and keep 1e-5.
constexpr double kInnerTolPressure = 3.0e-6;
constexpr double kInnerTolEnergy = 1.0e-4;
constexpr double kInnerTolTransport = 1.0e-5;

// The mixed T* solve starts with FP64 defect correction around the transform
// inverse of its constant-coefficient part I/dt - alpha L when the terms that
// inverse leaves out are small: every cooled wall's coefficient at most this
// fraction of 1/dt (Robin films in the workloads: ~0.4%; the half-cell
// Dirichlet walls of Example 2 are comparable to 1/dt and keep BiCGSTAB
// alone). Measured on the oracle's T* system at 64x48x48, a sweep reduces
// the residual by ~1.6e-3 (BiCGSTAB needed 16 inner iterations); three
// sweeps reach the benchmark tolerance from the T* initial guess. A fourth
// is allowed for the steps without that guess (the first one, and the first
// after a state write), where it costs less than the BiCGSTAB iterations
// that would finish the solve instead; the sweeps stop once the tolerance is
// met.
constexpr double kHelmholtzWallFraction = 0.05;
constexpr int kHelmholtzSweeps = 4;
// The transforms cost 2 (n_x + n_y) multiply-adds per cell and sweep: beyond
// this many modes three sweeps cost more than the BiCGSTAB iterations they
// replace (measured: 128 + 96 on the box, 0.58 -> 0.36 ms; 384 + 256 on the
// ingot, 8.1 -> 11.9 ms).
constexpr int kHelmholtzMaxModes = 320;

bool transform_energy_solve(const ss_case* c) {
  if (c->g.precision != SS_MIXED || !c->dct.tables || !c->dct.fp32) return false;
  if (c->pr.nx + (c->pr.dim == 3 ? c->pr.ny : 0) > kHelmholtzMaxModes) return false;
  for (int q = 0; q < 6; ++q)
    if (c->pr.wall_coef[q] > kHelmholtzWallFraction * c->pr.idt) return false;
  return true;
}

ss_status stage_solve(ss_case* c, int sys, bool fuse_project = false) {
  SolverCtl ctl;
  ctl.mixed = c->g.precision == SS_MIXED;
  ctl.block_cap = c->block_cap;
  ctl.stat_index = sys;
  ctl.inner_tol = sys == SS_SYS_P ? kInnerTolPressure : sys == SS_SYS_T ? kInnerTolEnergy : kInnerTolTransport;
  cudaError_t e;
  if (sys == SS_SYS_P) {
    ctl.tol = c->g.tol_p;
    ctl.max_it = c->g.max_it_p;
    // the correction of the previous step (zero in a new case and after
    // ss_set_fields) starts the mixed multigrid solve; the Jacobi and FP64
    // solves start from zero
    // (the FP64 transform solve converges in one sweep: a warm start would
    // only add a residual pass)
    ctl.warm_start = !(c->g.precond_p == SS_PRECOND_DCT && c->g.precision == SS_FP64);
    StageTimer tm(c, SS_PROF_SOLVE + sys, 1);
    if (c->g.precond_p == SS_PRECOND_MG)
      e = launch_pcg_mg(c->mg, c->pr, c->pb, c->pc, ctl, c->sc[0], c->st, c->stream);
    else if (c->g.precond_p == SS_PRECOND_DCT) {
      ProjectPtrs pj{{c->u, c->v, c->w}, {c->ustar[0], c->ustar[1], c->ustar[2]}, c->p};
      e = launch_poisson_dct(c->dct, c->pr, c->pb, c->pc, ctl, c->sc[0], c->st, fuse_project ? &pj : nullptr,
                             c->stream);
    }
    else
      e = launch_pcg_poisson(c->pr, c->pb, c->pc, ctl, c->sc[0], c->st, c->stream);
  } else if (sys >= 0 && sys < SS_NSYS) {
    if (sys == SS_SYS_W && c->pr.dim != 3) return SS_OK;
    ctl.tol = c->g.tol_t;
    ctl.max_it = c->g.max_it_t;
    ctl.jacobi = sys != SS_SYS_T;   // T* is diffusion-dominated: a Jacobi sweep gains little
    e = cudaSuccess;
    if (sys == SS_SYS_T && transform_energy_solve(c)) {
      ctl.after_presolve = 1;
      StageTimer pre(c, SS_PROF_PRESOLVE_T, 1);
      e = launch_helmholtz_dct(c->dct, c->pr, c->sys[sys], c->pr.dim == 3, kHelmholtzSweeps, ctl, c->sc[0], c->st,
                               c->stream);
    }
    if (e == cudaSuccess) {
      StageTimer tm(c, SS_PROF_SOLVE + sys, 1);
      e = launch_bicgstab(c->sys[sys], c->pr.dim == 3, ctl, c->sc[0], c->st, c->stream);
    }
  } else {
    return fail(SS_EINVAL, "unknown system %d", sys);
  }
  if (e != cudaSuccess) return fail(SS_ECUDA, "solve of system %d: %s", sys, cudaGetErrorString(e));
  return SS_OK;
}

ss_status stage_project(ss_case* c) {
  StageTimer tm(c, SS_PROF_PROJECT, 1);
  double* vel[3] = {c->u, c->v, c->w};
  const double* us[3] = {c->ustar[0], c->ustar[1], c->ustar[2]};
  cudaError_t e = launch_project(c->pr, vel, us, c->pc, c->p, c->stream);
  if (e != cudaSuccess) return fail(SS_ECUDA, "projection: %s", cudaGetErrorString(e));
  return SS_OK;
}

ss_status stage_lever(ss_case* c) {
  StageTimer tm(c, SS_PROF_LEVER, 1);
  cudaError_t e = launch_lever(c->pr, &c->st->time, c->T, c->gl, c->C, c->Cl, c->Cs, c->Kinv, c->Ag, c->Tinc,
                               c->tinc_pending, c->stream);
  c->tinc_pending = 0;
  if (e != cudaSuccess) return fail(SS_ECUDA, "lever update: %s", cudaGetErrorString(e));
  return SS_OK;
}

#define STAGE_TRY(expr)            \
  do {                             \
    ss_status s_ = (expr);         \
    if (s_ != SS_OK) return s_;    \
  } while (0)

// The u*, v*, w* systems of Eq. 3.3 are independent (each uses u^n only):
// one cooperative launch solves all of them, one team of blocks per
// component. Its time and its launch are counted under solve_u. Used where
// joint_momentum() says so.
ss_status stage_solve_momentum(ss_case* c) {
  StageTimer tm(c, SS_PROF_SOLVE + SS_SYS_U, 1);
  const int ncomp = c->pr.dim;
  SolverCtl ctl[kMaxTeams];
  const Sys* sys[kMaxTeams];
  Scratch* sc[kMaxTeams];
  for (int q = 0; q < ncomp; ++q) {
    ctl[q].mixed = c->g.precision == SS_MIXED;
    ctl[q].block_cap = c->block_cap;
    ctl[q].stat_index = q;
    ctl[q].inner_tol = kInnerTolTransport;
    ctl[q].tol = c->g.tol_t;
    ctl[q].max_it = c->g.max_it_t;
    ctl[q].jacobi = 1;
    sys[q] = &c->sys[q];
    sc[q] = &c->sc[q];
  }
  cudaError_t e = launch_bicgstab_multi(sys, ncomp, ncomp == 3, ctl, sc, c->st, c->stream);
  if (e != cudaSuccess) return fail(SS_ECUDA, "joint momentum solve: %s", cudaGetErrorString(e));
  return SS_OK;
}

// When the momentum systems are solved in one joint launch. Measured on the
// 1.2 M-cell box: mixed, 0.44 ms joint against 0.49 ms for three sequential
// solves (each solve is bound by its FP64 residual passes and its barriers;
// three teams overlap their barrier waits); FP64, 0.64 against ~0.9 ms. A
// case under a solver block cap (a batch or a server running cases side by
// side) gains ~10% from the joint launch, and so does a small case, whose
// solves are latency-bound. At 25 M cells the joint launch was 15% slower
// (each team streams its own vectors from HBM on a third of the SMs, and the
// team with the most iterations sets the time).
constexpr long long kJointMomentumMaxCells = 1LL << 22;

bool joint_momentum(const ss_case* c) { return c->n_cell <= kJointMomentumMaxCells; }

ss_status one_step(ss_case* c) {
  const int ncomp = c->pr.dim;
  if (joint_momentum(c)) {  // 1: intermediate velocity (Eq. 3.3)
    for (int a = 0; a < ncomp; ++a) STAGE_TRY(stage_assemble(c, a));
    STAGE_TRY(stage_solve_momentum(c));
  } else {
    for (int a = 0; a < ncomp; ++a) {
      STAGE_TRY(stage_assemble(c, a));
      STAGE_TRY(stage_solve(c, a));
    }
  }
  STAGE_TRY(stage_assemble(c, SS_SYS_P));     // 2: pressure correction (Eq. 3.4)
  if (c->g.precond_p == SS_PRECOND_DCT) {
    STAGE_TRY(stage_solve(c, SS_SYS_P, true)); // 3: the transform solve ends with the projection (Eq. 3.5)
  } else {
    STAGE_TRY(stage_solve(c, SS_SYS_P));
    STAGE_TRY(stage_project(c));              // 3: projection (Eq. 3.5)
  }
  STAGE_TRY(stage_assemble(c, SS_SYS_C));     // 4: solute (Eq. 3.10)
  STAGE_TRY(stage_solve(c, SS_SYS_C));
  STAGE_TRY(stage_assemble(c, SS_SYS_T));     // 5-6: T* (Eq. 3.12); T_l is formed in the lever stage
  STAGE_TRY(stage_solve(c, SS_SYS_T));
  STAGE_TRY(stage_lever(c));                  // 7-8: lever rule, T, g_l, C_l, C_s (Eq. 3.13-3.19)
  return SS_OK;
}

void drop_graph(ss_case* c) {
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
}

ss_status read_status(ss_case* c, DevStatus* host) {
  CUDA_TRY(cudaMemcpyAsync(host, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  CUDA_TRY(cudaMemsetAsync(&c->st->sticky, 0, sizeof(int), c->stream));
  CUDA_TRY(cudaMemsetAsync(&c->st->err, 0, sizeof(int), c->stream));
  if (host->err != kErrNone) return fail(SS_ETIMEOUT, "a device-side grid barrier timed out; the solve returned early");
  if (host->sticky == SS_ENAN) return fail(SS_ENAN, "a non-finite residual appeared in a solve");
  if (host->sticky == SS_ENOTCONV) return fail(SS_ENOTCONV, "a solve reached its iteration cap");
  return SS_OK;
}

}  // namespace

// ---------------------------------------------------------------- packed batches
//
// A batch steps many cases with one launch per stage of Algorithm 1: the
// assembly and pointwise stages take a packed list of (case, row tile) items,
// the solves one cooperative launch in which each case is solved by its own
// team of blocks (sized from its cells by the schedule). The batch's device
// tables live in a workspace the caller provides; the cases keep their own.
struct ss_batch {
  std::vector<ss_case*>* cases;
  cudaStream_t stream;
  char* ws;
  size_t ws_bytes;
  CaseRows* rows;                             // [n]
  char* bcg[3];                               // PackedBcgTeam [n]: momentum, solute, temperature
  char* dct;                                  // DctArgs<float> [n]
  char* helm;                                 // the T* pre-solve's arguments [n]
  int* first;                                 // [n + 1] first block of each team
  PackedTile* tiles[kNumPackedStages];
  int ntiles[kNumPackedStages];
  int cap_tiles[kNumPackedStages];
  std::vector<int>* team_blocks;              // host copy of the team sizes
  int max_blocks;                             // blocks one packed solve launch may keep resident
  int nblocks;                                // blocks of the packed solve launches
  size_t dct_smem;
  double gamma;                               // team size ~ cells^gamma
  int tile_rows;                              // rows per tile of the packed stages
  cudaGraphExec_t graph;
  long long launches;
};

namespace {

constexpr int kMinTileRows = 256;
constexpr int kPackedLaunchesPerStep = 10;
constexpr int kMaxTileRows = 1 << 24;

int stage_parts(int stage, const ss_case* c) { return stage == kStageMomentum ? c->pr.dim : 1; }

long long stage_tiles(int stage, const ss_case* c, int tile_rows) {
  long long t = 0;
  for (int part = 0; part < stage_parts(stage, c); ++part)
    t += (packed_stage_rows(stage, c->pr, part) + tile_rows - 1) / tile_rows;
  return t;
}

// Walk of the batch workspace (the same walk sizes it and places the tables).
template <class F>
size_t batch_layout(ss_case* const* cs, int n, char* base, F&& place) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += (bytes + 255) & ~(size_t)255;
    return p;
  };
  place(0, take((size_t)n * sizeof(CaseRows)));
  for (int q = 0; q < 3; ++q) place(1 + q, take((size_t)n * packed_bcg_team_bytes()));
  place(4, take((size_t)n * packed_dct_args_bytes()));
  place(5, take((size_t)(n + 1) * sizeof(int)));
  for (int st = 0; st < kNumPackedStages; ++st) {
    long long t = 0;
    for (int q = 0; q < n && st != kStageProject; ++q) t += stage_tiles(st, cs[q], kMinTileRows);
    place(6 + st, take((size_t)t * sizeof(PackedTile)));
  }
  place(6 + kNumPackedStages, take((size_t)n * packed_helm_args_bytes()));
  return off;
}

ss_status batch_check(ss_case* const* cs, int n) {
  if (!cs || n < 1) return fail(SS_EINVAL, "a batch needs at least one case");
  for (int q = 0; q < n; ++q) {
    const ss_case* c = cs[q];
    if (!c) return fail(SS_EINVAL, "case %d is NULL", q);
    if (!c->alloy_set) return fail(SS_ESTATE, "case %d: set_alloy first", q);
    if (c->g.precision != SS_MIXED || c->g.precond_p != SS_PRECOND_DCT)
      return fail(SS_EINVAL, "case %d: packed batches take SS_MIXED cases with the SS_PRECOND_DCT pressure solver", q);
    for (int r = 0; r < q; ++r)
      if (cs[r] == c) return fail(SS_EINVAL, "case %d appears twice", q);
  }
  return SS_OK;
}

// Team sizes (blocks per case) and row tiles for the current schedule, uploaded.
ss_status batch_schedule(ss_batch* b) {
  std::vector<ss_case*>& cs = *b->cases;
  const int n = (int)cs.size();
  std::vector<double> w(n);
  std::vector<long long> want(n);
  double wsum = 0.0;
  for (int q = 0; q < n; ++q) {
    w[q] = std::pow((double)cs[q]->n_cell, b->gamma);
    wsum += w[q];
    want[q] = blocks_wanted(cs[q]->n_cell);
  }
  std::vector<int>& blk = *b->team_blocks;
  blk.assign(n, 1);
  long long tot = 0;
  for (int q = 0; q < n; ++q) {
    long long v = (long long)std::floor((double)b->max_blocks * w[q] / wsum);
    blk[q] = (int)std::max(1LL, std::min(v, want[q]));
    tot += blk[q];
  }
  while (tot > b->max_blocks) {            // the floor of 1 block per case can overshoot
    int big = 0;
    for (int q = 1; q < n; ++q) if (blk[q] > blk[big]) big = q;
    if (blk[big] <= 1) return fail(SS_EINVAL, "%d cases exceed the %d resident blocks of a packed launch", n,
                                   b->max_blocks);
    --blk[big];
    --tot;
  }
  while (tot < b->max_blocks) {            // hand spare blocks to the case with most cells per block
    int best = -1;
    for (int q = 0; q < n; ++q)
      if (blk[q] < want[q] && (best < 0 || (double)cs[q]->n_cell / blk[q] > (double)cs[best]->n_cell / blk[best]))
        best = q;
    if (best < 0) break;
    ++blk[best];
    ++tot;
  }
  std::vector<int> first(n + 1, 0);
  for (int q = 0; q < n; ++q) first[q + 1] = first[q] + blk[q];
  b->nblocks = first[n];
  CUDA_TRY(cudaMemcpyAsync(b->first, first.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, b->stream));
  for (int st = 0; st < kNumPackedStages; ++st) {
    std::vector<PackedTile> t;
    for (int q = 0; q < n && st != kStageProject; ++q)   // the pressure solve projects
      for (int part = 0; part < stage_parts(st, cs[q]); ++part) {
        const long long rows = packed_stage_rows(st, cs[q]->pr, part);
        for (long long r0 = 0; r0 < rows; r0 += b->tile_rows)
          t.push_back({q, part, (int)r0, (int)std::min(rows, r0 + (long long)b->tile_rows)});
      }
    if ((int)t.size() > b->cap_tiles[st]) return fail(SS_EINVAL, "tile table of stage %d overflows", st);
    b->ntiles[st] = (int)t.size();
    if (!t.empty())
      CUDA_TRY(cudaMemcpyAsync(b->tiles[st], t.data(), t.size() * sizeof(PackedTile), cudaMemcpyHostToDevice,
                               b->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  return SS_OK;
}

ss_status batch_one_step(ss_batch* b) {
  const int n = (int)b->cases->size();
  cudaStream_t s = b->stream;
  cudaError_t e;
#define PACKED_TRY(expr)                                                              \
  do {                                                                                \
    if ((e = (expr)) != cudaSuccess) return fail(SS_ECUDA, "%s: %s", #expr, cudaGetErrorString(e)); \
  } while (0)
  PACKED_TRY(launch_packed_rows(kStageMomentum, b->rows, b->tiles[kStageMomentum], b->ntiles[kStageMomentum], s));
  PACKED_TRY(launch_bicgstab_packed(b->bcg[0], b->first, n, b->nblocks, s));
  PACKED_TRY(launch_packed_rows(kStageRhs, b->rows, b->tiles[kStageRhs], b->ntiles[kStageRhs], s));
  PACKED_TRY(launch_poisson_dct_packed(b->dct, b->first, n, b->nblocks, b->dct_smem, s));   // ends with Eq. 3.5
  PACKED_TRY(launch_packed_rows(kStageSolute, b->rows, b->tiles[kStageSolute], b->ntiles[kStageSolute], s));
  PACKED_TRY(launch_bicgstab_packed(b->bcg[1], b->first, n, b->nblocks, s));
  PACKED_TRY(launch_packed_rows(kStageTemperature, b->rows, b->tiles[kStageTemperature],
                                b->ntiles[kStageTemperature], s));
  PACKED_TRY(launch_helmholtz_dct_packed(b->helm, b->first, n, b->nblocks, b->dct_smem, s));
  PACKED_TRY(launch_bicgstab_packed(b->bcg[2], b->first, n, b->nblocks, s));
  PACKED_TRY(launch_packed_rows(kStageLever, b->rows, b->tiles[kStageLever], b->ntiles[kStageLever], s));
#undef PACKED_TRY
  b->launches += kPackedLaunchesPerStep;
  return SS_OK;
}

void batch_drop_graph(ss_batch* b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
}

}  // namespace

extern "C" {

const char* ss_last_error(void) { return g_err; }

ss_status ss_workspace_bytes(const ss_grid* grid, size_t* bytes) {
  char why[256];
  if (!bytes) return fail(SS_EINVAL, "bytes is NULL");
  if (!grid_ok(grid, why, sizeof why)) return fail(SS_EINVAL, "%s", why);
  ss_case tmp;
  memset(&tmp, 0, sizeof tmp);
  tmp.g = *grid;
  Planner pl(nullptr, guard_of(grid));
  plan(&tmp, pl);
  *bytes = pl.off;
  return SS_OK;
}

ss_status ss_create_case(const ss_grid* grid, void* workspace, size_t workspace_bytes, void* stream, ss_case** out) {
  char why[256];
  if (!out) return fail(SS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!grid_ok(grid, why, sizeof why)) return fail(SS_EINVAL, "%s", why);
  if (!workspace) return fail(SS_EINVAL, "workspace is NULL");
  if (((uintptr_t)workspace & 255) != 0) return fail(SS_EINVAL, "workspace must be 256-byte aligned");
  size_t need = 0;
  ss_status s = ss_workspace_bytes(grid, &need);
  if (s != SS_OK) return s;
  if (workspace_bytes < need) return fail(SS_ENOMEM, "workspace has %zu bytes, needs %zu", workspace_bytes, need);
  ss_case* c = new (std::nothrow) ss_case;
  if (!c) return fail(SS_ENOMEM, "host allocation failed");
  memset(c, 0, sizeof *c);
  c->g = *grid;
  if (c->g.dim == 2) c->g.nz = 1;
  c->pool = new (std::nothrow) std::vector<cudaEvent_t>();
  c->pending = new (std::nothrow) std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>>();
  if (!c->pool || !c->pending) {
    delete c->pool;
    delete c->pending;
    delete c;
    return fail(SS_ENOMEM, "host allocation failed");
  }
  c->stream = (cudaStream_t)stream;
  c->ws = (char*)workspace;
  c->ws_bytes = workspace_bytes;
  Planner pl(c->ws, guard_of(grid));
  plan(c, pl);
  fill_params(c, nullptr);
  cudaError_t e = cudaMemsetAsync(c->ws, 0, need, c->stream);   // zero fields and guard bands
  if (e == cudaSuccess && c->mg.cinv) {
    const size_t nn = (size_t)c->cinv_n * c->cinv_n;
    const void* src = c->cinv_host;
    if (c->mg.fp32) {
      for (size_t q = 0; q < nn; ++q) c->cinv_host32[q] = (float)c->cinv_host[q];
      src = c->cinv_host32;
    }
    e = cudaMemcpyAsync(c->mg.cinv, src, nn * (c->mg.fp32 ? sizeof(float) : sizeof(double)), cudaMemcpyHostToDevice,
                        c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  }
  if (e == cudaSuccess && c->dct.tables) {
    // cosine matrices and eigenvalues of the transform solver, formed in FP64 on the host
    std::vector<double> tab(dct_table_elems(c->dct));
    dct_tables(c->dct, c->pr, tab.data());
    std::vector<float> tab32;
    const void* src = tab.data();
    size_t bytes = tab.size() * sizeof(double);
    if (c->dct.fp32) {
      tab32.assign(tab.begin(), tab.end());
      src = tab32.data();
      bytes = tab32.size() * sizeof(float);
    }
    e = cudaMemcpyAsync(c->dct.tables, src, bytes, cudaMemcpyHostToDevice, c->stream);
    std::vector<unsigned char> img;
    if (e == cudaSuccess && c->dct.img) {
      // the constant operands of the tensor-core transforms, staged once
      img.resize(dct_image_bytes(c->dct));
      dct_images(c->dct, tab32.data(), tab32.data() + (size_t)c->dct.Mx * c->dct.Mx, img.data());
      e = cudaMemcpyAsync(c->dct.img, img.data(), img.size(), cudaMemcpyHostToDevice, c->stream);
    }
    // the slab solves' factorisations, formed from the tables just copied
    if (e == cudaSuccess) e = dct_thomas_ensure(c->dct, c->pr, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  }
  if (e != cudaSuccess) {
    delete c->pool;
    delete c->pending;
    delete c;
    return fail(SS_ECUDA, "workspace clear: %s", cudaGetErrorString(e));
  }
  *out = c;
  return SS_OK;
}

ss_status ss_set_alloy(ss_case* c, const ss_alloy* al) {
  STAGE_TRY(check_case(c));
  drop_graph(c);
  if (!al) return fail(SS_EINVAL, "alloy is NULL");
  if (c->steps > 0) return fail(SS_ESTATE, "set_alloy after the first step");
  if (!(al->kp > 0 && al->kp < 1)) return fail(SS_EINVAL, "kp must be in (0, 1)");
  if (!(al->rho > 0 && al->k > 0 && al->cp > 0 && al->L > 0 && al->mu > 0 && al->K0 > 0 && al->darcy_eps > 0))
    return fail(SS_EINVAL, "rho, k, cp, L, mu, K0, darcy_eps must be > 0");
  if (al->Dl < 0) return fail(SS_EINVAL, "Dl must be >= 0");
  c->alloy_set = 1;
  fill_params(c, al);
  CUDA_TRY(dct_thomas_ensure(c->dct, c->pr, c->stream));   // the T* operator's shift depends on the alloy
  const long long nf[3] = {c->n_face[0], c->n_face[1], c->n_face[2]};
  CUDA_TRY(cudaMemsetAsync(c->u, 0, nf[0] * sizeof(double), c->stream));
  CUDA_TRY(cudaMemsetAsync(c->v, 0, nf[1] * sizeof(double), c->stream));
  CUDA_TRY(cudaMemsetAsync(c->w, 0, nf[2] * sizeof(double), c->stream));
  CUDA_TRY(cudaMemsetAsync(c->p, 0, c->n_cell * sizeof(double), c->stream));
  CUDA_TRY(cudaMemsetAsync(c->Tinc, 0, c->n_cell * sizeof(double), c->stream));
  c->tinc_pending = 0;
  k_fill<<<256, 256, 0, c->stream>>>(c->T, al->Tref, c->n_cell);
  k_fill<<<256, 256, 0, c->stream>>>(c->C, al->C0, c->n_cell);
  CUDA_TRY(cudaGetLastError());
  return ss_equilibrate(c);
}

ss_status ss_set_boundary(ss_case* c, int face, const ss_bc* bc) {
  STAGE_TRY(check_case(c));
  drop_graph(c);
  if (!bc) return fail(SS_EINVAL, "bc is NULL");
  if (face < 0 || face > 5) return fail(SS_EINVAL, "face must be 0..5");
  if (bc->thermal != SS_ADIABATIC && bc->thermal != SS_ROBIN && bc->thermal != SS_DIRICHLET)
    return fail(SS_EINVAL, "unknown thermal condition");
  if (bc->thermal == SS_ROBIN && !(bc->h > 0)) return fail(SS_EINVAL, "Robin h must be > 0");
  if (bc->flow != SS_NOSLIP && bc->flow != SS_FREESLIP) return fail(SS_EINVAL, "unknown flow condition");
  if (!std::isfinite(bc->Text) || !std::isfinite(bc->dTdt)) return fail(SS_EINVAL, "wall temperature not finite");
  c->bc[face] = *bc;
  fill_params(c, nullptr);
  return SS_OK;
}

ss_status ss_step(ss_case* c, int n) {
  STAGE_TRY(check_case(c));
  if (n < 0) return fail(SS_EINVAL, "n must be >= 0");
  if (!c->alloy_set) return fail(SS_ESTATE, "set_alloy before stepping");
  for (int q = 0; q < n; ++q) {
    STAGE_TRY(one_step(c));
    c->steps++;
  }
  return SS_OK;
}

ss_status ss_step_graph(ss_case* c, int n) {
  STAGE_TRY(check_case(c));
  if (n < 0) return fail(SS_EINVAL, "n must be >= 0");
  if (!c->alloy_set) return fail(SS_ESTATE, "set_alloy before stepping");
  if (c->stream == nullptr) return fail(SS_EINVAL, "graph steps need a non-default stream");
  if (!c->graph) {
    const int prof = c->profiling;
    long long before = 0;
    for (int q = 0; q < SS_NPROF; ++q) before += c->launches[q];
    c->profiling = 0;
    CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    ss_status s = one_step(c);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    c->profiling = prof;
    long long after = 0;
    for (int q = 0; q < SS_NPROF; ++q) after += c->launches[q];
    c->graph_kernels = after - before;
    for (int q = 0; q < SS_NPROF; ++q) c->launches[q] = 0;   // capture launched nothing
    c->launches[SS_PROF_SOLVE + SS_SYS_P] = 0;
    if (s != SS_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) return fail(SS_ECUDA, "step capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      c->graph = nullptr;
      return fail(SS_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
  }
  for (int q = 0; q < n; ++q) {
    CUDA_TRY(cudaGraphLaunch(c->graph, c->stream));
    c->steps++;
  }
  c->launches[SS_PROF_SOLVE + SS_SYS_P] += c->graph_kernels * n;   // counted under one stage
  return SS_OK;
}

ss_status ss_sync(ss_case* c) {
  STAGE_TRY(check_case(c));
  DevStatus h;
  return read_status(c, &h);
}

ss_status ss_get_fields(ss_case* c, unsigned mask, void* const* dst, int dst_is_device) {
  STAGE_TRY(check_case(c));
  if (!dst) return fail(SS_EINVAL, "dst is NULL");
  for (int id = 0; id < SS_NFIELDS; ++id) {
    if (!(mask & (1u << id))) continue;
    if (id == SS_W && c->pr.dim != 3) continue;
    if (!dst[id]) return fail(SS_EINVAL, "dst[%d] is NULL", id);
    CUDA_TRY(cudaMemcpyAsync(dst[id], field_ptr(c, id), field_len(c, id) * sizeof(double),
                             dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  }
  if (!dst_is_device) CUDA_TRY(cudaStreamSynchronize(c->stream));   // device copies stay stream-ordered
  return SS_OK;
}

ss_status ss_set_fields(ss_case* c, unsigned mask, const void* const* src, int src_is_device) {
  STAGE_TRY(check_case(c));
  if (!src) return fail(SS_EINVAL, "src is NULL");
  for (int id = 0; id < SS_NFIELDS; ++id) {
    if (!(mask & (1u << id))) continue;
    if (id == SS_W && c->pr.dim != 3) continue;
    if (!src[id]) return fail(SS_EINVAL, "src[%d] is NULL", id);
    CUDA_TRY(cudaMemcpyAsync(field_ptr(c, id), src[id], field_len(c, id) * sizeof(double),
                             src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  }
  // a new state clears the pressure solve's warm start, so the next step
  // depends on the state alone (as in a new case)
  CUDA_TRY(cudaMemsetAsync(c->pc, 0, c->n_cell * sizeof(double), c->stream));
  // and the T* initial guess's increment, for the same reason
  CUDA_TRY(cudaMemsetAsync(c->Tinc, 0, c->n_cell * sizeof(double), c->stream));
  c->tinc_pending = 0;
  if ((mask & (1u << SS_GL)) && c->alloy_set) {
    // keep K^{-1} and A_g consistent with the new g_l; C_l and C_s stay as they are
    cudaError_t e = launch_equilibrate(c->pr, c->T, c->C, c->gl, c->Cl, c->Cs, c->Kinv, c->Ag, 0, 0, c->stream);
    if (e != cudaSuccess) return fail(SS_ECUDA, "derived fields: %s", cudaGetErrorString(e));
  }
  if (!src_is_device) CUDA_TRY(cudaStreamSynchronize(c->stream));
  return SS_OK;
}

ss_status ss_equilibrate(ss_case* c) {
  STAGE_TRY(check_case(c));
  if (!c->alloy_set) return fail(SS_ESTATE, "set_alloy first");
  cudaError_t e = launch_equilibrate(c->pr, c->T, c->C, c->gl, c->Cl, c->Cs, c->Kinv, c->Ag, 1, 1, c->stream);
  if (e != cudaSuccess) return fail(SS_ECUDA, "equilibrate: %s", cudaGetErrorString(e));
  return SS_OK;
}

ss_status ss_set_block_cap(ss_case* c, int max_blocks) {
  STAGE_TRY(check_case(c));
  if (max_blocks < 0) return fail(SS_EINVAL, "max_blocks must be >= 0");
  drop_graph(c);   // launch configurations are part of a captured step
  c->block_cap = max_blocks;
  return SS_OK;
}

ss_status ss_set_tensor_cores(ss_case* c, int mode) {
  STAGE_TRY(check_case(c));
  if (mode != SS_TC_AUTO && mode != SS_TC_ON && mode != SS_TC_OFF) return fail(SS_EINVAL, "unknown mode %d", mode);
  drop_graph(c);   // launch configurations are part of a captured step
  c->dct.tc_mode = mode;
  return SS_OK;
}

ss_status ss_set_time(ss_case* c, double t) {
  STAGE_TRY(check_case(c));
  if (!std::isfinite(t)) return fail(SS_EINVAL, "time must be finite");
  k_fill<<<1, 32, 0, c->stream>>>(&c->st->time, t, 1);
  CUDA_TRY(cudaGetLastError());
  return SS_OK;
}

ss_status ss_get_time(ss_case* c, double* t) {
  STAGE_TRY(check_case(c));
  if (!t) return fail(SS_EINVAL, "t is NULL");
  CUDA_TRY(cudaMemcpyAsync(t, &c->st->time, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return SS_OK;
}

ss_status ss_get_stats(ss_case* c, ss_stats* out) {
  STAGE_TRY(check_case(c));
  if (!out) return fail(SS_EINVAL, "out is NULL");
  DevStatus h;
  ss_status s = read_status(c, &h);
  out->steps = c->steps;
  for (int q = 0; q < SS_NSYS; ++q) {
    out->iters[q] = h.stat[q].iters;
    out->refinements[q] = h.stat[q].refinements;
    out->relres[q] = h.stat[q].relres;
    out->jacobi[q] = h.stat[q].jacobi;
  }
  out->status = (s == SS_OK) ? SS_OK : (int)s;
  return s;
}

ss_status ss_set_profiling(ss_case* c, int on) {
  STAGE_TRY(check_case(c));
  c->profiling = on ? 1 : 0;
  return SS_OK;
}

ss_status ss_get_profile(ss_case* c, ss_profile* out) {
  STAGE_TRY(check_case(c));
  if (!out) return fail(SS_EINVAL, "out is NULL");
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  memset(out, 0, sizeof *out);
  for (auto& pe : *c->pending) {
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, pe.second.first, pe.second.second));
    out->ms[pe.first] += ms;
    c->pool->push_back(pe.second.first);
    c->pool->push_back(pe.second.second);
  }
  c->pending->clear();
  for (int q = 0; q < SS_NPROF; ++q) {
    out->launches[q] = c->launches[q];
    out->kernels += c->launches[q];
    c->launches[q] = 0;
  }
  DevStatus h;
  CUDA_TRY(cudaMemcpy(&h, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost));
  for (int s = 0; s < SS_NSYS; ++s) {
    out->iters[s] = h.stat[s].iters_total;
    out->jacobi[s] = h.stat[s].jacobi_total;
    CUDA_TRY(cudaMemsetAsync(&c->st->stat[s].iters_total, 0, 2 * sizeof(long long), c->stream));
  }
  out->presolve_sweeps = h.presolve_sweeps;
  CUDA_TRY(cudaMemsetAsync(&c->st->presolve_sweeps, 0, sizeof(long long), c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return SS_OK;
}

ss_status ss_destroy(ss_case* c) {
  if (!c) return SS_OK;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  for (auto& pe : *c->pending) {
    cudaEventDestroy(pe.second.first);
    cudaEventDestroy(pe.second.second);
  }
  for (auto ev : *c->pool) cudaEventDestroy(ev);
  drop_graph(c);
  delete c->pool;
  delete c->pending;
  delete c;
  if (e != cudaSuccess) return fail(SS_ECUDA, "destroy: %s", cudaGetErrorString(e));
  return SS_OK;
}

ss_status ss_assemble(ss_case* c, int sys) {
  STAGE_TRY(check_case(c));
  if (!c->alloy_set) return fail(SS_ESTATE, "set_alloy first");
  if (sys == SS_SYS_W && c->pr.dim != 3) return fail(SS_EINVAL, "no w system in 2D");
  return stage_assemble(c, sys);
}

ss_status ss_solve(ss_case* c, int sys) {
  STAGE_TRY(check_case(c));
  if (!c->alloy_set) return fail(SS_ESTATE, "set_alloy first");
  if (sys == SS_SYS_W && c->pr.dim != 3) return fail(SS_EINVAL, "no w system in 2D");
  STAGE_TRY(stage_solve(c, sys));
  return ss_sync(c);
}

ss_status ss_get_system(ss_case* c, int sys, void* const* dst, int dst_is_device) {
  STAGE_TRY(check_case(c));
  if (!dst) return fail(SS_EINVAL, "dst is NULL");
  if (sys < 0 || sys >= SS_NSYS) return fail(SS_EINVAL, "unknown system %d", sys);
  const Sys& S = c->sys[sys];
  const double* src[9] = {S.a.P, S.a.W, S.a.E, S.a.S, S.a.N, S.a.B, S.a.T_, S.b, S.x};
  const cudaMemcpyKind kind = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  for (int q = 0; q < 9; ++q) {
    if (!dst[q]) continue;
    if (sys == SS_SYS_P && q < 7) continue;
    if ((q == 5 || q == 6) && c->pr.dim != 3) {   // no z diagonals in 2D
      if (dst_is_device) CUDA_TRY(cudaMemsetAsync(dst[q], 0, S.d.n * sizeof(double), c->stream));
      else memset(dst[q], 0, S.d.n * sizeof(double));
      continue;
    }
    CUDA_TRY(cudaMemcpyAsync(dst[q], src[q], S.d.n * sizeof(double), kind, c->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return SS_OK;
}

ss_status ss_assemble_forward(ss_case* c, int sys) {
  STAGE_TRY(check_case(c));
  if (!c->alloy_set) return fail(SS_ESTATE, "set_alloy first");
  if (sys < 0 || sys >= SS_NSYS || sys == SS_SYS_P) return fail(SS_EINVAL, "system %d has no planes to assemble", sys);
  if (sys == SS_SYS_W && c->pr.dim != 3) return fail(SS_EINVAL, "no w system in 2D");
  const double* vel[3];
  vel_of(c, vel);
  cudaError_t e = launch_forward_assemble(sys, c->pr, c->sys[sys], vel, c->p, c->T, c->C, c->Cl, c->gl, c->Kinv,
                                          c->Ag, &c->st->time, c->stream);
  if (e != cudaSuccess) return fail(SS_ECUDA, "forward assembly of system %d: %s", sys, cudaGetErrorString(e));
  if (sys <= SS_SYS_W) {   // the predictor's initial guess, as the term-wise assembly sets it
    const long long nf = c->n_face[sys];
    CUDA_TRY(cudaMemcpyAsync(c->ustar[sys], vel[sys], nf * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  }
  return SS_OK;
}

ss_status ss_get_system_f32(ss_case* c, int sys, void* const* dst, int dst_is_device) {
  STAGE_TRY(check_case(c));
  if (!dst) return fail(SS_EINVAL, "dst is NULL");
  if (sys < 0 || sys >= SS_NSYS) return fail(SS_EINVAL, "unknown system %d", sys);
  if (sys == SS_SYS_P) return fail(SS_EINVAL, "the pressure system has no planes");
  const Sys& S = c->sys[sys];
  if (!S.af.P) return fail(SS_ESTATE, "FP32 planes exist in SS_MIXED cases only");
  const float* src[8] = {S.af.P, S.af.W, S.af.E, S.af.S, S.af.N, S.af.B, S.af.T_, S.af.idiag};
  const cudaMemcpyKind kind = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  for (int q = 0; q < 8; ++q) {
    if (!dst[q]) continue;
    if ((q == 5 || q == 6) && c->pr.dim != 3) {
      if (dst_is_device) CUDA_TRY(cudaMemsetAsync(dst[q], 0, S.d.n * sizeof(float), c->stream));
      else memset(dst[q], 0, S.d.n * sizeof(float));
      continue;
    }
    CUDA_TRY(cudaMemcpyAsync(dst[q], src[q], S.d.n * sizeof(float), kind, c->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return SS_OK;
}

ss_status ss_convert_f64_to_f32(const double* src, float* dst, long long n, void* stream) {
  if (n < 0) return fail(SS_EINVAL, "n must be >= 0");
  if (n > 0 && (!src || !dst)) return fail(SS_EINVAL, "src/dst is NULL");
  if (n == 0) return SS_OK;
  cudaError_t e = launch_to_f32(src, dst, n, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(SS_ECUDA, "convert: %s", cudaGetErrorString(e));
  return SS_OK;
}

ss_status ss_set_wait_limit(ss_case* c, long long polls) {
  STAGE_TRY(check_case(c));
  if (polls < 0 || polls > kMaxSpinLimit)
    return fail(SS_EINVAL, "polls must be in [0, %lld] (0: the default)", kMaxSpinLimit);
  k_set_spin_limit<<<1, 1, 0, c->stream>>>(c->st, polls);
  CUDA_TRY(cudaGetLastError());
  return SS_OK;
}

ss_status ss_wait_selftest(ss_case* c) {
  STAGE_TRY(check_case(c));
  CUDA_TRY(cudaMemsetAsync(&c->st->selftest_counter, 0, sizeof(unsigned int), c->stream));
  k_wait_selftest<<<1, 32, 0, c->stream>>>(c->st);
  CUDA_TRY(cudaGetLastError());
  return SS_OK;
}

ss_status ss_tc_selftest(ss_case* c, const float* a, const float* b, float* d, int n, int k, int transposed) {
  STAGE_TRY(check_case(c));
  if (!a || !b || !d) return fail(SS_EINVAL, "a, b and d must be device pointers");
  if (n < 16 || n > 256 || n % 16 != 0) return fail(SS_EINVAL, "n = %d: need a multiple of 16 in [16, 256]", n);
  if (k < 1 || k > 4096) return fail(SS_EINVAL, "k = %d: need 1 <= k <= 4096", k);
  CUDA_TRY(launch_tc_selftest(a, b, d, n, k, transposed ? 1 : 0, c->st, c->stream));
  return SS_OK;
}

ss_status ss_batch_workspace_bytes(ss_case* const* cases, int n, size_t* bytes) {
  if (!bytes) return fail(SS_EINVAL, "bytes is NULL");
  STAGE_TRY(batch_check(cases, n));
  *bytes = batch_layout(cases, n, nullptr, [](int, char*) {});
  return SS_OK;
}

ss_status ss_batch_create(ss_case* const* cases, int n, void* workspace, size_t workspace_bytes, void* stream,
                          ss_batch** out) {
  if (!out) return fail(SS_EINVAL, "out is NULL");
  *out = nullptr;
  size_t need = 0;
  STAGE_TRY(ss_batch_workspace_bytes(cases, n, &need));
  if (!workspace) return fail(SS_EINVAL, "workspace is NULL");
  if (((uintptr_t)workspace & 255) != 0) return fail(SS_EINVAL, "workspace must be 256-byte aligned");
  if (workspace_bytes < need) return fail(SS_ENOMEM, "batch workspace has %zu bytes, needs %zu", workspace_bytes, need);
  ss_batch* b = new (std::nothrow) ss_batch;
  if (!b) return fail(SS_ENOMEM, "host allocation failed");
  memset(b, 0, sizeof *b);
  b->cases = new (std::nothrow) std::vector<ss_case*>(cases, cases + n);
  b->team_blocks = new (std::nothrow) std::vector<int>();
  if (!b->cases || !b->team_blocks) {
    delete b->cases;
    delete b->team_blocks;
    delete b;
    return fail(SS_ENOMEM, "host allocation failed");
  }
  b->stream = (cudaStream_t)stream;
  b->ws = (char*)workspace;
  b->ws_bytes = workspace_bytes;
  b->gamma = 1.0;
  b->tile_rows = 4096;
  char* slot[7 + kNumPackedStages] = {nullptr};
  batch_layout(cases, n, b->ws, [&](int k, char* p) { slot[k] = p; });
  b->rows = reinterpret_cast<CaseRows*>(slot[0]);
  for (int q = 0; q < 3; ++q) b->bcg[q] = slot[1 + q];
  b->dct = slot[4];
  b->helm = slot[6 + kNumPackedStages];
  b->first = reinterpret_cast<int*>(slot[5]);
  for (int st = 0; st < kNumPackedStages; ++st) {
    b->tiles[st] = reinterpret_cast<PackedTile*>(slot[6 + st]);
    long long t = 0;
    for (int q = 0; q < n && st != kStageProject; ++q) t += stage_tiles(st, cases[q], kMinTileRows);
    b->cap_tiles[st] = (int)t;
  }
  // per-case descriptions and solver arguments, built on the host once
  const size_t bt = packed_bcg_team_bytes(), da = packed_dct_args_bytes();
  std::vector<CaseRows> rows(n);
  const size_t ha = packed_helm_args_bytes();
  std::vector<char> bcg(3 * (size_t)n * bt), dct((size_t)n * da), helm((size_t)n * ha);
  b->dct_smem = 0;
  for (int q = 0; q < n; ++q) {
    ss_case* c = cases[q];
    CaseRows& r = rows[q];
    memset(&r, 0, sizeof r);
    r.pr = c->pr;
    for (int k = 0; k < SS_NSYS; ++k) r.sys[k] = c->sys[k];
    r.u = c->u; r.v = c->v; r.w = c->w; r.p = c->p; r.T = c->T; r.C = c->C; r.gl = c->gl; r.Cl = c->Cl;
    r.Cs = c->Cs; r.Kinv = c->Kinv; r.Ag = c->Ag; r.pc = c->pc; r.pb = c->pb; r.Tinc = c->Tinc;
    for (int a = 0; a < 3; ++a) r.ustar[a] = c->ustar[a];
    r.st = c->st;
    SolverCtl ctl[3];
    const Sys* sys[3];
    for (int a = 0; a < c->pr.dim; ++a) {
      ctl[a].mixed = 1; ctl[a].block_cap = 0; ctl[a].stat_index = a; ctl[a].inner_tol = kInnerTolTransport;
      ctl[a].tol = c->g.tol_t; ctl[a].max_it = c->g.max_it_t; ctl[a].jacobi = 1;
      sys[a] = &c->sys[a];
    }
    fill_packed_bcg_team(&bcg[(0 * (size_t)n + q) * bt], sys, c->pr.dim, c->pr.dim == 3, ctl, c->sc[0], c->st);
    SolverCtl cc = ctl[0];
    cc.stat_index = SS_SYS_C;
    sys[0] = &c->sys[SS_SYS_C];
    fill_packed_bcg_team(&bcg[(1 * (size_t)n + q) * bt], sys, 1, c->pr.dim == 3, &cc, c->sc[0], c->st);
    SolverCtl ct = ctl[0];
    ct.stat_index = SS_SYS_T;
    ct.inner_tol = kInnerTolEnergy;
    ct.after_presolve = transform_energy_solve(c) ? 1 : 0;
    ct.jacobi = 0;
    sys[0] = &c->sys[SS_SYS_T];
    fill_packed_bcg_team(&bcg[(2 * (size_t)n + q) * bt], sys, 1, c->pr.dim == 3, &ct, c->sc[0], c->st);
    SolverCtl cp;
    cp.mixed = 1; cp.block_cap = 0; cp.stat_index = SS_SYS_P; cp.inner_tol = kInnerTolPressure;
    cp.warm_start = 1;
    cp.tol = c->g.tol_p; cp.max_it = c->g.max_it_p;
    ProjectPtrs pj{{c->u, c->v, c->w}, {c->ustar[0], c->ustar[1], c->ustar[2]}, c->p};
    const size_t sm = fill_packed_dct_args(&dct[(size_t)q * da], c->dct, c->pr, c->pb, c->pc, cp, c->sc[0], c->st, &pj);
    b->dct_smem = std::max(b->dct_smem, sm);
    const size_t hm = fill_packed_helm_args(&helm[(size_t)q * ha], c->dct, c->pr, c->sys[SS_SYS_T], c->pr.dim == 3,
                                            transform_energy_solve(c) ? kHelmholtzSweeps : 0, ct, c->sc[0], c->st);
    b->dct_smem = std::max(b->dct_smem, hm);
  }
  const int lim_d = std::min(packed_dct_max_blocks(b->dct_smem), packed_helm_max_blocks(b->dct_smem));
  b->max_blocks = std::min(packed_bcg_max_blocks(), lim_d);
  for (int q = 0; q < n; ++q) b->max_blocks = std::min(b->max_blocks, cases[q]->sc[0].max_blocks);
  cudaError_t e = cudaSuccess;
  for (int q = 0; q < n && e == cudaSuccess; ++q) e = cudaStreamSynchronize(cases[q]->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->rows, rows.data(), n * sizeof(CaseRows), cudaMemcpyHostToDevice, b->stream);
  for (int q = 0; q < 3 && e == cudaSuccess; ++q)
    e = cudaMemcpyAsync(b->bcg[q], &bcg[(size_t)q * n * bt], n * bt, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->dct, dct.data(), n * da, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->helm, helm.data(), n * ha, cudaMemcpyHostToDevice, b->stream);
  ss_status s = SS_OK;
  if (e != cudaSuccess) s = fail(SS_ECUDA, "batch tables: %s", cudaGetErrorString(e));
  else if (b->max_blocks < n) s = fail(SS_EINVAL, "%d cases exceed the %d resident blocks of a packed launch", n,
                                       b->max_blocks);
  else s = batch_schedule(b);
  if (s != SS_OK) {
    delete b->cases;
    delete b->team_blocks;
    delete b;
    return s;
  }
  *out = b;
  return SS_OK;
}

ss_status ss_batch_set_schedule(ss_batch* b, double gamma, int tile_rows) {
  if (!b) return fail(SS_EINVAL, "batch is NULL");
  if (!(gamma >= 0.0 && gamma <= 2.0)) return fail(SS_EINVAL, "gamma must be in [0, 2]");
  if (tile_rows < kMinTileRows || tile_rows > kMaxTileRows)
    return fail(SS_EINVAL, "tile_rows must be in [%d, %d]", kMinTileRows, kMaxTileRows);
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  batch_drop_graph(b);
  b->gamma = gamma;
  b->tile_rows = tile_rows;
  return batch_schedule(b);
}

ss_status ss_batch_get_teams(ss_batch* b, int* blocks) {
  if (!b || !blocks) return fail(SS_EINVAL, "batch or blocks is NULL");
  for (size_t q = 0; q < b->team_blocks->size(); ++q) blocks[q] = (*b->team_blocks)[q];
  return SS_OK;
}

ss_status ss_batch_step(ss_batch* b, int n) {
  if (!b) return fail(SS_EINVAL, "batch is NULL");
  if (n < 0) return fail(SS_EINVAL, "n must be >= 0");
  if (n == 0) return SS_OK;
  if (b->stream == nullptr) {                  // the legacy default stream cannot be captured
    for (int k = 0; k < n; ++k) STAGE_TRY(batch_one_step(b));
  } else {
    if (!b->graph) {
      const long long before = b->launches;
      CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      ss_status s = batch_one_step(b);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(b->stream, &g);
      b->launches = before;                    // the capture launched nothing
      if (s != SS_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
      }
      if (e != cudaSuccess) return fail(SS_ECUDA, "batch capture: %s", cudaGetErrorString(e));
      e = cudaGraphInstantiate(&b->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        b->graph = nullptr;
        return fail(SS_ECUDA, "batch graph instantiate: %s", cudaGetErrorString(e));
      }
    }
    for (int k = 0; k < n; ++k) CUDA_TRY(cudaGraphLaunch(b->graph, b->stream));
    b->launches += (long long)kPackedLaunchesPerStep * n;
  }
  for (ss_case* c : *b->cases) {
    c->steps += n;
    c->tinc_pending = 0;
  }
  return SS_OK;
}

ss_status ss_batch_sync(ss_batch* b, long long* launches) {
  if (!b) return fail(SS_EINVAL, "batch is NULL");
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  if (launches) *launches = b->launches;
  ss_status worst = SS_OK;
  char msg[512] = "";
  for (ss_case* c : *b->cases) {
    DevStatus h;
    ss_status s = read_status(c, &h);
    if (s != SS_OK && (worst == SS_OK || s > worst)) {
      worst = s;
      snprintf(msg, sizeof msg, "%s", g_err);
    }
  }
  if (worst != SS_OK) return fail(worst, "%s", msg);
  return SS_OK;
}

ss_status ss_batch_destroy(ss_batch* b) {
  if (!b) return SS_OK;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  batch_drop_graph(b);
  delete b->cases;
  delete b->team_blocks;
  delete b;
  if (e != cudaSuccess) return fail(SS_ECUDA, "batch destroy: %s", cudaGetErrorString(e));
  return SS_OK;
}

ss_status ss_project(ss_case* c) {
  STAGE_TRY(check_case(c));
  return stage_project(c);
}

ss_status ss_lever(ss_case* c) {
  STAGE_TRY(check_case(c));
  if (!c->alloy_set) return fail(SS_ESTATE, "set_alloy first");
  return stage_lever(c);
}

}  // extern "C"
