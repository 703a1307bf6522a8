// Term-wise assembly of the DIA systems and the pointwise stages of one step.
//
//   k_assemble_momentum<A>   rows of the intermediate-velocity system for
//                            component A (Eq. 3.3 with the momentum form Eq. 2.7)
//   k_assemble_cells<SOLUTE> solute system (Eq. 3.6-3.10) or T* system (Eq. 3.12)
//   k_poisson_rhs            -(rho/dt) div u* (Eq. 3.4)
//   k_project                u^{n+1} = u* - (dt/rho) grad p', p += p' (Eq. 3.5)
//   k_lever                  latent-heat correction and quadratic lever rule
//                            (Eq. 3.13-3.19), plus K^{-1} (Eq. 2.8) and A_g
//                            (Eq. 3.8) for the next step
//   k_equilibrate            equilibrium g_l, C_l, C_s of given (T, C) (Eq. 3.15, 3.18-3.19)
//
// One thread per row, grid-stride. Each row is written once with coalesced
// stores (consecutive threads own consecutive x). The constant diffusion
// parts of the stencils (Sec. 4, term-wise strategy) are launch constants;
// per step only the velocity-, fraction- and field-dependent terms are read.
//
// Coefficients follow the vectorised form of Eq. 4.3-4.4: per axis the
// convection tuple [-max(F_b,0); max(F_f,0) - min(F_b,0); min(F_f,0)]/h and
// the diffusion tuple [-D_b; D_b + D_f; -D_f]/h^2 (sign of -div(D grad)),
// where F_b/F_f are the advecting velocities on the back/front faces of the
// control volume and a neighbour that is not an unknown drops its coupling.
#include "solid_internal.cuh"

namespace solid {
namespace {

// The pointwise and assembly kernels of this file use smaller blocks than the
// cooperative solvers: one row per thread, no block-wide reductions.
constexpr int kBlockA = 256;

inline int grid_for(long long n) {
  long long b = (n + kBlockA - 1) / kBlockA;
  if (b > 152LL * 32) b = 152LL * 32;
  if (b < 1) b = 1;
  return (int)b;
}

struct Axes {
  int n[3];
  double ih[3], ih2[3];
};

__device__ __forceinline__ Axes axes_of(const Params& pr) {
  Axes ax;
  ax.n[0] = pr.nx; ax.n[1] = pr.ny; ax.n[2] = pr.nz;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    ax.ih[a] = pr.ih[a];
    ax.ih2[a] = pr.ih2[a];
  }
  return ax;
}

// flat index of (i, j, k) in the face array of velocity component d
__device__ __forceinline__ int fidx(const Params& pr, int d, int i, int j, int k) {
  const int fx = pr.nx + (d == 0), fy = pr.ny + (d == 1);
  return i + fx * (j + fy * k);
}

__device__ __forceinline__ int cidx(const Params& pr, int i, int j, int k) { return i + pr.nx * (j + pr.ny * k); }

// These kernels are bound by the FP64 pipe (a small fraction of the FP32
// rate on GB300), so work that needs no FP64 arithmetic is done on the
// integer pipes: the sign split of an advecting velocity and the FP64 -> FP32
// rounding of the plane copies.

// max(F, 0) and min(F, 0) by the sign bit (a -0 goes to the negative side,
// which changes no coefficient).
struct Split {
  double pos, neg;
};
__device__ __forceinline__ Split split(double F) {
  const bool negative = __double2hiint(F) < 0;
  return {negative ? 0.0 : F, negative ? F : 0.0};
}

// to_f32 (solid_internal.cuh): the FP64 -> FP32 rounding on the integer pipes.

// The mixed path's FP64 residual never reads the FP64 inverse diagonal: it is
// written on the FP64 path only, and the FP32 one is an FP32 reciprocal
// (both are Jacobi preconditioners; the residuals use the planes).
__device__ __forceinline__ void write_row(const Sys& s, int r, int dim, double P, const double nbB[3],
                                          const double nbF[3], double b) {
  s.a.P[r] = P;
  s.a.W[r] = nbB[0];
  s.a.E[r] = nbF[0];
  s.a.S[r] = nbB[1];
  s.a.N[r] = nbF[1];
  if (dim == 3) {
    s.a.B[r] = nbB[2];
    s.a.T_[r] = nbF[2];
  }
  s.b[r] = b;
  if (s.af.P) {   // FP32 copies for the mixed-precision inner solve
    const float Pf = to_f32(P);
    s.af.P[r] = Pf;
    s.af.W[r] = to_f32(nbB[0]);
    s.af.E[r] = to_f32(nbF[0]);
    s.af.S[r] = to_f32(nbB[1]);
    s.af.N[r] = to_f32(nbF[1]);
    if (dim == 3) {
      s.af.B[r] = to_f32(nbB[2]);
      s.af.T_[r] = to_f32(nbF[2]);
    }
    s.af.idiag[r] = 1.0f / Pf;
  } else {
    s.a.idiag[r] = 1.0 / P;
  }
}

// Rows first, first + stride, ... below end of the momentum system of
// component A (the bodies below take a row range so that one launch can also
// serve many cases of a packed batch).
template <int A>
__device__ __forceinline__ void assemble_momentum_rows(const Params& pr, const Sys& s, const double* __restrict__ u,
                                                       const double* __restrict__ v, const double* __restrict__ w,
                                                       double* ustar, const double* __restrict__ p,
                                                       const double* __restrict__ T, const double* __restrict__ Cl,
                                                       const double* __restrict__ Kinv, int first, int stride,
                                                       int end) {
  const Axes ax = axes_of(pr);
  const double* vel[3] = {u, v, w};
  const int mx = s.d.mx, my = s.d.my;
  const int sA = (A == 0) ? 1 : (A == 1) ? mx : mx * my;    // stride of axis A in the row grid
  const double idt = pr.idt;
  for (int r = first; r < end; r += stride) {
    int i, j, k;
    decompose3(r, s.d.fmx, s.d.fmy, i, j, k);
    const int idx[3] = {i, j, k};
    const int f = idx[A];
    const double own = vel[A][r];
    ustar[r] = own;   // initial guess of the predictor solve: u^n
    double nbB[3] = {0.0, 0.0, 0.0}, nbF[3] = {0.0, 0.0, 0.0};
    if (f == 0 || f == ax.n[A]) {   // wall face: identity row, datum 0
      write_row(s, r, pr.dim, 1.0, nbB, nbF, 0.0);
      continue;
    }
    // the two cells sharing this face along A
    int lo[3] = {i, j, k};
    lo[A] -= 1;
    const int c_lo = cidx(pr, lo[0], lo[1], lo[2]);
    const int c_hi = cidx(pr, i, j, k);
    double P = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (d >= pr.dim) break;
      // sums (not means) of the two velocities that advect across the back and
      // front faces of this control volume; the 1/2 is folded into hh = 1/(2h)
      double sb, sf, Db, Df;   // Db, Df: diffusion coefficient / h^2 of the two faces
      bool hb, hf;
      if (d == A) {
        sb = vel[A][r - sA] + own;
        sf = own + vel[A][r + sA];
        hb = (f - 1 >= 1);
        hf = (f + 1 <= ax.n[A] - 1);
        Db = pr.nu_ih2[d];
        Df = pr.nu_ih2[d];
      } else {
        int lo_f[3] = {lo[0], lo[1], lo[2]}, hi_f[3] = {i, j, k};
        lo_f[d] += 1;
        hi_f[d] += 1;
        sb = vel[d][fidx(pr, d, lo[0], lo[1], lo[2])] + vel[d][fidx(pr, d, i, j, k)];
        sf = vel[d][fidx(pr, d, lo_f[0], lo_f[1], lo_f[2])] + vel[d][fidx(pr, d, hi_f[0], hi_f[1], hi_f[2])];
        hb = (idx[d] >= 1);
        hf = (idx[d] <= ax.n[d] - 2);
        // beyond a wall the ghost is -interior (no-slip: the wall face then
        // carries 2 nu) or +interior (free-slip: no viscous flux)
        Db = hb ? pr.nu_ih2[d] : (pr.slip[2 * d] ? 0.0 : pr.two_nu_ih2[d]);
        Df = hf ? pr.nu_ih2[d] : (pr.slip[2 * d + 1] ? 0.0 : pr.two_nu_ih2[d]);
      }
      const Split b_ = split(sb), f_ = split(sf);
      P += fma(f_.pos - b_.neg, pr.hh[d], Db + Df);
      nbB[d] = hb ? fma(-b_.pos, pr.hh[d], -Db) : 0.0;
      nbF[d] = hf ? fma(f_.neg, pr.hh[d], -Df) : 0.0;
    }
    P += idt + pr.half_nu * (Kinv[c_lo] + Kinv[c_hi]);
    double b = fma(own, idt, -(p[c_hi] - p[c_lo]) * pr.ih_irho[A]);
    if (A == pr.vert) {
      const double Tf = 0.5 * (T[c_lo] + T[c_hi]);
      const double Cf = 0.5 * (Cl[c_lo] + Cl[c_hi]);
      b += pr.gravity * (pr.betaT * (Tf - pr.Tref) + pr.betaC * (Cf - pr.C0));
    }
    write_row(s, r, pr.dim, P, nbB, nbF, b);
  }
}

// ---- mixed-path assembly in double-float arithmetic
//
// The same rows as above with the plane coefficients computed in double-float
// (about 48 significant bits on the FP32 pipe, inputs split on the integer
// pipe) and converted to FP64 with one FP64 add per plane: GB300's FP64 pipe
// bounds the FP64 kernels at ~30 FP64 operations per row. The right-hand side
// stays FP64 (its pressure difference and Boussinesq deviations cancel). The
// planes agree with the FP64 ones to ~1e-14 relative to the row's scale, and
// the FP32 copies are their IEEE rounding as before (formed from the pairs,
// see df_round).

// max(F, 0) and min(F, 0) of a double-float by the sign of its leading part
struct SplitDf {
  dfl pos, neg;
};
__device__ __forceinline__ SplitDf split_df(dfl F) {
  const dfl z = {0.f, 0.f};
  const bool negative = __float_as_int(F.hi) < 0;
  return {negative ? z : F, negative ? F : z};
}

// The FP64 planes are the pairs' sums (exact widening, one FP64 add). The
// FP32 copies are the same sums rounded once in FP32: rounding hi + lo to
// binary64 and then to binary32 gives the binary32 rounding of hi + lo itself
// (double rounding through 53 bits is innocuous for a sum of two 24-bit
// numbers, as 53 >= 2 * 24 + 1), so they equal the FP64 planes' IEEE
// rounding bit for bit, without the integer-pipe conversion.
__device__ __forceinline__ float df_round(dfl a) { return __fadd_rn(a.hi, a.lo); }

__device__ __forceinline__ void write_row_df(const Sys& s, int r, int dim, dfl P, const dfl nbB[3], const dfl nbF[3],
                                             double b) {
  s.a.P[r] = df_to_f64(P);
  s.a.W[r] = df_to_f64(nbB[0]);
  s.a.E[r] = df_to_f64(nbF[0]);
  s.a.S[r] = df_to_f64(nbB[1]);
  s.a.N[r] = df_to_f64(nbF[1]);
  if (dim == 3) {
    s.a.B[r] = df_to_f64(nbB[2]);
    s.a.T_[r] = df_to_f64(nbF[2]);
  }
  s.b[r] = b;
  if (s.af.P) {
    const float Pf = df_round(P);
    s.af.P[r] = Pf;
    s.af.W[r] = df_round(nbB[0]);
    s.af.E[r] = df_round(nbF[0]);
    s.af.S[r] = df_round(nbB[1]);
    s.af.N[r] = df_round(nbF[1]);
    if (dim == 3) {
      s.af.B[r] = df_round(nbB[2]);
      s.af.T_[r] = df_round(nbF[2]);
    }
    s.af.idiag[r] = 1.0f / Pf;
  } else {
    s.a.idiag[r] = 1.0 / df_to_f64(P);
  }
}

template <int A>
__device__ __forceinline__ void assemble_momentum_rows_df(const Params& pr, const Sys& s, const double* __restrict__ u,
                                                          const double* __restrict__ v, const double* __restrict__ w,
                                                          double* ustar, const double* __restrict__ p,
                                                          const double* __restrict__ T,
                                                          const double* __restrict__ Cl,
                                                          const double* __restrict__ Kinv, int first, int stride,
                                                          int end) {
  const Axes ax = axes_of(pr);
  const double* vel[3] = {u, v, w};
  const int mx = s.d.mx, my = s.d.my;
  const int sA = (A == 0) ? 1 : (A == 1) ? mx : mx * my;
  const double idt = pr.idt;
  const dfl zero = {0.f, 0.f};
  for (int r = first; r < end; r += stride) {
    int i, j, k;
    decompose3(r, s.d.fmx, s.d.fmy, i, j, k);
    const int idx[3] = {i, j, k};
    const int f = idx[A];
    const double own = vel[A][r];
    ustar[r] = own;   // initial guess of the predictor solve: u^n
    if (f == 0 || f == ax.n[A]) {   // wall face: identity row, datum 0
      const double zb[3] = {0.0, 0.0, 0.0};
      write_row(s, r, pr.dim, 1.0, zb, zb, 0.0);
      continue;
    }
    int lo[3] = {i, j, k};
    lo[A] -= 1;
    const int c_lo = cidx(pr, lo[0], lo[1], lo[2]);
    const int c_hi = cidx(pr, i, j, k);
    const dfl own_d = df_from(own);
    dfl P = df_add(pr.df_idt, df_mul(pr.df_half_nu, df_add(df_from(Kinv[c_lo]), df_from(Kinv[c_hi]))));
    dfl nbB[3] = {zero, zero, zero}, nbF[3] = {zero, zero, zero};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (d >= pr.dim) break;
      dfl sb, sf, Db, Df;
      bool hb, hf;
      if (d == A) {
        sb = df_add(df_from(vel[A][r - sA]), own_d);
        sf = df_add(own_d, df_from(vel[A][r + sA]));
        hb = (f - 1 >= 1);
        hf = (f + 1 <= ax.n[A] - 1);
        Db = pr.df_nu_ih2[d];
        Df = pr.df_nu_ih2[d];
      } else {
        int lo_f[3] = {lo[0], lo[1], lo[2]}, hi_f[3] = {i, j, k};
        lo_f[d] += 1;
        hi_f[d] += 1;
        sb = df_add(df_from(vel[d][fidx(pr, d, lo[0], lo[1], lo[2])]), df_from(vel[d][fidx(pr, d, i, j, k)]));
        sf = df_add(df_from(vel[d][fidx(pr, d, lo_f[0], lo_f[1], lo_f[2])]),
                    df_from(vel[d][fidx(pr, d, hi_f[0], hi_f[1], hi_f[2])]));
        hb = (idx[d] >= 1);
        hf = (idx[d] <= ax.n[d] - 2);
        Db = hb ? pr.df_nu_ih2[d] : (pr.slip[2 * d] ? zero : pr.df_two_nu_ih2[d]);
        Df = hf ? pr.df_nu_ih2[d] : (pr.slip[2 * d + 1] ? zero : pr.df_two_nu_ih2[d]);
      }
      const SplitDf b_ = split_df(sb), f_ = split_df(sf);
      P = df_add(P, df_add(df_mul(df_sub(f_.pos, b_.neg), pr.df_hh[d]), df_add(Db, Df)));
      if (hb) nbB[d] = df_neg(df_add(df_mul(b_.pos, pr.df_hh[d]), Db));
      if (hf) nbF[d] = df_sub(df_mul(f_.neg, pr.df_hh[d]), Df);
    }
    double b = fma(own, idt, -(p[c_hi] - p[c_lo]) * pr.ih_irho[A]);
    if (A == pr.vert) {
      const double Tf = 0.5 * (T[c_lo] + T[c_hi]);
      const double Cf = 0.5 * (Cl[c_lo] + Cl[c_hi]);
      b += pr.gravity * (pr.betaT * (Tf - pr.Tref) + pr.betaC * (Cf - pr.C0));
    }
    write_row_df(s, r, pr.dim, P, nbB, nbF, b);
  }
}

template <int A>
__global__ void __launch_bounds__(kBlockA) k_assemble_momentum_df(Params pr, Sys s, const double* __restrict__ u,
                                                                 const double* __restrict__ v,
                                                                 const double* __restrict__ w, double* ustar,
                                                                 const double* __restrict__ p,
                                                                 const double* __restrict__ T,
                                                                 const double* __restrict__ Cl,
                                                                 const double* __restrict__ Kinv) {
  assemble_momentum_rows_df<A>(pr, s, u, v, w, ustar, p, T, Cl, Kinv, blockIdx.x * blockDim.x + threadIdx.x,
                               gridDim.x * blockDim.x, (int)s.d.n);
}

template <int A>
__global__ void __launch_bounds__(kBlockA) k_assemble_momentum(Params pr, Sys s, const double* __restrict__ u,
                                                              const double* __restrict__ v,
                                                              const double* __restrict__ w, double* ustar,
                                                              const double* __restrict__ p,
                                                              const double* __restrict__ T,
                                                              const double* __restrict__ Cl,
                                                              const double* __restrict__ Kinv) {
  assemble_momentum_rows<A>(pr, s, u, v, w, ustar, p, T, Cl, Kinv, blockIdx.x * blockDim.x + threadIdx.x,
                            gridDim.x * blockDim.x, (int)s.d.n);
}

// Cell-centred systems. SOLUTE = true: solute (Eq. 3.10) with diffusivity
// g_l^n D_l on faces and column scaling by A_g = 1/(1 - (1-k_p)(1-g_l^n));
// false: T* (Eq. 3.12) with diffusivity k/(rho c_p) and cooled walls, whose
// temperature is taken at the new time level *time + dt.
// `Ag` holds A_g per cell (kept current by k_lever / k_equilibrate).
// T* only (Tinc non-null): the solve's initial guess replaces T^n in place,
// T^n + Tinc (the previous step's T* - T^{n-1}, or 0) when use_guess, else
// T^n; Tinc then holds -T^n, which the lever stage completes to T* - T^n.
// Each row reads and writes T and Tinc only at itself.
template <bool SOLUTE>
__device__ __forceinline__ void assemble_cells_rows(const Params& pr, const Sys& s, const double* __restrict__ u,
                                                    const double* __restrict__ v, const double* __restrict__ w,
                                                    double* phi_n, const double* __restrict__ gl,
                                                    const double* __restrict__ Ag, const double* __restrict__ time,
                                                    double* Tinc, int use_guess, int first, int rstride, int end) {
  const Axes ax = axes_of(pr);
  const double* vel[3] = {u, v, w};
  const int nx = pr.nx, ny = pr.ny;
  const int stride[3] = {1, nx, nx * ny};
  const double idt = pr.idt;
  for (int r = first; r < end; r += rstride) {
    int i, j, k;
    decompose3(r, pr.fnx, pr.fny, i, j, k);
    const int idx[3] = {i, j, k};
    double m0 = 0.0, nbB[3] = {0.0, 0.0, 0.0}, nbF[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a >= pr.dim) break;
      int fr[3] = {i, j, k};
      fr[a] += 1;
      const Split b_ = split(vel[a][fidx(pr, a, i, j, k)]);
      const Split f_ = split(vel[a][fidx(pr, a, fr[0], fr[1], fr[2])]);
      const bool hb = idx[a] >= 1, hf = idx[a] <= ax.n[a] - 2;
      double Db, Df;   // diffusion coefficient / h^2 of the back and front faces
      if (SOLUTE) {
        Db = hb ? pr.half_Dl_ih2[a] * (gl[r - stride[a]] + gl[r]) : 0.0;
        Df = hf ? pr.half_Dl_ih2[a] * (gl[r] + gl[r + stride[a]]) : 0.0;
      } else {
        Db = hb ? pr.alpha_ih2[a] : 0.0;
        Df = hf ? pr.alpha_ih2[a] : 0.0;
      }
      m0 += fma(f_.pos - b_.neg, ax.ih[a], Db + Df);
      double cb = hb ? fma(-b_.pos, ax.ih[a], -Db) : 0.0;
      double cf = hf ? fma(f_.neg, ax.ih[a], -Df) : 0.0;
      if (SOLUTE) {
        cb = hb ? cb * Ag[r - stride[a]] : 0.0;
        cf = hf ? cf * Ag[r + stride[a]] : 0.0;
      }
      nbB[a] = cb;
      nbF[a] = cf;
    }
    const double phi = phi_n[r];
    double P, b = phi * idt;
    if (!SOLUTE && Tinc) {
      const double inc = Tinc[r];
      phi_n[r] = use_guess ? phi + inc : phi;
      Tinc[r] = -phi;
    }
    if (SOLUTE) {
      P = idt + m0 * Ag[r];
    } else {
      P = m0 + idt;
      // cooled walls: flux coef (T_P - T_w(t^{n+1})) (Robin through the film and
      // half a cell; Dirichlet through half a cell)
      const int wall[6] = {i == 0, i == nx - 1, j == 0, j == ny - 1, pr.dim == 3 && k == 0,
                           pr.dim == 3 && k == pr.nz - 1};
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        if (wall[q] && ((pr.wall_mask >> q) & 1)) {   // boundary rows only: no FP64 work elsewhere
          const double t_new = *time + pr.dt;
          P += pr.wall_coef[q];
          b += pr.wall_coef[q] * (pr.wall_T0[q] + pr.wall_rate[q] * t_new);
        }
      }
    }
    write_row(s, r, pr.dim, P, nbB, nbF, b);
  }
}

template <bool SOLUTE>
__device__ __forceinline__ void assemble_cells_rows_df(const Params& pr, const Sys& s, const double* __restrict__ u,
                                                       const double* __restrict__ v, const double* __restrict__ w,
                                                       double* phi_n, const double* __restrict__ gl,
                                                       const double* __restrict__ Ag,
                                                       const double* __restrict__ time, double* Tinc, int use_guess,
                                                       int first, int rstride, int end) {
  const Axes ax = axes_of(pr);
  const double* vel[3] = {u, v, w};
  const int nx = pr.nx, ny = pr.ny;
  const int stride[3] = {1, nx, nx * ny};
  const double idt = pr.idt;
  const dfl zero = {0.f, 0.f};
  for (int r = first; r < end; r += rstride) {
    int i, j, k;
    decompose3(r, pr.fnx, pr.fny, i, j, k);
    const int idx[3] = {i, j, k};
    dfl m0 = zero, nbB[3] = {zero, zero, zero}, nbF[3] = {zero, zero, zero};
    dfl g0 = zero, agc = zero;
    if (SOLUTE) {
      g0 = df_from(gl[r]);
      agc = df_from(Ag[r]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a >= pr.dim) break;
      int fr[3] = {i, j, k};
      fr[a] += 1;
      const SplitDf b_ = split_df(df_from(vel[a][fidx(pr, a, i, j, k)]));
      const SplitDf f_ = split_df(df_from(vel[a][fidx(pr, a, fr[0], fr[1], fr[2])]));
      const bool hb = idx[a] >= 1, hf = idx[a] <= ax.n[a] - 2;
      dfl Db = zero, Df = zero;   // diffusion coefficient / h^2 of the back and front faces
      if (SOLUTE) {
        if (hb) Db = df_mul(pr.df_half_Dl_ih2[a], df_add(df_from(gl[r - stride[a]]), g0));
        if (hf) Df = df_mul(pr.df_half_Dl_ih2[a], df_add(g0, df_from(gl[r + stride[a]])));
      } else {
        if (hb) Db = pr.df_alpha_ih2[a];
        if (hf) Df = pr.df_alpha_ih2[a];
      }
      m0 = df_add(m0, df_add(df_mul(df_sub(f_.pos, b_.neg), pr.df_ih[a]), df_add(Db, Df)));
      dfl cb = zero, cf = zero;
      if (hb) cb = df_neg(df_add(df_mul(b_.pos, pr.df_ih[a]), Db));
      if (hf) cf = df_sub(df_mul(f_.neg, pr.df_ih[a]), Df);
      if (SOLUTE) {
        if (hb) cb = df_mul(cb, df_from(Ag[r - stride[a]]));
        if (hf) cf = df_mul(cf, df_from(Ag[r + stride[a]]));
      }
      nbB[a] = cb;
      nbF[a] = cf;
    }
    const double phi = phi_n[r];
    double b = phi * idt;
    if (!SOLUTE && Tinc) {
      const double inc = Tinc[r];
      phi_n[r] = use_guess ? phi + inc : phi;
      Tinc[r] = -phi;
    }
    dfl P;
    if (SOLUTE) {
      P = df_add(pr.df_idt, df_mul(m0, agc));
    } else {
      P = df_add(m0, pr.df_idt);
      const int wall[6] = {i == 0, i == nx - 1, j == 0, j == ny - 1, pr.dim == 3 && k == 0,
                           pr.dim == 3 && k == pr.nz - 1};
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        if (wall[q] && ((pr.wall_mask >> q) & 1)) {   // boundary rows only
          const double t_new = *time + pr.dt;
          P = df_add(P, pr.df_wall_coef[q]);
          b += pr.wall_coef[q] * (pr.wall_T0[q] + pr.wall_rate[q] * t_new);
        }
      }
    }
    write_row_df(s, r, pr.dim, P, nbB, nbF, b);
  }
}

template <bool SOLUTE>
__global__ void __launch_bounds__(kBlockA) k_assemble_cells_df(Params pr, Sys s, const double* __restrict__ u,
                                                              const double* __restrict__ v,
                                                              const double* __restrict__ w, double* phi_n,
                                                              const double* __restrict__ gl,
                                                              const double* __restrict__ Ag,
                                                              const double* __restrict__ time, double* Tinc,
                                                              int use_guess) {
  assemble_cells_rows_df<SOLUTE>(pr, s, u, v, w, phi_n, gl, Ag, time, Tinc, use_guess,
                                 blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, (int)s.d.n);
}

template <bool SOLUTE>
__global__ void __launch_bounds__(kBlockA) k_assemble_cells(Params pr, Sys s, const double* __restrict__ u,
                                                           const double* __restrict__ v,
                                                           const double* __restrict__ w,
                                                           double* phi_n,
                                                           const double* __restrict__ gl,
                                                           const double* __restrict__ Ag,
                                                           const double* __restrict__ time, double* Tinc,
                                                           int use_guess) {
  assemble_cells_rows<SOLUTE>(pr, s, u, v, w, phi_n, gl, Ag, time, Tinc, use_guess,
                              blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, (int)s.d.n);
}

__device__ __forceinline__ void poisson_rhs_rows(const Params& pr, const double* __restrict__ us,
                                                 const double* __restrict__ vs, const double* __restrict__ ws,
                                                 double* b, int first, int stride, int end) {
  const Axes ax = axes_of(pr);
  const double scale = pr.rhs_scale;
  for (int r = first; r < end; r += stride) {
    int i, j, k;
    decompose3(r, pr.fnx, pr.fny, i, j, k);
    double div = (us[fidx(pr, 0, i + 1, j, k)] - us[fidx(pr, 0, i, j, k)]) * ax.ih[0] +
                 (vs[fidx(pr, 1, i, j + 1, k)] - vs[fidx(pr, 1, i, j, k)]) * ax.ih[1];
    if (pr.dim == 3) div += (ws[fidx(pr, 2, i, j, k + 1)] - ws[fidx(pr, 2, i, j, k)]) * ax.ih[2];
    b[r] = scale * div;
  }
}

__global__ void __launch_bounds__(kBlockA) k_poisson_rhs(Params pr, const double* __restrict__ us,
                                                        const double* __restrict__ vs,
                                                        const double* __restrict__ ws, double* b) {
  poisson_rhs_rows(pr, us, vs, ws, b, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x,
                   pr.nx * pr.ny * pr.nz);
}

// Faces of u, v, w then cells of p, one flat index space of project_size() entries.
__host__ __device__ __forceinline__ int project_size(const Params& pr) {
  const int nx = pr.nx, ny = pr.ny, nz = pr.nz;
  return (nx + 1) * ny * nz + nx * (ny + 1) * nz + ((pr.dim == 3) ? nx * ny * (nz + 1) : 0) + nx * ny * nz;
}

__device__ __forceinline__ void project_rows(const Params& pr, double* u, double* v, double* w,
                                             const double* __restrict__ us, const double* __restrict__ vs,
                                             const double* __restrict__ ws, const double* __restrict__ pc, double* p,
                                             int first, int stride, int total) {
  const int nx = pr.nx, ny = pr.ny, nz = pr.nz;
  const int nu_ = (nx + 1) * ny * nz, nv = nx * (ny + 1) * nz, nw = (pr.dim == 3) ? nx * ny * (nz + 1) : 0;
  const double kk = pr.proj_k;
  for (int q = first; q < total; q += stride) {
    if (q < nu_ + nv + nw) {
      int d, r;
      if (q < nu_) { d = 0; r = q; }
      else if (q < nu_ + nv) { d = 1; r = q - nu_; }
      else { d = 2; r = q - nu_ - nv; }
      const int fx = nx + (d == 0), fy = ny + (d == 1);
      const int i = r % fx, t = r / fx, j = t % fy, k = t / fy;
      // position along d, cell count along d and cell stride along d, without
      // arrays indexed by the runtime axis (they would live in local memory)
      const int f = (d == 0) ? i : (d == 1) ? j : k;
      const int nd = (d == 0) ? nx : (d == 1) ? ny : nz;
      const int sd = (d == 0) ? 1 : (d == 1) ? nx : nx * ny;
      double* out = (d == 0) ? u : (d == 1) ? v : w;
      const double* in = (d == 0) ? us : (d == 1) ? vs : ws;
      if (f == 0 || f == nd) { out[r] = 0.0; continue; }
      const int c_hi = cidx(pr, i, j, k);
      const double grad = (pc[c_hi] - pc[c_hi - sd]) * pr.ih[d];
      out[r] = in[r] - kk * grad;
    } else {
      const int c = q - (nu_ + nv + nw);
      p[c] += pc[c];
    }
  }
}

__global__ void __launch_bounds__(kBlockA) k_project(Params pr, double* u, double* v, double* w,
                                                    const double* __restrict__ us,
                                                    const double* __restrict__ vs,
                                                    const double* __restrict__ ws,
                                                    const double* __restrict__ pc, double* p) {
  project_rows(pr, u, v, w, us, vs, ws, pc, p, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x,
               project_size(pr));
}

struct Phase {
  double Cl, Kinv, Ag;
};

__device__ __forceinline__ Phase phase_of(const Params& pr, double C, double g) {
  Phase o;
  const double s = 1.0 - g;
  if (s == 0.0) {
    // fully liquid: the two divisions below give exactly A_g = 1 and K^-1 = 0
    o.Ag = 1.0;
    o.Cl = C;
    o.Kinv = 0.0;
  } else {
    // g + kp (1 - g) = 1 - (1 - kp)(1 - g): the denominator of Eq. 3.18 is 1/A_g (Eq. 3.8);
    // both quotients from one reciprocal (a few ulps, where two divisions
    // would cost the FP64 pipe twice)
    const double d1 = 1.0 - pr.lev_a * s;            // 1 / A_g
    const double d2 = pr.K0 * (g * g * g + pr.eps);  // Carman-Kozeny denominator, regularised
    const double inv = 1.0 / (d1 * d2);
    o.Ag = d2 * inv;                                 // Eq. 3.8, for the next solute step
    o.Cl = C * o.Ag;                                 // Eq. 3.18
    o.Kinv = s * s * (d1 * inv);                     // Eq. 2.8
  }
  if (pr.has_eutectic) o.Cl = fmin(o.Cl, pr.Ce);
  return o;
}

// The lever update closes a step: it also advances the case's time by dt
// (done by the thread whose first row is 0).
// Tinc (may be null): T* - T^n for the next step's initial guess when
// form_inc (Tinc holds -T^n from this step's T* assembly), else 0.
__device__ __forceinline__ void lever_rows(const Params& pr, double* time, double* T, double* gl,
                                           const double* __restrict__ C, double* Cl, double* Cs, double* Kinv,
                                           double* Ag, double* Tinc, int form_inc, int first, int stride, int n) {
  if (first == 0) *time += pr.dt;
  const double kp = pr.kp, Tm = pr.Tm;
  const double cpL = pr.cpL, Lcp = pr.Lcp;
  const double a = pr.lev_a;
  const double Te = pr.Te;
  for (int r = first; r < n; r += stride) {
    const double Ts = T[r], gn = gl[r], Cn = C[r];
    const double Tl = Tm + pr.m * Cn;                                       // Eq. 3.14
    double g, Tn;
    if (gn == 1.0 && Ts >= Tl) {
      // a fully liquid cell at or above its liquidus stays liquid: the lever
      // solution is g = 1 and T = T* (the root of Eq. 3.16 is >= 1 and is
      // clamped to 1, so Eq. 3.13 leaves T* unchanged)
      g = 1.0;
      Tn = Ts;
    } else {
      const double b = kp - gn * a + pr.lev_cpLa * (Tm - Ts);              // Eq. 3.17
      const double c = -(gn + cpL * Ts) * kp + cpL * (Tl - pr.lev_aTm);
      const double sq = sqrt(fmax(b * b - pr.lev_4a * c, 0.0));
      // larger root of Eq. 3.16 (a > 0), in the form free of cancellation
      g = (b > 0.0) ? (2.0 * c) / (-b - sq) : (-b + sq) * pr.lev_inv2a;
      g = fmin(fmax(g, 0.0), 1.0);
      Tn = Ts - Lcp * (g - gn);                                              // Eq. 3.13
    }
    if (pr.has_eutectic && Tn < Te && g > 0.0) {   // isothermal eutectic plateau
      const double ge = gn - cpL * (Te - Ts);
      if (ge >= 0.0) { g = ge; Tn = Te; }
      else { g = 0.0; Tn = Ts + Lcp * gn; }
    }
    const Phase ph = phase_of(pr, Cn, g);
    if (Tinc) Tinc[r] = form_inc ? Ts + Tinc[r] : 0.0;
    T[r] = Tn;
    gl[r] = g;
    Cl[r] = ph.Cl;
    Cs[r] = kp * ph.Cl;                                                      // Eq. 3.19
    Kinv[r] = ph.Kinv;
    Ag[r] = ph.Ag;
  }
}

__global__ void __launch_bounds__(kBlockA) k_lever(Params pr, double* time, double* T, double* gl,
                                                  const double* __restrict__ C, double* Cl, double* Cs, double* Kinv,
                                                  double* Ag, int n, double* Tinc, int form_inc) {
  lever_rows(pr, time, T, gl, C, Cl, Cs, Kinv, Ag, Tinc, form_inc, blockIdx.x * blockDim.x + threadIdx.x,
             gridDim.x * blockDim.x, n);
}

__global__ void __launch_bounds__(kBlockA) k_equilibrate(Params pr, const double* __restrict__ T,
                                                        const double* __restrict__ C, double* gl, double* Cl,
                                                        double* Cs, double* Kinv, double* Ag, int n, int from_T,
                                                        int write_cl) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    double g = gl[r];
    if (from_T) {
      const double Tv = T[r], Tl = pr.Tm + pr.m * C[r];
      g = 1.0 - (Tv - Tl) / ((1.0 - pr.kp) * (Tv - pr.Tm));                 // Eq. 3.15
      g = (Tv >= Tl) ? 1.0 : fmin(fmax(g, 0.0), 1.0);
      gl[r] = g;
    }
    const Phase ph = phase_of(pr, C[r], g);
    if (write_cl) {
      Cl[r] = ph.Cl;
      Cs[r] = pr.kp * ph.Cl;
    }
    Kinv[r] = ph.Kinv;
    Ag[r] = ph.Ag;
  }
}


// ---- Forward assembly (Sec. 4, Eq. 4.5-4.7), a validation mode.
//
// The discrete equation of each row, Eq_r(phi), is written straight from its
// fluxes and wall ghosts (independently of the term-wise kernels above).
// Eq is affine, Eq(phi) = A phi - b, so b = -Eq(0), and the coefficient of
// row r on stencil point q is Eq_r(e) - Eq_r(0) for the trial vector e that
// is 1 on the cells of q's colour (colour = (i mod 3, j mod 3, k mod 3)): the
// seven points of a stencil have seven distinct colours. A trial vector is a
// function of the indices, so no probe vector is stored.
__device__ __forceinline__ int colour_of(int i, int j, int k) { return (i % 3) + 3 * (j % 3) + 9 * (k % 3); }

// (phi F) on a face with phi_back behind and phi_front in front: first-order upwind
__device__ __forceinline__ double upwind_flux(double F, double back, double front) {
  return (F >= 0.0 ? back : front) * F;
}

// Eq_r of component A of the intermediate velocity (Eq. 3.3) at the face
// (i, j, k), for the trial vector that is 1 on colour c (c < 0: all zero).
template <int A>
__device__ double momentum_equation(const Params& pr, const double* const vel[3], const double* p, const double* T,
                                    const double* Cl, const double* Kinv, int i, int j, int k, int c) {
  const int n[3] = {pr.nx, pr.ny, pr.nz};
  const int idx[3] = {i, j, k};
  const double h[3] = {pr.hx, pr.hy, pr.hz};
  const int fx = pr.nx + (A == 0), fy = pr.ny + (A == 1);
  auto trial = [&](int ii, int jj, int kk) -> double { return (c >= 0 && colour_of(ii, jj, kk) == c) ? 1.0 : 0.0; };
  auto u_at = [&](int d, int ii, int jj, int kk) -> double {
    const int gx = pr.nx + (d == 0), gy = pr.ny + (d == 1);
    return vel[d][ii + gx * (jj + gy * kk)];
  };
  const double P = trial(i, j, k);
  if (idx[A] == 0 || idx[A] == n[A]) return P;            // wall face: phi - 0
  const double nu = pr.mu / pr.rho;
  int lo[3] = {i, j, k};
  lo[A] -= 1;                                               // the cells on either side of the face
  const double own = vel[A][i + fx * (j + fy * k)];
  double r = (P - own) / pr.dt;
  for (int d = 0; d < pr.dim; ++d) {
    int f[3] = {i, j, k}, b[3] = {i, j, k};
    f[d] += 1;
    b[d] -= 1;
    double Uf, Ub, Pf, Pb;
    if (d == A) {
      Uf = 0.5 * (own + u_at(A, f[0], f[1], f[2]));
      Ub = 0.5 * (u_at(A, b[0], b[1], b[2]) + own);
      Pf = (f[A] == n[A]) ? 0.0 : trial(f[0], f[1], f[2]);  // the wall face holds 0
      Pb = (b[A] == 0) ? 0.0 : trial(b[0], b[1], b[2]);
    } else {
      int lf[3] = {lo[0], lo[1], lo[2]}, hf[3] = {i, j, k};
      lf[d] += 1;
      hf[d] += 1;
      Uf = 0.5 * (u_at(d, lf[0], lf[1], lf[2]) + u_at(d, hf[0], hf[1], hf[2]));
      Ub = 0.5 * (u_at(d, lo[0], lo[1], lo[2]) + u_at(d, i, j, k));
      // beyond a wall: ghost = -phi (no-slip) or +phi (free-slip)
      const double gf = pr.slip[2 * d + 1] ? P : -P, gb = pr.slip[2 * d] ? P : -P;
      Pf = (idx[d] + 1 <= n[d] - 1) ? trial(f[0], f[1], f[2]) : gf;
      Pb = (idx[d] - 1 >= 0) ? trial(b[0], b[1], b[2]) : gb;
    }
    r += (upwind_flux(Uf, P, Pf) - upwind_flux(Ub, Pb, P)) / h[d];
    r -= nu * ((Pf - P) - (P - Pb)) / (h[d] * h[d]);
  }
  const int clo = lo[0] + pr.nx * (lo[1] + pr.ny * lo[2]), chi = i + pr.nx * (j + pr.ny * k);
  r += nu * 0.5 * (Kinv[clo] + Kinv[chi]) * P;
  r += (p[chi] - p[clo]) / (h[A] * pr.rho);
  if (A == pr.vert) {
    const double Tf = 0.5 * (T[clo] + T[chi]), Cf = 0.5 * (Cl[clo] + Cl[chi]);
    r -= pr.gravity * (pr.betaT * (Tf - pr.Tref) + pr.betaC * (Cf - pr.C0));
  }
  return r;
}

// Eq_r of the solute step (SOLUTE: Eq. 3.7 with C_l = A_g C, Eq. 3.8-3.10)
// or of T* (Eq. 3.12 with its cooled walls) at cell (i, j, k), for the trial
// vector that is 1 on colour c (c < 0: all zero).
template <bool SOLUTE>
__device__ double cell_equation(const Params& pr, const double* const vel[3], const double* phi_n, const double* gl,
                                const double* Ag, double t_new, int i, int j, int k, int c) {
  const int n[3] = {pr.nx, pr.ny, pr.nz};
  const int idx[3] = {i, j, k};
  const double h[3] = {pr.hx, pr.hy, pr.hz};
  const int cell = i + pr.nx * (j + pr.ny * k);
  auto trial = [&](int ii, int jj, int kk) -> double { return (c >= 0 && colour_of(ii, jj, kk) == c) ? 1.0 : 0.0; };
  // the transported quantity: C_l = A_g C for the solute, T itself for energy
  auto q_at = [&](int ii, int jj, int kk) -> double {
    const double v = trial(ii, jj, kk);
    return SOLUTE ? v * Ag[ii + pr.nx * (jj + pr.ny * kk)] : v;
  };
  const double P = q_at(i, j, k);
  double r = (trial(i, j, k) - phi_n[cell]) / pr.dt;
  const double alpha = pr.k / (pr.rho * pr.cp);
  for (int a = 0; a < pr.dim; ++a) {
    int f[3] = {i, j, k}, b[3] = {i, j, k};
    f[a] += 1;
    b[a] -= 1;
    const int gx = pr.nx + (a == 0), gy = pr.ny + (a == 1);
    const double Uf = vel[a][f[0] + gx * (f[1] + gy * f[2])], Ub = vel[a][i + gx * (j + gy * k)];
    const bool has_f = idx[a] + 1 <= n[a] - 1, has_b = idx[a] - 1 >= 0;
    const double Qf = has_f ? q_at(f[0], f[1], f[2]) : 0.0, Qb = has_b ? q_at(b[0], b[1], b[2]) : 0.0;
    r += (upwind_flux(Uf, P, Qf) - upwind_flux(Ub, Qb, P)) / h[a];
    double Df = 0.0, Db = 0.0;   // zero-flux walls
    if (SOLUTE) {
      if (has_f) Df = pr.Dl * 0.5 * (gl[cell] + gl[f[0] + pr.nx * (f[1] + pr.ny * f[2])]);
      if (has_b) Db = pr.Dl * 0.5 * (gl[b[0] + pr.nx * (b[1] + pr.ny * b[2])] + gl[cell]);
    } else {
      if (has_f) Df = alpha;
      if (has_b) Db = alpha;
    }
    r -= (Df * (Qf - P) - Db * (P - Qb)) / (h[a] * h[a]);
  }
  if (!SOLUTE) {   // cooled walls: coef (T_P - T_w(t^{n+1}))
    const bool wall[6] = {i == 0, i == pr.nx - 1, j == 0, j == pr.ny - 1, pr.dim == 3 && k == 0,
                          pr.dim == 3 && k == pr.nz - 1};
    for (int w = 0; w < 6; ++w)
      if (wall[w] && pr.wall_coef[w] != 0.0)
        r += pr.wall_coef[w] * (trial(i, j, k) - (pr.wall_T0[w] + pr.wall_rate[w] * t_new));
  }
  return r;
}

// Probe the row's equation: b = -Eq(0); each stencil coefficient from the
// trial vector of its point's colour (0 for points outside the row grid).
template <typename EqF>
__device__ __forceinline__ void probe_row(const Sys& s, int r, int dim, int i, int j, int k, int mx, int my, int mz,
                                          EqF eq) {
  const double base = eq(-1);
  const double P = eq(colour_of(i, j, k)) - base;
  double nbB[3] = {0.0, 0.0, 0.0}, nbF[3] = {0.0, 0.0, 0.0};
  const int m[3] = {mx, my, mz};
  const int idx[3] = {i, j, k};
  for (int a = 0; a < dim; ++a) {
    int f[3] = {i, j, k}, b[3] = {i, j, k};
    f[a] += 1;
    b[a] -= 1;
    if (idx[a] - 1 >= 0) nbB[a] = eq(colour_of(b[0], b[1], b[2])) - base;
    if (idx[a] + 1 <= m[a] - 1) nbF[a] = eq(colour_of(f[0], f[1], f[2])) - base;
  }
  write_row(s, r, dim, P, nbB, nbF, -base);
}

template <int A>
__global__ void __launch_bounds__(kBlockA) k_forward_momentum(Params pr, Sys s, const double* __restrict__ u,
                                                             const double* __restrict__ v,
                                                             const double* __restrict__ w,
                                                             const double* __restrict__ p,
                                                             const double* __restrict__ T,
                                                             const double* __restrict__ Cl,
                                                             const double* __restrict__ Kinv) {
  const double* vel[3] = {u, v, w};
  const int mx = s.d.mx, my = s.d.my, mz = s.d.mz, n = (int)s.d.n;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const int i = r % mx, t = r / mx, j = t % my, k = t / my;
    probe_row(s, r, pr.dim, i, j, k, mx, my, mz,
              [&](int c) { return momentum_equation<A>(pr, vel, p, T, Cl, Kinv, i, j, k, c); });
  }
}

template <bool SOLUTE>
__global__ void __launch_bounds__(kBlockA) k_forward_cells(Params pr, Sys s, const double* __restrict__ u,
                                                          const double* __restrict__ v,
                                                          const double* __restrict__ w,
                                                          const double* __restrict__ phi_n,
                                                          const double* __restrict__ gl,
                                                          const double* __restrict__ Ag,
                                                          const double* __restrict__ time) {
  const double* vel[3] = {u, v, w};
  const int nx = pr.nx, ny = pr.ny, n = (int)s.d.n;
  const double t_new = SOLUTE ? 0.0 : *time + pr.dt;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const int i = r % nx, t = r / nx, j = t % ny, k = t / ny;
    probe_row(s, r, pr.dim, i, j, k, nx, ny, pr.nz,
              [&](int c) { return cell_equation<SOLUTE>(pr, vel, phi_n, gl, Ag, t_new, i, j, k, c); });
  }
}

// One launch of a packed stage: block b takes tiles[b], stages its case's
// description in shared memory and runs the stage's rows of that tile. The
// assembly stages also zero the barrier counters of their case for the
// solve launch that follows them.
template <int STAGE>
__global__ void __launch_bounds__(kBlockA) k_packed_rows(const CaseRows* __restrict__ cases,
                                                        const PackedTile* __restrict__ tiles) {
  __shared__ __align__(16) unsigned long long buf[(sizeof(CaseRows) + 7) / 8];
  const PackedTile t = tiles[blockIdx.x];
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(cases + t.c);
  for (int q = threadIdx.x; q < (int)(sizeof(CaseRows) / 8); q += blockDim.x) buf[q] = src[q];
  __syncthreads();
  const CaseRows& cs = *reinterpret_cast<const CaseRows*>(buf);
  const int first = t.r0 + threadIdx.x, stride = blockDim.x, end = t.r1;
  if (STAGE == kStageMomentum) {
    // packed batches are mixed-precision: the double-float assembly
    if (t.part == 0)
      assemble_momentum_rows_df<0>(cs.pr, cs.sys[0], cs.u, cs.v, cs.w, cs.ustar[0], cs.p, cs.T, cs.Cl, cs.Kinv,
                                   first, stride, end);
    else if (t.part == 1)
      assemble_momentum_rows_df<1>(cs.pr, cs.sys[1], cs.u, cs.v, cs.w, cs.ustar[1], cs.p, cs.T, cs.Cl, cs.Kinv,
                                   first, stride, end);
    else
      assemble_momentum_rows_df<2>(cs.pr, cs.sys[2], cs.u, cs.v, cs.w, cs.ustar[2], cs.p, cs.T, cs.Cl, cs.Kinv,
                                   first, stride, end);
  } else if (STAGE == kStageRhs) {
    poisson_rhs_rows(cs.pr, cs.ustar[0], cs.ustar[1], cs.ustar[2], cs.pb, first, stride, end);
  } else if (STAGE == kStageProject) {
    project_rows(cs.pr, cs.u, cs.v, cs.w, cs.ustar[0], cs.ustar[1], cs.ustar[2], cs.pc, cs.p, first, stride, end);
  } else if (STAGE == kStageSolute) {
    assemble_cells_rows_df<true>(cs.pr, cs.sys[SS_SYS_C], cs.u, cs.v, cs.w, cs.C, cs.gl, cs.Ag, nullptr, nullptr, 0,
                                 first, stride, end);
  } else if (STAGE == kStageTemperature) {
    assemble_cells_rows_df<false>(cs.pr, cs.sys[SS_SYS_T], cs.u, cs.v, cs.w, cs.T, nullptr, nullptr, &cs.st->time,
                                  cs.Tinc, 1, first, stride, end);
  } else {
    lever_rows(cs.pr, &cs.st->time, cs.T, cs.gl, cs.C, cs.Cl, cs.Cs, cs.Kinv, cs.Ag, cs.Tinc, 1, first, stride, end);
  }
  if (STAGE != kStageProject && STAGE != kStageLever && t.part == 0 && t.r0 == 0 && threadIdx.x == 0) {
    cs.st->barrier = 0u;
    for (int q = 0; q < kMaxTeams; ++q) cs.st->team_arrivals[q] = 0u;
  }
}

__global__ void __launch_bounds__(kBlockA) k_to_f32(const double* __restrict__ src, float* dst, long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    dst[q] = to_f32(src[q]);
}

}  // namespace

long long packed_stage_rows(int stage, const Params& pr, int part) {
  const long long nx = pr.nx, ny = pr.ny, nz = pr.nz;
  switch (stage) {
    case kStageMomentum:
      return part == 0 ? (nx + 1) * ny * nz : part == 1 ? nx * (ny + 1) * nz : nx * ny * (nz + 1);
    case kStageProject: return project_size(pr);
    default: return nx * ny * nz;
  }
}

cudaError_t launch_packed_rows(int stage, const CaseRows* cases, const PackedTile* tiles, int ntiles, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  switch (stage) {
    case kStageMomentum: k_packed_rows<kStageMomentum><<<ntiles, kBlockA, 0, st>>>(cases, tiles); break;
    case kStageRhs: k_packed_rows<kStageRhs><<<ntiles, kBlockA, 0, st>>>(cases, tiles); break;
    case kStageProject: k_packed_rows<kStageProject><<<ntiles, kBlockA, 0, st>>>(cases, tiles); break;
    case kStageSolute: k_packed_rows<kStageSolute><<<ntiles, kBlockA, 0, st>>>(cases, tiles); break;
    case kStageTemperature: k_packed_rows<kStageTemperature><<<ntiles, kBlockA, 0, st>>>(cases, tiles); break;
    case kStageLever: k_packed_rows<kStageLever><<<ntiles, kBlockA, 0, st>>>(cases, tiles); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_to_f32(const double* src, float* dst, long long n, cudaStream_t st) {
  k_to_f32<<<grid_for(n), kBlockA, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_forward_assemble(int sys, const Params& pr, const Sys& sy, const double* const vel[3],
                                    const double* p, const double* T, const double* C, const double* Cl,
                                    const double* gl, const double* Kinv, const double* Ag, const double* time,
                                    cudaStream_t st) {
  const int g = grid_for(sy.d.n);
  switch (sys) {
    case SS_SYS_U: k_forward_momentum<0><<<g, kBlockA, 0, st>>>(pr, sy, vel[0], vel[1], vel[2], p, T, Cl, Kinv); break;
    case SS_SYS_V: k_forward_momentum<1><<<g, kBlockA, 0, st>>>(pr, sy, vel[0], vel[1], vel[2], p, T, Cl, Kinv); break;
    case SS_SYS_W: k_forward_momentum<2><<<g, kBlockA, 0, st>>>(pr, sy, vel[0], vel[1], vel[2], p, T, Cl, Kinv); break;
    case SS_SYS_C: k_forward_cells<true><<<g, kBlockA, 0, st>>>(pr, sy, vel[0], vel[1], vel[2], C, gl, Ag, time); break;
    case SS_SYS_T: k_forward_cells<false><<<g, kBlockA, 0, st>>>(pr, sy, vel[0], vel[1], vel[2], T, gl, Ag, time); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_assemble_momentum(int comp, const Params& pr, const Sys& sys, const double* const vel[3],
                                     double* ustar, const double* p, const double* T, const double* Cl,
                                     const double* Kinv, cudaStream_t st) {
  const int g = grid_for(sys.d.n);
  if (sys.af.P) {   // mixed path: double-float coefficients
    if (comp == 0)
      k_assemble_momentum_df<0><<<g, kBlockA, 0, st>>>(pr, sys, vel[0], vel[1], vel[2], ustar, p, T, Cl, Kinv);
    else if (comp == 1)
      k_assemble_momentum_df<1><<<g, kBlockA, 0, st>>>(pr, sys, vel[0], vel[1], vel[2], ustar, p, T, Cl, Kinv);
    else
      k_assemble_momentum_df<2><<<g, kBlockA, 0, st>>>(pr, sys, vel[0], vel[1], vel[2], ustar, p, T, Cl, Kinv);
    return cudaGetLastError();
  }
  if (comp == 0)
    k_assemble_momentum<0><<<g, kBlockA, 0, st>>>(pr, sys, vel[0], vel[1], vel[2], ustar, p, T, Cl, Kinv);
  else if (comp == 1)
    k_assemble_momentum<1><<<g, kBlockA, 0, st>>>(pr, sys, vel[0], vel[1], vel[2], ustar, p, T, Cl, Kinv);
  else
    k_assemble_momentum<2><<<g, kBlockA, 0, st>>>(pr, sys, vel[0], vel[1], vel[2], ustar, p, T, Cl, Kinv);
  return cudaGetLastError();
}

cudaError_t launch_assemble_solute(const Params& pr, const Sys& sys, const double* const vel[3], const double* gl,
                                   const double* C, const double* Ag, cudaStream_t st) {
  if (sys.af.P)
    k_assemble_cells_df<true><<<grid_for(sys.d.n), kBlockA, 0, st>>>(pr, sys, vel[0], vel[1], vel[2],
                                                                     const_cast<double*>(C), gl, Ag, nullptr,
                                                                     nullptr, 0);
  else
    k_assemble_cells<true><<<grid_for(sys.d.n), kBlockA, 0, st>>>(pr, sys, vel[0], vel[1], vel[2],
                                                                  const_cast<double*>(C), gl, Ag, nullptr, nullptr, 0);
  return cudaGetLastError();
}

cudaError_t launch_assemble_temperature(const Params& pr, const Sys& sys, const double* const vel[3],
                                        const double* time, double* T, double* Tinc, int use_guess,
                                        cudaStream_t st) {
  if (sys.af.P)
    k_assemble_cells_df<false><<<grid_for(sys.d.n), kBlockA, 0, st>>>(pr, sys, vel[0], vel[1], vel[2], T, nullptr,
                                                                      nullptr, time, Tinc, use_guess);
  else
    k_assemble_cells<false><<<grid_for(sys.d.n), kBlockA, 0, st>>>(pr, sys, vel[0], vel[1], vel[2], T, nullptr,
                                                                   nullptr, time, Tinc, use_guess);
  return cudaGetLastError();
}

cudaError_t launch_poisson_rhs(const Params& pr, const double* const ustar[3], double* b, cudaStream_t st) {
  const long long n = (long long)pr.nx * pr.ny * pr.nz;
  k_poisson_rhs<<<grid_for(n), kBlockA, 0, st>>>(pr, ustar[0], ustar[1], ustar[2], b);
  return cudaGetLastError();
}

cudaError_t launch_project(const Params& pr, double* const vel[3], const double* const ustar[3], const double* pc,
                           double* p, cudaStream_t st) {
  const long long total = project_size(pr);
  k_project<<<grid_for(total), kBlockA, 0, st>>>(pr, vel[0], vel[1], vel[2], ustar[0], ustar[1], ustar[2], pc, p);
  return cudaGetLastError();
}

cudaError_t launch_lever(const Params& pr, double* time, double* T, double* gl, const double* C, double* Cl,
                         double* Cs, double* Kinv, double* Ag, double* Tinc, int form_inc, cudaStream_t st) {
  const int n = pr.nx * pr.ny * pr.nz;
  k_lever<<<grid_for(n), kBlockA, 0, st>>>(pr, time, T, gl, C, Cl, Cs, Kinv, Ag, n, Tinc, form_inc);
  return cudaGetLastError();
}

cudaError_t launch_equilibrate(const Params& pr, const double* T, const double* C, double* gl, double* Cl,
                               double* Cs, double* Kinv, double* Ag, int from_T, int write_cl, cudaStream_t st) {
  const int n = pr.nx * pr.ny * pr.nz;
  k_equilibrate<<<grid_for(n), kBlockA, 0, st>>>(pr, T, C, gl, Cl, Cs, Kinv, Ag, n, from_T, write_cl);
  return cudaGetLastError();
}

}  // namespace solid
