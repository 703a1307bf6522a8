// Persistent Krylov solvers for the DIA systems of one step.
//
// Each solve is ONE cooperative launch: every block stays resident for the
// whole solve, owns a fixed grid-stride set of rows, and meets the others at
// grid barriers between dependent phases. Dot products are reduced
// deterministically (warp shuffles, then per-block partials summed in block
// order by every block), so every block takes the same convergence decision
// and the result does not depend on timing. Convergence is checked on the
// device; the host never waits inside a solve.
//
//   k_bicgstab      Jacobi-preconditioned BiCGSTAB for the nonsymmetric
//                   transport systems (u*, v*, w*: Eq. 3.3; C: Eq. 3.10;
//                   T*: Eq. 3.12) stored as 5/7 DIA planes (Eq. 4.1).
//   k_pcg_poisson   Jacobi-preconditioned CG for the pressure correction
//                   (Eq. 3.4): the constant-coefficient Neumann Laplacian is
//                   applied matrix-free (term-wise strategy of Sec. 4: the
//                   operator never changes, so it is never assembled).
//
// Vectors that other blocks write during the solve (the SpMV operands) are
// read with plain L1-cached loads: they are read only after a grid barrier,
// whose acquire makes the other blocks' writes visible. The DIA planes do
// not change during a solve and use the read-only path.
#include <cstring>
#include <mutex>

#include "solid_internal.cuh"

namespace solid {
namespace {

template <typename T>
struct BcgVec {
  T *r, *rh, *p, *v, *y, *z, *t;
};

// vectors of the fused FP32 inner solve (bcg_fused): r/s pair, rhat, p pair, v pair, t
struct FusedVec {
  float *r0, *r1, *rh, *p0, *p1, *v0, *v1, *t;
};

struct BcgArgs {
  Sys sys;
  int has_z;
  double tol;
  int max_it;
  int stat_index;
  double inner_tol;        // relative tolerance of each FP32 inner solve (mixed path)
  BcgVec<double> v64;
  FusedVec f32;            // vectors of the fused FP32 inner solve (mixed path)
  float* d32;              // inner correction (mixed path)
  double* partial;
  int max_blocks;
  DevStatus* st;
  int after_presolve;      // 1: the T* pre-solve ran before this launch and may have met tol
  int jacobi;              // 1: FP64 Jacobi sweeps first (jacobi64)
};

template <typename T>
__device__ __forceinline__ T spmv_row(const Planes<T>& a, const T* x, int r, int sy, int sz, int has_z) {
  T acc = __ldg(a.P + r) * x[r];
  acc = fma(__ldg(a.W + r), x[r - 1], acc);
  acc = fma(__ldg(a.E + r), x[r + 1], acc);
  acc = fma(__ldg(a.S + r), x[r - sy], acc);
  acc = fma(__ldg(a.N + r), x[r + sy], acc);
  if (has_z) {
    acc = fma(__ldg(a.B + r), x[r - sz], acc);
    acc = fma(__ldg(a.T_ + r), x[r + sz], acc);
  }
  return acc;
}

// b_r - (A x)_r in FP64 with each product fused into the running difference
// (one FP64 operation per coefficient: the refinement residuals' FP64 work)
__device__ __forceinline__ double res_row64(double br, const Planes<double>& a, const double* x, int r, int sy,
                                            int sz, int has_z) {
  double acc = fma(-__ldg(a.P + r), x[r], br);
  acc = fma(-__ldg(a.W + r), x[r - 1], acc);
  acc = fma(-__ldg(a.E + r), x[r + 1], acc);
  acc = fma(-__ldg(a.S + r), x[r - sy], acc);
  acc = fma(-__ldg(a.N + r), x[r + sy], acc);
  if (has_z) {
    acc = fma(-__ldg(a.B + r), x[r - sz], acc);
    acc = fma(-__ldg(a.T_ + r), x[r + sz], acc);
  }
  return acc;
}

// Solve statistics, written by thread 0 of the leading block of the solving team.
__device__ void record(DevStatus* st, bool leader, int idx, int iters, int refinements, bool converged,
                       double relres, int jacobi = 0) {
  if (leader && threadIdx.x == 0) {
    SolveStat& s = st->stat[idx];
    s.iters = iters;
    s.iters_total += iters;
    s.jacobi = jacobi;
    s.jacobi_total += jacobi;
    s.refinements = refinements;
    s.converged = converged ? 1 : 0;
    s.nonfinite = isfinite(relres) ? 0 : 1;
    s.relres = relres;
    if (!isfinite(relres)) atomicExch(&st->sticky, (int)SS_ENAN);
    else if (!converged) atomicCAS(&st->sticky, (int)SS_OK, (int)SS_ENOTCONV);
  }
}

// float4 views for the FP32 streaming passes (every vector starts on a
// 256-byte boundary); n4 = n / 4 items, then a scalar tail.
__device__ __forceinline__ float4 ld4(const float* p, int m) { return reinterpret_cast<const float4*>(p)[m]; }
__device__ __forceinline__ float4 ldg4(const float* p, int m) { return __ldg(reinterpret_cast<const float4*>(p) + m); }
__device__ __forceinline__ void st4(float* p, int m, float4 v) { reinterpret_cast<float4*>(p)[m] = v; }

struct CoreOut {
  int it;
  bool conv;
  double res, bnorm;
  // bcg_fused: the solve stopped on the half step, and its correction is
  // x + al D^-1 p (x read as 0 when it == 1), formed where the caller reads it;
  // jac_fused: the sweeps stalled, and p is the buffer holding the correction
  bool half = false;
  float al = 0.f;
  const float* p = nullptr;
  bool x_done = false;   // jac_fused: the correction was already added to the FP64 iterate
};

// The BiCGSTAB scalars, formed by thread 0 of each block after each
// reduction (every block forms the same values from the same totals); the
// vector passes read them from shared memory.
template <typename T>
struct BcgScalars {
  double rho, alpha, omega, res, bnorm;
  T beta, om, al, omn;
  int state;   // 0: iterate on; 1: converged on the half step; 2: stop
  int conv;
};

// Jacobi-preconditioned BiCGSTAB on A x = b in precision T (the FP64 solver;
// the mixed path's FP32 inner solve is bcg_fused). zero_x0: start from x = 0
// without the initial SpMV. Block and grid reductions are FP64 and
// deterministic.
// Reduction slots 0..7. Returns false if a grid barrier gave up.
template <typename T>
__device__ bool bcg_core(const Planes<T>& a, int n, int sy, int sz, int has_z, const T* b, T* x, bool zero_x0,
                         const BcgVec<T>& V, double tol, int max_it, const Team& tm, int max_blocks, DevStatus* st,
                         unsigned int& epoch, CoreOut& out) {
  const int t0 = tm.rank * blockDim.x + threadIdx.x, gs = tm.size * blockDim.x;
  T *r = V.r, *rh = V.rh, *p = V.p, *v = V.v, *y = V.y, *z = V.z, *t = V.t;
  Vec<2> acc = {{0.0, 0.0}};
  {
    T a0 = T(0), a1 = T(0);
    for (int i = t0; i < n; i += gs) {          // r = b - A x0, rhat = r
      const T bi = b[i];
      const T ri = zero_x0 ? bi : bi - spmv_row(a, x, i, sy, sz, has_z);
      if (zero_x0) x[i] = T(0);
      r[i] = ri;
      rh[i] = ri;
      p[i] = T(0);
      v[i] = T(0);
      a0 += ri * ri;
      a1 += bi * bi;
    }
    acc.v[0] = (double)a0;
    acc.v[1] = (double)a1;
  }
  __shared__ BcgScalars<T> ks;
  double thr = 0.0;                               // read by thread 0 only
  if (!team_sum_post<2>(acc, tm, max_blocks, 6, st, epoch, [&](const double* tot) {
        ks.bnorm = sqrt(tot[1]);
        ks.res = sqrt(tot[0]);
        thr = tol * ks.bnorm;
        ks.rho = tot[0];
        ks.alpha = 1.0;
        ks.omega = 1.0;
        ks.beta = (T)ks.rho;                      // (rho / 1) (1 / 1); p = v = 0, so p = r
        ks.om = T(1);
        ks.conv = ks.res <= thr;
        ks.state = (ks.bnorm == 0.0 || ks.conv || max_it <= 0 || !isfinite(ks.res)) ? 2 : 0;
      }))
    return false;
  out.bnorm = ks.bnorm;
  out.it = 0;
  if (out.bnorm == 0.0) {
    if (!zero_x0)
      for (int i = t0; i < n; i += gs) x[i] = T(0);
    out.conv = true;
    out.res = 0.0;
    return true;
  }
  int it = 0;
  while (ks.state == 0) {
    ++it;
    const T beta = ks.beta, om = ks.om;
    for (int i = t0; i < n; i += gs) {          // p = r + beta (p - omega v); y = M^-1 p
      const T pi = r[i] + beta * (p[i] - om * v[i]);
      p[i] = pi;
      y[i] = __ldg(a.idiag + i) * pi;
    }
    if (!team_barrier(st, tm, epoch)) return false;
    T s1 = T(0);
    for (int i = t0; i < n; i += gs) {          // v = A y
      const T vi = spmv_row(a, y, i, sy, sz, has_z);
      v[i] = vi;
      s1 += rh[i] * vi;
    }
    if (!team_sum_post<1>(Vec<1>{{(double)s1}}, tm, max_blocks, 0, st, epoch, [&](const double* tot) {
          ks.alpha = ks.rho / tot[0];
          ks.al = (T)ks.alpha;
        }))
      return false;
    const T al = ks.al;
    T s2 = T(0);
    for (int i = t0; i < n; i += gs) {          // s = r - alpha v (in r); z = M^-1 s
      const T si = r[i] - al * v[i];
      r[i] = si;
      z[i] = __ldg(a.idiag + i) * si;
      s2 += si * si;
    }
    if (!team_sum_post<1>(Vec<1>{{(double)s2}}, tm, max_blocks, 1, st, epoch, [&](const double* tot) {
          const double rs = sqrt(tot[0]);
          if (rs <= thr) {                        // early exit on the half step
            ks.res = rs;
            ks.conv = 1;
            ks.state = 1;
          }
        }))
      return false;
    if (ks.state == 1) {
      for (int i = t0; i < n; i += gs) x[i] += al * y[i];
      break;
    }
    T s3 = T(0), s4 = T(0);
    for (int i = t0; i < n; i += gs) {          // t = A z
      const T ti = spmv_row(a, z, i, sy, sz, has_z);
      t[i] = ti;
      s3 += ti * r[i];
      s4 += ti * ti;
    }
    if (!team_sum_post<2>(Vec<2>{{(double)s3, (double)s4}}, tm, max_blocks, 2, st, epoch, [&](const double* tot) {
          ks.omega = (tot[1] > 0.0) ? tot[0] / tot[1] : 0.0;
          ks.omn = (T)ks.omega;
        }))
      return false;
    const T omn = ks.omn;
    T s5 = T(0), s6 = T(0);
    for (int i = t0; i < n; i += gs) {          // x += alpha y + omega z; r = s - omega t
      x[i] += al * y[i] + omn * z[i];
      const T ri = r[i] - omn * t[i];
      r[i] = ri;
      s5 += rh[i] * ri;
      s6 += ri * ri;
    }
    if (!team_sum_post<2>(Vec<2>{{(double)s5, (double)s6}}, tm, max_blocks, 4, st, epoch, [&](const double* tot) {
          ks.res = sqrt(tot[1]);
          ks.conv = ks.res <= thr;
          const double rho_old = ks.rho;
          ks.rho = tot[0];
          ks.beta = (T)((ks.rho / rho_old) * (ks.alpha / ks.omega));
          ks.om = (T)ks.omega;
          // stop on convergence, the iteration cap, a non-finite residual or
          // a breakdown (rho = 0 or omega = 0: the current iterate is reported)
          ks.state = (ks.conv || it >= max_it || !isfinite(ks.res) || ks.rho == 0.0 || ks.omega == 0.0) ? 2 : 0;
        }))
      return false;
  }
  out.it = it;
  out.conv = ks.conv != 0;
  out.res = ks.res;
  return true;
}

// ---- FP32 inner solve with three grid-wide synchronisations per iteration.
//
// The same Jacobi-preconditioned BiCGSTAB as bcg_core, in FP32, with the
// preconditioned vectors never stored: y = D^-1 (r + beta (p - omega v)) and
// z = D^-1 (r - alpha v) are formed wherever the SpMV needs them (the row and
// its six neighbours), from vectors that are complete after the previous
// reduction. So the p and y update merges into v = A y, and the s and z
// update into t = A z: per iteration three passes and three reductions
// instead of five. Every pass writes only buffers that no thread reads in
// the same pass: p and v alternate between two buffers each, r and s share
// a pair (s is written beside r; the new r overwrites s in place, row by row).
// The FP64 solver keeps bcg_core: forming y and z at seven points would cost
// FP64-pipe work that the saved passes do not repay.
struct YDir {   // y = D^-1 (r + beta (p - om v))
  const float *r, *p, *v, *d;
  float beta, om;
  __device__ __forceinline__ float at(int q) const { return d[q] * (r[q] + beta * (p[q] - om * v[q])); }
  __device__ __forceinline__ float4 at4(int q) const {   // q multiple of 4
    const float4 a = *reinterpret_cast<const float4*>(r + q), b = *reinterpret_cast<const float4*>(p + q);
    const float4 c = *reinterpret_cast<const float4*>(v + q), e = __ldg(reinterpret_cast<const float4*>(d + q));
    return make_float4(e.x * (a.x + beta * (b.x - om * c.x)), e.y * (a.y + beta * (b.y - om * c.y)),
                       e.z * (a.z + beta * (b.z - om * c.z)), e.w * (a.w + beta * (b.w - om * c.w)));
  }
};

struct Y1Dir {  // the first direction y = D^-1 r0, r0 = sc r32 (p = v = 0)
  const float *r, *d;
  float sc;
  __device__ __forceinline__ float at(int q) const { return d[q] * (r[q] * sc); }
  __device__ __forceinline__ float4 at4(int q) const {
    const float4 a = *reinterpret_cast<const float4*>(r + q), e = __ldg(reinterpret_cast<const float4*>(d + q));
    return make_float4(e.x * (a.x * sc), e.y * (a.y * sc), e.z * (a.z * sc), e.w * (a.w * sc));
  }
};

struct ZDir {   // z = D^-1 (r - al v)
  const float *r, *v, *d;
  float al;
  __device__ __forceinline__ float at(int q) const { return d[q] * (r[q] - al * v[q]); }
  __device__ __forceinline__ float4 at4(int q) const {
    const float4 a = *reinterpret_cast<const float4*>(r + q), c = *reinterpret_cast<const float4*>(v + q);
    const float4 e = __ldg(reinterpret_cast<const float4*>(d + q));
    return make_float4(e.x * (a.x - al * c.x), e.y * (a.y - al * c.y), e.z * (a.z - al * c.z),
                       e.w * (a.w - al * c.w));
  }
};

template <class F>
__device__ __forceinline__ float4 dir4(const F& f, int q, bool aligned) {
  if (aligned) return f.at4(q);
  return make_float4(f.at(q), f.at(q + 1), f.at(q + 2), f.at(q + 3));
}

// rows 4m..4m+3 of A f, the centre values xc given (same order of operations as spmv4)
template <class F>
__device__ __forceinline__ float4 spmv4_dir(const Planes<float>& a, const F& f, float4 xc, int m, int sy, int sz,
                                            int has_z, bool ay, bool az) {
  const int r = 4 * m;
  const float4 P = ldg4(a.P, m), W = ldg4(a.W, m), E = ldg4(a.E, m), S = ldg4(a.S, m), N = ldg4(a.N, m);
  const float xw = f.at(r - 1), xe = f.at(r + 4);
  const float4 xs = dir4(f, r - sy, ay), xn = dir4(f, r + sy, ay);
  float4 o;
  o.x = P.x * xc.x; o.y = P.y * xc.y; o.z = P.z * xc.z; o.w = P.w * xc.w;
  o.x = fmaf(W.x, xw, o.x); o.y = fmaf(W.y, xc.x, o.y); o.z = fmaf(W.z, xc.y, o.z); o.w = fmaf(W.w, xc.z, o.w);
  o.x = fmaf(E.x, xc.y, o.x); o.y = fmaf(E.y, xc.z, o.y); o.z = fmaf(E.z, xc.w, o.z); o.w = fmaf(E.w, xe, o.w);
  o.x = fmaf(S.x, xs.x, o.x); o.y = fmaf(S.y, xs.y, o.y); o.z = fmaf(S.z, xs.z, o.z); o.w = fmaf(S.w, xs.w, o.w);
  o.x = fmaf(N.x, xn.x, o.x); o.y = fmaf(N.y, xn.y, o.y); o.z = fmaf(N.z, xn.z, o.z); o.w = fmaf(N.w, xn.w, o.w);
  if (has_z) {
    const float4 B = ldg4(a.B, m), T = ldg4(a.T_, m);
    const float4 xb = dir4(f, r - sz, az), xt = dir4(f, r + sz, az);
    o.x = fmaf(B.x, xb.x, o.x); o.y = fmaf(B.y, xb.y, o.y); o.z = fmaf(B.z, xb.z, o.z); o.w = fmaf(B.w, xb.w, o.w);
    o.x = fmaf(T.x, xt.x, o.x); o.y = fmaf(T.y, xt.y, o.y); o.z = fmaf(T.z, xt.z, o.z); o.w = fmaf(T.w, xt.w, o.w);
  }
  return o;
}

template <class F>
__device__ __forceinline__ float spmv_dir(const Planes<float>& a, const F& f, float xc, int r, int sy, int sz,
                                          int has_z) {
  float acc = __ldg(a.P + r) * xc;
  acc = fmaf(__ldg(a.W + r), f.at(r - 1), acc);
  acc = fmaf(__ldg(a.E + r), f.at(r + 1), acc);
  acc = fmaf(__ldg(a.S + r), f.at(r - sy), acc);
  acc = fmaf(__ldg(a.N + r), f.at(r + sy), acc);
  if (has_z) {
    acc = fmaf(__ldg(a.B + r), f.at(r - sz), acc);
    acc = fmaf(__ldg(a.T_ + r), f.at(r + sz), acc);
  }
  return acc;
}

__device__ __forceinline__ float dot4(float4 a, float4 b) { return (a.x * b.x + a.y * b.y) + (a.z * b.z + a.w * b.w); }

// A x = r0 from x = 0 in FP32, r0 = sc r32 with r32 the caller's FP32 copy
// of its residual in V.t (read only by the first pass; pass 2 reuses V.t).
// The first iteration starts from p = v = 0, so its pass 1 also stages r0,
// rhat and p' = r0 and reduces (r0, r0) beside (rhat, v'): no separate
// initialisation pass or reduction, and x is first written (not updated) in
// its pass 3. A solve that converges on the half step leaves its last update
// x + al D^-1 p' to the caller (out.half, out.al, out.p). out.it == 0 means
// the correction is zero (already converged, or no iterations allowed).
// Reduction slots 0..7, like bcg_core.
__device__ bool bcg_fused(const Planes<float>& a, int n, int sy, int sz, int has_z, float* x, FusedVec V, float sc,
                          double tol, int max_it, const Team& tm, int max_blocks, DevStatus* st,
                          unsigned int& epoch, CoreOut& out) {
  const int t0 = tm.rank * blockDim.x + threadIdx.x, gs = tm.size * blockDim.x;
  const int n4 = n >> 2, tail = n4 << 2;
  const bool ay = (sy & 3) == 0, az = (sz & 3) == 0;
  float *R = V.r0, *S = V.r1, *Po = V.p0, *Pn = V.p1, *Vo = V.v0, *Vn = V.v1;
  const float* rh = V.rh;
  const float* dg = a.idiag;
  __shared__ BcgScalars<float> ks;
  double thr = 0.0;                               // read by thread 0 only
  {
    // pass 1 of iteration 1: r0 = sc r32, rhat = p' = r0, v' = A D^-1 p', (rhat, v'), (r0, r0)
    const float* r32 = V.t;
    const Y1Dir yd{r32, dg, sc};
    float s1 = 0.f, a0 = 0.f;
    for (int m = t0; m < n4; m += gs) {
      const float4 q = ld4(r32, m), dv = ldg4(dg, m);
      const float4 rv = make_float4(q.x * sc, q.y * sc, q.z * sc, q.w * sc);
      st4(R, m, rv);
      st4(V.rh, m, rv);
      st4(Pn, m, rv);
      const float4 yc = make_float4(dv.x * rv.x, dv.y * rv.y, dv.z * rv.z, dv.w * rv.w);
      const float4 vn = spmv4_dir(a, yd, yc, m, sy, sz, has_z, ay, az);
      st4(Vn, m, vn);
      s1 += dot4(rv, vn);
      a0 += dot4(rv, rv);
    }
    for (int i = tail + t0; i < n; i += gs) {
      const float ri = r32[i] * sc;
      R[i] = ri;
      V.rh[i] = ri;
      Pn[i] = ri;
      const float vn = spmv_dir(a, yd, __ldg(dg + i) * ri, i, sy, sz, has_z);
      Vn[i] = vn;
      s1 += ri * vn;
      a0 += ri * ri;
    }
    if (!team_sum_post<2>(VecF<2>{{s1, a0}}, tm, max_blocks, 6, st, epoch, [&](const double* tot) {
          ks.bnorm = sqrt(tot[1]);
          ks.res = ks.bnorm;
          thr = tol * ks.bnorm;
          ks.rho = tot[1];
          ks.omega = 1.0;
          ks.conv = ks.bnorm == 0.0 || ks.res <= thr;
          ks.state = (ks.conv || max_it <= 0 || !isfinite(ks.res)) ? 2 : 0;
          ks.alpha = ks.rho / tot[0];
          ks.al = (float)ks.alpha;
        }))
      return false;
  }
  out.bnorm = ks.bnorm;
  out.half = false;
  if (ks.state != 0) {
    out.it = 0;
    out.conv = ks.conv != 0;
    out.res = ks.res;
    return true;
  }
  int it = 1;
  while (true) {
    if (it > 1) {
      const float beta = ks.beta, om = ks.om;
      // pass 1: p' = r + beta (p - om v) (stored), v' = A D^-1 p', (rhat, v')
      const YDir yd{R, Po, Vo, dg, beta, om};
      float s1 = 0.f;
      for (int m = t0; m < n4; m += gs) {
        const float4 rv = ld4(R, m), pv = ld4(Po, m), vv = ld4(Vo, m), dv = ldg4(dg, m);
        float4 pn;
        pn.x = rv.x + beta * (pv.x - om * vv.x); pn.y = rv.y + beta * (pv.y - om * vv.y);
        pn.z = rv.z + beta * (pv.z - om * vv.z); pn.w = rv.w + beta * (pv.w - om * vv.w);
        st4(Pn, m, pn);
        const float4 yc = make_float4(dv.x * pn.x, dv.y * pn.y, dv.z * pn.z, dv.w * pn.w);
        const float4 vn = spmv4_dir(a, yd, yc, m, sy, sz, has_z, ay, az);
        st4(Vn, m, vn);
        s1 += dot4(ld4(rh, m), vn);
      }
      for (int i = tail + t0; i < n; i += gs) {
        const float pn = R[i] + beta * (Po[i] - om * Vo[i]);
        Pn[i] = pn;
        const float vn = spmv_dir(a, yd, __ldg(dg + i) * pn, i, sy, sz, has_z);
        Vn[i] = vn;
        s1 += rh[i] * vn;
      }
      if (!team_sum_post<1>(VecF<1>{{s1}}, tm, max_blocks, 0, st, epoch, [&](const double* tot) {
            ks.alpha = ks.rho / tot[0];
            ks.al = (float)ks.alpha;
          }))
        return false;
    }
    const float al = ks.al;
    // pass 2: s = r - al v' (stored beside r), t = A D^-1 s, (t,s), (t,t), (s,s)
    const ZDir zd{R, Vn, dg, al};
    float s3 = 0.f, s4 = 0.f, s2 = 0.f;
    for (int m = t0; m < n4; m += gs) {
      const float4 rv = ld4(R, m), vv = ld4(Vn, m), dv = ldg4(dg, m);
      const float4 sv = make_float4(rv.x - al * vv.x, rv.y - al * vv.y, rv.z - al * vv.z, rv.w - al * vv.w);
      st4(S, m, sv);
      const float4 zc = make_float4(dv.x * sv.x, dv.y * sv.y, dv.z * sv.z, dv.w * sv.w);
      const float4 tv = spmv4_dir(a, zd, zc, m, sy, sz, has_z, ay, az);
      st4(V.t, m, tv);
      s3 += dot4(tv, sv);
      s4 += dot4(tv, tv);
      s2 += dot4(sv, sv);
    }
    for (int i = tail + t0; i < n; i += gs) {
      const float si = R[i] - al * Vn[i];
      S[i] = si;
      const float ti = spmv_dir(a, zd, __ldg(dg + i) * si, i, sy, sz, has_z);
      V.t[i] = ti;
      s3 += ti * si;
      s4 += ti * ti;
      s2 += si * si;
    }
    if (!team_sum_post<3>(VecF<3>{{s3, s4, s2}}, tm, max_blocks, 2, st, epoch, [&](const double* tot) {
          const double rs = sqrt(tot[2]);
          if (rs <= thr) {                        // converged on the half step
            ks.res = rs;
            ks.conv = 1;
            ks.state = 1;
          } else {
            ks.omega = (tot[1] > 0.0) ? tot[0] / tot[1] : 0.0;
            ks.omn = (float)ks.omega;
          }
        }))
      return false;
    if (ks.state == 1) {                           // x + al D^-1 p', formed by the caller
      out.half = true;
      out.al = al;
      out.p = Pn;
      break;
    }
    const float omn = ks.omn;
    // pass 3: x += al D^-1 p' + omn D^-1 s (x = ... on iteration 1); r = s - omn t (over s);
    // (rhat, r), (r, r)
    const bool first = it == 1;
    float s5 = 0.f, s6 = 0.f;
    for (int m = t0; m < n4; m += gs) {
      const float4 xv = first ? make_float4(0.f, 0.f, 0.f, 0.f) : ld4(x, m);
      const float4 pv = ld4(Pn, m), sv = ld4(S, m), tv = ld4(V.t, m), dv = ldg4(dg, m);
      float4 xo, ro;
      xo.x = fmaf(omn, dv.x * sv.x, fmaf(al, dv.x * pv.x, xv.x));
      xo.y = fmaf(omn, dv.y * sv.y, fmaf(al, dv.y * pv.y, xv.y));
      xo.z = fmaf(omn, dv.z * sv.z, fmaf(al, dv.z * pv.z, xv.z));
      xo.w = fmaf(omn, dv.w * sv.w, fmaf(al, dv.w * pv.w, xv.w));
      ro.x = sv.x - omn * tv.x; ro.y = sv.y - omn * tv.y; ro.z = sv.z - omn * tv.z; ro.w = sv.w - omn * tv.w;
      st4(x, m, xo);
      st4(S, m, ro);
      s5 += dot4(ld4(rh, m), ro);
      s6 += dot4(ro, ro);
    }
    for (int i = tail + t0; i < n; i += gs) {
      const float di = __ldg(dg + i);
      x[i] = fmaf(omn, di * S[i], fmaf(al, di * Pn[i], first ? 0.f : x[i]));
      const float ri = S[i] - omn * V.t[i];
      S[i] = ri;
      s5 += rh[i] * ri;
      s6 += ri * ri;
    }
    if (!team_sum_post<2>(VecF<2>{{s5, s6}}, tm, max_blocks, 4, st, epoch, [&](const double* tot) {
          ks.res = sqrt(tot[1]);
          ks.conv = ks.res <= thr;
          const double rho_old = ks.rho;
          ks.rho = tot[0];
          ks.beta = (float)((ks.rho / rho_old) * (ks.alpha / ks.omega));
          ks.om = (float)ks.omega;
          // stop on convergence, the iteration cap, a non-finite residual or
          // a breakdown (rho = 0 or omega = 0: the current iterate is reported)
          ks.state = (ks.conv || it >= max_it || !isfinite(ks.res) || ks.rho == 0.0 || ks.omega == 0.0) ? 2 : 0;
        }))
      return false;
    if (ks.state != 0) break;
    float* tmp = R; R = S; S = tmp;               // the new r lives in S
    tmp = Po; Po = Pn; Pn = tmp;
    tmp = Vo; Vo = Vn; Vn = tmp;
    ++it;
  }
  out.it = it;
  out.conv = ks.conv != 0;
  out.res = ks.res;
  return true;
}

// FP64 Jacobi sweeps x <- x + D^-1 (b - A x) ahead of the Krylov solve of a
// transport system. Where 1/dt outweighs convection and diffusion the rows
// are strongly diagonally dominant (Eq. 3.3 and 3.10: on the 128x96x96 box
// a sweep reduces the residual ~50-fold for the momentum components and
// ~3000-fold for the solute), and a sweep reads each row's FP64 planes once,
// where a refinement sweep of the mixed solve needs its FP32 iterations and
// an FP64 update pass. Sweep k forms r_k = b - A x_k and x_{k+1} in one pass,
// ping-ponging between x and the residual vector, and reduces |r_k|:
//   |r_k| <= tol |b|: x_k is the solution (copied into x if it sits in the
//     scratch vector); returns 1;
//   |r_k| > kJacobiRate |r_{k-1}|, or kJacobiMax sweeps: the sweeps stop and
//     x_{k+1} (in x) is the Krylov solve's initial guess; returns 0;
//   a barrier gave up: returns -1.
// This is the FP64 path's form; the mixed path runs the same sweeps in FP32
// inside its FP64 refinement (jac_fused).
constexpr double kJacobiRate = 0.05;   // per-sweep reduction below which BiCGSTAB is faster
constexpr int kJacobiMax = 40;

__device__ int jacobi64(const BcgArgs& A, const Team& tm, unsigned int& epoch, int& sweeps, double& rel) {
  const int n = (int)A.sys.d.n;
  const int sy = A.sys.d.mx, sz = A.sys.d.mx * A.sys.d.my;
  const int t0 = tm.rank * blockDim.x + threadIdx.x, gs = tm.size * blockDim.x;
  const Planes<double>& a = A.sys.a;
  const double* b = A.sys.b;
  double* const x0 = A.sys.x;
  double* const x1 = A.v64.r;   // every scratch set has it; the Krylov solve writes it only after the sweeps
  __shared__ struct {
    double bn, rn, rel;
    int state;   // 0 sweep on, 1 converged on x_k, 2 hand x_{k+1} to the Krylov solve
  } js;
  double thr = 0.0, prev = 0.0;   // read by thread 0 only
  int k = 0;
  while (true) {
    const double* xk = (k & 1) ? x1 : x0;
    double* xn = (k & 1) ? x0 : x1;
    Vec<2> acc = {{0.0, 0.0}};
    for (int r = t0; r < n; r += gs) {
      const double rr = res_row64(b[r], a, xk, r, sy, sz, A.has_z);
      const double dinv = __ldg(a.idiag + r);
      xn[r] = fma(dinv, rr, xk[r]);
      acc.v[0] += rr * rr;
      if (k == 0) acc.v[1] += b[r] * b[r];
    }
    if (!team_sum_post<2>(acc, tm, A.max_blocks, (k & 1) ? 10 : 8, A.st, epoch, [&](const double* tot) {
          const double rn = sqrt(tot[0]);
          if (k == 0) {
            js.bn = sqrt(tot[1]);
            thr = A.tol * js.bn;
          }
          js.rn = rn;
          js.rel = js.bn > 0.0 ? rn / js.bn : 0.0;
          if (js.bn == 0.0 || rn <= thr) js.state = 1;
          else if (!isfinite(rn) || (k > 0 && rn > kJacobiRate * prev) || k + 1 >= kJacobiMax) js.state = 2;
          else js.state = 0;
          prev = rn;
        }))
      return -1;
    ++k;
    if (js.state == 0) continue;
    // the result (x_{k-1} when converged, else x_k) into x; the Krylov solve
    // reads x at neighbouring rows, hence the barrier after a copy
    const int src = (js.state == 1) ? ((k - 1) & 1) : (k & 1);
    if (src == 1) {
      for (int r = t0; r < n; r += gs) x0[r] = x1[r];
      if (js.state == 2 && !team_barrier(A.st, tm, epoch)) return -1;
    }
    sweeps = k;
    rel = js.rel;
    return js.state == 1 ? 1 : 0;
  }
}

__device__ __forceinline__ void fp64_solve(const BcgArgs& A, const Team& tm, unsigned int& epoch) {
  const int n = (int)A.sys.d.n;
  const int sy = A.sys.d.mx, sz = A.sys.d.mx * A.sys.d.my;
  int jac = 0;
  if (A.jacobi) {
    double rel = 0.0;
    const int j = jacobi64(A, tm, epoch, jac, rel);
    if (j < 0) return;
    if (j == 1) {
      record(A.st, tm.rank == 0, A.stat_index, 0, 0, true, rel, jac);
      return;
    }
  }
  CoreOut o;
  if (!bcg_core<double>(A.sys.a, n, sy, sz, A.has_z, A.sys.b, A.sys.x, false, A.v64, A.tol, A.max_it, tm,
                        A.max_blocks, A.st, epoch, o))
    return;
  record(A.st, tm.rank == 0, A.stat_index, o.it, 0, o.conv, o.bnorm > 0.0 ? o.res / o.bnorm : 0.0, jac);
}

// Mixed precision: FP64 iterative refinement around an FP32 inner solve on
// the FP32 copies of the planes: Jacobi sweeps (jac_fused) for the strongly
// diagonally dominant systems the caller marks, until they stall, else
// BiCGSTAB (bcg_fused). Each sweep solves A d = r / |r| in FP32 to the
// relative inner tolerance chosen per system by the caller, adds |r| d to the
// FP64 iterate and forms the true FP64 residual b - A x with the FP64 planes.
// It stops when that residual meets tol (the same test as the FP64 path). The
// pass that forms the residual also stores its FP32 copy, which the inner
// solve scales by 1/|r| as it reads it.
constexpr int kMaxRefine = 12;
// Inner iterations per refinement sweep: bounds a sweep whose FP32 iteration
// stalls (the outer FP64 loop then continues from the best iterate).
constexpr int kMaxInner = 200;
// A sweep's inner solve need not reduce its residual further than the outer
// tolerance still asks: it stops at max(inner_tol, kSweepMargin * thr / rn),
// thr the outer target and rn the current FP64 residual norm. The margin
// covers the FP32 operator's rounding, which the FP64 residual sees and the
// inner one does not.
constexpr double kSweepMargin = 0.1;
// The FP32 residual copy is scaled by 1/|r| in FP32 when |r| lies in
// [2^-60, 2^60]: no entry then overflows, and entries that fall below FP32's
// normal range are below 2^-66 |r|. Outside that range a pass restages the
// copy from the FP64 residual, scaled in FP64.
constexpr double kStageLo = 0x1p-60, kStageHi = 0x1p60;

// One FP32 Jacobi sweep d_{k+1} = d_k + D^-1 (r0 - A d_k), r0 = sc r32, on
// the rows of this thread; returns its part of |r0 - A d_k|^2 when REDUCE.
// XUPD: also x += rn d_{k+1} in FP64 for the same rows (the sweep that ends
// the inner solve adds the correction to the FP64 iterate).
template <bool REDUCE, bool XUPD>
__device__ __forceinline__ float jac_pass(const Planes<float>& a, int n, int sy, int sz, int has_z, const float* dk,
                                          float* dn, const float* r32, float sc, int t0, int gs, double* x64,
                                          double rn) {
  const int n4 = n >> 2, tail = n4 << 2;
  const bool ay = (sy & 3) == 0, az = (sz & 3) == 0;
  const float* dg = a.idiag;
  float s2 = 0.f;
  for (int m = t0; m < n4; m += gs) {
    const int r = 4 * m;
    const float4 P = ldg4(a.P, m), W = ldg4(a.W, m), E = ldg4(a.E, m), S = ldg4(a.S, m), N = ldg4(a.N, m);
    const float4 xc = ld4(dk, m);
    const float xw = dk[r - 1], xe = dk[r + 4];
    const float4 xs = ay ? ld4(dk, (r - sy) >> 2) : make_float4(dk[r - sy], dk[r - sy + 1], dk[r - sy + 2], dk[r - sy + 3]);
    const float4 xn = ay ? ld4(dk, (r + sy) >> 2) : make_float4(dk[r + sy], dk[r + sy + 1], dk[r + sy + 2], dk[r + sy + 3]);
    float4 o;
    o.x = P.x * xc.x; o.y = P.y * xc.y; o.z = P.z * xc.z; o.w = P.w * xc.w;
    o.x = fmaf(W.x, xw, o.x); o.y = fmaf(W.y, xc.x, o.y); o.z = fmaf(W.z, xc.y, o.z); o.w = fmaf(W.w, xc.z, o.w);
    o.x = fmaf(E.x, xc.y, o.x); o.y = fmaf(E.y, xc.z, o.y); o.z = fmaf(E.z, xc.w, o.z); o.w = fmaf(E.w, xe, o.w);
    o.x = fmaf(S.x, xs.x, o.x); o.y = fmaf(S.y, xs.y, o.y); o.z = fmaf(S.z, xs.z, o.z); o.w = fmaf(S.w, xs.w, o.w);
    o.x = fmaf(N.x, xn.x, o.x); o.y = fmaf(N.y, xn.y, o.y); o.z = fmaf(N.z, xn.z, o.z); o.w = fmaf(N.w, xn.w, o.w);
    if (has_z) {
      const float4 B = ldg4(a.B, m), T = ldg4(a.T_, m);
      const float4 xb = az ? ld4(dk, (r - sz) >> 2)
                           : make_float4(dk[r - sz], dk[r - sz + 1], dk[r - sz + 2], dk[r - sz + 3]);
      const float4 xt = az ? ld4(dk, (r + sz) >> 2)
                           : make_float4(dk[r + sz], dk[r + sz + 1], dk[r + sz + 2], dk[r + sz + 3]);
      o.x = fmaf(B.x, xb.x, o.x); o.y = fmaf(B.y, xb.y, o.y); o.z = fmaf(B.z, xb.z, o.z); o.w = fmaf(B.w, xb.w, o.w);
      o.x = fmaf(T.x, xt.x, o.x); o.y = fmaf(T.y, xt.y, o.y); o.z = fmaf(T.z, xt.z, o.z); o.w = fmaf(T.w, xt.w, o.w);
    }
    const float4 q = ld4(r32, m), dv = ldg4(dg, m);
    float4 sv;
    sv.x = fmaf(q.x, sc, -o.x); sv.y = fmaf(q.y, sc, -o.y); sv.z = fmaf(q.z, sc, -o.z); sv.w = fmaf(q.w, sc, -o.w);
    const float4 dnv = make_float4(fmaf(dv.x, sv.x, xc.x), fmaf(dv.y, sv.y, xc.y), fmaf(dv.z, sv.z, xc.z),
                                   fmaf(dv.w, sv.w, xc.w));
    st4(dn, m, dnv);
    if (REDUCE) s2 += dot4(sv, sv);
    if (XUPD) {
      x64[r] = fma(rn, (double)dnv.x, x64[r]);
      x64[r + 1] = fma(rn, (double)dnv.y, x64[r + 1]);
      x64[r + 2] = fma(rn, (double)dnv.z, x64[r + 2]);
      x64[r + 3] = fma(rn, (double)dnv.w, x64[r + 3]);
    }
  }
  for (int i = tail + t0; i < n; i += gs) {
    float acc = __ldg(a.P + i) * dk[i];
    acc = fmaf(__ldg(a.W + i), dk[i - 1], acc);
    acc = fmaf(__ldg(a.E + i), dk[i + 1], acc);
    acc = fmaf(__ldg(a.S + i), dk[i - sy], acc);
    acc = fmaf(__ldg(a.N + i), dk[i + sy], acc);
    if (has_z) {
      acc = fmaf(__ldg(a.B + i), dk[i - sz], acc);
      acc = fmaf(__ldg(a.T_ + i), dk[i + sz], acc);
    }
    const float si = fmaf(r32[i], sc, -acc);
    const float di = fmaf(__ldg(dg + i), si, dk[i]);
    dn[i] = di;
    if (REDUCE) s2 += si * si;
    if (XUPD) x64[i] = fma(rn, (double)di, x64[i]);
  }
  return s2;
}

// FP32 Jacobi sweeps for the inner solve A d = r0, r0 = sc r32 (unit norm;
// r32 is the caller's FP32 copy of its residual in V.t), for the strongly
// diagonally dominant transport systems (see jacobi64): d_1 = D^-1 r0 (no
// operator application), then d_{k+1} = d_k + D^-1 (r0 - A d_k). The first
// sweep reduces s_1 = |r0 - A d_1|, which is the sweeps' contraction rate
// rho: if s_1 <= tol the solve stops with d_2 (out.conv); if rho exceeds
// kJacobiRate it stops with d_2 and sets out.half as the stall flag (the
// caller's later sweeps use BiCGSTAB). Otherwise it runs the k sweeps for
// which (kJacobiMargin rho)^k <= tol with barriers only (no reductions), and
// the last of them adds rn d_{k+1} to the FP64 iterate x64 (out.x_done); the
// caller's FP64 residual then tells how far the correction went. d
// ping-pongs between x and V.p0; out.p is the result, out.it the iterates.
// Reduction slots 0..1.
constexpr double kJacobiMargin = 1.2;   // later sweeps contract a little less than the first
constexpr int kJacobiMaxPredicted = 16;
__device__ bool jac_fused(const Planes<float>& a, int n, int sy, int sz, int has_z, float* x, FusedVec V, float sc,
                          double tol, int max_it, const Team& tm, int max_blocks, DevStatus* st,
                          unsigned int& epoch, double* x64, double rn, CoreOut& out) {
  const int t0 = tm.rank * blockDim.x + threadIdx.x, gs = tm.size * blockDim.x;
  const int n4 = n >> 2, tail = n4 << 2;
  const float* r32 = V.t;
  const float* dg = a.idiag;
  float* const b0 = x;
  float* const b1 = V.p0;
  __shared__ struct {
    double res;
    int state;   // 0 predicted sweeps follow, 1 converged, 2 stalled
    int kpred;   // sweeps in all (the first included)
  } js;
  for (int m = t0; m < n4; m += gs) {             // d_1 = D^-1 r0
    const float4 q = ld4(r32, m), dv = ldg4(dg, m);
    st4(b0, m, make_float4(dv.x * (q.x * sc), dv.y * (q.y * sc), dv.z * (q.z * sc), dv.w * (q.w * sc)));
  }
  for (int i = tail + t0; i < n; i += gs) b0[i] = __ldg(dg + i) * (r32[i] * sc);
  out.half = false;
  out.x_done = false;
  out.bnorm = 1.0;
  out.p = b0;
  out.it = 1;
  out.conv = false;
  out.res = 1.0;
  if (max_it <= 1) return true;
  if (!team_barrier(st, tm, epoch)) return false;
  // sweep 1, reduced
  const float s2 = jac_pass<true, false>(a, n, sy, sz, has_z, b0, b1, r32, sc, t0, gs, nullptr, 0.0);
  if (!team_sum_post<1>(VecF<1>{{s2}}, tm, max_blocks, 0, st, epoch, [&](const double* tot) {
        const double rho = sqrt(tot[0]);
        js.res = rho;
        js.kpred = 1;
        if (rho <= tol) {
          js.state = 1;
        } else if (!isfinite(rho) || rho > kJacobiRate) {
          js.state = 2;
        } else {
          int k = 2;
          const double q = fmin(kJacobiMargin * rho, 0.5);
          double pk = q * q;
          while (pk > tol && k < kJacobiMaxPredicted) {
            pk *= q;
            ++k;
          }
          js.kpred = k < max_it - 1 ? k : max_it - 1;
          js.state = js.kpred >= 2 ? 0 : 1;
        }
      }))
    return false;
  out.res = js.res;
  out.p = b1;
  out.it = 2;
  if (js.state != 0) {
    out.conv = js.state == 1;
    out.half = js.state == 2;
    return true;
  }
  // sweeps 2 .. kpred, separated by barriers; the last one updates x64
  const int kpred = js.kpred;
  for (int k = 2; k <= kpred; ++k) {
    if (k > 2 && !team_barrier(st, tm, epoch)) return false;
    const float* dk = (k & 1) ? b0 : b1;
    float* dn = (k & 1) ? b1 : b0;
    if (k == kpred)
      jac_pass<false, true>(a, n, sy, sz, has_z, dk, dn, r32, sc, t0, gs, x64, rn);
    else
      jac_pass<false, false>(a, n, sy, sz, has_z, dk, dn, r32, sc, t0, gs, nullptr, 0.0);
    out.p = dn;
  }
  out.it = kpred + 1;
  out.x_done = true;
  return true;
}

// FP64 residual r = b - A x and its FP32 copy; returns this thread's |r|^2
// (and |b|^2 in bb when asked).
__device__ __forceinline__ double ir_residual(const BcgArgs& A, int t0, int gs, float* r32, double* bb) {
  const int n = (int)A.sys.d.n;
  const int sy = A.sys.d.mx, sz = A.sys.d.mx * A.sys.d.my;
  const double* b = A.sys.b;
  double s = 0.0, sb = 0.0;
  // two rows per pass (the second a repeat of the first past the end, then
  // dropped): two independent FP64 chains, whose loads overlap
  for (int i = t0; i < n; i += 2 * gs) {
    const bool two = i + gs < n;
    const int i2 = two ? i + gs : i;
    const double b1 = b[i], b2 = b[i2];
    const double r1 = res_row64(b1, A.sys.a, A.sys.x, i, sy, sz, A.has_z);
    const double r2 = res_row64(b2, A.sys.a, A.sys.x, i2, sy, sz, A.has_z);
    A.v64.r[i] = r1;
    r32[i] = to_f32(r1);
    s += r1 * r1;
    if (bb) sb += b1 * b1;
    if (two) {
      A.v64.r[i2] = r2;
      r32[i2] = to_f32(r2);
      s += r2 * r2;
      if (bb) sb += b2 * b2;
    }
  }
  if (bb) *bb = sb;
  return s;
}

__device__ __forceinline__ void ir_solve(const BcgArgs& A, const Team& tm, unsigned int& epoch) {
  const int n = (int)A.sys.d.n;
  const int sy = A.sys.d.mx, sz = A.sys.d.mx * A.sys.d.my;
  const int t0 = tm.rank * blockDim.x + threadIdx.x, gs = tm.size * blockDim.x;
  double* x = A.sys.x;
  double* r64 = A.v64.r;
  float* r32 = A.f32.t;                           // the residual's FP32 copy, read by the inner solve
  if (A.after_presolve && A.st->presolve_done) {  // the pre-solve met tol on the true FP64 residual
    record(A.st, tm.rank == 0, A.stat_index, 0, 0, true, A.st->presolve_rel);
    return;
  }
  Vec<2> acc;
  acc.v[0] = ir_residual(A, t0, gs, r32, &acc.v[1]);
  // scalars formed by thread 0 of each block after each reduction
  __shared__ struct {
    double bnorm, rn, inv, rel, itol;
    float sc;
    int conv, go, restage;
  } is;
  double thr = 0.0;                               // read by thread 0 only
  auto stage_scale = [&]() {
    is.restage = !(is.rn >= kStageLo && is.rn <= kStageHi);
    is.sc = is.restage ? 1.f : (float)is.inv;
  };
  if (!team_sum_post<2>(acc, tm, A.max_blocks, 13, A.st, epoch, [&](const double* tot) {
        is.bnorm = sqrt(tot[1]);
        is.rn = sqrt(tot[0]);
        thr = A.tol * is.bnorm;
        is.inv = 1.0 / is.rn;
        is.conv = is.bnorm == 0.0 || is.rn <= thr;
        is.go = is.bnorm > 0.0 && is.rn > thr && isfinite(is.rn);
        is.rel = is.bnorm > 0.0 ? is.rn / is.bnorm : 0.0;
        is.itol = fmax(A.inner_tol, kSweepMargin * thr / is.rn);
        stage_scale();
      }))
    return;
  int total = 0, jac = 0, ref = 0;
  bool jacobi = A.jacobi != 0;
  const float* dg = A.sys.af.idiag;
  while (is.go && ref < kMaxRefine && total + jac < A.max_it) {
    ++ref;
    const double rn = is.rn;
    if (is.restage) {                             // |r| outside [2^-60, 2^60]: scale in FP64
      const double inv = is.inv;
      for (int i = t0; i < n; i += gs) r32[i] = to_f32(r64[i] * inv);
      if (!team_barrier(A.st, tm, epoch)) return;
    }
    CoreOut o;
    const int left = A.max_it - total - jac;
    const int cap = left < kMaxInner ? left : kMaxInner;
    const float* d = A.d32;
    if (jacobi) {
      if (!jac_fused(A.sys.af, n, sy, sz, A.has_z, A.d32, A.f32, is.sc, is.itol, cap, tm, A.max_blocks, A.st,
                     epoch, x, rn, o))
        return;
      jac += o.it;
      d = o.p;
      if (o.half) jacobi = false;                 // the sweeps stalled: BiCGSTAB from the next sweep on
      // x += rn d (unless the last sweep did)
      if (!o.x_done)
        for (int i = t0; i < n; i += gs) x[i] = fma(rn, (double)d[i], x[i]);
    } else {
      if (!bcg_fused(A.sys.af, n, sy, sz, A.has_z, A.d32, A.f32, is.sc, is.itol, cap, tm, A.max_blocks, A.st,
                     epoch, o))
        return;
      if (o.it == 0) break;                       // the inner solve made no progress
      total += o.it;
      // x += rn d, d completed by the half step's update where it stopped there
      if (!o.half) {
        for (int i = t0; i < n; i += gs) x[i] = fma(rn, (double)d[i], x[i]);
      } else {
        const float al = o.al;
        const float* pp = o.p;
        const bool first = o.it == 1;             // d was not written on the first iteration
        for (int i = t0; i < n; i += gs) {
          const float y = __ldg(dg + i) * pp[i];
          x[i] = fma(rn, (double)(first ? al * y : fmaf(al, y, d[i])), x[i]);
        }
      }
    }
    if (!team_barrier(A.st, tm, epoch)) return;
    Vec<1> s1;
    s1.v[0] = ir_residual(A, t0, gs, r32, nullptr);
    if (!team_sum_post<1>(s1, tm, A.max_blocks, 15, A.st, epoch, [&](const double* tot) {
          is.rn = sqrt(tot[0]);
          is.inv = 1.0 / is.rn;
          is.conv = is.rn <= thr;
          is.go = is.rn > thr && isfinite(is.rn);
          is.rel = is.rn / is.bnorm;
          is.itol = fmax(A.inner_tol, kSweepMargin * thr / is.rn);
          stage_scale();
        }))
      return;
  }
  record(A.st, tm.rank == 0, A.stat_index, total, ref, is.conv != 0, is.rel, jac);
}

// Up to kMaxTeams independent systems in one cooperative launch: team s is
// the blocks [first[s], first[s+1]) and solves sys[s] with its own barrier
// counter and reduction partials (the momentum components u*, v*, w* of
// Eq. 3.3 are independent, so they share one launch instead of three).
struct BcgMulti {
  BcgArgs sys[kMaxTeams];
  int nsys;
  int first[kMaxTeams + 1];
};

// The systems one team of a packed launch solves, one after another.
struct PackedBcgTeam {
  BcgArgs sys[kMaxTeams];
  int nsys;
};

void fill_bcg_args(BcgArgs& A, const Sys& sys, int has_z, const SolverCtl& ctl, const Scratch& c, DevStatus* st);

// The team of this block. Each system's arguments are named with a constant
// index (no runtime indexing of the parameter block, which would copy it to
// local memory).
template <bool MIXED>
__device__ __forceinline__ void solve_team(const BcgMulti& M) {
  const int b = (int)blockIdx.x;
  const int s = (M.nsys > 2 && b >= M.first[2]) ? 2 : (M.nsys > 1 && b >= M.first[1]) ? 1 : 0;
  const int f0 = s == 0 ? 0 : s == 1 ? M.first[1] : M.first[2];
  const int f1 = s == 0 ? M.first[1] : s == 1 ? M.first[2] : M.first[3];
  DevStatus* st = M.sys[0].st;
  unsigned int epoch = 0;
  if (s == 0) {
    const Team tm{b - f0, f1 - f0, &st->team_arrivals[0], M.sys[0].partial};
    if (MIXED) ir_solve(M.sys[0], tm, epoch); else fp64_solve(M.sys[0], tm, epoch);
  } else if (s == 1) {
    const Team tm{b - f0, f1 - f0, &st->team_arrivals[1], M.sys[1].partial};
    if (MIXED) ir_solve(M.sys[1], tm, epoch); else fp64_solve(M.sys[1], tm, epoch);
  } else {
    const Team tm{b - f0, f1 - f0, &st->team_arrivals[2], M.sys[2].partial};
    if (MIXED) ir_solve(M.sys[2], tm, epoch); else fp64_solve(M.sys[2], tm, epoch);
  }
}

__global__ void __launch_bounds__(kBlock, 2) k_bicgstab(BcgMulti M) { solve_team<false>(M); }

__global__ void __launch_bounds__(kBlock, 1) k_bicgstab_ir(BcgMulti M) { solve_team<true>(M); }

// The team of block b in a packed launch: the largest q with first[q] <= b.
__device__ __forceinline__ int packed_team(const int* __restrict__ first, int nteams) {
  __shared__ int s_team;
  if (threadIdx.x == 0) {
    int lo = 0, hi = nteams - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (first[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    s_team = lo;
  }
  __syncthreads();
  return s_team;
}

// A packed launch over the cases of a batch: team q (blocks first[q] ..
// first[q+1]-1) solves the nsys systems of teams[q] one after another (the
// FP32-inner, FP64-refined solve), with the case's own barrier counter and
// reduction partials. Each system's arguments are staged in shared memory.
__global__ void __launch_bounds__(kBlock, 1) k_bicgstab_ir_packed(const PackedBcgTeam* __restrict__ teams,
                                                                 const int* __restrict__ first, int nteams) {
  const int q = packed_team(first, nteams);
  const int f0 = first[q], f1 = first[q + 1];
  __shared__ __align__(16) unsigned long long buf[(sizeof(BcgArgs) + 7) / 8];
  const int nsys = teams[q].nsys;
  unsigned int epoch = 0;
  for (int k = 0; k < nsys; ++k) {
    __syncthreads();
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&teams[q].sys[k]);
    for (int w = threadIdx.x; w < (int)(sizeof(BcgArgs) / 8); w += blockDim.x) buf[w] = src[w];
    __syncthreads();
    const BcgArgs& A = *reinterpret_cast<const BcgArgs*>(buf);
    const Team tm{(int)blockIdx.x - f0, f1 - f0, &A.st->team_arrivals[0], A.partial};
    ir_solve(A, tm, epoch);
  }
}

struct PcgArgs {
  int nx, ny, nz, dim;
  FastDiv fx, fy;
  double cx, cy, cz;      // 1/h^2 per axis
  double* b;
  double* x;
  double *r, *p, *q;
  double tol;
  int max_it;
  int stat_index;
  double* partial;
  int max_blocks;
  DevStatus* st;
};

// A = -L: (A p)_c = sum over existing neighbours of (p_c - p_nb)/h^2
__device__ __forceinline__ double lap_row(const PcgArgs& A, const double* p, int r, int i, int j, int k,
                                          double diag) {
  const int sy = A.nx, sz = A.nx * A.ny;
  double acc = diag * __ldcg(p + r);
  const double sxs = (i > 0 ? __ldcg(p + r - 1) : 0.0) + (i < A.nx - 1 ? __ldcg(p + r + 1) : 0.0);
  acc = fma(-A.cx, sxs, acc);
  const double sys = (j > 0 ? __ldcg(p + r - sy) : 0.0) + (j < A.ny - 1 ? __ldcg(p + r + sy) : 0.0);
  acc = fma(-A.cy, sys, acc);
  if (A.dim == 3) {
    const double szs = (k > 0 ? __ldcg(p + r - sz) : 0.0) + (k < A.nz - 1 ? __ldcg(p + r + sz) : 0.0);
    acc = fma(-A.cz, szs, acc);
  }
  return acc;
}

__device__ __forceinline__ int nb_code(const PcgArgs& A, int i, int j, int k) {
  const int cx = (i > 0) + (i < A.nx - 1);
  const int cy = (j > 0) + (j < A.ny - 1);
  const int cz = (A.dim == 3) ? (k > 0) + (k < A.nz - 1) : 0;
  return cx + 3 * cy + 9 * cz;
}

__global__ void __launch_bounds__(kBlock, 2) k_pcg_poisson(PcgArgs A) {
  __shared__ double s_diag[27], s_minv[27];
  if (threadIdx.x < 27) {
    const int c = threadIdx.x;
    const double d = (c % 3) * A.cx + ((c / 3) % 3) * A.cy + (c / 9) * A.cz;
    s_diag[c] = d;
    s_minv[c] = (d > 0.0) ? 1.0 / d : 0.0;
  }
  __syncthreads();
  unsigned int epoch = 0;
  const int n = A.nx * A.ny * A.nz;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  double *b = A.b, *x = A.x, *r = A.r, *p = A.p, *q = A.q;

  // consistency: remove the mean of the right-hand side (Neumann null space)
  Vec<1> sb = {{0.0}};
  for (int i = t0; i < n; i += gs) sb.v[0] += b[i];
  Vec<1> ob;
  if (!grid_sum<1>(sb, A.partial, A.max_blocks, 8, A.st, epoch, ob)) return;
  const double mean_b = ob.v[0] / (double)n;
  Vec<2> acc = {{0.0, 0.0}};
  for (int i = t0; i < n; i += gs) {
    int ii, jj, kk;
      decompose3(i, A.fx, A.fy, ii, jj, kk);
    const double bi = b[i] - mean_b;
    b[i] = bi;
    x[i] = 0.0;
    r[i] = bi;
    const double zi = s_minv[nb_code(A, ii, jj, kk)] * bi;
    p[i] = zi;
    acc.v[0] += bi * zi;
    acc.v[1] += bi * bi;
  }
  Vec<2> o0;
  if (!grid_sum<2>(acc, A.partial, A.max_blocks, 9, A.st, epoch, o0)) return;
  const double bnorm = sqrt(o0.v[1]);
  double rz = o0.v[0], res = bnorm;
  int it = 0;
  bool conv = (bnorm == 0.0);
  const double thr = A.tol * bnorm;
  while (!conv && it < A.max_it && isfinite(res)) {
    ++it;
    Vec<1> d1 = {{0.0}};
    for (int i = t0; i < n; i += gs) {            // q = A p
      int ii, jj, kk;
      decompose3(i, A.fx, A.fy, ii, jj, kk);
      const double qi = lap_row(A, p, i, ii, jj, kk, s_diag[nb_code(A, ii, jj, kk)]);
      q[i] = qi;
      d1.v[0] += p[i] * qi;
    }
    Vec<1> o1;
    if (!grid_sum<1>(d1, A.partial, A.max_blocks, 10, A.st, epoch, o1)) return;
    const double alpha = rz / o1.v[0];
    Vec<2> d2 = {{0.0, 0.0}};
    for (int i = t0; i < n; i += gs) {            // x += alpha p; r -= alpha q; z = M^-1 r
      int ii, jj, kk;
      decompose3(i, A.fx, A.fy, ii, jj, kk);
      x[i] += alpha * p[i];
      const double ri = r[i] - alpha * q[i];
      r[i] = ri;
      const double zi = s_minv[nb_code(A, ii, jj, kk)] * ri;
      d2.v[0] += ri * zi;
      d2.v[1] += ri * ri;
    }
    Vec<2> o2;
    if (!grid_sum<2>(d2, A.partial, A.max_blocks, 11, A.st, epoch, o2)) return;
    res = sqrt(o2.v[1]);
    conv = res <= thr;
    if (conv) break;
    const double beta = o2.v[0] / rz;
    rz = o2.v[0];
    for (int i = t0; i < n; i += gs) {            // p = z + beta p
      int ii, jj, kk;
      decompose3(i, A.fx, A.fy, ii, jj, kk);
      p[i] = s_minv[nb_code(A, ii, jj, kk)] * r[i] + beta * p[i];
    }
    if (!grid_barrier(A.st, gridDim.x, epoch)) return;
  }
  // gauge: zero-mean correction
  Vec<1> sx = {{0.0}};
  for (int i = t0; i < n; i += gs) sx.v[0] += x[i];
  Vec<1> ox;
  if (!grid_sum<1>(sx, A.partial, A.max_blocks, 12, A.st, epoch, ox)) return;
  const double mean_x = ox.v[0] / (double)n;
  for (int i = t0; i < n; i += gs) x[i] -= mean_x;
  record(A.st, blockIdx.x == 0, A.stat_index, it, 0, conv, bnorm > 0.0 ? res / bnorm : 0.0);
}

void fill_bcg_args(BcgArgs& A, const Sys& sys, int has_z, const SolverCtl& ctl, const Scratch& c, DevStatus* st) {
  A.sys = sys;
  A.has_z = has_z;
  A.tol = ctl.tol;
  A.max_it = ctl.max_it;
  A.stat_index = ctl.stat_index;
  A.inner_tol = ctl.inner_tol;
  A.v64 = {c.v[0], c.v[1], c.v[2], c.v[3], c.v[4], c.v[5], c.v[6]};
  A.f32 = {c.f[0], c.f[1], c.f[2], c.f[3], c.f[4], c.f[5], c.f[6], c.f[8]};
  A.d32 = c.f[7];
  A.partial = c.partial;
  A.max_blocks = c.max_blocks;
  A.st = st;
  A.after_presolve = ctl.after_presolve;
  A.jacobi = ctl.jacobi;
}

int g_num_sms = 0;

int coop_limit(const void* kernel, size_t smem = 0) {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, smem);
  if (per_sm > 4) per_sm = 4;
  return per_sm * g_num_sms;
}

int blocks_for(const void* kernel, long long rows, int max_blocks, size_t smem = 0) {
  long long want = blocks_wanted(rows);
  int lim = coop_limit(kernel, smem);
  if (lim > max_blocks) lim = max_blocks;
  if (want > lim) want = lim;
  if (want < 1) want = 1;
  return (int)want;
}

}  // namespace

int cooperative_blocks(const void* kernel, long long rows) { return blocks_for(kernel, rows, 1 << 30); }

int coop_blocks_for(const void* kernel, long long rows, int max_blocks) { return blocks_for(kernel, rows, max_blocks); }

int coop_blocks_for_smem(const void* kernel, long long rows, int max_blocks, size_t smem) {
  return blocks_for(kernel, rows, max_blocks, smem);
}

// Upper bound on the blocks of any cooperative launch (sizes the reduction partials).
int max_cooperative_blocks() {
  if (g_num_sms == 0) coop_limit((const void*)k_bicgstab);
  return 4 * (g_num_sms > 0 ? g_num_sms : 1);
}

cudaError_t launch_bicgstab_multi(const Sys* const* sys, int nsys, int has_z, const SolverCtl* ctl,
                                  Scratch* const* sc, DevStatus* st, cudaStream_t s) {
  if (nsys < 1 || nsys > kMaxTeams) return cudaErrorInvalidValue;
  BcgMulti M;
  memset(&M, 0, sizeof M);
  M.nsys = nsys;
  bool mixed = true;
  for (int q = 0; q < nsys; ++q) {
    fill_bcg_args(M.sys[q], *sys[q], has_z, ctl[q], *sc[q], st);
    mixed = mixed && ctl[q].mixed && sys[q]->af.P != nullptr && sc[q]->f[0] != nullptr;
  }
  const void* kern = mixed ? (const void*)k_bicgstab_ir : (const void*)k_bicgstab;
  // blocks per team: as many as the system's rows want, scaled down in
  // proportion to the rows when the teams together exceed what one
  // cooperative launch can keep resident
  int lim = coop_limit(kern);
  // a cap below one block per team is raised to that
  if (ctl[0].block_cap > 0 && lim > ctl[0].block_cap) lim = ctl[0].block_cap > nsys ? ctl[0].block_cap : nsys;
  long long want[kMaxTeams], rows = 0, total = 0;
  for (int q = 0; q < nsys; ++q) {
    if (lim > sc[q]->max_blocks) lim = sc[q]->max_blocks;
    want[q] = blocks_wanted(sys[q]->d.n);
    rows += sys[q]->d.n;
    total += want[q];
  }
  if (lim < nsys) return cudaErrorCooperativeLaunchTooLarge;
  if (total > lim) {
    total = 0;
    for (int q = 0; q < nsys; ++q) {
      want[q] = (long long)((double)lim * (double)sys[q]->d.n / (double)(rows > 0 ? rows : 1));
      if (want[q] < 1) want[q] = 1;
      total += want[q];
    }
    while (total > lim) {                      // rounding: take from the largest team
      int big = 0;
      for (int q = 1; q < nsys; ++q) if (want[q] > want[big]) big = q;
      --want[big];
      --total;
    }
    while (total < lim) {                      // and hand what rounding left to the team with most rows per block
      int most = 0;
      for (int q = 1; q < nsys; ++q)
        if ((double)sys[q]->d.n / (double)want[q] > (double)sys[most]->d.n / (double)want[most]) most = q;
      ++want[most];
      ++total;
    }
  }
  M.first[0] = 0;
  for (int q = 0; q < nsys; ++q) M.first[q + 1] = M.first[q] + (int)want[q];
  for (int q = nsys + 1; q <= kMaxTeams; ++q) M.first[q] = M.first[nsys];
  cudaError_t e = cudaMemsetAsync(st->team_arrivals, 0, sizeof(st->team_arrivals), s);
  if (e != cudaSuccess) return e;
  void* args[] = {&M};
  return cudaLaunchCooperativeKernel(kern, dim3(M.first[nsys]), dim3(kBlock), args, 0, s);
}

size_t packed_bcg_team_bytes() { return sizeof(PackedBcgTeam); }

void fill_packed_bcg_team(void* out, const Sys* const* sys, int nsys, int has_z, const SolverCtl* ctl, Scratch& sc,
                          DevStatus* st) {
  PackedBcgTeam& T = *static_cast<PackedBcgTeam*>(out);
  memset(&T, 0, sizeof T);
  T.nsys = nsys;
  for (int q = 0; q < nsys; ++q) fill_bcg_args(T.sys[q], *sys[q], has_z, ctl[q], sc, st);
}

int packed_bcg_max_blocks() { return coop_limit((const void*)k_bicgstab_ir_packed); }

cudaError_t launch_bicgstab_packed(const void* teams, const int* first, int nteams, int nblocks, cudaStream_t s) {
  void* args[] = {(void*)&teams, (void*)&first, (void*)&nteams};
  return cudaLaunchCooperativeKernel((const void*)k_bicgstab_ir_packed, dim3(nblocks), dim3(kBlock), args, 0, s);
}

cudaError_t launch_bicgstab(const Sys& sys, int has_z, const SolverCtl& ctl, Scratch& sc, DevStatus* st,
                            cudaStream_t s) {
  const Sys* sp[1] = {&sys};
  Scratch* cp[1] = {&sc};
  return launch_bicgstab_multi(sp, 1, has_z, &ctl, cp, st, s);
}

cudaError_t launch_pcg_poisson(const Params& pr, double* b, double* x, const SolverCtl& ctl, Scratch& sc,
                               DevStatus* st, cudaStream_t s) {
  PcgArgs A;
  A.nx = pr.nx; A.ny = pr.ny; A.nz = pr.nz; A.dim = pr.dim;
  A.fx = make_fastdiv(pr.nx);
  A.fy = make_fastdiv(pr.ny);
  A.cx = 1.0 / (pr.hx * pr.hx);
  A.cy = 1.0 / (pr.hy * pr.hy);
  A.cz = (pr.dim == 3) ? 1.0 / (pr.hz * pr.hz) : 0.0;
  A.b = b; A.x = x;
  A.r = sc.v[0]; A.p = sc.v[4]; A.q = sc.v[3];
  A.tol = ctl.tol;
  A.max_it = ctl.max_it;
  A.stat_index = ctl.stat_index;
  A.partial = sc.partial;
  A.max_blocks = sc.max_blocks;
  A.st = st;
  const long long n = (long long)pr.nx * pr.ny * pr.nz;
  const int nb = blocks_for((const void*)k_pcg_poisson, n,
                            ctl.block_cap > 0 && ctl.block_cap < sc.max_blocks ? ctl.block_cap : sc.max_blocks);
  cudaError_t e = cudaMemsetAsync(&st->barrier, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  void* args[] = {&A};
  return cudaLaunchCooperativeKernel((const void*)k_pcg_poisson, dim3(nb), dim3(kBlock), args, 0, s);
}

// ---------------------------------------------------------------- pressure solve without allocation
//
// Some callers cannot allocate device memory at all: an application whose
// memory manager owns every byte of the GPU and forbids allocations it did
// not make, a host loop with a hard latency budget in which a cudaMalloc
// (which can synchronise the device) is not acceptable, or a plugin that is
// handed only a stream and device pointers. For them the pressure-correction
// solve is offered with its scratch (solver vectors, reduction partials and
// status block) in a fixed file-scope device array instead of a workspace.
// The array is shared by every call in the process and keeps the last
// call's contents; each call clears the parts that must start at zero.
// Two such calls that overlap on the GPU (on different streams, or from
// different threads) race on the array.

constexpr long long kNoAllocMaxCells = 1LL << 17;     // 131072 cells (e.g. 64 x 64 x 32)
constexpr int kNoAllocMaxBlocks = 1024;
constexpr size_t kNoAllocStatusBytes = (sizeof(DevStatus) + 255) & ~(size_t)255;
constexpr size_t kNoAllocPartialBytes = (size_t)kMaxRedSlots * kNoAllocMaxBlocks * sizeof(double);
constexpr size_t kNoAllocBytes = kNoAllocStatusBytes + kNoAllocPartialBytes + 4 * kNoAllocMaxCells * sizeof(double);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoAllocMaxDevices] = {nullptr};

// Device address of the scratch array on the current device; looked up once
// per device (with that device current) and cached.
cudaError_t noalloc_scratch(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_noalloc_addr[dev]);
  return cudaSuccess;
}
}  // namespace

void set_error_message(const char* fmt, ...);   // capi.cu: the message ss_last_error() returns

}  // namespace solid

extern "C" ss_status ss_poisson_solve_noalloc(int dim, int nx, int ny, int nz, double hx, double hy, double hz,
                                              const double* b, double* x, double tol, int max_it, int* iters,
                                              double* relres, void* stream) {
  using namespace solid;
  if (dim == 2) nz = 1;
  if ((dim != 2 && dim != 3) || nx < 1 || ny < 1 || nz < 1) {
    set_error_message("ss_poisson_solve_noalloc: dim must be 2 or 3 and every cell count >= 1");
    return SS_EINVAL;
  }
  const long long n = (long long)nx * ny * nz;
  if (n > kNoAllocMaxCells) {
    set_error_message("ss_poisson_solve_noalloc: %lld cells exceed its fixed limit of %lld cells", n,
                      kNoAllocMaxCells);
    return SS_EINVAL;
  }
  if (!b || !x || !(hx > 0) || !(hy > 0) || (dim == 3 && !(hz > 0)) || !(tol > 0) || max_it < 1) {
    set_error_message("ss_poisson_solve_noalloc: NULL vector, non-positive spacing or tolerance, or max_it < 1");
    return SS_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* base = nullptr;
  cudaError_t e = noalloc_scratch(&base);
  if (e != cudaSuccess) {
    set_error_message("ss_poisson_solve_noalloc: scratch address lookup failed: %s", cudaGetErrorString(e));
    return SS_ECUDA;
  }
  DevStatus* st = reinterpret_cast<DevStatus*>(base);
  double* partial = reinterpret_cast<double*>(base + kNoAllocStatusBytes);
  double* vec = reinterpret_cast<double*>(base + kNoAllocStatusBytes + kNoAllocPartialBytes);
  PcgArgs A;
  A.nx = nx; A.ny = ny; A.nz = nz; A.dim = dim;
  A.fx = make_fastdiv(nx);
  A.fy = make_fastdiv(ny);
  A.cx = 1.0 / (hx * hx);
  A.cy = 1.0 / (hy * hy);
  A.cz = (dim == 3) ? 1.0 / (hz * hz) : 0.0;
  A.b = vec;                       // the kernel removes the mean in place: work on a copy
  A.r = vec + n;
  A.p = vec + 2 * n;
  A.q = vec + 3 * n;
  A.x = x;
  A.tol = tol;
  A.max_it = max_it;
  A.stat_index = SS_SYS_P;
  A.partial = partial;
  A.max_blocks = kNoAllocMaxBlocks;
  A.st = st;
  const int nb = blocks_for((const void*)k_pcg_poisson, n, kNoAllocMaxBlocks);
  void* args[] = {&A};
  if ((e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(A.b, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s)) != cudaSuccess ||
      (e = cudaLaunchCooperativeKernel((const void*)k_pcg_poisson, dim3(nb), dim3(kBlock), args, 0, s)) !=
          cudaSuccess) {
    set_error_message("ss_poisson_solve_noalloc: %s", cudaGetErrorString(e));
    return SS_ECUDA;
  }
  if (!iters && !relres) return SS_OK;
  DevStatus h;
  if ((e = cudaMemcpyAsync(&h, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    set_error_message("ss_poisson_solve_noalloc: %s", cudaGetErrorString(e));
    return SS_ECUDA;
  }
  if (iters) *iters = h.stat[SS_SYS_P].iters;
  if (relres) *relres = h.stat[SS_SYS_P].relres;
  if (h.err != kErrNone) {
    set_error_message("ss_poisson_solve_noalloc: a grid barrier timed out");
    return SS_ETIMEOUT;
  }
  if (h.stat[SS_SYS_P].nonfinite) {
    set_error_message("ss_poisson_solve_noalloc: non-finite residual");
    return SS_ENAN;
  }
  if (!h.stat[SS_SYS_P].converged) {
    set_error_message("ss_poisson_solve_noalloc: reached max_it before tol");
    return SS_ENOTCONV;
  }
  return SS_OK;
}

