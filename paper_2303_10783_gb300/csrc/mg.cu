// Geometric-multigrid-preconditioned CG for the pressure correction (Eq. 3.4).
//
// One cooperative launch runs the whole solve.
//   FP64 path   CG in FP64 preconditioned by an FP64 V-cycle.
//   mixed path  FP64 iterative refinement: each sweep forms the FP64 residual
//               r = b - A x, solves A d = r to a relative 1e-5 with CG in FP32
//               preconditioned by an FP32 V-cycle, and adds d to the FP64 x.
//               Every inner iteration is FP32; the FP64 work is one residual
//               per sweep, so the solve leaves GB300's narrow FP64 pipe.
// Both stop on the same test: the FP64 residual below tol * |b|.
//
// Hierarchy: cell-centred, each level halves every axis whose cell count is
// even and >= 4 (semi-coarsening when only some axes qualify). Each level
// rediscretises the Neumann Laplacian A = -L with its own spacings (the
// operator is constant, Sec. 4 term-wise strategy: nothing is assembled).
//   smoother      2 weighted-Jacobi sweeps before and 2 after, weights of a
//                 degree-2 Chebyshev polynomial (see kChebLo)
//   prolongation  trilinear in cell centres (per axis 3/4 parent, 1/4 the
//                 neighbour on the child's side; a wall mirrors the parent)
//   restriction   R = P^T / 2^(coarsened axes) (per axis weights 1/8 3/8 3/8 1/8)
//   coarsest      one product with the pseudo-inverse of its operator when it
//                 has at most kExactCoarse cells, else nu_c weighted-Jacobi
//                 sweeps from zero
// Jacobi smoothing is self-adjoint in the A inner product and R is a scaled
// P^T, so the V-cycle is a fixed symmetric positive-definite operator and
// plain CG applies. The small levels are run by block 0 alone, resident in
// its shared memory; the others grid-wide between grid barriers.
//
// Loads are plain (L1-cached): every phase that reads data another block
// wrote follows a grid barrier whose acquire makes those writes visible.
#include <cmath>
#include <cstring>
#include <utility>
#include <vector>

#include "solid_internal.cuh"

namespace solid {
namespace {

// Smoothing: the two sweeps before and after the coarse correction form a
// degree-2 Chebyshev polynomial in D^-1 A on [kChebLo, kChebHi]: the
// spectrum of the Jacobi-scaled Neumann Laplacian lies in [0, 2]
// (Gershgorin, every row), and the sweeps must damp its upper part, which
// the coarse level cannot represent. Weights are the reciprocals of the
// polynomial's roots, omega_1,2 = 1 / (c -+ d cos(pi/4)), c = (hi+lo)/2,
// d = (hi-lo)/2. Both sweeps are polynomials in D^-1 A, so pre- and
// post-smoothing commute and the V-cycle stays symmetric. The coarsest level
// takes nu_c weighted-Jacobi sweeps with kOmega.
constexpr double kOmega = 0.9;
constexpr double kChebLo = 0.4;
constexpr double kChebHi = 2.0;
constexpr double kOmega1 = 1.0 / (0.5 * (kChebHi + kChebLo) + 0.5 * (kChebHi - kChebLo) * 0.70710678118654752);
constexpr double kOmega2 = 1.0 / (0.5 * (kChebHi + kChebLo) - 0.5 * (kChebHi - kChebLo) * 0.70710678118654752);
constexpr int kMaxRefineP = 12;
// Inner iterations per refinement sweep of the mixed path: the V-cycle-
// preconditioned CG needs 5-8 per sweep; the cap only bounds a sweep whose
// FP32 iteration cannot make progress (the outer FP64 loop continues).
constexpr int kMaxInnerP = 100;
// A sweep's inner solve need not reduce its residual further than the outer
// tolerance still asks: it stops at max(inner_tol, kSweepMargin * thr / rn),
// with thr the outer target and rn the current FP64 residual. The margin
// covers the FP32 operator's rounding, which the FP64 residual sees and the
// inner one does not.
constexpr double kSweepMargin = 0.1;

template <typename TP>
struct Level {
  int nx, ny, nz, n;
  FastDiv fx, fy;          // division by nx and ny
  int cx, cy, cz;          // 1 if the next level halves this axis
  TP ax, ay, az;           // 1/h^2 per axis
  TP *b, *x, *t, *r;       // rhs, iterate, alternate iterate, residual
  int local;               // run by block 0 alone (from shared memory)
  int soff;                // offset (elements) of the level's four arrays in shared memory
  int v4;                  // nx % 4 == 0: FP32 passes take 4 consecutive cells per thread
  FastDiv fx4;             // division by nx / 4
};

template <typename TP>
struct MGArgs {
  int nl;                  // number of levels
  int nu_c;                // sweeps on the coarsest level (even)
  int G;                   // first local level (nl if none)
  int mixed;               // iterative refinement around an inner solve of type TP
  Level<TP> lev[kMaxLevels];
  double cx, cy, cz;       // FP64 1/h^2 of the fine grid
  double* b;               // right-hand side (mean removed in place)
  double *x, *r, *p, *p2, *q;  // FP64 vectors (solution, residual, CG vectors of the FP64 path;
                               // p and p2 alternate as old and new search direction)
  TP *ri, *pi, *pi2, *qi, *di; // inner CG vectors (mixed path)
  double tol;
  double inner_tol;        // relative tolerance of each FP32 inner solve (mixed path)
  int warm;                // mixed path: start from the x in place instead of 0
  int max_it;
  int stat_index;
  double* partial;
  int max_blocks;
  DevStatus* st;
  const TP* cinv;          // pseudo-inverse of the coarsest level, or nullptr (sweeps)
};

struct Range {
  int begin, stride;
};

template <typename TP>
__device__ __forceinline__ int code_of(const Level<TP>& L, int i, int j, int k) {
  return ((i > 0) + (i < L.nx - 1)) + 3 * ((j > 0) + (j < L.ny - 1)) + 9 * ((k > 0) + (k < L.nz - 1));
}

// (A v)_c for a Neumann Laplacian with per-axis coefficients a*
template <typename T>
__device__ __forceinline__ T lap(const T* v, int c, int i, int j, int k, int nx, int ny, int nz, T ax, T ay, T az,
                                 T diag) {
  const int sy = nx, sz = nx * ny;
  T acc = diag * v[c];
  acc = fma(-ax, (i > 0 ? v[c - 1] : T(0)) + (i < nx - 1 ? v[c + 1] : T(0)), acc);
  acc = fma(-ay, (j > 0 ? v[c - sy] : T(0)) + (j < ny - 1 ? v[c + sy] : T(0)), acc);
  if (nz > 1) acc = fma(-az, (k > 0 ? v[c - sz] : T(0)) + (k < nz - 1 ? v[c + sz] : T(0)), acc);
  return acc;
}

template <typename TP>
struct Tables {
  TP diag[kMaxLevels][27];
  TP wid[kMaxLevels][27];   // omega_1 / diag (0 for an isolated cell)
  TP wid2[kMaxLevels][27];  // omega_2 / diag
  TP widc[kMaxLevels][27];  // kOmega / diag (coarsest-level sweeps)
  double diag64[27];        // fine-grid FP64 diagonal
};

// Rows per thread per batch: a phase issues the loads of U rows before any
// dependent arithmetic. U > 1 buys memory-level parallelism with registers;
// in this kernel the extra registers spill, so U = 1.
template <typename T>
struct Batch {
  static constexpr int U = 1;
};

// the 7-point neighbour sums of v at cell c, per axis
template <typename T>
struct Nb {
  T c0, sx, sy, sz;
};

template <typename T>
__device__ __forceinline__ Nb<T> load_nb(const T* v, int c, int i, int j, int k, int nx, int ny, int nz) {
  const int sy = nx, sz = nx * ny;
  Nb<T> o;
  o.c0 = v[c];
  const T w = i > 0 ? v[c - 1] : T(0), e = i < nx - 1 ? v[c + 1] : T(0);
  const T s_ = j > 0 ? v[c - sy] : T(0), n_ = j < ny - 1 ? v[c + sy] : T(0);
  T b_ = T(0), t_ = T(0);
  if (nz > 1) {
    b_ = k > 0 ? v[c - sz] : T(0);
    t_ = k < nz - 1 ? v[c + sz] : T(0);
  }
  o.sx = w + e;
  o.sy = s_ + n_;
  o.sz = b_ + t_;
  return o;
}

template <typename T>
__device__ __forceinline__ T apply_nb(const Nb<T>& q, T ax, T ay, T az, T diag) {
  T acc = diag * q.c0;
  acc = fma(-ax, q.sx, acc);
  acc = fma(-ay, q.sy, acc);
  acc = fma(-az, q.sz, acc);
  return acc;
}

// ---- 4-cells-per-thread FP32 passes (levels with nx % 4 == 0; vectors start
// on 256-byte boundaries, so item m's float4 at 4m is aligned, and so are the
// float4 at 4m +- nx and 4m +- nx*ny)
__device__ __forceinline__ float4 ld4(const float* p, int c) { return *reinterpret_cast<const float4*>(p + c); }
__device__ __forceinline__ void st4(float* p, int c, float4 v) { *reinterpret_cast<float4*>(p + c) = v; }
__device__ __forceinline__ float comp(const float4& v, int l) { return l == 0 ? v.x : l == 1 ? v.y : l == 2 ? v.z : v.w; }

struct Item4 {
  int c, i0, j, k;
};

template <typename TP>
__device__ __forceinline__ Item4 item4(const Level<TP>& L, int m) {
  Item4 it;
  const int t = fdiv(m, L.fx4);
  it.i0 = (m - t * (int)L.fx4.d) * 4;
  it.k = fdiv(t, L.fy);
  it.j = t - it.k * (int)L.fy.d;
  it.c = 4 * m;
  return it;
}

// lane codes of 4 consecutive cells: the y/z part is shared, the x part differs only at the walls
template <typename TP>
__device__ __forceinline__ void codes4(const Level<TP>& L, const Item4& it, int code[4]) {
  const int yz = 3 * ((it.j > 0) + (it.j < L.ny - 1)) + 9 * ((it.k > 0) + (it.k < L.nz - 1));
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    const int i = it.i0 + l;
    code[l] = yz + (i > 0) + (i < L.nx - 1);
  }
}

// A v for 4 consecutive cells (coefficients ax, ay, az; diagonal table dg)
__device__ __forceinline__ void lap4(const float* v, const Item4& it, int nx, int ny, int nz, float ax, float ay,
                                     float az, const float* dg, const int code[4], float in[4], float Av[4]) {
  const int c = it.c, sz = nx * ny;
  const float4 c4 = ld4(v, c);
  const float W = it.i0 > 0 ? v[c - 1] : 0.f, E = it.i0 + 4 < nx ? v[c + 4] : 0.f;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 S = it.j > 0 ? ld4(v, c - nx) : z4, N = it.j < ny - 1 ? ld4(v, c + nx) : z4;
  const float4 B = (nz > 1 && it.k > 0) ? ld4(v, c - sz) : z4, T = (nz > 1 && it.k < nz - 1) ? ld4(v, c + sz) : z4;
  in[0] = c4.x; in[1] = c4.y; in[2] = c4.z; in[3] = c4.w;
  const float sx[4] = {W + c4.y, c4.x + c4.z, c4.y + c4.w, c4.z + E};
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    float acc = dg[code[l]] * in[l];
    acc = fmaf(-ax, sx[l], acc);
    acc = fmaf(-ay, comp(S, l) + comp(N, l), acc);
    acc = fmaf(-az, comp(B, l) + comp(T, l), acc);
    Av[l] = acc;
  }
}

template <typename TP, bool RESIDUAL>
__device__ void sweep4(const Level<TP>& L, const Tables<TP>& tb, int l, const float* in, float* out, Range rg,
                       const TP* wt) {
  const int n4 = L.n >> 2;
  for (int m = rg.begin; m < n4; m += rg.stride) {
    const Item4 it = item4(L, m);
    int code[4];
    codes4(L, it, code);
    float vin[4], Av[4];
    lap4(in, it, L.nx, L.ny, L.nz, (float)L.ax, (float)L.ay, (float)L.az, (const float*)tb.diag[l], code, vin, Av);
    const float4 b4 = ld4((const float*)L.b, it.c);
    const float bb[4] = {b4.x, b4.y, b4.z, b4.w};
    float o[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float res = bb[q] - Av[q];
      o[q] = RESIDUAL ? res : vin[q] + (float)wt[code[q]] * res;
    }
    st4(RESIDUAL ? (float*)L.r : out, it.c, make_float4(o[0], o[1], o[2], o[3]));
  }
}

// out = in + omega D^-1 (b - A in)      (residual_only: L.r = b - A in)
template <typename TP, bool RESIDUAL>
__device__ void sweep(const Level<TP>& L, const Tables<TP>& tb, int l, const TP* in, TP* out, Range rg,
                      const TP* wt) {
  if constexpr (sizeof(TP) == 4) {
    if (L.v4) {
      sweep4<TP, RESIDUAL>(L, tb, l, (const float*)in, (float*)out, rg, wt);
      return;
    }
  }
  constexpr int U = Batch<TP>::U;
  for (int base = rg.begin; base < L.n; base += U * rg.stride) {
    Nb<TP> q[U];
    TP bb[U];
    int code[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int c = base + u * rg.stride;
      if (c < L.n) {
        int i, j, k;
        decompose3(c, L.fx, L.fy, i, j, k);
        code[u] = code_of(L, i, j, k);
        q[u] = load_nb(in, c, i, j, k, L.nx, L.ny, L.nz);
        bb[u] = L.b[c];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int c = base + u * rg.stride;
      if (c < L.n) {
        const TP res = bb[u] - apply_nb(q[u], L.ax, L.ay, L.az, tb.diag[l][code[u]]);
        if (RESIDUAL) L.r[c] = res;
        else out[c] = q[u].c0 + wt[code[u]] * res;
      }
    }
  }
}

// one weighted-Jacobi sweep with the weight table wt (tb.wid, tb.wid2 or tb.widc of level l)
template <typename TP>
__device__ __forceinline__ void smooth(const Level<TP>& L, const Tables<TP>& tb, int l, const TP* in, TP* out,
                                       Range rg, const TP* wt) {
  sweep<TP, false>(L, tb, l, in, out, rg, wt);
}

template <typename TP>
__device__ __forceinline__ void residual(const Level<TP>& L, const Tables<TP>& tb, int l, const TP* in, Range rg) {
  sweep<TP, true>(L, tb, l, in, nullptr, rg, tb.wid[l]);
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// b_{l+1} = R r_l, and the first (pointwise) smoothing sweep of level l+1 from zero.
// Per coarsened axis the fine cells 2I-1 .. 2I+2 carry weights 1/8 3/8 3/8 1/8;
// clamping the out-of-range ones onto the wall cell reproduces R = P^T/2 there
// (1/2 on the wall cell). An axis that is not coarsened reads its one cell four
// times with weight 1/4.
template <typename TP>
__device__ void restrict_to(const Level<TP>& F, const Level<TP>& Cl, const Tables<TP>& tb, int lc, Range rg) {
  const TP wc[4] = {TP(0.125), TP(0.375), TP(0.375), TP(0.125)};
  const TP wn = TP(0.25);
  for (int c = rg.begin; c < Cl.n; c += rg.stride) {
    int I, J, K;
    decompose3(c, Cl.fx, Cl.fy, I, J, K);
    int fi[4], fj[4], fk[4];
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      fi[o] = F.cx ? clampi(2 * I - 1 + o, 0, F.nx - 1) : I;
      fj[o] = F.cy ? clampi(2 * J - 1 + o, 0, F.ny - 1) : J;
      fk[o] = F.cz ? clampi(2 * K - 1 + o, 0, F.nz - 1) : K;
    }
    TP acc = TP(0);
#pragma unroll
    for (int oz = 0; oz < 4; ++oz) {
      const TP wz = F.cz ? wc[oz] : wn;
      TP sy = TP(0);
#pragma unroll
      for (int oy = 0; oy < 4; ++oy) {
        const TP wy = F.cy ? wc[oy] : wn;
        const TP* row = F.r + (size_t)(fj[oy] + F.ny * fk[oz]) * F.nx;
        TP sx = TP(0);
#pragma unroll
        for (int ox = 0; ox < 4; ++ox) sx += (F.cx ? wc[ox] : wn) * row[fi[ox]];
        sy += wy * sx;
      }
      acc += wz * sy;
    }
    Cl.b[c] = acc;
    Cl.x[c] = tb.wid[lc][code_of(Cl, I, J, K)] * acc;
  }
}

// out_l += P e_{l+1}. Per axis the parent carries 3/4 and the coarse
// neighbour on the child's side 1/4; clamping a neighbour beyond the wall
// onto the parent gives the parent weight 1 there. An axis that is not
// coarsened reads its one cell twice (3/4 + 1/4).
//
// On float4 levels (x is then always coarsened) a thread takes 4 consecutive
// fine cells 4m..4m+3 of one x-row: their parents and x-neighbours are the
// coarse cells i0/2 - 1 .. i0/2 + 2, four per coarse row, so 16 coarse loads
// serve 4 cells. The arithmetic per cell is the same as in the scalar loop.
template <typename TP>
__device__ void prolong4(const Level<TP>& F, const Level<TP>& Cl, const float* e, float* out, Range rg) {
  const float w0 = 0.75f, w1 = 0.25f;
  const int n4 = F.n >> 2;
  for (int m = rg.begin; m < n4; m += rg.stride) {
    const Item4 it = item4(F, m);
    const int j = it.j, k = it.k;
    const int J0 = F.cy ? j >> 1 : j, K0 = F.cz ? k >> 1 : k;
    const int J1 = F.cy ? clampi((j & 1) ? J0 + 1 : J0 - 1, 0, Cl.ny - 1) : j;
    const int K1 = F.cz ? clampi((k & 1) ? K0 + 1 : K0 - 1, 0, Cl.nz - 1) : k;
    const int I = it.i0 >> 1;
    const int xa = clampi(I - 1, 0, Cl.nx - 1), xb = I, xc = I + 1, xd = clampi(I + 2, 0, Cl.nx - 1);
    const float* rows[4] = {e + (size_t)(J0 + Cl.ny * K0) * Cl.nx, e + (size_t)(J1 + Cl.ny * K0) * Cl.nx,
                            e + (size_t)(J0 + Cl.ny * K1) * Cl.nx, e + (size_t)(J1 + Cl.ny * K1) * Cl.nx};
    float c[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      c[q][0] = rows[q][xa];
      c[q][1] = rows[q][xb];
      c[q][2] = rows[q][xc];
      c[q][3] = rows[q][xd];
    }
    const float4 cur = ld4(out, it.c);
    // per lane: parent (I0) and x-neighbour (I1) column of the 4 coarse values
    const int par[4] = {1, 1, 2, 2}, nbr[4] = {0, 2, 1, 3};
    float o[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const float y0 = w0 * (w0 * c[0][par[l]] + w1 * c[0][nbr[l]]) + w1 * (w0 * c[1][par[l]] + w1 * c[1][nbr[l]]);
      const float y1 = w0 * (w0 * c[2][par[l]] + w1 * c[2][nbr[l]]) + w1 * (w0 * c[3][par[l]] + w1 * c[3][nbr[l]]);
      o[l] = comp(cur, l) + (w0 * y0 + w1 * y1);
    }
    st4(out, it.c, make_float4(o[0], o[1], o[2], o[3]));
  }
}

template <typename TP>
__device__ void prolong_add(const Level<TP>& F, const Level<TP>& Cl, const TP* e, TP* out, Range rg) {
  if constexpr (sizeof(TP) == 4) {
    if (F.v4 && F.cx) {
      prolong4(F, Cl, (const float*)e, (float*)out, rg);
      return;
    }
  }
  constexpr int U = Batch<TP>::U;
  const TP w0 = TP(0.75), w1 = TP(0.25);
  for (int base = rg.begin; base < F.n; base += U * rg.stride) {
    TP v[U][8], cur[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int c = base + u * rg.stride;
      if (c < F.n) {
        int i, j, k;
        decompose3(c, F.fx, F.fy, i, j, k);
        const int I0 = F.cx ? i >> 1 : i, J0 = F.cy ? j >> 1 : j, K0 = F.cz ? k >> 1 : k;
        const int I1 = F.cx ? clampi((i & 1) ? I0 + 1 : I0 - 1, 0, Cl.nx - 1) : i;
        const int J1 = F.cy ? clampi((j & 1) ? J0 + 1 : J0 - 1, 0, Cl.ny - 1) : j;
        const int K1 = F.cz ? clampi((k & 1) ? K0 + 1 : K0 - 1, 0, Cl.nz - 1) : k;
        const TP* r00 = e + (size_t)(J0 + Cl.ny * K0) * Cl.nx;
        const TP* r01 = e + (size_t)(J1 + Cl.ny * K0) * Cl.nx;
        const TP* r10 = e + (size_t)(J0 + Cl.ny * K1) * Cl.nx;
        const TP* r11 = e + (size_t)(J1 + Cl.ny * K1) * Cl.nx;
        v[u][0] = r00[I0]; v[u][1] = r00[I1];
        v[u][2] = r01[I0]; v[u][3] = r01[I1];
        v[u][4] = r10[I0]; v[u][5] = r10[I1];
        v[u][6] = r11[I0]; v[u][7] = r11[I1];
        cur[u] = out[c];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int c = base + u * rg.stride;
      if (c < F.n) {
        const TP y0 = w0 * (w0 * v[u][0] + w1 * v[u][1]) + w1 * (w0 * v[u][2] + w1 * v[u][3]);
        const TP y1 = w0 * (w0 * v[u][4] + w1 * v[u][5]) + w1 * (w0 * v[u][6] + w1 * v[u][7]);
        out[c] = cur[u] + (w0 * y0 + w1 * y1);
      }
    }
  }
}

struct GridSync {
  DevStatus* st;
  unsigned int* epoch;
  __device__ bool operator()() const { return grid_barrier(st, gridDim.x, *epoch); }
};

struct BlockSync {
  __device__ bool operator()() const {
    __syncthreads();
    return true;
  }
};

// Coarsest level: nu_c weighted-Jacobi sweeps in total, the first already
// done (pointwise) by the restriction into x; nu_c is even, so the result
// ends in t.
template <typename TP, typename SyncF>
__device__ bool coarsest(const Level<TP>* lev, int l, int nu_c, const Tables<TP>& tb, Range rg, SyncF sync,
                         const TP* cinv) {
  const Level<TP>& L = lev[l];
  if (cinv) {   // exact: t = pinv(A) b, one product with the precomputed pseudo-inverse
    if (!sync()) return false;
    for (int c = rg.begin; c < L.n; c += rg.stride) {
      const TP* row = cinv + (size_t)c * L.n;
      TP acc = TP(0);
      for (int q = 0; q < L.n; ++q) acc += row[q] * L.b[q];
      L.t[c] = acc;
    }
    return true;
  }
  TP* a = L.x;
  TP* b = L.t;
  for (int s = 1; s < nu_c; ++s) {
    if (!sync()) return false;
    smooth(L, tb, l, a, b, rg, tb.widc[l]);
    TP* tmp = a;
    a = b;
    b = tmp;
  }
  return true;
}

// Pre-smoothing, residual and restriction on levels [lo, hi): level lo's x
// holds the first sweep on entry.
template <typename TP, typename SyncF>
__device__ bool down(const Level<TP>* lev, const Tables<TP>& tb, int lo, int hi, Range rg, SyncF sync) {
  for (int l = lo; l < hi; ++l) {
    const Level<TP>& L = lev[l];
    if (!sync()) return false;
    smooth(L, tb, l, L.x, L.t, rg, tb.wid2[l]);   // second pre-smoothing sweep -> t
    if (!sync()) return false;
    residual(L, tb, l, L.t, rg);
    if (!sync()) return false;
    restrict_to(L, lev[l + 1], tb, l + 1, rg);
  }
  return true;
}

// Prolongation, correction and post-smoothing on levels hi down to lo. The
// caller guarantees that level hi + 1's result is complete on entry.
template <typename TP, typename SyncF>
__device__ bool up(const Level<TP>* lev, const Tables<TP>& tb, int hi, int lo, Range rg, SyncF sync) {
  for (int l = hi; l >= lo; --l) {
    const Level<TP>& L = lev[l];
    if (l != hi && !sync()) return false;
    prolong_add(L, lev[l + 1], lev[l + 1].t, L.t, rg);
    if (!sync()) return false;
    smooth(L, tb, l, L.t, L.x, rg, tb.wid2[l]);   // post-smoothing sweep 1 -> x
    if (!sync()) return false;
    smooth(L, tb, l, L.x, L.t, rg, tb.wid[l]);    // post-smoothing sweep 2 -> t
  }
  return true;
}

// Scalars the device functions need, passed by value (taking the address of
// the kernel's parameter block would copy all of it to local memory).
struct Ctx {
  int nl, nu_c, G;
  DevStatus* st;
  double* partial;
  int max_blocks;
  const void* cinv;        // pseudo-inverse of the coarsest level (TP), or nullptr
};

// One V-cycle. On entry level 0 holds b and the first sweep x = omega D^-1 b
// (written by the caller on each thread's own rows). On exit the result is in
// lev[0].t; each thread may read its own rows of it (a later reader of other
// rows needs a barrier). Levels from G on are run by block 0 in its shared
// memory (slev) while the other blocks wait at one barrier. glev and slev are
// level tables in shared memory (global and shared-memory arrays).
template <typename TP>
__device__ __noinline__ bool vcycle(const Ctx& X, const Level<TP>* glev, const Level<TP>* slev, const Tables<TP>& tb,
                       unsigned int& epoch) {
  const int nl = X.nl, G = X.G;
  const Range grid_rg{(int)(blockIdx.x * blockDim.x + threadIdx.x), (int)(gridDim.x * blockDim.x)};
  const Range blk_rg{(int)threadIdx.x, (int)blockDim.x};
  const GridSync gs{X.st, &epoch};
  const BlockSync bs;
  const int top = (G < nl - 1) ? G : nl - 1;   // first level not handled grid-wide on the way down
  if (!down(glev, tb, 0, top, grid_rg, gs)) return false;
  if (G < nl) {
    if (!gs()) return false;
    if (blockIdx.x == 0) {
      // level G's b and first sweep x were written grid-wide: stage them in shared memory
      const Level<TP>& Lg = glev[G];
      for (int c = threadIdx.x; c < Lg.n; c += blockDim.x) {
        slev[G].b[c] = Lg.b[c];
        slev[G].x[c] = Lg.x[c];
      }
      down(slev, tb, G, nl - 1, blk_rg, bs);
      __syncthreads();
      coarsest(slev, nl - 1, X.nu_c, tb, blk_rg, bs, (const TP*)X.cinv);
      __syncthreads();
      if (nl - 2 >= G) up(slev, tb, nl - 2, G, blk_rg, bs);
      __syncthreads();
      for (int c = threadIdx.x; c < Lg.n; c += blockDim.x) Lg.t[c] = slev[G].t[c];
    }
    if (!gs()) return false;                  // level G's result is read by every block next
  } else {
    if (!coarsest(glev, nl - 1, X.nu_c, tb, grid_rg, gs, (const TP*)X.cinv)) return false;
    if (top >= 1 && !gs()) return false;
  }
  return up(glev, tb, top - 1, 0, grid_rg, gs);
}

// Sums (r.z, r.r, sum z, sum r) over this thread's rows of z = lev[0].t. The
// rows are taken with the same thread-to-cell mapping as the level-0 sweep
// that wrote z (4 cells per thread on float4 levels), so no barrier is needed
// between that sweep and this pass.
template <typename TV, typename TP>
__device__ __forceinline__ void zr_sums(const Level<TP>& L0, const TV* r, int t0, int gsz, TV& a0, TV& a1, TV& a2,
                                        TV& a3) {
  const int n = L0.n;
  int begin = t0;
  if constexpr (sizeof(TV) == 4 && sizeof(TP) == 4) {
    if (L0.v4) {
      for (int m = t0; m < (n >> 2); m += gsz) {
        const float4 zv = ld4((const float*)L0.t, 4 * m), rv = ld4((const float*)r, 4 * m);
        a0 += (rv.x * zv.x + rv.y * zv.y) + (rv.z * zv.z + rv.w * zv.w);
        a1 += (rv.x * rv.x + rv.y * rv.y) + (rv.z * rv.z + rv.w * rv.w);
        a2 += (zv.x + zv.y) + (zv.z + zv.w);
        a3 += (rv.x + rv.y) + (rv.z + rv.w);
      }
      begin = n;
    }
  }
  for (int c = begin; c < n; c += gsz) {
    const TV zc = (TV)L0.t[c], rc = r[c];
    a0 += rc * zc;
    a1 += rc * rc;
    a2 += zc;
    a3 += rc;
  }
}

// The new search direction p' = (z - mz) + beta p at one point (beta and p
// unused in the first iteration, where p' = z - mz).
template <typename T>
struct Dir {
  const T* z;
  const T* p;
  T mz, beta;
  bool first;
  __device__ __forceinline__ T at(int c) const { return first ? z[c] - mz : (z[c] - mz) + beta * p[c]; }
  __device__ __forceinline__ float4 at4(int c) const {
    const float4 a = ld4((const float*)z, c);
    float4 o = make_float4(a.x - (float)mz, a.y - (float)mz, a.z - (float)mz, a.w - (float)mz);
    if (!first) {
      const float4 b = ld4((const float*)p, c);
      const float bt = (float)beta;
      o.x = o.x + bt * b.x; o.y = o.y + bt * b.y; o.z = o.z + bt * b.z; o.w = o.w + bt * b.w;
    }
    return o;
  }
};

// load_nb of the direction p' (same sums, same order, as load_nb of a stored p')
template <typename T>
__device__ __forceinline__ Nb<T> load_nb_dir(const Dir<T>& d, int c, int i, int j, int k, int nx, int ny, int nz) {
  const int sy = nx, sz = nx * ny;
  Nb<T> o;
  o.c0 = d.at(c);
  const T w = i > 0 ? d.at(c - 1) : T(0), e = i < nx - 1 ? d.at(c + 1) : T(0);
  const T s_ = j > 0 ? d.at(c - sy) : T(0), n_ = j < ny - 1 ? d.at(c + sy) : T(0);
  T b_ = T(0), t_ = T(0);
  if (nz > 1) {
    b_ = k > 0 ? d.at(c - sz) : T(0);
    t_ = k < nz - 1 ? d.at(c + sz) : T(0);
  }
  o.sx = w + e;
  o.sy = s_ + n_;
  o.sz = b_ + t_;
  return o;
}

// lap4 of the direction p' (same arithmetic as lap4 of a stored p')
__device__ __forceinline__ void lap4_dir(const Dir<float>& d, const Item4& it, int nx, int ny, int nz, float ax,
                                         float ay, float az, const float* dg, const int code[4], float in[4],
                                         float Av[4]) {
  const int c = it.c, sz = nx * ny;
  const float4 c4 = d.at4(c);
  const float W = it.i0 > 0 ? d.at(c - 1) : 0.f, E = it.i0 + 4 < nx ? d.at(c + 4) : 0.f;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 S = it.j > 0 ? d.at4(c - nx) : z4, N = it.j < ny - 1 ? d.at4(c + nx) : z4;
  const float4 B = (nz > 1 && it.k > 0) ? d.at4(c - sz) : z4, T = (nz > 1 && it.k < nz - 1) ? d.at4(c + sz) : z4;
  in[0] = c4.x; in[1] = c4.y; in[2] = c4.z; in[3] = c4.w;
  const float sx[4] = {W + c4.y, c4.x + c4.z, c4.y + c4.w, c4.z + E};
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    float acc = dg[code[l]] * in[l];
    acc = fmaf(-ax, sx[l], acc);
    acc = fmaf(-ay, comp(S, l) + comp(N, l), acc);
    acc = fmaf(-az, comp(B, l) + comp(T, l), acc);
    Av[l] = acc;
  }
}

struct PcgOut {
  int it;
  bool conv;
  double res, bnorm;
};

// The CG scalars, formed by thread 0 of each block after each reduction
// (every block forms the same values from the same totals).
template <typename TV>
struct PcgScalars {
  double rz, res, bnorm, inv_n;
  TV alpha, beta, mz;
  int state;   // 0: iterate on; 2: stop
  int conv;
};

// Reduction input: FP32 partial sums reduce in FP32 within a block.
template <typename TV, int K>
struct RedIn { using type = Vec<K>; };
template <int K>
struct RedIn<float, K> { using type = VecF<K>; };

// CG with the V-cycle preconditioner on A x = bscale * (b - bshift) (b is FP64), vectors
// of type TV (double: FP64 path; float: inner solve of the mixed path), x
// from 0. The fine-grid operator uses coefficients (cx, cy, cz) and the
// diagonal table dg of type TV. z is kept orthogonal to the constants (the
// Neumann null space): its mean is removed, so p and x never accumulate a
// constant that would swamp the FP32 arithmetic of the inner solve.
//
// One iteration has two grid-wide reductions and the V-cycle, and no other
// barrier: the new search direction p' = (z - mz) + beta p is formed on the
// fly wherever q = A p' needs it (z is complete after the reduction that
// gave beta), and written to the other of the two p buffers, so no block
// overwrites an old p value that another block still reads. The arithmetic
// is the same, operation for operation, as forming p' in a pass of its own.
// Reduction slots 0..11.
template <typename TV, typename TP>
__device__ __noinline__ bool pcg(const Ctx& X, const Level<TP>* glev, const Level<TP>* slev, const Tables<TP>& tb,
                    const double* b, double bshift, double bscale, TV* x, TV* r, TV* p_a, TV* p_b, TV* q, TV cx,
                    TV cy, TV cz,
                    const TV* dg, double tol, int max_it, unsigned int& epoch, PcgOut& out) {
  constexpr int U = Batch<TV>::U;
  const Level<TP>& L0 = glev[0];
  const int nx = L0.nx, ny = L0.ny, nz = L0.nz, n = L0.n;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x, gsz = gridDim.x * blockDim.x;
  for (int c = t0; c < n; c += gsz) {
    int i, j, k;
    decompose3(c, L0.fx, L0.fy, i, j, k);
    const TV bc = (TV)((b[c] - bshift) * bscale);
    r[c] = bc;
    x[c] = TV(0);
    L0.b[c] = (TP)bc;
    L0.x[c] = tb.wid[0][code_of(L0, i, j, k)] * (TP)bc;
  }
  if (!vcycle(X, glev, slev, tb, epoch)) return false;
  TV a0 = TV(0), a1 = TV(0), a2 = TV(0), a3 = TV(0);
  zr_sums(L0, r, t0, gsz, a0, a1, a2, a3);
  __shared__ PcgScalars<TV> ps;
  double thr = 0.0;                               // read by thread 0 only
  int it = 0;
  if (!grid_sum_post<4>(typename RedIn<TV, 4>::type{{a0, a1, a2, a3}}, X.partial, X.max_blocks, 0, X.st, epoch,
                        [&](const double* tot) {
                          ps.inv_n = 1.0 / (double)n;
                          const double mz = tot[2] * ps.inv_n;
                          ps.bnorm = sqrt(tot[1]);
                          ps.rz = tot[0] - mz * tot[3];
                          ps.res = ps.bnorm;
                          thr = tol * ps.bnorm;
                          ps.mz = (TV)mz;
                          ps.beta = TV(0);
                          ps.conv = ps.bnorm == 0.0;
                          ps.state = (ps.conv || max_it <= 0 || !isfinite(ps.res)) ? 2 : 0;
                        }))
    return false;
  out.bnorm = ps.bnorm;
  TV* p_old = p_a;
  TV* p = p_b;
  const bool v4 = (sizeof(TV) == 4) && L0.v4;
  // FP64 vectors: forming p' at the 7 stencil points would cost ~14 FP64
  // operations per cell on a pipe far slower than the FP32 one, so the FP64
  // path keeps p' in a pass of its own (and one more barrier).
  constexpr bool kFused = sizeof(TV) == 4;
  if constexpr (!kFused) {
    const TV mz = ps.mz;
    for (int c = t0; c < n; c += gsz) p[c] = (TV)L0.t[c] - mz;
    if (!grid_barrier(X.st, gridDim.x, epoch)) return false;
  }
  while (ps.state == 0) {
    const Dir<TV> dir{(const TV*)L0.t, p_old, ps.mz, ps.beta, it == 0};
    ++it;
    TV s1 = TV(0);
    if constexpr (sizeof(TV) == 4) {
      if (v4) {
        for (int m = t0; m < (n >> 2); m += gsz) {    // p' and q = A p', 4 cells per thread
          const Item4 itm = item4(L0, m);
          int code[4];
          codes4(L0, itm, code);
          float pin[4], qv[4];
          lap4_dir(dir, itm, nx, ny, nz, (float)cx, (float)cy, (float)cz, (const float*)dg, code, pin, qv);
          st4((float*)p, itm.c, make_float4(pin[0], pin[1], pin[2], pin[3]));
          st4((float*)q, itm.c, make_float4(qv[0], qv[1], qv[2], qv[3]));
          s1 += (pin[0] * qv[0] + pin[1] * qv[1]) + (pin[2] * qv[2] + pin[3] * qv[3]);
        }
      }
    }
    for (int base = v4 ? n : t0; base < n; base += U * gsz) {   // p' and q = A p'
      Nb<TV> nb[U];
      int code[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int c = base + u * gsz;
        if (c < n) {
          int i, j, k;
          decompose3(c, L0.fx, L0.fy, i, j, k);
          code[u] = code_of(L0, i, j, k);
          nb[u] = kFused ? load_nb_dir(dir, c, i, j, k, nx, ny, nz) : load_nb(p, c, i, j, k, nx, ny, nz);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int c = base + u * gsz;
        if (c < n) {
          const TV qc = apply_nb(nb[u], cx, cy, cz, dg[code[u]]);
          if (kFused) p[c] = nb[u].c0;
          q[c] = qc;
          s1 += nb[u].c0 * qc;
        }
      }
    }
    if (!grid_sum_post<1>(typename RedIn<TV, 1>::type{{s1}}, X.partial, X.max_blocks, 4, X.st, epoch,
                          [&](const double* tot) { ps.alpha = (TV)(ps.rz / tot[0]); }))
      return false;
    const TV alpha = ps.alpha;
    if constexpr (sizeof(TV) == 4) {
      if (v4) {
        for (int m = t0; m < (n >> 2); m += gsz) {    // x += alpha p; r -= alpha q; first V-cycle sweep
          const Item4 itm = item4(L0, m);
          int code[4];
          codes4(L0, itm, code);
          const float4 pv = ld4((const float*)p, itm.c), qv = ld4((const float*)q, itm.c);
          const float4 xv = ld4((const float*)x, itm.c), rv = ld4((const float*)r, itm.c);
          float4 xo, ro, x0;
          xo.x = xv.x + alpha * pv.x; xo.y = xv.y + alpha * pv.y; xo.z = xv.z + alpha * pv.z; xo.w = xv.w + alpha * pv.w;
          ro.x = rv.x - alpha * qv.x; ro.y = rv.y - alpha * qv.y; ro.z = rv.z - alpha * qv.z; ro.w = rv.w - alpha * qv.w;
          x0.x = (float)tb.wid[0][code[0]] * ro.x; x0.y = (float)tb.wid[0][code[1]] * ro.y;
          x0.z = (float)tb.wid[0][code[2]] * ro.z; x0.w = (float)tb.wid[0][code[3]] * ro.w;
          st4((float*)x, itm.c, xo);
          st4((float*)r, itm.c, ro);
          st4((float*)L0.b, itm.c, ro);
          st4((float*)L0.x, itm.c, x0);
        }
      }
    }
    for (int base = v4 ? n : t0; base < n; base += U * gsz) {   // x += alpha p; r -= alpha q; first V-cycle sweep
      TV pv[U], qv[U], xv[U], rv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int c = base + u * gsz;
        if (c < n) {
          pv[u] = p[c];
          qv[u] = q[c];
          xv[u] = x[c];
          rv[u] = r[c];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int c = base + u * gsz;
        if (c < n) {
          int i, j, k;
          decompose3(c, L0.fx, L0.fy, i, j, k);
          x[c] = xv[u] + alpha * pv[u];
          const TV rc = rv[u] - alpha * qv[u];
          r[c] = rc;
          L0.b[c] = (TP)rc;
          L0.x[c] = tb.wid[0][code_of(L0, i, j, k)] * (TP)rc;
        }
      }
    }
    if (!vcycle(X, glev, slev, tb, epoch)) return false;
    TV s2 = TV(0), s3 = TV(0), s4 = TV(0), s5 = TV(0);
    zr_sums(L0, r, t0, gsz, s2, s3, s4, s5);
    if (!grid_sum_post<4>(typename RedIn<TV, 4>::type{{s2, s3, s4, s5}}, X.partial, X.max_blocks, 8, X.st, epoch,
                          [&](const double* tot) {
                            ps.res = sqrt(tot[1]);
                            ps.conv = ps.res <= thr;
                            if (ps.conv) {
                              ps.state = 2;
                              return;
                            }
                            const double mz = tot[2] * ps.inv_n;
                            const double rz_new = tot[0] - mz * tot[3];
                            ps.beta = (TV)(rz_new / ps.rz);
                            ps.rz = rz_new;
                            ps.mz = (TV)mz;
                            ps.state = (it >= max_it || !isfinite(ps.res)) ? 2 : 0;
                          }))
      return false;
    if (ps.state != 0) break;
    if constexpr (kFused) {
      TV* tmp = p_old;  // this iteration's p' is the next iteration's old p
      p_old = p;
      p = tmp;
    } else {
      const TV mzt = ps.mz, beta = ps.beta;
      for (int c = t0; c < n; c += gsz) p[c] = ((TV)L0.t[c] - mzt) + beta * p[c];
      if (!grid_barrier(X.st, gridDim.x, epoch)) return false;
    }
  }
  out.it = it;
  out.conv = ps.conv != 0;
  out.res = ps.res;
  return true;
}

template <typename TP>
__global__ void __launch_bounds__(kBlock, 1) k_pcg_mg(MGArgs<TP> A) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ Tables<TP> tb;
  __shared__ Level<TP> glev[kMaxLevels];
  __shared__ Level<TP> slev[kMaxLevels];
  for (int q = threadIdx.x; q < A.nl * 27; q += blockDim.x) {
    const int l = q / 27, c = q % 27;
    const double ax = (double)A.lev[l].ax, ay = (double)A.lev[l].ay, az = (double)A.lev[l].az;
    const double d = (double)(c % 3) * ax + (double)((c / 3) % 3) * ay + (double)(c / 9) * az;
    tb.diag[l][c] = (TP)d;
    tb.wid[l][c] = d > 0.0 ? (TP)(kOmega1 / d) : TP(0);
    tb.wid2[l][c] = d > 0.0 ? (TP)(kOmega2 / d) : TP(0);
    tb.widc[l][c] = d > 0.0 ? (TP)(kOmega / d) : TP(0);
  }
  if (threadIdx.x < 27) {
    const int c = threadIdx.x;
    tb.diag64[c] = (c % 3) * A.cx + ((c / 3) % 3) * A.cy + (c / 9) * A.cz;
  }
  if (threadIdx.x == 0) {
    for (int l = 0; l < A.nl; ++l) {
      glev[l] = A.lev[l];
      slev[l] = A.lev[l];
      if (l >= A.G) {
        TP* base = reinterpret_cast<TP*>(dsm) + A.lev[l].soff;
        const int nl_ = A.lev[l].n;
        slev[l].b = base;
        slev[l].x = base + nl_;
        slev[l].t = base + 2 * nl_;
        slev[l].r = base + 3 * nl_;
      }
    }
  }
  __syncthreads();
  const Ctx X{A.nl, A.nu_c, A.G, A.st, A.partial, A.max_blocks, A.cinv};
  unsigned int epoch = 0;
  const Level<TP>& L0 = glev[0];
  const int n = L0.n;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x, gsz = gridDim.x * blockDim.x;
  double* b = A.b;
  double* x = A.x;
  double* r = A.r;

  // Scalars of this driver, formed by thread 0 of each block after each
  // reduction (divisions and square roots once per block, not per thread).
  __shared__ struct {
    double mean, bn, rn, rmean, inv, itol;
    int conv;
  } ds;
  // consistency: remove the mean of the right-hand side (Neumann null space)
  Vec<1> sb = {{0.0}};
  for (int c = t0; c < n; c += gsz) sb.v[0] += b[c];
  if (!grid_sum_post<1>(sb, X.partial, X.max_blocks, 12, X.st, epoch,
                        [&](const double* tot) { ds.mean = tot[0] / (double)n; }))
    return;
  const double mean_b = ds.mean;
  for (int c = t0; c < n; c += gsz) b[c] -= mean_b;

  int iters = 0, refs = 0;
  bool conv = false;
  double res = 0.0, bnorm = 0.0;   // relative residual res / bnorm
  // TP = double: the FP64 path; TP = float: the mixed path (refinement)
  if constexpr (sizeof(TP) == 8) {
    PcgOut o;
    if (!pcg<double, TP>(X, glev, slev, tb, b, 0.0, 1.0, x, r, A.p, A.p2, A.q, A.cx, A.cy, A.cz, tb.diag64, A.tol,
                         A.max_it, epoch, o))
      return;
    iters = o.it;
    conv = o.conv;
    res = o.res;
    bnorm = o.bnorm;
  } else {
    // Warm start: the x in place (the previous step's pressure correction,
    // which predicts this step's to a relative residual of ~1e-2 once the
    // flow has developed) is the initial iterate, so the refinement has less
    // to remove. Cold start: x = 0 and r = b.
    const double cx = A.cx, cy = A.cy, cz = A.cz;
    const bool warm = A.warm != 0;
    Vec<3> s = {{0.0, 0.0, 0.0}};
    for (int c = t0; c < n; c += gsz) {
      const double bc = b[c];
      double rc = bc;
      if (warm) {
        int i, j, k;
        decompose3(c, L0.fx, L0.fy, i, j, k);
        rc = bc - lap(x, c, i, j, k, L0.nx, L0.ny, L0.nz, cx, cy, cz, tb.diag64[code_of(L0, i, j, k)]);
      } else {
        x[c] = 0.0;
      }
      r[c] = rc;
      s.v[0] += bc * bc;
      s.v[1] += rc * rc;
      s.v[2] += rc;
    }
    double thr = 0.0;                             // read by thread 0 only
    if (!grid_sum_post<3>(s, X.partial, X.max_blocks, 13, X.st, epoch, [&](const double* tot) {
          ds.bn = sqrt(tot[0]);
          thr = A.tol * ds.bn;
          if (warm) {                             // range part of r, as after each sweep
            ds.rmean = tot[2] / (double)n;
            ds.rn = sqrt(fmax(tot[1] - (double)n * ds.rmean * ds.rmean, 0.0));
          } else {
            ds.rmean = 0.0;                       // b is mean-free
            ds.rn = ds.bn;
          }
          ds.inv = 1.0 / ds.rn;
          ds.conv = ds.bn == 0.0 || ds.rn <= thr;
          ds.itol = fmax(A.inner_tol, kSweepMargin * thr / ds.rn);
        }))
      return;
    conv = ds.conv != 0;
    while (!conv && refs < kMaxRefineP && iters < A.max_it && isfinite(ds.rn)) {
      const double rn = ds.rn;
      ++refs;
      // The inner solve sees the residual without its mean and scaled to unit
      // norm (no FP32 under- or overflow). The mean is the part of the FP64
      // residual in the operator's null space (the constants): it is rounding
      // of A x, no correction can remove it, and left in the inner right-hand
      // side it would stall the inner iteration once the rest falls below it.
      PcgOut io;
      const int cap = (A.max_it - iters < kMaxInnerP) ? A.max_it - iters : kMaxInnerP;
      if (!pcg<TP, TP>(X, glev, slev, tb, r, ds.rmean, ds.inv, A.di, A.ri, A.pi, A.pi2, A.qi, L0.ax, L0.ay, L0.az,
                       tb.diag[0], ds.itol, cap, epoch, io))
        return;
      iters += io.it;
      for (int c = t0; c < n; c += gsz) x[c] += rn * (double)A.di[c];
      if (!grid_barrier(X.st, gridDim.x, epoch)) return;
      Vec<2> s2 = {{0.0, 0.0}};
      for (int c = t0; c < n; c += gsz) {        // FP64 residual of the refined iterate
        int i, j, k;
        decompose3(c, L0.fx, L0.fy, i, j, k);
        const double rc = b[c] - lap(x, c, i, j, k, L0.nx, L0.ny, L0.nz, cx, cy, cz, tb.diag64[code_of(L0, i, j, k)]);
        r[c] = rc;
        s2.v[0] += rc * rc;
        s2.v[1] += rc;
      }
      if (!grid_sum_post<2>(s2, X.partial, X.max_blocks, 14, X.st, epoch, [&](const double* tot) {
            // norm of the residual's range part: sum (r - mean)^2 = sum r^2 - n mean^2
            ds.rmean = tot[1] / (double)n;
            ds.rn = sqrt(fmax(tot[0] - (double)n * ds.rmean * ds.rmean, 0.0));
            ds.inv = 1.0 / ds.rn;
            ds.conv = ds.rn <= thr;
            ds.itol = fmax(A.inner_tol, kSweepMargin * thr / ds.rn);
          }))
        return;
      conv = ds.conv != 0;
      if (io.it == 0) break;                     // the inner solve made no progress
    }
    res = ds.rn;
    bnorm = ds.bn;
  }
  // gauge: zero-mean correction
  Vec<1> sx = {{0.0}};
  for (int c = t0; c < n; c += gsz) sx.v[0] += x[c];
  if (!grid_sum_post<1>(sx, X.partial, X.max_blocks, 15, X.st, epoch,
                        [&](const double* tot) { ds.mean = tot[0] / (double)n; }))
    return;
  const double mean_x = ds.mean;
  for (int c = t0; c < n; c += gsz) x[c] -= mean_x;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const double rel = bnorm > 0.0 ? res / bnorm : 0.0;
    SolveStat& st = A.st->stat[A.stat_index];
    st.iters = iters;
    st.iters_total += iters;
    st.refinements = refs;
    st.converged = conv ? 1 : 0;
    st.nonfinite = isfinite(rel) ? 0 : 1;
    st.relres = rel;
    if (!isfinite(rel)) atomicExch(&A.st->sticky, (int)SS_ENAN);
    else if (!conv) atomicCAS(&A.st->sticky, (int)SS_OK, (int)SS_ENOTCONV);
  }
}

template <typename TP>
MGArgs<TP> make_args(const MGPlan& pl, const Params& pr, double* b, double* x, const SolverCtl& ctl, Scratch& sc,
                     DevStatus* st, size_t& smem) {
  MGArgs<TP> A;
  memset(&A, 0, sizeof A);
  A.nl = pl.nl;
  A.nu_c = 8;
  A.G = pl.nl;
  smem = 0;
  for (int l = 0; l < pl.nl; ++l) {
    Level<TP>& L = A.lev[l];
    L.nx = pl.n[l][0]; L.ny = pl.n[l][1]; L.nz = pl.n[l][2];
    L.n = L.nx * L.ny * L.nz;
    L.fx = make_fastdiv(L.nx);
    L.fy = make_fastdiv(L.ny);
    L.cx = pl.c[l][0]; L.cy = pl.c[l][1]; L.cz = pl.c[l][2];
    L.ax = (TP)(1.0 / (pl.h[l][0] * pl.h[l][0]));
    L.ay = (TP)(1.0 / (pl.h[l][1] * pl.h[l][1]));
    L.az = pr.dim == 3 ? (TP)(1.0 / (pl.h[l][2] * pl.h[l][2])) : TP(0);
    L.b = (TP*)pl.vec[l][0]; L.x = (TP*)pl.vec[l][1]; L.t = (TP*)pl.vec[l][2]; L.r = (TP*)pl.vec[l][3];
    L.local = pl.local[l];
    L.v4 = (sizeof(TP) == 4) && (L.nx % 4 == 0);
    L.fx4 = make_fastdiv(L.nx >= 4 ? L.nx / 4 : 1);
    if (L.local && A.G == pl.nl) A.G = l;
    if (l >= A.G) {
      L.soff = (int)(smem / sizeof(TP));
      smem += 4 * (size_t)L.n * sizeof(TP);
    }
  }
  A.mixed = pl.fp32;
  A.cx = 1.0 / (pr.hx * pr.hx);
  A.cy = 1.0 / (pr.hy * pr.hy);
  A.cz = pr.dim == 3 ? 1.0 / (pr.hz * pr.hz) : 0.0;
  A.b = b; A.x = x;
  A.r = sc.v[0]; A.p = sc.v[4]; A.p2 = sc.v[5]; A.q = sc.v[3];
  if (pl.fp32) {
    A.ri = (TP*)sc.f[1]; A.pi = (TP*)sc.f[2]; A.pi2 = (TP*)sc.f[5]; A.qi = (TP*)sc.f[3]; A.di = (TP*)sc.f[4];
  }
  A.tol = ctl.tol;
  A.inner_tol = ctl.inner_tol;
  A.warm = ctl.warm_start;
  A.max_it = ctl.max_it;
  A.stat_index = ctl.stat_index;
  A.partial = sc.partial;
  A.max_blocks = sc.max_blocks;
  A.st = st;
  A.cinv = (const TP*)pl.cinv;
  return A;
}

template <typename TP>
cudaError_t launch_t(const MGPlan& pl, const Params& pr, double* b, double* x, const SolverCtl& ctl, Scratch& sc,
                     DevStatus* st, cudaStream_t s) {
  size_t smem = 0;
  MGArgs<TP> A = make_args<TP>(pl, pr, b, x, ctl, sc, st, smem);
  const void* kern = (const void*)k_pcg_mg<TP>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long n = (long long)pr.nx * pr.ny * pr.nz;
  const int nb = coop_blocks_for_smem(kern, n, ctl.block_cap > 0 && ctl.block_cap < sc.max_blocks ? ctl.block_cap
                                                                                          : sc.max_blocks, smem);
  if ((e = cudaMemsetAsync(&st->barrier, 0, sizeof(unsigned int), s)) != cudaSuccess) return e;
  void* args[] = {&A};
  return cudaLaunchCooperativeKernel(kern, dim3(nb), dim3(kBlock), args, smem, s);
}

}  // namespace

void plan_multigrid(const Params& pr, MGPlan& pl, int fp32) {
  memset(&pl, 0, sizeof pl);
  int n[3] = {pr.nx, pr.ny, pr.dim == 3 ? pr.nz : 1};
  double h[3] = {pr.hx, pr.hy, pr.dim == 3 ? pr.hz : 1.0};
  const long long local_max = fp32 ? 4096 : 512;
  int l = 0;
  while (true) {
    pl.n[l][0] = n[0]; pl.n[l][1] = n[1]; pl.n[l][2] = n[2];
    pl.h[l][0] = h[0]; pl.h[l][1] = h[1]; pl.h[l][2] = h[2];
    const long long cells = (long long)n[0] * n[1] * n[2];
    pl.local[l] = cells <= local_max;
    int c[3] = {0, 0, 0};
    bool any = false;
    for (int a = 0; a < pr.dim; ++a) {
      if (n[a] % 2 == 0 && n[a] >= 4) { c[a] = 1; any = true; }
    }
    if (!any || cells <= 32 || l == kMaxLevels - 1) break;
    pl.c[l][0] = c[0]; pl.c[l][1] = c[1]; pl.c[l][2] = c[2];
    for (int a = 0; a < 3; ++a)
      if (c[a]) { n[a] /= 2; h[a] *= 2.0; }
    ++l;
  }
  pl.nl = l + 1;
  // once a level is local every coarser level is too
  for (int q = 1; q < pl.nl; ++q) pl.local[q] = pl.local[q] || pl.local[q - 1];
  pl.fp32 = fp32;
}

int coarse_pseudo_inverse(const MGPlan& pl, int dim, double* out) {
  const int L = pl.nl - 1;
  const int nx = pl.n[L][0], ny = pl.n[L][1], nz = pl.n[L][2];
  const int n = nx * ny * nz;
  if (n > kExactCoarse || pl.nl < 2) return 0;
  const double cx = 1.0 / (pl.h[L][0] * pl.h[L][0]), cy = 1.0 / (pl.h[L][1] * pl.h[L][1]);
  const double cz = dim == 3 ? 1.0 / (pl.h[L][2] * pl.h[L][2]) : 0.0;
  // B = A + J/n beside the identity, reduced by Gauss-Jordan with partial pivoting
  std::vector<double> a((size_t)n * 2 * n, 0.0);
  auto B = [&](int r, int q) -> double& { return a[(size_t)r * 2 * n + q]; };
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const int r = i + nx * (j + ny * k);
        const int nbs[6][2] = {{i > 0, r - 1}, {i < nx - 1, r + 1}, {j > 0, r - nx}, {j < ny - 1, r + nx},
                               {k > 0, r - nx * ny}, {k < nz - 1, r + nx * ny}};
        const double coef[6] = {cx, cx, cy, cy, cz, cz};
        for (int q = 0; q < 6; ++q)
          if (nbs[q][0] && coef[q] != 0.0) {
            B(r, r) += coef[q];
            B(r, nbs[q][1]) -= coef[q];
          }
      }
  for (int r = 0; r < n; ++r) {
    for (int q = 0; q < n; ++q) B(r, q) += 1.0 / n;
    B(r, n + r) = 1.0;
  }
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(B(r, col)) > std::fabs(B(piv, col))) piv = r;
    if (piv != col)
      for (int q = 0; q < 2 * n; ++q) std::swap(B(piv, q), B(col, q));
    const double d = B(col, col);
    for (int q = 0; q < 2 * n; ++q) B(col, q) /= d;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const double f = B(r, col);
      if (f != 0.0)
        for (int q = 0; q < 2 * n; ++q) B(r, q) -= f * B(col, q);
    }
  }
  for (int r = 0; r < n; ++r)
    for (int q = 0; q < n; ++q) out[(size_t)r * n + q] = B(r, n + q) - 1.0 / n;
  return n;
}

cudaError_t launch_pcg_mg(const MGPlan& pl, const Params& pr, double* b, double* x, const SolverCtl& ctl, Scratch& sc,
                          DevStatus* st, cudaStream_t s) {
  if (pl.fp32) return launch_t<float>(pl, pr, b, x, ctl, sc, st, s);
  return launch_t<double>(pl, pr, b, x, ctl, sc, st, s);
}

}  // namespace solid
