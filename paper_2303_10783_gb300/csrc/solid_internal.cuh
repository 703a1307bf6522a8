// Internal declarations shared by the CUDA translation units of libsolid.
//
// Layout in HBM (all carved from the caller's workspace, 256-byte aligned):
//   * every vector (field, DIA plane, solver vector) is a flat FP64 (or FP32)
//     array on its own row grid, x fastest, with a zero guard band of G
//     entries in front and behind, so that the 7-point stencil of any row
//     (offsets +-1, +-mx, +-mx*my) reads inside the allocation without
//     branches; the coefficient of a neighbour outside the grid is 0.
//   * DIA systems store 7 planes P, W, E, S, N, B, T (Eq. 4.1), the right-hand
//     side b and the inverse diagonal used by the Jacobi preconditioner.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/solid.h"

namespace solid {

constexpr int kBlock = 512;              // threads per block of every kernel
constexpr int kMaxRedSlots = 16;         // reduction slots (one per reduction site)
constexpr long long kSpinLimit = 1LL << 21;  // default barrier polls before giving up (about a second)
constexpr long long kMaxSpinLimit = 1LL << 24;  // largest limit a caller may set (several seconds)

// Systems of at most this many rows are solved by one block: its barriers
// are block barriers, which costs far less than the grid barriers that a few
// blocks would need for a few rows each.
constexpr long long kSingleBlockRows = 4096;
inline long long blocks_wanted(long long rows) {
  return rows <= kSingleBlockRows ? 1 : (rows + kBlock - 1) / kBlock;
}

// device-side error codes (sticky word in DevStatus::err)
enum : int { kErrNone = 0, kErrBarrier = 1 };

// Division by a runtime constant (make_fastdiv / fdiv below).
struct FastDiv {
  unsigned int d, m, s;
};

struct Dims {
  int mx, my, mz;      // row grid of a system / field
  long long n;         // mx * my * mz
  FastDiv fmx, fmy;    // division by mx and my (row -> i, j, k)
};

// Per-solve outcome written by the solver kernels.
struct SolveStat {
  long long iters_total;   // summed over solves since the host last read it
  long long jacobi_total;  // FP64 Jacobi sweeps, summed likewise
  int iters;
  int jacobi;              // FP64 Jacobi sweeps before the Krylov iterations (transport systems)
  int refinements;
  int converged;       // 1 converged, 0 hit the cap
  int nonfinite;       // 1 if a non-finite residual appeared
  double relres;
};

// Device status block (one per case).
// Largest number of independent systems one cooperative solve launch handles
// (the three momentum components), each by its own team of blocks.
constexpr int kMaxTeams = 3;

struct DevStatus {
  unsigned int barrier;          // grid-barrier arrival counter (reset before each cooperative launch)
  unsigned int pad0;
  int err;                       // sticky kErr* code of device-side waits
  int sticky;                    // sticky ss_status of solves since the last read
  SolveStat stat[SS_NSYS];
  double scal[kMaxRedSlots * 4]; // broadcast scalars (unused by the all-blocks reduction)
  double time;                   // simulated time of the fields; k_lever advances it by dt
  unsigned int team_arrivals[kMaxTeams]; // barrier counters of the teams of a multi-system solve
  unsigned int selftest_counter; // counter of the wait self-test (ss_wait_selftest)
  long long presolve_sweeps;     // T* transform pre-solve sweeps since the host last read them
  long long spin_limit;          // polls a barrier waits before giving up (0: kSpinLimit)
  double presolve_rel;           // relative FP64 residual the last T* pre-solve reached
  int presolve_done;             // 1: the last T* pre-solve met the tolerance (its BiCGSTAB has nothing to do)
};

template <typename T>
struct Planes {
  T *P, *W, *E, *S, *N, *B, *T_, *idiag;
};

struct Sys {
  Dims d;
  Planes<double> a;      // FP64 planes
  Planes<float> af;      // FP32 copies for the mixed-precision inner solve (may be null)
  double* b;
  double* x;             // solution (aliases a field or a scratch vector)
};

// A double-float: the value hi + lo held as two FP32s (operations below).
struct dfl {
  float hi, lo;
};

// Physical and numerical parameters passed by value to kernels.
struct Params {
  int dim, nx, ny, nz, vert;
  double hx, hy, hz, dt;
  double Tm, m, kp, C0, rho, k, cp, L, mu, Dl, betaT, betaC, K0, Ce, gravity, eps, Tref;
  int has_eutectic;
  // Thermal walls: flux coef (T_P - T_w(t)) per unit volume and rho c_p, with
  // T_w(t) = wall_T0 + wall_rate t (coef 0: adiabatic). Robin: coef = U/(rho cp h),
  // U = 1/(1/h_c + h/2k), rate 0; Dirichlet: coef = 2k/(rho cp h^2).
  double wall_coef[6], wall_T0[6], wall_rate[6];
  FastDiv fnx, fny;          // division by nx and ny (cell -> i, j, k)
  int slip[6];   // 1: free-slip wall (tangential ghost = interior), 0: no-slip
  int wall_mask; // bit q set when wall q is cooled (wall_coef[q] != 0): an integer test per row
  // Launch constants formed once on the host (IEEE division rounds the same
  // there): the FP64 pipe is the bound of the assembly kernels, so no thread
  // recomputes them.
  double ih[3], ih2[3];      // 1/h and 1/h^2 per axis
  double idt;                // 1/dt
  double nu;                 // mu/rho
  double irho;               // 1/rho
  double alphaT;             // k/(rho cp)
  double rhs_scale;          // -rho/dt (pressure right-hand side)
  double proj_k;             // dt/rho (projection)
  double cpL, Lcp;           // cp/L and L/cp (lever rule)
  double hh[3];              // 0.5/h (face averages of the advecting velocity folded in)
  double nu_ih2[3];          // nu/h^2 (momentum diffusion across one face)
  double two_nu_ih2[3];      // 2 nu/h^2 (no-slip wall face: ghost = -interior)
  double half_nu;            // nu/2 (face mean of the Darcy term)
  double ih_irho[3];         // 1/(h rho) (pressure gradient)
  double alpha_ih2[3];       // k/(rho cp h^2) (energy diffusion across one face)
  double half_Dl_ih2[3];     // D_l/(2 h^2) (solute diffusion: face mean of g_l D_l)
  // lever rule (Eq. 3.16-3.17): a = 1 - kp and products of constants with it
  double lev_a, lev_cpLa, lev_aTm, lev_4a, lev_2a, lev_inv2a;
  double Te;                 // eutectic temperature Tm + m Ce
  // the assembly constants as double-floats (mixed-path assembly)
  dfl df_hh[3], df_ih[3], df_nu_ih2[3], df_two_nu_ih2[3], df_alpha_ih2[3], df_half_Dl_ih2[3];
  dfl df_idt, df_half_nu;
  dfl df_wall_coef[6];
};

// Krylov scratch: 8 FP64 vectors + 9 FP32 vectors, each of `nmax` rows with guards.
struct Scratch {
  double* v[8];
  float* f[9];
  double* partial;       // [kMaxRedSlots][max_blocks]
  int max_blocks;
};

// ---------------------------------------------------------------- device helpers

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned int atom_add_acq_rel_u32(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// A team: the blocks [first, first + size) of a cooperative launch that work
// on one system. It has its own barrier counter and reduction partials, so
// teams of one launch proceed independently. A whole grid is one team.
struct Team {
  int rank;                 // this block's index within the team
  int size;                 // blocks in the team
  unsigned int* counter;    // the team's arrival counter (zeroed by the host before the launch)
  double* partial;          // the team's reduction partials, [kMaxRedSlots][max_blocks]
};

// Barrier over the blocks of a team. `epoch` counts barriers passed by this
// block. Thread 0 arrives with an acq_rel atomic (publishing the block's
// writes) and polls with acquire loads. A poll limit bounds the wait (the
// case's st->spin_limit, read once a block has polled 256 times; 0 means
// kSpinLimit): on expiry the sticky error is set and every block returns
// false from then on, so the kernel unwinds instead of hanging. The error
// flag is shared by all teams, so one team's failure unwinds every team.
__device__ __forceinline__ bool team_barrier(DevStatus* st, const Team& t, unsigned int& epoch) {
  if (t.size == 1) {   // a team of one block: a block barrier orders its own writes
    __threadfence_block();
    __syncthreads();
    return true;
  }
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    epoch += 1u;
    const unsigned int target = epoch * (unsigned int)t.size;
    __threadfence();
    const unsigned int old = atom_add_acq_rel_u32(t.counter, 1u);
    int ok = 1;
    if (old + 1u != target) {
      long long spins = 0, limit = 0;
      while (ld_acquire_u32(t.counter) < target) {
        if ((++spins & 255) == 0) {
          if (*(volatile int*)&st->err != kErrNone) { ok = 0; break; }
          if (limit == 0) {
            const long long l = st->spin_limit;
            limit = (l > 0 && l <= kMaxSpinLimit) ? l : kSpinLimit;
          }
          if (spins >= limit) { atomicExch(&st->err, kErrBarrier); ok = 0; break; }
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Grid-wide barrier for cooperative launches (the whole grid as one team,
// counting on st->barrier).
__device__ __forceinline__ bool grid_barrier(DevStatus* st, unsigned int nblocks, unsigned int& epoch) {
  const Team t{(int)blockIdx.x, (int)nblocks, &st->barrier, nullptr};
  return team_barrier(st, t, epoch);
}

template <int K>
struct Vec { double v[K]; };

// Block-wide sum of K doubles; the result is valid in thread 0 only.
template <int K>
__device__ __forceinline__ Vec<K> block_sum0(Vec<K> x) {
  __shared__ double sh[K][kBlock / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    double s = x.v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) sh[q][wid] = s;
  }
  __syncthreads();
  Vec<K> r;
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      double s = lane < kBlock / 32 ? sh[q][lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      r.v[q] = s;
    }
  }
  return r;
}

template <int K>
struct VecF { float v[K]; };

// Block-wide sum of K floats, returned as doubles in thread 0. The warp sums
// and the sum of the 16 warp sums are formed in FP32: the inputs are FP32
// partial sums of FP32 vectors, and an FP64 shuffle tree would cost each
// warp 16 clocks of the SM's two-lane FP64 pipe per step.
template <int K>
__device__ __forceinline__ Vec<K> block_sum0(VecF<K> x) {
  static_assert(kBlock / 32 <= 32 && (kBlock & (kBlock - 1)) == 0, "one warp holds the warp sums");
  __shared__ float shf[K][kBlock / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    float s = x.v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) shf[q][wid] = s;
  }
  __syncthreads();
  Vec<K> r;
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      float s = lane < kBlock / 32 ? shf[q][lane] : 0.f;
#pragma unroll
      for (int o = kBlock / 64; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      r.v[q] = (double)s;
    }
  }
  return r;
}

// Second half of a team reduction: after the barrier, warp q of every block
// sums slot q's partials in block order (the same order everywhere, so all
// blocks get bit-identical totals) into tot[q]; valid after a __syncthreads.
template <int K>
__device__ __forceinline__ void team_total(const Team& t, int max_blocks, int slot, double* tot) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (wid < K) {
    const double* pp = t.partial + (size_t)(slot + wid) * max_blocks;
    const int nb = t.size;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int i = lane;
    for (; i + 96 < nb; i += 128) {
      s0 += __ldcg(pp + i);
      s1 += __ldcg(pp + i + 32);
      s2 += __ldcg(pp + i + 64);
      s3 += __ldcg(pp + i + 96);
    }
    for (; i < nb; i += 32) s0 += __ldcg(pp + i);
    double s = (s0 + s1) + (s2 + s3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) tot[wid] = s;
  }
}

// Deterministic reduction of K values over a team: every block writes its
// partial sums to slots [slot, slot+K), passes the team barrier, and forms
// the totals with team_total. Returns false if the barrier gave up.
template <int K>
__device__ __forceinline__ bool team_sum(Vec<K> x, const Team& t, int max_blocks, int slot, DevStatus* st,
                                         unsigned int& epoch, Vec<K>& out) {
  static_assert(K <= kBlock / 32, "one warp per reduced value");
  Vec<K> b = block_sum0<K>(x);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) t.partial[(size_t)(slot + q) * max_blocks + t.rank] = b.v[q];
  }
  if (!team_barrier(st, t, epoch)) return false;
  __shared__ double tot[K];
  team_total<K>(t, max_blocks, slot, tot);
  __syncthreads();
#pragma unroll
  for (int q = 0; q < K; ++q) out.v[q] = tot[q];
  __syncthreads();
  return true;
}

// The same reduction (x a Vec<K> of doubles or a VecF<K> of floats), with
// the totals handed to post(const double* tot), run by thread 0 of each
// block: the Krylov scalars (divisions, square roots, stopping tests) are
// formed once per block instead of once per thread, which on GB300's narrow
// FP64 pipe (two lanes per clock per SM) costs microseconds per iteration. What post writes to
// shared memory is visible to every thread of the block on return.
template <int K, class In, class Post>
__device__ __forceinline__ bool team_sum_post(const In& x, const Team& t, int max_blocks, int slot, DevStatus* st,
                                              unsigned int& epoch, Post&& post) {
  static_assert(K <= kBlock / 32, "one warp per reduced value");
  const Vec<K> b = block_sum0(x);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) t.partial[(size_t)(slot + q) * max_blocks + t.rank] = b.v[q];
  }
  if (!team_barrier(st, t, epoch)) return false;
  __shared__ double tot[K];
  team_total<K>(t, max_blocks, slot, tot);
  __syncthreads();
  if (threadIdx.x == 0) post(static_cast<const double*>(tot));
  __syncthreads();
  return true;
}

// The same over the whole grid (counting on st->barrier).
template <int K>
__device__ __forceinline__ bool grid_sum(Vec<K> x, double* partial, int max_blocks, int slot, DevStatus* st,
                                         unsigned int& epoch, Vec<K>& out) {
  const Team t{(int)blockIdx.x, (int)gridDim.x, &st->barrier, partial};
  return team_sum<K>(x, t, max_blocks, slot, st, epoch, out);
}

template <int K, class In, class Post>
__device__ __forceinline__ bool grid_sum_post(const In& x, double* partial, int max_blocks, int slot, DevStatus* st,
                                              unsigned int& epoch, Post&& post) {
  const Team t{(int)blockIdx.x, (int)gridDim.x, &st->barrier, partial};
  return team_sum_post<K>(x, t, max_blocks, slot, st, epoch, post);
}

// IEEE-754 binary64 -> binary32 rounding to nearest, ties to even, on the
// integer pipes for values whose result is a normal float (exponent of d in
// [-126, 127]) and for zeros; other values (subnormal, overflowing, non-finite
// results) take the hardware conversion. The 52-bit fraction keeps its top 23
// bits; the 29 dropped bits decide the rounding; a carry out of the fraction
// correctly increments the exponent (up to infinity). GB300's FP64 pipe is
// narrow, so conversions that need no FP64 arithmetic stay off it.
__device__ __forceinline__ float to_f32(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  const unsigned e = (hi >> 20) & 0x7FFu;
  const unsigned sign = hi & 0x80000000u;
  if (e - 897u <= 253u) {
    const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1FFFFFFFu;
    unsigned bits = sign | ((e - 896u) << 23) | m;
    bits += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
    return __uint_as_float(bits);
  }
  if ((u << 1) == 0ull) return __uint_as_float(sign);
  return __double2float_rn(d);
}

// to_f32(d * p) for p = 2^e: where d is a normal FP64 value and d * 2^e has
// an exponent that FP32 holds as a normal number, the power of two goes into
// the exponent field on the integer pipes (d * 2^e is exact in FP64 there, so
// the result is bit-identical); other values take the FP64 product.
__device__ __forceinline__ float to_f32_scaled(double d, int e, double p) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  const unsigned ed = (hi >> 20) & 0x7FFu;
  const unsigned es = ed + (unsigned)e;   // biased exponent of d * 2^e (wraps when negative)
  if (ed - 1u < 2046u && es - 897u <= 253u) {
    const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1FFFFFFFu;
    unsigned bits = (hi & 0x80000000u) | ((es - 896u) << 23) | m;
    bits += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
    return __uint_as_float(bits);
  }
  return to_f32(d * p);
}

// binary32 -> binary64 (exact) on the integer pipes for normal floats and
// zeros: the exponent is rebiased (127 -> 1023) and the fraction shifted into
// place; subnormal and non-finite values take the hardware conversion.
__device__ __forceinline__ double to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  if (e - 1u < 254u)
    return __longlong_as_double((long long)(sign | ((unsigned long long)(e + 896u) << 52) |
                                            ((unsigned long long)(u & 0x7FFFFFu) << 29)));
  if ((u << 1) == 0u) return __longlong_as_double((long long)sign);
  return (double)f;
}

// ---- double-float: a value hi + lo held as two FP32s (about 48 significant
// bits; Dekker's exact sum and product, with the product's error from an
// FMA). The rounding intrinsics keep the compiler from contracting or
// reordering the error-free steps.
// a + b = s + e exactly (Knuth's two-sum)
__device__ __forceinline__ dfl df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  const dfl s = df_two_sum(a.hi, b.hi);
  return df_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float e = __fmaf_rn(a.hi, b.hi, -p);
  return df_two_sum(p, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e)));
}

// FP64 -> double-float on the integer pipes: hi keeps the top 24 bits of
// the significand (truncated), lo the next 29 rounded to 24, so the pair is
// within 2^-48 of x. Values outside FP32's normal range take to_f32 with
// lo = 0, and lo is 0 where it would fall below FP32's normal range
// (|x| < 2^-74): absolute errors there are below 2^-122.
__device__ __forceinline__ dfl df_from(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned hi32 = (unsigned)(u >> 32), lo32 = (unsigned)u;
  const unsigned e = (hi32 >> 20) & 0x7FFu;
  const unsigned sign = hi32 & 0x80000000u;
  if (e - 897u <= 253u) {
    const unsigned m23 = ((hi32 & 0xFFFFFu) << 3) | (lo32 >> 29);
    const float h = __uint_as_float(sign | ((e - 896u) << 23) | m23);
    const unsigned rest = lo32 & 0x1FFFFFFFu;        // rest * 2^(e - 1023 - 52)
    float l = 0.f;
    if (rest != 0u && e >= 949u)
      l = __uint_as_float(__float_as_uint(__fmul_rn(__uint2float_rn(rest), __uint_as_float((e - 948u) << 23))) | sign);
    return {h, l};
  }
  return {to_f32(x), 0.f};
}

// double-float -> FP64: both halves widened exactly, one FP64 add
__device__ __forceinline__ double df_to_f64(dfl a) { return to_f64(a.hi) + to_f64(a.lo); }

// an FP64 constant as a double-float, on the host
inline dfl df_const(double c) {
  const float hi = (float)c;
  return {hi, (float)(c - (double)hi)};
}

// Division by a runtime constant d >= 1 for 0 <= n < 2^31 with a multiply-high
// and a shift: q = (umulhi(n, m) + n) >> s, s = ceil(log2 d),
// m = floor(2^32 (2^s - d) / d) + 1 (round-up method of Granlund & Montgomery).
inline FastDiv make_fastdiv(unsigned int d) {
  FastDiv f;
  f.d = d;
  if (d <= 1) {
    f.d = 1;
    f.m = 0;
    f.s = 0;
    return f;
  }
  unsigned int s = 0;
  while ((1ull << s) < d) ++s;
  f.s = s;
  f.m = (unsigned int)((((unsigned long long)1 << 32) * (((unsigned long long)1 << s) - d)) / d + 1);
  return f;
}

__device__ __forceinline__ int fdiv(int n, const FastDiv& f) {
  return (int)((__umulhi((unsigned int)n, f.m) + (unsigned int)n) >> f.s);
}

// (i, j, k) of flat index c on an nx * ny * nz grid
__device__ __forceinline__ void decompose3(int c, const FastDiv& fx, const FastDiv& fy, int& i, int& j, int& k) {
  const int t = fdiv(c, fx);
  i = c - t * (int)fx.d;
  k = fdiv(t, fy);
  j = t - k * (int)fy.d;
}

// ---------------------------------------------------------------- host-side launchers

// assemble.cu
cudaError_t launch_assemble_momentum(int comp, const Params& pr, const Sys& sys, const double* const vel[3],
                                     double* ustar, const double* p, const double* T, const double* Cl,
                                     const double* Kinv, cudaStream_t s);
cudaError_t launch_assemble_solute(const Params& pr, const Sys& sys, const double* const vel[3], const double* gl,
                                   const double* C, const double* Ag, cudaStream_t s);
// T is replaced in place by the solve's initial guess (T + Tinc when
// use_guess, else T) and Tinc by -T (see k_assemble_cells).
cudaError_t launch_assemble_temperature(const Params& pr, const Sys& sys, const double* const vel[3],
                                        const double* time, double* T, double* Tinc, int use_guess,
                                        cudaStream_t s);
cudaError_t launch_poisson_rhs(const Params& pr, const double* const ustar[3], double* b, cudaStream_t s);
cudaError_t launch_project(const Params& pr, double* const vel[3], const double* const ustar[3], const double* pc,
                           double* p, cudaStream_t s);
// `time` is advanced by dt (the lever update closes a step); Tinc becomes
// T* - T^n when form_inc, else 0.
cudaError_t launch_lever(const Params& pr, double* time, double* T, double* gl, const double* C, double* Cl,
                         double* Cs, double* Kinv, double* Ag, double* Tinc, int form_inc, cudaStream_t s);
// from_T: recompute g_l from (T, C) in equilibrium; write_cl: recompute C_l, C_s.
// K^{-1} and A_g are always refreshed from g_l.
// Forward (residual-probing) assembly of system sys into its planes (validation mode).
cudaError_t launch_forward_assemble(int sys, const Params& pr, const Sys& sy, const double* const vel[3],
                                    const double* p, const double* T, const double* C, const double* Cl,
                                    const double* gl, const double* Kinv, const double* Ag, const double* time,
                                    cudaStream_t st);
// The FP64 -> FP32 rounding of the FP32 plane copies, on n device values.
cudaError_t launch_to_f32(const double* src, float* dst, long long n, cudaStream_t s);
cudaError_t launch_equilibrate(const Params& pr, const double* T, const double* C, double* gl, double* Cl,
                               double* Cs, double* Kinv, double* Ag, int from_T, int write_cl, cudaStream_t s);

// krylov.cu
struct SolverCtl {
  double tol;
  int max_it;
  int mixed;             // 1: FP32 inner iterations in FP64 iterative refinement
  int stat_index;        // SS_SYS_* slot of DevStatus::stat
  double inner_tol;      // relative tolerance of each FP32 inner solve (mixed path)
  int block_cap;         // > 0: at most this many blocks in the cooperative launch
  int warm_start = 0;    // 1: the solution buffer holds the initial guess (multigrid pressure, mixed path)
  int after_presolve = 0;  // 1: the T* pre-solve ran just before on this stream (mixed path)
  int jacobi = 0;          // 1: FP64 Jacobi sweeps first, while they contract fast (transport systems)
};
cudaError_t launch_bicgstab(const Sys& sys, int has_z, const SolverCtl& ctl, Scratch& sc, DevStatus* st,
                            cudaStream_t s);
// nsys (<= kMaxTeams) independent systems in one cooperative launch, each
// solved by its own team of blocks with its own scratch sc[q].
cudaError_t launch_bicgstab_multi(const Sys* const* sys, int nsys, int has_z, const SolverCtl* ctl,
                                  Scratch* const* sc, DevStatus* st, cudaStream_t s);
cudaError_t launch_pcg_poisson(const Params& pr, double* b, double* x, const SolverCtl& ctl, Scratch& sc,
                               DevStatus* st, cudaStream_t s);
int cooperative_blocks(const void* kernel, long long rows);
int max_cooperative_blocks();
// blocks for a cooperative launch of `kernel` over `rows` rows: at most the
// co-resident limit (capped at 4 per SM) and at most max_blocks
int coop_blocks_for(const void* kernel, long long rows, int max_blocks);
int coop_blocks_for_smem(const void* kernel, long long rows, int max_blocks, size_t smem);

// mg.cu: geometric multigrid hierarchy of the pressure Laplacian
constexpr int kMaxLevels = 12;
struct MGPlan {
  int nl;                      // levels (level 0 = the grid itself)
  int n[kMaxLevels][3];        // cells per axis
  int c[kMaxLevels][3];        // 1: the next level halves this axis
  double h[kMaxLevels][3];     // spacings
  int local[kMaxLevels];       // run by one block
  void* vec[kMaxLevels][4];    // b, x, t, r of the level (float or double)
  int fp32;                    // V-cycle vectors in FP32
  void* cinv;                  // coarsest level of at most kExactCoarse cells: its pseudo-inverse
                               // (row-major, float or double), else nullptr
};
// Coarsest levels up to this many cells are solved exactly (one product with
// the pseudo-inverse of their Neumann operator) instead of by sweeps.
constexpr int kExactCoarse = 64;
void plan_multigrid(const Params& pr, MGPlan& pl, int fp32);
// The pseudo-inverse of the coarsest level's Neumann operator, row-major
// (pinv(A) = (A + J/n)^-1 - J/n, J the all-ones matrix), into out[n*n];
// returns n, or 0 when the coarsest level has more than kExactCoarse cells.
int coarse_pseudo_inverse(const MGPlan& pl, int dim, double* out);
cudaError_t launch_pcg_mg(const MGPlan& pl, const Params& pr, double* b, double* x, const SolverCtl& ctl,
                          Scratch& sc, DevStatus* st, cudaStream_t s);

// ---- packed batches: one launch per stage for many cases
//
// The device-side description of one case of a packed batch: what the
// assembly and pointwise stages of a step read and write.
struct CaseRows {
  Params pr;
  Sys sys[SS_NSYS];
  double *u, *v, *w, *p, *T, *C, *gl, *Cl, *Cs, *Kinv, *Ag, *pc, *pb, *Tinc;
  double* ustar[3];
  DevStatus* st;
};
// A work item of a packed stage: rows [r0, r1) of part `part` (the momentum
// component; 0 otherwise) of case c.
struct PackedTile {
  int c, part, r0, r1;
};
enum { kStageMomentum = 0, kStageRhs = 1, kStageProject = 2, kStageSolute = 3, kStageTemperature = 4,
       kStageLever = 5, kNumPackedStages = 6 };
// Rows of case q that a packed stage covers (part: momentum component).
long long packed_stage_rows(int stage, const Params& pr, int part);
cudaError_t launch_packed_rows(int stage, const CaseRows* cases, const PackedTile* tiles, int ntiles, cudaStream_t s);
// krylov.cu: the transport solves of a packed batch, one team of blocks per case
size_t packed_bcg_team_bytes();
void fill_packed_bcg_team(void* out, const Sys* const* sys, int nsys, int has_z, const SolverCtl* ctl, Scratch& sc,
                          DevStatus* st);
int packed_bcg_max_blocks();
cudaError_t launch_bicgstab_packed(const void* teams, const int* first, int nteams, int nblocks, cudaStream_t s);

// dct.cu: the pressure correction by cosine transforms along x (and y in 3D)
// and tridiagonal solves along the last axis, inside FP64 refinement
struct DctPlan {
  int dim;
  int Mx, My, Mt;        // cells along x, along y (1 in 2D) and along the tridiagonal axis
  int fp32;              // transforms in FP32 (mixed cases) or FP64
  void* T1;              // work arrays of Mx*My*Mt elements (float or double)
  void* T2;
  void* tables;          // cosine matrices Cx [Mx][Mx], Cy [My][My], eigenvalues lx [Mx], ly [My]
  void* img;             // FP32 plans: Cx, Cx^T, Cy, Cy^T in the tensor cores' staged layout
  int tc_mode;           // SS_TC_AUTO, SS_TC_ON or SS_TC_OFF
  // 3D FP32 plans: the tridiagonal factorisations of the slab solves (1/d_t
  // per column), [Mx][Mt][My] for the pressure operator, then the same for
  // the T* operator with the shift thomas_shift
  void* thomas;
  int thomas_p, thomas_h;   // which half is formed
  double thomas_shift;
};
void plan_dct(const Params& pr, DctPlan& pl, int fp32);
size_t dct_table_elems(const DctPlan& pl);
// the tables in FP64, packed as above, into out[dct_table_elems]
void dct_tables(const DctPlan& pl, const Params& pr, double* out);
// bytes of the staged images of an FP32 plan (0 otherwise), and the images
// built from the FP32 tables (Cx [Mx][Mx] and Cy [My][My] as packed above)
size_t dct_image_bytes(const DctPlan& pl);
// bytes of the slab solves' factorisations (0 for 2D and FP64 plans), and
// forming them on stream s for the current parameters where not yet formed
// (after the tables are on the device; stream-ordered)
size_t dct_thomas_bytes(const DctPlan& pl);
cudaError_t dct_thomas_ensure(DctPlan& pl, const Params& pr, cudaStream_t s);
void dct_images(const DctPlan& pl, const float* Cx, const float* Cy, unsigned char* out);
// The fields of the projection (Eq. 3.5) that the transform solve can end with.
struct ProjectPtrs {
  double* vel[3];          // u^{n+1} (written)
  const double* us[3];     // u*
  double* p;               // p (p += p')
};
// proj: when not null, the solve ends with the projection (u^{n+1} from u* and
// the zero-mean p', and p += p'), bit for bit what the projection stage gives.
cudaError_t launch_poisson_dct(const DctPlan& pl, const Params& pr, double* b, double* x, const SolverCtl& ctl,
                               Scratch& sc, DevStatus* st, const ProjectPtrs* proj, cudaStream_t s);
// The T* system (mixed path) by FP64 defect correction around the FP32
// transform inverse of I/dt - alpha L, at most max_sweeps sweeps, starting
// from the x in place; the BiCGSTAB refinement follows it.
// tcgemm.cu: one block forms D (128 x n) = A (128 x k) B (n x k)^T on the tensor cores
// (transposed: A and B stored k x 128 and k x n)
cudaError_t launch_tc_selftest(const float* a, const float* b, float* d, int n, int k, int transposed,
                               DevStatus* st, cudaStream_t s);
cudaError_t launch_helmholtz_dct(const DctPlan& pl, const Params& pr, const Sys& sys, int has_z, int max_sweeps,
                                 const SolverCtl& ctl, Scratch& sc, DevStatus* st, cudaStream_t s);
// the same for a packed batch, one team per case (max_sweeps = 0: none)
size_t packed_helm_args_bytes();
size_t fill_packed_helm_args(void* out, const DctPlan& pl, const Params& pr, const Sys& sys, int has_z,
                             int max_sweeps, const SolverCtl& ctl, Scratch& sc, DevStatus* st);
int packed_helm_max_blocks(size_t smem);
cudaError_t launch_helmholtz_dct_packed(const void* args, const int* first, int nteams, int nblocks, size_t smem,
                                        cudaStream_t s);
// the pressure solves of a packed batch (FP32 transforms), one team per case
size_t packed_dct_args_bytes();
size_t fill_packed_dct_args(void* out, const DctPlan& pl, const Params& pr, double* b, double* x, const SolverCtl& ctl,
                            Scratch& sc, DevStatus* st, const ProjectPtrs* proj);
int packed_dct_max_blocks(size_t smem);
cudaError_t launch_poisson_dct_packed(const void* args, const int* first, int nteams, int nblocks, size_t smem,
                                      cudaStream_t s);

}  // namespace solid
