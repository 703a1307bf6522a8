// Pressure-correction solve (Eq. 3.4) by cosine transforms.
//
// The operator of Eq. 3.4 is the Laplacian with constant coefficients per
// axis and zero-flux walls on a box of cells (the term-wise strategy of
// Sec. 4 keeps it fixed for the whole run). Such an operator is diagonalised
// by the orthonormal DCT-II basis along each axis: along an axis of n cells
// and spacing h, the 1D operator (-p_{i-1} + 2 p_i - p_{i+1})/h^2, with the
// missing neighbour dropped at a wall, has the eigenvectors
// v_k(i) = s_k cos(pi k (i + 1/2) / n) and the eigenvalues
// lambda_k = (4/h^2) sin^2(pi k / (2n)). So A = -L is inverted exactly by
//   transform along x and y (3D) or x (2D),
//   for every transformed column, a tridiagonal solve along the last axis
//     (T_t + (lambda_x + lambda_y) I) p = f  (Thomas algorithm; the one
//     column with lambda_x + lambda_y = 0 is the Neumann null space: its last
//     unknown is pinned to 0, then its mean is removed),
//   transform back.
// The transforms are dense products with the n x n cosine matrices: GEMMs,
// computed by tiles in shared memory. Their cost is arithmetic, not
// synchronisation: one application has three passes and two grid barriers.
//
// The solve is FP64 iterative refinement around that inverse: each sweep
// forms the FP64 residual r = b - A x (and its norm), applies the inverse in
// the precision TP of the transforms, and adds the correction to x. TP =
// float on the mixed path (the inverse is then exact to FP32 rounding, and a
// sweep reduces the residual by 1e-4 to 1e-7), TP = double on the FP64 path.
// The stopping test is the same as the other pressure solvers': the FP64
// residual (its part outside the constants) below tol * |b|.
//
// Data flow of one application (Mx, My, Mt: cells along the transform axes x
// and y and along the tridiagonal axis; My = 1 in 2D; R = My * Mt lines
// along x; a line's index is row = j + My * t):
//   pass A   T1[kx][row] = sum_i Cx[kx][i] r[i + Mx row]          (tiles over kx, row)
//   pass B   per kx: T2[kx][t][ky] = sum_j Cy[ky][j] T1[kx][j + My t];
//            tridiagonal solves along t for every ky (in shared memory);
//            T1[kx][j + My t] = sum_ky Cy[ky][j] T2[kx][t][ky]   (one block per kx)
//            (2D: the tridiagonal solves run on T1 directly)
//   pass C   d[i + Mx row] = sum_kx Cx[kx][i] T1[kx][row]; x += |r| d
#include <cmath>
#include <cstring>
#include <vector>

#include "solid_internal.cuh"
#include "umma.cuh"

namespace solid {
namespace {

// GEMM tile: BM x BN outputs per block, K in chunks of BK; each of the 512
// threads owns 4 x 4 outputs. Shared-memory rows are padded by 4 elements
// (fewer bank conflicts on the transposing stores, 16-byte aligned rows).
constexpr int BM = 64, BN = 128, BK = 16;
constexpr int AS = BM + 4, BS = BN + 4;
constexpr int kGemmSmemElems = 2 * BK * AS + 2 * BK * BS;
static_assert(kBlock == 512, "the GEMM tile assumes 512 threads");
constexpr int kMaxSweeps = 20;
// shared memory for the tridiagonal solves of one chunk of columns
constexpr size_t kThomasSmemBytes = 96 * 1024;

template <typename TP>
struct DctArgs {
  int Mx, My, Mt, R, dim;
  int nx, ny, nz, n;
  FastDiv fx, fy;
  double cx, cy, cz;        // FP64 1/h^2 per axis (the residual's stencil)
  TP at;                    // 1/h^2 along the tridiagonal axis
  const TP* Cx;             // [Mx][Mx] cosine matrix (row k: mode k)
  const TP* Cy;             // [My][My]
  const TP* lx;             // [Mx] eigenvalues along x
  const TP* ly;             // [My] eigenvalues along y
  TP* T1;                   // [Mx][R]
  TP* T2;                   // [Mx][Mt][My]
  double* b;                // right-hand side (mean removed in place)
  double* x;                // solution
  double* r;                // FP64 residual
  double tol;
  int max_sweeps;
  int stat_index;
  int warm;                 // start from the x in place (else from 0)
  int thomas_cols;          // columns per shared-memory chunk of the tridiagonal solves
  int slab_smem;            // 1: pass B keeps each slab in shared memory (FP32 slabs that fit)
  int tc;                   // 1: the kernel opens the tensor cores (some pass below uses them)
  int tc_ac;                // 1: the FP32 transforms of passes A and C run on the tensor cores
  int tc_slab;              // 1: so do pass B's, with the slab's tridiagonal solves in shared memory
  // the constant operands of the tensor-core passes in their staged layout
  const unsigned char *img_cx, *img_cxt, *img_cy, *img_cyt;
  int img_gx, img_gy;       // 8-row groups per half of a chunk of the x and y images
  // Helmholtz mode (the T* pre-solve): the transforms invert s0 I - L instead
  // of -L (no null space), s0 = shift, for the operator I/dt - alpha L
  double shift;
  int helm;
  // 3D FP32 slab solves: 1/d_t of the tridiagonal factorisation of every
  // (kx, ky) column, [Mx][Mt][My], formed once for this operator (or null:
  // formed on the fly)
  const float* tinv;
  double* partial;
  int max_blocks;
  DevStatus* st;
  // projection (Eq. 3.5) after the solve, when p is not null:
  // u^{n+1} = u* - (dt/rho) grad p' on the faces, p += p'
  double* p;
  double* vel[3];
  const double* us[3];
  double proj_k;
  double ih[3];
  FastDiv ffx[3], ffy[3];   // division by the face grid's extents along x and y, per component
};

template <typename T>
__device__ __forceinline__ void lds4(const T* p, T v[4]);
template <>
__device__ __forceinline__ void lds4<float>(const float* p, float v[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
template <>
__device__ __forceinline__ void lds4<double>(const double* p, double v[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// FP64 <-> transform type, the FP32 conversions on the integer pipes
// (v * p for p = 2^e, narrowed)
template <typename TP>
__device__ __forceinline__ TP narrow_scaled(double v, int e, double p);
template <>
__device__ __forceinline__ float narrow_scaled<float>(double v, int e, double p) { return to_f32_scaled(v, e, p); }
template <>
__device__ __forceinline__ double narrow_scaled<double>(double v, int, double p) { return v * p; }
__device__ __forceinline__ double widen(float v) { return to_f64(v); }
__device__ __forceinline__ double widen(double v) { return v; }

// One BM x BN tile of C(m, n) = sum_k A(m, k) B(k, n), m in [m0, m0+BM) and
// n in [n0, n0+BN), entries beyond M, N, K taken as 0. la(m, k) and lb(k, n)
// load one operand element; st(m, n, v) stores one result. *_k_fast say
// whether consecutive k are adjacent in memory (else consecutive m or n),
// and out_m_fast whether consecutive m of the result are: the thread
// mappings of the loads and of the outputs follow, so that neighbouring
// threads touch neighbouring addresses. Chunk k+1 is fetched into registers
// while chunk k is multiplied (two shared-memory buffers).
template <typename TP, class LA, class LB, class ST>
__device__ __forceinline__ void gemm_tile(int M, int N, int K, int m0, int n0, LA la, bool a_k_fast, LB lb,
                                          bool b_k_fast, ST st, bool out_m_fast, TP* sm) {
  TP* As = sm;                   // [2][BK][AS]
  TP* Bs = sm + 2 * BK * AS;     // [2][BK][BS]
  const int tid = threadIdx.x;
  const int tm = out_m_fast ? (tid & 15) : (tid >> 5);
  const int tn = out_m_fast ? (tid >> 4) : (tid & 31);
  TP acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = TP(0);
  TP ra[2], rb[4];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int e = tid + q * kBlock;
      const int m = a_k_fast ? (e >> 4) : (e & (BM - 1));
      const int k = a_k_fast ? (e & (BK - 1)) : (e >> 6);
      const int gm = m0 + m, gk = k0 + k;
      ra[q] = (gm < M && gk < K) ? la(gm, gk) : TP(0);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + q * kBlock;
      const int n = b_k_fast ? (e >> 4) : (e & (BN - 1));
      const int k = b_k_fast ? (e & (BK - 1)) : (e >> 7);
      const int gn = n0 + n, gk = k0 + k;
      rb[q] = (gn < N && gk < K) ? lb(gk, gn) : TP(0);
    }
  };
  auto stash = [&](int buf) {
    TP* as = As + buf * BK * AS;
    TP* bs = Bs + buf * BK * BS;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int e = tid + q * kBlock;
      const int m = a_k_fast ? (e >> 4) : (e & (BM - 1));
      const int k = a_k_fast ? (e & (BK - 1)) : (e >> 6);
      as[k * AS + m] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + q * kBlock;
      const int n = b_k_fast ? (e >> 4) : (e & (BN - 1));
      const int k = b_k_fast ? (e & (BK - 1)) : (e >> 7);
      bs[k * BS + n] = rb[q];
    }
  };
  fetch(0);
  stash(0);
  __syncthreads();
  const int nk = (K + BK - 1) / BK;
  for (int c = 0; c < nk; ++c) {
    const int buf = c & 1;
    if (c + 1 < nk) fetch((c + 1) * BK);
    const TP* as = As + buf * BK * AS + tm * 4;
    const TP* bs = Bs + buf * BK * BS + tn * 4;
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      TP a[4], bv[4];
      lds4(as + k * AS, a);
      lds4(bs + k * BS, bv);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
    }
    if (c + 1 < nk) stash(buf ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + tm * 4 + i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tn * 4 + j;
      if (gm < M && gn < N) st(gm, gn, acc[i][j]);
    }
  }
}

// Tridiagonal solves along t for the columns [c0, c0 + w) of one group:
// column c's entry t is at buf[t * st + c * sc], its shift is sig(c) and it
// is the singular (null-space) column when sing(c). Staged in shared memory:
// values ys[c][t] and the eliminated super-diagonal cs[c][t], rows of odd
// length P (conflict-free column walks).
template <typename TP, class SIG, class SING>
__device__ void thomas_chunk(TP* buf, long long st, long long sc, int Mt, int c0, int w, TP at, SIG sig, SING sing,
                             TP* sm) {
  const int P = (Mt & 1) ? Mt : Mt + 1;
  TP* ys = sm;
  TP* cs = sm + (size_t)w * P;
  const int tot = w * Mt;
  const bool t_fast = (st == 1);
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int t = t_fast ? e % Mt : e / w;
    const int c = t_fast ? e / Mt : e % w;
    ys[c * P + t] = buf[(long long)t * st + (long long)(c0 + c) * sc];
  }
  __syncthreads();
  for (int c = threadIdx.x; c < w; c += blockDim.x) {
    TP* y = ys + c * P;
    TP* cp = cs + c * P;
    const TP s = sig(c0 + c);
    const bool singular = sing(c0 + c);
    // the singular column solves its first Mt - 1 rows with the last unknown
    // pinned to 0 (the system is consistent: its right-hand side sums to 0)
    const int m = singular ? Mt - 1 : Mt;
    if (m <= 0) {
      y[0] = TP(0);
    } else {
      TP prev_c = TP(0), prev_y = TP(0);
      for (int t = 0; t < m; ++t) {
        const TP nb = TP((t > 0) + (t < Mt - 1));
        const TP d = fma(at, prev_c, fma(at, nb, s));   // a nb + s + a c'_{t-1} (c' <= 0)
        const TP inv = TP(1) / d;
        prev_y = fma(at, prev_y, y[t]) * inv;
        prev_c = -at * inv;
        y[t] = prev_y;
        cp[t] = prev_c;
      }
      TP next = TP(0);
      if (singular) y[Mt - 1] = TP(0);
      for (int t = m - 1; t >= 0; --t) {
        next = y[t] - cp[t] * next;
        y[t] = next;
      }
      if (singular) {
        TP sum = TP(0);
        for (int t = 0; t < Mt; ++t) sum += y[t];
        const TP mean = sum / TP(Mt);
        for (int t = 0; t < Mt; ++t) y[t] -= mean;
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int t = t_fast ? e % Mt : e / w;
    const int c = t_fast ? e / Mt : e % w;
    buf[(long long)t * st + (long long)(c0 + c) * sc] = ys[c * P + t];
  }
  __syncthreads();
}

// b_c - (A v)_c, A = -L with zero-flux walls (FP64, the refinement residual):
// each product is fused into the running difference (one FP64 operation per
// neighbour pair and one for the centre; GB300's FP64 pipe bounds this loop)
__device__ __forceinline__ double res_lap64(double bc, const double* v, int c, int i, int j, int k, int nx, int ny,
                                            int nz, double ax, double ay, double az, double diag) {
  const int sy = nx, sz = nx * ny;
  double acc = fma(-diag, v[c], bc);
  acc = fma(ax, (i > 0 ? v[c - 1] : 0.0) + (i < nx - 1 ? v[c + 1] : 0.0), acc);
  acc = fma(ay, (j > 0 ? v[c - sy] : 0.0) + (j < ny - 1 ? v[c + sy] : 0.0), acc);
  if (nz > 1) acc = fma(az, (k > 0 ? v[c - sz] : 0.0) + (k < nz - 1 ? v[c + sz] : 0.0), acc);
  return acc;
}

// The FP32 transform path sums the staged residual r * 2^e (a few units at
// most) in FP32 partial sums of at most kNormChunk terms, each added to an
// FP64 total: a partial is within kNormChunk * 2^-24 of its exact value, so a
// norm is within ~1e-6 of the FP64 one, and convergence is declared only when
// the norm times kNormMargin meets the tolerance. The FP64 path sums in FP64.
constexpr int kNormChunk = 16;
constexpr double kNormMargin = 1.0 + 1.0 / 65536.0;

// Pass A: T1 = (Cx ⊗ I) (rs * sc + off): rs is the residual staged in T2 in
// the transform type, scaled by a power of two (exactly) when it was formed;
// sc and off turn it into (r - mean) / |r| (unit norm, no FP32 under- or
// overflow) in the transform type, once per element and tile.
template <typename TP>
__device__ void pass_a(const DctArgs<TP>& A, const Team& tm, TP sc, TP off, TP* sm) {
  const int Mx = A.Mx, R = A.R;
  const int mt = (Mx + BM - 1) / BM, nt = (R + BN - 1) / BN;
  const TP* Cx = A.Cx;
  const TP* rs = A.T2;
  TP* T1 = A.T1;
  for (int tile = tm.rank; tile < mt * nt; tile += tm.size) {
    const int m0 = (tile % mt) * BM, n0 = (tile / mt) * BN;
    gemm_tile<TP>(
        Mx, R, Mx, m0, n0, [&](int m, int k) { return Cx[(size_t)m * Mx + k]; }, true,
        [&](int k, int n) { return fma(rs[(size_t)n * Mx + k], sc, off); }, true,
        [&](int m, int n, TP v) { T1[(size_t)m * R + n] = v; }, false, sm);
  }
}

// Pass B: per mode kx, the transform along y, the tridiagonal solves along t
// and the inverse transform along y (3D); in 2D only the tridiagonal solves.
// Shared-memory GEMM of a whole slab: out(m, n) = sum_k a[k*lda + m] b[k*ldb + n]
// (both operands k-major), 4 x 4 outputs per thread strided over the output.
template <class ST>
__device__ __forceinline__ void smem_gemm(int M, int N, int K, const float* a, int lda, const float* b, int ldb,
                                          ST st) {
  const int mb = (M + 3) >> 2, nb = (N + 3) >> 2;
  const bool v4 = ((M | N | lda | ldb) & 3) == 0;
  for (int o = threadIdx.x; o < mb * nb; o += blockDim.x) {
    const int m0 = (o % mb) * 4, n0 = (o / mb) * 4;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k = 0; k < K; ++k) {
      float av[4], bv[4];
      if (v4) {
        lds4(a + (size_t)k * lda + m0, av);
        lds4(b + (size_t)k * ldb + n0, bv);
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          av[i] = (m0 + i < M) ? a[(size_t)k * lda + m0 + i] : 0.f;
          bv[i] = (n0 + i < N) ? b[(size_t)k * ldb + n0 + i] : 0.f;
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (m0 + i < M && n0 + j < N) st(m0 + i, n0 + j, acc[i][j]);
  }
}

// Shared memory (floats) of the slab-resident pass B: the slab and the cosine
// matrix (rows padded by 4: 16-byte aligned, fewer bank conflicts in the
// transposing copies), the transformed slab (rows of odd length) and the
// eliminated super-diagonal of the tridiagonal solves.
__host__ __device__ __forceinline__ size_t slab_smem_floats(int My, int Mt) {
  const size_t P = (size_t)(My | 1);
  return (size_t)My * (Mt + 4) + (size_t)My * (My + 4) + 2 * (size_t)Mt * P;
}

// The tridiagonal solves along t of slab kx, one column ky per thread: Ts
// holds the transformed slab [t][ky] (rows of P floats) and receives the
// solution; Ps takes the eliminated super-diagonal.
// inv: where the factorisation is a constant of the operator (A.tinv), the
// slab's 1/d_t, [Mt][My], in shared memory or straight from A.tinv; only the
// substitutions remain then.
__device__ __forceinline__ void slab_thomas(const DctArgs<float>& A, int kx, float* Ts, float* Ps, int P,
                                            const float* inv = nullptr) {
  const int My = A.My, Mt = A.Mt;
  const float at = A.at;
  const float sx = A.lx[kx];
  if (A.tinv) {
    if (!inv) inv = A.tinv + (size_t)kx * Mt * My;
    for (int c = threadIdx.x; c < My; c += blockDim.x) {
      const bool singular = !A.helm && kx == 0 && c == 0;
      const int m = singular ? Mt - 1 : Mt;
      float y = 0.f;
#pragma unroll 8
      for (int t = 0; t < m; ++t) {
        y = fmaf(at, y, Ts[(size_t)t * P + c]) * inv[(size_t)t * My + c];
        Ts[(size_t)t * P + c] = y;
      }
      float next = 0.f;
      if (singular) Ts[(size_t)(Mt - 1) * P + c] = 0.f;
#pragma unroll 8
      for (int t = m - 1; t >= 0; --t) {
        next = fmaf(at * inv[(size_t)t * My + c], next, Ts[(size_t)t * P + c]);
        Ts[(size_t)t * P + c] = next;
      }
      if (singular) {
        float sum = 0.f;
        for (int t = 0; t < Mt; ++t) sum += Ts[(size_t)t * P + c];
        const float mean = sum / (float)Mt;
        for (int t = 0; t < Mt; ++t) Ts[(size_t)t * P + c] -= mean;
      }
    }
    return;
  }
  for (int c = threadIdx.x; c < My; c += blockDim.x) {
    const float s = sx + A.ly[c] + (float)A.shift;
    const bool singular = !A.helm && kx == 0 && c == 0;
    const int m = singular ? Mt - 1 : Mt;
    if (m <= 0) {
      Ts[c] = 0.f;
    } else {
      float prev_c = 0.f, prev_y = 0.f;
      for (int t = 0; t < m; ++t) {
        const float nb = (float)((t > 0) + (t < Mt - 1));
        const float d = fmaf(at, prev_c, fmaf(at, nb, s));
        const float inv = 1.f / d;
        prev_y = fmaf(at, prev_y, Ts[(size_t)t * P + c]) * inv;
        prev_c = -at * inv;
        Ts[(size_t)t * P + c] = prev_y;
        Ps[(size_t)t * P + c] = prev_c;
      }
      float next = 0.f;
      if (singular) Ts[(size_t)(Mt - 1) * P + c] = 0.f;
      for (int t = m - 1; t >= 0; --t) {
        next = Ts[(size_t)t * P + c] - Ps[(size_t)t * P + c] * next;
        Ts[(size_t)t * P + c] = next;
      }
      if (singular) {
        float sum = 0.f;
        for (int t = 0; t < Mt; ++t) sum += Ts[(size_t)t * P + c];
        const float mean = sum / (float)Mt;
        for (int t = 0; t < Mt; ++t) Ts[(size_t)t * P + c] -= mean;
      }
    }
  }
}

// Pass B with the whole slab in shared memory (FP32, 3D): the transform along
// y, the tridiagonal solves along t and the inverse transform never wait on
// global memory between their steps.
__device__ void pass_b_slab(const DctArgs<float>& A, const Team& tm, float* sm) {
  const int Mx = A.Mx, My = A.My, Mt = A.Mt, R = A.R;
  const int P = My | 1;                           // odd row length of the transformed slab
  const int LX = Mt + 4, LC = My + 4;             // padded rows of Xs and Cs
  float* Xs = sm;                                 // [My][LX]: the slab, j-major; later the solution, ky-major
  float* Cs = Xs + (size_t)My * LX;               // [My][LC]: Cy transposed (GEMM 1), then Cy (GEMM 2)
  float* Ts = Cs + (size_t)My * LC;               // [Mt][P]: transformed slab, ky fastest
  float* Ps = Ts + (size_t)Mt * P;                // [Mt][P]: c' of the tridiagonal solves
  for (int kx = tm.rank; kx < Mx; kx += tm.size) {
    float* S1 = A.T1 + (size_t)kx * R;            // [t][j] in global memory
    for (int e = threadIdx.x; e < My * Mt; e += blockDim.x) {
      const int t = e / My, j = e - t * My;       // coalesced over j
      Xs[(size_t)j * LX + t] = S1[e];
    }
    for (int e = threadIdx.x; e < My * My; e += blockDim.x) {
      const int ky = e / My, j = e - ky * My;
      Cs[(size_t)j * LC + ky] = A.Cy[e];          // Cy^T: k-major for GEMM 1
    }
    __syncthreads();
    // GEMM 1: Ts[t][ky] = sum_j Cy[ky][j] S[t][j]
    smem_gemm(My, Mt, My, Cs, LC, Xs, LX, [&](int ky, int t, float v) { Ts[(size_t)t * P + ky] = v; });
    __syncthreads();
    for (int e = threadIdx.x; e < My * My; e += blockDim.x) {
      const int ky = e / My, j = e - ky * My;
      Cs[(size_t)ky * LC + j] = A.Cy[e];          // Cy: k-major for GEMM 2
    }
    slab_thomas(A, kx, Ts, Ps, P);
    __syncthreads();
    for (int e = threadIdx.x; e < My * Mt; e += blockDim.x) {
      const int ky = e / Mt, t = e - ky * Mt;
      Xs[(size_t)ky * LX + t] = Ts[(size_t)t * P + ky];   // the solution, ky-major for GEMM 2
    }
    __syncthreads();
    // GEMM 2: S[t][j] = sum_ky Cy[ky][j] Xs[ky][t]
    smem_gemm(My, Mt, My, Cs, LC, Xs, LX, [&](int j, int t, float v) { S1[(size_t)t * My + j] = v; });
    __syncthreads();
  }
}

// ---- The FP32 transforms on the tensor cores (umma.cuh): the same products
// as gemm_tile and smem_gemm, as 128-row accumulator tiles in TMEM.
constexpr int kTcMaxWidth = 128;   // accumulator width of passes A and C (two staging buffers: 133 KB)
// Passes A and C take the tensor cores from this many multiply-adds per
// transform (Mx * Mx * My * Mt) on: a tile's K chunks are latency-bound
// (~2 us of staging and ~1 us of MMA issue each, measured on GB300), which
// only pays where each block has several tiles. Measured per sweep: 128 x 96
// x 96, pass A 12.3 us (FP32 pipes 12.9), pass C 23.7 (17.3); 384 x 256 x
// 256, pass A 0.51 ms (0.68), pass C 0.83 ms (0.94).
constexpr long long kTcAcMinWork = 1ll << 30;

// Accumulator width (a multiple of 16, at most kTcMaxWidth) for an output of
// `extent` columns by `row_tiles` tiles of 128 rows on a team of `blocks`:
// the fewest rounds of tiles per block, then the least staging per round
// (each tile stages its 128 x K operand and its w x K one).
__device__ __forceinline__ int tc_width(int extent, int row_tiles, int blocks) {
  int best = 16;
  long long best_cost = -1;
  const int top = ((extent + 15) & ~15) < kTcMaxWidth ? ((extent + 15) & ~15) : kTcMaxWidth;
  for (int w = top; w >= 16; w -= 16) {
    const long long tiles = (long long)row_tiles * ((extent + w - 1) / w);
    const long long rounds = (tiles + blocks - 1) / blocks;
    const long long cost = rounds * (kTcM + w);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = w;
    }
  }
  return best;
}

// Pass A: T1[m][n] = sum_k Cx[m][k] (rs[n][k] sc + off), as D[n][m]: rows
// are 128 lines n, columns the modes m of the tile.
__device__ bool pass_a_tc(const DctArgs<float>& A, const Team& tm, float sc, float off, float* sm, TcState& tc) {
  const int Mx = A.Mx, R = A.R;
  const int lt = (R + kTcM - 1) / kTcM;
  const int w = tc_width(Mx, lt, tm.size);
  const int mt = (Mx + w - 1) / w;
  float* T1 = A.T1;
  const TcOperand data{A.T2, Mx, 1, R, Mx, sc, off, 0};     // (line n, k) = rs[n Mx + k] sc + off
  const TcOperand cx{A.Cx, Mx, 1, Mx, Mx, 1.f, 0.f, 0, A.img_cx, A.img_gx};     // (mode m, k) = Cx[m Mx + k]
  for (int tile = tm.rank; tile < lt * mt; tile += tm.size) {
    const int n0 = (tile % lt) * kTcM, m0 = (tile / lt) * w;
    if (!tc_gemm(tc, w, Mx, data, n0, cx, m0, sm, A.st)) return false;
    tc_store(tc, w, [&](int r, int c, float v) {
      const int n = n0 + r, m = m0 + c;
      if (n < R && m < Mx) T1[(size_t)m * R + n] = v;
    });
  }
  return true;
}

// Pass C: x[n][i] += rn sum_m Cx[m][i] T1[m][n], as D[i][n]: rows are 128
// points i along x, columns the lines n of the tile.
__device__ bool pass_c_tc(const DctArgs<float>& A, const Team& tm, double rn, float* sm, TcState& tc) {
  const int Mx = A.Mx, R = A.R;
  const int xt = (Mx + kTcM - 1) / kTcM;
  const int w = tc_width(R, xt, tm.size);
  const int nt = (R + w - 1) / w;
  double* x = A.x;
  const TcOperand cxt{A.Cx, 1, Mx, Mx, Mx, 1.f, 0.f, 1, A.img_cxt, A.img_gx};   // (point i, mode m) = Cx[m Mx + i]
  const TcOperand t1{A.T1, 1, R, R, Mx, 1.f, 0.f, 1};       // (line n, mode m) = T1[m R + n]
  for (int tile = tm.rank; tile < xt * nt; tile += tm.size) {
    const int i0 = (tile % xt) * kTcM, n0 = (tile / xt) * w;
    if (!tc_gemm(tc, w, Mx, cxt, i0, t1, n0, sm, A.st)) return false;
    tc_store(tc, w, [&](int r, int c, float v) {
      const int i = i0 + r, n = n0 + c;
      if (i < Mx && n < R) {
        const size_t q = (size_t)n * Mx + i;
        x[q] = fma(rn, widen(v), x[q]);
      }
    });
  }
  return true;
}

// Rows of the transformed slab of the tensor-core pass B: 16-byte aligned
// (the staging loads read them four at a time).
__host__ __device__ constexpr int tc_slab_row(int My) { return (My + 3) & ~3; }

// Pass B (3D, My <= 128, Mt <= 256) with the transforms along y on the
// tensor cores: per mode kx, Ts[t][ky] = sum_j Cy[ky][j] S[t][j] (rows ky),
// the tridiagonal solves along t in shared memory, then
// S[t][j] = sum_ky Cy[ky][j] Ts[t][ky] (rows j) back into T1.
__device__ bool pass_b_tc(const DctArgs<float>& A, const Team& tm, float* sm, TcState& tc) {
  const int Mx = A.Mx, My = A.My, Mt = A.Mt, R = A.R;
  const int P = tc_slab_row(My);
  const int w = (Mt + 15) & ~15;
  float* Ts = sm + tc_smem_bytes(w) / sizeof(float);   // [Mt][P]
  float* Ps = Ts + (size_t)Mt * P;                       // [Mt][P]
  const TcOperand cy{A.Cy, My, 1, My, My, 1.f, 0.f, 0, A.img_cy, A.img_gy};    // (ky, j) = Cy[ky My + j]
  const TcOperand cyt{A.Cy, 1, My, My, My, 1.f, 0.f, 1, A.img_cyt, A.img_gy};  // (j, ky) = Cy[ky My + j]
  const TcOperand ts{Ts, P, 1, Mt, My, 1.f, 0.f, 0};       // (t, ky) = Ts[t P + ky]
  // the slab's factorisation (when formed) comes into Ps by the copy engine
  // during the first product, where its offsets keep 16-byte alignment
  const uint32_t inv_bytes = (uint32_t)Mt * My * sizeof(float);
  const bool inv_async = A.tinv && (inv_bytes & 15u) == 0 && (reinterpret_cast<uintptr_t>(A.tinv) & 15u) == 0;
  for (int kx = tm.rank; kx < Mx; kx += tm.size) {
    float* S1 = A.T1 + (size_t)kx * R;   // [t][j]
    const TcOperand slab{S1, My, 1, Mt, My, 1.f, 0.f, 0};  // (t, j) = S1[t My + j]
    if (inv_async && threadIdx.x == 0) {
      fence_async_smem();   // Ps was last written by the threads
      mbar_expect_tx(tc.xbar, inv_bytes);
      bulk_g2s(smem_u32(Ps), A.tinv + (size_t)kx * Mt * My, inv_bytes, tc.xbar);
    }
    const bool ok = tc_gemm(tc, w, My, cy, 0, slab, 0, sm, A.st);
    if (inv_async) {   // the copy has been issued: wait for it (bounded) on every way on
      const bool got = mbar_wait(tc.xbar, tc.xphase);
      if (!got) mbar_wait(tc.xbar, tc.xphase);
      tc.xphase ^= 1u;
      if (__syncthreads_or(!got)) {
        if (threadIdx.x == 0) atomicExch(&A.st->err, kErrBarrier);
        return false;
      }
    }
    if (!ok) return false;
    tc_store(tc, w, [&](int ky, int t, float v) {
      if (ky < My && t < Mt) Ts[(size_t)t * P + ky] = v;
    });
    slab_thomas(A, kx, Ts, Ps, P, inv_async ? Ps : nullptr);
    __syncthreads();
    if (!tc_gemm(tc, w, My, cyt, 0, ts, 0, sm, A.st)) return false;
    tc_store(tc, w, [&](int j, int t, float v) {
      if (j < My && t < Mt) S1[(size_t)t * My + j] = v;
    });
  }
  return true;
}

template <typename TP>
__device__ void pass_b(const DctArgs<TP>& A, const Team& tm, TP* sm) {
  if constexpr (sizeof(TP) == 4) {
    if (A.slab_smem) {
      pass_b_slab(A, tm, sm);
      return;
    }
  }
  const int Mx = A.Mx, My = A.My, Mt = A.Mt, R = A.R;
  const TP* lx = A.lx;
  const TP* ly = A.ly;
  const TP* Cy = A.Cy;
  const TP at = A.at;
  const int w = A.thomas_cols;
  if (A.dim == 2) {
    // columns are the modes kx, each a contiguous line of Mt values in T1
    for (int c0 = tm.rank * w; c0 < Mx; c0 += tm.size * w) {
      const int cw = (Mx - c0 < w) ? Mx - c0 : w;
      thomas_chunk<TP>(
          A.T1, 1, R, Mt, c0, cw, at, [&](int c) { return lx[c] + (TP)A.shift; },
          [&](int c) { return !A.helm && c == 0; }, sm);
    }
    return;
  }
  const int mt = (My + BM - 1) / BM, nt = (Mt + BN - 1) / BN;
  for (int kx = tm.rank; kx < Mx; kx += tm.size) {
    TP* S1 = A.T1 + (size_t)kx * R;   // [t][j]
    TP* S2 = A.T2 + (size_t)kx * R;   // [t][ky]
    for (int tile = 0; tile < mt * nt; ++tile) {
      const int m0 = (tile % mt) * BM, n0 = (tile / mt) * BN;
      gemm_tile<TP>(
          My, Mt, My, m0, n0, [&](int m, int k) { return Cy[(size_t)m * My + k]; }, true,
          [&](int k, int n) { return S1[(size_t)n * My + k]; }, true,
          [&](int m, int n, TP v) { S2[(size_t)n * My + m] = v; }, true, sm);
    }
    __syncthreads();
    const TP sx = lx[kx];
    for (int c0 = 0; c0 < My; c0 += w) {
      const int cw = (My - c0 < w) ? My - c0 : w;
      thomas_chunk<TP>(
          S2, My, 1, Mt, c0, cw, at, [&](int c) { return sx + ly[c] + (TP)A.shift; },
          [&](int c) { return !A.helm && kx == 0 && c == 0; },
          sm);
    }
    for (int tile = 0; tile < mt * nt; ++tile) {
      const int m0 = (tile % mt) * BM, n0 = (tile / mt) * BN;
      gemm_tile<TP>(
          My, Mt, My, m0, n0, [&](int m, int k) { return Cy[(size_t)k * My + m]; }, false,
          [&](int k, int n) { return S2[(size_t)n * My + k]; }, true,
          [&](int m, int n, TP v) { S1[(size_t)n * My + m] = v; }, true, sm);
    }
    __syncthreads();
  }
}

// Pass C: x += rn * (Cx^T ⊗ I) T1
template <typename TP>
__device__ void pass_c(const DctArgs<TP>& A, const Team& tm, double rn, TP* sm) {
  const int Mx = A.Mx, R = A.R;
  const int mt = (Mx + BM - 1) / BM, nt = (R + BN - 1) / BN;
  const TP* Cx = A.Cx;
  const TP* T1 = A.T1;
  double* x = A.x;
  for (int tile = tm.rank; tile < mt * nt; tile += tm.size) {
    const int m0 = (tile % mt) * BM, n0 = (tile / mt) * BN;
    gemm_tile<TP>(
        Mx, R, Mx, m0, n0, [&](int m, int k) { return Cx[(size_t)k * Mx + m]; }, false,
        [&](int k, int n) { return T1[(size_t)k * R + n]; }, false,
        [&](int m, int n, TP v) {
          const size_t c = (size_t)n * Mx + m;
          x[c] = fma(rn, widen(v), x[c]);
        },
        true, sm);
  }
}

// The passes on the tensor cores where the kernel opened them (tc not null;
// FP32 only), else on the FP32 / FP64 pipes. False if a wait ran out.
template <typename TP>
__device__ __forceinline__ bool run_pass_a(const DctArgs<TP>& A, const Team& tm, TP sc, TP off, TP* sm,
                                           TcState* tc) {
  if constexpr (sizeof(TP) == 4) {
    if (tc && A.tc_ac) return pass_a_tc(A, tm, sc, off, sm, *tc);
  }
  pass_a<TP>(A, tm, sc, off, sm);
  return true;
}

template <typename TP>
__device__ __forceinline__ bool run_pass_b(const DctArgs<TP>& A, const Team& tm, TP* sm, TcState* tc) {
  if constexpr (sizeof(TP) == 4) {
    if (tc && A.tc_slab) return pass_b_tc(A, tm, sm, *tc);
  }
  pass_b<TP>(A, tm, sm);
  return true;
}

template <typename TP>
__device__ __forceinline__ bool run_pass_c(const DctArgs<TP>& A, const Team& tm, double rn, TP* sm, TcState* tc) {
  if constexpr (sizeof(TP) == 4) {
    if (tc && A.tc_ac) return pass_c_tc(A, tm, rn, sm, *tc);
  }
  pass_c<TP>(A, tm, rn, sm);
  return true;
}

// The whole solve by one team of blocks (a whole grid is one team); sm is the
// block's dynamic shared memory. Returns false if a barrier gave up.
template <typename TP>
__device__ bool poisson_dct_team(const DctArgs<TP>& A, const Team& tm, TP* sm, TcState* tc) {
  __shared__ double s_diag[27];
  if (threadIdx.x < 27) {
    const int c = threadIdx.x;
    s_diag[c] = (c % 3) * A.cx + ((c / 3) % 3) * A.cy + (c / 9) * A.cz;
  }
  __syncthreads();
  unsigned int epoch = 0;
  const int n = A.n;
  const int t0 = tm.rank * blockDim.x + threadIdx.x, gsz = tm.size * blockDim.x;
  double* b = A.b;
  double* x = A.x;
  double* r = A.r;
  __shared__ struct {
    double mean, bn, rn, rmean, sc, off, pscale;
    int pexp, go, conv;   // pscale = 2^pexp
  } ds;
  double thr = 0.0;   // read by thread 0 only
  TP* rs = A.T2;       // the residual of the next sweep, staged in the transform type (T2 is free outside pass B)
  // consistency: remove the mean of the right-hand side (Neumann null space);
  // its norm, from the same sums, sets the power of two that scales the
  // first staged residual
  Vec<2> sb = {{0.0, 0.0}};
  for (int c = t0; c < n; c += gsz) {
    const double bc = b[c];
    sb.v[0] += bc;
    sb.v[1] += bc * bc;
  }
  if (!team_sum_post<2>(sb, tm, A.max_blocks, 0, A.st, epoch, [&](const double* tot) {
        ds.mean = tot[0] / (double)n;
        int e = 0;
        frexp(sqrt(fmax(tot[1] - (double)n * ds.mean * ds.mean, 0.0)), &e);
        ds.pscale = ldexp(1.0, -e);
        ds.pexp = -e;
      }))
    return false;
  const double mean_b = ds.mean;
  // Warm start: the x in place (the previous step's correction) is the first
  // iterate and r = b - A x the first residual; cold start: x = 0 and the
  // first residual is b itself.
  const bool warm = A.warm != 0;
  double ps = ds.pscale;   // the staged residual is r * ps (ps a power of two: exact)
  int pe = ds.pexp;
  Vec<3> s2 = {{0.0, 0.0, 0.0}};
  for (int c = t0; c < n; c += gsz) {
    const double bc = b[c] - mean_b;
    b[c] = bc;
    s2.v[0] += bc * bc;
    double rc = bc;
    if (warm) {
      int i, j, k;
      decompose3(c, A.fx, A.fy, i, j, k);
      const int code = ((i > 0) + (i < A.nx - 1)) + 3 * ((j > 0) + (j < A.ny - 1)) + 9 * ((k > 0) + (k < A.nz - 1));
      rc = res_lap64(bc, x, c, i, j, k, A.nx, A.ny, A.nz, A.cx, A.cy, A.cz, s_diag[code]);
      r[c] = rc;
      s2.v[1] += rc;
      s2.v[2] += rc * rc;
    } else {
      x[c] = 0.0;
    }
    rs[c] = narrow_scaled<TP>(rc, pe, ps);
  }
  if (!team_sum_post<3>(s2, tm, A.max_blocks, 1, A.st, epoch, [&](const double* tot) {
        ds.bn = sqrt(tot[0]);
        thr = A.tol * ds.bn;
        if (warm) {   // the part of r outside the constants, as after each sweep
          ds.rmean = tot[1] / (double)n;
          ds.rn = sqrt(fmax(tot[2] - (double)n * ds.rmean * ds.rmean, 0.0));
        } else {
          ds.rmean = 0.0;
          ds.rn = ds.bn;
        }
        ds.conv = ds.bn == 0.0 || ds.rn <= thr;
        ds.go = !ds.conv && isfinite(ds.rn);
        ds.sc = 1.0 / (ds.pscale * ds.rn);
        ds.off = -ds.rmean / ds.rn;
        int e = 0;
        frexp(ds.rn, &e);
        ds.pscale = ldexp(1.0, -e);   // for the residual of the next sweep
        ds.pexp = -e;
      }))
    return false;
  int sweeps = 0;
  while (ds.go && sweeps < A.max_sweeps) {
    ++sweeps;
    const double rn = ds.rn;
    ps = ds.pscale;
    pe = ds.pexp;
    if (!run_pass_a<TP>(A, tm, (TP)ds.sc, (TP)ds.off, sm, tc)) return false;
    if (!team_barrier(A.st, tm, epoch)) return false;
    if (!run_pass_b<TP>(A, tm, sm, tc)) return false;
    if (!team_barrier(A.st, tm, epoch)) return false;
    if (!run_pass_c<TP>(A, tm, rn, sm, tc)) return false;
    if (!team_barrier(A.st, tm, epoch)) return false;
    constexpr bool f32 = sizeof(TP) == 4;
    Vec<2> s = {{0.0, 0.0}};
    float f0 = 0.f, f1 = 0.f;   // FP32 partial sums of r * ps (FP32 path)
    int nf = 0;
    // two rows per pass (the second a repeat of the first past the end, then
    // dropped): two independent FP64 chains, whose loads overlap
    auto code_of = [&](int i, int j, int k) {
      return ((i > 0) + (i < A.nx - 1)) + 3 * ((j > 0) + (j < A.ny - 1)) + 9 * ((k > 0) + (k < A.nz - 1));
    };
    for (int c = t0; c < n; c += 2 * gsz) {
      const bool two = c + gsz < n;
      const int c2 = two ? c + gsz : c;
      int i, j, k, i2, j2, k2;
      decompose3(c, A.fx, A.fy, i, j, k);
      decompose3(c2, A.fx, A.fy, i2, j2, k2);
      const double r1 = res_lap64(b[c], x, c, i, j, k, A.nx, A.ny, A.nz, A.cx, A.cy, A.cz, s_diag[code_of(i, j, k)]);
      const double r2 =
          res_lap64(b[c2], x, c2, i2, j2, k2, A.nx, A.ny, A.nz, A.cx, A.cy, A.cz, s_diag[code_of(i2, j2, k2)]);
      const TP v1 = narrow_scaled<TP>(r1, pe, ps), v2 = narrow_scaled<TP>(r2, pe, ps);
      rs[c] = v1;
      if (two) rs[c2] = v2;
      if constexpr (f32) {
        const float w2 = two ? v2 : 0.f;
        f0 += v1;
        f0 += w2;
        f1 = fmaf(w2, w2, fmaf(v1, v1, f1));
        nf += 2;
        if (nf >= kNormChunk) {
          s.v[0] += f0;
          s.v[1] += f1;
          f0 = f1 = 0.f;
          nf = 0;
        }
      } else {
        s.v[0] += r1;
        s.v[1] += r1 * r1;
        if (two) {
          s.v[0] += r2;
          s.v[1] += r2 * r2;
        }
      }
    }
    if constexpr (f32) {
      s.v[0] += f0;
      s.v[1] += f1;
    }
    if (!team_sum_post<2>(s, tm, A.max_blocks, 2, A.st, epoch, [&](const double* tot) {
          // norm of the part of r outside the constants: sum (r - mean)^2 (the
          // FP32 path's sums are of r * ps: 1 / ps is exact)
          const double us = f32 ? 1.0 / ps : 1.0;
          const double m = tot[0] / (double)n;
          const double rmean = m * us;
          const double rn_new = us * sqrt(fmax(tot[1] - (double)n * m * m, 0.0));
          ds.conv = rn_new * (f32 ? kNormMargin : 1.0) <= thr;
          // stop when a sweep no longer halves the residual (rounding floor)
          ds.go = !ds.conv && isfinite(rn_new) && rn_new < 0.5 * ds.rn;
          ds.rn = rn_new;
          ds.rmean = rmean;
          ds.sc = 1.0 / (ds.pscale * rn_new);
          ds.off = -rmean / rn_new;
          int e = 0;
          frexp(rn_new, &e);
          ds.pscale = ldexp(1.0, -e);
          ds.pexp = -e;
        }))
      return false;
  }
  // gauge: zero-mean correction
  Vec<1> sx = {{0.0}};
  for (int c = t0; c < n; c += gsz) sx.v[0] += x[c];
  if (!team_sum_post<1>(sx, tm, A.max_blocks, 3, A.st, epoch,
                        [&](const double* tot) { ds.mean = tot[0] / (double)n; }))
    return false;
  const double mean_x = ds.mean;
  double* pp = A.p;
  for (int c = t0; c < n; c += gsz) {
    const double xc = x[c] - mean_x;
    x[c] = xc;
    if (pp) pp[c] += xc;
  }
  if (pp) {
    // the projection: every face reads p' on both sides, written above by any block
    if (!team_barrier(A.st, tm, epoch)) return false;
    const int nx = A.nx, ny = A.ny, nz = A.nz;
    const int nf[3] = {(nx + 1) * ny * nz, nx * (ny + 1) * nz, A.dim == 3 ? nx * ny * (nz + 1) : 0};
    const double kk = A.proj_k;
    for (int d = 0; d < 3; ++d) {
      if (nf[d] == 0) continue;
      const int nd = (d == 0) ? nx : (d == 1) ? ny : nz;
      const int sd = (d == 0) ? 1 : (d == 1) ? nx : nx * ny;
      double* out = A.vel[d];
      const double* in = A.us[d];
      const double ih = A.ih[d];
      const FastDiv ffx = A.ffx[d], ffy = A.ffy[d];
      for (int r = t0; r < nf[d]; r += gsz) {
        int i, j, k;
        decompose3(r, ffx, ffy, i, j, k);
        const int f = (d == 0) ? i : (d == 1) ? j : k;
        if (f == 0 || f == nd) {
          out[r] = 0.0;
          continue;
        }
        const int c_hi = i + nx * (j + ny * k);
        const double grad = (x[c_hi] - x[c_hi - sd]) * ih;
        out[r] = in[r] - kk * grad;
      }
    }
  }
  if (tm.rank == 0 && threadIdx.x == 0) {
    const double rel = ds.bn > 0.0 ? ds.rn / ds.bn : 0.0;
    SolveStat& so = A.st->stat[A.stat_index];
    so.iters = sweeps;
    so.iters_total += sweeps;
    so.refinements = sweeps;
    so.converged = ds.conv ? 1 : 0;
    so.nonfinite = isfinite(rel) ? 0 : 1;
    so.relres = rel;
    if (!isfinite(rel)) atomicExch(&A.st->sticky, (int)SS_ENAN);
    else if (!ds.conv) atomicCAS(&A.st->sticky, (int)SS_OK, (int)SS_ENOTCONV);
  }
  return true;
}

// b_r - (A x)_r for one row of a DIA system in FP64, each product fused into
// the running difference (the guard bands make every neighbour read valid; an
// absent neighbour's coefficient is 0).
__device__ __forceinline__ double res64(double br, const Planes<double>& a, const double* x, int r, int sy, int sz,
                                        int has_z) {
  double acc = fma(-a.P[r], x[r], br);
  acc = fma(-a.W[r], x[r - 1], acc);
  acc = fma(-a.E[r], x[r + 1], acc);
  acc = fma(-a.S[r], x[r - sy], acc);
  acc = fma(-a.N[r], x[r + sy], acc);
  if (has_z) {
    acc = fma(-a.B[r], x[r - sz], acc);
    acc = fma(-a.T_[r], x[r + sz], acc);
  }
  return acc;
}

// The T* system (Eq. 3.12) by FP64 defect correction around the inverse of
// its constant-coefficient part I/dt - alpha L (zero-flux walls), by the
// same transforms with the shift 1/(alpha dt): each sweep forms the FP64
// residual b - A x with the system's own FP64 planes (upwind convection and
// cooled walls included), applies the inverse and adds the correction. The
// parts the inverse leaves out are small beside 1/dt where this is used, so
// a sweep reduces the residual by ~1e-3. The caller's BiCGSTAB refinement
// follows: when the sweeps met the tolerance on the true FP64 residual
// (status block: presolve_done, presolve_rel) it only records that, else it
// continues from x. The sweeps are counted in the status block's pre-solve
// counter. x holds the initial guess.
__device__ bool helmholtz_team(const DctArgs<float>& A, const Sys& S, int has_z, double inv_alpha, int max_sweeps,
                               const Team& tm, float* sm, TcState* tc) {
  unsigned int epoch = 0;
  const int n = (int)S.d.n;
  const int sy = S.d.mx, sz = S.d.mx * S.d.my;
  const int t0 = tm.rank * blockDim.x + threadIdx.x, gsz = tm.size * blockDim.x;
  const double* b = S.b;
  double* x = S.x;
  float* rs = A.T2;
  __shared__ struct {
    double rn, bn, sc, pscale;
    int pexp, go, conv;   // pscale = 2^pexp
  } hs;
  double thr = 0.0;   // read by thread 0 only
  double ps = 1.0;    // the first staged residual is not scaled (T* residuals are O(1) in K/s)
  if (tm.rank == 0 && threadIdx.x == 0) A.st->presolve_done = 0;
  Vec<2> s0 = {{0.0, 0.0}};
  for (int c = t0; c < n; c += gsz) {
    const double rc = res64(b[c], S.a, x, c, sy, sz, has_z);
    rs[c] = to_f32(rc);
    s0.v[0] += b[c] * b[c];
    s0.v[1] += rc * rc;
  }
  if (!team_sum_post<2>(s0, tm, A.max_blocks, 0, A.st, epoch, [&](const double* tot) {
        const double bn = sqrt(tot[0]);
        hs.bn = bn;
        hs.rn = sqrt(tot[1]);
        thr = A.tol * bn;
        hs.conv = bn == 0.0 || hs.rn <= thr;
        hs.go = bn > 0.0 && hs.rn > thr && isfinite(hs.rn);
        hs.sc = 1.0 / hs.rn;
        int e = 0;
        frexp(hs.rn, &e);
        hs.pscale = ldexp(1.0, -e);
        hs.pexp = -e;
      }))
    return false;
  int sweeps = 0;
  while (hs.go && sweeps < max_sweeps) {
    ++sweeps;
    const double rn = hs.rn;
    if (!run_pass_a<float>(A, tm, (float)hs.sc, 0.f, sm, tc)) return false;
    if (!team_barrier(A.st, tm, epoch)) return false;
    if (!run_pass_b<float>(A, tm, sm, tc)) return false;
    if (!team_barrier(A.st, tm, epoch)) return false;
    if (!run_pass_c<float>(A, tm, rn * inv_alpha, sm, tc)) return false;
    if (!team_barrier(A.st, tm, epoch)) return false;
    ps = hs.pscale;
    const int pe = hs.pexp;
    // the norm from FP32 partial sums of the staged r * ps (see kNormChunk)
    Vec<1> s1 = {{0.0}};
    float f1 = 0.f;
    int nf = 0;
    // two rows per pass (the second a repeat of the first past the end, then
    // dropped): two independent FP64 chains, whose loads overlap
    for (int c = t0; c < n; c += 2 * gsz) {
      const bool two = c + gsz < n;
      const int c2 = two ? c + gsz : c;
      const double r1 = res64(b[c], S.a, x, c, sy, sz, has_z);
      const double r2 = res64(b[c2], S.a, x, c2, sy, sz, has_z);
      const float v1 = to_f32_scaled(r1, pe, ps), v2 = two ? to_f32_scaled(r2, pe, ps) : 0.f;
      rs[c] = v1;
      if (two) rs[c2] = v2;
      f1 = fmaf(v2, v2, fmaf(v1, v1, f1));
      nf += 2;
      if (nf >= kNormChunk) {
        s1.v[0] += f1;
        f1 = 0.f;
        nf = 0;
      }
    }
    s1.v[0] += f1;
    if (!team_sum_post<1>(s1, tm, A.max_blocks, 1, A.st, epoch, [&](const double* tot) {
          const double rn_new = sqrt(tot[0]) / ps;
          hs.conv = rn_new * kNormMargin <= thr;
          hs.go = !hs.conv && isfinite(rn_new) && rn_new < 0.5 * hs.rn;
          hs.sc = 1.0 / (hs.pscale * rn_new);
          hs.rn = rn_new;
          int e = 0;
          frexp(rn_new, &e);
          hs.pscale = ldexp(1.0, -e);
          hs.pexp = -e;
        }))
      return false;
  }
  if (tm.rank == 0 && threadIdx.x == 0) {
    A.st->presolve_sweeps += sweeps;
    A.st->presolve_rel = hs.bn > 0.0 ? hs.rn / hs.bn : 0.0;
    A.st->presolve_done = hs.conv;
  }
  return true;
}

struct HelmArgs {
  DctArgs<float> dct;
  Sys sys;
  int has_z;
  double inv_alpha;
  int max_sweeps;
};

// Runs f(tc) with the block's tensor cores opened (TMEM allocated, closed
// again on every way out) when on, else f(nullptr).
template <class F>
__device__ __forceinline__ void with_tc(bool on, F f) {
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) unsigned long long s_mbar[kTcBarriers];
  if (on) {
    TcState tc;
    tc_open(tc, &s_tmem, s_mbar);
    f(&tc);
    tc_close(tc);
  } else {
    f(nullptr);
  }
}

__global__ void __launch_bounds__(kBlock, 1) k_helmholtz_dct(HelmArgs H) {
  extern __shared__ __align__(16) unsigned char dsm[];
  const Team tm{(int)blockIdx.x, (int)gridDim.x, &H.dct.st->barrier, H.dct.partial};
  with_tc(H.dct.tc != 0, [&](TcState* tc) {
    helmholtz_team(H.dct, H.sys, H.has_z, H.inv_alpha, H.max_sweeps, tm, reinterpret_cast<float*>(dsm), tc);
  });
}

// The T* pre-solve of a packed batch: team q runs case q's sweeps (none
// where the case's walls or size rule it out: max_sweeps = 0).
__global__ void __launch_bounds__(kBlock, 1) k_helmholtz_dct_packed(const HelmArgs* __restrict__ args,
                                                                   const int* __restrict__ first, int nteams) {
  extern __shared__ __align__(16) unsigned char dsm[];
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
  const int q = s_team;
  __shared__ __align__(16) unsigned long long buf[(sizeof(HelmArgs) + 7) / 8];
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(args + q);
  for (int w = threadIdx.x; w < (int)(sizeof(HelmArgs) / 8); w += blockDim.x) buf[w] = src[w];
  __syncthreads();
  const HelmArgs& H = *reinterpret_cast<const HelmArgs*>(buf);
  if (H.max_sweeps <= 0) return;
  const Team tm{(int)blockIdx.x - first[q], first[q + 1] - first[q], &H.dct.st->barrier, H.dct.partial};
  with_tc(H.dct.tc != 0, [&](TcState* tc) {
    helmholtz_team(H.dct, H.sys, H.has_z, H.inv_alpha, H.max_sweeps, tm, reinterpret_cast<float*>(dsm), tc);
  });
}

template <typename TP>
__global__ void __launch_bounds__(kBlock, 1) k_poisson_dct(DctArgs<TP> A) {
  extern __shared__ __align__(16) unsigned char dsm[];
  const Team tm{(int)blockIdx.x, (int)gridDim.x, &A.st->barrier, A.partial};
  if constexpr (sizeof(TP) == 4) {
    with_tc(A.tc != 0, [&](TcState* tc) { poisson_dct_team<TP>(A, tm, reinterpret_cast<TP*>(dsm), tc); });
  } else {
    poisson_dct_team<TP>(A, tm, reinterpret_cast<TP*>(dsm), nullptr);
  }
}

// Rows of a staged image of an n x n matrix: whole tiles of 128 rows plus
// one more, so that any tile of rows the passes stage lies inside it (the
// rows beyond n are zero).
size_t tc_image_rows(int n) { return (size_t)((n + kTcM - 1) / kTcM) * kTcM + kTcM; }

// Bytes of that image: per chunk of kTcKc values of K, the hi and the lo half.
size_t tc_image_bytes(int n) {
  const size_t chunks = (size_t)(n + kTcKc - 1) / kTcKc;
  return chunks * 2 * (tc_image_rows(n) / 8) * kTcSbo;
}

// FP32 -> TF32, round to nearest, ties to even (the device's tf32_rn, on the host)
float tf32_rn_host(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u += 0xFFFu + ((u >> 13) & 1u);
  u &= 0xFFFFE000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

// The image of the n x n operand f(r, k) in the staged layout of tc_stage.
template <class F>
void tc_image(int n, F f, unsigned char* out) {
  const size_t rows = tc_image_rows(n), half = rows / 8 * kTcSbo;
  const int chunks = (n + kTcKc - 1) / kTcKc;
  std::memset(out, 0, tc_image_bytes(n));
  for (int c = 0; c < chunks; ++c) {
    unsigned char* hi = out + (size_t)c * 2 * half;
    unsigned char* lo = hi + half;
    for (int r = 0; r < n; ++r)
      for (int kk = 0; kk < kTcKc && c * kTcKc + kk < n; ++kk) {
        const float v = f(r, c * kTcKc + kk);
        const float h = tf32_rn_host(v), l = tf32_rn_host(v - h);
        const size_t off = (size_t)(r >> 3) * kTcSbo + (size_t)(kk >> 2) * 128 + (size_t)(r & 7) * 16 + (kk & 3) * 4;
        std::memcpy(hi + off, &h, 4);
        std::memcpy(lo + off, &l, 4);
      }
  }
}

// Shared memory a block may give the slab-resident pass B.
constexpr size_t kSlabSmemBytes = 200 * 1024;

template <typename TP>
size_t smem_bytes(const DctPlan& pl, int* cols, int* slab, int* tc, int* tc_ac, int* tc_slab) {
  const int P = (pl.Mt & 1) ? pl.Mt : pl.Mt + 1;
  const int ncols = pl.dim == 3 ? pl.My : pl.Mx;
  long long w = (long long)(kThomasSmemBytes / (2 * (size_t)P * sizeof(TP)));
  if (w > ncols) w = ncols;
  if (w > 4 * kBlock) w = 4 * kBlock;
  if (w < 1) w = 1;
  *cols = (int)w;
  const size_t thomas = 2 * (size_t)w * P * sizeof(TP);
  const size_t gemm = (size_t)kGemmSmemElems * sizeof(TP);
  size_t need = thomas > gemm ? thomas : gemm;
  const size_t slab_bytes = slab_smem_floats(pl.My, pl.Mt) * sizeof(float);
  *slab = sizeof(TP) == 4 && pl.dim == 3 && slab_bytes <= kSlabSmemBytes;
  if (*slab && slab_bytes > need) need = slab_bytes;
  // the tensor-core passes (FP32): tiles of width up to kTcMaxWidth in A and
  // C, where the grid is large enough; in B the slab's accumulator width,
  // its transformed slab and the eliminated super-diagonal
  *tc_ac = sizeof(TP) == 4 && pl.tc_mode != SS_TC_OFF &&
           (pl.tc_mode == SS_TC_ON || (long long)pl.Mx * pl.Mx * pl.My * pl.Mt >= kTcAcMinWork);
  *tc_slab = 0;
  if (*tc_ac) {
    const size_t ac = tc_smem_bytes(kTcMaxWidth);
    if (ac > need) need = ac;
  }
  if (sizeof(TP) == 4 && pl.tc_mode != SS_TC_OFF) {
    const int wt = (pl.Mt + 15) & ~15;
    const size_t b = tc_smem_bytes(wt) + 2 * (size_t)pl.Mt * tc_slab_row(pl.My) * sizeof(float);
    if (pl.dim == 3 && pl.My <= kTcM && wt <= kTcCols && b <= kSlabSmemBytes) {
      *tc_slab = 1;
      *slab = 0;
      if (b > need) need = b;
    }
  }
  *tc = *tc_ac || *tc_slab;
  return need;
}

// A packed launch over the cases of a batch: team q (blocks first[q] ..
// first[q+1]-1) solves case q's pressure correction with its own arguments
// (staged in shared memory), barrier counter and reduction partials.
__global__ void __launch_bounds__(kBlock, 1) k_poisson_dct_packed(const DctArgs<float>* __restrict__ args,
                                                                 const int* __restrict__ first, int nteams) {
  extern __shared__ __align__(16) unsigned char dsm[];
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
  const int q = s_team;
  __shared__ __align__(16) unsigned long long buf[(sizeof(DctArgs<float>) + 7) / 8];
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(args + q);
  for (int w = threadIdx.x; w < (int)(sizeof(DctArgs<float>) / 8); w += blockDim.x) buf[w] = src[w];
  __syncthreads();
  const DctArgs<float>& A = *reinterpret_cast<const DctArgs<float>*>(buf);
  const Team tm{(int)blockIdx.x - first[q], first[q + 1] - first[q], &A.st->barrier, A.partial};
  with_tc(A.tc != 0, [&](TcState* tc) { poisson_dct_team<float>(A, tm, reinterpret_cast<float*>(dsm), tc); });
}

// The arguments of one solve; returns the dynamic shared memory it needs.
template <typename TP>
size_t make_args(DctArgs<TP>& A, const DctPlan& pl, const Params& pr, double* b, double* x, const SolverCtl& ctl,
                 Scratch& sc, DevStatus* st, const ProjectPtrs* proj) {
  memset(&A, 0, sizeof A);
  if (proj) {
    A.p = proj->p;
    for (int d = 0; d < 3; ++d) {
      A.vel[d] = proj->vel[d];
      A.us[d] = proj->us[d];
      A.ih[d] = pr.ih[d];
      A.ffx[d] = make_fastdiv(pr.nx + (d == 0));
      A.ffy[d] = make_fastdiv(pr.ny + (d == 1));
    }
    A.proj_k = pr.proj_k;
  }
  A.Mx = pl.Mx; A.My = pl.My; A.Mt = pl.Mt; A.R = pl.My * pl.Mt; A.dim = pl.dim;
  A.nx = pr.nx; A.ny = pr.ny; A.nz = pr.nz; A.n = pr.nx * pr.ny * pr.nz;
  A.fx = make_fastdiv(pr.nx);
  A.fy = make_fastdiv(pr.ny);
  A.cx = 1.0 / (pr.hx * pr.hx);
  A.cy = 1.0 / (pr.hy * pr.hy);
  A.cz = pr.dim == 3 ? 1.0 / (pr.hz * pr.hz) : 0.0;
  const double ht = pr.dim == 3 ? pr.hz : pr.hy;
  A.at = (TP)(1.0 / (ht * ht));
  const TP* tab = (const TP*)pl.tables;
  A.Cx = tab;
  A.Cy = tab + (size_t)pl.Mx * pl.Mx;
  A.lx = A.Cy + (size_t)pl.My * pl.My;
  A.ly = A.lx + pl.Mx;
  A.T1 = (TP*)pl.T1;
  A.T2 = (TP*)pl.T2;
  A.tinv = (sizeof(TP) == 4 && pl.thomas && pl.thomas_p) ? (const float*)pl.thomas : nullptr;
  A.b = b; A.x = x; A.r = sc.v[0];
  A.tol = ctl.tol;
  A.warm = ctl.warm_start;
  A.max_sweeps = ctl.max_it < kMaxSweeps ? ctl.max_it : kMaxSweeps;
  A.stat_index = ctl.stat_index;
  A.partial = sc.partial;
  A.max_blocks = sc.max_blocks;
  A.st = st;
  const size_t need = smem_bytes<TP>(pl, &A.thomas_cols, &A.slab_smem, &A.tc, &A.tc_ac, &A.tc_slab);
  if (A.tc && pl.img) {
    const unsigned char* img = (const unsigned char*)pl.img;
    A.img_gx = (int)(tc_image_rows(pl.Mx) / 8);
    A.img_gy = (int)(tc_image_rows(pl.My) / 8);
    A.img_cx = img;
    A.img_cxt = A.img_cx + tc_image_bytes(pl.Mx);
    A.img_cy = pl.dim == 3 ? A.img_cxt + tc_image_bytes(pl.Mx) : nullptr;
    A.img_cyt = pl.dim == 3 ? A.img_cy + tc_image_bytes(pl.My) : nullptr;
  }
  return need;
}

template <typename TP>
cudaError_t launch_t(const DctPlan& pl, const Params& pr, double* b, double* x, const SolverCtl& ctl, Scratch& sc,
                     DevStatus* st, const ProjectPtrs* proj, cudaStream_t s) {
  DctArgs<TP> A;
  const size_t smem = make_args<TP>(A, pl, pr, b, x, ctl, sc, st, proj);
  const void* kern = (const void*)k_poisson_dct<TP>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int cap = ctl.block_cap > 0 && ctl.block_cap < sc.max_blocks ? ctl.block_cap : sc.max_blocks;
  const int nb = coop_blocks_for_smem(kern, (long long)A.n, cap, smem);
  if ((e = cudaMemsetAsync(&st->barrier, 0, sizeof(unsigned int), s)) != cudaSuccess) return e;
  void* args[] = {&A};
  return cudaLaunchCooperativeKernel(kern, dim3(nb), dim3(kBlock), args, smem, s);
}

}  // namespace

void plan_dct(const Params& pr, DctPlan& pl, int fp32) {
  memset(&pl, 0, sizeof pl);
  pl.dim = pr.dim;
  pl.Mx = pr.nx;
  pl.My = pr.dim == 3 ? pr.ny : 1;
  pl.Mt = pr.dim == 3 ? pr.nz : pr.ny;
  pl.fp32 = fp32;
}

size_t dct_table_elems(const DctPlan& pl) {
  return (size_t)pl.Mx * pl.Mx + (size_t)pl.My * pl.My + pl.Mx + pl.My;
}

// Orthonormal DCT-II matrices and the eigenvalues of the 1D operators, in
// FP64 on the host: C[k][i] = s_k cos(pi k (2i + 1) / (2n)), s_0 = sqrt(1/n),
// s_k = sqrt(2/n); lambda_k = (4/h^2) sin^2(pi k / (2n)).
void dct_tables(const DctPlan& pl, const Params& pr, double* out) {
  const double pi = 3.14159265358979323846;
  auto fill = [&](int nn, double h, double* C, double* lam) {
    for (int k = 0; k < nn; ++k) {
      const double s = std::sqrt((k == 0 ? 1.0 : 2.0) / nn);
      for (int i = 0; i < nn; ++i) C[(size_t)k * nn + i] = s * std::cos(pi * k * (2.0 * i + 1.0) / (2.0 * nn));
      const double sn = std::sin(pi * k / (2.0 * nn));
      lam[k] = 4.0 * sn * sn / (h * h);
    }
  };
  double* Cx = out;
  double* Cy = Cx + (size_t)pl.Mx * pl.Mx;
  double* lx = Cy + (size_t)pl.My * pl.My;
  double* ly = lx + pl.Mx;
  fill(pl.Mx, pr.hx, Cx, lx);
  if (pl.dim == 3) {
    fill(pl.My, pr.hy, Cy, ly);
  } else {
    Cy[0] = 1.0;
    ly[0] = 0.0;
  }
}

size_t dct_image_bytes(const DctPlan& pl) {
  if (!pl.fp32) return 0;
  return 2 * tc_image_bytes(pl.Mx) + (pl.dim == 3 ? 2 * tc_image_bytes(pl.My) : 0);
}

// Cx as rows m (K along i), Cx^T as rows i (K along m), and in 3D Cy as rows
// ky (K along j), Cy^T as rows j (K along ky): the constant operands of
// passes A, C and B.
void dct_images(const DctPlan& pl, const float* Cx, const float* Cy, unsigned char* out) {
  if (!pl.fp32) return;
  const int Mx = pl.Mx, My = pl.My;
  unsigned char* p = out;
  tc_image(Mx, [&](int r, int k) { return Cx[(size_t)r * Mx + k]; }, p);
  p += tc_image_bytes(Mx);
  tc_image(Mx, [&](int r, int k) { return Cx[(size_t)k * Mx + r]; }, p);
  p += tc_image_bytes(Mx);
  if (pl.dim == 3) {
    tc_image(My, [&](int r, int k) { return Cy[(size_t)r * My + k]; }, p);
    p += tc_image_bytes(My);
    tc_image(My, [&](int r, int k) { return Cy[(size_t)k * My + r]; }, p);
  }
}

namespace {
// 1/d_t of the factorisation of T_t + (lx[kx] + ly[c] + shift) I for every
// column (kx, c): the recurrence of slab_thomas, once per operator
__global__ void k_thomas_table(float* inv, const float* lx, const float* ly, float at, float shift, int helm, int Mx,
                               int My, int Mt) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)Mx * My) return;
  const int kx = (int)(id / My), c = (int)(id - (long long)kx * My);
  const float s = lx[kx] + ly[c] + shift;
  const bool singular = !helm && kx == 0 && c == 0;
  const int m = singular ? Mt - 1 : Mt;
  float* o = inv + (size_t)kx * Mt * My + c;
  float prev_c = 0.f;
  for (int t = 0; t < Mt; ++t) {
    float v = 0.f;
    if (t < m) {
      const float nb = (float)((t > 0) + (t < Mt - 1));
      const float d = fmaf(at, prev_c, fmaf(at, nb, s));
      v = 1.f / d;
      prev_c = -at * v;
    }
    o[(size_t)t * My] = v;
  }
}
}  // namespace

size_t dct_thomas_bytes(const DctPlan& pl) {
  if (!pl.fp32 || pl.dim != 3) return 0;
  // only the slab solves read the tables: the tensor-core slab (any mode but
  // off) or the shared-memory slab (tensor cores off)
  DctPlan q = pl;
  int cols, slab, tc, tc_ac, tc_slab;
  q.tc_mode = SS_TC_AUTO;
  smem_bytes<float>(q, &cols, &slab, &tc, &tc_ac, &tc_slab);
  const bool slab_tc = tc_slab != 0;
  q.tc_mode = SS_TC_OFF;
  smem_bytes<float>(q, &cols, &slab, &tc, &tc_ac, &tc_slab);
  if (!slab_tc && !slab) return 0;
  return 2 * (size_t)pl.Mx * pl.My * pl.Mt * sizeof(float);
}

cudaError_t dct_thomas_ensure(DctPlan& pl, const Params& pr, cudaStream_t s) {
  if (!pl.thomas || !pl.tables || !pl.fp32 || pl.dim != 3) return cudaSuccess;
  const size_t n = (size_t)pl.Mx * pl.My * pl.Mt;
  const float* lx = (const float*)pl.tables + (size_t)pl.Mx * pl.Mx + (size_t)pl.My * pl.My;
  const float* ly = lx + pl.Mx;
  const float at = (float)(1.0 / (pr.hz * pr.hz));   // the transforms' 1/h^2 along the tridiagonal axis
  const int threads = 256;
  const int blocks = (int)(((long long)pl.Mx * pl.My + threads - 1) / threads);
  float* tab = (float*)pl.thomas;
  if (!pl.thomas_p) {
    k_thomas_table<<<blocks, threads, 0, s>>>(tab, lx, ly, at, 0.f, 0, pl.Mx, pl.My, pl.Mt);
    pl.thomas_p = 1;
  }
  const double sh = 1.0 / (pr.alphaT * pr.dt);   // the T* pre-solve's shift (as in its arguments)
  if (std::isfinite(sh) && (!pl.thomas_h || sh != pl.thomas_shift)) {
    k_thomas_table<<<blocks, threads, 0, s>>>(tab + n, lx, ly, at, (float)sh, 1, pl.Mx, pl.My, pl.Mt);
    pl.thomas_h = 1;
    pl.thomas_shift = sh;
  }
  return cudaGetLastError();
}

namespace {
size_t make_helm_args(HelmArgs& H, const DctPlan& pl, const Params& pr, const Sys& sys, int has_z, int max_sweeps,
                      const SolverCtl& ctl, Scratch& sc, DevStatus* st) {
  memset(&H, 0, sizeof H);
  const size_t smem = make_args<float>(H.dct, pl, pr, sys.b, sys.x, ctl, sc, st, nullptr);
  H.dct.helm = 1;
  H.dct.shift = 1.0 / (pr.alphaT * pr.dt);   // 1/(alpha dt), in the 1/h^2 units of the transforms
  H.dct.tinv = (pl.thomas && pl.thomas_h && pl.thomas_shift == H.dct.shift)
                   ? (const float*)pl.thomas + (size_t)pl.Mx * pl.My * pl.Mt
                   : nullptr;
  H.sys = sys;
  H.has_z = has_z;
  H.inv_alpha = 1.0 / pr.alphaT;
  H.max_sweeps = max_sweeps;
  return smem;
}
}  // namespace

size_t packed_helm_args_bytes() { return sizeof(HelmArgs); }

size_t fill_packed_helm_args(void* out, const DctPlan& pl, const Params& pr, const Sys& sys, int has_z,
                             int max_sweeps, const SolverCtl& ctl, Scratch& sc, DevStatus* st) {
  HelmArgs& H = *static_cast<HelmArgs*>(out);
  if (!pl.fp32 || !pl.tables) {
    memset(&H, 0, sizeof H);
    return 0;
  }
  return make_helm_args(H, pl, pr, sys, has_z, max_sweeps, ctl, sc, st);
}

cudaError_t launch_helmholtz_dct_packed(const void* args, const int* first, int nteams, int nblocks, size_t smem,
                                        cudaStream_t s) {
  const void* kern = (const void*)k_helmholtz_dct_packed;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* a[] = {(void*)&args, (void*)&first, (void*)&nteams};
  return cudaLaunchCooperativeKernel(kern, dim3(nblocks), dim3(kBlock), a, smem, s);
}

int packed_helm_max_blocks(size_t smem) {
  const void* kern = (const void*)k_helmholtz_dct_packed;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  return coop_blocks_for_smem(kern, 1LL << 40, 1 << 30, smem);
}

cudaError_t launch_helmholtz_dct(const DctPlan& pl, const Params& pr, const Sys& sys, int has_z, int max_sweeps,
                                 const SolverCtl& ctl, Scratch& sc, DevStatus* st, cudaStream_t s) {
  if (!pl.fp32) return cudaErrorInvalidValue;
  HelmArgs H;
  const size_t smem = make_helm_args(H, pl, pr, sys, has_z, max_sweeps, ctl, sc, st);
  const void* kern = (const void*)k_helmholtz_dct;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int cap = ctl.block_cap > 0 && ctl.block_cap < sc.max_blocks ? ctl.block_cap : sc.max_blocks;
  const int nb = coop_blocks_for_smem(kern, (long long)sys.d.n, cap, smem);
  if ((e = cudaMemsetAsync(&st->barrier, 0, sizeof(unsigned int), s)) != cudaSuccess) return e;
  void* args[] = {&H};
  return cudaLaunchCooperativeKernel(kern, dim3(nb), dim3(kBlock), args, smem, s);
}

size_t packed_dct_args_bytes() { return sizeof(DctArgs<float>); }

size_t fill_packed_dct_args(void* out, const DctPlan& pl, const Params& pr, double* b, double* x, const SolverCtl& ctl,
                            Scratch& sc, DevStatus* st, const ProjectPtrs* proj) {
  return make_args<float>(*static_cast<DctArgs<float>*>(out), pl, pr, b, x, ctl, sc, st, proj);
}

int packed_dct_max_blocks(size_t smem) {
  const void* kern = (const void*)k_poisson_dct_packed;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  return coop_blocks_for_smem(kern, 1LL << 40, 1 << 30, smem);
}

cudaError_t launch_poisson_dct_packed(const void* args, const int* first, int nteams, int nblocks, size_t smem,
                                      cudaStream_t s) {
  const void* kern = (const void*)k_poisson_dct_packed;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* a[] = {(void*)&args, (void*)&first, (void*)&nteams};
  return cudaLaunchCooperativeKernel(kern, dim3(nblocks), dim3(kBlock), a, smem, s);
}

cudaError_t launch_poisson_dct(const DctPlan& pl, const Params& pr, double* b, double* x, const SolverCtl& ctl,
                               Scratch& sc, DevStatus* st, const ProjectPtrs* proj, cudaStream_t s) {
  if (pl.fp32) return launch_t<float>(pl, pr, b, x, ctl, sc, st, proj, s);
  return launch_t<double>(pl, pr, b, x, ctl, sc, st, proj, s);
}

}  // namespace solid
