// tcgen05 (fifth-generation tensor core) building blocks for FP32 GEMM
// tiles: operands staged in shared memory as pairs of TF32 values
// (hi = x rounded to TF32, lo = x - hi rounded to TF32), the product formed
// as hi*hi + hi*lo + lo*hi by three tcgen05.mma of kind::tf32 per K step
// into one FP32 accumulator in tensor memory (TMEM). The dropped lo*lo term
// and the truncation of lo leave a relative error of a few 2^-22 per
// product, about FP32's own rounding, against 2^-11 for plain TF32.
//
// Layout: both operands K-major in the canonical no-swizzle form of the
// shared-memory matrix descriptor: core matrices of 8 rows x 16 bytes
// (4 FP32), the core matrices along K 128 bytes apart (leading byte offset),
// so one K step of 8 is two adjacent core matrices, and 8-row groups
// kTcSbo = 32 kTcKc + 16 bytes apart (stride byte offset) for a chunk of
// kTcKc values of K. The extra 16 bytes put the rows of a group and the
// groups on different shared-memory banks, so the 16-byte stores of the
// staging threads are conflict-free. Constant operands (cosine matrices)
// are stored once in exactly this layout and come into the staging buffers
// by bulk copies (cp.async.bulk) that complete on an mbarrier per buffer,
// while the threads stage the data operand.
//
// Accumulator: M = 128 rows, row i in TMEM lane i, column j in TMEM column
// j (32-bit). Warp w reads lanes 32 (w % 4) .. 32 (w % 4) + 31.
//
// Every wait is bounded: a wait that runs out sets the case's error flag,
// and the caller's next team barrier unwinds the kernel (which still frees
// its TMEM on the way out).
#pragma once

#include <cstdint>

#include "solid_internal.cuh"

namespace solid {

constexpr int kTcM = 128;            // accumulator rows (one TMEM lane each)
constexpr int kTcCols = 256;         // TMEM columns a block allocates (the widest accumulator)
constexpr int kTcKc = 32;            // K values per staged chunk
constexpr int kTcSbo = 32 * kTcKc + 16;   // bytes between 8-row groups of a chunk
constexpr long long kTcWaitPolls = 1ll << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// FP32 -> TF32 (10-bit significand), round to nearest, ties to even, on the
// integer pipes; finite inputs of moderate size (the transform operands).
__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t u = __float_as_uint(x);
  u += 0xFFFu + ((u >> 13) & 1u);
  return __uint_as_float(u & 0xFFFFE000u);
}

// byte offset of the 16-byte group k4 (values 4 k4 .. 4 k4 + 3) of row r of
// a staged K-major chunk
__device__ __forceinline__ uint32_t kmaj_off4(int r, int k4) {
  return (uint32_t)((r >> 3) * kTcSbo + k4 * 128 + (r & 7) * 16);
}

// shared-memory matrix descriptor of a K-major chunk starting at saddr
// (16-byte aligned): no swizzle, leading byte offset 128, stride byte
// offset kTcSbo, descriptor version 1
__device__ __forceinline__ uint64_t kmaj_desc(uint32_t saddr) {
  const uint64_t lbo = 128, sbo = kTcSbo;
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((lbo >> 4) << 16) | ((sbo >> 4) << 32) | (1ull << 46);
}

// instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B,
// both K-major, no negation, M x N
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes -> visible to the tensor core's reads
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D (+)= A B^T for one K step (issued by one thread)
__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// the mbarrier at mbar receives one arrival when the MMAs issued so far complete
__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one arrival on the mbarrier that also expects `bytes` of asynchronous copies
// to complete on it (the phase ends when both have happened)
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// bulk copy (the copy engine, no threads) of `bytes` from global memory to
// this block's shared memory, completing on mbar; both addresses 16-byte
// aligned and bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

// bounded wait for the phase with the given parity to complete
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (long long i = 0; i < kTcWaitPolls; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// 16 consecutive 32-bit columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}


// The block's tensor-core state: its TMEM columns and one mbarrier per
// staging buffer (the MMAs of a chunk complete on its buffer's barrier).
// Set up by tc_open (all threads) at the start of a kernel and released by
// tc_close (all threads) at its end.
struct TcState {
  uint32_t tmem;       // TMEM address of column 0, lane 0
  uint32_t mbar[2];    // shared addresses of the two mbarriers the MMAs complete on
  uint32_t phase[2];   // parity of the next phase to wait for on each
  uint32_t cbar[2];    // and of the two the bulk copies of constant operands complete on
  uint32_t cphase[2];
  uint32_t xbar;       // one more for a caller's own bulk copies
  uint32_t xphase;
};

// mbarriers tc_open sets up (s_mbar of tc_open holds this many)
constexpr int kTcBarriers = 5;

__device__ __forceinline__ void tc_open(TcState& tc, uint32_t* s_tmem, unsigned long long* s_mbar) {
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                 "r"((uint32_t)kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 32)
    for (int q = 0; q < kTcBarriers; ++q) mbar_init(smem_u32(s_mbar + q), 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  tc.tmem = *s_tmem;
  tc.mbar[0] = smem_u32(s_mbar);
  tc.mbar[1] = smem_u32(s_mbar + 1);
  tc.phase[0] = tc.phase[1] = 0;
  tc.cbar[0] = smem_u32(s_mbar + 2);
  tc.cbar[1] = smem_u32(s_mbar + 3);
  tc.cphase[0] = tc.cphase[1] = 0;
  tc.xbar = smem_u32(s_mbar + 4);
  tc.xphase = 0;
}

__device__ __forceinline__ void tc_close(const TcState& tc) {
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tc.tmem), "r"((uint32_t)kTcCols)
                 : "memory");
  }
}

// A GEMM operand in global or shared memory: element (r, k) at
// p[r * rs + k * ks], the value p[..] * sc + off for r < rows and k < cols
// and 0 elsewhere. rfast: consecutive rows are adjacent (rs = 1), else
// consecutive k (ks = 1).
struct TcOperand {
  const float* p;
  long long rs, ks;
  int rows, cols;
  float sc, off;
  int rfast;
  // or, for a constant operand, its image in the staged layout (per chunk of
  // kTcKc values of K: the hi then the lo half, each img_groups 8-row groups
  // of kTcSbo bytes), which the copy engine brings in (tc_image_async)
  const unsigned char* img = nullptr;
  int img_groups = 0;
};

__device__ __forceinline__ float tc_elem(const TcOperand& o, int r, int k) {
  return (r < o.rows && k < o.cols) ? fmaf(o.p[(long long)r * o.rs + (long long)k * o.ks], o.sc, o.off) : 0.f;
}

// 16-byte loads are possible when the pointer and the strided dimension
// keep every group of four on a 16-byte boundary
__device__ __forceinline__ bool tc_vec(const TcOperand& o) {
  return ((reinterpret_cast<uintptr_t>(o.p) & 15) == 0) && (((o.rfast ? o.ks : o.rs) & 3) == 0);
}

// Splits four values into TF32 hi and lo and stores them as one 16-byte
// group of the hi and lo chunks.
__device__ __forceinline__ void tc_put4(unsigned char* hi, unsigned char* lo, uint32_t off, float4 v) {
  float4 h, l;
  h.x = tf32_rn(v.x); l.x = tf32_rn(v.x - h.x);
  h.y = tf32_rn(v.y); l.y = tf32_rn(v.y - h.y);
  h.z = tf32_rn(v.z); l.z = tf32_rn(v.z - h.z);
  h.w = tf32_rn(v.w); l.w = tf32_rn(v.w - h.w);
  *reinterpret_cast<float4*>(hi + off) = h;
  *reinterpret_cast<float4*>(lo + off) = l;
}

// Stages rows [r0, r0 + nrows) (nrows a multiple of 16) and K values
// [k0, k0 + kc) (kc a multiple of 8) of operand o as TF32 pairs. Each warp
// takes blocks of 8 rows x 4 groups of four k (k-adjacent operands: a lane
// loads one row's four k) or 32 rows x 4 groups (row-adjacent operands: a
// lane loads four rows at each of four k and transposes them in registers).
__device__ __forceinline__ void tc_stage(const TcOperand& o, int r0, int nrows, int k0, int kc, unsigned char* hi,
                                         unsigned char* lo) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nk4 = kc >> 2, kg = (nk4 + 3) >> 2;
  const bool vec = tc_vec(o);
  if (!o.rfast) {
    const int nblk = (nrows >> 3) * kg;
    for (int b = warp; b < nblk; b += nw) {
      const int r = (b / kg) * 8 + (lane & 7);
      const int k4 = (b % kg) * 4 + (lane >> 3);
      if (k4 >= nk4) continue;
      const int gr = r0 + r, gk = k0 + 4 * k4;
      float4 v;
      if (vec && gr < o.rows && gk + 3 < o.cols) {
        v = *reinterpret_cast<const float4*>(o.p + (long long)gr * o.rs + gk);
        v.x = fmaf(v.x, o.sc, o.off); v.y = fmaf(v.y, o.sc, o.off);
        v.z = fmaf(v.z, o.sc, o.off); v.w = fmaf(v.w, o.sc, o.off);
      } else {
        v = make_float4(tc_elem(o, gr, gk), tc_elem(o, gr, gk + 1), tc_elem(o, gr, gk + 2), tc_elem(o, gr, gk + 3));
      }
      tc_put4(hi, lo, kmaj_off4(r, k4), v);
    }
  } else {
    const int nblk = ((nrows + 31) >> 5) * kg;
    for (int b = warp; b < nblk; b += nw) {
      const int r = (b / kg) * 32 + (lane & 7) * 4;
      const int k4 = (b % kg) * 4 + (lane >> 3);
      if (k4 >= nk4 || r >= nrows) continue;
      const int gr = r0 + r, gk = k0 + 4 * k4;
      float4 c[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (vec && gr + 3 < o.rows && gk + q < o.cols) {
          c[q] = *reinterpret_cast<const float4*>(o.p + gr + (long long)(gk + q) * o.ks);
          c[q].x = fmaf(c[q].x, o.sc, o.off); c[q].y = fmaf(c[q].y, o.sc, o.off);
          c[q].z = fmaf(c[q].z, o.sc, o.off); c[q].w = fmaf(c[q].w, o.sc, o.off);
        } else {
          c[q] = make_float4(tc_elem(o, gr, gk + q), tc_elem(o, gr + 1, gk + q), tc_elem(o, gr + 2, gk + q),
                             tc_elem(o, gr + 3, gk + q));
        }
      }
      tc_put4(hi, lo, kmaj_off4(r, k4), make_float4(c[0].x, c[1].x, c[2].x, c[3].x));
      tc_put4(hi, lo, kmaj_off4(r + 1, k4), make_float4(c[0].y, c[1].y, c[2].y, c[3].y));
      tc_put4(hi, lo, kmaj_off4(r + 2, k4), make_float4(c[0].z, c[1].z, c[2].z, c[3].z));
      tc_put4(hi, lo, kmaj_off4(r + 3, k4), make_float4(c[0].w, c[1].w, c[2].w, c[3].w));
    }
  }
}

// A constant operand's rows [r0, r0 + nrows) (r0 a multiple of 8, nrows of
// 16) of the chunk at k0, copied from its image by the copy engine: two
// contiguous runs of (nrows / 8) groups, the hi and the lo half, completing
// on mbar. Issued by one thread; the image holds a whole 128-row tile past
// any r0 and its offsets are multiples of 16 bytes.
__device__ __forceinline__ void tc_image_async(const TcOperand& o, int r0, int nrows, int k0, unsigned char* hi,
                                               unsigned char* lo, uint32_t mbar) {
  const size_t half = (size_t)o.img_groups * kTcSbo;
  const unsigned char* src = o.img + (size_t)(k0 / kTcKc) * 2 * half + (size_t)(r0 >> 3) * kTcSbo;
  const uint32_t bytes = (uint32_t)(nrows >> 3) * kTcSbo;
  bulk_g2s(smem_u32(hi), src, bytes, mbar);
  bulk_g2s(smem_u32(lo), src + half, bytes, mbar);
}

// Bytes of one staging buffer for an accumulator of width N: the hi and lo
// chunks of A (128 rows) and of B (N rows).
__host__ __device__ constexpr size_t tc_buffer_bytes(int N) { return 2 * (size_t)((kTcM + N) / 8) * kTcSbo; }
// Bytes of shared memory tc_gemm uses: two buffers.
__host__ __device__ constexpr size_t tc_smem_bytes(int N) { return 2 * tc_buffer_bytes(N); }

// One accumulator tile: D[r][n] = sum_k A(a_r0 + r, k) B(b_r0 + n, k) for
// r < 128, n < N (N a multiple of 16, at most kTcCols) and k < K. K goes in
// chunks of kTcKc through two staging buffers, so that chunk c + 1 is staged
// while the tensor cores multiply chunk c; sm holds tc_smem_bytes(N) bytes.
// The result stays in TMEM columns [0, N). Returns false (error flag set)
// if a wait ran out; the block then leaves together.
__device__ inline bool tc_gemm(TcState& tc, int N, int K, const TcOperand& a, int a_r0, const TcOperand& b, int b_r0,
                               float* sm, DevStatus* st) {
  unsigned char* base = reinterpret_cast<unsigned char*>(sm);
  const uint32_t a_bytes = (uint32_t)(kTcM / 8) * kTcSbo, b_bytes = (uint32_t)(N / 8) * kTcSbo;
  const uint32_t buf_bytes = 2 * (a_bytes + b_bytes);
  const uint32_t idesc = idesc_tf32(kTcM, N);
  const int nchunks = (K + kTcKc - 1) / kTcKc;
  auto wait_buffer = [&](int q) {   // (selects, not indexing: TcState stays in registers)
    const bool done = mbar_wait(q ? tc.mbar[1] : tc.mbar[0], q ? tc.phase[1] : tc.phase[0]);
    if (q) tc.phase[1] ^= 1u; else tc.phase[0] ^= 1u;
    if (!done) atomicExch(&st->err, kErrBarrier);
    return !__syncthreads_or(!done);
  };
  for (int c = 0; c < nchunks; ++c) {
    const int q = c & 1;
    if (c >= 2 && !wait_buffer(q)) return false;   // buffer q was last read by chunk c - 2
    unsigned char* Ahi = base + q * buf_bytes;
    unsigned char* Alo = Ahi + a_bytes;
    unsigned char* Bhi = Alo + a_bytes;
    unsigned char* Blo = Bhi + b_bytes;
    const int k0 = c * kTcKc;
    const int kc = (K - k0 < kTcKc) ? ((K - k0 + 7) & ~7) : kTcKc;   // the last chunk, padded to a K step
    // constant operands by the copy engine (in flight while the threads stage
    // the data operand), data operands by the threads
    const uint32_t tx = (a.img ? 2 * a_bytes : 0u) + (b.img ? 2 * b_bytes : 0u);
    const uint32_t cb = q ? tc.cbar[1] : tc.cbar[0];
    if (tx && threadIdx.x == 0) {
      fence_async_smem();   // this buffer's earlier generic-proxy writes before the copy's
      mbar_expect_tx(cb, tx);
      if (a.img) tc_image_async(a, a_r0, kTcM, k0, Ahi, Alo, cb);
      if (b.img) tc_image_async(b, b_r0, N, k0, Bhi, Blo, cb);
    }
    if (!a.img) tc_stage(a, a_r0, kTcM, k0, kc, Ahi, Alo);
    if (!b.img) tc_stage(b, b_r0, N, k0, kc, Bhi, Blo);
    bool copied = true;
    if (tx) {
      const uint32_t par = q ? tc.cphase[1] : tc.cphase[0];
      copied = mbar_wait(cb, par);
      if (!copied) mbar_wait(cb, par);   // gave up: a second bounded wait for the copies in flight
      if (q) tc.cphase[1] ^= 1u; else tc.cphase[0] ^= 1u;
    }
    fence_async_smem();
    if (__syncthreads_or(!copied)) {
      if (threadIdx.x == 0) atomicExch(&st->err, kErrBarrier);
      // the MMAs already issued complete on their barriers: bounded waits before leaving
      for (int p = c >= 1 ? c - 1 : 0; p < c; ++p) wait_buffer(p & 1);
      return false;
    }
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
      for (int s = 0; s < kc / 8; ++s) {
        const uint32_t off = (uint32_t)s * 256;   // two core matrices of 128 bytes per K step
        const uint64_t dah = kmaj_desc(ah + off), dal = kmaj_desc(al + off);
        const uint64_t dbh = kmaj_desc(bh + off), dbl = kmaj_desc(bl + off);
        umma_tf32(tc.tmem, dah, dbh, idesc, (c > 0 || s > 0) ? 1u : 0u);
        umma_tf32(tc.tmem, dah, dbl, idesc, 1u);
        umma_tf32(tc.tmem, dal, dbh, idesc, 1u);
      }
      umma_commit(q ? tc.mbar[1] : tc.mbar[0]);
    }
  }
  // the chunks not waited for yet: the accumulator is read next, and the
  // next tile restages both buffers
  for (int c = nchunks >= 2 ? nchunks - 2 : 0; c < nchunks; ++c)
    if (!wait_buffer(c & 1)) return false;
  tc_fence_after();
  return true;
}

// Hands the accumulator's columns [0, N) to st(r, n, v), 16 columns per
// TMEM load: warp w reads the lanes of quadrant w % 4 and the 16-column
// groups g = w / 4, w / 4 + nw / 4, ... (nw warps in the block). Then
// orders the reads before the next tile's MMAs.
template <class ST>
__device__ __forceinline__ void tc_store(const TcState& tc, int N, ST st) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = w & 3, nw = blockDim.x >> 5;
  const int r = q * 32 + lane;
  for (int c = (w >> 2) * 16; c < N; c += (nw >> 2) * 16) {
    float v[16];
    tmem_ld16(tc.tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
#pragma unroll
    for (int j = 0; j < 16; ++j) st(r, c + j, v[j]);
  }
  tc_fence_before();
  __syncthreads();
}

}  // namespace solid
