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
// (4 FP32), the two core matrices of one K step of 8 next to each other
// (leading byte offset 128), 8-row groups Kc/4 * 128 bytes apart (stride
// byte offset) for a chunk of Kc values of K.
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

// byte offset of element (r, k) of a K-major operand chunk of Kc columns
// (Kc a multiple of 8) in the canonical no-swizzle layout
__device__ __forceinline__ uint32_t kmaj_off(int r, int k, int Kc) {
  return (uint32_t)((r >> 3) * (Kc * 32) + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

// shared-memory matrix descriptor of a K-major chunk starting at saddr
// (16-byte aligned): no swizzle, leading byte offset 128, stride byte
// offset 32 Kc, descriptor version 1
__device__ __forceinline__ uint64_t kmaj_desc(uint32_t saddr, int Kc) {
  const uint64_t lbo = 128, sbo = 32ull * (uint64_t)Kc;
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

// The block's tensor-core state: its TMEM columns and the mbarrier the MMAs
// complete on. Set up by tc_open (all threads) at the start of a kernel and
// released by tc_close (all threads) at its end.
struct TcState {
  uint32_t tmem;      // TMEM address of column 0, lane 0
  uint32_t mbar;      // shared address of the mbarrier
  uint32_t phase;     // parity of the next phase to wait for
};

__device__ __forceinline__ void tc_open(TcState& tc, uint32_t* s_tmem, unsigned long long* s_mbar) {
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                 "r"((uint32_t)kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 32) mbar_init(smem_u32(s_mbar), 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  tc.tmem = *s_tmem;
  tc.mbar = smem_u32(s_mbar);
  tc.phase = 0;
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

// One accumulator tile: D[r][n] = sum_k A(r, k) B(n, k), r < 128, n < N
// (N a multiple of 16, at most kTcCols), k < K. la(r, k) and lb(n, k) load
// one FP32 operand value (0 outside the operand); a_rfast / b_rfast say
// whether consecutive rows (else consecutive k) are adjacent in memory, and
// the staging threads walk that index fastest. K is taken in chunks of Kc
// (a multiple of 8); sm holds 2 (128 + N) Kc floats. The result stays in
// TMEM columns [0, N). Returns false if a wait ran out (error flag set).
template <class LA, class LB>
__device__ bool tc_gemm(TcState& tc, int N, int K, int Kc, LA la, bool a_rfast, LB lb, bool b_rfast, float* sm,
                        DevStatus* st) {
  unsigned char* base = reinterpret_cast<unsigned char*>(sm);
  const uint32_t a_bytes = (uint32_t)kTcM * Kc * 4, b_bytes = (uint32_t)N * Kc * 4;
  unsigned char* Ahi = base;
  unsigned char* Alo = Ahi + a_bytes;
  unsigned char* Bhi = Alo + a_bytes;
  unsigned char* Blo = Bhi + b_bytes;
  const uint32_t idesc = idesc_tf32(kTcM, N);
  bool ok = true;
  for (int k0 = 0; k0 < K; k0 += Kc) {
    const int kc = (K - k0 < Kc) ? ((K - k0 + 7) & ~7) : Kc;   // the last chunk, padded to a K step
    const int na = kTcM * kc, nb = N * kc;
    for (int e = threadIdx.x; e < na; e += blockDim.x) {
      const int r = a_rfast ? e % kTcM : e / kc;
      const int k = a_rfast ? e / kTcM : e % kc;
      const float v = la(r, k0 + k);
      const float hi = tf32_rn(v);
      const uint32_t o = kmaj_off(r, k, Kc);
      *reinterpret_cast<float*>(Ahi + o) = hi;
      *reinterpret_cast<float*>(Alo + o) = tf32_rn(v - hi);
    }
    for (int e = threadIdx.x; e < nb; e += blockDim.x) {
      const int n = b_rfast ? e % N : e / kc;
      const int k = b_rfast ? e / N : e % kc;
      const float v = lb(n, k0 + k);
      const float hi = tf32_rn(v);
      const uint32_t o = kmaj_off(n, k, Kc);
      *reinterpret_cast<float*>(Bhi + o) = hi;
      *reinterpret_cast<float*>(Blo + o) = tf32_rn(v - hi);
    }
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
      for (int s = 0; s < kc / 8; ++s) {
        const uint32_t off = (uint32_t)s * 256;   // two core matrices of 128 bytes per K step
        const uint64_t dah = kmaj_desc(ah + off, Kc), dal = kmaj_desc(al + off, Kc);
        const uint64_t dbh = kmaj_desc(bh + off, Kc), dbl = kmaj_desc(bl + off, Kc);
        umma_tf32(tc.tmem, dah, dbh, idesc, (k0 > 0 || s > 0) ? 1u : 0u);
        umma_tf32(tc.tmem, dah, dbl, idesc, 1u);
        umma_tf32(tc.tmem, dal, dbh, idesc, 1u);
      }
      umma_commit(tc.mbar);
    }
    // every thread waits: the chunk's shared memory is reused by the next
    // chunk, and the accumulator is read after the last one
    const bool done = mbar_wait(tc.mbar, tc.phase);
    if (!done) atomicExch(&st->err, kErrBarrier);
    tc.phase ^= 1u;
    tc_fence_after();
    if (__syncthreads_or(!done)) {   // the block leaves together
      ok = false;
      break;
    }
  }
  return ok;
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
