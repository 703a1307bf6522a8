// Self-test of the tensor-core GEMM tile (umma.cuh): one block forms
// D = A B^T for A of 128 x k and B of n x k (FP32 device memory; row-major,
// or both stored transposed so that the staging takes its row-adjacent path)
// by three TF32 products per K step, and writes D (128 x n, row-major).
#include "umma.cuh"

namespace solid {
namespace {

__global__ void __launch_bounds__(kBlock, 1) k_tc_selftest(const float* __restrict__ a, const float* __restrict__ b,
                                                           float* __restrict__ d, int n, int k, int transposed,
                                                           DevStatus* st) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) unsigned long long s_mbar[kTcBarriers];
  TcState tc;
  tc_open(tc, &s_tmem, s_mbar);
  const TcOperand oa = transposed ? TcOperand{a, 1, kTcM, kTcM, k, 1.f, 0.f, 1} : TcOperand{a, k, 1, kTcM, k, 1.f, 0.f, 0};
  const TcOperand ob = transposed ? TcOperand{b, 1, n, n, k, 1.f, 0.f, 1} : TcOperand{b, k, 1, n, k, 1.f, 0.f, 0};
  if (tc_gemm(tc, n, k, oa, 0, ob, 0, reinterpret_cast<float*>(dsm), st))
    tc_store(tc, n, [&](int r, int c, float v) { d[(size_t)r * n + c] = v; });
  tc_close(tc);
}

}  // namespace

cudaError_t launch_tc_selftest(const float* a, const float* b, float* d, int n, int k, int transposed,
                               DevStatus* st, cudaStream_t s) {
  const size_t smem = tc_smem_bytes(n);
  cudaError_t e = cudaFuncSetAttribute(k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_tc_selftest<<<1, kBlock, smem, s>>>(a, b, d, n, k, transposed, st);
  return cudaGetLastError();
}

}  // namespace solid
