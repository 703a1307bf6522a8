// Self-test of the tensor-core GEMM tile (umma.cuh): one block forms
// D = A B^T for A of 128 x k and B of n x k (FP32, row-major, device
// memory) by three TF32 products per K step, and writes D (128 x n).
#include "umma.cuh"

namespace solid {
namespace {

constexpr int kSelftestKc = 32;

__global__ void __launch_bounds__(kBlock, 1) k_tc_selftest(const float* __restrict__ a, const float* __restrict__ b,
                                                           float* __restrict__ d, int n, int k, DevStatus* st) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) unsigned long long s_mbar;
  TcState tc;
  tc_open(tc, &s_tmem, &s_mbar);
  const bool ok = tc_gemm(
      tc, n, k, kSelftestKc, [&](int r, int kk) { return kk < k ? a[(size_t)r * k + kk] : 0.f; }, false,
      [&](int c, int kk) { return kk < k ? b[(size_t)c * k + kk] : 0.f; }, false, reinterpret_cast<float*>(dsm),
      st);
  if (ok) tc_store(tc, n, [&](int r, int c, float v) { d[(size_t)r * n + c] = v; });
  tc_close(tc);
}

}  // namespace

size_t tc_selftest_smem(int n) { return 2 * (size_t)(kTcM + n) * kSelftestKc * sizeof(float); }

cudaError_t launch_tc_selftest(const float* a, const float* b, float* d, int n, int k, DevStatus* st,
                               cudaStream_t s) {
  const size_t smem = tc_selftest_smem(n);
  cudaError_t e = cudaFuncSetAttribute(k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_tc_selftest<<<1, kBlock, smem, s>>>(a, b, d, n, k, st);
  return cudaGetLastError();
}

}  // namespace solid
