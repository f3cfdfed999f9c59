// closure.cu -- the learned MPCD->LB closure: a 4-layer 3x3 convolutional
// network (24 -> 64 -> 64 -> 64 -> 3 channels on 16 x 16 patches of MPCD
// cells) with bf16 weights and activations and fp32 accumulation.  Every
// contraction (forward, backward-data, backward-weights) is an implicit-GEMM
// on the tcgen05 tensor cores (tc_gemm.cuh).
#include <cuda_bf16.h>

#include "../../include/lbmpcd.h"
#include "kernels.h"
#include "tc_gemm.cuh"

namespace lbm {

template <int BN>
static cudaError_t gemm_bn(const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, int M, int N, int K, int ldc,
                           float alpha, float beta, int* err, cudaStream_t st) {
  static const cudaError_t attr =
      cudaFuncSetAttribute(tc_gemm_bf16<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_gemm_smem<BN>());
  if (attr != cudaSuccess) return attr;
  dim3 grid(N / BN, M / tc::BM);
  tc_gemm_bf16<BN><<<grid, 128, tc_gemm_smem<BN>(), st>>>(A, B, C, M, N, K, ldc, alpha, beta, err);
  return cudaGetLastError();
}

// C (M x N, fp32, row stride ldc) = alpha A B^T + beta C; picks the widest N tile.
cudaError_t tc_gemm(const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, int M, int N, int K, int ldc,
                    float alpha, float beta, int* err, cudaStream_t st) {
  if (N % 256 == 0) return gemm_bn<256>(A, B, C, M, N, K, ldc, alpha, beta, err, st);
  if (N % 128 == 0) return gemm_bn<128>(A, B, C, M, N, K, ldc, alpha, beta, err, st);
  if (N % 64 == 0) return gemm_bn<64>(A, B, C, M, N, K, ldc, alpha, beta, err, st);
  if (N % 32 == 0) return gemm_bn<32>(A, B, C, M, N, K, ldc, alpha, beta, err, st);
  return gemm_bn<16>(A, B, C, M, N, K, ldc, alpha, beta, err, st);
}

}  // namespace lbm

using namespace lbm;

extern "C" int lbmpcd_tc_gemm_bf16(const void* A, const void* B, float* C, int M, int N, int K, float alpha,
                                   float beta, int* err_dev, void* stream) {
  if (!A || !B || !C || !err_dev || M <= 0 || N <= 0 || K <= 0) return LBMPCD_ERR_INVALID_ARG;
  if (M % 128 || N % 16 || N > 4096 || K % 64) return LBMPCD_ERR_INVALID_ARG;
  const cudaError_t e = tc_gemm((const __nv_bfloat16*)A, (const __nv_bfloat16*)B, C, M, N, K, N, alpha, beta,
                                err_dev, (cudaStream_t)stream);
  return e == cudaSuccess ? LBMPCD_OK : LBMPCD_ERR_CUDA;
}
