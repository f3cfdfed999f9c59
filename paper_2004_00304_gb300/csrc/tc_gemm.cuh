// tc_gemm.cuh -- BF16 GEMM on the 5th-generation tensor cores (tcgen05):
//     C[M][N] (fp32) = A[M][K] (bf16, K contiguous) * B[N][K]^T (bf16, K contiguous)
// M a multiple of 128, N a multiple of 16 in [16, 256], K a multiple of 64.
//
// One CTA of 128 threads per 128 x N tile of C.  The K loop stages 64-wide
// slabs of A and B in shared memory in the canonical no-swizzle K-major layout
// (core matrices of 8 rows x 16 bytes), one elected thread issues four
// tcgen05.mma (M=128, N, K=16, kind::f16 with bf16 inputs) per slab with the
// accumulator in tensor memory, and tcgen05.commit signals an mbarrier when
// the slab has been consumed; two slabs are in flight.  The epilogue reads the
// accumulator with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = rows) and
// applies C = alpha * acc + beta * C.  Every mbarrier wait is bounded; a
// timeout sets the error word and the CTA returns after releasing its TMEM.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace lbm {
namespace tc {

constexpr int BM = 128, BK = 64;

__device__ __forceinline__ uint32_t s_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor, no swizzle, K-major: start address, the
// byte distance between core matrices adjacent in K (leading) and in M/N (stride)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the 5th-generation tensor cores
  return d;                // base offset 0, swizzle mode 0 (none)
}

// instruction descriptor of kind::f16: fp32 accumulator, bf16 A and B, both K-major
__host__ __device__ constexpr uint32_t instr_desc(int m, int n) {
  return (1u << 4)                    // D: f32
         | (1u << 7)                  // A: bf16
         | (1u << 10)                 // B: bf16
         | ((uint32_t)(n >> 3) << 17) // N / 8
         | ((uint32_t)(m >> 4) << 24);// M / 16
}

__device__ __forceinline__ void mbar_init(uint64_t* m, uint32_t c) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_addr(m)), "r"(c) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t* m, uint32_t parity) {
  const uint32_t a = s_addr(m);
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

}  // namespace tc

// C = alpha * A B^T + beta * C, fp32 C with leading dimension ldc.
// Tiles: blockIdx.x over N / bn, blockIdx.y over M / 128.
template <int BN>
__global__ void __launch_bounds__(128) tc_gemm_bf16(const __nv_bfloat16* __restrict__ A,
                                                    const __nv_bfloat16* __restrict__ B, float* __restrict__ C,
                                                    int M, int N, int K, int ldc, float alpha, float beta,
                                                    int* err) {
  using namespace tc;
  constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
  constexpr int STAGE = A_BYTES + B_BYTES;
  constexpr uint32_t TCOLS = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
  // two stages plus a full spare stage of slack after them
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(&tmem_base)),
                 "r"(TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = instr_desc(BM, BN);

  const int nk = K / BK;
  for (int kb = 0; kb < nk; ++kb) {
    const int s = kb & 1;
    unsigned char* sa = sm + s * STAGE;
    unsigned char* sb = sa + A_BYTES;
    if (kb >= 2) {   // the MMAs that read this stage two slabs ago must be done
      const bool ok = mbar_wait(&mbar[s], ((kb - 2) >> 1) & 1);
      if (__syncthreads_or(!ok)) { if (tid == 0) atomicExch(err, 1); s_fail = 1; break; }
    }
    // stage A (128 x 64) and B (BN x 64): core matrix (row group g, k group c)
    // at byte (g * 8 + c) * 128, its 8 rows of 16 bytes contiguous
    for (int idx = tid; idx < (BM + BN) * (BK / 8); idx += blockDim.x) {
      const int row = idx / (BK / 8), c = idx % (BK / 8);
      const bool isA = row < BM;
      const int r = isA ? row : row - BM;
      const __nv_bfloat16* src = isA ? A + (size_t)(m0 + r) * K + kb * BK + c * 8
                                     : B + (size_t)(n0 + r) * K + kb * BK + c * 8;
      const uint4 v = *reinterpret_cast<const uint4*>(src);
      unsigned char* dst = (isA ? sa : sb) + ((r >> 3) * (BK / 8) + c) * 128 + (r & 7) * 16;
      *reinterpret_cast<uint4*>(dst) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        // K = 16 = two core matrices: advance the start by two along K
        const uint64_t ad = smem_desc(s_addr(sa) + kk * 256, 128, (BK / 8) * 128);
        const uint64_t bd = smem_desc(s_addr(sb) + kk * 256, 128, (BK / 8) * 128);
        const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       s_addr(&mbar[s]))
                   : "memory");
    }
  }
  if (!s_fail && nk > 0) {
    // the last slab's commit also covers every earlier MMA
    const int s = (nk - 1) & 1;
    const bool ok = mbar_wait(&mbar[s], ((nk - 1) >> 1) & 1);
    if (__syncthreads_or(!ok)) { if (tid == 0) atomicExch(err, 1); s_fail = 1; }
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!s_fail) {
    const int row = m0 + warp * 32 + lane;
#pragma unroll
    for (int c0 = 0; c0 < BN; c0 += 16) {
      uint32_t v[16];
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(ta)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < M) {
        float* cr = C + (size_t)row * ldc + n0 + c0;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float a = __uint_as_float(v[j]);
          cr[j] = beta == 0.0f ? alpha * a : alpha * a + beta * cr[j];
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
  }
}

// dynamic shared memory of a launch: two stages plus one stage of slack
template <int BN>
constexpr int tc_gemm_smem() {
  return 3 * (tc::BM * tc::BK * 2 + BN * tc::BK * 2);
}

}  // namespace lbm
