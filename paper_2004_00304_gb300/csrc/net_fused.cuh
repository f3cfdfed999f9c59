// net_fused.cuh -- the closure network's forward pass fused into one kernel
// for in-loop inference: one CTA of 128 threads per 16 x 16 patch, every
// activation resident in shared memory, every contraction a tcgen05.mma.
//
// Each layer is a 3 x 3 convolution = 9 taps.  The patch's 256 pixels are the
// two 128-row M tiles (row m = 16 y + x).  A tap (dy, dx) reads pixel
// m + 16 dy + dx, so the layer input is kept three times, pre-shifted by
// dx = -1, 0, +1 (zero where x + dx leaves the patch), each with a zero halo
// of 16 rows above and below: then every tap's A operand is one of the
// copies at a row offset 16 dy, a multiple of the 8-row core-matrix height,
// and the MMAs read it in place (no im2col).  Copies use the canonical
// no-swizzle K-major layout (core matrix = 8 rows x 16 bytes; K-adjacent core
// matrices 128 bytes apart, 8-row groups KC * 128 bytes apart).  Layer 0 has
// 24 input channels, padded to 32.  Weights are staged per layer from an image
// already in the same layout ([n][tap][channel], zero padded), the two M tiles
// accumulate in TMEM columns 0..63 and 64..127, and the epilogue (bias, ReLU,
// bf16) writes the next layer's three copies; the last layer (3 outputs,
// padded to N = 16) adds the mean of the 8 input frames and writes y.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include "tc_gemm.cuh"

namespace lbm {
namespace fz {

constexpr int ROWS = 288;                        // pixel rows -16 .. 271
constexpr int COPY_BYTES = ROWS * 64 * 2;        // one copy at 64 channels
constexpr int W_BYTES = 64 * 576 * 2;            // largest weight image
constexpr int SMEM = 3 * COPY_BYTES + W_BYTES;   // 184320 bytes of dynamic shared memory

__host__ __device__ constexpr int cinp(int l) { return l == 0 ? 32 : 64; }   // padded input channels
__host__ __device__ constexpr int cinr(int l) { return l == 0 ? 24 : 64; }   // real input channels
__host__ __device__ constexpr int nout(int l) { return l == 3 ? 16 : 64; }   // padded outputs (MMA N)
__host__ __device__ constexpr int coutr(int l) { return l == 3 ? 3 : 64; }   // real outputs
__host__ __device__ constexpr long long img_bytes(int l) { return (long long)nout(l) * 9 * cinp(l) * 2; }
__host__ __device__ constexpr long long img_off(int l) {
  return l == 0 ? 0 : img_off(l - 1) + img_bytes(l - 1);
}
constexpr long long IMG_TOTAL = img_off(4);

struct Meta { long long woff[4], boff[4]; };

// byte offset of (row j in [-16, 272), channel group c) in a copy with KC groups
__device__ __forceinline__ uint32_t cp_off(int j, int c, int KC) {
  const int jj = j + 16;
  return (uint32_t)((((jj >> 3) * KC + c) << 7) + ((jj & 7) << 4));
}

// one 16-byte channel group of pixel p into the three shifted copies
__device__ __forceinline__ void put3(unsigned char* const* cp, int p, int c, int KC, uint4 v) {
  *reinterpret_cast<uint4*>(cp[1] + cp_off(p, c, KC)) = v;                            // dx = 0
  if ((p & 15) >= 1) *reinterpret_cast<uint4*>(cp[2] + cp_off(p - 1, c, KC)) = v;     // dx = +1
  if ((p & 15) <= 14) *reinterpret_cast<uint4*>(cp[0] + cp_off(p + 1, c, KC)) = v;    // dx = -1
}

__device__ __forceinline__ uint32_t pack2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

}  // namespace fz

// weight images of the four layers, bf16, core-matrix layout:
// element (n, k) of layer l at ((n/8 * KB + k/8) * 8 + n%8) * 8 + k%8,
// KB = 9 cinp / 8, k = tap * cinp + channel
__global__ void k_pack_fused(const float* __restrict__ theta, fz::Meta meta, __nv_bfloat16* __restrict__ img) {
  using namespace fz;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= IMG_TOTAL / 2) return;
  int l = 0;
  while (l < 3 && i >= img_off(l + 1) / 2) ++l;
  const long long e = i - img_off(l) / 2;
  const int KB = 9 * cinp(l) / 8;
  const int q = (int)(e & 7), r = (int)((e >> 3) & 7);
  const long long rest = e >> 6;
  const int c = (int)(rest % KB), g = (int)(rest / KB);
  const int n = 8 * g + r, k = 8 * c + q;
  const int tap = k / cinp(l), ci = k % cinp(l);
  float v = 0.0f;
  if (n < coutr(l) && ci < cinr(l)) v = theta[meta.woff[l] + ((long long)n * 9 + tap) * cinr(l) + ci];
  img[i] = __float2bfloat16_rn(v);
}

// y[P][256][3] = network(x[P][256][24]); grid = P, 128 threads, fz::SMEM bytes
// of dynamic shared memory.  Every mbarrier wait is bounded; a timeout sets
// *err, and the CTA releases its TMEM and returns.
__global__ void __launch_bounds__(128, 1) net_fused_fwd(const float* __restrict__ x,
                                                        const __nv_bfloat16* __restrict__ img,
                                                        const float* __restrict__ theta, fz::Meta meta,
                                                        float* __restrict__ y, int* err) {
  using namespace fz;
  using namespace tc;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  unsigned char* cp[3] = {sm, sm + COPY_BYTES, sm + 2 * COPY_BYTES};   // dx = -1, 0, +1
  unsigned char* wsm = sm + 3 * COPY_BYTES;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float* xp = x + (long long)blockIdx.x * 256 * 24;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(&tmem_base)),
                 "r"(128u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  const uint4 z4 = make_uint4(0, 0, 0, 0);
  for (int i = tid; i < 3 * COPY_BYTES / 16; i += 128) reinterpret_cast<uint4*>(sm)[i] = z4;
  __syncthreads();
  // layer-0 input: 24 fp32 channels -> bf16, padded to 32 (4 groups of 8)
  for (int it = tid; it < 256 * 4; it += 128) {
    const int p = it >> 2, c = it & 3;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = (c < 3) ? xp[p * 24 + 8 * c + e] : 0.0f;
    put3(cp, p, c, 4, make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7])));
  }
  for (int i = tid; i < (int)(img_bytes(0) / 16); i += 128)
    reinterpret_cast<uint4*>(wsm)[i] = reinterpret_cast<const uint4*>(img)[i];
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  for (int l = 0; l < 4 && !s_fail; ++l) {
    const int KC = cinp(l) / 8, N = nout(l);
    const uint32_t sbo_a = (uint32_t)KC * 128u, sbo_b = (uint32_t)(9 * KC) * 128u;
    if (tid == 0) {
      const uint32_t idesc = instr_desc(128, N);
      for (int t = 0; t < 2; ++t) {
        uint32_t acc = 0;
        for (int tap = 0; tap < 9; ++tap) {
          const int dy = tap / 3 - 1, dx = tap % 3 - 1;
          const uint32_t a0 = s_addr(cp[dx + 1]) + (uint32_t)((16 + 128 * t + 16 * dy) >> 3) * sbo_a;
          const uint32_t b0 = s_addr(wsm) + (uint32_t)(tap * KC) * 128u;
          for (int s = 0; s < KC / 2; ++s) {
            const uint64_t ad = smem_desc(a0 + s * 256, 128, sbo_a);
            const uint64_t bd = smem_desc(b0 + s * 256, 128, sbo_b);
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + 64u * t),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                : "memory");
            acc = 1;
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       s_addr(&mbar))
                   : "memory");
    }
    const bool ok = mbar_wait(&mbar, (uint32_t)(l & 1));
    if (__syncthreads_or(!ok)) {
      if (tid == 0) { atomicExch(err, 1); s_fail = 1; }
      __syncthreads();
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (l == 0) {   // the hidden layers use 8 channel groups: clear the 4-group layout first
      for (int i = tid; i < 3 * COPY_BYTES / 16; i += 128) reinterpret_cast<uint4*>(sm)[i] = z4;
      __syncthreads();
    }
    const float* bias = theta + meta.boff[l];
#pragma unroll 1
    for (int t = 0; t < 2; ++t) {
      const int m = 128 * t + 32 * warp + lane;
#pragma unroll 1
      for (int c0 = 0; c0 < N; c0 += 16) {
        uint32_t v[16];
        const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + 64u * t + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(ta)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (l < 3) {
          float a[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float s = __uint_as_float(v[j]) + bias[c0 + j];
            a[j] = s > 0.0f ? s : 0.0f;
          }
          put3(cp, m, c0 / 8, 8, make_uint4(pack2(a[0], a[1]), pack2(a[2], a[3]), pack2(a[4], a[5]), pack2(a[6], a[7])));
          put3(cp, m, c0 / 8 + 1, 8,
               make_uint4(pack2(a[8], a[9]), pack2(a[10], a[11]), pack2(a[12], a[13]), pack2(a[14], a[15])));
        } else {
          float* yr = y + ((long long)blockIdx.x * 256 + m) * 3;
          const float* xr = xp + (long long)m * 24;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            float s = 0.0f;
#pragma unroll
            for (int f = 0; f < 8; ++f) s += xr[3 * f + c];
            yr[c] = (__uint_as_float(v[c]) + bias[c]) + 0.125f * s;
          }
        }
      }
    }
    if (l < 3) {   // this layer's MMAs are complete: stage the next layer's weights
      const uint4* src = reinterpret_cast<const uint4*>(img + img_off(l + 1) / 2);
      for (int i = tid; i < (int)(img_bytes(l + 1) / 16); i += 128) reinterpret_cast<uint4*>(wsm)[i] = src[i];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128u) : "memory");
  }
}

}  // namespace lbm
