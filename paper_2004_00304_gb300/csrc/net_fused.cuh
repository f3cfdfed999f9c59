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
// padded to N = 16) subtracts its own mean over each patch column (16 rows)
// per field and adds the mean of the 8 input frames.  The kernel that runs
// these layers inside the coupled step is closure_step (closure_coupling.cu).
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include "kernels.h"
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

using Meta = NetMeta;   // parameter offsets of each layer's weights and biases

// byte offset of (row j in [-16, 272), channel group c) in a copy with KC groups
__device__ __forceinline__ uint32_t cp_off(int j, int c, int KC) {
  const int jj = j + 16;
  return (uint32_t)((((jj >> 3) * KC + c) << 7) + ((jj & 7) << 4));
}

// one 16-byte channel group of pixel p into the three shifted copies, which
// sit at cp + (dx + 1) COPY_BYTES
__device__ __forceinline__ void put3(unsigned char* cp, int p, int c, int KC, uint4 v) {
  *reinterpret_cast<uint4*>(cp + COPY_BYTES + cp_off(p, c, KC)) = v;                              // dx = 0
  if ((p & 15) >= 1) *reinterpret_cast<uint4*>(cp + 2 * COPY_BYTES + cp_off(p - 1, c, KC)) = v;   // dx = +1
  if ((p & 15) <= 14) *reinterpret_cast<uint4*>(cp + cp_off(p + 1, c, KC)) = v;                   // dx = -1
}

// weight image of one layer -> shared memory by one bulk (TMA) copy that
// completes on mbarrier wb; issued by one thread
__device__ __forceinline__ void bulk_weights(unsigned char* wsm, const __nv_bfloat16* src, uint32_t bytes,
                                             uint64_t* wb) {
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(wb);
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(b),
               "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(wsm)),
               "l"(src), "r"(bytes), "r"(b)
               : "memory");
}

// Clear the positions of the three copies that no write of a layer input
// covers, for a layout of KC channel groups: the 16 halo rows above and below
// (all copies), the rows whose x + dx leaves the patch (x = 15 in the dx = +1
// copy, x = 0 in the dx = -1 copy).  Every other position is written.
__device__ __forceinline__ void zero_unwritten(unsigned char* cp, int KC) {
  const uint4 z = make_uint4(0, 0, 0, 0);
  const int halo = 2 * KC * 8;   // 16-byte units in the 16 halo rows of one side
  for (int i = threadIdx.x; i < 3 * 2 * halo; i += blockDim.x) {
    const int k = i / (2 * halo), r = i % (2 * halo);
    const int off = r < halo ? r : (34 * KC * 8) + (r - halo);   // groups 0-1 and 34-35
    reinterpret_cast<uint4*>(cp + k * COPY_BYTES)[off] = z;
  }
  for (int i = threadIdx.x; i < 2 * 16 * KC; i += blockDim.x) {
    const int side = i / (16 * KC), r = (i / KC) % 16, c = i % KC;
    const int j = 16 * r + (side ? 15 : 0);   // dx = +1 copy: x = 15; dx = -1 copy: x = 0
    *reinterpret_cast<uint4*>(cp + (side ? 2 : 0) * COPY_BYTES + cp_off(j, c, KC)) = z;
  }
}

__device__ __forceinline__ uint32_t pack2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

}  // namespace fz


namespace fz {

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// All MMAs of one layer: tile t (rows 128 t .. 128 t + 127) accumulates in
// TMEM columns 64 t.., over 9 taps x KC/2 K-steps of 16.  dA / dB are the
// descriptors of the first copy / the weight image; a descriptor's start
// field is the byte address / 16, so an offset is added as offset / 16.
template <int KC, int N>
__device__ __forceinline__ void issue_layer(uint32_t tmem, uint64_t dA, uint64_t dB) {
  constexpr uint32_t idesc = tc::instr_desc(128, N);
#pragma unroll
  for (int t = 0; t < 2; ++t) {
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int dy = tap / 3 - 1, dx = tap % 3 - 1;
      const uint32_t a_off = (uint32_t)((dx + 1) * COPY_BYTES + ((16 + 128 * t + 16 * dy) >> 3) * KC * 128);
#pragma unroll
      for (int s = 0; s < KC / 2; ++s)
        mma_f16(tmem + 64u * t, dA + ((a_off + 256u * s) >> 4), dB + ((uint32_t)(tap * KC * 128 + 256 * s) >> 4),
                idesc, (tap | s) ? 1u : 0u);
    }
  }
}

// 16 consecutive fp32 accumulator columns of this warp's 32 lanes
#define FZ_TMEM_LD16(v, addr)                                                                                  \
  asm volatile(                                                                                                \
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];" \
      : "=r"((v)[0]), "=r"((v)[1]), "=r"((v)[2]), "=r"((v)[3]), "=r"((v)[4]), "=r"((v)[5]), "=r"((v)[6]),    \
        "=r"((v)[7]), "=r"((v)[8]), "=r"((v)[9]), "=r"((v)[10]), "=r"((v)[11]), "=r"((v)[12]),               \
        "=r"((v)[13]), "=r"((v)[14]), "=r"((v)[15])                                                          \
      : "r"(addr)                                                                                              \
      : "memory")

// hidden-layer epilogue of one tile: bias, ReLU, bf16 into the next layer's copies
__device__ __forceinline__ void epilogue_hidden(unsigned char* cp, uint32_t ta, int m, const float* bias) {
  uint32_t v[64];
  FZ_TMEM_LD16(v, ta);
  FZ_TMEM_LD16(v + 16, ta + 16);
  FZ_TMEM_LD16(v + 32, ta + 32);
  FZ_TMEM_LD16(v + 48, ta + 48);
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int g = 0; g < 8; ++g) {
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float s = __uint_as_float(v[8 * g + j]) + bias[8 * g + j];
      a[j] = s > 0.0f ? s : 0.0f;
    }
    put3(cp, m, g, 8, make_uint4(pack2(a[0], a[1]), pack2(a[2], a[3]), pack2(a[4], a[5]), pack2(a[6], a[7])));
  }
}

}  // namespace fz

}  // namespace lbm
