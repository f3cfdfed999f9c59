// net_fused.cuh -- the closure network's forward pass fused into one kernel
// for in-loop inference: a cluster of two CTAs of 256 threads per 16 x 16
// patch, every activation resident in shared memory, every contraction a
// tcgen05.mma.
//
// Each layer is a 3 x 3 convolution = 9 taps.  Pixel m = 16 y + x of the
// patch; CTA h of the pair (its rank in the cluster) computes the 128 pixels
// m = 128 h + p (image rows 8 h .. 8 h + 7), one M tile whose row p is TMEM
// lane p.  A tap (dy, dx) reads pixel
// m + 16 dy + dx, so the layer input is kept three times, pre-shifted by
// dx = -1, 0, +1 (zero where x + dx leaves the patch), each with 16 halo rows
// above and below the tile (the neighbouring image row): every tap's A
// operand is then one of the copies at a row offset 16 dy, a multiple of the
// 8-row core-matrix height, read in place by the MMAs (no im2col).  The halo
// rows toward the other CTA hold its pixels: each CTA writes the image row
// next to the cut into the other's copies through distributed shared memory
// after both have finished the layer's MMAs; the halo rows at the patch edge
// stay zero.  Copies use the canonical no-swizzle K-major layout (core matrix
// = 8 rows x 16 bytes; K-adjacent core matrices 128 bytes apart, 8-row groups
// KC * 128 bytes apart).  Layer 0 has 24 input channels, padded to 32.  The
// weight images are already in the same layout ([n][tap][channel], zero
// padded) and are staged by bulk copies into two buffers, so that the copy of
// layer l + 2 runs under layers l + 1; the accumulator of a layer is TMEM
// columns 0..63, and the epilogue (bias, ReLU, bf16) writes the next layer's
// three copies.  The last layer (3 outputs, padded to N = 16) subtracts its
// own mean over each patch column (16 rows, summed over both CTAs) per field
// and adds the mean of the 8 input frames.  The kernel that runs these layers
// inside the coupled step is closure_step (closure_coupling.cu).
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include "kernels.h"
#include "tc_gemm.cuh"

namespace lbm {
namespace fz {

constexpr int HALF = 128;                        // pixels per CTA (one M tile)
constexpr int ROWS = HALF + 32;                  // local rows -16 .. 143 (16 halo rows each side)
constexpr int COPY_BYTES = ROWS * 64 * 2;        // one copy at 64 channels
constexpr int W_BYTES = 64 * 576 * 2;            // largest weight image
constexpr int SMEM = 3 * COPY_BYTES + 2 * W_BYTES;   // 208896 bytes of dynamic shared memory

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

// byte offset of (local row j in [-16, 144), channel group c) in a copy with KC groups
__device__ __forceinline__ uint32_t cp_off(int j, int c, int KC) {
  const int jj = j + 16;
  return (uint32_t)((((jj >> 3) * KC + c) << 7) + ((jj & 7) << 4));
}

// this CTA's shared address -> the same address in the other CTA of the pair
__device__ __forceinline__ uint32_t peer_addr(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cluster(uint32_t a, uint4 v) {
  asm volatile("st.shared::cluster.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w)
               : "memory");
}
__device__ __forceinline__ void st_cluster_f32(uint32_t a, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}

// Every thread of both CTAs: the writes before (to either CTA's shared
// memory, also those the tensor cores read next) are visible after.
__device__ __forceinline__ void pair_sync() {
  asm volatile("fence.proxy.async.shared::cluster;" ::: "memory");
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// one 16-byte store to this CTA's shared memory (peer < 0) or, through
// distributed shared memory, to the same address in CTA `peer` of the pair
__device__ __forceinline__ void st16(uint32_t a, uint4 v, int peer) {
  if (peer < 0)
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
  else
    st_cluster(peer_addr(a, (uint32_t)peer), v);
}

// one 16-byte channel group of local pixel row p (x = p mod 16) into the
// three shifted copies at cp + (dx + 1) COPY_BYTES, of this CTA (peer < 0)
// or of CTA `peer`; for p in [-16, 144) every store stays in rows -16 .. 143
__device__ __forceinline__ void put3(unsigned char* cp, int p, int c, int KC, uint4 v, int peer) {
  const int x = p & 15;
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(cp);
  st16(base + COPY_BYTES + cp_off(p, c, KC), v, peer);                        // dx = 0
  if (x >= 1) st16(base + 2 * COPY_BYTES + cp_off(p - 1, c, KC), v, peer);    // dx = +1
  if (x <= 14) st16(base + cp_off(p + 1, c, KC), v, peer);                    // dx = -1
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
// covers, for a layout of KC channel groups, in CTA h of the pair: the 16
// halo rows at the patch edge (above the tile for h = 0, below it for
// h = 1; all copies), and every row whose x + dx leaves the patch (x = 15 in
// the dx = +1 copy, x = 0 in the dx = -1 copy, halo rows included).
__device__ __forceinline__ void zero_unwritten(unsigned char* cp, int KC, int h) {
  const uint4 z = make_uint4(0, 0, 0, 0);
  const int j0 = h == 0 ? -16 : HALF;
  for (int i = threadIdx.x; i < 3 * 16 * KC; i += blockDim.x) {
    const int k = i / (16 * KC), r = (i / KC) % 16, c = i % KC;
    *reinterpret_cast<uint4*>(cp + k * COPY_BYTES + cp_off(j0 + r, c, KC)) = z;
  }
  for (int i = threadIdx.x; i < 2 * (ROWS / 16) * KC; i += blockDim.x) {
    const int side = i / ((ROWS / 16) * KC), r = (i / KC) % (ROWS / 16), c = i % KC;
    const int j = 16 * r - 16 + (side ? 15 : 0);   // dx = +1 copy: x = 15; dx = -1 copy: x = 0
    *reinterpret_cast<uint4*>(cp + (side ? 2 : 0) * COPY_BYTES + cp_off(j, c, KC)) = z;
  }
}

__device__ __forceinline__ uint32_t pack2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// All MMAs of one layer for the CTA's tile (TMEM columns 0..N-1), over 9 taps
// x KC/2 K-steps of 16.  dA / dB are the descriptors of the first copy / the
// weight image; a descriptor's start field is the byte address / 16, so an
// offset is added as offset / 16.  Tap dy reads local rows 16 dy .. 16 dy + 127.
template <int KC, int N>
__device__ __forceinline__ void issue_layer(uint32_t tmem, uint64_t dA, uint64_t dB) {
  constexpr uint32_t idesc = tc::instr_desc(128, N);
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) {
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const uint32_t a_off = (uint32_t)((dx + 1) * COPY_BYTES + ((16 + 16 * dy) >> 3) * KC * 128);
#pragma unroll
    for (int s = 0; s < KC / 2; ++s)
      mma_f16(tmem, dA + ((a_off + 256u * s) >> 4), dB + ((uint32_t)(tap * KC * 128 + 256 * s) >> 4), idesc,
              (tap | s) ? 1u : 0u);
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

// hidden-layer epilogue of this thread's pixel row and 32 of the 64 channels
// (TMEM address ta, their biases): bias, ReLU, bf16, as 4 channel groups g[4]
// of the next layer's input
__device__ __forceinline__ void epilogue_hidden(uint32_t ta, const float* bias, uint4 (&g)[4]) {
  uint32_t v[32];
  FZ_TMEM_LD16(v, ta);
  FZ_TMEM_LD16(v + 16, ta + 16);
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float s = __uint_as_float(v[8 * q + j]) + bias[8 * q + j];
      a[j] = s > 0.0f ? s : 0.0f;
    }
    g[q] = make_uint4(pack2(a[0], a[1]), pack2(a[2], a[3]), pack2(a[4], a[5]), pack2(a[6], a[7]));
  }
}

}  // namespace fz

}  // namespace lbm
