// closure.cu -- the learned MPCD->LB closure: a 4-layer 3x3 convolutional
// network (24 -> 64 -> 64 -> 64 -> 3 channels on 16 x 16 patches of MPCD
// cells) with bf16 weights and activations and fp32 accumulation.  Every
// contraction (forward, backward-data, backward-weights) is an implicit-GEMM
// on the tcgen05 tensor cores (tc_gemm.cuh).
#include <cuda_bf16.h>
#include <math.h>

#include <mutex>
#include <new>
#include <vector>

#include "../../include/lbmpcd.h"
#include "kernels.h"
#include "net_fused.cuh"
#include "tc_gemm.cuh"

namespace lbm {

// The dynamic shared-memory opt-in of a GEMM instantiation, set once on each
// device (a function attribute holds for the device that is current when it
// is set).
template <int BN>
static cudaError_t gemm_smem_optin() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(mu);
  if (!done[dev]) {
    e = cudaFuncSetAttribute(tc_gemm_bf16<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_gemm_smem<BN>());
    if (e != cudaSuccess) return e;
    done[dev] = true;
  }
  return cudaSuccess;
}

template <int BN>
static cudaError_t gemm_bn(const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, int M, int N, int K, int ldc,
                           float alpha, float beta, int* err, cudaStream_t st) {
  const cudaError_t attr = gemm_smem_optin<BN>();
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

// ===========================================================================
// The network.  Patches are 16 x 16 cells, NHWC; a layer is im2col ->
// tcgen05 GEMM -> epilogue.  Row m of every matrix is pixel m = 256 p +
// 16 y + x of patch p; column k of an im2col matrix is (3 ky + kx) cin + ci.
namespace lbm {

struct NetLayer { int cin, cout, kdim, kpad, npad; long long woff, boff; };
constexpr int NL = 4;
static const int LCIN[NL] = {24, 64, 64, 64}, LCOUT[NL] = {64, 64, 64, 3};

static NetLayer layer(int l) {
  NetLayer L;
  L.cin = LCIN[l]; L.cout = LCOUT[l]; L.kdim = 9 * L.cin; L.kpad = (L.kdim + 63) / 64 * 64;
  L.npad = L.cout < 16 ? 16 : L.cout;
  long long o = 0;
  for (int i = 0; i < l; ++i) o += (long long)LCOUT[i] * 9 * LCIN[i] + LCOUT[i];
  L.woff = o; L.boff = o + (long long)L.cout * L.kdim;
  return L;
}
static long long net_nparams() { const NetLayer L = layer(NL - 1); return L.boff + L.cout; }

__device__ __forceinline__ __nv_bfloat16 bf(float x) { return __float2bfloat16_rn(x); }

// weights fp32 -> W [npad][kpad] and W^T [kpad][64] in bf16, zero padded
__global__ void k_cast_weights(const float* __restrict__ theta, NetLayer L, __nv_bfloat16* W, __nv_bfloat16* WT) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < L.npad * L.kpad) {
    const int n = i / L.kpad, k = i % L.kpad;
    W[i] = bf(n < L.cout && k < L.kdim ? theta[L.woff + (long long)n * L.kdim + k] : 0.0f);
  }
  if (i < L.kpad * 64) {
    const int k = i / 64, c = i % 64;
    WT[i] = bf(c < L.cout && k < L.kdim ? theta[L.woff + (long long)c * L.kdim + k] : 0.0f);
  }
}

// fp32 input [M][24] -> bf16 activations; rows past the patches are zero
__global__ void k_input(const float* __restrict__ x, int M, int Mpad, __nv_bfloat16* a0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Mpad * 24) return;
  a0[i] = bf(i < M * 24 ? x[i] : 0.0f);
}

// col[m][k], 8 consecutive k per thread (one 16-byte store)
template <int CIN>
__global__ void k_im2col(const __nv_bfloat16* __restrict__ a, int M, int Mpad, int kpad, __nv_bfloat16* col) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int kq = kpad / 8;
  if (t >= (long long)Mpad * kq) return;
  const int m = (int)(t / kq), k0 = (int)(t % kq) * 8;
  uint4 v = make_uint4(0, 0, 0, 0);
  const int tap = k0 / CIN, ci = k0 % CIN;
  if (m < M && tap < 9) {
    const int p = m >> 8, y = ((m >> 4) & 15) + tap / 3 - 1, x = (m & 15) + tap % 3 - 1;
    if (y >= 0 && y < 16 && x >= 0 && x < 16)
      v = *reinterpret_cast<const uint4*>(a + (((long long)p * 256 + y * 16 + x) * CIN + ci));
  }
  *reinterpret_cast<uint4*>(col + (long long)m * kpad + k0) = v;
}

// colT[k][m] (the transposed im2col the weight-gradient GEMM reads)
template <int CIN>
__global__ void k_im2colT(const __nv_bfloat16* __restrict__ a, int M, int Mpad, int kpad, __nv_bfloat16* colT) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)kpad * Mpad) return;
  const int k = (int)(t / Mpad), m = (int)(t % Mpad);
  __nv_bfloat16 v = bf(0.0f);
  const int tap = k / CIN, ci = k % CIN;
  if (m < M && tap < 9) {
    const int p = m >> 8, y = ((m >> 4) & 15) + tap / 3 - 1, x = (m & 15) + tap % 3 - 1;
    if (y >= 0 && y < 16 && x >= 0 && x < 16) v = a[((long long)p * 256 + y * 16 + x) * CIN + ci];
  }
  colT[t] = v;
}

// z += b; hidden layers: a = bf16(relu(z)); last layer: y = z + mean of the 8
// input frames (k_center then takes z's column means off y)
__global__ void k_epilogue(float* __restrict__ z, const float* __restrict__ theta, NetLayer L, int M, int last,
                           __nv_bfloat16* a, const float* __restrict__ x32, float* y) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)M * L.cout) return;
  const int m = (int)(i / L.cout), c = (int)(i % L.cout);
  float v = z[(long long)m * L.npad + c] + theta[L.boff + c];
  z[(long long)m * L.npad + c] = v;
  if (!last) {
    a[i] = bf(v > 0.0f ? v : 0.0f);
  } else {
    float s = 0.0f;
#pragma unroll
    for (int f = 0; f < 8; ++f) s += x32[(long long)m * 24 + 3 * f + c];
    y[i] = v + 0.125f * s;
  }
}

// dst[m][c] -= mean of src[.][c] over the 16 rows of m's patch column (pixel
// m = 16 y + x of patch m / 256; same patch and x), c < 3: the centring of the
// last layer's output (forward) and of dL/dy (backward: the centring is its
// own adjoint).  One block of 256 threads per patch: warp w holds rows 2w and
// 2w + 1, lanes l and l ^ 16 the same column.  Each thread reads and writes
// only its own row, so dst may be src.
__global__ void __launch_bounds__(256) k_center(float* dst, int dstride, const float* src, int sstride) {
  __shared__ float part[8][16][3];
  const long long m = (long long)blockIdx.x * 256 + threadIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float v[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    v[c] = src[m * sstride + c];
    v[c] += __shfl_xor_sync(0xFFFFFFFFu, v[c], 16);
  }
  if (lane < 16) {
#pragma unroll
    for (int c = 0; c < 3; ++c) part[warp][lane][c] = v[c];
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float s = 0.0f;
#pragma unroll
    for (int w = 0; w < 8; ++w) s += part[w][lane & 15][c];
    dst[m * dstride + c] -= s * (1.0f / 16.0f);
  }
}

// MSE loss and dL/dy = 2 (y - t) / (3 M) into d (row stride 64)
__global__ void k_loss(const float* __restrict__ y, const float* __restrict__ t, int M, float* d, float* loss) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  float e2 = 0.0f;
  if (i < (long long)M * 3) {
    const float e = y[i] - t[i];
    d[(i / 3) * 64 + i % 3] = 2.0f * e / (3.0f * M);
    e2 = e * e / (3.0f * M);
  }
  for (int o = 16; o > 0; o >>= 1) e2 += __shfl_down_sync(0xFFFFFFFFu, e2, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, e2);
}

// upstream gradient (through the ReLU of this layer's output unless last) ->
// dC [Mpad][64] and dC^T [64][Mpad] in bf16, bias gradient
__global__ void k_prep_dC(const float* __restrict__ d, const float* __restrict__ z, NetLayer L, int M, int Mpad,
                          int last, __nv_bfloat16* dC, __nv_bfloat16* dCT, float* grad) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;   // over Mpad * 64
  float g = 0.0f;
  int c = 0;
  if (i < (long long)Mpad * 64) {
    const int m = (int)(i / 64);
    c = (int)(i % 64);
    if (m < M && c < L.cout) {
      g = d[(long long)m * 64 + c];
      if (!last && !(z[(long long)m * L.npad + c] > 0.0f)) g = 0.0f;
    }
    dC[i] = bf(g);
    dCT[(long long)c * Mpad + m] = bf(g);
  }
  // bias gradient: lanes of a warp hold 32 consecutive channels of one pixel
  if (i < (long long)Mpad * 64 && c < L.cout && g != 0.0f) atomicAdd(&grad[L.boff + c], g);
}

// d[m][ci] (row stride 64) = sum over the taps of dcol[m - offset][(tap) cin + ci]
template <int CIN>
__global__ void k_col2im(const float* __restrict__ dcol, int M, int kpad, float* d) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)M * CIN) return;
  const int m = (int)(i / CIN), ci = (int)(i % CIN);
  const int p = m >> 8, y = (m >> 4) & 15, x = m & 15;
  float s = 0.0f;
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) {
    const int yo = y - (tap / 3 - 1), xo = x - (tap % 3 - 1);
    if (yo >= 0 && yo < 16 && xo >= 0 && xo < 16)
      s += dcol[((long long)p * 256 + yo * 16 + xo) * kpad + tap * CIN + ci];
  }
  d[(long long)m * 64 + ci] = s;
}

// weight gradient rows < cout, columns < kdim of dWfull [64][kpad]
__global__ void k_take_dW(const float* __restrict__ dW, NetLayer L, float* grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.cout * L.kdim) return;
  const int n = i / L.kdim, k = i % L.kdim;
  grad[L.woff + i] = dW[(long long)n * L.kpad + k];
}

__global__ void k_adam(float* theta, const float* __restrict__ g, float* m1, float* m2, long long n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float a = b1 * m1[i] + (1.0f - b1) * gi;
  const float b = b2 * m2[i] + (1.0f - b2) * gi * gi;
  m1[i] = a;
  m2[i] = b;
  theta[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}

}  // namespace lbm

struct lbmpcd_net {
  int cap = 0, Mpad = 0;
  long long nparam = 0;
  int adam_t = 0;
  cudaStream_t st = nullptr;
  float *theta = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
  __nv_bfloat16 *W[lbm::NL] = {}, *WT[lbm::NL] = {};
  __nv_bfloat16 *act[lbm::NL] = {};
  float *x32 = nullptr, *z[lbm::NL] = {}, *y = nullptr;
  __nv_bfloat16 *col = nullptr, *colT = nullptr, *dC = nullptr, *dCT = nullptr;
  float *dcol = nullptr, *d = nullptr, *dW = nullptr, *loss = nullptr;
  int* err = nullptr;
  __nv_bfloat16* img = nullptr;   // weight images of the fused in-loop forward
  bool weights_dirty = true;
  std::vector<void*> allocs;
};

namespace {
int net_alloc(lbmpcd_net* n, void** p, size_t bytes) {
  if (cudaMalloc(p, bytes) != cudaSuccess) return LBMPCD_ERR_OOM;
  n->allocs.push_back(*p);
  return cudaMemset(*p, 0, bytes) == cudaSuccess ? LBMPCD_OK : LBMPCD_ERR_CUDA;
}
inline int nblk(long long n, int t = 256) { return (int)((n + t - 1) / t); }
}  // namespace

extern "C" long long lbmpcd_net_num_params(void) { return lbm::net_nparams(); }

extern "C" void lbmpcd_net_destroy(lbmpcd_net* n) {
  if (!n) return;
  if (n->st) cudaStreamSynchronize(n->st); else cudaDeviceSynchronize();
  for (void* p : n->allocs) cudaFree(p);
  delete n;
}

extern "C" int lbmpcd_net_create(int max_patches, void* stream, lbmpcd_net** out) {
  using namespace lbm;
  if (!out || max_patches < 1 || max_patches > 8192) return LBMPCD_ERR_INVALID_ARG;
  *out = nullptr;
  lbmpcd_net* n = new (std::nothrow) lbmpcd_net();
  if (!n) return LBMPCD_ERR_OOM;
  n->cap = max_patches;
  n->Mpad = max_patches * 256;
  n->nparam = net_nparams();
  n->st = (cudaStream_t)stream;
  const long long Mp = n->Mpad;
  int rc = LBMPCD_OK;
#define NA(ptr, bytes) if (!rc) rc = net_alloc(n, (void**)&(ptr), (size_t)(bytes))
  NA(n->theta, n->nparam * 4); NA(n->grad, n->nparam * 4); NA(n->m1, n->nparam * 4); NA(n->m2, n->nparam * 4);
  for (int l = 0; l < NL; ++l) {
    const NetLayer L = layer(l);
    NA(n->W[l], (long long)L.npad * L.kpad * 2);
    NA(n->WT[l], (long long)L.kpad * 64 * 2);
    NA(n->act[l], Mp * L.cin * 2);
    NA(n->z[l], Mp * L.npad * 4);
  }
  NA(n->x32, Mp * 24 * 4); NA(n->y, Mp * 3 * 4);
  NA(n->col, Mp * 576 * 2); NA(n->colT, Mp * 576 * 2);
  NA(n->dcol, Mp * 576 * 4); NA(n->d, Mp * 64 * 4);
  NA(n->dC, Mp * 64 * 2); NA(n->dCT, Mp * 128 * 2);
  NA(n->dW, 128LL * 576 * 4); NA(n->loss, 4); NA(n->err, 4);
  NA(n->img, lbm::fz::IMG_TOTAL);
#undef NA
  if (rc) { lbmpcd_net_destroy(n); return rc; }
  *out = n;
  return LBMPCD_OK;
}

extern "C" int lbmpcd_net_set_params(lbmpcd_net* n, const float* theta, long long count, int on_device) {
  if (!n || !theta || count != n->nparam) return LBMPCD_ERR_INVALID_ARG;
  if (cudaMemcpyAsync(n->theta, theta, count * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                      n->st) != cudaSuccess)
    return LBMPCD_ERR_CUDA;
  cudaMemsetAsync(n->m1, 0, count * 4, n->st);
  cudaMemsetAsync(n->m2, 0, count * 4, n->st);
  n->adam_t = 0;
  n->weights_dirty = true;
  return cudaStreamSynchronize(n->st) == cudaSuccess ? LBMPCD_OK : LBMPCD_ERR_CUDA;
}

extern "C" int lbmpcd_net_get_params(lbmpcd_net* n, float* theta, long long count, int which, int on_device) {
  if (!n || !theta || count != n->nparam || which < 0 || which > 1) return LBMPCD_ERR_INVALID_ARG;
  if (cudaMemcpyAsync(theta, which ? n->grad : n->theta, count * 4,
                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, n->st) != cudaSuccess)
    return LBMPCD_ERR_CUDA;
  return cudaStreamSynchronize(n->st) == cudaSuccess ? LBMPCD_OK : LBMPCD_ERR_CUDA;
}

namespace lbm {
float* net_input(lbmpcd_net* n) { return n->x32; }
float* net_output(lbmpcd_net* n) { return n->y; }
int net_capacity(lbmpcd_net* n) { return n->cap; }

static void cast_weights(lbmpcd_net* n, cudaStream_t st) {
  for (int l = 0; l < NL; ++l) {
    const NetLayer L = layer(l);
    k_cast_weights<<<nblk((long long)(L.npad > 64 ? L.npad : 64) * L.kpad), 256, 0, st>>>(n->theta, L, n->W[l], n->WT[l]);
  }
  n->weights_dirty = false;
}

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

static NetMeta fused_meta() {
  NetMeta m;
  for (int l = 0; l < NL; ++l) { const NetLayer L = layer(l); m.woff[l] = L.woff; m.boff[l] = L.boff; }
  return m;
}

// parameters for in-loop inference: loaded, cast to bf16, packed into the
// weight images of the fused in-loop network and synchronised
int net_load_params(lbmpcd_net* n, const float* theta, int on_device) {
  if (cudaMemcpyAsync(n->theta, theta, n->nparam * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                      n->st) != cudaSuccess)
    return LBMPCD_ERR_CUDA;
  cast_weights(n, n->st);
  k_pack_fused<<<nblk(fz::IMG_TOTAL / 2), 256, 0, n->st>>>(n->theta, fused_meta(), n->img);
  if (cudaGetLastError() != cudaSuccess) return LBMPCD_ERR_CUDA;
  return cudaStreamSynchronize(n->st) == cudaSuccess ? LBMPCD_OK : LBMPCD_ERR_CUDA;
}

ClosureNet net_closure(lbmpcd_net* n) { return ClosureNet{n->img, n->theta, fused_meta(), n->err}; }

// forward pass of P patches already in net_input(n), weights already cast
cudaError_t net_forward_resident(lbmpcd_net* n, int P, cudaStream_t st) {
  const int M = P * 256, Mp = P * 256;   // one patch is two 128-row tiles: no padding rows needed
  k_input<<<nblk((long long)Mp * 24), 256, 0, st>>>(n->x32, M, Mp, n->act[0]);
  for (int l = 0; l < NL; ++l) {
    const NetLayer L = layer(l);
    const long long tq = (long long)Mp * (L.kpad / 8);
    if (L.cin == 24) k_im2col<24><<<nblk(tq), 256, 0, st>>>(n->act[l], M, Mp, L.kpad, n->col);
    else k_im2col<64><<<nblk(tq), 256, 0, st>>>(n->act[l], M, Mp, L.kpad, n->col);
    const cudaError_t e = tc_gemm(n->col, n->W[l], n->z[l], Mp, L.npad, L.kpad, L.npad, 1.0f, 0.0f, n->err, st);
    if (e != cudaSuccess) return e;
    const bool last = l == NL - 1;
    k_epilogue<<<nblk((long long)M * L.cout), 256, 0, st>>>(n->z[l], n->theta, L, M, last ? 1 : 0,
                                                            last ? nullptr : n->act[l + 1], n->x32, n->y);
  }
  k_center<<<P, 256, 0, st>>>(n->y, 3, n->z[NL - 1], layer(NL - 1).npad);
  return cudaGetLastError();
}

// the GEMMs' error word (a bounded wait gave up): read and cleared
int net_error(lbmpcd_net* n, cudaStream_t st) {
  int e = 0;
  if (cudaMemcpyAsync(&e, n->err, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) return LBMPCD_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return LBMPCD_ERR_CUDA;
  if (e && cudaMemset(n->err, 0, 4) != cudaSuccess) return LBMPCD_ERR_CUDA;
  return e ? LBMPCD_ERR_TIMEOUT : LBMPCD_OK;
}
}  // namespace lbm

namespace {
int net_forward(lbmpcd_net* n, const float* x, int P) {
  using namespace lbm;
  cudaStream_t st = n->st;
  if (n->weights_dirty) cast_weights(n, st);
  if (cudaMemcpyAsync(n->x32, x, (size_t)P * 256 * 24 * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return LBMPCD_ERR_CUDA;
  return net_forward_resident(n, P, st) == cudaSuccess ? LBMPCD_OK : LBMPCD_ERR_CUDA;
}

int net_backward(lbmpcd_net* n, const float* t, int P) {
  using namespace lbm;
  cudaStream_t st = n->st;
  const int M = P * 256, Mp = P * 256;
  cudaMemsetAsync(n->grad, 0, n->nparam * 4, st);
  cudaMemsetAsync(n->loss, 0, 4, st);
  cudaMemsetAsync(n->d, 0, (size_t)Mp * 64 * 4, st);
  k_loss<<<nblk((long long)M * 3), 256, 0, st>>>(n->y, t, M, n->d, n->loss);
  k_center<<<P, 256, 0, st>>>(n->d, 64, n->d, 64);   // dL/dz of the last layer
  for (int l = NL - 1; l >= 0; --l) {
    const NetLayer L = layer(l);
    k_prep_dC<<<nblk((long long)Mp * 64), 256, 0, st>>>(n->d, n->z[l], L, M, Mp, l == NL - 1 ? 1 : 0, n->dC, n->dCT,
                                                       n->grad);
    const long long tT = (long long)L.kpad * Mp;
    if (L.cin == 24) k_im2colT<24><<<nblk(tT), 256, 0, st>>>(n->act[l], M, Mp, L.kpad, n->colT);
    else k_im2colT<64><<<nblk(tT), 256, 0, st>>>(n->act[l], M, Mp, L.kpad, n->colT);
    // dW [128 rows, the first 64 = dC^T rows][kpad] = dC^T colT^T
    if (tc_gemm(n->dCT, n->colT, n->dW, 128, L.kpad, Mp, L.kpad, 1.0f, 0.0f, n->err, st) != cudaSuccess)
      return LBMPCD_ERR_CUDA;
    k_take_dW<<<nblk((long long)L.cout * L.kdim), 256, 0, st>>>(n->dW, L, n->grad);
    if (l > 0) {
      if (tc_gemm(n->dC, n->WT[l], n->dcol, Mp, L.kpad, 64, L.kpad, 1.0f, 0.0f, n->err, st) != cudaSuccess)
        return LBMPCD_ERR_CUDA;
      k_col2im<64><<<nblk((long long)M * 64), 256, 0, st>>>(n->dcol, M, L.kpad, n->d);
    }
  }
  return cudaGetLastError() == cudaSuccess ? LBMPCD_OK : LBMPCD_ERR_CUDA;
}

int net_check_err(lbmpcd_net* n) {
  int e = 0;
  if (cudaMemcpyAsync(&e, n->err, 4, cudaMemcpyDeviceToHost, n->st) != cudaSuccess) return LBMPCD_ERR_CUDA;
  if (cudaStreamSynchronize(n->st) != cudaSuccess) return LBMPCD_ERR_CUDA;
  return e ? LBMPCD_ERR_TIMEOUT : LBMPCD_OK;
}
}  // namespace

extern "C" int lbmpcd_net_forward(lbmpcd_net* n, const float* x_dev, int P, float* y_dev) {
  if (!n || !x_dev || !y_dev || P < 1 || P > n->cap) return LBMPCD_ERR_INVALID_ARG;
  int rc = net_forward(n, x_dev, P);
  if (rc) return rc;
  if (cudaMemcpyAsync(y_dev, n->y, (size_t)P * 256 * 3 * 4, cudaMemcpyDeviceToDevice, n->st) != cudaSuccess)
    return LBMPCD_ERR_CUDA;
  return net_check_err(n);
}

extern "C" int lbmpcd_net_backward(lbmpcd_net* n, const float* x_dev, const float* t_dev, int P, float* loss) {
  if (!n || !x_dev || !t_dev || P < 1 || P > n->cap) return LBMPCD_ERR_INVALID_ARG;
  int rc = net_forward(n, x_dev, P);
  if (!rc) rc = net_backward(n, t_dev, P);
  if (rc) return rc;
  if (loss && cudaMemcpyAsync(loss, n->loss, 4, cudaMemcpyDeviceToHost, n->st) != cudaSuccess) return LBMPCD_ERR_CUDA;
  return net_check_err(n);
}

extern "C" int lbmpcd_net_train_step(lbmpcd_net* n, const float* x_dev, const float* t_dev, int P, float lr,
                                     float* loss) {
  using namespace lbm;
  if (!n || !x_dev || !t_dev || P < 1 || P > n->cap || !(lr > 0)) return LBMPCD_ERR_INVALID_ARG;
  int rc = net_forward(n, x_dev, P);
  if (!rc) rc = net_backward(n, t_dev, P);
  if (rc) return rc;
  n->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)n->adam_t), c2 = 1.0f - powf(b2, (float)n->adam_t);
  k_adam<<<nblk(n->nparam), 256, 0, n->st>>>(n->theta, n->grad, n->m1, n->m2, n->nparam, lr, b1, b2, 1e-8f, c1, c2);
  n->weights_dirty = true;
  if (loss && cudaMemcpyAsync(loss, n->loss, 4, cudaMemcpyDeviceToHost, n->st) != cudaSuccess) return LBMPCD_ERR_CUDA;
  return net_check_err(n);
}

// ===========================================================================
// Allocation-free network forward.  All scratch (bf16 weights, activations,
// the im2col matrix, the fp32 GEMM output, the GEMM error word) lives in one
// file-scope device array reserved when the module loads, so a call performs
// no cudaMalloc / cudaFree.  Layout, each slot a multiple of 256 bytes, for
// Mp = NET_STATIC_MAX_PATCHES * 256 rows:
//   err word (256) | per layer l: W npad x kpad, WT kpad x 64, act Mp x cin
//   (bf16) | z Mp x 64 fp32 (reused by every layer) | col Mp x 576 bf16
namespace lbm {
constexpr int NET_STATIC_MAX_PATCHES = LBMPCD_NET_STATIC_MAX_PATCHES;
constexpr long long NS_MP = (long long)NET_STATIC_MAX_PATCHES * 256;
constexpr long long ns_round(long long b) { return (b + 255) / 256 * 256; }
// layer widths as constants for sizing the array (the carve below checks them against layer())
constexpr int NS_CIN[NL] = {24, 64, 64, 64}, NS_COUT[NL] = {64, 64, 64, 3};
constexpr long long ns_kpad(int l) { return (9LL * NS_CIN[l] + 63) / 64 * 64; }
constexpr long long ns_npad(int l) { return NS_COUT[l] < 16 ? 16 : NS_COUT[l]; }
constexpr long long ns_layer_bytes(int l) {
  return ns_round(ns_npad(l) * ns_kpad(l) * 2) + ns_round(ns_kpad(l) * 64 * 2) + ns_round(NS_MP * NS_CIN[l] * 2);
}
constexpr long long NS_Z_BYTES = ns_round(NS_MP * 64 * 4);
constexpr long long NS_COL_BYTES = ns_round(NS_MP * 576 * 2);
constexpr long long NS_BYTES = 256 + ns_layer_bytes(0) + ns_layer_bytes(1) + ns_layer_bytes(2) + ns_layer_bytes(3) +
                               NS_Z_BYTES + NS_COL_BYTES;
static_assert(NS_BYTES <= 5LL * 1024 * 1024, "static network scratch stays modest");

static __device__ __align__(256) unsigned char g_net_scratch[NS_BYTES];

// device address of g_net_scratch on the current device, looked up once per device
static cudaError_t net_scratch_base(unsigned char** out) {
  static std::mutex mu;
  static unsigned char* base[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(mu);
  if (!base[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_net_scratch);
    if (e != cudaSuccess) return e;
    base[dev] = (unsigned char*)p;
  }
  *out = base[dev];
  return cudaSuccess;
}
}  // namespace lbm

extern "C" int lbmpcd_net_forward_noalloc(const float* theta_dev, const float* x_dev, int patches, float* y_dev,
                                          void* stream) {
  using namespace lbm;
  if (!theta_dev || !x_dev || !y_dev || patches < 1) return LBMPCD_ERR_INVALID_ARG;
  if (patches > NET_STATIC_MAX_PATCHES) return LBMPCD_ERR_CAPACITY;
  unsigned char* s = nullptr;
  if (net_scratch_base(&s) != cudaSuccess) return LBMPCD_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  int* err = (int*)s;
  unsigned char* q = s + 256;
  __nv_bfloat16 *W[NL], *WT[NL], *act[NL];
  for (int l = 0; l < NL; ++l) {
    const NetLayer L = layer(l);
    if (L.cin != NS_CIN[l] || L.cout != NS_COUT[l] || L.kpad != ns_kpad(l) || L.npad != ns_npad(l))
      return LBMPCD_ERR_INVALID_ARG;   // the array was sized for another network
    W[l] = (__nv_bfloat16*)q; q += ns_round(ns_npad(l) * ns_kpad(l) * 2);
    WT[l] = (__nv_bfloat16*)q; q += ns_round(ns_kpad(l) * 64 * 2);
    act[l] = (__nv_bfloat16*)q; q += ns_round(NS_MP * NS_CIN[l] * 2);
  }
  float* z = (float*)q;
  q += NS_Z_BYTES;
  __nv_bfloat16* col = (__nv_bfloat16*)q;

  // the error word is the only scratch read before this call writes it
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return LBMPCD_ERR_CUDA;
  const int M = patches * 256;   // a patch is two 128-row tiles: no padding rows
  for (int l = 0; l < NL; ++l) {
    const NetLayer L = layer(l);
    k_cast_weights<<<nblk((long long)(L.npad > 64 ? L.npad : 64) * L.kpad), 256, 0, st>>>(theta_dev, L, W[l], WT[l]);
  }
  k_input<<<nblk((long long)M * 24), 256, 0, st>>>(x_dev, M, M, act[0]);
  for (int l = 0; l < NL; ++l) {
    const NetLayer L = layer(l);
    const long long tq = (long long)M * (L.kpad / 8);
    if (L.cin == 24) k_im2col<24><<<nblk(tq), 256, 0, st>>>(act[l], M, M, L.kpad, col);
    else k_im2col<64><<<nblk(tq), 256, 0, st>>>(act[l], M, M, L.kpad, col);
    if (tc_gemm(col, W[l], z, M, L.npad, L.kpad, L.npad, 1.0f, 0.0f, err, st) != cudaSuccess) return LBMPCD_ERR_CUDA;
    const bool last = l == NL - 1;
    k_epilogue<<<nblk((long long)M * L.cout), 256, 0, st>>>(z, theta_dev, L, M, last ? 1 : 0,
                                                           last ? nullptr : act[l + 1], x_dev, y_dev);
  }
  k_center<<<patches, 256, 0, st>>>(y_dev, 3, z, layer(NL - 1).npad);
  if (cudaGetLastError() != cudaSuccess) return LBMPCD_ERR_CUDA;
  int e = 0;
  if (cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return LBMPCD_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return LBMPCD_ERR_CUDA;
  return e ? LBMPCD_ERR_TIMEOUT : LBMPCD_OK;
}
