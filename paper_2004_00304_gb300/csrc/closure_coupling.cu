// closure_coupling.cu -- the learned closure inside the coupled step
// (feedback = 2, D2Q9; not in the paper, which couples one way).
//
// particle_pass(n) adds 1 and v of every particle whose home cell lies in a
// strip (the 16 fine columns nearest each x-edge of the region, xi = distance
// from the edge) to that cell's frame, half n & 1 of a double buffer.  The
// fields of step n per strip cell,
//     phi_0 = n / ppc - 1,
//     phi_1 = +-(sum v_x / n) / sqrt(kT/m)   (- on the right strip, seen in a mirror),
//     phi_2 = (sum v_y / n) / sqrt(kT/m)     (velocities 0 in an empty cell),
// go into slot n mod 8 of a ring of the last 8 steps (binary32) and the
// moving average e <- e + (phi - e) / 500 (binary64, e = phi at n = 0), the
// training target, by work items of the LB launch of step n + 1
// (cell_core.cuh), which also clear the half.  Patches: side-major,
// ceil(Hy/16) per side; patch py covers rows 16 py .. 16 py + 15 except the
// last, which covers Hy - 16 .. Hy - 1 and "owns" only its rows from
// 16 (npy - 1) on.
//
// On evaluation steps (n = n0, n0 + K, n0 + 2K, ... for the inference
// interval K, n0 = max(7, the step at which the parameters were loaded))
// closure_step runs once after the particle pass, one CTA per patch of the
// batch: the network input built from the ring (steps n - 7 .. n - 1) and the
// frame of step n straight into shared memory, the network (the tcgen05 layers
// of net_fused.cuh), the output and u_bar = sqrt(kT/m) times the mean
// predicted velocity over each inner-buffer node's r x r cells.  From the LB
// update after the first evaluation on, every update gives the inner-buffer
// nodes f_eq(rho_LB, u_bar) with the latest u_bar (lb_core.cuh), so the steps
// between evaluations launch nothing for the closure.
#include "cell_core.cuh"
#include "net_fused.cuh"

namespace lbm {

// network input of one replica's patches after step n, [P][16][16][24]
// binary64: frame f (oldest first) of step n - 7 + f is ring slot (n + 1 + f)
// mod 8 for f < 7; the newest, of step n, is still the frame the next LB
// launch folds in, so its fields are formed here
__global__ void closure_in_out(RepDev rd, uint32_t n, double* __restrict__ out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= 2LL * rd.cl_npy * CL_W * CL_W) return;
  const int p = (int)(i / (CL_W * CL_W)), yy = (int)((i / CL_W) % CL_W), xi = (int)(i % CL_W);
  const int side = p / rd.cl_npy, py = p % rd.cl_npy;
  const long long ncl = 32LL * rd.Hy;
  const long long c = ((long long)side * rd.Hy + cl_row0(rd, py) + yy) * CL_W + xi;
#pragma unroll
  for (int f = 0; f < CL_F - 1; ++f) {
    const float* r = rd.cring + ((long long)((n + 1u + (uint32_t)f) & (CL_F - 1)) * ncl + c) * 3;
#pragma unroll
    for (int k = 0; k < 3; ++k) out[24 * i + 3 * f + k] = (double)r[k];
  }
  double phi[3];
  cl_phi(rd, rd.cframe + 4 * ((n & 1) * ncl + c), side, phi);
#pragma unroll
  for (int k = 0; k < 3; ++k) out[24 * i + 3 * (CL_F - 1) + k] = (double)(float)phi[k];
}

// moving averages after step n of one replica in patch layout
// [P][16][16][3], binary64: the stored average runs to step n - 1, the frame
// of step n is added here as the next LB launch will
__global__ void closure_target_out(RepDev rd, uint32_t n, double* __restrict__ out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= 2LL * rd.cl_npy * CL_W * CL_W) return;
  const int p = (int)(i / (CL_W * CL_W)), yy = (int)((i / CL_W) % CL_W), xi = (int)(i % CL_W);
  const int side = p / rd.cl_npy, py = p % rd.cl_npy;
  const long long ncl = 32LL * rd.Hy;
  const long long c = ((long long)side * rd.Hy + cl_row0(rd, py) + yy) * CL_W + xi;
  double phi[3];
  cl_phi(rd, rd.cframe + 4 * ((n & 1) * ncl + c), side, phi);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double e = rd.cema[3 * c + k];
    out[3 * i + k] = n == 0 ? phi[k] : e + (phi[k] - e) * CL_EMA_A;
  }
}

// One CTA per patch of the batch (ptab: replica, side, py), 128 threads,
// fz::SMEM bytes of dynamic shared memory.  Thread (warp w, lane) handles the
// pixels m = 128 t + 32 w + lane, t = 0, 1, both for the input and for the
// output.  Every mbarrier wait is bounded; a timeout sets *err, and the CTA
// releases its TMEM and returns.
template <typename S>
__global__ void __launch_bounds__(128, 1) closure_step(const RepDev* __restrict__ reps,
                                                       const StepInfo* __restrict__ si, int k, int nrep,
                                                       const int4* __restrict__ ptab,
                                                       const __nv_bfloat16* __restrict__ img,
                                                       const float* __restrict__ theta, fz::Meta meta, int* err) {
  using namespace fz;
  using namespace tc;
  using R = typename Store<S>::R;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ RepDev rd;
  __shared__ StepInfo st;
  __shared__ __align__(8) uint64_t mbar;   // MMAs of a layer complete
  __shared__ __align__(8) uint64_t wbar;   // weight image of a layer arrived
  __shared__ float s_bias[4][64];
  __shared__ float s_zsum[4][16][3];      // per-warp column sums of the last layer's output
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  unsigned char* cp = sm;   // copies for dx = -1, 0, +1 at cp + (dx + 1) COPY_BYTES
  unsigned char* wsm = sm + 3 * COPY_BYTES;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int4 pt = ptab[blockIdx.x];
  const int side = pt.y, py = pt.z;
  load_block_records(rd, st, reps, si, pt.x, k, nrep);   // ends with a barrier
  const uint32_t n = st.n;
  const long long ncl = 32LL * rd.Hy;
  const int row0 = cl_row0(rd, py), own0 = py == rd.cl_npy - 1 ? CL_W * py : row0;
  const int rows_end = py == rd.cl_npy - 1 ? rd.Hy : own0 + CL_W;
  const int nodes = (rows_end - own0) / rd.r;   // inner-buffer nodes per column whose rows this patch owns
  const uint32_t first = (uint32_t)rd.cl_first;
  const bool eval = n >= first && (n - first) % (uint32_t)rd.cl_interval == 0u;
  if (!eval) return;   // launched on evaluation steps only (the chunk graphs disable the rest)

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(&tmem_base)),
                 "r"(128u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&mbar, 1);
    mbar_init(&wbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
    bulk_weights(wsm, img, (uint32_t)img_bytes(0), &wbar);
  }
  if (tid < 64) {
#pragma unroll
    for (int l = 0; l < 4; ++l) s_bias[l][tid] = tid < coutr(l) ? theta[meta.boff[l] + tid] : 0.0f;
  }
  zero_unwritten(cp, 4);
  __syncthreads();   // zeros and barrier initialisation before anyone writes or waits

  // input: the 8 frames of this thread's two pixels (all loads first, so that
  // they are in flight together): steps n - 7 .. n - 1 from the ring, step n
  // from its frame (folded into the ring by the next LB launch)
  float mean8[2][3];
  float v[2][3 * CL_F + 8];
  double fr[2][3];
  long long cc[2];
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const int m = 128 * t + 32 * warp + lane;
    cc[t] = ((long long)side * rd.Hy + row0 + (m >> 4)) * CL_W + (m & 15);
#pragma unroll
    for (int f = 0; f < CL_F - 1; ++f) {
      const float* r = rd.cring + ((long long)((n + 1u + (uint32_t)f) & (CL_F - 1)) * ncl + cc[t]) * 3;
#pragma unroll
      for (int q = 0; q < 3; ++q) v[t][3 * f + q] = r[q];
    }
    const double* fp = rd.cframe + 4 * ((n & 1) * ncl + cc[t]);
#pragma unroll
    for (int q = 0; q < 3; ++q) fr[t][q] = fp[q];
  }
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const int m = 128 * t + 32 * warp + lane;
    double phi[3];
    cl_phi(rd, fr[t], side, phi);
#pragma unroll
    for (int q = 0; q < 3; ++q) v[t][3 * (CL_F - 1) + q] = (float)phi[q];
#pragma unroll
    for (int q = 24; q < 32; ++q) v[t][q] = 0.0f;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float s = 0.0f;
#pragma unroll
      for (int f = 0; f < CL_F; ++f) s += v[t][3 * f + q];
      mean8[t][q] = 0.125f * s;
    }
#pragma unroll
    for (int g = 0; g < 4; ++g)
      put3(cp, m, g, 4,
           make_uint4(pack2(v[t][8 * g], v[t][8 * g + 1]), pack2(v[t][8 * g + 2], v[t][8 * g + 3]),
                      pack2(v[t][8 * g + 4], v[t][8 * g + 5]), pack2(v[t][8 * g + 6], v[t][8 * g + 7])));
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  for (int l = 0; l < 4; ++l) {
    const bool wok = mbar_wait(&wbar, (uint32_t)(l & 1));   // this layer's weights are in
    if (__syncthreads_or(!wok)) { s_fail = 1; break; }
    if (tid == 0) {
      const uint32_t a0 = s_addr(cp), b0 = s_addr(wsm);
      if (l == 0) issue_layer<4, 64>(tmem, smem_desc(a0, 128, 4 * 128), smem_desc(b0, 128, 36 * 128));
      else if (l < 3) issue_layer<8, 64>(tmem, smem_desc(a0, 128, 8 * 128), smem_desc(b0, 128, 72 * 128));
      else issue_layer<8, 16>(tmem, smem_desc(a0, 128, 8 * 128), smem_desc(b0, 128, 72 * 128));
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       s_addr(&mbar))
                   : "memory");
    }
    const bool mok = mbar_wait(&mbar, (uint32_t)(l & 1));
    if (__syncthreads_or(!mok)) { s_fail = 1; break; }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // this layer's MMAs are complete: the next layer's weights may overwrite
    // the staging buffer while the epilogue runs
    if (l < 3 && tid == 0) bulk_weights(wsm, img + img_off(l + 1) / 2, (uint32_t)img_bytes(l + 1), &wbar);
    if (l == 0) {   // the hidden layers use 8 channel groups: clear their unwritten positions
      zero_unwritten(cp, 8);
      __syncthreads();
    }
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    if (l < 3) {
      epilogue_hidden(cp, trow, 32 * warp + lane, s_bias[l]);
      epilogue_hidden(cp, trow + 64u, 128 + 32 * warp + lane, s_bias[l]);
    } else {
      // output: global (the CLOSURE_OUT field) and shared memory (the
      // imposition below); the copies are free once the last MMAs are done
      uint32_t v0[16], v1[16];
      FZ_TMEM_LD16(v0, trow);
      FZ_TMEM_LD16(v1, trow + 64u);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      // the correction less its mean over the 16 rows of its patch column
      // (per field) plus the 8-frame mean.  Pixel m = 16 y + x: this warp's
      // pixels are rows 8t + 2 warp + lane / 16, column lane % 16.
      float z[2][3], zs[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        z[0][c] = __uint_as_float(v0[c]) + s_bias[3][c];
        z[1][c] = __uint_as_float(v1[c]) + s_bias[3][c];
        zs[c] = z[0][c] + z[1][c];
        zs[c] += __shfl_xor_sync(0xFFFFFFFFu, zs[c], 16);
      }
      if (lane < 16) {
#pragma unroll
        for (int c = 0; c < 3; ++c) s_zsum[warp][lane][c] = zs[c];
      }
      __syncthreads();
      float* s_y = reinterpret_cast<float*>(sm);
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int m = 128 * t + 32 * warp + lane;
        float* yr = rd.cl_y + ((long long)blockIdx.x * 256 + m) * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int x = lane & 15;
          const float zm = (s_zsum[0][x][c] + s_zsum[1][x][c] + s_zsum[2][x][c] + s_zsum[3][x][c]) * (1.0f / 16.0f);
          const float yv = (z[t][c] - zm) + mean8[t][c];
          yr[c] = yv;
          s_y[3 * m + c] = yv;
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }

  // u_bar of the inner-buffer nodes whose fine rows this patch owns; the LB
  // updates from step n + 1 on impose it
  if (!s_fail) {
    const float* s_y = reinterpret_cast<const float*>(sm);
    for (int i = tid; i < nodes * rd.n_in; i += blockDim.x) {
      const int col = i / nodes, yn = 1 + own0 / rd.r + i % nodes;
      R su0 = R(0), su1 = R(0);
      for (int a = 0; a < rd.r; ++a)
        for (int b = 0; b < rd.r; ++b) {
          const int m = ((yn - 1) * rd.r + a - row0) * CL_W + (rd.n_out + col) * rd.r + b;
          su0 += (R)s_y[3 * m + 1];
          su1 += (R)s_y[3 * m + 2];
        }
      const R scale = (R)rd.sig / (R)(rd.r * rd.r);
      const R ux = (side ? -su0 : su0) * scale, uy = su1 * scale;
      double* u = rd.cl_u + 2 * (((long long)side * rd.n_in + col) * (rd.ny - 2) + (yn - 1));
      u[0] = (double)ux;   // imposed until the next evaluation
      u[1] = (double)uy;
    }
  }
  if (s_fail && tid == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128u) : "memory");
  }
}

template <typename S>
static cudaError_t go_step(const Launch& L, const int4* ptab, int P, int k, const ClosureNet& cn) {
  static const cudaError_t attr =
      cudaFuncSetAttribute(closure_step<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, fz::SMEM);
  if (attr != cudaSuccess) return attr;
  closure_step<S><<<P, 128, fz::SMEM, L.stream>>>(L.reps, L.si, k, L.nrep, ptab, cn.img, cn.theta, cn.meta,
                                                 cn.err);
  return cudaGetLastError();
}

cudaError_t launch_closure_step(int prec, const Launch& L, const int4* ptab, int P, int k, const ClosureNet& cn) {
  if (P == 0) return cudaSuccess;
  if (prec == P_FP64) return go_step<double>(L, ptab, P, k, cn);
  if (prec == P_FP32) return go_step<float>(L, ptab, P, k, cn);
  return go_step<__half>(L, ptab, P, k, cn);
}

cudaError_t launch_closure_in_out(const RepDev& rd, uint32_t n, double* out, cudaStream_t st) {
  const long long np = 2LL * rd.cl_npy * CL_W * CL_W;
  closure_in_out<<<(int)((np + 255) / 256), 256, 0, st>>>(rd, n, out);
  return cudaGetLastError();
}

cudaError_t launch_closure_target_out(const RepDev& rd, uint32_t n, double* out, cudaStream_t st) {
  const long long np = 2LL * rd.cl_npy * CL_W * CL_W;
  closure_target_out<<<(int)((np + 255) / 256), 256, 0, st>>>(rd, n, out);
  return cudaGetLastError();
}

}  // namespace lbm
