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

// A cluster of two CTAs per patch of the batch (ptab: replica, side, py),
// 256 threads each, fz::SMEM bytes of dynamic shared memory.  CTA h (rank in
// the pair) computes pixels m = 128 h + p, p = 0..127: thread p < 128 stages
// the input of pixel m and writes its output; threads 128 .. 143 stage the
// input of the image row across the cut (pixel 128 + t for h = 0, 112 + t
// for h = 1); in the hidden epilogues warp w reads TMEM lanes 32 (w mod 4) ..
// (pixel rows) and columns 32 (w / 4) .. (channels), and the threads holding
// the image row next to the cut also send it to the other CTA's halo rows
// (distributed shared memory).  Both CTAs pass the same sequence of cluster
// barriers on every path, so neither waits for a partner that has left; the
// mbarrier waits are bounded; a timeout sets *err, the CTA skips its
// remaining work (but not the barriers), releases its TMEM and returns.
// ONE: a single-replica handle, whose record comes as a kernel parameter
// (constant-bank operands, no dependent load before the input can be read).
template <typename S, bool ONE>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(256, 1)
    closure_step(const RepDev* __restrict__ reps, const __grid_constant__ RepDev one,
                 const StepInfo* __restrict__ si, int k, int nrep, const int4* __restrict__ ptab,
                 const __nv_bfloat16* __restrict__ img, const float* __restrict__ theta, fz::Meta meta, int* err) {
  using namespace fz;
  using namespace tc;
  using R = typename Store<S>::R;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ RepDev rd_s;
  __shared__ StepInfo st;
  __shared__ __align__(8) uint64_t mbar;      // MMAs of a layer complete
  __shared__ __align__(8) uint64_t wbar[2];   // weight image in buffer b arrived
  __shared__ float s_bias[4][64];
  __shared__ float s_zsum[4][16][3];          // per-warp column sums of the last layer's output
  __shared__ float s_zcol[2][16][3];          // column sums of the two CTAs (the other's written by it)
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  unsigned char* cp = sm;                     // copies for dx = -1, 0, +1 at cp + (dx + 1) COPY_BYTES
  unsigned char* wsm = sm + 3 * COPY_BYTES;   // weight buffers b at wsm + b W_BYTES
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int h = (int)(blockIdx.x & 1u), other = h ^ 1;
  const int patch = (int)(blockIdx.x >> 1);

  // what needs no record first: the first two weight images, TMEM, biases,
  // the unwritten positions of layer 0's input; then the records
  if (tid == 0) {
    mbar_init(&mbar, 1);
    mbar_init(&wbar[0], 1);
    mbar_init(&wbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
    bulk_weights(wsm, img, (uint32_t)img_bytes(0), &wbar[0]);
    bulk_weights(wsm + W_BYTES, img + img_off(1) / 2, (uint32_t)img_bytes(1), &wbar[1]);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(&tmem_base)),
                 "r"(64u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  {
    const int l = tid >> 6, c = tid & 63;
    s_bias[l][c] = c < coutr(l) ? theta[meta.boff[l] + c] : 0.0f;
  }
  zero_unwritten(cp, 4, h);
  const int4 pt = ptab[patch];
  const int side = pt.y, py = pt.z;
  if (ONE) {
    const int* c = (const int*)(si + k);
    int* d = (int*)&st;
    for (int i = threadIdx.x; i < (int)(sizeof(StepInfo) / 4); i += blockDim.x) d[i] = c[i];
    __syncthreads();
  } else {
    load_block_records(rd_s, st, reps, si, pt.x, k, nrep);   // ends with a barrier
  }
  const RepDev& rd = ONE ? one : rd_s;
  const uint32_t n = st.n;
  const long long ncl = 32LL * rd.Hy;
  const int row0 = cl_row0(rd, py), own0 = py == rd.cl_npy - 1 ? CL_W * py : row0;
  const int rows_end = py == rd.cl_npy - 1 ? rd.Hy : own0 + CL_W;
  const int nodes = (rows_end - own0) / rd.r;   // inner-buffer nodes per column whose rows this patch owns
  const uint32_t first = (uint32_t)rd.cl_first;
  const bool eval = n >= first && (n - first) % (uint32_t)rd.cl_interval == 0u;
  if (!eval) {   // both CTAs of every pair, before any cluster barrier: let the copies land, free TMEM
    if (tid == 0) {
      mbar_wait(&wbar[0], 0);
      mbar_wait(&wbar[1], 0);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(64u) : "memory");
    return;
  }

  // input: the 8 frames of this thread's pixel (all loads first, so that they
  // are in flight together): steps n - 7 .. n - 1 from the ring, step n from
  // its frame (folded into the ring by the next LB launch)
  float mean8[3] = {0.0f, 0.0f, 0.0f};
  if (tid < 144) {
    const int m = tid < 128 ? 128 * h + tid : (h == 0 ? tid : tid - 16);   // 128 + t or 112 + t across the cut
    const int lrow = tid < 128 ? tid : (h == 0 ? tid : tid - 144);         // local row
    const long long cc = ((long long)side * rd.Hy + row0 + (m >> 4)) * CL_W + (m & 15);
    float v[3 * CL_F + 8];
#pragma unroll
    for (int f = 0; f < CL_F - 1; ++f) {
      const float* r = rd.cring + ((long long)((n + 1u + (uint32_t)f) & (CL_F - 1)) * ncl + cc) * 3;
#pragma unroll
      for (int c = 0; c < 3; ++c) v[3 * f + c] = r[c];
    }
    double fr[3];
    const double* fp = rd.cframe + 4 * ((n & 1) * ncl + cc);
#pragma unroll
    for (int c = 0; c < 3; ++c) fr[c] = fp[c];
    double phi[3];
    cl_phi(rd, fr, side, phi);
#pragma unroll
    for (int c = 0; c < 3; ++c) v[3 * (CL_F - 1) + c] = (float)phi[c];
#pragma unroll
    for (int c = 24; c < 32; ++c) v[c] = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float s = 0.0f;
#pragma unroll
      for (int f = 0; f < CL_F; ++f) s += v[3 * f + c];
      mean8[c] = 0.125f * s;
    }
#pragma unroll
    for (int g = 0; g < 4; ++g)
      put3(cp, lrow, g, 4,
           make_uint4(pack2(v[8 * g], v[8 * g + 1]), pack2(v[8 * g + 2], v[8 * g + 3]),
                      pack2(v[8 * g + 4], v[8 * g + 5]), pack2(v[8 * g + 6], v[8 * g + 7])),
           -1);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  // epilogue role of this thread: pixel row p (TMEM lane), channel half c2
  const int p = 32 * (warp & 3) + lane, c2 = warp >> 2;
  const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + 32u * (uint32_t)c2;
  const bool cut_row = h == 0 ? p >= 112 : p < 16;   // the image row next to the other CTA
  float z[3] = {0.0f, 0.0f, 0.0f};

  for (int l = 0; l < 4; ++l) {
    // this layer's weights, its MMAs (one thread), their completion
    bool ok = !s_fail && mbar_wait(&wbar[l & 1], (uint32_t)((l >> 1) & 1));
    if (__syncthreads_or(!ok) && tid == 0) s_fail = 1;
    __syncthreads();
    const bool run = !s_fail;
    if (run && tid == 0) {
      const uint32_t a0 = s_addr(cp), b0 = s_addr(wsm + (l & 1) * W_BYTES);
      if (l == 0) issue_layer<4, 64>(tmem, smem_desc(a0, 128, 4 * 128), smem_desc(b0, 128, 36 * 128));
      else if (l < 3) issue_layer<8, 64>(tmem, smem_desc(a0, 128, 8 * 128), smem_desc(b0, 128, 72 * 128));
      else issue_layer<8, 16>(tmem, smem_desc(a0, 128, 8 * 128), smem_desc(b0, 128, 72 * 128));
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       s_addr(&mbar))
                   : "memory");
    }
    ok = !run || mbar_wait(&mbar, (uint32_t)(l & 1));
    if (__syncthreads_or(!ok) && tid == 0) s_fail = 1;
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool go = !s_fail;
    // the weight buffer of this layer is free: the image of layer l + 2
    if (go && l + 2 < 4 && tid == 0)
      bulk_weights(wsm + (l & 1) * W_BYTES, img + img_off(l + 2) / 2, (uint32_t)img_bytes(l + 2), &wbar[l & 1]);
    if (go && l == 0) {   // the hidden layers use 8 channel groups: clear their unwritten positions
      zero_unwritten(cp, 8, h);
      __syncthreads();
    }
    // this CTA is done with the layer's inputs: the other may write its halo
    // rows once it has waited for this arrival
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    if (l < 3) {
      uint4 g[4];
      if (go) {
        epilogue_hidden(trow, s_bias[l] + 32 * c2, g);
#pragma unroll
        for (int q = 0; q < 4; ++q) put3(cp, p, 4 * c2 + q, 8, g[q], -1);
      }
      asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
      if (go && cut_row) {   // the image row next to the cut, into the other CTA's halo rows
        const int pp = h == 0 ? p - 128 : p + 128;
#pragma unroll
        for (int q = 0; q < 4; ++q) put3(cp, pp, 4 * c2 + q, 8, g[q], other);
      }
    } else {
      // output: the correction less its mean over the 16 rows of its patch
      // column (per field) plus the 8-frame mean.  Warps 0-3 hold pixels p =
      // tid, image rows 8 h + 2 warp + lane / 16, column lane % 16; the
      // column sums of this CTA's 8 rows go to both CTAs.
      if (go && warp < 4) {
        uint32_t v0[16];
        FZ_TMEM_LD16(v0, trow);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float zs[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          z[c] = __uint_as_float(v0[c]) + s_bias[3][c];
          zs[c] = z[c] + __shfl_xor_sync(0xFFFFFFFFu, z[c], 16);
        }
        if (lane < 16) {
#pragma unroll
          for (int c = 0; c < 3; ++c) s_zsum[warp][lane][c] = zs[c];
        }
      }
      __syncthreads();
      asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
      if (go && tid < 48) {
        const int x = tid / 3, c = tid % 3;
        const float cs = s_zsum[0][x][c] + s_zsum[1][x][c] + s_zsum[2][x][c] + s_zsum[3][x][c];
        s_zcol[h][x][c] = cs;
        st_cluster_f32(peer_addr(s_addr(&s_zcol[h][x][c]), (uint32_t)other), cs);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    pair_sync();   // every halo row (and column sum) written by either CTA is visible
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }

  // y of this thread's pixel (global: the CLOSURE_OUT field; shared: u_bar)
  const bool done = !s_fail;
  float* s_y = reinterpret_cast<float*>(sm);   // the copies are free once the last MMAs are done
  if (done && tid < 128) {
    const int m = 128 * h + tid, x = tid & 15;
    float* yr = rd.cl_y + ((long long)patch * 256 + m) * 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float zm = (s_zcol[0][x][c] + s_zcol[1][x][c]) * (1.0f / 16.0f);
      const float yv = (z[c] - zm) + mean8[c];
      yr[c] = yv;
      s_y[3 * tid + c] = yv;
    }
  }
  __syncthreads();

  // u_bar of the inner-buffer nodes whose fine rows this patch owns and which
  // lie in this CTA's 8 image rows; the LB updates from step n + 1 on impose it
  if (done) {
    for (int i = tid; i < nodes * rd.n_in; i += blockDim.x) {
      const int col = i / nodes, yn = 1 + own0 / rd.r + i % nodes;
      const int pr = (yn - 1) * rd.r - row0;   // patch row of the node's first fine row
      if (pr < 8 * h || pr >= 8 * h + 8) continue;
      R su0 = R(0), su1 = R(0);
      for (int a = 0; a < rd.r; ++a)
        for (int b = 0; b < rd.r; ++b) {
          const int ml = (pr + a - 8 * h) * CL_W + (rd.n_out + col) * rd.r + b;
          su0 += (R)s_y[3 * ml + 1];
          su1 += (R)s_y[3 * ml + 2];
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64u) : "memory");
  }
}

template <typename S>
static cudaError_t go_step(const Launch& L, const int4* ptab, int P, int k, const ClosureNet& cn) {
  static const cudaError_t attr =
      cudaFuncSetAttribute(closure_step<S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, fz::SMEM);
  static const cudaError_t attr1 =
      cudaFuncSetAttribute(closure_step<S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, fz::SMEM);
  if (attr != cudaSuccess) return attr;
  if (attr1 != cudaSuccess) return attr1;
  if (L.nrep == 1 && L.host)
    closure_step<S, true><<<2 * P, 256, fz::SMEM, L.stream>>>(L.reps, *L.host, L.si, k, L.nrep, ptab, cn.img,
                                                              cn.theta, cn.meta, cn.err);
  else
    closure_step<S, false><<<2 * P, 256, fz::SMEM, L.stream>>>(L.reps, RepDev{}, L.si, k, L.nrep, ptab, cn.img,
                                                               cn.theta, cn.meta, cn.err);
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
