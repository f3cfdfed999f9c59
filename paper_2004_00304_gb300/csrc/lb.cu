// lb.cu -- a1: the lattice Boltzmann update (Eq. 1 with the equilibrium of
// Eq. 2) as one fused pull kernel per step.
//
// Each thread owns one fluid node.  It pulls f*_i(x - c_i) from the
// post-collision buffer of the previous step (structure of arrays
// f[i][z][y][x]: for a fixed i, a warp reads 32 consecutive x, one coalesced
// segment), substitutes f*_{-i}(x) where x - c_i is a wall node (half-way
// bounce-back), forms rho and u = (sum f c + F/2)/rho with F = rho g (Guo
// forcing), relaxes to f_eq with rate 1/tau, adds the Guo source and writes
// f*_i(x) to the other buffer.  Populations are kept as deviations
// d_i = f_i - w_i (rho0 = 1) so that small body-force increments survive
// binary32 / scaled binary16 storage.  HBM traffic: one read and one write of
// q populations per node.
#include "lb_core.cuh"
#include "tc_gemm.cuh"

namespace lbm {

template <int Q, typename S, int V>
__global__ void __launch_bounds__(128, Q == 9 ? 7 : 5) lb_pull(const RepDev* __restrict__ reps, const int4* __restrict__ bmap,
                                               int nwork, const StepInfo* __restrict__ si, int k, int nrep) {
  for_each_item_direct(bmap, nwork, reps, si, k, nrep,
                       [&](const RepDev& rd, const StepInfo& st, const int4 bm) { lb_row<Q, S, V>(rd, st, bm); });
}

// single-replica form (see for_each_item_one)
// items from the block map (computing (tile, y, z) from the index takes
// integer divisions that cost more than the load)
template <int Q, typename S, int V>
// 7 resident blocks per SM for D2Q9 (72 registers, one 4-byte spill): the 2040
// row tiles of the 2048 x 512 channel take 1.92 rounds of the resident grid
// instead of 2.24 (72.8 against 73.7 us per step; 5 per SM was slower still)
__global__ void __launch_bounds__(128, Q == 9 ? 7 : 5) lb_pull_one(const __grid_constant__ RepDev rd, const int4* __restrict__ bmap,
                                                   int nwork, const StepInfo* __restrict__ si, int k) {
  __shared__ StepInfo st;
  for_each_item_one([bmap](int wi) { return bmap[wi]; }, nwork, si, k, st,
                    [&](const int4 bm) { lb_row<Q, S, V>(rd, st, bm); });
}

// LB rows of the overlapped form: items taken from the counter ctr[k] (one
// atomic per item, the next one fetched while the current one runs), so that
// the blocks that start beside the particle pass take as many rows as they
// can and the rest start when the pass ends; each block ends with the
// programmatic-dependency wait for the pass it was launched after.
template <typename Body>
__device__ __forceinline__ void rows_from_counter(const int4* __restrict__ bmap, int nwork, int* ctr, Body&& body) {
  __shared__ int s_next[2];
  if (threadIdx.x == 0) s_next[0] = atomicAdd(ctr, 1);
  __syncthreads();
  for (int it = 0;; ++it) {
    const int wi = s_next[it & 1];
    if (wi >= nwork) break;
    if (threadIdx.x == 0) s_next[(it + 1) & 1] = atomicAdd(ctr, 1);
    body(bmap[wi]);
    __syncthreads();
  }
  allow_dependent_launch();   // the table / a8 launch may start its blocks now
  wait_for_prerequisite();
}

#ifndef LBM_ROWS_MINB
#define LBM_ROWS_MINB 7
#endif
template <int Q, typename S, int V>
__global__ void __launch_bounds__(128, Q == 9 ? LBM_ROWS_MINB : 5) lb_rows_one(const __grid_constant__ RepDev rd,
                                                   const int4* __restrict__ bmap, int nwork,
                                                   const StepInfo* __restrict__ si, int k, int* ctr) {
  __shared__ StepInfo st;
  {
    const int* c = (const int*)(si + k);
    int* d = (int*)&st;
    for (int i = threadIdx.x; i < (int)(sizeof(StepInfo) / 4); i += blockDim.x) d[i] = c[i];
  }
  rows_from_counter(bmap, nwork, ctr + k, [&](const int4 bm) { lb_row<Q, S, V>(rd, st, bm); });
}

template <int Q, typename S, int V>
__global__ void __launch_bounds__(128, Q == 9 ? 7 : 5) lb_rows(const RepDev* __restrict__ reps,
                                               const int4* __restrict__ bmap, int nwork,
                                               const StepInfo* __restrict__ si, int k, int nrep, int* ctr) {
  rows_from_counter(bmap, nwork, ctr + k, [&](const int4 bm) {
    lb_row<Q, S, V>(reps[bm.x], si[(long long)k * nrep + bm.x], bm);
  });
}

template <int Q, typename S, int V>
static cudaError_t go_lb_rows(const Launch& L, const int4* bmap, int nwork, int k, int* ctr) {
  if (nwork == 0) return cudaSuccess;
  if (L.nrep == 1 && L.host) {
    static const int g1 = grid_for(lb_rows_one<Q, S, V>, 128, 1 << 30);
    return launch_pdl(lb_rows_one<Q, S, V>, g1 < nwork ? g1 : nwork, 128, L.stream, true, *L.host, bmap, nwork,
                      L.si, k, ctr);
  }
  static const int g = grid_for(lb_rows<Q, S, V>, 128, 1 << 30);
  return launch_pdl(lb_rows<Q, S, V>, g < nwork ? g : nwork, 128, L.stream, true, L.reps, bmap, nwork, L.si, k,
                    L.nrep, ctr);
}

// The table / a8 launch of the overlapped form (items of lb_item only, so
// without the row code's registers).  Launched as a programmatic dependent of
// the LB rows (pdl), its blocks may be placed while the particle pass still
// runs; they wait for the rows (which wait for the pass) before any work,
// and let the next particle pass be placed at once.
#ifndef LBM_ITEMS_MINB
#define LBM_ITEMS_MINB 8
#endif
template <int Q, typename S>
__global__ void __launch_bounds__(128, LBM_ITEMS_MINB) lb_items_one(const __grid_constant__ RepDev rd,
                                                    const int4* __restrict__ bmap, int nwork,
                                                    const StepInfo* __restrict__ si, int k) {
  __shared__ StepInfo st;
  wait_for_prerequisite();
  allow_dependent_launch();
  {
    const int* c = (const int*)(si + k);
    int* d = (int*)&st;
    for (int i = threadIdx.x; i < (int)(sizeof(StepInfo) / 4); i += blockDim.x) d[i] = c[i];
    __syncthreads();
  }
  for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) lb_item<Q, S>(rd, st, bmap[wi]);
}

template <int Q, typename S>
__global__ void __launch_bounds__(128, LBM_ITEMS_MINB) lb_items(const RepDev* __restrict__ reps,
                                                const int4* __restrict__ bmap, int nwork,
                                                const StepInfo* __restrict__ si, int k, int nrep) {
  wait_for_prerequisite();
  allow_dependent_launch();
  for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
    const int4 bm = bmap[wi];
    lb_item<Q, S>(reps[bm.x], si[(long long)k * nrep + bm.x], bm);
  }
}

template <int Q, typename S>
static cudaError_t go_lb_items(const Launch& L, const int4* bmap, int nwork, int k, bool pdl) {
  if (nwork == 0) return cudaSuccess;
  if (L.nrep == 1 && L.host) {
    static const int g1 = grid_for(lb_items_one<Q, S>, 128, 1 << 30);
    return launch_pdl(lb_items_one<Q, S>, g1 < nwork ? g1 : nwork, 128, L.stream, pdl, *L.host, bmap, nwork, L.si, k);
  }
  static const int g = grid_for(lb_items<Q, S>, 128, 1 << 30);
  return launch_pdl(lb_items<Q, S>, g < nwork ? g : nwork, 128, L.stream, pdl, L.reps, bmap, nwork, L.si, k, L.nrep);
}

template <int Q, typename S, int V>
static cudaError_t go_lb(const Launch& L, const int4* bmap, int nwork, int k) {
  if (nwork == 0) return cudaSuccess;
  if (L.nrep == 1 && L.host) {
    static const int g1 = grid_cap(grid_for(lb_pull_one<Q, S, V>, 128, 1 << 30));
    lb_pull_one<Q, S, V><<<g1 < nwork ? g1 : nwork, 128, 0, L.stream>>>(*L.host, bmap, nwork, L.si, k);
    return cudaGetLastError();
  }
  static const int g = grid_cap(grid_for(lb_pull<Q, S, V>, 128, 1 << 30));
  lb_pull<Q, S, V><<<g < nwork ? g : nwork, 128, 0, L.stream>>>(L.reps, bmap, nwork, L.si, k, L.nrep);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a1 for D2Q9 binary32 rows with TMA staging.  A work item is a tile of up to
// TL_W = 512 nodes of one row (128 threads x 4 nodes).  Its 9 source segments
// (population i of row y - c_iy, or population opp(i) of row y where that row
// is a wall: half-way bounce-back) are brought into shared memory by bulk
// copies, each with a 4-node halo on both sides (wrapped periodically in x),
// into a ring of TL_STAGES stages; one thread issues the copies of the item
// TL_STAGES items ahead as soon as a stage is free, so that several rows per
// block are in flight without holding registers.  The collision is lb_finish,
// the same code as lb_pull.  Every mbarrier wait is bounded; a timeout sets
// *err, and the block waits (bounded) for its copies in flight and returns.
constexpr int TL_W = 512, TL_SEG = TL_W + 8, TL_STAGES = 3;
constexpr int TL_SMEM = TL_STAGES * 9 * TL_SEG * 4;

__device__ __forceinline__ void tl_copy(float* dst, const float* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(bytes), "r"((uint32_t)__cvta_generic_to_shared(bar))
               : "memory");
}

// issue the copies of one item into one stage (one thread)
__device__ __forceinline__ void tl_issue(const RepDev* __restrict__ reps, const StepInfo* __restrict__ si, int k,
                                         int nrep, const int4 bm, float* stage, uint64_t* bar) {
  using L = Lattice<9>;
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
  if (bm.y < 0) {   // a cell-table item: nothing to stage, complete the stage's phase
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(b) : "memory");
    return;
  }
  const RepDev& r = reps[bm.x];
  const int nx = r.nx, ny = r.ny, y = bm.z;
  const long long N = r.nnode;
  const float* src = (const float*)r.f[si[(long long)k * nrep + bm.x].n & 1];
  const int x0 = bm.y * TL_W, len = min(TL_W, nx - x0);
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(b),
               "r"((uint32_t)(9 * (len + 8) * 4))
               : "memory");
  const int xl = x0 == 0 ? nx - 4 : x0 - 4, xr = x0 + len == nx ? 0 : x0 + len;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int sy = y - L::cy(i);
    const bool bounce = (sy == 0) | (sy == ny - 1);
    const float* row = bounce ? src + L::opp(i) * N + (long long)y * nx : src + i * N + (long long)sy * nx;
    float* seg = stage + i * TL_SEG;
    tl_copy(seg, row + xl, 16u, bar);
    tl_copy(seg + 4, row + x0, (uint32_t)len * 4u, bar);
    tl_copy(seg + 4 + len, row + xr, 16u, bar);
  }
}

__global__ void __launch_bounds__(128) lb_pull_tma(const RepDev* __restrict__ reps, const int4* __restrict__ bmap,
                                                   int nwork, const StepInfo* __restrict__ si, int k, int nrep,
                                                   int* err) {
  using L = Lattice<9>;
  extern __shared__ __align__(16) float tsm[];
  __shared__ __align__(8) uint64_t full[TL_STAGES];
  __shared__ RepDev rd;
  __shared__ StepInfo st;
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < TL_STAGES; ++s) tc::mbar_init(&full[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int j = 0; j < TL_STAGES; ++j) {
      const int wi = blockIdx.x + j * gridDim.x;
      if (wi < nwork) tl_issue(reps, si, k, nrep, bmap[wi], tsm + j * 9 * TL_SEG, &full[j]);
    }
  }
  __syncthreads();
  int cur = -1, it = 0;
  for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x, ++it) {
    const int s = it % TL_STAGES;
    const int4 bm = bmap[wi];
    if (bm.x != cur) {
      __syncthreads();
      load_block_records(rd, st, reps, si, bm.x, k, nrep);
      cur = bm.x;
    }
    const bool ok = tc::mbar_wait(&full[s], (uint32_t)((it / TL_STAGES) & 1));
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicExch(err, 1);
        for (int q = 0; q < TL_STAGES; ++q) tc::mbar_wait(&full[q], (uint32_t)(((it + q) / TL_STAGES) & 1));
      }
      __syncthreads();
      return;
    }
    const int x0 = bm.y * TL_W, len = min(TL_W, rd.nx - x0), xl = 4 * tid;
    if (bm.y < 0) {
      if (st.cells)
        cell_table_item<9, float>(rd, st.n - 1u, st.prev_f[1] > 0.0f, (long long)(-1 - bm.y) * blockDim.x * CPT,
                                  rd.ncell);
    } else if (xl < len) {
      const float* stage = tsm + s * 9 * TL_SEG;
      const int y = bm.z;
      float d[9][4];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const int sy = y - L::cy(i);
        const bool bounce = (sy == 0) | (sy == rd.ny - 1);
        const float* seg = stage + i * TL_SEG + 4 + xl;   // node x0 + xl
        const float4 c = *reinterpret_cast<const float4*>(seg);
        if (L::cx(i) == 0 || bounce) {
          d[i][0] = c.x; d[i][1] = c.y; d[i][2] = c.z; d[i][3] = c.w;
        } else if (L::cx(i) > 0) {   // source x - 1
          d[i][0] = seg[-1]; d[i][1] = c.x; d[i][2] = c.y; d[i][3] = c.z;
        } else {                     // source x + 1
          d[i][0] = c.y; d[i][1] = c.z; d[i][2] = c.w; d[i][3] = seg[4];
        }
      }
      lb_finish<9, float, 4>(rd, st, d, x0 + xl, rd.nx * y, y, 0);
    }
    __syncthreads();   // every thread is done with stage s
    if (tid == 0) {
      const int nxt = wi + TL_STAGES * gridDim.x;
      if (nxt < nwork) tl_issue(reps, si, k, nrep, bmap[nxt], tsm + s * 9 * TL_SEG, &full[s]);
    }
  }
}

static cudaError_t go_lb_tma(const Launch& L, const int4* bmap, int nwork, int k) {
  if (nwork == 0) return cudaSuccess;
  static int g = 0;
  if (!g) {
    if (cudaFuncSetAttribute(lb_pull_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, TL_SMEM) != cudaSuccess)
      return cudaErrorInvalidValue;
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lb_pull_tma, 128, TL_SMEM);
    g = (occ > 0 ? occ : 1) * (sms > 0 ? sms : 1);
  }
  lb_pull_tma<<<g < nwork ? g : nwork, 128, TL_SMEM, L.stream>>>(L.reps, bmap, nwork, L.si, k, L.nrep, L.err);
  return cudaGetLastError();
}

// Nodes per thread: 4 for D2Q9 rows, 2 for D3Q19 rows (19 populations per
// node), 1 in binary64 or when the row length is not a multiple.
int lb_vector_width(int q, int prec, int nx) {
  if (prec == P_FP64) return 1;
  const int v = q == 9 ? 4 : 2;
  return nx % v == 0 ? v : 1;
}

bool lb_tma_ok(int q, int prec, int vec) { return q == 9 && prec == P_FP32 && vec == 4; }

cudaError_t launch_lb(int q, int prec, int vec, bool tma, const Launch& L, const int4* bmap, int nblocks, int k) {
  if (tma && lb_tma_ok(q, prec, vec)) return go_lb_tma(L, bmap, nblocks, k);
  if (q == 9) {
    if (prec == P_FP64) return go_lb<9, double, 1>(L, bmap, nblocks, k);
    if (prec == P_FP32) return vec == 4 ? go_lb<9, float, 4>(L, bmap, nblocks, k) : go_lb<9, float, 1>(L, bmap, nblocks, k);
    return vec == 4 ? go_lb<9, __half, 4>(L, bmap, nblocks, k) : go_lb<9, __half, 1>(L, bmap, nblocks, k);
  }
  if (prec == P_FP64) return go_lb<19, double, 1>(L, bmap, nblocks, k);
  if (prec == P_FP32) return vec == 2 ? go_lb<19, float, 2>(L, bmap, nblocks, k) : go_lb<19, float, 1>(L, bmap, nblocks, k);
  return vec == 2 ? go_lb<19, __half, 2>(L, bmap, nblocks, k) : go_lb<19, __half, 1>(L, bmap, nblocks, k);
}

cudaError_t launch_lb_rows(int q, int prec, int vec, const Launch& L, const int4* bmap, int nwork, int k, int* ctr) {
  if (q == 9) {
    if (prec == P_FP64) return go_lb_rows<9, double, 1>(L, bmap, nwork, k, ctr);
    if (prec == P_FP32)
      return vec == 4 ? go_lb_rows<9, float, 4>(L, bmap, nwork, k, ctr) : go_lb_rows<9, float, 1>(L, bmap, nwork, k, ctr);
    return vec == 4 ? go_lb_rows<9, __half, 4>(L, bmap, nwork, k, ctr) : go_lb_rows<9, __half, 1>(L, bmap, nwork, k, ctr);
  }
  if (prec == P_FP64) return go_lb_rows<19, double, 1>(L, bmap, nwork, k, ctr);
  if (prec == P_FP32)
    return vec == 2 ? go_lb_rows<19, float, 2>(L, bmap, nwork, k, ctr) : go_lb_rows<19, float, 1>(L, bmap, nwork, k, ctr);
  return vec == 2 ? go_lb_rows<19, __half, 2>(L, bmap, nwork, k, ctr) : go_lb_rows<19, __half, 1>(L, bmap, nwork, k, ctr);
}

cudaError_t launch_lb_items(int q, int prec, const Launch& L, const int4* bmap, int nwork, int k, bool pdl) {
  if (q == 9) {
    if (prec == P_FP64) return go_lb_items<9, double>(L, bmap, nwork, k, pdl);
    if (prec == P_FP32) return go_lb_items<9, float>(L, bmap, nwork, k, pdl);
    return go_lb_items<9, __half>(L, bmap, nwork, k, pdl);
  }
  if (prec == P_FP64) return go_lb_items<19, double>(L, bmap, nwork, k, pdl);
  if (prec == P_FP32) return go_lb_items<19, float>(L, bmap, nwork, k, pdl);
  return go_lb_items<19, __half>(L, bmap, nwork, k, pdl);
}

// ---- copy-out / copy-in of populations and LB-side diagnostics ------------
template <int Q, typename S>
__global__ void pops_out(const S* __restrict__ f, long long N, float inv, double* __restrict__ out) {
  using L = Lattice<Q>;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= Q * N) return;
  const int i = (int)(idx / N);
  double w = 0;
#pragma unroll
  for (int j = 0; j < Q; ++j) if (j == i) w = L::w(j);
  out[idx] = w + (double)Store<S>::ld(f + idx, inv);
}

template <int Q, typename S>
__global__ void pops_in(S* __restrict__ f0, S* __restrict__ f1, long long N, float scale,
                        const double* __restrict__ in) {
  using L = Lattice<Q>;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= Q * N) return;
  const int i = (int)(idx / N);
  double w = 0;
#pragma unroll
  for (int j = 0; j < Q; ++j) if (j == i) w = L::w(j);
  const double d = in[idx] - w;
  Store<S>::st(f0 + idx, (typename Store<S>::R)d, scale);
  Store<S>::st(f1 + idx, (typename Store<S>::R)d, scale);
}

// LB mass and momentum of the stored populations over fluid nodes (binary64).
template <int Q, typename S>
__global__ void lb_diag(const S* __restrict__ f, int nx, int ny, int nz, float inv, double* out) {
  using L = Lattice<Q>;
  const long long N = (long long)nx * ny * nz;
  double m = 0, px = 0, py = 0, pz = 0;
  for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < N;
       node += (long long)gridDim.x * blockDim.x) {
    const int y = (int)((node / nx) % ny);
    if (y == 0 || y == ny - 1) continue;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const double fv = L::w(i) + (double)Store<S>::ld(f + i * N + node, inv);
      m += fv; px += L::cx(i) * fv; py += L::cy(i) * fv; pz += L::cz(i) * fv;
    }
  }
  double v[4] = {m, px, py, pz};
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    double t = v[a];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&out[a], t);
  }
}

template <int Q, typename S>
static cudaError_t go_pops(const RepDev& rd, int parity, double* out, const double* in, double* diag,
                           cudaStream_t st) {
  const long long n = Q * rd.nnode;
  const int nb = (int)((n + 255) / 256);
  if (out) pops_out<Q, S><<<nb, 256, 0, st>>>((const S*)rd.f[parity], rd.nnode, rd.fp16_inv, out);
  if (in) pops_in<Q, S><<<nb, 256, 0, st>>>((S*)rd.f[0], (S*)rd.f[1], rd.nnode, rd.fp16_scale, in);
  if (diag) {
    const int g = (int)((rd.nnode + 255) / 256);
    lb_diag<Q, S><<<g < 1024 ? g : 1024, 256, 0, st>>>((const S*)rd.f[parity], rd.nx, rd.ny, rd.nz,
                                                       rd.fp16_inv, diag);
  }
  return cudaGetLastError();
}

static cudaError_t dispatch_pops(int q, int prec, const RepDev& rd, int parity, double* out, const double* in,
                                 double* diag, cudaStream_t st) {
  if (q == 9) {
    if (prec == P_FP64) return go_pops<9, double>(rd, parity, out, in, diag, st);
    if (prec == P_FP32) return go_pops<9, float>(rd, parity, out, in, diag, st);
    return go_pops<9, __half>(rd, parity, out, in, diag, st);
  }
  if (prec == P_FP64) return go_pops<19, double>(rd, parity, out, in, diag, st);
  if (prec == P_FP32) return go_pops<19, float>(rd, parity, out, in, diag, st);
  return go_pops<19, __half>(rd, parity, out, in, diag, st);
}

cudaError_t launch_pops_out(int q, int prec, const RepDev& rd, int parity, double* out, cudaStream_t st) {
  return dispatch_pops(q, prec, rd, parity, out, nullptr, nullptr, st);
}
// populations at equilibrium f_eq(rho0 = 1, u) (Eq. 2) from a velocity field
// u [3][nnode], written to both buffers: the way a flow is started from a
// prescribed velocity profile
template <int Q, typename S>
__global__ void pops_from_u(S* __restrict__ f0, S* __restrict__ f1, long long N, float scale,
                            const double* __restrict__ u) {
  using L = Lattice<Q>;
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const double ux = u[n], uy = u[N + n], uz = u[2 * N + n];
  const double uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const double cu = L::cx(i) * ux + L::cy(i) * uy + L::cz(i) * uz;
    const double d = L::w(i) * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    Store<S>::st(f0 + i * N + n, (typename Store<S>::R)d, scale);
    Store<S>::st(f1 + i * N + n, (typename Store<S>::R)d, scale);
  }
}

cudaError_t launch_pops_from_u(int q, int prec, const RepDev& rd, const double* u, cudaStream_t st) {
  const int nb = (int)((rd.nnode + 255) / 256);
#define LBM_PFU(QQ, SS) pops_from_u<QQ, SS><<<nb, 256, 0, st>>>((SS*)rd.f[0], (SS*)rd.f[1], rd.nnode, rd.fp16_scale, u)
  if (q == 9) {
    if (prec == P_FP64) LBM_PFU(9, double); else if (prec == P_FP32) LBM_PFU(9, float); else LBM_PFU(9, __half);
  } else {
    if (prec == P_FP64) LBM_PFU(19, double); else if (prec == P_FP32) LBM_PFU(19, float); else LBM_PFU(19, __half);
  }
#undef LBM_PFU
  return cudaGetLastError();
}

cudaError_t launch_pops_in(int q, int prec, const RepDev& rd, const double* in, cudaStream_t st) {
  return dispatch_pops(q, prec, rd, 0, nullptr, in, nullptr, st);
}
cudaError_t launch_diag_lb(int q, int prec, const RepDev& rd, int parity, double* out4, cudaStream_t st) {
  return dispatch_pops(q, prec, rd, parity, nullptr, nullptr, out4, st);
}

template <typename R>
__global__ void real_out(const R* __restrict__ src, long long n, double* __restrict__ out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (double)src[i];
}

template <typename R>
__global__ void fill_real(R* __restrict__ dst, long long n, double value) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (R)value;
}

cudaError_t launch_fill_real(int prec, void* dst, long long n, double value, cudaStream_t st) {
  const int nb = (int)((n + 255) / 256);
  if (n == 0) return cudaSuccess;
  if (prec == P_FP64) fill_real<double><<<nb, 256, 0, st>>>((double*)dst, n, value);
  else fill_real<float><<<nb, 256, 0, st>>>((float*)dst, n, value);
  return cudaGetLastError();
}

cudaError_t launch_real_out(int prec, const void* src, long long n, double* out, cudaStream_t st) {
  const int nb = (int)((n + 255) / 256);
  if (n == 0) return cudaSuccess;
  if (prec == P_FP64) real_out<double><<<nb, 256, 0, st>>>((const double*)src, n, out);
  else real_out<float><<<nb, 256, 0, st>>>((const float*)src, n, out);
  return cudaGetLastError();
}

}  // namespace lbm
