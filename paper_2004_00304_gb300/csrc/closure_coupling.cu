// closure_coupling.cu -- the learned closure inside the coupled step
// (feedback = 2, D2Q9; not in the paper, which couples one way).
//
// Per step n, after cell_pass(n):
//   closure_in      one thread per strip cell: this step's count and momentum
//                   (sampled by particle_pass right after streaming, the
//                   instant of a6) -> the three fields
//                       phi_0 = n / ppc - 1,
//                       phi_1 = +-(sum v_x / n) / sqrt(kT/m)   (- on the right strip),
//                       phi_2 = (sum v_y / n) / sqrt(kT/m),
//                   stored in an 8-slot ring (binary32); the moving average
//                   e <- e + (phi - e) / 500 (binary64, e = phi at n = 0) is
//                   the training target; the last 8 frames, oldest first, are
//                   written as the network's 24 input channels of every patch
//                   holding the cell;
//   network forward (closure.cu) over the patches of all replicas at once;
//   closure_impose  one thread per inner-buffer LB node: u_bar = sqrt(kT/m)
//                   times the mean predicted velocity of its r x r fine cells,
//                   f_eq(rho_LB, u_bar) written into the buffer lb_pull(n+1)
//                   reads, from step 7 on (8 frames present).
// Strips: the 16 fine columns nearest each x-edge of the region, xi = distance
// from the edge.  Patches: side-major, ceil(Hy/16) per side, patch py covers
// rows 16 py .. 16 py + 15 except the last, which covers Hy - 16 .. Hy - 1.
#include "kernels.h"

namespace lbm {

constexpr int CL_W = 16;          // strip width and patch side, fine cells
constexpr int CL_F = 8;           // frames in the network input
constexpr double CL_EMA_T = 500.0;

__device__ __forceinline__ int cl_row0(const RepDev& rd, int py) {
  return py == rd.cl_npy - 1 ? rd.Hy - CL_W : CL_W * py;
}

// the 24 channels of one pixel: 6 float4 stores into a 96-byte run
__device__ __forceinline__ void cl_put(const RepDev& rd, int patch, int yy, int xi, const float* v) {
  float4* dst = (float4*)(rd.cl_x + (((long long)patch * CL_W + yy) * CL_W + xi) * (3 * CL_F));
#pragma unroll
  for (int q = 0; q < 6; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

__device__ __forceinline__ void closure_in_item(const RepDev& rd, const StepInfo& st, const int2 bm) {
  const long long ncl = 2LL * rd.Hy * CL_W;
  const long long c = (long long)bm.y * blockDim.x + threadIdx.x;
  if (c >= ncl) return;
  const int side = (int)(c / ((long long)rd.Hy * CL_W));
  const int row = (int)((c / CL_W) % rd.Hy), xi = (int)(c % CL_W);
  double* fr = rd.cframe + 4 * c;
  const double n = fr[0], px = fr[1], py = fr[2];
  fr[0] = 0.0; fr[1] = 0.0; fr[2] = 0.0;
  double phi[3];
  phi[0] = n / (double)rd.ppc - 1.0;
  phi[1] = n > 0 ? (side ? -1.0 : 1.0) * ((px / n) / rd.sig) : 0.0;
  phi[2] = n > 0 ? (py / n) / rd.sig : 0.0;
  double* e = rd.cema + 3 * c;
  float* ring = rd.cring;
  const uint32_t slot = st.n & (CL_F - 1);
  float v[3 * CL_F];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    ring[((long long)slot * ncl + c) * 3 + k] = (float)phi[k];
    e[k] = st.n == 0 ? phi[k] : e[k] + (phi[k] - e[k]) / CL_EMA_T;
    v[3 * (CL_F - 1) + k] = (float)phi[k];
  }
  // frame f (oldest first) of step n - 7 + f sits in slot (n + 1 + f) mod 8
#pragma unroll
  for (int f = 0; f < CL_F - 1; ++f) {
    const uint32_t s = (st.n + 1u + (uint32_t)f) & (CL_F - 1);
#pragma unroll
    for (int k = 0; k < 3; ++k) v[3 * f + k] = ring[((long long)s * ncl + c) * 3 + k];
  }
  const int pa = min(row / CL_W, rd.cl_npy - 1);
  cl_put(rd, rd.cl_p0 + side * rd.cl_npy + pa, row - cl_row0(rd, pa), xi, v);
  if (pa != rd.cl_npy - 1 && row >= rd.Hy - CL_W)   // also in the (overlapping) last patch
    cl_put(rd, rd.cl_p0 + side * rd.cl_npy + rd.cl_npy - 1, row - (rd.Hy - CL_W), xi, v);
}

__global__ void __launch_bounds__(256) closure_in(const RepDev* __restrict__ reps, const int2* __restrict__ bmap,
                                                  int nwork, const StepInfo* __restrict__ si, int k, int nrep) {
  __shared__ RepDev rd;
  __shared__ StepInfo st;
  for_each_item(bmap, nwork, reps, si, k, nrep, rd, st, [&](const int2 bm) { closure_in_item(rd, st, bm); });
}

template <typename S>
__device__ __forceinline__ void closure_impose_item(const RepDev& rd, const StepInfo& st, const int2 bm) {
  using R = typename Store<S>::R;
  using L = Lattice<9>;
  const long long b = (long long)bm.y * blockDim.x + threadIdx.x;
  if (b >= rd.nbuf || st.n < (uint32_t)(CL_F - 1)) return;
  long long t = b;
  const int yn = 1 + (int)(t % (rd.ny - 2));
  t /= (rd.ny - 2);
  const int col = (int)(t % rd.n_in), side = (int)(t / rd.n_in);
  double su0 = 0.0, su1 = 0.0;
  for (int a = 0; a < rd.r; ++a)
    for (int bb = 0; bb < rd.r; ++bb) {
      const int row = (yn - 1) * rd.r + a, xi = (rd.n_out + col) * rd.r + bb;
      const int py = min(row / CL_W, rd.cl_npy - 1);
      const long long p = rd.cl_p0 + side * rd.cl_npy + py;
      const long long m = (p * CL_W + (row - cl_row0(rd, py))) * CL_W + xi;
      su0 += (double)rd.cl_y[3 * m + 1];
      su1 += (double)rd.cl_y[3 * m + 2];
    }
  const double rr = (double)(rd.r * rd.r);
  R u[3];
  u[0] = (R)((side ? -1.0 : 1.0) * rd.sig * su0 / rr);
  u[1] = (R)(rd.sig * su1 / rr);
  u[2] = R(0);
  const int x = side == 0 ? rd.x0 + rd.n_out + col : rd.x1 - 1 - rd.n_out - col;
  const long long node = x + (long long)rd.nx * yn;
  S* dst = (S*)rd.f[(st.n & 1) ^ 1];
  const R rl = ((const R*)rd.rho)[node];
  const R uu = u[0] * u[0] + u[1] * u[1];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const R cu = L::cx(i) * u[0] + L::cy(i) * u[1];
    const R dev = (R)L::w(i) * ((rl - R(1)) + rl * (R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu));
    Store<S>::st(dst + i * rd.nnode + node, dev, rd.fp16_scale,
                 sizeof(S) == 2 ? (mix32((uint32_t)node * 19u + (uint32_t)i + st.n * 0x632BE5ABu) | 1u) : 0u);
  }
}

template <typename S>
__global__ void __launch_bounds__(256) closure_impose(const RepDev* __restrict__ reps,
                                                      const int2* __restrict__ bmap, int nwork,
                                                      const StepInfo* __restrict__ si, int k, int nrep) {
  __shared__ RepDev rd;
  __shared__ StepInfo st;
  for_each_item(bmap, nwork, reps, si, k, nrep, rd, st, [&](const int2 bm) { closure_impose_item<S>(rd, st, bm); });
}

// moving averages of one replica in patch layout [P][16][16][3], binary64
__global__ void closure_target_out(RepDev rd, double* __restrict__ out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long npx = 2LL * rd.cl_npy * CL_W * CL_W;
  if (i >= npx) return;
  const int p = (int)(i / (CL_W * CL_W)), yy = (int)((i / CL_W) % CL_W), xi = (int)(i % CL_W);
  const int side = p / rd.cl_npy, py = p % rd.cl_npy;
  const long long c = ((long long)side * rd.Hy + cl_row0(rd, py) + yy) * CL_W + xi;
#pragma unroll
  for (int k = 0; k < 3; ++k) out[3 * i + k] = rd.cema[3 * c + k];
}

cudaError_t launch_closure_in(const Launch& L, const int2* bmap, int nwork, int k) {
  if (nwork == 0) return cudaSuccess;
  static const int g = grid_cap(grid_for(closure_in, 256, 1 << 30));
  closure_in<<<g < nwork ? g : nwork, 256, 0, L.stream>>>(L.reps, bmap, nwork, L.si, k, L.nrep);
  return cudaGetLastError();
}

template <typename S>
static void go_impose(const Launch& L, const int2* bmap, int nwork, int k) {
  static const int g = grid_cap(grid_for(closure_impose<S>, 256, 1 << 30));
  closure_impose<S><<<g < nwork ? g : nwork, 256, 0, L.stream>>>(L.reps, bmap, nwork, L.si, k, L.nrep);
}

cudaError_t launch_closure_impose(int prec, const Launch& L, const int2* bmap, int nwork, int k) {
  if (nwork == 0) return cudaSuccess;
  if (prec == P_FP64) go_impose<double>(L, bmap, nwork, k);
  else if (prec == P_FP32) go_impose<float>(L, bmap, nwork, k);
  else go_impose<__half>(L, bmap, nwork, k);
  return cudaGetLastError();
}

cudaError_t launch_closure_target_out(const RepDev& rd, double* out, cudaStream_t st) {
  const long long n = 2LL * rd.cl_npy * CL_W * CL_W;
  closure_target_out<<<(int)((n + 255) / 256), 256, 0, st>>>(rd, out);
  return cudaGetLastError();
}

}  // namespace lbm
