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
#include "kernels.h"

namespace lbm {

// V consecutive populations of one row: aligned vector load/store (V = 4 for
// binary32 and scaled binary16 rows whose length is a multiple of 4), scalar
// otherwise.
template <typename S, int V> struct Row;
template <typename S> struct Row<S, 1> {
  using R = typename Store<S>::R;
  __device__ static void ld(const S* p, R* o, float inv) { o[0] = Store<S>::ld(p, inv); }
  __device__ static void st(S* p, const R* v, float sc, uint32_t h) { Store<S>::st(p, v[0], sc, h); }
};
template <> struct Row<float, 4> {
  __device__ static void ld(const float* p, float* o, float) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
  }
  __device__ static void st(float* p, const float* v, float, uint32_t) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <> struct Row<float, 2> {
  __device__ static void ld(const float* p, float* o, float) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    o[0] = t.x; o[1] = t.y;
  }
  __device__ static void st(float* p, const float* v, float, uint32_t) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  }
};
template <> struct Row<__half, 2> {
  __device__ static void ld(const __half* p, float* o, float inv) {
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(p));
    o[0] = a.x * inv; o[1] = a.y * inv;
  }
  __device__ static void st(__half* p, const float* v, float sc, uint32_t h) {
    __half2 t;
    t.x = sr_half(v[0] * sc, h);
    t.y = sr_half(v[1] * sc, h ? mix32(h + 1u) : 0u);
    *reinterpret_cast<__half2*>(p) = t;
  }
};
template <> struct Row<__half, 4> {
  __device__ static void ld(const __half* p, float* o, float inv) {
    const uint2 t = *reinterpret_cast<const uint2*>(p);
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&t.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&t.y));
    o[0] = a.x * inv; o[1] = a.y * inv; o[2] = b.x * inv; o[3] = b.y * inv;
  }
  __device__ static void st(__half* p, const float* v, float sc, uint32_t h) {
    __half2 a, b;
    a.x = sr_half(v[0] * sc, h);
    a.y = sr_half(v[1] * sc, h ? mix32(h + 1u) : 0u);
    b.x = sr_half(v[2] * sc, h ? mix32(h + 2u) : 0u);
    b.y = sr_half(v[3] * sc, h ? mix32(h + 3u) : 0u);
    uint2 t;
    t.x = *reinterpret_cast<const uint32_t*>(&a);
    t.y = *reinterpret_cast<const uint32_t*>(&b);
    *reinterpret_cast<uint2*>(p) = t;
  }
};

__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// One thread owns V consecutive nodes x0 .. x0+V-1 of one row (y, z); a
// work item (replica, tile, y, z) is one block-wide tile of a row.
template <int Q, typename S, int V>
__device__ __forceinline__ void lb_row(const RepDev& rd, const StepInfo& st, const int4 bm) {
  using L = Lattice<Q>;
  using R = typename Store<S>::R;
  const int nx = rd.nx, ny = rd.ny, nz = rd.nz;
  const int y = bm.z, z = bm.w;
  const int tpr = nx / V;
  const int tx = bm.y * blockDim.x + threadIdx.x;
  const bool active = tx < tpr;
  const int lane = threadIdx.x & 31;
  const int x0 = tx * V;
  const int par = st.n & 1;
  const S* __restrict__ src = (const S*)rd.f[par];
  S* __restrict__ dst = (S*)rd.f[par ^ 1];
  const int N = (int)rd.nnode;
  const int row = nx * (y + ny * z);
  const float inv = rd.fp16_inv, scale = rd.fp16_scale;

  // phase 1: every load of the thread (Q aligned rows plus the scalar edge
  // values at warp boundaries), branch-free so that all of them are in flight
  // together: inactive tail lanes read a clamped, valid position and discard it,
  // bounce-back rows are selected, not branched to.
  const int xa = active ? x0 : (tpr - 1) * V;
  const int xprev = xa == 0 ? nx - 1 : xa - 1;
  const int xnext = xa + V >= nx ? 0 : xa + V;
  R d[Q][V], edge[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int sy = y - L::cy(i);
    const bool bounce = (sy == 0) | (sy == ny - 1);
    int sz = z - L::cz(i);
    sz = sz < 0 ? sz + nz : (sz >= nz ? sz - nz : sz);
    const S* srow_i = src + i * N + nx * (sy + ny * sz);
    const S* rp = bounce ? src + L::opp(i) * N + row : srow_i;
    if (V == 1) {
      int sx = xa - L::cx(i);
      sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
      d[i][0] = Store<S>::ld(rp + (bounce ? xa : sx), inv);
    } else {
      Row<S, V>::ld(rp + xa, d[i], inv);
    }
    edge[i] = R(0);
    if (V > 1 && L::cx(i) > 0) edge[i] = Store<S>::ld(rp + xprev, inv);
    if (V > 1 && L::cx(i) < 0) edge[i] = Store<S>::ld(rp + xnext, inv);
  }
  // phase 2: shift the rows with cx != 0 by one node through the neighbour lanes
  if (V > 1) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int sy = y - L::cy(i);
      if (L::cx(i) == 0 || sy == 0 || sy == ny - 1) continue;
      if (L::cx(i) > 0) {                    // source x - 1: previous lane's last node
        R prev = __shfl_up_sync(0xFFFFFFFFu, d[i][V - 1], 1);
        if (lane == 0) prev = edge[i];
#pragma unroll
        for (int v = V - 1; v > 0; --v) d[i][v] = d[i][v - 1];
        d[i][0] = prev;
      } else {                               // source x + 1: next lane's first node
        R next = __shfl_down_sync(0xFFFFFFFFu, d[i][0], 1);
        if (lane == 31 || tx + 1 >= tpr) next = edge[i];
#pragma unroll
        for (int v = 0; v < V - 1; ++v) d[i][v] = d[i][v + 1];
        d[i][V - 1] = next;
      }
    }
  }
  if (!active) return;

  const R om = Cst<R>::omega(rd), om1 = R(1) - om, cf = R(1) - R(0.5) * om;
  const R gx = Cst<R>::g(rd, 0), gy = Cst<R>::g(rd, 1), gz = Cst<R>::g(rd, 2);
  R mr[V], mu[3][V];   // post-collision values overwrite d in place
#pragma unroll
  for (int v = 0; v < V; ++v) {
    R drho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      drho += d[i][v];
      if (L::cx(i) > 0) jx += d[i][v]; else if (L::cx(i) < 0) jx -= d[i][v];
      if (L::cy(i) > 0) jy += d[i][v]; else if (L::cy(i) < 0) jy -= d[i][v];
      if (L::cz(i) > 0) jz += d[i][v]; else if (L::cz(i) < 0) jz -= d[i][v];
    }
    const R rho = R(1) + drho;
    const R ir = recip(rho);
    const R ux = jx * ir + R(0.5) * gx, uy = jy * ir + R(0.5) * gy, uz = jz * ir + R(0.5) * gz;
    const R Gx = rho * gx, Gy = rho * gy, Gz = rho * gz;              // F = rho g
    const R uu = ux * ux + uy * uy + uz * uz;
    const R uF = ux * Gx + uy * Gy + uz * Gz;
    // f*_i = (1-om) d_i + w_i (E_i + O_i): E even, O odd in c_i
    //   E = om drho - 1.5 om rho u.u - 3 cf u.F + cu (4.5 om rho cu + 9 cf cF)
    //   O = 3 (om rho cu + cf cF)
    const R K0 = om * drho - R(1.5) * om * rho * uu - R(3) * cf * uF;
    const R A = R(4.5) * om * rho, B = om * rho, C9 = R(9) * cf;
    d[0][v] = om1 * d[0][v] + (R)L::w(0) * K0;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int o = L::opp(i);
      if (o < i) continue;
      const R cu = L::cx(i) * ux + L::cy(i) * uy + L::cz(i) * uz;
      const R cF = L::cx(i) * Gx + L::cy(i) * Gy + L::cz(i) * Gz;
      const R cfF = cf * cF;
      const R E = K0 + cu * (A * cu + C9 * cF);
      const R Od = R(3) * (B * cu + cfF);
      const R w = (R)L::w(i);
      const R pe = w * E, po = w * Od;
      const R fi = om1 * d[i][v] + (pe + po);
      const R fo = om1 * d[o][v] + (pe - po);
      d[i][v] = fi;
      d[o][v] = fo;
    }
    mr[v] = rho; mu[0][v] = ux; mu[1][v] = uy; mu[2][v] = uz;
  }
  // random bits of the binary16 stochastic rounding: per node, population, step
  const uint32_t hb = sizeof(S) == 2 ? mix32((uint32_t)(row + x0) * 0x9E3779B1u ^ (st.n * 0x632BE5ABu + rd.rep)) : 0u;
#pragma unroll
  for (int i = 0; i < Q; ++i)
    Row<S, V>::st(dst + i * N + row + x0, d[i], scale, hb ? (mix32(hb + 0x27D4EB2Fu * (uint32_t)i) | 1u) : 0u);

  // rho, u: every node on request; otherwise the columns the coupling reads
  // (x0-1 .. x0+cw and x1-cw-1 .. x1, periodic in x).
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int x = x0 + v;
    bool want = st.write_moments;
    if (!want && rd.has_region) {
      int da = x - (rd.x0 - 1), db = x - (rd.x1 - rd.cw - 1);
      da = da < 0 ? da + nx : (da >= nx ? da - nx : da);
      db = db < 0 ? db + nx : (db >= nx ? db - nx : db);
      want = da <= rd.cw + 1 || db <= rd.cw + 1;
    }
    if (want) {
      R* rh = (R*)rd.rho;
      R* uv = (R*)rd.u;
      rh[row + x] = mr[v];
      uv[row + x] = mu[0][v];
      uv[N + row + x] = mu[1][v];
      uv[2 * N + row + x] = mu[2][v];
    }
  }
}


template <int Q, typename S, int V>
__global__ void __launch_bounds__(128, 5) lb_pull(const RepDev* __restrict__ reps, const int4* __restrict__ bmap,
                                               int nwork, const StepInfo* __restrict__ si, int k, int nrep) {
  __shared__ RepDev rd;
  __shared__ StepInfo st;
  for_each_item(bmap, nwork, reps, si, k, nrep, rd, st, [&](const int4 bm) { lb_row<Q, S, V>(rd, st, bm); });
}

template <int Q, typename S, int V>
static cudaError_t go_lb(const Launch& L, const int4* bmap, int nwork, int k) {
  if (nwork == 0) return cudaSuccess;
  static const int g = grid_cap(grid_for(lb_pull<Q, S, V>, 128, 1 << 30));
  lb_pull<Q, S, V><<<g < nwork ? g : nwork, 128, 0, L.stream>>>(L.reps, bmap, nwork, L.si, k, L.nrep);
  return cudaGetLastError();
}

// Nodes per thread: 4 for D2Q9 rows, 2 for D3Q19 rows (19 populations per
// node), 1 in binary64 or when the row length is not a multiple.
int lb_vector_width(int q, int prec, int nx) {
  if (prec == P_FP64) return 1;
  const int v = q == 9 ? 4 : 2;
  return nx % v == 0 ? v : 1;
}

cudaError_t launch_lb(int q, int prec, int vec, const Launch& L, const int4* bmap, int nblocks, int k) {
  if (q == 9) {
    if (prec == P_FP64) return go_lb<9, double, 1>(L, bmap, nblocks, k);
    if (prec == P_FP32) return vec == 4 ? go_lb<9, float, 4>(L, bmap, nblocks, k) : go_lb<9, float, 1>(L, bmap, nblocks, k);
    return vec == 4 ? go_lb<9, __half, 4>(L, bmap, nblocks, k) : go_lb<9, __half, 1>(L, bmap, nblocks, k);
  }
  if (prec == P_FP64) return go_lb<19, double, 1>(L, bmap, nblocks, k);
  if (prec == P_FP32) return vec == 2 ? go_lb<19, float, 2>(L, bmap, nblocks, k) : go_lb<19, float, 1>(L, bmap, nblocks, k);
  return vec == 2 ? go_lb<19, __half, 2>(L, bmap, nblocks, k) : go_lb<19, __half, 1>(L, bmap, nblocks, k);
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
