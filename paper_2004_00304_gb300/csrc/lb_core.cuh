// lb_core.cuh -- the per-row LB update (a1) shared by the per-step lb_pull
// kernel (lb.cu) and the persistent step kernel (mpcd.cu).  The same launch
// carries the collision-cell table of the previous step and its imposition
// (cell_core.cuh).
#pragma once
#include "cell_core.cuh"

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
    const float4 t = ld_hint(reinterpret_cast<const float4*>(p), l2_stream());
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
    t.y = sr_half(v[1] * sc, h ? sr_next(h) : 0u);
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
    const uint32_t h1 = h ? sr_next(h) : 0u, h2 = h ? sr_next(h1) : 0u, h3 = h ? sr_next(h2) : 0u;
    a.x = sr_half(v[0] * sc, h);
    a.y = sr_half(v[1] * sc, h1);
    b.x = sr_half(v[2] * sc, h2);
    b.y = sr_half(v[3] * sc, h3);
    uint2 t;
    t.x = *reinterpret_cast<const uint32_t*>(&a);
    t.y = *reinterpret_cast<const uint32_t*>(&b);
    *reinterpret_cast<uint2*>(p) = t;
  }
};

__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// a8 of step m on inner-buffer node b (LB node index `node`, LB density rl of
// this update): the window takes frame m (sampled by the particle pass of
// step m), and with feedback = 1 the node's post-collision populations become
// f_eq(rl, u_bar) (Eq. 2) with the window mean u_bar, written over the BGK
// values its thread has stored; nothing is imposed from the window of step 0.
// With the learned closure (feedback = 2) u_bar is the latest prediction
// (cl_u), from the update after the first evaluation on.
template <int Q, typename S>
__device__ __noinline__ void a8_node(const RepDev& rd, uint32_t m, long long b, int node, typename Store<S>::R rl) {
  using L = Lattice<Q>;
  using R = typename Store<S>::R;
  double W4[4];
  window_sums(rd, m, b, true, W4);
  R rb, ub[3];
  const R M = window_mean<L::D, R>(rd, m, W4, rb, ub);
  const bool net = rd.feedback == 2 && rd.cl_imp && m >= (uint32_t)rd.cl_first;
  if (net) {
    ub[0] = (R)rd.cl_u[2 * b];
    ub[1] = (R)rd.cl_u[2 * b + 1];
    ub[2] = R(0);
  }
  if (!((rd.feedback == 1 && m >= 1u && M > R(0)) || net)) return;
  S* dst = (S*)rd.f[((m + 1u) & 1) ^ 1];
  const R uu = ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const R cu = L::cx(i) * ub[0] + L::cy(i) * ub[1] + L::cz(i) * ub[2];
    const R dev = (R)L::w(i) * ((rl - R(1)) + rl * (R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu));
    Store<S>::st(dst + i * rd.nnode + node, dev, rd.fp16_scale,
                 sizeof(S) == 2 ? (mix32((uint32_t)node * 19u + (uint32_t)i + (m + 1u) * 0x632BE5ABu) | 1u) : 0u);
  }
}

// Collision (BGK + Guo source, Eq. 1-2) of V consecutive nodes x0.. of the
// row (y, z) starting at node index `row`, whose arrived populations are
// d[i][v]; the post-collision values go to the other buffer, rho / u where
// requested.  Inner-buffer nodes take a8 of the previous step instead (below).
template <int Q, typename S, int V>
__device__ __forceinline__ void lb_finish(const RepDev& rd, const StepInfo& st, typename Store<S>::R (&d)[Q][V],
                                          int x0, int row, int y, int z) {
  using L = Lattice<Q>;
  using R = typename Store<S>::R;
  const int nx = rd.nx;
  const int N = (int)rd.nnode;
  const float scale = rd.fp16_scale;
  S* dst = (S*)rd.f[(st.n & 1) ^ 1];
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
  // one stream of rounding words per thread, V words per population (the
  // first from the node's hash, the rest from sr_next)
  uint32_t hs = hb;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (sizeof(S) == 2) hs = sr_next(hs + (uint32_t)V * 0x9E3779B9u);
    Row<S, V>::st(dst + i * N + row + x0, d[i], scale, sizeof(S) == 2 ? hs : 0u);
  }

  // rho, u: every node on request; otherwise the columns the coupling reads
  // (x0-1 .. x0+cw and x1-cw-1 .. x1, periodic in x), or for a near-wall strip
  // the rows y1-cw-1 .. y1.
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int x = x0 + v;
    bool want = st.write_moments || (rd.strip && y >= rd.y1 - rd.cw - 1 && y <= rd.y1);
    if (!want && rd.has_region && !rd.strip) {
      int da = x - (rd.x0 - 1), db = x - (rd.x1 - rd.cw - 1);
      da = da < 0 ? da + nx : (da >= nx ? da - nx : da);
      db = db < 0 ? db + nx : (db >= nx ? db - nx : db);
      want = da <= rd.cw + 1 || db <= rd.cw + 1;
    }
    if (want) {
      R* rh = rho_of<R>(rd, st.n);
      R* uv = u_of<R>(rd, st.n);
      rh[row + x] = mr[v];
      uv[row + x] = mu[0][v];
      uv[N + row + x] = mu[1][v];
      uv[2 * N + row + x] = mu[2][v];
    }
  }
  // a8 of step m = n - 1 on the inner-buffer nodes (a few lanes of a few
  // rows; after the stores above, in a function of its own so that it does
  // not add to the row's register allocation), unless a8 items of a launch
  // after this one apply it (the overlapped form, below)
  if (rd.nbuf > 0 && st.n >= 1u && st.lb_a8) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const long long b = inner_index(rd, x0 + v, y, z);
      if (b >= 0 && x0 + v >= rd.own_lo && x0 + v < rd.own_hi) a8_node<Q, S>(rd, st.n - 1u, b, row + x0 + v, mr[v]);
    }
  }
}

// LB column, row and z of inner-buffer node b (the inverse of inner_index);
// for a piece of a divided region the column may lie outside the lattice.
__device__ __forceinline__ void inner_xyz(const RepDev& rd, long long b, int& x, int& y, int& z) {
  if (rd.strip) {
    x = (int)(b % rd.nx);
    const long long t = b / rd.nx;
    z = (int)(t % rd.nz);
    y = rd.y1 - 1 - rd.n_out - (int)(t / rd.nz);
    return;
  }
  y = 1 + (int)(b % (rd.ny - 2));
  const long long t = b / (rd.ny - 2);
  z = (int)(t % rd.nz);
  const long long t2 = t / rd.nz;
  const int col = (int)(t2 % rd.n_in), side = (int)(t2 / rd.n_in);
  x = side ? rd.x1 - 1 - rd.n_out - col : rd.x0 + rd.n_out + col;
}

// a8 of step m as a work item of its own (the overlapped form, where the LB
// update of step m + 1 runs beside the particle pass of step m): inner-buffer
// node b takes frame m into the window and, with feedback, gets f_eq(rho_LB,
// u_bar) over the post-collision populations the update of step m + 1 wrote,
// rho_LB being that update's density of the node.  The same arithmetic as the
// in-launch form.  A piece of a divided region imposes on the columns it owns
// only.
template <int Q, typename S>
__device__ __forceinline__ void a8_item(const RepDev& rd, uint32_t m, long long b) {
  using R = typename Store<S>::R;
  if (b >= rd.nbuf) return;
  int x, y, z;
  inner_xyz(rd, b, x, y, z);
  if (x < rd.own_lo || x >= rd.own_hi) return;
  const long long node = x + (long long)rd.nx * (y + (long long)rd.ny * z);
  a8_node<Q, S>(rd, m, b, (int)node, rho_of<R>(rd, m + 1u)[node]);
}

// One thread owns V consecutive nodes x0 .. x0+V-1 of one row (y, z).  A
// work item (replica, tile, y, z | k << 24) is one block-wide tile of a row
// (k = 0), or, for rows of tpr = nx / V < blockDim threads (tpr a power of
// two dividing blockDim), the 2^k = blockDim / tpr rows y, y + 1, ... with
// tpr threads each, so that narrow replicas do not leave most of a block
// idle.
// A work item other than an LB row (bm.y < 0), of block b = -1 - bm.y: the
// strip cells of the closure frame (bm.z = -1), the collision-cell table
// (bm.z = 0, blockDim CPT cells) or the a8 imposition of the inner-buffer
// nodes (bm.z = -2).  bm.w = 0: of step n - 1, in the LB launch of step n;
// bm.w = 1: of step n, in a launch after the particle pass of step n (the
// overlapped form).
template <int Q, typename S>
__device__ __forceinline__ void lb_item(const RepDev& rd, const StepInfo& st, const int4 bm) {
  const long long blk = -1 - bm.y;
  const bool now = bm.w != 0;
  const uint32_t m = now ? st.n : st.n - 1u;
  if (bm.z == -1) {
    if (now || st.n >= 1u) closure_fold_item(rd, m, blk * blockDim.x, 32LL * rd.Hy);
  } else if (bm.z == -2) {
    a8_item<Q, S>(rd, st.n, blk * blockDim.x + threadIdx.x);
  } else if (now || st.cells) {
    cell_table_item<Q, S>(rd, m, (now ? st.shift_f[1] : st.prev_f[1]) > 0.0f, blk * blockDim.x * CPT, rd.ncell);
  }
}

template <int Q, typename S, int V>
__device__ __forceinline__ void lb_row(const RepDev& rd, const StepInfo& st, const int4 bm) {
  using L = Lattice<Q>;
  using R = typename Store<S>::R;
  if (bm.y < 0) {
    lb_item<Q, S>(rd, st, bm);
    return;
  }
  const int nx = rd.nx, ny = rd.ny, nz = rd.nz;
  const int z = bm.w & 0xFFFFFF, rlog = bm.w >> 24;
  const int tpr = nx / V;
  const int lt = rlog ? __ffs(tpr) - 1 : 0;             // tpr = 2^lt when rows share the block
  const int tx = rlog ? (int)threadIdx.x & (tpr - 1) : bm.y * (int)blockDim.x + (int)threadIdx.x;
  const int yr = bm.z + (rlog ? (int)threadIdx.x >> lt : 0);
  const bool row_ok = yr < ny - 1;
  const int y = row_ok ? yr : ny - 2;                    // rows past the last fluid row load a valid one
  const bool active = tx < tpr && row_ok;
  const int lane = threadIdx.x & 31;
  const int x0 = tx * V;
  const int par = st.n & 1;
  // plain (coherent) loads: in the persistent kernel this buffer is written
  // by other blocks of the same launch between grid barriers
  const S* src = (const S*)rd.f[par];
  const int N = (int)rd.nnode;
  const int row = nx * (y + ny * z);
  const float inv = rd.fp16_inv;

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
  // phase 2: shift the rows with cx != 0 by one node through the neighbour
  // lanes.  Every lane takes part in every shuffle: the lanes of one warp may
  // hold different rows (multi-row items), of which some read a bounce-back
  // row that is not shifted.
  if (V > 1) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (L::cx(i) == 0) continue;
      const int sy = y - L::cy(i);
      const bool shift = !((sy == 0) | (sy == ny - 1));
      if (L::cx(i) > 0) {                    // source x - 1: previous lane's last node
        R prev = __shfl_up_sync(0xFFFFFFFFu, d[i][V - 1], 1);
        if (lane == 0 || tx == 0) prev = edge[i];
        if (shift) {
#pragma unroll
          for (int v = V - 1; v > 0; --v) d[i][v] = d[i][v - 1];
          d[i][0] = prev;
        }
      } else {                               // source x + 1: next lane's first node
        R next = __shfl_down_sync(0xFFFFFFFFu, d[i][0], 1);
        if (lane == 31 || tx + 1 >= tpr) next = edge[i];
        if (shift) {
#pragma unroll
          for (int v = 0; v < V - 1; ++v) d[i][v] = d[i][v + 1];
          d[i][V - 1] = next;
        }
      }
    }
  }
  if (!active) return;
  lb_finish<Q, S, V>(rd, st, d, x0, row, y, z);
}

}  // namespace lbm
