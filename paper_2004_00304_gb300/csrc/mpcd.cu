// mpcd.cu -- the MPCD half of the coupled step and both coupling directions.
//
// Per step n the handle runs   lb_pull(n) -> particle_pass(n):
//   particle_pass  one thread per particle, structure-of-arrays state
//                  (packed integer home cell, offsets, velocities):
//                    a7(n-1)  rotate v about the v_cm of its collision cell
//                             of step n-1 (table written by cell_pass(n-1)),
//                    a2+a3    outer-buffer particles: v = u_fine + sqrt(kT/m) xi,
//                             u_fine by bilinear/trilinear interpolation of
//                             the LB velocity (Algorithms 1-2, Sec. 2.3),
//                    a4       kick-drift streaming (Eq. 3), bounce-back walls,
//                             periodic wrap in the region,
//                    a6       inner-buffer particles add m, m v to the frame
//                             (with the learned closure, strip particles add
//                             1, v to their fine cell's closure frame),
//                    a5       binning under the step's random shift and a
//                             warp-aggregated reduction (__match_any_sync
//                             groups, one atomic per group and cell);
//   lb_pull(n + 1) carries the cell half of a7(n) (v_cm with virtual wall
//                  particles, rotation draw of Eq. 4, accumulators cleared)
//                  as extra work items, and a8(n) (window-mean MPCD velocity
//                  of the inner buffer -> f_eq(rho_LB, u_bar)) as the
//                  collision of the inner-buffer nodes (cell_core.cuh).
// The collision of the last step is applied lazily (flush) before particle
// state is read out, so the visible state is always post-collision.
// Every graph chunk starts with a counting sort of the particles by home cell
// (sort_count -> sort_scan_tiles -> sort_scan_top -> sort_scatter into the
// *_alt arrays; the chunk's first particle_pass reads them back), which keeps
// the particles of a warp in a few neighbouring cells so that the warp-level
// aggregation and the cell-table reads stay local.
//
// Streaming and binning use the add/mul helpers below: in binary64 they are
// the non-contractible __dadd_rn/__dmul_rn, so FP64 runs bin every particle
// into the same cell as a binary64 reference would; in binary32 the compiler
// may fuse them.
#include <type_traits>

#include "lb_core.cuh"

namespace lbm {

template <typename R> struct Num;
template <> struct Num<double> { static constexpr double one_minus = 1.0 - 1.0 / 9007199254740992.0; };
template <> struct Num<float> { static constexpr float one_minus = 1.0f - 1.0f / 16777216.0f; };

__device__ __forceinline__ int wrap(int a, int m) { a %= m; return a < 0 ? a + m : a; }

__device__ __forceinline__ double xadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double xsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double xmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float xadd(float a, float b) { return a + b; }
__device__ __forceinline__ float xsub(float a, float b) { return a - b; }
__device__ __forceinline__ float xmul(float a, float b) { return a * b; }

// Particle offsets and velocities: in 2D each is one array of interleaved
// (x, y) pairs (one 8- or 16-byte access per particle), in 3D one array per axis.
template <typename R> struct Pair;
template <> struct Pair<float> { using T = float2; };
template <> struct Pair<double> { using T = double2; };
template <int D, typename R> struct PState;
template <typename R> struct PState<2, R> {
  using T2 = typename Pair<R>::T;
  __device__ static void ld(void* const* base, uint32_t j, R* x) {
    T2 t;
    if constexpr (sizeof(R) == 4) t = ld_hint((const float2*)base[0] + j, l2_stream());
    else t = ((const T2*)base[0])[j];
    x[0] = t.x; x[1] = t.y;
  }
  __device__ static void st(void* const* base, uint32_t j, const R* x) {
    T2 t; t.x = x[0]; t.y = x[1];
    if constexpr (sizeof(R) == 4) st_hint((float2*)base[0] + j, t, l2_stream());
    else ((T2*)base[0])[j] = t;
  }
};
template <typename R> struct PState<3, R> {
  __device__ static void ld(void* const* base, uint32_t j, R* x) {
#pragma unroll
    for (int a = 0; a < 3; ++a) x[a] = ((const R*)base[a])[j];
  }
  __device__ static void st(void* const* base, uint32_t j, const R* x) {
#pragma unroll
    for (int a = 0; a < 3; ++a) ((R*)base[a])[j] = x[a];
  }
};

// ---------------------------------------------------------------------------
// prep: one block; per (step k of the chunk, replica) the global step index,
// the random shift of that step and of the previous one, and whether the
// previous collision is still pending.  overlap: the chunk runs the
// overlapped form (the LB update of step n + 1 beside the particle pass of
// step n, a launch after both for the table and a8 of step n): only the
// chunk's first LB launch applies a8 of the step before it, and the chunk
// leaves the table of its last step built; its work counters (ctr, one per
// step) start at zero.  The sort, when one ran since the
// last chunk, left d_sorted[r] = 1: the chunk's first step then reads the
// sorted copy, and the flag is cleared for the next chunk.
__global__ void prep_steps(const RepDev* __restrict__ reps, int nrep, int dim, int kcount, int* d_sorted,
                           StepInfo* __restrict__ si, uint32_t* d_step, int* d_pending, int* d_cells,
                           double* d_last_shift, int overlap, int* ctr) {
  const uint32_t n0 = *d_step;
  if (ctr)
    for (int k = threadIdx.x; k < kcount; k += blockDim.x) ctr[k] = 0;
  for (int idx = threadIdx.x; idx < kcount * nrep; idx += blockDim.x) {
    const int k = idx / nrep, r = idx % nrep;
    const RepDev& rd = reps[r];
    StepInfo s;
    s.n = n0 + k;
    s.pending = (k == 0) ? d_pending[r] : 1;
    s.cells = (k == 0) ? d_cells[r] : (rd.has_region ? 1 : 0);
    s.write_moments = (k == kcount - 1);
    s.lb_a8 = overlap ? (k == 0) : 1;
    s.src_alt = (k == 0) && d_sorted[r] && rd.has_region;
    const uint4 w = philox(0u, s.n, rd.rep, TAG_SHIFT, rd.key0, rd.key1);
    s.shift[0] = unit24(w.x);
    s.shift[1] = unit24(w.y);
    s.shift[2] = dim == 3 ? unit24(w.z) : 0.0;
    if (k == 0) {
      for (int a = 0; a < 3; ++a) s.prev[a] = d_last_shift[3 * r + a];
    } else {
      const uint4 p = philox(0u, s.n - 1, rd.rep, TAG_SHIFT, rd.key0, rd.key1);
      s.prev[0] = unit24(p.x);
      s.prev[1] = unit24(p.y);
      s.prev[2] = dim == 3 ? unit24(p.z) : 0.0;
    }
    for (int a = 0; a < 3; ++a) { s.shift_f[a] = (float)s.shift[a]; s.prev_f[a] = (float)s.prev[a]; }
    si[idx] = s;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < nrep; r += blockDim.x) {
    if (d_sorted[r] && reps[r].pooled) reps[r].pool[0] = reps[r].pool[2];   // the sort compacted the pool
    d_sorted[r] = 0;
    const StepInfo& last = si[(kcount - 1) * nrep + r];
    for (int a = 0; a < 3; ++a) d_last_shift[3 * r + a] = last.shift[a];
    d_pending[r] = reps[r].has_region ? 1 : 0;
    d_cells[r] = reps[r].has_region && !overlap ? 1 : 0;
  }
  if (threadIdx.x == 0) *d_step = n0 + kcount;
}

cudaError_t launch_prep(int dim, const Launch& L, StepInfo* si, int kcount, int* d_sorted, uint32_t* d_step,
                        int* d_pending, int* d_cells, double* d_last_shift, int overlap, int* ctr) {
  prep_steps<<<1, 256, 0, L.stream>>>(L.reps, L.nrep, dim, kcount, d_sorted, si, d_step, d_pending, d_cells,
                                      d_last_shift, overlap, ctr);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a5: the collision cell of a particle under shift s: per axis the home
// index plus one when offset + s >= 1 (the sum rounded in storage precision),
// wrapped in x and z.  id = cx + Wx (cy + (Hy+1) cz).
template <int D, typename R>
__device__ __forceinline__ uint32_t collision_cell(const RepDev& rd, int X, int Y, int Z, const R* o,
                                                   const R* s) {
  int cx = X + (xadd(o[0], s[0]) >= R(1) ? 1 : 0);
  if (cx >= rd.Wx) cx -= rd.Wx;
  const int cy = Y + (xadd(o[1], s[1]) >= R(1) ? 1 : 0);
  int cz = 0;
  if (D == 3) {
    cz = Z + (xadd(o[2], s[2]) >= R(1) ? 1 : 0);
    if (cz >= rd.Wz) cz -= rd.Wz;
  }
  return (uint32_t)(cx + rd.Wx * (cy + (rd.Hy + 1) * cz));
}

// a7, particle side: v <- v_cm + R (v - v_cm).  2D: R = rotation by theta
// with sin(theta) stored per cell; 3D: Rodrigues' formula about the cell axis.
// MPCD-AT: v holds the particle's random velocity and the table v_cm minus the
// cell's mean random velocity, so the collision is their sum.
template <int D, typename R>
__device__ __forceinline__ void rotate(const RepDev& rd, uint32_t c, R* v) {
  using T4 = typename Vec4<R>::T;
  const R ca = Cst<R>::cos_a(rd);
  const T4* tab = (const T4*)rd.tab;
  if (rd.collision == 1) {
    const T4 t = tab[D == 2 ? (size_t)c : 2 * (size_t)c];
    v[0] += t.x;
    v[1] += t.y;
    if (D == 3) v[2] += t.z;
    return;
  }
  if (D == 2) {
    const T4 t = tab[c];
    const R wx = v[0] - t.x, wy = v[1] - t.y;
    v[0] = t.x + (ca * wx - t.z * wy);
    v[1] = t.y + (t.z * wx + ca * wy);
  } else {
    const R sa = Cst<R>::sin_a(rd);
    const T4 t0 = tab[2 * (size_t)c], t1 = tab[2 * (size_t)c + 1];
    const R vc[3] = {t0.x, t0.y, t0.z}, n[3] = {t1.x, t1.y, t1.z};
    const R w[3] = {v[0] - vc[0], v[1] - vc[1], v[2] - vc[2]};
    const R cr[3] = {n[1] * w[2] - n[2] * w[1], n[2] * w[0] - n[0] * w[2], n[0] * w[1] - n[1] * w[0]};
    const R nw = n[0] * w[0] + n[1] * w[1] + n[2] * w[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) v[a] = vc[a] + (w[a] * ca + cr[a] * sa + n[a] * nw * (R(1) - ca));
  }
}

// LB velocity at node (x,y,z) with periodic x, z and the wall ghost
// u(0) = -u(1), u(ny-1) = -u(ny-2) that puts u = 0 on the half-way walls.
template <typename R>
__device__ __forceinline__ R u_node(const RepDev& rd, uint32_t n, int a, int x, int y, int z) {
  x = wrap(x, rd.nx);
  z = wrap(z, rd.nz);
  R sgn = R(1);
  if (y <= 0) { y = 1; sgn = R(-1); }
  if (y >= rd.ny - 1) { y = rd.ny - 2; sgn = R(-1); }
  const R* u = u_of<R>(rd, n);
  return sgn * u[a * rd.nnode + x + (long long)rd.nx * (y + (long long)rd.ny * z)];
}

// a2: bilinear (2D) / trilinear (3D) interpolation of the LB velocity, known
// at node centres (the LB update of step n), to the centre of MPCD cell
// (X,Y,Z) (Algorithm 2).  In the
// kernel's precision: for refinement ratios that are powers of two the
// positions and weights are exact in binary32.
template <int D, typename R>
__device__ void u_fine(const RepDev& rd, uint32_t n, int X, int Y, int Z, R* out) {
  const R r = Cst<R>::r(rd);
  const R px = (R)rd.x0 + ((R)X + R(0.5)) / r - R(0.5);
  const R py = R(1) + ((R)Y + R(0.5)) / r - R(0.5);
  const R pz = (D == 3) ? ((R)Z + R(0.5)) / r - R(0.5) : R(0);
  const int i0 = (int)floor(px), j0 = (int)floor(py), k0 = (int)floor(pz);
  const R tx = px - (R)i0, ty = py - (R)j0, tz = pz - (R)k0;
  for (int a = 0; a < D; ++a) {
    R acc = R(0);
    for (int di = 0; di < 2; ++di)
      for (int dj = 0; dj < 2; ++dj)
        for (int dk = 0; dk < (D == 3 ? 2 : 1); ++dk) {
          R wgt = (di ? tx : R(1) - tx) * (dj ? ty : R(1) - ty);
          if (D == 3) wgt *= (dk ? tz : R(1) - tz);
          acc += wgt * u_node<R>(rd, n, a, i0 + di, j0 + dj, k0 + dk);
        }
    out[a] = acc;
  }
}

// a3, Chapman-Enskog form (redraw = 1): the peculiar velocity C of a redrawn
// particle in cell (X,Y,Z) follows f_MB(C; kT/m) (1 + b : zz), z = C / sigma,
// b = pi' / (2 sigma^2), pi' the traceless part of (1 - 1/(2 tau)) Pi_neq / rho
// of the LB node holding the cell, Pi_neq = sum_i (f_i - f_i^eq) c_i c_i over
// the populations after this step's streaming.  Those are pulled again here
// from the buffer the LB step read (its sources, with the half-way
// bounce-back rule), in the storage precision (binary64 or binary32
// deviations).  Acceptance-rejection keyed by (particle id, step, replica,
// TAG_CE + 16 t), as the oracle draws it.
template <int D, typename R>
__device__ __noinline__ void ce_peculiar(const RepDev& rd, const StepInfo& st, int X, int Y, int Z, uint32_t id,
                                         R* C) {
  constexpr int Q = D == 2 ? 9 : 19;
  using L = Lattice<Q>;
  const int x = rd.x0 + X / rd.r, y = 1 + Y / rd.r, z = D == 3 ? Z / rd.r : 0;
  const R* src = (const R*)rd.f[st.n & 1];
  const long long N = rd.nnode, here = x + (long long)rd.nx * (y + (long long)rd.ny * z);
  R drho = R(0), j[3] = {R(0), R(0), R(0)}, P[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int sy = y - L::cy(i);
    R d;
    if (sy == 0 || sy == rd.ny - 1) {
      d = src[L::opp(i) * N + here];
    } else {
      const int sx = wrap(x - L::cx(i), rd.nx), sz = wrap(z - L::cz(i), rd.nz);
      d = src[i * N + sx + (long long)rd.nx * (sy + (long long)rd.ny * sz)];
    }
    drho += d;
    j[0] += L::cx(i) * d; j[1] += L::cy(i) * d; j[2] += L::cz(i) * d;
    P[0] += L::cx(i) * L::cx(i) * d; P[1] += L::cy(i) * L::cy(i) * d; P[2] += L::cz(i) * L::cz(i) * d;
    P[3] += L::cx(i) * L::cy(i) * d; P[4] += L::cx(i) * L::cz(i) * d; P[5] += L::cy(i) * L::cz(i) * d;
  }
  // deviations d_i = f_i - w_i: sum f c c = sum d c c + cs^2 I, and the
  // equilibrium's second moment is rho cs^2 I + rho u u
  const R rho = R(1) + drho, ir = R(1) / rho;
  const R u[3] = {j[0] * ir + R(0.5) * Cst<R>::g(rd, 0), j[1] * ir + R(0.5) * Cst<R>::g(rd, 1),
                  j[2] * ir + R(0.5) * Cst<R>::g(rd, 2)};
  const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
  const R fac = (R(1) - R(0.5) * Cst<R>::omega(rd)) * ir;
  R pi[6];
#pragma unroll
  for (int m = 0; m < 6; ++m)
    pi[m] = fac * (P[m] - (m < 3 ? drho / R(3) : R(0)) - rho * u[ia[m]] * u[ib[m]]);
  const R tr = (pi[0] + pi[1] + (D == 3 ? pi[2] : R(0))) / R(D);
  pi[0] -= tr; pi[1] -= tr;
  if (D == 3) pi[2] -= tr; else pi[2] = pi[4] = pi[5] = R(0);
  const R sg = Cst<R>::sig(rd), i2s = R(1) / (R(2) * sg * sg);
  R bmax = R(0);
#pragma unroll
  for (int m = 0; m < 6; ++m) { pi[m] *= i2s; bmax = fmax(bmax, fabs(pi[m])); }   // pi now holds b
  const R A = R(1) + R(30) * bmax;
  R zz[3] = {R(0), R(0), R(0)};
  for (int t = 0; t < CE_TRIES; ++t) {
    const uint4 w = philox(id, st.n, rd.rep, TAG_CE + 16u * (uint32_t)t, rd.key0, rd.key1);
    R z3, U;
    normal_pair(w.x, w.y, zz[0], zz[1]);
    if (D == 3) {
      normal_pair(w.z, w.w, zz[2], z3);
      const uint4 w2 = philox(id, st.n, rd.rep, TAG_CE + 1u + 16u * (uint32_t)t, rd.key0, rd.key1);
      U = sizeof(R) == 8 ? (R)unit24(w2.x) : (R)unit24f(w2.x);
    } else {
      U = sizeof(R) == 8 ? (R)unit24(w.z) : (R)unit24f(w.z);
    }
    const R q = pi[0] * zz[0] * zz[0] + pi[1] * zz[1] * zz[1] + R(2) * pi[3] * zz[0] * zz[1] +
                (D == 3 ? pi[2] * zz[2] * zz[2] + R(2) * pi[4] * zz[0] * zz[2] + R(2) * pi[5] * zz[1] * zz[2] : R(0));
    if (A * U <= R(1) + q) break;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) C[a] = sg * zz[a];
}

// a4: kick (v += g) then drift r += v dt (Eq. 3, dt = 1, r in cell units so the
// displacement is v r); a wall crossing reverses v and retraces the rest of
// the step; x (and z) wrap periodically in the region.
template <int D, typename R>
__device__ __forceinline__ void stream(const RepDev& rd, int& X, int& Y, int& Z, R* o, R* v) {
  v[0] = xadd(v[0], Cst<R>::g(rd, 0));
  v[1] = xadd(v[1], Cst<R>::g(rd, 1));
  if (D == 3) v[2] = xadd(v[2], Cst<R>::g(rd, 2));
  const R rr = Cst<R>::r(rd);
  const R dx = xmul(v[0], rr), dy = xmul(v[1], rr), dz = (D == 3) ? xmul(v[2], rr) : R(0);
  const R ty = xadd(o[1], dy);
  int ky = (ty >= R(1) ? 1 : 0) - (ty < R(0) ? 1 : 0);      // floor(ty) for ty in [-1, 2)
  if (ty < R(-1) || ty >= R(2)) ky = (int)floor(ty);
  const int nyc = Y + ky;
  R dxe = dx, dze = dz;
  if (nyc < 0 || nyc >= rd.Hy) {
    const R Lw = (nyc < 0) ? (R)(-Y) : (R)(rd.Hy - Y);   // wall, local units
    const R tr = xsub(Lw, xsub(ty, Lw));                 // mirrored end point
    if (rd.strip && nyc >= rd.Hy) {                      // top edge of a near-wall strip: specular
      v[1] = -v[1];
    } else {
      const R ts = (Lw - o[1]) / dy;                     // fraction before the hit
#pragma unroll
      for (int a = 0; a < D; ++a) v[a] = -v[a];
      dxe = xsub(xmul(dx, ts), xmul(dx, xsub(R(1), ts)));
      dze = xsub(xmul(dz, ts), xmul(dz, xsub(R(1), ts)));
    }
    const int kr = (int)floor(tr);
    Y += kr;
    o[1] = xsub(tr, (R)kr);
    if (Y >= rd.Hy) { Y = rd.Hy - 1; o[1] = Num<R>::one_minus; }
    if (Y < 0) { Y = 0; o[1] = R(0); }
  } else {
    Y = nyc;
    o[1] = xsub(ty, (R)ky);
  }
  if (o[1] >= R(1)) {
    o[1] = xsub(o[1], R(1));
    Y += 1;
    if (Y >= rd.Hy) { Y = rd.Hy - 1; o[1] = Num<R>::one_minus; }
  }
  const R tx = xadd(o[0], dxe);
  int kx = (tx >= R(1) ? 1 : 0) - (tx < R(0) ? 1 : 0);
  if (tx < R(-1) || tx >= R(2)) kx = (int)floor(tx);
  o[0] = xsub(tx, (R)kx);
  if (o[0] >= R(1)) { o[0] = xsub(o[0], R(1)); kx += 1; }
  X += kx;
  if (X < 0 || X >= rd.Wx) X = wrap(X, rd.Wx);
  if (D == 3) {
    const R tz = xadd(o[2], dze);
    int kz = (tz >= R(1) ? 1 : 0) - (tz < R(0) ? 1 : 0);
    if (tz < R(-1) || tz >= R(2)) kz = (int)floor(tz);
    o[2] = xsub(tz, (R)kz);
    if (o[2] >= R(1)) { o[2] = xsub(o[2], R(1)); kz += 1; }
    Z += kz;
    if (Z < 0 || Z >= rd.Wz) Z = wrap(Z, rd.Wz);
  }
}

// One work item = PP_ITEM consecutive particles; thread t handles particles
// t, t + 256, ... (PPT of them) of the item, so that every round of the warp
// covers 32 consecutive particles.  All state loads of the thread's particles
// are issued first, then their cell-table loads, before any arithmetic, so
// they are in flight together instead of forming one dependent chain.
// shared memory of particle_pass: staging of the warp-aggregated reduction
// read-only (L1-cached) load of a cell-table entry: particles of one block are
// sorted by home cell, so neighbouring threads read the same entries
template <typename T> __device__ __forceinline__ T ld_ro(const T* p) {
  if constexpr (std::is_same<T, float4>::value) return __ldg(p);
  else return *p;
}

template <int D, typename R> struct PassShared {
  R sv[D][256];
};

// a7 of step n-1, particle side, from the entries of the particle's collision
// cell in the table (2D: t0 = {v_cm, sin theta, n}; 3D: t0 = {v_cm, n},
// t1 = {axis, 0}): v <- v_cm + R (v - v_cm) (Eq. 4), rotation by theta in 2D,
// Rodrigues' formula about the axis in 3D.  MPCD-AT: v holds the particle's
// random velocity and t0 v_cm - <v_ran>, so the collision is their sum.
template <int D, typename R, bool AT, typename T4>
__device__ __forceinline__ void collide_from_table(const RepDev& rd, const T4& t0, const T4& t1, R* v) {
  const R ca = Cst<R>::cos_a(rd), sa = Cst<R>::sin_a(rd);
  if (AT) {
    v[0] += t0.x;
    v[1] += t0.y;
    if (D == 3) v[2] += t0.z;
  } else if (D == 2) {
    const R wx = v[0] - t0.x, wy = v[1] - t0.y;
    v[0] = t0.x + (ca * wx - t0.z * wy);
    v[1] = t0.y + (t0.z * wx + ca * wy);
  } else {
    const R vc[3] = {t0.x, t0.y, t0.z}, n[3] = {t1.x, t1.y, t1.z};
    const R w[3] = {v[0] - vc[0], v[1] - vc[1], v[2] - vc[2]};
    const R cr[3] = {n[1] * w[2] - n[2] * w[1], n[2] * w[0] - n[0] * w[2], n[0] * w[1] - n[1] * w[0]};
    const R nw = n[0] * w[0] + n[1] * w[1] + n[2] * w[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) v[a] = vc[a] + (w[a] * ca + cr[a] * sa + n[a] * nw * (R(1) - ca));
  }
}

constexpr uint32_t NO_CELL = 0xFFFFFFFFu;   // a particle that adds nothing to the cell sums

// One particle j of step n after its collision of step n-1: a3' removal
// (density resampling), a2 + a3 redraw in the outer buffer, a4 streaming, a6
// inner-buffer sampling and the closure strips, a5 binning under this step's
// shift, and the stores of its new state (MPCD-AT: with the random velocity of
// this step's collision in place of v).  alt: the state was read from the
// sorted copy; fresh: created by this step's spawn.  Returns the collision
// cell, or NO_CELL for a removed particle.  v keeps what the cell sums take
// (with SRD the velocity of the sampling instant, which add_strip_sums uses).
template <int D, typename R, bool RS, bool AT, bool CE>
__device__ __forceinline__ uint32_t move_particle(const RepDev& rd, const StepInfo& st, uint32_t j, bool alt,
                                                  bool fresh, int& X, int& Y, int& Z, R* o, R* v) {
  const bool outer = X < rd.xo_lo || X >= rd.xo_hi || Y >= rd.yo;
  if (RS && rd.resample && outer && !fresh) {   // a3': replaced by this step's spawn
    rd.home[j] = HOME_DEAD;
    return NO_CELL;
  }
  // a2 + a3: Maxwellian redraw in the outer buffer columns
  if (!(RS && rd.resample) && outer) {
    R uf[3] = {R(0), R(0), R(0)};
    u_fine<D, R>(rd, st.n, X, Y, Z, uf);
    const uint32_t id = (alt ? rd.pid_alt : rd.pid)[j];
    if (CE && rd.redraw == 1) {
      R C[3];
      ce_peculiar<D, R>(rd, st, X, Y, Z, id, C);
      v[0] = uf[0] + C[0];
      v[1] = uf[1] + C[1];
      if (D == 3) v[2] = uf[2] + C[2];
    } else {
      const uint4 w = philox(id, st.n, rd.rep, TAG_RESAMPLE, rd.key0, rd.key1);
      R z0, z1, z2, z3;
      normal_pair(w.x, w.y, z0, z1);
      normal_pair(w.z, w.w, z2, z3);
      const R sg = Cst<R>::sig(rd);
      v[0] = uf[0] + sg * z0;
      v[1] = uf[1] + sg * z1;
      if (D == 3) v[2] = uf[2] + sg * z2;
    }
  }
  if (RS && fresh) rd.pid[j] = PID_SPAWNED;
  else if (alt) rd.pid[j] = rd.pid_alt[j];
  // a4
  stream<D, R>(rd, X, Y, Z, o, v);
  // a6: inner-buffer sample (unshifted cells), binary64 atomics
  const bool left = X >= rd.xi_lo0 && X < rd.xi_hi0, right = X >= rd.xi_lo1 && X < rd.xi_hi1;
  const bool row_in = Y >= rd.yi_lo && Y < rd.yi_hi;   // inner rows of a near-wall strip
  if (left || right || row_in) {
    const int xn = X / rd.r, wcols = rd.x1 - rd.x0;
    const int zl = (D == 3) ? Z / rd.r : 0;
    long long b;
    if (row_in) {   // b = (row nz + z) nx + x, row counted down from the buffer's top
      const int row = rd.y1 - 2 - rd.n_out - Y / rd.r;
      b = ((long long)row * rd.nz + zl) * rd.nx + xn;
    } else {
      const int col = left ? xn - rd.n_out : wcols - 1 - rd.n_out - xn;
      b = (((long long)(right ? 1 : 0) * rd.n_in + col) * rd.nz + zl) * (rd.ny - 2) + Y / rd.r;
    }
    double* fr = rd.frame + 4 * b;
    atomicAdd(fr, rd.mass);
#pragma unroll
    for (int a = 0; a < D; ++a) atomicAdd(fr + 1 + a, rd.mass * (double)v[a]);
  }
  // learned-closure strips (feedback = 2), same instant as a6: with MPCD-AT
  // (whose v is replaced below) count and momentum per strip cell here; with
  // SRD the caller sums them per warp (add_strip_sums)
  if (D == 2 && AT && rd.cl_on) {
    const int xs = X < 16 ? X : rd.Wx - 1 - X;
    if (xs < 16) {
      const long long ncl = 32LL * rd.Hy;
      double* fr = rd.cframe + 4 * ((st.n & 1) * ncl + ((long long)(X < 16 ? 0 : 1) * rd.Hy + Y) * 16 + xs);
      atomicAdd(fr, 1.0);
      atomicAdd(fr + 1, (double)v[0]);
      atomicAdd(fr + 2, (double)v[1]);
    }
  }
  // a5: binning under this step's shift
  const uint32_t cid = collision_cell<D, R>(rd, X, Y, Z, o, Cst<R>::shift(st));
  st_hint(rd.home + j, HomePack<D>::pack(X, Y, Z), l2_stream());
  PState<D, R>::st(rd.off, j, o);
  if (AT) {
    // a7 (MPCD-AT), first half: v_ran from Philox(id, n, replica, TAG_AT)
    const uint4 w = philox((alt ? rd.pid_alt : rd.pid)[j], st.n, rd.rep, TAG_AT, rd.key0, rd.key1);
    R z[4];
    normal_pair(w.x, w.y, z[0], z[1]);
    if (D == 3) normal_pair(w.z, w.w, z[2], z[3]);
    const R sg = Cst<R>::sig(rd);
    R xi[3] = {sg * z[0], sg * z[1], D == 3 ? sg * z[2] : R(0)};
    PState<D, R>::st(rd.vel, j, xi);
#pragma unroll
    for (int a = 0; a < D; ++a) v[a] -= xi[a];
  } else {
    PState<D, R>::st(rd.vel, j, v);
  }
  return cid;
}

// Cell sums of the thread's PPT particles (cid[p] = NO_CELL adds nothing).
// Binary32: one vector atomic {n, sum v} per group of lanes; lanes are first
// merged with their xor-1 and then xor-2 neighbours when they share the
// collision cell (particles are sorted by home cell, so neighbours often do).
// The merge removes a part of the atomics for a few shuffles, where the full
// warp aggregation below cost as much as it saved.  Binary64: warp-aggregated
// reduction, one round per particle slot: lanes sharing a collision cell are
// summed by their lowest lane, which issues one atomic per accumulator.
template <int D, typename R>
__device__ __forceinline__ void add_cell_sums(const RepDev& rd, const uint32_t (&cid)[PPT], R (&v)[PPT][3],
                                              PassShared<D, R>& red) {
  if (sizeof(R) == 4) {
    // a lane with nothing to add (inactive, or merged into its partner) holds
    // the cell id NO_CELL, which matches no partner; in 2D the fourth
    // component is zero and is not exchanged
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
      uint32_t c = cid[p];
      float4 a = make_float4(1.0f, (float)v[p][0], (float)v[p][1], D == 3 ? (float)v[p][D - 1] : 0.0f);
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int m = 1 << r;
        const uint32_t co = __shfl_xor_sync(0xFFFFFFFFu, c, m);
        const float ax = __shfl_xor_sync(0xFFFFFFFFu, a.x, m), ay = __shfl_xor_sync(0xFFFFFFFFu, a.y, m);
        const float az = __shfl_xor_sync(0xFFFFFFFFu, a.z, m);
        const float aw = D == 3 ? __shfl_xor_sync(0xFFFFFFFFu, a.w, m) : 0.0f;
        if (c != NO_CELL && co == c) {
          if ((lane & m) == 0) { a.x += ax; a.y += ay; a.z += az; if (D == 3) a.w += aw; } else c = NO_CELL;
        }
      }
      if (c != NO_CELL) atomicAdd(rd.acc4 + c, a);
    }
    return;
  }
  const int lane = threadIdx.x & 31, wbase = threadIdx.x & ~31;
#pragma unroll
  for (int p = 0; p < PPT; ++p) {
    const unsigned grp = __match_any_sync(0xFFFFFFFFu, cid[p]);
    __syncwarp();
#pragma unroll
    for (int a = 0; a < D; ++a) red.sv[a][threadIdx.x] = v[p][a];
    __syncwarp();
    if (cid[p] != NO_CELL && lane == __ffs(grp) - 1) {
      R acc[D];
#pragma unroll
      for (int a = 0; a < D; ++a) acc[a] = R(0);
      unsigned m = grp;
      while (m) {
        const int l = __ffs(m) - 1;
        m &= m - 1;
#pragma unroll
        for (int a = 0; a < D; ++a) acc[a] += red.sv[a][wbase + l];
      }
      if (sizeof(R) == 4) {
        float4 g4;
        g4.x = (float)__popc(grp);
        g4.y = (float)acc[0];
        g4.z = (float)acc[1];
        g4.w = D == 3 ? (float)acc[D - 1] : 0.0f;
        atomicAdd(rd.acc4 + cid[p], g4);
      } else {
        atomicAdd(rd.acc_n + cid[p], (uint32_t)__popc(grp));
#pragma unroll
        for (int a = 0; a < D; ++a) atomicAdd((R*)rd.acc_v[a] + cid[p], acc[a]);
      }
    }
  }
}

// Learned-closure strip frame (feedback = 2, SRD): count and momentum per
// strip cell (the 16 fine columns at each x-edge of the region) of the moved
// particles (home X, Y after streaming, velocity v of the sampling instant;
// cid NO_CELL: nothing to add), binary64 atomics into half n & 1.  Particles
// are sorted by home cell and strip cells are home cells, so lanes are first
// merged with their xor-1 and xor-2 neighbours of the same cell; only warps
// holding a strip particle (an eighth of them on the benchmark channels) take
// this path.
template <typename R>
__device__ __forceinline__ void add_strip_sums(const RepDev& rd, const StepInfo& st, const uint32_t (&cid)[PPT],
                                               const int (&X)[PPT], const int (&Y)[PPT], const R (&v)[PPT][3]) {
  const long long ncl = 32LL * rd.Hy;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int p = 0; p < PPT; ++p) {
    const int xs = X[p] < 16 ? X[p] : rd.Wx - 1 - X[p];
    int c = (cid[p] != NO_CELL && xs < 16) ? ((X[p] < 16 ? 0 : 1) * rd.Hy + Y[p]) * 16 + xs : -1;
    if (!__any_sync(0xFFFFFFFFu, c >= 0)) continue;
    double a0 = c >= 0 ? 1.0 : 0.0, a1 = (double)v[p][0], a2 = (double)v[p][1];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int m = 1 << r;
      const int co = __shfl_xor_sync(0xFFFFFFFFu, c, m);
      const double b0 = __shfl_xor_sync(0xFFFFFFFFu, a0, m), b1 = __shfl_xor_sync(0xFFFFFFFFu, a1, m);
      const double b2 = __shfl_xor_sync(0xFFFFFFFFu, a2, m);
      if (c >= 0 && co == c) {
        if ((lane & m) == 0) { a0 += b0; a1 += b1; a2 += b2; } else c = -1;
      }
    }
    if (c >= 0) {
      double* fr = rd.cframe + 4 * ((st.n & 1) * ncl + c);
      atomicAdd(fr, a0);
      atomicAdd(fr + 1, a1);
      atomicAdd(fr + 2, a2);
    }
  }
}

// RS: density resampling compiled in; AT: MPCD-AT collision (Eq. 6) instead of
// SRD; CE: the Chapman-Enskog redraw compiled in (the plain pass keeps only the
// Maxwellian one).  MPCD-AT needs the cell mean of the particles' random velocities
// before any particle can leave the collision; as the old relative velocity
// plays no part in it, the binning pass draws each particle's random velocity
// v_ran, adds v - v_ran to its cell sum and stores v_ran in place of v.  The
// cell-table items turn the sums into v_cm - <v_ran>, and the next pass adds
// that to the stored v_ran: v_cm + v_ran - <v_ran> (virtual wall particles
// enter the table).
template <int D, typename R, bool RS, bool AT, bool CE>
__device__ __forceinline__ void particle_item(const RepDev& rd, const StepInfo& st, const uint32_t start,
                                              const uint32_t end, PassShared<D, R>& red) {
  using T4 = typename Vec4<R>::T;
  const uint32_t j0 = start + threadIdx.x;
  const bool alt = st.src_alt;
  const uint32_t* hsrc = alt ? rd.home_alt : rd.home;   // plain loads (see lb_row)
  int X[PPT], Y[PPT], Z[PPT];
  R o[PPT][3], v[PPT][3];
  bool act[PPT];
  // branch-free loads: a lane past the end reads the last particle and discards it
  void* const* offs = alt ? rd.off_alt : rd.off;
  void* const* vels = alt ? rd.vel_alt : rd.vel;
  const uint32_t np32 = min(RS ? pool_end(rd) : (uint32_t)rd.np, end), last = np32 ? np32 - 1u : 0u;
  // density resampling: removed particles (HOME_DEAD) are skipped, particles
  // created this step (PID_FRESH) are neither rotated nor removed
  bool fresh[PPT];
#pragma unroll
  for (int p = 0; p < PPT; ++p) {
    const uint32_t j = j0 + 256u * p;
    act[p] = j < np32;
    fresh[p] = false;
    const uint32_t jl = act[p] ? j : last;
    uint32_t hp = ld_hint(hsrc + jl, l2_stream());
    if (RS && rd.pooled) {
      if (hp == HOME_DEAD) { act[p] = false; hp = 0u; }
      fresh[p] = act[p] && rd.resample && (alt ? rd.pid_alt : rd.pid)[jl] == PID_FRESH;
    }
    HomePack<D>::unpack(hp, X[p], Y[p], Z[p]);
#pragma unroll
    for (int a = 0; a < 3; ++a) { o[p][a] = R(0); v[p][a] = R(0); }
    PState<D, R>::ld(offs, jl, o[p]);
    PState<D, R>::ld(vels, jl, v[p]);
  }
  // a7 of step n-1: cell-table loads for all particles, then the collisions
  if (st.pending) {
    const T4* tab = (const T4*)rd.tab;
    T4 t0[PPT], t1[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
      const uint32_t c = collision_cell<D, R>(rd, X[p], Y[p], Z[p], o[p], Cst<R>::prev(st));
      if (D == 2) t0[p] = ld_ro(tab + c);
      else { t0[p] = ld_ro(tab + 2 * (size_t)c); if (!AT) t1[p] = ld_ro(tab + 2 * (size_t)c + 1); }
    }
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
      if (RS && fresh[p]) continue;
      collide_from_table<D, R, AT>(rd, t0[p], t1[p], v[p]);
    }
  }
  uint32_t cid[PPT];
#pragma unroll
  for (int p = 0; p < PPT; ++p) {
    cid[p] = NO_CELL;
    if (!act[p]) continue;
    cid[p] = move_particle<D, R, RS, AT, CE>(rd, st, j0 + 256u * p, alt, fresh[p], X[p], Y[p], Z[p], o[p], v[p]);
  }
  if (D == 2 && !AT && rd.cl_on) add_strip_sums<R>(rd, st, cid, X, Y, v);
  add_cell_sums<D, R>(rd, cid, v, red);
}

// resident blocks per SM: 6 in 2D (40 registers, no spills); 5 in 3D, whose
// state needs more registers (at 6 the 3D pass spilled and ran 13 % slower);
// the single-replica 2D form runs at 8 (32 registers, no spills except in the
// Chapman-Enskog variant, which keeps 6): 71.8 against 72.8 us per step at
// 2048 x 512, the pass being bound by the latency of its dependent loads
template <int D, typename R, bool RS, bool AT, bool CE>
__global__ void __launch_bounds__(256, D == 2 ? 6 : 5) particle_pass(const RepDev* __restrict__ reps, const int2* __restrict__ bmap,
                                                     int nwork, const StepInfo* __restrict__ si, int k, int nrep) {
  __shared__ RepDev rd;
  __shared__ StepInfo st;
  __shared__ PassShared<D, R> red;
  wait_for_prerequisite();    // launched as a programmatic dependent: the table of step n - 1 is complete
  allow_dependent_launch();   // the LB update of step n + 1 may start beside this pass
  for_each_item<true>(bmap, nwork, reps, si, k, nrep, rd, st,
                      [&](const int2 bm) { particle_item<D, R, RS, AT, CE>(rd, st, (uint32_t)bm.y * PP_ITEM, ~0u, red); });
}

// single-replica form (see for_each_item_one)
template <int D, typename R, bool RS, bool AT, bool CE>
__global__ void __launch_bounds__(256, (D == 2 && !CE && sizeof(R) == 4) ? 8 : (D == 2 ? 6 : 5))
    particle_pass_one(const __grid_constant__ RepDev rd, int nwork,
                                                         const StepInfo* __restrict__ si, int k) {
  __shared__ StepInfo st;
  __shared__ PassShared<D, R> red;
  wait_for_prerequisite();    // launched as a programmatic dependent: the table of step n - 1 is complete
  allow_dependent_launch();   // the LB update of step n + 1 may start beside this pass
  {
    const int* c = (const int*)(si + k);
    int* d = (int*)&st;
    for (int i = threadIdx.x; i < (int)(sizeof(StepInfo) / 4); i += blockDim.x) d[i] = c[i];
    __syncthreads();
  }
  // an even share of the particles per block (a multiple of 32), walked in
  // PP_ITEM chunks: every block ends with the same amount of work, where
  // whole items left some blocks one item longer than the rest
  const uint32_t np = RS ? pool_end(rd) : (uint32_t)rd.np;
  const uint32_t per = ((np + gridDim.x - 1u) / gridDim.x + 31u) & ~31u;
  const uint32_t b0 = blockIdx.x * per, b1 = min(np, b0 + per);
  for (uint32_t s = b0; s < b1; s += PP_ITEM) particle_item<D, R, RS, AT, CE>(rd, st, s, b1, red);
}

// bps > 0: that many blocks per SM at most (the overlapped form leaves room
// for the LB update beside the pass), else the occupancy limit
template <int D, typename R, bool RS, bool AT, bool CE>
static void go_particles(const Launch& L, const int2* bmap, int nwork, int k, int bps, bool pdl) {
  const int cap = bps > 0 ? bps * sm_count() : 1 << 30;
  if (L.nrep == 1 && L.host) {
    static const int g1 = grid_cap(grid_for(particle_pass_one<D, R, RS, AT, CE>, 256, 1 << 30));
    const int g = min(min(g1, cap), nwork);
    launch_pdl(particle_pass_one<D, R, RS, AT, CE>, g, 256, L.stream, pdl, *L.host, nwork, L.si, k);
    return;
  }
  static const int gm = grid_cap(grid_for(particle_pass<D, R, RS, AT, CE>, 256, 1 << 30));
  const int g = min(min(gm, cap), nwork);
  launch_pdl(particle_pass<D, R, RS, AT, CE>, g, 256, L.stream, pdl, L.reps, bmap, nwork, L.si, k, L.nrep);
}

template <int D, typename R>
static void go_particles_mode(bool rs, bool at, bool ce, const Launch& L, const int2* bmap, int nwork, int k,
                              int bps, bool pdl) {
  if (ce) {
    if (at) go_particles<D, R, false, true, true>(L, bmap, nwork, k, bps, pdl);
    else go_particles<D, R, false, false, true>(L, bmap, nwork, k, bps, pdl);
  } else if (at) {
    go_particles<D, R, false, true, false>(L, bmap, nwork, k, bps, pdl);
  } else if (rs) {
    go_particles<D, R, true, false, false>(L, bmap, nwork, k, bps, pdl);
  } else {
    go_particles<D, R, false, false, false>(L, bmap, nwork, k, bps, pdl);
  }
}

// rs: some replica of the handle uses density resampling (the pass then checks
// each replica's mode; without it the resampling code is not compiled in);
// at: the handle's replicas collide by MPCD-AT (never together with rs);
// ce: some replica redraws by Chapman-Enskog (never together with rs)
cudaError_t launch_particles(int dim, int prec, bool rs, bool at, bool ce, const Launch& L, const int2* bmap,
                             int nwork, int k, int bps, bool pdl) {
  if (nwork == 0) return cudaSuccess;
  if (dim == 2) {
    if (prec == P_FP64) go_particles_mode<2, double>(rs, at, ce, L, bmap, nwork, k, bps, pdl);
    else go_particles_mode<2, float>(rs, at, ce, L, bmap, nwork, k, bps, pdl);
  } else {
    if (prec == P_FP64) go_particles_mode<3, double>(rs, at, ce, L, bmap, nwork, k, bps, pdl);
    else go_particles_mode<3, float>(rs, at, ce, L, bmap, nwork, k, bps, pdl);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a3' (resample_density = 1): one thread per outer-buffer cell, run before the
// particle pass.  N = floor(x) + [u < x - floor(x)], x = ppc rho_LB of the LB
// node holding the cell (rho0 = 1), u from Philox(c, n, replica,
// TAG_DENSITY), capped at SPAWN_MAX ppc; new particle k gets 24-bit uniform
// offsets from Philox(c SPAWN_MAX ppc + k, n, replica, TAG_SPAWN_POS) and the
// velocity u_fine + sqrt(kT/m) xi from Philox(..., TAG_SPAWN_VEL), and is
// appended to the pool (the arrays this step's particle pass reads) with
// PID_FRESH.  c = X + Wx (Y + Hy Z) is the home-cell index.  The particle pass
// removes the particles that were in these cells.  Past the pool capacity no
// particle is written and pool[1] is set.
template <int D, typename R>
__device__ __forceinline__ void spawn_item(const RepDev& rd, const StepInfo& st, const int2 bm) {
  const int nl = rd.xo_lo, nr = rd.Wx - rd.xo_hi, ncol = nl + nr;
  const long long t = (long long)bm.y * blockDim.x + threadIdx.x;
  if (t >= (long long)ncol * rd.Hy * rd.Wz) return;
  const int xi = (int)(t % ncol);
  const long long rest = t / ncol;
  const int Y = (int)(rest % rd.Hy), Z = (int)(rest / rd.Hy);
  const int X = xi < nl ? xi : rd.xo_hi + (xi - nl);
  const uint32_t c = (uint32_t)(X + (long long)rd.Wx * (Y + (long long)rd.Hy * Z));
  const long long node = (rd.x0 + X / rd.r) + (long long)rd.nx * ((1 + Y / rd.r) + (long long)rd.ny * (D == 3 ? Z / rd.r : 0));
  const double x = (double)rd.ppc * (double)rho_of<R>(rd, st.n)[node];
  const uint4 wd = philox(c, st.n, rd.rep, TAG_DENSITY, rd.key0, rd.key1);
  const double fl = floor(x);
  const uint32_t nmax = (uint32_t)(SPAWN_MAX * rd.ppc);
  long long nn = (long long)fl + (unit24(wd.x) < x - fl ? 1 : 0);
  if (nn < 0) nn = 0;
  uint32_t n = nn > (long long)nmax ? nmax : (uint32_t)nn;
  if (n == 0) return;
  R uf[3] = {R(0), R(0), R(0)};
  u_fine<D, R>(rd, st.n, X, Y, Z, uf);
  const uint32_t base = atomicAdd(rd.pool, n);
  const bool alt = st.src_alt;
  uint32_t* home = alt ? rd.home_alt : rd.home;
  uint32_t* pid = alt ? rd.pid_alt : rd.pid;
  void* const* offs = alt ? rd.off_alt : rd.off;
  void* const* vels = alt ? rd.vel_alt : rd.vel;
  const R sg = Cst<R>::sig(rd);
  const uint32_t hp = HomePack<D>::pack(X, Y, Z);
  for (uint32_t k = 0; k < n; ++k) {
    const uint32_t j = base + k;
    if (j >= rd.cap) { atomicExch(rd.pool + 1, 1u); break; }
    const uint32_t id = c * nmax + k;
    const uint4 wp = philox(id, st.n, rd.rep, TAG_SPAWN_POS, rd.key0, rd.key1);
    const uint4 wv = philox(id, st.n, rd.rep, TAG_SPAWN_VEL, rd.key0, rd.key1);
    R z0, z1, z2, z3;
    normal_pair(wv.x, wv.y, z0, z1);
    normal_pair(wv.z, wv.w, z2, z3);
    R o[3] = {(R)unit24(wp.x), (R)unit24(wp.y), D == 3 ? (R)unit24(wp.z) : R(0)};
    R v[3] = {uf[0] + sg * z0, uf[1] + sg * z1, D == 3 ? uf[2] + sg * z2 : R(0)};
    home[j] = hp;
    pid[j] = PID_FRESH;
    PState<D, R>::st(offs, j, o);
    PState<D, R>::st(vels, j, v);
  }
}

template <int D, typename R>
__global__ void __launch_bounds__(256) spawn_pass(const RepDev* __restrict__ reps, const int2* __restrict__ bmap,
                                                  int nwork, const StepInfo* __restrict__ si, int k, int nrep) {
  __shared__ RepDev rd;
  __shared__ StepInfo st;
  for_each_item(bmap, nwork, reps, si, k, nrep, rd, st, [&](const int2 bm) { spawn_item<D, R>(rd, st, bm); });
}

cudaError_t launch_spawn(int dim, int prec, const Launch& L, const int2* bmap, int nwork, int k) {
  if (nwork == 0) return cudaSuccess;
  const int g = nwork < 4096 ? nwork : 4096;
  if (dim == 2) {
    if (prec == P_FP64) spawn_pass<2, double><<<g, 256, 0, L.stream>>>(L.reps, bmap, nwork, L.si, k, L.nrep);
    else spawn_pass<2, float><<<g, 256, 0, L.stream>>>(L.reps, bmap, nwork, L.si, k, L.nrep);
  } else {
    if (prec == P_FP64) spawn_pass<3, double><<<g, 256, 0, L.stream>>>(L.reps, bmap, nwork, L.si, k, L.nrep);
    else spawn_pass<3, float><<<g, 256, 0, L.stream>>>(L.reps, bmap, nwork, L.si, k, L.nrep);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The collision-cell table of step m for the read-outs between calls (the
// step itself builds it inside the next LB launch): every cell of one
// replica, blocks of 256 CPT cells.
template <int Q, typename S>
__global__ void __launch_bounds__(256) cell_table_one(const __grid_constant__ RepDev rd, uint32_t m, int shift_y_pos) {
  cell_table_item<Q, S>(rd, m, shift_y_pos != 0, (long long)blockIdx.x * 256 * CPT, rd.ncell);
}

cudaError_t launch_cell_table(int q, int prec, const RepDev& rd, uint32_t m, bool shift_y_pos, cudaStream_t st) {
  const long long nb = (rd.ncell + 256 * CPT - 1) / (256 * CPT);
  if (nb == 0) return cudaSuccess;
  const int sp = shift_y_pos ? 1 : 0;
#define LBM_CT(QQ, SS) cell_table_one<QQ, SS><<<(int)nb, 256, 0, st>>>(rd, m, sp)
  if (q == 9) {
    if (prec == P_FP64) LBM_CT(9, double);
    else if (prec == P_FP32) LBM_CT(9, float);
    else LBM_CT(9, __half);
  } else {
    if (prec == P_FP64) LBM_CT(19, double);
    else if (prec == P_FP32) LBM_CT(19, float);
    else LBM_CT(19, __half);
  }
#undef LBM_CT
  return cudaGetLastError();
}

// WINDOW_MEAN after step m: rho_bar, u_bar of the last min(m + 1, W) frames
// of every inner-buffer node, from the window state (frame m is folded in by
// the next LB update, so it is added here without moving the window).
template <int D, typename R>
__global__ void window_out(const __grid_constant__ RepDev rd, uint32_t m, double* __restrict__ out) {
  const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (b >= rd.nbuf) return;
  double W4[4];
  window_sums(rd, m, b, false, W4);
  R rho, u[3];
  window_mean<D, R>(rd, m, W4, rho, u);
  out[4 * b] = (double)rho;
  out[4 * b + 1] = (double)u[0]; out[4 * b + 2] = (double)u[1]; out[4 * b + 3] = (double)u[2];
}

cudaError_t launch_window_out(int dim, int prec, const RepDev& rd, uint32_t m, double* out, cudaStream_t st) {
  const int nb = (int)((rd.nbuf + 255) / 256);
  if (nb == 0) return cudaSuccess;
  if (dim == 2) {
    if (prec == P_FP64) window_out<2, double><<<nb, 256, 0, st>>>(rd, m, out);
    else window_out<2, float><<<nb, 256, 0, st>>>(rd, m, out);
  } else {
    if (prec == P_FP64) window_out<3, double><<<nb, 256, 0, st>>>(rd, m, out);
    else window_out<3, float><<<nb, 256, 0, st>>>(rd, m, out);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Persistent form of a chunk: one cooperative launch runs kcount steps, each
// as the two phases lb_pull (with the cell-table items of the previous step)
// -> particle_pass over the same block maps (the LB map with 256-thread row
// tiles and 256 CPT-cell items), separated by a grid barrier.  The barrier is a counter and a generation word in global memory;
// every wait is bounded: after `spin` polls (PB_SPIN unless the handle set
// another limit) a block records the failure in *err and leaves the launch,
// and a block that finds *err set leaves too, so a stuck barrier ends the
// kernel instead of hanging the GPU.  Co-residency of all blocks comes from the
// cooperative launch.
constexpr unsigned PB_SPIN = 1u << 24;

__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned* gen, unsigned nblocks, int* err,
                                             unsigned spin) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g = atomicAdd(gen, 0u);
    __threadfence();
    int ok = 1;
    if (atomicAdd(count, 1u) + 1u == nblocks) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      unsigned it = 0;
      const volatile unsigned* vg = gen;
      const volatile int* ve = err;
      while (*vg == g) {   // plain polling loads (L2), no atomic traffic on the word
        if (++it >= spin || *ve != 0) { ok = 0; break; }
        __nanosleep(32);
      }
      if (!ok) atomicExch(err, 1);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <int Q, typename S, int V>
__global__ void __launch_bounds__(256, 2) step_persistent(const RepDev* __restrict__ reps, int nrep,
                                                         const StepInfo* __restrict__ si, int kcount,
                                                         const int4* __restrict__ bm_lb, int nb_lb,
                                                         const int2* __restrict__ bm_p, int nb_p,
                                                         unsigned* bar, int* err, unsigned spin) {
  constexpr int D = Q == 9 ? 2 : 3;
  using R = typename std::conditional<sizeof(S) == 8, double, float>::type;
  __shared__ RepDev rd;
  __shared__ StepInfo st;
  __shared__ PassShared<D, R> red;
  for (int k = 0; k < kcount; ++k) {
    for_each_item(bm_lb, nb_lb, reps, si, k, nrep, rd, st, [&](const int4 bm) { lb_row<Q, S, V>(rd, st, bm); });
    if (!grid_barrier(bar, bar + 1, gridDim.x, err, spin)) return;
    for_each_item(bm_p, nb_p, reps, si, k, nrep, rd, st, [&](const int2 bm) { particle_item<D, R, false, false, false>(rd, st, (uint32_t)bm.y * PP_ITEM, ~0u, red); });
    if (!grid_barrier(bar, bar + 1, gridDim.x, err, spin)) return;
  }
}

template <int Q, typename S, int V>
static cudaError_t go_persistent(const Launch& L, int kcount, const PersistentMaps& m, int blocks_per_sm,
                                 int* grid_out) {
  static int occ = -1, sms = 0;
  if (occ < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, step_persistent<Q, S, V>, 256, 0) != cudaSuccess) occ = 0;
  }
  if (occ < 1) return cudaErrorCooperativeLaunchTooLarge;
  const int bps = blocks_per_sm > 0 && blocks_per_sm < occ ? blocks_per_sm : occ;
  const int grid = bps * sms;
  if (grid_out) *grid_out = grid;
  const RepDev* reps = L.reps;
  int nrep = L.nrep;
  const StepInfo* si = L.si;
  const int4* bl = m.lb;
  const int2* bp = m.p;
  int nl = m.nb_lb, np = m.nb_p;
  unsigned* bar = m.bar;
  int* err = m.err;
  unsigned spin = m.spin ? m.spin : PB_SPIN;
  void* args[] = {(void*)&reps, (void*)&nrep, (void*)&si, (void*)&kcount, (void*)&bl, (void*)&nl,
                  (void*)&bp,   (void*)&np,   (void*)&bar, (void*)&err, (void*)&spin};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = L.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, (const void*)step_persistent<Q, S, V>, args);
}

cudaError_t launch_persistent(int q, int prec, int vec, const Launch& L, int kcount, const PersistentMaps& m,
                              int blocks_per_sm, int* grid_out) {
  if (q == 9) {
    if (prec == P_FP64) return go_persistent<9, double, 1>(L, kcount, m, blocks_per_sm, grid_out);
    if (prec == P_FP32)
      return vec == 4 ? go_persistent<9, float, 4>(L, kcount, m, blocks_per_sm, grid_out)
                      : go_persistent<9, float, 1>(L, kcount, m, blocks_per_sm, grid_out);
    return vec == 4 ? go_persistent<9, __half, 4>(L, kcount, m, blocks_per_sm, grid_out)
                    : go_persistent<9, __half, 1>(L, kcount, m, blocks_per_sm, grid_out);
  }
  if (prec == P_FP64) return go_persistent<19, double, 1>(L, kcount, m, blocks_per_sm, grid_out);
  if (prec == P_FP32)
    return vec == 2 ? go_persistent<19, float, 2>(L, kcount, m, blocks_per_sm, grid_out)
                    : go_persistent<19, float, 1>(L, kcount, m, blocks_per_sm, grid_out);
  return vec == 2 ? go_persistent<19, __half, 2>(L, kcount, m, blocks_per_sm, grid_out)
                  : go_persistent<19, __half, 1>(L, kcount, m, blocks_per_sm, grid_out);
}

// ---------------------------------------------------------------------------
// flush: a7 of the last step for every particle of one replica.
template <int D, typename R>
__global__ void flush_collision(const RepDev* __restrict__ rdp, double s0, double s1, double s2) {
  const RepDev& rd = *rdp;
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= pool_end(rd)) return;
  const R s[3] = {(R)s0, (R)s1, (R)s2};     // shifts are exact in binary32
  int X, Y, Z;
  const uint32_t hp = rd.home[j];
  if (hp == HOME_DEAD) return;
  HomePack<D>::unpack(hp, X, Y, Z);
  R o[3] = {R(0), R(0), R(0)}, v[3] = {R(0), R(0), R(0)};
  PState<D, R>::ld(rd.off, (uint32_t)j, o);
  PState<D, R>::ld(rd.vel, (uint32_t)j, v);
  rotate<D, R>(rd, collision_cell<D, R>(rd, X, Y, Z, o, s), v);
  PState<D, R>::st(rd.vel, (uint32_t)j, v);
}

cudaError_t launch_flush(int dim, int prec, const RepDev* rd_dev, const RepDev& rd, const double* ls,
                         cudaStream_t st) {
  const int nb = (int)(((rd.pooled ? (long long)rd.cap : rd.np) + 255) / 256);
  if (nb == 0) return cudaSuccess;
  if (dim == 2) {
    if (prec == P_FP64) flush_collision<2, double><<<nb, 256, 0, st>>>(rd_dev, ls[0], ls[1], ls[2]);
    else flush_collision<2, float><<<nb, 256, 0, st>>>(rd_dev, ls[0], ls[1], ls[2]);
  } else {
    if (prec == P_FP64) flush_collision<3, double><<<nb, 256, 0, st>>>(rd_dev, ls[0], ls[1], ls[2]);
    else flush_collision<3, float><<<nb, 256, 0, st>>>(rd_dev, ls[0], ls[1], ls[2]);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// initial particles: ppc per cell in cell order, offsets from 24-bit Philox
// uniforms, Maxwellian velocities (variance kT/m) from Box-Muller pairs.
template <int D, typename R>
__global__ void init_particles(const RepDev* __restrict__ rdp) {
  const RepDev& rd = *rdp;
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= rd.np) return;
  const long long cell = j / rd.ppc;
  const int X = (int)(cell % rd.Wx), Y = (int)((cell / rd.Wx) % rd.Hy), Z = (int)(cell / ((long long)rd.Wx * rd.Hy));
  const uint4 wp = philox((uint32_t)j, 0u, rd.rep, TAG_INIT_POS, rd.key0, rd.key1);
  const uint4 wv = philox((uint32_t)j, 0u, rd.rep, TAG_INIT_VEL, rd.key0, rd.key1);
  double z[4];
  normal_pair(wv.x, wv.y, z[0], z[1]);
  normal_pair(wv.z, wv.w, z[2], z[3]);
  const uint32_t wo[3] = {wp.x, wp.y, wp.z};
  rd.home[j] = HomePack<D>::pack(X, Y, Z);
  rd.pid[j] = (uint32_t)j;
  R o[3], v[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    o[a] = (R)unit24(wo[a]);
    v[a] = (R)(rd.sig * z[a]);
  }
  PState<D, R>::st(rd.off, (uint32_t)j, o);
  PState<D, R>::st(rd.vel, (uint32_t)j, v);
}

cudaError_t launch_init_particles(int dim, int prec, const RepDev* rd_dev, const RepDev& rd, cudaStream_t st) {
  const int nb = (int)((rd.np + 255) / 256);
  if (nb == 0) return cudaSuccess;
  if (dim == 2) {
    if (prec == P_FP64) init_particles<2, double><<<nb, 256, 0, st>>>(rd_dev);
    else init_particles<2, float><<<nb, 256, 0, st>>>(rd_dev);
  } else {
    if (prec == P_FP64) init_particles<3, double><<<nb, 256, 0, st>>>(rd_dev);
    else init_particles<3, float><<<nb, 256, 0, st>>>(rd_dev);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// particle fields in id order (binary64 / int32) and back.
enum { F_POS = 3, F_VEL = 4, F_CELL = 5, F_HOME = 10, F_ID = 12 };

// With density resampling the live particles come out in pool order (rank =
// compaction index from live_scan_*), PART_ID giving each one's id (initial
// index, or PID_SPAWNED for particles created by the resampling).
template <int D, typename R>
__global__ void part_out(RepDev rd, int field, double s0, double s1, double s2, void* out) {
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= pool_end(rd)) return;
  const uint32_t hp = rd.home[j];
  if (rd.pooled && hp == HOME_DEAD) return;
  const long long id = rd.pooled ? (long long)rd.rank[j] : (long long)rd.pid[j];
  int X, Y, Z;
  HomePack<D>::unpack(hp, X, Y, Z);
  if (field == F_POS || field == F_VEL) {
    double* o = (double*)out;
    R x[3] = {R(0), R(0), R(0)};
    PState<D, R>::ld(field == F_POS ? rd.off : rd.vel, (uint32_t)j, x);
    for (int a = 0; a < 3; ++a) o[3 * id + a] = (double)x[a];
  } else if (field == F_HOME) {
    int* o = (int*)out;
    o[3 * id] = X; o[3 * id + 1] = Y; o[3 * id + 2] = Z;
  } else if (field == F_CELL) {
    R of[3] = {R(0), R(0), R(0)};
    PState<D, R>::ld(rd.off, (uint32_t)j, of);
    const R s[3] = {(R)s0, (R)s1, (R)s2};
    ((int*)out)[id] = (int)collision_cell<D, R>(rd, X, Y, Z, of, s);
  } else {
    ((int*)out)[id] = rd.pooled ? (int)rd.pid[j] : (int)id;
  }
}

template <int D, typename R>
__global__ void part_in(RepDev rd, int field, const void* in, int* bad) {
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= rd.np) return;
  const long long id = rd.pid[j];
  if (field == F_POS || field == F_VEL) {
    const double* s = (const double*)in;
    R x3[3] = {R(0), R(0), R(0)};
    for (int a = 0; a < D; ++a) {
      const double x = s[3 * id + a];
      if (field == F_POS && !(x >= 0.0 && x < 1.0)) atomicExch(bad, 1);
      const R xr = (R)x;
      x3[a] = (field == F_POS && xr >= R(1)) ? Num<R>::one_minus : xr;
    }
    PState<D, R>::st(field == F_POS ? rd.off : rd.vel, (uint32_t)j, x3);
  } else {
    const int* s = (const int*)in;
    const int X = s[3 * id], Y = s[3 * id + 1], Z = D == 3 ? s[3 * id + 2] : 0;
    if (X < 0 || X >= rd.Wx || Y < 0 || Y >= rd.Hy || Z < 0 || Z >= rd.Wz) {
      atomicExch(bad, 1);
      return;
    }
    rd.home[j] = HomePack<D>::pack(X, Y, Z);
  }
}

cudaError_t launch_part_out(int dim, int prec, const RepDev& rd, int field, const double* ls, void* out,
                            cudaStream_t st) {
  const int nb = (int)(((rd.pooled ? (long long)rd.cap : rd.np) + 255) / 256);
  if (nb == 0) return cudaSuccess;
  if (dim == 2) {
    if (prec == P_FP64) part_out<2, double><<<nb, 256, 0, st>>>(rd, field, ls[0], ls[1], ls[2], out);
    else part_out<2, float><<<nb, 256, 0, st>>>(rd, field, ls[0], ls[1], ls[2], out);
  } else {
    if (prec == P_FP64) part_out<3, double><<<nb, 256, 0, st>>>(rd, field, ls[0], ls[1], ls[2], out);
    else part_out<3, float><<<nb, 256, 0, st>>>(rd, field, ls[0], ls[1], ls[2], out);
  }
  return cudaGetLastError();
}

cudaError_t launch_part_in(int dim, int prec, const RepDev& rd, int field, const void* in, int* bad,
                           cudaStream_t st) {
  const int nb = (int)((rd.np + 255) / 256);
  if (nb == 0) return cudaSuccess;
  if (dim == 2) {
    if (prec == P_FP64) part_in<2, double><<<nb, 256, 0, st>>>(rd, field, in, bad);
    else part_in<2, float><<<nb, 256, 0, st>>>(rd, field, in, bad);
  } else {
    if (prec == P_FP64) part_in<3, double><<<nb, 256, 0, st>>>(rd, field, in, bad);
    else part_in<3, float><<<nb, 256, 0, st>>>(rd, field, in, bad);
  }
  return cudaGetLastError();
}

// A piece of a region divided over x-slabs keeps the particles whose home
// cell column X lies in [lo, hi) modulo the region's width Wx; the others
// are removed (HOME_DEAD; the next sort compacts the pool).
template <int D>
__global__ void keep_columns(RepDev rd, int lo, int hi) {
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= pool_end(rd)) return;
  const uint32_t hp = rd.home[j];
  if (hp == HOME_DEAD) return;
  int X, Y, Z;
  HomePack<D>::unpack(hp, X, Y, Z);
  const int dx = wrap(X - lo, rd.Wx);
  if (dx >= hi - lo) rd.home[j] = HOME_DEAD;
}

cudaError_t launch_keep_columns(int dim, const RepDev& rd, int lo, int hi, cudaStream_t st) {
  const int nb = (int)(((long long)rd.cap + 255) / 256);
  if (nb == 0) return cudaSuccess;
  if (dim == 2) keep_columns<2><<<nb, 256, 0, st>>>(rd, lo, hi);
  else keep_columns<3><<<nb, 256, 0, st>>>(rd, lo, hi);
  return cudaGetLastError();
}

// Pooled particles replaced by n given ones (home cells int32 [n][3],
// offsets and velocities binary64 [n][3], ids int32 [n]) in slots 0 .. n-1,
// all in the sorted order the caller gives; the pool ends at n.  A home cell
// outside the region, or an offset outside [0, 1), sets *bad and the slot is
// written as removed (HOME_DEAD).
template <int D, typename R>
__global__ void pool_in(RepDev rd, long long n, const int* __restrict__ home, const double* __restrict__ off,
                        const double* __restrict__ vel, const int* __restrict__ pid, int* bad) {
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int X = home[3 * j], Y = home[3 * j + 1], Z = D == 3 ? home[3 * j + 2] : 0;
  R o[3], v[3];
  bool ok = X >= 0 && X < rd.Wx && Y >= 0 && Y < rd.Hy && Z >= 0 && Z < rd.Wz;
  for (int a = 0; a < 3; ++a) {
    o[a] = (R)off[3 * j + a];
    v[a] = (R)vel[3 * j + a];
    if (a < D && !(o[a] >= R(0) && o[a] < R(1))) ok = false;
  }
  if (!ok) {
    rd.home[j] = HOME_DEAD;
    atomicExch(bad, 1);
    return;
  }
  rd.home[j] = HomePack<D>::pack(X, Y, Z);
  rd.pid[j] = (uint32_t)pid[j];
  PState<D, R>::st(rd.off, (uint32_t)j, o);
  PState<D, R>::st(rd.vel, (uint32_t)j, v);
}

cudaError_t launch_pool_in(int dim, int prec, const RepDev& rd, long long n, const int* home, const double* off,
                           const double* vel, const int* pid, int* bad, cudaStream_t st) {
  const int nb = (int)((n + 255) / 256);
  if (nb == 0) return cudaSuccess;
  if (dim == 2) {
    if (prec == P_FP64) pool_in<2, double><<<nb, 256, 0, st>>>(rd, n, home, off, vel, pid, bad);
    else pool_in<2, float><<<nb, 256, 0, st>>>(rd, n, home, off, vel, pid, bad);
  } else {
    if (prec == P_FP64) pool_in<3, double><<<nb, 256, 0, st>>>(rd, n, home, off, vel, pid, bad);
    else pool_in<3, float><<<nb, 256, 0, st>>>(rd, n, home, off, vel, pid, bad);
  }
  return cudaGetLastError();
}

// particle count, momentum and kinetic energy (binary64) into out[4..8].
template <int D, typename R>
__global__ void part_diag(RepDev rd, double* out) {
  double p[3] = {0, 0, 0}, e = 0, cnt = 0;
  const long long end = pool_end(rd);
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < end;
       j += (long long)gridDim.x * blockDim.x) {
    if (rd.pooled && rd.home[j] == HOME_DEAD) continue;
    cnt += 1.0;
    R vv[3] = {R(0), R(0), R(0)};
    PState<D, R>::ld(rd.vel, (uint32_t)j, vv);
    for (int a = 0; a < D; ++a) {
      const double v = (double)vv[a];
      p[a] += rd.mass * v;
      e += 0.5 * rd.mass * v * v;
    }
  }
  double vals[5] = {cnt, p[0], p[1], p[2], e};
  for (int a = 0; a < 5; ++a) {
    double t = vals[a];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&out[4 + a], t);
  }
}

cudaError_t launch_diag_particles(int dim, int prec, const RepDev& rd, double* out9, cudaStream_t st) {
  const long long nslots = rd.pooled ? (long long)rd.cap : rd.np;
  if (nslots == 0) return cudaSuccess;
  long long g = (nslots + 255) / 256;
  const int nb = (int)(g < 1024 ? g : 1024);
  if (dim == 2) {
    if (prec == P_FP64) part_diag<2, double><<<nb, 256, 0, st>>>(rd, out9);
    else part_diag<2, float><<<nb, 256, 0, st>>>(rd, out9);
  } else {
    if (prec == P_FP64) part_diag<3, double><<<nb, 256, 0, st>>>(rd, out9);
    else part_diag<3, float><<<nb, 256, 0, st>>>(rd, out9);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Counting sort of the particles by home cell (row-major X fastest).
// sort_count: rank of every particle inside its home cell (warp-aggregated
// atomics on the per-cell counters); sort_scan_tiles: exclusive prefix of the
// counters inside tiles of SORT_TILE cells, tile totals, counters cleared;
// sort_scan_top: exclusive prefix of the tile totals (one block per replica);
// sort_scatter: every particle copied to its sorted slot in the *_alt arrays.
template <int D>
__device__ __forceinline__ uint32_t home_index(const RepDev& rd, uint32_t packed) {
  int X, Y, Z;
  HomePack<D>::unpack(packed, X, Y, Z);
  return (uint32_t)(X + rd.Wx * (Y + rd.Hy * Z));
}

template <int D>
__device__ __forceinline__ void sort_count_one(const RepDev& rd, const long long j) {
  const uint32_t hp = j < pool_end(rd) ? rd.home[j] : HOME_DEAD;
  const bool active = hp != HOME_DEAD;   // removed particles are dropped (pool compaction)
  const uint32_t h = active ? home_index<D>(rd, hp) : 0xFFFFFFFFu;
  const unsigned grp = __match_any_sync(0xFFFFFFFFu, h);
  const int lane = threadIdx.x & 31, leader = __ffs(grp) - 1;
  uint32_t base = 0;
  if (active && lane == leader) base = atomicAdd(rd.hcount + h, (uint32_t)__popc(grp));
  base = __shfl_sync(0xFFFFFFFFu, base, leader);
  if (active) rd.rank[j] = base + (uint32_t)__popc(grp & ((1u << lane) - 1u));
}

template <int D>
__device__ __forceinline__ void sort_count_item(const RepDev& rd, const int2 bm) {
#pragma unroll
  for (int p = 0; p < PPT; ++p) sort_count_one<D>(rd, (long long)bm.y * PP_ITEM + 256 * p + threadIdx.x);
}

template <int D>
__global__ void __launch_bounds__(256) sort_count(const RepDev* __restrict__ reps, const int2* __restrict__ bmap,
                                                  int nwork) {
  __shared__ RepDev rd;
  __shared__ StepInfo unused;
  for_each_item(bmap, nwork, reps, (const StepInfo*)nullptr, 0, 0, rd, unused,
                [&](const int2 bm) { sort_count_item<D>(rd, bm); });
}

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* warp_tot, uint32_t& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < nw ? warp_tot[lane] : 0u, ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, ti, o);
      if (lane >= o) ti += u;
    }
    if (lane < nw) warp_tot[lane] = ti - t;
    if (lane == 31) warp_tot[32] = ti;
  }
  __syncthreads();
  total = warp_tot[32];
  return inc - x + warp_tot[w];
}

__global__ void __launch_bounds__(SORT_TILE) sort_scan_tiles(const RepDev* __restrict__ reps, const int2* __restrict__ bmap) {
  __shared__ RepDev rd;
  __shared__ StepInfo unused;
  __shared__ uint32_t wt[33];
  const int2 bm = bmap[blockIdx.x];
  load_block_records(rd, unused, reps, nullptr, bm.x, 0, 0);
  const long long c = (long long)bm.y * SORT_TILE + threadIdx.x;
  const uint32_t x = c < rd.nhome ? rd.hcount[c] : 0u;
  uint32_t total;
  const uint32_t ex = block_exclusive_scan(x, wt, total);
  if (c < rd.nhome) { rd.hoff[c] = ex; rd.hcount[c] = 0u; }
  if (threadIdx.x == 0) rd.tsum[bm.y] = total;
}

__global__ void __launch_bounds__(1024) sort_scan_top(const RepDev* __restrict__ reps, int* d_sorted) {
  __shared__ RepDev rd;
  __shared__ StepInfo unused;
  __shared__ uint32_t wt[33];
  load_block_records(rd, unused, reps, nullptr, blockIdx.x, 0, 0);
  if (!rd.has_region) return;
  if (threadIdx.x == 0) d_sorted[blockIdx.x] = 1;   // read (and cleared) by the next prep
  uint32_t carry = 0;
  for (int base = 0; base < rd.ntile; base += blockDim.x) {
    const int t = base + threadIdx.x;
    const uint32_t x = t < rd.ntile ? rd.tsum[t] : 0u;
    uint32_t total;
    const uint32_t ex = block_exclusive_scan(x, wt, total);
    if (t < rd.ntile) rd.tsum[t] = carry + ex;
    carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0 && rd.pooled) rd.pool[2] = carry;   // live particles after the sort
}

template <int D, typename R>
__device__ __forceinline__ void sort_scatter_one(const RepDev& rd, const long long j) {
  if (j >= pool_end(rd)) return;
  const uint32_t hp = rd.home[j];
  if (hp == HOME_DEAD) return;
  const uint32_t h = home_index<D>(rd, hp);
  const long long dst = (long long)rd.tsum[h / SORT_TILE] + rd.hoff[h] + rd.rank[j];
  rd.home_alt[dst] = hp;
  rd.pid_alt[dst] = rd.pid[j];
  R o[3], v[3];
  PState<D, R>::ld(rd.off, (uint32_t)j, o);
  PState<D, R>::ld(rd.vel, (uint32_t)j, v);
  PState<D, R>::st(rd.off_alt, (uint32_t)dst, o);
  PState<D, R>::st(rd.vel_alt, (uint32_t)dst, v);
}

template <int D, typename R>
__device__ __forceinline__ void sort_scatter_item(const RepDev& rd, const int2 bm) {
#pragma unroll
  for (int p = 0; p < PPT; ++p) sort_scatter_one<D, R>(rd, (long long)bm.y * PP_ITEM + 256 * p + threadIdx.x);
}

template <int D, typename R>
__global__ void __launch_bounds__(256) sort_scatter(const RepDev* __restrict__ reps, const int2* __restrict__ bmap,
                                                    int nwork) {
  __shared__ RepDev rd;
  __shared__ StepInfo unused;
  for_each_item(bmap, nwork, reps, (const StepInfo*)nullptr, 0, 0, rd, unused,
                [&](const int2 bm) { sort_scatter_item<D, R>(rd, bm); });
}

cudaError_t launch_sort(int dim, int prec, const Launch& L, const int2* bmap_p, int nb_p, const int2* bmap_t,
                        int nb_t, int* d_sorted) {
  if (nb_p == 0) return cudaSuccess;
  static const int gc2 = grid_cap(grid_for(sort_count<2>, 256, 1 << 30)), gc3 = grid_cap(grid_for(sort_count<3>, 256, 1 << 30));
  if (dim == 2) sort_count<2><<<gc2 < nb_p ? gc2 : nb_p, 256, 0, L.stream>>>(L.reps, bmap_p, nb_p);
  else sort_count<3><<<gc3 < nb_p ? gc3 : nb_p, 256, 0, L.stream>>>(L.reps, bmap_p, nb_p);
  sort_scan_tiles<<<nb_t, SORT_TILE, 0, L.stream>>>(L.reps, bmap_t);
  sort_scan_top<<<L.nrep, 1024, 0, L.stream>>>(L.reps, d_sorted);
  static const int gs2 = grid_cap(grid_for(sort_scatter<2, float>, 256, 1 << 30));
  const int gs = nb_p < gs2 ? nb_p : gs2;
  if (dim == 2) {
    if (prec == P_FP64) sort_scatter<2, double><<<gs, 256, 0, L.stream>>>(L.reps, bmap_p, nb_p);
    else sort_scatter<2, float><<<gs, 256, 0, L.stream>>>(L.reps, bmap_p, nb_p);
  } else {
    if (prec == P_FP64) sort_scatter<3, double><<<gs, 256, 0, L.stream>>>(L.reps, bmap_p, nb_p);
    else sort_scatter<3, float><<<gs, 256, 0, L.stream>>>(L.reps, bmap_p, nb_p);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Readout order with density resampling: rank[j] = the number of live
// particles in the pool slots below j (stable, so that separate readouts of
// one state agree), ltile the per-tile totals of SORT_TILE slots, pool[2] the
// live count.
__global__ void __launch_bounds__(SORT_TILE) live_scan_tiles(RepDev rd) {
  __shared__ uint32_t wt[33];
  const long long j = (long long)blockIdx.x * SORT_TILE + threadIdx.x;
  const bool live = j < pool_end(rd) && rd.home[j] != HOME_DEAD;
  uint32_t total;
  const uint32_t ex = block_exclusive_scan(live ? 1u : 0u, wt, total);
  if (j < rd.cap) rd.rank[j] = ex;
  if (threadIdx.x == 0) rd.ltile[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) live_scan_top(RepDev rd, int ntile) {
  __shared__ uint32_t wt[33];
  uint32_t carry = 0;
  for (int base = 0; base < ntile; base += blockDim.x) {
    const int t = base + threadIdx.x;
    const uint32_t x = t < ntile ? rd.ltile[t] : 0u;
    uint32_t total;
    const uint32_t ex = block_exclusive_scan(x, wt, total);
    if (t < ntile) rd.ltile[t] = carry + ex;
    carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) rd.pool[2] = carry;
}

__global__ void live_scan_add(RepDev rd) {
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= rd.cap) return;
  rd.rank[j] += rd.ltile[j / SORT_TILE];
}

cudaError_t launch_live_index(const RepDev& rd, cudaStream_t st) {
  const int ntile = (int)((rd.cap + SORT_TILE - 1) / SORT_TILE);
  live_scan_tiles<<<ntile, SORT_TILE, 0, st>>>(rd);
  live_scan_top<<<1, 1024, 0, st>>>(rd, ntile);
  live_scan_add<<<(int)((rd.cap + 255) / 256), 256, 0, st>>>(rd);
  return cudaGetLastError();
}

// collision-cell table -> CELL_COUNT (int32) or CELL_VCM ([ncell][3] binary64)
template <int D, typename R>
__global__ void tab_out(RepDev rd, int field, void* out) {
  using T4 = typename Vec4<R>::T;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= rd.ncell) return;
  const T4 t = ((const T4*)rd.tab)[(D == 2 ? 1 : 2) * c];
  if (field == 7) {
    ((int*)out)[c] = (int)t.w;
  } else {
    double* o = (double*)out;
    o[3 * c] = (double)t.x;
    o[3 * c + 1] = (double)t.y;
    o[3 * c + 2] = D == 3 ? (double)t.z : 0.0;
  }
}

cudaError_t launch_tab_out(int dim, int prec, const RepDev& rd, int field, void* out, cudaStream_t st) {
  const int nb = (int)((rd.ncell + 255) / 256);
  if (nb == 0) return cudaSuccess;
  if (dim == 2) {
    if (prec == P_FP64) tab_out<2, double><<<nb, 256, 0, st>>>(rd, field, out);
    else tab_out<2, float><<<nb, 256, 0, st>>>(rd, field, out);
  } else {
    if (prec == P_FP64) tab_out<3, double><<<nb, 256, 0, st>>>(rd, field, out);
    else tab_out<3, float><<<nb, 256, 0, st>>>(rd, field, out);
  }
  return cudaGetLastError();
}

}  // namespace lbm
