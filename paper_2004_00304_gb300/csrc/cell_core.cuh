// cell_core.cuh -- the per-cell half of the collision (a7) and the windowed
// MPCD -> LB imposition (a8), as work items of the LB launch of the next step.
//
// The collision-cell table of step m (v_cm with virtual wall particles, the
// rotation draw of Eq. 4, accumulators cleared) needs every particle of step
// m binned; the particles need it only in the particle pass of step m + 1.
// The LB update of step m + 1 lies between the two, so the table is built by
// extra work items of that launch instead of a kernel of its own.  The
// imposition of a8 needs the sampling frame of step m, complete only after
// the particle pass of step m; it is applied by the LB update of step m + 1
// as the collision rule of the inner-buffer nodes (post-collision populations
// f_eq(rho_LB, u_bar)), where the same thread also moves the window on.
#pragma once
#include "kernels.h"

namespace lbm {

// Cells [start, end) of the table of step m, CPT per thread (c = start + tid
// + blockDim p), all accumulator loads first.  shift_y_pos: the random shift
// of step m has a non-zero y component (only then do the wall rows of cells
// straddle a wall).
template <int Q, typename S>
__device__ __forceinline__ void cell_table_item(const RepDev& rd, uint32_t m, bool shift_y_pos, long long start,
                                                long long end) {
  using R = typename Store<S>::R;
  using T4 = typename Vec4<R>::T;
  using L = Lattice<Q>;
  constexpr int D = L::D;
  const long long c0 = start + threadIdx.x;
  const int bs = blockDim.x;
  uint32_t nn[CPT];
  R V[CPT][3];
#pragma unroll
  for (int p = 0; p < CPT; ++p) {
    const long long c = c0 + (long long)bs * p;
    const long long cl = c < end ? c : end - 1;
    if (sizeof(R) == 4) {
      const float4 g4 = rd.acc4[cl];
      nn[p] = (uint32_t)g4.x;
      V[p][0] = (R)g4.y; V[p][1] = (R)g4.z; V[p][2] = (R)g4.w;
    } else {
      nn[p] = rd.acc_n[cl];
#pragma unroll
      for (int a = 0; a < 3; ++a) V[p][a] = a < D ? ((const R*)rd.acc_v[a])[cl] : R(0);
    }
  }
#pragma unroll
  for (int p = 0; p < CPT; ++p) {
    const long long c = c0 + (long long)bs * p;
    if (c >= end) break;
    const uint32_t n = nn[p];
    R vc[3] = {R(0), R(0), R(0)}, rt[3] = {R(0), R(0), R(0)};
    if (n > 0) {
      const uint32_t ci = (uint32_t)c, row = ci / (uint32_t)rd.Wx;
      const uint32_t cy = D == 2 ? row : row % (uint32_t)(rd.Hy + 1);
      const bool cut = (cy == 0 || (cy == (uint32_t)rd.Hy && !rd.strip)) && shift_y_pos;
      if (cut && (int)n < rd.ppc) {
        // Lamura-type wall: ppc - n virtual particles at rest, summed momentum
        // drawn from N(0, (ppc - n) m kT) per component.  MPCD-AT: they are
        // members of the cell, so the sum of their random velocities (same
        // law, TAG_AT_VIRT) is taken off as well: the sums hold v - v_ran.
        const int nv = rd.ppc - (int)n;
        const uint4 w = philox((uint32_t)c, m, rd.rep, TAG_VIRT, rd.key0, rd.key1);
        R z[4];
        normal_pair(w.x, w.y, z[0], z[1]);
        normal_pair(w.z, w.w, z[2], z[3]);
        const R sd = sqrt((R)nv * Cst<R>::kT_over_m(rd));
#pragma unroll
        for (int a = 0; a < D; ++a) V[p][a] += sd * z[a];
        if (rd.collision == 1) {
          const uint4 wa = philox((uint32_t)c, m, rd.rep, TAG_AT_VIRT, rd.key0, rd.key1);
          normal_pair(wa.x, wa.y, z[0], z[1]);
          normal_pair(wa.z, wa.w, z[2], z[3]);
#pragma unroll
          for (int a = 0; a < D; ++a) V[p][a] -= sd * z[a];
        }
#pragma unroll
        for (int a = 0; a < D; ++a) vc[a] = V[p][a] / (R)rd.ppc;
      } else {
        const R inv_n = R(1) / (R)n;
#pragma unroll
        for (int a = 0; a < D; ++a) vc[a] = V[p][a] * inv_n;
      }
      if (rd.collision == 1) {
        // MPCD-AT: no rotation; the table holds v_cm - <v_ran>
      } else if (D == 2) {
        const uint4 w = philox((uint32_t)c, m, rd.rep, TAG_SIGN, rd.key0, rd.key1);
        rt[0] = (w.x >> 31) ? Cst<R>::sin_a(rd) : -Cst<R>::sin_a(rd);
      } else {
        const uint4 w = philox((uint32_t)c, m, rd.rep, TAG_AXIS, rd.key0, rd.key1);
        if (sizeof(R) == 8) {
          const double zc = 2.0 * unit24(w.x) - 1.0;
          double sp, cp;
          sincospi(2.0 * unit24(w.y), &sp, &cp);
          const double rh = sqrt(1.0 - zc * zc);
          rt[0] = (R)(rh * cp); rt[1] = (R)(rh * sp); rt[2] = (R)zc;
        } else {
          const float zc = 2.0f * unit24f(w.x) - 1.0f;
          float sp, cp;
          sincospif(2.0f * unit24f(w.y), &sp, &cp);
          const float rh = sqrtf(1.0f - zc * zc);
          rt[0] = (R)(rh * cp); rt[1] = (R)(rh * sp); rt[2] = (R)zc;
        }
      }
    }
    T4* tab = (T4*)rd.tab;
    if (D == 2) {
      T4 t; t.x = vc[0]; t.y = vc[1]; t.z = rt[0]; t.w = (R)n;
      tab[c] = t;
    } else {
      T4 t0, t1;
      t0.x = vc[0]; t0.y = vc[1]; t0.z = vc[2]; t0.w = (R)n;
      t1.x = rt[0]; t1.y = rt[1]; t1.z = rt[2]; t1.w = R(0);
      tab[2 * c] = t0;
      tab[2 * c + 1] = t1;
    }
    if (sizeof(R) == 4) {
      rd.acc4[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
#pragma unroll
      for (int a = 0; a < D; ++a) ((R*)rd.acc_v[a])[c] = R(0);
      rd.acc_n[c] = 0u;
    }
  }
}

// ---------------------------------------------------------------------------
// Learned-closure strips (feedback = 2): the particle pass of step m adds 1
// and v of every particle in a strip cell (the 16 fine columns nearest each
// x-edge of the region) to half m & 1 of the frame; the LB launch of step
// m + 1 turns it into the fields of step m, puts them in the 8-step ring and
// the moving average (the training target) and clears the half for step m + 2.
constexpr int CL_W = 16;                 // strip width and patch side, fine cells
constexpr int CL_F = 8;                  // frames in the network input
constexpr double CL_EMA_A = 1.0 / 500.0; // moving-average weight of the newest frame

__device__ __forceinline__ int cl_row0(const RepDev& rd, int py) {
  return py == rd.cl_npy - 1 ? rd.Hy - CL_W : CL_W * py;
}

// this step's fields of one strip cell from its frame {count, sum vx, sum vy}
__device__ __forceinline__ void cl_phi(const RepDev& rd, const double* fr, int side, double phi[3]) {
  const double n = fr[0];
  phi[0] = n * rd.cl_inv_ppc - 1.0;
  phi[1] = 0.0;
  phi[2] = 0.0;
  if (n > 0) {
    const double s = rd.cl_inv_sig / n;
    phi[1] = (side ? -fr[1] : fr[1]) * s;
    phi[2] = fr[2] * s;
  }
}

// ring slot n mod 8 and moving average of strip cell c
__device__ __forceinline__ void cl_update(const RepDev& rd, uint32_t n, long long c, const double phi[3]) {
  const long long ncl = 32LL * rd.Hy;
  float* ring = rd.cring + ((long long)(n & (CL_F - 1)) * ncl + c) * 3;
  double* e = rd.cema + 3 * c;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    ring[k] = (float)phi[k];
    e[k] = n == 0 ? phi[k] : e[k] + (phi[k] - e[k]) * CL_EMA_A;
  }
}

// Strip cells [start, end) of the frame of step m, one per thread.
__device__ __forceinline__ void closure_fold_item(const RepDev& rd, uint32_t m, long long start, long long end) {
  const long long ncl = 32LL * rd.Hy;
  const long long c = start + threadIdx.x;
  if (c >= end) return;
  double* fr = rd.cframe + 4 * ((m & 1) * ncl + c);
  double phi[3];
  cl_phi(rd, fr, (int)(c / (16LL * rd.Hy)), phi);
  cl_update(rd, m, c, phi);
  fr[0] = 0.0; fr[1] = 0.0; fr[2] = 0.0;
}

// Index b of the inner-buffer LB node (x, y, z) in the window arrays, or -1:
// slab  b = ((side n_in + col) nz + z)(ny - 2) + y - 1, col counted inwards
//       from the region's edge (left: x = x0 + n_out + col, right:
//       x = x1 - 1 - n_out - col);
// strip b = (row nz + z) nx + x, row counted down from the buffer's top
//       (y = y1 - 1 - n_out - row).
__device__ __forceinline__ long long inner_index(const RepDev& rd, int x, int y, int z) {
  if (rd.strip) {
    const int row = rd.y1 - 1 - rd.n_out - y;
    if (row < 0 || row >= rd.n_in) return -1;
    return ((long long)row * rd.nz + z) * rd.nx + x;
  }
  int side, col;
  if (x >= rd.x0 + rd.n_out && x < rd.x0 + rd.n_out + rd.n_in) {
    side = 0; col = x - rd.x0 - rd.n_out;
  } else if (x >= rd.x1 - rd.n_out - rd.n_in && x < rd.x1 - rd.n_out) {
    side = 1; col = rd.x1 - 1 - rd.n_out - x;
  } else {
    return -1;
  }
  return (((long long)side * rd.n_in + col) * rd.nz + z) * (rd.ny - 2) + (y - 1);
}

// Window sums of inner-buffer node b after frame m: W = W_{m-1} + frame_m -
// frame_{m-W} (binary64; the ring holds the last W frames, frame m - W in
// slot m mod W).  commit: move the window on (running sum, ring slot, frame
// cleared for the next sampling); otherwise only read.
__device__ __forceinline__ void window_sums(const RepDev& rd, uint32_t m, long long b, bool commit, double W4[4]) {
  double* fr = rd.frame + 4 * b;
  double* ws = rd.wsum + 4 * b;
  double* rg = rd.ring + 4 * ((long long)(m % (uint32_t)rd.window) * rd.nbuf + b);
  double xf[4], xw[4], xr[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) { xf[a] = fr[a]; xw[a] = ws[a]; xr[a] = rg[a]; }
#pragma unroll
  for (int a = 0; a < 4; ++a) W4[a] = xw[a] + (xf[a] - xr[a]);
  if (commit) {
#pragma unroll
    for (int a = 0; a < 4; ++a) { ws[a] = W4[a]; rg[a] = xf[a]; fr[a] = 0.0; }
  }
}

// Window mean of the last min(m + 1, W) frames in the kernel's precision:
// rho_bar = M / (ppc m r^d W_m), u_bar = P / M (0 where M = 0).  Returns M.
template <int D, typename R>
__device__ __forceinline__ R window_mean(const RepDev& rd, uint32_t m, const double W4[4], R& rho, R u[3]) {
  const uint32_t nf = min(m + 1u, (uint32_t)rd.window);
  const R rdim = (D == 3) ? (R)(rd.r * rd.r * rd.r) : (R)(rd.r * rd.r);
  const R M = (R)W4[0];
  rho = M / ((R)rd.ppc * (R)Cst<R>::mass(rd) * rdim * (R)nf);
  u[0] = u[1] = u[2] = R(0);
  if (M > R(0)) {
    const R iM = R(1) / M;
    u[0] = (R)W4[1] * iM; u[1] = (R)W4[2] * iM; u[2] = (R)W4[3] * iM;
  }
  return M;
}

}  // namespace lbm
