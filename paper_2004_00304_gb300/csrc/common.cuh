// common.cuh -- device-side building blocks of the coupled LB-MPCD step:
// the counter-based generator, uniform/normal maps, lattice tables, the
// per-replica descriptor and the per-step record read by every kernel.
#pragma once
#include <utility>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <stdlib.h>

#define LBM_HD __host__ __device__ __forceinline__

namespace lbm {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11).  Counter words: (id, step, replica,
// tag), key: the 64-bit seed.  Same stream on host and device.
enum : uint32_t { TAG_SHIFT = 1, TAG_SIGN = 2, TAG_AXIS = 3, TAG_VIRT = 4,
                  TAG_RESAMPLE = 5, TAG_INIT_POS = 6, TAG_INIT_VEL = 7,
                  TAG_DENSITY = 8, TAG_SPAWN_POS = 9, TAG_SPAWN_VEL = 10,
                  TAG_AT = 11, TAG_AT_VIRT = 12, TAG_CE = 13 };
constexpr int CE_TRIES = 64;   // Chapman-Enskog redraw: attempts before the last candidate is kept

// density resampling of the outer buffer (resample_density = 1): a removed
// particle's home is HOME_DEAD until the next sort compacts the pool; a new
// particle carries PID_FRESH until its first particle pass, PID_SPAWNED after.
constexpr uint32_t HOME_DEAD = 0xFFFFFFFFu, PID_FRESH = 0xFFFFFFFEu, PID_SPAWNED = 0xFFFFFFFDu;
constexpr int SPAWN_MAX = 4;   // at most SPAWN_MAX ppc new particles per cell and step

LBM_HD uint32_t mul_hi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

LBM_HD uint4 philox(uint32_t id, uint32_t step, uint32_t rep, uint32_t tag, uint32_t k0, uint32_t k1) {
  uint32_t x = id, y = step, z = rep, w = tag;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t a = 0xD2511F53u * x, ah = mul_hi32(0xD2511F53u, x);
    const uint32_t b = 0xCD9E8D57u * z, bh = mul_hi32(0xCD9E8D57u, z);
    x = bh ^ y ^ k0;
    y = b;
    z = ah ^ w ^ k1;
    w = a;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return make_uint4(x, y, z, w);
}

// 24-bit uniform in [0,1): exact in binary32 and binary64.
LBM_HD double unit24(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }

LBM_HD float unit24f(uint32_t w) { return (float)(w >> 8) * (1.0f / 16777216.0f); }

// Box-Muller pair: u1 = (a+1) 2^-32 in (0,1], u2 = b 2^-32,
// z0 = sqrt(-2 ln u1) cos(2 pi u2), z1 = sqrt(-2 ln u1) sin(2 pi u2).
// binary64 version:
__device__ __forceinline__ void normal_pair(uint32_t a, uint32_t b, double& z0, double& z1) {
  const double u1 = ((double)a + 1.0) * (1.0 / 4294967296.0);
  const double u2 = (double)b * (1.0 / 4294967296.0);
  const double rad = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  z0 = rad * c;
  z1 = rad * s;
}
// binary32 version, within ~1e-6 of the binary64 outputs: ln u1 is logf(u1)
// for u1 < 1/2 and log1pf(-m 2^-32), m = 2^32 - 1 - a, for u1 >= 1/2, so that
// neither tail loses the bits that rounding the 32-bit word to binary32 drops.
__device__ __forceinline__ void normal_pair(uint32_t a, uint32_t b, float& z0, float& z1) {
  const float lnu = a < 0x80000000u ? logf((float)(a + 1u) * (1.0f / 4294967296.0f))
                                    : log1pf(-(float)(0xFFFFFFFFu - a) * (1.0f / 4294967296.0f));
  const float rad = sqrtf(-2.0f * lnu);
  float s, c;
  sincospif(2.0f * ((float)b * (1.0f / 4294967296.0f)), &s, &c);
  z0 = rad * c;
  z1 = rad * s;
}

// L2 eviction priority for data streamed once per step (createpolicy +
// L2::cache_hint, evict_first): the particle state, and the LB populations
// as they are read.  The populations an LB update writes keep the normal
// priority, so that they are still in L2 when the next update reads them
// (the particle state, which would crowd them out, goes first), and so do
// the cell table and sums, which every particle touches.
__device__ __forceinline__ uint64_t l2_stream() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint32_t ld_hint(const uint32_t* a, uint64_t pol) {
  uint32_t v;
  asm volatile("ld.global.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ void st_hint(uint32_t* a, uint32_t v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(a), "r"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ float2 ld_hint(const float2* a, uint64_t pol) {
  float2 v;
  asm volatile("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ void st_hint(float2* a, float2 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(a), "f"(v.x), "f"(v.y), "l"(pol)
               : "memory");
}
__device__ __forceinline__ float4 ld_hint(const float4* a, uint64_t pol) {
  float4 v;
  asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(a), "l"(pol));
  return v;
}

// ---------------------------------------------------------------------------
// Lattices: D2Q9 (the paper's, Sec. 2.1) and D3Q19.
template <int Q> struct Lattice;
template <> struct Lattice<9> {
  static constexpr int D = 2;
  LBM_HD static constexpr int cx(int i) { constexpr int t[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1}; return t[i]; }
  LBM_HD static constexpr int cy(int i) { constexpr int t[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1}; return t[i]; }
  LBM_HD static constexpr int cz(int) { return 0; }
  LBM_HD static constexpr int opp(int i) { constexpr int t[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6}; return t[i]; }
  LBM_HD static constexpr double w(int i) { return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0); }
};
template <> struct Lattice<19> {
  static constexpr int D = 3;
  LBM_HD static constexpr int cx(int i) {
    constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[i];
  }
  LBM_HD static constexpr int cy(int i) {
    constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[i];
  }
  LBM_HD static constexpr int cz(int i) {
    constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return t[i];
  }
  LBM_HD static constexpr int opp(int i) {
    constexpr int t[19] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};
    return t[i];
  }
  LBM_HD static constexpr double w(int i) { return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }
};

// ---------------------------------------------------------------------------
// Per-replica descriptor (device copy).  Every array of a replica is its own
// allocation; the kernels of one launch walk all replicas through a block map.
struct RepDev {
  // LB lattice
  int nx, ny, nz, q;
  double omega;            // 1 / tau
  double g[3];             // body acceleration
  long long nnode;         // nx ny nz
  float fp16_scale;        // binary16 deviation scale 2^k (1 for the other storages)
  float fp16_inv;
  void* f[2];              // populations [q][nnode], ping-pong by step parity
  void* rho;               // [2][nnode]     by step parity (rho_of)
  void* u;                 // [2][3][nnode]  by step parity (u_of)
  // MPCD region, cell units: [0,Wx) x [0,Hy) x [0,Wz)
  int has_region, x0, x1, Wx, Hy, Wz, r, n_out, n_in, cw, ppc, feedback, window;
  double kT, mass, sig;    // sig = sqrt(kT / m)
  double cos_a, sin_a, alpha;
  // binary32 copies of the constants the binary32 kernels use (binary64
  // arithmetic, conversions included, is slow on this GPU)
  float omega_f, g_f[3], r_f, cos_f, sin_f, kT_f, mass_f, sig_f;
  long long np;            // particles
  long long ncell;         // collision cells: Wx (Hy+1) Wz
  long long nbuf;          // inner-buffer LB nodes
  uint32_t key0, key1, rep;
  // coupling columns in cell units: outer X < xo_lo or X >= xo_hi; inner
  // [xi_lo0, xi_hi0) (left side) and [xi_lo1, xi_hi1) (right side)
  int xo_lo, xo_hi, xi_lo0, xi_hi0, xi_lo1, xi_hi1;
  // near-wall strip (Sec. 3.3): region = all columns x LB rows [1, y1); outer
  // buffer rows Y >= yo (Hy when there is no strip), inner rows [yi_lo, yi_hi)
  int strip, y1, yo, yi_lo, yi_hi;
  // pooled particles (density resampling, or a piece of a region divided
  // over x-slabs): particles live in a pool of cap slots, a removed one
  // marked HOME_DEAD; pool[0] is its end, pool[1] an overflow flag, pool[2]
  // the live count of the last sort or compaction; ltile scratch of the
  // readout compaction.  resample: density resampling (a3') itself.
  int pooled;
  int resample;
  // LB columns whose inner-buffer nodes this handle imposes on (a8): all of
  // them, or for a piece of a divided region the columns the handle owns
  int own_lo, own_hi;
  // collision rule: 0 SRD (Eq. 4), 1 MPCD-AT (Eq. 6)
  int collision;
  // outer-buffer redraw: 0 Maxwellian, 1 Chapman-Enskog
  int redraw;
  uint32_t cap;
  uint32_t* pool;
  uint32_t* ltile;
  // particles (structure of arrays); *_alt receive the sorted copy
  uint32_t* home;          // packed integer home cell
  void* off[3];            // offsets in [0,1), storage precision (2D: off[0] holds (x,y) pairs)
  void* vel[3];            // velocities, storage precision (2D: vel[0] holds (x,y) pairs)
  uint32_t* pid;           // particle id (Philox counter of the redraw)
  uint32_t* home_alt;
  void* off_alt[3];
  void* vel_alt[3];
  uint32_t* pid_alt;
  // counting sort by home cell
  long long nhome;         // Wx Hy Wz
  int ntile;               // ceil(nhome / SORT_TILE)
  uint32_t* hcount;        // [nhome] particles per home cell (zero between sorts)
  uint32_t* hoff;          // [nhome] exclusive prefix inside the tile
  uint32_t* tsum;          // [ntile] tile totals -> exclusive tile offsets
  uint32_t* rank;          // [np] rank of the particle inside its home cell
  // collision cells
  // accumulators of the current binning: binary32 storage keeps one float4
  // {n, sum vx, sum vy, sum vz} per cell in acc4 (one vector atomic per group
  // of particles); binary64 keeps acc_n and acc_v[d]
  float4* acc4;
  uint32_t* acc_n;
  void* acc_v[3];
  void* tab;               // table of the last collision, vec4 of the storage
                           // precision: 2D {vcm.x, vcm.y, sin(theta), n};
                           // 3D {vcm.x, vcm.y, vcm.z, n}, {axis.x, axis.y, axis.z, 0}
  // inner buffer sampling window (binary64)
  double* frame;           // [nbuf][4] this step's mass, momentum
  double* ring;            // [window][nbuf][4]
  double* wsum;            // [nbuf][4]
  // learned closure (feedback = 2, 2D): strips of 16 fine columns per side,
  // strip cell c = (side Hy + row) 16 + xi
  int cl_on;               // strip sampling active
  int cl_npy;              // patches per side, ceil(Hy / 16)
  int cl_p0;               // first patch of this replica in the handle's batch
  int cl_pad;
  double cl_inv_ppc, cl_inv_sig;   // 1 / ppc, 1 / sqrt(kT/m)
  int cl_interval;                 // steps between network evaluations
  int cl_first;                    // first evaluation: max(7, step of the parameter load)
  int cl_imp;                      // network loaded: the LB imposes cl_u after the first evaluation
  double* cl_u;                    // [nbuf][2] velocity imposed from the latest evaluation
  double* cframe;          // [2][2 Hy 16][4] count, sum vx, sum vy of step n in half n & 1
                           // (binary64 atomics; folded and cleared by the LB launch of n + 1)
  float* cring;            // [8][2 Hy 16][3] fields of the last 8 steps
  double* cema;            // [2 Hy 16][3] moving averages (training target)
  float* cl_y;             // network output of the handle's batch [P][16][16][3]
};

constexpr int SORT_TILE = 1024;

// rho and u of the LB update of step n: two copies, by step parity, so that
// the particle pass of step n reads them while the LB update of step n + 1
// writes the other copy
template <typename R> __device__ __forceinline__ R* rho_of(const RepDev& rd, uint32_t n) {
  return (R*)rd.rho + (long long)(n & 1u) * rd.nnode;
}
template <typename R> __device__ __forceinline__ R* u_of(const RepDev& rd, uint32_t n) {
  return (R*)rd.u + (long long)(n & 1u) * 3 * rd.nnode;
}

// end of the particle slots in use: the pool end for pooled particles, the
// fixed count otherwise
__device__ __forceinline__ uint32_t pool_end(const RepDev& rd) {
  if (!rd.pooled) return (uint32_t)rd.np;
  const uint32_t e = *(volatile const uint32_t*)rd.pool;
  return e < rd.cap ? e : rd.cap;
}

template <typename R> struct Vec4;
template <> struct Vec4<float> { using T = float4; };
template <> struct Vec4<double> { using T = double4_32a; };

// One record per (step of the chunk, replica), written by the prep kernel.
struct StepInfo {
  uint32_t n;              // global step index
  int pending;             // collision of step n-1 not yet applied to particles
  int write_moments;       // write rho/u on every node this step
  int src_alt;             // particle state of this step is in the *_alt (sorted) arrays
  int cells;               // the collision-cell table of step n - 1 is still to be built (LB launch)
  int lb_a8;               // the LB launch of step n applies a8 of step n - 1 on the inner-buffer nodes
                           // (otherwise a launch after the particle pass of step n - 1 does)
  double shift[3], prev[3];
  float shift_f[3], prev_f[3];   // the same shifts (exact in binary32)
};

// The per-replica and per-step constants in the kernel's precision.
template <typename R> struct Cst;
template <> struct Cst<double> {
  __device__ static double omega(const RepDev& d) { return d.omega; }
  __device__ static double g(const RepDev& d, int a) { return d.g[a]; }
  __device__ static double r(const RepDev& d) { return (double)d.r; }
  __device__ static double cos_a(const RepDev& d) { return d.cos_a; }
  __device__ static double sin_a(const RepDev& d) { return d.sin_a; }
  __device__ static double sig(const RepDev& d) { return d.sig; }
  __device__ static double kT_over_m(const RepDev& d) { return d.kT / d.mass; }
  __device__ static double mass(const RepDev& d) { return d.mass; }
  __device__ static const double* shift(const StepInfo& s) { return s.shift; }
  __device__ static const double* prev(const StepInfo& s) { return s.prev; }
};
template <> struct Cst<float> {
  __device__ static float omega(const RepDev& d) { return d.omega_f; }
  __device__ static float g(const RepDev& d, int a) { return d.g_f[a]; }
  __device__ static float r(const RepDev& d) { return d.r_f; }
  __device__ static float cos_a(const RepDev& d) { return d.cos_f; }
  __device__ static float sin_a(const RepDev& d) { return d.sin_f; }
  __device__ static float sig(const RepDev& d) { return d.sig_f; }
  __device__ static float kT_over_m(const RepDev& d) { return d.kT_f / d.mass_f; }
  __device__ static float mass(const RepDev& d) { return d.mass_f; }
  __device__ static const float* shift(const StepInfo& s) { return s.shift_f; }
  __device__ static const float* prev(const StepInfo& s) { return s.prev_f; }
};

// packed home cell: 2D x | y << 16 ; 3D x | y << 10 | z << 21
template <int D> struct HomePack;
template <> struct HomePack<2> {
  static constexpr int XMAX = 65535, YMAX = 65535, ZMAX = 1;
  LBM_HD static uint32_t pack(int x, int y, int) { return (uint32_t)x | ((uint32_t)y << 16); }
  LBM_HD static void unpack(uint32_t h, int& x, int& y, int& z) { x = h & 0xFFFF; y = h >> 16; z = 0; }
};
template <> struct HomePack<3> {
  static constexpr int XMAX = 1023, YMAX = 2047, ZMAX = 2047;
  LBM_HD static uint32_t pack(int x, int y, int z) {
    return (uint32_t)x | ((uint32_t)y << 10) | ((uint32_t)z << 21);
  }
  LBM_HD static void unpack(uint32_t h, int& x, int& y, int& z) {
    x = h & 0x3FF; y = (h >> 10) & 0x7FF; z = h >> 21;
  }
};

// Storage of LB populations as deviations d_i = f_i - w_i (rho0 = 1).
template <typename S> struct Store;
// 32-bit integer mix (the MurmurHash3 finaliser): the random bits of the
// stochastic rounding below; not part of the method's random numbers.
LBM_HD uint32_t mix32(uint32_t x) {
  x ^= x >> 16; x *= 0x85EBCA6Bu;
  x ^= x >> 13; x *= 0xC2B2AE35u;
  x ^= x >> 16;
  return x;
}

// binary32 -> binary16 with stochastic rounding: round up (in magnitude)
// with probability (|y| - down) / (up - down), so that the stored value is
// unbiased and updates far below one binary16 ulp (the per-step body-force
// increments) still accumulate.  For y in binary16's normal range the 13
// low mantissa bits that binary16 drops are exactly that fraction; adding 13
// uniform random bits to them and truncating toward zero rounds up with
// exactly that probability (the carry moves into the kept bits, or the
// exponent).  Below 2^-14 (binary16 subnormals: deviations under 2^-28 at the
// 2^14 scale) more bits are dropped and the rounding leans toward zero.
// h = 0 selects round-to-nearest (used when loading a state); h's top 13
// bits are the random bits.
__device__ __forceinline__ __half sr_half(float y, uint32_t h) {
  if (h == 0u) return __float2half_rn(y);
  return __float2half_rz(__uint_as_float(__float_as_uint(y) + (h >> 19)));
}

// next word of the stochastic-rounding stream of one thread (a 32-bit linear
// congruential step, Numerical Recipes' constants; its top bits are the ones
// sr_half uses); never 0, which would select round-to-nearest
__device__ __forceinline__ uint32_t sr_next(uint32_t h) { return (h * 1664525u + 1013904223u) | 1u; }

template <> struct Store<double> {
  using R = double;
  __device__ static double ld(const double* p, float) { return *p; }
  __device__ static void st(double* p, double v, float, uint32_t = 0) { *p = v; }
};
template <> struct Store<float> {
  using R = float;
  __device__ static float ld(const float* p, float) { return *p; }
  __device__ static void st(float* p, float v, float, uint32_t = 0) { *p = v; }
};
template <> struct Store<__half> {
  using R = float;   // binary16 holds d_i * scale; arithmetic in binary32
  __device__ static float ld(const __half* p, float inv) { return __half2float(*p) * inv; }
  __device__ static void st(__half* p, float v, float scale, uint32_t h = 0) { *p = sr_half(v * scale, h); }
};

// Programmatic dependent launch: a kernel launched after this one with the
// programmatic-serialization attribute may start once every block of this
// one has passed allow_dependent_launch; such a kernel calls
// wait_for_prerequisite before it ends, so that it completes only after this
// one has (and sees its writes).  Both are no-ops without such a launch.
__device__ __forceinline__ void allow_dependent_launch() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void wait_for_prerequisite() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch with or without the programmatic-serialization attribute (pdl).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), int grid, int block, cudaStream_t st, bool pdl,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// Copy a block's descriptor and step record to shared memory (all threads
// call it; it ends with a barrier).  si == nullptr skips the step record.
__device__ __forceinline__ void load_block_records(RepDev& srd, StepInfo& sst, const RepDev* reps,
                                                   const StepInfo* si, int rep, int k, int nrep) {
  const int* a = (const int*)(reps + rep);
  int* b = (int*)&srd;
  for (int i = threadIdx.x; i < (int)(sizeof(RepDev) / 4); i += blockDim.x) b[i] = a[i];
  if (si) {
    const int* c = (const int*)(si + (long long)k * nrep + rep);
    int* d = (int*)&sst;
    for (int i = threadIdx.x; i < (int)(sizeof(StepInfo) / 4); i += blockDim.x) d[i] = c[i];
  }
  __syncthreads();
}

// Walk over a block map.  Grid-stride (CONTIG = false): block b processes
// items b, b + gridDim.x, ...; contiguous (CONTIG = true): the items
// [b per, (b + 1) per), per = ceil(nwork / gridDim.x).  The map lists each
// replica's items contiguously and a block reloads the replica's records into
// shared memory only when the replica changes: with the contiguous split a
// block of the particle pass meets one replica or a few, where the
// grid-stride walk changed replica on almost every item of an ensemble of
// small replicas (a barrier and a dependent load each).  The LB launch keeps
// the grid-stride walk, so that its cell-table items, listed first, run first
// on every SM.  The body runs with the records of its item's replica.
template <bool CONTIG = false, typename Item, typename Body>
__device__ __forceinline__ void for_each_item(const Item* __restrict__ bmap, int nwork, const RepDev* reps,
                                              const StepInfo* si, int k, int nrep, RepDev& rd, StepInfo& st,
                                              Body&& body) {
  int cur = -1;
  const int per = CONTIG ? (nwork + (int)gridDim.x - 1) / (int)gridDim.x : 1;
  const int w0 = CONTIG ? (int)blockIdx.x * per : (int)blockIdx.x;
  const int w1 = CONTIG ? min(nwork, w0 + per) : nwork;
  const int dw = CONTIG ? 1 : (int)gridDim.x;
  for (int wi = w0; wi < w1; wi += dw) {
    const Item bm = bmap[wi];
    if (bm.x != cur) {
      __syncthreads();
      load_block_records(rd, st, reps, si, bm.x, k, nrep);
      cur = bm.x;
    }
    body(bm);
  }
}

// The same walks with the records read in place from global memory (through
// the read-only path; they do not change during a launch) instead of staged
// in shared memory: no barrier when the replica changes.  The body receives
// the item's records.
template <bool CONTIG = false, typename Item, typename Body>
__device__ __forceinline__ void for_each_item_direct(const Item* __restrict__ bmap, int nwork,
                                                     const RepDev* __restrict__ reps,
                                                     const StepInfo* __restrict__ si, int k, int nrep, Body&& body) {
  const int per = CONTIG ? (nwork + (int)gridDim.x - 1) / (int)gridDim.x : 1;
  const int w0 = CONTIG ? (int)blockIdx.x * per : (int)blockIdx.x;
  const int w1 = CONTIG ? min(nwork, w0 + per) : nwork;
  const int dw = CONTIG ? 1 : (int)gridDim.x;
  for (int wi = w0; wi < w1; wi += dw) {
    const Item bm = bmap[wi];
    body(reps[bm.x], si[(long long)k * nrep + bm.x], bm);
  }
}

// The same walk for single-replica launches, which take the replica record by
// value (a __grid_constant__ kernel parameter, read as constant-bank operands
// instead of shared-memory loads); only the step record is staged in shared
// memory.  The record is fixed between graph rebuilds.
// The items of a single replica are computed from their index (item_of)
// rather than read from the block map, which saves a dependent load.
template <typename ItemOf, typename Body>
__device__ __forceinline__ void for_each_item_one(ItemOf&& item_of, int nwork, const StepInfo* si, int k,
                                                  StepInfo& st, Body&& body) {
  const int* c = (const int*)(si + k);
  int* d = (int*)&st;
  for (int i = threadIdx.x; i < (int)(sizeof(StepInfo) / 4); i += blockDim.x) d[i] = c[i];
  __syncthreads();
  for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) body(item_of(wi));
}

// Resident-grid size for a kernel; LBMPCD_GRID_BLOCKS_PER_ITEM=1 in the
// environment switches every kernel to one block per work item instead
// (for measurement).
inline int grid_cap(int resident) {
  static int mode = -1;
  if (mode < 0) {
    const char* e = getenv("LBMPCD_GRID_BLOCKS_PER_ITEM");
    mode = (e && e[0] == '1') ? 1 : 0;
  }
  return mode ? (1 << 30) : resident;
}

// streaming multiprocessors of the current device (read once)
inline int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

// Blocks to launch for nwork items: enough to fill every SM at the kernel's
// occupancy, never more than the items.
template <typename K>
inline int grid_for(K kernel, int threads, int nwork) {
  const int sms = sm_count();
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, 0) != cudaSuccess || occ < 1) occ = 1;
  const long long cap = (long long)occ * sms;
  return (int)(nwork < cap ? nwork : cap);
}

}  // namespace lbm
