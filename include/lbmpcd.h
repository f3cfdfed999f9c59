/*
 * lbmpcd.h -- C ABI of the GB300 (sm_103a) coupled lattice Boltzmann /
 * multiparticle-collision-dynamics time stepper (liblbmpcd.so).
 *
 * The method is that of Montessori, Tiribocchi, Lauricella and Succi, "A
 * coupled lattice Boltzmann-multiparticle collision method for
 * multi-resolution hydrodynamics": the LB equation (Eq. 1) with the
 * second-order equilibrium (Eq. 2) runs on the whole channel; MPCD particles
 * (streaming Eq. 3, stochastic-rotation collision Eq. 4) run in a sub-region;
 * a coupling buffer of whole LB columns on each side of the sub-region passes
 * LB -> MPCD by redrawing particle velocities from a Maxwellian about the
 * (interpolated) LB velocity (Sec. 2.3, Algorithms 1 and 2) and MPCD -> LB by
 * imposing equilibrium populations built from windowed cell moments.
 *
 * Conventions shared by every entry point:
 *  - return 0 on success, a negative LBMPCD_ERR_* code on failure; no C++
 *    exception ever crosses this boundary; lbmpcd_last_error() gives text;
 *  - the library owns all device memory it allocates; callers own every
 *    pointer they pass in (params, region bounds, dst/src buffers);
 *  - a handle is not thread-safe; all its work is ordered on the CUDA stream
 *    given at creation (NULL = the legacy default stream);
 *  - units are LB units: spacing 1, time step 1; MPCD cells have side 1/refine.
 *
 * Geometry: LB node (x,y,z) covers [x,x+1)x[y,y+1)x[z,z+1); rows y = 0 and
 * y = ny-1 are solid (half-way bounce-back walls at y = 1 and y = ny-1),
 * x and z are periodic.  The MPCD sub-region is a slab of LB columns
 * [x0,x1) over all fluid rows and all z.
 */
#ifndef LBMPCD_H
#define LBMPCD_H
#include <stddef.h>
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

enum { LBMPCD_D2Q9 = 9, LBMPCD_D3Q19 = 19 };
/* LB population storage / particle arithmetic.  FP64: binary64 everywhere.
 * FP32: populations stored as binary32 deviations f_i - w_i rho0, particles
 * as integer cell + binary32 offset.  FP16DEV: populations stored as scaled
 * binary16 deviations, arithmetic in binary32, particles as for FP32. */
enum { LBMPCD_FP64 = 0, LBMPCD_FP32 = 1, LBMPCD_FP16DEV = 2 };

enum {
  LBMPCD_OK = 0,
  LBMPCD_ERR_INVALID_ARG = -1,
  LBMPCD_ERR_OOM = -2,
  LBMPCD_ERR_CUDA = -3,
  LBMPCD_ERR_TIMEOUT = -4,
  LBMPCD_ERR_STATE = -5,
  LBMPCD_ERR_CAPACITY = -6
};

/* Field ids for lbmpcd_get_fields / lbmpcd_set_state.  Element type is
 * double for floating-point fields and int32 for integer ones, whatever the
 * storage precision; shapes are per replica:
 *  RHO [nz][ny][nx], U [3][nz][ny][nx]    LB density / velocity of the last
 *                                         step (moments of the streamed
 *                                         populations, u with the half-force
 *                                         shift); Eq. 1-2, Sec. 2.1
 *  POPS [q][nz][ny][nx]                   stored post-collision populations f_i
 *  PART_POS [np][3] (double)              offset of each particle in its cell, [0,1)
 *  PART_VEL [np][3] (double)              particle velocities (LB units)
 *  PART_CELL [np] (int32)                 collision cell of the last binning
 *  SHIFT [3] (double)                     last random grid shift, cell units
 *  CELL_COUNT [ncell] (int32)             particles per collision cell, last binning
 *  WINDOW_MEAN [nbuf][4] (double)         rho_bar, u_bar of the inner buffer nodes
 *  DIAG [9] (double)                      LB mass, LB momentum (3), particle count,
 *                                         particle momentum (3), kinetic energy
 *  PART_HOME [np][3] (int32)              integer home cell of each particle
 *  CELL_VCM [ncell][3] (double)           centre-of-mass velocity of the last collision (MPCD-AT: v_cm - <v_ran>)
 *  PART_ID [np] (int32)                   identity: particle fields come back in id order
 *                                         (with resample_density = 1: the live particles
 *                                         in pool order, the same for every field read
 *                                         between two steps; PART_ID is the initial index
 *                                         or -3 for particles created by the resampling)
 *  CELL_LIST [np] (int32)                 cell lists of the last binning: for the collision
 *                                         cells in increasing id, the rows of the particle
 *                                         fields (= particle ids without resampling) of its
 *                                         particles in increasing order; cell c's entries
 *                                         start at the sum of CELL_COUNT below c (assembled
 *                                         on the host from PART_CELL)
 *  CLOSURE_IN [P][16][16][24] (double)    learned-closure network input of the last step
 *  CLOSURE_OUT [P][16][16][3] (double)    network output of the last step (with parameters)
 *  CLOSURE_TARGET [P][16][16][3] (double) moving averages of the strip fields (training target)
 *                                         -- the three CLOSURE fields exist with feedback = 2;
 *                                         P = 2 ceil(Hy/16) patches, see lbmpcd_set_closure
 * Collision cells: ncell = Wx (Hy+1) Wz, id = cx + Wx (cy + (Hy+1) cz), with
 * Wx = (x1-x0) refine, Hy = (ny-2) refine (a near-wall strip: (y1-1) refine),
 * Wz = nz refine (1 in 2D).
 * Inner buffer nodes: nbuf = 2 * floor(cw/2) * (ny-2) * nz, index
 * ((side * floor(cw/2) + col) * nz + z) * (ny-2) + (y-1); for a near-wall
 * strip floor(cw/2) * nz * nx, index (row * nz + z) * nx + x. */
enum {
  LBMPCD_RHO = 0, LBMPCD_U = 1, LBMPCD_POPS = 2, LBMPCD_PART_POS = 3, LBMPCD_PART_VEL = 4,
  LBMPCD_PART_CELL = 5, LBMPCD_SHIFT = 6, LBMPCD_CELL_COUNT = 7, LBMPCD_WINDOW_MEAN = 8,
  LBMPCD_DIAG = 9, LBMPCD_PART_HOME = 10, LBMPCD_CELL_VCM = 11, LBMPCD_PART_ID = 12,
  LBMPCD_CLOSURE_IN = 13, LBMPCD_CLOSURE_OUT = 14, LBMPCD_CLOSURE_TARGET = 15, LBMPCD_CELL_LIST = 17
};

typedef struct lbmpcd lbmpcd; /* opaque handle */

/* Problem statement of one replica (Sec. 2-3 of the paper; Table 1 lists the
 * same quantities).  All replicas of one handle share lattice and precision. */
typedef struct {
  int lattice;          /* LBMPCD_D2Q9 (nz must be 1) or LBMPCD_D3Q19 (Sec. 2.1) */
  int nx, ny, nz;       /* LB nodes, walls included in ny */
  double tau;           /* BGK relaxation time, nu = (tau - 1/2)/3 (Sec. 2.1) */
  double force[3];      /* body acceleration g driving the flow (Sec. 3) */
  int refine;           /* r = LB spacing / MPCD cell side a (Sec. 2.3, Algorithm 2) */
  int ppc;              /* mean particles per MPCD cell (Table 1 "N") */
  double alpha;         /* SRD rotation angle, radians (Eq. 4) */
  double kT, mass;      /* MPCD thermal energy and particle mass (Eq. 4-5, Algorithm 1) */
  int coupling_width;   /* LB columns of coupling buffer per side (2 in Sec. 2.3) */
  int precision;        /* LBMPCD_FP64 | LBMPCD_FP32 | LBMPCD_FP16DEV */
  int feedback;         /* 0: one-way LB -> MPCD as in the paper; 1: plus windowed MPCD -> LB;
                           2: plus MPCD -> LB from the learned closure (D2Q9; lbmpcd_set_closure) */
  int window;           /* samples in the averaging window (Table 1 N_s) */
  int resample_density; /* 0: outer-buffer velocities redrawn, particles kept (the paper, Sec. 2.3);
                           1: outer-buffer particles replaced each step by
                           N = stochastic-round(ppc rho_LB) new ones (see below) */
  uint64_t seed;        /* Philox key */
  int collision;        /* 0: SRD, stochastic rotation (Eq. 4); 1: MPCD-AT, Andersen thermostat
                           (Eq. 6, the rule the paper's runs use; see below).  All replicas of a
                           handle share it; 1 excludes resample_density = 1 */
  int redraw;           /* 0: Maxwellian redraw of the outer buffer (Algorithm 1); 1: Chapman-Enskog
                           redraw carrying the LB's non-equilibrium momentum flux (the Enskog
                           sampling Sec. 2.3 names for strong gradients; see below).  1 excludes
                           resample_density = 1 and LBMPCD_FP16DEV */
} lbmpcd_params;

/* Chapman-Enskog redraw (redraw = 1): the peculiar velocity C = v - u_fine of a
 * redrawn particle follows f_MB(C; kT/m) (1 + b : zz), z = C / sqrt(kT/m),
 * b = pi' / (2 kT/m), where pi' is the traceless part (over the MPCD
 * dimensions) of (1 - 1/(2 tau)) Pi_neq / rho and Pi_neq = sum_i (f_i - f_i^eq)
 * c_i c_i over the populations of the LB node holding the cell after this
 * step's streaming, so that <C C> = (kT/m) I + pi'.  Acceptance-rejection:
 * attempt t takes z from the Box-Muller normals of Philox(particle id, n,
 * replica, 13 + 16 t) (3D: z2 from words 2, 3) and U = (w >> 8) 2^-24 of
 * word 2 (3D: word 0 of Philox(..., 14 + 16 t)), accepted when
 * A U <= 1 + b : zz, A = 1 + 30 max |b_ab|; after 64 rejections the last
 * candidate is kept. */

/* MPCD-AT (collision = 1): each particle leaves the collision with
 * v_cm + v_ran - <v_ran>, v_ran a fresh Maxwellian velocity (variance kT/m per
 * component, Box-Muller of Philox(particle id, n, replica, 11)), the mean over
 * its collision cell.  In a wall-cut cell with n_c < ppc the ppc - n_c virtual
 * particles are members of the cell: their velocity sum (Philox tag 4, as for
 * SRD) enters v_cm and the sum of their random velocities (tag 12) enters
 * <v_ran>.  Field CELL_VCM then holds v_cm - <v_ran>.  The persistent launch
 * form is not available in this mode. */

/* Density resampling (resample_density = 1; a reading of "resampling from the
 * local LB density": the paper keeps its particles and redraws velocities):
 * each step, before streaming, every particle whose home cell lies in an
 * outer-buffer column is removed and each outer-buffer cell c (home-cell
 * index X + Wx (Y + Hy Z)) receives N = floor(x) + [u < x - floor(x)] new
 * particles, x = ppc rho_LB of the LB node holding the cell, u from
 * Philox(c, n, replica, 8), at most 4 ppc; particle k has uniform offsets
 * from Philox(c 4 ppc + k, n, replica, 9) and velocity u_fine + sqrt(kT/m) xi
 * (Box-Muller of Philox(c 4 ppc + k, n, replica, 10)).  Particles live in a
 * pool with room for 65 steps of new particles at twice the mean rate,
 * compacted at the start of every call and graph chunk; lbmpcd_step returns
 * ERR_CAPACITY (results invalid) if it ever fills, and synchronises the
 * stream to check.  Particle state cannot be loaded (lbmpcd_set_state) and
 * the persistent launch form is not available in this mode. */

/* Create a handle holding n_replicas independent channels; params points to
 * n_replicas structs (replica i uses params[i]).  cuda_stream is a
 * cudaStream_t (NULL for the default stream).  LB populations start at
 * f_eq(rho = 1, u = 0).  Errors: INVALID_ARG (bad sizes / mixed lattice or
 * precision), OOM, CUDA.  On failure *out is NULL. */
int lbmpcd_create(const lbmpcd_params* params, int n_replicas, void* cuda_stream, lbmpcd** out);

/* Declare the MPCD sub-region of a replica (LB node bounds, half-open).  Two
 * forms (lo[1] <= 1 and z spanning 0..nz in both):
 *  - slab of whole columns, hi[1] >= ny - 1: LB columns [lo[0], hi[0]), all
 *    fluid rows; periodic in x inside the region; coupling buffers of
 *    coupling_width columns at both x-ends (Sec. 2.3);
 *  - near-wall strip, hi[1] = y1 < ny - 1 (the two-level geometry of Sec. 3.3):
 *    all columns (lo[0] = 0, hi[0] = nx, periodic in x) and LB rows [1, y1);
 *    the coupling buffer lies along the top edge: the outer ceil(cw/2) rows
 *    below y1 are redrawn from the LB, the inner floor(cw/2) rows under them
 *    are sampled and (feedback = 1) imposed, WINDOW_MEAN entries ordered
 *    (row from the buffer's top, z, x).  The top edge is not a wall: particles
 *    reaching it are reflected specularly (v_y -> -v_y) and its cut cells get
 *    no virtual particles.  Needs y1 - 1 > coupling_width; not with
 *    feedback = 2 or resample_density = 1.
 * Seeds ppc particles in every MPCD cell with offsets uniform in the cell and
 * Maxwellian velocities (variance kT/m).  Must precede the first lbmpcd_step
 * (else ERR_STATE).  Errors: INVALID_ARG (bounds of neither form, region
 * narrower than 2 coupling widths, cell index range too large), OOM, CUDA. */
int lbmpcd_set_region(lbmpcd* h, int replica, const int lo[3], const int hi[3]);

/* A piece of a slab region divided over x-slabs of one channel (Sec. 3.1.1:
 * larger systems call for a parallel implementation; one handle per slab).
 * lo / hi: the whole region in this handle's LB columns, which may extend
 * beyond [0, nx) (the region is cut by the slab); the particles, the cells,
 * the coupling buffers and the periodic wrap in x are those of the whole
 * region, in its own cell coordinates.  [own_lo, own_hi) (inside [0, nx)):
 * the LB columns this handle owns, the only ones whose inner-buffer nodes it
 * imposes on (a8).  [keep_lo, keep_hi): the region cell columns (modulo the
 * region's width Wx = (hi[0] - lo[0]) r, a range of at most Wx) whose
 * particles this handle keeps: its own columns and the ghost columns around
 * them.  The whole region is seeded exactly as lbmpcd_set_region seeds it
 * (same particle ids, positions and velocities) and the particles outside
 * the kept columns are removed, so a set of pieces holds the undivided run's
 * particles.  Particles are pooled (lbmpcd_set_particles replaces them);
 * their read-outs list the live particles with their ids (PART_ID).  Not for
 * near-wall strips, the learned closure, density resampling, MPCD-AT or the
 * Chapman-Enskog redraw, nor the persistent launch form (INVALID_ARG).
 * Errors: as lbmpcd_set_region, plus INVALID_ARG for an empty owned range or
 * kept range. */
int lbmpcd_set_region_piece(lbmpcd* h, int replica, const int lo[3], const int hi[3], int own_lo, int own_hi,
                            int keep_lo, int keep_hi);

/* Replace the pooled particles of a replica (a region piece) by n given ones,
 * host arrays: home cell (X, Y, Z) int32 [n][3] in region cells, offsets in
 * [0, 1) and velocities binary64 [n][3] (the read-out layouts of PART_HOME,
 * PART_POS and PART_VEL), ids int32 [n] (PART_ID); the state is taken as
 * after the collision of the last step (a pending collision of the particles
 * replaced is applied to them first, and the collision-cell table built).
 * Used by the x-slab driver to hand particles between the pieces of a
 * divided region (Sec. 3.1.1).  Errors: INVALID_ARG (bad replica, count,
 * null array; a home cell outside the region or an offset outside [0, 1):
 * that particle is dropped), STATE (not a pooled replica), CAPACITY (n above
 * the pool), CUDA. */
int lbmpcd_set_particles(lbmpcd* h, int replica, long long n, const int* home, const double* off, const double* vel,
                         const int* pid);

/* Advance every replica by nsteps coupled time steps (one step = LB
 * stream-collide, interpolation + Maxwellian redraw in the outer buffer, MPCD
 * streaming, inner-buffer sampling, random-shift binning, SRD collision,
 * imposition).  A replica without a region runs the LB part only.
 * Asynchronous on the handle's stream.  Errors: INVALID_ARG, CUDA. */
int lbmpcd_step(lbmpcd* h, int nsteps);

/* Same work as lbmpcd_step, launched without graph replay and with a CUDA
 * event pair on the handle's stream around every kernel; adds each kernel
 * family's elapsed milliseconds to phase_ms[0..5] = {prep, lb_pull,
 * particle_pass, cell_pass, particle sort, learned closure} (caller-owned,
 * 6 entries; not zeroed here) and the number of kernel launches to *launches (may be NULL).  Synchronises the stream.  For
 * measurement only: the per-kernel events add small gaps between kernels.
 * Errors: INVALID_ARG, CUDA. */
int lbmpcd_step_profiled(lbmpcd* h, int nsteps, double* phase_ms, long long* launches);

/* Copy one field of one replica (layouts above) to dst, which holds exactly
 * `bytes` bytes (else INVALID_ARG); dst_on_device = 1 for device memory.
 * A host dst is filled through a device staging buffer that the handle keeps
 * between calls, grown to the largest host array seen and released by
 * lbmpcd_destroy (pinned host memory copies fastest).  Synchronises the
 * handle's stream before returning. */
int lbmpcd_get_fields(lbmpcd* h, int replica, int field, void* dst, size_t bytes, int dst_on_device);

/* Load POPS, PART_POS, PART_VEL or PART_HOME of one replica from src (same
 * layouts and element types as get_fields; particle arrays in id order; a
 * host src goes through the handle's staging buffer, as for get_fields), or
 * start the LB from a velocity field: U [3][nz][ny][nx] sets the populations
 * of every node to f_eq(rho0 = 1, u) (Eq. 2).
 * Positions must satisfy 0 <= offset < 1 and lie inside the region.  Errors:
 * INVALID_ARG (field, size, values), STATE (particles before set_region). */
int lbmpcd_set_state(lbmpcd* h, int replica, int field, const void* src, size_t bytes, int src_on_device);

/* Halo exchange of the x-slab decomposition of one channel over ranks (not
 * in the paper, which runs one domain; the LB update of Sec. 2.1 is local
 * to a node and its neighbours, so a channel cut into slabs of whole
 * columns, each held by one rank with H ghost columns per side, runs H
 * pull steps exactly between two exchanges of H columns per cut).
 * Populations of LB columns [x, x + ncols), all q, z and y, of the buffer
 * the next step reads, in the handle's storage: binary64 f_i; binary32
 * deviations f_i - w_i; binary16 deviations times 2^14
 * (lbmpcd_population_bytes gives 8, 4 or 2).  Layout [q][nz][ny][ncols],
 * ncols values per row.  dst / src are caller-owned, host or device
 * (flag); the copy is exact (raw storage), between handles of the same
 * lattice, precision and ny, nz.  Synchronous on the handle's stream.
 * Errors: INVALID_ARG (NULL handle or buffer, bad replica, columns outside
 * [0, nx)), CUDA. */
int lbmpcd_population_bytes(const lbmpcd* h);
int lbmpcd_get_columns(lbmpcd* h, int replica, int x, int ncols, void* dst, int dst_on_device);
int lbmpcd_set_columns(lbmpcd* h, int replica, int x, int ncols, const void* src, int src_on_device);

/* Tensor-core GEMM of the learned closure (not a step of the paper's method):
 * C[M][N] = alpha * A[M][K] B[N][K]^T + beta * C, A and B bf16 with K
 * contiguous, C fp32 with row stride N; all device pointers, launched on
 * `stream` (a cudaStream_t, may be NULL).  M a multiple of 128, N of 16
 * (<= 4096), K of 64, else INVALID_ARG.  err_dev is a device int set to 1 if
 * a bounded wait inside the kernel gave up (C then invalid).  Asynchronous. */
int lbmpcd_tc_gemm_bf16(const void* A, const void* B, float* C, int M, int N, int K, float alpha, float beta,
                        int* err_dev, void* stream);

/* The learned closure network (not in the paper; the MPCD->LB feedback of
 * the coupled step may use it in place of the long averaging window): a
 * 3x3 convolutional net 24 -> 64 -> 64 -> 64 -> 3 channels on 16 x 16 patches
 * of MPCD cells, ReLU between layers; the output is the mean of its 8 input
 * frames plus the last layer's output less that output's mean over the 16
 * rows of each patch column (per field), so that every column mean of every
 * predicted field is that of the 8-frame mean and the closure cannot add or
 * drain mass or momentum on average in any column of the coupling strip (the
 * head's bias therefore has no effect and a zero gradient);
 * bf16 weights and activations, fp32 accumulation, every contraction on the
 * tcgen05 tensor cores.  Tensors are fp32, NHWC, device pointers: input
 * x[P][16][16][24] (frame f, field c at channel 3f + c: density deviation
 * n/ppc - 1, u_x / sqrt(kT/m), u_y / sqrt(kT/m)), output / target
 * [P][16][16][3].  Parameters: one fp32 vector, per layer W[cout][3][3][cin]
 * then b[cout].  All calls synchronise the net's stream; a bounded wait that
 * gave up inside a kernel returns ERR_TIMEOUT. */
typedef struct lbmpcd_net lbmpcd_net;
long long lbmpcd_net_num_params(void);
int lbmpcd_net_create(int max_patches, void* cuda_stream, lbmpcd_net** out);
/* which = 0 parameters, 1 gradient of the last backward / train step */
int lbmpcd_net_get_params(lbmpcd_net* net, float* dst, long long count, int which, int dst_on_device);
int lbmpcd_net_set_params(lbmpcd_net* net, const float* src, long long count, int src_on_device);
int lbmpcd_net_forward(lbmpcd_net* net, const float* x_dev, int patches, float* y_dev);
/* forward, then the MSE loss against t and its parameter gradient */
int lbmpcd_net_backward(lbmpcd_net* net, const float* x_dev, const float* t_dev, int patches, float* loss_host);
/* backward plus one Adam step (beta 0.9, 0.999, eps 1e-8) with rate lr */
int lbmpcd_net_train_step(lbmpcd_net* net, const float* x_dev, const float* t_dev, int patches, float lr,
                          float* loss_host);
void lbmpcd_net_destroy(lbmpcd_net* net);

/* Allocation-free network forward (no counterpart in the paper): the same
 * output as lbmpcd_net_forward for parameters theta_dev (device fp32, the
 * layout above), input x_dev and output y_dev (device fp32), with every piece
 * of scratch in one device array of the library (about 4 MiB) reserved when
 * the module loads.  No call allocates or frees device or host memory, which
 * is what a caller needs that already holds nearly all of the GPU's memory in
 * its own pool (a PyTorch caching allocator, a solver that reserves HBM up
 * front) and so cannot risk a hidden cudaMalloc failing, or that steps in a
 * loop where cudaMalloc / cudaFree may synchronise the device.
 *  - patches in [1, LBMPCD_NET_STATIC_MAX_PATCHES], else ERR_CAPACITY (larger
 *    batches: call once per slice of at most that many patches); NULL
 *    pointers or patches < 1: ERR_INVALID_ARG.
 *  - Runs on `stream` (a cudaStream_t, may be NULL) and synchronises it
 *    before returning, so it cannot be called while that stream is being
 *    captured into a graph (the call then fails with ERR_CUDA); a bounded
 *    wait that gave up returns ERR_TIMEOUT.
 *  - The scratch's error word must be zero when the GEMMs start: each call
 *    clears it itself, first on its stream.  Nothing else in the scratch is
 *    read before the call writes it, so no state carries between calls.
 *  - The first call on a device looks up the scratch address
 *    (cudaGetSymbolAddress) and sets the GEMM kernels' shared-memory limit:
 *    make it with that device current, before any stream capture begins.
 *  - One scratch per device: calls that overlap in time on the same device
 *    (two host threads, or two streams) race on it and give wrong results;
 *    serialise them. */
#define LBMPCD_NET_STATIC_MAX_PATCHES 8
int lbmpcd_net_forward_noalloc(const float* theta_dev, const float* x_dev, int patches, float* y_dev,
                               void* cuda_stream);

/* The learned closure in the coupled step (feedback = 2; not in the paper,
 * which couples one way).  Every step, right after streaming (the instant of
 * the inner-buffer sampling), the particles in the 16 fine columns nearest
 * each x-edge of the region ("strips"; xi = distance from the edge, the right
 * strip seen in a mirror so its u_x changes sign) give per fine cell
 *     phi_0 = n/ppc - 1,  phi_1 = +-(sum v_x / n)/sqrt(kT/m),  phi_2 = (sum v_y / n)/sqrt(kT/m)
 * (velocities 0 in an empty cell).  The fields of the last 8 steps (zeros
 * before step 0), oldest first, are the 24 input channels of the network's
 * 16 x 16 patches: side-major, ceil(Hy/16) per side, patch py covering fine
 * rows 16 py .. 16 py + 15 except the last, which covers Hy-16 .. Hy-1.  The
 * training target is the moving average e <- e + (phi - e)/500 (e = phi at
 * step 0; the mean lag and white-noise variance of a 1000-step trailing mean).
 * With parameters loaded, the network runs on steps n0, n0 + K, n0 + 2K, ...
 * (K = interval >= 1, n0 = max(7, the step count at the load)), the patches of
 * all replicas as one batch; from n0 on every step gives each inner-buffer LB
 * node f_eq(rho_LB, u_bar), u_bar = sqrt(kT/m) times the latest prediction's
 * mean velocity over the node's r x r fine cells (fine row R read from patch
 * min(R/16, ceil(Hy/16)-1)).  K = 1 evaluates every step; K = 8 once per
 * window of 8 input frames.  Needs >= 32 fine columns and >= 16 fine rows in
 * the region, refine in {1, 2, 4, 8} and coupling_width * refine <= 16
 * (set_region returns INVALID_ARG otherwise).
 *
 * Load the network parameters (layout of lbmpcd_net_get_params, count =
 * lbmpcd_net_num_params()) from host or device memory; theta = NULL unloads
 * them, leaving the sampling only (one-way coupling plus the CLOSURE fields:
 * the mode that records training data).  CLOSURE_OUT holds the latest
 * prediction.  With parameters loaded,
 * lbmpcd_step synchronises the stream at its end and returns ERR_TIMEOUT if a
 * bounded wait inside the network's tensor-core kernels gave up.  Errors:
 * STATE (no replica with feedback = 2 and a region), INVALID_ARG, CUDA. */
int lbmpcd_set_closure(lbmpcd* h, const float* theta, long long count, int src_on_device, int interval);

/* Launch form of the step (batching of the step launches; not in the paper).  mode 0
 * (default): per-kernel launches over all replicas, captured once into CUDA
 * graphs of 1, 2, 3, ..., 64 steps (a call replays one graph per 64 steps
 * and one for the rest).  By default mode 0 runs the overlapped
 * form: the LB update of step n + 1, which needs only the populations of
 * step n, runs beside the particle pass of step n (launched as a
 * programmatic dependent of the pass, taking its row tiles from a work
 * counter, with the pass capped at blocks_per_sm blocks per SM -- 0 = the
 * occupancy limit, where the LB blocks take the SMs the pass's blocks leave
 * as they finish), and a third launch per step builds the
 * collision-cell table and applies the MPCD->LB imposition of step n.  The
 * learned closure, density resampling, the Chapman-Enskog redraw and the
 * TMA-staged LB rows run the serial form instead (one LB launch carrying
 * the previous step's table and imposition, then the particle pass), as does
 * every run with flags & LBMPCD_LAUNCH_SERIAL.  mode 1: each chunk of steps is
 * one persistent cooperative kernel running the LB and particle phases per
 * step with a grid barrier between phases (bounded waits: a barrier that
 * times out ends the launch and lbmpcd_step returns ERR_TIMEOUT), captured
 * into the chunk's graph when the driver allows the capture, launched
 * directly otherwise; lbmpcd_step then synchronises the stream at its end;
 * blocks_per_sm: persistent blocks per SM (0 = the occupancy limit).  Every
 * form computes the same results (same per-step records, same item code,
 * the same operations in the same order per element).  Mode 1 is not
 * available with the learned closure, density resampling, MPCD-AT or the
 * Chapman-Enskog redraw (INVALID_ARG).  flags: LBMPCD_LAUNCH_LB_TMA runs the
 * LB update of D2Q9 binary32 channels (4 nodes per thread) with its source
 * rows staged in shared memory by bulk (TMA) copies, three rows ahead per
 * block; ignored for other lattices and precisions.  A bounded wait in that
 * kernel that gives up is reported by the next lbmpcd_get_fields as
 * ERR_TIMEOUT. */
#define LBMPCD_LAUNCH_LB_TMA 1   /* flags: D2Q9 binary32 LB rows staged by bulk (TMA) copies */
#define LBMPCD_LAUNCH_SERIAL 2   /* flags: mode 0 without the overlapped form */
int lbmpcd_set_launch_mode(lbmpcd* h, int mode, int blocks_per_sm, int flags);

/* Poll limit of the grid-barrier waits of the persistent launch form (mode 1;
 * not a step of the paper's method): a block that has polled the barrier this
 * many times without the other blocks arriving gives up, records the failure
 * and leaves the launch, and every block that sees the record leaves at its
 * next barrier, so lbmpcd_step returns LBMPCD_ERR_TIMEOUT instead of the GPU
 * hanging.  polls = 0 restores the default (2^24 polls, seconds of waiting).
 * A small limit makes the waits run out on purpose, which is how the tests
 * drive this error path; the step's results are then invalid, the barrier
 * words are reset and the handle can be stepped or destroyed as usual. */
int lbmpcd_set_wait_limit(lbmpcd* h, unsigned polls);

/* Time the launch forms {mode 0 with the default LB row width (overlapped,
 * with the particle pass at the occupancy limit, 6 and 7 blocks per SM where
 * the overlapped form applies, and serial), with TMA rows (where they apply), with
 * one LB node per thread; mode 1 at the occupancy limit and with one block per
 * SM} for `steps` steps each (after a 64-step
 * warm-up) on a fresh copy of the handle built from the same parameters and
 * regions -- the handle's own state is not touched -- and keep the fastest.
 * choice (may be NULL) receives {mode, blocks_per_sm, LB nodes per thread,
 * flags, candidates timed}.  Needs the memory of a second handle for the
 * duration of the call.  Errors: INVALID_ARG, OOM, CUDA. */
int lbmpcd_autotune(lbmpcd* h, int steps, int choice[5]);

/* Element count of a field for a replica (or a negative error code). */
long long lbmpcd_field_size(const lbmpcd* h, int replica, int field);

/* Release every resource of the handle; NULL is accepted. */
void lbmpcd_destroy(lbmpcd* h);

/* Text of the last error on this handle (never NULL; "" when none).  With
 * h == NULL, the last error of a failed lbmpcd_create on this thread. */
const char* lbmpcd_last_error(const lbmpcd* h);

#ifdef __cplusplus
}
#endif
#endif
