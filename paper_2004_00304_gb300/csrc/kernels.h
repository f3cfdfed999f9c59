// kernels.h -- host-side launchers of the device kernels (one translation
// unit per kernel family, called by the C ABI in lbmpcd_api.cu).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include "common.cuh"

typedef struct lbmpcd_net lbmpcd_net;

namespace lbm {

// precision codes (match LBMPCD_FP64 / FP32 / FP16DEV)
enum { P_FP64 = 0, P_FP32 = 1, P_FP16 = 2 };

constexpr int PPT = 2;                       // particles per thread in particle_pass (swept: 2, 4, 8)
constexpr int PP_ITEM = 256 * PPT;           // particles per work item
constexpr int CPT = 4;                       // collision cells per thread in cell_pass

struct Launch {
  const RepDev* reps;     // device descriptor table
  int nrep;
  const StepInfo* si;     // device [kcount][nrep]
  cudaStream_t stream;
  int* err;               // set by a kernel whose bounded wait gave up
  const RepDev* host;     // host copy of the table (single-replica kernels take it by value)
};

// a1: fused pull stream + BGK collide (+ Guo force, bounce-back walls).
// vec = nodes per thread (lb_vector_width); one vec for all replicas of a handle.
// tma: D2Q9 binary32 rows of 4 nodes per thread staged by bulk copies
// (lb_tma_ok); same 512-node tiles as vec 4.
int lb_vector_width(int q, int prec, int nx);
bool lb_tma_ok(int q, int prec, int vec);
cudaError_t launch_lb(int q, int prec, int vec, bool tma, const Launch& L, const int4* bmap, int nblocks, int k);

// The overlapped form of a step (the LB update of step n + 1 runs beside the
// particle pass of step n, which it does not depend on):
// launch_lb_rows: the LB row items of step slot k, launched as a programmatic
// dependent of the particle pass just launched on the same stream (it starts
// while the pass runs, takes its rows from the work counter ctr[k], and ends
// only after the pass has); launch_lb_items: a kernel over a map of non-row
// LB items (closure strip frame, collision-cell table, a8) of step slot k,
// after both (pdl: as a programmatic dependent of the rows just launched).
cudaError_t launch_lb_rows(int q, int prec, int vec, const Launch& L, const int4* bmap, int nwork, int k, int* ctr);
cudaError_t launch_lb_items(int q, int prec, const Launch& L, const int4* bmap, int nwork, int k, bool pdl);

// prep: per-step records (shift, pending flag) for kcount steps.  d_sorted[r]
// (set by the sort, cleared here) says that replica r's current particle state
// is the sorted copy in the *_alt arrays, which the chunk's first step reads.
cudaError_t launch_prep(int dim, const Launch& L, StepInfo* si, int kcount, int* d_sorted, uint32_t* d_step,
                        int* d_pending, int* d_cells, double* d_last_shift, int overlap, int* ctr);

// counting sort of the particles by home cell into the *_alt arrays; sets
// d_sorted[r] for every replica with a region.
cudaError_t launch_sort(int dim, int prec, const Launch& L, const int2* bmap_p, int nb_p, const int2* bmap_t,
                        int nb_t, int* d_sorted);

// collision-cell table -> CELL_COUNT (field 7, int32) or CELL_VCM (field 11, [ncell][3] binary64).
cudaError_t launch_tab_out(int dim, int prec, const RepDev& rd, int field, void* out, cudaStream_t st);

// a7(n-1) + a2 + a3 + a4 + a6 + a5 over every particle; bps > 0 caps the
// blocks per SM (the overlapped form), 0 takes the occupancy limit.
cudaError_t launch_particles(int dim, int prec, bool rs, bool at, bool ce, const Launch& L, const int2* bmap,
                             int nblocks, int k, int bps, bool pdl = false);

// a7 cell part of step m (v_cm, virtual particles, rotation draw) for the
// read-outs between calls (the step builds it inside the next LB launch).
cudaError_t launch_cell_table(int q, int prec, const RepDev& rd, uint32_t m, bool shift_y_pos, cudaStream_t st);

// WINDOW_MEAN after step m ([nbuf][4] binary64).
cudaError_t launch_window_out(int dim, int prec, const RepDev& rd, uint32_t m, double* out, cudaStream_t st);

// learned closure (feedback = 2): the LB launch folds the strip frames into
// the ring and moving averages and imposes the latest prediction;
// closure_step runs the network on evaluation steps; read-outs of input and
// target after step n.
struct NetMeta { long long woff[4], boff[4]; };
struct ClosureNet {                 // what closure_step reads of the network
  const __nv_bfloat16* img;         // weight images (net_fused.cuh layout)
  const float* theta;               // fp32 parameters (biases)
  NetMeta meta;
  int* err;                         // set when a bounded wait gave up
};
cudaError_t launch_closure_step(int prec, const Launch& L, const int4* ptab, int P, int k, const ClosureNet& cn);
cudaError_t launch_closure_in_out(const RepDev& rd, uint32_t n, double* out, cudaStream_t st);
cudaError_t launch_closure_target_out(const RepDev& rd, uint32_t n, double* out, cudaStream_t st);

// the closure network (closure.cu) as the coupled step uses it: input and
// output buffers of the handle's batch, weights cast once per parameter load,
// and the forward pass of P resident patches on a given stream.
float* net_input(lbmpcd_net* n);
float* net_output(lbmpcd_net* n);
int net_capacity(lbmpcd_net* n);
int net_load_params(lbmpcd_net* n, const float* theta, int on_device);
cudaError_t net_forward_resident(lbmpcd_net* n, int P, cudaStream_t st);
ClosureNet net_closure(lbmpcd_net* n);
int net_error(lbmpcd_net* n, cudaStream_t st);

// persistent form of a chunk: kcount steps of lb_pull (with the cell-table
// items) -> particle_pass in one cooperative launch with bounded grid
// barriers between phases (bar: two zeroed words, err: set on a barrier
// timeout, spin: polls before a barrier wait gives up, 0 for the default).
// The LB map has 256-thread row tiles.  blocks_per_sm <= 0 takes the
// occupancy limit.
struct PersistentMaps {
  const int4* lb; int nb_lb;
  const int2* p; int nb_p;
  unsigned* bar;
  int* err;
  unsigned spin;
};
cudaError_t launch_persistent(int q, int prec, int vec, const Launch& L, int kcount, const PersistentMaps& m,
                              int blocks_per_sm, int* grid_out);

// a3' (density resampling): new particles of the outer-buffer cells, before
// the particle pass of the same step; readout order of the pooled particles
// (rank, pool[2] = live count).
cudaError_t launch_spawn(int dim, int prec, const Launch& L, const int2* bmap, int nwork, int k);
cudaError_t launch_live_index(const RepDev& rd, cudaStream_t st);

// pieces of a region divided over x-slabs: keep the particles of home cell
// columns [lo, hi) mod Wx (the others removed); replace the pooled particles
// by n given ones (device arrays: home [n][3] int32, offsets and velocities
// [n][3] binary64, ids [n] int32; *bad set for a value out of range).
cudaError_t launch_keep_columns(int dim, const RepDev& rd, int lo, int hi, cudaStream_t st);
cudaError_t launch_pool_in(int dim, int prec, const RepDev& rd, long long n, const int* home, const double* off,
                           const double* vel, const int* pid, int* bad, cudaStream_t st);

// apply the pending collision of the last step to every particle of a replica.
cudaError_t launch_flush(int dim, int prec, const RepDev* rd_dev, const RepDev& rd, const double* last_shift,
                         cudaStream_t st);

// seed particles of a replica (ppc per cell, Maxwellian velocities).
cudaError_t launch_init_particles(int dim, int prec, const RepDev* rd_dev, const RepDev& rd, cudaStream_t st);

// copy-out / copy-in helpers (binary64 / int32 host-facing layouts).
cudaError_t launch_pops_out(int q, int prec, const RepDev& rd, int parity, double* out, cudaStream_t st);
cudaError_t launch_pops_in(int q, int prec, const RepDev& rd, const double* in, cudaStream_t st);
cudaError_t launch_pops_from_u(int q, int prec, const RepDev& rd, const double* u, cudaStream_t st);
cudaError_t launch_fill_real(int prec, void* dst, long long n, double value, cudaStream_t st);
cudaError_t launch_real_out(int prec, const void* src, long long n, double* out, cudaStream_t st);
cudaError_t launch_part_out(int dim, int prec, const RepDev& rd, int field, const double* last_shift,
                            void* out, cudaStream_t st);
cudaError_t launch_part_in(int dim, int prec, const RepDev& rd, int field, const void* in, int* bad,
                           cudaStream_t st);
cudaError_t launch_diag_lb(int q, int prec, const RepDev& rd, int parity, double* out4, cudaStream_t st);
cudaError_t launch_diag_particles(int dim, int prec, const RepDev& rd, double* out9, cudaStream_t st);

}  // namespace lbm
