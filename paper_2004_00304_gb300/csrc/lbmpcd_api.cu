// lbmpcd_api.cu -- the C ABI declared in include/lbmpcd.h.
//
// A handle owns R replicas.  Every replica's arrays are separate device
// allocations described by a RepDev record; one device table of these records
// plus a block map per kernel family lets a single launch of each kernel
// cover all replicas.  lbmpcd_step runs the steps in chunks of KCHUNK steps
// and one chunk of what is left of a call; every chunk length (a prep kernel
// plus the step kernels) is captured once into a CUDA graph and replayed.
// The step kernels are, in the serial form, lb_pull (which also builds the
// collision-cell table of step n - 1 and applies its MPCD -> LB imposition)
// then particle_pass; in the overlapped form (the default where it applies)
// the LB rows of step n + 1 run beside the particle pass of step n and a
// third launch builds the table and applies the imposition of step n.  The
// particles are sorted by home cell whenever KCHUNK steps have passed since
// the last sort, between chunks.  With the learned closure (feedback = 2) the
// network runs as one more kernel (closure_step) on its evaluation steps.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbmpcd.h"
#include "kernels.h"

using namespace lbm;

namespace {
constexpr int KCHUNK = 64;   // longest captured chunk; steps between particle sorts
constexpr int NGRAPH = KCHUNK;   // chunk graphs of 1, 2, 3, ..., KCHUNK steps
thread_local std::string g_create_error;
}  // namespace

struct lbmpcd {
  std::vector<lbmpcd_params> P;
  int nrep = 0, q = 9, dim = 2, prec = 0, lbvec = 1;
  cudaStream_t stream = nullptr;
  std::vector<RepDev> rd;
  std::vector<std::vector<void*>> rep_allocs;   // per replica, region arrays
  std::vector<void*> allocs;                    // handle-wide
  RepDev* d_reps = nullptr;
  int4* bm_lb = nullptr;
  int2 *bm_p = nullptr, *bm_t = nullptr;
  int4* ptab = nullptr;                         // closure patches of the batch: (replica, side, py)
  int4* bm_lb256 = nullptr;                     // LB map with 256-thread row tiles (persistent kernel)
  int nb_lb256 = 0;
  // overlapped form: LB row items alone; the items of the launch after the
  // particle pass of step n (closure strip frame, table and a8 of step n),
  // without a8 for the last step of a chunk
  int4 *bm_rows = nullptr, *bm_c = nullptr, *bm_c_last = nullptr;
  int nb_rows = 0, nb_c = 0, nb_c_last = 0;
  bool serial = false;                          // overlapped form switched off (LBMPCD_LAUNCH_SERIAL)
  int ov_bps = 0;                               // particle-pass blocks per SM in the overlapped form (0: default)
  int* d_ctr = nullptr;                         // [KCHUNK] work counters of the overlapped LB rows
  int2* bm_s = nullptr;                         // outer-buffer cells of the density resampling
  int nb_s = 0;
  int mode = 0;                                 // 0: per-kernel launches in graphs, 1: persistent
  bool at = false;                              // replicas collide by MPCD-AT (Eq. 6)
  bool ce = false;                              // some replica redraws by Chapman-Enskog
  bool lb_tma = false;                          // D2Q9 binary32 LB rows staged by bulk copies
  int pers_bps = 0;                             // persistent blocks per SM (0: occupancy limit)
  bool pers_graph = true;                       // the persistent launch captures into a graph
  unsigned* d_bar = nullptr;                    // grid barrier: count, generation, error
  unsigned bar_spin = 0;                        // polls before a barrier wait gives up (0: default)
  int nb_lb = 0, nb_p = 0, nb_t = 0, n_ptab = 0;
  bool has_cl = false;                          // some replica samples closure strips (feedback = 2)
  lbmpcd_net* net = nullptr;                    // learned closure, batch of all replicas' patches
  int cl_P = 0;                                 // patches in the batch
  bool cl_params = false;                       // parameters loaded: impose from the network
  std::vector<float> cl_theta;                  // host copy of the parameters
  StepInfo* d_si = nullptr;
  uint32_t* d_step = nullptr;
  int* d_pending = nullptr;
  int* d_cells = nullptr;                       // per replica: the cell table of the last step is not built yet
  double* d_last_shift = nullptr;
  int* d_flag = nullptr;
  long long nstep = 0;
  bool maps_dirty = true;
  std::vector<char> pending;                    // host mirror of d_pending
  std::vector<char> cells;                      // host mirror of d_cells
  cudaGraphExec_t graphs[NGRAPH] = {};          // chunk of i + 1 steps (no closure network)
  cudaGraphExec_t g_eval = nullptr;             // one step with the closure network
  cudaGraphExec_t g_period = nullptr;           // `period` steps, the network on every K-th from the first
  int period = 0;                               // K floor(KCHUNK / K) for K <= KCHUNK, else 0
  bool graphs_ready = false;
  int* d_sorted = nullptr;                      // per replica: the sort ran since the last chunk
  long long last_sort = 0;                      // step count at the last sort (the seeded state is sorted)
  void* stage = nullptr;                        // device staging buffer of the host-side set / get calls
  size_t stage_cap = 0;
  std::string err;
};

static int fail(lbmpcd* h, int code, const std::string& msg) {
  if (h) h->err = msg; else g_create_error = msg;
  return code;
}
static int cuda_fail(lbmpcd* h, cudaError_t e, const char* where) {
  return fail(h, LBMPCD_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// The device buffer through which host arrays are set and read, kept by the
// handle and grown to the largest request: an allocation and a release per
// call cost milliseconds for the particle fields, and every cudaFree waits
// for the whole device.  Only the handle's stream uses it; the stream is
// synchronised first, so that no copy of an earlier call that returned early
// on an error is still in flight.
static cudaError_t staging(lbmpcd* h, size_t bytes, void** out) {
  cudaError_t s = cudaStreamSynchronize(h->stream);
  if (s != cudaSuccess) return s;
  if (bytes > h->stage_cap) {
    if (h->stage) {
      cudaError_t e = cudaFree(h->stage);
      h->stage = nullptr;
      h->stage_cap = 0;
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaMalloc(&h->stage, bytes);
    if (e != cudaSuccess) { h->stage = nullptr; return e; }
    h->stage_cap = bytes;
  }
  *out = h->stage;
  return cudaSuccess;
}
#define CK(h, call)                                            \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);   \
  } while (0)

static size_t real_size(int prec) { return prec == P_FP64 ? 8 : 4; }
static size_t store_size(int prec) { return prec == P_FP64 ? 8 : (prec == P_FP32 ? 4 : 2); }

static cudaError_t dalloc(std::vector<void*>& list, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) { *p = nullptr; return e; }
  list.push_back(*p);
  return cudaMemset(*p, 0, bytes);
}

static void free_list(std::vector<void*>& list) {
  for (void* p : list) cudaFree(p);
  list.clear();
}

// the captured chunks hold the kernels' arguments: drop them when those change
static void drop_graphs(lbmpcd* h) {
  for (auto& g : h->graphs)
    if (g) { cudaGraphExecDestroy(g); g = nullptr; }
  for (auto* g : {&h->g_eval, &h->g_period})
    if (*g) { cudaGraphExecDestroy(*g); *g = nullptr; }
  h->period = 0;
  h->graphs_ready = false;
}

extern "C" void lbmpcd_destroy(lbmpcd* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream); else cudaDeviceSynchronize();
  drop_graphs(h);
  if (h->net) lbmpcd_net_destroy(h->net);
  for (auto& l : h->rep_allocs) free_list(l);
  free_list(h->allocs);
  if (h->stage) cudaFree(h->stage);
  delete h;
}

extern "C" const char* lbmpcd_last_error(const lbmpcd* h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

static int validate(const lbmpcd_params& p, std::string& why) {
  if (p.lattice != LBMPCD_D2Q9 && p.lattice != LBMPCD_D3Q19) { why = "lattice must be 9 or 19"; return 0; }
  if (p.nx < 1 || p.ny < 3 || p.nz < 1) { why = "need nx >= 1, ny >= 3, nz >= 1"; return 0; }
  if (p.lattice == LBMPCD_D2Q9 && p.nz != 1) { why = "D2Q9 needs nz == 1"; return 0; }
  if ((long long)p.nx * p.ny * p.nz > (1LL << 31)) { why = "lattice too large"; return 0; }
  if (!(p.tau > 0.5)) { why = "tau must exceed 1/2"; return 0; }
  if (p.refine < 1 || p.refine > 16) { why = "refine must be in [1,16]"; return 0; }
  if (p.ppc < 1) { why = "ppc must be >= 1"; return 0; }
  if (!(p.kT >= 0) || !(p.mass > 0)) { why = "need kT >= 0, mass > 0"; return 0; }
  if (p.coupling_width < 0) { why = "coupling_width must be >= 0"; return 0; }
  if (p.precision < 0 || p.precision > 2) { why = "precision must be 0, 1 or 2"; return 0; }
  if (p.feedback < 0 || p.feedback > 2) { why = "feedback must be 0, 1 or 2"; return 0; }
  if (p.feedback == 2 && (p.lattice != LBMPCD_D2Q9 || !(p.kT > 0)))
    { why = "feedback = 2 (learned closure) needs D2Q9 and kT > 0"; return 0; }
  if (p.window < 1) { why = "window must be >= 1"; return 0; }
  if (p.resample_density < 0 || p.resample_density > 1) { why = "resample_density must be 0 or 1"; return 0; }
  if (p.collision < 0 || p.collision > 1) { why = "collision must be 0 (SRD) or 1 (MPCD-AT)"; return 0; }
  // MPCD-AT draws by particle id, and density resampling gives new particles no id
  if (p.collision == 1 && p.resample_density)
    { why = "collision = 1 (MPCD-AT) cannot be combined with resample_density = 1"; return 0; }
  if (p.redraw < 0 || p.redraw > 1) { why = "redraw must be 0 (Maxwellian) or 1 (Chapman-Enskog)"; return 0; }
  if (p.redraw == 1 && (p.resample_density || p.precision == LBMPCD_FP16DEV))
    { why = "redraw = 1 (Chapman-Enskog) needs resample_density = 0 and FP64 or FP32 storage"; return 0; }
  return 1;
}

extern "C" int lbmpcd_create(const lbmpcd_params* params, int n_replicas, void* cuda_stream, lbmpcd** out) {
  if (out) *out = nullptr;
  if (!params || !out || n_replicas < 1 || n_replicas > 65535)
    return fail(nullptr, LBMPCD_ERR_INVALID_ARG, "null argument or bad replica count");
  std::string why;
  for (int r = 0; r < n_replicas; ++r) {
    if (!validate(params[r], why)) return fail(nullptr, LBMPCD_ERR_INVALID_ARG, "replica " + std::to_string(r) + ": " + why);
    if (params[r].lattice != params[0].lattice || params[r].precision != params[0].precision ||
        params[r].collision != params[0].collision)
      return fail(nullptr, LBMPCD_ERR_INVALID_ARG, "all replicas must share lattice, precision and collision rule");
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(nullptr, LBMPCD_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  lbmpcd* h = new (std::nothrow) lbmpcd();
  if (!h) return fail(nullptr, LBMPCD_ERR_OOM, "host allocation failed");
  h->P.assign(params, params + n_replicas);
  h->nrep = n_replicas;
  h->q = params[0].lattice;
  h->dim = h->q == 9 ? 2 : 3;
  h->prec = params[0].precision;
  h->at = params[0].collision == 1;
  for (int r = 0; r < n_replicas; ++r) h->ce = h->ce || params[r].redraw == 1;
  h->stream = (cudaStream_t)cuda_stream;
  h->rd.resize(n_replicas);
  h->rep_allocs.resize(n_replicas);
  h->pending.assign(n_replicas, 0);
  h->cells.assign(n_replicas, 0);
  const size_t ss = store_size(h->prec), rs = real_size(h->prec);
  h->lbvec = 4;
  for (int r = 0; r < n_replicas; ++r) h->lbvec = std::min(h->lbvec, lb_vector_width(h->q, h->prec, params[r].nx));
  for (int r = 0; r < n_replicas; ++r) {
    const lbmpcd_params& p = params[r];
    RepDev& d = h->rd[r];
    memset(&d, 0, sizeof(d));
    d.nx = p.nx; d.ny = p.ny; d.nz = p.nz; d.q = h->q;
    d.omega = 1.0 / p.tau;
    for (int a = 0; a < 3; ++a) d.g[a] = p.force[a];
    if (h->dim == 2) d.g[2] = 0.0;
    d.nnode = (long long)p.nx * p.ny * p.nz;
    // binary16 deviations are stored times 2^14: |d| up to ~0.5 stays below the
    // binary16 maximum and increments down to ~1e-8 stay in its normal range
    d.fp16_scale = h->prec == P_FP16 ? 16384.0f : 1.0f;
    d.fp16_inv = 1.0f / d.fp16_scale;
    d.r = p.refine; d.ppc = p.ppc; d.cw = p.coupling_width;
    d.n_out = (p.coupling_width + 1) / 2; d.n_in = p.coupling_width / 2;
    d.feedback = p.feedback; d.window = p.window;
    d.collision = p.collision;
    d.redraw = p.redraw;
    d.kT = p.kT; d.mass = p.mass; d.sig = sqrt(p.kT / p.mass);
    d.alpha = p.alpha; d.cos_a = cos(p.alpha); d.sin_a = sin(p.alpha);
    d.omega_f = (float)d.omega; d.r_f = (float)p.refine;
    d.cos_f = (float)d.cos_a; d.sin_f = (float)d.sin_a;
    d.kT_f = (float)p.kT; d.mass_f = (float)p.mass; d.sig_f = (float)d.sig;
    for (int a = 0; a < 3; ++a) d.g_f[a] = (float)d.g[a];
    d.key0 = (uint32_t)(p.seed & 0xFFFFFFFFu); d.key1 = (uint32_t)(p.seed >> 32); d.rep = (uint32_t)r;
    std::vector<void*>& L = h->allocs;
    e = dalloc(L, &d.f[0], h->q * d.nnode * ss);
    if (e == cudaSuccess) e = dalloc(L, &d.f[1], h->q * d.nnode * ss);
    if (e == cudaSuccess) e = dalloc(L, &d.rho, 2 * d.nnode * rs);   // two copies by step parity
    if (e == cudaSuccess) e = dalloc(L, &d.u, 2 * 3 * d.nnode * rs);
    if (e == cudaSuccess) e = launch_fill_real(h->prec, d.rho, 2 * d.nnode, 1.0, nullptr);   // rho0 = 1
    if (e != cudaSuccess) {
      int code = e == cudaErrorMemoryAllocation ? LBMPCD_ERR_OOM : LBMPCD_ERR_CUDA;
      std::string m = std::string("allocating LB arrays: ") + cudaGetErrorString(e);
      lbmpcd_destroy(h);
      return fail(nullptr, code, m);
    }
  }
  void* tmp = nullptr;
  e = dalloc(h->allocs, &tmp, sizeof(RepDev) * n_replicas); h->d_reps = (RepDev*)tmp;
  if (e == cudaSuccess) { e = dalloc(h->allocs, &tmp, sizeof(StepInfo) * KCHUNK * n_replicas); h->d_si = (StepInfo*)tmp; }
  if (e == cudaSuccess) { e = dalloc(h->allocs, &tmp, sizeof(uint32_t)); h->d_step = (uint32_t*)tmp; }
  if (e == cudaSuccess) { e = dalloc(h->allocs, &tmp, sizeof(int) * n_replicas); h->d_pending = (int*)tmp; }
  if (e == cudaSuccess) { e = dalloc(h->allocs, &tmp, sizeof(int) * n_replicas); h->d_sorted = (int*)tmp; }
  if (e == cudaSuccess) { e = dalloc(h->allocs, &tmp, sizeof(int) * n_replicas); h->d_cells = (int*)tmp; }
  if (e == cudaSuccess) { e = dalloc(h->allocs, &tmp, sizeof(double) * 3 * n_replicas); h->d_last_shift = (double*)tmp; }
  if (e == cudaSuccess) { e = dalloc(h->allocs, &tmp, sizeof(int) * 16); h->d_flag = (int*)tmp; }
  if (e == cudaSuccess) { e = dalloc(h->allocs, &tmp, sizeof(unsigned) * 4); h->d_bar = (unsigned*)tmp; }
  if (e == cudaSuccess) { e = dalloc(h->allocs, &tmp, sizeof(int) * KCHUNK); h->d_ctr = (int*)tmp; }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    std::string m = std::string("allocating handle arrays: ") + cudaGetErrorString(e);
    lbmpcd_destroy(h);
    return fail(nullptr, LBMPCD_ERR_CUDA, m);
  }
  *out = h;
  return LBMPCD_OK;
}

// Block maps, one work item per entry, each replica's items contiguous:
// LB (replica, tile, y, z), preceded by the replica's cell-table items
// (replica, -1 - b, 0, 0) for block b of blockDim CPT collision cells (the
// table of the previous step, built in the same launch); particles / sort
// (replica, block of PP_ITEM particles); sort tiles (replica, tile of
// SORT_TILE home cells).
template <typename T>
static int upload_map(lbmpcd* h, T** dst, int* cnt, const std::vector<T>& src) {
  if (*dst) {
    cudaFree(*dst);
    for (auto it = h->allocs.begin(); it != h->allocs.end(); ++it)
      if (*it == (void*)*dst) { h->allocs.erase(it); break; }
    *dst = nullptr;
  }
  *cnt = (int)src.size();
  if (src.empty()) return LBMPCD_OK;
  void* p = nullptr;
  CK(h, dalloc(h->allocs, &p, sizeof(T) * src.size()));
  *dst = (T*)p;
  CK(h, cudaMemcpy(p, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
  return LBMPCD_OK;
}

// The closure network holds the patches of every replica with strip sampling
// in one batch; it is (re)created when the batch outgrows it.
static int closure_batch(lbmpcd* h) {
  int P = 0;
  for (int r = 0; r < h->nrep; ++r) {
    RepDev& d = h->rd[r];
    if (!d.cl_on) continue;
    d.cl_p0 = P;
    P += 2 * d.cl_npy;
  }
  h->cl_P = P;
  if (P == 0) return LBMPCD_OK;
  if (!h->net || net_capacity(h->net) < P) {
    if (h->net) { CK(h, cudaStreamSynchronize(h->stream)); lbmpcd_net_destroy(h->net); h->net = nullptr; }
    const int rc = lbmpcd_net_create(P, h->stream, &h->net);
    if (rc) return fail(h, rc, "creating the closure network");
    if (h->cl_params) {
      const int rc2 = net_load_params(h->net, h->cl_theta.data(), 0);
      if (rc2) return fail(h, rc2, "loading the closure parameters");
    }
  }
  for (int r = 0; r < h->nrep; ++r) {
    RepDev& d = h->rd[r];
    if (!d.cl_on) continue;
    d.cl_y = net_output(h->net);
  }
  return LBMPCD_OK;
}

static int build_maps(lbmpcd* h) {
  int rc0 = closure_batch(h);
  if (rc0) return rc0;
  std::vector<int4> lb;
  std::vector<int2> pp, tt, sp;
  std::vector<int4> pt, lb256, rows_only, cit, cit_last;
  h->has_cl = false;
  for (int r = 0; r < h->nrep; ++r) {
    const RepDev& d = h->rd[r];
    if (d.cl_on) {   // closure strip cells: the frame of the previous step folded into ring and average
      const long long ncl = 32LL * d.Hy;
      for (long long b = 0; b < (ncl + 127) / 128; ++b) lb.push_back(make_int4(r, (int)(-1 - b), -1, 0));
      for (long long b = 0; b < (ncl + 255) / 256; ++b) lb256.push_back(make_int4(r, (int)(-1 - b), -1, 0));
      h->has_cl = true;
    }
    if (d.has_region) {   // cell-table items first: their accumulators are still in L2
      for (long long b = 0; b < (d.ncell + 128 * CPT - 1) / (128 * CPT); ++b) lb.push_back(make_int4(r, (int)(-1 - b), 0, 0));
      for (long long b = 0; b < (d.ncell + 256 * CPT - 1) / (256 * CPT); ++b) lb256.push_back(make_int4(r, (int)(-1 - b), 0, 0));
      // the overlapped form's items of step n after its particle pass (bm.w = 1):
      // a8 of the inner-buffer nodes first (the longest chain of dependent
      // loads) and only in the map for steps that are not the last of their
      // chunk; strip frame and table in both maps
      for (long long b = 0; b < (d.nbuf + 127) / 128; ++b) cit.push_back(make_int4(r, (int)(-1 - b), -2, 1));
      for (auto* m : {&cit, &cit_last}) {
        if (d.cl_on)
          for (long long b = 0; b < (32LL * d.Hy + 127) / 128; ++b) m->push_back(make_int4(r, (int)(-1 - b), -1, 1));
        for (long long b = 0; b < (d.ncell + 128 * CPT - 1) / (128 * CPT); ++b)
          m->push_back(make_int4(r, (int)(-1 - b), 0, 1));
      }
    }
    // row items for blocks of bd threads: tiles of one row, or 2^k whole rows
    // per item where a row has tpr = nx / vec threads, tpr a power of two
    // below bd (not for the TMA-staged form, which stages one row per item)
    auto rows = [&](std::vector<int4>& out, int bd) {
      const int tpr = d.nx / h->lbvec;
      int k = 0;
      if (!h->lb_tma && tpr < bd && (tpr & (tpr - 1)) == 0)
        while ((tpr << (k + 1)) <= bd) ++k;
      const int ntx = k ? 1 : (tpr + bd - 1) / bd;
      for (int z = 0; z < d.nz; ++z)
        for (int y = 1; y < d.ny - 1; y += 1 << k)
          for (int t = 0; t < ntx; ++t) out.push_back(make_int4(r, t, y, z | (k << 24)));
    };
    rows(lb, 128);
    rows(lb256, 256);
    rows(rows_only, 128);
    if (!d.has_region) continue;
    const long long nslot = d.pooled ? (long long)d.cap : d.np;
    const long long npb = (nslot + PP_ITEM - 1) / PP_ITEM;
    for (long long b = 0; b < npb; ++b) pp.push_back(make_int2(r, (int)b));
    for (int b = 0; b < d.ntile; ++b) tt.push_back(make_int2(r, b));
    if (d.resample) {
      const long long nouter = (long long)(d.xo_lo + (d.Wx - d.xo_hi)) * d.Hy * d.Wz;
      for (long long b = 0; b < (nouter + 255) / 256; ++b) sp.push_back(make_int2(r, (int)b));
    }
    if (d.cl_on) {
      for (int side = 0; side < 2; ++side)
        for (int py = 0; py < d.cl_npy; ++py) pt.push_back(make_int4(r, side, py, 0));   // batch order
    }
  }
  int rc = upload_map(h, &h->bm_lb, &h->nb_lb, lb);
  if (!rc) rc = upload_map(h, &h->bm_p, &h->nb_p, pp);
  if (!rc) rc = upload_map(h, &h->bm_t, &h->nb_t, tt);
  if (!rc) rc = upload_map(h, &h->ptab, &h->n_ptab, pt);
  if (!rc) rc = upload_map(h, &h->bm_lb256, &h->nb_lb256, lb256);
  if (!rc) rc = upload_map(h, &h->bm_s, &h->nb_s, sp);
  if (!rc) rc = upload_map(h, &h->bm_rows, &h->nb_rows, rows_only);
  if (!rc) rc = upload_map(h, &h->bm_c, &h->nb_c, cit);
  if (!rc) rc = upload_map(h, &h->bm_c_last, &h->nb_c_last, cit_last);
  if (rc) return rc;
  CK(h, cudaMemcpy(h->d_reps, h->rd.data(), sizeof(RepDev) * h->nrep, cudaMemcpyHostToDevice));
  drop_graphs(h);
  h->maps_dirty = false;
  return LBMPCD_OK;
}

// piece = {own_lo, own_hi, keep_lo, keep_hi} for a piece of a region divided
// over x-slabs (lbmpcd_set_region_piece), else null
static int set_region_impl(lbmpcd* h, int replica, const int lo[3], const int hi[3], const int* piece) {
  if (!h) return LBMPCD_ERR_INVALID_ARG;
  if (replica < 0 || replica >= h->nrep || !lo || !hi) return fail(h, LBMPCD_ERR_INVALID_ARG, "bad replica or null bounds");
  if (h->nstep > 0) return fail(h, LBMPCD_ERR_STATE, "set_region must precede the first step");
  RepDev& d = h->rd[replica];
  const lbmpcd_params& p = h->P[replica];
  if (d.has_region) return fail(h, LBMPCD_ERR_STATE, "region already set for this replica");
  const int x0 = lo[0], x1 = hi[0];
  if (!(lo[1] <= 1 && lo[2] <= 0 && hi[2] >= p.nz))
    return fail(h, LBMPCD_ERR_INVALID_ARG, "region must start at the bottom wall and span all z");
  // hi[1] below the top wall: the near-wall strip of Sec. 3.3 (all columns,
  // LB rows [1, hi[1]), coupling buffer along its top edge)
  const bool strip = hi[1] < p.ny - 1;
  const int y1 = strip ? hi[1] : p.ny - 1;
  if (strip) {
    if (x0 != 0 || x1 != p.nx)
      return fail(h, LBMPCD_ERR_INVALID_ARG, "a near-wall strip spans all columns");
    if (y1 - 1 <= p.coupling_width)
      return fail(h, LBMPCD_ERR_INVALID_ARG, "near-wall strip not taller than its coupling buffer");
    if (p.feedback == 2 || p.resample_density)
      return fail(h, LBMPCD_ERR_INVALID_ARG, "a near-wall strip runs neither the learned closure nor density resampling");
  } else if ((!piece && (x0 < 0 || x1 > p.nx)) || x1 - x0 < 2 * p.coupling_width || x1 <= x0) {
    return fail(h, LBMPCD_ERR_INVALID_ARG, "region columns out of range or narrower than two coupling widths");
  }
  if (piece) {
    if (strip) return fail(h, LBMPCD_ERR_INVALID_ARG, "a near-wall strip is not divided into pieces");
    if (p.feedback == 2 || p.resample_density || p.redraw == 1 || p.collision == 1)
      return fail(h, LBMPCD_ERR_INVALID_ARG,
                  "a piece of a region runs neither the learned closure, density resampling, the Chapman-Enskog "
                  "redraw nor MPCD-AT");
    if (piece[0] < 0 || piece[1] > p.nx || piece[0] >= piece[1] || x0 < -(1 << 20) || x1 > (1 << 20))
      return fail(h, LBMPCD_ERR_INVALID_ARG, "owned columns of a piece must be a non-empty range of the lattice");
  }
  d.x0 = x0; d.x1 = x1;
  d.strip = strip ? 1 : 0; d.y1 = y1;
  d.Wx = (x1 - x0) * p.refine; d.Hy = (y1 - 1) * p.refine; d.Wz = h->dim == 3 ? p.nz * p.refine : 1;
  const bool fits = h->dim == 2 ? (d.Wx <= HomePack<2>::XMAX && d.Hy <= HomePack<2>::YMAX)
                                : (d.Wx <= HomePack<3>::XMAX + 1 && d.Hy <= HomePack<3>::YMAX + 1 &&
                                   d.Wz <= HomePack<3>::ZMAX + 1);
  if (!fits) return fail(h, LBMPCD_ERR_INVALID_ARG, "region has more cells per axis than the packed home index holds");
  d.nhome = (long long)d.Wx * d.Hy * d.Wz;
  d.ntile = (int)((d.nhome + SORT_TILE - 1) / SORT_TILE);
  d.np = d.nhome * p.ppc;
  {
    const int r = p.refine, w = x1 - x0;
    if (strip) {   // buffer rows under the top edge; no buffer columns
      d.xo_lo = 0; d.xo_hi = d.Wx;
      d.xi_lo0 = d.xi_hi0 = d.xi_lo1 = d.xi_hi1 = 0;
      d.yo = d.Hy - d.n_out * r;
      d.yi_lo = d.Hy - p.coupling_width * r; d.yi_hi = d.yo;
    } else {
      d.xo_lo = d.n_out * r; d.xo_hi = (w - d.n_out) * r;
      d.xi_lo0 = d.n_out * r; d.xi_hi0 = p.coupling_width * r;
      d.xi_lo1 = (w - p.coupling_width) * r; d.xi_hi1 = (w - d.n_out) * r;
      d.yo = d.Hy;
      d.yi_lo = d.yi_hi = 0;
    }
  }
  if (d.np >= (1LL << 32) - 1) return fail(h, LBMPCD_ERR_INVALID_ARG, "too many particles");
  // density resampling: a pool with room for KCHUNK + 1 steps of new particles
  // at twice the mean rate (the pool is compacted at the start of every chunk)
  long long cap = d.np;
  if (piece && (piece[2] >= piece[3] || piece[3] - piece[2] > d.Wx || piece[2] <= -d.Wx || piece[3] > 2 * d.Wx))
    return fail(h, LBMPCD_ERR_INVALID_ARG, "kept cell columns of a piece must be a non-empty range of at most the region's width");
  if (p.resample_density) {
    const long long nouter = (long long)(d.xo_lo + (d.Wx - d.xo_hi)) * d.Hy * d.Wz;
    if ((double)d.nhome * SPAWN_MAX * p.ppc >= 4294967296.0)
      return fail(h, LBMPCD_ERR_INVALID_ARG, "density resampling: region too large for 32-bit particle draws");
    cap = d.np + (KCHUNK + 1) * nouter * 2LL * p.ppc;
    if (cap >= (1LL << 32) - 8) return fail(h, LBMPCD_ERR_INVALID_ARG, "density resampling: pool too large");
  }
  if (p.feedback == 2 && (d.Wx < 32 || d.Hy < 16 || p.coupling_width * p.refine > 16 || 16 % p.refine))
    return fail(h, LBMPCD_ERR_INVALID_ARG,
                "learned closure needs >= 32 fine columns, >= 16 fine rows, refine in {1, 2, 4, 8} and "
                "coupling_width * refine <= 16");
  d.ncell = (long long)d.Wx * (d.Hy + 1) * d.Wz;
  d.nbuf = strip ? (long long)d.n_in * p.nx * p.nz : 2LL * d.n_in * (p.ny - 2) * p.nz;
  const size_t rs = real_size(h->prec);
  std::vector<void*>& L = h->rep_allocs[replica];
  void* t = nullptr;
  cudaError_t e = cudaSuccess;
#define A(ptr, bytes) if (e == cudaSuccess) { e = dalloc(L, &t, (bytes)); ptr = t; }
  A(*(void**)&d.home, cap * 4);
  A(*(void**)&d.pid, cap * 4);
  A(*(void**)&d.home_alt, cap * 4);
  A(*(void**)&d.pid_alt, cap * 4);
  if (h->dim == 2) {   // interleaved (x, y) pairs
    A(d.off[0], cap * 2 * rs); A(d.vel[0], cap * 2 * rs);
    A(d.off_alt[0], cap * 2 * rs); A(d.vel_alt[0], cap * 2 * rs);
  } else {
    for (int a = 0; a < 3; ++a) {
      A(d.off[a], cap * rs); A(d.vel[a], cap * rs);
      A(d.off_alt[a], cap * rs); A(d.vel_alt[a], cap * rs);
    }
  }
  A(*(void**)&d.rank, cap * 4);
  if (p.resample_density || piece) {
    A(*(void**)&d.pool, 4 * 4);
    A(*(void**)&d.ltile, ((cap + SORT_TILE - 1) / SORT_TILE) * 4);
    d.pooled = 1;
    d.resample = p.resample_density ? 1 : 0;
    d.cap = (uint32_t)cap;
    const uint32_t init[4] = {(uint32_t)d.np, 0u, (uint32_t)d.np, 0u};
    if (e == cudaSuccess) e = cudaMemcpy(d.pool, init, sizeof(init), cudaMemcpyHostToDevice);
  } else {
    d.cap = (uint32_t)d.np;
  }
  A(*(void**)&d.hcount, d.nhome * 4);
  A(*(void**)&d.hoff, d.nhome * 4);
  A(*(void**)&d.tsum, (long long)d.ntile * 4);
  if (h->prec == P_FP64) {
    A(*(void**)&d.acc_n, d.ncell * 4);
    for (int a = 0; a < h->dim; ++a) A(d.acc_v[a], d.ncell * rs);
  } else {
    A(*(void**)&d.acc4, d.ncell * 16);
  }
  A(d.tab, d.ncell * rs * 4 * (h->dim == 2 ? 1 : 2));
  const long long nb4 = (d.nbuf > 0 ? d.nbuf : 1) * 4;
  A(*(void**)&d.frame, nb4 * 8);
  A(*(void**)&d.ring, nb4 * 8 * (long long)p.window);
  A(*(void**)&d.wsum, nb4 * 8);
  if (p.feedback == 2) {
    const long long ncl = 2LL * d.Hy * 16;
    A(*(void**)&d.cframe, 2 * ncl * 4 * 8);
    A(*(void**)&d.cring, 8 * ncl * 3 * 4);
    A(*(void**)&d.cema, ncl * 3 * 8);
    A(*(void**)&d.cl_u, (d.nbuf > 0 ? d.nbuf : 1) * 2 * 8);
  }
#undef A
  if (e != cudaSuccess) {
    free_list(L);
    return fail(h, e == cudaErrorMemoryAllocation ? LBMPCD_ERR_OOM : LBMPCD_ERR_CUDA,
                std::string("allocating region arrays: ") + cudaGetErrorString(e));
  }
  d.has_region = 1;
  d.own_lo = piece ? piece[0] : 0;
  d.own_hi = piece ? piece[1] : p.nx;
  if (p.feedback == 2) {
    d.cl_on = 1;
    d.cl_npy = (d.Hy + 15) / 16;
    d.cl_inv_ppc = 1.0 / p.ppc;
    d.cl_inv_sig = 1.0 / d.sig;
    d.cl_interval = 1;
    d.cl_first = 7;
  }
  int rc = build_maps(h);
  if (rc) return rc;
  CK(h, launch_init_particles(h->dim, h->prec, h->d_reps + replica, d, h->stream));
  // a piece keeps the particles of the whole region's seeding (same ids,
  // positions and velocities as the undivided run) in its kept cell columns
  if (piece) CK(h, launch_keep_columns(h->dim, d, piece[2], piece[3], h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return LBMPCD_OK;
}

extern "C" int lbmpcd_set_region(lbmpcd* h, int replica, const int lo[3], const int hi[3]) {
  return set_region_impl(h, replica, lo, hi, nullptr);
}

extern "C" int lbmpcd_set_region_piece(lbmpcd* h, int replica, const int lo[3], const int hi[3], int own_lo,
                                       int own_hi, int keep_lo, int keep_hi) {
  const int pc[4] = {own_lo, own_hi, keep_lo, keep_hi};
  return set_region_impl(h, replica, lo, hi, pc);
}

// One chunk of kcount steps (the sort, when due, runs before it: run_sort).
static bool persistent(const lbmpcd* h) { return h->mode == 1 && !h->has_cl; }

// The overlapped form of the per-kernel launches: the LB update of step n + 1
// needs only the populations of step n, so it runs beside the particle pass
// of step n (a programmatic dependent of the pass, on the pass's stream, with
// the pass capped at ov_bps blocks per SM so that LB blocks fit beside it);
// the table and a8 of step n, which need both, follow in a launch of their
// own.  A chunk is L(n0); then per step P(n) with L(n + 1) beside it, then
// the table and a8 of step n; the last step's a8 is left to the next chunk's
// first LB launch, as in the serial form.  Not with the learned closure
// (its network runs between the pass and the table), density resampling (its
// spawn runs before the pass) or the Chapman-Enskog redraw (the pass reads
// the populations the LB update of step n + 1 overwrites), nor with the
// TMA-staged LB rows.
// some replica keeps its particles in a pool (density resampling or a region
// piece): the particle pass is compiled with the pool handling
static bool pooled_any(const lbmpcd* h) {
  for (int r = 0; r < h->nrep; ++r)
    if (h->rd[r].pooled) return true;
  return false;
}

static bool overlapped(const lbmpcd* h) {
  return h->mode == 0 && !h->serial && !h->has_cl && h->nb_s == 0 && !h->ce && !h->lb_tma && h->nb_p > 0;
}

// particle-pass blocks per SM in the overlapped form: the handle's setting,
// else the occupancy limit (the LB blocks then take the SMs the pass leaves
// as its blocks finish: measured faster on the 2048 x 512 channel than
// capping the pass at 7 or 6 blocks per SM to make room for them)
static int ov_blocks(const lbmpcd* h) { return h->pers_bps > 0 ? h->pers_bps : 0; }

// Programmatic dependencies inside an overlapped chunk: bit 0, the table / a8
// launch after the LB rows (its blocks are placed while the pass ends); bit
// 1, the next particle pass after that launch.
#ifndef LBM_OV_PDL
#define LBM_OV_PDL 3
#endif

// The kernels of one overlapped chunk of kcount steps (after its prep);
// around(phase, fn) wraps each launch group (the profiled form brackets them
// with events, which also makes each group wait for the previous one).
template <typename Around>
static cudaError_t overlapped_chunk(lbmpcd* h, const Launch& L, int kcount, Around&& around) {
  cudaError_t e = around(1, [&] { return launch_lb(h->q, h->prec, h->lbvec, false, L, h->bm_lb, h->nb_lb, 0); });
  for (int k = 0; k < kcount && e == cudaSuccess; ++k) {
    const bool last = k + 1 == kcount;
    e = around(2, [&] {
      cudaError_t x = launch_particles(h->dim, h->prec, pooled_any(h), h->at, false, L, h->bm_p, h->nb_p, k, ov_blocks(h),
                                       k > 0 && (LBM_OV_PDL & 2));
      if (x == cudaSuccess && !last) x = launch_lb_rows(h->q, h->prec, h->lbvec, L, h->bm_rows, h->nb_rows, k + 1, h->d_ctr);
      return x;
    });
    if (e == cudaSuccess)
      e = around(3, [&] {
        return launch_lb_items(h->q, h->prec, L, last ? h->bm_c_last : h->bm_c, last ? h->nb_c_last : h->nb_c, k,
                               !last && (LBM_OV_PDL & 1));
      });
  }
  return e;
}

// the closure network runs on step n (handle-wide: every closure replica
// shares the first evaluation and the interval)
static bool closure_eval(const lbmpcd* h, long long n) {
  for (int r = 0; r < h->nrep; ++r) {
    const RepDev& d = h->rd[r];
    if (!d.cl_on) continue;
    return n >= d.cl_first && (n - d.cl_first) % d.cl_interval == 0;
  }
  return false;
}

// Which steps of a chunk run the closure network: none, the first only, every
// K-th from the first (the periodic graph), or as the step count says (a
// chunk launched directly).
enum { CL_NONE = 0, CL_FIRST = 1, CL_EVERY_K = 2, CL_BY_STEP = 3 };

static int closure_interval(const lbmpcd* h) {
  for (int r = 0; r < h->nrep; ++r)
    if (h->rd[r].cl_on) return h->rd[r].cl_interval;
  return 1;
}

static int run_chunk(lbmpcd* h, int kcount, int cl_mode) {
  Launch L{h->d_reps, h->nrep, h->d_si, h->stream, h->d_flag + 8, h->rd.data()};
  const bool ov = overlapped(h);
  CK(h, launch_prep(h->dim, L, h->d_si, kcount, h->d_sorted, h->d_step, h->d_pending, h->d_cells,
                    h->d_last_shift, ov ? 1 : 0, ov ? h->d_ctr : nullptr));
  if (ov) {
    CK(h, overlapped_chunk(h, L, kcount, [](int, auto&& fn) { return fn(); }));
    return LBMPCD_OK;
  }
  if (persistent(h)) {
    const PersistentMaps m{h->bm_lb256, h->nb_lb256, h->bm_p, h->nb_p, h->d_bar, (int*)(h->d_bar + 2), h->bar_spin};
    CK(h, launch_persistent(h->q, h->prec, h->lbvec, L, kcount, m, h->pers_bps, nullptr));
    return LBMPCD_OK;
  }
  for (int k = 0; k < kcount; ++k) {
    CK(h, launch_lb(h->q, h->prec, h->lbvec, h->lb_tma, L, h->bm_lb, h->nb_lb, k));
    if (h->nb_s) CK(h, launch_spawn(h->dim, h->prec, L, h->bm_s, h->nb_s, k));
    CK(h, launch_particles(h->dim, h->prec, pooled_any(h), h->at, h->ce, L, h->bm_p, h->nb_p, k, 0));
    if (h->has_cl && h->cl_params) {
      const bool net = cl_mode == CL_FIRST ? k == 0
                     : cl_mode == CL_EVERY_K ? k % closure_interval(h) == 0
                     : cl_mode == CL_BY_STEP ? closure_eval(h, h->nstep + k) : false;
      if (net) CK(h, launch_closure_step(h->prec, L, h->ptab, h->n_ptab, k, net_closure(h->net)));
    }
  }
  return LBMPCD_OK;
}

// The counting sort of the particles by home cell is due before a chunk when
// KCHUNK steps have passed since the last one (it keeps the particles of a
// warp in a few neighbouring cells; the seeded state is sorted); density
// resampling compacts its particle pool with it before every chunk.
static bool sort_due(const lbmpcd* h) {
  if (h->nb_p == 0) return false;
  return h->nb_s > 0 || h->nstep - h->last_sort >= KCHUNK;
}

static int run_sort(lbmpcd* h) {
  Launch L{h->d_reps, h->nrep, h->d_si, h->stream, h->d_flag + 8, h->rd.data()};
  CK(h, launch_sort(h->dim, h->prec, L, h->bm_p, h->nb_p, h->bm_t, h->nb_t, h->d_sorted));
  h->last_sort = h->nstep;
  return LBMPCD_OK;
}

// Capture a chunk of kcount steps (closure network per cl_mode) into *out.
static int capture_chunk(lbmpcd* h, int kcount, int cl_mode, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  cudaStream_t cap = h->stream;
  bool own = false;
  if (!cap) { CK(h, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)); own = true; }
  if (own) CK(h, cudaDeviceSynchronize());
  CK(h, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
  cudaStream_t keep = h->stream;
  h->stream = cap;
  int rc = run_chunk(h, kcount, cl_mode);
  h->stream = keep;
  cudaError_t e = cudaStreamEndCapture(cap, &g);
  if (!rc && e == cudaSuccess) {
    e = cudaGraphInstantiate(out, g, 0);
    if (e != cudaSuccess) *out = nullptr;
  }
  if (g) cudaGraphDestroy(g);
  if (own) cudaStreamDestroy(cap);
  if (rc) return rc;
  if (e != cudaSuccess || !*out) return cuda_fail(h, e != cudaSuccess ? e : cudaErrorUnknown, "graph capture");
  return LBMPCD_OK;
}

// Every graph is captured at the first step after the maps were (re)built,
// so that no later call pays for a capture: the chunk lengths without the
// closure network and, with it loaded, one evaluation step and the periodic
// chunk (the network only where it runs: a disabled node in a graph still
// cost ~3.5 us per step).
static int capture_all(lbmpcd* h) {
  int rc = LBMPCD_OK;
  for (int i = 0; i < NGRAPH && !rc; ++i) rc = capture_chunk(h, i + 1, CL_NONE, &h->graphs[i]);
  if (!rc && h->has_cl && h->cl_params) {
    rc = capture_chunk(h, 1, CL_FIRST, &h->g_eval);
    const int K = closure_interval(h);
    if (!rc && K <= KCHUNK) {
      h->period = K * (KCHUNK / K);
      rc = capture_chunk(h, h->period, CL_EVERY_K, &h->g_period);
    }
  }
  if (rc) {
    drop_graphs(h);
    if (!persistent(h)) return rc;
    // the cooperative launch did not capture: launch the persistent chunks directly
    cudaGetLastError();
    h->pers_graph = false;
    h->err.clear();
    return LBMPCD_OK;
  }
  h->graphs_ready = true;
  return LBMPCD_OK;
}

// steps from n to the next step that runs the closure network (0: n does)
static long long to_next_eval(const lbmpcd* h, long long n) {
  for (int r = 0; r < h->nrep; ++r) {
    const RepDev& d = h->rd[r];
    if (!d.cl_on) continue;
    if (n < d.cl_first) return d.cl_first - n;
    const long long ph = (n - d.cl_first) % d.cl_interval;
    return ph ? d.cl_interval - ph : 0;
  }
  return 1LL << 40;
}

// a call is cut into chunks of KCHUNK steps and one of the rest (each
// chunk one graph replay; the first LB launch of a chunk is not overlapped)
static int chunk_len(int left) { return left < KCHUNK ? left : KCHUNK; }

extern "C" int lbmpcd_step(lbmpcd* h, int nsteps) {
  if (!h) return LBMPCD_ERR_INVALID_ARG;
  if (nsteps < 0) return fail(h, LBMPCD_ERR_INVALID_ARG, "nsteps < 0");
  if (h->maps_dirty) { int rc = build_maps(h); if (rc) return rc; }
  const bool use_graph = !persistent(h) || h->pers_graph;
  if (nsteps > 0 && use_graph && !h->graphs_ready) {
    const int rc = capture_all(h);
    if (rc) return rc;
  }
  const bool net = h->has_cl && h->cl_params;
  int left = nsteps;
  while (left > 0) {
    if (sort_due(h)) { const int rc = run_sort(h); if (rc) return rc; }
    int kc;
    if (!h->graphs_ready) {
      kc = chunk_len(left);
      const int rc = run_chunk(h, kc, CL_BY_STEP);
      if (rc) return rc;
    } else if (net && to_next_eval(h, h->nstep) == 0) {
      // an evaluation step: the periodic chunk when it fits, else the single step
      const bool per = h->g_period && left >= h->period;
      kc = per ? h->period : 1;
      CK(h, cudaGraphLaunch(per ? h->g_period : h->g_eval, h->stream));
    } else {
      const long long gap = net ? to_next_eval(h, h->nstep) : (long long)left;
      kc = chunk_len((int)(gap < left ? gap : left));
      CK(h, cudaGraphLaunch(h->graphs[kc - 1], h->stream));
    }
    left -= kc;
    h->nstep += kc;
  }
  if (nsteps > 0)
    for (int r = 0; r < h->nrep; ++r) {
      h->pending[r] = h->rd[r].has_region ? 1 : 0;
      h->cells[r] = h->rd[r].has_region && !overlapped(h) ? 1 : 0;   // the overlapped form builds the last table
    }
  if (nsteps > 0 && h->cl_params) {   // a bounded wait inside a closure GEMM gave up
    const int rc = net_error(h->net, h->stream);
    if (rc) return fail(h, rc, "closure network: a tensor-core wait timed out");
  }
  if (nsteps > 0 && h->nb_s) {   // a density-resampling pool ran out of slots
    for (int r = 0; r < h->nrep; ++r) {
      if (!h->rd[r].resample) continue;
      uint32_t pf[4];
      CK(h, cudaMemcpyAsync(pf, h->rd[r].pool, sizeof(pf), cudaMemcpyDeviceToHost, h->stream));
      CK(h, cudaStreamSynchronize(h->stream));
      if (pf[1]) return fail(h, LBMPCD_ERR_CAPACITY, "density resampling: particle pool full (replica " +
                                                         std::to_string(r) + "); results invalid");
    }
  }
  if (nsteps > 0 && persistent(h)) {   // a bounded grid-barrier wait gave up
    unsigned bar[4] = {0, 0, 0, 0};
    CK(h, cudaMemcpyAsync(bar, h->d_bar, sizeof(bar), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (bar[2]) {
      CK(h, cudaMemset(h->d_bar, 0, sizeof(bar)));
      return fail(h, LBMPCD_ERR_TIMEOUT, "persistent step: a grid-barrier wait timed out");
    }
  }
  return LBMPCD_OK;
}

extern "C" int lbmpcd_step_profiled(lbmpcd* h, int nsteps, double* phase_ms, long long* launches) {
  if (!h) return LBMPCD_ERR_INVALID_ARG;
  if (nsteps < 0 || !phase_ms) return fail(h, LBMPCD_ERR_INVALID_ARG, "nsteps < 0 or null phase_ms");
  if (h->maps_dirty) { int rc = build_maps(h); if (rc) return rc; }
  const int nev = 2 * (2 + 5 * KCHUNK);
  std::vector<cudaEvent_t> ev(nev, nullptr);
  for (auto& x : ev) CK(h, cudaEventCreate(&x));
  Launch L{h->d_reps, h->nrep, h->d_si, h->stream, h->d_flag + 8, h->rd.data()};
  int rc = LBMPCD_OK;
  long long nl = 0;
  int left = nsteps;
  cudaError_t e = cudaSuccess;
  while (left > 0 && e == cudaSuccess) {
    const int kc = chunk_len(left);
    int ie = 0;
    std::vector<int> phase;
    auto bracket = [&](int ph, auto&& fn) {
      if (e != cudaSuccess) return;
      e = cudaEventRecord(ev[ie++], h->stream);
      if (e == cudaSuccess) e = fn();
      if (e == cudaSuccess) e = cudaEventRecord(ev[ie++], h->stream);
      phase.push_back(ph);
      ++nl;
    };
    if (sort_due(h)) {
      bracket(4, [&] { return launch_sort(h->dim, h->prec, L, h->bm_p, h->nb_p, h->bm_t, h->nb_t, h->d_sorted); });
      h->last_sort = h->nstep;
    }
    const bool ov = overlapped(h);
    bracket(0, [&] { return launch_prep(h->dim, L, h->d_si, kc, h->d_sorted, h->d_step, h->d_pending,
                                        h->d_cells, h->d_last_shift, ov ? 1 : 0, ov ? h->d_ctr : nullptr); });
    if (ov) {
      // phase 1: the chunk's first LB launch; 2: each particle pass with the
      // LB update of the next step beside it (one bracket: they overlap);
      // 3: the table and a8 launch of each step
      int inner = 0;
      overlapped_chunk(h, L, kc, [&](int ph, auto&& fn) {
        bracket(ph, [&] { return fn(); });
        if (ph == 2 && inner++ + 1 < kc) ++nl;   // the LB rows launched inside the bracket
        return e;
      });
    }
    for (int k = 0; k < kc && !ov; ++k) {
      bracket(1, [&] { return launch_lb(h->q, h->prec, h->lbvec, h->lb_tma, L, h->bm_lb, h->nb_lb, k); });
      if (h->nb_s) bracket(2, [&] { return launch_spawn(h->dim, h->prec, L, h->bm_s, h->nb_s, k); });
      if (h->nb_p) bracket(2, [&] { return launch_particles(h->dim, h->prec, pooled_any(h), h->at, h->ce, L, h->bm_p, h->nb_p, k, 0); });
      if (h->has_cl && h->cl_params && closure_eval(h, h->nstep + k))
        bracket(5, [&] { return launch_closure_step(h->prec, L, h->ptab, h->n_ptab, k, net_closure(h->net)); });
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    for (size_t i = 0; i < phase.size() && e == cudaSuccess; ++i) {
      float ms = 0;
      e = cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
      phase_ms[phase[i]] += ms;
      if (phase[i] == 4) nl += 3;   // the sort is four kernels
    }
    left -= kc;
    h->nstep += kc;
  }
  for (auto& x : ev) cudaEventDestroy(x);
  if (e != cudaSuccess) rc = cuda_fail(h, e, "step_profiled");
  if (nsteps > 0)
    for (int r = 0; r < h->nrep; ++r) {
      h->pending[r] = h->rd[r].has_region ? 1 : 0;
      h->cells[r] = h->rd[r].has_region && !overlapped(h) ? 1 : 0;
    }
  if (launches) *launches += nl;
  return rc;
}

// live particles of a density-resampling replica; also leaves the readout
// order of the pool in rank (valid until the next step)
static long long live_particles(lbmpcd* h, int r) {
  const RepDev& d = h->rd[r];
  if (launch_live_index(d, h->stream) != cudaSuccess) return -1;
  uint32_t n = 0;
  if (cudaMemcpyAsync(&n, d.pool + 2, sizeof(n), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess) return -1;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return -1;
  return n;
}

static long long field_elems(const lbmpcd* h, int r, int field) {
  const RepDev& d = h->rd[r];
  const bool pf = field == LBMPCD_PART_POS || field == LBMPCD_PART_VEL || field == LBMPCD_PART_HOME ||
                  field == LBMPCD_PART_CELL || field == LBMPCD_PART_ID || field == LBMPCD_CELL_LIST;
  const bool scalar = field == LBMPCD_PART_CELL || field == LBMPCD_PART_ID || field == LBMPCD_CELL_LIST;
  if (pf && d.has_region && d.pooled) {
    const long long n = live_particles(const_cast<lbmpcd*>(h), r);
    if (n < 0) return -1;
    return scalar ? n : 3 * n;
  }
  switch (field) {
    case LBMPCD_RHO: return d.nnode;
    case LBMPCD_U: return 3 * d.nnode;
    case LBMPCD_POPS: return (long long)h->q * d.nnode;
    case LBMPCD_PART_POS: case LBMPCD_PART_VEL: case LBMPCD_PART_HOME: return d.has_region ? 3 * d.np : -1;
    case LBMPCD_PART_CELL: case LBMPCD_PART_ID: case LBMPCD_CELL_LIST: return d.has_region ? d.np : -1;
    case LBMPCD_SHIFT: return 3;
    case LBMPCD_CELL_COUNT: return d.has_region ? d.ncell : -1;
    case LBMPCD_CELL_VCM: return d.has_region ? 3 * d.ncell : -1;
    case LBMPCD_WINDOW_MEAN: return d.has_region ? 4 * d.nbuf : -1;
    case LBMPCD_DIAG: return 9;
    case LBMPCD_CLOSURE_IN: return d.cl_on ? 2LL * d.cl_npy * 256 * 24 : -1;
    case LBMPCD_CLOSURE_OUT: case LBMPCD_CLOSURE_TARGET: return d.cl_on ? 2LL * d.cl_npy * 256 * 3 : -1;
  }
  return -1;
}
static bool int_field(int f) {
  return f == LBMPCD_PART_CELL || f == LBMPCD_CELL_COUNT || f == LBMPCD_PART_HOME || f == LBMPCD_PART_ID ||
         f == LBMPCD_CELL_LIST;
}

extern "C" int lbmpcd_population_bytes(const lbmpcd* h) {
  if (!h) return LBMPCD_ERR_INVALID_ARG;
  return h->prec == P_FP64 ? 8 : (h->prec == P_FP32 ? 4 : 2);
}

namespace {
// Raw population columns [x, x + ncols) of the buffer the next step reads:
// rows (i, z, y) of ncols storage values, nx apart in the lattice.
int copy_columns(lbmpcd* h, int replica, int x, int ncols, void* host_or_dev, int on_device, bool to_lattice) {
  if (!h) return LBMPCD_ERR_INVALID_ARG;
  if (replica < 0 || replica >= h->nrep || !host_or_dev) return fail(h, LBMPCD_ERR_INVALID_ARG, "bad replica or null buffer");
  const RepDev& d = h->rd[replica];
  if (ncols < 1 || x < 0 || x + ncols > d.nx) return fail(h, LBMPCD_ERR_INVALID_ARG, "column range outside the lattice");
  const size_t esz = (size_t)lbmpcd_population_bytes(h);
  char* lat = (char*)d.f[h->nstep & 1] + (size_t)x * esz;
  const size_t pitch = (size_t)d.nx * esz, width = (size_t)ncols * esz, rows = (size_t)d.q * d.nz * d.ny;
  const cudaMemcpyKind k = to_lattice ? (on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice)
                                      : (on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
  cudaError_t e = to_lattice ? cudaMemcpy2DAsync(lat, pitch, host_or_dev, width, width, rows, k, h->stream)
                             : cudaMemcpy2DAsync(host_or_dev, width, lat, pitch, width, rows, k, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? LBMPCD_OK : cuda_fail(h, e, to_lattice ? "set_columns" : "get_columns");
}
}  // namespace

static int flush_if_pending(lbmpcd* h, int r);

extern "C" int lbmpcd_set_particles(lbmpcd* h, int replica, long long n, const int* home, const double* off,
                                    const double* vel, const int* pid) {
  if (!h) return LBMPCD_ERR_INVALID_ARG;
  if (replica < 0 || replica >= h->nrep || n < 0 || (n > 0 && (!home || !off || !vel || !pid)))
    return fail(h, LBMPCD_ERR_INVALID_ARG, "bad replica, count or null array");
  RepDev& d = h->rd[replica];
  if (!d.has_region || !d.pooled) return fail(h, LBMPCD_ERR_STATE, "set_particles needs pooled particles (a region piece)");
  if (n > (long long)d.cap) return fail(h, LBMPCD_ERR_CAPACITY, "more particles than the pool holds");
  if (h->maps_dirty) { int rc = build_maps(h); if (rc) return rc; }
  int rc = flush_if_pending(h, replica);   // the table of the last step built, its accumulators cleared
  if (rc) return rc;
  // one device buffer: offsets and velocities (binary64) first, so that
  // every array starts aligned to its element size whatever n is
  void* tmp = nullptr;
  const size_t bh = (size_t)n * 3 * 4, bo = (size_t)n * 3 * 8, bp = (size_t)n * 4;
  if (n > 0) CK(h, staging(h, 2 * bo + bh + bp, &tmp));
  char* t = (char*)tmp;
  double* t_off = (double*)t;
  double* t_vel = (double*)(t + bo);
  int* t_home = (int*)(t + 2 * bo);
  int* t_pid = (int*)(t + 2 * bo + bh);
  cudaError_t e = cudaSuccess;
  if (n > 0) {
    e = cudaMemcpyAsync(t_off, off, bo, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t_vel, vel, bo, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t_home, home, bh, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t_pid, pid, bp, cudaMemcpyHostToDevice, h->stream);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream);
  if (e == cudaSuccess && n > 0)
    e = launch_pool_in(h->dim, h->prec, d, n, t_home, t_off, t_vel, t_pid, h->d_flag, h->stream);
  const uint32_t pool[4] = {(uint32_t)n, 0u, (uint32_t)n, 0u};
  if (e == cudaSuccess) e = cudaMemcpyAsync(d.pool, pool, sizeof(pool), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_sorted + replica, 0, sizeof(int), h->stream);
  int bad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "set_particles");
  if (bad) return fail(h, LBMPCD_ERR_INVALID_ARG, "particle home cell or offset out of range (removed)");
  return LBMPCD_OK;
}

extern "C" int lbmpcd_get_columns(lbmpcd* h, int replica, int x, int ncols, void* dst, int dst_on_device) {
  return copy_columns(h, replica, x, ncols, dst, dst_on_device, false);
}

extern "C" int lbmpcd_set_columns(lbmpcd* h, int replica, int x, int ncols, const void* src, int src_on_device) {
  return copy_columns(h, replica, x, ncols, const_cast<void*>(src), src_on_device, true);
}

extern "C" long long lbmpcd_field_size(const lbmpcd* h, int replica, int field) {
  if (!h || replica < 0 || replica >= h->nrep) return LBMPCD_ERR_INVALID_ARG;
  long long n = field_elems(h, replica, field);
  return n < 0 ? LBMPCD_ERR_INVALID_ARG : n;
}

// The collision-cell table of the last step, which the step builds only in
// the next LB launch, for a read-out or the flush below.
static int cells_if_pending(lbmpcd* h, int r) {
  if (!h->cells[r] || !h->rd[r].has_region) return LBMPCD_OK;
  double ls[3];
  CK(h, cudaMemcpyAsync(ls, h->d_last_shift + 3 * r, sizeof(ls), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  CK(h, launch_cell_table(h->q, h->prec, h->rd[r], (uint32_t)(h->nstep - 1), (float)ls[1] > 0.0f, h->stream));
  CK(h, cudaMemsetAsync(h->d_cells + r, 0, sizeof(int), h->stream));
  h->cells[r] = 0;
  return LBMPCD_OK;
}

// Apply the collision of the last step to the particles (the step leaves it
// to the next particle pass) before their state is read or replaced.
static int flush_if_pending(lbmpcd* h, int r) {
  if (!h->pending[r] || !h->rd[r].has_region) return LBMPCD_OK;
  const int rc = cells_if_pending(h, r);
  if (rc) return rc;
  double ls[3];
  CK(h, cudaMemcpyAsync(ls, h->d_last_shift + 3 * r, sizeof(ls), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  CK(h, launch_flush(h->dim, h->prec, h->d_reps + r, h->rd[r], ls, h->stream));
  CK(h, cudaMemsetAsync(h->d_pending + r, 0, sizeof(int), h->stream));
  h->pending[r] = 0;
  return LBMPCD_OK;
}

extern "C" int lbmpcd_get_fields(lbmpcd* h, int replica, int field, void* dst, size_t bytes, int dst_on_device) {
  if (!h) return LBMPCD_ERR_INVALID_ARG;
  if (replica < 0 || replica >= h->nrep || !dst) return fail(h, LBMPCD_ERR_INVALID_ARG, "bad replica or null dst");
  const long long n = field_elems(h, replica, field);
  if (n < 0) return fail(h, LBMPCD_ERR_INVALID_ARG, "unknown field (or no region set)");
  const size_t esz = int_field(field) ? 4 : 8;
  if (bytes != (size_t)n * esz) return fail(h, LBMPCD_ERR_INVALID_ARG, "dst size does not match the field");
  if (h->maps_dirty) { int rc = build_maps(h); if (rc) return rc; }
  const RepDev& d = h->rd[replica];
  if (field == LBMPCD_CELL_LIST) {
    // stable counting sort of the particle rows by their collision cell (host)
    std::vector<int32_t> cell((size_t)n), list((size_t)n);
    std::vector<long long> start((size_t)d.ncell + 1, 0);
    int rc = n ? lbmpcd_get_fields(h, replica, LBMPCD_PART_CELL, cell.data(), (size_t)n * 4, 0) : LBMPCD_OK;
    if (rc) return rc;
    for (long long j = 0; j < n; ++j) {
      if (cell[j] < 0 || cell[j] >= d.ncell) return fail(h, LBMPCD_ERR_STATE, "particle without a collision cell");
      ++start[cell[j] + 1];
    }
    for (long long c = 0; c < d.ncell; ++c) start[c + 1] += start[c];
    for (long long j = 0; j < n; ++j) list[start[cell[j]]++] = (int32_t)j;
    if (n == 0) return LBMPCD_OK;
    CK(h, cudaMemcpyAsync(dst, list.data(), bytes, dst_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost,
                          h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return LBMPCD_OK;
  }
  void* buf = dst;
  void* tmp = nullptr;
  if (!dst_on_device && n > 0) {
    CK(h, staging(h, bytes, &tmp));
    buf = tmp;
  }
  int rc = LBMPCD_OK;
  cudaError_t e = cudaSuccess;
  const int parity = (int)(h->nstep & 1);
  double ls[3] = {0, 0, 0};
  switch (field) {
    case LBMPCD_RHO: case LBMPCD_U: {   // the copy of the last LB update (parity of step nstep - 1)
      const long long mp = h->nstep > 0 ? ((h->nstep - 1) & 1) : 0;
      const size_t rs = real_size(h->prec);
      e = field == LBMPCD_RHO ? launch_real_out(h->prec, (char*)d.rho + mp * d.nnode * rs, d.nnode, (double*)buf, h->stream)
                              : launch_real_out(h->prec, (char*)d.u + mp * 3 * d.nnode * rs, 3 * d.nnode, (double*)buf, h->stream);
      break;
    }
    case LBMPCD_POPS: e = launch_pops_out(h->q, h->prec, d, parity, (double*)buf, h->stream); break;
    case LBMPCD_PART_POS: case LBMPCD_PART_VEL: case LBMPCD_PART_HOME: case LBMPCD_PART_CELL:
    case LBMPCD_PART_ID:
      rc = flush_if_pending(h, replica);
      if (rc) break;
      e = cudaMemcpyAsync(ls, h->d_last_shift + 3 * replica, sizeof(ls), cudaMemcpyDeviceToHost, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
      if (e == cudaSuccess) e = launch_part_out(h->dim, h->prec, d, field, ls, buf, h->stream);
      break;
    case LBMPCD_SHIFT:
      e = cudaMemcpyAsync(buf, h->d_last_shift + 3 * replica, 3 * sizeof(double),
                          dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToDevice, h->stream);
      break;
    case LBMPCD_CELL_COUNT:
    case LBMPCD_CELL_VCM:
      rc = cells_if_pending(h, replica);
      if (!rc) e = launch_tab_out(h->dim, h->prec, d, field, buf, h->stream);
      break;
    case LBMPCD_WINDOW_MEAN:
      if (h->nstep == 0) e = cudaMemsetAsync(buf, 0, d.nbuf * 4 * 8, h->stream);
      else e = launch_window_out(h->dim, h->prec, d, (uint32_t)(h->nstep - 1), (double*)buf, h->stream);
      break;
    case LBMPCD_CLOSURE_IN:
      if (h->nstep == 0) e = cudaMemsetAsync(buf, 0, (size_t)n * 8, h->stream);
      else e = launch_closure_in_out(d, (uint32_t)(h->nstep - 1), (double*)buf, h->stream);
      break;
    case LBMPCD_CLOSURE_OUT:
      e = launch_real_out(P_FP32, net_output(h->net) + (long long)d.cl_p0 * 256 * 3, n, (double*)buf, h->stream);
      break;
    case LBMPCD_CLOSURE_TARGET:
      if (h->nstep == 0) e = cudaMemsetAsync(buf, 0, (size_t)n * 8, h->stream);
      else e = launch_closure_target_out(d, (uint32_t)(h->nstep - 1), (double*)buf, h->stream);
      break;
    case LBMPCD_DIAG: {
      double* o = (double*)buf;
      e = cudaMemsetAsync(o, 0, 9 * 8, h->stream);
      if (e == cudaSuccess) e = launch_diag_lb(h->q, h->prec, d, parity, o, h->stream);
      if (e == cudaSuccess && d.has_region) {
        rc = flush_if_pending(h, replica);
        if (!rc) e = launch_diag_particles(h->dim, h->prec, d, o, h->stream);
      }
      break;
    }
  }
  if (rc == LBMPCD_OK && e == cudaSuccess && tmp) e = cudaMemcpyAsync(dst, tmp, bytes, cudaMemcpyDeviceToHost, h->stream);
  int kerr = 0;   // a bounded wait inside a step kernel gave up (reported here, where the stream is synchronised)
  if (rc == LBMPCD_OK && e == cudaSuccess && h->lb_tma)
    e = cudaMemcpyAsync(&kerr, h->d_flag + 8, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (rc == LBMPCD_OK && e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (rc == LBMPCD_OK && e == cudaSuccess && kerr) {
    cudaMemset(h->d_flag + 8, 0, sizeof(int));
    return fail(h, LBMPCD_ERR_TIMEOUT, "a bounded wait in the TMA-staged LB kernel gave up; results invalid");
  }
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_fail(h, e, "get_fields");
  return LBMPCD_OK;
}

extern "C" int lbmpcd_set_state(lbmpcd* h, int replica, int field, const void* src, size_t bytes, int src_on_device) {
  if (!h) return LBMPCD_ERR_INVALID_ARG;
  if (replica < 0 || replica >= h->nrep || !src) return fail(h, LBMPCD_ERR_INVALID_ARG, "bad replica or null src");
  if (field != LBMPCD_POPS && field != LBMPCD_U && field != LBMPCD_PART_POS && field != LBMPCD_PART_VEL &&
      field != LBMPCD_PART_HOME)
    return fail(h, LBMPCD_ERR_INVALID_ARG, "only POPS, U, PART_POS, PART_VEL and PART_HOME can be set");
  const RepDev& d = h->rd[replica];
  const bool lbf = field == LBMPCD_POPS || field == LBMPCD_U;
  if (!lbf && !d.has_region) return fail(h, LBMPCD_ERR_STATE, "particles need a region first");
  if (!lbf && d.pooled)
    return fail(h, LBMPCD_ERR_INVALID_ARG,
                "particle state of pooled particles (density resampling, a region piece) is loaded by lbmpcd_set_particles");
  const long long n = field_elems(h, replica, field);
  const size_t esz = int_field(field) ? 4 : 8;
  if (bytes != (size_t)n * esz) return fail(h, LBMPCD_ERR_INVALID_ARG, "src size does not match the field");
  if (h->maps_dirty) { int rc = build_maps(h); if (rc) return rc; }
  if (!lbf) { int rc = flush_if_pending(h, replica); if (rc) return rc; }
  const void* buf = src;
  void* tmp = nullptr;
  if (!src_on_device) {
    CK(h, staging(h, bytes, &tmp));
    cudaError_t e = cudaMemcpyAsync(tmp, src, bytes, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_state copy");
    buf = tmp;
  }
  cudaError_t e = cudaSuccess;
  if (field == LBMPCD_POPS) {
    e = launch_pops_in(h->q, h->prec, d, (const double*)buf, h->stream);
  } else if (field == LBMPCD_U) {
    e = launch_pops_from_u(h->q, h->prec, d, (const double*)buf, h->stream);
  } else {
    e = cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) e = launch_part_in(h->dim, h->prec, d, field, buf, h->d_flag, h->stream);
  }
  int bad = 0;
  if (e == cudaSuccess && !lbf)
    e = cudaMemcpyAsync(&bad, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "set_state");
  if (bad) return fail(h, LBMPCD_ERR_INVALID_ARG, "particle positions out of range (state partly written)");
  return LBMPCD_OK;
}

extern "C" int lbmpcd_set_closure(lbmpcd* h, const float* theta, long long count, int src_on_device, int interval) {
  if (!h) return LBMPCD_ERR_INVALID_ARG;
  bool any = false;
  for (int r = 0; r < h->nrep; ++r) any = any || h->rd[r].cl_on;
  if (!any) return fail(h, LBMPCD_ERR_STATE, "no replica has a region with feedback = 2");
  if (theta && count != lbmpcd_net_num_params())
    return fail(h, LBMPCD_ERR_INVALID_ARG, "parameter count does not match the closure network");
  if (theta && interval < 1) return fail(h, LBMPCD_ERR_INVALID_ARG, "interval must be >= 1");
  for (int r = 0; r < h->nrep; ++r)
    if (h->rd[r].cl_on) {
      if (theta) {
        h->rd[r].cl_interval = interval;
        h->rd[r].cl_first = (int)std::max<long long>(7, h->nstep);
      }
      h->rd[r].cl_imp = theta ? 1 : 0;   // the LB imposes the prediction once one exists
      h->maps_dirty = true;
    }
  if (h->maps_dirty) { int rc = build_maps(h); if (rc) return rc; }
  if (!theta) {
    h->cl_params = false;
  } else {
    h->cl_theta.resize((size_t)count);
    CK(h, cudaMemcpyAsync(h->cl_theta.data(), theta, (size_t)count * 4,
                          src_on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    const int rc = net_load_params(h->net, h->cl_theta.data(), 0);
    if (rc) return fail(h, rc, "loading the closure parameters");
    h->cl_params = true;
  }
  drop_graphs(h);   // the step's kernels changed
  return LBMPCD_OK;
}

extern "C" int lbmpcd_set_wait_limit(lbmpcd* h, unsigned polls) {
  if (!h) return LBMPCD_ERR_INVALID_ARG;
  h->bar_spin = polls;
  drop_graphs(h);   // the persistent kernel takes the limit as an argument
  return LBMPCD_OK;
}

extern "C" int lbmpcd_set_launch_mode(lbmpcd* h, int mode, int blocks_per_sm, int flags) {
  if (!h) return LBMPCD_ERR_INVALID_ARG;
  if (mode < 0 || mode > 1 || blocks_per_sm < 0 || (flags & ~(LBMPCD_LAUNCH_LB_TMA | LBMPCD_LAUNCH_SERIAL)))
    return fail(h, LBMPCD_ERR_INVALID_ARG, "mode must be 0 or 1, flags a set of LBMPCD_LAUNCH_*");
  if (mode == 1)
    for (int r = 0; r < h->nrep; ++r)
      if (h->rd[r].cl_on || h->rd[r].pooled || h->at || h->ce)
        return fail(h, LBMPCD_ERR_INVALID_ARG,
                    "the persistent form runs neither the learned closure, the density resampling, MPCD-AT "
                    "nor the Chapman-Enskog redraw");
  h->mode = mode;
  h->pers_bps = blocks_per_sm;
  const bool tma = (flags & LBMPCD_LAUNCH_LB_TMA) && lb_tma_ok(h->q, h->prec, h->lbvec);
  if (tma != h->lb_tma) h->maps_dirty = true;   // the TMA form takes single-row items
  h->lb_tma = tma;
  h->serial = (flags & LBMPCD_LAUNCH_SERIAL) != 0;
  h->pers_graph = true;
  drop_graphs(h);
  return LBMPCD_OK;
}

// Time each candidate launch configuration on a fresh copy of the handle (same
// parameters and regions, so the handle's own state is untouched) and keep the
// fastest: per-kernel graphs with the default LB row width, with TMA-staged LB
// rows (D2Q9 binary32), with one LB node per thread; the persistent kernel at
// the occupancy limit and at one block per SM.
extern "C" int lbmpcd_autotune(lbmpcd* h, int steps, int* choice) {
  if (!h) return LBMPCD_ERR_INVALID_ARG;
  if (steps < 1) return fail(h, LBMPCD_ERR_INVALID_ARG, "steps must be >= 1");
  bool closure = false;
  for (int r = 0; r < h->nrep; ++r) closure = closure || h->rd[r].cl_on || h->rd[r].pooled || h->at || h->ce;
  struct Cand { int mode, bps, vec, flags; };
  const int vdef = h->lbvec;
  std::vector<Cand> cands = {{0, 0, vdef, 0}};
  if (!closure) {   // the overlapped form at other particle-pass shares of the SMs, and the serial form
    cands.push_back({0, 6, vdef, 0});
    cands.push_back({0, 7, vdef, 0});
    cands.push_back({0, 0, vdef, LBMPCD_LAUNCH_SERIAL});
  }
  if (lb_tma_ok(h->q, h->prec, vdef)) cands.push_back({0, 0, vdef, LBMPCD_LAUNCH_LB_TMA});
  if (vdef != 1) cands.push_back({0, 0, 1, 0});
  if (!closure) {
    cands.push_back({1, 0, vdef, 0});
    cands.push_back({1, 1, vdef, 0});
  }
  lbmpcd* c = nullptr;
  int rc = lbmpcd_create(h->P.data(), h->nrep, h->stream, &c);
  if (rc) return fail(h, rc, std::string("autotune copy: ") + g_create_error);
  for (int r = 0; r < h->nrep && !rc; ++r) {
    if (!h->rd[r].has_region) continue;
    const int lo[3] = {h->rd[r].x0, 0, 0}, hi[3] = {h->rd[r].x1, h->P[r].ny, h->P[r].nz};
    rc = lbmpcd_set_region(c, r, lo, hi);
  }
  std::vector<float> ms(cands.size(), 1e30f);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = LBMPCD_ERR_CUDA;
  for (size_t i = 0; i < cands.size() && !rc; ++i) {
    c->lbvec = cands[i].vec;
    c->maps_dirty = true;
    rc = lbmpcd_set_launch_mode(c, cands[i].mode, cands[i].bps, cands[i].flags);
    if (!rc) rc = lbmpcd_step(c, KCHUNK);   // warm-up, graph capture
    if (!rc && cudaEventRecord(e0, c->stream) != cudaSuccess) rc = LBMPCD_ERR_CUDA;
    if (!rc) rc = lbmpcd_step(c, steps);
    if (!rc && cudaEventRecord(e1, c->stream) != cudaSuccess) rc = LBMPCD_ERR_CUDA;
    if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = LBMPCD_ERR_CUDA;
    if (!rc) cudaEventElapsedTime(&ms[i], e0, e1);
    if (rc == LBMPCD_ERR_TIMEOUT || (rc == LBMPCD_ERR_CUDA && cands[i].mode == 1)) {
      rc = LBMPCD_OK;   // a candidate that cannot run is skipped
      ms[i] = 1e30f;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  const std::string why = rc ? std::string(c->err) : std::string();
  lbmpcd_destroy(c);
  if (rc) return fail(h, rc, "autotune: " + why);
  size_t best = 0;
  for (size_t i = 1; i < cands.size(); ++i) if (ms[i] < ms[best]) best = i;
  if (ms[best] >= 1e30f) return fail(h, LBMPCD_ERR_CUDA, "autotune: no candidate ran");
  h->lbvec = cands[best].vec;
  h->maps_dirty = true;
  rc = lbmpcd_set_launch_mode(h, cands[best].mode, cands[best].bps, cands[best].flags);
  if (rc) return rc;
  if (choice) {
    choice[0] = cands[best].mode;
    choice[1] = cands[best].bps;
    choice[2] = cands[best].vec;
    choice[3] = cands[best].flags;
    choice[4] = (int)cands.size();
  }
  return LBMPCD_OK;
}
