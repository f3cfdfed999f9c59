/*
 * oracle.h -- plain FP64 CPU oracle of the coupled lattice Boltzmann /
 * multiparticle-collision (LB-MPCD) time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this code; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no source with the CUDA path.
 *
 * The step it computes, in this order (Montessori et al., "A coupled lattice
 * Boltzmann-multiparticle collision method for multi-resolution hydrodynamics"):
 *   a1  LB stream + BGK collide, Eq. 1 with the equilibrium of Eq. 2, D2Q9 or
 *       D3Q19, half-way bounce-back walls (Sec. 3), Guo body force;
 *   a2  coarse->fine bilinear (trilinear) interpolation of u (Algorithm 2);
 *   a3  LB->MPCD Maxwellian redraw of outer-buffer particle velocities,
 *       Box-Muller normals (Sec. 2.3, Algorithm 1), or with redraw = 1 the
 *       Chapman-Enskog draw carrying the LB's non-equilibrium momentum flux
 *       (the Enskog sampling Sec. 2.3 names); with resample_density = 1 the
 *       outer-buffer particles are replaced instead;
 *   a4  MPCD streaming, Eq. 3, with body-force kick, bounce-back walls and
 *       periodic wrap inside the MPCD region (Sec. 2.3);
 *   a6  inner-buffer sampling of mass and momentum into a per-step frame;
 *   a5  random grid shift and binning into collision cells;
 *   a7  SRD collision, Eq. 4 (2D +-alpha, 3D random axis), or the MPCD-AT
 *       collision of Eq. 6 (collision = 1), with virtual wall particles in
 *       wall-cut cells;
 *   a8  MPCD->LB imposition of equilibrium populations built from the
 *       windowed cell moments on the inner buffer column.
 * The MPCD region is a slab of whole columns with buffers at its x-ends, or
 * (orc_set_strip) the near-wall strip of Sec. 3.3 with its buffer along y1.
 * With feedback = 2 (D2Q9 only; not in the paper) a8 is replaced by the
 * learned closure: each step records the instantaneous fine-cell fields of
 * the two 16-column strips at the region's x-edges, keeps the last 8 of them
 * and their exponential moving average, and lays them out as the network's
 * 16 x 16 patches; orc_closure_impose then has the next LB update impose
 * f_eq from a network output that the caller computes (oracle/closure.py).
 * All random numbers come from Philox4x32-10 keyed by (seed) with counter
 * (id, step, replica, tag); every floating-point step is IEEE binary64.
 */
#ifndef LBMPCD_ORACLE_H
#define LBMPCD_ORACLE_H
#include <stdint.h>
#include <stddef.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int lattice;          /* 9 = D2Q9, 19 = D3Q19 */
  int nx, ny, nz;       /* LB nodes; rows y = 0 and y = ny-1 are solid walls */
  double tau;           /* BGK relaxation time (Eq. 1) */
  double force[3];      /* body acceleration g (LB units / step^2) */
  int refine;           /* r = LB spacing / MPCD cell size a */
  int ppc;              /* mean particles per MPCD cell */
  double alpha;         /* SRD rotation angle, radians (Eq. 4) */
  double kT, mass;      /* thermal energy and particle mass (LB units) */
  int coupling_width;   /* LB columns of coupling buffer per side */
  int precision;        /* 0 FP64, 1 FP32, 2 FP16 deviations: decides binning precision only */
  int feedback;         /* 0 one-way (the paper), 1 windowed MPCD->LB imposition,
                           2 learned closure (sampling here, imposition by
                           orc_closure_impose) */
  int window;           /* averaging window W in steps */
  int resample_density; /* 0: outer-buffer velocities redrawn (the paper); 1: outer-buffer
                           particles replaced, their number drawn from the LB density */
  uint64_t seed;
  int collision;        /* 0: SRD (Eq. 4); 1: MPCD with the Andersen thermostat (MPCD-AT, Eq. 6) */
  int redraw;           /* 0: Maxwellian redraw (Algorithm 1); 1: Chapman-Enskog redraw carrying the
                           LB's non-equilibrium momentum flux (the Enskog sampling of Sec. 2.3) */
} orc_params;

typedef struct orc_sim orc_sim;

/* field ids (same numbering as the product's get_fields) */
enum {
  ORC_RHO = 0, ORC_U = 1, ORC_POPS = 2, ORC_PART_POS = 3, ORC_PART_VEL = 4,
  ORC_PART_CELL = 5, ORC_SHIFT = 6, ORC_CELL_COUNT = 7, ORC_WINDOW_MEAN = 8,
  ORC_DIAG = 9, ORC_PART_HOME = 10,
  ORC_CELL_VCM = 11,        /* [ncell][3] SRD: v_cm; MPCD-AT: v_cm minus the cell's mean random velocity */
  ORC_PART_ID = 12,
  ORC_CLOSURE_IN = 13,      /* [P][16][16][24] network input of the last step */
  ORC_CLOSURE_TARGET = 15,  /* [P][16][16][3] moving averages, patch layout */
  ORC_PI = 16,              /* [6][nz][ny][nx] traceless kinematic non-equilibrium momentum flux
                               (xx, yy, zz, xy, xz, yz) of the last LB step (redraw = 1) */
  ORC_CELL_LIST = 17        /* [np] particle indices grouped by collision cell (increasing cell,
                               then increasing index) */
};

orc_sim* orc_create(const orc_params* p, int replica);
int  orc_set_region(orc_sim* s, int x0, int x1);
/* near-wall strip (Sec. 3.3): all columns, LB rows [1, y1), coupling buffer along y1 */
int  orc_set_strip(orc_sim* s, int y1);
int  orc_step(orc_sim* s, int nsteps);
long orc_field_size(const orc_sim* s, int field);   /* element count */
int  orc_get_field(const orc_sim* s, int field, void* dst); /* double or int32 */
int  orc_set_field(orc_sim* s, int field, const void* src);
void orc_destroy(orc_sim* s);
long orc_num_particles(const orc_sim* s);
/* threads of the OpenMP loops (1 unless built with -fopenmp, for timing) */
int orc_num_threads(void);
long orc_step_count(const orc_sim* s);
/* Closure patches per replica (0 unless feedback = 2 with a region). */
long orc_closure_patches(const orc_sim* s);
/* a8 of the learned closure for the step just completed: y [P][16][16][3]
 * is the network output in patch layout; the LB update of the next step
 * imposes it (as the windowed a8).  No-op before 8 frames exist.  Returns -1
 * if the replica has no closure sampling. */
int  orc_closure_impose(orc_sim* s, const double* y);

/* building blocks exposed for the pin tests */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_box_muller(uint32_t w0, uint32_t w1, double* z0, double* z1);
void orc_feq(int lattice, double rho, const double u[3], double* out);
int  orc_lattice_table(int lattice, int* c /* q*3 */, double* w /* q */);
int  orc_bin_offset(double off, double s, int precision);
void orc_srd_rotate_2d(double vx, double vy, double cx, double cy, double alpha,
                       int sign, double* ox, double* oy);
void orc_srd_rotate_3d(const double v[3], const double vcm[3], const double axis[3],
                       double alpha, double out[3]);
void orc_random_axis(uint32_t w0, uint32_t w1, double axis[3]);
/* a2 interpolation of the current U field to the centre of MPCD cell (X,Y,Z) */
void orc_u_fine(const orc_sim* s, int X, int Y, int Z, double out[3]);

#ifdef __cplusplus
}
#endif
#endif
