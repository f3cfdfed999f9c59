/*
 * oracle.c -- plain FP64 CPU oracle of the coupled LB-MPCD step.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
 * baseline of the benchmark, never by the product library.  Written for a
 * reader who checks it against the paper by eye: plain loops, one step of the
 * method per function, no blocking, no fusion.  Compile with
 * -ffp-contract=off so that no multiply-add is fused.
 *
 * Units: LB spacing and LB time step are 1.  MPCD cells have side a = 1/r;
 * MPCD positions are kept as an integer home cell plus an offset in [0,1) in
 * cell units; velocities are in LB units per step; delta_t_MPCD = 1.
 *
 * Geometry: LB node (x,y,z) covers [x,x+1)x[y,y+1)x[z,z+1); rows y=0 and
 * y=ny-1 are solid, so the half-way walls sit at y=1 and y=ny-1.  The MPCD
 * region spans LB columns [x0,x1), all fluid rows and all z; in cell units it
 * is [0,Wx)x[0,Hy)x[0,Wz) with Wx=(x1-x0)r, Hy=(ny-2)r, Wz=nz*r (Wz=1 in 2D).
 * Each x-side has a coupling buffer of coupling_width LB columns: the outer
 * ceil(cw/2) columns take the LB->MPCD redraw, the inner floor(cw/2) columns
 * give the MPCD->LB imposition.
 *
 * Near-wall strip (orc_set_strip; the two-level geometry of Sec. 3.3): the
 * MPCD region spans all columns (periodic in x) and the LB rows [1, y1) next
 * to the bottom wall, Hy = (y1-1) r; the coupling buffer lies along its top
 * edge: the outer ceil(cw/2) LB rows below y1 take the redraw, the inner
 * floor(cw/2) rows under them the imposition.  The top edge is not a wall: a
 * particle that reaches it is turned back by specular reflection (v_y -> -v_y,
 * x and z motion kept), and cells cut by it get no virtual particles (they hold
 * outer-buffer particles only, whose velocities are redrawn before they move).
 */
#include "oracle.h"
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

#define TAG_SHIFT 1u
#define TAG_SIGN 2u
#define TAG_AXIS 3u
#define TAG_VIRT 4u
#define TAG_RESAMPLE 5u
#define TAG_INIT_POS 6u
#define TAG_INIT_VEL 7u
#define TAG_DENSITY 8u
#define TAG_SPAWN_POS 9u
#define TAG_SPAWN_VEL 10u
#define TAG_AT 11u
#define TAG_AT_VIRT 12u
#define TAG_CE 13u       /* attempt k uses tag TAG_CE + 16 k (and TAG_CE + 1 + 16 k in 3D) */
#define CE_TRIES 64
#define SPAWN_MAX 4     /* at most SPAWN_MAX * ppc new particles per cell and step */

static const double PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from its published definition (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of
 * (hi,lo) = M*x products on words 0 and 2, xor-mixed with words 1, 3 and the
 * key; the key is bumped by the Weyl constants between rounds.              */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter layout used everywhere: (id, step, replica, tag); key = seed. */
static void draw(const orc_sim* s, uint32_t id, uint32_t step, uint32_t tag, uint32_t w[4]);

/* Box-Muller (Box & Muller 1958, the transform Sec. 2.3 names):
 * u1 = (w0+1)/2^32 in (0,1], u2 = w1/2^32 in [0,1),
 * z0 = sqrt(-2 ln u1) cos(2 pi u2), z1 = sqrt(-2 ln u1) sin(2 pi u2).      */
void orc_box_muller(uint32_t w0, uint32_t w1, double* z0, double* z1) {
  double u1 = ((double)w0 + 1.0) * (1.0 / 4294967296.0);
  double u2 = (double)w1 * (1.0 / 4294967296.0);
  double rad = sqrt(-2.0 * log(u1));
  double ang = 2.0 * PI * u2;
  *z0 = rad * cos(ang);
  *z1 = rad * sin(ang);
}

/* 24-bit uniform in [0,1): exact in binary32 and binary64. */
static double u24(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }

/* uniformly distributed unit vector: n_z = 2u-1, azimuth 2 pi u'. */
void orc_random_axis(uint32_t w0, uint32_t w1, double axis[3]) {
  double z = 2.0 * u24(w0) - 1.0;
  double phi = 2.0 * PI * u24(w1);
  double rho = sqrt(1.0 - z * z);
  axis[0] = rho * cos(phi);
  axis[1] = rho * sin(phi);
  axis[2] = z;
}

/* ------------------------------------------------------------------------ */
/* Lattices (Sec. 2.1).  D2Q9 is the paper's; D3Q19 is the standard
 * three-dimensional second-order lattice with the same equilibrium form.    */
static const int C9[9][3] = {{0,0,0},{1,0,0},{0,1,0},{-1,0,0},{0,-1,0},
                             {1,1,0},{-1,1,0},{-1,-1,0},{1,-1,0}};
static const double W9[9] = {4.0/9, 1.0/9, 1.0/9, 1.0/9, 1.0/9,
                             1.0/36, 1.0/36, 1.0/36, 1.0/36};
static const int C19[19][3] = {{0,0,0},{1,0,0},{-1,0,0},{0,1,0},{0,-1,0},{0,0,1},{0,0,-1},
                               {1,1,0},{-1,-1,0},{1,-1,0},{-1,1,0},{1,0,1},{-1,0,-1},
                               {1,0,-1},{-1,0,1},{0,1,1},{0,-1,-1},{0,1,-1},{0,-1,1}};
static const double W19[19] = {1.0/3, 1.0/18, 1.0/18, 1.0/18, 1.0/18, 1.0/18, 1.0/18,
                               1.0/36, 1.0/36, 1.0/36, 1.0/36, 1.0/36, 1.0/36,
                               1.0/36, 1.0/36, 1.0/36, 1.0/36, 1.0/36, 1.0/36};

int orc_lattice_table(int lattice, int* c, double* w) {
  int q = lattice == 9 ? 9 : (lattice == 19 ? 19 : 0);
  for (int i = 0; i < q; ++i) {
    for (int a = 0; a < 3; ++a) c[3*i+a] = (q == 9) ? C9[i][a] : C19[i][a];
    w[i] = (q == 9) ? W9[i] : W19[i];
  }
  return q;
}

/* Eq. 2 with c_s^2 = 1/3. */
void orc_feq(int lattice, double rho, const double u[3], double* out) {
  int c[19*3]; double w[19];
  int q = orc_lattice_table(lattice, c, w);
  const double cs2 = 1.0 / 3.0;
  double uu = u[0]*u[0] + u[1]*u[1] + u[2]*u[2];
  for (int i = 0; i < q; ++i) {
    double cu = c[3*i]*u[0] + c[3*i+1]*u[1] + c[3*i+2]*u[2];
    out[i] = w[i] * rho * (1.0 + cu / cs2 + (cu*cu) / (2.0*cs2*cs2) - uu / (2.0*cs2));
  }
}

/* ------------------------------------------------------------------------ */
struct orc_sim {
  orc_params p;
  int replica, dim, q;
  int c[19*3]; double w[19]; int opp[19];
  long nnode;
  double *f, *fn, *rho, *u;          /* f[q][nz][ny][nx]; u[3][...] */
  double *pi;                         /* redraw = 1: [6][nz][ny][nx] traceless pi' (xx yy zz xy xz yz) */
  long step;                          /* global step counter n */
  /* MPCD */
  int has_region, x0, x1, Wx, Hy, Wz, r, n_out, n_in;
  int strip, y1;                      /* near-wall strip: rows [1, y1), buffer along y1 */
  long np, cap;                       /* particles, allocated slots */
  int *home;                          /* [np][3] integer home cell */
  double *off, *vel;                  /* [np][3] offsets in [0,1), velocities */
  int *pcell;                         /* [np] collision cell of last binning */
  int ncx, ncy, ncz; long ncell;
  int *cnt; double *sumv, *vcm;      /* per collision cell */
  double *vran, *ranm;               /* MPCD-AT: [np][3] random velocities, [ncell][3] their cell means */
  double shift[3];
  /* coupling */
  long nbuf;                          /* inner-buffer LB nodes */
  double *frames;                     /* [W][nbuf][4] ring of per-step samples */
  double *wmean;                      /* [nbuf][4] rho_bar, u_bar of last step */
  double *imp;                        /* [nbuf][4] imposition pending for the next LB update:
                                         flag, u_bar (set by a8, applied by a1 of the next step) */
  long nframes;                       /* frames written so far */
  /* learned closure (feedback = 2): strips of CL_W fine columns per side */
  int cl_on, cl_npy;                  /* patches per side: ceil(Hy / 16) */
  long cl_ncell;                      /* 2 Hy CL_W strip cells */
  double *cl_frame;                   /* [ncl][3] count, sum vx, sum vy of this step */
  double *cl_hist;                    /* [8][ncl][3] fields of the last 8 steps, oldest first */
  double *cl_ema;                     /* [ncl][3] exponential moving average */
  double *cl_x;                       /* [P][16][16][24] network input */
  long cl_nframes;
};

#define CL_W 16          /* strip width and patch side, fine cells */
#define CL_FRAMES 8      /* frames in the network input */
#define CL_EMA_T 500.0   /* moving-average time constant, steps */

static void draw(const orc_sim* s, uint32_t id, uint32_t step, uint32_t tag, uint32_t w[4]) {
  uint32_t ctr[4] = {id, step, (uint32_t)s->replica, tag};
  uint32_t key[2] = {(uint32_t)(s->p.seed & 0xffffffffu), (uint32_t)(s->p.seed >> 32)};
  orc_philox4x32_10(ctr, key, w);
}

static long nidx(const orc_sim* s, int x, int y, int z) {
  return (long)x + (long)s->p.nx * ((long)y + (long)s->p.ny * (long)z);
}
static int imod(int a, int m) { int b = a % m; return b < 0 ? b + m : b; }

orc_sim* orc_create(const orc_params* p, int replica) {
  if (!(p->lattice == 9 || p->lattice == 19)) return NULL;
  if (p->nx < 1 || p->ny < 3 || p->nz < 1) return NULL;
  if (p->lattice == 9 && p->nz != 1) return NULL;
  if (p->tau <= 0.5 || p->refine < 1 || p->ppc < 1 || p->resample_density < 0 || p->resample_density > 1)
    return NULL;
  /* MPCD-AT draws by particle index, which density resampling renumbers */
  if (p->collision < 0 || p->collision > 1 || (p->collision == 1 && p->resample_density)) return NULL;
  if (p->redraw < 0 || p->redraw > 1 || (p->redraw == 1 && p->resample_density)) return NULL;
  orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
  s->p = *p; s->replica = replica;
  s->dim = p->lattice == 9 ? 2 : 3;
  s->q = orc_lattice_table(p->lattice, s->c, s->w);
  for (int i = 0; i < s->q; ++i)
    for (int j = 0; j < s->q; ++j)
      if (s->c[3*j] == -s->c[3*i] && s->c[3*j+1] == -s->c[3*i+1] && s->c[3*j+2] == -s->c[3*i+2])
        s->opp[i] = j;
  s->nnode = (long)p->nx * p->ny * p->nz;
  s->f = (double*)malloc(sizeof(double) * s->q * s->nnode);
  s->fn = (double*)malloc(sizeof(double) * s->q * s->nnode);
  s->rho = (double*)malloc(sizeof(double) * s->nnode);
  s->u = (double*)calloc(3 * s->nnode, sizeof(double));
  s->pi = (double*)calloc(6 * s->nnode, sizeof(double));
  /* initial state: f = f_eq(rho0 = 1, u = 0) everywhere (walls included). */
  double feq[19], zero[3] = {0, 0, 0};
  orc_feq(p->lattice, 1.0, zero, feq);
  for (int i = 0; i < s->q; ++i)
    for (long n = 0; n < s->nnode; ++n) { s->f[i*s->nnode + n] = feq[i]; s->fn[i*s->nnode + n] = feq[i]; }
  for (long n = 0; n < s->nnode; ++n) s->rho[n] = 1.0;
  return s;
}

void orc_destroy(orc_sim* s) {
  if (!s) return;
  free(s->f); free(s->fn); free(s->rho); free(s->u); free(s->pi);
  free(s->home); free(s->off); free(s->vel); free(s->pcell);
  free(s->cnt); free(s->sumv); free(s->vcm); free(s->vran); free(s->ranm); free(s->frames); free(s->wmean); free(s->imp);
  free(s->cl_frame); free(s->cl_hist); free(s->cl_ema); free(s->cl_x);
  free(s);
}

long orc_num_particles(const orc_sim* s) { return s->np; }

/* threads the loops marked for OpenMP run on: 1 in the parity build */
int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
long orc_step_count(const orc_sim* s) { return s->step; }

/* Seed the MPCD region: exactly ppc particles in every cell, offsets uniform
 * in the cell (24-bit Philox uniforms), velocities Maxwellian with variance
 * kT/m per component and zero mean (Box-Muller). */
static int setup_region(orc_sim* s, int x0, int x1, int strip, int y1);
int orc_set_region(orc_sim* s, int x0, int x1) {
  const orc_params* p = &s->p;
  if (x0 < 0 || x1 > p->nx || x1 - x0 < 2 * p->coupling_width || p->coupling_width < 0) return -1;
  return setup_region(s, x0, x1, 0, p->ny - 1);
}

/* the near-wall strip: all columns, LB rows [1, y1), buffer rows below y1;
 * needs interior rows under the buffer and y1 below the top wall */
int orc_set_strip(orc_sim* s, int y1) {
  const orc_params* p = &s->p;
  if (p->coupling_width < 0 || y1 - 1 <= p->coupling_width || y1 >= p->ny - 1) return -1;
  if (p->feedback == 2 || p->resample_density) return -1;
  return setup_region(s, 0, p->nx, 1, y1);
}

static int setup_region(orc_sim* s, int x0, int x1, int strip, int y1) {
  const orc_params* p = &s->p;
  int cw = p->coupling_width;
  s->has_region = 1; s->x0 = x0; s->x1 = x1; s->r = p->refine;
  s->strip = strip; s->y1 = y1;
  s->Wx = (x1 - x0) * s->r; s->Hy = (y1 - 1) * s->r; s->Wz = s->dim == 3 ? p->nz * s->r : 1;
  s->n_out = (cw + 1) / 2; s->n_in = cw / 2;
  long ncell_home = (long)s->Wx * s->Hy * s->Wz;
  s->np = ncell_home * p->ppc;
  if (p->resample_density && (double)ncell_home * SPAWN_MAX * p->ppc >= 4294967296.0) return -1;
  s->cap = s->np > 0 ? s->np : 1;
  s->home = (int*)malloc(sizeof(int) * 3 * s->cap);
  s->off = (double*)malloc(sizeof(double) * 3 * s->cap);
  s->vel = (double*)malloc(sizeof(double) * 3 * s->cap);
  s->pcell = (int*)malloc(sizeof(int) * s->cap);
  s->ncx = s->Wx; s->ncy = s->Hy + 1; s->ncz = s->Wz;
  s->ncell = (long)s->ncx * s->ncy * s->ncz;
  s->cnt = (int*)calloc(s->ncell, sizeof(int));
  s->sumv = (double*)calloc(3 * s->ncell, sizeof(double));
  s->vcm = (double*)calloc(3 * s->ncell, sizeof(double));
  s->vran = (double*)calloc(3 * s->cap, sizeof(double));
  s->ranm = (double*)calloc(3 * s->ncell, sizeof(double));
  s->nbuf = strip ? (long)s->n_in * p->nx * p->nz : 2L * s->n_in * (p->ny - 2) * p->nz;
  int W = p->window > 0 ? p->window : 1;
  s->frames = (double*)calloc((size_t)W * (s->nbuf > 0 ? s->nbuf : 1) * 4, sizeof(double));
  s->wmean = (double*)calloc((size_t)(s->nbuf > 0 ? s->nbuf : 1) * 4, sizeof(double));
  s->imp = (double*)calloc((size_t)(s->nbuf > 0 ? s->nbuf : 1) * 4, sizeof(double));
  if (p->feedback == 2) {
    /* the closure needs two disjoint strips, 16 rows, an inner column inside
       the strip, LB nodes that do not straddle patches (r divides 16)
       and a thermal velocity to scale by */
    if (s->dim != 2 || s->Wx < 2 * CL_W || s->Hy < CL_W || cw * s->r > CL_W || CL_W % s->r || !(p->kT > 0))
      return -1;
    s->cl_on = 1;
    s->cl_npy = (s->Hy + CL_W - 1) / CL_W;
    s->cl_ncell = 2L * s->Hy * CL_W;
    s->cl_frame = (double*)calloc((size_t)s->cl_ncell * 3, sizeof(double));
    s->cl_hist = (double*)calloc((size_t)CL_FRAMES * s->cl_ncell * 3, sizeof(double));
    s->cl_ema = (double*)calloc((size_t)s->cl_ncell * 3, sizeof(double));
    s->cl_x = (double*)calloc((size_t)2 * s->cl_npy * CL_W * CL_W * 3 * CL_FRAMES, sizeof(double));
    s->cl_nframes = 0;
  }
  double sig = sqrt(p->kT / p->mass);
  for (long k = 0; k < s->np; ++k) {
    long cell = k / p->ppc;
    int hx = (int)(cell % s->Wx), hy = (int)((cell / s->Wx) % s->Hy), hz = (int)(cell / ((long)s->Wx * s->Hy));
    uint32_t w[4], v[4];
    draw(s, (uint32_t)k, 0u, TAG_INIT_POS, w);
    draw(s, (uint32_t)k, 0u, TAG_INIT_VEL, v);
    s->home[3*k] = hx; s->home[3*k+1] = hy; s->home[3*k+2] = hz;
    s->off[3*k] = u24(w[0]); s->off[3*k+1] = u24(w[1]);
    s->off[3*k+2] = s->dim == 3 ? u24(w[2]) : 0.0;
    double z0, z1, z2, z3;
    orc_box_muller(v[0], v[1], &z0, &z1);
    orc_box_muller(v[2], v[3], &z2, &z3);
    s->vel[3*k] = sig * z0; s->vel[3*k+1] = sig * z1;
    s->vel[3*k+2] = s->dim == 3 ? sig * z2 : 0.0;
    s->pcell[k] = -1;
  }
  s->nframes = 0;
  return 0;
}

/* LB node (x, y, z) of inner-buffer entry b: slab b = ((side n_in + col) nz
 * + z)(ny - 2) + y - 1, col counted inwards from the region's edge; strip
 * b = (row nz + z) nx + x, row counted down from the buffer's top. */
static void buffer_node(const orc_sim* s, long b, int* x, int* y, int* z) {
  const orc_params* p = &s->p;
  long t = b;
  if (s->strip) {
    *x = (int)(t % p->nx); t /= p->nx;
    *z = (int)(t % p->nz); t /= p->nz;
    *y = s->y1 - 1 - s->n_out - (int)t;
  } else {
    *y = 1 + (int)(t % (p->ny - 2)); t /= (p->ny - 2);
    *z = (int)(t % p->nz); t /= p->nz;
    int col = (int)(t % s->n_in), side = (int)(t / s->n_in);
    *x = side == 0 ? s->x0 + s->n_out + col : s->x1 - 1 - s->n_out - col;
  }
}

/* ------------------------------------------------------------------------ */
/* a1: LB step, Eq. 1.  Pull form: the population arriving at x along c_i is
 * the post-collision value stored at x - c_i; if x - c_i is a wall node, it is
 * the population that left x along -c_i and bounced back half-way (Sec. 3).
 * Moments of the arrived set: rho = sum f, rho u = sum f c + F/2 with F = rho g
 * (Guo et al. forcing), then f* = f - (f - f_eq)/tau + S with
 * S_i = (1 - 1/(2 tau)) w_i [(c_i - u)/cs^2 + (c_i.u) c_i / cs^4] . F.        */
static void lb_step(orc_sim* s) {
  const orc_params* p = &s->p;
  const double cs2 = 1.0 / 3.0, tau = p->tau;
  /* nodes are independent (each writes only its own populations and moments);
     the pragma takes effect only in the all-cores timing build (-fopenmp) */
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < p->nz; ++z)
    for (int y = 1; y < p->ny - 1; ++y)
      for (int x = 0; x < p->nx; ++x) {
        double fi[19];
        long here = nidx(s, x, y, z);
        for (int i = 0; i < s->q; ++i) {
          int sx = imod(x - s->c[3*i], p->nx);
          int sy = y - s->c[3*i+1];
          int sz = imod(z - s->c[3*i+2], p->nz);
          if (sy == 0 || sy == p->ny - 1)
            fi[i] = s->f[s->opp[i] * s->nnode + here];
          else
            fi[i] = s->f[i * s->nnode + nidx(s, sx, sy, sz)];
        }
        double rho = 0, jx = 0, jy = 0, jz = 0;
        for (int i = 0; i < s->q; ++i) {
          rho += fi[i];
          jx += fi[i] * s->c[3*i]; jy += fi[i] * s->c[3*i+1]; jz += fi[i] * s->c[3*i+2];
        }
        double F[3] = {rho * p->force[0], rho * p->force[1], rho * p->force[2]};
        double u[3] = {(jx + 0.5 * F[0]) / rho, (jy + 0.5 * F[1]) / rho, (jz + 0.5 * F[2]) / rho};
        double feq[19];
        orc_feq(p->lattice, rho, u, feq);
        for (int i = 0; i < s->q; ++i) {
          double ci[3] = {s->c[3*i], s->c[3*i+1], s->c[3*i+2]};
          double cu = ci[0]*u[0] + ci[1]*u[1] + ci[2]*u[2];
          double S = 0;
          for (int a = 0; a < 3; ++a)
            S += ((ci[a] - u[a]) / cs2 + cu * ci[a] / (cs2 * cs2)) * F[a];
          S *= (1.0 - 1.0 / (2.0 * tau)) * s->w[i];
          s->fn[i * s->nnode + here] = fi[i] - (fi[i] - feq[i]) / tau + S;
        }
        s->rho[here] = rho;
        s->u[here] = u[0]; s->u[s->nnode + here] = u[1]; s->u[2*s->nnode + here] = u[2];
        if (p->redraw == 1) {
          /* pi = (1 - 1/(2 tau)) Pi_neq / rho, Pi_neq = sum_i (f_i - f_i^eq) c_i c_i of the
             populations after streaming; its traceless part over the MPCD dimensions */
          const int ab[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
          double pv[6];
          for (int m = 0; m < 6; ++m) {
            double acc = 0;
            for (int i = 0; i < s->q; ++i) acc += (fi[i] - feq[i]) * s->c[3*i+ab[m][0]] * s->c[3*i+ab[m][1]];
            pv[m] = (1.0 - 1.0 / (2.0 * tau)) * acc / rho;
          }
          double tr = (pv[0] + pv[1] + (s->dim == 3 ? pv[2] : 0.0)) / s->dim;
          pv[0] -= tr; pv[1] -= tr;
          if (s->dim == 3) pv[2] -= tr; else { pv[2] = pv[4] = pv[5] = 0.0; }
          for (int m = 0; m < 6; ++m) s->pi[m * s->nnode + here] = pv[m];
        }
      }
  double* t = s->f; s->f = s->fn; s->fn = t;
  /* keep the (unused) wall rows identical in both buffers */
  for (int i = 0; i < s->q; ++i)
    for (int z = 0; z < p->nz; ++z)
      for (int x = 0; x < p->nx; ++x) {
        s->f[i*s->nnode + nidx(s, x, 0, z)] = s->fn[i*s->nnode + nidx(s, x, 0, z)];
        s->f[i*s->nnode + nidx(s, x, p->ny-1, z)] = s->fn[i*s->nnode + nidx(s, x, p->ny-1, z)];
      }
  /* a8 of the previous step, applied as the collision of the inner-buffer
     nodes: their post-collision populations become f_eq(rho_LB, u_bar), rho_LB
     the node's density of this update, u_bar the window mean a8 recorded */
  for (long b = 0; b < s->nbuf; ++b) {
    if (s->imp[4*b] == 0.0) continue;
    int x, y, z;
    buffer_node(s, b, &x, &y, &z);
    double feq[19];
    orc_feq(p->lattice, s->rho[nidx(s, x, y, z)], &s->imp[4*b+1], feq);
    for (int i = 0; i < s->q; ++i) s->f[i * s->nnode + nidx(s, x, y, z)] = feq[i];
  }
}

/* LB velocity with a ghost row behind each wall, u_ghost = -u_fluid, so that
 * the interpolated velocity vanishes on the half-way wall. */
static double u_node(const orc_sim* s, int a, int x, int y, int z) {
  const orc_params* p = &s->p;
  x = imod(x, p->nx); z = imod(z, p->nz);
  if (y <= 0) return -s->u[a * s->nnode + nidx(s, x, 1, z)];
  if (y >= p->ny - 1) return -s->u[a * s->nnode + nidx(s, x, p->ny - 2, z)];
  return s->u[a * s->nnode + nidx(s, x, y, z)];
}

/* a2 (Algorithm 2): bilinear (trilinear in 3D) interpolation of the LB
 * velocity, known at node centres (x+1/2, y+1/2, z+1/2), to the centre of
 * MPCD cell (X,Y,Z).  At r = 1 the two centres coincide. */
static void u_fine(const orc_sim* s, int X, int Y, int Z, double out[3]) {
  double r = s->r;
  double px = s->x0 + (X + 0.5) / r - 0.5;
  double py = 1.0 + (Y + 0.5) / r - 0.5;
  double pz = (s->dim == 3) ? (Z + 0.5) / r - 0.5 : 0.0;
  int i0 = (int)floor(px), j0 = (int)floor(py), k0 = (int)floor(pz);
  double tx = px - i0, ty = py - j0, tz = pz - k0;
  for (int a = 0; a < 3; ++a) {
    double acc = 0;
    for (int di = 0; di < 2; ++di)
      for (int dj = 0; dj < 2; ++dj)
        for (int dk = 0; dk < (s->dim == 3 ? 2 : 1); ++dk) {
          double wgt = (di ? tx : 1 - tx) * (dj ? ty : 1 - ty);
          if (s->dim == 3) wgt *= (dk ? tz : 1 - tz);
          acc += wgt * u_node(s, a, i0 + di, j0 + dj, k0 + dk);
        }
    out[a] = acc;
  }
}

static int lb_column_of(const orc_sim* s, int X) { return s->x0 + X / s->r; }
/* outer buffer: the n_out LB columns at each x-end of the region, or the n_out
 * LB rows under the top edge of a near-wall strip */
static int in_outer(const orc_sim* s, int X, int Y) {
  if (s->strip) return 1 + Y / s->r >= s->y1 - s->n_out;
  int x = lb_column_of(s, X);
  return x < s->x0 + s->n_out || x >= s->x1 - s->n_out;
}
/* index of the inner-buffer LB node holding MPCD cell (X,Y,Z), or -1.
 * Strip: b = (row nz + z) nx + x, row counted down from the buffer's top. */
static long inner_node(const orc_sim* s, int X, int Y, int Z) {
  const orc_params* p = &s->p;
  if (s->strip) {
    int y = 1 + Y / s->r;
    if (y < s->y1 - p->coupling_width || y >= s->y1 - s->n_out) return -1;
    int row = s->y1 - 1 - s->n_out - y, z = (s->dim == 3) ? Z / s->r : 0;
    return ((long)row * p->nz + z) * p->nx + X / s->r;
  }
  int x = lb_column_of(s, X);
  int side, col;
  if (x >= s->x0 + s->n_out && x < s->x0 + p->coupling_width) { side = 0; col = x - s->x0 - s->n_out; }
  else if (x < s->x1 - s->n_out && x >= s->x1 - p->coupling_width) { side = 1; col = s->x1 - 1 - s->n_out - x; }
  else return -1;
  int y = 1 + Y / s->r, z = (s->dim == 3) ? Z / s->r : 0;
  return (((long)side * s->n_in + col) * p->nz + z) * (p->ny - 2) + (y - 1);
}

/* a3' (resample_density = 1; the paper redraws velocities only and keeps the
 * particles, Sec. 2.3, so this mode reads "resampling from the local LB
 * density" literally): every particle whose home cell lies in an
 * outer-buffer column is removed; then each outer-buffer cell c (home cell
 * index c = X + Wx (Y + Hy Z), taken in increasing c) receives
 *   N_c = floor(x) + [u < x - floor(x)],  x = ppc rho_LB / rho0 (rho0 = 1),
 * rho_LB the density of the LB node holding the cell in this step and
 * u = (w0 >> 8) 2^-24 of Philox(c, n, replica, TAG_DENSITY), capped at
 * SPAWN_MAX ppc.  New particle k of cell c has the offsets (w >> 8) 2^-24 of
 * the words of Philox(c SPAWN_MAX ppc + k, n, replica, TAG_SPAWN_POS) and the
 * velocity u_fine + sqrt(kT/m) (z0, z1, z2) of the Box-Muller normals of
 * Philox(c SPAWN_MAX ppc + k, n, replica, TAG_SPAWN_VEL), as in a3. */
static void grow(orc_sim* s, long n) {
  if (n <= s->cap) return;
  long c = s->cap * 2 > n ? s->cap * 2 : n;
  s->home = (int*)realloc(s->home, sizeof(int) * 3 * c);
  s->off = (double*)realloc(s->off, sizeof(double) * 3 * c);
  s->vel = (double*)realloc(s->vel, sizeof(double) * 3 * c);
  s->pcell = (int*)realloc(s->pcell, sizeof(int) * c);
  s->cap = c;
}

static void resample_density(orc_sim* s) {
  const orc_params* p = &s->p;
  long w = 0;
  for (long k = 0; k < s->np; ++k) {
    if (in_outer(s, s->home[3*k], s->home[3*k+1])) continue;
    for (int a = 0; a < 3; ++a) {
      s->home[3*w+a] = s->home[3*k+a]; s->off[3*w+a] = s->off[3*k+a]; s->vel[3*w+a] = s->vel[3*k+a];
    }
    s->pcell[w] = s->pcell[k];
    ++w;
  }
  s->np = w;
  double sig = sqrt(p->kT / p->mass);
  long nmax = (long)SPAWN_MAX * p->ppc;
  for (int Z = 0; Z < s->Wz; ++Z)
    for (int Y = 0; Y < s->Hy; ++Y)
      for (int X = 0; X < s->Wx; ++X) {
        if (!in_outer(s, X, Y)) continue;
        long c = X + (long)s->Wx * (Y + (long)s->Hy * Z);
        int lx = lb_column_of(s, X), ly = 1 + Y / s->r, lz = s->dim == 3 ? Z / s->r : 0;
        double x = (double)p->ppc * s->rho[nidx(s, lx, ly, lz)];
        uint32_t wd[4]; draw(s, (uint32_t)c, (uint32_t)s->step, TAG_DENSITY, wd);
        double fl = floor(x);
        long n = (long)fl + (u24(wd[0]) < x - fl ? 1 : 0);
        if (n > nmax) n = nmax;
        if (n < 0) n = 0;
        double uf[3]; u_fine(s, X, Y, Z, uf);
        grow(s, s->np + n);
        for (long k = 0; k < n; ++k) {
          uint32_t id = (uint32_t)(c * nmax + k), wp[4], wv[4];
          draw(s, id, (uint32_t)s->step, TAG_SPAWN_POS, wp);
          draw(s, id, (uint32_t)s->step, TAG_SPAWN_VEL, wv);
          double z0, z1, z2, z3;
          orc_box_muller(wv[0], wv[1], &z0, &z1);
          orc_box_muller(wv[2], wv[3], &z2, &z3);
          long j = s->np++;
          s->home[3*j] = X; s->home[3*j+1] = Y; s->home[3*j+2] = Z;
          s->off[3*j] = u24(wp[0]); s->off[3*j+1] = u24(wp[1]);
          s->off[3*j+2] = s->dim == 3 ? u24(wp[2]) : 0.0;
          s->vel[3*j] = uf[0] + sig * z0;
          s->vel[3*j+1] = uf[1] + sig * z1;
          s->vel[3*j+2] = s->dim == 3 ? uf[2] + sig * z2 : 0.0;
          s->pcell[j] = -1;
        }
      }
}

/* a3 with the Chapman-Enskog distribution (redraw = 1; Sec. 2.3 names Enskog
 * sampling for flows whose gradients the Maxwellian redraw misses).  The new
 * peculiar velocity C = v - u_fine follows f_MB(C; kT/m) (1 + b : zz), z = C /
 * sqrt(kT/m), b = pi' / (2 kT/m), pi' the traceless non-equilibrium momentum
 * flux of the LB node holding the cell, so that <C C> = (kT/m) I + pi'.  It is
 * drawn by acceptance-rejection: attempt t takes z from the Box-Muller normals
 * of Philox(id, n, replica, TAG_CE + 16 t) (3D: z0, z1 from words 0, 1 and z2
 * from words 2, 3) and U = (w >> 8) 2^-24 of word 2 (3D: word 0 of
 * Philox(id, n, replica, TAG_CE + 1 + 16 t)), and is accepted when
 * A U <= 1 + b : zz with A = 1 + 30 max |b_ab|; after CE_TRIES rejections the
 * last candidate is kept. */
static void ce_peculiar(const orc_sim* s, uint32_t id, long node, double sig, double C[3]) {
  const int ab[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
  double b[3][3] = {{0}}, bmax = 0.0;
  for (int m = 0; m < 6; ++m) {
    double v = s->pi[m * s->nnode + node] / (2.0 * sig * sig);
    b[ab[m][0]][ab[m][1]] = v; b[ab[m][1]][ab[m][0]] = v;
    if (fabs(v) > bmax) bmax = fabs(v);
  }
  double A = 1.0 + 30.0 * bmax, z[3] = {0, 0, 0};
  for (int t = 0; t < CE_TRIES; ++t) {
    uint32_t w[4]; draw(s, id, (uint32_t)s->step, TAG_CE + 16u * (uint32_t)t, w);
    double z3, U;
    orc_box_muller(w[0], w[1], &z[0], &z[1]);
    if (s->dim == 3) {
      orc_box_muller(w[2], w[3], &z[2], &z3);
      uint32_t w2[4]; draw(s, id, (uint32_t)s->step, TAG_CE + 1u + 16u * (uint32_t)t, w2);
      U = u24(w2[0]);
    } else {
      z[2] = 0.0;
      U = u24(w[2]);
    }
    double q = 0.0;
    for (int a = 0; a < s->dim; ++a)
      for (int c = 0; c < s->dim; ++c) q += b[a][c] * z[a] * z[c];
    if (A * U <= 1.0 + q) break;
  }
  for (int a = 0; a < 3; ++a) C[a] = sig * z[a];
}

/* a3 (Sec. 2.3, Algorithm 1): particles whose home cell is in an outer buffer
 * column get v = u_fine + sqrt(kT/m) xi, xi ~ N(0, I) by Box-Muller (or the
 * Chapman-Enskog draw above with redraw = 1). */
static void resample(orc_sim* s) {
  double sig = sqrt(s->p.kT / s->p.mass);
  /* particles are independent: each draws by its own index (timing build only) */
#pragma omp parallel for schedule(static)
  for (long k = 0; k < s->np; ++k) {
    int X = s->home[3*k], Y = s->home[3*k+1], Z = s->home[3*k+2];
    if (!in_outer(s, X, Y)) continue;
    double uf[3]; u_fine(s, X, Y, Z, uf);
    if (s->p.redraw == 1) {
      long node = nidx(s, lb_column_of(s, X), 1 + Y / s->r, (s->dim == 3) ? Z / s->r : 0);
      double C[3]; ce_peculiar(s, (uint32_t)k, node, sig, C);
      for (int a = 0; a < 3; ++a) s->vel[3*k+a] = (a < s->dim) ? uf[a] + C[a] : 0.0;
      continue;
    }
    uint32_t w[4]; draw(s, (uint32_t)k, (uint32_t)s->step, TAG_RESAMPLE, w);
    double z0, z1, z2, z3;
    orc_box_muller(w[0], w[1], &z0, &z1);
    orc_box_muller(w[2], w[3], &z2, &z3);
    s->vel[3*k] = uf[0] + sig * z0;
    s->vel[3*k+1] = uf[1] + sig * z1;
    s->vel[3*k+2] = s->dim == 3 ? uf[2] + sig * z2 : 0.0;
  }
}

/* a4: Eq. 3 streaming with a body-force kick first (v += g, then r += v dt),
 * bounce-back on the walls y = 0 and y = Hy (velocity reversed, the rest of
 * the path retraced), periodic wrap in x inside the region and in z. */
static void stream(orc_sim* s) {
  const orc_params* p = &s->p;
  const double r = s->r;
  const double one_minus = 1.0 - 1.0 / 9007199254740992.0; /* largest double below 1 */
  /* particles are independent (timing build only, as in lb_step) */
#pragma omp parallel for schedule(static)
  for (long k = 0; k < s->np; ++k) {
    double* v = &s->vel[3*k];
    double* o = &s->off[3*k];
    int* h = &s->home[3*k];
    v[0] += p->force[0]; v[1] += p->force[1];
    if (s->dim == 3) v[2] += p->force[2];
    double dx = v[0] * r, dy = v[1] * r, dz = (s->dim == 3) ? v[2] * r : 0.0;
    /* y, in the local coordinate of the home cell */
    double ty = o[1] + dy;
    int ky = (int)floor(ty);
    int ny_ = h[1] + ky;
    double dxe = dx, dze = dz;
    if (ny_ < 0 || ny_ >= s->Hy) {
      double L = (ny_ < 0) ? (double)(-h[1]) : (double)(s->Hy - h[1]); /* wall, local units */
      double ts = (L - o[1]) / dy;          /* fraction of the step before the hit */
      double tr = L - (ty - L);             /* mirrored end point */
      if (s->strip && ny_ >= s->Hy) {       /* top edge of a strip: specular */
        v[1] = -v[1];
      } else {
        v[0] = -v[0]; v[1] = -v[1]; v[2] = -v[2];
        dxe = dx * ts - dx * (1.0 - ts);
        dze = dz * ts - dz * (1.0 - ts);
      }
      int kr = (int)floor(tr);
      h[1] += kr; o[1] = tr - (double)kr;
      if (h[1] >= s->Hy) { h[1] = s->Hy - 1; o[1] = one_minus; }
      if (h[1] < 0) { h[1] = 0; o[1] = 0.0; }
    } else {
      h[1] = ny_; o[1] = ty - (double)ky;
    }
    if (o[1] >= 1.0) { o[1] -= 1.0; h[1] += 1; if (h[1] >= s->Hy) { h[1] = s->Hy - 1; o[1] = one_minus; } }
    /* x, periodic inside the region (Sec. 2.3: no particle leaves it) */
    double tx = o[0] + dxe;
    int kx = (int)floor(tx);
    o[0] = tx - (double)kx;
    if (o[0] >= 1.0) { o[0] -= 1.0; kx += 1; }
    h[0] = imod(h[0] + kx, s->Wx);
    if (s->dim == 3) {
      double tz = o[2] + dze;
      int kz = (int)floor(tz);
      o[2] = tz - (double)kz;
      if (o[2] >= 1.0) { o[2] -= 1.0; kz += 1; }
      h[2] = imod(h[2] + kz, s->Wz);
    }
  }
}

/* a6: mass and momentum of the particles whose (unshifted) home cell lies in
 * an inner-buffer column, summed per LB node into this step's frame. */
static void sample_inner(orc_sim* s) {
  if (s->nbuf == 0) return;
  int W = s->p.window > 0 ? s->p.window : 1;
  double* fr = &s->frames[(size_t)(s->nframes % W) * s->nbuf * 4];
  memset(fr, 0, sizeof(double) * s->nbuf * 4);
  double m = s->p.mass;
  for (long k = 0; k < s->np; ++k) {
    long b = inner_node(s, s->home[3*k], s->home[3*k+1], s->home[3*k+2]);
    if (b < 0) continue;
    fr[4*b] += m;
    for (int a = 0; a < 3; ++a) fr[4*b+1+a] += m * s->vel[3*k+a];
  }
  s->nframes++;
}

/* binning decision of R10: the offset plus the shift, in the storage
 * precision, reaches the next cell when it is >= 1. */
int orc_bin_offset(double off, double sh, int precision) {
  if (precision == 0) return (off + sh) >= 1.0;
  float fo = (float)off, fs = (float)sh;
  float t = fo + fs;
  return t >= 1.0f;
}

/* a5: one random shift s in [0,1)^d per step (24-bit quanta, exact in both
 * precisions), cell index floor(r + s) per axis, counts and velocity sums. */
static void shift_and_bin(orc_sim* s) {
  uint32_t w[4];
  draw(s, 0u, (uint32_t)s->step, TAG_SHIFT, w);
  s->shift[0] = u24(w[0]); s->shift[1] = u24(w[1]);
  s->shift[2] = s->dim == 3 ? u24(w[2]) : 0.0;
  memset(s->cnt, 0, sizeof(int) * s->ncell);
  memset(s->sumv, 0, sizeof(double) * 3 * s->ncell);
  for (long k = 0; k < s->np; ++k) {
    int cx = imod(s->home[3*k] + orc_bin_offset(s->off[3*k], s->shift[0], s->p.precision), s->ncx);
    int cy = s->home[3*k+1] + orc_bin_offset(s->off[3*k+1], s->shift[1], s->p.precision);
    int cz = 0;
    if (s->dim == 3) cz = imod(s->home[3*k+2] + orc_bin_offset(s->off[3*k+2], s->shift[2], s->p.precision), s->ncz);
    long c = (long)cx + (long)s->ncx * ((long)cy + (long)s->ncy * cz);
    s->pcell[k] = (int)c;
    s->cnt[c] += 1;
    for (int a = 0; a < 3; ++a) s->sumv[3*c+a] += s->vel[3*k+a];
  }
}

/* Eq. 4 in 2D: v' = v_cm + R(+-alpha)(v - v_cm). */
void orc_srd_rotate_2d(double vx, double vy, double cx, double cy, double alpha,
                       int sign, double* ox, double* oy) {
  double th = sign > 0 ? alpha : -alpha;
  double wx = vx - cx, wy = vy - cy;
  *ox = cx + (cos(th) * wx - sin(th) * wy);
  *oy = cy + (sin(th) * wx + cos(th) * wy);
}

/* Eq. 4 in 3D: rotation by alpha about a unit axis n (Rodrigues' formula):
 * R w = w cos(alpha) + (n x w) sin(alpha) + n (n.w)(1 - cos(alpha)). */
void orc_srd_rotate_3d(const double v[3], const double vcm[3], const double n[3],
                       double alpha, double out[3]) {
  double w[3] = {v[0] - vcm[0], v[1] - vcm[1], v[2] - vcm[2]};
  double cr[3] = {n[1]*w[2] - n[2]*w[1], n[2]*w[0] - n[0]*w[2], n[0]*w[1] - n[1]*w[0]};
  double nw = n[0]*w[0] + n[1]*w[1] + n[2]*w[2];
  double ca = cos(alpha), sa = sin(alpha);
  for (int a = 0; a < 3; ++a) out[a] = vcm[a] + (w[a] * ca + cr[a] * sa + n[a] * nw * (1.0 - ca));
}

/* a7: SRD collision (Eq. 4).  A cell cut by a wall (rows 0 and Hy under a
 * nonzero shift) holding n_c < ppc particles gets ppc - n_c virtual wall
 * particles whose total momentum is drawn from N(0, (ppc - n_c) m kT) per
 * component (wall at rest); they enter v_cm only. */
static void collide_at(orc_sim* s);
static void collide(orc_sim* s) {
  const orc_params* p = &s->p;
  if (p->collision == 1) { collide_at(s); return; }
  for (long c = 0; c < s->ncell; ++c) {
    int n = s->cnt[c];
    for (int a = 0; a < 3; ++a) s->vcm[3*c+a] = 0.0;
    if (n == 0) continue;
    int cy = (int)((c / s->ncx) % s->ncy);
    int cut = (cy == 0 || (cy == s->Hy && !s->strip)) && s->shift[1] > 0.0;
    double P[3] = {s->sumv[3*c], s->sumv[3*c+1], s->sumv[3*c+2]};
    int ntot = n;
    if (cut && n < p->ppc) {
      int nv = p->ppc - n;
      uint32_t w[4]; draw(s, (uint32_t)c, (uint32_t)s->step, TAG_VIRT, w);
      double z0, z1, z2, z3;
      orc_box_muller(w[0], w[1], &z0, &z1);
      orc_box_muller(w[2], w[3], &z2, &z3);
      double sd = sqrt((double)nv * p->kT / p->mass);
      P[0] += sd * z0; P[1] += sd * z1;
      if (s->dim == 3) P[2] += sd * z2;
      ntot += nv;
    }
    for (int a = 0; a < 3; ++a) s->vcm[3*c+a] = P[a] / (double)ntot;
  }
  for (long k = 0; k < s->np; ++k) {
    long c = s->pcell[k];
    double* v = &s->vel[3*k];
    const double* vc = &s->vcm[3*c];
    if (s->dim == 2) {
      uint32_t w[4]; draw(s, (uint32_t)c, (uint32_t)s->step, TAG_SIGN, w);
      int sign = (w[0] >> 31) ? 1 : -1;
      double ox, oy;
      orc_srd_rotate_2d(v[0], v[1], vc[0], vc[1], p->alpha, sign, &ox, &oy);
      v[0] = ox; v[1] = oy;
    } else {
      uint32_t w[4]; draw(s, (uint32_t)c, (uint32_t)s->step, TAG_AXIS, w);
      double axis[3]; orc_random_axis(w[0], w[1], axis);
      double out[3]; orc_srd_rotate_3d(v, vc, axis, p->alpha, out);
      v[0] = out[0]; v[1] = out[1]; v[2] = out[2];
    }
  }
}

/* a7 with the Andersen thermostat, MPCD-AT (Eq. 6; collision = 1).  Every
 * particle k draws a random velocity v_ran,k with components N(0, kT/m)
 * (Box-Muller of Philox(k, n, replica, TAG_AT)) and leaves the collision with
 * v_k = v_cm + v_ran,k - <v_ran>, the mean taken over its collision cell: the
 * relative velocity is replaced, the cell momentum kept.  A wall-cut cell with
 * n_c < ppc holds ppc - n_c virtual particles that take part like real ones:
 * their velocity sum, N(0, (ppc - n_c) kT/m) per component from TAG_VIRT as for
 * SRD, enters v_cm, the sum of their random velocities, drawn the same way from
 * TAG_AT_VIRT, enters <v_ran>, and both means run over ppc particles. */
static void collide_at(orc_sim* s) {
  const orc_params* p = &s->p;
  const double sig = sqrt(p->kT / p->mass);
  for (long k = 0; k < s->np; ++k) {
    uint32_t w[4]; draw(s, (uint32_t)k, (uint32_t)s->step, TAG_AT, w);
    double z0, z1, z2, z3;
    orc_box_muller(w[0], w[1], &z0, &z1);
    orc_box_muller(w[2], w[3], &z2, &z3);
    s->vran[3*k] = sig * z0;
    s->vran[3*k+1] = sig * z1;
    s->vran[3*k+2] = s->dim == 3 ? sig * z2 : 0.0;
  }
  for (long c = 0; c < 3 * s->ncell; ++c) s->ranm[c] = 0.0;
  for (long k = 0; k < s->np; ++k)
    for (int a = 0; a < 3; ++a) s->ranm[3 * (long)s->pcell[k] + a] += s->vran[3*k+a];
  for (long c = 0; c < s->ncell; ++c) {
    int n = s->cnt[c];
    double P[3] = {s->sumv[3*c], s->sumv[3*c+1], s->sumv[3*c+2]};
    double X[3] = {s->ranm[3*c], s->ranm[3*c+1], s->ranm[3*c+2]};
    for (int a = 0; a < 3; ++a) { s->vcm[3*c+a] = 0.0; s->ranm[3*c+a] = 0.0; }
    if (n == 0) continue;
    int cy = (int)((c / s->ncx) % s->ncy);
    int cut = (cy == 0 || (cy == s->Hy && !s->strip)) && s->shift[1] > 0.0;
    int ntot = n;
    if (cut && n < p->ppc) {
      int nv = p->ppc - n;
      double sd = sqrt((double)nv * p->kT / p->mass);
      double z[4];
      uint32_t w[4]; draw(s, (uint32_t)c, (uint32_t)s->step, TAG_VIRT, w);
      orc_box_muller(w[0], w[1], &z[0], &z[1]);
      orc_box_muller(w[2], w[3], &z[2], &z[3]);
      for (int a = 0; a < s->dim; ++a) P[a] += sd * z[a];
      draw(s, (uint32_t)c, (uint32_t)s->step, TAG_AT_VIRT, w);
      orc_box_muller(w[0], w[1], &z[0], &z[1]);
      orc_box_muller(w[2], w[3], &z[2], &z[3]);
      for (int a = 0; a < s->dim; ++a) X[a] += sd * z[a];
      ntot += nv;
    }
    for (int a = 0; a < 3; ++a) { s->vcm[3*c+a] = P[a] / (double)ntot; s->ranm[3*c+a] = X[a] / (double)ntot; }
  }
  for (long k = 0; k < s->np; ++k) {
    long c = s->pcell[k];
    for (int a = 0; a < 3; ++a) s->vel[3*k+a] = s->vcm[3*c+a] + s->vran[3*k+a] - s->ranm[3*c+a];
  }
}

/* a8: on each inner-buffer LB node, rho_bar = rho0 M_W / (ppc m r^d W_n) and
 * u_bar = P_W / M_W from the last W_n = min(n+1, W) frames; the LB update of
 * the next step (a1, lb_step) gives the node the post-collision populations
 * f_eq(rho_LB, u_bar) (Eq. 2), rho_LB being the node's LB density of that
 * update: the imposition acts as the collision rule of the inner-buffer
 * nodes, since the frame of step n is complete only after step n's LB update.
 * The MPCD density is reported, not imposed: the two fluids have different
 * equations of state (LB pressure rho/3, MPCD pressure n kT), so MPCD density
 * fluctuations imposed on the LB become pressure gradients thousands of times
 * too strong and the coupled step diverges.  Nothing is imposed from the
 * first step's window (n = 0). */
static void impose(orc_sim* s) {
  const orc_params* p = &s->p;
  if (s->nbuf == 0) return;
  int W = p->window > 0 ? p->window : 1;
  long nf = s->nframes < W ? s->nframes : W;
  double rd = (s->dim == 3) ? (double)s->r * s->r * s->r : (double)s->r * s->r;
  for (long b = 0; b < s->nbuf; ++b) {
    double M = 0, P[3] = {0, 0, 0};
    for (long f = 0; f < nf; ++f) {
      const double* fr = &s->frames[(size_t)f * s->nbuf * 4 + 4*b];
      M += fr[0]; P[0] += fr[1]; P[1] += fr[2]; P[2] += fr[3];
    }
    double rho = M / ((double)p->ppc * p->mass * rd * (double)nf);
    double u[3] = {0, 0, 0};
    if (M > 0) { u[0] = P[0] / M; u[1] = P[1] / M; u[2] = P[2] / M; }
    s->wmean[4*b] = rho; s->wmean[4*b+1] = u[0]; s->wmean[4*b+2] = u[1]; s->wmean[4*b+3] = u[2];
    s->imp[4*b] = (p->feedback == 1 && s->step >= 1 && M > 0) ? 1.0 : 0.0;
    for (int a = 0; a < 3; ++a) s->imp[4*b+1+a] = u[a];
  }
}

/* ------------------------------------------------------------------------ */
/* Learned closure (feedback = 2, D2Q9; not in the paper).
 *
 * Strips: on each x-side, the CL_W fine columns nearest the region's edge;
 * xi = distance from the edge in fine cells (left: xi = X; right:
 * xi = Wx - 1 - X, the right strip seen in a mirror, so its u_x changes sign).
 * Strip cell c = (side Hy + Y) CL_W + xi.
 * Fields of one step, per strip cell, from the particles whose (unshifted)
 * home cell is c after streaming (the same instant as a6):
 *   phi_0 = n / ppc - 1,  phi_1 = +-(sum v_x / n) / sqrt(kT/m),
 *   phi_2 = (sum v_y / n) / sqrt(kT/m)   (velocities 0 in an empty cell).
 * Patches: side-major, ceil(Hy/16) per side; patch py covers rows
 * 16 py .. 16 py + 15, the last one rows Hy - 16 .. Hy - 1 (it may overlap the
 * one before).  Input pixel (row, xi) of a patch, channel 3 f + k = phi_k of
 * the f-th of the last 8 steps, oldest first (zeros for steps before 0).
 * Target: exponential moving average e <- e + (phi - e) / 500, e = phi at the
 * first frame (time constant 500 steps: the mean lag and the white-noise
 * variance of a 1000-step trailing mean). */
static long cl_row0(const orc_sim* s, int py) {
  return py == s->cl_npy - 1 ? s->Hy - CL_W : (long)CL_W * py;
}

static void closure_sample(orc_sim* s) {
  const long ncl = s->cl_ncell;
  memset(s->cl_frame, 0, sizeof(double) * ncl * 3);
  for (long k = 0; k < s->np; ++k) {
    int X = s->home[3*k], Y = s->home[3*k+1], side, xi;
    if (X < CL_W) { side = 0; xi = X; }
    else if (X >= s->Wx - CL_W) { side = 1; xi = s->Wx - 1 - X; }
    else continue;
    long c = ((long)side * s->Hy + Y) * CL_W + xi;
    s->cl_frame[3*c] += 1.0;
    s->cl_frame[3*c+1] += s->vel[3*k];
    s->cl_frame[3*c+2] += s->vel[3*k+1];
  }
  /* drop the oldest frame, append this one */
  memmove(s->cl_hist, s->cl_hist + ncl * 3, sizeof(double) * (CL_FRAMES - 1) * ncl * 3);
  double* nw = s->cl_hist + (size_t)(CL_FRAMES - 1) * ncl * 3;
  double sig = sqrt(s->p.kT / s->p.mass);
  for (long c = 0; c < ncl; ++c) {
    double n = s->cl_frame[3*c];
    double mirror = c >= (long)s->Hy * CL_W ? -1.0 : 1.0;
    double phi[3];
    phi[0] = n / (double)s->p.ppc - 1.0;
    phi[1] = n > 0 ? mirror * ((s->cl_frame[3*c+1] / n) / sig) : 0.0;
    phi[2] = n > 0 ? (s->cl_frame[3*c+2] / n) / sig : 0.0;
    for (int k = 0; k < 3; ++k) {
      nw[3*c+k] = phi[k];
      if (s->cl_nframes == 0) s->cl_ema[3*c+k] = phi[k];
      else s->cl_ema[3*c+k] += (phi[k] - s->cl_ema[3*c+k]) / CL_EMA_T;
    }
  }
  s->cl_nframes++;
  /* lay the history out as the network input */
  for (int pch = 0; pch < 2 * s->cl_npy; ++pch) {
    int side = pch / s->cl_npy, py = pch % s->cl_npy;
    long row0 = cl_row0(s, py);
    for (int y = 0; y < CL_W; ++y)
      for (int x = 0; x < CL_W; ++x) {
        long c = ((long)side * s->Hy + row0 + y) * CL_W + x;
        double* px = s->cl_x + (((size_t)pch * CL_W + y) * CL_W + x) * 3 * CL_FRAMES;
        for (int f = 0; f < CL_FRAMES; ++f)
          for (int k = 0; k < 3; ++k) px[3*f+k] = s->cl_hist[((size_t)f * ncl + c) * 3 + k];
      }
  }
}

long orc_closure_patches(const orc_sim* s) { return s->cl_on ? 2L * s->cl_npy : 0; }

/* Imposition from the network output: on each inner-buffer LB node, u_bar =
 * sqrt(kT/m) times the mean predicted velocity over the node's r x r fine
 * cells (u_x mirrored back on the right side).  As for a8, the LB update of
 * the next step gives the node the post-collision populations
 * f_eq(rho_LB, u_bar), rho_LB its density of that update (the MPCD density
 * is not imposed); this records u_bar for it.  Fine cell (row, xi) is read
 * from patch min(row / 16, npy - 1) of its side. */
int orc_closure_impose(orc_sim* s, const double* y) {
  const orc_params* p = &s->p;
  if (!s->cl_on) return -1;
  if (s->cl_nframes < CL_FRAMES) return 0;
  double sig = sqrt(p->kT / p->mass);
  for (int side = 0; side < 2; ++side)
    for (int col = 0; col < s->n_in; ++col)
      for (int yn = 1; yn < p->ny - 1; ++yn) {
        double su[2] = {0, 0};
        for (int a = 0; a < s->r; ++a)
          for (int b = 0; b < s->r; ++b) {
            int row = (yn - 1) * s->r + a, xi = (s->n_out + col) * s->r + b;
            int py = row / CL_W < s->cl_npy - 1 ? row / CL_W : s->cl_npy - 1;
            long pch = (long)side * s->cl_npy + py;
            long m = (pch * CL_W + (row - cl_row0(s, py))) * CL_W + xi;
            su[0] += y[3*m+1]; su[1] += y[3*m+2];
          }
        /* inner-buffer entry of the node (slab form, nz = 1) */
        long bi = ((long)side * s->n_in + col) * (p->ny - 2) + (yn - 1);
        s->imp[4*bi] = 1.0;
        s->imp[4*bi+1] = (side ? -1.0 : 1.0) * sig * su[0] / (double)(s->r * s->r);
        s->imp[4*bi+2] = sig * su[1] / (double)(s->r * s->r);
        s->imp[4*bi+3] = 0.0;
      }
  return 0;
}

void orc_u_fine(const orc_sim* s, int X, int Y, int Z, double out[3]) { u_fine(s, X, Y, Z, out); }

int orc_step(orc_sim* s, int nsteps) {
  for (int it = 0; it < nsteps; ++it) {
    lb_step(s);                       /* a1 */
    if (s->has_region) {
      if (s->p.resample_density) resample_density(s);   /* a2 + a3' */
      else resample(s);               /* a2 + a3 */
      stream(s);                      /* a4 */
      sample_inner(s);                /* a6 */
      if (s->cl_on) closure_sample(s);  /* closure input of the same instant */
      shift_and_bin(s);               /* a5 */
      collide(s);                     /* a7 */
      impose(s);                      /* a8 */
    }
    s->step++;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
long orc_field_size(const orc_sim* s, int field) {
  switch (field) {
    case ORC_RHO: return s->nnode;
    case ORC_U: return 3 * s->nnode;
    case ORC_POPS: return (long)s->q * s->nnode;
    case ORC_PART_POS: case ORC_PART_VEL: case ORC_PART_HOME: return 3 * s->np;
    case ORC_PART_CELL: case ORC_PART_ID: return s->np;
    case ORC_SHIFT: return 3;
    case ORC_CELL_COUNT: return s->ncell;
    case ORC_CELL_VCM: return 3 * s->ncell;
    case ORC_WINDOW_MEAN: return 4 * s->nbuf;
    case ORC_DIAG: return 9;
    case ORC_CLOSURE_IN: return s->cl_on ? 2L * s->cl_npy * CL_W * CL_W * 3 * CL_FRAMES : -1;
    case ORC_CLOSURE_TARGET: return s->cl_on ? 2L * s->cl_npy * CL_W * CL_W * 3 : -1;
    case ORC_PI: return 6 * s->nnode;
    case ORC_CELL_LIST: return s->np;
  }
  return -1;
}

/* DIAG: LB mass, LB momentum (x,y,z) of the stored populations over fluid
 * nodes; particle count, particle momentum (x,y,z), particle kinetic energy. */
static void diag(const orc_sim* s, double* d) {
  const orc_params* p = &s->p;
  for (int a = 0; a < 9; ++a) d[a] = 0;
  for (int z = 0; z < p->nz; ++z)
    for (int y = 1; y < p->ny - 1; ++y)
      for (int x = 0; x < p->nx; ++x)
        for (int i = 0; i < s->q; ++i) {
          double fv = s->f[i * s->nnode + nidx(s, x, y, z)];
          d[0] += fv; d[1] += fv * s->c[3*i]; d[2] += fv * s->c[3*i+1]; d[3] += fv * s->c[3*i+2];
        }
  d[4] = (double)s->np;
  for (long k = 0; k < s->np; ++k) {
    const double* v = &s->vel[3*k];
    d[5] += p->mass * v[0]; d[6] += p->mass * v[1]; d[7] += p->mass * v[2];
    d[8] += 0.5 * p->mass * (v[0]*v[0] + v[1]*v[1] + v[2]*v[2]);
  }
}

int orc_get_field(const orc_sim* s, int field, void* dst) {
  long n = orc_field_size(s, field);
  if (n < 0) return -1;
  double* D = (double*)dst; int* I = (int*)dst;
  switch (field) {
    case ORC_RHO: memcpy(D, s->rho, sizeof(double) * n); break;
    case ORC_U: memcpy(D, s->u, sizeof(double) * n); break;
    case ORC_POPS: memcpy(D, s->f, sizeof(double) * n); break;
    case ORC_PART_POS: memcpy(D, s->off, sizeof(double) * n); break;
    case ORC_PART_VEL: memcpy(D, s->vel, sizeof(double) * n); break;
    case ORC_PART_HOME: memcpy(I, s->home, sizeof(int) * n); break;
    case ORC_PART_CELL: memcpy(I, s->pcell, sizeof(int) * n); break;
    case ORC_PART_ID: for (long k = 0; k < n; ++k) I[k] = (int)k; break;
    case ORC_SHIFT: memcpy(D, s->shift, sizeof(double) * 3); break;
    case ORC_CELL_COUNT: memcpy(I, s->cnt, sizeof(int) * n); break;
    case ORC_CELL_VCM:   /* MPCD-AT: v_cm - <v_ran>, what each particle's own v_ran is added to */
      if (s->p.collision == 1) { for (long i = 0; i < n; ++i) D[i] = s->vcm[i] - s->ranm[i]; }
      else memcpy(D, s->vcm, sizeof(double) * n);
      break;
    case ORC_WINDOW_MEAN: memcpy(D, s->wmean, sizeof(double) * n); break;
    case ORC_PI: memcpy(D, s->pi, sizeof(double) * n); break;
    case ORC_CELL_LIST: {   /* for each cell in increasing order, its particles in increasing index */
      long m = 0;
      for (long c = 0; c < s->ncell; ++c)
        for (long k = 0; k < s->np; ++k)
          if (s->pcell[k] == c) I[m++] = (int)k;
      break;
    }
    case ORC_DIAG: diag(s, D); break;
    case ORC_CLOSURE_IN: memcpy(D, s->cl_x, sizeof(double) * n); break;
    case ORC_CLOSURE_TARGET:
      for (int pch = 0; pch < 2 * s->cl_npy; ++pch) {
        int side = pch / s->cl_npy, py = pch % s->cl_npy;
        for (int y = 0; y < CL_W; ++y)
          for (int x = 0; x < CL_W; ++x) {
            long c = ((long)side * s->Hy + cl_row0(s, py) + y) * CL_W + x;
            for (int k = 0; k < 3; ++k) D[(((long)pch * CL_W + y) * CL_W + x) * 3 + k] = s->cl_ema[3*c+k];
          }
      }
      break;
    default: return -1;
  }
  return 0;
}

int orc_set_field(orc_sim* s, int field, const void* src) {
  long n = orc_field_size(s, field);
  const double* D = (const double*)src; const int* I = (const int*)src;
  switch (field) {
    case ORC_POPS: memcpy(s->f, D, sizeof(double) * n); memcpy(s->fn, D, sizeof(double) * n); break;
    case ORC_PART_POS: memcpy(s->off, D, sizeof(double) * n); break;
    case ORC_PART_VEL: memcpy(s->vel, D, sizeof(double) * n); break;
    case ORC_PART_HOME: memcpy(s->home, I, sizeof(int) * n); break;
    case ORC_U: memcpy(s->u, D, sizeof(double) * n); break;
    default: return -1;
  }
  return 0;
}
