/*
 * CPU oracle for the patch-AMR wave-propagation method (ForestClaw,
 * Calhoun & Burstedde, arXiv 1703.03116).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is a plain, slow, FP64 restatement of
 * the method used to check the CUDA path.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant with the CUDA path.
 *
 * Geometry is done by brute force: every ghost cell is located by searching
 * the leaf set for the quadrant that contains its centre (Sec. 2.2 "Ghost
 * regions"), instead of using a precomputed neighbour list.
 *
 * Refluxing (or_params.reflux) is not in the paper: it is the standard
 * correction of Berger and Colella (J. Comput. Phys. 82, 1989), which replaces
 * the flux a coarse cell used at a coarse/fine face by the fine fluxes through
 * that face, summed over the face's fine cells and the fine substeps.  On the
 * cubed sphere it also makes the fluxes through cube edges single-valued (the
 * block of lower index keeps its flux, the other side takes it).  Pinned by
 * first-order closed forms, by exact conservation of mass, and by the
 * constant state where all fluxes of a step share one velocity field.
 *
 * The sphere's deformational flow (OR_VEL_DEFORM, Sec. 5.3) takes its edge
 * volume fluxes from the time-dependent streamfunction at each step's half
 * time.  Pinned against the published velocity components of that flow, the
 * solid-body rotation it reduces to at half period, and the return of a
 * tracer after one period.
 *
 * The multirate time interpolation of coarse data is pinned by exactness on
 * linear data (a linear field translated by a constant velocity through an
 * adaptive forest).  The capacity form on the sphere is pinned through its
 * behaviour: capacities tiling the sphere, a rotated tracer landing where
 * the rotation puts it, convergence, the deformational flow's return.
 *
 * The metrics of a sphere patch's ghost cells (its own mapping extended past
 * its block) are pinned like its interior's: capacities against the
 * solid-angle closed form, edge fluxes against the published velocity.
 *
 * Parity unpinned (checked only against the same stated reading): the fill
 * of the corner ghost block at three-valent cube corners.
 */
#ifndef FC_ORACLE_H
#define FC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_WALLS = 0, OR_PERIODIC = 1, OR_SPHERE = 2, OR_BRICK = 3 };
enum { OR_VEL_CONST = 0, OR_VEL_SWIRL = 1, OR_VEL_ROTATION = 2 /* sphere: vel[0..2] = omega */,
       OR_VEL_DEFORM = 3 /* sphere: vel[0..2] = kappa, T, T_f of the Sec. 5.3 streamfunction */ };

#define OR_MAXLEV 18

typedef struct {
  int domain;      /* OR_WALLS, OR_PERIODIC, OR_SPHERE, OR_BRICK */
  int nforests;    /* independent forests (one block each for the square) */
  int mx, mbc;     /* interior cells per side, ghost layers */
  int lmin, lmax;  /* level range of the whole run */
  int vel_kind;    /* OR_VEL_CONST (vel[0]=u, vel[1]=v) or OR_VEL_SWIRL (vel[0]=T) */
  double vel[4];
  int order;       /* 1: first order, 2: second-order corrections */
  int limiter;     /* 0: unlimited (Lax-Wendroff), 1: MC */
  int transverse;  /* 0: none, 1: fluctuations, 2: fluctuations + corrections */
  double vel_scale; /* every edge speed is multiplied by this (0 is read as 1) */
  int indicator;   /* regrid indicator: 0 max |grad q| / 2, 1 max q - min q (Sec. 5.1) */
  int smooth;      /* 1: smooth grading of target levels before refining (Sec. 3.3) */
  int reflux;      /* 1: conservative correction of coarse cells at coarse/fine faces and, on
                      the sphere, of one side of every cube edge (an extension: the paper's
                      scheme has none) */
  int brick[2];    /* OR_BRICK (Sec. 5.1): blocks per row and per column; block b covers
                      [b % brick[0], +1] x [b / brick[0], +1] of the brick, whose outer
                      faces are periodic */
} or_params;

typedef struct or_forest or_forest;

/* leaves: n rows of (forest, block, level, ix, iy) */
or_forest* or_create(const or_params* P, int n, const int* leaves);
void or_destroy(or_forest* F);
/* take the velocity scale of P (the layout parameters cannot change) */
void or_set_params(or_forest* F, const or_params* P);
int or_num_leaves(const or_forest* F);
void or_get_leaves(const or_forest* F, int* out);
/* interior data, [leaf][j][i], leaves in the order of or_get_leaves */
void or_set_q(or_forest* F, const double* q);
void or_get_q(const or_forest* F, double* q);
/* full arrays with ghosts, [leaf][j][i] over (mx+2mbc)^2 */
void or_get_q_full(const or_forest* F, double* q);
void or_set_q_full(or_forest* F, const double* q);

int or_fill_ghosts(or_forest* F);                       /* Alg. 1 */
int or_step_global(or_forest* F, double t, double dt);  /* global time stepping */
int or_step_multirate(or_forest* F, double t, double dt_coarse);
int or_tag(or_forest* F, double* delta);                /* ghost fill + per-leaf indicator */
int or_regrid(or_forest* F, double tau_r, double tau_c, const int* lmax_f, int* changed);
void or_mass(const or_forest* F, double* per_forest);

/* Adjoint of global time stepping (reverse mode, a.e. derivatives of the
 * limiter and of the minmod interpolation slopes, branches taken from the
 * forward state).  Starting from the forest's current interior state q0, run
 * nsteps global steps (t0, dt), form L = 1/2 sum over interior cells of
 * (q_N - q_target)^2, and return dL/dq0 (interior layout, leaf order) and
 * dL/d(velocity scale) at the current scale.  The forest's state is left at
 * q0.  Every intermediate state is stored (test sizes only). */
int or_adjoint_global(or_forest* F, int nsteps, double t0, double dt, const double* q_target,
                      double* grad_q0, double* grad_scale, double* loss);

/* one adjoint step: given lam (interior, adjoint of q^{n+1}) and the current
 * state q^n, overwrite lam with the adjoint of q^n and add the step's
 * velocity-scale derivative to *dscale */
int or_adjoint_step_global(or_forest* F, double t, double dt, double* lam, double* dscale);

/* Adjoint of one coarse multirate step (Sec. 4 recursion, coarse level
 * first, time-interpolated coarse ghosts): given lam (interior, adjoint of
 * the state after the step) and the forest at the step's start, overwrite lam
 * with the adjoint of the start state and add the velocity-scale derivative
 * to *dscale.  The forest is left at the start state.  Square domains. */
int or_adjoint_step_multirate(or_forest* F, double t, double dt_coarse, double* lam,
                              double* dscale);
/* as or_adjoint_global, over ncoarse coarse multirate steps */
int or_adjoint_multirate(or_forest* F, int ncoarse, double t0, double dt_coarse,
                         const double* q_target, double* grad_q0, double* grad_scale,
                         double* loss);

/* cubed sphere: unit-sphere positions of every interior cell centre
 * (n x mx x mx x 3) and the cell capacities (n x mx x mx) */
void or_sphere_centres(const or_forest* F, double* xyz);
void or_get_kappa(const or_forest* F, double* kappa);
/* the capacities over the extended range, ghost cells included (n x S x S) */
void or_get_kappa_full(const or_forest* F, double* kappa);

/* refluxing's pairing: per leaf, face (-x, +x, -y, +y) and face cell, 5
 * ints (kind, leaf across, its face on the edge, j0, j1): kind 1 finer
 * across (j0, j1: its cells beside the lower and upper half of the cell),
 * 2 same level across a cube edge with this side on the block of higher index
 * (j0: its cell), 0 none (-1 elsewhere) */
void or_reflux_pairs(const or_forest* F, int* out);

/* cubed sphere: the edge volume fluxes of every leaf at time t (leaf order;
 * per leaf (S+1)*S x-edges then S*(S+1) y-edges over the extended range, as
 * or_sphere_metrics lays them out) */
void or_sphere_edge_fluxes(const or_forest* F, double t, double* phix, double* phiy);

/* one uniform periodic N x N grid, used to check the forest against it */
int or_single_grid_periodic(const or_params* P, int N, double* q, double t0,
                            double dt, int nsteps);

/* scalar building blocks, exposed for table checks */
double or_mc_phi(double theta);
double or_minmod(double a, double b);

const char* or_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
