/* Oracle internals (test infrastructure only; see oracle.h). */
#ifndef FC_ORACLE_INTERNAL_H
#define FC_ORACLE_INTERNAL_H

#include "oracle.h"
#include <stdint.h>

/* Loops over patches marked PATCH_LOOP touch each patch's own arrays only
 * (reading the others' interiors), so their iterations are independent.  The
 * plain build runs them in order; the OpenMP build of the same sources (the
 * all-cores timing baseline) splits them over host threads, with the same
 * results, since no iteration reads what another writes. */
#ifdef _OPENMP
#define PATCH_LOOP _Pragma("omp parallel for schedule(dynamic, 4)")
#else
#define PATCH_LOOP
#endif

typedef struct {
  int f, b, l, x, y;   /* forest, block, level, quadrant coordinates */
} or_leaf;

struct or_forest {
  or_params P;
  int n;
  int S;             /* mx + 2 mbc */
  or_leaf* lv;       /* leaves in (forest, block, Morton) order */
  int* byKey;        /* leaf indices sorted by (f, b, l, x, y) */
  double* q;         /* n * S * S, current solution with ghosts */
  double* qold;      /* state saved before a leaf's last advance (multirate) */
  double* qT;        /* time-interpolated coarse data (multirate) */
  void* gcache;      /* memoised ghost-cell holders of the current mesh */
  /* cubed sphere: per-leaf metric terms over the extended index range */
  double* kappa;     /* n * S * S cell capacities (spherical areas) */
  double* phix;      /* n * (S+1) * S x-edge volume fluxes */
  double* phiy;      /* n * S * (S+1) y-edge volume fluxes */
  /* refluxing: per leaf, two substep slots of the final fluxes through its
   * four faces ([slot][face][cell], faces -x, +x, -y, +y, mx cells each) */
  double* bflux;
  int nbflux;        /* leaves bflux is sized for */
  int fslot;         /* the slot the next leaf update writes */
};

/* sphere.c */
int or_sphere_fold(int* b, double* x, double* y);
void or_sphere_box(const or_leaf* a, int LF, long lo[3], long hi[3]);
void or_sphere_point(int b, double x, double y, double X[3]);
void or_sphere_metrics(const or_leaf* a, int mx, int mbc, const double* omega, double* kappa,
                       double* phix, double* phiy);
/* the edge volume fluxes of a leaf from the streamfunction of P at time t
 * (OR_VEL_DEFORM): phi = difference of psi between the edge's end points */
void or_sphere_psi_fluxes(const or_leaf* a, const or_params* P, double t, double* phix,
                          double* phiy);
void or_claw_step_capacity(const or_params* P, double* q, int mx, int mbc, double dt,
                           const double* kappa, const double* phix, const double* phiy,
                           double* bflux);
/* (re)compute the metric terms of every leaf (sphere only) */
void or_update_metrics(or_forest* F);

/* relation of the leaf that holds a ghost cell to the ghost's owner */
enum { REL_SAME = 0, REL_FINE = 1, REL_COARSE = -1, REL_EXTERIOR = -100,
       REL_CORNER3 = -101, REL_NONE = -102 };

#define OR_IDX(F, i, j) (((i) + (F)->P.mbc) + (F)->S * ((j) + (F)->P.mbc))

void or_set_error(const char* fmt, ...);

/* forest.c */
int or_find(const or_forest* F, int f, int b, int l, int x, int y);
/* locate the leaf of forest f holding block point (x, y) of block b.
 * Returns the leaf index, or -1.  May move the point into another block
 * (periodic wrap, cube-face crossing); *b, *x, *y are updated.
 * Returns -2 for a point outside the physical domain (walls) and -3 for a
 * point beyond a three-valent cube corner. */
int or_locate(const or_forest* F, int f, int* b, double* x, double* y);
void or_sort_leaves(or_leaf* lv, int n);
void or_build_index(or_forest* F);
int or_touch(const or_forest* F, const or_leaf* a, const or_leaf* c);

/* claw.c */
void or_claw_step(const or_params* P, double* q, int mx, int mbc, double h,
                  double dt, double t, long gx0, long gy0);
/* as or_claw_step; bflux (4 mx, may be NULL) receives the final fluxes through
 * the patch's faces: F at x-edges 0 and mx of each row, then G at y-edges 0
 * and mx of each column */
void or_claw_step_flux(const or_params* P, double* q, int mx, int mbc, double h, double dt,
                       double t, long gx0, long gy0, double* bflux);
/* edge speeds at velocity time t (the half step of the step using them) */
double or_u_edge(const or_params* P, double h, double t, long gx0, long gy0, int i, int j);
double or_v_edge(const or_params* P, double h, double t, long gx0, long gy0, int i, int j);

/* ghost.c: Alg. 1 that also returns the state after phase 2 (the data that
 * the interpolation reads), and the ghost-holder map of the current mesh */
int or_fill_all_snapshot(or_forest* F, double* snapshot);
int or_ghost_holder(or_forest* F, int p, int k, int* rel, int* src, double* x, double* y);

/* ghost.c */
int or_fill_all(or_forest* F);
int or_fill_level(or_forest* F, int level, double alpha);
/* the wave-propagation step of leaf p (flat or capacity form) */
void or_advance_leaf(or_forest* F, int p, double t, double dt);
void or_drop_cache(or_forest* F);

#endif
