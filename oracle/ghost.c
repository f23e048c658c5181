/*
 * Oracle: ghost-cell filling.  Test infrastructure only (see oracle.h).
 *
 * Follows Alg. 1 (update_ghost, Sec. 2.3) literally:
 *   1. fill all coarse ghost regions (copy from a same-size neighbour,
 *      Eq. transform with I_n = A I_c + F; average of four fine cells,
 *      Eq. ghost_coarse),
 *   2. physical boundary conditions on exterior ghosts,
 *   3. fill all fine ghost regions by interpolation from the coarse
 *      neighbour, q_f = q_c + (h/4) grad(q_c) . d_k (Eq. ghost_fine), with the
 *      gradient from one-sided differences limited by minmod (the "monotone"
 *      interpolation of Sec. 3.1),
 *   4. physical boundary conditions again.
 * Every ghost cell is located geometrically: its centre is mapped to the
 * leaf that contains it, and the level difference of that leaf decides
 * whether it is copied (same level), averaged (one finer) or interpolated
 * (one coarser).  All ghosts start as NaN, so a value that the algorithm
 * reads before it is valid shows up as NaN in the result.
 *
 * Physical boundary (walls): zeroth-order extrapolation.  An exterior ghost
 * takes the value of the owner's own cell whose index is clamped into the
 * interior along each direction that leaves the domain; the other index is
 * kept, so the source may be an edge ghost filled in phase 1 or 3.
 */
#include "internal.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int rel, src;
  double x, y; /* ghost centre in the source leaf's block coordinates */
} gmap;

static int nghost(const or_forest* F) { return F->S * F->S - F->P.mx * F->P.mx; }

static int is_ghost(const or_forest* F, int i, int j) {
  return i < 0 || j < 0 || i >= F->P.mx || j >= F->P.mx;
}

/* locate the holder of ghost cell (i,j) of leaf p */
static gmap classify(const or_forest* F, int p, int i, int j) {
  const or_leaf* a = &F->lv[p];
  int mx = F->P.mx;
  double h = 1.0 / ldexp((double)mx, a->l);
  double x = ((double)a->x * mx + i + 0.5) * h;
  double y = ((double)a->y * mx + j + 0.5) * h;
  int b = a->b;
  gmap g;
  int k = or_locate(F, a->f, &b, &x, &y);
  g.x = x;
  g.y = y;
  g.src = k;
  if (k == -2) g.rel = REL_EXTERIOR;
  else if (k == -3) g.rel = REL_CORNER3;
  else if (k < 0) g.rel = REL_NONE;
  else {
    int d = F->lv[k].l - a->l;
    g.rel = (d == 0) ? REL_SAME : (d == 1) ? REL_FINE : (d == -1) ? REL_COARSE : REL_NONE;
  }
  return g;
}

/* value of the cell of leaf n (array src) that contains block point (x, y) */
static double cell_at(const or_forest* F, int n, const double* src, double x, double y) {
  const or_leaf* c = &F->lv[n];
  int mx = F->P.mx;
  double s = ldexp((double)mx, c->l);
  int i = (int)floor(x * s) - c->x * mx;
  int j = (int)floor(y * s) - c->y * mx;
  return src[OR_IDX(F, i, j)];
}

static double copy_value(const or_forest* F, const gmap* g, double* const* srcp) {
  return cell_at(F, g->src, srcp[g->src], g->x, g->y);
}

/* Eq. ghost_coarse: mean of the four fine cells inside the coarse ghost cell;
 * on the sphere the mean is weighted by the cell areas (Sec. 2.5: cell areas
 * are needed to average onto a coarse ghost region of a mapped grid) */
static double average_value(const or_forest* F, const gmap* g, double* const* srcp) {
  const or_leaf* c = &F->lv[g->src];
  double hf = 1.0 / ldexp((double)F->P.mx, c->l);
  const double* src = srcp[g->src];
  double a0 = cell_at(F, g->src, src, g->x - 0.5 * hf, g->y - 0.5 * hf);
  double a1 = cell_at(F, g->src, src, g->x + 0.5 * hf, g->y - 0.5 * hf);
  double a2 = cell_at(F, g->src, src, g->x - 0.5 * hf, g->y + 0.5 * hf);
  double a3 = cell_at(F, g->src, src, g->x + 0.5 * hf, g->y + 0.5 * hf);
  if (F->P.domain == OR_SPHERE) {
    const double* K = F->kappa + (size_t)g->src * F->S * F->S;
    double k0 = cell_at(F, g->src, K, g->x - 0.5 * hf, g->y - 0.5 * hf);
    double k1 = cell_at(F, g->src, K, g->x + 0.5 * hf, g->y - 0.5 * hf);
    double k2 = cell_at(F, g->src, K, g->x - 0.5 * hf, g->y + 0.5 * hf);
    double k3 = cell_at(F, g->src, K, g->x + 0.5 * hf, g->y + 0.5 * hf);
    return (((k0 * a0 + k1 * a1) + k2 * a2) + k3 * a3) / (((k0 + k1) + k2) + k3);
  }
  return 0.25 * (((a0 + a1) + a2) + a3);
}

/* Three-valent cube corner (no corner neighbour; a stated reading): the
 * corner ghost cell takes the mean of the two edge ghosts that share its
 * row and column next to the patch, once the edge ghosts are final. */
static void corner3_fill(or_forest* F, const gmap* G, int p, double* Q);

double or_minmod(double a, double b) {
  if (a * b <= 0.0) return 0.0;
  return fabs(a) < fabs(b) ? a : b;
}

/* Eq. ghost_fine in the coarse leaf's index space */
static double interp_value(const or_forest* F, const gmap* g, double* const* srcp) {
  const or_leaf* c = &F->lv[g->src];
  int mx = F->P.mx;
  double s = ldexp((double)mx, c->l);
  int ic = (int)floor(g->x * s) - c->x * mx;
  int jc = (int)floor(g->y * s) - c->y * mx;
  double xc = ((double)c->x * mx + ic + 0.5) / s;
  double yc = ((double)c->y * mx + jc + 0.5) / s;
  double dx = (g->x > xc) ? 1.0 : -1.0;
  double dy = (g->y > yc) ? 1.0 : -1.0;
  const double* Q = srcp[g->src];
  double q0 = Q[OR_IDX(F, ic, jc)];
  double sx = or_minmod(Q[OR_IDX(F, ic + 1, jc)] - q0, q0 - Q[OR_IDX(F, ic - 1, jc)]);
  double sy = or_minmod(Q[OR_IDX(F, ic, jc + 1)] - q0, q0 - Q[OR_IDX(F, ic, jc - 1)]);
  return q0 + 0.25 * (sx * dx + sy * dy);
}

/* zeroth-order extrapolation at walls */
static void apply_bc(const or_forest* F, int p, double* Q) {
  if (F->P.domain != OR_WALLS) return;
  const or_leaf* a = &F->lv[p];
  int mx = F->P.mx, mbc = F->P.mbc;
  int nb = 1 << a->l;
  for (int j = -mbc; j < mx + mbc; ++j)
    for (int i = -mbc; i < mx + mbc; ++i) {
      if (!is_ghost(F, i, j)) continue;
      int gi = a->x * mx + i, gj = a->y * mx + j; /* global cell index at this level */
      int outx = gi < 0 || gi >= nb * mx, outy = gj < 0 || gj >= nb * mx;
      if (!outx && !outy) continue;
      int ic = i, jc = j;
      if (outx) ic = (gi < 0) ? 0 : mx - 1;
      if (outy) jc = (gj < 0) ? 0 : mx - 1;
      Q[OR_IDX(F, i, j)] = Q[OR_IDX(F, ic, jc)];
    }
}

static void set_ghosts_nan(const or_forest* F, double* Q) {
  int mx = F->P.mx, mbc = F->P.mbc;
  for (int j = -mbc; j < mx + mbc; ++j)
    for (int i = -mbc; i < mx + mbc; ++i)
      if (is_ghost(F, i, j)) Q[OR_IDX(F, i, j)] = NAN;
}

/* classify every ghost cell of every leaf; memoised per mesh */
static const gmap* classify_all(or_forest* F) {
  if (F->gcache) return (const gmap*)F->gcache;
  int ng = nghost(F);
  gmap* G = (gmap*)malloc(sizeof(gmap) * (size_t)(F->n > 0 ? F->n : 1) * ng);
  int mx = F->P.mx, mbc = F->P.mbc;
  PATCH_LOOP
  for (int p = 0; p < F->n; ++p) {
    int k = 0;
    for (int j = -mbc; j < mx + mbc; ++j)
      for (int i = -mbc; i < mx + mbc; ++i)
        if (is_ghost(F, i, j)) G[(size_t)p * ng + k++] = classify(F, p, i, j);
  }
  F->gcache = G;
  return G;
}

void or_drop_cache(or_forest* F) {
  free(F->gcache);
  F->gcache = NULL;
}

static int check_map(const or_forest* F, const gmap* G, int p) {
  int ng = nghost(F);
  for (int k = 0; k < ng; ++k) {
    int r = G[(size_t)p * ng + k].rel;
    if (r == REL_NONE) {
      or_set_error("leaf %d: ghost cell %d has no valid holder (forest not 2:1 balanced?)", p, k);
      return -1;
    }
  }
  return 0;
}

/* phase 1 or 3 for one leaf: write ghosts of relation `want` into dst */
static void fill_regions(const or_forest* F, const gmap* G, int p, double* dst,
                         double* const* srcp, int want) {
  int ng = nghost(F), mx = F->P.mx, mbc = F->P.mbc, k = 0;
  for (int j = -mbc; j < mx + mbc; ++j)
    for (int i = -mbc; i < mx + mbc; ++i) {
      if (!is_ghost(F, i, j)) continue;
      const gmap* g = &G[(size_t)p * ng + k++];
      if (g->rel != want) continue;
      double v;
      if (want == REL_SAME) v = copy_value(F, g, srcp);
      else if (want == REL_FINE) v = average_value(F, g, srcp);
      else v = interp_value(F, g, srcp);
      dst[OR_IDX(F, i, j)] = v;
    }
}

int or_fill_all(or_forest* F) { return or_fill_all_snapshot(F, NULL); }

int or_ghost_holder(or_forest* F, int p, int k, int* rel, int* src, double* x, double* y) {
  const gmap* G = classify_all(F);
  const gmap* g = &G[(size_t)p * nghost(F) + k];
  *rel = g->rel;
  *src = g->src;
  *x = g->x;
  *y = g->y;
  return 0;
}

int or_fill_all_snapshot(or_forest* F, double* snapshot) {
  size_t S2 = (size_t)F->S * F->S;
  const gmap* G = classify_all(F);
  for (int p = 0; p < F->n; ++p)
    if (check_map(F, G, p)) return -1;
  double** cur = (double**)malloc(sizeof(double*) * (size_t)(F->n > 0 ? F->n : 1));
  for (int p = 0; p < F->n; ++p) {
    cur[p] = F->q + p * S2;
    set_ghosts_nan(F, cur[p]);
  }
  /* phase 1: copy and average into coarse ghost regions, all levels */
  PATCH_LOOP
  for (int p = 0; p < F->n; ++p) {
    fill_regions(F, G, p, cur[p], cur, REL_SAME);
    fill_regions(F, G, p, cur[p], cur, REL_FINE);
  }
  /* phase 2 */
  PATCH_LOOP
  for (int p = 0; p < F->n; ++p) apply_bc(F, p, cur[p]);
  /* phase 3: interpolate fine ghost regions from a snapshot of phase 2 */
  double* snap = (double*)malloc(sizeof(double) * (S2 * F->n > 0 ? S2 * F->n : 1));
  memcpy(snap, F->q, sizeof(double) * S2 * F->n);
  double** sp = (double**)malloc(sizeof(double*) * (size_t)(F->n > 0 ? F->n : 1));
  for (int p = 0; p < F->n; ++p) sp[p] = snap + p * S2;
  PATCH_LOOP
  for (int p = 0; p < F->n; ++p) fill_regions(F, G, p, cur[p], sp, REL_COARSE);
  /* phase 4 */
  PATCH_LOOP
  for (int p = 0; p < F->n; ++p) apply_bc(F, p, cur[p]);
  PATCH_LOOP
  for (int p = 0; p < F->n; ++p) corner3_fill(F, G, p, cur[p]);
  if (snapshot) memcpy(snapshot, snap, sizeof(double) * S2 * F->n);
  free(sp);
  free(snap);
  free(cur);
  return 0;
}

/* Ghost fill for one multirate substep of level L at a time that lies a
 * fraction alpha into the last step of level L-1.  Level L-1 data are
 * linearly interpolated in time from its saved and current states into qT;
 * their coarse ghost regions are filled from qT (same level) and from level
 * L (finer), then level L's own coarse ghost regions, then level L's fine
 * ghost regions by interpolation from qT.  Ghosts of qT whose holder is
 * coarser than L-1 are left NaN. */
int or_fill_level(or_forest* F, int L, double alpha) {
  size_t S2 = (size_t)F->S * F->S;
  int mx = F->P.mx;
  const gmap* G = classify_all(F);
  for (int p = 0; p < F->n; ++p)
    if ((F->lv[p].l == L || F->lv[p].l == L - 1) && check_map(F, G, p)) return -1;
  double** srcp = (double**)malloc(sizeof(double*) * (size_t)(F->n > 0 ? F->n : 1));
  for (int p = 0; p < F->n; ++p) {
    srcp[p] = (F->lv[p].l == L - 1) ? F->qT + p * S2 : F->q + p * S2;
    if (F->lv[p].l == L - 1) {
      double* T = F->qT + p * S2;
      const double* o = F->qold + p * S2;
      const double* c = F->q + p * S2;
      for (size_t k = 0; k < S2; ++k) T[k] = NAN;
      for (int j = 0; j < mx; ++j)
        for (int i = 0; i < mx; ++i) {
          size_t id = OR_IDX(F, i, j);
          T[id] = (1.0 - alpha) * o[id] + alpha * c[id];
        }
    } else if (F->lv[p].l == L) {
      set_ghosts_nan(F, F->q + p * S2);
    }
  }
  PATCH_LOOP
  for (int p = 0; p < F->n; ++p)
    if (F->lv[p].l == L - 1 || F->lv[p].l == L) {
      fill_regions(F, G, p, srcp[p], srcp, REL_SAME);
      fill_regions(F, G, p, srcp[p], srcp, REL_FINE);
    }
  PATCH_LOOP
  for (int p = 0; p < F->n; ++p)
    if (F->lv[p].l == L - 1 || F->lv[p].l == L) apply_bc(F, p, srcp[p]);
  PATCH_LOOP
  for (int p = 0; p < F->n; ++p)
    if (F->lv[p].l == L) fill_regions(F, G, p, srcp[p], srcp, REL_COARSE);
  PATCH_LOOP
  for (int p = 0; p < F->n; ++p)
    if (F->lv[p].l == L) apply_bc(F, p, srcp[p]);
  PATCH_LOOP
  for (int p = 0; p < F->n; ++p)
    if (F->lv[p].l == L - 1 || F->lv[p].l == L) corner3_fill(F, G, p, srcp[p]);
  free(srcp);
  return 0;
}

static void corner3_fill(or_forest* F, const gmap* G, int p, double* Q) {
  if (F->P.domain != OR_SPHERE) return;
  int ng = nghost(F), mx = F->P.mx, mbc = F->P.mbc, k = 0;
  for (int j = -mbc; j < mx + mbc; ++j)
    for (int i = -mbc; i < mx + mbc; ++i) {
      if (!is_ghost(F, i, j)) continue;
      const gmap* g = &G[(size_t)p * ng + k++];
      if (g->rel != REL_CORNER3) continue;
      int ic = i < 0 ? 0 : mx - 1, jc = j < 0 ? 0 : mx - 1;
      Q[OR_IDX(F, i, j)] = 0.5 * (Q[OR_IDX(F, i, jc)] + Q[OR_IDX(F, ic, j)]);
    }
}
