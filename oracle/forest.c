/*
 * Oracle: forest of quadtrees, leaf search, adjacency, and brute-force 2:1
 * balance.  Test infrastructure only (see oracle.h).
 *
 * Sec. 2 ("A quadtree layout"): a level-l quadrant of a unit block has edge
 * 2^-l; only leaves are stored; leaves are enumerated in Morton order.
 * Sec. 3 ("Dynamic grid adaptation"): refine/coarsen tags, then a 2:1 balance
 * step that may add refinement, so coarsening is not guaranteed.
 */
#include "internal.h"

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

static char g_err[512];

void or_set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

const char* or_last_error(void) { return g_err; }

#define LFINE 20 /* common resolution for Morton keys and adjacency tests */

static uint64_t spread(uint32_t v) {
  uint64_t r = 0;
  for (int k = 0; k < 32; ++k) r |= (uint64_t)((v >> k) & 1u) << (2 * k);
  return r;
}

static uint64_t morton(const or_leaf* a) {
  uint32_t X = (uint32_t)a->x << (LFINE - a->l);
  uint32_t Y = (uint32_t)a->y << (LFINE - a->l);
  return spread(X) | (spread(Y) << 1);
}

static int cmp_morton(const void* pa, const void* pb) {
  const or_leaf* a = (const or_leaf*)pa;
  const or_leaf* b = (const or_leaf*)pb;
  if (a->f != b->f) return a->f < b->f ? -1 : 1;
  if (a->b != b->b) return a->b < b->b ? -1 : 1;
  uint64_t ka = morton(a), kb = morton(b);
  if (ka != kb) return ka < kb ? -1 : 1;
  return a->l < b->l ? -1 : (a->l > b->l);
}

void or_sort_leaves(or_leaf* lv, int n) { qsort(lv, (size_t)n, sizeof(or_leaf), cmp_morton); }

static const or_forest* g_sort_forest;

static int key_cmp(const or_leaf* a, const or_leaf* b) {
  if (a->f != b->f) return a->f < b->f ? -1 : 1;
  if (a->b != b->b) return a->b < b->b ? -1 : 1;
  if (a->l != b->l) return a->l < b->l ? -1 : 1;
  if (a->x != b->x) return a->x < b->x ? -1 : 1;
  if (a->y != b->y) return a->y < b->y ? -1 : 1;
  return 0;
}

static int cmp_key_idx(const void* pa, const void* pb) {
  int ia = *(const int*)pa, ib = *(const int*)pb;
  return key_cmp(&g_sort_forest->lv[ia], &g_sort_forest->lv[ib]);
}

void or_build_index(or_forest* F) {
  free(F->byKey);
  F->byKey = (int*)malloc(sizeof(int) * (size_t)(F->n > 0 ? F->n : 1));
  for (int k = 0; k < F->n; ++k) F->byKey[k] = k;
  g_sort_forest = F;
  qsort(F->byKey, (size_t)F->n, sizeof(int), cmp_key_idx);
}

int or_find(const or_forest* F, int f, int b, int l, int x, int y) {
  or_leaf key = {f, b, l, x, y};
  int lo = 0, hi = F->n - 1;
  while (lo <= hi) {
    int mid = (lo + hi) / 2;
    int c = key_cmp(&F->lv[F->byKey[mid]], &key);
    if (c == 0) return F->byKey[mid];
    if (c < 0) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

int or_locate(const or_forest* F, int f, int* b, double* x, double* y) {
  int outx = (*x < 0.0 || *x >= 1.0), outy = (*y < 0.0 || *y >= 1.0);
  if (outx || outy) {
    if (F->P.domain == OR_WALLS) return -2;
    if (F->P.domain == OR_PERIODIC) {
      *x -= floor(*x);
      *y -= floor(*y);
    } else if (F->P.domain == OR_BRICK) {
      /* the point's place in the brick, wrapped periodically, gives its block */
      const int nx = F->P.brick[0], ny = F->P.brick[1];
      double X = (*b % nx) + *x, Y = (*b / nx) + *y;
      X -= nx * floor(X / nx);
      Y -= ny * floor(Y / ny);
      int bx = (int)floor(X), by = (int)floor(Y);
      if (bx >= nx) bx = nx - 1;
      if (by >= ny) by = ny - 1;
      *x = X - bx;
      *y = Y - by;
      *b = by * nx + bx;
    } else {
      int r = or_sphere_fold(b, x, y);
      if (r != 0) return r; /* -3: beyond a three-valent cube corner */
    }
  }
  for (int l = F->P.lmin; l <= F->P.lmax; ++l) {
    double s = ldexp(1.0, l);
    int xi = (int)floor(*x * s), yi = (int)floor(*y * s);
    int k = or_find(F, f, *b, l, xi, yi);
    if (k >= 0) return k;
  }
  return -1;
}

/* Do the closed squares of two distinct leaves intersect?  Brute force in a
 * common integer frame; for the periodic square the second leaf is also tried
 * shifted by one block length in each direction. */
int or_touch(const or_forest* F, const or_leaf* a, const or_leaf* c) {
  if (a->f != c->f) return 0;
  if (F->P.domain == OR_SPHERE) { /* closed boxes on the cube surface */
    long alo[3], ahi[3], clo[3], chi[3];
    or_sphere_box(a, LFINE, alo, ahi);
    or_sphere_box(c, LFINE, clo, chi);
    for (int k = 0; k < 3; ++k)
      if (alo[k] > chi[k] || clo[k] > ahi[k]) return 0;
    return 1;
  }
  long R = 1L << LFINE;
  long ax0 = (long)a->x << (LFINE - a->l), ax1 = (long)(a->x + 1) << (LFINE - a->l);
  long ay0 = (long)a->y << (LFINE - a->l), ay1 = (long)(a->y + 1) << (LFINE - a->l);
  long cx0 = (long)c->x << (LFINE - c->l), cx1 = (long)(c->x + 1) << (LFINE - c->l);
  long cy0 = (long)c->y << (LFINE - c->l), cy1 = (long)(c->y + 1) << (LFINE - c->l);
  /* the brick: both squares placed in the brick's frame (block (bx, by) at
   * (bx R, by R)), the brick's extent being the period */
  long PX = R, PY = R;
  if (F->P.domain == OR_BRICK) {
    const int nx = F->P.brick[0];
    PX = R * nx;
    PY = R * F->P.brick[1];
    ax0 += (a->b % nx) * R, ax1 += (a->b % nx) * R, ay0 += (a->b / nx) * R, ay1 += (a->b / nx) * R;
    cx0 += (c->b % nx) * R, cx1 += (c->b % nx) * R, cy0 += (c->b / nx) * R, cy1 += (c->b / nx) * R;
  } else if (a->b != c->b) {
    return 0;
  }
  int nshift = (F->P.domain == OR_PERIODIC || F->P.domain == OR_BRICK) ? 1 : 0;
  for (int sx = -nshift; sx <= nshift; ++sx)
    for (int sy = -nshift; sy <= nshift; ++sy) {
      long dx = sx * PX, dy = sy * PY;
      if (ax0 <= cx1 + dx && cx0 + dx <= ax1 && ay0 <= cy1 + dy && cy0 + dy <= ay1) return 1;
    }
  return 0;
}

or_forest* or_create(const or_params* P, int n, const int* leaves) {
  if (P->mbc * 4 > P->mx) {
    or_set_error("Proposition 1 needs mbc <= mx/4 (mx=%d, mbc=%d)", P->mx, P->mbc);
    return NULL;
  }
  if (P->lmin < 0 || P->lmax > OR_MAXLEV || P->lmin > P->lmax) {
    or_set_error("bad level range");
    return NULL;
  }
  if (P->vel_kind == OR_VEL_DEFORM &&
      (P->domain != OR_SPHERE || !(P->vel[1] != 0.0) || !(P->vel[2] != 0.0))) {
    or_set_error("the deformational velocity is for the sphere, with nonzero T and T_f");
    return NULL;
  }
  if (P->domain == OR_SPHERE && P->vel_kind != OR_VEL_ROTATION && P->vel_kind != OR_VEL_DEFORM) {
    or_set_error("the sphere takes the solid-body rotation or the deformational velocity");
    return NULL;
  }
  or_forest* F = (or_forest*)calloc(1, sizeof(or_forest));
  F->P = *P;
  F->n = n;
  F->S = P->mx + 2 * P->mbc;
  F->lv = (or_leaf*)malloc(sizeof(or_leaf) * (size_t)(n > 0 ? n : 1));
  for (int k = 0; k < n; ++k) {
    or_leaf a = {leaves[5 * k], leaves[5 * k + 1], leaves[5 * k + 2], leaves[5 * k + 3],
                 leaves[5 * k + 4]};
    F->lv[k] = a;
  }
  or_sort_leaves(F->lv, n);
  or_build_index(F);
  size_t cells = (size_t)n * F->S * F->S;
  F->q = (double*)malloc(sizeof(double) * (cells ? cells : 1));
  F->qold = (double*)malloc(sizeof(double) * (cells ? cells : 1));
  F->qT = (double*)malloc(sizeof(double) * (cells ? cells : 1));
  for (size_t c = 0; c < cells; ++c) F->q[c] = F->qold[c] = F->qT[c] = NAN;
  or_update_metrics(F);
  return F;
}

void or_update_metrics(or_forest* F) {
  free(F->kappa);
  free(F->phix);
  free(F->phiy);
  F->kappa = F->phix = F->phiy = NULL;
  if (F->P.domain != OR_SPHERE) return;
  size_t S = (size_t)F->S, n = (size_t)(F->n > 0 ? F->n : 1);
  F->kappa = (double*)malloc(sizeof(double) * n * S * S);
  F->phix = (double*)malloc(sizeof(double) * n * (S + 1) * S);
  F->phiy = (double*)malloc(sizeof(double) * n * S * (S + 1));
  double scale = F->P.vel_scale != 0.0 ? F->P.vel_scale : 1.0;
  double om[3] = {scale * F->P.vel[0], scale * F->P.vel[1], scale * F->P.vel[2]};
  const int deform = F->P.vel_kind == OR_VEL_DEFORM;
  if (deform) om[0] = om[1] = om[2] = 0.0;
  for (int p = 0; p < F->n; ++p) {
    or_sphere_metrics(&F->lv[p], F->P.mx, F->P.mbc, om, F->kappa + p * S * S,
                      F->phix + p * (S + 1) * S, F->phiy + p * S * (S + 1));
    /* time-dependent fluxes: those of t = 0 until a step sets its own */
    if (deform)
      or_sphere_psi_fluxes(&F->lv[p], &F->P, 0.0, F->phix + p * (S + 1) * S,
                           F->phiy + p * S * (S + 1));
  }
}

void or_destroy(or_forest* F) {
  if (!F) return;
  or_drop_cache(F);
  free(F->kappa);
  free(F->phix);
  free(F->phiy);
  free(F->bflux);
  free(F->lv);
  free(F->byKey);
  free(F->q);
  free(F->qold);
  free(F->qT);
  free(F);
}

int or_num_leaves(const or_forest* F) { return F->n; }

void or_set_params(or_forest* F, const or_params* P) {
  F->P.vel_scale = P->vel_scale;
  or_update_metrics(F); /* sphere fluxes carry the scale */
}

void or_get_leaves(const or_forest* F, int* out) {
  for (int k = 0; k < F->n; ++k) {
    out[5 * k] = F->lv[k].f;
    out[5 * k + 1] = F->lv[k].b;
    out[5 * k + 2] = F->lv[k].l;
    out[5 * k + 3] = F->lv[k].x;
    out[5 * k + 4] = F->lv[k].y;
  }
}

void or_set_q(or_forest* F, const double* q) {
  int mx = F->P.mx;
  for (int p = 0; p < F->n; ++p)
    for (int j = 0; j < mx; ++j)
      for (int i = 0; i < mx; ++i)
        F->q[(size_t)p * F->S * F->S + OR_IDX(F, i, j)] = q[((size_t)p * mx + j) * mx + i];
}

void or_get_q(const or_forest* F, double* q) {
  int mx = F->P.mx;
  for (int p = 0; p < F->n; ++p)
    for (int j = 0; j < mx; ++j)
      for (int i = 0; i < mx; ++i)
        q[((size_t)p * mx + j) * mx + i] = F->q[(size_t)p * F->S * F->S + OR_IDX(F, i, j)];
}

void or_get_q_full(const or_forest* F, double* q) {
  memcpy(q, F->q, sizeof(double) * (size_t)F->n * F->S * F->S);
}

void or_set_q_full(or_forest* F, const double* q) {
  memcpy(F->q, q, sizeof(double) * (size_t)F->n * F->S * F->S);
}
