/*
 * Oracle: time stepping, tagging, regridding and mass.
 * Test infrastructure only (see oracle.h).
 *
 * Global time stepping (Sec. 5.1 runs): one time step for every grid, ghost
 * fill of all levels by Alg. 1 before each step.
 *
 * Multirate stepping (Sec. 4, local time stepping): 2^(lmax-lmin) steps of
 * the finest level per coarse step.  Reading used here: recursive order,
 * coarse level first; before each substep of level L, Alg. 1 restricted to
 * levels L-1 and L, with level L-1 data linearly interpolated in time between
 * its state before and after its own last step.
 *
 * Regridding (Sec. 3.1): a grid is tagged for refinement when its indicator
 * exceeds tau_r; a family of four sibling leaves is tagged for coarsening
 * when all four indicators are below tau_c.  The indicator is the largest
 * undivided gradient magnitude over the interior,
 *   delta = max 1/2 sqrt((q(i+1,j)-q(i-1,j))^2 + (q(i,j+1)-q(i,j-1))^2).
 * The new layout: tagged grids refined, then 2:1 balance by refinement only
 * (Sec. 2: face and corner neighbours differ by at most one level), then each
 * tagged family coarsened if its parent is balanced against that layout.
 * New fine grids are filled by the ghost-fill interpolation (Eq. ghost_fine
 * in the parent's index space), new coarse grids by averaging (Eq.
 * ghost_coarse), unchanged grids are copied.
 */
#include "internal.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static double cell_h(const or_forest* F, int l) { return 1.0 / ldexp((double)F->P.mx, l); }

void or_advance_leaf(or_forest* F, int p, double t, double dt) {
  const or_leaf* a = &F->lv[p];
  size_t S2 = (size_t)F->S * F->S, S = (size_t)F->S;
  double* bf = (F->P.reflux && F->bflux) ? F->bflux + ((size_t)p * 2 + F->fslot) * 4 * F->P.mx
                                          : NULL;
  if (F->P.domain == OR_SPHERE) {
    /* a time-dependent streamfunction: the fluxes of the step's half time */
    if (F->P.vel_kind == OR_VEL_DEFORM)
      or_sphere_psi_fluxes(a, &F->P, t + 0.5 * dt, F->phix + p * (S + 1) * S,
                           F->phiy + p * S * (S + 1));
    or_claw_step_capacity(&F->P, F->q + p * S2, F->P.mx, F->P.mbc, dt, F->kappa + p * S2,
                          F->phix + p * (S + 1) * S, F->phiy + p * S * (S + 1), bf);
    return;
  }
  or_claw_step_flux(&F->P, F->q + p * S2, F->P.mx, F->P.mbc, cell_h(F, a->l), dt, t,
                    (long)a->x * F->P.mx, (long)a->y * F->P.mx, bf);
}

/* the face-flux store of the current leaves (refluxing) */
static void flux_store(or_forest* F) {
  if (!F->P.reflux || (F->bflux && F->nbflux == F->n)) return;
  free(F->bflux);
  size_t m = (size_t)(F->n > 0 ? F->n : 1) * 2 * 4 * F->P.mx;
  F->bflux = (double*)malloc(sizeof(double) * m);
  for (size_t c = 0; c < m; ++c) F->bflux[c] = NAN;
  F->nbflux = F->n;
}

/* the leaf across a face and the cell it holds at a point there: located from
 * the point at depth d beyond the face and the point one cell of that leaf
 * deeper (cell: that leaf's cell width), whose step gives the leaf's face on
 * the shared edge (g: 0 -x, 1 +x, 2 -y, 3 +y) and the cell's index along it.
 * Returns the leaf or -1; with cell = 0 only the leaf is located. */
static int across(const or_forest* F, const or_leaf* a, int dir, double along, double d,
                  double cell, int* g, int* jn) {
  const int mx = F->P.mx;
  const double h = cell_h(F, a->l);
  const double x0 = a->x * mx * h, y0 = a->y * mx * h, x1 = x0 + mx * h, y1 = y0 + mx * h;
  int leaf[2], ix[2], iy[2];
  for (int c = 0; c < 2; ++c) {
    double dd = d + c * cell, x, y;
    if (dir < 2) {
      x = dir == 0 ? x0 - dd : x1 + dd;
      y = y0 + along;
    } else {
      x = x0 + along;
      y = dir == 2 ? y0 - dd : y1 + dd;
    }
    int b = a->b;
    leaf[c] = or_locate(F, a->f, &b, &x, &y);
    if (leaf[c] < 0) return -1;
    const or_leaf* n = &F->lv[leaf[c]];
    double hn = cell_h(F, n->l);
    ix[c] = (int)floor(x / hn) - n->x * mx;
    iy[c] = (int)floor(y / hn) - n->y * mx;
  }
  if (leaf[0] != leaf[1]) return -1;
  if (cell == 0.0) return leaf[0]; /* the leaf only */
  int di = ix[1] - ix[0], dj = iy[1] - iy[0];
  if (di == 1 && dj == 0) *g = 0;
  else if (di == -1 && dj == 0) *g = 1;
  else if (di == 0 && dj == 1) *g = 2;
  else if (di == 0 && dj == -1) *g = 3;
  else return -1;
  *jn = *g < 2 ? iy[0] : ix[0];
  return leaf[0];
}

/*
 * Refluxing of level L (Berger and Colella's correction; the paper's scheme
 * has none), after one level-L update of length dt whose face fluxes are in
 * slot cslot.  With s_f = -1 on a -x or -y face and +1 on a +x or +y face, a
 * cell's update took out = s_f F through each face.  Across a face whose
 * other side is finer, the fine side's fluxes are the ones kept: the coarse
 * cell's outflow becomes out' = -w sum s_g F_fine over the two fine cells
 * across it and the nfs fine substeps (g the fine leaf's face on that edge;
 * w = (fine dt / dt) times the length ratio of a fine face for fluxes per
 * unit length -- 1/4 and 1/2 on the square with two substeps or one --, or
 * fine dt / dt for the sphere's volume fluxes), by q += c (out - out'), c =
 * dt/h on the square, dt/kappa of the cell on the sphere.  Across a cube
 * edge between two leaves of the same level (each side computes that edge's
 * flux from its own ghost cells), the side on the block of lower index keeps
 * its flux and the other takes out' = -s_g F_nb of the same substep.  Leaves
 * across are found by locating points beyond the face.  Faces are corrected
 * in the order -x, +x, -y, +y (a corner cell takes two).
 */
/* What refluxing exchanges at coarse face cell k of leaf p, face dir: kind 1
 * (finer across: leaf *pn's face *g, its cells *j0 and *j1 beside the lower
 * and upper half of cell k), kind 2 (same level across a cube edge, this side
 * on the block of higher index: leaf *pn's face *g, cell *j0), else 0. */
static int reflux_pair(const or_forest* F, int p, int dir, int k, int* pn, int* g, int* j0,
                       int* j1) {
  const or_leaf* a = &F->lv[p];
  const double h = cell_h(F, a->l);
  int gg, jn;
  /* the level across: at a quarter cell beyond the face, a fine cell's
   * centre, or inside a same-size or coarser cell */
  int n = across(F, a, dir, (k + 0.5) * h, 0.25 * h, 0.0, &gg, &jn);
  if (n < 0) return 0;
  if (F->lv[n].l == a->l + 1) {
    /* the two fine cells across coarse cell k */
    int g0, g1, i0, i1;
    int n1 = across(F, a, dir, (k + 0.75) * h, 0.25 * h, 0.5 * h, &g1, &i1);
    int n0 = across(F, a, dir, (k + 0.25) * h, 0.25 * h, 0.5 * h, &g0, &i0);
    if (n0 != n || n1 != n || g0 != g1) return 0;
    *pn = n;
    *g = g0;
    *j0 = i0;
    *j1 = i1;
    return 1;
  }
  if (F->lv[n].l == a->l && F->P.domain == OR_SPHERE && F->lv[n].b < a->b) {
    n = across(F, a, dir, (k + 0.5) * h, 0.5 * h, h, &gg, &jn);
    if (n < 0) return 0;
    *pn = n;
    *g = gg;
    *j0 = jn;
    *j1 = -1;
    return 2;
  }
  return 0;
}

void or_reflux_pairs(const or_forest* F, int* out) {
  const int mx = F->P.mx;
  for (int p = 0; p < F->n; ++p)
    for (int dir = 0; dir < 4; ++dir)
      for (int k = 0; k < mx; ++k) {
        int* o = out + (((size_t)p * 4 + dir) * mx + k) * 5;
        int pn = -1, g = -1, j0 = -1, j1 = -1;
        o[0] = reflux_pair(F, p, dir, k, &pn, &g, &j0, &j1);
        o[1] = o[0] ? pn : -1;
        o[2] = o[0] ? g : -1;
        o[3] = o[0] ? j0 : -1;
        o[4] = o[0] == 1 ? j1 : -1;
      }
}

static void reflux_level(or_forest* F, int L, double dt, int cslot, int nfs, double wt) {
  const int mx = F->P.mx;
  const int sphere = F->P.domain == OR_SPHERE;
  const size_t S2 = (size_t)F->S * F->S, fs = 4 * (size_t)mx;
  const double h = cell_h(F, L);
  const double w = sphere ? wt : 0.5 * wt;
  for (int p = 0; p < F->n; ++p) {
    const or_leaf* a = &F->lv[p];
    if (a->l != L) continue;
    double* Q = F->q + p * S2;
    for (int dir = 0; dir < 4; ++dir)
      for (int k = 0; k < mx; ++k) {
        const double sf = (dir & 1) ? 1.0 : -1.0;
        int pn, g, j0, j1;
        const int kind = reflux_pair(F, p, dir, k, &pn, &g, &j0, &j1);
        if (!kind) continue;
        const double sg = (g & 1) ? 1.0 : -1.0;
        double target;
        if (kind == 1) {
          double fsum = 0.0;
          for (int s = 0; s < nfs; ++s)
            fsum += F->bflux[((size_t)pn * 2 + s) * fs + (size_t)g * mx + j0] +
                    F->bflux[((size_t)pn * 2 + s) * fs + (size_t)g * mx + j1];
          target = -sg * (w * fsum);
        } else {
          target = -sg * F->bflux[((size_t)pn * 2 + cslot) * fs + (size_t)g * mx + j0];
        }
        const double out = sf * F->bflux[((size_t)p * 2 + cslot) * fs + (size_t)dir * mx + k];
        const int i = dir == 0 ? 0 : dir == 1 ? mx - 1 : k;
        const int j = dir == 2 ? 0 : dir == 3 ? mx - 1 : k;
        const double c = sphere ? dt / F->kappa[p * S2 + OR_IDX(F, i, j)] : dt / h;
        Q[OR_IDX(F, i, j)] += c * (out - target);
      }
  }
}

int or_fill_ghosts(or_forest* F) { return or_fill_all(F); }

int or_step_global(or_forest* F, double t, double dt) {
  if (or_fill_all(F)) return -1;
  flux_store(F);
  F->fslot = 0;
  PATCH_LOOP
  for (int p = 0; p < F->n; ++p) or_advance_leaf(F, p, t, dt);
  if (F->P.reflux) /* every level took one step of dt: one fine step of the same dt */
    for (int L = F->P.lmin; L <= F->P.lmax; ++L) reflux_level(F, L, dt, 0, 1, 1.0);
  return 0;
}

static int mr_level(or_forest* F, int L, double t, double dt, double alpha) {
  size_t S2 = (size_t)F->S * F->S;
  if (or_fill_level(F, L, alpha)) return -1;
  const int slot = alpha != 0.0; /* the second substep of a pair */
  F->fslot = slot;
  PATCH_LOOP
  for (int p = 0; p < F->n; ++p)
    if (F->lv[p].l == L) {
      memcpy(F->qold + p * S2, F->q + p * S2, sizeof(double) * S2);
      or_advance_leaf(F, p, t, dt);
    }
  if (L < F->P.lmax) {
    if (mr_level(F, L + 1, t, 0.5 * dt, 0.0)) return -1;
    if (mr_level(F, L + 1, t + 0.5 * dt, 0.5 * dt, 0.5)) return -1;
  }
  /* after both finer substeps of this step (two slots of dt/2) */
  if (F->P.reflux) reflux_level(F, L, dt, slot, 2, 0.5);
  return 0;
}

int or_step_multirate(or_forest* F, double t, double dt_coarse) {
  flux_store(F);
  return mr_level(F, F->P.lmin, t, dt_coarse, 0.0);
}

int or_tag(or_forest* F, double* delta) {
  if (or_fill_all(F)) return -1;
  size_t S2 = (size_t)F->S * F->S;
  int mx = F->P.mx;
  if (F->P.indicator == 1) {
    /* Sec. 5.1: the spread of the patch's values, largest minus smallest */
    for (int p = 0; p < F->n; ++p) {
      const double* Q = F->q + p * S2;
      double lo = Q[OR_IDX(F, 0, 0)], hi = lo;
      for (int j = 0; j < mx; ++j)
        for (int i = 0; i < mx; ++i) {
          double v = Q[OR_IDX(F, i, j)];
          if (v < lo) lo = v;
          if (v > hi) hi = v;
        }
      delta[p] = hi - lo;
    }
    return 0;
  }
  for (int p = 0; p < F->n; ++p) {
    const double* Q = F->q + p * S2;
    double m = 0.0;
    for (int j = 0; j < mx; ++j)
      for (int i = 0; i < mx; ++i) {
        double gx = Q[OR_IDX(F, i + 1, j)] - Q[OR_IDX(F, i - 1, j)];
        double gy = Q[OR_IDX(F, i, j + 1)] - Q[OR_IDX(F, i, j - 1)];
        double d = 0.5 * sqrt(gx * gx + gy * gy);
        if (d > m) m = d;
      }
    delta[p] = m;
  }
  return 0;
}

/* ---- new layout ---- */

typedef struct {
  or_leaf* a;
  int n, cap;
} leafvec;

static void push(leafvec* v, or_leaf x) {
  if (v->n == v->cap) {
    v->cap = v->cap ? 2 * v->cap : 64;
    v->a = (or_leaf*)realloc(v->a, sizeof(or_leaf) * (size_t)v->cap);
  }
  v->a[v->n++] = x;
}

static void push_children(leafvec* v, const or_leaf* p) {
  for (int c = 0; c < 4; ++c) {
    or_leaf k = {p->f, p->b, p->l + 1, 2 * p->x + (c & 1), 2 * p->y + (c >> 1)};
    push(v, k);
  }
}

/* refine (once) every leaf that touches a leaf two or more levels finer, until none */
static void balance(const or_forest* F, leafvec* v) {
  for (;;) {
    char* mark = (char*)calloc((size_t)(v->n > 0 ? v->n : 1), 1);
    int any = 0;
    for (int a = 0; a < v->n; ++a)
      for (int c = 0; c < v->n; ++c) {
        if (a == c) continue;
        if (v->a[c].l >= v->a[a].l + 2 && or_touch(F, &v->a[a], &v->a[c])) {
          mark[a] = 1;
          any = 1;
          break;
        }
      }
    if (!any) {
      free(mark);
      return;
    }
    leafvec w = {0, 0, 0};
    for (int a = 0; a < v->n; ++a) {
      if (mark[a]) push_children(&w, &v->a[a]);
      else push(&w, v->a[a]);
    }
    free(mark);
    free(v->a);
    *v = w;
  }
}

static int is_first_child(const or_leaf* a) { return (a->x % 2 == 0) && (a->y % 2 == 0); }

int or_regrid(or_forest* F, double tau_r, double tau_c, const int* lmax_f, int* changed) {
  int n = F->n, mx = F->P.mx;
  size_t S2 = (size_t)F->S * F->S;
  double* delta = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (or_tag(F, delta)) {
    free(delta);
    return -1;
  }
  char* refine = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
  for (int p = 0; p < n; ++p) {
    int lm = lmax_f ? lmax_f[F->lv[p].f] : F->P.lmax;
    refine[p] = (delta[p] > tau_r) && (F->lv[p].l < lm);
  }
  /* Sec. 3.3 smooth grading: each leaf's target level (one finer if tagged to
     refine, one coarser if below tau_c, else its own) is raised to the
     largest target among the leaves it touches; a leaf refines when its
     graded target is finer than it, and a family coarsens only when every
     sibling's graded target is coarser */
  int* target = NULL;
  if (F->P.smooth) {
    int* t0 = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    target = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    for (int p = 0; p < n; ++p) {
      int l = F->lv[p].l;
      t0[p] = refine[p] ? l + 1 : (delta[p] < tau_c && l > F->P.lmin) ? l - 1 : l;
    }
    for (int p = 0; p < n; ++p) {
      int t = t0[p];
      for (int q = 0; q < n; ++q)
        if (q != p && t0[q] > t && or_touch(F, &F->lv[p], &F->lv[q])) t = t0[q];
      target[p] = t;
    }
    for (int p = 0; p < n; ++p) {
      int lm = lmax_f ? lmax_f[F->lv[p].f] : F->P.lmax;
      refine[p] = target[p] > F->lv[p].l && F->lv[p].l < lm;
    }
    free(t0);
  }
  /* candidate families: four sibling leaves, none tagged to refine, all below
     tau_c (graded: all four with a coarser target) */
  int* fam = (int*)malloc(sizeof(int) * 4 * (size_t)(n > 0 ? n : 1));
  int nfam = 0;
  for (int p = 0; p < n; ++p) {
    const or_leaf* a = &F->lv[p];
    if (a->l <= F->P.lmin || !is_first_child(a)) continue;
    int s[4], ok = 1;
    for (int c = 0; c < 4 && ok; ++c) {
      s[c] = or_find(F, a->f, a->b, a->l, a->x + (c & 1), a->y + (c >> 1));
      if (s[c] < 0 || refine[s[c]]) ok = 0;
      else if (target ? !(target[s[c]] < a->l) : !(delta[s[c]] < tau_c)) ok = 0;
    }
    if (!ok) continue;
    for (int c = 0; c < 4; ++c) fam[4 * nfam + c] = s[c];
    ++nfam;
  }
  /* refine, then balance */
  leafvec v = {0, 0, 0};
  for (int p = 0; p < n; ++p) {
    if (refine[p]) push_children(&v, &F->lv[p]);
    else push(&v, F->lv[p]);
  }
  balance(F, &v);
  /* coarsen families whose parent is balanced against the refined layout */
  char* gone = (char*)calloc((size_t)(v.n > 0 ? v.n : 1), 1);
  leafvec parents = {0, 0, 0};
  for (int k = 0; k < nfam; ++k) {
    const or_leaf* c0 = &F->lv[fam[4 * k]];
    int idx[4], ok = 1;
    for (int c = 0; c < 4; ++c) {
      const or_leaf* s = &F->lv[fam[4 * k + c]];
      idx[c] = -1;
      for (int m = 0; m < v.n; ++m)
        if (v.a[m].f == s->f && v.a[m].b == s->b && v.a[m].l == s->l && v.a[m].x == s->x &&
            v.a[m].y == s->y) {
          idx[c] = m;
          break;
        }
      if (idx[c] < 0) ok = 0; /* a sibling was refined by balance */
    }
    if (!ok) continue;
    or_leaf par = {c0->f, c0->b, c0->l - 1, c0->x / 2, c0->y / 2};
    for (int m = 0; m < v.n && ok; ++m) {
      if (m == idx[0] || m == idx[1] || m == idx[2] || m == idx[3]) continue;
      if (v.a[m].l > par.l + 1 && or_touch(F, &par, &v.a[m])) ok = 0;
    }
    if (!ok) continue;
    for (int c = 0; c < 4; ++c) gone[idx[c]] = 1;
    push(&parents, par);
  }
  leafvec nw = {0, 0, 0};
  for (int m = 0; m < v.n; ++m)
    if (!gone[m]) push(&nw, v.a[m]);
  for (int k = 0; k < parents.n; ++k) push(&nw, parents.a[k]);
  or_sort_leaves(nw.a, nw.n);

  /* remap data onto the new layout */
  double* q2 = (double*)malloc(sizeof(double) * S2 * (size_t)(nw.n > 0 ? nw.n : 1));
  for (size_t c = 0; c < S2 * (size_t)nw.n; ++c) q2[c] = NAN;
  int status = 0, nchanged = 0;
  for (int m = 0; m < nw.n && status == 0; ++m) {
    const or_leaf* a = &nw.a[m];
    double* D = q2 + m * S2;
    int old = or_find(F, a->f, a->b, a->l, a->x, a->y);
    if (old >= 0) {
      for (int j = 0; j < mx; ++j)
        for (int i = 0; i < mx; ++i) D[OR_IDX(F, i, j)] = F->q[old * S2 + OR_IDX(F, i, j)];
      continue;
    }
    ++nchanged;
    int par = (a->l > 0) ? or_find(F, a->f, a->b, a->l - 1, a->x / 2, a->y / 2) : -1;
    if (par >= 0) {
      const double* Q = F->q + par * S2;
      int cx = a->x & 1, cy = a->y & 1;
      for (int j = 0; j < mx; ++j)
        for (int i = 0; i < mx; ++i) {
          int ic = cx * mx / 2 + i / 2, jc = cy * mx / 2 + j / 2;
          double dx = (i & 1) ? 1.0 : -1.0, dy = (j & 1) ? 1.0 : -1.0;
          double q0 = Q[OR_IDX(F, ic, jc)];
          double sx = or_minmod(Q[OR_IDX(F, ic + 1, jc)] - q0, q0 - Q[OR_IDX(F, ic - 1, jc)]);
          double sy = or_minmod(Q[OR_IDX(F, ic, jc + 1)] - q0, q0 - Q[OR_IDX(F, ic, jc - 1)]);
          D[OR_IDX(F, i, j)] = q0 + 0.25 * (sx * dx + sy * dy);
        }
      continue;
    }
    int ch[4], ok = 1;
    for (int c = 0; c < 4; ++c) {
      ch[c] = or_find(F, a->f, a->b, a->l + 1, 2 * a->x + (c & 1), 2 * a->y + (c >> 1));
      if (ch[c] < 0) ok = 0;
    }
    if (!ok) {
      or_set_error("regrid: new leaf (%d,%d,%d,%d,%d) has neither an old parent nor four old "
                   "children", a->f, a->b, a->l, a->x, a->y);
      status = -1;
      break;
    }
    for (int j = 0; j < mx; ++j)
      for (int i = 0; i < mx; ++i) {
        int cx = (2 * i >= mx), cy = (2 * j >= mx);
        const double* C = F->q + ch[cx + 2 * cy] * S2;
        int fi = 2 * i - cx * mx, fj = 2 * j - cy * mx;
        double a0 = C[OR_IDX(F, fi, fj)], a1 = C[OR_IDX(F, fi + 1, fj)];
        double a2 = C[OR_IDX(F, fi, fj + 1)], a3 = C[OR_IDX(F, fi + 1, fj + 1)];
        if (F->P.domain == OR_SPHERE) { /* area-weighted, as the ghost average */
          const double* K = F->kappa + ch[cx + 2 * cy] * S2;
          double k0 = K[OR_IDX(F, fi, fj)], k1 = K[OR_IDX(F, fi + 1, fj)];
          double k2 = K[OR_IDX(F, fi, fj + 1)], k3 = K[OR_IDX(F, fi + 1, fj + 1)];
          D[OR_IDX(F, i, j)] =
              (((k0 * a0 + k1 * a1) + k2 * a2) + k3 * a3) / (((k0 + k1) + k2) + k3);
        } else {
          D[OR_IDX(F, i, j)] = 0.25 * (((a0 + a1) + a2) + a3);
        }
      }
  }
  if (status == 0) {
    /* new leaves plus the old leaves that disappeared */
    nchanged += n - (nw.n - nchanged);
    free(F->lv);
    F->lv = nw.a;
    F->n = nw.n;
    free(F->q);
    F->q = q2;
    free(F->qold);
    free(F->qT);
    F->qold = (double*)malloc(sizeof(double) * S2 * (size_t)(nw.n > 0 ? nw.n : 1));
    F->qT = (double*)malloc(sizeof(double) * S2 * (size_t)(nw.n > 0 ? nw.n : 1));
    for (size_t c = 0; c < S2 * (size_t)nw.n; ++c) F->qold[c] = F->qT[c] = NAN;
    or_build_index(F);
    or_drop_cache(F);
    or_update_metrics(F);
    if (changed) *changed = nchanged;
  } else {
    free(nw.a);
    free(q2);
  }
  free(v.a);
  free(parents.a);
  free(gone);
  free(fam);
  free(refine);
  free(target);
  free(delta);
  return status;
}

void or_mass(const or_forest* F, double* per_forest) {
  size_t S2 = (size_t)F->S * F->S;
  int mx = F->P.mx;
  for (int f = 0; f < F->P.nforests; ++f) per_forest[f] = 0.0;
  for (int p = 0; p < F->n; ++p) {
    double h = cell_h(F, F->lv[p].l), s = 0.0;
    if (F->P.domain == OR_SPHERE) { /* capacity-weighted: sum kappa q */
      for (int j = 0; j < mx; ++j)
        for (int i = 0; i < mx; ++i)
          s += F->kappa[p * S2 + OR_IDX(F, i, j)] * F->q[p * S2 + OR_IDX(F, i, j)];
      per_forest[F->lv[p].f] += s;
      continue;
    }
    for (int j = 0; j < mx; ++j)
      for (int i = 0; i < mx; ++i) s += F->q[p * S2 + OR_IDX(F, i, j)];
    per_forest[F->lv[p].f] += h * h * s;
  }
}

int or_single_grid_periodic(const or_params* P, int N, double* q, double t0, double dt,
                            int nsteps) {
  int mbc = P->mbc, S = N + 2 * mbc;
  double* a = (double*)malloc(sizeof(double) * (size_t)S * S);
  double h = 1.0 / N;
  for (int n = 0; n < nsteps; ++n) {
    for (int j = -mbc; j < N + mbc; ++j)
      for (int i = -mbc; i < N + mbc; ++i) {
        int ii = ((i % N) + N) % N, jj = ((j % N) + N) % N;
        a[(i + mbc) + S * (j + mbc)] = q[ii + N * jj];
      }
    or_claw_step(P, a, N, mbc, h, dt, t0 + n * dt, 0, 0);
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N; ++i) q[i + N * j] = a[(i + mbc) + S * (j + mbc)];
  }
  free(a);
  return 0;
}
