/*
 * Oracle: reverse-mode adjoint of global time stepping.
 * Test infrastructure only (see oracle.h).
 *
 * The forward map of one step is q^{n+1} = S(Fill(q^n)): Alg. 1 fills every
 * ghost cell, then every patch takes the wave-propagation step.  Both maps are
 * piecewise linear in q (the MC limiter and the minmod slopes of the ghost
 * interpolation choose a linear piece), so the adjoint applies the transpose
 * of each elementary operation, in reverse order, with the pieces chosen by
 * the forward state (the a.e. derivative).  The velocity-scale derivative
 * sums, over every use of an edge speed s_e = sigma u_e, dL/ds_e * u_e.
 */
#include "internal.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* piece of the MC-limited wave lim(W, Wup) = phi(Wup/W) W, in the order the
 * forward evaluates phi: dW, dWup are the partial derivatives on that piece */
static void mc_piece(double W, double Wup, double* dW, double* dWup) {
  *dW = *dWup = 0.0;
  if (W == 0.0) return;
  double th = Wup / W;
  double a = 0.5 * (1.0 + th);
  int piece = 0; /* 0: (1+th)/2, 1: 2, 2: 2 th */
  double m = a;
  if (!(a < 2.0)) {
    m = 2.0;
    piece = 1;
  }
  if (!(m < 2.0 * th)) {
    m = 2.0 * th;
    piece = 2;
  }
  if (!(m > 0.0)) return;
  if (piece == 0) {
    *dW = 0.5;
    *dWup = 0.5;
  } else if (piece == 1) {
    *dW = 2.0;
  } else {
    *dWup = 2.0;
  }
}

typedef struct {
  double s, W, Wup, lim, dW, dWup, c, dc, Ft, Pf, Mf;
  int up; /* 1: upwind cell behind (s >= 0) */
} edgefw;

/* forward quantities of one edge (cells a,b behind / c,d ahead as in claw.c) */
static edgefw edge_forward(const or_params* P, double s, double qa, double qb, double qc,
                           double qd, double nu) {
  edgefw e;
  e.s = s;
  e.W = qc - qb;
  e.up = s >= 0.0;
  e.Wup = e.up ? qb - qa : qd - qc;
  e.lim = e.W;
  e.dW = 1.0;
  e.dWup = 0.0;
  if (P->limiter == 1) {
    e.lim = (e.W == 0.0) ? 0.0 : or_mc_phi(e.Wup / e.W) * e.W;
    mc_piece(e.W, e.Wup, &e.dW, &e.dWup);
  }
  double as = fabs(s);
  e.c = 0.5 * as * (1.0 - nu * as);
  e.dc = 0.5 * (s > 0.0 ? 1.0 : (s < 0.0 ? -1.0 : 0.0)) * (1.0 - 2.0 * nu * as);
  if (P->order < 2) {
    e.c = 0.0;
    e.dc = 0.0;
  }
  if (P->limiter == 1 && e.W == 0.0) e.Ft = 0.0;
  else e.Ft = e.c * e.lim;
  double sp = s > 0.0 ? s : 0.0, sm = s < 0.0 ? s : 0.0;
  e.Pf = sp * e.W;
  e.Mf = sm * e.W;
  if (P->transverse > 1) {
    e.Pf -= e.Ft;
    e.Mf += e.Ft;
  }
  return e;
}

/* Adjoint of one edge given the adjoints of its outputs (normal flux lF,
 * fluctuations lP, lM): adds to the four cell adjoints, returns dL/ds_e for
 * the edge's own speed. */
static double edge_reverse(const or_params* P, const edgefw* e, double qb, double qc, double lF,
                           double lP, double lM, double* la, double* lb, double* lc,
                           double* ld) {
  double sp = e->s > 0.0 ? e->s : 0.0, sm = e->s < 0.0 ? e->s : 0.0;
  double ip = e->s > 0.0 ? 1.0 : 0.0, im = e->s < 0.0 ? 1.0 : 0.0;
  double lFt = lF, lW = 0.0, lWup = 0.0, ds = 0.0;
  if (P->transverse > 0) {
    lW += sp * lP + sm * lM;
    ds += lP * ip * e->W + lM * im * e->W;
    if (P->transverse > 1) lFt += -lP + lM;
  }
  /* F = sp qb + sm qc + Ft */
  *lb += sp * lF;
  *lc += sm * lF;
  ds += lF * (ip * qb + im * qc);
  /* Ft = c(s) lim(W, Wup) */
  if (!(P->limiter == 1 && e->W == 0.0)) {
    lW += e->c * e->dW * lFt;
    lWup += e->c * e->dWup * lFt;
    ds += lFt * e->dc * e->lim;
  }
  /* W = qc - qb */
  *lc += lW;
  *lb -= lW;
  /* Wup */
  if (e->up) {
    *lb += lWup;
    *la -= lWup;
  } else {
    *ld += lWup;
    *lc -= lWup;
  }
  return ds;
}

/* Adjoint of or_claw_step for one patch.  q: the forward input (with
 * ghosts); lnew: adjoint of the new interior (mx x mx, [j][i]); lq: adjoint
 * of the input array (S x S), accumulated.  Returns sum_e dL/ds_e * s_e. */
static double claw_step_adjoint(const or_params* P, const double* q, int mx, int mbc, double h,
                                double dt, double t, long gx0, long gy0, const double* lnew,
                                double* lq) {
  int S = mx + 2 * mbc, SE = S + 1;
  double nu = dt / h, th = t + 0.5 * dt, sum = 0.0;
  double* lF = (double*)calloc((size_t)SE * SE, sizeof(double));
  double* lG = (double*)calloc((size_t)SE * SE, sizeof(double));
#define Q(i, j) q[((i) + mbc) + S * ((j) + mbc)]
#define LQ(i, j) lq[((i) + mbc) + S * ((j) + mbc)]
#define LF(i, j) lF[((i) + mbc) + SE * ((j) + mbc)]
#define LG(i, j) lG[((i) + mbc) + SE * ((j) + mbc)]
#define U(i, j) or_u_edge(P, h, th, gx0, gy0, i, j)
#define V(i, j) or_v_edge(P, h, th, gx0, gy0, i, j)
  /* update: Q(i,j) - nu (F(i+1,j) - F(i,j)) - nu (G(i,j+1) - G(i,j)) */
  for (int j = 0; j < mx; ++j)
    for (int i = 0; i < mx; ++i) {
      double l = lnew[j * mx + i];
      LQ(i, j) += l;
      LF(i + 1, j) -= nu * l;
      LF(i, j) += nu * l;
      LG(i, j + 1) -= nu * l;
      LG(i, j) += nu * l;
    }
  /* y-sweep, reversed */
  for (int i = mx; i >= -1; --i)
    for (int j = mx; j >= 0; --j) {
      edgefw e = edge_forward(P, V(i, j), Q(i, j - 2), Q(i, j - 1), Q(i, j), Q(i, j + 1), nu);
      double lP = 0.0, lM = 0.0;
      if (P->transverse > 0) {
        double u1 = U(i + 1, j), u0 = U(i, j), u3 = U(i + 1, j - 1), u2 = U(i, j - 1);
        double c1 = -0.5 * nu * (u1 > 0 ? u1 : 0), c0 = -0.5 * nu * (u0 < 0 ? u0 : 0);
        double c3 = -0.5 * nu * (u3 > 0 ? u3 : 0), c2 = -0.5 * nu * (u2 < 0 ? u2 : 0);
        lP = c1 * LF(i + 1, j) + c0 * LF(i, j);
        lM = c3 * LF(i + 1, j - 1) + c2 * LF(i, j - 1);
        /* the transverse coefficients use other edges' speeds */
        sum += c1 * LF(i + 1, j) * e.Pf + c0 * LF(i, j) * e.Pf + c3 * LF(i + 1, j - 1) * e.Mf +
               c2 * LF(i, j - 1) * e.Mf;
      }
      double la = 0, lb = 0, lc = 0, ld = 0;
      double ds = edge_reverse(P, &e, Q(i, j - 1), Q(i, j), LG(i, j), lP, lM, &la, &lb, &lc, &ld);
      sum += ds * e.s;
      LQ(i, j - 2) += la;
      LQ(i, j - 1) += lb;
      LQ(i, j) += lc;
      LQ(i, j + 1) += ld;
    }
  /* x-sweep, reversed */
  for (int j = mx; j >= -1; --j)
    for (int i = mx; i >= 0; --i) {
      edgefw e = edge_forward(P, U(i, j), Q(i - 2, j), Q(i - 1, j), Q(i, j), Q(i + 1, j), nu);
      double lP = 0.0, lM = 0.0;
      if (P->transverse > 0) {
        double v1 = V(i, j + 1), v0 = V(i, j), v3 = V(i - 1, j + 1), v2 = V(i - 1, j);
        double c1 = -0.5 * nu * (v1 > 0 ? v1 : 0), c0 = -0.5 * nu * (v0 < 0 ? v0 : 0);
        double c3 = -0.5 * nu * (v3 > 0 ? v3 : 0), c2 = -0.5 * nu * (v2 < 0 ? v2 : 0);
        lP = c1 * LG(i, j + 1) + c0 * LG(i, j);
        lM = c3 * LG(i - 1, j + 1) + c2 * LG(i - 1, j);
        sum += c1 * LG(i, j + 1) * e.Pf + c0 * LG(i, j) * e.Pf + c3 * LG(i - 1, j + 1) * e.Mf +
               c2 * LG(i - 1, j) * e.Mf;
      }
      double la = 0, lb = 0, lc = 0, ld = 0;
      double ds = edge_reverse(P, &e, Q(i - 1, j), Q(i, j), LF(i, j), lP, lM, &la, &lb, &lc, &ld);
      sum += ds * e.s;
      LQ(i - 2, j) += la;
      LQ(i - 1, j) += lb;
      LQ(i, j) += lc;
      LQ(i + 1, j) += ld;
    }
#undef Q
#undef LQ
#undef LF
#undef LG
#undef U
#undef V
  free(lF);
  free(lG);
  return sum;
}

static int is_ghost_cell(const or_forest* F, int i, int j) {
  return i < 0 || j < 0 || i >= F->P.mx || j >= F->P.mx;
}

/* transpose of the wall boundary condition for leaf p (see apply_bc) */
static void bc_reverse(const or_forest* F, int p, double* L) {
  if (F->P.domain != OR_WALLS) return;
  const or_leaf* a = &F->lv[p];
  int mx = F->P.mx, mbc = F->P.mbc, nb = 1 << a->l;
  for (int j = -mbc; j < mx + mbc; ++j)
    for (int i = -mbc; i < mx + mbc; ++i) {
      if (!is_ghost_cell(F, i, j)) continue;
      int gi = a->x * mx + i, gj = a->y * mx + j;
      int outx = gi < 0 || gi >= nb * mx, outy = gj < 0 || gj >= nb * mx;
      if (!outx && !outy) continue;
      int ic = i, jc = j;
      if (outx) ic = (gi < 0) ? 0 : mx - 1;
      if (outy) jc = (gj < 0) ? 0 : mx - 1;
      L[OR_IDX(F, ic, jc)] += L[OR_IDX(F, i, j)];
      L[OR_IDX(F, i, j)] = 0.0;
    }
}

static int cell_index(const or_forest* F, int n, double x, double y) {
  const or_leaf* c = &F->lv[n];
  int mx = F->P.mx;
  double s = ldexp((double)mx, c->l);
  int i = (int)floor(x * s) - c->x * mx;
  int j = (int)floor(y * s) - c->y * mx;
  return OR_IDX(F, i, j);
}

static void minmod_grad(double a, double b, double* da, double* db) {
  *da = *db = 0.0;
  if (a * b <= 0.0) return;
  if (fabs(a) < fabs(b)) *da = 1.0;
  else *db = 1.0;
}

/* transpose of Alg. 1 (or_fill_all).  L: adjoint of every leaf array with
 * ghosts; snap: the forward state after phase 2.  On return the adjoint of
 * every ghost cell is zero and the interiors hold the adjoint of q. */
static void fill_reverse(or_forest* F, double* L, const double* snap) {
  size_t S2 = (size_t)F->S * F->S;
  int mx = F->P.mx, mbc = F->P.mbc;
  /* phase 4 */
  for (int p = 0; p < F->n; ++p) bc_reverse(F, p, L + p * S2);
  /* phase 3: interpolation from the snapshot of the coarse leaf */
  for (int p = 0; p < F->n; ++p) {
    int k = 0;
    for (int j = -mbc; j < mx + mbc; ++j)
      for (int i = -mbc; i < mx + mbc; ++i) {
        if (!is_ghost_cell(F, i, j)) continue;
        int rel, n;
        double x, y;
        or_ghost_holder(F, p, k++, &rel, &n, &x, &y);
        if (rel != REL_COARSE) continue;
        double lg = L[p * S2 + OR_IDX(F, i, j)];
        L[p * S2 + OR_IDX(F, i, j)] = 0.0;
        const or_leaf* c = &F->lv[n];
        double s = ldexp((double)mx, c->l);
        int ic = (int)floor(x * s) - c->x * mx, jc = (int)floor(y * s) - c->y * mx;
        double xc = ((double)c->x * mx + ic + 0.5) / s, yc = ((double)c->y * mx + jc + 0.5) / s;
        double dx = (x > xc) ? 1.0 : -1.0, dy = (y > yc) ? 1.0 : -1.0;
        const double* Qn = snap + n * S2;
        double* Ln = L + n * S2;
        double q0 = Qn[OR_IDX(F, ic, jc)];
        double ax = Qn[OR_IDX(F, ic + 1, jc)] - q0, bx = q0 - Qn[OR_IDX(F, ic - 1, jc)];
        double ay = Qn[OR_IDX(F, ic, jc + 1)] - q0, by = q0 - Qn[OR_IDX(F, ic, jc - 1)];
        double dax, dbx, day, dby;
        minmod_grad(ax, bx, &dax, &dbx);
        minmod_grad(ay, by, &day, &dby);
        double lsx = 0.25 * dx * lg, lsy = 0.25 * dy * lg;
        Ln[OR_IDX(F, ic, jc)] += lg + lsx * (dbx - dax) + lsy * (dby - day);
        Ln[OR_IDX(F, ic + 1, jc)] += lsx * dax;
        Ln[OR_IDX(F, ic - 1, jc)] -= lsx * dbx;
        Ln[OR_IDX(F, ic, jc + 1)] += lsy * day;
        Ln[OR_IDX(F, ic, jc - 1)] -= lsy * dby;
      }
  }
  /* phase 2 */
  for (int p = 0; p < F->n; ++p) bc_reverse(F, p, L + p * S2);
  /* phase 1: copy and average */
  for (int p = 0; p < F->n; ++p) {
    int k = 0;
    for (int j = -mbc; j < mx + mbc; ++j)
      for (int i = -mbc; i < mx + mbc; ++i) {
        if (!is_ghost_cell(F, i, j)) continue;
        int rel, n;
        double x, y;
        or_ghost_holder(F, p, k++, &rel, &n, &x, &y);
        double lg = L[p * S2 + OR_IDX(F, i, j)];
        if (rel == REL_SAME) {
          L[n * S2 + cell_index(F, n, x, y)] += lg;
        } else if (rel == REL_FINE) {
          double hf = 1.0 / ldexp((double)mx, F->lv[n].l);
          for (int q = 0; q < 4; ++q) {
            double ox = (q & 1) ? 0.5 * hf : -0.5 * hf, oy = (q & 2) ? 0.5 * hf : -0.5 * hf;
            L[n * S2 + cell_index(F, n, x + ox, y + oy)] += 0.25 * lg;
          }
        } else {
          continue;
        }
        L[p * S2 + OR_IDX(F, i, j)] = 0.0;
      }
  }
}

static double scale_of(const or_params* P) { return P->vel_scale != 0.0 ? P->vel_scale : 1.0; }

int or_adjoint_step_global(or_forest* F, double t, double dt, double* lam, double* dscale) {
  if (F->P.reflux) {
    or_set_error("the adjoint is stated without refluxing");
    return -1;
  }
  size_t S2 = (size_t)F->S * F->S;
  int mx = F->P.mx;
  double* snap = (double*)malloc(sizeof(double) * S2 * (size_t)(F->n > 0 ? F->n : 1));
  if (or_fill_all_snapshot(F, snap)) {
    free(snap);
    return -1;
  }
  double* L = (double*)calloc(S2 * (size_t)(F->n > 0 ? F->n : 1), sizeof(double));
  double sum = 0.0;
  for (int p = 0; p < F->n; ++p) {
    const or_leaf* a = &F->lv[p];
    double h = 1.0 / ldexp((double)mx, a->l);
    sum += claw_step_adjoint(&F->P, F->q + p * S2, mx, F->P.mbc, h, dt, t, (long)a->x * mx,
                             (long)a->y * mx, lam + (size_t)p * mx * mx, L + p * S2);
  }
  fill_reverse(F, L, snap);
  for (int p = 0; p < F->n; ++p)
    for (int j = 0; j < mx; ++j)
      for (int i = 0; i < mx; ++i) lam[((size_t)p * mx + j) * mx + i] = L[p * S2 + OR_IDX(F, i, j)];
  *dscale += sum / scale_of(&F->P);
  free(L);
  free(snap);
  return 0;
}

int or_adjoint_global(or_forest* F, int nsteps, double t0, double dt, const double* q_target,
                      double* grad_q0, double* grad_scale, double* loss) {
  int mx = F->P.mx;
  size_t ni = (size_t)F->n * mx * mx;
  double* states = (double*)malloc(sizeof(double) * ni * (size_t)(nsteps > 0 ? nsteps + 1 : 1));
  or_get_q(F, states);
  for (int n = 0; n < nsteps; ++n) {
    if (or_step_global(F, t0 + n * dt, dt)) {
      free(states);
      return -1;
    }
    or_get_q(F, states + (size_t)(n + 1) * ni);
  }
  double* lam = grad_q0;
  double l = 0.0;
  for (size_t k = 0; k < ni; ++k) {
    double d = states[(size_t)nsteps * ni + k] - q_target[k];
    lam[k] = d;
    l += 0.5 * d * d;
  }
  *loss = l;
  *grad_scale = 0.0;
  for (int n = nsteps - 1; n >= 0; --n) {
    or_set_q(F, states + (size_t)n * ni);
    if (or_adjoint_step_global(F, t0 + n * dt, dt, lam, grad_scale)) {
      free(states);
      return -1;
    }
  }
  or_set_q(F, states);
  free(states);
  return 0;
}

/* ------------------------------------------------------------------------
 * Adjoint of multirate stepping (Sec. 4 local time stepping, coarse-first
 * recursion; the reading of the forward is in drive.c).
 *
 * State of the forward: per leaf the current interior q and the interior
 * qold of its level's previous state.  One substep of level L with weight
 * alpha:
 *   qT(c) = (1 - alpha) qold(c) + alpha q(c)     for leaves c of level L-1,
 *   ghosts of L-1 (in qT) and of L (in q) by Alg. 1 restricted to L-1, L,
 *   qold(p) = q(p), q(p) = step(q(p) with ghosts)  for leaves p of level L.
 * Its transpose, with lam (adjoint of q) and mu (adjoint of qold):
 *   lt(p) = step^T lam(p)  (a whole tile with ghosts),
 *   lam(p) = mu(p) + interior of lt(p), mu(p) = 0  (qold(p) was overwritten),
 *   the ghosts of lt and of the qT tiles' adjoint lT, through Alg. 1
 *   backwards: boundary condition of L, interpolation (into lT), boundary
 *   condition of L-1 and L, copy/average (into lT for sources of level L-1,
 *   else into lam),
 *   mu(c) += (1 - alpha) lT(c), lam(c) += alpha lT(c).
 * The substeps are reversed in the opposite order of the recursion; each is
 * replayed from the stored state before it (test sizes only).
 * ------------------------------------------------------------------------ */

typedef struct {
  int L;
  double t, dt, alpha;
} mr_sub;

static int mr_list(const or_forest* F, int L, double t, double dt, double alpha, mr_sub* out,
                   int k) {
  out[k].L = L;
  out[k].t = t;
  out[k].dt = dt;
  out[k].alpha = alpha;
  ++k;
  if (L < F->P.lmax) {
    k = mr_list(F, L + 1, t, 0.5 * dt, 0.0, out, k);
    k = mr_list(F, L + 1, t + 0.5 * dt, 0.5 * dt, 0.5, out, k);
  }
  return k;
}

/* transpose of or_fill_level(F, L, alpha) for the ghosts of level L (in Lq)
 * and of level L-1 (in LT); qT holds the forward's time-interpolated tiles */
static void fill_level_reverse(or_forest* F, int L, double* Lq, double* LT) {
  size_t S2 = (size_t)F->S * F->S;
  int mx = F->P.mx, mbc = F->P.mbc;
  /* phase 4: boundary condition of level L */
  for (int p = 0; p < F->n; ++p)
    if (F->lv[p].l == L) bc_reverse(F, p, Lq + p * S2);
  /* phase 3: interpolation of level L's coarse ghosts from qT */
  for (int p = 0; p < F->n; ++p) {
    if (F->lv[p].l != L) continue;
    int k = 0;
    for (int j = -mbc; j < mx + mbc; ++j)
      for (int i = -mbc; i < mx + mbc; ++i) {
        if (!is_ghost_cell(F, i, j)) continue;
        int rel, n;
        double x, y;
        or_ghost_holder(F, p, k++, &rel, &n, &x, &y);
        if (rel != REL_COARSE) continue;
        double lg = Lq[p * S2 + OR_IDX(F, i, j)];
        Lq[p * S2 + OR_IDX(F, i, j)] = 0.0;
        const or_leaf* c = &F->lv[n];
        double s = ldexp((double)mx, c->l);
        int ic = (int)floor(x * s) - c->x * mx, jc = (int)floor(y * s) - c->y * mx;
        double xc = ((double)c->x * mx + ic + 0.5) / s, yc = ((double)c->y * mx + jc + 0.5) / s;
        double dx = (x > xc) ? 1.0 : -1.0, dy = (y > yc) ? 1.0 : -1.0;
        const double* Qn = F->qT + n * S2;
        double* Ln = LT + n * S2;
        double q0 = Qn[OR_IDX(F, ic, jc)];
        double ax = Qn[OR_IDX(F, ic + 1, jc)] - q0, bx = q0 - Qn[OR_IDX(F, ic - 1, jc)];
        double ay = Qn[OR_IDX(F, ic, jc + 1)] - q0, by = q0 - Qn[OR_IDX(F, ic, jc - 1)];
        double dax, dbx, day, dby;
        minmod_grad(ax, bx, &dax, &dbx);
        minmod_grad(ay, by, &day, &dby);
        double lsx = 0.25 * dx * lg, lsy = 0.25 * dy * lg;
        Ln[OR_IDX(F, ic, jc)] += lg + lsx * (dbx - dax) + lsy * (dby - day);
        Ln[OR_IDX(F, ic + 1, jc)] += lsx * dax;
        Ln[OR_IDX(F, ic - 1, jc)] -= lsx * dbx;
        Ln[OR_IDX(F, ic, jc + 1)] += lsy * day;
        Ln[OR_IDX(F, ic, jc - 1)] -= lsy * dby;
      }
  }
  /* phase 2: boundary condition of levels L-1 (qT) and L */
  for (int p = 0; p < F->n; ++p) {
    if (F->lv[p].l == L) bc_reverse(F, p, Lq + p * S2);
    if (F->lv[p].l == L - 1) bc_reverse(F, p, LT + p * S2);
  }
  /* phase 1: copy and average into the ghosts of levels L-1 and L */
  for (int p = 0; p < F->n; ++p) {
    int lp = F->lv[p].l;
    if (lp != L && lp != L - 1) continue;
    double* Lp = (lp == L ? Lq : LT) + p * S2;
    int k = 0;
    for (int j = -mbc; j < mx + mbc; ++j)
      for (int i = -mbc; i < mx + mbc; ++i) {
        if (!is_ghost_cell(F, i, j)) continue;
        int rel, n;
        double x, y;
        or_ghost_holder(F, p, k++, &rel, &n, &x, &y);
        if (rel != REL_SAME && rel != REL_FINE) continue;
        double lg = Lp[OR_IDX(F, i, j)];
        Lp[OR_IDX(F, i, j)] = 0.0;
        double* Ln = (F->lv[n].l == L - 1 ? LT : Lq) + n * S2;
        if (rel == REL_SAME) {
          Ln[cell_index(F, n, x, y)] += lg;
        } else {
          double hf = 1.0 / ldexp((double)mx, F->lv[n].l);
          for (int q = 0; q < 4; ++q) {
            double ox = (q & 1) ? 0.5 * hf : -0.5 * hf, oy = (q & 2) ? 0.5 * hf : -0.5 * hf;
            Ln[cell_index(F, n, x + ox, y + oy)] += 0.25 * lg;
          }
        }
      }
  }
}

int or_adjoint_step_multirate(or_forest* F, double t, double dt_coarse, double* lam,
                              double* dscale) {
  if (F->P.domain == OR_SPHERE) {
    or_set_error("the adjoint is stated for the square domains");
    return -1;
  }
  if (F->P.reflux) {
    or_set_error("the adjoint is stated without refluxing");
    return -1;
  }
  size_t S2 = (size_t)F->S * F->S, nS = S2 * (size_t)(F->n > 0 ? F->n : 1);
  int mx = F->P.mx, nsub = (1 << (F->P.lmax - F->P.lmin + 1)) - 1;
  mr_sub* sub = (mr_sub*)malloc(sizeof(mr_sub) * (size_t)nsub);
  mr_list(F, F->P.lmin, t, dt_coarse, 0.0, sub, 0);
  /* forward, keeping the state (q, qold) before every substep */
  double* keep = (double*)malloc(sizeof(double) * nS * 2 * (size_t)nsub);
  int status = 0;
  for (int k = 0; k < nsub && status == 0; ++k) {
    memcpy(keep + 2 * k * nS, F->q, sizeof(double) * nS);
    memcpy(keep + (2 * k + 1) * nS, F->qold, sizeof(double) * nS);
    const mr_sub* s = &sub[k];
    if (or_fill_level(F, s->L, s->alpha)) status = -1;
    for (int p = 0; p < F->n && status == 0; ++p)
      if (F->lv[p].l == s->L) {
        memcpy(F->qold + p * S2, F->q + p * S2, sizeof(double) * S2);
        or_advance_leaf(F, p, s->t, s->dt);
      }
  }
  double* Lq = (double*)calloc(nS, sizeof(double));  /* adjoint of q (tiles) */
  double* Lo = (double*)calloc(nS, sizeof(double));  /* adjoint of qold */
  double* LT = (double*)calloc(nS, sizeof(double));  /* adjoint of qT */
  double* lnew = (double*)malloc(sizeof(double) * (size_t)mx * mx);
  for (int p = 0; p < F->n; ++p)
    for (int j = 0; j < mx; ++j)
      for (int i = 0; i < mx; ++i)
        Lq[p * S2 + OR_IDX(F, i, j)] = lam[((size_t)p * mx + j) * mx + i];
  double sum = 0.0;
  for (int k = nsub - 1; k >= 0 && status == 0; --k) {
    const mr_sub* s = &sub[k];
    memcpy(F->q, keep + 2 * k * nS, sizeof(double) * nS);
    memcpy(F->qold, keep + (2 * k + 1) * nS, sizeof(double) * nS);
    if (or_fill_level(F, s->L, s->alpha)) {
      status = -1;
      break;
    }
    memset(LT, 0, sizeof(double) * nS);
    for (int p = 0; p < F->n; ++p) {
      const or_leaf* a = &F->lv[p];
      if (a->l != s->L) continue;
      double* Lp = Lq + p * S2;
      for (int j = 0; j < mx; ++j)
        for (int i = 0; i < mx; ++i) {
          lnew[j * mx + i] = Lp[OR_IDX(F, i, j)];
          Lp[OR_IDX(F, i, j)] = 0.0;
        }
      double h = 1.0 / ldexp((double)mx, a->l);
      sum += claw_step_adjoint(&F->P, F->q + p * S2, mx, F->P.mbc, h, s->dt, s->t,
                               (long)a->x * mx, (long)a->y * mx, lnew, Lp);
      for (int j = 0; j < mx; ++j)
        for (int i = 0; i < mx; ++i) {
          Lp[OR_IDX(F, i, j)] += Lo[p * S2 + OR_IDX(F, i, j)];
          Lo[p * S2 + OR_IDX(F, i, j)] = 0.0;
        }
    }
    fill_level_reverse(F, s->L, Lq, LT);
    for (int p = 0; p < F->n; ++p)
      if (F->lv[p].l == s->L - 1)
        for (int j = 0; j < mx; ++j)
          for (int i = 0; i < mx; ++i) {
            double g = LT[p * S2 + OR_IDX(F, i, j)];
            Lo[p * S2 + OR_IDX(F, i, j)] += (1.0 - s->alpha) * g;
            Lq[p * S2 + OR_IDX(F, i, j)] += s->alpha * g;
          }
  }
  /* the state is left at the start of the coarse step */
  if (status == 0) {
    memcpy(F->q, keep, sizeof(double) * nS);
    memcpy(F->qold, keep + nS, sizeof(double) * nS);
    for (int p = 0; p < F->n; ++p)
      for (int j = 0; j < mx; ++j)
        for (int i = 0; i < mx; ++i)
          lam[((size_t)p * mx + j) * mx + i] = Lq[p * S2 + OR_IDX(F, i, j)];
    *dscale += sum / scale_of(&F->P);
  }
  free(lnew);
  free(LT);
  free(Lo);
  free(Lq);
  free(keep);
  free(sub);
  return status;
}

int or_adjoint_multirate(or_forest* F, int ncoarse, double t0, double dt_coarse,
                         const double* q_target, double* grad_q0, double* grad_scale,
                         double* loss) {
  int mx = F->P.mx;
  size_t ni = (size_t)F->n * mx * mx;
  double* states = (double*)malloc(sizeof(double) * ni * (size_t)(ncoarse + 1));
  or_get_q(F, states);
  for (int n = 0; n < ncoarse; ++n) {
    if (or_step_multirate(F, t0 + n * dt_coarse, dt_coarse)) {
      free(states);
      return -1;
    }
    or_get_q(F, states + (size_t)(n + 1) * ni);
  }
  double l = 0.0;
  for (size_t k = 0; k < ni; ++k) {
    double d = states[(size_t)ncoarse * ni + k] - q_target[k];
    grad_q0[k] = d;
    l += 0.5 * d * d;
  }
  *loss = l;
  *grad_scale = 0.0;
  for (int n = ncoarse - 1; n >= 0; --n) {
    or_set_q(F, states + (size_t)n * ni);
    if (or_adjoint_step_multirate(F, t0 + n * dt_coarse, dt_coarse, grad_q0, grad_scale)) {
      free(states);
      return -1;
    }
  }
  or_set_q(F, states);
  free(states);
  return 0;
}
