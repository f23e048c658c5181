/*
 * Oracle: the cubed-sphere multiblock domain (Sec. 2.4 "Multiblock indexing",
 * Sec. 5.3 advection on a sphere).  Test infrastructure only (see oracle.h).
 *
 * Six blocks are the faces of the cube [-1,1]^3.  Face b has a corner O_b and
 * edge vectors E1_b, E2_b of length 2: block point (x, y) in [0,1]^2 sits at
 * O_b + x E1_b + y E2_b.  The block coordinates carry the equiangular
 * gnomonic grid: angle (x - 1/2) pi/2 along each axis, projected from the
 * cube face onto the unit sphere.
 *
 * Locating a point outside a block (one coordinate out) folds it across the
 * cube edge in index space (Sec. 2.4): the overshoot normal to the edge
 * becomes depth into the adjacent face and the coordinate along the edge is
 * carried over, so cell rows normal to the edge continue into the next face.
 * A point outside in both coordinates lies beyond a cube vertex, where only
 * three blocks meet: it has no holder (REL_CORNER3).
 *
 * Reading for the metric terms (the paper relies on Clawpack's mapped-grid
 * solvers, Sec. 5.3): cell capacity kappa = spherical area of the mapped
 * cell (two spherical triangles); edge volume flux of the solid-body
 * rotation u = omega x X = psi difference with psi = -omega . X, i.e. across an
 * x-edge from corner a (below) to b (above): omega . (X_b - X_a), across a
 * y-edge from corner a (left) to b (right): omega . (X_a - X_b).  Ghost cells
 * use the owner's own mapping evaluated at their (extended) block
 * coordinates.
 */
#include "internal.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static const double kO[6][3] = {{-1, -1, 1}, {-1, 1, -1}, {1, -1, -1},
                                {-1, 1, -1}, {1, 1, -1},  {-1, -1, -1}};
static const double kE1[6][3] = {{2, 0, 0}, {2, 0, 0}, {0, 2, 0},
                                 {0, -2, 0}, {-2, 0, 0}, {2, 0, 0}};
static const double kE2[6][3] = {{0, 2, 0}, {0, -2, 0}, {0, 0, 2},
                                 {0, 0, 2}, {0, 0, 2},  {0, 0, 2}};

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void normal_of(int b, double n[3]) {
  /* outward unit normal: E1 x E2 / |E1 x E2| */
  const double* a = kE1[b];
  const double* c = kE2[b];
  double x[3] = {a[1] * c[2] - a[2] * c[1], a[2] * c[0] - a[0] * c[2], a[0] * c[1] - a[1] * c[0]};
  double l = sqrt(dot3(x, x));
  for (int k = 0; k < 3; ++k) n[k] = x[k] / l;
}

int or_sphere_fold(int* b, double* x, double* y) {
  int outx = (*x < 0.0 || *x >= 1.0), outy = (*y < 0.0 || *y >= 1.0);
  if (outx && outy) return -3;
  if (!outx && !outy) return 0;
  int B = *b;
  double xe = *x, ye = *y, depth, dir[3];
  if (outx) {
    xe = *x < 0.0 ? 0.0 : 1.0;
    depth = *x < 0.0 ? -*x : *x - 1.0;
    for (int k = 0; k < 3; ++k) dir[k] = (*x < 0.0 ? -1.0 : 1.0) * kE1[B][k] / 2.0;
  } else {
    ye = *y < 0.0 ? 0.0 : 1.0;
    depth = *y < 0.0 ? -*y : *y - 1.0;
    for (int k = 0; k < 3; ++k) dir[k] = (*y < 0.0 ? -1.0 : 1.0) * kE2[B][k] / 2.0;
  }
  double n[3], P[3];
  normal_of(B, n);
  for (int k = 0; k < 3; ++k)
    P[k] = kO[B][k] + xe * kE1[B][k] + ye * kE2[B][k] - n[k] * 2.0 * depth;
  /* the adjacent face is the one whose outward normal is dir */
  for (int c = 0; c < 6; ++c) {
    double m[3];
    normal_of(c, m);
    if (dot3(m, dir) > 0.5) {
      double d[3] = {P[0] - kO[c][0], P[1] - kO[c][1], P[2] - kO[c][2]};
      *b = c;
      *x = dot3(d, kE1[c]) / 4.0;
      *y = dot3(d, kE2[c]) / 4.0;
      return 0;
    }
  }
  return -4;
}

/* closed 3D box of a leaf on the cube surface, in units of 2^-LF of the
 * half-edge (integers) */
void or_sphere_box(const or_leaf* a, int LF, long lo[3], long hi[3]) {
  long R = 1L << LF;
  long sx0 = (long)a->x << (LF - a->l), sx1 = (long)(a->x + 1) << (LF - a->l);
  long sy0 = (long)a->y << (LF - a->l), sy1 = (long)(a->y + 1) << (LF - a->l);
  for (int k = 0; k < 3; ++k) {
    long o = (long)kO[a->b][k] * R, e1 = (long)kE1[a->b][k] / 2, e2 = (long)kE2[a->b][k] / 2;
    /* point = O + (x/R) E1 + (y/R) E2, E = 2 e  ->  in units of 1/R: O R + 2 e x */
    long v0 = o + 2 * e1 * sx0 + 2 * e2 * sy0, v1 = o + 2 * e1 * sx1 + 2 * e2 * sy1;
    long v2 = o + 2 * e1 * sx0 + 2 * e2 * sy1, v3 = o + 2 * e1 * sx1 + 2 * e2 * sy0;
    long mn = v0, mx = v0;
    if (v1 < mn) mn = v1;
    if (v2 < mn) mn = v2;
    if (v3 < mn) mn = v3;
    if (v1 > mx) mx = v1;
    if (v2 > mx) mx = v2;
    if (v3 > mx) mx = v3;
    lo[k] = mn;
    hi[k] = mx;
  }
}

/* equiangular gnomonic map of block point (x, y) of face b to the unit sphere */
void or_sphere_point(int b, double x, double y, double X[3]) {
  double ta = tan((x - 0.5) * M_PI / 2.0), tb = tan((y - 0.5) * M_PI / 2.0);
  double n[3], P[3];
  normal_of(b, n);
  for (int k = 0; k < 3; ++k) P[k] = n[k] + ta * kE1[b][k] / 2.0 + tb * kE2[b][k] / 2.0;
  double l = sqrt(dot3(P, P));
  for (int k = 0; k < 3; ++k) X[k] = P[k] / l;
}

/* area of the spherical triangle (a, b, c) (Van Oosterom & Strackee).  The
 * triple product a . (b x c) equals a . ((b - a) x (c - a)); the second form
 * keeps its relative accuracy for small triangles (the first cancels from
 * O(1) terms down to O(h^2)). */
static double tri_area(const double* a, const double* b, const double* c) {
  double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  double v[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
  double uv[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
  double num = fabs(dot3(a, uv));
  double den = 1.0 + dot3(a, b) + dot3(b, c) + dot3(c, a);
  return 2.0 * atan2(num, den);
}

/* metric terms of a leaf over its extended index range: kappa[S*S] (cells
 * -mbc..mx+mbc-1), phix[(S+1)*S] (x-edge i-1/2 of row j, i = -mbc..mx+mbc),
 * phiy[S*(S+1)] (y-edge j-1/2 of column i), for rotation vector omega */
void or_sphere_metrics(const or_leaf* a, int mx, int mbc, const double* omega, double* kappa,
                       double* phix, double* phiy) {
  int S = mx + 2 * mbc, SN = S + 1;
  double h = 1.0 / ldexp((double)mx, a->l);
  double* X = (double*)malloc(sizeof(double) * 3 * (size_t)SN * SN);
  for (int j = 0; j < SN; ++j)
    for (int i = 0; i < SN; ++i) {
      double x = ((double)a->x * mx + (i - mbc)) * h, y = ((double)a->y * mx + (j - mbc)) * h;
      or_sphere_point(a->b, x, y, X + 3 * (j * SN + i));
    }
#define N(i, j) (X + 3 * ((j) * SN + (i)))
  for (int j = 0; j < S; ++j)
    for (int i = 0; i < S; ++i)
      kappa[j * S + i] = tri_area(N(i, j), N(i + 1, j), N(i + 1, j + 1)) +
                         tri_area(N(i, j), N(i + 1, j + 1), N(i, j + 1));
  for (int j = 0; j < S; ++j)
    for (int i = 0; i < SN; ++i) {
      double d[3] = {N(i, j + 1)[0] - N(i, j)[0], N(i, j + 1)[1] - N(i, j)[1],
                     N(i, j + 1)[2] - N(i, j)[2]};
      phix[j * SN + i] = dot3(omega, d);
    }
  for (int j = 0; j < SN; ++j)
    for (int i = 0; i < S; ++i) {
      double d[3] = {N(i, j)[0] - N(i + 1, j)[0], N(i, j)[1] - N(i + 1, j)[1],
                     N(i, j)[2] - N(i + 1, j)[2]};
      phiy[j * S + i] = dot3(omega, d);
    }
#undef N
  free(X);
}

/* Sec. 5.3's deformational streamfunction at unit-sphere point X, time t:
 *   psi = k sin^2(rho - 2 pi t/T) cos^2(theta) cos(pi t/T) - 2 pi sin(theta)/T_f
 * with longitude rho and latitude theta of X; since X = cos(theta)(cos rho,
 * sin rho) + sin(theta) e_z, sin(rho - a) cos(theta) = Y cos a - X sin a =: s
 * and sin(theta) = Z (no angle is formed: smooth at the poles).  The velocity
 * is e_r x grad psi, as for the rotation, whose psi is -omega . X.  An edge's
 * flux is psi(b) - psi(a) = k c (s_b - s_a)(s_b + s_a) - (2 pi/T_f)(Z_b - Z_a)
 * (c = cos(pi t/T)), formed from the end points' differences: psi is O(1),
 * the flux O(h). */
static double deform_flux(const or_params* P, double t, const double* A, const double* B) {
  double k = P->vel[0], T = P->vel[1], Tf = P->vel[2];
  double a = 2.0 * M_PI * t / T, ca = cos(a), sa = sin(a);
  double scale = P->vel_scale != 0.0 ? P->vel_scale : 1.0;
  double ds = (B[1] - A[1]) * ca - (B[0] - A[0]) * sa;
  double ss = (B[1] + A[1]) * ca - (B[0] + A[0]) * sa;
  return scale * (k * cos(M_PI * t / T) * (ds * ss) - 2.0 * M_PI / Tf * (B[2] - A[2]));
}

void or_sphere_psi_fluxes(const or_leaf* a, const or_params* P, double t, double* phix,
                          double* phiy) {
  int mx = P->mx, mbc = P->mbc, S = mx + 2 * mbc, SN = S + 1;
  double h = 1.0 / ldexp((double)mx, a->l);
  double* X = (double*)malloc(sizeof(double) * 3 * (size_t)SN * SN);
  for (int j = 0; j < SN; ++j)
    for (int i = 0; i < SN; ++i) {
      double x = ((double)a->x * mx + (i - mbc)) * h, y = ((double)a->y * mx + (j - mbc)) * h;
      or_sphere_point(a->b, x, y, X + 3 * (j * SN + i));
    }
#define N(i, j) (X + 3 * ((j) * SN + (i)))
  /* the rotation's orientation: x-edge psi(bottom) - psi(top), y-edge
   * psi(right) - psi(left) (for psi = -omega . X these are omega . (X_top -
   * X_bottom) and omega . (X_left - X_right)) */
  for (int j = 0; j < S; ++j)
    for (int i = 0; i < SN; ++i) phix[j * SN + i] = deform_flux(P, t, N(i, j + 1), N(i, j));
  for (int j = 0; j < SN; ++j)
    for (int i = 0; i < S; ++i) phiy[j * S + i] = deform_flux(P, t, N(i, j), N(i + 1, j));
#undef N
  free(X);
}

void or_sphere_edge_fluxes(const or_forest* F, double t, double* phix, double* phiy) {
  size_t S = (size_t)F->S;
  for (int p = 0; p < F->n; ++p) {
    if (F->P.vel_kind == OR_VEL_DEFORM) {
      or_sphere_psi_fluxes(&F->lv[p], &F->P, t, phix + p * (S + 1) * S, phiy + p * S * (S + 1));
    } else {
      memcpy(phix + p * (S + 1) * S, F->phix + p * (S + 1) * S, sizeof(double) * (S + 1) * S);
      memcpy(phiy + p * S * (S + 1), F->phiy + p * S * (S + 1), sizeof(double) * S * (S + 1));
    }
  }
}

/* Capacity-form wave-propagation step of one patch (the flat step with cell
 * capacities kappa and edge volume fluxes phi in place of h^2 and h s):
 *   W = Q_R - Q_L, F = phi+ Q_L + phi- Q_R + Ft,
 *   Ft = 1/2 |phi| (1 - dt |phi| (1/kappa_L + 1/kappa_R)/2) phi(theta) W,
 *   P = phi+ W - Ft into R, M = phi- W + Ft into L, each carried across the
 *   transverse edges of its cell with 1/2 dt/kappa_cell phi_transverse,
 *   Q -= dt/kappa (F(i+1/2) - F(i-1/2) + G(j+1/2) - G(j-1/2)). */
void or_claw_step_capacity(const or_params* P, double* q, int mx, int mbc, double dt,
                           const double* kappa, const double* phix, const double* phiy,
                           double* bflux) {
  int S = mx + 2 * mbc, SE = S + 1;
  double* Fa = (double*)calloc((size_t)SE * SE, sizeof(double));
  double* Ga = (double*)calloc((size_t)SE * SE, sizeof(double));
#define Q(i, j) q[((i) + mbc) + S * ((j) + mbc)]
#define K(i, j) kappa[((i) + mbc) + S * ((j) + mbc)]
#define PX(i, j) phix[((i) + mbc) + SE * ((j) + mbc)]
#define PY(i, j) phiy[((i) + mbc) + S * ((j) + mbc)]
#define FX(i, j) Fa[((i) + mbc) + SE * ((j) + mbc)]
#define GY(i, j) Ga[((i) + mbc) + SE * ((j) + mbc)]
#define POS(a) ((a) > 0.0 ? (a) : 0.0)
#define NEG(a) ((a) < 0.0 ? (a) : 0.0)
  for (int j = -1; j <= mx; ++j)
    for (int i = 0; i <= mx; ++i) {
      double s = PX(i, j);
      double W = Q(i, j) - Q(i - 1, j);
      double Wup = (s >= 0.0) ? Q(i - 1, j) - Q(i - 2, j) : Q(i + 1, j) - Q(i, j);
      double Ft = 0.0;
      if (P->order >= 2) {
        double lim = W;
        if (P->limiter == 1) lim = (W == 0.0) ? 0.0 : or_mc_phi(Wup / W) * W;
        double as = fabs(s);
        double cr = dt * as * 0.5 * (1.0 / K(i - 1, j) + 1.0 / K(i, j));
        Ft = 0.5 * as * (1.0 - cr) * lim;
      }
      FX(i, j) += POS(s) * Q(i - 1, j) + NEG(s) * Q(i, j) + Ft;
      if (P->transverse > 0) {
        double Pf = POS(s) * W, Mf = NEG(s) * W;
        if (P->transverse > 1) {
          Pf -= Ft;
          Mf += Ft;
        }
        GY(i, j + 1) -= 0.5 * dt / K(i, j) * POS(PY(i, j + 1)) * Pf;
        GY(i, j) -= 0.5 * dt / K(i, j) * NEG(PY(i, j)) * Pf;
        GY(i - 1, j + 1) -= 0.5 * dt / K(i - 1, j) * POS(PY(i - 1, j + 1)) * Mf;
        GY(i - 1, j) -= 0.5 * dt / K(i - 1, j) * NEG(PY(i - 1, j)) * Mf;
      }
    }
  for (int i = -1; i <= mx; ++i)
    for (int j = 0; j <= mx; ++j) {
      double s = PY(i, j);
      double W = Q(i, j) - Q(i, j - 1);
      double Wup = (s >= 0.0) ? Q(i, j - 1) - Q(i, j - 2) : Q(i, j + 1) - Q(i, j);
      double Gt = 0.0;
      if (P->order >= 2) {
        double lim = W;
        if (P->limiter == 1) lim = (W == 0.0) ? 0.0 : or_mc_phi(Wup / W) * W;
        double as = fabs(s);
        double cr = dt * as * 0.5 * (1.0 / K(i, j - 1) + 1.0 / K(i, j));
        Gt = 0.5 * as * (1.0 - cr) * lim;
      }
      GY(i, j) += POS(s) * Q(i, j - 1) + NEG(s) * Q(i, j) + Gt;
      if (P->transverse > 0) {
        double Pf = POS(s) * W, Mf = NEG(s) * W;
        if (P->transverse > 1) {
          Pf -= Gt;
          Mf += Gt;
        }
        FX(i + 1, j) -= 0.5 * dt / K(i, j) * POS(PX(i + 1, j)) * Pf;
        FX(i, j) -= 0.5 * dt / K(i, j) * NEG(PX(i, j)) * Pf;
        FX(i + 1, j - 1) -= 0.5 * dt / K(i, j - 1) * POS(PX(i + 1, j - 1)) * Mf;
        FX(i, j - 1) -= 0.5 * dt / K(i, j - 1) * NEG(PX(i, j - 1)) * Mf;
      }
    }
  /* the fluxes through the patch's faces, as the update below uses them */
  if (bflux)
    for (int k = 0; k < mx; ++k) {
      bflux[k] = FX(0, k);
      bflux[mx + k] = FX(mx, k);
      bflux[2 * mx + k] = GY(k, 0);
      bflux[3 * mx + k] = GY(k, mx);
    }
  for (int j = 0; j < mx; ++j)
    for (int i = 0; i < mx; ++i)
      Q(i, j) = Q(i, j) - dt / K(i, j) * ((FX(i + 1, j) - FX(i, j)) + (GY(i, j + 1) - GY(i, j)));
#undef Q
#undef K
#undef PX
#undef PY
#undef FX
#undef GY
#undef POS
#undef NEG
  free(Fa);
  free(Ga);
}

void or_sphere_centres(const or_forest* F, double* xyz) {
  int mx = F->P.mx;
  for (int p = 0; p < F->n; ++p) {
    const or_leaf* a = &F->lv[p];
    double h = 1.0 / ldexp((double)mx, a->l);
    for (int j = 0; j < mx; ++j)
      for (int i = 0; i < mx; ++i)
        or_sphere_point(a->b, ((double)a->x * mx + i + 0.5) * h, ((double)a->y * mx + j + 0.5) * h,
                        xyz + 3 * (((size_t)p * mx + j) * mx + i));
  }
}

void or_get_kappa_full(const or_forest* F, double* kappa) {
  size_t n = (size_t)F->n * F->S * F->S;
  for (size_t c = 0; c < n; ++c) kappa[c] = F->kappa ? F->kappa[c] : 0.0;
}

void or_get_kappa(const or_forest* F, double* kappa) {
  int mx = F->P.mx;
  for (int p = 0; p < F->n; ++p)
    for (int j = 0; j < mx; ++j)
      for (int i = 0; i < mx; ++i)
        kappa[((size_t)p * mx + j) * mx + i] =
            F->kappa ? F->kappa[(size_t)p * F->S * F->S + OR_IDX(F, i, j)] : 0.0;
}
