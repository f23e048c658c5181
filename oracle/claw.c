/*
 * Oracle: the single-grid wave-propagation update of one patch.
 * Test infrastructure only (see oracle.h).
 *
 * The paper uses Clawpack's wave-propagation algorithms without restating
 * them (Sec. 5, "Scaling results").  This is the published 2D unsplit method
 * (LeVeque, J. Comput. Phys. 131, 1997; Finite Volume Methods for Hyperbolic
 * Problems, 2002, Ch. 6 and 20) for the conservative scalar advection
 * equation q_t + (u q)_x + (v q)_y = 0, written in flux form:
 *
 *   x-edge (i-1/2, j), speed s:  W = Q(i,j) - Q(i-1,j)
 *     F(i-1/2,j) = s+ Q(i-1,j) + s- Q(i,j) + Ft,
 *     Ft = 1/2 |s| (1 - dt/h |s|) phi(theta) W,  theta = W_upwind / W,
 *     fluctuation into cell i:   P = s+ W - Ft,
 *     fluctuation into cell i-1: M = s- W + Ft,
 *   each fluctuation is carried across the y-edges of the cell it enters
 *   (transverse propagation):  G(edge above) -= 1/2 dt/h v+ P,
 *                              G(edge below) -= 1/2 dt/h v- P,
 *   and symmetrically for the y-edges, then
 *   Q(i,j) -= dt/h (F(i+1/2,j) - F(i-1/2,j)) + dt/h (G(i,j+1/2) - G(i,j-1/2)).
 *
 * Edge speeds come from a streamfunction psi at the cell corners
 * (Sec. 5.1: the velocity field is defined by a streamfunction):
 *   u(i-1/2, j) =  (psi(x_{i-1/2}, y_{j+1/2}) - psi(x_{i-1/2}, y_{j-1/2})) / h
 *   v(i, j-1/2) = -(psi(x_{i+1/2}, y_{j-1/2}) - psi(x_{i-1/2}, y_{j-1/2})) / h
 * For a constant velocity the differences are exact and the constants are
 * used directly.  Swirl: psi = sin^2(pi x) sin^2(pi y) cos(pi t / T) / pi,
 * evaluated at the half step.  Corner coordinates are (global index) * h.
 */
#include "internal.h"

#include <math.h>
#include <stdlib.h>

double or_mc_phi(double theta) {
  double a = 0.5 * (1.0 + theta);
  double m = a < 2.0 ? a : 2.0;
  m = m < 2.0 * theta ? m : 2.0 * theta;
  return m > 0.0 ? m : 0.0;
}

typedef struct {
  const or_params* P;
  double h, thalf;
  long gx0, gy0;
} velctx;

/* The swirl streamfunction is separable, psi = s(x) s(y) cos(pi t/T) / pi
 * with s(z) = sin^2(pi z), so the corner difference along an edge is
 * s(x) (s(y1) - s(y0)) cos(pi t/T) / pi.  The difference of the two squares is
 * evaluated as sin(pi (y1 + y0)) sin(pi (y1 - y0)) -- the same number in
 * exact arithmetic, without the cancellation that subtracting two O(1) values
 * to get an O(h) result would cost (about 1e-16 / h relative). */
static double s2(long I, double h) {
  double s = sin(M_PI * ((double)I * h));
  return s * s;
}

static double dsq(long J0, double h) { /* s(y_{J0+1}) - s(y_{J0}) */
  return sin(M_PI * ((double)(2 * J0 + 1) * h)) * sin(M_PI * h);
}

static double scale_of(const or_params* P) { return P->vel_scale != 0.0 ? P->vel_scale : 1.0; }

/* speed at x-edge (i-1/2, j) */
static double u_edge(const velctx* c, int i, int j) {
  if (c->P->vel_kind == OR_VEL_CONST) return scale_of(c->P) * c->P->vel[0];
  long I = c->gx0 + i, J = c->gy0 + j;
  double ct = cos(M_PI * c->thalf / c->P->vel[0]) / M_PI;
  return scale_of(c->P) * (ct * s2(I, c->h) * dsq(J, c->h) / c->h);
}

/* speed at y-edge (i, j-1/2) */
static double v_edge(const velctx* c, int i, int j) {
  if (c->P->vel_kind == OR_VEL_CONST) return scale_of(c->P) * c->P->vel[1];
  long I = c->gx0 + i, J = c->gy0 + j;
  double ct = cos(M_PI * c->thalf / c->P->vel[0]) / M_PI;
  return scale_of(c->P) * (-ct * s2(J, c->h) * dsq(I, c->h) / c->h);
}

double or_u_edge(const or_params* P, double h, double t, long gx0, long gy0, int i, int j) {
  velctx c = {P, h, t, gx0, gy0};
  return u_edge(&c, i, j);
}

double or_v_edge(const or_params* P, double h, double t, long gx0, long gy0, int i, int j) {
  velctx c = {P, h, t, gx0, gy0};
  return v_edge(&c, i, j);
}

static double pos(double a) { return a > 0.0 ? a : 0.0; }
static double neg(double a) { return a < 0.0 ? a : 0.0; }

/* second-order correction flux for one edge */
static double correction(const or_params* P, double s, double W, double Wup, double nu) {
  if (P->order < 2) return 0.0;
  double phi = 1.0;
  if (P->limiter == 1) {
    if (W == 0.0) return 0.0;
    phi = or_mc_phi(Wup / W);
  }
  double as = fabs(s);
  return 0.5 * as * (1.0 - nu * as) * phi * W;
}

void or_claw_step(const or_params* P, double* q, int mx, int mbc, double h, double dt,
                  double t, long gx0, long gy0) {
  or_claw_step_flux(P, q, mx, mbc, h, dt, t, gx0, gy0, NULL);
}

void or_claw_step_flux(const or_params* P, double* q, int mx, int mbc, double h, double dt,
                       double t, long gx0, long gy0, double* bflux) {
  int S = mx + 2 * mbc;
  int SE = S + 1;
  double nu = dt / h;
  velctx c = {P, h, t + 0.5 * dt, gx0, gy0};
  /* F(i,j): x-edge i-1/2 of row j;  G(i,j): y-edge j-1/2 of column i */
  double* Fa = (double*)calloc((size_t)SE * SE, sizeof(double));
  double* Ga = (double*)calloc((size_t)SE * SE, sizeof(double));
#define Q(i, j) q[((i) + mbc) + S * ((j) + mbc)]
#define FX(i, j) Fa[((i) + mbc) + SE * ((j) + mbc)]
#define GY(i, j) Ga[((i) + mbc) + SE * ((j) + mbc)]
  /* x-sweep */
  for (int j = -1; j <= mx; ++j)
    for (int i = 0; i <= mx; ++i) {
      double s = u_edge(&c, i, j);
      double W = Q(i, j) - Q(i - 1, j);
      double Wup = (s >= 0.0) ? Q(i - 1, j) - Q(i - 2, j) : Q(i + 1, j) - Q(i, j);
      double Ft = correction(P, s, W, Wup, nu);
      FX(i, j) += pos(s) * Q(i - 1, j) + neg(s) * Q(i, j) + Ft;
      if (P->transverse > 0) {
        double Pf = pos(s) * W, Mf = neg(s) * W;
        if (P->transverse > 1) {
          Pf -= Ft;
          Mf += Ft;
        }
        GY(i, j + 1) -= 0.5 * nu * pos(v_edge(&c, i, j + 1)) * Pf;
        GY(i, j) -= 0.5 * nu * neg(v_edge(&c, i, j)) * Pf;
        GY(i - 1, j + 1) -= 0.5 * nu * pos(v_edge(&c, i - 1, j + 1)) * Mf;
        GY(i - 1, j) -= 0.5 * nu * neg(v_edge(&c, i - 1, j)) * Mf;
      }
    }
  /* y-sweep */
  for (int i = -1; i <= mx; ++i)
    for (int j = 0; j <= mx; ++j) {
      double s = v_edge(&c, i, j);
      double W = Q(i, j) - Q(i, j - 1);
      double Wup = (s >= 0.0) ? Q(i, j - 1) - Q(i, j - 2) : Q(i, j + 1) - Q(i, j);
      double Gt = correction(P, s, W, Wup, nu);
      GY(i, j) += pos(s) * Q(i, j - 1) + neg(s) * Q(i, j) + Gt;
      if (P->transverse > 0) {
        double Pf = pos(s) * W, Mf = neg(s) * W;
        if (P->transverse > 1) {
          Pf -= Gt;
          Mf += Gt;
        }
        FX(i + 1, j) -= 0.5 * nu * pos(u_edge(&c, i + 1, j)) * Pf;
        FX(i, j) -= 0.5 * nu * neg(u_edge(&c, i, j)) * Pf;
        FX(i + 1, j - 1) -= 0.5 * nu * pos(u_edge(&c, i + 1, j - 1)) * Mf;
        FX(i, j - 1) -= 0.5 * nu * neg(u_edge(&c, i, j - 1)) * Mf;
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
  /* conservative update of the interior */
  for (int j = 0; j < mx; ++j)
    for (int i = 0; i < mx; ++i)
      Q(i, j) = Q(i, j) - nu * (FX(i + 1, j) - FX(i, j)) - nu * (GY(i, j + 1) - GY(i, j));
#undef Q
#undef FX
#undef GY
  free(Fa);
  free(Ga);
}
