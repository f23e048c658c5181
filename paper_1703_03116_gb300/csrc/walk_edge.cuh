// One edge of the wave-propagation method, in the form the row-walking
// update kernels (walk, band) evaluate it: per edge the upwind normal flux
// with its MC-limited second-order correction, and the two fluctuations
// that the transverse terms carry into the neighbouring edges (the flux form
// of the unsplit method of Sec. 5, with the correction waves propagated
// transversely when transverse = 2).
#pragma once

#include "device_util.cuh"

namespace fc {

template <typename real>
struct Scheme {
  real nu;    // dt / h
  real tfac;  // 1/2 dt/h with transverse propagation, else 0
  real t2;    // 1 when correction waves are propagated transversely, else 0
  bool order2, mc;
};

template <typename real>
__device__ __forceinline__ Scheme<real> make_scheme(int order, int limiter, int transverse,
                                                    double nu) {
  Scheme<real> sc;
  sc.nu = real(nu);
  sc.tfac = transverse > 0 ? real(0.5 * nu) : real(0);
  sc.t2 = transverse > 1 ? real(1) : real(0);
  sc.order2 = order > 1;
  sc.mc = limiter != 0;
  return sc;
}

// one edge between cells qb (upwind-left/below) and qc, with the outer
// neighbours qa (behind qb) and qd (beyond qc): normal flux and the two
// fluctuations entering the right/upper (P) and left/lower (M) cell; nu the
// edge's dt/h in the correction (capacity form: dt (1/kappa_b + 1/kappa_c)/2)
template <typename real>
__device__ __forceinline__ void edge(real s, real qa, real qb, real qc, real qd, real nu,
                                     const Scheme<real>& sc, real& Fn, real& P, real& M) {
  const real sp = fmax(s, real(0)), sm = fmin(s, real(0));
  const real W = qc - qb;
  const real Wup = s >= real(0) ? qb - qa : qd - qc;
  const real as = fabs(s);
  const real cf = sc.order2 ? real(0.5) * as * (real(1) - nu * as) : real(0);
  const real Ft = cf * (sc.mc ? mc_limited(W, Wup) : W);
  Fn = sp * qb + sm * qc + Ft;
  P = sp * W - sc.t2 * Ft;
  M = sm * W + sc.t2 * Ft;
}

template <typename real>
__device__ __forceinline__ void edge(real s, real qa, real qb, real qc, real qd,
                                     const Scheme<real>& sc, real& Fn, real& P, real& M) {
  edge(s, qa, qb, qc, qd, sc.nu, sc, Fn, P, M);
}

}  // namespace fc
