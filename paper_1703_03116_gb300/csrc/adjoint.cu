// Adjoint (reverse mode) of one global time step: q^{n+1} = S(Fill(q^n)).
//
// Both maps are piecewise linear in q: the MC limiter and the minmod slopes of
// the ghost interpolation select a linear piece.  The adjoint applies the
// transpose of every operation in reverse order, on the piece the forward
// state selects (the a.e. derivative):
//
//  adj_advance     per patch: forward tile and adjoint of the new interior
//                  in shared memory; transpose of the update, of the
//                  transverse increments, and of every edge; then the
//                  transpose of the second wall-BC pass.  Writes the adjoint
//                  of the whole input tile (interior + ghosts) and adds
//                  sum_e dL/ds_e * s_e to an FP64 accumulator (the velocity
//                  scale derivative times the scale).
//  adj_interp      transpose of the interpolation (Eq. ghost_fine): each
//                  fine ghost's adjoint goes to the coarse cells it read
//                  (atomic adds into the coarse patch's tile).
//  adj_bc          transpose of the first wall-BC pass (local to a patch).
//  adj_copy        transpose of copy / average (Eq. transform,
//                  Eq. ghost_coarse): ghost adjoints go to the neighbours'
//                  interior cells (atomic adds).
//
// Multirate substep of level L (launch_adjoint_substep), two kernels: the
// update's transpose followed, in the same CTA, by that of the patch's ghost
// fill (adj_advance); the transposes of the ghosts of the level L-1 patches
// read through the time-interpolated tiles and of qT = (1 - alpha) q_old +
// alpha q (adj_coarse_tiles; sources read on the fly split their share
// inside the copy transpose).  Each level's
// adjoint of one state accumulates in one of two buffers (AdjAcc), every
// contribution an atomic add into a zeroed accumulator, so the substeps of
// different levels can run side by side wherever their forward substeps
// could.
// The adjoint tiles use the patch-store layout ((mx+4)^2 per patch).
#include <atomic>

#include "ghost_gather.cuh"

namespace fc {
namespace {

// limited wave piece of the division-free MC form and its partials
template <typename real>
__device__ __forceinline__ real mc_piece(real W, real Wup, real& dW, real& dWup) {
  dW = dWup = real(0);
  if (!(W * Wup > real(0))) return real(0);
  const real a = real(0.5) * fabs(W + Wup);
  const real b = real(2) * fabs(W), c = real(2) * fabs(Wup);
  if (a <= b && a <= c) {
    dW = dWup = real(0.5);
    return copysign(a, W);
  }
  if (b <= c) {
    dW = real(2);
    return copysign(b, W);
  }
  dWup = real(2);
  return copysign(c, W);
}

template <typename real>
struct EdgeFw {
  real W, Wup, lim, dW, dWup, c, dc, Ft, P, M;
  bool up;
};

template <typename real>
__device__ __forceinline__ EdgeFw<real> edge_fw(int order, int limiter, int transverse, real s,
                                                real qa, real qb, real qc, real qd, real nu) {
  EdgeFw<real> e;
  e.W = qc - qb;
  e.up = s >= real(0);
  e.Wup = e.up ? qb - qa : qd - qc;
  if (limiter) {
    e.lim = mc_piece(e.W, e.Wup, e.dW, e.dWup);
  } else {
    e.lim = e.W;
    e.dW = real(1);
    e.dWup = real(0);
  }
  const real as = fabs(s);
  e.c = order > 1 ? real(0.5) * as * (real(1) - nu * as) : real(0);
  e.dc = order > 1 ? real(0.5) * (s > real(0) ? real(1) : (s < real(0) ? real(-1) : real(0))) *
                         (real(1) - real(2) * nu * as)
                   : real(0);
  e.Ft = e.c * e.lim;
  const real sp = s > real(0) ? s : real(0), sm = s < real(0) ? s : real(0);
  e.P = sp * e.W - (transverse > 1 ? e.Ft : real(0));
  e.M = sm * e.W + (transverse > 1 ? e.Ft : real(0));
  return e;
}

// ---------------------------------------------------------------------
// Transposes of Alg. 1, per patch (threads tid, stride nt of a group that
// holds the patch's staged neighbour entries).  Each consumes (zeroes) the
// adjoint of the patch's own ghost cells it handles and scatters it, with
// atomics, to the cells those ghosts were computed from.

// transpose of a wall-BC pass: exterior ghost adjoint -> the clamped cell (an
// exterior ghost copies a non-exterior cell, so one pass in any order)
template <typename real, int MX>
__device__ void adj_bc_patch(const PatchMeta& pm, real* L, int tid, int nt) {
  constexpr int S = MX + 4;
  const int N = MX << pm.level;
  for (int k = tid; k < num_ghosts<MX>(); k += nt) {
    int i, j;
    ghost_ij<MX>(k, i, j);
    const int gx = pm.x * MX + i, gy = pm.y * MX + j;
    const bool ox = gx < 0 || gx >= N, oy = gy < 0 || gy >= N;
    if (!ox && !oy) continue;
    const int ic = ox ? (gx < 0 ? 0 : MX - 1) : i;
    const int jc = oy ? (gy < 0 ? 0 : MX - 1) : j;
    atomicAdd(&L[(jc + kMbc) * S + ic + kMbc], L[(j + kMbc) * S + i + kMbc]);
    L[(j + kMbc) * S + i + kMbc] = real(0);
  }
}

// transpose of the interpolation (Eq. ghost_fine): each coarse ghost's
// adjoint goes to the coarse cells it read, on the minmod pieces the forward
// data select.  A coarse patch on `tlevel` was read through the time-
// interpolated tiles (coarse_src: patch c at coarse_src + (c - coarse_p0)
// tiles, else D.qT) and takes the adjoint in lamT; else from the store, lam.
template <typename real, int MX>
__device__ void adj_interp_patch(const DevForest<real>& D, const NbrStage& st, const PatchMeta& pm,
                                 real* L, real* lam, int tlevel, real* lamT, const real* coarse_src,
                                 int coarse_p0, int tid, int nt) {
  constexpr int S = MX + 4;
  for (int k = tid; k < num_ghosts<MX>(); k += nt) {
    int i, j;
    ghost_ij<MX>(k, i, j);
    const int r = region_of<MX>(i, j);
    const NbrEntry& e = st.e[r];
    if (e.kind != NB_COARSE) continue;
    const int2 Ip = apply_a(e.a, pm.x * MX + i, pm.y * MX + j);
    const int gx = Ip.x + e.fx, gy = Ip.y + e.fy;
    const PatchMeta& nm = st.m0[r];
    const int ic = (gx >> 1) - nm.x * MX, jc = (gy >> 1) - nm.y * MX;
    if (ic < 0 || ic >= MX || jc < 0 || jc >= MX) continue;
    const real dx = (gx & 1) ? real(1) : real(-1);
    const real dy = (gy & 1) ? real(1) : real(-1);
    const size_t o = (size_t)(jc + kMbc) * S + ic + kMbc;
    const bool viaT = nm.level == tlevel;
    const real* C = (viaT ? (coarse_src ? coarse_src + (size_t)(e.n0 - coarse_p0) * S * S
                                        : patch_ptr(D.qT, e.n0, S))
                          : patch_ptr(D.buf[D.cur[nm.level]], e.n0, S)) +
                    o;
    real* LC = (viaT ? lamT : lam) + (size_t)e.n0 * S * S + o;
    const real lg = L[(j + kMbc) * S + i + kMbc];
    L[(j + kMbc) * S + i + kMbc] = real(0);
    const real q0 = C[0];
    const real ax = C[1] - q0, bx = q0 - C[-1], ay = C[S] - q0, by = q0 - C[-S];
    const real dax = (ax * bx > real(0) && fabs(ax) < fabs(bx)) ? real(1) : real(0);
    const real dbx = (ax * bx > real(0) && !(fabs(ax) < fabs(bx))) ? real(1) : real(0);
    const real day = (ay * by > real(0) && fabs(ay) < fabs(by)) ? real(1) : real(0);
    const real dby = (ay * by > real(0) && !(fabs(ay) < fabs(by))) ? real(1) : real(0);
    const real lsx = real(0.25) * dx * lg, lsy = real(0.25) * dy * lg;
    atomicAdd(LC, lg + lsx * (dbx - dax) + lsy * (dby - day));
    atomicAdd(LC + 1, lsx * dax);
    atomicAdd(LC - 1, -lsx * dbx);
    atomicAdd(LC + S, lsy * day);
    atomicAdd(LC - S, -lsy * dby);
  }
}

// Where the transposes of copies and averages add: a neighbour on the
// coarser level tlevel was read as (1 - alpha) q_old + alpha q (its shares
// go to the accumulators of its older and newer states); a same-size one at
// `same`, a finer one at `fine` (accumulators of those levels' states at the
// substep's time).
template <typename real>
struct AdjTargets {
  real* same;
  real* fine;
  real* t_old;
  real* t_new;
};

template <typename real>
__device__ __forceinline__ void adj_src_add(const AdjTargets<real>& g, bool viaT, bool fine,
                                            real alpha, size_t o, real v) {
  if (viaT) {
    atomicAdd(g.t_old + o, (real(1) - alpha) * v);
    if (alpha != real(0)) atomicAdd(g.t_new + o, alpha * v);
  } else {
    atomicAdd((fine ? g.fine : g.same) + o, v);
  }
}

// transpose of copy / average (Eq. transform, Eq. ghost_coarse): ghost
// adjoint (in L, the patch's own tile) -> neighbour interiors
template <typename real, int MX>
__device__ void adj_copy_patch(const NbrStage& st, const PatchMeta& pm, real* L,
                               const AdjTargets<real>& g, int tlevel, real alpha, int tid, int nt) {
  constexpr int S = MX + 4;
  for (int k = tid; k < num_ghosts<MX>(); k += nt) {
    int i, j;
    ghost_ij<MX>(k, i, j);
    const int r = region_of<MX>(i, j);
    const NbrEntry& e = st.e[r];
    if (e.kind != NB_SAME && e.kind != NB_FINE) continue;
    const real lg = L[(j + kMbc) * S + i + kMbc];
    L[(j + kMbc) * S + i + kMbc] = real(0);
    const int2 Ip = apply_a(e.a, pm.x * MX + i, pm.y * MX + j);
    const int gx = Ip.x + e.fx, gy = Ip.y + e.fy;
    if (e.kind == NB_SAME) {
      const PatchMeta& nm = st.m0[r];
      const int lx = gx - nm.x * MX, ly = gy - nm.y * MX;
      if (lx < 0 || lx >= MX || ly < 0 || ly >= MX) continue;
      adj_src_add(g, nm.level == tlevel, false, alpha,
                  (size_t)e.n0 * S * S + (ly + kMbc) * S + lx + kMbc, lg);
    } else {
      int n = e.n0;
      const PatchMeta* nm = &st.m0[r];
      int lx = 2 * gx - nm->x * MX, ly = 2 * gy - nm->y * MX;
      if (lx < 0 || lx >= MX || ly < 0 || ly >= MX) {
        if (e.n1 < 0) continue;
        n = e.n1;
        nm = &st.m1[r];
        lx = 2 * gx - nm->x * MX;
        ly = 2 * gy - nm->y * MX;
        if (lx < 0 || lx >= MX || ly < 0 || ly >= MX) continue;
      }
      for (int q = 0; q < 4; ++q)
        adj_src_add(g, nm->level == tlevel, true, alpha,
                    (size_t)n * S * S + (ly + (q >> 1) + kMbc) * S + lx + (q & 1) + kMbc,
                    real(0.25) * lg);
    }
  }
}

// Where the update transpose of a multirate substep also transposes its
// patches' ghost fill (the level's Alg. 1, reversed: interpolation from the
// coarse tiles into lamT, then copies and averages into the accumulators of
// level L, lam_out, and of level L+1, lam_fine) straight from the tile's
// adjoint in shared memory.
template <typename real>
struct AdjGhosts {
  real* lam_fine;
  real* lamT;
  const real* coarse_src;
  int coarse_p0, tlevel;
};

// The forward tile of patch p is read from the store, or from
// tiles + (p - tiles_p0) tiles when `tiles` is given (kept copies).  acc
// (multirate accumulators, with g): lam_in's tile is cleared once read, the
// ghost ring of the input tile's adjoint is transposed through the level's
// ghost fill at once (g), and its interior is added to lam_out's (other
// levels' and neighbours' transposes add there too).
template <typename real, int MX, int NT>
__global__ void __launch_bounds__(NT) adj_advance_kernel(DevForest<real> D, AdvArgs a,
                                                         real* lam_in, real* lam_out,
                                                         double* dscale, double dfac, int p0,
                                                         int p1, const real* tiles, int tiles_p0,
                                                         int acc, AdjGhosts<real> g) {
  constexpr int S = MX + 4;
  constexpr int NE = (MX + 1) * (MX + 2);
  constexpr int NV = MX + 3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real* Q = reinterpret_cast<real*>(smem_raw);
  real* LQ = Q + S * S;       // adjoint of the input tile
  real* LN = LQ + S * S;      // adjoint of the new interior (MX*MX)
  real* LF = LN + MX * MX;    // adjoint of x-edge normal flux / final flux
  real* LG = LF + NE;         // same for y-edges
  real* YS = LG + NE;         // forward y-fluctuation into each cell column -1..MX, rows 0..MX-1
  real* XS = YS + (MX + 2) * MX;  // forward x-fluctuation into cells, columns 0..MX-1, rows -1..MX
  real* LY = XS + MX * (MX + 2);  // adjoint of Y
  real* LX = LY + (MX + 2) * MX;  // adjoint of X
  real* Sx = LX + MX * (MX + 2);
  real* Sy = Sx + NV;
  real* Tx = Sy + NV;
  real* Ty = Tx + NV;
  __shared__ double red[NT / 32];
  __shared__ real ucoef_s;
  __shared__ NbrStage st;  // acc: the patch's neighbour entries
  const int order = D.order, limiter = D.limiter, transverse = D.transverse;
  const bool swirl = D.vel_kind == FC_VEL_SWIRL;
  const real cu = real(D.vel[0]), cv = real(D.vel[1]);
  const real nu = real(a.nu), hn = real(0.5 * a.nu), h = real(a.h);
  if (threadIdx.x == 0 && swirl) {
    const double t = a.t0_dev ? *a.t0_dev + a.t_off : a.t_half;  // graph replay: time on device
    ucoef_s = cospi_ratio<real>(t, a.period) * real(a.sfac);
  }
  __syncthreads();
  const real ucoef = swirl ? ucoef_s : real(0);
  // velocity-scale derivative: per-thread partial sums in the field's
  // precision (FP64 arithmetic is scarce on this GPU), FP64 from the block
  // reduction on
  real dsum = 0;

  for (int p = p0 + blockIdx.x; p < p1; p += gridDim.x) {
    const PatchMeta pm = D.meta[p];
    const real* src = tiles ? tiles + (size_t)(p - tiles_p0) * S * S
                            : D.buf[D.cur[pm.level]] + (size_t)p * S * S;
    real* lin = lam_in + (size_t)p * S * S;
    if (acc) stage_neighbours(D.meta, D.nbr, p, st, threadIdx.x);
    for (int k = threadIdx.x; k < S * S; k += NT) {
      Q[k] = src[k];
      LQ[k] = real(0);
    }
    for (int k = threadIdx.x; k < MX * MX; k += NT) {
      const int o = (k / MX + 2) * S + (k % MX) + 2;
      LN[k] = lin[o];
      if (acc) lin[o] = real(0);  // consumed: the buffer's next state starts from zero
    }
    if (swirl)
      for (int k = threadIdx.x; k < NV; k += NT) {
        const real xs = sinpi_r(real(pm.x * MX + k - 1) * h);
        const real ys = sinpi_r(real(pm.y * MX + k - 1) * h);
        Sx[k] = xs * xs;
        Sy[k] = ys * ys;
        Tx[k] = sinpi_r(real(2 * (pm.x * MX + k - 1) + 1) * h);
        Ty[k] = sinpi_r(real(2 * (pm.y * MX + k - 1) + 1) * h);
      }
    __syncthreads();
    auto q = [&](int i, int j) -> real { return Q[(j + 2) * S + (i + 2)]; };
    auto lq = [&](int i, int j) -> real* { return &LQ[(j + 2) * S + (i + 2)]; };
    auto uvel = [&](int i, int j) -> real { return swirl ? ucoef * Sx[i + 1] * Ty[j + 1] : cu; };
    auto vvel = [&](int i, int j) -> real { return swirl ? -ucoef * Sy[j + 1] * Tx[i + 1] : cv; };
    auto ln = [&](int i, int j) -> real {
      return (i >= 0 && i < MX && j >= 0 && j < MX) ? LN[j * MX + i] : real(0);
    };
    auto xe = [](int i, int j) { return (j + 1) * (MX + 1) + i; };
    auto ye = [](int i, int j) { return j * (MX + 2) + (i + 1); };
    // forward transverse inputs: Y(c, j) for c in [-1,MX], j in [0,MX); X(i, r) for i in [0,MX), r in [-1,MX]
    for (int k = threadIdx.x; k < 2 * (MX + 2) * MX; k += NT) {
      if (k < (MX + 2) * MX) {
        const int c = k % (MX + 2) - 1, j = k / (MX + 2);
        real Y = 0;
        for (int r = j; r <= j + 1; ++r) {  // y-edges (c, j) [P into (c,j)] and (c, j+1) [M into (c,j)]
          const real s = vvel(c, r);
          const EdgeFw<real> e =
              edge_fw(order, limiter, transverse, s, q(c, r - 2), q(c, r - 1), q(c, r), q(c, r + 1), nu);
          Y += (r == j) ? e.P : e.M;
        }
        YS[k] = Y;
      } else {
        const int f = k - (MX + 2) * MX;
        const int i = f % MX, r = f / MX - 1;
        real X = 0;
        for (int c = i; c <= i + 1; ++c) {
          const real s = uvel(c, r);
          const EdgeFw<real> e =
              edge_fw(order, limiter, transverse, s, q(c - 2, r), q(c - 1, r), q(c, r), q(c + 1, r), nu);
          X += (c == i) ? e.P : e.M;
        }
        XS[f] = X;
      }
    }
    // transpose of the update: Q_new = Q - nu dF - nu dG
    for (int k = threadIdx.x; k < 2 * NE; k += NT) {
      if (k < NE) {
        const int i = k % (MX + 1), j = k / (MX + 1) - 1;  // x-edge (i, j)
        LF[k] = (j >= 0 && j < MX) ? nu * (ln(i, j) - ln(i - 1, j)) : real(0);
      } else {
        const int f = k - NE;
        const int i = f % (MX + 2) - 1, j = f / (MX + 2);  // y-edge (i, j)
        LG[f] = (i >= 0 && i < MX) ? nu * (ln(i, j) - ln(i, j - 1)) : real(0);
      }
    }
    for (int k = threadIdx.x; k < MX * MX; k += NT) LQ[(k / MX + 2) * S + (k % MX) + 2] += LN[k];
    __syncthreads();
    // transpose of the transverse increments: F = Fn - nu/2 (u+ Y(i-1) + u- Y(i)), G likewise
    if (transverse > 0) {
      for (int k = threadIdx.x; k < 2 * (MX + 2) * MX; k += NT) {
        if (k < (MX + 2) * MX) {  // adjoint of Y(c, j): used by x-edges (c+1, j) [u+] and (c, j) [u-]
          const int c = k % (MX + 2) - 1, j = k / (MX + 2);
          real l = 0;
          if (c + 1 <= MX) {
            const real s = uvel(c + 1, j);
            l -= hn * (s > real(0) ? s : real(0)) * LF[xe(c + 1, j)];
          }
          if (c >= 0) {
            const real s = uvel(c, j);
            l -= hn * (s < real(0) ? s : real(0)) * LF[xe(c, j)];
          }
          LY[k] = l;
        } else {  // adjoint of X(i, r): used by y-edges (i, r+1) [v+] and (i, r) [v-]
          const int f = k - (MX + 2) * MX;
          const int i = f % MX, r = f / MX - 1;
          real l = 0;
          if (r + 1 <= MX) {
            const real s = vvel(i, r + 1);
            l -= hn * (s > real(0) ? s : real(0)) * LG[ye(i, r + 1)];
          }
          if (r >= 0) {
            const real s = vvel(i, r);
            l -= hn * (s < real(0) ? s : real(0)) * LG[ye(i, r)];
          }
          LX[f] = l;
        }
      }
      // speed derivative of the transverse coefficients (their own edges' speeds)
      for (int k = threadIdx.x; k < 2 * MX * (MX + 1); k += NT) {
        if (k < MX * (MX + 1)) {
          const int i = k % (MX + 1), j = k / (MX + 1);
          const real s = uvel(i, j);
          const real yl = YS[j * (MX + 2) + i], yr = YS[j * (MX + 2) + i + 1];  // Y(i-1,j), Y(i,j)
          dsum -= hn * ((s > real(0) ? s : real(0)) * yl + (s < real(0) ? s : real(0)) * yr) *
                  LF[xe(i, j)];
        } else {
          const int f = k - MX * (MX + 1);
          const int i = f % MX, j = f / MX;
          const real s = vvel(i, j);
          const real xb = XS[j * MX + i], xt = XS[(j + 1) * MX + i];  // X(i,j-1), X(i,j)
          dsum -= hn * ((s > real(0) ? s : real(0)) * xb + (s < real(0) ? s : real(0)) * xt) *
                  LG[ye(i, j)];
        }
      }
    }
    __syncthreads();
    // transpose of every edge: x-edges (i, j), i in [0,MX], j in [-1,MX]
    for (int k = threadIdx.x; k < 2 * NE; k += NT) {
      const bool xdir = k < NE;
      int i, j;
      real s, lF, lP = 0, lM = 0;
      if (xdir) {
        i = k % (MX + 1);
        j = k / (MX + 1) - 1;
        s = uvel(i, j);
        lF = LF[k];
        if (transverse > 0) {
          if (i < MX) lP = LX[(j + 1) * MX + i];        // P enters cell (i, j): X(i, j)
          if (i > 0) lM = LX[(j + 1) * MX + i - 1];     // M enters cell (i-1, j): X(i-1, j)
        }
      } else {
        const int f = k - NE;
        i = f % (MX + 2) - 1;
        j = f / (MX + 2);
        s = vvel(i, j);
        lF = LG[f];
        if (transverse > 0) {
          if (j < MX) lP = LY[j * (MX + 2) + i + 1];      // P enters (i, j): Y(i, j)
          if (j > 0) lM = LY[(j - 1) * (MX + 2) + i + 1];  // M enters (i, j-1): Y(i, j-1)
        }
      }
      // cells a (behind b), b, c, d (beyond c) along the edge normal
      real qa, qb, qc, qd;
      real *la, *lb, *lc, *ld;
      if (xdir) {
        qa = q(i - 2, j); qb = q(i - 1, j); qc = q(i, j); qd = q(i + 1, j);
        la = lq(i - 2, j); lb = lq(i - 1, j); lc = lq(i, j); ld = lq(i + 1, j);
      } else {
        qa = q(i, j - 2); qb = q(i, j - 1); qc = q(i, j); qd = q(i, j + 1);
        la = lq(i, j - 2); lb = lq(i, j - 1); lc = lq(i, j); ld = lq(i, j + 1);
      }
      const EdgeFw<real> e = edge_fw(order, limiter, transverse, s, qa, qb, qc, qd, nu);
      const real sp = s > real(0) ? s : real(0), sm = s < real(0) ? s : real(0);
      const real ip = s > real(0) ? real(1) : real(0), im = s < real(0) ? real(1) : real(0);
      real lFt = lF, lW = 0, lWup = 0;
      real ds = 0;
      if (transverse > 0) {
        lW += sp * lP + sm * lM;
        ds += lP * ip * e.W + lM * im * e.W;
        if (transverse > 1) lFt += -lP + lM;
      }
      atomicAdd(lb, sp * lF);
      atomicAdd(lc, sm * lF);
      ds += lF * (ip * qb + im * qc);
      lW += e.c * e.dW * lFt;
      lWup += e.c * e.dWup * lFt;
      ds += lFt * e.dc * e.lim;
      atomicAdd(lc, lW);
      atomicAdd(lb, -lW);
      if (e.up) {
        atomicAdd(lb, lWup);
        atomicAdd(la, -lWup);
      } else {
        atomicAdd(ld, lWup);
        atomicAdd(lc, -lWup);
      }
      dsum += ds * s;
    }
    __syncthreads();
    // transpose of the second wall-BC pass
    if (D.domain == FC_DOMAIN_WALLS) {
      const int N = MX << pm.level;
      for (int k = threadIdx.x; k < num_ghosts<MX>(); k += NT) {
        int i, j;
        ghost_ij<MX>(k, i, j);
        const int gx = pm.x * MX + i, gy = pm.y * MX + j;
        const bool ox = gx < 0 || gx >= N, oy = gy < 0 || gy >= N;
        if (!ox && !oy) continue;
        const int ic = ox ? (gx < 0 ? 0 : MX - 1) : i;
        const int jc = oy ? (gy < 0 ? 0 : MX - 1) : j;
        atomicAdd(lq(ic, jc), *lq(i, j));
        *lq(i, j) = real(0);
      }
      __syncthreads();
    }
    real* lout = lam_out + (size_t)p * S * S;
    if (acc) {
      // the level's ghost fill reversed (its wall passes' transposes add
      // nothing once the exterior adjoint has moved to the clamped cells
      // above): interpolation from the coarse tiles, then copies / averages
      adj_interp_patch<real, MX>(D, st, pm, LQ, lam_out, g.tlevel, g.lamT, g.coarse_src,
                                 g.coarse_p0, threadIdx.x, NT);
      __syncthreads();
      adj_copy_patch<real, MX>(st, pm, LQ, AdjTargets<real>{lam_out, g.lam_fine, nullptr, nullptr},
                               g.tlevel, real(0), threadIdx.x, NT);
      __syncthreads();
      for (int k = threadIdx.x; k < MX * MX; k += NT) {
        const int o = (k / MX + 2) * S + (k % MX) + 2;
        atomicAdd(lout + o, LQ[o]);
      }
    } else {
      for (int k = threadIdx.x; k < S * S; k += NT) lout[k] = LQ[k];
    }
    __syncthreads();
  }
  // within warps by shuffles, then the warps' partial sums in FP64
  for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xffffffffu, dsum, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)dsum;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < NT / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) atomicAdd(dscale, v * dfac);
  }
}

// --------------------------------------------------------------- kernels

// global step: the whole transpose of Alg. 1 is split by phase over all
// patches (the phases scatter into other patches' ghost cells)
template <typename real, int MX>
__global__ void adj_interp_kernel(DevForest<real> D, const int* targets, int ntargets,
                                  real* lam) {
  constexpr int S = MX + 4;
  __shared__ NbrStage st;
  for (int t = blockIdx.x; t < ntargets; t += gridDim.x) {
    const int p = targets[t];
    stage_neighbours(D.meta, D.nbr, p, st, threadIdx.x);
    const PatchMeta pm = D.meta[p];
    __syncthreads();
    adj_interp_patch<real, MX>(D, st, pm, lam + (size_t)p * S * S, lam, -1, nullptr, nullptr, 0,
                               threadIdx.x, blockDim.x);
    __syncthreads();
  }
}

template <typename real, int MX>
__global__ void adj_bc_kernel(DevForest<real> D, real* lam) {
  constexpr int S = MX + 4;
  for (int p = blockIdx.x; p < D.npatch; p += gridDim.x)
    adj_bc_patch<real, MX>(D.meta[p], lam + (size_t)p * S * S, threadIdx.x, blockDim.x);
}

template <typename real, int MX>
__global__ void adj_copy_kernel(DevForest<real> D, real* lam) {
  constexpr int S = MX + 4;
  __shared__ NbrStage st;
  for (int p = blockIdx.x; p < D.npatch; p += gridDim.x) {
    stage_neighbours(D.meta, D.nbr, p, st, threadIdx.x);
    const PatchMeta pm = D.meta[p];
    __syncthreads();
    adj_copy_patch<real, MX>(st, pm, lam + (size_t)p * S * S,
                             AdjTargets<real>{lam, lam, nullptr, nullptr}, -1, real(0),
                             threadIdx.x, blockDim.x);
    __syncthreads();
  }
}

// multirate substep, the level L-1 patches read through the time-
// interpolated tiles (each listed once): the transposes of their ghosts
// (boundary condition, copy / average: same-size neighbours on level L-1
// split between the accumulators of its older and newer states, lam_old and
// lam_new; finer ones, on level L, into lam) and of the time interpolation
// of their interiors; their lamT tiles are cleared
template <typename real, int MX>
__global__ void adj_coarse_tiles_kernel(DevForest<real> D, const int* targets, int n, real* lam,
                                        real* lam_old, real* lam_new, int tlevel, real alpha,
                                        real* lamT) {
  constexpr int S = MX + 4;
  __shared__ NbrStage st;
  const bool walls = D.domain == FC_DOMAIN_WALLS;
  for (int t = blockIdx.x; t < n; t += gridDim.x) {
    const int p = targets[t];
    stage_neighbours(D.meta, D.nbr, p, st, threadIdx.x);
    const PatchMeta pm = D.meta[p];
    real* T = lamT + (size_t)p * S * S;
    __syncthreads();
    if (walls) {
      adj_bc_patch<real, MX>(pm, T, threadIdx.x, blockDim.x);
      __syncthreads();
    }
    adj_copy_patch<real, MX>(st, pm, T, AdjTargets<real>{lam, lam, lam_old, lam_new}, tlevel,
                             alpha, threadIdx.x, blockDim.x);
    __syncthreads();
    const size_t base = (size_t)p * S * S;
    // (the interpolation stencils of the finer level read only the cells
    // within two of the tile's edge, so most of the tile's adjoint is zero:
    // those cells add nothing and need no clearing)
    for (int k = threadIdx.x; k < S * S; k += blockDim.x) {
      const int i = k % S - 2, j = k / S - 2;
      const real v = T[k];
      if (v == real(0)) continue;
      T[k] = real(0);
      if (i >= 0 && i < MX && j >= 0 && j < MX) {  // other CTAs may add here too
        atomicAdd(lam_old + base + k, (real(1) - alpha) * v);
        if (alpha != real(0)) atomicAdd(lam_new + base + k, alpha * v);
      }
    }
    __syncthreads();
  }
}

template <typename real, int MX>
constexpr size_t adj_smem() {
  return sizeof(real) * (size_t)(2 * (MX + 4) * (MX + 4) + MX * MX + 2 * (MX + 1) * (MX + 2) +
                                 4 * (MX + 2) * MX + 4 * (MX + 3));
}

inline int grid_for(int n) { return n < 1 ? 1 : (n < 65535 * 8 ? n : 65535 * 8); }

// transpose of the update of level L's patches [p0, p1) over (t, t + dt)
template <typename real, int MX>
cudaError_t adj_advance_level(const DevForest<real>& D, int L, int p0, int p1, double t, double dt,
                              double period, double scale, double dfac, real* lam_in,
                              real* lam_out, double* dscale, cudaStream_t s,
                              const double* t0_dev = nullptr, const real* tiles = nullptr,
                              int tiles_p0 = 0, int acc = 0,
                              AdjGhosts<real> g = AdjGhosts<real>{}) {
  // a whole CTA per patch, 512 threads at mx = 32: two CTAs per SM hold a
  // finest level's patches in one wave while the coarser levels' reversed
  // substeps run beside it (1024 threads, one CTA per SM, measured slower
  // once the levels overlapped; 256 too)
  constexpr int NT = MX >= 16 ? 512 : 256;
  // set once per process; concurrent first calls both set it (idempotent)
  static std::atomic<bool> attr{false};
  constexpr size_t smem = adj_smem<real, MX>();
  if (!attr.load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(adj_advance_kernel<real, MX, NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr.store(true, std::memory_order_release);
  }
  if (p1 <= p0) return cudaSuccess;
  AdvArgs al{};
  al.h = ldexp(1.0, -L) / MX;
  al.nu = dt / al.h;
  al.period = period;
  al.t_half = t + 0.5 * dt;
  al.t_off = t + 0.5 * dt;  // with t0_dev: t is relative to the replayed step's start
  al.t0_dev = t0_dev;
  al.sfac = D.vel_kind == FC_VEL_SWIRL ? scale * sin(M_PI * al.h) / (M_PI * al.h) : 0.0;
  adj_advance_kernel<real, MX, NT><<<p1 - p0, NT, smem, s>>>(D, al, lam_in, lam_out, dscale, dfac,
                                                               p0, p1, tiles, tiles_p0, acc, g);
  ++launch_counter();
  return cudaGetLastError();
}

template <typename real, int MX>
cudaError_t adjoint_mx(const DevForest<real>& D, const AdjArgs& g, const real* lam_in,
                       real* lam_out, double* dscale, cudaStream_t s) {
  // one launch per level (per-level h and dt/h); all read the pre-step state
  for (int L = 0; L <= kMaxLevel; ++L) {
    cudaError_t e = adj_advance_level<real, MX>(D, L, g.lev_start[L], g.lev_start[L + 1], g.t,
                                                g.dt, g.period, g.scale, g.dscale_factor,
                                                const_cast<real*>(lam_in), lam_out, dscale, s);
    if (e != cudaSuccess) return e;
  }
  if (g.ncoarse > 0) {
    adj_interp_kernel<real, MX><<<grid_for(g.ncoarse), 128, 0, s>>>(D, g.coarse_list, g.ncoarse,
                                                                     lam_out);
    ++launch_counter();
  }
  if (D.domain == FC_DOMAIN_WALLS) {
    adj_bc_kernel<real, MX><<<grid_for(D.npatch), 128, 0, s>>>(D, lam_out);
    ++launch_counter();
  }
  adj_copy_kernel<real, MX><<<grid_for(D.npatch), 128, 0, s>>>(D, lam_out);
  ++launch_counter();
  return cudaGetLastError();
}

// adjoint of one multirate substep of level L (see launch_adjoint_substep)
template <typename real, int MX>
cudaError_t adjoint_sub_mx(const DevForest<real>& D, const AdjSubArgs& g, const AdjAcc<real>& c,
                           double* dscale, cudaStream_t s) {
  const int n = g.p1 - g.p0;
  if (n <= 0) return cudaSuccess;
  const real alpha = real(g.alpha);
  cudaError_t e = adj_advance_level<real, MX>(
      D, g.L, g.p0, g.p1, g.t, g.dt, g.period, g.scale, g.dscale_factor, c.lam_in, c.lam_out,
      dscale, s, g.t0_dev, static_cast<const real*>(g.tiles), g.tiles_p0, 1,
      AdjGhosts<real>{c.lam_fine, c.lamT, static_cast<const real*>(g.coarse), g.coarse_p0,
                      g.tlevel});
  if (e != cudaSuccess) return e;
  if (g.nt > 0) {
    adj_coarse_tiles_kernel<real, MX><<<grid_for(g.nt), 256, 0, s>>>(
        D, g.list_t, g.nt, c.lam_out, c.lam_old, c.lam_new, g.tlevel, alpha, c.lamT);
    ++launch_counter();
  }
  return cudaGetLastError();
}

}  // namespace

template <typename real>
cudaError_t launch_adjoint_substep(const DevForest<real>& D, const AdjSubArgs& g,
                                   const AdjAcc<real>& c, double* dscale, cudaStream_t s) {
  switch (D.mx) {
    case 8: return adjoint_sub_mx<real, 8>(D, g, c, dscale, s);
    case 16: return adjoint_sub_mx<real, 16>(D, g, c, dscale, s);
    case 32: return adjoint_sub_mx<real, 32>(D, g, c, dscale, s);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_adjoint_substep<float>(const DevForest<float>&, const AdjSubArgs&,
                                                   const AdjAcc<float>&, double*, cudaStream_t);
template cudaError_t launch_adjoint_substep<double>(const DevForest<double>&, const AdjSubArgs&,
                                                    const AdjAcc<double>&, double*, cudaStream_t);

template <typename real>
cudaError_t launch_adjoint_step(const DevForest<real>& D, const AdjArgs& g, const real* lam_in,
                                real* lam_out, double* dscale, cudaStream_t s) {
  switch (D.mx) {
    case 8: return adjoint_mx<real, 8>(D, g, lam_in, lam_out, dscale, s);
    case 16: return adjoint_mx<real, 16>(D, g, lam_in, lam_out, dscale, s);
    case 32: return adjoint_mx<real, 32>(D, g, lam_in, lam_out, dscale, s);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_adjoint_step<float>(const DevForest<float>&, const AdjArgs&,
                                                const float*, float*, double*, cudaStream_t);
template cudaError_t launch_adjoint_step<double>(const DevForest<double>&, const AdjArgs&,
                                                 const double*, double*, double*, cudaStream_t);

}  // namespace fc
