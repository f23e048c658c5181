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

// One edge's transpose: e is the forward edge at speed s between cells a, b,
// c, d along its normal (qb, qc the middle two); lF, lP, lM the adjoints of
// its normal flux and of the fluctuations it sends into c's and b's side.
// Returns the four cells' adjoint contributions and, in ds, the derivative
// with respect to the edge speed times the speed.
template <typename real>
struct EdgeAdj {
  real a, b, c, d, ds;
};

template <typename real>
__device__ __forceinline__ EdgeAdj<real> edge_transpose(const EdgeFw<real>& e, int transverse,
                                                       real s, real qb, real qc, real lF,
                                                       real lP, real lM) {
  const real sp = s > real(0) ? s : real(0), sm = s < real(0) ? s : real(0);
  const real ip = s > real(0) ? real(1) : real(0), im = s < real(0) ? real(1) : real(0);
  real lFt = lF, lW = 0, lWup = 0, ds = 0;
  if (transverse > 0) {
    lW += sp * lP + sm * lM;
    ds += lP * ip * e.W + lM * im * e.W;
    if (transverse > 1) lFt += -lP + lM;
  }
  EdgeAdj<real> o;
  o.b = sp * lF;
  o.c = sm * lF;
  ds += lF * (ip * qb + im * qc);
  lW += e.c * e.dW * lFt;
  lWup += e.c * e.dWup * lFt;
  ds += lFt * e.dc * e.lim;
  o.c += lW;
  o.b -= lW;
  o.a = real(0);
  o.d = real(0);
  if (e.up) {
    o.b += lWup;
    o.a = -lWup;
  } else {
    o.d = lWup;
    o.c -= lWup;
  }
  o.ds = ds * s;
  return o;
}

template <typename real>
__device__ __forceinline__ real pos(real s) { return s > real(0) ? s : real(0); }
template <typename real>
__device__ __forceinline__ real neg(real s) { return s < real(0) ? s : real(0); }

// Transpose of the update of one patch (its final fluxes, their transverse
// increments and every edge), as a row walk: thread tid's lane li owns
// column li of the band of R rows starting at r0 = (tid / MX) R and walks
// rows r0 - 1 .. r0 + R, recomputing the forward edges it needs from the
// tile Q (x-edge (li, j) and y-edge (li, j + 1) at row j), taking the
// neighbouring column's values by shuffles, and transposing the x-edges of
// rows [r0, r0 + R) and the y-edges of rows [r0, r0 + R) (band 0 also the
// x-edges of row -1, the last band those of row MX and its y-edges).  The
// contributions to a cell's adjoint gather in a four-row register window of
// the lane's column and reach LQ (zeroed) by one shared atomic add per cell
// and band; ghost columns take theirs directly.  The edges of column MX (x)
// and of ghost columns -1 and MX (y) are side_transpose's.  LN: adjoint of
// the new interior; XMe[j + 1]: forward M of x-edge (MX, j); YPm[j], YMm[j]:
// forward P, M of y-edge (-1, j).  Returns the lane's share of sum ds.
template <typename real, int MX, int R, class UV, class VV>
__device__ __forceinline__ real band_transpose(const real* Q, real* LQ, const real* LN,
                                               const real* XMe, const real* YPm, const real* YMm,
                                               int order, int limiter, int transverse, real nu,
                                               real hn, UV uvel, VV vvel, int tid) {
  constexpr int S = MX + 4;
  constexpr unsigned FULL = 0xffffffffu;
  const int li = tid % MX, r0 = (tid / MX) * R, r1 = r0 + R;
  const bool last = r1 == MX;
  auto q = [&](int i, int j) -> real { return Q[(j + kMbc) * S + i + kMbc]; };
  auto ln = [&](int j) -> real { return (j >= 0 && j < MX) ? LN[j * MX + li] : real(0); };
  auto flush = [&](int row, real v) {
    if (row >= -kMbc && row <= MX + 1) atomicAdd(&LQ[(row + kMbc) * S + li + kMbc], v);
  };
  real dsum = 0;
  real A0 = 0, A1 = 0, A2 = 0, A3 = 0;  // contributions to rows j-2 .. j+1
  real qa = q(li, r0 - 2), qb = q(li, r0 - 1), qc = q(li, r0), qd = 0;
  real ln_cur = ln(r0 - 1);
  real v_cur = r0 - 1 >= 0 ? vvel(li, r0 - 1) : real(0);
  real lGf_cur = r0 - 1 >= 0 ? nu * (ln_cur - ln(r0 - 2)) : real(0);
  real YP_prev = 0, X_prev = 0, lY_prev = 0;
  EdgeFw<real> ey{};  // forward y-edge (li, j)
#pragma unroll(R <= 8 ? R + 2 : 2)
  for (int it = 0; it < R + 2; ++it) {
    const int j = r0 - 1 + it;
    const bool xrow = (j >= r0 && j < r1) || j == -1 || (last && j == MX);
    const bool yrow = (j >= r0 && j < r1) || (last && j == MX);
    if (j + 2 <= MX + 1) qd = q(li, j + 2);
    // forward: x-edge (li, j), y-edge (li, j + 1)
    const real su = uvel(li, j);
    const EdgeFw<real> ex =
        edge_fw(order, limiter, transverse, su, q(li - 2, j), q(li - 1, j), qb, q(li + 1, j), nu);
    real vn = 0;
    EdgeFw<real> eyn{};
    if (j + 1 <= MX) {
      vn = vvel(li, j + 1);
      eyn = edge_fw(order, limiter, transverse, vn, qa, qb, qc, qd, nu);
    }
    // adjoints of the final fluxes and of the fluctuation sums
    const real ln_next = ln(j + 1);
    const real lGf_next = j + 1 <= MX ? nu * (ln_next - ln_cur) : real(0);  // y-edge (li, j+1)
    real ln_left = __shfl_up_sync(FULL, ln_cur, 1, MX);
    if (li == 0) ln_left = real(0);
    const bool frow = j >= 0 && j < MX;
    const real lFf = frow ? nu * (ln_cur - ln_left) : real(0);  // x-edge (li, j)
    real lFf_r = __shfl_down_sync(FULL, lFf, 1, MX);            // x-edge (li+1, j)
    real su_r = __shfl_down_sync(FULL, su, 1, MX);
    if (li == MX - 1) {
      lFf_r = frow ? -nu * ln_cur : real(0);
      su_r = uvel(MX, j);
    }
    const real lY = frow ? -hn * (pos(su_r) * lFf_r + neg(su) * lFf) : real(0);  // Y(li, j)
    const real lX = -hn * (pos(vn) * lGf_next + (j >= 0 ? neg(v_cur) * lGf_cur : real(0)));
    real lX_l = __shfl_up_sync(FULL, lX, 1, MX);  // X(li-1, j)
    if (li == 0) lX_l = real(0);
    // forward fluctuation sums X(li, j), Y(li, j), Y(li-1, j)
    real XM_r = __shfl_down_sync(FULL, ex.M, 1, MX);
    if (li == MX - 1) XM_r = XMe[j + 1];
    const real X = ex.P + XM_r;
    const real Y = YP_prev + eyn.M;
    real Y_l = __shfl_up_sync(FULL, Y, 1, MX);
    if (li == 0) Y_l = frow ? YPm[j] + YMm[j + 1] : real(0);
    // x-edge (li, j)
    EdgeAdj<real> ox =
        edge_transpose(ex, transverse, su, q(li - 1, j), qb, lFf, transverse > 0 ? lX : real(0),
                       transverse > 0 ? lX_l : real(0));
    if (!xrow) ox = EdgeAdj<real>{0, 0, 0, 0, 0};
    dsum += ox.ds;
    if (transverse > 0 && xrow && frow) dsum -= hn * (pos(su) * Y_l + neg(su) * Y) * lFf;
    real T = ox.c;
    {
      const real b1 = __shfl_down_sync(FULL, ox.b, 1, MX);
      const real a2 = __shfl_down_sync(FULL, ox.a, 2, MX);
      const real d1 = __shfl_up_sync(FULL, ox.d, 1, MX);
      if (li + 1 < MX) T += b1;
      if (li + 2 < MX) T += a2;
      if (li >= 1) T += d1;
    }
    if (xrow) {  // contributions to the ghost columns
      if (li == 0) {
        atomicAdd(&LQ[(j + kMbc) * S + 0], ox.a);
        atomicAdd(&LQ[(j + kMbc) * S + 1], ox.b);
      }
      if (li == 1) atomicAdd(&LQ[(j + kMbc) * S + 1], ox.a);
      if (li == MX - 1) atomicAdd(&LQ[(j + kMbc) * S + MX + kMbc], ox.d);
    }
    // y-edge (li, j)
    if (yrow) {
      const EdgeAdj<real> oy =
          edge_transpose(ey, transverse, v_cur, qa, qb, lGf_cur,
                         transverse > 0 && j < MX ? lY : real(0),
                         transverse > 0 && j > 0 ? lY_prev : real(0));
      dsum += oy.ds;
      if (transverse > 0) dsum -= hn * (pos(v_cur) * X_prev + neg(v_cur) * X) * lGf_cur;
      A0 += oy.a;
      A1 += oy.b;
      A2 += oy.c;
      A3 += oy.d;
    }
    A2 += T;
    if (j >= r0 && j < r1) A2 += ln_cur;  // the update's identity part
    flush(j - 2, A0);
    A0 = A1;
    A1 = A2;
    A2 = A3;
    A3 = real(0);
    X_prev = X;
    lY_prev = lY;
    ey = eyn;
    YP_prev = eyn.P;
    v_cur = vn;
    lGf_cur = lGf_next;
    ln_cur = ln_next;
    qa = qb;
    qb = qc;
    qc = qd;
  }
  const int jl = r0 + R;  // the last row walked
  flush(jl - 1, A0);
  flush(jl, A1);
  flush(jl + 1, A2);
  return dsum;
}

// The edges band_transpose leaves: x-edge (MX, j), j in [-1, MX], and the
// y-edges of ghost columns -1 and MX, j in [0, MX] (threads tid, stride
// nt, one edge each, contributions by shared atomic adds).  Returns the
// threads' share of sum ds.
template <typename real, int MX, class UV, class VV>
__device__ __forceinline__ real side_transpose(const real* Q, real* LQ, const real* LN, int order,
                                               int limiter, int transverse, real nu, real hn,
                                               UV uvel, VV vvel, int tid, int nt) {
  constexpr int S = MX + 4;
  auto q = [&](int i, int j) -> real { return Q[(j + kMbc) * S + i + kMbc]; };
  auto ln = [&](int i, int j) -> real {
    return (i >= 0 && i < MX && j >= 0 && j < MX) ? LN[j * MX + i] : real(0);
  };
  auto add = [&](int i, int j, real v) { atomicAdd(&LQ[(j + kMbc) * S + i + kMbc], v); };
  // adjoints of the final fluxes of x-edge (i, j) and y-edge (i, j)
  auto lFf = [&](int i, int j) -> real {
    return (j >= 0 && j < MX) ? nu * (ln(i, j) - ln(i - 1, j)) : real(0);
  };
  auto lGf = [&](int i, int j) -> real {
    return (i >= 0 && i < MX && j >= 0 && j <= MX) ? nu * (ln(i, j) - ln(i, j - 1)) : real(0);
  };
  auto yedge = [&](int c, int j) {
    return edge_fw(order, limiter, transverse, vvel(c, j), q(c, j - 2), q(c, j - 1), q(c, j),
                   q(c, j + 1), nu);
  };
  real dsum = 0;
  for (int k = tid; k < 3 * MX + 4; k += nt) {
    if (k < MX + 2) {  // x-edge (MX, j): its P enters no updated cell; M enters (MX-1, j)
      const int j = k - 1;
      const real s = uvel(MX, j);
      const EdgeFw<real> e = edge_fw(order, limiter, transverse, s, q(MX - 2, j), q(MX - 1, j),
                                     q(MX, j), q(MX + 1, j), nu);
      const real lF = lFf(MX, j);
      real lM = 0;
      if (transverse > 0)
        lM = -hn * ((j + 1 <= MX ? pos(vvel(MX - 1, j + 1)) * lGf(MX - 1, j + 1) : real(0)) +
                    (j >= 0 ? neg(vvel(MX - 1, j)) * lGf(MX - 1, j) : real(0)));
      const EdgeAdj<real> o = edge_transpose(e, transverse, s, q(MX - 1, j), q(MX, j), lF,
                                             real(0), lM);
      add(MX - 2, j, o.a);
      add(MX - 1, j, o.b);
      add(MX, j, o.c);
      add(MX + 1, j, o.d);
      dsum += o.ds;
      if (transverse > 0 && j >= 0 && j < MX) {  // its transverse increment's speed
        const real Yl = yedge(MX - 1, j).P + yedge(MX - 1, j + 1).M;
        const real Yr = yedge(MX, j).P + yedge(MX, j + 1).M;
        dsum -= hn * (pos(s) * Yl + neg(s) * Yr) * lF;
      }
    } else {  // y-edge (c, j) of ghost column c = -1 or MX (no flux of its own updates a cell)
      const bool right = k >= 2 * MX + 3;
      const int j = k - (right ? 2 * MX + 3 : MX + 2);
      const int c = right ? MX : -1;
      const real s = vvel(c, j);
      const EdgeFw<real> e = yedge(c, j);
      // adjoint of Y(c, r): from x-edge (0, r)'s u+ (c = -1) or (MX, r)'s u- (c = MX)
      auto lY = [&](int r) -> real {
        if (r < 0 || r >= MX) return real(0);
        return right ? -hn * neg(uvel(MX, r)) * lFf(MX, r) : -hn * pos(uvel(0, r)) * lFf(0, r);
      };
      const real lP = transverse > 0 ? lY(j) : real(0);
      const real lM = transverse > 0 ? lY(j - 1) : real(0);
      const EdgeAdj<real> o =
          edge_transpose(e, transverse, s, q(c, j - 1), q(c, j), real(0), lP, lM);
      add(c, j - 2, o.a);
      add(c, j - 1, o.b);
      add(c, j, o.c);
      add(c, j + 1, o.d);
      dsum += o.ds;
    }
  }
  return dsum;
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
// (FP32 at mx = 32: two CTAs of 384 threads per SM, so a finest level's
// patches run in one wave)
template <typename real, int MX, int R, int NT, int NS>
__global__ void __launch_bounds__(NT, sizeof(real) == 4 && NT >= 384 ? 2 : 1)
    adj_advance_kernel(DevForest<real> D, AdvArgs a,
                                                         real* lam_in, real* lam_out,
                                                         double* dscale, double dfac, int p0,
                                                         int p1, const real* tiles, int tiles_p0,
                                                         int acc, AdjGhosts<real> g) {
  constexpr int S = MX + 4;
  constexpr int NV = MX + 3;
  constexpr int NW = MX * MX / R;  // threads that walk a band of R rows; NS more take the side edges
  static_assert(MX % R == 0 && NW + NS == NT && NW % 32 == 0 && NS % 32 == 0,
                "bands of R rows and the side edges, whole warps");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real* Q = reinterpret_cast<real*>(smem_raw);
  real* LQ = Q + S * S;       // adjoint of the input tile
  real* LN = LQ + S * S;      // adjoint of the new interior (MX*MX)
  real* XMe = LN + MX * MX;   // forward M of x-edge (MX, j) at [j + 1]
  real* YPm = XMe + MX + 2;   // forward P, M of y-edge (-1, j)
  real* YMm = YPm + MX + 1;
  real* Sx = YMm + MX + 1;
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
  // the swirl coefficient, by the last thread while the first patch's data
  // load (graph replay: the time is on the device); read after the barrier
  if (threadIdx.x == NT - 1 && swirl) {
    const double t = a.t0_dev ? *a.t0_dev + a.t_off : a.t_half;
    ucoef_s = cospi_ratio<real>(t, a.period) * real(a.sfac);
  }
  real ucoef = real(0);
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
    // every load of a thread is issued before any is used
    constexpr int NQ = (S * S + NT - 1) / NT, NL = (MX * MX + NT - 1) / NT;
    real vq[NQ], vl[NL];
#pragma unroll
    for (int u = 0; u < NQ; ++u) {
      const int k = (int)threadIdx.x + u * NT;
      vq[u] = k < S * S ? src[k] : real(0);
    }
#pragma unroll
    for (int u = 0; u < NL; ++u) {
      const int k = (int)threadIdx.x + u * NT;
      vl[u] = k < MX * MX ? lin[(k / MX + 2) * S + (k % MX) + 2] : real(0);
    }
    if (swirl)  // the tables, one entry a thread
      for (int k = threadIdx.x; k < 4 * NV; k += NT) {
        const int tb = k / NV, c = k % NV;
        const int z = (tb & 1 ? pm.y : pm.x) * MX + c - 1;
        real v;
        if (tb < 2) {
          v = sinpi_r(real(z) * h);
          v *= v;
        } else {
          v = sinpi_r(real(2 * z + 1) * h);
        }
        (tb == 0 ? Sx : tb == 1 ? Sy : tb == 2 ? Tx : Ty)[c] = v;
      }
#pragma unroll
    for (int u = 0; u < NQ; ++u) {
      const int k = (int)threadIdx.x + u * NT;
      if (k < S * S) {
        Q[k] = vq[u];
        LQ[k] = real(0);
      }
    }
#pragma unroll
    for (int u = 0; u < NL; ++u) {
      const int k = (int)threadIdx.x + u * NT;
      if (k < MX * MX) {
        LN[k] = vl[u];
        if (acc) lin[(k / MX + 2) * S + (k % MX) + 2] = real(0);  // consumed: next state from zero
      }
    }
    __syncthreads();
    ucoef = swirl ? ucoef_s : real(0);
    auto q = [&](int i, int j) -> real { return Q[(j + 2) * S + (i + 2)]; };
    auto lq = [&](int i, int j) -> real* { return &LQ[(j + 2) * S + (i + 2)]; };
    auto uvel = [&](int i, int j) -> real { return swirl ? ucoef * Sx[i + 1] * Ty[j + 1] : cu; };
    auto vvel = [&](int i, int j) -> real { return swirl ? -ucoef * Sy[j + 1] * Tx[i + 1] : cv; };
    // the side quantities the band walk reads, then the walk (rows of
    // bands) and the edges beside it (columns MX and -1)
    for (int k = threadIdx.x; k < 2 * MX + 3; k += NT) {
      if (k < MX + 2) {
        const int j = k - 1;
        XMe[k] = edge_fw(order, limiter, transverse, uvel(MX, j), q(MX - 2, j), q(MX - 1, j),
                         q(MX, j), q(MX + 1, j), nu)
                     .M;
      } else {
        const int j = k - (MX + 2);
        const EdgeFw<real> e = edge_fw(order, limiter, transverse, vvel(-1, j), q(-1, j - 2),
                                       q(-1, j - 1), q(-1, j), q(-1, j + 1), nu);
        YPm[j] = e.P;
        YMm[j] = e.M;
      }
    }
    __syncthreads();
    if (threadIdx.x < NW)
      dsum += band_transpose<real, MX, R>(Q, LQ, LN, XMe, YPm, YMm, order, limiter, transverse, nu,
                                          hn, uvel, vvel, threadIdx.x);
    else
      dsum += side_transpose<real, MX>(Q, LQ, LN, order, limiter, transverse, nu, hn, uvel, vvel,
                                       threadIdx.x - NW, NS);
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
__global__ void __launch_bounds__(256) adj_coarse_tiles_kernel(DevForest<real> D,
                                                               const int* targets, int n,
                                                               real* lam, real* lam_old,
                                                               real* lam_new, int tlevel,
                                                               real alpha, real* lamT) {
  constexpr int S = MX + 4, NT = 256, NQ = (S * S + NT - 1) / NT;
  __shared__ NbrStage st;
  __shared__ real L[S * S];  // the tile's adjoint, staged
  const bool walls = D.domain == FC_DOMAIN_WALLS;
  const int tid = threadIdx.x;
  for (int t = blockIdx.x; t < n; t += gridDim.x) {
    const int p = targets[t];
    stage_neighbours(D.meta, D.nbr, p, st, tid);
    const PatchMeta pm = D.meta[p];
    real* T = lamT + (size_t)p * S * S;
    // the whole tile in (every load issued before any is used); it is left
    // cleared for its next use (the interpolation stencils of the finer
    // level read only the cells within two of the tile's edge, so most of
    // it is zero and needs no store)
    real v[NQ];
#pragma unroll
    for (int u = 0; u < NQ; ++u) {
      const int k = tid + u * NT;
      v[u] = k < S * S ? T[k] : real(0);
    }
#pragma unroll
    for (int u = 0; u < NQ; ++u) {
      const int k = tid + u * NT;
      if (k < S * S) {
        L[k] = v[u];
        if (v[u] != real(0)) T[k] = real(0);
      }
    }
    __syncthreads();
    if (walls) {
      adj_bc_patch<real, MX>(pm, L, tid, NT);
      __syncthreads();
    }
    adj_copy_patch<real, MX>(st, pm, L, AdjTargets<real>{lam, lam, lam_old, lam_new}, tlevel,
                             alpha, tid, NT);
    __syncthreads();
    const size_t base = (size_t)p * S * S;
    for (int k = tid; k < MX * MX; k += NT) {  // other CTAs may add here too
      const int o = (k / MX + kMbc) * S + k % MX + kMbc;
      const real w = L[o];
      if (w == real(0)) continue;
      atomicAdd(lam_old + base + o, (real(1) - alpha) * w);
      if (alpha != real(0)) atomicAdd(lam_new + base + o, alpha * w);
    }
    __syncthreads();
  }
}

template <typename real, int MX>
constexpr size_t adj_smem() {
  return sizeof(real) * (size_t)(2 * (MX + 4) * (MX + 4) + MX * MX + 3 * MX + 4 + 4 * (MX + 3));
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
  // a whole CTA per patch whose warps walk bands of R rows (4 at mx = 32,
  // 2 below) while more warps transpose the side edges
  constexpr int R = MX == 32 ? 4 : 2;
  constexpr int NS = (3 * MX + 4 + 31) / 32 * 32;  // a thread per side edge
  constexpr int NT = MX * MX / R + NS;
  // set once per process; concurrent first calls both set it (idempotent)
  static std::atomic<bool> attr{false};
  constexpr size_t smem = adj_smem<real, MX>();
  if (!attr.load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(adj_advance_kernel<real, MX, R, NT, NS>,
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
  adj_advance_kernel<real, MX, R, NT, NS><<<p1 - p0, NT, smem, s>>>(
      D, al, lam_in, lam_out, dscale, dfac, p0, p1, tiles, tiles_p0, acc, g);
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
