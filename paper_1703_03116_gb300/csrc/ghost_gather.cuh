// Ghost-cell rules of Alg. 1 (Sec. 2.3), shared by the standalone fill
// kernels (which write the ghost ring of a patch array in HBM) and by the
// patch-update kernels (which fill the ghost ring of the tile they hold in
// shared memory before computing).
//
//  copy     (same-size neighbour):  q_c(I_c) = q_n(A I_c + F)      Eq. transform
//  average  (finer neighbour):      q_c(I_c) = 1/4 sum_k q_f(I_f^k) Eq. ghost_coarse
//  interp.  (coarser neighbour):    q_f = q_c + 1/4 (s_x d_x + s_y d_y),
//           s = minmod of the one-sided differences in the coarse index
//           space                                                   Eq. ghost_fine
//  walls    zeroth-order extrapolation: an exterior ghost copies the owner's
//           cell with each out-of-domain index clamped into the interior.
#pragma once

#include "device_util.cuh"

namespace fc {

// the eight face/corner entries of one patch and the layout of their patches
struct NbrStage {
  NbrEntry e[8];
  PatchMeta m0[8], m1[8];
};

// threads tid = 0..7 of a cooperating group stage the entries of patch p
// (the neighbours' level and coordinates travel in the entries: one read)
__device__ __forceinline__ void stage_neighbours(const PatchMeta* meta, const NbrEntry* nbr,
                                                 int p, NbrStage& st, int tid) {
  (void)meta;
  if (tid < 8) {
    const NbrEntry e = nbr[(size_t)p * 8 + tid];
    st.e[tid] = e;
    st.m0[tid] = PatchMeta{e.lev, e.x0, e.y0, 0, 0, 0};
    st.m1[tid] = PatchMeta{e.lev, e.x1, e.y1, 0, 0, 0};
  }
}

// interior cell (i, j) of source patch n (level nlev), time-interpolated when
// n lies on the level read through the interpolation buffer
template <typename real>
__device__ __forceinline__ real src_interior(const DevForest<real>& D, int tlevel, real alpha,
                                             int n, int nlev, int i, int j) {
  const size_t o = (size_t)n * D.S * D.S + (size_t)(j + kMbc) * D.S + (i + kMbc);
  const int c = D.cur[nlev];
  if (nlev == tlevel) {
    // alpha = 0 reads the older state alone: the newer one may still be
    // being written (the fill can run beside the update that makes it)
    if (alpha == real(0)) return D.buf[c ^ 1][o];
    return (real(1) - alpha) * D.buf[c ^ 1][o] + alpha * D.buf[c][o];
  }
  return D.buf[c][o];
}

// Ghost (i, j) of the owner (layout pm) from a same-size or finer neighbour,
// e being the entry of the ghost's face/corner region (the neighbours' level
// and positions travel in it).  Returns false when the region is not of
// that kind (or the entry is malformed).
template <typename real, int MX>
__device__ __forceinline__ bool copy_or_average_entry(const DevForest<real>& D, const NbrEntry& e,
                                                      const PatchMeta& pm, int tlevel, real alpha,
                                                      int i, int j, real& v) {
  if (e.kind != NB_SAME && e.kind != NB_FINE) return false;
  const int2 Ip = apply_a(e.a, pm.x * MX + i, pm.y * MX + j);
  const int gx = Ip.x + e.fx, gy = Ip.y + e.fy;
  if (e.kind == NB_SAME) {
    const int lx = gx - e.x0 * MX, ly = gy - e.y0 * MX;
    if (lx < 0 || lx >= MX || ly < 0 || ly >= MX) return false;
    v = src_interior(D, tlevel, alpha, e.n0, e.lev, lx, ly);
    return true;
  }
  int n = e.n0;
  int lx = 2 * gx - e.x0 * MX, ly = 2 * gy - e.y0 * MX;
  if (lx < 0 || lx >= MX || ly < 0 || ly >= MX) {
    if (e.n1 < 0) return false;
    n = e.n1;
    lx = 2 * gx - e.x1 * MX;
    ly = 2 * gy - e.y1 * MX;
    if (lx < 0 || lx >= MX || ly < 0 || ly >= MX) return false;
  }
  // the four fine cells, in the neighbour's frame: (0,0), (1,0), (0,1), (1,1)
  real s[4];
#pragma unroll
  for (int q = 0; q < 4; ++q)
    s[q] = src_interior(D, tlevel, alpha, n, e.lev, lx + (q & 1), ly + (q >> 1));
  if (D.metric) {  // mapped grid: weighted by the fine cells' areas
    const double* K = D.metric + (size_t)n * metric_stride(D.S) + (ly + kMbc) * D.S + lx + kMbc;
    const double k0 = K[0], k1 = K[1], k2 = K[D.S], k3 = K[D.S + 1];
    v = real((((k0 * double(s[0]) + k1 * double(s[1])) + k2 * double(s[2])) + k3 * double(s[3])) /
             (((k0 + k1) + k2) + k3));
    return true;
  }
  v = real(0.25) * (((s[0] + s[1]) + s[2]) + s[3]);
  return true;
}

// the same from the owner's staged entries
template <typename real, int MX>
__device__ __forceinline__ bool copy_or_average(const DevForest<real>& D, const NbrStage& st,
                                                const PatchMeta& pm, int tlevel, real alpha,
                                                int i, int j, real& v) {
  return copy_or_average_entry<real, MX>(D, st.e[region_of<MX>(i, j)], pm, tlevel, alpha, i, j,
                                         v);
}

// Ghost (i, j) of the owner from its coarser neighbour (e: the entry of the
// ghost's region); the coarse patch is read through the interpolation buffer
// when it lies on `tlevel`.
template <typename real, int MX>
__device__ __forceinline__ bool interpolate_entry(const DevForest<real>& D, const NbrEntry& e,
                                                  const PatchMeta& pm, int tlevel, int i, int j,
                                                  real& v) {
  constexpr int S = MX + 4;
  if (e.kind != NB_COARSE) return false;
  const int2 Ip = apply_a(e.a, pm.x * MX + i, pm.y * MX + j);
  const int gx = Ip.x + e.fx, gy = Ip.y + e.fy;
  const int ic = (gx >> 1) - e.x0 * MX, jc = (gy >> 1) - e.y0 * MX;
  if (ic < 0 || ic >= MX || jc < 0 || jc >= MX) return false;
  const real dx = (gx & 1) ? real(1) : real(-1);
  const real dy = (gy & 1) ? real(1) : real(-1);
  const real* C = patch_ptr(e.lev == tlevel ? D.qT : D.buf[D.cur[e.lev]], e.n0, S) +
                  (jc + kMbc) * S + ic + kMbc;
  const real q0 = C[0];
  const real sx = minmod(C[1] - q0, q0 - C[-1]);
  const real sy = minmod(C[S] - q0, q0 - C[-S]);
  v = q0 + real(0.25) * (sx * dx + sy * dy);
  return true;
}

// the same from the owner's staged entries
template <typename real, int MX>
__device__ __forceinline__ bool interpolate(const DevForest<real>& D, const NbrStage& st,
                                            const PatchMeta& pm, int tlevel, int i, int j,
                                            real& v) {
  return interpolate_entry<real, MX>(D, st.e[region_of<MX>(i, j)], pm, tlevel, i, j, v);
}

// The value the coarse-neighbour fill of a multirate substep (phases 1-2 at
// tlevel and alpha, then the wall condition) leaves in cell (i, j) of the
// time-interpolated tile of patch c (on tlevel; cm: its level and
// position): the interior (1 - alpha) q_old + alpha q_new, ghosts copied
// from same-size or averaged from finer neighbours, exterior ghosts from the
// cell the wall condition clamps them to; any other ghost keeps what the
// tile holds (that fill leaves it alone).  An update that computes the few
// coarse cells its interpolation reads this way needs no fill launch before
// it.  The interpolation's stencil is centred in c's interior, so it reads
// c's face ghosts at most, never the corners (on the cubed sphere, the
// corners beyond a cube vertex are the only ghosts that fill computes from
// other ghosts).
//
// Split in two: coarse_cell_interior applies the wall condition's clamp and
// says whether the cell is interior (then src_interior reads it); a ghost
// of c is coarse_ghost, which reads c's entry for its region from the table
// itself, so only the stencils that leave c's interior wait for that read.
template <typename real, int MX>
__device__ __forceinline__ bool coarse_cell_interior(const DevForest<real>& D,
                                                     const PatchMeta& cm, int& i, int& j) {
  if (D.domain == FC_DOMAIN_WALLS) {
    const int N = MX << cm.level;
    const int gx = cm.x * MX + i, gy = cm.y * MX + j;
    const bool ox = gx < 0 || gx >= N, oy = gy < 0 || gy >= N;
    if (ox) i = gx < 0 ? 0 : MX - 1;
    if (oy) j = gy < 0 ? 0 : MX - 1;
  }
  return i >= 0 && i < MX && j >= 0 && j < MX;
}

template <typename real, int MX>
__device__ __forceinline__ real coarse_ghost(const DevForest<real>& D, const PatchMeta& cm, int c,
                                             int tlevel, real alpha, int i, int j) {
  constexpr int S = MX + 4;
  real v;
  const NbrEntry e = D.nbr[(size_t)c * 8 + region_of<MX>(i, j)];
  if (copy_or_average_entry<real, MX>(D, e, cm, tlevel, alpha, i, j, v)) return v;
  return D.qT[(size_t)c * S * S + (j + kMbc) * S + i + kMbc];
}

// The value the coarse-neighbour fill gives ghost (ci, cj) of patch c by a
// rule of NbrEntry::code (1 copy of cell (lx, ly) of patch n, on tlevel; 2
// average of the 2 x 2 block at (lx, ly) of patch n, one level finer than
// tlevel, area-weighted on a mapped grid; 3 the tile's value): the
// arithmetic of copy_or_average_entry and coarse_ghost.
template <typename real, int MX>
__device__ __forceinline__ real fill_rule(const DevForest<real>& D, int tlevel, real alpha,
                                          int rule, int n, int lx, int ly, int c, int ci,
                                          int cj) {
  constexpr int S = MX + 4;
  if (rule == 1) return src_interior(D, tlevel, alpha, n, tlevel, lx, ly);
  if (rule == 3) return D.qT[(size_t)c * S * S + (cj + kMbc) * S + ci + kMbc];
  real s[4];
#pragma unroll
  for (int q = 0; q < 4; ++q)
    s[q] = src_interior(D, tlevel, alpha, n, tlevel + 1, lx + (q & 1), ly + (q >> 1));
  if (D.metric) {
    const double* K = D.metric + (size_t)n * metric_stride(D.S) + (ly + kMbc) * D.S + lx + kMbc;
    const double k0 = K[0], k1 = K[1], k2 = K[D.S], k3 = K[D.S + 1];
    return real((((k0 * double(s[0]) + k1 * double(s[1])) + k2 * double(s[2])) +
                 k3 * double(s[3])) /
                (((k0 + k1) + k2) + k3));
  }
  return real(0.25) * (((s[0] + s[1]) + s[2]) + s[3]);
}

// Ghost (ci, cj) of coarse neighbour c (entry e of the owner p's region r,
// ghost (i, j) of the owner) as the coarse-neighbour fill leaves it, from
// the sources listed in the region's entry (NbrEntry::src, code): one of the
// two listed ghosts, or the block of the owner's cells beside the ghost's
// coarse cell (region r a face, the list complete), else from c's own entry
// (coarse_ghost).  Only that last case waits on a read of c's table.
template <typename real, int MX>
__device__ __forceinline__ real coarse_ghost_at(const DevForest<real>& D, const NbrEntry& e,
                                                const PatchMeta& cm, int p, int tlevel,
                                                real alpha, int i, int j, int ci, int cj) {
  const int key = (ci + 1) | ((cj + 1) << 6);
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int code = e.code[q], rule = (code >> 24) & 3;
    if (rule && (code & 0xFFF) == key)
      return fill_rule<real, MX>(D, tlevel, alpha, rule, e.src[q], (code >> 12) & 63,
                                 (code >> 18) & 63, e.n0, ci, cj);
  }
  const int r = region_of<MX>(i, j);
  if ((e.code[0] & kSrcComplete) && r < 4) {
    const int bi = r == 0 ? 0 : r == 1 ? MX - 2 : (i & ~1);
    const int bj = r == 2 ? 0 : r == 3 ? MX - 2 : (j & ~1);
    return fill_rule<real, MX>(D, tlevel, alpha, 2, p, bi, bj, e.n0, ci, cj);
  }
  return coarse_ghost<real, MX>(D, cm, e.n0, tlevel, alpha, ci, cj);
}

// interpolate_entry(), reading a coarse neighbour on tlevel through the
// cells the coarse-neighbour fill would leave (above): the stencil's
// interior cells, then any ghost of the coarse patch from the sources the
// region's entry lists (coarse_ghost_at), all issued before any is used (the
// same values in any order); p is the owner.  keep_t non-null: each stencil cell
// is also stored where that fill would have left it in the coarse patch's
// tile at keep_t + (patch - keep_t_p0) tiles (the adjoint's replay keeps
// what the interpolation read; several writers store the same value)
template <typename real, int MX>
__device__ __forceinline__ bool interpolate_direct_entry(const DevForest<real>& D,
                                                         const NbrEntry& e, const PatchMeta& pm,
                                                         int tlevel, real alpha, int i, int j,
                                                         real& v, int p,
                                                         real* keep_t = nullptr,
                                                         int keep_t_p0 = 0) {
  if (e.kind != NB_COARSE) return false;
  if (e.lev != tlevel) return interpolate_entry<real, MX>(D, e, pm, tlevel, i, j, v);
  const int2 Ip = apply_a(e.a, pm.x * MX + i, pm.y * MX + j);
  const int gx = Ip.x + e.fx, gy = Ip.y + e.fy;
  const int ic = (gx >> 1) - e.x0 * MX, jc = (gy >> 1) - e.y0 * MX;
  if (ic < 0 || ic >= MX || jc < 0 || jc >= MX) return false;
  const real dx = (gx & 1) ? real(1) : real(-1);
  const real dy = (gy & 1) ? real(1) : real(-1);
  const PatchMeta cm{e.lev, e.x0, e.y0, 0, 0, 0};
  // stencil cells (0,0), (+1,0), (-1,0), (0,+1), (0,-1)
  int ci[5], cj[5];
  bool in[5];
  real c[5];
#pragma unroll
  for (int m = 0; m < 5; ++m) {
    ci[m] = ic + (m == 1 ? 1 : m == 2 ? -1 : 0);
    cj[m] = jc + (m == 3 ? 1 : m == 4 ? -1 : 0);
    in[m] = coarse_cell_interior<real, MX>(D, cm, ci[m], cj[m]);
    c[m] = in[m] ? src_interior(D, tlevel, alpha, e.n0, e.lev, ci[m], cj[m]) : real(0);
  }
#pragma unroll
  for (int m = 0; m < 5; ++m)
    if (!in[m])
      c[m] = coarse_ghost_at<real, MX>(D, e, cm, p, tlevel, alpha, i, j, ci[m], cj[m]);
  if (keep_t) {
    constexpr int S = MX + 4;
    real* K = keep_t + (size_t)(e.n0 - keep_t_p0) * S * S;
#pragma unroll
    for (int m = 0; m < 5; ++m) {  // at the cell's own place (an exterior one unclamped)
      const int oi = ic + (m == 1 ? 1 : m == 2 ? -1 : 0), oj = jc + (m == 3 ? 1 : m == 4 ? -1 : 0);
      K[(oj + kMbc) * S + oi + kMbc] = c[m];
    }
  }
  const real q0 = c[0];
  const real sx = minmod(c[1] - q0, q0 - c[2]);
  const real sy = minmod(c[3] - q0, q0 - c[4]);
  v = q0 + real(0.25) * (sx * dx + sy * dy);
  return true;
}

// the same from the owner's staged entries
template <typename real, int MX>
__device__ __forceinline__ bool interpolate_direct(const DevForest<real>& D, const NbrStage& st,
                                                   const PatchMeta& pm, int p, int tlevel,
                                                   real alpha, int i, int j, real& v) {
  return interpolate_direct_entry<real, MX>(D, st.e[region_of<MX>(i, j)], pm, tlevel, alpha, i,
                                            j, v, p);
}

// The neighbour reads of Alg. 1 for one patch (its copy/average and
// interpolation rules), made while the patch's own tile is still in flight:
// slot k of ring / ring_w gets ghost k's value and whether a rule set it (an
// exterior ghost is left to the wall condition).  entry_of(r) gives the
// entry of face/corner region r (staged in shared memory, or read from the
// table) of patch p.  Threads tid, stride nt.  direct: coarse neighbours on
// tlevel are read through the cells their fill would leave
// (interpolate_direct_entry; keep_t, keep_t_p0: where it also stores them).
template <typename real, int MX, class EntryOf>
__device__ __forceinline__ void gather_ring(const DevForest<real>& D, EntryOf entry_of, int p,
                                            const PatchMeta& pm, int tlevel, real alpha,
                                            bool direct, real* ring, bool* ring_w, int tid,
                                            int nt, real* keep_t = nullptr,
                                            int keep_t_p0 = 0) {
#pragma unroll 1
  for (int k = tid; k < num_ghosts<MX>(); k += nt) {
    int i, j;
    ghost_ij<MX>(k, i, j);
    const NbrEntry e = entry_of(region_of<MX>(i, j));
    real v;
    const bool w =
        copy_or_average_entry<real, MX>(D, e, pm, tlevel, alpha, i, j, v) ||
        (direct ? interpolate_direct_entry<real, MX>(D, e, pm, tlevel, alpha, i, j, v, p,
                                                     keep_t, keep_t_p0)
                : interpolate_entry<real, MX>(D, e, pm, tlevel, i, j, v));
    ring[k] = w ? v : real(0);
    ring_w[k] = w;
  }
}

// the gathered ghosts into the landed tile Q (each thread its own slots)
template <typename real, int MX>
__device__ __forceinline__ void store_ring(real* Q, const real* ring, const bool* ring_w, int tid,
                                           int nt) {
  constexpr int S = MX + 4;
  for (int k = tid; k < num_ghosts<MX>(); k += nt)
    if (ring_w[k]) {
      int i, j;
      ghost_ij<MX>(k, i, j);
      Q[(j + kMbc) * S + i + kMbc] = ring[k];
    }
}

// walls: exterior ghosts of the owner's array Q (threads tid, stride nt)
template <typename real, int MX>
__device__ __forceinline__ void wall_bc(const PatchMeta& pm, real* Q, int tid, int nt) {
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
    Q[(j + kMbc) * S + i + kMbc] = Q[(jc + kMbc) * S + ic + kMbc];
  }
}

// Cubed sphere, corner regions beyond a cube vertex (no block holds them; a
// stated reading of Sec. 2.4): each of the 2 x 2 corner ghosts takes the mean
// of the two edge ghosts in its row and column next to the patch, once the
// edge ghosts are final.  Threads tid, stride nt.
template <typename real, int MX, class KindOf>
__device__ __forceinline__ void corner3_fill_k(KindOf kind_of, real* Q, int tid, int nt) {
  constexpr int S = MX + 4;
  for (int k = tid; k < 16; k += nt) {
    const int r = 4 + (k >> 2);
    if (kind_of(r) != NB_CORNER3) continue;
    // corners (-,-), (+,-), (-,+), (+,+)
    const int i = (r & 1) ? MX + (k & 1) : -2 + (k & 1);
    const int j = (r & 2) ? MX + ((k >> 1) & 1) : -2 + ((k >> 1) & 1);
    const int ic = i < 0 ? 0 : MX - 1, jc = j < 0 ? 0 : MX - 1;
    Q[(j + kMbc) * S + i + kMbc] =
        real(0.5) * (Q[(jc + kMbc) * S + i + kMbc] + Q[(j + kMbc) * S + ic + kMbc]);
  }
}

// the same with the owner's staged entries
template <typename real, int MX>
__device__ __forceinline__ void corner3_fill(const NbrStage& st, real* Q, int tid, int nt) {
  corner3_fill_k<real, MX>([&](int r) { return st.e[r].kind; }, Q, tid, nt);
}

}  // namespace fc
