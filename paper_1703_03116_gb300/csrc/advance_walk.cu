// The wave-propagation patch update, "walk" variant (sm_103a).
//
// Same scheme as the staged variant (flux-form 2D wave propagation with
// MC-limited corrections and transverse propagation of both fluctuations),
// organised for the fewest instructions per cell:
//
//  * A warp works on 32/MX patches at a time; lane li of a patch's segment
//    owns interior column li and walks up the rows, keeping the column's
//    values in a four-row register window.  Per row it computes its x-edge
//    (left edge of its cell) and the y-edge above its window row; the
//    neighbouring column's results arrive by warp shuffles.
//  * The one x-edge and the two y-edge columns that fall outside the lanes
//    (x-edge MX, y-edges of ghost columns -1 and MX) are computed first by a
//    side pass in which lanes own rows, into small shared arrays.
//  * Each finished row of cells goes straight to HBM (coalesced); nothing
//    else is written to shared memory.
//  * Tiles arrive by 1D TMA bulk copies (cp.async.bulk + mbarrier), double
//    buffered per warp: the next group of patches is in flight while the
//    current one is computed.  Grids are persistent (CTAs loop over groups).
#include <atomic>
#include <cstdint>

#include "ghost_gather.cuh"
#include "walk_edge.cuh"

namespace fc {
namespace {

template <int MX>
constexpr int tile_stride() {
  // pad so that the 4 tiles of a warp at MX = 8 start on different banks
  return MX == 8 ? 168 : (MX + 4) * (MX + 4);
}

template <int MX>
constexpr int side_reals() {
  return ((2 * (MX + 3) + 3 * (MX + 2) + 4 * (MX + 1)) + 3) & ~3;
}

// NB tile buffers per warp: 2 overlap the next group's copy with this
// group's compute; 1 halves the shared memory, so twice the warps fit on an
// SM and other warps hide the copy instead
template <typename real, int MX, int NB>
constexpr int warp_reals() {
  return NB * (32 / MX) * tile_stride<MX>() + (32 / MX) * side_reals<MX>();
}

template <typename real, int MX, int NW, bool SWIRL, int NB>
__global__ void __launch_bounds__(NW * 32) advance_walk_kernel(DevForest<real> D, int p0, int p1,
                                                               AdvArgs a, int* err) {
  constexpr int S = MX + 4;
  constexpr int PPW = 32 / MX;
  constexpr int TILE = S * S;
  constexpr int TS = tile_stride<MX>();
  constexpr int NS = MX + 3;
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[NW][2];
  __shared__ real ucoef_s;
  __shared__ NbrStage nst[NW][PPW];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int seg = lane / MX, li = lane % MX;
  real* wbase = reinterpret_cast<real*>(smem_raw) + (size_t)warp * warp_reals<real, MX, NB>();
  real* side = wbase + NB * PPW * TS + seg * side_reals<MX>();
  real* TyS = side;           // sin(pi (y_r + y_{r+1})), r = -1..MX+1 at [r+1]
  real* SyS = TyS + NS;       // sin^2(pi y_r), r = -1..MX+1 at [r+1]
  real* FeN = SyS + NS;       // x-edge MX: normal flux, rows -1..MX at [r+1]
  real* FeU = FeN + (MX + 2);  //            speed
  real* XMe = FeU + (MX + 2);  //            fluctuation into cell MX-1
  real* YPm = XMe + (MX + 2);  // y-edges of column -1, rows 0..MX
  real* YMm = YPm + (MX + 1);
  real* YPp = YMm + (MX + 1);  // y-edges of column MX, rows 0..MX
  real* YMp = YPp + (MX + 1);

  if (threadIdx.x == 0 && SWIRL) {
    const double t = a.t0_dev ? *a.t0_dev + a.t_off : a.t_half;
    ucoef_s = cospi_ratio<real>(t, a.period) * real(a.sfac);
  }
  if (lane == 0) {
    mbar_init(&bars[warp][0], 1);
    mbar_init(&bars[warp][1], 1);
  }
  __syncthreads();

  const real ucoef = SWIRL ? ucoef_s : real(0);
  const real cu = real(D.vel[0]), cv = real(D.vel[1]);
  const real h = real(a.h);
  const Scheme<real> sc = make_scheme<real>(D.order, D.limiter, D.transverse, a.nu);

  const int ngroups = (p1 - p0 + PPW - 1) / PPW;
  const int TW = gridDim.x * NW;
  auto tile = [&](int b, int s) { return wbase + (b * PPW + s) * TS; };
  auto issue = [&](int g, int b) {  // lane 0: TMA loads of group g into buffer b
    const int nvalid = min(PPW, p1 - p0 - g * PPW);
    fence_proxy_async();
    mbar_expect_tx(&bars[warp][b], (uint32_t)(nvalid * TILE * sizeof(real)));
    for (int s = 0; s < nvalid; ++s) {
      const int p = p0 + g * PPW + s;
      const real* src = D.buf[D.cur[D.meta[p].level]] + (size_t)p * TILE;
      bulk_load(tile(b, s), src, (uint32_t)(TILE * sizeof(real)), &bars[warp][b]);
    }
  };

  uint32_t par0 = 0, par1 = 0;
  int b = 0;
  const int g_first = blockIdx.x * NW + warp;
  int g = g_first;
  if (g < ngroups && lane == 0) issue(g, 0);
  for (; g < ngroups; g += TW, b ^= (NB - 1)) {
    const bool prefetch = NB == 2 && g + TW < ngroups;
    // one buffer: the group's copy starts once the warp left the previous one
    if (NB == 1 && g != g_first && lane == 0) issue(g, 0);
    if (prefetch && lane == 0) issue(g + TW, b ^ 1);
    const int p = p0 + g * PPW + seg;
    const bool valid = p < p1;
    const int pc = valid ? p : p0 + g * PPW;
    const PatchMeta pm = D.meta[pc];
    real* dst = D.buf[D.cur[pm.level] ^ 1] + (size_t)pc * TILE;
    const int x0 = pm.x * MX, y0 = pm.y * MX;
    // column factors of this lane's edges (streamfunction tables)
    real Sx_i = 0, Tx_i = 0, SxE = 0, TxM = 0, TxP = 0;
    if (SWIRL) {
      real s = sinpi_r(real(x0 + li) * h);
      Sx_i = s * s;
      Tx_i = sinpi_r(real(2 * (x0 + li) + 1) * h);
      s = sinpi_r(real(x0 + MX) * h);
      SxE = s * s;
      TxM = sinpi_r(real(2 * (x0 - 1) + 1) * h);
      TxP = sinpi_r(real(2 * (x0 + MX) + 1) * h);
    }
    uint32_t& par = b ? par1 : par0;
    const bool ok = mbar_wait(&bars[warp][b], par, a.wait_limit);
    if (!__all_sync(FULL, ok)) {
      if (lane == 0) atomicOr(err, kErrTimeout);
      // let every copy in flight land before leaving
      mbar_wait(&bars[warp][b], par, kWaitLimit);
      if (prefetch) mbar_wait(&bars[warp][b ^ 1], b ? par0 : par1, kWaitLimit);
      return;
    }
    par ^= 1;
    real* T = tile(b, seg);
    if (a.gather) {  // Alg. 1 for this segment's patch, into the tile's ghost ring
      stage_neighbours(D.meta, D.nbr, pc, nst[warp][seg], li);
      __syncwarp();
      // every ghost by its own rule in one pass (the phases of Alg. 1 write
      // different ghosts, and an interpolation reads the coarse patch, not
      // this tile), then the wall condition once: the bits of the phased fill
      const NbrStage& ns = nst[warp][seg];
      for (int k = li; k < num_ghosts<MX>(); k += MX) {
        int i, j;
        ghost_ij<MX>(k, i, j);
        const NbrEntry& e = ns.e[region_of<MX>(i, j)];
        real v;
        if (copy_or_average_entry<real, MX>(D, e, pm, a.tlevel, real(a.alpha), i, j, v) ||
            interpolate_entry<real, MX>(D, e, pm, a.tlevel, i, j, v))
          T[(j + kMbc) * S + i + kMbc] = v;
      }
      __syncwarp();
      if (D.domain == FC_DOMAIN_WALLS) {
        wall_bc<real, MX>(pm, T, li, MX);
        __syncwarp();
      }
    }
    if (a.keep && valid) {  // the adjoint's replay keeps the ghost-filled input tile
      real* kp = static_cast<real*>(a.keep) + (size_t)(p - a.keep_p0) * TILE;
      for (int k = li; k < TILE; k += MX) kp[k] = T[k];
    }
    auto Q = [&](int i, int j) -> real { return T[(j + 2) * S + (i + 2)]; };

    // side pass: lanes own rows r = -1..MX+1
    for (int r = li - 1; r <= MX + 1; r += MX) {
      const real ty = SWIRL ? sinpi_r(real(2 * (y0 + r) + 1) * h) : real(0);
      real sy = SWIRL ? sinpi_r(real(y0 + r) * h) : real(0);
      sy *= sy;
      TyS[r + 1] = ty;
      SyS[r + 1] = sy;
      real Fn, P, M;
      if (r <= MX) {  // x-edge MX of row r
        const real s = SWIRL ? ucoef * SxE * ty : cu;
        edge(s, Q(MX - 2, r), Q(MX - 1, r), Q(MX, r), Q(MX + 1, r), sc, Fn, P, M);
        FeN[r + 1] = Fn;
        FeU[r + 1] = s;
        XMe[r + 1] = M;
      }
      if (r >= 0 && r <= MX) {  // y-edges of ghost columns -1 and MX at row r
        const real sl = SWIRL ? -ucoef * sy * TxM : cv;
        edge(sl, Q(-1, r - 2), Q(-1, r - 1), Q(-1, r), Q(-1, r + 1), sc, Fn, P, M);
        YPm[r] = P;
        YMm[r] = M;
        const real sr = SWIRL ? -ucoef * sy * TxP : cv;
        edge(sr, Q(MX, r - 2), Q(MX, r - 1), Q(MX, r), Q(MX, r + 1), sc, Fn, P, M);
        YPp[r] = P;
        YMp[r] = M;
      }
    }
    __syncwarp();

    // main walk: lane li owns column li; iteration r computes x-edge (li, r)
    // and y-edge (li, r+1), finishes the fluxes of row r and updates row r-1
    real qa = Q(li, -2), qb = Q(li, -1), qc = Q(li, 0), qd = 0;
    real X_prev = 0, Gn_cur = 0, v_cur = 0, YP_cur = 0, Gf_prev = 0, dF_prev = 0;
#pragma unroll 2  // fully unrolled, the row walk overflowed the instruction cache
    for (int r = -1; r <= MX; ++r) {
      if (r + 2 <= MX + 1) qd = Q(li, r + 2);
      // x-edge (li, r): cells (li-1, r) | (li, r)
      const real su = SWIRL ? ucoef * Sx_i * TyS[r + 1] : cu;
      real Fn_r, XP_r, XM_r;
      edge(su, Q(li - 2, r), Q(li - 1, r), qb, Q(li + 1, r), sc, Fn_r, XP_r, XM_r);
      real XMn = __shfl_down_sync(FULL, XM_r, 1, MX);
      if (li == MX - 1) XMn = XMe[r + 1];
      const real X_r = XP_r + XMn;  // x-fluctuation into cell (li, r)
      // y-edge (li, r+1): cells (li, r) | (li, r+1)
      real Gn_n = 0, YP_n = 0, YM_n = 0, v_n = 0;
      if (r + 1 <= MX) {
        v_n = SWIRL ? -ucoef * SyS[r + 2] * Tx_i : cv;
        edge(v_n, qa, qb, qc, qd, sc, Gn_n, YP_n, YM_n);
      }
      // final flux at y-edge (li, r)
      real Gf_r = 0;
      if (r >= 0)
        Gf_r = Gn_cur - sc.tfac * (fmax(v_cur, real(0)) * X_prev + fmin(v_cur, real(0)) * X_r);
      // final fluxes at x-edges (li, r) and (li+1, r)
      real dF_r = 0;
      if (r >= 0 && r < MX) {
        const real Y_r = YP_cur + YM_n;  // y-fluctuation into cell (li, r)
        real Yl = __shfl_up_sync(FULL, Y_r, 1, MX);
        if (li == 0) Yl = YPm[r] + YMm[r + 1];
        const real Ff = Fn_r - sc.tfac * (fmax(su, real(0)) * Yl + fmin(su, real(0)) * Y_r);
        real Fr = __shfl_down_sync(FULL, Ff, 1, MX);
        if (li == MX - 1) {
          const real ue = FeU[r + 1];
          Fr = FeN[r + 1] -
               sc.tfac * (fmax(ue, real(0)) * Y_r + fmin(ue, real(0)) * (YPp[r] + YMp[r + 1]));
        }
        dF_r = Fr - Ff;
      }
      // conservative update of cell (li, r-1)
      if (r >= 1 && valid)
        dst[(r + 1) * S + (li + 2)] = qa - sc.nu * dF_prev - sc.nu * (Gf_r - Gf_prev);
      X_prev = X_r;
      Gn_cur = Gn_n;
      v_cur = v_n;
      YP_cur = YP_n;
      Gf_prev = Gf_r;
      dF_prev = dF_r;
      qa = qb;
      qb = qc;
      qc = qd;
    }
    __syncwarp();
  }
}

template <typename real, int MX, int NW, bool SWIRL, int NB>
cudaError_t walk_launch(const DevForest<real>& D, int p0, int p1, const AdvArgs& a, int* err,
                        cudaStream_t s) {
  // computed once per process; concurrent first calls compute the same value
  static std::atomic<int> max_ctas_once{0};
  int max_ctas = max_ctas_once.load(std::memory_order_acquire);
  constexpr size_t smem = sizeof(real) * (size_t)NW * warp_reals<real, MX, NB>();
  auto kern = advance_walk_kernel<real, MX, NW, SWIRL, NB>;
  if (max_ctas == 0) {
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NW * 32, smem);
    if (e != cudaSuccess) return e;
    max_ctas = nsm * (per_sm > 0 ? per_sm : 1);
    max_ctas_once.store(max_ctas, std::memory_order_release);
  }
  constexpr int PPW = 32 / MX;
  const int groups = (p1 - p0 + PPW - 1) / PPW;
  int ctas = (groups + NW - 1) / NW;
  const int cap = a.ctas > 0 ? a.ctas : max_ctas;
  if (ctas > cap) ctas = cap;
  kern<<<ctas, NW * 32, smem, s>>>(D, p0, p1, a, err);
  ++launch_counter();
  return cudaGetLastError();
}

template <typename real, int MX, int NW>
cudaError_t walk_vel(const DevForest<real>& D, int p0, int p1, const AdvArgs& a, int* err,
                     cudaStream_t s) {
  const bool one = a.variant == ADV_WALK1;
  if (D.vel_kind == FC_VEL_SWIRL)
    return one ? walk_launch<real, MX, NW, true, 1>(D, p0, p1, a, err, s)
               : walk_launch<real, MX, NW, true, 2>(D, p0, p1, a, err, s);
  return one ? walk_launch<real, MX, NW, false, 1>(D, p0, p1, a, err, s)
             : walk_launch<real, MX, NW, false, 2>(D, p0, p1, a, err, s);
}

template <typename real, int MX>
cudaError_t walk_nw(const DevForest<real>& D, int p0, int p1, const AdvArgs& a, int* err,
                    cudaStream_t s) {
  switch (a.warps) {
    case 2: return walk_vel<real, MX, 2>(D, p0, p1, a, err, s);
    case 8: return walk_vel<real, MX, 8>(D, p0, p1, a, err, s);
    default: return walk_vel<real, MX, 4>(D, p0, p1, a, err, s);
  }
}

}  // namespace

template <typename real>
cudaError_t launch_advance_walk(const DevForest<real>& D, int p0, int p1, const AdvArgs& a,
                                int* err, cudaStream_t s) {
  switch (D.mx) {
    case 8: return walk_nw<real, 8>(D, p0, p1, a, err, s);
    case 16: return walk_nw<real, 16>(D, p0, p1, a, err, s);
    case 32: return walk_nw<real, 32>(D, p0, p1, a, err, s);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_advance_walk<float>(const DevForest<float>&, int, int,
                                                const AdvArgs&, int*, cudaStream_t);
template cudaError_t launch_advance_walk<double>(const DevForest<double>&, int, int,
                                                 const AdvArgs&, int*, cudaStream_t);

}  // namespace fc
