// The wave-propagation patch update, "band" variant (sm_103a).
//
// One CTA per patch, as in the staged variant, so that a launch of few
// patches still takes about one patch's latency; inside the CTA the update
// is the walk variant's row walk, divided among the warps.  Warp segment b
// (MX lanes) owns the band of R rows [bR, (b+1)R): lane li owns column li and
// walks the band's rows, keeping a four-row register window of its column,
// taking the neighbouring column's edge results by warp shuffles and writing
// each finished row of cells straight to HBM.  A band also computes the
// x-edges of the row below it and of the row above it, which the transverse
// increments of its first and last y-edge read: R + 2 rows of x-edges and
// R + 1 rows of y-edges per band.  The staged variant instead passes over
// every edge in shared memory, with a CTA barrier between phases.
//
// Before the walk, the CTA fills the tile's ghost ring (Alg. 1: the
// neighbour reads are made while the tile's TMA copy is in flight). It then
// computes what every band reads at the patch's sides: for each row, the
// x = MX edge (normal flux, speed, and the fluctuation into the last
// column); and the fluctuations of the y-edges of ghost columns -1 and MX.
// Then the bands run with no further CTA barrier.
//
// Refluxing: the final fluxes through the patch's faces are recorded as the
// staged variant does.
#include <atomic>
#include <cstdint>

#include "ghost_gather.cuh"
#include "walk_edge.cuh"

namespace fc {
namespace {

// threads of a CTA: one per column of each band, and at least one per
// ghost cell (the extra warps gather ghosts and then idle in the walk), so
// that no thread gathers two ghosts one after the other: each gather is a
// chain of dependent reads of other patches' cells
template <typename real, int MX, int R>
constexpr int band_threads() {
  return MX * MX / R > (num_ghosts<MX>() + 31) / 32 * 32 ? MX * MX / R
                                                         : (num_ghosts<MX>() + 31) / 32 * 32;
}

// resident CTAs the register budget is sized for: 1024 FP32 / 512 FP64
// threads per SM at most 64 / 128 registers a thread
template <typename real, int MX, int R>
constexpr int band_min_blocks() {
  return (sizeof(real) == 4 ? 1024 : 512) / band_threads<real, MX, R>() > 0
             ? (sizeof(real) == 4 ? 1024 : 512) / band_threads<real, MX, R>()
             : 1;
}

// CAP: the capacity form of the cubed sphere (Sec. 5.3) -- the patch's FP64
// metric block (kappa, phi_x, phi_y) arrives in dynamic shared memory by a
// second bulk copy; edge speeds are the edge volume fluxes phi, the
// correction's dt/h is dt (1/kappa_L + 1/kappa_R)/2, a fluctuation's
// transverse increment is scaled by dt/2 over the area of the cell it
// enters, and the update by dt over the cell's area.
template <typename real, int MX, int R, bool SWIRL, bool CAP>
__global__ void __launch_bounds__(band_threads<real, MX, R>(), band_min_blocks<real, MX, R>())
    advance_band_kernel(DevForest<real> D, int p0, int p1, AdvArgs a, int* err) {
  constexpr int S = MX + 4;
  constexpr int MS = CAP ? metric_stride(S) : 0;
  constexpr uint32_t mbytes = sizeof(double) * MS;
  extern __shared__ __align__(16) double Ms[];  // CAP: kappa, phi_x, phi_y
  constexpr int NT = band_threads<real, MX, R>();
  constexpr int NW = MX * MX / R;  // threads that walk a band
  constexpr int NV = MX + 3;  // corner nodes -1..MX+1 of a row or column
  constexpr int NG = num_ghosts<MX>();
  constexpr unsigned FULL = 0xffffffffu;
  constexpr uint32_t bytes = sizeof(real) * S * S;
  static_assert(MX % R == 0 && NW % 32 == 0 && NT % 32 == 0, "bands of R rows, whole warps");
  __shared__ __align__(128) real Q[S * S];
  __shared__ __align__(8) uint64_t bar;
  __shared__ real ucoef_s;
  __shared__ real ring[NG];    // ghost values gathered while the tile loads
  __shared__ bool ring_w[NG];
  // streamfunction tables over corner nodes k = 0..MX+2 (index k - 1):
  // Sx = sin^2(pi x_node), Tx = sin(pi (x_{c} + x_{c+1})) of column c = k - 1
  __shared__ real Sx[NV], Sy[NV], Tx[NV], Ty[NV];
  // the patch's sides: x-edge MX of rows -1..MX at [r + 1] (final-flux
  // inputs: normal flux, speed; fluctuation into cell MX - 1), and the
  // y-edges of ghost columns -1 / MX at rows 0..MX (fluctuations up / down)
  __shared__ real FeN[MX + 2], FeU[MX + 2], XMe[MX + 2];
  __shared__ real YPm[MX + 1], YMm[MX + 1], YPp[MX + 1], YMp[MX + 1];

  const int tid = threadIdx.x;
  const int li = tid % MX;  // column of this lane
  const int r0 = (tid / MX) * R;  // first row of this lane's band
  // thread 0 initialises the copy barrier, issues the copies and waits for
  // them; the other threads touch the barrier only after a CTA barrier
  if (tid == 0) mbar_init(&bar, 1);
  const real cu = real(D.vel[0]), cv = real(D.vel[1]);
  const real h = real(a.h);
  const Scheme<real> sc = make_scheme<real>(D.order, D.limiter, D.transverse, a.nu);
  const real dt = real(a.dt), tdt = D.transverse > 0 ? real(0.5 * a.dt) : real(0);
  auto q = [&](int i, int j) -> real { return Q[(j + kMbc) * S + (i + kMbc)]; };
  // capacity form: 1/kappa of cell (i, j), volume flux of x-edge (i, j) /
  // y-edge (i, j), and an edge's correction dt/h from its two cells
  auto ik = [&](int i, int j) -> real { return real(1) / real(Ms[(j + kMbc) * S + i + kMbc]); };
  auto phx = [&](int i, int j) -> real {
    return real(Ms[S * S + (j + kMbc) * (S + 1) + i + kMbc]);
  };
  auto phy = [&](int i, int j) -> real {
    return real(Ms[S * S + S * (S + 1) + (j + kMbc) * S + i + kMbc]);
  };
  auto nu_e = [&](real ika, real ikb) -> real { return dt * (real(0.5) * (ika + ikb)); };

  uint32_t parity = 0;
  for (int p = p0 + blockIdx.x; p < p1; p += gridDim.x, parity ^= 1) {
    const PatchMeta pm = D.meta[p];
    const real* src = D.buf[D.cur[pm.level]] + (size_t)p * S * S;
    real* dst = D.buf[D.cur[pm.level] ^ 1] + (size_t)p * S * S;
    if (tid == 0) {
      fence_proxy_async();
      mbar_expect_tx(&bar, bytes + mbytes);
      bulk_load(Q, src, bytes, &bar);
      if (CAP) bulk_load(Ms, D.metric + (size_t)p * MS, mbytes, &bar);
    }
    // the swirl coefficient, by the last thread (it gathers at most one
    // ghost); read after the barrier below
    if (SWIRL && tid == NT - 1 && p == p0 + (int)blockIdx.x) {
      const double t = a.t0_dev ? *a.t0_dev + a.t_off : a.t_half;
      ucoef_s = cospi_ratio<real>(t, a.period) * real(a.sfac);
    }
    if (SWIRL) {  // the tables, while the tile is in flight
      for (int k = tid; k < 4 * NV; k += NT) {
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
    }
    // each gathering thread reads the entry of its ghost's region from the
    // table itself: no staging pass, no barrier before the gather
    if (a.gather)
      gather_ring<real, MX>(
          D, [&](int r) { return D.nbr[(size_t)p * 8 + r]; }, p, pm, a.tlevel, real(a.alpha),
          a.direct != 0, ring, ring_w, tid, NT, static_cast<real*>(a.keep_t), a.keep_t_p0);
    // thread 0 observes the copy's completion (bounded), the others after the
    // barrier (at once); the CTA leaves together if it gave up
    const bool landed = tid == 0 ? mbar_wait(&bar, parity, a.wait_limit) : true;
    if (!__syncthreads_and(landed)) {
      if (tid == 0) atomicOr(err, kErrTimeout);
      mbar_wait(&bar, parity, kWaitLimit);  // let the copy land before leaving
      return;
    }
    if (tid != 0) mbar_wait(&bar, parity, kWaitLimit);
    if (a.gather) {
      store_ring<real, MX>(Q, ring, ring_w, tid, NT);
      __syncthreads();
      if (D.domain == FC_DOMAIN_WALLS) {
        wall_bc<real, MX>(pm, Q, tid, NT);
        __syncthreads();
      }
      if (CAP && D.domain == FC_DOMAIN_SPHERE) {  // corners beyond a cube vertex
        corner3_fill_k<real, MX>([&](int r) { return D.nbr[(size_t)p * 8 + r].kind; }, Q, tid,
                                 NT);
        __syncthreads();
      }
    }
    if (a.keep) {  // the adjoint's replay keeps the ghost-filled input tile
      real* kp = static_cast<real*>(a.keep) + (size_t)(p - a.keep_p0) * S * S;
      for (int k = tid; k < S * S; k += NT) kp[k] = Q[k];
    }
    const real ucoef = SWIRL ? ucoef_s : real(0);
    // the sides: x-edge MX of rows -1..MX, y-edges of ghost columns -1 and
    // MX at rows 0..MX (one edge a thread)
    for (int k = tid; k < 3 * MX + 4; k += NT) {
      real Fn, P, M;
      if (k < MX + 2) {
        const int r = k - 1;
        const real s = CAP ? phx(MX, r) : SWIRL ? ucoef * Sx[MX + 1] * Ty[r + 1] : cu;
        const real nu = CAP ? nu_e(ik(MX - 1, r), ik(MX, r)) : sc.nu;
        edge(s, q(MX - 2, r), q(MX - 1, r), q(MX, r), q(MX + 1, r), nu, sc, Fn, P, M);
        FeN[k] = Fn;
        FeU[k] = s;
        XMe[k] = M;
      } else {
        const bool right = k >= 2 * MX + 3;
        const int r = k - (right ? 2 * MX + 3 : MX + 2);
        const int c = right ? MX : -1;
        const real s = CAP ? phy(c, r) : SWIRL ? -ucoef * Sy[r + 1] * Tx[c + 1] : cv;
        const real nu = CAP ? nu_e(ik(c, r - 1), ik(c, r)) : sc.nu;
        edge(s, q(c, r - 2), q(c, r - 1), q(c, r), q(c, r + 1), nu, sc, Fn, P, M);
        (right ? YPp : YPm)[r] = P;
        (right ? YMp : YMm)[r] = M;
      }
    }
    __syncthreads();
    // the band walk: iteration it works on row r = r0 - 1 + it; it computes
    // x-edge (li, r) and y-edge (li, r + 1), finishes the final fluxes of
    // row r and updates cell (li, r - 1)
    real* bf = a.bflux ? static_cast<real*>(a.bflux) + ((size_t)p * 2 + a.bslot) * 4 * MX
                       : nullptr;
    if (tid < NW) {  // (the warps beyond the bands only gathered ghosts)
      const real Sx_i = SWIRL ? Sx[li + 1] : real(0), Tx_i = SWIRL ? Tx[li + 1] : real(0);
      real qa = q(li, r0 - 2), qb = q(li, r0 - 1), qc = q(li, r0), qd = 0;
      real X_prev = 0, Gn_cur = 0, v_cur = 0, YP_cur = 0, Gf_prev = 0, dF_prev = 0;
      // capacity form: 1/kappa of this column's cells in rows r-1, r
      real ik_prev = CAP ? ik(li, r0 - 2) : real(0), ik_cur = CAP ? ik(li, r0 - 1) : real(0);
#pragma unroll(R <= 8 ? R + 2 : 2)
      for (int it = 0; it < R + 2; ++it) {
        const int r = r0 - 1 + it;
        if (it <= R) qd = q(li, r + 2);
        const real ik_next = CAP && it <= R ? ik(li, r + 1) : real(0);
        real ik_left = CAP ? __shfl_up_sync(FULL, ik_cur, 1, MX) : real(0);  // cell (li-1, r)
        if (CAP && li == 0) ik_left = ik(-1, r);
        // x-edge (li, r): cells (li-1, r) | (li, r)
        const real su = CAP ? phx(li, r) : SWIRL ? ucoef * Sx_i * Ty[r + 1] : cu;
        real Fn_r, XP_r, XM_r;
        edge(su, q(li - 2, r), q(li - 1, r), qb, q(li + 1, r),
             CAP ? nu_e(ik_left, ik_cur) : sc.nu, sc, Fn_r, XP_r, XM_r);
        real XMn = __shfl_down_sync(FULL, XM_r, 1, MX);
        if (li == MX - 1) XMn = XMe[r + 1];
        const real X_r = XP_r + XMn;  // x-fluctuation into cell (li, r)
        // y-edge (li, r+1): cells (li, r) | (li, r+1); the last row's is the
        // next band's
        real Gn_n = 0, YP_n = 0, YM_n = 0, v_n = 0;
        if (it <= R) {
          v_n = CAP ? phy(li, r + 1) : SWIRL ? -ucoef * Sy[r + 2] * Tx_i : cv;
          edge(v_n, qa, qb, qc, qd, CAP ? nu_e(ik_cur, ik_next) : sc.nu, sc, Gn_n, YP_n, YM_n);
        }
        // final flux at y-edge (li, r)
        real Gf_r = 0;
        if (it >= 1) {
          if (CAP)
            Gf_r = Gn_cur - tdt * (fmax(v_cur, real(0)) * X_prev * ik_prev +
                                   fmin(v_cur, real(0)) * X_r * ik_cur);
          else
            Gf_r = Gn_cur - sc.tfac * (fmax(v_cur, real(0)) * X_prev + fmin(v_cur, real(0)) * X_r);
          if (bf && r == 0) bf[2 * MX + li] = Gf_r;
          if (bf && r == MX) bf[3 * MX + li] = Gf_r;
        }
        // final fluxes at x-edges (li, r) and (li+1, r), rows of the band
        real dF_r = 0;
        if (it >= 1 && it <= R) {
          const real Y_r = YP_cur + YM_n;  // y-fluctuation into cell (li, r)
          real Yl = __shfl_up_sync(FULL, Y_r, 1, MX);
          if (li == 0) Yl = YPm[r] + YMm[r + 1];
          const real Ff =
              CAP ? Fn_r - tdt * (fmax(su, real(0)) * Yl * ik_left + fmin(su, real(0)) * Y_r * ik_cur)
                  : Fn_r - sc.tfac * (fmax(su, real(0)) * Yl + fmin(su, real(0)) * Y_r);
          real Fr = __shfl_down_sync(FULL, Ff, 1, MX);
          if (li == MX - 1) {
            const real ue = FeU[r + 1];
            if (CAP)
              Fr = FeN[r + 1] - tdt * (fmax(ue, real(0)) * Y_r * ik_cur +
                                       fmin(ue, real(0)) * (YPp[r] + YMp[r + 1]) * ik(MX, r));
            else
              Fr = FeN[r + 1] - sc.tfac * (fmax(ue, real(0)) * Y_r +
                                           fmin(ue, real(0)) * (YPp[r] + YMp[r + 1]));
          }
          dF_r = Fr - Ff;
          if (bf && li == 0) bf[r] = Ff;
          if (bf && li == MX - 1) bf[MX + r] = Fr;
        }
        // conservative update of cell (li, r-1)
        if (it >= 2)
          dst[(r + 1) * S + (li + kMbc)] =
              CAP ? qa - dt * ik_prev * (dF_prev + (Gf_r - Gf_prev))
                  : qa - sc.nu * dF_prev - sc.nu * (Gf_r - Gf_prev);
        X_prev = X_r;
        Gn_cur = Gn_n;
        v_cur = v_n;
        YP_cur = YP_n;
        Gf_prev = Gf_r;
        dF_prev = dF_r;
        qa = qb;
        qb = qc;
        qc = qd;
        ik_prev = ik_cur;
        ik_cur = ik_next;
      }
    }
    __syncthreads();  // the next patch's copy overwrites the tile
  }
}

template <typename real, int MX, int R, bool SWIRL, bool CAP>
cudaError_t band_launch_t(const DevForest<real>& D, int p0, int p1, const AdvArgs& a, int* err,
                          cudaStream_t s) {
  constexpr size_t dyn = CAP ? sizeof(double) * (size_t)metric_stride(MX + 4) : 0;
  auto kern = advance_band_kernel<real, MX, R, SWIRL, CAP>;
  if (CAP) {  // set once per process; concurrent first calls both set it (idempotent)
    static std::atomic<bool> attr_set{false};
    if (!attr_set.load(std::memory_order_acquire)) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)dyn);
      if (e != cudaSuccess) return e;
      attr_set.store(true, std::memory_order_release);
    }
  }
  kern<<<p1 - p0, band_threads<real, MX, R>(), dyn, s>>>(D, p0, p1, a, err);
  ++launch_counter();
  return cudaGetLastError();
}

template <typename real, int MX, int R>
cudaError_t band_launch(const DevForest<real>& D, int p0, int p1, const AdvArgs& a, int* err,
                        cudaStream_t s) {
  if (D.metric) return band_launch_t<real, MX, R, false, true>(D, p0, p1, a, err, s);
  if (D.vel_kind == FC_VEL_SWIRL)
    return band_launch_t<real, MX, R, true, false>(D, p0, p1, a, err, s);
  return band_launch_t<real, MX, R, false, false>(D, p0, p1, a, err, s);
}

}  // namespace

// rows per band from the requested warps per CTA: a.warps x 32 threads, at
// most one lane per interior cell
template <typename real>
cudaError_t launch_advance_band(const DevForest<real>& D, int p0, int p1, const AdvArgs& a,
                                int* err, cudaStream_t s) {
  switch (D.mx) {
    case 8: return band_launch<real, 8, 1>(D, p0, p1, a, err, s);
    case 16:
      return a.warps <= 2 ? band_launch<real, 16, 4>(D, p0, p1, a, err, s)
             : a.warps == 4 ? band_launch<real, 16, 2>(D, p0, p1, a, err, s)
                            : band_launch<real, 16, 1>(D, p0, p1, a, err, s);
    case 32:
      return a.warps <= 4  ? band_launch<real, 32, 8>(D, p0, p1, a, err, s)
             : a.warps == 8 ? band_launch<real, 32, 4>(D, p0, p1, a, err, s)
                            : band_launch<real, 32, 2>(D, p0, p1, a, err, s);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_advance_band<float>(const DevForest<float>&, int, int,
                                                const AdvArgs&, int*, cudaStream_t);
template cudaError_t launch_advance_band<double>(const DevForest<double>&, int, int,
                                                 const AdvArgs&, int*, cudaStream_t);

}  // namespace fc
