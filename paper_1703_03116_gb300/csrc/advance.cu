// The wave-propagation patch update (sm_103a): "staged" variant and the
// variant dispatcher.
//
// Scheme: the 2D unsplit wave-propagation method for q_t + (uq)_x + (vq)_y = 0
// in flux form (the Clawpack algorithms the paper runs, Sec. 5): per edge the
// upwind flux, an MC-limited second-order correction, and the two
// fluctuations, each carried across the transverse edges of the cell it
// enters; then the conservative update of the interior.
//
// Staged variant: one CTA per patch.  The whole (MX+4)^2 array (interior + 2
// ghost layers, contiguous in HBM) arrives in shared memory by one 1D TMA
// bulk copy; edge quantities of both sweeps are computed once into shared
// arrays; final edge fluxes are formed in a second pass; each interior cell
// then reads its four fluxes.  Every thread works on every phase, so a patch
// finishes quickly -- the better choice when a launch has few patches.
//
// Capacity form (CAP, the cubed sphere, Sec. 5.3): the patch's FP64 metric
// block arrives by a second bulk copy.  Edge speeds become edge volume fluxes
// phi, and every 1/h becomes 1/kappa of the cell concerned: the correction
// 1/2 |phi| (1 - dt |phi| (1/kappa_L + 1/kappa_R)/2) phi(theta) W, the
// transverse increments 1/2 dt/kappa_cell phi^-+ (fluctuation entering that
// cell), and the update Q -= dt/kappa (F(i+1/2) - F(i-1/2) + G(j+1/2) -
// G(j-1/2)).
#include <atomic>
#include <cstdint>

#include "ghost_gather.cuh"

namespace fc {
namespace {

template <typename real>
__device__ __forceinline__ real correction(int order, int limiter, real s, real W, real Wup,
                                           real nu) {
  if (order < 2) return real(0);
  const real as = fabs(s);
  const real lim = limiter ? mc_limited(W, Wup) : W;
  return real(0.5) * as * (real(1) - nu * as) * lim;
}

// x-edge (i,j) lies between cells (i-1,j) and (i,j): i in [0,MX], j in [-1,MX]
// y-edge (i,j) lies between cells (i,j-1) and (i,j): j in [0,MX], i in [-1,MX]
template <typename real, int MX, int NT, bool CAP>
// (resident CTAs per SM: 3 of 512 FP32 threads, at most 42 registers a
// thread; 2 FP64; 8 of 128 and 16 of 64 threads, at most 64 registers)
__global__ void __launch_bounds__(NT, NT >= 512 ? (sizeof(real) == 4 ? 3 : 2)
                                                : (NT >= 128 ? 8 : 16))
    advance_staged_kernel(DevForest<real> D, int p0, int p1, AdvArgs a, int* err) {
  constexpr int S = MX + 4;
  constexpr int NE = (MX + 1) * (MX + 2);
  constexpr int NV = MX + 3;  // corner nodes -1..MX+1
  constexpr int MS = CAP ? metric_stride(S) : 0;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ real ucoef_s;
  __shared__ NbrStage st;
  __shared__ real ring[num_ghosts<MX>()];  // ghost values gathered while the tile loads
  __shared__ bool ring_w[num_ghosts<MX>()];
  // Warp roles when the CTA has warps to spare beyond the ghost ring (mx =
  // 32): the first NGT threads gather the ghosts while the others already
  // compute the edges that read interior cells only (x-edges 2..MX-2 and
  // y-edges 2..MX-2 of the interior rows / columns), taken in warp-sized
  // chunks from a shared counter that the gathering warps join once their
  // ghosts are stored; every edge is computed once, by the same formula, so
  // the results are those of one pass over all edges.
  constexpr int NGT = (num_ghosts<MX>() + 31) / 32 * 32;
  constexpr bool SPLIT = NT - NGT >= 128;
  constexpr int NI = (MX - 3) * MX;           // interior edges per direction
  constexpr int NCHUNK = (2 * NI + 31) / 32;  // warp-sized chunks of them
  constexpr int NB = 6 * MX + 2;              // boundary edges per direction
  __shared__ int chunk_next;
  // capacity form: kappa, phi_x, phi_y of the patch (MS doubles) come first
  const double* Ms = reinterpret_cast<const double*>(smem_raw);
  real* Q = reinterpret_cast<real*>(smem_raw + sizeof(double) * MS);
  real* Fn = Q + S * S;
  real* XP = Fn + NE;
  real* XM = XP + NE;
  real* Gn = XM + NE;
  real* YP = Gn + NE;
  real* YM = YP + NE;
  real* Sx = YM + NE;
  real* Sy = Sx + NV;
  real* Tx = Sy + NV;
  real* Ty = Tx + NV;
  const int order = D.order, limiter = D.limiter, transverse = D.transverse;
  const bool swirl = !CAP && D.vel_kind == FC_VEL_SWIRL;
  const real cu = real(D.vel[0]), cv = real(D.vel[1]);
  const real nu = real(a.nu), half_nu = real(0.5 * a.nu), h = real(a.h);
  constexpr uint32_t bytes = sizeof(real) * S * S;
  constexpr uint32_t mbytes = sizeof(double) * MS;
  const real dt = real(a.dt), half_dt = real(0.5 * a.dt);

  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    chunk_next = 0;
  }
  __syncthreads();
  // the swirl coefficient: computed by the last thread (no ghost to gather)
  // while the first patch's tile is in flight, read after the next barrier
  real ucoef = real(0);
  uint32_t parity = 0;
  for (int p = p0 + blockIdx.x; p < p1; p += gridDim.x, parity ^= 1) {
    const PatchMeta pm = D.meta[p];
    const real* src = D.buf[D.cur[pm.level]] + (size_t)p * S * S;
    real* dst = D.buf[D.cur[pm.level] ^ 1] + (size_t)p * S * S;
    if (threadIdx.x == 0) {
      fence_proxy_async();
      mbar_expect_tx(&bar, bytes + mbytes);
      bulk_load(Q, src, bytes, &bar);
      if (CAP) bulk_load(smem_raw, D.metric + (size_t)p * MS, mbytes, &bar);
    }
    if (swirl && threadIdx.x == NT - 1 && p == p0 + (int)blockIdx.x) {
      const double t = a.t0_dev ? *a.t0_dev + a.t_off : a.t_half;
      ucoef_s = cospi_ratio<real>(t, a.period) * real(a.sfac);
    }
    auto q = [&](int i, int j) -> real { return Q[(j + 2) * S + (i + 2)]; };
    // capacity form: kappa of cell (i,j), flux through x-edge / y-edge (i,j)
    auto kap = [&](int i, int j) -> real { return real(Ms[(j + 2) * S + (i + 2)]); };
    auto uvel = [&](int i, int j) -> real {
      if (CAP) return real(Ms[S * S + (j + 2) * (S + 1) + (i + 2)]);
      return swirl ? ucoef * Sx[i + 1] * Ty[j + 1] : cu;
    };
    auto vvel = [&](int i, int j) -> real {
      if (CAP) return real(Ms[S * S + S * (S + 1) + (j + 2) * S + (i + 2)]);
      return swirl ? -ucoef * Sy[j + 1] * Tx[i + 1] : cv;
    };
    // dt |phi| (1/kappa_L + 1/kappa_R)/2 = nu_e |phi| in the correction
    auto nu_x = [&](int i, int j) -> real {
      return CAP ? dt * (real(0.5) * (real(1) / kap(i - 1, j) + real(1) / kap(i, j))) : nu;
    };
    auto nu_y = [&](int i, int j) -> real {
      return CAP ? dt * (real(0.5) * (real(1) / kap(i, j - 1) + real(1) / kap(i, j))) : nu;
    };
    // normal flux and fluctuations of x-edge (i, j) (cells (i-1,j) | (i,j))
    // and of y-edge (i, j) (cells (i,j-1) | (i,j))
    auto xedge = [&](int i, int j) {
      const int e = (j + 1) * (MX + 1) + i;
      const real s = uvel(i, j);
      const real sp = s > real(0) ? s : real(0), sm = s < real(0) ? s : real(0);
      const real qm = q(i - 1, j), q0 = q(i, j);
      const real W = q0 - qm;
      const real Wup = s >= real(0) ? qm - q(i - 2, j) : q(i + 1, j) - q0;
      const real Ft = correction(order, limiter, s, W, Wup, nu_x(i, j));
      Fn[e] = sp * qm + sm * q0 + Ft;
      XP[e] = transverse > 1 ? sp * W - Ft : sp * W;
      XM[e] = transverse > 1 ? sm * W + Ft : sm * W;
    };
    auto yedge = [&](int i, int j) {
      const int f = j * (MX + 2) + (i + 1);
      const real s = vvel(i, j);
      const real sp = s > real(0) ? s : real(0), sm = s < real(0) ? s : real(0);
      const real qm = q(i, j - 1), q0 = q(i, j);
      const real W = q0 - qm;
      const real Wup = s >= real(0) ? qm - q(i, j - 2) : q(i, j + 1) - q0;
      const real Gt = correction(order, limiter, s, W, Wup, nu_y(i, j));
      Gn[f] = sp * qm + sm * q0 + Gt;
      YP[f] = transverse > 1 ? sp * W - Gt : sp * W;
      YM[f] = transverse > 1 ? sm * W + Gt : sm * W;
    };
    // streamfunction tables (thread k0 + k for corner node k):
    // psi = s(x) s(y) cos(pi t/T)/pi, s = sin^2(pi .); along an edge the
    // corner difference is s(corner) * sin(pi (z0 + z1)) * sin(pi h)
    auto tables = [&](int k0) {
      if (!swirl) return;
      const int k = (int)threadIdx.x - k0;
      if (k >= 0 && k < NV) {
        const real xs = sinpi_r(real(pm.x * MX + k - 1) * h);
        const real ys = sinpi_r(real(pm.y * MX + k - 1) * h);
        Sx[k] = xs * xs;
        Sy[k] = ys * ys;
        Tx[k] = sinpi_r(real(2 * (pm.x * MX + k - 1) + 1) * h);
        Ty[k] = sinpi_r(real(2 * (pm.y * MX + k - 1) + 1) * h);
      }
    };
    // Alg. 1 for this patch, its neighbour reads while the tile is in
    // flight: each thread computes the values of its ghost cells (copied from
    // same-size or averaged from finer neighbours, interpolated from coarser
    // ones; every ghost is one of these or exterior) into registers, stored
    // into the tile once it has landed; then the wall condition (the
    // exterior ghosts copy cells that are final by then) and, on the sphere,
    // the corners beyond a cube vertex
    auto gather = [&](int nthreads) {
      gather_ring<real, MX>(
          D, [&](int r) -> const NbrEntry& { return st.e[r]; }, p, pm, a.tlevel, real(a.alpha),
          a.direct != 0, ring, ring_w, threadIdx.x, nthreads, static_cast<real*>(a.keep_t),
          a.keep_t_p0);
    };
    bool split_done = false;
    if constexpr (SPLIT) {
      if (a.gather) {
        if (threadIdx.x < 8) stage_neighbours(D.meta, D.nbr, p, st, threadIdx.x);
        tables(NGT);
        __syncthreads();  // the patch's entries, the tables, the swirl coefficient
        ucoef = swirl ? ucoef_s : real(0);
        bool landed;
        if (threadIdx.x < NGT) {  // gathering warps
          gather(NGT);
          landed = mbar_wait(&bar, parity, a.wait_limit);
          if (landed) store_ring<real, MX>(Q, ring, ring_w, threadIdx.x, NGT);
        } else {
          landed = mbar_wait(&bar, parity, a.wait_limit);
        }
        // interior edges in warp-sized chunks (the gathering warps join late)
        const unsigned lane = threadIdx.x & 31;
        if (__all_sync(0xffffffffu, landed)) {
          for (;;) {
            int c = 0;
            if (lane == 0) c = atomicAdd(&chunk_next, 1);
            c = __shfl_sync(0xffffffffu, c, 0);
            if (c >= NCHUNK) break;
            const int t = c * 32 + (int)lane;
            if (t < NI) {
              xedge(2 + t % (MX - 3), t / (MX - 3));
            } else if (t < 2 * NI) {
              const int u = t - NI;
              yedge(u % MX, 2 + u / MX);
            }
          }
        }
        // every thread observes the copy's completion (bounded); the CTA
        // leaves together if any thread gave up
        if (!__syncthreads_and(landed)) {
          if (threadIdx.x == 0) atomicOr(err, kErrTimeout);
          mbar_wait(&bar, parity, kWaitLimit);  // let the copy land before leaving
          return;
        }
        if (threadIdx.x == 0) chunk_next = 0;  // (its next use is after later barriers)
        if (D.domain == FC_DOMAIN_WALLS) {
          wall_bc<real, MX>(pm, Q, threadIdx.x, NT);
          __syncthreads();
        }
        if (D.domain == FC_DOMAIN_SPHERE) {
          corner3_fill<real, MX>(st, Q, threadIdx.x, NT);
          __syncthreads();
        }
        split_done = true;
      }
    }
    if (!split_done) {
      if (a.gather) stage_neighbours(D.meta, D.nbr, p, st, threadIdx.x);
      tables(0);
      if (a.gather) {
        __syncthreads();  // the patch's entries
        gather(NT);
      }
      // every thread observes the copy's completion (bounded); the CTA leaves
      // together if any thread gave up
      const bool landed = mbar_wait(&bar, parity, a.wait_limit);
      if (!__syncthreads_and(landed)) {
        if (threadIdx.x == 0) atomicOr(err, kErrTimeout);
        mbar_wait(&bar, parity, kWaitLimit);  // let the copy land before leaving
        return;
      }
      ucoef = swirl ? ucoef_s : real(0);
      if (a.gather) {
        store_ring<real, MX>(Q, ring, ring_w, threadIdx.x, NT);
        __syncthreads();
        if (D.domain == FC_DOMAIN_WALLS) {
          wall_bc<real, MX>(pm, Q, threadIdx.x, NT);
          __syncthreads();
        }
        if (D.domain == FC_DOMAIN_SPHERE) {
          corner3_fill<real, MX>(st, Q, threadIdx.x, NT);
          __syncthreads();
        }
      }
    }
    if (a.keep) {  // the adjoint's replay keeps the ghost-filled input tile
      real* kp = static_cast<real*>(a.keep) + (size_t)(p - a.keep_p0) * S * S;
      for (int k = threadIdx.x; k < S * S; k += NT) kp[k] = Q[k];
    }
    if (split_done) {
      // the edges that read ghost cells: full rows j = -1, MX and the columns
      // i = 0, 1, MX-1, MX of the interior rows (x); the same for y
      for (int b = threadIdx.x; b < 2 * NB; b += NT) {
        const bool y = b >= NB;
        const int c = y ? b - NB : b;
        int u, v;  // (along, across) the edge's direction of travel
        if (c < 2 * (MX + 1)) {
          u = c % (MX + 1);
          v = c < MX + 1 ? -1 : MX;
        } else {
          const int d = c - 2 * (MX + 1);
          v = d >> 2;
          u = (d & 3) < 2 ? (d & 3) : MX - 3 + (d & 3);  // 0, 1, MX-1, MX
        }
        if (y) yedge(v, u);  // column i = v, edge j = u
        else xedge(u, v);    // edge i = u, row j = v
      }
    } else {
      // both sweeps: normal flux and fluctuations of every edge
      for (int e = threadIdx.x; e < 2 * NE; e += NT) {
        if (e < NE) {
          xedge(e % (MX + 1), e / (MX + 1) - 1);
        } else {
          const int f = e - NE;
          yedge(f % (MX + 2) - 1, f / (MX + 2));
        }
      }
    }
    __syncthreads();
    auto xe = [](int i, int j) { return (j + 1) * (MX + 1) + i; };
    auto ye = [](int i, int j) { return j * (MX + 2) + (i + 1); };
    // final fluxes: each fluctuation's transverse increment, gathered per edge
    if (transverse > 0) {
      for (int e = threadIdx.x; e < 2 * MX * (MX + 1); e += NT) {
        if (e < MX * (MX + 1)) {  // x-edges i in [0,MX], interior rows
          const int i = e % (MX + 1), j = e / (MX + 1);
          const real s = uvel(i, j);
          const real sp = s > real(0) ? s : real(0), sm = s < real(0) ? s : real(0);
          const real yl = YP[ye(i - 1, j)] + YM[ye(i - 1, j + 1)];  // into cell (i-1,j)
          const real yr = YP[ye(i, j)] + YM[ye(i, j + 1)];          // into cell (i,j)
          if (CAP)
            Fn[xe(i, j)] -= half_dt * (sp * yl / kap(i - 1, j) + sm * yr / kap(i, j));
          else
            Fn[xe(i, j)] -= half_nu * (sp * yl + sm * yr);
        } else {  // y-edges j in [0,MX], interior columns
          const int f = e - MX * (MX + 1);
          const int i = f % MX, j = f / MX;
          const real s = vvel(i, j);
          const real sp = s > real(0) ? s : real(0), sm = s < real(0) ? s : real(0);
          const real xb = XP[xe(i, j - 1)] + XM[xe(i + 1, j - 1)];  // into cell (i,j-1)
          const real xt = XP[xe(i, j)] + XM[xe(i + 1, j)];          // into cell (i,j)
          if (CAP)
            Gn[ye(i, j)] -= half_dt * (sp * xb / kap(i, j - 1) + sm * xt / kap(i, j));
          else
            Gn[ye(i, j)] -= half_nu * (sp * xb + sm * xt);
        }
      }
      __syncthreads();
    }
    if (a.bflux) {  // refluxing: the final fluxes through the patch's faces
      real* bf = static_cast<real*>(a.bflux) + ((size_t)p * 2 + a.bslot) * 4 * MX;
      for (int k = threadIdx.x; k < 4 * MX; k += NT) {
        const int f = k / MX, c = k % MX;
        bf[k] = f == 0 ? Fn[xe(0, c)] : f == 1 ? Fn[xe(MX, c)] : f == 2 ? Gn[ye(c, 0)] : Gn[ye(c, MX)];
      }
    }
    for (int k = threadIdx.x; k < MX * MX; k += NT) {
      const int i = k % MX, j = k / MX;
      real v;
      if (CAP)
        v = q(i, j) - dt / kap(i, j) *
                          ((Fn[xe(i + 1, j)] - Fn[xe(i, j)]) + (Gn[ye(i, j + 1)] - Gn[ye(i, j)]));
      else
        v = q(i, j) - nu * (Fn[xe(i + 1, j)] - Fn[xe(i, j)]) -
            nu * (Gn[ye(i, j + 1)] - Gn[ye(i, j)]);
      dst[(j + 2) * S + (i + 2)] = v;
    }
    __syncthreads();
  }
}

template <typename real, int MX, bool CAP>
constexpr size_t staged_smem() {
  return sizeof(double) * (size_t)(CAP ? metric_stride(MX + 4) : 0) +
         sizeof(real) * (size_t)((MX + 4) * (MX + 4) + 6 * (MX + 1) * (MX + 2) + 4 * (MX + 3));
}

template <typename real, int MX, int NT, bool CAP>
cudaError_t staged_launch_t(const DevForest<real>& D, int p0, int p1, const AdvArgs& a, int* err,
                            cudaStream_t s) {
  // set once per process; concurrent first calls both set it (idempotent)
  static std::atomic<bool> attr_set{false};
  constexpr size_t smem = staged_smem<real, MX, CAP>();
  if (!attr_set.load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(advance_staged_kernel<real, MX, NT, CAP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set.store(true, std::memory_order_release);
  }
  advance_staged_kernel<real, MX, NT, CAP><<<p1 - p0, NT, smem, s>>>(D, p0, p1, a, err);
  ++launch_counter();
  return cudaGetLastError();
}

template <typename real, int MX, int NT>
cudaError_t staged_launch(const DevForest<real>& D, int p0, int p1, const AdvArgs& a, int* err,
                          cudaStream_t s) {
  if (D.metric) return staged_launch_t<real, MX, NT, true>(D, p0, p1, a, err, s);
  return staged_launch_t<real, MX, NT, false>(D, p0, p1, a, err, s);
}

template <typename real>
cudaError_t launch_advance_staged(const DevForest<real>& D, int p0, int p1, const AdvArgs& a,
                                  int* err, cudaStream_t s) {
  switch (D.mx) {
    case 8: return staged_launch<real, 8, 64>(D, p0, p1, a, err, s);
    case 16: return staged_launch<real, 16, 128>(D, p0, p1, a, err, s);
    case 32: return staged_launch<real, 32, 512>(D, p0, p1, a, err, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

template <typename real>
cudaError_t launch_advance(const DevForest<real>& D, int p0, int p1, const AdvArgs& a, int* err,
                           cudaStream_t s) {
  if (p1 <= p0) return cudaSuccess;
  // the walk variant has no capacity form and records no face fluxes:
  // mapped grids and refluxing run staged or band
  if ((a.variant == ADV_WALK || a.variant == ADV_WALK1) && !D.metric && !a.bflux)
    return launch_advance_walk(D, p0, p1, a, err, s);
  // the band variant records face fluxes and has the capacity form
  if (a.variant == ADV_BAND) return launch_advance_band(D, p0, p1, a, err, s);
  return launch_advance_staged(D, p0, p1, a, err, s);
}

template cudaError_t launch_advance<float>(const DevForest<float>&, int, int, const AdvArgs&,
                                           int*, cudaStream_t);
template cudaError_t launch_advance<double>(const DevForest<double>&, int, int, const AdvArgs&,
                                            int*, cudaStream_t);

}  // namespace fc
