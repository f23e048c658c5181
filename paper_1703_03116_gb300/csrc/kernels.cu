// CUDA kernels of the patch-AMR hot path (sm_103a): ghost fill (Alg. 1
// phases), the wave-propagation patch update, tagging, regrid remap, mass,
// and field packing.
//
// Store layout: every patch is one contiguous (mx+4)^2 block ([j][i], i
// fastest) holding interior and two ghost layers (Sec. 2: "a grid with 8^2
// interior cells and two layers of ghost cells stores solution data in a
// contiguous array of 12^2").  Two such stores are kept; level l's current
// data live in buf[cur[l]] and its previous state in buf[cur[l]^1].
#include <cmath>

#include "fc_internal.hpp"

namespace fc {

uint64_t& launch_counter() {
  static thread_local uint64_t c = 0;
  return c;
}

namespace {

template <typename real>
__device__ __forceinline__ real minmod(real a, real b) {
  if (a * b <= real(0)) return real(0);
  return fabs(a) < fabs(b) ? a : b;
}

template <typename real>
__device__ __forceinline__ real mc_phi(real th) {
  real a = real(0.5) * (real(1) + th);
  real m = a < real(2) ? a : real(2);
  m = m < real(2) * th ? m : real(2) * th;
  return m > real(0) ? m : real(0);
}

__device__ __forceinline__ int2 apply_a(int a, int x, int y) {
  int u = (a & 1) ? y : x;
  int v = (a & 1) ? x : y;
  if (a & 2) u = -u;
  if (a & 4) v = -v;
  return make_int2(u, v);
}

// k-th ghost cell of a patch: rows -2,-1 and mx,mx+1 (full width), then
// columns -2,-1,mx,mx+1 of the interior rows.
__device__ __forceinline__ void ghost_ij(int k, int mx, int& i, int& j) {
  const int S = mx + 4;
  if (k < 2 * S) {
    j = k / S - 2;
    i = k % S - 2;
    return;
  }
  k -= 2 * S;
  if (k < 2 * S) {
    j = mx + k / S;
    i = k % S - 2;
    return;
  }
  k -= 2 * S;
  j = k >> 2;
  const int c = k & 3;
  i = c < 2 ? c - 2 : mx + c - 2;
}

__device__ __forceinline__ int region_of(int i, int j, int mx) {
  const int dx = i < 0 ? -1 : (i >= mx ? 1 : 0);
  const int dy = j < 0 ? -1 : (j >= mx ? 1 : 0);
  if (dy == 0) return dx < 0 ? 0 : 1;
  if (dx == 0) return dy < 0 ? 2 : 3;
  return 4 + (dx > 0 ? 1 : 0) + (dy > 0 ? 2 : 0);
}

template <typename real>
__device__ __forceinline__ size_t cell(const DevForest<real>& D, int p, int i, int j) {
  return (size_t)p * D.S * D.S + (size_t)(j + kMbc) * D.S + (i + kMbc);
}

// interior value of source patch n for copy/average: time-interpolated when
// n is on the level that the fill reads through the interpolation buffer
template <typename real>
__device__ __forceinline__ real src_interior(const DevForest<real>& D, const FillArgs& A, int n,
                                             int i, int j) {
  const int lev = D.meta[n].level;
  const size_t o = cell(D, n, i, j);
  if (lev == A.tlevel) {
    const int c = D.cur[lev];
    return (real(1) - real(A.alpha)) * D.buf[c ^ 1][o] + real(A.alpha) * D.buf[c][o];
  }
  return D.buf[D.cur[lev]][o];
}

// array of patch n as a coarse interpolation source (interior + ghosts)
template <typename real>
__device__ __forceinline__ const real* src_array(const DevForest<real>& D, const FillArgs& A,
                                                 int n) {
  const int lev = D.meta[n].level;
  const real* base = (lev == A.tlevel) ? D.qT : D.buf[D.cur[lev]];
  return base + (size_t)n * D.S * D.S;
}

template <typename real>
__device__ __forceinline__ real* dst_array(const DevForest<real>& D, const FillArgs& A, int p) {
  const int lev = D.meta[p].level;
  real* base = (lev == A.tlevel) ? D.qT : D.buf[D.cur[lev]];
  return base + (size_t)p * D.S * D.S;
}

// zeroth-order extrapolation at walls: an exterior ghost copies the owner's
// cell with the out-of-domain index clamped to the nearest interior index
template <typename real>
__device__ void wall_bc(const DevForest<real>& D, const PatchMeta& pm, real* Q) {
  const int mx = D.mx, S = D.S;
  const int N = mx << pm.level;
  const int NG = 4 * S + 4 * mx;
  for (int k = threadIdx.x; k < NG; k += blockDim.x) {
    int i, j;
    ghost_ij(k, mx, i, j);
    const int gx = pm.x * mx + i, gy = pm.y * mx + j;
    const bool ox = gx < 0 || gx >= N, oy = gy < 0 || gy >= N;
    if (!ox && !oy) continue;
    const int ic = ox ? (gx < 0 ? 0 : mx - 1) : i;
    const int jc = oy ? (gy < 0 ? 0 : mx - 1) : j;
    Q[(j + kMbc) * S + i + kMbc] = Q[(jc + kMbc) * S + ic + kMbc];
  }
}

// Alg. 1 phases 1-2 for a list of patches: copy (Eq. transform), average
// (Eq. ghost_coarse), then the physical boundary condition.  Patches on the
// time-interpolated level also get their interior (1-alpha) old + alpha new.
template <typename real>
__global__ void __launch_bounds__(256) fill_coarse_kernel(DevForest<real> D, FillArgs A) {
  const int mx = D.mx, S = D.S;
  const int NG = 4 * S + 4 * mx;
  for (int t = blockIdx.x; t < A.ntargets; t += gridDim.x) {
    const int p = A.targets[t];
    const PatchMeta pm = D.meta[p];
    real* Q = dst_array(D, A, p);
    if (pm.level == A.tlevel) {
      for (int k = threadIdx.x; k < mx * mx; k += blockDim.x) {
        const int i = k % mx, j = k / mx;
        Q[(j + kMbc) * S + i + kMbc] = src_interior(D, A, p, i, j);
      }
    }
    for (int k = threadIdx.x; k < NG; k += blockDim.x) {
      int i, j;
      ghost_ij(k, mx, i, j);
      const NbrEntry e = D.nbr[(size_t)p * 8 + region_of(i, j, mx)];
      if (e.kind != NB_SAME && e.kind != NB_FINE) continue;
      const int2 Ip = apply_a(e.a, pm.x * mx + i, pm.y * mx + j);
      const int gx = Ip.x + e.fx, gy = Ip.y + e.fy;
      real v;
      if (e.kind == NB_SAME) {
        const PatchMeta nm = D.meta[e.n0];
        const int lx = gx - nm.x * mx, ly = gy - nm.y * mx;
        if (lx < 0 || lx >= mx || ly < 0 || ly >= mx) continue;  // malformed entry
        v = src_interior(D, A, e.n0, lx, ly);
      } else {
        int n = e.n0;
        PatchMeta nm = D.meta[n];
        int lx = 2 * gx - nm.x * mx, ly = 2 * gy - nm.y * mx;
        if (lx < 0 || lx >= mx || ly < 0 || ly >= mx) {
          if (e.n1 < 0) continue;  // malformed entry
          n = e.n1;
          nm = D.meta[n];
          lx = 2 * gx - nm.x * mx;
          ly = 2 * gy - nm.y * mx;
          if (lx < 0 || lx >= mx || ly < 0 || ly >= mx) continue;
        }
        real s[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int2 d = apply_a(e.a, (q & 1) ? 1 : -1, (q & 2) ? 1 : -1);
          s[q] = src_interior(D, A, n, lx + (d.x > 0), ly + (d.y > 0));
        }
        v = real(0.25) * (((s[0] + s[1]) + s[2]) + s[3]);
      }
      Q[(j + kMbc) * S + i + kMbc] = v;
    }
    if (D.domain == FC_DOMAIN_WALLS) {
      __syncthreads();
      wall_bc(D, pm, Q);
    }
    __syncthreads();
  }
}

// Alg. 1 phases 3-4: interpolation from the coarser neighbour (Eq.
// ghost_fine, minmod-limited one-sided slopes in the coarse index space),
// then the physical boundary condition again.
template <typename real>
__global__ void __launch_bounds__(256) fill_fine_kernel(DevForest<real> D, FillArgs A) {
  const int mx = D.mx, S = D.S;
  const int NG = 4 * S + 4 * mx;
  for (int t = blockIdx.x; t < A.ntargets; t += gridDim.x) {
    const int p = A.targets[t];
    const PatchMeta pm = D.meta[p];
    real* Q = dst_array(D, A, p);
    for (int k = threadIdx.x; k < NG; k += blockDim.x) {
      int i, j;
      ghost_ij(k, mx, i, j);
      const NbrEntry e = D.nbr[(size_t)p * 8 + region_of(i, j, mx)];
      if (e.kind != NB_COARSE) continue;
      const int2 Ip = apply_a(e.a, pm.x * mx + i, pm.y * mx + j);
      const int gx = Ip.x + e.fx, gy = Ip.y + e.fy;
      const PatchMeta nm = D.meta[e.n0];
      const int ic = (gx >> 1) - nm.x * mx, jc = (gy >> 1) - nm.y * mx;
      if (ic < 0 || ic >= mx || jc < 0 || jc >= mx) continue;  // malformed entry
      const real dx = (gx & 1) ? real(1) : real(-1);
      const real dy = (gy & 1) ? real(1) : real(-1);
      const real* C = src_array(D, A, e.n0);
      const real q0 = C[(jc + kMbc) * S + ic + kMbc];
      const real sx = minmod(C[(jc + kMbc) * S + ic + 1 + kMbc] - q0,
                             q0 - C[(jc + kMbc) * S + ic - 1 + kMbc]);
      const real sy = minmod(C[(jc + 1 + kMbc) * S + ic + kMbc] - q0,
                             q0 - C[(jc - 1 + kMbc) * S + ic + kMbc]);
      Q[(j + kMbc) * S + i + kMbc] = q0 + real(0.25) * (sx * dx + sy * dy);
    }
    if (D.domain == FC_DOMAIN_WALLS) {
      __syncthreads();
      wall_bc(D, pm, Q);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ advance

template <typename real>
__device__ __forceinline__ real correction(int order, int limiter, real s, real W, real Wup,
                                           real nu) {
  if (order < 2) return real(0);
  real phi = real(1);
  if (limiter) {
    if (W == real(0)) return real(0);
    phi = mc_phi(Wup / W);
  }
  const real as = fabs(s);
  return real(0.5) * as * (real(1) - nu * as) * phi * W;
}

template <typename real>
__device__ __forceinline__ real sinpi_r(real x);
template <>
__device__ __forceinline__ float sinpi_r<float>(float x) { return sinpif(x); }
template <>
__device__ __forceinline__ double sinpi_r<double>(double x) { return sinpi(x); }

// One patch per CTA (grid-stride over the level's patches).  The whole
// (mx+4)^2 tile is staged in shared memory; edge quantities of both sweeps
// are computed once into shared arrays; each interior cell then gathers the
// transverse increments of its four edges and writes its new value.
//
// x-edge (i,j) sits between cells (i-1,j) and (i,j), i in [0,MX], j in [-1,MX];
// y-edge (i,j) sits between cells (i,j-1) and (i,j), j in [0,MX], i in [-1,MX].
template <typename real, int MX>
__global__ void __launch_bounds__(256) advance_kernel(DevForest<real> D, int p0, int p1,
                                                      double t_half, double dt) {
  constexpr int S = MX + 4;
  constexpr int NE = (MX + 1) * (MX + 2);
  constexpr int NT = MX + 3;  // corner nodes -1..MX+1
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real* Q = reinterpret_cast<real*>(smem_raw);
  real* Fn = Q + S * S;
  real* XP = Fn + NE;
  real* XM = XP + NE;
  real* Gn = XM + NE;
  real* YP = Gn + NE;
  real* YM = YP + NE;
  real* Sx = YM + NE;
  real* Sy = Sx + NT;
  real* Tx = Sy + NT;
  real* Ty = Tx + NT;
  const int order = D.order, limiter = D.limiter, transverse = D.transverse;
  const bool swirl = D.vel_kind == FC_VEL_SWIRL;
  const real cu = real(D.vel[0]), cv = real(D.vel[1]);

  for (int p = p0 + blockIdx.x; p < p1; p += gridDim.x) {
    const PatchMeta pm = D.meta[p];
    const real* src = D.buf[D.cur[pm.level]] + (size_t)p * S * S;
    real* dst = D.buf[D.cur[pm.level] ^ 1] + (size_t)p * S * S;
    const double hd = ldexp(1.0, -pm.level) / MX;
    const real nu = real(dt / hd);
    for (int k = threadIdx.x; k < S * S; k += blockDim.x) Q[k] = src[k];
    // Swirl: psi = s(x) s(y) cos(pi t/T)/pi with s = sin^2(pi .), so the
    // corner difference along an edge is s(corner) (s(y1) - s(y0)) and
    // s(y1) - s(y0) = sin(pi (y0 + y1)) sin(pi h): corner tables S, edge
    // tables T, no cancellation.
    real ucoef = real(0);
    if (swirl) {
      ucoef = real(cospi(t_half / D.vel[0]) / M_PI * sinpi(hd) / hd);
      for (int k = threadIdx.x; k < NT; k += blockDim.x) {
        const real xs = sinpi_r(real((pm.x * MX + k - 1) * hd));
        const real ys = sinpi_r(real((pm.y * MX + k - 1) * hd));
        Sx[k] = xs * xs;
        Sy[k] = ys * ys;
        Tx[k] = sinpi_r(real((2 * (pm.x * MX + k - 1) + 1) * hd));
        Ty[k] = sinpi_r(real((2 * (pm.y * MX + k - 1) + 1) * hd));
      }
    }
    __syncthreads();
    auto q = [&](int i, int j) -> real { return Q[(j + 2) * S + (i + 2)]; };
    auto uvel = [&](int i, int j) -> real {  // x-edge (i,j): corners (i,j), (i,j+1)
      return swirl ? ucoef * Sx[i + 1] * Ty[j + 1] : cu;
    };
    auto vvel = [&](int i, int j) -> real {  // y-edge (i,j): corners (i,j), (i+1,j)
      return swirl ? -ucoef * Sy[j + 1] * Tx[i + 1] : cv;
    };
    // x-sweep
    for (int e = threadIdx.x; e < NE; e += blockDim.x) {
      const int i = e % (MX + 1), j = e / (MX + 1) - 1;
      const real s = uvel(i, j);
      const real sp = s > real(0) ? s : real(0), sm = s < real(0) ? s : real(0);
      const real W = q(i, j) - q(i - 1, j);
      const real Wup = s >= real(0) ? q(i - 1, j) - q(i - 2, j) : q(i + 1, j) - q(i, j);
      const real Ft = correction(order, limiter, s, W, Wup, nu);
      Fn[e] = sp * q(i - 1, j) + sm * q(i, j) + Ft;
      real P = sp * W, M = sm * W;
      if (transverse > 1) {
        P -= Ft;
        M += Ft;
      }
      XP[e] = P;
      XM[e] = M;
    }
    // y-sweep
    for (int e = threadIdx.x; e < NE; e += blockDim.x) {
      const int i = e % (MX + 2) - 1, j = e / (MX + 2);
      const real s = vvel(i, j);
      const real sp = s > real(0) ? s : real(0), sm = s < real(0) ? s : real(0);
      const real W = q(i, j) - q(i, j - 1);
      const real Wup = s >= real(0) ? q(i, j - 1) - q(i, j - 2) : q(i, j + 1) - q(i, j);
      const real Ft = correction(order, limiter, s, W, Wup, nu);
      Gn[e] = sp * q(i, j - 1) + sm * q(i, j) + Ft;
      real P = sp * W, M = sm * W;
      if (transverse > 1) {
        P -= Ft;
        M += Ft;
      }
      YP[e] = P;
      YM[e] = M;
    }
    __syncthreads();
    const real half_nu = real(0.5) * nu;
    auto xe = [](int i, int j) { return (j + 1) * (MX + 1) + i; };
    auto ye = [](int i, int j) { return j * (MX + 2) + (i + 1); };
    // total x-fluctuation into cell (i,j), and y-fluctuation
    auto Xc = [&](int i, int j) -> real { return XP[xe(i, j)] + XM[xe(i + 1, j)]; };
    auto Yc = [&](int i, int j) -> real { return YP[ye(i, j)] + YM[ye(i, j + 1)]; };
    auto Fx = [&](int i, int j) -> real {
      real f = Fn[xe(i, j)];
      if (transverse > 0) {
        const real s = uvel(i, j);
        const real sp = s > real(0) ? s : real(0), sm = s < real(0) ? s : real(0);
        f -= half_nu * (sp * Yc(i - 1, j) + sm * Yc(i, j));
      }
      return f;
    };
    auto Gy = [&](int i, int j) -> real {
      real g = Gn[ye(i, j)];
      if (transverse > 0) {
        const real s = vvel(i, j);
        const real sp = s > real(0) ? s : real(0), sm = s < real(0) ? s : real(0);
        g -= half_nu * (sp * Xc(i, j - 1) + sm * Xc(i, j));
      }
      return g;
    };
    for (int k = threadIdx.x; k < MX * MX; k += blockDim.x) {
      const int i = k % MX, j = k / MX;
      const real v = q(i, j) - nu * (Fx(i + 1, j) - Fx(i, j)) - nu * (Gy(i, j + 1) - Gy(i, j));
      dst[(j + 2) * S + (i + 2)] = v;
    }
    __syncthreads();
  }
}

template <typename real, int MX>
size_t advance_smem() {
  constexpr int S = MX + 4;
  constexpr int NE = (MX + 1) * (MX + 2);
  return sizeof(real) * (size_t)(S * S + 6 * NE + 4 * (MX + 3));
}

template <typename real, int MX>
cudaError_t advance_mx(const DevForest<real>& D, int p0, int p1, double t, double dt,
                       cudaStream_t s) {
  static bool attr_set = false;
  const size_t smem = advance_smem<real, MX>();
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(advance_kernel<real, MX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int n = p1 - p0;
  advance_kernel<real, MX><<<n, 256, smem, s>>>(D, p0, p1, t + 0.5 * dt, dt);
  ++launch_counter();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ tag

template <typename real>
__global__ void tag_kernel(DevForest<real> D, double* delta) {
  __shared__ double red[256];
  const int mx = D.mx, S = D.S;
  for (int p = blockIdx.x; p < D.npatch; p += gridDim.x) {
    const real* Q = D.buf[D.cur[D.meta[p].level]] + (size_t)p * S * S;
    double m = 0.0;
    for (int k = threadIdx.x; k < mx * mx; k += blockDim.x) {
      const int i = k % mx + 2, j = k / mx + 2;
      const double gx = (double)Q[j * S + i + 1] - (double)Q[j * S + i - 1];
      const double gy = (double)Q[(j + 1) * S + i] - (double)Q[(j - 1) * S + i];
      const double d = 0.5 * sqrt(gx * gx + gy * gy);
      m = d > m ? d : m;
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
      __syncthreads();
    }
    if (threadIdx.x == 0) delta[p] = red[0];
    __syncthreads();
  }
}

// ------------------------------------------------------------------ mass

template <typename real>
__global__ void patch_sum_kernel(DevForest<real> D, double* sums) {
  __shared__ double red[256];
  const int mx = D.mx, S = D.S;
  for (int p = blockIdx.x; p < D.npatch; p += gridDim.x) {
    const PatchMeta pm = D.meta[p];
    const real* Q = D.buf[D.cur[pm.level]] + (size_t)p * S * S;
    double s = 0.0;
    for (int k = threadIdx.x; k < mx * mx; k += blockDim.x)
      s += (double)Q[(k / mx + 2) * S + k % mx + 2];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const double h = ldexp(1.0, -pm.level) / mx;
      sums[p] = h * h * red[0];
    }
    __syncthreads();
  }
}

__global__ void forest_sum_kernel(const double* sums, const int* api_to_dev, const int* fstart,
                                  int nforests, double* out) {
  __shared__ double red[256];
  for (int f = blockIdx.x; f < nforests; f += gridDim.x) {
    double s = 0.0;
    for (int k = fstart[f] + threadIdx.x; k < fstart[f + 1]; k += blockDim.x)
      s += sums[api_to_dev[k]];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[f] = red[0];
    __syncthreads();
  }
}

// ------------------------------------------------------------------ pack / unpack

template <typename real>
__global__ void pack_kernel(DevForest<real> D, const int* api_to_dev, real* out, int full) {
  const int mx = D.mx, S = D.S;
  const int per = full ? S * S : mx * mx;
  const size_t total = (size_t)D.npatch * per;
  for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(g / per), r = (int)(g % per);
    const int p = api_to_dev[k];
    const real* Q = D.buf[D.cur[D.meta[p].level]] + (size_t)p * S * S;
    out[g] = full ? Q[r] : Q[(r / mx + 2) * S + r % mx + 2];
  }
}

template <typename real>
__global__ void unpack_kernel(DevForest<real> D, const int* api_to_dev, const real* in) {
  const int mx = D.mx, S = D.S;
  const size_t total = (size_t)D.npatch * mx * mx;
  for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(g / (mx * mx)), r = (int)(g % (mx * mx));
    const int p = api_to_dev[k];
    real* Q = D.buf[D.cur[D.meta[p].level]] + (size_t)p * S * S;
    Q[(r / mx + 2) * S + r % mx + 2] = in[g];
  }
}

// ------------------------------------------------------------------ remap

template <typename real>
__global__ void remap_kernel(DevForest<real> Old, DevForest<real> New, const RemapEntry* rm) {
  const int mx = New.mx, S = New.S;
  for (int p = blockIdx.x; p < New.npatch; p += gridDim.x) {
    const RemapEntry e = rm[p];
    real* Dq = New.buf[New.cur[New.meta[p].level]] + (size_t)p * S * S;
    for (int k = threadIdx.x; k < mx * mx; k += blockDim.x) {
      const int i = k % mx, j = k / mx;
      real v;
      if (e.kind == RM_COPY) {
        const int s = e.src[0];
        v = Old.buf[Old.cur[Old.meta[s].level]][(size_t)s * S * S + (j + 2) * S + i + 2];
      } else if (e.kind == RM_INTERP) {
        const int s = e.src[0];
        const real* C = Old.buf[Old.cur[Old.meta[s].level]] + (size_t)s * S * S;
        const int ic = e.cx * (mx / 2) + (i >> 1) + 2, jc = e.cy * (mx / 2) + (j >> 1) + 2;
        const real dx = (i & 1) ? real(1) : real(-1), dy = (j & 1) ? real(1) : real(-1);
        const real q0 = C[jc * S + ic];
        const real sx = minmod(C[jc * S + ic + 1] - q0, q0 - C[jc * S + ic - 1]);
        const real sy = minmod(C[(jc + 1) * S + ic] - q0, q0 - C[(jc - 1) * S + ic]);
        v = q0 + real(0.25) * (sx * dx + sy * dy);
      } else {
        const int cx = (2 * i >= mx), cy = (2 * j >= mx);
        const int s = e.src[cx + 2 * cy];
        const real* C = Old.buf[Old.cur[Old.meta[s].level]] + (size_t)s * S * S;
        const int fi = 2 * i - cx * mx + 2, fj = 2 * j - cy * mx + 2;
        v = real(0.25) * (((C[fj * S + fi] + C[fj * S + fi + 1]) + C[(fj + 1) * S + fi]) +
                          C[(fj + 1) * S + fi + 1]);
      }
      Dq[(j + 2) * S + i + 2] = v;
    }
  }
}

inline int grid_for(int n) { return n < 1 ? 1 : (n < 65535 * 8 ? n : 65535 * 8); }

}  // namespace

// ------------------------------------------------------------------ launchers

template <typename real>
cudaError_t launch_fill_coarse(const DevForest<real>& D, const FillArgs& A, cudaStream_t s) {
  if (A.ntargets <= 0) return cudaSuccess;
  fill_coarse_kernel<real><<<grid_for(A.ntargets), 128, 0, s>>>(D, A);
  ++launch_counter();
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_fill_fine(const DevForest<real>& D, const FillArgs& A, cudaStream_t s) {
  if (A.ntargets <= 0) return cudaSuccess;
  fill_fine_kernel<real><<<grid_for(A.ntargets), 128, 0, s>>>(D, A);
  ++launch_counter();
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_advance(const DevForest<real>& D, int level, int p0, int p1, double t,
                           double dt, cudaStream_t s) {
  (void)level;
  if (p1 <= p0) return cudaSuccess;
  switch (D.mx) {
    case 8: return advance_mx<real, 8>(D, p0, p1, t, dt, s);
    case 16: return advance_mx<real, 16>(D, p0, p1, t, dt, s);
    case 32: return advance_mx<real, 32>(D, p0, p1, t, dt, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename real>
cudaError_t launch_tag(const DevForest<real>& D, double* delta, cudaStream_t s) {
  if (D.npatch <= 0) return cudaSuccess;
  tag_kernel<real><<<grid_for(D.npatch), 256, 0, s>>>(D, delta);
  ++launch_counter();
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_mass(const DevForest<real>& D, const int* api_to_dev, const int* fstart,
                        int nforests, double* patch_sums, double* out, cudaStream_t s) {
  if (D.npatch > 0) {
    patch_sum_kernel<real><<<grid_for(D.npatch), 256, 0, s>>>(D, patch_sums);
    ++launch_counter();
  }
  forest_sum_kernel<<<grid_for(nforests), 256, 0, s>>>(patch_sums, api_to_dev, fstart, nforests,
                                                        out);
  ++launch_counter();
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_pack(const DevForest<real>& D, const int* api_to_dev, real* out, int full,
                        cudaStream_t s) {
  if (D.npatch <= 0) return cudaSuccess;
  pack_kernel<real><<<1216, 256, 0, s>>>(D, api_to_dev, out, full);
  ++launch_counter();
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_unpack(const DevForest<real>& D, const int* api_to_dev, const real* in,
                          cudaStream_t s) {
  if (D.npatch <= 0) return cudaSuccess;
  unpack_kernel<real><<<1216, 256, 0, s>>>(D, api_to_dev, in);
  ++launch_counter();
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_remap(const DevForest<real>& Old, const DevForest<real>& New,
                         const RemapEntry* rm, cudaStream_t s) {
  if (New.npatch <= 0) return cudaSuccess;
  remap_kernel<real><<<grid_for(New.npatch), 256, 0, s>>>(Old, New, rm);
  ++launch_counter();
  return cudaGetLastError();
}

#define FC_INSTANTIATE(real)                                                                   \
  template cudaError_t launch_fill_coarse<real>(const DevForest<real>&, const FillArgs&,      \
                                                cudaStream_t);                                 \
  template cudaError_t launch_fill_fine<real>(const DevForest<real>&, const FillArgs&,        \
                                              cudaStream_t);                                   \
  template cudaError_t launch_advance<real>(const DevForest<real>&, int, int, int, double,    \
                                            double, cudaStream_t);                             \
  template cudaError_t launch_tag<real>(const DevForest<real>&, double*, cudaStream_t);        \
  template cudaError_t launch_mass<real>(const DevForest<real>&, const int*, const int*, int, \
                                         double*, double*, cudaStream_t);                      \
  template cudaError_t launch_pack<real>(const DevForest<real>&, const int*, real*, int,      \
                                         cudaStream_t);                                        \
  template cudaError_t launch_unpack<real>(const DevForest<real>&, const int*, const real*,   \
                                           cudaStream_t);                                      \
  template cudaError_t launch_remap<real>(const DevForest<real>&, const DevForest<real>&,     \
                                          const RemapEntry*, cudaStream_t);

FC_INSTANTIATE(float)
FC_INSTANTIATE(double)

}  // namespace fc
