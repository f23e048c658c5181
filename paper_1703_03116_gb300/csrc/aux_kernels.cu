// Auxiliary kernels: tagging (Sec. 3.1 indicator), FP64 mass sums, field
// packing between the store and the caller's layout, and the regrid remap
// (copy, Eq. ghost_fine interpolation into new children, Eq. ghost_coarse
// averaging into new parents).  On the cubed sphere mass is sum(kappa q) and
// new parents take the area-weighted mean of their children.
#include <cmath>

#include "device_util.cuh"

namespace fc {

uint64_t& launch_counter() {
  static thread_local uint64_t c = 0;
  return c;
}

namespace {
// ------------------------------------------------------------------ tag

// The indicator is max over cells of |grad q| / 2 (central differences),
// computed in the field's precision (FP64 on a GPU whose FP64 rate is a
// small fraction of FP32 would bound this memory-bound pass by arithmetic).
// The square root is monotone, so it is taken once per patch, of the largest
// squared difference: the same value, bit for bit, as the maximum of the
// per-cell roots.
// kind 1 (Sec. 5.1): the spread max q - min q of the interior instead, in
// the field's precision (exact: a difference of two stored values).
template <typename real>
__global__ void tag_kernel(DevForest<real> D, int kind, double* delta) {
  __shared__ real red[256], red2[256];
  const int mx = D.mx, S = D.S;
  for (int p = blockIdx.x; p < D.npatch; p += gridDim.x) {
    const real* Q = D.buf[D.cur[D.meta[p].level]] + (size_t)p * S * S;
    if (kind == 1) {
      real hi = Q[2 * S + 2], lo = hi;
      for (int k = threadIdx.x; k < mx * mx; k += blockDim.x) {
        const real v = Q[(k / mx + 2) * S + k % mx + 2];
        hi = v > hi ? v : hi;
        lo = v < lo ? v : lo;
      }
      red[threadIdx.x] = hi;
      red2[threadIdx.x] = lo;
      __syncthreads();
      for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
          if (red[threadIdx.x + w] > red[threadIdx.x]) red[threadIdx.x] = red[threadIdx.x + w];
          if (red2[threadIdx.x + w] < red2[threadIdx.x]) red2[threadIdx.x] = red2[threadIdx.x + w];
        }
        __syncthreads();
      }
      if (threadIdx.x == 0) delta[p] = (double)red[0] - (double)red2[0];
      __syncthreads();
      continue;
    }
    real m = real(0);
    for (int k = threadIdx.x; k < mx * mx; k += blockDim.x) {
      const int i = k % mx + 2, j = k / mx + 2;
      const real gx = Q[j * S + i + 1] - Q[j * S + i - 1];
      const real gy = Q[(j + 1) * S + i] - Q[(j - 1) * S + i];
      const real d2 = gx * gx + gy * gy;
      m = d2 > m ? d2 : m;
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) {
        const real o = red[threadIdx.x + w];
        if (o > red[threadIdx.x]) red[threadIdx.x] = o;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) delta[p] = 0.5 * sqrt((double)red[0]);
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
    if (D.metric) {  // mapped grid: sum of kappa q
      const double* K = D.metric + (size_t)p * metric_stride(S);
      for (int k = threadIdx.x; k < mx * mx; k += blockDim.x) {
        const int o = (k / mx + 2) * S + k % mx + 2;
        s += K[o] * (double)Q[o];
      }
    } else {
      for (int k = threadIdx.x; k < mx * mx; k += blockDim.x)
        s += (double)Q[(k / mx + 2) * S + k % mx + 2];
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const double h = ldexp(1.0, -pm.level) / mx;
      sums[p] = D.metric ? red[0] : h * h * red[0];
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
  const size_t total = (size_t)D.napi * per;
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
  const size_t total = (size_t)D.napi * mx * mx;
  for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(g / (mx * mx)), r = (int)(g % (mx * mx));
    const int p = api_to_dev[k];
    real* Q = D.buf[D.cur[D.meta[p].level]] + (size_t)p * S * S;
    Q[(r / mx + 2) * S + r % mx + 2] = in[g];
  }
}

// Test aid (an executable Prop. 1): value into every ghost cell of both
// state buffers and every cell of the time-interpolation tiles -- the cells
// a rule of Alg. 1 must write before any update may read them.
template <typename real>
__global__ void poison_kernel(DevForest<real> D, real value) {
  const int mx = D.mx, S = D.S;
  const size_t total = (size_t)D.npatch * S * S;
  for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(g % ((size_t)S * S)), i = r % S - kMbc, j = r / S - kMbc;
    D.qT[g] = value;
    if (i < 0 || i >= mx || j < 0 || j >= mx) {
      D.buf[0][g] = value;
      D.buf[1][g] = value;
    }
  }
}

// interior capacities in field order: kappa from the metric block on a
// mapped grid, h^2 on the square domains
template <typename real>
__global__ void pack_capacity_kernel(DevForest<real> D, const int* api_to_dev, double* out) {
  const int mx = D.mx, S = D.S;
  const size_t total = (size_t)D.napi * mx * mx;
  for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(g / (mx * mx)), r = (int)(g % (mx * mx));
    const int p = api_to_dev[k];
    if (D.metric) {
      out[g] = D.metric[(size_t)p * metric_stride(S) + (r / mx + 2) * S + r % mx + 2];
    } else {
      const double h = ldexp(1.0, -D.meta[p].level) / mx;
      out[g] = h * h;
    }
  }
}

// halo exchange of a partition: the interiors of the listed patches (local
// device indices, each read from its level's current state) to a contiguous
// buffer [k][j][i], and back into the listed mirrors' current states
template <typename real>
__global__ void halo_pack_kernel(DevForest<real> D, const int* list, int n, real* out) {
  const int mx = D.mx, S = D.S;
  const size_t total = (size_t)n * mx * mx;
  for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(g / (mx * mx)), r = (int)(g % (mx * mx));
    const int p = list[k];
    out[g] = D.buf[D.cur[D.meta[p].level]][(size_t)p * S * S + (r / mx + 2) * S + r % mx + 2];
  }
}

template <typename real>
__global__ void halo_unpack_kernel(DevForest<real> D, const int* list, int n, const real* in) {
  const int mx = D.mx, S = D.S;
  const size_t total = (size_t)n * mx * mx;
  for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(g / (mx * mx)), r = (int)(g % (mx * mx));
    const int p = list[k];
    D.buf[D.cur[D.meta[p].level]][(size_t)p * S * S + (r / mx + 2) * S + r % mx + 2] = in[g];
  }
}

// dst += src elementwise (n values)
template <typename real>
__global__ void add_store_kernel(real* dst, const real* src, size_t n) {
  for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < n;
       g += (size_t)gridDim.x * blockDim.x)
    dst[g] += src[g];
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
        if (Old.metric) {  // mapped grid: area-weighted, as the ghost average
          const double* K = Old.metric + (size_t)s * metric_stride(S);
          const double k0 = K[fj * S + fi], k1 = K[fj * S + fi + 1];
          const double k2 = K[(fj + 1) * S + fi], k3 = K[(fj + 1) * S + fi + 1];
          v = real((((k0 * double(C[fj * S + fi]) + k1 * double(C[fj * S + fi + 1])) +
                     k2 * double(C[(fj + 1) * S + fi])) +
                    k3 * double(C[(fj + 1) * S + fi + 1])) /
                   (((k0 + k1) + k2) + k3));
        } else {
          v = real(0.25) * (((C[fj * S + fi] + C[fj * S + fi + 1]) + C[(fj + 1) * S + fi]) +
                            C[(fj + 1) * S + fi + 1]);
        }
      }
      Dq[(j + 2) * S + i + 2] = v;
    }
  }
}

inline int grid_for(int n) { return n < 1 ? 1 : (n < 65535 * 8 ? n : 65535 * 8); }

// Refluxing (Berger and Colella's correction; the paper's scheme has none):
// one warp per level-L patch, lane k on face cell k.  A face whose other side
// is finer (an NB_FINE face entry: n0 holds the half of the face at cells
// 0..MX/2-1, n1 the other half, the square domains' identity orientation)
// gives coarse cell k the fine fluxes of fine cells 2k - half*MX and the next
// through the fine patch's opposite face, summed over nfs substep slots and
// scaled by w, in place of its own flux Fc of slot cslot.  The faces go one
// after the other (-x, +x, -y, +y): a corner cell takes two corrections, from
// two lanes, ordered by the warp barrier between faces.
template <typename real, int MX>
__global__ void reflux_kernel(DevForest<real> D, int p0, int p1, const real* __restrict__ bflux,
                              int cslot, int nfs, real w, real nu) {
  const int lane = threadIdx.x & 31;
  const int p = p0 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (p >= p1) return;  // whole warps leave together
  real* Q = D.buf[D.cur[D.meta[p].level]] + (size_t)p * D.S * D.S;
  for (int dir = 0; dir < 4; ++dir) {
    const NbrEntry& e = D.nbr[(size_t)p * 8 + dir];
    if (e.kind == NB_FINE && lane < MX) {
      const int k = lane, half = k >= MX / 2 ? 1 : 0;
      const int n = half ? e.n1 : e.n0;
      const int jf = 2 * k - half * MX;
      const int ff = dir ^ 1;  // the fine patch's face on the shared edge
      real acc = real(0);
      for (int s = 0; s < nfs; ++s) {
        const real* b = bflux + (((size_t)n * 2 + s) * 4 + ff) * MX + jf;
        acc += b[0] + b[1];
      }
      const real Fbar = w * acc;
      const real Fc = bflux[(((size_t)p * 2 + cslot) * 4 + dir) * MX + k];
      const int i = dir == 0 ? 0 : (dir == 1 ? MX - 1 : k);
      const int j = dir == 2 ? 0 : (dir == 3 ? MX - 1 : k);
      real* c = Q + (size_t)(j + kMbc) * D.S + (i + kMbc);
      *c = (dir == 0 || dir == 2) ? *c + nu * (Fbar - Fc) : *c + nu * (Fc - Fbar);
    }
    __syncwarp();
  }
}

// Refluxing on the cubed sphere, from the host's pairing (per patch, face
// and face cell: kind, patch across, its face g on the shared edge, its cells
// j0, j1): a cell beside a finer patch (kind 1) takes the fine side's volume
// fluxes summed over nfs substep slots with weight w (the time ratio); a
// cell on a cube edge whose same-size neighbour lies on a block of lower
// index (kind 2) takes that neighbour's flux of the same substep.  Fluxes are
// signed outward on each side; the correction is dt / kappa of the cell.
// One warp per patch, lane k on face cell k, faces in order (-x, +x, -y, +y).
template <typename real, int MX>
__global__ void reflux_pairs_kernel(DevForest<real> D, int p0, int p1,
                                    const real* __restrict__ bflux, const int* __restrict__ pairs,
                                    int cslot, int nfs, double w, double dt) {
  const int lane = threadIdx.x & 31;
  const int p = p0 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (p >= p1) return;  // whole warps leave together
  const int S = D.S;
  real* Q = D.buf[D.cur[D.meta[p].level]] + (size_t)p * S * S;
  const double* K = D.metric + (size_t)p * metric_stride(S);
  for (int dir = 0; dir < 4; ++dir) {
    if (lane < MX) {
      const int* e = pairs + (((size_t)p * 4 + dir) * MX + lane) * 5;
      const int kind = e[0];
      if (kind != 0) {
        const int n = e[1], g = e[2], j0 = e[3], j1 = e[4];
        const double sg = (g & 1) ? 1.0 : -1.0, sf = (dir & 1) ? 1.0 : -1.0;
        double target;
        if (kind == 1) {
          double fsum = 0.0;
          for (int s = 0; s < nfs; ++s) {
            const real* b = bflux + (((size_t)n * 2 + s) * 4 + g) * MX;
            fsum += double(b[j0]) + double(b[j1]);
          }
          target = -sg * (w * fsum);
        } else {
          target = -sg * double(bflux[(((size_t)n * 2 + cslot) * 4 + g) * MX + j0]);
        }
        const double out = sf * double(bflux[(((size_t)p * 2 + cslot) * 4 + dir) * MX + lane]);
        const int i = dir == 0 ? 0 : (dir == 1 ? MX - 1 : lane);
        const int j = dir == 2 ? 0 : (dir == 3 ? MX - 1 : lane);
        const int o = (j + kMbc) * S + (i + kMbc);
        Q[o] = real(double(Q[o]) + dt / K[o] * (out - target));
      }
    }
    __syncwarp();
  }
}

}  // namespace

template <typename real>
cudaError_t launch_reflux(const DevForest<real>& D, int p0, int p1, const real* bflux, int cslot,
                          int nfs, double w, double nu, cudaStream_t s) {
  if (p1 <= p0) return cudaSuccess;
  constexpr int kWarps = 4;
  const int grid = (p1 - p0 + kWarps - 1) / kWarps;
  switch (D.mx) {
    case 8:
      reflux_kernel<real, 8><<<grid, 32 * kWarps, 0, s>>>(D, p0, p1, bflux, cslot, nfs, real(w),
                                                           real(nu));
      break;
    case 16:
      reflux_kernel<real, 16><<<grid, 32 * kWarps, 0, s>>>(D, p0, p1, bflux, cslot, nfs, real(w),
                                                            real(nu));
      break;
    case 32:
      reflux_kernel<real, 32><<<grid, 32 * kWarps, 0, s>>>(D, p0, p1, bflux, cslot, nfs, real(w),
                                                            real(nu));
      break;
    default: return cudaErrorInvalidValue;
  }
  ++launch_counter();
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_tag(const DevForest<real>& D, int kind, double* delta, cudaStream_t s) {
  if (D.npatch <= 0) return cudaSuccess;
  tag_kernel<real><<<grid_for(D.npatch), 256, 0, s>>>(D, kind, delta);
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
cudaError_t launch_poison(const DevForest<real>& D, double value, cudaStream_t s) {
  if (D.npatch <= 0) return cudaSuccess;
  poison_kernel<real><<<1216, 256, 0, s>>>(D, real(value));
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
cudaError_t launch_halo(const DevForest<real>& D, const int* list, int n, real* buf, int pack,
                        cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const size_t total = (size_t)n * D.mx * D.mx;
  const int grid = (int)std::min<size_t>((total + 255) / 256, 1216);
  if (pack)
    halo_pack_kernel<real><<<grid, 256, 0, s>>>(D, list, n, buf);
  else
    halo_unpack_kernel<real><<<grid, 256, 0, s>>>(D, list, n, buf);
  ++launch_counter();
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_add_store(real* dst, const real* src, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  add_store_kernel<real><<<1216, 256, 0, s>>>(dst, src, n);
  ++launch_counter();
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_pack_capacity(const DevForest<real>& D, const int* api_to_dev, double* out,
                                 cudaStream_t s) {
  if (D.npatch <= 0) return cudaSuccess;
  pack_capacity_kernel<real><<<1216, 256, 0, s>>>(D, api_to_dev, out);
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

template <typename real>
cudaError_t launch_reflux_pairs(const DevForest<real>& D, int p0, int p1, const real* bflux,
                                const int* pairs, int cslot, int nfs, double w, double dt,
                                cudaStream_t s) {
  if (p1 <= p0) return cudaSuccess;
  constexpr int kWarps = 4;
  const int grid = (p1 - p0 + kWarps - 1) / kWarps;
  switch (D.mx) {
    case 8:
      reflux_pairs_kernel<real, 8><<<grid, 32 * kWarps, 0, s>>>(D, p0, p1, bflux, pairs, cslot,
                                                                 nfs, w, dt);
      break;
    case 16:
      reflux_pairs_kernel<real, 16><<<grid, 32 * kWarps, 0, s>>>(D, p0, p1, bflux, pairs, cslot,
                                                                  nfs, w, dt);
      break;
    case 32:
      reflux_pairs_kernel<real, 32><<<grid, 32 * kWarps, 0, s>>>(D, p0, p1, bflux, pairs, cslot,
                                                                  nfs, w, dt);
      break;
    default: return cudaErrorInvalidValue;
  }
  ++launch_counter();
  return cudaGetLastError();
}

#define FC_INSTANTIATE(real)                                                                   \
  template cudaError_t launch_tag<real>(const DevForest<real>&, int, double*, cudaStream_t);        \
  template cudaError_t launch_reflux<real>(const DevForest<real>&, int, int, const real*, int, int, \
                                           double, double, cudaStream_t);                          \
  template cudaError_t launch_mass<real>(const DevForest<real>&, const int*, const int*, int, \
                                         double*, double*, cudaStream_t);                      \
  template cudaError_t launch_pack<real>(const DevForest<real>&, const int*, real*, int,      \
                                         cudaStream_t);                                        \
  template cudaError_t launch_unpack<real>(const DevForest<real>&, const int*, const real*,   \
                                           cudaStream_t);                                      \
  template cudaError_t launch_add_store<real>(real*, const real*, size_t, cudaStream_t);      \
  template cudaError_t launch_reflux_pairs<real>(const DevForest<real>&, int, int, const real*, \
                                                 const int*, int, int, double, double,         \
                                                 cudaStream_t);                                \
  template cudaError_t launch_halo<real>(const DevForest<real>&, const int*, int, real*, int,  \
                                        cudaStream_t);                                         \
  template cudaError_t launch_pack_capacity<real>(const DevForest<real>&, const int*, double*, \
                                                  cudaStream_t);                               \
  template cudaError_t launch_remap<real>(const DevForest<real>&, const DevForest<real>&,     \
                                          const RemapEntry*, cudaStream_t);                      \
  template cudaError_t launch_poison<real>(const DevForest<real>&, double, cudaStream_t);

FC_INSTANTIATE(float)
FC_INSTANTIATE(double)

}  // namespace fc

namespace fc {
namespace {
__global__ void set_time_kernel(double* t0_dev, double t0) { *t0_dev = t0; }
__global__ void add_double_kernel(double* dst, const double* src) { *dst += *src; }
}  // namespace

cudaError_t launch_add_double(double* dst, const double* src, cudaStream_t s) {
  add_double_kernel<<<1, 1, 0, s>>>(dst, src);
  ++launch_counter();
  return cudaGetLastError();
}

// Sec. 2.3 (interpolation) with the coarse neighbours' time-interpolated
// cells computed where they are read: for each region of a patch filled
// from a coarser neighbour c (entry e), the ghosts of c that the
// interpolation stencils of the region's ghosts reach beyond the owner's own
// cells, and the rule of c's coarse-neighbour fill for each (from c's face
// entries: copy of a same-size neighbour's cell, average of a finer one's
// 2 x 2 block; a coarser one leaves the tile's value) -- NbrEntry::src and
// code, one thread an entry, written in place (a thread writes its entry's
// src and code and reads only other fields of the entries).  The stencil and
// the wall clamp are interpolate_direct_entry's.  The four ghosts of an
// aligned 2 x 2 group share their coarse cell, its stencil and their block
// of the owner, so one stands for all; along a face only the two end groups
// are visited: a group between them has its stencil inside c but towards
// the owner, where c's ghost is the average of the owner's block beside it,
// as each end group shows for its own.
__global__ void coarse_sources_kernel(NbrEntry* nbr, const PatchMeta* meta, int n, int mx,
                                      int walls) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * 8) return;
  const int p = t >> 3, r = t & 7;
  NbrEntry& e = nbr[t];
  if (e.kind != NB_COARSE) return;
  const PatchMeta o = meta[p];
  const int c = e.n0;
  const int dxr = r == 0 || r == 4 || r == 6 ? -1 : r == 1 || r == 5 || r == 7 ? 1 : 0;
  const int dyr = r == 2 || r == 4 || r == 5 ? -1 : r == 3 || r == 6 || r == 7 ? 1 : 0;
  const int i0 = dxr < 0 ? -2 : dxr > 0 ? mx : 0, i1 = dxr == 0 ? mx : i0 + 2;
  const int j0 = dyr < 0 ? -2 : dyr > 0 ? mx : 0, j1 = dyr == 0 ? mx : j0 + 2;
  const int step_i = r < 4 && dxr == 0 ? mx - 2 : 2, step_j = r < 4 && dyr == 0 ? mx - 2 : 2;
  auto region = [mx](int i, int j) {
    const int dx = i < 0 ? -1 : (i >= mx ? 1 : 0), dy = j < 0 ? -1 : (j >= mx ? 1 : 0);
    if (dy == 0) return dx < 0 ? 0 : 1;
    if (dx == 0) return dy < 0 ? 2 : 3;
    return 4 + (dx > 0 ? 1 : 0) + (dy > 0 ? 2 : 0);
  };
  int ext = 0, cc[2] = {0, 0}, src[2] = {-1, -1}, code[2] = {0, 0};
  bool complete = true;
  for (int j = j0; j < j1 && complete; j += step_j)
    for (int i = i0; i < i1 && complete; i += step_i) {
      bool own = r >= 4;  // a face's group has the owner's block among its reads
      const int2 I = apply_a(e.a, o.x * mx + i, o.y * mx + j);
      const int gx = I.x + e.fx, gy = I.y + e.fy;
      const int ic = (gx >> 1) - e.x0 * mx, jc = (gy >> 1) - e.y0 * mx;
      if (ic < 0 || ic >= mx || jc < 0 || jc >= mx) continue;  // not interpolated
      for (int m = 1; m < 5 && complete; ++m) {
        int ci = ic + (m == 1 ? 1 : m == 2 ? -1 : 0), cj = jc + (m == 3 ? 1 : m == 4 ? -1 : 0);
        if (walls) {  // the exterior ghosts of c are its clamped cells
          const int N = mx << e.lev, X = e.x0 * mx + ci, Y = e.y0 * mx + cj;
          if (X < 0 || X >= N) ci = X < 0 ? 0 : mx - 1;
          if (Y < 0 || Y >= N) cj = Y < 0 ? 0 : mx - 1;
        }
        if (ci >= 0 && ci < mx && cj >= 0 && cj < mx) continue;  // c's interior
        const NbrEntry& f = nbr[(size_t)c * 8 + region(ci, cj)];  // c's fill of (ci, cj)
        int rule = 3, sp = -1, lx = 0, ly = 0;
        if (f.kind == NB_SAME || f.kind == NB_FINE) {
          const int2 H = apply_a(f.a, e.x0 * mx + ci, e.y0 * mx + cj);
          const int hx = H.x + f.fx, hy = H.y + f.fy;
          if (f.kind == NB_SAME) {
            rule = 1;
            sp = f.n0;
            lx = hx - f.x0 * mx;
            ly = hy - f.y0 * mx;
          } else {
            rule = 2;
            sp = f.n0;
            lx = 2 * hx - f.x0 * mx;
            ly = 2 * hy - f.y0 * mx;
            if (lx < 0 || lx >= mx || ly < 0 || ly >= mx) {
              sp = f.n1;
              lx = 2 * hx - f.x1 * mx;
              ly = 2 * hy - f.y1 * mx;
            }
          }
          if (sp < 0 || lx < 0 || lx >= mx || ly < 0 || ly >= mx) {
            complete = false;  // (a malformed entry: the update reads c's)
            break;
          }
        }
        // next to the owner: a block of its own cells, the one the update
        // takes (region r a face; the block beside the ghost's coarse cell,
        // towards the owner)
        if (rule == 2 && sp == p && r < 4) {
          const int bi = r == 0 ? 0 : r == 1 ? mx - 2 : (i & ~1);
          const int bj = r == 2 ? 0 : r == 3 ? mx - 2 : (j & ~1);
          if (lx == bi && ly == bj) {
            own = true;
            continue;
          }
        }
        const int key = (ci + 1) | ((cj + 1) << 6);
        int slot = -1;
        for (int q = 0; q < ext; ++q)
          if (cc[q] == key) slot = q;
        if (slot < 0) {
          if (ext == 2) {
            complete = false;
            break;
          }
          slot = ext++;
          cc[slot] = key;
          src[slot] = sp;
          code[slot] = key | (lx << 12) | (ly << 18) | (rule << 24);
        }
      }
      if (!own) complete = false;
    }
  if (!complete) {  // no list: the update reads c's entries
    src[0] = src[1] = -1;
    code[0] = code[1] = 0;
  }
  e.src[0] = src[0];
  e.src[1] = src[1];
  e.code[0] = code[0] | (complete ? kSrcComplete : 0);
  e.code[1] = code[1];
}

cudaError_t launch_coarse_sources(NbrEntry* nbr, const PatchMeta* meta, int n, int mx, int walls,
                                  cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  coarse_sources_kernel<<<(n * 8 + 255) / 256, 256, 0, s>>>(nbr, meta, n, mx, walls);
  ++launch_counter();
  return cudaGetLastError();
}

// Stores the start time of a replayed coarse step in device memory (one
// thread); kernels captured in a graph read it there.
cudaError_t launch_set_time(double* t0_dev, double t0, cudaStream_t s) {
  set_time_kernel<<<1, 1, 0, s>>>(t0_dev, t0);
  ++launch_counter();
  return cudaGetLastError();
}
}  // namespace fc
