// Ghost-cell fill kernels (Alg. 1, Sec. 2.3), one CTA per target patch.
//
// fill_coarse: phases 1-2 -- copy from same-size neighbours (Eq. transform),
//   average four fine cells (Eq. ghost_coarse), then the physical boundary
//   condition.  Patches on the time-interpolated level also receive their
//   interior (1 - alpha) q_old + alpha q_new.
// fill_fine: phases 3-4 -- interpolate from the coarser neighbour (Eq.
//   ghost_fine, minmod-limited one-sided slopes in the coarse index space),
//   then the boundary condition again.
//
// The eight face/corner entries of the target and the layout of their
// neighbour patches are staged in shared memory once per patch, so each
// ghost cell costs one dependent load of source data.
#include "device_util.cuh"

namespace fc {
namespace {

struct NbrStage {
  NbrEntry e[8];
  PatchMeta m0[8], m1[8];
  PatchMeta self;
};

__device__ __forceinline__ void stage_neighbours(const PatchMeta* meta, const NbrEntry* nbr,
                                                 int p, NbrStage& st) {
  const int t = threadIdx.x;
  if (t < 8) {
    const NbrEntry e = nbr[(size_t)p * 8 + t];
    st.e[t] = e;
    if (e.n0 >= 0) st.m0[t] = meta[e.n0];
    if (e.n1 >= 0) st.m1[t] = meta[e.n1];
  } else if (t == 8) {
    st.self = meta[p];
  }
}

// source value for copy/average: interior cell of patch n, time-interpolated
// when n lies on the level read through the interpolation buffer
template <typename real>
__device__ __forceinline__ real src_interior(const DevForest<real>& D, int tlevel, real alpha,
                                             int n, int nlev, int i, int j) {
  const size_t o = (size_t)n * D.S * D.S + (size_t)(j + kMbc) * D.S + (i + kMbc);
  const int c = D.cur[nlev];
  if (nlev == tlevel) return (real(1) - alpha) * D.buf[c ^ 1][o] + alpha * D.buf[c][o];
  return D.buf[c][o];
}

// zeroth-order extrapolation at walls: an exterior ghost copies the owner's
// cell with each out-of-domain index clamped to the nearest interior index
template <typename real, int MX>
__device__ __forceinline__ void wall_bc(const PatchMeta& pm, real* Q) {
  constexpr int S = MX + 4;
  const int N = MX << pm.level;
  for (int k = threadIdx.x; k < num_ghosts<MX>(); k += blockDim.x) {
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

template <typename real, int MX>
__global__ void __launch_bounds__(256) fill_coarse_kernel(DevForest<real> D, FillArgs A) {
  constexpr int S = MX + 4;
  __shared__ NbrStage st;
  const real alpha = real(A.alpha);
  for (int t = blockIdx.x; t < A.ntargets; t += gridDim.x) {
    const int p = A.targets[t];
    stage_neighbours(D.meta, D.nbr, p, st);
    __syncthreads();
    const PatchMeta pm = st.self;
    real* Q = patch_ptr((pm.level == A.tlevel) ? D.qT : D.buf[D.cur[pm.level]], p, S);
    if (pm.level == A.tlevel) {
      for (int k = threadIdx.x; k < MX * MX; k += blockDim.x) {
        const int i = k % MX, j = k / MX;
        Q[(j + kMbc) * S + i + kMbc] = src_interior(D, A.tlevel, alpha, p, pm.level, i, j);
      }
    }
    for (int k = threadIdx.x; k < num_ghosts<MX>(); k += blockDim.x) {
      int i, j;
      ghost_ij<MX>(k, i, j);
      const int r = region_of<MX>(i, j);
      const NbrEntry& e = st.e[r];
      if (e.kind != NB_SAME && e.kind != NB_FINE) continue;
      const int2 Ip = apply_a(e.a, pm.x * MX + i, pm.y * MX + j);
      const int gx = Ip.x + e.fx, gy = Ip.y + e.fy;
      real v;
      if (e.kind == NB_SAME) {
        const PatchMeta& nm = st.m0[r];
        const int lx = gx - nm.x * MX, ly = gy - nm.y * MX;
        if (lx < 0 || lx >= MX || ly < 0 || ly >= MX) continue;  // malformed entry
        v = src_interior(D, A.tlevel, alpha, e.n0, nm.level, lx, ly);
      } else {
        int n = e.n0;
        const PatchMeta* nm = &st.m0[r];
        int lx = 2 * gx - nm->x * MX, ly = 2 * gy - nm->y * MX;
        if (lx < 0 || lx >= MX || ly < 0 || ly >= MX) {
          if (e.n1 < 0) continue;  // malformed entry
          n = e.n1;
          nm = &st.m1[r];
          lx = 2 * gx - nm->x * MX;
          ly = 2 * gy - nm->y * MX;
          if (lx < 0 || lx >= MX || ly < 0 || ly >= MX) continue;
        }
        real s[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int2 d = apply_a(e.a, (q & 1) ? 1 : -1, (q & 2) ? 1 : -1);
          s[q] = src_interior(D, A.tlevel, alpha, n, nm->level, lx + (d.x > 0), ly + (d.y > 0));
        }
        v = real(0.25) * (((s[0] + s[1]) + s[2]) + s[3]);
      }
      Q[(j + kMbc) * S + i + kMbc] = v;
    }
    if (D.domain == FC_DOMAIN_WALLS) {
      __syncthreads();
      wall_bc<real, MX>(pm, Q);
    }
    __syncthreads();
  }
}

template <typename real, int MX>
__global__ void __launch_bounds__(256) fill_fine_kernel(DevForest<real> D, FillArgs A) {
  constexpr int S = MX + 4;
  __shared__ NbrStage st;
  for (int t = blockIdx.x; t < A.ntargets; t += gridDim.x) {
    const int p = A.targets[t];
    stage_neighbours(D.meta, D.nbr, p, st);
    __syncthreads();
    const PatchMeta pm = st.self;
    real* Q = patch_ptr((pm.level == A.tlevel) ? D.qT : D.buf[D.cur[pm.level]], p, S);
    for (int k = threadIdx.x; k < num_ghosts<MX>(); k += blockDim.x) {
      int i, j;
      ghost_ij<MX>(k, i, j);
      const int r = region_of<MX>(i, j);
      const NbrEntry& e = st.e[r];
      if (e.kind != NB_COARSE) continue;
      const int2 Ip = apply_a(e.a, pm.x * MX + i, pm.y * MX + j);
      const int gx = Ip.x + e.fx, gy = Ip.y + e.fy;
      const PatchMeta& nm = st.m0[r];
      const int ic = (gx >> 1) - nm.x * MX, jc = (gy >> 1) - nm.y * MX;
      if (ic < 0 || ic >= MX || jc < 0 || jc >= MX) continue;  // malformed entry
      const real dx = (gx & 1) ? real(1) : real(-1);
      const real dy = (gy & 1) ? real(1) : real(-1);
      const real* C = patch_ptr(nm.level == A.tlevel ? D.qT : D.buf[D.cur[nm.level]], e.n0, S) +
                      (jc + kMbc) * S + ic + kMbc;
      const real q0 = C[0];
      const real sx = minmod(C[1] - q0, q0 - C[-1]);
      const real sy = minmod(C[S] - q0, q0 - C[-S]);
      Q[(j + kMbc) * S + i + kMbc] = q0 + real(0.25) * (sx * dx + sy * dy);
    }
    if (D.domain == FC_DOMAIN_WALLS) {
      __syncthreads();
      wall_bc<real, MX>(pm, Q);
    }
    __syncthreads();
  }
}

inline int grid_for(int n) { return n < 1 ? 1 : (n < 65535 * 8 ? n : 65535 * 8); }

template <typename real, int MX>
cudaError_t fill_mx(const DevForest<real>& D, const FillArgs& A, bool fine, cudaStream_t s) {
  constexpr int threads = MX >= 32 ? 256 : 128;
  if (fine)
    fill_fine_kernel<real, MX><<<grid_for(A.ntargets), threads, 0, s>>>(D, A);
  else
    fill_coarse_kernel<real, MX><<<grid_for(A.ntargets), threads, 0, s>>>(D, A);
  ++launch_counter();
  return cudaGetLastError();
}

template <typename real>
cudaError_t fill_dispatch(const DevForest<real>& D, const FillArgs& A, bool fine,
                          cudaStream_t s) {
  if (A.ntargets <= 0) return cudaSuccess;
  switch (D.mx) {
    case 8: return fill_mx<real, 8>(D, A, fine, s);
    case 16: return fill_mx<real, 16>(D, A, fine, s);
    case 32: return fill_mx<real, 32>(D, A, fine, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

template <typename real>
cudaError_t launch_fill_coarse(const DevForest<real>& D, const FillArgs& A, cudaStream_t s) {
  return fill_dispatch(D, A, false, s);
}

template <typename real>
cudaError_t launch_fill_fine(const DevForest<real>& D, const FillArgs& A, cudaStream_t s) {
  return fill_dispatch(D, A, true, s);
}

template cudaError_t launch_fill_coarse<float>(const DevForest<float>&, const FillArgs&,
                                               cudaStream_t);
template cudaError_t launch_fill_coarse<double>(const DevForest<double>&, const FillArgs&,
                                                cudaStream_t);
template cudaError_t launch_fill_fine<float>(const DevForest<float>&, const FillArgs&,
                                             cudaStream_t);
template cudaError_t launch_fill_fine<double>(const DevForest<double>&, const FillArgs&,
                                              cudaStream_t);

}  // namespace fc
