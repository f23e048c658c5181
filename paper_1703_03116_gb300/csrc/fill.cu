// Standalone ghost-cell fill kernels (Alg. 1, Sec. 2.3), one CTA per target
// patch, writing the ghost ring of the patch arrays in HBM.
//
// fill_coarse: phases 1-2 -- copy from same-size neighbours, average fine
//   neighbours, then the physical boundary condition.  Patches on the
//   time-interpolated level also receive their interior (1 - alpha) q_old +
//   alpha q_new (multirate: the coarse data a finer level interpolates from).
// fill_fine: phases 3-4 -- interpolation from the coarser neighbour, then
//   the boundary condition again.
// On the cubed sphere the corner ghosts beyond a cube vertex are set last,
// by whichever kernel finishes the patch's edge ghosts.
//
// The rules themselves live in ghost_gather.cuh, shared with the patch-update
// kernels, which apply them to the tile they hold in shared memory.
#include "ghost_gather.cuh"

namespace fc {
namespace {

template <typename real, int MX>
__global__ void __launch_bounds__(256) fill_coarse_kernel(DevForest<real> D, FillArgs A) {
  constexpr int S = MX + 4;
  __shared__ NbrStage st;
  const real alpha = real(A.alpha);
  for (int t = blockIdx.x; t < A.ntargets; t += gridDim.x) {
    const int p = A.targets[t];
    stage_neighbours(D.meta, D.nbr, p, st, threadIdx.x);
    const PatchMeta pm = D.meta[p];
    __syncthreads();
    real* Q = patch_ptr((pm.level == A.tlevel) ? D.qT : D.buf[D.cur[pm.level]], p, S);
    if (pm.level == A.tlevel) {
      if (A.full_interior) {
        for (int k = threadIdx.x; k < MX * MX; k += blockDim.x) {
          const int i = k % MX, j = k / MX;
          Q[(j + kMbc) * S + i + kMbc] = src_interior(D, A.tlevel, alpha, p, pm.level, i, j);
        }
      } else {
        // the cells within two of the patch's edge: rows 0, 1, MX-2, MX-1,
        // then columns 0, 1, MX-2, MX-1 of the rows between
        constexpr int NR = 4 * MX + 4 * (MX - 4);
        for (int k = threadIdx.x; k < NR; k += blockDim.x) {
          int i, j;
          if (k < 4 * MX) {
            const int r = k / MX;
            j = r < 2 ? r : MX - 4 + r;
            i = k % MX;
          } else {
            const int c = (k - 4 * MX) & 3;
            j = 2 + ((k - 4 * MX) >> 2);
            i = c < 2 ? c : MX - 4 + c;
          }
          Q[(j + kMbc) * S + i + kMbc] = src_interior(D, A.tlevel, alpha, p, pm.level, i, j);
        }
      }
    }
    for (int k = threadIdx.x; k < num_ghosts<MX>(); k += blockDim.x) {
      int i, j;
      ghost_ij<MX>(k, i, j);
      real v;
      if (copy_or_average<real, MX>(D, st, pm, A.tlevel, alpha, i, j, v))
        Q[(j + kMbc) * S + i + kMbc] = v;
    }
    if (D.domain == FC_DOMAIN_WALLS) {
      __syncthreads();
      wall_bc<real, MX>(pm, Q, threadIdx.x, blockDim.x);
    }
    if (D.domain == FC_DOMAIN_SPHERE && !(pm.flags & 1)) {  // edge ghosts are final
      __syncthreads();
      corner3_fill<real, MX>(st, Q, threadIdx.x, blockDim.x);
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
    stage_neighbours(D.meta, D.nbr, p, st, threadIdx.x);
    const PatchMeta pm = D.meta[p];
    __syncthreads();
    real* Q = patch_ptr((pm.level == A.tlevel) ? D.qT : D.buf[D.cur[pm.level]], p, S);
    for (int k = threadIdx.x; k < num_ghosts<MX>(); k += blockDim.x) {
      int i, j;
      ghost_ij<MX>(k, i, j);
      real v;
      if (interpolate<real, MX>(D, st, pm, A.tlevel, i, j, v)) Q[(j + kMbc) * S + i + kMbc] = v;
    }
    if (D.domain == FC_DOMAIN_WALLS) {
      __syncthreads();
      wall_bc<real, MX>(pm, Q, threadIdx.x, blockDim.x);
    }
    if (D.domain == FC_DOMAIN_SPHERE) {
      __syncthreads();
      corner3_fill<real, MX>(st, Q, threadIdx.x, blockDim.x);
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
