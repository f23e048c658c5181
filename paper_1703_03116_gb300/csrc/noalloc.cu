// Mass reduction that allocates nothing: fc_mass_noalloc.
//
// Some callers cannot allocate device memory at the point where they need a
// mass sum -- for example code running inside a host allocator callback, a
// process whose device memory is carved up by another runtime, or a driver
// loop that must not touch the allocator once it is running.  This entry
// point takes a packed field that the caller already holds on the device and
// keeps its per-leaf partial sums in a fixed, file-scope device array instead
// of forest-owned scratch.  It is the same two-stage FP64 reduction as
// fc_forest_mass: one CTA per leaf sums its cells (weighted by the caller's
// cell capacities when given) in a fixed order, then one CTA per forest sums
// its leaves in a fixed order.
#include <cstdint>
#include <mutex>

#include "fc_internal.hpp"

namespace fc {
namespace {

// Per-leaf partial sums.  Every GPU that loads this library keeps this array
// (FC_NOALLOC_MAX_LEAVES doubles) until the process exits.  A call writes
// slots [0, nleaves) and its forest totals read only slots in that range (a
// forest_start entry outside [0, nleaves] is clamped into it), so no slot
// left by an earlier call is read and nothing needs clearing; calls whose
// work overlaps on the GPU share the array and race.
static __device__ __align__(256) double g_leaf_sums[FC_NOALLOC_MAX_LEAVES];

template <typename real>
__global__ void leaf_sum_kernel(const real* q, const double* capacity, int mx, int nleaves,
                                const int* level, double* sums) {
  __shared__ double red[256];
  const int cells = mx * mx;
  for (int k = blockIdx.x; k < nleaves; k += gridDim.x) {
    const real* Q = q + (size_t)k * cells;
    double s = 0.0;
    if (capacity) {  // mapped grid: sum of kappa q, in fc_forest_mass's order
      const double* K = capacity + (size_t)k * cells;
      for (int c = threadIdx.x; c < cells; c += blockDim.x) s += K[c] * (double)Q[c];
    } else {
      for (int c = threadIdx.x; c < cells; c += blockDim.x) s += (double)Q[c];
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const double h = ldexp(1.0, -level[k]) / mx;
      sums[k] = capacity ? red[0] : h * h * red[0];
    }
    __syncthreads();
  }
}

__global__ void forest_total_kernel(const double* sums, const int* fstart, int nforests,
                                    int nleaves, double* out) {
  __shared__ double red[256];
  for (int f = blockIdx.x; f < nforests; f += gridDim.x) {
    // a malformed table reads no slot outside this call's [0, nleaves)
    const int k0 = min(max(fstart[f], 0), nleaves), k1 = min(max(fstart[f + 1], k0), nleaves);
    double s = 0.0;
    for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) s += sums[k];
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

// Device address of g_leaf_sums, looked up once per device with that device
// current.  Host code must not pass the symbol itself: on the host it names a
// stand-in, not device memory.
constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
double* g_addr[kMaxDevices] = {nullptr};

cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_leaf_sums);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

cudaError_t noalloc_mass(const void* q, const double* capacity, int dtype, int mx, int nleaves,
                         const int* level, const int* fstart, int nforests, double* out,
                         cudaStream_t s) {
  double* sums = nullptr;
  cudaError_t e = scratch_address(&sums);
  if (e != cudaSuccess) return e;
  const int g1 = nleaves < 4096 ? nleaves : 4096;
  if (dtype == FC_F32)
    leaf_sum_kernel<float><<<g1, 256, 0, s>>>(static_cast<const float*>(q), capacity, mx,
                                              nleaves, level, sums);
  else
    leaf_sum_kernel<double><<<g1, 256, 0, s>>>(static_cast<const double*>(q), capacity, mx,
                                               nleaves, level, sums);
  ++launch_counter();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int g2 = nforests < 4096 ? nforests : 4096;
  forest_total_kernel<<<g2, 256, 0, s>>>(sums, fstart, nforests, nleaves, out);
  ++launch_counter();
  return cudaGetLastError();
}

}  // namespace fc
