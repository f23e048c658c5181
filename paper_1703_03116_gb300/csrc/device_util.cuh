// Small device helpers shared by the kernels of this library.
#pragma once

#include "fc_internal.hpp"

namespace fc {

template <typename real>
__device__ __forceinline__ real minmod(real a, real b) {
  if (a * b <= real(0)) return real(0);
  return fabs(a) < fabs(b) ? a : b;
}

// Signed permutation A of Eq. (transform): bit 0 swaps the axes, bits 1 and
// 2 negate the first and second output component.
__device__ __forceinline__ int2 apply_a(int a, int x, int y) {
  int u = (a & 1) ? y : x;
  int v = (a & 1) ? x : y;
  if (a & 2) u = -u;
  if (a & 4) v = -v;
  return make_int2(u, v);
}

// k-th ghost cell of an MX x MX patch with two ghost layers: rows -2, -1 and
// MX, MX+1 (full width), then columns -2, -1, MX, MX+1 of the interior rows.
template <int MX>
__device__ __forceinline__ void ghost_ij(int k, int& i, int& j) {
  constexpr int S = MX + 4;
  if (k < 2 * S) {
    j = k / S - 2;
    i = k % S - 2;
    return;
  }
  k -= 2 * S;
  if (k < 2 * S) {
    j = MX + k / S;
    i = k % S - 2;
    return;
  }
  k -= 2 * S;
  j = k >> 2;
  const int c = k & 3;
  i = c < 2 ? c - 2 : MX + c - 2;
}

template <int MX>
__host__ __device__ constexpr int num_ghosts() {
  return 4 * (MX + 4) + 4 * MX;
}

// face / corner region of a ghost cell, in the order of kDirX/kDirY
template <int MX>
__device__ __forceinline__ int region_of(int i, int j) {
  const int dx = i < 0 ? -1 : (i >= MX ? 1 : 0);
  const int dy = j < 0 ? -1 : (j >= MX ? 1 : 0);
  if (dy == 0) return dx < 0 ? 0 : 1;
  if (dx == 0) return dy < 0 ? 2 : 3;
  return 4 + (dx > 0 ? 1 : 0) + (dy > 0 ? 2 : 0);
}

template <typename real>
__device__ __forceinline__ real* patch_ptr(real* base, int p, int S) {
  return base + (size_t)p * S * S;
}

// ---------------------------------------------------------------- TMA / mbarrier

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// bounded wait: gives up after `limit` polls (each poll may suspend briefly)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}


// 1D bulk copy global -> shared (TMA), completion counted on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst_smem)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <typename real>
__device__ __forceinline__ real sinpi_r(real x);
template <>
__device__ __forceinline__ float sinpi_r<float>(float x) { return sinpif(x); }
template <>
__device__ __forceinline__ double sinpi_r<double>(double x) { return sinpi(x); }

// cos(pi t / T) in the field's precision (a CTA evaluates it once, on one
// thread, while the others wait: FP64 is slow on this GPU)
template <typename real>
__device__ __forceinline__ real cospi_ratio(double t, double T);
template <>
__device__ __forceinline__ float cospi_ratio<float>(double t, double T) {
  return cospif(float(t) / float(T));
}
template <>
__device__ __forceinline__ double cospi_ratio<double>(double t, double T) { return cospi(t / T); }

// phi(W_up / W) W for the MC limiter without a division:
// 0 unless W and W_up share a sign, else sign(W) min(|W + W_up|/2, 2|W|, 2|W_up|)
template <typename real>
__device__ __forceinline__ real mc_limited(real W, real Wup) {
  const real m = fmin(real(0.5) * fabs(W + Wup), real(2) * fmin(fabs(W), fabs(Wup)));
  return (W * Wup > real(0)) ? copysign(m, W) : real(0);
}

}  // namespace fc
