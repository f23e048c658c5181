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

}  // namespace fc
