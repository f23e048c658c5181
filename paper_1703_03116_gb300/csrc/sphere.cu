// Cubed-sphere metric terms (Sec. 5.3: advection on the mapped unit sphere).
//
// The wave-propagation update on a mapped grid runs in capacity form: each
// cell carries its area kappa on the sphere, each edge the volume flux of
// the velocity through it.  For the solid-body rotation u = omega x X the
// velocity has the stream function psi = -omega . X on the unit sphere, so
// the flux through an edge is a difference of psi at its two end points;
// across an x-edge (from its lower end a to its upper end b) it is
// omega . (X_b - X_a), across a y-edge (from its left end a to its right end
// b) omega . (X_a - X_b), positive along +x and +y.  The difference is taken
// of the end points before the dot product (psi itself is O(1), the flux
// O(h)).  Cells are bounded by great circles (gnomonic grid lines), so the
// area is exactly that of two spherical triangles, each by the formula of
// Van Oosterom and Strackee (1983): tan(E/2) = |a . (b x c)| /
// (1 + a.b + b.c + c.a).
//
// The metrics of a patch cover its ghost cells too (the patch's own mapping
// extended past its block), are computed in FP64 once per layout, and are
// stored per patch in the order kappa, phi_x, phi_y (metric_stride doubles).
//
// The deformational flow of Sec. 5.3 has a time-dependent streamfunction
// psi = k sin^2(rho - 2 pi t/T) cos^2(theta) cos(pi t/T) - 2 pi sin(theta)/T_f.
// With s = Y cos a - X sin a (a = 2 pi t/T), which is sin(rho - a) cos(theta),
// and sin(theta) = Z, psi = k c s^2 - (2 pi/T_f) Z (c = cos(pi t/T)); an edge
// flux psi(b) - psi(a) = k c (s_b - s_a)(s_b + s_a) - (2 pi/T_f)(Z_b - Z_a) is
// again formed from the end points' differences.  Its fluxes are refreshed
// for each substep's half time from the corners kept per patch.
#include <atomic>
#include <cmath>

#include "device_util.cuh"

namespace fc {
namespace {

__device__ __forceinline__ double axis_component(int code, int k) {
  return (code == k + 1) ? 1.0 : (code == -(k + 1)) ? -1.0 : 0.0;
}

// the triple product as a . ((b - a) x (c - a)): equal to a . (b x c), but
// without cancelling from O(1) terms down to O(h^2) for a small triangle
__device__ __forceinline__ double tri_area(const double* a, const double* b, const double* c) {
  const double u0 = b[0] - a[0], u1 = b[1] - a[1], u2 = b[2] - a[2];
  const double v0 = c[0] - a[0], v1 = c[1] - a[1], v2 = c[2] - a[2];
  const double w0 = u1 * v2 - u2 * v1;
  const double w1 = u2 * v0 - u0 * v2;
  const double w2 = u0 * v1 - u1 * v0;
  const double num = fabs(a[0] * w0 + a[1] * w1 + a[2] * w2);
  const double ab = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
  const double bcd = b[0] * c[0] + b[1] * c[1] + b[2] * c[2];
  const double ca = c[0] * a[0] + c[1] * a[1] + c[2] * a[2];
  return 2.0 * atan2(num, 1.0 + ab + bcd + ca);
}

// one CTA per patch; X: the (S+1)^2 grid corners on the sphere, in shared
// memory as three planes.  After a regrid (rm != null) a patch that kept its
// quadrant copies its block from the old layout's store instead.
__global__ void __launch_bounds__(256) metrics_kernel(const PatchMeta* meta, int npatch, int mx,
                                                      double w0, double w1, double w2,
                                                      double* metric, const RemapEntry* rm,
                                                      const double* old_metric,
                                                      double* corner_out) {
  extern __shared__ double Xs[];
  const int S = mx + 2 * kMbc, SN = S + 1;
  double* X0 = Xs;
  double* X1 = X0 + SN * SN;
  double* X2 = X1 + SN * SN;
  for (int p = blockIdx.x; p < npatch; p += gridDim.x) {
    if (rm && rm[p].kind == RM_COPY) {
      const double2* src =
          reinterpret_cast<const double2*>(old_metric + (size_t)rm[p].src[0] * metric_stride(S));
      double2* dst = reinterpret_cast<double2*>(metric + (size_t)p * metric_stride(S));
      for (int k = threadIdx.x; k < metric_stride(S) / 2; k += blockDim.x) dst[k] = src[k];
      continue;
    }
    const PatchMeta pm = meta[p];
    int n, ex, ey;
    cube_face(pm.block, &n, &ex, &ey);
    const double h = 1.0 / ldexp((double)mx, pm.level);
    for (int k = threadIdx.x; k < SN * SN; k += blockDim.x) {
      const int i = k % SN, j = k / SN;
      const double x = ((double)pm.x * mx + (i - kMbc)) * h;
      const double y = ((double)pm.y * mx + (j - kMbc)) * h;
      const double ta = tan((x - 0.5) * M_PI / 2.0), tb = tan((y - 0.5) * M_PI / 2.0);
      double P[3];
      for (int c = 0; c < 3; ++c)
        P[c] = axis_component(n, c) + ta * axis_component(ex, c) + tb * axis_component(ey, c);
      const double len = sqrt(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
      X0[k] = P[0] / len;
      X1[k] = P[1] / len;
      X2[k] = P[2] / len;
      if (corner_out) {
        double* C = corner_out + (size_t)p * 3 * SN * SN;
        C[k] = X0[k];
        C[SN * SN + k] = X1[k];
        C[2 * SN * SN + k] = X2[k];
      }
    }
    __syncthreads();
    double* K = metric + (size_t)p * metric_stride(S);
    double* PX = K + S * S;
    double* PY = PX + S * SN;
    auto corner = [&](int i, int j, double* v) {
      const int k = j * SN + i;
      v[0] = X0[k];
      v[1] = X1[k];
      v[2] = X2[k];
    };
    for (int k = threadIdx.x; k < S * S; k += blockDim.x) {
      const int i = k % S, j = k / S;
      double a[3], b[3], c[3], d[3];
      corner(i, j, a);
      corner(i + 1, j, b);
      corner(i + 1, j + 1, c);
      corner(i, j + 1, d);
      K[k] = tri_area(a, b, c) + tri_area(a, c, d);
    }
    for (int k = threadIdx.x; k < S * SN; k += blockDim.x) {
      // x-edge i-1/2 of row j: corners (i, j) below, (i, j+1) above
      const int i = k % SN, j = k / SN;
      double a[3], b[3];
      corner(i, j, a);
      corner(i, j + 1, b);
      PX[k] = w0 * (b[0] - a[0]) + w1 * (b[1] - a[1]) + w2 * (b[2] - a[2]);
    }
    for (int k = threadIdx.x; k < SN * S; k += blockDim.x) {
      // y-edge j-1/2 of column i: corners (i, j) left, (i+1, j) right
      const int i = k % S, j = k / S;
      double a[3], b[3];
      corner(i, j, a);
      corner(i + 1, j, b);
      PY[k] = w0 * (a[0] - b[0]) + w1 * (a[1] - b[1]) + w2 * (a[2] - b[2]);
    }
    __syncthreads();
  }
}

// one CTA per patch of [p0, p1): phi_x, phi_y of its metric block at time t
__global__ void __launch_bounds__(256) deform_fluxes_kernel(int p0, int p1, int mx,
                                                            const double* __restrict__ corner,
                                                            double* metric, double kc, double T,
                                                            double rot, double t_half,
                                                            const double* t0_dev, double t_off) {
  const double t = t0_dev ? *t0_dev + t_off : t_half;
  const double a = 2.0 * M_PI * t / T;
  const double ca = cos(a), sa = sin(a), kcc = kc * cos(M_PI * t / T);
  const int S = mx + 2 * kMbc, SN = S + 1;
  for (int p = p0 + blockIdx.x; p < p1; p += gridDim.x) {
    const double* X0 = corner + (size_t)p * 3 * SN * SN;
    const double* X1 = X0 + SN * SN;
    const double* X2 = X1 + SN * SN;
    double* PX = metric + (size_t)p * metric_stride(S) + S * S;
    double* PY = PX + S * SN;
    // psi(corner kb) - psi(corner ka)
    auto dpsi = [&](int ka, int kb) -> double {
      const double ds = (X1[kb] - X1[ka]) * ca - (X0[kb] - X0[ka]) * sa;
      const double ss = (X1[kb] + X1[ka]) * ca - (X0[kb] + X0[ka]) * sa;
      return kcc * (ds * ss) - rot * (X2[kb] - X2[ka]);
    };
    for (int k = threadIdx.x; k < S * SN; k += blockDim.x) {
      // x-edge i-1/2 of row j: psi(corner (i, j)) - psi(corner (i, j+1))
      const int i = k % SN, j = k / SN;
      PX[k] = dpsi((j + 1) * SN + i, j * SN + i);
    }
    for (int k = threadIdx.x; k < SN * S; k += blockDim.x) {
      // y-edge j-1/2 of column i: psi(corner (i+1, j)) - psi(corner (i, j))
      const int i = k % S, j = k / S;
      PY[k] = dpsi(j * SN + i, j * SN + i + 1);
    }
  }
}

}  // namespace

cudaError_t launch_deform_fluxes(int p0, int p1, int mx, const double* corner, double* metric,
                                 double kc, double T, double rot, double t_half,
                                 const double* t0_dev, double t_off, cudaStream_t s) {
  if (p1 <= p0) return cudaSuccess;
  const int grid = p1 - p0 < 65535 * 8 ? p1 - p0 : 65535 * 8;
  deform_fluxes_kernel<<<grid, 256, 0, s>>>(p0, p1, mx, corner, metric, kc, T, rot, t_half,
                                            t0_dev, t_off);
  ++launch_counter();
  return cudaGetLastError();
}

cudaError_t launch_sphere_metrics(const PatchMeta* meta, int npatch, int mx, const double* omega,
                                  double* metric, const RemapEntry* rm, const double* old_metric,
                                  double* corner_out, cudaStream_t s) {
  if (npatch <= 0) return cudaSuccess;
  const int SN = mx + 2 * kMbc + 1;
  const size_t smem = sizeof(double) * 3 * (size_t)SN * SN;
  // set once per process; concurrent first calls both set it (idempotent)
  static std::atomic<bool> attr_set{false};
  if (!attr_set.load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(metrics_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    if (e != cudaSuccess) return e;
    attr_set.store(true, std::memory_order_release);
  }
  if (smem > 64 * 1024) return cudaErrorInvalidValue;
  const int grid = npatch < 65535 * 8 ? npatch : 65535 * 8;
  metrics_kernel<<<grid, 256, smem, s>>>(meta, npatch, mx, omega[0], omega[1], omega[2], metric,
                                         rm, old_metric, corner_out);
  ++launch_counter();
  return cudaGetLastError();
}

}  // namespace fc
