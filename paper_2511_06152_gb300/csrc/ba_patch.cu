// Patch transfer between images (Sec. 3.1): the patch centres of image 0
// moved to images k, either through the GNSS/IMU poses at a nominal depth
// (Eq. 3) or by the footprints' in-plane rotation and displacement (Eq. 4).
// One thread per (patch, target image); binary64.  Outputs are [m][n]
// arrays of target-major order, so that each target image's patches are
// contiguous and the stores coalesce.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ba_internal.h"

namespace bagpu {

namespace {

// Eq. 3: X = T_0 + lambda R_0 K_0^-1 [u v 1]^T (lambda: depth along image 0's
// optical axis), seen by image k: pi(K_k R_k^T (X - T_k)); K is the pinhole
// part (f, cx, cy) of the intrinsics, as Eq. 3 has no distortion term.  A
// point behind image k gives NaN and inside = 0; inside = 1 when the
// transferred centre lies in [0, width) x [0, height).
__global__ void k_patch_poses(int n, const double2* __restrict__ p0, const double* __restrict__ intr0,
                              const double* __restrict__ R0, const double* __restrict__ T0, double lambda, int m,
                              const double* __restrict__ intr, const double* __restrict__ R,
                              const double* __restrict__ T, double width, double height, double2* __restrict__ p,
                              uint8_t* __restrict__ inside) {
  const double f0i = 1.0 / intr0[0], cx0 = intr0[1], cy0 = intr0[2];
  for (int k = blockIdx.y; k < m; k += gridDim.y) {
    const double* Rk = R + 9 * (size_t)k;
    const double* Tk = T + 3 * (size_t)k;
    const double fk = intr[7 * (size_t)k], cxk = intr[7 * (size_t)k + 1], cyk = intr[7 * (size_t)k + 2];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      const double2 q = p0[i];
      const double r0 = (q.x - cx0) * f0i, r1 = (q.y - cy0) * f0i;  // K_0^-1 p_bar = (r0, r1, 1)
      double d[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) d[a] = T0[a] + lambda * (R0[3 * a] * r0 + R0[3 * a + 1] * r1 + R0[3 * a + 2]) - Tk[a];
      const double x = Rk[0] * d[0] + Rk[3] * d[1] + Rk[6] * d[2];  // R_k^T (X - T_k)
      const double y = Rk[1] * d[0] + Rk[4] * d[1] + Rk[7] * d[2];
      const double z = Rk[2] * d[0] + Rk[5] * d[1] + Rk[8] * d[2];
      double2 out = make_double2(nan(""), nan(""));
      uint8_t in = 0;
      if (z > 0.0) {
        const double iz = 1.0 / z;
        out = make_double2(fk * x * iz + cxk, fk * y * iz + cyk);
        in = out.x >= 0.0 && out.x < width && out.y >= 0.0 && out.y < height;
      }
      const size_t o = (size_t)k * n + i;
      p[o] = out;
      if (inside) inside[o] = in;
    }
  }
}

// Eq. 4: q_k = R(theta_k) (q_0 - c) + c + g_k - g_0, R(theta) = [cos -sin; sin cos]
// (the sine and cosine of each target image once, in shared memory).
__global__ void k_patch_planar(int n, const double2* __restrict__ q0, double cx, double cy, double g0x, double g0y,
                               int m, const double* __restrict__ theta, const double2* __restrict__ g,
                               double2* __restrict__ q) {
  __shared__ double cs[2];
  for (int k = blockIdx.y; k < m; k += gridDim.y) {
    __syncthreads();  // the previous target's cs is no longer read
    if (threadIdx.x == 0) sincos(theta[k], &cs[1], &cs[0]);
    __syncthreads();
    const double c = cs[0], s = cs[1];
    const double2 gk = g[k];
    const double tx = cx + gk.x - g0x, ty = cy + gk.y - g0y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      const double2 a = q0[i];
      const double dx = a.x - cx, dy = a.y - cy;
      q[(size_t)k * n + i] = make_double2((c * dx - s * dy) + tx, (s * dx + c * dy) + ty);
    }
  }
}

dim3 patch_grid(int n, int m) {
  const int bx = (n + 255) / 256;
  return dim3(bx < 1 ? 1 : (bx > 1024 ? 1024 : bx), m < 1 ? 1 : (m > 65535 ? 65535 : m));
}

}  // namespace

void launch_patch_poses(int n, const double* p0, const double* intr0, const double* R0, const double* T0,
                        double lambda, int m, const double* intr, const double* R, const double* T, double width,
                        double height, double* p, uint8_t* inside, cudaStream_t st) {
  LAUNCH(KK_OTHER, st,
         k_patch_poses<<<patch_grid(n, m), 256, 0, st>>>(n, reinterpret_cast<const double2*>(p0), intr0, R0, T0,
                                                            lambda, m, intr, R, T, width, height,
                                                            reinterpret_cast<double2*>(p), inside));
}

void launch_patch_planar(int n, const double* q0, const double* c, const double* g0, int m, const double* theta,
                         const double* g, double* q, cudaStream_t st) {
  LAUNCH(KK_OTHER, st,
         k_patch_planar<<<patch_grid(n, m), 256, 0, st>>>(n, reinterpret_cast<const double2*>(q0), c[0], c[1], g0[0],
                                                             g0[1], m, theta, reinterpret_cast<const double2*>(g),
                                                             reinterpret_cast<double2*>(q)));
}

}  // namespace bagpu
