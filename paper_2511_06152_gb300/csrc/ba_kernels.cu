// Kernels of one LM iteration, batched over many clusters.
//
//   k_lin_schur      one CTA per chunk of consecutive tiles (a tile is up to 32
//                    observations of whole points, one warp).  Each warp
//                    linearises its tiles: residual, Jacobians (Eq. 5-7),
//                    point blocks V = sum Jp^T Jp and g_p = -sum Jp^T r by
//                    segmented warp reductions, V* = V + mu D_p = L L^T,
//                    M = L^-1, q = M g_p and Z = Jc^T Jp M^T, so that
//                    W V*^-1 W^T = Z Z^T and W V*^-1 g_p = Z q; one record per
//                    observation goes to shared memory.  The CTA then runs the
//                    chunk's reduction jobs: per free image the sums of
//                    Jc^T Jc - Z Z^T, -Jc^T r, Z q, diag(Jc^T Jc), and per
//                    co-visible image pair the sum of Z_a Z_b^T, each job on a
//                    run of lanes sized by its cost.  One partial sum per job.
//   k_partial_reduce the chunks' partial sums of each image and each pair,
//                    added in chunk order (FP64).
//   k_factor_solve   per cluster (FP64): assemble S = U* - W V*^-1 W^T and
//                    rhs = g_c - W V*^-1 g_p with priors and damping, blocked
//                    Cholesky in shared memory, solve, iterative refinement,
//                    candidate camera poses.  (Clusters of more than 32 free
//                    images: the global-memory solver of ba_big.cu.)
//   k_backsub_cost   per tile: linearise again (same arithmetic, same values),
//                    dX = M^T (q - sum_k Z_k^T dc_k), candidate points, cost
//                    at the candidate and the predicted reduction; the warp
//                    that finishes a cluster's last tile takes its LM step:
//                    gain ratio, accept/reject, Nielsen update.
//   Four launches per LM iteration.
//
// Precision.  MIXED = false: every step in binary64.  MIXED = true: the
// per-observation linearisation, the Schur reductions and the back-
// substitution run in binary32; the state (points and cameras) is held in
// double-float, and the cost F(x) that decides the gain ratio is evaluated
// per observation in double-float and summed in binary64; the reduced
// camera system is assembled, factored and refined in binary64.
//
// Every sum runs in an order fixed by the cluster's presorted tables; the
// only atomic is the back-substitution's per-cluster tile counter, which
// chooses the warp that takes the LM step and enters no sum.
#include <cuda_runtime.h>
#include <stdio.h>

#include <algorithm>
#include <type_traits>

#include "ba_device.cuh"
#include "ba_bulk.cuh"
#include "ba_camera.cuh"
#include "ba_dfloat.cuh"
#include "ba_internal.h"

namespace bagpu {

template <bool MIXED> struct RealOf { using T = double; };
template <> struct RealOf<true> { using T = float; };

template <typename Real> struct Vec2;
template <> struct Vec2<float> { using T = float2; };
template <> struct Vec2<double> { using T = double2; };

// ------------------------------------------------------------------ state access

__device__ __forceinline__ const float2* xdf_ptr(const DevCluster& C, int buf, int j) {
  return reinterpret_cast<const float2*>(C.X) + ((size_t)buf * C.n_pts + j) * 3;
}
__device__ __forceinline__ float2* xdf_wptr(const DevCluster& C, int buf, int j) {
  return reinterpret_cast<float2*>(C.X) + ((size_t)buf * C.n_pts + j) * 3;
}

// double-float camera record
struct CamDf {
  dfl R[9], T[3], f, k1, k2, p1, p2;
  float free_flag;
};

// Camera record layout (kCamDf = 40 floats): the part the binary32
// linearisation reads first, in six float4: R.hi [0, 9), T.hi [9, 12),
// T.lo [12, 15), f.hi 15, k1 k2 p1 p2 .hi [16, 20), free flag 20, pad; then
// R.lo [24, 33), f.lo 33, k1 k2 p1 p2 .lo [34, 38), pad.
__device__ __forceinline__ void load_f4(const float* p, int n4, float* v) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int i = 0; i < n4; ++i) {
    const float4 w = q[i];
    v[4 * i] = w.x; v[4 * i + 1] = w.y; v[4 * i + 2] = w.z; v[4 * i + 3] = w.w;
  }
}

// the linearisation's part: high words of R, f and the distortion, T in full
__device__ __forceinline__ CamDf load_camdf_lin(const float* p) {
  CamDf c;
  float v[24];
  load_f4(p, 6, v);
#pragma unroll
  for (int i = 0; i < 9; ++i) c.R[i] = dfl{v[i], 0.f};
#pragma unroll
  for (int i = 0; i < 3; ++i) c.T[i] = dfl{v[9 + i], v[12 + i]};
  c.f = dfl{v[15], 0.f};
  c.k1 = dfl{v[16], 0.f};
  c.k2 = dfl{v[17], 0.f};
  c.p1 = dfl{v[18], 0.f};
  c.p2 = dfl{v[19], 0.f};
  c.free_flag = v[20];
  return c;
}

// the whole double-float record
__device__ __forceinline__ CamDf load_camdf(const float* p) {
  CamDf c;
  float v[kCamDf];
  load_f4(p, kCamDf / 4, v);
#pragma unroll
  for (int i = 0; i < 9; ++i) c.R[i] = dfl{v[i], v[24 + i]};
#pragma unroll
  for (int i = 0; i < 3; ++i) c.T[i] = dfl{v[9 + i], v[12 + i]};
  c.f = dfl{v[15], v[33]};
  c.k1 = dfl{v[16], v[34]};
  c.k2 = dfl{v[17], v[35]};
  c.p1 = dfl{v[18], v[36]};
  c.p2 = dfl{v[19], v[37]};
  c.free_flag = v[20];
  return c;
}

__device__ __forceinline__ const float* camdf_ptr(const DevCluster& C, int buf, int k) {
  return C.camdf + ((size_t)buf * C.n_cams + k) * kCamDf;
}

// Eq. 5 with Brown distortion in double-float: residual (u - cx, v - cy) - c
// for a double-float point, every term in double-float.  X - T and the final
// difference with the observation, where the result is much smaller than the
// operands, use the accurate sum; the other sums (the rotation, the
// distortion terms, all far below the pixel accuracy the cost needs in their
// cancellation) the sloppy one; one reciprocal of the depth.
__device__ __forceinline__ bool df_residual(const CamDf& c, dfl X0, dfl X1, dfl X2, dfl c0, dfl c1, dfl& e0,
                                            dfl& e1) {
  const dfl d0 = df_sub(X0, c.T[0]), d1 = df_sub(X1, c.T[1]), d2 = df_sub(X2, c.T[2]);
  const dfl z = df_add_fast(df_add_fast(df_mul(c.R[2], d0), df_mul(c.R[5], d1)), df_mul(c.R[8], d2));
  if (!(z.hi > (float)kMinDepth)) return false;
  const dfl x = df_add_fast(df_add_fast(df_mul(c.R[0], d0), df_mul(c.R[3], d1)), df_mul(c.R[6], d2));
  const dfl y = df_add_fast(df_add_fast(df_mul(c.R[1], d0), df_mul(c.R[4], d1)), df_mul(c.R[7], d2));
  const dfl iz = df_recip(z);
  const dfl xn = df_mul(x, iz), yn = df_mul(y, iz);
  const dfl xx = df_mul(xn, xn), yy = df_mul(yn, yn), xy2 = df_mul_f(df_mul(xn, yn), 2.0f);
  const dfl r2 = df_add_fast(xx, yy);
  const dfl radm1 = df_mul(r2, df_add_fast(c.k1, df_mul(c.k2, r2)));  // rad - 1
  const dfl ddx = df_add_fast(df_add_fast(df_mul(xn, radm1), df_mul(c.p1, xy2)),
                              df_mul(c.p2, df_add_fast(r2, df_mul_f(xx, 2.0f))));
  const dfl ddy = df_add_fast(df_add_fast(df_mul(yn, radm1), df_mul(c.p1, df_add_fast(r2, df_mul_f(yy, 2.0f)))),
                              df_mul(c.p2, xy2));
  e0 = df_sub(df_mul(c.f, df_add_fast(xn, ddx)), c0);
  e1 = df_sub(df_mul(c.f, df_add_fast(yn, ddy)), c1);
  return true;
}

// 1/2 rho(s) / sigma^2 in double-float, s = e0^2 + e1^2 (Eq. 6: rho on the squared norm)
__device__ __forceinline__ dfl df_robust_cost(dfl e0, dfl e1, float delta, float half_inv_s2) {
  const dfl s = df_add_fast(df_mul(e0, e0), df_mul(e1, e1));
  const float d2 = delta * delta;
  dfl rho;
  if (s.hi <= d2) {
    rho = s;
  } else {
    rho = df_add_f(df_mul_f(df_sqrt(s), 2.0f * delta), -d2);
  }
  return df_mul_f(rho, half_inv_s2);
}

// ------------------------------------------------------------------ camera copies

// FP64 path: camera records in binary64 for the per-observation kernels.
__global__ void k_camreal(BatchView bv) {
  for (int s = blockIdx.x; s < bv.n; s += gridDim.x) {
    const DevCluster& C = bv.cl[s];
    const int cur = C.lm->cur;
    double* cr = (double*)C.camreal;
    for (int k = threadIdx.x; k < C.n_cams; k += blockDim.x) {
      const double* R = C.R + ((size_t)cur * C.n_cams + k) * 9;
      const double* T = C.T + ((size_t)cur * C.n_cams + k) * 3;
      double* o = cr + (size_t)kCamReal * k;
      for (int i = 0; i < 9; ++i) o[i] = R[i];
      for (int i = 0; i < 3; ++i) o[9 + i] = T[i];
      for (int i = 0; i < 7; ++i) o[12 + i] = C.intr[7 * k + i];
      o[19] = C.free_idx[k] >= 0 ? 1.0 : 0.0;
    }
  }
}

// both buffers of the mixed camera records from the binary64 cameras
__global__ void k_camdf_all(BatchView bv) {
  for (int s = blockIdx.x; s < bv.n; s += gridDim.x) {
    const DevCluster& C = bv.cl[s];
    for (int idx = threadIdx.x; idx < 2 * C.n_cams; idx += blockDim.x) {
      const int buf = idx / C.n_cams, k = idx - buf * C.n_cams;
      write_camdf(C, buf, k, C.R + ((size_t)buf * C.n_cams + k) * 9, C.T + ((size_t)buf * C.n_cams + k) * 3);
    }
  }
}

// ------------------------------------------------------------------ per-tile linearisation

__device__ __forceinline__ void ld4(const float* r, int at, float* o) {
  const float4 v = *reinterpret_cast<const float4*>(r + at);
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld4(const double* r, int at, double* o) {
  const double2 a = *reinterpret_cast<const double2*>(r + at);
  const double2 b = *reinterpret_cast<const double2*>(r + at + 2);
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}

// What one lane knows after linearising its observation of a tile: the
// whitened, robust-weighted Jacobians and residual, Z = Jc^T Jp L^-T, and
// (broadcast from the point's first lane) L^-1 and q = L^-1 g_p of the damped
// point block; D_p and g_p are valid on the point's first lane.
template <bool MIXED>
struct TileLin {
  using Real = typename RealOf<MIXED>::T;
  bool act, head;
  int o, k, j, seg_start, seg_end, span;
  Real Jc[12], r0, r1, Z[18];
  Real P[6];  // P = Jp M^T (2x3, row-major), so that Z = Jc^T P
  Real m00, m10, m11, m20, m21, m22, q0, q1, q2;
  Real d0, d1, d2, g0, g1, g2;
};

// Where the mixed linearisation reads a chunk's observations (camera, point,
// observation relative to the principal point) and the current points:
// the cluster's arrays in global memory, or a shared-memory copy of the
// chunk's ranges (index o - o0, point j - j0).
struct ObsView {
  const int* cam;
  const int* pt;
  const float2* chi;
  const float2* x;  // 3 float2 (hi, lo) per point
  int o0, j0;
};

__device__ __forceinline__ ObsView global_view(const DevCluster& C, int cur) {
  return ObsView{C.obs_cam, C.obs_pt, C.obs_chi, reinterpret_cast<const float2*>(C.X) + (size_t)cur * C.n_pts * 3,
                 0, 0};
}

// Linearise one tile (one warp).  The same arithmetic wherever it is called
// (the back-substitution linearises again rather than storing the result).
// PT_BUF: the point blocks' M, q, D_p and g_p are read from C.ptblk, where
// the linearise+Schur kernel of the same iteration stored them (same values),
// instead of being reduced and factored again.
template <bool MIXED, bool WANT_Z = true, bool PT_BUF = false>
__device__ __forceinline__ void linearize_tile(const DevCluster& C, LmState* lm, const Tile& tl, int lane,
                                               bool report_fail, TileLin<MIXED>& L, const ObsView& V) {
  using Real = typename RealOf<MIXED>::T;
  L.act = lane < tl.n_obs;
  L.o = tl.obs_begin + (L.act ? lane : 0);
  if constexpr (MIXED) {
    L.k = L.act ? V.cam[L.o - V.o0] : 0;
    L.j = L.act ? V.pt[L.o - V.o0] : -1 - lane;
  } else {
    L.k = L.act ? C.obs_cam[L.o] : 0;
    L.j = L.act ? C.obs_pt[L.o] : -1 - lane;
  }
  segments(L.j, lane, L.seg_start, L.seg_end);
  L.span = segment_span(L.seg_start, L.seg_end);
  L.head = L.act && lane == L.seg_start;
  const int cur = lm->cur;
  Real mu, inv_sigma, delta;
  if constexpr (MIXED) {
    mu = lm->mu_f;
    inv_sigma = C.inv_sigma_f;
    delta = C.delta_f;
  } else {
    mu = lm->mu;
    inv_sigma = 1.0 / C.sigma_px;
    delta = C.huber_delta;
  }
  Real Jp[6];
  L.r0 = 0;
  L.r1 = 0;
#pragma unroll
  for (int i = 0; i < 12; ++i) L.Jc[i] = 0;
#pragma unroll
  for (int i = 0; i < 6; ++i) Jp[i] = 0;
  if (L.act) {
    Real Rm[9], in[7], dx, dy, dz, uo, vo;
    bool is_free;
    if constexpr (MIXED) {
      const CamDf cd = load_camdf_lin(camdf_ptr(C, cur, L.k));
      const float2* xp = V.x + (size_t)(L.j - V.j0) * 3;
      const float2 a = xp[0], b = xp[1], c = xp[2];
      dx = df_to_f(df_sub(dfl{a.x, a.y}, cd.T[0]));
      dy = df_to_f(df_sub(dfl{b.x, b.y}, cd.T[1]));
      dz = df_to_f(df_sub(dfl{c.x, c.y}, cd.T[2]));
#pragma unroll
      for (int i = 0; i < 9; ++i) Rm[i] = cd.R[i].hi;
      in[0] = cd.f.hi; in[1] = 0.f; in[2] = 0.f;
      in[3] = cd.k1.hi; in[4] = cd.k2.hi; in[5] = cd.p1.hi; in[6] = cd.p2.hi;
      const float2 ch = V.chi[L.o - V.o0];  // observation relative to the principal point
      uo = ch.x; vo = ch.y;
      is_free = cd.free_flag != 0.0f;
    } else {
      const double* cr = (const double*)C.camreal + (size_t)kCamReal * L.k;
#pragma unroll
      for (int i = 0; i < 9; ++i) Rm[i] = cr[i];
#pragma unroll
      for (int i = 0; i < 7; ++i) in[i] = cr[12 + i];
      const double* Xd = C.X + ((size_t)cur * C.n_pts + L.j) * 3;
      dx = Xd[0] - cr[9]; dy = Xd[1] - cr[10]; dz = Xd[2] - cr[11];
      const double2 u = reinterpret_cast<const double2*>(C.obs_uv)[L.o];
      uo = u.x; vo = u.y;
      is_free = cr[19] != 0.0;
    }
    obs_linearize<Real>(Rm, dx, dy, dz, in, uo, vo, inv_sigma, delta, L.r0, L.r1, L.Jc, Jp);
    if (!is_free) {
#pragma unroll
      for (int i = 0; i < 12; ++i) L.Jc[i] = 0;
    }
  }
  if constexpr (PT_BUF) {
    // every lane of a point reads its block (one address per point); an
    // inactive lane reads point 0 and keeps P = 0 (its Jp is 0)
    const Real* pb = reinterpret_cast<const Real*>(C.ptblk) + (size_t)(L.act ? L.j : 0) * 16;
    Real w[16];
    ld4(pb, 0, w); ld4(pb, 4, w + 4); ld4(pb, 8, w + 8); ld4(pb, 12, w + 12);
    L.m00 = w[0]; L.m10 = w[1]; L.m11 = w[2]; L.m20 = w[3]; L.m21 = w[4]; L.m22 = w[5];
    L.q0 = w[6]; L.q1 = w[7]; L.q2 = w[8];
    L.d0 = w[9]; L.d1 = w[10]; L.d2 = w[11];
    L.g0 = w[12]; L.g1 = w[13]; L.g2 = w[14];
  } else {
    // point blocks by segmented reduction
    Real v00 = Jp[0] * Jp[0] + Jp[3] * Jp[3];
    Real v01 = Jp[0] * Jp[1] + Jp[3] * Jp[4];
    Real v02 = Jp[0] * Jp[2] + Jp[3] * Jp[5];
    Real v11 = Jp[1] * Jp[1] + Jp[4] * Jp[4];
    Real v12 = Jp[1] * Jp[2] + Jp[4] * Jp[5];
    Real v22 = Jp[2] * Jp[2] + Jp[5] * Jp[5];
    Real g0 = -(Jp[0] * L.r0 + Jp[3] * L.r1);
    Real g1 = -(Jp[1] * L.r0 + Jp[4] * L.r1);
    Real g2 = -(Jp[2] * L.r0 + Jp[5] * L.r1);
    v00 = seg_reduce(v00, lane, L.seg_start, L.seg_end, L.span);
    v01 = seg_reduce(v01, lane, L.seg_start, L.seg_end, L.span);
    v02 = seg_reduce(v02, lane, L.seg_start, L.seg_end, L.span);
    v11 = seg_reduce(v11, lane, L.seg_start, L.seg_end, L.span);
    v12 = seg_reduce(v12, lane, L.seg_start, L.seg_end, L.span);
    v22 = seg_reduce(v22, lane, L.seg_start, L.seg_end, L.span);
    g0 = seg_reduce(g0, lane, L.seg_start, L.seg_end, L.span);
    g1 = seg_reduce(g1, lane, L.seg_start, L.seg_end, L.span);
    g2 = seg_reduce(g2, lane, L.seg_start, L.seg_end, L.span);
    // head: damp, factor V* = L L^T, M = L^-1, q = M g_p
    Real m00 = 0, m10 = 0, m11 = 0, m20 = 0, m21 = 0, m22 = 0, q0 = 0, q1 = 0, q2 = 0;
    L.d0 = L.d1 = L.d2 = 0;
    L.g0 = g0; L.g1 = g1; L.g2 = g2;
    if (L.head) {
      const Real d0 = clamp_diag(v00), d1 = clamp_diag(v11), d2 = clamp_diag(v22);
      const Real a00 = v00 + mu * d0, a11 = v11 + mu * d1, a22 = v22 + mu * d2;
      // V* = L L^T with M = L^-1 from reciprocal square roots of the pivots
      bool ok = a00 > Real(0);
      m00 = pivot_rsqrt(ok ? a00 : Real(1));
      const Real l10 = v01 * m00, l20 = v02 * m00;
      const Real t11 = a11 - l10 * l10;
      ok = ok && t11 > Real(0);
      m11 = pivot_rsqrt(t11 > Real(0) ? t11 : Real(1));
      const Real l21 = (v12 - l20 * l10) * m11;
      const Real t22 = a22 - l20 * l20 - l21 * l21;
      ok = ok && t22 > Real(0);
      m22 = pivot_rsqrt(t22 > Real(0) ? t22 : Real(1));
      if (!ok && report_fail) lm->pt_fail = 1;  // point block not positive definite: reject this step
      m10 = -l10 * m00 * m11;
      m21 = -l21 * m11 * m22;
      m20 = -(l20 * m00 + l21 * m10) * m22;
      q0 = m00 * g0;
      q1 = m10 * g0 + m11 * g1;
      q2 = m20 * g0 + m21 * g1 + m22 * g2;
      L.d0 = d0; L.d1 = d1; L.d2 = d2;
    }
    L.m00 = __shfl_sync(BA_FULL_MASK, m00, L.seg_start);
    L.m10 = __shfl_sync(BA_FULL_MASK, m10, L.seg_start);
    L.m11 = __shfl_sync(BA_FULL_MASK, m11, L.seg_start);
    L.m20 = __shfl_sync(BA_FULL_MASK, m20, L.seg_start);
    L.m21 = __shfl_sync(BA_FULL_MASK, m21, L.seg_start);
    L.m22 = __shfl_sync(BA_FULL_MASK, m22, L.seg_start);
    L.q0 = __shfl_sync(BA_FULL_MASK, q0, L.seg_start);
    L.q1 = __shfl_sync(BA_FULL_MASK, q1, L.seg_start);
    L.q2 = __shfl_sync(BA_FULL_MASK, q2, L.seg_start);
  }
  // P = Jp M^T (2x3), Z = Jc^T P (6x3)
  const Real P00 = Jp[0] * L.m00;
  const Real P01 = Jp[0] * L.m10 + Jp[1] * L.m11;
  const Real P02 = Jp[0] * L.m20 + Jp[1] * L.m21 + Jp[2] * L.m22;
  const Real P10 = Jp[3] * L.m00;
  const Real P11 = Jp[3] * L.m10 + Jp[4] * L.m11;
  const Real P12 = Jp[3] * L.m20 + Jp[4] * L.m21 + Jp[5] * L.m22;
  L.P[0] = P00; L.P[1] = P01; L.P[2] = P02;
  L.P[3] = P10; L.P[4] = P11; L.P[5] = P12;
  if constexpr (WANT_Z) {
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      L.Z[3 * m + 0] = L.Jc[m] * P00 + L.Jc[6 + m] * P10;
      L.Z[3 * m + 1] = L.Jc[m] * P01 + L.Jc[6 + m] * P11;
      L.Z[3 * m + 2] = L.Jc[m] * P02 + L.Jc[6 + m] * P12;
    }
  }
}

// ------------------------------------------------------------------ K1: linearise + Schur reductions, one CTA per chunk

// Shared record of one observation, kSrec = 28 Real, 16-byte aligned:
// Jc [0, 12), r [12, 14), u = P q [14, 16), W = I - P P^T as
// (w00, w01, w11) [16, 19), pad, P [20, 26) (P = Jp M^T, 2x3), pad.  Since
// Z = Jc^T P, the observation's share of the image block is
// Jc^T Jc - Z Z^T = Jc^T W Jc, of the right-hand side Z q = Jc^T u, and of a
// pair block Z_a Z_b^T = Jc_a^T (P_a P_b^T) Jc_b.  An image job reads the
// first five 16-byte groups, a pair job groups 0-2, 5 and 6.
// Jc (12) and P (6)
template <typename Real>
__device__ __forceinline__ void ld_rec_jcp(const Real* r, Real Jc[12], Real P[6]) {
  ld4(r, 0, Jc);
  ld4(r, 4, Jc + 4);
  ld4(r, 8, Jc + 8);
  Real t[4];
  ld4(r, 20, P);
  ld4(r, 24, t);
  P[4] = t[0];
  P[5] = t[1];
}
// Jc (12), r (2), u (2), W (3)
template <typename Real>
__device__ __forceinline__ void ld_rec_cam(const Real* r, Real Jc[12], Real rr[2], Real u[2], Real w[3]) {
  ld4(r, 0, Jc);
  ld4(r, 4, Jc + 4);
  ld4(r, 8, Jc + 8);
  Real a[4], b[4];
  ld4(r, 12, a);
  ld4(r, 16, b);
  rr[0] = a[0]; rr[1] = a[1];
  u[0] = a[2]; u[1] = a[3];
  w[0] = b[0]; w[1] = b[1]; w[2] = b[2];
}

// Store one observation's record (vector stores): Jc, r, u = P q,
// W = I - P P^T and P.
template <bool MIXED>
__device__ __forceinline__ void st_rec(typename RealOf<MIXED>::T* r, const TileLin<MIXED>& L) {
  using Real = typename RealOf<MIXED>::T;
  const Real* P = L.P;
  const Real u0 = P[0] * L.q0 + P[1] * L.q1 + P[2] * L.q2;
  const Real u1 = P[3] * L.q0 + P[4] * L.q1 + P[5] * L.q2;
  const Real w00 = Real(1) - (P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
  const Real w01 = -(P[0] * P[3] + P[1] * P[4] + P[2] * P[5]);
  const Real w11 = Real(1) - (P[3] * P[3] + P[4] * P[4] + P[5] * P[5]);
  const Real v[28] = {L.Jc[0], L.Jc[1], L.Jc[2], L.Jc[3], L.Jc[4], L.Jc[5], L.Jc[6], L.Jc[7], L.Jc[8], L.Jc[9],
                      L.Jc[10], L.Jc[11], L.r0, L.r1, u0, u1, w00, w01, w11, Real(0),
                      P[0], P[1], P[2], P[3], P[4], P[5], Real(0), Real(0)};
  if constexpr (MIXED) {
    float4* o = reinterpret_cast<float4*>(r);
#pragma unroll
    for (int i = 0; i < 7; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
  } else {
    double2* o = reinterpret_cast<double2*>(r);
#pragma unroll
    for (int i = 0; i < 14; ++i) o[i] = make_double2(v[2 * i], v[2 * i + 1]);
  }
}

// The point's block for the back-substitution (head lane of the point).
template <bool MIXED>
__device__ __forceinline__ void st_ptblk(const DevCluster& C, const TileLin<MIXED>& L) {
  using Real = typename RealOf<MIXED>::T;
  const Real v[16] = {L.m00, L.m10, L.m11, L.m20, L.m21, L.m22, L.q0, L.q1,
                      L.q2,  L.d0,  L.d1,  L.d2,  L.g0,  L.g1,  L.g2, Real(0)};
  Real* pb = reinterpret_cast<Real*>(C.ptblk) + (size_t)L.j * 16;
  if constexpr (MIXED) {
    float4* o = reinterpret_cast<float4*>(pb);
#pragma unroll
    for (int i = 0; i < 4; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
  } else {
    double2* o = reinterpret_cast<double2*>(pb);
#pragma unroll
    for (int i = 0; i < 8; ++i) o[i] = make_double2(v[2 * i], v[2 * i + 1]);
  }
}

// One job's sums over its items [i0, i1).  Image job: the upper triangle of
// sum Jc^T W Jc (21), -sum Jc^T r (6), sum Jc^T u (6), diag sum Jc^T Jc (6).
// Pair job: sum Jc_a^T (P_a P_b^T) Jc_b (36, row-major).
template <typename Real>
__device__ __forceinline__ void job_sums(const DevCluster& C, const Job& J, bool cam, int i0, int i1,
                                         const Real* srec, Real acc[39]) {
#pragma unroll
  for (int i = 0; i < 39; ++i) acc[i] = 0;
  if (cam) {
    for (int e = i0; e < i1; ++e) {
      const Real* r = srec + (size_t)C.cm_list[J.item_begin + e] * kSrec;
      Real Jc[12], rr[2], u[2], w[3];
      ld_rec_cam(r, Jc, rr, u, w);
      Real WJ0[6], WJ1[6];
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        WJ0[m] = w[0] * Jc[m] + w[1] * Jc[6 + m];
        WJ1[m] = w[1] * Jc[m] + w[2] * Jc[6 + m];
      }
      int t = 0;
#pragma unroll
      for (int a = 0; a < 6; ++a)
#pragma unroll
        for (int b = a; b < 6; ++b) acc[t++] += Jc[a] * WJ0[b] + Jc[6 + a] * WJ1[b];
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        acc[21 + a] -= Jc[a] * rr[0] + Jc[6 + a] * rr[1];
        acc[27 + a] += Jc[a] * u[0] + Jc[6 + a] * u[1];
        acc[33 + a] += Jc[a] * Jc[a] + Jc[6 + a] * Jc[6 + a];
      }
    }
  } else {
    for (int e = i0; e < i1; ++e) {
      const unsigned int it = C.pent[J.item_begin + e];
      Real Ja[12], Pa[6], Jb[12], Pb[6];
      ld_rec_jcp(srec + (size_t)(it & 0xffffu) * kSrec, Ja, Pa);
      ld_rec_jcp(srec + (size_t)(it >> 16) * kSrec, Jb, Pb);
      // G = P_a P_b^T (2x2), H = G Jc_b (2x6)
      const Real g00 = Pa[0] * Pb[0] + Pa[1] * Pb[1] + Pa[2] * Pb[2];
      const Real g01 = Pa[0] * Pb[3] + Pa[1] * Pb[4] + Pa[2] * Pb[5];
      const Real g10 = Pa[3] * Pb[0] + Pa[4] * Pb[1] + Pa[5] * Pb[2];
      const Real g11 = Pa[3] * Pb[3] + Pa[4] * Pb[4] + Pa[5] * Pb[5];
      Real H0[6], H1[6];
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        H0[m] = g00 * Jb[m] + g01 * Jb[6 + m];
        H1[m] = g10 * Jb[m] + g11 * Jb[6 + m];
      }
#pragma unroll
      for (int a = 0; a < 6; ++a)
#pragma unroll
        for (int b = 0; b < 6; ++b) acc[6 * a + b] += Ja[a] * H0[b] + Ja[6 + a] * H1[b];
    }
  }
}

// One job's partial sums as 16-byte stores (the rows are 16-byte aligned:
// kCamPart and kPairPart are multiples of 16 bytes); a camera row's last
// group carries a zero in its pad word.
static_assert(kCamPart % 4 == 0 && kPairPart % 4 == 0, "partial rows of 16-byte groups");
__device__ __forceinline__ void store_job_row(float* out, bool cam, const float acc[39]) {
  float4* o = reinterpret_cast<float4*>(out);
#pragma unroll
  for (int i = 0; i < 9; ++i) o[i] = make_float4(acc[4 * i], acc[4 * i + 1], acc[4 * i + 2], acc[4 * i + 3]);
  if (cam) o[9] = make_float4(acc[36], acc[37], acc[38], 0.f);
}
__device__ __forceinline__ void store_job_row(double* out, bool cam, const double acc[39]) {
  double2* o = reinterpret_cast<double2*>(out);
#pragma unroll
  for (int i = 0; i < 18; ++i) o[i] = make_double2(acc[2 * i], acc[2 * i + 1]);
  if (cam) {
    o[18] = make_double2(acc[36], acc[37]);
    o[19] = make_double2(acc[38], 0.0);
  }
}

template <typename Real>
__device__ __forceinline__ void store_job(const DevCluster& C, const Job& J, bool cam, const Real acc[39]) {
  Real* out = cam ? (Real*)C.campart + (size_t)kCamPart * J.slot : (Real*)C.pairpart + (size_t)kPairPart * J.slot;
  store_job_row(out, cam, acc);
}

// bytes of the per-observation records (and, overlaid, the lane partials)
__host__ __device__ constexpr size_t chunk_records_bytes(bool mixed) {
  return (mixed ? sizeof(float) : sizeof(double)) *
         ((size_t)(mixed ? kChunkObsMixed : kChunkObsF64) * kSrec > (size_t)kChunkThreads * kLanePart
              ? (size_t)(mixed ? kChunkObsMixed : kChunkObsF64) * kSrec
              : (size_t)kChunkThreads * kLanePart);
}
__device__ __forceinline__ float4 vadd(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ double2 vadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// Shared-memory staging of one chunk's observations and points (mixed path):
// camera and point indices (int), observations relative to the principal
// point (float2 hi), points (3 float2 each), each range rounded outward to
// 16 bytes.  A chunk spanning more than kStagePts points reads its points
// from global memory instead.  Double-buffered beside them, so that the next
// chunk's copies land while this chunk's jobs still read its own: the chunk's
// head (cluster slot, state buffer, chunk record; written by the issuing
// thread), its tile headers, its job records and the job of each lane (the
// last two for chunks of at most kChunkThreads jobs).
constexpr int kStagePts = 512;
constexpr uint32_t kStageIdxBytes = kChunkObsMixed * 4 + 32;
constexpr uint32_t kStageChiBytes = kChunkObsMixed * 8 + 32;
constexpr uint32_t kStageXBytes = kStagePts * 24 + 32;
struct ChunkHead {
  int s, cur, pad0, pad1;
  Chunk ch;
};
constexpr uint32_t kHeadBytes = (sizeof(ChunkHead) + 15) / 16 * 16;
constexpr uint32_t kStageTileBytes = kChunkTilesMixed * sizeof(Tile) + 32;
constexpr uint32_t kStageJobBytes = kChunkThreads * sizeof(Job) + 32;
constexpr uint32_t kStageLaneBytes = kChunkThreads;  // one byte per lane
constexpr uint32_t kTableBytes = kHeadBytes + kStageTileBytes + kStageJobBytes + kStageLaneBytes;
constexpr uint32_t kStageBytes = 2 * kStageIdxBytes + kStageChiBytes + kStageXBytes + 2 * kTableBytes;
constexpr uint64_t kCopyWaitNs = 200000000ull;  // give up on a staged copy after 200 ms
constexpr uint64_t kInjectWaitNs = 1000000ull;  // the injected wait's limit (kInjectCopyTimeout)
static_assert(kTableBytes % 16 == 0 && kStageTileBytes % 16 == 0 && kStageJobBytes % 16 == 0, "16-byte staging");

struct Stage {
  char* idx_cam;
  char* idx_pt;
  char* chi;
  char* x;
  char* tab;  // two table buffers of kTableBytes
  uint64_t* bar;
  int* ok;
  uint64_t* never;  // failure injection: a barrier no copy or thread completes
  __device__ ChunkHead* head(int b) const { return reinterpret_cast<ChunkHead*>(tab + b * kTableBytes); }
  __device__ char* tiles(int b) const { return tab + b * kTableBytes + kHeadBytes; }
  __device__ char* jobs(int b) const { return tab + b * kTableBytes + kHeadBytes + kStageTileBytes; }
  __device__ unsigned char* lanes(int b) const {
    return reinterpret_cast<unsigned char*>(tab + b * kTableBytes + kHeadBytes + kStageTileBytes + kStageJobBytes);
  }
};

__device__ __forceinline__ bool job_table_mode(const Chunk& ch) {
  const int nj = ch.n_lc + ch.n_lp;
  return nj > 0 && nj <= kChunkThreads;
}

// Issue the copies of chunk g into table buffer b (one thread) and write its
// head.  The barrier's transaction count covers exactly the bytes issued.
__device__ __forceinline__ void stage_issue(const BatchView& bv, int g, const Stage& S, int b) {
  const int s = find_slot(bv.chunk_pre, bv.n, g);
  const DevCluster& C = bv.cl[s];
  const int local = g - bv.chunk_pre[s];
  const Chunk ch = C.chunks[local];
  const int cur = C.lm->cur;
  ChunkHead* hd = S.head(b);
  hd->s = s;
  hd->cur = cur;
  hd->ch = ch;
  const BulkRange rc = bulk_range(C.obs_cam + ch.obs_begin, (size_t)ch.n_obs * 4);
  const BulkRange rp = bulk_range(C.obs_pt + ch.obs_begin, (size_t)ch.n_obs * 4);
  const BulkRange rh = bulk_range(C.obs_chi + ch.obs_begin, (size_t)ch.n_obs * 8);
  const bool stage_x = ch.n_pts <= kStagePts;
  const float2* xb = reinterpret_cast<const float2*>(C.X) + ((size_t)cur * C.n_pts + ch.pt_begin) * 3;
  const BulkRange rx = bulk_range(xb, stage_x ? (size_t)ch.n_pts * 24 : 0);
  const BulkRange rt = bulk_range(C.tiles + ch.tile_begin, (size_t)ch.n_tiles * sizeof(Tile));
  const bool tab = job_table_mode(ch);
  const BulkRange rj = bulk_range(C.jobs + ch.job_begin, tab ? (size_t)(ch.n_lc + ch.n_lp) * sizeof(Job) : 0);
  const unsigned char* lj = C.lane_job + (size_t)local * kChunkThreads;
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(S.bar, rc.bytes + rp.bytes + rh.bytes + (stage_x ? rx.bytes : 0u) + rt.bytes +
                                   (tab ? rj.bytes + kStageLaneBytes : 0u));
  bulk_copy_g2s(S.idx_cam, rc.src, rc.bytes, S.bar);
  bulk_copy_g2s(S.idx_pt, rp.src, rp.bytes, S.bar);
  bulk_copy_g2s(S.chi, rh.src, rh.bytes, S.bar);
  if (stage_x && rx.bytes) bulk_copy_g2s(S.x, rx.src, rx.bytes, S.bar);
  bulk_copy_g2s(S.tiles(b), rt.src, rt.bytes, S.bar);
  if (tab) {
    bulk_copy_g2s(S.jobs(b), rj.src, rj.bytes, S.bar);
    bulk_copy_g2s(S.lanes(b), lj, kStageLaneBytes, S.bar);
  }
}

// The view of the staged chunk (same rounding as stage_issue).
__device__ __forceinline__ ObsView stage_view(const DevCluster& C, const Chunk& ch, int cur, const Stage& S) {
  ObsView V;
  V.cam = reinterpret_cast<const int*>(S.idx_cam + bulk_range(C.obs_cam + ch.obs_begin, 4).lead);
  V.pt = reinterpret_cast<const int*>(S.idx_pt + bulk_range(C.obs_pt + ch.obs_begin, 4).lead);
  V.chi = reinterpret_cast<const float2*>(S.chi + bulk_range(C.obs_chi + ch.obs_begin, 8).lead);
  V.o0 = ch.obs_begin;
  const float2* xb = reinterpret_cast<const float2*>(C.X) + ((size_t)cur * C.n_pts + ch.pt_begin) * 3;
  if (ch.n_pts <= kStagePts) {
    V.x = reinterpret_cast<const float2*>(S.x + bulk_range(xb, 24).lead);
    V.j0 = ch.pt_begin;
  } else {
    V.x = reinterpret_cast<const float2*>(C.X) + (size_t)cur * C.n_pts * 3;
    V.j0 = 0;
  }
  return V;
}

template <bool MIXED>
__global__ void __launch_bounds__(kChunkThreads, MIXED ? kLinSchurMinBlocksMixed : 1)
    k_lin_schur(BatchView bv, int diag) {
  using Real = typename RealOf<MIXED>::T;
  extern __shared__ __align__(16) unsigned char smraw[];
  // [chunk_obs][kSrec] records; once every job has read them, the same
  // memory holds the lane partials of multi-lane jobs ([threads][kLanePart])
  Real* srec = reinterpret_cast<Real*>(smraw);
  Real* lanepart = srec;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int total = bv.tot[1];
  // a contiguous run of chunks per CTA: neighbouring chunks (Morton order of
  // the points) share images and points in the caches
  const int per = (total + (int)gridDim.x - 1) / (int)gridDim.x;
  const int g0 = (int)blockIdx.x * per, g1 = min(total, g0 + per);
  // mixed path: the next chunk's observations and points are copied into
  // shared memory by the copy engine while this chunk is reduced
  Stage S{};
  uint32_t phase = 0;
  if constexpr (MIXED) {
    char* st = reinterpret_cast<char*>(smraw) + chunk_records_bytes(true);
    S.idx_cam = st;
    S.idx_pt = st + kStageIdxBytes;
    S.chi = st + 2 * kStageIdxBytes;
    S.x = st + 2 * kStageIdxBytes + kStageChiBytes;
    S.tab = st + 2 * kStageIdxBytes + kStageChiBytes + kStageXBytes;
    S.bar = reinterpret_cast<uint64_t*>(st + kStageBytes);
    S.ok = reinterpret_cast<int*>(st + kStageBytes + 8);
    S.never = reinterpret_cast<uint64_t*>(st + kStageBytes + 16);
    if (threadIdx.x == 0) {
      mbar_init(S.bar, 1);
      mbar_init(S.never, 1);
      fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && g0 < g1) stage_issue(bv, g0, S, 0);
  }
  int b = 0;  // table buffer of the current chunk (mixed path)
  for (int g = g0; g < g1; ++g, b ^= 1) {
    int s;
    Chunk ch;
    if constexpr (!MIXED) {
      s = find_slot(bv.chunk_pre, bv.n, g);
      ch = bv.cl[s].chunks[g - bv.chunk_pre[s]];
    }
    ObsView V{};
    if constexpr (MIXED) {
      if (threadIdx.x == 0) {
        const bool ok = (bv.inject & kInjectCopyTimeout) ? mbar_wait_bounded(S.never, 0u, kInjectWaitNs)
                                                         : mbar_wait_bounded(S.bar, phase, kCopyWaitNs);
        *S.ok = ok ? 1 : 0;
      }
      __syncthreads();
      phase ^= 1u;
      if (!*S.ok) {
        // the copy did not complete in time: flag every cluster whose chunks
        // this CTA has still to process (their steps are rejected), wait once
        // more for the copies in flight, and stop
        if (threadIdx.x == 0) {
          for (int h = g; h < g1; ++h) {
            LmState* hl = bv.cl[find_slot(bv.chunk_pre, bv.n, h)].lm;
            hl->dev_error = kDevErrTimeout;
            hl->pt_fail = 1;
          }
          mbar_wait_bounded(S.bar, phase ^ 1u, kCopyWaitNs);
        }
        return;
      }
      const ChunkHead* hd = S.head(b);
      s = hd->s;
      ch = hd->ch;
      V = stage_view(bv.cl[s], ch, hd->cur, S);
    }
    const DevCluster& C = bv.cl[s];
    LmState* lm = C.lm;
    const bool active = lm->active != 0;
    // 1. linearise the chunk's tiles into shared memory
    if (active) {
      for (int t = warp; t < ch.n_tiles; t += nw) {
        Tile tl;
        if constexpr (MIXED) {
          tl = reinterpret_cast<const Tile*>(S.tiles(b) + bulk_range(C.tiles + ch.tile_begin, 8).lead)[t];
        } else {
          tl = C.tiles[ch.tile_begin + t];
        }
        TileLin<MIXED> L;
        linearize_tile<MIXED, false>(C, lm, tl, lane, true, L, V);
        if (L.act) st_rec<MIXED>(srec + (size_t)(L.o - ch.obs_begin) * kSrec, L);
        if (L.head) st_ptblk<MIXED>(C, L);
        if (diag) {  // largest |g_p| of the tile, for the gradient norm
          double gm = L.head ? fmax(fabs((double)L.g0), fmax(fabs((double)L.g1), fabs((double)L.g2))) : 0.0;
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) gm = fmax(gm, __shfl_down_sync(BA_FULL_MASK, gm, off));
          if (lane == 0) C.tilepart[2 * (ch.tile_begin + t) + 1] = gm;
        }
      }
    }
    __syncthreads();
    if constexpr (MIXED) {  // staging is free: start the copies of this CTA's next chunk
      if (threadIdx.x == 0 && g + 1 < g1) stage_issue(bv, g + 1, S, b ^ 1);
    }
    if (!active) continue;
    // 2. Schur reductions of the chunk.  Jobs: each free camera (sum of
    //    Jc^T Jc - Z Z^T, -Jc^T r, Z q, diag(Jc^T Jc) over its observations) and
    //    each co-visible camera pair (sum of Z_a Z_b^T over its point pairs).
    //    The host gave every job a run of lanes in proportion to its cost;
    //    lane i of a job sums a contiguous range of the job's items, and the
    //    lanes' partial sums are added in lane order.  A chunk with more jobs
    //    than threads runs one lane per job.
    const int n_jobs = ch.n_lc + ch.n_lp;  // 0 when every observation of the chunk is of a fixed camera
    if (n_jobs > 0 && n_jobs <= (int)blockDim.x) {
      // job whose lane run holds this thread: the last job starting at or
      // before it (jobs are in lane order); staged by the host's table on the
      // mixed path, a binary search on the other
      int lo;
      Job J;
      if constexpr (MIXED) {
        lo = S.lanes(b)[threadIdx.x];
        J = reinterpret_cast<const Job*>(S.jobs(b) + bulk_range(C.jobs + ch.job_begin, 16).lead)[lo];
      } else {
        lo = 0;
        int hi = n_jobs - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (C.jobs[ch.job_begin + mid].lane_begin <= (int)threadIdx.x) lo = mid; else hi = mid - 1;
        }
        J = C.jobs[ch.job_begin + lo];
      }
      const bool mine = (int)threadIdx.x < J.lane_begin + J.n_lanes;
      const int part = threadIdx.x - J.lane_begin;
      const bool cam = lo < ch.n_lc;
      Real acc[39];
      if (mine) {
        const int i0 = (int)(((long long)J.count * part) / J.n_lanes);
        const int i1 = (int)(((long long)J.count * (part + 1)) / J.n_lanes);
        job_sums<Real>(C, J, cam, i0, i1, srec, acc);
        if (J.n_lanes == 1) store_job<Real>(C, J, cam, acc);
      }
      __syncthreads();  // every record has been read: the lane partials may overwrite them
      if (mine && J.n_lanes > 1) {
        Real* lp = lanepart + (size_t)threadIdx.x * kLanePart;
        if constexpr (MIXED) {
          float4* o = reinterpret_cast<float4*>(lp);
#pragma unroll
          for (int i = 0; i < 9; ++i) o[i] = make_float4(acc[4 * i], acc[4 * i + 1], acc[4 * i + 2], acc[4 * i + 3]);
          o[9] = make_float4(acc[36], acc[37], acc[38], 0.f);
        } else {
          double2* o = reinterpret_cast<double2*>(lp);
#pragma unroll
          for (int i = 0; i < 19; ++i) o[i] = make_double2(acc[2 * i], acc[2 * i + 1]);
          o[19] = make_double2(acc[38], 0.0);
        }
      }
      __syncthreads();
      // multi-lane jobs: the job's own lanes add its lane partials, each lane
      // a share of the 16-byte groups of the row, every element summed over
      // the job's lanes in lane order
      if (mine && J.n_lanes > 1) {
        using Vec = typename std::conditional<MIXED, float4, double2>::type;
        constexpr int kPer = 16 / sizeof(Real);  // elements of a group
        const int groups = (cam ? kCamPart : kPairPart) / kPer;
        const Vec* rows = reinterpret_cast<const Vec*>(lanepart);
        Vec* out = reinterpret_cast<Vec*>(cam ? (Real*)C.campart + (size_t)kCamPart * J.slot
                                              : (Real*)C.pairpart + (size_t)kPairPart * J.slot);
        for (int q = part; q < groups; q += J.n_lanes) {
          Vec v = rows[(size_t)J.lane_begin * (kLanePart / kPer) + q];
          for (int l = J.lane_begin + 1; l < J.lane_begin + J.n_lanes; ++l) v = vadd(v, rows[(size_t)l * (kLanePart / kPer) + q]);
          out[q] = v;
        }
      }
    } else {
      for (int jb = threadIdx.x; jb < n_jobs; jb += blockDim.x) {
        const Job J = C.jobs[ch.job_begin + jb];
        const bool cam = jb < ch.n_lc;
        Real acc[39];
        job_sums<Real>(C, J, cam, 0, J.count, srec, acc);
        store_job<Real>(C, J, cam, acc);
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ partial sums -> per-camera / per-pair sums

// Running sum of binary32 partials kept in double-float (TwoSum, error-free
// to ~2^-48 of the total; binary64 adds run at 1/59 of the binary32 rate),
// or of binary64 partials in binary64.
struct AccF {
  dfl v{0.f, 0.f};
  __device__ __forceinline__ void add(float x) { v = df_add_f(v, x); }
  __device__ __forceinline__ double get() const { return (double)v.hi + (double)v.lo; }
};
struct AccD {
  double v = 0.0;
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ double get() const { return v; }
};
template <typename Real> struct AccOf { using T = AccD; };
template <> struct AccOf<float> { using T = AccF; };

// Item `it` of a cluster (a free camera, it < n_free, or a camera pair): sum
// its chunk partials in chunk order, by one warp (lane i owns element i and
// i + 32), into camsum / pairsum.
template <typename Real>
__device__ __forceinline__ void reduce_item_partials(const DevCluster& C, int it, int lane) {
  using Acc = typename AccOf<Real>::T;
  const bool cam = it < C.n_free;
  const int key = cam ? it : it - C.n_free;
  const int width = cam ? 39 : 36, stride = cam ? kCamPart : kPairPart;
  const int* slots = cam ? C.cam_slots : C.pair_slots;
  const int b = cam ? C.cam_slot_begin[key] : C.pair_slot_begin[key];
  const int e = cam ? C.cam_slot_begin[key + 1] : C.pair_slot_begin[key + 1];
  const Real* part = (const Real*)(cam ? C.campart : C.pairpart);
  double* out = cam ? C.camsum + (size_t)kCamPart * key : C.pairsum + (size_t)kPairPart * key;
  const bool two = lane + 32 < width;
  Acc v0, v1;
  int p = b;
  for (; p + 4 <= e; p += 4) {  // four independent loads in flight, added in slot order
    const Real* a0 = part + (size_t)stride * slots[p];
    const Real* a1 = part + (size_t)stride * slots[p + 1];
    const Real* a2 = part + (size_t)stride * slots[p + 2];
    const Real* a3 = part + (size_t)stride * slots[p + 3];
    const Real x0 = lane < width ? a0[lane] : Real(0), x1 = lane < width ? a1[lane] : Real(0);
    const Real x2 = lane < width ? a2[lane] : Real(0), x3 = lane < width ? a3[lane] : Real(0);
    const Real y0 = two ? a0[lane + 32] : Real(0), y1 = two ? a1[lane + 32] : Real(0);
    const Real y2 = two ? a2[lane + 32] : Real(0), y3 = two ? a3[lane + 32] : Real(0);
    v0.add(x0); v0.add(x1); v0.add(x2); v0.add(x3);
    v1.add(y0); v1.add(y1); v1.add(y2); v1.add(y3);
  }
  for (; p < e; ++p) {
    const Real* a0 = part + (size_t)stride * slots[p];
    if (lane < width) v0.add(a0[lane]);
    if (two) v1.add(a0[lane + 32]);
  }
  if (lane < width) out[lane] = v0.get();
  if (two) out[lane + 32] = v1.get();
}

// Warp per free camera or camera pair of every cluster of the batch.
template <typename Real>
__global__ void __launch_bounds__(256) k_partial_reduce(BatchView bv) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int total = bv.tot[2];
  for (int g = warp; g < total; g += nwarps) {
    const int s = find_slot(bv.item_pre, bv.n, g);
    const DevCluster& C = bv.cl[s];
    if (!C.lm->active) continue;
    reduce_item_partials<Real>(C, g - bv.item_pre[s], lane);
  }
}

// ------------------------------------------------------------------ K4 (FP64)

__device__ __forceinline__ int pk(int i, int j) { return (i * (i + 1)) / 2 + j; }  // packed lower, j <= i

size_t factor_smem_bytes(int max_n) {
  // packed A, per-camera sums and priors, x, b, t, inv_diag, the envelope and
  // scale exponents (ints), the double-float solves' block inverses
  const int nf = max_n / 6;
  const size_t doubles = (size_t)max_n * (max_n + 1) / 2 + (size_t)nf * 40 + (size_t)nf * 42 + 5 * (size_t)max_n +
                         (size_t)((max_n + 31) / 32) * (32 * 33 / 2) + 64;
  return doubles * sizeof(double);
}

#ifndef BA_FACTOR_THREADS
#define BA_FACTOR_THREADS 512
#endif
constexpr int kFactorThreads = BA_FACTOR_THREADS;  // threads of the shared-memory factor CTA

constexpr int kSolveNB = 32;   // diagonal block of the triangular solves (one warp)

// Blocked right-looking Cholesky A = L L^T of the packed lower matrix in
// shared memory, by the whole CTA.  Per column j of a panel of nb
// columns: warp 0 takes the pivot (square root and its reciprocal, once) and
// the scaled entries of the panel's own rows; then every thread scales its
// rows of column j and updates the panel's remaining columns.  After the
// panel the trailing matrix is updated with it in 4x4 register tiles.
// inv_diag[j] = 1 / L(j, j) is kept for the solves; colbuf: shared [n].
// efirst[i]: first column of row i inside the envelope of A.  The factor has
// no fill outside the envelope, so every product with an entry left of it
// is zero and is skipped (the sums are unchanged).
// Sets *fail (shared) when a pivot is not positive.
__device__ void chol_blocked(double* A, int n, double* inv_diag, double* colbuf, const int* efirst, int* fail,
                             int nb) {
  const int tid = threadIdx.x, bs = blockDim.x;
  for (int k0 = 0; k0 < n; k0 += nb) {
    const int k1 = min(k0 + nb, n);
    for (int j = k0; j < k1; ++j) {
      if (tid < 32) {
        const int lane = tid;
        double inv = 0.0;
        if (lane == 0) {
          const double d = A[pk(j, j)];
          if (!(d > 0.0)) *fail = 1;
          inv = pivot_rsqrt(d > 0.0 ? d : 1.0);  // one reciprocal square root per pivot
          const double r = (d > 0.0 ? d : 1.0) * inv;
          A[pk(j, j)] = r;
          inv_diag[j] = inv;
        }
        inv = __shfl_sync(BA_FULL_MASK, inv, 0);
        if (j + 1 + lane < k1) colbuf[j + 1 + lane] = A[pk(j + 1 + lane, j)] * inv;
      }
      __syncthreads();
      const double inv = inv_diag[j];
      for (int i = j + 1 + tid; i < n; i += bs) {
        if (efirst[i] > j) continue;  // L(i, j) = 0
        const double l = A[pk(i, j)] * inv;
        A[pk(i, j)] = l;
        const int cmax = min(i, k1 - 1);
        for (int c = j + 1; c <= cmax; ++c) A[pk(i, c)] -= l * colbuf[c];
      }
      __syncthreads();
    }
    if (*fail) return;
    const int m = n - k1;  // trailing matrix rows/cols k1..n-1
    if (m > 0) {
      const int nt = (m + 3) >> 2;
      const int ntiles = nt * (nt + 1) / 2;
      for (int t = tid; t < ntiles; t += bs) {
        int bi = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
        while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
        while (bi * (bi + 1) / 2 > t) --bi;
        const int bc = t - bi * (bi + 1) / 2;
        const int i0 = k1 + 4 * bi, c0 = k1 + 4 * bc;
        // columns of the panel that can be nonzero in both row groups
        int fi = n, fc = n;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          if (i0 + a < n) fi = min(fi, efirst[i0 + a]);
          if (c0 + a < n) fc = min(fc, efirst[c0 + a]);
        }
        const int qlo = max(k0, max(fi, fc));
        if (qlo >= k1) continue;
        double acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
        for (int q = qlo; q < k1; ++q) {
          double li[4], lc[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            li[a] = i0 + a < n ? A[pk(i0 + a, q)] : 0.0;
            lc[a] = c0 + a < n ? A[pk(c0 + a, q)] : 0.0;
          }
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] += li[a] * lc[b];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int i = i0 + a, c = c0 + b;
            if (i < n && c <= i) A[pk(i, c)] -= acc[a][b];
          }
      }
      __syncthreads();
    }
  }
}

// Cholesky with one panel of look-ahead.  Warps 0-3 (group P) factor the
// next panel while warps 4.. (group T) update the rest of the trailing matrix
// with the current panel, so that the panel's sequential pivot chain runs
// behind the trailing update.  Per panel p (columns [k0, k1), already
// factored) and next panel [k1, k2): group P first updates the next panel's
// columns with panel p, then factors them column by column, synchronising on
// a named barrier of its 128 threads; group T updates columns >= k2.  The
// writes of the two groups are disjoint and both only read panel p.  Same
// envelope skipping as chol_blocked.  Requires blockDim.x > 128.
__device__ __forceinline__ void bar_group_p() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// factor columns [k1, k2) (already updated by every earlier panel), group P only
__device__ void chol_panel_p(double* A, int n, int k1, int k2, double* inv_diag, double* colbuf, const int* efirst,
                             int* fail) {
  const int tid = threadIdx.x;
  for (int j = k1; j < k2; ++j) {
    if (tid < 32) {
      double inv = 0.0;
      if (tid == 0) {
        const double d = A[pk(j, j)];
        if (!(d > 0.0)) *fail = 1;
        inv = pivot_rsqrt(d > 0.0 ? d : 1.0);
        A[pk(j, j)] = (d > 0.0 ? d : 1.0) * inv;
        inv_diag[j] = inv;
      }
      inv = __shfl_sync(BA_FULL_MASK, inv, 0);
      if (j + 1 + tid < k2) colbuf[j + 1 + tid] = A[pk(j + 1 + tid, j)] * inv;
    }
    bar_group_p();
    const double inv = inv_diag[j];
    for (int i = j + 1 + tid; i < n; i += 128) {
      if (efirst[i] > j) continue;  // L(i, j) = 0
      const double l = A[pk(i, j)] * inv;
      A[pk(i, j)] = l;
      const int cmax = min(i, k2 - 1);
      for (int c = j + 1; c <= cmax; ++c) A[pk(i, c)] -= l * colbuf[c];
    }
    bar_group_p();
  }
}

__device__ void chol_lookahead(double* A, int n, double* inv_diag, double* colbuf, const int* efirst, int* fail,
                               int nb) {
  const int tid = threadIdx.x;
  const bool gp = tid < 128;
  if (gp) chol_panel_p(A, n, 0, min(nb, n), inv_diag, colbuf, efirst, fail);
  __syncthreads();
  for (int k0 = 0; k0 < n; k0 += nb) {
    if (*fail) return;
    const int k1 = min(k0 + nb, n), k2 = min(k1 + nb, n);
    if (gp) {
      if (k1 < n) {
        // the next panel's columns c in [k1, k2), rows i >= c, with panel p
        const int w = k2 - k1;
        for (int u = tid; u < (n - k1) * w; u += 128) {
          const int i = k1 + u / w, c = k1 + u % w;
          if (c > i) continue;
          const int qlo = max(k0, max(efirst[i], efirst[c]));
          double s = 0.0;
          for (int q = qlo; q < k1; ++q) s += A[pk(i, q)] * A[pk(c, q)];
          A[pk(i, c)] -= s;
        }
        bar_group_p();
        chol_panel_p(A, n, k1, k2, inv_diag, colbuf, efirst, fail);
      }
    } else if (k2 < n) {
      // trailing columns >= k2 with panel p, by the other warps
      const int tt = tid - 128, nt_thr = blockDim.x - 128;
      const int m = n - k2;
      const int nt = (m + 3) >> 2;
      const int ntiles = nt * (nt + 1) / 2;
      for (int t = tt; t < ntiles; t += nt_thr) {
        int bi = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
        while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
        while (bi * (bi + 1) / 2 > t) --bi;
        const int bc = t - bi * (bi + 1) / 2;
        const int i0 = k2 + 4 * bi, c0 = k2 + 4 * bc;
        int fi = n, fc = n;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          if (i0 + a < n) fi = min(fi, efirst[i0 + a]);
          if (c0 + a < n) fc = min(fc, efirst[c0 + a]);
        }
        const int qlo = max(k0, max(fi, fc));
        if (qlo >= k1) continue;
        double acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
        for (int q = qlo; q < k1; ++q) {
          double li[4], lc[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            li[a] = i0 + a < n ? A[pk(i0 + a, q)] : 0.0;
            lc[a] = c0 + a < n ? A[pk(c0 + a, q)] : 0.0;
          }
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] += li[a] * lc[b];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int i = i0 + a, c = c0 + b;
            if (i < n && c <= i) A[pk(i, c)] -= acc[a][b];
          }
      }
    }
    __syncthreads();
  }
}

// After the factorisation: L = Lu D with D = diag(L) and Lu unit lower
// triangular; the strictly lower part of A is scaled to Lu in place (the
// diagonal keeps L(j, j)), so that S = Lu D^2 Lu^T and the sweeps need no
// division.
__device__ void chol_unit_scale(double* A, const double* inv_diag, const int* efirst, int n) {
  const int total = n * (n + 1) / 2;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    int i = (int)((sqrtf(8.0f * (float)idx + 1.0f) - 1.0f) * 0.5f);  // row of packed entry idx
    while ((i + 1) * (i + 2) / 2 <= idx) ++i;
    while (i * (i + 1) / 2 > idx) --i;
    const int j = idx - i * (i + 1) / 2;
    if (j < i && j >= efirst[i]) A[idx] *= inv_diag[j];
  }
}

// Solve S x = b in place (b in shared memory) with S = Lu D^2 Lu^T, by the
// whole CTA.  Per diagonal block of kSolveNB rows, warp 0 sweeps the unit
// triangle (lane = row of the block); then one thread per row updates the
// rest of the vector with the block's columns.  Entries left of a row's
// envelope are zero and skipped.
__device__ void chol_solve_blocked(const double* A, const double* inv_diag, const int* efirst, double* b, int n) {
  const int tid = threadIdx.x, bs = blockDim.x, lane = tid & 31, wid = tid >> 5;
  for (int k0 = 0; k0 < n; k0 += kSolveNB) {  // Lu z = b
    const int k1 = min(k0 + kSolveNB, n);
    if (wid == 0) {
      const int i = k0 + lane;
      double v = i < k1 ? b[i] : 0.0;
      for (int j = k0; j < k1 - 1; ++j) {
        const double z = __shfl_sync(BA_FULL_MASK, v, j - k0);
        if (i > j && i < k1 && efirst[i] <= j) v -= A[pk(i, j)] * z;
      }
      if (i < k1) b[i] = v;
    }
    __syncthreads();
    for (int i = k1 + tid; i < n; i += bs) {  // b_i -= sum_{q in block} Lu(i, q) z_q
      const int q0 = max(k0, efirst[i]);
      double s = 0.0;
      for (int q = q0; q < k1; ++q) s += A[pk(i, q)] * b[q];
      b[i] -= s;
    }
    __syncthreads();
  }
  // w = D^-2 z, one factor 1 / L(i, i) at a time: the square of the
  // reciprocal of a tiny (even subnormal) pivot would overflow
  for (int i = tid; i < n; i += bs) b[i] = (b[i] * inv_diag[i]) * inv_diag[i];
  __syncthreads();
  const int nb = (n + kSolveNB - 1) / kSolveNB;
  for (int blk = nb - 1; blk >= 0; --blk) {  // Lu^T x = w
    const int k0 = blk * kSolveNB, k1 = min(k0 + kSolveNB, n);
    if (wid == 0) {
      const int i = k0 + lane;
      double v = i < k1 ? b[i] : 0.0;
      for (int j = k1 - 1; j > k0; --j) {
        const double xj = __shfl_sync(BA_FULL_MASK, v, j - k0);
        if (i < j && i >= k0 && efirst[j] <= i) v -= A[pk(j, i)] * xj;
      }
      if (i < k1) b[i] = v;
    }
    __syncthreads();
    int lo = k0;  // the block's rows have no entry left of their envelopes
    for (int q = k0; q < k1; ++q) lo = min(lo, efirst[q]);
    for (int i = lo + tid; i < k0; i += bs) {  // b_i -= sum_{q in block} Lu(q, i) x_q
      double s = 0.0;
      for (int q = k0; q < k1; ++q)
        if (efirst[q] <= i) s += A[pk(q, i)] * b[q];
      b[i] -= s;
    }
    __syncthreads();
  }
}

// ---- the same factorisation and solves in double-float (mixed path)
//
// The binary64 pipe of GB300 runs at 1/59 of the binary32 rate, and it bounds
// the binary64 factor of the largest clusters (about 2 DFMA per clock per
// SM).  The mixed path therefore factors an equilibrated copy of the system
// in double-float on the binary32 pipe: A' = E A E with E = diag(2^e_i)
// (powers of two, exact), e_i chosen so that A'(i, i) lies in [1/2, 4); the
// diagonal near 1 keeps every entry of the factor well inside the binary32
// exponent range whatever the scale of A.  A x = b is solved as A' y = E b,
// x = E y; the iterative refinement against the binary64 S (unchanged)
// removes the factor's rounding (double-float, about 2^-47 relative per
// operation).  Same blocking, look-ahead and envelope skipping as the binary64
// functions above; a pivot that is not positive sets *fail.

// A (binary64, packed lower, envelope entries) -> A' = E A E as double-float
// in the same bytes; escale[i] = e_i.  Entries left of a row's envelope are
// zero in both representations.
__device__ void chol_to_scaled_df(double* A, int n, const int* efirst, int* escale) {
  const int tid = threadIdx.x, bs = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = bs >> 5;
  for (int i = tid; i < n; i += bs) {
    const double d = A[pk(i, i)];
    escale[i] = (d > 0.0 && d < INFINITY) ? -(ilogb(d) / 2) : 0;
  }
  __syncthreads();
  dfl* Af = reinterpret_cast<dfl*>(A);
  for (int i = wid; i < n; i += nw) {
    const int ei = escale[i];
    for (int j = efirst[i] + lane; j <= i; j += 32) Af[pk(i, j)] = df_from_d_pow2(A[pk(i, j)], ei + escale[j]);
  }
  __syncthreads();
}

__device__ __forceinline__ dfl shfl_df(dfl v, int src) {
  return dfl{__shfl_sync(BA_FULL_MASK, v.hi, src), __shfl_sync(BA_FULL_MASK, v.lo, src)};
}

// factor columns [k1, k2) (already updated by every earlier panel), group P only
__device__ void chol_panel_p_df(dfl* A, int n, int k1, int k2, dfl* inv_diag, dfl* colbuf, const int* efirst,
                                int* fail) {
  const int tid = threadIdx.x;
  for (int j = k1; j < k2; ++j) {
    if (tid < 32) {
      dfl inv{0.0f, 0.0f};
      if (tid == 0) {
        dfl d = A[pk(j, j)];
        if (!(d.hi > 0.0f)) {
          *fail = 1;
          d = dfl{1.0f, 0.0f};
        }
        inv = df_rsqrt(d);
        A[pk(j, j)] = df_mul(d, inv);
        inv_diag[j] = inv;
      }
      inv = shfl_df(inv, 0);
      if (j + 1 + tid < k2) colbuf[j + 1 + tid] = df_mul(A[pk(j + 1 + tid, j)], inv);
    }
    bar_group_p();
    const dfl inv = inv_diag[j];
    for (int i = j + 1 + tid; i < n; i += 128) {
      if (efirst[i] > j) continue;  // L(i, j) = 0
      const dfl l = df_mul(A[pk(i, j)], inv);
      A[pk(i, j)] = l;
      const int cmax = min(i, k2 - 1);
      for (int c = j + 1; c <= cmax; ++c) A[pk(i, c)] = df_fms(A[pk(i, c)], l, colbuf[c]);
    }
    bar_group_p();
  }
}

__device__ void chol_lookahead_df(dfl* A, int n, dfl* inv_diag, dfl* colbuf, const int* efirst, int* fail, int nb) {
  const int tid = threadIdx.x;
  const bool gp = tid < 128;
  if (gp) chol_panel_p_df(A, n, 0, min(nb, n), inv_diag, colbuf, efirst, fail);
  __syncthreads();
  for (int k0 = 0; k0 < n; k0 += nb) {
    if (*fail) return;
    const int k1 = min(k0 + nb, n), k2 = min(k1 + nb, n);
    if (gp) {
      if (k1 < n) {
        const int w = k2 - k1;
        for (int u = tid; u < (n - k1) * w; u += 128) {
          const int i = k1 + u / w, c = k1 + u % w;
          if (c > i) continue;
          const int qlo = max(k0, max(efirst[i], efirst[c]));
          if (qlo >= k1) continue;
          Dot2 s;
          for (int q = qlo; q < k1; ++q) s.add(A[pk(i, q)], A[pk(c, q)]);
          A[pk(i, c)] = df_sub(A[pk(i, c)], s.get());
        }
        bar_group_p();
        chol_panel_p_df(A, n, k1, k2, inv_diag, colbuf, efirst, fail);
      }
    } else if (k2 < n) {
      const int tt = tid - 128, nt_thr = blockDim.x - 128;
      const int m = n - k2;
      const int nt = (m + 3) >> 2;
      const int ntiles = nt * (nt + 1) / 2;
      for (int t = tt; t < ntiles; t += nt_thr) {
        int bi = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
        while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
        while (bi * (bi + 1) / 2 > t) --bi;
        const int bc = t - bi * (bi + 1) / 2;
        const int i0 = k2 + 4 * bi, c0 = k2 + 4 * bc;
        int fi = n, fc = n;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          if (i0 + a < n) fi = min(fi, efirst[i0 + a]);
          if (c0 + a < n) fc = min(fc, efirst[c0 + a]);
        }
        const int qlo = max(k0, max(fi, fc));
        if (qlo >= k1) continue;
        Dot2 acc[4][4];
        for (int q = qlo; q < k1; ++q) {
          dfl li[4], lc[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            li[a] = i0 + a < n ? A[pk(i0 + a, q)] : dfl{0.0f, 0.0f};
            lc[a] = c0 + a < n ? A[pk(c0 + a, q)] : dfl{0.0f, 0.0f};
          }
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b].add(li[a], lc[b]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int i = i0 + a, c = c0 + b;
            if (i < n && c <= i) A[pk(i, c)] = df_sub(A[pk(i, c)], acc[a][b].get());
          }
      }
    }
    __syncthreads();
  }
}

__device__ void chol_unit_scale_df(dfl* A, const dfl* inv_diag, const int* efirst, int n) {
  const int tid = threadIdx.x, bs = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = bs >> 5;
  (void)bs;
  for (int i = wid; i < n; i += nw)
    for (int j = efirst[i] + lane; j < i; j += 32) A[pk(i, j)] = df_mul(A[pk(i, j)], inv_diag[j]);
}

// Inverses of the unit-lower diagonal blocks of kSolveNB rows of Lu, packed
// lower (entry (r, c) of a block at r (r + 1) / 2 + c, the unit diagonal
// stored), one warp per block, lane = column c:
// X(c, c) = 1, X(r, c) = -sum_{q=c}^{r-1} Lu(r, q) X(q, c) for r > c.
// The solves then apply each block as a product instead of a sequential
// substitution.
constexpr int kSolveTri = kSolveNB * (kSolveNB + 1) / 2;
__device__ void chol_block_inverses_df(const dfl* A, const int* efirst, dfl* binv, int n) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nb = (n + kSolveNB - 1) / kSolveNB;
  for (int blk = wid; blk < nb; blk += nw) {
    const int k0 = blk * kSolveNB, m = min(kSolveNB, n - k0);
    dfl* X = binv + (size_t)blk * kSolveTri;
    const int c = lane;
    if (c >= m) continue;
    X[c * (c + 1) / 2 + c] = dfl{1.0f, 0.0f};
    for (int r = c + 1; r < m; ++r) {
      const int qs = max(c, efirst[k0 + r] - k0);  // Lu(r, q) = 0 left of the envelope
      const dfl* Lr = A + pk(k0 + r, k0);
      Dot2 s0, s1;
      int q = qs;
      for (; q + 1 < r; q += 2) {
        s0.add(Lr[q], X[q * (q + 1) / 2 + c]);
        s1.add(Lr[q + 1], X[(q + 1) * (q + 2) / 2 + c]);
      }
      for (; q < r; ++q) s0.add(Lr[q], X[q * (q + 1) / 2 + c]);
      s0.merge(s1.s, s1.c);
      X[r * (r + 1) / 2 + c] = df_neg(s0.get());
    }
  }
}

// S' y = b in place with S' = Lu D^2 Lu^T (double-float): the sweeps of
// chol_solve_blocked, each diagonal block applied through its inverse (warp
// 0, lane = row), the rest of the vector updated thread per row, all sums
// compensated (Dot2)
__device__ void chol_solve_df(const dfl* A, const dfl* inv_diag, const int* efirst, const dfl* binv, dfl* b, int n) {
  const int tid = threadIdx.x, bs = blockDim.x, lane = tid & 31, wid = tid >> 5;
  for (int k0 = 0; k0 < n; k0 += kSolveNB) {  // Lu z = b
    const int k1 = min(k0 + kSolveNB, n);
    if (wid == 0) {
      const dfl* X = binv + (size_t)(k0 / kSolveNB) * kSolveTri;
      const int r = lane, i = k0 + r;
      dfl v{0.0f, 0.0f};
      if (i < k1) {  // z_r = sum_{q <= r} X(r, q) b_q
        const dfl* Xr = X + r * (r + 1) / 2;
        Dot2 s0, s1;
        int q = 0;
        for (; q + 1 <= r; q += 2) {
          s0.add(Xr[q], b[k0 + q]);
          s1.add(Xr[q + 1], b[k0 + q + 1]);
        }
        for (; q <= r; ++q) s0.add(Xr[q], b[k0 + q]);
        s0.merge(s1.s, s1.c);
        v = s0.get();
      }
      __syncwarp();
      if (i < k1) b[i] = v;
    }
    __syncthreads();
    for (int i = k1 + tid; i < n; i += bs) {
      const int q0 = max(k0, efirst[i]);
      if (q0 >= k1) continue;
      Dot2 s0, s1, s2, s3;  // four interleaved sums, merged in a fixed order
      int q = q0;
      for (; q + 3 < k1; q += 4) {
        s0.add(A[pk(i, q)], b[q]);
        s1.add(A[pk(i, q + 1)], b[q + 1]);
        s2.add(A[pk(i, q + 2)], b[q + 2]);
        s3.add(A[pk(i, q + 3)], b[q + 3]);
      }
      for (; q < k1; ++q) s0.add(A[pk(i, q)], b[q]);
      s0.merge(s1.s, s1.c);
      s2.merge(s3.s, s3.c);
      s0.merge(s2.s, s2.c);
      b[i] = df_sub(b[i], s0.get());
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += bs) b[i] = df_mul(df_mul(b[i], inv_diag[i]), inv_diag[i]);  // D^-2
  __syncthreads();
  const int nb = (n + kSolveNB - 1) / kSolveNB;
  for (int blk = nb - 1; blk >= 0; --blk) {  // Lu^T x = w
    const int k0 = blk * kSolveNB, k1 = min(k0 + kSolveNB, n), m = k1 - k0;
    if (wid == 0) {
      const dfl* X = binv + (size_t)blk * kSolveTri;
      const int r = lane, i = k0 + r;
      dfl v{0.0f, 0.0f};
      if (i < k1) {  // x_r = sum_{q >= r} X(q, r) w_q
        Dot2 s0, s1;
        int q = r;
        for (; q + 1 < m; q += 2) {
          s0.add(X[q * (q + 1) / 2 + r], b[k0 + q]);
          s1.add(X[(q + 1) * (q + 2) / 2 + r], b[k0 + q + 1]);
        }
        for (; q < m; ++q) s0.add(X[q * (q + 1) / 2 + r], b[k0 + q]);
        s0.merge(s1.s, s1.c);
        v = s0.get();
      }
      __syncwarp();
      if (i < k1) b[i] = v;
    }
    __syncthreads();
    int lo = k0;
    for (int q = k0; q < k1; ++q) lo = min(lo, efirst[q]);
    for (int i = lo + tid; i < k0; i += bs) {
      // the block's rows whose envelope reaches column i are a prefix
      // [k0, qe) of it (the envelope is monotone)
      int qe = k0;
      while (qe < k1 && efirst[qe] <= i) ++qe;
      if (qe == k0) continue;
      Dot2 s0, s1, s2, s3;
      int q = k0;
      for (; q + 3 < qe; q += 4) {
        s0.add(A[pk(q, i)], b[q]);
        s1.add(A[pk(q + 1, i)], b[q + 1]);
        s2.add(A[pk(q + 2, i)], b[q + 2]);
        s3.add(A[pk(q + 3, i)], b[q + 3]);
      }
      for (; q < qe; ++q) s0.add(A[pk(q, i)], b[q]);
      s0.merge(s1.s, s1.c);
      s2.merge(s3.s, s3.c);
      s0.merge(s2.s, s2.c);
      b[i] = df_sub(b[i], s0.get());
    }
    __syncthreads();
  }
}

// A x = v for the binary64 vector v (in place): scaled into double-float in
// the same bytes, solved, scaled back
__device__ void solve_scaled_df(const dfl* A, const dfl* inv_diag, const int* efirst, const int* escale,
                                const dfl* binv, double* v, int n) {
  dfl* vf = reinterpret_cast<dfl*>(v);
  for (int i = threadIdx.x; i < n; i += blockDim.x) vf[i] = df_from_d_pow2(v[i], escale[i]);
  __syncthreads();
  chol_solve_df(A, inv_diag, efirst, binv, vf, n);
  for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = ldexp(df_to_d(vf[i]), escale[i]);
  __syncthreads();
}

template <bool MIXED>
__global__ void __launch_bounds__(kFactorThreads) k_factor_solve(BatchView bv, int refine_steps, int assemble_only) {
  using Real = typename RealOf<MIXED>::T;
  extern __shared__ double sm[];
  __shared__ int fail;
  const int tid = threadIdx.x, bs = blockDim.x;
  for (int so = blockIdx.x; so < bv.n; so += gridDim.x) {
    const int s = bv.factor_order[so];  // largest systems first
    const DevCluster& C = bv.cl[s];
    LmState* lm = C.lm;
    if (!lm->active && !assemble_only) continue;
    if (C.n_free > kMaxFreeSmall) continue;  // the global-memory solver takes larger systems
    const int nf = C.n_free, n = 6 * nf, nc = C.n_cams;
    const double mu = lm->mu;
    const int cur = lm->cur;
    double* A = sm;
    double* cd = A + (size_t)n * (n + 1) / 2;  // [nf][40]
    double* pr = cd + (size_t)nf * 40;         // [nf][42]: JtJ 36, Jtr 6
    double* x = pr + (size_t)nf * 42;          // [n]
    double* b = x + n;                         // [n]
    double* t = b + n;                         // [n]
    double* inv_diag = t + n;                  // [n]
    const double* Rc = C.R + (size_t)cur * nc * 9;
    const double* Tc = C.T + (size_t)cur * nc * 3;

    if (tid == 0) lm->tiles_done = 0;  // the back-substitution counts its tiles from here
    // per-camera sums (k_partial_reduce)
    for (int idx = tid; idx < nf * 39; idx += bs) {
      const int f = idx / 39, e = idx - 39 * f;
      cd[40 * f + e] = C.camsum[(size_t)kCamPart * f + e];
    }
    for (int f = tid; f < nf; f += bs) {
      const int k = C.cam_of_free[f];
      prior_terms(Rc + 9 * k, Tc + 3 * k, C.R_prior + 9 * k, C.T_prior + 3 * k, C.sigma_imu, C.sigma_gnss,
                  pr + 42 * f, pr + 42 * f + 36);
    }
    for (int idx = tid; idx < n * (n + 1) / 2; idx += bs) A[idx] = 0.0;
    if (tid == 0) fail = lm->pt_fail;
    __syncthreads();
    // diagonal blocks: U + prior + mu D - sum Z Z^T
    for (int idx = tid; idx < nf * 21; idx += bs) {
      const int f = idx / 21;
      int e = idx - 21 * f, a = 0;
      while (e >= 6 - a) { e -= 6 - a; ++a; }
      const int bb = a + e;  // a <= bb, packed upper index of (a, bb)
      const int ui = idx - 21 * f;
      double v = cd[40 * f + ui] + pr[42 * f + 6 * a + bb];
      if (a == bb) {
        const double D = clamp_diag(cd[40 * f + 33 + a] + pr[42 * f + 7 * a]);
        v += mu * D;
        C.Dc[6 * f + a] = D;
      }
      const int p = C.fpos[f];
      A[pk(6 * p + bb, 6 * p + a)] = v;  // row bb >= col a
    }
    for (int idx = tid; idx < n; idx += bs) {
      const int f = idx / 6, a = idx - 6 * f;
      const double g = cd[40 * f + 21 + a] - pr[42 * f + 36 + a];
      C.gc[idx] = g;
      const double r = g - cd[40 * f + 27 + a];
      const int pi = 6 * C.fpos[f] + a;  // elimination order
      C.rhs[pi] = r;
      b[pi] = r;
    }
    // off-diagonal blocks: S(fb, fa) = -(sum Z_a Z_b^T)^T
    for (int idx = tid; idx < C.n_pairs * 36; idx += bs) {
      const int p = idx / 36, e = idx - 36 * p;
      const int i = e / 6, c = e - 6 * i;
      const double v = C.pairsum[(size_t)kPairPart * p + e];
      const int2 key = C.pair_key[p];
      const int pa = C.fpos[key.x], pb = C.fpos[key.y];
      if (pb > pa) A[pk(6 * pb + c, 6 * pa + i)] = -v;
      else A[pk(6 * pa + i, 6 * pb + c)] = -v;
    }
    __syncthreads();
    if (assemble_only || refine_steps > 0) {  // S in binary64 for the refinement (only the refinement reads it)
      for (int idx = tid; idx < n * n; idx += bs) {
        const int r = idx / n, c = idx - n * r;
        C.S[idx] = r >= c ? A[pk(r, c)] : A[pk(c, r)];
      }
    }
    if (assemble_only) {
      __syncthreads();
      continue;
    }
    __syncthreads();  // the copy of S above reads A
    // blocked right-looking Cholesky in shared memory (t[] is the column buffer)
    int* efirst = reinterpret_cast<int*>(inv_diag + n);  // [n]: first column of each row's envelope
    for (int idx = tid; idx < n; idx += bs) efirst[idx] = 6 * C.env_first[idx / 6];
    __syncthreads();
    // double-float factor of the equilibrated system (escale: its exponents):
    // the mixed path, and the binary64 path under BA_FLAG_SMALL_DF_FACTOR
    const bool use_df = MIXED || bv.factor_df;
    int* escale = efirst + n;
    dfl* binv = reinterpret_cast<dfl*>(inv_diag + 2 * n);  // inverses of the solves' diagonal blocks
    dfl* Af = reinterpret_cast<dfl*>(A);
    dfl* inv_f = reinterpret_cast<dfl*>(inv_diag);
    if (use_df) {
      chol_to_scaled_df(A, n, efirst, escale);
      if (!fail) chol_lookahead_df(Af, n, inv_f, reinterpret_cast<dfl*>(t), efirst, &fail, bv.factor_nb);
    } else {
#ifdef BA_FACTOR_NO_LOOKAHEAD
      if (!fail) chol_blocked(A, n, inv_diag, t, efirst, &fail, bv.factor_nb);
#else
      if (!fail) chol_lookahead(A, n, inv_diag, t, efirst, &fail, bv.factor_nb);
#endif
    }
    __syncthreads();
    const int status = fail ? BA_STATUS_NOT_PD : 0;
    if (!fail) {
      if (use_df) {
        chol_unit_scale_df(Af, inv_f, efirst, n);
        __syncthreads();
        chol_block_inverses_df(Af, efirst, binv, n);
        __syncthreads();
        solve_scaled_df(Af, inv_f, efirst, escale, binv, b, n);
      } else {
        chol_unit_scale(A, inv_diag, efirst, n);
        __syncthreads();
        chol_solve_blocked(A, inv_diag, efirst, b, n);
      }
      for (int idx = tid; idx < n; idx += bs) x[idx] = b[idx];
      __syncthreads();
      // iterative refinement against the FP64 system kept in global memory
      for (int it = 0; it < refine_steps; ++it) {
        const int lane = tid & 31, wid = tid >> 5, nw = bs >> 5;
        for (int r = wid; r < n; r += nw) {
          double acc = 0.0;
          for (int c = efirst[r] + lane; c < n; c += 32)  // zero blocks outside the envelope skipped
            if (c <= r || efirst[c] <= r) acc += C.S[(size_t)r * n + c] * x[c];
          acc = warp_sum(acc);
          if (lane == 0) t[r] = C.rhs[r] - acc;
        }
        __syncthreads();
        if (use_df) solve_scaled_df(Af, inv_f, efirst, escale, binv, t, n);
        else chol_solve_blocked(A, inv_diag, efirst, t, n);
        for (int idx = tid; idx < n; idx += bs) x[idx] += t[idx];
        __syncthreads();
      }
      for (int idx = tid; idx < n; idx += bs) {  // back to free-image order
        const double v = x[6 * C.fpos[idx / 6] + idx % 6];
        C.dc[idx] = v;
        if (MIXED) C.dc32[idx] = (float)v;
      }
    } else {
      for (int idx = tid; idx < n; idx += bs) {
        C.dc[idx] = 0.0;
        if (MIXED) C.dc32[idx] = 0.0f;
        x[idx] = 0.0;
      }
    }
    __syncthreads();
    // candidate cameras; per-camera prior cost and pred terms into t[]
    for (int k = tid; k < nc; k += bs) {
      const int f = C.free_idx[k];
      double pc, pn;
      candidate_camera<MIXED>(C, k, x, mu, cur, fail != 0, &pc, &pn);
      if (f >= 0) {
        t[2 * f] = pc;
        t[2 * f + 1] = pn;
      }
    }
    __syncthreads();
    if (tid == 0) {
      double pc = 0.0, pn = 0.0;
      for (int f = 0; f < nf; ++f) { pc += t[2 * f]; pn += t[2 * f + 1]; }
      lm->pred_cam = pc;
      lm->prior_new = pn;
      lm->status = lm->dev_error ? lm->dev_error : status;
      lm->dev_error = 0;
    }
    __syncthreads();
    // a cluster without observations has no back-substitution tile to count:
    // its LM step is taken here
    if (!assemble_only && C.n_tiles == 0 && tid < 32) lm_update_warp<MIXED>(C, tid);
    __syncthreads();
  }
}

// ------------------------------------------------------------------ K5

// Back-substitution and candidate cost, warp per tile.  The tile is
// linearised again (the same arithmetic as in k_lin_schur) instead of reading
// per-observation records back from memory.
template <bool MIXED>
__device__ void backsub_tile(const DevCluster& C, LmState* lm, int local, int lane);

// add a warp's count of finished tiles to its cluster's total; the warp that
// completes the total takes the cluster's LM decision
template <bool MIXED>
__device__ __forceinline__ void publish_tiles(const DevCluster& C, int count, int lane) {
  int done = 0;
  if (lane == 0) {
    __threadfence();  // this warp's partial sums before the count
    done = atomicAdd(&C.lm->tiles_done, count) + count;
  }
  done = __shfl_sync(BA_FULL_MASK, done, 0);
  if (done == C.n_tiles) {
    __threadfence();
    lm_update_warp<MIXED>(C, lane);
  }
}

template <bool MIXED>
__global__ void __launch_bounds__(256) k_backsub_cost(BatchView bv) {
  using Real = typename RealOf<MIXED>::T;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int total = bv.tot[0];
  // each warp takes a contiguous run of tiles, so that its tiles mostly
  // belong to one cluster: it counts them per cluster and publishes the
  // count once per cluster it leaves (one fence and one atomic each); the
  // warp whose count completes a cluster takes the cluster's LM decision,
  // every other tile's partial sums being written by then
  const int per = (total + nwarps - 1) / nwarps;
  const int g0 = warp * per, g1 = min(total, g0 + per);
  int s = g0 < g1 ? find_slot(bv.tile_pre, bv.n, g0) : 0;
  int pending = 0;
  for (int g = g0; g < g1; ++g) {
    while (g >= bv.tile_pre[s + 1]) {  // the next cluster: publish the count of this one
      if (pending) publish_tiles<MIXED>(bv.cl[s], pending, lane);
      pending = 0;
      ++s;
    }
    const DevCluster& C = bv.cl[s];
    LmState* lm = C.lm;
    if (!lm->active) continue;
    if (lm->status == 0) backsub_tile<MIXED>(C, lm, g - bv.tile_pre[s], lane);
    ++pending;
  }
  if (pending) publish_tiles<MIXED>(bv.cl[s], pending, lane);
}

// back-substitution and candidate cost of one tile (one warp)
template <bool MIXED>
__device__ void backsub_tile(const DevCluster& C, LmState* lm, int local, int lane) {
  using Real = typename RealOf<MIXED>::T;
  {
    const Tile tl = C.tiles[local];
    TileLin<MIXED> L;
    linearize_tile<MIXED, false, true>(C, lm, tl, lane, false, L, global_view(C, lm->cur));
    const int cur = lm->cur;
    Real mu_r;
    if constexpr (MIXED) mu_r = lm->mu_f; else mu_r = lm->mu;
    // t = Z^T dc_k = P^T (Jc dc_k)
    Real t0 = 0, t1 = 0, t2 = 0;
    const int f = L.act ? C.free_idx[L.k] : -1;
    if (f >= 0) {
      Real d[6];
      if constexpr (MIXED) {
        const float2* d2 = reinterpret_cast<const float2*>(C.dc32 + 6 * f);
        const float2 u0 = d2[0], u1 = d2[1], u2 = d2[2];
        d[0] = u0.x; d[1] = u0.y; d[2] = u1.x; d[3] = u1.y; d[4] = u2.x; d[5] = u2.y;
      } else {
#pragma unroll
        for (int m = 0; m < 6; ++m) d[m] = C.dc[6 * f + m];
      }
      Real u0 = 0, u1 = 0;
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        u0 += L.Jc[m] * d[m];
        u1 += L.Jc[6 + m] * d[m];
      }
      t0 = L.P[0] * u0 + L.P[3] * u1;
      t1 = L.P[1] * u0 + L.P[4] * u1;
      t2 = L.P[2] * u0 + L.P[5] * u1;
    }
    t0 = seg_reduce(t0, lane, L.seg_start, L.seg_end, L.span);
    t1 = seg_reduce(t1, lane, L.seg_start, L.seg_end, L.span);
    t2 = seg_reduce(t2, lane, L.seg_start, L.seg_end, L.span);
    // head: dX = M^T (q - t), candidate point, pred term
    Real dX0 = 0, dX1 = 0, dX2 = 0;
    Real pp = 0;  // dX^T (mu Dp dX + gp)
    if (L.head) {
      const Real v0 = L.q0 - t0, v1 = L.q1 - t1, v2 = L.q2 - t2;
      dX0 = L.m00 * v0 + L.m10 * v1 + L.m20 * v2;
      dX1 = L.m11 * v1 + L.m21 * v2;
      dX2 = L.m22 * v2;
      pp = dX0 * (mu_r * L.d0 * dX0 + L.g0) + dX1 * (mu_r * L.d1 * dX1 + L.g1) + dX2 * (mu_r * L.d2 * dX2 + L.g2);
    }
    const int o = L.o, k = L.k, j = L.j;
    const bool act = L.act;
    const int seg_start = L.seg_start;
    double cost = 0.0;
    if constexpr (MIXED) {
      dfl x0{0.f, 0.f}, x1{0.f, 0.f}, x2{0.f, 0.f};
      if (L.head) {
        const float2* xp = xdf_ptr(C, cur, j);
        const float2 a = xp[0], b = xp[1], c = xp[2];
        x0 = df_add_f(dfl{a.x, a.y}, dX0);
        x1 = df_add_f(dfl{b.x, b.y}, dX1);
        x2 = df_add_f(dfl{c.x, c.y}, dX2);
        float2* xn = xdf_wptr(C, cur ^ 1, j);
        xn[0] = make_float2(x0.hi, x0.lo);
        xn[1] = make_float2(x1.hi, x1.lo);
        xn[2] = make_float2(x2.hi, x2.lo);
      }
      x0.hi = __shfl_sync(BA_FULL_MASK, x0.hi, seg_start); x0.lo = __shfl_sync(BA_FULL_MASK, x0.lo, seg_start);
      x1.hi = __shfl_sync(BA_FULL_MASK, x1.hi, seg_start); x1.lo = __shfl_sync(BA_FULL_MASK, x1.lo, seg_start);
      x2.hi = __shfl_sync(BA_FULL_MASK, x2.hi, seg_start); x2.lo = __shfl_sync(BA_FULL_MASK, x2.lo, seg_start);
      dfl cst{0.f, 0.f};
      if (act) {
        const CamDf cdf = load_camdf(camdf_ptr(C, cur ^ 1, k));
        const float2 ch = C.obs_chi[o], cl = C.obs_clo[o];
        dfl e0, e1;
        if (df_residual(cdf, x0, x1, x2, dfl{ch.x, cl.x}, dfl{ch.y, cl.y}, e0, e1))
          cst = df_robust_cost(e0, e1, C.delta_f, C.half_inv_s2_f);
      }
      // fixed-order warp sum in double-float, one conversion per warp
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const dfl o2{__shfl_down_sync(BA_FULL_MASK, cst.hi, off), __shfl_down_sync(BA_FULL_MASK, cst.lo, off)};
        cst = df_add(cst, o2);
      }
      if (lane == 0) cost = df_to_d(cst);
    } else {
      double x0 = 0.0, x1 = 0.0, x2 = 0.0;
      if (L.head) {
        const double* X = C.X + ((size_t)cur * C.n_pts + j) * 3;
        x0 = X[0] + (double)dX0;
        x1 = X[1] + (double)dX1;
        x2 = X[2] + (double)dX2;
        double* Xn = C.X + ((size_t)(cur ^ 1) * C.n_pts + j) * 3;
        Xn[0] = x0; Xn[1] = x1; Xn[2] = x2;
      }
      x0 = __shfl_sync(BA_FULL_MASK, x0, seg_start);
      x1 = __shfl_sync(BA_FULL_MASK, x1, seg_start);
      x2 = __shfl_sync(BA_FULL_MASK, x2, seg_start);
      if (act) {
        const double Xn[3] = {x0, x1, x2};
        const double* Rn = C.R + ((size_t)(cur ^ 1) * C.n_cams + k) * 9;
        const double* Tn = C.T + ((size_t)(cur ^ 1) * C.n_cams + k) * 3;
        const double2 u = reinterpret_cast<const double2*>(C.obs_uv)[o];
        cost = obs_cost(Rn, Tn, C.intr + 7 * k, Xn, u.x, u.y, 0.5 / (C.sigma_px * C.sigma_px), C.huber_delta);
      }
      cost = warp_sum(cost);
    }
    double ppred;
    if constexpr (MIXED) {
      const float ps = warp_sum(pp);  // binary32 warp sum, one conversion per warp
      ppred = lane == 0 ? (double)ps : 0.0;
    } else {
      ppred = warp_sum((double)pp);
    }
    if (lane == 0) {
      C.tilepart[2 * local] = cost;
      C.tilepart[2 * local + 1] = ppred;
    }
  }
}

// ------------------------------------------------------------------ cost at the current state

template <bool MIXED>
__global__ void __launch_bounds__(256) k_cost_tiles(BatchView bv) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int total = bv.tot[0];
  for (int g = warp; g < total; g += nwarps) {
    const int s = find_slot(bv.tile_pre, bv.n, g);
    const DevCluster& C = bv.cl[s];
    const LmState* lm = C.lm;
    if (!lm->needs_init) continue;
    const int local = g - bv.tile_pre[s];
    const Tile tl = C.tiles[local];
    const int cur = lm->cur;
    double cost = 0.0;
    if constexpr (MIXED) {
      dfl cst{0.f, 0.f};
      if (lane < tl.n_obs) {
        const int o = tl.obs_begin + lane;
        const int k = C.obs_cam[o], j = C.obs_pt[o];
        const CamDf cdf = load_camdf(camdf_ptr(C, cur, k));
        const float2* xp = xdf_ptr(C, cur, j);
        const float2 a = xp[0], b = xp[1], c = xp[2];
        const float2 ch = C.obs_chi[o], cl = C.obs_clo[o];
        dfl e0, e1;
        if (df_residual(cdf, dfl{a.x, a.y}, dfl{b.x, b.y}, dfl{c.x, c.y}, dfl{ch.x, cl.x}, dfl{ch.y, cl.y}, e0, e1))
          cst = df_robust_cost(e0, e1, C.delta_f, C.half_inv_s2_f);
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const dfl o2{__shfl_down_sync(BA_FULL_MASK, cst.hi, off), __shfl_down_sync(BA_FULL_MASK, cst.lo, off)};
        cst = df_add(cst, o2);
      }
      if (lane == 0) cost = df_to_d(cst);
    } else {
      if (lane < tl.n_obs) {
        const int o = tl.obs_begin + lane;
        const int k = C.obs_cam[o], j = C.obs_pt[o];
        const double2 u = reinterpret_cast<const double2*>(C.obs_uv)[o];
        cost = obs_cost(C.R + ((size_t)cur * C.n_cams + k) * 9, C.T + ((size_t)cur * C.n_cams + k) * 3,
                        C.intr + 7 * k, C.X + ((size_t)cur * C.n_pts + j) * 3, u.x, u.y,
                        0.5 / (C.sigma_px * C.sigma_px), C.huber_delta);
      }
      cost = warp_sum(cost);
    }
    if (lane == 0) C.tilepart[2 * local] = cost;
  }
}

// fixed-order block sum of tilepart[:, which]
// Both per-tile sums (cost at the candidate, pred) over the cluster's tiles,
// in a fixed order: each thread a strided run of tiles, then a warp tree and
// the warps in order.  red: shared [2][blockDim / 32].  Valid in thread 0.
__device__ double2 block_sum_tiles2(const DevCluster& C, double* red) {
  double a = 0.0, b = 0.0;
  const double2* tp = reinterpret_cast<const double2*>(C.tilepart);
  for (int i = threadIdx.x; i < C.n_tiles; i += blockDim.x) {
    const double2 v = tp[i];
    a += v.x;
    b += v.y;
  }
  a = warp_sum(a);
  b = warp_sum(b);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    red[wid] = a;
    red[nw + wid] = b;
  }
  __syncthreads();
  double2 tot = make_double2(0.0, 0.0);
  if (threadIdx.x == 0)
    for (int w = 0; w < nw; ++w) {
      tot.x += red[w];
      tot.y += red[nw + w];
    }
  __syncthreads();
  return tot;
}

__device__ double block_sum_tiles(const DevCluster& C, int which, double* red) {
  double v = 0.0;
  for (int i = threadIdx.x; i < C.n_tiles; i += blockDim.x) v += C.tilepart[2 * i + which];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
  __syncthreads();
  return tot;  // valid in thread 0
}

// Fixed-order sum over the block (warp trees, then the warps in order);
// valid in thread 0.
__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
  __syncthreads();
  return tot;
}

__global__ void __launch_bounds__(256) k_cost_init(BatchView bv) {
  __shared__ double red[8];
  for (int s = blockIdx.x; s < bv.n; s += gridDim.x) {
    const DevCluster& C = bv.cl[s];
    LmState* lm = C.lm;
    if (!lm->needs_init) continue;
    const double F = block_sum_tiles(C, 0, red);
    // prior terms of the free images at the current state: thread t takes
    // images t, t + blockDim.x, ... in order
    const int cur = lm->cur;
    double pc = 0.0;
    for (int k = threadIdx.x; k < C.n_cams; k += blockDim.x) {
      if (C.free_idx[k] < 0) continue;
      pc += prior_terms(C.R + ((size_t)cur * C.n_cams + k) * 9, C.T + ((size_t)cur * C.n_cams + k) * 3,
                        C.R_prior + 9 * k, C.T_prior + 3 * k, C.sigma_imu, C.sigma_gnss, nullptr, nullptr);
    }
    pc = block_sum(pc, red);
    if (threadIdx.x == 0) {
      lm->needs_init = 0;
      lm->F = F + pc;
      lm->pt_fail = 0;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ K6

// ------------------------------------------------------------------ diagnostics

__global__ void k_grad_norm(BatchView bv, double* out) {
  __shared__ double red[8];
  for (int s = blockIdx.x; s < bv.n; s += gridDim.x) {
    const DevCluster& C = bv.cl[s];
    double m = 0.0;
    for (int i = threadIdx.x; i < 6 * C.n_free; i += blockDim.x) m = fmax(m, fabs(C.gc[i]));
    for (int t = threadIdx.x; t < C.n_tiles; t += blockDim.x) m = fmax(m, C.tilepart[2 * t + 1]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(BA_FULL_MASK, m, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      double v = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = fmax(v, red[w]);
      out[s] = v;
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void point_f64(const DevCluster& C, bool mixed, int buf, int j, double X[3]) {
  if (mixed) {
    const float2* p = xdf_ptr(C, buf, j);
    for (int i = 0; i < 3; ++i) X[i] = (double)p[i].x + (double)p[i].y;
  } else {
    const double* p = C.X + ((size_t)buf * C.n_pts + j) * 3;
    for (int i = 0; i < 3; ++i) X[i] = p[i];
  }
}

__global__ void k_reproj(const DevCluster* dcl, int mixed, double* err) {
  const DevCluster& C = *dcl;
  const int cur = C.lm->cur;
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < C.n_obs; o += gridDim.x * blockDim.x) {
    const int k = C.obs_cam[o], j = C.obs_pt[o];
    const double2 u = reinterpret_cast<const double2*>(C.obs_uv)[o];
    double X[3];
    point_f64(C, mixed, cur, j, X);
    err[o] = obs_error_norm(C.R + ((size_t)cur * C.n_cams + k) * 9, C.T + ((size_t)cur * C.n_cams + k) * 3,
                            C.intr + 7 * k, X, u.x, u.y);
  }
}

// The current state in the caller's layout, binary64: R [nc][9] and T [nc][3]
// of the current buffer, X [np][3] in the caller's point order (any output
// may be null).
__global__ void k_export_state(const DevCluster* dcl, int mixed, double* R, double* T, double* out) {
  const DevCluster& C = *dcl;
  const int cur = C.lm->cur;
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 12 * C.n_cams; i += stride) {
    if (i < 9 * C.n_cams) {
      if (R) R[i] = C.R[(size_t)cur * C.n_cams * 9 + i];
    } else if (T) {
      T[i - 9 * C.n_cams] = C.T[(size_t)cur * C.n_cams * 3 + i - 9 * C.n_cams];
    }
  }
  if (!out) return;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < C.n_pts; j += stride) {
    double X[3];
    point_f64(C, mixed, cur, j, X);
    const int u = C.pt_perm[j];  // caller's index
    out[3 * u] = X[0];
    out[3 * u + 1] = X[1];
    out[3 * u + 2] = X[2];
  }
}

// ------------------------------------------------------------------ run control

// Arm every cluster of the batch for `iters` more iterations (iters < 0:
// mark active without a target, for the diagnostic linearisation).
__global__ void k_arm(BatchView bv, int iters) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < bv.n; s += gridDim.x * blockDim.x) {
    LmState* lm = bv.cl[s].lm;
    if (iters >= 0) {
      lm->iters_target = lm->iter + iters;
      lm->active = iters > 0;
    } else {
      lm->active = iters == -1;
    }
    lm->needs_init = 1;
    lm->pt_fail = 0;
    lm->iter0 = lm->iter;
    lm->ftol = 0.0;
  }
}

// Serving slots: arm[s] > 0 starts arm[s] more iterations for slot s (and asks
// for F at its state first), ending early on convergence when ftol[s] > 0; 0
// leaves the slot as it is.
__global__ void k_arm_slots(BatchView bv, const int* arm, const double* ftol) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < bv.n; s += gridDim.x * blockDim.x) {
    const int a = arm[s];
    if (a <= 0) continue;
    LmState* lm = bv.cl[s].lm;
    lm->iters_target = lm->iter + a;
    lm->active = 1;
    lm->needs_init = 1;
    lm->pt_fail = 0;
    lm->iter0 = lm->iter;
    lm->ftol = ftol[s];
  }
}

// Warm start: copy the current state of shared cameras and points from a live
// cluster (src) into a new one (dst): both state buffers and the reset state.
// cams / pts hold (dst index, src index) pairs in internal order.  The copy is
// representation-agnostic (8-byte words), so both clusters must use the same
// precision.
// Cluster transition (Sec. 3.2, Eq. 8): an image free in dst and shared with
// src takes the weighted average of its two current poses, weights = its
// observations in each cluster; orientation at fraction w_dst / (w_src +
// w_dst) along the geodesic from the src orientation, position the weighted
// mean.  Binary64.  pairs[i] = (camera in dst, camera in src).
__global__ void k_transition(const DevCluster* dst, const DevCluster* src, const int2* pairs, int n) {
  const DevCluster& D = *dst;
  const DevCluster& S = *src;
  const int dcur = D.lm->cur, scur = S.lm->cur;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int kd = pairs[i].x, ks = pairs[i].y;
    if (D.free_idx[kd] < 0) continue;  // fixed in dst: already the src pose
    const double wo = (double)S.cam_nobs[ks], wn = (double)D.cam_nobs[kd];
    if (!(wo + wn > 0.0)) continue;
    const double t = wn / (wo + wn);
    const double* Ro = S.R + ((size_t)scur * S.n_cams + ks) * 9;
    const double* To = S.T + ((size_t)scur * S.n_cams + ks) * 3;
    double* Rn = D.R + ((size_t)dcur * D.n_cams + kd) * 9;
    double* Tn = D.T + ((size_t)dcur * D.n_cams + kd) * 3;
    double E[9], phi[3], Q[9], Rm[9];
    for (int a = 0; a < 3; ++a)  // E = Ro^T Rn
      for (int b = 0; b < 3; ++b) E[3 * a + b] = Ro[a] * Rn[b] + Ro[3 + a] * Rn[3 + b] + Ro[6 + a] * Rn[6 + b];
    so3_log(E, phi);
    for (int a = 0; a < 3; ++a) phi[a] *= t;
    so3_exp(phi, Q);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) Rm[3 * a + b] = Ro[3 * a] * Q[b] + Ro[3 * a + 1] * Q[3 + b] + Ro[3 * a + 2] * Q[6 + b];
    for (int a = 0; a < 9; ++a) Rn[a] = Rm[a];
    for (int a = 0; a < 3; ++a) Tn[a] = (wo * To[a] + wn * Tn[a]) / (wo + wn);
  }
}

__global__ void k_warm_copy(const DevCluster* dst, const DevCluster* src, const int2* cams, int n_cams,
                            const int2* pts, int n_pts) {
  const int scur = src->lm->cur;
  const int stride = gridDim.x * blockDim.x;
  if (blockIdx.x == 0 && threadIdx.x == 0) {  // the damping state goes with the poses and points
    LmState* dl = dst->lm;
    const LmState* sl = src->lm;
    dl->mu = dl->mu0 = sl->mu;
    dl->mu_f = (float)sl->mu;
    dl->nu = dl->nu0 = sl->nu;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pts; i += stride) {
    const int2 p = pts[i];
    const double* sx = src->X + ((size_t)scur * src->n_pts + p.y) * 3;
    for (int a = 0; a < 3; ++a) {
      const double v = sx[a];
      dst->X[(size_t)p.x * 3 + a] = v;
      dst->X[((size_t)dst->n_pts + p.x) * 3 + a] = v;
      const_cast<double*>(dst->X_init)[(size_t)p.x * 3 + a] = v;
    }
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_cams; i += stride) {
    const int2 p = cams[i];
    const double* sr = src->R + ((size_t)scur * src->n_cams + p.y) * 9;
    const double* st = src->T + ((size_t)scur * src->n_cams + p.y) * 3;
    for (int b = 0; b < 2; ++b) {
      for (int a = 0; a < 9; ++a) dst->R[((size_t)b * dst->n_cams + p.x) * 9 + a] = sr[a];
      for (int a = 0; a < 3; ++a) dst->T[((size_t)b * dst->n_cams + p.x) * 3 + a] = st[a];
    }
    for (int a = 0; a < 9; ++a) const_cast<double*>(dst->R_init)[(size_t)p.x * 9 + a] = sr[a];
    for (int a = 0; a < 3; ++a) const_cast<double*>(dst->T_init)[(size_t)p.x * 3 + a] = st[a];
  }
}

// Restore the state given at create into both state buffers and reset LM
// control.  The copy is representation-agnostic (8-byte words).
__global__ void k_reset(BatchView bv) {
  for (int s = blockIdx.y; s < bv.n; s += gridDim.y) {
    const DevCluster& C = bv.cl[s];
    const size_t nr = (size_t)C.n_cams * 9, nt = (size_t)C.n_cams * 3, nx = (size_t)C.n_pts * 3;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nx; i += (size_t)gridDim.x * blockDim.x) {
      const double v = C.X_init[i];
      C.X[i] = v;
      C.X[nx + i] = v;
    }
    if (blockIdx.x == 0) {
      for (size_t i = threadIdx.x; i < nr; i += blockDim.x) { C.R[i] = C.R_init[i]; C.R[nr + i] = C.R_init[i]; }
      for (size_t i = threadIdx.x; i < nt; i += blockDim.x) { C.T[i] = C.T_init[i]; C.T[nt + i] = C.T_init[i]; }
      if (threadIdx.x == 0) {
        LmState* lm = C.lm;
        lm->mu = lm->mu0;
        lm->mu_f = (float)lm->mu0;
        lm->nu = lm->nu0;
        lm->F = 0.0;
        lm->F_new = 0.0;
        lm->cur = 0;
        lm->status = 0;
        lm->iter = 0;
        lm->n_accepted = 0;
        lm->active = 0;
        lm->iters_target = 0;
        lm->pt_fail = 0;
        lm->dev_error = 0;
      }
    }
  }
}

// Copy LM control and the last `iters` trace records of every cluster into
// contiguous buffers ([n] and [n][iters]).
__global__ void k_gather(BatchView bv, int iters, LmState* lm_out, StepRec* trace_out) {
  for (int s = blockIdx.x; s < bv.n; s += gridDim.x) {
    const DevCluster& C = bv.cl[s];
    if (threadIdx.x == 0 && lm_out) lm_out[s] = *C.lm;
    if (trace_out && C.trace_cap > 0) {
      const int end = C.lm->iter;
      for (int i = threadIdx.x; i < iters; i += blockDim.x) {
        const int it = end - iters + i;
        if (it >= 0) trace_out[(size_t)s * iters + i] = C.trace[it % C.trace_cap];
      }
    }
  }
}

// ------------------------------------------------------------------ launchers
//
// Every launch goes through LAUNCH(kind, ...): it counts the launch (as a
// direct launch, or as a kernel node when the stream is being captured) and,
// when a probe is attached to the calling thread, brackets the kernel with
// CUDA events (captured as event-record nodes inside graphs).

static thread_local Probe* t_probe = nullptr;
static thread_local unsigned long long t_direct = 0, t_captured = 0;

void set_probe(Probe* p) { t_probe = p; }
unsigned long long take_direct_launches() {
  const unsigned long long v = t_direct;
  t_direct = 0;
  return v;
}
unsigned long long take_captured_launches() {
  const unsigned long long v = t_captured;
  t_captured = 0;
  return v;
}

static bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  return cs == cudaStreamCaptureStatusActive;
}

static void probe_mark(cudaStream_t st, cudaEvent_t* out) {
  cudaEventCreate(out);
  if (capturing(st)) cudaEventRecordWithFlags(*out, st, cudaEventRecordExternal);
  else cudaEventRecord(*out, st);
}

LaunchScope::LaunchScope(int k, cudaStream_t s) : kind(k), st(s) {
  if (t_probe) probe_mark(st, &e0);
}

LaunchScope::~LaunchScope() {
  if (capturing(st)) ++t_captured; else ++t_direct;
  if (t_probe) {
    cudaEvent_t e1;
    probe_mark(st, &e1);
    t_probe->recs.push_back(ProbeRec{kind, e0, e1});
  }
}

static int grid_for(int items, int per_block, int cap) {
  int g = (items + per_block - 1) / per_block;
  if (g > cap) g = cap;
  return g < 1 ? 1 : g;
}

static int g_num_sms = 0;
int num_sms() {
  if (!g_num_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

void launch_arm(const BatchView& bv, int iters, cudaStream_t st) {
  LAUNCH(KK_OTHER, st, k_arm<<<(bv.n + 127) / 128, 128, 0, st>>>(bv, iters));
}

void launch_arm_slots(const BatchView& bv, const int* arm, const double* ftol, cudaStream_t st) {
  LAUNCH(KK_OTHER, st, k_arm_slots<<<(bv.n + 127) / 128, 128, 0, st>>>(bv, arm, ftol));
}

void launch_warm_copy(const DevCluster* dst, const DevCluster* src, const int2* cams, int n_cams, const int2* pts,
                      int n_pts, cudaStream_t st) {
  const int n = n_pts > n_cams ? n_pts : n_cams;
  LAUNCH(KK_OTHER, st,
         k_warm_copy<<<grid_for(n, 256, num_sms() * 4), 256, 0, st>>>(dst, src, cams, n_cams, pts, n_pts));
}

void launch_transition(const DevCluster* dst, const DevCluster* src, const int2* pairs, int n, cudaStream_t st) {
  LAUNCH(KK_OTHER, st, k_transition<<<grid_for(n, 128, 1024), 128, 0, st>>>(dst, src, pairs, n));
}

void launch_camreal(const BatchView& bv, bool mixed, cudaStream_t st) {
  if (mixed) LAUNCH(KK_OTHER, st, k_camdf_all<<<grid_for(bv.n, 1, 65535), 64, 0, st>>>(bv));
  else LAUNCH(KK_OTHER, st, k_camreal<<<grid_for(bv.n, 1, 65535), 64, 0, st>>>(bv));
}

void launch_reset(const BatchView& bv, bool mixed, cudaStream_t st) {
  dim3 grid(64, bv.n < 65535 ? bv.n : 65535);
  LAUNCH(KK_OTHER, st, k_reset<<<grid, 256, 0, st>>>(bv));
  launch_camreal(bv, mixed, st);
}

void launch_gather(const BatchView& bv, int iters, LmState* lm_out, StepRec* trace_out, cudaStream_t st) {
  LAUNCH(KK_OTHER, st, k_gather<<<bv.n < 65535 ? bv.n : 65535, 128, 0, st>>>(bv, iters, lm_out, trace_out));
}

template <bool MIXED>
static void launch_cost_init_t(const BatchView& bv, cudaStream_t st) {
  const int sms = num_sms();
  LAUNCH(KK_COST_TILES, st, k_cost_tiles<MIXED><<<grid_for(bv.total_tiles, 8, sms * 16), 256, 0, st>>>(bv));
  LAUNCH(KK_COST_INIT, st, k_cost_init<<<grid_for(bv.n, 1, 65535), kCostInitThreads, 0, st>>>(bv));
}

void launch_cost_init(const BatchView& bv, bool mixed, cudaStream_t st) {
  if (mixed) launch_cost_init_t<true>(bv, st);
  else launch_cost_init_t<false>(bv, st);
}

int chunk_obs(bool mixed) { return mixed ? kChunkObsMixed : kChunkObsF64; }
int chunk_tiles(bool mixed) { return mixed ? kChunkTilesMixed : kChunkTilesF64; }

static size_t chunk_smem_bytes(bool mixed) {
  // records (later overlaid by the lane partials); mixed path: the chunk
  // staging, its barrier, a flag and the failure-injection barrier
  return chunk_records_bytes(mixed) + (mixed ? (size_t)kStageBytes + 24 : 0);
}

template <bool MIXED>
static void launch_lin_schur(const BatchView& bv, int diag, cudaStream_t st) {
  LAUNCH(KK_LIN_SCHUR, st,
         k_lin_schur<MIXED><<<grid_for(bv.total_chunks, 1, num_sms() * bv.lin_ctas_per_sm), kChunkThreads,
                              chunk_smem_bytes(MIXED),
                              st>>>(bv, diag));
}


template <bool MIXED>
static void launch_partial_reduce(const BatchView& bv, cudaStream_t st) {
  using Real = typename RealOf<MIXED>::T;
  LAUNCH(KK_PARTIAL_REDUCE, st, k_partial_reduce<Real><<<grid_for(bv.total_items, 8, num_sms() * 16), 256, 0, st>>>(bv));
}

template <bool MIXED>
static void launch_iteration_t(const BatchView& bv, int refine_steps, cudaStream_t st, const std::vector<BigRef>* big) {
  const int sms = num_sms();
  launch_lin_schur<MIXED>(bv, 0, st);
  launch_partial_reduce<MIXED>(bv, st);
  const size_t smem = factor_smem_bytes(bv.max_n);
  LAUNCH(KK_FACTOR, st,
         k_factor_solve<MIXED><<<grid_for(bv.n, 1, 65535), bv.factor_threads, smem, st>>>(bv, refine_steps, 0));
  if (big)
    for (const BigRef& b : *big) launch_big_solve(b, MIXED, refine_steps, 0, st);
  LAUNCH(KK_BACKSUB, st, k_backsub_cost<MIXED><<<grid_for(bv.total_tiles, 8, sms * bv.back_ctas_per_sm), 256, 0, st>>>(bv));
}

void launch_iteration(const BatchView& bv, bool mixed, int refine_steps, cudaStream_t st,
                      const std::vector<BigRef>* big) {
  if (mixed) launch_iteration_t<true>(bv, refine_steps, st, big);
  else launch_iteration_t<false>(bv, refine_steps, st, big);
}

template <bool MIXED>
static void launch_grad_norm_t(const BatchView& bv, double* out, cudaStream_t st, const std::vector<BigRef>* big) {
  launch_lin_schur<MIXED>(bv, 1, st);
  launch_partial_reduce<MIXED>(bv, st);
  LAUNCH(KK_FACTOR, st,
         k_factor_solve<MIXED><<<grid_for(bv.n, 1, 65535), bv.factor_threads, factor_smem_bytes(bv.max_n), st>>>(bv, 0, 1));
  if (big)
    for (const BigRef& b : *big) launch_big_solve(b, MIXED, 0, 1, st);
  LAUNCH(KK_OTHER, st, k_grad_norm<<<grid_for(bv.n, 1, 65535), 256, 0, st>>>(bv, out));
}

void launch_grad_norm(const BatchView& bv, bool mixed, double* out, cudaStream_t st, const std::vector<BigRef>* big) {
  if (mixed) launch_grad_norm_t<true>(bv, out, st, big);
  else launch_grad_norm_t<false>(bv, out, st, big);
}

void launch_reproj(const DevCluster* dcl, const DevCluster& hcl, bool mixed, double* err_pm, cudaStream_t st) {
  LAUNCH(KK_OTHER, st, k_reproj<<<grid_for(hcl.n_obs, 256, num_sms() * 8), 256, 0, st>>>(dcl, mixed, err_pm));
}

void launch_export_state(const DevCluster* dcl, const DevCluster& hcl, bool mixed, double* R, double* T, double* X,
                         cudaStream_t st) {
  const int items = hcl.n_pts > 12 * hcl.n_cams ? hcl.n_pts : 12 * hcl.n_cams;
  LAUNCH(KK_OTHER, st, k_export_state<<<grid_for(items, 256, num_sms() * 8), 256, 0, st>>>(dcl, mixed, R, T, X));
}

// binary32 FMA-rate probe: 16 independent chains per thread (enough to
// cover the pipe's latency), the result stored only if it comes out as an
// impossible value so that nothing is optimised away
__global__ void __launch_bounds__(512) k_fma_probe(int iters, float seed, float* sink) {
  float a[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i] = seed + (float)(threadIdx.x + i);
  const float m = 0.999999f, c = 1e-7f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = __fmaf_rn(a[i], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 16; ++i) s += a[i];
  if (s == -1.0f) *sink = s;
}

void launch_fma_probe(int ctas, int iters, float* sink, cudaStream_t st) {
  LAUNCH(KK_OTHER, st, k_fma_probe<<<ctas, 512, 0, st>>>(iters, 1.0f, sink));
}

cudaError_t set_kernel_attributes(int max_n) {
  const size_t smem = factor_smem_bytes(max_n);
  cudaError_t e = cudaFuncSetAttribute(k_factor_solve<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_factor_solve<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_lin_schur<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)chunk_smem_bytes(true));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_lin_schur<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)chunk_smem_bytes(false));
}

}  // namespace bagpu
