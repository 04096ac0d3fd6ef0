// Kernels of one LM iteration, batched over many clusters.
//
//   k_linearize     per observation (warp per tile of whole points): residual,
//                   Jacobians, point blocks V = sum Jp^T Jp, g_p = -sum Jp^T r
//                   by deterministic segmented warp reductions, the damped
//                   point block V* = V + mu Dp, its Cholesky factor L and
//                   Linv = L^-1, q = Linv g_p, and Z = W Linv^T = Jc^T (Jp Linv^T),
//                   so that W V*^-1 W^T = Z Z^T and W V*^-1 g_p = Z q.
//   k_cam_reduce    camera-major chunks: sum (Jc^T Jc - Z Z^T), -Jc^T r, Z q,
//                   diag(Jc^T Jc) of every observation of a free camera.
//   k_pair_reduce   camera-pair chunks: sum Z_a Z_b^T over co-visible points.
//   k_factor_solve  per cluster (FP64): assemble S = U* - W V*^-1 W^T and
//                   rhs = g_c - W V*^-1 g_p with priors and damping, Cholesky,
//                   solve, iterative refinement, candidate camera poses.
//   k_backsub_cost  per observation: dX = Linv^T (q - sum_k Z_k^T dc_k),
//                   candidate points, cost at the candidate, pred terms.
//   k_lm_update     per cluster: gain ratio, accept/reject, Nielsen update.
//
// Precision.  MIXED = false: every step in binary64.  MIXED = true: the
// per-observation linearisation, the Schur reductions and the back-
// substitution run in binary32; the state (points and cameras) is held in
// double-float, and the cost F(x) that decides the gain ratio is evaluated
// per observation in double-float and summed in binary64; the reduced
// camera system is assembled, factored and refined in binary64.
//
// Every sum runs in an order fixed by the cluster's presorted tables; there
// are no atomics.
#include <cuda_runtime.h>
#include <stdio.h>

#include "ba_device.cuh"
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

__device__ __forceinline__ CamDf load_camdf(const float* p) {
  CamDf c;
  float v[kCamDf];
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int i = 0; i < kCamDf / 4; ++i) {
    const float4 w = q[i];
    v[4 * i] = w.x; v[4 * i + 1] = w.y; v[4 * i + 2] = w.z; v[4 * i + 3] = w.w;
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) c.R[i] = dfl{v[2 * i], v[2 * i + 1]};
#pragma unroll
  for (int i = 0; i < 3; ++i) c.T[i] = dfl{v[18 + 2 * i], v[19 + 2 * i]};
  c.f = dfl{v[24], v[25]};
  c.k1 = dfl{v[26], v[27]};
  c.k2 = dfl{v[28], v[29]};
  c.p1 = dfl{v[30], v[31]};
  c.p2 = dfl{v[32], v[33]};
  c.free_flag = v[34];
  return c;
}

__device__ __forceinline__ const float* camdf_ptr(const DevCluster& C, int buf, int k) {
  return C.camdf + ((size_t)buf * C.n_cams + k) * kCamDf;
}

// Eq. 5 with Brown distortion in double-float: residual (u - cx, v - cy) - c
// for a double-float point, every term in double-float.
__device__ __forceinline__ bool df_residual(const CamDf& c, dfl X0, dfl X1, dfl X2, dfl c0, dfl c1, dfl& e0,
                                            dfl& e1) {
  const dfl d0 = df_sub(X0, c.T[0]), d1 = df_sub(X1, c.T[1]), d2 = df_sub(X2, c.T[2]);
  const dfl z = df_add(df_add(df_mul(c.R[2], d0), df_mul(c.R[5], d1)), df_mul(c.R[8], d2));
  if (!(z.hi > (float)kMinDepth)) return false;
  const dfl x = df_add(df_add(df_mul(c.R[0], d0), df_mul(c.R[3], d1)), df_mul(c.R[6], d2));
  const dfl y = df_add(df_add(df_mul(c.R[1], d0), df_mul(c.R[4], d1)), df_mul(c.R[7], d2));
  const dfl xn = df_div(x, z), yn = df_div(y, z);
  const dfl xx = df_mul(xn, xn), yy = df_mul(yn, yn), xy2 = df_mul_f(df_mul(xn, yn), 2.0f);
  const dfl r2 = df_add(xx, yy);
  const dfl radm1 = df_mul(r2, df_add(c.k1, df_mul(c.k2, r2)));  // rad - 1
  const dfl ddx = df_add(df_add(df_mul(xn, radm1), df_mul(c.p1, xy2)), df_mul(c.p2, df_add(r2, df_mul_f(xx, 2.0f))));
  const dfl ddy = df_add(df_add(df_mul(yn, radm1), df_mul(c.p1, df_add(r2, df_mul_f(yy, 2.0f)))), df_mul(c.p2, xy2));
  e0 = df_sub(df_mul(c.f, df_add(xn, ddx)), c0);
  e1 = df_sub(df_mul(c.f, df_add(yn, ddy)), c1);
  return true;
}

// 1/2 rho(s) / sigma^2 in double-float, s = e0^2 + e1^2 (Eq. 6: rho on the squared norm)
__device__ __forceinline__ dfl df_robust_cost(dfl e0, dfl e1, float delta, float half_inv_s2) {
  const dfl s = df_add(df_mul(e0, e0), df_mul(e1, e1));
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

// mixed path: double-float record of camera k from (R, T) in binary64
__device__ void write_camdf(const DevCluster& C, int buf, int k, const double* R, const double* T) {
  float* o = C.camdf + ((size_t)buf * C.n_cams + k) * kCamDf;
  for (int i = 0; i < 9; ++i) {
    const dfl v = df_from_d(R[i]);
    o[2 * i] = v.hi;
    o[2 * i + 1] = v.lo;
  }
  for (int i = 0; i < 3; ++i) {
    const dfl v = df_from_d(T[i]);
    o[18 + 2 * i] = v.hi;
    o[19 + 2 * i] = v.lo;
  }
  const dfl f = df_from_d(C.intr[7 * k]);
  o[24] = f.hi;
  o[25] = f.lo;
  for (int i = 0; i < 4; ++i) {
    const dfl v = df_from_d(C.intr[7 * k + 3 + i]);
    o[26 + 2 * i] = v.hi;
    o[27 + 2 * i] = v.lo;
  }
  o[34] = C.free_idx[k] >= 0 ? 1.0f : 0.0f;
  for (int i = 35; i < kCamDf; ++i) o[i] = 0.0f;
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

// ------------------------------------------------------------------ K1

template <bool MIXED>
__global__ void __launch_bounds__(256) k_linearize(BatchView bv) {
  using Real = typename RealOf<MIXED>::T;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int g = warp; g < bv.total_tiles; g += nwarps) {
    const int s = find_slot(bv.tile_pre, bv.n, g);
    const DevCluster& C = bv.cl[s];
    LmState* lm = C.lm;
    if (!lm->active) continue;
    const Tile tl = C.tiles[g - bv.tile_pre[s]];
    const bool act = lane < tl.n_obs;
    const int o = tl.obs_begin + (act ? lane : 0);
    const int k = act ? C.obs_cam[o] : 0;
    const int j = act ? C.obs_pt[o] : -1 - lane;
    int seg_start, seg_end;
    segments(j, lane, seg_start, seg_end);
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

    Real r0 = 0, r1 = 0, Jc[12], Jp[6];
#pragma unroll
    for (int i = 0; i < 12; ++i) Jc[i] = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) Jp[i] = 0;
    if (act) {
      Real Rm[9], in[7], dx, dy, dz, uo, vo;
      bool is_free;
      if constexpr (MIXED) {
        const CamDf cd = load_camdf(camdf_ptr(C, cur, k));
        const float2* xp = xdf_ptr(C, cur, j);
        const float2 a = xp[0], b = xp[1], c = xp[2];
        dx = df_to_f(df_sub(dfl{a.x, a.y}, cd.T[0]));
        dy = df_to_f(df_sub(dfl{b.x, b.y}, cd.T[1]));
        dz = df_to_f(df_sub(dfl{c.x, c.y}, cd.T[2]));
#pragma unroll
        for (int i = 0; i < 9; ++i) Rm[i] = cd.R[i].hi;
        in[0] = cd.f.hi; in[1] = 0.f; in[2] = 0.f;
        in[3] = cd.k1.hi; in[4] = cd.k2.hi; in[5] = cd.p1.hi; in[6] = cd.p2.hi;
        const float2 ch = C.obs_chi[o];  // observation relative to the principal point
        uo = ch.x; vo = ch.y;
        is_free = cd.free_flag != 0.0f;
      } else {
        const double* cr = (const double*)C.camreal + (size_t)kCamReal * k;
#pragma unroll
        for (int i = 0; i < 9; ++i) Rm[i] = cr[i];
#pragma unroll
        for (int i = 0; i < 7; ++i) in[i] = cr[12 + i];
        const double* Xd = C.X + ((size_t)cur * C.n_pts + j) * 3;
        dx = Xd[0] - cr[9]; dy = Xd[1] - cr[10]; dz = Xd[2] - cr[11];
        const double2 u = reinterpret_cast<const double2*>(C.obs_uv)[o];
        uo = u.x; vo = u.y;
        is_free = cr[19] != 0.0;
      }
      obs_linearize<Real>(Rm, dx, dy, dz, in, uo, vo, inv_sigma, delta, r0, r1, Jc, Jp);
      if (!is_free) {
#pragma unroll
        for (int i = 0; i < 12; ++i) Jc[i] = 0;
      }
    }
    // point blocks by segmented reduction
    Real v00 = Jp[0] * Jp[0] + Jp[3] * Jp[3];
    Real v01 = Jp[0] * Jp[1] + Jp[3] * Jp[4];
    Real v02 = Jp[0] * Jp[2] + Jp[3] * Jp[5];
    Real v11 = Jp[1] * Jp[1] + Jp[4] * Jp[4];
    Real v12 = Jp[1] * Jp[2] + Jp[4] * Jp[5];
    Real v22 = Jp[2] * Jp[2] + Jp[5] * Jp[5];
    Real g0 = -(Jp[0] * r0 + Jp[3] * r1);
    Real g1 = -(Jp[1] * r0 + Jp[4] * r1);
    Real g2 = -(Jp[2] * r0 + Jp[5] * r1);
    v00 = seg_reduce(v00, lane, seg_start, seg_end);
    v01 = seg_reduce(v01, lane, seg_start, seg_end);
    v02 = seg_reduce(v02, lane, seg_start, seg_end);
    v11 = seg_reduce(v11, lane, seg_start, seg_end);
    v12 = seg_reduce(v12, lane, seg_start, seg_end);
    v22 = seg_reduce(v22, lane, seg_start, seg_end);
    g0 = seg_reduce(g0, lane, seg_start, seg_end);
    g1 = seg_reduce(g1, lane, seg_start, seg_end);
    g2 = seg_reduce(g2, lane, seg_start, seg_end);

    // head: damp, factor V* = L L^T, M = L^-1, q = M g_p
    Real m00 = 0, m10 = 0, m11 = 0, m20 = 0, m21 = 0, m22 = 0;
    if (act && lane == seg_start) {
      const Real d0 = clamp_diag(v00), d1 = clamp_diag(v11), d2 = clamp_diag(v22);
      const Real a00 = v00 + mu * d0, a11 = v11 + mu * d1, a22 = v22 + mu * d2;
      bool ok = a00 > Real(0);
      const Real l00 = sqrt(ok ? a00 : Real(1));
      const Real l10 = v01 / l00, l20 = v02 / l00;
      const Real t11 = a11 - l10 * l10;
      ok = ok && t11 > Real(0);
      const Real l11 = sqrt(t11 > Real(0) ? t11 : Real(1));
      const Real l21 = (v12 - l20 * l10) / l11;
      const Real t22 = a22 - l20 * l20 - l21 * l21;
      ok = ok && t22 > Real(0);
      const Real l22 = sqrt(t22 > Real(0) ? t22 : Real(1));
      if (!ok) lm->pt_fail = 1;  // point block not positive definite: reject this step
      m00 = Real(1) / l00;
      m11 = Real(1) / l11;
      m22 = Real(1) / l22;
      m10 = -l10 * m00 * m11;
      m21 = -l21 * m11 * m22;
      m20 = -(l20 * m00 + l21 * m10) * m22;
      const Real q0 = m00 * g0;
      const Real q1 = m10 * g0 + m11 * g1;
      const Real q2 = m20 * g0 + m21 * g1 + m22 * g2;
      Real* pa = (Real*)C.paux + (size_t)kPaux * j;
      pa[0] = m00; pa[1] = m10; pa[2] = m11; pa[3] = m20; pa[4] = m21; pa[5] = m22;
      pa[6] = q0; pa[7] = q1; pa[8] = q2;
      pa[9] = d0; pa[10] = d1; pa[11] = d2;
      pa[12] = g0; pa[13] = g1; pa[14] = g2;
      pa[15] = 0;
    }
    m00 = __shfl_sync(BA_FULL_MASK, m00, seg_start);
    m10 = __shfl_sync(BA_FULL_MASK, m10, seg_start);
    m11 = __shfl_sync(BA_FULL_MASK, m11, seg_start);
    m20 = __shfl_sync(BA_FULL_MASK, m20, seg_start);
    m21 = __shfl_sync(BA_FULL_MASK, m21, seg_start);
    m22 = __shfl_sync(BA_FULL_MASK, m22, seg_start);
    if (!act) continue;
    // P = Jp M^T (2x3), Z = Jc^T P (6x3)
    const Real P00 = Jp[0] * m00;
    const Real P01 = Jp[0] * m10 + Jp[1] * m11;
    const Real P02 = Jp[0] * m20 + Jp[1] * m21 + Jp[2] * m22;
    const Real P10 = Jp[3] * m00;
    const Real P11 = Jp[3] * m10 + Jp[4] * m11;
    const Real P12 = Jp[3] * m20 + Jp[4] * m21 + Jp[5] * m22;
    Real rec[kRec];
#pragma unroll
    for (int i = 0; i < 12; ++i) rec[kRecJc + i] = Jc[i];
    rec[kRecR] = r0;
    rec[kRecR + 1] = r1;
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      rec[kRecZ + 3 * m + 0] = Jc[m] * P00 + Jc[6 + m] * P10;
      rec[kRecZ + 3 * m + 1] = Jc[m] * P01 + Jc[6 + m] * P11;
      rec[kRecZ + 3 * m + 2] = Jc[m] * P02 + Jc[6 + m] * P12;
    }
    using V2 = typename Vec2<Real>::T;
    V2* dst = reinterpret_cast<V2*>((Real*)C.rec + (size_t)kRec * o);
#pragma unroll
    for (int i = 0; i < kRec / 2; ++i) {
      V2 v;
      v.x = rec[2 * i];
      v.y = rec[2 * i + 1];
      dst[i] = v;
    }
  }
}

// ------------------------------------------------------------------ K2

template <typename Real>
__global__ void __launch_bounds__(128) k_cam_reduce(BatchView bv) {
  __shared__ Real red[4][40];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int g = blockIdx.x; g < bv.total_cchunks; g += gridDim.x) {
    const int s = find_slot(bv.cchunk_pre, bv.n, g);
    const DevCluster& C = bv.cl[s];
    if (!C.lm->active) continue;
    const int local = g - bv.cchunk_pre[s];
    const ChunkItem it = C.cchunks[local];
    Real acc[39];
#pragma unroll
    for (int i = 0; i < 39; ++i) acc[i] = 0;
    using V2 = typename Vec2<Real>::T;
    for (int e = threadIdx.x; e < it.count; e += blockDim.x) {
      const int o = C.cam_obs[it.begin + e];
      const V2* rp = reinterpret_cast<const V2*>((const Real*)C.rec + (size_t)kRec * o);
      Real rc[kRec];
#pragma unroll
      for (int i = 0; i < kRec / 2; ++i) {
        const V2 v = rp[i];
        rc[2 * i] = v.x;
        rc[2 * i + 1] = v.y;
      }
      const Real* pa = (const Real*)C.paux + (size_t)kPaux * C.obs_pt[o];
      const Real q0 = pa[6], q1 = pa[7], q2 = pa[8];
      const Real* Jc = rc + kRecJc;
      const Real* Z = rc + kRecZ;
      const Real r0 = rc[kRecR], r1 = rc[kRecR + 1];
      int t = 0;
#pragma unroll
      for (int a = 0; a < 6; ++a) {
#pragma unroll
        for (int b = a; b < 6; ++b) {
          acc[t++] += Jc[a] * Jc[b] + Jc[6 + a] * Jc[6 + b] -
                      (Z[3 * a] * Z[3 * b] + Z[3 * a + 1] * Z[3 * b + 1] + Z[3 * a + 2] * Z[3 * b + 2]);
        }
      }
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        acc[21 + a] -= Jc[a] * r0 + Jc[6 + a] * r1;
        acc[27 + a] += Z[3 * a] * q0 + Z[3 * a + 1] * q1 + Z[3 * a + 2] * q2;
        acc[33 + a] += Jc[a] * Jc[a] + Jc[6 + a] * Jc[6 + a];
      }
    }
#pragma unroll
    for (int i = 0; i < 39; ++i) {
      const Real v = warp_sum(acc[i]);
      if (lane == 0) red[wid][i] = v;
    }
    __syncthreads();
    if (threadIdx.x < 39) {
      const int i = threadIdx.x;
      const Real v = (red[0][i] + red[1][i]) + (red[2][i] + red[3][i]);
      ((Real*)C.campart)[(size_t)kCamPart * local + i] = v;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ K3

template <typename Real>
__global__ void __launch_bounds__(256) k_pair_reduce(BatchView bv) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  using V2 = typename Vec2<Real>::T;
  for (int g = warp; g < bv.total_pchunks; g += nwarps) {
    const int s = find_slot(bv.pchunk_pre, bv.n, g);
    const DevCluster& C = bv.cl[s];
    if (!C.lm->active) continue;
    const int local = g - bv.pchunk_pre[s];
    const ChunkItem it = C.pchunks[local];
    Real acc[36];
#pragma unroll
    for (int i = 0; i < 36; ++i) acc[i] = 0;
    for (int e = lane; e < it.count; e += 32) {
      const int2 ab = C.pair_ent[it.begin + e];
      const V2* pa = reinterpret_cast<const V2*>((const Real*)C.rec + (size_t)kRec * ab.x + kRecZ);
      const V2* pb = reinterpret_cast<const V2*>((const Real*)C.rec + (size_t)kRec * ab.y + kRecZ);
      Real Za[18], Zb[18];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const V2 x = pa[i], y = pb[i];
        Za[2 * i] = x.x; Za[2 * i + 1] = x.y;
        Zb[2 * i] = y.x; Zb[2 * i + 1] = y.y;
      }
#pragma unroll
      for (int a = 0; a < 6; ++a)
#pragma unroll
        for (int b = 0; b < 6; ++b)
          acc[6 * a + b] += Za[3 * a] * Zb[3 * b] + Za[3 * a + 1] * Zb[3 * b + 1] + Za[3 * a + 2] * Zb[3 * b + 2];
    }
#pragma unroll
    for (int i = 0; i < 36; ++i) {
      const Real v = warp_sum(acc[i]);
      if (lane == 0) ((Real*)C.pairpart)[(size_t)kPairPart * local + i] = v;
    }
  }
}

// ------------------------------------------------------------------ K4 (FP64)

__device__ __forceinline__ int pk(int i, int j) { return (i * (i + 1)) / 2 + j; }  // packed lower, j <= i

size_t factor_smem_bytes(int max_n) {
  const int nf = max_n / 6;
  const size_t doubles = (size_t)max_n * (max_n + 1) / 2 + (size_t)nf * 40 + (size_t)nf * 42 + 3 * (size_t)max_n + 64;
  return doubles * sizeof(double);
}

// Solve L L^T x = b in place (b in shared memory), one warp.
__device__ void chol_solve_warp(const double* A, double* b, int n, int lane) {
  for (int j = 0; j < n; ++j) {
    const double yj = b[j] / A[pk(j, j)];
    __syncwarp();
    if (lane == 0) b[j] = yj;
    for (int i = j + 1 + lane; i < n; i += 32) b[i] -= A[pk(i, j)] * yj;
    __syncwarp();
  }
  for (int j = n - 1; j >= 0; --j) {
    const double xj = b[j] / A[pk(j, j)];
    __syncwarp();
    if (lane == 0) b[j] = xj;
    for (int i = lane; i < j; i += 32) b[i] -= A[pk(j, i)] * xj;
    __syncwarp();
  }
}

template <bool MIXED>
__global__ void __launch_bounds__(512) k_factor_solve(BatchView bv, int refine_steps, int assemble_only) {
  using Real = typename RealOf<MIXED>::T;
  extern __shared__ double sm[];
  __shared__ int fail;
  const int tid = threadIdx.x, bs = blockDim.x;
  for (int s = blockIdx.x; s < bv.n; s += gridDim.x) {
    const DevCluster& C = bv.cl[s];
    LmState* lm = C.lm;
    if (!lm->active && !assemble_only) continue;
    const int nf = C.n_free, n = 6 * nf, nc = C.n_cams;
    const double mu = lm->mu;
    const int cur = lm->cur;
    double* A = sm;
    double* cd = A + (size_t)n * (n + 1) / 2;  // [nf][40]
    double* pr = cd + (size_t)nf * 40;         // [nf][42]: JtJ 36, Jtr 6
    double* x = pr + (size_t)nf * 42;          // [n]
    double* b = x + n;                         // [n]
    double* t = b + n;                         // [n]
    const double* Rc = C.R + (size_t)cur * nc * 9;
    const double* Tc = C.T + (size_t)cur * nc * 3;

    // camera chunk partials, summed in chunk order
    for (int idx = tid; idx < nf * 39; idx += bs) {
      const int f = idx / 39, e = idx - 39 * f;
      double v = 0.0;
      for (int p = C.cam_part_begin[f]; p < C.cam_part_begin[f + 1]; ++p)
        v += (double)((const Real*)C.campart)[(size_t)kCamPart * p + e];
      cd[40 * f + e] = v;
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
      A[pk(6 * f + bb, 6 * f + a)] = v;  // row bb >= col a
    }
    for (int idx = tid; idx < n; idx += bs) {
      const int f = idx / 6, a = idx - 6 * f;
      const double g = cd[40 * f + 21 + a] - pr[42 * f + 36 + a];
      C.gc[idx] = g;
      const double r = g - cd[40 * f + 27 + a];
      C.rhs[idx] = r;
      b[idx] = r;
    }
    // off-diagonal blocks: S(fb, fa) = -(sum Z_a Z_b^T)^T
    for (int idx = tid; idx < C.n_pairs * 36; idx += bs) {
      const int p = idx / 36, e = idx - 36 * p;
      const int i = e / 6, c = e - 6 * i;
      double v = 0.0;
      for (int q = C.pair_part_begin[p]; q < C.pair_part_begin[p + 1]; ++q)
        v += (double)((const Real*)C.pairpart)[(size_t)kPairPart * q + e];
      const int2 key = C.pair_key[p];
      A[pk(6 * key.y + c, 6 * key.x + i)] = -v;
    }
    __syncthreads();
    for (int idx = tid; idx < n * n; idx += bs) {
      const int r = idx / n, c = idx - n * r;
      C.S[idx] = r >= c ? A[pk(r, c)] : A[pk(c, r)];
    }
    if (assemble_only) {
      __syncthreads();
      continue;
    }
    // right-looking Cholesky in shared memory
    for (int j = 0; j < n; ++j) {
      if (tid == 0) {
        const double d = A[pk(j, j)];
        if (!(d > 0.0)) fail = 1;
        A[pk(j, j)] = sqrt(d > 0.0 ? d : 1.0);
      }
      __syncthreads();
      if (fail) break;
      const double inv = 1.0 / A[pk(j, j)];
      for (int i = j + 1 + tid; i < n; i += bs) A[pk(i, j)] *= inv;
      __syncthreads();
      const int m = n - j - 1;
      const int total = m * (m + 1) / 2;
      for (int u = tid; u < total; u += bs) {
        int ii = (int)((sqrtf(8.0f * (float)u + 1.0f) - 1.0f) * 0.5f);
        while ((ii + 1) * (ii + 2) / 2 <= u) ++ii;
        while (ii * (ii + 1) / 2 > u) --ii;
        const int cc = u - ii * (ii + 1) / 2;
        const int row = j + 1 + ii, col = j + 1 + cc;
        A[pk(row, col)] -= A[pk(row, j)] * A[pk(col, j)];
      }
      __syncthreads();
    }
    __syncthreads();
    const int status = fail ? BA_STATUS_NOT_PD : 0;
    if (!fail) {
      if (tid < 32) chol_solve_warp(A, b, n, tid);
      __syncthreads();
      for (int idx = tid; idx < n; idx += bs) x[idx] = b[idx];
      __syncthreads();
      // iterative refinement against the FP64 system kept in global memory
      for (int it = 0; it < refine_steps; ++it) {
        const int lane = tid & 31, wid = tid >> 5, nw = bs >> 5;
        for (int r = wid; r < n; r += nw) {
          double acc = 0.0;
          for (int c = lane; c < n; c += 32) acc += C.S[(size_t)r * n + c] * x[c];
          acc = warp_sum(acc);
          if (lane == 0) t[r] = C.rhs[r] - acc;
        }
        __syncthreads();
        if (tid < 32) chol_solve_warp(A, t, n, tid);
        __syncthreads();
        for (int idx = tid; idx < n; idx += bs) x[idx] += t[idx];
        __syncthreads();
      }
      for (int idx = tid; idx < n; idx += bs) {
        C.dc[idx] = x[idx];
        if (MIXED) C.dc32[idx] = (float)x[idx];
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
    double* Rn = C.R + (size_t)(cur ^ 1) * nc * 9;
    double* Tn = C.T + (size_t)(cur ^ 1) * nc * 3;
    for (int k = tid; k < nc; k += bs) {
      const int f = C.free_idx[k];
      if (f < 0 || fail) {
        for (int i = 0; i < 9; ++i) Rn[9 * k + i] = Rc[9 * k + i];
        for (int i = 0; i < 3; ++i) Tn[3 * k + i] = Tc[3 * k + i];
        if (f >= 0) { t[2 * f] = 0.0; t[2 * f + 1] = 0.0; }
      } else {
        const double* d = x + 6 * f;
        double E[9];
        so3_exp(d, E);
        const double* R0 = Rc + 9 * k;
        for (int r = 0; r < 3; ++r)
          for (int c = 0; c < 3; ++c)
            Rn[9 * k + 3 * r + c] = R0[3 * r] * E[c] + R0[3 * r + 1] * E[3 + c] + R0[3 * r + 2] * E[6 + c];
        for (int i = 0; i < 3; ++i) Tn[3 * k + i] = Tc[3 * k + i] + d[3 + i];
        double pc = 0.0;
        for (int a = 0; a < 6; ++a) pc += d[a] * (mu * C.Dc[6 * f + a] * d[a] + C.gc[6 * f + a]);
        t[2 * f] = pc;
        t[2 * f + 1] = prior_terms(Rn + 9 * k, Tn + 3 * k, C.R_prior + 9 * k, C.T_prior + 3 * k, C.sigma_imu,
                                   C.sigma_gnss, nullptr, nullptr);
      }
      if constexpr (MIXED) write_camdf(C, cur ^ 1, k, Rn + 9 * k, Tn + 3 * k);
    }
    __syncthreads();
    if (tid == 0) {
      double pc = 0.0, pn = 0.0;
      for (int f = 0; f < nf; ++f) { pc += t[2 * f]; pn += t[2 * f + 1]; }
      lm->pred_cam = pc;
      lm->prior_new = pn;
      lm->status = status;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ K5

template <bool MIXED>
__global__ void __launch_bounds__(256) k_backsub_cost(BatchView bv) {
  using Real = typename RealOf<MIXED>::T;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  using V2 = typename Vec2<Real>::T;
  for (int g = warp; g < bv.total_tiles; g += nwarps) {
    const int s = find_slot(bv.tile_pre, bv.n, g);
    const DevCluster& C = bv.cl[s];
    const LmState* lm = C.lm;
    if (!lm->active || lm->status != 0) continue;
    const int local = g - bv.tile_pre[s];
    const Tile tl = C.tiles[local];
    const bool act = lane < tl.n_obs;
    const int o = tl.obs_begin + (act ? lane : 0);
    const int k = act ? C.obs_cam[o] : 0;
    const int j = act ? C.obs_pt[o] : -1 - lane;
    int seg_start, seg_end;
    segments(j, lane, seg_start, seg_end);
    const int cur = lm->cur;
    Real mu_r;
    if constexpr (MIXED) mu_r = lm->mu_f; else mu_r = lm->mu;
    // t = Z^T dc_k
    Real t0 = 0, t1 = 0, t2 = 0;
    const int f = act ? C.free_idx[k] : -1;
    if (f >= 0) {
      const V2* zp = reinterpret_cast<const V2*>((const Real*)C.rec + (size_t)kRec * o + kRecZ);
      Real Z[18];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const V2 v = zp[i];
        Z[2 * i] = v.x;
        Z[2 * i + 1] = v.y;
      }
      Real d[6];
      if constexpr (MIXED) {
        const float2* d2 = reinterpret_cast<const float2*>(C.dc32 + 6 * f);
        const float2 u0 = d2[0], u1 = d2[1], u2 = d2[2];
        d[0] = u0.x; d[1] = u0.y; d[2] = u1.x; d[3] = u1.y; d[4] = u2.x; d[5] = u2.y;
      } else {
#pragma unroll
        for (int m = 0; m < 6; ++m) d[m] = C.dc[6 * f + m];
      }
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        const Real dm = d[m];
        t0 += Z[3 * m] * dm;
        t1 += Z[3 * m + 1] * dm;
        t2 += Z[3 * m + 2] * dm;
      }
    }
    t0 = seg_reduce(t0, lane, seg_start, seg_end);
    t1 = seg_reduce(t1, lane, seg_start, seg_end);
    t2 = seg_reduce(t2, lane, seg_start, seg_end);
    // head: dX = M^T (q - t), candidate point, pred term
    Real dX0 = 0, dX1 = 0, dX2 = 0;
    Real pp = 0;  // dX^T (mu Dp dX + gp), summed below in FP64
    if (act && lane == seg_start) {
      const Real* pa = (const Real*)C.paux + (size_t)kPaux * j;
      const Real v0 = pa[6] - t0, v1 = pa[7] - t1, v2 = pa[8] - t2;
      dX0 = pa[0] * v0 + pa[1] * v1 + pa[3] * v2;
      dX1 = pa[2] * v1 + pa[4] * v2;
      dX2 = pa[5] * v2;
      const Real m = mu_r;
      pp = dX0 * (m * pa[9] * dX0 + pa[12]) + dX1 * (m * pa[10] * dX1 + pa[13]) + dX2 * (m * pa[11] * dX2 + pa[14]);
    }
    double cost = 0.0;
    if constexpr (MIXED) {
      dfl x0{0.f, 0.f}, x1{0.f, 0.f}, x2{0.f, 0.f};
      if (act && lane == seg_start) {
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
      if (act && lane == seg_start) {
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
  for (int g = warp; g < bv.total_tiles; g += nwarps) {
    const int s = find_slot(bv.tile_pre, bv.n, g);
    const DevCluster& C = bv.cl[s];
    const LmState* lm = C.lm;
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

__global__ void __launch_bounds__(256) k_cost_init(BatchView bv) {
  __shared__ double red[8];
  for (int s = blockIdx.x; s < bv.n; s += gridDim.x) {
    const DevCluster& C = bv.cl[s];
    LmState* lm = C.lm;
    const double F = block_sum_tiles(C, 0, red);
    if (threadIdx.x == 0) {
      const int cur = lm->cur;
      double pc = 0.0;
      for (int k = 0; k < C.n_cams; ++k) {
        if (C.free_idx[k] < 0) continue;
        pc += prior_terms(C.R + ((size_t)cur * C.n_cams + k) * 9, C.T + ((size_t)cur * C.n_cams + k) * 3,
                          C.R_prior + 9 * k, C.T_prior + 3 * k, C.sigma_imu, C.sigma_gnss, nullptr, nullptr);
      }
      lm->F = F + pc;
      lm->pt_fail = 0;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ K6

template <bool MIXED>
__global__ void __launch_bounds__(256) k_lm_update(BatchView bv) {
  __shared__ double red[8];
  __shared__ int s_cur, s_act;
  for (int s = blockIdx.x; s < bv.n; s += gridDim.x) {
    const DevCluster& C = bv.cl[s];
    LmState* lm = C.lm;
    if (!lm->active) continue;
    const bool ok = lm->status == 0;
    double Fo = 0.0, pp = 0.0;
    if (ok) {
      Fo = block_sum_tiles(C, 0, red);
      pp = block_sum_tiles(C, 1, red);
    }
    if (threadIdx.x == 0) {
      const double F = lm->F;
      const double Fn = ok ? Fo + lm->prior_new : F;
      const double pred = ok ? 0.5 * (pp + lm->pred_cam) : 0.0;
      const double gain = pred > 0.0 ? (F - Fn) / pred : 0.0;
      const int accepted = ok && pred > 0.0 && gain > 0.0;
      const double mu_used = lm->mu;
      if (accepted) {
        const double tt = 2.0 * gain - 1.0;
        const double fct = 1.0 - tt * tt * tt;
        lm->mu = mu_used * (fct > 1.0 / 3.0 ? fct : 1.0 / 3.0);
        lm->nu = 2.0;
        lm->cur ^= 1;
        lm->F = Fn;
        lm->n_accepted += 1;
      } else {
        lm->mu = mu_used * lm->nu;
        lm->nu *= 2.0;
      }
      if (C.trace_cap > 0) {
        StepRec& r = C.trace[lm->iter % C.trace_cap];
        r.accepted = accepted;
        r.status = lm->status;
        r.F_before = F;
        r.F_after = Fn;
        r.predicted = pred;
        r.gain = gain;
        r.mu_used = mu_used;
        r.mu = lm->mu;
        r.nu = lm->nu;
      }
      lm->iter += 1;
      if (lm->iter >= lm->iters_target) lm->active = 0;
      lm->pt_fail = 0;
      lm->mu_f = (float)lm->mu;
      s_cur = lm->cur;
      s_act = accepted;
    }
    __syncthreads();
    if (!MIXED && s_act) {  // refresh the binary64 camera records for the new state
      double* cr = (double*)C.camreal;
      for (int k = threadIdx.x; k < C.n_cams; k += blockDim.x) {
        const double* R = C.R + ((size_t)s_cur * C.n_cams + k) * 9;
        const double* T = C.T + ((size_t)s_cur * C.n_cams + k) * 3;
        double* o = cr + (size_t)kCamReal * k;
        for (int i = 0; i < 9; ++i) o[i] = R[i];
        for (int i = 0; i < 3; ++i) o[9 + i] = T[i];
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ diagnostics

template <typename Real>
__global__ void k_grad_norm(BatchView bv, double* out) {
  __shared__ double red[8];
  for (int s = blockIdx.x; s < bv.n; s += gridDim.x) {
    const DevCluster& C = bv.cl[s];
    double m = 0.0;
    for (int i = threadIdx.x; i < 6 * C.n_free; i += blockDim.x) m = fmax(m, fabs(C.gc[i]));
    for (int j = threadIdx.x; j < C.n_pts; j += blockDim.x) {
      const Real* pa = (const Real*)C.paux + (size_t)kPaux * j;
      m = fmax(m, fmax(fabs((double)pa[12]), fmax(fabs((double)pa[13]), fabs((double)pa[14]))));
    }
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

__global__ void k_export_points(const DevCluster* dcl, int mixed, double* out) {
  const DevCluster& C = *dcl;
  const int cur = C.lm->cur;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < C.n_pts; j += gridDim.x * blockDim.x) {
    double X[3];
    point_f64(C, mixed, cur, j, X);
    out[3 * j] = X[0];
    out[3 * j + 1] = X[1];
    out[3 * j + 2] = X[2];
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
    lm->pt_fail = 0;
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
        lm->nu = 2.0;
        lm->F = 0.0;
        lm->F_new = 0.0;
        lm->cur = 0;
        lm->status = 0;
        lm->iter = 0;
        lm->n_accepted = 0;
        lm->active = 0;
        lm->iters_target = 0;
        lm->pt_fail = 0;
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

struct LaunchScope {
  int kind;
  cudaStream_t st;
  cudaEvent_t e0 = nullptr;
  LaunchScope(int k, cudaStream_t s) : kind(k), st(s) {
    if (t_probe) probe_mark(st, &e0);
  }
  ~LaunchScope() {
    if (capturing(st)) ++t_captured; else ++t_direct;
    if (t_probe) {
      cudaEvent_t e1;
      probe_mark(st, &e1);
      t_probe->recs.push_back(ProbeRec{kind, e0, e1});
    }
  }
};

#define LAUNCH(kind, st, ...) \
  do {                          \
    LaunchScope ls__(kind, st); \
    __VA_ARGS__;                \
  } while (0)

static int grid_for(int items, int per_block, int cap) {
  int g = (items + per_block - 1) / per_block;
  if (g > cap) g = cap;
  return g < 1 ? 1 : g;
}

static int g_num_sms = 0;
static int num_sms() {
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
  LAUNCH(KK_COST_INIT, st, k_cost_init<<<grid_for(bv.n, 1, 65535), 256, 0, st>>>(bv));
}

void launch_cost_init(const BatchView& bv, bool mixed, cudaStream_t st) {
  if (mixed) launch_cost_init_t<true>(bv, st);
  else launch_cost_init_t<false>(bv, st);
}

template <bool MIXED>
static void launch_iteration_t(const BatchView& bv, int refine_steps, cudaStream_t st) {
  using Real = typename RealOf<MIXED>::T;
  const int sms = num_sms();
  LAUNCH(KK_LINEARIZE, st, k_linearize<MIXED><<<grid_for(bv.total_tiles, 8, sms * 16), 256, 0, st>>>(bv));
  LAUNCH(KK_CAM_REDUCE, st, k_cam_reduce<Real><<<grid_for(bv.total_cchunks, 1, sms * 32), 128, 0, st>>>(bv));
  if (bv.total_pchunks > 0)
    LAUNCH(KK_PAIR_REDUCE, st, k_pair_reduce<Real><<<grid_for(bv.total_pchunks, 8, sms * 16), 256, 0, st>>>(bv));
  const size_t smem = factor_smem_bytes(bv.max_n);
  LAUNCH(KK_FACTOR, st, k_factor_solve<MIXED><<<grid_for(bv.n, 1, 65535), 512, smem, st>>>(bv, refine_steps, 0));
  LAUNCH(KK_BACKSUB, st, k_backsub_cost<MIXED><<<grid_for(bv.total_tiles, 8, sms * 16), 256, 0, st>>>(bv));
  LAUNCH(KK_LM_UPDATE, st, k_lm_update<MIXED><<<grid_for(bv.n, 1, 65535), 256, 0, st>>>(bv));
}

void launch_iteration(const BatchView& bv, bool mixed, int refine_steps, cudaStream_t st) {
  if (mixed) launch_iteration_t<true>(bv, refine_steps, st);
  else launch_iteration_t<false>(bv, refine_steps, st);
}

template <bool MIXED>
static void launch_grad_norm_t(const BatchView& bv, double* out, cudaStream_t st) {
  using Real = typename RealOf<MIXED>::T;
  const int sms = num_sms();
  LAUNCH(KK_LINEARIZE, st, k_linearize<MIXED><<<grid_for(bv.total_tiles, 8, sms * 16), 256, 0, st>>>(bv));
  LAUNCH(KK_CAM_REDUCE, st, k_cam_reduce<Real><<<grid_for(bv.total_cchunks, 1, sms * 32), 128, 0, st>>>(bv));
  if (bv.total_pchunks > 0)
    LAUNCH(KK_PAIR_REDUCE, st, k_pair_reduce<Real><<<grid_for(bv.total_pchunks, 8, sms * 16), 256, 0, st>>>(bv));
  LAUNCH(KK_FACTOR, st,
         k_factor_solve<MIXED><<<grid_for(bv.n, 1, 65535), 512, factor_smem_bytes(bv.max_n), st>>>(bv, 0, 1));
  LAUNCH(KK_OTHER, st, k_grad_norm<Real><<<grid_for(bv.n, 1, 65535), 256, 0, st>>>(bv, out));
}

void launch_grad_norm(const BatchView& bv, bool mixed, double* out, cudaStream_t st) {
  if (mixed) launch_grad_norm_t<true>(bv, out, st);
  else launch_grad_norm_t<false>(bv, out, st);
}

void launch_reproj(const DevCluster* dcl, const DevCluster& hcl, bool mixed, double* err_pm, cudaStream_t st) {
  LAUNCH(KK_OTHER, st, k_reproj<<<grid_for(hcl.n_obs, 256, num_sms() * 8), 256, 0, st>>>(dcl, mixed, err_pm));
}

void launch_export_points(const DevCluster* dcl, const DevCluster& hcl, bool mixed, double* out, cudaStream_t st) {
  LAUNCH(KK_OTHER, st, k_export_points<<<grid_for(hcl.n_pts, 256, num_sms() * 8), 256, 0, st>>>(dcl, mixed, out));
}

cudaError_t set_kernel_attributes(int max_n) {
  const size_t smem = factor_smem_bytes(max_n);
  cudaError_t e = cudaFuncSetAttribute(k_factor_solve<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_factor_solve<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace bagpu
