// Device helpers: SO(3), the camera model of Eq. 5 with Brown distortion,
// the Huber weight of Eq. 6, and deterministic warp reductions.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "ba_internal.h"

namespace bagpu {

#define BA_FULL_MASK 0xffffffffu

__device__ __forceinline__ float rsqrt_any(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_any(double x) { return rsqrt(x); }

// 1 / sqrt(d) of a Cholesky pivot d > 0.  A pivot can be positive but tiny
// (a block whose only term is mu * D with a tiny damping mu, down to
// subnormal values): the reciprocal square root is taken of d scaled by an
// even power of two into the normal range, and the result is scaled back.
__device__ __forceinline__ double pivot_rsqrt(double d) {
  return d < 0x1p-960 ? rsqrt(d * 0x1p960) * 0x1p480 : rsqrt(d);
}
__device__ __forceinline__ float pivot_rsqrt(float d) {
  return d < 0x1p-100f ? rsqrtf(d * 0x1p100f) * 0x1p50f : rsqrtf(d);
}
__device__ __forceinline__ float recip_any(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip_any(double x) { return 1.0 / x; }

// largest s in [0, n) with pre[s] <= g (pre is non-decreasing)
__device__ __forceinline__ int find_slot(const int* __restrict__ pre, int n, int g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(pre + mid) <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Reduce v over lanes [seg_start, seg_end) of a warp to lane seg_start by a
// binary tree whose shape depends only on the segment: deterministic.
// span = the warp's longest segment (warp-uniform): the levels at or above
// it add nothing and are skipped, which leaves every sum unchanged.
template <typename T>
__device__ __forceinline__ T seg_reduce(T v, int lane, int seg_start, int seg_end, int span = 32) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    if (off >= span) break;
    const T o = __shfl_down_sync(BA_FULL_MASK, v, off);
    if (((lane - seg_start) & (2 * off - 1)) == 0 && lane + off < seg_end) v += o;
  }
  return v;
}

// Whole-warp tree sum to lane 0 (fixed order).
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(BA_FULL_MASK, v, off);
  return v;
}

// Segment bounds of each lane from the point index of its observation
// (inactive lanes carry a unique negative key and are their own segment).
__device__ __forceinline__ void segments(int key, int lane, int& seg_start, int& seg_end) {
  const int prev = __shfl_up_sync(BA_FULL_MASK, key, 1);
  const bool head = (lane == 0) || (key != prev) || key < 0;
  const unsigned heads = __ballot_sync(BA_FULL_MASK, head);
  const unsigned upto = (2u << lane) - 1u;  // lanes 0..lane (lane 31 wraps to all ones)
  seg_start = 31 - __clz(heads & upto);
  const unsigned after = heads & ~upto;
  seg_end = after ? __ffs(after) - 1 : 32;
}

// longest segment of the warp
__device__ __forceinline__ int segment_span(int seg_start, int seg_end) {
  return (int)__reduce_max_sync(BA_FULL_MASK, (unsigned)(seg_end - seg_start));
}

template <typename Real>
__device__ __forceinline__ Real clamp_diag(Real v) {
  return v < Real(kDiagMin) ? Real(kDiagMin) : (v > Real(kDiagMax) ? Real(kDiagMax) : v);
}

// ------------------------------------------------------------------ SO(3), FP64

// R = Exp(w) = I + a [w]x + b [w]x^2, [w]x^2 = w w^T - |w|^2 I
__device__ inline void so3_exp(const double w[3], double R[9]) {
  const double t2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double a, b;
  if (t2 < 1e-16) {
    a = 1.0 - t2 / 6.0;
    b = 0.5 - t2 / 24.0;
  } else {
    const double t = sqrt(t2);
    double s, c;
    sincos(t, &s, &c);
    a = s / t;
    b = (1.0 - c) / t2;
  }
  const double d = 1.0 - b * t2;
  R[0] = d + b * w[0] * w[0];
  R[4] = d + b * w[1] * w[1];
  R[8] = d + b * w[2] * w[2];
  R[1] = b * w[0] * w[1] - a * w[2];
  R[3] = b * w[0] * w[1] + a * w[2];
  R[2] = b * w[0] * w[2] + a * w[1];
  R[6] = b * w[0] * w[2] - a * w[1];
  R[5] = b * w[1] * w[2] - a * w[0];
  R[7] = b * w[1] * w[2] + a * w[0];
}

__device__ inline void so3_log(const double R[9], double w[3]) {
  double c = 0.5 * (R[0] + R[4] + R[8] - 1.0);
  c = fmin(1.0, fmax(-1.0, c));
  const double t = acos(c);
  const double v0 = R[7] - R[5], v1 = R[2] - R[6], v2 = R[3] - R[1];
  if (t < 1e-8) {
    const double s = 0.5 * (1.0 + t * t / 6.0);
    w[0] = s * v0; w[1] = s * v1; w[2] = s * v2;
  } else if (t > 3.14159165358979 /* pi - 1e-6 */) {
    // axis from the column of R + I with the largest norm
    int col = 0;
    double best = -1.0;
    for (int j = 0; j < 3; ++j) {
      const double a0 = R[j] + (j == 0), a1 = R[3 + j] + (j == 1), a2 = R[6 + j] + (j == 2);
      const double nn = a0 * a0 + a1 * a1 + a2 * a2;
      if (nn > best) { best = nn; col = j; }
    }
    const double inv = 1.0 / sqrt(best);
    double ax0 = (R[col] + (col == 0)) * inv, ax1 = (R[3 + col] + (col == 1)) * inv,
           ax2 = (R[6 + col] + (col == 2)) * inv;
    if (ax0 * v0 + ax1 * v1 + ax2 * v2 < 0.0) { ax0 = -ax0; ax1 = -ax1; ax2 = -ax2; }
    w[0] = t * ax0; w[1] = t * ax1; w[2] = t * ax2;
  } else {
    const double s = t / (2.0 * sin(t));
    w[0] = s * v0; w[1] = s * v1; w[2] = s * v2;
  }
}

// inverse right Jacobian: I + 1/2 [w]x + c2 [w]x^2
__device__ inline void so3_jr_inv(const double w[3], double J[9]) {
  const double t2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double c2;
  if (t2 < 1e-10) {
    c2 = 1.0 / 12.0 + t2 / 720.0;
  } else {
    const double t = sqrt(t2);
    double s, c;
    sincos(t, &s, &c);
    c2 = 1.0 / t2 - (1.0 + c) / (2.0 * t * s);
  }
  const double d = 1.0 - c2 * t2;
  J[0] = d + c2 * w[0] * w[0];
  J[4] = d + c2 * w[1] * w[1];
  J[8] = d + c2 * w[2] * w[2];
  J[1] = c2 * w[0] * w[1] - 0.5 * w[2];
  J[3] = c2 * w[0] * w[1] + 0.5 * w[2];
  J[2] = c2 * w[0] * w[2] + 0.5 * w[1];
  J[6] = c2 * w[0] * w[2] - 0.5 * w[1];
  J[5] = c2 * w[1] * w[2] - 0.5 * w[0];
  J[7] = c2 * w[1] * w[2] + 0.5 * w[0];
}

// GNSS/IMU prior of one camera at (R, T): residual phi = Log(Rp^T R),
// e = T - Tp, whitened.  Fills J^T J (6x6 row-major) and J^T r (6), and
// returns the prior cost 1/2 |r|^2.
__device__ inline double prior_terms(const double* R, const double* T, const double* Rp, const double* Tp,
                                     double sigma_imu, double sigma_gnss, double* JtJ, double* Jtr) {
  double cost = 0.0;
  if (JtJ) for (int i = 0; i < 36; ++i) JtJ[i] = 0.0;
  if (Jtr) for (int i = 0; i < 6; ++i) Jtr[i] = 0.0;
  if (sigma_imu > 0.0) {
    double E[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) E[3 * i + j] = Rp[i] * R[j] + Rp[3 + i] * R[3 + j] + Rp[6 + i] * R[6 + j];
    double phi[3];
    so3_log(E, phi);
    const double iv = 1.0 / (sigma_imu * sigma_imu);
    cost += 0.5 * iv * (phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]);
    if (JtJ || Jtr) {
      double Jr[9];
      so3_jr_inv(phi, Jr);
      for (int a = 0; a < 3; ++a) {
        if (Jtr) Jtr[a] = iv * (Jr[a] * phi[0] + Jr[3 + a] * phi[1] + Jr[6 + a] * phi[2]);
        if (JtJ)
          for (int b = 0; b < 3; ++b)
            JtJ[6 * a + b] = iv * (Jr[a] * Jr[b] + Jr[3 + a] * Jr[3 + b] + Jr[6 + a] * Jr[6 + b]);
      }
    }
  }
  if (sigma_gnss > 0.0) {
    const double ig = 1.0 / (sigma_gnss * sigma_gnss);
    for (int a = 0; a < 3; ++a) {
      const double e = T[a] - Tp[a];
      cost += 0.5 * ig * e * e;
      if (Jtr) Jtr[3 + a] = ig * e;
      if (JtJ) JtJ[6 * (3 + a) + 3 + a] = ig;
    }
  }
  return cost;
}

// ------------------------------------------------------------------ Eq. 5 + Brown, Eq. 6

// FP64 robust cost term 1/2 rho(s) / sigma^2 of one observation (0 behind the camera).
__device__ __forceinline__ double obs_cost(const double* R, const double* T, const double* in, const double* X,
                                           double uo, double vo, double half_inv_s2, double delta) {
  const double dx = X[0] - T[0], dy = X[1] - T[1], dz = X[2] - T[2];
  const double x = R[0] * dx + R[3] * dy + R[6] * dz;
  const double y = R[1] * dx + R[4] * dy + R[7] * dz;
  const double z = R[2] * dx + R[5] * dy + R[8] * dz;
  if (!(z > kMinDepth)) return 0.0;
  const double iz = 1.0 / z;
  const double xn = x * iz, yn = y * iz;
  const double r2 = xn * xn + yn * yn;
  const double rad = 1.0 + r2 * (in[3] + in[4] * r2);
  const double xd = xn * rad + 2.0 * in[5] * xn * yn + in[6] * (r2 + 2.0 * xn * xn);
  const double yd = yn * rad + in[5] * (r2 + 2.0 * yn * yn) + 2.0 * in[6] * xn * yn;
  const double e0 = in[0] * xd + in[1] - uo, e1 = in[0] * yd + in[2] - vo;
  const double s = e0 * e0 + e1 * e1;
  const double d2 = delta * delta;
  const double rho = s <= d2 ? s : 2.0 * delta * sqrt(s) - d2;
  return half_inv_s2 * rho;
}

__device__ __forceinline__ double obs_error_norm(const double* R, const double* T, const double* in, const double* X,
                                                 double uo, double vo) {
  const double dx = X[0] - T[0], dy = X[1] - T[1], dz = X[2] - T[2];
  const double x = R[0] * dx + R[3] * dy + R[6] * dz;
  const double y = R[1] * dx + R[4] * dy + R[7] * dz;
  const double z = R[2] * dx + R[5] * dy + R[8] * dz;
  const double iz = 1.0 / z;
  const double xn = x * iz, yn = y * iz;
  const double r2 = xn * xn + yn * yn;
  const double rad = 1.0 + r2 * (in[3] + in[4] * r2);
  const double xd = xn * rad + 2.0 * in[5] * xn * yn + in[6] * (r2 + 2.0 * xn * xn);
  const double yd = yn * rad + in[5] * (r2 + 2.0 * yn * yn) + 2.0 * in[6] * xn * yn;
  return hypot(in[0] * xd + in[1] - uo, in[0] * yd + in[2] - vo);
}

// Whitened, robust-weighted residual and Jacobians of one observation.
// d = X - T (world), Rm camera->world (row-major), in = (f, cx, cy, k1, k2, p1, p2).
// Jc is 2x6 row-major over [dtheta, dT] (right perturbation), Jp is 2x3.
template <typename Real>
__device__ __forceinline__ bool obs_linearize(const Real* Rm, Real dx, Real dy, Real dz, const Real* in, Real uo,
                                              Real vo, Real inv_sigma, Real delta, Real& r0, Real& r1, Real Jc[12],
                                              Real Jp[6]) {
  const Real x = Rm[0] * dx + Rm[3] * dy + Rm[6] * dz;
  const Real y = Rm[1] * dx + Rm[4] * dy + Rm[7] * dz;
  const Real z = Rm[2] * dx + Rm[5] * dy + Rm[8] * dz;
  if (!(z > Real(kMinDepth))) {
    r0 = r1 = Real(0);
#pragma unroll
    for (int i = 0; i < 12; ++i) Jc[i] = Real(0);
#pragma unroll
    for (int i = 0; i < 6; ++i) Jp[i] = Real(0);
    return false;
  }
  const Real f = in[0], k1 = in[3], k2 = in[4], p1 = in[5], p2 = in[6];
  const Real iz = recip_any(z);
  const Real xn = x * iz, yn = y * iz;
  const Real r2 = xn * xn + yn * yn;
  const Real rad = Real(1) + r2 * (k1 + k2 * r2);
  const Real xd = xn * rad + Real(2) * p1 * xn * yn + p2 * (r2 + Real(2) * xn * xn);
  const Real yd = yn * rad + p1 * (r2 + Real(2) * yn * yn) + Real(2) * p2 * xn * yn;
  const Real e0 = f * xd + in[1] - uo;
  const Real e1 = f * yd + in[2] - vo;
  const Real s = e0 * e0 + e1 * e1;
  // IRLS weight w = rho'(s); scale = sqrt(w) / sigma
  Real scale = inv_sigma;
  if (s > delta * delta) scale *= sqrt(delta * rsqrt_any(s));
  r0 = scale * e0;
  r1 = scale * e1;
  // d(xd, yd)/d(xn, yn)
  const Real drad = Real(2) * k1 + Real(4) * k2 * r2;
  const Real D00 = rad + drad * xn * xn + Real(2) * p1 * yn + Real(6) * p2 * xn;
  const Real D01 = drad * xn * yn + Real(2) * p1 * xn + Real(2) * p2 * yn;
  const Real D11 = rad + drad * yn * yn + Real(6) * p1 * yn + Real(2) * p2 * xn;
  // A = f D d(xn,yn)/dXc, scaled
  const Real a = scale * f * iz;
  const Real A00 = a * D00, A01 = a * D01, A02 = -a * (D00 * xn + D01 * yn);
  const Real A10 = a * D01, A11 = a * D11, A12 = -a * (D01 * xn + D11 * yn);
  // dXc/dX = R^T: Jp[r][b] = sum_c A[r][c] R[b][c]
  Jp[0] = A00 * Rm[0] + A01 * Rm[1] + A02 * Rm[2];
  Jp[1] = A00 * Rm[3] + A01 * Rm[4] + A02 * Rm[5];
  Jp[2] = A00 * Rm[6] + A01 * Rm[7] + A02 * Rm[8];
  Jp[3] = A10 * Rm[0] + A11 * Rm[1] + A12 * Rm[2];
  Jp[4] = A10 * Rm[3] + A11 * Rm[4] + A12 * Rm[5];
  Jp[5] = A10 * Rm[6] + A11 * Rm[7] + A12 * Rm[8];
  // dXc/ddtheta = [Xc]x
  Jc[0] = A01 * z - A02 * y;
  Jc[1] = A02 * x - A00 * z;
  Jc[2] = A00 * y - A01 * x;
  Jc[6] = A11 * z - A12 * y;
  Jc[7] = A12 * x - A10 * z;
  Jc[8] = A10 * y - A11 * x;
  // dXc/dT = -R^T
  Jc[3] = -Jp[0]; Jc[4] = -Jp[1]; Jc[5] = -Jp[2];
  Jc[9] = -Jp[3]; Jc[10] = -Jp[4]; Jc[11] = -Jp[5];
  return true;
}

// The LM decision of one cluster, by one warp, once every tile of its
// back-substitution is done: F(x + d) and pred from the tiles' partial sums
// (in k_cost_init's summation order), the gain ratio,
// accept or reject, Nielsen's update of mu and nu, the step record; on
// acceptance in binary64 the camera records of the new state.
template <bool MIXED>
__device__ __forceinline__ void lm_update_warp(const DevCluster& C, int lane) {
  LmState* lm = C.lm;
  const bool ok = lm->status == 0;
  double Fo = 0.0, pp = 0.0;
  if (ok) {
    // the order of k_cost_init's sum over a 256-thread CTA (thread t of warp
    // t / 32 adds tiles t, t + 256, ... in turn; a warp tree; the 8 warps in
    // order), so that F carried from one iteration to the next equals F
    // evaluated afresh at the start of a solve, bit for bit
    const double2* tp = reinterpret_cast<const double2*>(C.tilepart);
    for (int w = 0; w < kCostInitThreads / 32; ++w) {
      double a = 0.0, b = 0.0;
      for (int i = 32 * w + lane; i < C.n_tiles; i += kCostInitThreads) {
        const double2 v = tp[i];
        a += v.x;
        b += v.y;
      }
      Fo += warp_sum(a);
      pp += warp_sum(b);
    }
  }
  int accepted = 0, cur = 0;
  if (lane == 0) {
    const double F = lm->F;
    const double Fn = ok ? Fo + lm->prior_new : F;
    const double pred = ok ? 0.5 * (pp + lm->pred_cam) : 0.0;
    const double gain = pred > 0.0 ? (F - Fn) / pred : 0.0;
    accepted = ok && pred > 0.0 && gain > 0.0;
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
    // converged (serving): an accepted step, not the first since arming, that
    // lowered F by at most ftol * F
    if (lm->ftol > 0.0 && accepted && lm->iter - lm->iter0 >= 2 && F - Fn <= lm->ftol * F) lm->active = 0;
    lm->pt_fail = 0;
    lm->mu_f = (float)lm->mu;
    cur = lm->cur;
  }
  accepted = __shfl_sync(BA_FULL_MASK, accepted, 0);
  cur = __shfl_sync(BA_FULL_MASK, cur, 0);
  if (!MIXED && accepted) {  // refresh the binary64 camera records for the new state
    double* cr = (double*)C.camreal;
    for (int k = lane; k < C.n_cams; k += 32) {
      const double* R = C.R + ((size_t)cur * C.n_cams + k) * 9;
      const double* T = C.T + ((size_t)cur * C.n_cams + k) * 3;
      double* o = cr + (size_t)kCamReal * k;
      for (int i = 0; i < 9; ++i) o[i] = R[i];
      for (int i = 0; i < 3; ++i) o[9 + i] = T[i];
    }
  }
}

}  // namespace bagpu
