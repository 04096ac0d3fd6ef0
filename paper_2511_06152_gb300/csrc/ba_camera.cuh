// Camera records and candidate poses, shared by the reduced-system solvers.
#pragma once
#include "ba_device.cuh"
#include "ba_dfloat.cuh"
#include "ba_internal.h"

namespace bagpu {

// mixed path: double-float record of camera k from (R, T) in binary64, in the
// layout the kernels read (high words of the linearisation's inputs first)
__device__ inline void write_camdf(const DevCluster& C, int buf, int k, const double* R, const double* T) {
  float* o = C.camdf + ((size_t)buf * C.n_cams + k) * kCamDf;
  for (int i = 0; i < 9; ++i) {
    const dfl v = df_from_d(R[i]);
    o[i] = v.hi;
    o[24 + i] = v.lo;
  }
  for (int i = 0; i < 3; ++i) {
    const dfl v = df_from_d(T[i]);
    o[9 + i] = v.hi;
    o[12 + i] = v.lo;
  }
  const dfl f = df_from_d(C.intr[7 * k]);
  o[15] = f.hi;
  o[33] = f.lo;
  for (int i = 0; i < 4; ++i) {
    const dfl v = df_from_d(C.intr[7 * k + 3 + i]);
    o[16 + i] = v.hi;
    o[34 + i] = v.lo;
  }
  o[20] = C.free_idx[k] >= 0 ? 1.0f : 0.0f;
  for (int i = 21; i < 24; ++i) o[i] = 0.0f;
  for (int i = 38; i < kCamDf; ++i) o[i] = 0.0f;
}

// Candidate pose of camera k for the step x (in the elimination order,
// 6 per free image): R Exp(dtheta), T + dT in binary64, written to state
// buffer cur ^ 1 (and its double-float record in the mixed path).  A fixed
// camera, or any camera when fail is set, keeps its pose.  For a free camera
// *pc = d^T (mu D d + g) of its block and *pn = its prior cost at the
// candidate; 0 otherwise.
template <bool MIXED>
__device__ inline void candidate_camera(const DevCluster& C, int k, const double* x, double mu, int cur, bool fail,
                                        double* pc, double* pn) {
  const int nc = C.n_cams;
  const double* Rc = C.R + (size_t)cur * nc * 9 + 9 * k;
  const double* Tc = C.T + (size_t)cur * nc * 3 + 3 * k;
  double* Rn = C.R + (size_t)(cur ^ 1) * nc * 9 + 9 * k;
  double* Tn = C.T + (size_t)(cur ^ 1) * nc * 3 + 3 * k;
  const int f = C.free_idx[k];
  *pc = 0.0;
  *pn = 0.0;
  if (f < 0 || fail) {
    for (int i = 0; i < 9; ++i) Rn[i] = Rc[i];
    for (int i = 0; i < 3; ++i) Tn[i] = Tc[i];
  } else {
    const double* d = x + 6 * C.fpos[f];
    double E[9];
    so3_exp(d, E);
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) Rn[3 * r + c] = Rc[3 * r] * E[c] + Rc[3 * r + 1] * E[3 + c] + Rc[3 * r + 2] * E[6 + c];
    for (int i = 0; i < 3; ++i) Tn[i] = Tc[i] + d[3 + i];
    double s = 0.0;
    for (int a = 0; a < 6; ++a) s += d[a] * (mu * C.Dc[6 * f + a] * d[a] + C.gc[6 * f + a]);
    *pc = s;
    *pn = prior_terms(Rn, Tn, C.R_prior + 9 * k, C.T_prior + 3 * k, C.sigma_imu, C.sigma_gnss, nullptr, nullptr);
  }
  if constexpr (MIXED) write_camdf(C, cur ^ 1, k, Rn, Tn);
}

}  // namespace bagpu
