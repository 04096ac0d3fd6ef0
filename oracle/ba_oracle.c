/*
 * Plain FP64 CPU oracle for the local bundle-adjustment LM iteration.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the GPU path computes.  Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * What it follows:
 *   - Eq. 5 (Sec. 3.2): observation p_kj = pi(K R_k^T (X_j - T_k)), R_k
 *     camera->world, T_k the camera centre, pi(x,y,z) = (x/z, y/z) (Sec. 3.1).
 *     K is extended with Brown radial (k1,k2) and tangential (p1,p2) terms
 *     applied to the normalised coordinates before the focal length.
 *   - Eq. 6 / Eq. 7: robust cost sum_k sum_j rho(||p_kj - pi(...)||^2), rho
 *     acting on the squared 2-D norm of each observation.  rho is Huber with
 *     threshold delta (pixels); residuals are whitened by sigma_px.
 *   - Sec. 3.2 (initial values from GNSS/IMU): GNSS position and IMU attitude
 *     priors, whitened by sigma_gnss and sigma_imu, are added to the cost for
 *     every free camera.  A sigma of 0 switches that prior off.
 *   - Sec. 3.2 (cluster overlap): fixed cameras keep their pose; their
 *     observations still constrain the points.
 *   - The optimiser, which the paper leaves unnamed, is Levenberg-Marquardt
 *     with Marquardt diagonal scaling and Nielsen's damping update (Nielsen
 *     1999; Madsen, Nielsen & Tingleff 2004), solved by eliminating the 3x3
 *     point blocks (Schur complement) and a dense Cholesky of the reduced
 *     camera system.  Robust weights enter by iteratively reweighted least
 *     squares (w = rho'(s)).
 *
 * Parameter update (right perturbation): R <- R Exp(dtheta), T <- T + dT,
 * X <- X + dX; a camera's 6-vector is ordered [dtheta, dT].
 *
 * Every function is pinned by the tests in tests/test_oracle_*.py: finite
 * differences, closed forms, a dense normal-equation solve, zero-noise
 * convergence and cost monotonicity.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "ba_oracle.h"

/* ------------------------------------------------------------------ */
/* small linear algebra                                                */
/* ------------------------------------------------------------------ */

static void mat3_mul(const double A[9], const double B[9], double C[9]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
      C[3 * i + j] = s;
    }
}

/* C = A^T B */
static void mat3_tmul(const double A[9], const double B[9], double C[9]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[3 * k + i] * B[3 * k + j];
      C[3 * i + j] = s;
    }
}

static void skew(const double w[3], double S[9]) {
  S[0] = 0.0;   S[1] = -w[2]; S[2] = w[1];
  S[3] = w[2];  S[4] = 0.0;   S[5] = -w[0];
  S[6] = -w[1]; S[7] = w[0];  S[8] = 0.0;
}

/* ------------------------------------------------------------------ */
/* SO(3): Rodrigues' formula and its inverse; the inverse right        */
/* Jacobian in the closed form of Barfoot, State Estimation for        */
/* Robotics (2017), Sec. 7.1.                                          */
/* ------------------------------------------------------------------ */

void orc_so3_exp(const double w[3], double R[9]) {
  double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double th = sqrt(th2);
  double a, b; /* R = I + a [w]x + b [w]x^2 */
  if (th < 1e-8) {
    a = 1.0 - th2 / 6.0;
    b = 0.5 - th2 / 24.0;
  } else {
    a = sin(th) / th;
    b = (1.0 - cos(th)) / th2;
  }
  double S[9], S2[9];
  skew(w, S);
  mat3_mul(S, S, S2);
  for (int i = 0; i < 9; ++i) R[i] = a * S[i] + b * S2[i];
  R[0] += 1.0; R[4] += 1.0; R[8] += 1.0;
}

void orc_so3_log(const double R[9], double w[3]) {
  double tr = R[0] + R[4] + R[8];
  double c = 0.5 * (tr - 1.0);
  if (c > 1.0) c = 1.0;
  if (c < -1.0) c = -1.0;
  double th = acos(c);
  double v[3] = {R[7] - R[5], R[2] - R[6], R[3] - R[1]}; /* 2 sin(th) * axis */
  if (th < 1e-8) {
    /* R ~ I + [w]x: take the skew part, with the first correction term */
    double s = 0.5 * (1.0 + th * th / 6.0);
    for (int i = 0; i < 3; ++i) w[i] = s * v[i];
  } else if (th > M_PI - 1e-6) {
    /* near pi the skew part vanishes; read the axis off R + I */
    double B[9];
    for (int i = 0; i < 9; ++i) B[i] = R[i];
    B[0] += 1.0; B[4] += 1.0; B[8] += 1.0;
    int col = 0;
    double best = -1.0;
    for (int j = 0; j < 3; ++j) {
      double n = B[j] * B[j] + B[3 + j] * B[3 + j] + B[6 + j] * B[6 + j];
      if (n > best) { best = n; col = j; }
    }
    double nn = sqrt(best);
    double ax[3] = {B[col] / nn, B[3 + col] / nn, B[6 + col] / nn};
    /* fix the sign with the (small) skew part */
    if (ax[0] * v[0] + ax[1] * v[1] + ax[2] * v[2] < 0.0) {
      ax[0] = -ax[0]; ax[1] = -ax[1]; ax[2] = -ax[2];
    }
    for (int i = 0; i < 3; ++i) w[i] = th * ax[i];
  } else {
    double s = th / (2.0 * sin(th));
    for (int i = 0; i < 3; ++i) w[i] = s * v[i];
  }
}

void orc_so3_jr_inv(const double w[3], double J[9]) {
  double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double th = sqrt(th2);
  double c2; /* coefficient of [w]x^2 */
  if (th < 1e-5) {
    c2 = 1.0 / 12.0 + th2 / 720.0;
  } else {
    c2 = 1.0 / th2 - (1.0 + cos(th)) / (2.0 * th * sin(th));
  }
  double S[9], S2[9];
  skew(w, S);
  mat3_mul(S, S, S2);
  for (int i = 0; i < 9; ++i) J[i] = 0.5 * S[i] + c2 * S2[i];
  J[0] += 1.0; J[4] += 1.0; J[8] += 1.0;
}

/* ------------------------------------------------------------------ */
/* Eq. 5 with Brown distortion                                         */
/* ------------------------------------------------------------------ */

int orc_project(const double intr[7], const double R[9], const double T[3], const double X[3],
                double uv[2]) {
  double d[3] = {X[0] - T[0], X[1] - T[1], X[2] - T[2]};
  double Xc[3];
  for (int i = 0; i < 3; ++i) Xc[i] = R[i] * d[0] + R[3 + i] * d[1] + R[6 + i] * d[2]; /* R^T d */
  if (Xc[2] <= ORC_MIN_DEPTH) {
    uv[0] = uv[1] = 0.0;
    return 0;
  }
  double xn = Xc[0] / Xc[2], yn = Xc[1] / Xc[2];
  double f = intr[0], cx = intr[1], cy = intr[2];
  double k1 = intr[3], k2 = intr[4], p1 = intr[5], p2 = intr[6];
  double r2 = xn * xn + yn * yn;
  double rad = 1.0 + k1 * r2 + k2 * r2 * r2;
  double xd = xn * rad + 2.0 * p1 * xn * yn + p2 * (r2 + 2.0 * xn * xn);
  double yd = yn * rad + p1 * (r2 + 2.0 * yn * yn) + 2.0 * p2 * xn * yn;
  uv[0] = f * xd + cx;
  uv[1] = f * yd + cy;
  return 1;
}

/* ------------------------------------------------------------------ */
/* Huber on the squared norm s (Eq. 6: rho acts on ||r||^2)             */
/* ------------------------------------------------------------------ */

double orc_huber_rho(double s, double delta) {
  double d2 = delta * delta;
  if (s <= d2) return s;
  return 2.0 * delta * sqrt(s) - d2;
}

double orc_huber_weight(double s, double delta) { /* rho'(s) */
  if (s <= delta * delta) return 1.0;
  return delta / sqrt(s);
}

/* ------------------------------------------------------------------ */
/* one observation: whitened, robust-weighted residual and Jacobians   */
/* ------------------------------------------------------------------ */

int orc_linearize_obs(const orc_problem* P, const double* R, const double* T, const double* X, int i,
                      double r[2], double Jc[12], double Jp[6], double* s_out) {
  int k = P->obs_cam[i], j = P->obs_pt[i];
  const double* Rk = R + 9 * k;
  const double* Tk = T + 3 * k;
  const double* Xj = X + 3 * j;
  const double* in = P->intr + 7 * k;
  double d[3] = {Xj[0] - Tk[0], Xj[1] - Tk[1], Xj[2] - Tk[2]};
  double Xc[3];
  for (int a = 0; a < 3; ++a) Xc[a] = Rk[a] * d[0] + Rk[3 + a] * d[1] + Rk[6 + a] * d[2];
  memset(r, 0, 2 * sizeof(double));
  memset(Jc, 0, 12 * sizeof(double));
  memset(Jp, 0, 6 * sizeof(double));
  if (Xc[2] <= ORC_MIN_DEPTH) { /* behind the camera: weight 0 */
    if (s_out) *s_out = 0.0;
    return 0;
  }
  double x = Xc[0], y = Xc[1], z = Xc[2];
  double xn = x / z, yn = y / z;
  double f = in[0], cx = in[1], cy = in[2], k1 = in[3], k2 = in[4], p1 = in[5], p2 = in[6];
  double r2 = xn * xn + yn * yn;
  double rad = 1.0 + k1 * r2 + k2 * r2 * r2;
  double xd = xn * rad + 2.0 * p1 * xn * yn + p2 * (r2 + 2.0 * xn * xn);
  double yd = yn * rad + p1 * (r2 + 2.0 * yn * yn) + 2.0 * p2 * xn * yn;
  double res[2] = {f * xd + cx - P->obs_uv[2 * i], f * yd + cy - P->obs_uv[2 * i + 1]};
  double s = res[0] * res[0] + res[1] * res[1];
  if (s_out) *s_out = s;

  /* d(xd,yd)/d(xn,yn) */
  double drad_dx = 2.0 * k1 * xn + 4.0 * k2 * r2 * xn;
  double drad_dy = 2.0 * k1 * yn + 4.0 * k2 * r2 * yn;
  double D[4];
  D[0] = rad + xn * drad_dx + 2.0 * p1 * yn + 6.0 * p2 * xn;
  D[1] = xn * drad_dy + 2.0 * p1 * xn + 2.0 * p2 * yn;
  D[2] = yn * drad_dx + 2.0 * p1 * xn + 2.0 * p2 * yn;
  D[3] = rad + yn * drad_dy + 6.0 * p1 * yn + 2.0 * p2 * xn;
  /* d(xn,yn)/dXc */
  double Pn[6] = {1.0 / z, 0.0, -x / (z * z), 0.0, 1.0 / z, -y / (z * z)};
  /* A = f * D * Pn : d(u,v)/dXc, 2x3 */
  double A[6];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 3; ++b) A[3 * a + b] = f * (D[2 * a] * Pn[b] + D[2 * a + 1] * Pn[3 + b]);

  /* dXc/ddtheta = [Xc]x, dXc/dT = -R^T, dXc/dX = R^T */
  double Sx[9];
  skew(Xc, Sx);
  double scale = sqrt(orc_huber_weight(s, P->huber_delta)) / P->sigma_px;
  for (int a = 0; a < 2; ++a) {
    for (int b = 0; b < 3; ++b) {
      double jt = 0.0, jx = 0.0;
      for (int c = 0; c < 3; ++c) {
        jt += A[3 * a + c] * Sx[3 * c + b];
        jx += A[3 * a + c] * Rk[3 * b + c]; /* (R^T)[c][b] = R[b][c] */
      }
      Jc[6 * a + b] = scale * jt;
      Jc[6 * a + 3 + b] = -scale * jx;
      Jp[3 * a + b] = scale * jx;
    }
    r[a] = scale * res[a];
  }
  return 1;
}

/* prior residual (6) and Jacobian (6x6, rows [r_R; r_T], cols [dtheta, dT]) */
void orc_linearize_prior(const orc_problem* P, const double* R, const double* T, int k, double r[6],
                         double J[36]) {
  memset(r, 0, 6 * sizeof(double));
  memset(J, 0, 36 * sizeof(double));
  if (P->sigma_imu > 0.0) {
    double E[9], phi[3], Jr[9];
    mat3_tmul(P->R_prior + 9 * k, R + 9 * k, E); /* R_imu^T R */
    orc_so3_log(E, phi);
    orc_so3_jr_inv(phi, Jr);
    for (int a = 0; a < 3; ++a) {
      r[a] = phi[a] / P->sigma_imu;
      for (int b = 0; b < 3; ++b) J[6 * a + b] = Jr[3 * a + b] / P->sigma_imu;
    }
  }
  if (P->sigma_gnss > 0.0) {
    for (int a = 0; a < 3; ++a) {
      r[3 + a] = (T[3 * k + a] - P->T_prior[3 * k + a]) / P->sigma_gnss;
      J[6 * (3 + a) + 3 + a] = 1.0 / P->sigma_gnss;
    }
  }
}

/* ------------------------------------------------------------------ */
/* cost F(x) = 1/2 sum rho(s)/sigma_px^2 + 1/2 sum_free ||prior||^2    */
/* ------------------------------------------------------------------ */

double orc_cost(const orc_problem* P, const double* R, const double* T, const double* X) {
  double F = 0.0;
  for (int i = 0; i < P->n_obs; ++i) {
    int k = P->obs_cam[i], j = P->obs_pt[i];
    double uv[2];
    if (!orc_project(P->intr + 7 * k, R + 9 * k, T + 3 * k, X + 3 * j, uv)) continue;
    double e0 = uv[0] - P->obs_uv[2 * i], e1 = uv[1] - P->obs_uv[2 * i + 1];
    F += 0.5 * orc_huber_rho(e0 * e0 + e1 * e1, P->huber_delta) / (P->sigma_px * P->sigma_px);
  }
  for (int k = 0; k < P->n_cams; ++k) {
    if (P->fixed[k]) continue;
    double r[6], J[36];
    orc_linearize_prior(P, R, T, k, r, J);
    for (int a = 0; a < 6; ++a) F += 0.5 * r[a] * r[a];
  }
  return F;
}

/* ------------------------------------------------------------------ */
/* dense Cholesky (lower, in place) and triangular solves               */
/* ------------------------------------------------------------------ */

static int cholesky(int n, double* A) {
  for (int j = 0; j < n; ++j) {
    double d = A[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
    if (!(d > 0.0)) return -1;
    d = sqrt(d);
    A[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double s = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) s -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
      A[(size_t)i * n + j] = s / d;
    }
  }
  return 0;
}

static void cholesky_solve(int n, const double* L, double* b) {
  for (int i = 0; i < n; ++i) { /* L y = b */
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * b[k];
    b[i] = s / L[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) { /* L^T x = y */
    double s = b[i];
    for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * b[k];
    b[i] = s / L[(size_t)i * n + i];
  }
}

/* inverse of a symmetric positive definite 3x3 through its Cholesky factor */
static int spd3_inverse(const double V[9], double Vi[9]) {
  double L[9];
  memcpy(L, V, sizeof(L));
  if (cholesky(3, L)) return -1;
  for (int c = 0; c < 3; ++c) {
    double e[3] = {0.0, 0.0, 0.0};
    e[c] = 1.0;
    cholesky_solve(3, L, e);
    for (int r = 0; r < 3; ++r) Vi[3 * r + c] = e[r];
  }
  return 0;
}

static double clamp_diag(double v) {
  if (v < ORC_DIAG_MIN) return ORC_DIAG_MIN;
  if (v > ORC_DIAG_MAX) return ORC_DIAG_MAX;
  return v;
}

/* observation order sorted by (point, camera): stable counting sort */
static int* sorted_obs(const orc_problem* P) {
  int* cnt = (int*)calloc((size_t)P->n_pts + 1, sizeof(int));
  int* order = (int*)malloc(sizeof(int) * (size_t)(P->n_obs > 0 ? P->n_obs : 1));
  for (int i = 0; i < P->n_obs; ++i) cnt[P->obs_pt[i] + 1]++;
  for (int j = 0; j < P->n_pts; ++j) cnt[j + 1] += cnt[j];
  for (int i = 0; i < P->n_obs; ++i) order[cnt[P->obs_pt[i]]++] = i;
  /* within a point, order by camera (insertion sort: tracks are short) */
  int s = 0;
  for (int j = 0; j < P->n_pts; ++j) {
    int e = cnt[j];
    for (int a = s + 1; a < e; ++a) {
      int v = order[a], b = a - 1;
      while (b >= s && P->obs_cam[order[b]] > P->obs_cam[v]) { order[b + 1] = order[b]; --b; }
      order[b + 1] = v;
    }
    s = e;
  }
  free(cnt);
  return order;
}

/* ------------------------------------------------------------------ */
/* damped Gauss-Newton step by the Schur complement                    */
/*                                                                    */
/* H = J^T J with blocks U (6x6 per free camera), V (3x3 per point),   */
/* W (6x3 per observation of a free camera); g = -J^T r.  Damping      */
/* H* = H + mu D, D = clamp(diag H, 1e-6, 1e32).  Eliminating the      */
/* points: S = U* - W V*^-1 W^T, rhs = g_c - W V*^-1 g_p,              */
/* S dc = rhs, dX_j = V*_j^-1 (g_p,j - sum_k W_kj^T dc_k).             */
/* ------------------------------------------------------------------ */

int orc_solve_damped(const orc_problem* P, const double* R, const double* T, const double* X, double mu,
                     double* dc, double* dp, double* gc_out, double* gp_out, double* Dc_out,
                     double* Dp_out) {
  int nc = P->n_cams, np = P->n_pts;
  int* free_idx = (int*)malloc(sizeof(int) * (size_t)nc);
  int nf = 0;
  for (int k = 0; k < nc; ++k) free_idx[k] = P->fixed[k] ? -1 : nf++;
  int n = 6 * nf;
  double* U = (double*)calloc((size_t)nc * 36, sizeof(double));
  double* gc = (double*)calloc((size_t)nc * 6, sizeof(double));
  double* V = (double*)calloc((size_t)np * 9, sizeof(double));
  double* gp = (double*)calloc((size_t)np * 3, sizeof(double));
  double* W = (double*)calloc((size_t)(P->n_obs > 0 ? P->n_obs : 1) * 18, sizeof(double));
  int* order = sorted_obs(P);

  /* accumulate the blocks over observations in (point, camera) order */
  for (int t = 0; t < P->n_obs; ++t) {
    int i = order[t];
    int k = P->obs_cam[i], j = P->obs_pt[i];
    double r[2], Jc[12], Jp[6];
    orc_linearize_obs(P, R, T, X, i, r, Jc, Jp, NULL);
    for (int a = 0; a < 3; ++a) {
      for (int b = 0; b < 3; ++b) V[9 * j + 3 * a + b] += Jp[a] * Jp[b] + Jp[3 + a] * Jp[3 + b];
      gp[3 * j + a] -= Jp[a] * r[0] + Jp[3 + a] * r[1];
    }
    if (free_idx[k] >= 0) {
      for (int a = 0; a < 6; ++a) {
        for (int b = 0; b < 6; ++b) U[36 * k + 6 * a + b] += Jc[a] * Jc[b] + Jc[6 + a] * Jc[6 + b];
        gc[6 * k + a] -= Jc[a] * r[0] + Jc[6 + a] * r[1];
        for (int b = 0; b < 3; ++b) W[18 * i + 3 * a + b] = Jc[a] * Jp[b] + Jc[6 + a] * Jp[3 + b];
      }
    }
  }
  /* the pose priors of the free cameras */
  for (int k = 0; k < nc; ++k) {
    if (free_idx[k] < 0) continue;
    double r[6], J[36];
    orc_linearize_prior(P, R, T, k, r, J);
    for (int a = 0; a < 6; ++a) {
      for (int b = 0; b < 6; ++b) {
        double s = 0.0;
        for (int c = 0; c < 6; ++c) s += J[6 * c + a] * J[6 * c + b];
        U[36 * k + 6 * a + b] += s;
      }
      double s = 0.0;
      for (int c = 0; c < 6; ++c) s += J[6 * c + a] * r[c];
      gc[6 * k + a] -= s;
    }
  }

  /* damping */
  double* Dc = (double*)calloc((size_t)nc * 6, sizeof(double));
  double* Dp = (double*)calloc((size_t)np * 3, sizeof(double));
  for (int k = 0; k < nc; ++k) {
    if (free_idx[k] < 0) continue;
    for (int a = 0; a < 6; ++a) Dc[6 * k + a] = clamp_diag(U[36 * k + 7 * a]);
  }
  for (int j = 0; j < np; ++j)
    for (int a = 0; a < 3; ++a) Dp[3 * j + a] = clamp_diag(V[9 * j + 4 * a]);

  /* reduced camera system */
  double* S = (double*)calloc((size_t)(n > 0 ? n : 1) * (n > 0 ? n : 1), sizeof(double));
  double* rhs = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  double* Vinv = (double*)calloc((size_t)np * 9, sizeof(double));
  int status = 0;
  for (int k = 0; k < nc; ++k) {
    int fk = free_idx[k];
    if (fk < 0) continue;
    for (int a = 0; a < 6; ++a) {
      for (int b = 0; b < 6; ++b) S[(size_t)(6 * fk + a) * n + 6 * fk + b] = U[36 * k + 6 * a + b];
      S[(size_t)(6 * fk + a) * n + 6 * fk + a] += mu * Dc[6 * k + a];
      rhs[6 * fk + a] = gc[6 * k + a];
    }
  }
  int t0 = 0;
  for (int j = 0; j < np; ++j) {
    int t1 = t0;
    while (t1 < P->n_obs && P->obs_pt[order[t1]] == j) ++t1;
    double Vs[9];
    memcpy(Vs, V + 9 * j, sizeof(Vs));
    for (int a = 0; a < 3; ++a) Vs[4 * a] += mu * Dp[3 * j + a];
    if (spd3_inverse(Vs, Vinv + 9 * j)) status = ORC_ERR_NOT_PD;
    const double* Vi = Vinv + 9 * j;
    for (int ta = t0; ta < t1; ++ta) {
      int ia = order[ta], ka = P->obs_cam[ia], fa = free_idx[ka];
      if (fa < 0) continue;
      double Y[18]; /* Y = W_a V*^-1 */
      for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 3; ++b) {
          double s = 0.0;
          for (int c = 0; c < 3; ++c) s += W[18 * ia + 3 * a + c] * Vi[3 * c + b];
          Y[3 * a + b] = s;
        }
      for (int a = 0; a < 6; ++a) {
        double s = 0.0;
        for (int c = 0; c < 3; ++c) s += Y[3 * a + c] * gp[3 * j + c];
        rhs[6 * fa + a] -= s;
      }
      for (int tb = t0; tb < t1; ++tb) {
        int ib = order[tb], kb = P->obs_cam[ib], fb = free_idx[kb];
        if (fb < 0) continue;
        for (int a = 0; a < 6; ++a)
          for (int b = 0; b < 6; ++b) {
            double s = 0.0;
            for (int c = 0; c < 3; ++c) s += Y[3 * a + c] * W[18 * ib + 3 * b + c];
            S[(size_t)(6 * fa + a) * n + 6 * fb + b] -= s;
          }
      }
    }
    t0 = t1;
  }

  if (status == 0 && n > 0 && cholesky(n, S)) status = ORC_ERR_NOT_PD;
  if (status == 0 && n > 0) cholesky_solve(n, S, rhs);

  /* camera steps (fixed cameras do not move) */
  for (int k = 0; k < nc; ++k)
    for (int a = 0; a < 6; ++a) dc[6 * k + a] = (status == 0 && free_idx[k] >= 0) ? rhs[6 * free_idx[k] + a] : 0.0;

  /* back-substitution for the points */
  t0 = 0;
  for (int j = 0; j < np; ++j) {
    int t1 = t0;
    while (t1 < P->n_obs && P->obs_pt[order[t1]] == j) ++t1;
    double b[3] = {gp[3 * j], gp[3 * j + 1], gp[3 * j + 2]};
    for (int ta = t0; ta < t1; ++ta) {
      int ia = order[ta], ka = P->obs_cam[ia];
      if (free_idx[ka] < 0) continue;
      for (int c = 0; c < 3; ++c) {
        double s = 0.0;
        for (int a = 0; a < 6; ++a) s += W[18 * ia + 3 * a + c] * dc[6 * ka + a];
        b[c] -= s;
      }
    }
    for (int a = 0; a < 3; ++a) {
      double s = 0.0;
      for (int c = 0; c < 3; ++c) s += Vinv[9 * j + 3 * a + c] * b[c];
      dp[3 * j + a] = status == 0 ? s : 0.0;
    }
    t0 = t1;
  }

  if (gc_out) memcpy(gc_out, gc, sizeof(double) * 6 * (size_t)nc);
  if (gp_out) memcpy(gp_out, gp, sizeof(double) * 3 * (size_t)np);
  if (Dc_out) memcpy(Dc_out, Dc, sizeof(double) * 6 * (size_t)nc);
  if (Dp_out) memcpy(Dp_out, Dp, sizeof(double) * 3 * (size_t)np);
  free(free_idx); free(U); free(gc); free(V); free(gp); free(W); free(order);
  free(Dc); free(Dp); free(S); free(rhs); free(Vinv);
  return status;
}

/* retraction x (+) delta */
void orc_apply_step(const orc_problem* P, const double* R, const double* T, const double* X, const double* dc,
                    const double* dp, double* Rn, double* Tn, double* Xn) {
  for (int k = 0; k < P->n_cams; ++k) {
    double E[9];
    orc_so3_exp(dc + 6 * k, E);
    mat3_mul(R + 9 * k, E, Rn + 9 * k);
    for (int a = 0; a < 3; ++a) Tn[3 * k + a] = T[3 * k + a] + dc[6 * k + 3 + a];
  }
  for (int j = 0; j < P->n_pts; ++j)
    for (int a = 0; a < 3; ++a) Xn[3 * j + a] = X[3 * j + a] + dp[3 * j + a];
}

/* ------------------------------------------------------------------ */
/* one LM iteration                                                    */
/*   pred = 1/2 delta^T (mu D delta + g)                               */
/*   gain = (F(x) - F(x+)) / pred; accept when gain > 0 and pred > 0   */
/*   accept: mu *= max(1/3, 1 - (2 gain - 1)^3), nu = 2                */
/*   reject: mu *= nu, nu *= 2                                         */
/* ------------------------------------------------------------------ */

int orc_lm_step(const orc_problem* P, double* R, double* T, double* X, double* mu, double* nu,
                orc_step_info* info) {
  int nc = P->n_cams, np = P->n_pts;
  double* dc = (double*)calloc((size_t)nc * 6, sizeof(double));
  double* dp = (double*)calloc((size_t)np * 3 + 1, sizeof(double));
  double* gc = (double*)calloc((size_t)nc * 6, sizeof(double));
  double* gp = (double*)calloc((size_t)np * 3 + 1, sizeof(double));
  double* Dc = (double*)calloc((size_t)nc * 6, sizeof(double));
  double* Dp = (double*)calloc((size_t)np * 3 + 1, sizeof(double));
  double* Rn = (double*)malloc(sizeof(double) * 9 * (size_t)nc);
  double* Tn = (double*)malloc(sizeof(double) * 3 * (size_t)nc);
  double* Xn = (double*)malloc(sizeof(double) * (3 * (size_t)np + 1));

  double F = orc_cost(P, R, T, X);
  int status = orc_solve_damped(P, R, T, X, *mu, dc, dp, gc, gp, Dc, Dp);
  double pred = 0.0, Fn = F;
  int accepted = 0;
  double gain = 0.0;
  if (status == 0) {
    for (int k = 0; k < nc; ++k)
      for (int a = 0; a < 6; ++a) pred += dc[6 * k + a] * (*mu * Dc[6 * k + a] * dc[6 * k + a] + gc[6 * k + a]);
    for (int j = 0; j < np; ++j)
      for (int a = 0; a < 3; ++a) pred += dp[3 * j + a] * (*mu * Dp[3 * j + a] * dp[3 * j + a] + gp[3 * j + a]);
    pred *= 0.5;
    orc_apply_step(P, R, T, X, dc, dp, Rn, Tn, Xn);
    Fn = orc_cost(P, Rn, Tn, Xn);
    gain = pred > 0.0 ? (F - Fn) / pred : 0.0;
    accepted = (pred > 0.0 && gain > 0.0);
  }
  double mu_before = *mu;
  if (accepted) {
    memcpy(R, Rn, sizeof(double) * 9 * (size_t)nc);
    memcpy(T, Tn, sizeof(double) * 3 * (size_t)nc);
    memcpy(X, Xn, sizeof(double) * 3 * (size_t)np);
    double t = 2.0 * gain - 1.0;
    double f = 1.0 - t * t * t;
    *mu *= (f > 1.0 / 3.0) ? f : 1.0 / 3.0;
    *nu = 2.0;
  } else {
    *mu *= *nu;
    *nu *= 2.0;
  }
  if (info) {
    info->accepted = accepted;
    info->status = status;
    info->F = F;
    info->F_new = Fn;
    info->pred = pred;
    info->gain = gain;
    info->mu_used = mu_before;
    info->mu = *mu;
    info->nu = *nu;
  }
  free(dc); free(dp); free(gc); free(gp); free(Dc); free(Dp); free(Rn); free(Tn); free(Xn);
  return status;
}

int orc_lm_run(const orc_problem* P, double* R, double* T, double* X, int iters, double mu0,
               orc_step_info* trace) {
  double mu = mu0, nu = 2.0;
  int last = 0;
  for (int it = 0; it < iters; ++it) last = orc_lm_step(P, R, T, X, &mu, &nu, trace ? trace + it : NULL);
  return last;
}

/* Cluster transition, Sec. 3.2 Eq. 8: an overlap image adjusted in both the
 * previous and the new cluster takes the weighted average of its two poses,
 * weights in proportion to its feature matches (observations) in each.
 * Position: the weighted arithmetic mean.  Orientation: the weighted mean on
 * SO(3), which for two rotations is the point at fraction
 * t = w_new / (w_old + w_new) along the geodesic from R_old to R_new:
 * R_old Exp(t Log(R_old^T R_new)). */
void orc_transition(const double R_old[9], const double T_old[3], double w_old, const double R_new[9],
                    const double T_new[3], double w_new, double R_out[9], double T_out[3]) {
  const double t = w_new / (w_old + w_new);
  double E[9], phi[3], D[9];
  for (int i = 0; i < 3; ++i)  /* E = R_old^T R_new */
    for (int j = 0; j < 3; ++j)
      E[3 * i + j] = R_old[i] * R_new[j] + R_old[3 + i] * R_new[3 + j] + R_old[6 + i] * R_new[6 + j];
  orc_so3_log(E, phi);
  for (int i = 0; i < 3; ++i) phi[i] *= t;
  orc_so3_exp(phi, D);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      R_out[3 * i + j] = R_old[3 * i] * D[j] + R_old[3 * i + 1] * D[3 + j] + R_old[3 * i + 2] * D[6 + j];
  for (int i = 0; i < 3; ++i) T_out[i] = (w_old * T_old[i] + w_new * T_new[i]) / (w_old + w_new);
}

/* ---- Image footprints on a DSM (Sec. 3.1) and their overlap (Sec. 3.1 cross-strip
 * detection, Sec. 3.2 cluster formation). ---- */

/* Height of the DSM at (x, y): bilinear interpolation of the raster, the
 * position clamped to the raster. */
double orc_dsm_height(const orc_dsm* D, double x, double y) {
  double fx = (x - D->x0) / D->dx, fy = (y - D->y0) / D->dy;
  if (fx < 0.0) fx = 0.0;
  if (fy < 0.0) fy = 0.0;
  if (fx > D->nx - 1) fx = D->nx - 1;
  if (fy > D->ny - 1) fy = D->ny - 1;
  int ix = (int)fx, iy = (int)fy;
  if (ix > D->nx - 2) ix = D->nx - 2;
  if (iy > D->ny - 2) iy = D->ny - 2;
  const double ax = fx - ix, ay = fy - iy;
  const double* h = D->h + (size_t)iy * D->nx + ix;
  const double h0 = h[0] * (1.0 - ax) + h[1] * ax;
  const double h1 = h[D->nx] * (1.0 - ax) + h[D->nx + 1] * ax;
  return h0 * (1.0 - ay) + h1 * ay;
}

/* Ground point of pixel (u, v): the ray from the camera centre T along
 * R [(u - cx)/f, (v - cy)/f, 1] (lens distortion not applied) meets the DSM
 * surface.  The ray is sampled from where it enters the raster's height range
 * to where it leaves it, in steps of at most half a raster cell horizontally
 * (ORC_DSM_MAX_STEPS at most); the first sample at or below the surface
 * brackets the crossing, which ORC_DSM_BISECT bisections refine.  Returns 0,
 * or -1 for a ray that does not point down. */
int orc_ray_dsm(const double intr[7], const double R[9], const double T[3], double u, double v, const orc_dsm* D,
                double hmin, double hmax, double P[3]) {
  const double a = (u - intr[1]) / intr[0], b = (v - intr[2]) / intr[0];
  double d[3];
  for (int i = 0; i < 3; ++i) d[i] = R[3 * i] * a + R[3 * i + 1] * b + R[3 * i + 2];
  if (!(d[2] < 0.0)) return -1;
  double t0 = (T[2] - hmax) / (-d[2]), t1 = (T[2] - hmin) / (-d[2]);
  if (t0 < 0.0) t0 = 0.0;
  const double dxy = sqrt(d[0] * d[0] + d[1] * d[1]);
  const double cell = D->dx < D->dy ? D->dx : D->dy;
  int n = 1;
  if (dxy > 0.0) {
    const double steps = ceil((t1 - t0) * dxy / (0.5 * cell));
    n = steps < 1.0 ? 1 : (steps > ORC_DSM_MAX_STEPS ? ORC_DSM_MAX_STEPS : (int)steps);
  }
  double lo = t0, hi = t1;
  for (int i = 1; i <= n; ++i) {
    const double t = t0 + (t1 - t0) * i / n;
    const double g = T[2] + t * d[2] - orc_dsm_height(D, T[0] + t * d[0], T[1] + t * d[1]);
    if (g <= 0.0) {
      hi = t;
      lo = t0 + (t1 - t0) * (i - 1) / n;
      break;
    }
  }
  for (int it = 0; it < ORC_DSM_BISECT; ++it) {
    const double t = 0.5 * (lo + hi);
    const double g = T[2] + t * d[2] - orc_dsm_height(D, T[0] + t * d[0], T[1] + t * d[1]);
    if (g <= 0.0) hi = t; else lo = t;
  }
  for (int i = 0; i < 3; ++i) P[i] = T[i] + hi * d[i];
  return 0;
}

/* Footprint of an image of width x height pixels: the ground points of its
 * four corners (0,0), (w,0), (w,h), (0,h), as corners[4][3]. */
int orc_footprint(const double intr[7], double width, double height, const double R[9], const double T[3],
                  const orc_dsm* D, double corners[12]) {
  double hmin = D->h[0], hmax = D->h[0];
  for (size_t i = 0; i < (size_t)D->nx * D->ny; ++i) {
    if (D->h[i] < hmin) hmin = D->h[i];
    if (D->h[i] > hmax) hmax = D->h[i];
  }
  const double uv[4][2] = {{0.0, 0.0}, {width, 0.0}, {width, height}, {0.0, height}};
  for (int c = 0; c < 4; ++c)
    if (orc_ray_dsm(intr, R, T, uv[c][0], uv[c][1], D, hmin, hmax, corners + 3 * c) != 0) return -1;
  return 0;
}

/* signed area of a polygon (x, y pairs) */
static double poly_area(const double* p, int n) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) {
    const int j = (i + 1) % n;
    s += p[2 * i] * p[2 * j + 1] - p[2 * j] * p[2 * i + 1];
  }
  return 0.5 * s;
}

/* Area of the intersection of two convex quadrilaterals in the ground plane
 * (x, y of the footprint corners, any orientation): Sutherland-Hodgman
 * clipping of one by the other, then the shoelace formula. */
double orc_quad_overlap(const double qa[12], const double qb[12]) {
  double A[8], B[8];
  for (int i = 0; i < 4; ++i) {
    A[2 * i] = qa[3 * i]; A[2 * i + 1] = qa[3 * i + 1];
    B[2 * i] = qb[3 * i]; B[2 * i + 1] = qb[3 * i + 1];
  }
  const double sb = poly_area(B, 4) >= 0.0 ? 1.0 : -1.0;  /* orientation of the clipper */
  double P[32], Q[32];
  int np = 4;
  for (int i = 0; i < 8; ++i) P[i] = A[i];
  for (int e = 0; e < 4 && np > 0; ++e) {
    const double ex = B[2 * e], ey = B[2 * e + 1];
    const double fx = B[2 * ((e + 1) % 4)], fy = B[2 * ((e + 1) % 4) + 1];
    int nq = 0;
    for (int i = 0; i < np; ++i) {
      const double* s = P + 2 * i;
      const double* t = P + 2 * ((i + 1) % np);
      const double ds = sb * ((fx - ex) * (s[1] - ey) - (fy - ey) * (s[0] - ex));
      const double dt = sb * ((fx - ex) * (t[1] - ey) - (fy - ey) * (t[0] - ex));
      if (ds >= 0.0) { Q[2 * nq] = s[0]; Q[2 * nq + 1] = s[1]; ++nq; }
      if ((ds >= 0.0) != (dt >= 0.0)) {
        const double w = ds / (ds - dt);
        Q[2 * nq] = s[0] + w * (t[0] - s[0]);
        Q[2 * nq + 1] = s[1] + w * (t[1] - s[1]);
        ++nq;
      }
    }
    np = nq;
    for (int i = 0; i < 2 * np; ++i) P[i] = Q[i];
  }
  return np >= 3 ? fabs(poly_area(P, np)) : 0.0;
}

double orc_quad_area(const double q[12]) {
  double A[8];
  for (int i = 0; i < 4; ++i) { A[2 * i] = q[3 * i]; A[2 * i + 1] = q[3 * i + 1]; }
  return fabs(poly_area(A, 4));
}

/* ---- Patch transfer (Sec. 3.1, Eq. 3 and Eq. 4). ---- */

/* Eq. 3, written as it reads: X = T_0 + lambda R_0 K_0^-1 [u v 1]^T, then
 * pi(K_k R_k^T (X - T_k)) with pi(x, y, z) = (x / z, y / z).  K has no
 * distortion term in Eq. 3, so none is applied. */
int orc_patch_transfer_poses(const double intr0[7], const double R0[9], const double T0[3], const double p0[2],
                             double lambda, const double intrk[7], const double Rk[9], const double Tk[3],
                             double pk[2]) {
  /* K_0^-1 p_bar: K = [f 0 cx; 0 f cy; 0 0 1] */
  const double ray[3] = {(p0[0] - intr0[1]) / intr0[0], (p0[1] - intr0[2]) / intr0[0], 1.0};
  double X[3], d[3], xc[3], h[3];
  for (int i = 0; i < 3; ++i) X[i] = T0[i] + lambda * (R0[3 * i] * ray[0] + R0[3 * i + 1] * ray[1] + R0[3 * i + 2] * ray[2]);
  for (int i = 0; i < 3; ++i) d[i] = X[i] - Tk[i];
  for (int i = 0; i < 3; ++i) xc[i] = Rk[i] * d[0] + Rk[3 + i] * d[1] + Rk[6 + i] * d[2]; /* R_k^T (X - T_k) */
  if (!(xc[2] > 0.0)) return 0;
  h[0] = intrk[0] * xc[0] + intrk[1] * xc[2]; /* K_k x_c */
  h[1] = intrk[0] * xc[1] + intrk[2] * xc[2];
  h[2] = xc[2];
  pk[0] = h[0] / h[2];
  pk[1] = h[1] / h[2];
  return 1;
}

/* Eq. 4 with R(theta) = [cos(theta) sin(-theta); sin(theta) cos(theta)]. */
void orc_patch_transfer_planar(const double q0[2], const double c[2], double theta, const double g0[2],
                               const double gk[2], double qk[2]) {
  const double a = cos(theta), b = sin(theta);
  const double dx = q0[0] - c[0], dy = q0[1] - c[1];
  qk[0] = (a * dx - b * dy) + c[0] + gk[0] - g0[0];
  qk[1] = (b * dx + a * dy) + c[1] + gk[1] - g0[1];
}
