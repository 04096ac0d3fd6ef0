/*
 * Plain FP64 CPU oracle for the local bundle-adjustment LM iteration.
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the
 * benchmark's CPU-baseline leg, never by the CUDA library.
 *
 * Arrays are row-major FP64 in caller-owned host memory:
 *   intr     [n_cams][7]  f, cx, cy, k1, k2, p1, p2 (pixels; Brown terms on
 *                         normalised coordinates)
 *   R        [n_cams][9]  camera->world rotation (Eq. 5 uses R^T)
 *   T        [n_cams][3]  camera centre, local ENU metres
 *   X        [n_pts][3]   points, local ENU metres
 *   R_prior, T_prior      IMU attitude / GNSS position per camera
 *   fixed    [n_cams]     1 = pose held fixed (cluster overlap, Sec. 3.2)
 *   obs_cam, obs_pt, obs_uv[n_obs][2]  observations in pixels
 * sigma_gnss / sigma_imu of 0 switch that prior off.
 */
#ifndef BA_ORACLE_H
#define BA_ORACLE_H

#define ORC_MIN_DEPTH 1e-6
#define ORC_DIAG_MIN 1e-6
#define ORC_DIAG_MAX 1e32
#define ORC_ERR_NOT_PD (-3)

typedef struct {
  int n_cams, n_pts, n_obs;
  const double* intr;
  const double* R_prior;
  const double* T_prior;
  const unsigned char* fixed;
  const int* obs_cam;
  const int* obs_pt;
  const double* obs_uv;
  double sigma_px, huber_delta, sigma_gnss, sigma_imu;
} orc_problem;

typedef struct {
  int accepted, status;
  double F, F_new, pred, gain, mu_used, mu, nu;
} orc_step_info;

void orc_so3_exp(const double w[3], double R[9]);
void orc_so3_log(const double R[9], double w[3]);
void orc_so3_jr_inv(const double w[3], double J[9]);
int orc_project(const double intr[7], const double R[9], const double T[3], const double X[3], double uv[2]);
double orc_huber_rho(double s, double delta);
double orc_huber_weight(double s, double delta);
int orc_linearize_obs(const orc_problem* P, const double* R, const double* T, const double* X, int i,
                      double r[2], double Jc[12], double Jp[6], double* s_out);
void orc_linearize_prior(const orc_problem* P, const double* R, const double* T, int k, double r[6],
                         double J[36]);
double orc_cost(const orc_problem* P, const double* R, const double* T, const double* X);
int orc_solve_damped(const orc_problem* P, const double* R, const double* T, const double* X, double mu,
                     double* dc, double* dp, double* gc_out, double* gp_out, double* Dc_out, double* Dp_out);
void orc_apply_step(const orc_problem* P, const double* R, const double* T, const double* X, const double* dc,
                    const double* dp, double* Rn, double* Tn, double* Xn);
int orc_lm_step(const orc_problem* P, double* R, double* T, double* X, double* mu, double* nu,
                orc_step_info* info);
int orc_lm_run(const orc_problem* P, double* R, double* T, double* X, int iters, double mu0,
               orc_step_info* trace);
/* DSM raster: heights h[iy * nx + ix] at (x0 + ix dx, y0 + iy dy), bilinear between nodes. */
typedef struct {
  int nx, ny;
  double x0, y0, dx, dy;
  const double* h;
} orc_dsm;

#define ORC_DSM_MAX_STEPS 100000
#define ORC_DSM_BISECT 60

double orc_dsm_height(const orc_dsm* D, double x, double y);
int orc_ray_dsm(const double intr[7], const double R[9], const double T[3], double u, double v, const orc_dsm* D,
                double hmin, double hmax, double P[3]);
int orc_footprint(const double intr[7], double width, double height, const double R[9], const double T[3],
                  const orc_dsm* D, double corners[12]);
double orc_quad_overlap(const double qa[12], const double qb[12]);
double orc_quad_area(const double q[12]);

/* Eq. 8: weighted pose average of an overlap image (weights w_old, w_new > 0). */
void orc_transition(const double R_old[9], const double T_old[3], double w_old, const double R_new[9],
                    const double T_new[3], double w_new, double R_out[9], double T_out[3]);

/* Patch transfer (Sec. 3.1).  Eq. 3: the centre p0 (pixels) of a patch of
 * image 0 moved to image k through the poses, at depth lambda along image
 * 0's optical axis; K is the pinhole part of intr (f, cx, cy).  Returns 1
 * (and writes pk) when the point is in front of image k, else 0. */
int orc_patch_transfer_poses(const double intr0[7], const double R0[9], const double T0[3], const double p0[2],
                             double lambda, const double intrk[7], const double Rk[9], const double Tk[3],
                             double pk[2]);
/* Eq. 4: a patch centre q0 (ground plane) moved by the in-plane rotation
 * theta about the patch-grid centre c and the image-centre displacement
 * gk - g0. */
void orc_patch_transfer_planar(const double q0[2], const double c[2], double theta, const double g0[2],
                               const double gk[2], double qk[2]);

#endif
