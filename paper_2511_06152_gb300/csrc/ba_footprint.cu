// Image footprints on a DSM and their overlaps (Sec. 3.1: the four image
// corners projected onto the surface model; cross-strip overlap detection by
// comparing projected footprints, used to form the clusters of Sec. 3.2).
//
//   k_footprint  one thread per (image, corner): the ray from the camera
//                centre through the corner pixel (no lens distortion) is
//                sampled from where it enters the DSM's height range, in
//                steps of at most half a raster cell horizontally; the first
//                sample at or below the bilinear surface brackets the first
//                hit, refined by a fixed number of bisections.  Binary64.
//   k_overlap    one thread per (footprint a, footprint b): area of the
//                intersection of the two convex ground quadrilaterals by
//                Sutherland-Hodgman clipping and the shoelace formula.
#include <cuda_runtime.h>
#include <math.h>

#include "ba_internal.h"

namespace bagpu {

namespace {

__device__ double dsm_height(const DsmView& D, double x, double y) {
  double fx = (x - D.x0) / D.dx, fy = (y - D.y0) / D.dy;
  fx = fmin(fmax(fx, 0.0), (double)(D.nx - 1));
  fy = fmin(fmax(fy, 0.0), (double)(D.ny - 1));
  int ix = (int)fx, iy = (int)fy;
  ix = min(ix, D.nx - 2);
  iy = min(iy, D.ny - 2);
  const double ax = fx - ix, ay = fy - iy;
  const double* h = D.h + (size_t)iy * D.nx + ix;
  const double h0 = h[0] * (1.0 - ax) + h[1] * ax;
  const double h1 = h[D.nx] * (1.0 - ax) + h[D.nx + 1] * ax;
  return h0 * (1.0 - ay) + h1 * ay;
}

__global__ void k_footprint(int n, const double* intr, double width, double height, const double* R,
                            const double* T, DsmView D, double* corners) {
  for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < 4 * n; id += gridDim.x * blockDim.x) {
    const int k = id >> 2, c = id & 3;
    const double* in = intr + 7 * k;
    const double* Rk = R + 9 * k;
    const double* Tk = T + 3 * k;
    const double u = (c == 1 || c == 2) ? width : 0.0, v = (c >= 2) ? height : 0.0;
    const double a = (u - in[1]) / in[0], b = (v - in[2]) / in[0];
    double d[3];
    for (int i = 0; i < 3; ++i) d[i] = Rk[3 * i] * a + Rk[3 * i + 1] * b + Rk[3 * i + 2];
    double* P = corners + 3 * id;
    if (!(d[2] < 0.0)) {  // the ray does not point down
      P[0] = P[1] = P[2] = nan("");
      continue;
    }
    double t0 = (Tk[2] - D.hmax) / (-d[2]);
    const double t1 = (Tk[2] - D.hmin) / (-d[2]);
    if (t0 < 0.0) t0 = 0.0;
    const double dxy = sqrt(d[0] * d[0] + d[1] * d[1]);
    const double cell = fmin(D.dx, D.dy);
    int m = 1;
    if (dxy > 0.0) {
      const double steps = ceil((t1 - t0) * dxy / (0.5 * cell));
      m = steps < 1.0 ? 1 : (steps > (double)kDsmMaxSteps ? kDsmMaxSteps : (int)steps);
    }
    double lo = t0, hi = t1;
    for (int i = 1; i <= m; ++i) {
      const double t = t0 + (t1 - t0) * i / m;
      const double g = Tk[2] + t * d[2] - dsm_height(D, Tk[0] + t * d[0], Tk[1] + t * d[1]);
      if (g <= 0.0) {
        hi = t;
        lo = t0 + (t1 - t0) * (i - 1) / m;
        break;
      }
    }
    for (int it = 0; it < kDsmBisect; ++it) {
      const double t = 0.5 * (lo + hi);
      const double g = Tk[2] + t * d[2] - dsm_height(D, Tk[0] + t * d[0], Tk[1] + t * d[1]);
      if (g <= 0.0) hi = t; else lo = t;
    }
    for (int i = 0; i < 3; ++i) P[i] = Tk[i] + hi * d[i];
  }
}

__device__ double poly_area2(const double* p, int n) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) {
    const int j = (i + 1 == n) ? 0 : i + 1;
    s += p[2 * i] * p[2 * j + 1] - p[2 * j] * p[2 * i + 1];
  }
  return 0.5 * s;
}

__global__ void k_overlap(int na, const double* qa, int nb, const double* qb, double* area) {
  for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < na * nb; id += gridDim.x * blockDim.x) {
    const int ia = id / nb, ib = id - ia * nb;
    const double* A = qa + 12 * ia;
    const double* B = qb + 12 * ib;
    double Bx[8];
    for (int i = 0; i < 4; ++i) {
      Bx[2 * i] = B[3 * i];
      Bx[2 * i + 1] = B[3 * i + 1];
    }
    const double sb = poly_area2(Bx, 4) >= 0.0 ? 1.0 : -1.0;  // orientation of the clipper
    double P[16], Q[16];  // a convex quadrilateral clipped by four half-planes has at most 8 vertices
    int np = 4;
    for (int i = 0; i < 4; ++i) {
      P[2 * i] = A[3 * i];
      P[2 * i + 1] = A[3 * i + 1];
    }
    for (int e = 0; e < 4 && np > 0; ++e) {
      const double ex = Bx[2 * e], ey = Bx[2 * e + 1];
      const double fx = Bx[2 * ((e + 1) & 3)], fy = Bx[2 * ((e + 1) & 3) + 1];
      int nq = 0;
      for (int i = 0; i < np; ++i) {
        const double* s = P + 2 * i;
        const double* t = P + 2 * ((i + 1 == np) ? 0 : i + 1);
        const double ds = sb * ((fx - ex) * (s[1] - ey) - (fy - ey) * (s[0] - ex));
        const double dt = sb * ((fx - ex) * (t[1] - ey) - (fy - ey) * (t[0] - ex));
        if (ds >= 0.0 && nq < 8) {
          Q[2 * nq] = s[0];
          Q[2 * nq + 1] = s[1];
          ++nq;
        }
        if ((ds >= 0.0) != (dt >= 0.0) && nq < 8) {
          const double w = ds / (ds - dt);
          Q[2 * nq] = s[0] + w * (t[0] - s[0]);
          Q[2 * nq + 1] = s[1] + w * (t[1] - s[1]);
          ++nq;
        }
      }
      np = nq;
      for (int i = 0; i < 2 * np; ++i) P[i] = Q[i];
    }
    area[id] = np >= 3 ? fabs(poly_area2(P, np)) : 0.0;
  }
}

int grid_of(int items, int per) {
  const int g = (items + per - 1) / per, cap = num_sms() * 8;
  return g < 1 ? 1 : (g > cap ? cap : g);
}

}  // namespace

void launch_footprints(int n, const double* intr, double width, double height, const double* R, const double* T,
                       const DsmView& D, double* corners, cudaStream_t st) {
  LAUNCH(KK_OTHER, st, k_footprint<<<grid_of(4 * n, 128), 128, 0, st>>>(n, intr, width, height, R, T, D, corners));
}

void launch_overlaps(int na, const double* qa, int nb, const double* qb, double* area, cudaStream_t st) {
  LAUNCH(KK_OTHER, st, k_overlap<<<grid_of(na * nb, 128), 128, 0, st>>>(na, qa, nb, qb, area));
}

}  // namespace bagpu
