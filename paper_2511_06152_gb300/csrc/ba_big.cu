// Reduced camera systems larger than one CTA's shared memory holds (more than
// kMaxFreeSmall free images, n = 6 n_free > 192; the 400-image large block
// has n = 2400), solved in global memory.  Same system and elimination order
// as the shared-memory solver of ba_kernels.cu: S assembled in binary64 in
// the reverse Cuthill-McKee order, Cholesky restricted to the envelope of S
// (no fill outside it), a solve, refinement steps against S in binary64.
//
//   k_big_prior   per free image: priors, damping D, g_c, rhs, diagonal block
//   k_big_pairs   off-diagonal blocks of S from the co-visible pairs' sums
//
// Factorisation on the tensor cores (default).  GB300 runs binary64 at about
// 1/59 of its binary32 rate, so the factor is kept as double-float (binary32
// pairs, ~48 bits) and its dense products run on the tcgen05 tensor cores as
// exact products of 8-bit digit matrices (ba_tc.cuh):
//   k_big_split      S -> F (lower triangle, double-float, zeros outside the envelope)
//   per block column k of kBigNB columns (right-looking):
//     k_big_panel      every CTA factors the diagonal block and inverts it
//                      (double-float); CTA 0 stores both, CTA b stores the
//                      panel L_ik = A_ik L_kk^-T of row block k + b and its
//                      Ozaki digits
//     k_big_update_tc  A_ij -= L_ik L_jk^T on 128 x 32 tiles inside the
//                      envelope: digit products on the tensor cores,
//                      double-float subtraction
//   k_big_solve_df   forward and backward substitution (one CTA, double-float,
//                    the inverted diagonal blocks and the panels)
//   k_big_resid      t = rhs - S x in binary64
//   k_big_finish     dc, candidate poses, pred and prior terms, status
//
// Binary64 factorisation on the CUDA cores (BA_FLAG_BIG_FP64_FACTOR):
//   (F = S)
//   per block column k:
//     k_big_diag    factor the diagonal block (one CTA)
//     k_big_trsm    L_ik = A_ik L_kk^-T for the row blocks inside the envelope
//     k_big_update  A_ij -= L_ik L_jk^T for the tiles inside the envelope
//   k_big_solve   forward and backward substitution (one CTA)
//   k_big_resid, k_big_finish
//
// The envelope is non-decreasing: row r's first nonzero column is
// ef(r) = 6 env_first[r / 6]; the rows of a column block that can be nonzero
// below it form one contiguous run of row blocks, whose length per block
// column the host passes in (it fixes the grid sizes).
#include <cuda_runtime.h>

#include <algorithm>

#include "ba_camera.cuh"
#include "ba_device.cuh"
#include "ba_internal.h"
#include "ba_tc.cuh"

namespace bagpu {

namespace {

__device__ __forceinline__ int ef_row(const DevCluster& C, int r) { return 6 * C.env_first[r / 6]; }

// last row (or column) c with ef_row(c) <= r: the envelope of S is symmetric
__device__ __forceinline__ int env_last(const DevCluster& C, int r) {
  const int nb = C.n_free;
  int lo = r / 6, hi = nb - 1;  // env_first[p] <= p, so block r / 6 qualifies
  const int lim = r / 6;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (C.env_first[mid] <= lim) lo = mid; else hi = mid - 1;
  }
  return 6 * lo + 5;
}

// per free image: JtJ and Jtr of its priors, D, g_c, rhs and its diagonal block of S
__global__ void k_big_prior(const DevCluster* dcl) {
  const DevCluster& C = *dcl;
  const LmState* lm = C.lm;
  const int nf = C.n_free, n = 6 * nf, cur = lm->cur;
  const double mu = lm->mu;
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
    const int k = C.cam_of_free[f], p = C.fpos[f];
    double JtJ[36], Jtr[6];
    prior_terms(C.R + (size_t)cur * C.n_cams * 9 + 9 * k, C.T + (size_t)cur * C.n_cams * 3 + 3 * k,
                C.R_prior + 9 * k, C.T_prior + 3 * k, C.sigma_imu, C.sigma_gnss, JtJ, Jtr);
    const double* cd = C.camsum + (size_t)kCamPart * f;
    int ui = 0;
    for (int a = 0; a < 6; ++a)
      for (int b = a; b < 6; ++b, ++ui) {
        double v = cd[ui] + JtJ[6 * a + b];
        if (a == b) {
          const double D = clamp_diag(cd[33 + a] + JtJ[7 * a]);
          v += mu * D;
          C.Dc[6 * f + a] = D;
        }
        C.S[(size_t)(6 * p + b) * n + 6 * p + a] = v;
        C.S[(size_t)(6 * p + a) * n + 6 * p + b] = v;
      }
    for (int a = 0; a < 6; ++a) {
      const double g = cd[21 + a] - Jtr[a];
      C.gc[6 * f + a] = g;
      C.rhs[6 * p + a] = g - cd[27 + a];
    }
  }
}

// S(a, b) = -sum Z_a Z_b^T for every co-visible pair, both triangles
__global__ void k_big_pairs(const DevCluster* dcl) {
  const DevCluster& C = *dcl;
  const int n = 6 * C.n_free;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < C.n_pairs * 36; idx += gridDim.x * blockDim.x) {
    const int p = idx / 36, e = idx - 36 * p;
    const int i = e / 6, c = e - 6 * i;
    const double v = -C.pairsum[(size_t)kPairPart * p + e];
    const int2 key = C.pair_key[p];
    const int ra = 6 * C.fpos[key.x] + i, rb = 6 * C.fpos[key.y] + c;
    C.S[(size_t)rb * n + ra] = v;
    C.S[(size_t)ra * n + rb] = v;
  }
}

// Factor the diagonal block of block column k (one CTA): right-looking, one
// column at a time, reciprocal square root pivots (kept in bx[3n + j]).
__global__ void __launch_bounds__(256) k_big_diag(const DevCluster* dcl, int k) {
  const DevCluster& C = *dcl;
  const int n = 6 * C.n_free, r0 = kBigNB * k, nb = min(kBigNB, n - r0);
  __shared__ double L[kBigNB][kBigNB + 1];
  __shared__ double s_inv;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < nb * nb; idx += blockDim.x) {
    const int r = idx / nb, c = idx - r * nb;
    L[r][c] = c <= r ? C.F[(size_t)(r0 + r) * n + r0 + c] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (tid == 0) {
      const double d = L[j][j];
      if (!(d > 0.0)) *C.bflag = 1;
      const double dd = d > 0.0 ? d : 1.0;
      const double inv = pivot_rsqrt(dd);
      L[j][j] = dd * inv;
      C.bx[3 * n + r0 + j] = inv;
      s_inv = inv;
    }
    __syncthreads();
    const double inv = s_inv;
    for (int r = j + 1 + tid; r < nb; r += blockDim.x) L[r][j] *= inv;
    __syncthreads();
    const int w = nb - j - 1;
    for (int idx = tid; idx < w * w; idx += blockDim.x) {
      const int r = j + 1 + idx / w, c = j + 1 + idx % w;
      if (c <= r) L[r][c] -= L[r][j] * L[c][j];
    }
    __syncthreads();
  }
  for (int idx = tid; idx < nb * nb; idx += blockDim.x) {
    const int r = idx / nb, c = idx - r * nb;
    if (c <= r) C.F[(size_t)(r0 + r) * n + r0 + c] = L[r][c];
  }
}

// Row blocks i = k + 1 + blockIdx.x: L_ik = A_ik L_kk^-T by column sweeps.
__global__ void __launch_bounds__(256) k_big_trsm(const DevCluster* dcl, int k) {
  const DevCluster& C = *dcl;
  const int n = 6 * C.n_free, c0 = kBigNB * k, nb = min(kBigNB, n - c0);
  const int r0 = kBigNB * (k + 1 + blockIdx.x), nr = min(kBigNB, n - r0);
  if (nr <= 0) return;
  __shared__ double Lk[kBigNB][kBigNB + 1];
  __shared__ double X[kBigNB][kBigNB + 1];
  const int tid = threadIdx.x;
  for (int idx = tid; idx < kBigNB * kBigNB; idx += blockDim.x) {
    const int r = idx / kBigNB, c = idx - r * kBigNB;
    Lk[r][c] = (r < nb && c <= r) ? C.F[(size_t)(c0 + r) * n + c0 + c] : 0.0;
    X[r][c] = (r < nr && c < nb) ? C.F[(size_t)(r0 + r) * n + c0 + c] : 0.0;
  }
  __shared__ double inv[kBigNB];
  for (int c = tid; c < nb; c += blockDim.x) inv[c] = C.bx[3 * n + c0 + c];
  __syncthreads();
  for (int c = 0; c < nb; ++c) {
    for (int r = tid; r < nr; r += blockDim.x) X[r][c] *= inv[c];
    __syncthreads();
    const int w = nb - c - 1;
    for (int idx = tid; idx < nr * w; idx += blockDim.x) {
      const int r = idx / w, cc = c + 1 + idx % w;
      X[r][cc] -= X[r][c] * Lk[cc][c];
    }
    __syncthreads();
  }
  for (int idx = tid; idx < nr * nb; idx += blockDim.x) {
    const int r = idx / nb, c = idx - r * nb;
    C.F[(size_t)(r0 + r) * n + c0 + c] = X[r][c];
  }
}

// Tiles (i, j), k < j <= i < k + 1 + m: A_ij -= L_ik L_jk^T, each tile as two
// CTAs of 16 rows (twice the CTAs of the step over twice the SMs).  Each
// thread computes two entries of a row.
constexpr int kHalf = kBigNB / 2;
__global__ void __launch_bounds__(256) k_big_update(const DevCluster* dcl, int k) {
  const DevCluster& C = *dcl;
  const int n = 6 * C.n_free, c0 = kBigNB * k, nb = min(kBigNB, n - c0);
  const int t = blockIdx.x >> 1, half = blockIdx.x & 1;
  int ii = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while ((ii + 1) * (ii + 2) / 2 <= t) ++ii;
  while (ii * (ii + 1) / 2 > t) --ii;
  const int jj = t - ii * (ii + 1) / 2;
  const int ri = kBigNB * (k + 1 + ii) + kHalf * half, rj = kBigNB * (k + 1 + jj);
  const int ni = min(kHalf, n - ri), nj = min(kBigNB, n - rj);
  if (ni <= 0 || nj <= 0) return;
  __shared__ double Li[kHalf][kBigNB + 1];
  __shared__ double Lj[kBigNB][kBigNB + 1];
  const int tid = threadIdx.x;
  for (int idx = tid; idx < kHalf * kBigNB; idx += blockDim.x) {
    const int r = idx / kBigNB, q = idx - r * kBigNB;
    Li[r][q] = (r < ni && q < nb) ? C.F[(size_t)(ri + r) * n + c0 + q] : 0.0;
  }
  for (int idx = tid; idx < kBigNB * kBigNB; idx += blockDim.x) {
    const int r = idx / kBigNB, q = idx - r * kBigNB;
    Lj[r][q] = (r < nj && q < nb) ? C.F[(size_t)(rj + r) * n + c0 + q] : 0.0;
  }
  __syncthreads();
  const int r = tid >> 4, cb = (tid & 15) * 2;
  double acc[2] = {0.0, 0.0};
  for (int q = 0; q < nb; ++q) {
    const double a = Li[r][q];
#pragma unroll
    for (int u = 0; u < 2; ++u) acc[u] += a * Lj[cb + u][q];
  }
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int c = cb + u;
    if (r < ni && c < nj && (ri - kHalf * half != rj || c <= r + kHalf * half))
      C.F[(size_t)(ri + r) * n + rj + c] -= acc[u];
  }
}

// Shared memory of the solve: v (n), the pivots' reciprocals (n), and the
// strictly lower triangle of the current diagonal block.
constexpr int kBlkLd = kBigNB + 1;
size_t big_solve_smem(int n) { return sizeof(double) * (2 * (size_t)n + (size_t)kBigNB * kBlkLd); }

// the strictly lower triangle of diagonal block r0 (nb rows) into blk (all threads)
__device__ __forceinline__ void stage_diag_block(const DevCluster& C, int n, int r0, int nb, double* blk) {
  for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
    const int r = idx / nb, c = idx - r * nb;
    blk[r * kBlkLd + c] = c < r ? C.F[(size_t)(r0 + r) * n + r0 + c] : 0.0;
  }
}

// Solve S y = v with the factor (one CTA; v and y in shared memory, y
// overwrites v).  Per block of kBigNB rows: the block's triangle is staged in
// shared memory and warp 0 sweeps it (lane = row), then one thread per row
// updates the rows inside the envelope with the block's columns.
__device__ void big_solve_cta(const DevCluster& C, double* v, double* inv, double* blk) {
  const int n = 6 * C.n_free, tid = threadIdx.x, bs = blockDim.x, lane = tid & 31, wid = tid >> 5;
  for (int i = tid; i < n; i += bs) inv[i] = C.bx[3 * n + i];
  const int nblk = (n + kBigNB - 1) / kBigNB;
  for (int k = 0; k < nblk; ++k) {  // L y = v
    const int r0 = kBigNB * k, nb = min(kBigNB, n - r0);
    stage_diag_block(C, n, r0, nb, blk);
    __syncthreads();
    if (wid == 0) {
      double y = lane < nb ? v[r0 + lane] : 0.0;
      for (int j = 0; j < nb; ++j) {
        const double yj = __shfl_sync(BA_FULL_MASK, y * inv[r0 + j], j);
        if (lane == j) y = yj;
        else if (lane > j && lane < nb) y -= blk[lane * kBlkLd + j] * yj;
      }
      if (lane < nb) v[r0 + lane] = y;
    }
    __syncthreads();
    const int last = min(n - 1, env_last(C, r0 + nb - 1));  // rows whose envelope reaches this block
    for (int i = r0 + nb + tid; i <= last; i += bs) {
      double s = 0.0;
      for (int q = max(r0, ef_row(C, i)); q < r0 + nb; ++q) s += C.F[(size_t)i * n + q] * v[q];
      v[i] -= s;
    }
    __syncthreads();
  }
  for (int k = nblk - 1; k >= 0; --k) {  // L^T x = y
    const int r0 = kBigNB * k, nb = min(kBigNB, n - r0);
    stage_diag_block(C, n, r0, nb, blk);
    __syncthreads();
    if (wid == 0) {
      double x = lane < nb ? v[r0 + lane] : 0.0;
      for (int j = nb - 1; j >= 0; --j) {
        const double xj = __shfl_sync(BA_FULL_MASK, x * inv[r0 + j], j);
        if (lane == j) x = xj;
        else if (lane < j) x -= blk[j * kBlkLd + lane] * xj;
      }
      if (lane < nb) v[r0 + lane] = x;
    }
    __syncthreads();
    for (int i = ef_row(C, r0) + tid; i < r0; i += bs) {  // columns of the block's rows
      double s = 0.0;
      for (int q = r0; q < r0 + nb; ++q)
        if (ef_row(C, q) <= i) s += C.F[(size_t)q * n + i] * v[q];
      v[i] -= s;
    }
    __syncthreads();
  }
}

// x = S^-1 rhs (mode 0), or x += S^-1 t (mode 1)
__global__ void __launch_bounds__(1024) k_big_solve(const DevCluster* dcl, int mode) {
  const DevCluster& C = *dcl;
  extern __shared__ double v[];
  const int n = 6 * C.n_free;
  const double* src = mode == 0 ? C.rhs : C.bx + 2 * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = src[i];
  big_solve_cta(C, v, v + n, v + 2 * n);
  double* x = C.bx + n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = mode == 0 ? v[i] : x[i] + v[i];
}

// t = rhs - S x over the envelope (warp per row)
__global__ void __launch_bounds__(256) k_big_resid(const DevCluster* dcl) {
  const DevCluster& C = *dcl;
  const int n = 6 * C.n_free, lane = threadIdx.x & 31;
  const double* x = C.bx + n;
  double* t = C.bx + 2 * n;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += (gridDim.x * blockDim.x) >> 5) {
    const int c1 = min(n - 1, env_last(C, r));
    double acc = 0.0;
    for (int c = ef_row(C, r) + lane; c <= c1; c += 32) acc += C.S[(size_t)r * n + c] * x[c];
    acc = warp_sum(acc);
    if (lane == 0) t[r] = C.rhs[r] - acc;
  }
}

// dc (free-image order), candidate poses, pred and prior terms, status
template <bool MIXED>
__global__ void __launch_bounds__(512) k_big_finish(const DevCluster* dcl) {
  const DevCluster& C = *dcl;
  LmState* lm = C.lm;
  const int n = 6 * C.n_free, tid = threadIdx.x;
  const bool fail = lm->pt_fail != 0 || *C.bflag != 0;
  const double* x = C.bx + n;
  for (int idx = tid; idx < n; idx += blockDim.x) {
    const double v = fail ? 0.0 : x[6 * C.fpos[idx / 6] + idx % 6];
    C.dc[idx] = v;
    if (MIXED) C.dc32[idx] = (float)v;
  }
  double pc = 0.0, pn = 0.0;
  for (int k = tid; k < C.n_cams; k += blockDim.x) {
    double a, b;
    candidate_camera<MIXED>(C, k, x, lm->mu, lm->cur, fail, &a, &b);
    pc += a;
    pn += b;
  }
  __shared__ double red[2][16];
  pc = warp_sum(pc);
  pn = warp_sum(pn);
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = pc;
    red[1][tid >> 5] = pn;
  }
  __syncthreads();
  if (tid == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      s0 += red[0][w];
      s1 += red[1][w];
    }
    lm->pred_cam = s0;
    lm->prior_new = s1;
    lm->status = lm->dev_error ? lm->dev_error : (fail ? BA_STATUS_NOT_PD : 0);
    lm->dev_error = 0;
    lm->tiles_done = 0;  // the back-substitution counts its tiles from here
    *C.bflag = 0;
  }
  __syncthreads();
  // a cluster without observations has no back-substitution tile to count:
  // its LM step is taken here
  if (C.n_tiles == 0 && lm->active && tid < 32) lm_update_warp<MIXED>(C, tid);
}

// ------------------------------------------------------------------ tensor-core factorisation

__device__ __forceinline__ float* df_hi(const DevCluster& C) { return reinterpret_cast<float*>(C.F); }
__device__ __forceinline__ float* df_lo(const DevCluster& C) {
  const int n = 6 * C.n_free;
  return reinterpret_cast<float*>(C.F) + (size_t)n * n;
}

// F = S on the lower triangle as double-float (entries outside the envelope
// are zero in S and become zero here), one CTA per row.
__global__ void __launch_bounds__(256) k_big_split(const DevCluster* dcl) {
  const DevCluster& C = *dcl;
  const int n = 6 * C.n_free;
  float* Fh = df_hi(C);
  float* Fl = df_lo(C);
  for (int r = blockIdx.x; r < n; r += gridDim.x) {
    const double* srow = C.S + (size_t)r * n;
    for (int c = threadIdx.x; c <= r; c += blockDim.x) {
      const double v = srow[c];
      float h = 0.0f, l = 0.0f;
      if (v != 0.0) {
        h = __double2float_rn(v);
        l = __double2float_rn(v - (double)h);
      }
      Fh[(size_t)r * n + c] = h;
      Fl[(size_t)r * n + c] = l;
    }
  }
}

constexpr int kPanelThreads = 1024;
constexpr int kPld = kBigNB + 1;  // padded leading dimension of the shared blocks

// Block column k: the diagonal block factored and inverted by every CTA
// (double-float; rows past n padded with the identity), then CTA 0 stores
// the factor and the inverse, CTA b (1 <= b <= m) the panel of row block
// k + b, L_ik = A_ik (L_kk^-1)^T, and its Ozaki digits and row scales.
//
// The factor and its inverse come out of one right-looking sweep: W starts
// as the identity and receives the same row operations as the matrix, so
// that row j of W, scaled by 1 / L(j, j) once the column j is final, is row
// j of L^-1 (forward substitution of L X = I, one row at a time).  Columns
// go in blocks of pw (a divisor of 32): one warp factors a block (the
// pivots' reciprocal square roots, the block's columns of L, its rows of X)
// with warp-level synchronisation only, then the whole CTA applies the
// block's rank-pw update below it: two block-wide barriers per block.
__global__ void __launch_bounds__(kPanelThreads) k_big_panel(const DevCluster* dcl, int k, int pw) {
  const DevCluster& C = *dcl;
  const int n = 6 * C.n_free, r0 = kBigNB * k, nb = min(kBigNB, n - r0);
  float* Fh = df_hi(C);
  float* Fl = df_lo(C);
  __shared__ float Lh[kBigNB][kPld], Ll[kBigNB][kPld];  // factor
  __shared__ float Wh[kBigNB][kPld], Wl[kBigNB][kPld];  // identity -> inverse of the factor
  __shared__ float Ph[kBigNB][kPld], Pl[kBigNB][kPld];  // A_ik
  const int tid = threadIdx.x;
  const int b = blockIdx.x;
  const int ri = r0 + kBigNB * b, nr = b == 0 ? nb : min(kBigNB, n - ri);
  for (int idx = tid; idx < kBigNB * kBigNB; idx += kPanelThreads) {
    const int r = idx >> 5, c = idx & 31;
    float h = 0.0f, l = 0.0f;
    if (r < nb && c < nb) {
      if (c <= r) {
        h = Fh[(size_t)(r0 + r) * n + r0 + c];
        l = Fl[(size_t)(r0 + r) * n + r0 + c];
      }
    } else if (r == c) {
      h = 1.0f;
    }
    Lh[r][c] = h;
    Ll[r][c] = l;
    Wh[r][c] = r == c ? 1.0f : 0.0f;
    Wl[r][c] = 0.0f;
    if (b > 0) {
      float ph = 0.0f, pl = 0.0f;
      if (r < nr && c < nb) {
        ph = Fh[(size_t)(ri + r) * n + r0 + c];
        pl = Fl[(size_t)(ri + r) * n + r0 + c];
      }
      Ph[r][c] = ph;
      Pl[r][c] = pl;
    }
  }
  __shared__ float Dh[kBigNB], Dl[kBigNB];  // L(j, j), kept apart until the sweep ends
  __syncthreads();
  bool fail = false;
  // blocks of pw columns: warp 0 factors the block's columns (lane = row,
  // warp-level synchronisation only) and finishes the block's rows of X;
  // then every thread applies the block's rank-pw update to the rows below
  // it (entry (tr, tc) of the trailing matrix, or of W left of it)
  const int tr = tid >> 5, tc = tid & 31, lane = tid & 31;
  for (int jb = 0; jb < kBigNB; jb += pw) {
    const int je = jb + pw - 1;  // last column of the block
    if (tid < 32) {
      for (int j = jb; j <= je; ++j) {
        dfl d{Lh[j][j], Ll[j][j]};
        if (!(d.hi > 0.0f)) {
          fail = true;
          d = dfl{1.0f, 0.0f};
        }
        const dfl iv = df_rsqrt(d);
        if (lane > j) {
          const dfl v = df_mul(dfl{Lh[lane][j], Ll[lane][j]}, iv);
          Lh[lane][j] = v.hi;
          Ll[lane][j] = v.lo;
        } else {
          if (lane == j) {
            const dfl sq = df_mul(d, iv);
            Dh[j] = sq.hi;
            Dl[j] = sq.lo;
          }
          const dfl x = df_mul(dfl{Wh[j][lane], Wl[j][lane]}, iv);  // row j of X
          Wh[j][lane] = x.hi;
          Wl[j][lane] = x.lo;
        }
        __syncwarp();
        if (lane > j) {  // the block's later columns, rows below j
          const dfl lr{Lh[lane][j], Ll[lane][j]};
          for (int c = j + 1; c <= je && c <= lane; ++c) {
            const dfl a = df_fms(dfl{Lh[lane][c], Ll[lane][c]}, lr, dfl{Lh[c][j], Ll[c][j]});
            Lh[lane][c] = a.hi;
            Ll[lane][c] = a.lo;
          }
        }
        if (lane <= j) {  // the block's later rows of W, column lane
          const dfl xj{Wh[j][lane], Wl[j][lane]};
          for (int r = j + 1; r <= je; ++r) {
            const dfl a = df_fms(dfl{Wh[r][lane], Wl[r][lane]}, dfl{Lh[r][j], Ll[r][j]}, xj);
            Wh[r][lane] = a.hi;
            Wl[r][lane] = a.lo;
          }
        }
        __syncwarp();
      }
    }
    __syncthreads();
    if (tr > je && tc <= tr) {
      if (tc <= je) {  // W(tr, tc) -= sum_j L(tr, j) X(j, tc) over the block's columns
        dfl a{Wh[tr][tc], Wl[tr][tc]};
        for (int i = 0; i < pw; ++i) {
          const int j = jb + i;
          if (j >= tc) a = df_fms(a, dfl{Lh[tr][j], Ll[tr][j]}, dfl{Wh[j][tc], Wl[j][tc]});
        }
        Wh[tr][tc] = a.hi;
        Wl[tr][tc] = a.lo;
      } else {  // L(tr, tc) -= sum_j L(tr, j) L(tc, j)
        dfl a{Lh[tr][tc], Ll[tr][tc]};
        for (int i = 0; i < pw; ++i) a = df_fms(a, dfl{Lh[tr][jb + i], Ll[tr][jb + i]}, dfl{Lh[tc][jb + i], Ll[tc][jb + i]});
        Lh[tr][tc] = a.hi;
        Ll[tr][tc] = a.lo;
      }
    }
    __syncthreads();
  }
  if (tid < kBigNB) {
    Lh[tid][tid] = Dh[tid];
    Ll[tid][tid] = Dl[tid];
  }
  __syncthreads();
  if (b == 0) {
    if (tid == 0 && fail) *C.bflag = 1;
    float* lv = C.linv + (size_t)k * 2 * kBigNB * kBigNB;
    for (int idx = tid; idx < kBigNB * kBigNB; idx += kPanelThreads) {
      const int r = idx >> 5, c = idx & 31;
      lv[idx] = Wh[r][c];
      lv[kBigNB * kBigNB + idx] = Wl[r][c];
      if (r < nb && c <= r) {
        Fh[(size_t)(r0 + r) * n + r0 + c] = Lh[r][c];
        Fl[(size_t)(r0 + r) * n + r0 + c] = Ll[r][c];
      }
    }
    return;
  }
  // the panel: L_ik(r, c) = sum_{q <= c} A_ik(r, q) X(c, q), thread (r, c)
  const int r = tid >> 5, c = tid & 31;
  Dot2 acc;
  for (int q = 0; q <= c; ++q) acc.add(dfl{Ph[r][q], Pl[r][q]}, dfl{Wh[c][q], Wl[c][q]});
  const dfl out = acc.get();
  int E = df_exp_bound(out.hi);
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) E = max(E, __shfl_xor_sync(BA_FULL_MASK, E, off));
  const int row = ri + r;  // < big_dig_rows(n): ri < n and rows of a block column are padded to kBigNB
  const size_t slice = (size_t)C.dig_groups * (kGroupBytes / 2);  // uint16 per digit matrix
  const bool live = r < nr && c < nb;
  if (live) {
    Fh[(size_t)row * n + r0 + c] = out.hi;
    Fl[(size_t)row * n + r0 + c] = out.lo;
  }
  uint16_t dg[kSlices];
  df_digits(live ? out : dfl{0.0f, 0.0f}, E, dg);
  const size_t off = canon_off(row, c) / 2;
#pragma unroll
  for (int t = 0; t < kSlices; ++t) C.dig[(size_t)t * slice + off] = dg[t];
  if (c == 0) C.dexp[row] = E;
}

constexpr int kUpdThreads = 512;  // 16 warps: 4 per tensor-memory lane quarter, 8 columns each
constexpr int kUpdM = 128, kUpdN = 32;
constexpr uint32_t kUpdA = kUpdM / 8 * kGroupBytes;  // bytes of one digit matrix of the 128-row operand
constexpr uint32_t kUpdB = kUpdN / 8 * kGroupBytes;  // of the 32-row operand
constexpr uint32_t kUpdTmemCols = 256;               // kDiags accumulators of kUpdN columns
constexpr size_t kUpdOperandBytes = (size_t)kSlices * (kUpdA + kUpdB);
// Dynamic shared memory requested per CTA: more than a third of the SM's
// 228 KB, so that at most two CTAs share an SM and their tensor-memory
// allocations (2 x 256 of the 512 columns) always succeed at once.
constexpr size_t kUpdSmem = 96 * 1024;
static_assert(kUpdOperandBytes + 256 <= kUpdSmem && 3 * kUpdSmem > 228 * 1024, "update kernel shared memory");
static_assert(kDiags * kUpdN <= (int)kUpdTmemCols, "accumulators fit the allocation");
constexpr uint64_t kTcWaitNs = 200000000ull;  // give up on a copy or the products after 200 ms

// Block column k, m row blocks below it: tile (column block jb, row group
// rg) holds rows [R0 + 128 rg, + 128) x columns [R0 + 32 jb, + 32) of the
// trailing matrix, R0 = 32 (k + 1).  A_ij -= L_ik L_jk^T by the digit
// products on the tensor cores (accumulators in tensor memory), combined
// per entry in double-float and subtracted from the factor.
__global__ void __launch_bounds__(kUpdThreads, 1) k_big_update_tc(const DevCluster* dcl, int k, int m) {
  const DevCluster& C = *dcl;
  const int n = 6 * C.n_free;
  const int R0 = kBigNB * (k + 1), band_end = min(n, R0 + kBigNB * m);
  const int jb = blockIdx.x, rg = blockIdx.y;
  const int rA = R0 + kUpdM * rg, cB = R0 + kUpdN * jb;
  if (rA >= band_end || rA + kUpdM - 1 < cB) return;  // past the band, or above the diagonal
  extern __shared__ __align__(1024) unsigned char smu[];
  unsigned char* sa = smu;
  unsigned char* sb = smu + (size_t)kSlices * kUpdA;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smu + kUpdOperandBytes);  // [0] copies, [1] products
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bars + 2);
  int* s_ok = reinterpret_cast<int*>(s_tmem + 1);
  int* s_ecol = s_ok + 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(s_tmem, kUpdTmemCols);
  if (tid < kUpdN) s_ecol[tid] = C.dexp[cB + tid];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  const size_t slice_bytes = (size_t)C.dig_groups * kGroupBytes;
  const unsigned char* dig = reinterpret_cast<const unsigned char*>(C.dig);
  if (tid == 0) {
    mbar_arrive_expect_tx(&bars[0], (uint32_t)kUpdOperandBytes);
    for (int t = 0; t < kSlices; ++t) {
      bulk_copy_g2s(sa + (size_t)t * kUpdA, dig + t * slice_bytes + (size_t)(rA / 8) * kGroupBytes, kUpdA, &bars[0]);
      bulk_copy_g2s(sb + (size_t)t * kUpdB, dig + t * slice_bytes + (size_t)(cB / 8) * kGroupBytes, kUpdB, &bars[0]);
    }
    int ok = mbar_wait_bounded(&bars[0], 0, kTcWaitNs) ? 1 : 0;
    if (ok) {
      issue_digit_products<kUpdM, kUpdN>(tmem, smem_u32(sa), kUpdA, smem_u32(sb), kUpdB);
      mma_commit(&bars[1]);
      ok = mbar_wait_bounded(&bars[1], 0, kTcWaitNs) ? 1 : 0;
      if (!ok) mbar_wait_bounded(&bars[1], 0, kTcWaitNs);  // the products still running, once more
    } else {
      mbar_wait_bounded(&bars[0], 0, kTcWaitNs);  // the copies in flight, once more
    }
    *s_ok = ok;
    if (!ok) C.lm->dev_error = kDevErrTimeout;
  }
  __syncthreads();
  tc_fence_after();
  if (*s_ok) {
    // warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (rows) and columns
    // 8 (w / 4) .. + 7 of every accumulator
    const int quarter = warp & 3, cb = 8 * (warp >> 2);
    const int row = rA + 32 * quarter + lane;
    const bool live = row < band_end;
    const int er = live ? C.dexp[row] : 0;
    float* Fh = df_hi(C);
    float* Fl = df_lo(C);
    const size_t o0 = (size_t)row * n + cB + cb;
    const int ncol = live ? min(8, row - (cB + cb) + 1) : 0;  // columns on or left of the diagonal
    float fh[8], fl[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      fh[i] = i < ncol ? Fh[o0 + i] : 0.0f;
      fl[i] = i < ncol ? Fl[o0 + i] : 0.0f;
    }
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    float acc[kDiags][8];
#pragma unroll
    for (int c = 0; c < kDiags; ++c) tmem_ld8(lane_base + (uint32_t)(c * kUpdN + cb), acc[c]);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float a[kDiags];
#pragma unroll
      for (int c = 0; c < kDiags; ++c) a[c] = acc[c][i];
      const dfl v = df_ldexp(combine_diags(a), er + s_ecol[cb + i]);
      const dfl f = df_sub(dfl{fh[i], fl[i]}, v);
      if (i < ncol) {
        Fh[o0 + i] = f.hi;
        Fl[o0 + i] = f.lo;
      }
    }
  }
  (void)lane;
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kUpdTmemCols);
}

// Dot2 partial sums of a warp (or of aligned groups of `width` lanes)
// merged by a butterfly: every lane ends with the group's total.
__device__ __forceinline__ Dot2 warp_merge(Dot2 d, int width) {
  for (int off = 1; off < width; off <<= 1)
    d.merge(__shfl_xor_sync(BA_FULL_MASK, d.s, off), __shfl_xor_sync(BA_FULL_MASK, d.c, off));
  return d;
}

size_t big_solve_df_smem(int n) { return sizeof(float) * (2 * (size_t)n + 2 * kBigNB); }

constexpr int kSolveChunk = 12;  // entries a lane loads before it sums them

// Solve S y = v with the double-float factor (one CTA of 1024 threads; v in
// shared memory).  Both sweeps read, per block k of 32 rows, the rows' own
// entries left of the diagonal block, L(r0 + r, lo .. r0), lo = the block's
// first envelope column (contiguous in memory: coalesced across a warp), and
// the inverted diagonal block X = L_kk^-1 (loaded one block ahead).
//   forward  (k ascending):  u = v_k - L(k, lo .. r0) v(lo .. r0); v_k = X u
//   backward (k descending): x_k = X^T v_k; v(lo .. r0) -= L(k, lo .. r0)^T x_k
// Every dot product is compensated (Dot2); each lane issues its loads in
// groups of kSolveChunk before it sums them.  x = S^-1 rhs (mode 0) or
// x += S^-1 t (mode 1), binary64 in and out.
__global__ void __launch_bounds__(1024) k_big_solve_df(const DevCluster* dcl, int mode) {
  const DevCluster& C = *dcl;
  extern __shared__ float sv[];
  const int n = 6 * C.n_free, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  float* vh = sv;
  float* vl = sv + n;
  float* yh = sv + 2 * n;
  float* yl = yh + kBigNB;
  const float* Fh = df_hi(C);
  const float* Fl = df_lo(C);
  const double* src = mode == 0 ? C.rhs : C.bx + 2 * n;
  for (int i = tid; i < n; i += blockDim.x) {
    const dfl v = df_from_d(src[i]);
    vh[i] = v.hi;
    vl[i] = v.lo;
  }
  const int nblk = (n + kBigNB - 1) / kBigNB;
  const size_t xs = 2 * kBigNB * kBigNB;
  // this thread's entry of X: (wid, lane) in the forward sweep, (lane, wid) in the backward one
  float xh = C.linv[wid * kBigNB + lane], xl = C.linv[kBigNB * kBigNB + wid * kBigNB + lane];
  __syncthreads();
  for (int k = 0; k < nblk; ++k) {  // L y = v
    const int r0 = kBigNB * k, nb = min(kBigNB, n - r0), lo = ef_row(C, r0);
    const float cxh = xh, cxl = xl;
    if (k + 1 < nblk) {
      xh = C.linv[(k + 1) * xs + wid * kBigNB + lane];
      xl = C.linv[(k + 1) * xs + kBigNB * kBigNB + wid * kBigNB + lane];
    }
    if (wid < nb) {  // warp r: u_r = v_r - sum_j L(r0 + r, j) v_j
      const size_t ro = (size_t)(r0 + wid) * n;
      Dot2 acc;
      for (int base = lo; base < r0; base += 32 * kSolveChunk) {
        float ah[kSolveChunk], al[kSolveChunk];
#pragma unroll
        for (int i = 0; i < kSolveChunk; ++i) {
          const int j = base + lane + 32 * i;
          ah[i] = j < r0 ? Fh[ro + j] : 0.0f;
          al[i] = j < r0 ? Fl[ro + j] : 0.0f;
        }
#pragma unroll
        for (int i = 0; i < kSolveChunk; ++i) {
          const int j = base + lane + 32 * i;
          if (j < r0) acc.add(dfl{ah[i], al[i]}, dfl{vh[j], vl[j]});
        }
      }
      acc = warp_merge(acc, 32);
      if (lane == 0) {
        const dfl u = df_sub(dfl{vh[r0 + wid], vl[r0 + wid]}, acc.get());
        yh[wid] = u.hi;
        yl[wid] = u.lo;
      }
    }
    __syncthreads();
    {  // warp r: v_r = sum_q X(r, q) u_q
      Dot2 acc;
      if (lane < nb) acc.add(dfl{cxh, cxl}, dfl{yh[lane], yl[lane]});
      acc = warp_merge(acc, 32);
      if (lane == 0 && wid < nb) {
        const dfl y = acc.get();
        vh[r0 + wid] = y.hi;
        vl[r0 + wid] = y.lo;
      }
    }
    __syncthreads();
  }
  xh = C.linv[(nblk - 1) * xs + lane * kBigNB + wid];
  xl = C.linv[(nblk - 1) * xs + kBigNB * kBigNB + lane * kBigNB + wid];
  for (int k = nblk - 1; k >= 0; --k) {  // L^T x = y
    const int r0 = kBigNB * k, nb = min(kBigNB, n - r0), lo = ef_row(C, r0);
    {  // warp r: x_r = sum_q X(q, r) y_q
      Dot2 acc;
      if (lane < nb) acc.add(dfl{xh, xl}, dfl{vh[r0 + lane], vl[r0 + lane]});
      acc = warp_merge(acc, 32);
      if (lane == 0) {
        const dfl x = acc.get();
        yh[wid] = x.hi;
        yl[wid] = x.lo;
      }
    }
    if (k > 0) {
      xh = C.linv[(k - 1) * xs + lane * kBigNB + wid];
      xl = C.linv[(k - 1) * xs + kBigNB * kBigNB + lane * kBigNB + wid];
    }
    __syncthreads();
    if (tid < nb) {
      vh[r0 + tid] = yh[tid];
      vl[r0 + tid] = yl[tid];
    }
    for (int j = lo + tid; j < r0; j += blockDim.x) {  // v_j -= sum_r L(r0 + r, j) x_r
      Dot2 acc;
      for (int q0 = 0; q0 < nb; q0 += kSolveChunk) {
        float ah[kSolveChunk], al[kSolveChunk];
#pragma unroll
        for (int i = 0; i < kSolveChunk; ++i) {
          const size_t o = (size_t)(r0 + q0 + i) * n + j;
          ah[i] = q0 + i < nb ? Fh[o] : 0.0f;
          al[i] = q0 + i < nb ? Fl[o] : 0.0f;
        }
#pragma unroll
        for (int i = 0; i < kSolveChunk; ++i)
          if (q0 + i < nb) acc.add(dfl{ah[i], al[i]}, dfl{yh[q0 + i], yl[q0 + i]});
      }
      const dfl v = df_sub(dfl{vh[j], vl[j]}, acc.get());
      vh[j] = v.hi;
      vl[j] = v.lo;
    }
    __syncthreads();
  }
  double* x = C.bx + n;
  for (int i = tid; i < n; i += blockDim.x) {
    const double v = (double)vh[i] + (double)vl[i];
    x[i] = mode == 0 ? v : x[i] + v;
  }
}

}  // namespace

static int grid_for_big(int items, int per_block) {
  const int g = (items + per_block - 1) / per_block, cap = num_sms() * 8;
  return g < 1 ? 1 : (g > cap ? cap : g);
}

// The launches of one iteration's reduced-system solve for one large cluster
// (captured into the caller's graph).  assemble_only: priors, g_c and S only.
void launch_big_solve(const BigRef& b, bool mixed, int refine_steps, int assemble_only, cudaStream_t st) {
  const int n = b.n;
  const size_t nn = (size_t)n * n;
  cudaMemsetAsync(b.S, 0, nn * sizeof(double), st);
  LAUNCH(KK_FACTOR, st, k_big_prior<<<(b.nf + 63) / 64, 64, 0, st>>>(b.d));
  LAUNCH(KK_FACTOR, st, k_big_pairs<<<grid_for_big(b.n_pairs * 36, 256), 256, 0, st>>>(b.d));
  if (assemble_only) return;
  const int nblk = (n + kBigNB - 1) / kBigNB;
  if (b.tc) {
    LAUNCH(KK_FACTOR, st, k_big_split<<<std::min(n, num_sms() * 8), 256, 0, st>>>(b.d));
    for (int k = 0; k < nblk; ++k) {
      const int m = b.below[k];
      LAUNCH(KK_FACTOR, st, k_big_panel<<<1 + m, kPanelThreads, 0, st>>>(b.d, k, b.panel_w));
      if (m > 0) {
        const dim3 grid(m, (kBigNB * m + kUpdM - 1) / kUpdM);
        LAUNCH(KK_FACTOR, st, k_big_update_tc<<<grid, kUpdThreads, kUpdSmem, st>>>(b.d, k, m));
      }
    }
    const size_t sm = big_solve_df_smem(n);
    LAUNCH(KK_FACTOR, st, k_big_solve_df<<<1, 1024, sm, st>>>(b.d, 0));
    for (int it = 0; it < refine_steps; ++it) {
      LAUNCH(KK_FACTOR, st, k_big_resid<<<grid_for_big(n * 32, 256), 256, 0, st>>>(b.d));
      LAUNCH(KK_FACTOR, st, k_big_solve_df<<<1, 1024, sm, st>>>(b.d, 1));
    }
  } else {
    cudaMemcpyAsync(b.F, b.S, nn * sizeof(double), cudaMemcpyDeviceToDevice, st);
    for (int k = 0; k < nblk; ++k) {
      LAUNCH(KK_FACTOR, st, k_big_diag<<<1, 256, 0, st>>>(b.d, k));
      const int m = b.below[k];
      if (m > 0) {
        LAUNCH(KK_FACTOR, st, k_big_trsm<<<m, 256, 0, st>>>(b.d, k));
        LAUNCH(KK_FACTOR, st, k_big_update<<<m * (m + 1), 256, 0, st>>>(b.d, k));
      }
    }
    const size_t sm = big_solve_smem(n);
    LAUNCH(KK_FACTOR, st, k_big_solve<<<1, 1024, sm, st>>>(b.d, 0));
    for (int it = 0; it < refine_steps; ++it) {
      LAUNCH(KK_FACTOR, st, k_big_resid<<<grid_for_big(n * 32, 256), 256, 0, st>>>(b.d));
      LAUNCH(KK_FACTOR, st, k_big_solve<<<1, 1024, sm, st>>>(b.d, 1));
    }
  }
  if (mixed) LAUNCH(KK_FACTOR, st, k_big_finish<true><<<1, 512, 0, st>>>(b.d));
  else LAUNCH(KK_FACTOR, st, k_big_finish<false><<<1, 512, 0, st>>>(b.d));
}

cudaError_t set_big_attributes(int max_n) {
  const int smem = (int)big_solve_smem(max_n);
  cudaError_t e =
      cudaFuncSetAttribute(k_big_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, smem > 48 * 1024 ? smem : 48 * 1024);
  if (e != cudaSuccess) return e;
  const int smem_df = (int)big_solve_df_smem(max_n);
  e = cudaFuncSetAttribute(k_big_solve_df, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           smem_df > 48 * 1024 ? smem_df : 48 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_big_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUpdSmem);
}

}  // namespace bagpu
