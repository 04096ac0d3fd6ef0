// Reduced camera systems larger than one CTA's shared memory holds (more than
// kMaxFreeSmall free images, n = 6 n_free > 192; the 400-image large block
// has n = 2400), solved in binary64 in global memory.  Same system, order and
// algorithm as the shared-memory solver of ba_kernels.cu: S assembled in the
// reverse Cuthill-McKee elimination order, Cholesky restricted to the
// envelope of S (no fill outside it), a solve, one refinement step against S.
//
//   k_big_prior   per free image: priors, damping D, g_c, rhs, diagonal block
//   k_big_pairs   off-diagonal blocks of S from the co-visible pairs' sums
//   (F = S)
//   per block column k of kBigNB columns (right-looking):
//     k_big_diag    factor the diagonal block (one CTA)
//     k_big_trsm    L_ik = A_ik L_kk^-T for the row blocks inside the envelope
//     k_big_update  A_ij -= L_ik L_jk^T for the tiles inside the envelope
//   k_big_solve   forward and backward substitution (one CTA)
//   k_big_resid   t = rhs - S x
//   k_big_finish  dc, candidate poses, pred and prior terms, status
//
// The envelope is non-decreasing: row r's first nonzero column is
// ef(r) = 6 env_first[r / 6]; the rows of a column block that can be nonzero
// below it form one contiguous run of row blocks, whose length per block
// column the host passes in (it fixes the grid sizes).
#include <cuda_runtime.h>

#include "ba_camera.cuh"
#include "ba_device.cuh"
#include "ba_internal.h"

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
    *C.bflag = 0;
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
  cudaMemcpyAsync(b.F, b.S, nn * sizeof(double), cudaMemcpyDeviceToDevice, st);
  const int nblk = (n + kBigNB - 1) / kBigNB;
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
  if (mixed) LAUNCH(KK_FACTOR, st, k_big_finish<true><<<1, 512, 0, st>>>(b.d));
  else LAUNCH(KK_FACTOR, st, k_big_finish<false><<<1, 512, 0, st>>>(b.d));
}

cudaError_t set_big_attributes(int max_n) {
  const int smem = (int)big_solve_smem(max_n);
  return cudaFuncSetAttribute(k_big_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, smem > 48 * 1024 ? smem : 48 * 1024);
}

}  // namespace bagpu
