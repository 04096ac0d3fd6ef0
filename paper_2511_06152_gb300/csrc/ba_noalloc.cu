// ba_cost_noalloc: the robust cost F(x) of a cluster from caller-owned
// device arrays, with no device or host allocation.
//
// Some callers cannot allocate once they are running: onboard flight
// software that reserves all of its memory at start-up and forbids
// allocation afterwards (the setting the paper's real-time pipeline targets),
// or a host process whose device memory is owned by another allocator.  This
// entry point serves them.  It is the same computation as the library's cost
// pass (per-chunk partial sums, then a fixed-order total plus the GNSS/IMU
// prior terms), but its partial sums live in the file-scope device array
// below instead of memory the library allocates.
//
// Scratch: kNoAllocMaxPartials doubles (512 KiB).  Every GPU that loads the
// library holds the array until the process exits.  One partial covers
// kNoAllocChunk observations, so a call accepts at most
// kNoAllocChunk * kNoAllocMaxPartials = 67,108,864 observations.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/ba.h"
#include "ba_device.cuh"

namespace {

constexpr int kNoAllocChunk = 1024;         // observations per partial sum
constexpr int kNoAllocThreads = 256;        // threads per chunk block
constexpr int kNoAllocMaxPartials = 65536;  // scratch capacity (doubles)
constexpr long long kNoAllocMaxObs = (long long)kNoAllocChunk * kNoAllocMaxPartials;
constexpr int kMaxDevices = 64;

// Shared by every call on a device; keeps the last call's contents.  Each
// call writes partials [0, n_chunks) before it reads them, so nothing needs
// clearing; calls that overlap on the GPU race on this array.
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxPartials];

std::mutex g_setup_mu;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device.  In host code the array's name is only a host-side stand-in.
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// One block per chunk of kNoAllocChunk observations: each thread sums its
// observations in a fixed order, then a fixed tree over the block.
__global__ void __launch_bounds__(kNoAllocThreads)
k_cost_chunks_noalloc(const double* __restrict__ intr, const double* __restrict__ R, const double* __restrict__ T,
                      const double* __restrict__ X, const int32_t* __restrict__ obs_cam,
                      const int32_t* __restrict__ obs_pt, const double* __restrict__ obs_uv, int n_cams, int n_pts,
                      int n_obs, double half_inv_s2, double delta, double* partials) {
  __shared__ double red[kNoAllocThreads / 32];
  const int c = blockIdx.x;
  double v = 0.0;
  for (int i = 0; i < kNoAllocChunk / kNoAllocThreads; ++i) {
    const long long o = (long long)c * kNoAllocChunk + (long long)i * kNoAllocThreads + threadIdx.x;
    if (o >= n_obs) break;
    const int k = obs_cam[o], j = obs_pt[o];
    if (k < 0 || k >= n_cams || j < 0 || j >= n_pts) {  // invalid index: poison the result, never fault
      v += __longlong_as_double(0x7ff8000000000000ULL);
      continue;
    }
    v += bagpu::obs_cost(R + 9 * (size_t)k, T + 3 * (size_t)k, intr + 7 * (size_t)k, X + 3 * (size_t)j,
                         obs_uv[2 * o], obs_uv[2 * o + 1], half_inv_s2, delta);
  }
  v = bagpu::warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kNoAllocThreads / 32; ++w) s += red[w];
    partials[c] = s;
  }
}

// One block: the partials in a fixed order, plus the prior terms of the free
// cameras in camera order.
__global__ void __launch_bounds__(kNoAllocThreads)
k_cost_finish_noalloc(const double* partials, int n_chunks, const double* __restrict__ R, const double* __restrict__ T,
                      const double* __restrict__ R_prior, const double* __restrict__ T_prior,
                      const uint8_t* __restrict__ fixed, int n_cams, double sigma_imu, double sigma_gnss,
                      double* F_out) {
  __shared__ double red[kNoAllocThreads / 32];
  double v = 0.0;
  for (int i = threadIdx.x; i < n_chunks; i += blockDim.x) v += partials[i];
  v = bagpu::warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double F = 0.0;
    for (int w = 0; w < kNoAllocThreads / 32; ++w) F += red[w];
    for (int k = 0; k < n_cams; ++k) {
      if (fixed && fixed[k]) continue;
      F += bagpu::prior_terms(R + 9 * (size_t)k, T + 3 * (size_t)k, R_prior + 9 * (size_t)k, T_prior + 3 * (size_t)k,
                              sigma_imu, sigma_gnss, nullptr, nullptr);
    }
    *F_out = F;
  }
}

}  // namespace

extern "C" BA_API ba_status ba_cost_noalloc(const ba_cluster_desc* d, void* stream, double* F_out) {
  if (!d || !F_out || d->ptr_kind != BA_PTR_DEVICE) return BA_ERR_INVALID;
  if (d->n_cams < 1 || d->n_pts < 0 || d->n_obs < 0 || (long long)d->n_obs > kNoAllocMaxObs) return BA_ERR_INVALID;
  if (!(d->sigma_px > 0.0) || !(d->huber_delta_px > 0.0) || !(d->sigma_gnss_m >= 0.0) || !(d->sigma_imu_rad >= 0.0))
    return BA_ERR_INVALID;
  if (!d->intr || !d->R || !d->T || !d->R_prior || !d->T_prior || (d->n_pts > 0 && !d->X) ||
      (d->n_obs > 0 && (!d->obs_cam || !d->obs_pt || !d->obs_uv)))
    return BA_ERR_INVALID;
  double* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return BA_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int n_chunks = (int)((d->n_obs + (long long)kNoAllocChunk - 1) / kNoAllocChunk);
  const double half_inv_s2 = 0.5 / (d->sigma_px * d->sigma_px);
  if (n_chunks > 0)
    k_cost_chunks_noalloc<<<n_chunks, kNoAllocThreads, 0, st>>>(d->intr, d->R, d->T, d->X, d->obs_cam, d->obs_pt,
                                                                d->obs_uv, d->n_cams, d->n_pts, d->n_obs, half_inv_s2,
                                                                d->huber_delta_px, scratch);
  k_cost_finish_noalloc<<<1, kNoAllocThreads, 0, st>>>(scratch, n_chunks, d->R, d->T, d->R_prior, d->T_prior, d->fixed,
                                                        d->n_cams, d->sigma_imu_rad, d->sigma_gnss_m, F_out);
  return cudaGetLastError() == cudaSuccess ? BA_OK : BA_ERR_CUDA;
}
