// Internal layout shared by the kernels and the host side of the library.
//
// One cluster lives in one device arena.  Points are reordered along a
// Morton curve of their initial ground position, and observations are stored
// in point-major order (sorted by point, then camera), so the observations of
// a point are contiguous and nearby points share cameras.  "Tiles" cut that
// order into runs of at most 32 observations holding whole points (one warp
// each); "chunks" group consecutive tiles (one CTA each).  Per chunk, a
// presorted table lists the observations of each free camera and the
// observation pairs of each co-visible camera pair; the chunk reduces its
// observations into per-camera and per-pair partial sums in that fixed order,
// and the reduced camera system sums the partials in chunk order.  No
// reduction depends on anything but the cluster itself.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace bagpu {

constexpr int kSrec = 28;         // per-observation shared record: Jc[12], r[2], u[2], W[3], pad, P[6], pad
#ifndef BA_LIN_SCHUR_MIN_BLOCKS
#define BA_LIN_SCHUR_MIN_BLOCKS 2
#endif
constexpr int kLinSchurMinBlocksMixed = BA_LIN_SCHUR_MIN_BLOCKS;  // CTAs per SM the mixed linearise+Schur kernel is compiled for
constexpr int kCamPart = 40;      // camera partial: A[21], gobs[6], Zq[6], Udiag[6], pad
constexpr int kPairPart = 36;     // pair partial: sum Z_a Z_b^T (6x6 row-major)
constexpr int kChunkTilesMixed = 16;  // tiles per chunk (two per warp), binary32 records
constexpr int kChunkTilesF64 = 8;     // tiles per chunk (one per warp), binary64 records
constexpr int kChunkObsMixed = 32 * kChunkTilesMixed;  // at most this many observations per chunk
constexpr int kChunkObsF64 = 32 * kChunkTilesF64;
constexpr int kChunkThreads = 256;
constexpr int kMaxTrack = 32;
constexpr int kMaxFreeSmall = 32;  // free cameras the single-CTA factor handles (n <= 192)
constexpr int kMaxBatchChains = 8;  // concurrent launch chains of a batch's LM iterations, at most
constexpr int kMaxFree = 1024;     // free cameras of one cluster (larger systems: the global-memory solver)
constexpr int kBigNB = 32;         // block size of the global-memory factorisation
constexpr int kSlicesHost = 6;     // Ozaki digits per double-float entry (kSlices of ba_tc.cuh)
constexpr double kDiagMin = 1e-6;
constexpr double kDiagMax = 1e32;
constexpr double kMinDepth = 1e-6;
constexpr int BA_STATUS_NOT_PD = -3;  // same value as BA_ERR_NOT_PD in ba.h
constexpr int kTraceCap = 256;
constexpr int kCostInitThreads = 256;  // threads of k_cost_init's CTA (its sums' order)
// double-float camera record (floats): high words of R [0, 9), T.hi [9, 12),
// T.lo [12, 15), f.hi 15, k1 k2 p1 p2 .hi [16, 20), free flag 20, pad; then
// the low words of R [24, 33), f.lo 33, k1 k2 p1 p2 .lo [34, 38), pad to 40
constexpr int kCamDf = 40;
constexpr int kCamReal = 20;

struct Tile {
  int obs_begin;
  int n_obs;  // <= 32, whole points
};

struct Chunk {
  int obs_begin, n_obs;     // point-major observation range (whole tiles)
  int tile_begin, n_tiles;  // its tiles
  int job_begin;            // its jobs: n_lc free cameras, then n_lp co-visible camera pairs
  int n_lc, n_lp;
  int pt_begin, n_pts;      // internal point range spanned by its observations
};

// One reduction job of a chunk: a free camera (items: its observations, as
// chunk-local indices into cm_list) or a camera pair (items: the chunk-local
// observation index pairs a | b << 16 in pent), summed by a run of lanes.
struct Job {
  int slot;        // camera or pair partial slot
  int item_begin;  // into cm_list (camera) or pent (pair)
  int count;       // items
  short lane_begin, n_lanes;
};
static_assert(sizeof(Job) == 16, "jobs are staged as 16-byte records");

// shared-memory row per lane for multi-lane jobs: 44 words, so that the
// 16-byte stores of the eight lanes of a quarter-warp fall on distinct banks
constexpr int kLanePart = 44;

// Per-cluster LM control state, resident on the device.
struct LmState {
  double mu, nu;
  double F;          // cost at the current state
  double F_new;      // cost at the candidate
  double pred_cam;   // camera part of d^T (mu D d + g)
  double prior_new;  // prior cost at the candidate
  double mu0;        // damping a reset restores (mu0 at create, or the warm start's)
  double nu0;        // nu a reset restores (2 at create, or the warm start's)
  int cur;           // which of the double-buffered states is current
  int status;        // status of the last factorisation
  int iter;          // iterations run
  int n_accepted;
  int active;        // 1 while the cluster still has iterations to run
  int iters_target;
  int pt_fail;       // a damped point block was not positive definite this iteration
  float mu_f;        // mu rounded to binary32 (mixed-path kernels)
  int needs_init;    // F must be evaluated at the current state before the next iteration
  int dev_error;     // a kernel gave up on a bounded wait this iteration (kDevErrTimeout); rejects the step
  int tiles_done;    // back-substitution tiles finished this iteration; the warp that finishes the last
                     // one takes the cluster's LM decision (zeroed by the factor kernels)
  int iter0;         // iter when the cluster was last armed
  double ftol;       // serving: an accepted step after the first that lowers F by at most ftol * F
                     // ends the solve (0: off)
};

constexpr int kDevErrTimeout = -4;  // = BA_ERR_TIMEOUT

// Same layout as ba_step_info.
struct StepRec {
  int accepted, status;
  double F_before, F_after, predicted, gain, mu_used, mu, nu;
};

// Device-side descriptor of one cluster (plain pointers into its arena).
struct DevCluster {
  int n_cams, n_pts, n_obs, n_free;
  int n_tiles, n_chunks, n_pairs, n_cslots, n_pslots, pad_i;
  double sigma_px, huber_delta, sigma_gnss, sigma_imu;
  float inv_sigma_f, delta_f, half_inv_s2_f, pad_f;  // binary32 copies of 1/sigma_px, delta, 1/(2 sigma_px^2)

  const double* intr;      // [nc][7]
  double* R;               // [2][nc][9]
  double* T;               // [2][nc][3]
  // Points (internal order), double-buffered.  FP64 path: binary64 [2][np][3].
  // Mixed path: double-float [2][np][3] of (hi, lo) binary32 pairs (same 24 B).
  double* X;
  const double* R_prior;   // [nc][9]
  const double* T_prior;   // [nc][3]
  const double* R_init;    // [nc][9] state given at create (for reset)
  const double* T_init;    // [nc][3]
  const double* X_init;    // [np][3], same representation as X, internal order
  const int* pt_perm;      // [np] internal point -> caller's point index
  const int* free_idx;     // [nc] -> free index or -1
  const int* cam_of_free;  // [nf]
  const int* cam_nobs;     // [nc] observations of each camera
  // elimination order of the reduced camera system: free image f sits at
  // block position fpos[f]; env_first[p] = first block column of block row
  // p inside the envelope of S (and of its Cholesky factor)
  const int* fpos;         // [nf]
  const int* env_first;    // [nf], non-decreasing
  // global-memory solver (more than kMaxFreeSmall free images), else null:
  double* F;               // [n][n] Cholesky factor (lower), elimination order
  double* bx;              // [4][n]: right-hand side / work, solution, correction, 1 / L(j, j)
  int* bflag;              // nonzero: a pivot was not positive
  // tensor-core factorisation of the global-memory solver: F holds the factor
  // as double-float (binary32 high words [n][n], then low words [n][n]);
  // dig: Ozaki digits of the current panel's rows, [kSlices][dig_groups]
  // groups of 8 rows x 32 columns in the canonical shared-memory layout
  // (512 bytes each); dexp: each row's power-of-two scale; linv: the inverse
  // of each 32 x 32 diagonal block of the factor, [nblk][hi, lo][32][32]
  unsigned short* dig;
  int* dexp;
  float* linv;
  void* camreal;           // FP64 path: double [nc][20]: R[9], T[3], intr[7], free flag
  float* camdf;            // mixed path: [2][nc][kCamDf] double-float cameras

  // per point, from the current iteration's linearisation: M = L^-1 of the
  // damped point block (m00 m10 m11 m20 m21 m22), q = M g_p, D_p, g_p, pad;
  // Real [n_pts][16], written by the linearise+Schur kernel for the
  // back-substitution
  void* ptblk;
  const Tile* tiles;       // [n_tiles]
  const int* obs_cam;      // [no] point-major
  const int* obs_pt;       // [no] point-major, internal point index
  const double* obs_uv;    // [no][2] point-major, binary64 pixels
  const float2* obs_chi;   // mixed path: [no] hi part of (u - cx, v - cy)
  const float2* obs_clo;   // mixed path: [no] lo part of (u - cx, v - cy)

  const Chunk* chunks;         // [n_chunks]
  const Job* jobs;             // per chunk, in lane order
  const unsigned char* lane_job;  // [n_chunks][kChunkThreads] job of each lane (chunks of at most kChunkThreads jobs)
  const unsigned short* cm_list;  // chunk-local observation lists per camera job
  const unsigned int* pent;       // chunk-local observation pairs per pair job
  void* campart;               // Real [n_cslots][kCamPart]
  void* pairpart;              // Real [n_pslots][kPairPart]
  const int* cam_slot_begin;   // [nf + 1]
  const int* cam_slots;        // [n_cslots] camera partial slots by free camera, chunk order
  const int2* pair_key;        // [n_pairs] (free a, free b), a < b
  const int* pair_slot_begin;  // [n_pairs + 1]
  const int* pair_slots;       // [n_pslots] pair partial slots by pair, chunk order
  double* camsum;              // [nf][kCamPart] per-camera sums of the partials
  double* pairsum;             // [n_pairs][kPairPart] per-pair sums of the partials

  double* S;        // [n][n], n = 6 nf, row-major, full
  double* rhs;      // [n]
  double* gc;       // [n]
  double* Dc;       // [n]
  double* dc;       // [n]
  float* dc32;      // [n] binary32 copy of dc (mixed path)
  double* tilepart; // [n_tiles][2]: cost, point pred (or max |g_p| in the diagnostic pass)
  LmState* lm;
  StepRec* trace;   // [trace_cap]
  int trace_cap;
  int dig_groups;   // groups of 8 rows in dig (rows of the factor rounded up to 32, plus 128)
};

struct BatchView {
  const DevCluster* cl;  // [n]
  const int* tile_pre;   // [n + 1]
  const int* chunk_pre;  // [n + 1]
  const int* item_pre;   // [n + 1] free cameras + camera pairs
  const int* factor_order;  // [n] clusters by decreasing reduced-system size
  const int* tot;        // device [3]: total tiles, chunks, reduction items (kernels read these)
  int n;
  int total_tiles, total_chunks, total_items;
  int max_n;             // largest 6 * n_free in the batch
  int inject;            // failure injection for tests (kInject* bits); 0 in normal use
  // launch parameters the autotuner chooses (TuneParams)
  int lin_ctas_per_sm;   // linearise+Schur grid: at most this many CTAs per SM (grid-stride beyond)
  int back_ctas_per_sm;  // back-substitution grid: at most this many CTAs per SM
  int factor_nb;         // panel width of the shared-memory Cholesky
  int factor_threads;    // threads of the shared-memory factor CTA
  int factor_df;         // 1: the shared-memory factor in double-float (mixed path, or BA_FLAG_SMALL_DF_FACTOR)
};

// Launch and presort parameters chosen by the autotuner (ba_tune in ba.h).
struct TuneParams {
  int chunk_tiles = 0;       // tiles per linearise+Schur chunk (0: the precision's maximum)
  int lin_ctas_per_sm = 8;
  int back_ctas_per_sm = 16;
  int factor_nb = 8;
  int factor_threads = 512;
  int big_panel_w = 4;       // columns of a block of the global-memory solver's panel factorisation
  int batch_chains = 4;      // concurrent launch chains of a batch's LM iterations
};

// kInjectCopyTimeout: the mixed linearise+Schur kernel waits for its first
// staged chunk on a barrier that nothing completes, with a 1 ms limit, so
// that its bounded-wait failure path runs (BA_FLAG_INJECT_COPY_TIMEOUT).
constexpr int kInjectCopyTimeout = 1;

// Kernel kinds, for launch counting and per-kernel timing.
enum KernelKind {
  KK_LIN_SCHUR = 0,
  KK_PARTIAL_REDUCE,  // chunk partials -> per-camera / per-pair sums
  KK_FACTOR,
  KK_BACKSUB,
  KK_LM_UPDATE,
  KK_COST_TILES,
  KK_COST_INIT,
  KK_OTHER,
  KK_COUNT
};

// CUDA events bracketing each launch while a probe is attached to the thread.
struct ProbeRec {
  int kind;
  cudaEvent_t e0, e1;
};
struct Probe {
  std::vector<ProbeRec> recs;
};
void set_probe(Probe* p);                       // attach to the calling thread (nullptr detaches)
unsigned long long take_direct_launches();      // launches outside capture since the last call
unsigned long long take_captured_launches();    // kernel nodes captured since the last call

// Every kernel launch goes through LAUNCH(kind, stream, launch): it counts the
// launch (direct, or as a captured graph node) and, with a probe attached to
// the calling thread, brackets it with events for per-kind timing.
struct LaunchScope {
  int kind;
  cudaStream_t st;
  cudaEvent_t e0 = nullptr;
  LaunchScope(int k, cudaStream_t s);
  ~LaunchScope();
};
#define LAUNCH(kind, st, ...)   \
  do {                          \
    LaunchScope ls__(kind, st); \
    __VA_ARGS__;                \
  } while (0)

int num_sms();

// A cluster whose reduced system is solved in global memory (more than
// kMaxFreeSmall free images): what the host needs to emit its launches.
struct BigRef {
  const DevCluster* d;     // device descriptor
  int n, nf, n_pairs;
  double* S;               // device [n][n]
  double* F;               // device [n][n]
  std::vector<int> below;  // per block column of kBigNB: row blocks below it inside the envelope
  bool tc = true;          // tensor-core double-float factor (else the binary64 CUDA-core one)
  int panel_w = 4;         // column-block width of the panel factorisation (1, 2, 4, 8, 16 or 32)
};
void launch_big_solve(const BigRef& b, bool mixed, int refine_steps, int assemble_only, cudaStream_t st);
// rows of the digit buffer of a system of order n: n rounded up to kBigNB, plus
// one 128-row tile, so that every tile the update kernel copies lies inside
__host__ __device__ constexpr int big_dig_rows(int n) { return (n + kBigNB - 1) / kBigNB * kBigNB + 128; }
cudaError_t set_big_attributes(int max_n);

// Kernel launchers (ba_kernels.cu).  All run on `st`.
cudaError_t set_kernel_attributes(int max_n);
void launch_arm(const BatchView& bv, int iters, cudaStream_t st);
void launch_arm_slots(const BatchView& bv, const int* arm, const double* ftol, cudaStream_t st);
// DSM raster on the device (heights h[iy * nx + ix] at (x0 + ix dx, y0 + iy dy)),
// with its height range
struct DsmView {
  int nx, ny;
  double x0, y0, dx, dy, hmin, hmax;
  const double* h;
};
constexpr int kDsmMaxSteps = 100000;  // ray samples before the bisection, at most
constexpr int kDsmBisect = 60;        // bisections of the bracketed first hit
void launch_footprints(int n, const double* intr, double width, double height, const double* R, const double* T,
                       const DsmView& D, double* corners, cudaStream_t st);
void launch_overlaps(int na, const double* qa, int nb, const double* qb, double* area, cudaStream_t st);

// Eq. 8 on the (dst camera, src camera) pairs of pairs[n]
void launch_transition(const DevCluster* dst, const DevCluster* src, const int2* pairs, int n, cudaStream_t st);
void launch_warm_copy(const DevCluster* dst, const DevCluster* src, const int2* cams, int n_cams, const int2* pts,
                      int n_pts, cudaStream_t st);
void launch_reset(const BatchView& bv, bool mixed, cudaStream_t st);
void launch_gather(const BatchView& bv, int iters, LmState* lm_out, StepRec* trace_out, cudaStream_t st);
void launch_camreal(const BatchView& bv, bool mixed, cudaStream_t st);
void launch_cost_init(const BatchView& bv, bool mixed, cudaStream_t st);
// big: the batch's clusters with more than kMaxFreeSmall free images (their
// reduced systems are solved by launch_big_solve), or null
void launch_iteration(const BatchView& bv, bool mixed, int refine_steps, cudaStream_t st,
                      const std::vector<BigRef>* big = nullptr);
void launch_grad_norm(const BatchView& bv, bool mixed, double* out, cudaStream_t st,
                      const std::vector<BigRef>* big = nullptr);
void launch_reproj(const DevCluster* dcl, const DevCluster& hcl, bool mixed, double* err_pm, cudaStream_t st);
void launch_export_state(const DevCluster* dcl, const DevCluster& hcl, bool mixed, double* R, double* T, double* X,
                         cudaStream_t st);
void launch_patch_poses(int n, const double* p0, const double* intr0, const double* R0, const double* T0,
                        double lambda, int m, const double* intr, const double* R, const double* T, double width,
                        double height, double* p, uint8_t* inside, cudaStream_t st);
// c, g0: host arrays of 2
void launch_patch_planar(int n, const double* q0, const double* c, const double* g0, int m, const double* theta,
                         const double* g, double* q, cudaStream_t st);
size_t factor_smem_bytes(int max_n);
void launch_fma_probe(int ctas, int iters, float* sink, cudaStream_t st);
int chunk_obs(bool mixed);
int chunk_tiles(bool mixed);

}  // namespace bagpu
