// Host side of the C ABI declared in include/ba.h: validation, the presort
// that builds the deterministic reduction tables, device arenas, batch plans
// with CUDA-graph replay, and the serving scheduler.
#include <cuda_runtime.h>

#include <fstream>
#include <sstream>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/ba.h"
#include "ba_internal.h"

static_assert(bagpu::kDevErrTimeout == BA_ERR_TIMEOUT, "device and ABI timeout codes differ");

using namespace bagpu;

namespace {

struct Cluster {
  ba_cluster_id id = 0;
  int nc = 0, np = 0, no = 0, nf = 0;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  DevCluster h{};                 // descriptor with device pointers
  DevCluster* d_desc = nullptr;   // device copy of h
  std::vector<int> pm_to_user;    // point-major position -> caller observation index
  std::vector<int> pt_inv;        // caller point index -> internal point index
  std::atomic<int> in_service{0}; // queued or running in the serving scheduler
  ba_cluster_info info{};         // table sizes, filled at creation
  std::vector<int> big_below;     // global-memory solver: row blocks below each block column (else empty)
};

struct GraphRec {
  cudaGraphExec_t exec = nullptr;
  unsigned long long kernels = 0;  // kernel nodes in the graph
  Probe* probe = nullptr;          // event pairs captured with the graph (timing mode)
};

// One of a batch's concurrent iteration chains: a view of part of the
// batch (its own descriptor copies, prefix sums and factor order) and the
// part's clusters that go to the global-memory solver.
struct Chain {
  BatchView bv{};
  std::vector<BigRef> big;
};

struct Plan {
  std::vector<ba_cluster_id> ids;
  char* dbuf = nullptr;
  size_t dbuf_bytes = 0;
  BatchView bv{};
  std::vector<Chain> chains;     // the LM iterations' launches, one stream each (empty: one chain, bv)
  LmState* lm_out = nullptr;     // device [n]
  double* gnorm = nullptr;       // device [n]
  std::map<int, GraphRec> graphs;
  GraphRec* last = nullptr;      // graph of the last launch (for timing readout)
  cudaEvent_t done = nullptr;    // recorded behind a batch's result copies
  std::vector<BigRef> big;       // clusters whose reduced systems are solved in global memory
};

struct Ticket {
  ba_cluster_id id = 0;
  int iters = 0;
  double ftol = 0.0;   // relative cost decrease that ends the solve (0: off; tested on the device)
  int done = 0;
  ba_result res{};
  std::chrono::steady_clock::time_point t_submit;
  cudaEvent_t ready = nullptr;  // recorded on the context's stream at submit
};

// Serving slots (see scheduler_loop).
struct SlotTable {
  int n = 0;
  int tune_gen = -1;  // ctx->tune_gen the serving graph was captured with
  char* dbuf = nullptr;
  size_t bytes = 0;
  char* hbuf = nullptr;  // two pinned host mirrors of dbuf's layout, one per round parity: the table
                         // goes up, the LM states come back, in copies that do not stage through the
                         // driver, while the other parity's round may still be in flight
  size_t o_lm = 0;       // offset of the LM states (everything before it is the uploaded table)
  cudaEvent_t done[2] = {nullptr, nullptr};  // end of the round of each parity
  cudaEvent_t tail = nullptr;  // end of the last round launched: a completed ticket orders the
                               // context's stream after it (the cluster may still be read, inert,
                               // by a round in flight)
  BatchView bv{};
  DevCluster* d_desc = nullptr;
  int* d_pre = nullptr;
  int* d_order = nullptr;
  int* d_arm = nullptr;
  double* d_ftol = nullptr;
  LmState* d_lm = nullptr;
  DevCluster empty{};
  std::vector<DevCluster> descs;
  std::vector<int> arm;
  std::vector<double> ftol;
  std::vector<long long> first_round;  // per slot: the round its cluster first ran in
  std::vector<ba_cluster_id> occ;
  std::vector<ba_ticket> occ_ticket;
  std::vector<LmState> lm;
  GraphRec graph;
  bool dirty = true;
};

}  // namespace

struct ba_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  uint64_t budget = 0;
  bool mixed = false;
  int n_slots = 64;
  int refine = 1;
  std::map<ba_cluster_id, Cluster*> clusters;
  uint64_t next_id = 1;
  uint64_t mem = 0;
  std::map<std::vector<ba_cluster_id>, Plan*> plans;
  int attr_max_n = 0;
  bool timing = false;
  int inject = 0;  // failure-injection bits for the kernels (BA_FLAG_INJECT_*)
  bool big_fp64 = false;  // global-memory solver: binary64 CUDA-core factor instead of the tensor-core one
  bool small_df = false;  // BA_FP64: shared-memory factor in double-float (as in the mixed path)
  TuneParams tune;        // launch and presort parameters (ba_set_tune, ba_autotune, the tuning table)
  std::atomic<int> tune_gen{0};  // bumped by every change of tune: the serving graph is captured again
  std::mutex stats_mu;  // kernel statistics (API threads and the scheduler)
  // pinned host staging buffers of cluster creation, reused across calls (one
  // per concurrent creation; taken and returned under stage_mu)
  std::atomic<int> creating{0};  // cluster creations in flight (host presort threads)
  std::mutex stage_mu;
  std::vector<std::pair<char*, size_t>> stage_free;
  double kms[KK_COUNT] = {0};
  uint64_t klaunch[KK_COUNT] = {0};
  std::atomic<uint64_t> launches{0};
  std::mutex api_mu;  // cluster table, plans, budget; never held across a serving round
  cudaMemPool_t pool = nullptr;  // device memory of clusters and plans (stream-ordered)

  // serving
  std::mutex sv_mu;
  std::condition_variable sv_cv;
  std::deque<ba_ticket> queue;
  std::map<ba_ticket, Ticket> tickets;
  uint64_t next_ticket = 1;
  std::thread sched;
  bool sched_stop = false;
  bool sched_started = false;
  cudaStream_t sched_stream = nullptr;  // the scheduler's rounds
  cudaStream_t plan_stream = nullptr;   // plan tables (allocated and uploaded without waiting for the solves)
  cudaStream_t copy_stream = nullptr;   // result copies issued without the API lock: never the caller's
                                        // stream, which another thread may be capturing into a graph
  double* hstage = nullptr;             // pinned host staging of ba_get_state (grown on demand)
  std::mutex hstage_mu;                 // the staging's user (taken before api_mu)
  cudaEvent_t state_done = nullptr;     // end of a ba_get_state_batch group's copy
  size_t hstage_bytes = 0;
  SlotTable slots;
  // forked streams of a batch graph's concurrent chains (capture only: no
  // work is ever issued to them outside a capture), with the fork and join
  // events; created on first use
  std::vector<cudaStream_t> chain_streams;
  std::vector<cudaEvent_t> chain_join;
  cudaEvent_t chain_fork = nullptr;
};

namespace {

// message of the calling thread's last failing call (like errno: the API is
// called from several threads, the scheduler among them)
thread_local std::string t_last_error;

ba_status set_err(ba_ctx* ctx, ba_status st, const std::string& msg) {
  (void)ctx;
  t_last_error = msg;
  return st;
}

#define CUDA_TRY(ctx, call)                                                            \
  do {                                                                                 \
    cudaError_t e__ = (call);                                                          \
    if (e__ != cudaSuccess)                                                            \
      return set_err(ctx, BA_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e__)); \
  } while (0)

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

struct Layout {
  size_t off = 0;
  size_t add(size_t bytes) {
    const size_t o = off;
    off += align_up(bytes);
    return o;
  }
};

// A read-only input array of ba_create_cluster: the caller's host memory in
// place, or a host copy of the caller's device memory.
template <typename T>
struct In {
  const T* p = nullptr;
  size_t n = 0;
  std::vector<T> own;
  const T& operator[](size_t i) const { return p[i]; }
  const T* data() const { return p; }
  size_t size() const { return n; }
};

template <typename T>
bool fetch(const T* src, size_t n, int kind, In<T>& out) {
  out.n = n;
  if (n == 0) {
    out.p = out.own.data();
    return true;
  }
  if (!src) return false;
  if (kind == BA_PTR_DEVICE) {
    out.own.resize(n);
    out.p = out.own.data();
    return cudaMemcpy(out.own.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost) == cudaSuccess;
  }
  out.p = src;
  return true;
}

// every value finite: no exponent field of all ones (a branch-free pass the
// compiler vectorises)
bool all_finite(const In<double>& v) {
  uint64_t bad = 0;
  for (size_t i = 0; i < v.n; ++i) {
    uint64_t x;
    std::memcpy(&x, v.p + i, sizeof(x));
    bad |= (uint64_t)(((x >> 52) & 0x7ffu) == 0x7ffu);
  }
  return bad == 0;
}

Cluster* find_cluster(ba_ctx* ctx, ba_cluster_id id) {
  auto it = ctx->clusters.find(id);
  return it == ctx->clusters.end() ? nullptr : it->second;
}

ba_status ensure_attrs(ba_ctx* ctx, int max_n) {
  if (max_n <= ctx->attr_max_n) return BA_OK;
  const int want = std::max(max_n, 6 * kMaxFreeSmall);
  CUDA_TRY(ctx, set_kernel_attributes(std::min(want, 6 * kMaxFreeSmall)));
  if (want > 6 * kMaxFreeSmall) CUDA_TRY(ctx, set_big_attributes(want));
  ctx->attr_max_n = want;
  return BA_OK;
}

void free_probe(Probe* pr) {
  if (!pr) return;
  for (auto& r : pr->recs) {
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
  }
  delete pr;
}

void note_direct(ba_ctx* ctx) { ctx->launches += take_direct_launches(); }

// Host copies (pinned staging -> caller arrays) on up to max_threads threads,
// each taking one contiguous share of the bytes of the list taken as one
// sequence; small totals stay on the calling thread.
struct HostCopy {
  void* dst;
  const void* src;
  size_t bytes;
};
void copy_out(const std::vector<HostCopy>& items, int max_threads) {
  size_t total = 0;
  for (const HostCopy& c : items) total += c.bytes;
  constexpr size_t kPerThread = (size_t)4 << 20;  // below this a thread does not pay for itself
  const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  const int n_thr = (int)std::max<size_t>(1, std::min<size_t>({(size_t)max_threads, (size_t)hw, total / kPerThread}));
  auto part = [&](size_t b0, size_t b1) {  // bytes [b0, b1) of the sequence
    size_t at = 0;
    for (const HostCopy& c : items) {
      const size_t lo = std::max(b0, at), hi = std::min(b1, at + c.bytes);
      if (lo < hi) std::memcpy((char*)c.dst + (lo - at), (const char*)c.src + (lo - at), hi - lo);
      at += c.bytes;
      if (at >= b1) break;
    }
  };
  std::vector<std::thread> th;
  size_t started = 0;  // bytes handed to helper threads
  if (n_thr > 1) {
    const size_t share = (total + n_thr - 1) / n_thr;
    try {
      for (int t = 1; t < n_thr; ++t) {
        const size_t b0 = std::min(total, (size_t)t * share), b1 = std::min(total, b0 + share);
        th.emplace_back(part, b0, b1);
        started = b1;
      }
    } catch (...) {  // a helper that cannot start leaves its share to this thread
    }
    part(0, std::min(total, share));
    if (started < total) part(std::max(share, started), total);
  } else {
    part(0, total);
  }
  for (auto& x : th) x.join();
}

// Device memory of clusters and plans comes from the context's own pool,
// stream-ordered: a free is queued behind the work already on its stream and
// never waits for the device, so retiring a cluster does not stall a serving
// round.  The pool keeps what it has reserved (no release threshold).
cudaError_t pool_alloc(ba_ctx* ctx, void** p, size_t bytes, cudaStream_t st) {
  return cudaMallocFromPoolAsync(p, bytes, ctx->pool, st);
}

bool tune_in_range(const ba_tune& t, bool mixed, std::string* why) {
  const int cmax = chunk_tiles(mixed);
  auto bad = [&](const char* m) {
    *why = m;
    return false;
  };
  if (t.chunk_tiles != 0 && (t.chunk_tiles < 4 || t.chunk_tiles > cmax))
    return bad("chunk_tiles must be 0 or 4 .. 16 (mixed) / 8 (FP64)");
  if (t.lin_ctas_per_sm < 1 || t.lin_ctas_per_sm > 32) return bad("lin_ctas_per_sm must be 1 .. 32");
  if (t.back_ctas_per_sm < 1 || t.back_ctas_per_sm > 32) return bad("back_ctas_per_sm must be 1 .. 32");
  if (t.factor_nb < 2 || t.factor_nb > 32) return bad("factor_nb must be 2 .. 32");
  if (t.factor_threads != 256 && t.factor_threads != 384 && t.factor_threads != 512)
    return bad("factor_threads must be 256, 384 or 512");
  if (t.big_panel_w < 1 || t.big_panel_w > 32 || (32 % t.big_panel_w) != 0)
    return bad("big_panel_w must be 1, 2, 4, 8, 16 or 32");
  if (t.batch_chains < 1 || t.batch_chains > kMaxBatchChains) return bad("batch_chains must be 1 .. 8");
  return true;
}

TuneParams tune_from_abi(const ba_tune& t) {
  TuneParams p;
  p.chunk_tiles = t.chunk_tiles;
  p.lin_ctas_per_sm = t.lin_ctas_per_sm;
  p.back_ctas_per_sm = t.back_ctas_per_sm;
  p.factor_nb = t.factor_nb;
  p.factor_threads = t.factor_threads;
  p.big_panel_w = t.big_panel_w;
  p.batch_chains = t.batch_chains;
  return p;
}

ba_tune tune_to_abi(const TuneParams& p) {
  ba_tune t{};
  t.chunk_tiles = p.chunk_tiles;
  t.lin_ctas_per_sm = p.lin_ctas_per_sm;
  t.back_ctas_per_sm = p.back_ctas_per_sm;
  t.factor_nb = p.factor_nb;
  t.factor_threads = p.factor_threads;
  t.big_panel_w = p.big_panel_w;
  t.batch_chains = p.batch_chains;
  return t;
}

// the autotuned launch parameters into a batch view (grids and CTA shapes
// are fixed when a plan's graph is captured)
void apply_tune(const ba_ctx* ctx, BatchView& bv) {
  bv.lin_ctas_per_sm = ctx->tune.lin_ctas_per_sm;
  bv.back_ctas_per_sm = ctx->tune.back_ctas_per_sm;
  bv.factor_nb = ctx->tune.factor_nb;
  bv.factor_threads = ctx->tune.factor_threads;
  bv.factor_df = ctx->mixed || ctx->small_df;
}

void free_plan(ba_ctx* ctx, Plan* p) {
  for (auto& kv : p->graphs) {
    cudaGraphExecDestroy(kv.second.exec);  // an executing graph is freed when it completes
    free_probe(kv.second.probe);
  }
  if (p->dbuf) cudaFreeAsync(p->dbuf, ctx->stream);
  if (p->done) cudaEventDestroy(p->done);
  delete p;
}

void drop_plans_with(ba_ctx* ctx, ba_cluster_id id) {
  for (auto it = ctx->plans.begin(); it != ctx->plans.end();) {
    if (std::find(it->first.begin(), it->first.end(), id) != it->first.end()) {
      ctx->mem -= it->second->dbuf_bytes;
      free_plan(ctx, it->second);
      it = ctx->plans.erase(it);
    } else {
      ++it;
    }
  }
}

ba_status get_plan(ba_ctx* ctx, const std::vector<ba_cluster_id>& ids, Plan** out) {
  auto it = ctx->plans.find(ids);
  if (it != ctx->plans.end()) {
    *out = it->second;
    return BA_OK;
  }
  const int n = (int)ids.size();
  std::vector<DevCluster> descs(n);
  std::vector<int> pre(3 * (size_t)(n + 1), 0);
  int max_n = 6, big_max = 0;
  for (int i = 0; i < n; ++i) {
    Cluster* c = find_cluster(ctx, ids[i]);
    if (!c) return set_err(ctx, BA_ERR_NOT_FOUND, "unknown cluster id in batch");
    descs[i] = c->h;
    pre[i + 1] = pre[i] + c->h.n_tiles;
    pre[(n + 1) + i + 1] = pre[(n + 1) + i] + c->h.n_chunks;
    pre[2 * (n + 1) + i + 1] = pre[2 * (n + 1) + i] + c->h.n_free + c->h.n_pairs;
    if (c->nf <= kMaxFreeSmall) max_n = std::max(max_n, 6 * c->h.n_free);
    else big_max = std::max(big_max, 6 * c->nf);
  }
  ba_status st = ensure_attrs(ctx, std::max(max_n, big_max));
  if (st != BA_OK) return st;
  Plan* p = new Plan();
  p->ids = ids;
  auto big_ref = [&](const Cluster* c) {
    return BigRef{c->d_desc, 6 * c->nf, c->nf, c->h.n_pairs, c->h.S, c->h.F, c->big_below, !ctx->big_fp64,
                  ctx->tune.big_panel_w};
  };
  for (int i = 0; i < n; ++i) {
    Cluster* c = find_cluster(ctx, ids[i]);
    if (c->nf > kMaxFreeSmall) p->big.push_back(big_ref(c));
  }
  pre.push_back(pre[n]);  // totals, read by the kernels
  pre.push_back(pre[(n + 1) + n]);
  pre.push_back(pre[2 * (n + 1) + n]);
  Layout L;
  const size_t o_desc = L.add(sizeof(DevCluster) * n);
  const size_t o_pre = L.add(sizeof(int) * pre.size());
  const size_t o_lm = L.add(sizeof(LmState) * n);
  const size_t o_gn = L.add(sizeof(double) * n);
  const size_t o_ord = L.add(sizeof(int) * n);
  std::vector<int> order(n);  // factor kernel: largest reduced systems first
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return descs[a].n_free > descs[b].n_free; });
  // The LM iterations run as tune.batch_chains concurrent chains of launches over
  // disjoint parts of the batch, so that one chain's kernels fill the SMs
  // another chain's kernels leave idle (the factor's largest systems, the
  // grids' last waves, the gaps between launches).  Clusters are dealt to
  // the chains in order of decreasing reduced-system size; a chain lists its
  // clusters in batch order.  Every cluster's arithmetic is its own, so the
  // results do not depend on the split.
  struct ChainHost {
    std::vector<int> mem;  // batch indices
    std::vector<DevCluster> descs;
    std::vector<int> pre, ord;
    size_t o_desc = 0, o_pre = 0, o_ord = 0;
    int max_n = 6;
  };
  const int n_chains = std::min(n, ctx->tune.batch_chains);
  std::vector<ChainHost> chh(n_chains > 1 ? n_chains : 0);
  for (int r = 0; r < n && n_chains > 1; ++r) chh[r % n_chains].mem.push_back(order[r]);
  for (ChainHost& h : chh) {
    std::sort(h.mem.begin(), h.mem.end());
    const int m = (int)h.mem.size();
    h.pre.assign(3 * (size_t)(m + 1), 0);
    for (int i = 0; i < m; ++i) {
      const DevCluster& d = descs[h.mem[i]];
      h.descs.push_back(d);
      h.pre[i + 1] = h.pre[i] + d.n_tiles;
      h.pre[(m + 1) + i + 1] = h.pre[(m + 1) + i] + d.n_chunks;
      h.pre[2 * (m + 1) + i + 1] = h.pre[2 * (m + 1) + i] + d.n_free + d.n_pairs;
      if (find_cluster(ctx, ids[h.mem[i]])->nf <= kMaxFreeSmall) h.max_n = std::max(h.max_n, 6 * d.n_free);
    }
    h.pre.push_back(h.pre[m]);
    h.pre.push_back(h.pre[(m + 1) + m]);
    h.pre.push_back(h.pre[2 * (m + 1) + m]);
    h.ord.resize(m);
    for (int i = 0; i < m; ++i) h.ord[i] = i;
    std::stable_sort(h.ord.begin(), h.ord.end(),
                     [&](int a, int b) { return h.descs[a].n_free > h.descs[b].n_free; });
    h.o_desc = L.add(sizeof(DevCluster) * m);
    h.o_pre = L.add(sizeof(int) * h.pre.size());
    h.o_ord = L.add(sizeof(int) * m);
  }
  p->dbuf_bytes = L.off;
  if (ctx->budget && ctx->mem + p->dbuf_bytes > ctx->budget) {
    delete p;
    return set_err(ctx, BA_ERR_BUDGET, "batch plan exceeds the device-memory budget");
  }
  // allocated and filled on the plan stream and waited for there: the
  // solves already queued on the context's stream (another batch still on
  // the device) are not waited for
  cudaError_t e = pool_alloc(ctx, (void**)&p->dbuf, p->dbuf_bytes, ctx->plan_stream);
  if (e != cudaSuccess) {
    delete p;
    return set_err(ctx, BA_ERR_CUDA, std::string("plan allocation: ") + cudaGetErrorString(e));
  }
  ctx->mem += p->dbuf_bytes;
  const cudaStream_t ps = ctx->plan_stream;
  e = cudaMemcpyAsync(p->dbuf + o_desc, descs.data(), sizeof(DevCluster) * n, cudaMemcpyHostToDevice, ps);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->dbuf + o_pre, pre.data(), sizeof(int) * pre.size(), cudaMemcpyHostToDevice, ps);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->dbuf + o_ord, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice, ps);
  for (const ChainHost& h : chh) {
    const size_t m = h.mem.size();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(p->dbuf + h.o_desc, h.descs.data(), sizeof(DevCluster) * m, cudaMemcpyHostToDevice, ps);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(p->dbuf + h.o_pre, h.pre.data(), sizeof(int) * h.pre.size(), cudaMemcpyHostToDevice, ps);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(p->dbuf + h.o_ord, h.ord.data(), sizeof(int) * m, cudaMemcpyHostToDevice, ps);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(ps);
  if (e != cudaSuccess) {
    ctx->mem -= p->dbuf_bytes;
    free_plan(ctx, p);
    return set_err(ctx, BA_ERR_CUDA, std::string("plan upload: ") + cudaGetErrorString(e));
  }
  const int* dpre = (const int*)(p->dbuf + o_pre);
  p->bv.cl = (const DevCluster*)(p->dbuf + o_desc);
  p->bv.tile_pre = dpre;
  p->bv.chunk_pre = dpre + (n + 1);
  p->bv.item_pre = dpre + 2 * (n + 1);
  p->bv.factor_order = (const int*)(p->dbuf + o_ord);
  p->bv.tot = dpre + 3 * (n + 1);
  p->bv.n = n;
  p->bv.total_tiles = pre[n];
  p->bv.total_chunks = pre[(n + 1) + n];
  p->bv.total_items = pre[2 * (n + 1) + n];
  p->bv.max_n = max_n;
  p->bv.inject = ctx->inject;
  apply_tune(ctx, p->bv);
  for (const ChainHost& h : chh) {
    const int m = (int)h.mem.size();
    Chain c;
    const int* cpre = (const int*)(p->dbuf + h.o_pre);
    c.bv.cl = (const DevCluster*)(p->dbuf + h.o_desc);
    c.bv.tile_pre = cpre;
    c.bv.chunk_pre = cpre + (m + 1);
    c.bv.item_pre = cpre + 2 * (m + 1);
    c.bv.factor_order = (const int*)(p->dbuf + h.o_ord);
    c.bv.tot = cpre + 3 * (m + 1);
    c.bv.n = m;
    c.bv.total_tiles = h.pre[m];
    c.bv.total_chunks = h.pre[(m + 1) + m];
    c.bv.total_items = h.pre[2 * (m + 1) + m];
    c.bv.max_n = h.max_n;
    c.bv.inject = ctx->inject;
    apply_tune(ctx, c.bv);
    for (int i : h.mem) {
      const Cluster* cc = find_cluster(ctx, ids[i]);
      if (cc->nf > kMaxFreeSmall) c.big.push_back(big_ref(cc));
    }
    p->chains.push_back(std::move(c));
  }
  p->lm_out = (LmState*)(p->dbuf + o_lm);
  p->gnorm = (double*)(p->dbuf + o_gn);
  ctx->plans[ids] = p;
  *out = p;
  return BA_OK;
}

// Streams and events for forking k - 1 chains off the context's stream
// inside a capture (created once, kept until shutdown).
ba_status ensure_chain_streams(ba_ctx* ctx, int k) {
  if (!ctx->chain_fork) CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->chain_fork, cudaEventDisableTiming));
  while ((int)ctx->chain_streams.size() < k - 1) {
    cudaStream_t cs = nullptr;
    cudaEvent_t ce = nullptr;
    CUDA_TRY(ctx, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    const cudaError_t e = cudaEventCreateWithFlags(&ce, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      cudaStreamDestroy(cs);
      return set_err(ctx, BA_ERR_CUDA, std::string("chain event: ") + cudaGetErrorString(e));
    }
    ctx->chain_streams.push_back(cs);
    ctx->chain_join.push_back(ce);
  }
  return BA_OK;
}

// Inside a capture on the context's stream: the plan's chains, chain 0 on
// the context's stream and chain c on chain_streams[c - 1], forked after
// what the stream holds and joined back into it.
cudaError_t capture_chains(ba_ctx* ctx, Plan* p, int iters) {
  const int k = (int)p->chains.size();
  cudaError_t e = cudaEventRecord(ctx->chain_fork, ctx->stream);
  for (int c = 1; c < k && e == cudaSuccess; ++c) e = cudaStreamWaitEvent(ctx->chain_streams[c - 1], ctx->chain_fork, 0);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < iters; ++i)
    for (int c = 0; c < k; ++c)
      launch_iteration(p->chains[c].bv, ctx->mixed, ctx->refine, c == 0 ? ctx->stream : ctx->chain_streams[c - 1],
                       &p->chains[c].big);
  for (int c = 1; c < k && e == cudaSuccess; ++c) {
    e = cudaEventRecord(ctx->chain_join[c - 1], ctx->chain_streams[c - 1]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->chain_join[c - 1], 0);
  }
  return e;
}

// iters LM iterations on the plan's clusters as one graph launch:
// arm -> cost at the current state -> iters x (K1..K6), the iterations as
// the plan's concurrent chains when it has more than one.
ba_status run_plan(ba_ctx* ctx, Plan* p, int iters) {
  auto it = p->graphs.find(iters);
  if (it == p->graphs.end()) {
    GraphRec g;
    cudaGraph_t graph = nullptr;
    if (!p->chains.empty()) {
      const ba_status cst = ensure_chain_streams(ctx, (int)p->chains.size());
      if (cst != BA_OK) return cst;
    }
    note_direct(ctx);
    take_captured_launches();
    if (ctx->timing) {
      g.probe = new Probe();
      set_probe(g.probe);
    }
    CUDA_TRY(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    launch_arm(p->bv, iters, ctx->stream);
    launch_cost_init(p->bv, ctx->mixed, ctx->stream);
    cudaError_t ec = cudaSuccess;
    if (p->chains.empty()) {
      for (int i = 0; i < iters; ++i) launch_iteration(p->bv, ctx->mixed, ctx->refine, ctx->stream, &p->big);
    } else {
      ec = capture_chains(ctx, p, iters);
    }
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
    if (e == cudaSuccess && ec != cudaSuccess) {
      cudaGraphDestroy(graph);
      graph = nullptr;
      e = ec;
    }
    set_probe(nullptr);
    g.kernels = take_captured_launches();
    if (e != cudaSuccess) {
      free_probe(g.probe);
      return set_err(ctx, BA_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      free_probe(g.probe);
      return set_err(ctx, BA_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    it = p->graphs.emplace(iters, g).first;
  }
  CUDA_TRY(ctx, cudaGraphLaunch(it->second.exec, ctx->stream));
  ctx->launches += it->second.kernels;
  p->last = &it->second;
  return BA_OK;
}

// After the stream has synchronised: fold the last graph's event times into
// the per-kernel statistics.
void fold_probe(ba_ctx* ctx, const Probe* pr) {
  std::lock_guard<std::mutex> g(ctx->stats_mu);
  for (auto& r : pr->recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.e0, r.e1) == cudaSuccess) ctx->kms[r.kind] += ms;
    ctx->klaunch[r.kind] += 1;
  }
}

void collect_timing(ba_ctx* ctx, Plan* p) {
  if (!ctx->timing || !p->last || !p->last->probe) return;
  fold_probe(ctx, p->last->probe);
}

void fill_step(const StepRec& r, ba_step_info* o) {
  o->accepted = r.accepted;
  o->status = r.status;
  o->F_before = r.F_before;
  o->F_after = r.F_after;
  o->predicted = r.predicted;
  o->gain = r.gain;
  o->mu_used = r.mu_used;
  o->mu = r.mu;
  o->nu = r.nu;
}

// Runs iters iterations on ids and returns per-cluster LM state and traces.
// With lk (holding the context's lock), the lock is released while the host
// waits for the device and taken again before returning; the caller keeps
// the batch's clusters out of every other call meanwhile (in_service).
ba_status run_and_collect(ba_ctx* ctx, const std::vector<ba_cluster_id>& ids, int iters, std::vector<LmState>* lm,
                          std::vector<StepRec>* trace, std::unique_lock<std::mutex>* lk = nullptr) {
  Plan* p = nullptr;
  ba_status st = get_plan(ctx, ids, &p);
  if (st != BA_OK) return st;
  const int n = (int)ids.size();
  st = run_plan(ctx, p, iters);
  if (st != BA_OK) return st;
  StepRec* dtrace = nullptr;
  const int tcap = std::min(iters, kTraceCap);
  if (trace && tcap > 0) {
    CUDA_TRY(ctx, cudaMallocAsync((void**)&dtrace, sizeof(StepRec) * (size_t)n * tcap, ctx->stream));
  }
  launch_gather(p->bv, tcap, p->lm_out, dtrace, ctx->stream);
  // The results go to pageable host memory, a copy that waits on the host
  // for the whole batch.  It is issued on the context's copy stream behind
  // the batch's event, and with lk after the lock has been released: other
  // threads (cluster creation) are not held up for the duration of the
  // solve, and nothing lands on the context's stream without the lock.
  struct Relock {
    std::unique_lock<std::mutex>* lk;
    ~Relock() {
      if (lk && !lk->owns_lock()) lk->lock();
    }
  } relock{lk};
  // the waiting thread sleeps instead of spinning: the host threads stay
  // free for cluster creation meanwhile
  if (!p->done) CUDA_TRY(ctx, cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming | cudaEventBlockingSync));
  CUDA_TRY(ctx, cudaEventRecord(p->done, ctx->stream));
  if (lk) lk->unlock();
  const cudaStream_t cs = ctx->copy_stream;
  CUDA_TRY(ctx, cudaEventSynchronize(p->done));
  if (lm) {
    lm->resize(n);
    CUDA_TRY(ctx, cudaMemcpyAsync(lm->data(), p->lm_out, sizeof(LmState) * n, cudaMemcpyDeviceToHost, cs));
  }
  if (trace && dtrace) {
    trace->assign((size_t)n * tcap, StepRec{});
    CUDA_TRY(ctx, cudaMemcpyAsync(trace->data(), dtrace, sizeof(StepRec) * (size_t)n * tcap, cudaMemcpyDeviceToHost, cs));
    CUDA_TRY(ctx, cudaFreeAsync(dtrace, cs));
  }
  CUDA_TRY(ctx, cudaStreamSynchronize(cs));
  if (lk) lk->lock();
  CUDA_TRY(ctx, cudaGetLastError());
  note_direct(ctx);
  collect_timing(ctx, p);
  return BA_OK;
}

// ------------------------------------------------------------------ cluster creation

// f(begin, end) over [0, n) in n_thr contiguous ranges, the first on the
// calling thread; a helper that cannot start leaves its range to the calling
// thread.  f must write disjoint outputs per range.
template <class F>
void par_ranges(int n_thr, size_t n, const F& f) {
  if (n_thr <= 1 || n < 2) {
    f((size_t)0, n);
    return;
  }
  const size_t share = (n + n_thr - 1) / n_thr;
  std::vector<std::thread> th;
  size_t started = std::min(n, share);  // [0, share) is the calling thread's
  try {
    for (int t = 1; t < n_thr && started < n; ++t) {
      const size_t b0 = started, b1 = std::min(n, b0 + share);
      th.emplace_back([&f, b0, b1] { f(b0, b1); });
      started = b1;
    }
  } catch (...) {
  }
  f((size_t)0, std::min(n, share));
  if (started < n) f(started, n);
  for (auto& x : th) x.join();
}

// ------------------------------------------------------------------ presort self-check

// ba_presort_host runs build_cluster with a probe: the chunk tables on a
// given number of threads, and instead of the upload a check of the tables.
struct PresortProbe {
  int threads = 0;  // > 0: the chunk tables on exactly this many threads
  ba_presort_info* out = nullptr;
};

// The presorted tables of one cluster, as build_cluster holds them before
// staging.
struct PresortView {
  int nc, np, no, nf, tiles_per_chunk, obs_per_chunk;
  const int32_t* ocam;
  const int32_t* opt;
  const std::vector<int>& free_idx;
  const std::vector<int>& perm;
  const std::vector<int>& inv;
  const std::vector<int>& pm;
  const std::vector<int>& pt_start;
  const std::vector<int>& pcam;
  const std::vector<int>& ppt;
  const std::vector<Tile>& tiles;
  const std::vector<Chunk>& chunks;
  const std::vector<Job>& jobs;
  const std::vector<unsigned short>& cm_list;
  const std::vector<unsigned char>& lane_job;
  const std::vector<unsigned int>& pent;
  const std::vector<int2>& pair_key;
  const std::vector<int>& cam_slot_begin;
  const std::vector<int>& cam_slots;
  const std::vector<int>& pair_slot_begin;
  const std::vector<int>& pair_slots;
  const std::vector<int>& fpos;
  const std::vector<int>& env_first;
};

// Checks every table against what the observations alone imply, the
// expected contents rebuilt here by brute force (not by the presort's own
// steps), and reports the sizes and an FNV-1a digest of the tables.  A
// failed check counts in checks_failed; message names the first.
void check_presort(const PresortView& V, ba_presort_info* o) {
  int failed = 0;
  auto fail = [&](const char* what) {
    if (failed++ == 0) std::snprintf(o->message, sizeof(o->message), "%s", what);
  };
  const int no = V.no, np = V.np, nf = V.nf;
  // caller <-> internal point order, point-major order (points ascending,
  // cameras strictly ascending within a point)
  {
    bool ok = (int)V.perm.size() == np && (int)V.inv.size() == np;
    for (int j = 0; ok && j < np; ++j) ok = V.perm[j] >= 0 && V.perm[j] < np && V.inv[V.perm[j]] == j;
    if (!ok) fail("point order: perm and inv are not inverse permutations");
  }
  {
    std::vector<char> seen(no, 0);
    bool ok = (int)V.pm.size() == no;
    for (int p = 0; ok && p < no; ++p) {
      const int i = V.pm[p];
      if (i < 0 || i >= no || seen[i]) {
        ok = false;
        break;
      }
      seen[i] = 1;
      ok = V.pcam[p] == V.ocam[i] && V.ppt[p] == V.inv[V.opt[i]] &&
           (p == 0 || V.ppt[p] > V.ppt[p - 1] || (V.ppt[p] == V.ppt[p - 1] && V.pcam[p] > V.pcam[p - 1]));
    }
    if (!ok) fail("point-major order");
    std::vector<int> cnt(np + 1, 0);
    for (int i = 0; i < no; ++i) ++cnt[V.inv[V.opt[i]] + 1];
    for (int j = 0; j < np; ++j) cnt[j + 1] += cnt[j];
    if (V.pt_start != cnt) fail("point starts");
  }
  // tiles: consecutive runs of whole points, 1..32 observations, covering all
  {
    int at = 0;
    bool ok = true;
    for (const Tile& t : V.tiles) {
      ok = ok && t.obs_begin == at && t.n_obs >= 1 && t.n_obs <= 32 &&
           (at == 0 || V.ppt[at] != V.ppt[at - 1]);
      at += t.n_obs;
    }
    if (!ok || at != no) fail("tiles");
  }
  // chunks: consecutive tiles; jobs consecutive, image jobs first
  {
    int tt = 0, jb = 0;
    bool ok = true;
    for (const Chunk& ch : V.chunks) {
      int n_obs = 0;
      for (int t = ch.tile_begin; t < ch.tile_begin + ch.n_tiles && t < (int)V.tiles.size(); ++t)
        n_obs += V.tiles[t].n_obs;
      ok = ok && ch.tile_begin == tt && ch.n_tiles >= 1 && ch.n_tiles <= V.tiles_per_chunk &&
           tt + ch.n_tiles <= (int)V.tiles.size() && ch.obs_begin == V.tiles[tt].obs_begin && ch.n_obs == n_obs &&
           ch.n_obs <= V.obs_per_chunk && ch.pt_begin == V.ppt[ch.obs_begin] &&
           ch.n_pts == V.ppt[ch.obs_begin + ch.n_obs - 1] - ch.pt_begin + 1 && ch.job_begin == jb &&
           ch.n_lc >= 0 && ch.n_lp >= 0;
      if (!ok) break;
      tt += ch.n_tiles;
      jb += ch.n_lc + ch.n_lp;
    }
    if (!ok || tt != (int)V.tiles.size() || jb != (int)V.jobs.size()) {
      fail("chunks");
      o->checks_failed = failed;
      return;  // the job checks below walk the chunks
    }
  }
  // slot -> free camera and slot -> pair, from the grouped slot lists
  const int n_pairs = (int)V.pair_key.size();
  int n_cslots = 0, n_pslots = 0;
  for (const Chunk& ch : V.chunks) {
    n_cslots += ch.n_lc;
    n_pslots += ch.n_lp;
  }
  std::vector<int> slot_cam(n_cslots, -1), slot_pair(n_pslots, -1);
  {
    bool ok = (int)V.cam_slot_begin.size() == nf + 1 && V.cam_slot_begin[0] == 0 &&
              V.cam_slot_begin[nf] == n_cslots && (int)V.cam_slots.size() == n_cslots;
    for (int f = 0; ok && f < nf; ++f)
      for (int k = V.cam_slot_begin[f]; ok && k < V.cam_slot_begin[f + 1]; ++k) {
        const int sl = V.cam_slots[k];
        ok = sl >= 0 && sl < n_cslots && slot_cam[sl] < 0 && (k == V.cam_slot_begin[f] || sl > V.cam_slots[k - 1]);
        if (ok) slot_cam[sl] = f;
      }
    ok = ok && (int)V.pair_slot_begin.size() == n_pairs + 1 && V.pair_slot_begin[0] == 0 &&
         V.pair_slot_begin[n_pairs] == n_pslots && (int)V.pair_slots.size() == n_pslots;
    for (int q = 0; ok && q < n_pairs; ++q)
      for (int k = V.pair_slot_begin[q]; ok && k < V.pair_slot_begin[q + 1]; ++k) {
        const int sl = V.pair_slots[k];
        ok = sl >= 0 && sl < n_pslots && slot_pair[sl] < 0 && (k == V.pair_slot_begin[q] || sl > V.pair_slots[k - 1]);
        if (ok) slot_pair[sl] = q;
      }
    if (!ok) {
      fail("slot groups");
      o->checks_failed = failed;
      return;
    }
  }
  // jobs: per chunk, one image job per free camera observed in it and one
  // pair job per co-visible free pair, with exactly the items the
  // observations imply, counts non-increasing (ties by camera / key), slots
  // in job order; pairs numbered by first appearance
  {
    bool ok = true;
    int cs = 0, ps = 0;
    std::vector<char> pair_seen(n_pairs, 0);
    int next_pair = 0;
    for (size_t c = 0; ok && c < V.chunks.size(); ++c) {
      const Chunk& ch = V.chunks[c];
      std::map<int, std::vector<unsigned>> want_cam, want_pair;
      for (int j = ch.pt_begin; j < ch.pt_begin + ch.n_pts; ++j)
        for (int a = V.pt_start[j]; a < V.pt_start[j + 1]; ++a) {
          const int fa = V.free_idx[V.pcam[a]];
          if (fa < 0) continue;
          want_cam[fa].push_back((unsigned)(a - ch.obs_begin));
          for (int b = a + 1; b < V.pt_start[j + 1]; ++b) {
            const int fb = V.free_idx[V.pcam[b]];
            if (fb >= 0)
              want_pair[fa * nf + fb].push_back((unsigned)(a - ch.obs_begin) | ((unsigned)(b - ch.obs_begin) << 16));
          }
        }
      for (auto& kv : want_cam)  // items of a camera, ascending
        std::sort(kv.second.begin(), kv.second.end());
      ok = ch.n_lc == (int)want_cam.size() && ch.n_lp == (int)want_pair.size();
      for (int q = 0; ok && q < ch.n_lc; ++q) {
        const Job& jb = V.jobs[ch.job_begin + q];
        ok = jb.slot == cs++;
        if (!ok) break;
        const int f = slot_cam[jb.slot];
        auto it = want_cam.find(f);
        ok = it != want_cam.end() && jb.count == (int)it->second.size() && jb.item_begin >= 0 &&
             jb.item_begin + (size_t)jb.count <= V.cm_list.size();
        for (int k = 0; ok && k < jb.count; ++k) ok = V.cm_list[jb.item_begin + k] == it->second[k];
        if (ok && q > 0) {
          const Job& pv = V.jobs[ch.job_begin + q - 1];
          ok = pv.count > jb.count || (pv.count == jb.count && slot_cam[pv.slot] < f);
        }
      }
      for (int q = 0; ok && q < ch.n_lp; ++q) {
        const Job& jb = V.jobs[ch.job_begin + ch.n_lc + q];
        ok = jb.slot == ps++;
        if (!ok) break;
        const int pi = slot_pair[jb.slot];
        const int key = V.pair_key[pi].x * nf + V.pair_key[pi].y;
        if (!pair_seen[pi]) {  // first appearance: the next pair index
          ok = pi == next_pair++;
          pair_seen[pi] = 1;
        }
        auto it = want_pair.find(key);
        ok = ok && V.pair_key[pi].x < V.pair_key[pi].y && it != want_pair.end() &&
             jb.count == (int)it->second.size() && jb.item_begin >= 0 &&
             jb.item_begin + (size_t)jb.count <= V.pent.size();
        for (int k = 0; ok && k < jb.count; ++k) ok = V.pent[jb.item_begin + k] == it->second[k];
        if (ok && q > 0) {
          const Job& pv = V.jobs[ch.job_begin + ch.n_lc + q - 1];
          const int pkey = V.pair_key[slot_pair[pv.slot]].x * nf + V.pair_key[slot_pair[pv.slot]].y;
          ok = pv.count > jb.count || (pv.count == jb.count && pkey < key);
        }
      }
    }
    if (ok) ok = next_pair == n_pairs;
    size_t cm_total = 0, pe_total = 0;
    for (const Chunk& ch : V.chunks) {
      for (int q = 0; q < ch.n_lc; ++q) cm_total += V.jobs[ch.job_begin + q].count;
      for (int q = 0; q < ch.n_lp; ++q) pe_total += V.jobs[ch.job_begin + ch.n_lc + q].count;
    }
    if (ok) ok = cm_total == V.cm_list.size() && pe_total == V.pent.size();
    if (!ok) fail("jobs and their items");
  }
  // lanes: a run of at least one lane (at most one per item) per job, runs in
  // job order within the CTA; lane t runs the last job whose run starts at or
  // before t; chunks with more jobs than threads: one lane per job
  int max_lanes = 0, fallback = 0;
  {
    bool ok = V.lane_job.size() == V.chunks.size() * (size_t)kChunkThreads;
    for (size_t c = 0; ok && c < V.chunks.size(); ++c) {
      const Chunk& ch = V.chunks[c];
      const int nj = ch.n_lc + ch.n_lp;
      const unsigned char* row = V.lane_job.data() + c * kChunkThreads;
      if (nj == 0 || nj > kChunkThreads) {
        fallback += nj > kChunkThreads;
        for (int q = 0; ok && q < nj; ++q)
          ok = V.jobs[ch.job_begin + q].lane_begin == 0 && V.jobs[ch.job_begin + q].n_lanes == 1;
        for (int t = 0; ok && t < kChunkThreads; ++t) ok = row[t] == 0;
        continue;
      }
      int end = 0;
      for (int q = 0; ok && q < nj; ++q) {
        const Job& jb = V.jobs[ch.job_begin + q];
        ok = jb.n_lanes >= 1 && jb.n_lanes <= std::max(1, jb.count) && jb.lane_begin >= end &&
             (q > 0 || jb.lane_begin == 0);
        end = jb.lane_begin + jb.n_lanes;
      }
      ok = ok && end <= kChunkThreads;
      max_lanes = std::max(max_lanes, end);
      for (int t = 0, q = 0; ok && t < kChunkThreads; ++t) {
        while (q + 1 < nj && V.jobs[ch.job_begin + q + 1].lane_begin <= t) ++q;
        ok = row[t] == q;
      }
    }
    if (!ok) fail("lanes");
  }
  // elimination order: a permutation whose envelope holds every co-visible pair
  {
    bool ok = (int)V.fpos.size() == nf && (int)V.env_first.size() == nf;
    std::vector<char> seen(nf, 0);
    for (int f = 0; ok && f < nf; ++f) {
      ok = V.fpos[f] >= 0 && V.fpos[f] < nf && !seen[V.fpos[f]];
      if (ok) seen[V.fpos[f]] = 1;
    }
    for (int p = 0; ok && p < nf; ++p) ok = V.env_first[p] >= 0 && V.env_first[p] <= p && (p == 0 || V.env_first[p] >= V.env_first[p - 1]);
    for (const int2& k : V.pair_key) {
      if (!ok) break;
      const int a = V.fpos[k.x], b = V.fpos[k.y];
      ok = V.env_first[std::max(a, b)] <= std::min(a, b);
    }
    if (!ok) fail("elimination order and envelope");
  }
  // sizes and digest
  unsigned long long h = 1469598103934665603ull;
  auto mix = [&](const void* p, size_t bytes) {
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < bytes; ++i) {
      h ^= b[i];
      h *= 1099511628211ull;
    }
  };
  mix(V.pm.data(), sizeof(int) * V.pm.size());
  mix(V.tiles.data(), sizeof(Tile) * V.tiles.size());
  mix(V.chunks.data(), sizeof(Chunk) * V.chunks.size());
  mix(V.jobs.data(), sizeof(Job) * V.jobs.size());
  mix(V.cm_list.data(), sizeof(unsigned short) * V.cm_list.size());
  mix(V.lane_job.data(), V.lane_job.size());
  mix(V.pent.data(), sizeof(unsigned int) * V.pent.size());
  mix(V.pair_key.data(), sizeof(int2) * V.pair_key.size());
  mix(V.cam_slots.data(), sizeof(int) * V.cam_slots.size());
  mix(V.pair_slots.data(), sizeof(int) * V.pair_slots.size());
  mix(V.fpos.data(), sizeof(int) * V.fpos.size());
  mix(V.env_first.data(), sizeof(int) * V.env_first.size());
  o->n_free = nf;
  o->n_tiles = (int32_t)V.tiles.size();
  o->n_chunks = (int32_t)V.chunks.size();
  o->n_pairs = n_pairs;
  o->n_cam_jobs = n_cslots;
  o->n_pair_jobs = n_pslots;
  o->max_lanes = max_lanes;
  o->fallback_chunks = fallback;
  o->tiles_per_chunk = V.tiles_per_chunk;
  o->checks_failed = failed;
  o->n_free_obs = (int64_t)V.cm_list.size();
  o->n_pair_entries = (int64_t)V.pent.size();
  o->digest = h;
}

// A one-cluster view for the kernels that only walk the descriptor table
// (camera records, warm start): no prefix sums, no device allocation.
BatchView one_view(const DevCluster* d_desc, int n_free) {
  BatchView bv{};
  bv.cl = d_desc;
  bv.n = 1;
  bv.max_n = 6 * n_free;
  return bv;
}

// Host copy of the mixed path's camera record (write_camdf's layout and
// values: hi = the binary64 value rounded to binary32, lo = the remainder
// rounded to binary32)
void host_camdf(float* o, const double* R, const double* T, const double* intr, bool is_free) {
  auto split = [](double v, float* hi, float* lo) {
    *hi = (float)v;
    *lo = (float)(v - (double)*hi);
  };
  for (int i = 0; i < 9; ++i) split(R[i], &o[i], &o[24 + i]);
  for (int i = 0; i < 3; ++i) split(T[i], &o[9 + i], &o[12 + i]);
  split(intr[0], &o[15], &o[33]);
  for (int i = 0; i < 4; ++i) split(intr[3 + i], &o[16 + i], &o[34 + i]);
  o[20] = is_free ? 1.0f : 0.0f;
  for (int i = 21; i < 24; ++i) o[i] = 0.0f;
  for (int i = 38; i < kCamDf; ++i) o[i] = 0.0f;
}

ba_status build_cluster(ba_ctx* ctx, const ba_cluster_desc* d, Cluster* c, const PresortProbe* probe = nullptr) {
  const auto t_start = std::chrono::steady_clock::now();
  struct InFlight {
    std::atomic<int>& n;
    explicit InFlight(std::atomic<int>& v) : n(v) { ++n; }
    ~InFlight() { --n; }
  } in_flight(ctx->creating);
  const int nc = d->n_cams, np = d->n_pts, no = d->n_obs;
  if (nc < 1 || np < 0 || no < 0) return set_err(ctx, BA_ERR_INVALID, "n_cams must be >= 1, n_pts and n_obs >= 0");
  if (d->ptr_kind != BA_PTR_HOST && d->ptr_kind != BA_PTR_DEVICE) return set_err(ctx, BA_ERR_INVALID, "bad ptr_kind");
  if (!(d->sigma_px > 0.0) || !(d->huber_delta_px > 0.0) || !(d->sigma_gnss_m >= 0.0) || !(d->sigma_imu_rad >= 0.0))
    return set_err(ctx, BA_ERR_INVALID, "sigma_px and huber_delta_px must be > 0, prior sigmas >= 0");
  const int kind = d->ptr_kind;
  In<double> intr, R, T, X, Rp, Tp, uv;
  In<int32_t> ocam, opt;
  In<uint8_t> fixed;
  if (!fetch(d->intr, (size_t)nc * 7, kind, intr) || !fetch(d->R, (size_t)nc * 9, kind, R) ||
      !fetch(d->T, (size_t)nc * 3, kind, T) || !fetch(d->X, (size_t)np * 3, kind, X) ||
      !fetch(d->R_prior, (size_t)nc * 9, kind, Rp) || !fetch(d->T_prior, (size_t)nc * 3, kind, Tp) ||
      !fetch(d->obs_uv, (size_t)no * 2, kind, uv) || !fetch(d->obs_cam, (size_t)no, kind, ocam) ||
      !fetch(d->obs_pt, (size_t)no, kind, opt))
    return set_err(ctx, BA_ERR_INVALID, "missing input array (NULL pointer or failed device read)");
  if (d->fixed) {
    if (!fetch(d->fixed, (size_t)nc, kind, fixed)) return set_err(ctx, BA_ERR_INVALID, "bad fixed array");
  } else {
    fixed.own.assign(nc, 0);
    fixed.p = fixed.own.data();
    fixed.n = nc;
  }
  if (!all_finite(intr) || !all_finite(R) || !all_finite(T) || !all_finite(X) || !all_finite(Rp) ||
      !all_finite(Tp) || !all_finite(uv))
    return set_err(ctx, BA_ERR_INVALID, "non-finite value in the input");
  {
    unsigned bad = 0;  // one branch-free pass over both index arrays
    for (int i = 0; i < no; ++i)
      bad |= (unsigned)((uint32_t)ocam[i] >= (uint32_t)nc) | (unsigned)((uint32_t)opt[i] >= (uint32_t)np);
    if (bad) return set_err(ctx, BA_ERR_INVALID, "observation index out of range");
  }
  // threads for the staging gathers: a few when few creations share the host
  // (hardware threads / creations in flight, at most 4), none for small
  // clusters (a thread start costs tens of microseconds); no result depends
  // on the split
  const int hw_threads = (int)std::max(1u, std::thread::hardware_concurrency());
  const int par = probe && probe->threads > 0 ? probe->threads
                                              : std::max(1, std::min(4, hw_threads / std::max(1, ctx->creating.load())));
  auto par_for = [&](size_t n, const auto& f) { par_ranges(n >= ((size_t)1 << 16) ? par : 1, n, f); };

  // free cameras, in camera order
  std::vector<int> free_idx(nc, -1), cam_of_free;
  for (int k = 0; k < nc; ++k)
    if (!fixed[k]) {
      free_idx[k] = (int)cam_of_free.size();
      cam_of_free.push_back(k);
    }
  const int nf = (int)cam_of_free.size();
  if (nf == 0) return set_err(ctx, BA_ERR_INVALID, "no free camera");
  if (nf > kMaxFree) return set_err(ctx, BA_ERR_INVALID, "more than 1024 free cameras in one cluster");

  // internal point order: Morton code of the initial ground position (x, y),
  // ties by the caller's index, so that consecutive points share cameras
  std::vector<int> perm(np), inv(np);  // internal -> caller, caller -> internal
  {
    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
    for (int j = 0; j < np; ++j) {
      xmin = std::min(xmin, X[3 * (size_t)j]); xmax = std::max(xmax, X[3 * (size_t)j]);
      ymin = std::min(ymin, X[3 * (size_t)j + 1]); ymax = std::max(ymax, X[3 * (size_t)j + 1]);
    }
    const double sx = xmax > xmin ? 65535.0 / (xmax - xmin) : 0.0, sy = ymax > ymin ? 65535.0 / (ymax - ymin) : 0.0;
    auto spread = [](uint32_t v) {
      v &= 0xffffu;
      v = (v | (v << 8)) & 0x00ff00ffu;
      v = (v | (v << 4)) & 0x0f0f0f0fu;
      v = (v | (v << 2)) & 0x33333333u;
      v = (v | (v << 1)) & 0x55555555u;
      return v;
    };
    // stable LSD radix sort of the codes, 11 bits per pass (three passes,
    // histograms of all three digits in one sweep), on packed (code, caller
    // index) keys, starting from the caller's order (so ties stay in caller
    // order)
    std::vector<uint64_t> key(np), key2(np);
    uint32_t hist[3][2049] = {{0}};
    for (int j = 0; j < np; ++j) {
      const uint32_t qx = (uint32_t)((X[3 * (size_t)j] - xmin) * sx), qy = (uint32_t)((X[3 * (size_t)j + 1] - ymin) * sy);
      const uint32_t code = spread(qx) | (spread(qy) << 1);
      key[j] = ((uint64_t)code << 32) | (uint32_t)j;
      ++hist[0][(code & 2047u) + 1];
      ++hist[1][((code >> 11) & 2047u) + 1];
      ++hist[2][(code >> 22) + 1];
    }
    for (int d = 0; d < 3; ++d) {
      uint32_t* c = hist[d];
      for (int b = 0; b < 2048; ++b) c[b + 1] += c[b];
      const int shift = 32 + 11 * d;
      for (int j = 0; j < np; ++j) {
        const uint64_t k = key[j];
        key2[c[(k >> shift) & 2047u]++] = k;
      }
      key.swap(key2);
    }
    for (int i = 0; i < np; ++i) {
      const int j = (int)(uint32_t)key[i];
      perm[i] = j;
      inv[j] = i;
    }
  }

  // point-major order: counting sort by internal point, then by camera within
  // a point.  The scatter writes one packed word per observation (camera in
  // the high half, observation index in the low half), so the per-point sort
  // by camera moves single words and, with ties in observation order, is the
  // stable sort by camera; the point of each entry follows from the counts.
  std::vector<int> cnt((size_t)np + 1, 0), pm(no), pcam(no), ppt(no);
  {
    std::vector<int> okey(no);  // internal point of each observation
    for (int i = 0; i < no; ++i) {
      const int j = inv[opt[i]];
      okey[i] = j;
      cnt[j + 1]++;
    }
    for (int j = 0; j < np; ++j) cnt[j + 1] += cnt[j];
    std::vector<int> pos(cnt.begin(), cnt.end() - 1);
    std::vector<uint64_t> ent(no);
    for (int i = 0; i < no; ++i) ent[pos[okey[i]]++] = ((uint64_t)(uint32_t)ocam[i] << 32) | (uint32_t)i;
    for (int j = 0; j < np; ++j) {
      const int s = cnt[j], e = cnt[j + 1];
      if (e - s > kMaxTrack) return set_err(ctx, BA_ERR_INVALID, "a point has more than 32 observations");
      for (int a = s + 1; a < e; ++a) {  // insertion sort of the point's words
        const uint64_t v = ent[a];
        int b = a - 1;
        while (b >= s && ent[b] > v) {
          ent[b + 1] = ent[b];
          --b;
        }
        ent[b + 1] = v;
      }
      for (int q = s; q < e; ++q) {
        pm[q] = (int)(uint32_t)ent[q];
        pcam[q] = (int)(ent[q] >> 32);
        ppt[q] = j;
      }
      for (int a = s + 1; a < e; ++a)
        if (pcam[a] == pcam[a - 1]) return set_err(ctx, BA_ERR_INVALID, "repeated (camera, point) observation");
    }
  }
  std::vector<int> pt_start(cnt);

  // tiles: runs of whole points with at most 32 observations
  std::vector<Tile> tiles;
  {
    int tb = 0, tn = 0;
    for (int j = 0; j < np; ++j) {
      const int L = pt_start[j + 1] - pt_start[j];
      if (L == 0) continue;
      if (tn + L > 32) {
        tiles.push_back(Tile{tb, tn});
        tn = 0;
      }
      if (tn == 0) tb = pt_start[j];
      tn += L;
    }
    if (tn > 0) tiles.push_back(Tile{tb, tn});
  }

  // chunks of consecutive tiles with at most chunk_obs() observations, and per
  // chunk the observation lists of its free cameras and the observation pairs
  // of its co-visible camera pairs (all in increasing point-major order)
  const bool mixed = ctx->mixed;
  const int ch_tiles = ctx->tune.chunk_tiles > 0 ? ctx->tune.chunk_tiles : chunk_tiles(mixed);
  std::vector<Chunk> chunks;
  for (size_t t = 0; t < tiles.size();) {
    Chunk ch{};
    ch.obs_begin = tiles[t].obs_begin;
    ch.tile_begin = (int)t;
    while (t < tiles.size() && ch.n_tiles < ch_tiles) {
      ch.n_obs += tiles[t].n_obs;
      ++t;
      ++ch.n_tiles;
    }
    ch.pt_begin = ppt[ch.obs_begin];  // observations are sorted by internal point
    ch.n_pts = ppt[ch.obs_begin + ch.n_obs - 1] - ch.pt_begin + 1;
    chunks.push_back(ch);
  }
  const int n_chunks = (int)chunks.size();
  // Per chunk, on its own: the jobs (its free cameras, then its co-visible
  // camera pairs, each by decreasing item count, ties by index / key), their
  // item lists (increasing point-major order), lanes and lane-to-job table.
  struct ChunkJobs {
    std::vector<int> cam;            // free camera of each image job
    std::vector<int> key;            // fa * nf + fb of each pair job
    std::vector<int> count;          // items of each job, image jobs first
    std::vector<unsigned short> cm;  // the image jobs' items, job after job
    std::vector<unsigned int> pe;    // the pair jobs' items, job after job
    std::vector<short> lane_begin, n_lanes;
    unsigned char lane_job[kChunkThreads];
  };
  struct Scratch {
    std::vector<int> cam_cnt, cam_off;  // by free camera
    std::vector<int> local_pair_of;     // fa * nf + fb -> local pair, -1 between chunks
    std::vector<int> pf;                // free camera of each observation of the chunk, or -1
    std::vector<int> lp_keys, lp_cnt, lp_off, order;
    std::vector<int> item_lp;           // local pair of each pair item, in point-major order (grown, not cleared)
    std::vector<unsigned int> item_val;
    std::vector<double> cost;
    std::vector<int> lanes;
    std::vector<int2> runs;
    std::vector<int> l_lo, l_hi, l_mid;
    explicit Scratch(int nf_) : cam_cnt(nf_, 0), cam_off(nf_), local_pair_of((size_t)nf_ * nf_, -1) {}
  };
  std::vector<ChunkJobs> cj(n_chunks);
  auto build_chunk = [&](int c, Scratch& S) {
    const Chunk& ch = chunks[c];
    ChunkJobs& J = cj[c];
    const int o0 = ch.obs_begin, o1 = ch.obs_begin + ch.n_obs;
    S.pf.resize(ch.n_obs);  // free camera of each of the chunk's observations, or -1
    int* const pf = S.pf.data();
    for (int p = o0; p < o1; ++p) pf[p - o0] = free_idx[pcam[p]];
    J.cam.reserve(nf);
    J.count.reserve(nf + 64);
    J.key.reserve(64);
    // image jobs: items counted, jobs ordered, then each item placed at its
    // job's next position (a stable counting sort: point-major order kept)
    for (int i = 0; i < ch.n_obs; ++i) {
      const int f = pf[i];
      if (f >= 0 && S.cam_cnt[f]++ == 0) J.cam.push_back(f);
    }
    std::sort(J.cam.begin(), J.cam.end(), [&](int x, int y) {
      return S.cam_cnt[x] != S.cam_cnt[y] ? S.cam_cnt[x] > S.cam_cnt[y] : x < y;
    });
    {
      int off = 0;
      for (int f : J.cam) {
        J.count.push_back(S.cam_cnt[f]);
        S.cam_off[f] = off;
        off += S.cam_cnt[f];
      }
      J.cm.resize(off);
      for (int i = 0; i < ch.n_obs; ++i)
        if (pf[i] >= 0) J.cm[S.cam_off[pf[i]]++] = (unsigned short)i;
      for (int f : J.cam) S.cam_cnt[f] = 0;
    }
    // pair jobs, the same way; pairs point by point (observations of a point
    // are sorted by camera), local pairs numbered by first appearance
    S.lp_keys.clear();
    S.lp_cnt.clear();
    size_t max_items = 0;  // k (k - 1) / 2 per point of k observations
    for (int j = ch.pt_begin; j < ch.pt_begin + ch.n_pts; ++j) {
      const size_t k = (size_t)(pt_start[j + 1] - pt_start[j]);
      max_items += k > 1 ? k * (k - 1) / 2 : 0;
    }
    if (S.item_lp.size() < max_items) {
      S.item_lp.resize(max_items);
      S.item_val.resize(max_items);
    }
    int* const item_lp = S.item_lp.data();
    unsigned int* const item_val = S.item_val.data();
    size_t n_items = 0;
    for (int j = ch.pt_begin; j < ch.pt_begin + ch.n_pts; ++j) {
      const int s0 = pt_start[j] - o0, e0 = pt_start[j + 1] - o0;
      for (int a = s0; a < e0; ++a) {
        const int fa = pf[a];
        if (fa < 0) continue;
        int* const row = S.local_pair_of.data() + (size_t)fa * nf;
        for (int b = a + 1; b < e0; ++b) {
          const int fb = pf[b];
          if (fb < 0) continue;
          int lp = row[fb];
          if (lp < 0) {
            lp = row[fb] = (int)S.lp_keys.size();
            S.lp_keys.push_back(fa * nf + fb);
            S.lp_cnt.push_back(0);
          }
          ++S.lp_cnt[lp];
          item_lp[n_items] = lp;
          item_val[n_items] = (unsigned)a | ((unsigned)b << 16);
          ++n_items;
        }
      }
    }
    const int n_lp_used = (int)S.lp_keys.size();
    S.order.resize(n_lp_used);
    for (int i = 0; i < n_lp_used; ++i) S.order[i] = i;
    std::sort(S.order.begin(), S.order.end(), [&](int x, int y) {
      if (S.lp_cnt[x] != S.lp_cnt[y]) return S.lp_cnt[x] > S.lp_cnt[y];
      return S.lp_keys[x] < S.lp_keys[y];
    });
    {
      S.lp_off.resize(n_lp_used);
      int off = 0;
      for (int li : S.order) {
        const int key = S.lp_keys[li];
        J.key.push_back(key);
        J.count.push_back(S.lp_cnt[li]);
        S.lp_off[li] = off;
        off += S.lp_cnt[li];
        S.local_pair_of[key] = -1;
      }
      J.pe.resize(off);
      for (size_t i = 0; i < n_items; ++i) J.pe[S.lp_off[item_lp[i]]++] = item_val[i];
    }
    // Lanes per job: every lane of every job gets about the same work, a
    // quantum Q of instructions (camera item ~165, pair item ~123), the
    // smallest Q whose lanes fit the CTA; the pair jobs start on a warp
    // boundary so that no warp runs both loop bodies.  A job has at least
    // one lane and at most one per item; chunks with more jobs than threads
    // run one lane per job (the kernel's fallback mode).
    const int n_lc = (int)J.cam.size(), n_lp = (int)J.key.size(), nj = n_lc + n_lp;
    J.lane_begin.assign(nj, 0);
    J.n_lanes.assign(nj, 1);
    std::memset(J.lane_job, 0, sizeof(J.lane_job));
    if (nj > 0 && nj <= kChunkThreads) {
      S.cost.resize(nj);
      for (int q = 0; q < nj; ++q) S.cost[q] = J.count[q] * (q < n_lc ? 165.0 : 123.0);
      S.lanes.resize(nj);
      auto alloc = [&](double Q, bool align) {
        int nc = 0, np_ = 0;
        for (int q = 0; q < nj; ++q) {
          const int cnt = J.count[q];
          int l = (int)std::ceil(S.cost[q] / Q);
          l = std::max(1, std::min(l, std::max(1, cnt)));
          S.lanes[q] = l;
          (q < n_lc ? nc : np_) += l;
        }
        return (align && n_lp > 0 ? (nc + 31) / 32 * 32 : nc) + np_;
      };
      // alloc(Q, align) <= kChunkThreads.  Jobs of one kind are sorted by
      // count, so equal jobs are runs that get equal lanes: one term per run,
      // stopping as soon as the partial count exceeds the CTA.
      S.runs.clear();  // (first job, jobs) of each run; the camera runs first
      int n_cam_runs = 0;
      for (int q = 0; q < nj; ++q) {
        if (q == 0 || q == n_lc || J.count[q] != J.count[q - 1]) {
          S.runs.push_back(make_int2(q, 0));
          if (q < n_lc) ++n_cam_runs;
        }
        ++S.runs.back().y;
      }
      // Lanes never grow with Q (a correctly rounded division is monotone):
      // a run's lanes at lo (or its cap, while lo = 0) and at hi bound them at
      // every Q between, and a run whose bounds agree needs no division.
      const int nr = (int)S.runs.size();
      S.l_lo.resize(nr);
      S.l_hi.resize(nr);
      S.l_mid.resize(nr);
      auto lanes_at = [&](int r, double Q) {
        const int q = S.runs[r].x;
        return std::max(1, std::min((int)std::ceil(S.cost[q] / Q), std::max(1, J.count[q])));
      };
      int evaluated = 0;  // runs whose l_mid the last fits() call set
      auto fits = [&](double Q, bool align) {
        int nc = 0, r = 0;
        for (; r < n_cam_runs; ++r) {
          const int l = S.l_lo[r] == S.l_hi[r] ? S.l_lo[r] : lanes_at(r, Q);
          S.l_mid[r] = l;
          nc += S.runs[r].y * l;
          if (nc > kChunkThreads) {
            evaluated = r + 1;
            return false;
          }
        }
        int tot = align && n_lp > 0 ? (nc + 31) / 32 * 32 : nc;
        for (; r < nr; ++r) {
          const int l = S.l_lo[r] == S.l_hi[r] ? S.l_lo[r] : lanes_at(r, Q);
          S.l_mid[r] = l;
          tot += S.runs[r].y * l;
          if (tot > kChunkThreads) {
            evaluated = r + 1;
            return false;
          }
        }
        evaluated = nr;
        return tot <= kChunkThreads;
      };
      // one lane each must fit (alloc at an unbounded quantum, in closed form)
      bool align = (n_lp > 0 ? (n_lc + 31) / 32 * 32 : n_lc) + n_lp <= kChunkThreads;
      double lo = 0.0, hi = 1.0;
      for (int q = 0; q < nj; ++q) hi = std::max(hi, S.cost[q]);
      for (int r = 0; r < nr; ++r) {
        S.l_lo[r] = std::max(1, J.count[S.runs[r].x]);
        S.l_hi[r] = lanes_at(r, hi);
      }
      for (int it = 0; it < 24; ++it) {  // smallest quantum that fits (to 2^-24 of the largest cost)
        const double mid = 0.5 * (lo + hi);
        if (mid > 0.0 && fits(mid, align)) {
          hi = mid;
          for (int r = 0; r < evaluated; ++r) S.l_hi[r] = S.l_mid[r];
        } else {
          lo = mid;
          if (mid > 0.0)
            for (int r = 0; r < evaluated; ++r) S.l_lo[r] = S.l_mid[r];
        }
      }
      alloc(hi, align);
      int lb = 0;
      for (int q = 0; q < nj; ++q) {
        if (align && q == n_lc && q > 0) lb = (lb + 31) / 32 * 32;
        J.lane_begin[q] = (short)lb;
        J.n_lanes[q] = (short)S.lanes[q];
        lb += S.lanes[q];
      }
      // lane t runs the last job whose lane run starts at or before t
      int q = 0;
      for (int t2 = 0; t2 < kChunkThreads; ++t2) {
        while (q + 1 < nj && J.lane_begin[q + 1] <= t2) ++q;
        J.lane_job[t2] = (unsigned char)q;
      }
    }
  };
  {
    // the chunks on a few threads when few creations share the host (the
    // result does not depend on the split); one thread otherwise
    const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
    const int busy = std::max(1, ctx->creating.load());
    const int n_thr = probe && probe->threads > 0 ? probe->threads
                                                  : (n_chunks >= 32 ? std::max(1, std::min(4, hw / busy)) : 1);
    std::atomic<int> next{0};
    auto worker = [&]() {
      Scratch S(nf);
      for (int c; (c = next.fetch_add(1)) < n_chunks;) build_chunk(c, S);
    };
    std::vector<std::thread> th;
    try {  // helpers beside the calling thread; if one cannot start, the others finish the chunks
      for (int i = 1; i < n_thr; ++i) th.emplace_back(worker);
    } catch (...) {
    }
    worker();
    for (auto& x : th) x.join();
  }
  // merge, in chunk order: partial-sum slots, item offsets, pair indices
  std::vector<Job> jobs;
  std::vector<unsigned short> cm_list;
  std::vector<unsigned char> lane_job((size_t)n_chunks * kChunkThreads);  // per chunk: the job of each lane
  std::vector<unsigned int> pent;
  std::vector<int> pair_of((size_t)nf * nf, -1);  // (fa, fb) -> pair index
  std::vector<int2> pair_key;
  std::vector<int2> cam_slot_ent, pair_slot_ent;  // (free camera or pair, slot), in chunk order
  int n_cslots = 0, n_pslots = 0;
  {
    size_t n_lc = 0, n_lp = 0, n_cm = 0, n_pe = 0;
    for (const ChunkJobs& J : cj) {
      n_lc += J.cam.size();
      n_lp += J.key.size();
      n_cm += J.cm.size();
      n_pe += J.pe.size();
    }
    jobs.reserve(n_lc + n_lp);
    cam_slot_ent.reserve(n_lc);
    pair_slot_ent.reserve(n_lp);
    cm_list.reserve(n_cm);
    pent.reserve(n_pe);
  }
  for (int c = 0; c < n_chunks; ++c) {
    Chunk& ch = chunks[c];
    const ChunkJobs& J = cj[c];
    ch.job_begin = (int)jobs.size();
    ch.n_lc = (int)J.cam.size();
    ch.n_lp = (int)J.key.size();
    int off = (int)cm_list.size();  // the chunk's item lists are its jobs' lists, job after job
    for (int q = 0; q < ch.n_lc; ++q) {
      Job jb{n_cslots++, off, J.count[q], J.lane_begin[q], J.n_lanes[q]};
      cam_slot_ent.push_back(make_int2(J.cam[q], jb.slot));
      off += J.count[q];
      jobs.push_back(jb);
    }
    cm_list.insert(cm_list.end(), J.cm.begin(), J.cm.end());
    off = (int)pent.size();
    for (int i = 0; i < ch.n_lp; ++i) {
      const int q = ch.n_lc + i, key = J.key[i];
      if (pair_of[key] < 0) {
        pair_of[key] = (int)pair_key.size();
        pair_key.push_back(make_int2(key / nf, key % nf));
      }
      Job jb{n_pslots++, off, J.count[q], J.lane_begin[q], J.n_lanes[q]};
      pair_slot_ent.push_back(make_int2(pair_of[key], jb.slot));
      off += J.count[q];
      jobs.push_back(jb);
    }
    pent.insert(pent.end(), J.pe.begin(), J.pe.end());
    std::memcpy(lane_job.data() + (size_t)c * kChunkThreads, J.lane_job, kChunkThreads);
  }
  // pairs in key order (the reduced system does not depend on this order, but a
  // fixed one keeps the tables reproducible)
  // slots grouped by camera / pair, each group in chunk order (stable counting sort)
  auto group = [](const std::vector<int2>& ent, int n_groups, std::vector<int>& begin, std::vector<int>& out) {
    begin.assign((size_t)n_groups + 1, 0);
    for (const int2& e : ent) ++begin[e.x + 1];
    for (int i = 0; i < n_groups; ++i) begin[i + 1] += begin[i];
    out.resize(ent.size());
    std::vector<int> pos(begin.begin(), begin.end() - 1);
    for (const int2& e : ent) out[pos[e.x]++] = e.y;
  };
  std::vector<int> cam_slot_begin, cam_slots;
  group(cam_slot_ent, nf, cam_slot_begin, cam_slots);
  const int n_pairs = (int)pair_key.size();
  std::vector<int> pair_slot_begin, pair_slots;
  group(pair_slot_ent, n_pairs, pair_slot_begin, pair_slots);

  // Elimination order of the reduced camera system: reverse Cuthill-McKee
  // (Cuthill & McKee 1969; George 1971) on the co-visibility graph of the
  // free images, which keeps the envelope of S, and with it the fill of its
  // Cholesky factor, narrow for images along strips.  The envelope of each
  // block row starts at its first co-visible block in that order.
  std::vector<int> fpos(nf), env_first(nf);
  {
    std::vector<std::vector<int>> adj(nf);
    for (const int2& k : pair_key) {
      adj[k.x].push_back(k.y);
      adj[k.y].push_back(k.x);
    }
    for (auto& v : adj) std::sort(v.begin(), v.end(), [&](int a, int b) {
      return adj[a].size() != adj[b].size() ? adj[a].size() < adj[b].size() : a < b;
    });
    std::vector<int> order;
    std::vector<char> seen(nf, 0);
    while ((int)order.size() < nf) {  // one BFS per connected component, from a least-connected image
      int start = -1;
      for (int f = 0; f < nf; ++f)
        if (!seen[f] && (start < 0 || adj[f].size() < adj[start].size())) start = f;
      seen[start] = 1;
      size_t head = order.size();
      order.push_back(start);
      while (head < order.size()) {
        const int u = order[head++];
        for (int v : adj[u])
          if (!seen[v]) {
            seen[v] = 1;
            order.push_back(v);
          }
      }
    }
    std::reverse(order.begin(), order.end());
    for (int p = 0; p < nf; ++p) fpos[order[p]] = p;
    for (int f = 0; f < nf; ++f) {
      int first = fpos[f];
      for (int g : adj[f]) first = std::min(first, fpos[g]);
      env_first[fpos[f]] = first;
    }
    // widen to a non-decreasing envelope (a superset: still no fill outside)
    for (int p = nf - 2; p >= 0; --p) env_first[p] = std::min(env_first[p], env_first[p + 1]);
  }
  // global-memory solver: per block column of kBigNB, the row blocks below it
  // whose first row reaches into it (contiguous, as the envelope is monotone)
  std::vector<int> big_below;
  const bool big = nf > kMaxFreeSmall;
  if (big) {
    const int n = 6 * nf, nblk = (n + kBigNB - 1) / kBigNB;
    big_below.assign(nblk, 0);
    for (int k = 0; k < nblk; ++k) {
      const int last_col = std::min(n, kBigNB * (k + 1)) - 1;
      int i = k + 1;
      while (i < nblk && 6 * env_first[(kBigNB * i) / 6] <= last_col) ++i;
      big_below[k] = i - (k + 1);
    }
  }

  if (probe) {  // ba_presort_host: the tables are checked instead of staged
    check_presort(PresortView{nc, np, no, nf, ch_tiles, chunk_obs(mixed), ocam.data(), opt.data(), free_idx, perm, inv,
                              pm, pt_start, pcam, ppt, tiles, chunks, jobs, cm_list, lane_job, pent, pair_key,
                              cam_slot_begin, cam_slots, pair_slot_begin, pair_slots, fpos, env_first},
                  probe->out);
    return BA_OK;
  }

  // arena layout: static (uploaded) part first
  const size_t rs = mixed ? sizeof(float) : sizeof(double);
  const int n = 6 * nf;
  Layout Lo;
  const size_t o_intr = Lo.add(sizeof(double) * nc * 7);
  const size_t o_R = Lo.add(sizeof(double) * 2 * nc * 9);
  const size_t o_T = Lo.add(sizeof(double) * 2 * nc * 3);
  const size_t o_X = Lo.add(sizeof(double) * 2 * (size_t)np * 3);
  const size_t o_Rp = Lo.add(sizeof(double) * nc * 9);
  const size_t o_Tp = Lo.add(sizeof(double) * nc * 3);
  const size_t o_Ri = Lo.add(sizeof(double) * nc * 9);
  const size_t o_Ti = Lo.add(sizeof(double) * nc * 3);
  const size_t o_Xi = Lo.add(sizeof(double) * (size_t)np * 3);
  const size_t o_perm = Lo.add(sizeof(int) * (size_t)np);
  const size_t o_free = Lo.add(sizeof(int) * nc);
  const size_t o_cof = Lo.add(sizeof(int) * nf);
  const size_t o_fpos = Lo.add(sizeof(int) * nf);
  const size_t o_cnobs = Lo.add(sizeof(int) * nc);
  const size_t o_envf = Lo.add(sizeof(int) * nf);
  const size_t o_tiles = Lo.add(sizeof(Tile) * tiles.size());
  const size_t o_ocam = Lo.add(sizeof(int) * (size_t)no);
  const size_t o_opt = Lo.add(sizeof(int) * (size_t)no);
  const size_t o_uv = Lo.add(sizeof(double) * 2 * (size_t)no);
  const size_t o_chi = Lo.add(mixed ? sizeof(float2) * (size_t)no : 0);
  const size_t o_clo = Lo.add(mixed ? sizeof(float2) * (size_t)no : 0);
  const size_t o_chunks = Lo.add(sizeof(Chunk) * chunks.size());
  const size_t o_jobs = Lo.add(sizeof(Job) * jobs.size());
  const size_t o_ljob = Lo.add(lane_job.size());
  const size_t o_cml = Lo.add(sizeof(unsigned short) * cm_list.size());
  const size_t o_pent = Lo.add(sizeof(unsigned int) * pent.size());
  const size_t o_csb = Lo.add(sizeof(int) * cam_slot_begin.size());
  const size_t o_cs = Lo.add(sizeof(int) * cam_slots.size());
  const size_t o_pkey = Lo.add(sizeof(int2) * pair_key.size());
  const size_t o_psb = Lo.add(sizeof(int) * pair_slot_begin.size());
  const size_t o_ps = Lo.add(sizeof(int) * pair_slots.size());
  const size_t o_lm = Lo.add(sizeof(LmState));
  const size_t o_bflag = Lo.add(big ? sizeof(int) : 0);  // zero from the staging
  const size_t o_camreal = Lo.add(mixed ? 0 : sizeof(double) * kCamReal * nc);
  const size_t o_camdf = Lo.add(mixed ? sizeof(float) * 2 * kCamDf * nc : 0);
  const size_t static_bytes = Lo.off;
  const size_t o_cpart = Lo.add(rs * kCamPart * (size_t)n_cslots);
  const size_t o_ppart = Lo.add(rs * kPairPart * (size_t)n_pslots);
  const size_t o_csum = Lo.add(sizeof(double) * kCamPart * (size_t)nf);
  const size_t o_psum = Lo.add(sizeof(double) * kPairPart * (size_t)n_pairs);
  const size_t o_S = Lo.add(sizeof(double) * (size_t)n * n);
  const size_t o_rhs = Lo.add(sizeof(double) * n);
  const size_t o_gc = Lo.add(sizeof(double) * n);
  const size_t o_Dc = Lo.add(sizeof(double) * n);
  const size_t o_dc = Lo.add(sizeof(double) * n);
  const size_t o_dc32 = Lo.add(sizeof(float) * n);
  const size_t o_tp = Lo.add(sizeof(double) * 2 * tiles.size());
  const size_t o_ptblk = Lo.add(rs * 16 * (size_t)np);
  const size_t o_trace = Lo.add(sizeof(StepRec) * kTraceCap);
  const size_t o_desc = Lo.add(sizeof(DevCluster));
  const size_t o_F = Lo.add(big ? sizeof(double) * (size_t)n * n : 0);
  const size_t o_bx = Lo.add(big ? sizeof(double) * 4 * (size_t)n : 0);
  const int dig_rows = big ? big_dig_rows(n) : 0;
  const size_t o_dig = Lo.add(big ? (size_t)kSlicesHost * dig_rows * 32 * sizeof(uint16_t) : 0);
  const size_t o_dexp = Lo.add(big ? sizeof(int) * (size_t)dig_rows : 0);
  const size_t o_linv = Lo.add(big ? sizeof(float) * 2 * kBigNB * kBigNB * (size_t)((n + kBigNB - 1) / kBigNB) : 0);
  const size_t total = Lo.off;

  // a pinned staging buffer of the context (every byte the kernels read is
  // written below; alignment padding may keep an earlier cluster's bytes):
  // the smallest free one that holds this cluster, else a new one.  Buffers
  // are only freed at shutdown: freeing pinned memory waits for the device,
  // which would stall a creation behind a batch that is being solved.
  std::pair<char*, size_t> stage{nullptr, 0};
  {
    std::lock_guard<std::mutex> g(ctx->stage_mu);
    int best = -1;
    for (int i = 0; i < (int)ctx->stage_free.size(); ++i)
      if (ctx->stage_free[i].second >= static_bytes &&
          (best < 0 || ctx->stage_free[i].second < ctx->stage_free[best].second))
        best = i;
    if (best >= 0) {
      stage = ctx->stage_free[best];
      ctx->stage_free.erase(ctx->stage_free.begin() + best);
    }
  }
  if (!stage.first) {
    const size_t want = (static_bytes + ((size_t)1 << 20) - 1) & ~(((size_t)1 << 20) - 1);
    if (cudaMallocHost((void**)&stage.first, want) != cudaSuccess)
      return set_err(ctx, BA_ERR_CUDA, "pinned staging buffer");
    stage.second = want;
  }
  struct StageBack {  // returns the buffer to the context once the upload is done (or abandoned)
    ba_ctx* ctx;
    std::pair<char*, size_t> s;
    ~StageBack() {
      std::lock_guard<std::mutex> g(ctx->stage_mu);
      ctx->stage_free.push_back(s);
    }
  } stage_back{ctx, stage};
  char* const stage_ptr = stage.first;
  auto put = [&](size_t off, const void* src, size_t bytes) {
    if (bytes) std::memcpy(stage_ptr + off, src, bytes);
  };
  put(o_intr, intr.data(), sizeof(double) * intr.size());
  put(o_R, R.data(), sizeof(double) * R.size());
  put(o_R + sizeof(double) * R.size(), R.data(), sizeof(double) * R.size());
  put(o_T, T.data(), sizeof(double) * T.size());
  put(o_T + sizeof(double) * T.size(), T.data(), sizeof(double) * T.size());
  // points in internal order: binary64, or double-float (hi, lo) pairs in the
  // mixed path; written once, then copied to the second state buffer and the
  // initial state
  const size_t xbytes = sizeof(double) * (size_t)np * 3;
  {
    double* xs = reinterpret_cast<double*>(stage_ptr + o_X);
    float* xf = reinterpret_cast<float*>(xs);
    par_for((size_t)np, [&](size_t b, size_t e) {
      for (size_t i = b; i < e; ++i)
        for (int a = 0; a < 3; ++a) {
          const double v = X[3 * (size_t)perm[i] + a];
          if (mixed) {
            const float hi = (float)v;
            xf[2 * (3 * i + a)] = hi;
            xf[2 * (3 * i + a) + 1] = (float)(v - (double)hi);
          } else {
            xs[3 * i + a] = v;
          }
        }
    });
  }
  put(o_X + xbytes, stage_ptr + o_X, xbytes);
  put(o_Rp, Rp.data(), sizeof(double) * Rp.size());
  put(o_Tp, Tp.data(), sizeof(double) * Tp.size());
  put(o_Ri, R.data(), sizeof(double) * R.size());
  put(o_Ti, T.data(), sizeof(double) * T.size());
  put(o_Xi, stage_ptr + o_X, xbytes);
  put(o_perm, perm.data(), sizeof(int) * perm.size());
  put(o_free, free_idx.data(), sizeof(int) * nc);
  put(o_cof, cam_of_free.data(), sizeof(int) * nf);
  put(o_fpos, fpos.data(), sizeof(int) * nf);
  {
    std::vector<int> cnobs(nc, 0);
    for (int i = 0; i < no; ++i) ++cnobs[ocam[i]];
    put(o_cnobs, cnobs.data(), sizeof(int) * nc);
  }
  put(o_envf, env_first.data(), sizeof(int) * nf);
  put(o_tiles, tiles.data(), sizeof(Tile) * tiles.size());
  put(o_ocam, pcam.data(), sizeof(int) * (size_t)no);
  put(o_opt, ppt.data(), sizeof(int) * (size_t)no);
  {
    double* su = (double*)(stage_ptr + o_uv);
    float2* chi = mixed ? (float2*)(stage_ptr + o_chi) : nullptr;
    float2* clo = mixed ? (float2*)(stage_ptr + o_clo) : nullptr;
    par_for((size_t)no, [&](size_t b, size_t e) {
      for (size_t p = b; p < e; ++p) {
        const size_t i = (size_t)pm[p];
        su[2 * p] = uv[2 * i];
        su[2 * p + 1] = uv[2 * i + 1];
        if (chi) {  // observation relative to the principal point, double-float
          const double cu = uv[2 * i] - intr[7 * (size_t)ocam[i] + 1];
          const double cv = uv[2 * i + 1] - intr[7 * (size_t)ocam[i] + 2];
          const float hu = (float)cu, hv = (float)cv;
          chi[p] = make_float2(hu, hv);
          clo[p] = make_float2((float)(cu - (double)hu), (float)(cv - (double)hv));
        }
      }
    });
  }
  put(o_chunks, chunks.data(), sizeof(Chunk) * chunks.size());
  put(o_jobs, jobs.data(), sizeof(Job) * jobs.size());
  put(o_ljob, lane_job.data(), lane_job.size());
  put(o_cml, cm_list.data(), sizeof(unsigned short) * cm_list.size());
  put(o_pent, pent.data(), sizeof(unsigned int) * pent.size());
  put(o_csb, cam_slot_begin.data(), sizeof(int) * cam_slot_begin.size());
  put(o_cs, cam_slots.data(), sizeof(int) * cam_slots.size());
  put(o_pkey, pair_key.data(), sizeof(int2) * pair_key.size());
  put(o_psb, pair_slot_begin.data(), sizeof(int) * pair_slot_begin.size());
  put(o_ps, pair_slots.data(), sizeof(int) * pair_slots.size());
  {
    LmState lm{};
    lm.mu0 = d->mu0 > 0.0 ? d->mu0 : 1e-4;
    lm.mu = lm.mu0;
    lm.mu_f = (float)lm.mu0;
    lm.nu = 2.0;
    lm.nu0 = 2.0;
    put(o_lm, &lm, sizeof(lm));
  }
  if (big) {
    const int zero = 0;
    put(o_bflag, &zero, sizeof(int));
  }
  // the camera records the kernels read, formed here rather than by a kernel
  // at creation (a kernel would wait for SMs behind any batch being solved):
  // the same values as write_camdf / k_camreal, both state buffers equal
  if (mixed) {
    float* o = reinterpret_cast<float*>(stage_ptr + o_camdf);
    for (int k = 0; k < nc; ++k) host_camdf(o + (size_t)k * kCamDf, &R[9 * (size_t)k], &T[3 * (size_t)k], &intr[7 * (size_t)k],
                                            free_idx[k] >= 0);
    std::memcpy(o + (size_t)nc * kCamDf, o, sizeof(float) * kCamDf * nc);
  } else {
    double* o = reinterpret_cast<double*>(stage_ptr + o_camreal);
    for (int k = 0; k < nc; ++k) {
      double* r = o + (size_t)kCamReal * k;
      for (int i = 0; i < 9; ++i) r[i] = R[9 * (size_t)k + i];
      for (int i = 0; i < 3; ++i) r[9 + i] = T[3 * (size_t)k + i];
      for (int i = 0; i < 7; ++i) r[12 + i] = intr[7 * (size_t)k + i];
      r[19] = free_idx[k] >= 0 ? 1.0 : 0.0;
    }
  }

  const auto t_staged = std::chrono::steady_clock::now();
  // Everything above is host work.  The budget is reserved under the API
  // lock; allocation, upload and the camera records run on a stream of this
  // call without the lock, so creation overlaps other calls and serving.
  {
    std::lock_guard<std::mutex> g(ctx->api_mu);
    if (ctx->budget && ctx->mem + total > ctx->budget)
      return set_err(ctx, BA_ERR_BUDGET, "cluster exceeds the device-memory budget");
    ctx->mem += total;
  }
  auto unreserve = [&]() {
    std::lock_guard<std::mutex> g(ctx->api_mu);
    ctx->mem -= total;
  };
  cudaStream_t up = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    unreserve();
    return set_err(ctx, BA_ERR_CUDA, std::string("upload stream: ") + cudaGetErrorString(e));
  }
  char* arena = nullptr;
  e = pool_alloc(ctx, (void**)&arena, total, up);
  if (e != cudaSuccess) {
    cudaStreamDestroy(up);
    unreserve();
    return set_err(ctx, BA_ERR_BUDGET, std::string("cluster allocation: ") + cudaGetErrorString(e));
  }
  auto fail = [&](const char* what, cudaError_t err) {
    cudaFreeAsync(arena, up);
    cudaStreamSynchronize(up);
    cudaStreamDestroy(up);
    unreserve();
    return set_err(ctx, BA_ERR_CUDA, std::string(what) + cudaGetErrorString(err));
  };
  e = cudaMemcpyAsync(arena, stage_ptr, static_bytes, cudaMemcpyHostToDevice, up);
  if (e != cudaSuccess) return fail("cluster upload: ", e);

  DevCluster& h = c->h;
  h = DevCluster{};
  h.n_cams = nc; h.n_pts = np; h.n_obs = no; h.n_free = nf;
  h.n_tiles = (int)tiles.size(); h.n_chunks = (int)chunks.size(); h.n_pairs = n_pairs;
  h.n_cslots = n_cslots; h.n_pslots = n_pslots;
  h.sigma_px = d->sigma_px; h.huber_delta = d->huber_delta_px; h.sigma_gnss = d->sigma_gnss_m;
  h.sigma_imu = d->sigma_imu_rad;
  h.inv_sigma_f = (float)(1.0 / d->sigma_px);
  h.delta_f = (float)d->huber_delta_px;
  h.half_inv_s2_f = (float)(0.5 / (d->sigma_px * d->sigma_px));
  h.intr = (const double*)(arena + o_intr);
  h.R = (double*)(arena + o_R);
  h.T = (double*)(arena + o_T);
  h.X = (double*)(arena + o_X);
  h.R_prior = (const double*)(arena + o_Rp);
  h.T_prior = (const double*)(arena + o_Tp);
  h.R_init = (const double*)(arena + o_Ri);
  h.T_init = (const double*)(arena + o_Ti);
  h.X_init = (const double*)(arena + o_Xi);
  h.pt_perm = (const int*)(arena + o_perm);
  h.free_idx = (const int*)(arena + o_free);
  h.cam_of_free = (const int*)(arena + o_cof);
  h.fpos = (const int*)(arena + o_fpos);
  h.cam_nobs = (const int*)(arena + o_cnobs);
  h.env_first = (const int*)(arena + o_envf);
  h.F = big ? (double*)(arena + o_F) : nullptr;
  h.bx = big ? (double*)(arena + o_bx) : nullptr;
  h.bflag = big ? (int*)(arena + o_bflag) : nullptr;
  h.dig = big ? (unsigned short*)(arena + o_dig) : nullptr;
  h.dexp = big ? (int*)(arena + o_dexp) : nullptr;
  h.linv = big ? (float*)(arena + o_linv) : nullptr;
  h.dig_groups = dig_rows / 8;
  h.camreal = mixed ? nullptr : arena + o_camreal;
  h.camdf = mixed ? (float*)(arena + o_camdf) : nullptr;
  h.tiles = (const Tile*)(arena + o_tiles);
  h.ptblk = arena + o_ptblk;
  h.obs_cam = (const int*)(arena + o_ocam);
  h.obs_pt = (const int*)(arena + o_opt);
  h.obs_uv = (const double*)(arena + o_uv);
  h.obs_chi = mixed ? (const float2*)(arena + o_chi) : nullptr;
  h.obs_clo = mixed ? (const float2*)(arena + o_clo) : nullptr;
  h.chunks = (const Chunk*)(arena + o_chunks);
  h.jobs = (const Job*)(arena + o_jobs);
  h.lane_job = (const unsigned char*)(arena + o_ljob);
  h.cm_list = (const unsigned short*)(arena + o_cml);
  h.pent = (const unsigned int*)(arena + o_pent);
  h.campart = arena + o_cpart;
  h.pairpart = arena + o_ppart;
  h.cam_slot_begin = (const int*)(arena + o_csb);
  h.cam_slots = (const int*)(arena + o_cs);
  h.pair_key = (const int2*)(arena + o_pkey);
  h.pair_slot_begin = (const int*)(arena + o_psb);
  h.pair_slots = (const int*)(arena + o_ps);
  h.camsum = (double*)(arena + o_csum);
  h.pairsum = (double*)(arena + o_psum);
  h.S = (double*)(arena + o_S);
  h.rhs = (double*)(arena + o_rhs);
  h.gc = (double*)(arena + o_gc);
  h.Dc = (double*)(arena + o_Dc);
  h.dc = (double*)(arena + o_dc);
  h.dc32 = (float*)(arena + o_dc32);
  h.tilepart = (double*)(arena + o_tp);
  h.lm = (LmState*)(arena + o_lm);
  h.trace = (StepRec*)(arena + o_trace);
  h.trace_cap = kTraceCap;
  c->d_desc = (DevCluster*)(arena + o_desc);
  e = cudaMemcpyAsync(c->d_desc, &h, sizeof(DevCluster), cudaMemcpyHostToDevice, up);
  if (e == cudaSuccess) e = cudaStreamSynchronize(up);
  if (e != cudaSuccess) return fail("cluster upload: ", e);
  cudaStreamDestroy(up);
  c->nc = nc; c->np = np; c->no = no; c->nf = nf;
  c->arena = arena;
  c->arena_bytes = total;
  c->info.n_cams = nc; c->info.n_free = nf; c->info.n_pts = np; c->info.n_obs = no;
  c->info.n_tiles = (int)tiles.size();
  c->info.n_chunks = (int)chunks.size();
  c->info.n_cam_slots = n_cslots;
  c->info.n_pair_slots = n_pslots;
  c->info.n_pairs = n_pairs;
  c->info.n_free_obs = (int64_t)cm_list.size();
  c->info.n_pair_entries = (int64_t)pent.size();
  c->info.arena_bytes = (int64_t)total;
  const auto t_end = std::chrono::steady_clock::now();
  c->info.presort_ms = std::chrono::duration<double, std::milli>(t_staged - t_start).count();
  c->info.upload_ms = std::chrono::duration<double, std::milli>(t_end - t_staged).count();
  c->pm_to_user = std::move(pm);
  c->pt_inv = std::move(inv);
  c->big_below = std::move(big_below);
  return BA_OK;
}

// single-cluster view for kernels that take a BatchView
ba_status single_view(ba_ctx* ctx, Cluster* c, Plan** p) { return get_plan(ctx, {c->id}, p); }

// Warm start: the current state of the cameras and points that c shares with
// src, copied on the device (caller indices -> internal indices), into both
// state buffers and the reset state of c.  Enqueued on the context's stream.
ba_status warm_copy(ba_ctx* ctx, Cluster* c, Cluster* src, const int32_t* cam_map, const int32_t* pt_map) {
  std::vector<int2> pairs;
  for (int k = 0; k < c->nc; ++k) {
    const int m = cam_map[k];
    if (m >= 0 && m < src->nc) pairs.push_back(make_int2(k, m));
  }
  const int n_cam_pairs = (int)pairs.size();
  for (int ju = 0; ju < c->np; ++ju) {
    const int mu_ = pt_map[ju];
    if (mu_ >= 0 && mu_ < src->np) pairs.push_back(make_int2(c->pt_inv[ju], src->pt_inv[mu_]));
  }
  // the kernel also carries the damping (mu, nu) over, so it runs even when
  // no camera or point is shared
  int2* dp = nullptr;
  if (!pairs.empty()) {
    CUDA_TRY(ctx, cudaMallocAsync((void**)&dp, sizeof(int2) * pairs.size(), ctx->stream));
    CUDA_TRY(ctx, cudaMemcpyAsync(dp, pairs.data(), sizeof(int2) * pairs.size(), cudaMemcpyHostToDevice, ctx->stream));
  }
  launch_warm_copy(c->d_desc, src->d_desc, dp, n_cam_pairs, dp ? dp + n_cam_pairs : nullptr,
                   (int)pairs.size() - n_cam_pairs, ctx->stream);
  note_direct(ctx);
  if (dp) CUDA_TRY(ctx, cudaFreeAsync(dp, ctx->stream));
  return BA_OK;
}

// ------------------------------------------------------------------ serving scheduler
//
// Continuous batching at LM-iteration granularity.  The running clusters sit
// in a fixed table of n_slots slots in device memory (descriptors, prefix
// sums, totals, factor order, arm counts); one CUDA graph, captured once,
// runs one LM iteration for every slot, reading the table as data.  Every
// round the scheduler (1) admits queued clusters into free slots and uploads
// the table if it changed, (2) launches the graph, (3) reads back the slots'
// LM states of the round before (rounds are pipelined one deep; see
// scheduler_loop) and retires the clusters that stopped on the device.
// Requests that arrive while others run join at the next round.  A cluster's
// iterations are exactly those of ba_run: every reduction is per cluster and
// fixed-order, so results do not depend on which clusters share a round.

ba_status slots_setup(ba_ctx* ctx) {
  SlotTable& T = ctx->slots;
  if (T.dbuf) return BA_OK;
  const int n = ctx->n_slots;
  ba_status st = ensure_attrs(ctx, 6 * kMaxFreeSmall);
  if (st != BA_OK) return st;
  Layout L;
  const size_t o_desc = L.add(sizeof(DevCluster) * n);
  const size_t o_pre = L.add(sizeof(int) * (3 * (size_t)(n + 1) + 3));
  const size_t o_ord = L.add(sizeof(int) * n);
  const size_t o_arm = L.add(sizeof(int) * n);
  const size_t o_ftol = L.add(sizeof(double) * n);
  const size_t o_lm = L.add(sizeof(LmState) * n);
  const size_t o_dummy = L.add(sizeof(LmState));
  T.bytes = L.off;
  T.o_lm = o_lm;
  CUDA_TRY(ctx, cudaMalloc((void**)&T.dbuf, T.bytes));
  CUDA_TRY(ctx, cudaMemset(T.dbuf, 0, T.bytes));
  CUDA_TRY(ctx, cudaMallocHost((void**)&T.hbuf, 2 * T.bytes));
  std::memset(T.hbuf, 0, 2 * T.bytes);
  for (auto& ev : T.done) CUDA_TRY(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  CUDA_TRY(ctx, cudaEventCreateWithFlags(&T.tail, cudaEventDisableTiming));
  ctx->mem += T.bytes;
  T.n = n;
  T.d_desc = (DevCluster*)(T.dbuf + o_desc);
  T.d_pre = (int*)(T.dbuf + o_pre);
  T.d_order = (int*)(T.dbuf + o_ord);
  T.d_arm = (int*)(T.dbuf + o_arm);
  T.d_ftol = (double*)(T.dbuf + o_ftol);
  T.d_lm = (LmState*)(T.dbuf + o_lm);
  T.empty = DevCluster{};
  T.empty.lm = (LmState*)(T.dbuf + o_dummy);  // zeroed: inactive, nothing to evaluate
  T.descs.assign(n, T.empty);
  T.arm.assign(n, 0);
  T.ftol.assign(n, 0.0);
  T.first_round.assign(n, -1);
  T.occ.assign(n, 0);
  T.occ_ticket.assign(n, 0);
  T.lm.assign(n, LmState{});
  BatchView& bv = T.bv;
  bv.cl = T.d_desc;
  bv.tile_pre = T.d_pre;
  bv.chunk_pre = T.d_pre + (n + 1);
  bv.item_pre = T.d_pre + 2 * (n + 1);
  bv.tot = T.d_pre + 3 * (n + 1);
  bv.factor_order = T.d_order;
  bv.n = n;
  bv.total_tiles = bv.total_chunks = bv.total_items = 1 << 30;  // the graph uses the largest grids
  bv.max_n = 6 * kMaxFreeSmall;
  bv.inject = ctx->inject;
  apply_tune(ctx, bv);
  T.dirty = true;
  return BA_OK;
}

ba_status slots_upload(ba_ctx* ctx, int parity) {
  SlotTable& T = ctx->slots;
  const int n = T.n;
  std::vector<int> pre(3 * (size_t)(n + 1) + 3, 0), order(n);
  for (int i = 0; i < n; ++i) {
    const DevCluster& h = T.descs[i];
    pre[i + 1] = pre[i] + h.n_tiles;
    pre[(n + 1) + i + 1] = pre[(n + 1) + i] + h.n_chunks;
    pre[2 * (n + 1) + i + 1] = pre[2 * (n + 1) + i] + h.n_free + h.n_pairs;
    order[i] = i;
  }
  pre[3 * (n + 1)] = pre[n];
  pre[3 * (n + 1) + 1] = pre[(n + 1) + n];
  pre[3 * (n + 1) + 2] = pre[2 * (n + 1) + n];
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return T.descs[a].n_free > T.descs[b].n_free; });
  // the whole table through this parity's pinned mirror in one copy (the
  // mirror's last copy, two rounds ago, has completed: that round has been
  // collected)
  char* const h = T.hbuf + parity * T.bytes;
  auto at = [&](const void* dev) { return h + ((const char*)dev - T.dbuf); };
  std::memcpy(at(T.d_desc), T.descs.data(), sizeof(DevCluster) * n);
  std::memcpy(at(T.d_pre), pre.data(), sizeof(int) * pre.size());
  std::memcpy(at(T.d_order), order.data(), sizeof(int) * n);
  std::memcpy(at(T.d_arm), T.arm.data(), sizeof(int) * n);
  std::memcpy(at(T.d_ftol), T.ftol.data(), sizeof(double) * n);
  CUDA_TRY(ctx, cudaMemcpyAsync(T.dbuf, h, T.o_lm, cudaMemcpyHostToDevice, ctx->sched_stream));
  T.dirty = false;
  return BA_OK;
}

// Launch one round on the scheduler's stream: arm -> F for newly armed slots
// -> one LM iteration -> gather; then the LM states go back to this parity's
// pinned mirror and the parity's event is recorded.  Nothing here waits for
// the device.
ba_status slots_launch(ba_ctx* ctx, int parity) {
  SlotTable& T = ctx->slots;
  const int gen = ctx->tune_gen.load();
  if (T.graph.exec && T.tune_gen != gen) {  // launch parameters changed since the capture
    cudaGraphExecDestroy(T.graph.exec);      // freed once a launch of it in flight completes
    T.graph.exec = nullptr;
    free_probe(T.graph.probe);
    T.graph.probe = nullptr;
  }
  if (!T.graph.exec) {
    apply_tune(ctx, T.bv);
    T.tune_gen = gen;
    cudaGraph_t graph = nullptr;
    note_direct(ctx);
    take_captured_launches();
    if (ctx->timing) {
      T.graph.probe = new Probe();
      set_probe(T.graph.probe);
    }
    CUDA_TRY(ctx, cudaStreamBeginCapture(ctx->sched_stream, cudaStreamCaptureModeThreadLocal));
    launch_arm_slots(T.bv, T.d_arm, T.d_ftol, ctx->sched_stream);
    launch_cost_init(T.bv, ctx->mixed, ctx->sched_stream);
    launch_iteration(T.bv, ctx->mixed, ctx->refine, ctx->sched_stream);
    launch_gather(T.bv, 0, T.d_lm, nullptr, ctx->sched_stream);
    cudaError_t e = cudaStreamEndCapture(ctx->sched_stream, &graph);
    set_probe(nullptr);
    T.graph.kernels = take_captured_launches();
    if (e != cudaSuccess) return set_err(ctx, BA_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&T.graph.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return set_err(ctx, BA_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  if (T.dirty) {
    ba_status st = slots_upload(ctx, parity);
    if (st != BA_OK) return st;
  }
  CUDA_TRY(ctx, cudaGraphLaunch(T.graph.exec, ctx->sched_stream));
  ctx->launches += T.graph.kernels;
  CUDA_TRY(ctx, cudaMemcpyAsync(T.hbuf + parity * T.bytes + T.o_lm, T.d_lm, sizeof(LmState) * T.n,
                                cudaMemcpyDeviceToHost, ctx->sched_stream));
  CUDA_TRY(ctx, cudaEventRecord(T.done[parity], ctx->sched_stream));
  CUDA_TRY(ctx, cudaEventRecord(T.tail, ctx->sched_stream));
  // the slots armed for this round are not armed again by the next one
  bool armed = false;
  for (int s = 0; s < T.n; ++s)
    if (T.arm[s]) {
      T.arm[s] = 0;
      armed = true;
    }
  if (armed) T.dirty = true;
  return BA_OK;
}

// Wait for the round of this parity and take its LM states.
ba_status slots_collect(ba_ctx* ctx, int parity) {
  SlotTable& T = ctx->slots;
  CUDA_TRY(ctx, cudaEventSynchronize(T.done[parity]));
  CUDA_TRY(ctx, cudaGetLastError());
  if (ctx->timing && T.graph.probe) fold_probe(ctx, T.graph.probe);
  std::memcpy(T.lm.data(), T.hbuf + parity * T.bytes + T.o_lm, sizeof(LmState) * T.n);
  return BA_OK;
}

// The scheduler thread.  Rounds are pipelined one deep: round r is launched
// before the results of round r - 1 are read, so the host's work between
// rounds (reading the states, retiring and admitting clusters, the table
// upload) overlaps the device's next round.  A cluster whose state shows it
// finished (its iteration count reached, converged on the device, or an
// error) leaves the table for the next launch and its ticket completes at
// once, although it may still sit, inert (inactive), in the round already in
// flight, which reads its LM state: ba_poll therefore orders the context's
// stream after the last round launched before it hands a result back, so
// that nothing the caller then queues on the cluster (freeing it, a reset, a
// warm start) overtakes that round.  With per-kernel timing the rounds run
// one at a time (a graph's event probes are read after each round).
void scheduler_loop(ba_ctx* ctx) {
  SlotTable& T = ctx->slots;
  cudaSetDevice(ctx->device);
  int occupied = 0;          // slots holding a cluster
  long long launched = 0;    // rounds launched
  long long collected = 0;   // rounds read
  std::vector<cudaEvent_t> admitted;
  auto finish_ticket = [&](int s, const std::chrono::steady_clock::time_point& now) {
    Ticket& tk = ctx->tickets[T.occ_ticket[s]];
    tk.done = 1;
    tk.res.latency_ms = std::chrono::duration<double, std::milli>(now - tk.t_submit).count();
    {
      std::lock_guard<std::mutex> g(ctx->api_mu);
      Cluster* c = find_cluster(ctx, T.occ[s]);
      if (c) c->in_service = 0;
    }
    T.occ[s] = 0;
    T.first_round[s] = -1;
    --occupied;
  };
  for (;;) {
    admitted.clear();
    {
      std::unique_lock<std::mutex> lk(ctx->sv_mu);
      ctx->sv_cv.wait(lk, [&] { return ctx->sched_stop || !ctx->queue.empty() || occupied > 0 || launched > collected; });
      if (ctx->sched_stop && occupied == 0 && launched == collected) return;
      for (int s = 0; s < T.n && !ctx->queue.empty(); ++s) {
        if (T.occ[s]) continue;
        const ba_ticket t = ctx->queue.front();
        ctx->queue.pop_front();
        Ticket& tk = ctx->tickets[t];
        Cluster* c = nullptr;
        {
          std::lock_guard<std::mutex> g(ctx->api_mu);
          c = find_cluster(ctx, tk.id);
        }
        if (!c) {  // destroyed while queued
          tk.done = 1;
          tk.res.status = BA_ERR_NOT_FOUND;
          continue;
        }
        T.occ[s] = tk.id;
        T.occ_ticket[s] = t;
        T.descs[s] = c->h;
        T.arm[s] = tk.iters;
        T.ftol[s] = tk.ftol;
        T.first_round[s] = launched;  // it runs from the next round on
        T.dirty = true;
        ++occupied;
        admitted.push_back(tk.ready);
        tk.ready = nullptr;
      }
    }
    // The rounds run without the API lock: the clusters in the slots are
    // marked in service, which every call that writes or frees a cluster
    // refuses.  Work the caller queued on the context's stream before
    // submitting (creation, warm start, reset) is ordered before the round.
    ba_status st = BA_OK;
    for (cudaEvent_t ev : admitted) {
      if (cudaStreamWaitEvent(ctx->sched_stream, ev, 0) != cudaSuccess) st = BA_ERR_CUDA;
      cudaEventDestroy(ev);
    }
    // launch the next round while one may still be in flight (the mirrors
    // of its parity are free: the round two back has been read)
    if (st == BA_OK && occupied > 0) {
      st = slots_launch(ctx, (int)(launched & 1));
      if (st == BA_OK) ++launched;
    }
    // read the older round in flight: always when two are, otherwise when no
    // further round follows it, or right away with per-kernel timing
    long long reading = -1;
    const long long pending = launched - collected;
    if (st == BA_OK && (pending >= 2 || (pending == 1 && (occupied == 0 || ctx->timing)))) {
      reading = collected;
      st = slots_collect(ctx, (int)(reading & 1));
      collected = reading + 1;
    }
    if (st != BA_OK) {  // let whatever was queued end before the clusters are handed back
      cudaStreamSynchronize(ctx->sched_stream);
      collected = launched;
    }
    {
      std::lock_guard<std::mutex> lk(ctx->sv_mu);
      const auto now = std::chrono::steady_clock::now();
      for (int s = 0; s < T.n; ++s) {
        if (!T.occ[s]) continue;
        if (st != BA_OK) {  // the round failed: every occupied slot ends with the error
          ctx->tickets[T.occ_ticket[s]].res.status = st;
          T.descs[s] = T.empty;
          T.dirty = true;
          finish_ticket(s, now);
          continue;
        }
        if (reading < 0 || T.first_round[s] > reading) continue;  // not in the round read
        const LmState& L = T.lm[s];
        if (L.active) continue;
        // finished in the round read: its result; out of the table from the
        // next launch on
        Ticket& tk = ctx->tickets[T.occ_ticket[s]];
        tk.res.status = L.status;
        tk.res.iters = L.iter - L.iter0;
        tk.res.final_cost = L.F;
        tk.res.accepted = L.n_accepted;
        T.descs[s] = T.empty;
        T.dirty = true;
        finish_ticket(s, now);
      }
      ctx->sv_cv.notify_all();
    }
  }
}

}  // namespace

// ====================================================================== C ABI

extern "C" {

BA_API const char* ba_status_string(ba_status s) {
  switch (s) {
    case BA_OK: return "ok";
    case BA_PENDING: return "pending";
    case BA_ERR_INVALID: return "invalid argument or problem data";
    case BA_ERR_BUDGET: return "device-memory budget or slots exhausted";
    case BA_ERR_NOT_PD: return "damped system not positive definite";
    case BA_ERR_TIMEOUT: return "bounded wait expired";
    case BA_ERR_CUDA: return "CUDA runtime error";
    case BA_ERR_NOT_FOUND: return "unknown cluster id or ticket";
    default: return "unknown status";
  }
}

BA_API const char* ba_last_error(ba_ctx* ctx) { return ctx ? t_last_error.c_str() : "null context"; }

BA_API ba_status ba_init(ba_ctx** out, const ba_config* cfg) {
  if (!out || !cfg) return BA_ERR_INVALID;
  if (cfg->precision != BA_FP64 && cfg->precision != BA_MIXED) return BA_ERR_INVALID;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) return BA_ERR_CUDA;
  if (cudaSetDevice(cfg->device) != cudaSuccess) return BA_ERR_CUDA;
  ba_ctx* ctx = new ba_ctx();
  ctx->device = cfg->device;
  ctx->budget = cfg->hbm_budget_bytes;
  ctx->mixed = cfg->precision == BA_MIXED;
  ctx->n_slots = cfg->n_slots > 0 ? cfg->n_slots : 64;
  // mixed: the double-float factor's rounding lies far below the binary32
  // rounding of the per-observation terms the system is built from, so a
  // binary64 refinement pass would not change the step beyond that
  ctx->refine = cfg->refine_steps >= 0 ? cfg->refine_steps : (ctx->mixed ? 0 : 1);
  ctx->timing = (cfg->flags & BA_FLAG_KERNEL_TIMING) != 0;
  ctx->inject = (cfg->flags & BA_FLAG_INJECT_COPY_TIMEOUT) ? kInjectCopyTimeout : 0;
  ctx->big_fp64 = (cfg->flags & BA_FLAG_BIG_FP64_FACTOR) != 0;
  ctx->small_df = (cfg->flags & BA_FLAG_SMALL_DF_FACTOR) != 0;
  if (cfg->tune_table) {  // this GPU's entry of the tuning table, if it has one
    cudaDeviceProp prop{};
    ba_tune t{};
    if (cudaGetDeviceProperties(&prop, cfg->device) == cudaSuccess &&
        ba_tune_table_lookup(cfg->tune_table, prop.name, prop.multiProcessorCount, cfg->precision, &t) == BA_OK)
      ctx->tune = tune_from_abi(t);
  }
  if (cfg->stream) {
    ctx->stream = (cudaStream_t)cfg->stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return BA_ERR_CUDA;
    }
    ctx->own_stream = true;
  }
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = cfg->device;
  const uint64_t keep = UINT64_MAX;
  if (cudaStreamCreateWithFlags(&ctx->sched_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->plan_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMemPoolCreate(&ctx->pool, &props) != cudaSuccess ||
      cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, (void*)&keep) != cudaSuccess) {
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    if (ctx->sched_stream) cudaStreamDestroy(ctx->sched_stream);
    if (ctx->plan_stream) cudaStreamDestroy(ctx->plan_stream);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return BA_ERR_CUDA;
  }
  *out = ctx;
  return BA_OK;
}

BA_API ba_status ba_create_cluster(ba_ctx* ctx, const ba_cluster_desc* d, ba_cluster_id* out) {
  if (!ctx || !d || !out) return BA_ERR_INVALID;
  cudaSetDevice(ctx->device);
  Cluster* c = new Cluster();
  ba_status st = build_cluster(ctx, d, c);  // presort, upload and camera records, without the API lock
  if (st != BA_OK) {
    delete c;
    return st;
  }
  std::lock_guard<std::mutex> g(ctx->api_mu);
  if (d->warm_from) {
    Cluster* src = find_cluster(ctx, d->warm_from);
    st = (src && d->warm_cam_map && d->warm_pt_map && !src->in_service)
             ? warm_copy(ctx, c, src, d->warm_cam_map, d->warm_pt_map)
             : set_err(ctx, BA_ERR_NOT_FOUND, "warm_from cluster not found, in service, or maps missing");
    if (st == BA_OK) {
      launch_camreal(one_view(c->d_desc, c->nf), ctx->mixed, ctx->stream);
      note_direct(ctx);
      if (cudaGetLastError() != cudaSuccess) st = set_err(ctx, BA_ERR_CUDA, "warm start launch failed");
    }
    if (st != BA_OK) {
      ctx->mem -= c->arena_bytes;
      cudaFreeAsync(c->arena, ctx->stream);
      delete c;
      return st;
    }
  }
  c->id = ctx->next_id++;
  ctx->clusters[c->id] = c;
  *out = c->id;
  return BA_OK;
}

BA_API ba_status ba_warm_start(ba_ctx* ctx, ba_cluster_id dst, ba_cluster_id src, const int32_t* cam_map,
                               const int32_t* pt_map) {
  if (!ctx || !cam_map || !pt_map) return BA_ERR_INVALID;
  std::lock_guard<std::mutex> g(ctx->api_mu);
  Cluster* c = find_cluster(ctx, dst);
  Cluster* s = find_cluster(ctx, src);
  if (!c || !s) return BA_ERR_NOT_FOUND;
  if (c->in_service || s->in_service) return set_err(ctx, BA_ERR_INVALID, "cluster is in service");
  ba_status st = warm_copy(ctx, c, s, cam_map, pt_map);
  if (st != BA_OK) return st;
  launch_camreal(one_view(c->d_desc, c->nf), ctx->mixed, ctx->stream);
  note_direct(ctx);
  CUDA_TRY(ctx, cudaGetLastError());
  return BA_OK;
}

BA_API ba_status ba_transition(ba_ctx* ctx, ba_cluster_id dst, ba_cluster_id src, const int32_t* cam_map) {
  if (!ctx || !cam_map) return BA_ERR_INVALID;
  std::lock_guard<std::mutex> g(ctx->api_mu);
  Cluster* c = find_cluster(ctx, dst);
  Cluster* s = find_cluster(ctx, src);
  if (!c || !s) return BA_ERR_NOT_FOUND;
  if (c->in_service || s->in_service) return set_err(ctx, BA_ERR_INVALID, "cluster is in service");
  std::vector<int2> pairs;
  for (int k = 0; k < c->nc; ++k) {
    const int m = cam_map[k];
    if (m < -1 || m >= s->nc) return set_err(ctx, BA_ERR_INVALID, "cam_map index out of range");
    if (m >= 0) pairs.push_back(make_int2(k, m));
  }
  if (pairs.empty()) return BA_OK;
  int2* dp = nullptr;
  CUDA_TRY(ctx, cudaMallocAsync((void**)&dp, sizeof(int2) * pairs.size(), ctx->stream));
  CUDA_TRY(ctx, cudaMemcpyAsync(dp, pairs.data(), sizeof(int2) * pairs.size(), cudaMemcpyHostToDevice, ctx->stream));
  launch_transition(c->d_desc, s->d_desc, dp, (int)pairs.size(), ctx->stream);
  launch_camreal(one_view(c->d_desc, c->nf), ctx->mixed, ctx->stream);  // camera records of the new poses
  note_direct(ctx);
  CUDA_TRY(ctx, cudaFreeAsync(dp, ctx->stream));
  CUDA_TRY(ctx, cudaGetLastError());
  return BA_OK;
}

BA_API ba_status ba_footprints(ba_ctx* ctx, int32_t n, const double* intr, double width, double height,
                               const double* R, const double* T, const ba_dsm* dsm, double* corners) {
  if (!ctx || n < 0 || !dsm || (n > 0 && (!intr || !R || !T || !corners))) return BA_ERR_INVALID;
  if (dsm->nx < 2 || dsm->ny < 2 || !dsm->h || !(dsm->dx > 0.0) || !(dsm->dy > 0.0) || !(width > 0.0) ||
      !(height > 0.0))
    return set_err(ctx, BA_ERR_INVALID, "ba_footprints: bad DSM or image size");
  if (n == 0) return BA_OK;
  std::lock_guard<std::mutex> g(ctx->api_mu);
  const size_t nh = (size_t)dsm->nx * dsm->ny;
  DsmView D{dsm->nx, dsm->ny, dsm->x0, dsm->y0, dsm->dx, dsm->dy, dsm->h[0], dsm->h[0], nullptr};
  for (size_t i = 0; i < nh; ++i) {
    if (!std::isfinite(dsm->h[i])) return set_err(ctx, BA_ERR_INVALID, "ba_footprints: non-finite DSM height");
    D.hmin = std::min(D.hmin, dsm->h[i]);
    D.hmax = std::max(D.hmax, dsm->h[i]);
  }
  const size_t b_in = sizeof(double) * (size_t)n * (7 + 9 + 3), b_h = sizeof(double) * nh,
               b_out = sizeof(double) * (size_t)n * 12;
  char* buf = nullptr;
  CUDA_TRY(ctx, cudaMallocAsync((void**)&buf, b_in + b_h + b_out, ctx->stream));
  double* d_intr = (double*)buf;
  double* d_R = d_intr + 7 * (size_t)n;
  double* d_T = d_R + 9 * (size_t)n;
  double* d_h = d_T + 3 * (size_t)n;
  double* d_out = d_h + nh;
  CUDA_TRY(ctx, cudaMemcpyAsync(d_intr, intr, sizeof(double) * 7 * n, cudaMemcpyHostToDevice, ctx->stream));
  CUDA_TRY(ctx, cudaMemcpyAsync(d_R, R, sizeof(double) * 9 * n, cudaMemcpyHostToDevice, ctx->stream));
  CUDA_TRY(ctx, cudaMemcpyAsync(d_T, T, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, ctx->stream));
  CUDA_TRY(ctx, cudaMemcpyAsync(d_h, dsm->h, b_h, cudaMemcpyHostToDevice, ctx->stream));
  D.h = d_h;
  launch_footprints(n, d_intr, width, height, d_R, d_T, D, d_out, ctx->stream);
  note_direct(ctx);
  CUDA_TRY(ctx, cudaMemcpyAsync(corners, d_out, b_out, cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaFreeAsync(buf, ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  CUDA_TRY(ctx, cudaGetLastError());
  return BA_OK;
}

BA_API ba_status ba_patch_transfer_poses(ba_ctx* ctx, int32_t n, const double* p0, const double* intr0,
                                         const double* R0, const double* T0, double lambda, int32_t m,
                                         const double* intr, const double* R, const double* T, double width,
                                         double height, double* p, uint8_t* inside) {
  if (!ctx || n < 0 || m < 0) return BA_ERR_INVALID;
  if (n == 0 || m == 0) return BA_OK;
  if (!p0 || !intr0 || !R0 || !T0 || !intr || !R || !T || !p || !std::isfinite(lambda) || !(width > 0.0) ||
      !(height > 0.0) || !(intr0[0] != 0.0))
    return set_err(ctx, BA_ERR_INVALID, "ba_patch_transfer_poses: null pointer, bad size or bad depth");
  if ((int64_t)n * m > (int64_t)1 << 30) return set_err(ctx, BA_ERR_INVALID, "ba_patch_transfer_poses: too many");
  std::lock_guard<std::mutex> g(ctx->api_mu);
  const size_t np0 = 2 * (size_t)n, ncam = 19, nk = 19 * (size_t)m, nout = 2 * (size_t)n * m;
  const size_t bytes = sizeof(double) * (np0 + ncam + nk + nout) + (inside ? (size_t)n * m : 0);
  char* buf = nullptr;
  CUDA_TRY(ctx, cudaMallocAsync((void**)&buf, bytes, ctx->stream));
  // the double2 arrays (centres in and out) first, at even offsets of the
  // allocation's 256-byte aligned start
  double* d_p0 = (double*)buf;
  double* d_out = d_p0 + np0;
  double* d_c0 = d_out + nout;  // intr0 7, R0 9, T0 3
  double* d_intr = d_c0 + ncam;
  double* d_R = d_intr + 7 * (size_t)m;
  double* d_T = d_R + 9 * (size_t)m;
  uint8_t* d_in = inside ? (uint8_t*)(d_T + 3 * (size_t)m) : nullptr;
  const cudaStream_t st = ctx->stream;
  CUDA_TRY(ctx, cudaMemcpyAsync(d_p0, p0, sizeof(double) * np0, cudaMemcpyHostToDevice, st));
  CUDA_TRY(ctx, cudaMemcpyAsync(d_c0, intr0, sizeof(double) * 7, cudaMemcpyHostToDevice, st));
  CUDA_TRY(ctx, cudaMemcpyAsync(d_c0 + 7, R0, sizeof(double) * 9, cudaMemcpyHostToDevice, st));
  CUDA_TRY(ctx, cudaMemcpyAsync(d_c0 + 16, T0, sizeof(double) * 3, cudaMemcpyHostToDevice, st));
  CUDA_TRY(ctx, cudaMemcpyAsync(d_intr, intr, sizeof(double) * 7 * m, cudaMemcpyHostToDevice, st));
  CUDA_TRY(ctx, cudaMemcpyAsync(d_R, R, sizeof(double) * 9 * m, cudaMemcpyHostToDevice, st));
  CUDA_TRY(ctx, cudaMemcpyAsync(d_T, T, sizeof(double) * 3 * m, cudaMemcpyHostToDevice, st));
  launch_patch_poses(n, d_p0, d_c0, d_c0 + 7, d_c0 + 16, lambda, m, d_intr, d_R, d_T, width, height, d_out, d_in, st);
  note_direct(ctx);
  CUDA_TRY(ctx, cudaMemcpyAsync(p, d_out, sizeof(double) * nout, cudaMemcpyDeviceToHost, st));
  if (inside) CUDA_TRY(ctx, cudaMemcpyAsync(inside, d_in, (size_t)n * m, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(ctx, cudaFreeAsync(buf, st));
  CUDA_TRY(ctx, cudaStreamSynchronize(st));
  CUDA_TRY(ctx, cudaGetLastError());
  return BA_OK;
}

BA_API ba_status ba_patch_transfer_planar(ba_ctx* ctx, int32_t n, const double* q0, const double* c,
                                          const double* g0, int32_t m, const double* theta, const double* g,
                                          double* q) {
  if (!ctx || n < 0 || m < 0) return BA_ERR_INVALID;
  if (n == 0 || m == 0) return BA_OK;
  if (!q0 || !c || !g0 || !theta || !g || !q)
    return set_err(ctx, BA_ERR_INVALID, "ba_patch_transfer_planar: null pointer");
  if ((int64_t)n * m > (int64_t)1 << 30) return set_err(ctx, BA_ERR_INVALID, "ba_patch_transfer_planar: too many");
  std::lock_guard<std::mutex> gl(ctx->api_mu);
  const size_t nq = 2 * (size_t)n, nout = 2 * (size_t)n * m;
  char* buf = nullptr;
  CUDA_TRY(ctx, cudaMallocAsync((void**)&buf, sizeof(double) * (nq + 3 * (size_t)m + nout), ctx->stream));
  // the double2 arrays (centres, displacements, output) first, at even offsets
  double* d_q0 = (double*)buf;
  double* d_g = d_q0 + nq;
  double* d_out = d_g + 2 * (size_t)m;
  double* d_th = d_out + nout;
  const cudaStream_t st = ctx->stream;
  CUDA_TRY(ctx, cudaMemcpyAsync(d_q0, q0, sizeof(double) * nq, cudaMemcpyHostToDevice, st));
  CUDA_TRY(ctx, cudaMemcpyAsync(d_th, theta, sizeof(double) * m, cudaMemcpyHostToDevice, st));
  CUDA_TRY(ctx, cudaMemcpyAsync(d_g, g, sizeof(double) * 2 * m, cudaMemcpyHostToDevice, st));
  launch_patch_planar(n, d_q0, c, g0, m, d_th, d_g, d_out, st);
  note_direct(ctx);
  CUDA_TRY(ctx, cudaMemcpyAsync(q, d_out, sizeof(double) * nout, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(ctx, cudaFreeAsync(buf, st));
  CUDA_TRY(ctx, cudaStreamSynchronize(st));
  CUDA_TRY(ctx, cudaGetLastError());
  return BA_OK;
}

BA_API ba_status ba_footprint_overlaps(ba_ctx* ctx, int32_t na, const double* qa, int32_t nb, const double* qb,
                                       double* area) {
  if (!ctx || na < 0 || nb < 0 || (na > 0 && nb > 0 && (!qa || !qb || !area))) return BA_ERR_INVALID;
  if ((int64_t)na * nb > (int64_t)1 << 30) return set_err(ctx, BA_ERR_INVALID, "ba_footprint_overlaps: too many pairs");
  if (na == 0 || nb == 0) return BA_OK;
  std::lock_guard<std::mutex> g(ctx->api_mu);
  const size_t ba_ = sizeof(double) * 12 * (size_t)na, bb = sizeof(double) * 12 * (size_t)nb,
               bo = sizeof(double) * (size_t)na * nb;
  char* buf = nullptr;
  CUDA_TRY(ctx, cudaMallocAsync((void**)&buf, ba_ + bb + bo, ctx->stream));
  double* d_a = (double*)buf;
  double* d_b = d_a + 12 * (size_t)na;
  double* d_o = d_b + 12 * (size_t)nb;
  CUDA_TRY(ctx, cudaMemcpyAsync(d_a, qa, ba_, cudaMemcpyHostToDevice, ctx->stream));
  CUDA_TRY(ctx, cudaMemcpyAsync(d_b, qb, bb, cudaMemcpyHostToDevice, ctx->stream));
  launch_overlaps(na, d_a, nb, d_b, d_o, ctx->stream);
  note_direct(ctx);
  CUDA_TRY(ctx, cudaMemcpyAsync(area, d_o, bo, cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaFreeAsync(buf, ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  CUDA_TRY(ctx, cudaGetLastError());
  return BA_OK;
}

BA_API ba_status ba_linearize(ba_ctx* ctx, ba_cluster_id id, ba_lin_info* out) {
  if (!ctx || !out) return BA_ERR_INVALID;
  std::lock_guard<std::mutex> g(ctx->api_mu);
  Cluster* c = find_cluster(ctx, id);
  if (!c) return BA_ERR_NOT_FOUND;
  if (c->in_service) return set_err(ctx, BA_ERR_INVALID, "cluster is in service");
  Plan* p = nullptr;
  ba_status st = single_view(ctx, c, &p);
  if (st != BA_OK) return st;
  launch_arm(p->bv, -1, ctx->stream);
  launch_cost_init(p->bv, ctx->mixed, ctx->stream);
  launch_grad_norm(p->bv, ctx->mixed, p->gnorm, ctx->stream, &p->big);
  launch_arm(p->bv, -2, ctx->stream);
  note_direct(ctx);
  LmState lm{};
  double gn = 0.0;
  CUDA_TRY(ctx, cudaMemcpyAsync(&lm, c->h.lm, sizeof(LmState), cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaMemcpyAsync(&gn, p->gnorm, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  CUDA_TRY(ctx, cudaGetLastError());
  out->cost = lm.F;
  out->grad_inf = gn;
  out->n_free = c->nf;
  return BA_OK;
}

BA_API ba_status ba_run(ba_ctx* ctx, ba_cluster_id id, int32_t iters, ba_step_info* trace) {
  if (!ctx || iters < 0) return BA_ERR_INVALID;
  std::lock_guard<std::mutex> g(ctx->api_mu);
  Cluster* c = find_cluster(ctx, id);
  if (!c) return BA_ERR_NOT_FOUND;
  if (c->in_service) return set_err(ctx, BA_ERR_INVALID, "cluster is in service");
  if (iters == 0) return BA_OK;
  std::vector<StepRec> tr;
  ba_status st = run_and_collect(ctx, {id}, iters, nullptr, trace ? &tr : nullptr);
  if (st != BA_OK) return st;
  if (trace) {
    const int tcap = std::min(iters, kTraceCap);
    for (int i = 0; i < iters; ++i) trace[i] = ba_step_info{};
    for (int i = 0; i < tcap; ++i) fill_step(tr[i], trace + (iters - tcap) + i);
  }
  return BA_OK;
}

BA_API ba_status ba_solve_step(ba_ctx* ctx, ba_cluster_id id, ba_step_info* out) {
  ba_step_info tmp;
  ba_status st = ba_run(ctx, id, 1, &tmp);
  if (st == BA_OK && out) *out = tmp;
  return st;
}

BA_API ba_status ba_solve_batch(ba_ctx* ctx, const ba_cluster_id* ids, int32_t n, int32_t iters, ba_result* results,
                         ba_step_info* trace) {
  if (!ctx || !ids || n <= 0 || iters < 0) return BA_ERR_INVALID;
  std::unique_lock<std::mutex> g(ctx->api_mu);
  std::vector<ba_cluster_id> v(ids, ids + n);
  for (auto id : v) {
    Cluster* c = find_cluster(ctx, id);
    if (!c) return BA_ERR_NOT_FOUND;
    if (c->in_service) return set_err(ctx, BA_ERR_INVALID, "cluster is in service");
  }
  {
    std::vector<ba_cluster_id> s(v);
    std::sort(s.begin(), s.end());
    if (std::adjacent_find(s.begin(), s.end()) != s.end()) return set_err(ctx, BA_ERR_INVALID, "repeated id in batch");
  }
  std::vector<LmState> lm;
  std::vector<StepRec> tr;
  const int tcap = std::min(iters, kTraceCap);
  // The device runs the batch without the lock (other threads may create,
  // read or solve other clusters meanwhile); the batch's own clusters are in
  // service until it returns.
  for (auto id : v) find_cluster(ctx, id)->in_service = 1;
  ba_status st = run_and_collect(ctx, v, iters, &lm, trace ? &tr : nullptr, &g);
  for (auto id : v) find_cluster(ctx, id)->in_service = 0;
  if (st != BA_OK) return st;
  for (int i = 0; i < n; ++i) {
    if (results) {
      ba_result& r = results[i];
      r = ba_result{};
      r.status = lm[i].status;
      r.iters = iters;
      r.accepted = lm[i].n_accepted;
      r.final_cost = lm[i].F;
      r.initial_cost = 0.0;
    }
    if (trace) {
      for (int t = 0; t < iters; ++t) trace[(size_t)i * iters + t] = ba_step_info{};
      for (int t = 0; t < tcap; ++t) fill_step(tr[(size_t)i * tcap + t], trace + (size_t)i * iters + (iters - tcap) + t);
      if (results && iters > 0 && tcap == iters) results[i].initial_cost = tr[(size_t)i * tcap].F_before;
    }
  }
  return BA_OK;
}

BA_API ba_status ba_reset(ba_ctx* ctx, ba_cluster_id id) {
  if (!ctx) return BA_ERR_INVALID;
  std::lock_guard<std::mutex> g(ctx->api_mu);
  Cluster* c = find_cluster(ctx, id);
  if (!c) return BA_ERR_NOT_FOUND;
  if (c->in_service) return set_err(ctx, BA_ERR_INVALID, "cluster is in service");
  Plan* p = nullptr;
  ba_status st = single_view(ctx, c, &p);
  if (st != BA_OK) return st;
  launch_reset(p->bv, ctx->mixed, ctx->stream);
  note_direct(ctx);
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  CUDA_TRY(ctx, cudaGetLastError());
  return BA_OK;
}

BA_API ba_status ba_reset_batch(ba_ctx* ctx, const ba_cluster_id* ids, int32_t n) {
  if (!ctx || !ids || n <= 0) return BA_ERR_INVALID;
  std::lock_guard<std::mutex> g(ctx->api_mu);
  std::vector<ba_cluster_id> v(ids, ids + n);
  for (auto id : v) {
    Cluster* c = find_cluster(ctx, id);
    if (!c) return BA_ERR_NOT_FOUND;
    if (c->in_service) return set_err(ctx, BA_ERR_INVALID, "cluster is in service");
  }
  Plan* p = nullptr;
  ba_status st = get_plan(ctx, v, &p);
  if (st != BA_OK) return st;
  launch_reset(p->bv, ctx->mixed, ctx->stream);
  note_direct(ctx);
  CUDA_TRY(ctx, cudaGetLastError());
  return BA_OK;
}

BA_API ba_status ba_launch_count(ba_ctx* ctx, uint64_t* out) {
  if (!ctx || !out) return BA_ERR_INVALID;
  std::lock_guard<std::mutex> g(ctx->api_mu);
  note_direct(ctx);
  *out = ctx->launches;
  return BA_OK;
}

BA_API ba_status ba_kernel_stats(ba_ctx* ctx, double* ms, uint64_t* launches, int32_t n, int32_t reset) {
  if (!ctx || n < 0 || n > KK_COUNT) return BA_ERR_INVALID;
  std::lock_guard<std::mutex> g(ctx->stats_mu);
  for (int i = 0; i < n; ++i) {
    if (ms) ms[i] = ctx->kms[i];
    if (launches) launches[i] = ctx->klaunch[i];
  }
  if (reset)
    for (int i = 0; i < KK_COUNT; ++i) {
      ctx->kms[i] = 0.0;
      ctx->klaunch[i] = 0;
    }
  return BA_OK;
}

BA_API ba_status ba_presort_host(const ba_cluster_desc* d, int32_t precision, int32_t threads, ba_presort_info* out) {
  if (!out) return BA_ERR_INVALID;
  std::memset(out, 0, sizeof(*out));
  auto reject = [&](const char* why) {
    std::snprintf(out->message, sizeof(out->message), "%s", why);
    return BA_ERR_INVALID;
  };
  if (!d) return reject("null cluster description");
  if (precision != BA_FP64 && precision != BA_MIXED) return reject("precision must be BA_FP64 or BA_MIXED");
  if (d->ptr_kind != BA_PTR_HOST) return reject("ba_presort_host reads host arrays only");
  if (threads < 0 || threads > 64) return reject("threads must be 0 (the library's choice) to 64");
  ba_ctx ctx;  // host bookkeeping only: no device, stream or pool is touched
  ctx.mixed = precision == BA_MIXED;
  Cluster c;
  PresortProbe probe;
  probe.threads = threads;
  probe.out = out;
  const ba_status st = build_cluster(&ctx, d, &c, &probe);
  if (st != BA_OK) std::snprintf(out->message, sizeof(out->message), "%s", t_last_error.c_str());
  return st;
}

BA_API ba_status ba_submit(ba_ctx* ctx, ba_cluster_id id, const ba_solve_opts* opts, ba_ticket* out) {
  if (!ctx || !opts || !out || opts->max_iters <= 0) return BA_ERR_INVALID;
  if (!(opts->ftol >= 0.0) || !std::isfinite(opts->ftol)) return set_err(ctx, BA_ERR_INVALID, "ftol must be finite and >= 0");
  cudaEvent_t ready = nullptr;
  {
    std::lock_guard<std::mutex> g(ctx->api_mu);
    Cluster* c = find_cluster(ctx, id);
    if (!c) return BA_ERR_NOT_FOUND;
    if (6 * c->nf > 6 * kMaxFreeSmall) return set_err(ctx, BA_ERR_INVALID, "cluster too large for a serving slot");
    ba_status st = slots_setup(ctx);
    if (st != BA_OK) return st;
    CUDA_TRY(ctx, cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    if (cudaEventRecord(ready, ctx->stream) != cudaSuccess) {
      cudaEventDestroy(ready);
      return set_err(ctx, BA_ERR_CUDA, "ba_submit: event record failed");
    }
    int expect = 0;
    if (!c->in_service.compare_exchange_strong(expect, 1)) {
      cudaEventDestroy(ready);
      return set_err(ctx, BA_ERR_INVALID, "cluster already submitted");
    }
  }
  std::lock_guard<std::mutex> lk(ctx->sv_mu);
  if (!ctx->sched_started) {
    ctx->sched_started = true;
    ctx->sched = std::thread(scheduler_loop, ctx);
  }
  const ba_ticket t = ctx->next_ticket++;
  Ticket tk;
  tk.id = id;
  tk.iters = opts->max_iters;
  tk.ftol = opts->ftol;
  tk.t_submit = std::chrono::steady_clock::now();
  tk.ready = ready;
  ctx->tickets[t] = tk;
  ctx->queue.push_back(t);
  ctx->sv_cv.notify_all();
  *out = t;
  return BA_OK;
}

BA_API ba_status ba_poll(ba_ctx* ctx, ba_ticket t, ba_result* out) {
  if (!ctx) return BA_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(ctx->sv_mu);
    auto it = ctx->tickets.find(t);
    if (it == ctx->tickets.end()) return BA_ERR_NOT_FOUND;
    if (!it->second.done) return BA_PENDING;
  }
  // The cluster may still be read (inert) by the serving round in flight:
  // whatever the caller queues on it from now on waits for that round (under
  // the API lock, so that the wait cannot land in another thread's capture of
  // the context's stream).
  cudaError_t e = cudaSuccess;
  {
    std::lock_guard<std::mutex> g(ctx->api_mu);
    if (ctx->slots.tail) e = cudaStreamWaitEvent(ctx->stream, ctx->slots.tail, 0);
  }
  std::lock_guard<std::mutex> lk(ctx->sv_mu);
  auto it = ctx->tickets.find(t);
  if (it == ctx->tickets.end()) return BA_ERR_NOT_FOUND;
  if (e != cudaSuccess) {
    ctx->tickets.erase(it);
    return set_err(ctx, BA_ERR_CUDA, std::string("ordering after the serving round: ") + cudaGetErrorString(e));
  }
  if (out) *out = it->second.res;
  ctx->tickets.erase(it);
  return BA_OK;
}

BA_API ba_status ba_get_state(ba_ctx* ctx, ba_cluster_id id, double* R, double* T, double* X, int32_t ptr_kind) {
  if (!ctx) return BA_ERR_INVALID;
  std::lock_guard<std::mutex> hs(ctx->hstage_mu);
  std::lock_guard<std::mutex> g(ctx->api_mu);
  Cluster* c = find_cluster(ctx, id);
  if (!c) return BA_ERR_NOT_FOUND;
  // one kernel writes the requested parts of the current state into one
  // device block (it reads the current buffer's index itself); host
  // destinations get it through one copy into pinned staging
  const size_t nr = (size_t)c->nc * 9, nt = (size_t)c->nc * 3, nx = (size_t)c->np * 3;
  const size_t total = nr + nt + nx;
  double* tmp = nullptr;
  CUDA_TRY(ctx, cudaMallocAsync((void**)&tmp, sizeof(double) * total, ctx->stream));
  launch_export_state(c->d_desc, c->h, ctx->mixed, R ? tmp : nullptr, T ? tmp + nr : nullptr,
                      X && nx ? tmp + nr + nt : nullptr, ctx->stream);
  note_direct(ctx);
  if (ptr_kind == BA_PTR_DEVICE) {
    if (R) CUDA_TRY(ctx, cudaMemcpyAsync(R, tmp, sizeof(double) * nr, cudaMemcpyDeviceToDevice, ctx->stream));
    if (T) CUDA_TRY(ctx, cudaMemcpyAsync(T, tmp + nr, sizeof(double) * nt, cudaMemcpyDeviceToDevice, ctx->stream));
    if (X && nx)
      CUDA_TRY(ctx, cudaMemcpyAsync(X, tmp + nr + nt, sizeof(double) * nx, cudaMemcpyDeviceToDevice, ctx->stream));
    CUDA_TRY(ctx, cudaFreeAsync(tmp, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return BA_OK;
  }
  if (ctx->hstage_bytes < sizeof(double) * total) {
    if (ctx->hstage) cudaFreeHost(ctx->hstage);
    ctx->hstage = nullptr;
    ctx->hstage_bytes = 0;
    const size_t want = std::max(sizeof(double) * total, (size_t)1 << 20);
    CUDA_TRY(ctx, cudaMallocHost((void**)&ctx->hstage, want));
    ctx->hstage_bytes = want;
  }
  CUDA_TRY(ctx, cudaMemcpyAsync(ctx->hstage, tmp, sizeof(double) * total, cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaFreeAsync(tmp, ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  if (R) std::memcpy(R, ctx->hstage, sizeof(double) * nr);
  if (T) std::memcpy(T, ctx->hstage + nr, sizeof(double) * nt);
  if (X && nx) std::memcpy(X, ctx->hstage + nr + nt, sizeof(double) * nx);
  return BA_OK;
}

BA_API ba_status ba_get_state_batch(ba_ctx* ctx, const ba_cluster_id* ids, int32_t n, double* const* R,
                                    double* const* T, double* const* X) {
  if (!ctx || (n > 0 && !ids) || n < 0) return BA_ERR_INVALID;
  std::lock_guard<std::mutex> hs(ctx->hstage_mu);  // (taken before the API lock, as in ba_get_state)
  std::unique_lock<std::mutex> g(ctx->api_mu);
  std::vector<Cluster*> cs(n);
  for (int i = 0; i < n; ++i) {
    cs[i] = find_cluster(ctx, ids[i]);
    if (!cs[i]) return BA_ERR_NOT_FOUND;
    if (cs[i]->in_service) return set_err(ctx, BA_ERR_INVALID, "cluster is in service");
  }
  // The batch's clusters are in service for the call.  Each group's work is
  // queued on the context's stream under the lock; the wait for it and the
  // host copies run without the lock (other threads may create or solve
  // other clusters meanwhile).
  for (Cluster* c : cs) c->in_service = 1;
  struct Release {
    ba_ctx* ctx;
    std::vector<Cluster*>& cs;
    std::unique_lock<std::mutex>& g;
    ~Release() {
      if (!g.owns_lock()) g.lock();
      for (Cluster* c : cs) c->in_service = 0;
    }
  } release{ctx, cs, g};
  if (!ctx->state_done) CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->state_done, cudaEventDisableTiming | cudaEventBlockingSync));
  // groups of clusters whose states fit the pinned staging (at most
  // kStateStageBytes, or one cluster's state if that is larger): per group,
  // one device export per cluster into one block, one copy, one wait
  constexpr size_t kStateStageBytes = (size_t)32 << 20;
  auto doubles_of = [&](int i) { return (size_t)cs[i]->nc * 12 + (size_t)cs[i]->np * 3; };
  for (int i0 = 0; i0 < n;) {
    size_t total = doubles_of(i0);
    int i1 = i0 + 1;
    while (i1 < n && sizeof(double) * (total + doubles_of(i1)) <= kStateStageBytes) total += doubles_of(i1++);
    if (!g.owns_lock()) g.lock();
    if (ctx->hstage_bytes < sizeof(double) * total) {
      if (ctx->hstage) cudaFreeHost(ctx->hstage);
      ctx->hstage = nullptr;
      ctx->hstage_bytes = 0;
      const size_t want = std::max(sizeof(double) * total, std::min(kStateStageBytes, (size_t)1 << 20));
      CUDA_TRY(ctx, cudaMallocHost((void**)&ctx->hstage, want));
      ctx->hstage_bytes = want;
    }
    double* tmp = nullptr;
    CUDA_TRY(ctx, cudaMallocAsync((void**)&tmp, sizeof(double) * total, ctx->stream));
    size_t off = 0;
    for (int i = i0; i < i1; ++i) {
      const Cluster* c = cs[i];
      double* b = tmp + off;
      launch_export_state(c->d_desc, c->h, ctx->mixed, b, b + (size_t)c->nc * 9,
                          c->np ? b + (size_t)c->nc * 12 : nullptr, ctx->stream);
      off += doubles_of(i);
    }
    note_direct(ctx);
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->hstage, tmp, sizeof(double) * total, cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(ctx, cudaFreeAsync(tmp, ctx->stream));
    CUDA_TRY(ctx, cudaEventRecord(ctx->state_done, ctx->stream));
    g.unlock();
    CUDA_TRY(ctx, cudaEventSynchronize(ctx->state_done));
    off = 0;
    std::vector<HostCopy> out;
    for (int i = i0; i < i1; ++i) {
      const Cluster* c = cs[i];
      const double* b = ctx->hstage + off;
      const size_t nr = (size_t)c->nc * 9, nt = (size_t)c->nc * 3, nx = (size_t)c->np * 3;
      if (R && R[i]) out.push_back(HostCopy{R[i], b, sizeof(double) * nr});
      if (T && T[i]) out.push_back(HostCopy{T[i], b + nr, sizeof(double) * nt});
      if (X && X[i] && nx) out.push_back(HostCopy{X[i], b + nr + nt, sizeof(double) * nx});
      off += doubles_of(i);
    }
    copy_out(out, 8);
    i0 = i1;
  }
  return BA_OK;
}

BA_API ba_status ba_reprojection_errors(ba_ctx* ctx, ba_cluster_id id, double* err) {
  if (!ctx || !err) return BA_ERR_INVALID;
  std::lock_guard<std::mutex> g(ctx->api_mu);
  Cluster* c = find_cluster(ctx, id);
  if (!c) return BA_ERR_NOT_FOUND;
  if (c->no == 0) return BA_OK;
  double* d = nullptr;
  CUDA_TRY(ctx, cudaMallocAsync((void**)&d, sizeof(double) * c->no, ctx->stream));
  launch_reproj(c->d_desc, c->h, ctx->mixed, d, ctx->stream);
  note_direct(ctx);
  std::vector<double> pmv(c->no);
  CUDA_TRY(ctx, cudaMemcpyAsync(pmv.data(), d, sizeof(double) * c->no, cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaFreeAsync(d, ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  CUDA_TRY(ctx, cudaGetLastError());
  for (int p = 0; p < c->no; ++p) err[c->pm_to_user[p]] = pmv[p];
  return BA_OK;
}

BA_API ba_status ba_memory_in_use(ba_ctx* ctx, uint64_t* bytes) {
  if (!ctx || !bytes) return BA_ERR_INVALID;
  std::lock_guard<std::mutex> g(ctx->api_mu);
  *bytes = ctx->mem;
  return BA_OK;
}

BA_API ba_status ba_get_cluster_info(ba_ctx* ctx, ba_cluster_id id, ba_cluster_info* out) {
  if (!ctx || !out) return BA_ERR_INVALID;
  std::lock_guard<std::mutex> g(ctx->api_mu);
  Cluster* c = find_cluster(ctx, id);
  if (!c) return BA_ERR_NOT_FOUND;
  *out = c->info;
  return BA_OK;
}

BA_API ba_status ba_get_tune(ba_ctx* ctx, ba_tune* out) {
  if (!ctx || !out) return BA_ERR_INVALID;
  std::lock_guard<std::mutex> g(ctx->api_mu);
  *out = tune_to_abi(ctx->tune);
  return BA_OK;
}

BA_API ba_status ba_set_tune(ba_ctx* ctx, const ba_tune* t) {
  if (!ctx || !t) return BA_ERR_INVALID;
  std::string why;
  if (!tune_in_range(*t, ctx->mixed, &why)) return set_err(ctx, BA_ERR_INVALID, why);
  std::lock_guard<std::mutex> g(ctx->api_mu);
  for (auto& kv : ctx->clusters)
    if (kv.second->in_service) return set_err(ctx, BA_ERR_INVALID, "a cluster is in service");
  ctx->tune = tune_from_abi(*t);
  // plans hold graphs captured with the old launch shapes: rebuilt on demand
  for (auto& kv : ctx->plans) {
    ctx->mem -= kv.second->dbuf_bytes;
    free_plan(ctx, kv.second);
  }
  ctx->plans.clear();
  ctx->tune_gen.fetch_add(1);  // and the serving graph is captured again before its next round
  return BA_OK;
}

BA_API ba_status ba_autotune(ba_ctx* ctx, const ba_cluster_desc* descs, int32_t n, int32_t iters, ba_tune* out) {
  if (!ctx || !descs || n <= 0 || iters <= 0 || !out) return BA_ERR_INVALID;
  std::vector<ba_cluster_id> ids;
  int created = -1;  // chunk_tiles the current tuning clusters were created with
  bool has_big = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto destroy_all = [&]() {
    for (ba_cluster_id id : ids) ba_destroy_cluster(ctx, id);
    ids.clear();
  };
  auto finish = [&](ba_status st) {
    destroy_all();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return st;
  };
  CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return finish(set_err(ctx, BA_ERR_CUDA, "ba_autotune: event creation failed"));
  // device time of one batch solve with t: the fastest of three after a warm-up
  auto measure = [&](const TuneParams& t, double* ms) -> ba_status {
    ba_tune bt = tune_to_abi(t);
    ba_status st = ba_set_tune(ctx, &bt);
    if (st != BA_OK) return st;
    const int ct = t.chunk_tiles > 0 ? t.chunk_tiles : chunk_tiles(ctx->mixed);
    if (ct != created) {
      destroy_all();
      for (int i = 0; i < n; ++i) {
        ba_cluster_id id = 0;
        st = ba_create_cluster(ctx, &descs[i], &id);
        if (st != BA_OK) return st;
        ids.push_back(id);
        ba_cluster_info info{};
        if (ba_get_cluster_info(ctx, id, &info) == BA_OK && info.n_free > kMaxFreeSmall) has_big = true;
      }
      created = ct;
    }
    double best = 1e300;
    for (int rep = 0; rep < 4; ++rep) {
      st = ba_reset_batch(ctx, ids.data(), n);
      if (st != BA_OK) return st;
      CUDA_TRY(ctx, cudaEventRecord(e0, ctx->stream));
      st = ba_solve_batch(ctx, ids.data(), n, iters, nullptr, nullptr);
      if (st != BA_OK) return st;
      CUDA_TRY(ctx, cudaEventRecord(e1, ctx->stream));
      CUDA_TRY(ctx, cudaEventSynchronize(e1));
      float el = 0.f;
      CUDA_TRY(ctx, cudaEventElapsedTime(&el, e0, e1));
      if (rep > 0) best = std::min(best, (double)el);  // rep 0 captures the graphs
    }
    *ms = best;
    return BA_OK;
  };
  TuneParams cur;  // the defaults
  cur.chunk_tiles = chunk_tiles(ctx->mixed);
  double cur_ms = 0.0;
  ba_status st = measure(cur, &cur_ms);
  if (st != BA_OK) return finish(st);
  const double ms_default = cur_ms;
  // one parameter at a time; a candidate replaces the current value only
  // when it is faster by more than 1 % (timing noise keeps the default)
  struct Knob {
    int TuneParams::*field;
    std::vector<int> cands;
    bool big_only;
  };
  const bool mixed = ctx->mixed;
  const std::vector<Knob> knobs = {
      {&TuneParams::chunk_tiles, mixed ? std::vector<int>{12, 8} : std::vector<int>{6, 4}, false},
      {&TuneParams::lin_ctas_per_sm, {4, 2}, false},
      {&TuneParams::back_ctas_per_sm, {8, 4}, false},
      {&TuneParams::factor_nb, {4, 16}, false},
      {&TuneParams::factor_threads, {384, 256}, false},
      {&TuneParams::big_panel_w, {2, 8}, true},
      {&TuneParams::batch_chains, {2, 8}, false},
  };
  for (const Knob& k : knobs) {
    if (k.big_only && !has_big) continue;
    TuneParams best = cur;
    double best_ms = cur_ms;
    for (int v : k.cands) {
      TuneParams t = cur;
      t.*(k.field) = v;
      double ms = 0.0;
      st = measure(t, &ms);
      if (st != BA_OK) return finish(st);
      if (ms < best_ms * 0.99) {
        best = t;
        best_ms = ms;
      }
    }
    cur = best;
    cur_ms = best_ms;
  }
  ba_tune bt = tune_to_abi(cur);
  st = ba_set_tune(ctx, &bt);
  if (st != BA_OK) return finish(st);
  bt.ms_default = ms_default;
  bt.ms_tuned = cur_ms;
  *out = bt;
  return finish(BA_OK);
}

BA_API ba_status ba_tune_table_lookup(const char* path, const char* gpu_name, int32_t sm_count, int32_t precision,
                                      ba_tune* out) {
  if (!path || !gpu_name || !out || (precision != BA_FP64 && precision != BA_MIXED)) return BA_ERR_INVALID;
  std::ifstream f(path);
  if (!f) return BA_ERR_NOT_FOUND;
  std::string want(gpu_name);
  std::replace(want.begin(), want.end(), ' ', '_');
  const std::string prec = precision == BA_MIXED ? "mixed" : "fp64";
  bool found = false;
  ba_tune result{};
  std::string line;
  while (std::getline(f, line)) {
    const size_t hash = line.find('#');
    if (hash != std::string::npos) line.resize(hash);
    std::istringstream in(line);
    std::string name, pr;
    int sms = 0;
    if (!(in >> name >> sms >> pr)) continue;
    if (name != want || sms != sm_count || pr != prec) continue;
    ba_tune t = tune_to_abi(TuneParams{});
    std::string kv;
    while (in >> kv) {
      const size_t eq = kv.find('=');
      if (eq == std::string::npos) return BA_ERR_INVALID;
      const std::string key = kv.substr(0, eq), val = kv.substr(eq + 1);
      char* end = nullptr;
      const double v = std::strtod(val.c_str(), &end);
      if (end == val.c_str() || *end != '\0') return BA_ERR_INVALID;
      if (key == "chunk_tiles") t.chunk_tiles = (int)v;
      else if (key == "lin_ctas_per_sm") t.lin_ctas_per_sm = (int)v;
      else if (key == "back_ctas_per_sm") t.back_ctas_per_sm = (int)v;
      else if (key == "factor_nb") t.factor_nb = (int)v;
      else if (key == "factor_threads") t.factor_threads = (int)v;
      else if (key == "big_panel_w") t.big_panel_w = (int)v;
      else if (key == "batch_chains") t.batch_chains = (int)v;
      else if (key == "ms_default") t.ms_default = v;
      else if (key == "ms_tuned") t.ms_tuned = v;
      else return BA_ERR_INVALID;
    }
    std::string why;
    if (!tune_in_range(t, precision == BA_MIXED, &why)) return BA_ERR_INVALID;
    result = t;
    found = true;  // the last matching line wins
  }
  if (!found) return BA_ERR_NOT_FOUND;
  *out = result;
  return BA_OK;
}

BA_API ba_status ba_probe_fp32_fma(ba_ctx* ctx, int32_t ctas_per_sm, int32_t iters, double* tflops, double* ms) {
  if (!ctx || !tflops || !ms || ctas_per_sm < 1 || iters < 1) return BA_ERR_INVALID;
  CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  float* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(ctx, cudaMallocAsync((void**)&sink, sizeof(float), ctx->stream));
  CUDA_TRY(ctx, cudaEventCreate(&e0));
  CUDA_TRY(ctx, cudaEventCreate(&e1));
  const int ctas = ctas_per_sm * num_sms();
  launch_fma_probe(ctas, iters, sink, ctx->stream);  // warm-up
  cudaEventRecord(e0, ctx->stream);
  launch_fma_probe(ctas, iters, sink, ctx->stream);
  cudaEventRecord(e1, ctx->stream);
  note_direct(ctx);
  const cudaError_t e = cudaEventSynchronize(e1);
  float el = 0.f;
  if (e == cudaSuccess) cudaEventElapsedTime(&el, e0, e1);
  cudaFreeAsync(sink, ctx->stream);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || !(el > 0.f)) return set_err(ctx, BA_ERR_CUDA, "ba_probe_fp32_fma: timing failed");
  *ms = el;
  *tflops = 2.0 * 16.0 * (double)iters * 512.0 * (double)ctas / (el * 1e-3) / 1e12;
  return BA_OK;
}

BA_API ba_status ba_destroy_cluster(ba_ctx* ctx, ba_cluster_id id) {
  if (!ctx) return BA_ERR_INVALID;
  std::lock_guard<std::mutex> g(ctx->api_mu);
  Cluster* c = find_cluster(ctx, id);
  if (!c) return BA_ERR_NOT_FOUND;
  if (c->in_service) return set_err(ctx, BA_ERR_INVALID, "cluster is in service");
  // stream-ordered: the arena is released after the work already queued on
  // the context's stream; serving rounds that used it have completed
  drop_plans_with(ctx, id);
  ctx->clusters.erase(id);
  ctx->mem -= c->arena_bytes;
  // a serving round in flight may still read the cluster (inert, after its
  // ticket completed): the memory goes back once that round has ended
  if (ctx->slots.tail) CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->stream, ctx->slots.tail, 0));
  CUDA_TRY(ctx, cudaFreeAsync(c->arena, ctx->stream));
  delete c;
  return BA_OK;
}

BA_API ba_status ba_shutdown(ba_ctx* ctx) {
  if (!ctx) return BA_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(ctx->sv_mu);
    ctx->sched_stop = true;
    ctx->sv_cv.notify_all();
  }
  if (ctx->sched.joinable()) ctx->sched.join();
  for (auto& kv : ctx->tickets)
    if (kv.second.ready) cudaEventDestroy(kv.second.ready);
  cudaStreamSynchronize(ctx->sched_stream);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->slots.graph.exec) cudaGraphExecDestroy(ctx->slots.graph.exec);
  free_probe(ctx->slots.graph.probe);
  if (ctx->slots.dbuf) cudaFree(ctx->slots.dbuf);
  if (ctx->slots.hbuf) cudaFreeHost(ctx->slots.hbuf);
  for (auto& ev : ctx->slots.done)
    if (ev) cudaEventDestroy(ev);
  if (ctx->slots.tail) cudaEventDestroy(ctx->slots.tail);
  for (auto& kv : ctx->plans) free_plan(ctx, kv.second);
  for (auto& kv : ctx->clusters) {
    cudaFreeAsync(kv.second->arena, ctx->stream);
    delete kv.second;
  }
  cudaStreamSynchronize(ctx->stream);
  cudaMemPoolDestroy(ctx->pool);
  cudaStreamDestroy(ctx->sched_stream);
  cudaStreamDestroy(ctx->plan_stream);
  cudaStreamDestroy(ctx->copy_stream);
  for (cudaStream_t cs : ctx->chain_streams) cudaStreamDestroy(cs);
  for (cudaEvent_t ce : ctx->chain_join) cudaEventDestroy(ce);
  if (ctx->chain_fork) cudaEventDestroy(ctx->chain_fork);
  if (ctx->hstage) cudaFreeHost(ctx->hstage);
  if (ctx->state_done) cudaEventDestroy(ctx->state_done);
  for (auto& b : ctx->stage_free) cudaFreeHost(b.first);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return BA_OK;
}

}  // extern "C"
