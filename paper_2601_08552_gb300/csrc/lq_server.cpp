// lq_server.cpp -- continuous-batching serving loop for simulation requests.
//
// A host thread owns one CUDA stream, a stream-ordered memory pool and a
// table of active requests, each a one-chain simulation with its own device
// arena.  Every tick it (1) admits queued requests while their device
// footprint fits the HBM budget and a slot is free, (2) runs every active
// request in a single persistent launch over a gathered descriptor array, so
// requests that arrive while others run join the next launch and their work
// overlaps on the device, and (3) retires requests that have done their
// sweeps: their records become a result (sign-weighted means and jackknife
// errors) and their memory returns to the budget.
//
// Within a tick each chain runs as many of its remaining sweeps as fit in the
// tick's time budget (at least one), so small requests are not held to one
// sweep while a large one finishes its sweep.  The budget is the longest
// expected single sweep among the active requests (measured on the device by
// the kernel, or estimated from a cost model for new ones), and at least the
// tick target.  Per-sweep latency samples are the chains' own sweep times.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/lecqmc.h"
#include "lq_device.h"
#include "lq_internal.h"
#include "lq_kernels.h"
#include "lq_lattice.h"

namespace {

struct Pending {
  uint64_t id;
  lq_lattice* lat;  // owned copy
  lq_params params;
  int32_t n_sweeps;
  uint32_t chain_id;
  size_t footprint;
  double t_submit;
  int waited_for_memory;
};

struct Active {
  uint64_t id;
  lq_lattice* lat;
  lq_sim* sim;
  LqChainDev desc;  // authoritative copy of the chain descriptor between ticks
  int32_t n_sweeps, done;
  size_t footprint;
  double t_submit, t_admit;
  long long updates_per_sweep;
  double cost;          // cost-model units per sweep
  long long last_ns;    // measured duration of its latest sweep (0 until one ran)
  double sweep_ms_sum;
  int active_at_admit;  // requests already on the device when this one was admitted
  int waited_for_memory;  // 1 if it reached the head of the queue and had to wait for memory to be freed
};

// Latency samples in a fixed histogram: 200 logarithmic bins per decade from
// 1 microsecond to 10^4 s (a bin is 1.2 % wide), so the store does not grow
// with the number of sweeps and a percentile costs one pass over the bins.
struct LatencyHist {
  static constexpr int kPerDecade = 200, kDecades = 10;
  static constexpr double kLo = 1e-3;  // ms
  std::vector<long long> bins = std::vector<long long>(kPerDecade * kDecades + 2, 0);
  long long n = 0;
  double lo = 0.0, hi = 0.0;
  void add(double ms, long long count = 1) {
    if (count <= 0 || !(ms >= 0.0)) return;
    int b;
    if (ms < kLo) b = 0;
    else {
      b = 1 + (int)std::floor(std::log10(ms / kLo) * kPerDecade);
      if (b > kPerDecade * kDecades) b = kPerDecade * kDecades + 1;
    }
    bins[b] += count;
    if (n == 0 || ms < lo) lo = ms;
    if (n == 0 || ms > hi) hi = ms;
    n += count;
  }
  // the q-quantile as the geometric centre of its bin (clamped to the extremes seen)
  double quantile(double q) const {
    if (n == 0) return 0.0;
    const long long want = (long long)std::ceil(q * (double)n);
    long long c = 0;
    for (size_t b = 0; b < bins.size(); ++b) {
      c += bins[b];
      if (c >= std::max(want, 1LL)) {
        double v = b == 0 ? lo : kLo * std::pow(10.0, ((double)b - 0.5) / kPerDecade);
        return std::min(std::max(v, lo), hi);
      }
    }
    return hi;
  }
};

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct lq_server {
  int device = 0, prec = 0, max_active = 0, queue_cap = 0;
  size_t budget = 0, in_use = 0;
  cudaStream_t st = nullptr;
  cudaMemPool_t pool = nullptr;
  lq_allocator alloc;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::thread worker;
  uint64_t next_id = 1;
  std::deque<Pending> queue;
  std::vector<Active> active;
  std::map<uint64_t, lq_result> done;
  std::map<uint64_t, int> state;  // 0 queued, 1 active, 2 done
  // device descriptor table, order list and per-chain sweep caps of the gathered launch
  LqChainDev* d_slots = nullptr;
  int* d_order = nullptr;
  int* d_caps = nullptr;
  int* d_queue = nullptr;
  int* d_queue2 = nullptr;                // chain queue of the large-plan launch
  cudaStream_t st2 = nullptr;             // its stream, forked from and joined to st
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  char* d_ws = nullptr;  // workspace of big plans for the gathered launches (grown on demand)
  size_t ws_cap = 0;
  int dev_sms = 1;
  double tick_target_ms = 20.0;
  double ns_per_cost = 0.0;  // running estimate of sweep nanoseconds per cost unit
  // statistics
  LatencyHist sweep_ms;       // one sample per sweep: that sweep's own device time
  LatencyHist tick_ms;        // one sample per batched launch
  LatencyHist wall_sweep_ms;  // one sample per request: (retirement - submission) / sweeps
  long long submitted = 0, admitted = 0, completed = 0, rejected = 0;
  double updates_done = 0.0, busy_s = 0.0, t_start = 0.0, admit_s = 0.0, retire_s = 0.0;
  std::string last_err;
};

static lq_status srv_fail(lq_status s, const std::string& msg) { return lq_internal_fail(s, msg); }

// Stream-ordered device memory for the request arenas: allocation and release
// on the server stream never synchronize the device.
static void* srv_alloc(void* ctx, size_t bytes, void* stream) {
  lq_server* S = (lq_server*)ctx;
  void* p = nullptr;
  if (cudaMallocFromPoolAsync(&p, bytes, S->pool, (cudaStream_t)stream) != cudaSuccess) return nullptr;
  return p;
}
static void srv_free(void*, void* ptr, size_t, void* stream) { cudaFreeAsync(ptr, (cudaStream_t)stream); }

// Workspace for a gathered launch of `grid` CTAs (stream-ordered, from the pool).
static cudaError_t ensure_ws(lq_server* S, size_t bytes) {
  if (bytes <= S->ws_cap) return cudaSuccess;
  if (S->d_ws) cudaFreeAsync(S->d_ws, S->st);
  S->d_ws = nullptr;
  S->ws_cap = 0;
  void* p = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, S->pool, S->st);
  if (e != cudaSuccess) return e;
  S->d_ws = (char*)p;
  S->ws_cap = bytes;
  return cudaSuccess;
}

static void finish_failed(lq_server* S, uint64_t id, size_t footprint, lq_status st) {
  lq_result r;
  std::memset(&r, 0, sizeof(r));
  r.status = st;
  std::lock_guard<std::mutex> g(S->mu);
  S->in_use -= footprint;
  S->done[id] = r;
  S->state[id] = 2;
  S->completed++;
}

static void retire_impl(lq_server* S, Active& a);

static void retire(lq_server* S, Active& a) {
  const double t0 = now_s();
  retire_impl(S, a);
  std::lock_guard<std::mutex> g(S->mu);
  S->retire_s += now_s() - t0;
}

static void retire_impl(lq_server* S, Active& a) {
  lq_result r;
  std::memset(&r, 0, sizeof(r));
  // hand the descriptor back to the simulation object, then read it out
  const lq_sim_launch_info inf = lq_internal_sim_info(a.sim);
  lq_status st = LQ_OK;
  if (cudaMemcpyAsync(inf.d_chains, &a.desc, sizeof(LqChainDev), cudaMemcpyHostToDevice, S->st) != cudaSuccess ||
      cudaStreamSynchronize(S->st) != cudaSuccess)
    st = LQ_ECUDA;
  lq_internal_sim_invalidate(a.sim);
  if (st == LQ_OK) st = lq_sim_sync(a.sim);  // device errors of the chain (bad input, numerics)
  std::vector<double> rec((size_t)std::max(a.n_sweeps, 1) * LQ_NOBS);
  int32_t nrec = 0;
  if (st == LQ_OK && a.n_sweeps > 0) st = lq_sim_records(a.sim, 0, a.n_sweeps, &nrec, rec.data());
  if (st == LQ_OK) {
    r.n_records = std::min(nrec, a.n_sweeps);
    lq_internal_obs_stats(rec.data(), r.n_records, std::min(r.n_records, 16), r.obs_mean, r.obs_err);
    st = lq_sim_tracked_weight(a.sim, 0, &r.log_weight, &r.sign);
  }
  if (st == LQ_OK) st = lq_sim_stats(a.sim, 0, r.counts);
  r.status = st;
  r.queue_ms = 1e3 * (a.t_admit - a.t_submit);
  r.total_ms = 1e3 * (now_s() - a.t_submit);
  r.sweep_ms_mean = a.done ? a.sweep_ms_sum / a.done : 0.0;
  r.wall_ms_per_sweep = a.done ? r.total_ms / a.done : 0.0;
  r.active_at_admit = a.active_at_admit;
  r.waited_for_memory = a.waited_for_memory;
  lq_sim_destroy(a.sim);
  lq_lattice_destroy(a.lat);
  std::lock_guard<std::mutex> g(S->mu);
  if (a.done) S->wall_sweep_ms.add(r.wall_ms_per_sweep);
  S->in_use -= a.footprint;
  S->done[a.id] = r;
  S->state[a.id] = 2;
  S->completed++;
}

// Admit queued requests (first come, first served; a request that does not
// fit waits, and later ones wait behind it).  The new requests' fields and
// Fock states are drawn and their QR chains built in one gathered launch each.
static void admit(lq_server* S) {
  std::vector<Pending> take;
  {
    std::lock_guard<std::mutex> g(S->mu);
    size_t in_use = S->in_use;
    while (!S->queue.empty() && (int)(S->active.size() + take.size()) < S->max_active &&
           in_use + S->queue.front().footprint <= S->budget) {
      take.push_back(S->queue.front());
      in_use += S->queue.front().footprint;
      S->queue.pop_front();
    }
    // the head of the queue that does not fit waits for a retirement
    if (!S->queue.empty() && in_use + S->queue.front().footprint > S->budget) S->queue.front().waited_for_memory = 1;
    S->in_use = in_use;
  }
  if (take.empty()) return;
  std::vector<Active> fresh;
  int M = 1, Nmax = 1, buf = 0;
  for (const Pending& p : take) {
    lq_sim* sim = nullptr;
    lq_status st = lq_internal_sim_create_unbuilt(p.lat, &p.params, p.chain_id, S->st, &S->alloc, &sim);
    if (st != LQ_OK) {
      lq_lattice_destroy(p.lat);
      finish_failed(S, p.id, p.footprint, st);
      continue;
    }
    const lq_sim_launch_info inf = lq_internal_sim_info(sim);
    Active a;
    a.desc = *lq_internal_sim_host_desc(sim);
    a.cost = inf.cost;
    a.id = p.id; a.lat = p.lat; a.sim = sim; a.n_sweeps = p.n_sweeps; a.done = 0; a.footprint = p.footprint;
    a.t_submit = p.t_submit;
    a.updates_per_sweep = 2LL * (long long)std::lround(p.params.beta / p.params.dtau) * lq_lattice_get_view(p.lat).N;
    a.last_ns = 0;
    a.sweep_ms_sum = 0.0;
    a.active_at_admit = (int)S->active.size();
    a.waited_for_memory = p.waited_for_memory;
    fresh.push_back(a);
    M = std::max(M, inf.M);
    Nmax = std::max(Nmax, inf.Nmax);
    buf = std::max(buf, inf.buf_bytes);
  }
  const int n = (int)fresh.size();
  if (n == 0) return;
  std::vector<LqChainDev> desc(n);
  std::vector<int> order(n);
  for (int k = 0; k < n; ++k) {
    desc[k] = fresh[k].desc;
    order[k] = k;
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return fresh[x].cost > fresh[y].cost; });
  const size_t smem = lq::smem_bytes(M, Nmax, buf);
  const int per_sm = std::max(1, lq::max_active_sweep_ctas(S->prec, M, smem));
  cudaError_t e = cudaMemcpyAsync(S->d_slots, desc.data(), sizeof(LqChainDev) * n, cudaMemcpyHostToDevice, S->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S->d_order, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice, S->st);
  const int grid = std::min(n, S->dev_sms * per_sm);
  if (e == cudaSuccess) e = ensure_ws(S, (size_t)grid * lq::workspace_bytes(M, Nmax, buf));
  if (e == cudaSuccess) e = lq::launch_init(S->d_slots, S->d_order, n, std::min(n, 1024), S->st);
  if (e == cudaSuccess)
    e = lq::launch_build(S->prec, S->d_slots, S->d_order, n, M, Nmax, buf, grid, S->st, S->d_ws, S->ws_cap);
  if (e == cudaSuccess) e = cudaMemcpyAsync(desc.data(), S->d_slots, sizeof(LqChainDev) * n, cudaMemcpyDeviceToHost, S->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(S->st);
  const double t_admit = now_s();
  for (int k = 0; k < n; ++k) {
    Active& a = fresh[k];
    a.t_admit = t_admit;
    if (e == cudaSuccess) a.desc = desc[k];
    a.desc.sweep_ns_sum = 0;
    {
      std::lock_guard<std::mutex> g(S->mu);
      S->state[a.id] = 1;
      S->admitted++;
    }
    if (e != cudaSuccess || a.desc.err) {
      a.n_sweeps = 0;  // the build failed: report it through the simulation's own error path
      retire(S, a);
      continue;
    }
    std::lock_guard<std::mutex> g(S->mu);
    S->active.push_back(a);
  }
}

// One launch over every active request of each plan class (at most
// LQ_NS_SMALL particles per spin, then the larger ones): each request runs
// its remaining sweeps up to its class's time budget (at least one).
static void tick(lq_server* S) {
  const int n = (int)S->active.size();
  if (n == 0) return;
  std::vector<LqChainDev> desc(n);
  std::vector<int> order(n), caps(n);
  std::vector<double> est(n);
  std::vector<char> big(n);
  double target_ms;
  {
    std::lock_guard<std::mutex> g(S->mu);
    target_ms = S->tick_target_ms;
  }
  for (int k = 0; k < n; ++k) {
    const Active& a = S->active[k];
    desc[k] = a.desc;
    big[k] = std::max(a.desc.ns[0], a.desc.ns[1]) > LQ_NS_SMALL;
    est[k] = a.last_ns > 0 ? (double)a.last_ns : S->ns_per_cost * a.cost;
    order[k] = k;
  }
  // small class first, each longest first, so the persistent CTAs take the
  // long chains before the short ones
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    if (big[x] != big[y]) return !big[x];
    return est[x] != est[y] ? est[x] > est[y] : S->active[x].cost > S->active[y].cost;
  });
  for (int q = 0; q < n; ++q) caps[q] = S->active[order[q]].n_sweeps - S->active[order[q]].done;
  cudaMemcpyAsync(S->d_slots, desc.data(), sizeof(LqChainDev) * n, cudaMemcpyHostToDevice, S->st);
  cudaMemcpyAsync(S->d_order, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice, S->st);
  cudaMemcpyAsync(S->d_caps, caps.data(), sizeof(int) * n, cudaMemcpyHostToDevice, S->st);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, S->st);
  cudaError_t e = cudaSuccess;
  // the classes' ranges in the order array and their plans
  int qa[3] = {0, 0, n}, Mc[2] = {1, 1}, Nc[2] = {1, 1}, bc[2] = {0, 0}, gc[2] = {0, 0};
  long long budget[2];
  while (qa[1] < n && !big[order[qa[1]]]) ++qa[1];
  for (int cls = 0; cls < 2; ++cls) {
    budget[cls] = std::max(1LL, (long long)(target_ms * 1e6));  // 0 would mean no budget in the kernel
    for (int q = qa[cls]; q < qa[cls + 1]; ++q) {
      const lq_sim_launch_info inf = lq_internal_sim_info(S->active[order[q]].sim);
      Mc[cls] = std::max(Mc[cls], inf.M);
      Nc[cls] = std::max(Nc[cls], inf.Nmax);
      bc[cls] = std::max(bc[cls], inf.buf_bytes);
      budget[cls] = std::max(budget[cls], (long long)est[order[q]]);
    }
    if (qa[cls + 1] > qa[cls]) {
      const size_t smem = lq::smem_bytes(Mc[cls], Nc[cls], bc[cls]);
      const int per_sm = std::max(1, lq::max_active_sweep_ctas(S->prec, Mc[cls], smem));
      gc[cls] = std::min(qa[cls + 1] - qa[cls], S->dev_sms * per_sm);
    }
  }
  if (gc[1]) e = ensure_ws(S, (size_t)gc[1] * lq::workspace_bytes(Mc[1], Nc[1], bc[1]));
  // with both classes, the large one runs on the second stream (its own chain
  // queue) concurrently with the small one, joined by events
  const bool both = gc[0] && gc[1];
  bool forked = false;
  if (e == cudaSuccess && both) {
    e = cudaEventRecord(S->ev_fork, S->st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(S->st2, S->ev_fork, 0);
    forked = e == cudaSuccess;
  }
  for (int cls = 1; cls >= 0 && e == cudaSuccess; --cls) {
    if (!gc[cls]) continue;
    const int q0 = qa[cls], nq = qa[cls + 1] - qa[cls];
    cudaStream_t st = (both && cls == 1) ? S->st2 : S->st;
    int* queue = (both && cls == 1) ? S->d_queue2 : S->d_queue;
    e = lq::launch_sweep(S->prec, S->d_slots, S->d_order + q0, nq, queue, 1, 1, Mc[cls], Nc[cls], bc[cls], gc[cls], st,
                         cls ? S->d_ws : nullptr, cls ? S->ws_cap : 0, S->d_caps + q0, budget[cls]);
  }
  if (forked) {
    // join even if a launch failed: later work on st (a workspace release
    // among it) must not overtake what st2 still runs
    cudaError_t ej = cudaEventRecord(S->ev_join, S->st2);
    if (ej == cudaSuccess) ej = cudaStreamWaitEvent(S->st, S->ev_join, 0);
    if (ej != cudaSuccess) cudaStreamSynchronize(S->st2);
    if (e == cudaSuccess) e = ej;
  }
  cudaEventRecord(e1, S->st);
  cudaMemcpyAsync(desc.data(), S->d_slots, sizeof(LqChainDev) * n, cudaMemcpyDeviceToHost, S->st);
  cudaError_t e2 = cudaStreamSynchronize(S->st);
  if (e == cudaSuccess) e = e2;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::vector<std::pair<double, long long>> samples;  // (ms, count)
  double upd = 0.0, ratio_sum = 0.0;
  int ratio_n = 0;
  for (int k = 0; k < n; ++k) {
    Active& a = S->active[k];
    const int d = (int)(desc[k].sweep - a.desc.sweep);
    if (d > 0) {
      // each sweep's own time from the descriptor's ring; a chain that ran
      // more sweeps than the ring holds gives the rest their mean
      const int kept = std::min(d, LQ_SWEEP_RING);
      double kept_ns = 0.0;
      for (int t = d - kept; t < d; ++t) {
        const long long ns = desc[k].sweep_ns_ring[(a.desc.sweep + (uint32_t)t) % LQ_SWEEP_RING];
        kept_ns += (double)ns;
        samples.emplace_back(1e-6 * (double)ns, 1);
      }
      if (d > kept) samples.emplace_back(1e-6 * ((double)desc[k].sweep_ns_sum - kept_ns) / (d - kept), d - kept);
      a.sweep_ms_sum += 1e-6 * (double)desc[k].sweep_ns_sum;
      a.last_ns = desc[k].sweep_ns_last;
      if (a.cost > 0) { ratio_sum += (double)desc[k].sweep_ns_last / a.cost; ++ratio_n; }
      upd += (double)d * (double)a.updates_per_sweep;
      a.done += d;
    }
    a.desc = desc[k];
    a.desc.sweep_ns_sum = 0;
  }
  if (ratio_n) S->ns_per_cost = ratio_sum / ratio_n;
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->busy_s += ms * 1e-3;
    S->tick_ms.add(ms);
    for (const auto& sm : samples) S->sweep_ms.add(sm.first, sm.second);
    S->updates_done += upd;
    if (e != cudaSuccess) S->last_err = cudaGetErrorString(e);
  }
  std::vector<Active> keep;
  for (Active& a : S->active) {
    if (e != cudaSuccess || a.done >= a.n_sweeps) retire(S, a);
    else keep.push_back(a);
  }
  std::lock_guard<std::mutex> g(S->mu);
  S->active.swap(keep);
}

static void run_loop(lq_server* S) {
  cudaSetDevice(S->device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait_for(lk, std::chrono::milliseconds(2),
                     [&] { return S->stop || !S->queue.empty() || !S->active.empty(); });
      if (S->stop && S->queue.empty() && S->active.empty()) break;
      if (S->stop) {  // drop what was never admitted
        for (const Pending& p : S->queue) {
          lq_lattice_destroy(p.lat);
          S->state[p.id] = 2;
          lq_result r;
          std::memset(&r, 0, sizeof(r));
          r.status = LQ_ETIMEOUT;
          S->done[p.id] = r;
        }
        S->queue.clear();
      }
    }
    const double t0 = now_s();
    admit(S);
    const double t1 = now_s();
    tick(S);
    std::lock_guard<std::mutex> g(S->mu);
    S->admit_s += t1 - t0;
  }
}

extern "C" lq_status lq_server_create(int32_t device, size_t hbm_budget, int32_t precision, int32_t max_active,
                                      int32_t queue_capacity, lq_server** out) {
  if (!out || hbm_budget == 0 || max_active < 1 || queue_capacity < 1) return srv_fail(LQ_EINVAL, "bad server arguments");
  if (precision != LQ_FP64 && precision != LQ_MIXED && precision != LQ_MIXED_DW) return srv_fail(LQ_EINVAL, "bad precision");
  lq_server* S = new (std::nothrow) lq_server();
  if (!S) return srv_fail(LQ_ENOMEM, "host allocation");
  S->device = device; S->prec = precision; S->max_active = max_active; S->queue_cap = queue_capacity;
  S->budget = hbm_budget;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc((void**)&S->d_slots, sizeof(LqChainDev) * max_active);
  if (e == cudaSuccess) e = cudaMalloc((void**)&S->d_order, sizeof(int) * max_active);
  if (e == cudaSuccess) e = cudaMalloc((void**)&S->d_caps, sizeof(int) * max_active);
  if (e == cudaSuccess) e = cudaMalloc((void**)&S->d_queue, sizeof(int) * (1 + 1024));
  if (e == cudaSuccess) e = cudaMalloc((void**)&S->d_queue2, sizeof(int) * (1 + 1024));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->st2, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&S->dev_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    e = cudaMemPoolCreate(&S->pool, &props);
    uint64_t keep_all = UINT64_MAX;  // keep released memory in the pool for the next request
    if (e == cudaSuccess) e = cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep_all);
  }
  S->alloc.ctx = S;
  S->alloc.alloc = srv_alloc;
  S->alloc.free = srv_free;
  if (e != cudaSuccess) {
    lq_server_destroy(S);
    return srv_fail(LQ_ECUDA, std::string("server set-up: ") + cudaGetErrorString(e));
  }
  S->t_start = now_s();
  S->worker = std::thread(run_loop, S);
  *out = S;
  return LQ_OK;
}

extern "C" lq_status lq_server_submit(lq_server* S, const lq_request* req, uint64_t* id) {
  if (!S || !req || !req->lattice || !id || req->n_sweeps < 1) return srv_fail(LQ_EINVAL, "bad request");
  if (req->params.precision != S->prec) return srv_fail(LQ_EINVAL, "request precision differs from the server's");
  const size_t fp = lq_internal_footprint(req->lattice, &req->params);
  if (fp > S->budget) return srv_fail(LQ_EINVAL, "request needs more device memory than the server budget");
  const lq_lattice_view v = lq_lattice_get_view(req->lattice);
  // owned copy of the lattice, so the caller may destroy theirs
  std::vector<int> bi(v.nb), bj(v.nb);
  std::vector<double> kb(v.nb);
  lq_lattice_bonds(req->lattice, bi.data(), bj.data(), kb.data(), nullptr);
  lq_lattice* copy = nullptr;
  lq_status st = lq_lattice_from_bonds(v.N, v.nb, bi.data(), bj.data(), kb.data(), v.has_eps ? v.eps : nullptr,
                                       v.sub, &copy);
  if (st != LQ_OK) return st;
  std::lock_guard<std::mutex> g(S->mu);
  if ((int)S->queue.size() >= S->queue_cap) {
    lq_lattice_destroy(copy);
    S->rejected++;
    return srv_fail(LQ_EBUSY, "request queue is full");
  }
  Pending p;
  p.id = S->next_id++;
  p.lat = copy;
  p.params = req->params;
  p.n_sweeps = req->n_sweeps;
  p.chain_id = req->chain_id;
  p.footprint = fp;
  p.t_submit = now_s();
  p.waited_for_memory = 0;
  S->queue.push_back(p);
  S->state[p.id] = 0;
  S->submitted++;
  *id = p.id;
  S->cv.notify_one();
  return LQ_OK;
}

extern "C" lq_status lq_server_poll(lq_server* S, uint64_t id, lq_result* out) {
  if (!S || !out) return srv_fail(LQ_EINVAL, "bad arguments");
  std::lock_guard<std::mutex> g(S->mu);
  auto it = S->done.find(id);
  if (it == S->done.end()) {
    if (!S->state.count(id)) return srv_fail(LQ_EINVAL, "unknown request id");
    return srv_fail(LQ_ENOTFOUND, "request not finished");
  }
  *out = it->second;
  S->done.erase(it);
  S->state.erase(id);
  return LQ_OK;
}

extern "C" lq_status lq_server_stats(lq_server* S, lq_server_info* out) {
  if (!S || !out) return srv_fail(LQ_EINVAL, "bad arguments");
  std::lock_guard<std::mutex> g(S->mu);
  std::memset(out, 0, sizeof(*out));
  out->p50_sweep_ms = S->sweep_ms.quantile(0.50);
  out->p99_sweep_ms = S->sweep_ms.quantile(0.99);
  out->p50_tick_ms = S->tick_ms.quantile(0.50);
  out->p99_tick_ms = S->tick_ms.quantile(0.99);
  out->p50_wall_sweep_ms = S->wall_sweep_ms.quantile(0.50);
  out->p99_wall_sweep_ms = S->wall_sweep_ms.quantile(0.99);
  out->sweeps = S->sweep_ms.n;
  out->ticks = (int64_t)S->tick_ms.n;
  out->submitted = S->submitted;
  out->admitted = S->admitted;
  out->completed = S->completed;
  out->rejected = S->rejected;
  out->active = (int64_t)S->active.size();
  out->queued = (int64_t)S->queue.size();
  out->busy_s = S->busy_s;
  out->wall_s = now_s() - S->t_start;
  out->updates_per_s = S->busy_s > 0 ? S->updates_done / S->busy_s : 0.0;
  out->admit_s = S->admit_s;
  out->retire_s = S->retire_s;
  out->hbm_in_use = S->in_use;
  return LQ_OK;
}

extern "C" lq_status lq_server_set_tick_target(lq_server* S, double ms) {
  if (!S || !(ms >= 0.0) || !std::isfinite(ms)) return srv_fail(LQ_EINVAL, "tick target must be a finite number >= 0");
  std::lock_guard<std::mutex> g(S->mu);
  S->tick_target_ms = ms;
  return LQ_OK;
}

extern "C" lq_status lq_server_destroy(lq_server* S) {
  if (!S) return LQ_OK;
  if (S->worker.joinable()) {
    {
      std::lock_guard<std::mutex> g(S->mu);
      S->stop = true;
    }
    S->cv.notify_one();
    S->worker.join();
  }
  if (S->d_ws && S->st) cudaFreeAsync(S->d_ws, S->st);
  if (S->st) cudaStreamSynchronize(S->st);
  cudaFree(S->d_slots);
  cudaFree(S->d_order);
  cudaFree(S->d_caps);
  cudaFree(S->d_queue);
  cudaFree(S->d_queue2);
  if (S->st2) {
    cudaStreamSynchronize(S->st2);
    cudaStreamDestroy(S->st2);
  }
  if (S->ev_fork) cudaEventDestroy(S->ev_fork);
  if (S->ev_join) cudaEventDestroy(S->ev_join);
  if (S->pool) cudaMemPoolDestroy(S->pool);
  if (S->st) cudaStreamDestroy(S->st);
  delete S;
  return LQ_OK;
}
