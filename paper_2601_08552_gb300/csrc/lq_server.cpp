// lq_server.cpp -- continuous-batching serving loop for simulation requests.
//
// A host thread owns one CUDA stream and a table of active requests, each a
// one-chain simulation with its own device arena.  Every tick it (1) admits
// queued requests while their device footprint fits the HBM budget and a
// slot is free, (2) runs ONE sweep of every active request in a single
// persistent launch over a gathered descriptor array, so requests that
// arrive while others run join the next launch and their work overlaps on
// the device, and (3) retires requests that have done their sweeps: their
// records become a result (sign-weighted means and jackknife errors) and
// their memory returns to the budget.  The tick time, taken with CUDA events
// on the server stream, is the per-sweep latency every active request saw.
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
};

struct Active {
  uint64_t id;
  lq_lattice* lat;
  lq_sim* sim;
  int32_t n_sweeps, done;
  size_t footprint;
  double t_submit, t_admit;
  long long updates_per_sweep;
  double sweep_ms_sum;
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
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::thread worker;
  uint64_t next_id = 1;
  std::deque<Pending> queue;
  std::vector<Active> active;
  std::map<uint64_t, lq_result> done;
  std::map<uint64_t, int> state;  // 0 queued, 1 active, 2 done
  // device descriptor table and order list for the gathered launch
  LqChainDev* d_slots = nullptr;
  int* d_order = nullptr;
  int* d_queue = nullptr;
  // statistics
  std::vector<double> tick_ms;  // per-sweep latency samples (one per active request per tick)
  long long submitted = 0, admitted = 0, completed = 0, rejected = 0;
  double updates_done = 0.0, busy_s = 0.0, t_start = 0.0;
  std::string last_err;
};

static lq_status srv_fail(lq_status s, const std::string& msg) { return lq_internal_fail(s, msg); }

static void retire(lq_server* S, Active& a) {
  lq_result r;
  std::memset(&r, 0, sizeof(r));
  r.status = LQ_OK;
  std::vector<double> rec((size_t)std::max(a.n_sweeps, 1) * LQ_NOBS);
  int32_t nrec = 0;
  lq_status st = lq_sim_records(a.sim, 0, a.n_sweeps, &nrec, rec.data());
  if (st == LQ_OK) {
    r.n_records = std::min(nrec, a.n_sweeps);
    lq_internal_obs_stats(rec.data(), r.n_records, std::min(r.n_records, 16), r.obs_mean, r.obs_err);
    st = lq_sim_tracked_weight(a.sim, 0, &r.log_weight, &r.sign);
  }
  if (st == LQ_OK) st = lq_sim_stats(a.sim, 0, r.counts);
  if (st == LQ_OK) st = lq_sim_sync(a.sim);
  r.status = st;
  r.queue_ms = 1e3 * (a.t_admit - a.t_submit);
  r.total_ms = 1e3 * (now_s() - a.t_submit);
  r.sweep_ms_mean = a.done ? a.sweep_ms_sum / a.done : 0.0;
  lq_sim_destroy(a.sim);
  lq_lattice_destroy(a.lat);
  std::lock_guard<std::mutex> g(S->mu);
  S->in_use -= a.footprint;
  S->done[a.id] = r;
  S->state[a.id] = 2;
  S->completed++;
}

// Admit queued requests (first come, first served; a request that does not
// fit waits, and later ones wait behind it).
static void admit(lq_server* S) {
  for (;;) {
    Pending p;
    {
      std::lock_guard<std::mutex> g(S->mu);
      if (S->queue.empty() || (int)S->active.size() >= S->max_active) return;
      if (S->in_use + S->queue.front().footprint > S->budget) return;
      p = S->queue.front();
      S->queue.pop_front();
      S->in_use += p.footprint;
    }
    lq_sim* sim = nullptr;
    const lq_lattice* lp = p.lat;
    lq_status st = lq_sim_create(&lp, &p.params, 1, &p.chain_id, S->st, nullptr, &sim);
    if (st == LQ_OK) st = lq_sim_init(sim);
    if (st != LQ_OK) {
      lq_result r;
      std::memset(&r, 0, sizeof(r));
      r.status = st;
      if (sim) lq_sim_destroy(sim);
      lq_lattice_destroy(p.lat);
      std::lock_guard<std::mutex> g(S->mu);
      S->in_use -= p.footprint;
      S->done[p.id] = r;
      S->state[p.id] = 2;
      S->completed++;
      continue;
    }
    Active a;
    a.id = p.id; a.lat = p.lat; a.sim = sim; a.n_sweeps = p.n_sweeps; a.done = 0; a.footprint = p.footprint;
    a.t_submit = p.t_submit; a.t_admit = now_s();
    a.updates_per_sweep = 2LL * (long long)std::lround(p.params.beta / p.params.dtau) * lq_lattice_get_view(p.lat).N;
    a.sweep_ms_sum = 0.0;
    std::lock_guard<std::mutex> g(S->mu);
    S->active.push_back(a);
    S->state[a.id] = 1;
    S->admitted++;
  }
}

// One sweep of every active request in one launch.
static void tick(lq_server* S) {
  const int n = (int)S->active.size();
  if (n == 0) return;
  int M = 1, Nmax = 1, buf = 0;
  std::vector<LqChainDev> desc(n);
  std::vector<int> order(n);
  for (int k = 0; k < n; ++k) {
    const lq_sim_launch_info inf = lq_internal_sim_info(S->active[k].sim);
    cudaMemcpyAsync(&desc[k], inf.d_chains, sizeof(LqChainDev), cudaMemcpyDeviceToHost, S->st);
    M = std::max(M, inf.M);
    Nmax = std::max(Nmax, inf.Nmax);
    buf = std::max(buf, inf.buf_bytes);
    order[k] = k;
  }
  cudaStreamSynchronize(S->st);
  // longest first
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (double)desc[a].L * desc[a].N > (double)desc[b].L * desc[b].N;
  });
  cudaMemcpyAsync(S->d_slots, desc.data(), sizeof(LqChainDev) * n, cudaMemcpyHostToDevice, S->st);
  cudaMemcpyAsync(S->d_order, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice, S->st);
  int dev_sms = 1;
  cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, S->device);
  const size_t smem = lq::smem_bytes(M, Nmax, buf);
  const int per_sm = std::max(1, lq::max_active_sweep_ctas(S->prec, smem));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, S->st);
  cudaError_t e = lq::launch_sweep(S->prec, S->d_slots, S->d_order, n, S->d_queue, 1, 1, M, Nmax, buf,
                                   std::min(n, dev_sms * per_sm), S->st);
  cudaEventRecord(e1, S->st);
  cudaMemcpyAsync(desc.data(), S->d_slots, sizeof(LqChainDev) * n, cudaMemcpyDeviceToHost, S->st);
  cudaStreamSynchronize(S->st);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int k = 0; k < n; ++k) {
    const lq_sim_launch_info inf = lq_internal_sim_info(S->active[k].sim);
    cudaMemcpyAsync(inf.d_chains, &desc[k], sizeof(LqChainDev), cudaMemcpyHostToDevice, S->st);
    lq_internal_sim_invalidate(S->active[k].sim);
  }
  cudaStreamSynchronize(S->st);
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->busy_s += ms * 1e-3;
    for (int k = 0; k < n; ++k) {
      S->tick_ms.push_back(ms);
      S->updates_done += (double)S->active[k].updates_per_sweep;
    }
    if (e != cudaSuccess) S->last_err = cudaGetErrorString(e);
  }
  std::vector<Active> keep;
  for (Active& a : S->active) {
    a.done++;
    a.sweep_ms_sum += ms;
    if (a.done >= a.n_sweeps) retire(S, a);
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
    admit(S);
    tick(S);
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
  if (e == cudaSuccess) e = cudaMalloc((void**)&S->d_queue, sizeof(int) * (1 + 1024));
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
  std::vector<double> t = S->tick_ms;
  if (!t.empty()) {
    std::sort(t.begin(), t.end());
    out->p50_sweep_ms = t[(size_t)(0.50 * (t.size() - 1))];
    out->p99_sweep_ms = t[(size_t)(0.99 * (t.size() - 1))];
  }
  out->submitted = S->submitted;
  out->admitted = S->admitted;
  out->completed = S->completed;
  out->rejected = S->rejected;
  out->active = (int64_t)S->active.size();
  out->queued = (int64_t)S->queue.size();
  out->busy_s = S->busy_s;
  out->wall_s = now_s() - S->t_start;
  out->updates_per_s = S->busy_s > 0 ? S->updates_done / S->busy_s : 0.0;
  out->hbm_in_use = S->in_use;
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
  if (S->st) cudaStreamSynchronize(S->st);
  cudaFree(S->d_slots);
  cudaFree(S->d_order);
  cudaFree(S->d_queue);
  if (S->st) cudaStreamDestroy(S->st);
  delete S;
  return LQ_OK;
}
