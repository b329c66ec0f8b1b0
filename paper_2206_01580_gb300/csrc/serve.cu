// Continuous-batching server for energy + force prediction (host runtime).
//
// The paper observes that one configuration leaves the GPU mostly idle and
// that batching 1000 configurations cuts the cost per configuration by two
// orders of magnitude (timings section). The server turns a stream of
// independent requests into such batches while requests keep arriving:
//   * admission: a request is accepted only while the number of requests and
//     of atoms held by the server (queued, running or finished but not yet
//     collected) stay within the configured limits (QMLR_EBUSY otherwise);
//   * a batcher thread owns n_lanes "lanes" (a CUDA stream, a prediction
//     workspace and pinned/device staging buffers each). Whenever a lane is
//     idle it packs the queued requests in arrival order into one CSR batch,
//     copies it to the device, runs the prediction and copies E and F back,
//     so up to n_lanes batches overlap on the device while new requests queue;
//   * each batch is padded to a size bucket (4 buckets per octave) with
//     isolated padding atoms and empty molecules, so the prediction can be
//     captured once per (lane, bucket) as a CUDA graph and replayed;
//   * a host callback enqueued after the copies marks the lane finished; the
//     batcher hands the results to the requests and records their latency.
// A molecule's result does not depend on what else is in its batch: every
// kernel of the prediction computes a molecule's (or atom's) values in an
// order fixed by that molecule alone.
#include "model_internal.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

struct qmlr_server;

namespace qmlr {

static double now_us() {
  using namespace std::chrono;
  return duration<double, std::micro>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  uint64_t ticket = 0;
  int n_atoms = 0;
  std::vector<float> coords;
  std::vector<int32_t> elem;
  double E = 0.0;
  std::vector<float> F;
  int state = 0;   // 0 queued, 1 running, 2 done, 3 failed
  double t_submit = 0, t_done = 0;
};

struct Lane {
  cudaStream_t stream = nullptr;
  PredictWorkspace ws;
  float* d_coords = nullptr;
  int32_t* d_elem = nullptr;
  int32_t* d_mol_ptr = nullptr;
  double* d_E = nullptr;
  float* d_F = nullptr;
  float* h_coords = nullptr;
  int32_t* h_elem = nullptr;
  int32_t* h_mol_ptr = nullptr;
  double* h_E = nullptr;
  float* h_F = nullptr;
  std::vector<std::shared_ptr<Request>> reqs;
  int bucket = 0;
  bool busy = false;
  std::atomic<bool> done{false};
  std::unordered_map<int, cudaGraphExec_t> graphs;
  std::unordered_map<int, size_t> graph_kernels;   // kernel nodes per graph (launch accounting)
  std::unordered_map<int, bool> warmed;
  ::qmlr_server* server = nullptr;
};

}  // namespace qmlr

struct qmlr_server {
  qmlr_model* m = nullptr;
  qmlr_serve_config cfg{};
  std::vector<qmlr::Lane*> lanes;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<qmlr::Request>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<qmlr::Request>> held;   // admitted, not yet collected
  uint64_t next_ticket = 1;
  int64_t atoms_held = 0;
  bool stop = false;
  int device = 0;
  int pad_reserve = 2;   // molecules kept free in every batch for padding
  std::thread worker;
  std::vector<float> latencies_us;
  std::vector<int32_t> latency_atoms;   // atoms of the request behind each latency
  int64_t completed = 0, rejected = 0, batches = 0, batch_atoms = 0;
  double atoms_done = 0, t_first = -1, t_last = 0;
  int fatal = QMLR_OK;
  char fatal_msg[256] = "";
};

namespace qmlr {

static void CUDART_CB lane_finished(void* p) {
  Lane* l = static_cast<Lane*>(p);
  l->done.store(true, std::memory_order_release);
  l->server->cv_work.notify_all();
}

// Batch-size buckets: 64 * 2^(q/8), rounded up to a multiple of 32, capped at max_batch_atoms.
static int bucket_for(int atoms, int cap) {
  double b = 64.0;
  while (b < atoms) b *= 1.0905077326652577;   // 2^(1/8)
  int v = ((int)std::ceil(b) + 31) & ~31;
  return std::min(std::max(v, 32), cap);
}

static int run_prediction(qmlr_server* S, Lane& L, int bucket) {
  const int nm = S->cfg.max_batch_mols;
  auto direct = [&]() {
    return predict_ef_ws(S->m, L.ws, L.d_coords, L.d_elem, L.d_mol_ptr, nm, bucket, L.d_E, L.d_F, L.stream);
  };
  if (!S->cfg.use_graphs) return direct();
  auto it = L.graphs.find(bucket);
  if (it == L.graphs.end()) {
    if (!L.warmed[bucket]) {   // first use of this size: run once outside capture
      L.warmed[bucket] = true;
      return direct();
    }
    cudaGraph_t g = nullptr;
    QMLR_CUDA_TRY(cudaStreamBeginCapture(L.stream, cudaStreamCaptureModeThreadLocal));
    int rc = direct();
    cudaError_t e = cudaStreamEndCapture(L.stream, &g);
    if (rc) return rc;
    if (e != cudaSuccess) {
      set_error("graph capture failed: %s", cudaGetErrorString(e));
      return QMLR_ECUDA;
    }
    size_t n_nodes = 0;
    cudaGraphGetNodes(g, nullptr, &n_nodes);
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      set_error("graph instantiate failed: %s", cudaGetErrorString(e));
      return QMLR_ECUDA;
    }
    it = L.graphs.emplace(bucket, ex).first;
    L.graph_kernels[bucket] = n_nodes;
  }
  QMLR_CUDA_TRY(cudaGraphLaunch(it->second, L.stream));
  for (size_t q = 0; q < L.graph_kernels[bucket]; ++q) count_launch();
  return QMLR_OK;
}

// Pack queued requests into lane L and launch (called with S->mu held).
static int dispatch(qmlr_server* S, Lane& L) {
  const int cap = S->cfg.max_batch_atoms, nm = S->cfg.max_batch_mols;
  int atoms = 0, mols = 0;
  L.reqs.clear();
  while (!S->queue.empty()) {
    auto& r = S->queue.front();
    // room for the request plus the padding molecules of the bucket
    if (atoms + r->n_atoms > cap || mols + 1 + S->pad_reserve > nm) break;
    atoms += r->n_atoms;
    ++mols;
    L.reqs.push_back(r);
    S->queue.pop_front();
  }
  if (L.reqs.empty()) return QMLR_OK;
  const int bucket = bucket_for(atoms, cap);
  // pack real molecules
  int a = 0, mm = 0;
  L.h_mol_ptr[0] = 0;
  for (auto& r : L.reqs) {
    std::copy(r->coords.begin(), r->coords.end(), L.h_coords + 3 * (size_t)a);
    std::copy(r->elem.begin(), r->elem.end(), L.h_elem + a);
    a += r->n_atoms;
    L.h_mol_ptr[++mm] = a;
    r->state = 1;
  }
  // padding atoms: isolated (10 A apart, far from the molecules), one per molecule so
  // that no kernel walks a long padding molecule
  int k = 0;
  while (a < bucket) {
    const int take = 1;
    for (int q = 0; q < take; ++q, ++k) {
      L.h_coords[3 * (size_t)(a + q) + 0] = 1.0e5f + 10.0f * (float)k;
      L.h_coords[3 * (size_t)(a + q) + 1] = 0.f;
      L.h_coords[3 * (size_t)(a + q) + 2] = 0.f;
      L.h_elem[a + q] = 0;
    }
    a += take;
    if (mm < nm) L.h_mol_ptr[++mm] = a;
  }
  while (mm < nm) L.h_mol_ptr[++mm] = a;   // empty molecules up to the fixed count
  L.bucket = bucket;
  cudaStream_t s = L.stream;
  QMLR_CUDA_TRY(cudaMemcpyAsync(L.d_coords, L.h_coords, sizeof(float) * 3 * bucket, cudaMemcpyHostToDevice, s));
  QMLR_CUDA_TRY(cudaMemcpyAsync(L.d_elem, L.h_elem, sizeof(int32_t) * bucket, cudaMemcpyHostToDevice, s));
  QMLR_CUDA_TRY(cudaMemcpyAsync(L.d_mol_ptr, L.h_mol_ptr, sizeof(int32_t) * (nm + 1), cudaMemcpyHostToDevice, s));
  int rc = run_prediction(S, L, bucket);
  if (rc) return rc;
  QMLR_CUDA_TRY(cudaMemcpyAsync(L.h_E, L.d_E, sizeof(double) * L.reqs.size(), cudaMemcpyDeviceToHost, s));
  QMLR_CUDA_TRY(cudaMemcpyAsync(L.h_F, L.d_F, sizeof(float) * 3 * (size_t)atoms, cudaMemcpyDeviceToHost, s));
  L.done.store(false);
  QMLR_CUDA_TRY(cudaLaunchHostFunc(s, lane_finished, &L));
  L.busy = true;
  ++S->batches;
  S->batch_atoms += atoms;
  return QMLR_OK;
}

static void finish(qmlr_server* S, Lane& L) {
  const double t = now_us();
  size_t a = 0;
  for (size_t q = 0; q < L.reqs.size(); ++q) {
    auto& r = L.reqs[q];
    r->E = L.h_E[q];
    r->F.assign(L.h_F + 3 * a, L.h_F + 3 * (a + r->n_atoms));
    a += r->n_atoms;
    r->state = 2;
    r->t_done = t;
    S->latencies_us.push_back((float)(t - r->t_submit));
    S->latency_atoms.push_back(r->n_atoms);
    S->atoms_done += r->n_atoms;
    ++S->completed;
  }
  S->t_last = t;
  L.reqs.clear();
  L.busy = false;
}

static void worker_loop(qmlr_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    bool progressed = false;
    for (Lane* L : S->lanes)
      if (L->busy && L->done.load(std::memory_order_acquire)) {
        finish(S, *L);
        progressed = true;
      }
    if (progressed) S->cv_done.notify_all();
    if (S->fatal == QMLR_OK)
      for (Lane* L : S->lanes)
        if (!L->busy && !S->queue.empty()) {
          int rc = dispatch(S, *L);
          if (rc) {
            S->fatal = rc;
            snprintf(S->fatal_msg, sizeof(S->fatal_msg), "%s", qmlr_last_error());
            for (auto& r : L->reqs) r->state = 3;
            for (auto& r : S->queue) r->state = 3;
            S->queue.clear();
            S->cv_done.notify_all();
          }
        }
    bool any_busy = false;
    for (Lane* L : S->lanes) any_busy |= L->busy;
    if (S->stop && !any_busy) break;
    S->cv_work.wait_for(lk, std::chrono::microseconds(any_busy ? 200 : 2000));
  }
}

static void destroy_lane(Lane* L) {
  if (!L) return;
  if (L->stream) cudaStreamSynchronize(L->stream);
  for (auto& g : L->graphs) cudaGraphExecDestroy(g.second);
  L->ws.release();
  cudaFree(L->d_coords);
  cudaFree(L->d_elem);
  cudaFree(L->d_mol_ptr);
  cudaFree(L->d_E);
  cudaFree(L->d_F);
  cudaFreeHost(L->h_coords);
  cudaFreeHost(L->h_elem);
  cudaFreeHost(L->h_mol_ptr);
  cudaFreeHost(L->h_E);
  cudaFreeHost(L->h_F);
  if (L->stream) cudaStreamDestroy(L->stream);
  delete L;
}

}  // namespace qmlr

using namespace qmlr;

extern "C" int qmlr_serve_create(qmlr_model* m, const qmlr_serve_config* cfg, qmlr_server** out) {
  QMLR_REQUIRE(m && cfg && out, "NULL pointer argument");
  QMLR_REQUIRE(cfg->n_lanes >= 1 && cfg->n_lanes <= 8, "n_lanes must be in 1..8");
  QMLR_REQUIRE(cfg->max_batch_atoms >= m->max_mol_atoms,
               "max_batch_atoms (%d) must hold the largest molecule (%d)", cfg->max_batch_atoms,
               m->max_mol_atoms);
  // padding is at most 9.1 % of a bucket (8 buckets per octave) plus rounding to 32
  const int pad_reserve = (int)std::ceil(0.091 * cfg->max_batch_atoms) + 33;
  QMLR_REQUIRE(cfg->max_batch_mols >= pad_reserve + 1,
               "max_batch_mols must be >= %d (one molecule plus padding)", pad_reserve + 1);
  QMLR_REQUIRE(cfg->max_batch_mols <= cfg->max_batch_atoms + 4096,
               "max_batch_mols must be <= max_batch_atoms + 4096");
  QMLR_REQUIRE(cfg->max_slots >= 1 && cfg->max_inflight_atoms >= m->max_mol_atoms, "bad admission limits");
  const size_t per_atom = PredictWorkspace::bytes_per_atom(m) + 3 * 4 + 4 + 12;
  const int64_t need = (int64_t)cfg->n_lanes * ((int64_t)per_atom * cfg->max_batch_atoms +
                                                (int64_t)cfg->max_batch_mols * 12 + (1 << 20));
  QMLR_REQUIRE(cfg->mem_budget_bytes <= 0 || need <= cfg->mem_budget_bytes,
               "the lanes need %lld bytes, over the memory budget of %lld", (long long)need,
               (long long)cfg->mem_budget_bytes);
  qmlr_server* S = new qmlr_server();
  S->m = m;
  S->cfg = *cfg;
  S->pad_reserve = pad_reserve;
  QMLR_CUDA_TRY(cudaGetDevice(&S->device));
  const size_t na = cfg->max_batch_atoms, nm = cfg->max_batch_mols;
  for (int i = 0; i < cfg->n_lanes; ++i) {
    Lane* L = new Lane();
    L->server = S;
    cudaError_t e = cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&L->d_coords, 12 * na);
    if (e == cudaSuccess) e = cudaMalloc(&L->d_elem, 4 * na);
    if (e == cudaSuccess) e = cudaMalloc(&L->d_mol_ptr, 4 * (nm + 1));
    if (e == cudaSuccess) e = cudaMalloc(&L->d_E, 8 * nm);
    if (e == cudaSuccess) e = cudaMalloc(&L->d_F, 12 * na);
    if (e == cudaSuccess) e = cudaMallocHost(&L->h_coords, 12 * na);
    if (e == cudaSuccess) e = cudaMallocHost(&L->h_elem, 4 * na);
    if (e == cudaSuccess) e = cudaMallocHost(&L->h_mol_ptr, 4 * (nm + 1));
    if (e == cudaSuccess) e = cudaMallocHost(&L->h_E, 8 * nm);
    if (e == cudaSuccess) e = cudaMallocHost(&L->h_F, 12 * na);
    int rc = (e == cudaSuccess) ? L->ws.reserve(m, cfg->max_batch_atoms) : QMLR_ECUDA;
    S->lanes.push_back(L);
    if (rc != QMLR_OK) {
      if (e != cudaSuccess) set_error("server allocation failed: %s", cudaGetErrorString(e));
      for (Lane* x : S->lanes) destroy_lane(x);
      delete S;
      return rc == QMLR_OK ? QMLR_ENOMEM : rc;
    }
  }
  S->worker = std::thread(worker_loop, S);
  *out = S;
  return QMLR_OK;
}

extern "C" int qmlr_serve_submit(qmlr_server* S, const float* host_coords, const int32_t* host_elem,
                                 int32_t n_atoms, uint64_t* ticket) {
  QMLR_REQUIRE(S && ticket, "NULL pointer argument");
  QMLR_REQUIRE(n_atoms >= 1 && host_coords && host_elem, "a request needs at least one atom");
  QMLR_REQUIRE(n_atoms <= S->m->max_mol_atoms, "molecule of %d atoms exceeds the model's limit %d", n_atoms,
               S->m->max_mol_atoms);
  auto r = std::make_shared<Request>();
  r->n_atoms = n_atoms;
  r->coords.assign(host_coords, host_coords + 3 * (size_t)n_atoms);
  r->elem.assign(host_elem, host_elem + n_atoms);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->fatal) {
      set_error("server stopped after an error: %s", S->fatal_msg);
      return S->fatal;
    }
    if ((int64_t)S->held.size() >= S->cfg.max_slots || S->atoms_held + n_atoms > S->cfg.max_inflight_atoms) {
      ++S->rejected;
      set_error("request not admitted: %zu requests and %lld atoms held", S->held.size(),
                (long long)S->atoms_held);
      return QMLR_EBUSY;
    }
    r->ticket = S->next_ticket++;
    r->t_submit = now_us();
    if (S->t_first < 0) S->t_first = r->t_submit;
    S->held.emplace(r->ticket, r);
    S->atoms_held += n_atoms;
    S->queue.push_back(r);
    *ticket = r->ticket;
  }
  S->cv_work.notify_all();
  return QMLR_OK;
}

extern "C" int qmlr_serve_poll(qmlr_server* S, uint64_t ticket, double* host_E, float* host_F,
                               int64_t timeout_us) {
  QMLR_REQUIRE(S, "server is NULL");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->held.find(ticket);
  QMLR_REQUIRE(it != S->held.end(), "unknown or already collected ticket %llu", (unsigned long long)ticket);
  auto r = it->second;
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::microseconds(std::min<int64_t>(std::max<int64_t>(timeout_us, 0), 600000000LL));
  while (r->state < 2) {
    if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && r->state < 2) {
      set_error("request %llu not finished within %lld us", (unsigned long long)ticket, (long long)timeout_us);
      return QMLR_ETIMEOUT;
    }
  }
  if (r->state == 3) {
    S->held.erase(it);
    S->atoms_held -= r->n_atoms;
    set_error("request failed: %s", S->fatal_msg);
    return S->fatal ? S->fatal : QMLR_ECUDA;
  }
  if (host_E) *host_E = r->E;
  if (host_F) std::copy(r->F.begin(), r->F.end(), host_F);
  S->held.erase(it);
  S->atoms_held -= r->n_atoms;
  return QMLR_OK;
}

extern "C" int qmlr_serve_stats(qmlr_server* S, qmlr_serve_report* out) {
  QMLR_REQUIRE(S && out, "NULL pointer argument");
  std::lock_guard<std::mutex> lk(S->mu);
  qmlr_serve_report st{};
  st.completed = S->completed;
  st.rejected = S->rejected;
  st.batches = S->batches;
  if (!S->latencies_us.empty()) {
    std::vector<float> v(S->latencies_us);
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) { return (double)v[std::min(v.size() - 1, (size_t)(q * (v.size() - 1) + 0.5))]; };
    st.p50_us = pct(0.50);
    st.p99_us = pct(0.99);
    st.max_us = v.back();
    double sum = 0;
    for (float x : v) sum += x;
    st.mean_us = sum / v.size();
  }
  const double span = S->t_last - S->t_first;
  if (span > 0) {
    st.throughput_rps = S->completed / (span * 1e-6);
    st.us_per_atom = S->atoms_done > 0 ? span / S->atoms_done : 0;
  }
  st.mean_batch_atoms = S->batches ? (double)S->batch_atoms / S->batches : 0;
  *out = st;
  return QMLR_OK;
}

extern "C" int qmlr_serve_latencies(qmlr_server* S, float* host_latency_us, int32_t* host_atoms, int64_t capacity,
                                    int64_t* count) {
  QMLR_REQUIRE(S && count, "NULL pointer argument");
  QMLR_REQUIRE(capacity >= 0, "capacity must be >= 0");
  std::lock_guard<std::mutex> lk(S->mu);
  const int64_t n = (int64_t)S->latencies_us.size();
  *count = n;
  const int64_t k = std::min(n, capacity);
  if (k > 0) {
    QMLR_REQUIRE(host_latency_us && host_atoms, "NULL output array");
    std::copy(S->latencies_us.begin(), S->latencies_us.begin() + k, host_latency_us);
    std::copy(S->latency_atoms.begin(), S->latency_atoms.begin() + k, host_atoms);
  }
  return QMLR_OK;
}

extern "C" int qmlr_serve_reset_stats(qmlr_server* S) {
  QMLR_REQUIRE(S, "server is NULL");
  std::lock_guard<std::mutex> lk(S->mu);
  S->latencies_us.clear();
  S->latency_atoms.clear();
  S->completed = S->rejected = S->batches = S->batch_atoms = 0;
  S->atoms_done = 0;
  S->t_first = -1;
  S->t_last = 0;
  return QMLR_OK;
}

extern "C" int qmlr_serve_destroy(qmlr_server* S) {
  if (!S) return QMLR_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (Lane* L : S->lanes) destroy_lane(L);
  delete S;
  return QMLR_OK;
}

extern "C" int qmlr_serve_replay(qmlr_server* S, const float* host_coords, const int32_t* host_elem,
                                 const int32_t* host_mol_ptr, int32_t n_pool, const double* arrival_us,
                                 const int32_t* pick, int32_t n_req, int64_t* rejected,
                                 qmlr_serve_report* out) {
  QMLR_REQUIRE(S && host_coords && host_elem && host_mol_ptr && arrival_us && pick && out, "NULL pointer argument");
  QMLR_REQUIRE(n_pool >= 1 && n_req >= 0, "bad sizes");
  for (int i = 0; i < n_req; ++i)
    QMLR_REQUIRE(pick[i] >= 0 && pick[i] < n_pool, "pick[%d] = %d out of range", i, pick[i]);
  int rc = qmlr_serve_reset_stats(S);
  if (rc) return rc;
  // collector: polls tickets in submission order
  std::mutex qm;
  std::condition_variable qcv;
  std::deque<std::pair<uint64_t, int>> pending;
  bool done_submitting = false;
  int first_err = QMLR_OK;
  std::thread collector([&]() {
    std::vector<float> F;
    for (;;) {
      std::pair<uint64_t, int> item;
      {
        std::unique_lock<std::mutex> lk(qm);
        qcv.wait(lk, [&] { return !pending.empty() || done_submitting; });
        if (pending.empty()) return;
        item = pending.front();
        pending.pop_front();
      }
      F.resize(3 * (size_t)item.second);
      double E;
      const int r = qmlr_serve_poll(S, item.first, &E, F.data(), 60000000);
      if (r != QMLR_OK && first_err == QMLR_OK) first_err = r;
    }
  });
  int64_t rej = 0;
  const double t0 = now_us();
  for (int i = 0; i < n_req; ++i) {
    while (now_us() - t0 < arrival_us[i]) {
    }
    const int k = pick[i];
    const int a = host_mol_ptr[k], n = host_mol_ptr[k + 1] - a;
    uint64_t t;
    const int r = qmlr_serve_submit(S, host_coords + 3 * (size_t)a, host_elem + a, n, &t);
    if (r == QMLR_EBUSY) {
      ++rej;
      continue;
    }
    if (r != QMLR_OK) {
      if (first_err == QMLR_OK) first_err = r;
      break;
    }
    {
      std::lock_guard<std::mutex> lk(qm);
      pending.emplace_back(t, n);
    }
    qcv.notify_one();
  }
  {
    std::lock_guard<std::mutex> lk(qm);
    done_submitting = true;
  }
  qcv.notify_one();
  collector.join();
  if (rejected) *rejected = rej;
  rc = qmlr_serve_stats(S, out);
  if (rc) return rc;
  if (first_err) {
    set_error("replay failed with status %d", first_err);
    return first_err;
  }
  return QMLR_OK;
}
