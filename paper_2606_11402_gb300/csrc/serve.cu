// Serving engine: continuous batching of generate / whiten / logdet / NLL-
// gradient requests over resident GraphGP instances (graph + factor).
//
// A native scheduler thread owns a set of stream slots.  Requests are queued
// by graphgp_server_submit with their arrival time; the scheduler admits them
// in arrival order while a slot is free and the device bytes of the requests
// in flight stay within the HBM budget (one request per instance at a time,
// since an instance's work vectors and level barrier are shared).  An admitted
// request runs on its slot's stream: host-to-device copy of its input, the
// operation, device-to-host copy of its results, then an event.  Requests on
// different slots overlap on the device.  The first request of each
// (instance, operation, slot) is captured into a CUDA graph, which later
// requests replay; if capture is refused the operation runs as plain
// launches.  Completion is detected by polling the events; arrival, admission
// and completion times are kept per request (host monotonic clock).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>

#include "common.cuh"

namespace ggp {
int run_generate(graphgp_graph_t g, graphgp_factor_t f, const float* xi, float* v, cudaStream_t s);
int run_whiten(graphgp_graph_t g, graphgp_factor_t f, const float* v, float* xi, double* sq,
               cudaStream_t s);
}  // namespace ggp

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Req {
  uint64_t id = 0;
  int inst = -1;
  int op = 0;
  const float* in_h = nullptr;
  float* out_h = nullptr;
  double* scal_h = nullptr;   // [4]: op-dependent scalars
  double t_arrival = 0, t_admit = 0, t_done = 0;
  int status = 1;             // 1 queued, 2 running, 0 done, <0 error
  int slot = -1;
  size_t footprint = 0;
};

struct Slot {
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  float* in_d = nullptr;
  float* out_d = nullptr;
  double* scal_d = nullptr;   // [4]
  float* out_h = nullptr;     // pinned staging for results
  double* scal_h = nullptr;   // pinned [4]
  size_t cap = 0;             // floats
  Req* req = nullptr;
  std::map<std::pair<int, int>, cudaGraphExec_t> graphs;
  std::map<std::pair<int, int>, bool> no_graph;
};

struct Inst {
  graphgp_graph_t g;
  graphgp_factor_t f;
  int64_t N;
  bool busy = false;
};

}  // namespace

struct graphgp_server_s {
  std::vector<Inst> inst;
  std::vector<Slot> slots;
  std::deque<Req*> queue;
  std::unordered_map<uint64_t, Req*> reqs;
  std::mutex mu;
  std::condition_variable cv, done_cv;
  std::thread worker;
  bool stop = false;
  bool started = false;
  bool use_graphs = true;
  size_t budget = 0, in_use = 0;
  uint64_t next_id = 1;
  int64_t completed = 0, errors = 0;
  int device = 0;
};

namespace {

// Device bytes a request needs beyond the resident instance: its input and
// output vectors, and for gradients the instance's work vectors.
size_t footprint(const Inst& in, int op) {
  size_t n = (size_t)in.N * sizeof(float);
  switch (op) {
    case GRAPHGP_OP_GENERATE:
    case GRAPHGP_OP_WHITEN: return 2 * n;
    case GRAPHGP_OP_LOGDET: return 64;
    default: return 4 * n;
  }
}

// Enqueues one request's work on the slot's stream (captured or not).
int enqueue_op(const Inst& in, int op, Slot& sl) {
  cudaStream_t s = sl.s;
  switch (op) {
    case GRAPHGP_OP_GENERATE:
      return ggp::run_generate(in.g, in.f, sl.in_d, sl.out_d, s);
    case GRAPHGP_OP_WHITEN:
      return ggp::run_whiten(in.g, in.f, sl.in_d, sl.out_d, nullptr, s);
    case GRAPHGP_OP_LOGDET:
      return graphgp_logdet(in.f, sl.scal_d, s);
    case GRAPHGP_OP_NLL_GRAD: {
      GGP_CUDA(cudaMemsetAsync(sl.scal_d, 0, 4 * sizeof(double), s));
      GGP_TRY(graphgp_nll(in.g, in.f, sl.in_d, sl.scal_d, s));
      GGP_TRY(graphgp_nll_backward(in.g, in.f, sl.in_d, 1.0, sl.out_d, sl.scal_d + 1, s));
      return GRAPHGP_OK;
    }
  }
  return GRAPHGP_ERR_INVALID;
}

size_t in_floats(const Inst& in, int op) { return op == GRAPHGP_OP_LOGDET ? 0 : (size_t)in.N; }
size_t out_floats(const Inst& in, int op) { return op == GRAPHGP_OP_LOGDET ? 0 : (size_t)in.N; }

// Starts a request on a free slot.  Called with the lock held.
int launch(graphgp_server_s* sv, Req* r, int slot_id) {
  Slot& sl = sv->slots[slot_id];
  Inst& in = sv->inst[r->inst];
  cudaStream_t s = sl.s;
  size_t nin = in_floats(in, r->op), nout = out_floats(in, r->op);
  if (nin) GGP_CUDA(cudaMemcpyAsync(sl.in_d, r->in_h, nin * 4, cudaMemcpyHostToDevice, s));
  auto key = std::make_pair(r->inst, r->op);
  bool graphs = sv->use_graphs && !sl.no_graph.count(key);
  if (graphs) {
    auto it = sl.graphs.find(key);
    if (it == sl.graphs.end()) {
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      bool ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      int rc = ok ? enqueue_op(in, r->op, sl) : GRAPHGP_ERR_CUDA;
      cudaError_t e = cudaStreamEndCapture(s, &graph);
      ok = ok && rc == GRAPHGP_OK && e == cudaSuccess && graph &&
           cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      if (ok) {
        sl.graphs[key] = exec;
        it = sl.graphs.find(key);
      } else {
        sl.no_graph[key] = true;
        graphs = false;
      }
    }
    if (graphs) GGP_CUDA(cudaGraphLaunch(it->second, s));
  }
  if (!graphs) GGP_TRY(enqueue_op(in, r->op, sl));
  if (nout) {
    float* dst = r->out_h ? r->out_h : sl.out_h;
    GGP_CUDA(cudaMemcpyAsync(dst, sl.out_d, nout * 4, cudaMemcpyDeviceToHost, s));
  }
  if (r->op == GRAPHGP_OP_LOGDET || r->op == GRAPHGP_OP_NLL_GRAD) {
    double* dst = r->scal_h ? r->scal_h : sl.scal_h;
    GGP_CUDA(cudaMemcpyAsync(dst, sl.scal_d, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  GGP_CUDA(cudaEventRecord(sl.ev, s));
  return GRAPHGP_OK;
}

void worker_loop(graphgp_server_s* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    bool progress = false;
    // completions
    for (size_t i = 0; i < sv->slots.size(); i++) {
      Slot& sl = sv->slots[i];
      if (!sl.req) continue;
      cudaError_t e = cudaEventQuery(sl.ev);
      if (e == cudaErrorNotReady) continue;
      Req* r = sl.req;
      r->t_done = now_s();
      r->status = (e == cudaSuccess) ? GRAPHGP_OK : GRAPHGP_ERR_CUDA;
      if (e != cudaSuccess) {
        cudaGetLastError();
        sv->errors++;
      }
      sv->inst[r->inst].busy = false;
      sv->in_use -= r->footprint;
      sv->completed++;
      sl.req = nullptr;
      progress = true;
    }
    if (progress) sv->done_cv.notify_all();
    if (sv->stop && sv->queue.empty()) {
      bool idle = true;
      for (auto& sl : sv->slots) idle = idle && !sl.req;
      if (idle) break;
    }
    // admissions, in arrival order; a request whose instance is busy waits
    // without blocking later ones
    for (auto it = sv->queue.begin(); it != sv->queue.end();) {
      int free_slot = -1;
      for (size_t i = 0; i < sv->slots.size(); i++)
        if (!sv->slots[i].req) {
          free_slot = (int)i;
          break;
        }
      if (free_slot < 0) break;
      Req* r = *it;
      Inst& in = sv->inst[r->inst];
      if (in.busy || (sv->in_use + r->footprint > sv->budget && sv->in_use > 0)) {
        ++it;
        continue;
      }
      in.busy = true;
      sv->in_use += r->footprint;
      r->slot = free_slot;
      r->status = 2;
      r->t_admit = now_s();
      sv->slots[free_slot].req = r;
      int rc = launch(sv, r, free_slot);
      if (rc < 0) {
        r->status = rc;
        r->t_done = now_s();
        in.busy = false;
        sv->in_use -= r->footprint;
        sv->slots[free_slot].req = nullptr;
        sv->errors++;
        sv->completed++;
        sv->done_cv.notify_all();
      }
      it = sv->queue.erase(it);
      progress = true;
    }
    if (!progress) {
      bool any_busy = false;
      for (auto& sl : sv->slots) any_busy = any_busy || sl.req;
      if (any_busy)
        sv->cv.wait_for(lk, std::chrono::microseconds(20));
      else
        sv->cv.wait_for(lk, std::chrono::milliseconds(2));
    }
  }
}

}  // namespace

using namespace ggp;

extern "C" int graphgp_server_create(int n_slots, size_t hbm_budget, int use_graphs,
                                     graphgp_server_t* out) {
  if (!out || n_slots < 1 || n_slots > 64) return GRAPHGP_ERR_INVALID;
  *out = nullptr;
  auto* sv = new (std::nothrow) graphgp_server_s();
  if (!sv) return GRAPHGP_ERR_OOM;
  sv->budget = hbm_budget ? hbm_budget : (size_t)8 << 30;
  sv->use_graphs = use_graphs != 0;
  sv->slots.resize(n_slots);
  cudaGetDevice(&sv->device);
  *out = sv;
  return GRAPHGP_OK;
}

extern "C" int graphgp_server_register(graphgp_server_t sv, graphgp_graph_t g, graphgp_factor_t f,
                                       int* instance_id) {
  if (!sv || !g || !f || f->g != g || f->row_end >= 0 || !instance_id) return GRAPHGP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->started) return GRAPHGP_ERR_INVALID;
  GGP_CUDA(cudaDeviceSynchronize());
  sv->inst.push_back(Inst{g, f, g->N, false});
  *instance_id = (int)sv->inst.size() - 1;
  return GRAPHGP_OK;
}

extern "C" int graphgp_server_start(graphgp_server_t sv) {
  if (!sv) return GRAPHGP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->started) return GRAPHGP_ERR_INVALID;
  size_t cap = 1;
  for (auto& in : sv->inst) cap = std::max(cap, (size_t)in.N);
  for (auto& sl : sv->slots) {
    GGP_CUDA(cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking));
    GGP_CUDA(cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming));
    GGP_CUDA(cudaMalloc(&sl.in_d, cap * 4));
    GGP_CUDA(cudaMalloc(&sl.out_d, cap * 4));
    GGP_CUDA(cudaMalloc(&sl.scal_d, 4 * sizeof(double)));
    GGP_CUDA(cudaMallocHost(&sl.out_h, cap * 4));
    GGP_CUDA(cudaMallocHost(&sl.scal_h, 4 * sizeof(double)));
    sl.cap = cap;
  }
  sv->started = true;
  sv->worker = std::thread(worker_loop, sv);
  return GRAPHGP_OK;
}

extern "C" int graphgp_server_submit(graphgp_server_t sv, int instance_id, int op,
                                     const float* in_h, float* out_h, double* scal_h,
                                     double arrival_s, uint64_t* ticket) {
  if (!sv || !ticket || op < GRAPHGP_OP_GENERATE || op > GRAPHGP_OP_NLL_GRAD)
    return GRAPHGP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (!sv->started || sv->stop || instance_id < 0 || instance_id >= (int)sv->inst.size())
    return GRAPHGP_ERR_INVALID;
  if (op != GRAPHGP_OP_LOGDET && !in_h) return GRAPHGP_ERR_INVALID;
  Req* r = new (std::nothrow) Req();
  if (!r) return GRAPHGP_ERR_OOM;
  r->id = sv->next_id++;
  r->inst = instance_id;
  r->op = op;
  r->in_h = in_h;
  r->out_h = out_h;
  r->scal_h = scal_h;
  r->t_arrival = arrival_s > 0 ? arrival_s : now_s();
  r->footprint = footprint(sv->inst[instance_id], op);
  sv->reqs[r->id] = r;
  sv->queue.push_back(r);
  *ticket = r->id;
  sv->cv.notify_one();
  return GRAPHGP_OK;
}

extern "C" int graphgp_server_wait(graphgp_server_t sv, uint64_t ticket, double timeout_s,
                                   double* times_out) {
  if (!sv) return GRAPHGP_ERR_INVALID;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return GRAPHGP_ERR_INVALID;
  Req* r = it->second;
  auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  while (r->status > 0) {
    if (sv->done_cv.wait_until(lk, deadline) == std::cv_status::timeout && r->status > 0)
      return GRAPHGP_ERR_TIMEOUT;
  }
  if (times_out) {
    times_out[0] = r->t_arrival;
    times_out[1] = r->t_admit;
    times_out[2] = r->t_done;
  }
  return r->status;
}

extern "C" int graphgp_server_stats(graphgp_server_t sv, int64_t* completed, int64_t* errors,
                                    int64_t* queued, size_t* bytes_in_flight) {
  if (!sv) return GRAPHGP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (completed) *completed = sv->completed;
  if (errors) *errors = sv->errors;
  if (queued) *queued = (int64_t)sv->queue.size();
  if (bytes_in_flight) *bytes_in_flight = sv->in_use;
  return GRAPHGP_OK;
}

extern "C" void graphgp_server_destroy(graphgp_server_t sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    sv->cv.notify_all();
  }
  if (sv->worker.joinable()) sv->worker.join();
  for (auto& sl : sv->slots) {
    for (auto& kv : sl.graphs) cudaGraphExecDestroy(kv.second);
    if (sl.s) cudaStreamSynchronize(sl.s);
    if (sl.in_d) cudaFree(sl.in_d);
    if (sl.out_d) cudaFree(sl.out_d);
    if (sl.scal_d) cudaFree(sl.scal_d);
    if (sl.out_h) cudaFreeHost(sl.out_h);
    if (sl.scal_h) cudaFreeHost(sl.scal_h);
    if (sl.ev) cudaEventDestroy(sl.ev);
    if (sl.s) cudaStreamDestroy(sl.s);
  }
  for (auto& kv : sv->reqs) delete kv.second;
  delete sv;
}
