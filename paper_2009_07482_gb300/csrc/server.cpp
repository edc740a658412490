// server.cpp -- continuous-batching serving loop over the DAG executor.
//
// A model is an inference DAG at a fixed batch size: its weights are RESIDENT
// inputs (uploaded once per slot and kept), its activations are streamed
// inputs, its sinks are read back.  A slot is one planned instance of a model
// (a dag_handle with its own buffers and stream).  Requests wait in arrival
// order; dag_server_progress admits a request as soon as its model has an
// idle slot, or a new slot fits in the free device memory (cudaMemGetInfo,
// less a reserve) and under the slot limit.  An admitted request is
// launched at once: its activations go up on the copy engines and its
// persistent executor launch is queued on the slot's stream, so requests that
// arrive while others run start as SMs free up and overlap them on the device
// (no batch boundary to wait for).  Completion = the slot's readback is done.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <list>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dag_internal.h"
#include "dagexec.h"

namespace {

using Clock = std::chrono::steady_clock;

double now_s() {
  return std::chrono::duration<double>(Clock::now().time_since_epoch()).count();
}

struct Model {
  std::vector<dag_node_desc> nodes;
  std::vector<dag_buffer_desc> bufs;
  std::vector<const void *> weights;  // per buffer: host data of resident inputs
  std::vector<int> streamed, outputs;
  std::vector<const void *> def_in;   // default request inputs (simulation)
  std::vector<void *> def_out;
  size_t footprint = 0;               // bytes of one slot's buffers
  dag_options opt{};
  std::vector<float> costs;
};

struct Request {
  uint64_t ticket = 0;
  int model = 0;
  std::vector<const void *> in;
  std::vector<void *> out;
  double t_arrive = 0, t_launch = 0, t_done = 0;
  dag_status status = DAG_OK;
  bool done = false;
};

struct Slot {
  dag_handle *h = nullptr;
  cudaStream_t st = nullptr;
  int model = 0;
  Request *req = nullptr;
  double last_used = 0;
};

size_t esz(int dt) { return dt == DAG_BF16 ? 2 : 4; }

}  // namespace

struct dag_server {
  std::vector<Model> models;
  std::list<Slot> slots;  // stable addresses: requests point at their slot's handle
  std::deque<Request *> pending;
  std::unordered_map<uint64_t, Request *> reqs;
  std::mutex mu;
  uint64_t next_ticket = 1;
  int max_slots = 0;
  size_t reserve = 0;
  int max_in_flight = 0, in_flight = 0;
};

static dag_status make_slot(dag_server *s, int m, Slot *out) {
  Model &M = s->models[m];
  Slot sl;
  sl.model = m;
  dag_options o = M.opt;
  if (!M.costs.empty()) {
    o.node_cost_us = M.costs.data();
    o.scheduler = DAG_SCHED_RANK_GIVEN;
  }
  dag_status st = dag_create(M.nodes.data(), (int)M.nodes.size(), nullptr, 0, M.bufs.data(), (int)M.bufs.size(), &o,
                             &sl.h);
  if (st) return st;
  for (size_t b = 0; b < M.bufs.size(); ++b)
    if (M.weights[b] && (st = dag_set_input(sl.h, (int)b, M.weights[b]))) {
      dag_destroy(sl.h);
      return st;
    }
  if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess) {
    dag_destroy(sl.h);
    return dagx::report_error(DAG_EDEVICE, "server: stream");
  }
  *out = sl;
  return DAG_OK;
}

extern "C" dag_status dag_server_create(const dag_model_desc *models, int n_models, int max_slots,
                                        size_t hbm_reserve_bytes, const dag_options *opts, dag_server **out) {
  if (!out || n_models < 1 || !models || max_slots < 1)
    return dagx::report_error(DAG_EINVAL, "dag_server_create: arguments");
  dag_server *s = new dag_server();
  s->max_slots = max_slots;
  s->reserve = hbm_reserve_bytes;
  for (int m = 0; m < n_models; ++m) {
    const dag_model_desc &d = models[m];
    Model M;
    M.nodes.assign(d.nodes, d.nodes + d.n_nodes);
    M.bufs.assign(d.buffers, d.buffers + d.n_buffers);
    M.weights.assign(d.n_buffers, nullptr);
    if (opts) M.opt = *opts;
    if (d.node_cost_us) M.costs.assign(d.node_cost_us, d.node_cost_us + d.n_nodes);
    for (int b = 0; b < d.n_buffers; ++b) {
      const dag_buffer_desc &bd = d.buffers[b];
      if (bd.view_of < 0) M.footprint += (size_t)bd.rows * ((bd.cols + 15) / 16 * 16) * esz(bd.dtype);
      if ((bd.flags & DAG_BUF_INPUT) && (bd.flags & DAG_BUF_RESIDENT)) {
        if (!d.weights || !d.weights[b]) {
          delete s;
          return dagx::report_error(DAG_EINVAL, "dag_server_create: a resident input has no host data");
        }
        M.weights[b] = d.weights[b];
      } else if (bd.flags & DAG_BUF_INPUT) {
        M.streamed.push_back(b);
      }
      if (bd.flags & DAG_BUF_OUTPUT) M.outputs.push_back(b);
    }
    M.def_in.assign(M.streamed.size(), nullptr);
    M.def_out.assign(M.outputs.size(), nullptr);
    s->models.push_back(std::move(M));
  }
  *out = s;
  return DAG_OK;
}

extern "C" dag_status dag_server_set_io(dag_server *s, int model, const void *const *inputs, void *const *outputs) {
  if (!s || model < 0 || model >= (int)s->models.size()) return dagx::report_error(DAG_EINVAL, "bad model");
  Model &M = s->models[model];
  for (size_t i = 0; i < M.streamed.size(); ++i) M.def_in[i] = inputs ? inputs[i] : nullptr;
  for (size_t i = 0; i < M.outputs.size(); ++i) M.def_out[i] = outputs ? outputs[i] : nullptr;
  return DAG_OK;
}

extern "C" dag_status dag_server_warm(dag_server *s, int model, int n_slots) {
  if (!s || model < 0 || model >= (int)s->models.size()) return dagx::report_error(DAG_EINVAL, "bad model");
  std::lock_guard<std::mutex> lock(s->mu);
  for (int i = 0; i < n_slots && (int)s->slots.size() < s->max_slots; ++i) {
    Slot sl;
    dag_status st = make_slot(s, model, &sl);
    if (st) return st;
    s->slots.push_back(sl);
  }
  return DAG_OK;
}

extern "C" dag_status dag_server_submit(dag_server *s, int model, const void *const *inputs, void *const *outputs,
                                        uint64_t *ticket) {
  if (!s || model < 0 || model >= (int)s->models.size()) return dagx::report_error(DAG_EINVAL, "bad model");
  Request *r = new Request();
  r->model = model;
  const Model &M = s->models[model];
  r->in.assign(M.streamed.size(), nullptr);
  r->out.assign(M.outputs.size(), nullptr);
  for (size_t i = 0; i < M.streamed.size(); ++i) r->in[i] = inputs ? inputs[i] : M.def_in[i];
  for (size_t i = 0; i < M.outputs.size(); ++i) r->out[i] = outputs ? outputs[i] : M.def_out[i];
  r->t_arrive = now_s();
  std::lock_guard<std::mutex> lock(s->mu);
  r->ticket = s->next_ticket++;
  s->pending.push_back(r);
  s->reqs[r->ticket] = r;
  if (ticket) *ticket = r->ticket;
  return DAG_OK;
}

static int progress_locked(dag_server *s) {
  int completed = 0;
  // 1. completions
  for (auto &sl : s->slots) {
    if (!sl.req) continue;
    const dag_status st = dag_poll(sl.h);
    if (st == DAG_EBUSY) continue;
    sl.req->status = st;
    sl.req->t_done = now_s();
    sl.req->done = true;
    sl.req = nullptr;
    s->in_flight--;
    ++completed;
  }
  // 2. admission, in arrival order: a request takes an idle slot of its model,
  //    or a new slot if device memory and the slot limit allow; when they do
  //    not, the least recently used idle slot of another model is released
  //    first, so every model keeps making progress
  // one device-memory query per pass, updated as slots come and go; idle
  // slots indexed by model
  size_t free_mem = 0, total_mem = 0;
  bool mem_known = false;
  auto fits = [&](int m) {
    if (!mem_known) {
      cudaMemGetInfo(&free_mem, &total_mem);
      mem_known = true;
    }
    return (int)s->slots.size() < s->max_slots && free_mem > s->reserve + s->models[m].footprint + (64u << 20);
  };
  std::vector<std::vector<Slot *>> idle(s->models.size());
  for (auto &sl : s->slots)
    if (!sl.req && sl.h) idle[sl.model].push_back(&sl);
  bool blocked_new = false;  // a slot could not be made this pass: do not retry for later requests
  for (auto it = s->pending.begin(); it != s->pending.end();) {
    Request *r = *it;
    Slot *free_slot = nullptr;
    if (!idle[r->model].empty()) {
      free_slot = idle[r->model].back();
      idle[r->model].pop_back();
    } else if (!blocked_new) {
      // evict only when evicting every idle slot of the other models would
      // make room: otherwise warm slots would be torn down for nothing
      if (!fits(r->model)) {
        size_t freeable = 0;
        int evictable = 0;
        for (auto &sl : s->slots)
          if (!sl.req && sl.model != r->model) {
            freeable += s->models[sl.model].footprint;
            ++evictable;
          }
        const bool room = (int)s->slots.size() - evictable < s->max_slots &&
                          free_mem + freeable > s->reserve + s->models[r->model].footprint + (64u << 20);
        if (!room) {
          blocked_new = true;
          ++it;
          continue;
        }
      }
      while (!fits(r->model)) {
        auto victim = s->slots.end();
        for (auto sit = s->slots.begin(); sit != s->slots.end(); ++sit)
          if (!sit->req && sit->model != r->model && (victim == s->slots.end() || sit->last_used < victim->last_used))
            victim = sit;
        if (victim == s->slots.end()) break;
        auto &vl = idle[victim->model];
        vl.erase(std::remove(vl.begin(), vl.end(), &*victim), vl.end());
        dag_destroy(victim->h);
        cudaStreamDestroy(victim->st);
        s->slots.erase(victim);
        mem_known = false;
      }
      if (fits(r->model)) {
        Slot sl;
        if (make_slot(s, r->model, &sl) == DAG_OK) {
          s->slots.push_back(sl);
          free_slot = &s->slots.back();
          mem_known = false;
        }
      }
      if (!free_slot) blocked_new = true;
    }
    if (!free_slot) { ++it; continue; }
    free_slot->last_used = now_s();
    // 3. launch
    const Model &M = s->models[r->model];
    dag_status st = DAG_OK;
    for (size_t i = 0; i < M.streamed.size() && !st; ++i) st = dag_set_input(free_slot->h, M.streamed[i], r->in[i]);
    for (size_t i = 0; i < M.outputs.size() && !st; ++i) st = dag_set_output(free_slot->h, M.outputs[i], r->out[i]);
    if (!st) st = dag_submit(free_slot->h, free_slot->st);
    r->t_launch = now_s();
    if (st) {
      r->status = st;
      r->done = true;
      r->t_done = r->t_launch;
      ++completed;
    } else {
      free_slot->req = r;
      s->in_flight++;
      s->max_in_flight = std::max(s->max_in_flight, s->in_flight);
    }
    it = s->pending.erase(it);
  }
  return completed;
}

extern "C" int dag_server_progress(dag_server *s) {
  if (!s) return -1;
  std::lock_guard<std::mutex> lock(s->mu);
  return progress_locked(s);
}

extern "C" dag_status dag_server_wait(dag_server *s, uint64_t ticket, uint64_t timeout_ns, dag_request_info *info) {
  if (!s) return dagx::report_error(DAG_EINVAL, "null server");
  const double t_end = now_s() + (timeout_ns ? timeout_ns * 1e-9 : 1e30);
  for (;;) {
    {
      std::lock_guard<std::mutex> lock(s->mu);
      auto it = s->reqs.find(ticket);
      if (it == s->reqs.end()) return dagx::report_error(DAG_EINVAL, "unknown ticket");
      progress_locked(s);
      Request *r = it->second;
      if (r->done) {
        if (info) *info = dag_request_info{r->model, r->status, r->t_arrive, r->t_launch, r->t_done};
        const dag_status st = r->status;
        s->reqs.erase(it);
        delete r;
        return st;
      }
    }
    if (now_s() > t_end) return dagx::report_error(DAG_ETIMEOUT, "dag_server_wait timed out");
    std::this_thread::yield();
  }
}

extern "C" dag_status dag_server_simulate(dag_server *s, const int32_t *model_seq, int n, double rate_hz,
                                          uint64_t seed, double *latency_us, double *wall_s, int *max_in_flight) {
  if (!s || !model_seq || n < 1 || rate_hz <= 0) return dagx::report_error(DAG_EINVAL, "dag_server_simulate: arguments");
  // Poisson arrivals: exponential gaps -ln(u)/rate, u in (0,1] from SplitMix64
  std::vector<double> arrive(n);
  double t = 0;
  for (int i = 0; i < n; ++i) {
    uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double u = ((double)(z >> 11) + 1.0) * 0x1p-53;
    t += -std::log(u) / rate_hz;
    arrive[i] = t;
  }
  std::vector<uint64_t> tickets(n, 0);
  s->max_in_flight = 0;
  const double t0 = now_s();
  int next = 0, done = 0;
  std::vector<char> got(n, 0);
  while (done < n) {
    const double el = now_s() - t0;
    while (next < n && arrive[next] <= el) {
      dag_status st = dag_server_submit(s, model_seq[next], nullptr, nullptr, &tickets[next]);
      if (st) return st;
      std::lock_guard<std::mutex> lock(s->mu);
      s->reqs[tickets[next]]->t_arrive = t0 + arrive[next];  // latency counts from the scheduled arrival
      ++next;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    progress_locked(s);
    for (int i = 0; i < next; ++i) {
      if (got[i]) continue;
      auto it = s->reqs.find(tickets[i]);
      if (it == s->reqs.end() || !it->second->done) continue;
      Request *r = it->second;
      if (r->status) return dagx::report_error(r->status, "dag_server_simulate: a request failed");
      if (latency_us) latency_us[i] = (r->t_done - r->t_arrive) * 1e6;
      s->reqs.erase(it);
      delete r;
      got[i] = 1;
      ++done;
    }
  }
  if (wall_s) *wall_s = now_s() - t0;
  if (max_in_flight) *max_in_flight = s->max_in_flight;
  return DAG_OK;
}

extern "C" int dag_server_slots(dag_server *s) {
  if (!s) return 0;
  std::lock_guard<std::mutex> lock(s->mu);
  return (int)s->slots.size();
}

extern "C" dag_status dag_server_destroy(dag_server *s) {
  if (!s) return DAG_OK;
  for (auto &sl : s->slots) {
    if (sl.h) dag_destroy(sl.h);
    if (sl.st) cudaStreamDestroy(sl.st);
  }
  for (auto *r : s->pending) delete r;
  for (auto &kv : s->reqs) {
    bool queued = std::find(s->pending.begin(), s->pending.end(), kv.second) != s->pending.end();
    if (!queued) delete kv.second;
  }
  delete s;
  return DAG_OK;
}
