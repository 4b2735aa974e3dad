// Continuous-batching request engine: lanes of (context, server set) that
// evaluate up to four requests together by a carousel over the set's layers
// (contract in include/pepsi.h, pepsi_engine_*).
//
// A lane step takes the next chunk [pos, pos + L) of the set's layers.  The
// multiply-accumulate of the chunk runs for the lane's requests in launches
// of up to the schedule's batch_requests (one read of the chunk's
// plaintexts per launch), then each request's equality
// circuits (Algorithm 1) and its share of the layer sum (Algorithm 2) run on
// the lane's stream.  A request that joins at layer p sees layers p .. mu-1,
// then 0 .. p-1: its layer sum is the same sum in another order, which is
// the same result as long as the layers are rounded one by one or all
// together (the only rounding runs a lane accepts).  Its final step also
// runs the output stage (relinearisation, (h!)^-1, mask, response switch).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "context.h"

using namespace pepsi_detail;

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kMaxSlots = PEPSI_MAC_MAX_REQUESTS;
constexpr size_t kStepsAhead = 2;  // lane steps queued ahead of the GPU

struct Request {
  int lane = 0;
  const u64* cts = nullptr;
  int mode = 0;
  u64 mask_seed = 0;
  u64* out = nullptr;
  Clock::time_point t_submit, t_done;
  int status = -1;  // -1 while pending, then a PEPSI_* code
};

// Device state of one admitted request, from the engine's memory pool.
struct Slot {
  bool busy = false;
  u64 ticket = 0;
  int mode = 0;
  u64 mask_seed = 0;
  u64* out = nullptr;
  u64* C = nullptr;    // [ell][2][k][N] request, NTT form, split operand format
  u64* H = nullptr;    // [Lc][2][k][N] h' of the current chunk
  u64* acc = nullptr;  // [3][k][N] layer sum
  u64* X = nullptr;    // [3][k+kb][N] run sum of the exact products (lazy rescaling)
  size_t bytes = 0;
  u32 done = 0;        // layers seen
  LazyRun lr{};
};

// A queued step: its completion event, the lane's device error word as the
// step left it (copied to pinned host memory by the step itself), and what
// completes with it.
struct Step {
  cudaEvent_t ev = nullptr;
  int* err = nullptr;          // pinned word of the lane's ring
  std::vector<u64> finishing;  // tickets whose output stage ran in this step
  size_t released = 0;         // bytes of state given back with them
};

struct Lane {
  pepsi_ctx* c = nullptr;  // the lane's own context (shares the parent's tables)
  int set = 0;             // internal server set (one block)
  u32 mu = 0, mu_res = 0, pos = 0;
  int nslots = 1, Lc = 1;
  EvalBufs b{};
  Slot slot[kMaxSlots];
  std::deque<u64> queue;   // tickets waiting for a slot
  std::deque<Step> inflight;
  std::vector<cudaEvent_t> spare;
  int* err_ring = nullptr;  // pinned host words, one per queued step
  u64 nsteps = 0;
  int fail_next = 0;        // test hook: the next admission reports this status instead of running
};

}  // namespace

struct pepsi_engine {
  std::vector<Lane> lanes;
  cudaMemPool_t pool = nullptr;
  size_t budget = 0, used = 0, peak = 0;
  uint64_t steps = 0, submitted = 0, completed = 0;
  std::mutex mu;               // guards reqs, incoming and the counters read by other threads
  std::condition_variable cv;  // signalled on submissions and completions
  std::unordered_map<u64, Request> reqs;
  std::deque<u64> incoming;
  u64 next_ticket = 1;
  std::thread th;
  bool thread_on = false, stop = false;
  std::mutex pump_mu;          // one pump at a time
};

// A captured engine schedule (pepsi_engine_capture).
struct pepsi_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t own = nullptr;  // capture and launch stream when the caller gives none
  cudaStream_t last = nullptr; // stream of the last launch
  int* err = nullptr;          // pinned: each lane's error word after the last launch
  int nlanes = 0;
  int device = -1;             // the lanes' device (its graph memory pool)
};

namespace {

// Bytes of a request's device state on a lane (lazy: with its run sum).
size_t request_bytes(const Lane& L, bool lazy) {
  const pepsi_ctx* c = L.c;
  const size_t kN = (size_t)c->k * c->N;
  size_t w = request_prepared_words(c->ell, kN) + (size_t)L.Lc * 2 * kN + 3 * kN;
  if (lazy) w += (size_t)3 * (c->k + c->kb) * c->N;
  return w * 8;
}

cudaError_t pool_alloc(pepsi_engine* e, u64** p, size_t words, cudaStream_t st) {
  return cudaMallocFromPoolAsync((void**)p, words * 8, e->pool, st);
}

// Admit the head of the lane's queue into slot s (the engine lock is not
// held: only the pumping thread touches lanes).
int admit(pepsi_engine* e, Lane& L, int s, u64 ticket, const Request& r, size_t bytes) {
  if (L.fail_next) {  // an injected failure, made on the host
    const int rc = L.fail_next;
    L.fail_next = 0;
    return rc;
  }
  pepsi_ctx* c = L.c;
  cudaStream_t st = c->stream;
  const size_t kN = (size_t)c->k * c->N;
  Slot& S = L.slot[s];
  S = Slot{};
  S.ticket = ticket;
  S.mode = r.mode;
  S.mask_seed = r.mask_seed;
  S.out = r.out;
  S.bytes = bytes;
  const u32 G = rescale_run(c, L.mu, r.mode);
  cudaError_t err = pool_alloc(e, &S.C, request_prepared_words(c->ell, kN), st);
  if (err == cudaSuccess) err = pool_alloc(e, &S.H, (size_t)L.Lc * 2 * kN, st);
  if (err == cudaSuccess) err = pool_alloc(e, &S.acc, 3 * kN, st);
  if (err == cudaSuccess && G > 1) err = pool_alloc(e, &S.X, (size_t)3 * (c->k + c->kb) * c->N, st);
  if (err == cudaSuccess) err = prepare_request(c, r.cts, S.C, st);
  if (err != cudaSuccess) return cuda_status(err);
  if (G > 1) {
    S.lr.X = S.X;
    S.lr.acc = S.acc;
    S.lr.G = G;
  }
  S.busy = true;
  return PEPSI_OK;
}

void release(Slot& S, cudaStream_t st) {
  for (u64* p : {S.C, S.H, S.acc, S.X})
    if (p) cudaFreeAsync(p, st);
  S.C = S.H = S.acc = S.X = nullptr;
  S.busy = false;
}

// Queue one step of the lane: the multiply-accumulate of the next chunk for
// every busy slot, then each slot's circuits and layer sum; a slot that has
// seen all layers also runs the output stage and is released.
int enqueue_step(Lane& L, Step& step, bool capturing = false) {
  pepsi_ctx* c = L.c;
  cudaStream_t st = c->stream;
  ServerSet& S = c->sets[L.set];
  const size_t kN = (size_t)c->k * c->N, vstride = (size_t)(c->k + c->kb) * c->N;
  u32 n = std::min<u32>((u32)L.Lc, L.mu - L.pos);
  if (L.pos < L.mu_res) n = std::min<u32>(n, L.mu_res - L.pos);
  const int nl = (int)n;
  const u64* Cs[kMaxSlots];
  u64* Hs[kMaxSlots];
  int act[kMaxSlots], na = 0;
  for (int s = 0; s < L.nslots; ++s)
    if (L.slot[s].busy) {
      Cs[na] = L.slot[s].C;
      Hs[na] = L.slot[s].H;
      act[na++] = s;
    }
  if (!na) return PEPSI_OK;
  PlainTab P;
  if (L.pos < L.mu_res) {
    P = S.plain(kN, c->ell, L.pos);
  } else {
    {
      Prof p(c, PC_PTGEN, st);
      launch_ptgen(c->V, S.dpos + (size_t)L.pos * c->N * c->h, nl, c->ell, c->h, L.b.Pc, st);
    }
    P = plain_words(L.b.Pc);
  }
  for (int q0 = 0; q0 < na; q0 += c->batch_requests) {  // launches of at most batch_requests requests
    Prof p(c, PC_MAC, st);
    const int nq = std::min(c->batch_requests, na - q0);
    const cudaError_t me = mac_status(launch_mac_requests(c->V, nq, Cs + q0, P, Hs + q0, c->ell, nl, c->mac_fold,
                                                          c->d_err, st, c->batch_points, c->batch_groups));
    if (me != cudaSuccess) return cuda_status(me);
  }
  for (int i = 0; i < na; ++i) {
    Slot& T = L.slot[act[i]];
    const bool valued = T.mode >= PEPSI_MODE_LABELS;
    const u64* VP = valued ? S.dVP + (size_t)L.pos * vstride : nullptr;
    const bool last = T.done + n == L.mu;
    L.b.H = T.H;
    if (T.lr.G > 1) {
      const LastMult m = eq_circuit_front(c, L.b, nl, st);
      lazy_chunk(c, L.b, m, VP, nl, last, T.lr, st);
    } else {
      eq_circuit(c, L.b, nl, st);
      if (valued) {
        ntt(c, true, L.b.D, L.b.D, (size_t)nl * 3, c->k, 0, kN, kN, st);
        Prof p(c, PC_POINTWISE, st);
        launch_accum_val(c->V, L.b.D, VP, nl, T.acc, T.done == 0, st);
      } else {
        Prof p(c, PC_POINTWISE, st);
        launch_accum(c->V, L.b.D, nl, T.acc, T.done == 0, st);
      }
    }
    T.done += n;
    if (last) {
      const cudaError_t fe = finish_request(c, L.b, T.acc, valued && T.lr.G <= 1, T.mode, T.mask_seed, T.out, st);
      if (fe != cudaSuccess) return cuda_status(fe);
      step.finishing.push_back(T.ticket);
      step.released += T.bytes;
      release(T, st);
    }
  }
  L.pos = (L.pos + n) % L.mu;
  if (capturing) return cuda_status(cudaGetLastError());  // completion is the graph's
  if (L.spare.empty()) {
    cudaEvent_t ev;
    const cudaError_t ce = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (ce != cudaSuccess) return cuda_status(ce);
    L.spare.push_back(ev);
  }
  step.ev = L.spare.back();
  L.spare.pop_back();
  // the error word as this step leaves it, then cleared for the next step
  step.err = L.err_ring + (L.nsteps++ % (kStepsAhead + 1));
  cudaError_t re = cudaMemcpyAsync(step.err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (re == cudaSuccess) re = cudaMemsetAsync(c->d_err, 0, sizeof(int), st);
  if (re == cudaSuccess) re = cudaEventRecord(step.ev, st);
  if (re != cudaSuccess) return cuda_status(re);
  return cuda_status(cudaGetLastError());
}

// Retire the lane's completed steps; returns how many requests completed.
int retire(pepsi_engine* e, Lane& L, bool* progressed) {
  int done = 0;
  while (!L.inflight.empty()) {
    Step& s = L.inflight.front();
    const cudaError_t q = cudaEventQuery(s.ev);
    if (q == cudaErrorNotReady) break;
    int status = PEPSI_OK;
    if (q != cudaSuccess) {
      status = cuda_status(q);
    } else if (*s.err) {  // a bounded wait of this step expired
      status = PEPSI_E_TIMEOUT;
    }
    const Clock::time_point now = Clock::now();
    {
      std::lock_guard<std::mutex> lock(e->mu);
      for (u64 t : s.finishing) {
        Request& r = e->reqs.at(t);
        r.status = status;
        r.t_done = now;
        ++e->completed;
        ++done;
      }
      e->used -= s.released;
    }
    L.spare.push_back(s.ev);
    L.inflight.pop_front();
    *progressed = true;
  }
  return done;
}

// Complete a request with an error status: its slot's state goes back to the
// pool and its bytes to the budget (a failed admission or step; the next
// requests are still served).
void fail_slot(pepsi_engine* e, Lane& L, int s, int status) {
  Slot& S = L.slot[s];
  release(S, L.c->stream);
  std::lock_guard<std::mutex> lock(e->mu);
  Request& r = e->reqs.at(S.ticket);
  r.status = status;
  r.t_done = Clock::now();
  ++e->completed;
  e->used -= S.bytes;
  S = Slot{};
}

int pump_once(pepsi_engine* e, uint64_t* pending) {
  std::lock_guard<std::mutex> pl(e->pump_mu);
  bool progressed = false;
  int completed = 0;
  // route new submissions to their lanes
  std::vector<std::pair<int, u64>> routed;
  {
    std::lock_guard<std::mutex> lock(e->mu);
    while (!e->incoming.empty()) {
      const u64 t = e->incoming.front();
      e->incoming.pop_front();
      routed.push_back({e->reqs.at(t).lane, t});
    }
  }
  for (auto& rt : routed) e->lanes[rt.first].queue.push_back(rt.second);
  int rc = PEPSI_OK;
  for (Lane& L : e->lanes) {
    completed += retire(e, L, &progressed);
    while (L.inflight.size() < kStepsAhead && rc == PEPSI_OK) {
      // admit waiting requests into free slots while the budget holds them
      for (int s = 0; s < L.nslots && !L.queue.empty(); ++s) {
        if (L.slot[s].busy) continue;
        const u64 t = L.queue.front();
        Request r;
        size_t bytes = 0;
        {
          std::lock_guard<std::mutex> lock(e->mu);
          r = e->reqs.at(t);
          bytes = request_bytes(L, rescale_run(L.c, L.mu, r.mode) > 1);
          if (e->used + bytes > e->budget && e->used > 0) break;  // wait for memory to come back
          e->used += bytes;
          e->peak = std::max(e->peak, e->used);
        }
        L.queue.pop_front();
        const int arc = admit(e, L, s, t, r, bytes);
        progressed = true;
        if (arc != PEPSI_OK) {
          if (rc == PEPSI_OK) rc = arc;
          L.slot[s].ticket = t;
          L.slot[s].bytes = bytes;
          fail_slot(e, L, s, arc);
          ++completed;
        }
      }
      bool busy = false;
      for (int s = 0; s < L.nslots; ++s) busy |= L.slot[s].busy;
      if (!busy) break;
      Step step;
      const int src = enqueue_step(L, step);
      {
        std::lock_guard<std::mutex> lock(e->mu);
        ++e->steps;
      }
      if (src != PEPSI_OK) {  // the lane's requests in flight fail with the step
        if (rc == PEPSI_OK) rc = src;
        for (int s = 0; s < L.nslots; ++s)
          if (L.slot[s].busy) {
            fail_slot(e, L, s, src);
            ++completed;
          }
        break;
      }
      L.inflight.push_back(std::move(step));
      progressed = true;
    }
  }
  {
    std::lock_guard<std::mutex> lock(e->mu);
    if (pending) *pending = e->submitted - e->completed;
  }
  if (completed) e->cv.notify_all();
  return rc;
}

void engine_thread(pepsi_engine* e) {
  for (;;) {
    uint64_t pending = 0;
    pump_once(e, &pending);
    std::unique_lock<std::mutex> lock(e->mu);
    if (e->stop && e->submitted == e->completed) return;
    if (pending)  // work in flight: poll again shortly
      e->cv.wait_for(lock, std::chrono::microseconds(20));
    else
      e->cv.wait_for(lock, std::chrono::milliseconds(5), [&] { return e->stop || !e->incoming.empty(); });
  }
}

}  // namespace

extern "C" {

int pepsi_engine_create(const pepsi_lane* lanes, int nlanes, uint64_t hbm_budget, pepsi_engine** out) {
  if (!out || !lanes || nlanes <= 0) return PEPSI_E_PARAM;
  *out = nullptr;
  for (int i = 0; i < nlanes; ++i) {
    pepsi_ctx* p = lanes[i].ctx;
    if (!p || lanes[i].slots < 1 || lanes[i].slots > (uint32_t)kMaxSlots) return PEPSI_E_PARAM;
    if (lanes[i].set_id < 0 || lanes[i].set_id >= (int)p->groups.size() || !p->groups[lanes[i].set_id].live ||
        p->groups[lanes[i].set_id].blk.size() != 1)
      return PEPSI_E_PARAM;
    const u32 mu = p->groups[lanes[i].set_id].mu;
    for (int mode = PEPSI_MODE_INDICATOR; mode <= PEPSI_MODE_SUM; ++mode) {
      const u32 G = rescale_run(p, mu, mode);
      if (G > 1 && G < mu) return PEPSI_E_PARAM;  // runs that depend on where a request starts
    }
  }
  auto* e = new pepsi_engine();
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  if (err == cudaSuccess) err = cudaMemPoolCreate(&e->pool, &props);
  if (err == cudaSuccess) {  // keep freed state in the pool for the next requests
    uint64_t keep = UINT64_MAX;
    err = cudaMemPoolSetAttribute(e->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  int rc = err == cudaSuccess ? PEPSI_OK : cuda_status(err);
  for (int i = 0; i < nlanes && rc == PEPSI_OK; ++i) {
    pepsi_ctx* p = lanes[i].ctx;
    Lane L;
    L.c = ctx_fork(p, &err);
    if (!L.c) {
      rc = cuda_status(err);
      break;
    }
    L.set = p->groups[lanes[i].set_id].blk[0];
    const ServerSet& S = L.c->sets[L.set];
    L.mu = S.mu;
    L.mu_res = S.mu_res;
    L.nslots = (int)lanes[i].slots;
    L.Lc = balanced_chunk(L.c->chunk, L.mu);
    err = eval_bufs(L.c, L.Lc, L.mu_res < L.mu, &L.b);
    if (err == cudaSuccess) err = cudaHostAlloc((void**)&L.err_ring, (kStepsAhead + 1) * sizeof(int), 0);
    if (err == cudaSuccess) memset(L.err_ring, 0, (kStepsAhead + 1) * sizeof(int));
    if (err != cudaSuccess) rc = cuda_status(err);
    e->lanes.push_back(std::move(L));
  }
  if (rc == PEPSI_OK) {
    size_t freeb = 0, totalb = 0;
    cudaMemGetInfo(&freeb, &totalb);
    e->budget = hbm_budget ? (size_t)hbm_budget : freeb / 2;
  }
  if (rc != PEPSI_OK) {
    pepsi_engine_destroy(e);
    return rc;
  }
  *out = e;
  return PEPSI_OK;
}

int pepsi_engine_submit(pepsi_engine* e, int lane, const uint64_t* cts, int mode, uint64_t mask_seed,
                        uint64_t* out_ct, uint64_t* ticket) {
  if (!e || !cts || !out_ct || !ticket || lane < 0 || lane >= (int)e->lanes.size()) return PEPSI_E_PARAM;
  if (mode < PEPSI_MODE_INDICATOR || mode > PEPSI_MODE_SUM) return PEPSI_E_PARAM;
  const Lane& L = e->lanes[lane];
  if (mode >= PEPSI_MODE_LABELS && !L.c->sets[L.set].has_values) return PEPSI_E_PARAM;
  Request r;
  r.lane = lane;
  r.cts = cts;
  r.mode = mode;
  r.mask_seed = mask_seed;
  r.out = out_ct;
  r.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lock(e->mu);
    const u64 t = e->next_ticket++;
    e->reqs.emplace(t, r);
    e->incoming.push_back(t);
    ++e->submitted;
    *ticket = t;
  }
  e->cv.notify_all();
  return PEPSI_OK;
}

int pepsi_engine_pump(pepsi_engine* e, uint64_t* pending) {
  if (!e) return PEPSI_E_PARAM;
  return pump_once(e, pending);
}

int pepsi_engine_run(pepsi_engine* e) {
  if (!e) return PEPSI_E_PARAM;
  int first = PEPSI_OK;  // the first failed request's status
  for (;;) {
    uint64_t pending = 0;
    const int rc = pump_once(e, &pending);
    if (first == PEPSI_OK) first = rc;
    if (!pending) return first;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

int pepsi_engine_start(pepsi_engine* e) {
  if (!e) return PEPSI_E_PARAM;
  std::lock_guard<std::mutex> lock(e->mu);
  if (e->thread_on) return PEPSI_OK;
  e->stop = false;
  e->thread_on = true;
  e->th = std::thread(engine_thread, e);
  return PEPSI_OK;
}

int pepsi_engine_stop(pepsi_engine* e) {
  if (!e) return PEPSI_E_PARAM;
  {
    std::lock_guard<std::mutex> lock(e->mu);
    if (!e->thread_on) return PEPSI_OK;
    e->stop = true;
  }
  e->cv.notify_all();
  e->th.join();
  std::lock_guard<std::mutex> lock(e->mu);
  e->thread_on = false;
  return PEPSI_OK;
}

int pepsi_engine_wait(pepsi_engine* e, uint64_t ticket, double* latency_ms) {
  if (!e) return PEPSI_E_PARAM;
  for (;;) {
    bool self_pump = false;
    {
      std::unique_lock<std::mutex> lock(e->mu);
      auto it = e->reqs.find(ticket);
      if (it == e->reqs.end()) return PEPSI_E_PARAM;
      if (it->second.status >= 0) {  // done: report it and forget the ticket
        if (latency_ms)
          *latency_ms =
              std::chrono::duration<double, std::milli>(it->second.t_done - it->second.t_submit).count();
        const int status = it->second.status;
        e->reqs.erase(it);
        return status;
      }
      if (e->thread_on)
        e->cv.wait_for(lock, std::chrono::milliseconds(1));
      else
        self_pump = true;
    }
    if (self_pump) {  // failures complete their requests: this one reports its own status
      uint64_t pending = 0;
      pump_once(e, &pending);
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  }
}

int pepsi_engine_fail_next(pepsi_engine* e, int lane, int status) {
  if (!e || lane < 0 || lane >= (int)e->lanes.size() || status <= PEPSI_OK || status > PEPSI_E_NOISE)
    return PEPSI_E_PARAM;
  std::lock_guard<std::mutex> pl(e->pump_mu);
  e->lanes[lane].fail_next = status;
  return PEPSI_OK;
}

int pepsi_engine_get_stats(pepsi_engine* e, pepsi_engine_stats* out) {
  if (!e || !out) return PEPSI_E_PARAM;
  std::lock_guard<std::mutex> lock(e->mu);
  out->submitted = e->submitted;
  out->completed = e->completed;
  out->steps = e->steps;
  out->bytes_in_use = e->used;
  out->bytes_peak = e->peak;
  out->budget = e->budget;
  return PEPSI_OK;
}

int pepsi_engine_capture(pepsi_engine* e, void* stream, pepsi_graph** out) {
  if (!e || !out) return PEPSI_E_PARAM;
  *out = nullptr;
  std::lock_guard<std::mutex> pl(e->pump_mu);
  std::vector<std::pair<int, u64>> routed;
  {
    std::lock_guard<std::mutex> lock(e->mu);
    if (e->thread_on) return PEPSI_E_PARAM;
    for (const Lane& L : e->lanes) {
      if (!L.inflight.empty()) return PEPSI_E_PARAM;
      for (int s = 0; s < L.nslots; ++s)
        if (L.slot[s].busy) return PEPSI_E_PARAM;
    }
    for (u64 t : e->incoming) {  // captured requests read and write device memory only
      const Request& r = e->reqs.at(t);
      if (!is_device_ptr(r.cts) || !is_device_ptr(r.out)) return PEPSI_E_PARAM;
    }
    for (const Lane& L : e->lanes)
      for (u64 t : L.queue)
        if (!is_device_ptr(e->reqs.at(t).cts) || !is_device_ptr(e->reqs.at(t).out)) return PEPSI_E_PARAM;
    while (!e->incoming.empty()) {
      const u64 t = e->incoming.front();
      e->incoming.pop_front();
      routed.push_back({e->reqs.at(t).lane, t});
    }
  }
  for (auto& rt : routed) e->lanes[rt.first].queue.push_back(rt.second);
  auto* g = new pepsi_graph();
  g->nlanes = (int)e->lanes.size();
  g->device = e->lanes.empty() ? -1 : e->lanes[0].c->device;
  cudaError_t err = cudaHostAlloc((void**)&g->err, g->nlanes * sizeof(int), 0);
  if (err == cudaSuccess) memset(g->err, 0, g->nlanes * sizeof(int));
  cudaStream_t origin = (cudaStream_t)stream;
  if (err == cudaSuccess && !origin) {
    err = cudaStreamCreateWithFlags(&g->own, cudaStreamNonBlocking);
    origin = g->own;
  }
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins(e->lanes.size(), nullptr);
  if (err == cudaSuccess) err = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  for (auto& j : joins)
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
  bool capturing = false;
  if (err == cudaSuccess) err = cudaStreamBeginCapture(origin, cudaStreamCaptureModeRelaxed);
  capturing = err == cudaSuccess;
  if (err == cudaSuccess) err = cudaEventRecord(fork, origin);
  for (Lane& L : e->lanes)
    if (err == cudaSuccess) err = cudaStreamWaitEvent(L.c->stream, fork, 0);
  int rc = err == cudaSuccess ? PEPSI_OK : cuda_status(err);
  // the whole schedule, open loop: a request's state goes back to the budget
  // as soon as its final step is queued (later steps of the graph reuse it)
  std::vector<u64> captured;
  for (bool work = true; work && rc == PEPSI_OK;) {
    work = false;
    for (Lane& L : e->lanes) {
      for (int s = 0; s < L.nslots && !L.queue.empty() && rc == PEPSI_OK; ++s) {
        if (L.slot[s].busy) continue;
        const u64 t = L.queue.front();
        Request r;
        size_t bytes = 0;
        {
          std::lock_guard<std::mutex> lock(e->mu);
          r = e->reqs.at(t);
          bytes = request_bytes(L, rescale_run(L.c, L.mu, r.mode) > 1);
          if (e->used + bytes > e->budget && e->used > 0) break;
          e->used += bytes;
          e->peak = std::max(e->peak, e->used);
        }
        L.queue.pop_front();
        rc = admit(e, L, s, t, r, bytes);
      }
      bool busy = false;
      for (int s = 0; s < L.nslots; ++s) busy |= L.slot[s].busy;
      if (!busy || rc != PEPSI_OK) continue;
      Step step;
      rc = enqueue_step(L, step, true);
      std::lock_guard<std::mutex> lock(e->mu);
      ++e->steps;
      e->used -= step.released;
      for (u64 t : step.finishing) captured.push_back(t);
      work = true;
    }
    for (const Lane& L : e->lanes) work |= !L.queue.empty();
  }
  // join every lane back to the origin; each lane's error word is read and cleared there
  for (size_t i = 0; i < e->lanes.size() && rc == PEPSI_OK; ++i) {
    pepsi_ctx* c = e->lanes[i].c;
    err = cudaEventRecord(joins[i], c->stream);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(origin, joins[i], 0);
    if (err == cudaSuccess) err = cudaMemcpyAsync(g->err + i, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, origin);
    if (err == cudaSuccess) err = cudaMemsetAsync(c->d_err, 0, sizeof(int), origin);
    if (err != cudaSuccess) rc = cuda_status(err);
  }
  if (capturing) {
    const cudaError_t ee = cudaStreamEndCapture(origin, &g->graph);
    if (rc == PEPSI_OK && ee != cudaSuccess) rc = cuda_status(ee);
  }
  if (rc == PEPSI_OK) {
    err = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (err != cudaSuccess) rc = cuda_status(err);
  }
  cudaEventDestroy(fork);
  for (auto j : joins) cudaEventDestroy(j);
  {  // the captured requests are handed over to the graph: their tickets are done
    std::lock_guard<std::mutex> lock(e->mu);
    const Clock::time_point now = Clock::now();
    for (u64 t : captured) {
      Request& r = e->reqs.at(t);
      r.status = rc;
      r.t_done = now;
      ++e->completed;
    }
  }
  e->cv.notify_all();
  if (rc != PEPSI_OK) {
    for (Lane& L : e->lanes)  // a failed capture leaves no request behind
      for (int s = 0; s < L.nslots; ++s) L.slot[s] = Slot{};
    pepsi_graph_destroy(g);
    return rc;
  }
  *out = g;
  return PEPSI_OK;
}

int pepsi_graph_launch(pepsi_graph* g, void* stream, int synchronize) {
  if (!g || !g->exec) return PEPSI_E_PARAM;
  cudaStream_t st = stream ? (cudaStream_t)stream : g->own;
  if (!st) return PEPSI_E_PARAM;
  cudaError_t err = cudaGraphLaunch(g->exec, st);
  g->last = st;
  if (err != cudaSuccess) return cuda_status(err);
  if (!synchronize) return PEPSI_OK;
  err = cudaStreamSynchronize(st);
  if (err != cudaSuccess) return cuda_status(err);
  for (int i = 0; i < g->nlanes; ++i)
    if (g->err[i]) return PEPSI_E_TIMEOUT;
  return PEPSI_OK;
}

void pepsi_graph_destroy(pepsi_graph* g) {
  if (!g) return;
  if (g->last) cudaStreamSynchronize(g->last);
  const int trim = g->exec ? g->device : -1;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->own) cudaStreamDestroy(g->own);
  if (g->err) cudaFreeHost(g->err);
  delete g;
  // the graph's request state came from the device's graph memory pool,
  // which keeps its physical memory until trimmed
  if (trim >= 0) cudaDeviceGraphMemTrim(trim);
}

void pepsi_engine_destroy(pepsi_engine* e) {
  if (!e) return;
  pepsi_engine_stop(e);
  for (int guard = 0; guard < 1000000; ++guard) {  // finish what is in flight
    uint64_t pending = 0;
    pump_once(e, &pending);
    if (!pending) break;
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  for (Lane& L : e->lanes) {
    if (L.c) cudaStreamSynchronize(L.c->stream);
    for (int s = 0; s < kMaxSlots; ++s)
      if (L.slot[s].busy && L.c) release(L.slot[s], L.c->stream);
    for (Step& s : L.inflight) L.spare.push_back(s.ev);
    for (cudaEvent_t ev : L.spare) cudaEventDestroy(ev);
    if (L.err_ring) cudaFreeHost(L.err_ring);
    if (L.c) {
      cudaStreamSynchronize(L.c->stream);
      pepsi_destroy(L.c);
    }
  }
  if (e->pool) cudaMemPoolDestroy(e->pool);
  delete e;
}

}  // extern "C"
