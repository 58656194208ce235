// lsas_server.cu -- a serving loop around the fused receiver.
//
// Frames of several receiver configurations (antenna count, FFT length, QAM
// order, ...) arrive one at a time in host memory.  A configuration is
// registered once: that is where memory is admitted (its plan and its
// staging buffers must fit the server's budget) and where its stream lives.
// Submitted frames wait in a per-configuration queue.  Each configuration
// has two lanes (a stream with its own staging buffers), and a lane holds one
// batch from dispatch until its results are home.  A worker thread takes the
// configuration with the oldest waiting frame among those with a free lane,
// gathers up to max_batch of its frames (or fewer once the oldest has waited
// max_wait_us), uploads them into the lane's staging buffers, runs the fused
// receiver on the batch and copies each frame's results back to its own host
// buffers.  A host callback after the copies records the completion time,
// frees the lane and wakes waiters.  While both lanes of a configuration are
// busy its frames accumulate, so under load the batches grow to max_batch
// instead of queueing many small launches (a launch of one frame costs about
// as much device time as one of a full wave); the two lanes let one batch's
// upload overlap the other's kernel.
// Memory is admitted twice: a configuration when it is registered (its
// plan, both lanes' staging and, for the learned form, the refinement's
// buffers), and every frame when it is submitted: a frame is charged its
// device footprint (input, H, bits and, when asked for, z) from submission
// until its results are home, against the frame budget (by default what the
// memory budget leaves after registration).  A frame that does not fit is
// refused with LSAS_ERR_CAPACITY, or waits a bounded time for room, so the
// queue can never hold more work than the device memory it stands for.
// A configuration registered with refinement parameters runs the learned
// form: LS estimate -> tensor-core refinement -> MRC and demap with the
// refined channel (lsas_estimate, lsas_dn_apply_tc, lsas_demodulate).
// Each frame is processed exactly as it would be alone (frames are
// independent in the kernels, and a configuration's plan splits every batch
// smaller than a wave into the same number of antenna shards), so the
// results do not depend on the mix.
// Device-side conditions (zero channel energy, a bounded wait that ran out)
// latch in the configuration's plan and are returned by lsas_server_destroy.
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "lsas.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket;
  int config;
  const void* h_in;
  float* h_H;
  uint8_t* h_bits;
  float* h_eq;
  Clock::time_point submitted;
  size_t bytes;   // device footprint charged against the frame budget
};

struct Done {
  bool done = false;
  lsas_status status = LSAS_OK;
  double latency_us = 0.0;
};

// One stream with staging for max_batch frames; busy while a batch is on it.
struct Lane {
  void* d_in = nullptr;
  float* d_H = nullptr;
  uint8_t* d_bits = nullptr;
  float* d_eq = nullptr;
  // learned form: the LS estimate, the refinement's scratch and its status
  float* d_Hls = nullptr;
  float* d_work = nullptr;
  int* d_status = nullptr;
  cudaStream_t stream = nullptr;
  bool busy = false;
};
constexpr int kLanes = 2;

struct Config {
  lsas_plan plan = nullptr;   // shared by the lanes (read-only tables, latched status)
  const uint16_t* dn_params = nullptr;   // bf16 refinement parameters (learned form)
  int M, N, cp, S, Q, D;
  lsas_input_fmt fmt;
  size_t in_b, h_b, bits_b, eq_b;   // bytes per frame
  Lane lanes[kLanes];
  std::deque<Request> queue;
  size_t bytes = 0;
  int free_lane() const {
    for (int l = 0; l < kLanes; ++l)
      if (!lanes[l].busy) return l;
    return -1;
  }
};

struct Batch;

}  // namespace

struct lsas_server_s {
  size_t budget = 0, used = 0;
  size_t frame_budget = 0;   // 0: what the budget leaves after registration
  double admit_wait_ms = 0;  // how long a submit may wait for room
  size_t inflight = 0;       // bytes of frames queued or on the device
  int max_batch = 1;
  double max_wait_us = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::vector<std::unique_ptr<Config>> configs;
  std::map<uint64_t, Done> done;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  uint64_t launched = 0, frames = 0;
};

namespace {

// Completion of one batch: a host callback after the batch's result copies.
struct Batch {
  lsas_server_s* s;
  std::vector<std::pair<uint64_t, Clock::time_point>> items;
  int config, lane;
  size_t bytes;
};

// Runs on a CUDA callback thread (no CUDA calls here): marks the batch's
// frames done with their submit-to-results latency and frees its lane.
void CUDART_CB batch_done(void* arg) {
  Batch* b = static_cast<Batch*>(arg);
  lsas_server_s* s = b->s;
  const Clock::time_point now = Clock::now();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    for (auto& it : b->items) {
      Done& d = s->done[it.first];
      d.done = true;
      d.status = LSAS_OK;
      d.latency_us = std::chrono::duration<double, std::micro>(now - it.second).count();
    }
    s->configs[b->config]->lanes[b->lane].busy = false;
    s->inflight -= b->bytes;
  }
  s->cv_done.notify_all();
  s->cv_work.notify_one();
  delete b;
}

void fail_batch(lsas_server_s* s, const std::vector<Request>& reqs, lsas_status st) {
  {
    std::lock_guard<std::mutex> lock(s->mu);
    for (const Request& r : reqs) {
      Done& d = s->done[r.ticket];
      d.done = true;
      d.status = st;
      s->inflight -= r.bytes;
    }
  }
  s->cv_done.notify_all();
}

// The frame budget in force: the one set, else what registration left.
size_t frame_budget(const lsas_server_s* s) {
  if (s->frame_budget) return s->frame_budget;
  return s->budget > s->used ? s->budget - s->used : 0;
}

// Charge `bytes` of frames against the frame budget (caller holds the lock):
// LSAS_OK once they fit, LSAS_ERR_CAPACITY if they never can or the admission
// wait runs out.
lsas_status admit(lsas_server_s* s, std::unique_lock<std::mutex>& lock, size_t bytes) {
  if (bytes > frame_budget(s)) return LSAS_ERR_CAPACITY;
  if (s->inflight + bytes > frame_budget(s)) {
    if (s->admit_wait_ms <= 0) return LSAS_ERR_CAPACITY;
    const auto until = Clock::now() + std::chrono::duration<double, std::milli>(s->admit_wait_ms);
    while (s->inflight + bytes > frame_budget(s)) {
      if (s->cv_done.wait_until(lock, until) == std::cv_status::timeout &&
          s->inflight + bytes > frame_budget(s))
        return LSAS_ERR_CAPACITY;
      if (s->stop) return LSAS_ERR_INVALID_ARG;
    }
  }
  s->inflight += bytes;
  return LSAS_OK;
}

size_t frame_bytes_of(const Config& cf, bool eq) {
  return cf.in_b + cf.h_b + cf.bits_b + (eq ? cf.eq_b : 0);
}

void worker_loop(lsas_server_s* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lock(s->mu);
  for (;;) {
    // the configuration with a free lane whose oldest waiting frame is oldest
    int pick = -1;
    Clock::time_point oldest;
    for (size_t c = 0; c < s->configs.size(); ++c) {
      Config& cf = *s->configs[c];
      if (cf.queue.empty() || cf.free_lane() < 0) continue;
      if (pick < 0 || cf.queue.front().submitted < oldest) {
        pick = static_cast<int>(c);
        oldest = cf.queue.front().submitted;
      }
    }
    if (pick < 0) {
      // nothing to dispatch: every queue is empty or waits for a busy lane
      // (a lane frees when its batch's callback runs, which notifies us)
      bool pending = false;
      for (const auto& c : s->configs) pending = pending || !c->queue.empty();
      if (s->stop && !pending) return;
      s->cv_work.wait_for(lock, std::chrono::milliseconds(50));
      continue;
    }
    Config& cf = *s->configs[pick];
    const auto deadline = oldest + std::chrono::duration<double, std::micro>(s->max_wait_us);
    if (static_cast<int>(cf.queue.size()) < s->max_batch && !s->stop && Clock::now() < deadline) {
      s->cv_work.wait_until(lock, deadline);   // gather more of this configuration
      continue;
    }
    std::vector<Request> reqs;
    while (!cf.queue.empty() && static_cast<int>(reqs.size()) < s->max_batch) {
      reqs.push_back(cf.queue.front());
      cf.queue.pop_front();
    }
    const int li = cf.free_lane();
    Lane& ln = cf.lanes[li];
    ln.busy = true;
    lock.unlock();
    // upload, run, download on the lane's stream; as in lsas_run_frame_host,
    // only the samples after each cyclic prefix cross the host link once rows
    // of N samples span at least 1 KB (the receiver never reads the prefixes)
    lsas_status st = LSAS_OK;
    const int F = static_cast<int>(reqs.size());
    const size_t bps = cf.fmt == LSAS_IN_SC16 ? 4 : 8;
    const size_t pitch = static_cast<size_t>(cf.N + cf.cp) * bps;
    const size_t keep = static_cast<size_t>(cf.N) * bps, skip = static_cast<size_t>(cf.cp) * bps;
    const bool strip = cf.cp > 0 && keep >= 1024;
    for (int i = 0; i < F && st == LSAS_OK; ++i) {
      unsigned char* dst = static_cast<unsigned char*>(ln.d_in) + i * cf.in_b;
      const unsigned char* src = static_cast<const unsigned char*>(reqs[i].h_in);
      const cudaError_t e =
          strip ? cudaMemcpy2DAsync(dst + skip, pitch, src + skip, pitch, keep,
                                    static_cast<size_t>(cf.M) * cf.S, cudaMemcpyHostToDevice, ln.stream)
                : cudaMemcpyAsync(dst, src, cf.in_b, cudaMemcpyHostToDevice, ln.stream);
      if (e != cudaSuccess) st = LSAS_ERR_CUDA;
    }
    if (st == LSAS_OK) {
      bool eq = false;   // z is computed when any frame of the batch asks for it
      for (const Request& r : reqs) eq = eq || r.h_eq != nullptr;
      if (cf.dn_params) {
        // learned form: LS, refinement on the tensor cores, MRC with it
        st = lsas_estimate(cf.plan, ln.d_in, F, ln.d_Hls, ln.stream);
        if (st == LSAS_OK)
          st = lsas_dn_apply_tc(cf.dn_params, ln.d_Hls, F * cf.M, cf.N, ln.d_work, ln.d_H,
                                ln.d_status, ln.stream);
        if (st == LSAS_OK)
          st = lsas_demodulate(cf.plan, ln.d_in, ln.d_H, F, ln.d_bits, eq ? ln.d_eq : nullptr,
                               ln.stream);
      } else {
        st = lsas_run_frame(cf.plan, ln.d_in, F, ln.d_H, ln.d_bits, eq ? ln.d_eq : nullptr,
                            ln.stream);
      }
    }
    for (int i = 0; i < F && st == LSAS_OK; ++i) {
      const Request& r = reqs[i];
      if (cudaMemcpyAsync(r.h_H, reinterpret_cast<unsigned char*>(ln.d_H) + i * cf.h_b, cf.h_b,
                          cudaMemcpyDeviceToHost, ln.stream) != cudaSuccess ||
          cudaMemcpyAsync(r.h_bits, ln.d_bits + i * cf.bits_b, cf.bits_b, cudaMemcpyDeviceToHost,
                          ln.stream) != cudaSuccess ||
          (r.h_eq && cudaMemcpyAsync(r.h_eq, reinterpret_cast<unsigned char*>(ln.d_eq) + i * cf.eq_b,
                                     cf.eq_b, cudaMemcpyDeviceToHost, ln.stream) != cudaSuccess))
        st = LSAS_ERR_CUDA;
    }
    if (st == LSAS_OK) {
      Batch* b = new Batch{s, {}, pick, li, 0};
      for (const Request& r : reqs) {
        b->items.emplace_back(r.ticket, r.submitted);
        b->bytes += r.bytes;
      }
      if (cudaLaunchHostFunc(ln.stream, batch_done, b) != cudaSuccess) {
        delete b;
        st = LSAS_ERR_CUDA;
      }
    }
    if (st != LSAS_OK) {
      // nothing will call back for this batch: wait for what was queued on
      // the lane, then free it
      cudaStreamSynchronize(ln.stream);
      fail_batch(s, reqs, st);
    }
    lock.lock();
    if (st != LSAS_OK) ln.busy = false;
    s->launched += 1;
    s->frames += F;
  }
}

}  // namespace

extern "C" {

lsas_status lsas_server_create(size_t mem_budget_bytes, int max_batch, double max_wait_us,
                               lsas_server* out) {
  if (!out) return LSAS_ERR_INVALID_ARG;
  *out = nullptr;
  if (max_batch < 1 || max_batch > 1024 || max_wait_us < 0) return LSAS_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return LSAS_ERR_CUDA;
  }
  lsas_server_s* s = new (std::nothrow) lsas_server_s();
  if (!s) return LSAS_ERR_OOM;
  s->budget = mem_budget_bytes;
  s->max_batch = max_batch;
  s->max_wait_us = max_wait_us;
  s->device = dev;
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return LSAS_OK;
}

}  // extern "C"

namespace {

lsas_status register_config(lsas_server s, int M, int N, int cp_len, int n_sym, int pilot_idx,
                            int qam_order, lsas_input_fmt fmt, const float* host_pilot_iq,
                            const uint16_t* dn_params, int* config_id) {
  if (!s || !config_id) return LSAS_ERR_INVALID_ARG;
  lsas_status st = lsas_check_config(M, N, cp_len, n_sym, pilot_idx, qam_order);
  if (st != LSAS_OK) return st;
  // the refinement runs over rows of N subcarriers in tiles of 128
  if (dn_params && (N % 128 != 0)) return LSAS_ERR_UNSUPPORTED;
  size_t fb[4];
  st = lsas_frame_bytes(M, N, cp_len, n_sym, qam_order, fmt, fb);
  if (st != LSAS_OK) return st;
  auto cf = std::make_unique<Config>();
  cf->M = M;
  cf->N = N;
  cf->cp = cp_len;
  cf->S = n_sym;
  cf->Q = qam_order;
  cf->D = n_sym - 1;
  cf->fmt = fmt;
  cf->in_b = fb[0];
  cf->h_b = fb[1];
  cf->bits_b = fb[2];
  cf->eq_b = fb[3];
  cf->dn_params = dn_params;
  const size_t B = static_cast<size_t>(s->max_batch);
  size_t work_floats = 0;
  if (dn_params) {
    st = lsas_dn_work_size(static_cast<int>(B) * M, N, &work_floats);
    if (st != LSAS_OK) return st;
  }
  // admission: staging for max_batch frames on each lane (plus, for the
  // learned form, the LS estimate and the refinement's scratch) and the
  // plan's own memory (estimated here, replaced by what the plan reports
  // once it exists)
  const size_t plan_b = static_cast<size_t>(N) * 64 + (1u << 20);
  const size_t lane_b = B * (fb[0] + fb[1] + fb[2] + fb[3]) +
                        (dn_params ? B * fb[1] + work_floats * 4 + 256 : 0);
  cf->bytes = kLanes * lane_b + plan_b;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->used + cf->bytes > s->budget) return LSAS_ERR_CAPACITY;
    s->used += cf->bytes;
  }
  auto undo = [&](lsas_status e) {
    if (cf->plan) lsas_plan_destroy(cf->plan);
    for (Lane& ln : cf->lanes) {
      cudaFree(ln.d_in);
      cudaFree(ln.d_H);
      cudaFree(ln.d_bits);
      cudaFree(ln.d_eq);
      cudaFree(ln.d_Hls);
      cudaFree(ln.d_work);
      cudaFree(ln.d_status);
      if (ln.stream) cudaStreamDestroy(ln.stream);
    }
    std::lock_guard<std::mutex> lock(s->mu);
    s->used -= cf->bytes;
    return e;
  };
  if (cudaSetDevice(s->device) != cudaSuccess) return undo(LSAS_ERR_CUDA);
  st = lsas_plan_create(M, N, cp_len, n_sym, pilot_idx, qam_order, &cf->plan);
  if (st != LSAS_OK) return undo(st);
  st = lsas_plan_set(cf->plan, fmt, s->max_batch);
  if (st == LSAS_OK && host_pilot_iq) st = lsas_plan_set_pilot(cf->plan, host_pilot_iq);
  if (st != LSAS_OK) return undo(st);
  // batches smaller than a wave run split into antenna shards, with one shard
  // count for every batch size, so that a frame's results do not depend on
  // how many frames share its batch
  if (st == LSAS_OK) st = lsas_plan_set_batch_split(cf->plan, 2);
  if (st != LSAS_OK) return undo(st);
  {
    // the plan's own allocation (tables, split-tail scratch) replaces the
    // estimate, and is admitted against the budget like the rest
    size_t held = 0;
    if (lsas_plan_device_bytes(cf->plan, &held) != LSAS_OK) return undo(LSAS_ERR_CUDA);
    std::lock_guard<std::mutex> lock(s->mu);
    const size_t actual = cf->bytes - plan_b + held;
    if (s->used - cf->bytes + actual > s->budget) {
      s->used -= cf->bytes;
      cf->bytes = 0;
    } else {
      s->used += actual - cf->bytes;
      cf->bytes = actual;
    }
  }
  if (cf->bytes == 0) return undo(LSAS_ERR_CAPACITY);
  for (Lane& ln : cf->lanes) {
    if (cudaMalloc(&ln.d_in, B * cf->in_b) != cudaSuccess ||
        cudaMalloc(&ln.d_H, B * cf->h_b) != cudaSuccess ||
        cudaMalloc(&ln.d_bits, B * cf->bits_b) != cudaSuccess ||
        cudaMalloc(&ln.d_eq, B * cf->eq_b) != cudaSuccess ||
        (dn_params && (cudaMalloc(&ln.d_Hls, B * cf->h_b) != cudaSuccess ||
                       cudaMalloc(&ln.d_work, work_floats * 4) != cudaSuccess ||
                       cudaMalloc(&ln.d_status, sizeof(int)) != cudaSuccess))) {
      cudaGetLastError();
      return undo(LSAS_ERR_OOM);
    }
    if (dn_params && cudaMemset(ln.d_status, 0, sizeof(int)) != cudaSuccess)
      return undo(LSAS_ERR_CUDA);
    if (cudaStreamCreateWithFlags(&ln.stream, cudaStreamNonBlocking) != cudaSuccess)
      return undo(LSAS_ERR_CUDA);
  }
  std::lock_guard<std::mutex> lock(s->mu);
  s->configs.push_back(std::move(cf));
  *config_id = static_cast<int>(s->configs.size()) - 1;
  return LSAS_OK;
}

}  // namespace

extern "C" {

lsas_status lsas_server_register(lsas_server s, int M, int N, int cp_len, int n_sym,
                                 int pilot_idx, int qam_order, lsas_input_fmt fmt,
                                 const float* host_pilot_iq, int* config_id) {
  return register_config(s, M, N, cp_len, n_sym, pilot_idx, qam_order, fmt, host_pilot_iq,
                         nullptr, config_id);
}

lsas_status lsas_server_register_refined(lsas_server s, int M, int N, int cp_len, int n_sym,
                                         int pilot_idx, int qam_order, lsas_input_fmt fmt,
                                         const float* host_pilot_iq,
                                         const uint16_t* d_params_bf16, int* config_id) {
  if (!d_params_bf16) return LSAS_ERR_INVALID_ARG;
  return register_config(s, M, N, cp_len, n_sym, pilot_idx, qam_order, fmt, host_pilot_iq,
                         d_params_bf16, config_id);
}

lsas_status lsas_server_set_admission(lsas_server s, size_t frame_budget_bytes, double wait_ms) {
  if (!s || wait_ms < 0) return LSAS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  s->frame_budget = frame_budget_bytes;
  s->admit_wait_ms = wait_ms;
  return LSAS_OK;
}

lsas_status lsas_server_submit(lsas_server s, int config_id, const void* h_in, float* h_H,
                               uint8_t* h_bits, float* h_eq, uint64_t* ticket) {
  if (!s || !h_in || !h_H || !h_bits || !ticket) return LSAS_ERR_INVALID_ARG;
  {
    std::unique_lock<std::mutex> lock(s->mu);
    if (config_id < 0 || config_id >= static_cast<int>(s->configs.size())) return LSAS_ERR_INVALID_ARG;
    if (s->stop) return LSAS_ERR_INVALID_ARG;
    const size_t fb = frame_bytes_of(*s->configs[config_id], h_eq != nullptr);
    const lsas_status st = admit(s, lock, fb);
    if (st != LSAS_OK) return st;
    Config& cf = *s->configs[config_id];
    const uint64_t t = s->next_ticket++;
    cf.queue.push_back(Request{t, config_id, h_in, h_H, h_bits, h_eq, Clock::now(), fb});
    s->done[t] = Done{};
    *ticket = t;
  }
  s->cv_work.notify_one();
  return LSAS_OK;
}

lsas_status lsas_server_submit_many(lsas_server s, int n, const int* config_ids,
                                    const void* const* h_in, float* const* h_H,
                                    uint8_t* const* h_bits, float* const* h_eq,
                                    uint64_t* tickets) {
  if (!s || n < 0 || (n > 0 && (!config_ids || !h_in || !h_H || !h_bits || !tickets)))
    return LSAS_ERR_INVALID_ARG;
  {
    std::unique_lock<std::mutex> lock(s->mu);
    if (s->stop) return LSAS_ERR_INVALID_ARG;
    // validate and admit everything first: either all frames are queued or none
    size_t total = 0;
    for (int i = 0; i < n; ++i) {
      if (config_ids[i] < 0 || config_ids[i] >= static_cast<int>(s->configs.size()) || !h_in[i] ||
          !h_H[i] || !h_bits[i])
        return LSAS_ERR_INVALID_ARG;
      total += frame_bytes_of(*s->configs[config_ids[i]], h_eq && h_eq[i]);
    }
    const lsas_status st = admit(s, lock, total);
    if (st != LSAS_OK) return st;
    const Clock::time_point now = Clock::now();
    for (int i = 0; i < n; ++i) {
      const uint64_t t = s->next_ticket++;
      float* eq = h_eq ? h_eq[i] : nullptr;
      s->configs[config_ids[i]]->queue.push_back(
          Request{t, config_ids[i], h_in[i], h_H[i], h_bits[i], eq, now,
                  frame_bytes_of(*s->configs[config_ids[i]], eq != nullptr)});
      s->done[t] = Done{};
      tickets[i] = t;
    }
  }
  if (n > 0) s->cv_work.notify_one();
  return LSAS_OK;
}

lsas_status lsas_server_wait_many(lsas_server s, int n, const uint64_t* tickets,
                                  double timeout_ms, double* latency_us, lsas_status* status) {
  if (!s || n < 0 || (n > 0 && !tickets)) return LSAS_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lock(s->mu);
  for (int i = 0; i < n; ++i)
    if (s->done.find(tickets[i]) == s->done.end()) return LSAS_ERR_INVALID_ARG;
  const auto until = Clock::now() + std::chrono::duration<double, std::milli>(timeout_ms);
  for (int i = 0; i < n; ++i) {
    while (!s->done[tickets[i]].done) {
      if (s->cv_done.wait_until(lock, until) == std::cv_status::timeout && !s->done[tickets[i]].done)
        return LSAS_ERR_TIMEOUT;   // every ticket stays valid
    }
  }
  lsas_status first = LSAS_OK;
  for (int i = 0; i < n; ++i) {
    const Done d = s->done[tickets[i]];
    s->done.erase(tickets[i]);
    if (latency_us) latency_us[i] = d.latency_us;
    if (status) status[i] = d.status;
    if (d.status != LSAS_OK && first == LSAS_OK) first = d.status;
  }
  return first;
}

lsas_status lsas_server_wait(lsas_server s, uint64_t ticket, double timeout_ms,
                             double* latency_us) {
  if (!s) return LSAS_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->done.find(ticket);
  if (it == s->done.end()) return LSAS_ERR_INVALID_ARG;
  const auto until = Clock::now() + std::chrono::duration<double, std::milli>(timeout_ms);
  while (!s->done[ticket].done) {
    if (s->cv_done.wait_until(lock, until) == std::cv_status::timeout && !s->done[ticket].done)
      return LSAS_ERR_TIMEOUT;
  }
  Done d = s->done[ticket];
  s->done.erase(ticket);
  if (latency_us) *latency_us = d.latency_us;
  return d.status;
}

lsas_status lsas_server_stats(lsas_server s, uint64_t out[4]) {
  if (!s || !out) return LSAS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  out[0] = s->launched;
  out[1] = s->frames;
  out[2] = s->used;
  out[3] = s->configs.size();
  return LSAS_OK;
}

lsas_status lsas_server_frame_bytes(lsas_server s, uint64_t out[2]) {
  if (!s || !out) return LSAS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  out[0] = s->inflight;
  out[1] = frame_budget(s);
  return LSAS_OK;
}

lsas_status lsas_server_destroy(lsas_server s) {
  if (!s) return LSAS_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  lsas_status st = LSAS_OK;
  for (auto& cf : s->configs) {
    for (Lane& ln : cf->lanes)
      if (ln.stream) cudaStreamSynchronize(ln.stream);
    const lsas_status ps = lsas_plan_sync(cf->plan, cf->lanes[0].stream);
    if (ps != LSAS_OK && st == LSAS_OK) st = ps;
    lsas_plan_destroy(cf->plan);
    for (Lane& ln : cf->lanes) {
      if (ln.d_status) {
        // the refinement's bounded waits latch here
        int code = 0;
        if (cudaMemcpy(&code, ln.d_status, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess &&
            code != 0 && st == LSAS_OK)
          st = static_cast<lsas_status>(code);
      }
      cudaFree(ln.d_in);
      cudaFree(ln.d_H);
      cudaFree(ln.d_bits);
      cudaFree(ln.d_eq);
      cudaFree(ln.d_Hls);
      cudaFree(ln.d_work);
      cudaFree(ln.d_status);
      if (ln.stream) cudaStreamDestroy(ln.stream);
    }
  }
  delete s;
  return st;
}

}  // extern "C"
