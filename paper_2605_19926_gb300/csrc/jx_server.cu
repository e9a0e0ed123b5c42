// jx_server.cu — the continuous-batching step server declared in
// include/jx.h (jx_server_*).
//
// Clients open sessions (a group of envs with one config, state resident in
// device memory for the session's life) and submit step requests with host
// actions. A dispatcher thread merges the pending requests of all sessions
// into batched launches of the persistent kernel (jx_batch's kernel, one
// group per session) on a small set of launch slots, each with its own
// stream, work-queue counters, action staging and maze work space, so that
// launches of requests that arrive while others run overlap on the device.
// Session memory (env state, frames, rewards, dones) comes from one device
// arena sized by the byte budget: a session is admitted only if its block
// fits, and its block returns to the arena when the session closes.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "jx_host.h"

using jx::host::cuda_fail;
using jx::host::DeviceGuard;
using jx::host::fail;

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

constexpr size_t kArenaAlign = 256;
size_t arena_align(size_t x) { return (x + kArenaAlign - 1) & ~(kArenaAlign - 1); }

// First-fit allocator over one device range: free ranges keyed by offset,
// merged with their neighbours on release.
class Arena {
 public:
  void init(uint8_t* base, size_t bytes) {
    base_ = base;
    free_.clear();
    used_ = 0;
    if (bytes) free_[0] = bytes;
  }
  uint8_t* alloc(size_t bytes) {
    bytes = arena_align(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t off = it->first, len = it->second;
      free_.erase(it);
      if (len > bytes) free_[off + bytes] = len - bytes;
      used_ += bytes;
      return base_ + off;
    }
    return nullptr;
  }
  void release(uint8_t* p, size_t bytes) {
    bytes = arena_align(bytes);
    size_t off = (size_t)(p - base_);
    used_ -= bytes;
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + bytes == next->first) {
      bytes += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += bytes;
        return;
      }
    }
    free_[off] = bytes;
  }
  size_t used() const { return used_; }

 private:
  uint8_t* base_ = nullptr;
  size_t used_ = 0;
  std::map<size_t, size_t> free_;
};

struct Request {
  uint32_t seq;
  double t_submit;
  std::vector<uint8_t> actions;
};

struct Session {
  int32_t id = 0;
  jx_env* env = nullptr;
  jx::Params p{};  // laid out for the server's tiling; outputs point at the session buffers
  uint8_t* block = nullptr;
  size_t block_bytes = 0;
  uint8_t* d_frames = nullptr;
  float* d_rewards = nullptr;
  uint8_t* d_dones = nullptr;
  std::deque<Request> pending;
  bool ready = false, in_flight = false, closing = false;
  uint32_t next_seq = 0, done_seq = 0;
};

struct InFlight {
  Session* s;
  uint32_t seq;
  double t_submit;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  uint32_t* queue = nullptr;    // work-queue counters of the batched kernel
  uint8_t* scratch = nullptr;   // maze work space, one slot per warp
  uint8_t* h_actions = nullptr;  // pinned staging of the launch's actions
  uint8_t* d_actions = nullptr;
  bool busy = false;
  std::vector<InFlight> reqs;
};

}  // namespace

struct jx_server {
  int device = 0;
  int num_sms = 0;
  size_t smem_per_sm = 0, reserved = 0;
  jx_tiling tiling{};
  int max_map_side = 0;
  size_t scratch_stride = 0;
  int max_warps = 0;
  int64_t max_launch_envs = 0;
  size_t budget = 0;
  uint8_t* arena_mem = nullptr;
  Arena arena;
  size_t peak_used = 0;
  int32_t max_sessions = 0;
  int32_t next_id = 1;
  std::unordered_map<int32_t, Session*> sessions;
  std::vector<Slot> slots;
  cudaStream_t admin = nullptr;  // resets of newly opened sessions
  std::map<int, int> occupancy;  // 2 x block shared memory bytes + kernel spec -> blocks per SM
  std::mutex mu;
  std::mutex open_mu;  // serialises the admin stream
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  bool paused = false;
  jx_status worker_status = JX_OK;
  std::string worker_msg;
  // counters
  uint64_t submitted = 0, completed = 0, launches = 0, env_steps = 0, groups = 0, rejected = 0;
  int inflight = 0, peak_inflight = 0, peak_sessions = 0;
  std::vector<double> latencies;
};

namespace {

void free_session(jx_server* sv, Session* s) {
  if (s->env) jx_destroy(s->env);  // memory is the arena's: no device call
  if (s->block) sv->arena.release(s->block, s->block_bytes);
  sv->sessions.erase(s->id);
  delete s;
}

int blocks_per_sm(jx_server* sv, int smem, int spec) {
  const int key = smem * 2 + spec;
  auto it = sv->occupancy.find(key);
  if (it != sv->occupancy.end()) return it->second;
  int b = 0;
  if (jx::batch_blocks_per_sm(jx::MODE_STEP, sv->tiling.cols_per_lane, spec, sv->tiling.warps_per_block, smem, &b) !=
      cudaSuccess)
    b = 0;
  sv->occupancy[key] = b;
  return b;
}

// One batched launch of the head requests of `chosen` on slot `sl` (lock held).
jx_status dispatch(jx_server* sv, Slot& sl, std::vector<Session*>& chosen) {
  std::stable_sort(chosen.begin(), chosen.end(), [](const Session* a, const Session* b) {
    const int64_t fa = (int64_t)a->p.H * a->p.W, fb = (int64_t)b->p.H * b->p.W;
    return fa != fb ? fa > fb : a->p.S > b->p.S;
  });
  jx::BatchParams bp{};
  size_t off = 0;
  int warp_bytes = 0;
  int64_t total = 0;
  sl.reqs.clear();
  for (size_t i = 0; i < chosen.size(); ++i) {
    Session* s = chosen[i];
    Request& r = s->pending.front();
    std::memcpy(sl.h_actions + off, r.actions.data(), r.actions.size());
    jx::Params p = s->p;
    p.actions = sl.d_actions + off;
    p.gen_scratch = sv->scratch_stride ? sl.scratch : nullptr;
    p.gen_scratch_stride = sv->scratch_stride;
    bp.g[i] = p;
    warp_bytes = std::max(warp_bytes, p.warp_bytes);
    off += (r.actions.size() + 15) & ~(size_t)15;
    total += p.n;
    sl.reqs.push_back({s, r.seq, r.t_submit});
    s->pending.pop_front();
    s->in_flight = true;
  }
  bp.n_groups = (int32_t)chosen.size();
  bp.warp_bytes = warp_bytes;
  bp.queue = sl.queue;
  const int wpb = sv->tiling.warps_per_block, smem = warp_bytes * wpb;
  const int bps = blocks_per_sm(sv, smem, jx::batch_spec(bp));
  if (bps < 1) return fail(JX_ECUDA, "batched kernel cannot be resident with %d bytes of shared memory", smem);
  const int64_t grid = std::min<int64_t>((int64_t)bps * sv->num_sms, (total + wpb - 1) / wpb);
  cudaError_t err = cudaMemcpyAsync(sl.d_actions, sl.h_actions, off, cudaMemcpyHostToDevice, sl.stream);
  if (err != cudaSuccess) return cuda_fail(err, "copy of request actions");
  if ((err = jx::batch_launch(bp, jx::MODE_STEP, sv->tiling.cols_per_lane, wpb, (int)grid, sl.stream)) !=
      cudaSuccess)
    return cuda_fail(err, "batched kernel launch");
  if ((err = cudaEventRecord(sl.done, sl.stream)) != cudaSuccess) return cuda_fail(err, "cudaEventRecord");
  sl.busy = true;
  sv->inflight++;
  sv->peak_inflight = std::max(sv->peak_inflight, sv->inflight);
  sv->launches++;
  sv->env_steps += (uint64_t)total;
  sv->groups += chosen.size();
  return JX_OK;
}

void worker_loop(jx_server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  std::vector<Session*> ready;
  while (!sv->stop) {
    bool progress = false;
    for (Slot& sl : sv->slots) {
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess && sv->worker_status == JX_OK) {
        sv->worker_status = cuda_fail(q, "batched step");
        sv->worker_msg = jx_last_error();
      }
      const double t = now_s();
      for (InFlight& r : sl.reqs) {
        r.s->done_seq = r.seq;
        r.s->in_flight = false;
        sv->latencies.push_back(t - r.t_submit);
        sv->completed++;
        if (r.s->closing && r.s->pending.empty()) free_session(sv, r.s);
      }
      sl.reqs.clear();
      sl.busy = false;
      sv->inflight--;
      progress = true;
    }
    if (progress) sv->cv_done.notify_all();
    if (sv->worker_status == JX_OK && !sv->paused) {
      for (Slot& sl : sv->slots) {
        if (sl.busy) continue;
        ready.clear();
        for (auto& kv : sv->sessions) {
          Session* s = kv.second;
          if (s->ready && !s->in_flight && !s->pending.empty()) ready.push_back(s);
        }
        if (ready.empty()) break;
        // oldest requests first, as many groups as one launch takes
        std::sort(ready.begin(), ready.end(), [](const Session* a, const Session* b) {
          return a->pending.front().t_submit < b->pending.front().t_submit;
        });
        std::vector<Session*> chosen;
        int64_t envs = 0;
        for (Session* s : ready) {
          if ((int)chosen.size() == jx::kMaxGroups) break;
          if (envs + s->p.n > sv->max_launch_envs) continue;
          chosen.push_back(s);
          envs += s->p.n;
        }
        jx_status st = dispatch(sv, sl, chosen);
        if (st != JX_OK) {
          sv->worker_status = st;
          sv->worker_msg = jx_last_error();
          sv->cv_done.notify_all();
          break;
        }
        progress = true;
      }
    }
    if (progress) continue;
    if (sv->inflight > 0) {
      // kernels in flight: poll their events
      lk.unlock();
      std::this_thread::yield();
      lk.lock();
    } else {
      sv->cv_work.wait_for(lk, std::chrono::milliseconds(2));
    }
  }
}

jx_status check_server(const jx_server* sv) {
  if (!sv) return fail(JX_EINVAL, "server is NULL");
  return JX_OK;
}

void destroy_slots(jx_server* sv) {
  for (Slot& sl : sv->slots) {
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.queue) cudaFree(sl.queue);
    if (sl.scratch) cudaFree(sl.scratch);
    if (sl.d_actions) cudaFree(sl.d_actions);
    if (sl.h_actions) cudaFreeHost(sl.h_actions);
  }
  sv->slots.clear();
}

}  // namespace

extern "C" {

jx_status jx_server_create(int device, uint64_t budget_bytes, int32_t max_sessions, int32_t max_inflight,
                           int32_t max_map_side, const jx_tiling* tiling, jx_server** out) {
  if (!out) return fail(JX_EINVAL, "out is NULL");
  *out = nullptr;
  if (budget_bytes < kArenaAlign) return fail(JX_EINVAL, "budget_bytes must be >= %zu", kArenaAlign);
  if (max_sessions < 1) return fail(JX_EINVAL, "max_sessions must be >= 1 (got %d)", max_sessions);
  if (max_inflight < 1 || max_inflight > 16)
    return fail(JX_EINVAL, "max_inflight must be in [1, 16] (got %d)", max_inflight);
  if (max_map_side < 3 || max_map_side > jx::kMaxSide)
    return fail(JX_EINVAL, "max_map_side must be in [3, %d] (got %d)", jx::kMaxSide, max_map_side);
  jx_tiling t;
  if (tiling) {
    t = *tiling;
  } else {
    jx_tiling_default(&t);
  }
  if (t.warps_per_block != 1 && t.warps_per_block != 2 && t.warps_per_block != 4)
    return fail(JX_EINVAL, "warps_per_block must be 1, 2 or 4");
  if (t.cols_per_lane != 1 && t.cols_per_lane != 2) return fail(JX_EINVAL, "cols_per_lane must be 1 or 2");
  if (t.bits_min_side < 0 || t.max_rows_per_block < 1 || t.max_rows_per_block > 64 ||
      (t.staging_buffers != 1 && t.staging_buffers != 2))
    return fail(JX_EINVAL, "bad tiling");
  int ndev = 0;
  cudaError_t err = cudaGetDeviceCount(&ndev);
  if (err != cudaSuccess) return cuda_fail(err, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) return fail(JX_EINVAL, "device %d out of range (%d devices)", device, ndev);
  DeviceGuard dg(device);
  if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
  cudaDeviceProp prop;
  if ((err = cudaGetDeviceProperties(&prop, device)) != cudaSuccess) return cuda_fail(err, "cudaGetDeviceProperties");

  jx_server* sv = new (std::nothrow) jx_server();
  if (!sv) return fail(JX_ENOMEM, "host allocation failed");
  sv->device = device;
  sv->num_sms = prop.multiProcessorCount;
  sv->smem_per_sm = prop.sharedMemPerMultiprocessor;
  sv->reserved = prop.reservedSharedMemPerBlock;
  sv->tiling = t;
  sv->max_map_side = max_map_side;
  sv->scratch_stride = jx::gen_scratch_bytes(JX_TASK_MAZE_KEYDOOR, max_map_side & ~1);
  sv->max_warps = jx::kMinBlocksPerSm * sv->num_sms;
  sv->max_launch_envs = 1 << 20;
  sv->budget = (size_t)budget_bytes;
  sv->max_sessions = max_sessions;
  auto bail = [&](jx_status st) {
    destroy_slots(sv);
    if (sv->admin) cudaStreamDestroy(sv->admin);
    if (sv->arena_mem) cudaFree(sv->arena_mem);
    delete sv;
    return st;
  };
  if ((err = cudaMalloc(&sv->arena_mem, sv->budget)) != cudaSuccess) {
    sv->arena_mem = nullptr;
    return bail(fail(JX_ENOMEM, "cudaMalloc of the %zu-byte session arena failed", sv->budget));
  }
  sv->arena.init(sv->arena_mem, sv->budget);
  if ((err = cudaStreamCreateWithFlags(&sv->admin, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(cuda_fail(err, "cudaStreamCreate"));
  sv->slots.resize(max_inflight);
  for (Slot& sl : sv->slots) {
    const size_t qbytes = sizeof(uint32_t) * (jx::kMaxGroups + 1);
    const size_t scratch = sv->scratch_stride * (size_t)sv->max_warps;
    if ((err = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (err = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming)) != cudaSuccess ||
        (err = cudaMalloc(&sl.queue, qbytes)) != cudaSuccess ||
        (err = cudaMemset(sl.queue, 0, qbytes)) != cudaSuccess ||
        (scratch && (err = cudaMalloc(&sl.scratch, scratch)) != cudaSuccess) ||
        (err = cudaMalloc(&sl.d_actions, (size_t)sv->max_launch_envs + 16 * jx::kMaxGroups)) != cudaSuccess ||
        (err = cudaHostAlloc(&sl.h_actions, (size_t)sv->max_launch_envs + 16 * jx::kMaxGroups,
                             cudaHostAllocDefault)) != cudaSuccess)
      return bail(fail(JX_ENOMEM, "launch slot allocation failed: %s", cudaGetErrorString(err)));
  }
  if ((err = cudaDeviceSynchronize()) != cudaSuccess) return bail(cuda_fail(err, "server create"));
  try {
    sv->worker = std::thread(worker_loop, sv);
  } catch (...) {
    return bail(fail(JX_ENOMEM, "cannot start the dispatcher thread"));
  }
  *out = sv;
  return JX_OK;
}

jx_status jx_server_destroy(jx_server* sv) {
  if (!sv) return JX_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  DeviceGuard dg(sv->device);
  cudaDeviceSynchronize();
  std::vector<Session*> all;
  for (auto& kv : sv->sessions) all.push_back(kv.second);
  for (Session* s : all) free_session(sv, s);
  destroy_slots(sv);
  if (sv->admin) cudaStreamDestroy(sv->admin);
  if (sv->arena_mem) cudaFree(sv->arena_mem);
  delete sv;
  return JX_OK;
}

}  // extern "C"

namespace {

jx_status open_session(jx_server* sv, const jx_config* cfg, const char* ascii, int32_t* session) {
  if (jx_status st = check_server(sv)) return st;
  if (!session) return fail(JX_EINVAL, "session is NULL");
  *session = 0;
  size_t env_bytes = 0;
  if (jx_status st = jx::host::env_bytes(cfg, ascii, sv->device, &env_bytes)) return st;
  if (cfg->map_side > sv->max_map_side)
    return fail(JX_EINVAL, "map_side %d above the server's max_map_side %d", cfg->map_side, sv->max_map_side);
  if (cfg->n_envs > sv->max_launch_envs)
    return fail(JX_EINVAL, "n_envs %d above the server's per-launch limit %lld", cfg->n_envs,
                (long long)sv->max_launch_envs);
  const size_t n = (size_t)cfg->n_envs, fb = n * jx::host::frame_bytes(*cfg);
  const size_t off_frames = arena_align(env_bytes), off_rewards = off_frames + arena_align(fb);
  const size_t off_dones = off_rewards + arena_align(4 * n), total = off_dones + arena_align(n);
  Session* s = new (std::nothrow) Session();
  if (!s) return fail(JX_ENOMEM, "host allocation failed");
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if ((int32_t)sv->sessions.size() >= sv->max_sessions) {
      sv->rejected++;
      delete s;
      return fail(JX_EBUDGET, "all %d session slots are in use", sv->max_sessions);
    }
    s->block = sv->arena.alloc(total);
    if (!s->block) {
      sv->rejected++;
      delete s;
      return fail(JX_EBUDGET, "session needs %zu bytes; %zu of the %zu-byte budget in use", total, sv->arena.used(),
                  sv->budget);
    }
    s->block_bytes = total;
    sv->peak_used = std::max(sv->peak_used, sv->arena.used());
    s->id = sv->next_id++;
    sv->sessions[s->id] = s;  // not ready: the dispatcher skips it
    sv->peak_sessions = std::max(sv->peak_sessions, (int)sv->sessions.size());
  }
  DeviceGuard dg(sv->device);
  jx_status st = jx::host::create_in(cfg, ascii, sv->device, s->block, env_bytes, &s->env);
  s->d_frames = s->block + off_frames;
  s->d_rewards = reinterpret_cast<float*>(s->block + off_rewards);
  s->d_dones = s->block + off_dones;
  if (st == JX_OK) {
    std::lock_guard<std::mutex> olk(sv->open_mu);
    st = jx_reset(s->env, sv->admin, s->d_frames);
    cudaError_t err = cudaSuccess;
    if (st == JX_OK && (err = cudaMemsetAsync(s->d_rewards, 0, 5 * n, sv->admin)) != cudaSuccess)
      st = cuda_fail(err, "clearing the session outputs");
    if (st == JX_OK && (err = cudaStreamSynchronize(sv->admin)) != cudaSuccess) st = cuda_fail(err, "session reset");
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  if (st != JX_OK) {
    free_session(sv, s);
    return st;
  }
  jx::Params p = s->env->base;
  p.map_bits = sv->tiling.bits_min_side > 0 && cfg->map_side >= sv->tiling.bits_min_side && cfg->map_side % 8 == 0;
  p.staging = sv->tiling.staging_buffers;
  jx::host::choose_rows(p, sv->tiling.max_rows_per_block, sv->tiling.warps_per_block, jx::kMinBlocksPerSm,
                        sv->smem_per_sm, sv->reserved);
  p.frames = s->d_frames;
  p.rewards = s->d_rewards;
  p.dones = s->d_dones;
  p.steps = 1;
  s->p = p;
  s->ready = true;
  *session = s->id;
  return JX_OK;
}

}  // namespace

extern "C" {

jx_status jx_server_open(jx_server* sv, const jx_config* cfg, int32_t* session) {
  return open_session(sv, cfg, nullptr, session);
}

jx_status jx_server_open_ascii(jx_server* sv, const jx_config* cfg, const char* ascii, int32_t* session) {
  if (!ascii) return fail(JX_EINVAL, "ascii is NULL");
  return open_session(sv, cfg, ascii, session);
}

jx_status jx_server_close(jx_server* sv, int32_t session) {
  if (jx_status st = check_server(sv)) return st;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->sessions.find(session);
  if (it == sv->sessions.end() || !it->second->ready) return fail(JX_EINVAL, "no open session %d", session);
  Session* s = it->second;
  s->closing = true;
  if (!s->in_flight && s->pending.empty()) free_session(sv, s);
  sv->cv_work.notify_all();
  return JX_OK;
}

jx_status jx_server_session(jx_server* sv, int32_t session, jx_env** env, uint8_t** d_frames, float** d_rewards,
                            uint8_t** d_dones) {
  if (jx_status st = check_server(sv)) return st;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->sessions.find(session);
  if (it == sv->sessions.end() || !it->second->ready || it->second->closing)
    return fail(JX_EINVAL, "no open session %d", session);
  Session* s = it->second;
  if (env) *env = s->env;
  if (d_frames) *d_frames = s->d_frames;
  if (d_rewards) *d_rewards = s->d_rewards;
  if (d_dones) *d_dones = s->d_dones;
  return JX_OK;
}

jx_status jx_server_submit(jx_server* sv, int32_t session, const uint8_t* h_actions, uint64_t* ticket) {
  if (jx_status st = check_server(sv)) return st;
  if (!h_actions) return fail(JX_EINVAL, "h_actions is NULL");
  std::unique_lock<std::mutex> lk(sv->mu);
  if (sv->worker_status != JX_OK) return fail(sv->worker_status, "%s", sv->worker_msg.c_str());
  auto it = sv->sessions.find(session);
  if (it == sv->sessions.end() || !it->second->ready || it->second->closing)
    return fail(JX_EINVAL, "no open session %d", session);
  Session* s = it->second;
  Request r;
  r.seq = ++s->next_seq;
  r.t_submit = now_s();
  r.actions.assign(h_actions, h_actions + s->p.n);
  s->pending.push_back(std::move(r));
  sv->submitted++;
  if (ticket) *ticket = ((uint64_t)(uint32_t)session << 32) | s->next_seq;
  lk.unlock();
  sv->cv_work.notify_one();
  return JX_OK;
}

jx_status jx_server_wait(jx_server* sv, uint64_t ticket, double timeout_s) {
  if (jx_status st = check_server(sv)) return st;
  const int32_t session = (int32_t)(ticket >> 32);
  const uint32_t seq = (uint32_t)ticket;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto done = [&]() {
    if (sv->worker_status != JX_OK) return true;
    auto it = sv->sessions.find(session);
    return it == sv->sessions.end() || it->second->done_seq >= seq;
  };
  const auto limit = std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0.0);
  if (!sv->cv_done.wait_for(lk, limit, done))
    return fail(JX_ETIMEOUT, "request %u of session %d not done after %g s", seq, session, timeout_s);
  if (sv->worker_status != JX_OK) return fail(sv->worker_status, "%s", sv->worker_msg.c_str());
  return JX_OK;
}

jx_status jx_server_pause(jx_server* sv, int32_t paused) {
  if (jx_status st = check_server(sv)) return st;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->paused = paused != 0;
  }
  sv->cv_work.notify_all();
  return JX_OK;
}

jx_status jx_server_stats(jx_server* sv, jx_server_counters* out) {
  if (jx_status st = check_server(sv)) return st;
  if (!out) return fail(JX_EINVAL, "out is NULL");
  std::lock_guard<std::mutex> lk(sv->mu);
  std::memset(out, 0, sizeof(*out));
  out->requests_submitted = sv->submitted;
  out->requests_done = sv->completed;
  out->launches = sv->launches;
  out->env_steps = sv->env_steps;
  out->groups_launched = sv->groups;
  out->rejected_opens = sv->rejected;
  out->budget_bytes = sv->budget;
  out->bytes_in_use = sv->arena.used();
  out->peak_bytes_in_use = sv->peak_used;
  out->sessions_open = (int32_t)sv->sessions.size();
  out->peak_sessions = sv->peak_sessions;
  out->inflight_launches = sv->inflight;
  out->peak_inflight_launches = sv->peak_inflight;
  return JX_OK;
}

jx_status jx_server_latencies(jx_server* sv, double* out, uint64_t capacity, uint64_t* count) {
  if (jx_status st = check_server(sv)) return st;
  if (!count || (!out && capacity)) return fail(JX_EINVAL, "NULL pointer");
  std::lock_guard<std::mutex> lk(sv->mu);
  const uint64_t n = std::min<uint64_t>(capacity, sv->latencies.size());
  if (n) std::memcpy(out, sv->latencies.data(), n * sizeof(double));
  sv->latencies.erase(sv->latencies.begin(), sv->latencies.begin() + (ptrdiff_t)n);
  *count = n;
  return JX_OK;
}

}  // extern "C"
