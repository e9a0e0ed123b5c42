// jx_batch.cu — host side of the batch API declared in include/jx.h: env
// groups of different map and frame sizes stepped in one persistent launch,
// the tiling autotuner, and CUDA-graph capture of step sequences.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>
#include <vector>

#include "jx_host.h"

using jx::host::aligned16;
using jx::host::cuda_fail;
using jx::host::DeviceGuard;
using jx::host::fail;

struct jx_batch {
  int device = 0;
  int num_sms = 0;
  size_t smem_per_sm = 0, reserved = 0, optin = 0;
  std::vector<jx_env*> envs;  // the groups, in the order given
  std::vector<int64_t> env_off, frame_off;
  int64_t n_total = 0, frame_total = 0;
  std::vector<int> order;  // launch order of the groups (indices into envs): largest frames first
  jx_tiling tiling{};
  jx::BatchParams bp{};  // groups in launch order; per-call pointers unset
  int block_smem = 0;
  int grid[5] = {};  // per mode
  uint32_t* queue = nullptr;
  uint8_t* scratch = nullptr;
  size_t scratch_bytes = 0;
  std::atomic<uint64_t> launches{0};
};

struct jx_graph {
  int device = 0;
  jx_batch* batch = nullptr;
  int32_t steps = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

constexpr int kModes[] = {jx::MODE_STEP, jx::MODE_RESET, jx::MODE_RENDER, jx::MODE_ROLLOUT};

jx_status check_tiling(const jx_tiling& t) {
  if (t.warps_per_block != 1 && t.warps_per_block != 2 && t.warps_per_block != 4)
    return fail(JX_EINVAL, "warps_per_block must be 1, 2 or 4 (got %d)", t.warps_per_block);
  if (t.cols_per_lane != 1 && t.cols_per_lane != 2)
    return fail(JX_EINVAL, "cols_per_lane must be 1 or 2 (got %d)", t.cols_per_lane);
  if (t.bits_min_side < 0) return fail(JX_EINVAL, "bits_min_side must be >= 0 (got %d)", t.bits_min_side);
  if (t.max_rows_per_block < 1 || t.max_rows_per_block > 64)
    return fail(JX_EINVAL, "max_rows_per_block must be in [1, 64] (got %d)", t.max_rows_per_block);
  if (t.staging_buffers != 1 && t.staging_buffers != 2)
    return fail(JX_EINVAL, "staging_buffers must be 1 or 2 (got %d)", t.staging_buffers);
  return JX_OK;
}

// Lay out every group for tiling t, size the launch and (re)allocate the
// maze work space. Leaves the batch unchanged on failure.
jx_status apply_tiling(jx_batch* b, const jx_tiling& t) {
  if (jx_status st = check_tiling(t)) return st;
  jx::BatchParams bp{};
  bp.n_groups = (int32_t)b->order.size();
  size_t stride = 0;
  int warp_bytes = 0;
  for (int i = 0; i < bp.n_groups; ++i) {
    const jx_env* env = b->envs[b->order[i]];
    jx::Params p = env->base;
    const int S = env->cfg.map_side;
    p.map_bits = t.bits_min_side > 0 && S >= t.bits_min_side && S % 8 == 0;
    p.staging = t.staging_buffers;
    jx::host::choose_rows(p, t.max_rows_per_block, t.warps_per_block, jx::kMinBlocksPerSm, b->smem_per_sm,
                          b->reserved);
    p.out_stride = (int32_t)b->n_total;
    p.frame_step = (size_t)b->frame_total;
    stride = std::max(stride, jx::gen_scratch_bytes(env->cfg.task, S));
    warp_bytes = std::max(warp_bytes, p.warp_bytes);
    bp.g[i] = p;
  }
  bp.warp_bytes = warp_bytes;
  const int smem = warp_bytes * t.warps_per_block;
  if ((size_t)smem > b->optin)
    return fail(JX_EINVAL, "tiling needs %d bytes of shared memory per block (limit %zu)", smem, b->optin);
  int grid[5] = {};
  int max_grid = 0;
  for (int mode : kModes) {
    int bps = 0;
    cudaError_t err = jx::batch_blocks_per_sm(mode, t.cols_per_lane, jx::batch_spec(bp), t.warps_per_block, smem, &bps);
    if (err != cudaSuccess) return cuda_fail(err, "occupancy query");
    if (bps < 1) return fail(JX_EINVAL, "batched kernel cannot be resident with %d bytes of shared memory", smem);
    const int64_t need = (b->n_total + t.warps_per_block - 1) / t.warps_per_block;
    const int64_t cap = (int64_t)bps * b->num_sms;
    grid[mode] = (int)std::min(need, cap);
    max_grid = std::max(max_grid, grid[mode]);
  }
  const size_t scratch_need = stride * (size_t)max_grid * t.warps_per_block;
  if (scratch_need > b->scratch_bytes) {
    uint8_t* fresh = nullptr;
    cudaError_t err = cudaMalloc(&fresh, scratch_need);
    if (err != cudaSuccess) return fail(JX_ENOMEM, "cudaMalloc of %zu scratch bytes failed", scratch_need);
    if (b->scratch) {
      cudaDeviceSynchronize();  // launches in flight may still use the old work space
      cudaFree(b->scratch);
    }
    b->scratch = fresh;
    b->scratch_bytes = scratch_need;
  }
  for (int i = 0; i < bp.n_groups; ++i) {
    bp.g[i].gen_scratch = stride > 0 ? b->scratch : nullptr;
    bp.g[i].gen_scratch_stride = stride;
  }
  bp.queue = b->queue;
  b->bp = bp;
  b->tiling = t;
  b->block_smem = smem;
  std::memcpy(b->grid, grid, sizeof(grid));
  return JX_OK;
}

jx_status check_batch(const jx_batch* b) {
  if (!b) return fail(JX_EINVAL, "batch is NULL");
  return JX_OK;
}

// One launch of the batched kernel with the per-call pointers of every group.
jx_status batch_run(jx_batch* b, int mode, cudaStream_t stream, const uint8_t* actions, uint8_t* frames,
                    float* rewards, uint8_t* dones, int32_t steps, bool count = true) {
  jx::BatchParams bp = b->bp;
  for (int i = 0; i < bp.n_groups; ++i) {
    const int g = b->order[i];
    jx::Params& p = bp.g[i];
    p.actions = actions ? actions + b->env_off[g] : nullptr;
    p.rewards = rewards ? rewards + b->env_off[g] : nullptr;
    p.dones = dones ? dones + b->env_off[g] : nullptr;
    p.frames = frames + b->frame_off[g];
    p.steps = steps;
  }
  DeviceGuard dg(b->device);
  if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
  if (mode == jx::MODE_STEP || mode == jx::MODE_ROLLOUT || mode == jx::MODE_RESET) {
    for (int i = 0; i < bp.n_groups; ++i) {  // groups whose next episodes are built ahead
      if (!bp.g[i].nx_ep) continue;
      cudaError_t err = jx::pregen_launch(bp.g[i], mode == jx::MODE_ROLLOUT ? steps : 1, mode == jx::MODE_RESET, stream);
      if (err != cudaSuccess) return cuda_fail(err, "pre-generation launch");
      if (count) b->launches.fetch_add(jx::kPregenKernels, std::memory_order_relaxed);
    }
  }
  cudaError_t err = jx::batch_launch(bp, mode, b->tiling.cols_per_lane, b->tiling.warps_per_block, b->grid[mode],
                                     stream);
  if (err != cudaSuccess) {
    // The kernel's last warp clears the work-queue counters for the next
    // launch; a launch that failed may not have got there, so clear them here
    // (on the same stream) or every later launch would find drained queues.
    (void)cudaMemsetAsync(bp.queue, 0, sizeof(uint32_t) * (jx::kMaxGroups + 1), stream);
    return cuda_fail(err, "batched kernel launch");
  }
  if (count) b->launches.fetch_add(1, std::memory_order_relaxed);
  return JX_OK;
}

jx_status check_outputs(const uint8_t* actions, const uint8_t* frames, const float* rewards, const uint8_t* dones) {
  if (!actions || !rewards || !dones) return fail(JX_EINVAL, "NULL device pointer");
  if (!frames || !aligned16(frames)) return fail(JX_EINVAL, "d_frames must be a 16-byte aligned device pointer");
  return JX_OK;
}

// The autotuner's search space, the default tiling first.
std::vector<jx_tiling> search_space() {
  jx_tiling def;
  jx_tiling_default(&def);
  std::vector<jx_tiling> out{def};
  for (int w : {1, 2, 4})
    for (int c : {1, 2})
      for (int bits : {0, 128, 64, 32, 8})
        for (int rows : {8, 16, 32})
          for (int staging : {1, 2}) {
            jx_tiling t{w, c, bits, rows, staging};
            if (std::memcmp(&t, &def, sizeof(t)) != 0) out.push_back(t);
          }
  return out;
}

// Device buffers of one autotuning run.
struct TuneBuffers {
  uint8_t* base = nullptr;
  uint8_t *actions = nullptr, *frames = nullptr, *dones = nullptr;
  float* rewards = nullptr;
  ~TuneBuffers() {
    if (base) cudaFree(base);
  }
};

}  // namespace

extern "C" {

jx_status jx_tiling_default(jx_tiling* out) {
  if (!out) return fail(JX_EINVAL, "out is NULL");
  out->warps_per_block = 1;
  out->cols_per_lane = 1;
  out->bits_min_side = 128;
  out->max_rows_per_block = 32;
  out->staging_buffers = 1;
  return JX_OK;
}

jx_status jx_batch_create(jx_env* const* groups, int32_t n_groups, const jx_tiling* tiling, jx_batch** out) {
  if (!out) return fail(JX_EINVAL, "out is NULL");
  *out = nullptr;
  if (!groups) return fail(JX_EINVAL, "groups is NULL");
  if (n_groups < 1 || n_groups > jx::kMaxGroups)
    return fail(JX_EINVAL, "n_groups must be in [1, %d] (got %d)", jx::kMaxGroups, n_groups);
  for (int i = 0; i < n_groups; ++i) {
    if (!groups[i]) return fail(JX_EINVAL, "group %d is NULL", i);
    if (groups[i]->device != groups[0]->device)
      return fail(JX_EINVAL, "group %d is on device %d, group 0 on device %d", i, groups[i]->device,
                  groups[0]->device);
    for (int j = 0; j < i; ++j)
      if (groups[j] == groups[i]) return fail(JX_EINVAL, "groups %d and %d are the same env", j, i);
  }
  jx_tiling t;
  if (tiling)
    t = *tiling;
  else
    jx_tiling_default(&t);
  if (jx_status st = check_tiling(t)) return st;

  jx_batch* b = new (std::nothrow) jx_batch();
  if (!b) return fail(JX_ENOMEM, "host allocation failed");
  b->device = groups[0]->device;
  b->envs.assign(groups, groups + n_groups);
  for (jx_env* env : b->envs) {
    b->env_off.push_back(b->n_total);
    b->frame_off.push_back(b->frame_total);
    b->n_total += env->cfg.n_envs;
    b->frame_total += (int64_t)env->cfg.n_envs * (int64_t)jx::host::frame_bytes(env->cfg);
  }
  if (b->n_total > INT32_MAX) {
    delete b;
    return fail(JX_EINVAL, "a batch holds at most 2^31 - 1 envs");
  }
  for (int i = 0; i < n_groups; ++i) b->order.push_back(i);
  std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
    const jx_config &a = b->envs[x]->cfg, &c = b->envs[y]->cfg;
    const int64_t fa = (int64_t)a.frame_h * a.frame_w, fc = (int64_t)c.frame_h * c.frame_w;
    if (fa != fc) return fa > fc;
    return a.map_side > c.map_side;
  });
  DeviceGuard dg(b->device);
  cudaDeviceProp prop;
  cudaError_t err = dg.err;
  if (err == cudaSuccess) err = cudaGetDeviceProperties(&prop, b->device);
  if (err != cudaSuccess) {
    delete b;
    return cuda_fail(err, "cudaGetDeviceProperties");
  }
  b->num_sms = prop.multiProcessorCount;
  b->smem_per_sm = prop.sharedMemPerMultiprocessor;
  b->reserved = prop.reservedSharedMemPerBlock;
  b->optin = prop.sharedMemPerBlockOptin;
  const size_t qbytes = sizeof(uint32_t) * (jx::kMaxGroups + 1);
  if ((err = cudaMalloc(&b->queue, qbytes)) != cudaSuccess) {
    delete b;
    return fail(JX_ENOMEM, "cudaMalloc of the work queues failed");
  }
  if ((err = cudaMemset(b->queue, 0, qbytes)) != cudaSuccess) {
    jx_batch_destroy(b);
    return cuda_fail(err, "cudaMemset of the work queues");
  }
  if (jx_status st = apply_tiling(b, t)) {
    jx_batch_destroy(b);
    return st;
  }
  if ((err = cudaDeviceSynchronize()) != cudaSuccess) {
    jx_batch_destroy(b);
    return cuda_fail(err, "batch create");
  }
  *out = b;
  return JX_OK;
}

jx_status jx_batch_destroy(jx_batch* batch) {
  if (!batch) return JX_OK;
  {
    DeviceGuard dg(batch->device);
    cudaDeviceSynchronize();
    if (batch->queue) cudaFree(batch->queue);
    if (batch->scratch) cudaFree(batch->scratch);
  }
  delete batch;
  return JX_OK;
}

jx_status jx_batch_info(const jx_batch* batch, int64_t* n_envs, int64_t* frame_bytes_per_step) {
  if (jx_status st = check_batch(batch)) return st;
  if (n_envs) *n_envs = batch->n_total;
  if (frame_bytes_per_step) *frame_bytes_per_step = batch->frame_total;
  return JX_OK;
}

jx_status jx_batch_group(const jx_batch* batch, int32_t group, int64_t* env_offset, int64_t* frame_offset) {
  if (jx_status st = check_batch(batch)) return st;
  if (group < 0 || group >= (int32_t)batch->envs.size())
    return fail(JX_EINVAL, "group %d outside [0, %zu)", group, batch->envs.size());
  if (env_offset) *env_offset = batch->env_off[group];
  if (frame_offset) *frame_offset = batch->frame_off[group];
  return JX_OK;
}

jx_status jx_batch_set_tiling(jx_batch* batch, const jx_tiling* tiling) {
  if (jx_status st = check_batch(batch)) return st;
  if (!tiling) return fail(JX_EINVAL, "tiling is NULL");
  DeviceGuard dg(batch->device);
  if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
  return apply_tiling(batch, *tiling);
}

jx_status jx_batch_get_tiling(const jx_batch* batch, jx_tiling* tiling) {
  if (jx_status st = check_batch(batch)) return st;
  if (!tiling) return fail(JX_EINVAL, "tiling is NULL");
  *tiling = batch->tiling;
  return JX_OK;
}

jx_status jx_batch_launch_shape(const jx_batch* batch, int32_t* grid, int32_t* block, int32_t* smem_bytes) {
  if (jx_status st = check_batch(batch)) return st;
  if (grid) *grid = batch->grid[jx::MODE_STEP];
  if (block) *block = 32 * batch->tiling.warps_per_block;
  if (smem_bytes) *smem_bytes = batch->block_smem;
  return JX_OK;
}

jx_status jx_batch_launch_count(const jx_batch* batch, uint64_t* count) {
  if (jx_status st = check_batch(batch)) return st;
  if (!count) return fail(JX_EINVAL, "count is NULL");
  *count = batch->launches.load(std::memory_order_relaxed);
  return JX_OK;
}

jx_status jx_batch_reset(jx_batch* batch, void* stream, uint8_t* d_frames) {
  if (jx_status st = check_batch(batch)) return st;
  if (!d_frames || !aligned16(d_frames)) return fail(JX_EINVAL, "d_frames must be a 16-byte aligned device pointer");
  return batch_run(batch, jx::MODE_RESET, static_cast<cudaStream_t>(stream), nullptr, d_frames, nullptr, nullptr, 1);
}

jx_status jx_batch_step(jx_batch* batch, void* stream, const uint8_t* d_actions, uint8_t* d_frames,
                        float* d_rewards, uint8_t* d_dones) {
  if (jx_status st = check_batch(batch)) return st;
  if (jx_status st = check_outputs(d_actions, d_frames, d_rewards, d_dones)) return st;
  return batch_run(batch, jx::MODE_STEP, static_cast<cudaStream_t>(stream), d_actions, d_frames, d_rewards, d_dones,
                   1);
}

jx_status jx_batch_rollout(jx_batch* batch, void* stream, const uint8_t* d_actions, int32_t steps,
                           uint8_t* d_frames, float* d_rewards, uint8_t* d_dones) {
  if (jx_status st = check_batch(batch)) return st;
  if (steps < 1) return fail(JX_EINVAL, "steps must be >= 1 (got %d)", steps);
  if (jx_status st = check_outputs(d_actions, d_frames, d_rewards, d_dones)) return st;
  return batch_run(batch, jx::MODE_ROLLOUT, static_cast<cudaStream_t>(stream), d_actions, d_frames, d_rewards,
                   d_dones, steps);
}

jx_status jx_batch_render(jx_batch* batch, void* stream, uint8_t* d_frames) {
  if (jx_status st = check_batch(batch)) return st;
  if (!d_frames || !aligned16(d_frames)) return fail(JX_EINVAL, "d_frames must be a 16-byte aligned device pointer");
  return batch_run(batch, jx::MODE_RENDER, static_cast<cudaStream_t>(stream), nullptr, d_frames, nullptr, nullptr, 1);
}

jx_status jx_batch_autotune(jx_batch* batch, void* stream, int32_t mode, int32_t steps, int32_t max_trials,
                            int32_t* n_trials, jx_tiling* trials, float* ms_per_step) {
  if (jx_status st = check_batch(batch)) return st;
  if (mode != 0 && mode != 1) return fail(JX_EINVAL, "mode must be 0 (steps) or 1 (rollout) (got %d)", mode);
  if (steps < 1 || steps > 1024) return fail(JX_EINVAL, "steps must be in [1, 1024] (got %d)", steps);
  if (max_trials < 1) return fail(JX_EINVAL, "max_trials must be >= 1 (got %d)", max_trials);
  if (n_trials) *n_trials = 0;
  DeviceGuard dg(batch->device);
  if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t N = (size_t)batch->n_total, F = (size_t)batch->frame_total, T = (size_t)steps;
  TuneBuffers buf;
  const size_t off_frames = jx::host::align256(T * N);
  const size_t off_rewards = off_frames + jx::host::align256(T * F);
  const size_t off_dones = off_rewards + jx::host::align256(4 * T * N);
  cudaError_t err = cudaMalloc(&buf.base, off_dones + jx::host::align256(T * N));
  if (err != cudaSuccess) {
    buf.base = nullptr;
    return fail(JX_ENOMEM, "cudaMalloc of %zu autotuning bytes failed", off_dones + T * N);
  }
  buf.actions = buf.base;
  buf.frames = buf.base + off_frames;
  buf.rewards = reinterpret_cast<float*>(buf.base + off_rewards);
  buf.dones = buf.base + off_dones;
  {
    std::vector<uint8_t> act(T * N);
    for (size_t i = 0; i < act.size(); ++i) act[i] = jx::host::tune_action(i);
    if ((err = cudaMemcpy(buf.actions, act.data(), act.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_fail(err, "copy of autotuning actions");
  }
  cudaEvent_t e0, e1;
  if ((err = cudaEventCreate(&e0)) != cudaSuccess) return cuda_fail(err, "cudaEventCreate");
  if ((err = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(err, "cudaEventCreate");
  }
  const jx_tiling before = batch->tiling;
  jx_tiling best = before;
  float best_ms = -1.f;
  int done = 0;
  jx_status st = JX_OK;
  for (const jx_tiling& t : search_space()) {
    if (done >= max_trials) break;
    if (apply_tiling(batch, t) != JX_OK) continue;  // does not fit: not a candidate
    auto run = [&]() -> jx_status {
      if (mode == 1)
        return batch_run(batch, jx::MODE_ROLLOUT, s, buf.actions, buf.frames, buf.rewards, buf.dones, steps, false);
      for (size_t k = 0; k < T; ++k)
        if (jx_status r = batch_run(batch, jx::MODE_STEP, s, buf.actions + k * N, buf.frames + k * F,
                                    buf.rewards + k * N, buf.dones + k * N, 1, false))
          return r;
      return JX_OK;
    };
    if ((st = batch_run(batch, jx::MODE_RESET, s, nullptr, buf.frames, nullptr, nullptr, 1, false)) != JX_OK) break;
    if ((st = run()) != JX_OK) break;
    cudaEventRecord(e0, s);
    if ((st = run()) != JX_OK) break;
    cudaEventRecord(e1, s);
    if ((err = cudaEventSynchronize(e1)) != cudaSuccess) {
      st = cuda_fail(err, "autotuning trial");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= (float)T;
    if (trials) trials[done] = t;
    if (ms_per_step) ms_per_step[done] = ms;
    ++done;
    if (best_ms < 0.f || ms < best_ms) {
      best_ms = ms;
      best = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (n_trials) *n_trials = done;
  jx_status st2 = apply_tiling(batch, st == JX_OK ? best : before);
  if (st2 == JX_OK) st2 = batch_run(batch, jx::MODE_RESET, s, nullptr, buf.frames, nullptr, nullptr, 1, false);
  if (st2 == JX_OK && (err = cudaStreamSynchronize(s)) != cudaSuccess) st2 = cuda_fail(err, "autotuning reset");
  if (st != JX_OK) return st;
  if (done == 0) return fail(JX_EINVAL, "no tiling of the search space fits this batch");
  return st2;
}

jx_status jx_batch_capture(jx_batch* batch, int32_t steps, const uint8_t* d_actions, uint8_t* d_frames,
                           float* d_rewards, uint8_t* d_dones, jx_graph** out) {
  if (jx_status st = check_batch(batch)) return st;
  if (!out) return fail(JX_EINVAL, "out is NULL");
  *out = nullptr;
  if (steps < 1) return fail(JX_EINVAL, "steps must be >= 1 (got %d)", steps);
  if (jx_status st = check_outputs(d_actions, d_frames, d_rewards, d_dones)) return st;
  DeviceGuard dg(batch->device);
  if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
  jx_graph* g = new (std::nothrow) jx_graph();
  if (!g) return fail(JX_ENOMEM, "host allocation failed");
  g->device = batch->device;
  g->batch = batch;
  g->steps = steps;
  cudaStream_t s;
  cudaError_t err = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (err != cudaSuccess) {
    delete g;
    return cuda_fail(err, "cudaStreamCreate");
  }
  jx_status st = JX_OK;
  err = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (err != cudaSuccess) st = cuda_fail(err, "cudaStreamBeginCapture");
  const size_t N = (size_t)batch->n_total, F = (size_t)batch->frame_total;
  for (int32_t t = 0; st == JX_OK && t < steps; ++t)
    st = batch_run(batch, jx::MODE_STEP, s, d_actions + t * N, d_frames + t * F, d_rewards + t * N, d_dones + t * N,
                   1, false);
  if (err == cudaSuccess) {
    cudaError_t e2 = cudaStreamEndCapture(s, &g->graph);
    if (st == JX_OK && e2 != cudaSuccess) st = cuda_fail(e2, "cudaStreamEndCapture");
  }
  if (st == JX_OK && (err = cudaGraphInstantiate(&g->exec, g->graph, 0)) != cudaSuccess)
    st = cuda_fail(err, "cudaGraphInstantiate");
  cudaStreamDestroy(s);
  if (st != JX_OK) {
    jx_graph_destroy(g);
    return st;
  }
  *out = g;
  return JX_OK;
}

jx_status jx_graph_launch(jx_graph* graph, void* stream) {
  if (!graph) return fail(JX_EINVAL, "graph is NULL");
  DeviceGuard dg(graph->device);
  if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
  cudaError_t err = cudaGraphLaunch(graph->exec, static_cast<cudaStream_t>(stream));
  if (err != cudaSuccess) return cuda_fail(err, "cudaGraphLaunch");
  graph->batch->launches.fetch_add((uint64_t)graph->steps, std::memory_order_relaxed);
  return JX_OK;
}

jx_status jx_graph_destroy(jx_graph* graph) {
  if (!graph) return JX_OK;
  {
    DeviceGuard dg(graph->device);
    if (graph->exec) cudaGraphExecDestroy(graph->exec);
    if (graph->graph) cudaGraphDestroy(graph->graph);
  }
  delete graph;
  return JX_OK;
}

}  // extern "C"
