// jx_api.cu — host side of the C ABI declared in include/jx.h: argument
// validation, the struct-of-arrays state block in device memory, per-env
// constant tables, launch shapes and the checkpoint / test hooks.
#include <atomic>
#include <cmath>
#include <mutex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "jx_host.h"

using jx::host::aligned16;
using jx::host::align256;
using jx::host::cuda_fail;
using jx::host::DeviceGuard;
using jx::host::fail;

namespace {

// The ASCII task's map, parsed on the host: the S x S cells, then the spawn
// candidates, the goal candidates and the keys (cell * 4 + colour), each in
// row-major order.
struct AsciiMap {
  std::vector<uint8_t> cells;
  std::vector<int32_t> spawn, goal, keys;
};

jx_status parse_ascii(const char* text, int S, AsciiMap& m) {
  if (!text) return fail(JX_EINVAL, "ascii is NULL");
  m.cells.assign((size_t)S * S, 1);
  int row = 0, col = 0, n_floor = 0;
  for (const char* q = text; *q; ++q) {
    const unsigned char ch = (unsigned char)*q;
    if (ch == '\n') {
      ++row;
      col = 0;
      continue;
    }
    if (ch == '\r') continue;
    if (ch < 32 || ch > 126) return fail(JX_EINVAL, "ascii map: character %d at row %d is not printable", ch, row);
    if (row >= S || col >= S) return fail(JX_EINVAL, "ascii map: cell (%d, %d) outside the %d x %d map", col, row, S, S);
    const int32_t cell = row * S + col;
    int v;
    if (ch == '#') {
      v = 1;
    } else if (ch == '.' || ch == ' ') {
      v = 0;
    } else if (ch == 'S' || ch == 'G') {
      v = 0;
      (ch == 'S' ? m.spawn : m.goal).push_back(cell);
    } else if (ch == 'r' || ch == 'b' || ch == 'y') {
      v = 0;
      m.keys.push_back(cell * 4 + (ch == 'r' ? 0 : (ch == 'b' ? 1 : 2)));
    } else if (ch == '"' || ch == '\\') {
      v = JX_UNLOCKED + (ch == '"' ? 1 : 2);
    } else if (ch == 'R' || ch == 'B' || ch == 'Y') {
      v = JX_LOCKED + (ch == 'R' ? 0 : (ch == 'B' ? 1 : 2));
    } else if (ch >= '1' && ch <= '9') {
      v = ch - '0';
    } else {
      v = 1 + ch % 9;  // other symbols (generated DMLab maps): coloured static walls
    }
    m.cells[cell] = (uint8_t)v;
    n_floor += v == 0;
    ++col;
  }
  if (m.keys.size() > (size_t)jx::kMaxSprites)
    return fail(JX_EINVAL, "ascii map: %zu keys, at most %d", m.keys.size(), jx::kMaxSprites);
  if (n_floor == 0) return fail(JX_EINVAL, "ascii map: no floor cell");
  return JX_OK;
}

jx_status validate(const jx_config* c, const AsciiMap* am = nullptr) {
  if (!c) return fail(JX_EINVAL, "config is NULL");
  if (c->n_envs < 1) return fail(JX_EINVAL, "n_envs must be >= 1 (got %d)", c->n_envs);
  if (c->task != JX_TASK_ROOMS && c->task != JX_TASK_MAZE_KEYDOOR && c->task != JX_TASK_MAZE_ROOMS &&
      c->task != JX_TASK_ASCII)
    return fail(JX_EINVAL, "unknown task %d", c->task);
  if ((c->task == JX_TASK_ASCII) != (am != nullptr))
    return fail(JX_EINVAL, c->task == JX_TASK_ASCII ? "the ASCII task needs jx_create_ascii and its map"
                                                     : "a map text needs task JX_TASK_ASCII");
  const bool maze = c->task == JX_TASK_MAZE_KEYDOOR || c->task == JX_TASK_MAZE_ROOMS;
  if (c->map_side < 3 || c->map_side > jx::kMaxSide)
    return fail(JX_EINVAL, "map_side must be in [3, %d] (got %d)", jx::kMaxSide, c->map_side);
  if (maze && (c->map_side < 6 || c->map_side % 2 != 0))
    return fail(JX_EINVAL, "maze map_side must be even and >= 6 (got %d)", c->map_side);
  if (c->frame_h < 1 || c->frame_h > jx::kMaxH)
    return fail(JX_EINVAL, "frame_h must be in [1, %d] (got %d)", jx::kMaxH, c->frame_h);
  if (c->frame_w < 16 || c->frame_w > jx::kMaxW || c->frame_w % 16 != 0)
    return fail(JX_EINVAL, "frame_w must be a multiple of 16 in [16, %d] (got %d)", jx::kMaxW, c->frame_w);
  if (c->max_sprites < 0 || c->max_sprites > jx::kMaxSprites)
    return fail(JX_EINVAL, "max_sprites must be in [0, %d] (got %d)", jx::kMaxSprites, c->max_sprites);
  if (maze && c->max_sprites < 2)
    return fail(JX_EINVAL, "the maze task needs max_sprites >= 2 (key and goal)");
  if (c->horizon < 0) return fail(JX_EINVAL, "horizon must be >= 0");
  if (c->turns_per_rev < 1 || c->turns_per_rev > 32767) return fail(JX_EINVAL, "turns_per_rev must be in [1, 32767]");
  if (!(c->wall_prob >= 0.0 && c->wall_prob <= 1.0)) return fail(JX_EINVAL, "wall_prob must be in [0, 1]");
  if (!(c->fov_deg > 0.0 && c->fov_deg < 180.0)) return fail(JX_EINVAL, "fov_deg must be in (0, 180)");
  if (!(c->move_step >= 0.0 && c->move_step <= 0.5)) return fail(JX_EINVAL, "move_step must be in [0, 0.5]");
  if (!(c->radius >= 0.0 && c->radius <= 0.49)) return fail(JX_EINVAL, "radius must be in [0, 0.49]");
  if (!std::isfinite(c->step_reward) || !std::isfinite(c->key_reward) || !std::isfinite(c->goal_reward))
    return fail(JX_EINVAL, "rewards must be finite");
  if (am && c->max_sprites < (int)am->keys.size() + (am->goal.empty() ? 0 : 1))
    return fail(JX_EINVAL, "the map has %zu keys%s: max_sprites must be at least %zu", am->keys.size(),
                am->goal.empty() ? "" : " and a goal", am->keys.size() + (am->goal.empty() ? 0 : 1));
  return JX_OK;
}

// Field sizes of the state block, in JX_F_* order.
void layout(jx_env* env) {
  const size_t N = env->cfg.n_envs, K = env->cfg.max_sprites, S = env->cfg.map_side;
  const size_t sizes[JX_F_COUNT] = {
      2 * N,      // cell_x
      2 * N,      // cell_y
      4 * N,      // frac_x
      4 * N,      // frac_y
      4 * N,      // theta0
      2 * N,      // turn
      4 * N,      // t
      4 * N,      // episode
      N,          // flags
      12 * N,     // obj
      N,          // nspr
      4 * N * K,  // spr_x
      4 * N * K,  // spr_y
      N * K,      // spr_type
      N * S * S,  // map
      4 * N,      // cos0
      4 * N,      // sin0
      env->cfg.gray_stack ? 4 * N * (size_t)env->cfg.frame_h * env->cfg.frame_w : 0,  // gray
  };
  size_t off = 0;
  for (int f = 0; f < JX_F_COUNT; ++f) {
    env->field_off[f] = off;
    env->field_size[f] = sizes[f];
    off += align256(sizes[f] > 0 ? sizes[f] : 1);
  }
  env->state_bytes = off;
}

template <class T>
T* field_ptr(jx_env* env, int f) {
  return reinterpret_cast<T*>(env->state + env->field_off[f]);
}

jx_status check_env(const jx_env* env) {
  if (!env) return fail(JX_EINVAL, "env is NULL");
  return JX_OK;
}

// Steps per hand-off chunk of a rollout launch of the env kernel (0: each
// warp runs whole envs). Measured on the 4096-env maze workload (10,000 steps
// in 128-step launches): chunks of 12 steps on 5/8 of the resident warps run
// at 9.10-9.16 us per step against 9.44-9.46 us for whole envs on all of
// them (the warps of an SM are served unequally, and the hand-off lets the
// faster ones take more chunks; with fewer warps than envs a warp always finds
// an item whose env is free). Rollouts of 20 steps lose more to the hand-off
// latency than they gain. Envs with a grayscale stack run whole: their planes
// are written by bulk copies four steps apart, which two warps could reorder.
int rollout_chunk(const jx_env* env, int steps) {
  if (env->cfg.gray_stack || steps < jx::kHandoffMinSteps) return 0;
  int chunk = jx::kHandoffChunk;
  const int64_t n = env->cfg.n_envs;
  while (n * ((steps + chunk - 1) / chunk) >= (int64_t)1 << 31) chunk *= 2;  // item numbers stay below 2^31
  return chunk < steps ? chunk : steps;
}

jx_status run(jx_env* env, const jx::Params& p, int mode, void* stream) {
  DeviceGuard g(env->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p.nx_ep && (mode == jx::MODE_STEP || mode == jx::MODE_ROLLOUT || mode == jx::MODE_RESET)) {
    cudaError_t err = jx::pregen_launch(p, mode == jx::MODE_ROLLOUT ? p.steps : 1, mode == jx::MODE_RESET, s);
    if (err != cudaSuccess) return cuda_fail(err, "pre-generation launch");
    env->launches.fetch_add(jx::kPregenKernels, std::memory_order_relaxed);
  }
  cudaError_t err = jx::launch(p, mode, mode == jx::MODE_ROLLOUT && p.chunk > 0 ? env->grid_handoff : env->grid, s);
  if (err != cudaSuccess) {
    // a failed rollout launch may leave the hand-off words set (the kernel
    // zeroes them as it ends): clear them on the same stream
    if (mode == jx::MODE_ROLLOUT && p.chunk > 0) (void)cudaMemsetAsync(p.work, 0, env->work_bytes, s);
    return cuda_fail(err, "kernel launch");
  }
  env->launches.fetch_add(1, std::memory_order_relaxed);
  return JX_OK;
}

}  // namespace

namespace jx {
namespace host {

thread_local std::string g_last_error;

jx_status fail(jx_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

jx_status cuda_fail(cudaError_t err, const char* what) {
  return fail(JX_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(err), cudaGetErrorString(err));
}

void choose_rows(Params& p, int max_rows, int warps, int blocks, size_t smem_per_sm, size_t reserved) {
  const int rowb = 3 * p.W;
  // candidates: up to max_rows (or the whole frame when it is shorter); the
  // largest with which `blocks` warps fit, else the smallest. A block need not
  // be whole fill passes (the lanes past its last row idle in the last pass):
  // wide frames leave room for few rows, and every block costs a copy-out and
  // a pass over the sprites.
  const int top = p.H < max_rows ? p.H : max_rows;
  int best = 0, smallest = 0;
  for (int rows = top; rows >= 1; --rows) {
    smallest = rows;
    Params q = p;
    q.rows_per_block = rows;
    q.frame_block_bytes = rows * rowb;
    q.gray_block_bytes = q.gray ? rows * p.W : 0;
    layout_warp_smem(q);
    const int per_block = q.warp_bytes * warps;
    if (!best && (size_t)(per_block + reserved) * (size_t)((blocks + warps - 1) / warps) <= smem_per_sm) best = rows;
  }
  const int rows = best ? best : (smallest ? smallest : 1);
  p.rows_per_block = rows;
  p.frame_block_bytes = rows * rowb;
  p.gray_block_bytes = p.gray ? rows * p.W : 0;
  layout_warp_smem(p);
}

}  // namespace host
}  // namespace jx

extern "C" {

const char* jx_last_error(void) { return jx::host::g_last_error.c_str(); }

}  // extern "C"

// Staging for jx_step_host_static: a fixed array in every device's memory,
// held until the process exits. Host code cannot use the name as a device
// address; the per-device address comes from cudaGetSymbolAddress, which
// jx_create (every path that keeps an env) calls with the env's device
// current. Under CUDA's lazy module loading that lookup is what loads this
// file's module and so reserves the array: it happens when the env is made,
// not inside the first jx_step_host_static call.
static __device__ __align__(256) uint8_t g_static_staging[JX_STATIC_STAGING_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
void* g_static_ptr[kMaxDevices] = {};

// Address of the staging array on `device`, which must be the current device
// (looked up once per device).
jx_status static_staging(int device, uint8_t** out) {
  if (device < 0 || device >= kMaxDevices) return fail(JX_EINVAL, "device %d beyond %d", device, kMaxDevices);
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_ptr[device]) {
    void* ptr = nullptr;
    cudaError_t err = cudaGetSymbolAddress(&ptr, g_static_staging);
    if (err != cudaSuccess) return cuda_fail(err, "cudaGetSymbolAddress of the static staging array");
    g_static_ptr[device] = ptr;
  }
  *out = static_cast<uint8_t*>(g_static_ptr[device]);
  return JX_OK;
}
}  // namespace

namespace {

// jx_create / jx_env_bytes / jx_create_in. Everything that does not need
// device memory is decided first (layout, tables, launch shape); then the
// env's one device block (state | aux | maze scratch) is allocated, or placed
// in the caller's memory `ext`. With `bytes_only` the block size is returned
// in *bytes and nothing is kept.
jx_status create_impl(const jx_config* cfg, int device, void* ext, size_t ext_bytes, bool bytes_only, size_t* bytes,
                      jx_env** out, const AsciiMap* am = nullptr) {
  jx_status st = validate(cfg, am);
  if (st != JX_OK) return st;
  int ndev = 0;
  cudaError_t err = cudaGetDeviceCount(&ndev);
  if (err != cudaSuccess) return cuda_fail(err, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) return fail(JX_EINVAL, "device %d out of range (%d devices)", device, ndev);

  jx_env* env = new (std::nothrow) jx_env();
  if (!env) return fail(JX_ENOMEM, "host allocation failed");
  env->cfg = *cfg;
  env->device = device;
  DeviceGuard g(device);
  if (g.err != cudaSuccess) {
    delete env;
    return cuda_fail(g.err, "cudaSetDevice");
  }
  layout(env);

  const jx_config& c = *cfg;
  const int W = c.frame_w, tpr = c.turns_per_rev;
  // aux block: error word | turn table | column table | ASCII map and
  // candidates | rollout hand-off words (zero between launches)
  const size_t aux_err = 0, aux_turn = 256, aux_col = align256(aux_turn + 8 * (size_t)tpr);
  const size_t aux_tmpl = align256(aux_col + 4 * (size_t)W);
  const size_t n_cand = am ? am->spawn.size() + am->goal.size() + am->keys.size() : 0;
  const size_t aux_cand = align256(aux_tmpl + (am ? am->cells.size() : 0));
  const size_t aux_work = align256(aux_cand + 4 * n_cand);
  const size_t aux_bytes = align256(aux_work + 4 * (2 + (size_t)c.n_envs));

  jx::Params& p = env->base;
  p.n = c.n_envs;
  p.S = c.map_side;
  p.H = c.frame_h;
  p.W = W;
  p.K = c.max_sprites;
  p.horizon = c.horizon;
  p.tpr = tpr;
  p.task = c.task;
  p.move = (float)c.move_step;
  p.radius = (float)c.radius;
  p.tan_half = (float)std::tan(0.5 * c.fov_deg * 3.14159265358979323846 / 180.0);
  p.inv_tan_half = (float)(1.0 / std::tan(0.5 * c.fov_deg * 3.14159265358979323846 / 180.0));
  for (int ev = 0; ev < 4; ++ev)
    p.reward_lut[ev] =
        (float)(c.step_reward + ((ev & 1) ? c.key_reward : 0.0) + ((ev & 2) ? c.goal_reward : 0.0));
  p.seed = c.seed;
  p.bulk_wait_rounds = jx::kBulkWaitRounds;
  p.handoff_polls = jx::kHandoffPolls;
  // wall iff k * 2^-53 < wall_prob for the 53-bit integer k = draw >> 11
  p.wall_thr = (uint64_t)std::ceil(c.wall_prob * 9007199254740992.0);

  cudaDeviceProp prop;
  if ((err = cudaGetDeviceProperties(&prop, device)) != cudaSuccess) {
    delete env;
    return cuda_fail(err, "cudaGetDeviceProperties");
  }
  env->num_sms = prop.multiProcessorCount;
  // Frame staging: one buffer per warp (each row block waits for the copy-out
  // of the one before), the largest row block (at most 32 rows) with which
  // kMinBlocksPerSm warps still fit in one SM's shared memory: fewer, larger
  // blocks beat double buffering at the same shared memory. The map is held
  // as a bit plane when that buys fewer row blocks per frame (the smaller map
  // leaves room for more rows), and always at side 128 (2 KB instead of 16 KB).
  p.gray = c.gray_stack != 0;
  p.shading = c.shading != 0;
  p.out_stride = c.n_envs;
  p.frame_step = (size_t)c.n_envs * jx::host::frame_bytes(c);
  p.staging = 1;
  {
    auto rows_with = [&](bool bits) {
      jx::Params q = p;
      q.map_bits = bits;
      jx::host::choose_rows(q, 32, jx::kWarpsPerBlock, jx::kMinBlocksPerSm, prop.sharedMemPerMultiprocessor,
                            prop.reservedSharedMemPerBlock);
      return q;
    };
    const bool bits_ok = c.map_side % 8 == 0;
    const jx::Params with_bytes = rows_with(false);
    const jx::Params with_bits = bits_ok ? rows_with(true) : with_bytes;
    auto blocks = [&](const jx::Params& q) { return (c.frame_h + q.rows_per_block - 1) / q.rows_per_block; };
    const bool bits = bits_ok && (c.map_side >= 128 || blocks(with_bits) < blocks(with_bytes));
    p = bits ? with_bits : with_bytes;
  }
  env->smem_block = jx::block_smem_bytes(p);
  const int smem_block = env->smem_block;
  if ((size_t)smem_block > prop.sharedMemPerBlockOptin) {
    delete env;
    return fail(JX_EINVAL, "configuration needs %d bytes of shared memory per block (limit %zu)", smem_block,
                prop.sharedMemPerBlockOptin);
  }
  int bps = 0;
  for (int mode = 0; mode < 5; ++mode) {
    int b = 0;
    if ((err = jx::kernel_blocks_per_sm(p, mode, &b)) != cudaSuccess) {
      delete env;
      return cuda_fail(err, "occupancy query");
    }
    bps = mode == 0 || b < bps ? b : bps;
  }
  if (bps < 1) {
    delete env;
    return fail(JX_EINVAL, "kernel cannot be resident with %d bytes of shared memory", smem_block);
  }
  env->blocks_per_sm = bps;
  const long need = (c.n_envs + jx::kWarpsPerBlock - 1) / jx::kWarpsPerBlock;
  const long cap = (long)bps * env->num_sms;
  env->grid = (int)(need < cap ? need : cap);
  {
    // hand-off rollouts: 5/8 of the resident warps, and at most 5 warps per 8 envs
    const long by_sm = cap * 5 / 8, by_envs = ((long)c.n_envs * 5 / 8 + jx::kWarpsPerBlock - 1) / jx::kWarpsPerBlock;
    env->grid_handoff = (int)(by_sm < by_envs ? by_sm : by_envs);
    if (env->grid_handoff < 1) env->grid_handoff = 1;
  }
  // maze work space: one slot per warp of the grid
  p.gen_scratch_stride = jx::gen_scratch_bytes(c.task, c.map_side);
  const size_t scratch_bytes = p.gen_scratch_stride * (size_t)env->grid * jx::kWarpsPerBlock;

  // the device block: state | aux | scratch
  const size_t off_aux = align256(env->state_bytes), off_scratch = off_aux + aux_bytes;
  const size_t total = off_scratch + align256(scratch_bytes);
  if (bytes) *bytes = total;
  if (bytes_only) {
    delete env;
    return JX_OK;
  }
  if (ext) {
    if (ext_bytes < total || (reinterpret_cast<uintptr_t>(ext) & 255u)) {
      delete env;
      return fail(JX_EINVAL, "external block must be 256-byte aligned and hold %zu bytes (got %zu)", total, ext_bytes);
    }
    env->mem = static_cast<uint8_t*>(ext);
    env->owns_mem = false;
  } else {
    if ((err = cudaMalloc(&env->mem, total)) != cudaSuccess) {
      env->mem = nullptr;
      delete env;
      return fail(JX_ENOMEM, "cudaMalloc of %zu env bytes failed: %s", total, cudaGetErrorString(err));
    }
    env->owns_mem = true;
  }
  env->mem_bytes = total;
  {
    // reserve the static staging array of this device now (see static_staging)
    uint8_t* unused = nullptr;
    if (jx_status st2 = static_staging(device, &unused)) {
      if (env->owns_mem) cudaFree(env->mem);
      delete env;
      return st2;
    }
  }
  env->state = env->mem;
  env->aux = env->mem + off_aux;
  env->scratch = scratch_bytes ? env->mem + off_scratch : nullptr;
  if ((err = cudaMemset(env->state, 0, env->state_bytes)) != cudaSuccess) {
    jx_destroy(env);
    return cuda_fail(err, "cudaMemset of the state");
  }
  {
    // per-env constant tables, computed in double and rounded once
    std::string host(aux_bytes, '\0');
    const double two_pi = 2.0 * 3.14159265358979323846;
    float* turn = reinterpret_cast<float*>(&host[aux_turn]);
    for (int k = 0; k < tpr; ++k) {
      double a = two_pi * (double)k / (double)tpr;
      turn[2 * k] = (float)std::cos(a);
      turn[2 * k + 1] = (float)std::sin(a);
    }
    float* colk = reinterpret_cast<float*>(&host[aux_col]);
    const double t = std::tan(0.5 * c.fov_deg * 3.14159265358979323846 / 180.0);
    for (int col = 0; col < W; ++col) colk[col] = (float)((2.0 * (col + 0.5) / W - 1.0) * t);
    if (am) {
      std::memcpy(&host[aux_tmpl], am->cells.data(), am->cells.size());
      int32_t* cand = reinterpret_cast<int32_t*>(&host[aux_cand]);
      for (int32_t v : am->spawn) *cand++ = v;
      for (int32_t v : am->goal) *cand++ = v;
      for (int32_t v : am->keys) *cand++ = v;
    }
    err = cudaMemcpy(env->aux, host.data(), aux_bytes, cudaMemcpyHostToDevice);
    if (err != cudaSuccess) {
      jx_destroy(env);
      return cuda_fail(err, "cudaMemcpy of tables");
    }
  }
  p.st.cell_x = field_ptr<int16_t>(env, JX_F_CELL_X);
  p.st.cell_y = field_ptr<int16_t>(env, JX_F_CELL_Y);
  p.st.frac_x = field_ptr<float>(env, JX_F_FRAC_X);
  p.st.frac_y = field_ptr<float>(env, JX_F_FRAC_Y);
  p.st.theta0 = field_ptr<float>(env, JX_F_THETA0);
  p.st.turn = field_ptr<int16_t>(env, JX_F_TURN);
  p.st.t = field_ptr<int32_t>(env, JX_F_T);
  p.st.episode = field_ptr<uint32_t>(env, JX_F_EPISODE);
  p.st.flags = field_ptr<uint8_t>(env, JX_F_FLAGS);
  p.st.obj = field_ptr<int16_t>(env, JX_F_OBJ);
  p.st.nspr = field_ptr<uint8_t>(env, JX_F_NSPR);
  p.st.spr_x = field_ptr<float>(env, JX_F_SPR_X);
  p.st.spr_y = field_ptr<float>(env, JX_F_SPR_Y);
  p.st.spr_type = field_ptr<uint8_t>(env, JX_F_SPR_TYPE);
  p.st.map = field_ptr<uint8_t>(env, JX_F_MAP);
  p.st.cos0 = field_ptr<float>(env, JX_F_COS0);
  p.st.sin0 = field_ptr<float>(env, JX_F_SIN0);
  p.st.gray = c.gray_stack ? field_ptr<uint8_t>(env, JX_F_GRAY) : nullptr;
  p.err = reinterpret_cast<uint32_t*>(env->aux + aux_err);
  p.turn_cs = reinterpret_cast<const float2*>(env->aux + aux_turn);
  p.col_k = reinterpret_cast<const float*>(env->aux + aux_col);
  p.work = reinterpret_cast<uint32_t*>(env->aux + aux_work);
  env->work_bytes = 4 * (2 + (size_t)c.n_envs);
  if (am) {
    p.tmpl = env->aux + aux_tmpl;
    p.cand = reinterpret_cast<const int32_t*>(env->aux + aux_cand);
    p.n_spawn = (int32_t)am->spawn.size();
    p.n_goal = (int32_t)am->goal.size();
    p.n_keys = (int32_t)am->keys.size();
  }
  p.gen_scratch = env->scratch;
  if (env->owns_mem && jx::pregen_wanted(c.task, c.map_side, c.horizon)) {
    // next-episode block: the state fields before the grayscale stack, the
    // episode each env's entry holds, and one walk work slot per env; without
    // the memory, episodes are built where they start, as for other configs
    const size_t N = c.n_envs, nx_bytes = env->field_off[JX_F_GRAY];
    const size_t stride = jx::pregen_work_bytes(c.map_side);
    const size_t off_ep = align256(nx_bytes), off_count = off_ep + align256(4 * N);
    const size_t off_work = off_count + 256;
    const size_t off_words = align256(off_work + stride * N);
    const size_t words_bytes = jx::pregen_words_bytes(c.map_side) * N;
    if (cudaMalloc(&env->nx_mem, off_words + words_bytes) == cudaSuccess &&
        cudaMemset(env->nx_mem + off_ep, 0xFF, 4 * N) == cudaSuccess &&
        cudaMemset(env->nx_mem + off_work, 0, stride * N) == cudaSuccess) {
      auto nx = [&](int f) { return env->nx_mem + env->field_off[f]; };
      p.nx = jx::State{reinterpret_cast<int16_t*>(nx(JX_F_CELL_X)), reinterpret_cast<int16_t*>(nx(JX_F_CELL_Y)),
                       reinterpret_cast<float*>(nx(JX_F_FRAC_X)), reinterpret_cast<float*>(nx(JX_F_FRAC_Y)),
                       reinterpret_cast<float*>(nx(JX_F_THETA0)), reinterpret_cast<int16_t*>(nx(JX_F_TURN)),
                       reinterpret_cast<int32_t*>(nx(JX_F_T)), reinterpret_cast<uint32_t*>(nx(JX_F_EPISODE)),
                       nx(JX_F_FLAGS), reinterpret_cast<int16_t*>(nx(JX_F_OBJ)), nx(JX_F_NSPR),
                       reinterpret_cast<float*>(nx(JX_F_SPR_X)), reinterpret_cast<float*>(nx(JX_F_SPR_Y)),
                       nx(JX_F_SPR_TYPE), nx(JX_F_MAP), reinterpret_cast<float*>(nx(JX_F_COS0)),
                       reinterpret_cast<float*>(nx(JX_F_SIN0)), nullptr};
      p.nx_ep = reinterpret_cast<uint32_t*>(env->nx_mem + off_ep);
      p.nx_work = env->nx_mem + off_work;
      p.nx_work_stride = stride;
      p.nx_words = reinterpret_cast<uint32_t*>(env->nx_mem + off_words);
      int lanes = 0;
      (void)jx::pregen_resident_lanes(c.map_side, env->num_sms, &lanes);
      p.nx_lanes = (int32_t)((size_t)lanes < N ? (size_t)lanes : N);
      p.nx_count = reinterpret_cast<uint32_t*>(env->nx_mem + off_count);
      // one lane builds a maze in about three times a warp's time: ahead of
      // the launch pays once a launch would start mazes on about three times
      // as many envs as there are resident warps
      p.nx_min = 3 * env->num_sms * jx::kMinBlocksPerSm;
    } else {
      if (env->nx_mem) cudaFree(env->nx_mem);
      env->nx_mem = nullptr;
      (void)cudaGetLastError();
    }
  }
  // the memset and the table copy are done before the handle is returned
  if ((err = cudaStreamSynchronize(0)) != cudaSuccess) {
    jx_destroy(env);
    return cuda_fail(err, "create");
  }
  *out = env;
  return JX_OK;
}

}  // namespace

extern "C" {

jx_status jx_create(const jx_config* cfg, int device, jx_env** out) {
  if (!out) return fail(JX_EINVAL, "out is NULL");
  *out = nullptr;
  return create_impl(cfg, device, nullptr, 0, false, nullptr, out);
}

jx_status jx_create_ascii(const jx_config* cfg, const char* ascii, int device, jx_env** out) {
  if (!out) return fail(JX_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfg) return fail(JX_EINVAL, "config is NULL");
  if (cfg->map_side < 3 || cfg->map_side > jx::kMaxSide)
    return fail(JX_EINVAL, "map_side must be in [3, %d] (got %d)", jx::kMaxSide, cfg->map_side);
  AsciiMap am;
  if (jx_status st = parse_ascii(ascii, cfg->map_side, am)) return st;
  return create_impl(cfg, device, nullptr, 0, false, nullptr, out, &am);
}

}  // extern "C"

namespace jx {
namespace host {

jx_status env_bytes(const jx_config* cfg, const char* ascii, int device, size_t* bytes) {
  if (!bytes) return fail(JX_EINVAL, "bytes is NULL");
  *bytes = 0;
  if (!ascii) return create_impl(cfg, device, nullptr, 0, true, bytes, nullptr);
  if (!cfg) return fail(JX_EINVAL, "config is NULL");
  if (cfg->map_side < 3 || cfg->map_side > jx::kMaxSide)
    return fail(JX_EINVAL, "map_side must be in [3, %d] (got %d)", jx::kMaxSide, cfg->map_side);
  AsciiMap am;
  if (jx_status st = parse_ascii(ascii, cfg->map_side, am)) return st;
  return create_impl(cfg, device, nullptr, 0, true, bytes, nullptr, &am);
}

jx_status create_in(const jx_config* cfg, const char* ascii, int device, void* d_mem, size_t bytes, jx_env** out) {
  if (!out) return fail(JX_EINVAL, "out is NULL");
  *out = nullptr;
  if (!d_mem) return fail(JX_EINVAL, "d_mem is NULL");
  if (!ascii) return create_impl(cfg, device, d_mem, bytes, false, nullptr, out);
  if (!cfg) return fail(JX_EINVAL, "config is NULL");
  if (cfg->map_side < 3 || cfg->map_side > jx::kMaxSide)
    return fail(JX_EINVAL, "map_side must be in [3, %d] (got %d)", jx::kMaxSide, cfg->map_side);
  AsciiMap am;
  if (jx_status st = parse_ascii(ascii, cfg->map_side, am)) return st;
  return create_impl(cfg, device, d_mem, bytes, false, nullptr, out, &am);
}

}  // namespace host
}  // namespace jx

extern "C" {

jx_status jx_env_bytes(const jx_config* cfg, int device, size_t* bytes) {
  if (!bytes) return fail(JX_EINVAL, "bytes is NULL");
  *bytes = 0;
  return create_impl(cfg, device, nullptr, 0, true, bytes, nullptr);
}

jx_status jx_create_in(const jx_config* cfg, int device, void* d_mem, size_t bytes, jx_env** out) {
  if (!out) return fail(JX_EINVAL, "out is NULL");
  *out = nullptr;
  if (!d_mem) return fail(JX_EINVAL, "d_mem is NULL");
  return create_impl(cfg, device, d_mem, bytes, false, nullptr, out);
}

jx_status jx_destroy(jx_env* env) {
  if (!env) return JX_OK;
  if (env->tuned) jx_batch_destroy(env->tuned);
  {
    DeviceGuard g(env->device);
    // an env in caller memory frees nothing on the device: no synchronisation
    if (env->owns_mem || env->stage) cudaDeviceSynchronize();
    if (env->owns_mem && env->mem) cudaFree(env->mem);
    if (env->nx_mem) cudaFree(env->nx_mem);
    if (env->stage) cudaFree(env->stage);
  }
  delete env;
  return JX_OK;
}

jx_status jx_reset(jx_env* env, void* stream, uint8_t* d_frames) {
  if (jx_status st = check_env(env)) return st;
  if (env->use_batch) return jx_batch_reset(env->tuned, stream, d_frames);
  if (!d_frames || !aligned16(d_frames)) return fail(JX_EINVAL, "d_frames must be a 16-byte aligned device pointer");
  jx::Params p = env->base;
  p.frames = d_frames;
  return run(env, p, jx::MODE_RESET, stream);
}

jx_status jx_step(jx_env* env, void* stream, const uint8_t* d_actions, uint8_t* d_frames, float* d_rewards,
                  uint8_t* d_dones) {
  if (jx_status st = check_env(env)) return st;
  if (env->use_batch) return jx_batch_step(env->tuned, stream, d_actions, d_frames, d_rewards, d_dones);
  if (!d_actions || !d_rewards || !d_dones) return fail(JX_EINVAL, "NULL device pointer");
  if (!d_frames || !aligned16(d_frames)) return fail(JX_EINVAL, "d_frames must be a 16-byte aligned device pointer");
  jx::Params p = env->base;
  p.actions = d_actions;
  p.frames = d_frames;
  p.rewards = d_rewards;
  p.dones = d_dones;
  return run(env, p, jx::MODE_STEP, stream);
}

jx_status jx_rollout(jx_env* env, void* stream, const uint8_t* d_actions, int32_t steps, uint8_t* d_frames,
                     float* d_rewards, uint8_t* d_dones) {
  if (jx_status st = check_env(env)) return st;
  if (env->use_batch) return jx_batch_rollout(env->tuned, stream, d_actions, steps, d_frames, d_rewards, d_dones);
  if (steps < 1) return fail(JX_EINVAL, "steps must be >= 1 (got %d)", steps);
  if (!d_actions || !d_rewards || !d_dones) return fail(JX_EINVAL, "NULL device pointer");
  if (!d_frames || !aligned16(d_frames)) return fail(JX_EINVAL, "d_frames must be a 16-byte aligned device pointer");
  jx::Params p = env->base;
  p.actions = d_actions;
  p.frames = d_frames;
  p.rewards = d_rewards;
  p.dones = d_dones;
  p.steps = steps;
  p.chunk = rollout_chunk(env, steps);
  return run(env, p, jx::MODE_ROLLOUT, stream);
}

jx_status jx_render(jx_env* env, void* stream, uint8_t* d_frames) {
  if (jx_status st = check_env(env)) return st;
  if (env->use_batch) return jx_batch_render(env->tuned, stream, d_frames);
  if (!d_frames || !aligned16(d_frames)) return fail(JX_EINVAL, "d_frames must be a 16-byte aligned device pointer");
  jx::Params p = env->base;
  p.frames = d_frames;
  return run(env, p, jx::MODE_RENDER, stream);
}

jx_status jx_debug_rays(jx_env* env, void* stream, int32_t* d_hits, float* d_perp) {
  if (jx_status st = check_env(env)) return st;
  if (!d_hits || !d_perp || !aligned16(d_hits)) return fail(JX_EINVAL, "d_hits (16-byte aligned) and d_perp needed");
  jx::Params p = env->base;
  p.dbg_hits = d_hits;
  p.dbg_perp = d_perp;
  return run(env, p, jx::MODE_RAYS, stream);
}

jx_status jx_step_host(jx_env* env, void* stream, const uint8_t* h_actions, uint8_t* h_frames, float* h_rewards,
                       uint8_t* h_dones) {
  if (jx_status st = check_env(env)) return st;
  if (!h_actions || !h_frames || !h_rewards || !h_dones) return fail(JX_EINVAL, "NULL host pointer");
  DeviceGuard g(env->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  const size_t N = env->cfg.n_envs;
  const size_t frame_bytes = N * 3 * (size_t)env->cfg.frame_h * env->cfg.frame_w;
  if (!env->stage) {
    env->stage_frames_off = align256(N);
    env->stage_rewards_off = env->stage_frames_off + align256(frame_bytes);
    env->stage_dones_off = env->stage_rewards_off + align256(4 * N);
    cudaError_t err = cudaMalloc(&env->stage, env->stage_dones_off + align256(N));
    if (err != cudaSuccess) {
      env->stage = nullptr;
      return fail(JX_ENOMEM, "cudaMalloc of host-step staging failed");
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint8_t* d_act = env->stage;
  uint8_t* d_frames = env->stage + env->stage_frames_off;
  float* d_rew = reinterpret_cast<float*>(env->stage + env->stage_rewards_off);
  uint8_t* d_done = env->stage + env->stage_dones_off;
  cudaError_t err = cudaMemcpyAsync(d_act, h_actions, N, cudaMemcpyHostToDevice, s);
  if (err != cudaSuccess) return cuda_fail(err, "copy of actions");
  jx_status st = jx_step(env, stream, d_act, d_frames, d_rew, d_done);
  if (st != JX_OK) return st;
  if ((err = cudaMemcpyAsync(h_frames, d_frames, frame_bytes, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (err = cudaMemcpyAsync(h_rewards, d_rew, 4 * N, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (err = cudaMemcpyAsync(h_dones, d_done, N, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(err, "copy of results");
  if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(err, "host step");
  return JX_OK;
}

jx_status jx_step_host_static(jx_env* env, void* stream, const uint8_t* h_actions, uint8_t* h_frames,
                              float* h_rewards, uint8_t* h_dones) {
  if (jx_status st = check_env(env)) return st;
  if (!h_actions || !h_frames || !h_rewards || !h_dones) return fail(JX_EINVAL, "NULL host pointer");
  const size_t N = env->cfg.n_envs;
  const size_t frame_bytes = N * 3 * (size_t)env->cfg.frame_h * env->cfg.frame_w;
  const size_t off_frames = align256(N);
  const size_t off_rewards = off_frames + align256(frame_bytes);
  const size_t off_dones = off_rewards + align256(4 * N);
  const size_t need = off_dones + align256(N);
  if (need > (size_t)JX_STATIC_STAGING_BYTES)
    return fail(JX_EINVAL, "this batch needs %zu bytes of staging; the static staging array holds %zu", need,
                (size_t)JX_STATIC_STAGING_BYTES);
  DeviceGuard g(env->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  uint8_t* base = nullptr;
  if (jx_status st = static_staging(env->device, &base)) return st;
  // every byte the step reads is written first in this call: nothing to clear
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint8_t* d_act = base;
  uint8_t* d_frames = base + off_frames;
  float* d_rew = reinterpret_cast<float*>(base + off_rewards);
  uint8_t* d_done = base + off_dones;
  cudaError_t err = cudaMemcpyAsync(d_act, h_actions, N, cudaMemcpyHostToDevice, s);
  if (err != cudaSuccess) return cuda_fail(err, "copy of actions");
  jx_status st = jx_step(env, stream, d_act, d_frames, d_rew, d_done);
  if (st != JX_OK) return st;
  if ((err = cudaMemcpyAsync(h_frames, d_frames, frame_bytes, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (err = cudaMemcpyAsync(h_rewards, d_rew, 4 * N, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (err = cudaMemcpyAsync(h_dones, d_done, N, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(err, "copy of results");
  if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(err, "host step");
  return JX_OK;
}

jx_status jx_autotune(jx_env* env, void* stream, int32_t mode, int32_t steps, int32_t max_trials, int32_t* n_trials,
                      jx_tiling* trials, float* ms_per_step) {
  if (jx_status st = check_env(env)) return st;
  if (mode != 0 && mode != 1) return fail(JX_EINVAL, "mode must be 0 (steps) or 1 (rollout) (got %d)", mode);
  if (steps < 1 || steps > 1024) return fail(JX_EINVAL, "steps must be in [1, 1024] (got %d)", steps);
  if (max_trials < 1) return fail(JX_EINVAL, "max_trials must be >= 1 (got %d)", max_trials);
  if (n_trials) *n_trials = 0;
  DeviceGuard g(env->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  if (!env->tuned) {
    jx_env* self = env;
    if (jx_status st = jx_batch_create(&self, 1, nullptr, &env->tuned)) return st;
  }
  env->use_batch = false;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t N = env->cfg.n_envs, T = steps, F = N * jx::host::frame_bytes(env->cfg);
  // trial 0: the env's own kernel, under the batched trials' protocol
  float env_ms = 0.f;
  {
    uint8_t* base = nullptr;
    const size_t off_frames = align256(T * N), off_rewards = off_frames + align256(T * F);
    const size_t off_dones = off_rewards + align256(4 * T * N);
    cudaError_t err = cudaMalloc(&base, off_dones + align256(T * N));
    if (err != cudaSuccess) return fail(JX_ENOMEM, "cudaMalloc of the autotuning buffers failed");
    std::string act(T * N, '\0');
    for (size_t i = 0; i < act.size(); ++i) act[i] = (char)jx::host::tune_action(i);
    uint8_t* frames = base + off_frames;
    float* rewards = reinterpret_cast<float*>(base + off_rewards);
    uint8_t* dones = base + off_dones;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    jx_status st = JX_OK;
    if ((err = cudaMemcpy(base, act.data(), act.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (err = cudaEventCreate(&e0)) != cudaSuccess || (err = cudaEventCreate(&e1)) != cudaSuccess)
      st = cuda_fail(err, "autotuning setup");
    auto run_steps = [&]() -> jx_status {
      jx::Params p = env->base;
      p.rewards = rewards;
      p.dones = dones;
      if (mode == 1) {
        p.actions = base;
        p.frames = frames;
        p.steps = steps;
        p.chunk = rollout_chunk(env, steps);  // the launch jx_rollout makes
        return run(env, p, jx::MODE_ROLLOUT, s);
      }
      for (size_t k = 0; k < T; ++k) {
        p.actions = base + k * N;
        p.frames = frames + k * F;
        p.rewards = rewards + k * N;
        p.dones = dones + k * N;
        if (jx_status r = run(env, p, jx::MODE_STEP, s)) return r;
      }
      return JX_OK;
    };
    if (st == JX_OK) {
      jx::Params p = env->base;
      p.frames = frames;
      st = run(env, p, jx::MODE_RESET, s);
    }
    if (st == JX_OK) st = run_steps();
    if (st == JX_OK && (err = cudaEventRecord(e0, s)) != cudaSuccess) st = cuda_fail(err, "cudaEventRecord");
    if (st == JX_OK) st = run_steps();
    if (st == JX_OK && (err = cudaEventRecord(e1, s)) != cudaSuccess) st = cuda_fail(err, "cudaEventRecord");
    if (st == JX_OK && (err = cudaEventSynchronize(e1)) != cudaSuccess) st = cuda_fail(err, "autotuning trial");
    if (st == JX_OK) cudaEventElapsedTime(&env_ms, e0, e1);
    env_ms /= (float)T;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(base);
    if (st != JX_OK) return st;
  }
  std::vector<jx_tiling> bt(max_trials > 1 ? max_trials - 1 : 0);
  std::vector<float> bms(bt.size());
  int32_t nb = 0;
  if (!bt.empty()) {
    if (jx_status st = jx_batch_autotune(env->tuned, stream, mode, steps, (int32_t)bt.size(), &nb, bt.data(),
                                         bms.data()))
      return st;
  } else {
    // no batched trial: leave every env reset as promised
    jx::Params p = env->base;
    uint8_t* frames = nullptr;
    cudaError_t err = cudaMalloc(&frames, F);
    if (err != cudaSuccess) return fail(JX_ENOMEM, "cudaMalloc of a reset frame buffer failed");
    p.frames = frames;
    jx_status st = run(env, p, jx::MODE_RESET, s);
    if (st == JX_OK && (err = cudaStreamSynchronize(s)) != cudaSuccess) st = cuda_fail(err, "autotuning reset");
    cudaFree(frames);
    if (st != JX_OK) return st;
  }
  float best = env_ms;
  for (int i = 0; i < nb; ++i) best = bms[i] < best ? bms[i] : best;
  env->use_batch = best < env_ms;
  if (trials) {
    trials[0] = jx_tiling{0, 0, 0, 0, 0};
    for (int i = 0; i < nb; ++i) trials[1 + i] = bt[i];
  }
  if (ms_per_step) {
    ms_per_step[0] = env_ms;
    for (int i = 0; i < nb; ++i) ms_per_step[1 + i] = bms[i];
  }
  if (n_trials) *n_trials = 1 + nb;
  return JX_OK;
}

jx_status jx_env_set_tiling(jx_env* env, const jx_tiling* tiling) {
  if (jx_status st = check_env(env)) return st;
  if (!tiling) return fail(JX_EINVAL, "tiling is NULL");
  const jx_tiling t = *tiling;
  if (t.warps_per_block == 0 && t.cols_per_lane == 0 && t.bits_min_side == 0 && t.max_rows_per_block == 0 &&
      t.staging_buffers == 0) {
    env->use_batch = false;
    return JX_OK;
  }
  DeviceGuard g(env->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  if (!env->tuned) {
    jx_env* self = env;
    if (jx_status st = jx_batch_create(&self, 1, &t, &env->tuned)) return st;
  } else if (jx_status st = jx_batch_set_tiling(env->tuned, &t)) {
    return st;
  }
  env->use_batch = true;
  return JX_OK;
}

jx_status jx_env_tiling(const jx_env* env, jx_tiling* tiling) {
  if (jx_status st = check_env(env)) return st;
  if (!tiling) return fail(JX_EINVAL, "tiling is NULL");
  if (env->use_batch) return jx_batch_get_tiling(env->tuned, tiling);
  *tiling = jx_tiling{0, 0, 0, 0, 0};
  return JX_OK;
}

jx_status jx_state_bytes(const jx_env* env, size_t* bytes) {
  if (jx_status st = check_env(env)) return st;
  if (!bytes) return fail(JX_EINVAL, "bytes is NULL");
  *bytes = env->state_bytes;
  return JX_OK;
}

jx_status jx_state_field(const jx_env* env, int32_t field, size_t* offset, size_t* bytes) {
  if (jx_status st = check_env(env)) return st;
  if (field < 0 || field >= JX_F_COUNT) return fail(JX_EINVAL, "unknown field %d", field);
  if (offset) *offset = env->field_off[field];
  if (bytes) *bytes = env->field_size[field];
  return JX_OK;
}

jx_status jx_get_state(jx_env* env, void* h_buf, size_t bytes) {
  if (jx_status st = check_env(env)) return st;
  if (!h_buf || bytes != env->state_bytes)
    return fail(JX_EINVAL, "buffer must be %zu bytes (got %zu)", env->state_bytes, bytes);
  DeviceGuard g(env->device);
  cudaError_t err = cudaDeviceSynchronize();
  if (err == cudaSuccess) err = cudaMemcpy(h_buf, env->state, bytes, cudaMemcpyDeviceToHost);
  return err == cudaSuccess ? JX_OK : cuda_fail(err, "get_state");
}

jx_status jx_set_state(jx_env* env, const void* h_buf, size_t bytes) {
  if (jx_status st = check_env(env)) return st;
  if (!h_buf || bytes != env->state_bytes)
    return fail(JX_EINVAL, "buffer must be %zu bytes (got %zu)", env->state_bytes, bytes);
  // a private copy: positions checked, derived heading fields recomputed
  std::string blob(static_cast<const char*>(h_buf), bytes);
  auto fld = [&](int f) { return &blob[env->field_off[f]]; };
  const int N = env->cfg.n_envs, S = env->cfg.map_side;
  const int16_t* cx = reinterpret_cast<const int16_t*>(fld(JX_F_CELL_X));
  const int16_t* cy = reinterpret_cast<const int16_t*>(fld(JX_F_CELL_Y));
  const float* fx = reinterpret_cast<const float*>(fld(JX_F_FRAC_X));
  const float* fy = reinterpret_cast<const float*>(fld(JX_F_FRAC_Y));
  const float* th = reinterpret_cast<const float*>(fld(JX_F_THETA0));
  const int16_t* turn = reinterpret_cast<const int16_t*>(fld(JX_F_TURN));
  const uint8_t* nspr = reinterpret_cast<const uint8_t*>(fld(JX_F_NSPR));
  float* c0 = reinterpret_cast<float*>(fld(JX_F_COS0));
  float* s0 = reinterpret_cast<float*>(fld(JX_F_SIN0));
  for (int i = 0; i < N; ++i) {
    if (cx[i] < 0 || cx[i] >= S || cy[i] < 0 || cy[i] >= S || !(fx[i] >= 0.f && fx[i] < 1.f) ||
        !(fy[i] >= 0.f && fy[i] < 1.f))
      return fail(JX_EINVAL, "env %d: position outside the map (cell %d,%d frac %g,%g)", i, cx[i], cy[i], fx[i], fy[i]);
    if (!std::isfinite(th[i])) return fail(JX_EINVAL, "env %d: theta0 is not finite", i);
    if (turn[i] < 0 || turn[i] >= env->cfg.turns_per_rev)
      return fail(JX_EINVAL, "env %d: turn %d outside [0, %d)", i, turn[i], env->cfg.turns_per_rev);
    if (nspr[i] > env->cfg.max_sprites)
      return fail(JX_EINVAL, "env %d: %d sprites in use, at most %d", i, nspr[i], env->cfg.max_sprites);
    c0[i] = (float)std::cos((double)th[i]);
    s0[i] = (float)std::sin((double)th[i]);
  }
  DeviceGuard g(env->device);
  cudaError_t err = cudaDeviceSynchronize();
  if (err == cudaSuccess) err = cudaMemcpy(env->state, blob.data(), bytes, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaDeviceSynchronize();
  return err == cudaSuccess ? JX_OK : cuda_fail(err, "set_state");
}

jx_status jx_sync_status(jx_env* env, void* stream) {
  if (jx_status st = check_env(env)) return st;
  DeviceGuard g(env->device);
  cudaError_t err = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (err != cudaSuccess) return cuda_fail(err, "stream");
  uint32_t word = 0;
  if ((err = cudaMemcpy(&word, env->base.err, 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(err, "error word");
  if (word) {
    cudaMemset(env->base.err, 0, 4);
    return fail(JX_EDEVICE, "device error word 0x%x (1: action outside 0..6; 2: a bulk map copy completed late, or "
                            "was lost and its warp left that env and its later envs unstepped; 4: a rollout hand-off between "
                            "warps ran out of its bounded wait)", word);
  }
  return JX_OK;
}

jx_status jx_debug_wait_limit(jx_env* env, int32_t rounds) {
  if (jx_status st = check_env(env)) return st;
  if (rounds < 0) return fail(JX_EINVAL, "rounds must be >= 0 (got %d)", rounds);
  env->base.bulk_wait_rounds = rounds;
  if (env->tuned) {  // the env's one-group batch copies its parameters when its tiling is applied
    jx_tiling t;
    if (jx_status st = jx_batch_get_tiling(env->tuned, &t)) return st;
    return jx_batch_set_tiling(env->tuned, &t);
  }
  return JX_OK;
}

jx_status jx_debug_handoff_limit(jx_env* env, int32_t polls) {
  if (jx_status st = check_env(env)) return st;
  if (polls < 0) return fail(JX_EINVAL, "polls must be >= 0 (got %d)", polls);
  env->base.handoff_polls = polls;
  return JX_OK;
}

jx_status jx_launch_count(const jx_env* env, uint64_t* count) {
  if (jx_status st = check_env(env)) return st;
  if (!count) return fail(JX_EINVAL, "count is NULL");
  uint64_t batched = 0;
  if (env->tuned) jx_batch_launch_count(env->tuned, &batched);
  *count = env->launches.load(std::memory_order_relaxed) + batched;
  return JX_OK;
}

jx_status jx_launch_shape(const jx_env* env, int32_t* grid, int32_t* block, int32_t* smem_bytes) {
  if (jx_status st = check_env(env)) return st;
  if (env->use_batch) return jx_batch_launch_shape(env->tuned, grid, block, smem_bytes);
  if (grid) *grid = env->grid;
  if (block) *block = jx::kThreads;
  if (smem_bytes) *smem_bytes = env->smem_block;
  return JX_OK;
}

jx_status jx_rollout_shape(const jx_env* env, int32_t steps, int32_t* grid, int32_t* block, int32_t* smem_bytes,
                           int32_t* chunk) {
  if (jx_status st = check_env(env)) return st;
  if (steps < 1) return fail(JX_EINVAL, "steps must be >= 1 (got %d)", steps);
  if (env->use_batch) {
    if (chunk) *chunk = 0;
    return jx_batch_launch_shape(env->tuned, grid, block, smem_bytes);
  }
  const int c = rollout_chunk(env, steps);
  if (grid) *grid = c > 0 ? env->grid_handoff : env->grid;
  if (block) *block = jx::kThreads;
  if (smem_bytes) *smem_bytes = env->smem_block;
  if (chunk) *chunk = c;
  return JX_OK;
}

}  // extern "C"
