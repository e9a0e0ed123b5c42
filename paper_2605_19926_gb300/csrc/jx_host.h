// jx_host.h — host-side internals shared by the env API (jx_api.cu) and the
// batch API (jx_batch.cu). Not part of the public ABI.
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <string>

#include "../../include/jx.h"
#include "jx_internal.h"

struct jx_env {
  jx_config cfg;
  int device = 0;
  int num_sms = 0;
  int blocks_per_sm = 0;
  int grid = 0;
  int grid_handoff = 0;  // blocks of a rollout launch in hand-off chunks (see rollout_chunk)
  int smem_block = 0;
  jx::Params base{};
  // one device block: state | aux | scratch (owned, or in the caller's memory)
  uint8_t* mem = nullptr;
  size_t mem_bytes = 0;
  bool owns_mem = true;
  // struct-of-arrays state block
  uint8_t* state = nullptr;
  size_t state_bytes = 0;
  size_t field_off[JX_F_COUNT] = {};
  size_t field_size[JX_F_COUNT] = {};
  // device error word, turn table, column table, rollout hand-off words
  uint8_t* aux = nullptr;
  size_t work_bytes = 0;
  // maze generation work space, one slot per resident warp
  uint8_t* scratch = nullptr;
  // next-episode block and work slots of the lane-parallel pre-generation
  // (owned mazes of side >= 64), or null
  uint8_t* nx_mem = nullptr;
  // staging buffers of jx_step_host
  uint8_t* stage = nullptr;
  size_t stage_frames_off = 0, stage_rewards_off = 0, stage_dones_off = 0;
  std::atomic<uint64_t> launches{0};
  // jx_autotune: a private one-group batch over this env, and whether the
  // env's launches go through it (the batched kernel with tuned tiles)
  jx_batch* tuned = nullptr;
  bool use_batch = false;
};

namespace jx {

// kernels one pregen_launch launches: the count, the walls and the build
constexpr int kPregenKernels = 3;

namespace host {

extern thread_local std::string g_last_error;

// Records the message for jx_last_error and returns st.
jx_status fail(jx_status st, const char* fmt, ...);
jx_status cuda_fail(cudaError_t err, const char* what);

// Makes a device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit DeviceGuard(int dev) {
    err = cudaGetDevice(&prev);
    if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Uniform random actions of the autotuners: action i = (SplitMix64 output i) * 7 >> 64.
inline uint8_t tune_action(uint64_t i) {
  uint64_t x = i + 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x ^= x >> 31;
  return (uint8_t)(((x >> 32) * 7) >> 32);
}
inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Bytes of one env's RGB frame.
inline size_t frame_bytes(const jx_config& c) { return (size_t)3 * c.frame_h * c.frame_w; }

// The largest frame row block (at most max_rows rows, a multiple of the rows
// one fill pass covers when it is below H) with which `blocks` warps of the
// layout fit in `smem_per_sm` bytes, each block of `warps` warps also taking
// `reserved` bytes. Sets rows_per_block, frame_block_bytes and the layout.
void choose_rows(Params& p, int max_rows, int warps, int blocks, size_t smem_per_sm, size_t reserved);

// jx_env_bytes / jx_create_in, for the ASCII task too (ascii: the map text, or null).
jx_status env_bytes(const jx_config* cfg, const char* ascii, int device, size_t* bytes);
jx_status create_in(const jx_config* cfg, const char* ascii, int device, void* d_mem, size_t bytes, jx_env** out);

}  // namespace host
}  // namespace jx
