// jx_internal.h — parameters shared by the host API (jx_api.cu) and the
// kernels (jx_kernels.cu). Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace jx {

constexpr int kMaxSprites = 16;
constexpr int kBulkWaitRounds = 1 << 16;  // default try_wait polls before a bulk map copy counts as late
constexpr int kMaxSide = 128;
constexpr int kMaxH = 256;
constexpr int kMaxW = 256;
constexpr int kWarpsPerBlock = 2;  // envs in flight per block of the env kernel (shares the per-block smem reserve)
constexpr int kThreads = kWarpsPerBlock * 32;
constexpr int kMaxStaging = 2;  // frame row-block staging buffers per warp: 1 or 2
constexpr int kMinBlocksPerSm = 28;  // register budget: 28 warps resident per SM
constexpr int kHandoffPolls = 1 << 22;  // default polls (about 0.25 us apart) before a rollout hand-off counts as late
constexpr int kHandoffMinSteps = 64;    // rollouts of at least this many steps run in hand-off chunks
constexpr int kHandoffChunk = 12;       // steps per hand-off chunk

enum Mode { MODE_STEP = 0, MODE_RESET = 1, MODE_RENDER = 2, MODE_RAYS = 3, MODE_ROLLOUT = 4 };

// How a warp holds its env's map in shared memory: one byte per cell, or one
// bit per cell (wall or closed door) with the wall type read from the state
// block at a ray's hit. MAP_RUNTIME takes the choice from Params::map_bits.
enum MapKind { MAP_BYTES = 0, MAP_BITS = 1, MAP_RUNTIME = 2 };

// Batched launches over env groups of different sizes.
constexpr int kMaxGroups = 32;
constexpr int kBatchMaxThreads = 128;  // up to 4 warps (envs in flight) per block
constexpr int kBatchMinBlocks = kMinBlocksPerSm * 32 / kBatchMaxThreads;

enum Purpose : uint32_t {
  P_WALL = 1,
  P_SPAWN = 2,
  P_HEADING = 3,
  P_DFS = 4,
  P_KEY = 5,
  P_NSPRITES = 6,
  P_SPRITE_CELL = 7,
  P_ROOM = 8,
  P_GOAL = 9
};

// Device pointers into the struct-of-arrays state block.
struct State {
  int16_t* cell_x;
  int16_t* cell_y;
  float* frac_x;
  float* frac_y;
  float* theta0;
  int16_t* turn;
  int32_t* t;
  uint32_t* episode;
  uint8_t* flags;
  int16_t* obj;  // [N][6]
  uint8_t* nspr;
  float* spr_x;  // [N][K]
  float* spr_y;
  uint8_t* spr_type;
  uint8_t* map;  // [N][S][S]
  float* cos0;   // [N] cos(theta0), derived
  float* sin0;   // [N] sin(theta0), derived
  uint8_t* gray; // [N][4][H][W] grayscale frame stack, or null
};

struct Params {
  State st;
  uint32_t* err;          // device error word
  const float2* turn_cs;  // [turns_per_rev] (cos, sin) of turn * 2 pi / turns_per_rev
  const float* col_k;     // [W] (2 (c + 1/2) / W - 1) * tan(fov / 2)
  uint8_t* gen_scratch;   // [warps][gen_scratch_stride], maze generation work space
  size_t gen_scratch_stride;
  // The next episode of each env, built ahead by the lane-parallel
  // pre-generation kernel (mazes of side >= kPregenMinSide), or all null:
  // the state fields generation writes, the episode number they hold
  // (0xFFFFFFFF: none), and one work slot per env (the build's counters, and
  // a build in progress between launches; zero at creation).
  State nx;
  uint32_t* nx_ep;
  uint8_t* nx_work;
  size_t nx_work_stride;
  uint32_t* nx_words;  // [pregen_lane_words][n]: the walk words of builds in progress
  int32_t nx_lanes;  // lanes of the pre-generation grid (a lane takes envs lane, lane + nx_lanes, ...)
  // nx_count[0]: the envs that need a pre-built episode, nx_count[1]: those
  // whose build starts, counted first (none: the walls or the build kernel
  // returns at once); batches of fewer than nx_min envs are built where
  // episodes start (one lane's build takes longer than a warp's)
  uint32_t* nx_count;
  int32_t nx_min;
  const uint8_t* actions;
  uint8_t* frames;
  float* rewards;
  uint8_t* dones;
  int32_t* dbg_hits;
  float* dbg_perp;
  int32_t n, S, H, W, K, horizon, tpr, task;
  int32_t steps;  // steps of one rollout launch (actions / outputs are [steps][out_stride][...])
  // Rollout hand-off (env kernel, MODE_ROLLOUT, chunk > 0): the launch's steps
  // are cut into chunks of `chunk` steps, and warps take (env, chunk) items in
  // chunk-major order from the counter work[0]; chunk k of env e starts once
  // work[2 + e] == k, which the warp that ran chunk k - 1 stores (0 after the
  // last chunk). work[1] counts the warps that finished; the last one zeroes
  // work[0] and work[1]. chunk == 0: each warp runs whole envs (e = warp,
  // warp + warps, ...).
  uint32_t* work;
  int32_t chunk;
  int32_t handoff_polls;  // polls of a hand-off wait before it counts as late (jx_debug_handoff_limit)
  int32_t out_stride;  // envs per step in the action / reward / done arrays (n, or a batch's total)
  size_t frame_step;   // bytes per step in the frame array (n frames, or a batch's total)
  int32_t map_bits;    // the map is staged as a bit plane (see MapKind)
  int32_t gray;        // the env keeps a grayscale frame stack (st.gray)
  int32_t shading;     // distance shading of wall colours
  // ASCII task: the parsed map [S*S] and its candidate cells: n_spawn spawn
  // cells, n_goal goal cells, n_keys keys (cell * 4 + colour), in that order
  const uint8_t* tmpl;
  const int32_t* cand;
  int32_t n_spawn, n_goal, n_keys;
  int32_t gray_block_bytes;  // rows_per_block * W when gray, else 0
  int32_t rows_per_block;  // rows per staged frame block
  int32_t staging;         // staging buffers per warp (1: each block waits for the last one's copy-out)
  int32_t frame_block_bytes;
  int32_t map_smem_bytes;  // S * S rounded up to 16
  // per-warp shared memory layout (byte offsets from the warp's base; set by layout_warp_smem)
  int32_t off_gray, off_pal, off_map, off_col_rgb, off_col_top, off_col_bot, off_zbuf, off_spr_in, off_spr_a, off_spr_rect,
      off_spr_ty, off_spr_rgb, off_spr_kind, off_order, off_spr_span, off_obj, warp_bytes;
  int32_t bulk_wait_rounds;  // try_wait polls before a bulk map copy counts as late (jx_debug_wait_limit)
  float move, radius, tan_half, inv_tan_half;
  float reward_lut[4];
  uint64_t seed;
  uint64_t wall_thr;  // an interior cell is a wall iff (draw >> 11) < wall_thr
};

// A launch over env groups: warps take envs from per-group work queues, the
// groups in the order given (largest envs first).
struct BatchParams {
  Params g[kMaxGroups];  // per group; actions / outputs already offset to the group's slice
  uint32_t* queue;       // [kMaxGroups + 1] next env per group, warps finished; zero between launches
  int32_t n_groups;
  int32_t warp_bytes;  // per-warp shared memory: the largest group's layout
};

// Fill in the per-warp shared memory layout of p (needs W, K, S, map_bits, frame_block_bytes).
void layout_warp_smem(Params& p);
// Dynamic shared memory bytes of one block.
int block_smem_bytes(const Params& p);
size_t gen_scratch_bytes(int task, int S);
// Lane-parallel pre-generation: for maze tasks of side >= kPregenMinSide (a
// multiple of 4), one lane per env advances the build of the env's next
// episode (reset: episode 0) into p.nx by its share of the launches left
// before the horizon (each launch runs `steps` steps).
constexpr int kPregenMinSide = 64;
constexpr int kPregenThreads = 32;  // pre-generation lanes per block (each with its walk state in shared memory)
constexpr int kPregenLaunches = 20;  // a build's walk goes into at most this many launches
bool pregen_wanted(int task, int S, int horizon);
size_t pregen_work_bytes(int S);
size_t pregen_words_bytes(int S);  // per env: the saved walk words of a build in progress
// Lanes of the pre-generation kernel resident at once on num_sms SMs (its grid).
cudaError_t pregen_resident_lanes(int S, int num_sms, int* lanes);
cudaError_t pregen_launch(const Params& p, int steps, bool reset, cudaStream_t stream);

// Configure (attributes) and query occupancy of the kernel for `mode`.
cudaError_t kernel_blocks_per_sm(const Params& p, int mode, int* blocks);
// Launch the fused kernel for `mode`.
cudaError_t launch(const Params& p, int mode, int grid, cudaStream_t stream);

// The batched kernel: blocks of `warps` warps, `cols` rays marched together per lane;
// spec 1 (every group with bit-plane maps and no grayscale stack) selects a
// specialised instance, 0 the general one (batch_spec gives it for a launch).
int batch_spec(const BatchParams& bp);
cudaError_t batch_blocks_per_sm(int mode, int cols, int spec, int warps, int smem_bytes, int* blocks);
cudaError_t batch_launch(const BatchParams& bp, int mode, int cols, int warps, int grid, cudaStream_t stream);

}  // namespace jx
