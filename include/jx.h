/*
 * jx.h — C ABI of the GB300-native batched first-person environment library.
 *
 * The library steps N independent Wolfenstein-3D-style environments at once
 * and renders one uint8 RGB frame per environment (JAXenstein, arxiv
 * 2605.19926: reset/step environment interface, Sec. 1 and Sec. 3.1; DDA
 * ray casting over a tile map, Sec. 2.1; wall slices shaded from the hit
 * distance, Sec. 2 and Sec. 2.1; fixed sprites, Fig. 1; key / locked door /
 * goal tasks, Table 1 and Table 2; native low-resolution frames, Sec. 3.1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All compute runs in hand-written CUDA kernels on the env's device. There
 *   is no CPU path: every entry point that computes fails with JX_ECUDA when
 *   no usable device is present.
 * - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *   stream. Calls taking device pointers only enqueue work on that stream and
 *   return at once (asynchronous); they never synchronise and never allocate,
 *   so they may be captured into a CUDA graph.
 * - Device pointers (prefix d_) must point to memory on the env's device.
 *   Host pointers (prefix h_) are ordinary or pinned host memory.
 * - The library owns all environment state (positions, headings, maps,
 *   sprites) in device memory; the caller owns its output buffers and streams.
 * - Status codes are returned; nothing traps. A human-readable message for
 *   the last failing call on the calling thread is in jx_last_error().
 * - Kernels that meet bad data (an action outside 0..6) record it in a device
 *   error word and treat the action as a no-op; jx_sync_status reads the word.
 *
 * Frame layout: [N][H][W][3] uint8 (NHWC, RGB), env-major and row-major; one
 * frame is 3*H*W bytes. Frame buffers must be 16-byte aligned.
 */
#ifndef JX_H
#define JX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct jx_env jx_env; /* opaque handle */

typedef enum {
  JX_OK = 0,
  JX_EINVAL = 1,   /* bad argument or configuration */
  JX_ENOMEM = 2,   /* device or host allocation failed */
  JX_ECUDA = 3,    /* a CUDA runtime call failed (no device, launch error, ...) */
  JX_ETIMEOUT = 4, /* a bounded wait gave up */
  JX_EBUDGET = 5,  /* refused by a memory budget */
  JX_EDEVICE = 6   /* the device error word was set by a kernel */
} jx_status;

enum { JX_TASK_ROOMS = 0, JX_TASK_MAZE_KEYDOOR = 1, JX_TASK_MAZE_ROOMS = 2, JX_TASK_ASCII = 3 };

/* Map cell values (JX_F_MAP): 0 floor; 1..9 static walls of colour 1..9;
 * JX_LOCKED + c a locked door and JX_UNLOCKED + c an unlocked door of colour
 * c (0 red, 1 blue, 2 yellow); any other value draws and blocks as wall 1.
 * A locked door is open while the key of its colour is held (Table 2); an
 * unlocked door opens (turns to floor) when the agent walks into it.
 * Sprite types (JX_F_SPR_TYPE): 0 none, 1 red key, 2 goal, 3 distractor,
 * 4 blue key, 5 yellow key. */
enum { JX_LOCKED = 16, JX_UNLOCKED = 20 };

enum {
  JX_ACT_NOOP = 0,
  JX_ACT_FORWARD = 1,
  JX_ACT_BACK = 2,
  JX_ACT_STRAFE_LEFT = 3,
  JX_ACT_STRAFE_RIGHT = 4,
  JX_ACT_TURN_LEFT = 5,
  JX_ACT_TURN_RIGHT = 6
};

/* Environment configuration (one value for all N environments).
 *  n_envs        number of environments N (>= 1)
 *  task          JX_TASK_ROOMS: border walls, interior walls with probability
 *                wall_prob, optional decorative sprites; JX_TASK_MAZE_KEYDOOR:
 *                random DFS maze with one key, one locked door and a goal at
 *                the cell farthest from the spawn (Table 1 "key-door");
 *                JX_TASK_MAZE_ROOMS: that maze with S*S/1024 open 8 x 8 rooms
 *                carved in (the door kept) and 0..K-2 distractor sprites after
 *                the key and the goal; JX_TASK_ASCII: a map given as text,
 *                see jx_create_ascii
 *  map_side      S, the map is S x S cells; rooms: 3..128; mazes: even, 6..128
 *  frame_h       H rows, 1..256
 *  frame_w       W columns, a multiple of 16, 16..256
 *  max_sprites   K sprite slots per env, 0..16 (mazes need >= 2: key and goal)
 *  horizon       episode length limit in steps, 0 = no limit
 *  turns_per_rev a turn action rotates by 2*pi / turns_per_rev (72 = 5 degrees)
 *  wall_prob     interior wall probability of the rooms task, [0, 1]
 *  fov_deg       horizontal field of view in degrees, (0, 180)
 *  move_step     cells moved by one move action, [0, 0.5]
 *  radius        half-size of the agent's collision box, [0, 0.49]
 *  step_reward, key_reward, goal_reward: reward of a step is
 *                step_reward + key_reward [key picked] + goal_reward [goal reached],
 *                rounded once to float32
 *  seed          master seed of all map, spawn and heading draws
 *  gray_stack    nonzero: keep a 4-frame grayscale stack per env in the state
 *                (field JX_F_GRAY, [N][4][H][W] uint8), written in the same
 *                pass as the RGB frame: the frame of episode step t goes to
 *                plane t mod 4 (integer BT.601 luma (77 R + 150 G + 29 B +
 *                128) >> 8 of each pixel), and an episode's first frame to all
 *                four planes. So after step t the planes t, t-1, t-2, t-3
 *                (mod 4) hold the last four frames, the first one repeated
 *                early in an episode.
 *  shading       nonzero: distance shading of walls (Sec. 2.1): each channel
 *                of the wall colour (after the 3/4 of y faces) is scaled by
 *                q / 256, q = 64 + floor(192 min(h, H) / H), h the slice
 *                height in rows. */
typedef struct {
  int32_t n_envs;
  int32_t task;
  int32_t map_side;
  int32_t frame_h;
  int32_t frame_w;
  int32_t max_sprites;
  int32_t horizon;
  int32_t turns_per_rev;
  double wall_prob;
  double fov_deg;
  double move_step;
  double radius;
  double step_reward;
  double key_reward;
  double goal_reward;
  uint64_t seed;
  int32_t gray_stack;
  int32_t shading;
} jx_config;

/* Create N environments on CUDA device `device` and allocate their state in
 * its memory (no episode is generated yet: call jx_reset). The config is
 * validated before any CUDA call, so JX_EINVAL needs no GPU. *out receives
 * the handle, owned by the caller until jx_destroy.
 * Maze tasks (JX_TASK_MAZE_KEYDOOR, JX_TASK_MAZE_ROOMS) with map_side >= 64
 * and a multiple of 4 also reserve a next-episode block (the state without
 * the grayscale stack, plus about 4.4 bytes per maze node per env of work
 * space): in batches of many envs with a horizon, one lane per env builds each
 * env's next episode there while the current one runs, its walk spread over
 * the launches before the horizon (all at once at a reset). Without that
 * memory the env works as for other configs. Results do not depend on it. */
jx_status jx_create(const jx_config* cfg, int device, jx_env** out);

/* jx_create for the ASCII task (cfg->task == JX_TASK_ASCII): the map is the
 * text `ascii` (rows separated by '\n', '\r' ignored) in the top-left corner
 * of an S x S grid of walls, S = cfg->map_side. Symbols (Table 2): '#' wall
 * 1; '1'..'9' wall of that colour; '.' and ' ' floor; 'S' spawn candidate;
 * 'G' goal candidate; 'r', 'b', 'y' red, blue and yellow keys; '"' and '\\'
 * blue and yellow unlocked doors; 'R', 'B', 'Y' red, blue and yellow locked
 * doors; any other printable character a wall of colour 1 + (code mod 9).
 * Every episode starts from this map: spawn uniform over the 'S' cells (over
 * all floor cells when there is none), the keys as sprites on their cells in
 * row-major order, then a goal sprite on one 'G' cell drawn uniformly per
 * episode (none without 'G'). Needs max_sprites >= keys + (1 if any 'G').
 * JX_EINVAL when the text does not fit, holds a control character, more than
 * 16 keys, or no floor. */
jx_status jx_create_ascii(const jx_config* cfg, const char* ascii, int device, jx_env** out);

/* Device bytes jx_create allocates for cfg on `device`: one block holding
 * the state, the per-env tables and the maze work space. Validates cfg like
 * jx_create. */
jx_status jx_env_bytes(const jx_config* cfg, int device, size_t* bytes);

/* jx_create with the env's device block placed in caller memory d_mem
 * (256-byte aligned, at least jx_env_bytes bytes, on `device`) instead of
 * allocated: for callers that manage device memory themselves (the step
 * server's arena). The env never frees d_mem. */
jx_status jx_create_in(const jx_config* cfg, int device, void* d_mem, size_t bytes, jx_env** out);

/* Free the env's device memory and the handle. NULL is accepted. Waits for
 * the env's outstanding work on the device first, unless the env lives in
 * caller memory (jx_create_in) and has no host-step staging, in which case
 * it touches the device not at all. */
jx_status jx_destroy(jx_env* env);

/* Start episode 0 of every environment: generate its map, spawn, heading and
 * sprites from (seed, env index, episode), then render the first frame of
 * each into d_frames ([N][H][W][3]). Asynchronous on `stream`.
 * Paper: the environment interface's reset returning the first observation
 * (Sec. 1, Sec. 3.1); key-door task layout (Table 1, Table 2). */
jx_status jx_reset(jx_env* env, void* stream, uint8_t* d_frames);

/* One environment step of all N environments, fused in one kernel:
 * action -> movement with wall collision -> key pickup / goal -> reward ->
 * episode end -> auto-reset of ended episodes (next episode's map) -> render.
 * Paper: the step of the environment interface, batched over environments
 * (Sec. 1, Sec. 3.1); keys, locked doors and the goal (Table 2); the render
 * as in jx_render (Sec. 2.1, Fig. 1).
 *  d_actions [N] uint8 in 0..6 (see JX_ACT_*), read;
 *  d_frames  [N][H][W][3] uint8, written: the frame after the step (for an
 *            env whose episode ended, the first frame of its next episode);
 *  d_rewards [N] float32, written: the reward of the step just taken;
 *  d_dones   [N] uint8, written: 1 where the step ended the episode.
 * Asynchronous on `stream`; allocates nothing; capturable in a CUDA graph. */
jx_status jx_step(jx_env* env, void* stream, const uint8_t* d_actions, uint8_t* d_frames, float* d_rewards,
                  uint8_t* d_dones);

/* `steps` consecutive calls of jx_step in one kernel launch, for action
 * streams known in advance (uniform random policies, as the paper's speed
 * measurements use, App. A.1; replayed or scripted actions): step t reads
 * d_actions + t*N and writes d_frames + t*N*H*W*3,
 * d_rewards + t*N and d_dones + t*N. The results are identical to the
 * sequence of jx_step calls.
 *  d_actions [steps][N] uint8; d_frames [steps][N][H][W][3] uint8;
 *  d_rewards [steps][N] float32; d_dones [steps][N] uint8.
 * Each env's pose stays in registers and its map in shared memory across the
 * steps. Rollouts of 64 steps or more (envs without a grayscale stack) are cut
 * into chunks of 12 steps that the launch's warps take in turn: a warp that
 * finishes a chunk takes the next free one, of any env, and the chunk after
 * it starts once its env's previous chunk has stored the state (a hand-off
 * through device memory that a late partner cannot stall for more than a
 * bounded wait; bit 2 of the device error word records one that ran out).
 * Asynchronous on `stream`; allocates nothing. steps >= 1. Launches of one
 * env must be ordered on one stream (they share its hand-off words). */
jx_status jx_rollout(jx_env* env, void* stream, const uint8_t* d_actions, int32_t steps, uint8_t* d_frames,
                     float* d_rewards, uint8_t* d_dones);

/* Render the current state of all environments into d_frames (no state
 * change): one DDA ray per screen column over the tile map (Sec. 2.1), a wall
 * slice from the perpendicular hit distance shaded per face (Sec. 2.1),
 * billboard sprites against the per-column depth buffer (Fig. 1), at the
 * frame's native resolution (Sec. 3.1). */
jx_status jx_render(jx_env* env, void* stream, uint8_t* d_frames);

/* jx_step with host buffers: copies h_actions to the device, steps, copies
 * frames, rewards and dones back into the host buffers and waits for the
 * stream. Uses device staging buffers owned by the env (allocated on first
 * use). Host buffers of pinned memory give the fastest copies. */
jx_status jx_step_host(jx_env* env, void* stream, const uint8_t* h_actions, uint8_t* h_frames, float* h_rewards,
                       uint8_t* h_dones);

/* jx_step_host for callers that must not allocate device memory, for example
 * a process whose device memory is already handed out to a framework's
 * caching allocator, or a loop that may not take the implicit
 * synchronisation of a first-use cudaMalloc. It behaves like jx_step_host but
 * stages actions, frames, rewards and dones in a fixed array inside the
 * library (JX_STATIC_STAGING_BYTES per device, kept until the process exits)
 * instead of buffers allocated on first use, and it calls no allocating
 * routine. The paper has no counterpart: this is a deployment convenience of
 * this library.
 *  - Limit: the batch needs N * (3 H W + 6) bytes plus 256-byte alignment of
 *    four buffers; larger batches return JX_EINVAL with the sizes.
 *  - The array of a device is reserved when the first env on that device is
 *    created: jx_create, jx_create_ascii and jx_create_in look up its device
 *    address (cudaGetSymbolAddress), which under CUDA's lazy module loading
 *    is what loads it. So this call itself reserves nothing, and the memory
 *    is taken while the caller can still afford it: create the env before
 *    handing the rest of the device to a caching allocator.
 *  - All calls on a device share the one array, which keeps the last call's
 *    contents; every byte a call reads is written earlier in the same call.
 *    Calls that overlap on the GPU (several envs or threads on different
 *    streams of one device) race on the array: serialise them.
 *  - Waits for `stream` before returning, like jx_step_host. */
#define JX_STATIC_STAGING_BYTES (16u << 20)
jx_status jx_step_host_static(jx_env* env, void* stream, const uint8_t* h_actions, uint8_t* h_frames,
                              float* h_rewards, uint8_t* h_dones);

/* Test and debug hook: the number of mbarrier polls a warp makes before a
 * bulk copy of a byte map (maps of 4 KB or more held as bytes) counts as
 * late (default 65536). A late copy sets bit 2 of the device error word (see
 * jx_sync_status) and is waited for up to a further fixed bound; a copy that
 * does not complete then counts as lost: its warp leaves that env and its
 * later envs of the launch unstepped (their outputs keep old contents) and
 * never reuses the copy's buffer. 0 makes every copy late, exercising that
 * path on a healthy device. Applies to later launches of the env (its own
 * kernel, and its tuned batch). JX_EINVAL for rounds < 0. */
jx_status jx_debug_wait_limit(jx_env* env, int32_t rounds);

/* Test and debug hook: the number of polls a warp makes, in a rollout in
 * hand-off chunks (see jx_rollout), for the warp that ran the previous chunk
 * of an env to publish its state, before the wait counts as late (default
 * 4194304, about a second). A late wait sets bit 2 of the device error word
 * and the chunk runs on whatever state the env holds then, so the results of
 * that launch are undefined; the launch still ends, and later launches start
 * from clean hand-off words. 0 makes every wait late, exercising that path on
 * a healthy device. Applies to later rollouts of the env's own kernel.
 * JX_EINVAL for polls < 0. */
jx_status jx_debug_handoff_limit(jx_env* env, int32_t polls);

/* Per-column ray results of the current state (test and debug hook):
 *  d_hits [N][W][4] int32: hit cell x, hit cell y, side (0: x face, 1: y face),
 *         slice height h in rows;
 *  d_perp [N][W] float32: perpendicular distance of the hit. */
jx_status jx_debug_rays(jx_env* env, void* stream, int32_t* d_hits, float* d_perp);

/* State access (checkpoint / resume and lockstep testing). The state is one
 * device block of struct-of-arrays fields; jx_state_field gives each field's
 * byte offset and size inside it (fields: JX_F_*). jx_get_state copies the
 * whole block to the host and waits; jx_set_state copies it back and waits.
 * `bytes` must equal jx_state_bytes. jx_set_state checks that every position
 * lies inside the map (cell in [0, S), fraction in [0, 1)), that turn lies in
 * [0, turns_per_rev) and the sprite count in [0, K], and returns JX_EINVAL
 * otherwise; it recomputes the derived fields (JX_F_COS0, JX_F_SIN0)
 * from theta0 and leaves the caller's buffer untouched. */
enum {
  JX_F_CELL_X = 0,   /* int16  [N]   cell column of the position            */
  JX_F_CELL_Y = 1,   /* int16  [N]   cell row of the position               */
  JX_F_FRAC_X = 2,   /* float  [N]   x - cell_x in [0, 1)                   */
  JX_F_FRAC_Y = 3,   /* float  [N]   y - cell_y in [0, 1)                   */
  JX_F_THETA0 = 4,   /* float  [N]   heading at episode start (radians)     */
  JX_F_TURN = 5,     /* int16  [N]   heading = theta0 + turn * 2pi/turns_per_rev */
  JX_F_T = 6,        /* int32  [N]   steps taken in the episode             */
  JX_F_EPISODE = 7,  /* uint32 [N]   episode counter                        */
  JX_F_FLAGS = 8,    /* uint8  [N]   keys held: bit 0 red, bit 1 blue, bit 2 yellow */
  JX_F_OBJ = 9,      /* int16  [N][6] key x, key y, goal x, goal y, door x, door y (-1: none) */
  JX_F_NSPR = 10,    /* uint8  [N]   sprites in use                         */
  JX_F_SPR_X = 11,   /* float  [N][K] sprite x (absolute map coordinate)    */
  JX_F_SPR_Y = 12,   /* float  [N][K] sprite y                              */
  JX_F_SPR_TYPE = 13, /* uint8 [N][K] sprite types (above)                 */
  JX_F_MAP = 14,     /* uint8  [N][S][S] cell values (JX_LOCKED, JX_UNLOCKED above) */
  JX_F_COS0 = 15,    /* float  [N]   cos(theta0), derived: jx_set_state recomputes it */
  JX_F_SIN0 = 16,    /* float  [N]   sin(theta0), derived: jx_set_state recomputes it */
  JX_F_GRAY = 17,    /* uint8  [N][4][H][W] grayscale frame stack (0 bytes unless gray_stack) */
  JX_F_COUNT = 18
};
jx_status jx_state_bytes(const jx_env* env, size_t* bytes);
jx_status jx_state_field(const jx_env* env, int32_t field, size_t* offset, size_t* bytes);
jx_status jx_get_state(jx_env* env, void* h_buf, size_t bytes);
jx_status jx_set_state(jx_env* env, const void* h_buf, size_t bytes);

/* Wait for `stream`, then read and clear the device error word: JX_OK, or
 * JX_EDEVICE when a kernel recorded bad data since the last call (bit 0: an
 * action outside 0..6, taken as a no-op; bit 1: a bulk map copy completed
 * late or was lost, see jx_debug_wait_limit; bit 2: a rollout hand-off
 * between warps ran out of its bounded wait, see jx_rollout). */
jx_status jx_sync_status(jx_env* env, void* stream);

/* Number of kernel launches this env has issued since creation. For maze
 * configs with a next-episode block (see jx_create), jx_reset, jx_step and
 * jx_rollout each also launch the three kernels that build episodes ahead (a
 * count, the walls of builds that start, then the build's share of the launch,
 * after a 4-byte cudaMemsetAsync on the same stream; all capturable in a CUDA
 * graph). */
jx_status jx_launch_count(const jx_env* env, uint64_t* count);

/* Launch shape of the fused step kernel: grid blocks, threads per block,
 * dynamic shared memory bytes per block. */
jx_status jx_launch_shape(const jx_env* env, int32_t* grid, int32_t* block, int32_t* smem_bytes);

/* Launch shape of a jx_rollout of `steps` steps: as jx_launch_shape, plus the
 * steps per hand-off chunk (0: every warp runs whole envs). For an env routed
 * through the batched kernel (jx_autotune), the batch's shape and chunk 0.
 * JX_EINVAL for steps < 1. */
jx_status jx_rollout_shape(const jx_env* env, int32_t steps, int32_t* grid, int32_t* block, int32_t* smem_bytes,
                           int32_t* chunk);

/* ------------------------------------------------------------------------
 * Batches: env groups of different map and frame sizes in one launch.
 *
 * A batch ties together G existing envs ("groups"; each is homogeneous, the
 * groups differ in map side, frame size, sprite count, task, seed, ...) and
 * steps all of their environments in ONE launch of a persistent kernel:
 * every warp drains per-group work queues (counters of handed-out envs), the
 * groups taken largest frames first, so warps that finish early move on to
 * the remaining envs. Results are bit-identical to stepping each group alone
 * with jx_step / jx_rollout / jx_reset / jx_render.
 *
 * Layout of a batch's arrays (the batch's env order): group g's envs occupy
 * env indices [env_offset(g), env_offset(g) + n_g) of the action, reward and
 * done arrays, and bytes [frame_offset(g), frame_offset(g) + n_g*3*H_g*W_g)
 * of the frame array, groups in the order given to jx_batch_create. Per step
 * the arrays hold n_envs (jx_batch_info) entries and frame_bytes_per_step
 * bytes; rollouts stack `steps` such steps.
 *
 * The batch references the group envs, it does not own them: they must
 * outlive it, and while a batch launch is in flight their own calls must not
 * run on another stream. Launches of one batch must be ordered on one stream
 * at a time (they share its work-queue counters). */
typedef struct jx_batch jx_batch;
typedef struct jx_graph jx_graph;

/* Tile choices of the batched kernel (set by hand or by jx_batch_autotune).
 *  warps_per_block     envs in flight per thread block: 1, 2 or 4
 *  cols_per_lane       DDA rays each lane marches together per pass: 1 or 2
 *  bits_min_side       maps whose side is >= this (and a multiple of 8) are
 *                      held in shared memory as bit planes (1 bit per cell)
 *                      instead of byte grids; 0 = byte grids for all
 *  max_rows_per_block  frame rows per staged shared-memory block (upper
 *                      bound, 1..64; lowered to fit 28 warps per SM)
 *  staging_buffers     row-block staging buffers per warp: 1 (a block waits
 *                      for the copy-out of the one before; larger blocks fit)
 *                      or 2 (fill one while the other drains) */
typedef struct {
  int32_t warps_per_block;
  int32_t cols_per_lane;
  int32_t bits_min_side;
  int32_t max_rows_per_block;
  int32_t staging_buffers;
} jx_tiling;

/* The fixed tiling (what a single env uses): 1 warp per block, 1 ray per
 * lane, byte maps below side 128, up to 32 rows per block, one staging buffer. */
jx_status jx_tiling_default(jx_tiling* out);

/* Make a batch of n_groups (1..32) distinct envs on one device. tiling NULL
 * = jx_tiling_default. Allocates the queue counters and the maze work space. */
jx_status jx_batch_create(jx_env* const* groups, int32_t n_groups, const jx_tiling* tiling, jx_batch** out);
/* Free the batch (not its groups). NULL is accepted. */
jx_status jx_batch_destroy(jx_batch* batch);
/* Total envs and frame bytes of one step of the batch. */
jx_status jx_batch_info(const jx_batch* batch, int64_t* n_envs, int64_t* frame_bytes_per_step);
/* Offsets of group g (in the order given) in the env and frame arrays. */
jx_status jx_batch_group(const jx_batch* batch, int32_t group, int64_t* env_offset, int64_t* frame_offset);
/* Change / read the tiling. Results do not depend on it, only speed does. */
jx_status jx_batch_set_tiling(jx_batch* batch, const jx_tiling* tiling);
jx_status jx_batch_get_tiling(const jx_batch* batch, jx_tiling* tiling);
/* Launch shape of the batched step kernel: grid, threads per block, dynamic
 * shared memory per block. */
jx_status jx_batch_launch_shape(const jx_batch* batch, int32_t* grid, int32_t* block, int32_t* smem_bytes);
/* Number of batched kernel launches issued since creation (graph replays
 * count their steps; autotuning trials do not count). */
jx_status jx_batch_launch_count(const jx_batch* batch, uint64_t* count);

/* jx_reset / jx_step / jx_rollout / jx_render of every env of every group in
 * one launch each, with the batch's array layout (above). Asynchronous on
 * `stream`; allocate nothing; capturable in a CUDA graph. */
jx_status jx_batch_reset(jx_batch* batch, void* stream, uint8_t* d_frames);
jx_status jx_batch_step(jx_batch* batch, void* stream, const uint8_t* d_actions, uint8_t* d_frames,
                        float* d_rewards, uint8_t* d_dones);
jx_status jx_batch_rollout(jx_batch* batch, void* stream, const uint8_t* d_actions, int32_t steps,
                           uint8_t* d_frames, float* d_rewards, uint8_t* d_dones);
jx_status jx_batch_render(jx_batch* batch, void* stream, uint8_t* d_frames);

/* Autotuner: times every tiling of the search space (warps_per_block 1, 2,
 * 4 x cols_per_lane 1, 2 x bits_min_side 0, 128, 64, 32, 8 x max_rows_per_block
 * 8, 16, 32 x staging_buffers 1, 2; the first max_trials of them, the
 * default first) on this batch
 * and keeps the fastest. mode 0 times `steps` jx_batch_step launches, mode 1
 * one jx_batch_rollout launch of `steps` steps; each trial starts from
 * jx_batch_reset and is timed with CUDA events after one untimed launch.
 * Uses uniform random actions and allocates its own buffers. Every env is
 * RESET (episode 0) when it returns. trials / ms_per_step (optional, room for
 * max_trials entries) receive each trial's tiling and time per step;
 * *n_trials the number run. Waits for `stream`. */
jx_status jx_batch_autotune(jx_batch* batch, void* stream, int32_t mode, int32_t steps, int32_t max_trials,
                            int32_t* n_trials, jx_tiling* trials, float* ms_per_step);

/* Autotuner of a single env: times the env's own kernel (trial 0, reported as
 * the all-zero tiling; for mode 1, the launch jx_rollout makes for `steps`,
 * in hand-off chunks from 64 steps) and the batched kernel over this env alone under every
 * tiling of jx_batch_autotune's search space (the first max_trials - 1), with
 * jx_batch_autotune's protocol, and keeps the fastest: afterwards jx_reset,
 * jx_step, jx_rollout and jx_render of the env launch the chosen kernel
 * (results are identical either way; jx_debug_rays always uses the env's own
 * kernel). Every env is RESET (episode 0) when it returns. Waits for `stream`. */
jx_status jx_autotune(jx_env* env, void* stream, int32_t mode, int32_t steps, int32_t max_trials,
                      int32_t* n_trials, jx_tiling* trials, float* ms_per_step);
/* The env's launch choice: the all-zero tiling for its own kernel, else the
 * batched kernel's tiling. jx_env_set_tiling pins it (all zero: the env's own
 * kernel); a bad tiling returns JX_EINVAL and changes nothing. */
jx_status jx_env_tiling(const jx_env* env, jx_tiling* tiling);
jx_status jx_env_set_tiling(jx_env* env, const jx_tiling* tiling);

/* CUDA graph of `steps` consecutive jx_batch_step launches (step t reads
 * d_actions + t*n_envs and writes step t's slice of d_frames, d_rewards,
 * d_dones, laid out as for jx_batch_rollout). jx_graph_launch replays it on
 * a stream: one submission for all the steps. The graph keeps the batch's
 * tiling and the pointers of the capture; it must not outlive the batch. */
jx_status jx_batch_capture(jx_batch* batch, int32_t steps, const uint8_t* d_actions, uint8_t* d_frames,
                           float* d_rewards, uint8_t* d_dones, jx_graph** out);
jx_status jx_graph_launch(jx_graph* graph, void* stream);
jx_status jx_graph_destroy(jx_graph* graph);

/* ------------------------------------------------------------------------
 * Step server: continuous batching of step requests.
 *
 * Clients (actor groups) open sessions: a session is a group of envs with one
 * config whose state, frames, rewards and dones stay in device memory for the
 * session's life. They submit step requests (one step of all the session's
 * envs, actions from host memory) as they arrive. A dispatcher thread inside
 * the server merges the oldest pending request of every idle session (up to
 * 32 sessions and 2^20 envs per launch) into one launch of the batched
 * persistent kernel (see jx_batch_*), on one of `max_inflight` launch slots,
 * each with its own stream; requests that arrive while launches run go into
 * the next launch on a free slot, so their work overlaps on the device. A
 * session has at most one request on the device; its later requests wait in
 * its FIFO. Results equal those of stepping the session's env alone with
 * jx_step, bit for bit.
 *
 * Admission: sessions live in one device arena of budget_bytes (allocated at
 * creation). jx_server_open returns JX_EBUDGET when the session's block does
 * not fit in the free arena or all max_sessions slots are taken; the block
 * returns to the arena when the session is closed and drained, so a later
 * open succeeds. The server's own launch slots (streams, maze work space,
 * action staging) are allocated outside the budget. */
typedef struct jx_server jx_server;

typedef struct {
  uint64_t requests_submitted;
  uint64_t requests_done;
  uint64_t launches;         /* batched kernel launches */
  uint64_t env_steps;        /* env steps of all launches */
  uint64_t groups_launched;  /* sum over launches of the sessions in the launch */
  uint64_t rejected_opens;   /* JX_EBUDGET answers of jx_server_open */
  uint64_t budget_bytes;
  uint64_t bytes_in_use;
  uint64_t peak_bytes_in_use;
  int32_t sessions_open;
  int32_t peak_sessions;
  int32_t inflight_launches;
  int32_t peak_inflight_launches;
} jx_server_counters;

/* Create a server on `device`: a budget_bytes session arena, max_sessions
 * session slots, max_inflight (1..16) launch slots, maps up to max_map_side,
 * the batched kernel's tiling (NULL = jx_tiling_default). Starts the
 * dispatcher thread. */
jx_status jx_server_create(int device, uint64_t budget_bytes, int32_t max_sessions, int32_t max_inflight,
                           int32_t max_map_side, const jx_tiling* tiling, jx_server** out);
/* Stop the dispatcher, wait for the device, free every session and the arena. */
jx_status jx_server_destroy(jx_server* server);
/* Admit a session of cfg.n_envs envs: create them in the arena and reset
 * them (episode 0; the first frames are in the session's frame buffer when
 * this returns). JX_EBUDGET: no room now (retry after a close). */
jx_status jx_server_open(jx_server* server, const jx_config* cfg, int32_t* session);
/* jx_server_open for the ASCII task: the session's envs play the map `ascii`
 * (see jx_create_ascii). */
jx_status jx_server_open_ascii(jx_server* server, const jx_config* cfg, const char* ascii, int32_t* session);
/* Close a session: no further submits; its memory returns to the arena once
 * its queued requests have run. */
jx_status jx_server_close(jx_server* server, int32_t session);
/* The session's env handle and its device output buffers (frames
 * [n][H][W][3], rewards [n], dones [n]), valid until close. After a request's
 * wait returns they hold that step's results, until the session's next
 * request runs. */
jx_status jx_server_session(jx_server* server, int32_t session, jx_env** env, uint8_t** d_frames,
                            float** d_rewards, uint8_t** d_dones);
/* Queue one step request: h_actions [n] (copied before returning). *ticket
 * identifies it for jx_server_wait. Never blocks on the device. */
jx_status jx_server_submit(jx_server* server, int32_t session, const uint8_t* h_actions, uint64_t* ticket);
/* Wait (at most timeout_s seconds: JX_ETIMEOUT) until the request's step has
 * completed on the device. */
jx_status jx_server_wait(jx_server* server, uint64_t ticket, double timeout_s);
/* Hold (paused != 0) or resume the dispatcher: while held, submitted
 * requests queue and launches already on the device complete. */
jx_status jx_server_pause(jx_server* server, int32_t paused);
jx_status jx_server_stats(jx_server* server, jx_server_counters* out);
/* Move up to `capacity` latencies (seconds from submit to completion seen
 * by the dispatcher) of completed requests, oldest first, into out. */
jx_status jx_server_latencies(jx_server* server, double* out, uint64_t capacity, uint64_t* count);

/* Message of the last failing call on this thread ("" if none). */
const char* jx_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* JX_H */
