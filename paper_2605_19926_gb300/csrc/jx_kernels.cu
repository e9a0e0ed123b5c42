// jx_kernels.cu — the env kernel (one env config per launch), the kernels
// that build next episodes ahead (a count, then one lane per env), and their
// host side: launch shape queries, launches, the per-warp shared memory layout.
#include "jx_device.cuh"

namespace jx {
namespace {

// ---- rollout hand-off (Params::work): a rollout launch's steps in chunks,
// (env, chunk) items handed out in chunk-major order, so that every warp
// stays busy until the launch's last items: warps of one SM are served
// unequally by the schedulers, and an env bound to a warp for all its steps
// would leave the launch waiting on the slowest warps.

__device__ __forceinline__ uint32_t take_item(const Params& p, int lane) {
  uint32_t v = 0;
  if (lane == 0) v = atomicAdd(p.work, 1u);
  return __shfl_sync(0xffffffffu, v, 0);
}

// Waits until chunk k - 1 of env e is published (work[2 + e] == k). The
// warp that holds it is running: it took the item before this warp took a
// later one, and waits only on earlier items itself. False after
// kHandoffPolls polls.
__device__ __forceinline__ bool await_chunk(const Params& p, int e, uint32_t k) {
  const uint32_t* f = p.work + 2 + e;
  for (int i = 0; i < kHandoffPolls; ++i) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
    if (__all_sync(0xffffffffu, v == k)) return true;
    __nanosleep(200);
  }
  return false;
}

// Publishes a finished chunk of env e: every lane's stores of the state (and
// of a new episode's map, objects and sprites) are visible before the flag.
__device__ __forceinline__ void publish_chunk(const Params& p, int e, uint32_t v, int lane) {
  __threadfence();
  __syncwarp();
  if (lane == 0) asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p.work + 2 + e), "r"(v) : "memory");
}

// Launched as a programmatic dependent of the kernel before it on the stream
// (see launch_mode): a launch may be scheduled while the one before it
// drains, and runs its prologue (the constant palette, the warp header in
// shared memory) meanwhile. griddepcontrol.wait then holds it until every
// earlier kernel on the stream has completed and its writes are visible;
// nothing before the wait reads memory that a kernel writes, or writes global
// memory. The single-step modes release their dependents at once (a step is
// one wave of blocks, so the next step's blocks take the slots the first
// finished ones leave); the long modes release them as their warps finish,
// so that no waiting block holds a slot through a rollout. Without the launch
// attribute these instructions do nothing.
// The end of a launch that hands out work from Params::work: the warp's bulk
// stores have read its shared memory, and the last warp to get here zeroes
// the counters for the next launch.
__device__ __forceinline__ void finish_items(const Params& p, int nw, int lane) {
  if (lane == 0) {
    bulk_wait_read_all();
    __threadfence();
    if (atomicAdd(p.work + 1, 1u) == (uint32_t)nw - 1) {
      atomicExch(p.work, 0u);
      atomicExch(p.work + 1, 0u);
    }
  }
}

template <int MODE, int MAPK, int GRAY>
__global__ void __launch_bounds__(kThreads, kMinBlocksPerSm / kWarpsPerBlock)
    env_kernel(const __grid_constant__ Params p) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  constexpr bool kEarlyRelease = MODE == MODE_STEP || MODE == MODE_RENDER || MODE == MODE_RAYS;
  if (kEarlyRelease) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint8_t* const wbase = smem_raw + warp * p.warp_bytes;
  write_palette(p, WarpSmem{wbase, FillLane{}}, lane);  // a constant table: before the wait
  // the header's mbarrier serves only bulk copies of byte maps of 4 KB or more
  if (!p.map_bits && p.S * p.S >= 4096) init_warp_header(wbase, lane);
  const uint3 pal = make_uint3(0u, 0u, 0u);  // stored above, not per env
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int gw = blockIdx.x * kWarpsPerBlock + warp;
  const int nw = gridDim.x * kWarpsPerBlock;
  uint8_t* scratch = p.gen_scratch ? p.gen_scratch + (size_t)gw * p.gen_scratch_stride : nullptr;
  int slot = 0;
  if (MODE == MODE_ROLLOUT && p.chunk > 0) {
    const uint32_t nch = (uint32_t)((p.steps + p.chunk - 1) / p.chunk);
    const uint32_t items = (uint32_t)p.n * nch;  // below 2^31 (the host caps it)
    bool lost = false;
    for (uint32_t item = take_item(p, lane); item < items;) {
      const uint32_t next = take_item(p, lane);  // its latency overlaps this item
      const int e = (int)(item % (uint32_t)p.n);
      const uint32_t k = item / (uint32_t)p.n;
      if (k > 0 && !await_chunk(p, e, k) && lane == 0) atomicOr(p.err, 4u);
      const int t0 = (int)k * p.chunk, t1 = t0 + p.chunk < p.steps ? t0 + p.chunk : p.steps;
      // after a lost map copy the warp only passes its items on (their envs
      // keep their state; the error word says so) and never touches the ring
      if (!lost) lost = !run_env<MODE, MAPK, 1, GRAY>(p, e, wbase, scratch, lane, slot, pal, false, t0, t1);
      publish_chunk(p, e, k + 1 == nch ? 0u : k + 1, lane);
      item = next;
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    finish_items(p, nw, lane);
    return;
  }
  for (int e = gw; e < p.n; e += nw)
    if (!run_env<MODE, MAPK, 1, GRAY>(p, e, wbase, scratch, lane, slot, pal, false, 0, p.steps))
      break;  // a copy was lost
  if (!kEarlyRelease) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  // shared memory stays allocated until the bulk stores have read it
  if (lane == 0) bulk_wait_read_all();
}

// Whether env e needs a pre-built episode, and which: the one it starts
// soon, or for a reset episode 0, unless the next-episode block holds it
// already. "Soon" spreads the builds of envs whose horizons coincide over the
// last kPregenSpread launches before it, a contiguous part of the envs in
// each (so a warp's lanes build together): env e of part q = e * kPregenSpread
// / n is built once its horizon falls within the next steps * (1 + q) steps.
__device__ __forceinline__ bool pregen_need(const Params& p, int e, int steps, int reset, uint32_t& ep) {
  if (reset) {
    ep = 0;
    return p.nx_ep[e] != 0u;
  }
  ep = p.st.episode[e] + 1;
  const int q = (int)(((int64_t)e * kPregenSpread) / p.n);
  return p.horizon > 0 && p.st.t[e] + steps * (1 + q) >= p.horizon && p.nx_ep[e] != ep;
}

// Counts the envs that need a pre-built episode into *p.nx_count (zeroed before).
__global__ void __launch_bounds__(128) pregen_count_kernel(const __grid_constant__ Params p, int steps, int reset) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t ep;
  const bool need = e < p.n && pregen_need(p, e, steps, reset, ep);
  const uint32_t b = __ballot_sync(0xffffffffu, need);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(p.nx_count, (uint32_t)__popc(b));
}

// Lane-parallel pre-generation: lane i builds, for envs i, i + lanes, ...,
// the episode each needs, when at least nx_min envs need one. Each lane keeps
// its walk's state in shared memory (kPregenThreads lanes a block,
// pregen_lane_words words each: under 48 KB a block for side 128).
__global__ void __launch_bounds__(kPregenThreads) pregen_kernel(const __grid_constant__ Params p, int steps, int reset) {
  extern __shared__ uint32_t pregen_sm[];
  if (*p.nx_count < (uint32_t)p.nx_min) return;  // the whole grid
  const int lane_id = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  // lanes below nx_lanes own a work slot; the loop runs the same iterations
  // in all lanes of a warp (its condition is the warp's first env)
  for (int e = lane_id; e - lane < p.n; e += p.nx_lanes) {
    uint32_t ep = 0;
    const bool need = lane_id < p.nx_lanes && e < p.n && pregen_need(p, e, steps, reset, ep);
    const uint32_t m = __ballot_sync(0xffffffffu, need);
    if (need) {
      gen_maze_lane(p, e, ep, p.nx_work + (size_t)lane_id * p.nx_work_stride, pregen_sm + threadIdx.x, blockDim.x, m);
      p.nx_ep[e] = ep;
    }
  }
}

// The env kernel of a mode for p's map kind and grayscale stack.
template <int MODE>
auto env_kernel_of(const Params& p) {
  if (p.map_bits) return p.gray ? env_kernel<MODE, MAP_BITS, 1> : env_kernel<MODE, MAP_BITS, 0>;
  return p.gray ? env_kernel<MODE, MAP_BYTES, 1> : env_kernel<MODE, MAP_BYTES, 0>;
}

template <int MODE>
cudaError_t blocks_per_sm_mode(const Params& p, int* blocks) {
  auto k = env_kernel_of<MODE>(p);
  cudaError_t err = raise_smem_limit(k);
  if (err != cudaSuccess) return err;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, kThreads, block_smem_bytes(p));
}

// Programmatic stream serialisation: the launch may overlap the tail of the
// kernel before it on the stream up to its griddepcontrol.wait (consecutive
// steps in a CUDA graph then start without a launch gap).
template <int MODE>
cudaError_t launch_mode(const Params& p, int grid, cudaStream_t stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = (size_t)block_smem_bytes(p);
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, env_kernel_of<MODE>(p), p);
}
}  // namespace

void layout_warp_smem(Params& p) {
  const int K = p.K > 0 ? p.K : 1;
  int q = kWarpHeader + p.staging * p.frame_block_bytes;
  auto take = [&](int bytes) {
    const int at = q;
    q += align16(bytes);
    return at;
  };
  p.map_smem_bytes = align16(p.map_bits ? (p.S * p.S + 7) / 8 : p.S * p.S);
  p.off_gray = take(p.staging * p.gray_block_bytes);
  p.off_pal = take(4 * kPaletteWords);
  p.off_map = take(p.map_smem_bytes);
  p.off_col_rgb = take(4 * p.W);
  p.off_col_top = take(p.W);
  p.off_col_bot = take(p.W);
  p.off_zbuf = take(4 * p.W);
  p.off_spr_in = take(16 * K);
  p.off_spr_a = take(16 * K);
  p.off_spr_rect = take(16 * K);
  p.off_spr_ty = take(4 * K);
  p.off_spr_rgb = take(4 * K);
  p.off_spr_kind = take(4 * K);
  p.off_order = take(4 * K);
  p.off_spr_span = take(4 * K);
  p.off_obj = take(4 * 8);
  p.warp_bytes = align16(q);
}

int block_smem_bytes(const Params& p) { return p.warp_bytes * kWarpsPerBlock; }

bool pregen_wanted(int task, int S, int horizon) {
  (void)horizon;  // a reset uses it too
  return (task == 1 || task == 2) && S >= kPregenMinSide && S % 4 == 0;
}

size_t pregen_work_bytes(int S) {
  const size_t n = (size_t)((S - 2) / 2) * ((S - 2) / 2);
  return (4 * n + 16 + 255) & ~(size_t)255;  // discovery and finish counters (uint16, the first 16-byte aligned)
}

cudaError_t pregen_launch(const Params& p, int steps, bool reset, cudaStream_t stream) {
  if (p.nx_ep == nullptr || p.nx_lanes <= 0) return cudaSuccess;
  cudaError_t err = cudaMemsetAsync(p.nx_count, 0, sizeof(uint32_t), stream);
  if (err != cudaSuccess) return err;
  pregen_count_kernel<<<(p.n + 127) / 128, 128, 0, stream>>>(p, steps, reset ? 1 : 0);
  const size_t lane_bytes = (size_t)kPregenThreads * pregen_lane_words(p.S) * sizeof(uint32_t);
  pregen_kernel<<<(p.nx_lanes + kPregenThreads - 1) / kPregenThreads, kPregenThreads, lane_bytes, stream>>>(
      p, steps, reset ? 1 : 0);
  return cudaGetLastError();
}

size_t gen_scratch_bytes(int task, int S) {
  if (task != 1 && task != 2) return 0;
  int nn = (S - 2) / 2;
  return (maze_scratch_bytes(nn * nn) + 255) & ~(size_t)255;
}

cudaError_t kernel_blocks_per_sm(const Params& p, int mode, int* blocks) {
  switch (mode) {
    case MODE_STEP: return blocks_per_sm_mode<MODE_STEP>(p, blocks);
    case MODE_RESET: return blocks_per_sm_mode<MODE_RESET>(p, blocks);
    case MODE_RENDER: return blocks_per_sm_mode<MODE_RENDER>(p, blocks);
    case MODE_ROLLOUT: return blocks_per_sm_mode<MODE_ROLLOUT>(p, blocks);
    default: return blocks_per_sm_mode<MODE_RAYS>(p, blocks);
  }
}

cudaError_t launch(const Params& p, int mode, int grid, cudaStream_t stream) {
  switch (mode) {
    case MODE_STEP: return launch_mode<MODE_STEP>(p, grid, stream);
    case MODE_RESET: return launch_mode<MODE_RESET>(p, grid, stream);
    case MODE_RENDER: return launch_mode<MODE_RENDER>(p, grid, stream);
    case MODE_ROLLOUT: return launch_mode<MODE_ROLLOUT>(p, grid, stream);
    default: return launch_mode<MODE_RAYS>(p, grid, stream);
  }
}
}  // namespace jx
