// jx_kernels.cu — the env kernel (one env config per launch, rollouts in
// hand-off chunks), the kernels that build next episodes ahead (a count, the
// walls of the builds that start, then one lane per env advancing its build),
// and their host side: launch shape queries, launches, the per-warp shared
// memory layout.
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
// p.handoff_polls polls (kHandoffPolls unless a test lowered it).
__device__ __forceinline__ bool await_chunk(const Params& p, int e, uint32_t k) {
  const uint32_t* f = p.work + 2 + e;
  for (int i = 0; i < p.handoff_polls; ++i) {
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
// the counters for the next launch, and the envs' hand-off words too when a
// hand-off ran late (two warps may then have published an env out of order).
__device__ __forceinline__ void finish_items(const Params& p, int nw, int lane) {
  if (lane == 0) {
    bulk_wait_read_all();
    __threadfence();
    if (atomicAdd(p.work + 1, 1u) == (uint32_t)nw - 1) {
      atomicExch(p.work, 0u);
      atomicExch(p.work + 1, 0u);
      if (*reinterpret_cast<volatile uint32_t*>(p.err) & 4u)
        for (int e = 0; e < p.n; ++e) p.work[2 + e] = 0u;
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
      if (!lost) lost = !run_env<MODE, MAPK, 1, GRAY>(p, e, wbase, scratch, lane, slot, t0, t1);
      publish_chunk(p, e, k + 1 == nch ? 0u : k + 1, lane);
      item = next;
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    finish_items(p, nw, lane);
    return;
  }
  for (int e = gw; e < p.n; e += nw)
    if (!run_env<MODE, MAPK, 1, GRAY>(p, e, wbase, scratch, lane, slot, 0, p.steps))
      break;  // a copy was lost
  if (!kEarlyRelease) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  // shared memory stays allocated until the bulk stores have read it
  if (lane == 0) bulk_wait_read_all();
}

// Whether env e needs a pre-built episode, and which: episode 0 at a reset,
// else the one after its current episode (with a horizon, which bounds when it
// starts), unless the next-episode block holds it already.
__device__ __forceinline__ bool pregen_need(const Params& p, int e, int reset, uint32_t& ep) {
  if (reset) {
    ep = 0;
    return p.nx_ep[e] != 0u;
  }
  ep = p.st.episode[e] + 1;
  return p.horizon > 0 && p.nx_ep[e] != ep;
}

// Whether env e's build of episode ep starts over in this launch: no walk of
// that episode is in progress in its work slot.
__device__ __forceinline__ bool pregen_fresh(const Params& p, int e, uint32_t ep) {
  const uint32_t* rec = reinterpret_cast<const uint32_t*>(p.nx_work + (size_t)e * p.nx_work_stride +
                                                          lane_slot(p.S).off_rec);
  return !(rec[1] == 1u && rec[0] == ep);
}

// Counts the envs that need a pre-built episode into nx_count[0], and those
// whose build starts in this launch into nx_count[1] (both zeroed before).
__global__ void __launch_bounds__(128) pregen_count_kernel(const __grid_constant__ Params p, int reset) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t ep = 0;
  const bool need = e < p.n && pregen_need(p, e, reset, ep);
  const bool fresh = need && pregen_fresh(p, e, ep);
  const uint32_t b = __ballot_sync(0xffffffffu, need), f = __ballot_sync(0xffffffffu, fresh);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(p.nx_count, (uint32_t)__popc(b));
  if ((threadIdx.x & 31) == 0 && f) atomicAdd(p.nx_count + 1, (uint32_t)__popc(f));
}

// The walls of the builds that start in this launch, 16 cells a thread (the
// draws of all cells at once, with the GPU's full occupancy; the walk needs
// them laid before its first step).
__global__ void __launch_bounds__(256) pregen_walls_kernel(const __grid_constant__ Params p, int reset) {
  if (p.nx_count[1] == 0u || p.n < p.nx_min) return;  // the whole grid: no build starts
  const int per_env = p.S * p.S / 16;
  const int64_t items = (int64_t)p.n * per_env;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < items;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(idx / per_env);
    uint32_t ep = 0;
    if (pregen_need(p, e, reset, ep) && pregen_fresh(p, e, ep)) lane_walls16(p, e, ep, (int)(idx % per_env) * 16);
  }
}

// Lane-parallel pre-generation, one lane per env (batches of at least nx_min
// envs; smaller ones build where episodes start, where one warp is faster
// than one lane). Each launch advances the build of every env's next episode
// by its share of the walk's steps: the steps left over the launches left
// before the one in which the episode can end at the horizon (that launch
// only takes the entry over), and at least 1 / kPregenLaunches of them; all
// of them at a reset or when one launch is left. The build of an episode is
// so spread over the first launches of the episode before it, and a finished
// entry is published by its episode number (nx_ep). Each lane keeps the walk's words in shared memory while it runs
// (kPregenThreads lanes a block, pregen_lane_words words each: under 48 KB a
// block for side 128) and in the words array between launches.
__global__ void __launch_bounds__(kPregenThreads) pregen_kernel(const __grid_constant__ Params p, int steps, int reset) {
  extern __shared__ uint32_t pregen_sm[];
  if (*p.nx_count == 0u || p.n < p.nx_min) return;  // the whole grid
  const LaneSlot L = lane_slot(p.S);
  const LaneWords W = lane_words(pregen_sm + threadIdx.x, blockDim.x, L);
  const int total = 2 * L.n - 1;
  // a block (one warp) takes 32 consecutive envs at a time, one a lane
  for (int base = blockIdx.x * kPregenThreads; base < p.n; base += gridDim.x * kPregenThreads) {
    const int e = base + (int)threadIdx.x;
    uint32_t ep = 0;
    const bool need = e < p.n && pregen_need(p, e, reset, ep);
    if (__ballot_sync(0xffffffffu, need) == 0u) continue;  // the whole warp
    uint8_t* work = p.nx_work + (size_t)(need ? e : 0) * p.nx_work_stride;
    const uint32_t* rec = reinterpret_cast<const uint32_t*>(work + L.off_rec);
    LaneWalk w{};
    int budget = 0;
    if (need) {
      const bool resume = rec[1] == 1u && rec[0] == ep;
      w = resume ? lane_walk_load(W, work, L, p.nx_words, e, p.n) : lane_walk_begin(p, e, ep, W, work, L);
      int launches = 1;  // the launches left for the remaining steps
      if (!reset) {
        const int left = p.horizon - p.st.t[e];
        launches = left > steps ? (left + steps - 1) / steps - 1 : 1;
      }
      // a build's steps go into at most kPregenLaunches launches after the
      // one that lays its walls (fewer saves and loads of the walk), and
      // always in time for the horizon
      const int share = (total + kPregenLaunches - 1) / kPregenLaunches;
      const int due = (total - w.it + launches - 1) / launches;
      budget = launches > 1 && !resume ? 0 : (share > due ? share : due);
      budget = budget < total - w.it ? budget : total - w.it;
    }
    // the warp's lanes step together (each its own walk), as many rounds as
    // the largest share
    const int rounds = __reduce_max_sync(0xffffffffu, budget);
    const uint64_t kd = stream_key(p.seed, (uint32_t)e, ep, P_DFS);
    uint8_t* smap = p.nx.map + (size_t)(need ? e : 0) * p.S * p.S;
    uint16_t* disc = reinterpret_cast<uint16_t*>(work);
    uint16_t* fin = reinterpret_cast<uint16_t*>(work + L.off_fin);
    for (int k = 0; k < rounds; ++k) {
      __syncwarp();
      if (k < budget) lane_walk_step(p, W, w, kd, smap, disc, fin, L.nn);
    }
    if (need) {
      if (w.it == total) {
        lane_walk_finish(p, e, ep, w, W, pregen_sm + threadIdx.x, blockDim.x, work, L);
        reinterpret_cast<uint32_t*>(work + L.off_rec)[1] = 0u;
        p.nx_ep[e] = ep;  // the entry is complete: read by later kernels only
      } else {
        lane_walk_save(W, w, work, L, ep, p.nx_words, e, p.n);
      }
    }
    __syncwarp();
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

size_t pregen_words_bytes(int S) { return 4 * (size_t)pregen_lane_words(S); }

cudaError_t pregen_resident_lanes(int S, int num_sms, int* lanes) {
  int blocks = 0;
  const size_t lane_bytes = (size_t)kPregenThreads * pregen_lane_words(S) * sizeof(uint32_t);
  cudaError_t err = cudaFuncSetAttribute(pregen_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lane_bytes);
  if (err == cudaSuccess)
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, pregen_kernel, kPregenThreads, lane_bytes);
  *lanes = (blocks > 0 ? blocks : 1) * num_sms * kPregenThreads;
  return err;
}

size_t pregen_work_bytes(int S) {
  // discovery and finish counters (uint16), the saved walk words and record
  return ((size_t)lane_slot(S).bytes + 255) & ~(size_t)255;
}

cudaError_t pregen_launch(const Params& p, int steps, bool reset, cudaStream_t stream) {
  if (p.nx_ep == nullptr || p.nx_lanes <= 0) return cudaSuccess;
  cudaError_t err = cudaMemsetAsync(p.nx_count, 0, 2 * sizeof(uint32_t), stream);
  if (err != cudaSuccess) return err;
  pregen_count_kernel<<<(p.n + 127) / 128, 128, 0, stream>>>(p, reset ? 1 : 0);
  const int64_t wall_blocks = ((int64_t)p.n * (p.S * p.S / 16) + 255) / 256;
  pregen_walls_kernel<<<(unsigned)(wall_blocks < 4096 ? wall_blocks : 4096), 256, 0, stream>>>(p, reset ? 1 : 0);
  const size_t lane_bytes = (size_t)kPregenThreads * pregen_lane_words(p.S) * sizeof(uint32_t);
  pregen_kernel<<<(p.nx_lanes + kPregenThreads - 1) / kPregenThreads, kPregenThreads, lane_bytes, stream>>>(
      p, steps, reset ? 1 : 0);  // nx_lanes: the resident lanes (pregen_resident_lanes)
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
