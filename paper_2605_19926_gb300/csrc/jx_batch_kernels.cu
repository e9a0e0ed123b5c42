// jx_batch_kernels.cu — the batched kernel (env groups of different sizes in
// one persistent launch over per-group work queues) and its launches.
#include "jx_device.cuh"

namespace jx {
namespace {

// One launch over the groups of a batch. Each group has a work queue (a
// counter of handed-out envs); a warp drains the groups' queues in order,
// one env at a time, fetching its next ticket while it works on the current
// env. The last warp to finish zeroes the counters for the next launch.
// SPEC 0: each group's map kind and grayscale stack as its Params say; SPEC 1:
// every group has bit-plane maps and no grayscale stack (compiled in).
template <int MODE, int COLS, int SPEC>
__global__ void __launch_bounds__(kBatchMaxThreads, kBatchMinBlocks)
    batch_kernel(const __grid_constant__ BatchParams bp) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  uint8_t* const wbase = smem_raw + warp * bp.warp_bytes;
  init_warp_header(wbase, lane);
  const int gw = blockIdx.x * wpb + warp;
  int slot = 0;
  bool fresh = true;  // nothing of an earlier group is pending in the ring
  bool lost = false;  // a map copy of this warp was lost: it takes no further env
  for (int g = 0; g < bp.n_groups && !lost; ++g) {
    const Params& p = bp.g[g];
    uint32_t ticket = 0;
    if (lane == 0) {
      // a drained queue is skipped without an atomic
      ticket = *reinterpret_cast<volatile uint32_t*>(bp.queue + g);
      if (ticket < (uint32_t)p.n) ticket = atomicAdd(bp.queue + g, 1u);
    }
    ticket = __shfl_sync(0xffffffffu, ticket, 0);
    if (ticket >= (uint32_t)p.n) continue;
    if (!fresh && lane == 0) bulk_wait_read_all();  // the layout changes under the ring
    __syncwarp();
    write_palette(p, WarpSmem{wbase, fill_lane(p, lane)}, lane);
    fresh = false;
    slot = 0;
    uint8_t* scratch = p.gen_scratch ? p.gen_scratch + (size_t)gw * p.gen_scratch_stride : nullptr;
    while (ticket < (uint32_t)p.n) {
      uint32_t next = 0;
      if (lane == 0) next = atomicAdd(bp.queue + g, 1u);
      const int e = (int)ticket;
      if (SPEC == 1)
        lost = !run_env<MODE, MAP_BITS, COLS, 0>(p, e, wbase, scratch, lane, slot, 0, p.steps);
      else
        lost = !run_env<MODE, MAP_RUNTIME, COLS, 2>(p, e, wbase, scratch, lane, slot, 0, p.steps);
      if (lost) break;  // the counters are still cleared below: every warp reaches the end
      ticket = __shfl_sync(0xffffffffu, next, 0);
    }
  }
  if (lane == 0) {
    bulk_wait_read_all();
    __threadfence();
    const uint32_t nw = gridDim.x * wpb;
    if (atomicAdd(bp.queue + kMaxGroups, 1u) == nw - 1) {
      for (int g = 0; g < bp.n_groups; ++g) atomicExch(bp.queue + g, 0u);
      atomicExch(bp.queue + kMaxGroups, 0u);
    }
  }
}

template <int MODE>
auto batch_kernel_for(int cols, int spec) {
  if (spec == 1) return cols == 2 ? batch_kernel<MODE, 2, 1> : batch_kernel<MODE, 1, 1>;
  return cols == 2 ? batch_kernel<MODE, 2, 0> : batch_kernel<MODE, 1, 0>;
}

auto batch_kernel_of(int mode, int cols, int spec) {
  switch (mode) {
    case MODE_RESET: return batch_kernel_for<MODE_RESET>(cols, spec);
    case MODE_ROLLOUT: return batch_kernel_for<MODE_ROLLOUT>(cols, spec);
    case MODE_RENDER: return batch_kernel_for<MODE_RENDER>(cols, spec);
    default: return batch_kernel_for<MODE_STEP>(cols, spec);
  }
}
}  // namespace

int batch_spec(const BatchParams& bp) {
  for (int g = 0; g < bp.n_groups; ++g)
    if (!bp.g[g].map_bits || bp.g[g].gray) return 0;
  return 1;
}

cudaError_t batch_blocks_per_sm(int mode, int cols, int spec, int warps, int smem_bytes, int* blocks) {
  auto k = batch_kernel_of(mode, cols, spec);
  cudaError_t err = raise_smem_limit(k);
  if (err != cudaSuccess) return err;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, 32 * warps, smem_bytes);
}

cudaError_t batch_launch(const BatchParams& bp, int mode, int cols, int warps, int grid, cudaStream_t stream) {
  auto k = batch_kernel_of(mode, cols, batch_spec(bp));
  k<<<grid, 32 * warps, (size_t)bp.warp_bytes * warps, stream>>>(bp);
  return cudaGetLastError();
}
}  // namespace jx
