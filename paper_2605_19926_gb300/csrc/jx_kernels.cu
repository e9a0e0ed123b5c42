// jx_kernels.cu — the fused environment kernel (sm_103a).
//
// One warp owns one environment at a time and walks the whole hot path for
// it: load the struct-of-arrays state, stage the map in shared memory, step
// (movement, collision, key / door / goal, reward, episode end), regenerate
// the map of an ended episode, cast one DDA ray per screen column, project
// the billboard sprites, and write the frame in row blocks that TMA bulk
// copies stream from shared memory to HBM. Warps are independent: no block
// barrier is ever taken, only warp-level synchronisation.
//
// Paper passages: DDA ray casting over the tile map (Sec. 2.1); the wall
// slice from the hit distance, shaded per face (Sec. 2, Sec. 2.1); objects
// as fixed sprites drawn against a depth buffer (Fig. 1); the key-door rules
// (Table 1, Table 2); native low-resolution rendering (Sec. 3.1).
#include <cstdint>

#include "jx_internal.h"

namespace jx {
namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr double kHeadingScale = (2.0 * 3.14159265358979323846) / 16777216.0;  // 2 pi / 2^24
constexpr int kHMax = 1 << 20;
constexpr int kDoor = 5;
constexpr int kSprKey = 1;
constexpr int kSprGoal = 2;
static_assert(kRingBuffers == 2, "bulk wait depth below assumes two staging buffers");

// ------------------------------------------------------------- palette ----
// Colours packed as 0x00BBGGRR so that the low three bytes are R, G, B.
constexpr uint32_t rgb(uint32_t r, uint32_t g, uint32_t b) { return r | (g << 8) | (b << 16); }
constexpr uint32_t shade34(uint32_t c) {  // y faces: each channel scaled by 3/4 (floor)
  return rgb((((c >> 0) & 255) * 3) >> 2, (((c >> 8) & 255) * 3) >> 2, (((c >> 16) & 255) * 3) >> 2);
}
constexpr uint32_t kWall1 = rgb(160, 160, 160);
constexpr uint32_t kWall2 = rgb(64, 160, 64);
constexpr uint32_t kWall3 = rgb(64, 96, 192);
constexpr uint32_t kWall4 = rgb(176, 144, 80);
constexpr uint32_t kDoorRgb = rgb(200, 32, 32);
constexpr uint32_t kCeil = rgb(48, 48, 56);
constexpr uint32_t kFloor = rgb(104, 96, 88);

// [side][cell value]; values above 5 draw as wall type 1
__constant__ uint32_t c_wall[2][8] = {
    {kWall1, kWall1, kWall2, kWall3, kWall4, kDoorRgb, kWall1, kWall1},
    {shade34(kWall1), shade34(kWall1), shade34(kWall2), shade34(kWall3), shade34(kWall4), shade34(kDoorRgb),
     shade34(kWall1), shade34(kWall1)}};
// by sprite type: 1 key, 2 goal, 3 distractor
__constant__ uint32_t c_sprite[4] = {rgb(144, 64, 192), rgb(224, 40, 40), rgb(240, 208, 32), rgb(144, 64, 192)};

// ------------------------------------------------------------ SplitMix64 --
// Steele, Lea & Flood (OOPSLA 2014): output n of the generator seeded with s
// is the 64-bit finaliser applied to s + n * gamma.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t splitmix(uint64_t seed, uint64_t n) { return mix64(seed + n * kGamma); }
// Key of the stream (seed, env, episode, purpose): chained generator outputs.
__device__ __forceinline__ uint64_t stream_key(uint64_t seed, uint32_t env, uint32_t ep, uint32_t purpose) {
  return splitmix(splitmix(splitmix(seed, (uint64_t)env + 1), (uint64_t)ep + 1), (uint64_t)purpose + 1);
}
__device__ __forceinline__ uint64_t draw_at(uint64_t key, uint32_t index) { return splitmix(key, (uint64_t)index + 1); }
// uniform integer below n from the high 32 bits (multiply-shift)
__device__ __forceinline__ uint32_t below32(uint32_t hi, uint32_t n) {
  return (uint32_t)(((uint64_t)hi * (uint64_t)n) >> 32);
}
__device__ __forceinline__ uint32_t below(uint64_t d, uint32_t n) { return below32((uint32_t)(d >> 32), n); }

// ------------------------------------------------------------- bulk copy --
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void bulk_store(void* gdst, const void* ssrc, uint32_t bytes) {
  uint32_t s = (uint32_t)__cvta_generic_to_shared(ssrc);
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(gdst), "r"(s), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}
// all but the newest group have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read_all_but_one() {
  asm volatile("cp.async.bulk.wait_group.read 1;\n" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

// ------------------------------------------------------------- warp smem --
__host__ __device__ __forceinline__ int align16(int x) { return (x + 15) & ~15; }

struct WarpSmem {
  uint8_t* ring;      // kRingBuffers * frame_block_bytes
  uint8_t* map;       // map_smem_bytes
  uint32_t* col_rgb;  // [W]
  uint32_t* col_tb;   // [W] top | bot << 16
  float* zbuf;        // [W]
  float4* spr_a;      // [K] x0, width, top, height (pixels)
  float* spr_ty;      // [K] depth
  uint32_t* spr_rgb;  // [K]
  int32_t* spr_kind;  // [K] type
  int32_t* order;     // [K] visible sprites, far to near
};

__host__ __device__ __forceinline__ int warp_bytes(const Params& p) {
  int b = kRingBuffers * p.frame_block_bytes;
  b += p.map_smem_bytes;
  b += align16(4 * p.W) * 3;
  int K = p.K > 0 ? p.K : 1;
  b += align16(16 * K) + align16(4 * K) * 4;
  return align16(b);
}

__device__ __forceinline__ WarpSmem carve(uint8_t* base, const Params& p) {
  WarpSmem w;
  int K = p.K > 0 ? p.K : 1;
  uint8_t* q = base;
  w.ring = q;
  q += kRingBuffers * p.frame_block_bytes;
  w.map = q;
  q += p.map_smem_bytes;
  w.col_rgb = (uint32_t*)q;
  q += align16(4 * p.W);
  w.col_tb = (uint32_t*)q;
  q += align16(4 * p.W);
  w.zbuf = (float*)q;
  q += align16(4 * p.W);
  w.spr_a = (float4*)q;
  q += align16(16 * K);
  w.spr_ty = (float*)q;
  q += align16(4 * K);
  w.spr_rgb = (uint32_t*)q;
  q += align16(4 * K);
  w.spr_kind = (int32_t*)q;
  q += align16(4 * K);
  w.order = (int32_t*)q;
  return w;
}

// ------------------------------------------------------------ env state ----
struct Env {
  int cx, cy;    // cell of the position
  float fx, fy;  // position inside the cell, [0, 1)
  float th0;
  int turn, t;
  uint32_t ep;
  int has_key;
  int key_x, key_y, goal_x, goal_y, door_x, door_y;
  int nspr;
};

__device__ __forceinline__ Env load_env(const Params& p, int e) {
  Env r;
  const State& st = p.st;
  r.cx = st.cell_x[e];
  r.cy = st.cell_y[e];
  r.fx = st.frac_x[e];
  r.fy = st.frac_y[e];
  r.th0 = st.theta0[e];
  int turn = st.turn[e] % p.tpr;
  r.turn = turn < 0 ? turn + p.tpr : turn;
  r.t = st.t[e];
  r.ep = st.episode[e];
  r.has_key = st.flags[e] & 1;
  const int16_t* o = st.obj + 6 * (size_t)e;
  r.key_x = o[0];
  r.key_y = o[1];
  r.goal_x = o[2];
  r.goal_y = o[3];
  r.door_x = o[4];
  r.door_y = o[5];
  int ns = st.nspr[e];
  r.nspr = ns > p.K ? p.K : ns;
  return r;
}

// heading = theta0 + turn * 2 pi / turns_per_rev, by rotating (cos, sin)(theta0)
__device__ __forceinline__ void heading(const Params& p, const Env& r, float& c, float& s) {
  float s0, c0;
  sincosf(r.th0, &s0, &c0);
  float2 cs = p.turn_cs[r.turn];
  c = fmaf(c0, cs.x, -s0 * cs.y);
  s = fmaf(s0, cs.x, c0 * cs.y);
}

__device__ __forceinline__ void stage_map(const Params& p, int e, uint8_t* smap, int lane) {
  const int n = p.S * p.S;
  const uint8_t* g = p.st.map + (size_t)e * n;
  if ((n & 15) == 0) {
    const uint4* src = reinterpret_cast<const uint4*>(g);
    uint4* dst = reinterpret_cast<uint4*>(smap);
    for (int i = lane; i < (n >> 4); i += 32) dst[i] = src[i];
  } else {
    for (int i = lane; i < n; i += 32) smap[i] = g[i];
  }
  __syncwarp();
}

__device__ __forceinline__ void store_map(const Params& p, int e, const uint8_t* smap, int lane) {
  const int n = p.S * p.S;
  uint8_t* g = p.st.map + (size_t)e * n;
  if ((n & 15) == 0) {
    const uint4* src = reinterpret_cast<const uint4*>(smap);
    uint4* dst = reinterpret_cast<uint4*>(g);
    for (int i = lane; i < (n >> 4); i += 32) dst[i] = src[i];
  } else {
    for (int i = lane; i < n; i += 32) g[i] = smap[i];
  }
}

// ------------------------------------------------------------ generators --
// Index of the r-th cell (row-major) of smap[0..n) satisfying pred, or -1.
template <class Pred>
__device__ __forceinline__ int nth_cell(int n, uint32_t r, int lane, Pred pred) {
  for (int base = 0; base < n; base += 32) {
    int i = base + lane;
    bool f = i < n && pred(i);
    uint32_t b = __ballot_sync(0xffffffffu, f);
    uint32_t c = __popc(b);
    if (r < c) {
      for (uint32_t k = 0; k < r; ++k) b &= b - 1;
      return base + __ffs(b) - 1;
    }
    r -= c;
  }
  return -1;
}

template <class Pred>
__device__ __forceinline__ int count_cells(int n, int lane, Pred pred) {
  int total = 0;
  for (int base = 0; base < n; base += 32) {
    int i = base + lane;
    total += __popc(__ballot_sync(0xffffffffu, i < n && pred(i)));
  }
  return total;
}

// Writes the scalar fields of a fresh episode (lane 0) and all K sprite slots.
__device__ void write_episode_state(const Params& p, int e, uint32_t ep, int cell, const int obj[6], int nspr,
                                    const int* spr_cell, const int* spr_type, int lane) {
  const State& st = p.st;
  const int S = p.S;
  const uint64_t kh = stream_key(p.seed, (uint32_t)e, ep, P_HEADING);
  if (lane == 0) {
    st.cell_x[e] = (int16_t)(cell % S);
    st.cell_y[e] = (int16_t)(cell / S);
    st.frac_x[e] = 0.5f;
    st.frac_y[e] = 0.5f;
    st.theta0[e] = (float)((double)(draw_at(kh, 0) >> 40) * kHeadingScale);
    st.turn[e] = 0;
    st.t[e] = 0;
    st.episode[e] = ep;
    st.flags[e] = 0;
    int16_t* o = st.obj + 6 * (size_t)e;
    for (int k = 0; k < 6; ++k) o[k] = (int16_t)obj[k];
    st.nspr[e] = (uint8_t)nspr;
  }
  for (int k = lane; k < p.K; k += 32) {
    size_t i = (size_t)e * p.K + k;
    if (k < nspr) {
      st.spr_x[i] = (float)(spr_cell[k] % S) + 0.5f;
      st.spr_y[i] = (float)(spr_cell[k] / S) + 0.5f;
      st.spr_type[i] = (uint8_t)spr_type[k];
    } else {
      st.spr_x[i] = 0.f;
      st.spr_y[i] = 0.f;
      st.spr_type[i] = 0;
    }
  }
}

// Rooms: border walls; interior wall iff a 53-bit uniform draw < wall_prob;
// wall type 1 + (draw mod 4); spawn and decorative sprites on uniformly
// chosen free cells (row-major enumeration).
__device__ void gen_rooms(const Params& p, int e, uint32_t ep, uint8_t* smap, int lane) {
  const int S = p.S, n = S * S;
  const uint64_t kw = stream_key(p.seed, (uint32_t)e, ep, P_WALL);
  for (int i = lane; i < n; i += 32) {
    uint64_t u = draw_at(kw, (uint32_t)i);
    int x = i % S, y = i / S;
    bool border = x == 0 || y == 0 || x == S - 1 || y == S - 1;
    bool wall = border || (u >> 11) < p.wall_thr;
    smap[i] = wall ? (uint8_t)(1 + (u & 3)) : (uint8_t)0;
  }
  __syncwarp();
  auto is_free = [&](int i) { return smap[i] == 0; };
  int n_free = count_cells(n, lane, is_free);
  if (n_free == 0) {
    if (lane == 0) smap[(S / 2) * S + S / 2] = 0;
    __syncwarp();
    n_free = 1;
  }
  uint32_t pick = below(draw_at(stream_key(p.seed, (uint32_t)e, ep, P_SPAWN), 0), (uint32_t)n_free);
  int spawn = nth_cell(n, pick, lane, is_free);
  int nspr = 0;
  int spr_cell[kMaxSprites], spr_type[kMaxSprites];
  if (p.K > 0) {
    nspr = (int)below(draw_at(stream_key(p.seed, (uint32_t)e, ep, P_NSPRITES), 0), (uint32_t)p.K + 1);
    const uint64_t kc = stream_key(p.seed, (uint32_t)e, ep, P_SPRITE_CELL);
    for (int k = 0; k < nspr; ++k) {
      uint32_t c = below(draw_at(kc, (uint32_t)k), (uint32_t)n_free);
      spr_cell[k] = nth_cell(n, c, lane, is_free);
      spr_type[k] = 3;
    }
  }
  const int obj[6] = {-1, -1, -1, -1, -1, -1};
  write_episode_state(p, e, ep, spawn, obj, nspr, spr_cell, spr_type, lane);
  __syncwarp();
  store_map(p, e, smap, lane);
  __syncwarp();
}

// Work space of one maze generation in global scratch (n = nodes).
struct MazeScratch {
  uint32_t* rnd;  // [n] high 32 bits of the per-carve draws
  uint16_t* stack;
  uint16_t* parent;
  uint16_t* depth;
  uint16_t* disc;
  uint16_t* fin;
  uint8_t* visited;
};
__host__ __device__ __forceinline__ size_t maze_scratch_bytes(int n) {
  return (size_t)align16(4 * n) + 5 * (size_t)align16(2 * n) + (size_t)align16(n);
}
__device__ __forceinline__ MazeScratch maze_scratch(uint8_t* q, int n) {
  MazeScratch m;
  m.rnd = (uint32_t*)q;
  q += align16(4 * n);
  m.stack = (uint16_t*)q;
  q += align16(2 * n);
  m.parent = (uint16_t*)q;
  q += align16(2 * n);
  m.depth = (uint16_t*)q;
  q += align16(2 * n);
  m.disc = (uint16_t*)q;
  q += align16(2 * n);
  m.fin = (uint16_t*)q;
  q += align16(2 * n);
  m.visited = q;
  return m;
}

// Key-door maze: depth-first backtracker over the nodes at odd coordinates,
// N/E/S/W neighbour order, one draw per carved passage. Because the maze is
// the DFS tree, a node's BFS distance from the spawn is its tree depth, and
// the nodes reachable without crossing the door are those outside the
// subtree below the door (a DFS discovery / finish interval test).
__device__ void gen_maze(const Params& p, int e, uint32_t ep, uint8_t* smap, uint8_t* scratch, int lane) {
  const int S = p.S, n_cells = S * S;
  const int nn = (S - 2) / 2, n = nn * nn;
  MazeScratch m = maze_scratch(scratch, n);
  const uint64_t kw = stream_key(p.seed, (uint32_t)e, ep, P_WALL);
  for (int i = lane; i < n_cells; i += 32) smap[i] = (uint8_t)(1 + (draw_at(kw, (uint32_t)i) & 3));
  const uint64_t kd = stream_key(p.seed, (uint32_t)e, ep, P_DFS);
  for (int j = lane; j < n - 1; j += 32) m.rnd[j] = (uint32_t)(draw_at(kd, (uint32_t)j) >> 32);
  for (int i = lane; i < n; i += 32) m.visited[i] = 0;
  const int start = (int)below(draw_at(stream_key(p.seed, (uint32_t)e, ep, P_SPAWN), 0), (uint32_t)n);
  __syncwarp();
  if (lane == 0) {
    int sp = 0, carved = 0, pushes = 0;
    m.stack[sp++] = (uint16_t)start;
    m.visited[start] = 1;
    m.parent[start] = (uint16_t)start;
    m.depth[start] = 0;
    m.disc[start] = (uint16_t)pushes++;
    smap[(2 * (start / nn) + 1) * S + 2 * (start % nn) + 1] = 0;
    while (sp > 0) {
      int v = m.stack[sp - 1];
      int vx = v % nn, vy = v / nn;
      int cand[4], k = 0;
      if (vy > 0 && !m.visited[v - nn]) cand[k++] = v - nn;
      if (vx < nn - 1 && !m.visited[v + 1]) cand[k++] = v + 1;
      if (vy < nn - 1 && !m.visited[v + nn]) cand[k++] = v + nn;
      if (vx > 0 && !m.visited[v - 1]) cand[k++] = v - 1;
      if (k == 0) {
        m.fin[v] = (uint16_t)pushes;
        --sp;
        continue;
      }
      int w = cand[below32(m.rnd[carved], (uint32_t)k)];
      ++carved;
      int cvx = 2 * vx + 1, cvy = 2 * vy + 1;
      int cwx = 2 * (w % nn) + 1, cwy = 2 * (w / nn) + 1;
      smap[((cvy + cwy) >> 1) * S + ((cvx + cwx) >> 1)] = 0;
      smap[cwy * S + cwx] = 0;
      m.visited[w] = 1;
      m.parent[w] = (uint16_t)v;
      m.depth[w] = (uint16_t)(m.depth[v] + 1);
      m.disc[w] = (uint16_t)pushes++;
      m.stack[sp++] = (uint16_t)w;
    }
  }
  __syncwarp();
  // goal: deepest node, ties to the smallest (row-major) index
  int best_d = -1, best_i = 0x7fffffff;
  for (int i = lane; i < n; i += 32) {
    int d = m.depth[i];
    if (d > best_d) {
      best_d = d;
      best_i = i;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    int od = __shfl_xor_sync(0xffffffffu, best_d, off);
    int oi = __shfl_xor_sync(0xffffffffu, best_i, off);
    if (od > best_d || (od == best_d && oi < best_i)) {
      best_d = od;
      best_i = oi;
    }
  }
  const int goal = best_i;
  // door on edge ceil(m/2) of the m-edge spawn-to-goal path
  const int medges = best_d;
  const int j = (medges + 1) / 2;
  int pj = goal;
  for (int k = 0; k < medges - j; ++k) pj = m.parent[pj];
  const int pj1 = m.parent[pj];
  const int dxc = (2 * (pj % nn) + 1 + 2 * (pj1 % nn) + 1) >> 1;
  const int dyc = (2 * (pj / nn) + 1 + 2 * (pj1 / nn) + 1) >> 1;
  if (lane == 0) smap[dyc * S + dxc] = (uint8_t)kDoor;
  // key: uniform over spawn-side nodes except the spawn
  const int d0 = m.disc[pj], d1 = m.fin[pj];
  auto side = [&](int v) {
    int dv = m.disc[v];
    return v != start && !(dv >= d0 && dv < d1);
  };
  const int n_side = n - (d1 - d0) - 1;
  int key = start;
  if (n_side > 0) {
    uint32_t r = below(draw_at(stream_key(p.seed, (uint32_t)e, ep, P_KEY), 0), (uint32_t)n_side);
    key = nth_cell(n, r, lane, side);
  }
  auto cell_of = [&](int v) { return (2 * (v / nn) + 1) * S + 2 * (v % nn) + 1; };
  const int kc = cell_of(key), gc = cell_of(goal);
  const int obj[6] = {kc % S, kc / S, gc % S, gc / S, dxc, dyc};
  const int spr_cell[2] = {kc, gc};
  const int spr_type[2] = {kSprKey, kSprGoal};
  __syncwarp();
  write_episode_state(p, e, ep, cell_of(start), obj, 2, spr_cell, spr_type, lane);
  store_map(p, e, smap, lane);
  __syncwarp();
}

__device__ __forceinline__ void generate(const Params& p, int e, uint32_t ep, uint8_t* smap, uint8_t* scratch,
                                         int lane) {
  if (p.task == 0)
    gen_rooms(p, e, ep, smap, lane);
  else
    gen_maze(p, e, ep, smap, scratch, lane);
}

// ------------------------------------------------------------------ step ----
__device__ __forceinline__ bool solid(const uint8_t* smap, int S, int x, int y, int has_key) {
  if (x < 0 || y < 0 || x >= S || y >= S) return true;
  int v = smap[y * S + x];
  return v != 0 && !(v == kDoor && has_key);
}

// Box of half-size r centred at (cx + fx, cy + fy) overlaps no solid cell
// (closed intervals).
__device__ __forceinline__ bool box_free(const uint8_t* smap, int S, int cx, float fx, int cy, float fy, float r,
                                         int has_key) {
  int i0 = cx + (int)floorf(fx - r), i1 = cx + (int)floorf(fx + r);
  int j0 = cy + (int)floorf(fy - r), j1 = cy + (int)floorf(fy + r);
  for (int j = j0; j <= j1; ++j)
    for (int i = i0; i <= i1; ++i)
      if (solid(smap, S, i, j, has_key)) return false;
  return true;
}

// keep the position split as an integer cell plus a fraction in [0, 1)
__device__ __forceinline__ void renormalise(int& c, float& f) {
  if (f < 0.f) {
    f += 1.f;
    c -= 1;
    if (f >= 1.f) {  // a tiny negative fraction rounded up to 1
      f = 0.f;
      c += 1;
    }
  } else if (f >= 1.f) {
    f -= 1.f;
    c += 1;
  }
}

// Returns true when the episode ended (the caller regenerates).
__device__ bool step_env(const Params& p, int e, Env& r, const uint8_t* smap, int lane) {
  int a = p.actions[e];
  if (a > 6) {
    if (lane == 0) atomicOr(p.err, 1u);
    a = 0;
  }
  if (a == 5) r.turn = r.turn == 0 ? p.tpr - 1 : r.turn - 1;
  if (a == 6) r.turn = r.turn + 1 == p.tpr ? 0 : r.turn + 1;
  float c, s;
  heading(p, r, c, s);
  const float ms = p.move;
  float dx = 0.f, dy = 0.f;
  if (a == 1) {
    dx = ms * c;
    dy = ms * s;
  } else if (a == 2) {
    dx = -(ms * c);
    dy = -(ms * s);
  } else if (a == 3) {
    dx = ms * s;
    dy = -(ms * c);
  } else if (a == 4) {
    dx = -(ms * s);
    dy = ms * c;
  }
  const int S = p.S;
  const float rad = p.radius;
  float nfx = r.fx + dx;
  if (box_free(smap, S, r.cx, nfx, r.cy, r.fy, rad, r.has_key)) {
    r.fx = nfx;
    renormalise(r.cx, r.fx);
  }
  float nfy = r.fy + dy;
  if (box_free(smap, S, r.cx, r.fx, r.cy, nfy, rad, r.has_key)) {
    r.fy = nfy;
    renormalise(r.cy, r.fy);
  }
  int ev = 0;
  if (!r.has_key && r.key_x >= 0 && r.cx == r.key_x && r.cy == r.key_y) ev |= 1;
  if (r.goal_x >= 0 && r.cx == r.goal_x && r.cy == r.goal_y) ev |= 2;
  if (ev & 1) r.has_key = 1;
  r.t += 1;
  const bool done = (ev & 2) || (p.horizon > 0 && r.t >= p.horizon);
  if (lane == 0) {
    p.rewards[e] = p.reward_lut[ev];
    p.dones[e] = done ? 1 : 0;
    if (!done) {
      const State& st = p.st;
      st.cell_x[e] = (int16_t)r.cx;
      st.cell_y[e] = (int16_t)r.cy;
      st.frac_x[e] = r.fx;
      st.frac_y[e] = r.fy;
      st.turn[e] = (int16_t)r.turn;
      st.t[e] = r.t;
      st.flags[e] = (uint8_t)r.has_key;
    }
  }
  return done;
}

// ---------------------------------------------------------------- render ----
struct Ray {
  int mx, my, sx, sy, kx, ky, side;
  float ax, ay, gx, gy, gxay, gyax;
  bool done;
};

__device__ __forceinline__ void ray_init(Ray& q, const Env& r, float rx, float ry) {
  q.mx = r.cx;
  q.my = r.cy;
  q.sx = rx < 0.f ? -1 : 1;
  q.sy = ry < 0.f ? -1 : 1;
  q.ax = fabsf(rx);
  q.ay = fabsf(ry);
  q.gx = rx < 0.f ? r.fx : 1.f - r.fx;
  q.gy = ry < 0.f ? r.fy : 1.f - r.fy;
  q.gxay = q.gx * q.ay;
  q.gyax = q.gy * q.ax;
  q.kx = q.ky = 0;
  q.side = -1;
  q.done = false;
}

// One DDA crossing: the next x boundary is at t = (kx + gx) / ax, the next y
// boundary at (ky + gy) / ay; compare the cross-multiplied forms.
__device__ __forceinline__ void ray_advance(Ray& q, const uint8_t* smap, int S) {
  float lhs = fmaf((float)q.kx, q.ay, q.gxay);
  float rhs = fmaf((float)q.ky, q.ax, q.gyax);
  bool take_x = q.ay == 0.f || (q.ax != 0.f && lhs < rhs);
  if (take_x) {
    q.mx += q.sx;
    q.kx += 1;
    q.side = 0;
  } else {
    q.my += q.sy;
    q.ky += 1;
    q.side = 1;
  }
  bool out = q.mx < 0 || q.my < 0 || q.mx >= S || q.my >= S;
  q.done = out || smap[q.my * S + q.mx] != 0;
}

__device__ __forceinline__ float ray_perp(const Ray& q) {
  if (q.side == 0) return ((float)(q.kx - 1) + q.gx) / q.ax;
  if (q.side == 1) return ((float)(q.ky - 1) + q.gy) / q.ay;
  return __int_as_float(0x7f800000);  // no hit
}

struct Column {
  int h, top, bot;
  uint32_t rgb;
};

__device__ __forceinline__ Column column_of(const Ray& q, float perp, const uint8_t* smap, int S, int H) {
  Column col;
  int h;
  if (perp > 0.f) {
    float v = (float)H / perp + 0.5f;
    h = v >= 1048576.f ? kHMax : (int)floorf(v);
  } else {
    h = kHMax;
  }
  int top = (H - h) >> 1;  // arithmetic shift: floor division by 2
  int bot = top + h;
  col.h = h;
  col.top = top < 0 ? 0 : (top > H ? H : top);
  col.bot = bot < 0 ? 0 : (bot > H ? H : bot);
  int v = 1;
  if (q.side >= 0 && q.mx >= 0 && q.my >= 0 && q.mx < S && q.my < S) v = smap[q.my * S + q.mx];
  col.rgb = c_wall[q.side == 1 ? 1 : 0][v > 7 ? 7 : v];
  return col;
}

// Cast every column's ray; lanes take columns lane, lane + 32, ...; two rays
// per lane advance together and the warp stops when a ballot says all hit.
template <int MODE>
__device__ void cast_columns(const Params& p, int e, const Env& r, float c, float s, const WarpSmem& ws, int lane) {
  const int W = p.W, S = p.S, H = p.H;
  const uint8_t* smap = ws.map;
  const int max_it = 4 * S + 8;
  for (int base = 0; base < W; base += 64) {
    const int c0 = base + lane, c1 = base + 32 + lane;
    Ray q0, q1;
    const bool v0 = c0 < W, v1 = c1 < W;
    {
      float k = v0 ? p.col_k[c0] : 0.f;
      ray_init(q0, r, fmaf(-k, s, c), fmaf(k, c, s));
      q0.done = !v0;
    }
    {
      float k = v1 ? p.col_k[c1] : 0.f;
      ray_init(q1, r, fmaf(-k, s, c), fmaf(k, c, s));
      q1.done = !v1;
    }
    for (int it = 0; it < max_it; ++it) {
      if (!q0.done) ray_advance(q0, smap, S);
      if (!q1.done) ray_advance(q1, smap, S);
      if (__all_sync(0xffffffffu, q0.done && q1.done)) break;
    }
    if (v0) {
      float perp = ray_perp(q0);
      Column col = column_of(q0, perp, smap, S, H);
      ws.col_rgb[c0] = col.rgb;
      ws.col_tb[c0] = (uint32_t)col.top | ((uint32_t)col.bot << 16);
      ws.zbuf[c0] = perp;
      if (MODE == MODE_RAYS) {
        int4 hv = make_int4(q0.side >= 0 ? q0.mx : -1, q0.side >= 0 ? q0.my : -1, q0.side, col.h);
        reinterpret_cast<int4*>(p.dbg_hits)[(size_t)e * W + c0] = hv;
        p.dbg_perp[(size_t)e * W + c0] = perp;
      }
    }
    if (v1) {
      float perp = ray_perp(q1);
      Column col = column_of(q1, perp, smap, S, H);
      ws.col_rgb[c1] = col.rgb;
      ws.col_tb[c1] = (uint32_t)col.top | ((uint32_t)col.bot << 16);
      ws.zbuf[c1] = perp;
      if (MODE == MODE_RAYS) {
        int4 hv = make_int4(q1.side >= 0 ? q1.mx : -1, q1.side >= 0 ? q1.my : -1, q1.side, col.h);
        reinterpret_cast<int4*>(p.dbg_hits)[(size_t)e * W + c1] = hv;
        p.dbg_perp[(size_t)e * W + c1] = perp;
      }
    }
  }
}

// Project sprites (lane j takes sprite j) and order the visible ones far to
// near (equal depths: higher index first, so the lower index is drawn last).
__device__ int project_sprites(const Params& p, int e, const Env& r, float c, float s, const WarpSmem& ws,
                               int lane) {
  const int W = p.W, H = p.H;
  bool vis = false;
  float ty = 0.f;
  if (lane < r.nspr) {
    size_t i = (size_t)e * p.K + lane;
    int type = p.st.spr_type[i];
    float vx = (p.st.spr_x[i] - (float)r.cx) - r.fx;
    float vy = (p.st.spr_y[i] - (float)r.cy) - r.fy;
    ty = fmaf(vx, c, vy * s);
    float tx = fmaf(-vx, s, vy * c) / p.tan_half;
    vis = type != 0 && !(type == kSprKey && r.has_key) && ty > 0.1f;
    if (vis) {
      float scx = 0.5f * (float)W * (1.f + tx / ty);
      float hw = 0.5f * (float)W * 0.25f / (p.tan_half * ty);
      ws.spr_a[lane] = make_float4(scx - hw, 2.f * hw, 0.5f * (float)H, 0.5f * (float)H / ty);
      ws.spr_ty[lane] = ty;
      ws.spr_rgb[lane] = c_sprite[type & 3];
      ws.spr_kind[lane] = type;
    }
  }
  const uint32_t vmask = __ballot_sync(0xffffffffu, vis);
  int rank = 0;
  for (int k = 0; k < r.nspr; ++k) {
    float tk = __shfl_sync(0xffffffffu, ty, k);
    bool vk = (vmask >> k) & 1;
    if (vis && vk && (tk > ty || (tk == ty && k > lane))) ++rank;
  }
  if (vis) ws.order[rank] = lane;
  __syncwarp();
  return __popc(vmask);
}

__device__ __forceinline__ bool sprite_mask(int kind, float u, float v) {
  float a = fmaf(2.f, u, -1.f), b = fmaf(2.f, v, -1.f);
  if (kind == kSprKey) return fabsf(a) + fabsf(b) < 1.f;
  if (kind == kSprGoal) return true;
  return fmaf(a, a, b * b) < 1.f;
}

// Fill rows [r0, r1) of the frame into `buf` (row-major RGB).
__device__ __forceinline__ void fill_block(const Params& p, const WarpSmem& ws, uint8_t* buf, int r0, int r1,
                                          int nvis, int lane) {
  const int W = p.W, rowb = 3 * W;
  const int lpr = W >> 4;     // lanes per row, 16 pixels (48 bytes) each
  const int rpp = 32 / lpr;   // rows per pass
  const int my_row = lane / lpr, chunk = lane - my_row * lpr;
  if (my_row < rpp) {
    uint32_t crgb[16], ctb[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      crgb[k] = ws.col_rgb[chunk * 16 + k];
      ctb[k] = ws.col_tb[chunk * 16 + k];
    }
    for (int row = r0 + my_row; row < r1; row += rpp) {
      uint32_t px[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        int top = (int)(ctb[k] & 0xffffu), bot = (int)(ctb[k] >> 16);
        px[k] = row < top ? kCeil : (row < bot ? crgb[k] : kFloor);
      }
      uint32_t w[12];
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        w[3 * g + 0] = __byte_perm(px[4 * g + 0], px[4 * g + 1], 0x4210);
        w[3 * g + 1] = __byte_perm(px[4 * g + 1], px[4 * g + 2], 0x5421);
        w[3 * g + 2] = __byte_perm(px[4 * g + 2], px[4 * g + 3], 0x6542);
      }
      uint4* dst = reinterpret_cast<uint4*>(buf + (row - r0) * rowb + chunk * 48);
      dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
      dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
      dst[2] = make_uint4(w[8], w[9], w[10], w[11]);
    }
  }
  __syncwarp();
  // sprites, far to near, each pixel tested at its centre
  for (int oi = 0; oi < nvis; ++oi) {
    const int j = ws.order[oi];
    const float4 a = ws.spr_a[j];
    const float ty = ws.spr_ty[j];
    const uint32_t col_rgb = ws.spr_rgb[j];
    const int kind = ws.spr_kind[j];
    int cA = (int)floorf(fmaxf(a.x - 1.f, -1.f));
    int cB = (int)floorf(fminf(a.x + a.y + 1.f, (float)W));
    int rA = (int)floorf(fmaxf(a.z - 1.f, -1.f));
    int rB = (int)floorf(fminf(a.z + a.w + 1.f, (float)p.H));
    cA = cA < 0 ? 0 : cA;
    cB = cB > W - 1 ? W - 1 : cB;
    rA = rA < r0 ? r0 : rA;
    rB = rB > r1 - 1 ? r1 - 1 : rB;
    if (cA > cB || rA > rB) continue;
    const int ncols = cB - cA + 1;
    const int npx = ncols * (rB - rA + 1);
    for (int i = lane; i < npx; i += 32) {
      int row = rA + i / ncols;
      int col = cA + (i - (row - rA) * ncols);
      float u = ((float)col + 0.5f - a.x) / a.y;
      float v = ((float)row + 0.5f - a.z) / a.w;
      if (u >= 0.f && u < 1.f && v >= 0.f && v < 1.f && sprite_mask(kind, u, v) && ty < ws.zbuf[col]) {
        uint8_t* px = buf + (row - r0) * rowb + col * 3;
        px[0] = (uint8_t)(col_rgb & 255);
        px[1] = (uint8_t)((col_rgb >> 8) & 255);
        px[2] = (uint8_t)((col_rgb >> 16) & 255);
      }
    }
    __syncwarp();
  }
}

template <int MODE>
__device__ void render_env(const Params& p, int e, const Env& r, const WarpSmem& ws, int lane, int& slot) {
  float c, s;
  heading(p, r, c, s);
  cast_columns<MODE>(p, e, r, c, s, ws, lane);
  if (MODE == MODE_RAYS) return;
  const int nvis = project_sprites(p, e, r, c, s, ws, lane);  // ends with __syncwarp
  const int H = p.H, rowb = 3 * p.W;
  uint8_t* frame = p.frames + (size_t)e * H * rowb;
  for (int r0 = 0; r0 < H; r0 += p.rows_per_block) {
    const int r1 = r0 + p.rows_per_block < H ? r0 + p.rows_per_block : H;
    uint8_t* buf = ws.ring + slot * p.frame_block_bytes;
    if (lane == 0) bulk_wait_read_all_but_one();
    __syncwarp();
    fill_block(p, ws, buf, r0, r1, nvis, lane);
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) bulk_store(frame + (size_t)r0 * rowb, buf, (uint32_t)((r1 - r0) * rowb));
    slot ^= 1;
  }
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) env_kernel(const __grid_constant__ Params p) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const WarpSmem ws = carve(smem_raw + warp * warp_bytes(p), p);
  const int gw = blockIdx.x * kWarpsPerBlock + warp;
  const int nw = gridDim.x * kWarpsPerBlock;
  uint8_t* scratch = p.gen_scratch ? p.gen_scratch + (size_t)gw * p.gen_scratch_stride : nullptr;
  int slot = 0;
  for (int e = gw; e < p.n; e += nw) {
    Env r;
    if (MODE == MODE_RESET) {
      generate(p, e, 0u, ws.map, scratch, lane);
      r = load_env(p, e);
    } else {
      r = load_env(p, e);
      stage_map(p, e, ws.map, lane);
      if (MODE == MODE_STEP) {
        if (step_env(p, e, r, ws.map, lane)) {
          const uint32_t ep = r.ep + 1;
          __syncwarp();
          generate(p, e, ep, ws.map, scratch, lane);
          r = load_env(p, e);
        }
      }
    }
    // the locked door opens (for rays) once the key is held
    if (r.has_key && r.door_x >= 0 && r.door_y >= 0 && r.door_x < p.S && r.door_y < p.S) {
      if (lane == 0 && ws.map[r.door_y * p.S + r.door_x] == kDoor) ws.map[r.door_y * p.S + r.door_x] = 0;
      __syncwarp();
    }
    render_env<MODE>(p, e, r, ws, lane, slot);
    __syncwarp();
  }
  if (lane == 0) bulk_wait_all();
}

template <int MODE>
cudaError_t blocks_per_sm_for(const Params& p, int* blocks) {
  int smem = block_smem_bytes(p);
  cudaError_t err = cudaFuncSetAttribute(env_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (err != cudaSuccess) return err;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, env_kernel<MODE>, kThreads, smem);
}

}  // namespace

int warp_smem_bytes(const Params& p) { return warp_bytes(p); }

size_t gen_scratch_bytes(int task, int S) {
  if (task != 1) return 0;
  int nn = (S - 2) / 2;
  return (maze_scratch_bytes(nn * nn) + 255) & ~(size_t)255;
}

cudaError_t kernel_blocks_per_sm(const Params& p, int mode, int* blocks) {
  switch (mode) {
    case MODE_STEP: return blocks_per_sm_for<MODE_STEP>(p, blocks);
    case MODE_RESET: return blocks_per_sm_for<MODE_RESET>(p, blocks);
    case MODE_RENDER: return blocks_per_sm_for<MODE_RENDER>(p, blocks);
    default: return blocks_per_sm_for<MODE_RAYS>(p, blocks);
  }
}

cudaError_t launch(const Params& p, int mode, int grid, cudaStream_t stream) {
  const int smem = block_smem_bytes(p);
  switch (mode) {
    case MODE_STEP: env_kernel<MODE_STEP><<<grid, kThreads, smem, stream>>>(p); break;
    case MODE_RESET: env_kernel<MODE_RESET><<<grid, kThreads, smem, stream>>>(p); break;
    case MODE_RENDER: env_kernel<MODE_RENDER><<<grid, kThreads, smem, stream>>>(p); break;
    default: env_kernel<MODE_RAYS><<<grid, kThreads, smem, stream>>>(p); break;
  }
  return cudaGetLastError();
}

}  // namespace jx
