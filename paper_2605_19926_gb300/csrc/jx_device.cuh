// jx_device.cuh — the device code of the fused environment kernels (sm_103a),
// shared by the env kernel (jx_kernels.cu) and the batched kernel
// (jx_batch_kernels.cu). Everything is internal to each translation unit.
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
#pragma once

#include <cstdint>

#include "jx_internal.h"

namespace jx {
namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr double kHeadingScale = (2.0 * 3.14159265358979323846) / 16777216.0;  // 2 pi / 2^24
constexpr int kHMax = 1 << 20;
constexpr int kLocked = 16;    // + colour (0 red, 1 blue, 2 yellow): locked doors
constexpr int kUnlocked = 20;  // + colour: unlocked doors
constexpr int kDoor = kLocked;  // the red locked door of the generated mazes
constexpr int kTaskAscii = 3;
constexpr int kSprKey = 1;
constexpr int kSprGoal = 2;
constexpr int kSprKeyBlue = 4;
constexpr int kSprKeyYellow = 5;
// colour of a key sprite type, -1 for other types
__host__ __device__ constexpr int key_colour(int type) {
  return type == kSprKey ? 0 : (type == kSprKeyBlue ? 1 : (type == kSprKeyYellow ? 2 : -1));
}
__device__ __forceinline__ bool is_locked(int v) { return (unsigned)(v - kLocked) < 3u; }
__device__ __forceinline__ bool is_unlocked(int v) { return (unsigned)(v - kUnlocked) < 3u; }

// ------------------------------------------------------------- palette ----
// Colours packed as 0xYYBBGGRR: the low three bytes are R, G, B and the top
// byte is the colour's integer BT.601 luma (77 R + 150 G + 29 B + 128) >> 8,
// the pixel's value in the grayscale frame stack.
__host__ __device__ constexpr uint32_t luma(uint32_t r, uint32_t g, uint32_t b) { return (77 * r + 150 * g + 29 * b + 128) >> 8; }
constexpr uint32_t rgb(uint32_t r, uint32_t g, uint32_t b) { return r | (g << 8) | (b << 16) | (luma(r, g, b) << 24); }
constexpr uint32_t shade34(uint32_t c) {  // y faces: each channel scaled by 3/4 (floor), luma of the result
  return rgb((((c >> 0) & 255) * 3) >> 2, (((c >> 8) & 255) * 3) >> 2, (((c >> 16) & 255) * 3) >> 2);
}
constexpr uint32_t kWall1 = rgb(160, 160, 160);
constexpr uint32_t kCeil = rgb(48, 48, 56);
constexpr uint32_t kFloor = rgb(104, 96, 88);

// Colour of a cell value: walls 1..9, locked and unlocked doors by colour,
// anything else as wall 1.
constexpr uint32_t cell_rgb(int v) {
  return v == 2 ? rgb(64, 160, 64)
       : v == 3 ? rgb(64, 96, 192)
       : v == 4 ? rgb(176, 144, 80)
       : v == 5 ? rgb(200, 100, 40)
       : v == 6 ? rgb(112, 64, 160)
       : v == 7 ? rgb(40, 160, 160)
       : v == 8 ? rgb(128, 128, 48)
       : v == 9 ? rgb(216, 216, 216)
       : v == kLocked + 0 ? rgb(200, 32, 32)
       : v == kLocked + 1 ? rgb(32, 64, 200)
       : v == kLocked + 2 ? rgb(208, 184, 32)
       : v == kUnlocked + 0 ? rgb(232, 120, 120)
       : v == kUnlocked + 1 ? rgb(120, 150, 232)
       : v == kUnlocked + 2 ? rgb(236, 222, 128)
       : kWall1;
}
constexpr int kCellColours = 32;  // palette entries per face; values above draw as wall 1
constexpr int kPaletteWords = 2 * kCellColours + 8;

// [face][cell value]: x faces, then y faces (3/4); then the sprite colours by
// type: 1 red key, 2 goal, 3 distractor, 4 blue key, 5 yellow key (others as
// distractor). In global memory, not the constant bank: every lane reads its
// own entries, which the constant cache would serve one address at a time.
#define JX_CELLS(f) f(0), f(1), f(2), f(3), f(4), f(5), f(6), f(7), f(8), f(9), f(10), f(11), f(12), f(13), f(14), \
    f(15), f(16), f(17), f(18), f(19), f(20), f(21), f(22), f(23), f(24), f(25), f(26), f(27), f(28), f(29), f(30), f(31)
#define JX_X_FACE(v) cell_rgb(v)
#define JX_Y_FACE(v) shade34(cell_rgb(v))
__device__ uint32_t g_palette[kPaletteWords] = {
    JX_CELLS(JX_X_FACE), JX_CELLS(JX_Y_FACE),
    rgb(144, 64, 192), rgb(224, 40, 40), rgb(240, 208, 32), rgb(144, 64, 192),
    rgb(40, 80, 224),  rgb(232, 200, 40), rgb(144, 64, 192), rgb(144, 64, 192)};
#undef JX_X_FACE
#undef JX_Y_FACE
#undef JX_CELLS

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
// Frames are written once and never read back here: the copy-out carries an
// L2 evict-first policy, so frame lines are the first to leave L2.
__device__ __forceinline__ void bulk_copy(void* gdst, const void* ssrc, uint32_t bytes) {
  uint32_t s = (uint32_t)__cvta_generic_to_shared(ssrc);
  uint64_t policy;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(policy));
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;\n" ::"l"(gdst), "r"(s),
               "r"(bytes), "l"(policy)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }

// Every warp's shared memory starts with a 16-byte header: the mbarrier that
// bulk global->shared map copies complete on (bytes 0..7), the phase parity
// the next copy waits for (8..11), and 1 once a copy was lost (12..15).
constexpr int kWarpHeader = 16;
constexpr int kBulkDrainLimit = 1 << 22;  // further rounds before a late copy counts as lost

// One bounded round of try_wait polls of the warp's mbarrier for `phase`;
// returns 1 once it has completed.
__device__ __forceinline__ uint32_t bulk_poll(uint32_t bar, uint32_t phase, int rounds, uint32_t done) {
  for (int it = 0; it < rounds && !done; ++it)
    asm volatile("{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n selp.u32 %0, 1, 0, q;\n}\n"
                 : "=r"(done)
                 : "r"(bar), "r"(phase)
                 : "memory");
  return done;
}

__device__ __forceinline__ void init_warp_header(uint8_t* wbase, int lane) {
  if (lane == 0) {
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(wbase);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
    reinterpret_cast<uint32_t*>(wbase)[2] = 0;
    reinterpret_cast<uint32_t*>(wbase)[3] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncwarp();
}

// n bytes (a multiple of 16, both addresses 16-byte aligned) from global
// memory to shared memory with one bulk copy issued by lane 0 and completed
// on the warp's mbarrier. Every lane waits at most first_rounds polls; a copy
// still pending then is late, and the lanes wait up to kBulkDrainLimit more
// polls for it before giving it up: its bytes may still land in `sdst` at any
// time, so the caller must not reuse the buffer (the header records it).
// Returns 0 (in time), 1 (late, complete now) or 2 (lost).
__device__ __forceinline__ int bulk_load(uint8_t* wbase, uint8_t* sdst, const uint8_t* gsrc, uint32_t n, int lane,
                                         int first_rounds) {
  volatile uint32_t* hdr = reinterpret_cast<volatile uint32_t*>(wbase);
  const uint32_t phase = hdr[2];
  const uint32_t bar = (uint32_t)__cvta_generic_to_shared(wbase);
  const uint32_t dst = (uint32_t)__cvta_generic_to_shared(sdst);
  __syncwarp();
  if (lane == 0) {
    // earlier generic-proxy accesses of the destination and the source come first
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("fence.proxy.async.global;\n" ::: "memory");
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(bar),
                 "r"(n)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                 "l"(gsrc), "r"(n), "r"(bar)
                 : "memory");
  }
  uint32_t done = bulk_poll(bar, phase, first_rounds, 0u);
  int state = 0;
  if (!__all_sync(0xffffffffu, done != 0)) {
    done = bulk_poll(bar, phase, kBulkDrainLimit, done);
    state = __all_sync(0xffffffffu, done != 0) ? 1 : 2;
  }
  if (lane == 0) {
    hdr[2] = phase ^ 1u;
    if (state == 2) hdr[3] = 1u;
  }
  __syncwarp();
  return state;
}
// the staging buffer about to be filled has been read out: with two buffers
// the other one may still be draining, with one every earlier copy is done
__device__ __forceinline__ void bulk_wait_staging(int staging) {
  if (staging == 1)
    asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
  else
    asm volatile("cp.async.bulk.wait_group.read 1;\n" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}

// ------------------------------------------------------------- warp smem --
__host__ __device__ __forceinline__ int align16(int x) { return (x + 15) & ~15; }

// Shared memory of a warp, addressed from one base with the layout offsets
// of Params (constants), so no pointer lives in a register:
//   header    16 bytes: the map-copy mbarrier and its phase (see kWarpHeader)
//   ring      staging * frame_block_bytes (also the maze work space)
//   gray      staging * gray_block_bytes: the row blocks of the grayscale frame
//   pal       [2][32] wall colours by face and cell value, then [8] sprite colours by type
//   map       S * S cell values, row-major
//   col_rgb   [W] wall colour, chunk-interleaved (see col_slot)
//   col_top   [W] bytes: 127 + first wall row (at most H/2), by column
//   col_bot   [W] bytes: 127 + first floor row - H/2 (at least 0), by column
//   zbuf      [W] perpendicular distance by column
//   spr_in    [K] float4 sprite x, y, type (as float)
//   spr_a     [K] float4 x0, top, 1 / width, 1 / height (pixels)
//   spr_rect  [K] int4 pixel rectangle to test: first/last column, first/last row
//   spr_ty    [K] depth;  spr_rgb [K] colour;  spr_kind [K] type
//   order     [K] visible sprites, far to near
//   spr_span  [K] first row << 16 | last row the oi-th sprite of that order can cover
//   obj       [8] int32 key x, key y, goal x, goal y, door x, door y, sprites in use
// The lane's place in the frame fill: lanes [0, groups * rows) are laid out
// as `rows` rows of `groups` 16-pixel groups (48 bytes: three 16-byte stores).
struct FillLane {
  int groups, rows, my_row, g;
};
__device__ __forceinline__ FillLane fill_lane(const Params& p, int lane) {
  FillLane f;
  f.groups = p.W >> 4;
  f.rows = 32 / f.groups;
  f.my_row = lane / f.groups;
  f.g = lane - f.my_row * f.groups;
  return f;
}

struct WarpSmem {
  uint8_t* base;
  FillLane fl;
  __device__ __forceinline__ uint8_t* ring() const { return base + kWarpHeader; }
  __device__ __forceinline__ uint8_t* gray_ring(const Params& p) const { return base + p.off_gray; }
  __device__ __forceinline__ uint32_t* pal(const Params& p) const { return (uint32_t*)(base + p.off_pal); }
  __device__ __forceinline__ uint8_t* map(const Params& p) const { return base + p.off_map; }
  __device__ __forceinline__ uint32_t* col_rgb(const Params& p) const { return (uint32_t*)(base + p.off_col_rgb); }
  __device__ __forceinline__ uint8_t* col_top(const Params& p) const { return base + p.off_col_top; }
  __device__ __forceinline__ uint8_t* col_bot(const Params& p) const { return base + p.off_col_bot; }
  __device__ __forceinline__ float* zbuf(const Params& p) const { return (float*)(base + p.off_zbuf); }
  __device__ __forceinline__ float4* spr_in(const Params& p) const { return (float4*)(base + p.off_spr_in); }
  __device__ __forceinline__ float4* spr_a(const Params& p) const { return (float4*)(base + p.off_spr_a); }
  __device__ __forceinline__ int4* spr_rect(const Params& p) const { return (int4*)(base + p.off_spr_rect); }
  __device__ __forceinline__ float* spr_ty(const Params& p) const { return (float*)(base + p.off_spr_ty); }
  __device__ __forceinline__ uint32_t* spr_rgb(const Params& p) const { return (uint32_t*)(base + p.off_spr_rgb); }
  __device__ __forceinline__ int32_t* spr_kind(const Params& p) const { return (int32_t*)(base + p.off_spr_kind); }
  __device__ __forceinline__ int32_t* order(const Params& p) const { return (int32_t*)(base + p.off_order); }
  __device__ __forceinline__ uint32_t* spr_span(const Params& p) const { return (uint32_t*)(base + p.off_spr_span); }
  __device__ __forceinline__ int32_t* obj(const Params& p) const { return (int32_t*)(base + p.off_obj); }
};

// Column data is stored so that the lanes filling one row (16 columns each)
// read consecutive 16-byte groups: quad q (columns 4q..4q+3 of the group) of
// column group c sits at word (q * groups + c) * 4.
__device__ __forceinline__ int col_slot(int col, int groups) {
  const int c = col >> 4, j = col & 15;
  return (((j >> 2) * groups + c) << 2) | (j & 3);
}

// The palette words of this lane: entries lane, 32 + lane and 64 + (lane & 7).
__device__ __forceinline__ uint3 load_palette(int lane) {
  return make_uint3(__ldg(g_palette + lane), __ldg(g_palette + 32 + lane), __ldg(g_palette + 64 + (lane & 7)));
}
__device__ __forceinline__ void store_palette(const Params& p, const WarpSmem& ws, const uint3& w, int lane) {
  ws.pal(p)[lane] = w.x;
  ws.pal(p)[32 + lane] = w.y;
  if (lane < 8) ws.pal(p)[64 + lane] = w.z;
}
__device__ __forceinline__ void write_palette(const Params& p, const WarpSmem& ws, int lane) {
  store_palette(p, ws, load_palette(lane), lane);
  __syncwarp();
}

// ------------------------------------------------------------ env state ----
// The scalar state of the env a warp is working on (identical in all lanes).
// Key, goal and door cells and the sprite table live in the warp's shared
// memory instead (see load_objects).
struct Env {
  int cx, cy;    // cell of the position
  float fx, fy;  // position inside the cell, [0, 1)
  float c0, s0;  // cos, sin of theta0
  int turn, t;
  int keys;  // keys held: bit c for colour c
};

__device__ __forceinline__ Env load_env(const Params& p, int e) {
  Env r;
  const State& st = p.st;
  r.cx = st.cell_x[e];
  r.cy = st.cell_y[e];
  r.fx = st.frac_x[e];
  r.fy = st.frac_y[e];
  r.c0 = st.cos0[e];
  r.s0 = st.sin0[e];
  r.turn = st.turn[e];  // in [0, turns_per_rev): generated so, checked by set_state
  r.t = st.t[e];
  r.keys = st.flags[e] & 7;
  return r;
}

// Key / goal / door cells (lanes 0..5) and sprite slots (lane j: slot j) into
// the warp's shared memory.
__device__ __forceinline__ void load_objects(const Params& p, const WarpSmem& ws, int e, int lane) {
  if (lane < 6) ws.obj(p)[lane] = p.st.obj[6 * (size_t)e + lane];
  if (lane == 6) {
    const int ns = p.st.nspr[e];
    ws.obj(p)[6] = ns > p.K ? p.K : ns;  // sprites in use
  }
  if (lane < p.K) {
    const size_t i = (size_t)e * p.K + lane;
    ws.spr_in(p)[lane] = make_float4(p.st.spr_x[i], p.st.spr_y[i], (float)p.st.spr_type[i], 0.f);
  }
}

// heading = theta0 + turn * 2 pi / turns_per_rev: (cos, sin)(theta0), kept in
// the state, rotated by the table entry of `turn`
__device__ __forceinline__ void heading_from(const Env& r, float2 cs, float& c, float& s) {
  c = fmaf(r.c0, cs.x, -r.s0 * cs.y);
  s = fmaf(r.s0, cs.x, r.c0 * cs.y);
}
__device__ __forceinline__ void heading(const Params& p, const Env& r, float& c, float& s) {
  heading_from(r, p.turn_cs[r.turn], c, s);
}

// Byte maps of 4 KB or more (side >= 64) are copied by one bulk copy, smaller
// ones by 16-byte loads of all lanes. The warp header is read only on the
// bulk path (kernels initialise it only where maps of that size occur). A
// late copy sets bit 2 of the error word; a lost one also returns false: the
// warp then leaves the env (and any later env) untouched.
__device__ __forceinline__ bool stage_map(const Params& p, int e, uint8_t* smap, int lane) {
  const int n = p.S * p.S;
  const uint8_t* g = p.st.map + (size_t)e * n;
  uint8_t* wbase = smap - p.off_map;
  if (n >= 4096 && (n & 15) == 0) {
    if (reinterpret_cast<volatile uint32_t*>(wbase)[3] != 0) return false;  // an earlier copy was lost
    const int st = bulk_load(wbase, smap, g, (uint32_t)n, lane, p.bulk_wait_rounds);
    if (st != 0 && lane == 0) atomicOr(p.err, 2u);
    return st != 2;
  }
  if ((n & 15) == 0) {
    const uint4* src = reinterpret_cast<const uint4*>(g);
    uint4* dst = reinterpret_cast<uint4*>(smap);
    for (int i = lane; i < (n >> 4); i += 32) dst[i] = src[i];
  } else {
    for (int i = lane; i < n; i += 32) smap[i] = g[i];
  }
  __syncwarp();
  return true;
}

__device__ __forceinline__ void store_map(const Params& p, int e, const uint8_t* smap, int lane) {
  const int n = p.S * p.S;
  uint8_t* g = p.st.map + (size_t)e * n;
  if (smap == g) return;  // generated in place
  if ((n & 15) == 0) {
    const uint4* src = reinterpret_cast<const uint4*>(smap);
    uint4* dst = reinterpret_cast<uint4*>(g);
    for (int i = lane; i < (n >> 4); i += 32) dst[i] = src[i];
  } else {
    for (int i = lane; i < n; i += 32) g[i] = smap[i];
  }
}

// bit k of the result is set iff byte k of x is nonzero
__device__ __forceinline__ uint32_t nonzero4(uint32_t x) {
  const uint32_t m = __vcmpne4(x, 0u) & 0x01010101u;
  return (m * 0x10204080u) >> 28;  // gathers bits 0, 8, 16, 24 into bits 28..31
}

// The map as a bit plane: bit i of word i / 32 is set iff cell i is nonzero
// (S * S is a multiple of 32; rows run on across word boundaries).
// The bytes are read from `src` (16-byte aligned; the state block's map when null).
__device__ __forceinline__ void stage_map_bits(const Params& p, int e, uint8_t* smap, int lane,
                                               const uint8_t* src = nullptr) {
  const int words = (p.S * p.S) >> 5;
  const uint4* g = reinterpret_cast<const uint4*>(src ? src : p.st.map + (size_t)e * p.S * p.S);
  uint32_t* w = reinterpret_cast<uint32_t*>(smap);
  for (int i = lane; i < words; i += 32) {
    const uint4 a = g[2 * i], b = g[2 * i + 1];
    w[i] = nonzero4(a.x) | nonzero4(a.y) << 4 | nonzero4(a.z) << 8 | nonzero4(a.w) << 12 | nonzero4(b.x) << 16 |
           nonzero4(b.y) << 20 | nonzero4(b.z) << 24 | nonzero4(b.w) << 28;
  }
  __syncwarp();
}

template <int MAPK>
__device__ __forceinline__ bool map_bits(const Params& p) {
  return MAPK == MAP_BITS || (MAPK == MAP_RUNTIME && p.map_bits != 0);
}

// cell i of the staged map blocks movement and rays (in bit mode the door's
// bit is cleared while the key is held, see open_door)
template <int MAPK>
__device__ __forceinline__ bool cell_set(const Params& p, const uint8_t* smap, int i) {
  if (map_bits<MAPK>(p)) return (reinterpret_cast<const uint32_t*>(smap)[i >> 5] >> (i & 31)) & 1u;
  return smap[i] != 0;
}

template <int MAPK>
__device__ __forceinline__ bool stage(const Params& p, int e, uint8_t* smap, int lane) {
  if (map_bits<MAPK>(p)) {
    stage_map_bits(p, e, smap, lane);
    return true;
  }
  return stage_map(p, e, smap, lane);
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

// Writes the scalar fields of a fresh episode (lane 0) and all K sprite slots
// (lanes lane, lane + kstep, ...) into st: the state, or the next-episode block.
__device__ void write_episode_state(const Params& p, const State& st, int e, uint32_t ep, int cell, const int obj[6],
                                    int nspr, const int* spr_cell, const int* spr_type, int lane, int kstep) {
  const int S = p.S;
  const uint64_t kh = stream_key(p.seed, (uint32_t)e, ep, P_HEADING);
  if (lane == 0) {
    st.cell_x[e] = (int16_t)(cell % S);
    st.cell_y[e] = (int16_t)(cell / S);
    st.frac_x[e] = 0.5f;
    st.frac_y[e] = 0.5f;
    const float th0 = (float)((double)(draw_at(kh, 0) >> 40) * kHeadingScale);
    double sd, cd;
    sincos((double)th0, &sd, &cd);
    st.theta0[e] = th0;
    st.cos0[e] = (float)cd;
    st.sin0[e] = (float)sd;
    st.turn[e] = 0;
    st.t[e] = 0;
    st.episode[e] = ep;
    st.flags[e] = 0;
    int16_t* o = st.obj + 6 * (size_t)e;
    for (int k = 0; k < 6; ++k) o[k] = (int16_t)obj[k];
    st.nspr[e] = (uint8_t)nspr;
  }
  for (int k = lane; k < p.K; k += kstep) {
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
__device__ __forceinline__ void gen_rooms(const Params& p, int e, uint32_t ep, uint8_t* smap, int lane) {
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
  write_episode_state(p, p.st, e, ep, spawn, obj, nspr, spr_cell, spr_type, lane, 32);
  __syncwarp();
  store_map(p, e, smap, lane);
  __syncwarp();
}

// Work space of one maze generation (n = nodes): the per-carve draws, the
// DFS stack of node cells, and each node's DFS discovery / finish counters.
struct MazeScratch {
  uint32_t* rnd;     // [n] high 32 bits of the per-carve draws
  uint16_t* stack;   // [n] node cells packed as y << 8 | x
  uint16_t* disc;    // [n] push counter when the node was discovered
  uint16_t* fin;     // [n] push counter when the node was finished
  int32_t* result;   // [4] goal node, its depth, the door's two path nodes (packed cells)
};
__host__ __device__ __forceinline__ size_t maze_scratch_bytes(int n) {
  return (size_t)align16(4 * n) + 3 * (size_t)align16(2 * n) + 16;
}
__device__ __forceinline__ MazeScratch maze_scratch(uint8_t* q, int n) {
  MazeScratch m;
  m.rnd = (uint32_t*)q;
  q += align16(4 * n);
  m.stack = (uint16_t*)q;
  q += align16(2 * n);
  m.disc = (uint16_t*)q;
  q += align16(2 * n);
  m.fin = (uint16_t*)q;
  q += align16(2 * n);
  m.result = (int32_t*)q;
  return m;
}

// Key-door maze: depth-first backtracker over the nodes at odd coordinates,
// N/E/S/W neighbour order, one draw per carved passage. A node is unvisited
// while its cell is still a wall. Because the maze is the DFS tree, a node's
// BFS distance from the spawn is its stack depth when pushed, and the stack at
// that moment is its path from the spawn: the goal (deepest node, ties to
// the smallest row-major index) and the two path nodes around the door are
// recorded during the walk. The nodes reachable without crossing the door are
// those outside the door's subtree (a discovery / finish interval test).
__device__ __forceinline__ void gen_maze(const Params& p, int e, uint32_t ep, uint8_t* smap, uint8_t* scratch, int lane) {
  const int S = p.S, n_cells = S * S;
  const int nn = (S - 2) / 2, n = nn * nn;
  MazeScratch m = maze_scratch(scratch, n);
  const uint64_t kw = stream_key(p.seed, (uint32_t)e, ep, P_WALL);
  for (int i = lane; i < n_cells; i += 32) smap[i] = (uint8_t)(1 + (draw_at(kw, (uint32_t)i) & 3));
  const uint64_t kd = stream_key(p.seed, (uint32_t)e, ep, P_DFS);
  for (int j = lane; j < n - 1; j += 32) m.rnd[j] = (uint32_t)(draw_at(kd, (uint32_t)j) >> 32);
  const int start = (int)below(draw_at(stream_key(p.seed, (uint32_t)e, ep, P_SPAWN), 0), (uint32_t)n);
  __syncwarp();
  if (lane == 0) {
    int vx = 2 * (start % nn) + 1, vy = 2 * (start / nn) + 1, v = start;
    smap[vy * S + vx] = 0;
    int sp = 0, pushes = 0, carved = 0;
    m.stack[sp++] = (uint16_t)(vy << 8 | vx);
    m.disc[v] = (uint16_t)pushes++;
    int best_v = start, best_d = 0, door_a = vy << 8 | vx, door_b = door_a;
    for (;;) {
      const int c = vy * S + vx;
      const uint32_t open = (uint32_t)(vy > 1 && smap[c - 2 * S] != 0) | ((uint32_t)(vx < S - 3 && smap[c + 2] != 0) << 1) |
                            ((uint32_t)(vy < S - 3 && smap[c + 2 * S] != 0) << 2) |
                            ((uint32_t)(vx > 1 && smap[c - 2] != 0) << 3);
      if (open == 0) {
        m.fin[v] = (uint16_t)pushes;
        if (--sp == 0) break;
        const int top = m.stack[sp - 1];
        vx = top & 0xff;
        vy = top >> 8;
        v = (vy >> 1) * nn + (vx >> 1);
        continue;
      }
      // the r-th unvisited neighbour in N, E, S, W order
      uint32_t bits = open;
      for (uint32_t r = below32(m.rnd[carved++], (uint32_t)__popc(open)); r > 0; --r) bits &= bits - 1;
      const int d = __ffs(bits) - 1;
      const int dx = d == 1 ? 1 : (d == 3 ? -1 : 0), dy = d == 0 ? -1 : (d == 2 ? 1 : 0);
      smap[c + dy * S + dx] = 0;
      vx += 2 * dx;
      vy += 2 * dy;
      smap[vy * S + vx] = 0;
      v = (vy >> 1) * nn + (vx >> 1);
      const int depth = sp;
      m.stack[sp++] = (uint16_t)(vy << 8 | vx);
      m.disc[v] = (uint16_t)pushes++;
      if (depth > best_d || (depth == best_d && v < best_v)) {
        best_v = v;
        best_d = depth;
        const int j = (depth + 1) / 2;  // the door sits on edge ceil(depth / 2) of the path
        door_a = m.stack[j - 1];
        door_b = m.stack[j];
      }
    }
    m.result[0] = best_v;
    m.result[1] = best_d;
    m.result[2] = door_a;
    m.result[3] = door_b;
  }
  __syncwarp();
  const int goal = m.result[0];
  const int door_a = m.result[2], door_b = m.result[3];
  const int dxc = ((door_a & 0xff) + (door_b & 0xff)) >> 1, dyc = ((door_a >> 8) + (door_b >> 8)) >> 1;
  if (lane == 0) smap[dyc * S + dxc] = (uint8_t)kDoor;
  // key: uniform over spawn-side nodes except the spawn
  const int pj = ((door_b >> 8) >> 1) * nn + ((door_b & 0xff) >> 1);
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
  int spr_cell[kMaxSprites], spr_type[kMaxSprites];
  spr_cell[0] = kc;
  spr_type[0] = kSprKey;
  spr_cell[1] = gc;
  spr_type[1] = kSprGoal;
  int nspr = 2;
  if (p.task == 2) {
    // open 8 x 8 rooms (the door kept), then distractors on floor cells
    __syncwarp();
    const uint64_t kr = stream_key(p.seed, (uint32_t)e, ep, P_ROOM);
    const int n_rooms = n_cells / 1024;
    for (int r = 0; r < n_rooms; ++r) {
      const int x0 = 1 + (int)below(draw_at(kr, (uint32_t)(2 * r)), (uint32_t)(S - 9));
      const int y0 = 1 + (int)below(draw_at(kr, (uint32_t)(2 * r + 1)), (uint32_t)(S - 9));
      for (int j = lane; j < 64; j += 32) {
        const int i = (y0 + (j >> 3)) * S + x0 + (j & 7);
        if (smap[i] != kDoor) smap[i] = 0;
      }
    }
    __syncwarp();
    auto is_free = [&](int i) { return smap[i] == 0; };
    const int n_free = count_cells(n_cells, lane, is_free);
    const int nd = (int)below(draw_at(stream_key(p.seed, (uint32_t)e, ep, P_NSPRITES), 0), (uint32_t)(p.K - 1));
    const uint64_t ks = stream_key(p.seed, (uint32_t)e, ep, P_SPRITE_CELL);
    for (int k = 0; k < nd; ++k) {
      const uint32_t c = below(draw_at(ks, (uint32_t)k), (uint32_t)n_free);
      spr_cell[2 + k] = nth_cell(n_cells, c, lane, is_free);
      spr_type[2 + k] = 3;
    }
    nspr = 2 + nd;
  }
  __syncwarp();
  write_episode_state(p, p.st, e, ep, cell_of(start), obj, nspr, spr_cell, spr_type, lane, 32);
  store_map(p, e, smap, lane);
  __syncwarp();
}

// Zero (floor) bytes among the 16 at q (16-byte aligned).
__device__ __forceinline__ int floor_bytes16(const uint8_t* q) {
  const uint4 v = *reinterpret_cast<const uint4*>(q);
  return 16 - __popc(nonzero4(v.x) | nonzero4(v.y) << 4 | nonzero4(v.z) << 8 | nonzero4(v.w) << 12);
}

// Shared-memory words one pre-generation lane needs for mazes of side S: the
// walk's visited bits (one per node) and parent directions (two bits per node).
__host__ __device__ __forceinline__ int pregen_lane_words(int S) {
  const int n = ((S - 2) / 2) * ((S - 2) / 2);
  return ((n + 31) >> 5) + ((n + 15) >> 4);
}

// One lane builds episode ep of env e into the next-episode block p.nx: the
// draws and steps of gen_maze, run serially by the lane, so that 32 mazes of
// a warp are built at once. S is a multiple of 4, so S * S is one of 16.
//
// The lane's shared-memory words (word w at sm[w * vstride]) hold the walk's
// state: a visited bit per node (a node is visited exactly when gen_maze's
// map byte of it is floor) and the direction back to the node's parent (two
// bits per node). Backtracking follows the parent directions, so no stack is
// kept; the stack depth is a counter, and the door's path nodes (at depths
// ceil(d / 2) - 1 and ceil(d / 2) on the path to the deepest node, depth d)
// are found afterwards by walking up from that node. The discovery and finish
// counters go to the env's work slot in global memory (written in the walk,
// read once for the key). After the walk the words hold the floor-cell counts
// of 256-cell chunks for the distractor draws.
//
// A build is resumable: lane_walk_begin lays the walls and starts the walk,
// lane_walk_step takes one of its 2 n - 1 steps (n - 1 carves, n
// backtracks), and lane_walk_finish places the door, key, rooms and sprites.
// Between launches the walk's scalars and shared-memory words are kept in the
// env's work slot (lane_walk_save, lane_walk_load), so that the building of
// an episode can be spread over the launches of the episode before it.
__device__ __forceinline__ uint32_t lds32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];\n" : "=r"(v) : "r"(addr));
  return v;
}
__device__ __forceinline__ void sts32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared.u32 [%0], %1;\n" ::"r"(addr), "r"(v) : "memory");
}

// The walk's scalars, all saved as 32-bit words.
struct LaneWalk {
  int vx, vy, v, sp, pushes, best_v, best_d, start, it, carved;
};
constexpr int kLaneWalkWords = 10;

// Byte offsets in an env's work slot for side S: the discovery counters, the
// finish counters, and the record (the episode being built, whether its walk
// is in progress, the walk's scalars). The walk's saved words live apart
// (lane_walk_save).
struct LaneSlot {
  int n, nn, vwords, dwords, off_fin, off_rec, bytes;
};
__host__ __device__ __forceinline__ LaneSlot lane_slot(int S) {
  LaneSlot L;
  L.nn = (S - 2) / 2;
  L.n = L.nn * L.nn;
  L.vwords = (L.n + 31) >> 5;
  L.dwords = (L.n + 15) >> 4;
  L.off_fin = align16(2 * L.n);
  L.off_rec = L.off_fin + align16(2 * L.n);
  L.bytes = L.off_rec + 4 * (2 + kLaneWalkWords);
  return L;
}

// The lane's visited and parent words in shared memory, through shared-space
// addresses: their loads need not wait for the lane's global stores (map
// bytes, counters), which never alias them.
struct LaneWords {
  uint32_t sbase, dbase, sstride;
  int vwords, dwords;
  __device__ uint32_t word(int w) const { return sbase + (uint32_t)w * sstride; }
  __device__ uint32_t seen(int u) const { return (lds32(word(u >> 5)) >> (u & 31)) & 1u; }
  __device__ void mark(int u) const {
    const uint32_t a = word(u >> 5);
    sts32(a, lds32(a) | 1u << (u & 31));
  }
  __device__ int parent_dir(int u) const {
    return (int)((lds32(dbase + (uint32_t)(u >> 4) * sstride) >> (2 * (u & 15))) & 3u);
  }
  __device__ void set_parent_dir(int u, int d) const {  // d: 0 N, 1 E, 2 S, 3 W; the old bits of u are 0
    const uint32_t a = dbase + (uint32_t)(u >> 4) * sstride;
    sts32(a, lds32(a) | (uint32_t)d << (2 * (u & 15)));
  }
};
__device__ __forceinline__ LaneWords lane_words(uint32_t* sm, int vstride, const LaneSlot& L) {
  LaneWords W;
  W.sbase = (uint32_t)__cvta_generic_to_shared(sm);
  W.sstride = 4u * (uint32_t)vstride;
  W.dbase = W.sbase + (uint32_t)L.vwords * W.sstride;
  W.vwords = L.vwords;
  W.dwords = L.dwords;
  return W;
}

// Sixteen wall cells i .. i + 15 of episode ep of env e (walls typed like
// gen_maze's), into its next-episode map.
__device__ __forceinline__ void lane_walls16(const Params& p, int e, uint32_t ep, int i) {
  const uint64_t kw = stream_key(p.seed, (uint32_t)e, ep, P_WALL);
  uint32_t q4[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t v = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) v |= (1u + (uint32_t)(draw_at(kw, (uint32_t)(i + 4 * q + b)) & 3)) << (8 * b);
    q4[q] = v;
  }
  *reinterpret_cast<uint4*>(p.nx.map + (size_t)e * p.S * p.S + i) = make_uint4(q4[0], q4[1], q4[2], q4[3]);
}

// The walk of episode ep of env e started at the spawn node (the walls are
// laid already, by lane_walls16), its words cleared.
__device__ LaneWalk lane_walk_begin(const Params& p, int e, uint32_t ep, const LaneWords& W, uint8_t* work,
                                    const LaneSlot& L) {
  const int S = p.S, n_cells = S * S, nn = L.nn;
  uint8_t* smap = p.nx.map + (size_t)e * n_cells;
  uint16_t* disc = reinterpret_cast<uint16_t*>(work);
  for (int w = 0; w < W.vwords + W.dwords; ++w) sts32(W.word(w), 0u);
  LaneWalk w;
  w.start = (int)below(draw_at(stream_key(p.seed, (uint32_t)e, ep, P_SPAWN), 0), (uint32_t)L.n);
  w.v = w.start;
  w.vx = 2 * (w.start % nn) + 1;
  w.vy = 2 * (w.start / nn) + 1;
  smap[w.vy * S + w.vx] = 0;
  W.mark(w.v);
  w.sp = 1;  // stack size: the current node's depth is sp - 1
  w.pushes = 0;
  w.carved = 0;
  disc[w.v] = (uint16_t)w.pushes++;
  w.best_v = w.start;
  w.best_d = 0;
  w.it = 0;
  return w;
}

// One step of the walk: a carve to the r-th unvisited neighbour in N, E, S, W
// order, or a backtrack to the parent when there is none.
__device__ __forceinline__ void lane_walk_step(const Params& p, const LaneWords& W, LaneWalk& w, uint64_t kd,
                                               uint8_t* smap, uint16_t* disc, uint16_t* fin, int nn) {
  const int S = p.S;
  // the draw a carve in this step takes (its high 32 bits), computed by every
  // lane of the warp together whether it carves or backtracks: lanes carve at
  // different steps, and a draw computed only where it is used would run once
  // for every different set of carving lanes
  uint32_t hi = (uint32_t)(draw_at(kd, (uint32_t)w.carved) >> 32);
  asm volatile("" : "+r"(hi));  // keeps the draw ahead of the branch
  ++w.it;
  const int vx = w.vx, vy = w.vy, v = w.v;
  const uint32_t open = (uint32_t)(vy > 1 && !W.seen(v - nn)) | ((uint32_t)(vx < S - 3 && !W.seen(v + 1)) << 1) |
                        ((uint32_t)(vy < S - 3 && !W.seen(v + nn)) << 2) | ((uint32_t)(vx > 1 && !W.seen(v - 1)) << 3);
  if (open == 0) {
    fin[v] = (uint16_t)w.pushes;
    if (--w.sp == 0) return;  // the spawn, finished: the walk's last step
    const int d = W.parent_dir(v);  // back to the parent
    w.vx += d == 1 ? 2 : (d == 3 ? -2 : 0);
    w.vy += d == 2 ? 2 : (d == 0 ? -2 : 0);
    w.v = (w.vy >> 1) * nn + (w.vx >> 1);
    return;
  }
  ++w.carved;
  uint32_t bits = open;
  const uint32_t r = below32(hi, (uint32_t)__popc(open));  // below 4: drop the r lowest set bits
  if (r > 0u) bits &= bits - 1u;
  if (r > 1u) bits &= bits - 1u;
  if (r > 2u) bits &= bits - 1u;
  const int d = __ffs(bits) - 1;
  const int dx = d == 1 ? 1 : (d == 3 ? -1 : 0), dy = d == 0 ? -1 : (d == 2 ? 1 : 0);
  smap[(vy + dy) * S + vx + dx] = 0;
  w.vx = vx + 2 * dx;
  w.vy = vy + 2 * dy;
  smap[w.vy * S + w.vx] = 0;
  w.v = (w.vy >> 1) * nn + (w.vx >> 1);
  W.mark(w.v);
  W.set_parent_dir(w.v, d ^ 2);
  const int depth = w.sp++;
  disc[w.v] = (uint16_t)w.pushes++;
  if (depth > w.best_d || (depth == w.best_d && w.v < w.best_v)) {
    w.best_v = w.v;
    w.best_d = depth;
  }
}

// A walk in progress into the env's record and the words array (word i of
// env e at words[i * n_envs + e], so that the lanes of a warp, consecutive
// envs, move consecutive words), or back into the lane's shared memory.
__device__ __forceinline__ void lane_walk_save(const LaneWords& W, const LaneWalk& w, uint8_t* work,
                                               const LaneSlot& L, uint32_t ep, uint32_t* words, int e, int n_envs) {
  for (int i = 0; i < W.vwords + W.dwords; ++i) words[(size_t)i * n_envs + e] = lds32(W.word(i));
  uint32_t* rec = reinterpret_cast<uint32_t*>(work + L.off_rec);
  const int s[kLaneWalkWords] = {w.vx, w.vy, w.v, w.sp, w.pushes, w.best_v, w.best_d, w.start, w.it, w.carved};
#pragma unroll
  for (int i = 0; i < kLaneWalkWords; ++i) rec[2 + i] = (uint32_t)s[i];
  rec[0] = ep;
  rec[1] = 1u;
}
__device__ __forceinline__ LaneWalk lane_walk_load(const LaneWords& W, const uint8_t* work, const LaneSlot& L,
                                                   const uint32_t* words, int e, int n_envs) {
  for (int i = 0; i < W.vwords + W.dwords; ++i) sts32(W.word(i), words[(size_t)i * n_envs + e]);
  const uint32_t* rec = reinterpret_cast<const uint32_t*>(work + L.off_rec);
  LaneWalk w;
  w.vx = (int)rec[2];
  w.vy = (int)rec[3];
  w.v = (int)rec[4];
  w.sp = (int)rec[5];
  w.pushes = (int)rec[6];
  w.best_v = (int)rec[7];
  w.best_d = (int)rec[8];
  w.start = (int)rec[9];
  w.it = (int)rec[10];
  w.carved = (int)rec[11];
  return w;
}

// The door, key, rooms and distractor sprites of a finished walk, and the
// episode's state fields into the next-episode block.
__device__ void lane_walk_finish(const Params& p, int e, uint32_t ep, const LaneWalk& w, const LaneWords& W,
                                 uint32_t* sm, int vstride, uint8_t* work, const LaneSlot& L) {
  const int S = p.S, n_cells = S * S;
  const int nn = L.nn, n = L.n;
  uint8_t* smap = p.nx.map + (size_t)e * n_cells;
  const uint16_t* disc = reinterpret_cast<const uint16_t*>(work);
  const uint16_t* fin = reinterpret_cast<const uint16_t*>(work + L.off_fin);
  const int best_v = w.best_v, best_d = w.best_d, start = w.start;
  auto parent_dir = [&](int u) { return W.parent_dir(u); };
  // the door sits on edge ceil(d / 2) of the path to the deepest node: between
  // its path nodes at depths j - 1 (a) and j (b), j = ceil(d / 2)
  const int j = (best_d + 1) / 2;
  int bx = 2 * (best_v % nn) + 1, by = 2 * (best_v / nn) + 1;
  for (int k = best_d; k > j; --k) {
    const int d = parent_dir((by >> 1) * nn + (bx >> 1));
    bx += d == 1 ? 2 : (d == 3 ? -2 : 0);
    by += d == 2 ? 2 : (d == 0 ? -2 : 0);
  }
  int ax = bx, ay = by;
  if (j > 0) {
    const int d = parent_dir((by >> 1) * nn + (bx >> 1));
    ax += d == 1 ? 2 : (d == 3 ? -2 : 0);
    ay += d == 2 ? 2 : (d == 0 ? -2 : 0);
  }
  const int dxc = (ax + bx) >> 1, dyc = (ay + by) >> 1;
  smap[dyc * S + dxc] = (uint8_t)kDoor;
  // key: uniform over spawn-side nodes except the spawn (outside the door's
  // subtree: discovery counter outside [disc, fin) of its path node b)
  const int pj = (by >> 1) * nn + (bx >> 1);
  const int d0 = disc[pj], d1 = fin[pj];
  const int n_side = n - (d1 - d0) - 1;
  int key = start;
  if (n_side > 0) {
    uint32_t r = below(draw_at(stream_key(p.seed, (uint32_t)e, ep, P_KEY), 0), (uint32_t)n_side);
    for (int u0 = 0; u0 < n; u0 += 8) {  // eight counters a load (the work slot is 16-byte aligned)
      const uint4 q = *reinterpret_cast<const uint4*>(disc + u0);
      const uint32_t dq[4] = {q.x, q.y, q.z, q.w};
      int found = -1;
#pragma unroll
      for (int h = 0; h < 8; ++h) {
        const int u = u0 + h;
        const int du = (int)((dq[h >> 1] >> (16 * (h & 1))) & 0xffffu);
        const bool side = u < n && u != start && !(du >= d0 && du < d1);
        if (side && found < 0) {
          if (r == 0)
            found = u;
          else
            --r;
        }
      }
      if (found >= 0) {
        key = found;
        break;
      }
    }
  }
  auto cell_of = [&](int u) { return (2 * (u / nn) + 1) * S + 2 * (u % nn) + 1; };
  const int kc = cell_of(key), gc = cell_of(best_v);
  const int obj[6] = {kc % S, kc / S, gc % S, gc / S, dxc, dyc};
  int spr_cell[kMaxSprites], spr_type[kMaxSprites];
  spr_cell[0] = kc;
  spr_type[0] = kSprKey;
  spr_cell[1] = gc;
  spr_type[1] = kSprGoal;
  int nspr = 2;
  if (p.task == 2) {
    // open 8 x 8 rooms (the door kept), then distractors on floor cells
    const uint64_t kr = stream_key(p.seed, (uint32_t)e, ep, P_ROOM);
    const int n_rooms = n_cells / 1024;
    for (int r = 0; r < n_rooms; ++r) {
      const int x0 = 1 + (int)below(draw_at(kr, (uint32_t)(2 * r)), (uint32_t)(S - 9));
      const int y0 = 1 + (int)below(draw_at(kr, (uint32_t)(2 * r + 1)), (uint32_t)(S - 9));
      for (int j2 = 0; j2 < 64; ++j2) {
        const int i = (y0 + (j2 >> 3)) * S + x0 + (j2 & 7);
        if (i != dyc * S + dxc) smap[i] = 0;  // the door cell is the only kDoor
      }
    }
    // floor cells per 256-cell chunk (the visited bits are no longer needed)
    const int n_chunks = n_cells >> 8;
    int n_free = 0;
    for (int ch = 0; ch < n_chunks; ++ch) {
      const uint4* g = reinterpret_cast<const uint4*>(smap + (ch << 8));
      uint4 q[16];
#pragma unroll
      for (int h = 0; h < 16; ++h) q[h] = g[h];
      int f = 0;
#pragma unroll
      for (int h = 0; h < 16; ++h)
        f += 16 - __popc(nonzero4(q[h].x) | nonzero4(q[h].y) << 4 | nonzero4(q[h].z) << 8 | nonzero4(q[h].w) << 12);
      sm[ch * vstride] = (uint32_t)f;
      n_free += f;
    }
    const int nd = (int)below(draw_at(stream_key(p.seed, (uint32_t)e, ep, P_NSPRITES), 0), (uint32_t)(p.K - 1));
    const uint64_t ks = stream_key(p.seed, (uint32_t)e, ep, P_SPRITE_CELL);
    for (int k = 0; k < nd && n_free > 0; ++k) {
      uint32_t r = below(draw_at(ks, (uint32_t)k), (uint32_t)n_free);
      int ch = 0;
      for (;; ++ch) {  // the chunk holding the r-th floor cell
        const uint32_t f = sm[ch * vstride];
        if (r < f) break;
        r -= f;
      }
      const uint4* g = reinterpret_cast<const uint4*>(smap + (ch << 8));
      uint4 q[16];
#pragma unroll
      for (int h = 0; h < 16; ++h) q[h] = g[h];
      int cell = -1;
#pragma unroll
      for (int h = 0; h < 16; ++h) {  // the r-th zero byte of the chunk
        const uint32_t z = ~(nonzero4(q[h].x) | nonzero4(q[h].y) << 4 | nonzero4(q[h].z) << 8 | nonzero4(q[h].w) << 12) &
                           0xffffu;
        const uint32_t c = (uint32_t)__popc(z);
        if (cell < 0) {
          if (r < c) {
            uint32_t zz = z;
            for (uint32_t t = 0; t < r; ++t) zz &= zz - 1;
            cell = (ch << 8) + 16 * h + __ffs(zz) - 1;
          } else {
            r -= c;
          }
        }
      }
      spr_cell[2 + k] = cell;
      spr_type[2 + k] = 3;
    }
    nspr = 2 + nd;
  }
  write_episode_state(p, p.nx, e, ep, cell_of(start), obj, nspr, spr_cell, spr_type, 0, 1);
}

// Takes over episode ep of env e from the next-episode block: the state
// fields generation writes, and the map staged into shared memory as bytes
// or as a bit plane (plain loads from the block, as gen writes them).
template <int MAPK>
__device__ __noinline__ void take_next(const Params& p, int e, uint32_t ep, uint8_t* wbase, int lane) {
  const WarpSmem ws{wbase, FillLane{}};
  const int n = p.S * p.S;
  const uint4* src = reinterpret_cast<const uint4*>(p.nx.map + (size_t)e * n);
  uint4* dst = reinterpret_cast<uint4*>(p.st.map + (size_t)e * n);
  uint4* sdst = reinterpret_cast<uint4*>(ws.map(p));
  for (int i = lane; i < (n >> 4); i += 32) {
    const uint4 v = src[i];
    dst[i] = v;
    if (!map_bits<MAPK>(p)) sdst[i] = v;
  }
  const State &st = p.st, &nx = p.nx;
  if (lane == 0) {
    st.cell_x[e] = nx.cell_x[e];
    st.cell_y[e] = nx.cell_y[e];
    st.frac_x[e] = 0.5f;
    st.frac_y[e] = 0.5f;
    st.theta0[e] = nx.theta0[e];
    st.cos0[e] = nx.cos0[e];
    st.sin0[e] = nx.sin0[e];
    st.turn[e] = 0;
    st.t[e] = 0;
    st.episode[e] = ep;
    st.flags[e] = 0;
    st.nspr[e] = nx.nspr[e];
  }
  if (lane < 6) st.obj[6 * (size_t)e + lane] = nx.obj[6 * (size_t)e + lane];
  for (int k = lane; k < p.K; k += 32) {
    const size_t i = (size_t)e * p.K + k;
    st.spr_x[i] = nx.spr_x[i];
    st.spr_y[i] = nx.spr_y[i];
    st.spr_type[i] = nx.spr_type[i];
  }
  __syncwarp();
  if (map_bits<MAPK>(p)) stage_map_bits(p, e, ws.map(p), lane, p.nx.map + (size_t)e * n);
}

// ASCII maps (Table 2): each episode copies the parsed map; the spawn is
// uniform over the 'S' cells (over all floor cells when there is none), the
// keys become sprites on their cells in row-major order, and a goal sprite
// goes on one 'G' cell drawn uniformly per episode.
__device__ __forceinline__ void gen_ascii(const Params& p, int e, uint32_t ep, uint8_t* smap, int lane) {
  const int S = p.S, n = S * S;
  for (int i = lane; i < n; i += 32) smap[i] = p.tmpl[i];
  __syncwarp();
  const uint64_t d = draw_at(stream_key(p.seed, (uint32_t)e, ep, P_SPAWN), 0);
  auto is_free = [&](int i) { return smap[i] == 0; };
  int cell;
  if (p.n_spawn > 0) {
    cell = p.cand[below(d, (uint32_t)p.n_spawn)];
  } else {
    const int n_free = count_cells(n, lane, is_free);
    cell = nth_cell(n, below(d, (uint32_t)n_free), lane, is_free);
  }
  int spr_cell[kMaxSprites], spr_type[kMaxSprites];
  int obj[6] = {-1, -1, -1, -1, -1, -1};
  const int32_t* keys = p.cand + p.n_spawn + p.n_goal;
  int k = 0;
  for (int i = 0; i < p.n_keys; ++i, ++k) {
    const int colour = keys[i] & 3;
    spr_cell[k] = keys[i] >> 2;
    spr_type[k] = colour == 0 ? kSprKey : (colour == 1 ? kSprKeyBlue : kSprKeyYellow);
  }
  if (p.n_keys > 0) {
    obj[0] = (keys[0] >> 2) % S;
    obj[1] = (keys[0] >> 2) / S;
  }
  if (p.n_goal > 0) {
    const int g = p.cand[p.n_spawn + below(draw_at(stream_key(p.seed, (uint32_t)e, ep, P_GOAL), 0),
                                           (uint32_t)p.n_goal)];
    spr_cell[k] = g;
    spr_type[k] = kSprGoal;
    ++k;
    obj[2] = g % S;
    obj[3] = g / S;
  }
  // the first locked door in row-major order
  for (int base = 0; base < n; base += 32) {
    const uint32_t b = __ballot_sync(0xffffffffu, base + lane < n && is_locked(smap[base + lane]));
    if (b) {
      const int c = base + __ffs(b) - 1;
      obj[4] = c % S;
      obj[5] = c / S;
      break;
    }
  }
  write_episode_state(p, p.st, e, ep, cell, obj, k, spr_cell, spr_type, lane, 32);
  __syncwarp();
  store_map(p, e, smap, lane);
  __syncwarp();
}

// The maze work space lives in the warp's frame staging ring when it fits
// (32 x 32 mazes need 2.3 KB), else in the global per-warp slot. Inlined
// behind unlikely branches: a call would make every value live across it
// spill in the hot loop. A byte map is generated in shared memory and copied
// out. In bit mode the byte map is generated in the ring, after the maze work
// space, when both fit there (the one-lane DFS then never waits on global
// memory), else in place in the state block; the bit plane is staged from it.
template <int MAPK>
__device__ __forceinline__ void generate(const Params& p, int e, uint32_t ep, uint8_t* wbase, uint8_t* scratch,
                                      int lane) {
  if (p.nx_ep != nullptr && p.nx_ep[e] == ep) {  // built ahead by the pre-generation kernel
    take_next<MAPK>(p, e, ep, wbase, lane);
    return;
  }
  const WarpSmem ws{wbase, fill_lane(p, lane)};
  const bool bits = map_bits<MAPK>(p);
  const bool maze = p.task != 0 && p.task != kTaskAscii;
  const size_t ring = (size_t)p.staging * p.frame_block_bytes;
  const size_t work_bytes = maze ? maze_scratch_bytes(((p.S - 2) / 2) * ((p.S - 2) / 2)) : 0;
  const bool work_in_ring = maze && work_bytes <= ring;
  const bool map_in_ring = bits && (size_t)align16((int)work_bytes) + (size_t)p.S * p.S <= ring;
  if (work_in_ring || map_in_ring) {
    if (lane == 0) bulk_wait_read_all();  // the ring's pending frame stores have read it
    __syncwarp();
  }
  uint8_t* smap = !bits ? ws.map(p) : (map_in_ring ? ws.ring() + align16((int)work_bytes) : p.st.map + (size_t)e * p.S * p.S);
  if (p.task == 0) {
    gen_rooms(p, e, ep, smap, lane);
  } else if (p.task == kTaskAscii) {
    gen_ascii(p, e, ep, smap, lane);
  } else {
    gen_maze(p, e, ep, smap, work_in_ring ? ws.ring() : scratch, lane);
  }
  if (bits) stage_map_bits(p, e, ws.map(p), lane, map_in_ring ? smap : nullptr);
}

// ------------------------------------------------------------------ step ----
template <int MAPK>
__device__ __forceinline__ bool solid(const Params& p, const uint8_t* smap, int S, int x, int y, int keys) {
  if (x < 0 || y < 0 || x >= S || y >= S) return true;
  if (map_bits<MAPK>(p)) return cell_set<MAPK>(p, smap, y * S + x);
  int v = smap[y * S + x];
  return v != 0 && !(is_locked(v) && ((keys >> (v - kLocked)) & 1));
}

// Box of half-size r centred at (cx + fx, cy + fy) overlaps no solid cell
// (closed intervals).
// floor(v) for v in [-1, 2): fractions stay in [0, 1) and a move or the box
// half-size is below 1/2, so every box edge lies in that range.
__device__ __forceinline__ int floor_small(float v) { return (v >= 1.f ? 1 : 0) - (v < 0.f ? 1 : 0); }

// Solidity of the 3 x 3 cells around cell (cx, cy), one lane per cell: bit
// 3 (dy + 1) + (dx + 1) for the cell at offset (dx, dy), dx, dy in {-1, 0, 1}.
// A move of at most half a cell by a box of half-size below one half keeps
// both axis tests of a step inside these cells (see box_hits).
template <int MAPK>
__device__ __forceinline__ uint32_t solid3x3(const Params& p, const uint8_t* smap, int cx, int cy, int keys,
                                             int lane) {
  const int k = lane < 9 ? lane : 4;
  const int dy = (k * 11 >> 5) - 1;  // k / 3 for k < 9
  const int dx = k - 3 * (dy + 1) - 1;
  const bool sld = lane < 9 && solid<MAPK>(p, smap, p.S, cx + dx, cy + dy, keys);
  return __ballot_sync(0xffffffffu, sld);
}

// The box of half-size r centred at (cx + fx, cy + fy) overlaps a solid cell
// of mask m (solid3x3 around cell (ox, oy)); closed intervals, touching counts.
__device__ __forceinline__ bool box_hits(uint32_t m, int ox, int oy, int cx, float fx, int cy, float fy, float r) {
  const int i0 = cx - ox + floor_small(fx - r), i1 = cx - ox + floor_small(fx + r);
  const int j0 = cy - oy + floor_small(fy - r), j1 = cy - oy + floor_small(fy + r);
  const uint32_t cols = ((2u << (i1 - i0)) - 1u) << (i0 + 1);  // offsets i0..i1 of one row
  bool hit = ((m >> (3 * (j0 + 1))) & cols) != 0u;
  if (j1 != j0) hit |= ((m >> (3 * (j1 + 1))) & cols) != 0u;
  return hit;
}

// An unlocked door opens when the agent walks into it: after a rejected axis
// move, every unlocked door cell under the box at (cx + fx, cy + fy) turns
// to floor, in the staged map and in the state block.
template <int MAPK>
__device__ __noinline__ void open_unlocked(const Params& p, int e, uint8_t* smap, int cx, float fx, int cy, float fy,
                                           int lane) {
  const int S = p.S;
  const float r = p.radius;
  const int i0 = cx + floor_small(fx - r), i1 = cx + floor_small(fx + r);
  const int j0 = cy + floor_small(fy - r), j1 = cy + floor_small(fy + r);
  uint8_t* g = p.st.map + (size_t)e * S * S;
  for (int j = j0; j <= j1; ++j)
    for (int i = i0; i <= i1; ++i) {
      if (i < 0 || j < 0 || i >= S || j >= S) continue;
      const int c = j * S + i;
      if (!is_unlocked(map_bits<MAPK>(p) ? g[c] : smap[c])) continue;
      if (lane == 0) {
        g[c] = 0;
        if (map_bits<MAPK>(p))
          reinterpret_cast<uint32_t*>(smap)[c >> 5] &= ~(1u << (c & 31));
        else
          smap[c] = 0;
      }
    }
  __syncwarp();
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

// An action outside 0..6 is recorded in the error word and taken as a no-op;
// a turn action moves `turn` one step around the circle of turns_per_rev.
__device__ __forceinline__ int turn_for(const Params& p, Env& r, int a, int lane) {
  if (a > 6) {
    if (lane == 0) atomicOr(p.err, 1u);
    a = 0;
  }
  if (a == 5) r.turn = r.turn == 0 ? p.tpr - 1 : r.turn - 1;
  if (a == 6) r.turn = r.turn + 1 == p.tpr ? 0 : r.turn + 1;
  return a;
}

// One step of env e under action a (already checked by turn_for, with the
// heading (c, s) of the turned agent); the reward and done flag go to output
// slot `out`. Returns true when the episode ended (the caller regenerates).
// The pose is written back to the state block only when write_state is set.
template <int MAPK>
__device__ __forceinline__ bool step_env(const Params& p, int e, Env& r, const uint8_t* smap, const int32_t* obj,
                                         const float4* spr_in, int lane, float c, float s, int a, size_t out,
                                         bool write_state) {
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
  const float rad = p.radius;
  const bool doors = p.task == kTaskAscii;  // maps with unlocked doors
  // both axis tests read the solidity of the cells around the start cell
  const int ox = r.cx, oy = r.cy;
  uint32_t m = solid3x3<MAPK>(p, smap, ox, oy, r.keys, lane);
  float nfx = r.fx + dx;
  if (!box_hits(m, ox, oy, r.cx, nfx, r.cy, r.fy, rad)) {
    r.fx = nfx;
    renormalise(r.cx, r.fx);
  } else if (__builtin_expect(doors, 0)) {
    open_unlocked<MAPK>(p, e, const_cast<uint8_t*>(smap), r.cx, nfx, r.cy, r.fy, lane);
    m = solid3x3<MAPK>(p, smap, ox, oy, r.keys, lane);  // opened doors are floor now
  }
  float nfy = r.fy + dy;
  if (!box_hits(m, ox, oy, r.cx, r.fx, r.cy, nfy, rad)) {
    r.fy = nfy;
    renormalise(r.cy, r.fy);
  } else if (__builtin_expect(doors, 0)) {
    open_unlocked<MAPK>(p, e, const_cast<uint8_t*>(smap), r.cx, r.fx, r.cy, nfy, lane);
  }
  // key and goal events from the sprite table (lane j looks at slot j): a key
  // of a colour not held yet on the agent's cell is picked up; a goal there
  // is reached
  uint32_t kbit = 0;
  bool goal = false;
  if (lane < obj[6]) {
    const float4 sp = spr_in[lane];
    if ((int)floorf(sp.x) == r.cx && (int)floorf(sp.y) == r.cy) {
      const int type = (int)sp.z;
      const int kc = key_colour(type);
      if (kc >= 0 && !((r.keys >> kc) & 1)) kbit = 1u << kc;
      goal = type == kSprGoal;
    }
  }
  const uint32_t picked = __reduce_or_sync(0xffffffffu, kbit);
  int ev = (picked ? 1 : 0) | (__any_sync(0xffffffffu, goal) ? 2 : 0);
  r.keys |= (int)picked;
  r.t += 1;
  const bool done = (ev & 2) || (p.horizon > 0 && r.t >= p.horizon);
  if (lane == 0) {
    p.rewards[out] = ev == 0 ? p.reward_lut[0] : (ev == 1 ? p.reward_lut[1] : (ev == 2 ? p.reward_lut[2] : p.reward_lut[3]));
    p.dones[out] = done ? 1 : 0;
    if (write_state && !done) {
      const State& st = p.st;
      st.cell_x[e] = (int16_t)r.cx;
      st.cell_y[e] = (int16_t)r.cy;
      st.frac_x[e] = r.fx;
      st.frac_y[e] = r.fy;
      st.turn[e] = (int16_t)r.turn;
      st.t[e] = r.t;
      st.flags[e] = (uint8_t)r.keys;
    }
  }
  return done;
}

// ---------------------------------------------------------------- render ----
// DDA (Sec. 2.1), one crossing per iteration. The next x boundary is at
// t = (kx + gx) / ax, the next y boundary at (ky + gy) / ay; the
// cross-multiplied forms are compared, so no division is needed.
struct Ray {
  int mx, my, sx, sy, side;
  float kx, ky;  // boundaries crossed so far (exact small integers)
  float ax, ay, gx, gy, gxay, gyax;
  bool done;
};

__device__ __forceinline__ void ray_init(Ray& q, const Env& r, float rx, float ry, bool valid) {
  q.mx = r.cx;
  q.my = r.cy;
  q.sx = rx < 0.f ? -1 : 1;
  q.sy = ry < 0.f ? -1 : 1;
  q.ax = fabsf(rx);
  q.ay = fabsf(ry);
  q.gx = rx < 0.f ? r.fx : 1.f - r.fx;
  q.gy = ry < 0.f ? r.fy : 1.f - r.fy;
  // an axis the ray never crosses compares as +infinity
  const float inf = __int_as_float(0x7f800000);
  q.gxay = q.ax == 0.f ? inf : q.gx * q.ay;
  q.gyax = q.ay == 0.f ? inf : q.gy * q.ax;
  q.kx = q.ky = 0.f;
  q.side = -1;
  q.done = !valid;
}

// One crossing. CHECK: a cell outside the map ends the ray (as wall 1);
// without it the map's border must be solid and the ray start inside it, so
// that every ray hits before it could leave (see mark_border).
template <int MAPK, bool CHECK>
__device__ __forceinline__ void ray_advance(const Params& p, Ray& q, const uint8_t* smap, int S) {
  const float lhs = fmaf(q.kx, q.ay, q.gxay);
  const float rhs = fmaf(q.ky, q.ax, q.gyax);
  const bool tx = lhs < rhs;
  q.mx += tx ? q.sx : 0;
  q.my += tx ? 0 : q.sy;
  q.kx += tx ? 1.f : 0.f;
  q.ky += tx ? 0.f : 1.f;
  q.side = tx ? 0 : 1;
  if (CHECK) {
    const bool out = (unsigned)q.mx >= (unsigned)S || (unsigned)q.my >= (unsigned)S;
    q.done = out || cell_set<MAPK>(p, smap, q.my * S + q.mx);
  } else {
    q.done = cell_set<MAPK>(p, smap, q.my * S + q.mx);
  }
}

// Whether rays of the staged map can skip the bounds test: every border cell
// is solid in the staged map (locked doors of held keys already cleared) and
// the agent's cell is not on the border, so a ray meets a solid cell before
// it could leave the map, and the agent, blocked by the border, stays inside.
// Kept in the warp's object words (obj[7]); recomputed whenever the staged map
// or the keys change. ASCII maps, whose unlocked doors open on contact, always
// take the bounds test.
template <int MAPK>
__device__ __forceinline__ void mark_border(const Params& p, const WarpSmem& ws, int cx, int cy, int lane) {
  const int S = p.S;
  bool ok = p.task != kTaskAscii && cx > 0 && cy > 0 && cx < S - 1 && cy < S - 1;
  if (ok) {
    const uint8_t* smap = ws.map(p);
    for (int i = lane; i < S; i += 32)
      ok = ok && cell_set<MAPK>(p, smap, i) && cell_set<MAPK>(p, smap, (S - 1) * S + i) &&
           cell_set<MAPK>(p, smap, i * S) && cell_set<MAPK>(p, smap, i * S + S - 1);
    ok = __all_sync(0xffffffffu, ok);
  }
  if (lane == 0) ws.obj(p)[7] = ok ? 1 : 0;
  __syncwarp();
}

// A finished ray's hit: perpendicular distance, face, and the hit cell's
// value. With bit-plane maps the value is a load from the state block; it is
// issued here and first used by finish_column, after the next pass's DDA, so
// that its latency overlaps that loop.
struct Hit {
  float perp;
  int side, v, col, mx, my;
};

template <int MAPK>
__device__ __forceinline__ Hit hit_of(const Params& p, int e, const Ray& q, int col, const WarpSmem& ws) {
  const int S = p.S;
  Hit h;
  if (q.side == 0)
    h.perp = __fdividef((q.kx - 1.f) + q.gx, q.ax);
  else if (q.side == 1)
    h.perp = __fdividef((q.ky - 1.f) + q.gy, q.ay);
  else
    h.perp = __int_as_float(0x7f800000);  // no hit
  h.side = q.side;
  h.col = col;
  h.mx = q.mx;
  h.my = q.my;
  h.v = 1;
  const bool inside = (unsigned)q.mx < (unsigned)S && (unsigned)q.my < (unsigned)S;
  if (q.side >= 0 && inside)
    h.v = map_bits<MAPK>(p) ? p.st.map[(size_t)e * S * S + q.my * S + q.mx] : ws.map(p)[q.my * S + q.mx];
  return h;
}

// Slice of a hit: rows and colour into the column arrays.
template <int MODE>
__device__ __forceinline__ void finish_column(const Params& p, int e, const Hit& q, const WarpSmem& ws) {
  const int H = p.H, col = q.col;
  const float perp = q.perp;
  // h = floor(H / perp + 1/2), clamped; top = floor((H - h) / 2)
  int h;
  if (perp > 0.f) {
    const float v = __fdividef((float)H, perp) + 0.5f;
    h = v >= 1048576.f ? kHMax : (int)floorf(v);
  } else {
    h = kHMax;
  }
  const int top = (H - h) >> 1;  // arithmetic shift: floor division by 2
  const int bot = top + h;
  const int v = q.v;
  const int slot = col_slot(col, p.W >> 4);
  uint32_t colour = ws.pal(p)[(q.side == 1 ? kCellColours : 0) + (v < kCellColours ? v : 1)];
  if (p.shading) {  // distance shading: channels scaled by q / 256, q = 64 + 192 min(h, H) / H
    const uint32_t qq = 64u + (uint32_t)(192 * (h < H ? h : H)) / (uint32_t)H;
    const uint32_t R = ((colour & 255u) * qq) >> 8, G = (((colour >> 8) & 255u) * qq) >> 8,
                   B = (((colour >> 16) & 255u) * qq) >> 8;
    colour = R | (G << 8) | (B << 16) | (luma(R, G, B) << 24);
  }
  ws.col_rgb(p)[slot] = colour;
  // h >= 0, so top <= H/2 <= bot: clamped to [0, H] they fit the byte offsets
  ws.col_top(p)[col] = (uint8_t)(127 + (top < 0 ? 0 : top));
  ws.col_bot(p)[col] = (uint8_t)(127 + (bot > H ? H : bot) - (H >> 1));
  ws.zbuf(p)[col] = perp;
  if (MODE == MODE_RAYS) {
    int4 hv = make_int4(q.side >= 0 ? q.mx : -1, q.side >= 0 ? q.my : -1, q.side, h);
    reinterpret_cast<int4*>(p.dbg_hits)[(size_t)e * p.W + col] = hv;
    p.dbg_perp[(size_t)e * p.W + col] = perp;
  }
}

// Cast every column's ray: in each pass lane l marches the rays of columns
// l + 32 j (j < COLS) together, and the warp leaves the DDA loop when a
// ballot says every ray has hit.
// The column table's entries lane and 32 + lane (0 beyond the frame), fetched
// ahead with the env's state: the first two passes of cast_columns use them.
__device__ __forceinline__ float2 col_k_pair(const Params& p, int lane) {
  return make_float2(__ldg(p.col_k + lane), lane + 32 < p.W ? __ldg(p.col_k + lane + 32) : 0.f);
}

template <int MODE, int MAPK, int COLS>
__device__ __forceinline__ void cast_columns(const Params& p, int e, const Env& r, float c, float s,
                                             const WarpSmem& ws, int lane, float2 k01) {
  const int W = p.W, S = p.S;
  const uint8_t* smap = ws.map(p);
  const int max_it = 4 * S + 8;
  const bool inside = ws.obj(p)[7] != 0;  // rays need no bounds test (mark_border)
  // single steps (latency-bound) finish a lane's hit after its next ray;
  // the other modes at once (a rollout keeps more state live across the loop)
  constexpr bool kDefer = MODE == MODE_STEP;
  Hit last;  // the lane's previous hit, finished after the next one is found
  bool pending = false;
  for (int col0 = lane; col0 - lane < W; col0 += 32 * COLS) {
    Ray q[COLS];
#pragma unroll
    for (int j = 0; j < COLS; ++j) {
      const int col = col0 + 32 * j;
      const bool valid = col < W;
      const int m = (col - lane) >> 5;  // column col = lane + 32 m
      const float k = m == 0 ? k01.x : (m == 1 ? k01.y : __ldg(p.col_k + (valid ? col : 0)));
      ray_init(q[j], r, fmaf(-k, s, c), fmaf(k, c, s), valid);
    }
    if (inside) {
      for (int it = 0; it < max_it; ++it) {
        bool all = true;
#pragma unroll
        for (int j = 0; j < COLS; ++j) {
          if (!q[j].done) ray_advance<MAPK, false>(p, q[j], smap, S);
          all = all && q[j].done;
        }
        if (__all_sync(0xffffffffu, all)) break;
      }
    } else {
      for (int it = 0; it < max_it; ++it) {
        bool all = true;
#pragma unroll
        for (int j = 0; j < COLS; ++j) {
          if (!q[j].done) ray_advance<MAPK, true>(p, q[j], smap, S);
          all = all && q[j].done;
        }
        if (__all_sync(0xffffffffu, all)) break;
      }
    }
#pragma unroll
    for (int j = 0; j < COLS; ++j)
      if (col0 + 32 * j < W) {
        const Hit h = hit_of<MAPK>(p, e, q[j], col0 + 32 * j, ws);
        if (!kDefer) {
          finish_column<MODE>(p, e, h, ws);
          continue;
        }
        if (pending) finish_column<MODE>(p, e, last, ws);
        last = h;
        pending = true;
      }
  }
  if (kDefer && pending) finish_column<MODE>(p, e, last, ws);
  __syncwarp();
}

// Project sprites (lane j takes sprite j) and order the visible ones far to
// near (equal depths: higher index first, so the lower index is drawn last).
// A sprite at depth ty is 0.25 W / (tan(fov/2) ty) columns wide, centred on
// column (W/2)(1 + tx/ty), and (H/2) / ty rows high from row H/2 down.
__device__ __forceinline__ int project_sprites(const Params& p, const Env& r, float c, float s, const WarpSmem& ws,
                                               int lane) {
  const int W = p.W, H = p.H;
  bool vis = false;
  float ty = 0.f;
  int cA = 0, cB = -1;
  const int nspr = ws.obj(p)[6];
  if (lane < nspr) {
    const float4 sp = ws.spr_in(p)[lane];
    const int type = (int)sp.z;
    const float vx = (sp.x - (float)r.cx) - r.fx;
    const float vy = (sp.y - (float)r.cy) - r.fy;
    ty = fmaf(vx, c, vy * s);
    const int kc = key_colour(type);
    if (type != 0 && !(kc >= 0 && ((r.keys >> kc) & 1)) && ty > 0.1f) {
      // 1/ty within an ulp or two: pixel positions move by far less than the
      // 1e-3 pixel the silhouette-edge tolerance allows
      const float inv_ty = __fdividef(1.f, ty);
      const float tx = fmaf(-vx, s, vy * c) * p.inv_tan_half;
      const float wd = 0.25f * (float)W * p.inv_tan_half * inv_ty;
      const float ht = 0.5f * (float)H * inv_ty;
      const float x0 = fmaf(0.5f * (float)W, fmaf(tx, inv_ty, 1.f), -0.5f * wd);
      const float top = 0.5f * (float)H;
      // pixel centres that can fall inside [x0, x0 + wd) x [top, top + ht), one pixel of slack
      cA = (int)floorf(fmaxf(x0 - 1.f, -1.f));
      cB = (int)floorf(fminf(x0 + wd + 1.f, (float)W));
      const int rA = (int)floorf(fmaxf(top - 1.f, -1.f));
      const int rB = (int)floorf(fminf(top + ht + 1.f, (float)H));
      cA = cA < 0 ? 0 : cA;
      cB = cB > W - 1 ? W - 1 : cB;
      vis = cA <= cB;  // some column of the screen
      if (vis) {
        ws.spr_a(p)[lane] = make_float4(x0, top, ty * (4.f * p.tan_half / (float)W), ty * (2.f / (float)H));
        ws.spr_rect(p)[lane] = make_int4(cA, cB, rA < 0 ? 0 : rA, rB > H - 1 ? H - 1 : rB);
        ws.spr_ty(p)[lane] = ty;
        ws.spr_rgb(p)[lane] = ws.pal(p)[2 * kCellColours + (type & 7)];
        ws.spr_kind(p)[lane] = kc >= 0 ? 1 : (type == kSprGoal ? 2 : 3);  // mask: diamond, rectangle, disc
      }
    }
  }
  const uint32_t cand = __ballot_sync(0xffffffffu, vis);
  if (cand == 0u) return 0;  // nothing on screen (warp-uniform)
  // A pixel is drawn only where the sprite is nearer than its column's wall:
  // a sprite behind the walls at every column it can cover is culled here
  // (the lanes scan its columns together).
  uint32_t vmask = 0u;
  for (uint32_t m = cand; m != 0u; m &= m - 1u) {
    const int j = __ffs(m) - 1;
    const int a = __shfl_sync(0xffffffffu, cA, j), b = __shfl_sync(0xffffffffu, cB, j);
    const float tj = __shfl_sync(0xffffffffu, ty, j);
    bool nearer = false;
    for (int col = a + lane; col <= b; col += 32) nearer |= tj < ws.zbuf(p)[col];
    if (__any_sync(0xffffffffu, nearer)) vmask |= 1u << j;
  }
  if (vmask == 0u) return 0;
  vis = (vmask >> lane) & 1u;
  int rank = 0;  // visible sprites farther than this one (or as far, of higher index)
  if (vmask & (vmask - 1u))
    for (uint32_t m = vmask; m != 0u; m &= m - 1u) {
      const int k = __ffs(m) - 1;
      const float tk = __shfl_sync(0xffffffffu, ty, k);
      if (vis && (tk > ty || (tk == ty && k > lane))) ++rank;
    }
  if (vis) ws.order(p)[rank] = lane;
  __syncwarp();
  return __popc(vmask);
}

// Four pixels of colour c as the three words of their 12 RGB bytes.
__host__ __device__ constexpr uint32_t rgb_word(uint32_t c, int k) {
  return k == 0 ? (c & 0xFFFFFFu) | (c << 24)                       // R G B R
         : k == 1 ? ((c >> 8) & 0xFFFFu) | ((c & 0xFFFFu) << 16)   // G B R G
                  : ((c >> 16) & 255u) | ((c & 0xFFFFFFu) << 8);   // B R G B
}

// prmt with every selector nibble's sign bit set: byte j of the result is
// 0xFF or 0x00 as bit 7 of byte (SEL >> 4j) & 3 of x is set or clear.
template <uint32_t SEL>
__device__ __forceinline__ uint32_t sign_bytes(uint32_t x) {
  uint32_t d;
  asm("prmt.b32 %0, %1, 0, %2;" : "=r"(d) : "r"(x), "n"(SEL));
  return d;
}
__device__ __forceinline__ uint32_t select_bytes(uint32_t m, uint32_t a, uint32_t b) { return (m & a) | (~m & b); }

// Fill rows [r0, r1) of the frame into `buf` (row-major RGB), then draw the
// sprites over them.
//
// A lane owns 16 columns of a row: four quads of 4 pixels, 12 bytes = 3 words
// each, stored as three 16-byte words. Because every slice is centred, a row
// above H/2 is ceiling or wall and a row at or below it is wall or floor.
// Byte k of d = (127 + top_k) - row (all bytes at once) is in [0, 255], so no
// borrow crosses bytes, and its bit 7 is set exactly when row < top_k;
// sign-replicating prmt turns those bits into byte masks laid out like the
// pixels' RGB bytes, and one select per word picks ceiling or wall. Rows
// below the middle do the same with 127 + bot_k - H/2 and row - H/2 (wall or
// floor).
#define JX_QUAD_WORDS(d, A0, A1, A2, B0, B1, B2)                                        \
  select_bytes(sign_bytes<0x9888>(d), A0, B0), select_bytes(sign_bytes<0xAA99>(d), A1, B1), \
      select_bytes(sign_bytes<0xBBBA>(d), A2, B2)
// GRAYF: the block also writes its rows of the grayscale frame into gbuf.
template <bool GRAYF>
__device__ __forceinline__ void fill_block(const Params& p, const WarpSmem& ws, uint8_t* buf, uint8_t* gbuf, int r0,
                                          int r1, int nvis, int lane) {
  const int W = p.W, H = p.H, rowb = 3 * W, mid = H >> 1;
  const int groups = ws.fl.groups;  // lanes per row, 16 pixels (48 bytes) each
  const int rpp = ws.fl.rows;       // rows per pass
  const int my_row = ws.fl.my_row, g = ws.fl.g;
  if (my_row < rpp) {
    const uint4 t16 = *reinterpret_cast<const uint4*>(ws.col_top(p) + 16 * g);
    const uint4 b16 = *reinterpret_cast<const uint4*>(ws.col_bot(p) + 16 * g);
    uint32_t wq[12], yq[4];  // wall RGB words of the four quads, wall luma bytes
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const uint4 c = *reinterpret_cast<const uint4*>(ws.col_rgb(p) + ((h * groups + g) << 2));
      wq[3 * h + 0] = __byte_perm(c.x, c.y, 0x4210);
      wq[3 * h + 1] = __byte_perm(c.y, c.z, 0x5421);
      wq[3 * h + 2] = __byte_perm(c.z, c.w, 0x6542);
      if (GRAYF) yq[h] = __byte_perm(__byte_perm(c.x, c.y, 0x0073), __byte_perm(c.z, c.w, 0x0073), 0x5410);
    }
    constexpr uint32_t C0 = rgb_word(kCeil, 0), C1 = rgb_word(kCeil, 1), C2 = rgb_word(kCeil, 2);
    constexpr uint32_t F0 = rgb_word(kFloor, 0), F1 = rgb_word(kFloor, 1), F2 = rgb_word(kFloor, 2);
    constexpr uint32_t CY = (kCeil >> 24) * 0x01010101u, FY = (kFloor >> 24) * 0x01010101u;
    const uint32_t step = (uint32_t)rpp * 0x01010101u;
    int row = r0 + my_row;
    // this lane's 48 RGB bytes (and 16 luma bytes) in its first row
    uint4* dst = reinterpret_cast<uint4*>(buf + my_row * rowb + g * 48);
    uint4* gdst = reinterpret_cast<uint4*>((GRAYF ? gbuf : buf) + my_row * W + g * 16);
    const int dstep = rpp * rowb / 16, gstep = rpp * W / 16;
    const int lim = r1 < mid ? r1 : mid;
    if (row < lim) {  // ceiling or wall
      const uint32_t rr = (uint32_t)row * 0x01010101u;
      uint32_t d0 = t16.x - rr, d1 = t16.y - rr, d2 = t16.z - rr, d3 = t16.w - rr;
      for (; row < lim; row += rpp, d0 -= step, d1 -= step, d2 -= step, d3 -= step, dst += dstep) {
        const uint32_t a[12] = {JX_QUAD_WORDS(d0, C0, C1, C2, wq[0], wq[1], wq[2]),
                                JX_QUAD_WORDS(d1, C0, C1, C2, wq[3], wq[4], wq[5]),
                                JX_QUAD_WORDS(d2, C0, C1, C2, wq[6], wq[7], wq[8]),
                                JX_QUAD_WORDS(d3, C0, C1, C2, wq[9], wq[10], wq[11])};
        dst[0] = make_uint4(a[0], a[1], a[2], a[3]);
        dst[1] = make_uint4(a[4], a[5], a[6], a[7]);
        dst[2] = make_uint4(a[8], a[9], a[10], a[11]);
        if (GRAYF) {
          *gdst = make_uint4(select_bytes(sign_bytes<0xBA98>(d0), CY, yq[0]), select_bytes(sign_bytes<0xBA98>(d1), CY, yq[1]),
                             select_bytes(sign_bytes<0xBA98>(d2), CY, yq[2]), select_bytes(sign_bytes<0xBA98>(d3), CY, yq[3]));
          gdst += gstep;
        }
      }
    }
    if (row < r1) {  // wall or floor
      const uint32_t rr = (uint32_t)(row - mid) * 0x01010101u;
      uint32_t d0 = b16.x - rr, d1 = b16.y - rr, d2 = b16.z - rr, d3 = b16.w - rr;
      for (; row < r1; row += rpp, d0 -= step, d1 -= step, d2 -= step, d3 -= step, dst += dstep) {
        const uint32_t a[12] = {JX_QUAD_WORDS(d0, wq[0], wq[1], wq[2], F0, F1, F2),
                                JX_QUAD_WORDS(d1, wq[3], wq[4], wq[5], F0, F1, F2),
                                JX_QUAD_WORDS(d2, wq[6], wq[7], wq[8], F0, F1, F2),
                                JX_QUAD_WORDS(d3, wq[9], wq[10], wq[11], F0, F1, F2)};
        dst[0] = make_uint4(a[0], a[1], a[2], a[3]);
        dst[1] = make_uint4(a[4], a[5], a[6], a[7]);
        dst[2] = make_uint4(a[8], a[9], a[10], a[11]);
        if (GRAYF) {
          *gdst = make_uint4(select_bytes(sign_bytes<0xBA98>(d0), yq[0], FY), select_bytes(sign_bytes<0xBA98>(d1), yq[1], FY),
                             select_bytes(sign_bytes<0xBA98>(d2), yq[2], FY), select_bytes(sign_bytes<0xBA98>(d3), yq[3], FY));
          gdst += gstep;
        }
      }
    }
  }
  __syncwarp();
  if (nvis == 0) return;  // warp-uniform
  // sprites, far to near; lanes take columns. For a column, the covered rows
  // are those whose centre has v in [0, 1) with |2v - 1| below the mask's
  // half-height at this u (key: 1 - |2u - 1|, disc: sqrt(1 - (2u - 1)^2)).
  // the sprites whose rows meet this block, far to near
  const uint32_t span = lane < nvis ? ws.spr_span(p)[lane] : 0xFFFF0000u;
  uint32_t hits = __ballot_sync(0xffffffffu, (int)(span >> 16) < r1 && (int)(span & 0xffffu) >= r0);
  while (hits) {
    const int oi = __ffs(hits) - 1;
    hits &= hits - 1;
    const int j = ws.order(p)[oi];
    const int4 rc = ws.spr_rect(p)[j];
    const int rA = rc.z < r0 ? r0 : rc.z;
    const int rB = rc.w > r1 - 1 ? r1 - 1 : rc.w;
    if (rc.x > rc.y || rA > rB) continue;
    const float4 a = ws.spr_a(p)[j];  // x0, top, 1/width, 1/height
    const float ty = ws.spr_ty(p)[j];
    const uint32_t rgbv = ws.spr_rgb(p)[j];
    const int kind = ws.spr_kind(p)[j];
    for (int col = rc.x + lane; col <= rc.y; col += 32) {
      const float u = ((float)col + 0.5f - a.x) * a.z;
      if (!(u >= 0.f && u < 1.f && ty < ws.zbuf(p)[col])) continue;
      const float au = fabsf(fmaf(2.f, u, -1.f));
      const float half = kind == 1 ? 1.f - au : (kind == 2 ? 2.f : sqrtf(fmaxf(0.f, fmaf(-au, au, 1.f))));
      uint8_t* px = buf + col * 3;
      for (int row = rA; row <= rB; ++row) {
        const float v = ((float)row + 0.5f - a.y) * a.w;
        if (v >= 0.f && v < 1.f && fabsf(fmaf(2.f, v, -1.f)) < half) {
          uint8_t* q = px + (row - r0) * rowb;
          q[0] = (uint8_t)(rgbv & 255);
          q[1] = (uint8_t)((rgbv >> 8) & 255);
          q[2] = (uint8_t)((rgbv >> 16) & 255);
          if (GRAYF) gbuf[(row - r0) * W + col] = (uint8_t)(rgbv >> 24);
        }
      }
    }
    __syncwarp();
  }
}
#undef JX_QUAD_WORDS

// GRAY: 0 no grayscale stack, 1 a stack, 2 as p.st.gray says (batched kernel).
template <int MODE, int MAPK, int COLS, int GRAY>
__device__ __forceinline__ void render_env(const Params& p, int e, const Env& r, float c, float s,
                                           const WarpSmem& ws, int lane, int& slot, uint8_t* frame, float2 k01) {
  cast_columns<MODE, MAPK, COLS>(p, e, r, c, s, ws, lane, k01);
  if (MODE == MODE_RAYS) return;
  const int nvis = project_sprites(p, r, c, s, ws, lane);  // ends with __syncwarp
  const int H = p.H, W = p.W, rowb = 3 * W;
  if (lane < nvis) {  // rows each sprite of the far-to-near order can cover
    const int4 rc = ws.spr_rect(p)[ws.order(p)[lane]];
    ws.spr_span(p)[lane] = rc.x <= rc.y ? ((uint32_t)rc.z << 16) | (uint32_t)rc.w : 0xFFFF0000u;
  }
  __syncwarp();
  const bool gray_on = GRAY == 1 || (GRAY == 2 && p.st.gray != nullptr);
  for (int r0 = 0; r0 < H; r0 += p.rows_per_block) {
    const int r1 = r0 + p.rows_per_block < H ? r0 + p.rows_per_block : H;
    uint8_t* buf = ws.ring() + slot * p.frame_block_bytes;
    uint8_t* gbuf = gray_on ? ws.gray_ring(p) + slot * p.gray_block_bytes : nullptr;
    if (lane == 0) bulk_wait_staging(p.staging);
    __syncwarp();
    if (gray_on)
      fill_block<true>(p, ws, buf, gbuf, r0, r1, nvis, lane);
    else
      fill_block<false>(p, ws, buf, gbuf, r0, r1, nvis, lane);
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) {
      bulk_copy(frame + (size_t)r0 * rowb, buf, (uint32_t)((r1 - r0) * rowb));
      if (gray_on) {
        // grayscale stack: plane t mod 4, or all four planes for an episode's first frame
        const size_t plane = (size_t)H * W;
        uint8_t* g0 = p.st.gray + (size_t)e * 4 * plane + (size_t)r0 * W;
        const uint32_t gbytes = (uint32_t)((r1 - r0) * W);
        if (r.t == 0) {
          for (int k = 0; k < 4; ++k) bulk_copy(g0 + k * plane, gbuf, gbytes);
        } else {
          bulk_copy(g0 + (size_t)(r.t & 3) * plane, gbuf, gbytes);
        }
      }
      bulk_commit();
    }
    slot = slot + 1 == p.staging ? 0 : slot + 1;
  }
}

// Locked doors of the colours held open for rays (and, in bit mode, for
// collisions): their cells are cleared in the staged map, which the state
// block keeps as written. Run after staging and whenever the keys change.
// Generated mazes have one red door (the door cell of the state); ASCII maps
// are scanned.
template <int MAPK>
__device__ __noinline__ void open_doors(const Params& p, int e, int keys, const WarpSmem& ws, int lane) {
  if (keys == 0) return;
  const int S = p.S, n = S * S;
  const uint8_t* g = p.st.map + (size_t)e * n;
  uint8_t* smap = ws.map(p);
  if (p.task == kTaskAscii) {
    for (int i = lane; i < n; i += 32) {
      const int v = map_bits<MAPK>(p) ? g[i] : smap[i];
      if (!(is_locked(v) && ((keys >> (v - kLocked)) & 1))) continue;
      if (map_bits<MAPK>(p))
        atomicAnd(reinterpret_cast<uint32_t*>(smap) + (i >> 5), ~(1u << (i & 31)));
      else
        smap[i] = 0;
    }
  } else if (keys & 1) {
    const int2 door = *reinterpret_cast<const int2*>(ws.obj(p) + 4);
    if (lane == 0 && door.x >= 0 && door.y >= 0 && door.x < S && door.y < S) {
      const int i = door.y * S + door.x;
      if (map_bits<MAPK>(p)) {
        if (g[i] == kDoor) reinterpret_cast<uint32_t*>(smap)[i >> 5] &= ~(1u << (i & 31));
      } else if (smap[i] == kDoor) {
        smap[i] = 0;
      }
    }
  }
  __syncwarp();
}

// What a launch reads of env e before its first step, fetched in one round of
// independent loads so that their latencies overlap: the scalar state, the
// key / goal / door cells and sprite count (lanes 0..6), the sprite slots
// (lane j: slot j), the map when it holds at most 1 KB (two 16-byte chunks a
// lane), the first action, the column table's first two entries of the lane,
// and for the single step the turn table's entries lane, 32 + lane and
// 64 + lane (tables of at most 96 turns).
struct Prefetch {
  Env r;
  int obj;
  float4 spr;
  uint4 m0, m1;
  float2 tc0, tc1, tc2;
  float2 k01;  // column table entries lane, 32 + lane
  int action;
};

template <int MAPK>
__device__ __forceinline__ bool small_map(const Params& p) {
  const int n = p.S * p.S;
  return n <= 1024 && (n & 31) == 0;
}

template <int MODE, int MAPK>
__device__ __forceinline__ Prefetch prefetch(const Params& p, int e, int t0, int lane) {
  Prefetch q;
  const State& st = p.st;
  q.r = load_env(p, e);
  q.obj = lane < 6 ? (int)st.obj[6 * (size_t)e + lane] : (lane == 6 ? (int)st.nspr[e] : 0);
  q.spr = make_float4(0.f, 0.f, 0.f, 0.f);
  if (lane < p.K) {
    const size_t i = (size_t)e * p.K + lane;
    q.spr = make_float4(st.spr_x[i], st.spr_y[i], (float)st.spr_type[i], 0.f);
  }
  q.m0 = q.m1 = make_uint4(0u, 0u, 0u, 0u);
  if (small_map<MAPK>(p)) {
    const int n = p.S * p.S;
    const uint4* g = reinterpret_cast<const uint4*>(st.map + (size_t)e * n);
    if (map_bits<MAPK>(p)) {  // word `lane` of the bit plane: cells 32 lane .. 32 lane + 31
      if (lane < (n >> 5)) {
        q.m0 = g[2 * lane];
        q.m1 = g[2 * lane + 1];
      }
    } else {
      if (lane < (n >> 4)) q.m0 = g[lane];
      if (lane + 32 < (n >> 4)) q.m1 = g[lane + 32];
    }
  }
  q.action = (MODE == MODE_STEP || MODE == MODE_ROLLOUT) ? (int)p.actions[(size_t)t0 * p.out_stride + e] : 0;
  q.k01 = col_k_pair(p, lane);
  q.tc0 = q.tc1 = q.tc2 = make_float2(0.f, 0.f);
  if (MODE == MODE_STEP && p.tpr <= 96) {
    if (lane < p.tpr) q.tc0 = p.turn_cs[lane];
    if (lane + 32 < p.tpr) q.tc1 = p.turn_cs[lane + 32];
    if (lane + 64 < p.tpr) q.tc2 = p.turn_cs[lane + 64];
  }
  return q;
}

// The prefetched objects, sprites and map into the warp's shared memory
// (maps too large to prefetch are staged here), and the border flag of
// mark_border (taken from the prefetched rows for 32 x 32 bit planes); ends
// with __syncwarp. False when the map's copy was lost (see stage_map).
template <int MAPK>
__device__ __forceinline__ bool stage_prefetched(const Params& p, const WarpSmem& ws, int e, const Prefetch& q,
                                                 int lane) {
  if (lane < 6) ws.obj(p)[lane] = q.obj;
  if (lane == 6) ws.obj(p)[6] = q.obj > p.K ? p.K : q.obj;  // sprites in use
  if (lane < p.K) ws.spr_in(p)[lane] = q.spr;
  if (!small_map<MAPK>(p)) {
    if (!stage<MAPK>(p, e, ws.map(p), lane)) return false;  // ends with __syncwarp
    mark_border<MAPK>(p, ws, q.r.cx, q.r.cy, lane);
    return true;
  }
  const int n = p.S * p.S;
  if (map_bits<MAPK>(p)) {
    const uint32_t w = nonzero4(q.m0.x) | nonzero4(q.m0.y) << 4 | nonzero4(q.m0.z) << 8 | nonzero4(q.m0.w) << 12 |
                       nonzero4(q.m1.x) << 16 | nonzero4(q.m1.y) << 20 | nonzero4(q.m1.z) << 24 |
                       nonzero4(q.m1.w) << 28;
    if (lane < (n >> 5)) reinterpret_cast<uint32_t*>(ws.map(p))[lane] = w;
    if (p.S == 32) {  // word `lane` is row `lane`: its end cells, and all of rows 0 and 31, solid
      const int S = 32, cx = q.r.cx, cy = q.r.cy;
      const bool row_ok = (w & 0x80000001u) == 0x80000001u && ((lane != 0 && lane != S - 1) || w == 0xffffffffu);
      const bool ok = __all_sync(0xffffffffu, row_ok) && p.task != kTaskAscii && cx > 0 && cy > 0 && cx < S - 1 &&
                      cy < S - 1;
      if (lane == 0) ws.obj(p)[7] = ok ? 1 : 0;
      __syncwarp();
      return true;
    }
  } else {
    uint4* dst = reinterpret_cast<uint4*>(ws.map(p));
    if (lane < (n >> 4)) dst[lane] = q.m0;
    if (lane + 32 < (n >> 4)) dst[lane + 32] = q.m1;
  }
  __syncwarp();
  mark_border<MAPK>(p, ws, q.r.cx, q.r.cy, lane);
  return true;
}

// Turn table entry `turn`: from the prefetched registers (lane turn mod 32
// holds it) when the table has at most 96 entries, else from global memory.
__device__ __forceinline__ float2 turn_entry(const Params& p, const Prefetch& q, int turn) {
  if (p.tpr > 96) return p.turn_cs[turn];
  const int src = turn & 31;
  const float2 a = make_float2(__shfl_sync(0xffffffffu, q.tc0.x, src), __shfl_sync(0xffffffffu, q.tc0.y, src));
  const float2 b = make_float2(__shfl_sync(0xffffffffu, q.tc1.x, src), __shfl_sync(0xffffffffu, q.tc1.y, src));
  const float2 c = make_float2(__shfl_sync(0xffffffffu, q.tc2.x, src), __shfl_sync(0xffffffffu, q.tc2.y, src));
  return turn < 32 ? a : (turn < 64 ? b : c);
}

// An ended episode: the next one (built here or taken over from the
// next-episode block), its state and objects reloaded, and its heading.
// Inlined behind the callers' unlikely branches (see generate).
template <int MAPK>
__device__ __forceinline__ void next_episode(const Params& p, int e, Env& r, const WarpSmem& ws, uint8_t* scratch,
                                          int lane, float& c, float& s) {
  const uint32_t ep = p.st.episode[e] + 1;
  __syncwarp();
  generate<MAPK>(p, e, ep, ws.base, scratch, lane);
  r = load_env(p, e);
  load_objects(p, ws, e, lane);
  __syncwarp();
  heading(p, r, c, s);
  mark_border<MAPK>(p, ws, r.cx, r.cy, lane);
}

// Everything one launch does for env e: MODE_ROLLOUT runs the launch's steps
// t0 .. t1 - 1 with the env's scalar state in registers and its map in shared
// memory (the state is loaded before step t0 and stored after step t1 - 1).
// Returns false when the env's map copy was lost: the warp must stop.
template <int MODE, int MAPK, int COLS, int GRAY>
__device__ __forceinline__ bool run_env(const Params& p, int e, uint8_t* wbase, uint8_t* scratch, int lane,
                                        int& slot, int t0 = 0, int t1 = 0) {
  const WarpSmem ws{wbase, fill_lane(p, lane)};
  const size_t frame_bytes = (size_t)3 * p.H * p.W;
  if (MODE == MODE_RESET) {
    generate<MAPK>(p, e, 0u, wbase, scratch, lane);
    const Env r = load_env(p, e);
    load_objects(p, ws, e, lane);
    __syncwarp();
    mark_border<MAPK>(p, ws, r.cx, r.cy, lane);
    float c, s;
    heading(p, r, c, s);
    render_env<MODE, MAPK, COLS, GRAY>(p, e, r, c, s, ws, lane, slot, p.frames + (size_t)e * frame_bytes,
                                       col_k_pair(p, lane));
    __syncwarp();
    return true;
  }
  const Prefetch q = prefetch<MODE, MAPK>(p, e, t0, lane);
  Env r = q.r;
  if (!stage_prefetched<MAPK>(p, ws, e, q, lane)) return false;  // ends with __syncwarp
  if (r.keys != 0) {  // doors of held keys open: the border flag again
    open_doors<MAPK>(p, e, r.keys, ws, lane);
    mark_border<MAPK>(p, ws, r.cx, r.cy, lane);
  }
  if (MODE == MODE_ROLLOUT) {
    int a_next = q.action;
    for (int t = t0; t < t1; ++t) {
      int a = a_next;
      if (t + 1 < t1) a_next = p.actions[(size_t)(t + 1) * p.out_stride + e];
      const size_t out = (size_t)t * p.out_stride + e;
      const int keys0 = r.keys;
      a = turn_for(p, r, a, lane);
      float c, s;
      heading(p, r, c, s);
      if (__builtin_expect(step_env<MAPK>(p, e, r, ws.map(p), ws.obj(p), ws.spr_in(p), lane, c, s, a, out, false), 0))
        next_episode<MAPK>(p, e, r, ws, scratch, lane, c, s);
      if (__builtin_expect(r.keys != keys0, 0)) {
        open_doors<MAPK>(p, e, r.keys, ws, lane);
        mark_border<MAPK>(p, ws, r.cx, r.cy, lane);
      }
      render_env<MODE, MAPK, COLS, GRAY>(p, e, r, c, s, ws, lane, slot,
                                         p.frames + (size_t)t * p.frame_step + (size_t)e * frame_bytes, q.k01);
      __syncwarp();
    }
    if (lane == 0) {
      const State& st = p.st;
      st.cell_x[e] = (int16_t)r.cx;
      st.cell_y[e] = (int16_t)r.cy;
      st.frac_x[e] = r.fx;
      st.frac_y[e] = r.fy;
      st.turn[e] = (int16_t)r.turn;
      st.t[e] = r.t;
      st.flags[e] = (uint8_t)r.keys;
    }
    __syncwarp();
    return true;
  }
  float c, s;
  if (MODE == MODE_STEP) {
    const int keys0 = r.keys;
    const int a = turn_for(p, r, q.action, lane);
    heading_from(r, turn_entry(p, q, r.turn), c, s);
    if (__builtin_expect(step_env<MAPK>(p, e, r, ws.map(p), ws.obj(p), ws.spr_in(p), lane, c, s, a, (size_t)e, true),
                         0))
      next_episode<MAPK>(p, e, r, ws, scratch, lane, c, s);
    else if (r.keys != keys0) {
      open_doors<MAPK>(p, e, r.keys, ws, lane);
      mark_border<MAPK>(p, ws, r.cx, r.cy, lane);
    }
  } else {
    heading(p, r, c, s);
  }
  render_env<MODE, MAPK, COLS, GRAY>(p, e, r, c, s, ws, lane, slot, p.frames + (size_t)e * frame_bytes, q.k01);
  __syncwarp();
  return true;
}

// A kernel's dynamic shared memory limit is a property of the function, shared
// by every env in the process: it is raised to the device's opt-in maximum (never
// lowered), so envs of different sizes can coexist.
template <class Kernel>
cudaError_t raise_smem_limit(Kernel kernel) {
  int dev = 0, optin = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (err == cudaSuccess) err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  return err;
}

}  // namespace
}  // namespace jx
