/*
 * jx_oracle.c — plain FP64 CPU oracle of the batched first-person environment
 * step + render (JAXenstein, arxiv 2605.19926).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline / reference leg, never by the product path.
 * It shares no code with the CUDA library.
 *
 * Each function below follows one passage of the paper (or, where the paper
 * is silent, one stated reading) and does it the slow, literal way: one
 * environment at a time, one ray per column, one pixel at a time, in double
 * precision. No blocking, no fusion, no precomputed tables.
 */
#include "jx_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define PI 3.14159265358979323846
#define HMAX (1 << 20) /* slice heights are clamped here (only reached for perp ~ 0) */

/* ---------------------------------------------------------------- RNG ----
 * SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): the state advances by the golden-ratio
 * increment and each output is the state passed through the 64-bit
 * finaliser. The n-th output of the generator seeded with s is therefore
 * mix(s + n * gamma). */
static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t jxo_splitmix64(uint64_t seed, uint64_t n) {
  return mix64(seed + n * 0x9E3779B97F4A7C15ULL);
}

/* Stream keys are chained: the env's key is output env+1 of the master
 * generator, the episode's key is output episode+1 of the env's generator,
 * and so on; draw `index` is output index+1 of the purpose's generator. */
uint64_t jxo_draw(uint64_t seed, uint32_t env, uint32_t episode, uint32_t purpose, uint32_t index) {
  uint64_t k_env = jxo_splitmix64(seed, (uint64_t)env + 1);
  uint64_t k_ep = jxo_splitmix64(k_env, (uint64_t)episode + 1);
  uint64_t k_p = jxo_splitmix64(k_ep, (uint64_t)purpose + 1);
  return jxo_splitmix64(k_p, (uint64_t)index + 1);
}

/* Uniform integer in [0, n): the high 32 bits of the draw scaled by n
 * (Lemire's multiply-shift). */
static uint32_t uniform_below(uint64_t draw, uint32_t n) {
  return (uint32_t)(((draw >> 32) * (uint64_t)n) >> 32);
}

/* Uniform heading in [0, 2*pi) from the top 24 bits of a draw. */
static double heading_from_draw(uint64_t draw) {
  double frac = (double)(draw >> 40) * (1.0 / 16777216.0);
  return (2.0 * PI) * frac;
}

int jxo_sizeof_env(void) { return (int)sizeof(jxo_env); }
int jxo_sizeof_config(void) { return (int)sizeof(jxo_config); }
int jxo_sizeof_ray(void) { return (int)sizeof(jxo_ray); }

/* ------------------------------------------------------------ palette ----
 * The paper renders untextured walls, a red key, a red locked door and a
 * yellow goal (Table 1, Table 2). The exact RGB values are this
 * implementation's choice; they are fixed. */
static void set_rgb(uint8_t rgb[3], int r, int g, int b) {
  rgb[0] = (uint8_t)r;
  rgb[1] = (uint8_t)g;
  rgb[2] = (uint8_t)b;
}
static void wall_rgb(int v, uint8_t rgb[3]) {
  switch (v) {
    case 2: set_rgb(rgb, 64, 160, 64); break;
    case 3: set_rgb(rgb, 64, 96, 192); break;
    case 4: set_rgb(rgb, 176, 144, 80); break;
    case 5: set_rgb(rgb, 200, 100, 40); break;
    case 6: set_rgb(rgb, 112, 64, 160); break;
    case 7: set_rgb(rgb, 40, 160, 160); break;
    case 8: set_rgb(rgb, 128, 128, 48); break;
    case 9: set_rgb(rgb, 216, 216, 216); break;
    case JXO_LOCKED + 0: set_rgb(rgb, 200, 32, 32); break;
    case JXO_LOCKED + 1: set_rgb(rgb, 32, 64, 200); break;
    case JXO_LOCKED + 2: set_rgb(rgb, 208, 184, 32); break;
    case JXO_UNLOCKED + 0: set_rgb(rgb, 232, 120, 120); break;
    case JXO_UNLOCKED + 1: set_rgb(rgb, 120, 150, 232); break;
    case JXO_UNLOCKED + 2: set_rgb(rgb, 236, 222, 128); break;
    default: set_rgb(rgb, 160, 160, 160); break; /* type 1 and anything else */
  }
}
static const uint8_t CEIL_RGB[3] = {48, 48, 56};
static const uint8_t FLOOR_RGB[3] = {104, 96, 88};
static void sprite_rgb(int type, uint8_t rgb[3]) {
  switch (type) {
    case JXO_SPR_KEY: set_rgb(rgb, 224, 40, 40); break;
    case JXO_SPR_GOAL: set_rgb(rgb, 240, 208, 32); break;
    case JXO_SPR_KEY_BLUE: set_rgb(rgb, 40, 80, 224); break;
    case JXO_SPR_KEY_YELLOW: set_rgb(rgb, 232, 200, 40); break;
    default: set_rgb(rgb, 144, 64, 192); break;
  }
}
/* colour of a key sprite type, -1 for other types */
static int key_colour(int type) {
  return type == JXO_SPR_KEY ? 0 : (type == JXO_SPR_KEY_BLUE ? 1 : (type == JXO_SPR_KEY_YELLOW ? 2 : -1));
}

/* ---------------------------------------------------------------- map ---- */
static int config_ok(const jxo_config* cfg) {
  int S = cfg->map_side;
  if (S < 3 || S > JXO_MAX_SIDE) return 0;
  if (cfg->frame_h < 1 || cfg->frame_w < 1) return 0;
  if (cfg->max_sprites < 0 || cfg->max_sprites > JXO_MAX_SPRITES) return 0;
  if (cfg->turns_per_rev < 1) return 0;
  if (cfg->task == JXO_TASK_MAZE_KEYDOOR || cfg->task == JXO_TASK_MAZE_ROOMS) {
    if (S < 6 || (S % 2) != 0 || cfg->max_sprites < 2) return 0;
  } else if (cfg->task == JXO_TASK_ASCII) {
    const jxo_ascii* a = (const jxo_ascii*)(uintptr_t)cfg->ascii;
    if (!a || a->side != S || cfg->max_sprites < a->n_keys + (a->n_goal > 0)) return 0;
  } else if (cfg->task != JXO_TASK_ROOMS) {
    return 0;
  }
  return 1;
}

/* A cell outside the map reads as a type-1 wall. */
static int cell_value(const jxo_config* cfg, const jxo_env* e, int x, int y) {
  int S = cfg->map_side;
  if (x < 0 || y < 0 || x >= S || y >= S) return 1;
  return e->map[y * S + x];
}

/* Walls and closed doors are solid; a locked door is open (floor) while the
 * key of its colour is held (Table 2: locked doors open with their key). */
static int is_solid(const jxo_config* cfg, const jxo_env* e, int x, int y) {
  int v = cell_value(cfg, e, x, y);
  if (v == JXO_FLOOR) return 0;
  if (v >= JXO_LOCKED && v < JXO_LOCKED + 3 && ((e->keys >> (v - JXO_LOCKED)) & 1)) return 0;
  return 1;
}

/* -------------------------------------------------------- generators ---- */
static int is_border(int S, int x, int y) { return x == 0 || y == 0 || x == S - 1 || y == S - 1; }

/* Rooms task: border walls; each interior cell is a wall when a uniform
 * draw in [0, 1) (53 bits) is below wall_prob; wall type 1 + (draw mod 4). */
static void gen_rooms(const jxo_config* cfg, int32_t env, uint32_t ep, jxo_env* e) {
  int S = cfg->map_side;
  uint64_t seed = cfg->seed;
  for (int y = 0; y < S; ++y)
    for (int x = 0; x < S; ++x) {
      uint64_t u = jxo_draw(seed, (uint32_t)env, ep, JXO_P_WALL, (uint32_t)(y * S + x));
      int wall;
      if (is_border(S, x, y)) {
        wall = 1;
      } else {
        double uniform = (double)(u >> 11) * (1.0 / 9007199254740992.0);
        wall = uniform < cfg->wall_prob;
      }
      e->map[y * S + x] = wall ? (uint8_t)(1 + (u & 3)) : JXO_FLOOR;
    }
  int n_free = 0;
  for (int i = 0; i < S * S; ++i) n_free += e->map[i] == JXO_FLOOR;
  if (n_free == 0) {
    e->map[(S / 2) * S + S / 2] = JXO_FLOOR;
    n_free = 1;
  }
  /* spawn: the centre of a uniformly chosen free cell (row-major enumeration) */
  uint32_t pick = uniform_below(jxo_draw(seed, (uint32_t)env, ep, JXO_P_SPAWN, 0), (uint32_t)n_free);
  int seen = 0;
  for (int i = 0; i < S * S; ++i) {
    if (e->map[i] != JXO_FLOOR) continue;
    if ((uint32_t)seen == pick) {
      e->x = (i % S) + 0.5;
      e->y = (i / S) + 0.5;
      break;
    }
    ++seen;
  }
  e->key_x = e->key_y = e->goal_x = e->goal_y = e->door_x = e->door_y = -1;
  /* decorative sprites: how many, then each on a uniformly chosen free cell */
  e->n_sprites = 0;
  if (cfg->max_sprites > 0) {
    uint32_t n = uniform_below(jxo_draw(seed, (uint32_t)env, ep, JXO_P_NSPRITES, 0),
                               (uint32_t)cfg->max_sprites + 1);
    for (uint32_t k = 0; k < n; ++k) {
      uint32_t c = uniform_below(jxo_draw(seed, (uint32_t)env, ep, JXO_P_SPRITE_CELL, k), (uint32_t)n_free);
      int s2 = 0;
      for (int i = 0; i < S * S; ++i) {
        if (e->map[i] != JXO_FLOOR) continue;
        if ((uint32_t)s2 == c) {
          e->spr_x[k] = (i % S) + 0.5;
          e->spr_y[k] = (i / S) + 0.5;
          e->spr_type[k] = JXO_SPR_DISTRACTOR;
          break;
        }
        ++s2;
      }
    }
    e->n_sprites = (int32_t)n;
  }
}

/* Key-door maze task: a random depth-first ("recursive backtracker") maze on
 * the nodes at odd coordinates 1, 3, ..., S-3, with 1-cell corridors. The DFS
 * starts at the spawn node; at each step it picks uniformly among the
 * unvisited neighbours listed in N, E, S, W order, using one draw per carved
 * passage. The goal is the cell farthest (BFS) from the spawn, ties to the
 * smallest (y, x). The locked door sits on the passage of edge ceil(m/2) of
 * the m-edge spawn-to-goal path. The key is uniform over the nodes reachable
 * from the spawn without crossing the door, the spawn itself excluded (the
 * spawn when there is no other). */
static int gen_maze(const jxo_config* cfg, int32_t env, uint32_t ep, jxo_env* e) {
  int S = cfg->map_side;
  int nn = (S - 2) / 2;
  int n_nodes = nn * nn;
  uint64_t seed = cfg->seed;
  for (int i = 0; i < S * S; ++i)
    e->map[i] = (uint8_t)(1 + (jxo_draw(seed, (uint32_t)env, ep, JXO_P_WALL, (uint32_t)i) & 3));

  int start = (int)uniform_below(jxo_draw(seed, (uint32_t)env, ep, JXO_P_SPAWN, 0), (uint32_t)n_nodes);
  int* stack = (int*)malloc(sizeof(int) * n_nodes);
  uint8_t* visited = (uint8_t*)calloc((size_t)n_nodes, 1);
  int sp = 0;
  uint32_t carved = 0;
  stack[sp++] = start;
  visited[start] = 1;
  e->map[(2 * (start / nn) + 1) * S + 2 * (start % nn) + 1] = JXO_FLOOR;
  while (sp > 0) {
    int v = stack[sp - 1];
    int vx = v % nn, vy = v / nn;
    int cand[4], k = 0;
    if (vy > 0 && !visited[v - nn]) cand[k++] = v - nn;      /* N */
    if (vx < nn - 1 && !visited[v + 1]) cand[k++] = v + 1;   /* E */
    if (vy < nn - 1 && !visited[v + nn]) cand[k++] = v + nn; /* S */
    if (vx > 0 && !visited[v - 1]) cand[k++] = v - 1;        /* W */
    if (k == 0) {
      --sp;
      continue;
    }
    int w = cand[uniform_below(jxo_draw(seed, (uint32_t)env, ep, JXO_P_DFS, carved), (uint32_t)k)];
    ++carved;
    int cvx = 2 * vx + 1, cvy = 2 * vy + 1;
    int cwx = 2 * (w % nn) + 1, cwy = 2 * (w / nn) + 1;
    e->map[((cvy + cwy) / 2) * S + (cvx + cwx) / 2] = JXO_FLOOR;
    e->map[cwy * S + cwx] = JXO_FLOOR;
    visited[w] = 1;
    stack[sp++] = w;
  }
  free(stack);
  free(visited);

  /* breadth-first distances over free cells from the spawn cell */
  int n_cells = S * S;
  int* dist = (int*)malloc(sizeof(int) * n_cells);
  int* parent = (int*)malloc(sizeof(int) * n_cells);
  int* queue = (int*)malloc(sizeof(int) * n_cells);
  for (int i = 0; i < n_cells; ++i) dist[i] = -1, parent[i] = -1;
  int s_cell = (2 * (start / nn) + 1) * S + 2 * (start % nn) + 1;
  int qh = 0, qt = 0;
  queue[qt++] = s_cell;
  dist[s_cell] = 0;
  while (qh < qt) {
    int c = queue[qh++];
    int cx = c % S, cy = c / S;
    const int dxs[4] = {0, 1, 0, -1}, dys[4] = {-1, 0, 1, 0};
    for (int d = 0; d < 4; ++d) {
      int nx = cx + dxs[d], ny = cy + dys[d];
      if (nx < 0 || ny < 0 || nx >= S || ny >= S) continue;
      int nc = ny * S + nx;
      if (e->map[nc] != JXO_FLOOR || dist[nc] >= 0) continue;
      dist[nc] = dist[c] + 1;
      parent[nc] = c;
      queue[qt++] = nc;
    }
  }
  int goal = s_cell;
  for (int i = 0; i < n_cells; ++i)
    if (dist[i] > dist[goal]) goal = i;

  /* spawn-to-goal path and the door on edge ceil(m/2) */
  int L = dist[goal];
  int* path = (int*)malloc(sizeof(int) * (L + 1));
  for (int i = L, c = goal; i >= 0; --i) {
    path[i] = c;
    c = parent[c];
  }
  int m = L / 2;
  int door = -1;
  if (m >= 1) {
    int j = (m + 1) / 2;
    door = path[2 * j - 1];
    e->map[door] = JXO_DOOR;
  }
  free(path);

  /* nodes reachable from the spawn with the door closed */
  uint8_t* reach = (uint8_t*)calloc((size_t)n_cells, 1);
  qh = qt = 0;
  queue[qt++] = s_cell;
  reach[s_cell] = 1;
  while (qh < qt) {
    int c = queue[qh++];
    int cx = c % S, cy = c / S;
    const int dxs[4] = {0, 1, 0, -1}, dys[4] = {-1, 0, 1, 0};
    for (int d = 0; d < 4; ++d) {
      int nx = cx + dxs[d], ny = cy + dys[d];
      if (nx < 0 || ny < 0 || nx >= S || ny >= S) continue;
      int nc = ny * S + nx;
      if (e->map[nc] != JXO_FLOOR || reach[nc]) continue;
      reach[nc] = 1;
      queue[qt++] = nc;
    }
  }
  int n_side = 0;
  for (int y = 1; y < S; y += 2)
    for (int x = 1; x < S; x += 2) {
      int c = y * S + x;
      if (y <= S - 3 && x <= S - 3 && reach[c] && c != s_cell) ++n_side;
    }
  int key = s_cell;
  if (n_side > 0) {
    uint32_t pick = uniform_below(jxo_draw(seed, (uint32_t)env, ep, JXO_P_KEY, 0), (uint32_t)n_side);
    int seen = 0;
    for (int y = 1; y <= S - 3 && key == s_cell; y += 2)
      for (int x = 1; x <= S - 3; x += 2) {
        int c = y * S + x;
        if (!reach[c] || c == s_cell) continue;
        if ((uint32_t)seen == pick) {
          key = c;
          break;
        }
        ++seen;
      }
  }
  free(reach);
  free(queue);
  free(parent);
  free(dist);

  e->x = (s_cell % S) + 0.5;
  e->y = (s_cell / S) + 0.5;
  e->key_x = key % S;
  e->key_y = key / S;
  e->goal_x = goal % S;
  e->goal_y = goal / S;
  e->door_x = door >= 0 ? door % S : -1;
  e->door_y = door >= 0 ? door / S : -1;
  e->n_sprites = 2;
  e->spr_x[0] = e->key_x + 0.5;
  e->spr_y[0] = e->key_y + 0.5;
  e->spr_type[0] = JXO_SPR_KEY;
  e->spr_x[1] = e->goal_x + 0.5;
  e->spr_y[1] = e->goal_y + 0.5;
  e->spr_type[1] = JXO_SPR_GOAL;
  return 0;
}

/* Maze with rooms (the large-scale workload): the key-door maze above, then
 * S*S/1024 open rooms of 8 x 8 cells, room r with its top-left cell at
 * (1 + u mod (S - 9), 1 + u' mod (S - 9)) from draws 2r and 2r+1 of the room
 * stream, every cell inside turned to floor except the locked door; then a
 * uniform number in [0, K-2] of distractor sprites after the key and the goal,
 * each on a uniformly chosen floor cell (row-major enumeration of the final
 * map). Rooms only add floor, so every floor cell stays reachable; they may
 * open a way around the door. */
static void gen_maze_rooms(const jxo_config* cfg, int32_t env, uint32_t ep, jxo_env* e) {
  int S = cfg->map_side;
  uint64_t seed = cfg->seed;
  gen_maze(cfg, env, ep, e);
  int n_rooms = (S * S) / 1024;
  for (int r = 0; r < n_rooms; ++r) {
    int x0 = 1 + (int)uniform_below(jxo_draw(seed, (uint32_t)env, ep, JXO_P_ROOM, (uint32_t)(2 * r)), (uint32_t)(S - 9));
    int y0 = 1 + (int)uniform_below(jxo_draw(seed, (uint32_t)env, ep, JXO_P_ROOM, (uint32_t)(2 * r + 1)),
                                    (uint32_t)(S - 9));
    for (int y = y0; y < y0 + 8; ++y)
      for (int x = x0; x < x0 + 8; ++x)
        if (e->map[y * S + x] != JXO_DOOR) e->map[y * S + x] = JXO_FLOOR;
  }
  int n_free = 0;
  for (int i = 0; i < S * S; ++i) n_free += e->map[i] == JXO_FLOOR;
  uint32_t n = uniform_below(jxo_draw(seed, (uint32_t)env, ep, JXO_P_NSPRITES, 0), (uint32_t)cfg->max_sprites - 1);
  for (uint32_t k = 0; k < n; ++k) {
    uint32_t c = uniform_below(jxo_draw(seed, (uint32_t)env, ep, JXO_P_SPRITE_CELL, k), (uint32_t)n_free);
    int seen = 0;
    for (int i = 0; i < S * S; ++i) {
      if (e->map[i] != JXO_FLOOR) continue;
      if ((uint32_t)seen == c) {
        e->spr_x[2 + k] = (i % S) + 0.5;
        e->spr_y[2 + k] = (i / S) + 0.5;
        e->spr_type[2 + k] = JXO_SPR_DISTRACTOR;
        break;
      }
      ++seen;
    }
  }
  e->n_sprites = 2 + (int32_t)n;
}

/* ASCII maps (Table 2): each episode starts from the parsed map: the spawn
 * uniform over the 'S' cells (over all floor cells when there is none), the
 * goal sprite on one 'G' cell drawn uniformly each episode (DMLab's random
 * goal; the only one when there is one), the keys as sprites on their cells
 * in row-major order, then the goal. Doors start as written. */
static void gen_ascii(const jxo_config* cfg, int32_t env, uint32_t ep, jxo_env* e) {
  const jxo_ascii* a = (const jxo_ascii*)(uintptr_t)cfg->ascii;
  int S = cfg->map_side;
  uint64_t seed = cfg->seed;
  memcpy(e->map, a->map, (size_t)S * S);
  uint64_t d = jxo_draw(seed, (uint32_t)env, ep, JXO_P_SPAWN, 0);
  int cell = 0;
  if (a->n_spawn > 0) {
    cell = a->spawn[uniform_below(d, (uint32_t)a->n_spawn)];
  } else {
    int n_free = 0;
    for (int i = 0; i < S * S; ++i) n_free += e->map[i] == JXO_FLOOR;
    uint32_t pick = uniform_below(d, (uint32_t)n_free);
    for (int i = 0, seen = 0; i < S * S; ++i) {
      if (e->map[i] != JXO_FLOOR) continue;
      if ((uint32_t)seen++ == pick) {
        cell = i;
        break;
      }
    }
  }
  e->x = (cell % S) + 0.5;
  e->y = (cell / S) + 0.5;
  int k = 0;
  const int key_type[3] = {JXO_SPR_KEY, JXO_SPR_KEY_BLUE, JXO_SPR_KEY_YELLOW};
  for (int i = 0; i < a->n_keys; ++i, ++k) {
    e->spr_x[k] = (a->key_cell[i] % S) + 0.5;
    e->spr_y[k] = (a->key_cell[i] / S) + 0.5;
    e->spr_type[k] = key_type[a->key_colour[i]];
  }
  e->key_x = a->n_keys ? a->key_cell[0] % S : -1;
  e->key_y = a->n_keys ? a->key_cell[0] / S : -1;
  e->goal_x = e->goal_y = -1;
  if (a->n_goal > 0) {
    int g = a->goal[uniform_below(jxo_draw(seed, (uint32_t)env, ep, JXO_P_GOAL, 0), (uint32_t)a->n_goal)];
    e->spr_x[k] = (g % S) + 0.5;
    e->spr_y[k] = (g / S) + 0.5;
    e->spr_type[k] = JXO_SPR_GOAL;
    ++k;
    e->goal_x = g % S;
    e->goal_y = g / S;
  }
  e->door_x = e->door_y = -1;
  for (int i = 0; i < S * S; ++i)
    if (e->map[i] >= JXO_LOCKED && e->map[i] < JXO_LOCKED + 3) {
      e->door_x = i % S;
      e->door_y = i / S;
      break;
    }
  e->n_sprites = k;
}

int jxo_sizeof_ascii(void) { return (int)sizeof(jxo_ascii); }

int jxo_parse_ascii(const char* text, int32_t side, jxo_ascii* a) {
  if (!text || !a || side < 3 || side > JXO_MAX_SIDE) return -1;
  memset(a, 0, sizeof(*a));
  a->side = side;
  for (int i = 0; i < side * side; ++i) a->map[i] = 1;
  int row = 0, col = 0, n_floor = 0;
  for (const char* q = text; *q; ++q) {
    char ch = *q;
    if (ch == '\n') {
      ++row;
      col = 0;
      continue;
    }
    if (ch == '\r') continue;
    if ((unsigned char)ch < 32 || (unsigned char)ch > 126) return -1;
    if (row >= side || col >= side) return -1;
    int cell = row * side + col, v;
    switch (ch) {
      case '#': v = 1; break;
      case '.': case ' ': v = JXO_FLOOR; break;
      case 'S': v = JXO_FLOOR; a->spawn[a->n_spawn++] = cell; break;
      case 'G': v = JXO_FLOOR; a->goal[a->n_goal++] = cell; break;
      case 'r': case 'b': case 'y':
        if (a->n_keys == JXO_MAX_SPRITES) return -1;
        v = JXO_FLOOR;
        a->key_cell[a->n_keys] = cell;
        a->key_colour[a->n_keys++] = ch == 'r' ? 0 : (ch == 'b' ? 1 : 2);
        break;
      case '"': v = JXO_UNLOCKED + 1; break;
      case '\\': v = JXO_UNLOCKED + 2; break;
      case 'R': v = JXO_LOCKED + 0; break;
      case 'B': v = JXO_LOCKED + 1; break;
      case 'Y': v = JXO_LOCKED + 2; break;
      default: v = (ch >= '1' && ch <= '9') ? ch - '0' : 1 + ((unsigned char)ch % 9); break;
    }
    a->map[cell] = (uint8_t)v;
    n_floor += v == JXO_FLOOR;
    ++col;
  }
  return n_floor > 0 ? 0 : -1;
}

void jxo_gray(const uint8_t* rgb, int64_t n, uint8_t* out) {
  for (int64_t i = 0; i < n; ++i)
    out[i] = (uint8_t)((77 * (int)rgb[3 * i] + 150 * (int)rgb[3 * i + 1] + 29 * (int)rgb[3 * i + 2] + 128) >> 8);
}

int jxo_generate(const jxo_config* cfg, int32_t env_index, uint32_t episode, jxo_env* out) {
  if (!config_ok(cfg)) return -1;
  memset(out, 0, sizeof(*out));
  out->episode = episode;
  out->t = 0;
  out->turn = 0;
  out->keys = 0;
  if (cfg->task == JXO_TASK_ROOMS)
    gen_rooms(cfg, env_index, episode, out);
  else if (cfg->task == JXO_TASK_ASCII)
    gen_ascii(cfg, env_index, episode, out);
  else if (cfg->task == JXO_TASK_MAZE_ROOMS)
    gen_maze_rooms(cfg, env_index, episode, out);
  else
    gen_maze(cfg, env_index, episode, out);
  out->theta0 = heading_from_draw(jxo_draw(cfg->seed, (uint32_t)env_index, episode, JXO_P_HEADING, 0));
  return 0;
}

/* ------------------------------------------------------------- camera ---- */
static double heading(const jxo_config* cfg, const jxo_env* e) {
  return e->theta0 + (double)e->turn * (2.0 * PI / (double)cfg->turns_per_rev);
}

/* ----------------------------------------------------------------- step ----
 * Movement with wall collision: the agent is an axis-aligned box of
 * half-size r; a move is tried along x, then along y, and each axis is
 * rejected on its own when the box at the new position overlaps a solid cell
 * (closed intervals, touching counts). */
static int box_free_margin(const jxo_config* cfg, const jxo_env* e, double px, double py, double grow) {
  double r = cfg->radius + grow;
  int x0 = (int)floor(px - r), x1 = (int)floor(px + r);
  int y0 = (int)floor(py - r), y1 = (int)floor(py + r);
  for (int j = y0; j <= y1; ++j)
    for (int i = x0; i <= x1; ++i)
      if (is_solid(cfg, e, i, j)) return 0;
  return 1;
}
static int box_free(const jxo_config* cfg, const jxo_env* e, double px, double py) {
  return box_free_margin(cfg, e, px, py, 0.0);
}
/* a collision decision that moving the box edges by JXO_EPS_CELL could flip */
static int box_near_tie(const jxo_config* cfg, const jxo_env* e, double px, double py) {
  return box_free_margin(cfg, e, px, py, JXO_EPS_CELL) != box_free_margin(cfg, e, px, py, -JXO_EPS_CELL);
}

/* An unlocked door opens when the agent walks into it (there is no separate
 * toggle action): every unlocked door cell the rejected box overlaps becomes
 * floor. */
static void open_unlocked(const jxo_config* cfg, jxo_env* e, double px, double py) {
  int S = cfg->map_side;
  double r = cfg->radius;
  int x0 = (int)floor(px - r), x1 = (int)floor(px + r);
  int y0 = (int)floor(py - r), y1 = (int)floor(py + r);
  for (int j = y0; j <= y1; ++j)
    for (int i = x0; i <= x1; ++i) {
      if (i < 0 || j < 0 || i >= S || j >= S) continue;
      int v = e->map[j * S + i];
      if (v >= JXO_UNLOCKED && v < JXO_UNLOCKED + 3) e->map[j * S + i] = JXO_FLOOR;
    }
}

/* Key and goal events at position (px, py): a key sprite whose cell is the
 * agent's cell and whose colour is not held yet is picked up (its colour
 * bit into *picked); a goal sprite there is reached. */
static int pickup_events(const jxo_env* e, double px, double py, int* picked) {
  int cx = (int)floor(px), cy = (int)floor(py);
  int ev = 0, bits = 0;
  for (int j = 0; j < e->n_sprites; ++j) {
    if ((int)floor(e->spr_x[j]) != cx || (int)floor(e->spr_y[j]) != cy) continue;
    int c = key_colour(e->spr_type[j]);
    if (c >= 0 && !((e->keys >> c) & 1)) {
      ev |= JXO_EV_KEY;
      bits |= 1 << c;
    }
    if (e->spr_type[j] == JXO_SPR_GOAL) ev |= JXO_EV_GOAL;
  }
  if (picked) *picked = bits;
  return ev;
}

/* A collision test with its finite-precision tie taken a chosen way: bias 0
 * the exact test; +1 a test that growing or shrinking the box by
 * JXO_EPS_CELL would flip lets the box move (the smaller box's answer), -1
 * blocks it (the larger box's answer). */
static int box_free_biased(const jxo_config* cfg, const jxo_env* e, double px, double py, int32_t bias) {
  if (bias != 0 && box_near_tie(cfg, e, px, py)) return bias > 0;
  return box_free(cfg, e, px, py);
}

/* One step (movement, collision, key / goal events, reward, episode end,
 * auto-reset). coll_x / coll_y bias the x and y collision tests as
 * box_free_biased; pick_x / pick_y (-1, 0, +1) move the point where key and
 * goal events are evaluated by that many JXO_EPS_CELL along x and y. All zero
 * is the exact step. */
static int step_impl(const jxo_config* cfg, int32_t env_index, jxo_env* e, int32_t action, int32_t coll_x,
                     int32_t coll_y, int32_t pick_x, int32_t pick_y, double* reward, int32_t* done,
                     int32_t* events) {
  if (!config_ok(cfg) || action < 0 || action > 6) return -1;
  double th = heading(cfg, e);
  double c = cos(th), s = sin(th);
  double ms = cfg->move_step;
  double dx = 0.0, dy = 0.0;
  switch (action) {
    case JXO_FWD: dx = ms * c; dy = ms * s; break;
    case JXO_BACK: dx = -ms * c; dy = -ms * s; break;
    case JXO_STRAFE_L: dx = ms * s; dy = -ms * c; break;  /* minus the right vector (-s, c) */
    case JXO_STRAFE_R: dx = -ms * s; dy = ms * c; break;
    case JXO_TURN_L: e->turn = (e->turn + cfg->turns_per_rev - 1) % cfg->turns_per_rev; break;
    case JXO_TURN_R: e->turn = (e->turn + 1) % cfg->turns_per_rev; break;
    default: break;
  }
  int near = 0;
  double nx = e->x + dx;
  near |= box_near_tie(cfg, e, nx, e->y);
  if (!box_free_biased(cfg, e, nx, e->y, coll_x)) {
    open_unlocked(cfg, e, nx, e->y);
    nx = e->x;
  }
  double ny = e->y + dy;
  near |= box_near_tie(cfg, e, nx, ny);
  if (!box_free_biased(cfg, e, nx, ny, coll_y)) {
    open_unlocked(cfg, e, nx, ny);
    ny = e->y;
  }
  e->x = nx;
  e->y = ny;

  int picked = 0;
  int ev = pickup_events(e, nx + pick_x * JXO_EPS_CELL, ny + pick_y * JXO_EPS_CELL, &picked);
  /* a key or goal event that moving the position by JXO_EPS_CELL could flip */
  int ev0 = pickup_events(e, nx, ny, NULL);
  for (int k = 0; k < 4; ++k) {
    double px = nx + ((k & 1) ? JXO_EPS_CELL : -JXO_EPS_CELL);
    double py = ny + ((k & 2) ? JXO_EPS_CELL : -JXO_EPS_CELL);
    if (pickup_events(e, px, py, NULL) != ev0) near = 1;
  }
  e->keys |= picked;
  *reward = cfg->step_reward + ((ev & JXO_EV_KEY) ? cfg->key_reward : 0.0) +
            ((ev & JXO_EV_GOAL) ? cfg->goal_reward : 0.0);
  e->t += 1;
  int d = (ev & JXO_EV_GOAL) || (cfg->horizon > 0 && e->t >= cfg->horizon);
  *done = d;
  *events = ev | (near ? JXO_EV_NEAR_TIE : 0);
  if (d) jxo_generate(cfg, env_index, e->episode + 1, e);
  return 0;
}

int jxo_step(const jxo_config* cfg, int32_t env_index, jxo_env* e, int32_t action, double* reward,
             int32_t* done, int32_t* events) {
  return step_impl(cfg, env_index, e, action, 0, 0, 0, 0, reward, done, events);
}

int jxo_step_biased(const jxo_config* cfg, int32_t env_index, jxo_env* e, int32_t action, int32_t coll_x,
                    int32_t coll_y, int32_t pick_x, int32_t pick_y, double* reward, int32_t* done,
                    int32_t* events) {
  if (coll_x < -1 || coll_x > 1 || coll_y < -1 || coll_y > 1 || pick_x < -1 || pick_x > 1 || pick_y < -1 ||
      pick_y > 1)
    return -1;
  return step_impl(cfg, env_index, e, action, coll_x, coll_y, pick_x, pick_y, reward, done, events);
}

/* ------------------------------------------------------------ raycast ----
 * DDA (Sec. 2.1): march from tile boundary to tile boundary along the ray
 * origin + t * (rx, ry). The next x boundary is reached at
 * t = (kx + gx) / |rx|, kx = 0, 1, ...; gx is the distance from the origin to
 * the first x boundary in the direction of travel (likewise for y). The
 * nearer boundary is crossed (x on a strict "less", y otherwise); the first
 * solid cell entered is the hit and its t is reported as perp. */
int jxo_cast(const jxo_config* cfg, const jxo_env* e, double ox, double oy, double rx, double ry,
             int32_t bias, jxo_ray* out) {
  int S = cfg->map_side;
  int mx = (int)floor(ox), my = (int)floor(oy);
  int sx = rx < 0 ? -1 : 1, sy = ry < 0 ? -1 : 1;
  double ax = fabs(rx), ay = fabs(ry);
  double gx = rx < 0 ? ox - mx : (mx + 1) - ox;
  double gy = ry < 0 ? oy - my : (my + 1) - oy;
  double len = sqrt(rx * rx + ry * ry);
  long kx = 0, ky = 0;
  memset(out, 0, sizeof(*out));
  out->cell_x = out->cell_y = -1;
  out->side = -1;
  out->perp = INFINITY;
  for (int it = 0; it < 4 * S + 8; ++it) {
    double tx = ax > 0 ? (kx + gx) / ax : INFINITY;
    double ty = ay > 0 ? (ky + gy) / ay : INFINITY;
    int take_x = tx < ty;
    if (bias != 0 && fabs(tx - ty) * len < JXO_EPS_CELL) take_x = bias > 0;
    double t;
    int side;
    if (take_x) {
      t = tx;
      ++kx;
      mx += sx;
      side = 0;
    } else {
      t = ty;
      ++ky;
      my += sy;
      side = 1;
    }
    if (is_solid(cfg, e, mx, my)) {
      out->cell_x = mx;
      out->cell_y = my;
      out->side = side;
      out->perp = t;
      return 0;
    }
  }
  return 0;
}

/* Slice from the hit distance: h = floor(H / perp + 1/2) rows, centred:
 * top = floor((H - h) / 2), bot = top + h, both clamped to [0, H]. */
static void slice_rows(int H, double perp, jxo_ray* r) {
  int h;
  double v = 0.0;
  if (!(perp > 0.0)) {
    h = HMAX;
  } else {
    v = (double)H / perp + 0.5;
    h = v >= (double)HMAX ? HMAX : (int)floor(v);
  }
  int top = (int)floor((double)(H - h) / 2.0);
  int bot = top + h;
  r->h = h;
  r->top = top < 0 ? 0 : (top > H ? H : top);
  r->bot = bot < 0 ? 0 : (bot > H ? H : bot);
  r->h_ambiguous = 0;
  if (perp > 0.0 && v < (double)HMAX) {
    double f = v - floor(v);
    double tol = JXO_EPS_REL * v;
    if (f < tol || 1.0 - f < tol) r->h_ambiguous = 1;
  }
}

/* a key whose colour is held is no longer drawn */
static int sprite_visible(const jxo_env* e, int j) {
  int type = e->spr_type[j];
  if (type == JXO_SPR_NONE) return 0;
  int c = key_colour(type);
  if (c >= 0 && ((e->keys >> c) & 1)) return 0;
  return 1;
}

/* Type masks over normalised sprite coordinates (u, v) in [0, 1)^2:
 * key = diamond, goal = full rectangle, distractor = disc. Returns the
 * signed margin (> 0 inside); the rectangle's own edges are tested apart. */
static double mask_margin(int type, double u, double v) {
  double a = 2.0 * u - 1.0, b = 2.0 * v - 1.0;
  if (key_colour(type) >= 0) return 1.0 - (fabs(a) + fabs(b));
  if (type == JXO_SPR_GOAL) return 1.0;
  return 1.0 - (a * a + b * b);
}

typedef struct {
  int ok;
  double ty, x0, w, top, hgt;
} sprite_screen;

/* Billboard sprites (Fig. 1): a sprite of world width and height 0.5
 * standing on the floor, drawn against the per-column depth buffer. With the
 * view direction d, the right vector r = (-sin, cos) and the camera plane
 * p = tan(fov/2) r, the sprite offset v = tx p + ty d gives depth ty and
 * screen centre column W/2 (1 + tx / ty). */
static sprite_screen project_sprite(const jxo_config* cfg, const jxo_env* e, int j, double c, double s,
                                    double T) {
  sprite_screen o;
  int H = cfg->frame_h, W = cfg->frame_w;
  double vx = e->spr_x[j] - e->x, vy = e->spr_y[j] - e->y;
  o.ty = vx * c + vy * s;
  double tx = (-vx * s + vy * c) / T;
  o.ok = o.ty > 0.1;
  double scx = 0.5 * W * (1.0 + tx / o.ty);
  double hw = 0.5 * W * 0.25 / (T * o.ty);
  o.x0 = scx - hw;
  o.w = 2.0 * hw;
  o.top = 0.5 * H;
  o.hgt = 0.5 * H / o.ty;
  return o;
}

/* The frame with every column's ray cast under `bias` (see jxo_cast): 0 the
 * exact frame. A biased frame is one of the frames a corner ray admits, so
 * its ambiguity flags leave out the whole-column flag of corner rays (the
 * caller compares such a column against the variant its ray took). */
static int render_impl(const jxo_config* cfg, const jxo_env* e, uint8_t* frame, jxo_ray* rays,
                       uint8_t* ambiguous, int32_t bias) {
  if (!config_ok(cfg)) return -1;
  int H = cfg->frame_h, W = cfg->frame_w;
  double th = heading(cfg, e);
  double c = cos(th), s = sin(th);
  double T = tan(0.5 * cfg->fov_deg * PI / 180.0);
  int want_flags = rays != NULL || ambiguous != NULL;
  jxo_ray* col_rays = (jxo_ray*)malloc(sizeof(jxo_ray) * W);
  if (ambiguous) memset(ambiguous, 0, (size_t)H * W);

  /* one ray per column through the pixel centre: cx = 2 (col + 1/2) / W - 1 */
  for (int col = 0; col < W; ++col) {
    double cx = 2.0 * (col + 0.5) / W - 1.0;
    double rx = c - cx * T * s, ry = s + cx * T * c;
    jxo_ray* r = &col_rays[col];
    jxo_cast(cfg, e, e->x, e->y, rx, ry, bias, r);
    slice_rows(H, r->perp, r);
    r->corner = 0;
    if (want_flags) {
      jxo_ray bx, by;
      jxo_cast(cfg, e, e->x, e->y, rx, ry, +1, &bx);
      jxo_cast(cfg, e, e->x, e->y, rx, ry, -1, &by);
      if (bx.cell_x != by.cell_x || bx.cell_y != by.cell_y || bx.side != by.side) r->corner = 1;
      if (r->side >= 0) {
        /* hit point within JXO_EPS_CELL of a lattice point */
        double hx = e->x + r->perp * rx, hy = e->y + r->perp * ry;
        double along = r->side == 0 ? hy : hx;
        if (fabs(along - floor(along + 0.5)) < JXO_EPS_CELL) r->corner = 1;
      }
    }
  }

  /* walls, ceiling and floor; the wall colour is scaled by 3/4 on y faces
   * and, with distance shading (Sec. 2.1: shading from the distance), by
   * q / 256 with q = 64 + floor(192 min(h, H) / H): full colour for a slice
   * of the whole frame height or more, a quarter of it far away */
  for (int col = 0; col < W; ++col) {
    const jxo_ray* r = &col_rays[col];
    uint8_t wall[3];
    wall_rgb(r->side >= 0 ? cell_value(cfg, e, r->cell_x, r->cell_y) : 1, wall);
    if (r->side == 1)
      for (int k = 0; k < 3; ++k) wall[k] = (uint8_t)((wall[k] * 3) >> 2);
    if (cfg->shading) {
      int q = 64 + (192 * (r->h < H ? r->h : H)) / H;
      for (int k = 0; k < 3; ++k) wall[k] = (uint8_t)((wall[k] * q) >> 8);
    }
    for (int row = 0; row < H; ++row) {
      const uint8_t* rgb = row < r->top ? CEIL_RGB : (row < r->bot ? wall : FLOOR_RGB);
      uint8_t* px = frame + ((size_t)row * W + col) * 3;
      px[0] = rgb[0];
      px[1] = rgb[1];
      px[2] = rgb[2];
    }
    if (ambiguous) {
      if (r->corner && bias == 0) {
        for (int row = 0; row < H; ++row) ambiguous[row * W + col] = 1;
      } else if (r->h_ambiguous && cfg->shading) {
        /* a one-row change of h recolours the whole slice */
        for (int row = r->top - 1; row <= r->bot; ++row)
          if (row >= 0 && row < H) ambiguous[row * W + col] = 1;
      } else if (r->h_ambiguous) {
        int rows[4] = {r->top - 1, r->top, r->bot - 1, r->bot};
        for (int k = 0; k < 4; ++k)
          if (rows[k] >= 0 && rows[k] < H) ambiguous[rows[k] * W + col] = 1;
      }
    }
  }

  /* sprites: per pixel, the nearest covering sprite in front of the wall */
  int ns = e->n_sprites;
  sprite_screen sp[JXO_MAX_SPRITES];
  for (int j = 0; j < ns; ++j) sp[j] = project_sprite(cfg, e, j, c, s, T);
  for (int row = 0; row < H && ns > 0; ++row) {
    for (int col = 0; col < W; ++col) {
      double px = col + 0.5, py = row + 0.5;
      double zb = col_rays[col].perp;
      int best = -1;
      double best_ty = 0.0;
      int amb = 0;
      for (int j = 0; j < ns; ++j) {
        if (!sprite_visible(e, j)) continue;
        const sprite_screen* q = &sp[j];
        int near_clip = fabs(q->ty - 0.1) < JXO_EPS_REL;
        if (!q->ok && !near_clip) continue;
        double u = (px - q->x0) / q->w, v = (py - q->top) / q->hgt;
        int in_rect = u >= 0.0 && u < 1.0 && v >= 0.0 && v < 1.0;
        double mm = mask_margin(e->spr_type[j], u, v);
        int covers = q->ok && in_rect && mm > 0.0 && q->ty < zb;
        if (ambiguous) {
          double du = fmin(fabs(px - q->x0), fabs(px - (q->x0 + q->w)));
          double dv = fmin(fabs(py - q->top), fabs(py - (q->top + q->hgt)));
          int near_rect = px > q->x0 - JXO_EPS_PIX && px < q->x0 + q->w + JXO_EPS_PIX &&
                          py > q->top - JXO_EPS_PIX && py < q->top + q->hgt + JXO_EPS_PIX;
          if (near_rect) {
            double scale = fmin(0.5 * q->w, 0.5 * q->hgt);
            if (du < JXO_EPS_PIX || dv < JXO_EPS_PIX) amb = 1;
            if (fabs(mm) * scale < 2.0 * JXO_EPS_PIX) amb = 1;
            if (fabs(q->ty - zb) < JXO_EPS_REL * q->ty) amb = 1;
            if (near_clip) amb = 1;
            if (covers && best >= 0 && fabs(q->ty - best_ty) < JXO_EPS_REL * q->ty) amb = 1;
          }
        }
        if (covers && (best < 0 || q->ty < best_ty)) {
          best = j;
          best_ty = q->ty;
        }
      }
      if (best >= 0) {
        uint8_t rgb[3];
        sprite_rgb(e->spr_type[best], rgb);
        uint8_t* p = frame + ((size_t)row * W + col) * 3;
        p[0] = rgb[0];
        p[1] = rgb[1];
        p[2] = rgb[2];
      }
      if (ambiguous && amb) ambiguous[row * W + col] = 1;
    }
  }
  if (rays) memcpy(rays, col_rays, sizeof(jxo_ray) * W);
  free(col_rays);
  return 0;
}

int jxo_render(const jxo_config* cfg, const jxo_env* e, uint8_t* frame, jxo_ray* rays, uint8_t* ambiguous) {
  return render_impl(cfg, e, frame, rays, ambiguous, 0);
}

int jxo_render_biased(const jxo_config* cfg, const jxo_env* e, uint8_t* frame, jxo_ray* rays, uint8_t* ambiguous,
                      int32_t bias) {
  if (bias < -1 || bias > 1) return -1;
  return render_impl(cfg, e, frame, rays, ambiguous, bias);
}

/* ------------------------------------------------------------ batches ---- */
static int clamp_threads(int32_t nthreads) { return nthreads < 1 ? 1 : nthreads; }

int jxo_step_render_batch(const jxo_config* cfg, const int32_t* env_index, jxo_env* envs, int32_t n,
                          const uint8_t* actions, float* rewards, uint8_t* dones, int32_t* events,
                          uint8_t* frames, jxo_ray* rays, uint8_t* ambiguous, int32_t nthreads) {
  if (!config_ok(cfg)) return -1;
  size_t fb = (size_t)cfg->frame_h * cfg->frame_w;
  int err = 0;
#pragma omp parallel for num_threads(clamp_threads(nthreads)) schedule(dynamic, 4) reduction(| : err)
  for (int32_t i = 0; i < n; ++i) {
    double r;
    int32_t d, ev;
    err |= jxo_step(cfg, env_index[i], &envs[i], actions[i], &r, &d, &ev) != 0;
    if (rewards) rewards[i] = (float)r;
    if (dones) dones[i] = (uint8_t)d;
    if (events) events[i] = ev;
    if (frames || rays || ambiguous)
      err |= jxo_render(cfg, &envs[i], frames ? frames + fb * 3 * i : NULL,
                        rays ? rays + (size_t)cfg->frame_w * i : NULL,
                        ambiguous ? ambiguous + fb * i : NULL) != 0;
  }
  return err ? -1 : 0;
}

int jxo_render_batch_biased(const jxo_config* cfg, const jxo_env* envs, int32_t n, uint8_t* frames, jxo_ray* rays,
                            uint8_t* ambiguous, int32_t bias, int32_t nthreads) {
  if (!config_ok(cfg) || bias < -1 || bias > 1) return -1;
  size_t fb = (size_t)cfg->frame_h * cfg->frame_w;
  int err = 0;
#pragma omp parallel for num_threads(clamp_threads(nthreads)) schedule(dynamic, 4) reduction(| : err)
  for (int32_t i = 0; i < n; ++i)
    err |= render_impl(cfg, &envs[i], frames + fb * 3 * i, rays ? rays + (size_t)cfg->frame_w * i : NULL,
                       ambiguous ? ambiguous + fb * i : NULL, bias) != 0;
  return err ? -1 : 0;
}

int jxo_render_batch(const jxo_config* cfg, const jxo_env* envs, int32_t n, uint8_t* frames, jxo_ray* rays,
                     uint8_t* ambiguous, int32_t nthreads) {
  return jxo_render_batch_biased(cfg, envs, n, frames, rays, ambiguous, 0, nthreads);
}

/* jxo_step_biased over n environments with one bias choice for all (no frames). */
int jxo_step_batch_biased(const jxo_config* cfg, const int32_t* env_index, jxo_env* envs, int32_t n,
                          const uint8_t* actions, int32_t coll_x, int32_t coll_y, int32_t pick_x, int32_t pick_y,
                          float* rewards, uint8_t* dones, int32_t* events, int32_t nthreads) {
  if (!config_ok(cfg)) return -1;
  int err = 0;
#pragma omp parallel for num_threads(clamp_threads(nthreads)) schedule(dynamic, 4) reduction(| : err)
  for (int32_t i = 0; i < n; ++i) {
    double r;
    int32_t d, ev;
    err |= jxo_step_biased(cfg, env_index[i], &envs[i], actions[i], coll_x, coll_y, pick_x, pick_y, &r, &d, &ev) != 0;
    rewards[i] = (float)r;
    dones[i] = (uint8_t)d;
    events[i] = ev;
  }
  return err ? -1 : 0;
}

int jxo_generate_batch(const jxo_config* cfg, const int32_t* env_index, const uint32_t* episode, jxo_env* out,
                       int32_t n, int32_t nthreads) {
  if (!config_ok(cfg)) return -1;
  int err = 0;
#pragma omp parallel for num_threads(clamp_threads(nthreads)) schedule(dynamic, 4) reduction(| : err)
  for (int32_t i = 0; i < n; ++i) err |= jxo_generate(cfg, env_index[i], episode[i], &out[i]) != 0;
  return err ? -1 : 0;
}
