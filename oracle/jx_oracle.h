/*
 * jx_oracle.h — plain FP64 CPU oracle of the batched first-person environment
 * step + render (JAXenstein, arxiv 2605.19926).
 *
 * TEST INFRASTRUCTURE ONLY. This code is the slow, obviously-correct
 * statement of what the GPU path must compute. Only the test suite, the
 * smoke check and the benchmark's CPU-baseline / reference leg may load it.
 * It shares no source, header, table or constant generator with the CUDA
 * library; the two agree only through the definitions written here.
 *
 * Everything is double precision. Positions are absolute map coordinates
 * (cell (i, j) is the unit square [i, i+1) x [j, j+1); x = column to the
 * right, y = row downwards); the heading is measured from +x towards +y.
 *
 * Paper passages followed: ray casting with DDA over a tile map (Sec. 2.1),
 * wall slice from hit distance (Sec. 2, Sec. 2.1), fixed sprites (Fig. 1),
 * keys / locked doors / goal (Table 1 "key-door", Table 2), native
 * low-resolution frames (Sec. 3.1). Constants the paper does not fix
 * (movement, collision radius, field of view, rewards, horizon, colours,
 * generators) are parameters or the readings listed beside each function.
 */
#ifndef JX_ORACLE_H
#define JX_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define JXO_MAX_SIDE 128
#define JXO_MAX_SPRITES 16

/* Tasks */
#define JXO_TASK_ROOMS 0        /* border walls + random interior walls       */
#define JXO_TASK_MAZE_KEYDOOR 1 /* DFS maze, one key, one locked door, a goal */
#define JXO_TASK_MAZE_ROOMS 2   /* the key-door maze with 8 x 8 open rooms carved in and distractor sprites */
#define JXO_TASK_ASCII 3        /* a map given as ASCII text (Table 2 symbols) */

/* Map cell values */
#define JXO_FLOOR 0
/* cell values: 1..9 static walls (colour by value); locked doors 16 + c and
 * unlocked doors 20 + c for colour c = 0 red, 1 blue, 2 yellow */
#define JXO_LOCKED 16
#define JXO_UNLOCKED 20
#define JXO_DOOR JXO_LOCKED /* the red locked door of the generated key-door mazes */

/* sprite types; keys of colour c: red 1, blue 4, yellow 5 */
#define JXO_SPR_NONE 0
#define JXO_SPR_KEY 1
#define JXO_SPR_GOAL 2
#define JXO_SPR_DISTRACTOR 3
#define JXO_SPR_KEY_BLUE 4
#define JXO_SPR_KEY_YELLOW 5

/* actions */
#define JXO_NOOP 0
#define JXO_FWD 1
#define JXO_BACK 2
#define JXO_STRAFE_L 3
#define JXO_STRAFE_R 4
#define JXO_TURN_L 5
#define JXO_TURN_R 6

/* Random-draw purposes (one SplitMix64 stream per purpose) */
#define JXO_P_WALL 1
#define JXO_P_SPAWN 2
#define JXO_P_HEADING 3
#define JXO_P_DFS 4
#define JXO_P_KEY 5
#define JXO_P_NSPRITES 6
#define JXO_P_SPRITE_CELL 7
#define JXO_P_ROOM 8
#define JXO_P_GOAL 9

/* Tolerances the oracle uses to flag decisions that finite precision may flip. */
#define JXO_EPS_CELL 1e-5   /* cells: DDA ties, hit near a lattice point, collision boundaries */
#define JXO_EPS_PIX 1e-3    /* pixels: sprite silhouette edges */
#define JXO_EPS_REL 1e-5    /* relative: slice height rounding, depth comparisons */

/* step events bits */
#define JXO_EV_KEY 1
#define JXO_EV_GOAL 2
#define JXO_EV_NEAR_TIE 4

typedef struct {
  int32_t task;
  int32_t map_side;
  int32_t frame_h, frame_w;
  int32_t max_sprites;
  int32_t horizon;       /* episode length limit in steps; 0 = none */
  int32_t turns_per_rev; /* a turn action rotates by 2*pi / turns_per_rev */
  int32_t shading;       /* 1: wall colours also scaled by the slice height (distance shading) */
  double wall_prob;      /* interior wall probability (rooms task) */
  double fov_deg;        /* horizontal field of view */
  double move_step;      /* cells per move action */
  double radius;         /* half-size of the agent's collision box */
  double step_reward, key_reward, goal_reward;
  uint64_t seed;
  uint64_t ascii;        /* JXO_TASK_ASCII: address of the parsed jxo_ascii map */
} jxo_config;

typedef struct {
  double x, y;           /* absolute position */
  double theta0;         /* heading at episode start (radians) */
  int32_t turn;          /* heading = theta0 + turn * 2*pi/turns_per_rev */
  int32_t t;             /* steps taken in this episode */
  uint32_t episode;
  int32_t keys;          /* keys held: bit c for colour c (0 red, 1 blue, 2 yellow) */
  int32_t key_x, key_y, goal_x, goal_y, door_x, door_y; /* -1 when absent */
  int32_t n_sprites;
  int32_t pad0;
  double spr_x[JXO_MAX_SPRITES], spr_y[JXO_MAX_SPRITES];
  int32_t spr_type[JXO_MAX_SPRITES];
  uint8_t map[JXO_MAX_SIDE * JXO_MAX_SIDE]; /* row-major, map[y*S + x] */
} jxo_env;

typedef struct {
  int32_t cell_x, cell_y; /* first solid cell the ray enters */
  int32_t side;           /* 0: crossed an x boundary (vertical face), 1: a y boundary */
  int32_t h;              /* slice height in rows */
  int32_t top, bot;       /* clamped slice rows [top, bot) */
  int32_t corner;         /* 1: a finite-precision tie could change (cell, side) */
  int32_t h_ambiguous;    /* 1: H/perp + 1/2 lies within tolerance of an integer */
  double perp;            /* perpendicular (camera-plane) distance of the hit */
} jxo_ray;

/* n-th output (n >= 1) of SplitMix64 seeded with `seed`. */
uint64_t jxo_splitmix64(uint64_t seed, uint64_t n);
/* The draw `index` of stream (seed, env, episode, purpose). */
uint64_t jxo_draw(uint64_t seed, uint32_t env, uint32_t episode, uint32_t purpose, uint32_t index);

int jxo_sizeof_env(void);
int jxo_sizeof_config(void);
int jxo_sizeof_ray(void);

/* Build episode `episode` of environment `env_index`. Returns 0, or -1 on an invalid config. */
int jxo_generate(const jxo_config* cfg, int32_t env_index, uint32_t episode, jxo_env* out);

/* An ASCII map (Table 2) laid out in the top-left corner of an S x S grid of
 * walls: '#' wall 1; '1'..'9' wall of that colour; '.' and ' ' floor; 'S'
 * spawn candidate; 'G' goal candidate; 'r', 'b', 'y' red, blue, yellow keys;
 * '"', '\\' blue and yellow unlocked doors; 'R', 'B', 'Y' locked doors; any
 * other printable character a static wall of colour 1 + (code mod 9) (the
 * generated DMLab symbols). Candidates and keys in row-major order. */
typedef struct {
  int32_t side;
  int32_t n_spawn, n_goal, n_keys;
  uint8_t map[JXO_MAX_SIDE * JXO_MAX_SIDE];
  int32_t spawn[JXO_MAX_SIDE * JXO_MAX_SIDE];
  int32_t goal[JXO_MAX_SIDE * JXO_MAX_SIDE];
  int32_t key_cell[JXO_MAX_SPRITES];
  int32_t key_colour[JXO_MAX_SPRITES];
} jxo_ascii;

/* 0 on success; -1 when the text does not fit S x S, holds a control
 * character, or more than JXO_MAX_SPRITES keys. */
int jxo_parse_ascii(const char* text, int32_t side, jxo_ascii* out);
int jxo_sizeof_ascii(void);

/* Grayscale of n RGB pixels: the integer BT.601 luma (77 R + 150 G + 29 B + 128) >> 8. */
void jxo_gray(const uint8_t* rgb, int64_t n, uint8_t* out);

/* One environment step with auto-reset. Returns 0 or -1. */
int jxo_step(const jxo_config* cfg, int32_t env_index, jxo_env* e, int32_t action,
             double* reward, int32_t* done, int32_t* events);

/* DDA cast from (ox, oy) along (rx, ry). bias 0: exact decisions; +1 / -1: decisions
 * within JXO_EPS_CELL of a tie go to the x / y boundary. Fills cell, side, perp. */
int jxo_cast(const jxo_config* cfg, const jxo_env* e, double ox, double oy, double rx, double ry,
             int32_t bias, jxo_ray* out);

/* jxo_step with the decisions finite precision may flip taken a chosen way,
 * to enumerate the outcomes a near tie (JXO_EV_NEAR_TIE) admits. coll_x,
 * coll_y in {-1, 0, +1} for the x and y collision tests: 0 exact; +1 a test
 * within JXO_EPS_CELL of flipping lets the box move; -1 blocks it. pick_x,
 * pick_y in {-1, 0, +1}: key and goal events are evaluated at the position
 * moved by that many JXO_EPS_CELL. All zero is jxo_step. Returns 0 or -1. */
int jxo_step_biased(const jxo_config* cfg, int32_t env_index, jxo_env* e, int32_t action, int32_t coll_x,
                    int32_t coll_y, int32_t pick_x, int32_t pick_y, double* reward, int32_t* done,
                    int32_t* events);

/* Render one frame [H][W][3]. rays (W entries) and ambiguous ([H][W]) may be NULL. */
int jxo_render(const jxo_config* cfg, const jxo_env* e, uint8_t* frame, jxo_ray* rays,
               uint8_t* ambiguous);
/* jxo_render with every ray cast under `bias` (-1, 0, +1; see jxo_cast): the
 * frame of one tie decision for all corner rays. Corner columns are then not
 * flagged as wholly ambiguous (only their slice edges, as other columns). */
int jxo_render_biased(const jxo_config* cfg, const jxo_env* e, uint8_t* frame, jxo_ray* rays,
                      uint8_t* ambiguous, int32_t bias);

/* Batched helpers over n environments (OpenMP over environments when nthreads > 1).
 * frames / rays / ambiguous may be NULL. rewards are rounded to float32. */
int jxo_step_render_batch(const jxo_config* cfg, const int32_t* env_index, jxo_env* envs, int32_t n,
                          const uint8_t* actions, float* rewards, uint8_t* dones, int32_t* events,
                          uint8_t* frames, jxo_ray* rays, uint8_t* ambiguous, int32_t nthreads);
int jxo_render_batch(const jxo_config* cfg, const jxo_env* envs, int32_t n, uint8_t* frames,
                     jxo_ray* rays, uint8_t* ambiguous, int32_t nthreads);
int jxo_render_batch_biased(const jxo_config* cfg, const jxo_env* envs, int32_t n, uint8_t* frames,
                            jxo_ray* rays, uint8_t* ambiguous, int32_t bias, int32_t nthreads);
int jxo_step_batch_biased(const jxo_config* cfg, const int32_t* env_index, jxo_env* envs, int32_t n,
                          const uint8_t* actions, int32_t coll_x, int32_t coll_y, int32_t pick_x, int32_t pick_y,
                          float* rewards, uint8_t* dones, int32_t* events, int32_t nthreads);
int jxo_generate_batch(const jxo_config* cfg, const int32_t* env_index, const uint32_t* episode,
                       jxo_env* out, int32_t n, int32_t nthreads);

#ifdef __cplusplus
}
#endif
#endif
