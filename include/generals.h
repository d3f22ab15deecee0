/*
 * libgenerals: batched Generals.io environment step on GB300 (sm_103a).
 *
 * One call advances every game of an environment by one turn: action
 * validation and application, combat and capture, general capture with land
 * transfer, army growth, termination and reward, auto-reset through the
 * seeded map generator, then per-player fog-of-war observations, the public
 * scoreboard and the legal-action mask (paper, Section IV; fixed H x W x 9
 * action space of Section IV-G; reward of Section III).
 *
 * Conventions shared by every entry point
 *  - Return 0 on success or a negative GEN_ERR_* code; gen_last_error()
 *    gives a one-line reason.  Illegal or out-of-range actions are not
 *    errors: they act as a pass and are counted per game.
 *  - Device pointers ("d_") must be 16-byte aligned device memory of the
 *    sizes stated; host pointers ("h_") are ordinary (preferably pinned)
 *    host memory.  The library never frees caller memory.
 *  - "stream" is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream.  Calls are stream-ordered and do not synchronise the device,
 *    except where a call is documented as synchronous.
 *  - The environment owns the game state (device arenas) until
 *    gen_destroy().  An environment must not be used from two host threads
 *    at once.
 *
 * Layout (ragged batches allowed: each game g has its own H_g x W_g board,
 * N_g = H_g * W_g cells, P_g players):
 *  - Npad_g = N_g rounded up to a multiple of 16.
 *  - Per-player planes (obs_army int16, obs_owner int8, obs_terrain int8,
 *    obs_vis uint8, mask uint8) hold, for game g and player p, Npad_g cells
 *    in row-major order starting at plane_off[g] + p * Npad_g.  Cells
 *    N_g .. Npad_g-1 are padding and read 0 (army), -2 (owner), 4 (terrain),
 *    0 (vis, mask).  A uniform batch is the array [G][P][Npad].
 *  - Per-player slots (actions, reward, scoreboard) of game g are
 *    player_off[g] + p.  A uniform batch is [G][P].
 *  - Codes: terrain 0 plain, 1 mountain, 2 castle, 3 general; observed
 *    terrain 4 = fog, 5 = fogged mountain or castle; owner -1 neutral,
 *    0..P-1 player, -2 hidden.  Mask byte: bit d (0 up, 1 down, 2 left,
 *    3 right) = all-but-one move legal, bit 4+d = half move legal; pass is
 *    always legal and not in the mask.
 *  - Action of a player: flat index a = cell * 9 + k into the H x W x 9
 *    action space; k = 0 pass, 1..4 all-but-one up/down/left/right, 5..8
 *    half up/down/left/right.
 */
#ifndef GENERALS_H
#define GENERALS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GEN_OK 0
#define GEN_ERR_BAD_ARG (-1)
#define GEN_ERR_OOM (-2)
#define GEN_ERR_CUDA (-3)
#define GEN_ERR_TIMEOUT (-4)
#define GEN_ERR_STATE (-5)

#define GEN_MODE_1V1 0
#define GEN_MODE_2V2 1
#define GEN_MODE_FFA 2

#define GEN_MAX_PLAYERS 8
#define GEN_MAX_SIDE 64

typedef struct gen_env gen_env;

/* Generator and episode parameters (Section IV-A map generation). */
typedef struct gen_params {
    uint64_t seed;             /* map seed of the counter hash */
    uint64_t game_id_base;     /* global id of local game 0 (sharding) */
    uint32_t mountain_thresh;  /* P(mountain) = thresh / 2^32; 858993459 = 20% */
    int32_t n_cities;          /* >= 0: neutral castles per map; < 0: use city_per_mille */
    int32_t city_per_mille;    /* castles = floor(N * per_mille / 1000) when n_cities < 0 */
    int32_t city_army_min;     /* castle army, inclusive range (40..50 in the paper) */
    int32_t city_army_max;
    int32_t min_general_dist;  /* Manhattan spacing of generals; <= 0: floor((H+W)/3) */
    int32_t max_turns;         /* 0 = no truncation; else done code 2 at this turn */
    int32_t auto_reset;        /* 1: a finished game is regenerated inside gen_step */
    int32_t max_general_dist;  /* spawn-distance curriculum cap (0 = none), Section V */
    int32_t bfs_distance;      /* 1: general spacing in BFS steps around mountains ("17 steps") */
    int32_t castle_radius;     /* > 0: a neutral castle within this many steps of every general (6) */
} gen_params;

/* Device output buffers of one frame (sizes from gen_layout): the
 * observation planes, mask, reward, scoreboard and done flags of
 * Sections III, IV-B and IV-G.  Fields are caller-provided device pointers;
 * where a call says so, a NULL field (or a NULL gen_outputs) selects the
 * environment's own buffer of that output (gen_outputs_get). */
typedef struct gen_outputs {
    int16_t *obs_army;    /* [plane_cells] army if visible else 0 */
    int8_t *obs_owner;    /* [plane_cells] owner if visible else -2 */
    int8_t *obs_terrain;  /* [plane_cells] terrain if visible else 4 / 5 */
    uint8_t *obs_vis;     /* [plane_cells] 1 if visible */
    uint8_t *mask;        /* [plane_cells] legal-move bits */
    float *reward;        /* [player_slots] reward of this step */
    int32_t *scoreboard;  /* [player_slots][2] land, army (public) */
    uint8_t *done;        /* [n_games] 0 running, 1 terminal, 2 truncated */
} gen_outputs;

/* Sizes of an environment's per-game arrays (see "Layout" above). */
typedef struct gen_layout_info {
    int32_t n_games;
    int32_t player_slots;  /* sum of P_g */
    int64_t plane_cells;   /* sum of P_g * Npad_g: elements of each per-player plane */
    int64_t state_cells;   /* sum of Npad_g */
    int32_t max_players;
    int32_t max_cells;     /* max N_g */
} gen_layout_info;

/* Fill *p with the defaults of the Section IV-A generator: seed 1, 20%
 * mountains, 8 castles of 40..50, spacing floor((H+W)/3), no truncation,
 * auto-reset on. */
int gen_default_params(gen_params *p);

/* Create a uniform batch of `batch` games of H x W in `mode` (0 1v1, 1 2v2,
 * 2 FFA with 8 players) with default parameters and the given seed.  Runs
 * the generator for every game (epoch 0).  Synchronous. */
int gen_create(gen_env **out, int batch, int H, int W, int mode, uint64_t seed);

/* Create a ragged batch: per-game host arrays h_H, h_W, h_mode and
 * h_n_players (players for FFA; ignored for 1v1 / 2v2), each of `batch`
 * entries; 1 <= H, W <= 64, P <= N.  Synchronous. */
int gen_create_ex(gen_env **out, const gen_params *p, int batch, const int32_t *h_H, const int32_t *h_W,
                  const int32_t *h_mode, const int32_t *h_n_players);

/* Layout sizes and, when the arrays are non-NULL, the per-game host offsets
 * (h_plane_off[g], h_player_off[g], h_npad[g], each [n_games]).  Interface
 * addition: the paper's per-player H x W observations (Section IV-B) and
 * H x W x 9 actions (Section IV-G) flattened into ragged arrays. */
int gen_layout(const gen_env *env, gen_layout_info *info, int64_t *h_plane_off, int32_t *h_player_off,
               int32_t *h_npad);

/* Regenerate games (next epoch, new map, turn 0; the frame counter runs on)
 * and write their observations, masks and scoreboard into `out` (reward 0,
 * done 0).  d_game_ids: device int32 [n] of distinct local game ids (ids
 * outside [0, n_games) are skipped), or NULL for all games.  Section IV-A.
 * `out` or any of its fields may be NULL: those outputs go to the
 * environment's own buffers (see gen_outputs_get). */
int gen_reset(gen_env *env, const int32_t *d_game_ids, int n, const gen_outputs *out, void *stream);

/* Write the current observations, masks and scoreboard of every game into
 * `out` without advancing (reward 0, done 0): the fogged view of Section
 * IV-B and the legal moves of Section IV-D.  NULL `out` or fields: the
 * environment's own buffers, as for gen_reset. */
int gen_observe(gen_env *env, const gen_outputs *out, void *stream);

/* Advance every game by one turn.  d_actions: device int32 [player_slots].
 * Writes every field of `out`.  Section IV-B..IV-E.  `out` may be NULL, or
 * have NULL fields: those outputs go to the environment's own buffers (see
 * gen_outputs_get), valid until the next call that writes them. */
int gen_step(gen_env *env, const int32_t *d_actions, const gen_outputs *out, void *stream);

/* The environment's own one-frame output buffers (device pointers, every
 * field set), which gen_step / gen_step_policy / gen_reset / gen_observe
 * write in place of NULL output fields and gen_step_host stages through.
 * Interface addition (the paper's environment returns its observations,
 * Sections III and IV-B).  Allocated on first use, by this call or by the
 * first call given a NULL field -- a synchronous cudaMalloc, so make that
 * first call outside any stream capture; held until gen_destroy.  Their
 * contents are those of the last call that wrote into them.
 * GEN_ERR_OOM when the allocation fails. */
int gen_outputs_get(gen_env *env, gen_outputs *out);

/* Device bytes the environment holds now: state arenas, game tables, size
 * buckets, and its own output and staging buffers once allocated (feature
 * builders hold their own).  Interface addition, no counterpart in the
 * paper: memory accounting for admission budgets. */
int gen_device_bytes(const gen_env *env, size_t *bytes);

/* gen_step (NULL outputs as there), then the benchmark policy for the
 * next step computed from the new masks in the same launch: d_next_actions [player_slots] receives, per
 * player, a uniformly drawn legal (cell, direction) pair (row-major cells,
 * then up, down, left, right; pass when none) sent whole, or halved with
 * probability 0.2, keyed by (policy_seed, global game id, frame, player).
 * d_next_actions may equal d_actions. */
int gen_step_policy(gen_env *env, const int32_t *d_actions, const gen_outputs *out, uint64_t policy_seed,
                    int32_t *d_next_actions, void *stream);

/* Rollout forms of gen_rollout. */
#define GEN_ROLLOUT_RESIDENT 0 /* one launch; each game's state stays in shared memory for all K frames */
#define GEN_ROLLOUT_GRAPH 1    /* K step launches replayed from a captured CUDA graph */
#define GEN_ROLLOUT_LAUNCHES 2 /* K step launches issued one by one */
#define GEN_ROLLOUT_AUTO 3     /* the form gen_autotune picked for this environment (resident until tuned) */

/* K frames of every game, the benchmark policy choosing every action (see
 * gen_step_policy).  Every array of `out` holds K consecutive frames: frame
 * f of a per-player plane starts at f * plane_cells, of reward at
 * f * player_slots, of scoreboard at 2 * f * player_slots, of done at
 * f * n_games.  d_actions [player_slots]: in, the first frame's actions;
 * out, the actions for the frame after the rollout.  d_action_log
 * [K][player_slots] (may be NULL) receives the actions each frame consumed.
 * All forms give identical results.  GEN_ROLLOUT_GRAPH captures on first use
 * and replays while K, the seed and every buffer stay the same; its first
 * call must not happen inside another stream capture. */
int gen_rollout(gen_env *env, int K, uint64_t policy_seed, int32_t *d_actions, const gen_outputs *out,
                int32_t *d_action_log, int form, void *stream);

/* The benchmark policy alone (the uniform random legal policy of gen_step_policy,
 * over the Section IV-G action space), from the current state of every game. */
int gen_policy(gen_env *env, uint64_t policy_seed, int32_t *d_actions, void *stream);

/* gen_step with host buffers (Section IV-B..IV-E step; interface addition
 * for host-side actors): copies h_actions [player_slots] to the device,
 * steps, copies every non-NULL output of `h_out` back into host memory (same
 * sizes as the device outputs) and synchronises the stream.  When
 * h_next_actions is non-NULL the benchmark policy of gen_step_policy runs in
 * the same launch and its actions are copied back too.  Host buffers should
 * be pinned (page-locked) for the copies to overlap.  A batch of 8,192 games
 * or more launched as one size bucket runs as four chunks of games whose
 * outputs are copied out on an internal stream while the later chunks step;
 * the results are the same bytes as gen_step_policy's. */
int gen_step_host(gen_env *env, const int32_t *h_actions, const gen_outputs *h_out, uint64_t policy_seed,
                  int32_t *h_next_actions, void *stream);

/* gen_step_host for callers that cannot allocate device memory.  The paper
 * has no counterpart: this is an interface addition.  gen_step_host stages
 * the actions and one frame of outputs in device buffers it cudaMallocs on
 * its first call; some callers cannot allow that: an actor process whose
 * device memory is already handed to a fixed-size pool, or a real-time loop
 * that must not take cudaMalloc's implicit device synchronisation or risk an
 * out-of-memory failure mid-rollout.  This entry point allocates nothing: it
 * stages through a static device array of 32 MiB that every GPU loading the
 * library holds until the process exits, with the same arguments, results
 * and synchronisation as gen_step_host.
 *  - A batch whose staging (actions, five planes, reward, scoreboard, done,
 *    each rounded up to 256 bytes) exceeds 32 MiB is rejected with
 *    GEN_ERR_BAD_ARG; use gen_step_host for it.
 *  - The first call on a device looks up the array's device address (once
 *    per device, with that device current, and again after the device's
 *    context has been recreated, as by cudaDeviceReset); make that first
 *    call before any stream capture.
 *  - Every call, from any environment, shares the one array: calls whose
 *    device work overlaps (other threads, other streams) race and must be
 *    serialised by the caller.  Each call overwrites every staged byte it
 *    reads, so no state carries over between calls. */
int gen_step_host_static(gen_env *env, const int32_t *h_actions, const gen_outputs *h_out, uint64_t policy_seed,
                         int32_t *h_next_actions, void *stream);

/* Copy the whole game state of Section IV (armies, owners, cell types,
 * per-game counters) to host memory: h_army [state_cells] int16,
 * h_owner / h_terrain [state_cells] int8 (game g at its state offset,
 * sum of Npad of earlier games), h_scalars [n_games][8] uint32 = turn,
 * frame, epoch, alive bits, finished, invalid actions, saturations, error.
 * Synchronous on `stream`. */
int gen_read_state(gen_env *env, int16_t *h_army, int8_t *h_owner, int8_t *h_terrain, uint32_t *h_scalars,
                   void *stream);

/* Overwrite the whole game state from host memory (same layout as
 * gen_read_state; the error word is ignored).  Every cell and counter is
 * checked against the rules' ranges (Section IV: cell types 0..3, owners
 * -1..P-1, armies >= 0, padding cells empty, alive bits of the game's
 * players); GEN_ERR_BAD_ARG names the first offender.  Synchronous on
 * `stream`. */
int gen_write_state(gen_env *env, const int16_t *h_army, const int8_t *h_owner, const int8_t *h_terrain,
                    const uint32_t *h_scalars, void *stream);

/* Save everything that determines the environment's future frames into one
 * opaque, versioned host blob: every board (Section IV), the per-game
 * counters (turn, frame, epoch, alive players, finished, invalid actions,
 * saturations, error word) and the generator and episode parameters,
 * spawn range included (Sections IV-A and V).  Interface addition for
 * checkpoint and resume.  With h_buf NULL only *used is set (the size);
 * else h_buf must hold cap >= that many bytes, and *used receives the size
 * written.  Synchronous on `stream`.  Feature builders keep their own
 * memory, which the blob does not hold. */
int gen_save_state(gen_env *env, void *h_buf, size_t cap, size_t *used, void *stream);

/* Restore a blob written by gen_save_state into an environment of the same
 * games (same count, and per game the same H, W, mode and players), which
 * then continues frame for frame as the saved one would have: its
 * generator parameters, seed and spawn range are replaced by the saved
 * ones.  The blob is checked (magic, version, sizes, a checksum, every cell
 * and counter within the rules' ranges) before anything changes;
 * GEN_ERR_BAD_ARG says what failed.  Synchronous on `stream`. */
int gen_load_state(gen_env *env, const void *h_buf, size_t size, void *stream);

/* Change the spawn spacing of every later map of this environment (the
 * spawn-distance curriculum of Section V raises max_dist over training):
 * min_dist <= 0 keeps floor((H+W)/3), max_dist 0 removes the cap.  Takes
 * effect at the next reset or auto-reset; synchronous. */
int gen_set_spawn_range(gen_env *env, int min_dist, int max_dist);

/* Tuning call, no counterpart in the paper.  Launch shape of this
 * environment's step kernel: warps per CTA, one of 1,
 * 2, 4, 8 that fits the shared-memory limit (a warp runs one game, or two or
 * four, see gen_set_lane_groups; launches of fewer games than fill every SM
 * once take fewer warps per CTA).  Used by the autotuner; results do not
 * depend on it. */
int gen_set_launch(gen_env *env, int warps_per_cta);

/* Tuning call, no counterpart in the paper (Section IV-G runs every board
 * size in one environment; this picks how).  Times, on a scratch batch of
 * the environment's own shapes and parameters (its games do not advance;
 * the scratch is freed before returning), and keeps for this environment:
 *  - games per warp (gen_set_lane_groups: by batch size, one, or several);
 *  - for batches of several size buckets, the batch form (gen_set_batch_form);
 *  - the rollout form that GEN_ROLLOUT_AUTO runs (8-frame rollouts, per frame);
 *  - the sampler form (gen_set_sample_form, on zero logits);
 *  - each size bucket's games per CTA among 2, 4, 8 in the bucket form.
 * Results are cached for the process per batch signature (bucket classes
 * and counts, SM count).  `steps` timed calls per candidate; a
 * one-line-per-choice report goes to `report` when non-NULL.  Synchronous.
 * Buckets: games are grouped by padded cells (<= 256, 512, 768, 1024, 1536,
 * 2048, 3072, 4096) and players (<= 2, 4, 8); each bucket launches with its
 * own shared-memory size, largest first, on forked streams.  No choice
 * changes a result. */
int gen_autotune(gen_env *env, int steps, char *report, size_t report_cap);

/* Measurement call, no counterpart in the paper: the HBM roofline
 * denominator.  Measure copy bandwidth of this GPU with the library's own 128-bit copy
 * kernel over `bytes` (rounded down to 16 B), best of `reps`; returns GB/s
 * counting read + write bytes in *gbps.  Synchronous. */
int gen_copy_peak(size_t bytes, int reps, double *gbps);

/* ---- env server: continuous batching of many clients' steps ------------
 * The games of every client session stay on the device.  A scheduler
 * thread folds all step requests waiting at a given moment into one tick
 * (one work-list launch over all their games, every size class at once, with the
 * benchmark policy fused); up to two ticks are in flight, one behind the
 * other on the device, so requests that arrive while one runs start the
 * moment it ends.  Sessions are admitted while the device bytes they need fit the
 * budget; otherwise gen_server_open waits for others to close.  Each game is
 * keyed by the global game id its session was opened with, so its results
 * do not depend on the other sessions.  Section IV rules throughout.  The
 * server calls are interface additions with no counterpart in the paper
 * (its simulator steps one fixed batch inside the training loop, Section
 * IV-G); each gen_server_* declaration below belongs to this addition. */
typedef struct gen_server gen_server;

typedef struct gen_server_config {
    size_t budget_bytes;     /* device bytes sessions may hold (state; outputs too when on the device) */
    int64_t max_games;       /* game slots */
    int64_t max_cells;       /* board cells (padded to 16 per game) over all open sessions */
    int64_t max_plane_cells; /* per-player output cells over all open sessions */
    int32_t host_outputs;    /* 1: outputs in mapped pinned host memory (host clients); 0: device memory */
    uint64_t policy_seed;    /* benchmark policy seed of every session */
} gen_server_config;

typedef struct gen_server_stats {
    uint64_t requests, frames, ticks;
    uint64_t sessions_open, sessions_admitted, sessions_waited;
    double seconds;          /* since creation or the last reset */
    double frames_per_s;     /* games stepped per second */
    double lat_p50_ms, lat_p99_ms, lat_mean_ms; /* submit to result in the caller's buffers */
    double tick_games_mean;  /* games per tick */
    double bytes_in_use, budget;
    uint64_t sessions_waited_budget; /* admissions that waited while the byte budget was full */
    double peak_bytes_in_use;        /* most bytes sessions held at once in the window */
    double service_p50_ms, service_p99_ms; /* submit to result, as seen by the server */
    double offered_requests_per_s;   /* simulations: the clients' request rate (open loop: arrivals) */
    double tick_gpu_ms_mean;         /* device time of a tick, from its first copy to its last kernel */
    double tick_host_ms_mean;        /* scheduler time spent issuing a tick */
} gen_server_stats;

/* Allocates the arenas for the configured capacities (device memory, and
 * pinned host memory in host-output mode) and starts the scheduler thread. */
int gen_server_create(gen_server **out, const gen_params *p, const gen_server_config *cfg);

/* Admit a session of n games (per-game host arrays as gen_create_ex), keyed
 * by global ids game_id_base + i; waits up to wait_ms for room.  Generates
 * the games (epoch 0).  h_first_actions [the session's player slots] (may be
 * NULL) receives the policy's actions for the first step.  GEN_ERR_OOM when
 * there is no room in time. */
int gen_server_open(gen_server *sv, int n, const int32_t *h_H, const int32_t *h_W, const int32_t *h_mode,
                    const int32_t *h_n_players, uint64_t game_id_base, int wait_ms, int32_t *h_first_actions,
                    int32_t *session_out);

/* Sizes of a session's outputs (as gen_layout; offsets start at 0 within the
 * session) and, when dev_outputs is non-NULL, device pointers to them. */
int gen_server_session_layout(gen_server *sv, int session, gen_layout_info *info, gen_outputs *dev_outputs);

/* One step of every game of the session: h_actions [slots] in; blocks until
 * the tick that carried it completes, then copies the non-NULL fields of
 * h_out (host memory, session layout) and the policy's next actions.  One
 * step per session at a time. */
int gen_server_step(gen_server *sv, int session, const int32_t *h_actions, const gen_outputs *h_out,
                    int32_t *h_next_actions, double *latency_ms);

/* Release a session's games; waiting sessions may then be admitted. */
int gen_server_close(gen_server *sv, int session);

/* Counters, throughput and latency percentiles; reset = 1 starts a new window. */
int gen_server_stats_get(gen_server *sv, gen_server_stats *st, int reset);

/* Stop the scheduler and free everything. */
void gen_server_destroy(gen_server *sv);

/* Reason for the last server failure on this thread (never NULL). */
const char *gen_server_last_error(void);

typedef struct gen_sim_config {
    int32_t clients;            /* simulated actor clients (threads) */
    double mean_interarrival_ms;/* exponential think time before each step */
    int32_t min_games, max_games;/* games per session, uniform */
    int32_t min_side, max_side; /* board sides, uniform, H and W independent */
    double frac_1v1, frac_2v2;  /* mode mix; the rest is FFA with 8 players */
    int32_t min_steps, max_steps;/* steps before a client closes its session and opens another */
    double seconds;             /* measured window (after a short warm-up) */
    uint64_t seed, policy_seed;
    size_t budget_bytes;        /* admission budget */
    int32_t host_outputs;       /* see gen_server_config */
    int32_t copy_outputs;       /* clients copy every output into their own host buffers */
    int32_t open_loop;          /* 1: Poisson arrivals at mean_interarrival_ms, independent of completions;
                                   latencies run from each request's scheduled arrival */
    int32_t reserved;           /* 0 */
} gen_sim_config;

/* Run a server with simulated clients and report its stats.  Closed loop
 * (open_loop 0): each client thinks for an exponential time after its
 * previous result, then steps.  Open loop (open_loop 1): each client's
 * requests arrive as a Poisson process at the mean interval whatever the
 * server does; a request that arrives while the session's previous step is
 * still out waits for it, and lat_* count from the scheduled arrival
 * (queueing included), service_* from the submission.  Interface addition,
 * no counterpart in the paper. */
int gen_server_simulate(const gen_params *p, const gen_sim_config *cfg, gen_server_stats *st);

/* ---- policy sampling over the H x W x 9 action space (Sec. IV-G, App. C) --
 * Logits: player plane q = plane_off[g] + p * Npad_g holds 9 * Npad_g float32
 * at q * 9, entry c * 9 + k for cell c and k = 0 pass, 1..4 all-but-one up,
 * down, left, right, 5..8 half (the action encoding of gen_step); entries of
 * padding cells are ignored.  Logits must be finite.
 * Legal entries of player p: (c, 0) where p owns c; (c, 1 + d) and (c, 5 + d)
 * where the move is legal (the compact mask's bits d and 4 + d).  The action
 * is drawn from exp(logit) over the legal entries by an exact integer
 * inverse CDF (weights floor(E(l - max) * 2^24) with a bit-reproducible
 * single-precision exponential E), keyed by (seed, global game id, frame of
 * the step that will consume it, p); a player without a legal entry gets 0
 * (pass).  The same logits and seed give the same actions on every device.
 * d_actions: player_slots int32 (the layout gen_step reads).  d_mask9
 * (optional, 16-byte aligned): the expanded legal mask, 9 * Npad_g bytes per
 * player plane at q * 9, 1 = legal.  With d_logits and d_actions NULL only
 * the mask is written.  Asynchronous on `stream`; order it after the step
 * that produced the state.  GEN_ERR_BAD_ARG for NULL env, inconsistent
 * pointers or misaligned buffers. */
int gen_sample_actions(gen_env *env, const float *d_logits, uint64_t seed, int32_t *d_actions, uint8_t *d_mask9,
                       void *stream);

/* Tuning call, no counterpart in the paper.  Games per warp in the step
 * kernels (the results are the same): 1 = one
 * warp per game; 2 = two games per warp (four in multi-frame launches)
 * wherever the games allow it -- at most two players, boards of at most
 * 1,024 padded cells (576 for four), no spawn options; 0 (default) = as 2 for
 * launches of at least 12 x the SM count games (24 x in multi-frame
 * launches), else 1.  GEN_ERR_BAD_ARG for NULL env or a mode outside 0..2. */
int gen_set_lane_groups(gen_env *env, int mode);

/* Tuning call, no counterpart in the paper (Section IV-G runs every board
 * size and mode in one environment; this picks how a batch of several size
 * buckets is launched; the results are the same): 1 = one launch per size
 * bucket, buckets after the first on side streams; 2 = one persistent
 * work-list launch per frame (per rollout in the resident form): CTAs take
 * items -- up to a CTA's worth of one bucket's games, largest boards first --
 * from an atomic counter and carve their shared memory per item; 0 (default)
 * = 2 for batches of more than four buckets, else 1.  Batches with spawn
 * options always take form 1.  The work list's
 * counter belongs to the environment: order its calls on one stream.
 * GEN_ERR_BAD_ARG for NULL env or a form outside 0..2. */
int gen_set_batch_form(gen_env *env, int form);

/* Tuning call, no counterpart in the paper.  How gen_sample_actions
 * spreads a game over the GPU (the results are the same): 1 = one warp per
 * game, players in turn; 2 = one CTA per game with a warp per player (as
 * many as fit in shared memory beside the board); 3 = one CTA per player
 * with a thread per (own cell, entry) pair; 0 (default) = 3 while games x
 * the most players per game is at most 8 x the SM count, else 2.
 * GEN_ERR_BAD_ARG for NULL env or a form outside 0..3. */
int gen_set_sample_form(gen_env *env, int form);

/* ---- feature tensor (App. A, table of observation channels) -------------
 * Per player C = 24 + 2 * hist float32 planes of Npad_g cells each, in the
 * table's order: 0 armies, 1 own army, 2 enemy army, 3 neutral army,
 * 4 seen, 5 enemy seen, 6 generals, 7 castles, 8 mountains (persistent
 * memory), 9 neutral cells, 10 owned cells, 11 opponent cells, 12 fog,
 * 13 structures in fog, 14 turn, 15 (turn mod 50) / 50, 16 own land,
 * 17 own army, 18 opponents' land, 19 opponents' army (public scoreboard),
 * 20 last enemy army seen, 21 log(1 + turns since an enemy was last seen)
 * / 5, 22 column / (W-1), 23 row / (H-1), 24 .. 24+hist-1 own army deltas
 * (newest first), 24+hist .. 24+2hist-1 enemy army deltas.  "Opponent" is
 * a player of another team; enemy planes are the fogged view.
 * Layout: the player plane q = plane_off[g] + p * Npad_g (as for the
 * observation planes) holds channel ch of cell c at float index
 * q * C + ch * Npad_g + c; a uniform batch is [G][P][C][Npad].  Padding
 * cells N_g .. Npad_g-1 read 0 in every channel.
 * Memory: the builder keeps per player and cell the five persistent masks,
 * the last enemy army and turn, and hist + 1 frames of own / enemy army
 * planes (about 15 + 4 * (hist + 1) bytes per plane cell, allocated at
 * creation).  Each build folds the current frame into that memory once
 * (keyed by the game's frame counter; a second build in the same frame
 * changes nothing) and clears a game's memory when its epoch changes (a
 * new episode).  Call it after every step for the paper's definition of
 * the memory and delta rows.  The environment must outlive the builder. */
typedef struct gen_features gen_features;

/* hist in [1, 16] (the paper's default is 7: 38 channels).  Allocates the
 * memory on the environment's device; synchronous.  GEN_ERR_BAD_ARG for a
 * NULL env or hist out of range, GEN_ERR_CUDA when allocation fails. */
int gen_features_create(gen_features **out, gen_env *env, int hist);

/* As gen_features_create, with the temporal tokens of App. A: per player
 * the opponents' summed army and land (public scoreboard) of the last
 * `window` builder frames (the paper's window: 512), kept in a device ring
 * of window int32 pairs per player.  window in [0, 4096]; 0 = none. */
int gen_features_create_ex(gen_features **out, gen_env *env, int hist, int window);

/* Channels C (24 + 2 * hist, App. A) and the number of floats the output
 * buffer must hold. */
int gen_features_layout(const gen_features *f, int32_t *channels, int64_t *n_floats);

/* Window T (App. A temporal tokens) and the int32 count of the
 * temporal-token output: player_slots * T * 2. */
int gen_features_series_layout(const gen_features *f, int32_t *window, int64_t *n_ints);

/* Fold the current frame into the memory and write every player's features
 * to d_out (device, 16-byte aligned, n_floats floats).  Asynchronous on
 * `stream`; order it after the step that produced the frame. */
int gen_features_build(gen_features *f, float *d_out, void *stream);

/* As gen_features_build, also writing the temporal tokens to d_series
 * (device, 8-byte aligned, NULL: not written): player slot s holds T
 * (army, land) int32 pairs at s * T * 2, entry k = k frames back (newest
 * first), 0 before the episode.  GEN_ERR_BAD_ARG when d_series is given to a
 * builder created without a window. */
int gen_features_build_ex(gen_features *f, float *d_out, int32_t *d_series, void *stream);

/* Tuning call, no counterpart in the paper.  Times `steps` builds in each
 * form (gen_features_set_form 1 and 2) into d_out and keeps the faster;
 * *form_out (may be NULL) receives it.  The first build folds the current
 * frame; the timed ones repeat it (a repeated build in one frame changes
 * nothing), so d_out holds this frame's features afterwards.  Synchronous. */
int gen_features_autotune(gen_features *f, float *d_out, int steps, int *form_out);

/* Tuning call, no counterpart in the paper.  How the builder spreads a
 * game over the GPU (the bytes written are the same): 1 = one warp per
 * game, players in turn; 2 = one CTA per (game, player), its warps sharing
 * the player's 128-cell chunks, for batches too small to fill the GPU one
 * warp per game; 0 (default) = 2 while games x the most players per game is
 * at most 56 x the SM count, else 1.  GEN_ERR_BAD_ARG outside 0..2. */
int gen_features_set_form(gen_features *f, int form);

/* Free a builder's memory (App. A feature memory). */
void gen_features_destroy(gen_features *f);

/* Reason for the last failure on this thread (never NULL).  Interface
 * addition: error reporting of the C-ABI. */
const char *gen_last_error(void);

/* Free the environment's device state and buffers (interface addition). */
void gen_destroy(gen_env *env);

#ifdef __cplusplus
}
#endif
#endif /* GENERALS_H */
