/*
 * Generals.io rules oracle: a plain, slow, single-threaded CPU statement of
 * the batched environment step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file.  It shares no code,
 * header, table or helper with the CUDA library; the two sides are written
 * separately from the same rule text.
 *
 * Every function follows the game description of the paper (Section IV):
 *   Sec. IV-A  grid of plain / mountain / general / castle cells, 20%
 *              mountains, neutral castles holding 40-50 units, generals
 *              placed apart from each other;
 *   Sec. IV-B  ownership (neutral or one player) and fog of war: a player
 *              sees its own cells and their Moore (8-cell) neighbourhood,
 *              plus a public scoreboard of land and army per player;
 *   Sec. IV-C  generals and owned castles +1 every other turn, every
 *              owned plain cell +1 every 50 turns;
 *   Sec. IV-D  one move per player per turn: all-but-one or half of a cell's
 *              units to a 4-neighbour, or pass; combat by subtraction, ties
 *              keep the previous owner; capturing a general wins;
 *   Sec. IV-E  free-for-all capture hands the loser's land and half its army
 *              to the captor and turns the general into a castle; 2v2 moves
 *              onto an ally cell pool units and take the cell over; a team
 *              loses when both its generals are captured;
 *   Sec. IV-G  fixed H x W x 9 action space for every mode;
 *   Sec. III   sparse terminal zero-sum reward +1 / -1.
 * Where the paper is silent the readings used are written next to the code
 * that applies them (Q-numbers refer to the list of readings kept with the
 * design notes).  Nothing here is blocked, fused or reordered: one cell at a
 * time, in the order the rules are stated.
 *
 * Parity pins (tests/): SplitMix64 published output vectors, hand-worked
 * tiny boards (tests/golden/), the all-pass growth closed form, fog against
 * a library 3x3 binary dilation, the mask against the step's own validator
 * tried action by action, generator statistics and BFS connectivity, policy
 * uniformity, and invariants over exhaustive joint actions on 3x3 boards.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- cell and observation codes (Sec. IV-A, IV-B) ---------------------- */
#define T_PLAIN 0
#define T_MOUNTAIN 1
#define T_CASTLE 2
#define T_GENERAL 3
#define OBS_FOG 4
#define OBS_FOG_OBSTACLE 5
#define OBS_OWNER_HIDDEN (-2)
#define NEUTRAL (-1)

#define MODE_1V1 0
#define MODE_2V2 1
#define MODE_FFA 2

#define MAXP 8
#define ARMY_MAX 32767

/* ---- hash purposes ----------------------------------------------------- */
#define PURPOSE_MOUNTAIN 1
#define PURPOSE_GENERAL 2
#define PURPOSE_CITY_POS 3
#define PURPOSE_CITY_ARMY 4
#define PURPOSE_NEAR_CASTLE_POS 5
#define PURPOSE_NEAR_CASTLE_ARMY 6

#define GEN_ATTEMPTS 64 /* R: bounded rejection attempts per level */

typedef struct orc_params {
    uint64_t seed;           /* map seed */
    uint64_t game_id_base;   /* global id of local game 0 */
    uint32_t mountain_thresh;/* u32 threshold: P(mountain) = thresh / 2^32 */
    int32_t n_cities;        /* >= 0: fixed count; < 0: use city_per_mille */
    int32_t city_per_mille;  /* cities = floor(N * per_mille / 1000) */
    int32_t city_army_min;   /* inclusive */
    int32_t city_army_max;   /* inclusive */
    int32_t min_general_dist;/* >= 1: Manhattan D_min; <= 0: floor((H+W)/3) */
    int32_t max_turns;       /* 0 = no truncation */
    int32_t auto_reset;      /* 1 = regenerate finished games inside step */
    int32_t max_general_dist;/* spawn-distance curriculum cap (0 = none) */
    int32_t bfs_distance;    /* 1: spacing measured in BFS steps around mountains */
    int32_t castle_radius;   /* > 0: each general gets a neutral castle this many steps away */
} orc_params;

typedef struct orc_game {
    int32_t H, W, N, P, mode;
    int16_t *army;
    int8_t *owner;
    int8_t *terrain;
    int32_t turn;
    uint32_t frame;
    uint32_t epoch;
    uint32_t alive;      /* bit p set while player p still holds a general */
    uint32_t finished;   /* game over and not regenerated (auto_reset off) */
    int32_t gpos[MAXP];  /* general cell per player (as placed) */
    uint32_t invalid;    /* actions turned into pass */
    uint32_t saturated;  /* additions clipped at ARMY_MAX */
    float reward[MAXP];  /* of the last step */
    uint8_t done;        /* of the last step: 0, 1 terminal, 2 truncated */
} orc_game;

typedef struct orc_env {
    int32_t G;
    orc_params prm;
    orc_game *games;
} orc_env;

/* ======================================================================
 * Counter-based hash.  SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014): the generator adds the
 * golden-ratio increment to its state and returns the mix of the new state.
 * orc_sm(s, n) is the n-th output (n = 0, 1, ...) of SplitMix64 seeded with
 * s, computed directly from its definition by stepping the generator.
 * ====================================================================== */
static uint64_t orc_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t orc_sm(uint64_t seed, uint64_t n) {
    /* after n+1 steps the state is seed + (n+1) * increment (mod 2^64) */
    uint64_t state = seed + (n + 1) * 0x9E3779B97F4A7C15ULL;
    return orc_mix64(state);
}

/* key(seed, a, b, c): three nested SplitMix64 streams. */
uint64_t orc_key(uint64_t seed, uint64_t a, uint64_t b, uint64_t c) {
    return orc_sm(orc_sm(orc_sm(seed, a), b), c);
}

/* 32-bit draw i of a key: the high half of the i-th stream output. */
uint32_t orc_draw(uint64_t key, uint64_t i) { return (uint32_t)(orc_sm(key, i) >> 32); }

/* Uniform integer in [0, n): multiply-shift of a 32-bit draw. */
static int32_t orc_uniform(uint32_t u, uint32_t n) {
    return (int32_t)(((uint64_t)u * (uint64_t)n) >> 32);
}

/* ---- small helpers ------------------------------------------------------ */
static int orc_team(const orc_game *g, int p) {
    return g->mode == MODE_2V2 ? (p >> 1) : p; /* Q20: {0,1} vs {2,3} */
}
static int orc_abs(int x) { return x < 0 ? -x : x; }

static int orc_cities_for(const orc_params *prm, int N) {
    if (prm->n_cities >= 0) return prm->n_cities;
    return (int)(((int64_t)N * prm->city_per_mille) / 1000);
}
static int orc_dmin_for(const orc_params *prm, int H, int W) {
    if (prm->min_general_dist >= 1) return prm->min_general_dist;
    int d = (H + W) / 3;
    return d < 1 ? 1 : d;
}

/* destination of a move from cell c in direction d (0 up, 1 down, 2 left,
 * 3 right), or -1 when it leaves the board */
static int orc_neighbour(const struct orc_game *g, int c, int d);

/* BFS distance in steps from src through non-mountain cells (4-neighbours);
 * -1 where unreachable.  queue holds N ints. */
static void orc_bfs(const orc_game *g, int src, int *dist, int *queue) {
    for (int c = 0; c < g->N; ++c) dist[c] = -1;
    int head = 0, tail = 0;
    dist[src] = 0;
    queue[tail++] = src;
    while (head < tail) {
        int c = queue[head++];
        for (int d = 0; d < 4; ++d) {
            int n = orc_neighbour(g, c, d);
            if (n >= 0 && g->terrain[n] != T_MOUNTAIN && dist[n] < 0) {
                dist[n] = dist[c] + 1;
                queue[tail++] = n;
            }
        }
    }
}

/* ======================================================================
 * Map generator (Sec. IV-A; Q13, Q15).  Every draw is an integer from the
 * hash keyed by (seed, global game id, epoch, purpose).
 * ====================================================================== */
static void orc_generate(const orc_params *prm, orc_game *g, uint64_t game_id) {
    const int H = g->H, W = g->W, N = g->N, P = g->P;
    for (int c = 0; c < N; ++c) {
        g->army[c] = 0;
        g->owner[c] = NEUTRAL;
        g->terrain[c] = T_PLAIN;
    }
    /* 1. mountains: independent per-cell Bernoulli */
    uint64_t kmtn = orc_key(prm->seed, game_id, g->epoch, PURPOSE_MOUNTAIN);
    for (int c = 0; c < N; ++c)
        if (orc_draw(kmtn, (uint64_t)c) < prm->mountain_thresh) g->terrain[c] = T_MOUNTAIN;

    /* 2. generals: rejection sampling, R attempts per distance level; the
     *    level drops by one after R failures; below 1 the first cell in
     *    row-major order that holds no general is taken. */
    uint64_t kgen = orc_key(prm->seed, game_id, g->epoch, PURPOSE_GENERAL);
    uint64_t i = 0;
    int D = orc_dmin_for(prm, H, W);
    const int bfs = prm->bfs_distance != 0;
    const int Dmax = prm->max_general_dist;  /* curriculum cap (Sec. V spawn-distance curriculum) */
    int *dist = (int *)malloc(sizeof(int) * (size_t)N * (P + 1));  /* BFS from each placed general */
    int *queue = dist + (size_t)N * P;
    for (int p = 0; p < P; ++p) {
        int placed = -1;
        while (placed < 0) {
            if (D >= 1) {
                for (int t = 0; t < GEN_ATTEMPTS && placed < 0; ++t) {
                    int c = orc_uniform(orc_draw(kgen, i), (uint32_t)N);
                    i += 1;
                    if (g->terrain[c] == T_MOUNTAIN) continue;
                    int ok = 1;
                    for (int q = 0; q < p; ++q) {
                        int d = bfs ? dist[(size_t)q * N + c]
                                    : orc_abs(c / W - g->gpos[q] / W) + orc_abs(c % W - g->gpos[q] % W);
                        if (d < 0 || d < D) ok = 0;           /* unreachable or too close */
                        if (Dmax > 0 && d > Dmax) ok = 0;     /* beyond the curriculum cap */
                    }
                    if (ok) placed = c;
                }
                if (placed < 0) D -= 1;
            } else {
                /* first row-major cell holding no general; in BFS mode first
                 * try cells reachable from every earlier general within the
                 * cap, then cells reachable from general 0, then any cell */
                for (int pass = bfs ? 0 : 2; pass < 3 && placed < 0; ++pass)
                    for (int c = 0; c < N && placed < 0; ++c) {
                        int taken = 0;
                        for (int q = 0; q < p; ++q)
                            if (g->gpos[q] == c) taken = 1;
                        if (taken) continue;
                        if (pass < 2 && g->terrain[c] == T_MOUNTAIN) continue;
                        int fits = 1;
                        for (int q = 0; q < p; ++q) {
                            const int d = dist[(size_t)q * N + c];
                            if (pass == 0 && (d < 0 || (Dmax > 0 && d > Dmax))) fits = 0;
                            if (pass == 1 && q == 0 && d < 0) fits = 0;
                        }
                        if (fits) placed = c;
                    }
            }
        }
        g->gpos[p] = placed;
        if (bfs) orc_bfs(g, placed, dist + (size_t)p * N, queue);
    }
    for (int p = P; p < MAXP; ++p) g->gpos[p] = -1;
    for (int p = 0; p < P; ++p) {
        g->terrain[g->gpos[p]] = T_GENERAL;
        g->owner[g->gpos[p]] = (int8_t)p;
        g->army[g->gpos[p]] = 1; /* Q11 */
    }

    /* 3. connectivity (Q15): an L-shaped path from general p to general p+1,
     *    rows first, then columns; mountains on it become plain.  In BFS mode
     *    only when some general cannot reach general 0. */
    int carve = !bfs;
    for (int p = 1; p < P && bfs; ++p)
        if (dist[g->gpos[p]] < 0) carve = 1;
    for (int p = 0; carve && p + 1 < P; ++p) {
        int r = g->gpos[p] / W, c = g->gpos[p] % W;
        int r1 = g->gpos[p + 1] / W, c1 = g->gpos[p + 1] % W;
        while (r != r1) {
            r += (r1 > r) ? 1 : -1;
            if (g->terrain[r * W + c] == T_MOUNTAIN) g->terrain[r * W + c] = T_PLAIN;
        }
        while (c != c1) {
            c += (c1 > c) ? 1 : -1;
            if (g->terrain[r * W + c] == T_MOUNTAIN) g->terrain[r * W + c] = T_PLAIN;
        }
    }

    /* 4. neutral castles on plain cells, R attempts each (a failure skips
     *    that castle); army uniform in [min, max]. */
    uint64_t kpos = orc_key(prm->seed, game_id, g->epoch, PURPOSE_CITY_POS);
    uint64_t karm = orc_key(prm->seed, game_id, g->epoch, PURPOSE_CITY_ARMY);
    int ncity = orc_cities_for(prm, N);
    uint64_t j = 0;
    uint32_t span = (uint32_t)(prm->city_army_max - prm->city_army_min + 1);
    for (int k = 0; k < ncity; ++k) {
        for (int t = 0; t < GEN_ATTEMPTS; ++t) {
            int c = orc_uniform(orc_draw(kpos, j), (uint32_t)N);
            j += 1;
            if (g->terrain[c] == T_PLAIN && g->owner[c] == NEUTRAL) {
                g->terrain[c] = T_CASTLE;
                g->army[c] = (int16_t)(prm->city_army_min + orc_uniform(orc_draw(karm, (uint64_t)k), span));
                break;
            }
        }
    }

    /* 5. castle near every general (Sec. IV-A): when no neutral castle lies
     *    within castle_radius BFS steps, one is placed on the k-th free plain
     *    cell (row-major) of that ball, k uniform. */
    if (prm->castle_radius > 0) {
        uint64_t knp = orc_key(prm->seed, game_id, g->epoch, PURPOSE_NEAR_CASTLE_POS);
        uint64_t kna = orc_key(prm->seed, game_id, g->epoch, PURPOSE_NEAR_CASTLE_ARMY);
        for (int p = 0; p < P; ++p) {
            orc_bfs(g, g->gpos[p], dist, queue);
            int have = 0, count = 0;
            for (int c = 0; c < N; ++c) {
                if (dist[c] < 0 || dist[c] > prm->castle_radius) continue;
                if (g->terrain[c] == T_CASTLE && g->owner[c] == NEUTRAL) have = 1;
                if (g->terrain[c] == T_PLAIN && g->owner[c] == NEUTRAL) count += 1;
            }
            if (have || count == 0) continue;
            int k = orc_uniform(orc_draw(knp, (uint64_t)p), (uint32_t)count);
            for (int c = 0; c < N; ++c) {
                if (dist[c] < 0 || dist[c] > prm->castle_radius) continue;
                if (g->terrain[c] != T_PLAIN || g->owner[c] != NEUTRAL) continue;
                if (k-- == 0) {
                    g->terrain[c] = T_CASTLE;
                    g->army[c] = (int16_t)(prm->city_army_min + orc_uniform(orc_draw(kna, (uint64_t)p), span));
                    break;
                }
            }
        }
    }
    free(dist);

    g->turn = 0;
    g->alive = (P >= 32) ? 0xFFFFFFFFu : ((1u << P) - 1u);
    g->finished = 0;
}

/* ======================================================================
 * One move (Sec. IV-D, IV-E; Q1-Q3, Q7-Q10, Q19).
 * Returns 1 when the action was executed, 0 when it became a pass.
 * `eliminated` collects players whose general fell during this turn.
 * ====================================================================== */
static int16_t orc_sat_add(orc_game *g, int a, int b) {
    int s = a + b;
    if (s > ARMY_MAX) {
        g->saturated += 1;
        s = ARMY_MAX;
    }
    return (int16_t)s;
}

/* destination of a move from cell c in direction d (0 up, 1 down, 2 left,
 * 3 right), or -1 when it leaves the board */
static int orc_neighbour(const orc_game *g, int c, int d) {
    int r = c / g->W, col = c % g->W;
    if (d == 0) r -= 1;
    if (d == 1) r += 1;
    if (d == 2) col -= 1;
    if (d == 3) col += 1;
    if (r < 0 || r >= g->H || col < 0 || col >= g->W) return -1;
    return r * g->W + col;
}

/* legality of moving out of c towards d for player p at this instant */
static int orc_move_legal(const orc_game *g, int p, int c, int d) {
    if (!(g->alive & (1u << p))) return 0;
    if (g->owner[c] != p) return 0;
    if (g->army[c] < 2) return 0; /* Q3 */
    int dst = orc_neighbour(g, c, d);
    if (dst < 0) return 0;
    if (g->terrain[dst] == T_MOUNTAIN) return 0;
    return 1;
}

static void orc_capture_general(orc_game *g, int dst, int loser, int captor, uint32_t *eliminated) {
    g->terrain[dst] = T_CASTLE;
    for (int c = 0; c < g->N; ++c) {
        if (c == dst) continue;
        if (g->owner[c] == loser) {
            g->owner[c] = (int8_t)captor;
            g->army[c] = (int16_t)(g->army[c] - (g->army[c] >> 1)); /* Q7 */
        }
    }
    g->alive &= ~(1u << loser);
    *eliminated |= (1u << loser);
}

static int orc_apply_move(orc_game *g, int p, int32_t action, uint32_t *eliminated) {
    const int N = g->N;
    if (action < 0 || (int64_t)action >= 9LL * N) return 0;
    int c = action / 9, k = action % 9;
    if (k == 0) return 1; /* pass */
    int d = (k - 1) % 4;
    int half = (k >= 5);
    if (!orc_move_legal(g, p, c, d)) return 0;
    int dst = orc_neighbour(g, c, d);
    int army = g->army[c];
    int moved = half ? (army >> 1) : (army - 1); /* Q2 */
    g->army[c] = (int16_t)(army - moved);

    int o = g->owner[dst];
    int def = g->army[dst];
    if (o == p) {
        g->army[dst] = orc_sat_add(g, def, moved);
    } else if (o >= 0 && g->mode == MODE_2V2 && orc_team(g, o) == orc_team(g, p)) {
        /* ally: pool the units; the mover takes the cell unless it is the
         * ally's general (Q9) */
        g->army[dst] = orc_sat_add(g, def, moved);
        if (g->terrain[dst] != T_GENERAL) g->owner[dst] = (int8_t)p;
    } else {
        if (moved > def) {
            g->owner[dst] = (int8_t)p;
            g->army[dst] = (int16_t)(moved - def);
            if (g->terrain[dst] == T_GENERAL && o >= 0) orc_capture_general(g, dst, o, p, eliminated);
        } else if (moved == def) {
            g->army[dst] = 0; /* Q10: tie keeps the previous owner */
        } else {
            g->army[dst] = (int16_t)(def - moved);
        }
    }
    return 1;
}

/* ======================================================================
 * Whole step of one game: moves, growth, termination, reward, reset.
 * ====================================================================== */
static void orc_step_game(const orc_params *prm, orc_game *g, uint64_t game_id, const int32_t *actions) {
    const int P = g->P;
    for (int p = 0; p < MAXP; ++p) g->reward[p] = 0.0f;
    g->done = 0;
    if (g->finished) {
        g->frame += 1;
        return;
    }

    /* moves in rotating priority (Q1), each checked when it executes */
    uint32_t eliminated = 0;
    for (int k = 0; k < P; ++k) {
        int p = (g->turn + k) % P;
        if (!(g->alive & (1u << p))) continue; /* Q18 */
        if (!orc_apply_move(g, p, actions[p], &eliminated)) g->invalid += 1;
    }

    /* growth (Sec. IV-C; Q4-Q6) */
    g->turn += 1;
    if (g->turn % 2 == 0)
        for (int c = 0; c < g->N; ++c)
            if (g->owner[c] >= 0 && (g->terrain[c] == T_GENERAL || g->terrain[c] == T_CASTLE))
                g->army[c] = orc_sat_add(g, g->army[c], 1);
    if (g->turn % 50 == 0)
        for (int c = 0; c < g->N; ++c)
            if (g->owner[c] >= 0 && g->terrain[c] == T_PLAIN) g->army[c] = orc_sat_add(g, g->army[c], 1);

    /* termination and reward (Sec. III, IV-D, IV-E; Q17) */
    if (g->mode == MODE_2V2) {
        int team_dead[2];
        for (int t = 0; t < 2; ++t)
            team_dead[t] = !(g->alive & (1u << (2 * t))) && !(g->alive & (1u << (2 * t + 1)));
        if (team_dead[0] || team_dead[1]) {
            g->done = 1;
            for (int p = 0; p < P; ++p) g->reward[p] = team_dead[orc_team(g, p)] ? -1.0f : 1.0f;
        }
    } else {
        int n_alive = 0;
        for (int p = 0; p < P; ++p)
            if (g->alive & (1u << p)) n_alive += 1;
        for (int p = 0; p < P; ++p)
            if (eliminated & (1u << p)) g->reward[p] = -1.0f;
        if (n_alive <= 1) {
            g->done = 1;
            for (int p = 0; p < P; ++p)
                if (g->alive & (1u << p)) g->reward[p] = 1.0f;
        }
    }
    if (!g->done && prm->max_turns > 0 && g->turn >= prm->max_turns) g->done = 2; /* Q21 */

    /* reset (Q16): the frame's observation is of the new game */
    if (g->done) {
        if (prm->auto_reset) {
            g->epoch += 1;
            orc_generate(prm, g, game_id);
        } else {
            g->finished = 1;
        }
    }
    g->frame += 1;
}

/* ======================================================================
 * Observation of player p (Sec. IV-B, App. A rows 0-3 and 9-13; Q12, Q18).
 * Each output is a plane of N cells in row-major order.
 * ====================================================================== */
static int orc_sees(const orc_game *g, int p, int c) {
    if (!(g->alive & (1u << p))) return 0; /* Q18 */
    int r = c / g->W, col = c % g->W;
    for (int dr = -1; dr <= 1; ++dr)
        for (int dc = -1; dc <= 1; ++dc) {
            int rr = r + dr, cc = col + dc;
            if (rr < 0 || rr >= g->H || cc < 0 || cc >= g->W) continue;
            int o = g->owner[rr * g->W + cc];
            if (o >= 0 && orc_team(g, o) == orc_team(g, p)) return 1;
        }
    return 0;
}

static void orc_observe(const orc_game *g, int p, int16_t *army, int8_t *owner, int8_t *terrain,
                        uint8_t *vis, uint8_t *mask) {
    for (int c = 0; c < g->N; ++c) {
        int v = orc_sees(g, p, c);
        int t = g->terrain[c];
        vis[c] = (uint8_t)v;
        army[c] = v ? g->army[c] : 0;
        owner[c] = v ? g->owner[c] : (int8_t)OBS_OWNER_HIDDEN;
        if (v)
            terrain[c] = (int8_t)t;
        else
            terrain[c] = (t == T_MOUNTAIN || t == T_CASTLE) ? OBS_FOG_OBSTACLE : OBS_FOG;
        /* legal-action mask: bit d = all-but-one towards d, bit 4+d = half;
         * both need the same conditions (Q3).  Pass is always legal. */
        uint8_t m = 0;
        if (!g->finished)
            for (int d = 0; d < 4; ++d)
                if (orc_move_legal(g, p, c, d)) m |= (uint8_t)((1u << d) | (1u << (4 + d)));
        mask[c] = m;
    }
}

/* public scoreboard (Sec. IV-B): land and army per player */
static void orc_scoreboard(const orc_game *g, int32_t *land, int32_t *army) {
    for (int p = 0; p < MAXP; ++p) {
        land[p] = 0;
        army[p] = 0;
    }
    for (int c = 0; c < g->N; ++c)
        if (g->owner[c] >= 0) {
            land[(int)g->owner[c]] += 1;
            army[(int)g->owner[c]] += g->army[c];
        }
}

/* ======================================================================
 * Benchmark policy (Q23): uniform over legal (cell, direction) pairs in
 * row-major cell order then up, down, left, right; pass when none; the
 * half-split is taken with probability 0.2 (threshold floor(0.2 * 2^32)).
 * The draws are keyed by the frame index of the step that consumes them.
 * ====================================================================== */
#define SPLIT_THRESH 858993459u

static int32_t orc_policy_action(const orc_game *g, int p, uint64_t policy_seed, uint64_t game_id) {
    int n = 0;
    if (!g->finished)
        for (int c = 0; c < g->N; ++c)
            for (int d = 0; d < 4; ++d) n += orc_move_legal(g, p, c, d);
    if (n == 0) return 0;
    uint64_t key = orc_key(policy_seed, game_id, g->frame, (uint64_t)p);
    int j = orc_uniform(orc_draw(key, 0), (uint32_t)n);
    int split = orc_draw(key, 1) < SPLIT_THRESH;
    for (int c = 0; c < g->N; ++c)
        for (int d = 0; d < 4; ++d)
            if (orc_move_legal(g, p, c, d)) {
                if (j == 0) return c * 9 + (split ? 5 + d : 1 + d);
                j -= 1;
            }
    return 0; /* unreachable */
}

/* ======================================================================
 * C-ABI used by the Python test harness (ctypes).
 * ====================================================================== */
static int orc_players_for(int mode, int n_players) {
    if (mode == MODE_1V1) return 2;
    if (mode == MODE_2V2) return 4;
    return n_players;
}

int orc_env_new(orc_env **out, int32_t G, const int32_t *H, const int32_t *W, const int32_t *mode,
                const int32_t *n_players, const orc_params *prm) {
    *out = NULL;
    if (G < 0) return -1;
    orc_env *e = (orc_env *)calloc(1, sizeof(orc_env));
    if (!e) return -2;
    e->G = G;
    e->prm = *prm;
    e->games = (orc_game *)calloc((size_t)(G > 0 ? G : 1), sizeof(orc_game));
    for (int g = 0; g < G; ++g) {
        orc_game *gm = &e->games[g];
        int P = orc_players_for(mode[g], n_players ? n_players[g] : 2);
        if (H[g] < 1 || W[g] < 1 || P < 2 || P > MAXP || H[g] * W[g] < P || mode[g] < 0 || mode[g] > 2) {
            for (int k = 0; k < g; ++k) {
                free(e->games[k].army);
                free(e->games[k].owner);
                free(e->games[k].terrain);
            }
            free(e->games);
            free(e);
            return -1;
        }
        gm->H = H[g];
        gm->W = W[g];
        gm->N = H[g] * W[g];
        gm->P = P;
        gm->mode = mode[g];
        gm->army = (int16_t *)calloc((size_t)gm->N, sizeof(int16_t));
        gm->owner = (int8_t *)calloc((size_t)gm->N, 1);
        gm->terrain = (int8_t *)calloc((size_t)gm->N, 1);
        gm->epoch = 0;
        gm->frame = 0;
        orc_generate(&e->prm, gm, prm->game_id_base + (uint64_t)g);
    }
    *out = e;
    return 0;
}

void orc_env_free(orc_env *e) {
    if (!e) return;
    for (int g = 0; g < e->G; ++g) {
        free(e->games[g].army);
        free(e->games[g].owner);
        free(e->games[g].terrain);
    }
    free(e->games);
    free(e);
}

/* manual reset: next epoch, new map, turn 0; the frame counter runs on */
int orc_reset(orc_env *e, const int32_t *game_ids, int32_t n) {
    int count = game_ids ? n : e->G;
    for (int k = 0; k < count; ++k) {
        int g = game_ids ? game_ids[k] : k;
        if (g < 0 || g >= e->G) return -1;
        e->games[g].epoch += 1;
        orc_generate(&e->prm, &e->games[g], e->prm.game_id_base + (uint64_t)g);
        for (int p = 0; p < MAXP; ++p) e->games[g].reward[p] = 0.0f;
        e->games[g].done = 0;
    }
    return 0;
}

/* actions: [G][8] int32, one per player slot (slots >= P ignored) */
void orc_step(orc_env *e, const int32_t *actions) {
    for (int g = 0; g < e->G; ++g)
        orc_step_game(&e->prm, &e->games[g], e->prm.game_id_base + (uint64_t)g, actions + 8 * g);
}

/* one game's observation of player p, planes of N cells each */
void orc_observe_player(const orc_env *e, int32_t g, int32_t p, int16_t *army, int8_t *owner, int8_t *terrain,
                        uint8_t *vis, uint8_t *mask) {
    orc_observe(&e->games[g], p, army, owner, terrain, vis, mask);
}

/* scoreboard of game g: land[8], army[8] */
void orc_get_scoreboard(const orc_env *e, int32_t g, int32_t *land, int32_t *army) {
    orc_scoreboard(&e->games[g], land, army);
}

/* actions for the next step of every game: [G][8] int32 (slots >= P = 0) */
void orc_policy(const orc_env *e, uint64_t policy_seed, int32_t *actions) {
    for (int g = 0; g < e->G; ++g) {
        const orc_game *gm = &e->games[g];
        for (int p = 0; p < 8; ++p)
            actions[8 * g + p] = (p < gm->P) ? orc_policy_action(gm, p, policy_seed, e->prm.game_id_base + (uint64_t)g) : 0;
    }
}

/* scalar state of game g: turn, frame, epoch, alive, finished, invalid,
 * saturated, done, then gpos[8]; reward[8] separately */
void orc_get_scalars(const orc_env *e, int32_t g, int64_t *s, float *reward) {
    const orc_game *gm = &e->games[g];
    s[0] = gm->turn;
    s[1] = gm->frame;
    s[2] = gm->epoch;
    s[3] = gm->alive;
    s[4] = gm->finished;
    s[5] = gm->invalid;
    s[6] = gm->saturated;
    s[7] = gm->done;
    for (int p = 0; p < 8; ++p) s[8 + p] = gm->gpos[p];
    for (int p = 0; p < 8; ++p) reward[p] = gm->reward[p];
}

void orc_get_board(const orc_env *e, int32_t g, int16_t *army, int8_t *owner, int8_t *terrain) {
    const orc_game *gm = &e->games[g];
    memcpy(army, gm->army, sizeof(int16_t) * (size_t)gm->N);
    memcpy(owner, gm->owner, (size_t)gm->N);
    memcpy(terrain, gm->terrain, (size_t)gm->N);
}

/* overwrite one game's board and scalars (hand-built test positions) */
void orc_set_game(orc_env *e, int32_t g, const int16_t *army, const int8_t *owner, const int8_t *terrain,
                  int32_t turn, uint32_t alive, uint32_t frame, uint32_t epoch) {
    orc_game *gm = &e->games[g];
    memcpy(gm->army, army, sizeof(int16_t) * (size_t)gm->N);
    memcpy(gm->owner, owner, (size_t)gm->N);
    memcpy(gm->terrain, terrain, (size_t)gm->N);
    gm->turn = turn;
    gm->alive = alive;
    gm->frame = frame;
    gm->epoch = epoch;
    gm->finished = 0;
    for (int p = 0; p < MAXP; ++p) gm->gpos[p] = -1;
    for (int c = 0; c < gm->N; ++c)
        if (terrain[c] == T_GENERAL && owner[c] >= 0) gm->gpos[(int)owner[c]] = c;
}

/* ======================================================================
 * Feature tensor (Appendix A, Table "Observation channels"): per player
 * C = 24 + 2 * hist float channels over the game's own H x W cells, in the
 * table's order.  Persistent memory (rows 4-8, 20-21) and the army-delta
 * history (rows 24 on) accumulate over the frames the builder is run on and
 * are cleared when the game's epoch changes (a new episode).  Readings
 * (Q26-Q33 in the design notes):
 *   Q26 "opponent" = a player of another team (1v1 and FFA: any other
 *       player; 2v2: the other team); an ally's cells appear only in
 *       row 0 (armies) of the instantaneous rows;
 *   Q27 enemy_army (row 2) and the enemy deltas use the fogged view: army
 *       on VISIBLE opponent cells, 0 elsewhere; own_army is the agent's
 *       own cells (always visible to a living agent);
 *   Q28 neutral_cells (row 9) = visible, unowned and not a mountain;
 *   Q29 structures_in_fog (row 13) = fogged and either shown as an
 *       obstacle by the fogged observation (mountain or castle) or a
 *       remembered general;
 *   Q30 rows 16-19 come from the public scoreboard (Sec. IV-B): own land
 *       and army, summed land and army of the opponents;
 *   Q31 last_enemy_army_seen (row 20) takes the enemy army of a cell each
 *       frame the cell is visible (0 when visible without an enemy) and
 *       keeps it while fogged; last_enemy_army_age (row 21) is
 *       log(1 + dt) / 5 with dt = turns since an enemy was last seen on
 *       the cell, 0 when the cell is visible or no enemy was ever seen
 *       there in this episode;
 *   Q32 coords: column / (W - 1) and row / (H - 1), 0 when the side is 1;
 *       each game uses its own H x W, so no padded border exists;
 *   Q33 deltas: row 24 + k = own(t - k) - own(t - k - 1) for k = 0 ..
 *       hist - 1 over consecutive builder frames; frames before the
 *       episode count as all-zero planes.  Row 14 is the turn counter.
 *   Q34 temporal tokens (App. A, the two non-spatial tokens): per player
 *       the opponents' summed army and land (rows 19 and 18) of the last
 *       `window` builder frames, entry k = k frames back (newest first),
 *       as (army, land) int32 pairs; frames before the episode are 0.
 * Float rows are evaluated in double and rounded to float once.
 * ====================================================================== */

typedef struct orc_pmem {
    int64_t epoch;          /* epoch folded in last; -1: none yet */
    int64_t frame;          /* frame folded in last */
    uint8_t *seen, *enemy_seen, *generals, *castles, *mountains; /* [N] */
    int32_t *last_enemy_army; /* [N] */
    int32_t *last_enemy_turn; /* [N], meaningful where enemy_seen */
    int32_t *own_hist;      /* [hist + 1][N]: [k] = own army plane of the k-th latest folded frame */
    int32_t *enemy_hist;    /* [hist + 1][N] */
    int32_t *series;        /* [window][2]: [k] = (opponents' army, land) k frames back */
} orc_pmem;

typedef struct orc_feat {
    const orc_env *e;       /* read by orc_feat_build only */
    int32_t G, hist, window;
    int32_t *P;             /* [G] players per game, kept for orc_feat_free */
    orc_pmem *mem;          /* [G][MAXP] */
} orc_feat;

static int orc_is_opponent(const orc_game *g, int p, int o) {
    return o >= 0 && orc_team(g, o) != orc_team(g, p);
}

int orc_feat_new(orc_feat **out, const orc_env *e, int32_t hist, int32_t window) {
    *out = NULL;
    if (hist < 1 || hist > 16 || window < 0 || window > 4096) return -1;
    orc_feat *f = (orc_feat *)calloc(1, sizeof(orc_feat));
    f->e = e;
    f->G = e->G;
    f->hist = hist;
    f->window = window;
    f->P = (int32_t *)calloc((size_t)(e->G > 0 ? e->G : 1), sizeof(int32_t));
    for (int g = 0; g < e->G; ++g) f->P[g] = e->games[g].P;
    f->mem = (orc_pmem *)calloc((size_t)(e->G > 0 ? e->G : 1) * MAXP, sizeof(orc_pmem));
    for (int g = 0; g < e->G; ++g)
        for (int p = 0; p < e->games[g].P; ++p) {
            orc_pmem *m = &f->mem[g * MAXP + p];
            size_t n = (size_t)e->games[g].N;
            m->epoch = -1;
            m->frame = -1;
            m->seen = (uint8_t *)calloc(n, 1);
            m->enemy_seen = (uint8_t *)calloc(n, 1);
            m->generals = (uint8_t *)calloc(n, 1);
            m->castles = (uint8_t *)calloc(n, 1);
            m->mountains = (uint8_t *)calloc(n, 1);
            m->last_enemy_army = (int32_t *)calloc(n, sizeof(int32_t));
            m->last_enemy_turn = (int32_t *)calloc(n, sizeof(int32_t));
            m->own_hist = (int32_t *)calloc(n * (size_t)(hist + 1), sizeof(int32_t));
            m->enemy_hist = (int32_t *)calloc(n * (size_t)(hist + 1), sizeof(int32_t));
            m->series = (int32_t *)calloc((size_t)(window > 0 ? window : 1) * 2, sizeof(int32_t));
        }
    *out = f;
    return 0;
}

void orc_feat_free(orc_feat *f) {
    if (!f) return;
    for (int g = 0; g < f->G; ++g)
        for (int p = 0; p < f->P[g]; ++p) {
            orc_pmem *m = &f->mem[g * MAXP + p];
            free(m->seen);
            free(m->enemy_seen);
            free(m->generals);
            free(m->castles);
            free(m->mountains);
            free(m->last_enemy_army);
            free(m->last_enemy_turn);
            free(m->own_hist);
            free(m->enemy_hist);
            free(m->series);
        }
    free(f->mem);
    free(f->P);
    free(f);
}

/* features of player p of game g into out[C][N]; folds the current frame
 * into the player's memory first (once per frame) */
static void orc_feat_player(orc_feat *f, int gi, int p, float *out, int32_t *series_out) {
    const orc_game *g = &f->e->games[gi];
    orc_pmem *m = &f->mem[gi * MAXP + p];
    const int N = g->N, W = g->W, H = g->H, hist = f->hist;
    float *ch[64];
    for (int k = 0; k < 24 + 2 * hist; ++k) ch[k] = out + (size_t)k * N;

    /* current frame, fogged as the observation shows it */
    int32_t *own = (int32_t *)calloc((size_t)N, sizeof(int32_t));
    int32_t *enemy = (int32_t *)calloc((size_t)N, sizeof(int32_t));
    uint8_t *vis = (uint8_t *)calloc((size_t)N, 1);
    for (int c = 0; c < N; ++c) {
        vis[c] = (uint8_t)orc_sees(g, p, c);
        own[c] = g->owner[c] == p ? g->army[c] : 0;
        enemy[c] = (vis[c] && orc_is_opponent(g, p, g->owner[c])) ? g->army[c] : 0;
    }

    /* a new episode clears the memory (Q33: the past counts as zero) */
    if (m->epoch != (int64_t)g->epoch) {
        memset(m->seen, 0, (size_t)N);
        memset(m->enemy_seen, 0, (size_t)N);
        memset(m->generals, 0, (size_t)N);
        memset(m->castles, 0, (size_t)N);
        memset(m->mountains, 0, (size_t)N);
        memset(m->last_enemy_army, 0, sizeof(int32_t) * (size_t)N);
        memset(m->last_enemy_turn, 0, sizeof(int32_t) * (size_t)N);
        memset(m->own_hist, 0, sizeof(int32_t) * (size_t)N * (size_t)(hist + 1));
        memset(m->enemy_hist, 0, sizeof(int32_t) * (size_t)N * (size_t)(hist + 1));
        if (f->window > 0) memset(m->series, 0, sizeof(int32_t) * 2 * (size_t)f->window);
        m->epoch = (int64_t)g->epoch;
        m->frame = -1;
    }
    const int fold = m->frame != (int64_t)g->frame;

    /* rows 4-8, 20: what this frame reveals (Q31) */
    if (fold)
        for (int c = 0; c < N; ++c) {
            if (!vis[c]) continue;
            m->seen[c] = 1;
            if (orc_is_opponent(g, p, g->owner[c])) {
                m->enemy_seen[c] = 1;
                m->last_enemy_turn[c] = g->turn;
            }
            if (g->terrain[c] == T_GENERAL) m->generals[c] = 1;
            if (g->terrain[c] == T_CASTLE) m->castles[c] = 1;
            if (g->terrain[c] == T_MOUNTAIN) m->mountains[c] = 1;
            m->last_enemy_army[c] = enemy[c];
        }
    /* history: the folded frame becomes plane 0, older planes move back */
    if (fold) {
        for (int k = hist; k >= 1; --k) {
            memcpy(m->own_hist + (size_t)k * N, m->own_hist + (size_t)(k - 1) * N, sizeof(int32_t) * (size_t)N);
            memcpy(m->enemy_hist + (size_t)k * N, m->enemy_hist + (size_t)(k - 1) * N, sizeof(int32_t) * (size_t)N);
        }
        memcpy(m->own_hist, own, sizeof(int32_t) * (size_t)N);
        memcpy(m->enemy_hist, enemy, sizeof(int32_t) * (size_t)N);
        m->frame = (int64_t)g->frame;
    }

    /* scoreboard (Q30) */
    int32_t land[MAXP], army[MAXP];
    orc_scoreboard(g, land, army);
    int64_t opp_land = 0, opp_army = 0;
    for (int q = 0; q < g->P; ++q)
        if (orc_is_opponent(g, p, q)) {
            opp_land += land[q];
            opp_army += army[q];
        }

    /* temporal tokens (Q34): the newest entry first, older ones move back */
    if (fold && f->window > 0) {
        for (int k = f->window - 1; k >= 1; --k) {
            m->series[2 * k] = m->series[2 * (k - 1)];
            m->series[2 * k + 1] = m->series[2 * (k - 1) + 1];
        }
        m->series[0] = (int32_t)opp_army;
        m->series[1] = (int32_t)opp_land;
    }
    if (series_out && f->window > 0)
        memcpy(series_out, m->series, sizeof(int32_t) * 2 * (size_t)f->window);

    for (int c = 0; c < N; ++c) {
        const int r = c / W, col = c % W, o = g->owner[c], t = g->terrain[c];
        const int v = vis[c];
        ch[0][c] = (float)(v ? g->army[c] : 0);
        ch[1][c] = (float)own[c];
        ch[2][c] = (float)enemy[c];
        ch[3][c] = (float)((v && o == NEUTRAL) ? g->army[c] : 0);
        ch[4][c] = (float)m->seen[c];
        ch[5][c] = (float)m->enemy_seen[c];
        ch[6][c] = (float)m->generals[c];
        ch[7][c] = (float)m->castles[c];
        ch[8][c] = (float)m->mountains[c];
        ch[9][c] = (float)(v && o == NEUTRAL && t != T_MOUNTAIN);
        ch[10][c] = (float)(o == p);
        ch[11][c] = (float)(v && orc_is_opponent(g, p, o));
        ch[12][c] = (float)(!v);
        ch[13][c] = (float)(!v && (t == T_MOUNTAIN || t == T_CASTLE || m->generals[c]));
        ch[14][c] = (float)g->turn;
        ch[15][c] = (float)((double)(g->turn % 50) / 50.0);
        ch[16][c] = (float)land[p];
        ch[17][c] = (float)army[p];
        ch[18][c] = (float)opp_land;
        ch[19][c] = (float)opp_army;
        ch[20][c] = (float)m->last_enemy_army[c];
        {
            int dt = 0;
            if (!v && m->enemy_seen[c]) dt = g->turn - m->last_enemy_turn[c];
            ch[21][c] = (float)(log(1.0 + (double)dt) / 5.0);
        }
        ch[22][c] = (float)(W > 1 ? (double)col / (double)(W - 1) : 0.0);
        ch[23][c] = (float)(H > 1 ? (double)r / (double)(H - 1) : 0.0);
        /* deltas (Q33) between consecutive folded frames */
        for (int k = 0; k < hist; ++k) {
            ch[24 + k][c] = (float)(m->own_hist[(size_t)k * N + c] - m->own_hist[(size_t)(k + 1) * N + c]);
            ch[24 + hist + k][c] =
                (float)(m->enemy_hist[(size_t)k * N + c] - m->enemy_hist[(size_t)(k + 1) * N + c]);
        }
    }

    free(own);
    free(enemy);
    free(vis);
}

/* every game and player, in order: out holds sum over games of P * C * N
 * floats, game g's player p at [C][N] after those of earlier pairs; series
 * (may be NULL) holds window * 2 int32 per player in the same order */
void orc_feat_build(orc_feat *f, float *out, int32_t *series) {
    const int C = 24 + 2 * f->hist;
    size_t off = 0, soff = 0;
    for (int g = 0; g < f->e->G; ++g)
        for (int p = 0; p < f->e->games[g].P; ++p) {
            orc_feat_player(f, g, p, out + off, series ? series + soff : NULL);
            off += (size_t)C * (size_t)f->e->games[g].N;
            soff += 2 * (size_t)f->window;
        }
}

/* ======================================================================
 * Policy sampling over the H x W x 9 action space (Sec. IV-G; App. C: the
 * policy head's H x W x 9 distribution).  Readings (Q35-Q37 in the design
 * notes):
 *   Q35 legal entries of player p: (c, 0) pass where p owns c; (c, 1 + d)
 *       all-but-one and (c, 5 + d) half where the move is legal (as the
 *       compact mask); a player with no legal entry passes (action 0);
 *   Q36 the categorical is exp(logit) over legal entries, sampled exactly
 *       with integer weights: m = max legal logit, w = floor(E(l - m) 2^24)
 *       with E the exponential below, r = floor(d * S / 2^64) for the
 *       64-bit draw d and S the sum of weights, and the first entry in
 *       index order whose running weight sum exceeds r;
 *   Q37 E(x) = 2^n * P(f) with t = x * log2(e) rounded to float, n =
 *       floor(t), f = t - n, and P the degree-7 Taylor polynomial of 2^f,
 *       sum of (f ln 2)^k / k!, in Horner form with fused multiply-adds;
 *       E = 0 below t = -25 (the weight would be 0).  Every step is an
 *       IEEE single-precision operation, so the result is reproducible.
 * The draw: d = sm(key(seed, global game id, frame, p), 7), the frame of
 * the step that consumes the action.
 * ====================================================================== */
static float orc_exp_q37(float x) {
    const float t = x * 1.4426950408889634f;
    if (t < -25.0f) return 0.0f;
    const float n = floorf(t);
    const float f = t - n;
    float p = 1.5252733804059838e-05f;
    p = fmaf(p, f, 0.00015403530393381606f);
    p = fmaf(p, f, 0.0013333558146428441f);
    p = fmaf(p, f, 0.009618129107628477f);
    p = fmaf(p, f, 0.055504108664821576f);
    p = fmaf(p, f, 0.2402265069591007f);
    p = fmaf(p, f, 0.6931471805599453f);
    p = fmaf(p, f, 1.0f);
    return ldexpf(p, (int)n);
}

/* the exponential of Q37, for the pins */
float orc_exp37(float x) { return orc_exp_q37(x); }

static uint64_t orc_mulhi64(uint64_t a, uint64_t b) {
    const uint64_t a0 = a & 0xFFFFFFFFu, a1 = a >> 32, b0 = b & 0xFFFFFFFFu, b1 = b >> 32;
    const uint64_t p00 = a0 * b0, p01 = a0 * b1, p10 = a1 * b0, p11 = a1 * b1;
    const uint64_t mid = (p00 >> 32) + (p01 & 0xFFFFFFFFu) + (p10 & 0xFFFFFFFFu);
    return p11 + (p01 >> 32) + (p10 >> 32) + (mid >> 32);
}

/* legal entry (c, k) of player p (Q35) */
static int orc_entry_legal(const orc_game *g, int p, int c, int k) {
    if (k == 0) return g->owner[c] == p;
    if (g->finished) return 0;
    return orc_move_legal(g, p, c, (k - 1) & 3);
}

/* logits: per game and player (in order) N * 9 floats; actions [G][8];
 * mask9 (may be NULL): per game and player N * 9 bytes of legal entries */
void orc_sample_actions(const orc_env *e, const float *logits, uint64_t seed, int32_t *actions, uint8_t *mask9) {
    size_t off = 0;
    for (int g = 0; g < e->G; ++g) {
        const orc_game *gm = &e->games[g];
        const uint64_t gid = e->prm.game_id_base + (uint64_t)g;
        for (int p = 0; p < 8; ++p) actions[8 * g + p] = 0;
        for (int p = 0; p < gm->P; ++p) {
            const float *l = logits + off;
            const int n9 = 9 * gm->N;
            int any = 0;
            float m = 0.0f;
            for (int i = 0; i < n9; ++i) {
                const int legal = orc_entry_legal(gm, p, i / 9, i % 9);
                if (mask9) mask9[off + i] = (uint8_t)legal;
                if (legal && (!any || l[i] > m)) m = l[i];
                if (legal) any = 1;
            }
            if (any) {
                uint64_t S = 0;
                for (int i = 0; i < n9; ++i)
                    if (orc_entry_legal(gm, p, i / 9, i % 9))
                        S += (uint64_t)floorf(orc_exp_q37(l[i] - m) * 16777216.0f);
                const uint64_t d = orc_sm(orc_key(seed, gid, gm->frame, (uint64_t)p), 7);
                const uint64_t r = orc_mulhi64(d, S);
                uint64_t run = 0;
                for (int i = 0; i < n9; ++i) {
                    if (!orc_entry_legal(gm, p, i / 9, i % 9)) continue;
                    run += (uint64_t)floorf(orc_exp_q37(l[i] - m) * 16777216.0f);
                    if (run > r) {
                        actions[8 * g + p] = i;
                        break;
                    }
                }
            }
            off += (size_t)n9;
        }
    }
}
