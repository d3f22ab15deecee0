// Device code of libgenerals: one group of lanes advances one Generals.io
// game -- a warp, or for two-player games on small boards a half (two games
// per warp) or, in multi-frame launches, a quarter of one (four per warp).
//
// Per game and step (paper Section IV) the group
//   1. stages the board (int16 armies, int8 owners, int8 terrain) in shared
//      memory with cp.async 16-byte copies;
//   2. resolves the players' moves one after another on its first lane
//      (Sec. IV-D, IV-E), with a group-wide pass for the land transfer of a
//      captured general;
//   3. applies growth (Sec. IV-C) while ballots turn the board into 32-cell
//      bitsets (ownership per player, army >= 2) and reductions total the
//      armies;
//   4. decides termination and reward (Sec. III) and regenerates finished
//      games (Sec. IV-A);
//   5. dilates the (team) ownership bitsets into fog-of-war visibility with
//      word shifts (Sec. IV-B);
//   6. expands bitsets and board bytes into 16-cell observation and mask
//      chunks written with 128-bit streaming stores;
//   7. optionally picks the next actions with the benchmark policy: legal
//      (cell, direction) counts per chunk, a group scan to find the chunk, a
//      scan over its 16 cells to find the cell.
//
// Terrain bytes carry the cell type in bits 0-1 and, in bits 2-5, whether
// the neighbour up / down / left / right exists and is not a mountain.  The
// generator sets these bits once per map (mountains never change), so move
// validation and the mask read them instead of the neighbours.  The public
// state (gen_read_state) shows bits 0-1 only.
//
// No floating point decides anything: all game arithmetic is integer.
#include <cuda_runtime.h>

#include <atomic>

#include <map>
#include <mutex>
#include <tuple>

#include "gk_internal.h"

namespace gk {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
// games with at most two players share a warp: two (16 lanes each) up to
// kPairMaxCells padded cells, and in multi-frame launches four (8 lanes each)
// up to kQuadMaxCells (measured: per-frame launches of small boards lose with
// four, resident rollouts gain)
constexpr int kQuadMaxCells = 576;
constexpr int kPairMaxCells = 1024;
constexpr int kPairMaxPlayers = 2;
constexpr int kPlain = 0, kMountain = 1, kCastle = 2, kGeneral = 3;
constexpr int kArmyMax = 32767;
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ULL;
constexpr uint32_t kSplitThresh = 858993459u;  // floor(0.2 * 2^32)

// ---- SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) as a counter hash -------
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
// n-th output of the SplitMix64 stream seeded with s
__device__ __forceinline__ uint64_t stream_out(uint64_t s, uint64_t n) { return mix64(s + (n + 1) * kGamma); }
__device__ __forceinline__ uint64_t hkey(uint64_t s, uint64_t a, uint64_t b, uint64_t c) {
    return stream_out(stream_out(stream_out(s, a), b), c);
}
__device__ __forceinline__ uint32_t hdraw(uint64_t k, uint64_t i) { return (uint32_t)(stream_out(k, i) >> 32); }
// uniform integer in [0, n) by multiply-shift
__device__ __forceinline__ int uniform_below(uint32_t u, uint32_t n) { return (int)__umulhi(u, n); }

// ---- a group of W lanes working on one game ----------------------------------
// The whole warp (W = 32) or one of its halves (W = 16, two games per warp).
// Collectives name only the group's lanes, so the two halves of a warp run
// their games independently (also through divergent branches).
template <int W>
struct Grp {
    int lane;       // 0 .. W-1
    int shift;      // the group's first lane in the warp
    unsigned mask;  // the group's lanes
    __device__ __forceinline__ explicit Grp(int warp_lane)
        : lane(warp_lane & (W - 1)), shift(W == 32 ? 0 : (warp_lane & (32 - W))),
          mask(W == 32 ? kFull : (((1u << W) - 1u) << (warp_lane & (32 - W)))) {}
    template <class T>
    __device__ __forceinline__ T shfl(T v, int src) const { return __shfl_sync(mask, v, src, W); }
    template <class T>
    __device__ __forceinline__ T shfl_up(T v, int d) const { return __shfl_up_sync(mask, v, d, W); }
    // bit i = lane i of the group (the other half's lanes are masked off)
    __device__ __forceinline__ unsigned ballot(bool pr) const {
        if (W == 32) return __ballot_sync(kFull, pr);
        return (__ballot_sync(mask, pr) & mask) >> shift;
    }
    __device__ __forceinline__ unsigned reduce_add(unsigned v) const {
        if constexpr (W == 32) {
            return __reduce_add_sync(kFull, v);
        } else {
#pragma unroll
            for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, W);
            return v;
        }
    }
    __device__ __forceinline__ bool any(bool pr) const {
        if (W == 32) return __any_sync(kFull, pr);
        return ballot(pr) != 0u;
    }
    __device__ __forceinline__ void sync() const { __syncwarp(mask); }
};

// ---- per-warp shared-memory view --------------------------------------------
struct Smem {
    int16_t* army;
    int8_t* owner;
    uint8_t* terrain;  // type | passable-neighbour bits << 2
    uint32_t* own;     // [pmax][stride]
    uint32_t* big;     // army >= 2
    uint32_t* col0;    // first column
    uint32_t* colL;    // last column
    uint32_t* vis;     // [pmax][stride]
    uint32_t* tmp;
    // legal moves per (player, 16-cell chunk), one region in one of two forms:
    // groups narrower than a warp (two-player games, issue-bound) keep each
    // chunk's 64-bit mask (bit 4j + d: cell j towards d); a warp per game
    // keeps only its count of legal pairs (a byte), which keeps 8-player
    // carves small, and the policy rebuilds the selected chunk's mask from
    // the board
    uint64_t* legal;   // [pmax][chunks], narrow groups
    uint8_t* cnt;      // [pmax][chunks], a warp per game (same bytes)
    int32_t* misc;     // [0..7] general cells, [8..15] land, [16..23] army
    int stride;
};

// bytes of the legal-move region of a carve: masks for narrow groups, counts for a warp per game
__host__ __device__ __forceinline__ int legal_region_bytes(int npad_max, int pmax, bool narrow) {
    return narrow ? 8 * pmax * (npad_max >> 4) : ((pmax * (npad_max >> 4) + 15) & ~15);
}

// A group's shared-memory geometry packed in one word: padded cells of the
// largest board (13 bits), bitset stride in words (8 bits), players (4 bits),
// and whether the group is narrower than a warp (bit 25: the mask form of
// the legal-move region).
__host__ __device__ __forceinline__ uint32_t pack_geom(int npad_max, int nw_stride, int pmax, bool narrow) {
    return (uint32_t)npad_max | ((uint32_t)nw_stride << 13) | ((uint32_t)pmax << 21) | (narrow ? 1u << 25 : 0u);
}
template <int LW>
__device__ __forceinline__ uint32_t geom_of(const KArgs& a) {
    return pack_geom(a.npad_max, a.nw_stride, a.pmax, LW < 32);
}

__device__ __forceinline__ Smem carve_dims(char* base, const int np, const int st, const int pm, const bool narrow) {
    Smem s;
    s.army = reinterpret_cast<int16_t*>(base);
    s.owner = reinterpret_cast<int8_t*>(base + 2 * np);
    s.terrain = reinterpret_cast<uint8_t*>(base + 3 * np);
    uint32_t* w = reinterpret_cast<uint32_t*>(base + 4 * np);
    s.own = w;
    w += pm * st;
    s.big = w;
    w += st;
    s.col0 = w;
    w += st;
    s.colL = w;
    w += st;
    s.vis = w;
    w += pm * st;
    s.tmp = w;
    w += st;
    s.legal = reinterpret_cast<uint64_t*>(w);  // 8-byte aligned: every region above is
    s.cnt = reinterpret_cast<uint8_t*>(w);
    w += legal_region_bytes(np, pm, narrow) >> 2;  // whole 16-byte units
    s.misc = reinterpret_cast<int32_t*>(w);
    s.stride = st;
    return s;
}
__device__ __forceinline__ Smem carve_geom(char* base, uint32_t geom) {
    return carve_dims(base, (int)(geom & 0x1FFFu), (int)((geom >> 13) & 0xFFu), (int)((geom >> 21) & 0xFu),
                      ((geom >> 25) & 1u) != 0u);
}
// the launch's own geometry, straight from the kernel parameters
template <int LW>
__device__ __forceinline__ Smem carve(char* base, const KArgs& a) {
    return carve_dims(base, a.npad_max, a.nw_stride, a.pmax, LW < 32);
}

struct Game {
    int H, W, N, Npad, nch, P, mode, nw;
    int64_t plane_off;
    int cell_off, player_off, n_cities, dmin;
};

__device__ __forceinline__ Game load_game(const GameInfo* gi) {
    Game g;
    g.H = gi->H;
    g.W = gi->W;
    g.N = gi->N;
    g.Npad = gi->Npad;
    g.nch = gi->Npad >> 4;
    g.P = gi->P;
    g.mode = gi->mode;
    g.nw = (gi->N + 31) >> 5;
    g.plane_off = gi->plane_off;
    g.cell_off = gi->cell_off;
    g.player_off = gi->player_off;
    g.n_cities = gi->n_cities;
    g.dmin = gi->dmin;
    return g;
}

// UNI: the launch's games all have the launch's shape (a.uniform), so every
// field is a kernel parameter or follows from gidx; a kernel compiled for it
// keeps none of them in registers.
template <bool UNI = false>
__device__ __forceinline__ Game game_of(const KArgs& a, int gidx) {
    if (!UNI && !a.uniform) return load_game(a.info + gidx);
    Game g = load_game(&a.ushape);
    g.cell_off = gidx * g.Npad;
    g.player_off = gidx * g.P;
    g.plane_off = (int64_t)gidx * g.P * g.Npad;
    return g;
}
template <bool UNI = false>
__device__ __forceinline__ uint64_t game_id_of(const KArgs& a, int gidx) {
    return (UNI || a.uniform) ? a.game_id_base + (uint64_t)gidx : a.info[gidx].game_id;
}

__device__ __forceinline__ uint32_t valid_bits(int N, int w) {
    int rem = N - 32 * w;
    if (rem >= 32) return kFull;
    if (rem <= 0) return 0u;
    return (1u << rem) - 1u;
}

// passable-neighbour bits of every cell (bits 2..5 of the terrain byte),
// from a mountain bitset so that no lane reads a byte another lane writes
template <int LW>
__device__ __forceinline__ void derive_passable(const Game& g, const Smem& s, const Grp<LW>& t) {
    const int N = g.N, W = g.W, H = g.H;
    for (int w = 0; w < g.nw; ++w) {
        unsigned m = 0;
        for (int h = 0; h < 32; h += LW) {
            const int c = 32 * w + h + t.lane;
            m |= t.ballot(c < N && (s.terrain[c] & 3) == kMountain) << h;
        }
        if (t.lane == 0) s.tmp[w] = m;
    }
    t.sync();
    for (int c = t.lane; c < N; c += LW) {
        const int r = c / W, col = c - r * W;
        auto mtn = [&](int x) { return (s.tmp[x >> 5] >> (x & 31)) & 1u; };
        uint32_t b = 0;
        if (r > 0 && !mtn(c - W)) b |= 1u;
        if (r < H - 1 && !mtn(c + W)) b |= 2u;
        if (col > 0 && !mtn(c - 1)) b |= 4u;
        if (col < W - 1 && !mtn(c + 1)) b |= 8u;
        s.terrain[c] = (uint8_t)((s.terrain[c] & 3) | (b << 2));
    }
    t.sync();
}

// ---- board geometry: first and last column bitsets -------------------------
// g_columns[W-1][0][w] has bit b set when cell 32w+b is in the first column
// of a W-wide board, [1] the last column; filled once per device.
constexpr int kColWords = (kMaxSide * kMaxSide) / 32;
__device__ __align__(16) uint32_t g_columns[kMaxSide][2][kColWords];

template <int LW>
__device__ __forceinline__ void column_pass(const Game& g, const Smem& s, const Grp<LW>& t) {
    const uint32_t* c0 = g_columns[g.W - 1][0];
    const uint32_t* cl = g_columns[g.W - 1][1];
    for (int w = t.lane; w < g.nw; w += LW) {
        s.col0[w] = c0[w];
        s.colL[w] = cl[w];
    }
    t.sync();
}

// ---- bitset BFS (generator options) ----------------------------------------
// Word arrays of nw words in shared memory, one lane per word.  Bit c of
// dilate4(x) is set when a 4-neighbour of cell c is set in x.
__device__ void dilate4(const uint32_t* x, uint32_t* out, const Game& g, const Smem& s, int lane) {
    const int nw = g.nw, q = g.W >> 5, sh = g.W & 31;
    for (int w = lane; w < nw; w += 32) {
        const uint32_t X = x[w];
        const uint32_t Xm = w > 0 ? x[w - 1] : 0u, Xp = w + 1 < nw ? x[w + 1] : 0u;
        const uint32_t L = (X << 1) | (Xm >> 31);  // bit c <- cell c-1
        const uint32_t R = (X >> 1) | (Xp << 31);  // bit c <- cell c+1
        uint32_t v = (L & ~s.col0[w]) | (R & ~s.colL[w]);
        const int wa = w - q;  // bit c <- cell c-W
        if (wa >= 0) v |= x[wa] << sh;
        if (sh && wa - 1 >= 0) v |= x[wa - 1] >> (32 - sh);
        const int wb = w + q;  // bit c <- cell c+W
        if (wb < nw) v |= x[wb] >> sh;
        if (sh && wb + 1 < nw) v |= x[wb + 1] << (32 - sh);
        out[w] = v & valid_bits(g.N, w);
    }
    __syncwarp();
}

__device__ __forceinline__ void set_single(uint32_t* x, int c, const Game& g, int lane) {
    for (int w = lane; w < g.nw; w += 32) x[w] = (w == (c >> 5)) ? (1u << (c & 31)) : 0u;
    __syncwarp();
}

// BFS from src through `pass`.  keep_out (when lo >= 0): cells within lo
// steps leave `allowed`; then `allowed` keeps only cells within hi steps
// (hi <= 0: all reachable cells).  vis / front / nxt are scratch.
__device__ void bfs_restrict(int src, int lo, int hi, const uint32_t* pass, uint32_t* allowed, uint32_t* vis,
                             uint32_t* front, uint32_t* nxt, const Game& g, const Smem& s, int lane) {
    set_single(vis, src, g, lane);
    set_single(front, src, g, lane);
    bool cut = false;
    if (lo == 0) {
        for (int w = lane; w < g.nw; w += 32) allowed[w] &= ~vis[w];
        cut = true;
    }
    for (int step = 1; hi <= 0 || step <= hi; ++step) {
        dilate4(front, nxt, g, s, lane);
        bool any = false;
        for (int w = lane; w < g.nw; w += 32) {
            const uint32_t n = nxt[w] & pass[w] & ~vis[w];
            front[w] = n;
            vis[w] |= n;
            any |= n != 0u;
        }
        __syncwarp();
        if (!__any_sync(kFull, any)) break;
        if (step == lo) {
            for (int w = lane; w < g.nw; w += 32) allowed[w] &= ~vis[w];
            cut = true;
        }
    }
    __syncwarp();
    for (int w = lane; w < g.nw; w += 32) allowed[w] &= (lo >= 0 && !cut) ? 0u : vis[w];
    __syncwarp();
}

// first set bit (row-major) of x, or -1
__device__ int first_bit(const uint32_t* x, const Game& g, int lane) {
    int best = 0x7FFFFFFF;
    for (int w = lane; w < g.nw; w += 32)
        if (x[w]) best = min(best, 32 * w + __ffs(x[w]) - 1);
    best = (int)__reduce_min_sync(kFull, (unsigned)best);
    return best == 0x7FFFFFFF ? -1 : best;
}

// cell of the k-th (0-based, row-major) set bit of x; x holds more than k bits
__device__ int kth_bit(const uint32_t* x, uint32_t k, const Game& g, int lane) {
    const int wpl = (g.nw + 31) >> 5, w0 = lane * wpl;
    uint32_t mine = 0;
    for (int w = w0; w < w0 + wpl && w < g.nw; ++w) mine += __popc(x[w]);
    uint32_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const int L = __ffs(__ballot_sync(kFull, incl > k)) - 1;
    int cell = 0;
    if (lane == L) {
        uint32_t r = k - (incl - mine);
        for (int w = w0; w < w0 + wpl && w < g.nw; ++w) {
            uint32_t v = x[w];
            const uint32_t n = __popc(v);
            if (r >= n) {
                r -= n;
                continue;
            }
            for (uint32_t z = 0; z < r; ++z) v &= v - 1;
            cell = 32 * w + __ffs(v) - 1;
            break;
        }
    }
    return __shfl_sync(kFull, cell, L);
}

// bitset of cells matching a predicate on (terrain type, owner), one ballot per word
template <class Pred>
__device__ void cell_bits(uint32_t* out, const Game& g, const Smem& s, int lane, Pred pred) {
    for (int w = 0; w < g.nw; ++w) {
        const int c = 32 * w + lane;
        const bool b = c < g.N && pred(s.terrain[c] & 3, (int)s.owner[c]);
        const unsigned m = __ballot_sync(kFull, b);
        if (lane == 0) out[w] = m;
    }
    __syncwarp();
}

// ---- map generator with spawn options (Sec. IV-A) --------------------------
// Scratch bitsets of the spawn options; the step rebuilds these arrays.
struct GenScratch {
    uint32_t *pass, *front, *nxt, *vis, *allowed, *gens;
};
__device__ __forceinline__ GenScratch gen_scratch(const Smem& s) {
    const int st = s.stride;
    return GenScratch{s.big, s.own, s.own + st, s.vis, s.vis + st, s.tmp};
}

// Generals at BFS distance (through non-mountain cells) in [D, dmax] of every
// earlier general, D falling by one after each kGenAttempts rejected draws;
// at D = 0 the first cell (row-major) within the cap of every earlier general,
// else reachable from general 0, else any free cell.  Lane p returns player
// p's general in the low 16 bits; bit 20 says whether a general cannot reach
// general 0 (the L-path carve is then needed).
__device__ __noinline__ int place_generals_bfs(const Game& g, const Smem& s, uint64_t kgen, int dmax, int lane) {
    const int N = g.N, P = g.P;
    const GenScratch z = gen_scratch(s);
    column_pass(g, s, Grp<32>(lane));
    cell_bits(z.pass, g, s, lane, [](int t, int) { return t != kMountain; });
    for (int w = lane; w < g.nw; w += 32) z.gens[w] = 0u;
    __syncwarp();
    uint32_t i = 0;
    int D = g.dmin;
    int my_gpos = -1;
    for (int p = 0; p < P; ++p) {
        int placed = -1;
        while (placed < 0) {
            if (D >= 1) {
                for (int w = lane; w < g.nw; w += 32) z.allowed[w] = z.pass[w];
                __syncwarp();
                for (int q = 0; q < p; ++q)
                    bfs_restrict(__shfl_sync(kFull, my_gpos, q), D - 1, dmax, z.pass, z.allowed, z.vis, z.front,
                                 z.nxt, g, s, lane);
                int found = -1;
                for (int base = 0; base < kGenAttempts; base += 32) {
                    const int t = base + lane;
                    const int c = uniform_below(hdraw(kgen, (uint64_t)(i + t)), (uint32_t)N);
                    const bool ok = t < kGenAttempts && ((z.allowed[c >> 5] >> (c & 31)) & 1u);
                    const unsigned b = __ballot_sync(kFull, ok);
                    if (b) {
                        const int l = __ffs(b) - 1;
                        found = base + l;
                        placed = __shfl_sync(kFull, c, l);
                        break;
                    }
                }
                if (found >= 0) {
                    i += (uint32_t)found + 1;
                } else {
                    i += kGenAttempts;
                    D -= 1;
                }
            } else {
                for (int w = lane; w < g.nw; w += 32) z.allowed[w] = z.pass[w] & ~z.gens[w];
                __syncwarp();
                for (int q = 0; q < p; ++q)
                    bfs_restrict(__shfl_sync(kFull, my_gpos, q), -1, dmax, z.pass, z.allowed, z.vis, z.front, z.nxt,
                                 g, s, lane);
                placed = first_bit(z.allowed, g, lane);
                if (placed < 0) {
                    for (int w = lane; w < g.nw; w += 32) z.allowed[w] = z.pass[w] & ~z.gens[w];
                    __syncwarp();
                    if (p > 0)
                        bfs_restrict(__shfl_sync(kFull, my_gpos, 0), -1, 0, z.pass, z.allowed, z.vis, z.front, z.nxt,
                                     g, s, lane);
                    placed = first_bit(z.allowed, g, lane);
                }
                if (placed < 0) {
                    for (int w = lane; w < g.nw; w += 32) z.allowed[w] = ~z.gens[w] & valid_bits(N, w);
                    __syncwarp();
                    placed = first_bit(z.allowed, g, lane);
                }
            }
        }
        if (lane == p) my_gpos = placed;
        if (lane == (placed >> 5)) z.gens[placed >> 5] |= 1u << (placed & 31);
        __syncwarp();
    }
    bool carve = false;
    if (P > 1) {
        for (int w = lane; w < g.nw; w += 32) z.allowed[w] = z.gens[w];
        __syncwarp();
        bfs_restrict(__shfl_sync(kFull, my_gpos, 0), -1, 0, z.pass, z.allowed, z.vis, z.front, z.nxt, g, s, lane);
        bool miss = false;
        for (int w = lane; w < g.nw; w += 32) miss |= z.allowed[w] != z.gens[w];
        carve = __any_sync(kFull, miss);
    }
    return (my_gpos & 0xFFFF) | (carve ? (1 << 20) : 0);
}

// A neutral castle within `radius` BFS steps of every general (s.misc holds
// the generals): where none is, one on a free plain cell of the ball, the
// k-th such cell in row-major order with k drawn uniformly.
__device__ __noinline__ void castle_guarantee(const KArgs& a, const Game& g, const Smem& s, uint64_t gid,
                                              uint32_t epoch, int radius, int lane) {
    const GenScratch z = gen_scratch(s);
    column_pass(g, s, Grp<32>(lane));
    uint32_t* free_plain = z.gens;
    cell_bits(z.pass, g, s, lane, [](int t, int) { return t != kMountain; });
    cell_bits(free_plain, g, s, lane, [](int t, int o) { return t == kPlain && o == -1; });
    const uint64_t knp = hkey(a.seed, gid, epoch, 5);
    const uint64_t kna = hkey(a.seed, gid, epoch, 6);
    for (int p = 0; p < g.P; ++p) {
        const int gp = s.misc[p];
        cell_bits(z.allowed, g, s, lane, [](int t, int o) { return t == kCastle && o == -1; });
        bfs_restrict(gp, -1, radius, z.pass, z.allowed, z.vis, z.front, z.nxt, g, s, lane);
        bool have = false;
        for (int w = lane; w < g.nw; w += 32) have |= z.allowed[w] != 0u;
        if (__any_sync(kFull, have)) continue;
        for (int w = lane; w < g.nw; w += 32) z.allowed[w] = free_plain[w] & z.vis[w];  // vis: the ball
        __syncwarp();
        uint32_t cnt = 0;
        for (int w = lane; w < g.nw; w += 32) cnt += __popc(z.allowed[w]);
        cnt = __reduce_add_sync(kFull, cnt);
        if (cnt == 0) continue;
        const int cell = kth_bit(z.allowed, (uint32_t)uniform_below(hdraw(knp, (uint64_t)p), cnt), g, lane);
        if (lane == 0) {
            s.terrain[cell] = kCastle;
            s.army[cell] = (int16_t)(a.city_min + uniform_below(hdraw(kna, (uint64_t)p), (uint32_t)a.city_span));
        }
        if (lane == (cell >> 5)) free_plain[cell >> 5] &= ~(1u << (cell & 31));
        __syncwarp();
    }
}

// The generator with spawn options (the launch's spawn_dmax, spawn_bfs,
// castle_radius).  It is a separate function of a separate kernel
// instantiation so that the options' register pressure never reaches the
// step kernel that runs without them.
__device__ __forceinline__ void generate_spawn_body(const KArgs& a, const Game& g, const Smem& s, uint64_t gid,
                                                   uint32_t epoch, int lane) {
    const int N = g.N, W = g.W, P = g.P;
    const uint64_t kmtn = hkey(a.seed, gid, epoch, 1);
    for (int c = lane; c < g.Npad; c += 32) {
        bool m = c < N && hdraw(kmtn, (uint64_t)c) < a.mtn_thresh;
        s.army[c] = 0;
        s.owner[c] = -1;
        s.terrain[c] = m ? kMountain : kPlain;
    }
    __syncwarp();

    // generals: 32 candidate draws evaluated at once; the first accepted in
    // draw order wins, so the draw counter advances exactly as one by one
    const uint64_t kgen = hkey(a.seed, gid, epoch, 2);
    const int dmax = a.spawn_dmax;
    int my_gpos = -1;  // lane p holds player p's general
    bool carve = true;
    if (a.spawn_bfs) {
        const int r = place_generals_bfs(g, s, kgen, dmax, lane);
        my_gpos = lane < P ? (r & 0xFFFF) : -1;
        carve = (r >> 20) & 1;
    } else {
        uint32_t i = 0;
        int D = g.dmin;
        for (int p = 0; p < P; ++p) {
            int placed = -1;
            while (placed < 0) {
                if (D >= 1) {
                    int found = -1;
                    for (int base = 0; base < kGenAttempts; base += 32) {
                        int t = base + lane;
                        int c = uniform_below(hdraw(kgen, (uint64_t)(i + t)), (uint32_t)N);
                        bool ok = (t < kGenAttempts) && s.terrain[c] != kMountain;
                        int rc = c / W, cc = c - rc * W;
                        for (int q = 0; q < p; ++q) {
                            int gq = __shfl_sync(kFull, my_gpos, q);
                            int rq = gq / W, cq = gq - rq * W;
                            const int d = abs(rc - rq) + abs(cc - cq);
                            if (d < D || (dmax > 0 && d > dmax)) ok = false;
                        }
                        unsigned b = __ballot_sync(kFull, ok);
                        if (b) {
                            int l = __ffs(b) - 1;
                            found = base + l;
                            placed = __shfl_sync(kFull, c, l);
                            break;
                        }
                    }
                    if (found >= 0) {
                        i += (uint32_t)found + 1;
                    } else {
                        i += kGenAttempts;
                        D -= 1;
                    }
                } else {
                    for (int base = 0; base < N && placed < 0; base += 32) {
                        int c = base + lane;
                        bool ok = c < N;
                        for (int q = 0; q < p; ++q)
                            if (__shfl_sync(kFull, my_gpos, q) == c) ok = false;
                        unsigned b = __ballot_sync(kFull, ok);
                        if (b) placed = base + __ffs(b) - 1;
                    }
                }
            }
            if (lane == p) my_gpos = placed;
        }
    }
    if (lane < P) {
        s.terrain[my_gpos] = kGeneral;
        s.owner[my_gpos] = (int8_t)lane;
        s.army[my_gpos] = 1;
        s.misc[lane] = my_gpos;
    }
    __syncwarp();

    // L-path rows first, then columns, between consecutive generals (in BFS
    // mode only when some general cannot reach general 0)
    if (carve && lane == 0) {
        for (int p = 0; p + 1 < P; ++p) {
            int r = s.misc[p] / W, c = s.misc[p] % W;
            int r1 = s.misc[p + 1] / W, c1 = s.misc[p + 1] % W;
            while (r != r1) {
                r += (r1 > r) ? 1 : -1;
                if (s.terrain[r * W + c] == kMountain) s.terrain[r * W + c] = kPlain;
            }
            while (c != c1) {
                c += (c1 > c) ? 1 : -1;
                if (s.terrain[r * W + c] == kMountain) s.terrain[r * W + c] = kPlain;
            }
        }
    }
    __syncwarp();

    // neutral castles on neutral plain cells
    const uint64_t kpos = hkey(a.seed, gid, epoch, 3);
    const uint64_t karm = hkey(a.seed, gid, epoch, 4);
    uint32_t j = 0;
    for (int k = 0; k < g.n_cities; ++k) {
        int found = -1, cell = 0;
        for (int base = 0; base < kGenAttempts; base += 32) {
            int t = base + lane;
            int c = uniform_below(hdraw(kpos, (uint64_t)(j + t)), (uint32_t)N);
            bool ok = (t < kGenAttempts) && s.terrain[c] == kPlain && s.owner[c] == -1;
            unsigned b = __ballot_sync(kFull, ok);
            if (b) {
                int l = __ffs(b) - 1;
                found = base + l;
                cell = __shfl_sync(kFull, c, l);
                break;
            }
        }
        if (found >= 0) {
            j += (uint32_t)found + 1;
            if (lane == 0) {
                s.terrain[cell] = kCastle;
                s.army[cell] = (int16_t)(a.city_min + uniform_below(hdraw(karm, (uint64_t)k), (uint32_t)a.city_span));
            }
            __syncwarp();
        } else {
            j += kGenAttempts;
        }
    }

    if (a.castle_radius > 0) castle_guarantee(a, g, s, gid, epoch, a.castle_radius, lane);
    derive_passable(g, s, Grp<32>(lane));
}

// ---- map generator (Sec. IV-A) ----------------------------------------------
template <int LW>
__device__ __forceinline__ void generate_body(const KArgs& a, const Game& g, const Smem& s, uint64_t gid,
                                             uint32_t epoch, const Grp<LW>& t) {
    const int N = g.N, W = g.W, P = g.P;
    const uint64_t kmtn = hkey(a.seed, gid, epoch, 1);
    for (int c = t.lane; c < g.Npad; c += LW) {
        bool m = c < N && hdraw(kmtn, (uint64_t)c) < a.mtn_thresh;
        s.army[c] = 0;
        s.owner[c] = -1;
        s.terrain[c] = m ? kMountain : kPlain;
    }
    t.sync();

    // generals: LW candidate draws evaluated at once; the first accepted in
    // draw order wins, so the draw counter advances exactly as one by one
    const uint64_t kgen = hkey(a.seed, gid, epoch, 2);
    uint32_t i = 0;
    int D = g.dmin;
    int my_gpos = -1;  // lane p holds player p's general
    for (int p = 0; p < P; ++p) {
        int placed = -1;
        while (placed < 0) {
            if (D >= 1) {
                int found = -1;
                for (int base = 0; base < kGenAttempts; base += LW) {
                    const int dr = base + t.lane;  // draw index
                    int c = uniform_below(hdraw(kgen, (uint64_t)(i + dr)), (uint32_t)N);
                    bool ok = (dr < kGenAttempts) && s.terrain[c] != kMountain;
                    int rc = c / W, cc = c - rc * W;
                    for (int q = 0; q < p; ++q) {
                        int gq = t.shfl(my_gpos, q);
                        int rq = gq / W, cq = gq - rq * W;
                        if (abs(rc - rq) + abs(cc - cq) < D) ok = false;
                    }
                    unsigned b = t.ballot(ok);
                    if (b) {
                        int l = __ffs(b) - 1;
                        found = base + l;
                        placed = t.shfl(c, l);
                        break;
                    }
                }
                if (found >= 0) {
                    i += (uint32_t)found + 1;
                } else {
                    i += kGenAttempts;
                    D -= 1;
                }
            } else {
                for (int base = 0; base < N && placed < 0; base += LW) {
                    int c = base + t.lane;
                    bool ok = c < N;
                    for (int q = 0; q < p; ++q)
                        if (t.shfl(my_gpos, q) == c) ok = false;
                    unsigned b = t.ballot(ok);
                    if (b) placed = base + __ffs(b) - 1;
                }
            }
        }
        if (t.lane == p) my_gpos = placed;
    }
    if (t.lane < P) {
        s.terrain[my_gpos] = kGeneral;
        s.owner[my_gpos] = (int8_t)t.lane;
        s.army[my_gpos] = 1;
        s.misc[t.lane] = my_gpos;
    }
    t.sync();

    // connectivity: L-path rows first, then columns, between consecutive generals
    if (t.lane == 0) {
        for (int p = 0; p + 1 < P; ++p) {
            int r = s.misc[p] / W, c = s.misc[p] % W;
            int r1 = s.misc[p + 1] / W, c1 = s.misc[p + 1] % W;
            while (r != r1) {
                r += (r1 > r) ? 1 : -1;
                if (s.terrain[r * W + c] == kMountain) s.terrain[r * W + c] = kPlain;
            }
            while (c != c1) {
                c += (c1 > c) ? 1 : -1;
                if (s.terrain[r * W + c] == kMountain) s.terrain[r * W + c] = kPlain;
            }
        }
    }
    t.sync();

    // neutral castles on neutral plain cells
    const uint64_t kpos = hkey(a.seed, gid, epoch, 3);
    const uint64_t karm = hkey(a.seed, gid, epoch, 4);
    uint32_t j = 0;
    for (int k = 0; k < g.n_cities; ++k) {
        int found = -1, cell = 0;
        for (int base = 0; base < kGenAttempts; base += LW) {
            const int dr = base + t.lane;  // draw index
            int c = uniform_below(hdraw(kpos, (uint64_t)(j + dr)), (uint32_t)N);
            bool ok = (dr < kGenAttempts) && s.terrain[c] == kPlain && s.owner[c] == -1;
            unsigned b = t.ballot(ok);
            if (b) {
                int l = __ffs(b) - 1;
                found = base + l;
                cell = t.shfl(c, l);
                break;
            }
        }
        if (found >= 0) {
            j += (uint32_t)found + 1;
            if (t.lane == 0) {
                s.terrain[cell] = kCastle;
                s.army[cell] = (int16_t)(a.city_min + uniform_below(hdraw(karm, (uint64_t)k), (uint32_t)a.city_span));
            }
            t.sync();
        } else {
            j += kGenAttempts;
        }
    }
    derive_passable(g, s, t);
}

// Out-of-line entry points of the cold paths take plain arguments and rebuild
// the game and shared-memory views themselves, so that the step kernel never
// materialises those structures in local memory for a call it rarely makes.
template <int LW, bool UNI>
__device__ __noinline__ void generate(const KArgs& a, int gidx, char* warp_base, uint32_t geom, uint64_t gid,
                                     uint32_t epoch, int warp_lane) {
    generate_body(a, game_of<UNI>(a, gidx), carve_geom(warp_base, geom), gid, epoch, Grp<LW>(warp_lane));
}
__device__ __noinline__ void generate_spawn(const KArgs& a, int gidx, char* warp_base, uint32_t geom, uint64_t gid,
                                           uint32_t epoch, int lane) {
    generate_spawn_body(a, game_of(a, gidx), carve_geom(warp_base, geom), gid, epoch, lane);
}
template <int LW, bool UNI>
__device__ __noinline__ void derive_passable_at(const KArgs& a, int gidx, char* warp_base, uint32_t geom,
                                               int warp_lane) {
    derive_passable(game_of<UNI>(a, gidx), carve_geom(warp_base, geom), Grp<LW>(warp_lane));
}

// ---- one move on lane 0 (Sec. IV-D, IV-E) ----------------------------------
// Returns the captured general's cell in the low 16 bits and the loser in
// bits 16..19 (+1), or 0 when no general fell.
__device__ int resolve_move(const Game& g, const Smem& s, int p, int32_t act, uint32_t& alive, uint32_t& invalid,
                            uint32_t& sat) {
    if (act < 0 || act >= 9 * g.N) {
        invalid += 1;
        return 0;
    }
    const int c = act / 9, k = act - 9 * c;
    if (k == 0) return 0;
    const int d = (k - 1) & 3;
    const int av = s.army[c];
    // bit 2+d: the neighbour towards d exists and is not a mountain
    if (s.owner[c] != p || av < 2 || !((s.terrain[c] >> (2 + d)) & 1u)) {
        invalid += 1;
        return 0;
    }
    const int dst = c + (d == 0 ? -g.W : d == 1 ? g.W : d == 2 ? -1 : 1);
    const int moved = (k >= 5) ? (av >> 1) : (av - 1);
    s.army[c] = (int16_t)(av - moved);
    const int o = s.owner[dst];
    const int def = s.army[dst];
    if (o == p || (o >= 0 && g.mode == 1 && (o >> 1) == (p >> 1))) {
        int sum = def + moved;
        if (sum > kArmyMax) {
            sum = kArmyMax;
            sat += 1;
        }
        s.army[dst] = (int16_t)sum;
        if (o != p && (s.terrain[dst] & 3) != kGeneral) s.owner[dst] = (int8_t)p;
        return 0;
    }
    if (moved > def) {
        s.owner[dst] = (int8_t)p;
        s.army[dst] = (int16_t)(moved - def);
        if ((s.terrain[dst] & 3) == kGeneral && o >= 0) {
            s.terrain[dst] = (uint8_t)((s.terrain[dst] & ~3u) | kCastle);
            alive &= ~(1u << o);
            return dst | ((o + 1) << 16);
        }
    } else if (moved == def) {
        s.army[dst] = 0;
    } else {
        s.army[dst] = (int16_t)(def - moved);
    }
    return 0;
}

// ---- growth + bitsets + army totals, 16 cells per lane ---------------------
// Bytes are compared four at a time inside 32-bit words: zero_bytes(x) has
// 0x80 in every byte of x that is zero (exact, no carries between bytes).
__device__ __forceinline__ uint32_t zero_bytes(uint32_t x) {
    const uint32_t t = (x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu;
    return ~(t | x) & 0x80808080u;
}
// bits 7, 15, 23, 31 of x -> bits 0..3
__device__ __forceinline__ uint32_t gather4(uint32_t x80) { return (x80 * 0x00204081u) >> 28; }

template <int PT, int LW>
__device__ uint32_t chunk_pass(const Game& g, const Smem& s, bool grow_s, bool grow_p, const Grp<LW>& t) {
    const int P = g.P, nch = g.nch, st2 = 2 * s.stride;
    const bool grow = grow_s || grow_p;
    uint32_t sat = 0;
    int arm[PT];
#pragma unroll
    for (int p = 0; p < PT; ++p) arm[p] = 0;
    uint16_t* own16 = reinterpret_cast<uint16_t*>(s.own);
    uint16_t* big16 = reinterpret_cast<uint16_t*>(s.big);
    for (int ch = t.lane; ch < nch; ch += LW) {
        const int c0 = ch << 4;
        const uint4 O = *reinterpret_cast<const uint4*>(s.owner + c0);
        const uint4 A0 = *reinterpret_cast<const uint4*>(s.army + c0);
        const uint4 A1 = *reinterpret_cast<const uint4*>(s.army + c0 + 8);
        const uint32_t ow[4] = {O.x, O.y, O.z, O.w};
        uint32_t aw[8] = {A0.x, A0.y, A0.z, A0.w, A1.x, A1.y, A1.z, A1.w};
        if (grow) {
            // owned generals / castles (+1 on even turns), owned plain (+1 every 50)
            const uint4 T = *reinterpret_cast<const uint4*>(s.terrain + c0);
            const uint32_t tw[4] = {T.x, T.y, T.z, T.w};
            bool changed = false;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t owned = ~zero_bytes(~ow[k]) & 0x80808080u;
                const uint32_t structure = (tw[k] << 6) & 0x80808080u;       // type bit 1
                const uint32_t plain = zero_bytes(tw[k] & 0x03030303u);
                const uint32_t g80 = owned & ((grow_s ? structure : 0u) | (grow_p ? plain : 0u));
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t inc = (__byte_perm(g80, 0, h ? 0x3322 : 0x1100) >> 15) & 0x00010001u;
                    uint32_t v = aw[2 * k + h] + inc;
                    const uint32_t ov = v & 0x80008000u;  // 32767 + 1
                    sat += __popc(ov);
                    v -= ov >> 15;
                    changed |= (inc != 0u);
                    aw[2 * k + h] = v;
                }
            }
            if (changed) {
                *reinterpret_cast<uint4*>(s.army + c0) = make_uint4(aw[0], aw[1], aw[2], aw[3]);
                *reinterpret_cast<uint4*>(s.army + c0 + 8) = make_uint4(aw[4], aw[5], aw[6], aw[7]);
            }
        }
        // army >= 2: bit 15 / 31 of army + 0x7FFE per halfword
        uint32_t big = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t y0 = aw[2 * k] + 0x7FFE7FFEu, y1 = aw[2 * k + 1] + 0x7FFE7FFEu;
            big |= gather4(__byte_perm(y0, y1, 0x7531) & 0x80808080u) << (4 * k);
        }
        big16[ch] = (uint16_t)big;
        // army totals: low and high bytes of 4 armies dotted with 0/1 owner bytes
        uint32_t lo4[4], hi4[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            lo4[k] = __byte_perm(aw[2 * k], aw[2 * k + 1], 0x6420);
            hi4[k] = __byte_perm(aw[2 * k], aw[2 * k + 1], 0x7531);
        }
#pragma unroll
        for (int p = 0; p < PT; ++p) {
            if (p < P) {
                uint32_t own = 0, slo = 0, shi = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t z = zero_bytes(ow[k] ^ (0x01010101u * (uint32_t)p));
                    own |= gather4(z) << (4 * k);
                    const uint32_t m = z >> 7;
                    slo = __dp4a(lo4[k], m, slo);
                    shi = __dp4a(hi4[k], m, shi);
                }
                arm[p] += (int)(slo + 256u * shi);
                own16[p * st2 + ch] = (uint16_t)own;
            }
        }
        if ((nch & 1) && ch == nch - 1) {  // unused upper half of the last word
            big16[nch] = 0;
#pragma unroll
            for (int p = 0; p < PT; ++p)
                if (p < P) own16[p * st2 + nch] = 0;
        }
    }
    if (t.lane == 0) {
#pragma unroll
        for (int p = 0; p < kMaxPlayers; ++p) s.misc[16 + p] = 0;
    }
#pragma unroll
    for (int p = 0; p < PT; ++p) {
        if (p < P) {
            const int tot = (int)t.reduce_add((unsigned)arm[p]);
            if (t.lane == 0) s.misc[16 + p] = tot;
        }
    }
    t.sync();
    return t.reduce_add(sat);
}

template <int LW>
__device__ __forceinline__ uint32_t cell_pass(const Game& g, const Smem& s, bool grow_s, bool grow_p, const Grp<LW>& t) {
    if constexpr (LW < 32) {  // groups narrower than a warp only run games of at most kPairMaxPlayers
        static_assert(kPairMaxPlayers == 2, "narrow groups compile the two-player cell pass only");
        return chunk_pass<2, LW>(g, s, grow_s, grow_p, t);
    } else {
        if (g.P <= 2) return chunk_pass<2, LW>(g, s, grow_s, grow_p, t);
        if (g.P <= 4) return chunk_pass<4, LW>(g, s, grow_s, grow_p, t);
        return chunk_pass<8, LW>(g, s, grow_s, grow_p, t);
    }
}

// ---- fog: 3x3 dilation of the (team) ownership bitset (Sec. IV-B) ----------
// Also counts each player's land for the scoreboard.
template <int LW>
__device__ void fog_pass(const Game& g, const Smem& s, uint32_t alive, const Grp<LW>& t) {
    const int N = g.N, W = g.W, nw = g.nw, st = s.stride;
    const int q = W >> 5, sh = W & 31;
    const bool team = g.mode == 1;
    for (int p = 0; p < g.P; ++p) {
        const uint32_t* own = s.own + p * st;
        const uint32_t* ally = s.own + (p ^ 1) * st;
        int land = 0;
        for (int w = t.lane; w < nw; w += LW) {
            const uint32_t mine = own[w];
            land += __popc(mine);
            const uint32_t T = mine | (team ? ally[w] : 0u);
            const uint32_t Tm = (w > 0) ? (own[w - 1] | (team ? ally[w - 1] : 0u)) : 0u;
            const uint32_t Tp = (w + 1 < nw) ? (own[w + 1] | (team ? ally[w + 1] : 0u)) : 0u;
            const uint32_t L = (T << 1) | (Tm >> 31);  // bit c <- cell c-1
            const uint32_t R = (T >> 1) | (Tp << 31);  // bit c <- cell c+1
            s.tmp[w] = (T | (L & ~s.col0[w]) | (R & ~s.colL[w])) & valid_bits(N, w);
        }
        land = (int)t.reduce_add((unsigned)land);
        if (t.lane == 0) s.misc[8 + p] = land;
        t.sync();
        const bool seeing = (alive >> p) & 1u;
        for (int w = t.lane; w < nw; w += LW) {
            const uint32_t h = s.tmp[w];
            // bit c <- cell c - W (row above) and cell c + W (row below)
            const int wa = w - q;
            uint32_t up = (wa >= 0 ? s.tmp[wa] << sh : 0u);
            if (sh && wa - 1 >= 0) up |= s.tmp[wa - 1] >> (32 - sh);
            const int wb = w + q;
            uint32_t dn = (wb < nw ? s.tmp[wb] >> sh : 0u);
            if (sh && wb + 1 < nw) dn |= s.tmp[wb + 1] << (32 - sh);
            s.vis[p * st + w] = seeing ? ((h | up | dn) & valid_bits(N, w)) : 0u;
        }
        t.sync();
    }
}

// 4 bits -> 4 bytes of 0x01
__device__ __forceinline__ uint32_t spread4(uint32_t nib) { return (nib * 0x00204081u) & 0x01010101u; }
// low nibbles of 4 bytes -> 16 bits (byte k's nibble at bits 4k..4k+3)
__device__ __forceinline__ uint32_t nibbles16(uint32_t x) {
    x &= 0x0F0F0F0Fu;
    const uint32_t y = (x | (x >> 4)) & 0x00FF00FFu;
    return (y | (y >> 8)) & 0xFFFFu;
}

// Legal moves of player p in chunk ch as 64 bits, 4 per cell in (cell,
// direction) order: the player owns the cell, it holds at least 2, and the
// neighbour towards the direction is passable.  The caller knows the player
// is alive and the game running.
__device__ __forceinline__ uint64_t chunk_legal64(const Smem& s, int p, int ch) {
    const int c0 = ch << 4;
    const int wi = c0 >> 5, sh = c0 & 16;
    const uint32_t mv = ((s.own[p * s.stride + wi] & s.big[wi]) >> sh) & 0xFFFFu;
    const uint4 T = *reinterpret_cast<const uint4*>(s.terrain + c0);
    const uint32_t tw[4] = {T.x, T.y, T.z, T.w};
    uint32_t nib[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) nib[k] = ((tw[k] >> 2) & 0x0F0F0F0Fu) & (spread4((mv >> (4 * k)) & 15u) * 0x0Fu);
    const uint32_t lo = nibbles16(nib[0]) | (nibbles16(nib[1]) << 16);
    const uint32_t hi = nibbles16(nib[2]) | (nibbles16(nib[3]) << 16);
    return ((uint64_t)hi << 32) | lo;
}

// ---- observation + mask chunks of 16 cells (Sec. IV-B, App. A, Sec. IV-G) --
// WRITE: store the planes; COUNT: legal (cell, direction) pairs per chunk.
template <bool WRITE, bool COUNT, int LW>
__device__ void output_pass(const KArgs& a, const Game& g, const Smem& s, uint32_t alive, bool finished, const Grp<LW>& t,
                            int64_t frame_off) {
    const int nch = g.nch, st = s.stride, P = g.P;
    int p = 0, ch = t.lane;
    while (p < P && ch >= nch) {
        ch -= nch;
        ++p;
    }
    while (p < P) {
        const int c0 = ch << 4;
        const int wi = c0 >> 5, sh = c0 & 16;
        uint32_t mv = 0;
        if (!finished && ((alive >> p) & 1u)) mv = ((s.own[p * st + wi] & s.big[wi]) >> sh) & 0xFFFFu;
        const uint4 T = *reinterpret_cast<const uint4*>(s.terrain + c0);
        const uint32_t tw[4] = {T.x, T.y, T.z, T.w};
        uint32_t om[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t dpb = ((tw[k] >> 2) & 0x0F0F0F0Fu) * 0x11u;
            om[k] = dpb & (spread4((mv >> (4 * k)) & 15u) * 0xFFu);
        }
        if (COUNT) {
            if (LW < 32) {
                // the chunk's legal moves as 64 bits: 4 per cell in (cell, direction) order
                const uint32_t lo = nibbles16(om[0]) | (nibbles16(om[1]) << 16);
                const uint32_t hi = nibbles16(om[2]) | (nibbles16(om[3]) << 16);
                s.legal[p * nch + ch] = ((uint64_t)hi << 32) | lo;
            } else {
                // legal (cell, direction) pairs of the chunk: the low nibble of each mask byte
                s.cnt[p * nch + ch] = (uint8_t)(__popc(om[0] & 0x0F0F0F0Fu) + __popc(om[1] & 0x0F0F0F0Fu) +
                                                __popc(om[2] & 0x0F0F0F0Fu) + __popc(om[3] & 0x0F0F0F0Fu));
            }
        }
        if (WRITE) {
            const uint32_t vis16 = (s.vis[p * st + wi] >> sh) & 0xFFFFu;
            const uint4 A0 = *reinterpret_cast<const uint4*>(s.army + c0);
            const uint4 A1 = *reinterpret_cast<const uint4*>(s.army + c0 + 8);
            const uint4 O = *reinterpret_cast<const uint4*>(s.owner + c0);
            const uint32_t aw[8] = {A0.x, A0.y, A0.z, A0.w, A1.x, A1.y, A1.z, A1.w};
            const uint32_t ow[4] = {O.x, O.y, O.z, O.w};
            uint32_t oa[8], oo[4], ot[4], ov[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t v1 = spread4((vis16 >> (4 * k)) & 15u);
                const uint32_t bm = v1 * 0xFFu;
                oo[k] = (ow[k] & bm) | (0xFEFEFEFEu & ~bm);
                const uint32_t tt = tw[k] & 0x03030303u;
                const uint32_t fogc = ((tt ^ (tt >> 1)) & 0x01010101u) | 0x04040404u;
                ot[k] = (tt & bm) | (fogc & ~bm);
                ov[k] = v1;
                oa[2 * k] = aw[2 * k] & __byte_perm(bm, 0, 0x1100);
                oa[2 * k + 1] = aw[2 * k + 1] & __byte_perm(bm, 0, 0x3322);
            }
            const int64_t off = frame_off + g.plane_off + (int64_t)p * g.Npad + c0;
            uint4* pa = reinterpret_cast<uint4*>(a.obs_army + off);
            __stcs(pa, make_uint4(oa[0], oa[1], oa[2], oa[3]));
            __stcs(pa + 1, make_uint4(oa[4], oa[5], oa[6], oa[7]));
            __stcs(reinterpret_cast<uint4*>(a.obs_owner + off), make_uint4(oo[0], oo[1], oo[2], oo[3]));
            __stcs(reinterpret_cast<uint4*>(a.obs_terrain + off), make_uint4(ot[0], ot[1], ot[2], ot[3]));
            __stcs(reinterpret_cast<uint4*>(a.obs_vis + off), make_uint4(ov[0], ov[1], ov[2], ov[3]));
            __stcs(reinterpret_cast<uint4*>(a.mask + off), make_uint4(om[0], om[1], om[2], om[3]));
        }
        ch += LW;
        while (p < P && ch >= nch) {
            ch -= nch;
            ++p;
        }
    }
    t.sync();
}

template <int LW>
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x, const Grp<LW>& t) {
#pragma unroll
    for (int o = 1; o < LW; o <<= 1) {
        const uint32_t y = t.shfl_up(x, o);
        if (t.lane >= o) x += y;
    }
    return x;
}

// ---- benchmark policy: uniform legal (cell, direction), split p = 0.2 -------
// Needs the chunk counts of output_pass<*, true>.  Players are scanned two at
// a time (16-bit counts packed in one 32-bit warp scan: a board has at most
// 4 x 4096 legal pairs); the lane holding pair j walks its chunks and selects
// the bit by popcount bisection.
// Returns, on lane p < P, player p's action; DIRECT also stores it.
template <bool DIRECT, int LW>
__device__ int32_t policy_pass(const KArgs& a, const Game& g, const Smem& s, uint32_t alive, bool finished,
                               uint32_t frame, uint64_t gid, const Grp<LW>& t) {
    int32_t mine_action = 0;
    const int nch = g.nch;
    constexpr bool masks = LW < 32;
    const int cpl = (nch + LW - 1) / LW;  // consecutive chunks per lane
    const int c_lo = t.lane * cpl;
    const int c_hi = min(c_lo + cpl, nch);
    // lane p hashes player p's two draws
    uint32_t u1 = 0, u2 = 0;
    if (t.lane < g.P) {
        const uint64_t K = hkey(a.policy_seed, gid, frame, (uint64_t)t.lane);
        u1 = hdraw(K, 0);
        u2 = hdraw(K, 1);
    }
    for (int p0 = 0; p0 < g.P; p0 += 2) {
        uint32_t mine = 0;
        for (int c = c_lo; c < c_hi; ++c) {
            if (masks) {
                mine += __popcll(s.legal[p0 * nch + c]);
                if (p0 + 1 < g.P) mine += (uint32_t)__popcll(s.legal[(p0 + 1) * nch + c]) << 16;
            } else {
                mine += s.cnt[p0 * nch + c];
                if (p0 + 1 < g.P) mine += (uint32_t)s.cnt[(p0 + 1) * nch + c] << 16;
            }
        }
        const uint32_t incl2 = warp_incl_scan(mine, t);
        const uint32_t total2 = t.shfl(incl2, LW - 1);
        for (int q = 0; q < 2 && p0 + q < g.P; ++q) {
            const int p = p0 + q;
            const uint32_t total = (total2 >> (16 * q)) & 0xFFFFu;
            const uint32_t incl = (incl2 >> (16 * q)) & 0xFFFFu;
            const uint32_t pu1 = t.shfl(u1, p);
            const uint32_t pu2 = t.shfl(u2, p);
            int32_t action = 0;
            if (total > 0 && !finished && ((alive >> p) & 1u)) {
                const uint32_t j = (uint32_t)uniform_below(pu1, total);
                const int L = __ffs(t.ballot(incl > j)) - 1;
                int32_t found = 0;
                if (t.lane == L) {
                    uint32_t jj = j - (incl - ((mine >> (16 * q)) & 0xFFFFu));
                    for (int c = c_lo; c < c_hi; ++c) {
                        const uint64_t mk = masks ? s.legal[p * nch + c] : 0ull;
                        const uint32_t n = masks ? (uint32_t)__popcll(mk) : (uint32_t)s.cnt[p * nch + c];
                        if (jj >= n) {
                            jj -= n;
                            continue;
                        }
                        const uint64_t m = masks ? mk : chunk_legal64(s, p, c);
                        uint32_t x = (uint32_t)m;
                        int bit = 0;
                        const uint32_t nlo = __popc(x);
                        if (jj >= nlo) {
                            jj -= nlo;
                            x = (uint32_t)(m >> 32);
                            bit = 32;
                        }
#pragma unroll
                        for (int w = 16; w >= 1; w >>= 1) {
                            const uint32_t cw = __popc(x & ((1u << w) - 1u));
                            if (jj >= cw) {
                                jj -= cw;
                                x >>= w;
                                bit += w;
                            }
                        }
                        const int d = bit & 3;
                        found = (c * 16 + (bit >> 2)) * 9 + ((pu2 < kSplitThresh) ? 5 + d : 1 + d);
                        break;
                    }
                }
                action = t.shfl(found, L);
            }
            if (DIRECT) {
                if (t.lane == 0) a.next_actions[g.player_off + p] = action;
            } else if (t.lane == p) {
                mine_action = action;
            }
        }
    }
    return mine_action;
}

// All of a board's 16-byte vectors (army, owner, terrain) copied global ->
// shared with cp.async: every copy is in flight at once and none passes
// through registers.  board_wait() completes them (a hardware wait).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
template <int LW>
__device__ __forceinline__ void board_issue(const KArgs& a, const Game& g, const Smem& s, const Grp<LW>& t) {
    const int n16 = g.Npad >> 4;  // 16-byte vectors per int8 plane
    const uint4* ga = reinterpret_cast<const uint4*>(a.army + g.cell_off);
    const uint4* go = reinterpret_cast<const uint4*>(a.owner + g.cell_off);
    const uint4* gt = reinterpret_cast<const uint4*>(a.terrain + g.cell_off);
    uint4* sa = reinterpret_cast<uint4*>(s.army);
    uint4* so = reinterpret_cast<uint4*>(s.owner);
    uint4* st = reinterpret_cast<uint4*>(s.terrain);
    for (int v = t.lane; v < 2 * n16; v += LW) cp_async16(sa + v, ga + v);
    for (int v = t.lane; v < n16; v += LW) {
        cp_async16(so + v, go + v);
        cp_async16(st + v, gt + v);
    }
    if (a.do_outputs) {
        // the board's first- and last-column bitsets for the fog pass, in
        // the same group of copies (8-byte pairs of words: both regions and
        // both table rows are 8-byte aligned, the region holds an even count)
        const uint32_t* c0 = g_columns[g.W - 1][0];
        const uint32_t* cl = g_columns[g.W - 1][1];
        for (int v = t.lane; 2 * v < g.nw; v += LW) {
            cp_async8(s.col0 + 2 * v, c0 + 2 * v);
            cp_async8(s.colL + 2 * v, cl + 2 * v);
        }
    }
}
template <int LW>
__device__ __forceinline__ void board_wait(const Grp<LW>& t) {
    asm volatile("cp.async.wait_all;" ::: "memory");
    t.sync();
}

template <int LW>
__device__ __forceinline__ void store_board(const KArgs& a, const Game& g, const Smem& s, const Grp<LW>& t) {
    const int n16 = g.Npad >> 4;
    uint4* ga = reinterpret_cast<uint4*>(a.army + g.cell_off);
    uint4* go = reinterpret_cast<uint4*>(a.owner + g.cell_off);
    uint4* gt = reinterpret_cast<uint4*>(a.terrain + g.cell_off);
    const uint4* sa = reinterpret_cast<const uint4*>(s.army);
    const uint4* so = reinterpret_cast<const uint4*>(s.owner);
    const uint4* st = reinterpret_cast<const uint4*>(s.terrain);
    for (int v = t.lane; v < 2 * n16; v += LW) ga[v] = sa[v];
    for (int v = t.lane; v < n16; v += LW) {
        go[v] = so[v];
        gt[v] = st[v];
    }
}

}  // namespace

namespace {


template <bool MULTI, bool SPAWN, int LW, bool UNI>
// geom: the packed carve geometry of the game's warp region, or 0 for the
// launch's own (kernel parameters); only the cold out-of-line paths use it.
__device__ __forceinline__ void run_game(const KArgs& a, const Smem& s, char* warp_base, const uint32_t geom,
                                         const int gidx, const Grp<LW>& t) {
    Game g = game_of<UNI>(a, gidx);
    if constexpr (LW < 32) {
        // narrow groups run only two-player games without teams: 1v1, or a
        // two-player free-for-all, whose rules are the same
        g.P = kPairMaxPlayers;
        g.mode = 0;
    }
    GameScalars* sc = a.scal + gidx;

    // every global load of the step is issued here, before any is used
    const bool board = a.op != OP_CREATE && a.op != OP_RESET;
    if (board) board_issue(a, g, s, t);
    uint4 s0 = make_uint4(0, 0, 0, 0), s1 = make_uint4(0, 0, 0, 0);
    if (a.op != OP_CREATE) {
        s0 = *reinterpret_cast<const uint4*>(sc);
        s1 = *(reinterpret_cast<const uint4*>(sc) + 1);
    }
    // player `lane`'s action for the next step (frame 0: from the caller)
    int32_t my_act = (a.op == OP_STEP && t.lane < g.P) ? a.actions[g.player_off + t.lane] : 0;
    if (board) board_wait(t);

    uint32_t turn = 0, frame = 0, epoch = 0, alive = 0, finished = 0, invalid = 0, saturated = 0, err = 0;
    if (a.op != OP_CREATE) {
        turn = s0.x;
        frame = s0.y;
        epoch = s0.z;
        alive = s0.w;
        finished = s1.x;
        invalid = s1.y;
        saturated = s1.z;
        err = s1.w;
    }
    const uint32_t all_alive = (1u << g.P) - 1u;
    bool wrote_state = false;

    if (a.op == OP_CREATE || a.op == OP_RESET) {
        if (a.op == OP_RESET) epoch += 1;
        if constexpr (SPAWN)
            generate_spawn(a, gidx, warp_base, geom ? geom : geom_of<LW>(a), game_id_of<UNI>(a, gidx), epoch, t.lane + t.shift);
        else
            generate<LW, UNI>(a, gidx, warp_base, geom ? geom : geom_of<LW>(a), game_id_of<UNI>(a, gidx), epoch, t.lane + t.shift);
        turn = 0;
        alive = all_alive;
        finished = 0;
        wrote_state = true;
    } else if (a.op == OP_DERIVE) {
        derive_passable_at<LW, UNI>(a, gidx, warp_base, geom ? geom : geom_of<LW>(a), t.lane + t.shift);
        wrote_state = true;
    }
    const int frames = (MULTI && a.op == OP_STEP) ? a.frames : 1;
    for (int f = 0; f < frames; ++f) {
        float my_reward = 0.0f;
        uint32_t done = 0;
        if (a.op == OP_STEP && !finished) {
            if (MULTI && a.action_log && t.lane < g.P)
                a.action_log[(int64_t)f * a.slot_stride + g.player_off + t.lane] = my_act;
            // moves in rotating priority, each checked when it runs (Q1)
            uint32_t eliminated = 0;
            uint32_t inv0 = 0, sat0 = 0;
            for (int k = 0; k < g.P; ++k) {
                const int p = (int)((turn + (uint32_t)k) % (uint32_t)g.P);
                const int32_t act = t.shfl(my_act, p);
                int cap = 0;
                if (t.lane == 0 && ((alive >> p) & 1u)) cap = resolve_move(g, s, p, act, alive, inv0, sat0);
                cap = t.shfl(cap, 0);
                alive = t.shfl(alive, 0);
                t.sync();
                if (cap) {
                    // land transfer: every other cell of the loser, army - army/2 (Q7)
                    const int dst = cap & 0xFFFF, q = (cap >> 16) - 1;
                    eliminated |= 1u << q;
                    for (int c = t.lane; c < g.N; c += LW) {
                        if (c != dst && s.owner[c] == q) {
                            s.owner[c] = (int8_t)p;
                            const int av = s.army[c];
                            s.army[c] = (int16_t)(av - (av >> 1));
                        }
                    }
                    t.sync();
                }
            }
            invalid += t.shfl(inv0, 0);
            saturated += t.shfl(sat0, 0);
            turn += 1;
            saturated += cell_pass(g, s, (turn % 2u) == 0u, (turn % 50u) == 0u, t);
            // termination and reward (Sec. III, IV-D, IV-E; Q17, Q21)
            if (g.mode == 1) {
                const bool dead0 = (alive & 0x3u) == 0u, dead1 = (alive & 0xCu) == 0u;
                if (dead0 || dead1) {
                    done = 1;
                    const bool mine_dead = ((t.lane >> 1) == 0) ? dead0 : dead1;
                    my_reward = mine_dead ? -1.0f : 1.0f;
                }
            } else {
                if ((eliminated >> t.lane) & 1u) my_reward = -1.0f;
                if (__popc(alive) <= 1) {
                    done = 1;
                    if ((alive >> t.lane) & 1u) my_reward = 1.0f;
                }
            }
            if (!done && a.max_turns > 0 && turn >= (uint32_t)a.max_turns) done = 2;
            if (done) {
                if (a.auto_reset) {
                    epoch += 1;
                    if constexpr (SPAWN)
                        generate_spawn(a, gidx, warp_base, geom ? geom : geom_of<LW>(a), game_id_of<UNI>(a, gidx), epoch, t.lane + t.shift);
                    else
                        generate<LW, UNI>(a, gidx, warp_base, geom ? geom : geom_of<LW>(a), game_id_of<UNI>(a, gidx), epoch, t.lane + t.shift);
                    turn = 0;
                    alive = all_alive;
                    cell_pass(g, s, false, false, t);
                } else {
                    finished = 1;
                }
            }
            wrote_state = true;
        } else {
            // create, reset, observe, policy, or a frozen game
            saturated += cell_pass(g, s, false, false, t);
        }
        if (a.op == OP_STEP) frame += 1;

        const bool fin = finished != 0;
        if constexpr (MULTI) {
            // reward and done before the output passes and the scoreboard
            // as soon as the fog pass has counted the land: fewer values
            // live through the passes (measured faster in multi-frame
            // launches, slower per frame)
            if (a.do_outputs) {
                const int64_t soff = (int64_t)f * a.slot_stride;
                if (t.lane < g.P) a.reward[soff + g.player_off + t.lane] = my_reward;
                if (t.lane == 0) a.done[(int64_t)f * a.game_stride + gidx] = (uint8_t)done;
            }
        }
        if (a.do_outputs) {
            const int64_t poff = (int64_t)f * a.plane_stride;
            const int64_t soff = (int64_t)f * a.slot_stride;
            if (!board) column_pass(g, s, t);  // else copied with the board
            fog_pass(g, s, alive, t);  // counts the land
            if constexpr (MULTI) {
                if (t.lane < g.P) {
                    a.scoreboard[2 * (soff + g.player_off + t.lane) + 0] = s.misc[8 + t.lane];
                    a.scoreboard[2 * (soff + g.player_off + t.lane) + 1] = s.misc[16 + t.lane];
                }
            }
            if (a.next_actions)
                output_pass<true, true, LW>(a, g, s, alive, fin, t, poff);
            else
                output_pass<true, false, LW>(a, g, s, alive, fin, t, poff);
            if constexpr (!MULTI) {
                if (t.lane < g.P) {
                    a.reward[soff + g.player_off + t.lane] = my_reward;
                    a.scoreboard[2 * (soff + g.player_off + t.lane) + 0] = s.misc[8 + t.lane];
                    a.scoreboard[2 * (soff + g.player_off + t.lane) + 1] = s.misc[16 + t.lane];
                }
                if (t.lane == 0) a.done[(int64_t)f * a.game_stride + gidx] = (uint8_t)done;
            }
        } else if (a.next_actions) {
            output_pass<false, true, LW>(a, g, s, alive, fin, t, 0);
        }
        if (a.next_actions) my_act = policy_pass<!MULTI, LW>(a, g, s, alive, fin, frame, game_id_of<UNI>(a, gidx), t);
    }
    if (MULTI && a.next_actions && t.lane < g.P) a.next_actions[g.player_off + t.lane] = my_act;
    if (wrote_state) {
        t.sync();
        store_board(a, g, s, t);
    }
    if (t.lane == 0 && a.op != OP_OBSERVE && a.op != OP_POLICY) {
        uint4* dst = reinterpret_cast<uint4*>(sc);
        dst[0] = make_uint4(turn, frame, epoch, alive);
        dst[1] = make_uint4(finished, invalid, saturated, a.op == OP_CREATE ? 0u : err);
    }
}


}  // namespace

// One game per group of LW lanes (32: a warp; 16 or 8: two or four games per
// warp); groups walk the item list with a grid stride.  MULTI: several frames
// per launch (rollouts) with the board kept in shared memory.  SPAWN: the map
// generator with spawn options (LW = 32 only).  UNI: every game of the launch
// has the launch's shape (uniform batches).
// Register budget: 64 per thread (4 CTAs of 8 warps per SM) for the per-frame
// form; the multi-frame form keeps more state live across frames and runs
// best with 85 (3 CTAs).
template <bool MULTI, bool SPAWN, int LW, bool UNI>
__global__ void __launch_bounds__(256, MULTI ? 3 : 4) k_generals(const KArgs a) {
    chain_entry();
    extern __shared__ __align__(16) char smem_raw[];
    constexpr int kGroups = 32 / LW;  // games per warp
    const int wl = threadIdx.x & 31;
    const Grp<LW> t(wl);
    const int grp = (threadIdx.x >> 5) * kGroups + wl / LW;  // group in the CTA
    const int gpc = (blockDim.x >> 5) * kGroups;                                // groups per CTA
    char* warp_base = smem_raw + grp * a.warp_smem;
    const Smem s = carve<LW>(warp_base, a);
    if constexpr (!MULTI) {  // the grid covers every item
        const int item = blockIdx.x * gpc + grp;
        if (item >= a.n_items) return;
        const int gidx = a.list ? a.list[item] : item;
        if (gidx < 0 || gidx >= a.n_games) return;
        run_game<MULTI, SPAWN, LW, UNI>(a, s, warp_base, 0u, gidx, t);
    } else {
        for (int item = blockIdx.x * gpc + grp; item < a.n_items; item += gridDim.x * gpc) {
            const int gidx = a.list ? a.list[item] : item;
            if (gidx < 0 || gidx >= a.n_games) continue;
            t.sync();
            run_game<MULTI, SPAWN, LW, UNI>(a, s, warp_base, 0u, gidx, t);
        }
    }
}

// Every size bucket of a ragged or mixed batch in one persistent launch.  A
// CTA takes one work item at a time (an atomic counter over a list ordered
// largest boards first), carves its shared memory for that item's bucket and
// runs one game per lane group: two per warp for two-player buckets of small
// boards, one per warp otherwise.  The CTA waits at a barrier between items,
// so that the next item may carve the same bytes differently.
template <bool MULTI>
__global__ void __launch_bounds__(256, MULTI ? 3 : 4) k_worklist(const KArgs a, const WArgs w) {
    chain_entry();
    extern __shared__ __align__(16) char smem_raw[];
    __shared__ int s_item;
    const int warp = threadIdx.x >> 5, wl = threadIdx.x & 31;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(w.counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= w.n_items) {  // the same for every thread of the CTA
            // the last CTA to run out zeroes the counters for the next launch:
            // every CTA has drawn its last index by then, and a chained launch
            // reads them only after this grid has completed
            if (threadIdx.x == 0) {
                __threadfence();  // this CTA's last draw is ordered before its exit count
                if (atomicAdd(w.counter + 1, 1) == (int)gridDim.x - 1) {
                    __threadfence();  // and every other CTA's before these stores
                    w.counter[0] = 0;
                    w.counter[1] = 0;
                }
            }
            return;
        }
        const WorkItem item = w.items[it];
        const BucketGeom bg = w.geoms[item.bucket];
        if (bg.lw == 16) {
            const Grp<16> t(wl);
            const int grp = 2 * warp + (wl >> 4);
            if (grp < item.count) {
                char* base = smem_raw + grp * bg.group_smem;
                run_game<MULTI, false, 16, false>(a, carve_geom(base, bg.geom), base, bg.geom,
                                                  w.order[item.first + grp], t);
            }
        } else {
            const Grp<32> t(wl);
            if (warp < item.count) {
                char* base = smem_raw + warp * bg.group_smem;
                run_game<MULTI, false, 32, false>(a, carve_geom(base, bg.geom), base, bg.geom,
                                                  w.order[item.first + warp], t);
            }
        }
        __syncthreads();
    }
}

__global__ void k_columns() {
    const int W = blockIdx.x + 1;
    for (int w = threadIdx.x; w < kColWords; w += blockDim.x) {
        uint32_t c0 = 0, cl = 0;
        for (int b = 0; b < 32; ++b) {
            const int c = 32 * w + b;
            if (c % W == 0) c0 |= 1u << b;
            if (c % W == W - 1) cl |= 1u << b;
        }
        g_columns[W - 1][0][w] = c0;
        g_columns[W - 1][1][w] = cl;
    }
}

__global__ void k_copy(const uint4* __restrict__ src, uint4* __restrict__ dst, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (; i < n; i += stride) __stcs(dst + i, __ldcs(src + i));
}

// Every step-kernel instantiation may take up to the per-CTA maximum of
// dynamic shared memory on the current device: set once per device, so no
// launch shape needs its own opt-in (the limit gates launches only).
int allow_max_smem() {
    static SmemLimit limit;
    const void* fns[14] = {
        (const void*)k_generals<false, false, 32, false>, (const void*)k_generals<true, false, 32, false>,
        (const void*)k_generals<false, false, 32, true>,  (const void*)k_generals<true, false, 32, true>,
        (const void*)k_generals<false, false, 16, false>, (const void*)k_generals<true, false, 16, false>,
        (const void*)k_generals<false, false, 16, true>,  (const void*)k_generals<true, false, 16, true>,
        (const void*)k_generals<false, false, 8, false>,  (const void*)k_generals<true, false, 8, false>,
        (const void*)k_generals<false, false, 8, true>,   (const void*)k_generals<true, false, 8, true>,
        (const void*)k_generals<false, true, 32, false>,  (const void*)k_generals<true, true, 32, false>};
    return limit.raise(fns, 14, 227 * 1024);
}

uint32_t bucket_geom(int npad_max, int nw_stride, int pmax, bool narrow) {
    return pack_geom(npad_max, nw_stride, pmax, narrow);
}

int worklist_shape(bool multi, int* cta_smem, int* ctas) {
    // four CTAs of 8 warps per SM per frame (the register budget's limit),
    // three in multi-frame launches; each takes an equal share of the SM's
    // shared memory less the per-CTA reservation
    const void* f = multi ? (const void*)k_worklist<true> : (const void*)k_worklist<false>;
    int dev = 0, sms = 0, smem_sm = 0, reserved = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return (int)e;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    const int want = multi ? 3 : 4;
    int bytes = ((smem_sm / want - reserved - 64) / 16) * 16;  // 64: the kernel's static item slot
    if (bytes > 227 * 1024) bytes = 227 * 1024;
    // the kernel's own static slot counts against the per-CTA limit too
    if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess)
        return (int)e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, 256, (size_t)bytes)) != cudaSuccess)
        return (int)e;
    if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
    *cta_smem = bytes;
    *ctas = per_sm * sms;
    return 0;
}

int launch_worklist(const KArgs& a, const WArgs& w, int cta_smem, int ctas, void* stream) {
    const cudaStream_t st = (cudaStream_t)stream;  // the counters arrive zeroed (see k_worklist)
    const bool multi = a.frames > 1 || a.action_log;
    const int grid = ctas < w.n_items ? ctas : w.n_items;
    if (grid <= 0) return 0;
    if (multi) return launch_chained(k_worklist<true>, dim3(grid), dim3(256), cta_smem, st, a, w);
    return launch_chained(k_worklist<false>, dim3(grid), dim3(256), cta_smem, st, a, w);
}

int warp_smem_bytes(int npad_max, int pmax, int* nw_stride, bool narrow) {
    int nw = (npad_max + 31) / 32;
    nw = (nw + 1) & ~1;  // even: the carve stays a multiple of 16 bytes
    if (nw_stride) *nw_stride = nw;
    return 4 * npad_max + 4 * nw * (2 * pmax + 4) + legal_region_bytes(npad_max, pmax, narrow) + 4 * 24;
}

int max_resident_ctas(int warps_per_cta, int smem_bytes, int* out) {
    cudaError_t e = (cudaError_t)allow_max_smem();
    if (e != cudaSuccess) return (int)e;
    int per_sm = 0, dev = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_generals<false, false, 32, false>, 32 * warps_per_cta,
                                                           smem_bytes)) != cudaSuccess)
        return (int)e;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    *out = per_sm * sms;
    return 0;
}

int init_tables() {
    static std::mutex mu;
    static bool ready[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (int)e;
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 64 && ready[dev]) return 0;
    k_columns<<<kMaxSide, 128>>>();
    if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return (int)e;
    if (dev >= 0 && dev < 64) ready[dev] = true;
    return 0;
}

// Resident CTAs of kernel f per SM for a launch shape, from the occupancy
// calculator; cached per (kernel, threads, bytes) for the process.
int ctas_per_sm(const void* f, int threads, int smem) {
    static std::mutex mu;
    static std::map<std::tuple<const void*, int, int, int>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(f, threads, smem, dev);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, threads, (size_t)smem) != cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = n;
    return n;
}

// Launch shape of one step launch: warps per CTA.  `fixed` > 0 is the
// caller's choice (gen_set_launch, the autotuner); otherwise the count among
// 8, 4, 2, 1 whose CTAs keep the most warps resident per SM (ties: more warps
// per CTA).  Either way, launches too small to give every SM a CTA take
// fewer warps per CTA.
int pick_warps(const void* f, int fixed, int games_per_warp, int warp_smem, int n_items, int sms) {
    int w = fixed;
    if (w <= 0) {
        int best = 0;
        w = 1;
        for (int cand : {8, 4, 2, 1}) {
            const int smem = cand * games_per_warp * warp_smem;
            if (smem > 227 * 1024) continue;
            const int warps = ctas_per_sm(f, 32 * cand, smem) * cand;
            if (warps > best) {
                best = warps;
                w = cand;
            }
        }
    }
    while (w > 1 && (n_items + games_per_warp * w - 1) / (games_per_warp * w) < sms) w >>= 1;
    return w;
}

// The plain-generator kernels of one lane-group width: per frame or
// multi-frame, for uniform or per-game shapes.
template <int LW>
const void* plain_kernel(bool multi, bool uniform) {
    if (multi && uniform) return (const void*)k_generals<true, false, LW, true>;
    if (multi) return (const void*)k_generals<true, false, LW, false>;
    if (uniform) return (const void*)k_generals<false, false, LW, true>;
    return (const void*)k_generals<false, false, LW, false>;
}

template <int LW>
int launch_plain(const KArgs& a, bool multi, int fixed_warps, int max_ctas, int sms, cudaStream_t st) {
    constexpr int kPerWarp = 32 / LW;
    const void* f = plain_kernel<LW>(multi, a.uniform != 0);
    const int warps = pick_warps(f, fixed_warps, kPerWarp, a.warp_smem, a.n_items, sms);
    const int games_per_cta = kPerWarp * warps;
    const int smem = a.warp_smem * games_per_cta;
    int blocks = (a.n_items + games_per_cta - 1) / games_per_cta;
    // multi-frame launches: a grid of many waves, groups stride over any items beyond it
    if (multi && max_ctas > 0 && blocks > 64 * max_ctas) blocks = 64 * max_ctas;
    const dim3 grid(blocks), block(32 * warps);
    if (multi && a.uniform) return launch_chained(k_generals<true, false, LW, true>, grid, block, smem, st, a);
    if (multi) return launch_chained(k_generals<true, false, LW, false>, grid, block, smem, st, a);
    if (a.uniform) return launch_chained(k_generals<false, false, LW, true>, grid, block, smem, st, a);
    return launch_chained(k_generals<false, false, LW, false>, grid, block, smem, st, a);
}

int launch_step(const KArgs& a, int warps_per_cta, int max_ctas, void* stream) {
    if (a.n_items <= 0) return 0;

    const bool spawn = a.spawn_dmax > 0 || a.spawn_bfs || a.castle_radius > 0;
    const bool multi = a.frames > 1 || a.action_log;
    const cudaStream_t st = (cudaStream_t)stream;
    {
        const int e = allow_max_smem();
        if (e != 0) return e;
    }
    static std::atomic<int> sm_count{0};  // of the first device used: only the launch shape depends on it
    int sms = sm_count.load(std::memory_order_relaxed);
    if (sms == 0) {
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        sms = n > 0 ? n : 1;
        sm_count.store(sms, std::memory_order_relaxed);
    }
    // several games per warp for small two-player boards, plain generator
    // only, once the batch is large enough: below it a warp per game is
    // faster (measured on 24x24 1v1: 1,024 games per frame 98 against 87 M
    // frames/s, resident 194 against 122 M; pairs win from 2,048 games per
    // frame and 4,096 resident)
    const bool large = a.n_items >= (multi ? 24 : 12) * sms;
    const bool small = !spawn && a.pmax <= kPairMaxPlayers && (a.lane_groups == 2 || (a.lane_groups == 0 && large));
    const int wcap = warps_per_cta > 0 ? warps_per_cta : 1;  // the fixed shape must fit too
    // narrow groups keep their legal moves as chunk masks: a larger carve
    const int ws_narrow = small ? warp_smem_bytes(a.npad_max, a.pmax, nullptr, true) : a.warp_smem;
    int per_warp = 1;
    if (small && multi && a.npad_max <= kQuadMaxCells && 4 * wcap * ws_narrow <= 227 * 1024)
        per_warp = 4;
    else if (small && a.npad_max <= kPairMaxCells && 2 * wcap * ws_narrow <= 227 * 1024)
        per_warp = 2;
    if (per_warp > 1) {
        KArgs n = a;
        n.warp_smem = ws_narrow;
        return per_warp == 4 ? launch_plain<8>(n, multi, warps_per_cta, max_ctas, sms, st)
                             : launch_plain<16>(n, multi, warps_per_cta, max_ctas, sms, st);
    }
    if (spawn) {  // one game per warp, shapes read per game
        const void* f = multi ? (const void*)k_generals<true, true, 32, false> : (const void*)k_generals<false, true, 32, false>;
        const int warps = pick_warps(f, warps_per_cta, 1, a.warp_smem, a.n_items, sms);
        const int smem = a.warp_smem * warps;
        int blocks = (a.n_items + warps - 1) / warps;
        if (multi && max_ctas > 0 && blocks > 64 * max_ctas) blocks = 64 * max_ctas;
        if (multi) return launch_chained(k_generals<true, true, 32, false>, dim3(blocks), dim3(32 * warps), smem, st, a);
        return launch_chained(k_generals<false, true, 32, false>, dim3(blocks), dim3(32 * warps), smem, st, a);
    }
    return launch_plain<32>(a, multi, warps_per_cta, max_ctas, sms, st);
}

int launch_copy(const void* src, void* dst, size_t n16, int blocks, void* stream) {
    k_copy<<<blocks, 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<const uint4*>(src),
                                                      reinterpret_cast<uint4*>(dst), n16);
    return (int)cudaGetLastError();
}

}  // namespace gk
