// Device code of libgenerals: one warp advances one Generals.io game.
//
// Per game and step (paper Section IV): the warp stages the board (int16
// armies, int8 owners, int8 terrain) in shared memory, lane 0 resolves the
// players' moves one after another (Sec. IV-D/IV-E), the warp applies
// growth (Sec. IV-C) while it turns the board into 32-cell bitsets with
// __ballot_sync (ownership per player, army >= 2, passable neighbour per
// direction, edge columns), decides termination and reward (Sec. III),
// regenerates finished games (Sec. IV-A), dilates ownership bitsets into
// fog-of-war visibility with word shifts (Sec. IV-B), and expands bitsets
// and board bytes into 16-cell observation and mask chunks written with
// 128-bit streaming stores.  Optionally the benchmark policy picks the next
// actions from the same bitsets (popc counts, a warp scan, a bit walk).
//
// No floating point decides anything: all game arithmetic is integer.
#include <cuda_runtime.h>

#include "gk_internal.h"

namespace gk {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
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

// ---- per-warp shared-memory view --------------------------------------------
struct Smem {
    int16_t* army;
    int8_t* owner;
    int8_t* terrain;
    uint32_t* own;   // [pmax][stride]
    uint32_t* big;   // army >= 2
    uint32_t* dp;    // [4][stride]: neighbour in direction d exists and is not a mountain
    uint32_t* col0;  // first column
    uint32_t* colL;  // last column
    uint32_t* vis;   // [pmax][stride]
    uint32_t* tmp;
    int32_t* misc;   // [0..7] general cells, [8..15] land, [16..23] army
    int stride;
};

__device__ __forceinline__ Smem carve(char* base, const KArgs& a) {
    Smem s;
    const int np = a.npad_max, st = a.nw_stride, pm = a.pmax;
    s.army = reinterpret_cast<int16_t*>(base);
    s.owner = reinterpret_cast<int8_t*>(base + 2 * np);
    s.terrain = reinterpret_cast<int8_t*>(base + 3 * np);
    uint32_t* w = reinterpret_cast<uint32_t*>(base + 4 * np);
    s.own = w;
    w += pm * st;
    s.big = w;
    w += st;
    s.dp = w;
    w += 4 * st;
    s.col0 = w;
    w += st;
    s.colL = w;
    w += st;
    s.vis = w;
    w += pm * st;
    s.tmp = w;
    w += st;
    s.misc = reinterpret_cast<int32_t*>(w);
    s.stride = st;
    return s;
}

struct Game {
    int H, W, N, Npad, P, mode, nw;
    int64_t plane_off;
    int cell_off, player_off, n_cities, dmin;
};

__device__ __forceinline__ Game load_game(const GameInfo* gi) {
    Game g;
    g.H = gi->H;
    g.W = gi->W;
    g.N = gi->N;
    g.Npad = gi->Npad;
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

__device__ __forceinline__ uint32_t valid_bits(int N, int w) {
    int rem = N - 32 * w;
    if (rem >= 32) return kFull;
    if (rem <= 0) return 0u;
    return (1u << rem) - 1u;
}

// ---- map generator (Sec. IV-A) ----------------------------------------------
__device__ void generate(const KArgs& a, const Game& g, const Smem& s, uint64_t gid, uint32_t epoch, int lane) {
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
    uint32_t i = 0;
    int D = g.dmin;
    int my_gpos = -1;  // lane p holds player p's general
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
                        if (abs(rc - rq) + abs(cc - cq) < D) ok = false;
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
    if (lane < P) {
        s.terrain[my_gpos] = kGeneral;
        s.owner[my_gpos] = (int8_t)lane;
        s.army[my_gpos] = 1;
        s.misc[lane] = my_gpos;
    }
    __syncwarp();

    // connectivity: L-path rows first, then columns, between consecutive generals
    if (lane == 0) {
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
}

// ---- one move on lane 0 (Sec. IV-D, IV-E) ----------------------------------
// Returns the captured general's cell in the low 16 bits and the loser in
// bits 16..19 (+1), or 0 when no general fell.
__device__ int resolve_move(const Game& g, const Smem& s, int p, int32_t act, uint32_t& alive, uint32_t& invalid,
                            uint32_t& sat) {
    const int N = g.N, W = g.W, H = g.H;
    if (act < 0 || act >= 9 * N) {
        invalid += 1;
        return 0;
    }
    const int c = act / 9, k = act - 9 * c;
    if (k == 0) return 0;
    const int d = (k - 1) & 3;
    const bool half = k >= 5;
    int r = c / W, col = c - r * W;
    if (d == 0) r -= 1;
    if (d == 1) r += 1;
    if (d == 2) col -= 1;
    if (d == 3) col += 1;
    const int av = s.army[c];
    if (s.owner[c] != p || av < 2 || r < 0 || r >= H || col < 0 || col >= W) {
        invalid += 1;
        return 0;
    }
    const int dst = r * W + col;
    if (s.terrain[dst] == kMountain) {
        invalid += 1;
        return 0;
    }
    const int moved = half ? (av >> 1) : (av - 1);
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
        if (o != p && s.terrain[dst] != kGeneral) s.owner[dst] = (int8_t)p;
        return 0;
    }
    if (moved > def) {
        s.owner[dst] = (int8_t)p;
        s.army[dst] = (int16_t)(moved - def);
        if (s.terrain[dst] == kGeneral && o >= 0) {
            s.terrain[dst] = kCastle;
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

// ---- growth + bitsets + scoreboard (one cell per lane per word) ------------
__device__ uint32_t cell_pass(const Game& g, const Smem& s, bool grow_s, bool grow_p, int lane) {
    const int N = g.N, W = g.W, H = g.H, P = g.P, nw = g.nw;
    const int q32 = 32 / W, r32 = 32 - q32 * W;
    int r = lane / W, col = lane - (lane / W) * W;
    uint32_t sat = 0;
    int land[kMaxPlayers], arm[kMaxPlayers];
#pragma unroll
    for (int p = 0; p < kMaxPlayers; ++p) land[p] = arm[p] = 0;
    for (int w = 0; w < nw; ++w) {
        const int c = 32 * w + lane;
        const bool valid = c < N;
        int t = kMountain, o = -1, av = 0;
        if (valid) {
            t = s.terrain[c];
            o = s.owner[c];
            av = s.army[c];
            if (o >= 0 && ((grow_s && (t == kGeneral || t == kCastle)) || (grow_p && t == kPlain))) {
                av += 1;
                if (av > kArmyMax) {
                    av = kArmyMax;
                    sat += 1;
                }
                s.army[c] = (int16_t)av;
            }
        }
        const bool up = valid && r > 0 && s.terrain[c - W] != kMountain;
        const bool dn = valid && r < H - 1 && s.terrain[c + W] != kMountain;
        const bool lf = valid && col > 0 && s.terrain[c - 1] != kMountain;
        const bool rt = valid && col < W - 1 && s.terrain[c + 1] != kMountain;
        const unsigned b_big = __ballot_sync(kFull, valid && av >= 2);
        const unsigned b_up = __ballot_sync(kFull, up);
        const unsigned b_dn = __ballot_sync(kFull, dn);
        const unsigned b_lf = __ballot_sync(kFull, lf);
        const unsigned b_rt = __ballot_sync(kFull, rt);
        const unsigned b_c0 = __ballot_sync(kFull, valid && col == 0);
        const unsigned b_cl = __ballot_sync(kFull, valid && col == W - 1);
        if (lane == 0) {
            s.big[w] = b_big;
            s.dp[0 * s.stride + w] = b_up;
            s.dp[1 * s.stride + w] = b_dn;
            s.dp[2 * s.stride + w] = b_lf;
            s.dp[3 * s.stride + w] = b_rt;
            s.col0[w] = b_c0;
            s.colL[w] = b_cl;
        }
#pragma unroll
        for (int p = 0; p < kMaxPlayers; ++p) {
            if (p < P) {
                const unsigned b_own = __ballot_sync(kFull, o == p);
                if (lane == 0) s.own[p * s.stride + w] = b_own;
                land[p] += __popc(b_own);
                arm[p] += __reduce_add_sync(kFull, (unsigned)(o == p ? av : 0));
            }
        }
        col += r32;
        r += q32;
        if (col >= W) {
            col -= W;
            r += 1;
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int p = 0; p < kMaxPlayers; ++p) {
            s.misc[8 + p] = land[p];
            s.misc[16 + p] = arm[p];
        }
    }
    __syncwarp();
    return __reduce_add_sync(kFull, sat);
}

// ---- fog: 3x3 dilation of the (team) ownership bitset (Sec. IV-B) ----------
__device__ void fog_pass(const Game& g, const Smem& s, uint32_t alive, int lane) {
    const int N = g.N, W = g.W, nw = g.nw, st = s.stride;
    const int q = W >> 5, sh = W & 31;
    for (int p = 0; p < g.P; ++p) {
        const bool team = g.mode == 1;
        const uint32_t* own = s.own + p * st;
        const uint32_t* ally = s.own + (p ^ 1) * st;
        for (int w = lane; w < nw; w += 32) {
            uint32_t T = own[w] | (team ? ally[w] : 0u);
            uint32_t Tm = (w > 0) ? (own[w - 1] | (team ? ally[w - 1] : 0u)) : 0u;
            uint32_t Tp = (w + 1 < nw) ? (own[w + 1] | (team ? ally[w + 1] : 0u)) : 0u;
            uint32_t L = (T << 1) | (Tm >> 31);  // bit c <- cell c-1
            uint32_t R = (T >> 1) | (Tp << 31);  // bit c <- cell c+1
            s.tmp[w] = (T | (L & ~s.col0[w]) | (R & ~s.colL[w])) & valid_bits(N, w);
        }
        __syncwarp();
        const bool seeing = (alive >> p) & 1u;
        for (int w = lane; w < nw; w += 32) {
            const uint32_t h = s.tmp[w];
            // bit c <- cell c - W (row above) and cell c + W (row below)
            int wa = w - q;
            uint32_t up = (wa >= 0 ? s.tmp[wa] << sh : 0u);
            if (sh && wa - 1 >= 0) up |= s.tmp[wa - 1] >> (32 - sh);
            int wb = w + q;
            uint32_t dn = (wb < nw ? s.tmp[wb] >> sh : 0u);
            if (sh && wb + 1 < nw) dn |= s.tmp[wb + 1] << (32 - sh);
            s.vis[p * st + w] = seeing ? ((h | up | dn) & valid_bits(N, w)) : 0u;
        }
        __syncwarp();
    }
}

// 4 bits -> 4 bytes of 0x01
__device__ __forceinline__ uint32_t spread4(uint32_t nib) { return (nib * 0x00204081u) & 0x01010101u; }

// ---- observation + mask chunks of 16 cells (Sec. IV-B, App. A, Sec. IV-G) --
__device__ void output_pass(const KArgs& a, const Game& g, const Smem& s, uint32_t alive, bool finished, int lane) {
    const int nch = g.Npad >> 4, st = s.stride;
    const int items = g.P * nch;
    for (int it = lane; it < items; it += 32) {
        const int p = it / nch;
        const int c0 = (it - p * nch) << 4;
        const int wi = c0 >> 5, sh = c0 & 16;
        const uint32_t vis16 = (s.vis[p * st + wi] >> sh) & 0xFFFFu;
        uint32_t mv = 0;
        if (!finished && ((alive >> p) & 1u)) mv = ((s.own[p * st + wi] & s.big[wi]) >> sh) & 0xFFFFu;
        const uint32_t mU = mv & (s.dp[0 * st + wi] >> sh);
        const uint32_t mD = mv & (s.dp[1 * st + wi] >> sh);
        const uint32_t mL = mv & (s.dp[2 * st + wi] >> sh);
        const uint32_t mR = mv & (s.dp[3 * st + wi] >> sh);
        const uint4 A0 = *reinterpret_cast<const uint4*>(s.army + c0);
        const uint4 A1 = *reinterpret_cast<const uint4*>(s.army + c0 + 8);
        const uint4 O = *reinterpret_cast<const uint4*>(s.owner + c0);
        const uint4 T = *reinterpret_cast<const uint4*>(s.terrain + c0);
        const uint32_t aw[8] = {A0.x, A0.y, A0.z, A0.w, A1.x, A1.y, A1.z, A1.w};
        const uint32_t ow[4] = {O.x, O.y, O.z, O.w};
        const uint32_t tw[4] = {T.x, T.y, T.z, T.w};
        uint32_t oa[8], oo[4], ot[4], ov[4], om[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t v1 = spread4((vis16 >> (4 * k)) & 15u);
            const uint32_t bm = v1 * 0xFFu;
            oo[k] = (ow[k] & bm) | (0xFEFEFEFEu & ~bm);
            const uint32_t fogc = ((tw[k] ^ (tw[k] >> 1)) & 0x01010101u) | 0x04040404u;
            ot[k] = (tw[k] & bm) | (fogc & ~bm);
            ov[k] = v1;
            oa[2 * k] = aw[2 * k] & __byte_perm(bm, 0, 0x1100);
            oa[2 * k + 1] = aw[2 * k + 1] & __byte_perm(bm, 0, 0x3322);
            const uint32_t m = spread4((mU >> (4 * k)) & 15u) | (spread4((mD >> (4 * k)) & 15u) << 1) |
                               (spread4((mL >> (4 * k)) & 15u) << 2) | (spread4((mR >> (4 * k)) & 15u) << 3);
            om[k] = m * 0x11u;
        }
        const int64_t off = g.plane_off + (int64_t)p * g.Npad + c0;
        uint4* pa = reinterpret_cast<uint4*>(a.obs_army + off);
        __stcs(pa, make_uint4(oa[0], oa[1], oa[2], oa[3]));
        __stcs(pa + 1, make_uint4(oa[4], oa[5], oa[6], oa[7]));
        __stcs(reinterpret_cast<uint4*>(a.obs_owner + off), make_uint4(oo[0], oo[1], oo[2], oo[3]));
        __stcs(reinterpret_cast<uint4*>(a.obs_terrain + off), make_uint4(ot[0], ot[1], ot[2], ot[3]));
        __stcs(reinterpret_cast<uint4*>(a.obs_vis + off), make_uint4(ov[0], ov[1], ov[2], ov[3]));
        __stcs(reinterpret_cast<uint4*>(a.mask + off), make_uint4(om[0], om[1], om[2], om[3]));
    }
}

// ---- benchmark policy: uniform legal (cell, direction), split p = 0.2 -------
__device__ void policy_pass(const KArgs& a, const Game& g, const Smem& s, uint32_t alive, bool finished,
                            uint32_t frame, uint64_t gid, int lane) {
    const int nw = g.nw, st = s.stride;
    const int wpl = (nw + 31) >> 5;
    const int w0 = lane * wpl;
    for (int p = 0; p < g.P; ++p) {
        const bool on = !finished && ((alive >> p) & 1u);
        uint32_t cnt = 0;
        if (on) {
            for (int w = w0; w < w0 + wpl && w < nw; ++w) {
                const uint32_t mv = s.own[p * st + w] & s.big[w];
                cnt += __popc(mv & s.dp[w]) + __popc(mv & s.dp[st + w]) + __popc(mv & s.dp[2 * st + w]) +
                       __popc(mv & s.dp[3 * st + w]);
            }
        }
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t total = __shfl_sync(kFull, incl, 31);
        int32_t action = 0;
        if (total > 0) {
            const uint64_t K = hkey(a.policy_seed, gid, frame, (uint64_t)p);
            const uint32_t j = (uint32_t)uniform_below(hdraw(K, 0), total);
            const bool split = hdraw(K, 1) < kSplitThresh;
            const unsigned b = __ballot_sync(kFull, incl > j);
            const int L = __ffs(b) - 1;
            int32_t found = 0;
            if (lane == L) {
                uint32_t jj = j - (incl - cnt);
                for (int w = w0; w < w0 + wpl && w < nw; ++w) {
                    const uint32_t mv = s.own[p * st + w] & s.big[w];
                    const uint32_t u = mv & s.dp[w], dn = mv & s.dp[st + w], l = mv & s.dp[2 * st + w],
                                   r = mv & s.dp[3 * st + w];
                    const uint32_t cw = __popc(u) + __popc(dn) + __popc(l) + __popc(r);
                    if (jj >= cw) {
                        jj -= cw;
                        continue;
                    }
                    uint32_t m = u | dn | l | r;
                    while (m) {
                        const int bit = __ffs(m) - 1;
                        const uint32_t dirs = ((u >> bit) & 1u) | (((dn >> bit) & 1u) << 1) |
                                              (((l >> bit) & 1u) << 2) | (((r >> bit) & 1u) << 3);
                        const uint32_t cb = __popc(dirs);
                        if (jj < cb) {
                            uint32_t dd = dirs;
                            for (uint32_t z = 0; z < jj; ++z) dd &= dd - 1;
                            const int d = __ffs(dd) - 1;
                            found = (32 * w + bit) * 9 + (split ? 5 + d : 1 + d);
                            break;
                        }
                        jj -= cb;
                        m &= m - 1;
                    }
                    break;
                }
            }
            action = __shfl_sync(kFull, found, L);
        }
        if (lane == 0) a.next_actions[g.player_off + p] = action;
    }
}

__device__ __forceinline__ void load_board(const KArgs& a, const Game& g, const Smem& s, int lane) {
    const int n16 = g.Npad >> 4;  // 16-byte vectors per int8 plane
    const uint4* ga = reinterpret_cast<const uint4*>(a.army + g.cell_off);
    const uint4* go = reinterpret_cast<const uint4*>(a.owner + g.cell_off);
    const uint4* gt = reinterpret_cast<const uint4*>(a.terrain + g.cell_off);
    uint4* sa = reinterpret_cast<uint4*>(s.army);
    uint4* so = reinterpret_cast<uint4*>(s.owner);
    uint4* st = reinterpret_cast<uint4*>(s.terrain);
    for (int v = lane; v < 2 * n16; v += 32) sa[v] = __ldcs(ga + v);
    for (int v = lane; v < n16; v += 32) {
        so[v] = __ldcs(go + v);
        st[v] = __ldcs(gt + v);
    }
    __syncwarp();
}

__device__ __forceinline__ void store_board(const KArgs& a, const Game& g, const Smem& s, int lane) {
    const int n16 = g.Npad >> 4;
    uint4* ga = reinterpret_cast<uint4*>(a.army + g.cell_off);
    uint4* go = reinterpret_cast<uint4*>(a.owner + g.cell_off);
    uint4* gt = reinterpret_cast<uint4*>(a.terrain + g.cell_off);
    const uint4* sa = reinterpret_cast<const uint4*>(s.army);
    const uint4* so = reinterpret_cast<const uint4*>(s.owner);
    const uint4* st = reinterpret_cast<const uint4*>(s.terrain);
    for (int v = lane; v < 2 * n16; v += 32) ga[v] = sa[v];
    for (int v = lane; v < n16; v += 32) {
        go[v] = so[v];
        gt[v] = st[v];
    }
}

}  // namespace

__global__ void __launch_bounds__(256) k_generals(const KArgs a) {
    extern __shared__ __align__(16) char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int item = blockIdx.x * (blockDim.x >> 5) + wid;
    if (item >= a.n_items) return;
    const int gidx = a.list ? a.list[item] : item;
    if (gidx < 0 || gidx >= a.n_games) return;
    const Game g = load_game(a.info + gidx);
    const Smem s = carve(smem_raw + wid * a.warp_smem, a);
    const uint64_t gid = a.game_id_base + (uint64_t)gidx;
    GameScalars* sc = a.scal + gidx;

    uint32_t turn, frame, epoch, alive, finished, invalid, saturated;
    if (a.op == OP_CREATE) {
        turn = frame = epoch = finished = invalid = saturated = 0;
    } else {
        turn = sc->turn;
        frame = sc->frame;
        epoch = sc->epoch;
        alive = sc->alive;
        finished = sc->finished;
        invalid = sc->invalid;
        saturated = sc->saturated;
    }
    const uint32_t all_alive = (1u << g.P) - 1u;
    bool wrote_state = false;
    float my_reward = 0.0f;
    uint32_t done = 0;

    if (a.op == OP_CREATE || a.op == OP_RESET) {
        if (a.op == OP_RESET) epoch += 1;
        generate(a, g, s, gid, epoch, lane);
        turn = 0;
        alive = all_alive;
        finished = 0;
        saturated += cell_pass(g, s, false, false, lane);
        wrote_state = true;
    } else {
        load_board(a, g, s, lane);
        if (a.op == OP_STEP) {
            if (!finished) {
                // moves in rotating priority, each checked when it runs (Q1)
                const int32_t my_act = (lane < g.P) ? a.actions[g.player_off + lane] : 0;
                uint32_t eliminated = 0;
                uint32_t inv0 = 0, sat0 = 0;
                for (int k = 0; k < g.P; ++k) {
                    const int p = (int)((turn + (uint32_t)k) % (uint32_t)g.P);
                    const int32_t act = __shfl_sync(kFull, my_act, p);
                    int cap = 0;
                    if (lane == 0 && ((alive >> p) & 1u)) cap = resolve_move(g, s, p, act, alive, inv0, sat0);
                    cap = __shfl_sync(kFull, cap, 0);
                    alive = __shfl_sync(kFull, alive, 0);
                    __syncwarp();
                    if (cap) {
                        // land transfer: every other cell of the loser, army - army/2 (Q7)
                        const int dst = cap & 0xFFFF, q = (cap >> 16) - 1;
                        eliminated |= 1u << q;
                        for (int c = lane; c < g.N; c += 32) {
                            if (c != dst && s.owner[c] == q) {
                                s.owner[c] = (int8_t)p;
                                const int av = s.army[c];
                                s.army[c] = (int16_t)(av - (av >> 1));
                            }
                        }
                        __syncwarp();
                    }
                }
                invalid += __shfl_sync(kFull, inv0, 0);
                saturated += __shfl_sync(kFull, sat0, 0);
                turn += 1;
                saturated += cell_pass(g, s, (turn % 2u) == 0u, (turn % 50u) == 0u, lane);
                // termination and reward (Sec. III, IV-D, IV-E; Q17, Q21)
                if (g.mode == 1) {
                    const bool dead0 = (alive & 0x3u) == 0u, dead1 = (alive & 0xCu) == 0u;
                    if (dead0 || dead1) {
                        done = 1;
                        const bool mine_dead = ((lane >> 1) == 0) ? dead0 : dead1;
                        my_reward = mine_dead ? -1.0f : 1.0f;
                    }
                } else {
                    if ((eliminated >> lane) & 1u) my_reward = -1.0f;
                    if (__popc(alive) <= 1) {
                        done = 1;
                        if ((alive >> lane) & 1u) my_reward = 1.0f;
                    }
                }
                if (!done && a.max_turns > 0 && turn >= (uint32_t)a.max_turns) done = 2;
                if (done) {
                    if (a.auto_reset) {
                        epoch += 1;
                        generate(a, g, s, gid, epoch, lane);
                        turn = 0;
                        alive = all_alive;
                        cell_pass(g, s, false, false, lane);
                    } else {
                        finished = 1;
                    }
                }
                wrote_state = true;
            } else {
                cell_pass(g, s, false, false, lane);  // frozen game: outputs only
            }
            frame += 1;
        } else {
            cell_pass(g, s, false, false, lane);
        }
    }

    if (a.op != OP_POLICY) {
        if (a.do_outputs) {
            fog_pass(g, s, alive, lane);
            output_pass(a, g, s, alive, finished != 0, lane);
            if (lane < g.P) {
                a.reward[g.player_off + lane] = my_reward;
                a.scoreboard[2 * (g.player_off + lane) + 0] = s.misc[8 + lane];
                a.scoreboard[2 * (g.player_off + lane) + 1] = s.misc[16 + lane];
            }
            if (lane == 0) a.done[gidx] = (uint8_t)done;
        }
    }
    if (a.next_actions) policy_pass(a, g, s, alive, finished != 0, frame, gid, lane);
    if (wrote_state) {
        __syncwarp();
        store_board(a, g, s, lane);
    }
    if (lane == 0 && a.op != OP_OBSERVE && a.op != OP_POLICY) {
        GameScalars o;
        o.turn = turn;
        o.frame = frame;
        o.epoch = epoch;
        o.alive = alive;
        o.finished = finished;
        o.invalid = invalid;
        o.saturated = saturated;
        o.err = (a.op == OP_CREATE) ? 0u : sc->err;
        *sc = o;
    }
}

__global__ void k_copy(const uint4* __restrict__ src, uint4* __restrict__ dst, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (; i < n; i += stride) __stcs(dst + i, __ldcs(src + i));
}

int warp_smem_bytes(int npad_max, int pmax, int* nw_stride) {
    int nw = (npad_max + 31) / 32;
    nw = (nw + 3) & ~3;
    if (nw_stride) *nw_stride = nw;
    return 4 * npad_max + 4 * nw * (2 * pmax + 8) + 4 * 24;
}

int launch_step(const KArgs& a, int warps_per_cta, void* stream) {
    if (a.n_items <= 0) return 0;
    const int smem = a.warp_smem * warps_per_cta;
    static int configured = 0;
    if (smem > 48 * 1024 && smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(k_generals, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return (int)e;
        configured = smem;
    }
    const int blocks = (a.n_items + warps_per_cta - 1) / warps_per_cta;
    k_generals<<<blocks, 32 * warps_per_cta, smem, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

int launch_copy(const void* src, void* dst, size_t n16, int blocks, void* stream) {
    k_copy<<<blocks, 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<const uint4*>(src),
                                                      reinterpret_cast<uint4*>(dst), n16);
    return (int)cudaGetLastError();
}

}  // namespace gk
