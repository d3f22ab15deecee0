// Feature tensor of every player (Appendix A, table of observation
// channels): C = 24 + 2K float planes per player over the game's own board.
//
// Rows 0-3 and 9-13 are the instantaneous fogged view, 4-8 and 20-21 the
// player's persistent memory, 14-19 broadcast scalars (turn, its phase in the
// 50-turn cycle, own and opponents' land and army from the public scoreboard),
// 22-23 coordinates and 24 on the last K differences of the own and the
// (fogged) enemy army planes.  The memory is folded once per frame (keyed by
// the game's frame counter) and cleared when the game's epoch changes.
// Readings: "opponent" = another team; enemy planes use the fogged view;
// neutral cells exclude mountains; structures in fog = fogged mountains and
// castles (shown as obstacles) and remembered generals; the age row is
// log(1 + dt) / 5 with dt the turns since an enemy was last seen on the cell,
// 0 when visible or never seen; coordinates col / (W - 1), row / (H - 1);
// frames before the episode count as zero planes.
//
// One warp per game: the board is staged in shared memory once, then each
// player in turn gets a visibility bitset (3x3 dilation of its team's cells)
// and a pass over the cells, four consecutive cells per lane, that reads the
// memory, writes the 24 + 2K channels with 16-byte streaming stores and
// writes the folded memory back.  HBM-bound: per player and cell it moves
// 4 (24 + 2K) bytes of output, 2 * 2K bytes of history and 15 bytes of memory.
#include <cuda_runtime.h>

#include <cstdint>

#include "gk_internal.h"

namespace gk {
namespace {

constexpr unsigned kAll = 0xFFFFFFFFu;
constexpr int kWarps = 8;

// shared memory of one warp: board (4 bytes per cell), team and visibility
// bitsets, scoreboard; a multiple of 16 bytes
__host__ __device__ __forceinline__ int warp_bytes(int npad_max) {
    const int nw_max = (npad_max + 31) >> 5;
    return (4 * npad_max + 8 * nw_max + 64 + 15) & ~15;
}

__device__ __forceinline__ uint32_t valid_word(int N, int w) {
    const int lo = 32 * w;
    if (lo + 32 <= N) return kAll;
    if (lo >= N) return 0u;
    return (1u << (N - lo)) - 1u;
}

// bits of word w whose cell index is congruent to r modulo W
__device__ __forceinline__ uint32_t column_word(int w, int W, int r) {
    const int c0 = 32 * w;
    int first = (r - c0 % W) % W;
    if (first < 0) first += W;
    uint32_t m = 0;
    for (int b = first; b < 32; b += W) m |= 1u << b;
    return m;
}

// x shifted so that bit c receives bit c - s of x (s may be negative), over
// an nw-word bitset in shared memory
__device__ __forceinline__ uint32_t shifted(const uint32_t* x, int nw, int w, int s) {
    if (s == 0) return x[w];
    if (s > 0) {
        const int q = s >> 5, r = s & 31;
        const int a = w - q;
        uint32_t v = a >= 0 ? x[a] << r : 0u;
        if (r && a - 1 >= 0) v |= x[a - 1] >> (32 - r);
        return v;
    }
    const int t = -s, q = t >> 5, r = t & 31;
    const int a = w + q;
    uint32_t v = a < nw ? x[a] >> r : 0u;
    if (r && a + 1 < nw) v |= x[a + 1] << (32 - r);
    return v;
}

__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d) {
    __stcs(reinterpret_cast<float4*>(p), make_float4(a, b, c, d));
}

__device__ __forceinline__ int lo16(uint32_t x) { return (int)(int16_t)(x & 0xFFFFu); }
__device__ __forceinline__ int hi16(uint32_t x) { return (int)(int16_t)(x >> 16); }

// age row: log(1 + dt) / 5 in double, rounded once
__device__ __forceinline__ float age_value(int dt) {
    return dt > 0 ? (float)(log(1.0 + (double)dt) / 5.0) : 0.0f;
}

__global__ void __launch_bounds__(256) k_features(const FArgs f) {
    extern __shared__ __align__(16) char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int gidx = blockIdx.x * kWarps + wid;
    if (gidx >= f.n_games) return;

    const int nw_max = (f.npad_max + 31) >> 5;
    char* base = smem + (size_t)wid * warp_bytes(f.npad_max);
    int16_t* s_army = reinterpret_cast<int16_t*>(base);
    int8_t* s_owner = reinterpret_cast<int8_t*>(base + 2 * f.npad_max);
    int8_t* s_terrain = reinterpret_cast<int8_t*>(base + 3 * f.npad_max);
    uint32_t* s_team = reinterpret_cast<uint32_t*>(base + 4 * f.npad_max);
    uint32_t* s_vis = s_team + nw_max;
    int32_t* s_score = reinterpret_cast<int32_t*>(s_vis + nw_max);  // land[8], army[8]

    const GameInfo gi = f.info[gidx];
    const int H = gi.H, W = gi.W, N = gi.N, Npad = gi.Npad, P = gi.P, mode = gi.mode;
    const int nw = (Npad + 31) >> 5;
    const GameScalars sc = f.scal[gidx];
    const int C = 24 + 2 * f.hist, K = f.hist, R = f.hist + 1;

    // board to shared memory, 16 bytes per lane and copy
    {
        const uint4* ga = reinterpret_cast<const uint4*>(f.army + gi.cell_off);
        const uint4* go = reinterpret_cast<const uint4*>(f.owner + gi.cell_off);
        const uint4* gt = reinterpret_cast<const uint4*>(f.terrain + gi.cell_off);
        const int n16 = Npad >> 4;
        for (int v = lane; v < 2 * n16; v += 32) reinterpret_cast<uint4*>(s_army)[v] = __ldg(ga + v);
        for (int v = lane; v < n16; v += 32) {
            reinterpret_cast<uint4*>(s_owner)[v] = __ldg(go + v);
            reinterpret_cast<uint4*>(s_terrain)[v] = __ldg(gt + v);
        }
    }
    __syncwarp();

    // public scoreboard (Sec. IV-B): land and army per player
    for (int q = 0; q < P; ++q) {
        int land = 0, army = 0;
        for (int c = lane; c < N; c += 32)
            if (s_owner[c] == q) {
                land += 1;
                army += s_army[c];
            }
        land = (int)__reduce_add_sync(kAll, (unsigned)land);
        army = (int)__reduce_add_sync(kAll, (unsigned)army);
        if (lane == 0) {
            s_score[q] = land;
            s_score[8 + q] = army;
        }
    }
    __syncwarp();

    const int turn = (int)sc.turn;
    const float f_turn = (float)turn;
    const float f_phase = (float)(turn % 50) / 50.0f;

    for (int p = 0; p < P; ++p) {
        const int tp = mode == 1 ? (p >> 1) : p;
        const bool alive = (sc.alive >> p) & 1u;
        // team cells, then their 3x3 dilation (Sec. IV-B)
        for (int w = 0; w < nw; ++w) {
            const int c = 32 * w + lane;
            const int o = c < N ? s_owner[c] : -1;
            const bool mine = alive && o >= 0 && (mode == 1 ? (o >> 1) : o) == tp;
            const unsigned b = __ballot_sync(kAll, mine);
            if (lane == 0) s_team[w] = b;
        }
        __syncwarp();
        for (int w = lane; w < nw; w += 32) {
            const uint32_t x = s_team[w];
            const uint32_t left = shifted(s_team, nw, w, 1) & ~column_word(w, W, 0);       // from c - 1
            const uint32_t right = shifted(s_team, nw, w, -1) & ~column_word(w, W, W - 1); // from c + 1
            s_vis[w] = x | left | right;
        }
        __syncwarp();
        uint32_t vis_w[4];
        for (int i = 0; i < 4; ++i) {
            const int w = lane + 32 * i;
            vis_w[i] = 0u;
            if (w < nw)
                vis_w[i] = (s_vis[w] | shifted(s_vis, nw, w, W) | shifted(s_vis, nw, w, -W)) & valid_word(N, w);
        }
        __syncwarp();
        for (int i = 0; i < 4; ++i) {
            const int w = lane + 32 * i;
            if (w < nw) s_vis[w] = vis_w[i];
        }
        __syncwarp();

        // scalars of this player (Q30)
        int opp_land = 0, opp_army = 0;
        for (int q = 0; q < P; ++q)
            if ((mode == 1 ? (q >> 1) : q) != tp) {
                opp_land += s_score[q];
                opp_army += s_score[8 + q];
            }
        const float f_own_land = (float)s_score[p], f_own_army = (float)s_score[8 + p];
        const float f_opp_land = (float)opp_land, f_opp_army = (float)opp_army;

        // memory header: clear on a new epoch, fold once per frame
        const int slot = gi.player_off + p;
        const uint4 h = f.hdr[slot];
        const bool cleared = h.x != sc.epoch + 1u;
        const bool fold = cleared || h.y != sc.frame;
        const int nvalid_old = cleared ? 0 : (int)h.w;
        const int head = fold ? (cleared ? 0 : (int)((h.z + 1u) % (uint32_t)R)) : (int)h.z;
        const int nvalid = fold ? min(nvalid_old + 1, R) : nvalid_old;

        const int64_t q0 = gi.plane_off + (int64_t)p * Npad;  // this player's plane
        float* out = f.out + q0 * C;
        for (int c = 4 * lane; c < Npad; c += 128) {
            const int64_t pc = q0 + c;
            // board of cells c..c+3
            const uint2 a2 = *reinterpret_cast<const uint2*>(s_army + c);
            const uint32_t ow = *reinterpret_cast<const uint32_t*>(s_owner + c);
            const uint32_t tw = *reinterpret_cast<const uint32_t*>(s_terrain + c);
            const uint32_t vbits = (s_vis[c >> 5] >> (c & 31)) & 0xFu;
            // memory of cells c..c+3
            uint32_t mb = cleared ? 0u : *reinterpret_cast<const uint32_t*>(f.mem_bits + pc);
            uint2 lea = make_uint2(0u, 0u);
            int4 let = make_int4(0, 0, 0, 0);
            if (!cleared) {
                lea = *reinterpret_cast<const uint2*>(f.mem_army + pc);
                let = *reinterpret_cast<const int4*>(f.mem_turn + pc);
            }
            int av[4], own[4], enemy[4], neut[4], lea_n[4], dt[4];
            uint32_t flags = 0;  // per cell byte: bit 0 in board, 1 visible, 2 own, 3 opponent, 5 neutral, 6 fog structure
            int let_n[4] = {let.x, let.y, let.z, let.w};
            const int lea_o[4] = {lo16(lea.x), hi16(lea.x), lo16(lea.y), hi16(lea.y)};
            const int arm[4] = {lo16(a2.x), hi16(a2.x), lo16(a2.y), hi16(a2.y)};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const bool in = c + i < N;
                const int o = (int)(int8_t)(ow >> (8 * i));
                const int t = (int)((tw >> (8 * i)) & 0x3u);
                const bool v = in && ((vbits >> i) & 1u);
                const bool isown = in && o == p;
                const bool isopp = in && o >= 0 && (mode == 1 ? (o >> 1) : o) != tp;
                const int a = in ? arm[i] : 0;
                av[i] = v ? a : 0;
                own[i] = isown ? a : 0;
                enemy[i] = (v && isopp) ? a : 0;
                neut[i] = (v && o == -1) ? a : 0;
                uint32_t m = (mb >> (8 * i)) & 0x1Fu;
                const bool seen_old = m & 1u;
                if (v) {
                    m |= 1u;
                    if (isopp) {
                        m |= 2u;
                        let_n[i] = turn;
                    }
                    if (t == 3) m |= 4u;
                    if (t == 2) m |= 8u;
                    if (t == 1) m |= 16u;
                }
                mb = (mb & ~(0xFFu << (8 * i))) | (m << (8 * i));
                lea_n[i] = v ? enemy[i] : (seen_old ? lea_o[i] : 0);
                dt[i] = (!v && (m & 2u)) ? turn - let_n[i] : 0;
                uint32_t fl = in ? 1u : 0u;
                if (v) fl |= 2u;
                if (isown) fl |= 4u;
                if (v && isopp) fl |= 8u;
                if (v && o == -1 && t != 1) fl |= 32u;
                if (in && !v && (t == 1 || t == 2 || (m & 4u))) fl |= 64u;
                flags |= fl << (8 * i);
            }
            auto flag = [&](int i, uint32_t b) { return (float)((flags >> (8 * i + b)) & 1u); };
            auto bit = [&](int i, int b) { return (float)((mb >> (8 * i + b)) & 1u); };
            auto row = [&](int ch) { return out + (int64_t)ch * Npad + c; };
            st4(row(0), (float)av[0], (float)av[1], (float)av[2], (float)av[3]);
            st4(row(1), (float)own[0], (float)own[1], (float)own[2], (float)own[3]);
            st4(row(2), (float)enemy[0], (float)enemy[1], (float)enemy[2], (float)enemy[3]);
            st4(row(3), (float)neut[0], (float)neut[1], (float)neut[2], (float)neut[3]);
#pragma unroll
            for (int b = 0; b < 5; ++b) st4(row(4 + b), bit(0, b), bit(1, b), bit(2, b), bit(3, b));
            st4(row(9), flag(0, 5), flag(1, 5), flag(2, 5), flag(3, 5));
            st4(row(10), flag(0, 2), flag(1, 2), flag(2, 2), flag(3, 2));
            st4(row(11), flag(0, 3), flag(1, 3), flag(2, 3), flag(3, 3));
            {
                auto fog = [&](int i) { return (float)(((flags >> (8 * i)) & 3u) == 1u); };  // in, not visible
                st4(row(12), fog(0), fog(1), fog(2), fog(3));
            }
            st4(row(13), flag(0, 6), flag(1, 6), flag(2, 6), flag(3, 6));
            {
                auto in_ = [&](int i, float x) { return ((flags >> (8 * i)) & 1u) ? x : 0.0f; };
                st4(row(14), in_(0, f_turn), in_(1, f_turn), in_(2, f_turn), in_(3, f_turn));
                st4(row(15), in_(0, f_phase), in_(1, f_phase), in_(2, f_phase), in_(3, f_phase));
                st4(row(16), in_(0, f_own_land), in_(1, f_own_land), in_(2, f_own_land), in_(3, f_own_land));
                st4(row(17), in_(0, f_own_army), in_(1, f_own_army), in_(2, f_own_army), in_(3, f_own_army));
                st4(row(18), in_(0, f_opp_land), in_(1, f_opp_land), in_(2, f_opp_land), in_(3, f_opp_land));
                st4(row(19), in_(0, f_opp_army), in_(1, f_opp_army), in_(2, f_opp_army), in_(3, f_opp_army));
                st4(row(20), (float)lea_n[0], (float)lea_n[1], (float)lea_n[2], (float)lea_n[3]);
                st4(row(21), age_value(dt[0]), age_value(dt[1]), age_value(dt[2]), age_value(dt[3]));
                // coordinates (Q32)
                float cx[4], cy[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int cc = c + i, r = cc / W, col = cc - r * W;
                    cx[i] = in_(i, W > 1 ? (float)col / (float)(W - 1) : 0.0f);
                    cy[i] = in_(i, H > 1 ? (float)r / (float)(H - 1) : 0.0f);
                }
                st4(row(22), cx[0], cx[1], cx[2], cx[3]);
                st4(row(23), cy[0], cy[1], cy[2], cy[3]);
            }
            // deltas (Q33): plane 0 is this frame, plane k >= 1 the ring slot k back
            {
                int po[4] = {own[0], own[1], own[2], own[3]};
                int pe[4] = {enemy[0], enemy[1], enemy[2], enemy[3]};
                for (int k = 0; k < K; ++k) {
                    int no[4] = {0, 0, 0, 0}, ne[4] = {0, 0, 0, 0};
                    if (k + 1 < nvalid) {
                        const int s = (head - (k + 1) + R) % R;
                        const uint2 xo = __ldcs(reinterpret_cast<const uint2*>(f.ring + (int64_t)(2 * s) * f.plane_cells + pc));
                        const uint2 xe =
                            __ldcs(reinterpret_cast<const uint2*>(f.ring + (int64_t)(2 * s + 1) * f.plane_cells + pc));
                        no[0] = lo16(xo.x), no[1] = hi16(xo.x), no[2] = lo16(xo.y), no[3] = hi16(xo.y);
                        ne[0] = lo16(xe.x), ne[1] = hi16(xe.x), ne[2] = lo16(xe.y), ne[3] = hi16(xe.y);
                    }
                    st4(row(24 + k), (float)(po[0] - no[0]), (float)(po[1] - no[1]), (float)(po[2] - no[2]),
                        (float)(po[3] - no[3]));
                    st4(row(24 + K + k), (float)(pe[0] - ne[0]), (float)(pe[1] - ne[1]), (float)(pe[2] - ne[2]),
                        (float)(pe[3] - ne[3]));
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        po[i] = no[i];
                        pe[i] = ne[i];
                    }
                }
            }
            if (fold) {
                *reinterpret_cast<uint32_t*>(f.mem_bits + pc) = mb;
                *reinterpret_cast<uint2*>(f.mem_army + pc) =
                    make_uint2(((uint32_t)lea_n[0] & 0xFFFFu) | ((uint32_t)lea_n[1] << 16),
                               ((uint32_t)lea_n[2] & 0xFFFFu) | ((uint32_t)lea_n[3] << 16));
                *reinterpret_cast<int4*>(f.mem_turn + pc) = make_int4(let_n[0], let_n[1], let_n[2], let_n[3]);
                *reinterpret_cast<uint2*>(f.ring + (int64_t)(2 * head) * f.plane_cells + pc) =
                    make_uint2(((uint32_t)own[0] & 0xFFFFu) | ((uint32_t)own[1] << 16),
                               ((uint32_t)own[2] & 0xFFFFu) | ((uint32_t)own[3] << 16));
                *reinterpret_cast<uint2*>(f.ring + (int64_t)(2 * head + 1) * f.plane_cells + pc) =
                    make_uint2(((uint32_t)enemy[0] & 0xFFFFu) | ((uint32_t)enemy[1] << 16),
                               ((uint32_t)enemy[2] & 0xFFFFu) | ((uint32_t)enemy[3] << 16));
            }
        }
        if (fold && lane == 0) f.hdr[slot] = make_uint4(sc.epoch + 1u, sc.frame, (uint32_t)head, (uint32_t)nvalid);
        __syncwarp();
    }
}

}  // namespace

int launch_features(const FArgs& f, void* stream) {
    if (f.n_games <= 0) return 0;
    const int smem = kWarps * warp_bytes(f.npad_max);
    static int configured = 48 * 1024;
    if (smem > configured) {
        const cudaError_t e = cudaFuncSetAttribute(k_features, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return (int)e;
        configured = smem;
    }
    const int blocks = (f.n_games + kWarps - 1) / kWarps;
    k_features<<<blocks, 32 * kWarps, smem, (cudaStream_t)stream>>>(f);
    return (int)cudaGetLastError();
}

}  // namespace gk
