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
// Two forms of the same computation.  k_features: one warp per game -- the
// board is staged in shared memory once, then each player in turn gets a
// visibility bitset (3x3 dilation of its team's cells) and a pass over the
// cells, four consecutive cells per lane, that reads the memory, writes the
// 24 + 2K channels with 16-byte streaming stores and writes the folded memory
// back.  k_features_cta, for batches too small to fill the GPU one warp per
// game: one CTA per (game, player); each warp stages the memory and history
// planes of two of the player's 128-cell chunks with cp.async while one warp
// builds the player's bitset and others the scoreboard, then writes those
// chunks; the player's memory header is read before the CTA's last barrier
// and written after it.
// HBM-bound: per player and cell it moves 4 (24 + 2K) bytes of output,
// 2 * 2K bytes of history and 15 bytes of memory.
#include <cuda_runtime.h>

#include <atomic>

#include <algorithm>
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
    return (4 * npad_max + 8 * nw_max + 64 + 8 * kMaxSide + 15) & ~15;
}

// the coordinate rows' values (Q32) by column and by row: column / (W - 1)
// and row / (H - 1), 0 when the side is 1; computed once per game
__device__ __forceinline__ void coord_table(float* s_coord, int H, int W, int tid, int nthreads) {
    for (int i = tid; i < 2 * kMaxSide; i += nthreads) {
        const int v = i < kMaxSide ? i : i - kMaxSide, side = i < kMaxSide ? W : H;
        s_coord[i] = side > 1 && v < side ? (float)v / (float)(side - 1) : 0.0f;
    }
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

// flag byte of one cell
constexpr uint32_t kFIn = 1u;          // on the board (not padding)
constexpr uint32_t kFVis = 2u;         // visible
constexpr uint32_t kFOwn = 4u;         // owned by the player
constexpr uint32_t kFOpp = 8u;         // visible and owned by an opponent
constexpr uint32_t kFUnowned = 16u;    // visible and unowned
constexpr uint32_t kFNeutral = 32u;    // visible, unowned, not a mountain
constexpr uint32_t kFFogStruct = 64u;  // fogged structure
constexpr uint32_t kFKeep = 128u;      // fogged and seen before: keep the last enemy army
static_assert(kFIn == 1u << 0 && kFVis == 1u << 1 && kFOwn == 1u << 2 && kFOpp == 1u << 3 &&
                  kFNeutral == 1u << 5 && kFFogStruct == 1u << 6,
              "st4b<S> call sites name these bit positions");

// four int16 values, each kept where the cell's flag byte has `bit`, else 0
__device__ __forceinline__ uint2 select16(uint2 x, uint32_t fl, uint32_t bit) {
    const uint32_t m0 = (fl & bit) ? 0x0000FFFFu : 0u;
    const uint32_t m1 = (fl & (bit << 8)) ? 0xFFFF0000u : 0u;
    const uint32_t m2 = (fl & (bit << 16)) ? 0x0000FFFFu : 0u;
    const uint32_t m3 = (fl & (bit << 24)) ? 0xFFFF0000u : 0u;
    return make_uint2(x.x & (m0 | m1), x.y & (m2 | m3));
}
__device__ __forceinline__ uint2 or2(uint2 a, uint2 b) { return make_uint2(a.x | b.x, a.y | b.y); }

__device__ __forceinline__ void st4i(float* p, uint2 x) {
    __stcs(reinterpret_cast<float4*>(p),
           make_float4((float)lo16(x.x), (float)hi16(x.x), (float)lo16(x.y), (float)hi16(x.y)));
}
// all ones where the sign bit of byte B of x is set, else 0 (prmt's sign
// replication: selector nibble 8 + B for every byte of the result)
template <int B>
__device__ __forceinline__ uint32_t byte_sign(uint32_t x) {
    uint32_t r;
    asm("prmt.b32 %0, %1, 0, %2;" : "=r"(r) : "r"(x), "n"(0x8888 + 0x1111 * B));
    return r;
}
// 1.0 where the byte of each cell has bit S: the bit is moved to each byte's
// sign position and spread over the word
template <int S>
__device__ __forceinline__ void st4b(float* p, uint32_t w) {
    const uint32_t t = w << (7 - S), one = 0x3F800000u;
    __stcs(reinterpret_cast<float4*>(p), make_float4(__uint_as_float(byte_sign<0>(t) & one),
                                                     __uint_as_float(byte_sign<1>(t) & one),
                                                     __uint_as_float(byte_sign<2>(t) & one),
                                                     __uint_as_float(byte_sign<3>(t) & one)));
}
// a broadcast scalar on board cells, 0 on padding
__device__ __forceinline__ void st4s(float* p, uint32_t fl, float x) {
    __stcs(reinterpret_cast<float4*>(p), make_float4((fl & kFIn) ? x : 0.0f, (fl & (kFIn << 8)) ? x : 0.0f,
                                                     (fl & (kFIn << 16)) ? x : 0.0f, (fl & (kFIn << 24)) ? x : 0.0f));
}
// four int16 values as floats
__device__ __forceinline__ float4 f4_16(uint2 x) {
    return make_float4((float)lo16(x.x), (float)hi16(x.x), (float)lo16(x.y), (float)hi16(x.y));
}

// age row: log(1 + dt) / 5 in double, rounded once (out of line: rare)
__device__ __noinline__ float age_log(int dt) { return (float)(log(1.0 + (double)dt) / 5.0); }
__device__ __forceinline__ float age_value(int dt) { return dt > 0 ? age_log(dt) : 0.0f; }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}

// land and army of player q on the board, by one warp
__device__ __forceinline__ void score_of(const int16_t* s_army, const int8_t* s_owner, int N, int q, int32_t* s_score,
                                         int lane) {
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

// player p's visibility bitset (Sec. IV-B): the 3x3 dilation of its team's
// cells, by one warp, through the scratch bitset s_team
__device__ __forceinline__ void vis_of(const int8_t* s_owner, uint32_t* s_team, uint32_t* s_vis, int N, int W, int nw,
                                       int mode, int tp, bool alive, int lane) {
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
        if (w < nw) vis_w[i] = (s_vis[w] | shifted(s_vis, nw, w, W) | shifted(s_vis, nw, w, -W)) & valid_word(N, w);
    }
    __syncwarp();
    for (int i = 0; i < 4; ++i) {
        const int w = lane + 32 * i;
        if (w < nw) s_vis[w] = vis_w[i];
    }
    __syncwarp();
}

// one player's frame: its scalars and memory-header state
struct PlayerFrame {
    int p, tp, slot;
    int opp_land, opp_army;
    float f_own_land, f_own_army, f_opp_land, f_opp_army;
    bool cleared, fold;
    uint32_t n_fold;  // frames folded this episode, this one included
    int head;         // ring slot of this frame
    int nvalid;       // ring slots holding frames of this episode
};

// LOAD_HDR: the player's memory header is read from global memory here (the
// warp form), else `h` holds it (the CTA form stages the headers)
template <bool LOAD_HDR>
__device__ __forceinline__ PlayerFrame player_frame_t(const FArgs& f, const GameInfo& gi, const GameScalars& sc,
                                                      const int32_t* s_score, int p, int R, uint4 h) {
    PlayerFrame x;
    x.p = p;
    x.tp = gi.mode == 1 ? (p >> 1) : p;
    x.slot = gi.player_off + p;
    // scalars of this player (Q30)
    int opp_land = 0, opp_army = 0;
    for (int q = 0; q < gi.P; ++q)
        if ((gi.mode == 1 ? (q >> 1) : q) != x.tp) {
            opp_land += s_score[q];
            opp_army += s_score[8 + q];
        }
    x.opp_land = opp_land;
    x.opp_army = opp_army;
    x.f_own_land = (float)s_score[p];
    x.f_own_army = (float)s_score[8 + p];
    x.f_opp_land = (float)opp_land;
    x.f_opp_army = (float)opp_army;
    // memory header: clear on a new epoch, fold once per frame
    if (LOAD_HDR) h = f.hdr[x.slot];
    x.cleared = h.x != sc.epoch + 1u;
    x.fold = x.cleared || h.y != sc.frame;
    x.n_fold = (x.cleared ? 0u : h.z) + (x.fold ? 1u : 0u);
    x.head = (int)((x.n_fold - 1u) % (uint32_t)R);
    x.nvalid = (int)min(x.n_fold, (uint32_t)R);
    return x;
}

// temporal tokens (App. A) of one player: the ring entry of this frame
// (once), and entries k0, k0 + dk, ... of the newest-first copy
__device__ __forceinline__ void player_tokens(const FArgs& f, const PlayerFrame& x, bool write_ring, uint32_t k0,
                                              uint32_t dk) {
    const uint32_t T = (uint32_t)f.window;
    int2* ring = f.series_ring + (int64_t)x.slot * T;
    if (write_ring && x.fold) ring[(x.n_fold - 1u) % T] = make_int2(x.opp_army, x.opp_land);
    if (f.series_out) {
        int2* so = f.series_out + (int64_t)x.slot * T;
        const uint32_t valid = min(x.n_fold, T);
        const uint32_t newest = (x.n_fold - 1u) % T;  // entry k back is (newest - k) mod T
        for (uint32_t k = k0; k < T; k += dk) {
            int2 v = make_int2(0, 0);
            if (k == 0)
                v = make_int2(x.opp_army, x.opp_land);
            else if (k < valid)
                v = ring[newest >= k ? newest - k : newest + T - k];
            so[k] = v;
        }
    }
}

// cells c .. c+3 of one player: read and fold the memory, write the 24 + 2K
// rows.  mem(mb, lea, let) supplies the memory of the four cells (zeros when
// cleared) and ring_pair(back, own, enemy) the army planes `back` frames ago
// (zeros where the episode has none): global loads for the warp form, a
// shared-memory staging for the CTA form.
template <class Mem, class Ring>
__device__ __forceinline__ void cell_quad_from(const FArgs& f, const GameInfo& gi, const PlayerFrame& x, int turn,
                                               float f_turn, float f_phase, const int16_t* s_army,
                                               const int8_t* s_owner, const int8_t* s_terrain, const uint32_t* s_vis,
                                               const float* s_coord, int c, Mem mem, Ring ring_pair) {
    const int H = gi.H, W = gi.W, N = gi.N, Npad = gi.Npad, mode = gi.mode, p = x.p, tp = x.tp;
    const int C = 24 + 2 * f.hist, K = f.hist;
    const int64_t q0 = gi.plane_off + (int64_t)p * Npad;  // this player's plane
    float* out = f.out + q0 * C;
    const int64_t pc = q0 + c;
    // memory of cells c..c+3 (loads first)
    uint32_t mb = 0u;
    uint2 lea = make_uint2(0u, 0u);
    int4 let = make_int4(0, 0, 0, 0);
    mem(mb, lea, let);
    // board of cells c..c+3
    const uint2 a2 = *reinterpret_cast<const uint2*>(s_army + c);
    const uint32_t ow = *reinterpret_cast<const uint32_t*>(s_owner + c);
    const uint32_t tw = *reinterpret_cast<const uint32_t*>(s_terrain + c);
    const uint32_t vbits = (s_vis[c >> 5] >> (c & 31)) & 0xFu;
    // one flag byte per cell (kF*) and the folded memory masks
    uint32_t fl = 0u;
    int lt[4] = {let.x, let.y, let.z, let.w};
    float age[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool in = c + i < N;
        const int o = (int)(int8_t)(ow >> (8 * i));
        const uint32_t t = (tw >> (8 * i)) & 0x3u;
        const bool v = in && ((vbits >> i) & 1u);
        const bool opp = in && o >= 0 && (mode == 1 ? (o >> 1) : o) != tp;
        uint32_t m = (mb >> (8 * i)) & 0x1Fu;
        const bool seen_old = m & 1u;
        if (v) {
            m |= 1u;
            if (opp) {
                m |= 2u;
                lt[i] = turn;
            }
            m |= t == 3u ? 4u : t == 2u ? 8u : t == 1u ? 16u : 0u;
        }
        mb = (mb & ~(0xFFu << (8 * i))) | (m << (8 * i));
        age[i] = age_value((!v && (m & 2u)) ? turn - lt[i] : 0);
        uint32_t b = in ? kFIn : 0u;
        if (v) b |= kFVis;
        if (in && o == p) b |= kFOwn;
        if (v && opp) b |= kFOpp;
        if (v && o == -1) b |= kFUnowned;
        if (v && o == -1 && t != 1u) b |= kFNeutral;
        if (in && !v && (t == 1u || t == 2u || (m & 4u))) b |= kFFogStruct;
        if (!v && seen_old) b |= kFKeep;
        fl |= b << (8 * i);
    }
    const uint2 own = select16(a2, fl, kFOwn);
    const uint2 ene = select16(a2, fl, kFOpp);
    const uint2 lea_n = or2(ene, select16(lea, fl, kFKeep));  // Q31
    if (x.fold) {
        *reinterpret_cast<uint32_t*>(f.mem_bits + pc) = mb;
        *reinterpret_cast<uint2*>(f.mem_army + pc) = lea_n;
        *reinterpret_cast<int4*>(f.mem_turn + pc) = make_int4(lt[0], lt[1], lt[2], lt[3]);
        *reinterpret_cast<uint2*>(f.ring + (int64_t)(2 * x.head) * f.plane_cells + pc) = own;
        *reinterpret_cast<uint2*>(f.ring + (int64_t)(2 * x.head + 1) * f.plane_cells + pc) = ene;
    }
    float* row = out + c;
    st4i(row, select16(a2, fl, kFVis));
    st4i(row += Npad, own);
    st4i(row += Npad, ene);
    st4i(row += Npad, select16(a2, fl, kFUnowned));
    st4b<0>(row += Npad, mb);
    st4b<1>(row += Npad, mb);
    st4b<2>(row += Npad, mb);
    st4b<3>(row += Npad, mb);
    st4b<4>(row += Npad, mb);
    st4b<5>(row += Npad, fl);                // kFNeutral
    st4b<2>(row += Npad, fl);                // kFOwn
    st4b<3>(row += Npad, fl);                // kFOpp
    st4b<0>(row += Npad, fl & ~(fl >> 1));   // kFIn and not kFVis: on the board and not visible
    st4b<6>(row += Npad, fl);                // kFFogStruct
    st4s(row += Npad, fl, f_turn);
    st4s(row += Npad, fl, f_phase);
    st4s(row += Npad, fl, x.f_own_land);
    st4s(row += Npad, fl, x.f_own_army);
    st4s(row += Npad, fl, x.f_opp_land);
    st4s(row += Npad, fl, x.f_opp_army);
    st4i(row += Npad, lea_n);
    st4(row += Npad, age[0], age[1], age[2], age[3]);
    {  // coordinates (Q32)
        float cx[4], cy[4];
        int r = c / W, col = c - r * W;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const bool in = (fl >> (8 * i)) & kFIn;
            cx[i] = in ? s_coord[col] : 0.0f;
            cy[i] = in ? s_coord[kMaxSide + min(r, H - 1)] : 0.0f;
            if (++col == W) {
                col = 0;
                ++r;
            }
        }
        st4(row += Npad, cx[0], cx[1], cx[2], cx[3]);
        st4(row += Npad, cy[0], cy[1], cy[2], cy[3]);
    }
    // deltas (Q33): plane 0 is this frame, plane k >= 1 the ring slot k back;
    // each pair is fetched two iterations ahead of the stores that use it
    // (armies are below 2^15: the float differences are exact)
    float4 po = f4_16(own), pe = f4_16(ene);
    uint2 o1, e1, o2, e2;
    ring_pair(1, o1, e1);
    ring_pair(2, o2, e2);
    float* rd = row + (int64_t)Npad;
    for (int k = 0; k < K; ++k, rd += Npad) {
        uint2 o3, e3;
        ring_pair(k + 3, o3, e3);
        const float4 qo = f4_16(o1), qe = f4_16(e1);
        st4(rd, po.x - qo.x, po.y - qo.y, po.z - qo.z, po.w - qo.w);
        st4(rd + (int64_t)K * Npad, pe.x - qe.x, pe.y - qe.y, pe.z - qe.z, pe.w - qe.w);
        po = qo;
        pe = qe;
        o1 = o2;
        e1 = e2;
        o2 = o3;
        e2 = e3;
    }
}

// the warp form's cells: memory and ring planes loaded from global memory
__device__ __forceinline__ void cell_quad(const FArgs& f, const GameInfo& gi, const PlayerFrame& x, int turn,
                                          float f_turn, float f_phase, const int16_t* s_army, const int8_t* s_owner,
                                          const int8_t* s_terrain, const uint32_t* s_vis, const float* s_coord,
                                          int c) {
    const int R = f.hist + 1;
    const int64_t pc = gi.plane_off + (int64_t)x.p * gi.Npad + c;
    auto mem = [&](uint32_t& mb, uint2& lea, int4& let) {
        if (!x.cleared) {
            mb = __ldcs(reinterpret_cast<const unsigned int*>(f.mem_bits + pc));
            lea = __ldcs(reinterpret_cast<const uint2*>(f.mem_army + pc));
            let = __ldcs(reinterpret_cast<const int4*>(f.mem_turn + pc));
        }
    };
    auto ring_pair = [&](int back, uint2& o, uint2& e) {  // own / enemy planes `back` frames ago
        o = make_uint2(0u, 0u);
        e = o;
        if (back < x.nvalid) {
            const int sl = (x.head - back + R) % R;
            o = __ldcs(reinterpret_cast<const uint2*>(f.ring + (int64_t)(2 * sl) * f.plane_cells + pc));
            e = __ldcs(reinterpret_cast<const uint2*>(f.ring + (int64_t)(2 * sl + 1) * f.plane_cells + pc));
        }
    };
    cell_quad_from(f, gi, x, turn, f_turn, f_phase, s_army, s_owner, s_terrain, s_vis, s_coord, c, mem, ring_pair);
}

__global__ void __launch_bounds__(256, 4) k_features(const FArgs f) {
    chain_entry();
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
    float* s_coord = reinterpret_cast<float*>(s_score + 16);         // [2 * kMaxSide]

    const GameInfo gi = f.info[gidx];
    const int N = gi.N, Npad = gi.Npad, P = gi.P;
    const int nw = (Npad + 31) >> 5;
    const GameScalars sc = f.scal[gidx];
    const int R = f.hist + 1;

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
    coord_table(s_coord, gi.H, gi.W, lane, 32);
    __syncwarp();

    // public scoreboard (Sec. IV-B): land and army per player
    for (int q = 0; q < P; ++q) score_of(s_army, s_owner, N, q, s_score, lane);
    __syncwarp();

    const int turn = (int)sc.turn;
    const float f_turn = (float)turn;
    const float f_phase = (float)(turn % 50) / 50.0f;

    for (int p = 0; p < P; ++p) {
        const int tp = gi.mode == 1 ? (p >> 1) : p;
        vis_of(s_owner, s_team, s_vis, N, gi.W, nw, gi.mode, tp, (sc.alive >> p) & 1u, lane);
        const PlayerFrame x = player_frame_t<true>(f, gi, sc, s_score, p, R, make_uint4(0u, 0u, 0u, 0u));
        if (f.window > 0) player_tokens(f, x, lane == 0, (uint32_t)lane, 32u);
        for (int c = 4 * lane; c < Npad; c += 128)
            cell_quad(f, gi, x, turn, f_turn, f_phase, s_army, s_owner, s_terrain, s_vis, s_coord, c);
        if (x.fold && lane == 0) f.hdr[x.slot] = make_uint4(sc.epoch + 1u, sc.frame, x.n_fold, 0u);
        __syncwarp();
    }
}

// shared memory of the one-player CTA: board, the player's visibility bitset
// and a scratch bitset, scoreboard, coordinate table, the player's memory
// header, then per warp the staging of kItemsPerBatch items; a multiple of
// 16 bytes
constexpr int kItemsPerBatch = 2;
__host__ __device__ __forceinline__ int cta_hdr_offset(int npad_max) {  // 16-byte aligned
    const int nw_max = (npad_max + 31) >> 5;
    return (4 * npad_max + 8 * nw_max + 64 + 8 * kMaxSide + 15) & ~15;
}
__host__ __device__ __forceinline__ int cta_head_bytes(int npad_max) { return cta_hdr_offset(npad_max) + 16; }
// one item's staging, lane-major: memory bits (4 B), last enemy army (8 B) and
// turn (16 B) of the lane's four cells, then K (own, enemy) ring plane pairs
// (8 + 8 B)
__host__ __device__ __forceinline__ int item_stage_bytes(int hist) { return 32 * (28 + 16 * hist); }
__host__ __device__ __forceinline__ int cta_bytes(int npad_max, int hist, int warps) {
    return cta_head_bytes(npad_max) + warps * kItemsPerBatch * item_stage_bytes(hist);
}

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)), "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)), "l"(gmem)
                 : "memory");
}

// the part of a player's memory header that decides what is read
struct HdrState {
    bool cleared;
    int head, nvalid;
};
__device__ __forceinline__ HdrState hdr_state(const uint4 h, const GameScalars& sc, int R) {
    HdrState y;
    y.cleared = h.x != sc.epoch + 1u;
    const bool fold = y.cleared || h.y != sc.frame;
    const uint32_t n_fold = (y.cleared ? 0u : h.z) + (fold ? 1u : 0u);
    y.head = (int)((n_fold - 1u) % (uint32_t)R);
    y.nvalid = (int)min(n_fold, (uint32_t)R);
    return y;
}

// issue the copies of one item's memory and older ring planes into `st`
// (this lane's share; completed by cp.async.wait_all)
__device__ __forceinline__ void stage_item(const FArgs& f, const HdrState& y, int64_t pc, char* st, int lane) {
    const int K = f.hist, R = f.hist + 1;
    if (!y.cleared) {
        cp_async4(st + 4 * lane, f.mem_bits + pc);
        cp_async8(st + 128 + 8 * lane, f.mem_army + pc);
        cp_async16(st + 384 + 16 * lane, f.mem_turn + pc);
    }
    for (int back = 1; back <= K && back < y.nvalid; ++back) {
        const int sl = (y.head - back + R) % R;
        char* d = st + 896 + 512 * (back - 1);
        cp_async8(d + 8 * lane, f.ring + (int64_t)(2 * sl) * f.plane_cells + pc);
        cp_async8(d + 256 + 8 * lane, f.ring + (int64_t)(2 * sl + 1) * f.plane_cells + pc);
    }
}

// One CTA per (game, player): CTA b takes player b mod pmax of game
// b / pmax (CTAs of absent players return at once).  The board and the
// player's header are staged first; the items' memory and history planes are
// in flight while one warp builds the player's visibility bitset and the
// others the scoreboard (a warp per player); then warp w takes the player's
// 128-cell chunks w, w + warps, ... kItemsPerBatch at a time.
__global__ void __launch_bounds__(1024) k_features_cta(const FArgs f, int pmax) {
    extern __shared__ __align__(16) char smem[];
    chain_entry();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int gidx = blockIdx.x / pmax, p = blockIdx.x - gidx * pmax;
    const GameInfo gi = f.info[gidx];
    const int N = gi.N, Npad = gi.Npad, P = gi.P;
    if (p >= P) return;  // the same for the whole CTA

    const int nw_max = (f.npad_max + 31) >> 5;
    int16_t* s_army = reinterpret_cast<int16_t*>(smem);
    int8_t* s_owner = reinterpret_cast<int8_t*>(smem + 2 * f.npad_max);
    int8_t* s_terrain = reinterpret_cast<int8_t*>(smem + 3 * f.npad_max);
    uint32_t* s_vis = reinterpret_cast<uint32_t*>(smem + 4 * f.npad_max);  // [nw_max]
    uint32_t* s_team = s_vis + nw_max;                                      // [nw_max] scratch
    int32_t* s_score = reinterpret_cast<int32_t*>(s_team + nw_max);         // land[8], army[8]
    float* s_coord = reinterpret_cast<float*>(s_score + 16);                // [2 * kMaxSide]
    uint4* s_hdr = reinterpret_cast<uint4*>(smem + cta_hdr_offset(f.npad_max));
    char* s_stage = smem + cta_head_bytes(f.npad_max) + (size_t)wid * kItemsPerBatch * item_stage_bytes(f.hist);

    const int nw = (Npad + 31) >> 5;
    const GameScalars sc = f.scal[gidx];
    const int R = f.hist + 1, K = f.hist;
    const int chunks = (Npad + 127) >> 7;  // 128 cells: four per lane
    const int64_t q0 = gi.plane_off + (int64_t)p * Npad;
    {  // board to shared memory, every 16-byte copy in flight at once
        const uint4* ga = reinterpret_cast<const uint4*>(f.army + gi.cell_off);
        const uint4* go = reinterpret_cast<const uint4*>(f.owner + gi.cell_off);
        const uint4* gt = reinterpret_cast<const uint4*>(f.terrain + gi.cell_off);
        const int n16 = Npad >> 4;
        for (int v = threadIdx.x; v < 2 * n16; v += blockDim.x) cp_async16(reinterpret_cast<uint4*>(s_army) + v, ga + v);
        for (int v = threadIdx.x; v < n16; v += blockDim.x) {
            cp_async16(reinterpret_cast<uint4*>(s_owner) + v, go + v);
            cp_async16(reinterpret_cast<uint4*>(s_terrain) + v, gt + v);
        }
    }
    coord_table(s_coord, gi.H, gi.W, threadIdx.x, blockDim.x);
    uint4 my_hdr = make_uint4(0u, 0u, 0u, 0u);
    if (threadIdx.x == 0) {  // read before the last barrier, written after it
        my_hdr = f.hdr[gi.player_off + p];
        *s_hdr = my_hdr;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    const uint4 h = *s_hdr;
    const HdrState y = hdr_state(h, sc, R);
    // this warp's chunks are wid, wid + nwarps, ...; batch b holds the
    // kItemsPerBatch of them from the (b * kItemsPerBatch)-th on
    auto stage_batch = [&](int b) {
        for (int j = 0; j < kItemsPerBatch; ++j) {
            const int k = wid + nwarps * (b * kItemsPerBatch + j), c = 128 * k + 4 * lane;
            if (k >= chunks) break;
            if (c < Npad) stage_item(f, y, q0 + c, s_stage + j * item_stage_bytes(f.hist), lane);
        }
    };
    stage_batch(0);  // in flight while the visibility and the scoreboard are built
    // task 0: the player's visibility bitset (Sec. IV-B); task 1 + q: player q's scoreboard entry
    for (int t = wid; t <= P; t += nwarps) {
        if (t == 0)
            vis_of(s_owner, s_team, s_vis, N, gi.W, nw, gi.mode, gi.mode == 1 ? (p >> 1) : p, (sc.alive >> p) & 1u, lane);
        else
            score_of(s_army, s_owner, N, t - 1, s_score, lane);
    }
    __syncthreads();

    const int turn = (int)sc.turn;
    const float f_turn = (float)turn;
    const float f_phase = (float)(turn % 50) / 50.0f;
    const PlayerFrame x = player_frame_t<false>(f, gi, sc, s_score, p, R, h);
    const int mine = chunks > wid ? (chunks - wid + nwarps - 1) / nwarps : 0;
    for (int b = 0; kItemsPerBatch * b < mine; ++b) {
        if (b > 0) stage_batch(b);
        asm volatile("cp.async.wait_all;" ::: "memory");
        for (int j = 0; j < kItemsPerBatch; ++j) {
            const int k = wid + nwarps * (b * kItemsPerBatch + j);
            if (k >= chunks) break;
            // the player's tokens are shared by its first min(chunks, warps) chunks
            if (f.window > 0) {
                const int per = min(chunks, nwarps);
                if (k < per) player_tokens(f, x, k == 0 && lane == 0, (uint32_t)(32 * k + lane), (uint32_t)(32 * per));
            }
            const int c = 128 * k + 4 * lane;
            if (c >= Npad) continue;
            const char* st = s_stage + j * item_stage_bytes(f.hist);
            auto mem = [&](uint32_t& mb, uint2& lea, int4& let) {
                if (!x.cleared) {
                    mb = *reinterpret_cast<const uint32_t*>(st + 4 * lane);
                    lea = *reinterpret_cast<const uint2*>(st + 128 + 8 * lane);
                    let = *reinterpret_cast<const int4*>(st + 384 + 16 * lane);
                }
            };
            auto ring_pair = [&](int back, uint2& o, uint2& e) {
                o = make_uint2(0u, 0u);
                e = o;
                if (back <= K && back < x.nvalid) {
                    const char* d = st + 896 + 512 * (back - 1);
                    o = *reinterpret_cast<const uint2*>(d + 8 * lane);
                    e = *reinterpret_cast<const uint2*>(d + 256 + 8 * lane);
                }
            };
            cell_quad_from(f, gi, x, turn, f_turn, f_phase, s_army, s_owner, s_terrain, s_vis, s_coord, c, mem,
                           ring_pair);
        }
        __syncwarp();  // this warp's staging is reused by its next batch
    }
    __syncthreads();  // every warp has read the header
    if (threadIdx.x == 0 && x.fold)
        f.hdr[gi.player_off + p] = make_uint4(sc.epoch + 1u, sc.frame, x.n_fold, 0u);
}

}  // namespace

int launch_features(const FArgs& f, int pmax, int form, void* stream) {
    if (f.n_games <= 0) return 0;
    static std::atomic<int> sm_count{0};  // of the first device used: only the launch shape depends on it
    int sms = sm_count.load(std::memory_order_relaxed);
    if (sms == 0) {
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        sms = n > 0 ? n : 1;
        sm_count.store(sms, std::memory_order_relaxed);
    }
    // the CTA form while the batch has at most 56 x the SM count players
    // (measured on 24x24 1v1, each build the first of its frame: 512 games
    // 28.5 against 69.3 us, 4,096 games 184.8 against 186.4 us, 8,192 games
    // 360 against 335 us)
    if (form == 0) form = (int64_t)f.n_games * pmax <= 56 * (int64_t)sms ? 2 : 1;
    if (form == 2) {
        // a CTA per (game, player) with a warp per kItemsPerBatch chunks, as
        // many as the staging leaves room for in shared memory
        const int chunks = (f.npad_max + 127) >> 7;
        const int per_warp = kItemsPerBatch * item_stage_bytes(f.hist);
        const int fit = (227 * 1024 - cta_head_bytes(f.npad_max)) / per_warp;
        const int warps = std::max(1, std::min(std::min(32, fit), (chunks + kItemsPerBatch - 1) / kItemsPerBatch));
        const int smem = cta_bytes(f.npad_max, f.hist, warps);
        static SmemLimit limit;
        const void* fn = (const void*)k_features_cta;
        const int e = limit.raise(&fn, 1, smem);
        if (e != 0) return e;
        return launch_chained(k_features_cta, dim3((unsigned)((int64_t)f.n_games * pmax)), dim3(32 * warps), smem,
                              (cudaStream_t)stream, f, pmax);
    }
    const int smem = kWarps * warp_bytes(f.npad_max);
    static SmemLimit limit;
    const void* fn = (const void*)k_features;
    const int e = limit.raise(&fn, 1, smem);
    if (e != 0) return e;
    const int blocks = (f.n_games + kWarps - 1) / kWarps;
    return launch_chained(k_features, dim3(blocks), dim3(32 * kWarps), smem, (cudaStream_t)stream, f);
}

}  // namespace gk
