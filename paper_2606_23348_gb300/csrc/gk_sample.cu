// Policy sampling over the H x W x 9 action space (Sec. IV-G; the policy
// head's H x W x 9 distribution, App. C) and the expanded legal mask.
//
// Legal entries of player p: (c, pass) where p owns c; (c, 1 + d) all-but-one
// and (c, 5 + d) half towards d where the move is legal (p alive and owning
// c, at least 2 units, the neighbour exists and is not a mountain, the game
// not finished).  Sampling is an exact integer inverse CDF, so that the same
// logits and seed pick the same action on every device:
//   m = max legal logit; w_e = floor(E(l_e - m) * 2^24) with E the
//   reproducible exponential below; S = sum of w_e (64-bit, exact);
//   r = floor(d * S / 2^64) for the 64-bit draw d = counter hash of (seed,
//   global game id, frame of the consuming step, p) at index 7; the action
//   is the first legal entry in index order whose running sum exceeds r.
// E(x) = 2^n * P(f): t = x * log2(e) in float, n = floor(t), f = t - n, P the
// degree-7 Taylor polynomial of 2^f (sum of (f ln 2)^k / k!) in Horner form
// with fused multiply-adds, 0 below t = -25.  Every operation is an IEEE
// single-precision operation with round-to-nearest written out explicitly
// (no contraction), so the weights are bit-reproducible.
//
// One CTA per game with a warp per player (k_sample_cta), one warp per game
// with the players in turn (k_sample), or, for small batches, one CTA per
// player with a thread per (own cell, entry) pair (k_sample_wide, described
// where it is defined).  The board is staged in
// shared memory (every 16-byte copy in flight at once); legal entries lie
// only on the player's own cells, so the warp first lists those cells in
// index order (a ballot per 32 cells, no global load) and the passes run over
// the list, 32 own cells at a time: pass 1 derives each cell's nine legal
// bits and takes the maximum; pass 2 (logits held in registers for the first
// 64 own cells, read again from L1/L2 beyond) sums each cell's weights,
// computing every exponential once (two entries per packed FMA chain), and
// keeps the sums per cell and per 32
// cells; pass 3 finds the group, the cell and (nine lanes weighing the cell's
// entries at once) the entry where the running sum first exceeds r.  Only the
// own cells' logits are read (36 bytes each).  The expanded mask, when asked
// for, is a dense pass over every cell (a cell's entries belong to its owner)
// written through shared memory with 16-byte stores.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>

#include "gk_internal.h"

namespace gk {
namespace {

constexpr unsigned kAll = 0xFFFFFFFFu;
constexpr int kWarps = 8;
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t stream_out(uint64_t s, uint64_t n) { return mix64(s + (n + 1) * kGamma); }
__device__ __forceinline__ uint64_t hkey(uint64_t s, uint64_t a, uint64_t b, uint64_t c) {
    return stream_out(stream_out(stream_out(s, a), b), c);
}

// weight of a legal entry: floor(E(l - m) * 2^24).  E = P * 2^n exactly
// (n >= -25, P in [1, 2)), so the floor is P's 24-bit significand shifted
// right by -(n + 1) bits; equal to the float floor of the exact product.
__device__ __forceinline__ uint32_t weight_shift(float l, float m) {
    const float t = __fmul_rn(__fsub_rn(l, m), 1.4426950408889634f);
    if (t < -25.0f) return 0u;
    const float nf = floorf(t);
    const float f = __fsub_rn(t, nf);
    float p = 1.5252733804059838e-05f;
    p = __fmaf_rn(p, f, 0.00015403530393381606f);
    p = __fmaf_rn(p, f, 0.0013333558146428441f);
    p = __fmaf_rn(p, f, 0.009618129107628477f);
    p = __fmaf_rn(p, f, 0.055504108664821576f);
    p = __fmaf_rn(p, f, 0.2402265069591007f);
    p = __fmaf_rn(p, f, 0.6931471805599453f);
    p = __fmaf_rn(p, f, 1.0f);
    const int n = (int)nf;                                          // -25 .. 0
    const uint32_t sig = (__float_as_uint(p) & 0x7FFFFFu) | 0x800000u;  // P * 2^23
    return n >= 0 ? sig << 1 : sig >> (-(n + 1));
}

// two weights at once: the same single-precision operations as
// weight_shift, issued as packed pairs (each half an IEEE round-to-nearest
// operation of its own, so the results are bit for bit those of two calls)
__device__ __forceinline__ uint64_t pack2(float a, float b) {
    return (uint64_t)__float_as_uint(a) | ((uint64_t)__float_as_uint(b) << 32);
}
__device__ __forceinline__ float lo2(uint64_t x) { return __uint_as_float((uint32_t)x); }
__device__ __forceinline__ float hi2(uint64_t x) { return __uint_as_float((uint32_t)(x >> 32)); }
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint32_t weight_from(float t, float nf, float p) {
    if (t < -25.0f) return 0u;
    const int n = (int)nf;
    const uint32_t sig = (__float_as_uint(p) & 0x7FFFFFu) | 0x800000u;
    return n >= 0 ? sig << 1 : sig >> (-(n + 1));
}
__device__ __forceinline__ uint2 weight_shift2(float l0, float l1, float m) {
    const float t0 = __fmul_rn(__fsub_rn(l0, m), 1.4426950408889634f);
    const float t1 = __fmul_rn(__fsub_rn(l1, m), 1.4426950408889634f);
    const float n0 = floorf(t0), n1 = floorf(t1);
    const uint64_t f = pack2(__fsub_rn(t0, n0), __fsub_rn(t1, n1));
    uint64_t p = pack2(1.5252733804059838e-05f, 1.5252733804059838e-05f);
    p = fma2(p, f, pack2(0.00015403530393381606f, 0.00015403530393381606f));
    p = fma2(p, f, pack2(0.0013333558146428441f, 0.0013333558146428441f));
    p = fma2(p, f, pack2(0.009618129107628477f, 0.009618129107628477f));
    p = fma2(p, f, pack2(0.055504108664821576f, 0.055504108664821576f));
    p = fma2(p, f, pack2(0.2402265069591007f, 0.2402265069591007f));
    p = fma2(p, f, pack2(0.6931471805599453f, 0.6931471805599453f));
    p = fma2(p, f, pack2(1.0f, 1.0f));
    return make_uint2(weight_from(t0, n0, lo2(p)), weight_from(t1, n1, hi2(p)));
}

// legal entries of one cell for player p as bits 0..8 (entry k of the cell)
__device__ __forceinline__ uint32_t legal9(int own_p, int army, uint32_t terrain, bool moves) {
    if (!own_p) return 0u;
    uint32_t b = 1u;  // pass
    if (moves && army >= 2) {
        const uint32_t dirs = (terrain >> 2) & 0xFu;  // neighbour exists and is not a mountain
        b |= (dirs << 1) | (dirs << 5);
    }
    return b;
}

// shared memory of one warp's player, sized for boards up to npad_max cells:
// the player's own cells in index order (2 B), their legal bits (2 B) and
// weight sums (4 B), the weight sum of every 32 of them (8 B), mask staging
// (288 B); a multiple of 16 bytes.  The board (4 B per cell) comes first.
__host__ __device__ __forceinline__ int sample_player_bytes(int npad_max) {
    const int rounds = (npad_max + 31) >> 5;
    return 8 * npad_max + 8 * ((rounds + 1) & ~1) + 288;
}
__host__ __device__ __forceinline__ int sample_warp_bytes(int npad_max) {
    return 4 * npad_max + sample_player_bytes(npad_max);
}

// the nine logits of one cell, every load issued before any is used
__device__ __forceinline__ void load9(float (&v)[9], const float* x) {
#pragma unroll
    for (int k = 0; k < 9; ++k) v[k] = __ldcg(x + k);
}

__device__ __forceinline__ uint64_t warp_sum64(uint64_t x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kAll, x, o);
    return x;
}
__device__ __forceinline__ uint64_t warp_incl64(uint64_t x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(kAll, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}

// a game's board in shared memory, by `nthreads` threads from `tid` on
__device__ __forceinline__ void stage_board(const SArgs& a, const GameInfo& gi, char* b, int np, int tid, int nthreads) {
    const uint4* ga = reinterpret_cast<const uint4*>(a.army + gi.cell_off);
    const uint4* go = reinterpret_cast<const uint4*>(a.owner + gi.cell_off);
    const uint4* gt = reinterpret_cast<const uint4*>(a.terrain + gi.cell_off);
    uint4* sa = reinterpret_cast<uint4*>(b);
    uint4* so = reinterpret_cast<uint4*>(b + 2 * np);
    uint4* st = reinterpret_cast<uint4*>(b + 3 * np);
    const int n16 = gi.Npad >> 4;
    for (int v = tid; v < 2 * n16; v += nthreads) cp_async16(sa + v, ga + v);
    for (int v = tid; v < n16; v += nthreads) {
        cp_async16(so + v, go + v);
        cp_async16(st + v, gt + v);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// expanded mask rows r0 = row0, row0 + drow, ... (32 cells each) of every
// player: a cell's legal entries belong to its owner only
__device__ __forceinline__ void mask_rows(const SArgs& a, const GameInfo& gi, const GameScalars& sc,
                                          const int16_t* s_army, const int8_t* s_owner, const uint8_t* s_terrain,
                                          uint8_t* s_mask, int row0, int drow, int lane) {
    const int N = gi.N, Npad = gi.Npad, P = gi.P;
    for (int r0 = row0; r0 < Npad; r0 += drow) {
        const int cells = min(32, Npad - r0), c = r0 + lane;
        int o = -1;
        uint32_t lb = 0u;
        if (c < N) {
            o = s_owner[c];
            if (o >= 0) {
                const bool moves = ((sc.alive >> o) & 1u) && !sc.finished;
                lb = legal9(true, s_army[c], s_terrain[c], moves);
            }
        }
        const int n16 = (9 * cells) >> 4;
        for (int p = 0; p < P; ++p) {
            const uint32_t bits = o == p ? lb : 0u;
            if (lane < cells)
#pragma unroll
                for (int k = 0; k < 9; ++k) s_mask[9 * lane + k] = (uint8_t)((bits >> k) & 1u);
            __syncwarp();
            const int64_t base = (gi.plane_off + (int64_t)p * Npad) * 9;
            if (lane < n16)
                reinterpret_cast<uint4*>(a.mask9 + base + 9 * r0)[lane] = reinterpret_cast<const uint4*>(s_mask)[lane];
            __syncwarp();
        }
    }
}

// player p's action, by one warp over its region `w` of shared memory
__device__ __forceinline__ int32_t sample_player(const SArgs& a, const GameInfo& gi, const GameScalars& sc, int p,
                                                 const int16_t* s_army, const int8_t* s_owner,
                                                 const uint8_t* s_terrain, char* w, int lane) {
    const int np = a.npad_max, N = gi.N, Npad = gi.Npad;
    uint32_t* s_w = reinterpret_cast<uint32_t*>(w);                // [np] per own cell
    uint16_t* s_list = reinterpret_cast<uint16_t*>(w + 4 * np);    // [np] own cells
    uint16_t* s_legal = reinterpret_cast<uint16_t*>(w + 6 * np);   // [np] per own cell
    uint64_t* s_round = reinterpret_cast<uint64_t*>(w + 8 * np);   // [rounds]
    const unsigned lt_mask = (1u << lane) - 1u;
    const bool moves = ((sc.alive >> p) & 1u) && !sc.finished;
    const float* lg = a.logits + (gi.plane_off + (int64_t)p * Npad) * 9;
    // the player's cells in index order (legal entries lie only there)
    int n = 0;
    for (int r0 = 0; r0 < N; r0 += 32) {
        const int c = r0 + lane;
        const bool mine = c < N && s_owner[c] == p;
        const unsigned bal = __ballot_sync(kAll, mine);
        if (mine) s_list[n + __popc(bal & lt_mask)] = (uint16_t)c;
        n += __popc(bal);
    }
    __syncwarp();
    if (n == 0) return 0;
    // pass 1: legal bits and the maximum legal logit; the first two groups'
    // logits stay in registers for pass 2
    float m = -3.402823466e38f;
    float v0[9], v1[9];
    for (int i = lane; i < n; i += 32) {
        const int c = s_list[i];
        const uint32_t lb = legal9(true, s_army[c], s_terrain[c], moves);
        s_legal[i] = (uint16_t)lb;
        float v[9];
        load9(v, lg + 9 * c);
#pragma unroll
        for (int k = 0; k < 9; ++k)
            if ((lb >> k) & 1u) m = fmaxf(m, v[k]);
        if (i < 32) {
#pragma unroll
            for (int k = 0; k < 9; ++k) v0[k] = v[k];
        } else if (i < 64) {
#pragma unroll
            for (int k = 0; k < 9; ++k) v1[k] = v[k];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kAll, m, o));
    __syncwarp();
    // pass 2: weight sums per own cell and per 32 of them (every exponential once)
    uint64_t S = 0;
    for (int i0 = 0; i0 < n; i0 += 32) {
        const int i = i0 + lane;
        uint32_t wsum = 0u;
        if (i < n) {
            const int c = s_list[i];
            const uint32_t lb = s_legal[i];
            float v[9];
            if (i0 == 0) {
#pragma unroll
                for (int k = 0; k < 9; ++k) v[k] = v0[k];
            } else if (i0 == 32) {
#pragma unroll
                for (int k = 0; k < 9; ++k) v[k] = v1[k];
            } else {
                load9(v, lg + 9 * c);
            }
#pragma unroll
            for (int k = 0; k < 8; k += 2) {
                const uint2 w2 = weight_shift2(v[k], v[k + 1], m);
                wsum += ((lb >> k) & 1u) ? w2.x : 0u;
                wsum += ((lb >> (k + 1)) & 1u) ? w2.y : 0u;
            }
            if ((lb >> 8) & 1u) wsum += weight_shift(v[8], m);
            s_w[i] = wsum;
        }
        const uint64_t rs = warp_sum64(wsum);
        if (lane == 0) s_round[i0 >> 5] = rs;
        S += rs;
    }
    __syncwarp();
    const uint64_t d = stream_out(hkey(a.seed, gi.game_id, sc.frame, (uint64_t)p), 7);
    const uint64_t r = __umul64hi(d, S);
    // pass 3: the group of 32, then the cell, then the entry where the running sum first exceeds r
    const int groups = (n + 31) >> 5;
    uint64_t run = 0;
    int jr = -1;
    for (int j0 = 0; j0 < groups && jr < 0; j0 += 32) {
        const uint64_t rs = j0 + lane < groups ? s_round[j0 + lane] : 0u;
        const uint64_t incl = warp_incl64(rs, lane);
        const unsigned hit = __ballot_sync(kAll, run + incl > r);
        if (hit) {
            const int L = __ffs(hit) - 1;
            jr = j0 + L;
            run += __shfl_sync(kAll, incl - rs, L);
        } else {
            run += __shfl_sync(kAll, incl, 31);
        }
    }
    if (jr < 0) return 0;  // S = 0: only when every legal logit is -inf (outside the documented domain)
    const int i = 32 * jr + lane;
    const uint64_t wi = i < n ? s_w[i] : 0u;
    const uint64_t incl = warp_incl64(wi, lane);
    const unsigned hit = __ballot_sync(kAll, run + incl > r);
    const int L = __ffs(hit) - 1;
    // the entry inside the chosen cell: lanes 0..8 take one entry each
    const uint64_t before = run + __shfl_sync(kAll, incl - wi, L);
    const int cL = s_list[32 * jr + L];
    const uint32_t lbL = s_legal[32 * jr + L];
    uint64_t we = 0;
    if (lane < 9 && ((lbL >> lane) & 1u)) we = weight_shift(__ldcg(lg + 9 * cL + lane), m);
    const uint64_t ein = warp_incl64(we, lane);
    const unsigned ehit = __ballot_sync(kAll, lane < 9 && before + ein > r);
    return 9 * cL + (__ffs(ehit) - 1);
}

// one warp per game, players in turn
__global__ void __launch_bounds__(256) k_sample(const SArgs a, int warps_per_cta) {
    chain_entry();
    extern __shared__ __align__(16) char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int gidx = blockIdx.x * warps_per_cta + wid;
    if (gidx >= a.n_games) return;
    const int np = a.npad_max;
    char* b = smem + (size_t)wid * sample_warp_bytes(np);
    char* w = b + 4 * np;
    const GameInfo gi = a.info[gidx];
    const GameScalars sc = a.scal[gidx];
    stage_board(a, gi, b, np, lane, 32);
    __syncwarp();
    const int16_t* s_army = reinterpret_cast<const int16_t*>(b);
    const int8_t* s_owner = reinterpret_cast<const int8_t*>(b + 2 * np);
    const uint8_t* s_terrain = reinterpret_cast<const uint8_t*>(b + 3 * np);
    if (a.mask9)
        mask_rows(a, gi, sc, s_army, s_owner, s_terrain, reinterpret_cast<uint8_t*>(w + sample_player_bytes(np) - 288),
                  0, 32, lane);
    if (!a.logits) return;
    for (int p = 0; p < gi.P; ++p) {
        const int32_t action = sample_player(a, gi, sc, p, s_army, s_owner, s_terrain, w, lane);
        if (lane == 0 && a.actions) a.actions[gi.player_off + p] = action;
        __syncwarp();
    }
}

// one CTA per game (small batches): warp q takes players q, q + warps, ...
// and mask rows q, q + warps, ... over its own region of shared memory
__global__ void __launch_bounds__(256) k_sample_cta(const SArgs a) {
    chain_entry();
    extern __shared__ __align__(16) char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int gidx = blockIdx.x;  // the grid is one CTA per game
    const int np = a.npad_max;
    char* w = smem + 4 * np + (size_t)wid * sample_player_bytes(np);
    const GameInfo gi = a.info[gidx];
    const GameScalars sc = a.scal[gidx];
    stage_board(a, gi, smem, np, threadIdx.x, blockDim.x);
    __syncthreads();
    const int16_t* s_army = reinterpret_cast<const int16_t*>(smem);
    const int8_t* s_owner = reinterpret_cast<const int8_t*>(smem + 2 * np);
    const uint8_t* s_terrain = reinterpret_cast<const uint8_t*>(smem + 3 * np);
    if (a.mask9)
        mask_rows(a, gi, sc, s_army, s_owner, s_terrain, reinterpret_cast<uint8_t*>(w + sample_player_bytes(np) - 288),
                  32 * wid, 32 * nwarps, lane);
    if (!a.logits) return;
    for (int p = wid; p < gi.P; p += nwarps) {
        const int32_t action = sample_player(a, gi, sc, p, s_army, s_owner, s_terrain, w, lane);
        if (lane == 0 && a.actions) a.actions[gi.player_off + p] = action;
        __syncwarp();
    }
}

// ---- entry-parallel form (small batches) --------------------------------
// One CTA of kWideThreads threads per (game, player): the player's own cells
// are listed in index order by contiguous ranges of cells per thread and a
// block scan; then every (own cell, entry) pair gets a thread of its own,
// entry e of the list being entry e mod 9 of own cell e / 9 -- index order.
// Pass 1 loads each legal entry's logit once (the first kWideRegRounds
// rounds of the block stay in registers) and takes the block maximum; pass 2
// forms the integer weights and each warp's sum per round; one warp then
// sums them (S), draws r and finds the (round, warp) where the running sum
// first exceeds r; that warp scans its own 32 weights for the entry.  A
// game's chain is a few dependent steps instead of a warp's walk over its
// own cells, which is what sets the time when a launch fills less than a
// wave.
constexpr int kWideThreads = 128;
constexpr int kWideWarps = kWideThreads / 32;
constexpr int kWideRegRounds = 4;
constexpr float kNegInf = -__builtin_huge_valf();

__host__ __device__ __forceinline__ int wide_rounds(int npad_max) {
    return (9 * npad_max + kWideThreads - 1) / kWideThreads;
}
// board (4 B per cell), own-cell list and legal bits (2 + 2 B per cell),
// per-round warp sums (4 B each), block scratch, one mask staging row per warp
__host__ __device__ __forceinline__ int wide_bytes(int npad_max) {
    const int rw = (4 * wide_rounds(npad_max) * kWideWarps + 15) & ~15;
    return 8 * npad_max + rw + 64 + 288 * kWideWarps;
}

__global__ void __launch_bounds__(kWideThreads) k_sample_wide(const SArgs a, int pmax) {
    chain_entry();
    extern __shared__ __align__(16) char smem[];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int gidx = blockIdx.x / pmax, p = blockIdx.x - gidx * pmax;
    const GameInfo gi = a.info[gidx];
    if (p >= gi.P) return;
    const GameScalars sc = a.scal[gidx];
    const int np = a.npad_max, N = gi.N, Npad = gi.Npad;
    uint16_t* s_list = reinterpret_cast<uint16_t*>(smem + 4 * np);
    uint16_t* s_legal = reinterpret_cast<uint16_t*>(smem + 6 * np);
    uint32_t* s_ws = reinterpret_cast<uint32_t*>(smem + 8 * np);  // [round][warp]
    const int rw = (4 * wide_rounds(np) * kWideWarps + 15) & ~15;
    uint32_t* s_misc = reinterpret_cast<uint32_t*>(smem + 8 * np + rw);  // 16 words
    uint8_t* s_mask = reinterpret_cast<uint8_t*>(smem + 8 * np + rw + 64) + 288 * wid;
    stage_board(a, gi, smem, np, tid, kWideThreads);
    __syncthreads();
    const int16_t* s_army = reinterpret_cast<const int16_t*>(smem);
    const int8_t* s_owner = reinterpret_cast<const int8_t*>(smem + 2 * np);
    const uint8_t* s_terrain = reinterpret_cast<const uint8_t*>(smem + 3 * np);
    const bool moves = ((sc.alive >> p) & 1u) && !sc.finished;
    if (a.mask9) {  // player p's plane: rows of 32 cells, one warp each
        for (int r0 = 32 * wid; r0 < Npad; r0 += 32 * kWideWarps) {
            const int cells = min(32, Npad - r0), c = r0 + lane;
            const uint32_t bits =
                c < N && s_owner[c] == p ? legal9(true, s_army[c], s_terrain[c], moves) : 0u;
            if (lane < cells)
#pragma unroll
                for (int k = 0; k < 9; ++k) s_mask[9 * lane + k] = (uint8_t)((bits >> k) & 1u);
            __syncwarp();
            const int64_t base = (gi.plane_off + (int64_t)p * Npad) * 9;
            if (lane < ((9 * cells) >> 4))
                reinterpret_cast<uint4*>(a.mask9 + base + 9 * r0)[lane] = reinterpret_cast<const uint4*>(s_mask)[lane];
            __syncwarp();
        }
    }
    if (!a.logits) return;
    // the player's cells in index order: a contiguous range of cells per thread
    const int cpt = (N + kWideThreads - 1) / kWideThreads;
    const int c0 = min(N, tid * cpt), c1 = min(N, c0 + cpt);
    int cnt = 0;
    for (int c = c0; c < c1; ++c) cnt += s_owner[c] == p;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kAll, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_misc[wid] = (uint32_t)incl;
    __syncthreads();
    int before = incl - cnt, n = 0;
#pragma unroll
    for (int q = 0; q < kWideWarps; ++q) {
        const int t = (int)s_misc[q];
        if (q < wid) before += t;
        n += t;
    }
    for (int c = c0, i = before; c < c1; ++c)
        if (s_owner[c] == p) {
            s_list[i] = (uint16_t)c;
            s_legal[i] = (uint16_t)legal9(true, s_army[c], s_terrain[c], moves);
            ++i;
        }
    __syncthreads();  // the list is complete; s_misc free again
    if (n == 0) {
        if (tid == 0 && a.actions) a.actions[gi.player_off + p] = 0;
        return;
    }
    const float* lg = a.logits + (gi.plane_off + (int64_t)p * Npad) * 9;
    const int ne = 9 * n, rounds = (ne + kWideThreads - 1) / kWideThreads;
    // entry e of the list: its logit if legal, else -inf
    auto logit_of = [&](int e) -> float {
        if (e >= ne) return kNegInf;
        const int i = e / 9, k = e - 9 * i;
        if (!((s_legal[i] >> k) & 1u)) return kNegInf;
        return __ldcg(lg + 9 * (int)s_list[i] + k);
    };
    // pass 1: the maximum legal logit
    float v[kWideRegRounds];
    float m = kNegInf;
#pragma unroll
    for (int j = 0; j < kWideRegRounds; ++j) {
        v[j] = j < rounds ? logit_of(tid + kWideThreads * j) : kNegInf;
        m = fmaxf(m, v[j]);
    }
    for (int j = kWideRegRounds; j < rounds; ++j) m = fmaxf(m, logit_of(tid + kWideThreads * j));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kAll, m, o));
    if (lane == 0) s_misc[wid] = __float_as_uint(m);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kWideWarps; ++q) m = fmaxf(m, __uint_as_float(s_misc[q]));
    // pass 2: integer weights (0 for illegal entries) and each warp's sum per round
    auto weight_of = [&](float x) -> uint32_t { return x == kNegInf ? 0u : weight_shift(x, m); };
    uint32_t w[kWideRegRounds];
#pragma unroll
    for (int j = 0; j < kWideRegRounds; ++j) {
        w[j] = weight_of(v[j]);
        if (j < rounds) {
            const uint32_t ws = __reduce_add_sync(kAll, w[j]);  // at most 32 * 2^24
            if (lane == 0) s_ws[j * kWideWarps + wid] = ws;
        }
    }
    for (int j = kWideRegRounds; j < rounds; ++j) {
        const uint32_t ws = __reduce_add_sync(kAll, weight_of(logit_of(tid + kWideThreads * j)));
        if (lane == 0) s_ws[j * kWideWarps + wid] = ws;
    }
    __syncthreads();
    // one warp: S, r, then the (round, warp) slot where the running sum first exceeds r
    if (wid == 0) {
        const int slots = rounds * kWideWarps;
        uint64_t S = 0;
        for (int t = lane; t < slots; t += 32) S += s_ws[t];
        S = warp_sum64(S);
        const uint64_t d = stream_out(hkey(a.seed, gi.game_id, sc.frame, (uint64_t)p), 7);
        const uint64_t r = __umul64hi(d, S);
        uint64_t run = 0;
        int found = -1;
        for (int t0 = 0; t0 < slots && found < 0; t0 += 32) {
            const uint64_t x = t0 + lane < slots ? s_ws[t0 + lane] : 0u;
            const uint64_t inc = warp_incl64(x, lane);
            const unsigned hit = __ballot_sync(kAll, run + inc > r);
            if (hit) {
                const int L = __ffs(hit) - 1;
                found = t0 + L;
                run += __shfl_sync(kAll, inc - x, L);
            } else {
                run += __shfl_sync(kAll, inc, 31);
            }
        }
        if (lane == 0) {
            s_misc[8] = (uint32_t)found;
            s_misc[10] = (uint32_t)run;
            s_misc[11] = (uint32_t)(run >> 32);
            s_misc[12] = (uint32_t)r;
            s_misc[13] = (uint32_t)(r >> 32);
        }
    }
    __syncthreads();
    const int found = (int)s_misc[8];
    if (found < 0) {  // S = 0: only when every legal logit is -inf (outside the documented domain)
        if (tid == 0 && a.actions) a.actions[gi.player_off + p] = 0;
        return;
    }
    const int jf = found / kWideWarps;
    if (wid != found - jf * kWideWarps) return;
    const uint64_t run = s_misc[10] | ((uint64_t)s_misc[11] << 32);
    const uint64_t r = s_misc[12] | ((uint64_t)s_misc[13] << 32);
    uint32_t wj = 0u;
#pragma unroll
    for (int j = 0; j < kWideRegRounds; ++j)
        if (j == jf) wj = w[j];
    if (jf >= kWideRegRounds) wj = weight_of(logit_of(tid + kWideThreads * jf));
    uint32_t inc = wj;  // at most 32 * 2^24: no overflow
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kAll, inc, o);
        if (lane >= o) inc += y;
    }
    const unsigned hit = __ballot_sync(kAll, run + inc > r);
    if (lane == __ffs(hit) - 1 && a.actions) {
        const int e = tid + kWideThreads * jf, i = e / 9;
        a.actions[gi.player_off + p] = 9 * (int)s_list[i] + (e - 9 * i);
    }
}

}  // namespace

int launch_sample(const SArgs& a, int pmax, int form, void* stream) {
    if (a.n_games <= 0) return 0;
    // by default a CTA per player with a thread per entry while the players
    // fill at most about one wave of those CTAs, else a CTA per game
    // (measured on 24x24 1v1 at mid-game: 512 games 6.1 against 7.8 us,
    // 1,024 games 9.8 against 8.8 us; from 2,048 games on the CTA per game
    // is the fastest form)
    if (form == 0) {
        static std::atomic<int> sm_count{0};  // of the first device used: only the form depends on it
        int sms = sm_count.load(std::memory_order_relaxed);
        if (sms == 0) {
            int dev = 0, n = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
            sms = n > 0 ? n : 1;
            sm_count.store(sms, std::memory_order_relaxed);
        }
        form = (int64_t)a.n_games * pmax <= 8 * (int64_t)sms ? 3 : 2;
    }
    if (form == 3) {
        const int smem = wide_bytes(a.npad_max);
        static SmemLimit limit;
        const void* fn = (const void*)k_sample_wide;
        const int e = limit.raise(&fn, 1, smem);
        if (e != 0) return e;
        return launch_chained(k_sample_wide, dim3((unsigned)((int64_t)a.n_games * pmax)), dim3(kWideThreads), smem,
                              (cudaStream_t)stream, a, pmax);
    }
    if (form == 2) {
        // a warp per player, as many as fit next to the board (at least one)
        const int fit = (227 * 1024 - 4 * a.npad_max) / sample_player_bytes(a.npad_max);
        const int warps = std::max(1, std::min(std::min(pmax, kWarps), fit));
        const int smem = 4 * a.npad_max + warps * sample_player_bytes(a.npad_max);
        static SmemLimit limit;
        const void* fn = (const void*)k_sample_cta;
        const int e = limit.raise(&fn, 1, smem);
        if (e != 0) return e;
        return launch_chained(k_sample_cta, dim3(a.n_games), dim3(32 * warps), smem, (cudaStream_t)stream, a);
    }
    const int per_warp = sample_warp_bytes(a.npad_max);
    const int wpc = std::max(1, std::min(kWarps, (200 * 1024) / per_warp));
    const int smem = wpc * per_warp;
    static SmemLimit limit;
    const void* fn = (const void*)k_sample;
    const int e = limit.raise(&fn, 1, smem);
    if (e != 0) return e;
    const int blocks = (a.n_games + wpc - 1) / wpc;
    return launch_chained(k_sample, dim3(blocks), dim3(32 * wpc), smem, (cudaStream_t)stream, a, wpc);
}

}  // namespace gk
