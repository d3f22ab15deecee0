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
// One warp per game, players in turn; three passes over the player's logits
// (maximum with the mask, weight sum, selection by a warp scan per 128
// entries), the second and third from L2.  HBM-bound: 36 bytes of logits per
// cell (plus 9 mask bytes when the expanded mask is written).
#include <cuda_runtime.h>

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

// the reproducible exponential (see the file comment)
__device__ __forceinline__ float exp_r(float x) {
    const float t = __fmul_rn(x, 1.4426950408889634f);
    if (t < -25.0f) return 0.0f;
    const float n = floorf(t);
    const float f = __fsub_rn(t, n);
    float p = 1.5252733804059838e-05f;
    p = __fmaf_rn(p, f, 0.00015403530393381606f);
    p = __fmaf_rn(p, f, 0.0013333558146428441f);
    p = __fmaf_rn(p, f, 0.009618129107628477f);
    p = __fmaf_rn(p, f, 0.055504108664821576f);
    p = __fmaf_rn(p, f, 0.2402265069591007f);
    p = __fmaf_rn(p, f, 0.6931471805599453f);
    p = __fmaf_rn(p, f, 1.0f);
    return __fmul_rn(p, __int_as_float((127 + (int)n) << 23));  // exact: n >= -25
}
__device__ __forceinline__ uint32_t weight(float l, float m) {
    return (uint32_t)floorf(__fmul_rn(exp_r(__fsub_rn(l, m)), 16777216.0f));
}

struct Player {
    const int16_t* army;
    const int8_t* owner;
    const int8_t* terrain;
    int N, p;
    bool moves;  // alive and the game not finished
};

// legality of the four entries e0 .. e0 + 3 as bits 0..3
__device__ __forceinline__ uint32_t legal4(const Player& q, int e0) {
    uint32_t bits = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int e = e0 + i;
        const int c = e / 9, k = e - 9 * c;
        if (c >= q.N) continue;
        const bool own = q.owner[c] == q.p;
        bool ok;
        if (k == 0)
            ok = own;
        else
            ok = q.moves && own && q.army[c] >= 2 && ((q.terrain[c] >> (2 + ((k - 1) & 3))) & 1);
        bits |= (ok ? 1u : 0u) << i;
    }
    return bits;
}

__global__ void __launch_bounds__(256) k_sample(const SArgs a) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int gidx = blockIdx.x * kWarps + wid;
    if (gidx >= a.n_games) return;
    const GameInfo gi = a.info[gidx];
    const GameScalars sc = a.scal[gidx];
    const int N = gi.N, Npad = gi.Npad;
    const int E = 9 * Npad;  // entries of one player plane (a multiple of 4)
    for (int p = 0; p < gi.P; ++p) {
        Player q;
        q.army = a.army + gi.cell_off;
        q.owner = a.owner + gi.cell_off;
        q.terrain = a.terrain + gi.cell_off;
        q.N = N;
        q.p = p;
        q.moves = ((sc.alive >> p) & 1u) && !sc.finished;
        const int64_t base = (gi.plane_off + (int64_t)p * Npad) * 9;
        const float* lg = a.logits ? a.logits + base : nullptr;

        // pass 1: legal mask (written when asked) and the maximum legal logit
        float m = -3.402823466e38f;
        bool any = false;
        for (int e0 = 4 * lane; e0 < E; e0 += 128) {
            const uint32_t bits = legal4(q, e0);
            if (a.mask9)
                *reinterpret_cast<uchar4*>(a.mask9 + base + e0) =
                    make_uchar4(bits & 1u, (bits >> 1) & 1u, (bits >> 2) & 1u, (bits >> 3) & 1u);
            if (lg && bits) {
                const float4 v = __ldg(reinterpret_cast<const float4*>(lg + e0));
                if (bits & 1u) m = fmaxf(m, v.x);
                if (bits & 2u) m = fmaxf(m, v.y);
                if (bits & 4u) m = fmaxf(m, v.z);
                if (bits & 8u) m = fmaxf(m, v.w);
                any = true;
            }
        }
        if (!lg) continue;
        any = __any_sync(kAll, any);
        int32_t action = 0;
        if (any) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kAll, m, o));
            // pass 2: the exact sum of the weights
            uint64_t S = 0;
            for (int e0 = 4 * lane; e0 < E; e0 += 128) {
                const uint32_t bits = legal4(q, e0);
                if (!bits) continue;
                const float4 v = *reinterpret_cast<const float4*>(lg + e0);
                if (bits & 1u) S += weight(v.x, m);
                if (bits & 2u) S += weight(v.y, m);
                if (bits & 4u) S += weight(v.z, m);
                if (bits & 8u) S += weight(v.w, m);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) S += __shfl_xor_sync(kAll, S, o);
            const uint64_t d = stream_out(hkey(a.seed, gi.game_id, sc.frame, (uint64_t)p), 7);
            const uint64_t r = __umul64hi(d, S);
            // pass 3: first entry whose running weight sum exceeds r, 128 entries per round
            uint64_t run = 0;
            for (int r0 = 0; r0 < E; r0 += 128) {
                const int e0 = r0 + 4 * lane;
                uint32_t w[4] = {0u, 0u, 0u, 0u};
                if (e0 < E) {
                    const uint32_t bits = legal4(q, e0);
                    if (bits) {
                        const float4 v = *reinterpret_cast<const float4*>(lg + e0);
                        if (bits & 1u) w[0] = weight(v.x, m);
                        if (bits & 2u) w[1] = weight(v.y, m);
                        if (bits & 4u) w[2] = weight(v.z, m);
                        if (bits & 8u) w[3] = weight(v.w, m);
                    }
                }
                const uint32_t mine = w[0] + w[1] + w[2] + w[3];  // <= 2^26
                uint32_t incl = mine;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(kAll, incl, o);
                    if (lane >= o) incl += y;
                }
                const unsigned hit = __ballot_sync(kAll, run + incl > r);
                if (hit) {
                    const int L = __ffs(hit) - 1;
                    int pick = 0;
                    if (lane == L) {
                        uint64_t acc = run + (incl - mine);
                        for (int i = 0; i < 4; ++i) {
                            acc += w[i];
                            if (acc > r) {
                                pick = e0 + i;
                                break;
                            }
                        }
                    }
                    action = __shfl_sync(kAll, pick, L);
                    break;
                }
                run += __shfl_sync(kAll, incl, 31);
            }
        }
        if (lane == 0 && a.actions) a.actions[gi.player_off + p] = action;
    }
}

}  // namespace

int launch_sample(const SArgs& a, void* stream) {
    if (a.n_games <= 0) return 0;
    const int blocks = (a.n_games + kWarps - 1) / kWarps;
    k_sample<<<blocks, 32 * kWarps, 0, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

}  // namespace gk
