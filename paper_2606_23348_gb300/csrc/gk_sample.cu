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
// One warp per game, players in turn, 32 cells per round with the round's
// 288 logits staged in shared memory by 16-byte loads: pass 1 derives each
// cell's nine legal bits once (and writes the expanded mask) and takes the
// maximum; pass 2 (from L2) sums each cell's weights, computing every
// exponential once; pass 3 scans the per-cell sums in shared memory and
// resolves the entry inside the chosen cell.  Rounds without a legal entry
// read no logits.  HBM-bound at most 36 bytes of logits per cell (plus 9 mask
// bytes when the expanded mask is written).
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

// shared memory of one warp, sized for boards up to npad_max cells
__host__ __device__ __forceinline__ int sample_warp_bytes(int npad_max) {
    return 4 * npad_max + 2 * npad_max + 4 * 288 + 288;  // weights, legal bits, logits and mask staging
}

// warp copy of `cells` cells x 9 logits (a multiple of 144 floats) to shared memory
__device__ __forceinline__ void stage_logits(float* dst, const float* src, int cells, int lane) {
    const int n4 = (9 * cells) >> 2;
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (int v = lane; v < n4; v += 32) d4[v] = __ldcg(s4 + v);
    __syncwarp();
}

__global__ void __launch_bounds__(256) k_sample(const SArgs a) {
    extern __shared__ __align__(16) char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int gidx = blockIdx.x * kWarps + wid;
    if (gidx >= a.n_games) return;
    char* base_s = smem + (size_t)wid * sample_warp_bytes(a.npad_max);
    uint32_t* s_w = reinterpret_cast<uint32_t*>(base_s);                              // [npad_max]
    float* s_stage = reinterpret_cast<float*>(base_s + 4 * a.npad_max);               // [288]
    uint16_t* s_legal = reinterpret_cast<uint16_t*>(base_s + 4 * a.npad_max + 1152);  // [npad_max]
    uint8_t* s_mask = reinterpret_cast<uint8_t*>(base_s + 6 * a.npad_max + 1152);     // [288]

    const GameInfo gi = a.info[gidx];
    const GameScalars sc = a.scal[gidx];
    const int N = gi.N, Npad = gi.Npad;
    const int16_t* army = a.army + gi.cell_off;
    const int8_t* owner = a.owner + gi.cell_off;
    const int8_t* terrain = a.terrain + gi.cell_off;
    for (int p = 0; p < gi.P; ++p) {
        const bool moves = ((sc.alive >> p) & 1u) && !sc.finished;
        const int64_t base = (gi.plane_off + (int64_t)p * Npad) * 9;
        const float* lg = a.logits ? a.logits + base : nullptr;

        // pass 1: legal bits per cell, the expanded mask, the maximum legal logit
        float m = -3.402823466e38f;
        bool any_all = false;
        for (int r0 = 0; r0 < Npad; r0 += 32) {
            const int cells = min(32, Npad - r0);
            const int c = r0 + lane;
            uint32_t lb = 0u;
            if (c < N) lb = legal9(owner[c] == p, army[c], (uint32_t)(uint8_t)terrain[c], moves);
            if (c < Npad) s_legal[c] = (uint16_t)lb;
            if (a.mask9) {
                if (lane < cells)
#pragma unroll
                    for (int k = 0; k < 9; ++k) s_mask[9 * lane + k] = (uint8_t)((lb >> k) & 1u);
                __syncwarp();
                const int n16 = (9 * cells) >> 4;
                if (lane < n16)
                    reinterpret_cast<uint4*>(a.mask9 + base + 9 * r0)[lane] = reinterpret_cast<const uint4*>(s_mask)[lane];
                __syncwarp();
            }
            const bool any = __any_sync(kAll, lb != 0u);
            if (!lg || !any) continue;
            any_all = true;
            stage_logits(s_stage, lg + 9 * r0, cells, lane);
#pragma unroll
            for (int k = 0; k < 9; ++k)
                if ((lb >> k) & 1u) m = fmaxf(m, s_stage[9 * lane + k]);
            __syncwarp();
        }
        if (!lg) continue;
        int32_t action = 0;
        if (any_all) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kAll, m, o));
            // pass 2: weight of each cell (sum of its legal entries' weights), exact total
            uint64_t S = 0;
            for (int r0 = 0; r0 < Npad; r0 += 32) {
                const int cells = min(32, Npad - r0);
                const int c = r0 + lane;
                const uint32_t lb = c < Npad ? s_legal[c] : 0u;
                uint32_t w = 0u;
                if (__any_sync(kAll, lb != 0u)) {
                    stage_logits(s_stage, lg + 9 * r0, cells, lane);
#pragma unroll
                    for (int k = 0; k < 9; ++k)
                        if ((lb >> k) & 1u) w += weight_shift(s_stage[9 * lane + k], m);
                    __syncwarp();
                }
                if (c < Npad) s_w[c] = w;
                S += w;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) S += __shfl_xor_sync(kAll, S, o);
            __syncwarp();
            const uint64_t d = stream_out(hkey(a.seed, gi.game_id, sc.frame, (uint64_t)p), 7);
            const uint64_t r = __umul64hi(d, S);
            // pass 3: the cell whose running weight sum first exceeds r, then the entry within it
            uint64_t run = 0;
            for (int r0 = 0; r0 < Npad; r0 += 32) {
                const int c = r0 + lane;
                const uint64_t w = c < Npad ? s_w[c] : 0u;
                uint64_t incl = w;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint64_t y = __shfl_up_sync(kAll, incl, o);
                    if (lane >= o) incl += y;
                }
                const unsigned hit = __ballot_sync(kAll, run + incl > r);
                if (hit) {
                    const int L = __ffs(hit) - 1;
                    int pick = 0;
                    if (lane == L) {
                        uint64_t acc = run + (incl - w);
                        const uint32_t lb = s_legal[c];
                        for (int k = 0; k < 9; ++k) {
                            if (!((lb >> k) & 1u)) continue;
                            acc += weight_shift(__ldcg(lg + 9 * c + k), m);
                            if (acc > r) {
                                pick = 9 * c + k;
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
        __syncwarp();
    }
}

}  // namespace

int launch_sample(const SArgs& a, void* stream) {
    if (a.n_games <= 0) return 0;
    const int smem = kWarps * sample_warp_bytes(a.npad_max);
    static int configured = 48 * 1024;
    if (smem > configured) {
        const cudaError_t e = cudaFuncSetAttribute(k_sample, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return (int)e;
        configured = smem;
    }
    const int blocks = (a.n_games + kWarps - 1) / kWarps;
    k_sample<<<blocks, 32 * kWarps, smem, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

}  // namespace gk
