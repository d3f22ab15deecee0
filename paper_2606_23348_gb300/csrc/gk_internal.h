// Internal structures shared by the kernels and the C-ABI layer of
// libgenerals.  Not part of the public interface (include/generals.h).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <mutex>

namespace gk {

constexpr int kMaxPlayers = 8;
constexpr int kMaxSide = 64;
constexpr int kGenAttempts = 64;  // rejection attempts per level (generator)

enum Op : int32_t {
    OP_CREATE = 0,   // epoch 0 map, counters cleared, outputs
    OP_RESET = 1,    // next epoch map, outputs
    OP_OBSERVE = 2,  // outputs only
    OP_STEP = 3,     // full step, outputs
    OP_POLICY = 4,   // benchmark policy only
    OP_DERIVE = 5,   // recompute cached per-map bits after a state upload
};

// Read-only description of one game (48 bytes).
struct alignas(16) GameInfo {
    int64_t plane_off;   // first cell of player 0's plane in every per-player output plane
    uint64_t game_id;    // global id keying the game's maps and policy draws
    int32_t cell_off;    // first cell in the state arenas
    int32_t player_off;  // first per-player slot (actions, reward, scoreboard)
    int16_t H, W;
    int16_t N, Npad;     // cells, cells rounded up to 16
    int8_t mode, P;
    int16_t n_cities;
    int16_t dmin;        // Manhattan spacing of generals
    int16_t pad0;
    int32_t pad1[2];
};
static_assert(sizeof(GameInfo) == 48, "GameInfo is 48 bytes");

// Mutable per-game scalars (32 bytes), one row of gen_read_state's h_scalars.
struct alignas(16) GameScalars {
    uint32_t turn, frame, epoch, alive, finished, invalid, saturated, err;
};
static_assert(sizeof(GameScalars) == 32, "GameScalars is 32 bytes");

struct KArgs {
    const GameInfo* info;
    const int32_t* list;  // optional list of local game ids, else item i = game i
    int32_t n_items;
    int32_t n_games;    // list entries outside [0, n_games) are skipped
    int32_t op;
    int16_t* army;
    int8_t* owner;
    int8_t* terrain;
    GameScalars* scal;
    const int32_t* actions;
    int16_t* obs_army;
    int8_t* obs_owner;
    int8_t* obs_terrain;
    uint8_t* obs_vis;
    uint8_t* mask;
    float* reward;
    int32_t* scoreboard;
    uint8_t* done;
    int32_t* next_actions;  // non-null: fused benchmark policy
    // multi-frame rollouts: frame f writes its outputs at base + f * stride
    int32_t frames;         // frames per launch (state stays in shared memory)
    int64_t plane_stride;   // elements of one frame of a per-player plane
    int32_t slot_stride;    // per-player slots of one frame (reward, actions log)
    int32_t game_stride;    // games of one frame (done)
    int32_t* action_log;    // optional [frames][slots]: actions each frame consumed
    // uniform batch: every game has ushape's board and mode; game g sits at
    // cell g * Npad, plane cell g * P * Npad, slot g * P, global id base + g
    int32_t uniform;
    GameInfo ushape;
    uint64_t policy_seed;
    uint64_t seed;
    uint64_t game_id_base;
    uint32_t mtn_thresh;
    int32_t city_min, city_span;
    int32_t max_turns;
    int32_t auto_reset;
    int32_t do_outputs;
    // shared-memory carve of one warp (one game)
    int32_t npad_max;   // cells
    int32_t nw_stride;  // 32-bit words per bitset
    int32_t pmax;
    int32_t warp_smem;  // bytes per warp (a warp per game; launches of narrower groups recompute it)
    // spawn options of the map generator (all zero: the plain generator)
    int32_t spawn_dmax;     // cap on a general's distance to every earlier one (0: none)
    int32_t spawn_bfs;      // 1: spacing in BFS steps around mountains
    int32_t castle_radius;  // > 0: a neutral castle within this many steps of every general
    // games per warp: 0 by batch size, 1 a warp per game, 2 two or four per
    // warp whenever the games allow (two players, small boards, no spawn options)
    int32_t lane_groups;
};

// Programmatic dependent launch.  Every kernel of the library is launched
// with launch_chained(), which lets the GPU place it while the kernel before
// it on the stream is still running, and begins with chain_entry():
// griddepcontrol.wait returns once that kernel has completed and its writes
// are visible (at once after an ordinary launch, a copy or an event), so no
// global memory is touched before it.  The kernels issue no early
// launch_dependents: a kernel's successor is placed as its CTAs exit, which
// hides the launch gap between dependent kernels of a stream (measured on the
// 512-game sample -> step -> features loop: 45.2 -> 38.4 us per frame with
// plain launches; triggering at kernel entry instead slowed the same loop
// inside a CUDA graph from 43.5 to 48.7 us).
__device__ __forceinline__ void chain_entry() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KP, typename... A>
inline int launch_chained(void (*k)(KP...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A&&... args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return (int)cudaLaunchKernelEx(&cfg, k, static_cast<A&&>(args)...);
}

// Dynamic shared memory above 48 KiB needs a per-kernel opt-in on each
// device.  raise() lifts the limit of n kernels to `want` bytes on the current
// device the first time a launch needs it; limits only grow, so launches
// sized earlier stay legal.  Thread-safe.  Returns a cudaError_t.
struct SmemLimit {
    std::mutex mu;
    int bytes[64] = {};
    int raise(const void* const* fns, int n, int want) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return (int)e;
        if (dev < 0 || dev >= 64) return (int)cudaErrorInvalidDevice;
        std::lock_guard<std::mutex> lk(mu);
        if (want <= 48 * 1024 || want <= bytes[dev]) return 0;
        for (int i = 0; i < n && e == cudaSuccess; ++i)
            e = cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, want);
        if (e != cudaSuccess) return (int)e;
        bytes[dev] = want;
        return 0;
    }
};

// Feature-tensor builder (App. A): one warp per game, players in turn.
struct FArgs {
    const GameInfo* info;
    const int16_t* army;
    const int8_t* owner;
    const int8_t* terrain;
    const GameScalars* scal;
    int32_t n_games;
    int32_t hist;          // delta history length K: channels 24 + 2K
    int64_t plane_cells;   // cells of the per-player plane set
    uint4* hdr;            // per player slot: epoch + 1 folded (0: none), frame folded, frames folded this episode
    uint8_t* mem_bits;     // per plane cell: bit 0 seen, 1 enemy seen, 2 general, 3 castle, 4 mountain
    int16_t* mem_army;     // per plane cell: last enemy army seen
    int32_t* mem_turn;     // per plane cell: turn an enemy was last seen
    int16_t* ring;         // [(K + 1) * 2][plane_cells]: own / enemy army planes of folded frames
    float* out;            // player plane q = plane_off + p * Npad: channel ch of cell c at q * C + ch * Npad + c
    int32_t npad_max;      // largest board (cells, multiple of 16)
    int32_t window;        // temporal-token window T (0: none)
    int2* series_ring;     // [slot][T]: (opponents' army, land), entry (n - 1) mod T = the n-th folded frame
    int2* series_out;      // optional [slot][T]: newest first, 0 before the episode
};

// Launch the feature builder over every game on `stream`: form 1 one warp
// per game, 2 one CTA per game, 0 by batch size.  pmax = the most players of
// any game.  Returns a cudaError_t.
int launch_features(const FArgs& f, int pmax, int form, void* stream);

// Policy sampling over the H x W x 9 action space: one warp per game.
struct SArgs {
    const GameInfo* info;
    const int16_t* army;
    const int8_t* owner;
    const int8_t* terrain;  // type | passable-neighbour bits << 2
    const GameScalars* scal;
    int32_t n_games;
    const float* logits;    // player plane q: 9 * Npad floats at q * 9 (NULL: mask only)
    uint64_t seed;
    int32_t* actions;       // [player slots] (NULL with logits NULL)
    uint8_t* mask9;         // optional: 9 * Npad legal-entry bytes per player plane at q * 9
    int32_t npad_max;       // largest board (cells, multiple of 16)
};

// Launch the sampler over every game on `stream`: form 1 one warp per game,
// 2 (and 0, the default) one CTA per game with a warp per player.  pmax = the most
// players of any game.  Returns a cudaError_t.
int launch_sample(const SArgs& a, int pmax, int form, void* stream);

// Bytes of shared memory one lane group needs for games up to npad_max
// cells and pmax players; also returns the bitset stride in words.  narrow:
// a group narrower than a warp (its legal moves kept as per-chunk masks).
int warp_smem_bytes(int npad_max, int pmax, int* nw_stride, bool narrow = false);

// CTAs of the step kernel that fit on the whole GPU at once (raises the
// kernel's shared-memory limit as a side effect).  Returns a cudaError_t.
int max_resident_ctas(int warps_per_cta, int smem_bytes, int* out);

// ---- work-list launch: every size bucket of a ragged batch in one launch --
// One item: `count` games of one bucket, entries first .. first+count-1 of
// the environment's game order (largest boards first).
struct WorkItem {
    int32_t first, count, bucket, pad;
};
// A bucket's shared-memory geometry (packed as the kernels' carve expects),
// bytes per lane group and lane-group width (16: two games per warp, 32).
struct BucketGeom {
    uint32_t geom;
    int32_t group_smem;
    int32_t lw;
    int32_t pad;
};
struct WArgs {
    const WorkItem* items;
    int32_t n_items;
    const BucketGeom* geoms;
    const int32_t* order;
    int32_t* counter;  // [0] next item, [1] CTAs done; the last CTA done zeroes both (zero when allocated)
};
// Packed geometry word of a bucket (as the kernels unpack it).
uint32_t bucket_geom(int npad_max, int nw_stride, int pmax, bool narrow);
// Dynamic shared memory per CTA and CTAs of the whole GPU for the work-list
// kernel (`multi`: multi-frame form).  Returns a cudaError_t.
int worklist_shape(bool multi, int* cta_smem, int* ctas);
// Zero the item counter, then one persistent launch of `ctas` CTAs that
// take items until the list is done.  Returns a cudaError_t.
int launch_worklist(const KArgs& a, const WArgs& w, int cta_smem, int ctas, void* stream);

// Launch the step kernel with `warps_per_cta` games per CTA on `stream`.
// Returns a cudaError_t value.
int launch_step(const KArgs& a, int warps_per_cta, int max_ctas, void* stream);

// Fill the device's constant tables (board column masks); once per device,
// synchronous.  Returns a cudaError_t value.
int init_tables();

// 128-bit copy kernel used to measure the HBM roofline denominator.
int launch_copy(const void* src, void* dst, size_t n16, int blocks, void* stream);

}  // namespace gk
