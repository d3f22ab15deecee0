// C-ABI of libgenerals (declared in include/generals.h): argument checks,
// device arenas, per-game layout, size buckets, launches, rollouts (plain,
// resident, CUDA graph) and the launch-shape autotuner.  All game work runs
// in the kernels of gk_kernels.cu; this file never computes a rule.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "generals.h"
#include "gk_internal.h"

using gk::GameInfo;
using gk::GameScalars;
using gk::KArgs;

namespace {

thread_local char g_err[512] = "no error";

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(GEN_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define CUDA_TRY(expr, what)                               \
    do {                                                   \
        cudaError_t e_ = (expr);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

constexpr int kMaxSmemPerCta = 227 * 1024;

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
bool aligned4(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 3u) == 0; }

// A group of games of similar size launched together with its own
// shared-memory carve and launch shape.
struct Bucket {
    int offset = 0;   // first entry in the env's game order
    int n = 0;        // games
    int npad_max = 0;
    int pmax = 0;
    int nw_stride = 0;
    int warp_smem = 0;
    int warps = 8;    // games (warps) per CTA
    bool tuned = false;  // warps set by gen_set_launch or the autotuner; else chosen per launch by occupancy
    int max_ctas = 0;
};

// process-wide cache of autotuned launch shapes: (cell class, player class, SMs) -> warps
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, int> g_tune_cache;

}  // namespace

struct gen_env {
    int G = 0;
    gen_params prm{};
    std::vector<GameInfo> h_info;
    int64_t plane_cells = 0;
    int64_t state_cells = 0;
    int player_slots = 0;
    int pmax = 0;
    int npad_max = 0;
    int sample_form = 0;  // gen_sample_actions: 1 a warp per game, 2 a CTA per game, 3 a CTA per player, 0 by batch size
    int rollout_form = GEN_ROLLOUT_RESIDENT;  // what GEN_ROLLOUT_AUTO runs (the autotuner's pick)
    int lane_groups = 0;  // step kernels: 0 by batch size, 1 a warp per game, 2 several per warp when allowed
    int nmax = 0;
    bool uniform = false;            // every game has the same board size and mode
    Bucket all;                      // every game, largest carve (used for game-id lists)
    std::vector<Bucket> buckets;     // size buckets covering every game once
    int32_t* d_order = nullptr;      // games sorted by bucket (NULL: identity, one bucket)
    std::vector<cudaStream_t> side;  // one per bucket beyond the first
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    GameInfo* d_info = nullptr;
    GameScalars* d_scal = nullptr;
    int16_t* d_army = nullptr;
    int8_t* d_owner = nullptr;
    int8_t* d_terrain = nullptr;
    // staging for gen_step_host
    int32_t* d_actions = nullptr;
    gen_outputs d_out{};
    bool have_out = false;
    // gen_step_host pipeline: game ids 0..G-1, a copy stream, one event per chunk
    int32_t* d_iota = nullptr;
    cudaStream_t copy = nullptr;
    cudaEvent_t chunk_ev[8] = {};
    cudaEvent_t copy_done = nullptr;
    // cached rollout graph
    cudaGraphExec_t graph = nullptr;
    std::vector<const void*> graph_key;
    size_t dev_bytes = 0;  // device memory this environment holds (gen_device_bytes)
    // work-list form: every bucket in one launch ([0] per frame, [1] multi-frame)
    int batch_form = 0;  // 0 auto, 1 one launch per bucket, 2 one work-list launch
    gk::BucketGeom* d_geoms = nullptr;
    gk::WorkItem* d_items[2] = {};
    int32_t* d_counter = nullptr;
    int wl_items[2] = {}, wl_smem[2] = {}, wl_ctas[2] = {};
};

namespace {

void free_env(gen_env* e) {
    if (!e) return;
    if (e->graph) cudaGraphExecDestroy(e->graph);
    e->graph = nullptr;
    for (auto s : e->side) cudaStreamDestroy(s);
    for (auto v : e->join) cudaEventDestroy(v);
    if (e->fork) cudaEventDestroy(e->fork);
    cudaFree(e->d_order);
    cudaFree(e->d_info);
    cudaFree(e->d_scal);
    cudaFree(e->d_army);
    cudaFree(e->d_owner);
    cudaFree(e->d_terrain);
    cudaFree(e->d_actions);
    cudaFree(e->d_iota);
    cudaFree(e->d_geoms);
    cudaFree(e->d_items[0]);
    cudaFree(e->d_items[1]);
    cudaFree(e->d_counter);
    if (e->copy) cudaStreamDestroy(e->copy);
    for (auto v : e->chunk_ev)
        if (v) cudaEventDestroy(v);
    if (e->copy_done) cudaEventDestroy(e->copy_done);
    if (e->have_out) {
        cudaFree(e->d_out.obs_army);
        cudaFree(e->d_out.obs_owner);
        cudaFree(e->d_out.obs_terrain);
        cudaFree(e->d_out.obs_vis);
        cudaFree(e->d_out.mask);
        cudaFree(e->d_out.reward);
        cudaFree(e->d_out.scoreboard);
        cudaFree(e->d_out.done);
    }
    delete e;
}

// cudaMalloc that counts the bytes against the environment
template <class T>
cudaError_t dev_alloc(gen_env* e, T** p, size_t bytes) {
    const cudaError_t ce = cudaMalloc(reinterpret_cast<void**>(p), bytes);
    if (ce == cudaSuccess) e->dev_bytes += bytes;
    return ce;
}

// A cached rollout graph holds kernel arguments captured by value (seed,
// generator parameters, launch shapes): drop it whenever one of them changes.
void drop_graph(gen_env* e) {
    if (e->graph) cudaGraphExecDestroy(e->graph);
    e->graph = nullptr;
    e->graph_key.clear();
}

// Mean device time, ms, of one call of `run` on `s` over `reps` calls after two warm-ups.
template <class Run>
float time_calls(Run run, int reps, cudaStream_t s, cudaEvent_t a, cudaEvent_t b) {
    for (int k = 0; k < 2; ++k)
        if (run() != GEN_OK) return 1e30f;
    cudaEventRecord(a, s);
    for (int k = 0; k < reps; ++k)
        if (run() != GEN_OK) return 1e30f;
    cudaEventRecord(b, s);
    if (cudaEventSynchronize(b) != cudaSuccess) return 1e30f;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms / (float)reps;
}

int check_params(const gen_params* p) {
    if (!p) return fail(GEN_ERR_BAD_ARG, "params is NULL");
    if (p->city_army_min < 0 || p->city_army_max < p->city_army_min || p->city_army_max > 32767)
        return fail(GEN_ERR_BAD_ARG, "castle army range [%d, %d] invalid", p->city_army_min, p->city_army_max);
    if (p->n_cities < 0 && (p->city_per_mille < 0 || p->city_per_mille > 1000))
        return fail(GEN_ERR_BAD_ARG, "city_per_mille %d outside [0, 1000]", p->city_per_mille);
    if (p->n_cities > 4096) return fail(GEN_ERR_BAD_ARG, "n_cities %d too large", p->n_cities);
    if (p->max_turns < 0) return fail(GEN_ERR_BAD_ARG, "max_turns < 0");
    if (p->max_general_dist < 0 || p->castle_radius < 0 || p->castle_radius > 127)
        return fail(GEN_ERR_BAD_ARG, "spawn cap %d or castle radius %d invalid", p->max_general_dist, p->castle_radius);
    return GEN_OK;
}

int check_outputs(const gen_outputs* o) {
    if (!o) return fail(GEN_ERR_BAD_ARG, "outputs is NULL");
    const void* ptrs[8] = {o->obs_army, o->obs_owner, o->obs_terrain, o->obs_vis,
                           o->mask,     o->reward,    o->scoreboard,  o->done};
    for (int i = 0; i < 8; ++i) {
        if (!ptrs[i]) return fail(GEN_ERR_BAD_ARG, "output field %d is NULL", i);
        if (i < 5 && !aligned16(ptrs[i])) return fail(GEN_ERR_BAD_ARG, "output plane %d not 16-byte aligned", i);
        if ((i == 5 || i == 6) && (reinterpret_cast<uintptr_t>(ptrs[i]) & 3u))  // float / int32 stores
            return fail(GEN_ERR_BAD_ARG, "output field %d not 4-byte aligned", i);
    }
    return GEN_OK;
}

int choose_warps(int warp_smem) {
    for (int w : {8, 4, 2, 1})
        if (w * warp_smem <= kMaxSmemPerCta) return w;
    return 0;
}

// fill a bucket's carve and launch shape; 0 or a GEN_ERR code
int shape_bucket(Bucket& b) {
    b.warp_smem = gk::warp_smem_bytes(b.npad_max, b.pmax, &b.nw_stride);
    if (b.warps == 0 || b.warps * b.warp_smem > kMaxSmemPerCta) b.warps = choose_warps(b.warp_smem);
    if (b.warps == 0)
        return fail(GEN_ERR_BAD_ARG, "a %d-cell board needs %d bytes of shared memory per game", b.npad_max,
                    b.warp_smem);
    const int rc = gk::max_resident_ctas(b.warps, b.warps * b.warp_smem, &b.max_ctas);
    if (rc != 0) return cuda_fail((cudaError_t)rc, "occupancy query");
    return GEN_OK;
}

KArgs base_args(const gen_env* e, const Bucket& b, int op) {
    KArgs a;
    memset(&a, 0, sizeof(a));
    a.info = e->d_info;
    a.list = (&b == &e->all || !e->d_order) ? nullptr : e->d_order + b.offset;
    a.n_items = b.n;
    a.n_games = e->G;
    a.op = op;
    a.army = e->d_army;
    a.owner = e->d_owner;
    a.terrain = e->d_terrain;
    a.scal = e->d_scal;
    a.seed = e->prm.seed;
    a.game_id_base = e->prm.game_id_base;
    a.mtn_thresh = e->prm.mountain_thresh;
    a.spawn_dmax = e->prm.max_general_dist;
    a.spawn_bfs = e->prm.bfs_distance ? 1 : 0;
    a.castle_radius = e->prm.castle_radius;
    a.lane_groups = e->lane_groups;
    a.city_min = e->prm.city_army_min;
    a.city_span = e->prm.city_army_max - e->prm.city_army_min + 1;
    a.max_turns = e->prm.max_turns;
    a.auto_reset = e->prm.auto_reset;
    a.frames = 1;
    a.plane_stride = e->plane_cells;
    a.slot_stride = e->player_slots;
    a.game_stride = e->G;
    a.npad_max = b.npad_max;
    a.nw_stride = b.nw_stride;
    a.pmax = b.pmax;
    a.warp_smem = b.warp_smem;
    if (e->uniform) {
        a.uniform = 1;
        a.ushape = e->h_info[0];
    }
    return a;
}

void set_outputs(KArgs& a, const gen_outputs* o) {
    a.obs_army = o->obs_army;
    a.obs_owner = o->obs_owner;
    a.obs_terrain = o->obs_terrain;
    a.obs_vis = o->obs_vis;
    a.mask = o->mask;
    a.reward = o->reward;
    a.scoreboard = o->scoreboard;
    a.done = o->done;
    a.do_outputs = 1;
}

int launch_one(const Bucket& b, const KArgs& a, void* stream, const char* what) {
    const int rc = gk::launch_step(a, b.tuned ? b.warps : 0, b.max_ctas, stream);
    if (rc != 0) return cuda_fail((cudaError_t)rc, what);
    return GEN_OK;
}

// Every game, one launch per size bucket; buckets after the first run on
// side streams forked from and joined back into `stream`.
// The work-list form serves batches of several buckets without spawn
// options (their generator runs in its own kernel).  By default it takes
// batches of more than four buckets: there the per-bucket launches are many
// and small (mixed 32,768 games, 15 buckets: 136 against 131 M frames/s per
// frame, resident 173 against 167 M), while a few large buckets overlap
// well on the forked streams (ragged 131,072 games, 4 buckets: 428 against
// 419 M, resident 627 against 606 M).
bool use_worklist(const gen_env* e) {
    const bool spawn = e->prm.max_general_dist > 0 || e->prm.bfs_distance || e->prm.castle_radius > 0;
    if (e->buckets.size() < 2 || !e->d_items[0] || spawn || e->batch_form == 1) return false;
    return e->batch_form == 2 || e->buckets.size() > 4;
}

template <class Fill>
int launch_buckets(gen_env* e, int op, Fill fill, void* stream, const char* what) {
    const size_t nb = e->buckets.size();
    if (use_worklist(e)) {
        KArgs a = base_args(e, e->all, op);
        fill(a);
        const int m = (a.frames > 1 || a.action_log) ? 1 : 0;
        gk::WArgs w;
        w.items = e->d_items[m];
        w.n_items = e->wl_items[m];
        w.geoms = e->d_geoms;
        w.order = e->d_order;
        w.counter = e->d_counter;
        const int rc = gk::launch_worklist(a, w, e->wl_smem[m], e->wl_ctas[m], stream);
        if (rc != 0) return cuda_fail((cudaError_t)rc, what);
        return GEN_OK;
    }
    if (nb == 1) {
        KArgs a = base_args(e, e->buckets[0], op);
        fill(a);
        return launch_one(e->buckets[0], a, stream, what);
    }
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaEventRecord(e->fork, s), "fork record");
    for (size_t i = 0; i < nb; ++i) {
        cudaStream_t si = i == 0 ? s : e->side[i - 1];
        if (i > 0) CUDA_TRY(cudaStreamWaitEvent(si, e->fork, 0), "fork wait");
        KArgs a = base_args(e, e->buckets[i], op);
        fill(a);
        int rc = launch_one(e->buckets[i], a, si, what);
        if (rc) return rc;
        if (i > 0) {
            CUDA_TRY(cudaEventRecord(e->join[i - 1], si), "join record");
            CUDA_TRY(cudaStreamWaitEvent(s, e->join[i - 1], 0), "join wait");
        }
    }
    return GEN_OK;
}

int players_for(int mode, int n_players) {
    if (mode == GEN_MODE_1V1) return 2;
    if (mode == GEN_MODE_2V2) return 4;
    return n_players;
}

// The environment's own output buffers (one frame) and action staging,
// allocated on first use: all of them or none.
int ensure_internal_outputs(gen_env* e) {
    if (e->have_out) return GEN_OK;
    const size_t pc = (size_t)e->plane_cells, ps = (size_t)e->player_slots;
    const size_t bytes[9] = {pc * 2, pc, pc, pc, pc, ps * 4, ps * 8, (size_t)e->G, ps * 4};
    void* p[9] = {};
    cudaError_t ce = cudaSuccess;
    size_t total = 0;
    for (int i = 0; i < 9 && ce == cudaSuccess; ++i) {
        ce = cudaMalloc(&p[i], bytes[i]);
        total += bytes[i];
    }
    if (ce != cudaSuccess) {
        for (void* x : p) cudaFree(x);
        return ce == cudaErrorMemoryAllocation ? fail(GEN_ERR_OOM, "device allocation of the output buffers failed")
                                               : cuda_fail(ce, "cudaMalloc outputs");
    }
    gen_outputs& o = e->d_out;
    o.obs_army = static_cast<int16_t*>(p[0]);
    o.obs_owner = static_cast<int8_t*>(p[1]);
    o.obs_terrain = static_cast<int8_t*>(p[2]);
    o.obs_vis = static_cast<uint8_t*>(p[3]);
    o.mask = static_cast<uint8_t*>(p[4]);
    o.reward = static_cast<float*>(p[5]);
    o.scoreboard = static_cast<int32_t*>(p[6]);
    o.done = static_cast<uint8_t*>(p[7]);
    e->d_actions = static_cast<int32_t*>(p[8]);
    e->dev_bytes += total;
    e->have_out = true;
    return GEN_OK;
}

// The outputs a call writes: the caller's buffers, with the environment's
// own buffers in place of every NULL field (of every field when out is NULL).
int resolve_outputs(gen_env* e, const gen_outputs* out, gen_outputs* res) {
    const gen_outputs none{};
    const gen_outputs& o = out ? *out : none;
    const bool need = !o.obs_army || !o.obs_owner || !o.obs_terrain || !o.obs_vis || !o.mask || !o.reward ||
                      !o.scoreboard || !o.done;
    if (need) {
        const int rc = ensure_internal_outputs(e);
        if (rc) return rc;
    }
    const gen_outputs& d = e->d_out;
    res->obs_army = o.obs_army ? o.obs_army : d.obs_army;
    res->obs_owner = o.obs_owner ? o.obs_owner : d.obs_owner;
    res->obs_terrain = o.obs_terrain ? o.obs_terrain : d.obs_terrain;
    res->obs_vis = o.obs_vis ? o.obs_vis : d.obs_vis;
    res->mask = o.mask ? o.mask : d.mask;
    res->reward = o.reward ? o.reward : d.reward;
    res->scoreboard = o.scoreboard ? o.scoreboard : d.scoreboard;
    res->done = o.done ? o.done : d.done;
    return check_outputs(res);
}

// Size class of a game: padded cells rounded up to a class edge, players
// rounded up to 2, 4 or 8.  Games of one class share a carve.
int cell_class(int npad) {
    for (int edge : {256, 512, 768, 1024, 1536, 2048, 3072, 4096})
        if (npad <= edge) return edge;
    return 4096;
}
int player_class(int P) { return P <= 2 ? 2 : (P <= 4 ? 4 : 8); }

std::pair<int, int> game_class(const GameInfo& gi) { return std::make_pair(cell_class(gi.Npad), player_class(gi.P)); }

int build_buckets(gen_env* e) {
    std::vector<int> order((size_t)e->G);
    for (int g = 0; g < e->G; ++g) order[(size_t)g] = g;
    auto key = [&](int g) { return game_class(e->h_info[(size_t)g]); };
    // largest class first (it finishes last), then game id
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return key(x) > key(y); });
    e->buckets.clear();
    for (int i = 0; i < e->G;) {
        const auto k = key(order[(size_t)i]);
        int j = i;
        Bucket b;
        b.offset = i;
        while (j < e->G && key(order[(size_t)j]) == k) {
            const GameInfo& gi = e->h_info[(size_t)order[(size_t)j]];
            b.npad_max = std::max(b.npad_max, (int)gi.Npad);
            b.pmax = std::max(b.pmax, (int)gi.P);
            ++j;
        }
        b.n = j - i;
        b.warps = 8;
        int rc = shape_bucket(b);
        if (rc) return rc;
        e->buckets.push_back(b);
        i = j;
    }
    if (e->buckets.size() > 1) {
        CUDA_TRY(dev_alloc(e, &e->d_order, sizeof(int32_t) * (size_t)e->G), "cudaMalloc order");
        CUDA_TRY(cudaMemcpy(e->d_order, order.data(), sizeof(int32_t) * (size_t)e->G, cudaMemcpyHostToDevice),
                 "upload order");
        CUDA_TRY(cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming), "event");
        for (size_t i = 1; i < e->buckets.size(); ++i) {
            cudaStream_t s;
            cudaEvent_t v;
            CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream");
            e->side.push_back(s);
            CUDA_TRY(cudaEventCreateWithFlags(&v, cudaEventDisableTiming), "event");
            e->join.push_back(v);
        }
    }
    return GEN_OK;
}

// The work lists of a batch of several buckets: per bucket its shared-memory
// geometry and lane-group width, and items of as many consecutive games (in
// the bucket order, largest boards first) as one CTA of the work-list kernel
// holds.  Rebuilt when the lane-group setting changes; synchronous.
int build_worklist(gen_env* e) {
    if (e->buckets.size() < 2) return GEN_OK;
    const size_t nb = e->buckets.size();
    std::vector<gk::BucketGeom> geoms(nb);
    for (size_t i = 0; i < nb; ++i) {
        const Bucket& b = e->buckets[i];
        geoms[i].lw = (b.pmax <= 2 && b.npad_max <= 1024 && e->lane_groups != 1) ? 16 : 32;
        geoms[i].group_smem = gk::warp_smem_bytes(b.npad_max, b.pmax, nullptr, geoms[i].lw < 32);
        geoms[i].geom = gk::bucket_geom(b.npad_max, b.nw_stride, b.pmax, geoms[i].lw < 32);
        geoms[i].pad = 0;
    }
    if (!e->d_geoms) {
        CUDA_TRY(dev_alloc(e, &e->d_geoms, sizeof(gk::BucketGeom) * nb), "cudaMalloc bucket geometry");
        CUDA_TRY(dev_alloc(e, &e->d_counter, 2 * sizeof(int32_t)), "cudaMalloc work counters");
        const int32_t zero[2] = {0, 0};  // afterwards each work-list launch leaves them zeroed
        CUDA_TRY(cudaMemcpy(e->d_counter, zero, sizeof(zero), cudaMemcpyHostToDevice), "zero work counters");
    }
    CUDA_TRY(cudaMemcpy(e->d_geoms, geoms.data(), sizeof(gk::BucketGeom) * nb, cudaMemcpyHostToDevice),
             "upload bucket geometry");
    for (int m = 0; m < 2; ++m) {
        int smem = 0, ctas = 0;
        const int rc = gk::worklist_shape(m == 1, &smem, &ctas);
        if (rc != 0) return cuda_fail((cudaError_t)rc, "work-list launch shape");
        std::vector<gk::WorkItem> items;
        for (size_t i = 0; i < nb; ++i) {
            const Bucket& b = e->buckets[i];
            const int groups = 8 * (32 / geoms[i].lw);
            const int gs = geoms[i].group_smem;
            const int per = std::max(1, std::min(groups, smem / gs));
            if (per * gs > smem)
                return fail(GEN_ERR_BAD_ARG, "a %d-cell board needs %d bytes of shared memory per game", b.npad_max, gs);
            for (int k = 0; k < b.n; k += per) {
                gk::WorkItem it;
                it.first = b.offset + k;
                it.count = std::min(per, b.n - k);
                it.bucket = (int)i;
                it.pad = 0;
                items.push_back(it);
            }
        }
        if (!e->d_items[m])  // at most one item per game, whatever the lane-group widths
            CUDA_TRY(dev_alloc(e, &e->d_items[m], sizeof(gk::WorkItem) * (size_t)e->G), "cudaMalloc work list");
        CUDA_TRY(cudaMemcpy(e->d_items[m], items.data(), sizeof(gk::WorkItem) * items.size(), cudaMemcpyHostToDevice),
                 "upload work list");
        e->wl_items[m] = (int)items.size();
        e->wl_smem[m] = smem;
        e->wl_ctas[m] = ctas;
    }
    return GEN_OK;
}

}  // namespace

extern "C" {

int gen_default_params(gen_params* p) {
    if (!p) return fail(GEN_ERR_BAD_ARG, "params is NULL");
    memset(p, 0, sizeof(*p));
    p->seed = 1;
    p->game_id_base = 0;
    p->mountain_thresh = 858993459u;
    p->n_cities = 8;
    p->city_per_mille = 0;
    p->city_army_min = 40;
    p->city_army_max = 50;
    p->min_general_dist = 0;
    p->max_turns = 0;
    p->auto_reset = 1;
    return GEN_OK;
}

int gen_create_ex(gen_env** out, const gen_params* p, int batch, const int32_t* h_H, const int32_t* h_W,
                  const int32_t* h_mode, const int32_t* h_n_players) {
    if (!out) return fail(GEN_ERR_BAD_ARG, "out is NULL");
    *out = nullptr;
    int rc = check_params(p);
    if (rc) return rc;
    if (batch < 1) return fail(GEN_ERR_BAD_ARG, "batch %d < 1", batch);
    if (!h_H || !h_W || !h_mode) return fail(GEN_ERR_BAD_ARG, "shape arrays are NULL");
    gen_env* e = new gen_env();
    e->G = batch;
    e->prm = *p;
    e->h_info.resize((size_t)batch);
    int64_t cell = 0, plane = 0;
    int slot = 0;
    for (int g = 0; g < batch; ++g) {
        const int H = h_H[g], W = h_W[g], mode = h_mode[g];
        const int P = players_for(mode, h_n_players ? h_n_players[g] : 8);
        if (H < 1 || W < 1 || H > GEN_MAX_SIDE || W > GEN_MAX_SIDE) {
            free_env(e);
            return fail(GEN_ERR_BAD_ARG, "game %d: side %dx%d outside 1..%d", g, H, W, GEN_MAX_SIDE);
        }
        if (mode < 0 || mode > 2 || P < 2 || P > GEN_MAX_PLAYERS || H * W < P) {
            free_env(e);
            return fail(GEN_ERR_BAD_ARG, "game %d: mode %d with %d players on %d cells", g, mode, P, H * W);
        }
        const int N = H * W, Npad = (N + 15) & ~15;
        GameInfo& gi = e->h_info[(size_t)g];
        memset(&gi, 0, sizeof(gi));
        gi.plane_off = plane;
        gi.game_id = p->game_id_base + (uint64_t)g;
        gi.cell_off = (int32_t)cell;
        gi.player_off = slot;
        gi.H = (int16_t)H;
        gi.W = (int16_t)W;
        gi.N = (int16_t)N;
        gi.Npad = (int16_t)Npad;
        gi.mode = (int8_t)mode;
        gi.P = (int8_t)P;
        const int nc = p->n_cities >= 0 ? p->n_cities : (int)(((int64_t)N * p->city_per_mille) / 1000);
        gi.n_cities = (int16_t)nc;
        int d = p->min_general_dist >= 1 ? p->min_general_dist : (H + W) / 3;
        gi.dmin = (int16_t)(d < 1 ? 1 : d);
        cell += Npad;
        plane += (int64_t)P * Npad;
        slot += P;
        e->pmax = std::max(e->pmax, P);
        e->npad_max = std::max(e->npad_max, Npad);
        e->nmax = std::max(e->nmax, N);
        if (cell > INT32_MAX) {
            free_env(e);
            return fail(GEN_ERR_BAD_ARG, "batch too large: more than 2^31 state cells");
        }
    }
    {
        const int trc = gk::init_tables();  // arguments are valid: now touch the device
        if (trc != 0) {
            free_env(e);
            return cuda_fail((cudaError_t)trc, "device tables");
        }
    }
    e->state_cells = cell;
    e->plane_cells = plane;
    e->player_slots = slot;
    e->uniform = true;
    for (int g = 1; g < batch && e->uniform; ++g) {
        const GameInfo& x = e->h_info[(size_t)g];
        const GameInfo& y = e->h_info[0];
        e->uniform = x.H == y.H && x.W == y.W && x.mode == y.mode && x.P == y.P && x.n_cities == y.n_cities &&
                     x.dmin == y.dmin;
    }
    e->all.n = batch;
    e->all.npad_max = e->npad_max;
    e->all.pmax = e->pmax;
    if ((rc = shape_bucket(e->all)) != GEN_OK || (rc = build_buckets(e)) != GEN_OK ||
        (rc = build_worklist(e)) != GEN_OK) {
        free_env(e);
        return rc;
    }

    cudaError_t ce;
    if ((ce = dev_alloc(e, &e->d_info, sizeof(GameInfo) * (size_t)batch)) != cudaSuccess ||
        (ce = dev_alloc(e, &e->d_scal, sizeof(GameScalars) * (size_t)batch)) != cudaSuccess ||
        (ce = dev_alloc(e, &e->d_army, 2 * (size_t)cell)) != cudaSuccess ||
        (ce = dev_alloc(e, &e->d_owner, (size_t)cell)) != cudaSuccess ||
        (ce = dev_alloc(e, &e->d_terrain, (size_t)cell)) != cudaSuccess) {
        free_env(e);
        return ce == cudaErrorMemoryAllocation ? fail(GEN_ERR_OOM, "device allocation failed")
                                               : cuda_fail(ce, "cudaMalloc");
    }
    if ((ce = cudaMemcpy(e->d_info, e->h_info.data(), sizeof(GameInfo) * (size_t)batch, cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (ce = cudaMemset(e->d_scal, 0, sizeof(GameScalars) * (size_t)batch)) != cudaSuccess) {
        free_env(e);
        return cuda_fail(ce, "upload game table");
    }
    rc = launch_buckets(e, gk::OP_CREATE, [](KArgs&) {}, nullptr, "create launch");
    if (rc == GEN_OK && (ce = cudaDeviceSynchronize()) != cudaSuccess) rc = cuda_fail(ce, "create kernel");
    if (rc) {
        free_env(e);
        return rc;
    }
    *out = e;
    return GEN_OK;
}

int gen_create(gen_env** out, int batch, int H, int W, int mode, uint64_t seed) {
    gen_params p;
    gen_default_params(&p);
    p.seed = seed;
    if (batch < 1) return fail(GEN_ERR_BAD_ARG, "batch %d < 1", batch);
    std::vector<int32_t> hh((size_t)batch, H), ww((size_t)batch, W), mm((size_t)batch, mode),
        pp((size_t)batch, 8);
    return gen_create_ex(out, &p, batch, hh.data(), ww.data(), mm.data(), pp.data());
}

int gen_layout(const gen_env* e, gen_layout_info* info, int64_t* h_plane_off, int32_t* h_player_off,
               int32_t* h_npad) {
    if (!e || !info) return fail(GEN_ERR_BAD_ARG, "env or info is NULL");
    info->n_games = e->G;
    info->player_slots = e->player_slots;
    info->plane_cells = e->plane_cells;
    info->state_cells = e->state_cells;
    info->max_players = e->pmax;
    info->max_cells = e->nmax;
    for (int g = 0; g < e->G; ++g) {
        const GameInfo& gi = e->h_info[(size_t)g];
        if (h_plane_off) h_plane_off[g] = gi.plane_off;
        if (h_player_off) h_player_off[g] = gi.player_off;
        if (h_npad) h_npad[g] = gi.Npad;
    }
    return GEN_OK;
}

int gen_reset(gen_env* e, const int32_t* d_game_ids, int n, const gen_outputs* out_arg, void* stream) {
    if (!e) return fail(GEN_ERR_BAD_ARG, "env is NULL");
    if (d_game_ids && (n < 0 || n > e->G)) return fail(GEN_ERR_BAD_ARG, "reset count %d outside [0, %d]", n, e->G);
    gen_outputs res;
    int rc = resolve_outputs(e, out_arg, &res);
    if (rc) return rc;
    const gen_outputs* out = &res;
    if (!d_game_ids)
        return launch_buckets(e, gk::OP_RESET, [&](KArgs& a) { set_outputs(a, out); }, stream, "reset launch");
    KArgs a = base_args(e, e->all, gk::OP_RESET);
    a.list = d_game_ids;
    a.n_items = n;
    set_outputs(a, out);
    return launch_one(e->all, a, stream, "reset launch");
}

int gen_observe(gen_env* e, const gen_outputs* out_arg, void* stream) {
    if (!e) return fail(GEN_ERR_BAD_ARG, "env is NULL");
    gen_outputs res;
    int rc = resolve_outputs(e, out_arg, &res);
    if (rc) return rc;
    const gen_outputs* out = &res;
    return launch_buckets(e, gk::OP_OBSERVE, [&](KArgs& a) { set_outputs(a, out); }, stream, "observe launch");
}

int gen_outputs_get(gen_env* e, gen_outputs* out) {
    if (!e || !out) return fail(GEN_ERR_BAD_ARG, "env or out is NULL");
    const int rc = ensure_internal_outputs(e);
    if (rc) return rc;
    *out = e->d_out;
    return GEN_OK;
}

int gen_device_bytes(const gen_env* e, size_t* bytes) {
    if (!e || !bytes) return fail(GEN_ERR_BAD_ARG, "env or bytes is NULL");
    *bytes = e->dev_bytes;
    return GEN_OK;
}

int gen_step_policy(gen_env* e, const int32_t* d_actions, const gen_outputs* out_arg, uint64_t policy_seed,
                    int32_t* d_next_actions, void* stream) {
    if (!e) return fail(GEN_ERR_BAD_ARG, "env is NULL");
    if (!d_actions) return fail(GEN_ERR_BAD_ARG, "actions is NULL");
    if (!aligned4(d_actions) || !aligned4(d_next_actions)) return fail(GEN_ERR_BAD_ARG, "actions not 4-byte aligned");
    gen_outputs res;
    int rc = resolve_outputs(e, out_arg, &res);
    if (rc) return rc;
    const gen_outputs* out = &res;
    return launch_buckets(e, gk::OP_STEP,
                          [&](KArgs& a) {
                              a.actions = d_actions;
                              set_outputs(a, out);
                              a.next_actions = d_next_actions;
                              a.policy_seed = policy_seed;
                          },
                          stream, "step launch");
}

int gen_step(gen_env* e, const int32_t* d_actions, const gen_outputs* out, void* stream) {
    return gen_step_policy(e, d_actions, out, 0, nullptr, stream);
}

int gen_policy(gen_env* e, uint64_t policy_seed, int32_t* d_actions, void* stream) {
    if (!e) return fail(GEN_ERR_BAD_ARG, "env is NULL");
    if (!d_actions) return fail(GEN_ERR_BAD_ARG, "actions is NULL");
    if (!aligned4(d_actions)) return fail(GEN_ERR_BAD_ARG, "actions not 4-byte aligned");
    return launch_buckets(e, gk::OP_POLICY,
                          [&](KArgs& a) {
                              a.next_actions = d_actions;
                              a.policy_seed = policy_seed;
                          },
                          stream, "policy launch");
}

int gen_rollout(gen_env* e, int K, uint64_t policy_seed, int32_t* d_actions, const gen_outputs* out,
                int32_t* d_action_log, int impl, void* stream) {
    if (!e) return fail(GEN_ERR_BAD_ARG, "env is NULL");
    if (K < 1) return fail(GEN_ERR_BAD_ARG, "K = %d < 1", K);
    if (!d_actions) return fail(GEN_ERR_BAD_ARG, "actions is NULL");
    if (!aligned4(d_actions) || !aligned4(d_action_log)) return fail(GEN_ERR_BAD_ARG, "actions not 4-byte aligned");
    // K frames of outputs: the environment's own buffers hold one, so every field is the caller's
    int rc = check_outputs(out);
    if (rc) return rc;
    if (impl == GEN_ROLLOUT_AUTO) impl = e->rollout_form;
    if (impl == GEN_ROLLOUT_RESIDENT) {
        return launch_buckets(e, gk::OP_STEP,
                              [&](KArgs& a) {
                                  a.actions = d_actions;
                                  set_outputs(a, out);
                                  a.next_actions = d_actions;
                                  a.policy_seed = policy_seed;
                                  a.frames = K;
                                  a.action_log = d_action_log;
                              },
                              stream, "rollout launch");
    }
    if (impl != GEN_ROLLOUT_GRAPH && impl != GEN_ROLLOUT_LAUNCHES)
        return fail(GEN_ERR_BAD_ARG, "unknown rollout form %d", impl);
    // K single-frame launches; launch k writes frame k of every output
    auto enqueue = [&](cudaStream_t s) -> int {
        for (int k = 0; k < K; ++k) {
            const int64_t pk = (int64_t)k * e->plane_cells, sk = (int64_t)k * e->player_slots;
            int r = launch_buckets(e, gk::OP_STEP,
                                   [&](KArgs& a) {
                                       a.actions = d_actions;
                                       set_outputs(a, out);
                                       a.obs_army += pk;
                                       a.obs_owner += pk;
                                       a.obs_terrain += pk;
                                       a.obs_vis += pk;
                                       a.mask += pk;
                                       a.reward += sk;
                                       a.scoreboard += 2 * sk;
                                       a.done += (int64_t)k * e->G;
                                       a.next_actions = d_actions;
                                       a.policy_seed = policy_seed;
                                       a.action_log = d_action_log ? d_action_log + sk : nullptr;
                                   },
                                   s, "rollout launch");
            if (r) return r;
        }
        return GEN_OK;
    };
    if (impl == GEN_ROLLOUT_LAUNCHES) return enqueue((cudaStream_t)stream);
    // CUDA graph of the K launches, captured once per (K, buffers, seed)
    const std::vector<const void*> key = {(const void*)(intptr_t)K, (const void*)(uintptr_t)policy_seed,
                                          d_actions,                d_action_log,
                                          out->obs_army,            out->obs_owner,
                                          out->obs_terrain,         out->obs_vis,
                                          out->mask,                out->reward,
                                          out->scoreboard,          out->done};
    if (!e->graph || e->graph_key != key) {
        if (e->graph) {
            cudaGraphExecDestroy(e->graph);
            e->graph = nullptr;
        }
        cudaStream_t cap;
        CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "capture stream");
        cudaGraph_t gr = nullptr;
        cudaError_t ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
            rc = enqueue(cap);
            cudaError_t ce2 = cudaStreamEndCapture(cap, &gr);
            if (rc == GEN_OK && ce2 != cudaSuccess) rc = cuda_fail(ce2, "end capture");
        } else {
            rc = cuda_fail(ce, "begin capture");
        }
        cudaStreamDestroy(cap);
        if (rc) {
            if (gr) cudaGraphDestroy(gr);
            return rc;
        }
        ce = cudaGraphInstantiate(&e->graph, gr, 0);
        cudaGraphDestroy(gr);
        if (ce != cudaSuccess) {
            e->graph = nullptr;
            return cuda_fail(ce, "graph instantiate");
        }
        e->graph_key = key;
    }
    CUDA_TRY(cudaGraphLaunch(e->graph, (cudaStream_t)stream), "graph launch");
    return GEN_OK;
}

// The outputs of games [g0, g1) copied device -> host on stream t: every
// per-game range is contiguous because offsets grow in game order.
static int copy_out_range(gen_env* e, const gen_outputs& h, int32_t* h_next, int g0, int g1, cudaStream_t t) {
    const gen_outputs& d = e->d_out;
    const size_t p0 = (size_t)e->h_info[g0].plane_off;
    const size_t p1 = g1 < e->G ? (size_t)e->h_info[g1].plane_off : (size_t)e->plane_cells;
    const size_t s0 = (size_t)e->h_info[g0].player_off;
    const size_t s1 = g1 < e->G ? (size_t)e->h_info[g1].player_off : (size_t)e->player_slots;
    const size_t np = p1 - p0, ns = s1 - s0;
    auto cp = [&](void* dst, const void* src, size_t bytes) {
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, t);
    };
    if (h_next) CUDA_TRY(cp(h_next + s0, e->d_actions + s0, ns * 4), "copy actions out");
    if (h.obs_army) CUDA_TRY(cp(h.obs_army + p0, d.obs_army + p0, np * 2), "copy out");
    if (h.obs_owner) CUDA_TRY(cp(h.obs_owner + p0, d.obs_owner + p0, np), "copy out");
    if (h.obs_terrain) CUDA_TRY(cp(h.obs_terrain + p0, d.obs_terrain + p0, np), "copy out");
    if (h.obs_vis) CUDA_TRY(cp(h.obs_vis + p0, d.obs_vis + p0, np), "copy out");
    if (h.mask) CUDA_TRY(cp(h.mask + p0, d.mask + p0, np), "copy out");
    if (h.reward) CUDA_TRY(cp(h.reward + s0, d.reward + s0, ns * 4), "copy out");
    if (h.scoreboard) CUDA_TRY(cp(h.scoreboard + 2 * s0, d.scoreboard + 2 * s0, ns * 8), "copy out");
    if (h.done) CUDA_TRY(cp(h.done + g0, d.done + g0, (size_t)(g1 - g0)), "copy out");
    return GEN_OK;
}

// Pipelined host step for a batch launched as one bucket in game order: the
// batch runs as K chunks of games on `s`, and each chunk's outputs leave on a
// copy stream as soon as its launch ends, so the copies (bound by the host
// link) overlap the remaining launches.
static int step_host_pipelined(gen_env* e, const gen_outputs& h, uint64_t policy_seed, int32_t* h_next,
                               cudaStream_t s, int K) {
    if (!e->d_iota) {
        std::vector<int32_t> iota((size_t)e->G);
        for (int g = 0; g < e->G; ++g) iota[(size_t)g] = g;
        CUDA_TRY(dev_alloc(e, &e->d_iota, sizeof(int32_t) * (size_t)e->G), "cudaMalloc game ids");
        CUDA_TRY(cudaMemcpy(e->d_iota, iota.data(), sizeof(int32_t) * (size_t)e->G, cudaMemcpyHostToDevice),
                 "upload game ids");
        CUDA_TRY(cudaStreamCreateWithFlags(&e->copy, cudaStreamNonBlocking), "copy stream");
        for (auto& v : e->chunk_ev) CUDA_TRY(cudaEventCreateWithFlags(&v, cudaEventDisableTiming), "chunk event");
        CUDA_TRY(cudaEventCreateWithFlags(&e->copy_done, cudaEventDisableTiming), "copy event");
    }
    const Bucket& b = e->buckets[0];
    for (int c = 0; c < K; ++c) {
        const int g0 = (int)((int64_t)e->G * c / K), g1 = (int)((int64_t)e->G * (c + 1) / K);
        KArgs a = base_args(e, b, gk::OP_STEP);
        a.list = e->d_iota + g0;
        a.n_items = g1 - g0;
        a.actions = e->d_actions;
        set_outputs(a, &e->d_out);
        a.next_actions = h_next ? e->d_actions : nullptr;
        a.policy_seed = policy_seed;
        int rc = launch_one(b, a, s, "step launch");
        if (rc) return rc;
        CUDA_TRY(cudaEventRecord(e->chunk_ev[c], s), "chunk record");
        CUDA_TRY(cudaStreamWaitEvent(e->copy, e->chunk_ev[c], 0), "chunk wait");
        rc = copy_out_range(e, h, h_next, g0, g1, e->copy);
        if (rc) return rc;
    }
    CUDA_TRY(cudaEventRecord(e->copy_done, e->copy), "copy record");
    CUDA_TRY(cudaStreamWaitEvent(s, e->copy_done, 0), "copy join");
    return GEN_OK;
}

int gen_step_host(gen_env* e, const int32_t* h_actions, const gen_outputs* h_out, uint64_t policy_seed,
                  int32_t* h_next_actions, void* stream) {
    if (!e) return fail(GEN_ERR_BAD_ARG, "env is NULL");
    if (!h_actions || !h_out) return fail(GEN_ERR_BAD_ARG, "host buffers are NULL");
    int rc = ensure_internal_outputs(e);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t pc = (size_t)e->plane_cells, ps = (size_t)e->player_slots;
    CUDA_TRY(cudaMemcpyAsync(e->d_actions, h_actions, ps * 4, cudaMemcpyHostToDevice, s), "copy actions in");
    if (e->buckets.size() == 1 && !e->d_order && e->G >= 8192) {
        rc = step_host_pipelined(e, *h_out, policy_seed, h_next_actions, s, 4);
        if (rc) return rc;
        CUDA_TRY(cudaStreamSynchronize(s), "step_host sync");
        return GEN_OK;
    }
    rc = gen_step_policy(e, e->d_actions, &e->d_out, policy_seed, h_next_actions ? e->d_actions : nullptr, stream);
    if (rc) return rc;
    if (h_next_actions)
        CUDA_TRY(cudaMemcpyAsync(h_next_actions, e->d_actions, ps * 4, cudaMemcpyDeviceToHost, s), "copy actions out");
    const gen_outputs& d = e->d_out;
    const gen_outputs& h = *h_out;
    if (h.obs_army) CUDA_TRY(cudaMemcpyAsync(h.obs_army, d.obs_army, pc * 2, cudaMemcpyDeviceToHost, s), "copy out");
    if (h.obs_owner) CUDA_TRY(cudaMemcpyAsync(h.obs_owner, d.obs_owner, pc, cudaMemcpyDeviceToHost, s), "copy out");
    if (h.obs_terrain)
        CUDA_TRY(cudaMemcpyAsync(h.obs_terrain, d.obs_terrain, pc, cudaMemcpyDeviceToHost, s), "copy out");
    if (h.obs_vis) CUDA_TRY(cudaMemcpyAsync(h.obs_vis, d.obs_vis, pc, cudaMemcpyDeviceToHost, s), "copy out");
    if (h.mask) CUDA_TRY(cudaMemcpyAsync(h.mask, d.mask, pc, cudaMemcpyDeviceToHost, s), "copy out");
    if (h.reward) CUDA_TRY(cudaMemcpyAsync(h.reward, d.reward, ps * 4, cudaMemcpyDeviceToHost, s), "copy out");
    if (h.scoreboard)
        CUDA_TRY(cudaMemcpyAsync(h.scoreboard, d.scoreboard, ps * 8, cudaMemcpyDeviceToHost, s), "copy out");
    if (h.done) CUDA_TRY(cudaMemcpyAsync(h.done, d.done, (size_t)e->G, cudaMemcpyDeviceToHost, s), "copy out");
    CUDA_TRY(cudaStreamSynchronize(s), "step_host sync");
    return GEN_OK;
}

}  // extern "C"

// ---- host-buffer step that allocates nothing --------------------------------
// gen_step_host stages actions and outputs in device buffers it allocates on
// its first call.  gen_step_host_static stages them instead in this
// file-scope array, reserved when the library is loaded on a GPU and held by
// every GPU that loads it until the process exits.  Host code must not use
// the symbol as an address: the per-device address comes from
// cudaGetSymbolAddress, looked up once per device with that device current.
namespace {

constexpr size_t kStaticStageBytes = size_t(32) << 20;  // 32 MiB
__device__ __align__(256) unsigned char g_static_stage[kStaticStageBytes];

constexpr int kMaxStageDevices = 64;
std::mutex g_stage_mu;
unsigned char* g_stage_addr[kMaxStageDevices] = {};
void* g_stage_ctx[kMaxStageDevices] = {};

// The calling thread's current CUDA context (a driver handle), or NULL when
// it cannot be read.  Read through the runtime's driver entry-point lookup,
// so the library needs no link to the driver library.
void* current_context() {
    using CtxGetCurrent = int (*)(void**);
    static const CtxGetCurrent fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return static_cast<CtxGetCurrent>(nullptr);
        return reinterpret_cast<CtxGetCurrent>(f);
    }();
    void* ctx = nullptr;
    if (fn && fn(&ctx) != 0) ctx = nullptr;
    return ctx;
}

// Device address of the staging array on the current device.  Looked up
// once per device with that device current, and again whenever the device's
// context has changed since (cudaDeviceReset recreates it and the module,
// and the array may then sit elsewhere).
int static_stage(unsigned char** out) {
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kMaxStageDevices) return fail(GEN_ERR_BAD_ARG, "device %d beyond %d", dev, kMaxStageDevices);
    std::lock_guard<std::mutex> lk(g_stage_mu);
    void* ctx = current_context();
    if (!g_stage_addr[dev] || !ctx || ctx != g_stage_ctx[dev]) {
        void* p = nullptr;
        const cudaError_t ce = cudaGetSymbolAddress(&p, g_static_stage);
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaGetSymbolAddress(static stage)");
        g_stage_addr[dev] = static_cast<unsigned char*>(p);
        g_stage_ctx[dev] = current_context();
    }
    *out = g_stage_addr[dev];
    return GEN_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" {

int gen_step_host_static(gen_env* e, const int32_t* h_actions, const gen_outputs* h_out, uint64_t policy_seed,
                         int32_t* h_next_actions, void* stream) {
    if (!e) return fail(GEN_ERR_BAD_ARG, "env is NULL");
    if (!h_actions || !h_out) return fail(GEN_ERR_BAD_ARG, "host buffers are NULL");
    const size_t pc = (size_t)e->plane_cells, ps = (size_t)e->player_slots, G = (size_t)e->G;
    // stage layout: actions, five planes, reward, scoreboard, done (256-byte aligned each)
    size_t off[9];
    const size_t sizes[9] = {ps * 4, pc * 2, pc, pc, pc, pc, ps * 4, ps * 8, G};
    size_t total = 0;
    for (int i = 0; i < 9; ++i) {
        off[i] = total;
        total += align256(sizes[i]);
    }
    if (total > kStaticStageBytes)
        return fail(GEN_ERR_BAD_ARG,
                    "batch needs %zu bytes of staging; gen_step_host_static holds at most %zu (use gen_step_host)",
                    total, kStaticStageBytes);
    unsigned char* base = nullptr;
    int rc = static_stage(&base);
    if (rc) return rc;
    int32_t* d_act = reinterpret_cast<int32_t*>(base + off[0]);
    gen_outputs d;
    d.obs_army = reinterpret_cast<int16_t*>(base + off[1]);
    d.obs_owner = reinterpret_cast<int8_t*>(base + off[2]);
    d.obs_terrain = reinterpret_cast<int8_t*>(base + off[3]);
    d.obs_vis = base + off[4];
    d.mask = base + off[5];
    d.reward = reinterpret_cast<float*>(base + off[6]);
    d.scoreboard = reinterpret_cast<int32_t*>(base + off[7]);
    d.done = base + off[8];
    // every staged byte the step reads is copied in first and every output it
    // returns is written by the step, so nothing needs clearing between calls
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(d_act, h_actions, ps * 4, cudaMemcpyHostToDevice, s), "copy actions in");
    rc = gen_step_policy(e, d_act, &d, policy_seed, h_next_actions ? d_act : nullptr, stream);
    if (rc) return rc;
    if (h_next_actions) CUDA_TRY(cudaMemcpyAsync(h_next_actions, d_act, ps * 4, cudaMemcpyDeviceToHost, s), "copy out");
    const gen_outputs& h = *h_out;
    if (h.obs_army) CUDA_TRY(cudaMemcpyAsync(h.obs_army, d.obs_army, pc * 2, cudaMemcpyDeviceToHost, s), "copy out");
    if (h.obs_owner) CUDA_TRY(cudaMemcpyAsync(h.obs_owner, d.obs_owner, pc, cudaMemcpyDeviceToHost, s), "copy out");
    if (h.obs_terrain)
        CUDA_TRY(cudaMemcpyAsync(h.obs_terrain, d.obs_terrain, pc, cudaMemcpyDeviceToHost, s), "copy out");
    if (h.obs_vis) CUDA_TRY(cudaMemcpyAsync(h.obs_vis, d.obs_vis, pc, cudaMemcpyDeviceToHost, s), "copy out");
    if (h.mask) CUDA_TRY(cudaMemcpyAsync(h.mask, d.mask, pc, cudaMemcpyDeviceToHost, s), "copy out");
    if (h.reward) CUDA_TRY(cudaMemcpyAsync(h.reward, d.reward, ps * 4, cudaMemcpyDeviceToHost, s), "copy out");
    if (h.scoreboard)
        CUDA_TRY(cudaMemcpyAsync(h.scoreboard, d.scoreboard, ps * 8, cudaMemcpyDeviceToHost, s), "copy out");
    if (h.done) CUDA_TRY(cudaMemcpyAsync(h.done, d.done, G, cudaMemcpyDeviceToHost, s), "copy out");
    CUDA_TRY(cudaStreamSynchronize(s), "step_host_static sync");
    return GEN_OK;
}

}  // extern "C"

namespace {

// Host state of every game in the public layout (terrain bits 0-1 only);
// synchronous on s.
int read_state_into(gen_env* e, int16_t* h_army, int8_t* h_owner, int8_t* h_terrain, uint32_t* h_scalars,
                    cudaStream_t s) {
    const size_t n = (size_t)e->state_cells;
    if (h_army) CUDA_TRY(cudaMemcpyAsync(h_army, e->d_army, 2 * n, cudaMemcpyDeviceToHost, s), "read army");
    if (h_owner) CUDA_TRY(cudaMemcpyAsync(h_owner, e->d_owner, n, cudaMemcpyDeviceToHost, s), "read owner");
    if (h_terrain) CUDA_TRY(cudaMemcpyAsync(h_terrain, e->d_terrain, n, cudaMemcpyDeviceToHost, s), "read terrain");
    if (h_scalars)
        CUDA_TRY(cudaMemcpyAsync(h_scalars, e->d_scal, sizeof(GameScalars) * (size_t)e->G, cudaMemcpyDeviceToHost, s),
                 "read scalars");
    CUDA_TRY(cudaStreamSynchronize(s), "read_state sync");
    // the device keeps per-map passable-neighbour bits above the cell type
    if (h_terrain)
        for (size_t i = 0; i < n; ++i) h_terrain[i] = (int8_t)(h_terrain[i] & 3);
    return GEN_OK;
}

// Every game's state within the rules' ranges (Section IV: cell types,
// owners, armies; alive bits of the game's players).
int validate_state(const gen_env* e, const int16_t* h_army, const int8_t* h_owner, const int8_t* h_terrain,
                   const uint32_t* h_scalars) {
    for (int g = 0; g < e->G; ++g) {
        const GameInfo& gi = e->h_info[(size_t)g];
        const uint32_t* sc = h_scalars + 8 * (size_t)g;
        const uint32_t full = (1u << gi.P) - 1u;
        if ((sc[3] & ~full) != 0u || sc[4] > 1u)
            return fail(GEN_ERR_BAD_ARG, "game %d: alive bits 0x%x or finished %u invalid", g, sc[3], sc[4]);
        for (int c = 0; c < gi.Npad; ++c) {
            const size_t k = (size_t)gi.cell_off + (size_t)c;
            const bool pad = c >= gi.N;
            if (h_terrain[k] < 0 || h_terrain[k] > 3 || h_owner[k] < -1 || h_owner[k] >= gi.P || h_army[k] < 0 ||
                (pad && (h_terrain[k] != 0 || h_army[k] != 0 || h_owner[k] != -1)))
                return fail(GEN_ERR_BAD_ARG, "game %d cell %d: invalid cell (terrain %d owner %d army %d)", g, c,
                            h_terrain[k], h_owner[k], h_army[k]);
        }
    }
    return GEN_OK;
}

// Upload validated host state, then recompute the per-map cached bits;
// synchronous on s.  keep_err: restore the error words as given (else 0).
int upload_state(gen_env* e, const int16_t* h_army, const int8_t* h_owner, const int8_t* h_terrain,
                 const uint32_t* h_scalars, bool keep_err, cudaStream_t s) {
    const size_t n = (size_t)e->state_cells;
    std::vector<GameScalars> sc((size_t)e->G);
    memcpy(sc.data(), h_scalars, sizeof(GameScalars) * (size_t)e->G);
    if (!keep_err)
        for (auto& x : sc) x.err = 0;
    CUDA_TRY(cudaMemcpyAsync(e->d_army, h_army, 2 * n, cudaMemcpyHostToDevice, s), "write army");
    CUDA_TRY(cudaMemcpyAsync(e->d_owner, h_owner, n, cudaMemcpyHostToDevice, s), "write owner");
    CUDA_TRY(cudaMemcpyAsync(e->d_terrain, h_terrain, n, cudaMemcpyHostToDevice, s), "write terrain");
    CUDA_TRY(cudaMemcpyAsync(e->d_scal, sc.data(), sizeof(GameScalars) * (size_t)e->G, cudaMemcpyHostToDevice, s),
             "write scalars");
    int rc = launch_buckets(e, gk::OP_DERIVE, [](KArgs&) {}, s, "derive launch");
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize(s), "write_state sync");
    return GEN_OK;
}

// ---- saved-state blob --------------------------------------------------
// Header (kBlobHeader bytes), then per game int32 H, W, mode, players; army
// int16 [state_cells]; owner int8 [state_cells]; terrain int8 [state_cells]
// (cell type only); scalars uint32 [n_games][8].  Host byte order.
constexpr char kBlobMagic[8] = {'G', 'E', 'N', 'S', 'T', 'A', 'T', 'E'};
constexpr uint32_t kBlobVersion = 1;

struct BlobHeader {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;
    uint64_t total_bytes;
    uint64_t checksum;  // FNV-1a 64 of every byte after the header
    int32_t n_games;
    int32_t player_slots;
    int64_t state_cells;
    gen_params params;  // generator and episode parameters, spawn range included
};

size_t blob_bytes(const gen_env* e) {
    const size_t G = (size_t)e->G, n = (size_t)e->state_cells;
    return sizeof(BlobHeader) + 16 * G + 4 * n + sizeof(GameScalars) * G;
}

// FNV-1a, 64-bit (Fowler, Noll, Vo)
uint64_t fnv1a64(const unsigned char* p, size_t n) {
    uint64_t h = 1469598103934665603ULL;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ULL;
    }
    return h;
}

// Per-game derived fields of the game table from the parameters.
void apply_params(gen_env* e, const gen_params& p) {
    e->prm = p;
    for (size_t g = 0; g < e->h_info.size(); ++g) {
        GameInfo& gi = e->h_info[g];
        gi.game_id = p.game_id_base + (uint64_t)g;
        const int nc = p.n_cities >= 0 ? p.n_cities : (int)(((int64_t)gi.N * p.city_per_mille) / 1000);
        gi.n_cities = (int16_t)nc;
        const int d = p.min_general_dist >= 1 ? p.min_general_dist : (gi.H + gi.W) / 3;
        gi.dmin = (int16_t)(d < 1 ? 1 : d);
    }
}

}  // namespace

extern "C" {

int gen_read_state(gen_env* e, int16_t* h_army, int8_t* h_owner, int8_t* h_terrain, uint32_t* h_scalars,
                   void* stream) {
    if (!e) return fail(GEN_ERR_BAD_ARG, "env is NULL");
    return read_state_into(e, h_army, h_owner, h_terrain, h_scalars, (cudaStream_t)stream);
}

int gen_write_state(gen_env* e, const int16_t* h_army, const int8_t* h_owner, const int8_t* h_terrain,
                    const uint32_t* h_scalars, void* stream) {
    if (!e) return fail(GEN_ERR_BAD_ARG, "env is NULL");
    if (!h_army || !h_owner || !h_terrain || !h_scalars) return fail(GEN_ERR_BAD_ARG, "host buffers are NULL");
    int rc = validate_state(e, h_army, h_owner, h_terrain, h_scalars);
    if (rc) return rc;
    return upload_state(e, h_army, h_owner, h_terrain, h_scalars, false, (cudaStream_t)stream);
}

int gen_save_state(gen_env* e, void* h_buf, size_t cap, size_t* used, void* stream) {
    if (!e || !used) return fail(GEN_ERR_BAD_ARG, "env or used is NULL");
    const size_t need = blob_bytes(e);
    *used = need;
    if (!h_buf) return GEN_OK;  // size query
    if (cap < need) return fail(GEN_ERR_BAD_ARG, "buffer of %zu bytes; the saved state needs %zu", cap, need);
    const size_t G = (size_t)e->G, n = (size_t)e->state_cells;
    unsigned char* b = static_cast<unsigned char*>(h_buf);
    unsigned char* shapes = b + sizeof(BlobHeader);
    int16_t* army = reinterpret_cast<int16_t*>(shapes + 16 * G);
    int8_t* owner = reinterpret_cast<int8_t*>(shapes + 16 * G + 2 * n);
    int8_t* terrain = owner + n;
    unsigned char* scal = reinterpret_cast<unsigned char*>(terrain + n);
    // army sits at an even offset (header and shapes are multiples of 16 bytes)
    static_assert(sizeof(BlobHeader) % 16 == 0, "blob sections stay aligned");
    std::vector<uint32_t> sc(8 * G);
    int rc = read_state_into(e, army, owner, terrain, sc.data(), (cudaStream_t)stream);
    if (rc) return rc;
    memcpy(scal, sc.data(), sizeof(uint32_t) * 8 * G);
    for (size_t g = 0; g < G; ++g) {
        const GameInfo& gi = e->h_info[g];
        const int32_t v[4] = {gi.H, gi.W, gi.mode, gi.P};
        memcpy(shapes + 16 * g, v, 16);
    }
    BlobHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, kBlobMagic, 8);
    h.version = kBlobVersion;
    h.header_bytes = (uint32_t)sizeof(BlobHeader);
    h.total_bytes = need;
    h.n_games = e->G;
    h.player_slots = e->player_slots;
    h.state_cells = e->state_cells;
    h.params = e->prm;
    h.checksum = fnv1a64(b + sizeof(BlobHeader), need - sizeof(BlobHeader));
    memcpy(b, &h, sizeof(h));
    return GEN_OK;
}

int gen_load_state(gen_env* e, const void* h_buf, size_t size, void* stream) {
    if (!e || !h_buf) return fail(GEN_ERR_BAD_ARG, "env or buffer is NULL");
    if (size < sizeof(BlobHeader)) return fail(GEN_ERR_BAD_ARG, "saved state of %zu bytes is truncated", size);
    const unsigned char* b = static_cast<const unsigned char*>(h_buf);
    BlobHeader h;
    memcpy(&h, b, sizeof(h));
    if (memcmp(h.magic, kBlobMagic, 8) != 0) return fail(GEN_ERR_BAD_ARG, "not a saved environment state");
    if (h.version != kBlobVersion || h.header_bytes != sizeof(BlobHeader))
        return fail(GEN_ERR_BAD_ARG, "saved-state version %u (header %u bytes); this library reads version %u",
                    h.version, h.header_bytes, kBlobVersion);
    const size_t need = blob_bytes(e);
    if (h.n_games != e->G || h.state_cells != e->state_cells || h.player_slots != e->player_slots ||
        h.total_bytes != need || size < need)
        return fail(GEN_ERR_BAD_ARG, "saved state of %d games / %lld cells (%zu bytes) does not fit this environment "
                    "(%d games / %lld cells, %zu bytes)", h.n_games, (long long)h.state_cells, size, e->G,
                    (long long)e->state_cells, need);
    if (fnv1a64(b + sizeof(BlobHeader), need - sizeof(BlobHeader)) != h.checksum)
        return fail(GEN_ERR_BAD_ARG, "saved state is corrupt (checksum mismatch)");
    const size_t G = (size_t)e->G, n = (size_t)e->state_cells;
    const unsigned char* shapes = b + sizeof(BlobHeader);
    for (size_t g = 0; g < G; ++g) {
        int32_t v[4];
        memcpy(v, shapes + 16 * g, 16);
        const GameInfo& gi = e->h_info[g];
        if (v[0] != gi.H || v[1] != gi.W || v[2] != gi.mode || v[3] != gi.P)
            return fail(GEN_ERR_BAD_ARG, "game %zu: saved %dx%d mode %d with %d players, environment %dx%d mode %d "
                        "with %d players", g, v[0], v[1], v[2], v[3], gi.H, gi.W, gi.mode, gi.P);
    }
    int rc = check_params(&h.params);
    if (rc) return rc;
    // copies: the blob need not be aligned for int16 / uint32 access
    std::vector<int16_t> army(n);
    std::vector<uint32_t> sc(8 * G);
    memcpy(army.data(), shapes + 16 * G, 2 * n);
    const int8_t* owner = reinterpret_cast<const int8_t*>(shapes + 16 * G + 2 * n);
    const int8_t* terrain = owner + n;
    memcpy(sc.data(), terrain + n, sizeof(uint32_t) * 8 * G);
    if ((rc = validate_state(e, army.data(), owner, terrain, sc.data())) != GEN_OK) return rc;
    drop_graph(e);
    apply_params(e, h.params);
    CUDA_TRY(cudaMemcpy(e->d_info, e->h_info.data(), sizeof(GameInfo) * G, cudaMemcpyHostToDevice),
             "upload game table");
    return upload_state(e, army.data(), owner, terrain, sc.data(), true, (cudaStream_t)stream);
}

int gen_set_spawn_range(gen_env* e, int min_dist, int max_dist) {
    if (!e) return fail(GEN_ERR_BAD_ARG, "env is NULL");
    if (max_dist < 0 || max_dist > 32767 || min_dist > 32767)
        return fail(GEN_ERR_BAD_ARG, "spawn range [%d, %d] invalid", min_dist, max_dist);
    drop_graph(e);
    gen_params p = e->prm;
    p.min_general_dist = min_dist;
    p.max_general_dist = max_dist;
    apply_params(e, p);
    CUDA_TRY(cudaMemcpy(e->d_info, e->h_info.data(), sizeof(GameInfo) * (size_t)e->G, cudaMemcpyHostToDevice),
             "upload game table");
    return GEN_OK;
}

struct gen_features {
    gen_env* env = nullptr;
    int hist = 0;
    int window = 0;
    int form = 0;  // 0 by batch size, 1 one warp per game, 2 one CTA per game
    void* d_mem = nullptr;  // one allocation: headers, masks, last army, last turn, ring
    gk::FArgs args{};
};

int gen_features_create(gen_features** out, gen_env* e, int hist) { return gen_features_create_ex(out, e, hist, 0); }

int gen_features_create_ex(gen_features** out, gen_env* e, int hist, int window) {
    if (!out) return fail(GEN_ERR_BAD_ARG, "out is NULL");
    *out = nullptr;
    if (!e) return fail(GEN_ERR_BAD_ARG, "env is NULL");
    if (hist < 1 || hist > 16) return fail(GEN_ERR_BAD_ARG, "hist %d outside [1, 16]", hist);
    if (window < 0 || window > 4096) return fail(GEN_ERR_BAD_ARG, "window %d outside [0, 4096]", window);
    const int64_t pc = e->plane_cells;
    const size_t hdr = (size_t)e->player_slots * sizeof(uint4);
    const size_t bits = ((size_t)pc + 15) & ~(size_t)15;
    const size_t army = ((size_t)pc * 2 + 15) & ~(size_t)15;
    const size_t turn = (size_t)pc * 4;
    const size_t ring = (size_t)(hist + 1) * 2 * (size_t)pc * 2;
    const size_t series = (size_t)e->player_slots * (size_t)window * sizeof(int2);
    auto* f = new gen_features();
    f->env = e;
    f->hist = hist;
    f->window = window;
    char* m = nullptr;
    cudaError_t ce = cudaMalloc(&m, hdr + bits + army + turn + ring + series);
    if (ce != cudaSuccess) {
        delete f;
        return cuda_fail(ce, "cudaMalloc feature memory");
    }
    if ((ce = cudaMemset(m, 0, hdr)) != cudaSuccess) {
        cudaFree(m);
        delete f;
        return cuda_fail(ce, "clear feature headers");
    }
    f->d_mem = m;
    gk::FArgs& a = f->args;
    a.info = e->d_info;
    a.army = e->d_army;
    a.owner = e->d_owner;
    a.terrain = e->d_terrain;
    a.scal = e->d_scal;
    a.n_games = e->G;
    a.hist = hist;
    a.plane_cells = pc;
    a.hdr = reinterpret_cast<uint4*>(m);
    a.mem_bits = reinterpret_cast<uint8_t*>(m + hdr);
    a.mem_army = reinterpret_cast<int16_t*>(m + hdr + bits);
    a.mem_turn = reinterpret_cast<int32_t*>(m + hdr + bits + army);
    a.ring = reinterpret_cast<int16_t*>(m + hdr + bits + army + turn);
    a.npad_max = e->npad_max;
    a.window = window;
    a.series_ring = window > 0 ? reinterpret_cast<int2*>(m + hdr + bits + army + turn + ring) : nullptr;
    a.series_out = nullptr;
    *out = f;
    return GEN_OK;
}

int gen_features_series_layout(const gen_features* f, int32_t* window, int64_t* n_ints) {
    if (!f) return fail(GEN_ERR_BAD_ARG, "features is NULL");
    if (window) *window = f->window;
    if (n_ints) *n_ints = (int64_t)f->env->player_slots * f->window * 2;
    return GEN_OK;
}

int gen_features_layout(const gen_features* f, int32_t* channels, int64_t* n_floats) {
    if (!f) return fail(GEN_ERR_BAD_ARG, "features is NULL");
    const int C = 24 + 2 * f->hist;
    if (channels) *channels = C;
    if (n_floats) *n_floats = f->env->plane_cells * C;
    return GEN_OK;
}

int gen_features_build(gen_features* f, float* d_out, void* stream) {
    return gen_features_build_ex(f, d_out, nullptr, stream);
}

int gen_features_build_ex(gen_features* f, float* d_out, int32_t* d_series, void* stream) {
    if (!f || !d_out) return fail(GEN_ERR_BAD_ARG, "NULL argument");
    if (reinterpret_cast<uintptr_t>(d_out) & 15u) return fail(GEN_ERR_BAD_ARG, "d_out is not 16-byte aligned");
    if (d_series && f->window == 0) return fail(GEN_ERR_BAD_ARG, "this builder has no temporal window");
    if (reinterpret_cast<uintptr_t>(d_series) & 7u) return fail(GEN_ERR_BAD_ARG, "d_series is not 8-byte aligned");
    gk::FArgs a = f->args;
    a.out = d_out;
    a.series_out = reinterpret_cast<int2*>(d_series);
    const int rc = gk::launch_features(a, f->env->pmax, f->form, stream);
    if (rc != 0) return cuda_fail((cudaError_t)rc, "feature launch");
    return GEN_OK;
}

int gen_features_autotune(gen_features* f, float* d_out, int steps, int* form_out) {
    if (!f || !d_out) return fail(GEN_ERR_BAD_ARG, "NULL argument");
    if (steps < 1) return fail(GEN_ERR_BAD_ARG, "steps < 1");
    cudaStream_t s = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "autotune stream");
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    // the first build folds the current frame; the timed ones repeat it, so
    // both forms do the same work and the memory is as one build leaves it
    int rc = gen_features_build_ex(f, d_out, nullptr, s);
    float best = 1e30f;
    int best_form = f->form;
    for (int form : {1, 2}) {
        if (rc) break;
        f->form = form;
        auto build = [&]() { return gen_features_build_ex(f, d_out, nullptr, s); };
        const float ms = time_calls(build, steps, s, a, b);
        if (ms < best) {
            best = ms;
            best_form = form;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamDestroy(s);
    f->form = best_form;
    if (rc) return rc;
    if (form_out) *form_out = best_form;
    return GEN_OK;
}

int gen_features_set_form(gen_features* f, int form) {
    if (!f) return fail(GEN_ERR_BAD_ARG, "features is NULL");
    if (form < 0 || form > 2) return fail(GEN_ERR_BAD_ARG, "form %d outside [0, 2]", form);
    f->form = form;
    return GEN_OK;
}

void gen_features_destroy(gen_features* f) {
    if (!f) return;
    cudaFree(f->d_mem);
    delete f;
}

int gen_sample_actions(gen_env* e, const float* d_logits, uint64_t seed, int32_t* d_actions, uint8_t* d_mask9,
                       void* stream) {
    if (!e) return fail(GEN_ERR_BAD_ARG, "env is NULL");
    if (!d_logits && d_actions) return fail(GEN_ERR_BAD_ARG, "actions need logits");
    if (d_logits && !d_actions) return fail(GEN_ERR_BAD_ARG, "logits need an actions buffer");
    if (!d_logits && !d_mask9) return fail(GEN_ERR_BAD_ARG, "nothing to compute");
    if (!aligned4(d_actions)) return fail(GEN_ERR_BAD_ARG, "actions not 4-byte aligned");
    if (!aligned16(d_logits) || !aligned16(d_mask9))  // the mask rows are written 16 bytes at a time
        return fail(GEN_ERR_BAD_ARG, "logits and mask9 must be 16-byte aligned");
    gk::SArgs a{};
    a.info = e->d_info;
    a.army = e->d_army;
    a.owner = e->d_owner;
    a.terrain = e->d_terrain;
    a.scal = e->d_scal;
    a.n_games = e->G;
    a.logits = d_logits;
    a.seed = seed;
    a.actions = d_actions;
    a.mask9 = d_mask9;
    a.npad_max = e->npad_max;
    const int rc = gk::launch_sample(a, e->pmax, e->sample_form, stream);
    if (rc != 0) return cuda_fail((cudaError_t)rc, "sampler launch");
    return GEN_OK;
}

int gen_set_lane_groups(gen_env* e, int mode) {
    if (!e) return fail(GEN_ERR_BAD_ARG, "env is NULL");
    if (mode < 0 || mode > 2) return fail(GEN_ERR_BAD_ARG, "mode %d outside [0, 2]", mode);
    drop_graph(e);
    e->lane_groups = mode;
    return build_worklist(e);  // the work lists' lane-group widths follow the setting
}

int gen_set_batch_form(gen_env* e, int form) {
    if (!e) return fail(GEN_ERR_BAD_ARG, "env is NULL");
    if (form < 0 || form > 2) return fail(GEN_ERR_BAD_ARG, "form %d outside [0, 2]", form);
    drop_graph(e);
    e->batch_form = form;
    return GEN_OK;
}

int gen_set_sample_form(gen_env* e, int form) {
    if (!e) return fail(GEN_ERR_BAD_ARG, "env is NULL");
    if (form < 0 || form > 3) return fail(GEN_ERR_BAD_ARG, "form %d outside [0, 3]", form);
    e->sample_form = form;
    return GEN_OK;
}

int gen_set_launch(gen_env* e, int warps_per_cta) {
    if (!e) return fail(GEN_ERR_BAD_ARG, "env is NULL");
    if (warps_per_cta != 1 && warps_per_cta != 2 && warps_per_cta != 4 && warps_per_cta != 8)
        return fail(GEN_ERR_BAD_ARG, "warps_per_cta %d not in {1, 2, 4, 8}", warps_per_cta);
    for (auto& b : e->buckets)
        if (warps_per_cta * b.warp_smem > kMaxSmemPerCta)
            return fail(GEN_ERR_BAD_ARG, "%d warps need %d bytes of shared memory", warps_per_cta,
                        warps_per_cta * b.warp_smem);
    drop_graph(e);
    for (auto& b : e->buckets) {
        b.warps = warps_per_cta;
        b.tuned = true;
        int rc = shape_bucket(b);
        if (rc) return rc;
    }
    return GEN_OK;
}

}  // extern "C"

// The environment-wide launch choices of the autotuner, per batch signature.
struct TunedForms {
    int lane_groups, batch_form, rollout_form, sample_form;
};
static std::map<std::string, TunedForms> g_forms_cache;  // under g_tune_mu

// Lane-group width, batch form, rollout form (K = 8 frames) and sampler
// form, each timed on a scratch batch of the environment's own shapes and
// parameters (its games do not advance); cached per batch signature.
static int tune_env_forms(gen_env* e, int steps, int sms, std::string& rep) {
    char line[256];
    std::string sig = std::to_string(sms) + ":" + std::to_string(e->G);
    for (const Bucket& b : e->buckets)
        sig += ":" + std::to_string(cell_class(b.npad_max)) + "/" + std::to_string(player_class(b.pmax)) + "x" +
               std::to_string(b.n);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_forms_cache.find(sig);
        if (it != g_forms_cache.end()) {
            const TunedForms& f = it->second;
            e->lane_groups = f.lane_groups;
            e->batch_form = f.batch_form;
            e->rollout_form = f.rollout_form;
            e->sample_form = f.sample_form;
            snprintf(line, sizeof(line), "forms (cached): lanes %d, batch %d, rollout %d, sampler %d\n", f.lane_groups,
                     f.batch_form, f.rollout_form, f.sample_form);
            rep += line;
            return build_worklist(e);
        }
    }
    std::vector<int32_t> hh, ww, mm, pp;
    for (const GameInfo& gi : e->h_info) {
        hh.push_back(gi.H);
        ww.push_back(gi.W);
        mm.push_back(gi.mode);
        pp.push_back(gi.P);
    }
    gen_env* t = nullptr;
    int rc = gen_create_ex(&t, &e->prm, e->G, hh.data(), ww.data(), mm.data(), pp.data());
    if (rc) return rc;
    constexpr int K = 8;
    gen_outputs ko{};
    float* logits = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    const size_t pc = (size_t)t->plane_cells, ps = (size_t)t->player_slots, G = (size_t)t->G;
    cudaError_t ce = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreate(&a);
    if (ce == cudaSuccess) ce = cudaEventCreate(&b);
    if (ce == cudaSuccess) ce = cudaMalloc(&ko.obs_army, K * pc * 2);
    if (ce == cudaSuccess) ce = cudaMalloc(&ko.obs_owner, K * pc);
    if (ce == cudaSuccess) ce = cudaMalloc(&ko.obs_terrain, K * pc);
    if (ce == cudaSuccess) ce = cudaMalloc(&ko.obs_vis, K * pc);
    if (ce == cudaSuccess) ce = cudaMalloc(&ko.mask, K * pc);
    if (ce == cudaSuccess) ce = cudaMalloc(&ko.reward, K * ps * 4);
    if (ce == cudaSuccess) ce = cudaMalloc(&ko.scoreboard, K * ps * 8);
    if (ce == cudaSuccess) ce = cudaMalloc(&ko.done, K * G);
    if (ce == cudaSuccess) ce = cudaMalloc(&logits, pc * 9 * sizeof(float));
    if (ce == cudaSuccess) ce = cudaMemsetAsync(logits, 0, pc * 9 * sizeof(float), s);
    if (ce != cudaSuccess) rc = cuda_fail(ce, "autotune scratch");
    if (rc == GEN_OK) rc = ensure_internal_outputs(t);
    if (rc == GEN_OK) rc = gen_policy(t, 1, t->d_actions, s);
    TunedForms best{e->lane_groups, e->batch_form, e->rollout_form, e->sample_form};
    auto step = [&]() { return gen_step_policy(t, t->d_actions, &t->d_out, 1, t->d_actions, s); };
    if (rc == GEN_OK) {
        // lane groups: by batch size, a warp per game, or several per warp where the games allow
        float bt = 1e30f;
        rep += "lanes:";
        for (int lg : {0, 1, 2}) {
            if ((rc = gen_set_lane_groups(t, lg)) != GEN_OK) break;
            const float ms = time_calls(step, steps, s, a, b);
            snprintf(line, sizeof(line), " %d=%.4fms", lg, ms);
            rep += line;
            if (ms < bt) {
                bt = ms;
                best.lane_groups = lg;
            }
        }
        rep += "\n";
    }
    if (rc == GEN_OK) rc = gen_set_lane_groups(t, best.lane_groups);
    if (rc == GEN_OK && t->buckets.size() > 1) {
        float bt = 1e30f;
        rep += "batch:";
        for (int bf : {1, 2}) {
            t->batch_form = bf;
            const float ms = time_calls(step, steps, s, a, b);
            snprintf(line, sizeof(line), " %d=%.4fms", bf, ms);
            rep += line;
            if (ms < bt) {
                bt = ms;
                best.batch_form = bf;
            }
        }
        rep += "\n";
        t->batch_form = best.batch_form;
    }
    if (rc == GEN_OK) {
        float bt = 1e30f;
        rep += "rollout (per frame, K = 8):";
        for (int form : {GEN_ROLLOUT_RESIDENT, GEN_ROLLOUT_GRAPH, GEN_ROLLOUT_LAUNCHES}) {
            auto roll = [&]() { return gen_rollout(t, K, 1, t->d_actions, &ko, nullptr, form, s); };
            const float ms = time_calls(roll, std::max(1, steps / K), s, a, b) / K;
            snprintf(line, sizeof(line), " %d=%.4fms", form, ms);
            rep += line;
            if (ms < bt) {
                bt = ms;
                best.rollout_form = form;
            }
        }
        rep += "\n";
    }
    if (rc == GEN_OK) {
        float bt = 1e30f;
        rep += "sampler:";
        for (int form : {1, 2, 3}) {
            t->sample_form = form;
            auto samp = [&]() { return gen_sample_actions(t, logits, 1, t->d_actions, nullptr, s); };
            const float ms = time_calls(samp, steps, s, a, b);
            snprintf(line, sizeof(line), " %d=%.4fms", form, ms);
            rep += line;
            if (ms < bt) {
                bt = ms;
                best.sample_form = form;
            }
        }
        rep += "\n";
    }
    cudaFree(ko.obs_army);
    cudaFree(ko.obs_owner);
    cudaFree(ko.obs_terrain);
    cudaFree(ko.obs_vis);
    cudaFree(ko.mask);
    cudaFree(ko.reward);
    cudaFree(ko.scoreboard);
    cudaFree(ko.done);
    cudaFree(logits);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (s) cudaStreamDestroy(s);
    free_env(t);
    if (rc) return rc;
    e->lane_groups = best.lane_groups;
    e->batch_form = best.batch_form;
    e->rollout_form = best.rollout_form;
    e->sample_form = best.sample_form;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_forms_cache[sig] = best;
    }
    return build_worklist(e);
}

extern "C" {

int gen_autotune(gen_env* e, int steps, char* report, size_t report_cap) {
    if (!e) return fail(GEN_ERR_BAD_ARG, "env is NULL");
    if (steps < 1) return fail(GEN_ERR_BAD_ARG, "steps < 1");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    drop_graph(e);
    std::string rep;
    char line[256];
    {
        const int rc = tune_env_forms(e, steps, sms, rep);
        if (rc) return rc;
    }
    for (size_t bi = 0; bi < e->buckets.size(); ++bi) {
        Bucket& b = e->buckets[bi];
        const auto cls = std::make_pair(cell_class(b.npad_max), player_class(b.pmax));
        const auto key = std::make_tuple(cls.first, cls.second, sms);
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) {
                b.warps = it->second;
                b.tuned = true;
                int rc = shape_bucket(b);
                if (rc) return rc;
                snprintf(line, sizeof(line), "bucket %zu (%d games, <=%d cells, <=%d players): %d warps/CTA (cached)\n",
                         bi, b.n, b.npad_max, b.pmax, b.warps);
                rep += line;
                continue;
            }
        }
        // a scratch batch of this bucket's shapes: same parameters, its own state
        std::vector<int32_t> hh, ww, mm, pp;
        for (int g = 0; g < e->G; ++g) {
            const GameInfo& gi = e->h_info[(size_t)g];
            if (game_class(gi) != cls) continue;
            hh.push_back(gi.H);
            ww.push_back(gi.W);
            mm.push_back(gi.mode);
            pp.push_back(gi.P);
        }
        gen_env* t = nullptr;
        int rc = gen_create_ex(&t, &e->prm, (int)hh.size(), hh.data(), ww.data(), mm.data(), pp.data());
        if (rc) return rc;
        rc = ensure_internal_outputs(t);
        if (rc) {
            free_env(t);
            return rc;
        }
        cudaStream_t s;
        cudaEvent_t t0, t1;
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        cudaEventCreate(&t0);
        cudaEventCreate(&t1);
        float best = 1e30f;
        int best_w = b.warps;
        std::string trials;
        gen_policy(t, 1, t->d_actions, s);
        for (int w : {2, 4, 8}) {
            if (w * b.warp_smem > kMaxSmemPerCta) continue;
            if (gen_set_launch(t, w) != GEN_OK) continue;
            for (int k = 0; k < 3; ++k) gen_step_policy(t, t->d_actions, &t->d_out, 1, t->d_actions, s);
            cudaEventRecord(t0, s);
            for (int k = 0; k < steps; ++k) gen_step_policy(t, t->d_actions, &t->d_out, 1, t->d_actions, s);
            cudaEventRecord(t1, s);
            if (cudaEventSynchronize(t1) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, t0, t1);
            snprintf(line, sizeof(line), " %dw=%.3fms", w, ms / steps);
            trials += line;
            if (ms < best) {
                best = ms;
                best_w = w;
            }
        }
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
        cudaStreamDestroy(s);
        free_env(t);
        cudaError_t ce = cudaGetLastError();
        if (ce != cudaSuccess) return cuda_fail(ce, "autotune");
        b.warps = best_w;
        b.tuned = true;
        if ((rc = shape_bucket(b)) != GEN_OK) return rc;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune_cache[key] = best_w;
        }
        snprintf(line, sizeof(line), "bucket %zu (%d games, <=%d cells, <=%d players): %d warps/CTA;", bi, b.n,
                 b.npad_max, b.pmax, best_w);
        rep += line + trials + "\n";
    }
    if (report && report_cap) {
        const size_t n = std::min(report_cap - 1, rep.size());
        memcpy(report, rep.data(), n);
        report[n] = 0;
    }
    return GEN_OK;
}

int gen_copy_peak(size_t bytes, int reps, double* gbps) {
    if (!gbps || bytes < 16 || reps < 1) return fail(GEN_ERR_BAD_ARG, "bad copy-peak arguments");
    const size_t n16 = bytes / 16;
    void *src = nullptr, *dst = nullptr;
    CUDA_TRY(cudaMalloc(&src, n16 * 16), "cudaMalloc copy src");
    if (cudaMalloc(&dst, n16 * 16) != cudaSuccess) {
        cudaFree(src);
        return fail(GEN_ERR_OOM, "cudaMalloc copy dst");
    }
    cudaMemset(src, 1, n16 * 16);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    double best = 0.0;
    int rc = GEN_OK;
    for (int r = 0; r < reps + 1 && rc == GEN_OK; ++r) {
        cudaEventRecord(t0, nullptr);
        int lr = gk::launch_copy(src, dst, n16, sms * 8, nullptr);
        cudaEventRecord(t1, nullptr);
        cudaError_t ce = cudaEventSynchronize(t1);
        if (lr != 0 || ce != cudaSuccess) {
            rc = cuda_fail(lr ? (cudaError_t)lr : ce, "copy kernel");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t0, t1);
        if (r > 0) best = std::max(best, 2.0 * (double)n16 * 16.0 / (ms * 1e-3) / 1e9);
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFree(src);
    cudaFree(dst);
    *gbps = best;
    return rc;
}

const char* gen_last_error(void) { return g_err; }

void gen_destroy(gen_env* e) { free_env(e); }

}  // extern "C"
