// C-ABI of libgenerals (declared in include/generals.h): argument checks,
// device arenas, per-game layout, launches.  All game work runs in the
// kernels of gk_kernels.cu; this file never computes a rule.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
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

#define CUDA_TRY(expr, what)                  \
    do {                                      \
        cudaError_t e_ = (expr);              \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

constexpr int kMaxSmemPerCta = 227 * 1024;

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

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
    int nmax = 0;
    int nw_stride = 0;
    int warp_smem = 0;
    int warps_per_cta = 8;
    GameInfo* d_info = nullptr;
    GameScalars* d_scal = nullptr;
    int16_t* d_army = nullptr;
    int8_t* d_owner = nullptr;
    int8_t* d_terrain = nullptr;
    // staging for gen_step_host
    int32_t* d_actions = nullptr;
    gen_outputs d_out{};
    bool have_out = false;
};

namespace {

void free_env(gen_env* e) {
    if (!e) return;
    cudaFree(e->d_info);
    cudaFree(e->d_scal);
    cudaFree(e->d_army);
    cudaFree(e->d_owner);
    cudaFree(e->d_terrain);
    cudaFree(e->d_actions);
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

int check_params(const gen_params* p) {
    if (!p) return fail(GEN_ERR_BAD_ARG, "params is NULL");
    if (p->city_army_min < 0 || p->city_army_max < p->city_army_min || p->city_army_max > 32767)
        return fail(GEN_ERR_BAD_ARG, "castle army range [%d, %d] invalid", p->city_army_min, p->city_army_max);
    if (p->n_cities < 0 && (p->city_per_mille < 0 || p->city_per_mille > 1000))
        return fail(GEN_ERR_BAD_ARG, "city_per_mille %d outside [0, 1000]", p->city_per_mille);
    if (p->n_cities > 4096) return fail(GEN_ERR_BAD_ARG, "n_cities %d too large", p->n_cities);
    if (p->max_turns < 0) return fail(GEN_ERR_BAD_ARG, "max_turns < 0");
    return GEN_OK;
}

int check_outputs(const gen_env* e, const gen_outputs* o) {
    if (!o) return fail(GEN_ERR_BAD_ARG, "outputs is NULL");
    const void* ptrs[8] = {o->obs_army, o->obs_owner, o->obs_terrain, o->obs_vis,
                           o->mask,     o->reward,    o->scoreboard,  o->done};
    for (int i = 0; i < 8; ++i) {
        if (!ptrs[i]) return fail(GEN_ERR_BAD_ARG, "output field %d is NULL", i);
        if (i < 5 && !aligned16(ptrs[i])) return fail(GEN_ERR_BAD_ARG, "output plane %d not 16-byte aligned", i);
    }
    (void)e;
    return GEN_OK;
}

KArgs base_args(const gen_env* e, int op) {
    KArgs a;
    memset(&a, 0, sizeof(a));
    a.info = e->d_info;
    a.list = nullptr;
    a.n_items = e->G;
    a.n_games = e->G;
    a.op = op;
    a.army = e->d_army;
    a.owner = e->d_owner;
    a.terrain = e->d_terrain;
    a.scal = e->d_scal;
    a.seed = e->prm.seed;
    a.game_id_base = e->prm.game_id_base;
    a.mtn_thresh = e->prm.mountain_thresh;
    a.city_min = e->prm.city_army_min;
    a.city_span = e->prm.city_army_max - e->prm.city_army_min + 1;
    a.max_turns = e->prm.max_turns;
    a.auto_reset = e->prm.auto_reset;
    a.npad_max = e->npad_max;
    a.nw_stride = e->nw_stride;
    a.pmax = e->pmax;
    a.warp_smem = e->warp_smem;
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

int launch(const gen_env* e, const KArgs& a, void* stream, const char* what) {
    int rc = gk::launch_step(a, e->warps_per_cta, stream);
    if (rc != 0) return cuda_fail((cudaError_t)rc, what);
    return GEN_OK;
}

int players_for(int mode, int n_players) {
    if (mode == GEN_MODE_1V1) return 2;
    if (mode == GEN_MODE_2V2) return 4;
    return n_players;
}

int choose_warps(int warp_smem) {
    for (int w : {8, 4, 2, 1})
        if (w * warp_smem <= kMaxSmemPerCta) return w;
    return 0;
}

int ensure_internal_outputs(gen_env* e) {
    if (e->have_out) return GEN_OK;
    gen_outputs& o = e->d_out;
    const size_t pc = (size_t)e->plane_cells, ps = (size_t)e->player_slots;
    CUDA_TRY(cudaMalloc(&o.obs_army, pc * 2), "cudaMalloc obs_army");
    CUDA_TRY(cudaMalloc(&o.obs_owner, pc), "cudaMalloc obs_owner");
    CUDA_TRY(cudaMalloc(&o.obs_terrain, pc), "cudaMalloc obs_terrain");
    CUDA_TRY(cudaMalloc(&o.obs_vis, pc), "cudaMalloc obs_vis");
    CUDA_TRY(cudaMalloc(&o.mask, pc), "cudaMalloc mask");
    CUDA_TRY(cudaMalloc(&o.reward, ps * 4), "cudaMalloc reward");
    CUDA_TRY(cudaMalloc(&o.scoreboard, ps * 8), "cudaMalloc scoreboard");
    CUDA_TRY(cudaMalloc(&o.done, (size_t)e->G), "cudaMalloc done");
    CUDA_TRY(cudaMalloc(&e->d_actions, ps * 4), "cudaMalloc actions");
    e->have_out = true;
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
    }
    if (cell > INT32_MAX) {
        free_env(e);
        return fail(GEN_ERR_BAD_ARG, "batch too large: %lld state cells", (long long)cell);
    }
    e->state_cells = cell;
    e->plane_cells = plane;
    e->player_slots = slot;
    e->warp_smem = gk::warp_smem_bytes(e->npad_max, e->pmax, &e->nw_stride);
    e->warps_per_cta = choose_warps(e->warp_smem);

    cudaError_t ce;
    if ((ce = cudaMalloc(&e->d_info, sizeof(GameInfo) * (size_t)batch)) != cudaSuccess ||
        (ce = cudaMalloc(&e->d_scal, sizeof(GameScalars) * (size_t)batch)) != cudaSuccess ||
        (ce = cudaMalloc(&e->d_army, 2 * (size_t)cell)) != cudaSuccess ||
        (ce = cudaMalloc(&e->d_owner, (size_t)cell)) != cudaSuccess ||
        (ce = cudaMalloc(&e->d_terrain, (size_t)cell)) != cudaSuccess) {
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
    KArgs a = base_args(e, gk::OP_CREATE);
    rc = launch(e, a, nullptr, "create launch");
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

int gen_reset(gen_env* e, const int32_t* d_game_ids, int n, const gen_outputs* out, void* stream) {
    if (!e) return fail(GEN_ERR_BAD_ARG, "env is NULL");
    int rc = check_outputs(e, out);
    if (rc) return rc;
    KArgs a = base_args(e, gk::OP_RESET);
    if (d_game_ids) {
        if (n < 0 || n > e->G) return fail(GEN_ERR_BAD_ARG, "reset count %d outside [0, %d]", n, e->G);
        a.list = d_game_ids;
        a.n_items = n;
    }
    set_outputs(a, out);
    return launch(e, a, stream, "reset launch");
}

int gen_observe(gen_env* e, const gen_outputs* out, void* stream) {
    if (!e) return fail(GEN_ERR_BAD_ARG, "env is NULL");
    int rc = check_outputs(e, out);
    if (rc) return rc;
    KArgs a = base_args(e, gk::OP_OBSERVE);
    set_outputs(a, out);
    return launch(e, a, stream, "observe launch");
}

int gen_step_policy(gen_env* e, const int32_t* d_actions, const gen_outputs* out, uint64_t policy_seed,
                    int32_t* d_next_actions, void* stream) {
    if (!e) return fail(GEN_ERR_BAD_ARG, "env is NULL");
    if (!d_actions) return fail(GEN_ERR_BAD_ARG, "actions is NULL");
    int rc = check_outputs(e, out);
    if (rc) return rc;
    KArgs a = base_args(e, gk::OP_STEP);
    a.actions = d_actions;
    set_outputs(a, out);
    a.next_actions = d_next_actions;
    a.policy_seed = policy_seed;
    return launch(e, a, stream, "step launch");
}

int gen_step(gen_env* e, const int32_t* d_actions, const gen_outputs* out, void* stream) {
    return gen_step_policy(e, d_actions, out, 0, nullptr, stream);
}

int gen_policy(gen_env* e, uint64_t policy_seed, int32_t* d_actions, void* stream) {
    if (!e) return fail(GEN_ERR_BAD_ARG, "env is NULL");
    if (!d_actions) return fail(GEN_ERR_BAD_ARG, "actions is NULL");
    KArgs a = base_args(e, gk::OP_POLICY);
    a.next_actions = d_actions;
    a.policy_seed = policy_seed;
    return launch(e, a, stream, "policy launch");
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

int gen_read_state(gen_env* e, int16_t* h_army, int8_t* h_owner, int8_t* h_terrain, uint32_t* h_scalars,
                   void* stream) {
    if (!e) return fail(GEN_ERR_BAD_ARG, "env is NULL");
    cudaStream_t s = (cudaStream_t)stream;
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

int gen_write_state(gen_env* e, const int16_t* h_army, const int8_t* h_owner, const int8_t* h_terrain,
                    const uint32_t* h_scalars, void* stream) {
    if (!e) return fail(GEN_ERR_BAD_ARG, "env is NULL");
    if (!h_army || !h_owner || !h_terrain || !h_scalars) return fail(GEN_ERR_BAD_ARG, "host buffers are NULL");
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
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)e->state_cells;
    std::vector<GameScalars> sc((size_t)e->G);
    memcpy(sc.data(), h_scalars, sizeof(GameScalars) * (size_t)e->G);
    for (auto& x : sc) x.err = 0;
    CUDA_TRY(cudaMemcpyAsync(e->d_army, h_army, 2 * n, cudaMemcpyHostToDevice, s), "write army");
    CUDA_TRY(cudaMemcpyAsync(e->d_owner, h_owner, n, cudaMemcpyHostToDevice, s), "write owner");
    CUDA_TRY(cudaMemcpyAsync(e->d_terrain, h_terrain, n, cudaMemcpyHostToDevice, s), "write terrain");
    CUDA_TRY(cudaMemcpyAsync(e->d_scal, sc.data(), sizeof(GameScalars) * (size_t)e->G, cudaMemcpyHostToDevice, s),
             "write scalars");
    KArgs a = base_args(e, gk::OP_DERIVE);
    int rc = launch(e, a, stream, "derive launch");
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize(s), "write_state sync");
    return GEN_OK;
}

int gen_set_launch(gen_env* e, int warps_per_cta) {
    if (!e) return fail(GEN_ERR_BAD_ARG, "env is NULL");
    if (warps_per_cta != 1 && warps_per_cta != 2 && warps_per_cta != 4 && warps_per_cta != 8)
        return fail(GEN_ERR_BAD_ARG, "warps_per_cta %d not in {1, 2, 4, 8}", warps_per_cta);
    if (warps_per_cta * e->warp_smem > kMaxSmemPerCta)
        return fail(GEN_ERR_BAD_ARG, "%d warps need %d bytes of shared memory", warps_per_cta,
                    warps_per_cta * e->warp_smem);
    e->warps_per_cta = warps_per_cta;
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
