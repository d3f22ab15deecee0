// Env server of libgenerals: the games of many client sessions stay resident
// on the device and are stepped by continuous batching.  Clients submit step
// requests as they please; a scheduler thread folds every request waiting at
// that moment into one tick (one work-list launch over all
// their games), keeps up to two ticks in flight on one stream so that
// requests arriving while a tick runs are launched behind it and start on
// the device the moment it ends, and completes each request when its tick's
// event fires.  New sessions are
// admitted against a byte budget of device memory as earlier ones close.
//
// Every game keys its maps and policy draws by the global game id its
// session was opened with, so a session's results do not depend on the slots
// it got or on the other sessions in its ticks.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <random>
#include <thread>
#include <vector>

#include "generals.h"
#include "gk_internal.h"

using gk::GameInfo;
using gk::GameScalars;
using gk::KArgs;

namespace {

thread_local char s_err[512] = "no error";

int sfail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(s_err, sizeof(s_err), fmt, ap);
    va_end(ap);
    return code;
}

#define SCUDA(expr, what)                                                                                      \
    do {                                                                                                       \
        cudaError_t e_ = (expr);                                                                               \
        if (e_ != cudaSuccess) return sfail(GEN_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e_),           \
                                            cudaGetErrorString(e_));                                           \
    } while (0)

using Clock = std::chrono::steady_clock;
double now_ms() { return std::chrono::duration<double, std::milli>(Clock::now().time_since_epoch()).count(); }

constexpr int kMaxSmemPerCta = 227 * 1024;
constexpr int kTicks = 2;  // ticks in flight at once, one behind the other on the tick stream
constexpr double kTickDeadlineMs = 30000.0;  // a tick still running after this fails its requests

// First-fit allocator of index ranges in [0, cap), with coalescing.
class RangeAlloc {
  public:
    void reset(int64_t cap) {
        free_.clear();
        if (cap > 0) free_[0] = cap;
    }
    int64_t alloc(int64_t n, int64_t align) {
        if (n <= 0) return 0;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            const int64_t off = it->first, len = it->second;
            const int64_t start = (off + align - 1) / align * align;
            if (start + n > off + len) continue;
            free_.erase(it);
            if (start > off) free_[off] = start - off;
            if (off + len > start + n) free_[start + n] = off + len - (start + n);
            return start;
        }
        return -1;
    }
    void release(int64_t off, int64_t n) {
        if (n <= 0) return;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

  private:
    std::map<int64_t, int64_t> free_;
};

struct Session {
    int id = 0;
    int n = 0;
    int64_t g0 = 0, c0 = 0, p0 = 0, s0 = 0;  // first game slot, cell, plane cell, player slot
    int64_t cells = 0, planes = 0, slots = 0;
    size_t bytes = 0;  // device bytes charged to the budget
    int npad_max = 0, pmax = 0;
    std::vector<GameInfo> info;
    std::vector<std::pair<int, std::vector<int32_t>>> by_class;  // class index -> game slots
    bool busy = false;
};

struct Request {
    int session = 0;
    double t_submit = 0;
    bool done = false;
    int rc = GEN_OK;
    std::mutex m;
    std::condition_variable cv;
};

struct ClassShape {
    int npad_max = 0, pmax = 0, nw_stride = 0, warp_smem = 0, warps = 2, max_ctas = 0;
};

struct Tick {
    cudaStream_t stream = nullptr;  // the server's tick stream (shared by every tick)
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr, done = nullptr;
    cudaEvent_t t_start = nullptr, t_end = nullptr;  // timing: the tick's device time
    int32_t* d_list = nullptr;
    int32_t* h_list = nullptr;  // pinned
    gk::WorkItem* d_items = nullptr;  // the tick's work list (one launch over every class)
    gk::WorkItem* h_items = nullptr;  // pinned
    int32_t* d_counter = nullptr;
    std::vector<Request*> reqs;
    bool busy = false;
    double t_launch = 0;
    int64_t games = 0;
};

int cell_class(int npad) {
    for (int edge : {256, 512, 768, 1024, 1536, 2048, 3072, 4096})
        if (npad <= edge) return edge;
    return 4096;
}
int player_class(int P) { return P <= 2 ? 2 : (P <= 4 ? 4 : 8); }

// size classes in launch order (largest first): 8 cell edges x 3 player classes
constexpr int kClasses = 24;
int class_index(int npad, int P) {
    int ci = 0;
    for (int edge : {256, 512, 768, 1024, 1536, 2048, 3072, 4096}) {
        if (npad <= edge) break;
        ++ci;
    }
    ci = ci > 7 ? 7 : ci;
    const int pi = P <= 2 ? 0 : (P <= 4 ? 1 : 2);
    return (7 - ci) * 3 + (2 - pi);
}
int class_edge(int idx) {
    static const int edges[8] = {256, 512, 768, 1024, 1536, 2048, 3072, 4096};
    return edges[7 - idx / 3];
}
int class_players(int idx) { return 8 >> (idx % 3); }

}  // namespace

struct gen_server {
    int device = 0;
    gen_params prm{};
    uint64_t policy_seed = 0;
    int host_outputs = 1;
    size_t budget = 0, in_use = 0;
    int64_t cap_games = 0, cap_cells = 0, cap_planes = 0, cap_slots = 0;
    RangeAlloc a_games, a_cells, a_planes, a_slots;
    GameInfo* d_info = nullptr;
    GameScalars* d_scal = nullptr;
    int16_t* d_army = nullptr;
    int8_t* d_owner = nullptr;
    int8_t* d_terrain = nullptr;
    // outputs and actions: mapped host memory (host clients) or device memory
    gen_outputs out_host{};  // host view (host mode) / NULLs
    gen_outputs out_dev{};   // device view used by the kernel
    int32_t* act_host = nullptr;
    int32_t* act_dev = nullptr;
    cudaStream_t admin = nullptr;
    Tick ticks[kTicks];
    // every tick runs on this one stream: a tick launched while another runs
    // waits behind it, so the device goes from one to the next without a gap
    // and two ticks never split its SMs
    cudaStream_t tick_stream = nullptr;
    std::map<std::pair<int, int>, ClassShape> shapes;
    // work-list launches: per size class its geometry, items of a CTA's worth of games
    gk::BucketGeom* d_geoms = nullptr;
    int class_per_item[kClasses] = {};
    int wl_smem = 0, wl_ctas = 0;
    std::mutex mu;
    std::condition_variable cv_req, cv_admit;
    std::deque<Request*> queue;
    std::map<int, Session> sessions;
    int next_id = 1;
    bool stop = false;
    std::thread sched;
    // statistics
    std::mutex stat_mu;
    std::vector<double> lat;
    uint64_t frames = 0, requests = 0, tick_count = 0, admitted = 0, waited = 0, waited_budget = 0;
    double tick_gpu_ms_sum = 0, tick_host_ms_sum = 0;
    size_t peak_in_use = 0;  // under mu
    double t0 = 0, tick_games_sum = 0;
    std::string fatal;
};

namespace {

int class_shape(gen_server* sv, int npad, int P, ClassShape* out) {
    const auto key = std::make_pair(cell_class(npad), player_class(P));
    auto it = sv->shapes.find(key);
    if (it != sv->shapes.end()) {
        *out = it->second;
        return GEN_OK;
    }
    ClassShape c;
    c.npad_max = key.first;
    c.pmax = key.second;
    c.warp_smem = gk::warp_smem_bytes(c.npad_max, c.pmax, &c.nw_stride);
    c.warps = 0;
    for (int w : {2, 1})  // 2 games per CTA: the autotuner's choice for mixed large boards
        if (w * c.warp_smem <= kMaxSmemPerCta) {
            c.warps = w;
            break;
        }
    if (c.warps == 0) return sfail(GEN_ERR_BAD_ARG, "board of %d cells does not fit shared memory", npad);
    const int rc = gk::max_resident_ctas(c.warps, c.warps * c.warp_smem, &c.max_ctas);
    if (rc) return sfail(GEN_ERR_CUDA, "occupancy query failed (%d)", rc);
    sv->shapes[key] = c;
    *out = c;
    return GEN_OK;
}

KArgs server_args(gen_server* sv, int op, const ClassShape& c) {
    KArgs a;
    memset(&a, 0, sizeof(a));
    a.info = sv->d_info;
    a.n_games = (int32_t)sv->cap_games;
    a.op = op;
    a.army = sv->d_army;
    a.owner = sv->d_owner;
    a.terrain = sv->d_terrain;
    a.scal = sv->d_scal;
    a.actions = sv->act_dev;
    a.obs_army = sv->out_dev.obs_army;
    a.obs_owner = sv->out_dev.obs_owner;
    a.obs_terrain = sv->out_dev.obs_terrain;
    a.obs_vis = sv->out_dev.obs_vis;
    a.mask = sv->out_dev.mask;
    a.reward = sv->out_dev.reward;
    a.scoreboard = sv->out_dev.scoreboard;
    a.done = sv->out_dev.done;
    a.do_outputs = 1;
    a.next_actions = sv->act_dev;
    a.policy_seed = sv->policy_seed;
    a.seed = sv->prm.seed;
    a.mtn_thresh = sv->prm.mountain_thresh;
    a.spawn_dmax = std::max(sv->prm.max_general_dist, 0);
    a.spawn_bfs = sv->prm.bfs_distance ? 1 : 0;
    a.castle_radius = std::max(sv->prm.castle_radius, 0);
    a.city_min = sv->prm.city_army_min;
    a.city_span = sv->prm.city_army_max - sv->prm.city_army_min + 1;
    a.max_turns = sv->prm.max_turns;
    a.auto_reset = sv->prm.auto_reset;
    a.frames = 1;
    a.plane_stride = sv->cap_planes;
    a.slot_stride = (int32_t)sv->cap_slots;
    a.game_stride = (int32_t)sv->cap_games;
    a.npad_max = c.npad_max;
    a.nw_stride = c.nw_stride;
    a.pmax = c.pmax;
    a.warp_smem = c.warp_smem;
    return a;
}

void finish_request(Request* r, int rc) {
    std::lock_guard<std::mutex> lk(r->m);
    r->rc = rc;
    r->done = true;
    r->cv.notify_all();
}

// Launch one tick over every game of the sessions `ss` (busy sessions: their
// game lists do not change).  With spawn options the per-class launches
// need sv->mu held (class shapes are cached in a shared map); the work-list
// launch reads nothing shared that can change and runs without it.
int launch_tick(gen_server* sv, Tick& t, const std::vector<const Session*>& ss, const ClassShape& base) {
    int64_t count[kClasses] = {0};
    int64_t games = 0;
    for (const Session* sp : ss) {
        for (auto& kv : sp->by_class) count[kv.first] += (int64_t)kv.second.size();
        games += sp->n;
    }
    int64_t start[kClasses], fill[kClasses];
    int64_t k = 0;
    for (int c = 0; c < kClasses; ++c) {
        start[c] = fill[c] = k;
        k += count[c];
    }
    for (const Session* s : ss)
        for (auto& kv : s->by_class) {
            memcpy(t.h_list + fill[kv.first], kv.second.data(), sizeof(int32_t) * kv.second.size());
            fill[kv.first] += (int64_t)kv.second.size();
        }
    SCUDA(cudaEventRecord(t.t_start, t.stream), "tick timing");
    SCUDA(cudaMemcpyAsync(t.d_list, t.h_list, sizeof(int32_t) * (size_t)k, cudaMemcpyHostToDevice, t.stream),
          "tick list upload");
    const bool spawn = sv->prm.max_general_dist > 0 || sv->prm.bfs_distance || sv->prm.castle_radius > 0;
    bool fits = true;
    for (int c = 0; c < kClasses; ++c) fits = fits && (count[c] == 0 || sv->class_per_item[c] >= 1);
    if (!spawn && fits) {
        // one persistent work-list launch over every class of the tick
        int n_items = 0;
        for (int c = 0; c < kClasses; ++c)
            for (int64_t j = 0; j < count[c]; j += sv->class_per_item[c]) {
                gk::WorkItem& it = t.h_items[n_items++];
                it.first = (int32_t)(start[c] + j);
                it.count = (int32_t)std::min<int64_t>(sv->class_per_item[c], count[c] - j);
                it.bucket = c;
                it.pad = 0;
            }
        SCUDA(cudaMemcpyAsync(t.d_items, t.h_items, sizeof(gk::WorkItem) * (size_t)n_items, cudaMemcpyHostToDevice,
                              t.stream),
              "tick work-list upload");
        KArgs a = server_args(sv, gk::OP_STEP, base);  // geometry comes with each item
        gk::WArgs w;
        int rc;
        w.items = t.d_items;
        w.n_items = n_items;
        w.geoms = sv->d_geoms;
        w.order = t.d_list;
        w.counter = t.d_counter;
        rc = gk::launch_worklist(a, w, sv->wl_smem, sv->wl_ctas, t.stream);
        if (rc) return sfail(GEN_ERR_CUDA, "tick launch: %s", cudaGetErrorString((cudaError_t)rc));
        SCUDA(cudaEventRecord(t.t_end, t.stream), "tick timing");
    SCUDA(cudaEventRecord(t.done, t.stream), "tick event");
        t.busy = true;
        t.games = games;
        t.t_launch = now_ms();
        return GEN_OK;
    }
    int used = 0;
    for (int c = 0; c < kClasses; ++c) used += count[c] > 0;
    if (used > 1) SCUDA(cudaEventRecord(t.fork, t.stream), "fork");
    int i = 0;
    for (int c = 0; c < kClasses; ++c) {
        if (!count[c]) continue;
        ClassShape cs;
        int rc = class_shape(sv, class_edge(c), class_players(c), &cs);
        if (rc) return rc;
        KArgs a = server_args(sv, gk::OP_STEP, cs);
        a.list = t.d_list + start[c];
        a.n_items = (int32_t)count[c];
        cudaStream_t s = i == 0 ? t.stream : t.side[(size_t)i - 1];
        if (i > 0) SCUDA(cudaStreamWaitEvent(s, t.fork, 0), "fork wait");
        rc = gk::launch_step(a, cs.warps, cs.max_ctas, s);
        if (rc) return sfail(GEN_ERR_CUDA, "tick launch: %s", cudaGetErrorString((cudaError_t)rc));
        if (i > 0) {
            SCUDA(cudaEventRecord(t.join[(size_t)i - 1], s), "join");
            SCUDA(cudaStreamWaitEvent(t.stream, t.join[(size_t)i - 1], 0), "join wait");
        }
        ++i;
    }
    SCUDA(cudaEventRecord(t.t_end, t.stream), "tick timing");
    SCUDA(cudaEventRecord(t.done, t.stream), "tick event");
    t.busy = true;
    t.games = games;
    t.t_launch = now_ms();
    return GEN_OK;
}

int busy_ticks(const gen_server* sv) {
    int n = 0;
    for (const Tick& t : sv->ticks) n += t.busy ? 1 : 0;
    return n;
}

void scheduler(gen_server* sv) {
    cudaSetDevice(sv->device);
    std::vector<std::pair<Request*, int>> finished;
    std::unique_lock<std::mutex> lk(sv->mu);
    while (true) {
        const bool any_busy = busy_ticks(sv) > 0;
        if (sv->stop && sv->queue.empty() && !any_busy) break;
        // complete finished ticks (poll with a deadline)
        for (Tick& t : sv->ticks) {
            if (!t.busy) continue;
            const cudaError_t q = cudaEventQuery(t.done);
            int rc = GEN_OK;
            if (q == cudaErrorNotReady) {
                if (now_ms() - t.t_launch < kTickDeadlineMs) continue;
                rc = sfail(GEN_ERR_TIMEOUT, "tick still running after %.0f ms", kTickDeadlineMs);
                sv->fatal = s_err;
            } else if (q != cudaSuccess) {
                rc = sfail(GEN_ERR_CUDA, "tick failed: %s", cudaGetErrorString(q));
                sv->fatal = s_err;
            }
            float gpu_ms = 0.f;
            if (rc == GEN_OK) cudaEventElapsedTime(&gpu_ms, t.t_start, t.t_end);
            {
                std::lock_guard<std::mutex> sl(sv->stat_mu);
                sv->tick_gpu_ms_sum += gpu_ms;
                sv->tick_count += 1;
                sv->tick_games_sum += (double)t.games;
                if (rc == GEN_OK) sv->frames += (uint64_t)t.games;
            }
            for (Request* r : t.reqs) {
                sv->sessions[r->session].busy = false;
                finished.emplace_back(r, rc);
            }
            t.reqs.clear();
            t.busy = false;
        }
        if (!finished.empty()) {  // wake the clients without holding the server lock
            lk.unlock();
            for (auto& fr : finished) finish_request(fr.first, fr.second);
            finished.clear();
            lk.lock();
        }
        // start a tick with every waiting request
        if (!sv->queue.empty()) {
            Tick* free_t = nullptr;
            for (Tick& t : sv->ticks)
                if (!t.busy && !free_t) free_t = &t;
            if (free_t && sv->fatal.empty()) {
                free_t->reqs.assign(sv->queue.begin(), sv->queue.end());
                sv->queue.clear();
                std::vector<const Session*> ss;
                ss.reserve(free_t->reqs.size());
                for (Request* r : free_t->reqs) ss.push_back(&sv->sessions.find(r->session)->second);
                ClassShape base;
                int rc = class_shape(sv, 256, 2, &base);
                const double h0 = now_ms();
                if (rc == GEN_OK) {
                    free_t->busy = true;  // taken: only this thread starts or completes ticks
                    const bool spawn = sv->prm.max_general_dist > 0 || sv->prm.bfs_distance || sv->prm.castle_radius > 0;
                    if (!spawn) lk.unlock();
                    rc = launch_tick(sv, *free_t, ss, base);
                    if (!spawn) lk.lock();
                }
                {
                    std::lock_guard<std::mutex> sl(sv->stat_mu);
                    sv->tick_host_ms_sum += now_ms() - h0;
                }
                if (rc) {
                    sv->fatal = s_err;
                    for (Request* r : free_t->reqs) {
                        sv->sessions[r->session].busy = false;
                        finish_request(r, rc);
                    }
                    free_t->reqs.clear();
                    free_t->busy = false;
                }
                continue;
            }
            if (!sv->fatal.empty()) {
                for (Request* r : sv->queue) {
                    sv->sessions[r->session].busy = false;
                    finish_request(r, GEN_ERR_STATE);
                }
                sv->queue.clear();
            }
        }
        // sleep until a request arrives or a running tick may have finished
        const bool busy_now = busy_ticks(sv) > 0;
        sv->cv_req.wait_for(lk, std::chrono::microseconds(busy_now ? 20 : 2000));
    }
}

void free_server(gen_server* sv) {
    if (!sv) return;
    for (Tick& t : sv->ticks) {
        for (auto s : t.side) cudaStreamDestroy(s);
        for (auto e : t.join) cudaEventDestroy(e);
        if (t.fork) cudaEventDestroy(t.fork);
        if (t.done) cudaEventDestroy(t.done);
        if (t.t_start) cudaEventDestroy(t.t_start);
        if (t.t_end) cudaEventDestroy(t.t_end);

        cudaFree(t.d_list);
        cudaFreeHost(t.h_list);
        cudaFree(t.d_items);
        cudaFreeHost(t.h_items);
        cudaFree(t.d_counter);
    }
    cudaFree(sv->d_geoms);
    if (sv->admin) cudaStreamDestroy(sv->admin);
    if (sv->tick_stream) cudaStreamDestroy(sv->tick_stream);
    cudaFree(sv->d_info);
    cudaFree(sv->d_scal);
    cudaFree(sv->d_army);
    cudaFree(sv->d_owner);
    cudaFree(sv->d_terrain);
    auto release = [&](void* p) {
        if (!p) return;
        if (sv->host_outputs)
            cudaFreeHost(p);
        else
            cudaFree(p);
    };
    gen_outputs& o = sv->host_outputs ? sv->out_host : sv->out_dev;
    release(o.obs_army);
    release(o.obs_owner);
    release(o.obs_terrain);
    release(o.obs_vis);
    release(o.mask);
    release(o.reward);
    release(o.scoreboard);
    release(o.done);
    if (sv->act_host) cudaFreeHost(sv->act_host);
    delete sv;
}

}  // namespace

extern "C" {

const char* gen_server_last_error(void) { return s_err; }

int gen_server_create(gen_server** out, const gen_params* p, const gen_server_config* cfg) {
    if (!out || !p || !cfg) return sfail(GEN_ERR_BAD_ARG, "NULL argument");
    *out = nullptr;
    if (cfg->max_games < 1 || cfg->max_games > (1 << 26))
        return sfail(GEN_ERR_BAD_ARG, "max_games %lld outside [1, 2^26]", (long long)cfg->max_games);
    if (cfg->max_cells < 16 || cfg->max_cells > (int64_t)INT32_MAX - 4096)
        return sfail(GEN_ERR_BAD_ARG, "max_cells %lld outside [16, 2^31 - 4096]", (long long)cfg->max_cells);
    if (cfg->max_plane_cells < 16) return sfail(GEN_ERR_BAD_ARG, "max_plane_cells below 16");
    if (cfg->budget_bytes < 4096) return sfail(GEN_ERR_BAD_ARG, "budget below 4 KiB");
    if (p->max_general_dist < 0 || p->castle_radius < 0 || p->castle_radius > 127)
        return sfail(GEN_ERR_BAD_ARG, "spawn cap %d or castle radius %d invalid", p->max_general_dist, p->castle_radius);
    {
        const int trc = gk::init_tables();
        if (trc != 0) return sfail(GEN_ERR_CUDA, "device tables: %s", cudaGetErrorString((cudaError_t)trc));
    }
    gen_server* sv = new gen_server();
    cudaGetDevice(&sv->device);
    sv->prm = *p;
    sv->policy_seed = cfg->policy_seed;
    sv->host_outputs = cfg->host_outputs ? 1 : 0;
    sv->budget = cfg->budget_bytes;
    sv->cap_games = cfg->max_games;
    sv->cap_cells = cfg->max_cells;
    sv->cap_planes = cfg->max_plane_cells;
    sv->cap_slots = 8 * cfg->max_games;
    sv->a_games.reset(sv->cap_games);
    sv->a_cells.reset(sv->cap_cells);
    sv->a_planes.reset(sv->cap_planes);
    sv->a_slots.reset(sv->cap_slots);
    cudaError_t ce = cudaSuccess;
    auto dev_alloc = [&](void** ptr, size_t n) {
        if (ce == cudaSuccess) ce = cudaMalloc(ptr, n);
    };
    dev_alloc((void**)&sv->d_info, sizeof(GameInfo) * (size_t)sv->cap_games);
    dev_alloc((void**)&sv->d_scal, sizeof(GameScalars) * (size_t)sv->cap_games);
    dev_alloc((void**)&sv->d_army, 2 * (size_t)sv->cap_cells);
    dev_alloc((void**)&sv->d_owner, (size_t)sv->cap_cells);
    dev_alloc((void**)&sv->d_terrain, (size_t)sv->cap_cells);
    const size_t pc = (size_t)sv->cap_planes, ps = (size_t)sv->cap_slots, G = (size_t)sv->cap_games;
    const size_t osz[9] = {pc * 2, pc, pc, pc, pc, ps * 4, ps * 8, G, ps * 4};
    void* optr[9] = {};
    // outputs: mapped host memory or device memory; actions: always mapped host
    // memory, so clients pass them without any CUDA call
    for (int i = 0; i < 9 && ce == cudaSuccess; ++i) {
        if (sv->host_outputs || i == 8) {
            ce = cudaHostAlloc(&optr[i], osz[i], cudaHostAllocMapped | cudaHostAllocPortable);
        } else {
            ce = cudaMalloc(&optr[i], osz[i]);
        }
    }
    gen_outputs& o = sv->host_outputs ? sv->out_host : sv->out_dev;
    o.obs_army = (int16_t*)optr[0];
    o.obs_owner = (int8_t*)optr[1];
    o.obs_terrain = (int8_t*)optr[2];
    o.obs_vis = (uint8_t*)optr[3];
    o.mask = (uint8_t*)optr[4];
    o.reward = (float*)optr[5];
    o.scoreboard = (int32_t*)optr[6];
    o.done = (uint8_t*)optr[7];
    if (sv->host_outputs) {
        sv->act_host = (int32_t*)optr[8];
        void* dp[9] = {};
        for (int i = 0; i < 9 && ce == cudaSuccess; ++i) ce = cudaHostGetDevicePointer(&dp[i], optr[i], 0);
        sv->out_dev.obs_army = (int16_t*)dp[0];
        sv->out_dev.obs_owner = (int8_t*)dp[1];
        sv->out_dev.obs_terrain = (int8_t*)dp[2];
        sv->out_dev.obs_vis = (uint8_t*)dp[3];
        sv->out_dev.mask = (uint8_t*)dp[4];
        sv->out_dev.reward = (float*)dp[5];
        sv->out_dev.scoreboard = (int32_t*)dp[6];
        sv->out_dev.done = (uint8_t*)dp[7];
        sv->act_dev = (int32_t*)dp[8];
    } else {
        sv->act_host = (int32_t*)optr[8];
        void* dp = nullptr;
        if (ce == cudaSuccess) ce = cudaHostGetDevicePointer(&dp, optr[8], 0);
        sv->act_dev = (int32_t*)dp;
    }
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&sv->admin, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&sv->tick_stream, cudaStreamNonBlocking);
    for (Tick& t : sv->ticks) {
        t.stream = sv->tick_stream;
        if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&t.fork, cudaEventDisableTiming);
        if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&t.done, cudaEventDisableTiming);
        if (ce == cudaSuccess) ce = cudaEventCreate(&t.t_start);
        if (ce == cudaSuccess) ce = cudaEventCreate(&t.t_end);
        if (ce == cudaSuccess) ce = cudaMalloc(&t.d_list, sizeof(int32_t) * G);
        if (ce == cudaSuccess) ce = cudaHostAlloc(&t.h_list, sizeof(int32_t) * G, cudaHostAllocPortable);
        if (ce == cudaSuccess) ce = cudaMalloc(&t.d_items, sizeof(gk::WorkItem) * G);
        if (ce == cudaSuccess) ce = cudaHostAlloc(&t.h_items, sizeof(gk::WorkItem) * G, cudaHostAllocPortable);
        if (ce == cudaSuccess) ce = cudaMalloc(&t.d_counter, 2 * sizeof(int32_t));
        if (ce == cudaSuccess) {  // afterwards each work-list launch leaves them zeroed
            const int32_t zero[2] = {0, 0};
            ce = cudaMemcpy(t.d_counter, zero, sizeof(zero), cudaMemcpyHostToDevice);
        }
        for (int i = 0; i < 24 && ce == cudaSuccess; ++i) {  // one per size class
            cudaStream_t s;
            cudaEvent_t v;
            ce = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
            if (ce == cudaSuccess) t.side.push_back(s);
            if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&v, cudaEventDisableTiming);
            if (ce == cudaSuccess) t.join.push_back(v);
        }
    }
    if (ce == cudaSuccess) {
        // the work-list kernel's launch shape and every size class's geometry
        int rc = gk::worklist_shape(false, &sv->wl_smem, &sv->wl_ctas);
        ce = (cudaError_t)rc;
        gk::BucketGeom geoms[kClasses];
        for (int c = 0; c < kClasses && ce == cudaSuccess; ++c) {
            int st = 0;
            const int npad = class_edge(c), P = class_players(c);
            geoms[c].lw = (P <= 2 && npad <= 1024) ? 16 : 32;
            const int bytes = gk::warp_smem_bytes(npad, P, &st, geoms[c].lw < 32);
            geoms[c].geom = gk::bucket_geom(npad, st, P, geoms[c].lw < 32);
            geoms[c].group_smem = bytes;
            geoms[c].pad = 0;
            sv->class_per_item[c] = std::min(8 * (32 / geoms[c].lw), sv->wl_smem / bytes);
        }
        if (ce == cudaSuccess) ce = cudaMalloc(&sv->d_geoms, sizeof(geoms));
        if (ce == cudaSuccess) ce = cudaMemcpy(sv->d_geoms, geoms, sizeof(geoms), cudaMemcpyHostToDevice);
    }
    if (ce != cudaSuccess) {
        free_server(sv);
        return ce == cudaErrorMemoryAllocation ? sfail(GEN_ERR_OOM, "server allocation failed")
                                               : sfail(GEN_ERR_CUDA, "server setup: %s", cudaGetErrorString(ce));
    }
    sv->t0 = now_ms();
    sv->sched = std::thread(scheduler, sv);
    *out = sv;
    return GEN_OK;
}

int gen_server_open(gen_server* sv, int n, const int32_t* h_H, const int32_t* h_W, const int32_t* h_mode,
                    const int32_t* h_n_players, uint64_t game_id_base, int wait_ms, int32_t* h_first_actions,
                    int32_t* session_out) {
    if (!sv || !session_out || !h_H || !h_W || !h_mode) return sfail(GEN_ERR_BAD_ARG, "NULL argument");
    if (n < 1) return sfail(GEN_ERR_BAD_ARG, "session of %d games", n);
    Session s;
    s.n = n;
    s.info.resize((size_t)n);
    for (int g = 0; g < n; ++g) {
        const int H = h_H[g], W = h_W[g], mode = h_mode[g];
        const int P = mode == GEN_MODE_1V1 ? 2 : mode == GEN_MODE_2V2 ? 4 : (h_n_players ? h_n_players[g] : 8);
        if (H < 1 || W < 1 || H > GEN_MAX_SIDE || W > GEN_MAX_SIDE || mode < 0 || mode > 2 || P < 2 ||
            P > GEN_MAX_PLAYERS || H * W < P)
            return sfail(GEN_ERR_BAD_ARG, "game %d: %dx%d mode %d with %d players", g, H, W, mode, P);
        GameInfo& gi = s.info[(size_t)g];
        memset(&gi, 0, sizeof(gi));
        const int N = H * W, Npad = (N + 15) & ~15;
        gi.H = (int16_t)H;
        gi.W = (int16_t)W;
        gi.N = (int16_t)N;
        gi.Npad = (int16_t)Npad;
        gi.mode = (int8_t)mode;
        gi.P = (int8_t)P;
        gi.game_id = game_id_base + (uint64_t)g;
        const int nc = sv->prm.n_cities >= 0 ? sv->prm.n_cities : (int)(((int64_t)N * sv->prm.city_per_mille) / 1000);
        gi.n_cities = (int16_t)nc;
        const int d = sv->prm.min_general_dist >= 1 ? sv->prm.min_general_dist : (H + W) / 3;
        gi.dmin = (int16_t)(d < 1 ? 1 : d);
        s.cells += Npad;
        s.planes += (int64_t)P * Npad;
        s.slots += P;
        s.npad_max = std::max(s.npad_max, Npad);
        s.pmax = std::max(s.pmax, P);
    }
    s.bytes = (size_t)s.cells * 4 + (size_t)n * (sizeof(GameInfo) + sizeof(GameScalars)) +
              (sv->host_outputs ? 0 : (size_t)s.planes * 6 + (size_t)s.slots * 16 + (size_t)n);
    if (s.bytes > sv->budget) return sfail(GEN_ERR_OOM, "session needs %zu bytes, budget is %zu", s.bytes, sv->budget);
    {
        std::unique_lock<std::mutex> lk(sv->mu);
        const auto deadline = Clock::now() + std::chrono::milliseconds(wait_ms > 0 ? wait_ms : 0);
        bool waited = false, over_budget = false;
        while (true) {
            if (!sv->fatal.empty()) return sfail(GEN_ERR_STATE, "server failed: %s", sv->fatal.c_str());
            if (sv->in_use + s.bytes > sv->budget) over_budget = true;
            if (sv->in_use + s.bytes <= sv->budget) {
                s.g0 = sv->a_games.alloc(n, 1);
                s.c0 = s.g0 >= 0 ? sv->a_cells.alloc(s.cells, 16) : -1;
                s.p0 = s.c0 >= 0 ? sv->a_planes.alloc(s.planes, 16) : -1;
                s.s0 = s.p0 >= 0 ? sv->a_slots.alloc(s.slots, 4) : -1;
                if (s.s0 >= 0) break;
                if (s.p0 >= 0) sv->a_planes.release(s.p0, s.planes);
                if (s.c0 >= 0) sv->a_cells.release(s.c0, s.cells);
                if (s.g0 >= 0) sv->a_games.release(s.g0, n);
            }
            waited = true;
            if (wait_ms <= 0 || sv->cv_admit.wait_until(lk, deadline) == std::cv_status::timeout)
                return sfail(GEN_ERR_OOM, "no room for %d games (%zu bytes) within %d ms", n, s.bytes, wait_ms);
        }
        sv->in_use += s.bytes;
        sv->peak_in_use = std::max(sv->peak_in_use, sv->in_use);
        s.id = sv->next_id++;
        int64_t c = s.c0, pl = s.p0, sl = s.s0;
        for (auto& gi : s.info) {
            gi.cell_off = (int32_t)c;
            gi.plane_off = pl;
            gi.player_off = (int32_t)sl;
            c += gi.Npad;
            pl += (int64_t)gi.P * gi.Npad;
            sl += gi.P;
        }
        {
            std::vector<int32_t> per[kClasses];
            for (int g = 0; g < n; ++g)
                per[class_index(s.info[(size_t)g].Npad, s.info[(size_t)g].P)].push_back((int32_t)(s.g0 + g));
            for (int c = 0; c < kClasses; ++c)
                if (!per[c].empty()) s.by_class.emplace_back(c, std::move(per[c]));
        }
        s.busy = true;  // until its games exist
        sv->sessions[s.id] = s;
        std::lock_guard<std::mutex> sl2(sv->stat_mu);
        sv->admitted += 1;
        sv->waited += waited ? 1 : 0;
        sv->waited_budget += over_budget ? 1 : 0;
    }
    // generate the session's games (epoch 0), write their first observations and policy actions
    ClassShape c;
    Session* sp = nullptr;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sp = &sv->sessions[s.id];  // map nodes stay put while other sessions come and go
        int rc = class_shape(sv, sp->npad_max, sp->pmax, &c);
        if (rc) return rc;
    }
    const Session& ss = *sp;
    SCUDA(cudaMemcpyAsync(sv->d_info + ss.g0, ss.info.data(), sizeof(GameInfo) * (size_t)n, cudaMemcpyHostToDevice,
                          sv->admin),
          "session table upload");
    SCUDA(cudaMemsetAsync(sv->d_scal + ss.g0, 0, sizeof(GameScalars) * (size_t)n, sv->admin), "session scalars");
    KArgs a = server_args(sv, gk::OP_CREATE, c);
    a.info = sv->d_info + ss.g0;
    a.scal = sv->d_scal + ss.g0;
    a.done = sv->out_dev.done + ss.g0;
    a.n_items = n;
    a.n_games = n;
    int rc = gk::launch_step(a, c.warps, c.max_ctas, sv->admin);
    if (rc) return sfail(GEN_ERR_CUDA, "session create launch: %s", cudaGetErrorString((cudaError_t)rc));
    SCUDA(cudaStreamSynchronize(sv->admin), "session create");
    if (h_first_actions) memcpy(h_first_actions, sv->act_host + ss.s0, sizeof(int32_t) * (size_t)ss.slots);
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->sessions[s.id].busy = false;
    }
    *session_out = s.id;
    return GEN_OK;
}

int gen_server_session_layout(gen_server* sv, int session, gen_layout_info* info, gen_outputs* dev_outputs) {
    if (!sv || !info) return sfail(GEN_ERR_BAD_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->sessions.find(session);
    if (it == sv->sessions.end()) return sfail(GEN_ERR_BAD_ARG, "no session %d", session);
    const Session& s = it->second;
    info->n_games = s.n;
    info->player_slots = (int32_t)s.slots;
    info->plane_cells = s.planes;
    info->state_cells = s.cells;
    info->max_players = s.pmax;
    int nmax = 0;
    for (auto& gi : s.info) nmax = std::max(nmax, (int)gi.N);
    info->max_cells = nmax;
    if (dev_outputs) {
        const gen_outputs& o = sv->out_dev;
        dev_outputs->obs_army = o.obs_army + s.p0;
        dev_outputs->obs_owner = o.obs_owner + s.p0;
        dev_outputs->obs_terrain = o.obs_terrain + s.p0;
        dev_outputs->obs_vis = o.obs_vis + s.p0;
        dev_outputs->mask = o.mask + s.p0;
        dev_outputs->reward = o.reward + s.s0;
        dev_outputs->scoreboard = o.scoreboard + 2 * s.s0;
        dev_outputs->done = o.done + s.g0;
    }
    return GEN_OK;
}

int gen_server_step(gen_server* sv, int session, const int32_t* h_actions, const gen_outputs* h_out,
                    int32_t* h_next_actions, double* latency_ms) {
    if (!sv || !h_actions) return sfail(GEN_ERR_BAD_ARG, "NULL argument");
    const double t_submit = now_ms();
    struct {
        int64_t g0, p0, s0, planes, slots;
        int n;
    } s;  // the session's ranges only: its game tables stay where they are
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->sessions.find(session);
        if (it == sv->sessions.end()) return sfail(GEN_ERR_BAD_ARG, "no session %d", session);
        if (it->second.busy) return sfail(GEN_ERR_STATE, "session %d already has a step in flight", session);
        if (!sv->fatal.empty()) return sfail(GEN_ERR_STATE, "server failed: %s", sv->fatal.c_str());
        it->second.busy = true;
        const Session& q = it->second;
        s = {q.g0, q.p0, q.s0, q.planes, q.slots, q.n};
    }
    // actions into the session's slots (mapped host memory)
    memcpy(sv->act_host + s.s0, h_actions, sizeof(int32_t) * (size_t)s.slots);
    Request r;
    r.session = session;
    r.t_submit = t_submit;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->queue.push_back(&r);
    }
    sv->cv_req.notify_one();
    {
        std::unique_lock<std::mutex> lk(r.m);
        r.cv.wait(lk, [&] { return r.done; });
    }
    if (r.rc != GEN_OK) {
        std::string why;
        {
            std::lock_guard<std::mutex> lk(sv->mu);  // the scheduler writes fatal under mu
            why = sv->fatal;
        }
        return sfail(r.rc, "step failed: %s", why.c_str());
    }
    // results out of the session's ranges
    if (sv->host_outputs) {
        const gen_outputs& o = sv->out_host;
        if (h_out) {
            const size_t pc = (size_t)s.planes, ps = (size_t)s.slots;
            if (h_out->obs_army) memcpy(h_out->obs_army, o.obs_army + s.p0, pc * 2);
            if (h_out->obs_owner) memcpy(h_out->obs_owner, o.obs_owner + s.p0, pc);
            if (h_out->obs_terrain) memcpy(h_out->obs_terrain, o.obs_terrain + s.p0, pc);
            if (h_out->obs_vis) memcpy(h_out->obs_vis, o.obs_vis + s.p0, pc);
            if (h_out->mask) memcpy(h_out->mask, o.mask + s.p0, pc);
            if (h_out->reward) memcpy(h_out->reward, o.reward + s.s0, ps * 4);
            if (h_out->scoreboard) memcpy(h_out->scoreboard, o.scoreboard + 2 * s.s0, ps * 8);
            if (h_out->done) memcpy(h_out->done, o.done + s.g0, (size_t)s.n);
        }
        if (h_next_actions) memcpy(h_next_actions, sv->act_host + s.s0, sizeof(int32_t) * (size_t)s.slots);
    } else {
        const gen_outputs& o = sv->out_dev;
        const size_t pc = (size_t)s.planes, ps = (size_t)s.slots;
        if (h_out) {
            if (h_out->obs_army) SCUDA(cudaMemcpy(h_out->obs_army, o.obs_army + s.p0, pc * 2, cudaMemcpyDefault), "out");
            if (h_out->obs_owner) SCUDA(cudaMemcpy(h_out->obs_owner, o.obs_owner + s.p0, pc, cudaMemcpyDefault), "out");
            if (h_out->obs_terrain)
                SCUDA(cudaMemcpy(h_out->obs_terrain, o.obs_terrain + s.p0, pc, cudaMemcpyDefault), "out");
            if (h_out->obs_vis) SCUDA(cudaMemcpy(h_out->obs_vis, o.obs_vis + s.p0, pc, cudaMemcpyDefault), "out");
            if (h_out->mask) SCUDA(cudaMemcpy(h_out->mask, o.mask + s.p0, pc, cudaMemcpyDefault), "out");
            if (h_out->reward) SCUDA(cudaMemcpy(h_out->reward, o.reward + s.s0, ps * 4, cudaMemcpyDefault), "out");
            if (h_out->scoreboard)
                SCUDA(cudaMemcpy(h_out->scoreboard, o.scoreboard + 2 * s.s0, ps * 8, cudaMemcpyDefault), "out");
            if (h_out->done) SCUDA(cudaMemcpy(h_out->done, o.done + s.g0, (size_t)s.n, cudaMemcpyDefault), "out");
        }
        if (h_next_actions) memcpy(h_next_actions, sv->act_host + s.s0, sizeof(int32_t) * ps);
    }
    const double lat = now_ms() - t_submit;
    if (latency_ms) *latency_ms = lat;
    {
        std::lock_guard<std::mutex> sl(sv->stat_mu);
        sv->lat.push_back(lat);
        sv->requests += 1;
    }
    return GEN_OK;
}

int gen_server_close(gen_server* sv, int session) {
    if (!sv) return sfail(GEN_ERR_BAD_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->sessions.find(session);
    if (it == sv->sessions.end()) return sfail(GEN_ERR_BAD_ARG, "no session %d", session);
    if (it->second.busy) return sfail(GEN_ERR_STATE, "session %d has a step in flight", session);
    const Session& s = it->second;
    sv->a_games.release(s.g0, s.n);
    sv->a_cells.release(s.c0, s.cells);
    sv->a_planes.release(s.p0, s.planes);
    sv->a_slots.release(s.s0, s.slots);
    sv->in_use -= s.bytes;
    sv->sessions.erase(it);
    sv->cv_admit.notify_all();
    return GEN_OK;
}

int gen_server_stats_get(gen_server* sv, gen_server_stats* st, int reset) {
    if (!sv || !st) return sfail(GEN_ERR_BAD_ARG, "NULL argument");
    std::vector<double> lat;
    {
        std::lock_guard<std::mutex> sl(sv->stat_mu);
        lat = sv->lat;
        st->requests = sv->requests;
        st->frames = sv->frames;
        st->ticks = sv->tick_count;
        st->sessions_admitted = sv->admitted;
        st->sessions_waited = sv->waited;
        st->sessions_waited_budget = sv->waited_budget;
        st->seconds = (now_ms() - sv->t0) * 1e-3;
        st->tick_games_mean = sv->tick_count ? sv->tick_games_sum / (double)sv->tick_count : 0.0;
        st->tick_gpu_ms_mean = sv->tick_count ? sv->tick_gpu_ms_sum / (double)sv->tick_count : 0.0;
        st->tick_host_ms_mean = sv->tick_count ? sv->tick_host_ms_sum / (double)sv->tick_count : 0.0;
        if (reset) {
            sv->lat.clear();
            sv->requests = sv->frames = sv->tick_count = sv->admitted = sv->waited = sv->waited_budget = 0;
            sv->tick_games_sum = 0;
            sv->tick_gpu_ms_sum = sv->tick_host_ms_sum = 0;
            sv->t0 = now_ms();
        }
    }
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        st->bytes_in_use = (double)sv->in_use;
        st->budget = (double)sv->budget;
        st->sessions_open = (uint64_t)sv->sessions.size();
        st->peak_bytes_in_use = (double)sv->peak_in_use;
        if (reset) sv->peak_in_use = sv->in_use;
    }
    st->frames_per_s = st->seconds > 0 ? (double)st->frames / st->seconds : 0.0;
    auto pct = [&](double q) {
        if (lat.empty()) return 0.0;
        const size_t k = std::min(lat.size() - 1, (size_t)(q * (double)(lat.size() - 1) + 0.5));
        std::nth_element(lat.begin(), lat.begin() + (long)k, lat.end());
        return lat[k];
    };
    st->lat_p50_ms = pct(0.50);
    st->lat_p99_ms = pct(0.99);
    double sum = 0;
    for (double x : lat) sum += x;
    st->lat_mean_ms = lat.empty() ? 0.0 : sum / (double)lat.size();
    st->service_p50_ms = st->lat_p50_ms;
    st->service_p99_ms = st->lat_p99_ms;
    st->offered_requests_per_s = 0.0;
    return GEN_OK;
}

void gen_server_destroy(gen_server* sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_req.notify_all();
    if (sv->sched.joinable()) sv->sched.join();
    cudaDeviceSynchronize();
    free_server(sv);
}

// Simulated actor clients.  Each holds one session, steps it with the
// actions the policy gave it last, and after a random number of steps closes
// it and opens a new one.  Closed loop: an exponential think time after each
// result.  Open loop: requests arrive as a Poisson process (exponential gaps
// on a schedule that runs on whatever the server does); a request whose
// arrival has passed is issued at once, and its latency counts from the
// scheduled arrival.
int gen_server_simulate(const gen_params* p, const gen_sim_config* cfg, gen_server_stats* st) {
    if (!p || !cfg || !st) return sfail(GEN_ERR_BAD_ARG, "NULL argument");
    if (cfg->clients < 1 || cfg->min_games < 1 || cfg->max_games < cfg->min_games || cfg->min_side < 1 ||
        cfg->max_side < cfg->min_side || cfg->max_side > GEN_MAX_SIDE || cfg->seconds <= 0)
        return sfail(GEN_ERR_BAD_ARG, "bad simulation config");
    gen_server* sv = nullptr;
    // room for every client to hold its largest session twice over (one closing, one opening)
    const int64_t max_games = (int64_t)cfg->clients * cfg->max_games * 2;
    const int64_t side = (int64_t)cfg->max_side;
    const int64_t mean_cells = ((int64_t)(cfg->min_side + cfg->max_side) / 2 + 1) * ((cfg->min_side + cfg->max_side) / 2 + 1);
    gen_server_config sc;
    memset(&sc, 0, sizeof(sc));
    sc.budget_bytes = cfg->budget_bytes;
    sc.max_games = max_games;
    sc.max_cells = std::min<int64_t>((int64_t)INT32_MAX - 4096, std::max<int64_t>(side * side * 64, 2 * max_games * mean_cells));
    const double mean_p = 2.0 * cfg->frac_1v1 + 4.0 * cfg->frac_2v2 + 8.0 * (1.0 - cfg->frac_1v1 - cfg->frac_2v2);
    sc.max_plane_cells = std::max<int64_t>(side * side * 8 * 64, (int64_t)((double)sc.max_cells * mean_p * 1.25));
    // with outputs on the device the budget caps the planes ever admitted at
    // budget / 6 bytes; arenas a little larger than that keep the budget the
    // binding limit without reserving memory no session could use
    if (!cfg->host_outputs)
        sc.max_plane_cells = std::min<int64_t>(sc.max_plane_cells,
                                               std::max<int64_t>(side * side * 8 * 64,
                                                                 (int64_t)((double)cfg->budget_bytes / 6.0 * 1.15)));
    sc.host_outputs = cfg->host_outputs;
    sc.policy_seed = cfg->policy_seed;
    int rc = gen_server_create(&sv, p, &sc);
    if (rc) return rc;
    std::atomic<bool> stop{false};
    std::atomic<bool> measuring{false};
    std::atomic<uint64_t> next_game_id{0};
    std::atomic<int> errors{0};
    std::mutex err_mu;
    std::string first_err;
    std::mutex lat_mu;
    std::vector<double> arrival_lat;  // open loop: scheduled arrival to result, measured window only
    const bool open_loop = cfg->open_loop != 0;
    auto client = [&](int id) {
        using SClock = std::chrono::steady_clock;
        auto next = SClock::now();
        std::vector<double> my_lat;
        std::mt19937_64 rng(cfg->seed * 1000003ULL + (uint64_t)id);
        std::exponential_distribution<double> think(1.0 / std::max(1e-6, cfg->mean_interarrival_ms));
        std::uniform_int_distribution<int> ngames(cfg->min_games, cfg->max_games);
        std::uniform_int_distribution<int> side(cfg->min_side, cfg->max_side);
        std::uniform_int_distribution<int> life(cfg->min_steps, std::max(cfg->min_steps, cfg->max_steps));
        std::uniform_real_distribution<double> u01(0.0, 1.0);
        while (!stop.load()) {
            const int n = ngames(rng);
            std::vector<int32_t> H((size_t)n), W((size_t)n), M((size_t)n), P((size_t)n, 8);
            for (int g = 0; g < n; ++g) {
                H[(size_t)g] = side(rng);
                W[(size_t)g] = side(rng);
                const double u = u01(rng);
                M[(size_t)g] = u < cfg->frac_1v1 ? 0 : (u < cfg->frac_1v1 + cfg->frac_2v2 ? 1 : 2);
            }
            const uint64_t base = next_game_id.fetch_add((uint64_t)n);
            int32_t sid = 0;
            std::vector<int32_t> acts((size_t)n * 8);
            int r = gen_server_open(sv, n, H.data(), W.data(), M.data(), P.data(), base, 60000, acts.data(), &sid);
            if (r) {
                if (errors.fetch_add(1) == 0) {
                    std::lock_guard<std::mutex> lk(err_mu);
                    first_err = s_err;
                }
                return;
            }
            gen_layout_info li;
            gen_server_session_layout(sv, sid, &li, nullptr);
            acts.resize((size_t)li.player_slots);
            std::vector<int16_t> oa((size_t)li.plane_cells);
            std::vector<uint8_t> ob((size_t)li.plane_cells * 4);
            std::vector<float> rw((size_t)li.player_slots);
            std::vector<int32_t> sb((size_t)li.player_slots * 2);
            std::vector<uint8_t> dn((size_t)n);
            gen_outputs ho;
            ho.obs_army = oa.data();
            ho.obs_owner = (int8_t*)ob.data();
            ho.obs_terrain = (int8_t*)ob.data() + li.plane_cells;
            ho.obs_vis = ob.data() + 2 * li.plane_cells;
            ho.mask = ob.data() + 3 * li.plane_cells;
            ho.reward = rw.data();
            ho.scoreboard = sb.data();
            ho.done = dn.data();
            const int steps = life(rng);
            for (int k = 0; k < steps && !stop.load(); ++k) {
                const std::chrono::duration<double, std::milli> gap(think(rng));
                if (open_loop) {
                    next += std::chrono::duration_cast<SClock::duration>(gap);
                    std::this_thread::sleep_until(next);
                } else {
                    std::this_thread::sleep_for(gap);
                }
                double lat = 0;
                r = gen_server_step(sv, sid, acts.data(), cfg->copy_outputs ? &ho : nullptr, acts.data(), &lat);
                if (open_loop && measuring.load())
                    my_lat.push_back(std::chrono::duration<double, std::milli>(SClock::now() - next).count());
                if (r) {
                    if (errors.fetch_add(1) == 0) {
                        std::lock_guard<std::mutex> lk(err_mu);
                        first_err = s_err;
                    }
                    break;
                }
            }
            gen_server_close(sv, sid);
        }
        std::lock_guard<std::mutex> lk(lat_mu);
        arrival_lat.insert(arrival_lat.end(), my_lat.begin(), my_lat.end());
    };
    std::vector<std::thread> th;
    for (int i = 0; i < cfg->clients; ++i) th.emplace_back(client, i);
    // warm up, then measure
    std::this_thread::sleep_for(std::chrono::duration<double>(std::min(2.0, 0.25 * cfg->seconds)));
    gen_server_stats tmp;
    gen_server_stats_get(sv, &tmp, 1);
    measuring.store(true);
    std::this_thread::sleep_for(std::chrono::duration<double>(cfg->seconds));
    gen_server_stats_get(sv, st, 0);
    measuring.store(false);
    stop.store(true);
    for (auto& t : th) t.join();
    gen_server_destroy(sv);
    st->offered_requests_per_s = (double)cfg->clients * 1e3 / std::max(1e-6, cfg->mean_interarrival_ms);
    if (open_loop && !arrival_lat.empty()) {
        auto pct = [&](double q) {
            const size_t k = std::min(arrival_lat.size() - 1, (size_t)(q * (double)(arrival_lat.size() - 1) + 0.5));
            std::nth_element(arrival_lat.begin(), arrival_lat.begin() + (long)k, arrival_lat.end());
            return arrival_lat[k];
        };
        st->lat_p50_ms = pct(0.50);
        st->lat_p99_ms = pct(0.99);
        double sum = 0;
        for (double x : arrival_lat) sum += x;
        st->lat_mean_ms = sum / (double)arrival_lat.size();
    }
    if (errors.load()) return sfail(GEN_ERR_STATE, "%d client errors; first: %s", errors.load(), first_err.c_str());
    return GEN_OK;
}

}  // extern "C"
