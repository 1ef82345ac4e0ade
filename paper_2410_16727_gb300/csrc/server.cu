// server.cu -- serving loop with continuous batching (host runtime) and the
// arena manager it places device memory with.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

// The ABI layer (abi.cu) keeps the thread-local error text; these two helpers
// are its public face inside the library.
namespace dseed {
int set_error(int code, const char *fmt, ...);
KRobot robot_params(const DseedRobot *robot);
KCost cost_params(const DseedCostParams &c);
KOpt opt_params(const DseedOptParams &o);
int check_cost_opt(const DseedCostParams &c, const DseedOptParams &o, float delta_t, float delta_r);
}  // namespace dseed

using dseed::set_error;

// ---------------------------------------------------------------------------- arena

struct DseedArena {
    size_t bytes = 0, used = 0, peak = 0;
    std::map<size_t, size_t> free_blocks;   // offset -> size
    std::map<size_t, size_t> taken;         // offset -> size
};

namespace {

constexpr size_t kUnit = 256;
size_t round_up(size_t v) { return (v + kUnit - 1) / kUnit * kUnit; }

bool arena_take(DseedArena *a, size_t bytes, size_t *off) {
    bytes = round_up(std::max<size_t>(bytes, 1));
    for (auto it = a->free_blocks.begin(); it != a->free_blocks.end(); ++it) {
        if (it->second >= bytes) {
            const size_t o = it->first, rest = it->second - bytes;
            a->free_blocks.erase(it);
            if (rest) a->free_blocks[o + bytes] = rest;
            a->taken[o] = bytes;
            a->used += bytes;
            a->peak = std::max(a->peak, a->used);
            *off = o;
            return true;
        }
    }
    return false;
}

bool arena_give(DseedArena *a, size_t off) {
    auto t = a->taken.find(off);
    if (t == a->taken.end()) return false;
    size_t o = off, sz = t->second;
    a->taken.erase(t);
    a->used -= sz;
    auto nx = a->free_blocks.lower_bound(o);
    if (nx != a->free_blocks.end() && nx->first == o + sz) {       // merge with the next block
        sz += nx->second;
        a->free_blocks.erase(nx);
    }
    auto pv = a->free_blocks.lower_bound(o);
    if (pv != a->free_blocks.begin()) {                              // merge with the previous block
        --pv;
        if (pv->first + pv->second == o) {
            o = pv->first;
            sz += pv->second;
            a->free_blocks.erase(pv);
        }
    }
    a->free_blocks[o] = sz;
    return true;
}

size_t arena_largest(const DseedArena *a) {
    size_t m = 0;
    for (const auto &kv : a->free_blocks) m = std::max(m, kv.second);
    return m;
}

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

extern "C" int dseed_arena_create(size_t bytes, DseedArena **out) {
    if (!out) return set_error(DSEED_EINVAL, "out is NULL");
    *out = nullptr;
    DseedArena *a = new (std::nothrow) DseedArena;
    if (!a) return set_error(DSEED_ENOMEM, "host allocation of the arena failed");
    a->bytes = bytes / kUnit * kUnit;
    if (a->bytes) a->free_blocks[0] = a->bytes;
    *out = a;
    return DSEED_OK;
}

extern "C" void dseed_arena_destroy(DseedArena *arena) { delete arena; }

extern "C" int dseed_arena_alloc(DseedArena *arena, size_t bytes, size_t *offset) {
    if (!arena || !offset) return set_error(DSEED_EINVAL, "arena or offset is NULL");
    if (!arena_take(arena, bytes, offset))
        return set_error(DSEED_ENOMEM, "no free block of %zu bytes (largest free %zu)", round_up(bytes),
                         arena_largest(arena));
    return DSEED_OK;
}

extern "C" int dseed_arena_free(DseedArena *arena, size_t offset) {
    if (!arena) return set_error(DSEED_EINVAL, "arena is NULL");
    if (!arena_give(arena, offset)) return set_error(DSEED_EINVAL, "offset %zu is not an allocated block", offset);
    return DSEED_OK;
}

extern "C" int dseed_arena_usage(const DseedArena *arena, size_t *used, size_t *peak, size_t *largest_free) {
    if (!arena) return set_error(DSEED_EINVAL, "arena is NULL");
    if (used) *used = arena->used;
    if (peak) *peak = arena->peak;
    if (largest_free) *largest_free = arena_largest(arena);
    return DSEED_OK;
}

// ---------------------------------------------------------------------------- server

namespace {

struct SceneRec {
    size_t off_cub = 0, off_esdf = 0;
    DseedGrid grid{};
    int n = 0;
    int users = 0;
};

struct Req {
    long long ticket = 0;
    DseedRequest r{};
    int state = 0;                 // 0 queued, 1 admitted, 2 done, -1 failed
    size_t off = 0;
    int iters_done = 0;
    double t_submit = 0, t_done = 0;
    unsigned long long *key_host = nullptr;   // pinned slot for the best-seed key
    int key_slot = -1;
    // every host buffer pinned: the device addresses of q_start, goal, seeds,
    // traj, cost, success, used by the batched copy kernel instead of copies
    bool mapped = false;
    void *dev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
};

struct Round {
    cudaEvent_t done = nullptr;
    std::vector<Req *> finishing;
};

constexpr int kClasses = 3;        // T <= 32, <= 64, <= 128

int t_class(int T) { return T <= 32 ? 0 : (T <= 64 ? 1 : 2); }

}  // namespace

struct DseedServer {
    dseed::KRobot rb{};
    dseed::KCost kc{};
    dseed::KOpt ko{};
    float delta_t = 0, delta_r = 0;
    int max_requests = 0, round_iters = 0;
    char *arena_dev = nullptr;
    DseedArena arena;
    size_t table_off = 0;          // reserved: kClasses x max_requests ServeEntry
    cudaStream_t stream = nullptr;
    // pinned staging of the round tables (two halves used in turn) and best keys
    dseed::ServeEntry *stage = nullptr;
    cudaEvent_t stage_free[2] = {nullptr, nullptr};
    int stage_half = 0;
    unsigned long long *keys = nullptr;
    unsigned long long *keys_dev = nullptr;   // the keys' mapped device address
    std::vector<int> free_keys;
    // request traffic through k_io_copies: pinned staging of the copy tables
    // (two halves with the round tables, uploads then downloads, 4 copies a
    // request each), their device copies at io_off in the arena, 16 bytes of
    // 0xff there (a fresh best-seed key), and the uploads of requests admitted
    // since the last round
    dseed::IoCopy *io_stage = nullptr;
    size_t io_off = 0;
    std::vector<dseed::IoCopy> up;
    std::unordered_map<int, SceneRec> scenes;
    std::deque<Req *> queue;
    std::vector<Req *> active;
    std::deque<Round> inflight;
    std::unordered_map<long long, std::unique_ptr<Req>> reqs;
    long long next_ticket = 1;
    double wait_limit_s = 60.0;    // limit of every wait on the GPU (dseed_server_set_wait_limit)
    DseedServerStats stats{};
};

namespace {

int cuda_err(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return DSEED_OK;
    return set_error(DSEED_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Wait for `ev` by polling cudaEventQuery, the host thread yielding between
// polls, for at most sv->wait_limit_s seconds.  On expiry DSEED_ETIMEOUT: the
// work stays in flight and the server's state is unchanged, so a later call can
// wait again.  The GPU never spins on the host's behalf.
int bounded_wait(const DseedServer *sv, cudaEvent_t ev, const char *what) {
    const double t0 = now_s();
    for (;;) {
        const cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return DSEED_OK;
        if (e != cudaErrorNotReady) return cuda_err(e, what);
        const double waited = now_s() - t0;
        if (waited >= sv->wait_limit_s)
            return set_error(DSEED_ETIMEOUT, "%s: not complete after %.3g s (limit %.3g s); it stays in flight", what,
                             waited, sv->wait_limit_s);
        std::this_thread::yield();
    }
}

size_t request_bytes(const DseedServer *sv, int S, int T) {
    return dseed::serve_layout(S, T, sv->ko.m).total * sizeof(float);
}

void finish(DseedServer *sv, Req *q, bool ok, double t) {
    q->state = ok ? 2 : -1;
    q->t_done = t;
    if (ok) {
        const unsigned long long k = *q->key_host;
        *q->r.best_host = k == ~0ull ? -1 : (int)(k & 0xffffffffull);
        sv->stats.completed += 1;
    } else {
        sv->stats.failed += 1;
    }
    if (q->key_host) sv->free_keys.push_back((int)(q->key_host - sv->keys));
    q->key_host = nullptr;
}

// retire rounds whose work (kernels and output copies) has completed
int retire(DseedServer *sv, bool wait_oldest, int *n_done) {
    bool first = true;
    while (!sv->inflight.empty()) {
        Round &rd = sv->inflight.front();
        if (wait_oldest && first) {
            const int r = bounded_wait(sv, rd.done, "serving round");
            if (r) return r;
        }
        first = false;
        const cudaError_t e = cudaEventQuery(rd.done);
        if (e == cudaErrorNotReady) break;
        if (e != cudaSuccess) return cuda_err(e, "serving round");
        const double t = now_s();
        for (Req *q : rd.finishing) {
            dseed_arena_free(&sv->arena, q->off);
            auto it = sv->scenes.find(q->r.scene_id);
            if (it != sv->scenes.end()) it->second.users -= 1;
            finish(sv, q, true, t);
            if (n_done) *n_done += 1;
        }
        cudaEventDestroy(rd.done);
        sv->inflight.pop_front();
    }
    return DSEED_OK;
}

// Device address of pinned host memory, nullptr for any other pointer.
void *mapped_address(const void *h) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

constexpr int kIoPerRequest = 4;

int admit(DseedServer *sv) {
    while (!sv->queue.empty() && (int)sv->active.size() < sv->max_requests && !sv->free_keys.empty()) {
        Req *q = sv->queue.front();
        auto it = sv->scenes.find(q->r.scene_id);
        const size_t need = request_bytes(sv, q->r.S, q->r.T);
        if (it == sv->scenes.end() || need > sv->arena.bytes - sv->table_off) {
            // cannot ever run: unknown scene, or larger than the whole arena
            sv->queue.pop_front();
            if (it != sv->scenes.end()) it->second.users -= 1;
            q->key_host = nullptr;
            finish(sv, q, false, now_s());
            continue;
        }
        size_t off;
        if (!arena_take(&sv->arena, need, &off)) break;          // wait for memory, keep arrival order
        sv->queue.pop_front();
        q->off = off;
        q->state = 1;
        q->iters_done = 0;
        const int slot = sv->free_keys.back();
        sv->free_keys.pop_back();
        q->key_host = sv->keys + slot;
        const dseed::ServeLayout L = dseed::serve_layout(q->r.S, q->r.T, sv->ko.m);
        float *R = reinterpret_cast<float *>(sv->arena_dev + off);
        const size_t n = 7 * (size_t)q->r.T;
        q->key_slot = slot;
        if (q->mapped) {
            const char *ff = sv->arena_dev + sv->io_off + 2 * sizeof(dseed::IoCopy) * kIoPerRequest * sv->max_requests;
            sv->up.push_back({q->dev[0], R + L.qs, 7 * sizeof(float)});
            sv->up.push_back({q->dev[1], R + L.goal, 7 * sizeof(float)});
            sv->up.push_back({q->dev[2], R + L.xt, (unsigned long long)q->r.S * n * sizeof(float)});
            sv->up.push_back({ff, R + L.key, sizeof(unsigned long long)});
            sv->active.push_back(q);
            sv->stats.admitted += 1;
            continue;
        }
        int r = cuda_err(cudaMemcpyAsync(R + L.qs, q->r.q_start_host, 7 * sizeof(float), cudaMemcpyHostToDevice,
                                         sv->stream), "request upload");
        if (!r) r = cuda_err(cudaMemcpyAsync(R + L.goal, q->r.goal_host, 7 * sizeof(float), cudaMemcpyHostToDevice,
                                             sv->stream), "request upload");
        if (!r) r = cuda_err(cudaMemcpyAsync(R + L.xt, q->r.seeds_host, (size_t)q->r.S * n * sizeof(float),
                                             cudaMemcpyHostToDevice, sv->stream), "request upload");
        if (!r) r = cuda_err(cudaMemsetAsync(R + L.key, 0xff, sizeof(unsigned long long), sv->stream), "request init");
        if (r) return r;
        sv->active.push_back(q);
        sv->stats.admitted += 1;
    }
    return DSEED_OK;
}

// Copy `n` entries of a copy table through staging half `half`, direction
// `dir` (0: uploads, 1: downloads), and launch the batched copy kernel.
int run_io(DseedServer *sv, int half, int dir, const dseed::IoCopy *entries, size_t n) {
    if (n == 0) return DSEED_OK;
    const size_t cap = (size_t)kIoPerRequest * sv->max_requests;
    if (n > cap) return set_error(DSEED_EINVAL, "%zu request copies exceed the table of %zu", n, cap);
    dseed::IoCopy *stage = sv->io_stage + ((size_t)half * 2 + dir) * cap;
    std::copy(entries, entries + n, stage);
    dseed::IoCopy *table = reinterpret_cast<dseed::IoCopy *>(sv->arena_dev + sv->io_off) + (size_t)dir * cap;
    int r = cuda_err(cudaMemcpyAsync(table, stage, n * sizeof(dseed::IoCopy), cudaMemcpyHostToDevice, sv->stream),
                     "copy table upload");
    if (!r) r = cuda_err((cudaError_t)dseed::launch_io_copies(table, (int)n, sv->stream), "request copies");
    return r;
}

int launch_round(DseedServer *sv) {
    // the staging half we fill must no longer be read by an earlier upload
    const int half = sv->stage_half;
    int r = bounded_wait(sv, sv->stage_free[half], "staging wait");
    if (r) return r;
    // inputs of the requests admitted since the last round
    r = run_io(sv, half, 0, sv->up.data(), sv->up.size());
    if (r) return r;
    sv->up.clear();
    dseed::ServeEntry *st = sv->stage + (size_t)half * kClasses * sv->max_requests;
    int counts[kClasses] = {0, 0, 0};
    long long warps[kClasses] = {0, 0, 0};
    Round rd;
    std::vector<Req *> still;
    for (Req *q : sv->active) {
        const int c = t_class(q->r.T);
        dseed::ServeEntry &E = st[(size_t)c * sv->max_requests + counts[c]];
        const SceneRec &sc = sv->scenes.at(q->r.scene_id);
        E.warp_begin = warps[c];
        E.region = reinterpret_cast<float *>(sv->arena_dev + q->off);
        E.scene.esdf_dev = reinterpret_cast<const float *>(sv->arena_dev + sc.off_esdf);
        E.scene.grid = sc.grid;
        E.scene.lipschitz = 1.0f;
        E.S = q->r.S;
        E.T = q->r.T;
        E.iters_done = q->iters_done;
        E.iters_round = std::min(sv->round_iters, sv->ko.iters - q->iters_done);
        E.final_round = q->iters_done + E.iters_round >= sv->ko.iters ? 1 : 0;
        E.pad = 0;
        q->iters_done += E.iters_round;
        counts[c] += 1;
        warps[c] += q->r.S;
        if (E.final_round) rd.finishing.push_back(q); else still.push_back(q);
    }
    dseed::ServeEntry *table_dev = reinterpret_cast<dseed::ServeEntry *>(sv->arena_dev + sv->table_off);
    r = cuda_err(cudaMemcpyAsync(table_dev, st, sizeof(dseed::ServeEntry) * kClasses * sv->max_requests,
                                 cudaMemcpyHostToDevice, sv->stream), "round table upload");
    if (r) return r;
    for (int c = 0; c < kClasses; ++c) {
        if (!counts[c]) continue;
        r = cuda_err((cudaError_t)dseed::launch_serve(sv->rb, sv->kc, sv->ko, sv->delta_t, sv->delta_r, 1 << c,
                                                      table_dev + (size_t)c * sv->max_requests, counts[c], warps[c],
                                                      sv->stream),
                     "serving kernel");
        if (r) return r;
    }
    // outputs of the requests that finish in this round
    std::vector<dseed::IoCopy> down;
    for (Req *q : rd.finishing) {
        const dseed::ServeLayout L = dseed::serve_layout(q->r.S, q->r.T, sv->ko.m);
        const float *R = reinterpret_cast<const float *>(sv->arena_dev + q->off);
        const size_t n = 7 * (size_t)q->r.T, S = q->r.S;
        if (q->mapped) {
            down.push_back({R + L.xa, q->dev[3], (unsigned long long)S * n * sizeof(float)});
            down.push_back({R + L.cost, q->dev[4], (unsigned long long)S * sizeof(float)});
            down.push_back({R + L.succ, q->dev[5], (unsigned long long)S});
            down.push_back({R + L.key, sv->keys_dev + q->key_slot, sizeof(unsigned long long)});
            continue;
        }
        r = cuda_err(cudaMemcpyAsync(q->r.traj_host, R + L.xa, S * n * sizeof(float), cudaMemcpyDeviceToHost,
                                     sv->stream), "output copy");
        if (!r) r = cuda_err(cudaMemcpyAsync(q->r.cost_host, R + L.cost, S * sizeof(float), cudaMemcpyDeviceToHost,
                                             sv->stream), "output copy");
        if (!r) r = cuda_err(cudaMemcpyAsync(q->r.success_host, R + L.succ, S, cudaMemcpyDeviceToHost, sv->stream),
                             "output copy");
        if (!r) r = cuda_err(cudaMemcpyAsync(q->key_host, R + L.key, sizeof(unsigned long long),
                                             cudaMemcpyDeviceToHost, sv->stream), "output copy");
        if (r) return r;
    }
    r = run_io(sv, half, 1, down.data(), down.size());
    // this half's staging has been read once the copies above are done
    if (!r) r = cuda_err(cudaEventRecord(sv->stage_free[half], sv->stream), "event");
    if (r) return r;
    sv->stage_half ^= 1;
    r = cuda_err(cudaEventCreateWithFlags(&rd.done, cudaEventDisableTiming), "event");
    if (!r) r = cuda_err(cudaEventRecord(rd.done, sv->stream), "event");
    if (r) return r;
    sv->active.swap(still);
    sv->inflight.push_back(std::move(rd));
    sv->stats.rounds += 1;
    return DSEED_OK;
}

}  // namespace

extern "C" int dseed_server_create(const DseedRobot *robot, const DseedServerDesc *desc, void *arena_dev,
                                   DseedServer **out) {
    if (!robot || !desc || !arena_dev || !out) return set_error(DSEED_EINVAL, "NULL argument");
    *out = nullptr;
    if (desc->max_requests < 1 || desc->round_iters < 1) return set_error(DSEED_EINVAL, "max_requests and round_iters must be >= 1");
    int r = dseed::check_cost_opt(desc->cost, desc->opt, desc->delta_t, desc->delta_r);
    if (r) return r;
    if (reinterpret_cast<uintptr_t>(arena_dev) % 256 != 0) return set_error(DSEED_EINVAL, "arena not 256-byte aligned");
    const size_t round_table_bytes = round_up(sizeof(dseed::ServeEntry) * kClasses * (size_t)desc->max_requests);
    const size_t io_bytes = round_up(sizeof(dseed::IoCopy) * 2 * kIoPerRequest * (size_t)desc->max_requests + 256);
    const size_t table_bytes = round_table_bytes + io_bytes;
    if (desc->arena_bytes < table_bytes + kUnit)
        return set_error(DSEED_ENOMEM, "arena of %zu bytes is smaller than the %zu-byte round tables", desc->arena_bytes,
                         table_bytes);
    std::unique_ptr<DseedServer> sv(new (std::nothrow) DseedServer);
    if (!sv) return set_error(DSEED_ENOMEM, "host allocation of the server failed");
    sv->rb = dseed::robot_params(robot);
    sv->kc = dseed::cost_params(desc->cost);
    sv->ko = dseed::opt_params(desc->opt);
    sv->delta_t = desc->delta_t;
    sv->delta_r = desc->delta_r;
    sv->max_requests = desc->max_requests;
    sv->round_iters = desc->round_iters;
    sv->arena_dev = static_cast<char *>(arena_dev);
    sv->arena.bytes = desc->arena_bytes / kUnit * kUnit;
    sv->arena.free_blocks[0] = sv->arena.bytes;
    size_t off;
    arena_take(&sv->arena, table_bytes, &off);
    sv->table_off = off;
    sv->io_off = off + round_table_bytes;
    r = cuda_err(cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking), "stream");
    if (!r) r = cuda_err(cudaMallocHost(reinterpret_cast<void **>(&sv->stage),
                                        sizeof(dseed::ServeEntry) * 2 * kClasses * (size_t)desc->max_requests),
                         "pinned staging");
    if (!r) r = cuda_err(cudaMallocHost(reinterpret_cast<void **>(&sv->keys),
                                        sizeof(unsigned long long) * (size_t)desc->max_requests * 2),
                         "pinned keys");
    if (!r) r = cuda_err(cudaHostGetDevicePointer(reinterpret_cast<void **>(&sv->keys_dev), sv->keys, 0),
                         "mapped keys");
    if (!r) r = cuda_err(cudaMallocHost(reinterpret_cast<void **>(&sv->io_stage),
                                        sizeof(dseed::IoCopy) * 2 * 2 * kIoPerRequest * (size_t)desc->max_requests),
                         "pinned copy tables");
    // the 0xff bytes a fresh best-seed key is copied from
    if (!r) r = cuda_err(cudaMemsetAsync(sv->arena_dev + sv->io_off +
                                             sizeof(dseed::IoCopy) * 2 * kIoPerRequest * (size_t)desc->max_requests,
                                         0xff, 16, sv->stream),
                         "key constant");
    for (int h = 0; h < 2 && !r; ++h) {
        r = cuda_err(cudaEventCreateWithFlags(&sv->stage_free[h], cudaEventDisableTiming), "event");
        if (!r) r = cuda_err(cudaEventRecord(sv->stage_free[h], sv->stream), "event");
    }
    if (r) {
        dseed_server_destroy(sv.release());
        return r;
    }
    // a key slot per admitted request and per request still draining
    for (int k = 2 * desc->max_requests - 1; k >= 0; --k) sv->free_keys.push_back(k);
    *out = sv.release();
    return DSEED_OK;
}

extern "C" void dseed_server_destroy(DseedServer *sv) {
    if (!sv) return;
    if (sv->stream) cudaStreamSynchronize(sv->stream);
    for (auto &rd : sv->inflight) cudaEventDestroy(rd.done);
    for (int h = 0; h < 2; ++h)
        if (sv->stage_free[h]) cudaEventDestroy(sv->stage_free[h]);
    if (sv->stage) cudaFreeHost(sv->stage);
    if (sv->keys) cudaFreeHost(sv->keys);
    if (sv->io_stage) cudaFreeHost(sv->io_stage);
    if (sv->stream) cudaStreamDestroy(sv->stream);
    delete sv;
}

extern "C" int dseed_server_add_scene(DseedServer *sv, int scene_id, const float *cuboids_host, int n,
                                      const DseedGrid *grid) {
    if (!sv || !grid) return set_error(DSEED_EINVAL, "NULL argument");
    if (sv->scenes.count(scene_id)) return set_error(DSEED_EINVAL, "scene %d already resident", scene_id);
    if (n < 0 || (n > 0 && !cuboids_host)) return set_error(DSEED_EINVAL, "bad cuboid count or NULL cuboids");
    if (grid->nx < 2 || grid->ny < 2 || grid->nz < 2 || !(grid->res > 0.f))
        return set_error(DSEED_EINVAL, "bad grid");
    const size_t esdf_bytes = sizeof(float) * (size_t)grid->nx * grid->ny * grid->nz;
    SceneRec sc;
    sc.grid = *grid;
    sc.n = n;
    if (!arena_take(&sv->arena, esdf_bytes, &sc.off_esdf))
        return set_error(DSEED_ENOMEM, "scene %d: ESDF of %zu bytes does not fit in the arena", scene_id, esdf_bytes);
    if (!arena_take(&sv->arena, std::max<size_t>(sizeof(float) * 6 * (size_t)n, 1), &sc.off_cub)) {
        arena_give(&sv->arena, sc.off_esdf);
        return set_error(DSEED_ENOMEM, "scene %d: cuboids do not fit in the arena", scene_id);
    }
    float *cub = reinterpret_cast<float *>(sv->arena_dev + sc.off_cub);
    int r = DSEED_OK;
    if (n > 0)
        r = cuda_err(cudaMemcpyAsync(cub, cuboids_host, sizeof(float) * 6 * (size_t)n, cudaMemcpyHostToDevice,
                                     sv->stream), "scene upload");
    if (!r) {
        DseedEsdfJob job;
        job.cuboids_dev = cub;
        job.n = n;
        job.grid = *grid;
        job.esdf_dev = reinterpret_cast<float *>(sv->arena_dev + sc.off_esdf);
        r = cuda_err((cudaError_t)dseed::launch_esdf_build(&job, 1, sv->stream), "scene ESDF");
    }
    if (r) {
        arena_give(&sv->arena, sc.off_esdf);
        arena_give(&sv->arena, sc.off_cub);
        return r;
    }
    sv->scenes[scene_id] = sc;
    return DSEED_OK;
}

extern "C" int dseed_server_remove_scene(DseedServer *sv, int scene_id) {
    if (!sv) return set_error(DSEED_EINVAL, "server is NULL");
    auto it = sv->scenes.find(scene_id);
    if (it == sv->scenes.end()) return set_error(DSEED_EINVAL, "scene %d is not resident", scene_id);
    if (it->second.users > 0) return set_error(DSEED_EINVAL, "scene %d is used by %d requests", scene_id, it->second.users);
    // stream-ordered: work already enqueued that reads the scene finishes first
    cudaEvent_t ev = nullptr;
    int r = cuda_err(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
    if (!r) r = cuda_err(cudaEventRecord(ev, sv->stream), "event");
    if (!r) r = bounded_wait(sv, ev, "remove scene");
    if (ev) cudaEventDestroy(ev);
    if (r) return r;
    arena_give(&sv->arena, it->second.off_esdf);
    arena_give(&sv->arena, it->second.off_cub);
    sv->scenes.erase(it);
    return DSEED_OK;
}

extern "C" int dseed_server_submit(DseedServer *sv, const DseedRequest *req, long long *ticket) {
    if (!sv || !req || !ticket) return set_error(DSEED_EINVAL, "NULL argument");
    if (req->S < 1 || req->T < 1 || req->T > DSEED_MAX_T) return set_error(DSEED_EINVAL, "bad S or T");
    if (!req->q_start_host || !req->goal_host || !req->seeds_host || !req->traj_host || !req->cost_host ||
        !req->success_host || !req->best_host)
        return set_error(DSEED_EINVAL, "a request buffer is NULL");
    std::unique_ptr<Req> q(new (std::nothrow) Req);
    if (!q) return set_error(DSEED_ENOMEM, "host allocation of the request failed");
    q->ticket = sv->next_ticket++;
    q->r = *req;
    q->t_submit = now_s();
    // with every host buffer pinned the request's traffic goes through the batched copy kernel
    const void *host[6] = {req->q_start_host, req->goal_host, req->seeds_host, req->traj_host, req->cost_host,
                           req->success_host};
    q->mapped = true;
    for (int i = 0; i < 6 && q->mapped; ++i) {
        q->dev[i] = mapped_address(host[i]);
        q->mapped = q->dev[i] != nullptr;
    }
    auto it = sv->scenes.find(req->scene_id);
    if (it != sv->scenes.end()) it->second.users += 1;
    sv->queue.push_back(q.get());
    *ticket = q->ticket;
    sv->reqs[q->ticket] = std::move(q);
    sv->stats.submitted += 1;
    return DSEED_OK;
}

extern "C" int dseed_server_step(DseedServer *sv, int wait, int *n_done) {
    if (!sv) return set_error(DSEED_EINVAL, "server is NULL");
    if (n_done) *n_done = 0;
    int r = retire(sv, wait != 0, n_done);
    if (r) return r;
    r = admit(sv);
    if (r) return r;
    if (!sv->active.empty() && sv->inflight.size() < 2) r = launch_round(sv);
    return r;
}

extern "C" int dseed_server_set_wait_limit(DseedServer *sv, double seconds) {
    if (!sv) return set_error(DSEED_EINVAL, "server is NULL");
    if (!(seconds >= 0.0)) return set_error(DSEED_EINVAL, "wait limit must be >= 0 seconds (got %g)", seconds);
    sv->wait_limit_s = seconds;
    return DSEED_OK;
}

extern "C" int dseed_server_poll(DseedServer *sv, long long ticket, int *state, double *t_submit, double *t_done) {
    if (!sv || !state) return set_error(DSEED_EINVAL, "NULL argument");
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return set_error(DSEED_EINVAL, "unknown ticket %lld", ticket);
    *state = it->second->state;
    if (t_submit) *t_submit = it->second->t_submit;
    if (t_done) *t_done = it->second->t_done;
    return DSEED_OK;
}

extern "C" int dseed_server_stats(const DseedServer *sv, DseedServerStats *out) {
    if (!sv || !out) return set_error(DSEED_EINVAL, "NULL argument");
    *out = sv->stats;
    out->queued = (int)sv->queue.size();
    out->active = (int)sv->active.size();
    for (const auto &rd : sv->inflight) out->active += (int)rd.finishing.size();
    out->arena_used = sv->arena.used;
    out->arena_peak = sv->arena.peak;
    return DSEED_OK;
}
