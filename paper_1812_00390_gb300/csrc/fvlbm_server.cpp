// Continuous-batching solve server.
//
// Requests (a mesh and its parameters) are queued in arrival order.  Every
// poll round admits queued requests while the device arena has a free block
// large enough for the request's workspace and a slot is free; advances every
// active request by one residual interval (the paper checks its velocity
// residual every 1000 steps, Sec. 3.2), with the requests' launches spread
// over several streams so that their kernels overlap on the GPU; then checks
// each request's residual and retires those that reached the tolerance or the
// step cap, copying rho and u to host memory and returning the workspace to
// the arena.  Each request is an ordinary solver over its own workspace, so its
// result does not depend on what else is running.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "fvlbm_internal.h"

using namespace fvlbm;

namespace {

// First-fit allocator over one device buffer (offsets only).
struct Arena {
    size_t size = 0;
    std::map<size_t, size_t> free_;  // offset -> length
    explicit Arena(size_t n = 0) : size(n) {
        if (n) free_[0] = n;
    }
    static size_t round(size_t n) { return (n + 255) / 256 * 256; }
    bool alloc(size_t n, size_t* off) {
        n = round(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n, o = it->first + n;
                free_.erase(it);
                if (rest) free_[o] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = round(n);
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
    size_t largest() const {
        size_t m = 0;
        for (auto& kv : free_) m = std::max(m, kv.second);
        return m;
    }
};

struct Request {
    int64_t id;
    const fvlbm_mesh* mesh;
    std::vector<fvlbm_params> params;
    size_t bytes = 0, off = 0;
    int stream = 0;
    fvlbm_solver* solver = nullptr;
    int state = FVLBM_REQ_QUEUED;
    int status = FVLBM_OK;
    int64_t steps = 0;
    double residual = INFINITY;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int64_t n_cell = 0;
    std::vector<double> rho, u;
};

double now_s(const std::chrono::steady_clock::time_point& t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct fvlbm_server {
    fvlbm_server_config cfg{};
    std::chrono::steady_clock::time_point t0;
    void* base = nullptr;
    Arena arena;
    std::vector<cudaStream_t> streams;
    std::deque<int64_t> queue;
    std::vector<int64_t> active;
    std::map<int64_t, Request> req;
    int64_t next_id = 0;
    int rr = 0;
    int64_t cell_steps = 0;
};

extern "C" int fvlbm_server_create(const fvlbm_server_config* cfg, fvlbm_server** out) {
    clear_error();
    if (!cfg || !out || cfg->arena_bytes == 0 || cfg->n_streams <= 0 || cfg->n_streams > 64 || cfg->max_active <= 0 ||
        cfg->check_interval <= 0 || !(cfg->residual_tol >= 0) || cfg->max_steps <= 0)
        return fail(FVLBM_ERR_ARG, "fvlbm_server_create: bad configuration");
    *out = nullptr;
    fvlbm_server* s = new (std::nothrow) fvlbm_server;
    if (!s) return fail(FVLBM_ERR_OOM, "fvlbm_server_create: out of host memory");
    s->cfg = *cfg;
    s->t0 = std::chrono::steady_clock::now();
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(cfg->device) != cudaSuccess) {
        delete s;
        return fail(FVLBM_ERR_UNSUPPORTED, "fvlbm_server_create: no CUDA device %d", cfg->device);
    }
    cudaError_t e = cudaMalloc(&s->base, cfg->arena_bytes);
    if (e != cudaSuccess) {
        delete s;
        if (prev >= 0) cudaSetDevice(prev);
        return fail(FVLBM_ERR_OOM, "fvlbm_server_create: arena of %zu bytes: %s", cfg->arena_bytes, cudaGetErrorString(e));
    }
    s->arena = Arena(cfg->arena_bytes);
    for (int k = 0; k < cfg->n_streams; k++) {
        cudaStream_t st;
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) break;
        s->streams.push_back(st);
    }
    if (prev >= 0) cudaSetDevice(prev);
    if ((int)s->streams.size() != cfg->n_streams) {
        fvlbm_server_destroy(s);
        return fail(FVLBM_ERR_CUDA, "fvlbm_server_create: streams: %s", cudaGetErrorString(e));
    }
    *out = s;
    return FVLBM_OK;
}

extern "C" void fvlbm_server_destroy(fvlbm_server* s) {
    if (!s) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->cfg.device);
    for (auto& kv : s->req)
        if (kv.second.solver) fvlbm_solver_destroy(kv.second.solver);
    for (cudaStream_t st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    if (s->base) cudaFree(s->base);
    if (prev >= 0) cudaSetDevice(prev);
    delete s;
}

extern "C" int fvlbm_server_submit(fvlbm_server* s, const fvlbm_mesh* mesh, const fvlbm_params* params,
                                   int32_t n_params, int64_t* id) {
    clear_error();
    if (!s || !mesh || !params || n_params <= 0 || !id) return fail(FVLBM_ERR_ARG, "fvlbm_server_submit: bad arguments");
    size_t bytes = 0;
    int rc = fvlbm_workspace_bytes(mesh, params, n_params, &bytes);
    if (rc) return rc;
    if (Arena::round(bytes) > s->cfg.arena_bytes)
        return fail(FVLBM_ERR_OOM, "request needs %zu bytes, the arena holds %zu", bytes, s->cfg.arena_bytes);
    for (int32_t k = 0; k < n_params; k++)
        if (params[k].device != s->cfg.device) return fail(FVLBM_ERR_ARG, "request device differs from the server's");
    Request r;
    r.id = s->next_id++;
    r.mesh = mesh;
    r.params.assign(params, params + n_params);
    r.bytes = bytes;
    r.t_submit = now_s(s->t0);
    fvlbm_mesh_info_t info;
    fvlbm_mesh_info(mesh, &info);
    r.n_cell = info.n_cell;
    s->req.emplace(r.id, std::move(r));
    s->queue.push_back(s->next_id - 1);
    *id = s->next_id - 1;
    return FVLBM_OK;
}

static void retire(fvlbm_server* s, Request& r, int status) {
    r.status = status;
    r.state = status == FVLBM_OK ? FVLBM_REQ_DONE : FVLBM_REQ_FAILED;
    if (status == FVLBM_OK) {
        r.rho.resize(r.n_cell);
        r.u.resize(2 * r.n_cell);
        int rc = fvlbm_macros(r.solver, r.rho.data(), r.u.data());
        if (rc) {
            r.status = rc;
            r.state = FVLBM_REQ_FAILED;
        }
    }
    fvlbm_solver_destroy(r.solver);
    r.solver = nullptr;
    s->arena.release(r.off, r.bytes);
    r.t_done = now_s(s->t0);
}

extern "C" int fvlbm_server_poll(fvlbm_server* s, int32_t* n_completed) {
    clear_error();
    if (!s) return fail(FVLBM_ERR_ARG, "fvlbm_server_poll: null server");
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->cfg.device);
    int32_t done = 0;
    // one residual interval for every active request, launched first so that
    // the GPU works while the host prepares new requests; the launches of
    // different requests go to different streams and overlap on the device
    std::vector<int64_t> stepping = s->active;
    for (int64_t id : stepping) {
        Request& r = s->req[id];
        const int64_t n = std::min<int64_t>(s->cfg.check_interval, s->cfg.max_steps - r.steps);
        int rc = fvlbm_step(r.solver, n);
        if (rc) r.status = rc;
        r.steps += n;
        s->cell_steps += n * r.n_cell;
    }
    // admission: first fit over the queue in arrival order, while a slot and
    // an arena block are free
    for (auto it = s->queue.begin(); it != s->queue.end() && (int)s->active.size() < s->cfg.max_active;) {
        Request& r = s->req[*it];
        size_t off;
        if (!s->arena.alloc(r.bytes, &off)) {
            ++it;
            continue;
        }
        r.off = off;
        r.stream = s->rr++ % (int)s->streams.size();
        int rc = fvlbm_init(r.mesh, r.params.data(), (int32_t)r.params.size(), s->streams[r.stream],
                            (unsigned char*)s->base + off, Arena::round(r.bytes), &r.solver);
        r.t_admit = now_s(s->t0);
        it = s->queue.erase(it);
        if (rc) {
            r.solver = nullptr;
            s->arena.release(off, r.bytes);
            r.state = FVLBM_REQ_FAILED;
            r.status = rc;
            r.t_done = r.t_admit;
            done++;
            continue;
        }
        r.state = FVLBM_REQ_ACTIVE;
        s->active.push_back(r.id);
    }
    // requests admitted this round stay active; the ones advanced are checked
    std::vector<int64_t> still;
    for (int64_t id : s->active)
        if (std::find(stepping.begin(), stepping.end(), id) == stepping.end()) still.push_back(id);
    for (int64_t id : stepping) {
        Request& r = s->req[id];
        double e = INFINITY;
        int rc = r.status ? r.status : fvlbm_residual(r.solver, &e);
        r.residual = e;
        if (rc) {
            retire(s, r, rc);
            done++;
        } else if (e <= s->cfg.residual_tol || r.steps >= s->cfg.max_steps) {
            retire(s, r, FVLBM_OK);
            done++;
        } else {
            still.push_back(id);
        }
    }
    s->active.swap(still);
    if (prev >= 0) cudaSetDevice(prev);
    if (n_completed) *n_completed = done;
    return FVLBM_OK;
}

extern "C" int fvlbm_server_request(fvlbm_server* s, int64_t id, fvlbm_request_info* info, double* rho, double* u) {
    clear_error();
    if (!s || !info) return fail(FVLBM_ERR_ARG, "fvlbm_server_request: null argument");
    auto it = s->req.find(id);
    if (it == s->req.end()) return fail(FVLBM_ERR_ARG, "unknown request %lld", (long long)id);
    const Request& r = it->second;
    info->state = r.state;
    info->status = r.status;
    info->steps = r.steps;
    info->n_cell = r.n_cell;
    info->residual = r.residual;
    info->t_submit = r.t_submit;
    info->t_admit = r.t_admit;
    info->t_done = r.t_done;
    info->workspace_bytes = r.bytes;
    if (r.state == FVLBM_REQ_DONE) {
        if (rho) std::memcpy(rho, r.rho.data(), sizeof(double) * r.n_cell);
        if (u) std::memcpy(u, r.u.data(), sizeof(double) * 2 * r.n_cell);
    }
    return FVLBM_OK;
}

extern "C" int fvlbm_server_stats(const fvlbm_server* s, fvlbm_server_stats_t* st) {
    clear_error();
    if (!s || !st) return fail(FVLBM_ERR_ARG, "fvlbm_server_stats: null argument");
    st->queued = (int32_t)s->queue.size();
    st->active = (int32_t)s->active.size();
    st->arena_free_largest = s->arena.largest();
    size_t fr = 0;
    for (auto& kv : s->arena.free_) fr += kv.second;
    st->arena_free = fr;
    st->cell_steps = s->cell_steps;
    st->t_now = now_s(s->t0);
    return FVLBM_OK;
}
