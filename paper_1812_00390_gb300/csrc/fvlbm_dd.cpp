// Partitioned solve of one mesh on one device: one solver per part of a
// fvlbm_partition plan, the halo exchange after every stage, and the FP64
// reductions summed over the parts.  See fvlbm_partition.cpp for the plan and
// fvlbm_exchange.cu for the exchange kernel.
#include <cmath>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "fvlbm_internal.h"

using namespace fvlbm;

struct fvlbm_dd {
    const fvlbm_partition* plan = nullptr;
    std::vector<fvlbm_solver*> part;
    int device = 0;
    int prec = FVLBM_FP64;
    void* stream = nullptr;   // the caller's: the halo exchange, and the order every call keeps
    // with more than one part, each part's stages run on a stream of its own,
    // so that the parts' kernels overlap; events order them with the exchange
    std::vector<cudaStream_t> part_stream;
    std::vector<cudaEvent_t> part_done;
    cudaEvent_t main_done = nullptr;
    int4* entries = nullptr;   // device: (src part, src internal cell, dst part, dst internal cell)
    int64_t n_entries = 0;
};

namespace {

int cuda_fail(cudaError_t e, const char* what) { return fail(FVLBM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e)); }

// The parts' streams wait for the work queued on the caller's stream.
int fork(fvlbm_dd* d) {
    if (d->part_stream.empty()) return FVLBM_OK;
    cudaError_t e = cudaEventRecord(d->main_done, (cudaStream_t)d->stream);
    for (size_t p = 0; e == cudaSuccess && p < d->part_stream.size(); p++)
        e = cudaStreamWaitEvent(d->part_stream[p], d->main_done, 0);
    return e == cudaSuccess ? FVLBM_OK : cuda_fail(e, "partitioned solve: stream order");
}

// The caller's stream waits for the work queued on every part's stream.
int join(fvlbm_dd* d) {
    cudaError_t e = cudaSuccess;
    for (size_t p = 0; e == cudaSuccess && p < d->part_stream.size(); p++) {
        e = cudaEventRecord(d->part_done[p], d->part_stream[p]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent((cudaStream_t)d->stream, d->part_done[p], 0);
    }
    return e == cudaSuccess ? FVLBM_OK : cuda_fail(e, "partitioned solve: stream order");
}

// Copy every ghost's state from its owner, each part's buffer given: on the
// caller's stream, after every part's queued work, and before any part's next.
int exchange(fvlbm_dd* d, void* const* bufs) {
    int rc = join(d);
    if (!rc) rc = launch_halo_copy(d->prec, d->stream, d->entries, d->n_entries, bufs, (int)d->part.size());
    return rc ? rc : fork(d);
}

// Exchange on the parts' current states.
int exchange_current(fvlbm_dd* d) {
    std::vector<void*> bufs(d->part.size());
    for (size_t p = 0; p < d->part.size(); p++) {
        SolverRef r;
        int rc = solver_ref(d->part[p], &r);
        if (rc) return rc;
        bufs[p] = r.view->fa;
    }
    return exchange(d, bufs.data());
}

int create_impl(fvlbm_dd* d, const fvlbm_partition* plan, const fvlbm_params* params, void* stream) {
    d->plan = plan;
    d->device = params->device;
    d->prec = params->precision;
    d->stream = stream;
    {
        DeviceGuard dg(d->device);
        if (plan->n_parts > 1) {
            cudaError_t e = cudaEventCreateWithFlags(&d->main_done, cudaEventDisableTiming);
            for (int32_t p = 0; e == cudaSuccess && p < plan->n_parts; p++) {
                cudaStream_t ps = nullptr;
                cudaEvent_t pe = nullptr;
                e = cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking);
                if (e == cudaSuccess) d->part_stream.push_back(ps);
                if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pe, cudaEventDisableTiming);
                if (e == cudaSuccess) d->part_done.push_back(pe);
            }
            if (e != cudaSuccess) return cuda_fail(e, "fvlbm_dd_create: part streams");
            int rc = fork(d);   // the parts start after the caller's queued work
            if (rc) return rc;
        }
    }
    for (int32_t p = 0; p < plan->n_parts; p++) {
        fvlbm_solver* s = nullptr;
        void* ps = d->part_stream.empty() ? stream : (void*)d->part_stream[p];
        int rc = fvlbm_init(plan->parts[p].mesh, params, 1, ps, nullptr, 0, &s);
        if (rc) return rc;
        d->part.push_back(s);
    }
    // exchange table in the parts' internal numbering
    std::vector<int4> host;
    for (const HaloMsg& m : plan->msgs) {
        const Mesh& S = plan->parts[m.src].mesh->m;
        const Mesh& D = plan->parts[m.dst].mesh->m;
        for (size_t e = 0; e < m.src_local.size(); e++)
            host.push_back(make_int4(m.src, (int)S.iperm[m.src_local[e]], m.dst, (int)D.iperm[m.dst_local[e]]));
    }
    d->n_entries = (int64_t)host.size();
    DeviceGuard dg(d->device);
    if (!host.empty()) {
        cudaError_t e = cudaMalloc(&d->entries, host.size() * sizeof(int4));
        if (e != cudaSuccess) {
            d->entries = nullptr;
            return fail(FVLBM_ERR_OOM, "fvlbm_dd_create: exchange table: %s", cudaGetErrorString(e));
        }
        e = cudaMemcpyAsync(d->entries, host.data(), host.size() * sizeof(int4), cudaMemcpyHostToDevice,
                            (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "fvlbm_dd_create: upload exchange table");
    }
    // Step 0 ran in every part's own cells; fill the ghosts
    int rc = exchange_current(d);
    if (rc) return rc;
    return fvlbm_dd_sync(d);
}

}  // namespace

extern "C" void fvlbm_dd_destroy(fvlbm_dd* d) {
    if (!d) return;
    for (fvlbm_solver* s : d->part) fvlbm_solver_destroy(s);
    DeviceGuard dg(d->device);
    if (d->entries) cudaFree(d->entries);
    for (cudaStream_t ps : d->part_stream) cudaStreamDestroy(ps);
    for (cudaEvent_t pe : d->part_done) cudaEventDestroy(pe);
    if (d->main_done) cudaEventDestroy(d->main_done);
    delete d;
}

extern "C" int fvlbm_dd_create(const fvlbm_partition* plan, const fvlbm_params* params, int32_t n_params, void* stream,
                               fvlbm_dd** out) {
    clear_error();
    if (!plan || !params || n_params != 1 || !out) return fail(FVLBM_ERR_ARG, "fvlbm_dd_create: bad arguments");
    *out = nullptr;
    fvlbm_dd* d = new (std::nothrow) fvlbm_dd;
    if (!d) return fail(FVLBM_ERR_OOM, "fvlbm_dd_create: out of host memory");
    int rc;
    try {
        rc = create_impl(d, plan, params, stream);
    } catch (const std::bad_alloc&) {
        rc = fail(FVLBM_ERR_OOM, "fvlbm_dd_create: out of host memory");
    }
    if (rc) {
        fvlbm_dd_destroy(d);
        return rc;
    }
    *out = d;
    return FVLBM_OK;
}

extern "C" int fvlbm_dd_step(fvlbm_dd* d, int64_t n) {
    clear_error();
    if (!d || n < 0) return fail(FVLBM_ERR_ARG, "fvlbm_dd_step: bad arguments");
    DeviceGuard dg(d->device);
    const int ns = solver_n_stages(d->part[0]);
    std::vector<void*> bufs(d->part.size());
    int frc = fork(d);   // after the work the caller queued on its stream
    if (frc) return frc;
    for (int64_t t = 0; t < n; t++)
        for (int k = 0; k < ns; k++) {
            for (size_t p = 0; p < d->part.size(); p++) {
                int rc = solver_stage(d->part[p], k, &bufs[p]);
                if (rc) return rc;
            }
            int rc = exchange(d, bufs.data());
            if (rc) return rc;
        }
    return FVLBM_OK;
}

extern "C" int fvlbm_dd_sync(fvlbm_dd* d) {
    clear_error();
    if (!d) return fail(FVLBM_ERR_ARG, "fvlbm_dd_sync: null argument");
    for (fvlbm_solver* s : d->part) {
        int rc = fvlbm_sync(s);
        if (rc) return rc;
    }
    DeviceGuard dg(d->device);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)d->stream);
    return e == cudaSuccess ? FVLBM_OK : cuda_fail(e, "fvlbm_dd_sync");
}

namespace {

// Per part: fetch its owned cells' rows (width values each) with `get` and
// scatter them to the caller's numbering of the whole mesh.
template <typename Get>
int gather_rows(fvlbm_dd* d, double* out, int width, Get get) {
    std::vector<double> buf;
    for (size_t p = 0; p < d->part.size(); p++) {
        const PartPlan& P = d->plan->parts[p];
        buf.assign((size_t)P.n_owned * width, 0.0);
        int rc = get(d->part[p], buf.data());
        if (rc) return rc;
        for (int64_t l = 0; l < P.n_owned; l++)
            for (int c = 0; c < width; c++) out[(size_t)P.cells[l] * width + c] = buf[(size_t)l * width + c];
    }
    return FVLBM_OK;
}

}  // namespace

extern "C" int fvlbm_dd_macros(fvlbm_dd* d, double* rho, double* u) {
    clear_error();
    if (!d) return fail(FVLBM_ERR_ARG, "fvlbm_dd_macros: null argument");
    if (rho) {
        int rc = gather_rows(d, rho, 1, [](fvlbm_solver* s, double* b) { return fvlbm_macros(s, b, nullptr); });
        if (rc) return rc;
    }
    if (u) return gather_rows(d, u, 2, [](fvlbm_solver* s, double* b) { return fvlbm_macros(s, nullptr, b); });
    return FVLBM_OK;
}

extern "C" int fvlbm_dd_get_f(fvlbm_dd* d, double* f) {
    clear_error();
    if (!d || !f) return fail(FVLBM_ERR_ARG, "fvlbm_dd_get_f: null argument");
    return gather_rows(d, f, FVLBM_Q, [](fvlbm_solver* s, double* b) { return fvlbm_get_f(s, b); });
}

extern "C" int fvlbm_dd_set_f(fvlbm_dd* d, const double* f) {
    clear_error();
    if (!d || !f) return fail(FVLBM_ERR_ARG, "fvlbm_dd_set_f: null argument");
    std::vector<double> buf;
    for (size_t p = 0; p < d->part.size(); p++) {
        const PartPlan& P = d->plan->parts[p];
        buf.resize((size_t)P.n_owned * FVLBM_Q);
        for (int64_t l = 0; l < P.n_owned; l++)
            for (int a = 0; a < FVLBM_Q; a++) buf[(size_t)l * FVLBM_Q + a] = f[(size_t)P.cells[l] * FVLBM_Q + a];
        int rc = fvlbm_set_f(d->part[p], buf.data());
        if (rc) return rc;
    }
    DeviceGuard dg(d->device);
    int rc = exchange_current(d);
    return rc ? rc : fvlbm_dd_sync(d);
}

extern "C" int fvlbm_dd_mass(fvlbm_dd* d, double* mass) {
    clear_error();
    if (!d || !mass) return fail(FVLBM_ERR_ARG, "fvlbm_dd_mass: null argument");
    double m = 0;
    std::vector<double> r;
    for (fvlbm_solver* s : d->part) {
        int rc = solver_sums(s, RED_MASS, r);
        if (rc) return rc;
        m += r[0];
    }
    *mass = m;
    return FVLBM_OK;
}

extern "C" int fvlbm_dd_residual(fvlbm_dd* d, double* e) {
    clear_error();
    if (!d || !e) return fail(FVLBM_ERR_ARG, "fvlbm_dd_residual: null argument");
    double num = 0, den = 0;
    std::vector<double> r;
    for (fvlbm_solver* s : d->part) {
        int rc = solver_sums(s, RED_RESIDUAL, r);
        if (rc) return rc;
        num += r[0];
        den += r[1];
    }
    *e = den == 0 ? (num == 0 ? 0.0 : INFINITY) : std::sqrt(num) / std::sqrt(den);
    return FVLBM_OK;
}

extern "C" int fvlbm_dd_stage_kernel(const fvlbm_dd* d, int32_t* kernel, int64_t* launches_per_step) {
    clear_error();
    if (!d || !kernel) return fail(FVLBM_ERR_ARG, "fvlbm_dd_stage_kernel: bad arguments");
    int rc = fvlbm_stage_kernel(d->part[0], kernel);
    if (rc) return rc;
    if (launches_per_step) {
        int64_t total = 0;
        for (fvlbm_solver* s : d->part) {
            int64_t l = 0;
            rc = fvlbm_launches_per_step(s, &l);
            if (rc) return rc;
            total += l;
        }
        *launches_per_step = total + (d->n_entries > 0 ? solver_n_stages(d->part[0]) : 0);
    }
    return FVLBM_OK;
}
