// C ABI of the batched solver: many independent instances stepped together.
#include <cstdint>
#include <cstring>
#include <new>

#include "batched.cuh"

namespace sfrd {
// defined in the single-instance translation units
extern template cudaError_t launch_load<float>(Plan&, const void*, cudaStream_t);
extern template cudaError_t launch_load<double>(Plan&, const void*, cudaStream_t);
extern template cudaError_t launch_store<float>(Plan&, void*, cudaStream_t);
extern template cudaError_t launch_store<double>(Plan&, void*, cudaStream_t);
}  // namespace sfrd

using sfrd::BatchPlan;
using sfrd::Plan;

struct sfrd_batch_s {
    BatchPlan b;
};

#define SFRD_BCUDA(call)                                                 \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return sfrd::cuda_fail(e_, #call);       \
    } while (0)

namespace {

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

void drop_graph(BatchPlan& b) {
    if (b.exec) cudaGraphExecDestroy(b.exec);
    if (b.graph) cudaGraphDestroy(b.graph);
    b.exec = nullptr;
    b.graph = nullptr;
}

void drop_streams(BatchPlan& b) {
    for (cudaStream_t s : b.side) cudaStreamDestroy(s);
    for (cudaEvent_t e : b.join) cudaEventDestroy(e);
    b.side.clear();
    b.join.clear();
}

cudaError_t step_direct(BatchPlan& b, cudaStream_t s) {
    return b.dtype == SFRD_F32 ? sfrd::batch_step<float>(b, s) : sfrd::batch_step<double>(b, s);
}

}  // namespace

extern "C" {

int sfrd_batch_plan(sfrd_batch_t* out, int64_t count, const sfrd_grid* grids, const int32_t* bcs,
                    const double* alpha, const double* kappa, double dt, int32_t dtype,
                    const sfrd_reaction* reaction) {
    if (!out) return SFRD_EINVAL;
    *out = nullptr;
    if (count < 1 || !grids || !bcs || !alpha || !kappa || !reaction) return SFRD_EINVAL;
    if (grids[0].dim == 1) return SFRD_EUNSUPPORTED;   // batched passes are the 2D/3D ones
    sfrd_batch_s* h = new (std::nothrow) sfrd_batch_s();
    if (!h) return SFRD_EINVAL;
    BatchPlan& b = h->b;
    const int S = reaction->nspecies;
    for (int64_t i = 0; i < count; ++i) {
        Plan* p = nullptr;
        const int rc = sfrd::create_plan(&p, &grids[i], bcs[i], alpha + i * S, kappa + i * S, dt, dtype, reaction);
        if (rc != SFRD_OK) {
            delete h;
            return rc;
        }
        bool ok = grids[i].dim == grids[0].dim;
        for (int d = 0; d < p->dim; ++d) ok = ok && p->Nint[d] <= sfrd::kBatchMaxN;
        if (!ok) {
            delete p;
            delete h;
            return grids[i].dim == grids[0].dim ? SFRD_EUNSUPPORTED : SFRD_EINVAL;
        }
        p->CC = dtype == SFRD_F32 ? sfrd::BatchCC<float>::v : sfrd::BatchCC<double>::v;
        b.inst.push_back(*p);
        delete p;
    }
    b.dim = b.inst[0].dim;
    b.S = S;
    b.dtype = dtype;
    // workspace: instance workspaces, then the pass tables, then the work counters
    size_t o = 0;
    for (const Plan& p : b.inst) {
        b.inst_off.push_back(o);
        o = up256(o + p.ws_bytes);
    }
    // table sizes are known once the instances are bound; reserve a generous upper bound
    const size_t per_inst = sizeof(sfrd::BatchX<double>) + 2 * sizeof(sfrd::BatchC<double>);
    size_t items = 0;
    for (const Plan& p : b.inst) items += (size_t)(p.n[1] * p.n[2] + 1) + 3 * (size_t)(p.pitch + 1) * (p.n[1] + p.n[2] + 1);
    b.off_tables = o;    // pass tables start here (filled at bind)
    o = up256(o + count * per_inst + items * sizeof(sfrd::BatchItem) + 64 * 256);
    b.off_counters = o;
    o = up256(o + sfrd::kBatchCounters * sizeof(int));
    b.ws_bytes = o;
    *out = h;
    return SFRD_OK;
}

int sfrd_batch_workspace_bytes(sfrd_batch_t batch, size_t* bytes) {
    if (!batch || !bytes) return SFRD_EINVAL;
    *bytes = batch->b.ws_bytes;
    return SFRD_OK;
}

int sfrd_batch_bind(sfrd_batch_t batch, void* workspace, size_t bytes, void* stream) {
    if (!batch) return SFRD_EINVAL;
    BatchPlan& b = batch->b;
    if (!workspace || bytes < b.ws_bytes || (reinterpret_cast<uintptr_t>(workspace) & 255u)) return SFRD_ENOWS;
    drop_graph(b);
    b.ws = static_cast<char*>(workspace);
    b.stream = static_cast<cudaStream_t>(stream);
    b.loaded = false;
    for (size_t i = 0; i < b.inst.size(); ++i) {
        const int rc = sfrd::bind_plan(&b.inst[i], b.ws + b.inst_off[i], b.inst[i].ws_bytes, stream);
        if (rc != SFRD_OK) return rc;
    }
    const size_t base = b.off_tables;
    std::vector<char>& host = b.host_tables;
    host.clear();
    if (b.dtype == SFRD_F32) sfrd::batch_tables<float>(b, host);
    else sfrd::batch_tables<double>(b, host);
    if (base + host.size() > b.off_counters) return SFRD_EUNSUPPORTED;
    for (sfrd::BatchPass* ps : {&b.px, &b.pmid, &b.pslow}) {
        ps->off_args += base;
        for (sfrd::BatchGroup& gr : ps->groups) gr.off_items += base;
    }
    SFRD_BCUDA(cudaMemcpyAsync(b.ws + base, host.data(), host.size(), cudaMemcpyHostToDevice, b.stream));
    SFRD_BCUDA(b.dtype == SFRD_F32 ? sfrd::batch_prepare<float>() : sfrd::batch_prepare<double>());
    int dev = 0;
    SFRD_BCUDA(cudaGetDevice(&dev));
    SFRD_BCUDA(cudaDeviceGetAttribute(&b.sms, cudaDevAttrMultiProcessorCount, dev));
    if (!b.cap_stream) SFRD_BCUDA(cudaStreamCreateWithFlags(&b.cap_stream, cudaStreamNonBlocking));
    SFRD_BCUDA(b.dtype == SFRD_F32 ? sfrd::batch_set_grids<float>(b) : sfrd::batch_set_grids<double>(b));
    // side streams and events for the launch groups of a pass (forked and joined inside the step graph)
    const int ng = sfrd::batch_max_groups(b.inst, b.dim);
    while ((int)b.side.size() < ng) {
        cudaStream_t st = nullptr;
        SFRD_BCUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        b.side.push_back(st);
    }
    while ((int)b.join.size() < ng + 1) {
        cudaEvent_t ev = nullptr;
        SFRD_BCUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        b.join.push_back(ev);
    }
    SFRD_BCUDA(cudaStreamSynchronize(b.stream));
    return SFRD_OK;
}

int sfrd_batch_load(sfrd_batch_t batch, const void* const* u0, double t0) {
    if (!batch || !u0) return SFRD_EINVAL;
    BatchPlan& b = batch->b;
    if (!b.ws) return SFRD_ENOWS;
    for (size_t i = 0; i < b.inst.size(); ++i) {
        if (!u0[i]) return SFRD_EINVAL;
        Plan& p = b.inst[i];
        SFRD_BCUDA(sfrd::launch_set_clock(p, t0, b.stream, 0));
        SFRD_BCUDA(b.dtype == SFRD_F32 ? sfrd::launch_load<float>(p, u0[i], b.stream)
                                       : sfrd::launch_load<double>(p, u0[i], b.stream));
        p.loaded = true;
    }
    b.loaded = true;
    return SFRD_OK;
}

int sfrd_batch_advance(sfrd_batch_t batch, int64_t nsteps) {
    if (!batch) return SFRD_EINVAL;
    BatchPlan& b = batch->b;
    if (!b.ws) return SFRD_ENOWS;
    if (!b.loaded) return SFRD_ESTATE;
    if (nsteps < 0) return SFRD_EINVAL;
    if (nsteps == 0) return SFRD_OK;
    if (!b.exec) {
        SFRD_BCUDA(cudaStreamBeginCapture(b.cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = step_direct(b, b.cap_stream);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(b.cap_stream, &g);
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return sfrd::cuda_fail(e, "batched step capture");
        }
        if (e2 != cudaSuccess) return sfrd::cuda_fail(e2, "cudaStreamEndCapture");
        b.graph = g;
        SFRD_BCUDA(cudaGraphInstantiate(&b.exec, g, 0));
    }
    for (int64_t k = 0; k < nsteps; ++k) SFRD_BCUDA(cudaGraphLaunch(b.exec, b.stream));
    return SFRD_OK;
}

int sfrd_batch_store(sfrd_batch_t batch, void* const* u) {
    if (!batch || !u) return SFRD_EINVAL;
    BatchPlan& b = batch->b;
    if (!b.ws) return SFRD_ENOWS;
    if (!b.loaded) return SFRD_ESTATE;
    for (size_t i = 0; i < b.inst.size(); ++i) {
        if (!u[i]) return SFRD_EINVAL;
        SFRD_BCUDA(b.dtype == SFRD_F32 ? sfrd::launch_store<float>(b.inst[i], u[i], b.stream)
                                       : sfrd::launch_store<double>(b.inst[i], u[i], b.stream));
    }
    return SFRD_OK;
}

int sfrd_batch_info(sfrd_batch_t batch, int64_t* count, int64_t* dof, int64_t* launches_per_step) {
    if (!batch) return SFRD_EINVAL;
    const BatchPlan& b = batch->b;
    int64_t d = 0;
    for (const Plan& p : b.inst) d += p.dense * p.S;
    if (count) *count = (int64_t)b.inst.size();
    if (dof) *dof = d;
    if (launches_per_step) *launches_per_step = sfrd::batch_launches_per_step(b.inst, b.dim);
    return SFRD_OK;
}

int sfrd_batch_autotune(sfrd_batch_t batch, int32_t steps, int32_t* chosen) {
    if (!batch || steps < 1) return SFRD_EINVAL;
    BatchPlan& b = batch->b;
    if (!b.ws) return SFRD_ENOWS;
    bool generic = false;
    for (const Plan& p : b.inst) generic = generic || sfrd::has_generic_axis(p);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SFRD_BCUDA(cudaEventCreate(&e0));
    SFRD_BCUDA(cudaEventCreate(&e1));
    float best = -1.0f;
    int best_k = 2, best_rule = 0, rc = SFRD_OK;
    for (int rule = 0; rule < (generic ? 4 : 1) && rc == SFRD_OK; ++rule) {
        bool fresh = rule == 0;
        for (Plan& p : b.inst) fresh = sfrd::apply_schedule(&p, p.CC, rule) || fresh;
        if (!fresh) continue;
        for (int k = 1; k <= 4 && rc == SFRD_OK; ++k) {
            b.blocks_per_sm = k;
            rc = sfrd_batch_bind(batch, b.ws, b.ws_bytes, b.stream);
            if (rc != SFRD_OK) break;
            cudaError_t e = step_direct(b, b.stream);   // warm-up (state is zero after binding)
            if (e == cudaSuccess) e = cudaEventRecord(e0, b.stream);
            for (int q = 0; q < steps && e == cudaSuccess; ++q) e = step_direct(b, b.stream);
            if (e == cudaSuccess) e = cudaEventRecord(e1, b.stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                rc = sfrd::cuda_fail(e, "sfrd_batch_autotune");
                break;
            }
            if (best < 0 || ms < best) {
                best = ms;
                best_k = k;
                best_rule = rule;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SFRD_OK) return rc;
    for (Plan& p : b.inst) sfrd::apply_schedule(&p, p.CC, best_rule);
    b.blocks_per_sm = best_k;
    rc = sfrd_batch_bind(batch, b.ws, b.ws_bytes, b.stream);
    if (rc != SFRD_OK) return rc;
    if (chosen) {
        chosen[0] = best_k;
        chosen[1] = best_rule;
    }
    return SFRD_OK;
}

void sfrd_batch_destroy(sfrd_batch_t batch) {
    if (!batch) return;
    drop_graph(batch->b);
    drop_streams(batch->b);
    if (batch->b.cap_stream) cudaStreamDestroy(batch->b.cap_stream);
    delete batch;
}

}  // extern "C"
