// Batched ETDRK4-P13 steps: many independent instances (each with its own grid
// size, boundary condition, orders alpha_s and coefficients) advanced together.
// Each pass of the step is split into launch groups: the instances whose pass
// axis has the same register-engine length form one group, run by the kernel
// compiled for that length (batch_kernels.cuh), and the instances on the
// shared-memory engine form one more, run by the generic kernel below with a
// fixed tile width.  The groups of a pass are independent, so they are issued on
// forked streams and become parallel branches of the step's CUDA graph: one
// group's tail overlaps the others.  Every launch is persistent (grid = resident
// blocks per SM x SMs, or fewer when it has fewer items) and takes its
// (instance, tile) items from its own device counter.
#pragma once

#include <algorithm>
#include <cstring>
#include <vector>

#include "batch_kernels.cuh"
#include "passes.cuh"

namespace sfrd {

// Tile width of the shared-memory engine inside batched passes.
template <typename T> struct BatchCC { static constexpr int v = sizeof(T) == 4 ? 8 : 4; };
constexpr int kBatchMaxN = 512;

namespace v2 {
#define SFRD_BATCH_EXTERN(T, N)                                                                                \
    extern template cudaError_t batch_grids2<T, N>(int, int, int, int, int*, bool);                             \
    extern template cudaError_t batch_launch2<T, N>(int, int, const void*, const BatchItem*, int, double, int*, \
                                                    int, cudaStream_t, bool, int);                              \
    extern template cudaError_t batch_prepare2<T, N>();
#define SFRD_BATCH_EXTERN_ALL(T)                                                                     \
    SFRD_BATCH_EXTERN(T, 64) SFRD_BATCH_EXTERN(T, 96) SFRD_BATCH_EXTERN(T, 128) SFRD_BATCH_EXTERN(T, 200) \
    SFRD_BATCH_EXTERN(T, 256) SFRD_BATCH_EXTERN(T, 384) SFRD_BATCH_EXTERN(T, 512)
SFRD_BATCH_EXTERN_ALL(float)
SFRD_BATCH_EXTERN_ALL(double)
}  // namespace v2

// ---- the shared-memory-engine group ---------------------------------------------------

template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads, 2) batch_xg_kernel(const BatchX<T>* __restrict__ insts,
                                                                const BatchItem* __restrict__ items, int nitems,
                                                                double stage_frac, int* counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) XArgs<T> s_args;
    __shared__ int s_w;
    batch_loop<true>(insts, items, nitems, counter, stage_frac, &s_args, &s_w,
                     [&](const XArgs<T>& a, const BatchItem& it) { x_body<T, BatchCC<T>::v, MODE>(a, it.bx, smem_raw); });
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads, 2) batch_colg_kernel(const BatchC<T>* __restrict__ insts,
                                                                  const BatchItem* __restrict__ items, int nitems,
                                                                  int* counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) ColArgs<T> s_args;
    __shared__ int s_w;
    batch_loop<false>(insts, items, nitems, counter, 0.0, &s_args, &s_w, [&](const ColArgs<T>& a, const BatchItem& it) {
        col_body<T, BatchCC<T>::v, MODE>(a, it.bx, it.by, smem_raw);
    });
}

// ---- host side ------------------------------------------------------------------------

template <typename T>
static size_t inst_smem(const Plan& p, int d) {
    if (!p.v2[d]) return tile_smem<T>(p, d);
    switch (p.Nint[d]) {
        case 64: return v2::TileOf<T, 64>::E::smem_bytes();
        case 128: return v2::TileOf<T, 128>::E::smem_bytes();
        case 256: return v2::TileOf<T, 256>::E::smem_bytes();
        case 96: return v2::TileOf<T, 96>::E::smem_bytes();
        case 200: return v2::TileOf<T, 200>::E::smem_bytes();
        case 384: return v2::TileOf<T, 384>::E::smem_bytes();
        default: return v2::TileOf<T, 512>::E::smem_bytes();
    }
}

// One launch group of a pass: its items (all of instances with the same engine and axis length).
struct BatchGroup {
    int engine = 0, N = 0;
    size_t off_items = 0;
    int nitems = 0;
    size_t smem = 0;   // shared-memory engine: the largest tile of its instances
    int grid[6] = {0, 0, 0, 0, 0, 0};   // x pass, then column modes PLAIN, TA, TB, TC, TD (set at bind)
    bool pair = false;   // register-engine stage passes on element pairs (FP32 two-species instances)
};

// Device tables of one batched pass kind.
struct BatchPass {
    size_t off_args = 0;
    std::vector<BatchGroup> groups;
};

struct BatchPlan {
    std::vector<Plan> inst;
    std::vector<size_t> inst_off;
    int dim = 0, S = 0, dtype = 0;
    BatchPass px, pmid, pslow;
    size_t off_tables = 0, off_counters = 0, ws_bytes = 0;
    std::vector<char> host_tables;   // staging kept alive for the async uploads
    char* ws = nullptr;
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    std::vector<cudaStream_t> side;  // forked streams of the groups of one pass
    std::vector<cudaEvent_t> join;   // their completion events, and (last) the fork event
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool loaded = false;
    int sms = 0;
    int blocks_per_sm = 0;   // resident blocks per SM of the persistent launches (0: as many as fit)
};

// (engine, length) of the groups of one pass axis, in a fixed order (register lengths ascending,
// then the shared-memory engine).
static std::vector<std::pair<int, int>> group_keys(const std::vector<Plan>& inst, int d) {
    std::vector<std::pair<int, int>> keys;
    for (const Plan& p : inst) {
        const std::pair<int, int> k(p.v2[d] ? 1 : 0, p.v2[d] ? (int)p.Nint[d] : 0);
        if (std::find(keys.begin(), keys.end(), k) == keys.end()) keys.push_back(k);
    }
    std::sort(keys.begin(), keys.end(), [](const std::pair<int, int>& a, const std::pair<int, int>& b) {
        return a.first != b.first ? a.first > b.first : a.second < b.second;
    });
    return keys;
}

// Launches of one batched step: the groups of every pass, over the four stages.
inline int batch_launches_per_step(const std::vector<Plan>& inst, int dim) {
    const int slow = dim == 3 ? 2 : 1;
    int n = (int)group_keys(inst, 0).size() + (int)group_keys(inst, slow).size();
    if (dim == 3) n += 2 * (int)group_keys(inst, 1).size();
    return 4 * n;
}

// Most groups of any pass (side streams needed).
inline int batch_max_groups(const std::vector<Plan>& inst, int dim) {
    size_t m = std::max(group_keys(inst, 0).size(), group_keys(inst, dim == 3 ? 2 : 1).size());
    if (dim == 3) m = std::max(m, group_keys(inst, 1).size());
    return (int)m;
}

template <typename T>
static void batch_tables(BatchPlan& b, std::vector<char>& host) {
    // per-instance arguments of the three pass kinds, then the items of every group, packed back to back
    const int n = (int)b.inst.size();
    std::vector<BatchX<T>> xa(n);
    std::vector<BatchC<T>> ma(n), sa(n);
    std::vector<std::vector<BatchItem>> xi(n), mi(n), si(n);   // items per instance
    const int slow = b.dim == 3 ? 2 : 1;
    for (int i = 0; i < n; ++i) {
        const Plan& p = b.inst[i];
        const Arr<T> W = internal_arr<T>(p, p.off_W);
        dim3 g;
        xa[i].a = x_args<T>(p, W, W, p.pitch, 0.0, g);
        xa[i].engine = p.v2[0] ? 1 : 0;
        xa[i].N = (int)p.Nint[0];
        for (unsigned bx = 0; bx < g.x; ++bx) xi[i].push_back(BatchItem{i, (int)bx, 0, (int)p.Nint[0], 0});
        // the batched step runs only the stage modes on the slow axis: element pairs where the
        // single-instance step uses them (species on grid z)
        sa[i].a = col_args<T>(p, slow, W, W, 1.0, g, true);
        sa[i].engine = p.v2[slow] ? 1 : 0;
        sa[i].N = (int)p.Nint[slow];
        for (unsigned bz = 0; bz < g.z; ++bz)
            for (unsigned by = 0; by < g.y; ++by)
                for (unsigned bx = 0; bx < g.x; ++bx)
                    si[i].push_back(BatchItem{i, (int)bx, (int)by, (int)p.Nint[slow], (int)bz});
        if (b.dim == 3) {
            ma[i].a = col_args<T>(p, 1, W, W, 1.0, g);
            ma[i].engine = p.v2[1] ? 1 : 0;
            ma[i].N = (int)p.Nint[1];
            for (unsigned by = 0; by < g.y; ++by)
                for (unsigned bx = 0; bx < g.x; ++bx) mi[i].push_back(BatchItem{i, (int)bx, (int)by, (int)p.Nint[1], 0});
        }
    }
    size_t o = 0;
    auto put = [&](const void* src, size_t bytes) {
        const size_t at = o;
        o = (o + bytes + 255) / 256 * 256;
        if (host.size() < o) host.resize(o);
        std::memcpy(host.data() + at, src, bytes);
        return at;
    };
    auto groups = [&](BatchPass& ps, int d, const std::vector<std::vector<BatchItem>>& items,
                      const std::vector<BatchC<T>>* cargs) {
        ps.groups.clear();
        for (const auto& key : group_keys(b.inst, d)) {
            BatchGroup gr;
            gr.engine = key.first;
            gr.N = key.second;
            std::vector<BatchItem> its;
            int npair = 0, nmember = 0;
            for (int i = 0; i < n; ++i) {
                const Plan& p = b.inst[i];
                if ((p.v2[d] ? 1 : 0) != key.first || (key.first && (int)p.Nint[d] != key.second)) continue;
                its.insert(its.end(), items[i].begin(), items[i].end());
                gr.smem = std::max(gr.smem, inst_smem<T>(p, d));
                ++nmember;
                if (cargs && (*cargs)[i].a.in_sp > 0) ++npair;
            }
            // one kernel per group: the pair layout depends only on the batch's dtype and species count
            // and on the register engine (col_args), so a group's instances all have it or none does
            gr.pair = key.first == 1 && npair > 0 && npair == nmember;
            // longest lines first (the shared-memory group mixes lengths)
            std::stable_sort(its.begin(), its.end(),
                             [](const BatchItem& x, const BatchItem& y) { return x.cost > y.cost; });
            gr.nitems = (int)its.size();
            gr.off_items = put(its.data(), its.size() * sizeof(BatchItem));
            ps.groups.push_back(gr);
        }
    };
    b.px.off_args = put(xa.data(), xa.size() * sizeof(BatchX<T>));
    groups(b.px, 0, xi, nullptr);
    b.pslow.off_args = put(sa.data(), sa.size() * sizeof(BatchC<T>));
    groups(b.pslow, slow, si, &sa);
    if (b.dim == 3) {
        b.pmid.off_args = put(ma.data(), ma.size() * sizeof(BatchC<T>));
        groups(b.pmid, 1, mi, nullptr);
    } else {
        b.pmid.off_args = 0;
        b.pmid.groups.clear();
    }
}

template <typename T>
cudaError_t batch_prepare() {
    const int m = 192 * 1024;   // leaves room for the static shared arguments of the batched kernels
    SFRD_TRY(cudaFuncSetAttribute(batch_xg_kernel<T, MODE_REACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, m));
    void (*cs[])(const BatchC<T>*, const BatchItem*, int, int*) = {
        batch_colg_kernel<T, MODE_PLAIN>, batch_colg_kernel<T, MODE_TA>, batch_colg_kernel<T, MODE_TB>,
        batch_colg_kernel<T, MODE_TC>, batch_colg_kernel<T, MODE_TD>};
    for (auto k : cs) SFRD_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, m));
    SFRD_TRY((v2::batch_prepare2<T, 64>()));
    SFRD_TRY((v2::batch_prepare2<T, 96>()));
    SFRD_TRY((v2::batch_prepare2<T, 128>()));
    SFRD_TRY((v2::batch_prepare2<T, 200>()));
    SFRD_TRY((v2::batch_prepare2<T, 256>()));
    SFRD_TRY((v2::batch_prepare2<T, 384>()));
    return v2::batch_prepare2<T, 512>();
}

// Column-pass modes in the order of BatchGroup::grid[1..5].
inline int batch_mode_slot(int axis, int mode) { return axis == BATCH_X ? 0 : (mode == MODE_PLAIN ? 1 : mode); }

// Grids of every launch of every group (at bind: resident blocks per SM from the occupancy of each kernel).
template <typename T>
static cudaError_t batch_set_grids(BatchPlan& b) {
    void (*kx)(const BatchX<T>*, const BatchItem*, int, double, int*) = batch_xg_kernel<T, MODE_REACT>;
    void (*kc[5])(const BatchC<T>*, const BatchItem*, int, int*) = {
        batch_colg_kernel<T, MODE_PLAIN>, batch_colg_kernel<T, MODE_TA>, batch_colg_kernel<T, MODE_TB>,
        batch_colg_kernel<T, MODE_TC>, batch_colg_kernel<T, MODE_TD>};
    for (BatchPass* ps : {&b.px, &b.pmid, &b.pslow}) {
        const int axis = ps == &b.px ? BATCH_X : BATCH_COL;
        for (BatchGroup& gr : ps->groups) {
            if (gr.engine == 1) {
                switch (gr.N) {
#define SFRD_BATCH_CASE(N) \
    case N: SFRD_TRY((v2::batch_grids2<T, N>(axis, b.blocks_per_sm, b.sms, gr.nitems, gr.grid, gr.pair))); break;
                    SFRD_BATCH_CASE(64) SFRD_BATCH_CASE(96) SFRD_BATCH_CASE(128) SFRD_BATCH_CASE(200)
                    SFRD_BATCH_CASE(256) SFRD_BATCH_CASE(384) SFRD_BATCH_CASE(512)
#undef SFRD_BATCH_CASE
                    default: return cudaErrorInvalidValue;
                }
                continue;
            }
            cudaError_t e = cudaSuccess;
            if (axis == BATCH_X) {
                gr.grid[0] = v2::batch_grid(reinterpret_cast<const void*>(kx), gr.smem, 0, b.sms, gr.nitems, &e);
            } else {
                for (int m = 0; m < 5 && e == cudaSuccess; ++m)
                    gr.grid[1 + m] = v2::batch_grid(reinterpret_cast<const void*>(kc[m]), gr.smem, b.blocks_per_sm,
                                                    b.sms, gr.nitems, &e);
            }
            SFRD_TRY(e);
        }
    }
    return cudaSuccess;
}

// One launch of group gr of a pass (axis BATCH_X or BATCH_COL, mode) on stream s.
template <typename T>
static cudaError_t batch_launch_group(const BatchPlan& b, const BatchPass& ps, const BatchGroup& gr, int axis,
                                      int mode, double frac, int* counter, cudaStream_t s) {
    const void* args = b.ws + ps.off_args;
    const BatchItem* items = reinterpret_cast<const BatchItem*>(b.ws + gr.off_items);
    const int grid = gr.grid[batch_mode_slot(axis, mode)];
    if (grid < 1) return cudaErrorInvalidConfiguration;
    if (gr.engine == 1) {
        // the instances of a batch share one reaction: two-species batches take its own x-pass kernel
        const int xkind = b.S == 2 ? b.inst[0].re.kind : -1;
        switch (gr.N) {
#define SFRD_BATCH_CASE(N) \
    case N: return v2::batch_launch2<T, N>(axis, mode, args, items, gr.nitems, frac, counter, grid, s, gr.pair, xkind);
            SFRD_BATCH_CASE(64) SFRD_BATCH_CASE(96) SFRD_BATCH_CASE(128) SFRD_BATCH_CASE(200)
            SFRD_BATCH_CASE(256) SFRD_BATCH_CASE(384) SFRD_BATCH_CASE(512)
#undef SFRD_BATCH_CASE
            default: return cudaErrorInvalidValue;
        }
    }
    if (axis == BATCH_X) {
        batch_xg_kernel<T, MODE_REACT><<<grid, kThreads, gr.smem, s>>>(static_cast<const BatchX<T>*>(args), items,
                                                                       gr.nitems, frac, counter);
        return cudaGetLastError();
    }
    switch (mode) {
        case MODE_PLAIN:
            batch_colg_kernel<T, MODE_PLAIN><<<grid, kThreads, gr.smem, s>>>(static_cast<const BatchC<T>*>(args), items,
                                                                             gr.nitems, counter);
            break;
        case MODE_TA:
            batch_colg_kernel<T, MODE_TA><<<grid, kThreads, gr.smem, s>>>(static_cast<const BatchC<T>*>(args), items,
                                                                          gr.nitems, counter);
            break;
        case MODE_TB:
            batch_colg_kernel<T, MODE_TB><<<grid, kThreads, gr.smem, s>>>(static_cast<const BatchC<T>*>(args), items,
                                                                          gr.nitems, counter);
            break;
        case MODE_TC:
            batch_colg_kernel<T, MODE_TC><<<grid, kThreads, gr.smem, s>>>(static_cast<const BatchC<T>*>(args), items,
                                                                          gr.nitems, counter);
            break;
        default:
            batch_colg_kernel<T, MODE_TD><<<grid, kThreads, gr.smem, s>>>(static_cast<const BatchC<T>*>(args), items,
                                                                          gr.nitems, counter);
            break;
    }
    return cudaGetLastError();
}

// One pass: its groups forked from stream s onto the side streams and joined back (a single group
// runs on s itself).
template <typename T>
static cudaError_t batch_pass(const BatchPlan& b, const BatchPass& ps, int axis, int mode, double frac, int* counters,
                              int& q, cudaStream_t s) {
    const int ng = (int)ps.groups.size();
    if (ng == 1) return batch_launch_group<T>(b, ps, ps.groups[0], axis, mode, frac, counters + q++, s);
    if (ng > (int)b.side.size() || ng >= (int)b.join.size()) return cudaErrorInvalidValue;
    cudaEvent_t fork = b.join.back();
    SFRD_TRY(cudaEventRecord(fork, s));
    for (int g = 0; g < ng; ++g) {
        SFRD_TRY(cudaStreamWaitEvent(b.side[g], fork, 0));
        SFRD_TRY(batch_launch_group<T>(b, ps, ps.groups[g], axis, mode, frac, counters + q++, b.side[g]));
        SFRD_TRY(cudaEventRecord(b.join[g], b.side[g]));
    }
    for (int g = 0; g < ng; ++g) SFRD_TRY(cudaStreamWaitEvent(s, b.join[g], 0));
    return cudaSuccess;
}

// Work counters of one step: one per launch (at most 4 stages x 4 passes x 8 groups = 128).
constexpr int kBatchCounters = 256;

// One batched step: per stage [middle] x [middle] slow, each pass one launch per group.
template <typename T>
cudaError_t batch_step(const BatchPlan& b, cudaStream_t s) {
    static const double frac[4] = {0.0, 0.5, 0.5, 1.0};
    int* counters = reinterpret_cast<int*>(b.ws + b.off_counters);
    SFRD_TRY(cudaMemsetAsync(counters, 0, kBatchCounters * sizeof(int), s));
    int q = 0;
    for (int st = 0; st < 4; ++st) {
        if (b.dim == 3) SFRD_TRY(batch_pass<T>(b, b.pmid, BATCH_COL, MODE_PLAIN, 0.0, counters, q, s));
        SFRD_TRY(batch_pass<T>(b, b.px, BATCH_X, MODE_REACT, frac[st], counters, q, s));
        if (b.dim == 3) SFRD_TRY(batch_pass<T>(b, b.pmid, BATCH_COL, MODE_PLAIN, 0.0, counters, q, s));
        SFRD_TRY(batch_pass<T>(b, b.pslow, BATCH_COL, MODE_TA + st, 0.0, counters, q, s));
    }
    return cudaSuccess;
}

}  // namespace sfrd
