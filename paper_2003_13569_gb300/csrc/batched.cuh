// Batched ETDRK4-P13 steps: many independent instances (each with its own grid
// size, boundary condition, orders alpha_s and coefficients) advanced by ONE
// launch per pass of the step.  Each launch is a persistent kernel: its blocks
// take (instance, tile) work items from a device counter, copy the instance's
// pass arguments into shared memory and run the same device body as the
// single-instance pass (register engine for power-of-two N <= 512, shared-memory
// engine with a fixed tile width otherwise).  Items are ordered longest first.
#pragma once

#include <algorithm>
#include <cstring>
#include <vector>

#include "passes.cuh"
#include "passes2.cuh"

namespace sfrd {

struct BatchItem {
    int inst, bx, by, cost;
};

template <typename T> struct BatchX {
    XArgs<T> a;
    int engine;   // 1 register engine, 0 shared-memory engine
    int N;
};

template <typename T> struct BatchC {
    ColArgs<T> a;
    int engine;
    int N;
};

// Tile width of the shared-memory engine inside batched passes.
template <typename T> struct BatchCC { static constexpr int v = sizeof(T) == 4 ? 8 : 4; };
constexpr int kBatchMaxN = 512;

template <typename A>
__device__ __forceinline__ void copy_args(A* dst, const A* src) {
    static_assert(sizeof(A) % 4 == 0, "argument block must be word sized");
    const int* s = reinterpret_cast<const int*>(src);
    int* d = reinterpret_cast<int*>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(A) / 4); i += blockDim.x) d[i] = s[i];
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads, 2) batch_x_kernel(const BatchX<T>* __restrict__ insts,
                                                               const BatchItem* __restrict__ items, int nitems,
                                                               double stage_frac, int* counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) XArgs<T> s_args;
    __shared__ int s_w, s_engine, s_N;
    for (;;) {
        if (threadIdx.x == 0) s_w = atomicAdd(counter, 1);
        __syncthreads();
        const int w = s_w;
        if (w >= nitems) break;
        const BatchItem it = items[w];
        copy_args(&s_args, &insts[it.inst].a);
        if (threadIdx.x == 0) {
            s_engine = insts[it.inst].engine;
            s_N = insts[it.inst].N;
        }
        __syncthreads();
        if (threadIdx.x == 0) s_args.stage_frac = stage_frac;
        __syncthreads();
        if (s_engine == 1) {
            switch (s_N) {
                case 64: v2::x2_body<T, 64, MODE>(s_args, it.bx, smem_raw); break;
                case 128: v2::x2_body<T, 128, MODE>(s_args, it.bx, smem_raw); break;
                case 256: v2::x2_body<T, 256, MODE>(s_args, it.bx, smem_raw); break;
                default: v2::x2_body<T, 512, MODE>(s_args, it.bx, smem_raw); break;
            }
        } else {
            x_body<T, BatchCC<T>::v, MODE>(s_args, it.bx, smem_raw);
        }
        __syncthreads();
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads, 2) batch_col_kernel(const BatchC<T>* __restrict__ insts,
                                                                 const BatchItem* __restrict__ items, int nitems,
                                                                 int* counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) ColArgs<T> s_args;
    __shared__ int s_w, s_engine, s_N;
    for (;;) {
        if (threadIdx.x == 0) s_w = atomicAdd(counter, 1);
        __syncthreads();
        const int w = s_w;
        if (w >= nitems) break;
        const BatchItem it = items[w];
        copy_args(&s_args, &insts[it.inst].a);
        if (threadIdx.x == 0) {
            s_engine = insts[it.inst].engine;
            s_N = insts[it.inst].N;
        }
        __syncthreads();
        if (s_engine == 1) {
            switch (s_N) {
                case 64: v2::col2_body<T, 64, MODE>(s_args, it.bx, it.by, smem_raw); break;
                case 128: v2::col2_body<T, 128, MODE>(s_args, it.bx, it.by, smem_raw); break;
                case 256: v2::col2_body<T, 256, MODE>(s_args, it.bx, it.by, smem_raw); break;
                default: v2::col2_body<T, 512, MODE>(s_args, it.bx, it.by, smem_raw); break;
            }
        } else {
            col_body<T, BatchCC<T>::v, MODE>(s_args, it.bx, it.by, smem_raw);
        }
        __syncthreads();
    }
}

// ---- host side ------------------------------------------------------------------------

template <typename T>
static size_t inst_smem(const Plan& p, int d) {
    if (!p.v2[d]) return tile_smem<T>(p, d);
    switch (p.Nint[d]) {
        case 64: return v2::TileOf<T, 64>::E::smem_bytes();
        case 128: return v2::TileOf<T, 128>::E::smem_bytes();
        case 256: return v2::TileOf<T, 256>::E::smem_bytes();
        default: return v2::TileOf<T, 512>::E::smem_bytes();
    }
}

// Device tables of one batched pass kind.
struct BatchPass {
    size_t off_args = 0, off_items = 0;
    int nitems = 0;
    size_t smem = 0;
    int axis = 0;   // 0 x, 1 middle, 2 slow
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
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool loaded = false;
    int max_blocks = 0;
    int blocks_per_sm = 0;   // resident blocks per SM of the persistent launches (0: default 2)
};

template <typename T>
static void batch_tables(BatchPlan& b, std::vector<char>& host) {
    // arguments and items of the three pass kinds, packed back to back
    const int n = (int)b.inst.size();
    std::vector<BatchX<T>> xa(n);
    std::vector<BatchC<T>> ma(n), sa(n);
    std::vector<BatchItem> xi, mi, si;
    size_t sx = 0, sm = 0, ss = 0;
    const int slow = b.dim == 3 ? 2 : 1;
    for (int i = 0; i < n; ++i) {
        const Plan& p = b.inst[i];
        const Arr<T> W = internal_arr<T>(p, p.off_W);
        dim3 g;
        xa[i].a = x_args<T>(p, W, W, p.pitch, 0.0, g);
        xa[i].engine = p.v2[0] ? 1 : 0;
        xa[i].N = (int)p.Nint[0];
        for (unsigned bx = 0; bx < g.x; ++bx) xi.push_back(BatchItem{i, (int)bx, 0, (int)p.Nint[0]});
        sx = std::max(sx, inst_smem<T>(p, 0));
        sa[i].a = col_args<T>(p, slow, W, W, 1.0, g);
        sa[i].engine = p.v2[slow] ? 1 : 0;
        sa[i].N = (int)p.Nint[slow];
        for (unsigned by = 0; by < g.y; ++by)
            for (unsigned bx = 0; bx < g.x; ++bx) si.push_back(BatchItem{i, (int)bx, (int)by, (int)p.Nint[slow]});
        ss = std::max(ss, inst_smem<T>(p, slow));
        if (b.dim == 3) {
            ma[i].a = col_args<T>(p, 1, W, W, 1.0, g);
            ma[i].engine = p.v2[1] ? 1 : 0;
            ma[i].N = (int)p.Nint[1];
            for (unsigned by = 0; by < g.y; ++by)
                for (unsigned bx = 0; bx < g.x; ++bx) mi.push_back(BatchItem{i, (int)bx, (int)by, (int)p.Nint[1]});
            sm = std::max(sm, inst_smem<T>(p, 1));
        }
    }
    auto longest_first = [](const BatchItem& x, const BatchItem& y) { return x.cost > y.cost; };
    std::stable_sort(xi.begin(), xi.end(), longest_first);
    std::stable_sort(mi.begin(), mi.end(), longest_first);
    std::stable_sort(si.begin(), si.end(), longest_first);
    size_t o = 0;
    auto put = [&](const void* src, size_t bytes) {
        const size_t at = o;
        o = (o + bytes + 255) / 256 * 256;
        if (host.size() < o) host.resize(o);
        std::memcpy(host.data() + at, src, bytes);
        return at;
    };
    b.px.off_args = put(xa.data(), xa.size() * sizeof(BatchX<T>));
    b.px.off_items = put(xi.data(), xi.size() * sizeof(BatchItem));
    b.px.nitems = (int)xi.size();
    b.px.smem = sx;
    b.pslow.off_args = put(sa.data(), sa.size() * sizeof(BatchC<T>));
    b.pslow.off_items = put(si.data(), si.size() * sizeof(BatchItem));
    b.pslow.nitems = (int)si.size();
    b.pslow.smem = ss;
    if (b.dim == 3) {
        b.pmid.off_args = put(ma.data(), ma.size() * sizeof(BatchC<T>));
        b.pmid.off_items = put(mi.data(), mi.size() * sizeof(BatchItem));
        b.pmid.nitems = (int)mi.size();
        b.pmid.smem = sm;
    } else {
        b.pmid.off_args = b.pmid.off_items = 0;
        b.pmid.nitems = 0;
    }
}

template <typename T>
cudaError_t batch_prepare() {
    const int m = 192 * 1024;   // leaves room for the static shared arguments of the batched kernels
    void (*xs[])(const BatchX<T>*, const BatchItem*, int, double, int*) = {batch_x_kernel<T, MODE_REACT>};
    for (auto k : xs) SFRD_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, m));
    void (*cs[])(const BatchC<T>*, const BatchItem*, int, int*) = {
        batch_col_kernel<T, MODE_PLAIN>, batch_col_kernel<T, MODE_TA>, batch_col_kernel<T, MODE_TB>,
        batch_col_kernel<T, MODE_TC>, batch_col_kernel<T, MODE_TD>};
    for (auto k : cs) SFRD_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, m));
    return cudaSuccess;
}

// One batched step: per stage [middle] x [middle] slow, each one persistent launch.
template <typename T>
cudaError_t batch_step(const BatchPlan& b, cudaStream_t s) {
    static const double frac[4] = {0.0, 0.5, 0.5, 1.0};
    int* counters = reinterpret_cast<int*>(b.ws + b.off_counters);
    SFRD_TRY(cudaMemsetAsync(counters, 0, 64 * sizeof(int), s));
    const int grid = b.max_blocks;
    int q = 0;
    const BatchX<T>* xa = reinterpret_cast<const BatchX<T>*>(b.ws + b.px.off_args);
    const BatchItem* xi = reinterpret_cast<const BatchItem*>(b.ws + b.px.off_items);
    const BatchC<T>* sa = reinterpret_cast<const BatchC<T>*>(b.ws + b.pslow.off_args);
    const BatchItem* si = reinterpret_cast<const BatchItem*>(b.ws + b.pslow.off_items);
    const BatchC<T>* ma = reinterpret_cast<const BatchC<T>*>(b.ws + b.pmid.off_args);
    const BatchItem* mi = reinterpret_cast<const BatchItem*>(b.ws + b.pmid.off_items);
    for (int st = 0; st < 4; ++st) {
        if (b.dim == 3) {
            batch_col_kernel<T, MODE_PLAIN><<<grid, kThreads, b.pmid.smem, s>>>(ma, mi, b.pmid.nitems, counters + q++);
            SFRD_TRY(cudaGetLastError());
        }
        batch_x_kernel<T, MODE_REACT><<<grid, kThreads, b.px.smem, s>>>(xa, xi, b.px.nitems, frac[st], counters + q++);
        SFRD_TRY(cudaGetLastError());
        if (b.dim == 3) {
            batch_col_kernel<T, MODE_PLAIN><<<grid, kThreads, b.pmid.smem, s>>>(ma, mi, b.pmid.nitems, counters + q++);
            SFRD_TRY(cudaGetLastError());
        }
        switch (st) {
            case 0: batch_col_kernel<T, MODE_TA><<<grid, kThreads, b.pslow.smem, s>>>(sa, si, b.pslow.nitems, counters + q++); break;
            case 1: batch_col_kernel<T, MODE_TB><<<grid, kThreads, b.pslow.smem, s>>>(sa, si, b.pslow.nitems, counters + q++); break;
            case 2: batch_col_kernel<T, MODE_TC><<<grid, kThreads, b.pslow.smem, s>>>(sa, si, b.pslow.nitems, counters + q++); break;
            default: batch_col_kernel<T, MODE_TD><<<grid, kThreads, b.pslow.smem, s>>>(sa, si, b.pslow.nitems, counters + q++); break;
        }
        SFRD_TRY(cudaGetLastError());
    }
    return cudaSuccess;
}

}  // namespace sfrd
