// Persistent kernels of the batched step, one per engine length and pass mode.
//
// A batched pass runs the instances whose pass axis has the same length on the
// register engine as one launch of a kernel compiled for that length (its
// register budget and tile exactly those of the single-instance pass), and the
// instances on the shared-memory engine as one launch of the generic kernel.
// Every block of a launch takes (instance, tile) work items from the launch's
// own device counter, copies the instance's pass arguments into shared memory
// and runs the single-instance device body on that tile.
#pragma once

#include "passes2.cuh"

namespace sfrd {

struct BatchItem {
    int inst, bx, by, cost;
    int bz;   // species of an element-pair tile (0 otherwise)
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

// Pass kinds of a batched launch.
enum BatchAxis { BATCH_X = 0, BATCH_COL = 1 };

template <typename A>
__device__ __forceinline__ void copy_args(A* dst, const A* src) {
    static_assert(sizeof(A) % 4 == 0, "argument block must be word sized");
    const int* s = reinterpret_cast<const int*>(src);
    int* d = reinterpret_cast<int*>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(A) / 4); i += blockDim.x) d[i] = s[i];
}

// The work loop of one persistent block: body(args, item) for every item it takes.  The x pass
// (XPASS) sets the stage fraction of the reaction time in the copied arguments.
template <bool XPASS, typename Args, typename Inst, class Body>
__device__ __forceinline__ void batch_loop(const Inst* __restrict__ insts, const BatchItem* __restrict__ items,
                                           int nitems, int* counter, double frac, Args* s_args, int* s_w,
                                           Body&& body) {
    for (;;) {
        if (threadIdx.x == 0) *s_w = atomicAdd(counter, 1);
        __syncthreads();
        const int w = *s_w;
        if (w >= nitems) break;
        const BatchItem it = items[w];
        copy_args(s_args, &insts[it.inst].a);
        __syncthreads();
        if constexpr (XPASS) {
            if (threadIdx.x == 0) s_args->stage_frac = frac;
            __syncthreads();
        }
        body(*s_args, it);
        __syncthreads();
    }
}

namespace v2 {

// KIND >= 0 (FP32 two-species batches, whose instances share one reaction): the reaction pass compiled
// for that reaction kind only, as the single-instance length-1024 pass.
template <typename T, int N, int MODE, int KIND = -1>
__global__ void __launch_bounds__(kThreads, (min_blocks<T, N, MODE>()))
    batch_x2_kernel(const BatchX<T>* __restrict__ insts, const BatchItem* __restrict__ items, int nitems,
                    double stage_frac, int* counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) XArgs<T> s_args;
    __shared__ int s_w;
    batch_loop<true>(insts, items, nitems, counter, stage_frac, &s_args, &s_w, [&](const XArgs<T>& a, const BatchItem& it) {
        x2_body<T, N, MODE, -1, KIND>(a, it.bx, smem_raw);
    });
}

// The length-N batched reaction pass for a batch's reaction: one kernel per two-species kind for FP32
// (kind < 0: the kernel of every kind, which also serves one-species batches).
template <typename T, int N>
void (*batch_x2_for(int kind))(const BatchX<T>*, const BatchItem*, int, double, int*) {
    if constexpr (sizeof(T) == 4) {
        switch (kind) {
            case SFRD_REACT_SCHNAKENBERG: return batch_x2_kernel<T, N, MODE_REACT, SFRD_REACT_SCHNAKENBERG>;
            case SFRD_REACT_GRAY_SCOTT: return batch_x2_kernel<T, N, MODE_REACT, SFRD_REACT_GRAY_SCOTT>;
            case SFRD_REACT_FHN: return batch_x2_kernel<T, N, MODE_REACT, SFRD_REACT_FHN>;
            case SFRD_REACT_GIERER_MEINHARDT: return batch_x2_kernel<T, N, MODE_REACT, SFRD_REACT_GIERER_MEINHARDT>;
            case SFRD_REACT_LINEAR: return batch_x2_kernel<T, N, MODE_REACT, SFRD_REACT_LINEAR>;
            case SFRD_REACT_NONE: return batch_x2_kernel<T, N, MODE_REACT, SFRD_REACT_NONE>;
            default: break;
        }
    }
    return batch_x2_kernel<T, N, MODE_REACT>;
}

// PAIR: the stage passes of FP32 two-species instances on element pairs (species = item.bz), as the
// single-instance slow-axis passes run them.
template <typename T, int N, int MODE, bool PAIR = false>
__global__ void __launch_bounds__(kThreads, (min_blocks<T, N, MODE>()))
    batch_col2_kernel(const BatchC<T>* __restrict__ insts, const BatchItem* __restrict__ items, int nitems,
                      int* counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) ColArgs<T> s_args;
    __shared__ int s_w;
    batch_loop<false>(insts, items, nitems, counter, 0.0, &s_args, &s_w, [&](const ColArgs<T>& a, const BatchItem& it) {
        col2_body<T, N, MODE, -1, false, PAIR>(a, it.bx, it.by, smem_raw, it.bz);
    });
}

// Grid of a persistent launch: blocks_per_sm resident blocks per SM (0: as many as fit), never more than
// the launch's items.
inline int batch_grid(const void* kernel, size_t smem, int blocks_per_sm, int sms, int nitems, cudaError_t* err) {
    int occ = 0;
    *err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kThreads, smem);
    if (occ < 1) occ = 1;
    const int bps = blocks_per_sm > 0 && blocks_per_sm < occ ? blocks_per_sm : occ;
    const long long g = (long long)bps * sms;
    return (int)(g < nitems ? g : nitems);
}

// Kernel of the length-N batched pass of kind `axis` and `mode` (`pair`: the element-pair stage passes).
template <typename T, int N>
const void* batch_kernel2(int axis, int mode, bool pair = false) {
    if (axis == BATCH_X) return reinterpret_cast<const void*>(batch_x2_kernel<T, N, MODE_REACT>);
    if constexpr (sizeof(T) == 4) {
        if (pair) {
            switch (mode) {
                case MODE_TA: return reinterpret_cast<const void*>(batch_col2_kernel<T, N, MODE_TA, true>);
                case MODE_TB: return reinterpret_cast<const void*>(batch_col2_kernel<T, N, MODE_TB, true>);
                case MODE_TC: return reinterpret_cast<const void*>(batch_col2_kernel<T, N, MODE_TC, true>);
                case MODE_TD: return reinterpret_cast<const void*>(batch_col2_kernel<T, N, MODE_TD, true>);
                default: break;
            }
        }
    }
    switch (mode) {
        case MODE_PLAIN: return reinterpret_cast<const void*>(batch_col2_kernel<T, N, MODE_PLAIN>);
        case MODE_TA: return reinterpret_cast<const void*>(batch_col2_kernel<T, N, MODE_TA>);
        case MODE_TB: return reinterpret_cast<const void*>(batch_col2_kernel<T, N, MODE_TB>);
        case MODE_TC: return reinterpret_cast<const void*>(batch_col2_kernel<T, N, MODE_TC>);
        default: return reinterpret_cast<const void*>(batch_col2_kernel<T, N, MODE_TD>);
    }
}

// Grids of the length-N batched launches (taken when the batch is bound, outside any capture):
// grid[0] the x pass, grid[1 + m] the column pass of mode m in (PLAIN, TA, TB, TC, TD).
template <typename T, int N>
cudaError_t batch_grids2(int axis, int blocks_per_sm, int sms, int nitems, int* grid, bool pair) {
    const size_t smem = TileOf<T, N>::E::smem_bytes();
    cudaError_t e = cudaSuccess;
    if (axis == BATCH_X) {   // the x passes run at their kernel's full occupancy (measured 1.5 % faster)
        grid[0] = batch_grid(batch_kernel2<T, N>(BATCH_X, MODE_REACT), smem, 0, sms, nitems, &e);
        return e;
    }
    const int modes[5] = {MODE_PLAIN, MODE_TA, MODE_TB, MODE_TC, MODE_TD};
    for (int m = 0; m < 5 && e == cudaSuccess; ++m)
        grid[1 + m] = batch_grid(batch_kernel2<T, N>(BATCH_COL, modes[m], pair), smem, blocks_per_sm, sms, nitems, &e);
    return e;
}

// One launch of the length-N kernel of pass kind `axis` and `mode` on stream s, `grid` blocks.
// xkind: the reaction kind of a two-species batch, or -1 (the x pass of every kind).
template <typename T, int N>
cudaError_t batch_launch2(int axis, int mode, const void* args, const BatchItem* items, int nitems, double frac,
                          int* counter, int grid, cudaStream_t s, bool pair, int xkind) {
    const size_t smem = TileOf<T, N>::E::smem_bytes();
    if (axis == BATCH_X) {
        batch_x2_for<T, N>(xkind)<<<grid, kThreads, smem, s>>>(static_cast<const BatchX<T>*>(args), items, nitems,
                                                               frac, counter);
        return cudaGetLastError();
    }
    auto k = reinterpret_cast<void (*)(const BatchC<T>*, const BatchItem*, int, int*)>(
        const_cast<void*>(batch_kernel2<T, N>(BATCH_COL, mode, pair)));
    k<<<grid, kThreads, smem, s>>>(static_cast<const BatchC<T>*>(args), items, nitems, counter);
    return cudaGetLastError();
}

// Shared-memory size attribute of the length-N batched kernels.
template <typename T, int N>
cudaError_t batch_prepare2() {
    const int m = (int)TileOf<T, N>::E::smem_bytes();
    cudaError_t e = cudaSuccess;
    const int xkinds[] = {-1, SFRD_REACT_NONE, SFRD_REACT_LINEAR, SFRD_REACT_FHN, SFRD_REACT_GRAY_SCOTT,
                          SFRD_REACT_SCHNAKENBERG, SFRD_REACT_GIERER_MEINHARDT};
    for (int kind : xkinds)
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(batch_x2_for<T, N>(kind), cudaFuncAttributeMaxDynamicSharedMemorySize, m);
    void (*ks[])(const BatchC<T>*, const BatchItem*, int, int*) = {
        batch_col2_kernel<T, N, MODE_PLAIN>, batch_col2_kernel<T, N, MODE_TA>, batch_col2_kernel<T, N, MODE_TB>,
        batch_col2_kernel<T, N, MODE_TC>, batch_col2_kernel<T, N, MODE_TD>};
    for (auto k : ks)
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, m);
    if constexpr (sizeof(T) == 4) {
        void (*kp[])(const BatchC<T>*, const BatchItem*, int, int*) = {
            batch_col2_kernel<T, N, MODE_TA, true>, batch_col2_kernel<T, N, MODE_TB, true>,
            batch_col2_kernel<T, N, MODE_TC, true>, batch_col2_kernel<T, N, MODE_TD, true>};
        for (auto k : kp)
            if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, m);
    }
    return e;
}

#define SFRD_BATCH_INSTANTIATE(T, N)                                                                     \
    template cudaError_t batch_grids2<T, N>(int, int, int, int, int*, bool);                              \
    template cudaError_t batch_launch2<T, N>(int, int, const void*, const BatchItem*, int, double, int*, int, \
                                             cudaStream_t, bool, int);                                    \
    template cudaError_t batch_prepare2<T, N>();

}  // namespace v2
}  // namespace sfrd
