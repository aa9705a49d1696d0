// Allocation-free variant of the forward transform (sfrd_forward).
//
// sfrd_forward needs device scratch (the padded intermediate field and the
// twiddle / permutation tables), which normally lives in the workspace the
// caller allocates and binds.  This variant keeps that scratch in a fixed
// file-scope device array instead, so it can be called by code that may not
// allocate device memory at all: for instance a plugin or solver component
// embedded in a host application that owns the GPU memory budget and forbids
// allocations after start-up, or a latency-critical loop that cannot afford
// the implicit synchronisation of cudaMalloc / cudaFree.
#include <cstring>
#include <mutex>

#include "sfrd_internal.h"

namespace sfrd {

// Maximum scratch of the allocation-free entry point (tables + one padded field).
constexpr size_t kNoAllocScratchBytes = 16u << 20;

// Device-resident scratch shared by every call on a device; every GPU that loads
// the library holds it until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up by the first call on each
// device (with that device current); that first call should come before any stream capture.
int scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return SFRD_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return SFRD_OK;
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace
}  // namespace sfrd

namespace sfrd {
Plan* plan_of(sfrd_plan_t h);
}

// The plan's workspace fields are pointed at the static scratch for the duration
// of the call and restored afterwards; nothing is allocated on the host or the
// device.
extern "C" int sfrd_forward_noalloc(sfrd_plan_t plan, const void* u, void* uhat, void* stream) {
    using namespace sfrd;
    if (!plan || !u || !uhat) return SFRD_EINVAL;
    Plan& p = *plan_of(plan);
    const size_t E = p.esize;
    // scratch layout: [padded field | twiddles x, y, z | permutations x, y, z]
    size_t off_tw[3], off_perm[3];
    size_t o = up256((size_t)p.S * p.plane * E);
    for (int d = 0; d < 3; ++d) {
        off_tw[d] = o;
        o = up256(o + (size_t)p.M[d] * 2 * E);
        off_perm[d] = o;
        o = up256(o + (size_t)p.M[d] * sizeof(int));
    }
    if (o > kNoAllocScratchBytes) return SFRD_EUNSUPPORTED;   // problem larger than the fixed scratch
    void* base = nullptr;
    const int rc = scratch_address(&base);
    if (rc != SFRD_OK) return rc;

    char* const save_ws = p.ws;
    const cudaStream_t save_stream = p.stream;
    const size_t save_W2 = p.off_W2;
    size_t save_tw[3], save_perm[3];
    for (int d = 0; d < 3; ++d) {
        save_tw[d] = p.off_tw[d];
        save_perm[d] = p.off_perm[d];
        p.off_tw[d] = off_tw[d];
        p.off_perm[d] = off_perm[d];
    }
    p.ws = static_cast<char*>(base);
    p.stream = static_cast<cudaStream_t>(stream);
    p.off_W2 = 0;
    cudaStream_t s = p.stream;
    cudaError_t e = cudaSuccess;
    for (int d = 0; d < 3 && e == cudaSuccess; ++d) {
        const void* tw = p.dtype == SFRD_F32 ? (const void*)p.tw32[d].data() : (const void*)p.tw64[d].data();
        e = cudaMemcpyAsync(p.ws + p.off_tw[d], tw, (size_t)p.M[d] * 2 * E, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p.ws + p.off_perm[d], p.perm[d].data(), (size_t)p.M[d] * sizeof(int),
                                cudaMemcpyHostToDevice, s);
    }
    // the field scratch starts at zero on every call (the previous call left its values there)
    if (e == cudaSuccess) e = cudaMemsetAsync(p.ws + p.off_W2, 0, (size_t)p.S * p.plane * E, s);
    if (e == cudaSuccess) e = p.dtype == SFRD_F32 ? prepare_kernels<float>(p) : prepare_kernels<double>(p);
    if (e == cudaSuccess)
        e = p.dtype == SFRD_F32 ? launch_forward<float>(p, u, uhat, s) : launch_forward<double>(p, u, uhat, s);
    // wait for the work queued on the shared array even when a launch or copy failed part way, so that
    // no kernel of this call is still using the array when the call returns
    const cudaError_t es = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = es;

    p.ws = save_ws;
    p.stream = save_stream;
    p.off_W2 = save_W2;
    for (int d = 0; d < 3; ++d) {
        p.off_tw[d] = save_tw[d];
        p.off_perm[d] = save_perm[d];
    }
    return e == cudaSuccess ? SFRD_OK : cuda_fail(e, "sfrd_forward_noalloc");
}
