// Shared helpers of the npvs CUDA library (device status word, error reporting, scans).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <utility>
#include <cstdarg>
#include <cstdio>

#include "npvs.h"

namespace npvs {

// ---- host-side error reporting ------------------------------------------------------------

void set_error(const char* fmt, ...);

inline npvs_status fail(npvs_status s, const char* msg) {
    set_error("%s", msg);
    return s;
}

// Counts kernel launches made by this library (for launch accounting by callers).
void count_launch();

inline npvs_status check_launch(const char* what) {
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("%s: %s", what, cudaGetErrorString(e));
        return NPVS_ERR_CUDA;
    }
    return NPVS_OK;
}

#define NPVS_REQUIRE(cond, code, msg)                 \
    do {                                              \
        if (!(cond)) return ::npvs::fail((code), (msg)); \
    } while (0)

#define NPVS_TRY(expr)                       \
    do {                                     \
        npvs_status _s = (expr);             \
        if (_s != NPVS_OK) return _s;        \
    } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Identifier of the CUDA context current on the calling thread, 0 if there is none or the driver
// cannot say (cuCtxGetCurrent / cuCtxGetId, reached through the runtime's entry-point query so that
// the library does not link libcuda). Ids are unique within a process and never reused: a cache
// keyed on one is refreshed after a device reset, which replaces the primary context.
unsigned long long current_context_id();

constexpr int kMaxDevices = 64;

// Bound, in SM clock cycles, of every mbarrier wait in the tensor-core kernels launched from now on
// (npvs_set_wait_limit; default kDefaultWaitCycles, about 2 s at the maximum SM clock).
constexpr long long kDefaultWaitCycles = 4000000000ll;
long long wait_limit_cycles();

// Raises `kernel`'s dynamic shared-memory limit to `bytes` in the current context. `seen` (one
// slot per device ordinal, kMaxDevices) remembers the context in which it was last raised, so the
// attribute is set once per context; concurrent first calls may both set it, which is harmless.
npvs_status ensure_dynamic_smem(const void* kernel, int bytes, std::atomic<unsigned long long>* seen,
                                const char* what);

// Every kernel of the library is launched with programmatic stream serialisation: the next kernel
// on the stream may be launched and scheduled while this one finishes. Each kernel therefore
// starts with pdl_begin(): griddepcontrol.wait (returns once every earlier kernel on the stream has
// completed and its writes are visible; a no-op without the attribute), then
// griddepcontrol.launch_dependents (lets the following kernel start its own launch).
// Programmatic dependent launch can be switched off for the whole process with NPVS_PDL=0.
bool pdl_enabled();

template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                            Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

constexpr int kNumSMs = 152;

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Bump allocator over a caller-provided workspace (256-byte aligned sub-buffers).
struct Arena {
    char* base;
    size_t size;
    size_t used = 0;
    Arena(void* b, size_t s) : base((char*)b), size(s) {}
    template <class T>
    T* take(size_t count) {
        size_t off = (used + 255) & ~size_t(255);
        size_t bytes = count * sizeof(T);
        if (base == nullptr || off + bytes > size) {
            used = off + bytes;
            return nullptr;
        }
        used = off + bytes;
        return reinterpret_cast<T*>(base + off);
    }
    static size_t round(size_t b) { return (b + 255) & ~size_t(255); }
};

// ---- device helpers -------------------------------------------------------------------------

__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ void raise_status(int32_t* status, npvs_status s) {
    if (status) atomicOr(status, 1 << (int)s);
}

// Linear index of a coarse site.
__device__ __forceinline__ long long site_lin(int b, int z, int y, int x, const npvs_dims& d) {
    return (((long long)b * d.Z + z) * d.Y + y) * d.X + x;
}

// Block-wide exclusive scan of one int per thread (blockDim.x multiple of 32, <= 1024).
// Returns the exclusive prefix; *total receives the block sum (all threads).
__device__ __forceinline__ int block_exclusive_scan(int v, int* smem_warp /* >= 32 ints */, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) smem_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nw ? smem_warp[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < nw) smem_warp[lane] = wi - w;  // exclusive warp offsets
        if (lane == 31) smem_warp[32] = wi;       // block total
    }
    __syncthreads();
    int res = smem_warp[warp] + incl - v;
    *total = smem_warp[32];
    __syncthreads();
    return res;
}

// Device-wide exclusive scan of block counts (single CTA): out[i] = sum_{j<i} in[i];
// *total_out = min(sum, cap) if cap >= 0 else sum; overflow raises NPVS_ERR_CAPACITY.
__global__ void scan_block_counts_kernel(const int* in, int* out, int n, int* total_out, int cap,
                                         int32_t* status);

npvs_status scan_block_counts(const int* in, int* out, int n, int* total_out, int cap,
                              int32_t* status, cudaStream_t st);

}  // namespace npvs
