// Status/error entry points, the host-side frustum setup (a1) and the shared scan kernel.
#include <cuda.h>

#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "common.cuh"

namespace npvs {

static thread_local char g_err[512] = "";
static std::atomic<unsigned long long> g_launches{0};
static std::atomic<long long> g_wait_limit{kDefaultWaitCycles};

long long wait_limit_cycles() { return g_wait_limit.load(std::memory_order_relaxed); }

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

bool pdl_enabled() {
    static const bool on = [] {
        const char* v = std::getenv("NPVS_PDL");
        return !(v && v[0] == '0');
    }();
    return on;
}

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

namespace {
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

template <typename Fn>
Fn driver_fn(const char* name) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        return reinterpret_cast<Fn>(f);
    return nullptr;
}
}  // namespace

unsigned long long current_context_id() {
    static const CtxGetCurrentFn get_current = driver_fn<CtxGetCurrentFn>("cuCtxGetCurrent");
    static const CtxGetIdFn get_id = driver_fn<CtxGetIdFn>("cuCtxGetId");
    if (!get_current || !get_id) return 0;
    CUcontext c = nullptr;
    if (get_current(&c) != CUDA_SUCCESS || c == nullptr) return 0;
    unsigned long long id = 0;
    if (get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

npvs_status ensure_dynamic_smem(const void* kernel, int bytes, std::atomic<unsigned long long>* seen,
                                const char* what) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error("%s: cudaGetDevice: %s", what, cudaGetErrorString(e));
        return NPVS_ERR_CUDA;
    }
    const bool slot = dev >= 0 && dev < kMaxDevices;
    unsigned long long id = current_context_id();
    if (slot && id != 0 && seen[dev].load(std::memory_order_acquire) == id) return NPVS_OK;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) {
        set_error("%s: cudaFuncSetAttribute: %s", what, cudaGetErrorString(e));
        return NPVS_ERR_CUDA;
    }
    if (id == 0) id = current_context_id();  // the runtime call above made the primary context current
    if (slot) seen[dev].store(id, std::memory_order_release);
    return NPVS_OK;
}

// One CTA of 1024 threads scans n block counts in chunks of 1024.
__global__ void scan_block_counts_kernel(const int* in, int* out, int n, int* total_out, int cap,
                                         int32_t* status) {
    pdl_begin();
    __shared__ int sw[33];
    int carry = 0;
    for (int base = 0; base < n; base += blockDim.x) {
        int i = base + threadIdx.x;
        int v = i < n ? in[i] : 0;
        int tot;
        int ex = block_exclusive_scan(v, sw, &tot);
        if (i < n) out[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        int t = carry;
        if (cap >= 0 && t > cap) {
            raise_status(status, NPVS_ERR_CAPACITY);
            t = cap;
        }
        *total_out = t;
    }
}

npvs_status scan_block_counts(const int* in, int* out, int n, int* total_out, int cap,
                              int32_t* status, cudaStream_t st) {
    launch_k(scan_block_counts_kernel, 1, 1024, 0, st, in, out, n, total_out, cap, status);
    return check_launch("scan_block_counts");
}

}  // namespace npvs

using namespace npvs;

extern "C" const char* npvs_last_error(void) { return g_err; }

extern "C" const char* npvs_version(void) { return "npvs 0.1 (sm_103a)"; }

extern "C" unsigned long long npvs_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

extern "C" npvs_status npvs_set_wait_limit(int64_t cycles, int64_t* previous) {
    NPVS_REQUIRE(cycles >= 0, NPVS_ERR_INVALID_ARG, "npvs_set_wait_limit: cycles < 0");
    const long long old = g_wait_limit.exchange(cycles > 0 ? (long long)cycles : kDefaultWaitCycles);
    if (previous) *previous = old;
    return NPVS_OK;
}

extern "C" npvs_status npvs_check_status(int32_t* status, void* stream) {
    NPVS_REQUIRE(status != nullptr, NPVS_ERR_INVALID_ARG, "npvs_check_status: status is NULL");
    int32_t h = 0;
    cudaStream_t st = as_stream(stream);
    if (cudaMemcpyAsync(&h, status, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemsetAsync(status, 0, sizeof(int32_t), st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        set_error("npvs_check_status: %s", cudaGetErrorString(cudaGetLastError()));
        return NPVS_ERR_CUDA;
    }
    if (h == 0) return NPVS_OK;
    for (int s = 1; s < 31; ++s)
        if (h & (1 << s)) {
            set_error("device status word 0x%x", h);
            return (npvs_status)s;
        }
    return NPVS_ERR_CUDA;
}

extern "C" npvs_status npvs_camera_setup(const npvs_viewcell* vc, int32_t n_slices, npvs_camera* out) {
    NPVS_REQUIRE(vc && out, NPVS_ERR_INVALID_ARG, "npvs_camera_setup: NULL argument");
    NPVS_REQUIRE(n_slices >= 1 && n_slices <= NPVS_MAX_SLICES, NPVS_ERR_INVALID_ARG,
                 "npvs_camera_setup: n_slices out of range");
    NPVS_REQUIRE(vc->near_ > 0 && vc->far_ > vc->near_ && vc->half_size >= 0, NPVS_ERR_INVALID_ARG,
                 "npvs_camera_setup: need 0 < near < far and half_size >= 0");
    const double pi = 3.14159265358979323846;
    const double deg = pi / 180.0;
    double theta = vc->fov_deg * deg;
    double beta = vc->rot_deg * deg;
    NPVS_REQUIRE(theta > 0 && theta + 2 * beta < pi, NPVS_ERR_INVALID_ARG,
                 "npvs_camera_setup: need 0 < theta and theta + 2 beta < 180 degrees");
    double phi = 0.5 * (theta + 2.0 * beta);
    double psi = vc->yaw;
    double f[3] = {std::sin(psi), 0.0, std::cos(psi)};
    double r[3] = {std::cos(psi), 0.0, -std::sin(psi)};
    double u[3] = {0.0, 1.0, 0.0};
    double h = vc->half_size;
    double delta = h / std::tan(0.5 * theta) + h;
    std::memset(out, 0, sizeof(*out));
    for (int i = 0; i < 3; ++i) {
        out->origin[i] = (float)(vc->centre[i] - delta * f[i]);
        out->right[i] = (float)r[i];
        out->up[i] = (float)u[i];
        out->fwd[i] = (float)f[i];
    }
    out->tan_half = (float)std::tan(phi);
    out->n_slices = n_slices;
    double nr = vc->near_, fr = vc->far_;
    for (int k = 0; k <= n_slices; ++k)
        out->slices[k] = (float)(nr * std::pow(fr / nr, (double)k / (double)n_slices));
    return NPVS_OK;
}
