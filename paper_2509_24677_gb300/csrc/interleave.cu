// a3: sparse 3-D interleave g_d and a7: de-interleave g_d^-1 + sigmoid + threshold + G mask
// (Sec. 3.3 "3D volume-preserving interleaving"; Sec. 3.1 threshold tau; Sec. 3.2 supp(V) in G).
//
// Interleave: three launches. (1) one thread per coarse site tests its d^3 occupancy bits (d
// divides 32, so each (z, y) row of a block is a bit field of one word) and each CTA counts its
// active sites; (2) one CTA scans the CTA counts; (3) each CTA re-tests its sites, ranks them
// with a block scan, writes coords / table, and then writes the feature rows of its active sites
// cooperatively, 8 channels (16 B of BF16) per thread, so consecutive threads store consecutive
// bytes of a row.
#include <cuda_bf16.h>

#include "common.cuh"

namespace npvs {
namespace {

constexpr int kSitesPerCta = 256;

struct ILParams {
    const uint32_t* bits;
    npvs_grid g;
    int d, in_ch, dtype, cap;
    int Xc, Yc, Zc;
    long long n_sites;
};

__device__ __forceinline__ bool site_active(const ILParams& p, long long site, int& b, int& Z, int& Y,
                                            int& X) {
    X = (int)(site % p.Xc);
    long long t = site / p.Xc;
    Y = (int)(t % p.Yc);
    t /= p.Yc;
    Z = (int)(t % p.Zc);
    b = (int)(t / p.Zc);
    const int d = p.d, WW = p.g.W >> 5, x0 = d * X;
    const uint32_t mask = d == 32 ? 0xffffffffu : (((1u << d) - 1u) << (x0 & 31));
    const uint32_t* w = p.bits + (((size_t)b * p.g.D + (size_t)d * Z) * p.g.H + (size_t)d * Y) * WW + (x0 >> 5);
    for (int dz = 0; dz < d; ++dz)
        for (int dy = 0; dy < d; ++dy)
            if (w[((size_t)dz * p.g.H + dy) * WW] & mask) return true;
    return false;
}

__global__ void __launch_bounds__(kSitesPerCta) il_count_kernel(ILParams p, int* __restrict__ counts) {
    long long site = (long long)blockIdx.x * kSitesPerCta + threadIdx.x;
    int b, Z, Y, X;
    int f = site < p.n_sites ? (int)site_active(p, site, b, Z, Y, X) : 0;
    int c = __syncthreads_count(f);
    if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

// value of interleaved channel ch of site (b, Z, Y, X)
__device__ __forceinline__ float il_value(const ILParams& p, int b, int Z, int Y, int X, int ch) {
    const int d = p.d, d3 = d * d * d;
    int c = ch / d3, r = ch - c * d3;
    int dz = r / (d * d), dy = (r / d) % d, dx = r % d;
    int x = d * X + dx, y = d * Y + dy, k = d * Z + dz;
    const int WW = p.g.W >> 5;
    uint32_t w = p.bits[(((size_t)b * p.g.D + k) * p.g.H + y) * WW + (x >> 5)];
    bool occ = (w >> (x & 31)) & 1u;
    if (c == 0) return occ ? 1.0f : 0.0f;
    return occ ? __fdiv_rn((float)(2 * k + 1), (float)(2 * p.g.D)) : 0.0f;
}

__global__ void __launch_bounds__(kSitesPerCta) il_write_kernel(ILParams p, const int* __restrict__ block_off,
                                                                int32_t* __restrict__ coords, void* __restrict__ feats,
                                                                int32_t* __restrict__ table, int32_t* status) {
    __shared__ int sw[33];
    __shared__ int4 s_site[kSitesPerCta];
    __shared__ int s_rank[kSitesPerCta];
    long long site = (long long)blockIdx.x * kSitesPerCta + threadIdx.x;
    int b = 0, Z = 0, Y = 0, X = 0;
    bool in = site < p.n_sites;
    int f = in ? (int)site_active(p, site, b, Z, Y, X) : 0;
    int nloc;
    int loc = block_exclusive_scan(f, sw, &nloc);
    int rank = block_off[blockIdx.x] + loc;
    if (in && table) table[site] = (f && rank < p.cap) ? rank : -1;
    if (f) {
        if (rank < p.cap) {
            reinterpret_cast<int4*>(coords)[rank] = make_int4(b, Z, Y, X);
        } else {
            raise_status(status, NPVS_ERR_CAPACITY);
        }
        s_site[loc] = make_int4(b, Z, Y, X);
        s_rank[loc] = rank;
    }
    __syncthreads();
    const int C = p.in_ch * p.d * p.d * p.d;
    const int vec = (C % 8 == 0) ? 8 : 1;
    const int chunks = C / vec;
    for (int e = threadIdx.x; e < nloc * chunks; e += kSitesPerCta) {
        int i = e / chunks, ch0 = (e - i * chunks) * vec;
        int r = s_rank[i];
        if (r >= p.cap) continue;
        int4 s = s_site[i];
        size_t off = (size_t)r * C + ch0;
        if (p.dtype == NPVS_BF16) {
            __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(feats) + off;
            if (vec == 8) {
                __align__(16) __nv_bfloat16 v[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) v[q] = __float2bfloat16_rn(il_value(p, s.x, s.y, s.z, s.w, ch0 + q));
                *reinterpret_cast<uint4*>(out) = *reinterpret_cast<uint4*>(v);
            } else {
                out[0] = __float2bfloat16_rn(il_value(p, s.x, s.y, s.z, s.w, ch0));
            }
        } else if (p.dtype == NPVS_F32) {
            float* out = reinterpret_cast<float*>(feats) + off;
            for (int q = 0; q < vec; ++q) out[q] = il_value(p, s.x, s.y, s.z, s.w, ch0 + q);
        } else {
            double* out = reinterpret_cast<double*>(feats) + off;
            for (int q = 0; q < vec; ++q) out[q] = (double)il_value(p, s.x, s.y, s.z, s.w, ch0 + q);
        }
    }
}

// ---- de-interleave ------------------------------------------------------------------------

__global__ void deinterleave_kernel(const float* __restrict__ logits, const int32_t* __restrict__ table,
                                    const int32_t* __restrict__ n_active, npvs_grid g, int d, float tau,
                                    const uint32_t* __restrict__ mask_bits, uint32_t* __restrict__ pvs) {
    const int WW = g.W >> 5;
    const long long n_words = (long long)g.B * g.D * g.H * WW;
    const int n = *n_active;
    const int Xc = g.W / d, Yc = g.H / d, Zc = g.D / d, d3 = d * d * d;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < n_words;
         w += (long long)gridDim.x * blockDim.x) {
        uint32_t m = mask_bits[w];
        uint32_t out = 0;
        if (m) {
            int xw = (int)(w % WW);
            long long t = w / WW;
            int y = (int)(t % g.H);
            t /= g.H;
            int k = (int)(t % g.D);
            int b = (int)(t / g.D);
            int Y = y / d, dy = y - Y * d, Z = k / d, dz = k - Z * d;
            long long rowbase = (((long long)b * Zc + Z) * Yc + Y) * Xc;
            while (m) {
                int i = __ffs(m) - 1;
                m &= m - 1;
                int x = xw * 32 + i, X = x / d, dx = x - X * d;
                int row = table[rowbase + X];
                if (row >= 0 && row < n) {
                    float z = logits[(size_t)row * d3 + (dz * d + dy) * d + dx];
                    float pr = 1.0f / (1.0f + expf(-z));
                    if (pr >= tau) out |= 1u << i;
                }
            }
        }
        pvs[w] = out;
    }
}

__global__ void sigmoid_rows_kernel(const float* __restrict__ logits, const int32_t* __restrict__ n_active,
                                    int d3, float* __restrict__ probs) {
    const long long n = (long long)(*n_active) * d3;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        probs[i] = 1.0f / (1.0f + expf(-logits[i]));
}

}  // namespace
}  // namespace npvs

using namespace npvs;

static bool valid_d(int d) { return d == 1 || d == 2 || d == 4 || d == 8 || d == 16 || d == 32; }

extern "C" size_t npvs_interleave_workspace_bytes(npvs_grid g, int32_t d) {
    if (!valid_d(d) || d <= 0) return 0;
    long long sites = (long long)g.B * (g.W / d) * (g.H / d) * (g.D / d);
    long long nb = (sites + kSitesPerCta - 1) / kSitesPerCta;
    return 2 * Arena::round((size_t)(nb + 1) * sizeof(int)) + 256;
}

extern "C" npvs_status npvs_interleave(const uint32_t* occ_bits, npvs_grid g, int32_t d, int32_t in_ch,
                                       int32_t feat_dtype, int32_t capacity, int32_t* coords, void* feats,
                                       int32_t* n_active, int32_t* table, int32_t* status, void* workspace,
                                       size_t workspace_bytes, void* stream) {
    NPVS_REQUIRE(occ_bits && coords && feats && n_active, NPVS_ERR_INVALID_ARG, "npvs_interleave: NULL pointer");
    NPVS_REQUIRE(valid_d(d), NPVS_ERR_UNSUPPORTED, "npvs_interleave: d must divide 32");
    NPVS_REQUIRE(g.W > 0 && g.H > 0 && g.D > 0 && g.B > 0 && g.W % 32 == 0 && g.W % d == 0 &&
                     g.H % d == 0 && g.D % d == 0,
                 NPVS_ERR_UNSUPPORTED, "npvs_interleave: grid must be a multiple of d (and W of 32)");
    NPVS_REQUIRE(in_ch == 1 || in_ch == 2, NPVS_ERR_UNSUPPORTED, "npvs_interleave: in_ch must be 1 or 2");
    NPVS_REQUIRE(feat_dtype == NPVS_F32 || feat_dtype == NPVS_BF16 || feat_dtype == NPVS_F64,
                 NPVS_ERR_UNSUPPORTED, "npvs_interleave: bad feat_dtype");
    NPVS_REQUIRE(capacity >= 0, NPVS_ERR_INVALID_ARG, "npvs_interleave: capacity < 0");
    NPVS_REQUIRE(workspace && workspace_bytes >= npvs_interleave_workspace_bytes(g, d), NPVS_ERR_WORKSPACE,
                 "npvs_interleave: workspace too small");
    cudaStream_t st = as_stream(stream);
    ILParams p;
    p.bits = occ_bits;
    p.g = g;
    p.d = d;
    p.in_ch = in_ch;
    p.dtype = feat_dtype;
    p.cap = capacity;
    p.Xc = g.W / d;
    p.Yc = g.H / d;
    p.Zc = g.D / d;
    p.n_sites = (long long)g.B * p.Xc * p.Yc * p.Zc;
    const int nb = ceil_div(p.n_sites, kSitesPerCta);
    Arena ar(workspace, workspace_bytes);
    int* counts = ar.take<int>(nb + 1);
    int* offs = ar.take<int>(nb + 1);
    il_count_kernel<<<nb, kSitesPerCta, 0, st>>>(p, counts);
    NPVS_TRY(check_launch("il_count_kernel"));
    NPVS_TRY(scan_block_counts(counts, offs, nb, n_active, capacity, status, st));
    il_write_kernel<<<nb, kSitesPerCta, 0, st>>>(p, offs, coords, feats, table, status);
    return check_launch("il_write_kernel");
}

extern "C" npvs_status npvs_deinterleave(const float* logits, const int32_t* table, const int32_t* n_active,
                                         npvs_grid g, int32_t d, float tau, const uint32_t* mask_bits,
                                         uint32_t* pvs_bits, float* probs_out, int32_t capacity, void* stream) {
    NPVS_REQUIRE(logits && table && n_active && mask_bits && pvs_bits, NPVS_ERR_INVALID_ARG,
                 "npvs_deinterleave: NULL pointer");
    NPVS_REQUIRE(valid_d(d) && g.W % 32 == 0 && g.W % d == 0 && g.H % d == 0 && g.D % d == 0 && g.B > 0,
                 NPVS_ERR_UNSUPPORTED, "npvs_deinterleave: unsupported grid / d");
    cudaStream_t st = as_stream(stream);
    long long words = (long long)g.B * g.D * g.H * (g.W / 32);
    int blocks = (int)std::min<long long>(ceil_div(words, 256), kNumSMs * 16);
    deinterleave_kernel<<<blocks, 256, 0, st>>>(logits, table, n_active, g, d, tau, mask_bits, pvs_bits);
    NPVS_TRY(check_launch("deinterleave_kernel"));
    if (probs_out) {
        int d3 = d * d * d;
        int pb = (int)std::min<long long>(ceil_div((long long)capacity * d3, 256), kNumSMs * 16);
        if (pb > 0) sigmoid_rows_kernel<<<pb, 256, 0, st>>>(logits, n_active, d3, probs_out);
        NPVS_TRY(check_launch("sigmoid_rows_kernel"));
    }
    return NPVS_OK;
}

// ---- interleave for callers that cannot allocate ----------------------------------------------
//
// npvs_interleave needs a small scratch area (per-CTA counts and their prefix sums) that the caller
// normally passes in. Some callers cannot hand out device memory at all: a renderer or game engine
// that reserves its whole GPU heap at start-up and forbids allocations during a frame, or code that
// runs where calling cudaMalloc is not permitted (inside a frame's time budget, or from a thread
// that must not synchronise the device, which cudaMalloc/cudaFree may do). For them
// npvs_interleave_noalloc keeps that scratch in a fixed array that lives in the library's own
// device memory for as long as the library is loaded.
#include <mutex>

namespace {
constexpr long long kNoAllocMaxSites = 1ll << 22;  // 4,194,304 coarse sites per call (all batches)
constexpr int kNoAllocMaxCtas = (int)(kNoAllocMaxSites / npvs::kSitesPerCta);
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
int* g_noalloc_ptr[kNoAllocMaxDevices] = {};
}  // namespace

// counts [kNoAllocMaxCtas + 1] then offsets [kNoAllocMaxCtas + 1] (128 KiB per device)
static __device__ __align__(256) int npvs_interleave_scratch[2 * (kNoAllocMaxCtas + 1)];

extern "C" npvs_status npvs_interleave_noalloc(const uint32_t* occ_bits, npvs_grid g, int32_t d, int32_t in_ch,
                                               int32_t feat_dtype, int32_t capacity, int32_t* coords, void* feats,
                                               int32_t* n_active, int32_t* table, int32_t* status, void* stream) {
    NPVS_REQUIRE(occ_bits && coords && feats && n_active, NPVS_ERR_INVALID_ARG,
                 "npvs_interleave_noalloc: NULL pointer");
    NPVS_REQUIRE(valid_d(d), NPVS_ERR_UNSUPPORTED, "npvs_interleave_noalloc: d must divide 32");
    NPVS_REQUIRE(g.W > 0 && g.H > 0 && g.D > 0 && g.B > 0 && g.W % 32 == 0 && g.W % d == 0 &&
                     g.H % d == 0 && g.D % d == 0,
                 NPVS_ERR_UNSUPPORTED, "npvs_interleave_noalloc: grid must be a multiple of d (and W of 32)");
    NPVS_REQUIRE(in_ch == 1 || in_ch == 2, NPVS_ERR_UNSUPPORTED, "npvs_interleave_noalloc: in_ch must be 1 or 2");
    NPVS_REQUIRE(feat_dtype == NPVS_F32 || feat_dtype == NPVS_BF16 || feat_dtype == NPVS_F64,
                 NPVS_ERR_UNSUPPORTED, "npvs_interleave_noalloc: bad feat_dtype");
    NPVS_REQUIRE(capacity >= 0, NPVS_ERR_INVALID_ARG, "npvs_interleave_noalloc: capacity < 0");
    const long long n_sites = (long long)g.B * (g.W / d) * (g.H / d) * (g.D / d);
    if (n_sites > kNoAllocMaxSites) {
        set_error("npvs_interleave_noalloc: %lld coarse sites exceed the fixed scratch limit of %lld "
                  "(use npvs_interleave with a workspace)",
                  n_sites, kNoAllocMaxSites);
        return NPVS_ERR_UNSUPPORTED;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("npvs_interleave_noalloc: no usable current device");
        return NPVS_ERR_CUDA;
    }
    int* scratch;
    {
        // the device address of the array, looked up once per device (with that device current)
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (g_noalloc_ptr[dev] == nullptr) {
            void* ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, npvs_interleave_scratch);
            if (e != cudaSuccess || ptr == nullptr) {
                set_error("npvs_interleave_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
                return NPVS_ERR_CUDA;
            }
            g_noalloc_ptr[dev] = static_cast<int*>(ptr);
        }
        scratch = g_noalloc_ptr[dev];
    }
    cudaStream_t st = as_stream(stream);
    ILParams p;
    p.bits = occ_bits;
    p.g = g;
    p.d = d;
    p.in_ch = in_ch;
    p.dtype = feat_dtype;
    p.cap = capacity;
    p.Xc = g.W / d;
    p.Yc = g.H / d;
    p.Zc = g.D / d;
    p.n_sites = n_sites;
    const int nb = ceil_div(p.n_sites, kSitesPerCta);
    int* counts = scratch;                      // fully rewritten by every call before it is read
    int* offs = scratch + kNoAllocMaxCtas + 1;  // likewise
    il_count_kernel<<<nb, kSitesPerCta, 0, st>>>(p, counts);
    NPVS_TRY(check_launch("il_count_kernel"));
    NPVS_TRY(scan_block_counts(counts, offs, nb, n_active, capacity, status, st));
    il_write_kernel<<<nb, kSitesPerCta, 0, st>>>(p, offs, coords, feats, table, status);
    return check_launch("il_write_kernel");
}
