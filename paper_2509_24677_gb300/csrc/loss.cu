// a8/a9: weighted Dice + repulsive visibility loss (Sec. 3.3) and its gradient w.r.t. the logits.
//
// Sums per sample b, with y the ground-truth bit and g the geometry bit of a froxel and
// p~ = sigmoid(z) * g the soft prediction masked by the geometry grid:
//   TP = sum y p~,  FP = sum (1 - y) p~,  GTP = popcount of the sample's ground-truth grid,
//   FN = GTP - TP,  NOCC = sum g,  BCE = sum g (max(z, 0) - z y + log1p(exp(-|z|)))
//   L_dice = 1 - (2 TP + eps) / (2 TP + alpha FN + (1 - alpha) FP + eps)
//   L_attr = FN / (GTP + eps),  L_rep = FP / (GTP + eps)
//   L_b = lambda L_dice + (1 - lambda)(L_attr + L_rep) + w_bce BCE / NOCC,   L = mean_b L_b.
// (The paper's prose and printed formulas name FN / FP the other way round and print the
// attraction term with the opposite sign; these are the readings of the library.)
//
// Determinism: every sum is taken in a fixed order that depends only on the row capacity and
// the data: a warp reduces one row's d^3 channels with a fixed butterfly, one CTA per sample then
// adds its rows in a fixed strided order and a fixed tree, and the last CTA averages the
// samples in index order. Integer counts are exact.
#include "common.cuh"

namespace npvs {
namespace {

constexpr int kRowsCta = 256;  // 8 warps, one row each per iteration
constexpr int kRedCta = 512;

struct LossGeom {
    npvs_grid g;
    int d, d3, WW;
};

// Bit of froxel channel j of coarse site c = (b, Z, Y, X) in a [B][D][H][W/32] grid.
__device__ __forceinline__ uint32_t site_bit(const uint32_t* __restrict__ bits, const LossGeom& G, int4 c, int j) {
    const int d = G.d;
    const int dz = j / (d * d), dy = (j / d) % d, dx = j % d;
    const int z = c.y * d + dz, y = c.z * d + dy, x = c.w * d + dx;
    const size_t w = (((size_t)c.x * G.g.D + z) * G.g.H + y) * G.WW + (x >> 5);
    return (__ldg(bits + w) >> (x & 31)) & 1u;
}

__device__ __forceinline__ float sigmoid_t(float z) { return 1.0f / (1.0f + expf(-z)); }
__device__ __forceinline__ double sigmoid_t(double z) { return 1.0 / (1.0 + exp(-z)); }
__device__ __forceinline__ float log1p_t(float v) { return log1pf(v); }
__device__ __forceinline__ double log1p_t(double v) { return log1p(v); }
__device__ __forceinline__ float exp_t(float v) { return expf(v); }
__device__ __forceinline__ double exp_t(double v) { return exp(v); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-row partial sums (TP, FP, BCE, NOCC) of rows < n.
template <typename T>
__global__ void __launch_bounds__(kRowsCta) loss_rows_kernel(const T* __restrict__ z, const int32_t* __restrict__ coords,
                                                             const int32_t* __restrict__ n_rows, int cap,
                                                             const uint32_t* __restrict__ gt, const uint32_t* __restrict__ gb,
                                                             LossGeom G, int with_bce, T* __restrict__ part,
                                                             unsigned int* __restrict__ counter) {
    pdl_begin();
    if (blockIdx.x == 0 && threadIdx.x == 0) *counter = 0u;
    const int n = min(*n_rows, cap);
    const int lane = threadIdx.x & 31;
    const int wpc = kRowsCta / 32;
    for (int r = blockIdx.x * wpc + (threadIdx.x >> 5); r < n; r += gridDim.x * wpc) {
        const int4 c = reinterpret_cast<const int4*>(coords)[r];
        T tp = 0, fp = 0, bce = 0, nocc = 0;
        for (int j = lane; j < G.d3; j += 32) {
            if (!site_bit(gb, G, c, j)) continue;
            const T zz = z[(size_t)r * G.d3 + j];
            const T p = sigmoid_t(zz);
            const bool y = site_bit(gt, G, c, j);
            if (y) tp += p; else fp += p;
            nocc += T(1);
            if (with_bce) bce += (zz > T(0) ? zz : T(0)) - (y ? zz : T(0)) + log1p_t(exp_t(-fabs(zz)));
        }
        tp = warp_sum(tp);
        fp = warp_sum(fp);
        bce = warp_sum(bce);
        nocc = warp_sum(nocc);
        if (lane == 0) {
            T* o = part + (size_t)r * 4;
            o[0] = tp;
            o[1] = fp;
            o[2] = bce;
            o[3] = nocc;
        }
    }
}

// First row index in [0, n) whose batch index is >= b (coords sorted by batch first).
__device__ __forceinline__ int lower_row(const int32_t* coords, int n, int b) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (coords[(size_t)mid * 4] < b) lo = mid + 1; else hi = mid;
    }
    return lo;
}

template <typename T>
__global__ void __launch_bounds__(kRedCta) loss_reduce_kernel(const T* __restrict__ part, const int32_t* __restrict__ coords,
                                                              const int32_t* __restrict__ n_rows, int cap,
                                                              const uint32_t* __restrict__ gt, LossGeom G,
                                                              npvs_loss_params prm, T* __restrict__ terms,
                                                              T* __restrict__ loss, unsigned int* __restrict__ counter) {
    pdl_begin();
    __shared__ T s[4][kRedCta];
    __shared__ unsigned long long sg[kRedCta];
    __shared__ bool last;
    const int b = blockIdx.x, B = gridDim.x, tid = threadIdx.x;
    const int n = min(*n_rows, cap);
    const int lo = lower_row(coords, n, b), hi = lower_row(coords, n, b + 1);
    T acc[4] = {0, 0, 0, 0};
    for (int r = lo + tid; r < hi; r += kRedCta) {
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] += part[(size_t)r * 4 + q];
    }
    const size_t words = (size_t)G.g.D * G.g.H * G.WW;
    const uint32_t* gw = gt + (size_t)b * words;
    unsigned long long pc = 0;
    for (size_t w = tid; w < words; w += kRedCta) pc += __popc(__ldg(gw + w));
#pragma unroll
    for (int q = 0; q < 4; ++q) s[q][tid] = acc[q];
    sg[tid] = pc;
    __syncthreads();
    for (int h = kRedCta / 2; h > 0; h >>= 1) {
        if (tid < h) {
#pragma unroll
            for (int q = 0; q < 4; ++q) s[q][tid] += s[q][tid + h];
            sg[tid] += sg[tid + h];
        }
        __syncthreads();
    }
    if (tid == 0) {
        const T tp = s[0][0], fp = s[1][0], bce = s[2][0], nocc = s[3][0];
        const T gtp = (T)sg[0];
        const T al = prm.alpha, ep = prm.eps, lam = prm.lam, wb = prm.w_bce;
        const T fn = gtp - tp;
        const T S = T(2) * tp + al * fn + (T(1) - al) * fp + ep;
        const T N = T(2) * tp + ep;
        const T dice = T(1) - N / S;
        const T attr = fn / (gtp + ep), rep = fp / (gtp + ep);
        const T bmean = (wb != T(0) && nocc > T(0)) ? bce / nocc : T(0);
        const T Lb = lam * dice + (T(1) - lam) * (attr + rep) + wb * bmean;
        T* t = terms + (size_t)b * NPVS_LOSS_TERMS;
        t[NPVS_LT_L] = Lb;
        t[NPVS_LT_DICE] = dice;
        t[NPVS_LT_ATTR] = attr;
        t[NPVS_LT_REP] = rep;
        t[NPVS_LT_BCE] = bmean;
        t[NPVS_LT_GTP] = gtp;
        t[NPVS_LT_TP] = tp;
        t[NPVS_LT_FN] = fn;
        t[NPVS_LT_FP] = fp;
        t[NPVS_LT_NOCC] = nocc;
        // dL/dTP and dL/dFP of the batch mean (FN = GTP - TP)
        t[NPVS_LT_DTP] = (lam * (-(T(2) * S - N * (T(2) - al)) / (S * S)) - (T(1) - lam) / (gtp + ep)) / T(B);
        t[NPVS_LT_DFP] = (lam * (N * (T(1) - al) / (S * S)) + (T(1) - lam) / (gtp + ep)) / T(B);
        __threadfence();
        last = atomicAdd(counter, 1u) == (unsigned)(B - 1);
    }
    __syncthreads();
    if (last && tid == 0) {
        __threadfence();
        T m = 0;
        for (int i = 0; i < B; ++i) m += ((volatile T*)terms)[(size_t)i * NPVS_LOSS_TERMS + NPVS_LT_L];
        *loss = m / T(B);
        *counter = 0u;
    }
}

template <typename T, typename O>
__device__ __forceinline__ void store_grad(O* out, size_t i, T v);
template <>
__device__ __forceinline__ void store_grad<float, float>(float* out, size_t i, float v) { out[i] = v; }
template <>
__device__ __forceinline__ void store_grad<float, __nv_bfloat16>(__nv_bfloat16* out, size_t i, float v) {
    out[i] = __float2bfloat16_rn(v);
}
template <>
__device__ __forceinline__ void store_grad<double, double>(double* out, size_t i, double v) { out[i] = v; }

// dL/dz = dloss * g * ( p (1 - p) (y dL/dTP + (1 - y) dL/dFP) + w_bce (p - y) / (B NOCC) ).
template <typename T, typename O>
__global__ void __launch_bounds__(256) loss_bwd_kernel(const T* __restrict__ z, const int32_t* __restrict__ coords,
                                                       const int32_t* __restrict__ n_rows, int cap,
                                                       const uint32_t* __restrict__ gt, const uint32_t* __restrict__ gb,
                                                       LossGeom G, T w_bce, const T* __restrict__ terms,
                                                       const T* __restrict__ dloss, O* __restrict__ dz) {
    pdl_begin();
    const int n = min(*n_rows, cap);
    const size_t total = (size_t)n * G.d3;
    const T dl = dloss ? *dloss : T(1);
    const T B = (T)G.g.B;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / G.d3), j = (int)(e - (size_t)r * G.d3);
        const int4 c = reinterpret_cast<const int4*>(coords)[r];
        T v = 0;
        if (site_bit(gb, G, c, j)) {
            const T* t = terms + (size_t)c.x * NPVS_LOSS_TERMS;
            const T zz = z[e];
            const T p = sigmoid_t(zz);
            const bool y = site_bit(gt, G, c, j);
            v = p * (T(1) - p) * (y ? t[NPVS_LT_DTP] : t[NPVS_LT_DFP]);
            if (w_bce != T(0)) v += w_bce * (p - (y ? T(1) : T(0))) / (B * t[NPVS_LT_NOCC]);
            v *= dl;
        }
        store_grad<T, O>(dz, e, v);
    }
}

npvs_status loss_geom(npvs_grid g, int d, int capacity, LossGeom* G, const char* who) {
    (void)who;
    NPVS_REQUIRE(g.W > 0 && g.H > 0 && g.D > 0 && g.B > 0 && g.W % 32 == 0, NPVS_ERR_INVALID_ARG,
                 "npvs_loss: grid needs W a positive multiple of 32 and positive H, D, B");
    NPVS_REQUIRE(d >= 1 && d <= 16 && g.W % d == 0 && g.H % d == 0 && g.D % d == 0, NPVS_ERR_UNSUPPORTED,
                 "npvs_loss: d must divide W, H and D (1 <= d <= 16)");
    NPVS_REQUIRE(capacity >= 0, NPVS_ERR_INVALID_ARG, "npvs_loss: negative capacity");
    G->g = g;
    G->d = d;
    G->d3 = d * d * d;
    G->WW = g.W / 32;
    return NPVS_OK;
}

int rows_grid(int cap) { return std::max(1, std::min(ceil_div(cap, kRowsCta / 32), kNumSMs * 8)); }

}  // namespace
}  // namespace npvs

using namespace npvs;

extern "C" size_t npvs_loss_workspace_bytes(int32_t capacity, int32_t dtype) {
    const size_t el = dtype == NPVS_F64 ? 8 : 4;
    return Arena::round((size_t)std::max(capacity, 1) * 4 * el) + Arena::round(sizeof(unsigned int)) + 256;
}

extern "C" npvs_status npvs_loss_fwd(int32_t dtype, const void* logits, const int32_t* coords, const int32_t* n_rows,
                                     int32_t capacity, const uint32_t* gt_bits, const uint32_t* g_bits, npvs_grid grid,
                                     int32_t d, const npvs_loss_params* prm, void* terms, void* loss, void* workspace,
                                     size_t workspace_bytes, void* stream) {
    NPVS_REQUIRE(logits && coords && n_rows && gt_bits && g_bits && prm && terms && loss, NPVS_ERR_INVALID_ARG,
                 "npvs_loss_fwd: NULL argument");
    NPVS_REQUIRE(dtype == NPVS_F32 || dtype == NPVS_F64, NPVS_ERR_UNSUPPORTED, "npvs_loss_fwd: dtype must be F32 or F64");
    LossGeom G;
    NPVS_TRY(loss_geom(grid, d, capacity, &G, "npvs_loss_fwd"));
    NPVS_REQUIRE(workspace && workspace_bytes >= npvs_loss_workspace_bytes(capacity, dtype), NPVS_ERR_WORKSPACE,
                 "npvs_loss_fwd: workspace smaller than npvs_loss_workspace_bytes()");
    cudaStream_t st = as_stream(stream);
    Arena ar(workspace, workspace_bytes);
    const int with_bce = prm->w_bce != 0.0f;
    if (dtype == NPVS_F32) {
        float* part = ar.take<float>((size_t)std::max(capacity, 1) * 4);
        unsigned int* cnt = ar.take<unsigned int>(1);
        launch_k(loss_rows_kernel<float>, rows_grid(capacity), kRowsCta, 0, st, (const float*)logits, coords, n_rows,
                 capacity, gt_bits, g_bits, G, with_bce, part, cnt);
        NPVS_TRY(check_launch("loss_rows_kernel"));
        launch_k(loss_reduce_kernel<float>, grid.B, kRedCta, 0, st, (const float*)part, coords, n_rows, capacity, gt_bits,
                 G, *prm, (float*)terms, (float*)loss, cnt);
    } else {
        double* part = ar.take<double>((size_t)std::max(capacity, 1) * 4);
        unsigned int* cnt = ar.take<unsigned int>(1);
        launch_k(loss_rows_kernel<double>, rows_grid(capacity), kRowsCta, 0, st, (const double*)logits, coords, n_rows,
                 capacity, gt_bits, g_bits, G, with_bce, part, cnt);
        NPVS_TRY(check_launch("loss_rows_kernel"));
        launch_k(loss_reduce_kernel<double>, grid.B, kRedCta, 0, st, (const double*)part, coords, n_rows, capacity,
                 gt_bits, G, *prm, (double*)terms, (double*)loss, cnt);
    }
    return check_launch("loss_reduce_kernel");
}

extern "C" npvs_status npvs_loss_bwd(int32_t dtype, const void* logits, const int32_t* coords, const int32_t* n_rows,
                                     int32_t capacity, const uint32_t* gt_bits, const uint32_t* g_bits, npvs_grid grid,
                                     int32_t d, const npvs_loss_params* prm, const void* terms, const void* dloss,
                                     int32_t dlogits_dtype, void* dlogits, void* stream) {
    NPVS_REQUIRE(logits && coords && n_rows && gt_bits && g_bits && prm && terms && dlogits, NPVS_ERR_INVALID_ARG,
                 "npvs_loss_bwd: NULL argument");
    LossGeom G;
    NPVS_TRY(loss_geom(grid, d, capacity, &G, "npvs_loss_bwd"));
    cudaStream_t st = as_stream(stream);
    const int nb = std::max(1, std::min(ceil_div((long long)capacity * G.d3, 256), kNumSMs * 16));
    if (dtype == NPVS_F32 && dlogits_dtype == NPVS_F32) {
        launch_k(loss_bwd_kernel<float, float>, nb, 256, 0, st, (const float*)logits, coords, n_rows, capacity, gt_bits,
                 g_bits, G, (float)prm->w_bce, (const float*)terms, (const float*)dloss, (float*)dlogits);
    } else if (dtype == NPVS_F32 && dlogits_dtype == NPVS_BF16) {
        launch_k(loss_bwd_kernel<float, __nv_bfloat16>, nb, 256, 0, st, (const float*)logits, coords, n_rows, capacity,
                 gt_bits, g_bits, G, (float)prm->w_bce, (const float*)terms, (const float*)dloss, (__nv_bfloat16*)dlogits);
    } else if (dtype == NPVS_F64 && dlogits_dtype == NPVS_F64) {
        launch_k(loss_bwd_kernel<double, double>, nb, 256, 0, st, (const double*)logits, coords, n_rows, capacity,
                 gt_bits, g_bits, G, (double)prm->w_bce, (const double*)terms, (const double*)dloss, (double*)dlogits);
    } else {
        return fail(NPVS_ERR_UNSUPPORTED, "npvs_loss_bwd: dtype pairs are F32->F32, F32->BF16, F64->F64");
    }
    return check_launch("loss_bwd_kernel");
}
