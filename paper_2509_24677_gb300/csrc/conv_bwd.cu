// a10: backward of the sparse convolutions (Sec. 2.3 layers, trained with Sec. 4.2's optimiser).
//
// For a layer y = act(b + sum_t W_t^T x[map(n, t)]) with ReLU mask m = 1[y > 0]:
//   g      = dy * m                                       (grad_mask_kernel, also the bias partials)
//   db     = sum_n g[n]
//   dW_t   = sum_n x[map(n, t)]^T g[n]                    (wgrad_kernel: one reduction GEMM per tap)
//   dx[i]  = sum_{(n, t): map(n, t) = i} W_t g[n]         (dgrad)
// The dgrad is itself a forward sparse convolution over the transposed rulebook, so it runs on
// the forward kernels (tensor cores for BF16): a submanifold conv's transpose is the submanifold
// conv with the opposite taps (the neighbour map is symmetric: map(n, t) = i iff
// map(i, 26 - t) = n) and weights W_{26-t}^T; a stride-2 down conv's transpose is the up conv on
// the same level pair with W_t^T and vice versa (2x2x2: the down map and the up map; 3x3x3 with
// padding 1: the two maps of a DOWN3 rulebook, input rows of each coarse output and coarse rows of
// each fine row and tap); a 1x1 conv's transpose is the 1x1 conv with W^T.
//
// Determinism: every sum has a fixed order. Rows are cut into a fixed number of chunks of the device
// row count; each chunk's partial sums are written to the workspace and added in chunk order.
#include <type_traits>

#include "common.cuh"
#include "conv_tc.cuh"

namespace npvs {
namespace {

template <typename T> struct AccOf { using type = float; };
template <> struct AccOf<double> { using type = double; };

__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ double to_acc(double v) { return v; }

constexpr int kMaskRows = 256;
constexpr int WK = 32;  // rows per shared-memory stage of the weight-gradient kernel

// g = dy * 1[y > 0] (rows < n; not written without ReLU) and per-chunk column sums of g. The rows
// are cut into gridDim.x equal chunks of the device row count.
template <typename T, typename A>
__global__ void __launch_bounds__(256) grad_mask_kernel(const T* __restrict__ dy, const T* __restrict__ y, int relu,
                                                        const int32_t* __restrict__ n_out, int cap, int cout,
                                                        T* __restrict__ g, A* __restrict__ part_db) {
    pdl_begin();
    __shared__ A s[256];
    const int n = min(*n_out, cap);
    const int rpc = (n + gridDim.x - 1) / gridDim.x;
    const int row0 = min((int)blockIdx.x * rpc, n);
    const int rend = min(row0 + rpc, n);
    for (int o0 = 0; o0 < cout; o0 += 256) {
        const int cw = min(256, cout - o0);
        const int ge = 256 / cw;  // row phases
        const int q = threadIdx.x / cw, o = o0 + threadIdx.x % cw;
        A acc = 0;
        if (q < ge) {
            for (int r = row0 + q; r < rend; r += ge) {
                const size_t i = (size_t)r * cout + o;
                const T v = dy[i];
                if (relu) {
                    const bool on = to_acc(y[i]) > A(0);
                    g[i] = on ? v : T(0.0f);
                    if (on) acc += to_acc(v);
                } else {
                    acc += to_acc(v);
                }
            }
        }
        s[threadIdx.x] = acc;
        __syncthreads();
        if (threadIdx.x < cw) {
            A t = 0;
            for (int qq = 0; qq < ge; ++qq) t += s[qq * cw + threadIdx.x];
            part_db[(size_t)blockIdx.x * cout + o0 + threadIdx.x] = t;
        }
        __syncthreads();
    }
}

// BF16 form of grad_mask_kernel: 8 channels (16 bytes) per thread, cout / 8 threads per row, 256 /
// (cout / 8) rows per pass; the column partials are added over the passes' rows in fixed order.
__global__ void __launch_bounds__(256) grad_mask_bf16_kernel(const __nv_bfloat16* __restrict__ dy,
                                                             const __nv_bfloat16* __restrict__ y, int relu,
                                                             const int32_t* __restrict__ n_out, int cap, int cout,
                                                             __nv_bfloat16* __restrict__ g, float* __restrict__ part_db) {
    pdl_begin();
    __shared__ float s[256 * 8];
    const int n = min(*n_out, cap);
    const int rpc = (n + gridDim.x - 1) / gridDim.x;
    const int row0 = min((int)blockIdx.x * rpc, n), rend = min(row0 + rpc, n);
    const int cg = cout >> 3, rpp = 256 / cg;
    const int q = threadIdx.x / cg, grp = threadIdx.x - q * cg;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (q < rpp) {
        for (int r = row0 + q; r < rend; r += rpp) {
            const size_t i = (size_t)r * cout + grp * 8;
            uint4 v = *reinterpret_cast<const uint4*>(dy + i);
            if (relu) {
                const uint4 m = *reinterpret_cast<const uint4*>(y + i);
                const uint32_t* mw = reinterpret_cast<const uint32_t*>(&m);
                uint32_t* vw = reinterpret_cast<uint32_t*>(&v);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    // a BF16 is > 0 iff its sign bit is clear and it is not +0
                    const uint32_t lo = mw[k] & 0xFFFFu, hi = mw[k] >> 16;
                    const uint32_t keep = ((lo != 0 && !(lo & 0x8000u)) ? 0xFFFFu : 0u) |
                                          ((hi != 0 && !(hi & 0x8000u)) ? 0xFFFF0000u : 0u);
                    vw[k] &= keep;
                }
                *reinterpret_cast<uint4*>(g + i) = v;
            }
            const __nv_bfloat16* b = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] += __bfloat162float(b[k]);
        }
    }
    if (q < rpp) {
#pragma unroll
        for (int k = 0; k < 8; ++k) s[q * cout + grp * 8 + k] = acc[k];
    }
    __syncthreads();
    for (int o = threadIdx.x; o < cout; o += 256) {
        float t = 0.f;
        for (int qq = 0; qq < rpp; ++qq) t += s[qq * cout + o];
        part_db[(size_t)blockIdx.x * cout + o] = t;
    }
}

// db[o] = sum over the chunks (in order) of the bias partials: 32 columns x 8 chunk phases per CTA.
template <typename A>
__global__ void __launch_bounds__(256) grad_db_reduce_kernel(const A* __restrict__ part_db, int n_db, int cout,
                                                             A* __restrict__ db) {
    pdl_begin();
    __shared__ A s[8][32];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int o = blockIdx.x * 32 + tx;
    A acc = 0;
    if (o < cout)
        for (int c = ty; c < n_db; c += 8) acc += part_db[(size_t)c * cout + o];
    s[ty][tx] = acc;
    __syncthreads();
    if (ty == 0 && o < cout) {
        A t = 0;
        for (int k = 0; k < 8; ++k) t += s[k][tx];
        db[o] = t;
    }
}

// Per (ci tile, co tile) x tap x row chunk: sum over the chunk's rows n of x[map(n, t)]^T g[n].
// The chunk's rows are cut from the device row count (n_chunks equal chunks), so the work spreads
// over every chunk whatever the occupancy. Rows are visited in windows of 256: the rows whose
// neighbour through tap t exists are compacted in order (ballot + block scan), then consumed 16 at a
// time from shared memory into a TT x TT register tile per thread (tile TILE = 16 TT channels).
template <typename T, typename A, int TT>
__global__ void __launch_bounds__(256) wgrad_kernel(int kind, const int32_t* __restrict__ map, const int32_t* __restrict__ n_out,
                                                    int cap, int cin, int cout, int n_chunks,
                                                    const T* __restrict__ x, const T* __restrict__ g,
                                                    A* __restrict__ part) {
    pdl_begin();
    constexpr int TILE = 16 * TT;
    __shared__ A sA[WK][TILE + 1];
    __shared__ A sB[WK][TILE + 1];
    __shared__ int sRow[256], sSrc[256];
    __shared__ int sw[33];
    const int taps = conv_taps(kind);
    const int tiles_co = (cout + TILE - 1) / TILE;
    const int ci0 = (blockIdx.x / tiles_co) * TILE, co0 = (blockIdx.x % tiles_co) * TILE;
    const int t = blockIdx.y, chunk = blockIdx.z;
    const int n = min(*n_out, cap);
    const int rpc = (n + n_chunks - 1) / n_chunks;
    const int rb = min(chunk * rpc, n), re = min(rb + rpc, n);
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    A acc[TT][TT];
#pragma unroll
    for (int i = 0; i < TT; ++i)
#pragma unroll
        for (int j = 0; j < TT; ++j) acc[i][j] = A(0);
    for (int w0 = rb; w0 < re; w0 += 256) {
        const int r = w0 + tid;
        const int src = r < re ? gather_row(kind, map, r, t) : -1;
        int nv;
        const int pos = block_exclusive_scan(src >= 0 ? 1 : 0, sw, &nv);
        if (src >= 0) {
            sRow[pos] = r;
            sSrc[pos] = src;
        }
        __syncthreads();
        for (int k0 = 0; k0 < nv; k0 += WK) {
            for (int e = tid; e < WK * TILE; e += 256) {
                const int k = e / TILE, c = e % TILE;
                const bool ok = k0 + k < nv;
                sA[k][c] = (ok && ci0 + c < cin) ? to_acc(x[(size_t)sSrc[k0 + k] * cin + ci0 + c]) : A(0);
                sB[k][c] = (ok && co0 + c < cout) ? to_acc(g[(size_t)sRow[k0 + k] * cout + co0 + c]) : A(0);
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < WK; ++k) {
                A a[TT], b[TT];
#pragma unroll
                for (int i = 0; i < TT; ++i) a[i] = sA[k][ty * TT + i];
#pragma unroll
                for (int j = 0; j < TT; ++j) b[j] = sB[k][tx * TT + j];
#pragma unroll
                for (int i = 0; i < TT; ++i)
#pragma unroll
                    for (int j = 0; j < TT; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
            __syncthreads();
        }
    }
    A* out = part + ((size_t)chunk * taps + t) * cin * cout;
#pragma unroll
    for (int i = 0; i < TT; ++i) {
        const int ci = ci0 + ty * TT + i;
        if (ci >= cin) continue;
#pragma unroll
        for (int j = 0; j < TT; ++j) {
            const int co = co0 + tx * TT + j;
            if (co < cout) out[(size_t)ci * cout + co] = acc[i][j];
        }
    }
}

// dw[e] = sum over chunks of the weight partials; db[o] = sum over chunks of the bias partials.
template <typename A>
__global__ void __launch_bounds__(256) grad_reduce_kernel(const A* __restrict__ part_w, int n_chunks, long long nW,
                                                          const A* __restrict__ part_db, int n_db, int cout,
                                                          A* __restrict__ dw, A* __restrict__ db) {
    pdl_begin();
    const long long total = nW + (db ? cout : 0);
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        A s = 0;
        if (e < nW) {
            for (int c = 0; c < n_chunks; ++c) s += part_w[(size_t)c * nW + e];
            dw[e] = s;
        } else {
            const int o = (int)(e - nW);
            for (int c = 0; c < n_db; ++c) s += part_db[(size_t)c * cout + o];
            db[o] = s;
        }
    }
}

// wt[t][co][ci] = w[s][ci][co], s = t or taps - 1 - t (flip).
template <typename T>
__global__ void __launch_bounds__(256) transpose_taps_kernel(const T* __restrict__ w, int taps, int cin, int cout, int flip,
                                                             T* __restrict__ wt) {
    pdl_begin();
    const long long total = (long long)taps * cin * cout;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)(e % cin);
        const long long r = e / cin;
        const int co = (int)(r % cout), t = (int)(r / cout);
        const int s = flip ? taps - 1 - t : t;
        wt[e] = w[((size_t)s * cin + ci) * cout + co];
    }
}

int host_taps(int kind) { return conv_taps(kind); }

bool strided(int kind) {
    return kind == NPVS_CONV_DOWN2 || kind == NPVS_CONV_UP2 || kind == NPVS_CONV_DOWN3 || kind == NPVS_CONV_UP3;
}

struct BwdPlan {
    int taps, n_db, n_chunks, tile, tiles;
    bool tc_wgrad;  // BF16: weight gradient on the tensor cores (wgrad_tc)
    size_t el, acc, g_bytes, db_bytes, w_bytes, wt_bytes, conv_bytes;
    npvs_conv_desc td;  // the transposed convolution (dgrad)
    int mode;           // weight transpose: 1 plain, 2 with reversed taps
};

BwdPlan plan_bwd(const npvs_conv_desc& d) {
    BwdPlan p;
    p.taps = host_taps(d.kind);
    p.el = d.dtype == NPVS_F64 ? 8 : (d.dtype == NPVS_BF16 ? 2 : 4);
    p.acc = d.dtype == NPVS_F64 ? 8 : 4;
    const int cap = std::max(d.cap_out, 1);
    p.n_db = std::min(ceil_div(cap, kMaskRows), 2 * kNumSMs);
    // 32-channel tiles when either side is narrow, 64 otherwise; about four CTAs per SM in total
    p.tile = std::min(d.cin, d.cout) <= 32 ? 32 : 64;
    p.tiles = ceil_div(d.cin, p.tile) * ceil_div(d.cout, p.tile);
    p.n_chunks = std::max(1, std::min(256, ceil_div(4LL * kNumSMs, (long long)p.tiles * p.taps)));
    p.n_chunks = std::min(p.n_chunks, std::max(1, ceil_div(cap, 64)));
    p.g_bytes = d.relu ? (size_t)cap * d.cout * p.el : 0;
    p.db_bytes = (size_t)p.n_db * d.cout * p.acc;
    p.tc_wgrad = wgrad_tc_supported(d);
    p.w_bytes = p.tc_wgrad ? wgrad_tc_bytes(d) : (size_t)p.n_chunks * p.taps * d.cin * d.cout * p.acc;

    npvs_conv_desc t = d;
    t.relu = 0;
    t.out_f32 = 0;
    t.cin = d.cout;
    t.cout = d.cin;
    t.n_out = d.n_in ? d.n_in : d.n_out;
    t.cap_out = d.cap_in > 0 ? d.cap_in : d.cap_out;
    t.n_in = d.n_out;
    t.cap_in = d.cap_out;
    t.tune_stages = t.tune_max_split = t.tune_lag = t.tune_gather = t.tune_gather_warps = t.tune_form = 0;
    if (d.kind == NPVS_CONV_SUBM3 && d.cin == d.cout && (d.tune_gather == 3 || d.tune_gather == 4)) {
        // the transposed submanifold conv has the forward's shape and neighbour map: keep its window gather
        t.tune_form = 1;
        t.tune_gather = d.tune_gather;
        t.tune_max_split = d.tune_max_split;
        t.tune_gather_warps = d.tune_gather_warps;
        t.tune_stages = d.tune_stages;
    }
    t.workspace = nullptr;
    t.workspace_bytes = 0;
    t.w_transposed = nullptr;
    t.kind = transposed_kind(d.kind, &p.mode);
    if (d.kind == NPVS_CONV_SUBM3) {
        t.map2 = nullptr;
    } else if (d.kind == NPVS_CONV_HEAD1) {
        t.map = nullptr;
        t.map2 = nullptr;
    } else {  // the strided pairs: the maps swap roles
        t.map = d.map2;
        t.map2 = d.map;
    }
    p.td = t;
    if (d.dtype == NPVS_BF16) {
        p.wt_bytes = npvs_packed_weight_bytes(t.kind, t.cin, t.cout);
        p.conv_bytes = npvs_conv_workspace_bytes(&t);
    } else {
        p.wt_bytes = (size_t)p.taps * d.cin * d.cout * p.el;
        p.conv_bytes = d.dtype == NPVS_F32 ? npvs_conv_workspace_bytes(&t) : 0;  // FP32 product tiles
    }
    return p;
}

template <typename T>
npvs_status run_dgrad(const npvs_conv_desc& d, BwdPlan& p, const void* w, const T* gg, void* dx, const void* dx_add,
                      Arena& ar, cudaStream_t st);

template <typename T>
npvs_status run_bwd(const npvs_conv_desc& d, BwdPlan& p, const void* x, const void* w, const void* y, const void* dy,
                    void* dx, const void* dx_add, void* dw, void* db, Arena& ar, cudaStream_t st) {
    using A = typename AccOf<T>::type;
    const int cap = d.cap_out;
    T* g = d.relu ? ar.take<T>((size_t)cap * d.cout) : nullptr;
    A* part_db = ar.take<A>((size_t)p.n_db * d.cout);
    const T* gg = d.relu ? g : (const T*)dy;
    if constexpr (std::is_same<T, __nv_bfloat16>::value) {
        if (p.tc_wgrad && d.cout <= 2048) {
            launch_k(grad_mask_bf16_kernel, p.n_db, 256, 0, st, (const T*)dy, (const T*)y, d.relu, d.n_out, cap, d.cout,
                     g, (float*)part_db);
            NPVS_TRY(check_launch("grad_mask_bf16_kernel"));
            Arena sub(ar.take<char>(p.w_bytes), p.w_bytes);
            NPVS_TRY(wgrad_tc(d, (const __nv_bfloat16*)x, gg, (float*)dw, sub, st));
            if (db) {
                launch_k(grad_db_reduce_kernel<A>, ceil_div(d.cout, 32), 256, 0, st, (const A*)part_db, p.n_db, d.cout,
                         (A*)db);
                NPVS_TRY(check_launch("grad_db_reduce_kernel"));
            }
            return run_dgrad<T>(d, p, w, gg, dx, dx_add, ar, st);
        }
    }
    launch_k(grad_mask_kernel<T, A>, p.n_db, 256, 0, st, (const T*)dy, (const T*)y, d.relu, d.n_out, cap, d.cout, g,
             part_db);
    NPVS_TRY(check_launch("grad_mask_kernel"));
    A* part_w = ar.take<A>((size_t)p.n_chunks * p.taps * d.cin * d.cout);
    dim3 wg(p.tiles, p.taps, p.n_chunks);
    if (p.tile == 32)
        launch_k(wgrad_kernel<T, A, 2>, wg, 256, 0, st, d.kind, d.map, d.n_out, cap, d.cin, d.cout, p.n_chunks,
                 (const T*)x, gg, part_w);
    else
        launch_k(wgrad_kernel<T, A, 4>, wg, 256, 0, st, d.kind, d.map, d.n_out, cap, d.cin, d.cout, p.n_chunks,
                 (const T*)x, gg, part_w);
    NPVS_TRY(check_launch("wgrad_kernel"));
    const long long nW = (long long)p.taps * d.cin * d.cout;
    const int rg = std::max(1, std::min(ceil_div(nW + d.cout, 256), kNumSMs * 8));
    launch_k(grad_reduce_kernel<A>, rg, 256, 0, st, (const A*)part_w, p.n_chunks, nW, (const A*)part_db, p.n_db, d.cout,
             (A*)dw, (A*)db);
    NPVS_TRY(check_launch("grad_reduce_kernel"));
    return run_dgrad<T>(d, p, w, gg, dx, dx_add, ar, st);
}

// dgrad: the transposed convolution of g
template <typename T>
npvs_status run_dgrad(const npvs_conv_desc& d, BwdPlan& p, const void* w, const T* gg, void* dx, const void* dx_add,
                      Arena& ar, cudaStream_t st) {
    if (!dx) return NPVS_OK;
    void* wt = ar.take<char>(p.wt_bytes);
    if (d.dtype == NPVS_BF16) {
        if (d.w_transposed) wt = const_cast<void*>(d.w_transposed);  // packed after the optimizer step
        else NPVS_TRY(pack_weights_mode(p.td.kind, p.td.cin, p.td.cout, (const float*)w, wt, p.mode, st));
        p.td.workspace = ar.take<char>(p.conv_bytes);
        p.td.workspace_bytes = p.conv_bytes;
    } else {
        const long long tot = (long long)p.taps * d.cin * d.cout;
        const int tg = std::max(1, std::min(ceil_div(tot, 256), kNumSMs * 8));
        launch_k(transpose_taps_kernel<T>, tg, 256, 0, st, (const T*)w, p.taps, d.cin, d.cout, p.mode == 2 ? 1 : 0,
                 (T*)wt);
        NPVS_TRY(check_launch("transpose_taps_kernel"));
        if (p.conv_bytes) {
            p.td.workspace = ar.take<char>(p.conv_bytes);
            p.td.workspace_bytes = p.conv_bytes;
        }
    }
    return npvs_sparse_conv_fwd(&p.td, gg, wt, nullptr, dx_add, dx, st);
}

size_t bwd_bytes(const BwdPlan& p) {
    return Arena::round(p.g_bytes) + Arena::round(p.db_bytes) + Arena::round(p.w_bytes) + Arena::round(p.wt_bytes) +
           Arena::round(p.conv_bytes) + 6 * 256;
}

}  // namespace
}  // namespace npvs

using namespace npvs;

extern "C" size_t npvs_conv_bwd_workspace_bytes(const npvs_conv_desc* desc) {
    if (!desc || !valid_conv_kind(desc->kind)) return 0;
    BwdPlan p = plan_bwd(*desc);
    return bwd_bytes(p);
}

extern "C" npvs_status npvs_sparse_conv_bwd(const npvs_conv_desc* desc, const void* x, const void* w, const void* y,
                                            const void* dy, void* dx, const void* dx_add, void* dw, void* db,
                                            void* workspace, size_t workspace_bytes, void* stream) {
    NPVS_REQUIRE(desc && x && w && dy && dw && desc->n_out, NPVS_ERR_INVALID_ARG, "npvs_sparse_conv_bwd: NULL argument");
    const npvs_conv_desc& d = *desc;
    NPVS_REQUIRE(valid_conv_kind(d.kind), NPVS_ERR_UNSUPPORTED, "npvs_sparse_conv_bwd: unknown kind");
    NPVS_REQUIRE(d.cin > 0 && d.cout > 0 && d.cap_out >= 0, NPVS_ERR_INVALID_ARG, "npvs_sparse_conv_bwd: bad sizes");
    NPVS_REQUIRE(d.kind == NPVS_CONV_HEAD1 || d.map, NPVS_ERR_INVALID_ARG, "npvs_sparse_conv_bwd: map is NULL");
    NPVS_REQUIRE(d.dtype != NPVS_BF16 || !bf16_narrow(d.cin, d.cout), NPVS_ERR_UNSUPPORTED,
                 "npvs_sparse_conv_bwd: BF16 needs cin and cout multiples of 8");
    NPVS_REQUIRE(!d.w_transposed || d.dtype == NPVS_BF16, NPVS_ERR_INVALID_ARG,
                 "npvs_sparse_conv_bwd: w_transposed is a BF16 image");
    NPVS_REQUIRE(!d.relu || y, NPVS_ERR_INVALID_ARG, "npvs_sparse_conv_bwd: a ReLU layer needs its output y");
    NPVS_REQUIRE(!(d.relu && d.out_f32), NPVS_ERR_UNSUPPORTED, "npvs_sparse_conv_bwd: ReLU with out_f32 is not supported");
    NPVS_REQUIRE(!dx || d.kind == NPVS_CONV_SUBM3 || d.kind == NPVS_CONV_HEAD1 || d.map2, NPVS_ERR_INVALID_ARG,
                 "npvs_sparse_conv_bwd: the dgrad of a stride-2 conv needs map2 (the other map of the level pair)");
    NPVS_REQUIRE(!dx || !strided(d.kind) || (d.n_in && d.cap_in > 0), NPVS_ERR_INVALID_ARG,
                 "npvs_sparse_conv_bwd: the dgrad of a stride-2 conv needs n_in and cap_in");
    BwdPlan p = plan_bwd(d);
    NPVS_REQUIRE(workspace && workspace_bytes >= bwd_bytes(p), NPVS_ERR_WORKSPACE,
                 "npvs_sparse_conv_bwd: workspace smaller than npvs_conv_bwd_workspace_bytes()");
    if (d.cap_out == 0) return NPVS_OK;
    cudaStream_t st = as_stream(stream);
    Arena ar(workspace, workspace_bytes);
    switch (d.dtype) {
        case NPVS_F32: return run_bwd<float>(d, p, x, w, y, dy, dx, dx_add, dw, db, ar, st);
        case NPVS_BF16: return run_bwd<__nv_bfloat16>(d, p, x, w, y, dy, dx, dx_add, dw, db, ar, st);
        case NPVS_F64: return run_bwd<double>(d, p, x, w, y, dy, dx, dx_add, dw, db, ar, st);
        default: return fail(NPVS_ERR_UNSUPPORTED, "npvs_sparse_conv_bwd: unknown dtype");
    }
}
