// a5/a6: sparse convolutions, SIMT FMA path (FP32 and FP64; BF16 shapes that do not fit the tensor-core
// tiles) and the npvs_sparse_conv_fwd entry.
//
// FP32 (when the descriptor's workspace holds the product tiles): the product form, as on the
// tensor cores but in FP32 FMA: a dense GEMM T[n][j * cout + o] = sum_c x[n][c] W_j[c][o] over the
// input rows (128 x 128 tiles, 8 x 8 per thread, double-buffered shared memory, the weights read
// straight from the [taps][cin][cout] master), then y[m] = b + sum_t T[map(m, t)][t] over existing
// neighbours in fixed tap order (+ReLU, +skip); a 1 x 1 conv writes y from the GEMM directly.
// Otherwise (and for FP64): an output-stationary gather-GEMM (Sec. 2.3, masked dense definition):
// a CTA owns a 64-row x 64-column output tile and walks the taps t and input-channel blocks; for
// each it gathers the 64 input rows x[map(n, t)] (zeros where the neighbour is absent) and the
// weight block W_t into shared memory and accumulates a 4 x 4 register tile per thread. Taps with
// no neighbour in the whole tile are skipped. The epilogue adds bias, applies ReLU, adds the skip
// input and stores each output row exactly once.
#include <algorithm>

#include "common.cuh"
#include "conv_tc.cuh"

namespace npvs {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;

template <typename T>
__global__ void __launch_bounds__(256) conv_simt_kernel(npvs_conv_desc dsc, const T* __restrict__ x,
                                                        const T* __restrict__ w, const T* __restrict__ bias,
                                                        const T* __restrict__ skip, T* __restrict__ y) {
    pdl_begin();
    __shared__ T sA[BK][BM + 1];
    __shared__ T sB[BK][BN];
    __shared__ int sRow[BM];
    const int n_out = min(*dsc.n_out, dsc.cap_out);
    const int row0 = blockIdx.x * BM, col0 = blockIdx.y * BN;
    if (row0 >= n_out) return;
    const int tid = threadIdx.x, tx = tid % (BN / TN), ty = tid / (BN / TN);
    const int taps = conv_taps(dsc.kind), cin = dsc.cin, cout = dsc.cout;
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
    for (int t = 0; t < taps; ++t) {
        int any = 0;
        if (tid < BM) {
            int n = row0 + tid;
            int r = n < n_out ? gather_row(dsc.kind, dsc.map, n, t) : -1;
            sRow[tid] = r;
            any = r >= 0;
        }
        if (!__syncthreads_or(any)) continue;
        for (int c0 = 0; c0 < cin; c0 += BK) {
            // A: BM x BK gathered rows (transposed into sA[k][m])
            for (int e = tid; e < BM * BK; e += 256) {
                int m = e / BK, k = e % BK;
                int r = sRow[m];
                sA[k][m] = (r >= 0 && c0 + k < cin) ? x[(size_t)r * cin + c0 + k] : T(0);
            }
            // B: BK x BN block of W_t
            for (int e = tid; e < BK * BN; e += 256) {
                int k = e / BN, j = e % BN;
                sB[k][j] = (c0 + k < cin && col0 + j < cout) ? w[((size_t)t * cin + c0 + k) * cout + col0 + j] : T(0);
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < BK; ++k) {
                T a[TM], b[TN];
#pragma unroll
                for (int i = 0; i < TM; ++i) a[i] = sA[k][ty * TM + i];
#pragma unroll
                for (int j = 0; j < TN; ++j) b[j] = sB[k][tx * TN + j];
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        int n = row0 + ty * TM + i;
        if (n >= n_out) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            int o = col0 + tx * TN + j;
            if (o >= cout) continue;
            T v = acc[i][j] + (bias ? T(bias[o]) : T(0));
            if (dsc.relu) v = v > T(0) ? v : T(0);
            if (skip) v += skip[(size_t)n * cout + o];
            y[(size_t)n * cout + o] = v;
        }
    }
}

// FP32 GEMM C = A B with A = x [rows][K] (row-major, K % 8 == 0), B[k][n] = w[(n / cout) * K + k]
// [n % cout] (the master weights [J][K][cout], cout % 4 == 0), N = J * cout columns. direct == 0:
// C is stored to T [rows][N]; direct == 1 (J == 1): y = relu?(C + b) (+ skip) is stored.
constexpr int GM = 128, GN = 128, GK = 8;

__global__ void __launch_bounds__(256) gemm_f32_kernel(const float* __restrict__ A, const int32_t* __restrict__ n_rows_p,
                                                       int cap_rows, int K, const float* __restrict__ W, int cout, int N,
                                                       float* __restrict__ C, int direct, const float* __restrict__ bias,
                                                       int relu, const float* __restrict__ skip) {
    pdl_begin();
    __shared__ __align__(16) float sA[2][GK][GM];
    __shared__ __align__(16) float sB[2][GK][GN];
    const int rows = min(*n_rows_p, cap_rows);
    const int m0 = blockIdx.x * GM, n0 = blockIdx.y * GN;
    if (m0 >= rows) return;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    // global -> register loads of one k-block: A row tid/2, k (tid%2)*4; B k tid/32, column (tid%32)*4
    const int a_row = tid >> 1, a_k = (tid & 1) * 4;
    const int b_k = tid >> 5, b_n = (tid & 31) * 4;
    const bool a_ok = m0 + a_row < rows;
    const int bn = n0 + b_n;
    const bool b_ok = bn < N;
    const float* a_src = A + (size_t)(m0 + a_row) * K + a_k;
    const float* b_src = b_ok ? W + ((size_t)(bn / cout) * K) * cout + (bn % cout) : W;
    float4 ra, rb;
    auto load = [&](int k0) {
        ra = a_ok ? __ldg(reinterpret_cast<const float4*>(a_src + k0)) : make_float4(0.f, 0.f, 0.f, 0.f);
        rb = b_ok ? __ldg(reinterpret_cast<const float4*>(b_src + (size_t)(k0 + b_k) * cout))
                  : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    auto store = [&](int buf) {
        sA[buf][a_k + 0][a_row] = ra.x;
        sA[buf][a_k + 1][a_row] = ra.y;
        sA[buf][a_k + 2][a_row] = ra.z;
        sA[buf][a_k + 3][a_row] = ra.w;
        *reinterpret_cast<float4*>(&sB[buf][b_k][b_n]) = rb;
    };
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    load(0);
    store(0);
    __syncthreads();
    const int nk = K / GK;
    for (int kb = 0; kb < nk; ++kb) {
        const int buf = kb & 1;
        if (kb + 1 < nk) load((kb + 1) * GK);
#pragma unroll
        for (int k = 0; k < GK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4*>(&sA[buf][k][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&sA[buf][k][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&sB[buf][k][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&sB[buf][k][64 + tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (kb + 1 < nk) {
            store(buf ^ 1);
            __syncthreads();
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
        if (m >= rows) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int n = n0 + h * 64 + tx * 4;
            if (n >= N) continue;
            float4 v = make_float4(acc[i][4 * h], acc[i][4 * h + 1], acc[i][4 * h + 2], acc[i][4 * h + 3]);
            if (direct) {
                const float4 bb = bias ? *reinterpret_cast<const float4*>(bias + n) : make_float4(0.f, 0.f, 0.f, 0.f);
                v.x += bb.x;
                v.y += bb.y;
                v.z += bb.z;
                v.w += bb.w;
                if (relu) {
                    v.x = fmaxf(v.x, 0.f);
                    v.y = fmaxf(v.y, 0.f);
                    v.z = fmaxf(v.z, 0.f);
                    v.w = fmaxf(v.w, 0.f);
                }
                if (skip) {
                    const float4 sk = *reinterpret_cast<const float4*>(skip + (size_t)m * N + n);
                    v.x += sk.x;
                    v.y += sk.y;
                    v.z += sk.z;
                    v.w += sk.w;
                }
            }
            *reinterpret_cast<float4*>(C + (size_t)m * N + n) = v;
        }
    }
}

// y[m][o] = b[o] + sum_t T[map[m][t]][t * cout + o] over existing neighbours in tap order (taps == 0:
// the transposed conv, T[u >> 3][(u & 7) * cout + o] with u = map[m]), then ReLU and the skip input.
// One thread per (row, 4 channels).
__global__ void __launch_bounds__(256) reduce_f32_kernel(const float* __restrict__ T, int ldT,
                                                         const int32_t* __restrict__ map, int taps,
                                                         const int32_t* __restrict__ n_out_p, int cap_out, int cout,
                                                         const float* __restrict__ bias, int relu,
                                                         const float* __restrict__ skip, float* __restrict__ y) {
    pdl_begin();
    const int n_out = min(*n_out_p, cap_out);
    const uint32_t G = (uint32_t)cout >> 2;
    const uint32_t total = (uint32_t)n_out * G;  // < 2^31: checked by the launcher
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int m = (int)(e / G), o = (int)(e - (uint32_t)m * G) * 4;
        float4 acc = bias ? *reinterpret_cast<const float4*>(bias + o) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (taps == 0) {
            const int u = __ldg(map + m);
            if (u >= 0) {
                const float4 v = __ldcg(reinterpret_cast<const float4*>(T + (size_t)(u >> 3) * ldT + (u & 7) * cout + o));
                acc.x += v.x;
                acc.y += v.y;
                acc.z += v.z;
                acc.w += v.w;
            }
        } else {
            const int32_t* mp = map + (size_t)m * taps;
#pragma unroll 9
            for (int t = 0; t < taps; ++t) {
                const int n = __ldg(mp + t);
                if (n >= 0) {
                    const float4 v = __ldcg(reinterpret_cast<const float4*>(T + (size_t)n * ldT + t * cout + o));
                    acc.x += v.x;
                    acc.y += v.y;
                    acc.z += v.z;
                    acc.w += v.w;
                }
            }
        }
        if (relu) {
            acc.x = fmaxf(acc.x, 0.f);
            acc.y = fmaxf(acc.y, 0.f);
            acc.z = fmaxf(acc.z, 0.f);
            acc.w = fmaxf(acc.w, 0.f);
        }
        const size_t off = (size_t)m * cout + o;
        if (skip) {
            const float4 sk = *reinterpret_cast<const float4*>(skip + off);
            acc.x += sk.x;
            acc.y += sk.y;
            acc.z += sk.z;
            acc.w += sk.w;
        }
        *reinterpret_cast<float4*>(y + off) = acc;
    }
}

// BF16 convolutions whose channel counts do not fit the tensor-core tiles (cin or cout not a
// multiple of 8: the stem and the head of a network without interleave, d = 1, have one or two
// input channels and one logit per site). One thread per output element (row n, channel o; o
// fastest, so a warp shares the row's neighbour rows and reads a contiguous weight row), FP32
// accumulation over the taps in order and the input channels in order (eight at a time from a
// 16-byte load when cin % 8 == 0), then bias, ReLU, skip and one rounding to the output type.
__global__ void __launch_bounds__(256) conv_narrow_bf16_kernel(npvs_conv_desc dsc, const __nv_bfloat16* __restrict__ x,
                                                               const __nv_bfloat16* __restrict__ w,
                                                               const float* __restrict__ bias,
                                                               const __nv_bfloat16* __restrict__ skip, void* __restrict__ y,
                                                               int vec8) {
    pdl_begin();
    const int n_out = min(*dsc.n_out, dsc.cap_out);
    const int taps = conv_taps(dsc.kind), cin = dsc.cin, cout = dsc.cout;
    const long long total = (long long)n_out * cout;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(e / cout), o = (int)(e - (long long)n * cout);
        float acc = 0.0f;
        for (int t = 0; t < taps; ++t) {
            const int r = gather_row(dsc.kind, dsc.map, n, t);
            if (r < 0) continue;
            const __nv_bfloat16* xr = x + (size_t)r * cin;
            const __nv_bfloat16* wt = w + (size_t)t * cin * cout + o;
            if (vec8) {
                for (int k = 0; k < cin; k += 8) {
                    const uint4 q = __ldg(reinterpret_cast<const uint4*>(xr + k));
                    const __nv_bfloat16* xv = reinterpret_cast<const __nv_bfloat16*>(&q);
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        acc = fmaf(__bfloat162float(xv[j]), __bfloat162float(wt[(size_t)(k + j) * cout]), acc);
                }
            } else {
                for (int k = 0; k < cin; ++k)
                    acc = fmaf(__bfloat162float(xr[k]), __bfloat162float(wt[(size_t)k * cout]), acc);
            }
        }
        float v = acc + (bias ? bias[o] : 0.0f);
        if (dsc.relu) v = fmaxf(v, 0.0f);
        if (skip) v += __bfloat162float(skip[e]);
        if (dsc.out_f32)
            static_cast<float*>(y)[e] = v;
        else
            static_cast<__nv_bfloat16*>(y)[e] = __float2bfloat16_rn(v);
    }
}

// The same convolution for few input channels (cin <= 8) and 16..256 output channels (the stem of a
// network without interleave): one warp per output row. Lane t < taps fetches the row's neighbour
// index and that neighbour's cin inputs once (the loads of all taps in flight together); the taps
// are then walked in order, the index and inputs broadcast by shuffle, and lane l accumulates the
// output channels l, l + 32, ... against weights staged in shared memory as FP32, in the summation
// order of conv_narrow_bf16_kernel.
constexpr int kNarrowMaxCin = 8;
template <int NJ>
__global__ void __launch_bounds__(256) conv_narrow_rows_kernel(npvs_conv_desc dsc, const __nv_bfloat16* __restrict__ x,
                                                               const __nv_bfloat16* __restrict__ w,
                                                               const float* __restrict__ bias,
                                                               const __nv_bfloat16* __restrict__ skip, void* __restrict__ y) {
    extern __shared__ float s_w[];  // [taps][cin][cout]
    const int taps = conv_taps(dsc.kind), cin = dsc.cin, cout = dsc.cout;
    const int nw = taps * cin * cout;
    pdl_begin();  // the weights may come from a packing kernel just before
    for (int i = threadIdx.x; i < nw; i += blockDim.x) s_w[i] = __bfloat162float(w[i]);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int n_out = min(*dsc.n_out, dsc.cap_out);
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int n = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); n < n_out; n += warps) {
        int r = -1;
        float xk[kNarrowMaxCin];
#pragma unroll
        for (int k = 0; k < kNarrowMaxCin; ++k) xk[k] = 0.0f;
        if (lane < taps) {
            r = gather_row(dsc.kind, dsc.map, n, lane);
            if (r >= 0) {
#pragma unroll
                for (int k = 0; k < kNarrowMaxCin; ++k)
                    if (k < cin) xk[k] = __bfloat162float(x[(size_t)r * cin + k]);
            }
        }
        float acc[NJ];
#pragma unroll
        for (int j = 0; j < NJ; ++j) acc[j] = 0.0f;
        for (int t = 0; t < taps; ++t) {
            const int rt = __shfl_sync(0xffffffffu, r, t);
            if (rt < 0) continue;  // warp-uniform
#pragma unroll
            for (int k = 0; k < kNarrowMaxCin; ++k) {
                if (k >= cin) break;
                const float xv = __shfl_sync(0xffffffffu, xk[k], t);
                const float* wr = s_w + (t * cin + k) * cout;
#pragma unroll
                for (int j = 0; j < NJ; ++j) {
                    const int o = lane + 32 * j;
                    if (o < cout) acc[j] = fmaf(xv, wr[o], acc[j]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            const int o = lane + 32 * j;
            if (o >= cout) continue;
            const size_t e = (size_t)n * cout + o;
            float v = acc[j] + (bias ? bias[o] : 0.0f);
            if (dsc.relu) v = fmaxf(v, 0.0f);
            if (skip) v += __bfloat162float(skip[e]);
            if (dsc.out_f32)
                static_cast<float*>(y)[e] = v;
            else
                static_cast<__nv_bfloat16*>(y)[e] = __float2bfloat16_rn(v);
        }
    }
}

template <int NJ>
npvs_status launch_narrow_rows(const npvs_conv_desc& d, const void* x, const void* w, const float* bias,
                               const void* skip, void* y, size_t smem, cudaStream_t st) {
    const int grid = (int)std::max<long long>(1, std::min<long long>(ceil_div((long long)d.cap_out, 8), (long long)kNumSMs * 8));
    launch_k(conv_narrow_rows_kernel<NJ>, grid, 256, smem, st, d, (const __nv_bfloat16*)x, (const __nv_bfloat16*)w,
             bias, (const __nv_bfloat16*)skip, y);
    return check_launch("conv_narrow_rows_kernel");
}

npvs_status conv_narrow_bf16(const npvs_conv_desc& d, const void* x, const void* w, const float* bias,
                             const void* skip, void* y, cudaStream_t st) {
    const int taps = conv_taps(d.kind);
    const size_t smem = (size_t)taps * d.cin * d.cout * sizeof(float);
    if (d.cin <= kNarrowMaxCin && d.cout >= 16 && d.cout <= 256 && smem <= 48 * 1024) {
        if (d.cout <= 32) return launch_narrow_rows<1>(d, x, w, bias, skip, y, smem, st);
        if (d.cout <= 64) return launch_narrow_rows<2>(d, x, w, bias, skip, y, smem, st);
        if (d.cout <= 128) return launch_narrow_rows<4>(d, x, w, bias, skip, y, smem, st);
        return launch_narrow_rows<8>(d, x, w, bias, skip, y, smem, st);
    }
    const long long total = (long long)d.cap_out * d.cout;
    const int grid = (int)std::max<long long>(1, std::min<long long>(ceil_div(total, 256), (long long)kNumSMs * 16));
    const int vec8 = d.cin % 8 == 0 && (reinterpret_cast<uintptr_t>(x) & 15) == 0;
    launch_k(conv_narrow_bf16_kernel, grid, 256, 0, st, d, (const __nv_bfloat16*)x, (const __nv_bfloat16*)w, bias,
             (const __nv_bfloat16*)skip, y, vec8);
    return check_launch("conv_narrow_bf16_kernel");
}

// The FP32 product form of npvs_sparse_conv_fwd; NPVS_ERR_UNSUPPORTED when it does not apply.
npvs_status conv_f32_product(const npvs_conv_desc& d, const float* x, const float* w, const float* bias,
                             const float* skip, float* y, cudaStream_t st) {
    if (d.tune_form == 1 || d.cin % 8 != 0 || d.cout % 4 != 0) return NPVS_ERR_UNSUPPORTED;
    if (d.kind == NPVS_CONV_HEAD1) {  // one tap: y directly
        const int rows_cap = d.cap_out;
        dim3 grid(ceil_div(rows_cap, GM), ceil_div(d.cout, GN));
        launch_k(gemm_f32_kernel, grid, 256, 0, st, x, d.n_out, rows_cap, d.cin, w, d.cout, d.cout, y, 1, bias,
                 d.relu, skip);
        return check_launch("gemm_f32_kernel");
    }
    float* T = conv_product_tiles(d);
    if (T == nullptr || d.n_in == nullptr || d.cap_in <= 0) return NPVS_ERR_UNSUPPORTED;
    const long long work = (long long)d.cap_out * (d.cout / 4);
    if (work >= (1LL << 31)) return NPVS_ERR_UNSUPPORTED;  // the gather kernel handles any size
    const int J = map27(d.kind) ? 27 : 8;
    const int N = J * d.cout;
    dim3 grid(ceil_div(d.cap_in, GM), ceil_div(N, GN));
    launch_k(gemm_f32_kernel, grid, 256, 0, st, x, d.n_in, d.cap_in, d.cin, w, d.cout, N, T, 0, nullptr, 0, nullptr);
    NPVS_TRY(check_launch("gemm_f32_kernel"));
    const int taps = d.kind == NPVS_CONV_UP2 ? 0 : conv_taps(d.kind);
    const int rg = (int)std::max<long long>(1, std::min<long long>(ceil_div(work, 256), kNumSMs * 8));
    launch_k(reduce_f32_kernel, rg, 256, 0, st, T, N, d.map, taps, d.n_out, d.cap_out, d.cout, bias, d.relu, skip, y);
    return check_launch("reduce_f32_kernel");
}

}  // namespace
}  // namespace npvs

using namespace npvs;

extern "C" npvs_status npvs_sparse_conv_fwd(const npvs_conv_desc* dsc, const void* x, const void* w,
                                            const void* bias, const void* skip, void* y, void* stream) {
    NPVS_REQUIRE(dsc && x && w && y && dsc->n_out, NPVS_ERR_INVALID_ARG, "npvs_sparse_conv_fwd: NULL argument");
    NPVS_REQUIRE(valid_conv_kind(dsc->kind), NPVS_ERR_UNSUPPORTED, "npvs_sparse_conv_fwd: unknown kind");
    NPVS_REQUIRE(!(dsc->kind == NPVS_CONV_DOWN3 || dsc->kind == NPVS_CONV_UP3) || (dsc->n_in && dsc->cap_in > 0),
                 NPVS_ERR_INVALID_ARG, "npvs_sparse_conv_fwd: DOWN3 / UP3 need n_in and cap_in");
    NPVS_REQUIRE(dsc->kind == NPVS_CONV_HEAD1 || dsc->map, NPVS_ERR_INVALID_ARG, "npvs_sparse_conv_fwd: map is NULL");
    NPVS_REQUIRE(dsc->cin > 0 && dsc->cout > 0 && dsc->cap_out >= 0, NPVS_ERR_INVALID_ARG,
                 "npvs_sparse_conv_fwd: bad sizes");
    cudaStream_t st = as_stream(stream);
    if (dsc->cap_out == 0) return NPVS_OK;
    if (dsc->dtype == NPVS_BF16)
        return bf16_narrow(dsc->cin, dsc->cout) ? conv_narrow_bf16(*dsc, x, w, (const float*)bias, skip, y, st)
                                                : conv_tc_fwd(*dsc, x, w, (const float*)bias, skip, y, st);
    if (dsc->dtype == NPVS_F32) {
        const npvs_status s = conv_f32_product(*dsc, (const float*)x, (const float*)w, (const float*)bias,
                                               (const float*)skip, (float*)y, st);
        if (s != NPVS_ERR_UNSUPPORTED) return s;
    }
    dim3 grid(ceil_div(dsc->cap_out, BM), ceil_div(dsc->cout, BN));
    if (dsc->dtype == NPVS_F32) {
        launch_k(conv_simt_kernel<float>, grid, 256, 0, st, *dsc, (const float*)x, (const float*)w, (const float*)bias, (const float*)skip,
                                                      (float*)y);
    } else if (dsc->dtype == NPVS_F64) {
        launch_k(conv_simt_kernel<double>, grid, 256, 0, st, *dsc, (const double*)x, (const double*)w, (const double*)bias,
                                                       (const double*)skip, (double*)y);
    } else {
        return fail(NPVS_ERR_UNSUPPORTED, "npvs_sparse_conv_fwd: unknown dtype");
    }
    return check_launch("conv_simt_kernel");
}
