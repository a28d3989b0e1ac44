// a5/a6: sparse convolutions, SIMT FMA path (FP32 and FP64) and the npvs_sparse_conv_fwd entry.
//
// Output-stationary gather-GEMM (Sec. 2.3, masked dense definition): a CTA owns a 64-row x
// 64-column output tile and walks the taps t and input-channel blocks; for each it gathers the
// 64 input rows x[map(n, t)] (zeros where the neighbour is absent) and the weight block W_t into
// shared memory and accumulates a 4 x 4 register tile per thread. Taps with no neighbour in the
// whole tile are skipped. The epilogue adds bias, applies ReLU, adds the skip input and stores
// each output row exactly once.
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

}  // namespace
}  // namespace npvs

using namespace npvs;

extern "C" npvs_status npvs_sparse_conv_fwd(const npvs_conv_desc* dsc, const void* x, const void* w,
                                            const void* bias, const void* skip, void* y, void* stream) {
    NPVS_REQUIRE(dsc && x && w && y && dsc->n_out, NPVS_ERR_INVALID_ARG, "npvs_sparse_conv_fwd: NULL argument");
    NPVS_REQUIRE(dsc->kind >= NPVS_CONV_SUBM3 && dsc->kind <= NPVS_CONV_HEAD1, NPVS_ERR_UNSUPPORTED,
                 "npvs_sparse_conv_fwd: unknown kind");
    NPVS_REQUIRE(dsc->kind == NPVS_CONV_HEAD1 || dsc->map, NPVS_ERR_INVALID_ARG, "npvs_sparse_conv_fwd: map is NULL");
    NPVS_REQUIRE(dsc->cin > 0 && dsc->cout > 0 && dsc->cap_out >= 0, NPVS_ERR_INVALID_ARG,
                 "npvs_sparse_conv_fwd: bad sizes");
    cudaStream_t st = as_stream(stream);
    if (dsc->cap_out == 0) return NPVS_OK;
    if (dsc->dtype == NPVS_BF16) return conv_tc_fwd(*dsc, x, w, (const float*)bias, skip, y, st);
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
