// a10, BF16 weight gradient on the tensor cores: dW_t = sum_j x[src_j]^T g[dst_j] over the pairs
// (dst_j = output row, src_j = the input row it reads through tap t) of each tap.
//
// Pair lists. For each tap the rows whose neighbour through that tap exists are compacted in row
// order (count per 256-row chunk, scan per tap, write), giving src / dst lists per tap. The order
// is fixed, so the sums below are deterministic.
//
// GEMM. For tap t, C[ci][co] = sum_j A[j][ci] B[j][co] with A = the gathered x rows and B = the
// gathered g rows: the reduction runs over the pairs, and both operands arrive exactly as stored
// (a row of x holds consecutive ci, a row of g consecutive co), i.e. MN-major. A k-block is 64
// pairs; each operand row (128 bytes of 64 channels) is written by cp.async into a 128-byte
// swizzle atom (8 pair-rows x 128 B), atoms of consecutive 8-row groups 1024 B apart (SBO) and
// atoms of consecutive 64-channel groups 8 KB apart (LBO); one MMA (M = 128 channels of x, N = the
// channel tile of g, K = 16 pairs) advances 2048 B. The accumulator lives in TMEM (two buffers);
// work units (tap, ci tile, co tile, k slice) are spread over a persistent grid; each unit writes
// its FP32 partial tile and a reduction adds the k slices in order.
//
// Warp roles: 4 producer warps (cp.async gathers), 4 epilogue warps (TMEM -> partial tiles), one
// MMA warp. Every wait is bounded; on expiry the kernel flags NPVS_ERR_TIMEOUT, issues nothing
// new, drains what is in flight and frees its TMEM.
#include <cstring>

#include "conv_tc.cuh"
#include "tc_ptx.cuh"

namespace npvs {
namespace {

constexpr int kPairChunk = 256;
constexpr int kPW = 4;                      // producer warps
constexpr int kWgThreads = 32 * (kPW + 5);  // + 4 epilogue warps + 1 MMA warp
constexpr int kLag = 2;

__global__ void __launch_bounds__(kPairChunk) pairs_count_kernel(int kind, const int32_t* __restrict__ map,
                                                                 const int32_t* __restrict__ n_out, int cap,
                                                                 int n_chunks, int* __restrict__ counts) {
    pdl_begin();
    const int n = min(*n_out, cap);
    const int t = blockIdx.y;
    const int nc = (n + kPairChunk - 1) / kPairChunk;
    for (int c = blockIdx.x; c < nc; c += gridDim.x) {
        const int r = c * kPairChunk + threadIdx.x;
        const bool v = r < n && gather_row(kind, map, r, t) >= 0;
        const int cnt = __syncthreads_count(v);
        if (threadIdx.x == 0) counts[(size_t)t * n_chunks + c] = cnt;
    }
}

// One CTA per tap: exclusive scan of the tap's chunk counts, and the tap's pair total.
__global__ void __launch_bounds__(1024) pairs_scan_kernel(const int32_t* __restrict__ n_out, int cap, int n_chunks,
                                                          int* __restrict__ counts, int* __restrict__ totals) {
    pdl_begin();
    __shared__ int sw[33];
    const int n = min(*n_out, cap);
    const int nc = (n + kPairChunk - 1) / kPairChunk;
    int* cnt = counts + (size_t)blockIdx.x * n_chunks;
    int carry = 0;
    for (int c0 = 0; c0 < nc; c0 += 1024) {
        const int c = c0 + threadIdx.x;
        const int v = c < nc ? cnt[c] : 0;
        int tot;
        const int ex = block_exclusive_scan(v, sw, &tot);
        if (c < nc) cnt[c] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

__global__ void __launch_bounds__(kPairChunk) pairs_write_kernel(int kind, const int32_t* __restrict__ map,
                                                                 const int32_t* __restrict__ n_out, int cap,
                                                                 int n_chunks, const int* __restrict__ offs,
                                                                 int32_t* __restrict__ src, int32_t* __restrict__ dst) {
    pdl_begin();
    __shared__ int sw[33];
    const int n = min(*n_out, cap);
    const int t = blockIdx.y;
    const int nc = (n + kPairChunk - 1) / kPairChunk;
    for (int c = blockIdx.x; c < nc; c += gridDim.x) {
        const int r = c * kPairChunk + threadIdx.x;
        const int s = r < n ? gather_row(kind, map, r, t) : -1;
        int tot;
        const int pos = offs[(size_t)t * n_chunks + c] + block_exclusive_scan(s >= 0 ? 1 : 0, sw, &tot);
        if (s >= 0) {
            src[(size_t)t * cap + pos] = s;
            dst[(size_t)t * cap + pos] = r;
        }
    }
}

struct WgParams {
    int taps, cin, cout, MT, NT, Ntile, ksplit, stages, cap, nbB;
    uint32_t acc_cols;
    const int* totals;
    const int32_t* src;
    const int32_t* dst;
    const __nv_bfloat16* x;
    const __nv_bfloat16* g;
    float* part;  // [units][128][Ntile]
    int32_t* status;
    long long wait_limit;  // bound of every mbarrier wait, SM cycles (npvs_set_wait_limit)
};

// Shared-memory descriptor of an MN-major operand in 128-byte swizzle atoms: LBO = bytes between
// 64-element MN groups, SBO = bytes between 8-row K groups.
__device__ __forceinline__ uint64_t make_sdesc_mn(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;  // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both MN-major.
__host__ __device__ constexpr uint32_t idesc_mn(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

struct Unit {
    int t, mt, nt, j0, j1, nkb;
};

__device__ __forceinline__ Unit decode_unit(const WgParams& p, int u) {
    Unit w;
    const int ks = u % p.ksplit;
    int r = u / p.ksplit;
    w.nt = r % p.NT;
    r /= p.NT;
    w.mt = r % p.MT;
    w.t = r / p.MT;
    const int cnt = min(p.totals[w.t], p.cap);
    const int kc = ((cnt + p.ksplit - 1) / p.ksplit + 63) & ~63;
    w.j0 = min(ks * kc, cnt);
    w.j1 = min(w.j0 + kc, cnt);
    w.nkb = (w.j1 - w.j0 + 63) / 64;
    return w;
}

constexpr uint32_t kAtom = 8192;  // one 64-channel group of a 64-row k-block

__global__ void __launch_bounds__(kWgThreads, 1) wgrad_tc_kernel(const WgParams p) {
    pdl_begin();
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int S = p.stages;
    const uint32_t a_bytes = 2 * kAtom, b_bytes = (uint32_t)p.nbB * kAtom;
    uint8_t* sA = smem;
    uint8_t* sB = smem + (size_t)S * a_bytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + (size_t)S * b_bytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 5);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + S);
    const uint32_t tfull0 = smem_u32(bars + 2 * S), tempty0 = smem_u32(bars + 2 * S + 2), mdone = smem_u32(bars + 2 * S + 4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int units = p.taps * p.MT * p.NT * p.ksplit;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full0 + 8 * s, kPW);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull0 + 8 * b, 1);
            mbar_init(tempty0 + 8 * b, 4);
        }
        mbar_init(mdone, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kPW + 4) {
        tmem_alloc(smem_u32(tmem_slot), 2 * p.acc_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < kPW) {
        // ---------------------------------------------------------------- producers
        // thread -> (pair row = tid & 63, operand = tid >> 6: 0 = x row (A), 1 = g row (B)); each
        // thread reads its row index once per k-block, prefetched one k-block ahead
        const int tid = threadIdx.x, row = tid & 63;
        const bool isA = tid < 64;
        uint32_t it = 0;
        bool stop = false;
        for (int u = blockIdx.x; u < units && !stop; u += gridDim.x) {
            const Unit w = decode_unit(p, u);
            if (w.nkb == 0) continue;
            const int ci0 = w.mt * 128, co0 = w.nt * p.Ntile;
            const int nc = isA ? min(16, (p.cin - ci0) >> 3) : (min(p.Ntile, p.cout - co0) >> 3);
            const int32_t* list = (isA ? p.src : p.dst) + (size_t)w.t * p.cap;
            const __nv_bfloat16* base = isA ? p.x + ci0 : p.g + co0;
            const int ld = isA ? p.cin : p.cout;
            int next = w.j0 + row < w.j1 ? list[w.j0 + row] : -1;
            for (int kb = 0; kb < w.nkb; ++kb, ++it) {
                const int cur = next;
                const int jn = w.j0 + (kb + 1) * 64 + row;
                next = (kb + 1 < w.nkb && jn < w.j1) ? list[jn] : -1;
                const int s = (int)(it % S);
                mbar_wait(empty0 + 8 * s, ((it / S) & 1) ^ 1, abort_flag, p.wait_limit);
                if (__any_sync(0xffffffffu, *abort_flag)) {
                    stop = true;
                    break;
                }
                uint8_t* st = isA ? sA + (size_t)s * a_bytes : sB + (size_t)s * b_bytes;
                const uint32_t roff = (uint32_t)(row >> 3) * 1024 + (uint32_t)(row & 7) * 128;
                const __nv_bfloat16* src = base + (size_t)(cur >= 0 ? cur : 0) * ld;
                for (int c = 0; c < nc; ++c) {
                    const uint32_t off = (uint32_t)(c >> 3) * kAtom + roff + ((uint32_t)((c & 7) ^ (row & 7)) << 4);
                    cp_async16(smem_u32(st + off), src + c * 8, cur >= 0 ? 16u : 0u);
                }
                cp_async_commit();
                if (it >= (uint32_t)kLag) {
                    cp_async_wait<kLag>();
                    fence_proxy_async();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(full0 + 8 * ((it - kLag) % S));
                }
            }
        }
        cp_async_wait<0>();
        fence_proxy_async();
        __syncwarp();
        if (lane == 0)
            for (uint32_t j = it >= (uint32_t)kLag ? it - kLag : 0; j < it; ++j) mbar_arrive(full0 + 8 * (j % S));
    } else if (warp < kPW + 4) {
        // ---------------------------------------------------------------- epilogue
        const int ew = warp - kPW, m = ew * 32 + lane;
        uint32_t tc = 0;
        for (int u = blockIdx.x; u < units; u += gridDim.x) {
            const Unit w = decode_unit(p, u);
            float* dst = p.part + ((size_t)u * 128 + m) * p.Ntile;
            if (w.nkb == 0) {
                for (int c = 0; c < p.Ntile; c += 4) *reinterpret_cast<float4*>(dst + c) = make_float4(0.f, 0.f, 0.f, 0.f);
                continue;
            }
            const uint32_t buf = tc & 1;
            mbar_wait(tfull0 + 8 * buf, (tc >> 1) & 1, abort_flag, p.wait_limit);
            if (__any_sync(0xffffffffu, *abort_flag)) break;
            tc_fence_after();
            const uint32_t taddr = tmem + buf * p.acc_cols + ((uint32_t)(ew * 32) << 16);
            for (int c0 = 0; c0 < p.Ntile; c0 += 16) {
                uint32_t v[16];
                tmem_ld16(taddr + (uint32_t)c0, v);
                tmem_ld_wait();
#pragma unroll
                for (int q = 0; q < 16; q += 4)
                    *reinterpret_cast<float4*>(dst + c0 + q) = make_float4(__uint_as_float(v[q]), __uint_as_float(v[q + 1]),
                                                                          __uint_as_float(v[q + 2]), __uint_as_float(v[q + 3]));
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty0 + 8 * buf);
            ++tc;
        }
    } else {
        // ---------------------------------------------------------------- MMA issue
        if (lane == 0) {
            const uint32_t idesc = idesc_mn(128, p.Ntile);
            uint32_t it = 0, tc = 0;
            bool stop = false;
            for (int u = blockIdx.x; u < units && !stop; u += gridDim.x) {
                const Unit w = decode_unit(p, u);
                if (w.nkb == 0) continue;
                const uint32_t buf = tc & 1;
                const uint32_t acc = tmem + buf * p.acc_cols;
                mbar_wait(tempty0 + 8 * buf, ((tc >> 1) & 1) ^ 1, abort_flag, p.wait_limit);
                if (*abort_flag) break;
                tc_fence_after();
                for (int kb = 0; kb < w.nkb; ++kb, ++it) {
                    const int s = (int)(it % S);
                    if (!mbar_wait_ok(full0 + 8 * s, (it / S) & 1, abort_flag, p.wait_limit)) {
                        stop = true;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sA + (size_t)s * a_bytes), b0 = smem_u32(sB + (size_t)s * b_bytes);
                    // descriptors advanced by adding the 2048-byte K steps (16 rows) to their address field
                    const uint64_t ad = make_sdesc_mn(a0, kAtom, 1024), bd = make_sdesc_mn(b0, kAtom, 1024);
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        tc_mma(acc, ad + 128 * k, bd + 128 * k, idesc, (kb > 0 || k > 0) ? 1u : 0u);
                    tc_commit(empty0 + 8 * s);
                }
                if (!stop) tc_commit(tfull0 + 8 * buf);
                ++tc;
            }
            tc_commit(mdone);
            mbar_wait(mdone, 0, abort_flag, p.wait_limit);
        }
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kPW + 4) {
        tc_fence_after();
        tmem_dealloc(tmem, 2 * p.acc_cols);
    }
    if (threadIdx.x == 0 && *abort_flag) raise_status(p.status, NPVS_ERR_TIMEOUT);
}

// dw[t][ci][co] = sum over the k slices (in order) of the partial tiles.
__global__ void __launch_bounds__(256) wgrad_tc_reduce_kernel(const float* __restrict__ part, int taps, int cin, int cout,
                                                              int MT, int NT, int Ntile, int ksplit, float* __restrict__ dw) {
    pdl_begin();
    const long long total = (long long)taps * cin * cout;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int co = (int)(e % cout);
        const long long r = e / cout;
        const int ci = (int)(r % cin), t = (int)(r / cin);
        const int mt = ci >> 7, nt = co / Ntile;
        const size_t u0 = ((size_t)(t * MT + mt) * NT + nt) * ksplit;
        const size_t in = (size_t)(ci & 127) * Ntile + (co - nt * Ntile);
        float s = 0.f;
        for (int k = 0; k < ksplit; ++k) s += part[(u0 + k) * 128 * Ntile + in];
        dw[e] = s;
    }
}

struct WgPlan {
    int taps, n_chunks, MT, NT, Ntile, ksplit, stages, nbB;
    uint32_t acc_cols;
    size_t smem;
};

WgPlan plan_wgrad(const npvs_conv_desc& d) {
    WgPlan w;
    w.taps = conv_taps(d.kind);
    w.n_chunks = std::max(1, ceil_div(std::max(d.cap_out, 1), kPairChunk));
    w.MT = ceil_div(d.cin, 128);
    w.Ntile = std::min(256, (d.cout + 15) / 16 * 16);
    w.NT = ceil_div(d.cout, w.Ntile);
    w.nbB = (w.Ntile + 63) / 64;
    // about one unit per SM: each CTA then streams one long k range (taps differ in length, so a
    // finer split would not balance better)
    const int base_units = w.taps * w.MT * w.NT;
    w.ksplit = std::max(1, std::min(64, kNumSMs / base_units));
    w.acc_cols = 32;
    while ((int)w.acc_cols < w.Ntile) w.acc_cols <<= 1;
    const size_t stage = 2 * kAtom + (size_t)w.nbB * kAtom;
    const size_t fixed = 1024 + 16 * 8 + 64;
    w.stages = (int)std::min<size_t>(8, (220 * 1024 - fixed) / stage);
    w.smem = fixed + (size_t)w.stages * stage + (2 * w.stages + 5) * 8 + 16;
    return w;
}

}  // namespace

bool wgrad_tc_supported(const npvs_conv_desc& d) {
    return d.dtype == NPVS_BF16 && d.cin % 8 == 0 && d.cout % 8 == 0 && d.cap_out > 0;
}

size_t wgrad_tc_bytes(const npvs_conv_desc& d) {
    const WgPlan w = plan_wgrad(d);
    const size_t lists = 2 * Arena::round((size_t)w.taps * std::max(d.cap_out, 1) * sizeof(int32_t));
    const size_t counts = Arena::round((size_t)w.taps * w.n_chunks * sizeof(int)) + Arena::round(w.taps * sizeof(int));
    const size_t part = Arena::round((size_t)w.taps * w.MT * w.NT * w.ksplit * 128 * w.Ntile * sizeof(float));
    return lists + counts + part + 4 * 256;
}

npvs_status wgrad_tc(const npvs_conv_desc& d, const __nv_bfloat16* x, const __nv_bfloat16* g, float* dw, Arena& ar,
                     cudaStream_t st) {
    const WgPlan w = plan_wgrad(d);
    int32_t* src = ar.take<int32_t>((size_t)w.taps * d.cap_out);
    int32_t* dst = ar.take<int32_t>((size_t)w.taps * d.cap_out);
    int* counts = ar.take<int>((size_t)w.taps * w.n_chunks);
    int* totals = ar.take<int>(w.taps);
    float* part = ar.take<float>((size_t)w.taps * w.MT * w.NT * w.ksplit * 128 * w.Ntile);
    NPVS_REQUIRE(src && dst && counts && totals && part, NPVS_ERR_WORKSPACE, "npvs_sparse_conv_bwd: workspace too small");
    const dim3 pg(std::min(w.n_chunks, 64), w.taps);
    launch_k(pairs_count_kernel, pg, kPairChunk, 0, st, (int)d.kind, d.map, d.n_out, d.cap_out, w.n_chunks, counts);
    NPVS_TRY(check_launch("pairs_count_kernel"));
    launch_k(pairs_scan_kernel, w.taps, 1024, 0, st, d.n_out, d.cap_out, w.n_chunks, counts, totals);
    NPVS_TRY(check_launch("pairs_scan_kernel"));
    launch_k(pairs_write_kernel, pg, kPairChunk, 0, st, (int)d.kind, d.map, d.n_out, d.cap_out, w.n_chunks,
             (const int*)counts, src, dst);
    NPVS_TRY(check_launch("pairs_write_kernel"));
    WgParams p;
    std::memset(&p, 0, sizeof(p));
    p.taps = w.taps;
    p.cin = d.cin;
    p.cout = d.cout;
    p.MT = w.MT;
    p.NT = w.NT;
    p.Ntile = w.Ntile;
    p.ksplit = w.ksplit;
    p.stages = w.stages;
    p.cap = d.cap_out;
    p.nbB = w.nbB;
    p.acc_cols = w.acc_cols;
    p.totals = totals;
    p.src = src;
    p.dst = dst;
    p.x = x;
    p.g = g;
    p.part = part;
    p.status = d.status;
    p.wait_limit = wait_limit_cycles();
    static std::atomic<unsigned long long> seen[kMaxDevices];
    NPVS_TRY(ensure_dynamic_smem((const void*)wgrad_tc_kernel, 227 * 1024, seen, "wgrad_tc_kernel"));
    const int units = w.taps * w.MT * w.NT * w.ksplit;
    launch_k(wgrad_tc_kernel, std::min(units, kNumSMs), kWgThreads, w.smem, st, p);
    NPVS_TRY(check_launch("wgrad_tc_kernel"));
    const long long tot = (long long)w.taps * d.cin * d.cout;
    launch_k(wgrad_tc_reduce_kernel, std::max(1, std::min(ceil_div(tot, 256), kNumSMs * 8)), 256, 0, st,
             (const float*)part, w.taps, d.cin, d.cout, w.MT, w.NT, w.Ntile, w.ksplit, dw);
    return check_launch("wgrad_tc_reduce_kernel");
}

}  // namespace npvs
