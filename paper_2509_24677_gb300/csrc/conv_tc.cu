// a5/a6: BF16 sparse convolution on the 5th-generation tensor cores (tcgen05, TMEM accumulators).
//
// Two formulations of y[p] = b + sum_t W_t^T x[p + delta_t] (Sec. 2.3, masked dense definition):
//  * product form (default for submanifold and strided convs): a dense GEMM over the input rows,
//    T[n][t * cout + o] = sum_c x[n][c] W_t[c][o], with A loaded as whole 128-row TMA tiles, then
//    a gather-reduce y[m] = b + sum_t T[map[m][t]][t] over existing neighbours only, in fixed tap
//    order (conv_reduce_kernel);
//  * gather form: an implicit GEMM whose 128-row output tile accumulates sum_t X_t W_t over k-blocks
//    of BKE flat (tap, channel) columns (BKE = 64, or 32 when cin = 32), gathering neighbour rows.
//   gather     when cin is a multiple of 32, warp 0 alone feeds the pipeline with the TMA engine:
//              per stage each lane issues one cp.async.bulk.tensor tile::gather4 that brings 4
//              neighbour rows x[map(n, t)] (absent neighbours are out-of-range rows, filled with
//              zeros) into the stage, swizzled by the tensor map (128B, or 64B for 64-byte rows),
//              and lane 0 adds the weight block with one cp.async.bulk from a pre-swizzled HBM
//              image; everything completes on the stage's transaction-count barrier. For cin of 8
//              or 16, warps 0-3 gather 16-byte chunks with cp.async instead.
//   warp 8     allocates TMEM and issues tcgen05.mma (M=128, N=BN, K=16, FP32 accumulate) from one
//              thread; tcgen05.commit releases stages and hands a finished tile over;
//   warps 4-7  epilogue: tcgen05.ld of their 32 TMEM lanes, bias, ReLU, skip add, store.
// The CTA is persistent over work units; stage and accumulator hand-offs use mbarriers and every
// wait is bounded in time (on expiry the kernel flags NPVS_ERR_TIMEOUT, issues nothing new,
// drains what is in flight, frees its TMEM and returns).
// The transposed stride-2 convolution (UP2) runs in scatter form: rows are coarse sites, the
// GEMM has 8 * cout columns (one block per child tap), and the epilogue stores block j to the
// child row given by the down map, so every output row is still written exactly once.
#include <cuda.h>
#include <cuda_bf16.h>

#include <climits>
#include <cstring>

#include "conv_tc.cuh"
#include "tc_ptx.cuh"

namespace npvs {

static inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

namespace {

// Warp roles: PW gather warps (4 or 8), then 4 epilogue warps (warp % 4 selects the TMEM lane
// quadrant they may read), then the MMA warp.
constexpr int threads_for(int PW) { return 32 * (PW + 5); }
constexpr int kBM = 128;
constexpr int kSplitSlots = kNumSMs;
constexpr uint32_t kOutTileBytes = 32 * 16 * 4;  // 32 rows x 16 FP32 columns (64-byte rows)
constexpr int kOutTilesPerWarp = 2;              // 32 columns per TMEM wait and bulk group
constexpr uint32_t kOutStageBytes = 4 * kOutTilesPerWarp * kOutTileBytes;

struct TcParams {
    int kind, cin, cout, relu, out_f32;
    int scatter;   // epilogue: GEMM column block j -> child row map2[n][j] (transposed stride-2 conv)
    int tout;      // epilogue: raw FP32 accumulators into T [rows][Ntot] (product form)
    int tout_split;  // product form: the k-blocks may be split (partials summed in chunk order)
    int tout_tma;    // product form: T leaves through staging tiles and TMA stores (Ntot % 16 == 0)
    int KB, Kflat, Ntot, Npad, BN, n_tiles, stages;
    int gmode;     // A operand: 0 cp.async gather, 1 TMA gather4, 2 TMA dense tile (rows m0..m0+127),
                   // 3 window gather (SUBM3: dense TMA windows of input rows, A built in shared memory)
    int win_rows;  // window gather: rows of one window (one window per dz plane)
    int ncb;       // window gather: channel blocks of x (cin / BKE)
    int G;         // k-blocks per pipeline stage (window gather: taps of one (dz, dy) row; else 1)
    int BKE, RB;   // k-block width (elements) and its row bytes
    int rows_x;    // rows of x (the out-of-range row used for absent neighbours)
    int taps;      // stride of the gather map (27, 8) or 0 when row n reads input row n
    uint32_t acc_cols;  // TMEM columns of one accumulator (two are allocated)
    const int32_t* map;
    const int32_t* map2;
    const int32_t* n_rows;
    int cap_rows;
    const __nv_bfloat16* x;
    const __nv_bfloat16* w;
    const float* bias;
    const __nv_bfloat16* skip;
    void* y;
    float* T;
    int32_t* status;
    int max_split;   // upper bound of the k-split factor
    float* part;     // split-K partial tiles [kSplitSlots][128][BN] (nullable: no split)
    int* counters;   // split-K arrival counters [4 * kSplitSlots], zero between launches
    long long wait_limit;  // bound of every mbarrier wait, SM cycles (npvs_set_wait_limit)
};

__device__ __forceinline__ void tma_gather4(uint32_t dst, const CUtensorMap* tm, int col, int r0, int r1, int r2,
                                            int r3, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(col), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(bar)
        : "memory");
}

// ---- the kernel -----------------------------------------------------------------------------

// Teardown of the gather warps in the modes where several warps issue copies that complete on one
// stage barrier (TMA gather4, window gather). After a timeout the warps may have stopped at
// different iterations, so the drain must cover the last S stages of the furthest one: every
// warp publishes its iteration count, the gather warps meet at hardware named barrier 1 (each of
// them reaches it: their loops hold bounded waits only), and thread 0 waits for those stages. A
// stage that a stopped warp never armed completely gives up after kDrainCycles (~10 ms), long
// after any copy issued before the named barrier has landed. Without a timeout every warp ran
// the same iterations and this is the plain wait for the last S stages.
__device__ __forceinline__ void gather_teardown(uint32_t it, volatile int* warp_its, int PW, int warp, int lane,
                                                uint32_t full0, int S, volatile int* abort_flag, long long limit) {
    if (lane == 0) warp_its[warp] = (int)it;
    __syncwarp();
    asm volatile("bar.sync 1, %0;" ::"r"(PW * 32) : "memory");
    if (warp == 0 && lane == 0) {
        uint32_t hi = 0;
        for (int w = 0; w < PW; ++w) hi = max(hi, (uint32_t)warp_its[w]);
        for (uint32_t j = hi >= (uint32_t)S ? hi - S : 0; j < hi; ++j)
            mbar_wait(full0 + 8 * (j % S), (j / S) & 1, abort_flag, limit);
    }
    __syncwarp();
}

// Epilogue for 16 consecutive GEMM columns (from ng; bias of those columns in sb) of GEMM row n:
// bias, ReLU, skip, store.
__device__ __forceinline__ void store16(const TcParams& p, int n, int ng, const float* sb, const float (&acc)[16]) {
    int orow = n, o0 = ng;
    if (p.scatter) {
        const int j = ng / p.cout;
        if (j >= 8) return;
        orow = p.map2[(size_t)n * 8 + j];
        o0 = ng - j * p.cout;
        if (orow < 0) return;
    }
    const size_t base = (size_t)orow * p.cout + o0;
    const bool full16 = o0 + 16 <= p.cout;
    float sk[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) sk[q] = 0.0f;
    if (p.skip) {
        if (full16) {
            __align__(16) __nv_bfloat16 h[16];
            *reinterpret_cast<uint4*>(h) = *reinterpret_cast<const uint4*>(p.skip + base);
            *reinterpret_cast<uint4*>(h + 8) = *reinterpret_cast<const uint4*>(p.skip + base + 8);
#pragma unroll
            for (int q = 0; q < 16; ++q) sk[q] = __bfloat162float(h[q]);
        } else {
            for (int q = 0; q < 16 && o0 + q < p.cout; ++q) sk[q] = __bfloat162float(p.skip[base + q]);
        }
    }
    float f[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        float a = acc[q] + sb[q];
        if (p.relu) a = fmaxf(a, 0.0f);
        f[q] = a + sk[q];
    }
    if (p.out_f32) {
        float* yo = reinterpret_cast<float*>(p.y) + base;
        if (full16) {
#pragma unroll
            for (int q = 0; q < 16; q += 4) *reinterpret_cast<float4*>(yo + q) = make_float4(f[q], f[q + 1], f[q + 2], f[q + 3]);
        } else {
            for (int q = 0; q < 16 && o0 + q < p.cout; ++q) yo[q] = f[q];
        }
    } else {
        __nv_bfloat16* yo = reinterpret_cast<__nv_bfloat16*>(p.y) + base;
        if (full16) {
            __align__(16) __nv_bfloat16 h[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) h[q] = __float2bfloat16_rn(f[q]);
            *reinterpret_cast<uint4*>(yo) = *reinterpret_cast<uint4*>(h);
            *reinterpret_cast<uint4*>(yo + 8) = *reinterpret_cast<uint4*>(h + 8);
        } else {
            for (int q = 0; q < 16 && o0 + q < p.cout; ++q) yo[q] = __float2bfloat16_rn(f[q]);
        }
    }
}

// Window gather: one warp stages the A tile of tap t (one channel block) for the 128 rows of a
// tile. Row r (< rvalid) reads its neighbour map[r][t] from the window of t's dz plane (rows
// loj ...), or from global memory past the window end; absent neighbours and rows are zeros. The tile is written with the
// k-block's shared-memory swizzle, in batches of 8 chunks per lane (loads before stores).
template <int CH>
__device__ __forceinline__ void window_build_a(uint8_t* a_stage, const uint8_t* wj, const int* map_s, int t, int loj,
                                               int win_rows, int rvalid, const __nv_bfloat16* __restrict__ x, int cin,
                                               int col0, int lane) {
    constexpr int RB = CH * 16, PER = kBM * CH / 32, BATCH = 8;
#pragma unroll 1
    for (int q0 = 0; q0 < PER; q0 += BATCH) {
        uint4 v[BATCH];
        int nr[BATCH];
        bool far = false;
#pragma unroll
        for (int q = 0; q < BATCH; ++q) {  // window rows: every load in bounds, absent ones discarded
            const int r = (lane + 32 * (q0 + q)) / CH, c = lane % CH;
            const int n = r < rvalid ? map_s[r * 27 + t] : -1;
            const int w = n - loj;  // >= 0 for present neighbours: loj is the plane's smallest
            const bool in = n >= 0 && w < win_rows;
            far |= n >= 0 && w >= win_rows;
            const uint4 u = *reinterpret_cast<const uint4*>(wj + min(max(w, 0), win_rows - 1) * RB + c * 16);
            v[q] = in ? u : make_uint4(0u, 0u, 0u, 0u);
            nr[q] = (n >= 0 && !in) ? n : -1;
        }
        if (__any_sync(0xffffffffu, far)) {  // neighbours past the window end: from global memory
#pragma unroll
            for (int q = 0; q < BATCH; ++q)
                if (nr[q] >= 0) v[q] = __ldg(reinterpret_cast<const uint4*>(x + (size_t)nr[q] * cin + col0) + lane % CH);
        }
#pragma unroll
        for (int q = 0; q < BATCH; ++q) {
            const int r = (lane + 32 * (q0 + q)) / CH, c = lane % CH;
            *reinterpret_cast<uint4*>(a_stage + r * RB + ((c ^ (((r * RB) >> 7) & (CH - 1))) << 4)) = v[q];
        }
    }
}

// Work units: (row tile, column tile, k-chunk). Layers with few row tiles may split their k-blocks
// over up to gridDim.x CTAs; each writes an FP32 partial tile, and for every 32-row slice the last
// epilogue warp to finish (atomic counter) sums the partials in k-chunk order, so results do not
// depend on timing.
//
// Synchronisation: stage hand-offs use mbarriers (TMA modes: one expect_tx arrival and the copies'
// transaction bytes; cp.async mode: one arrival per gather warp once all its lanes' groups completed
// and were fenced to the async proxy, and a transaction barrier for the weight block); stage release
// and accumulator hand-over use tcgen05.commit. Two TMEM accumulators alternate between units so
// the epilogue of one unit overlaps the MMAs of the next. Below the CTA level only warp-local
// barriers are used and abort decisions are warp-uniform, so a timed-out wait never strands
// another warp. After a timeout nothing new is issued; teardown waits for the outstanding copies
// and MMAs before TMEM is freed.
template <int LAG, int PW>
__global__ void __launch_bounds__(threads_for(PW), 1)
    conv_tc_kernel(const TcParams p, const __grid_constant__ CUtensorMap tmap,
                   const __grid_constant__ CUtensorMap tmap_t) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int S = p.stages;
    // one stage holds G k-blocks: G A tiles of 128 rows and G B tiles of BN rows
    const uint32_t a_sub = (uint32_t)kBM * p.RB, b_sub = (uint32_t)p.BN * p.RB;
    const uint32_t a_bytes = p.G * a_sub, b_bytes = p.G * b_sub;
    const uint32_t win1 = p.gmode == 3 ? (uint32_t)p.win_rows * p.RB : 0u;  // bytes of one window
    uint8_t* sA = smem;
    uint8_t* sB = smem + (size_t)S * a_bytes;
    // product form: per epilogue warp four 32-row x 16-column FP32 staging tiles for the T stores
    float* s_out = reinterpret_cast<float*>(sB + (size_t)S * b_bytes);
    uint8_t* win = sB + (size_t)S * b_bytes + (p.tout_tma ? kOutStageBytes : 0u);  // window gather: 3 windows
    int* map_s = reinterpret_cast<int*>(win + 3 * (size_t)win1);
    float* s_bias = reinterpret_cast<float*>(map_s + kBM * p.taps + 4);  // [4 warps][256]
    uint64_t* bars = reinterpret_cast<uint64_t*>(s_bias + 4 * 256);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * S + 8);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile int* warp_its = reinterpret_cast<volatile int*>(tmem_slot + 4);  // [PW] gather teardown
    const uint32_t full0 = smem_u32(bars), bfull0 = smem_u32(bars + S), empty0 = smem_u32(bars + 2 * S);
    const uint32_t tfull0 = smem_u32(bars + 3 * S), tempty0 = smem_u32(bars + 3 * S + 2);
    const uint32_t mdone = smem_u32(bars + 3 * S + 4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // Set-up that reads nothing an earlier kernel writes runs before griddepcontrol.wait, so it
    // overlaps the tail of the previous kernel on the stream.
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            // TMA: one expect_tx; cp.async: one arrival per gather warp; window gather: one arrival
            // by the warp that built the stage (its weight bytes are expected on the same barrier)
            mbar_init(full0 + 8 * s, p.gmode == 0 ? PW : 1);
            mbar_init(bfull0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull0 + 8 * b, 1);
            mbar_init(tempty0 + 8 * b, 4);  // one arrival per epilogue warp
        }
        mbar_init(mdone, 1);
        mbar_init(mdone + 8, PW);  // window gather: gather-warp rendezvous
        mbar_init(mdone + 16, 1);  // window gather: windows landed (transaction bytes)
        mbar_init(mdone + 24, 1);  // window gather: the tile's neighbour map landed
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == PW + 4) {
        tmem_alloc(smem_u32(tmem_slot), 2 * p.acc_cols);
        tmem_relinquish();
    }
    pdl_begin();

    const int n_rows = min(*p.n_rows, p.cap_rows);
    const int tiles = ((n_rows + kBM - 1) / kBM) * p.n_tiles;
    int ksplit = 1, kbc = p.KB;
    // units = tiles x ksplit index the partial tiles and counters: at most kSplitSlots of them
    const int slots = min((int)gridDim.x, kSplitSlots);
    if (p.part != nullptr && (!p.tout || p.tout_split) && tiles > 0 && 2 * tiles <= slots && p.max_split > 1) {
        ksplit = min(min(p.KB, p.max_split), slots / tiles);
        kbc = (p.KB + ksplit - 1) / ksplit;
        ksplit = (p.KB + kbc - 1) / kbc;
    }
    const int units = tiles * ksplit;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if ((int)blockIdx.x >= units) {
        // no work: straight to the teardown (TMEM was allocated above)
    } else     if (warp < PW && p.gmode == 2) {
        // ------------------------------------------------------------------ TMA dense A tile
        if (warp == 0) {
            uint32_t it = 0;
            bool stop = false;
            for (int u = blockIdx.x; u < units && !stop; u += gridDim.x) {
                const int tile = u / ksplit, kc = u - tile * ksplit;
                const int mt = tile / p.n_tiles, nt = tile - mt * p.n_tiles;
                const int kb0 = kc * kbc, kb1 = min(p.KB, kb0 + kbc);
                for (int kb = kb0; kb < kb1; ++kb, ++it) {
                    const int s = (int)(it % S);
                    mbar_wait(empty0 + 8 * s, ((it / S) & 1) ^ 1, abort_flag, p.wait_limit);
                    if (__any_sync(0xffffffffu, *abort_flag)) {
                        stop = true;
                        break;
                    }
                    if (lane == 0) {  // the stage's G k-blocks: weight blocks and 128-row tiles of x
                        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(full0 + 8 * s),
                                     "r"(a_bytes + b_bytes)
                                     : "memory");
                        for (int g = 0; g < p.G; ++g) {
                            const int kbb = kb * p.G + g;
                            const __nv_bfloat16* wsrc = p.w + ((size_t)kbb * p.Npad + (size_t)nt * p.BN) * p.BKE;
                            bulk_g2s(smem_u32(sB + (size_t)s * b_bytes + g * b_sub), wsrc, b_sub, full0 + 8 * s);
                            tma_tile2d(smem_u32(sA + (size_t)s * a_bytes + g * a_sub), &tmap, kbb * p.BKE, mt * kBM,
                                       full0 + 8 * s);
                        }
                    }
                    __syncwarp();
                }
            }
            if (lane == 0)  // nothing the TMA engine writes may still be landing when the CTA leaves
                for (uint32_t j = it >= (uint32_t)S ? it - S : 0; j < it; ++j)
                    mbar_wait(full0 + 8 * (j % S), (j / S) & 1, abort_flag, p.wait_limit);
            __syncwarp();
        }
    } else if (warp < PW && p.gmode == 1) {
        // ------------------------------------------------------------------ TMA gather
        // the 32 row quads of a tile are spread over the gather warps (32 / PW lanes each); a lane
        // stages its quad's neighbour-map rows (lane-private) and issues its gather4 each stage
        constexpr int QPW = 32 / PW;
        const bool act = lane < QPW;
        const int q4 = warp * QPW + (act ? lane : 0);
        uint32_t it = 0;
        bool stop = false;
        for (int u = blockIdx.x; u < units && !stop; u += gridDim.x) {
            const int tile = u / ksplit, kc = u - tile * ksplit;
            const int mt = tile / p.n_tiles, nt = tile - mt * p.n_tiles;
            const int m0 = mt * kBM;
            const int kb0 = kc * kbc, kb1 = min(p.KB, kb0 + kbc);
            if (p.taps && act) {
                for (int rr = 0; rr < 4; ++rr) {
                    const int r = 4 * q4 + rr;
                    const bool ok = m0 + r < n_rows;
                    const int32_t* src = p.map + (size_t)(m0 + r) * p.taps;
                    for (int t = 0; t < p.taps; ++t) map_s[r * p.taps + t] = ok ? src[t] : -1;
                }
            }
            for (int kb = kb0; kb < kb1; ++kb, ++it) {
                const int s = (int)(it % S);
                mbar_wait(empty0 + 8 * s, ((it / S) & 1) ^ 1, abort_flag, p.wait_limit);
                if (__any_sync(0xffffffffu, *abort_flag)) {
                    stop = true;
                    break;
                }
                if (warp == 0 && lane == 0) {
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(full0 + 8 * s),
                                 "r"(a_bytes + b_bytes)
                                 : "memory");
                    const __nv_bfloat16* wsrc = p.w + ((size_t)kb * p.Npad + (size_t)nt * p.BN) * p.BKE;
                    bulk_g2s(smem_u32(sB + (size_t)s * b_bytes), wsrc, b_bytes, full0 + 8 * s);
                }
                const int t = p.taps ? (kb * p.BKE) / p.cin : 0;
                const int ci = kb * p.BKE - t * p.cin;
                int rows[4];
#pragma unroll
                for (int rr = 0; rr < 4; ++rr) {
                    const int r = 4 * q4 + rr, n = m0 + r;
                    int src = -1;
                    if (n < n_rows) src = p.taps ? map_s[r * p.taps + t] : n;
                    rows[rr] = src >= 0 ? src : p.rows_x;
                }
                if (act)
                    tma_gather4(smem_u32(sA + (size_t)s * a_bytes + 4 * q4 * p.RB), &tmap, ci, rows[0], rows[1],
                                rows[2], rows[3], full0 + 8 * s);
            }
        }
        // nothing the TMA engine writes may still be landing when the CTA leaves
        gather_teardown(it, warp_its, PW, warp, lane, full0, S, abort_flag, p.wait_limit);
    } else if (warp < PW && p.gmode == 3) {
        // ------------------------------------------------------------------ window gather (SUBM3)
        // Rows are in linear site order, so the neighbours of a 128-row tile through the 9 taps of
        // one dz plane lie in a short run of input rows starting at the smallest of them. Per
        // channel block the three runs (windows of win_rows rows) come in as dense TMA tiles; each
        // k-block (tap t, channel block cb) then builds its A stage row by row from the window of
        // t's plane (a neighbour past the window end is read from global memory), so no row is
        // fetched from global memory once per tap. Gather warps meet at an mbarrier (bounded waits).
        const int tid = threadIdx.x;
        const uint32_t rdv = mdone + 8, wfull = mdone + 16, mfull = mdone + 24;
        const int NB = min(PW, S);  // warps that build stages
        const int TPS = 27 / p.G;   // stages per channel block (G taps of one (dz, dy) row per stage)
        uint32_t rdv_ph = 0, wf_ph = 0, mf_ph = 0, it = 0;
        int s_it = 0, own_it = 0;   // stage (it % S) and builder warp (it % NB) of iteration it
        uint32_t ph_it = 0;         // phase parity of iteration it on its stage ((it / S) & 1)
        bool stop = false;
        auto rendezvous = [&]() {
            __syncwarp();
            if (lane == 0) mbar_arrive(rdv);
            mbar_wait(rdv, rdv_ph & 1, abort_flag, p.wait_limit);
            ++rdv_ph;
            return __any_sync(0xffffffffu, *abort_flag) != 0;
        };
        for (int u = blockIdx.x; u < units && !stop; u += gridDim.x) {
            const int tile = u / ksplit, kc = u - tile * ksplit;
            const int mt = tile / p.n_tiles, nt = tile - mt * p.n_tiles;
            const int m0 = mt * kBM;
            const int kb0 = kc * kbc, kb1 = min(p.KB, kb0 + kbc);
            if (u != (int)blockIdx.x) {
                fence_proxy_async();
                if (rendezvous()) break;  // the previous unit's map, bounds and windows are no longer read
            }
            if (tid == 0) {
                // the tile's neighbour-map rows (contiguous) in one bulk copy; the copy size must be a
                // multiple of 16 bytes (4 rows), the last < 4 rows of the map come by plain loads
                const int rows = min(kBM, p.cap_rows - m0), rows4 = rows & ~3;
                for (int e = rows4 * 27; e < rows * 27; ++e) map_s[e] = __ldg(p.map + (size_t)m0 * 27 + e);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mfull),
                             "r"((uint32_t)rows4 * 108u)
                             : "memory");
                if (rows4 > 0) bulk_g2s(smem_u32(map_s), p.map + (size_t)m0 * 27, (uint32_t)rows4 * 108u, mfull);
            }
            mbar_wait(mfull, mf_ph & 1, abort_flag, p.wait_limit);
            ++mf_ph;
            const int rvalid = n_rows - m0;  // rows of the tile that exist (map rows past it are stale)
            // every warp finds the window starts (smallest neighbour row per dz plane) of the whole tile
            int mn0 = INT_MAX, mn1 = INT_MAX, mn2 = INT_MAX;
            for (int r = lane; r < min(rvalid, kBM); r += 32) {
                const int* mr = map_s + r * 27;
#pragma unroll
                for (int t = 0; t < 27; ++t) {
                    const int v = mr[t];
                    const int vv = v >= 0 ? v : INT_MAX;
                    if (t < 9) mn0 = min(mn0, vv);
                    else if (t < 18) mn1 = min(mn1, vv);
                    else mn2 = min(mn2, vv);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                mn0 = min(mn0, __shfl_xor_sync(0xffffffffu, mn0, o));
                mn1 = min(mn1, __shfl_xor_sync(0xffffffffu, mn1, o));
                mn2 = min(mn2, __shfl_xor_sync(0xffffffffu, mn2, o));
            }
            const int lo[3] = {mn0, mn1, mn2};
            int cur = -1;
            for (int kb = kb0; kb < kb1; ++kb, ++it) {
                const int s = s_it, own = own_it;
                const uint32_t ph = ph_it;
                if (++s_it == S) {
                    s_it = 0;
                    ph_it ^= 1u;
                }
                if (++own_it == NB) own_it = 0;
                const int cb = kb / TPS, t = (kb - cb * TPS) * p.G;  // first tap of the stage
                if (cb != cur) {
                    if (cur >= 0) {
                        fence_proxy_async();
                        if (rendezvous()) {  // every warp is done with the current windows
                            stop = true;
                            break;
                        }
                    }
                    if (tid == 0) {
                        // planes whose taps this unit runs in channel block cb (a k-split unit may hold a few taps)
                        const int t_lo = (max(kb0, cb * TPS) - cb * TPS) * p.G;
                        const int t_hi = (min(kb1, cb * TPS + TPS) - cb * TPS) * p.G - 1;
                        bool need[3];
                        uint32_t bytes = 0;
                        for (int j = 0; j < 3; ++j) {
                            need[j] = lo[j] != INT_MAX && 9 * j <= t_hi && 9 * j + 8 >= t_lo;
                            bytes += need[j] ? win1 : 0u;
                        }
                        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(wfull), "r"(bytes)
                                     : "memory");
                        for (int j = 0; j < 3; ++j)
                            if (need[j]) tma_tile2d(smem_u32(win + j * win1), &tmap, cb * p.BKE, lo[j], wfull);
                    }
                    mbar_wait(wfull, wf_ph & 1, abort_flag, p.wait_limit);
                    ++wf_ph;
                    if (__any_sync(0xffffffffu, *abort_flag)) {
                        stop = true;
                        break;
                    }
                    cur = cb;
                }
                // stage `it` is built by warp it % NB alone, so the warps' wait / build / publish chains
                // overlap. NB <= S keeps every wait within one phase of its barrier: the warp's
                // previous stage (it - NB) waited for the release of it - NB - S >= it - 2S.
                if (own != warp) continue;
                mbar_wait(empty0 + 8 * s, ph ^ 1u, abort_flag, p.wait_limit);
                if (__any_sync(0xffffffffu, *abort_flag)) {
                    stop = true;
                    break;
                }
                if (lane == 0) {  // the stage's weight blocks land on its own barrier
                    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(full0 + 8 * s),
                                 "r"(b_bytes)
                                 : "memory");
                    for (int g = 0; g < p.G; ++g) {
                        const __nv_bfloat16* wsrc =
                            p.w + ((size_t)((t + g) * p.ncb + cb) * p.Npad + (size_t)nt * p.BN) * p.BKE;
                        bulk_g2s(smem_u32(sB + (size_t)s * b_bytes + g * b_sub), wsrc, b_sub, full0 + 8 * s);
                    }
                }
                // the stage's taps share dz (and dy): one window
                const int j = t / 9, loj = j == 0 ? lo[0] : (j == 1 ? lo[1] : lo[2]);
                const uint8_t* wj = win + j * win1;
                uint8_t* a_stage = sA + (size_t)s * a_bytes;
                for (int g = 0; g < p.G; ++g) {
                    if (p.RB == 128)
                        window_build_a<8>(a_stage + g * a_sub, wj, map_s, t + g, loj, p.win_rows, rvalid, p.x, p.cin,
                                          cb * p.BKE, lane);
                    else
                        window_build_a<4>(a_stage + g * a_sub, wj, map_s, t + g, loj, p.win_rows, rvalid, p.x, p.cin,
                                          cb * p.BKE, lane);
                }
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) mbar_arrive(full0 + 8 * s);
            }
        }
        if (tid == 0) {  // nothing the TMA engine writes may still be landing when the CTA leaves
            if (wf_ph > 0) mbar_wait(wfull, (wf_ph - 1) & 1, abort_flag, p.wait_limit);
            if (mf_ph > 0) mbar_wait(mfull, (mf_ph - 1) & 1, abort_flag, p.wait_limit);
        }
        gather_teardown(it, warp_its, PW, warp, lane, full0, S, abort_flag, p.wait_limit);
    } else if (warp < PW) {
        // ------------------------------------------------------------------ cp.async gather
        // thread (warp w, lane): 16-byte chunk c = lane & 7 of rows r0 + 4 PW q, r0 = 4 w + lane / 8
        constexpr int RSTEP = 4 * PW, NQ = kBM / RSTEP;
        const int tid = threadIdx.x, c = tid & 7, r0 = tid >> 3;
        uint32_t it = 0;
        bool stop = false;
        for (int u = blockIdx.x; u < units && !stop; u += gridDim.x) {
            const int tile = u / ksplit, kc = u - tile * ksplit;
            const int mt = tile / p.n_tiles, nt = tile - mt * p.n_tiles;
            const int m0 = mt * kBM;
            const int kb0 = kc * kbc, kb1 = min(p.KB, kb0 + kbc);
            if (p.taps) {  // this warp's rows of the neighbour map, once per unit
                __syncwarp();
                for (int e = lane; e < 4 * NQ * p.taps; e += 32) {
                    const int j = e / p.taps, t = e - j * p.taps;
                    const int r = 4 * warp + (j & 3) + RSTEP * (j >> 2);
                    map_s[r * p.taps + t] = (m0 + r < n_rows) ? p.map[(size_t)(m0 + r) * p.taps + t] : -1;
                }
                __syncwarp();
            }
            for (int kb = kb0; kb < kb1; ++kb, ++it) {
                const int s = (int)(it % S);
                mbar_wait(empty0 + 8 * s, ((it / S) & 1) ^ 1, abort_flag, p.wait_limit);
                if (__any_sync(0xffffffffu, *abort_flag)) {
                    stop = true;
                    break;
                }
                if (tid == 0) {
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bfull0 + 8 * s),
                                 "r"(b_bytes)
                                 : "memory");
                    const __nv_bfloat16* wsrc = p.w + ((size_t)kb * p.Npad + (size_t)nt * p.BN) * p.BKE;
                    bulk_g2s(smem_u32(sB + (size_t)s * b_bytes), wsrc, b_bytes, bfull0 + 8 * s);
                }
                const int k = kb * 64 + c * 8;
                const bool kvalid = k < p.Kflat;
                const int t = p.taps ? k / p.cin : 0;
                const int ci = k - t * p.cin;
                uint8_t* a_stage = sA + (size_t)s * a_bytes;
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const int r = r0 + RSTEP * q, n = m0 + r;
                    int src_row = -1;
                    if (kvalid && n < n_rows) src_row = p.taps ? map_s[r * p.taps + t] : n;
                    const void* src = src_row >= 0 ? (const void*)(p.x + (size_t)src_row * p.cin + ci) : (const void*)p.x;
                    cp_async16(smem_u32(a_stage + r * 128 + ((c ^ (r & 7)) << 4)), src, src_row >= 0 ? 16u : 0u);
                }
                cp_async_commit();
                if (it >= (uint32_t)LAG) {
                    cp_async_wait<LAG>();
                    fence_proxy_async();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(full0 + 8 * ((it - LAG) % S));
                }
            }
        }
        cp_async_wait<0>();
        fence_proxy_async();
        __syncwarp();
        if (!stop && lane == 0)
            for (uint32_t j = it >= (uint32_t)LAG ? it - LAG : 0; j < it; ++j) mbar_arrive(full0 + 8 * (j % S));
        if (tid == 0)  // no weight copy may still be landing when the CTA leaves
            for (uint32_t j = it >= (uint32_t)S ? it - S : 0; j < it; ++j)
                mbar_wait(bfull0 + 8 * (j % S), (j / S) & 1, abort_flag, p.wait_limit);
    } else if (warp < PW + 4) {
        // ------------------------------------------------------------------ epilogue
        const int ew = warp - PW, r = ew * 32 + lane;
        float* wb = s_bias + ew * 256;
        uint32_t tc = 0;
        for (int u = blockIdx.x; u < units; u += gridDim.x, ++tc) {
            const int tile = u / ksplit;
            const int mt = tile / p.n_tiles, nt = tile - mt * p.n_tiles;
            const int n = mt * kBM + r;
            const uint32_t buf = tc & 1;
            const uint32_t taddr_row = tmem + buf * p.acc_cols + ((uint32_t)(ew * 32) << 16);
            if (!p.tout) {
                __syncwarp();
                for (int c2 = lane; c2 < p.BN; c2 += 32) {
                    const int col = nt * p.BN + c2;
                    const int o = p.scatter ? col % p.cout : col;
                    wb[c2] = (p.bias && o < p.cout && col < p.Ntot) ? p.bias[o] : 0.0f;
                }
                __syncwarp();
            }
            mbar_wait(tfull0 + 8 * buf, (tc >> 1) & 1, abort_flag, p.wait_limit);
            if (__any_sync(0xffffffffu, *abort_flag)) break;
            tc_fence_after();
            if (p.tout && ksplit == 1 && !p.tout_tma) {  // rows of 16 columns by plain stores
                for (int c0 = 0; c0 < p.BN; c0 += 16) {
                    uint32_t v[16];
                    tmem_ld16(taddr_row + (uint32_t)c0, v);
                    tmem_ld_wait();
                    const int ng = nt * p.BN + c0;
                    if (n >= n_rows || ng >= p.Ntot) continue;
                    float* dst = p.T + (size_t)n * p.Ntot + ng;
                    if (ng + 16 <= p.Ntot) {
#pragma unroll
                        for (int q = 0; q < 16; q += 4)
                            *reinterpret_cast<float4*>(dst + q) =
                                make_float4(__uint_as_float(v[q]), __uint_as_float(v[q + 1]),
                                            __uint_as_float(v[q + 2]), __uint_as_float(v[q + 3]));
                    } else {
                        for (int q = 0; q < 16 && ng + q < p.Ntot; ++q) dst[q] = __uint_as_float(v[q]);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(tempty0 + 8 * buf);
            } else if (p.tout && ksplit == 1) {
                // Per 64 columns the warp loads its 32 accumulator rows with up to four TMEM loads and
                // one wait; each 16-column chunk goes to a staging tile in the 64-byte swizzle (row r's
                // 16-byte chunk c at position c ^ ((r >> 1) & 3)) and leaves with one TMA tensor store
                // of 32 full 64-byte row segments (lane 0 issues the group and waits for the previous
                // group to have read its tiles before they are rewritten). Rows past n_rows (up to the
                // tile end) carry values of rows nothing reads; rows past T's capacity are clipped by
                // the tensor map.
                const int row0 = mt * kBM + ew * 32;
                float* grp = s_out + ew * (kOutTilesPerWarp * kOutTileBytes / 4);
                for (int c0 = 0; c0 < p.BN; c0 += 16 * kOutTilesPerWarp) {
                    const int nch = min(kOutTilesPerWarp, (p.BN - c0) >> 4);  // warp-uniform
                    uint32_t v[kOutTilesPerWarp][16];
#pragma unroll
                    for (int q = 0; q < kOutTilesPerWarp; ++q)
                        if (q < nch) tmem_ld16(taddr_row + (uint32_t)(c0 + 16 * q), v[q]);
                    tmem_ld_wait();
                    const int ng0 = nt * p.BN + c0;
                    if (row0 >= n_rows || ng0 >= p.Ntot) continue;  // warp-uniform
                    const int nst = min(nch, (p.Ntot - ng0) >> 4);   // chunks inside T (Ntot % 16 == 0)
                    if (lane == 0) bulk_wait_read0();  // the last group has read its tiles
                    __syncwarp();
#pragma unroll
                    for (int q = 0; q < kOutTilesPerWarp; ++q) {
                        if (q >= nst) break;
                        float* tile = grp + q * (kOutTileBytes / 4);
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            *reinterpret_cast<float4*>(tile + lane * 16 + ((c ^ ((lane >> 1) & 3)) << 2)) =
                                make_float4(__uint_as_float(v[q][4 * c]), __uint_as_float(v[q][4 * c + 1]),
                                            __uint_as_float(v[q][4 * c + 2]), __uint_as_float(v[q][4 * c + 3]));
                    }
                    fence_proxy_async_shared();
                    __syncwarp();
                    if (lane == 0) {
                        for (int q = 0; q < nst; ++q)
                            tma_store_2d(&tmap_t, ng0 + 16 * q, row0, smem_u32(grp + q * (kOutTileBytes / 4)));
                        bulk_commit();
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(tempty0 + 8 * buf);
            } else if (ksplit == 1) {
                for (int c0 = 0; c0 < p.BN; c0 += 16) {
                    uint32_t v[16];
                    tmem_ld16(taddr_row + (uint32_t)c0, v);
                    tmem_ld_wait();
                    if (n >= n_rows) continue;
                    float acc[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) acc[q] = __uint_as_float(v[q]);
                    store16(p, n, nt * p.BN + c0, wb + c0, acc);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(tempty0 + 8 * buf);
            } else {
                float* part = p.part + ((size_t)u * kBM + r) * p.BN;
                for (int c0 = 0; c0 < p.BN; c0 += 16) {
                    uint32_t v[16];
                    tmem_ld16(taddr_row + (uint32_t)c0, v);
                    tmem_ld_wait();
#pragma unroll
                    for (int q = 0; q < 16; q += 4)
                        __stcg(reinterpret_cast<float4*>(part + c0 + q),
                               make_float4(__uint_as_float(v[q]), __uint_as_float(v[q + 1]), __uint_as_float(v[q + 2]),
                                           __uint_as_float(v[q + 3])));
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(tempty0 + 8 * buf);  // the accumulator is free again
                __threadfence();
                __syncwarp();
                int last = 0;
                if (lane == 0) last = atomicAdd(p.counters + tile * 4 + ew, 1) == ksplit - 1;
                last = __shfl_sync(0xffffffffu, last, 0);
                if (last) {
                    __threadfence();
                    if (n < n_rows) {
                        const float* base = p.part + ((size_t)(tile * ksplit) * kBM + r) * p.BN;
                        for (int c0 = 0; c0 < p.BN; c0 += 16) {
                            float acc[16];
#pragma unroll
                            for (int q = 0; q < 16; ++q) acc[q] = 0.0f;
                            for (int k2 = 0; k2 < ksplit; ++k2) {
                                const float* src = base + (size_t)k2 * kBM * p.BN + c0;
#pragma unroll
                                for (int q = 0; q < 16; q += 4) {
                                    float4 v4 = __ldcg(reinterpret_cast<const float4*>(src + q));
                                    acc[q] += v4.x;
                                    acc[q + 1] += v4.y;
                                    acc[q + 2] += v4.z;
                                    acc[q + 3] += v4.w;
                                }
                            }
                            if (p.tout) {  // the summed product tile into T, no epilogue
                                const int ng = nt * p.BN + c0;
                                if (ng >= p.Ntot) continue;
                                float* dst = p.T + (size_t)n * p.Ntot + ng;
                                if (ng + 16 <= p.Ntot) {
#pragma unroll
                                    for (int q = 0; q < 16; q += 4)
                                        *reinterpret_cast<float4*>(dst + q) =
                                            make_float4(acc[q], acc[q + 1], acc[q + 2], acc[q + 3]);
                                } else {
                                    for (int q = 0; q < 16 && ng + q < p.Ntot; ++q) dst[q] = acc[q];
                                }
                            } else {
                                store16(p, n, nt * p.BN + c0, wb + c0, acc);
                            }
                        }
                    }
                    if (lane == 0) p.counters[tile * 4 + ew] = 0;
                }
            }
        }
        if (p.tout_tma && lane == 0) {  // the T stores have read their tiles and landed (also after a timeout)
            bulk_wait_all();
            fence_proxy_async_global();
        }
        __syncwarp();
    } else {
        if (lane == 0) {
            // -------------------------------------------------------------- MMA issuer
            const uint32_t idesc = make_idesc(kBM, p.BN);
            const int kk_steps = p.BKE / 16;  // MMAs (K = 16) per k-block
            const uint32_t sA_u32 = smem_u32(sA), sB_u32 = smem_u32(sB);
            uint32_t tc = 0;
            int s = 0;          // stage of the next k-block
            uint32_t ph = 0;    // its phase parity
            bool stop = false;
            for (int u = blockIdx.x; u < units && !stop; u += gridDim.x, ++tc) {
                const int kc = u - (u / ksplit) * ksplit;
                const int kb0 = kc * kbc, kb1 = min(p.KB, kb0 + kbc);
                const uint32_t buf = tc & 1;
                const uint32_t acc = tmem + buf * p.acc_cols;
                mbar_wait(tempty0 + 8 * buf, ((tc >> 1) & 1) ^ 1, abort_flag, p.wait_limit);
                if (*abort_flag) break;
                tc_fence_after();
                for (int kb = kb0; kb < kb1; ++kb) {
                    // this thread issues every MMA of the CTA: the loop is kept short (one probe of a
                    // completed stage, descriptors advanced by adding the 32-byte K steps to their
                    // address field), else issuing would take longer than the MMAs of a k-block
                    if (!mbar_wait_ok(full0 + 8 * s, ph, abort_flag, p.wait_limit) ||
                        (p.gmode == 0 && !mbar_wait_ok(bfull0 + 8 * s, ph, abort_flag, p.wait_limit))) {
                        stop = true;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t ad = make_sdesc(sA_u32 + (uint32_t)s * a_bytes, p.RB);
                    const uint64_t bd = make_sdesc(sB_u32 + (uint32_t)s * b_bytes, p.RB);
                    for (int g = 0; g < p.G; ++g)
                        for (int k = 0; k < kk_steps; ++k)
                            tc_mma(acc, ad + ((g * a_sub + 32 * k) >> 4), bd + ((g * b_sub + 32 * k) >> 4), idesc,
                                   (kb > kb0 || g > 0 || k > 0) ? 1u : 0u);
                    tc_commit(empty0 + 8 * s);
                    if (++s == S) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (!stop) tc_commit(tfull0 + 8 * buf);
            }
            // every MMA this CTA issued has completed before TMEM is released
            tc_commit(mdone);
            mbar_wait(mdone, 0, abort_flag, p.wait_limit);
        }
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == PW + 4) {
        tc_fence_after();
        tmem_dealloc(tmem, 2 * p.acc_cols);
    }
    if (threadIdx.x == 0 && *abort_flag) raise_status(p.status, NPVS_ERR_TIMEOUT);
}

// y[m][o] = b[o] + sum_t T[map[m][t]][t * cout + o] (taps in fixed order), then ReLU and skip.
// taps == 0: the transposed conv, y[m][o] = b[o] + T[u >> 3][(u & 7) * cout + o] with u = map[m] the
// up map (parent row * 8 + child tap). One thread per (row, 4 channels); only existing neighbours
// are read.
template <typename OutT>
__global__ void __launch_bounds__(256) conv_reduce_kernel(const float* __restrict__ T, int ldT,
                                                          const int32_t* __restrict__ map, int taps,
                                                          const int32_t* __restrict__ n_out_p, int cap_out, int cout,
                                                          const float* __restrict__ bias, int relu,
                                                          const __nv_bfloat16* __restrict__ skip, OutT* __restrict__ y) {
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
            // every neighbour index first, then every product row, then the sums in tap order (one
            // memory round trip each instead of one per batch of taps); taps <= 27
            const int32_t* mp = map + (size_t)m * taps;
            int nb[27];
#pragma unroll
            for (int t = 0; t < 27; ++t) nb[t] = t < taps ? __ldg(mp + t) : -1;
            float4 v[27];
#pragma unroll
            for (int t = 0; t < 27; ++t)
                v[t] = nb[t] >= 0 ? __ldcg(reinterpret_cast<const float4*>(T + (size_t)nb[t] * ldT + t * cout + o))
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int t = 0; t < 27; ++t)
                if (nb[t] >= 0) {
                    acc.x += v[t].x;
                    acc.y += v[t].y;
                    acc.z += v[t].z;
                    acc.w += v[t].w;
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
            __align__(8) __nv_bfloat16 h[4];
            *reinterpret_cast<uint2*>(h) = *reinterpret_cast<const uint2*>(skip + off);
            acc.x += __bfloat162float(h[0]);
            acc.y += __bfloat162float(h[1]);
            acc.z += __bfloat162float(h[2]);
            acc.w += __bfloat162float(h[3]);
        }
        if constexpr (sizeof(OutT) == 4) {
            *reinterpret_cast<float4*>(y + off) = acc;
        } else {
            __align__(8) __nv_bfloat16 h[4] = {__float2bfloat16_rn(acc.x), __float2bfloat16_rn(acc.y),
                                                __float2bfloat16_rn(acc.z), __float2bfloat16_rn(acc.w)};
            *reinterpret_cast<uint2*>(y + off) = *reinterpret_cast<uint2*>(h);
        }
    }
}

// Packed weights: per k-block a [Npad][BKE] BF16 tile, K-major, each row's 16-byte chunks permuted
// exactly as the 128-byte (BKE = 64) or 64-byte (BKE = 32) shared-memory swizzle places them, so a
// stage is one linear bulk copy. Column-block forms (the transposed conv and the product form)
// have n = j * cout + o and k = ci; the direct forms have n = o and k = t * cin + ci.
// Weight W_t[ci][co] of the convolution being packed. mode 0: w is [taps][cin][cout]. mode 1 / 2:
// the convolution is the transpose of a stored one, w is the stored [taps][cout][cin] and
// W_t[ci][co] = w_s[co][ci] with s = t (mode 1) or s = taps - 1 - t (mode 2: the tap of the
// opposite offset, for the transpose of a submanifold convolution).
__device__ __forceinline__ float weight_at(const float* __restrict__ w, int mode, int taps, int cin, int cout, int t,
                                           int ci, int co) {
    if (mode == 0) return w[((size_t)t * cin + ci) * cout + co];
    const int s = mode == 2 ? taps - 1 - t : t;
    return w[((size_t)s * cout + co) * cin + ci];
}

// One element e of the image of a (kind, cin, cout) convolution in form sh (plain = 1: the plain
// [taps][cin][cout] BF16 image of the SIMT-path convolutions, e indexes it directly).
struct PackImage {
    TcShape sh;
    const float* w;
    __nv_bfloat16* out;
    int kind, cin, cout, mode, plain;
    long long begin;  // first element of this image in the launch's element range
    long long size;   // its elements
};

__device__ __forceinline__ void pack_element(const PackImage& im, long long e) {
    if (im.plain) {
        im.out[e] = __float2bfloat16_rn(im.w[e]);
        return;
    }
    const TcShape& sh = im.sh;
    const int taps = conv_taps(im.kind);
    const int nchunk = sh.BKE / 8;
    const int kk = (int)(e % sh.BKE);
    const long long rest = e / sh.BKE;
    const int n = (int)(rest % sh.Npad), kb = (int)(rest / sh.Npad);
    const int k = kb * sh.BKE + kk;
    float v = 0.0f;
    if (k < sh.Kflat && n < sh.Ntot) {
        if (sh.J > 1) {  // column blocks: n = j * cout + o, k = ci
            const int j = n / im.cout, o = n - j * im.cout;
            v = weight_at(im.w, im.mode, taps, im.cin, im.cout, j, k, o);
        } else {         // n = o, k = t * cin + ci
            const int t = k / im.cin, ci = k - t * im.cin;
            v = weight_at(im.w, im.mode, taps, im.cin, im.cout, t, ci, n);
        }
    }
    const int sw = ((n * sh.RB) >> 7) & (nchunk - 1);
    const size_t dst = ((size_t)kb * sh.Npad + n) * sh.BKE + ((((kk >> 3) ^ sw) << 3) | (kk & 7));
    im.out[dst] = __float2bfloat16_rn(v);
}

constexpr int kMaxPackImages = 48;

struct PackBatch {
    PackImage im[kMaxPackImages];
    int n;
    long long total;
};

// Every image of the batch in one grid-stride loop over the concatenated element ranges.
__global__ void __launch_bounds__(256) pack_images_kernel(const __grid_constant__ PackBatch b) {
    pdl_begin();
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < b.total;
         e += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = b.n - 1;  // the last image that begins at or before e
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (b.im[mid].begin <= e) lo = mid;
            else hi = mid - 1;
        }
        pack_element(b.im[lo], e - b.im[lo].begin);
    }
}

int conv_taps_host(int kind) { return conv_taps(kind); }

constexpr int kMaxStages = 12;
constexpr size_t kMaxSmem = 227 * 1024;

// win: bytes of the three windows of the window gather (0 otherwise); G: k-blocks per stage.
// out: the product form's T staging tiles (kOutStageBytes), else 0
size_t tc_smem_bytes(int BN, int RB, int taps, int S, size_t win = 0, int G = 1, size_t out = 0) {
    return 1024 + (size_t)S * G * (kBM + BN) * RB + out + win + (size_t)kBM * taps * 4 + 16 + 4 * 256 * 4 +
           (3 * S + 8) * 8 + 16 + 8 * 3 * 4;
}

int tc_stages(int BN, int RB, int taps, size_t out = 0) {
    for (int S = kMaxStages; S > 4; --S)
        if (tc_smem_bytes(BN, RB, taps, S, 0, 1, out) <= kMaxSmem) return S;
    return 4;
}

// Window gather with G taps per stage: the longest window (256, 192 or 128 rows) that leaves room
// for at least three stages (two with shorter windows); 0 when not even that fits.
int win_rows_for(int BN, int RB, int G, int* stages) {
    for (int wr = 256; wr >= 128; wr -= 64) {
        const size_t win = 3 * (size_t)wr * RB;
        for (int S = kMaxStages; S >= (wr == 256 ? 3 : 2); --S)
            if (tc_smem_bytes(BN, RB, 27, S, win, G) <= kMaxSmem) {
                *stages = S;
                return wr;
            }
    }
    return 0;
}

template <int LAG, int PW>
npvs_status launch_tc(const TcParams& p, const CUtensorMap& tm, const CUtensorMap& tm_t, int grid, size_t smem,
                      cudaStream_t st) {
    static std::atomic<unsigned long long> seen[kMaxDevices];
    NPVS_TRY(ensure_dynamic_smem((const void*)conv_tc_kernel<LAG, PW>, (int)kMaxSmem, seen, "conv_tc_kernel"));
    launch_k(conv_tc_kernel<LAG, PW>, grid, threads_for(PW), smem, st, p, tm, tm_t);
    return check_launch("conv_tc_kernel");
}

template <int PW>
npvs_status launch_tc_lag(int lag, const TcParams& p, const CUtensorMap& tm, const CUtensorMap& tm_t, int grid,
                          size_t smem, cudaStream_t st) {
    switch (lag) {
        case 1: return launch_tc<1, PW>(p, tm, tm_t, grid, smem, st);
        case 2: return launch_tc<2, PW>(p, tm, tm_t, grid, smem, st);
        case 3: return launch_tc<3, PW>(p, tm, tm_t, grid, smem, st);
        case 4: return launch_tc<4, PW>(p, tm, tm_t, grid, smem, st);
        case 6: return launch_tc<6, PW>(p, tm, tm_t, grid, smem, st);
        default: return fail(NPVS_ERR_INVALID_ARG, "npvs_sparse_conv_fwd: unsupported pipeline lag");
    }
}

// Bytes of one packed image (form 0: direct / transposed; form 1: product form).
size_t packed_image_bytes(int kind, int cin, int cout, int form) {
    TcShape sh = tc_shape(kind, cin, cout, form);
    return Arena::round((size_t)sh.KB * sh.Npad * sh.BKE * sizeof(__nv_bfloat16));
}

bool has_product_form(int kind) { return map27(kind) || kind == NPVS_CONV_DOWN2; }

size_t split_region_bytes() {
    return Arena::round(4 * kSplitSlots * sizeof(int)) + Arena::round((size_t)kSplitSlots * kBM * 256 * sizeof(float));
}

size_t product_region_bytes(const npvs_conv_desc& d) {
    if (!has_product_form(d.kind) && d.kind != NPVS_CONV_UP2) return 0;
    if (d.dtype == NPVS_BF16 && bf16_narrow(d.cin, d.cout)) return 0;
    const int J = map27(d.kind) ? 27 : 8;
    const int rows = d.cap_in > 0 ? d.cap_in : d.cap_out;
    return Arena::round((size_t)rows * J * d.cout * sizeof(float));
}

// One tcgen05 GEMM launch.
npvs_status run_gemm(TcParams& p, const TcShape& sh, const npvs_conv_desc& d, const void* x, int lag, cudaStream_t st) {
    p.KB = sh.KB;
    p.Kflat = sh.Kflat;
    p.Ntot = sh.Ntot;
    p.Npad = sh.Npad;
    p.BN = sh.BN;
    p.n_tiles = sh.n_tiles;
    p.BKE = sh.BKE;
    p.RB = sh.RB;
    size_t win = 0;
    p.G = 1;
    if (p.gmode == 3) {
        p.G = d.tune_gather == 4 ? 3 : 1;
        p.win_rows = win_rows_for(sh.BN, sh.RB, p.G, &p.stages);
        if (p.win_rows == 0 && p.G > 1) {  // three taps per stage do not fit: one
            p.G = 1;
            p.win_rows = win_rows_for(sh.BN, sh.RB, p.G, &p.stages);
        }
        NPVS_REQUIRE(p.win_rows > 0, NPVS_ERR_UNSUPPORTED, "BF16 conv: window gather does not fit this shape");
        p.ncb = d.cin / sh.BKE;
        p.KB = 27 / p.G * p.ncb;  // pipeline stages of one tile
        win = 3 * (size_t)p.win_rows * sh.RB;
    } else {
        p.stages = tc_stages(sh.BN, sh.RB, p.taps, p.tout_tma ? kOutStageBytes : 0);
        // dense 128-row tiles: two k-blocks per stage halve the stage hand-offs (each costs a few
        // hundred cycles of the single MMA-issuing thread), with as many stages as fit (at least 2)
        if (p.gmode == 2 && sh.KB % 2 == 0 && sh.KB >= 4) {
            int S2 = 0;
            for (int S = kMaxStages; S >= 2 && S2 == 0; --S)
                if (tc_smem_bytes(sh.BN, sh.RB, p.taps, S, 0, 2, p.tout_tma ? kOutStageBytes : 0) <= kMaxSmem) S2 = S;
            if (S2 >= 2) {
                p.G = 2;
                p.KB = sh.KB / 2;  // pipeline stages of one tile
                p.stages = S2;
            }
        }
    }
    if (d.tune_stages >= (p.gmode == 3 || p.G > 1 ? 2 : 3) && d.tune_stages < p.stages) p.stages = d.tune_stages;
    lag = std::min(lag, p.stages - 1);
    if (lag == 5) lag = 4;  // instantiated lags: 1, 2, 3, 4, 6 (all < stages)
    p.acc_cols = 32;
    while ((int)p.acc_cols < sh.BN) p.acc_cols <<= 1;
    if (p.cap_rows <= 0) return NPVS_OK;
    const size_t smem = tc_smem_bytes(sh.BN, sh.RB, p.taps, p.stages, win, p.G, p.tout_tma ? kOutStageBytes : 0);
    alignas(64) CUtensorMap tm;
    std::memset(&tm, 0, sizeof(tm));
    alignas(64) CUtensorMap tm_t;  // product form: T [cap_rows][Ntot] FP32, 16 x 32 boxes, 64-byte swizzle
    std::memset(&tm_t, 0, sizeof(tm_t));
    if (p.tout_tma) {
        EncodeTiledFn enc = encode_tiled();
        NPVS_REQUIRE(enc != nullptr, NPVS_ERR_CUDA, "BF16 conv: cuTensorMapEncodeTiled unavailable");
        const cuuint64_t gdim[2] = {(cuuint64_t)p.Ntot, (cuuint64_t)p.cap_rows};
        const cuuint64_t gstride[1] = {(cuuint64_t)p.Ntot * 4};
        const cuuint32_t box[2] = {16, 32};
        const cuuint32_t estride[2] = {1, 1};
        CUresult r = enc(&tm_t, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, p.T, gdim, gstride, box, estride,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        NPVS_REQUIRE(r == CUDA_SUCCESS, NPVS_ERR_CUDA, "BF16 conv: product-tile tensor map encoding failed");
    }
    if (p.gmode != 0) {
        EncodeTiledFn enc = encode_tiled();
        NPVS_REQUIRE(enc != nullptr, NPVS_ERR_CUDA, "BF16 conv: cuTensorMapEncodeTiled unavailable");
        const cuuint64_t gdim[2] = {(cuuint64_t)d.cin, (cuuint64_t)p.rows_x};
        const cuuint64_t gstride[1] = {(cuuint64_t)d.cin * 2};
        const cuuint32_t box_rows = p.gmode == 2 ? (cuuint32_t)kBM : (p.gmode == 3 ? (cuuint32_t)p.win_rows : 1u);
        const cuuint32_t box[2] = {(cuuint32_t)sh.BKE, box_rows};
        const cuuint32_t estride[2] = {1, 1};
        // windows are read row by row from shared memory: unswizzled
        const CUtensorMapSwizzle swz = p.gmode == 3 ? CU_TENSOR_MAP_SWIZZLE_NONE
                                                    : (sh.RB == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B);
        CUresult r = enc(&tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(x), gdim, gstride, box, estride,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            set_error("BF16 conv: cuTensorMapEncodeTiled failed (%d)", (int)r);
            return NPVS_ERR_CUDA;
        }
    }
    const long long tiles_cap = (long long)ceil_div(p.cap_rows, kBM) * sh.n_tiles;
    const int grid = (int)std::min<long long>(tiles_cap * (p.part ? p.KB : 1), kNumSMs);
    // dense TMA tiles (gmode 2) are issued by warp 0 alone: four gather warps leave the epilogue warps
    // more registers (the block has 288 threads instead of 416)
    return (d.tune_gather_warps == 4 || p.gmode == 2) ? launch_tc_lag<4>(lag, p, tm, tm_t, grid, smem, st)
                                                     : launch_tc_lag<8>(lag, p, tm, tm_t, grid, smem, st);
}

}  // namespace

float* conv_product_tiles(const npvs_conv_desc& d) {
    if (d.workspace == nullptr) return nullptr;
    Arena ar(d.workspace, d.workspace_bytes);  // the layout of conv_tc_fwd: split-K region, then T
    if (!ar.take<int>(4 * kSplitSlots) || !ar.take<float>((size_t)kSplitSlots * kBM * 256)) return nullptr;
    const size_t tb = product_region_bytes(d);
    if (tb == 0 || ar.size - Arena::round(ar.used) < tb) return nullptr;
    return ar.take<float>(tb / sizeof(float));
}

TcShape tc_shape(int kind, int cin, int cout, int form) {
    TcShape s;
    s.form = form;
    if (form == 1) {  // product form of SUBM3 / DOWN2 / DOWN3 / UP3: T = x [W_0 | W_1 | ...]
        s.J = map27(kind) ? 27 : 8;
        s.taps_eff = 1;
        s.Ntot = s.J * cout;
    } else if (kind == NPVS_CONV_UP2) {
        s.J = 8;
        s.taps_eff = 1;
        s.Ntot = 8 * cout;
    } else {
        s.J = 1;
        s.taps_eff = conv_taps(kind);
        s.Ntot = cout;
    }
    s.tma = cin % 32 == 0;
    s.BKE = (s.tma && cin % 64 != 0) ? 32 : 64;
    s.RB = 2 * s.BKE;
    s.Kflat = s.taps_eff * cin;
    s.KB = (s.Kflat + s.BKE - 1) / s.BKE;
    s.BN = 0;
    // product form: 256-column tiles when the padding costs at most ~6 % of the columns (the widest
    // MMA per issued instruction, fewer tiles per SM), else the widest exact divisor, which keeps
    // the weight image free of padding columns (T itself is never padded)
    const bool pad256 = form == 1 && s.Ntot > 256 && (long long)round_up(s.Ntot, 256) * 100 <= (long long)s.Ntot * 106;
    if (form == 1 && !pad256)
        for (int bn = 256; bn >= 16; bn -= 16)
            if (s.Ntot % bn == 0) {
                s.BN = bn;
                break;
            }
    if (s.BN) {
        s.Npad = s.Ntot;
    } else if (s.Ntot <= 256) {
        s.BN = round_up(s.Ntot, 16);
        s.Npad = s.BN;
    } else {
        s.BN = 256;
        s.Npad = round_up(s.Ntot, 256);
    }
    s.n_tiles = s.Npad / s.BN;
    return s;
}

npvs_status conv_tc_fwd(const npvs_conv_desc& d, const void* x, const void* w, const float* bias, const void* skip,
                        void* y, cudaStream_t st) {
    NPVS_REQUIRE(d.cin % 8 == 0, NPVS_ERR_UNSUPPORTED, "BF16 conv: cin must be a multiple of 8");
    NPVS_REQUIRE(d.cout % 8 == 0, NPVS_ERR_UNSUPPORTED, "BF16 conv: cout must be a multiple of 8");
    const bool up = d.kind == NPVS_CONV_UP2;
    NPVS_REQUIRE(!up || (d.cout % 16 == 0 && d.map2 && d.n_in), NPVS_ERR_UNSUPPORTED,
                 "BF16 UP2 conv: needs cout % 16 == 0, the down map (map2) and n_in");
    const int rows_x = d.cap_in > 0 ? d.cap_in : ((d.kind == NPVS_CONV_SUBM3 || d.kind == NPVS_CONV_HEAD1) ? d.cap_out : 0);
    NPVS_REQUIRE(rows_x > 0, NPVS_ERR_INVALID_ARG, "BF16 conv: cap_in (rows of x) is required for this kind");
    const int* n_x = d.n_in ? d.n_in : ((d.kind == NPVS_CONV_SUBM3 || d.kind == NPVS_CONV_HEAD1) ? d.n_out : nullptr);

    // workspace: split-K region, then (product form) the FP32 product tiles T
    float* part = nullptr;
    int* counters = nullptr;
    float* T = nullptr;
    if (d.workspace != nullptr) {
        Arena ar(d.workspace, d.workspace_bytes);
        counters = ar.take<int>(4 * kSplitSlots);
        part = ar.take<float>((size_t)kSplitSlots * kBM * 256);
        NPVS_REQUIRE(counters && part, NPVS_ERR_WORKSPACE, "npvs_sparse_conv_fwd: workspace too small");
        const size_t tb = product_region_bytes(d);
        if (tb && ar.size - Arena::round(ar.used) >= tb) T = ar.take<float>(tb / sizeof(float));
    }
    // product form when asked for, or by default where it applies and the workspace holds T
    const bool product = (has_product_form(d.kind) || up) && d.tune_form != 1 && T != nullptr && n_x != nullptr;
    NPVS_REQUIRE(!(d.tune_form == 2 && !product), NPVS_ERR_WORKSPACE,
                 "npvs_sparse_conv_fwd: product form needs n_in and a workspace of npvs_conv_workspace_bytes()");

    TcParams p;
    std::memset(&p, 0, sizeof(p));
    p.kind = d.kind;
    p.cin = d.cin;
    p.cout = d.cout;
    p.relu = d.relu;
    p.out_f32 = d.out_f32;
    p.x = (const __nv_bfloat16*)x;
    p.bias = bias;
    p.skip = (const __nv_bfloat16*)skip;
    p.y = y;
    p.status = d.status;
    p.wait_limit = wait_limit_cycles();
    p.rows_x = rows_x;
    p.max_split = d.tune_max_split > 0 ? d.tune_max_split : 8;
    const int lag = d.tune_lag > 0 ? d.tune_lag : 2;
    const size_t img0 = packed_image_bytes(d.kind, d.cin, d.cout, 0);

    if (product) {
        // T[n][j*cout + o] = sum_c x[n][c] W_j[c][o] over the input rows, then the gather-reduce
        TcShape sh = tc_shape(d.kind, d.cin, d.cout, up ? 0 : 1);  // the up conv's packing is column blocks
        p.w = up ? (const __nv_bfloat16*)w
                 : reinterpret_cast<const __nv_bfloat16*>(reinterpret_cast<const char*>(w) + img0);
        p.taps = 0;
        p.tout = 1;
        // k-split only when asked for explicitly: the unsplit product tiles are what the layer chain
        // reproduces bit for bit
        p.tout_split = d.tune_form == 2 && d.tune_max_split > 1;
        if (p.tout_split) {  // the split-K partial tiles and counters (the workspace's first region)
            p.part = part;
            p.counters = counters;
        }
        p.T = T;
        // TMA stores need 16-byte rows and addresses (the arena aligns T to 256 bytes)
        p.tout_tma = sh.Ntot % 16 == 0 && (reinterpret_cast<uintptr_t>(T) & 255) == 0;
        p.n_rows = n_x;
        p.cap_rows = rows_x;
        p.gmode = sh.tma ? 2 : 0;
        NPVS_TRY(run_gemm(p, sh, d, x, lag, st));
        const int taps = up ? 0 : conv_taps(d.kind);
        const long long work = (long long)d.cap_out * (d.cout / 4);
        NPVS_REQUIRE(work < (1LL << 31), NPVS_ERR_UNSUPPORTED, "BF16 conv: more than 2^31 output groups");
        const int grid = (int)std::max<long long>(1, std::min<long long>(ceil_div(work, 256), kNumSMs * 8));
        if (d.out_f32)
            launch_k(conv_reduce_kernel<float>, grid, 256, 0, st, T, sh.Ntot, d.map, taps, d.n_out, d.cap_out, d.cout, bias,
                                                            d.relu, (const __nv_bfloat16*)skip, (float*)y);
        else
            launch_k(conv_reduce_kernel<__nv_bfloat16>, grid, 256, 0, st, T, sh.Ntot, d.map, taps, d.n_out, d.cap_out, d.cout,
                                                                    bias, d.relu, (const __nv_bfloat16*)skip,
                                                                    (__nv_bfloat16*)y);
        return check_launch("conv_reduce_kernel");
    }

    TcShape sh = tc_shape(d.kind, d.cin, d.cout, 0);
    p.w = (const __nv_bfloat16*)w;
    p.scatter = up;
    p.taps = (map27(d.kind) || d.kind == NPVS_CONV_DOWN2) ? conv_taps(d.kind) : 0;
    p.map = d.map;
    p.map2 = d.map2;
    p.n_rows = up ? d.n_in : d.n_out;
    p.cap_rows = up ? d.cap_in : d.cap_out;
    p.part = part;
    p.counters = counters;
    if (!sh.tma) p.gmode = 0;
    else if (p.taps == 0) p.gmode = 2;      // rows of x read in order: dense tiles
    else if ((d.tune_gather == 3 || d.tune_gather == 4) && d.kind == NPVS_CONV_SUBM3) p.gmode = 3;
    else p.gmode = (d.tune_gather == 2 && sh.BKE == 64) ? 0 : 1;
    return run_gemm(p, sh, d, x, lag, st);
}

}  // namespace npvs

using namespace npvs;

extern "C" size_t npvs_conv_workspace_bytes(const npvs_conv_desc* d) {
    return split_region_bytes() + (d ? product_region_bytes(*d) : 0) + 256;
}

extern "C" size_t npvs_packed_weight_bytes(int32_t kind, int32_t cin, int32_t cout) {
    if (!valid_conv_kind(kind) || cin <= 0 || cout <= 0) return 0;
    if (bf16_narrow(cin, cout)) {
        return Arena::round((size_t)conv_taps_host(kind) * cin * cout * sizeof(__nv_bfloat16));
    }
    size_t b = packed_image_bytes(kind, cin, cout, 0);
    if (has_product_form(kind)) b += packed_image_bytes(kind, cin, cout, 1);
    return b;
}

namespace npvs {

// The images of one weight tensor (mode as weight_at) appended to the batch: the plain image of a
// narrow convolution, else the direct (or transposed-conv) form and, where it exists, the product form.
static void add_images(PackBatch& b, int kind, int cin, int cout, const float* w, void* packed, int mode) {
    char* out = (char*)packed;
    auto push = [&](const PackImage& im) {
        b.im[b.n] = im;
        b.im[b.n].begin = b.total;
        b.total += im.size;
        ++b.n;
    };
    if (bf16_narrow(cin, cout)) {
        PackImage im{};
        im.w = w;
        im.out = (__nv_bfloat16*)out;
        im.plain = 1;
        im.size = (long long)conv_taps_host(kind) * cin * cout;
        push(im);
        return;
    }
    const int nforms = has_product_form(kind) ? 2 : 1;
    for (int f = 0; f < nforms; ++f) {
        PackImage im{};
        im.sh = tc_shape(kind, cin, cout, f);
        im.w = w;
        im.out = (__nv_bfloat16*)out;
        im.kind = kind;
        im.cin = cin;
        im.cout = cout;
        im.mode = mode;
        im.size = (long long)im.sh.KB * im.sh.Npad * im.sh.BKE;
        push(im);
        out += packed_image_bytes(kind, cin, cout, f);
    }
}

static npvs_status launch_pack(const PackBatch& b, cudaStream_t st) {
    if (b.n == 0 || b.total == 0) return NPVS_OK;
    const int grid = (int)std::min<long long>((b.total + 255) / 256, (long long)kNumSMs * 16);
    launch_k(pack_images_kernel, grid, 256, 0, st, b);
    return check_launch("pack_images_kernel");
}

npvs_status pack_weights_mode(int kind, int cin, int cout, const float* w, void* packed, int mode, cudaStream_t st) {
    NPVS_REQUIRE(w && packed && cin > 0 && cout > 0, NPVS_ERR_INVALID_ARG, "npvs_pack_weights: bad arguments");
    NPVS_REQUIRE(valid_conv_kind(kind), NPVS_ERR_UNSUPPORTED, "npvs_pack_weights: unknown kind");
    NPVS_REQUIRE(mode == 0 || !bf16_narrow(cin, cout), NPVS_ERR_UNSUPPORTED,
                 "BF16 conv: transposed packing needs cin and cout multiples of 8");
    PackBatch b{};
    add_images(b, kind, cin, cout, w, packed, mode);
    return launch_pack(b, st);
}

}  // namespace npvs

extern "C" npvs_status npvs_pack_weights(int32_t kind, int32_t cin, int32_t cout, const float* w, void* packed,
                                         void* stream) {
    return pack_weights_mode(kind, cin, cout, w, packed, 0, as_stream(stream));
}

extern "C" size_t npvs_packed_weight_bytes_transposed(int32_t kind, int32_t cin, int32_t cout) {
    if (!valid_conv_kind(kind) || cin <= 0 || cout <= 0 || bf16_narrow(cin, cout)) return 0;
    int mode;
    return npvs_packed_weight_bytes(transposed_kind(kind, &mode), cout, cin);
}

extern "C" npvs_status npvs_pack_weights_many(int32_t n, const npvs_pack_job* jobs, void* stream) {
    NPVS_REQUIRE(n >= 0 && (n == 0 || jobs), NPVS_ERR_INVALID_ARG, "npvs_pack_weights_many: bad arguments");
    for (int i = 0; i < n; ++i) {  // every job is checked before the first launch
        const npvs_pack_job& j = jobs[i];
        if (!(j.w && j.packed && j.cin > 0 && j.cout > 0 && (j.transposed == 0 || j.transposed == 1))) {
            set_error("npvs_pack_weights_many: bad job %d", i);
            return NPVS_ERR_INVALID_ARG;
        }
        if (!valid_conv_kind(j.kind) || (j.transposed && bf16_narrow(j.cin, j.cout))) {
            set_error("npvs_pack_weights_many: job %d: unknown kind, or a transposed image of a convolution whose "
                      "cin or cout is not a multiple of 8", i);
            return NPVS_ERR_UNSUPPORTED;
        }
    }
    cudaStream_t st = as_stream(stream);
    PackBatch b{};
    for (int i = 0; i < n; ++i) {
        const npvs_pack_job& j = jobs[i];
        if (b.n + 2 > kMaxPackImages) {  // a job adds at most two images
            NPVS_TRY(launch_pack(b, st));
            b = PackBatch{};
        }
        if (j.transposed) {
            int mode;
            const int tk = transposed_kind(j.kind, &mode);
            add_images(b, tk, j.cout, j.cin, j.w, j.packed, mode);
        } else {
            add_images(b, j.kind, j.cin, j.cout, j.w, j.packed, 0);
        }
    }
    return launch_pack(b, st);
}
