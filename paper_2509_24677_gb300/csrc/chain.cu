// A chain of sparse convolutions in one persistent launch: the layers of a frame's coarse levels.
//
// Below level 0 the active sites are few (about 2,000, 400 and 100 rows at levels 1-3 of a
// 256x256x128 frame), so a convolution launched on its own is latency: kernel hand-off, prologue,
// a first copy, a few MMAs, an epilogue, and for the product form a second kernel. This kernel runs
// a contiguous run of layers (the down conv into a level, every layer below it, and the up conv
// out of it) in the product form of Sec. 2.3's masked dense definition, each layer as two phases
// separated by grid-wide barriers:
//   GEMM    T[n][j*cout + o] = sum_c x[n][c] W_j[c][o] over the input rows (tcgen05, FP32 in TMEM;
//           A = 128-row TMA tiles of x, B = bulk copies of the packed weight image; warp 0 issues
//           the copies, warp 1 the MMAs, warps 4-7 move the accumulators to T through shared memory
//           with TMA tensor stores);
//   reduce  y[m] = act(b + sum_t T[map(m, t)][t*cout + o]) (+ skip), taps in fixed order
//           (transposed conv: y[m] = act(b + T[parent][tap*cout + o]) through the up map),
// with exactly the operations, in the same order, of the two-kernel product form (conv_tc_kernel
// with its T epilogue, then conv_reduce_kernel), so the results are bitwise those of the layers
// launched one by one in that form.
//
// The launch is cooperative (every CTA resident, one per SM), which the grid barriers need. A
// barrier is a counter in global memory: every CTA adds one and waits, bounded in time, for the
// count of all CTAs; the last CTA to leave the kernel sets the counter back to zero, so it is zero
// between launches. A CTA whose wait expires (an mbarrier of its pipeline or a grid barrier)
// records NPVS_ERR_TIMEOUT, stops issuing work, adds the arrivals it still owes to the counter so
// that no other CTA waits for it, waits for its copies and MMAs in flight, frees its tensor memory
// and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cstring>

#include "chain.cuh"
#include "conv_tc.cuh"
#include "tc_ptx.cuh"

namespace npvs {
namespace {

constexpr int kThreads = 256;       // warp 0 copies, warp 1 MMAs, warps 4-7 epilogue; all reduce
constexpr int kRows = 128;          // GEMM row tile (MMA M)
constexpr int kStages = 4;
constexpr uint32_t kAStride = kRows * 128;  // one A stage: 128 rows of the widest k-block (128 bytes)
constexpr uint32_t kBStride = 256 * 128;    // one B stage: up to 256 columns of 128 bytes

struct ChainLayer {
    CUtensorMap tmap;   // x [rows_x][cin] BF16, box (BKE, 128 rows), swizzle of RB
    CUtensorMap tmapT;  // T [rows_x][Ntot] FP32, box (32 columns, 32 rows), 128-byte swizzle (TMA stores)
    const __nv_bfloat16* w;  // packed image of the GEMM's B operand
    const float* bias;
    const __nv_bfloat16* skip;
    __nv_bfloat16* y;
    const int32_t* map;  // SUBM3 [cap_out][27] neighbours, DOWN2 [cap_out][8] children, UP2 [cap_out] up map
    const int32_t* n_in;
    const int32_t* n_out;
    int kind, cout, relu, taps;  // taps: 27, 8, or 0 for the transposed conv (one parent per row)
    int rows_x, cap_out;
    int KB, Ntot, Npad, BN, n_tiles, BKE, RB;
};

struct ChainParams {
    ChainLayer layers[kChainMaxLayers];
    int n_layers;
    float* T;
    unsigned int* bar;  // [0] barrier arrivals, [1] CTAs done; zero between launches
    int32_t* status;
    long long wait_limit;
    uint32_t acc_cols;
};

constexpr uint32_t kStageTile = 32 * 32 * 4;  // 32 rows x 32 FP32 columns, 128-byte rows, 128-byte swizzle

size_t chain_smem_bytes() {  // 4 epilogue warps x 2 staging tiles
    return 1024 + (size_t)kStages * (kAStride + kBStride) + 8 * kStageTile + (2 * kStages + 5) * 8 + 16;
}


__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__global__ void __launch_bounds__(kThreads, 1) conv_chain_kernel(const __grid_constant__ ChainParams P) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;
    uint8_t* sB = smem + (size_t)kStages * kAStride;
    float* stage_tiles = reinterpret_cast<float*>(sB + (size_t)kStages * kBStride);  // [4 warps][2][32][32]
    uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(stage_tiles) + 8 * kStageTile);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 5);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + kStages);
    const uint32_t tfull0 = smem_u32(bars + 2 * kStages), tempty0 = smem_u32(bars + 2 * kStages + 2);
    const uint32_t mdone = smem_u32(bars + 2 * kStages + 4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long lim = P.wait_limit;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full0 + 8 * s, 1);   // one expect_tx arrival plus the copies' bytes
            mbar_init(empty0 + 8 * s, 1);  // tcgen05.commit of the MMAs that read the stage
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull0 + 8 * b, 1);
            mbar_init(tempty0 + 8 * b, 4);  // one arrival per epilogue warp
        }
        mbar_init(mdone, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), 2 * P.acc_cols);
        tmem_relinquish();
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // pipeline state, carried from layer to layer
    uint32_t p_it = 0;     // producer: k-blocks issued (stage p_it % S, phase (p_it / S) & 1)
    int m_s = 0;           // MMA: stage of the next k-block and its phase parity
    uint32_t m_ph = 0;
    uint32_t tc = 0;       // accumulator hand-overs (the MMA thread and the epilogue count the same units)
    unsigned target = 0;   // grid-barrier count to wait for
    int bars_done = 0;
    const int total_bars = 2 * P.n_layers;

    // Grid-wide barrier: every thread's writes of the phase (T by the epilogue, y by the reduce)
    // are ordered before it; after the reduce also for the async proxy (TMA reads y next). One
    // thread of warp 2 (which has no role in the GEMM phase) adds the CTA's arrival and waits,
    // bounded, for all CTAs. Returns false once the CTA has timed out.
    constexpr int kBarThread = 64;
    auto grid_barrier = [&](bool async_readers) -> bool {
        if (async_readers) fence_proxy_async_global();
        __syncthreads();
        if (threadIdx.x == kBarThread) {
            __threadfence();
            target += gridDim.x;
            atomicAdd(P.bar, 1u);
            ++bars_done;
            if (ld_acquire_gpu(P.bar) < target) {
                const long long t0 = clock64();
                while (ld_acquire_gpu(P.bar) < target) {
                    if (clock64() - t0 > lim) {
                        *abort_flag = 1;
                        break;
                    }
                }
            }
            __threadfence();
        }
        __syncthreads();
        return *abort_flag == 0;
    };

    bool ok = true;
    for (int li = 0; li < P.n_layers && ok; ++li) {
        const ChainLayer& L = P.layers[li];
        const int n_in = min(*L.n_in, L.rows_x);
        const int tiles = ((n_in + kRows - 1) / kRows) * L.n_tiles;
        // ---------------------------------------------------------------- GEMM phase
        if (warp == 0) {
            bool stop = false;
            if (lane == 0) fence_proxy_async_global();  // x was written by generic stores (the last reduce)
            const uint32_t bytes = (uint32_t)kRows * L.RB + (uint32_t)L.BN * L.RB;
            for (int u = blockIdx.x; u < tiles && !stop; u += gridDim.x) {
                const int mt = u / L.n_tiles, nt = u - mt * L.n_tiles;
                for (int kb = 0; kb < L.KB; ++kb, ++p_it) {
                    const int s = (int)(p_it % kStages);
                    mbar_wait(empty0 + 8 * s, ((p_it / kStages) & 1) ^ 1, abort_flag, lim);
                    if (__any_sync(0xffffffffu, *abort_flag)) {
                        stop = true;
                        break;
                    }
                    if (lane == 0) {
                        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(full0 + 8 * s),
                                     "r"(bytes)
                                     : "memory");
                        const __nv_bfloat16* wsrc = L.w + ((size_t)kb * L.Npad + (size_t)nt * L.BN) * L.BKE;
                        bulk_g2s(smem_u32(sB + (size_t)s * kBStride), wsrc, (uint32_t)L.BN * L.RB, full0 + 8 * s);
                        tma_tile2d(smem_u32(sA + (size_t)s * kAStride), &L.tmap, kb * L.BKE, mt * kRows, full0 + 8 * s);
                    }
                    __syncwarp();
                }
            }
        } else if (warp == 1) {
            if (lane == 0) {
                const uint32_t idesc = make_idesc(kRows, L.BN);
                const int kk_steps = L.BKE / 16;
                bool stop = false;
                for (int u = blockIdx.x; u < tiles && !stop; u += gridDim.x, ++tc) {
                    const uint32_t buf = tc & 1;
                    const uint32_t acc = tmem + buf * P.acc_cols;
                    mbar_wait(tempty0 + 8 * buf, ((tc >> 1) & 1) ^ 1, abort_flag, lim);
                    if (*abort_flag) break;
                    tc_fence_after();
                    for (int kb = 0; kb < L.KB; ++kb) {
                        if (!mbar_wait_ok(full0 + 8 * m_s, m_ph, abort_flag, lim)) {
                            stop = true;
                            break;
                        }
                        tc_fence_after();
                        // descriptors advanced by adding the 32-byte K steps to their address field
                        const uint64_t ad = make_sdesc(smem_u32(sA) + (uint32_t)m_s * kAStride, L.RB);
                        const uint64_t bd = make_sdesc(smem_u32(sB) + (uint32_t)m_s * kBStride, L.RB);
                        for (int k = 0; k < kk_steps; ++k)
                            tc_mma(acc, ad + 2 * k, bd + 2 * k, idesc, (kb > 0 || k > 0) ? 1u : 0u);
                        tc_commit(empty0 + 8 * m_s);
                        if (++m_s == kStages) {
                            m_s = 0;
                            m_ph ^= 1u;
                        }
                    }
                    if (!stop) tc_commit(tfull0 + 8 * buf);
                }
            }
            __syncwarp();
        } else if (warp >= 4) {
            // Each lane holds one accumulator row (TMEM lane). Per 32-column chunk the warp's 32 rows
            // go to a shared-memory tile in the 128-byte swizzle layout and leave with one TMA
            // tensor store (two tiles alternate; lane 0 issues and tracks the bulk groups).
            const int q = warp - 4;  // warp % 4: the TMEM lane quadrant it may read
            float* tiles2 = stage_tiles + q * 2 * 32 * 32;
            int ci = 0;  // chunks stored by this warp in this layer (tile ci & 1)
            for (int u = blockIdx.x; u < tiles; u += gridDim.x, ++tc) {
                const int mt = u / L.n_tiles, nt = u - mt * L.n_tiles;
                const int row0 = mt * kRows + q * 32;  // first T row of this warp's 32 rows
                const uint32_t buf = tc & 1;
                mbar_wait(tfull0 + 8 * buf, (tc >> 1) & 1, abort_flag, lim);
                if (__any_sync(0xffffffffu, *abort_flag)) break;
                tc_fence_after();
                const uint32_t taddr = tmem + buf * P.acc_cols + ((uint32_t)(q * 32) << 16);
                for (int c0 = 0; c0 < L.BN; c0 += 32) {
                    const int cw = min(32, L.BN - c0);  // 32, or 16 at the end of a tile
                    uint32_t v[32];
                    tmem_ld16(taddr + (uint32_t)c0, *reinterpret_cast<uint32_t(*)[16]>(v));
                    if (cw == 32) tmem_ld16(taddr + (uint32_t)c0 + 16, *reinterpret_cast<uint32_t(*)[16]>(v + 16));
                    tmem_ld_wait();
                    const int ng = nt * L.BN + c0;
                    if (ng >= L.Ntot || row0 >= n_in) continue;  // nothing of this chunk is read later
                    if (cw == 32 && (ng & 31) == 0) {
                        float* tile = tiles2 + (ci & 1) * 32 * 32;
                        if (lane == 0) bulk_wait_read1();  // the store that last read this tile is done
                        __syncwarp();
#pragma unroll
                        for (int c = 0; c < 8; ++c)  // row `lane`, 16-byte chunk c at position c ^ (lane % 8)
                            *reinterpret_cast<float4*>(tile + lane * 32 + ((c ^ (lane & 7)) << 2)) =
                                make_float4(__uint_as_float(v[4 * c]), __uint_as_float(v[4 * c + 1]),
                                            __uint_as_float(v[4 * c + 2]), __uint_as_float(v[4 * c + 3]));
                        fence_proxy_async_shared();
                        __syncwarp();
                        if (lane == 0) {
                            tma_store_2d(&L.tmapT, ng, row0, smem_u32(tile));
                            bulk_commit();
                        }
                        ++ci;
                    } else {  // a 16-column tail (tile widths that are odd multiples of 16): plain stores
                        const int n = row0 + lane;
                        if (n < n_in)
#pragma unroll
                            for (int k = 0; k < 16; k += 4)
                                *reinterpret_cast<float4*>(P.T + (size_t)n * L.Ntot + ng + k) =
                                    make_float4(__uint_as_float(v[k]), __uint_as_float(v[k + 1]),
                                                __uint_as_float(v[k + 2]), __uint_as_float(v[k + 3]));
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(tempty0 + 8 * buf);
            }
            if (lane == 0) {  // this layer's tensor stores have landed; order them before the barrier
                bulk_wait_all();
                fence_proxy_async_global();
            }
            __syncwarp();
        }
        if (!grid_barrier(false)) {
            ok = false;
            break;
        }
        // ---------------------------------------------------------------- reduce phase
        {
            const int n_out = min(*L.n_out, L.cap_out);
            const uint32_t G = (uint32_t)L.cout >> 2;
            const uint32_t total = (uint32_t)n_out * G;
            for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
                const int m = (int)(e / G), o = (int)(e - (uint32_t)m * G) * 4;
                float4 acc = L.bias ? *reinterpret_cast<const float4*>(L.bias + o) : make_float4(0.f, 0.f, 0.f, 0.f);
                if (L.taps == 0) {
                    const int u = __ldg(L.map + m);
                    if (u >= 0) {
                        const float4 v =
                            __ldcg(reinterpret_cast<const float4*>(P.T + (size_t)(u >> 3) * L.Ntot + (u & 7) * L.cout + o));
                        acc.x += v.x;
                        acc.y += v.y;
                        acc.z += v.z;
                        acc.w += v.w;
                    }
                } else {
                    // every neighbour index first, then every product row, then the sums in tap
                    // order (one memory round trip each instead of one per batch of taps)
                    const int32_t* mp = L.map + (size_t)m * L.taps;
                    int nb[27];
#pragma unroll
                    for (int t = 0; t < 27; ++t) nb[t] = t < L.taps ? __ldg(mp + t) : -1;
                    float4 v[27];
#pragma unroll
                    for (int t = 0; t < 27; ++t)
                        v[t] = nb[t] >= 0 ? __ldcg(reinterpret_cast<const float4*>(P.T + (size_t)nb[t] * L.Ntot + t * L.cout + o))
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
                if (L.relu) {
                    acc.x = fmaxf(acc.x, 0.f);
                    acc.y = fmaxf(acc.y, 0.f);
                    acc.z = fmaxf(acc.z, 0.f);
                    acc.w = fmaxf(acc.w, 0.f);
                }
                const size_t off = (size_t)m * L.cout + o;
                if (L.skip) {  // written earlier in this launch by other CTAs: read through L2
                    const uint2 raw = __ldcg(reinterpret_cast<const uint2*>(L.skip + off));
                    __align__(8) __nv_bfloat16 h[4];
                    *reinterpret_cast<uint2*>(h) = raw;
                    acc.x += __bfloat162float(h[0]);
                    acc.y += __bfloat162float(h[1]);
                    acc.z += __bfloat162float(h[2]);
                    acc.w += __bfloat162float(h[3]);
                }
                __align__(8) __nv_bfloat16 h[4] = {__float2bfloat16_rn(acc.x), __float2bfloat16_rn(acc.y),
                                                    __float2bfloat16_rn(acc.z), __float2bfloat16_rn(acc.w)};
                *reinterpret_cast<uint2*>(L.y + off) = *reinterpret_cast<uint2*>(h);
            }
        }
        if (!grid_barrier(true)) ok = false;
    }

    // ---- teardown
    if (warp == 0 && lane == 0)  // nothing the TMA engine writes may still be landing when the CTA leaves
        for (uint32_t j = p_it >= (uint32_t)kStages ? p_it - kStages : 0; j < p_it; ++j)
            mbar_wait(full0 + 8 * (j % kStages), (j / kStages) & 1, abort_flag, lim);
    if (warp == 1 && lane == 0) {  // every MMA this CTA issued has completed before TMEM is released
        tc_commit(mdone);
        mbar_wait(mdone, 0, abort_flag, lim);
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 2 * P.acc_cols);
    }
    if (threadIdx.x == kBarThread) {
        if (*abort_flag) raise_status(P.status, NPVS_ERR_TIMEOUT);
        // arrivals this CTA still owes (after a timeout), so that no other CTA waits for it
        if (bars_done < total_bars) atomicAdd(P.bar, (unsigned)(total_bars - bars_done));
        __threadfence();
        // the last CTA to leave sets the barrier words back to zero for the next launch: every
        // other CTA has passed its last barrier wait by then
        if (atomicAdd(P.bar + 1, 1u) == gridDim.x - 1) {
            atomicExch(P.bar, 0u);
            atomicExch(P.bar + 1, 0u);
        }
    }
}

}  // namespace

bool chain_layer_supported(int kind, int cin, int cout) {
    return (kind == NPVS_CONV_SUBM3 || kind == NPVS_CONV_DOWN2 || kind == NPVS_CONV_UP2) && cin % 32 == 0 &&
           cout % 16 == 0 && cin <= 4096 && cout <= 4096;
}

size_t chain_tiles_bytes(int kind, int cin, int cout, int rows_x) {
    const TcShape sh = tc_shape(kind, cin, cout, kind == NPVS_CONV_UP2 ? 0 : 1);
    return (size_t)rows_x * sh.Ntot * sizeof(float);
}

npvs_status chain_launch(const ChainLayerHost* layers, int n_layers, float* T, size_t T_bytes, unsigned int* bar,
                         int32_t* status, cudaStream_t st) {
    NPVS_REQUIRE(n_layers >= 1 && n_layers <= kChainMaxLayers, NPVS_ERR_UNSUPPORTED,
                 "layer chain: 1 to 24 layers");
    NPVS_REQUIRE(T && bar, NPVS_ERR_WORKSPACE, "layer chain: no product tiles or barrier words in the workspace");
    EncodeTiledFn enc = encode_tiled();
    NPVS_REQUIRE(enc != nullptr, NPVS_ERR_CUDA, "layer chain: cuTensorMapEncodeTiled unavailable");
    static_assert(sizeof(ChainParams) < 32000, "kernel parameters must stay below the 32 KB limit");
    alignas(64) ChainParams P;  // passed by value: the launch copies it into the kernel's parameters
    std::memset(&P, 0, sizeof(P));
    int max_bn = 16;
    for (int i = 0; i < n_layers; ++i) {
        const ChainLayerHost& h = layers[i];
        NPVS_REQUIRE(chain_layer_supported(h.kind, h.cin, h.cout) && h.x && h.w && h.y && h.map && h.n_in &&
                         h.n_out && h.rows_x > 0 && h.cap_out >= 0 && (h.kind == NPVS_CONV_SUBM3 || h.map2),
                     NPVS_ERR_UNSUPPORTED, "layer chain: unsupported layer");
        const bool up = h.kind == NPVS_CONV_UP2;
        const TcShape sh = tc_shape(h.kind, h.cin, h.cout, up ? 0 : 1);
        NPVS_REQUIRE(sh.BN <= 256 && (size_t)h.rows_x * sh.Ntot * sizeof(float) <= T_bytes, NPVS_ERR_WORKSPACE,
                     "layer chain: product tiles do not fit the workspace");
        ChainLayer& L = P.layers[i];
        // the product image follows the direct image in the packed weights (npvs_pack_weights); the
        // transposed conv's column-block image is its direct image
        const TcShape sh0 = tc_shape(h.kind, h.cin, h.cout, 0);
        const size_t img0 = Arena::round((size_t)sh0.KB * sh0.Npad * sh0.BKE * sizeof(__nv_bfloat16));
        L.w = reinterpret_cast<const __nv_bfloat16*>(static_cast<const char*>(h.w) + (up ? 0 : img0));
        L.bias = h.bias;
        L.skip = static_cast<const __nv_bfloat16*>(h.skip);
        L.y = static_cast<__nv_bfloat16*>(h.y);
        L.map = h.map;
        L.kind = h.kind;
        L.n_in = h.n_in;
        L.n_out = h.n_out;
        L.cout = h.cout;
        L.relu = h.relu;
        L.taps = up ? 0 : conv_taps(h.kind);
        L.rows_x = h.rows_x;
        L.cap_out = h.cap_out;
        L.KB = sh.KB;
        L.Ntot = sh.Ntot;
        L.Npad = sh.Npad;
        L.BN = sh.BN;
        L.n_tiles = sh.n_tiles;
        L.BKE = sh.BKE;
        L.RB = sh.RB;
        max_bn = std::max(max_bn, sh.BN);
        const cuuint64_t gdim[2] = {(cuuint64_t)h.cin, (cuuint64_t)h.rows_x};
        const cuuint64_t gstride[1] = {(cuuint64_t)h.cin * 2};
        const cuuint32_t box[2] = {(cuuint32_t)sh.BKE, (cuuint32_t)kRows};
        const cuuint32_t estride[2] = {1, 1};
        CUresult r =
            enc(&L.tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(h.x), gdim, gstride, box, estride,
                CU_TENSOR_MAP_INTERLEAVE_NONE, sh.RB == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        const cuuint64_t tdim[2] = {(cuuint64_t)sh.Ntot, (cuuint64_t)h.rows_x};
        const cuuint64_t tstride[1] = {(cuuint64_t)sh.Ntot * 4};
        const cuuint32_t tbox[2] = {32, 32};
        if (r == CUDA_SUCCESS)
            r = enc(&L.tmapT, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, T, tdim, tstride, tbox, estride,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            set_error("layer chain: cuTensorMapEncodeTiled failed (%d)", (int)r);
            return NPVS_ERR_CUDA;
        }
    }
    P.n_layers = n_layers;
    P.T = T;
    P.bar = bar;
    P.status = status;
    P.wait_limit = wait_limit_cycles();
    P.acc_cols = 32;
    while ((int)P.acc_cols < max_bn) P.acc_cols <<= 1;

    const size_t smem = chain_smem_bytes();
    static std::atomic<unsigned long long> seen[kMaxDevices];
    NPVS_TRY(ensure_dynamic_smem((const void*)conv_chain_kernel, (int)smem, seen, "conv_chain_kernel"));
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv_chain_kernel, kThreads, smem) != cudaSuccess)
        return check_launch("conv_chain_kernel occupancy");
    NPVS_REQUIRE(per_sm >= 1, NPVS_ERR_UNSUPPORTED, "layer chain: the kernel does not fit an SM");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)sms);  // one CTA per SM, all resident (cooperative launch)
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, conv_chain_kernel, P);
    return check_launch("conv_chain_kernel");
}

}  // namespace npvs
