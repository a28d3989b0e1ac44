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
// grids of at most this many CTAs sum the counts before each CTA in the write kernel (no scan launch)
constexpr int kFusedScanCtas = 1024;

struct ILParams {
    const uint32_t* bits;
    npvs_grid g;
    int d, in_ch, dtype, cap;
    int Xc, Yc, Zc;
    long long n_sites;
    const uint8_t* flags;  // nullable: each site's activity, written by il_active_kernel (d >= 16)
};

// DD: the interleave factor as a compile-time constant (0: runtime p.d). The d row words of SG
// depth slices (SG = 4 for d >= 16, else 1) are loaded together and OR-ed; the test stops after
// the first occupied group.
__device__ __forceinline__ void site_coords(const ILParams& p, long long site, int& b, int& Z, int& Y, int& X) {
    X = (int)(site % p.Xc);
    long long t = site / p.Xc;
    Y = (int)(t % p.Yc);
    t /= p.Yc;
    Z = (int)(t % p.Zc);
    b = (int)(t / p.Zc);
}

// Whether the d^3 block of site (b, Z, Y, X) holds an occupied froxel: the given activity flag, else
// the d row words of SG depth slices (SG = 4 for d >= 16, else 1) loaded together and OR-ed, the
// test stopping after the first occupied group.
template <int DD>
__device__ __forceinline__ bool site_active(const ILParams& p, long long site, int b, int Z, int Y, int X) {
    if (p.flags) return p.flags[site] != 0;
    const int d = DD ? DD : p.d, WW = p.g.W >> 5, x0 = d * X;
    const uint32_t mask = d == 32 ? 0xffffffffu : (((1u << d) - 1u) << (x0 & 31));
    const uint32_t* w = p.bits + (((size_t)b * p.g.D + (size_t)d * Z) * p.g.H + (size_t)d * Y) * WW + (x0 >> 5);
    constexpr int SG = DD >= 16 ? 4 : 1;
    for (int dz0 = 0; dz0 < d; dz0 += SG) {
        uint32_t acc = 0;
#pragma unroll
        for (int q = 0; q < SG; ++q) {
#pragma unroll 16
            for (int dy = 0; dy < (DD ? DD : d); ++dy) acc |= __ldg(w + ((size_t)(dz0 + q) * p.g.H + dy) * WW);
        }
        if (acc & mask) return true;
    }
    return false;
}

// Activity of every site for d >= 16, one warp per site: the lanes share the d^2 row words of the
// site's block and the warp votes (a thread per site would walk up to 1,024 words alone).
__global__ void __launch_bounds__(256) il_active_kernel(ILParams p, uint8_t* __restrict__ flags) {
    pdl_begin();
    const int lane = threadIdx.x & 31;
    const int d = p.d, dd = d * d, WW = p.g.W >> 5;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long site = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); site < p.n_sites;
         site += warps) {  // warp-uniform bound
        int b, Z, Y, X;
        site_coords(p, site, b, Z, Y, X);
        const int x0 = d * X;
        const uint32_t mask = d == 32 ? 0xffffffffu : (((1u << d) - 1u) << (x0 & 31));
        const uint32_t* w = p.bits + (((size_t)b * p.g.D + (size_t)d * Z) * p.g.H + (size_t)d * Y) * WW + (x0 >> 5);
        uint32_t acc = 0;
#pragma unroll 8
        for (int j = lane; j < dd; j += 32) {
            const int dz = j / d, dy = j - dz * d;
            acc |= __ldg(w + ((size_t)dz * p.g.H + dy) * WW);
        }
        const bool any = __any_sync(0xffffffffu, (acc & mask) != 0u);
        if (lane == 0) flags[site] = any ? 1 : 0;
    }
}

template <int DD>
__global__ void __launch_bounds__(kSitesPerCta) il_count_kernel(ILParams p, int* __restrict__ counts) {
    pdl_begin();
    long long site = (long long)blockIdx.x * kSitesPerCta + threadIdx.x;
    int b = 0, Z = 0, Y = 0, X = 0, f = 0;
    if (site < p.n_sites) {
        site_coords(p, site, b, Z, Y, X);
        f = (int)site_active<DD>(p, site, b, Z, Y, X);
    }
    int c = __syncthreads_count(f);
    if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

// Store n (4 or 8, or 1) consecutive channel values of one feature row.
__device__ __forceinline__ void store_vals(void* feats, int dtype, size_t off, const float* v, int n) {
    if (dtype == NPVS_BF16) {
        __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(feats) + off;
        __align__(16) __nv_bfloat16 h[8];
        for (int q = 0; q < n; ++q) h[q] = __float2bfloat16_rn(v[q]);
        if (n == 8) *reinterpret_cast<uint4*>(out) = *reinterpret_cast<uint4*>(h);
        else if (n == 4) *reinterpret_cast<uint2*>(out) = *reinterpret_cast<uint2*>(h);
        else for (int q = 0; q < n; ++q) out[q] = h[q];
    } else if (dtype == NPVS_F32) {
        float* out = reinterpret_cast<float*>(feats) + off;
        if (n >= 4) {
            for (int q = 0; q < n; q += 4) *reinterpret_cast<float4*>(out + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
        } else {
            for (int q = 0; q < n; ++q) out[q] = v[q];
        }
    } else {
        double* out = reinterpret_cast<double*>(feats) + off;
        for (int q = 0; q < n; ++q) out[q] = (double)v[q];
    }
}

// DD: the interleave factor as a compile-time constant (0: runtime p.d)
// Writes the d^2 occupancy values (and, with in_ch = 2, the d^2 depth values) of slab dz of the
// active site st (b, Z, Y, X in .x .. .w) at feature row r.
template <int DD>
__device__ __forceinline__ void il_write_slab(const ILParams& p, int4 st, int r, int dz, void* __restrict__ feats) {
    const int d = DD ? DD : p.d, d2 = d * d, d3 = d2 * d, C = p.in_ch * d3, WW = p.g.W >> 5;
    const int grp = d2 >= 8 ? 8 : d2;  // values per vector store
    const int k = d * st.y + dz, x0 = d * st.w;
    const float dep = __fdiv_rn((float)(2 * k + 1), (float)(2 * p.g.D));
    const uint32_t* wrow = p.bits + (((size_t)st.x * p.g.D + k) * p.g.H + (size_t)d * st.z) * WW + (x0 >> 5);
    const size_t base = (size_t)r * C + (size_t)dz * d2;
    float vo[8], vd[8];
    int nv = 0, j0 = 0;
#pragma unroll
    for (int dy = 0; dy < (DD ? DD : d); ++dy) {
        const uint32_t wbits = wrow[(size_t)dy * WW] >> (x0 & 31);
#pragma unroll
        for (int dx = 0; dx < (DD ? DD : d); ++dx) {
            const bool occ = (wbits >> dx) & 1u;
            vo[nv] = occ ? 1.0f : 0.0f;
            vd[nv] = occ ? dep : 0.0f;
            if (++nv == grp) {
                store_vals(feats, p.dtype, base + j0, vo, grp);
                if (p.in_ch == 2) store_vals(feats, p.dtype, base + d3 + j0, vd, grp);
                j0 += grp;
                nv = 0;
            }
        }
    }
}

// write_feats == 0: coordinates and table only (the features follow in il_feats_kernel).
// block_off == nullptr: the CTA sums the counts of the CTAs before it itself (grids of at most
// kFusedScanCtas CTAs), and the last CTA writes the row count (n_active, clamped to the capacity)
// that the separate scan would have written.
template <int DD>
__global__ void __launch_bounds__(kSitesPerCta) il_write_kernel(ILParams p, const int* __restrict__ block_off,
                                                                const int* __restrict__ counts, int32_t* n_active,
                                                                int32_t* __restrict__ coords, void* __restrict__ feats,
                                                                int32_t* __restrict__ table, int32_t* status,
                                                                int write_feats) {
    pdl_begin();
    __shared__ int sw[33];
    __shared__ int4 s_site[kSitesPerCta];
    __shared__ int s_rank[kSitesPerCta];
    long long site = (long long)blockIdx.x * kSitesPerCta + threadIdx.x;
    int b = 0, Z = 0, Y = 0, X = 0;
    bool in = site < p.n_sites;
    int f = 0;
    if (in) {
        site_coords(p, site, b, Z, Y, X);
        f = (int)site_active<DD>(p, site, b, Z, Y, X);
    }
    int nloc;
    int loc = block_exclusive_scan(f, sw, &nloc);
    int off;
    if (block_off) {
        off = block_off[blockIdx.x];
    } else {
        int v = 0;
        for (int i = threadIdx.x; i < (int)blockIdx.x; i += kSitesPerCta) v += counts[i];
        block_exclusive_scan(v, sw, &off);  // the block total of v: the sites before this CTA
        if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
            int t = off + nloc;
            if (p.cap >= 0 && t > p.cap) {
                raise_status(status, NPVS_ERR_CAPACITY);
                t = p.cap;
            }
            *n_active = t;
        }
    }
    int rank = off + loc;
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
    // one thread per (active site, dz): the d x d occupancy bits of that slab (d words), written as
    // d^2 occupancy values and, with in_ch = 2, d^2 depth values (one quotient per slab)
    if (!write_feats) return;
    const int d = DD ? DD : p.d;
    for (int e = threadIdx.x; e < nloc * d; e += kSitesPerCta) {
        const int i = e / d, dz = e - i * d;
        const int r = s_rank[i];
        if (r >= p.cap) continue;
        il_write_slab<DD>(p, s_site[i], r, dz, feats);
    }
}

// The features of large interleave factors (d >= 16), spread over the whole device: one item per
// (feature row, slab dz, row dy) of the rows il_write_kernel compacted (n_active, device), writing
// the d occupancy values of that froxel row (and, with in_ch = 2, its d depth values) eight at a
// time; the values are those il_write_slab writes.
template <int DD>
__global__ void __launch_bounds__(256) il_feats_kernel(ILParams p, const int32_t* __restrict__ coords,
                                                       const int32_t* __restrict__ n_active, void* __restrict__ feats) {
    pdl_begin();
    const int d = DD ? DD : p.d, d2 = d * d, d3 = d2 * d, C = p.in_ch * d3, WW = p.g.W >> 5;
    const long long n = (long long)min(*n_active, p.cap) * d2;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / d2), q = (int)(e - (long long)r * d2), dz = q / d, dy = q - dz * d;
        const int4 st = reinterpret_cast<const int4*>(coords)[r];
        const int k = d * st.y + dz, x0 = d * st.w;
        const float dep = __fdiv_rn((float)(2 * k + 1), (float)(2 * p.g.D));
        const uint32_t wbits =
            p.bits[(((size_t)st.x * p.g.D + k) * p.g.H + (size_t)d * st.z + dy) * WW + (x0 >> 5)] >> (x0 & 31);
        const size_t base = (size_t)r * C + (size_t)dz * d2 + (size_t)dy * d;
        for (int j0 = 0; j0 < d; j0 += 8) {
            float vo[8], vd[8];
#pragma unroll
            for (int q2 = 0; q2 < 8; ++q2) {
                const bool occ = (wbits >> (j0 + q2)) & 1u;
                vo[q2] = occ ? 1.0f : 0.0f;
                vd[q2] = occ ? dep : 0.0f;
            }
            store_vals(feats, p.dtype, base + j0, vo, 8);
            if (p.in_ch == 2) store_vals(feats, p.dtype, base + d3 + j0, vd, 8);
        }
    }
}

// ---- de-interleave ------------------------------------------------------------------------

// One thread per PVS word (32 froxels along x); index arithmetic in 32 bits (the host checks that
// the word count fits) and shifts by log2(d) (d is a power of two).
__global__ void deinterleave_kernel(const float* __restrict__ logits, const int32_t* __restrict__ table,
                                    const int32_t* __restrict__ n_active, npvs_grid g, int d, int ld, float tau,
                                    const uint32_t* __restrict__ mask_bits, uint32_t* __restrict__ pvs) {
    pdl_begin();
    const uint32_t WW = (uint32_t)g.W >> 5, H = (uint32_t)g.H, D = (uint32_t)g.D;
    const uint32_t n_words = (uint32_t)g.B * D * H * WW;
    const int n = *n_active;
    const int Xc = g.W >> ld, Yc = g.H >> ld, Zc = g.D >> ld, d3 = d * d * d, dm = d - 1;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < n_words; w += gridDim.x * blockDim.x) {
        const uint32_t m = mask_bits[w];
        uint32_t out = 0;
        if (m) {
            const uint32_t xw = w % WW, t = w / WW;
            const int y = (int)(t % H);
            const uint32_t t2 = t / H;
            const int k = (int)(t2 % D), b = (int)(t2 / D);
            const int Y = y >> ld, dy = y & dm, Z = k >> ld, dz = k & dm;
            const long long rowbase = (((long long)b * Zc + Z) * Yc + Y) * Xc;
            const int chan = (dz * d + dy) * d;
            // the word's occupied froxels in two rounds of independent loads (their sites' rows,
            // then their logits) before any threshold, instead of a dependent pair per froxel
            int row[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                row[i] = -1;
                if ((m >> i) & 1u) row[i] = table[rowbase + ((xw * 32 + i) >> ld)];
            }
            float z[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                z[i] = 0.f;
                if (row[i] >= 0 && row[i] < n) z[i] = logits[(size_t)row[i] * d3 + chan + ((xw * 32 + i) & dm)];
            }
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                if (row[i] >= 0 && row[i] < n) {
                    const float pr = 1.0f / (1.0f + expf(-z[i]));
                    if (pr >= tau) out |= 1u << i;
                }
            }
        }
        pvs[w] = out;
    }
}

__global__ void sigmoid_rows_kernel(const float* __restrict__ logits, const int32_t* __restrict__ n_active,
                                    int d3, float* __restrict__ probs) {
    pdl_begin();
    const long long n = (long long)(*n_active) * d3;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        probs[i] = 1.0f / (1.0f + expf(-logits[i]));
}

}  // namespace
}  // namespace npvs

using namespace npvs;

static bool valid_d(int d) { return d == 1 || d == 2 || d == 4 || d == 8 || d == 16 || d == 32; }

// Compaction, coordinates and table; the features in the same kernel for d <= 8, in a separate
// device-wide kernel for d >= 16 (a site's d slabs of d^2 values are too much work for 256 sites
// per CTA). n_active: the device row count the compaction writes.
// offs == nullptr: il_write_kernel computes the CTA offsets from counts and writes n_active.
static void launch_il_write(const ILParams& p, int nb, const int* offs, const int* counts, int32_t* coords, void* feats,
                            int32_t* table, int32_t* status, int32_t* n_active, cudaStream_t st) {
    const int wf = p.d >= 16 ? 0 : 1;
#define NPVS_IL_WRITE(DDV) \
    launch_k(il_write_kernel<DDV>, nb, kSitesPerCta, 0, st, p, offs, counts, n_active, coords, feats, table, status, wf)
    switch (p.d) {
        case 2: NPVS_IL_WRITE(2); break;
        case 4: NPVS_IL_WRITE(4); break;
        case 8: NPVS_IL_WRITE(8); break;
        case 16: NPVS_IL_WRITE(16); break;
        default: NPVS_IL_WRITE(0);
    }
#undef NPVS_IL_WRITE
    if (wf) return;
    const int grid =
        (int)std::max<long long>(1, std::min<long long>(ceil_div((long long)p.cap * p.d * p.d, 256), kNumSMs * 8));
    if (p.d == 16) launch_k(il_feats_kernel<16>, grid, 256, 0, st, p, coords, n_active, feats);
    else launch_k(il_feats_kernel<0>, grid, 256, 0, st, p, coords, n_active, feats);
}

static void launch_il_count(const ILParams& p, int nb, int* counts, cudaStream_t st) {
    switch (p.d) {
        case 2: launch_k(il_count_kernel<2>, nb, kSitesPerCta, 0, st, p, counts); break;
        case 4: launch_k(il_count_kernel<4>, nb, kSitesPerCta, 0, st, p, counts); break;
        case 8: launch_k(il_count_kernel<8>, nb, kSitesPerCta, 0, st, p, counts); break;
        case 16: launch_k(il_count_kernel<16>, nb, kSitesPerCta, 0, st, p, counts); break;
        default: launch_k(il_count_kernel<0>, nb, kSitesPerCta, 0, st, p, counts);
    }
}

// The site activity pre-pass for large interleave factors (flags: one byte per site).
static bool il_flags_pass(int d) { return d >= 16; }

static void launch_il_active(const ILParams& p, uint8_t* flags, cudaStream_t st) {
    const int grid = (int)std::max<long long>(1, std::min<long long>(ceil_div(p.n_sites, 8), kNumSMs * 16));
    launch_k(il_active_kernel, grid, 256, 0, st, p, flags);
}

extern "C" size_t npvs_interleave_workspace_bytes(npvs_grid g, int32_t d) {
    if (!valid_d(d) || d <= 0) return 0;
    long long sites = (long long)g.B * (g.W / d) * (g.H / d) * (g.D / d);
    long long nb = (sites + kSitesPerCta - 1) / kSitesPerCta;
    const size_t flags = il_flags_pass(d) ? Arena::round((size_t)sites) : 0;
    return 2 * Arena::round((size_t)(nb + 1) * sizeof(int)) + flags + 256;
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
    p.flags = nullptr;
    Arena ar(workspace, workspace_bytes);
    int* counts = ar.take<int>(nb + 1);
    int* offs = ar.take<int>(nb + 1);
    if (il_flags_pass(d)) {
        uint8_t* flags = ar.take<uint8_t>((size_t)p.n_sites);
        launch_il_active(p, flags, st);
        NPVS_TRY(check_launch("il_active_kernel"));
        p.flags = flags;
    }
    launch_il_count(p, nb, counts, st);
    NPVS_TRY(check_launch("il_count_kernel"));
    if (nb <= kFusedScanCtas) {  // the write kernel sums the counts before each CTA itself
        launch_il_write(p, nb, nullptr, counts, coords, feats, table, status, n_active, st);
        return check_launch("il_write_kernel");
    }
    NPVS_TRY(scan_block_counts(counts, offs, nb, n_active, capacity, status, st));
    launch_il_write(p, nb, offs, counts, coords, feats, table, status, n_active, st);
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
    NPVS_REQUIRE(words < (1LL << 31), NPVS_ERR_UNSUPPORTED, "npvs_deinterleave: more than 2^31 PVS words");
    int ld = 0;
    while ((1 << ld) < d) ++ld;
    int blocks = (int)std::min<long long>(ceil_div(words, 256), kNumSMs * 16);
    launch_k(deinterleave_kernel, blocks, 256, 0, st, logits, table, n_active, g, d, ld, tau, mask_bits, pvs_bits);
    NPVS_TRY(check_launch("deinterleave_kernel"));
    if (probs_out) {
        int d3 = d * d * d;
        int pb = (int)std::min<long long>(ceil_div((long long)capacity * d3, 256), kNumSMs * 16);
        if (pb > 0) launch_k(sigmoid_rows_kernel, pb, 256, 0, st, logits, n_active, d3, probs_out);
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
std::mutex g_noalloc_mutex;
// per device ordinal: the context in which the array's address was looked up, and the address
struct NoAllocSlot {
    unsigned long long ctx;
    int* ptr;
};
NoAllocSlot g_noalloc[npvs::kMaxDevices] = {};
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
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_error("npvs_interleave_noalloc: no usable current device");
        return NPVS_ERR_CUDA;
    }
    int* scratch;
    {
        // The device address of the array, looked up with the device current, once per device
        // and context: a device reset makes a new primary context (a new id), and the address of
        // the old one must not be reused, so the look-up is repeated then.
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        const unsigned long long ctx = current_context_id();
        if (ctx == 0 || g_noalloc[dev].ctx != ctx || g_noalloc[dev].ptr == nullptr) {
            void* ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, npvs_interleave_scratch);
            if (e != cudaSuccess || ptr == nullptr) {
                set_error("npvs_interleave_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
                return NPVS_ERR_CUDA;
            }
            g_noalloc[dev].ctx = current_context_id();  // the look-up made the primary context current
            g_noalloc[dev].ptr = static_cast<int*>(ptr);
        }
        scratch = g_noalloc[dev].ptr;
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
    p.flags = nullptr;  // no room for the activity pre-pass: every site is tested where it is read
    const int nb = ceil_div(p.n_sites, kSitesPerCta);
    int* counts = scratch;                      // fully rewritten by every call before it is read
    int* offs = scratch + kNoAllocMaxCtas + 1;  // likewise
    launch_il_count(p, nb, counts, st);
    NPVS_TRY(check_launch("il_count_kernel"));
    if (nb <= kFusedScanCtas) {  // the write kernel sums the counts before each CTA itself
        launch_il_write(p, nb, nullptr, counts, coords, feats, table, status, n_active, st);
        return check_launch("il_write_kernel");
    }
    NPVS_TRY(scan_block_counts(counts, offs, nb, n_active, capacity, status, st));
    launch_il_write(p, nb, offs, counts, coords, feats, table, status, n_active, st);
    return check_launch("il_write_kernel");
}
