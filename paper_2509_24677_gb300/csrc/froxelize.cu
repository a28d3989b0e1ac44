// a2: froxelization of a box scene into the geometry grid G (Sec. 3.2, froxelization paragraph),
// and pruning: the test of every box's froxels against a PVS (Sec. 3.2 occlusion culling, Sec. 5.6
// temporal bounding volumes of dynamic objects).
//
// Work decomposition: every box face gets a conservative bounding rectangle of supersampled
// pixels (the face clipped against half the near distance and projected, two sub-pixels of margin:
// the float error of the projection is an order of magnitude smaller) and the froxel columns that
// rectangle touches; a prefix sum over the per-face column counts gives a flat list of
// (face, column) items; each item casts the rays of its column that lie in the face's rectangle
// against its one face (rays outside it cannot hit the face). Every floating-point step of the ray
// test is an explicit round-to-nearest binary32 intrinsic in a fixed order, so the resulting
// bits do not depend on how the work is split. A hit sets its bit with atomicOr.
#include "common.cuh"

namespace npvs {
namespace {

struct __align__(16) FaceRec {
    int b, axis;
    float P, lo1, hi1, lo2, hi2;
    int x0, y0, nx, ny;      // froxel columns touched
    int sa0, sa1, sb0, sb1;  // supersampled pixels of the rectangle (inclusive)
};

constexpr int kScanChunk = 1024;

__device__ __forceinline__ int batch_of_box(const int32_t* off, int B, int j) {
    int lo = 0, hi = B - 1;  // largest e with off[e] <= j
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= j) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void face_setup_kernel(const float* __restrict__ boxes, const int32_t* __restrict__ box_off,
                                  int n_boxes, const npvs_camera* __restrict__ cams, npvs_grid g, int s,
                                  FaceRec* __restrict__ faces, int* __restrict__ counts) {
    pdl_begin();
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n_boxes * 6) return;
    int j = f / 6, fl = f % 6, axis = fl >> 1, side = fl & 1;
    FaceRec rec;
    rec.nx = rec.ny = 0;
    rec.x0 = rec.y0 = 0;
    rec.sa0 = rec.sb0 = 0;
    rec.sa1 = rec.sb1 = -1;
    int cnt = 0;
    if (j >= box_off[0] && j < box_off[g.B]) {
        int b = batch_of_box(box_off, g.B, j);
        const npvs_camera& c = cams[b];
        const float* bx = boxes + 6 * (size_t)j;
        int j1 = (axis + 1) % 3, j2 = (axis + 2) % 3;
        rec.b = b;
        rec.axis = axis;
        rec.P = bx[axis + 3 * side];
        rec.lo1 = bx[j1];
        rec.hi1 = bx[j1 + 3];
        rec.lo2 = bx[j2];
        rec.hi2 = bx[j2 + 3];
        // face corners in camera coordinates
        float cx[4], cy[4], cz[4];
        for (int q = 0; q < 4; ++q) {
            float p[3];
            p[axis] = rec.P;
            p[j1] = (q & 1) ? rec.hi1 : rec.lo1;
            p[j2] = (q & 2) ? rec.hi2 : rec.lo2;
            float v0 = p[0] - c.origin[0], v1 = p[1] - c.origin[1], v2 = p[2] - c.origin[2];
            cx[q] = v0 * c.right[0] + v1 * c.right[1] + v2 * c.right[2];
            cy[q] = v0 * c.up[0] + v1 * c.up[1] + v2 * c.up[2];
            cz[q] = v0 * c.fwd[0] + v1 * c.fwd[1] + v2 * c.fwd[2];
        }
        const int order[4] = {0, 1, 3, 2};  // polygon order of the quad
        const float zc = 0.5f * c.slices[0];
        const float zfar = 1.01f * c.slices[c.n_slices];
        float xmin = 1e30f, xmax = -1e30f, ymin = 1e30f, ymax = -1e30f;
        bool any = false, all_far = true;
        for (int e = 0; e < 4; ++e) {
            int A = order[e], Bq = order[(e + 1) & 3];
            bool inA = cz[A] >= zc, inB = cz[Bq] >= zc;
            float px[2], py[2], pz[2];
            int np = 0;
            if (inA) { px[np] = cx[A]; py[np] = cy[A]; pz[np] = cz[A]; ++np; }
            if (inA != inB) {
                float t = (zc - cz[A]) / (cz[Bq] - cz[A]);
                px[np] = cx[A] + t * (cx[Bq] - cx[A]);
                py[np] = cy[A] + t * (cy[Bq] - cy[A]);
                pz[np] = zc;
                ++np;
            }
            for (int q = 0; q < np; ++q) {
                any = true;
                if (pz[q] < zfar) all_far = false;
                float sx = px[q] / (pz[q] * c.tan_half), sy = py[q] / (pz[q] * c.tan_half);
                xmin = fminf(xmin, sx); xmax = fmaxf(xmax, sx);
                ymin = fminf(ymin, sy); ymax = fmaxf(ymax, sy);
            }
        }
        if (any && !all_far) {
            // supersampled pixel coordinate (n + 1) / 2 * sW (pixel a has its centre at a + 1/2),
            // two pixels of margin each side; then the froxel columns of those pixels
            const int sW = s * g.W, sH = s * g.H;
            float gx0 = (xmin + 1.f) * 0.5f * sW, gx1 = (xmax + 1.f) * 0.5f * sW;
            float gy0 = (ymin + 1.f) * 0.5f * sH, gy1 = (ymax + 1.f) * 0.5f * sH;
            gx0 = fmaxf(fminf(gx0, 1e9f), -1e9f); gx1 = fmaxf(fminf(gx1, 1e9f), -1e9f);
            gy0 = fmaxf(fminf(gy0, 1e9f), -1e9f); gy1 = fmaxf(fminf(gy1, 1e9f), -1e9f);
            const int a0 = max((int)floorf(gx0) - 2, 0), a1 = min((int)floorf(gx1) + 2, sW - 1);
            const int b0 = max((int)floorf(gy0) - 2, 0), b1 = min((int)floorf(gy1) + 2, sH - 1);
            if (a0 <= a1 && b0 <= b1) {
                rec.sa0 = a0; rec.sa1 = a1; rec.sb0 = b0; rec.sb1 = b1;
                rec.x0 = a0 / s; rec.y0 = b0 / s;
                rec.nx = a1 / s - rec.x0 + 1; rec.ny = b1 / s - rec.y0 + 1;
                cnt = rec.nx * rec.ny;
            }
        }
    } else {
        rec.b = 0; rec.axis = 0; rec.P = rec.lo1 = rec.hi1 = rec.lo2 = rec.hi2 = 0.f;
    }
    faces[f] = rec;
    counts[f] = cnt;
}

// Per-chunk exclusive scan of counts into 64-bit offsets; chunk sums for the second level.
__global__ void chunk_scan_kernel(const int* __restrict__ counts, long long* __restrict__ offs, int n,
                                  int* __restrict__ chunk_sum) {
    pdl_begin();
    __shared__ int sw[33];
    int i = blockIdx.x * kScanChunk + threadIdx.x;
    int v = i < n ? counts[i] : 0;
    int tot;
    int ex = block_exclusive_scan(v, sw, &tot);
    if (i < n) offs[i] = ex;
    if (threadIdx.x == 0) chunk_sum[blockIdx.x] = tot;
}

__global__ void chunk_add_kernel(long long* __restrict__ offs, int n, const int* __restrict__ chunk_off,
                                 const int* __restrict__ counts, long long* __restrict__ total) {
    pdl_begin();
    int i = blockIdx.x * kScanChunk + threadIdx.x;
    if (i < n) {
        long long o = offs[i] + chunk_off[blockIdx.x];
        offs[i] = o;
        if (i == n - 1) *total = o + counts[i];
    }
}

// Slice of t given z[0] <= t < z[D]: a guess from the exponential spacing of the slice table
// (lz0 = log2 z[0], kscale = D / log2(z[D] / z[0])), verified against the stored bounds and
// corrected to a neighbour; any other table falls back to the binary search. The result is the
// unique k with z[k] <= t < z[k + 1] either way.
__device__ __forceinline__ int slice_of(const float* __restrict__ z, int D, float t);

__device__ __forceinline__ int slice_guess(const float* __restrict__ z, int D, float t, float lz0, float kscale) {
    int k = (int)((__log2f(t) - lz0) * kscale);
    k = min(max(k, 0), D - 1);
    const float lo = z[k], hi = z[k + 1];
    if (lo <= t && t < hi) return k;
    if (t < lo && k > 0 && z[k - 1] <= t) return k - 1;
    if (t >= hi && k + 1 < D && t < z[k + 2]) return k + 1;
    return slice_of(z, D, t);
}

__device__ __forceinline__ int slice_of(const float* __restrict__ z, int D, float t) {
    int lo = 0, hi = D - 1;  // max k in [0, D-1] with z[k] <= t (z[0] <= t holds)
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (z[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Normalised pixel centres n = (2a + 1 - S) / S of the supersampled raster, one binary32 division
// each: xs[a] for a < sW, then ys[b] for b < sH.
__global__ void __launch_bounds__(256) raster_centres_kernel(int sW, int sH, float* __restrict__ xs) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < sW) xs[i] = __fdiv_rn((float)(2 * i + 1 - sW), (float)sW);
    else if (i < sW + sH) xs[i] = __fdiv_rn((float)(2 * (i - sW) + 1 - sH), (float)sH);
}

// SS: the supersampling factor as a compile-time constant (0: runtime value s, up to 16).
// Items (face, froxel column) are numbered face by face; a warp's 32 consecutive items belong to
// one face or a few neighbouring ones, so lane 0 finds the face of the warp's first item by binary
// search and every lane walks forward from it.
// TEST = false: a hit sets its froxel's bit in `bits`. TEST = true (pruning): a hit whose froxel
// is set in `test_bits` marks the face's box (face index / 6) in `visible` and ends the item; items
// of boxes already marked are skipped. The rays and their rounding are the same in both modes.
template <int SS, bool TEST>
__global__ void __launch_bounds__(256, 4) froxel_items_kernel(
    const FaceRec* __restrict__ faces, const long long* __restrict__ offs, int n_faces,
    const long long* __restrict__ total_p, const npvs_camera* __restrict__ cams, npvs_grid g, int s_rt,
    const float* __restrict__ centres, uint32_t* __restrict__ bits, const uint32_t* __restrict__ test_bits,
    uint8_t* visible) {
    pdl_begin();
    constexpr int CAP = SS ? SS : 16;
    const int s = SS ? SS : s_rt;
    const long long total = *total_p;
    const int sW = s * g.W, WW = g.W >> 5;
    const float* ys = centres + sW;
    const int lane = threadIdx.x & 31;
    // the loop runs per warp (base = the warp's first item), so every lane reaches the shuffle
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < total;
         base += (long long)gridDim.x * blockDim.x) {
        const long long item = base + lane;
        // max f with offs[f] <= base (offs[0] = 0, non-decreasing), searched by the whole warp: each
        // round the lanes probe 32 evenly spaced faces of [flo, fhi] and a ballot keeps the span of
        // the last probe that is <= base, so about three rounds of loads instead of log2(n_faces)
        int flo = 0, fhi = n_faces - 1;
        while (fhi - flo >= 32) {
            const int step = (fhi - flo + 32) / 32;
            const int pos = min(flo + lane * step, fhi);
            const unsigned ok = __ballot_sync(0xffffffffu, offs[pos] <= base);  // lane 0 (pos = flo) holds
            const int k = 31 - __clz(ok);
            flo = min(flo + k * step, fhi);
            fhi = min(flo + step - 1, fhi);
        }
        {
            const int pos = flo + lane;
            const unsigned ok = __ballot_sync(0xffffffffu, pos <= fhi && offs[pos] <= base);
            flo += 31 - __clz(ok);
        }
        int lo = flo;
        if (item >= total) continue;
        while (lo + 1 < n_faces && offs[lo + 1] <= item) ++lo;
        if (TEST && *(volatile const uint8_t*)(visible + lo / 6)) continue;  // box already kept
        const FaceRec fr = faces[lo];
        int local = (int)(item - offs[lo]);
        int x = fr.x0 + local % fr.nx, y = fr.y0 + local / fr.nx;
        const npvs_camera& c = cams[fr.b];
        const int ax = fr.axis, j1 = ax == 2 ? 0 : ax + 1, j2 = ax == 0 ? 2 : ax - 1;
        const float o_ax = c.origin[ax], o1 = c.origin[j1], o2 = c.origin[j2];
        const float f_ax = c.fwd[ax], f1 = c.fwd[j1], f2 = c.fwd[j2];
        const float r_ax = c.right[ax], r1 = c.right[j1], r2 = c.right[j2];
        const float u_ax = c.up[ax], u1 = c.up[j1], u2 = c.up[j2];
        const float tanh_ = c.tan_half;
        const float* z = c.slices;
        const float z0 = z[0], zD = z[g.D];
        const float lz0 = __log2f(z0), kscale = (float)g.D / (__log2f(zD) - lz0);
        const float num = __fsub_rn(fr.P, o_ax);
        size_t word_base = (((size_t)fr.b * g.D) * g.H + y) * WW + (x >> 5);
        const uint32_t bit = 1u << (x & 31);
        // ray direction parts that depend on the sub-column a only: f_i + (n_x tan) r_i, each
        // operation rounded as in the per-ray definition
        float ca_ax[CAP], ca_1[CAP], ca_2[CAP];
#pragma unroll
        for (int i = 0; i < CAP; ++i) {
            if (i >= s) break;
            const float nx = centres[x * s + i];
            const float sx = __fmul_rn(nx, tanh_);
            ca_ax[i] = __fadd_rn(f_ax, __fmul_rn(sx, r_ax));
            ca_1[i] = __fadd_rn(f1, __fmul_rn(sx, r1));
            ca_2[i] = __fadd_rn(f2, __fmul_rn(sx, r2));
        }
        int last_k = -1;
        float zlo = 0.f, zhi = -1.f;  // slice interval of last_k
        bool kept = false;            // TEST: the item found a froxel of the PVS
        // the column's rays inside the face's pixel rectangle
        const int i0 = max(fr.sa0 - x * s, 0), i1 = min(fr.sa1 - x * s, s - 1);
        const int b_end = min(fr.sb1 + 1, y * s + s);
        for (int bb = max(y * s, fr.sb0); bb < b_end && !kept; ++bb) {
            const float ny = ys[bb];
            const float sy = __fmul_rn(ny, tanh_);
            const float su_ax = __fmul_rn(sy, u_ax), su_1 = __fmul_rn(sy, u1), su_2 = __fmul_rn(sy, u2);
#pragma unroll
            for (int i = 0; i < CAP; ++i) {
                if (i >= s) break;
                if (i < i0 || i > i1) continue;
                const float d_ax = __fadd_rn(ca_ax[i], su_ax);
                if (d_ax == 0.0f) continue;
                const float t = __fdiv_rn(num, d_ax);
                if (!(t >= z0 && t < zD)) continue;
                const float h1 = __fadd_rn(o1, __fmul_rn(t, __fadd_rn(ca_1[i], su_1)));
                if (!(h1 >= fr.lo1 && h1 <= fr.hi1)) continue;
                const float h2 = __fadd_rn(o2, __fmul_rn(t, __fadd_rn(ca_2[i], su_2)));
                if (!(h2 >= fr.lo2 && h2 <= fr.hi2)) continue;
                if (!(t >= zlo && t < zhi)) {
                    const int k = slice_guess(z, g.D, t, lz0, kscale);
                    if constexpr (TEST) {
                        if (__ldg(test_bits + word_base + (size_t)k * g.H * WW) & bit) {
                            visible[lo / 6] = 1;
                            kept = true;
                            break;
                        }
                    } else {
                        atomicOr(bits + word_base + (size_t)k * g.H * WW, bit);
                    }
                    last_k = k;
                    zlo = z[k];
                    zhi = z[k + 1];
                }
            }
        }
        (void)last_k;
    }
}

}  // namespace
}  // namespace npvs

using namespace npvs;

static size_t froxel_ws(int n_boxes) {
    size_t F = (size_t)n_boxes * 6;
    size_t nchunk = (F + kScanChunk - 1) / kScanChunk;
    return Arena::round(F * sizeof(FaceRec)) + Arena::round(F * sizeof(int)) +
           Arena::round(F * sizeof(long long)) + 2 * Arena::round((nchunk + 1) * sizeof(int)) +
           Arena::round(sizeof(long long)) + Arena::round(2 * 65536 * sizeof(float)) + 256;
}

extern "C" size_t npvs_froxelize_workspace_bytes(int32_t n_boxes) { return froxel_ws(n_boxes); }

// The face set-up, the scan of the per-face column counts and the item kernel; TEST: pruning.
static npvs_status froxel_run(const float* boxes, const int32_t* box_offsets, int32_t n_boxes, const npvs_camera* cams,
                              npvs_grid g, int32_t s, uint32_t* bits, const uint32_t* test_bits, uint8_t* visible,
                              void* workspace, size_t workspace_bytes, cudaStream_t st, const char* who) {
#define NPVS_CHECK_F(cond, code, what)        \
    do {                                      \
        if (!(cond)) {                        \
            set_error("%s: %s", who, (what)); \
            return (code);                    \
        }                                     \
    } while (0)
    NPVS_CHECK_F(box_offsets && cams, NPVS_ERR_INVALID_ARG, "NULL pointer");
    NPVS_CHECK_F(n_boxes >= 0 && (n_boxes == 0 || boxes), NPVS_ERR_INVALID_ARG, "bad boxes");
    NPVS_CHECK_F(g.W > 0 && g.H > 0 && g.D > 0 && g.B > 0 && g.W % 32 == 0, NPVS_ERR_UNSUPPORTED,
                 "need W % 32 == 0 and positive sizes");
    NPVS_CHECK_F(g.D <= NPVS_MAX_SLICES, NPVS_ERR_UNSUPPORTED, "D > NPVS_MAX_SLICES");
    NPVS_CHECK_F(s >= 1 && s <= 16 && (long long)s * g.W <= 65536 && (long long)s * g.H <= 65536, NPVS_ERR_UNSUPPORTED,
                 "supersampling must be 1..16 and s*W, s*H <= 65536");
    NPVS_CHECK_F(workspace_bytes >= froxel_ws(n_boxes) && workspace, NPVS_ERR_WORKSPACE, "workspace too small");
#undef NPVS_CHECK_F
    if (n_boxes == 0) return NPVS_OK;
    const int F = n_boxes * 6;
    const int nchunk = ceil_div(F, kScanChunk);
    Arena ar(workspace, workspace_bytes);
    FaceRec* faces = ar.take<FaceRec>(F);
    int* counts = ar.take<int>(F);
    long long* offs = ar.take<long long>(F);
    int* csum = ar.take<int>(nchunk + 1);
    int* coff = ar.take<int>(nchunk + 1);
    long long* total = ar.take<long long>(1);
    float* centres = ar.take<float>((size_t)s * g.W + (size_t)s * g.H);
    launch_k(raster_centres_kernel, ceil_div((long long)s * (g.W + g.H), 256), 256, 0, st, s * g.W, s * g.H, centres);
    NPVS_TRY(check_launch("raster_centres_kernel"));
    launch_k(face_setup_kernel, ceil_div(F, 256), 256, 0, st, boxes, box_offsets, n_boxes, cams, g, (int)s, faces, counts);
    NPVS_TRY(check_launch("face_setup_kernel"));
    launch_k(chunk_scan_kernel, nchunk, kScanChunk, 0, st, counts, offs, F, csum);
    NPVS_TRY(check_launch("chunk_scan_kernel"));
    NPVS_TRY(scan_block_counts(csum, coff, nchunk, csum + nchunk, -1, nullptr, st));
    launch_k(chunk_add_kernel, nchunk, kScanChunk, 0, st, offs, F, coff, counts, total);
    NPVS_TRY(check_launch("chunk_add_kernel"));
    const int grid = kNumSMs * 8;
#define NPVS_ITEMS(SSV, T)                                                                                           \
    launch_k(froxel_items_kernel<SSV, T>, grid, 256, 0, st, faces, offs, F, total, cams, g, s, centres, bits, test_bits, \
             visible)
    if (test_bits) {
        switch (s) {
            case 4: NPVS_ITEMS(4, true); break;
            case 8: NPVS_ITEMS(8, true); break;
            default: NPVS_ITEMS(0, true);
        }
    } else {
        switch (s) {
            case 1: NPVS_ITEMS(1, false); break;
            case 2: NPVS_ITEMS(2, false); break;
            case 4: NPVS_ITEMS(4, false); break;
            case 8: NPVS_ITEMS(8, false); break;
            default: NPVS_ITEMS(0, false);
        }
    }
#undef NPVS_ITEMS
    return check_launch("froxel_items_kernel");
}

extern "C" npvs_status npvs_froxelize(const float* boxes, const int32_t* box_offsets, int32_t n_boxes,
                                      const npvs_camera* cams, npvs_grid g, int32_t s, uint32_t* occ_bits,
                                      void* workspace, size_t workspace_bytes, void* stream) {
    NPVS_REQUIRE(occ_bits, NPVS_ERR_INVALID_ARG, "npvs_froxelize: NULL pointer");
    NPVS_REQUIRE(g.W > 0 && g.H > 0 && g.D > 0 && g.B > 0 && g.W % 32 == 0, NPVS_ERR_UNSUPPORTED,
                 "npvs_froxelize: need W % 32 == 0 and positive sizes");
    cudaStream_t st = as_stream(stream);
    const size_t nbytes = (size_t)g.B * g.D * g.H * (g.W / 32) * sizeof(uint32_t);
    if (cudaMemsetAsync(occ_bits, 0, nbytes, st) != cudaSuccess) return check_launch("npvs_froxelize memset");
    return froxel_run(boxes, box_offsets, n_boxes, cams, g, s, occ_bits, nullptr, nullptr, workspace, workspace_bytes,
                      st, "npvs_froxelize");
}

extern "C" npvs_status npvs_prune(const float* boxes, const int32_t* box_offsets, int32_t n_boxes,
                                  const npvs_camera* cams, npvs_grid g, int32_t s, const uint32_t* pvs_bits,
                                  uint8_t* visible, void* workspace, size_t workspace_bytes, void* stream) {
    NPVS_REQUIRE(pvs_bits && (n_boxes == 0 || visible), NPVS_ERR_INVALID_ARG, "npvs_prune: NULL pointer");
    NPVS_REQUIRE(n_boxes >= 0, NPVS_ERR_INVALID_ARG, "npvs_prune: bad boxes");
    cudaStream_t st = as_stream(stream);
    if (n_boxes > 0 && cudaMemsetAsync(visible, 0, (size_t)n_boxes, st) != cudaSuccess)
        return check_launch("npvs_prune memset");
    return froxel_run(boxes, box_offsets, n_boxes, cams, g, s, nullptr, pvs_bits, visible, workspace, workspace_bytes,
                      st, "npvs_prune");
}
