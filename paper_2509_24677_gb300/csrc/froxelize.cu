// a2: froxelization of a box scene into the geometry grid G (Sec. 3.2, froxelization paragraph),
// and pruning: the test of every box's froxels against a PVS (Sec. 3.2 occlusion culling, Sec. 5.6
// temporal bounding volumes of dynamic objects).
//
// Work decomposition: every box face gets a conservative bounding rectangle of supersampled
// pixels (the face clipped against half the near distance and projected, two sub-pixels of margin:
// the float error of the projection is an order of magnitude smaller) and the froxel columns that
// rectangle touches; a prefix sum over the per-face column counts gives a flat list of
// (face, column) items; each item tests the rays of its column that lie in the face's rectangle
// against its one face (rays outside it cannot hit the face). Every floating-point step of the ray
// test is an explicit round-to-nearest binary32 intrinsic in a fixed order, so the resulting
// bits do not depend on how the work is split. An item whose rays all miss the face, or all hit it
// inside one slice, is decided from bounds on those same rounded values without casting its rays;
// the other items' rays are cast one by one. A hit sets its bit with atomicOr.
#include <climits>

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

// The record of face f (box f / 6, face f % 6) and the number of froxel columns its pixel
// rectangle touches.
__device__ __forceinline__ int face_record(const float* __restrict__ boxes, const int32_t* __restrict__ box_off,
                                           const npvs_camera* __restrict__ cams, const npvs_grid& g, int s, int f,
                                           FaceRec& rec) {
    int j = f / 6, fl = f % 6, axis = fl >> 1, side = fl & 1;
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
    return cnt;
}

// One thread per face (64-thread blocks: the set-up is latency bound, so it is spread over as many
// SMs as the faces allow): the face record, its column count, the exclusive prefix of the counts
// within the block (offs) and the block's total (block_sum); it also clears the item kernel's work
// counter and, when given, the n_zero words of the output bit grid. Threads f < sW + sH also write the
// normalised pixel centre f of the supersampled raster, n = (2a + 1 - S) / S in one binary32
// division: xs[a] for a < sW, then ys[b].
constexpr int kSetupBlock = 64;

__global__ void __launch_bounds__(kSetupBlock) face_setup_kernel(
    const float* __restrict__ boxes, const int32_t* __restrict__ box_off, int n_boxes,
    const npvs_camera* __restrict__ cams, npvs_grid g, int s, FaceRec* __restrict__ faces, int* __restrict__ counts,
    long long* __restrict__ offs, long long* __restrict__ block_sum, float* __restrict__ xs,
    unsigned long long* __restrict__ work, uint32_t* __restrict__ zero_words, long long n_zero) {
    __shared__ long long warp_sum[kSetupBlock / 32];
    pdl_begin();
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f == 0) *work = 0ull;  // the item kernel's work counter
    // the bit grid the item kernel ORs into (froxelization only), cleared here
    for (long long w = f; w < n_zero; w += (long long)gridDim.x * blockDim.x) zero_words[w] = 0u;
    {
        const int sW = s * g.W, sH = s * g.H;
        if (f < sW) xs[f] = __fdiv_rn((float)(2 * f + 1 - sW), (float)sW);
        else if (f < sW + sH) xs[f] = __fdiv_rn((float)(2 * (f - sW) + 1 - sH), (float)sH);
    }
    const bool own = f < n_boxes * 6;
    int cnt = 0;
    if (own) {
        FaceRec rec;
        cnt = face_record(boxes, box_off, cams, g, s, f, rec);
        faces[f] = rec;
        counts[f] = cnt;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    long long before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < kSetupBlock / 32; ++w) {
        if (w < warp) before += warp_sum[w];
        all += warp_sum[w];
    }
    if (own) offs[f] = before + incl - cnt;
    if (threadIdx.x == 0) block_sum[blockIdx.x] = all;
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
                                 const int* __restrict__ counts, long long* __restrict__ total,
                                 unsigned long long* __restrict__ work) {
    pdl_begin();
    int i = blockIdx.x * kScanChunk + threadIdx.x;
    if (i == 0) *work = 0ull;  // the item kernel's work counter
    if (i < n) {
        long long o = offs[i] + chunk_off[blockIdx.x];
        offs[i] = o;
        if (i == n - 1) *total = o + counts[i];
    }
}

// Up to kFusedFaceMax faces (at most 1,024 set-up blocks), the item kernel adds the scanned block
// totals to the set-up kernel's block-local prefixes itself; more faces take the chunked scan.
constexpr int kFusedFaceMax = kSetupBlock * 1024;

// The global item offset of face f: offs[f], plus its set-up block's offset when offs holds the
// block-local prefixes (boff != nullptr).
__device__ __forceinline__ long long face_off(const long long* __restrict__ offs, const long long* boff, int f) {
    return boff ? offs[f] + boff[f / kSetupBlock] : offs[f];
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

// The camera's components along a face's axis (ax) and its two other axes (j1 = ax + 1, j2 = ax + 2,
// mod 3).
struct AxisFrame {
    float o_ax, o1, o2, f_ax, f1, f2, r_ax, r1, r2, u_ax, u1, u2;
};

__device__ __forceinline__ AxisFrame axis_frame(const npvs_camera& c, int ax) {
    const int j1 = ax == 2 ? 0 : ax + 1, j2 = ax == 0 ? 2 : ax - 1;
    AxisFrame A;
    A.o_ax = c.origin[ax]; A.o1 = c.origin[j1]; A.o2 = c.origin[j2];
    A.f_ax = c.fwd[ax];    A.f1 = c.fwd[j1];    A.f2 = c.fwd[j2];
    A.r_ax = c.right[ax];  A.r1 = c.right[j1];  A.r2 = c.right[j2];
    A.u_ax = c.up[ax];     A.u1 = c.up[j1];     A.u2 = c.up[j2];
    return A;
}

// The rays of froxel column (x, y) that lie in the face's pixel rectangle: sub-columns i0..i1 of
// the column and supersampled rows b0..b1 (inclusive; never empty for an item of the face).
struct ColumnSpan {
    int i0, i1, b0, b1;
};

__device__ __forceinline__ ColumnSpan column_span(const FaceRec& fr, int x, int y, int s) {
    ColumnSpan sp;
    sp.i0 = max(fr.sa0 - x * s, 0);
    sp.i1 = min(fr.sa1 - x * s, s - 1);
    sp.b0 = max(y * s, fr.sb0);
    sp.b1 = min(fr.sb1, y * s + s - 1);
    return sp;
}

// Slice constants of one camera: the table, its ends and the exponential-spacing guess.
struct SliceTable {
    const float* z;
    int D;
    float z0, zD, lz0, kscale;
};

__device__ __forceinline__ SliceTable slice_table(const npvs_camera& c, int D) {
    SliceTable T;
    T.z = c.slices;
    T.D = D;
    T.z0 = T.z[0];
    T.zD = T.z[D];
    T.lz0 = __log2f(T.z0);
    T.kscale = (float)D / (__log2f(T.zD) - T.lz0);
    return T;
}

// Bounds of one direction component over the rays of a span. Every rounded operation of
// ray_face_slice is monotone in each input (round-to-nearest is monotone; sx and sy grow with the
// pixel index since tan > 0), so the component's extremes over the span come from its end
// sub-columns (sxa, sxb) and end rows (sya, syb), combined by the same rounded addition.
__device__ __forceinline__ void dir_bounds(float f, float r, float u, float sxa, float sxb, float sya, float syb,
                                           float& lo, float& hi) {
    const float ca = __fadd_rn(f, __fmul_rn(sxa, r)), cb = __fadd_rn(f, __fmul_rn(sxb, r));
    const float ua = __fmul_rn(sya, u), ub = __fmul_rn(syb, u);
    lo = __fadd_rn(fminf(ca, cb), fminf(ua, ub));
    hi = __fadd_rn(fmaxf(ca, cb), fmaxf(ua, ub));
}

// Bounds of h = o + t d over t in [tlo, thi] (tlo > 0) and d in [dlo, dhi]: fl(t d) grows with d for
// t > 0 and is monotone in t for fixed d, so its extremes are products of the interval ends.
__device__ __forceinline__ void hit_bounds(float o, float tlo, float thi, float dlo, float dhi, float& lo,
                                           float& hi) {
    lo = __fadd_rn(o, fminf(__fmul_rn(tlo, dlo), __fmul_rn(thi, dlo)));
    hi = __fadd_rn(o, fmaxf(__fmul_rn(tlo, dhi), __fmul_rn(thi, dhi)));
}

__device__ __forceinline__ bool finite4(float a, float b, float c, float d) {
    return isfinite(a) && isfinite(b) && isfinite(c) && isfinite(d);
}

// Decides a span of rays against a face from interval bounds of ray_face_slice's intermediate values
// (dir_bounds, hit_bounds and the monotone division): 0 when no ray of the span can hit the face, 1
// when every ray hits it inside one slice (*k), 2 when the bounds do not decide. The bounds hold
// every ray's exact binary32 values, so 0 and 1 give the same bits as testing the rays one by one;
// any non-finite bound, or z_0 <= 0, gives 2.
__device__ __forceinline__ int classify_span(const FaceRec& fr, const AxisFrame& A, float num, float tanh_,
                                             const ColumnSpan& sp, int x, int s, const float* __restrict__ xs,
                                             const float* __restrict__ ys, const SliceTable& T, int* k) {
    if (!(T.z0 > 0.0f)) return 2;
    const float sxa = __fmul_rn(xs[x * s + sp.i0], tanh_), sxb = __fmul_rn(xs[x * s + sp.i1], tanh_);
    const float sya = __fmul_rn(ys[sp.b0], tanh_), syb = __fmul_rn(ys[sp.b1], tanh_);
    float dlo, dhi;
    dir_bounds(A.f_ax, A.r_ax, A.u_ax, sxa, sxb, sya, syb, dlo, dhi);
    if (!finite4(dlo, dhi, num, 0.0f) || !(dlo > 0.0f || dhi < 0.0f)) return 2;
    const float ta = __fdiv_rn(num, dlo), tb = __fdiv_rn(num, dhi);
    const float tlo = fminf(ta, tb), thi = fmaxf(ta, tb);
    if (thi < T.z0 || tlo >= T.zD) return 0;
    if (!(tlo >= T.z0 && thi < T.zD)) return 2;
    float e1lo, e1hi, e2lo, e2hi;
    dir_bounds(A.f1, A.r1, A.u1, sxa, sxb, sya, syb, e1lo, e1hi);
    dir_bounds(A.f2, A.r2, A.u2, sxa, sxb, sya, syb, e2lo, e2hi);
    if (!finite4(e1lo, e1hi, e2lo, e2hi)) return 2;
    float h1lo, h1hi, h2lo, h2hi;
    hit_bounds(A.o1, tlo, thi, e1lo, e1hi, h1lo, h1hi);
    hit_bounds(A.o2, tlo, thi, e2lo, e2hi, h2lo, h2hi);
    if (h1hi < fr.lo1 || h1lo > fr.hi1 || h2hi < fr.lo2 || h2lo > fr.hi2) return 0;
    if (!(h1lo >= fr.lo1 && h1hi <= fr.hi1 && h2lo >= fr.lo2 && h2hi <= fr.hi2)) return 2;
    const int kk = slice_guess(T.z, T.D, tlo, T.lz0, T.kscale);  // slices grow with t
    if (!(thi < T.z[kk + 1])) return 2;
    *k = kk;
    return 1;
}

// Casts the rays of one item (face lo, global item index item) one by one and sets (TEST: tests)
// the slices they hit. Every operation is rounded to nearest in binary32 in the order of the per-ray
// definition: direction component i = (f_i + (n_x tan) r_i) + (n_y tan) u_i, t = (P - o_ax) / dir_ax,
// a hit iff z_0 <= t < z_D and o_j + t dir_j lies in the face's closed rectangle for both other axes
// j. The sub-column parts f_i + (n_x tan) r_i are computed once per call; the call takes rows
// q, q + nq, q + 2 nq, ... of the item's span (several threads share an item's rays).
template <int SS, bool TEST>
__device__ __forceinline__ void cast_item_rays(const FaceRec* __restrict__ faces, const long long* __restrict__ offs,
                                               const long long* boff, int lo, long long item, int q, int nq,
                                               const npvs_camera* __restrict__ cams,
                                               const npvs_grid& g, int s, const float* __restrict__ xs,
                                               const float* __restrict__ ys, uint32_t* __restrict__ bits,
                                               const uint32_t* __restrict__ test_bits, uint8_t* visible) {
    constexpr int CAP = SS ? SS : 16;
    if (TEST && *(volatile const uint8_t*)(visible + lo / 6)) return;  // box already kept
    const int WW = g.W >> 5;
    const FaceRec fr = faces[lo];
    const int local = (int)(item - face_off(offs, boff, lo));
    const int x = fr.x0 + local % fr.nx, y = fr.y0 + local / fr.nx;
    const npvs_camera& c = cams[fr.b];
    const AxisFrame A = axis_frame(c, fr.axis);
    const SliceTable T = slice_table(c, g.D);
    const float tanh_ = c.tan_half;
    const float num = __fsub_rn(fr.P, A.o_ax);
    const ColumnSpan sp = column_span(fr, x, y, s);
    const size_t word_base = (((size_t)fr.b * g.D) * g.H + y) * WW + (x >> 5);
    const uint32_t bit = 1u << (x & 31);
    float ca_ax[CAP], ca_1[CAP], ca_2[CAP];
#pragma unroll
    for (int i = 0; i < CAP; ++i) {
        if (i >= s) break;
        const float sx = __fmul_rn(xs[x * s + i], tanh_);
        ca_ax[i] = __fadd_rn(A.f_ax, __fmul_rn(sx, A.r_ax));
        ca_1[i] = __fadd_rn(A.f1, __fmul_rn(sx, A.r1));
        ca_2[i] = __fadd_rn(A.f2, __fmul_rn(sx, A.r2));
    }
    float zlo = 0.f, zhi = -1.f;  // slice interval of the last slice set
    for (int bb = sp.b0 + q; bb <= sp.b1; bb += nq) {
        const float sy = __fmul_rn(ys[bb], tanh_);
        const float su_ax = __fmul_rn(sy, A.u_ax), su_1 = __fmul_rn(sy, A.u1), su_2 = __fmul_rn(sy, A.u2);
#pragma unroll
        for (int i = 0; i < CAP; ++i) {
            if (i >= s) break;
            if (i < sp.i0 || i > sp.i1) continue;
            const float d_ax = __fadd_rn(ca_ax[i], su_ax);
            if (d_ax == 0.0f) continue;
            const float t = __fdiv_rn(num, d_ax);
            if (!(t >= T.z0 && t < T.zD)) continue;
            const float h1 = __fadd_rn(A.o1, __fmul_rn(t, __fadd_rn(ca_1[i], su_1)));
            if (!(h1 >= fr.lo1 && h1 <= fr.hi1)) continue;
            const float h2 = __fadd_rn(A.o2, __fmul_rn(t, __fadd_rn(ca_2[i], su_2)));
            if (!(h2 >= fr.lo2 && h2 <= fr.hi2)) continue;
            if (!(t >= zlo && t < zhi)) {
                const int k = slice_guess(T.z, T.D, t, T.lz0, T.kscale);
                if constexpr (TEST) {
                    if (__ldg(test_bits + word_base + (size_t)k * g.H * WW) & bit) {
                        visible[lo / 6] = 1;
                        return;
                    }
                } else {
                    atomicOr(bits + word_base + (size_t)k * g.H * WW, bit);
                }
                zlo = T.z[k];
                zhi = T.z[k + 1];
            }
        }
    }
}

// SS: the supersampling factor as a compile-time constant (0: runtime value s, up to 16).
// Items (face, froxel column) are numbered face by face; a warp's 32 consecutive items belong to
// one face or a few neighbouring ones, found by a warp-wide search. Each thread first decides its
// item from interval bounds (classify_span): most columns lie wholly outside the face or wholly
// inside it within one slice, and set at most one bit. The block then gathers its undecided items
// into shared memory and casts their rays, each item's rows split over up to s threads, so that the
// threads that cast rays hold undecided items only, instead of waiting on a few edge columns among
// decided ones.
// TEST = false: a hit sets its froxel's bit in `bits`. TEST = true (pruning): a hit whose froxel
// is set in `test_bits` marks the face's box (face index / 6) in `visible`; items of boxes already
// marked are skipped. The rays and their rounding are the same in both modes.
constexpr int kItemsBlock = 256;

template <int SS, bool TEST>
__global__ void __launch_bounds__(kItemsBlock, 4) froxel_items_kernel(
    const FaceRec* __restrict__ faces, const long long* __restrict__ offs, int n_faces,
    const long long* __restrict__ total_p, const long long* __restrict__ block_sum,
    const npvs_camera* __restrict__ cams, npvs_grid g, int s_rt, const float* __restrict__ centres,
    uint32_t* __restrict__ bits, const uint32_t* __restrict__ test_bits, uint8_t* visible,
    unsigned long long* __restrict__ work) {
    __shared__ long long s_item[kItemsBlock];
    __shared__ int s_face[kItemsBlock];
    __shared__ int s_n;
    __shared__ long long s_base;
    __shared__ long long s_boff[kFusedFaceMax / kSetupBlock];
    __shared__ long long s_wsum[kItemsBlock / 32 + 1];
    pdl_begin();
    const int s = SS ? SS : s_rt;
    const int sW = s * g.W, WW = g.W >> 5;
    const float* ys = centres + sW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // block_sum != nullptr: offs holds the set-up kernel's block-local prefixes; every block scans
    // the block totals (four per thread) into s_boff and takes the total from it. Else offs holds
    // the global offsets and *total_p the total.
    const long long* boff = nullptr;
    long long total;
    if (block_sum) {
        static_assert((kFusedFaceMax / kSetupBlock) % kItemsBlock == 0, "block totals split evenly over threads");
        constexpr int kPer = kFusedFaceMax / kSetupBlock / kItemsBlock;
        const int nbs = (n_faces + kSetupBlock - 1) / kSetupBlock;
        long long v[kPer], sum = 0;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int i = threadIdx.x * kPer + j;
            v[j] = i < nbs ? block_sum[i] : 0;
            sum += v[j];
        }
        long long incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_wsum[warp] = incl;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long r = 0;
            for (int w = 0; w < kItemsBlock / 32; ++w) {
                const long long t = s_wsum[w];
                s_wsum[w] = r;
                r += t;
            }
            s_wsum[kItemsBlock / 32] = r;
        }
        __syncthreads();
        long long run = s_wsum[warp] + incl - sum;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            s_boff[threadIdx.x * kPer + j] = run;
            run += v[j];
        }
        total = s_wsum[kItemsBlock / 32];
        boff = s_boff;
        __syncthreads();
    } else {
        total = *total_p;
    }
    // The blocks take units of kItemsBlock items from a work counter (cleared before this launch),
    // so that blocks whose items take long do not leave the others idle at the end. The loop runs
    // per block: every thread reaches the barriers and the warp collectives.
    for (;;) {
        if (threadIdx.x == 0) {
            s_n = 0;
            s_base = (long long)atomicAdd(work, (unsigned long long)kItemsBlock);
        }
        __syncthreads();
        const long long block_base = s_base;
        if (block_base >= total) break;
        const long long base = block_base + (threadIdx.x & ~31);  // the warp's first item
        const long long item = base + lane;
        // max f with offs[f] <= base (offs[0] = 0, non-decreasing), searched by the whole warp: each
        // round the lanes probe 32 evenly spaced faces of [flo, fhi] and a ballot keeps the span of
        // the last probe that is <= base, so about three rounds of loads instead of log2(n_faces)
        int flo = 0, fhi = n_faces - 1;
        while (fhi - flo >= 32) {
            const int step = (fhi - flo + 32) / 32;
            const int pos = min(flo + lane * step, fhi);
            const unsigned ok = __ballot_sync(0xffffffffu, face_off(offs, boff, pos) <= base);  // lane 0 (pos = flo) holds
            const int k = 31 - __clz(ok);
            flo = min(flo + k * step, fhi);
            fhi = min(flo + step - 1, fhi);
        }
        {
            const int pos = flo + lane;
            const unsigned ok = __ballot_sync(0xffffffffu, pos <= fhi && face_off(offs, boff, pos) <= base);
            flo += 31 - __clz(ok);
        }
        // each lane's face, max f with offs[f] <= item: the warp loads the offsets of 32 faces from
        // flo at a time and every lane keeps the last one at or below its item; another window
        // follows while the window's last face starts at or before the warp's last item
        int lo = flo;
        for (int wf = flo;; wf += 32) {
            const long long o = wf + lane < n_faces ? face_off(offs, boff, wf + lane) : LLONG_MAX;
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (__shfl_sync(0xffffffffu, o, j) <= item) lo = wf + j;
            if (!(__shfl_sync(0xffffffffu, o, 31) <= base + 31)) break;
        }
        if (item < total) {
            if (!(TEST && *(volatile const uint8_t*)(visible + lo / 6))) {  // box not kept yet
                const FaceRec fr = faces[lo];
                const int local = (int)(item - face_off(offs, boff, lo));
                const int x = fr.x0 + local % fr.nx, y = fr.y0 + local / fr.nx;
                const npvs_camera& c = cams[fr.b];
                const AxisFrame A = axis_frame(c, fr.axis);
                const SliceTable T = slice_table(c, g.D);
                const ColumnSpan sp = column_span(fr, x, y, s);
                int k = -1;
                const int cls = (sp.i0 <= sp.i1 && sp.b0 <= sp.b1)
                                    ? classify_span(fr, A, __fsub_rn(fr.P, A.o_ax), c.tan_half, sp, x, s, centres,
                                                    ys, T, &k)
                                    : 0;
                if (cls == 1) {
                    const size_t w = (((size_t)fr.b * g.D + k) * g.H + y) * WW + (x >> 5);
                    const uint32_t bit = 1u << (x & 31);
                    if constexpr (TEST) {
                        if (__ldg(test_bits + w) & bit) visible[lo / 6] = 1;
                    } else {
                        atomicOr(bits + w, bit);
                    }
                } else if (cls == 2) {
                    const int j = atomicAdd(&s_n, 1);
                    s_item[j] = item;
                    s_face[j] = lo;
                }
            }
        }
        __syncthreads();
        // nq threads per undecided item (a power of two, at most s rows each), so that the whole
        // block casts rays when few items are undecided
        const int n_slow = s_n;
        if (n_slow > 0) {
            int nq = 1;
            while (2 * nq * n_slow <= kItemsBlock && 2 * nq <= s) nq *= 2;
            const int j = (int)threadIdx.x / nq;
            if (j < n_slow)
                cast_item_rays<SS, TEST>(faces, offs, boff, s_face[j], s_item[j], (int)threadIdx.x % nq, nq, cams, g, s,
                                         centres, ys, bits, test_bits, visible);
        }
        __syncthreads();  // the list and s_base are read before the next unit resets them
    }
}

}  // namespace
}  // namespace npvs

using namespace npvs;

static size_t froxel_ws(int n_boxes) {
    size_t F = (size_t)n_boxes * 6;
    size_t nchunk = (F + kScanChunk - 1) / kScanChunk;
    // block totals of the set-up kernel: its grid covers max(F, s W + s H <= 2 * 65536) threads
    size_t nsetup = (std::max<size_t>(F, 2 * 65536) + kSetupBlock - 1) / kSetupBlock;
    return Arena::round(F * sizeof(FaceRec)) + Arena::round(F * sizeof(int)) + Arena::round(nsetup * sizeof(long long)) +
           Arena::round(F * sizeof(long long)) + 2 * Arena::round((nchunk + 1) * sizeof(int)) +
           2 * Arena::round(sizeof(long long)) + Arena::round(2 * 65536 * sizeof(float)) + 256;
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
    unsigned long long* work = ar.take<unsigned long long>(1);
    const long long setup_threads = std::max<long long>(F, (long long)s * (g.W + g.H));
    long long* block_sum = ar.take<long long>((size_t)ceil_div(setup_threads, kSetupBlock));
    float* centres = ar.take<float>((size_t)s * g.W + (size_t)s * g.H);
    launch_k(face_setup_kernel, ceil_div(setup_threads, kSetupBlock), kSetupBlock, 0, st, boxes, box_offsets, n_boxes,
             cams, g, (int)s, faces, counts, offs, block_sum, centres, work, bits,
             bits ? (long long)g.B * g.D * g.H * (g.W / 32) : 0ll);
    NPVS_TRY(check_launch("face_setup_kernel"));
    const bool fused = F <= kFusedFaceMax;  // the item kernel adds the block offsets itself
    if (!fused) {  // the offsets again from the counts, by chunks
        launch_k(chunk_scan_kernel, nchunk, kScanChunk, 0, st, counts, offs, F, csum);
        NPVS_TRY(check_launch("chunk_scan_kernel"));
        NPVS_TRY(scan_block_counts(csum, coff, nchunk, csum + nchunk, -1, nullptr, st));
        launch_k(chunk_add_kernel, nchunk, kScanChunk, 0, st, offs, F, coff, counts, total, work);
        NPVS_TRY(check_launch("chunk_add_kernel"));
    }
    const int grid = kNumSMs * 4;  // resident blocks (4 per SM); the work counter balances them
#define NPVS_ITEMS(SSV, T)                                                                                           \
    launch_k(froxel_items_kernel<SSV, T>, grid, kItemsBlock, 0, st, faces, offs, F, total, fused ? block_sum : nullptr,  \
             cams, g, s, centres, bits, test_bits, visible, work)
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
    if (n_boxes == 0) {  // no face set-up kernel runs to clear the grid
        const size_t nbytes = (size_t)g.B * g.D * g.H * (g.W / 32) * sizeof(uint32_t);
        if (cudaMemsetAsync(occ_bits, 0, nbytes, st) != cudaSuccess) return check_launch("npvs_froxelize memset");
    }
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
