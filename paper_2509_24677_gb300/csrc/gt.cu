// Ground-truth PVS by from-region ray casting (Sec. 3.2: the training target is the set of
// froxels of the enclosing frustum that are visible from some point of the viewcell, estimated by
// casting rays from points sampled in the cell; Sec. 4.1 samples the cell densely).
//
// For every viewpoint p_m of batch element e and every pixel (a, b) of an (s W) x (s H) raster of
// the enclosing frustum's directions (dir = fwd + n_x tan right + n_y tan up, the same raster as
// the froxelization), the nearest hit t* > 0 of the ray p_m + t dir over e's boxes is found, the
// hit point is expressed in the frustum's camera frame (x_c, y_c, z_c) and, if it lies inside
// the frustum (near <= z_c < far, |x_c / z_c| <= tan, |y_c / z_c| <= tan), the froxel
// (floor((x_c / (z_c tan) + 1) / 2 W), floor((y_c / (z_c tan) + 1) / 2 H), slice(z_c)) is set.
// Optionally the result is ANDed with the geometry grid G (supp(PVS) within supp(G), Sec. 3.2).
//
// One thread per ray; the boxes of the batch element are streamed through shared memory in tiles
// that every thread of the CTA tests its ray against (slab test: a box is entered at
// tn = max(0, max_i min(t0_i, t1_i)), t_i = (bound_i - p_i) * (1 / dir_i), and hit first if it is
// left after that and before the best hit so far). Every floating-point step is one binary32
// operation rounded to nearest (__fadd_rn / __fmul_rn / __fdiv_rn, so nothing is contracted into
// an FMA) in a fixed order: dir_i = (f_i + (n_x tan) r_i) + (n_y tan) u_i as in the froxelization,
// v_i = (p_i + t* dir_i) - c'_i, x_c = (v_0 r_0 + v_1 r_1) + v_2 r_2 (y_c with u, z_c with f),
// x = floor((((x_c / z_c) / tan) + 1) * 0.5 * W). The minimum over boxes does not depend on their
// order, so the result is bit-for-bit the same whatever the tiling.
#include "common.cuh"

namespace npvs {
namespace {

constexpr int kGtCta = 256;
constexpr int kBoxTile = 256;

__device__ __forceinline__ int slice_index(const float* __restrict__ z, int D, float t) {
    int lo = 0, hi = D - 1;  // largest k with z[k] <= t, given z[0] <= t < z[D]
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (z[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kGtCta) gt_raycast_kernel(const float* __restrict__ boxes,
                                                            const int32_t* __restrict__ box_offsets,
                                                            const npvs_camera* __restrict__ cams,
                                                            const float* __restrict__ points, int M, npvs_grid g,
                                                            int s, uint32_t* __restrict__ bits) {
    pdl_begin();
    __shared__ float sb[6][kBoxTile];
    const int sW = s * g.W, sH = s * g.H;
    const long long per_elem = (long long)M * sW * sH;
    const long long first = (long long)blockIdx.x * kGtCta;   // a CTA never spans two elements
    const int e = (int)(first / per_elem);
    if (e >= g.B) return;
    const long long ray = first + threadIdx.x - (long long)e * per_elem;
    const bool live = ray < per_elem;
    const npvs_camera& cam = cams[e];
    float p[3] = {0.f, 0.f, 0.f}, dir[3] = {0.f, 0.f, 1.f};
    if (live) {
        const int m = (int)(ray / ((long long)sW * sH));
        const int rem = (int)(ray - (long long)m * sW * sH);
        const int b = rem / sW, a = rem - b * sW;
        const float nx = __fdiv_rn((float)(2 * a + 1 - sW), (float)sW);
        const float ny = __fdiv_rn((float)(2 * b + 1 - sH), (float)sH);
        const float sx = __fmul_rn(nx, cam.tan_half), sy = __fmul_rn(ny, cam.tan_half);
        const float* pm = points + ((size_t)e * M + m) * 3;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            p[i] = pm[i];
            dir[i] = __fadd_rn(__fadd_rn(cam.fwd[i], __fmul_rn(sx, cam.right[i])), __fmul_rn(sy, cam.up[i]));
        }
    }
    float inv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) inv[i] = __fdiv_rn(1.0f, dir[i]);  // +-inf on an axis-parallel ray
    float best = INFINITY;
    const int j0 = box_offsets[e], j1 = box_offsets[e + 1];
    for (int base = j0; base < j1; base += kBoxTile) {
        const int nt = min(kBoxTile, j1 - base);
        __syncthreads();
        for (int q = threadIdx.x; q < nt * 6; q += kGtCta) sb[q % 6][q / 6] = boxes[(size_t)base * 6 + q];
        __syncthreads();
        if (!live) continue;
        for (int k = 0; k < nt; ++k) {
            float tn = 0.0f, tf = best;  // entry after the origin, before the best hit so far
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float lo = sb[i][k], hi = sb[3 + i][k];
                if (dir[i] == 0.0f) {
                    if (p[i] < lo || p[i] > hi) tf = -1.0f;
                } else {
                    const float t0 = __fmul_rn(__fsub_rn(lo, p[i]), inv[i]);
                    const float t1 = __fmul_rn(__fsub_rn(hi, p[i]), inv[i]);
                    tn = fmaxf(tn, fminf(t0, t1));
                    tf = fminf(tf, fmaxf(t0, t1));
                }
            }
            if (tn <= tf && tn > 0.0f && tn < best) best = tn;
        }
    }
    if (!live || !(best < INFINITY)) return;
    float v[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) v[i] = __fsub_rn(__fadd_rn(p[i], __fmul_rn(best, dir[i])), cam.origin[i]);
    auto dot = [&](const float* e) {
        return __fadd_rn(__fadd_rn(__fmul_rn(v[0], e[0]), __fmul_rn(v[1], e[1])), __fmul_rn(v[2], e[2]));
    };
    const float xc = dot(cam.right), yc = dot(cam.up), zc = dot(cam.fwd);
    if (!(zc >= cam.slices[0] && zc < cam.slices[g.D])) return;
    const float ux = __fdiv_rn(__fdiv_rn(xc, zc), cam.tan_half), uy = __fdiv_rn(__fdiv_rn(yc, zc), cam.tan_half);
    if (!(fabsf(ux) <= 1.0f && fabsf(uy) <= 1.0f)) return;
    const int x = min((int)floorf(__fmul_rn(__fmul_rn(__fadd_rn(ux, 1.0f), 0.5f), (float)g.W)), g.W - 1);
    const int y = min((int)floorf(__fmul_rn(__fmul_rn(__fadd_rn(uy, 1.0f), 0.5f), (float)g.H)), g.H - 1);
    const int k = slice_index(cam.slices, g.D, zc);
    atomicOr(bits + (((size_t)e * g.D + k) * g.H + y) * (g.W / 32) + (x >> 5), 1u << (x & 31));
}

__global__ void __launch_bounds__(256) and_bits_kernel(uint32_t* __restrict__ a, const uint32_t* __restrict__ b,
                                                       long long n) {
    pdl_begin();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] &= b[i];
}

}  // namespace
}  // namespace npvs

using namespace npvs;

extern "C" npvs_status npvs_gt_raycast(const float* boxes, const int32_t* box_offsets, const npvs_camera* cams,
                                       const float* points, int32_t n_points, npvs_grid grid, int32_t s_gt,
                                       const uint32_t* g_bits, uint32_t* gt_bits, void* stream) {
    NPVS_REQUIRE(boxes && box_offsets && cams && points && gt_bits, NPVS_ERR_INVALID_ARG, "npvs_gt_raycast: NULL argument");
    NPVS_REQUIRE(grid.W > 0 && grid.W % 32 == 0 && grid.H > 0 && grid.D > 0 && grid.D <= NPVS_MAX_SLICES && grid.B > 0,
                 NPVS_ERR_INVALID_ARG, "npvs_gt_raycast: bad grid");
    NPVS_REQUIRE(n_points > 0 && s_gt >= 1 && (long long)s_gt * grid.W <= 65536 && (long long)s_gt * grid.H <= 65536,
                 NPVS_ERR_INVALID_ARG, "npvs_gt_raycast: bad n_points or s_gt");
    const long long per_elem = (long long)n_points * s_gt * grid.W * s_gt * grid.H;
    NPVS_REQUIRE(per_elem % kGtCta == 0, NPVS_ERR_UNSUPPORTED,
                 "npvs_gt_raycast: rays per batch element (n_points * s_gt^2 * W * H) must be a multiple of 256");
    const long long blocks = per_elem / kGtCta * grid.B;
    NPVS_REQUIRE(blocks <= 0x7fffffffLL, NPVS_ERR_UNSUPPORTED, "npvs_gt_raycast: too many rays");
    cudaStream_t st = as_stream(stream);
    const size_t words = (size_t)grid.B * grid.D * grid.H * (grid.W / 32);
    if (cudaMemsetAsync(gt_bits, 0, words * sizeof(uint32_t), st) != cudaSuccess) return check_launch("gt memset");
    launch_k(gt_raycast_kernel, (unsigned)blocks, kGtCta, 0, st, boxes, box_offsets, cams, points, (int)n_points, grid,
             (int)s_gt, gt_bits);
    NPVS_TRY(check_launch("gt_raycast_kernel"));
    if (!g_bits) return NPVS_OK;
    const int nb = std::max(1, std::min(ceil_div((long long)words, 256), kNumSMs * 8));
    launch_k(and_bits_kernel, nb, 256, 0, st, gt_bits, g_bits, (long long)words);
    return check_launch("and_bits_kernel");
}
