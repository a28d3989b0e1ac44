/*
 * Oracle (test infrastructure only): froxelization of an axis-aligned box scene and the
 * ray-cast ground-truth PVS, written as plain loops over the definitions.
 *
 * Only the test suite, the smoke check and the bench's CPU-baseline leg load this file's
 * library. It shares no code with the CUDA path.
 *
 * Camera vector (13 floats): origin c'[3], right r[3], up u[3], forward f[3], tan(phi),
 * where phi = (theta + 2 beta) / 2 is the half-angle of the widened frustum (Sec. 3.2).
 * Slice table z[0..D] (D+1 floats, increasing): froxel depth slice k covers [z[k], z[k+1]).
 *
 * Froxelization (Sec. 3.2, "froxelization" paragraph): every fragment is quantised to a froxel
 * and that froxel's bit is set; the scene is supersampled s x s per froxel column. Fragments
 * here are the hits of one ray per supersampled pixel (a, b) with every box face, front and
 * back, with no depth test:
 *   ray direction  dir = f + (n_x tan(phi)) r + (n_y tan(phi)) u,
 *                  n_x = (2a + 1 - sW) / (sW), n_y = (2b + 1 - sH) / (sH);
 *   face on axis i at coordinate P: t = (P - c'_i) / dir_i, hit if the other two coordinates
 *   c'_j + t dir_j lie in the closed face rectangle and z[0] <= t < z[D];
 *   froxel (floor(a / s), floor(b / s), k) with k = max{k : z[k] <= t}.
 * Bit layout of a grid: word ((k * H + y) * (W / 32) + x / 32), bit (x & 31).
 *
 * Two precisions: the FP32 mirror evaluates each operation above as one IEEE binary32 operation
 * with round-to-nearest in the written order (this file must be compiled with
 * -ffp-contract=off), which fixes the integer outcome of every floating-point decision; the
 * FP64 mode evaluates the same definition in binary64 on the same float32 inputs.
 *
 * Ground truth (Sec. 3.2, last paragraph): from each of M viewpoints p_m in the viewcell, one
 * ray per supersampled pixel of p_m's own frustum (same basis and tan(phi)) finds the nearest
 * face hit t* > 0; the hit point p_m + t* dir is reprojected into the c' frame and its froxel is
 * marked. Two precisions again: binary64 (the nearest hit over every face rectangle), and a
 * binary32 mirror that fixes one sequence of binary32 operations, each rounded to nearest: the
 * nearest entry t* = max_i min(t0_i, t1_i) over the boxes whose slab intervals overlap after the
 * origin (the Kay-Kajiya slab method, t_i = (bound_i - p_i) * (1 / dir_i)), then the reprojection.
 * The slab entry of a ray that starts outside a box is its first face hit, so the two agree up
 * to rounding; the mirror's sequence is what fixes every integer decision bit for bit.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define WORDS_PER_COLUMN(D) (((D) + 31) / 32)

/* ---------------------------------------------------------------------------------------- */
/* binary32 mirror                                                                           */
/* ---------------------------------------------------------------------------------------- */

static int slice_of_f(const float *z, int D, float t) {
    int k = 0;
    for (int i = 1; i < D; ++i)
        if (z[i] <= t) k = i;
    return k;
}

static void ray_dir_f(const float *cam, int a, int b, int sW, int sH, float dir[3]) {
    float nx = (float)(2 * a + 1 - sW) / (float)sW;
    float ny = (float)(2 * b + 1 - sH) / (float)sH;
    float sx = nx * cam[12];
    float sy = ny * cam[12];
    for (int i = 0; i < 3; ++i) {
        float t1 = sx * cam[3 + i];
        float t2 = cam[9 + i] + t1;
        float t3 = sy * cam[6 + i];
        dir[i] = t2 + t3;
    }
}

/* Calls mark(k) for every slice hit by ray (a, b); returns the number of hits. */
static int ray_slices_f(const float *cam, const float *z, int D, const float *boxes, int nb,
                        int a, int b, int sW, int sH, uint32_t *colbits /* WORDS_PER_COLUMN */) {
    float dir[3];
    ray_dir_f(cam, a, b, sW, sH, dir);
    int hits = 0;
    for (int j = 0; j < nb; ++j) {
        const float *bx = boxes + 6 * (size_t)j;
        for (int ax = 0; ax < 3; ++ax) {
            if (dir[ax] == 0.0f) continue;
            int j1 = (ax + 1) % 3, j2 = (ax + 2) % 3;
            for (int side = 0; side < 2; ++side) {
                float P = bx[ax + 3 * side];
                float num = P - cam[ax];
                float t = num / dir[ax];
                if (!(t >= z[0] && t < z[D])) continue;
                float m1 = t * dir[j1];
                float h1 = cam[j1] + m1;
                float m2 = t * dir[j2];
                float h2 = cam[j2] + m2;
                if (h1 >= bx[j1] && h1 <= bx[j1 + 3] && h2 >= bx[j2] && h2 <= bx[j2 + 3]) {
                    int k = slice_of_f(z, D, t);
                    colbits[k >> 5] |= 1u << (k & 31);
                    ++hits;
                }
            }
        }
    }
    return hits;
}

/* ---------------------------------------------------------------------------------------- */
/* binary64 evaluation of the same definition                                                */
/* ---------------------------------------------------------------------------------------- */

static int slice_of_d(const float *z, int D, double t) {
    int k = 0;
    for (int i = 1; i < D; ++i)
        if ((double)z[i] <= t) k = i;
    return k;
}

static void ray_dir_d(const float *cam, int a, int b, int sW, int sH, double dir[3]) {
    double nx = (double)(2 * a + 1 - sW) / (double)sW;
    double ny = (double)(2 * b + 1 - sH) / (double)sH;
    double tp = (double)cam[12];
    for (int i = 0; i < 3; ++i)
        dir[i] = (double)cam[9 + i] + nx * tp * (double)cam[3 + i] + ny * tp * (double)cam[6 + i];
}

static void ray_slices_d(const float *cam, const float *z, int D, const float *boxes, int nb,
                         int a, int b, int sW, int sH, uint32_t *colbits) {
    double dir[3];
    ray_dir_d(cam, a, b, sW, sH, dir);
    for (int j = 0; j < nb; ++j) {
        const float *bx = boxes + 6 * (size_t)j;
        for (int ax = 0; ax < 3; ++ax) {
            if (dir[ax] == 0.0) continue;
            int j1 = (ax + 1) % 3, j2 = (ax + 2) % 3;
            for (int side = 0; side < 2; ++side) {
                double t = ((double)bx[ax + 3 * side] - (double)cam[ax]) / dir[ax];
                if (!(t >= (double)z[0] && t < (double)z[D])) continue;
                double h1 = (double)cam[j1] + t * dir[j1];
                double h2 = (double)cam[j2] + t * dir[j2];
                if (h1 >= bx[j1] && h1 <= bx[j1 + 3] && h2 >= bx[j2] && h2 <= bx[j2 + 3]) {
                    int k = slice_of_d(z, D, t);
                    colbits[k >> 5] |= 1u << (k & 31);
                }
            }
        }
    }
}

/* ---------------------------------------------------------------------------------------- */
/* exported: whole grid, selected columns                                                    */
/* ---------------------------------------------------------------------------------------- */

/* bits: [D][H][W/32], zeroed here. precision: 32 = binary32 mirror, 64 = binary64. */
void oracle_froxelize(const float *cam, const float *z, int W, int H, int D, int s,
                      const float *boxes, int nb, int precision, uint32_t *bits) {
    const int WW = W / 32, sW = s * W, sH = s * H, nw = WORDS_PER_COLUMN(D);
    memset(bits, 0, sizeof(uint32_t) * (size_t)D * H * WW);
    /* one froxel row y per iteration: the words it writes belong to that row only */
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = 0; y < H; ++y) {
        uint32_t col[8];
        for (int x = 0; x < W; ++x) {
            memset(col, 0, sizeof(col));
            for (int b = y * s; b < (y + 1) * s; ++b)
                for (int a = x * s; a < (x + 1) * s; ++a) {
                    if (precision == 64)
                        ray_slices_d(cam, z, D, boxes, nb, a, b, sW, sH, col);
                    else
                        ray_slices_f(cam, z, D, boxes, nb, a, b, sW, sH, col);
                }
            for (int w = 0; w < nw; ++w) {
                uint32_t m = col[w];
                while (m) {
                    int k = 32 * w + __builtin_ctz(m);
                    m &= m - 1;
                    bits[((size_t)k * H + y) * WW + x / 32] |= 1u << (x & 31);
                }
            }
        }
    }
}

/* Slices of the listed froxel columns: cols [nc][2] = (x, y); out [nc][ceil(D/32)]. */
void oracle_froxel_columns(const float *cam, const float *z, int W, int H, int D, int s,
                           const float *boxes, int nb, int precision, const int32_t *cols, int nc,
                           uint32_t *out) {
    const int sW = s * W, sH = s * H, nw = WORDS_PER_COLUMN(D);
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < nc; ++i) {
        uint32_t col[8];
        memset(col, 0, sizeof(col));
        int x = cols[2 * i], y = cols[2 * i + 1];
        for (int b = y * s; b < (y + 1) * s; ++b)
            for (int a = x * s; a < (x + 1) * s; ++a) {
                if (precision == 64)
                    ray_slices_d(cam, z, D, boxes, nb, a, b, sW, sH, col);
                else
                    ray_slices_f(cam, z, D, boxes, nb, a, b, sW, sH, col);
            }
        for (int w = 0; w < nw; ++w) out[(size_t)i * nw + w] = col[w];
    }
}

/* The slice of one depth value t (binary32 compare against the table); -1 outside [z0, zD). */
int oracle_slice_of(const float *z, int D, float t) {
    if (!(t >= z[0] && t < z[D])) return -1;
    return slice_of_f(z, D, t);
}

/* One ray's direction in the binary32 mirror (for tests of the op order). */
void oracle_ray_dir_f32(const float *cam, int a, int b, int sW, int sH, float *dir) {
    ray_dir_f(cam, a, b, sW, sH, dir);
}

/* ---------------------------------------------------------------------------------------- */
/* ground truth: first hits from M viewpoints, reprojected into c' (binary64)                */
/* ---------------------------------------------------------------------------------------- */

/* Nearest hit t* > 0 of the ray p + t dir over all faces; returns +inf if none. */
static double first_hit(const double p[3], const double dir[3], const float *boxes, int nb) {
    double best = INFINITY;
    for (int j = 0; j < nb; ++j) {
        const float *bx = boxes + 6 * (size_t)j;
        for (int ax = 0; ax < 3; ++ax) {
            if (dir[ax] == 0.0) continue;
            int j1 = (ax + 1) % 3, j2 = (ax + 2) % 3;
            for (int side = 0; side < 2; ++side) {
                double t = ((double)bx[ax + 3 * side] - p[ax]) / dir[ax];
                if (!(t > 0.0) || !(t < best)) continue;
                double h1 = p[j1] + t * dir[j1];
                double h2 = p[j2] + t * dir[j2];
                if (h1 >= bx[j1] && h1 <= bx[j1 + 3] && h2 >= bx[j2] && h2 <= bx[j2 + 3]) best = t;
            }
        }
    }
    return best;
}

/*
 * bits: [D][H][W/32] raw ground truth (not yet intersected with G); zeroed here.
 * pts: [M][3] viewpoints. s_gt: rays per froxel column edge for each viewpoint.
 * Returns the number of rays that hit something.
 */
long long oracle_gt_raycast(const float *cam, const float *z, int W, int H, int D, int s_gt,
                            const double *pts, int M, const float *boxes, int nb,
                            uint32_t *bits) {
    const int WW = W / 32, sW = s_gt * W, sH = s_gt * H;
    const double tp = (double)cam[12];
    memset(bits, 0, sizeof(uint32_t) * (size_t)D * H * WW);
    long long nhit = 0;
    const long long nrays = (long long)M * sW * sH;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : nhit)
    for (long long ray = 0; ray < nrays; ++ray) {
        int m = (int)(ray / ((long long)sW * sH));
        int rem = (int)(ray % ((long long)sW * sH));
        int b = rem / sW, a = rem % sW;
        const double *p = pts + 3 * (size_t)m;
        double dir[3];
        ray_dir_d(cam, a, b, sW, sH, dir);
        double t = first_hit(p, dir, boxes, nb);
        if (!(t < INFINITY)) continue;
        ++nhit;
        double v[3];
        for (int i = 0; i < 3; ++i) v[i] = p[i] + t * dir[i] - (double)cam[i];
        double xc = 0, yc = 0, zc = 0;
        for (int i = 0; i < 3; ++i) {
            xc += v[i] * (double)cam[3 + i];
            yc += v[i] * (double)cam[6 + i];
            zc += v[i] * (double)cam[9 + i];
        }
        if (!(zc >= (double)z[0] && zc < (double)z[D])) continue;
        double nx = xc / zc / tp, ny = yc / zc / tp;
        if (!(fabs(nx) <= 1.0 && fabs(ny) <= 1.0)) continue;
        int x = (int)floor((nx + 1.0) / 2.0 * W);
        int y = (int)floor((ny + 1.0) / 2.0 * H);
        if (x > W - 1) x = W - 1;
        if (y > H - 1) y = H - 1;
        int k = slice_of_d(z, D, zc);
        __atomic_fetch_or(&bits[((size_t)k * H + y) * WW + x / 32], 1u << (x & 31),
                          __ATOMIC_RELAXED);
    }
    return nhit;
}

/* ---------------------------------------------------------------------------------------- */
/* ground truth: binary32 mirror                                                             */
/* ---------------------------------------------------------------------------------------- */

/* Nearest slab entry t* > 0 of the ray p + t dir over all boxes (inv = 1 / dir per axis, +-inf
 * where dir is 0); +inf if none. A box is entered at tn = max(0, max_i min(t0_i, t1_i)) and left
 * at tf = min(best, min_i max(t0_i, t1_i)); it is hit first if tn <= tf, tn > 0 and tn < best. */
static float first_hit_f(const float p[3], const float dir[3], const float inv[3], const float *boxes,
                         int nb) {
    float best = INFINITY;
    for (int j = 0; j < nb; ++j) {
        const float *bx = boxes + 6 * (size_t)j;
        float tn = 0.0f, tf = best;
        for (int i = 0; i < 3; ++i) {
            float lo = bx[i], hi = bx[3 + i];
            if (dir[i] == 0.0f) {
                if (p[i] < lo || p[i] > hi) tf = -1.0f;   /* parallel to the slab, outside it */
            } else {
                float d0 = lo - p[i];
                float t0 = d0 * inv[i];
                float d1 = hi - p[i];
                float t1 = d1 * inv[i];
                tn = fmaxf(tn, fminf(t0, t1));
                tf = fminf(tf, fmaxf(t0, t1));
            }
        }
        if (tn <= tf && tn > 0.0f && tn < best) best = tn;
    }
    return best;
}

/*
 * Binary32 mirror of oracle_gt_raycast. pts: [M][3] float viewpoints. Per ray (a, b) of
 * viewpoint m: dir as the froxelization's ray_dir_f, inv_i = 1 / dir_i, t* from first_hit_f,
 * v_i = (p_i + t* dir_i) - c'_i, x_c = (v_0 r_0 + v_1 r_1) + v_2 r_2 (likewise y_c with u, z_c
 * with f), inside iff z[0] <= z_c < z[D] and |(x_c / z_c) / tan| <= 1 and |(y_c / z_c) / tan| <= 1,
 * froxel x = min(floor(((x_c / z_c / tan) + 1) * 0.5 * W), W - 1) (likewise y), slice k of z_c.
 * bits: [D][H][W/32] raw ground truth, zeroed here. Returns the number of rays that hit.
 */
long long oracle_gt_raycast_f32(const float *cam, const float *z, int W, int H, int D, int s_gt,
                                const float *pts, int M, const float *boxes, int nb, uint32_t *bits) {
    const int WW = W / 32, sW = s_gt * W, sH = s_gt * H;
    const float tp = cam[12];
    memset(bits, 0, sizeof(uint32_t) * (size_t)D * H * WW);
    long long nhit = 0;
    const long long nrays = (long long)M * sW * sH;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : nhit)
    for (long long ray = 0; ray < nrays; ++ray) {
        int m = (int)(ray / ((long long)sW * sH));
        int rem = (int)(ray % ((long long)sW * sH));
        int b = rem / sW, a = rem % sW;
        const float *p = pts + 3 * (size_t)m;
        float dir[3], inv[3];
        ray_dir_f(cam, a, b, sW, sH, dir);
        for (int i = 0; i < 3; ++i) inv[i] = 1.0f / dir[i];
        float t = first_hit_f(p, dir, inv, boxes, nb);
        if (!(t < INFINITY)) continue;
        ++nhit;
        float v[3];
        for (int i = 0; i < 3; ++i) {
            float step = t * dir[i];
            float q = p[i] + step;
            v[i] = q - cam[i];
        }
        float c[3];
        for (int axis = 0; axis < 3; ++axis) {          /* 0: right (x_c), 1: up (y_c), 2: fwd (z_c) */
            const float *e = cam + 3 + 3 * axis;
            float s0 = v[0] * e[0];
            float s1 = v[1] * e[1];
            float s2 = v[2] * e[2];
            float acc = s0 + s1;
            c[axis] = acc + s2;
        }
        float xc = c[0], yc = c[1], zc = c[2];
        if (!(zc >= z[0] && zc < z[D])) continue;
        float qx = xc / zc, qy = yc / zc;
        float ux = qx / tp, uy = qy / tp;
        if (!(fabsf(ux) <= 1.0f && fabsf(uy) <= 1.0f)) continue;
        float hx = (ux + 1.0f) * 0.5f, hy = (uy + 1.0f) * 0.5f;
        float fx = hx * (float)W, fy = hy * (float)H;
        int x = (int)floorf(fx), y = (int)floorf(fy);
        if (x > W - 1) x = W - 1;
        if (y > H - 1) y = H - 1;
        int k = slice_of_f(z, D, zc);
        __atomic_fetch_or(&bits[((size_t)k * H + y) * WW + x / 32], 1u << (x & 31), __ATOMIC_RELAXED);
    }
    return nhit;
}
