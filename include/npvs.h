/*
 * npvs — C ABI of the GB300 (sm_103a) NeuralPVS hot path.
 *
 * The path (Sec. 3 of the paper): a viewcell defines an enclosing frustum (Sec. 3.2); the scene is
 * froxelized into a binary geometry grid G (Sec. 3.2); G is interleaved into a coarse sparse grid
 * with d^3 channels per site (Sec. 3.3, "3D volume-preserving interleaving"); a sparse 3-D
 * convolutional network f_theta runs on it (Sec. 3.3, Sec. 2.3); the result is de-interleaved,
 * passed through a sigmoid and thresholded at tau (Sec. 3.1), and ANDed with G (Sec. 3.2,
 * supp(V) within supp(G)). Training adds the weighted Dice + repulsive visibility loss
 * (Sec. 3.3), hand-written backward kernels and Adam (Sec. 4.2).
 *
 * Conventions for every entry point:
 *  - Pointers marked "device" are CUDA device (or managed) memory owned by the caller; the
 *    library never allocates, frees or retains them past the call. Pointers marked "host" are
 *    read during the call only.
 *  - `stream` is a cudaStream_t passed as void*. All device work is enqueued on it; no entry
 *    point synchronises the device except npvs_check_status.
 *  - Argument errors are returned synchronously (NPVS_ERR_INVALID_ARG / NPVS_ERR_UNSUPPORTED)
 *    and nothing is enqueued. A launch failure returns NPVS_ERR_CUDA. Data-dependent errors found
 *    on the device (a capacity overflow) are OR-ed as bit (1 << status) into the caller's
 *    device status word `status` (nullable); kernels never trap.
 *  - npvs_last_error() returns a message for the last non-OK status on the calling thread.
 *  - Row counts produced on the device (n_rows, n_active) are clamped to the capacity given;
 *    consumers read them from device memory, so a whole frame can be captured in a CUDA graph.
 *
 * Layouts:
 *  - Froxel bits: uint32 [B][D][H][W/32]; froxel (x, y, k) of batch b is bit (x & 31) of word
 *    ((b*D + k)*H + y)*(W/32) + x/32. x runs along the camera's right axis, y along up, k is the
 *    depth slice.
 *  - Sparse level: coords int32 [cap][4] = (b, z, y, x) sorted by the linear index
 *    ((b*Z + z)*Y + y)*X + x; feature rows [cap][C] row-major; table int32 [B*Z*Y*X] holding each
 *    site's row or -1 (a direct-mapped hash table keyed by the linear index).
 *  - Interleaved channel of froxel (d X + dx, d Y + dy, d Z + dz) in input channel c:
 *    c*d^3 + (dz*d + dy)*d + dx. Input channel 0 is occupancy in {0,1}; channel 1 (in_ch = 2) is
 *    the normalised depth (2k+1)/(2D) of slice k at occupied froxels and 0 elsewhere.
 *  - Weights (F32, F64): [taps][cin][cout] row-major, taps 27 (SubM3, tap ((dz+1)*3+(dy+1))*3+(dx+1)
 *    for neighbour offset (dz,dy,dx)), 8 (down/up, tap (cz*2+cy)*2+cx for child offset), 1 (head).
 *    BF16 weights are first packed by npvs_pack_weights into the tensor-core tile layout.
 */
#ifndef NPVS_H
#define NPVS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NPVS_OK = 0,
    NPVS_ERR_INVALID_ARG = 1,
    NPVS_ERR_UNSUPPORTED = 2,
    NPVS_ERR_CAPACITY = 3,
    NPVS_ERR_WORKSPACE = 4,
    NPVS_ERR_CUDA = 5,
    NPVS_ERR_TIMEOUT = 6
} npvs_status;

typedef enum { NPVS_F32 = 0, NPVS_BF16 = 1, NPVS_F64 = 2 } npvs_dtype;

#define NPVS_MAX_SLICES 256

/* Froxel grid: W (multiple of 32) x H x D depth slices, batch B. */
typedef struct {
    int32_t W, H, D, B;
} npvs_grid;

/* Coarse (sparse-level) grid: X x Y x Z sites, batch B. */
typedef struct {
    int32_t X, Y, Z, B;
} npvs_dims;

/* Cube viewcell (Sec. 3.2): centre, half-size, heading yaw (radians about +y; yaw 0 looks along
 * +z; pitch 0), camera FOV theta and rotation allowance beta in degrees, near / far distances. */
typedef struct {
    double centre[3];
    double half_size;
    double yaw;
    double fov_deg;
    double rot_deg;
    double near_;
    double far_;
} npvs_viewcell;

/* Enclosing frustum (Sec. 3.2): apex c', orthonormal basis, tan of the half-angle
 * phi = (theta + 2 beta)/2, and the D+1 increasing slice bounds (slice k covers
 * [slices[k], slices[k+1])). Plain old data; copy an array of them to the device for
 * npvs_froxelize. */
typedef struct {
    float origin[3];
    float right[3];
    float up[3];
    float fwd[3];
    float tan_half;
    int32_t n_slices;
    float slices[NPVS_MAX_SLICES + 1];
} npvs_camera;

/* A sparse level (device pointers; capacity = rows allocated). */
typedef struct {
    npvs_dims dims;
    int32_t capacity;
    int32_t* coords;  /* device [capacity][4] */
    int32_t* n_rows;  /* device scalar */
    int32_t* table;   /* device [B*Z*Y*X] */
} npvs_level;

typedef enum {
    NPVS_RB_SUBM3 = 0,
    NPVS_RB_DOWN2 = 1,
    NPVS_RB_SUBM3_TABLE = 2,
    NPVS_RB_DOWN3 = 3
} npvs_rulebook_kind;

typedef enum {
    NPVS_CONV_SUBM3 = 0, /* submanifold 3x3x3: output set = input set */
    NPVS_CONV_DOWN2 = 1, /* 2x2x2 stride 2: output set = parents */
    NPVS_CONV_UP2 = 2,   /* transposed 2x2x2 stride 2 onto the finer level's set */
    NPVS_CONV_HEAD1 = 3, /* 1x1x1 */
    NPVS_CONV_DOWN3 = 4, /* 3x3x3 stride 2 padding 1: output q gets input 2q + k - 1 through tap k;
                            output set = the dilated set of a DOWN3 rulebook */
    NPVS_CONV_UP3 = 5    /* its transpose: output p gets input q with p = 2q + k - 1, onto the
                            finer level's set */
} npvs_conv_kind;

/* One sparse convolution (Sec. 2.3; masked dense definition y[p] = b + sum_t W_t^T x[p + t]).
 *  map:  SUBM3 -> neighbour rows [cap_out][27] (-1 = none), from npvs_build_rulebook(SUBM3)
 *        DOWN2 -> child rows of each parent [cap_out][8]
 *        UP2   -> parent*8 + child-tap of each fine row [cap_out] (the "up map"); map2 -> the
 *                 child rows of each coarse row [cap_in][8] (the down map of the same level pair)
 *        HEAD1 -> NULL
 *        DOWN3 -> input rows of the 27 taps of each output [cap_out][27] (the map of a DOWN3
 *                 rulebook), map2 -> the rulebook's map2 (for the backward's dgrad);
 *        UP3   -> the map2 of that rulebook, [cap_out][27] coarse rows, map2 -> its map
 *        (DOWN3 / UP3: n_in and cap_in are required)
 *  n_out: device row count of the output level; cap_out its capacity (grid sizing).
 *  x: [cap_in][cin]; y: [cap_out][cout]; skip (nullable): [cap_out][cout] added after ReLU.
 *  dtype: F32 / F64 (SIMT FMA kernels, weights [taps][cin][cout]) or BF16 (tcgen05 kernels,
 *  weights packed by npvs_pack_weights, FP32 accumulation); out_f32: with BF16, write FP32 y.
 *  BF16 with cin or cout not a multiple of 8 (the one- or two-channel stem and the one-logit head of
 *  a network without interleave, d = 1): a SIMT kernel with FP32 accumulation, the packed image is
 *  plain BF16 [taps][cin][cout], the tune fields and the workspace are not used, and
 *  npvs_sparse_conv_bwd returns NPVS_ERR_UNSUPPORTED. */
typedef struct {
    int32_t kind;
    int32_t dtype;
    int32_t cin, cout;
    int32_t relu;
    int32_t out_f32;
    const int32_t* map;
    const int32_t* map2;
    const int32_t* n_out;
    int32_t cap_out;
    const int32_t* n_in;
    int32_t cap_in;
    int32_t* status; /* nullable device status word (NPVS_ERR_TIMEOUT from bounded waits) */
    void* workspace; /* nullable device scratch of npvs_conv_workspace_bytes(desc) bytes for BF16
                        and FP32 convs: split-K partial tiles and counters, and the product-form
                        tiles T (FP32 uses the product form when T fits, else the gather kernel).
                        It must be zero-filled before its first use; every call leaves the
                        counters at zero again. Calls sharing one workspace must not overlap on
                        the device. NULL: gather form without split-K. */
    size_t workspace_bytes;
    int32_t tune_stages;    /* BF16: shared-memory pipeline stages, 3..12 (window gather 2..12;
                               0 = the most that fit) */
    int32_t tune_max_split; /* BF16: largest split-K factor (0 = 8; 1 = never split). The product
                               form's GEMM splits only with tune_form 2 and tune_max_split >= 2
                               (its partial tiles are summed in chunk order, so T differs from the
                               unsplit tiles in rounding; the default keeps them unsplit) */
    int32_t tune_lag;       /* BF16 cp.async gather: groups in flight per thread before a stage is
                               published (0 = 2; clamped to stages - 1) */
    int32_t tune_gather;    /* BF16 gather form: 0 auto, 1 TMA tile::gather4 (cin % 32 == 0),
                               2 cp.async, 3 window gather (SUBM3, cin % 32 == 0: per 128-row tile
                               and dz plane a dense TMA window of input rows, the A operand built
                               from it in shared memory), 4 window gather with the three taps of
                               one (dz, dy) row per pipeline stage (one tap where three do not fit
                               in shared memory) */
    int32_t tune_gather_warps; /* BF16: gather warps per CTA, 4 or 8 (0 = 8) */
    int32_t tune_form;      /* BF16 SUBM3 / DOWN2 / UP2: 0 auto (product form when the workspace
                               holds T), 1 gather (UP2: scatter-epilogue) form, 2 product form */
    const void* w_transposed; /* npvs_sparse_conv_bwd with BF16, nullable: the image of the
                                 transposed convolution of the same weights (npvs_pack_weights_many,
                                 transposed = 1), read by the dgrad instead of packing it from w in
                                 the call. Must be NULL with F32 / F64 (NPVS_ERR_INVALID_ARG).
                                 The forward ignores it. */
} npvs_conv_desc;

/* ---- status and errors --------------------------------------------------------------------- */

/* Message for the last non-OK status returned on the calling thread ("" if none). */
const char* npvs_last_error(void);

/* Library version string. */
const char* npvs_version(void);

/* Number of CUDA kernel launches this library has issued in this process (memsets excluded). */
unsigned long long npvs_launch_count(void);

/* Synchronises `stream`, reads the device status word (int32, device) and clears it. Returns
 * NPVS_OK if it was 0, else the lowest status whose bit was set. */
npvs_status npvs_check_status(int32_t* status, void* stream);

/* Bound of the waits inside the tensor-core kernels (the BF16 convolutions of npvs_sparse_conv_fwd /
 * npvs_forward and the BF16 weight gradient of npvs_sparse_conv_bwd), in SM clock cycles, for every
 * kernel launched after the call (a CUDA graph keeps the bound it was captured with); the paper has
 * no counterpart. cycles = 0 restores the default (4e9 cycles, about 2 s at the maximum SM clock);
 * the previous bound is stored in *previous (nullable). A wait that outlasts the bound makes its CTA
 * stop issuing copies and MMAs, wait (at most ~1e7 SM cycles more per outstanding stage, whatever the
 * bound) for those already in flight, free its tensor memory and return; NPVS_ERR_TIMEOUT is OR-ed
 * into the convolution's status word. The outputs of a timed-out call are undefined, and a
 * convolution workspace it used must be zero-filled again before its next use. A bound of a few
 * cycles makes every wait that is not satisfied when first tested expire (bounds below 1e6 cycles
 * are kept by polling; each poll costs a few hundred cycles): that is how the timeout path is tested.
 * Returns NPVS_ERR_INVALID_ARG for cycles < 0. */
npvs_status npvs_set_wait_limit(int64_t cycles, int64_t* previous);

/* ---- a1: frustum setup (host) --------------------------------------------------------------- */

/* Sec. 3.2 first paragraph: c' = c - fwd * (h / tan(theta/2) + h) for a cube viewcell of
 * half-size h (lateral radius r = h, plus h to enclose the cube's depth); phi = (theta+2 beta)/2;
 * exponential slices z_k = near * (far/near)^(k/D). Computed in binary64 on the host, rounded
 * once to binary32. Returns NPVS_ERR_INVALID_ARG for D outside [1, NPVS_MAX_SLICES] or
 * non-positive near / far <= near. */
npvs_status npvs_camera_setup(const npvs_viewcell* vc, int32_t n_slices, npvs_camera* out);

/* ---- a2: froxelization ---------------------------------------------------------------------- */

/* Workspace bytes npvs_froxelize needs for n_boxes boxes. */
size_t npvs_froxelize_workspace_bytes(int32_t n_boxes);

/* Sec. 3.2 froxelization with s x s supersampling per froxel column: for every supersampled
 * pixel (a, b) of batch element e and every face of e's boxes (front and back, no depth test),
 * the ray c' + t dir, dir = fwd + (n_x tan) right + (n_y tan) up, n_x = (2a+1-sW)/(sW),
 * hits the face plane P at t = (P - c'_i)/dir_i; if the other two coordinates lie in the closed
 * face rectangle and slices[0] <= t < slices[D], bit (a/s, b/s, max{k: slices[k] <= t}) is set.
 * Every operation is one binary32 operation with round-to-nearest in that order, so the
 * result is bit-exact.
 *  boxes: device float [n_boxes][6] (min xyz, max xyz); box_offsets: device int32 [B+1], element
 *  e owns boxes [box_offsets[e], box_offsets[e+1]); cams: device npvs_camera [B] with
 *  n_slices == grid.D; occ_bits: device, zeroed and written here.
 *  Errors: W % 32 != 0, D > NPVS_MAX_SLICES, s < 1 or s > 16, s*W or s*H > 65536, workspace too
 *  small. */
npvs_status npvs_froxelize(const float* boxes, const int32_t* box_offsets, int32_t n_boxes,
                           const npvs_camera* cams, npvs_grid grid, int32_t supersample,
                           uint32_t* occ_bits, void* workspace, size_t workspace_bytes, void* stream);

/* Pruning (Sec. 3.2: the PVS culls occlusion at once, since a fragment that falls in a froxel the
 * PVS leaves empty can be discarded; Sec. 5.6: the temporal bounding volume of a dynamic object is
 * froxelized and the object is dropped when none of its froxels is visible). visible[i] = 1 iff
 * box i, froxelized alone by the rule of npvs_froxelize (same rays, same binary32 rounding), sets
 * at least one froxel whose bit is set in pvs_bits of the box's batch element; else 0. The boxes
 * may be the scene's primitives or bounding volumes of moving objects.
 *  boxes, box_offsets, cams, grid, supersample: as npvs_froxelize; pvs_bits: device
 *  [B][D][H][W/32] (for example npvs_deinterleave's output); visible: device uint8 [n_boxes],
 *  written here (boxes outside [box_offsets[0], box_offsets[B]) get 0). Workspace:
 *  npvs_froxelize_workspace_bytes(n_boxes). Errors: as npvs_froxelize, NULL pvs_bits / visible. */
npvs_status npvs_prune(const float* boxes, const int32_t* box_offsets, int32_t n_boxes,
                       const npvs_camera* cams, npvs_grid grid, int32_t supersample,
                       const uint32_t* pvs_bits, uint8_t* visible, void* workspace,
                       size_t workspace_bytes, void* stream);

/* ---- a3: interleave / a7: de-interleave ------------------------------------------------------ */

size_t npvs_interleave_workspace_bytes(npvs_grid grid, int32_t d);

/* Sec. 3.3 g_d on the sparse grid: the coarse site (X, Y, Z) of batch b is active iff any of its
 * d^3 froxels is occupied; active sites are compacted in linear order into coords and their
 * in_ch * d^3 features (layout above) are written as feat_dtype (F32 or BF16; the depth value is
 * the binary32 quotient (2k+1)/(2D), rounded to nearest-even for BF16). d must divide 32, W, H
 * and D. n_active (device) receives min(count, capacity); overflow sets NPVS_ERR_CAPACITY in
 * status. table (device [B*(D/d)*(H/d)*(W/d)], nullable) receives each site's row or -1. */
npvs_status npvs_interleave(const uint32_t* occ_bits, npvs_grid grid, int32_t d, int32_t in_ch,
                            int32_t feat_dtype, int32_t capacity, int32_t* coords, void* feats,
                            int32_t* n_active, int32_t* table, int32_t* status, void* workspace,
                            size_t workspace_bytes, void* stream);

/* npvs_interleave for callers that cannot allocate device memory (the paper has no counterpart;
 * this is an interface convenience). Same arguments and results as npvs_interleave, without the
 * workspace: the scratch lives in a fixed 128 KiB array inside the library's device memory, which
 * every GPU that loads the library keeps until the process exits. Meant for callers that must not
 * allocate or free device memory, e.g. an engine that reserves its whole GPU heap at start-up, or code
 * on a frame's critical path where cudaMalloc / cudaFree (which may synchronise the device) is not
 * allowed. It allocates nothing itself.
 *  - Limit: B * (W/d) * (H/d) * (D/d) <= 4,194,304 coarse sites; larger grids return
 *    NPVS_ERR_UNSUPPORTED with a message (use npvs_interleave and a workspace).
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with that
 *    device current; make that first call before any stream capture on the device. The address is
 *    cached per device and per CUDA context: after a device reset (cudaDeviceReset, which replaces
 *    the primary context) the next call looks it up again, so that call too belongs before any
 *    capture.
 *  - All calls on a device share the one array and it keeps the last call's contents; no part of it
 *    needs to start at zero (each call rewrites what it reads), but calls that overlap on the GPU (e.g.
 *    from two streams at once) race on it and must be serialised by the caller. */
npvs_status npvs_interleave_noalloc(const uint32_t* occ_bits, npvs_grid grid, int32_t d, int32_t in_ch,
                                    int32_t feat_dtype, int32_t capacity, int32_t* coords, void* feats,
                                    int32_t* n_active, int32_t* table, int32_t* status, void* stream);

/* Sec. 3.3 g_d^-1 with the Sec. 3.1 threshold and the Sec. 3.2 mask: for every froxel, p =
 * sigmoid(logit) of its site's channel (0 for inactive sites) in binary32 (CUDA expf);
 * pvs bit = (p >= tau) AND mask bit. logits: device float [cap][d^3]; table: level-0 table;
 * mask_bits / pvs_bits: froxel bits; probs_out (nullable) device float [cap][d^3] receives p for
 * rows < n_active. */
npvs_status npvs_deinterleave(const float* logits, const int32_t* table, const int32_t* n_active,
                              npvs_grid grid, int32_t d, float tau, const uint32_t* mask_bits,
                              uint32_t* pvs_bits, float* probs_out, int32_t capacity, void* stream);

/* ---- a4: rulebooks ------------------------------------------------------------------------- */

size_t npvs_rulebook_workspace_bytes(npvs_dims dims);

/* SUBM3 (out_level, map2 unused): fills in->table from in->coords (-1 elsewhere) and writes the
 * neighbour map map [in->capacity][27]: entry k of row n is the row of site coords[n] + offset_k
 * or -1 (absent or outside the grid).
 * SUBM3_TABLE: the same neighbour map, with in->table already filled for every site of the level
 * (as npvs_interleave's table output and a DOWN2 rulebook's out->table are).
 * DOWN2: from in->table builds the parent level: out->coords / out->n_rows / out->table for the
 * sites {floor(p/2)} in linear order (out->dims must be in->dims halved; all even), map
 * [out->capacity][8] = rows of each parent's children (tap (cz*2+cy)*2+cx, -1 if absent), and
 * map2 [in->capacity] = parent_row*8 + tap of every fine row (the up map). Overflow of
 * out->capacity sets NPVS_ERR_CAPACITY in status.
 * DOWN3 (Sec. 2.3: a sparse convolution whose outputs dilate onto the neighbours of active sites;
 * here a 3x3x3 kernel, stride 2, padding 1): the same
 * from in->table for the dilated output set {q : some 2q + k - 1 active, k in {0,1,2}^3} in linear
 * order (out->dims = in->dims halved), map [out->capacity][27] = the input row of 2q + k - 1 for tap
 * k = (kz*3 + ky)*3 + kx (-1 if absent) and map2 [in->capacity][27] = for every fine row p and tap
 * k the output row q with p = 2q + k - 1 (-1 if none): the map of the transposed convolution. */
npvs_status npvs_build_rulebook(int32_t kind, const npvs_level* in, const npvs_level* out,
                                int32_t* map, int32_t* map2, int32_t* status, void* workspace,
                                size_t workspace_bytes, void* stream);

/* ---- a5/a6: sparse convolution ------------------------------------------------------------- */

/* Bytes of the BF16 convolution workspace for this convolution (split-K region, plus for SUBM3 /
 * DOWN2 / UP2 / DOWN3 / UP3 the FP32 product tiles T of cap_in x taps x cout, taps 27 / 8 / 8 / 27
 * / 27). NULL: the split-K region only. */
size_t npvs_conv_workspace_bytes(const npvs_conv_desc* desc);

/* Bytes of a packed BF16 weight tensor for a forward conv of this shape. */
size_t npvs_packed_weight_bytes(int32_t kind, int32_t cin, int32_t cout);

/* Packs FP32 weights [taps][cin][cout] (device) into the BF16 tensor-core layout (device,
 * npvs_packed_weight_bytes) with round-to-nearest-even. */
npvs_status npvs_pack_weights(int32_t kind, int32_t cin, int32_t cout, const float* w,
                              void* packed, void* stream);

/* One weight tensor of npvs_pack_weights_many: FP32 [taps][cin][cout] (device) of a (kind, cin,
 * cout) convolution, packed into `packed` (device) as
 *  - transposed = 0: the forward image, exactly as npvs_pack_weights (npvs_packed_weight_bytes);
 *  - transposed = 1: the image of the convolution that the BF16 backward's dgrad runs (input and
 *    output channels swapped; SUBM3 with the taps reversed, DOWN2 <-> UP2, DOWN3 <-> UP3, HEAD1),
 *    npvs_packed_weight_bytes_transposed bytes, for npvs_conv_desc.w_transposed. */
typedef struct {
    int32_t kind, cin, cout, transposed;
    const float* w;
    void* packed;
} npvs_pack_job;

/* Bytes of the transposed image of a (kind, cin, cout) convolution's weights (0 when cin or cout
 * is not a multiple of 8: that backward is not on the tensor cores). */
size_t npvs_packed_weight_bytes_transposed(int32_t kind, int32_t cin, int32_t cout);

/* Packs n weight tensors (host array of jobs) in one launch per 24 jobs (round to nearest even,
 * the layouts of npvs_pack_weights): after an optimizer step, every forward and dgrad image of a
 * network at once. All jobs are checked before the first launch (NPVS_ERR_INVALID_ARG for a NULL
 * pointer or a non-positive size, NPVS_ERR_UNSUPPORTED for an unknown kind or a transposed image
 * of a convolution whose cin or cout is not a multiple of 8); n = 0 launches nothing. */
npvs_status npvs_pack_weights_many(int32_t n, const npvs_pack_job* jobs, void* stream);

/* y = act(b + conv(x)) (+ skip); see npvs_conv_desc. bias (nullable): [cout], FP32, or FP64 with
 * dtype F64. Output-stationary: every output row is written exactly once (no atomics); rows >=
 * *n_out are not touched. */
npvs_status npvs_sparse_conv_fwd(const npvs_conv_desc* desc, const void* x, const void* w,
                                 const void* bias, const void* skip, void* y, void* stream);

/* ---- a1-a7 as one call: the whole frame -------------------------------------------------- */

/* One layer of a network for npvs_forward, in canonical order (a plain SubM3 stack, or a U-Net:
 * stem, per level SubM3 layers and a DOWN2, then per decoder level an UP2 whose output gets the
 * output of the layer just before the matching DOWN2 added after its ReLU, SubM3 layers, and a
 * HEAD1 with d^3 outputs). A U-Net may use the k = 3 stride-2 pair instead (DOWN3 / UP3 in place
 * of every DOWN2 / UP2, each coarser level then being the dilated output set of a DOWN3
 * rulebook); the two pairs cannot be mixed in one network (NPVS_ERR_UNSUPPORTED), and such a
 * network has no layer chain. tune_*: as npvs_conv_desc (0 = defaults). */
typedef struct {
    int32_t kind, cin, cout, relu;
    const void* w;     /* device: BF16 packed image (npvs_pack_weights) or F32 [taps][cin][cout] */
    const float* bias; /* device [cout], nullable */
    int32_t tune_stages, tune_max_split, tune_lag, tune_gather, tune_gather_warps, tune_form;
} npvs_layer;

/* A frame plan: froxel grid (batch = number of viewcells), interleave factor d, input channels
 * (1 occupancy, 2 + depth), supersampling, dtype (BF16 or F32), threshold tau, the largest box
 * count of a call, level capacities in permille of each level's sites (0 = all sites: no overflow
 * possible), the layers (host array), and chain_level:
 *  - 0: every layer is its own launch (npvs_sparse_conv_fwd with the layer's tune fields);
 *  - k >= 1: the down conv into level k, every layer below it and the up conv out of it run as one
 *    persistent cooperative launch (one CTA per SM, grid-wide barriers between phases) in the
 *    product form (a tcgen05 GEMM T = x [W_0 | W_1 | ...], then the gather-reduce over existing
 *    neighbours in fixed tap order), bitwise equal to those layers launched one by one in the
 *    product form (tune_form 2). Their tune fields are not used. Needs BF16, cin % 32 == 0 and
 *    cout % 16 == 0 for each of those layers and at most 24 of them (else NPVS_ERR_UNSUPPORTED).
 *    A timed-out wait in it reports NPVS_ERR_TIMEOUT; the workspace must then be zero-filled again. */
typedef struct {
    npvs_grid grid;
    int32_t d, in_ch, supersample, dtype;
    float tau;
    int32_t max_boxes;
    int32_t capacity_permille;
    int32_t n_layers;
    const npvs_layer* layers;
    int32_t chain_level;
} npvs_net_desc;

/* Bytes of the npvs_forward workspace of a plan (0 if the plan is invalid). The workspace must be
 * zero-filled before its first use (it holds the convolutions' split-K counters and the layer
 * chain's barrier words, which every call leaves at zero again). */
size_t npvs_forward_workspace_bytes(const npvs_net_desc* net);

/* The whole per-frame path (Sec. 3.1-3.3): npvs_froxelize -> npvs_interleave -> neighbour maps and
 * down-sampling rulebooks of every level -> every layer (npvs_sparse_conv_fwd) -> npvs_deinterleave
 * (sigmoid, tau, AND G). Inputs as npvs_froxelize (boxes, box_offsets [B+1], cams [B], all
 * device); outputs occ_bits (G) and pvs_bits [B][D][H][W/32], probs (nullable, [cap0][d^3] FP32 per
 * level-0 row). All buffers (levels, rulebooks, activations, scratch) are carved from workspace in a
 * fixed layout; nothing is allocated; the sequence can be captured in a CUDA graph. The rulebooks of
 * the coarser levels are built on a library-owned second stream of the device (created by the first
 * call that is not inside a stream capture; a capturing first call keeps one stream), forked from
 * and joined back into `stream` within the call, so they overlap the level-0 layers; the results do
 * not depend on it (calls from several host threads enqueue their fork and join one at a time).
 * Calls sharing one workspace must not overlap. */
npvs_status npvs_forward(const npvs_net_desc* net, const float* boxes, const int32_t* box_offsets,
                         int32_t n_boxes, const npvs_camera* cams, uint32_t* occ_bits, uint32_t* pvs_bits,
                         float* probs, int32_t* status, void* workspace, size_t workspace_bytes,
                         void* stream);

/* Where npvs_forward keeps layer `layer`'s output rows (layer -1: the interleaved input features) in
 * a workspace: *rows (device [capacity][C], dtype; FP32 for the last layer), the level's capacity
 * and its device row count. Host-only: reads nothing from the device. */
npvs_status npvs_forward_layer_output(const npvs_net_desc* net, int32_t layer, void* workspace, void** rows,
                                      int32_t* capacity, int32_t** n_rows);

/* ---- training targets: ground-truth PVS (Sec. 3.2) ---------------------------------------- */

/* From-region visibility by ray casting: for each viewpoint p_m of batch element e (device
 * float [B][n_points][3], world positions outside every box) and each pixel of the (s_gt W) x
 * (s_gt H) raster of cams[e]'s directions (as npvs_froxelize), the nearest box hit t > 0 of
 * p_m + t dir is reprojected into cams[e]'s frame; a hit inside the frustum sets its froxel in
 * gt_bits [B][D][H][W/32] (zeroed here). With g_bits (nullable) the result is ANDed with the
 * geometry grid. Binary32 arithmetic, each step rounded to nearest in a fixed order (slab entry
 * t* = max(0, max_i min(t0_i, t1_i)) with t_i = (bound_i - p_i) * (1 / dir_i); v_i = (p_i + t* dir_i)
 * - c'_i; x_c = (v_0 r_0 + v_1 r_1) + v_2 r_2 and likewise y_c, z_c; x = min(floor((((x_c / z_c) /
 * tan) + 1) * 0.5 * W), W - 1)), so the bits are reproducible exactly by a binary32 program.
 * n_points * s_gt^2 * W * H must be a multiple of 256. */
npvs_status npvs_gt_raycast(const float* boxes, const int32_t* box_offsets, const npvs_camera* cams,
                            const float* points, int32_t n_points, npvs_grid grid, int32_t s_gt,
                            const uint32_t* g_bits, uint32_t* gt_bits, void* stream);

/* ---- a10: sparse convolution backward ---------------------------------------------------- */

/* Bytes of the workspace of npvs_sparse_conv_bwd for this convolution (the gradient g of the
 * pre-activation, fixed-order partial sums of dW and db, the transposed weights and, for BF16,
 * the workspace of the transposed forward convolution that computes dx). */
size_t npvs_conv_bwd_workspace_bytes(const npvs_conv_desc* desc);

/* Backward of npvs_sparse_conv_fwd with the same desc (Sec. 2.3 layers; gradients of the masked
 * dense definition). With g = dy * 1[y > 0] (g = dy without ReLU):
 *   db = sum_n g[n],   dW_t = sum_n x[map(n, t)]^T g[n],   dx = transposed convolution of g (+ dx_add)
 *  x:      the forward input [cap_in][cin] (dtype; rows < n_in).
 *  w:      master weights [taps][cin][cout]: FP32 for F32 and BF16, FP64 for F64 (not packed).
 *  y:      the layer's output after ReLU and before a skip addition [cap_out][cout] (dtype);
 *          read only with relu (NULL otherwise). ReLU with out_f32 is unsupported.
 *  dy:     gradient of the output [cap_out][cout] (dtype, also for an out_f32 layer).
 *  dx:     nullable [cap_in][cin] (dtype): gradient of x, rows < n_in written. dx_add (nullable,
 *          same shape) is added to it: a gradient reaching x by another path (a skip).
 *  dw, db: FP32 (FP64 for F64) [taps][cin][cout] and [cout], overwritten; db nullable.
 *  The stride-2 kinds (DOWN2, UP2, DOWN3, UP3) need map2 (the other map of the level pair), n_in and
 *  cap_in for dx: the dgrad of DOWN2 / DOWN3 is the UP2 / UP3 convolution of g with W_t^T on the same
 *  rulebook, and the other way round.
 *  Sums are taken in a fixed order: results are bitwise reproducible for the same capacities.
 *  desc->workspace is not used; workspace must hold npvs_conv_bwd_workspace_bytes(desc). */
npvs_status npvs_sparse_conv_bwd(const npvs_conv_desc* desc, const void* x, const void* w, const void* y,
                                 const void* dy, void* dx, const void* dx_add, void* dw, void* db,
                                 void* workspace, size_t workspace_bytes, void* stream);

/* ---- a8/a9: weighted Dice + repulsive visibility loss (Sec. 3.3) -------------------------- */

/* Readings of Sec. 3.3 (the prose and printed formulas disagree on FN / FP): with y the ground
 * truth bit, g the geometry bit and p~ = sigmoid(z) g per froxel of a sample,
 *   TP = sum y p~, FP = sum (1-y) p~, GTP = popcount(GT), FN = GTP - TP, NOCC = sum g,
 *   dice = 1 - (2TP + eps) / (2TP + alpha FN + (1-alpha) FP + eps)
 *   attr = FN / (GTP + eps), rep = FP / (GTP + eps), bce = sum_g BCE-with-logits / NOCC (w_bce != 0)
 *   L_b = lam dice + (1 - lam)(attr + rep) + w_bce bce, and the loss is the mean of L_b over the batch.
 * Defaults: alpha 0.9, eps 1, lam 0.99 (Sec. 4.2), w_bce 0. */
typedef struct {
    double alpha, eps, lam, w_bce;
} npvs_loss_params;

#define NPVS_LOSS_TERMS 12
enum {
    NPVS_LT_L = 0, NPVS_LT_DICE = 1, NPVS_LT_ATTR = 2, NPVS_LT_REP = 3, NPVS_LT_BCE = 4, NPVS_LT_GTP = 5,
    NPVS_LT_TP = 6, NPVS_LT_FN = 7, NPVS_LT_FP = 8, NPVS_LT_NOCC = 9,
    NPVS_LT_DTP = 10, /* dLoss/dTP of the batch mean */
    NPVS_LT_DFP = 11  /* dLoss/dFP of the batch mean */
};

/* Bytes of the npvs_loss_fwd workspace for `capacity` rows of logits of this dtype (F32 / F64). */
size_t npvs_loss_workspace_bytes(int32_t capacity, int32_t dtype);

/* Loss of the logits z [capacity][d^3] (dtype F32 or F64; rows < *n_rows, coarse sites `coords`
 * of the interleaved level, channel order as the interleave) against the ground-truth and
 * geometry grids gt_bits / g_bits [B][D][H][W/32] of `grid`. Writes terms [B][NPVS_LOSS_TERMS]
 * and the scalar loss (device, dtype). Sums are fixed-order (bitwise reproducible). */
npvs_status npvs_loss_fwd(int32_t dtype, const void* logits, const int32_t* coords, const int32_t* n_rows,
                          int32_t capacity, const uint32_t* gt_bits, const uint32_t* g_bits, npvs_grid grid,
                          int32_t d, const npvs_loss_params* prm, void* terms, void* loss, void* workspace,
                          size_t workspace_bytes, void* stream);

/* dLoss/dz from the terms of npvs_loss_fwd, times the device scalar dloss (dtype; NULL = 1):
 * dz = g (p(1-p)(y dL/dTP + (1-y) dL/dFP) + w_bce (p - y) / (B NOCC)). Rows < *n_rows written, in
 * dlogits_dtype: F32 or BF16 for F32 logits (BF16 feeds the tensor-core backward), F64 for F64. */
npvs_status npvs_loss_bwd(int32_t dtype, const void* logits, const int32_t* coords, const int32_t* n_rows,
                          int32_t capacity, const uint32_t* gt_bits, const uint32_t* g_bits, npvs_grid grid,
                          int32_t d, const npvs_loss_params* prm, const void* terms, const void* dloss,
                          int32_t dlogits_dtype, void* dlogits, void* stream);

/* ---- a11: Adam (Sec. 4.2) ----------------------------------------------------------------- */

/* Paper: Adam, lr 1e-3, "decay 1e-10" (read as L2 weight decay added to the gradient); betas and
 * eps unspecified (0.9, 0.999, 1e-8). */
typedef struct {
    float lr, beta1, beta2, eps, weight_decay;
} npvs_adam_params;

/* One Adam step on n FP32 master parameters (all device): g = grad + wd theta, m and v updated,
 * theta -= lr mhat / (sqrt(vhat) + eps) with bias corrections of step t. state: device int32[2],
 * zero before the first step; state[0] counts the steps taken (t = state[0] + 1 is used and stored
 * back by the last CTA), state[1] is scratch. Replaying a captured step advances t. */
npvs_status npvs_adam_step(float* theta, const float* grad, float* m, float* v, int64_t n,
                           const npvs_adam_params* prm, int32_t* state, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* NPVS_H */
