// tcgen05 (5th-generation tensor core) BF16 sparse convolution: launcher and weight packing.
#pragma once
#include "common.cuh"

namespace npvs {

// Convolutions whose map lists the input row of each of 27 taps per output row ([rows][27]).
__host__ __device__ __forceinline__ bool map27(int kind) {
    return kind == NPVS_CONV_SUBM3 || kind == NPVS_CONV_DOWN3 || kind == NPVS_CONV_UP3;
}

__host__ __device__ __forceinline__ int conv_taps(int kind) {
    return map27(kind) ? 27 : (kind == NPVS_CONV_HEAD1 ? 1 : 8);
}

inline bool valid_conv_kind(int kind) { return kind >= NPVS_CONV_SUBM3 && kind <= NPVS_CONV_UP3; }

// Input row feeding output row n through tap t (-1: none).
__device__ __forceinline__ int gather_row(int kind, const int32_t* __restrict__ map, int n, int t) {
    switch (kind) {
        case NPVS_CONV_SUBM3:
        case NPVS_CONV_DOWN3:
        case NPVS_CONV_UP3: return map[(size_t)n * 27 + t];
        case NPVS_CONV_DOWN2: return map[(size_t)n * 8 + t];
        case NPVS_CONV_UP2: {
            int u = map[n];
            return (u >= 0 && (u & 7) == t) ? (u >> 3) : -1;
        }
        default: return n;
    }
}

// BF16 convolutions with cin or cout not a multiple of 8 run on a SIMT kernel (FP32 accumulation)
// with plain BF16 weights [taps][cin][cout] as their packed image, not on the tensor cores.
inline bool bf16_narrow(int cin, int cout) { return cin % 8 != 0 || cout % 8 != 0; }

// GEMM view of a convolution: rows x (Kflat = taps_eff * cin) x Ntot.
//   G-form (SUBM3, DOWN2, HEAD1, DOWN3, UP3): row = output row, k = tap * cin + ci, n = co.
//   S-form (UP2): row = coarse input row, k = ci, n = child_tap * cout + co; the epilogue scatters
//   column block child_tap to the child's row (down map).
struct TcShape {
    int form;  // 0: direct / transposed, 1: product form (T = x [W_0 | W_1 | ...])
    int J;     // column blocks of the GEMM (1, 8 for the transposed conv, taps for the product form)
    int taps_eff, Kflat, KB, Ntot, Npad, BN, n_tiles;
    int tma;  // gather with TMA tile::gather4 (cin % 32 == 0) instead of cp.async
    int BKE;  // k-block width in elements (64; 32 when cin is an odd multiple of 32)
    int RB;   // bytes of one k-block row (2 * BKE)
};

TcShape tc_shape(int kind, int cin, int cout, int form);

// Packs FP32 weights into the BF16 tensor-core image of a (kind, cin, cout) convolution; mode 1 / 2
// read them as the transpose of a stored (kind, cout, cin) convolution (2: with the taps
// reversed, the transpose of a submanifold convolution).
npvs_status pack_weights_mode(int kind, int cin, int cout, const float* w, void* packed, int mode, cudaStream_t st);

// The convolution whose forward is the dgrad of `kind` (input and output channels swapped), and the
// packing mode that reads the stored weights as its weights: the submanifold conv is its own
// transpose with the taps reversed (mode 2), the strided pairs and the head swap (mode 1).
inline int transposed_kind(int kind, int* mode) {
    *mode = kind == NPVS_CONV_SUBM3 ? 2 : 1;
    switch (kind) {
        case NPVS_CONV_SUBM3: return NPVS_CONV_SUBM3;
        case NPVS_CONV_DOWN2: return NPVS_CONV_UP2;
        case NPVS_CONV_UP2: return NPVS_CONV_DOWN2;
        case NPVS_CONV_DOWN3: return NPVS_CONV_UP3;
        case NPVS_CONV_UP3: return NPVS_CONV_DOWN3;
        default: return NPVS_CONV_HEAD1;
    }
}

// BF16 weight gradient on the tensor cores (dW FP32 [taps][cin][cout]) from the layer input x and
// the masked output gradient g; scratch from `ar` (wgrad_tc_bytes).
bool wgrad_tc_supported(const npvs_conv_desc& d);
size_t wgrad_tc_bytes(const npvs_conv_desc& d);
npvs_status wgrad_tc(const npvs_conv_desc& d, const __nv_bfloat16* x, const __nv_bfloat16* g, float* dw, Arena& ar,
                     cudaStream_t st);

npvs_status conv_tc_fwd(const npvs_conv_desc& d, const void* x, const void* w, const float* bias,
                        const void* skip, void* y, cudaStream_t st);

// The FP32 product tiles T [rows][J * cout] of a convolution in its workspace (the region
// npvs_conv_workspace_bytes() reserves), or nullptr when the workspace lacks them.
float* conv_product_tiles(const npvs_conv_desc& d);

}  // namespace npvs
