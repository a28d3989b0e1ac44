// Host interface of the persistent layer chain (chain.cu): a run of a frame's sparse convolutions
// executed by one cooperative launch.
#pragma once
#include "common.cuh"

namespace npvs {

constexpr int kChainMaxLayers = 24;

// One layer of a chain, as npvs_forward describes it (BF16, product form).
struct ChainLayerHost {
    int kind, cin, cout, relu;
    const void* x;        // [rows_x][cin] BF16
    const void* w;        // packed weights (npvs_pack_weights)
    const float* bias;    // [cout] or nullptr
    const void* skip;     // [cap_out][cout] BF16 added after ReLU, or nullptr
    void* y;              // [cap_out][cout] BF16
    const int32_t* map;   // SUBM3 neighbours, DOWN2 children, UP2 up map
    const int32_t* map2;  // which product rows the reduce reads: SUBM3 nullptr (map itself), DOWN2 the
                          // up map of the finer level, UP2 the down map [rows_x][8]
    const int32_t* n_in;  // device row counts of x and y
    const int32_t* n_out;
    int rows_x, cap_out;
};

// Kinds and shapes a chain runs: SUBM3, DOWN2 and UP2 with cin % 32 == 0 and cout % 16 == 0.
bool chain_layer_supported(int kind, int cin, int cout);

// Bytes of the FP32 product tiles T of one chain layer with rows_x input rows.
size_t chain_tiles_bytes(int kind, int cin, int cout, int rows_x);

// Enqueues the chain on `st`: T (T_bytes, the largest layer's tiles) and bar (two words, zero
// between launches; the kernel leaves them zero) come from the caller's workspace. Bounded waits
// raise NPVS_ERR_TIMEOUT in `status`.
npvs_status chain_launch(const ChainLayerHost* layers, int n_layers, float* T, size_t T_bytes, unsigned int* bar,
                         int32_t* status, cudaStream_t st);

}  // namespace npvs
