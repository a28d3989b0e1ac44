// npvs_forward: one whole frame of the path on the device (Sec. 3.1: V = g_d^-1(f_theta(g_d(G)))
// thresholded at tau and masked by G, with G the froxelized scene of the viewcell's enclosing
// frustum, Sec. 3.2), as one call over a caller-provided workspace.
//
// The call enqueues exactly the sequence a caller would make through the individual entry points:
// froxelize -> interleave (level-0 coords, features, table) -> per level the neighbour map from the
// prebuilt table and, between levels, the down-sampling rulebook -> every layer of the network ->
// de-interleave. Row counts stay on the device, so the call can be captured in a CUDA graph.
// Every buffer is carved from the workspace in a fixed order (npvs_forward_workspace_bytes), the
// library allocates nothing, and the activations of every layer stay readable in the workspace
// (npvs_forward_layer_output) for inspection or a following backward pass.
#include <cstring>
#include <vector>

#include <mutex>

#include "chain.cuh"
#include "common.cuh"
#include "conv_tc.cuh"

namespace npvs {
namespace {

struct FwdLevel {
    npvs_dims dims;
    int cap;
    int32_t *coords, *n_rows, *table, *nbr, *down, *up;
};

struct FwdPlan {
    int n_levels = 0;
    std::vector<int> level_of;  // output level of each layer
    std::vector<int> skip_of;   // layer whose output is added after this layer's ReLU (-1: none)
    std::vector<size_t> act_off;
    size_t el = 2;
    int chain_first = -1, chain_last = -1;  // layers run as one persistent launch (chain_level)
    bool k3 = false;  // the levels are linked by the k = 3 stride-2 pair (DOWN3 / UP3), not DOWN2 / UP2
};

npvs_status plan_net(const npvs_net_desc& n, FwdPlan* P) {
    NPVS_REQUIRE(n.layers && n.n_layers > 0, NPVS_ERR_INVALID_ARG, "npvs_forward: no layers");
    NPVS_REQUIRE(n.dtype == NPVS_BF16 || n.dtype == NPVS_F32, NPVS_ERR_UNSUPPORTED, "npvs_forward: dtype must be BF16 or F32");
    NPVS_REQUIRE(n.grid.W > 0 && n.grid.W % 32 == 0 && n.grid.H > 0 && n.grid.D > 0 && n.grid.B > 0, NPVS_ERR_INVALID_ARG,
                 "npvs_forward: bad grid");
    NPVS_REQUIRE(n.d >= 1 && 32 % n.d == 0 && n.grid.W % n.d == 0 && n.grid.H % n.d == 0 && n.grid.D % n.d == 0,
                 NPVS_ERR_UNSUPPORTED, "npvs_forward: d must divide 32, W, H and D");
    NPVS_REQUIRE(n.in_ch >= 1 && n.in_ch <= 2 && n.supersample >= 1 && n.max_boxes >= 0, NPVS_ERR_INVALID_ARG,
                 "npvs_forward: bad in_ch, supersample or max_boxes");
    P->level_of.assign(n.n_layers, 0);
    P->skip_of.assign(n.n_layers, -1);
    std::vector<int> stack;
    int lv = 0, maxlv = 0;
    bool seen_pair = false;
    for (int i = 0; i < n.n_layers; ++i) {
        const npvs_layer& l = n.layers[i];
        NPVS_REQUIRE(l.kind >= NPVS_CONV_SUBM3 && l.kind <= NPVS_CONV_UP3 && l.w, NPVS_ERR_INVALID_ARG,
                     "npvs_forward: bad layer");
        const int cin_expected = i == 0 ? n.in_ch * n.d * n.d * n.d : n.layers[i - 1].cout;
        NPVS_REQUIRE(l.cin == cin_expected, NPVS_ERR_INVALID_ARG, "npvs_forward: layer cin differs from the input width");
        const bool down = l.kind == NPVS_CONV_DOWN2 || l.kind == NPVS_CONV_DOWN3;
        const bool up = l.kind == NPVS_CONV_UP2 || l.kind == NPVS_CONV_UP3;
        if (down || up) {  // one pair for the whole network: the level sets follow from it
            const bool k3 = l.kind == NPVS_CONV_DOWN3 || l.kind == NPVS_CONV_UP3;
            NPVS_REQUIRE(!seen_pair || k3 == P->k3, NPVS_ERR_UNSUPPORTED,
                         "npvs_forward: the 2x2x2 and the k = 3 stride-2 pairs cannot be mixed");
            P->k3 = k3;
            seen_pair = true;
        }
        if (down) {
            stack.push_back(i - 1);
            ++lv;
        } else if (up) {
            NPVS_REQUIRE(!stack.empty() && lv > 0, NPVS_ERR_INVALID_ARG, "npvs_forward: up conv without a matching down conv");
            const int src = stack.back();
            stack.pop_back();
            --lv;
            NPVS_REQUIRE(src >= 0 && n.layers[src].cout == l.cout, NPVS_ERR_INVALID_ARG,
                         "npvs_forward: skip width differs from the up conv's output");
            P->skip_of[i] = src;
        }
        P->level_of[i] = lv;
        maxlv = std::max(maxlv, lv);
    }
    NPVS_REQUIRE(lv == 0 && n.layers[n.n_layers - 1].cout == n.d * n.d * n.d, NPVS_ERR_INVALID_ARG,
                 "npvs_forward: the network must end at level 0 with d^3 logits per site");
    P->n_levels = maxlv + 1;
    int X = n.grid.W / n.d, Y = n.grid.H / n.d, Z = n.grid.D / n.d;
    for (int li = 1; li < P->n_levels; ++li) {
        NPVS_REQUIRE(X % 2 == 0 && Y % 2 == 0 && Z % 2 == 0, NPVS_ERR_UNSUPPORTED,
                     "npvs_forward: every level above the last must have even dimensions");
        X /= 2;
        Y /= 2;
        Z /= 2;
    }
    P->el = n.dtype == NPVS_BF16 ? 2 : 4;
    if (n.chain_level > 0) {
        // the down conv into level chain_level ... the up conv out of it
        NPVS_REQUIRE(n.dtype == NPVS_BF16 && n.chain_level < P->n_levels, NPVS_ERR_UNSUPPORTED,
                     "npvs_forward: chain_level needs BF16 and a level below the top");
        for (int i = 0; i < n.n_layers && P->chain_first < 0; ++i)
            if (n.layers[i].kind == NPVS_CONV_DOWN2 && P->level_of[i] == n.chain_level) P->chain_first = i;
        for (int i = P->chain_first + 1; P->chain_first >= 0 && i < n.n_layers && P->chain_last < 0; ++i)
            if (n.layers[i].kind == NPVS_CONV_UP2 && P->level_of[i] == n.chain_level - 1) P->chain_last = i;
        NPVS_REQUIRE(P->chain_first >= 0 && P->chain_last > P->chain_first &&
                         P->chain_last - P->chain_first < kChainMaxLayers,
                     NPVS_ERR_UNSUPPORTED, "npvs_forward: no chain of at most 24 layers at chain_level");
        for (int i = P->chain_first; i <= P->chain_last; ++i)
            NPVS_REQUIRE(chain_layer_supported(n.layers[i].kind, n.layers[i].cin, n.layers[i].cout),
                         NPVS_ERR_UNSUPPORTED, "npvs_forward: a chained layer needs cin % 32 == 0 and cout % 16 == 0");
    }
    return NPVS_OK;
}

npvs_dims level_dims(const npvs_net_desc& n, int li) {
    npvs_dims d;
    d.X = (n.grid.W / n.d) >> li;
    d.Y = (n.grid.H / n.d) >> li;
    d.Z = (n.grid.D / n.d) >> li;
    d.B = n.grid.B;
    return d;
}

long long sites_of(const npvs_dims& d) { return (long long)d.X * d.Y * d.Z * d.B; }

int level_cap(const npvs_net_desc& n, int li) {
    const long long s = sites_of(level_dims(n, li));
    const long long c = n.capacity_permille > 0 ? (s * n.capacity_permille + 999) / 1000 : s;
    return (int)std::max<long long>(1, std::min(c, s));
}

npvs_conv_desc layer_desc(const npvs_net_desc& n, const FwdPlan& P, const std::vector<FwdLevel>& L, int i,
                          int32_t* status) {
    const npvs_layer& l = n.layers[i];
    const int li = P.level_of[i];
    npvs_conv_desc d;
    std::memset(&d, 0, sizeof(d));
    d.kind = l.kind;
    d.dtype = n.dtype;
    d.cin = l.cin;
    d.cout = l.cout;
    d.relu = l.relu;
    d.out_f32 = i == n.n_layers - 1;
    d.n_out = L[li].n_rows;
    d.cap_out = L[li].cap;
    d.status = status;
    d.tune_stages = l.tune_stages;
    d.tune_max_split = l.tune_max_split;
    d.tune_lag = l.tune_lag;
    d.tune_gather = l.tune_gather;
    d.tune_gather_warps = l.tune_gather_warps;
    d.tune_form = l.tune_form;
    if (l.kind == NPVS_CONV_SUBM3 || l.kind == NPVS_CONV_HEAD1) {
        d.map = l.kind == NPVS_CONV_SUBM3 ? L[li].nbr : nullptr;
        d.n_in = L[li].n_rows;
        d.cap_in = L[li].cap;
    } else if (l.kind == NPVS_CONV_DOWN2 || l.kind == NPVS_CONV_DOWN3) {  // the input rows of each output
        d.map = L[li - 1].down;
        d.map2 = L[li - 1].up;
        d.n_in = L[li - 1].n_rows;
        d.cap_in = L[li - 1].cap;
    } else {
        d.map = L[li].up;
        d.map2 = L[li].down;
        d.n_in = L[li + 1].n_rows;
        d.cap_in = L[li + 1].cap;
    }
    return d;
}

// Carves the workspace; with base == nullptr only sizes it. Returns the bytes used.
size_t carve(const npvs_net_desc& n, FwdPlan& P, void* base, size_t size, std::vector<FwdLevel>& L, void** feats,
             std::vector<void*>& acts, void** conv_ws, size_t* conv_ws_bytes, void** scratch, size_t* scratch_bytes,
             unsigned int** chain_bar = nullptr) {
    Arena ar(base, base ? size : 0);
    unsigned int* cb = ar.take<unsigned int>(2);  // the layer chain's grid-barrier words
    if (chain_bar) *chain_bar = cb;
    L.assign(P.n_levels, FwdLevel());
    for (int li = 0; li < P.n_levels; ++li) {
        FwdLevel& v = L[li];
        v.dims = level_dims(n, li);
        v.cap = level_cap(n, li);
        v.coords = ar.take<int32_t>((size_t)v.cap * 4);
        v.n_rows = ar.take<int32_t>(1);
        v.table = ar.take<int32_t>((size_t)sites_of(v.dims));
        v.nbr = ar.take<int32_t>((size_t)v.cap * 27);
        v.down = v.up = nullptr;
    }
    for (int li = 0; li + 1 < P.n_levels; ++li) {  // k = 3 pair: 27 taps each way
        L[li].down = ar.take<int32_t>((size_t)L[li + 1].cap * (P.k3 ? 27 : 8));
        L[li].up = ar.take<int32_t>((size_t)L[li].cap * (P.k3 ? 27 : 1));
    }
    *feats = ar.take<char>((size_t)L[0].cap * n.in_ch * n.d * n.d * n.d * P.el);
    acts.assign(n.n_layers, nullptr);
    for (int i = 0; i < n.n_layers; ++i) {
        const size_t el = i == n.n_layers - 1 ? 4 : P.el;
        acts[i] = ar.take<char>((size_t)L[P.level_of[i]].cap * n.layers[i].cout * el);
    }
    size_t cw = 0;
    if (n.dtype == NPVS_BF16 || n.dtype == NPVS_F32) {
        for (int i = 0; i < n.n_layers; ++i) {
            npvs_conv_desc d = layer_desc(n, P, L, i, nullptr);
            cw = std::max(cw, npvs_conv_workspace_bytes(&d));
        }
    }
    *conv_ws_bytes = cw;
    *conv_ws = cw ? ar.take<char>(cw) : nullptr;
    size_t sb = npvs_froxelize_workspace_bytes(std::max(n.max_boxes, 1));
    sb = std::max(sb, npvs_interleave_workspace_bytes(n.grid, n.d));
    for (int li = 0; li + 1 < P.n_levels; ++li) sb = std::max(sb, npvs_rulebook_workspace_bytes(L[li + 1].dims));
    *scratch_bytes = sb;
    *scratch = ar.take<char>(sb);
    return ar.used + 256;
}

}  // namespace
}  // namespace npvs

using namespace npvs;

extern "C" size_t npvs_forward_workspace_bytes(const npvs_net_desc* net) {
    if (!net) return 0;
    FwdPlan P;
    if (plan_net(*net, &P) != NPVS_OK) return 0;
    std::vector<FwdLevel> L;
    std::vector<void*> acts;
    void *feats, *cw, *sc;
    size_t cwb, scb;
    return carve(*net, P, nullptr, 0, L, &feats, acts, &cw, &cwb, &sc, &scb);
}

// One library-owned side stream and two events per device (created on first use, never inside a
// stream capture: a capturing call that finds none keeps everything on the caller's stream).
struct SideStream {
    bool ok = false;
    cudaStream_t stream = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    std::mutex* order = nullptr;  // held from the fork record to the join wait of one call
};

SideStream side_stream(cudaStream_t st) {
    static std::mutex mu;
    static std::mutex order[64];
    static SideStream per_dev[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SideStream();
    std::lock_guard<std::mutex> lock(mu);
    SideStream& s = per_dev[dev];
    if (s.ok) return s;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return SideStream();
    if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess) return SideStream();
    if (cudaEventCreateWithFlags(&s.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return SideStream();
    }
    s.order = &order[dev];
    s.ok = true;
    return s;
}

extern "C" npvs_status npvs_forward(const npvs_net_desc* net, const float* boxes, const int32_t* box_offsets,
                                    int32_t n_boxes, const npvs_camera* cams, uint32_t* occ_bits, uint32_t* pvs_bits,
                                    float* probs, int32_t* status, void* workspace, size_t workspace_bytes,
                                    void* stream) {
    NPVS_REQUIRE(net && boxes && box_offsets && cams && occ_bits && pvs_bits, NPVS_ERR_INVALID_ARG,
                 "npvs_forward: NULL argument");
    const npvs_net_desc& n = *net;
    FwdPlan P;
    NPVS_TRY(plan_net(n, &P));
    NPVS_REQUIRE(n_boxes <= n.max_boxes, NPVS_ERR_INVALID_ARG, "npvs_forward: more boxes than the plan's max_boxes");
    std::vector<FwdLevel> L;
    std::vector<void*> acts;
    void *feats, *cw, *sc;
    size_t cwb, scb;
    const size_t need = carve(n, P, nullptr, 0, L, &feats, acts, &cw, &cwb, &sc, &scb);
    NPVS_REQUIRE(workspace && workspace_bytes >= need, NPVS_ERR_WORKSPACE,
                 "npvs_forward: workspace smaller than npvs_forward_workspace_bytes()");
    unsigned int* chain_bar = nullptr;
    carve(n, P, workspace, workspace_bytes, L, &feats, acts, &cw, &cwb, &sc, &scb, &chain_bar);
    cudaStream_t st = as_stream(stream);

    NPVS_TRY(npvs_froxelize(boxes, box_offsets, n_boxes, cams, n.grid, n.supersample, occ_bits, sc, scb, st));
    NPVS_TRY(npvs_interleave(occ_bits, n.grid, n.d, n.in_ch, n.dtype, L[0].cap, L[0].coords, feats, L[0].n_rows,
                             L[0].table, status, sc, scb, st));
    {
        npvs_level lv = {L[0].dims, L[0].cap, L[0].coords, L[0].n_rows, L[0].table};
        NPVS_TRY(npvs_build_rulebook(NPVS_RB_SUBM3_TABLE, &lv, nullptr, L[0].nbr, nullptr, status, sc, scb, st));
    }
    // The rulebooks of the coarser levels depend only on the level-0 sites: they are built on a
    // second stream while the level-0 convolutions run (those use the convolution workspace, the
    // rulebooks the scratch region), and the caller's stream waits for them before the first layer
    // that reads a coarser level.
    SideStream side = side_stream(st);
    cudaStream_t rs = side.ok ? side.stream : st;
    // calls from several host threads share the device's events: one call's fork ... join at a time
    std::unique_lock<std::mutex> in_order;
    if (side.ok) in_order = std::unique_lock<std::mutex>(*side.order);
    if (side.ok && P.n_levels > 1) {
        if (cudaEventRecord(side.fork, st) != cudaSuccess || cudaStreamWaitEvent(rs, side.fork, 0) != cudaSuccess)
            return check_launch("npvs_forward: fork");
    }
    for (int li = 0; li + 1 < P.n_levels; ++li) {
        npvs_level lv = {L[li].dims, L[li].cap, L[li].coords, L[li].n_rows, L[li].table};
        npvs_level nx = {L[li + 1].dims, L[li + 1].cap, L[li + 1].coords, L[li + 1].n_rows, L[li + 1].table};
        NPVS_TRY(npvs_build_rulebook(P.k3 ? NPVS_RB_DOWN3 : NPVS_RB_DOWN2, &lv, &nx, L[li].down, L[li].up, status, sc,
                                     scb, rs));
        NPVS_TRY(npvs_build_rulebook(NPVS_RB_SUBM3_TABLE, &nx, nullptr, L[li + 1].nbr, nullptr, status, sc, scb, rs));
    }
    bool joined = !(side.ok && P.n_levels > 1);
    if (!joined && cudaEventRecord(side.join, rs) != cudaSuccess) return check_launch("npvs_forward: join");
    const void* a = feats;
    for (int i = 0; i < n.n_layers; ++i) {
        const bool level0_only =
            P.level_of[i] == 0 && (n.layers[i].kind == NPVS_CONV_SUBM3 || n.layers[i].kind == NPVS_CONV_HEAD1);
        if (!joined && !level0_only) {  // the first layer that reads a coarser level's rulebooks
            if (cudaStreamWaitEvent(st, side.join, 0) != cudaSuccess) return check_launch("npvs_forward: join");
            joined = true;
        }
        if (i == P.chain_first) {  // the chained layers, one persistent launch
            ChainLayerHost cl[kChainMaxLayers];
            float* T = nullptr;
            for (int j = i; j <= P.chain_last; ++j) {
                npvs_conv_desc d = layer_desc(n, P, L, j, status);
                d.workspace = cw;
                d.workspace_bytes = cwb;
                if (!T) T = conv_product_tiles(d);
                ChainLayerHost& h = cl[j - i];
                h.kind = d.kind;
                h.cin = d.cin;
                h.cout = d.cout;
                h.relu = d.relu;
                h.x = a;
                h.w = n.layers[j].w;
                h.bias = n.layers[j].bias;
                h.skip = P.skip_of[j] >= 0 ? acts[P.skip_of[j]] : nullptr;
                h.y = acts[j];
                h.map = d.map;
                h.map2 = d.map2;
                h.n_in = d.n_in;
                h.n_out = d.n_out;
                h.rows_x = d.cap_in;
                h.cap_out = d.cap_out;
                a = acts[j];
            }
            NPVS_REQUIRE(T != nullptr, NPVS_ERR_WORKSPACE, "npvs_forward: no product tiles for the layer chain");
            const size_t T_bytes = (size_t)((const char*)cw + cwb - (const char*)T);
            NPVS_TRY(chain_launch(cl, P.chain_last - i + 1, T, T_bytes, chain_bar, status, st));
            i = P.chain_last;
            continue;
        }
        npvs_conv_desc d = layer_desc(n, P, L, i, status);
        d.workspace = cw;
        d.workspace_bytes = cwb;
        const void* skip = P.skip_of[i] >= 0 ? acts[P.skip_of[i]] : nullptr;
        NPVS_TRY(npvs_sparse_conv_fwd(&d, a, n.layers[i].w, n.layers[i].bias, skip, acts[i], st));
        a = acts[i];
    }
    if (!joined && cudaStreamWaitEvent(st, side.join, 0) != cudaSuccess) return check_launch("npvs_forward: join");
    return npvs_deinterleave((const float*)acts[n.n_layers - 1], L[0].table, L[0].n_rows, n.grid, n.d, n.tau, occ_bits,
                             pvs_bits, probs, L[0].cap, st);
}

extern "C" npvs_status npvs_forward_layer_output(const npvs_net_desc* net, int32_t layer, void* workspace,
                                                 void** rows, int32_t* capacity, int32_t** n_rows) {
    NPVS_REQUIRE(net && workspace && rows, NPVS_ERR_INVALID_ARG, "npvs_forward_layer_output: NULL argument");
    FwdPlan P;
    NPVS_TRY(plan_net(*net, &P));
    NPVS_REQUIRE(layer >= -1 && layer < net->n_layers, NPVS_ERR_INVALID_ARG, "npvs_forward_layer_output: bad layer");
    std::vector<FwdLevel> L;
    std::vector<void*> acts;
    void *feats, *cw, *sc;
    size_t cwb, scb;
    carve(*net, P, workspace, (size_t)-1, L, &feats, acts, &cw, &cwb, &sc, &scb);
    const int li = layer < 0 ? 0 : P.level_of[layer];
    *rows = layer < 0 ? feats : acts[layer];
    if (capacity) *capacity = L[li].cap;
    if (n_rows) *n_rows = L[li].n_rows;
    return NPVS_OK;
}
