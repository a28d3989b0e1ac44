// a4: rulebooks of the sparse convolutions (Sec. 2.3: hash-indexed sparse tensors; submanifold
// convolutions centred on active sites; strided convolutions to coarser levels: 2x2x2 onto the
// parents, and 3x3x3 with padding 1 onto the dilated output set).
//
// The site -> row index is a direct-mapped hash table: the key is the linear site index and the
// slot is the key itself, so an insert is one store and a probe one load, with no collisions.
// The largest level here has ~10^5-10^6 possible sites per batch (4 bytes each), which fits HBM
// many times over; every lookup is a single coalescing-friendly read.
#include "common.cuh"

namespace npvs {
namespace {

constexpr int kCta = 256;

__global__ void table_insert_kernel(const int32_t* __restrict__ coords, const int32_t* __restrict__ n_rows,
                                    int cap, npvs_dims d, int32_t* __restrict__ table) {
    pdl_begin();
    const int n = min(*n_rows, cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int4 c = reinterpret_cast<const int4*>(coords)[i];
        table[site_lin(c.x, c.y, c.z, c.w, d)] = i;
    }
}

__global__ void subm3_nbr_kernel(const int32_t* __restrict__ coords, const int32_t* __restrict__ n_rows, int cap,
                                 npvs_dims d, const int32_t* __restrict__ table, int32_t* __restrict__ nbr) {
    pdl_begin();
    const long long n = (long long)min(*n_rows, cap) * 27;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        int i = (int)(e / 27), k = (int)(e - (long long)i * 27);
        int4 c = reinterpret_cast<const int4*>(coords)[i];
        int z = c.y + k / 9 - 1, y = c.z + (k / 3) % 3 - 1, x = c.w + k % 3 - 1;
        int r = -1;
        if (z >= 0 && z < d.Z && y >= 0 && y < d.Y && x >= 0 && x < d.X) r = table[site_lin(c.x, z, y, x, d)];
        nbr[e] = r;
    }
}

struct DownParams {
    const int32_t* fine_table;
    npvs_dims fd, cd;
    long long n_sites;  // coarse sites
    int cap;
};

__device__ __forceinline__ void coarse_site(const DownParams& p, long long s, int& b, int& Z, int& Y, int& X) {
    X = (int)(s % p.cd.X);
    long long t = s / p.cd.X;
    Y = (int)(t % p.cd.Y);
    t /= p.cd.Y;
    Z = (int)(t % p.cd.Z);
    b = (int)(t / p.cd.Z);
}

__device__ __forceinline__ int child_row(const DownParams& p, int b, int Z, int Y, int X, int j) {
    int cz = j >> 2, cy = (j >> 1) & 1, cx = j & 1;
    return p.fine_table[site_lin(b, 2 * Z + cz, 2 * Y + cy, 2 * X + cx, p.fd)];
}

__global__ void __launch_bounds__(kCta) down_count_kernel(DownParams p, int* __restrict__ counts) {
    pdl_begin();
    long long s = (long long)blockIdx.x * kCta + threadIdx.x;
    int f = 0;
    if (s < p.n_sites) {
        int b, Z, Y, X;
        coarse_site(p, s, b, Z, Y, X);
        for (int j = 0; j < 8 && !f; ++j) f = child_row(p, b, Z, Y, X, j) >= 0;
    }
    int c = __syncthreads_count(f);
    if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

__global__ void __launch_bounds__(kCta) down_write_kernel(DownParams p, const int* __restrict__ block_off,
                                                          int32_t* __restrict__ coords, int32_t* __restrict__ table,
                                                          int32_t* __restrict__ down, int32_t* status) {
    pdl_begin();
    __shared__ int sw[33];
    long long s = (long long)blockIdx.x * kCta + threadIdx.x;
    int b = 0, Z = 0, Y = 0, X = 0;
    int ch[8];
    int f = 0;
    bool in = s < p.n_sites;
    if (in) {
        coarse_site(p, s, b, Z, Y, X);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            ch[j] = child_row(p, b, Z, Y, X, j);
            f |= ch[j] >= 0;
        }
    }
    int nloc;
    int rank = block_off[blockIdx.x] + block_exclusive_scan(f, sw, &nloc);
    if (in) table[s] = (f && rank < p.cap) ? rank : -1;
    if (f) {
        if (rank < p.cap) {
            reinterpret_cast<int4*>(coords)[rank] = make_int4(b, Z, Y, X);
            int4* dm = reinterpret_cast<int4*>(down + (size_t)rank * 8);
            dm[0] = make_int4(ch[0], ch[1], ch[2], ch[3]);
            dm[1] = make_int4(ch[4], ch[5], ch[6], ch[7]);
        } else {
            raise_status(status, NPVS_ERR_CAPACITY);
        }
    }
}

__global__ void up_map_kernel(const int32_t* __restrict__ fine_coords, const int32_t* __restrict__ n_fine, int cap,
                              npvs_dims cd, const int32_t* __restrict__ coarse_table, int32_t* __restrict__ up) {
    pdl_begin();
    const int n = min(*n_fine, cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int4 c = reinterpret_cast<const int4*>(fine_coords)[i];
        int pr = coarse_table[site_lin(c.x, c.y >> 1, c.z >> 1, c.w >> 1, cd)];
        int tap = ((c.y & 1) * 2 + (c.z & 1)) * 2 + (c.w & 1);
        up[i] = pr >= 0 ? pr * 8 + tap : -1;
    }
}

// DOWN3 (3x3x3, stride 2, padding 1): coarse site q reads the 27 fine sites 2q + k - 1 per axis,
// k in {0,1,2}; q is active iff one of them is. Fine dims are twice the coarse ones, so 2q + 1 is
// always inside the fine grid and only 2q - 1 < 0 falls outside.
__device__ __forceinline__ int foot_row(const DownParams& p, int b, int Z, int Y, int X, int k) {
    const int z = 2 * Z + k / 9 - 1, y = 2 * Y + (k / 3) % 3 - 1, x = 2 * X + k % 3 - 1;
    if (z < 0 || y < 0 || x < 0) return -1;
    return p.fine_table[site_lin(b, z, y, x, p.fd)];
}

__global__ void __launch_bounds__(kCta) down3_count_kernel(DownParams p, int* __restrict__ counts) {
    pdl_begin();
    long long s = (long long)blockIdx.x * kCta + threadIdx.x;
    int f = 0;
    if (s < p.n_sites) {
        int b, Z, Y, X;
        coarse_site(p, s, b, Z, Y, X);
        for (int k = 0; k < 27 && !f; ++k) f = foot_row(p, b, Z, Y, X, k) >= 0;
    }
    int c = __syncthreads_count(f);
    if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

__global__ void __launch_bounds__(kCta) down3_write_kernel(DownParams p, const int* __restrict__ block_off,
                                                           int32_t* __restrict__ coords, int32_t* __restrict__ table,
                                                           int32_t* __restrict__ down, int32_t* status) {
    pdl_begin();
    __shared__ int sw[33];
    long long s = (long long)blockIdx.x * kCta + threadIdx.x;
    int b = 0, Z = 0, Y = 0, X = 0;
    int f = 0;
    bool in = s < p.n_sites;
    if (in) {
        coarse_site(p, s, b, Z, Y, X);
        for (int k = 0; k < 27 && !f; ++k) f = foot_row(p, b, Z, Y, X, k) >= 0;
    }
    int nloc;
    int rank = block_off[blockIdx.x] + block_exclusive_scan(f, sw, &nloc);
    if (in) table[s] = (f && rank < p.cap) ? rank : -1;
    if (f) {
        if (rank < p.cap) {
            reinterpret_cast<int4*>(coords)[rank] = make_int4(b, Z, Y, X);
            int32_t* dm = down + (size_t)rank * 27;
            for (int k = 0; k < 27; ++k) dm[k] = foot_row(p, b, Z, Y, X, k);
        } else {
            raise_status(status, NPVS_ERR_CAPACITY);
        }
    }
}

// The transposed map of DOWN3: for fine row i and tap k the coarse row q with p = 2q + k - 1 per
// axis (p + 1 - k even and (p + 1 - k) / 2 inside the coarse grid), else -1.
__global__ void up3_map_kernel(const int32_t* __restrict__ fine_coords, const int32_t* __restrict__ n_fine, int cap,
                               npvs_dims cd, const int32_t* __restrict__ coarse_table, int32_t* __restrict__ up) {
    pdl_begin();
    const long long n = (long long)min(*n_fine, cap) * 27;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / 27), k = (int)(e - (long long)i * 27);
        const int4 c = reinterpret_cast<const int4*>(fine_coords)[i];
        const int tz = c.y + 1 - k / 9, ty = c.z + 1 - (k / 3) % 3, tx = c.w + 1 - k % 3;
        int r = -1;
        if (((tz | ty | tx) & 1) == 0 && (tz >> 1) < cd.Z && (ty >> 1) < cd.Y && (tx >> 1) < cd.X)
            r = coarse_table[site_lin(c.x, tz >> 1, ty >> 1, tx >> 1, cd)];
        up[e] = r;
    }
}

int grid_for(long long work) { return (int)std::max<long long>(1, std::min<long long>(ceil_div(work, kCta), kNumSMs * 16)); }

}  // namespace
}  // namespace npvs

using namespace npvs;

extern "C" size_t npvs_rulebook_workspace_bytes(npvs_dims d) {
    long long sites = (long long)d.B * d.X * d.Y * d.Z;  // coarse sites of a DOWN2 output <= this
    long long nb = (sites + kCta - 1) / kCta;
    return 2 * Arena::round((size_t)(nb + 1) * sizeof(int)) + 256;
}

extern "C" npvs_status npvs_build_rulebook(int32_t kind, const npvs_level* in, const npvs_level* out, int32_t* map,
                                           int32_t* map2, int32_t* status, void* workspace, size_t workspace_bytes,
                                           void* stream) {
    NPVS_REQUIRE(in && map && in->table, NPVS_ERR_INVALID_ARG, "npvs_build_rulebook: NULL argument");
    const npvs_dims fd = in->dims;
    NPVS_REQUIRE(fd.X > 0 && fd.Y > 0 && fd.Z > 0 && fd.B > 0, NPVS_ERR_INVALID_ARG, "npvs_build_rulebook: bad dims");
    cudaStream_t st = as_stream(stream);
    if (kind == NPVS_RB_SUBM3 || kind == NPVS_RB_SUBM3_TABLE) {
        NPVS_REQUIRE(in->coords && in->n_rows, NPVS_ERR_INVALID_ARG, "npvs_build_rulebook: level without coords");
        if (kind == NPVS_RB_SUBM3) {
            size_t tb = (size_t)fd.B * fd.X * fd.Y * fd.Z * sizeof(int32_t);
            if (cudaMemsetAsync(in->table, 0xFF, tb, st) != cudaSuccess) return check_launch("rulebook memset");
            launch_k(table_insert_kernel, grid_for(in->capacity), kCta, 0, st, in->coords, in->n_rows, in->capacity,
                     fd, in->table);
            NPVS_TRY(check_launch("table_insert_kernel"));
        }
        launch_k(subm3_nbr_kernel, grid_for((long long)in->capacity * 27), kCta, 0, st, in->coords, in->n_rows, in->capacity,
                                                                                 fd, in->table, map);
        return check_launch("subm3_nbr_kernel");
    }
    NPVS_REQUIRE(kind == NPVS_RB_DOWN2 || kind == NPVS_RB_DOWN3, NPVS_ERR_UNSUPPORTED, "npvs_build_rulebook: unknown kind");
    NPVS_REQUIRE(out && out->coords && out->n_rows && out->table && map2 && in->coords && in->n_rows,
                 NPVS_ERR_INVALID_ARG, "npvs_build_rulebook: DOWN2 / DOWN3 need both levels and both maps");
    const npvs_dims cd = out->dims;
    NPVS_REQUIRE(fd.X == 2 * cd.X && fd.Y == 2 * cd.Y && fd.Z == 2 * cd.Z && fd.B == cd.B, NPVS_ERR_UNSUPPORTED,
                 "npvs_build_rulebook: DOWN2 / DOWN3 need even fine dims and coarse = fine / 2");
    NPVS_REQUIRE(workspace && workspace_bytes >= npvs_rulebook_workspace_bytes(cd), NPVS_ERR_WORKSPACE,
                 "npvs_build_rulebook: workspace too small");
    DownParams p;
    p.fine_table = in->table;
    p.fd = fd;
    p.cd = cd;
    p.n_sites = (long long)cd.B * cd.X * cd.Y * cd.Z;
    p.cap = out->capacity;
    const int nb = ceil_div(p.n_sites, kCta);
    Arena ar(workspace, workspace_bytes);
    int* counts = ar.take<int>(nb + 1);
    int* offs = ar.take<int>(nb + 1);
    if (kind == NPVS_RB_DOWN3) {
        launch_k(down3_count_kernel, nb, kCta, 0, st, p, counts);
        NPVS_TRY(check_launch("down3_count_kernel"));
        NPVS_TRY(scan_block_counts(counts, offs, nb, out->n_rows, out->capacity, status, st));
        launch_k(down3_write_kernel, nb, kCta, 0, st, p, offs, out->coords, out->table, map, status);
        NPVS_TRY(check_launch("down3_write_kernel"));
        launch_k(up3_map_kernel, grid_for((long long)in->capacity * 27), kCta, 0, st, in->coords, in->n_rows,
                 in->capacity, cd, out->table, map2);
        return check_launch("up3_map_kernel");
    }
    launch_k(down_count_kernel, nb, kCta, 0, st, p, counts);
    NPVS_TRY(check_launch("down_count_kernel"));
    NPVS_TRY(scan_block_counts(counts, offs, nb, out->n_rows, out->capacity, status, st));
    launch_k(down_write_kernel, nb, kCta, 0, st, p, offs, out->coords, out->table, map, status);
    NPVS_TRY(check_launch("down_write_kernel"));
    launch_k(up_map_kernel, grid_for(in->capacity), kCta, 0, st, in->coords, in->n_rows, in->capacity, cd, out->table, map2);
    return check_launch("up_map_kernel");
}
