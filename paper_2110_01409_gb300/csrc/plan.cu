// Plan setup (untimed): CSR checks, out-degrees, the static vertex partition
// of Sec. III-A per launch shape, the out-edge CSR and weight normalisation.
#include <cub/device/device_radix_sort.cuh>
#include <cub/block/block_scan.cuh>
#include <cub/device/device_scan.cuh>

#include <algorithm>

#include "dag_internal.cuh"
#include "devmem.cuh"

namespace dag {

// ---------------------------------------------------------------------------
// CSR checks and per-vertex data
// ---------------------------------------------------------------------------
__global__ void k_check_rowptr(const int* rowptr, int n, long long m, int* bad)
{
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v > n) return;
    int x = rowptr[v];
    if (v == 0 && x != 0) atomicOr(bad, 1);
    if (v == n && (long long)x != m) atomicOr(bad, 1);
    if (v < n && rowptr[v + 1] < x) atomicOr(bad, 1);
}

// Out-degree histogram of the sources. Lanes of a warp holding the same source
// (hub vertices recur often) add their count with one atomic.
__global__ void k_out_degree(const int* colidx, long long m, int n, int* outdeg, int* bad)
{
    const unsigned lane_lt = (1u << (threadIdx.x & 31)) - 1u;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < m;
         e += (long long)gridDim.x * blockDim.x) {
        const int u = colidx[e];
        const bool ok = u >= 0 && u < n;
        if (!ok) atomicOr(bad, 2);
        const unsigned peers = __match_any_sync(__activemask(), ok ? u : -1);
        if (ok && (peers & lane_lt) == 0) atomicAdd(&outdeg[u], __popc(peers));
    }
}

__global__ void k_degf(const int* outdeg, float* degf, int n)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) degf[v] = (float)outdeg[v];
}

__global__ void k_iota(int* a, long long m)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < m; e += (long long)gridDim.x * blockDim.x)
        a[e] = (int)e;
}

static int bits_for(int n)
{
    int b = 1;
    while (b < 31 && (1LL << b) < n) ++b;
    return b;
}

// ---------------------------------------------------------------------------
// Partition: block p starts at min { v : v + rowptr[v] >= ceil(p (n+m) / P) }
// (every vertex weighs in-degree + 1), then each block is cut into merge-path
// tiles of TILE items; a tile's start is (rows ended before it, edges before it).
// ---------------------------------------------------------------------------
// row_w: weight of a row beside its in-edges (1: Sec. III-A's in-degree + 1;
// row-capped tiles weigh rows more, see get_partition); total = row_w n + m.
__global__ void k_cta_rows(const int* rowptr, int n, long long total, int P, int* cta_row, int row_w)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > P) return;
    if (p == 0) { cta_row[0] = 0; return; }
    if (p == P) { cta_row[P] = n; return; }
    long long target = ((long long)p * total + P - 1) / P;
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if ((long long)row_w * mid + rowptr[mid] >= target) hi = mid;
        else lo = mid + 1;
    }
    cta_row[p] = lo;
}

// Tile counts of the P blocks and their exclusive prefix (cta_tile[0..P]), and
// the largest block's row count; one CTA of CT_THREADS threads, chunk by chunk.
__global__ void __launch_bounds__(CT_THREADS) k_cta_tiles(const int* rowptr, const int* cta_row, int P,
                                                          int* cta_tile, int* max_rows)
{
    using Scan = cub::BlockScan<int, CT_THREADS>;
    __shared__ typename Scan::TempStorage tmp;
    __shared__ int carry, mr;
    if (threadIdx.x == 0) { carry = 0; mr = 0; }
    for (int base = 0; base < P; base += CT_THREADS) {
        const int p = base + threadIdx.x;
        int cnt = 0;
        if (p < P) {
            const int r0 = cta_row[p], r1 = cta_row[p + 1];
            const long long items = (long long)(r1 - r0) + (rowptr[r1] - rowptr[r0]);
            cnt = (int)((items + TILE - 1) / TILE);
            atomicMax(&mr, r1 - r0);
        }
        __syncthreads();  // carry of the previous chunk is final; tmp is free
        int excl = 0, chunk = 0;
        Scan(tmp).ExclusiveSum(cnt, excl, chunk);
        if (p < P) cta_tile[p] = carry + excl;
        __syncthreads();
        if (threadIdx.x == 0) carry += chunk;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        cta_tile[P] = carry;
        *max_rows = mr;
    }
}

__global__ void k_tile_coords(const int* rowptr, int n, long long m, const int* cta_row, const int* cta_tile,
                              int P, int tiles, int* tile_row, int* tile_nz)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > tiles) return;
    if (k == tiles) { tile_row[k] = n; tile_nz[k] = (int)m; return; }
    int lo = 0, hi = P - 1;  // owning block: last p with cta_tile[p] <= k
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (cta_tile[mid] <= k) lo = mid;
        else hi = mid - 1;
    }
    int p = lo;
    long long diag = (long long)cta_row[p] + rowptr[cta_row[p]] + (long long)(k - cta_tile[p]) * TILE;
    // rows whose end item lies before diag: first v with v + rowptr[v+1] >= diag
    int a = cta_row[p], b = cta_row[p + 1];
    while (a < b) {
        int mid = (a + b) >> 1;
        if ((long long)mid + rowptr[mid + 1] >= diag) b = mid;
        else a = mid + 1;
    }
    tile_row[k] = a;
    tile_nz[k] = (int)(diag - a);
}

// Tiles capped at R completed rows (delayed sweeps whose delta is below a
// tile's rows: a tile's rows are computed together, so a buffer of delta rows
// can only be flushed at a tile end, and capping the rows per tile lets it
// flush after about every delta rows). A tile of block p ends at the first of:
// TILE items, the item that ends its R-th row, the block end. One thread per
// block walks its tiles; `count` mode writes the tile count of the block,
// else the merge-path coordinates from tile_row/tile_nz[cta_tile[p]] on.
__device__ __forceinline__ int rows_ended_before(const int* rowptr, int a, int r1, long long diag)
{
    // first v in [a, r1] with v + rowptr[v+1] >= diag (v = r1: all of the block's rows ended)
    int lo = a, hi = r1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((long long)mid + rowptr[mid + 1] >= diag) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

__global__ void k_capped_tiles(const int* rowptr, const int* cta_row, int P, int R, int* cnt, const int* cta_tile,
                               int* tile_row, int* tile_nz)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int r0 = cta_row[p], r1 = cta_row[p + 1];
    const long long d_end = (long long)r1 + rowptr[r1];
    int a = r0;
    long long d = (long long)r0 + rowptr[r0];
    int k = 0;
    while (d < d_end) {
        if (tile_row) {
            tile_row[cta_tile[p] + k] = a;
            tile_nz[cta_tile[p] + k] = (int)(d - a);
        }
        long long dn = d + TILE;
        if (a + R - 1 < r1) {  // the item that ends row a + R - 1, the R-th row from a
            const long long dc = (long long)(a + R - 1) + rowptr[a + R] + 1;
            if (dc < dn) dn = dc;
        }
        if (dn > d_end) dn = d_end;
        a = rows_ended_before(rowptr, a, r1, dn);
        d = dn;
        ++k;
    }
    if (cnt) cnt[p] = k;
}

// Exclusive prefix of per-block tile counts into cta_tile[0..P] and the
// largest block's row count (one CTA of CT_THREADS threads).
__global__ void __launch_bounds__(CT_THREADS) k_prefix_tiles(const int* cnt, const int* cta_row, int P,
                                                             int* cta_tile, int* max_rows)
{
    using Scan = cub::BlockScan<int, CT_THREADS>;
    __shared__ typename Scan::TempStorage tmp;
    __shared__ int carry, mr;
    if (threadIdx.x == 0) { carry = 0; mr = 0; }
    for (int base = 0; base < P; base += CT_THREADS) {
        const int p = base + threadIdx.x;
        int c = 0;
        if (p < P) {
            c = cnt[p];
            atomicMax(&mr, cta_row[p + 1] - cta_row[p]);
        }
        __syncthreads();
        int excl = 0, chunk = 0;
        Scan(tmp).ExclusiveSum(c, excl, chunk);
        if (p < P) cta_tile[p] = carry + excl;
        __syncthreads();
        if (threadIdx.x == 0) carry += chunk;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        cta_tile[P] = carry;
        *max_rows = mr;
    }
}

__global__ void k_tile_end(int tiles, int n, long long m, int* tile_row, int* tile_nz)
{
    tile_row[tiles] = n;
    tile_nz[tiles] = (int)m;
}

int get_partition(dag_plan* plan, int P, Partition** out, cudaStream_t s, int row_cap)
{
    if (row_cap >= TILE) row_cap = 0;  // a tile never holds more than TILE rows
    const long long key = (long long)P | ((long long)row_cap << 32);
    auto it = plan->parts.find(key);
    if (it != plan->parts.end()) { *out = &it->second; return DAG_OK; }
    Partition part;
    part.nblocks = P;
    part.row_cap = row_cap;
    int* mr_dev = nullptr;
    int* cnt = nullptr;
    DAG_CUDA(dev_alloc(&part.cta_row, (P + 1) * sizeof(int)));
    DAG_CUDA(dev_alloc(&part.cta_tile, (P + 1) * sizeof(int)));
    DAG_CUDA(dev_alloc(&mr_dev, sizeof(int)));
    // Row-capped tiles cost a tile per row_cap rows even where rows have no
    // edges, so their blocks weigh each row ceil(TILE / row_cap) instead of 1:
    // a block's tile count then follows its weight, as it does uncapped.
    const int row_w = row_cap > 0 ? (TILE + row_cap - 1) / row_cap : 1;
    long long total = (long long)row_w * plan->n + plan->m;
    k_cta_rows<<<(P + 1 + 255) / 256, 256, 0, s>>>(plan->rowptr, plan->n, total, P, part.cta_row, row_w);
    if (row_cap > 0) {
        DAG_CUDA(dev_alloc(&cnt, P * sizeof(int)));
        k_capped_tiles<<<(P + 127) / 128, 128, 0, s>>>(plan->rowptr, part.cta_row, P, row_cap, cnt, nullptr,
                                                      nullptr, nullptr);
        k_prefix_tiles<<<1, CT_THREADS, 0, s>>>(cnt, part.cta_row, P, part.cta_tile, mr_dev);
    } else {
        k_cta_tiles<<<1, CT_THREADS, 0, s>>>(plan->rowptr, part.cta_row, P, part.cta_tile, mr_dev);
    }
    int tiles = 0;
    DAG_CUDA(cudaMemcpyAsync(&tiles, part.cta_tile + P, sizeof(int), cudaMemcpyDeviceToHost, s));
    DAG_CUDA(cudaMemcpyAsync(&part.max_rows, mr_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    DAG_CUDA(cudaStreamSynchronize(s));
    dev_free(mr_dev);
    part.tiles = tiles;
    DAG_CUDA(dev_alloc(&part.tile_row, (tiles + 1) * sizeof(int)));
    DAG_CUDA(dev_alloc(&part.tile_nz, (tiles + 1) * sizeof(int)));
    if (row_cap > 0) {
        k_capped_tiles<<<(P + 127) / 128, 128, 0, s>>>(plan->rowptr, part.cta_row, P, row_cap, nullptr,
                                                      part.cta_tile, part.tile_row, part.tile_nz);
        k_tile_end<<<1, 1, 0, s>>>(tiles, plan->n, plan->m, part.tile_row, part.tile_nz);
        DAG_CUDA(cudaStreamSynchronize(s));
        dev_free(cnt);
    } else {
        k_tile_coords<<<(tiles + 1 + 255) / 256, 256, 0, s>>>(plan->rowptr, plan->n, plan->m, part.cta_row,
                                                               part.cta_tile, P, tiles, part.tile_row,
                                                               part.tile_nz);
    }
    DAG_CUDA(cudaGetLastError());
    auto ins = plan->parts.emplace(key, part);
    *out = &ins.first->second;
    return DAG_OK;
}

// Warp-worker partition: tile k starts at diagonal k * tile of the whole merge
// path; its coordinates are (rows ended before it, edges before it).
__global__ void k_warp_tile_coords(const int* rowptr, int n, long long m, int tile, int tiles, int* tile_row,
                                   int* tile_nz)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > tiles) return;
    if (k == tiles) { tile_row[k] = n; tile_nz[k] = (int)m; return; }
    const long long diag = (long long)k * tile;
    int lo = 0, hi = n;  // first v with v + rowptr[v+1] >= diag
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((long long)mid + rowptr[mid + 1] >= diag) hi = mid;
        else lo = mid + 1;
    }
    tile_row[k] = lo;
    tile_nz[k] = (int)(diag - lo);
}
// Tile k of the merge path of rows [lo, hi): diagonal min(d_lo + k tile, d_hi).
__global__ void k_range_tile_coords(const int* rowptr, int lo, int hi, int tile, int tiles, int* tile_row,
                                    int* tile_nz)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > tiles) return;
    const long long d_lo = (long long)lo + rowptr[lo], d_hi = (long long)hi + rowptr[hi];
    const long long diag = k == tiles ? d_hi : d_lo + (long long)k * tile;
    int a = lo, b = hi;  // first v in [lo, hi] with v + rowptr[v+1] >= diag
    while (a < b) {
        const int mid = (a + b) >> 1;
        if ((long long)mid + rowptr[mid + 1] >= diag) b = mid;
        else a = mid + 1;
    }
    tile_row[k] = a;
    tile_nz[k] = (int)(diag - a);
}

__global__ void k_warp_runs(const int* tile_row, int tiles, int W, int* wtile, int* wrow)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w > W) return;
    const int t = (int)((long long)w * tiles / W);
    wtile[w] = t;
    wrow[w] = tile_row[t];
}

int get_warp_partition(dag_plan* plan, int W, int tile, Partition** out, cudaStream_t s)
{
    const long long key = (1LL << 62) | ((long long)tile << 32) | (long long)W;
    auto it = plan->parts.find(key);
    if (it != plan->parts.end()) { *out = &it->second; return DAG_OK; }
    Partition part;
    part.nblocks = W;
    const long long total = (long long)plan->n + plan->m;
    const long long T = (total + tile - 1) / tile;
    if (T >= (1LL << 31)) return set_error(DAG_ERR_INVALID, "graph too large for warp tiles");
    part.tiles = (int)T;
    DAG_CUDA(dev_alloc(&part.cta_row, (W + 1) * sizeof(int)));
    DAG_CUDA(dev_alloc(&part.cta_tile, (W + 1) * sizeof(int)));
    DAG_CUDA(dev_alloc(&part.tile_row, (T + 1) * sizeof(int)));
    DAG_CUDA(dev_alloc(&part.tile_nz, (T + 1) * sizeof(int)));
    DAG_CUDA(dev_alloc(&part.wpub, W * sizeof(unsigned long long)));
    k_warp_tile_coords<<<(unsigned)((T + 1 + 255) / 256), 256, 0, s>>>(plan->rowptr, plan->n, plan->m, tile, (int)T,
                                                                       part.tile_row, part.tile_nz);
    k_warp_runs<<<(W + 1 + 255) / 256, 256, 0, s>>>(part.tile_row, (int)T, W, part.cta_tile, part.cta_row);
    DAG_CUDA(cudaGetLastError());
    std::vector<int> wrow(W + 1);
    DAG_CUDA(cudaMemcpyAsync(wrow.data(), part.cta_row, (W + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    DAG_CUDA(cudaStreamSynchronize(s));
    for (int w = 0; w < W; ++w) part.max_rows = std::max(part.max_rows, wrow[w + 1] - wrow[w]);
    auto ins = plan->parts.emplace(key, part);
    *out = &ins.first->second;
    return DAG_OK;
}

int get_warp_partition_range(dag_plan* plan, int W, int tile, int lo, int hi, Partition** out, cudaStream_t s)
{
    const auto key = std::make_tuple(W, tile, lo, hi);
    auto it = plan->range_parts.find(key);
    if (it != plan->range_parts.end()) { *out = &it->second; return DAG_OK; }
    std::vector<int> rp(2);
    DAG_CUDA(cudaMemcpy(&rp[0], plan->rowptr + lo, sizeof(int), cudaMemcpyDeviceToHost));
    DAG_CUDA(cudaMemcpy(&rp[1], plan->rowptr + hi, sizeof(int), cudaMemcpyDeviceToHost));
    const long long items = (long long)(hi - lo) + (rp[1] - rp[0]);
    const long long T = std::max(1LL, (items + tile - 1) / tile);
    Partition part;
    part.nblocks = W;
    part.tiles = (int)T;
    DAG_CUDA(dev_alloc(&part.cta_row, (W + 1) * sizeof(int)));
    DAG_CUDA(dev_alloc(&part.cta_tile, (W + 1) * sizeof(int)));
    DAG_CUDA(dev_alloc(&part.tile_row, (T + 1) * sizeof(int)));
    DAG_CUDA(dev_alloc(&part.tile_nz, (T + 1) * sizeof(int)));
    DAG_CUDA(dev_alloc(&part.wpub, W * sizeof(unsigned long long)));
    k_range_tile_coords<<<(unsigned)((T + 1 + 255) / 256), 256, 0, s>>>(plan->rowptr, lo, hi, tile, (int)T,
                                                                        part.tile_row, part.tile_nz);
    k_warp_runs<<<(W + 1 + 255) / 256, 256, 0, s>>>(part.tile_row, (int)T, W, part.cta_tile, part.cta_row);
    DAG_CUDA(cudaGetLastError());
    DAG_CUDA(cudaStreamSynchronize(s));
    auto ins = plan->range_parts.emplace(key, part);
    *out = &ins.first->second;
    return DAG_OK;
}

// ---------------------------------------------------------------------------
// Out-edge CSR: a stable radix sort of the in-edges by source keeps, within
// each source, the in-CSR order, i.e. ascending targets.
// ---------------------------------------------------------------------------
// dst[e] = the row of in-edge e. One warp per 32 rows, all lanes on each row's
// edges in turn, so a hub row (tens of thousands of edges) is not one thread's.
__global__ void k_edge_dst(const int* rowptr, int n, int* dst)
{
    const int lane = threadIdx.x & 31;
    const long long v0 = ((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5) * 32;
    if (v0 >= n) return;
    const int v1 = (int)min(v0 + 32, (long long)n);
    for (int v = (int)v0; v < v1; ++v) {
        const int e1 = rowptr[v + 1];
        for (int e = rowptr[v] + lane; e < e1; e += 32) dst[e] = v;
    }
}

__global__ void k_gather_i32(const int* src, const int* idx, int* out, long long m)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < m; e += (long long)gridDim.x * blockDim.x)
        out[e] = src[idx[e]];
}


int launch_transpose(dag_plan* plan, int* out_rowptr, int* out_colidx, int* perm, cudaStream_t s)
{
    const int n = plan->n;
    const long long m = plan->m;
    // out_rowptr = exclusive prefix of out-degree, with the total at [n]
    // scan over n+1 entries (the last one 0) so that out_rowptr[n] = m
    void* tmp = nullptr;
    int* padded = nullptr;
    size_t tmp_bytes = 0;
    DAG_CUDA(dev_alloc(&padded, (size_t)(n + 1) * sizeof(int)));
    DAG_CUDA(cudaMemsetAsync(padded + n, 0, sizeof(int), s));
    DAG_CUDA(cudaMemcpyAsync(padded, plan->outdeg, (size_t)n * sizeof(int), cudaMemcpyDeviceToDevice, s));
    DAG_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, padded, out_rowptr, n + 1, s));
    DAG_CUDA(dev_alloc(&tmp, tmp_bytes));
    DAG_CUDA(cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, padded, out_rowptr, n + 1, s));
    DAG_CUDA(cudaStreamSynchronize(s));
    dev_free(tmp);
    dev_free(padded);
    if (m == 0) return DAG_OK;
    int *keys_out = nullptr, *vals_in = nullptr, *dst = nullptr;
    DAG_CUDA(dev_alloc(&keys_out, (size_t)m * sizeof(int)));
    DAG_CUDA(dev_alloc(&vals_in, (size_t)m * sizeof(int)));
    DAG_CUDA(dev_alloc(&dst, (size_t)m * sizeof(int)));
    k_iota<<<1024, 256, 0, s>>>(vals_in, m);
    k_edge_dst<<<(n + 255) / 256, 256, 0, s>>>(plan->rowptr, n, dst);
    tmp_bytes = 0;
    DAG_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, plan->colidx, keys_out, vals_in, perm, (int)m, 0,
                                             bits_for(n), s));
    DAG_CUDA(dev_alloc(&tmp, tmp_bytes));
    DAG_CUDA(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, plan->colidx, keys_out, vals_in, perm, (int)m, 0,
                                             bits_for(n), s));
    k_gather_i32<<<1024, 256, 0, s>>>(dst, perm, out_colidx, m);
    DAG_CUDA(cudaGetLastError());
    DAG_CUDA(cudaStreamSynchronize(s));
    dev_free(tmp);
    dev_free(keys_out);
    dev_free(vals_in);
    dev_free(dst);
    return DAG_OK;
}

// Frontier maps: for every out-edge u -> v, the tile holding its in-CSR
// position and the tile holding v's row end. A change of u makes the tiles
// between the two run again in the next sweep. The maps are read as one set
// per source, so the order of the edges inside a source's out-list is free:
// a counting sort by source fills them in one pass over the in-CSR.

// One warp per tile t: every in-edge e = (v <- u) of the tile (edges
// [tile_nz[t], tile_nz[t+1]) of rows [tile_row[t], tile_row[t+1]]) takes the
// next slot of u's out-list (cursor[u], one atomic per run of equal sources
// in the warp) and writes there t and the tile ending row v: t itself for the
// rows that end inside t, else the tile ending row tile_row[t+1] (oend may
// be null).
__global__ void k_frontier_scatter(const int* rowptr, const int* colidx, int n, const int* tile_row,
                                   const int* tile_nz, int tiles, int* cursor, int* otile, int* oend)
{
    const int lane = threadIdx.x & 31;
    const int nwarps = (int)(((long long)gridDim.x * blockDim.x) >> 5);
    for (int t = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5); t < tiles; t += nwarps) {
        const int r0 = tile_row[t], r1 = tile_row[t + 1];
        const int nz0 = tile_nz[t], nz1 = tile_nz[t + 1];
        if (nz0 >= nz1) continue;
        // the tile ending row r1: the first t' > t whose successor starts past r1
        int end1 = t;
        if (r1 < n) {
            int lo = t + 1, hi = tiles - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (tile_row[mid + 1] > r1) hi = mid; else lo = mid + 1;
            }
            end1 = lo;
        }
        const int vmax = min(r1, n - 1);
        for (int e0 = nz0; e0 < nz1; e0 += 32) {
            const int e = e0 + lane;
            const bool live = e < nz1;
            const unsigned act = __ballot_sync(0xffffffffu, live);
            if (!live) continue;
            // the row of e: the last row of the tile starting at or before e
            int lo = r0, hi = vmax;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (rowptr[mid] <= e) lo = mid; else hi = mid - 1;
            }
            const int u = colidx[e];
            const unsigned peers = __match_any_sync(act, u);
            const int leader = __ffs(peers) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(cursor + u, __popc(peers));
            base = __shfl_sync(peers, base, leader);
            const int pos = base + __popc(peers & ((1u << lane) - 1u));
            otile[pos] = t;
            if (oend) oend[pos] = lo < r1 ? t : end1;
        }
    }
}

// fr_orow[0] = 0, fr_orow[1 ..] = inclusive prefix of out-degree. with_end
// false leaves out fr_oend (the warp-tile frontier stamps one tile per edge).
static int build_frontier_maps(dag_plan* plan, Partition* part, cudaStream_t s, bool with_end)
{
    const int n = plan->n;
    const long long m = plan->m;
    size_t scan_bytes = 0;
    DAG_CUDA(cub::DeviceScan::InclusiveSum(nullptr, scan_bytes, plan->outdeg, (int*)nullptr, n, s));
    // fr_otile doubles as the scan's scratch before the scatter fills it
    const size_t otile_ints = std::max((size_t)std::max(m, 1LL), (scan_bytes + sizeof(int) - 1) / sizeof(int));
    if (!plan->fr_orow) DAG_CUDA(dev_alloc(&plan->fr_orow, (size_t)(n + 1) * sizeof(int)));
    DAG_CUDA(dev_alloc(&part->fr_otile, otile_ints * sizeof(int)));
    if (with_end) DAG_CUDA(dev_alloc(&part->fr_oend, (size_t)std::max(m, 1LL) * sizeof(int)));
    DAG_CUDA(dev_alloc(&part->fr_alist, (size_t)std::max(part->tiles, 1) * sizeof(int)));
    DAG_CUDA(dev_alloc(&part->fr_chg, (size_t)n * sizeof(int)));
    DAG_CUDA(dev_alloc(&part->fr_glist, (size_t)std::max(part->tiles, 1) * sizeof(int)));
    DAG_CUDA(dev_alloc(&part->fr_gchg, ((size_t)n + (size_t)std::max(part->tiles, 1)) * sizeof(int)));
    DAG_CUDA(cudaMemsetAsync(plan->fr_orow, 0, sizeof(int), s));
    DAG_CUDA(cub::DeviceScan::InclusiveSum(part->fr_otile, scan_bytes, plan->outdeg, plan->fr_orow + 1, n, s));
    if (m > 0 && part->tiles > 0) {
        // fr_chg (a per-sweep list, written before it is read) serves as the cursor
        DAG_CUDA(cudaMemcpyAsync(part->fr_chg, plan->fr_orow, (size_t)n * sizeof(int), cudaMemcpyDeviceToDevice, s));
        const int blocks = (int)std::min(((long long)part->tiles * 32 + 255) / 256, 152LL * 64);
        k_frontier_scatter<<<blocks, 256, 0, s>>>(plan->rowptr, plan->colidx, n, part->tile_row, part->tile_nz,
                                                  part->tiles, part->fr_chg, part->fr_otile, part->fr_oend);
        DAG_CUDA(cudaGetLastError());
    }
    DAG_CUDA(cudaStreamSynchronize(s));
    // allocated last: a set fr_act marks the maps complete
    DAG_CUDA(dev_alloc(&part->fr_act, (size_t)std::max(part->tiles, 1) * sizeof(int)));
    return DAG_OK;
}

int frontier_maps(dag_plan* plan, Partition* part, cudaStream_t s, bool with_end)
{
    if (part->fr_act) return DAG_OK;
    const int rc = build_frontier_maps(plan, part, s, with_end);
    if (rc != DAG_OK) {  // a failed build leaves nothing behind: the next frontier solve starts again
        int** arrays[] = {&part->fr_otile, &part->fr_oend, &part->fr_alist, &part->fr_chg,
                          &part->fr_glist, &part->fr_gchg, &part->fr_act};
        for (int** a : arrays) {
            dev_free(*a);
            *a = nullptr;
        }
    }
    return rc;
}

// s[u] = sum of w over u's out-edges, in a fixed order whatever the launch:
// a warp per source (lane j takes out-edges j, j + 32, ... in out-CSR order,
// then a butterfly of the lanes' sums); sources of more than NW_HUB out-edges
// are left to k_out_sum_hub, a whole block per source.
constexpr int NW_HUB = 2048;
constexpr int NW_HUB_THREADS = 256;
__global__ void k_out_sum(const int* orow, const int* perm, const float* w, int n, float* s)
{
    const int lane = threadIdx.x & 31;
    const long long u = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    if (u >= n) return;
    const int k0 = orow[u], k1 = orow[u + 1];
    if (k1 - k0 > NW_HUB) return;
    float acc = 0.0f;
    for (int k = k0 + lane; k < k1; k += 32) acc += w[perm[k]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) s[u] = acc;
}
__global__ void __launch_bounds__(NW_HUB_THREADS) k_out_sum_hub(const int* orow, const int* perm, const float* w,
                                                               const int* hubs, int nhubs, float* s)
{
    __shared__ float part[NW_HUB_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int h = blockIdx.x; h < nhubs; h += gridDim.x) {
        const int u = hubs[h];
        const int k1 = orow[u + 1];
        float acc = 0.0f;
        for (int k = orow[u] + threadIdx.x; k < k1; k += NW_HUB_THREADS) acc += w[perm[k]];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) part[wid] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.0f;
            for (int j = 0; j < NW_HUB_THREADS / 32; ++j) t += part[j];
            s[u] = t;
        }
        __syncthreads();
    }
}
// The sources of more than NW_HUB out-edges (list order free: each is summed alone).
__global__ void k_hub_list(const int* orow, int n, int* hubs, int* nhubs)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n && orow[u + 1] - orow[u] > NW_HUB) hubs[atomicAdd(nhubs, 1)] = u;
}
__global__ void k_div(const int* colidx, const float* w, const float* s, float* val, long long m)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < m; e += (long long)gridDim.x * blockDim.x)
        val[e] = w[e] / s[colidx[e]];
}

__global__ void k_gather_f32(const float* src, const int* idx, float* out, long long m)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < m; e += (long long)gridDim.x * blockDim.x)
        out[e] = src[idx[e]];
}

// The out-CSR order of the plan's edges (row pointers and permutation) is
// built on the first call and kept: only the weights change between calls.
int launch_normalize(dag_plan* plan, const float* w, float* val, float* s_out, cudaStream_t s)
{
    const int n = plan->n;
    const long long m = plan->m;
    if (!plan->nw_perm) {
        int* orow = plan->fr_orow;
        int *ocol = nullptr, *perm = nullptr, *hubs = nullptr;
        if (!orow) DAG_CUDA(dev_alloc(&orow, (size_t)(n + 1) * sizeof(int)));
        plan->fr_orow = orow;
        DAG_CUDA(dev_alloc(&ocol, (size_t)std::max(m, 1LL) * sizeof(int)));
        if (dev_alloc(&perm, (size_t)std::max(m, 1LL) * sizeof(int)) != cudaSuccess) {
            dev_free(ocol);
            return cuda_check(cudaGetLastError(), "normalisation out-CSR");
        }
        int rc = launch_transpose(plan, orow, ocol, perm, s);
        dev_free(ocol);
        if (rc == DAG_OK && dev_alloc(&hubs, (size_t)(n + 1) * sizeof(int)) != cudaSuccess)
            rc = cuda_check(cudaGetLastError(), "normalisation hub list");
        if (rc == DAG_OK) {
            // hubs[n] counts the list
            int nh = 0;
            cudaMemsetAsync(hubs + n, 0, sizeof(int), s);
            k_hub_list<<<(n + 255) / 256, 256, 0, s>>>(orow, n, hubs, hubs + n);
            cudaMemcpyAsync(&nh, hubs + n, sizeof(int), cudaMemcpyDeviceToHost, s);
            const cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) rc = cuda_check(e, "normalisation hub list");
            plan->nw_nhubs = nh;
        }
        if (rc != DAG_OK) {
            dev_free(perm);
            dev_free(hubs);
            return rc;
        }
        plan->nw_hubs = hubs;
        plan->nw_perm = perm;  // set last: a set nw_perm marks the out-CSR order complete
    }
    k_out_sum<<<(unsigned)(((long long)n * 32 + 255) / 256), 256, 0, s>>>(plan->fr_orow, plan->nw_perm, w, n, s_out);
    if (plan->nw_nhubs > 0)
        k_out_sum_hub<<<std::min(plan->nw_nhubs, 4 * plan->num_sms), NW_HUB_THREADS, 0, s>>>(
            plan->fr_orow, plan->nw_perm, w, plan->nw_hubs, plan->nw_nhubs, s_out);
    if (m) k_div<<<2048, 256, 0, s>>>(plan->colidx, w, s_out, val, m);
    DAG_CUDA(cudaGetLastError());
    return DAG_OK;
}

}  // namespace dag

// ---------------------------------------------------------------------------
// Plan life cycle (C ABI)
// ---------------------------------------------------------------------------
using namespace dag;

extern "C" int dag_plan_create(const dag_csr* csr, int32_t barrier_timeout_ms, dag_plan** out)
{
    if (!csr || !out) return set_error(DAG_ERR_INVALID, "null argument");
    *out = nullptr;
    if (csr->n < 1 || csr->m < 0 || csr->m >= (1LL << 31))
        return set_error(DAG_ERR_INVALID, "need n >= 1 and 0 <= m < 2^31");
    if (!csr->d_rowptr || (csr->m > 0 && !csr->d_colidx))
        return set_error(DAG_ERR_INVALID, "null CSR array");
    dag_plan* p = new dag_plan();
    p->n = csr->n;
    p->m = csr->m;
    p->rowptr = csr->d_rowptr;
    p->colidx = csr->d_colidx;
    if (barrier_timeout_ms > 0) p->timeout_ns = (long long)barrier_timeout_ms * 1000000LL;
    auto fail = [&](int rc) { dag_plan_destroy(p); return rc; };
    if (cudaGetDevice(&p->device) != cudaSuccess) return fail(cuda_check(cudaGetLastError(), "cudaGetDevice"));
    cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    const int n = p->n;
    int* bad = nullptr;
    if (dev_alloc(&p->outdeg, (size_t)n * sizeof(int)) != cudaSuccess ||
        dev_alloc(&p->degf, (size_t)n * sizeof(float)) != cudaSuccess ||
        dev_alloc(&p->x0, (size_t)n * 4) != cudaSuccess || dev_alloc(&p->x1, (size_t)n * 4) != cudaSuccess ||
        dev_alloc(&p->scratch_f, (size_t)n * 4) != cudaSuccess ||
        dev_alloc(&p->sync, sizeof(SyncBlock)) != cudaSuccess || dev_alloc(&bad, sizeof(int)) != cudaSuccess) {
        dev_free(bad);
        cudaGetLastError();
        return fail(set_error(DAG_ERR_NOMEM, "plan workspace allocation failed"));
    }
    cudaStream_t s = 0;
    cudaMemsetAsync(bad, 0, sizeof(int), s);
    cudaMemsetAsync(p->outdeg, 0, (size_t)n * sizeof(int), s);
    k_check_rowptr<<<(n + 1 + 255) / 256, 256, 0, s>>>(p->rowptr, n, p->m, bad);
    int hbad = 0;
    cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        dev_free(bad);
        return fail(cuda_check(cudaGetLastError(), "rowptr check"));
    }
    if (hbad) {
        dev_free(bad);
        return fail(set_error(DAG_ERR_INVALID, "rowptr must start at 0, not decrease and end at m"));
    }
    if (p->m > 0) k_out_degree<<<2048, 256, 0, s>>>(p->colidx, p->m, n, p->outdeg, bad);
    k_degf<<<(n + 255) / 256, 256, 0, s>>>(p->outdeg, p->degf, n);
    cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    dev_free(bad);
    if (e != cudaSuccess) return fail(cuda_check(e, "out-degree"));
    if (hbad) return fail(set_error(DAG_ERR_INVALID, "colidx entry outside [0, n)"));
    *out = p;
    return DAG_OK;
}

namespace dag {
void release_batched_graphs(const dag_plan* plan);  // batched.cu: the plan's CUDA graphs
}

extern "C" int dag_plan_destroy(dag_plan* p)
{
    if (!p) return DAG_OK;
    dag::release_batched_graphs(p);
    // the plan's memory goes back to its device's pool once every launch that may use it has finished
    int prev = 0;
    const bool have_prev = cudaGetDevice(&prev) == cudaSuccess;
    if (!have_prev || prev != p->device) cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    dev_free(p->outdeg);
    dev_free(p->degf);
    dev_free(p->x0);
    dev_free(p->x1);
    dev_free(p->scratch_f);
    dev_free(p->sync);
    cudaFree(p->bx);  // batched workspace: cudaMalloc (batched.cu)
    cudaFree(p->bsync);
    for (auto& kv : p->parts) {
        dev_free(kv.second.cta_row);
        dev_free(kv.second.cta_tile);
        dev_free(kv.second.tile_row);
        dev_free(kv.second.tile_nz);
        dev_free(kv.second.fr_otile);
        dev_free(kv.second.fr_oend);
        dev_free(kv.second.fr_act);
        dev_free(kv.second.fr_alist);
        dev_free(kv.second.fr_chg);
        dev_free(kv.second.fr_glist);
        dev_free(kv.second.fr_gchg);
        dev_free(kv.second.wpub);
        cudaFree(kv.second.tpub);  // cudaMalloc (sweep_warp.cu)
    }
    for (auto& kv : p->range_parts) {
        dev_free(kv.second.cta_row);
        dev_free(kv.second.cta_tile);
        dev_free(kv.second.tile_row);
        dev_free(kv.second.tile_nz);
        dev_free(kv.second.wpub);
    }
    dev_free(p->fr_orow);
    dev_free(p->nw_perm);
    dev_free(p->nw_hubs);
    dev_free(p->grad_coef);
    if (have_prev && prev != p->device) cudaSetDevice(prev);
    delete p;
    return DAG_OK;
}

extern "C" int dag_plan_out_degree(const dag_plan* p, int32_t* d_outdeg, void* stream)
{
    if (!p || !d_outdeg) return set_error(DAG_ERR_INVALID, "null argument");
    DAG_CUDA(cudaMemcpyAsync(d_outdeg, p->outdeg, (size_t)p->n * sizeof(int), cudaMemcpyDeviceToDevice,
                             (cudaStream_t)stream));
    return DAG_OK;
}

extern "C" int dag_partition(dag_plan* p, int32_t workers, int32_t* h_start)
{
    if (!p || !h_start || workers < 1) return set_error(DAG_ERR_INVALID, "bad argument");
    Partition* part = nullptr;
    int rc = get_partition(p, workers, &part, 0, 0);
    if (rc) return rc;
    DAG_CUDA(cudaMemcpy(h_start, part->cta_row, (size_t)(workers + 1) * sizeof(int), cudaMemcpyDeviceToHost));
    return DAG_OK;
}

extern "C" int dag_transpose(dag_plan* p, int32_t* d_out_rowptr, int32_t* d_out_colidx, int32_t* d_perm,
                             void* stream)
{
    if (!p || !d_out_rowptr || (p->m > 0 && (!d_out_colidx || !d_perm)))
        return set_error(DAG_ERR_INVALID, "null argument");
    return launch_transpose(p, d_out_rowptr, d_out_colidx, d_perm, (cudaStream_t)stream);
}

extern "C" int dag_normalize_weights(dag_plan* p, const float* d_w, float* d_val, float* d_s, void* stream)
{
    if (!p || !d_s || (p->m > 0 && (!d_w || !d_val))) return set_error(DAG_ERR_INVALID, "null argument");
    return launch_normalize(p, d_w, d_val, d_s, (cudaStream_t)stream);
}

extern "C" int dag_plan_set_worker_cap(dag_plan* p, int32_t max_workers)
{
    if (!p || max_workers < 0) return set_error(DAG_ERR_INVALID, "bad argument");
    p->worker_cap = max_workers;
    return DAG_OK;
}

extern "C" int dag_gather_f32(const float* d_src, const int32_t* d_idx, int64_t m, float* d_out, void* stream)
{
    if (m < 0 || (m > 0 && (!d_src || !d_idx || !d_out))) return set_error(DAG_ERR_INVALID, "bad argument");
    if (m == 0) return DAG_OK;
    k_gather_f32<<<2048, 256, 0, (cudaStream_t)stream>>>(d_src, d_idx, d_out, m);
    DAG_CUDA(cudaGetLastError());
    return DAG_OK;
}

extern "C" int dag_debug_stall_staging_once(dag_plan* p, int32_t timeout_ms)
{
    if (!p || timeout_ms < 1) return set_error(DAG_ERR_INVALID, "bad argument");
    p->stall_staging_once = 1;
    p->skip_timeout_ns = (long long)timeout_ms * 1000000LL;
    return DAG_OK;
}

extern "C" int dag_debug_skip_barrier_once(dag_plan* p, int32_t timeout_ms)
{
    if (!p || timeout_ms < 1) return set_error(DAG_ERR_INVALID, "bad argument");
    p->skip_barrier_once = 1;
    p->skip_timeout_ns = (long long)timeout_ms * 1000000LL;
    return DAG_OK;
}
