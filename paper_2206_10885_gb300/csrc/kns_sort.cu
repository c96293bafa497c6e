// kns_sort.cu -- per-wave counting sort of samples by cell (configuration independent).
//
// scan:    turns the wave's per-key sample counts into exclusive offsets off[0..nkeys] and per-key
//          tile offsets tile_off[0..nkeys] (ceil(count / tile) tiles per key), writes one descriptor
//          {key, first sample, samples} per tile, publishes the tile counts, and clears the next
//          wave's counters.  Two launches of up to 128 blocks: each block sums a contiguous range of
//          keys (wave_scan_part_kernel), then each block adds the sums of the blocks before it to a
//          block-wide scan of its range (wave_scan_final_kernel) -- no block waits for another.
// scatter: each sample goes to off[cell] + (its rank among the wave's samples of that cell);
//          lanes of a warp that share a cell take consecutive slots with one atomic.
#include "kns_wave.cuh"

namespace kns {

constexpr int SCAN_THREADS = 1024;

// Inclusive block-wide scan of two values at once (1024 threads).
__device__ __forceinline__ void block_scan2(int &a, int &b, int *wa, int *wb) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int ya = __shfl_up_sync(FULL, a, o), yb = __shfl_up_sync(FULL, b, o);
        if (lane >= o) {
            a += ya;
            b += yb;
        }
    }
    if (lane == 31) {
        wa[warp] = a;
        wb[warp] = b;
    }
    __syncthreads();
    if (warp == 0) {
        int sa = wa[lane], sb = wb[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int ya = __shfl_up_sync(FULL, sa, o), yb = __shfl_up_sync(FULL, sb, o);
            if (lane >= o) {
                sa += ya;
                sb += yb;
            }
        }
        wa[lane] = sa;
        wb[lane] = sb;
    }
    __syncthreads();
    if (warp > 0) {
        a += wa[warp - 1];
        b += wb[warp - 1];
    }
}

constexpr int SCAN_MAX_BLOCKS = 128;     // WaveCtrl::scan_part entries
constexpr int SCAN_KEYS_PER_BLOCK = 4096;
inline int scan_blocks(int nkeys) {
    const int b = (nkeys + SCAN_KEYS_PER_BLOCK - 1) / SCAN_KEYS_PER_BLOCK;
    return b < 1 ? 1 : (b > SCAN_MAX_BLOCKS ? SCAN_MAX_BLOCKS : b);
}
// keys [k0, k1) of scan block b
__device__ __forceinline__ void scan_range(int nkeys, int b, int &k0, int &k1) {
    const int per = (nkeys + gridDim.x - 1) / gridDim.x;
    k0 = min(nkeys, b * per);
    k1 = min(nkeys, k0 + per);
}
__device__ __forceinline__ int key_tile(const WaveArgs &a, int c) { return c < a.NC ? a.btile : a.btile_bf; }

// Block sums of the round's samples and tiles per key range; clears the next round's counters.
__global__ void __launch_bounds__(SCAN_THREADS) wave_scan_part_kernel(WaveArgs a, int cur) {
    __shared__ int wa[32], wb[32];
    const int nxt = cur ^ 1, NK = a.nkeys;
    int k0, k1;
    scan_range(NK, blockIdx.x, k0, k1);
    for (int c = k0 + threadIdx.x; c < k1; c += SCAN_THREADS) {  // nothing reads them during this round
        a.count[nxt][c] = 0;
        a.fill[nxt][c] = 0;
    }
    const int n_live = a.ctrl->n_live[cur];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctrl->n_live[nxt] = 0;
        a.ctrl->next_tile = 0;
        a.ctrl->next_tile_bf = 0;
        a.ctrl->n_pend[cur] = 0;  // this round's pending list (round k - 2's advance has read it)
        // a small round is finished one warp per ray (its count includes the rays the previous round left
        // in empty voxels, which join the next round: the same rule as the persistent BF16 trace)
        a.ctrl->tail = n_live + a.ctrl->n_pend[nxt] <= a.tail_max ? 1 : 0;
    }
    if (n_live == 0) return;
    int sum = 0, tiles = 0;
    for (int c = k0 + threadIdx.x; c < k1; c += SCAN_THREADS) {
        const int n = a.count[cur][c], bt = key_tile(a, c);
        sum += n;
        tiles += (n + bt - 1) / bt;
    }
    block_scan2(sum, tiles, wa, wb);
    if (threadIdx.x == SCAN_THREADS - 1) {
        a.ctrl->scan_part[0][blockIdx.x] = sum;
        a.ctrl->scan_part[1][blockIdx.x] = tiles;
    }
}

// Offsets, tile offsets and tile descriptors of each block's key range: the sums of the blocks before
// it plus a block-wide exclusive scan (each thread a contiguous run of keys, so descriptors come out
// in key order).
__global__ void __launch_bounds__(SCAN_THREADS) wave_scan_final_kernel(WaveArgs a, int cur) {
    __shared__ int wa[32], wb[32];
    __shared__ int base[2];
    const int NK = a.nkeys;
    if (a.ctrl->n_live[cur] == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.ctrl->n_tiles = 0;
            a.ctrl->n_tiles_fine = 0;
        }
        return;
    }
    if (threadIdx.x < 32) {
        int bs = 0, bt = 0;
        for (int i = threadIdx.x; i < (int)blockIdx.x; i += 32) {
            bs += a.ctrl->scan_part[0][i];
            bt += a.ctrl->scan_part[1][i];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            bs += __shfl_xor_sync(FULL, bs, o);
            bt += __shfl_xor_sync(FULL, bt, o);
        }
        if (threadIdx.x == 0) {
            base[0] = bs;
            base[1] = bt;
        }
    }
    __syncthreads();
    int k0, k1;
    scan_range(NK, blockIdx.x, k0, k1);
    const int per = (k1 - k0 + SCAN_THREADS - 1) / SCAN_THREADS;
    const int c0 = min(k1, k0 + (int)threadIdx.x * per), c1 = min(k1, c0 + per);
    int sum = 0, tiles = 0;
    for (int c = c0; c < c1; ++c) {
        const int n = a.count[cur][c], bt = key_tile(a, c);
        sum += n;
        tiles += (n + bt - 1) / bt;
    }
    int incl_s = sum, incl_t = tiles;
    block_scan2(incl_s, incl_t, wa, wb);
    int run_s = base[0] + incl_s - sum, run_t = base[1] + incl_t - tiles;
    for (int c = c0; c < c1; ++c) {
        const int n = a.count[cur][c], bt = key_tile(a, c);
        a.off[c] = run_s;
        a.tile_off[c] = run_t;
        if (c == a.NC) a.ctrl->n_tiles_fine = run_t;  // first BF16 key: FP32 tiles end here
        for (int i = 0; i < n; i += bt) a.tiles[run_t++] = make_int4(c, run_s + i, min(bt, n - i), 0);
        run_s += n;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == SCAN_THREADS - 1) {
        a.off[NK] = base[0] + incl_s;
        a.tile_off[NK] = base[1] + incl_t;
        a.ctrl->n_tiles = base[1] + incl_t;
        // FP32 renders: every tile is an FP32 tile; BF16 renders: every tile is a tensor-core tile
        if (NK == a.NC) a.ctrl->n_tiles_fine = a.coarse ? 0 : base[1] + incl_t;
    }
}

__global__ void __launch_bounds__(256) wave_scatter_kernel(WaveArgs a, int cur) {
    const int n = a.ctrl->n_live[cur];
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * blockDim.x;
    const int bound = (n + 31) & ~31;  // warp-uniform loop bound
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < bound; i += stride) {
        const bool pred = i < n;
        const int c = pred ? a.qcell[cur][i] : 0;
        const int r = pred ? a.q[cur][i] : 0;
        const unsigned m = __ballot_sync(FULL, pred);
        if (pred) {
            const unsigned grp = __match_any_sync(m, c);
            const int leader = __ffs(grp) - 1;
            int base = 0;
            if (lane == leader) base = __ldg(a.off + c) + atomicAdd(a.fill[cur] + c, __popc(grp));
            base = __shfl_sync(grp, base, leader);
            a.sorted[base + __popc(grp & lanemask_lt())] = r;
        }
    }
}

// Coarse occupancy: block (bx, by, bz) of 8^3 voxels is set iff any of its voxels is occupied.
// The 8 voxels of a block row are 8 consecutive bits of one 32-bit word (res % 8 == 0).
__global__ void coarse_occupancy_kernel(const uint32_t *occ, int res, uint32_t *coarse) {
    const int cres = res / 8;
    const int64_t nb = (int64_t)cres * cres * cres;
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool any = false;
    if (b < nb) {
        const int bx = (int)(b % cres), by = (int)((b / cres) % cres), bz = (int)(b / ((int64_t)cres * cres));
        for (int z = 0; z < 8 && !any; ++z)
            for (int y = 0; y < 8 && !any; ++y) {
                const int64_t v = 8 * bx + (int64_t)res * ((8 * by + y) + (int64_t)res * (8 * bz + z));
                any = ((occ[v >> 5] >> (v & 31)) & 0xffu) != 0;
            }
    }
    const unsigned ball = __ballot_sync(FULL, any);
    if ((threadIdx.x & 31) == 0 && b < nb) coarse[b >> 5] = ball;
}

// Index box of the occupied voxels: bounds[0..2] = the smallest x, y, z index of a set bit, bounds[3..5]
// the largest (the caller initialises them to res and -1).  One thread per 32-bit word.
__global__ void occ_bounds_kernel(const uint32_t *occ, int res, int *bounds) {
    const int64_t nvox = (int64_t)res * res * res, nw = (nvox + 31) / 32;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nw) return;
    uint32_t m = occ[i];
    int lo[3] = {res, res, res}, hi[3] = {-1, -1, -1};
    while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        const int64_t v = 32 * i + b;
        if (v >= nvox) break;
        const int c[3] = {(int)(v % res), (int)((v / res) % res), (int)(v / ((int64_t)res * res))};
        for (int k = 0; k < 3; ++k) {
            lo[k] = min(lo[k], c[k]);
            hi[k] = max(hi[k], c[k]);
        }
    }
    if (hi[0] >= 0)
        for (int k = 0; k < 3; ++k) {
            atomicMin(bounds + k, lo[k]);
            atomicMax(bounds + 3 + k, hi[k]);
        }
}

cudaError_t launch_occ_bounds(const uint32_t *occ, int res, int *bounds, cudaStream_t s) {
    const int64_t nw = ((int64_t)res * res * res + 31) / 32;
    occ_bounds_kernel<<<(unsigned)((nw + 127) / 128), 128, 0, s>>>(occ, res, bounds);
    return cudaGetLastError();
}

cudaError_t launch_coarse_occupancy(const uint32_t *occ, int res, uint32_t *coarse, cudaStream_t s) {
    const int64_t nb = (int64_t)(res / 8) * (res / 8) * (res / 8);
    coarse_occupancy_kernel<<<(unsigned)((nb + 127) / 128), 128, 0, s>>>(occ, res, coarse);
    return cudaGetLastError();
}

cudaError_t launch_wave_scan(const WaveArgs &a, int cur, cudaStream_t s) {
    const int nb = scan_blocks(a.nkeys);
    wave_scan_part_kernel<<<nb, SCAN_THREADS, 0, s>>>(a, cur);
    wave_scan_final_kernel<<<nb, SCAN_THREADS, 0, s>>>(a, cur);
    return cudaGetLastError();
}

cudaError_t launch_wave_scatter(const WaveArgs &a, int cur, int blocks, cudaStream_t s) {
    wave_scatter_kernel<<<blocks, 256, 0, s>>>(a, cur);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- hits by cell (shading tiles)
// After the last round: the hit list is counting-sorted by the cell of each hit into `sorted`, with
// off[c] / tile_off[c] (tiles of `tile` hits, the shading kernel's tile), one descriptor per tile in
// `tiles` and the tile count in ctrl->n_tiles.  Uses the wave's count[0], fill[0], off, tile_off and sorted buffers, which the
// rounds no longer need.
__global__ void __launch_bounds__(256) wave_hit_count_kernel(WaveArgs a) {
    const int n = a.ctrl->n_hits;
    const int bound = (n + 31) & ~31;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < bound; i += gridDim.x * blockDim.x) {
        const bool pred = i < n;
        const int c = pred ? a.cell_ray[a.hits[i]] : 0;
        warp_count_cells(a.count[0], pred, c);
    }
}

__global__ void __launch_bounds__(SCAN_THREADS) wave_hit_scan_kernel(WaveArgs a, int tile) {
    // one block walks the cells in chunks of SCAN_THREADS consecutive cells (coalesced loads), each
    // chunk scanned across the block and offset by the chunks before it
    __shared__ int wa[32], wb[32], s_base[2];
    const int NC = a.NC;
    if (threadIdx.x == 0) s_base[0] = s_base[1] = 0;
    __syncthreads();
    for (int c0 = 0; c0 < NC; c0 += SCAN_THREADS) {
        const int c = c0 + (int)threadIdx.x;
        const int n = c < NC ? a.count[0][c] : 0, nt = (n + tile - 1) / tile;
        int incl_s = n, incl_t = nt;
        block_scan2(incl_s, incl_t, wa, wb);
        const int base_s = s_base[0], base_t = s_base[1];
        if (c < NC) {
            int run_s = base_s + incl_s - n, run_t = base_t + incl_t - nt;
            a.off[c] = run_s;
            a.tile_off[c] = run_t;
            a.fill[0][c] = 0;
            for (int i = 0; i < n; i += tile) a.tiles[run_t++] = make_int4(c, run_s + i, min(tile, n - i), 0);
        }
        __syncthreads();  // every thread has read the bases (and block_scan2's partials)
        if (threadIdx.x == SCAN_THREADS - 1) {
            s_base[0] = base_s + incl_s;
            s_base[1] = base_t + incl_t;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.off[NC] = s_base[0];
        a.tile_off[NC] = s_base[1];
        a.ctrl->n_tiles = s_base[1];
    }
}

__global__ void __launch_bounds__(256) wave_hit_scatter_kernel(WaveArgs a) {
    const int n = a.ctrl->n_hits;
    const int lane = threadIdx.x & 31;
    const int bound = (n + 31) & ~31;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < bound; i += gridDim.x * blockDim.x) {
        const bool pred = i < n;
        const int r = pred ? a.hits[i] : 0;
        const int c = pred ? a.cell_ray[r] : 0;
        const unsigned m = __ballot_sync(FULL, pred);
        if (pred) {
            const unsigned grp = __match_any_sync(m, c);
            const int leader = __ffs(grp) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(a.fill[0] + c, __popc(grp));
            base = __shfl_sync(grp, base, leader);
            a.sorted[a.off[c] + base + __popc(grp & lanemask_lt())] = r;
        }
    }
}

cudaError_t launch_hit_sort(const WaveArgs &a, int tile, int sm_count, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(a.count[0], 0, sizeof(int) * (a.NC + 1), s);
    if (e != cudaSuccess) return e;
    wave_hit_count_kernel<<<sm_count * 4, 256, 0, s>>>(a);
    wave_hit_scan_kernel<<<1, SCAN_THREADS, 0, s>>>(a, tile);
    wave_hit_scatter_kernel<<<sm_count * 4, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// Rays whose last step left them in an empty occupancy voxel: the DDA to the next occupied voxel (or
// out of the grid: a miss), the cycle test on the position reached, and the emit -- what the tile
// kernels' advance_ray would have done in place, one round later.  One thread per ray: many
// independent voxel walks hide each other's memory latency, and the kernel runs beside the next
// round's tiles.
__global__ void __launch_bounds__(256) wave_advance_kernel(GridView g, WaveArgs a, int p) {
    const int n = a.ctrl->n_pend[p];
    const int stride = gridDim.x * blockDim.x;
    const int bound = (n + 31) & ~31;  // warp-uniform loop bound
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < bound; i += stride) advance_pending(g, a, p, p, i, n);
}

cudaError_t launch_wave_advance(const GridView &g, const WaveArgs &a, int p, int sm_count, cudaStream_t s) {
    wave_advance_kernel<<<sm_count * 4, 256, 0, s>>>(g, a, p);
    return cudaGetLastError();
}

}  // namespace kns
