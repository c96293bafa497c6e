// kns_tc.cu -- the BF16 precision form of the sphere trace on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory).
// kns:instantiate (compiled once per grid configuration)
//
// One round of a BF16 render: a block of 128 threads takes tiles of up to 128 same-cell samples and
// evaluates the cell's SDF MLP (Eq. 2, trace form: d only) for
// the whole tile as one [128 x K] x [K x W] product per hidden layer:
//   - thread s owns sample s = row s of the activation matrix = lane s of the accumulator;
//   - the cell's weights (BF16, in the canonical K-major layout of kns_tc.cuh) are staged in shared
//     memory by one TMA bulk copy, kept while consecutive tiles share the cell;
//   - every activation and weight is split into a BF16 high part and a BF16 low part
//     (x = hi + lo to ~16 bits), and a layer is the sum of three tensor-core products
//     A_hi W_hi + A_lo W_hi + A_hi W_lo accumulated in FP32 in tensor memory (the lo x lo term is
//     below the FP32 accumulation error of the others), so d carries ~1e-5 relative error instead of
//     plain BF16's ~4e-3 -- enough for the BF16 phase to take the trace to the surface itself;
//   - the activation matrices A_hi, A_lo live in tensor memory beside the accumulator (thread s
//     writes row s with tcgen05.st), so the MMA takes A from tensor memory and B from shared memory,
//     and a worker's shared memory holds only the cell's weights;
//   - one thread issues the layer's tcgen05.mma chain and commits it to an mbarrier; the block then
//     reads its accumulator rows with tcgen05.ld, adds the bias and applies the softplus in FP32,
//     and writes the next layer's A_hi / A_lo rows back to tensor memory (or, after the last hidden
//     layer, forms d with the FP32 d row);
//   - each sample is then tested and stepped: |d| < eps_coarse ends the BF16 trace -- the ray joins
//     the hit list at this t, where the shading re-evaluates it in FP32 (and kns_fp32.cu's refinement
//     takes the last FP32 steps when that evaluation is not within eps); a step into an empty
//     occupancy voxel goes to the round's pending list (wave_advance_kernel); other samples go to
//     the next round -- or, while enough of them stay in this cell, are evaluated again at once
//     (in-tile stepping).  Keys of a BF16 render are the cells; every tile is a tensor-core tile.
// Every wait (weights, tensor-core completion) is bounded and reports KNS_ERR_TIMEOUT.
#include <algorithm>

#include "kns_tc.cuh"
#include "kns_wave.cuh"

namespace kns {

// The cell layout of kns_tc.cuh for configuration C (a worker's shared memory), and the worker's
// tensor-memory columns: the FP32 accumulator (W columns), then the activation matrices A_hi and A_lo
// (128 lanes = rows, the widest layer input along the columns, two BF16 values per column).
template <class C>
struct TcLayout {
    static constexpr int W = C::W, H = C::H;
    static constexpr int K0 = tc::k0_of(C::IN);
    static constexpr int KA = K0 > W ? K0 : W;
    __host__ __device__ static constexpr int hi(int l) { return tc::w_hi(l, W, K0); }
    __host__ __device__ static constexpr int lo(int l) { return tc::w_lo(l, W, K0); }
    __host__ __device__ static constexpr int kin(int l) { return l == 0 ? K0 : W; }
    static constexpr int BIAS = tc::bias_off(W, H, K0);
    static constexpr int DROW = tc::drow_off(W, H, K0);
    static constexpr int SIZE = tc::cell_bytes(W, H, K0);
    static constexpr int SMEM = SIZE;
    static constexpr int ACOLS = KA / 2;            // tensor-memory columns of one activation matrix
    static constexpr int TCOLS = W + 2 * ACOLS;     // a worker's tensor-memory columns
};

// Writes values v[0..15] as columns k0..k0+15 of this thread's row of the activation matrices in
// tensor memory (ta: A_hi's first column in this warp's lanes; A_lo follows ACOLS columns later).
// Every thread of the warp takes part.
template <class T>
__device__ __forceinline__ void put16(uint32_t ta, int k0, const float *v) {
    uint32_t h[8], l[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        const __nv_bfloat162 ll =
            __floats2bfloat162_rn(v[2 * i] - __low2float(hh), v[2 * i + 1] - __high2float(hh));
        h[i] = *reinterpret_cast<const uint32_t *>(&hh);
        l[i] = *reinterpret_cast<const uint32_t *>(&ll);
    }
    tc::tmem_st8(ta + (uint32_t)(k0 / 2), h);
    tc::tmem_st8(ta + (uint32_t)(T::ACOLS + k0 / 2), l);
}

// Encoding of Eq. 1 for row `row` (K0 columns, zero beyond IN): sin and cos of pi p once, then the
// double-angle recurrences sin 2a = 2 sin a cos a, cos 2a = (cos a - sin a)(cos a + sin a) for the
// higher frequencies (error ~1e-6 at the highest, below the hi/lo split's resolution).
template <class C, class T>
__device__ __forceinline__ void encode_row(uint32_t ta, float px, float py, float pz) {
    float in[T::K0];
    in[0] = px;
    in[1] = py;
    in[2] = pz;
    float s[3], c[3];
    sincospif(px, &s[0], &c[0]);
    sincospif(py, &s[1], &c[1]);
    sincospif(pz, &s[2], &c[2]);
#pragma unroll
    for (int k = 0; k < C::L; ++k) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            in[3 + 6 * k + a] = s[a];
            in[3 + 6 * k + 3 + a] = c[a];
            const float s2 = 2.f * s[a] * c[a], c2 = (c[a] - s[a]) * (c[a] + s[a]);
            s[a] = s2;
            c[a] = c2;
        }
    }
#pragma unroll
    for (int k = C::IN; k < T::K0; ++k) in[k] = 0.f;
#pragma unroll
    for (int k0 = 0; k0 < T::K0; k0 += 16) put16<T>(ta, k0, in + k0);
}

// One hidden layer on the tensor cores: D = A_hi W_hi + A_lo W_hi + A_hi W_lo over K = kin(l), A in
// tensor memory (ta: A_hi's first column; one K = 16 slice is 8 columns), W in shared memory.
template <class T>
__device__ __forceinline__ void issue_layer(uint32_t tmem, uint32_t ta, uint32_t w_base, int l, uint64_t *bar) {
    constexpr uint32_t idesc = tc::idesc_bf16_f32(128, T::W);
    const int K = T::kin(l);
    const uint32_t sbo = 16u * K, w_hi = w_base + T::hi(l), w_lo = w_base + T::lo(l);
    for (int ks = 0; ks < K / 16; ++ks) {
        const uint32_t o = 256u * ks, ah = ta + 8u * ks, al = ta + (uint32_t)T::ACOLS + 8u * ks;
        const uint64_t bh = tc::smem_desc(w_hi + o, 128, sbo), bl = tc::smem_desc(w_lo + o, 128, sbo);
        tc::mma_bf16_ta(tmem, ah, bh, idesc, ks > 0 ? 1u : 0u);
        tc::mma_bf16_ta(tmem, al, bh, idesc, 1u);
        tc::mma_bf16_ta(tmem, ah, bl, idesc, 1u);
    }
    tc::mma_commit(bar);
}

// softplus_beta(s) = max(s, 0) + ln(1 + e^(-beta |s|)) / beta with the change of base to 2^x and log2 y
// on the multi-function unit (PTX ex2.approx / lg2.approx) and the constants folded:
// k_e = -beta log2(e), k_l = ln(2) / beta.
__device__ __forceinline__ float softplus_mufu(float s, float k_e, float k_l) {
    float e, l;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(k_e * fabsf(s)));
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(1.f + e));
    return fmaf(l, k_l, fmaxf(s, 0.f));
}

constexpr uint32_t kTcPolls = 1u << 26;    // bound of every mbarrier wait

// A warpgroup worker: 128 threads that evaluate tiles on their own weights, activation matrices,
// tensor-memory columns and mbarriers, synchronised by their own named barrier.
struct TcWorker {
    unsigned char *wsm;       // shared: the cell's weights
    uint64_t *bar_w, *bar_mma;
    int *s_tile;              // 4 ints: key, first sample, samples, fresh
    int *s_red;               // 8 ints: per-warp partial counts, two alternating sets
    int *s_fail;              // set by any thread whose wait ran out; read after the next barrier
    uint32_t tmem;            // first tensor-memory column of the worker's accumulator (A_hi, A_lo follow)
    int bar;                  // named barrier id
    int tid, warp;            // thread (0..127) and warp (0..3) within the worker
    int cached;               // cell of the staged weights
    uint32_t ph_w, ph_mma;    // mbarrier phases
    bool w_pending, mma_pending;  // a weight copy / a tensor-core chain in flight
    unsigned n_eval;          // samples this thread evaluated
    int red;                  // which set of s_red the next count uses
};

__device__ __forceinline__ void wg_bar(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }

// Threads of the worker whose p is true (every thread of the worker calls it).  The two sets of partial
// counts alternate: a set is written again only two counts later, after every thread has passed the
// barrier of the count in between, so one barrier per count suffices.
__device__ __forceinline__ int wg_count(TcWorker &w, bool p) {
    const unsigned b = __ballot_sync(FULL, p);
    int *set = w.s_red + 4 * w.red;
    w.red ^= 1;
    if ((w.tid & 31) == 0) set[w.warp] = __popc(b);
    wg_bar(w.bar);
    return set[0] + set[1] + set[2] + set[3];
}

// One round of the BF16 trace for one worker: tiles [0, n_tiles) of the round, a contiguous run per
// worker (gi of nw workers) or handed out one at a time.  Returns false when a wait ran out.
template <class C>
__device__ bool tc_round(TcWorker &w, const GridView &g, const WaveArgs &a, int cur, int n_tiles, int gi, int nw) {
    using T = TcLayout<C>;
    const int tid = w.tid, nxt = cur ^ 1;
    const uint32_t w_base = tc::saddr(w.wsm), ta = w.tmem + (uint32_t)T::W;  // A_hi's first column
    const uint32_t t_lane = w.tmem + ((uint32_t)(32 * w.warp) << 16);       // this warp's lanes
    const uint32_t ta_lane = ta + ((uint32_t)(32 * w.warp) << 16);
    const float *bias = reinterpret_cast<const float *>(w.wsm + T::BIAS);
    const float *drow = reinterpret_cast<const float *>(w.wsm + T::DROW);
    const int per = (n_tiles + nw - 1) / nw;
    int next_static = gi * per;
    const int end_static = min(n_tiles, next_static + per);
    const bool cycles = a.t_hist != nullptr;
    const float k_e = -g.beta * 1.44269504088896341f, k_l = 0.693147180559945309f * g.inv_beta;
    // thread 0 runs two tiles ahead: the next tile's descriptor is loaded and the one after it claimed
    // while this tile is evaluated, so neither the claim nor the descriptor load waits at a tile's start
    auto claim = [&]() -> int {
        const int tile = a.static_tiles ? (next_static < end_static ? next_static : n_tiles)
                                        : atomicAdd(&a.ctrl->next_tile_bf, 1);
        ++next_static;
        return tile;
    };
    int4 d_next = make_int4(-1, 0, 0, 0);
    int t_after = n_tiles;
    if (tid == 0) {
        const int t0 = claim();
        if (t0 < n_tiles) d_next = a.tiles[t0];
        t_after = claim();
    }
    for (;;) {
        if (tid == 0) {
            const int4 d = d_next;
            d_next = make_int4(-1, 0, 0, 0);
            if (d.x >= 0 && t_after < n_tiles) {
                d_next = a.tiles[t_after];
                t_after = claim();
            }
            const bool fresh = d.x >= 0 && d.x != w.cached;
            if (fresh) bulk_load(w.wsm, a.wb + (int64_t)d.x * a.wb_stride, T::SIZE, w.bar_w);
            w.s_tile[0] = d.x;
            w.s_tile[1] = d.y;
            w.s_tile[2] = d.z;
            w.s_tile[3] = fresh;
        }
        wg_bar(w.bar);
        const int c = w.s_tile[0], start = w.s_tile[1], len = w.s_tile[2];
        const bool fresh = w.s_tile[3] != 0;
        if (c < 0) break;
        w.cached = c;
        const GridView gt = sub_grid(g, c / g.ncl);  // the grid of the tile's cell (a stack of grids)
        bool active = tid < len;
        int r = 0, steps = 0;
        float t = 0.f, t0 = 0.f, tf = 0.f;
        float4 hist = no_history();
        int4 trap = trap_empty();
        Ray ray{};
        if (active) {
            r = a.sorted[start + tid];
            t = a.t_ray[r];
            steps = a.steps_ray[r];
            if (cycles) hist = a.t_hist[r];
            if (a.trap) trap = a.trap[r];
            int cam;
            ray = ray_of(a, r, cam);
            clip_box(gt, ray, t0, tf);
        }
        if (fresh) w.w_pending = true;
        for (int it = 0;; ++it) {
            // (tensor-memory stores are warp-wide: a warp with a live sample encodes every lane's row;
            // the rows of idle lanes are never read back)
            if (__any_sync(FULL, active))
                encode_row<C, T>(ta_lane, fmaf(t, ray.wx, ray.ox), fmaf(t, ray.wy, ray.oy), fmaf(t, ray.wz, ray.oz));
            tc::tmem_wait_st();
            // a wait that runs out raises the worker's failure flag, read after the next barrier, where the
            // worker leaves; the thread itself ignores its sample from then on (lost)
            bool lost = false;
            if (w.w_pending) {
                if (mbar_wait(w.bar_w, w.ph_w, kTcPolls)) {
                    w.ph_w ^= 1u;
                    w.w_pending = false;
                } else {
                    *w.s_fail = 1;
                    lost = true;
                }
            }
            // the hidden layers: products on the tensor cores, bias + softplus + split on the worker
            float d = 0.f;
            for (int l = 0; l < C::H; ++l) {
                wg_bar(w.bar);
                if (*w.s_fail) return false;
                if (tid == 0) {
                    tc::fence_after_sync();
                    issue_layer<T>(w.tmem, ta, w_base, l, w.bar_mma);
                }
                w.mma_pending = true;
                if (mbar_wait(w.bar_mma, w.ph_mma, kTcPolls)) {
                    w.ph_mma ^= 1u;
                    w.mma_pending = false;
                } else {
                    *w.s_fail = 1;
                    lost = true;
                }
                tc::fence_after_sync();
                if (__any_sync(FULL, active)) {
                    float dacc = drow[T::W];  // the d row's bias (stored right after the row)
#pragma unroll
                    for (int c0 = 0; c0 < T::W; c0 += 16) {
                        float v[16];
                        tc::tmem_ld16(t_lane + (uint32_t)c0, v);
                        const float4 *b4 = reinterpret_cast<const float4 *>(bias + l * T::W + c0);
#pragma unroll
                        for (int i = 0; i < 16; i += 4) {
                            const float4 b = b4[i / 4];
                            v[i] = softplus_mufu(v[i] + b.x, k_e, k_l);
                            v[i + 1] = softplus_mufu(v[i + 1] + b.y, k_e, k_l);
                            v[i + 2] = softplus_mufu(v[i + 2] + b.z, k_e, k_l);
                            v[i + 3] = softplus_mufu(v[i + 3] + b.w, k_e, k_l);
                        }
                        if (l + 1 < C::H) {
                            put16<T>(ta_lane, c0, v);
                        } else {
                            const float4 *d4 = reinterpret_cast<const float4 *>(drow + c0);
#pragma unroll
                            for (int i = 0; i < 16; i += 4) {
                                const float4 dw = d4[i / 4];
                                dacc = fmaf(dw.x, v[i], dacc);
                                dacc = fmaf(dw.y, v[i + 1], dacc);
                                dacc = fmaf(dw.z, v[i + 2], dacc);
                                dacc = fmaf(dw.w, v[i + 3], dacc);
                            }
                        }
                    }
                    d = dacc;
                }
                tc::tmem_wait_st();
                tc::fence_before_sync();
            }
            // outcome: 0 none, 1 converged (hit list), 2 miss (written), 3 pending, 4 emit to ncell
            int outcome = 0, ncell = -1;
            const float t_eval = t;
            if (lost) active = false;
            w.n_eval += active ? 1u : 0u;
            if (active) {
                ++steps;
                if (fabsf(d) < a.eps_coarse) {
                    outcome = 1;  // the BF16 trace has converged: FP32 re-evaluates this step
                } else if (a.trap && trap_step(trap, t, d, c, a.trap_span, 5.f * a.eps_coarse)) {
                    outcome = 2;  // trapped at a seam: the budget miss of the plain iteration
                    write_miss(a, r, a.max_steps);
                } else {
                    t += d;
                    if (t > tf || t < t0 || steps >= a.max_steps) {
                        outcome = 2;
                        write_miss(a, r, steps);
                    } else {
                        ncell = advance_fast(gt, ray, t);
                        if (ncell == -2) {
                            outcome = 3;
                        } else if (cycles && cycle_step_tol(hist, t_eval, t)) {
                            outcome = 2;
                            write_miss(a, r, a.max_steps);
                            ncell = -1;
                        } else {
                            outcome = 4;
                        }
                    }
                }
            }
            const bool cand = outcome == 4 && ncell == c && it + 1 < a.inner_steps_bf;
            const int n_cand = wg_count(w, cand);
            if (*w.s_fail) return false;
            const bool again = n_cand > 0 && n_cand >= a.min_active_bf;
            const bool stay = cand && again;
            {
                const bool hit = outcome == 1, emit = outcome == 4 && !stay, pend = outcome == 3;
                if (hit) a.cell_ray[r] = c;
                if (hit || emit || pend) {
                    a.t_ray[r] = t;
                    a.steps_ray[r] = steps;
                }
                if (cycles && emit) a.t_hist[r] = hist;
                if (a.trap && (emit || pend)) a.trap[r] = trap;
                const int hp = warp_append(&a.ctrl->n_hits, hit);
                if (hit) a.hits[hp] = r;
                const int qp = warp_append(&a.ctrl->n_live[nxt], emit);
                if (emit) {
                    a.q[nxt][qp] = r;
                    a.qcell[nxt][qp] = ncell;
                }
                warp_count_cells(a.count[nxt], emit, ncell);
                const int pp = warp_append(&a.ctrl->n_pend[cur], pend);
                if (pend) {
                    a.pend_r[cur][pp] = r;
                    a.pend_t[cur][pp] = t_eval;
                }
                active = stay;
            }
            if (!again) break;
        }
        wg_bar(w.bar);  // every thread is done with the weights and the tile's state
    }
    return true;
}

// The end of a worker: after a failed wait, report it and let what is in flight land (bounded); add
// the worker's evaluation count.
__device__ __forceinline__ void tc_worker_done(TcWorker &w, const WaveArgs &a, bool ok) {
    if (!ok) {
        if (w.tid == 0) atomicCAS(a.status, 0, (int)6 /* KNS_ERR_TIMEOUT */);
        if (w.w_pending) mbar_wait(w.bar_w, w.ph_w, kTcPolls);
        if (w.mma_pending) mbar_wait(w.bar_mma, w.ph_mma, kTcPolls);
    }
    const unsigned long long n = warp_sum_u64(w.n_eval);
    if ((w.tid & 31) == 0 && n) atomicAdd(&a.ctrl->samples_bf16, n);
}

// Tensor-memory columns allocated for n: the next power of two, at least 32.
__host__ __device__ constexpr uint32_t pow2_cols(int n) {
    return n <= 32 ? 32u : n <= 64 ? 64u : n <= 128 ? 128u : n <= 256 ? 256u : 512u;
}

// ---------------------------------------------------------------- one round per launch
template <class C>
__global__ void __launch_bounds__(128) wave_eval_tc_kernel(GridView g, WaveArgs a, int cur) {
    using T = TcLayout<C>;
    extern __shared__ __align__(1024) unsigned char dyn[];
    __shared__ __align__(8) uint64_t bar_w, bar_mma;
    __shared__ uint32_t s_tmem;
    __shared__ int s_tile[4], s_red[8], s_fail;
    const int n_tiles = a.ctrl->n_tiles;
    // uniform over the block, before any tensor memory is held; a small round (at most tail_rays rays)
    // is finished one warp per ray by wave_tail_warp_kernel
    if (n_tiles <= 0 || a.ctrl->tail) return;
    const int tid = threadIdx.x;
    constexpr uint32_t NCOL = pow2_cols(T::TCOLS);
    if (tid < 32) tc::tmem_alloc(&s_tmem, NCOL);
    if (tid == 0) {
        mbar_init(&bar_w, 1);
        mbar_init(&bar_mma, 1);
        s_fail = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    TcWorker w{dyn, &bar_w, &bar_mma, s_tile, s_red, &s_fail, s_tmem, 1, tid, tid >> 5, -1, 0u, 0u,
               false, false, 0u, 0};
    const bool ok = tc_round<C>(w, g, a, cur, n_tiles, blockIdx.x, gridDim.x);
    tc_worker_done(w, a, ok);
    tc::fence_before_sync();
    __syncthreads();
    if (tid < 32) tc::tmem_free(s_tmem, NCOL);
}

// ---------------------------------------------------------------- every round in one launch
// Inclusive scan of two values over the block (blockDim.x a multiple of 32, at most 1024 threads).
__device__ __forceinline__ void block_scan2_any(int &x, int &y, int *wx, int *wy) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(FULL, x, o), b = __shfl_up_sync(FULL, y, o);
        if (lane >= o) {
            x += a;
            y += b;
        }
    }
    if (lane == 31) {
        wx[warp] = x;
        wy[warp] = y;
    }
    __syncthreads();
    if (warp == 0) {
        int sx = lane < nw ? wx[lane] : 0, sy = lane < nw ? wy[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int a = __shfl_up_sync(FULL, sx, o), b = __shfl_up_sync(FULL, sy, o);
            if (lane >= o) {
                sx += a;
                sy += b;
            }
        }
        if (lane < nw) {
            wx[lane] = sx;
            wy[lane] = sy;
        }
    }
    __syncthreads();
    if (warp > 0) {
        x += wx[warp - 1];
        y += wy[warp - 1];
    }
    __syncthreads();
}

// Workers per block of the persistent trace: as many as shared memory and the 512 tensor-memory
// columns hold, at most 4 (four warpgroups of 128 threads: 128 registers a thread).
template <class C>
__host__ __device__ constexpr int tc_workers() {
    constexpr int by_smem = (227 * 1024 - 2048) / TcLayout<C>::SMEM, by_tmem = 512 / TcLayout<C>::TCOLS;
    constexpr int n = by_smem < by_tmem ? by_smem : by_tmem;
    return n < 1 ? 1 : (n > 4 ? 4 : n);
}

// The rounds of a BF16 render after ray generation, in one cooperative launch of one block per SM
// with NW warpgroup workers each.  Per round, separated by grid barriers: (1) per-block sums of the
// round's per-cell sample counts and tiles, clearing the next round's counters; (2) exclusive offsets
// and tile descriptors (each block adds the sums of the blocks before it to a scan of its cells);
// (3) the scatter of the round's samples into cell order; (4) the tiles, on the workers, after which
// each warp walks rays the previous round left in empty voxels to their next occupied voxel (they
// join the next round, two rounds after they were left, as in host-driven rounds).  The loop ends
// when a round emits nothing and leaves nothing pending, or hands the rest over: a round (after the
// first) of at most tail_rays rays is sorted and scattered, ctrl->tail set, and finished by
// wave_tail_warp_kernel.  Nothing is synchronised with the host.
template <class C, int NW>
__global__ void __launch_bounds__(NW * 128, 1) trace_tc_kernel(GridView g, WaveArgs a) {
    using T = TcLayout<C>;
    extern __shared__ __align__(1024) unsigned char dyn[];
    __shared__ __align__(8) uint64_t bar_w[NW], bar_mma[NW];
    __shared__ uint32_t s_tmem;
    __shared__ int s_tile[NW][4], s_red[NW][8], s_fail[NW];
    __shared__ int wx[32], wy[32], s_base[2], s_flag;
    WaveCtrl *ctrl = a.ctrl;
    const int tid = threadIdx.x, wk = tid >> 7;
    constexpr uint32_t NCOL = pow2_cols(NW * T::TCOLS);
    if (tid < 32) tc::tmem_alloc(&s_tmem, NCOL);
    if (tid < NW) {
        mbar_init(&bar_w[tid], 1);
        mbar_init(&bar_mma[tid], 1);
        s_fail[tid] = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    unsigned char *base = dyn + wk * T::SMEM;
    TcWorker w{base, &bar_w[wk], &bar_mma[wk], s_tile[wk], s_red[wk], &s_fail[wk],
               s_tmem + (uint32_t)(wk * T::TCOLS), 1 + wk, tid & 127, (tid & 127) >> 5, -1, 0u, 0u, false, false, 0u, 0};
    if (blockIdx.x == 0 && tid == 0) ctrl->start_ns = globaltimer_ns();
    unsigned gen = 0;
    bool ok = true;
    const int NK = a.nkeys, max_rounds = min(2 * a.max_steps + 2, kMaxTraceRounds);
    int round = 0;
    for (;; ++round) {
        const int cur = round & 1, nxt = cur ^ 1;
        // a round of at most tail_rays rays (after the first) is finished one warp per ray in FP32
        // (wave_tail_warp_kernel, launched after this kernel): it is sorted and scattered, then the loop ends
        const bool handover = round > 0 && ctrl->n_live[cur] + ctrl->n_pend[nxt] <= a.tail_max;
        if (handover) {
            // the rays the previous round left in empty voxels walk to their next occupied voxel first
            // and join this round, which the tail then finishes
            const int n = ctrl->n_pend[nxt], bound = (n + 31) & ~31;
            for (int i = blockIdx.x * blockDim.x + tid; i < bound; i += gridDim.x * blockDim.x)
                advance_pending(g, a, nxt, cur, i, n);
            if (!(ok = grid_sync(ctrl, gen, &s_flag))) break;
        }
        const int per = (NK + gridDim.x - 1) / gridDim.x;
        const int k0 = min(NK, (int)blockIdx.x * per), k1 = min(NK, k0 + per);
        // (1) block sums; the next round's counters cleared; the round's control words reset
        {
            int sum = 0, tiles = 0;
            for (int c = k0 + tid; c < k1; c += blockDim.x) {
                const int n = a.count[cur][c];
                sum += n;
                tiles += (n + 127) >> 7;
                a.count[nxt][c] = 0;
                a.fill[nxt][c] = 0;
            }
            if (blockIdx.x == 0 && tid == 0) {
                ctrl->n_live[nxt] = 0;
                ctrl->n_pend[cur] = 0;
                ctrl->next_tile_bf = 0;
                ctrl->next_adv = 0;
            }
            block_scan2_any(sum, tiles, wx, wy);
            if (tid == blockDim.x - 1) {
                ctrl->scan_part[0][blockIdx.x] = sum;
                ctrl->scan_part[1][blockIdx.x] = tiles;
            }
        }
        if (!(ok = grid_sync(ctrl, gen, &s_flag))) break;
        if (blockIdx.x == 0 && tid == 0) ctrl->round_phase_ns[round][0] = globaltimer_ns();
        // (2) offsets and tile descriptors of this block's cells
        {
            if (tid < 32) {
                int bs = 0, bt = 0;
                for (int i = tid; i < (int)blockIdx.x; i += 32) {
                    bs += ctrl->scan_part[0][i];
                    bt += ctrl->scan_part[1][i];
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    bs += __shfl_xor_sync(FULL, bs, o);
                    bt += __shfl_xor_sync(FULL, bt, o);
                }
                if (tid == 0) {
                    s_base[0] = bs;
                    s_base[1] = bt;
                }
            }
            __syncthreads();
            const int pt = (k1 - k0 + blockDim.x - 1) / blockDim.x;
            const int c0 = min(k1, k0 + tid * pt), c1 = min(k1, c0 + pt);
            int sum = 0, tiles = 0;
            for (int c = c0; c < c1; ++c) {
                const int n = a.count[cur][c];
                sum += n;
                tiles += (n + 127) >> 7;
            }
            int is = sum, it = tiles;
            block_scan2_any(is, it, wx, wy);
            int run_s = s_base[0] + is - sum, run_t = s_base[1] + it - tiles;
            for (int c = c0; c < c1; ++c) {
                const int n = a.count[cur][c];
                a.off[c] = run_s;
                for (int i = 0; i < n; i += 128) a.tiles[run_t++] = make_int4(c, run_s + i, min(128, n - i), 0);
                run_s += n;
            }
            if (blockIdx.x == gridDim.x - 1 && tid == blockDim.x - 1) {
                a.off[NK] = s_base[0] + is;
                ctrl->n_tiles = s_base[1] + it;
                ctrl->round_tiles[round] = s_base[1] + it;
            }
        }
        if (!(ok = grid_sync(ctrl, gen, &s_flag))) break;
        if (blockIdx.x == 0 && tid == 0) ctrl->round_phase_ns[round][1] = globaltimer_ns();
        // (3) scatter into cell order
        {
            const int n = ctrl->n_live[cur], lane = tid & 31, bound = (n + 31) & ~31;
            for (int i = blockIdx.x * blockDim.x + tid; i < bound; i += gridDim.x * blockDim.x) {
                const bool pred = i < n;
                const int c = pred ? a.qcell[cur][i] : 0, r = pred ? a.q[cur][i] : 0;
                const unsigned m = __ballot_sync(FULL, pred);
                if (pred) {
                    const unsigned grp = __match_any_sync(m, c);
                    const int leader = __ffs(grp) - 1;
                    int b = 0;
                    if (lane == leader) b = a.off[c] + atomicAdd(a.fill[cur] + c, __popc(grp));
                    b = __shfl_sync(grp, b, leader);
                    a.sorted[b + __popc(grp & lanemask_lt())] = r;
                }
            }
        }
        if (!(ok = grid_sync(ctrl, gen, &s_flag))) break;
        if (blockIdx.x == 0 && tid == 0) ctrl->round_phase_ns[round][2] = globaltimer_ns();
        if (handover) {
            if (blockIdx.x == 0 && tid == 0) {
                ctrl->tail = 1;
                ctrl->next_tile = 0;
                ctrl->round_phase_ns[round][3] = ctrl->round_end_ns[round] = globaltimer_ns();
                ctrl->round_live[round] = ctrl->n_live[cur];
                ctrl->tail_parity = cur;
            }
            break;
        }
        // (4) the tiles; then each warp takes rays the previous round left in empty voxels (32 at a time)
        // and walks them to their next occupied voxel: they join the next round, as with the side-stream
        // walk of host-driven rounds
        {
            const bool wok = tc_round<C>(w, g, a, cur, ctrl->n_tiles, blockIdx.x * NW + wk, gridDim.x * NW);
            if (__syncthreads_or(!wok)) {
                tc_worker_done(w, a, wok);
                ok = false;
                w.n_eval = 0;
                break;
            }
            const int n = ctrl->n_pend[nxt];
            for (;;) {
                int b = 0;
                if ((tid & 31) == 0) b = atomicAdd(&ctrl->next_adv, 32);
                b = __shfl_sync(FULL, b, 0);
                if (b >= n) break;
                advance_pending(g, a, nxt, nxt, b + (tid & 31), n);
            }
        }
        if (!(ok = grid_sync(ctrl, gen, &s_flag))) break;
        if (blockIdx.x == 0 && tid == 0) ctrl->round_phase_ns[round][3] = globaltimer_ns();
        if (blockIdx.x == 0 && tid == 0) {
            ctrl->round_live[round] = ctrl->n_live[cur];
            ctrl->round_end_ns[round] = globaltimer_ns();
        }
        // done when nothing was emitted and nothing waits in this round's pending list
        if ((ctrl->n_live[nxt] == 0 && ctrl->n_pend[cur] == 0) || round + 1 >= max_rounds) break;
    }
    if (blockIdx.x == 0 && tid == 0) {
        ctrl->rounds = round + 1;
        if (ok && !ctrl->tail && (ctrl->n_live[(round & 1) ^ 1] != 0 || ctrl->n_pend[round & 1] != 0))
            atomicCAS(a.status, 0, (int)8 /* KNS_ERR_INTERNAL */);
    }
    if (!ok && tid == 0) atomicCAS(a.status, 0, (int)6 /* KNS_ERR_TIMEOUT */);
    tc_worker_done(w, a, true);
    tc::fence_before_sync();
    __syncthreads();
    if (tid < 32) tc::tmem_free(s_tmem, NCOL);
}

template <class C>
cudaError_t launch_wave_eval_tc_cfg(const GridView &g, const WaveArgs &a, int cur, int sm_count, cudaStream_t s) {
    using T = TcLayout<C>;
    static_assert(T::SMEM <= 200 * 1024, "tensor-core tile does not fit in shared memory");
    // Resident blocks per SM from the kernel's own resources (registers, shared memory, threads) and the
    // tensor memory (accumulator and activation columns, of 512 per SM).  The occupancy query is not used here: it reports one
    // block per SM for every kernel that allocates tensor memory.
    static std::atomic<int> per_sm{0};
    int nb = per_sm.load();
    if (nb <= 0) {
        cudaError_t e = cudaFuncSetAttribute(wave_eval_tc_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, T::SMEM);
        cudaFuncAttributes fa{};
        int dev = 0, smem_sm = 0, reserved = 0, regs_sm = 0;
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, wave_eval_tc_kernel<C>);
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
        if (e != cudaSuccess) return e;
        const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;  // allocated per warp in units of 256
        const int by_regs = regs_sm / (regs_warp * 4);
        const int by_smem = smem_sm / (T::SMEM + (int)fa.sharedSizeBytes + reserved);
        nb = std::max(1, std::min(std::min(by_regs, by_smem), std::min(16, 512 / (int)pow2_cols(T::TCOLS))));
        per_sm.store(nb);
    }
    wave_eval_tc_kernel<C><<<sm_count * nb, 128, T::SMEM, s>>>(g, a, cur);
    return cudaGetLastError();
}

template <class C>
cudaError_t launch_trace_tc_cfg(const GridView &g, const WaveArgs &a, int sm_count, cudaStream_t s) {
    constexpr int NW = tc_workers<C>();
    constexpr int smem = NW * TcLayout<C>::SMEM;
    static_assert(smem <= 227 * 1024, "persistent trace does not fit in shared memory");
    auto kern = trace_tc_kernel<C, NW>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    GridView gv = g;
    WaveArgs av = a;
    void *args[] = {&gv, &av};
    // one block per SM: every block is resident (the barriers need it), and a kernel that allocates tensor
    // memory may have one block per SM in a cooperative launch
    return cudaLaunchCooperativeKernel((void *)kern, dim3(sm_count), dim3(NW * 128), args, smem, s);
}

#ifdef KNS_W
using InstCfg = Cfg<KNS_W, KNS_H, KNS_L, KNS_LD>;
template cudaError_t launch_wave_eval_tc_cfg<InstCfg>(const GridView &, const WaveArgs &, int, int, cudaStream_t);
template cudaError_t launch_trace_tc_cfg<InstCfg>(const GridView &, const WaveArgs &, int, cudaStream_t);
#endif

}  // namespace kns
