// kns_wave.cu -- wavefront render kernels (FP32): ray generation and the per-cell evaluation of
// the sphere trace (Eq. 2, trace form: d only) -- block tiles (the default), warp tiles, and the
// one-warp-per-ray tail.  Shading is in kns_shade.cu, the sort and the advance kernel in kns_sort.cu.
// kns:instantiate (compiled once per grid configuration)
//
// Warp tiles: a warp evaluates the SDF MLP of one cell for up to 16 samples at once as a
// register-blocked GEMM per layer.  Activations live in shared memory as h[k][s] (k = input unit,
// s = sample); lane (sg, ng) = (lane / 8, lane % 8) accumulates samples 4sg..4sg+3 against output
// units ng*W/8 .. ng*W/8 + W/8 - 1, so each shared-memory float4 of activations and each float4 of
// k-major weights feed 16 (W = 32) or 32 (W = 64) FMAs.
#include "kns_wave.cuh"

namespace kns {

// Activations of a 16-sample tile are sample-major: h[s][k] with a row stride S(K) floats, S(K)/4
// odd, so that the float4 accesses below are free of bank conflicts.
__host__ __device__ constexpr int act_stride(int K) {
    return round4(K) + (((round4(K) / 4) % 2 == 0) ? 4 : 0);
}

// One layer of the tile: hout[s][o] = softplus(b[o] + sum_k Wt[k][o] hin[s][k]), k ascending.
// Lane (sg, ng) = (lane / 8, lane % 8) owns samples sg, sg+4, sg+8, sg+12 and outputs
// NPL*ng .. NPL*ng + NPL - 1: per 4 inputs it loads 4 float4 of activations and NPL float4 of
// weights and issues 16*NPL FMAs.
template <int K, int W>
__device__ __forceinline__ void tile_layer_f32(const float *__restrict__ Wt, const float *__restrict__ b,
                                               const float *hin, float *hout, int lane, float beta,
                                               float inv_beta) {
    constexpr int NPL = W / 8;
    constexpr int SIN = act_stride(K), SOUT = act_stride(W);
    const int sg = lane >> 3, ng = lane & 7;
    float acc[4][NPL];
#pragma unroll
    for (int j = 0; j < NPL; j += 4) {
        const float4 bb = *reinterpret_cast<const float4 *>(b + ng * NPL + j);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            acc[i][j] = bb.x;
            acc[i][j + 1] = bb.y;
            acc[i][j + 2] = bb.z;
            acc[i][j + 3] = bb.w;
        }
    }
#pragma unroll 2
    for (int k0 = 0; k0 < K; k0 += 4) {
        float4 av[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) av[i] = *reinterpret_cast<const float4 *>(hin + (sg + 4 * i) * SIN + k0);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
            for (int j = 0; j < NPL; j += 4) {
                const float4 w = *reinterpret_cast<const float4 *>(Wt + (k0 + kk) * W + ng * NPL + j);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float a = kk == 0 ? av[i].x : kk == 1 ? av[i].y : kk == 2 ? av[i].z : av[i].w;
                    acc[i][j] = fmaf(a, w.x, acc[i][j]);
                    acc[i][j + 1] = fmaf(a, w.y, acc[i][j + 1]);
                    acc[i][j + 2] = fmaf(a, w.z, acc[i][j + 2]);
                    acc[i][j + 3] = fmaf(a, w.w, acc[i][j + 3]);
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int j = 0; j < NPL; j += 4) {
            float4 v;
            v.x = softplus_f32(acc[i][j], beta, inv_beta);
            v.y = softplus_f32(acc[i][j + 1], beta, inv_beta);
            v.z = softplus_f32(acc[i][j + 2], beta, inv_beta);
            v.w = softplus_f32(acc[i][j + 3], beta, inv_beta);
            *reinterpret_cast<float4 *>(hout + (sg + 4 * i) * SOUT + ng * NPL + j) = v;
        }
    }
}

// SDF trace form for a tile whose encoded inputs are in hin[s][k] (left intact); P and Q are the
// ping-pong activation buffers.  Returns d of sample lane % 16.
template <class C>
__device__ __forceinline__ float tile_sdf_f32(const float *__restrict__ wt, const float *hin, float *P, float *Q,
                                              int lane, float beta, float inv_beta) {
    tile_layer_f32<C::INP, C::W>(wt + C::tW0, wt + C::tb0, hin, P, lane, beta, inv_beta);
    __syncwarp();
    float *src = P, *dst = Q;
#pragma unroll
    for (int l = 1; l < C::H; ++l) {
        tile_layer_f32<C::W, C::W>(wt + C::tWl(l), wt + C::tbl(l), src, dst, lane, beta, inv_beta);
        __syncwarp();
        float *tmp = src;
        src = dst;
        dst = tmp;
    }
    // the d row: bias first, then one sequential FMA chain over k, the same order as the
    // per-thread evaluator, so a sample's d does not depend on which path evaluated it
    constexpr int S = act_stride(C::W);
    const int s = lane & 15;
    float acc = wt[C::tbL];
#pragma unroll
    for (int k = 0; k < C::W; k += 4) {
        const float4 h = *reinterpret_cast<const float4 *>(src + s * S + k);
        const float4 w = *reinterpret_cast<const float4 *>(wt + C::tdL + k);
        acc = fmaf(w.x, h.x, acc);
        acc = fmaf(w.y, h.y, acc);
        acc = fmaf(w.z, h.z, acc);
        acc = fmaf(w.w, h.w, acc);
    }
    __syncwarp();
    return acc;
}

// Wave 0: one thread per pixel (16x8 pixels per block, 8x4 per warp, blockIdx.z = view); clip,
// advance, emit.
template <class C>
__global__ void __launch_bounds__(128) wave_gen_kernel(GridView g, WaveArgs a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = blockIdx.x * 16 + (warp & 1) * 8 + (lane & 7);
    const int i = blockIdx.y * 8 + (warp >> 1) * 4 + (lane >> 3);
    const int view = blockIdx.z;
    const ViewDev &V = a.views[view];
    const int r = V.ray_base + i * V.W + j;
    const bool valid = i < V.H && j < V.W && (a.ray_o == nullptr || r < a.n_table);
    bool alive = false;
    int cell = -1;
    if (valid) {
        a.ray_view[r] = view;
        const Ray ray = a.ray_o ? table_ray(a, r) : make_ray(V.cam, i, j);
        const GridView gv = sub_grid(g, V.grid);
        float t0, tf;
        if (!clip_box(gv, ray, t0, tf)) {
            write_miss(a, r, 0);
        } else {
            float t = t0;
            cell = advance_ray(gv, ray, t, tf);
            if (cell < 0) {
                write_miss(a, r, 0);
            } else {
                alive = true;
                a.t_ray[r] = t;
                a.steps_ray[r] = 0;
                if (a.t_hist) a.t_hist[r] = no_history();
                if (a.trap) a.trap[r] = trap_empty();
            }
        }
    }
    const int qp = warp_append(&a.ctrl->n_live[0], alive);
    if (alive) {
        a.q[0][qp] = r;
        a.qcell[0][qp] = cell;
    }
    warp_count_cells(a.count[0], alive, cell);
}

// Round k: each warp (a block of its own) takes tiles of up to 16 cell-sorted samples of one cell,
// stages the cell's k-major weights in its shared memory with one TMA bulk copy (skipped when the
// next tile has the same cell), and evaluates the 16 samples as a tile GEMM.  A ray whose next
// sample lies in the same cell keeps stepping inside the tile (up to inner_steps evaluations this
// round, while at least min_active rays remain); the others are emitted to round k+1 with their
// next cell, converge (hit list) or terminate (miss written).  A round with few rays (tail) is
// finished one warp per ray by wave_tail_warp_kernel.
template <class C>
__host__ __device__ constexpr int eval_smem_bytes() {
    return (C::TSIZE + TILE * (act_stride(C::INP) + 2 * act_stride(C::W))) * (int)sizeof(float);
}

// ---------------------------------------------------------------- block tiles (FP32 renders)
// Round k with tiles of up to BT samples of one cell (BT = 128 or 256, the sort's granularity): a
// block of NT threads takes tiles whose descriptors {cell, first sample, samples} the scan wrote
// (thread 0 holds the next descriptor and the index after it in flight), stages the cell's k-major
// trace weights with one TMA bulk copy (kept while consecutive tiles share the cell), encodes the
// samples into shared rows h[k][s] (row stride BT + 4 floats, NT / BT threads per sample), and runs
// each layer as a [W x K] by [K x BT] block GEMM: warp w owns a slice of the output units, lane l a
// run of samples, so per input k one warp-uniform float4 of weights and one float4 of activations
// feed 16 or more FMAs per thread.  Every output is its bias followed by one FMA per input in
// ascending order and the d row is one sequential FMA chain, the order of the per-thread evaluator,
// so d does not depend on the tile shape.  Threads 0..BT-1 then test and step their sample: a hit,
// a miss, a step into an empty voxel (the round's pending list: wave_advance_kernel walks it to the
// next occupied voxel), or an emit to round k+1 with its next cell -- unless enough of the tile's
// samples stay in the cell, in which case those are evaluated again at once (inner_steps,
// min_active).
constexpr int BTHREADS = 256;  // default threads per block tile (two per sample in the encoding)
// shared row stride (floats) of a BT-sample tile: row r starts in bank group r mod 8
__host__ __device__ constexpr int block_rs(int BT) { return BT + 4; }

// rows of the buffer that holds the encoding and, after layer 0, the second activation buffer
template <class C>
__host__ __device__ constexpr int block_rows0() { return C::INP > C::W ? C::INP : C::W; }

template <class C, int BT>
__host__ __device__ constexpr int block_eval_smem_bytes() {
    return (C::TSIZE + (block_rows0<C>() + C::W) * block_rs(BT)) * (int)sizeof(float);
}

// encoding of sample column s (Eq. 1) split into NH parts (1 or 2 threads per sample): part 0
// writes x, part h frequencies [h L/NH, (h+1) L/NH); values as encode3
template <int L, int NH, int BRS>
__device__ __forceinline__ void encode_split(float *rows, int s, int half, float px, float py, float pz) {
    const float p[3] = {px, py, pz};
    if (half == 0) {
        rows[0 * BRS + s] = px;
        rows[1 * BRS + s] = py;
        rows[2 * BRS + s] = pz;
    }
#pragma unroll
    for (int kk = 0; kk < L / NH; ++kk) {
        const int k = half * (L / NH) + kk;
        const float f = (float)(1 << k);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float sn, cs;
            sincospif(f * p[c], &sn, &cs);
            rows[(3 + 6 * k + c) * BRS + s] = sn;
            rows[(3 + 6 * k + 3 + c) * BRS + s] = cs;
        }
    }
}

// out[o][s] = softplus(b[o] + sum_{k < K} Wt[k][o] in[k][s]) for this thread's W/8 outputs x BT/32
// samples
template <int K, int W, int BT, int NT>
__device__ __forceinline__ void block_layer(const float *Wt, const float *b, const float *in, float *out,
                                            float beta, float inv_beta) {
    constexpr int NO = W / (NT / 32), NS = BT / 32, BRS = block_rs(BT);
    const int o0 = (threadIdx.x >> 5) * NO, s0 = (threadIdx.x & 31) * NS;
    float acc[NO][NS];
#pragma unroll
    for (int i = 0; i < NO; ++i) {
        const float bi = b[o0 + i];
#pragma unroll
        for (int j = 0; j < NS; ++j) acc[i][j] = bi;
    }
#pragma unroll 2
    for (int k = 0; k < K; ++k) {
        float xa[NS];
#pragma unroll
        for (int j4 = 0; j4 < NS; j4 += 4) {
            const float4 x = *reinterpret_cast<const float4 *>(in + k * BRS + s0 + j4);
            xa[j4] = x.x;
            xa[j4 + 1] = x.y;
            xa[j4 + 2] = x.z;
            xa[j4 + 3] = x.w;
        }
#pragma unroll
        for (int i4 = 0; i4 < NO; i4 += 4) {
            const float4 w = *reinterpret_cast<const float4 *>(Wt + k * W + o0 + i4);
            const float wa[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < NS; ++j) acc[i4 + i][j] = fmaf(wa[i], xa[j], acc[i4 + i][j]);
        }
    }
#pragma unroll
    for (int i = 0; i < NO; ++i)
#pragma unroll
        for (int j4 = 0; j4 < NS; j4 += 4)
            *reinterpret_cast<float4 *>(out + (o0 + i) * BRS + s0 + j4) = make_float4(
                softplus_f32(acc[i][j4], beta, inv_beta), softplus_f32(acc[i][j4 + 1], beta, inv_beta),
                softplus_f32(acc[i][j4 + 2], beta, inv_beta), softplus_f32(acc[i][j4 + 3], beta, inv_beta));
}

// the block's next tile: the next of its own contiguous run (static), or the round's next (dynamic)
__device__ __forceinline__ int claim_tile(const WaveArgs &a, int n_tiles, int &next_static, int end_static) {
    if (a.static_tiles) return next_static < end_static ? next_static++ : n_tiles;
    return atomicAdd(&a.ctrl->next_tile, 1);
}

// blocks of a tile kernel that fit on one SM by shared memory (at most 4): the register budget
template <class C, int BT>
__host__ __device__ constexpr int block_min_blocks() {
    constexpr int by_smem = (227 * 1024) / (block_eval_smem_bytes<C, BT>() + 2048);
    return by_smem < 1 ? 1 : (by_smem > 4 ? 4 : by_smem);
}

template <class C, int BT, int NT>
__global__ void __launch_bounds__(NT, block_min_blocks<C, BT>()) wave_eval_block_kernel(GridView g, WaveArgs a, int cur) {
    constexpr int BRS = block_rs(BT), NH = NT / BT;  // NH threads encode one sample
    extern __shared__ __align__(128) float dyn[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_tile[4];  // cell, start, len, fresh
    __shared__ float s_x[3][BT];
    if (a.ctrl->tail) return;  // finished one warp per ray by wave_tail_warp_kernel
    const int n_tiles = a.ctrl->n_tiles_fine;
    if (n_tiles <= 0) return;
    const int tid = threadIdx.x, nxt = cur ^ 1;
    // the encoding rows A0 are dead after layer 0, so the second activation buffer Q reuses them
    float *wsm = dyn;
    float *A0 = dyn + C::TSIZE, *P = A0 + block_rows0<C>() * BRS, *Q = A0;
    if (tid == 0) mbar_init(&bar, 1);
    __syncthreads();
    const int per = (n_tiles + gridDim.x - 1) / gridDim.x;
    int next_static = blockIdx.x * per;
    const int end_static = min(n_tiles, next_static + per);
    int cached = -1;
    uint32_t phase = 0;
    // thread 0 keeps two tiles in flight: the descriptor of the next tile (loaded) and the index of
    // the one after it (claimed), so that neither the claim nor the load waits at the tile's start
    int4 nd = make_int4(-1, 0, 0, 0);
    int nt = n_tiles;
    unsigned n_eval = 0;  // samples this thread evaluated
    if (tid == 0) {
        const int t0 = claim_tile(a, n_tiles, next_static, end_static);
        if (t0 < n_tiles) nd = a.tiles[t0];
        nt = claim_tile(a, n_tiles, next_static, end_static);
    }
    for (;;) {
        if (tid == 0) {
            const int4 d = nd;
            nd = nt < n_tiles ? a.tiles[nt] : make_int4(-1, 0, 0, 0);
            if (d.x >= 0) nt = claim_tile(a, n_tiles, next_static, end_static);
            if (d.x >= 0 && d.x != cached)
                bulk_load(wsm, a.wt + (int64_t)d.x * a.wt_stride, C::TSIZE * sizeof(float), &bar);
            s_tile[0] = d.x;
            s_tile[1] = d.y;
            s_tile[2] = d.z;
            s_tile[3] = d.x != cached;
        }
        __syncthreads();
        const int c = s_tile[0], start = s_tile[1], len = s_tile[2];
        const bool fresh = s_tile[3] != 0;
        if (c < 0) break;
        cached = c;
        const GridView gt = sub_grid(g, c / g.ncl);  // the grid of the tile's cell (a stack of grids)
        // samples: threads 0..127 own sample s = tid
        bool active = tid < len;
        int r = 0, steps = 0, switched = 0;
        float t = 0.f, t0 = 0.f, tf = 0.f;
        float4 hist = no_history();
        const bool cycles = a.t_hist != nullptr && !a.coarse;
        Ray ray{};
        if (active) {
            r = a.sorted[start + tid];
            t = a.t_ray[r];
            if (cycles) hist = a.t_hist[r];
            steps = a.steps_ray[r];
            if (a.coarse) switched = a.cell_ray[r];
            int cam;
            ray = ray_of(a, r, cam);
            clip_box(gt, ray, t0, tf);
        }
        // Up to inner_steps evaluations of the tile: a sample whose step keeps it in this cell (an
        // emit to the same key) is evaluated again at once, while at least min_active of them do;
        // the others, and all of them at the last evaluation, leave as below.
        bool fresh_wait = fresh;
        for (int it = 0;; ++it) {
            if (tid < BT) {
                s_x[0][tid] = active ? fmaf(t, ray.wx, ray.ox) : 0.f;
                s_x[1][tid] = active ? fmaf(t, ray.wy, ray.oy) : 0.f;
                s_x[2][tid] = active ? fmaf(t, ray.wz, ray.oz) : 0.f;
            }
            __syncthreads();
            {
                const int s = tid & (BT - 1);
                encode_split<C::L, NH, BRS>(A0, s, tid / BT, s_x[0][s], s_x[1][s], s_x[2][s]);
                if (tid < BT)
#pragma unroll
                    for (int k = C::IN; k < C::INP; ++k) A0[k * BRS + s] = 0.f;  // encoding pad
            }
            if (fresh_wait) {
                const bool ok = mbar_wait(&bar, phase, 1u << 26);
                phase ^= 1u;
                fresh_wait = false;
                if (__syncthreads_or(!ok)) {  // the weights never landed: report and leave
                    if (tid == 0) atomicCAS(a.status, 0, (int)6 /* KNS_ERR_TIMEOUT */);
                    return;
                }
            } else {
                __syncthreads();
            }
            block_layer<C::INP, C::W, BT, NT>(wsm + C::tW0, wsm + C::tb0, A0, P, g.beta, g.inv_beta);
            float *src = P, *dst = Q;
#pragma unroll
            for (int l = 1; l < C::H; ++l) {
                __syncthreads();
                block_layer<C::W, C::W, BT, NT>(wsm + C::tWl(l), wsm + C::tbl(l), src, dst, g.beta, g.inv_beta);
                float *tmp = src;
                src = dst;
                dst = tmp;
            }
            __syncthreads();
            // outcome of this evaluation: 0 none (inactive), 1 hit, 2 miss (written), 3 pending,
            // 4 emit to ncell
            int outcome = 0, ncell = -1;
            float t_eval = t;
            if (tid < BT) {
                // the d row: bias first, then one sequential FMA chain over k
                float d = wsm[C::tbL];
#pragma unroll 8
                for (int k = 0; k < C::W; ++k) d = fmaf(wsm[C::tdL + k], src[k * BRS + tid], d);
                n_eval += active ? 1u : 0u;
                if (active) {
                    ++steps;
                    const bool last_refine = a.coarse && steps - switched >= a.refine_steps;
                    if (fabsf(d) < a.eps || (last_refine && fabsf(d) < a.eps_coarse)) {
                        outcome = 1;
                    } else if (last_refine) {
                        outcome = 2;
                        write_miss(a, r, steps);
                    } else {
                        t += d;
                        if (t > tf || t < t0 || steps >= a.max_steps) {
                            outcome = 2;
                            write_miss(a, r, steps);
                        } else {
                            // an occupied voxel gives the next cell at once; a ray that stepped into
                            // empty space goes on the round's pending list for wave_advance_kernel, so
                            // that no lane holds the block in a long voxel walk
                            ncell = advance_fast(gt, ray, t);
                            if (ncell == -2) {
                                outcome = 3;
                            } else if (cycles && cycle_step(hist, t_eval, t)) {
                                outcome = 2;
                                write_miss(a, r, a.max_steps);
                                ncell = -1;
                            } else {
                                outcome = 4;
                            }
                        }
                    }
                }
            }
            // samples that stay in this cell are evaluated again while enough of them do
            const bool cand = outcome == 4 && ncell == c && it + 1 < a.inner_steps;
            const int n_cand = __syncthreads_count(cand);
            const bool again = n_cand > 0 && n_cand >= a.min_active;
            const bool stay = cand && again;
            if (tid < BT) {
                const bool hit = outcome == 1, emit = outcome == 4 && !stay, pend = outcome == 3;
                if (hit) {
                    a.cell_ray[r] = c;
                    a.t_ray[r] = t;
                    a.steps_ray[r] = steps;
                } else if (pend) {
                    a.t_ray[r] = t;
                    a.steps_ray[r] = steps;
                } else if (emit) {
                    a.t_ray[r] = t;
                    a.steps_ray[r] = steps;
                    if (cycles) a.t_hist[r] = hist;
                }
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
        __syncthreads();
    }
    if (tid < BT) {  // evaluated samples, one atomic per warp
        const unsigned long long n = warp_sum_u64(n_eval);
        if ((tid & 31) == 0 && n) atomicAdd(&a.ctrl->samples_f32, n);
    }
}

// Tail: a warp runs one ray to its end.  The warp keeps the k-major trace weights of its ray's
// current cell in a shared-memory slot of its own (one bulk copy per change of cell: the rays left
// for the tail are mostly grazing rays that take many small steps inside one cell) and evaluates a
// sample as one matrix-vector product per layer: lane o computes output unit o (and o + 32 for width
// 64) with its weights read conflict-free from the slot and the layer input broadcast from a
// shared-memory row.  Every output is its bias followed by one FMA per input in ascending order and
// every lane forms the d row as one sequential chain -- the order of the tile evaluators, so d is
// bit-identical to theirs.  Rays are handed out one at a time in cell-sorted order.

// input k of the encoding (Eq. 1): x, y, z, then per frequency sin x, sin y, sin z, cos x, cos y, cos z
__device__ __forceinline__ float encoding_entry(int k, float px, float py, float pz) {
    if (k < 3) return k == 0 ? px : (k == 1 ? py : pz);
    const int f = (k - 3) / 6, c = (k - 3) % 6;
    const float p = (c % 3) == 0 ? px : ((c % 3) == 1 ? py : pz);
    float sn, cs;
    sincospif((float)(1 << f) * p, &sn, &cs);
    return c < 3 ? sn : cs;
}

// shared memory of a tail warp: the weight slot, the encoded input row, two activation rows
template <class C>
constexpr int tail_smem_floats() { return C::TSIZE + C::INP + 2 * C::W; }

// vector of NPL consecutive floats (NPL = 1, 2 or 4): one shared-memory access per lane
template <int NPL>
struct VecF;
template <>
struct VecF<1> {
    static __device__ __forceinline__ void load(const float *p, float *v) { v[0] = *p; }
    static __device__ __forceinline__ void store(float *p, const float *v) { *p = v[0]; }
};
template <>
struct VecF<2> {
    static __device__ __forceinline__ void load(const float *p, float *v) {
        const float2 x = *reinterpret_cast<const float2 *>(p);
        v[0] = x.x;
        v[1] = x.y;
    }
    static __device__ __forceinline__ void store(float *p, const float *v) {
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    }
};
template <>
struct VecF<4> {
    static __device__ __forceinline__ void load(const float *p, float *v) {
        const float4 x = *reinterpret_cast<const float4 *>(p);
        v[0] = x.x;
        v[1] = x.y;
        v[2] = x.z;
        v[3] = x.w;
    }
    static __device__ __forceinline__ void store(float *p, const float *v) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};

// One layer of the warp product, lane l owning the NPL = W/32 consecutive outputs NPL*l ...: one
// vector load of their k-major weights feeds NPL FMAs.  out[o] = softplus(b[o] + sum_k Wt[k][o] in[k]),
// one chain per output, k ascending -- the summation order of every FP32 evaluator, so d is
// bit-identical to the tiles' (and to the shading's re-evaluation of a BF16 render's tail hits).
// The inputs are taken in groups of G: the weights and inputs of group g + 1 are loaded into registers
// while group g's FMAs run, so the chain waits on neither (a lane's two chains at width 64 are the
// only dependence left).
template <int K, int W>
__device__ __forceinline__ void warp_layer(const float *__restrict__ Wt, const float *__restrict__ b,
                                           const float *in, float *out, int lane, float beta, float inv_beta) {
    constexpr int NPL = W / 32;
    static_assert(NPL == 1 || NPL == 2 || NPL == 4, "width must be 32, 64 or 128");
    static_assert(K % 4 == 0, "layer input must be padded to 4");
    constexpr int G = K % 8 == 0 ? 8 : 4, NG = K / G;
    const int o0 = NPL * lane;
    float acc[NPL], w[2][G][NPL], x[2][G];
    VecF<NPL>::load(b + o0, acc);
    auto fetch = [&](int g, int buf) {
#pragma unroll
        for (int c = 0; c < G; c += 4) VecF<4>::load(in + g * G + c, &x[buf][c]);
#pragma unroll
        for (int c = 0; c < G; ++c) VecF<NPL>::load(Wt + (g * G + c) * W + o0, w[buf][c]);
    };
    fetch(0, 0);
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        if (g + 1 < NG) fetch(g + 1, (g + 1) & 1);
#pragma unroll
        for (int c = 0; c < G; ++c)
#pragma unroll
            for (int u = 0; u < NPL; ++u) acc[u] = fmaf(w[g & 1][c][u], x[g & 1][c], acc[u]);
    }
#pragma unroll
    for (int u = 0; u < NPL; ++u) acc[u] = softplus_f32(acc[u], beta, inv_beta);
    VecF<NPL>::store(out + o0, acc);
    __syncwarp();
}

// The d row: its bias, then one sequential chain over the last hidden layer (every lane forms it);
// the row and the activations are loaded a group of 16 ahead of the chain.
template <int W>
__device__ __forceinline__ float warp_d_row(const float *__restrict__ drow, float bias, const float *h) {
    constexpr int G = 16, NG = W / G;
    float wv[2][G], hv[2][G];
    auto fetch = [&](int g, int buf) {
#pragma unroll
        for (int c = 0; c < G; c += 4) {
            VecF<4>::load(drow + g * G + c, &wv[buf][c]);
            VecF<4>::load(h + g * G + c, &hv[buf][c]);
        }
    };
    float d = bias;
    fetch(0, 0);
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        if (g + 1 < NG) fetch(g + 1, (g + 1) & 1);
#pragma unroll
        for (int c = 0; c < G; ++c) d = fmaf(wv[g & 1][c], hv[g & 1][c], d);
    }
    return d;
}

// The SDF trace form of one sample whose encoded input row is in xin.
template <class C>
__device__ __forceinline__ float warp_sdf_trace(const float *__restrict__ wsm, const float *xin, float *h0, float *h1,
                                                int lane, float beta, float inv_beta) {
    warp_layer<C::INP, C::W>(wsm + C::tW0, wsm + C::tb0, xin, h0, lane, beta, inv_beta);
    float *src = h0, *dst = h1;
#pragma unroll
    for (int l = 1; l < C::H; ++l) {
        warp_layer<C::W, C::W>(wsm + C::tWl(l), wsm + C::tbl(l), src, dst, lane, beta, inv_beta);
        float *tmp = src;
        src = dst;
        dst = tmp;
    }
    return warp_d_row<C::W>(wsm + C::tdL, wsm[C::tbL], src);
}

// A tail round: one warp (one block) per ray, to the end.  Rays come in cell-sorted order (the cell
// of a ray's position is its sort key); the round's tile counter hands them out.  In a BF16 render the
// rays left in the round take their last steps here in FP32, with the BF16 trace's cycle test and seam
// trap, and join the hit list when |d| < eps as the tensor-core tiles' rays do.
template <class C, bool STACK>
__global__ void __launch_bounds__(32) wave_tail_warp_kernel(GridView g, WaveArgs a, int cur) {
    extern __shared__ __align__(128) float dyn[];
    __shared__ __align__(8) uint64_t bar;
    if (!a.ctrl->tail) return;
    if (cur < 0) cur = a.ctrl->tail_parity;  // the round the persistent BF16 trace left to the tail
    const int n = a.ctrl->n_live[cur];
    const int lane = threadIdx.x;
    float *wsm = dyn, *xin = dyn + C::TSIZE, *h0 = xin + C::INP, *h1 = h0 + C::W;
    for (int k = C::IN + lane; k < C::INP; k += 32) xin[k] = 0.f;  // encoding pad stays zero
    if (lane == 0) mbar_init(&bar, 1);
    __syncwarp();
    const bool cycles = a.t_hist != nullptr;
    int cached = -1;
    uint32_t phase = 0;
    unsigned long long nsamples = 0;
    for (;;) {
        int q = 0;
        if (lane == 0) q = atomicAdd(&a.ctrl->next_tile, 1);
        q = __shfl_sync(FULL, q, 0);
        if (q >= n) break;
        const int r = a.sorted[q];
        int lo = 0, hi = a.NC;  // the key with off[key] <= q < off[key+1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(a.off + mid) <= q) lo = mid; else hi = mid;
        }
        int cell = lo;
        int cam;
        const Ray ray = ray_of(a, r, cam);
        GridView gs;
        if constexpr (STACK) gs = sub_grid(g, cell / g.ncl);  // the ray's grid in a stack of grids
        const GridView &gr = STACK ? gs : g;
        float t0, tf;
        clip_box(gr, ray, t0, tf);
        float t = a.t_ray[r];
        int steps = a.steps_ray[r];
        float4 hist = cycles ? a.t_hist[r] : no_history();
        int4 trap = a.trap ? a.trap[r] : trap_empty();
        bool hit = false;
        for (;;) {
            // a new cell's weights are copied while the sample is encoded
            const bool fresh = cell != cached;
            if (fresh) {
                __syncwarp();  // every lane is done with the slot's previous cell
                if (lane == 0) bulk_load(wsm, a.wt + (int64_t)cell * a.wt_stride, C::TSIZE * sizeof(float), &bar);
            }
            {
                const float px = fmaf(t, ray.wx, ray.ox), py = fmaf(t, ray.wy, ray.oy),
                            pz = fmaf(t, ray.wz, ray.oz);
                for (int k = lane; k < C::IN; k += 32) xin[k] = encoding_entry(k, px, py, pz);
            }
            if (fresh) {
                const bool ok = mbar_wait(&bar, phase, 1u << 26);
                phase ^= 1u;
                if (!__all_sync(FULL, ok)) {  // the weights never landed: report and leave
                    if (lane == 0) atomicCAS(a.status, 0, (int)6 /* KNS_ERR_TIMEOUT */);
                    return;
                }
                cached = cell;
            }
            __syncwarp();
            const float d = warp_sdf_trace<C>(wsm, xin, h0, h1, lane, g.beta, g.inv_beta);
            ++steps;
            ++nsamples;
            if (fabsf(d) < a.eps) {
                hit = true;
                break;
            }
            // BF16 renders: the trace's seam trap (a trapped ray is the plain iteration's budget miss)
            if (a.trap && trap_step(trap, t, d, cell, a.trap_span, 5.f * a.eps_coarse)) {
                steps = a.max_steps;
                break;
            }
            const float t_eval = t;
            t += d;
            if (t > tf || t < t0 || steps >= a.max_steps) break;
            cell = advance_ray(gr, ray, t, tf);
            if (cell < 0) break;
            if (cycles && (a.coarse ? cycle_step_tol(hist, t_eval, t) : cycle_step(hist, t_eval, t))) {
                steps = a.max_steps;
                break;
            }
            // an occupancy skip ends the trap's run of samples (the skip moved t by more than d)
            if (a.trap && t != t_eval + d) trap = trap_empty();
        }
        if (lane == 0) {
            if (hit) {
                a.cell_ray[r] = cell;
                a.t_ray[r] = t;
                a.steps_ray[r] = steps;
                a.hits[atomicAdd(&a.ctrl->n_hits, 1)] = r;
            } else {
                write_miss(a, r, steps);
            }
        }
    }
    if (lane == 0 && nsamples) {
        atomicAdd(&a.ctrl->samples_f32, nsamples);
        atomicAdd(&a.ctrl->samples_tail, nsamples);
    }
}

template <class C>
__global__ void __launch_bounds__(32) wave_eval_kernel(GridView g, WaveArgs a, int cur) {
    extern __shared__ __align__(128) float dyn[];
    __shared__ __align__(8) uint64_t bar;
    if (a.ctrl->tail) return;  // finished one warp per ray by wave_tail_warp_kernel
    const int lane = threadIdx.x;
    const int nxt = cur ^ 1;
    float *wsm = dyn;
    float *hin = dyn + C::TSIZE;
    float *P = hin + TILE * act_stride(C::INP), *Q = P + TILE * act_stride(C::W);
    constexpr int SIN = act_stride(C::INP);
    const int n_tiles = a.ctrl->n_tiles_fine;  // FP32 tiles (BF16 tiles follow them)
    if (n_tiles <= 0) return;
    if (lane == 0) mbar_init(&bar, 1);
    __syncwarp();
    // static schedule: block b owns tiles [b*per, (b+1)*per) so consecutive same-cell tiles reuse
    // one weight load; dynamic: tiles are handed out one at a time
    const int per = (n_tiles + gridDim.x - 1) / gridDim.x;
    int next_static = blockIdx.x * per;
    const int end_static = min(n_tiles, next_static + per);
    int cached = -1;
    uint32_t phase = 0;
    for (;;) {
        int tile = 0;
        if (lane == 0) tile = a.static_tiles ? (next_static < end_static ? next_static : n_tiles)
                                             : atomicAdd(&a.ctrl->next_tile, 1);
        tile = __shfl_sync(FULL, tile, 0);
        ++next_static;
        if (tile >= n_tiles) break;
        int c = 0, start = 0, len = 0;
        if (lane == 0) {
            int lo = 0, hi = a.NC;  // the cell c with tile_off[c] <= tile < tile_off[c+1]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(a.tile_off + mid) <= tile) lo = mid; else hi = mid;
            }
            c = lo;
            start = __ldg(a.off + lo) + (tile - __ldg(a.tile_off + lo)) * TILE;
            len = min(TILE, __ldg(a.off + lo + 1) - start);
            if (c != cached) bulk_load(wsm, a.wt + (int64_t)c * a.wt_stride, C::TSIZE * sizeof(float), &bar);
        }
        c = __shfl_sync(FULL, c, 0);
        start = __shfl_sync(FULL, start, 0);
        len = __shfl_sync(FULL, len, 0);
        const bool fresh = c != cached;
        cached = c;
        const GridView gt = sub_grid(g, c / g.ncl);  // the grid of the tile's cell (a stack of grids)
        const int s = lane & 15;
        bool active = lane < TILE && s < len;
        int r = 0, steps = 0, switched = 0;
        float t = 0.f, t0 = 0.f, tf = 0.f;
        float4 hist = no_history();
        const bool cycles = a.t_hist != nullptr && !a.coarse;
        Ray ray{};
        if (active) {
            r = a.sorted[start + s];
            t = a.t_ray[r];
            if (cycles) hist = a.t_hist[r];
            steps = a.steps_ray[r];
            if (a.coarse) switched = a.cell_ray[r];  // step count at the BF16 -> FP32 switch
            int cam;
            ray = ray_of(a, r, cam);
            clip_box(gt, ray, t0, tf);
        }
        if (fresh) {
            const bool ok = mbar_wait(&bar, phase, 1u << 26);
            phase ^= 1u;
            if (!__all_sync(FULL, ok)) {  // the weights never landed: report and leave
                if (lane == 0) atomicCAS(a.status, 0, (int)6 /* KNS_ERR_TIMEOUT */);
                return;
            }
        }
        for (int it = 0; it < a.inner_steps; ++it) {
            if (!__any_sync(FULL, active)) break;
            if (lane < TILE) {
                float in[C::INP];
                if (active) {
                    encode3<C::L>(fmaf(t, ray.wx, ray.ox), fmaf(t, ray.wy, ray.oy), fmaf(t, ray.wz, ray.oz), in);
                } else {
#pragma unroll
                    for (int k = 0; k < C::INP; ++k) in[k] = 0.f;
                }
#pragma unroll
                for (int k = 0; k < C::INP; k += 4)
                    *reinterpret_cast<float4 *>(hin + s * SIN + k) = make_float4(in[k], in[k + 1], in[k + 2], in[k + 3]);
            }
            __syncwarp();
            const float d = tile_sdf_f32<C>(wsm, hin, P, Q, lane, g.beta, g.inv_beta);
            {
                const unsigned n = __popc(__ballot_sync(FULL, active) & 0xffffu);
                if (lane == 0) atomicAdd(&a.ctrl->samples_f32, (unsigned long long)n);
            }
            bool hit = false, emit = false;
            int ncell = -1;
            // a thinned-out tile hands its remaining rays to the next round, where they are
            // regrouped into full tiles, instead of running 16-sample GEMMs for a few rays
            const bool sparse = __popc(__ballot_sync(FULL, active)) < a.min_active;
            if (active) {
                ++steps;
                // BF16 renders: after refine_steps FP32 evaluations the FP32 field decides: a hit
                // here if |d| is within the coarse threshold, else the BF16 hit was spurious
                const bool last_refine = a.coarse && steps - switched >= a.refine_steps;
                if (fabsf(d) < a.eps || (last_refine && fabsf(d) < a.eps_coarse)) {
                    hit = true;
                    a.cell_ray[r] = c;
                    a.t_ray[r] = t;
                    a.steps_ray[r] = steps;
                    active = false;
                } else if (last_refine) {
                    write_miss(a, r, steps);
                    active = false;
                } else {
                    const float t_eval = t;
                    t += d;
                    if (t > tf || t < t0 || steps >= a.max_steps) {
                        write_miss(a, r, steps);
                        active = false;
                    } else {
                        ncell = advance_ray(gt, ray, t, tf);
                        if (ncell < 0) {
                            write_miss(a, r, steps);
                            active = false;
                        } else if (cycles && cycle_step(hist, t_eval, t)) {
                            write_miss(a, r, a.max_steps);
                            active = false;
                            ncell = -1;
                        } else if (ncell != c || it + 1 >= a.inner_steps || sparse) {
                            emit = true;
                            a.t_ray[r] = t;
                            a.steps_ray[r] = steps;
                            if (cycles) a.t_hist[r] = hist;
                            active = false;
                        }
                    }
                }
            }
            const int hp = warp_append(&a.ctrl->n_hits, hit);
            if (hit) a.hits[hp] = r;
            const int qp = warp_append(&a.ctrl->n_live[nxt], emit);
            if (emit) {
                a.q[nxt][qp] = r;
                a.qcell[nxt][qp] = ncell;
            }
            warp_count_cells(a.count[nxt], emit, ncell);
        }
    }
}

template <class C>
cudaError_t launch_wave_gen_cfg(const GridView &g, const WaveArgs &a, cudaStream_t s) {
    dim3 grid((a.max_W + 15) / 16, (a.max_H + 7) / 8, a.n_views);
    wave_gen_kernel<C><<<grid, 128, 0, s>>>(g, a);
    return cudaGetLastError();
}
template <class C, int BT, int NT>
cudaError_t launch_block_eval(const GridView &g, const WaveArgs &a, int cur, int sm_count, cudaStream_t s) {
    constexpr int smem = block_eval_smem_bytes<C, BT>();
    static_assert(smem <= 220 * 1024, "block tile does not fit in shared memory");
    static std::atomic<int> per_sm{0};
    int nb = 0;
    cudaError_t e = resident_blocks(wave_eval_block_kernel<C, BT, NT>, NT, smem, per_sm, nb);
    if (e != cudaSuccess) return e;
    wave_eval_block_kernel<C, BT, NT><<<sm_count * nb, NT, smem, s>>>(g, a, cur);
    return cudaGetLastError();
}

template <class C>
cudaError_t launch_wave_eval_cfg(const GridView &g, const WaveArgs &a, int cur, int blocks, int block_tiles,
                                 int sm_count, cudaStream_t s) {
    cudaError_t e;
    if (block_tiles) {
        // the sort's tile size decides the kernel: 256- or 128-sample block tiles, the latter with 256
        // threads (two per sample in the encoding) or 128 (block_tiles == 4: one thread per sample)
        e = a.btile == 256 ? launch_block_eval<C, 256, 256>(g, a, cur, sm_count, s)
            : block_tiles == 4 ? launch_block_eval<C, 128, 128>(g, a, cur, sm_count, s)
                               : launch_block_eval<C, 128, 256>(g, a, cur, sm_count, s);
        if (e != cudaSuccess) return e;
    } else {
        constexpr int smem = eval_smem_bytes<C>();
        static_assert(smem <= 200 * 1024, "eval tile does not fit in shared memory");
        e = cudaFuncSetAttribute(wave_eval_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        wave_eval_kernel<C><<<blocks, 32, smem, s>>>(g, a, cur);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_wave_tail_cfg<C>(g, a, cur, sm_count, s);
}

template <class C>
cudaError_t launch_wave_tail_cfg(const GridView &g, const WaveArgs &a, int cur, int sm_count, cudaStream_t s) {
    // one-warp blocks, as many as fit on the SMs at once (each holds one cell's weights)
    constexpr int tsmem = tail_smem_floats<C>() * (int)sizeof(float);
    static_assert(tsmem <= 64 * 1024, "tail weight slot does not fit");
    static std::atomic<int> tail_per_sm{0};
    int tail_blocks = 0;
    cudaError_t e = resident_blocks(wave_tail_warp_kernel<C, false>, 32, tsmem, tail_per_sm, tail_blocks);
    if (e != cudaSuccess) return e;
    if (g.sub_boxes) {  // a stack of grids (same resources)
        e = cudaFuncSetAttribute(wave_tail_warp_kernel<C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, tsmem);
        if (e != cudaSuccess) return e;
        wave_tail_warp_kernel<C, true><<<sm_count * tail_blocks, 32, tsmem, s>>>(g, a, cur);
    } else {
        wave_tail_warp_kernel<C, false><<<sm_count * tail_blocks, 32, tsmem, s>>>(g, a, cur);
    }
    return cudaGetLastError();
}

#ifdef KNS_W
using InstCfg = Cfg<KNS_W, KNS_H, KNS_L, KNS_LD>;
template cudaError_t launch_wave_gen_cfg<InstCfg>(const GridView &, const WaveArgs &, cudaStream_t);
template cudaError_t launch_wave_eval_cfg<InstCfg>(const GridView &, const WaveArgs &, int, int, int, int,
                                                   cudaStream_t);
template cudaError_t launch_wave_tail_cfg<InstCfg>(const GridView &, const WaveArgs &, int, int, cudaStream_t);
#endif

}  // namespace kns
