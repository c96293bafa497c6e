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
//   - one thread issues the layer's tcgen05.mma chain and commits it to an mbarrier; the block then
//     reads its accumulator rows with tcgen05.ld, adds the bias and applies the softplus in FP32,
//     and writes the next layer's A_hi / A_lo rows back to shared memory (or, after the last hidden
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

// The cell layout of kns_tc.cuh for configuration C, and the block's shared memory: the weights,
// then the activation matrices A_hi, A_lo (128 rows x the widest layer input).
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
    static constexpr int ABYTES = 128 * KA * 2;
    static constexpr int SMEM = SIZE + 2 * ABYTES;
};

// Writes values v[0..7] as columns k0..k0+7 of row `row` of the K-column activation matrices
// (hi at A, lo at A + ABYTES): two 16-byte stores.
template <class T>
__device__ __forceinline__ void put8(unsigned char *A, int row, int K, int k0, const float *v) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        const __nv_bfloat162 ll =
            __floats2bfloat162_rn(v[2 * i] - __low2float(hh), v[2 * i + 1] - __high2float(hh));
        h[i] = *reinterpret_cast<const uint32_t *>(&hh);
        l[i] = *reinterpret_cast<const uint32_t *>(&ll);
    }
    const int o = tc::canon_off(row, k0, K);
    *reinterpret_cast<uint4 *>(A + o) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4 *>(A + T::ABYTES + o) = make_uint4(l[0], l[1], l[2], l[3]);
}

// Encoding of Eq. 1 for row `row` (K0 columns, zero beyond IN): sin and cos of pi p once, then the
// double-angle recurrences sin 2a = 2 sin a cos a, cos 2a = (cos a - sin a)(cos a + sin a) for the
// higher frequencies (error ~1e-6 at the highest, below the hi/lo split's resolution).
template <class C, class T>
__device__ __forceinline__ void encode_row(unsigned char *A, int row, float px, float py, float pz) {
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
    for (int k0 = 0; k0 < T::K0; k0 += 8) put8<T>(A, row, T::K0, k0, in + k0);
}

// One hidden layer on the tensor cores: D = A_hi W_hi + A_lo W_hi + A_hi W_lo over K = kin(l).
template <class T>
__device__ __forceinline__ void issue_layer(uint32_t tmem, uint32_t a_hi, uint32_t w_base, int l, uint64_t *bar) {
    constexpr uint32_t idesc = tc::idesc_bf16_f32(128, T::W);
    const int K = T::kin(l);
    const uint32_t sbo = 16u * K, a_lo = a_hi + T::ABYTES, w_hi = w_base + T::hi(l), w_lo = w_base + T::lo(l);
    for (int ks = 0; ks < K / 16; ++ks) {
        const uint32_t o = 256u * ks;
        const uint64_t ah = tc::smem_desc(a_hi + o, 128, sbo), al = tc::smem_desc(a_lo + o, 128, sbo);
        const uint64_t bh = tc::smem_desc(w_hi + o, 128, sbo), bl = tc::smem_desc(w_lo + o, 128, sbo);
        tc::mma_bf16(tmem, ah, bh, idesc, ks > 0 ? 1u : 0u);
        tc::mma_bf16(tmem, al, bh, idesc, 1u);
        tc::mma_bf16(tmem, ah, bl, idesc, 1u);
    }
    tc::mma_commit(bar);
}

constexpr uint32_t kTcPolls = 1u << 26;  // bound of every mbarrier wait

template <class C>
__global__ void __launch_bounds__(128) wave_eval_tc_kernel(GridView g, WaveArgs a, int cur) {
    using T = TcLayout<C>;
    extern __shared__ __align__(1024) unsigned char dyn[];
    __shared__ __align__(8) uint64_t bar_w, bar_mma;
    __shared__ uint32_t s_tmem;
    __shared__ int s_tile[4];  // key, start, len, fresh
    const int n_tiles = a.ctrl->n_tiles;
    if (n_tiles <= 0) return;  // uniform over the block, before any tensor memory is held
    const int tid = threadIdx.x, warp = tid >> 5, nxt = cur ^ 1;
    unsigned char *wsm = dyn, *A = dyn + T::SIZE;
    const uint32_t w_base = tc::saddr(wsm), a_base = tc::saddr(A);
    if (warp == 0) tc::tmem_alloc(&s_tmem, (uint32_t)T::W);
    if (tid == 0) {
        mbar_init(&bar_w, 1);
        mbar_init(&bar_mma, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    const uint32_t t_lane = tmem + ((uint32_t)(32 * warp) << 16);
    const float *bias = reinterpret_cast<const float *>(wsm + T::BIAS);
    const float *drow = reinterpret_cast<const float *>(wsm + T::DROW);
    const int per = (n_tiles + gridDim.x - 1) / gridDim.x;
    int next_static = blockIdx.x * per;
    const int end_static = min(n_tiles, next_static + per);
    int cached = -1;
    uint32_t ph_w = 0, ph_mma = 0;
    bool w_pending = false, mma_pending = false;  // a copy or a product in flight (for a timeout exit)
    bool failed = false;
    unsigned n_eval = 0;
    const bool cycles = a.t_hist != nullptr;
    for (;;) {
        if (tid == 0) {
            int tile = a.static_tiles ? (next_static < end_static ? next_static : n_tiles)
                                      : atomicAdd(&a.ctrl->next_tile_bf, 1);
            ++next_static;
            int4 d = make_int4(-1, 0, 0, 0);
            if (tile < n_tiles) d = a.tiles[tile];
            const bool fresh = d.x >= 0 && d.x != cached;
            if (fresh) bulk_load(wsm, a.wb + (int64_t)d.x * a.wb_stride, T::SIZE, &bar_w);
            s_tile[0] = d.x;
            s_tile[1] = d.y;
            s_tile[2] = d.z;
            s_tile[3] = fresh;
        }
        __syncthreads();
        const int key = s_tile[0], start = s_tile[1], len = s_tile[2];
        const bool fresh = s_tile[3] != 0;
        if (key < 0) break;
        cached = key;
        const int c = key;
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
            clip_box(g, ray, t0, tf);
        }
        if (fresh) w_pending = true;
        for (int it = 0;; ++it) {
            if (active) encode_row<C, T>(A, tid, fmaf(t, ray.wx, ray.ox), fmaf(t, ray.wy, ray.oy), fmaf(t, ray.wz, ray.oz));
            tc::fence_async_smem();
            if (w_pending) {
                const bool ok = mbar_wait(&bar_w, ph_w, kTcPolls);
                if (__syncthreads_or(!ok)) {
                    failed = true;
                    break;
                }
                ph_w ^= 1u;
                w_pending = false;
            }
            // the hidden layers: products on the tensor cores, bias + softplus + split on the block
            float d = 0.f;
            for (int l = 0; l < C::H; ++l) {
                __syncthreads();
                if (tid == 0) {
                    tc::fence_after_sync();
                    issue_layer<T>(tmem, a_base, w_base, l, &bar_mma);
                }
                mma_pending = true;
                const bool ok = mbar_wait(&bar_mma, ph_mma, kTcPolls);
                if (__syncthreads_or(!ok)) {
                    failed = true;
                    break;
                }
                ph_mma ^= 1u;
                mma_pending = false;
                tc::fence_after_sync();
                if (__any_sync(FULL, active)) {
                    float dacc = drow[T::W];  // the d row's bias (stored right after the row)
#pragma unroll
                    for (int c0 = 0; c0 < T::W; c0 += 32) {
                        float v[32];
                        tc::tmem_ld32(t_lane + (uint32_t)c0, v);
#pragma unroll
                        for (int i = 0; i < 32; ++i) v[i] = softplus_f32(v[i] + bias[l * T::W + c0 + i], g.beta, g.inv_beta);
                        if (l + 1 < C::H) {
#pragma unroll
                            for (int j = 0; j < 32; j += 8) put8<T>(A, tid, T::W, c0 + j, v + j);
                        } else {
#pragma unroll
                            for (int i = 0; i < 32; ++i) dacc = fmaf(drow[c0 + i], v[i], dacc);
                        }
                    }
                    d = dacc;
                }
                tc::fence_async_smem();
                tc::fence_before_sync();
            }
            if (failed) break;
            // outcome: 0 none, 1 converged (hit list), 2 miss (written), 3 pending, 4 emit to ncell
            int outcome = 0, ncell = -1;
            float t_eval = t;
            n_eval += active ? 1u : 0u;
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
                        ncell = advance_fast(g, ray, t);
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
            const int n_cand = __syncthreads_count(cand);
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
        if (failed) break;
        __syncthreads();  // every thread is done with the weights and the tile's state
    }
    if (failed) {
        if (tid == 0) atomicCAS(a.status, 0, (int)6 /* KNS_ERR_TIMEOUT */);
        // let what is in flight land before the block leaves (bounded as well)
        if (w_pending) mbar_wait(&bar_w, ph_w, kTcPolls);
        if (mma_pending) mbar_wait(&bar_mma, ph_mma, kTcPolls);
    }
    {
        const unsigned long long n = warp_sum_u64(n_eval);
        if ((tid & 31) == 0 && n) atomicAdd(&a.ctrl->samples_bf16, n);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, (uint32_t)T::W);
}

template <class C>
cudaError_t launch_wave_eval_tc_cfg(const GridView &g, const WaveArgs &a, int cur, int sm_count, cudaStream_t s) {
    using T = TcLayout<C>;
    static_assert(T::SMEM <= 200 * 1024, "tensor-core tile does not fit in shared memory");
    // Resident blocks per SM from the kernel's own resources (registers, shared memory, threads) and the
    // tensor memory (W of 512 columns per block).  The occupancy query is not used here: for this kernel
    // it reported one block per SM where its registers and shared memory allow five.
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
        nb = std::max(1, std::min(std::min(by_regs, by_smem), std::min(16, 512 / C::W)));
        per_sm.store(nb);
    }
    wave_eval_tc_kernel<C><<<sm_count * nb, 128, T::SMEM, s>>>(g, a, cur);
    return cudaGetLastError();
}

#ifdef KNS_W
using InstCfg = Cfg<KNS_W, KNS_H, KNS_L, KNS_LD>;
template cudaError_t launch_wave_eval_tc_cfg<InstCfg>(const GridView &, const WaveArgs &, int, int, cudaStream_t);
#endif

}  // namespace kns
