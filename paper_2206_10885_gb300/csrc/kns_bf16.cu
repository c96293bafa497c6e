// kns_bf16.cu -- BF16 tensor-core evaluation of the coarse sphere-trace phase.
// kns:instantiate (compiled once per grid configuration)
//
// A warp evaluates the SDF MLP of one cell (Eq. 2, trace form) for a tile of 16 samples with
// mma.sync.m16n8k16 (BF16 inputs, FP32 accumulation): the 16 samples are the M dimension, the layer
// outputs are N (tiles of 8), the layer inputs K (tiles of 16).  The FP32 accumulator fragments of
// one layer, after the softplus, are exactly the A fragments of the next layer (output columns
// 16t..16t+15 = input k-tile t), so activations never leave registers.  The B fragments (weights)
// and biases of the cell are staged in shared memory by one TMA bulk copy; the encoded inputs are
// staged as BF16 rows in shared memory for the first layer's A fragments.
//
// A sample whose BF16 |d| falls below eps_coarse switches its ray to the FP32 phase at the same t:
// FP32 evaluations then decide hit or miss (kns_wave.cu), and shading is FP32.
#include <cuda_bf16.h>

#include "kns_wave.cuh"

namespace kns {

__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], const uint32_t (&a)[4], uint2 b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// Encoding of Eq. 1 for the BF16 phase: sin and cos of pi p once, then the double-angle
// recurrences sin 2a = 2 sin a cos a, cos 2a = (cos a - sin a)(cos a + sin a) for the higher
// frequencies (error ~1e-6, far below BF16 rounding).
template <int L, int NOUT>
__device__ __forceinline__ void encode3_rec(float px, float py, float pz, float (&out)[NOUT]) {
    out[0] = px;
    out[1] = py;
    out[2] = pz;
    float s[3], c[3];
    sincospif(px, &s[0], &c[0]);
    sincospif(py, &s[1], &c[1]);
    sincospif(pz, &s[2], &c[2]);
#pragma unroll
    for (int k = 0; k < L; ++k) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            out[3 + 6 * k + a] = s[a];
            out[3 + 6 * k + 3 + a] = c[a];
            const float s2 = 2.f * s[a] * c[a], c2 = (c[a] - s[a]) * (c[a] + s[a]);
            s[a] = s2;
            c[a] = c2;
        }
    }
#pragma unroll
    for (int i = 3 + 6 * L; i < NOUT; ++i) out[i] = 0.f;
}

template <class C>
__host__ __device__ constexpr int pe_words() {  // BF16 input row stride in 32-bit words (bank-conflict free)
    return C::K0P / 2 + 4;
}

// d of the 16 samples whose BF16 inputs are in pe[s][k]; returns d of sample lane % 16.
template <class C>
__device__ __forceinline__ float tile_sdf_bf16(const unsigned char *wsm, const uint32_t *pe, int lane, float beta,
                                               float inv_beta) {
    constexpr int KA = C::KT0 > C::KTH ? C::KT0 : C::KTH;
    constexpr int PEW = pe_words<C>();
    const uint2 *fr = reinterpret_cast<const uint2 *>(wsm);
    const int r = lane >> 2, q = lane & 3;
    uint32_t A[KA][4];
#pragma unroll
    for (int kt = 0; kt < C::KT0; ++kt) {
        A[kt][0] = pe[r * PEW + 8 * kt + q];
        A[kt][1] = pe[(r + 8) * PEW + 8 * kt + q];
        A[kt][2] = pe[r * PEW + 8 * kt + 4 + q];
        A[kt][3] = pe[(r + 8) * PEW + 8 * kt + 4 + q];
    }
    float acc[C::NT][4];
    // layer 0
    {
        const float *bias = reinterpret_cast<const float *>(wsm + C::BBl(0));
#pragma unroll
        for (int nt = 0; nt < C::NT; ++nt) {
            const float b0 = bias[8 * nt + 2 * q], b1 = bias[8 * nt + 2 * q + 1];
            acc[nt][0] = b0;
            acc[nt][1] = b1;
            acc[nt][2] = b0;
            acc[nt][3] = b1;
#pragma unroll
            for (int kt = 0; kt < C::KT0; ++kt) mma_bf16_16816(acc[nt], A[kt], fr[(C::FR0 + kt * C::NT + nt) * 32 + lane]);
        }
    }
#pragma unroll
    for (int l = 1; l <= C::H; ++l) {
        // softplus of layer l-1, repacked as layer l's A fragments
#pragma unroll
        for (int kt = 0; kt < C::KTH; ++kt) {
            A[kt][0] = pack_bf16x2(softplus_f32(acc[2 * kt][0], beta, inv_beta), softplus_f32(acc[2 * kt][1], beta, inv_beta));
            A[kt][1] = pack_bf16x2(softplus_f32(acc[2 * kt][2], beta, inv_beta), softplus_f32(acc[2 * kt][3], beta, inv_beta));
            A[kt][2] = pack_bf16x2(softplus_f32(acc[2 * kt + 1][0], beta, inv_beta),
                                   softplus_f32(acc[2 * kt + 1][1], beta, inv_beta));
            A[kt][3] = pack_bf16x2(softplus_f32(acc[2 * kt + 1][2], beta, inv_beta),
                                   softplus_f32(acc[2 * kt + 1][3], beta, inv_beta));
        }
        if (l == C::H) break;
        const float *bias = reinterpret_cast<const float *>(wsm + C::BBl(l));
#pragma unroll
        for (int nt = 0; nt < C::NT; ++nt) {
            const float b0 = bias[8 * nt + 2 * q], b1 = bias[8 * nt + 2 * q + 1];
            acc[nt][0] = b0;
            acc[nt][1] = b1;
            acc[nt][2] = b0;
            acc[nt][3] = b1;
#pragma unroll
            for (int kt = 0; kt < C::KTH; ++kt) mma_bf16_16816(acc[nt], A[kt], fr[(C::FRl(l) + kt * C::NT + nt) * 32 + lane]);
        }
    }
    // last layer: only column 0 (d) is populated
    const float bd = *reinterpret_cast<const float *>(wsm + C::BBL);
    float dd[4] = {q == 0 ? bd : 0.f, 0.f, q == 0 ? bd : 0.f, 0.f};
#pragma unroll
    for (int kt = 0; kt < C::KTH; ++kt) mma_bf16_16816(dd, A[kt], fr[(C::FRL + kt) * 32 + lane]);
    // d of sample s sits in lane 4 (s % 8): c0 for s < 8, c2 for s >= 8
    const float d_lo = __shfl_sync(FULL, dd[0], 4 * (lane & 7));
    const float d_hi = __shfl_sync(FULL, dd[2], 4 * (lane & 7));
    return (lane & 8) ? d_hi : d_lo;
}

template <class C>
__host__ __device__ constexpr int bf16_eval_smem_bytes() {
    return C::BSIZE + TILE * pe_words<C>() * 4;
}

// One round of the BF16 phase: tiles of BF16 samples (keys NC..2NC-1), one warp per block.
template <class C>
__global__ void __launch_bounds__(32) wave_eval_bf16_kernel(GridView g, WaveArgs a, int cur) {
    extern __shared__ __align__(128) unsigned char dynb[];
    __shared__ __align__(8) uint64_t bar;
    const int lane = threadIdx.x;
    const int nxt = cur ^ 1;
    unsigned char *wsm = dynb;
    uint32_t *pe = reinterpret_cast<uint32_t *>(dynb + C::BSIZE);
    constexpr int PEW = pe_words<C>();
    const int t_first = a.ctrl->n_tiles_fine, t_end_all = a.ctrl->n_tiles;
    const int n_tiles = t_end_all - t_first;
    if (n_tiles <= 0) return;
    if (lane == 0) mbar_init(&bar, 1);
    __syncwarp();
    const int per = (n_tiles + gridDim.x - 1) / gridDim.x;
    int next_static = blockIdx.x * per;
    const int end_static = min(n_tiles, next_static + per);
    int cached = -1;
    uint32_t phase = 0;
    for (;;) {
        int tile = 0;
        if (lane == 0) tile = a.static_tiles ? (next_static < end_static ? next_static : n_tiles)
                                             : atomicAdd(&a.ctrl->next_tile_bf, 1);
        tile = __shfl_sync(FULL, tile, 0);
        ++next_static;
        if (tile >= n_tiles) break;
        tile += t_first;
        int key = 0, start = 0, len = 0;
        if (lane == 0) {
            int lo = a.NC, hi = a.nkeys;  // the key with tile_off[key] <= tile < tile_off[key+1]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(a.tile_off + mid) <= tile) lo = mid; else hi = mid;
            }
            key = lo;
            start = __ldg(a.off + lo) + (tile - __ldg(a.tile_off + lo)) * TILE;
            len = min(TILE, __ldg(a.off + lo + 1) - start);
            if (key != cached) bulk_load(wsm, a.wb + (int64_t)(key - a.NC) * a.wb_stride, C::BSIZE, &bar);
        }
        key = __shfl_sync(FULL, key, 0);
        start = __shfl_sync(FULL, start, 0);
        len = __shfl_sync(FULL, len, 0);
        const int c = key - a.NC;
        const bool fresh = key != cached;
        cached = key;
        const int s = lane & 15;
        bool active = lane < TILE && s < len;
        int r = 0, steps = 0;
        float t = 0.f, t0 = 0.f, tf = 0.f;
        // cycle test of the BF16 phase: its positions and d values come from this one evaluator, and a
        // cycle never meets |d| < eps_coarse, so it ends as a budget miss (the FP32 phase keeps none)
        const bool cycles = a.t_hist != nullptr;
        float4 hist = no_history();
        Ray ray{};
        if (active) {
            r = a.sorted[start + s];
            t = a.t_ray[r];
            steps = a.steps_ray[r];
            if (cycles) hist = a.t_hist[r];
            int cam;
            ray = ray_of(a, r, cam);
            clip_box(g, ray, t0, tf);
        }
        if (fresh) {
            const bool ok = mbar_wait(&bar, phase, 1u << 26);
            phase ^= 1u;
            if (!__all_sync(FULL, ok)) {
                if (lane == 0) atomicCAS(a.status, 0, (int)6 /* KNS_ERR_TIMEOUT */);
                return;
            }
        }
        for (int it = 0; it < a.inner_steps; ++it) {
            if (!__any_sync(FULL, active)) break;
            if (lane < TILE) {
                float in[C::K0P];
                if (active) {
                    encode3_rec<C::L>(fmaf(t, ray.wx, ray.ox), fmaf(t, ray.wy, ray.oy), fmaf(t, ray.wz, ray.oz), in);
                } else {
#pragma unroll
                    for (int k = 0; k < C::K0P; ++k) in[k] = 0.f;
                }
#pragma unroll
                for (int k = 0; k < C::K0P; k += 2) pe[s * PEW + k / 2] = pack_bf16x2(in[k], in[k + 1]);
            }
            __syncwarp();
            const float d = tile_sdf_bf16<C>(wsm, pe, lane, g.beta, g.inv_beta);
            {
                const unsigned n = __popc(__ballot_sync(FULL, active) & 0xffffu);
                if (lane == 0) atomicAdd(&a.ctrl->samples_bf16, (unsigned long long)n);
            }
            __syncwarp();
            bool emit = false;
            int nkey = -1;
            const bool sparse = __popc(__ballot_sync(FULL, active)) < a.min_active;
            if (active) {
                ++steps;
                if (fabsf(d) < a.eps_coarse) {
                    // coarse hit: the ray continues in FP32 at this t; cell_ray marks the step count
                    // of the switch so the FP32 phase can count its refinement evaluations
                    if (steps >= a.max_steps) {
                        write_miss(a, r, steps);
                    } else {
                        emit = true;
                        nkey = c;
                        a.cell_ray[r] = steps;
                        a.t_ray[r] = t;
                        a.steps_ray[r] = steps;
                    }
                    active = false;
                } else {
                    const float t_eval = t;
                    t += d;
                    if (t > tf || t < t0 || steps >= a.max_steps) {
                        write_miss(a, r, steps);
                        active = false;
                    } else {
                        const int ncell = advance_ray(g, ray, t, tf);
                        if (ncell < 0) {
                            write_miss(a, r, steps);
                            active = false;
                        } else if (cycles && cycle_step(hist, t_eval, t)) {
                            write_miss(a, r, a.max_steps);
                            active = false;
                        } else if (ncell != c || it + 1 >= a.inner_steps || sparse) {
                            emit = true;
                            nkey = ncell + a.NC;
                            a.t_ray[r] = t;
                            a.steps_ray[r] = steps;
                            if (cycles) a.t_hist[r] = hist;
                            active = false;
                        }
                    }
                }
            }
            const int qp = warp_append(&a.ctrl->n_live[nxt], emit);
            if (emit) {
                a.q[nxt][qp] = r;
                a.qcell[nxt][qp] = nkey;
            }
            warp_count_cells(a.count[nxt], emit, nkey);
        }
    }
}

template <class C>
cudaError_t launch_wave_eval_bf16_cfg(const GridView &g, const WaveArgs &a, int cur, int blocks, cudaStream_t s) {
    constexpr int smem = bf16_eval_smem_bytes<C>();
    cudaError_t e = cudaFuncSetAttribute(wave_eval_bf16_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    wave_eval_bf16_kernel<C><<<blocks, 32, smem, s>>>(g, a, cur);
    return cudaGetLastError();
}

#ifdef KNS_W
using InstCfg = Cfg<KNS_W, KNS_H, KNS_L, KNS_LD>;
template cudaError_t launch_wave_eval_bf16_cfg<InstCfg>(const GridView &, const WaveArgs &, int, int, cudaStream_t);
#endif

}  // namespace kns
