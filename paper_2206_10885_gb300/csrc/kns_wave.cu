// kns_wave.cu -- wavefront render kernels (FP32): ray generation, per-cell tile evaluation, shading.
// kns:instantiate (compiled once per grid configuration)
//
// Tile evaluation: a warp evaluates the SDF MLP of one cell (Eq. 2, trace form: d only) for up to
// 16 samples at once as a register-blocked GEMM per layer.  Activations live in shared memory as
// h[k][s] (k = input unit, s = sample); lane (sg, ng) = (lane / 8, lane % 8) accumulates samples
// 4sg..4sg+3 against output units ng*W/8 .. ng*W/8 + W/8 - 1, so each shared-memory float4 of
// activations and each float4 of k-major weights feed 16 (W = 32) or 32 (W = 64) FMAs.
#include "kns_wave.cuh"

namespace kns {

// One layer of the tile: hout[o][s] = softplus(sum_k Wt[k][o] hin[k][s] + b[o]).
template <int K, int W>
__device__ __forceinline__ void tile_layer_f32(const float *__restrict__ Wt, const float *__restrict__ b,
                                               const float *hin, float *hout, int lane, float beta,
                                               float inv_beta) {
    constexpr int NPL = W / 8;  // output units per lane
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
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
        const float4 a = *reinterpret_cast<const float4 *>(hin + k * TILE + 4 * sg);
#pragma unroll
        for (int j = 0; j < NPL; j += 4) {
            const float4 w = *reinterpret_cast<const float4 *>(Wt + k * W + ng * NPL + j);
            acc[0][j] = fmaf(a.x, w.x, acc[0][j]);
            acc[0][j + 1] = fmaf(a.x, w.y, acc[0][j + 1]);
            acc[0][j + 2] = fmaf(a.x, w.z, acc[0][j + 2]);
            acc[0][j + 3] = fmaf(a.x, w.w, acc[0][j + 3]);
            acc[1][j] = fmaf(a.y, w.x, acc[1][j]);
            acc[1][j + 1] = fmaf(a.y, w.y, acc[1][j + 1]);
            acc[1][j + 2] = fmaf(a.y, w.z, acc[1][j + 2]);
            acc[1][j + 3] = fmaf(a.y, w.w, acc[1][j + 3]);
            acc[2][j] = fmaf(a.z, w.x, acc[2][j]);
            acc[2][j + 1] = fmaf(a.z, w.y, acc[2][j + 1]);
            acc[2][j + 2] = fmaf(a.z, w.z, acc[2][j + 2]);
            acc[2][j + 3] = fmaf(a.z, w.w, acc[2][j + 3]);
            acc[3][j] = fmaf(a.w, w.x, acc[3][j]);
            acc[3][j + 1] = fmaf(a.w, w.y, acc[3][j + 1]);
            acc[3][j + 2] = fmaf(a.w, w.z, acc[3][j + 2]);
            acc[3][j + 3] = fmaf(a.w, w.w, acc[3][j + 3]);
        }
    }
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
        float4 v;
        v.x = softplus_f32(acc[0][j], beta, inv_beta);
        v.y = softplus_f32(acc[1][j], beta, inv_beta);
        v.z = softplus_f32(acc[2][j], beta, inv_beta);
        v.w = softplus_f32(acc[3][j], beta, inv_beta);
        *reinterpret_cast<float4 *>(hout + (ng * NPL + j) * TILE + 4 * sg) = v;
    }
}

// SDF trace form for a tile whose encoded inputs are in hA[k][s]; returns d of sample lane % 16.
template <class C>
__device__ __forceinline__ float tile_sdf_f32(const float *__restrict__ wt, float *hA, float *hB, int lane,
                                              float beta, float inv_beta) {
    tile_layer_f32<C::INP, C::W>(wt + C::tW0, wt + C::tb0, hA, hB, lane, beta, inv_beta);
    __syncwarp();
    float *src = hB, *dst = hA;
#pragma unroll
    for (int l = 1; l < C::H; ++l) {
        tile_layer_f32<C::W, C::W>(wt + C::tWl(l), wt + C::tbl(l), src, dst, lane, beta, inv_beta);
        __syncwarp();
        float *tmp = src;
        src = dst;
        dst = tmp;
    }
    const int s = lane & 15, half = lane >> 4;
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < C::W / 2; ++k) {
        const int kk = half * (C::W / 2) + k;
        acc = fmaf(wt[C::tdL + kk], src[kk * TILE + s], acc);
    }
    acc += __shfl_xor_sync(FULL, acc, 16);
    return acc + wt[C::tbL];
}

// Wave 0: one thread per pixel (16x8 pixels per block, 8x4 per warp); clip, advance, emit.
template <class C>
__global__ void __launch_bounds__(128) wave_gen_kernel(GridView g, WaveArgs a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = blockIdx.x * 16 + (warp & 1) * 8 + (lane & 7);
    const int i = blockIdx.y * 8 + (warp >> 1) * 4 + (lane >> 3);
    const int cam = blockIdx.z;
    const bool valid = i < a.H && j < a.W;
    const int r = cam * a.W * a.H + i * a.W + j;
    bool alive = false;
    int cell = -1;
    if (valid) {
        const Ray ray = make_ray(a.cams + 16 * cam, i, j);
        float t0, tf;
        if (!clip_box(g, ray, t0, tf)) {
            write_miss(a, r, 0);
        } else {
            float t = t0;
            cell = advance_ray(g, ray, t, tf);
            if (cell < 0) {
                write_miss(a, r, 0);
            } else {
                alive = true;
                a.t_ray[r] = t;
                a.steps_ray[r] = 0;
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

// Round k: each block takes a tile of up to 64 cell-sorted samples of one cell (dynamic
// scheduling), stages the cell's k-major weights in shared memory with one TMA bulk copy, and each
// of its 4 warps evaluates 16 samples.  Rays whose next sample stays in the same cell keep
// stepping inside the tile (up to inner_steps evaluations this round); the others are emitted to
// round k+1 (with their next cell), converge (hit list) or terminate (miss written).
constexpr int EVAL_WARPS = 4;

template <class C>
__host__ __device__ constexpr int eval_hrows() {
    return C::INP > C::W ? C::INP : C::W;
}
template <class C>
__host__ __device__ constexpr int eval_smem_bytes() {
    return (C::TSIZE + EVAL_WARPS * 2 * eval_hrows<C>() * TILE) * (int)sizeof(float);
}

template <class C>
__global__ void __launch_bounds__(EVAL_WARPS * 32) wave_eval_kernel(GridView g, WaveArgs a, int cur) {
    extern __shared__ __align__(128) float dyn[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_tile, s_cell, s_start, s_len;
    float *wsm = dyn;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *hA = dyn + C::TSIZE + warp * 2 * eval_hrows<C>() * TILE;
    float *hB = hA + eval_hrows<C>() * TILE;
    const int nxt = cur ^ 1;
    const int n_tiles = a.ctrl->n_tiles;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    int cached = -1;
    uint32_t phase = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            const int tile = atomicAdd(&a.ctrl->next_tile, 1);
            s_tile = tile;
            if (tile < n_tiles) {
                int lo = 0, hi = a.NC;  // the cell c with tile_off[c] <= tile < tile_off[c+1]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (__ldg(a.tile_off + mid) <= tile) lo = mid; else hi = mid;
                }
                const int start = __ldg(a.off + lo) + (tile - __ldg(a.tile_off + lo)) * a.btile;
                s_cell = lo;
                s_start = start;
                s_len = min(a.btile, __ldg(a.off + lo + 1) - start);
                if (lo != cached)
                    bulk_load(wsm, a.wt + (int64_t)lo * a.wt_stride, C::TSIZE * sizeof(float), &bar);
            }
        }
        __syncthreads();
        if (s_tile >= n_tiles) break;
        const int c = s_cell;
        const bool fresh = c != cached;
        cached = c;
        // this warp's samples
        const int wstart = s_start + warp * TILE;
        const int wlen = max(0, min(TILE, s_len - warp * TILE));
        const int s = lane & 15;
        bool active = lane < TILE && s < wlen;
        int r = 0, steps = 0;
        float t = 0.f, t0 = 0.f, tf = 0.f;
        Ray ray{};
        if (active) {
            r = a.sorted[wstart + s];
            t = a.t_ray[r];
            steps = a.steps_ray[r];
            int cam;
            ray = ray_of(a, r, cam);
            clip_box(g, ray, t0, tf);
        }
        if (fresh) {
            const bool ok = mbar_wait(&bar, phase, 1u << 26);
            phase ^= 1u;
            if (__syncthreads_or(!ok)) {  // the copy never landed: report and leave
                if (threadIdx.x == 0) atomicCAS(a.status, 0, (int)6 /* KNS_ERR_TIMEOUT */);
                mbar_wait(&bar, phase ^ 1u, 1u << 20);
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
                for (int k = 0; k < C::INP; ++k) hA[k * TILE + s] = in[k];
            }
            __syncwarp();
            const float d = tile_sdf_f32<C>(wsm, hA, hB, lane, g.beta, g.inv_beta);
            bool hit = false, emit = false, stay = false;
            int ncell = -1;
            if (active) {
                ++steps;
                if (fabsf(d) < a.eps) {
                    hit = true;
                    a.cell_ray[r] = c;
                    a.t_ray[r] = t;
                    a.steps_ray[r] = steps;
                } else {
                    t += d;
                    if (t > tf || t < t0 || steps >= a.max_steps) {
                        write_miss(a, r, steps);
                    } else {
                        ncell = advance_ray(g, ray, t, tf);
                        if (ncell < 0) {
                            write_miss(a, r, steps);
                        } else if (ncell == c && it + 1 < a.inner_steps) {
                            stay = true;
                        } else {
                            emit = true;
                            a.t_ray[r] = t;
                            a.steps_ray[r] = steps;
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
            active = stay;
            __syncwarp();
        }
        __syncthreads();  // the weights buffer and tile slots are reused by the next tile
    }
}

// Shading of converged rays: full SDF MLP with its input gradient (normal), colour MLP (Eq. 3).
template <class C>
__global__ void __launch_bounds__(128) wave_shade_kernel(GridView g, WaveArgs a) {
    const int n = a.ctrl->n_hits;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const int r = a.hits[q];
        const int c = a.cell_ray[r];
        const float t = a.t_ray[r];
        int cam;
        const Ray ray = ray_of(a, r, cam);
        const float x = fmaf(t, ray.wx, ray.ox), y = fmaf(t, ray.wy, ray.oy), z = fmaf(t, ray.wz, ray.oz);
        const float *cw = g.w + (int64_t)c * g.cell_stride;
        float feat[FEAT], grad[3], nrm[3], rgb[3];
        sdf_full_f32<C>(cw, x, y, z, g.beta, g.inv_beta, feat, grad);
        const float gn = sqrtf(fmaf(grad[0], grad[0], fmaf(grad[1], grad[1], grad[2] * grad[2])));
        const float inv = gn > 0.f ? 1.f / gn : 0.f;
        nrm[0] = grad[0] * inv;
        nrm[1] = grad[1] * inv;
        nrm[2] = grad[2] * inv;
        colour_f32<C>(cw, feat, nrm, ray.wx, ray.wy, ray.wz, x, y, z, rgb);
        a.rgb[3 * (int64_t)r + 0] = rgb[0];
        a.rgb[3 * (int64_t)r + 1] = rgb[1];
        a.rgb[3 * (int64_t)r + 2] = rgb[2];
        a.depth[r] = t;
        if (a.normal) {
            a.normal[3 * (int64_t)r + 0] = nrm[0];
            a.normal[3 * (int64_t)r + 1] = nrm[1];
            a.normal[3 * (int64_t)r + 2] = nrm[2];
        }
        if (a.cell_out) a.cell_out[r] = c;
        if (a.steps_out) a.steps_out[r] = a.steps_ray[r];
        if (a.hit_out) a.hit_out[r] = 1;
    }
}

template <class C>
cudaError_t launch_wave_gen_cfg(const GridView &g, const WaveArgs &a, cudaStream_t s) {
    dim3 grid((a.W + 15) / 16, (a.H + 7) / 8, a.n_cams);
    wave_gen_kernel<C><<<grid, 128, 0, s>>>(g, a);
    return cudaGetLastError();
}
template <class C>
cudaError_t launch_wave_eval_cfg(const GridView &g, const WaveArgs &a, int cur, int blocks, cudaStream_t s) {
    constexpr int smem = eval_smem_bytes<C>();
    static_assert(smem <= 200 * 1024, "eval tile does not fit in shared memory");
    cudaError_t e = cudaFuncSetAttribute(wave_eval_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    wave_eval_kernel<C><<<blocks, EVAL_WARPS * 32, smem, s>>>(g, a, cur);
    return cudaGetLastError();
}
template <class C>
cudaError_t launch_wave_shade_cfg(const GridView &g, const WaveArgs &a, int blocks, cudaStream_t s) {
    wave_shade_kernel<C><<<blocks, 128, 0, s>>>(g, a);
    return cudaGetLastError();
}

#ifdef KNS_W
using InstCfg = Cfg<KNS_W, KNS_H, KNS_L, KNS_LD>;
template cudaError_t launch_wave_gen_cfg<InstCfg>(const GridView &, const WaveArgs &, cudaStream_t);
template cudaError_t launch_wave_eval_cfg<InstCfg>(const GridView &, const WaveArgs &, int, int, cudaStream_t);
template cudaError_t launch_wave_shade_cfg<InstCfg>(const GridView &, const WaveArgs &, int, cudaStream_t);
#endif

}  // namespace kns
