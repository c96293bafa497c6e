// kns_train.cu -- the NeuS-style training step on a Kilo-grid: loss and hand-written backward.
//
// What is computed (Sec. 3.2.2 loss, Sec. 3.3 finite differences; NeuS volume rendering):
//   per ray, Ns stratified samples in the box interval, SDF at each (coarse pass), NeuS weights with
//   Phi = sigmoid(s_up d), Ni importance samples by inverting their CDF, all S = Ns + Ni merged;
//   at each sample the SDF d, feature z, a normal from central differences of d (step h, each point
//   in its own cell), the colour MLP, NeuS opacity alpha_i = max(1 - Phi(s d_{i+1}) / Phi(s d_i), 0),
//   C = sum_i T_i alpha_i c_i; L = mean |C - I|_1 + lambda mean (|grad d| - 1)^2 over eikonal points,
//   the gradient again by central differences.  Sample positions are not differentiated.
//
// How: every SDF evaluation is a record (a point and an id).  This file makes the records and
// counting-sorts them by the cell that evaluates them (chunks of at most CHUNK records of one cell
// are what the grouped MLP kernels of kns_train_tile.cu take), places the importance samples, and
// does the per-ray volume rendering, the loss and the upstream gradients of the rendered samples.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kns_kernels.h"
#include "kns_train.cuh"

namespace kns {
namespace {

using train::CHUNK;
using train::MAXS;
using train::fd_normal;
using train::grid_for;
using train::load3;

// ------------------------------------------------------------------ activations
__device__ __forceinline__ float sigm(float s) { return 1.f / (1.f + expf(-s)); }
// log sigmoid(x), stable for any x
__device__ __forceinline__ float log_sigm(float x) {
    return x < 0.f ? x - log1pf(expf(x)) : -log1pf(expf(-x));
}

// ------------------------------------------------------------------ geometry
__device__ __forceinline__ int axis_cell(float x, float bmin, float scale, int n) {
    float u = floorf((x - bmin) * scale);
    u = fminf(fmaxf(u, 0.f), (float)(n - 1));
    return (int)u;
}
__device__ __forceinline__ int cell_at(const TrainArgs &a, float x, float y, float z) {
    return axis_cell(x, a.bmin[0], a.cscale[0], a.N) +
           a.N * (axis_cell(y, a.bmin[1], a.cscale[1], a.N) + a.N * axis_cell(z, a.bmin[2], a.cscale[2], a.N));
}
// slab test: true with [tn, tf], tn = max(t_near, 0)
__device__ __forceinline__ bool clip_ray(const TrainArgs &a, const float *o, const float *w, float &tn, float &tf) {
    float lo = -INFINITY, hi = INFINITY;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (w[k] != 0.f) {
            const float t1 = (a.bmin[k] - o[k]) / w[k], t2 = (a.bmax[k] - o[k]) / w[k];
            lo = fmaxf(lo, fminf(t1, t2));
            hi = fminf(hi, fmaxf(t1, t2));
        } else if (o[k] < a.bmin[k] || o[k] > a.bmax[k]) {
            return false;
        }
    }
    if (lo > hi || hi < 0.f) return false;
    tn = fmaxf(lo, 0.f);
    tf = hi;
    return true;
}
__device__ __forceinline__ float strat_t(float tn, float tf, int i, float u, int Ns) {
    return tn + ((float)i + u) / (float)Ns * (tf - tn);
}

// ------------------------------------------------------------------ records
// coarse record rec = r * Ns + i: the i-th stratified sample of ray r
__device__ __forceinline__ bool coarse_record(const TrainArgs &a, int64_t rec, float3 &x, int &key) {
    const int64_t r = rec / a.Ns;
    const int i = (int)(rec - r * a.Ns);
    float o[3], w[3], tn, tf;
    load3(a.o + 3 * r, o);
    load3(a.w + 3 * r, w);
    if (!clip_ray(a, o, w, tn, tf)) return false;
    const float t = strat_t(tn, tf, i, __ldg(a.u_s + rec), a.Ns);
    x = make_float3(o[0] + t * w[0], o[1] + t * w[1], o[2] + t * w[2]);
    key = cell_at(a, x.x, x.y, x.z);
    return true;
}
// fine records: [0, 6 B S) difference points of the samples (6 q + k), [6 B S, 6 (B S + M)) those of
// the eikonal points, then the B S sample centres (key NC + cell).  k = 2 axis + (0: +h, 1: -h).
__device__ __forceinline__ bool fine_record(const TrainArgs &a, int64_t rec, float3 &x, int &key) {
    const int64_t nbs = a.B * a.S, nfd = 6 * (nbs + a.M);
    float p[3];
    if (rec < nfd) {
        const int64_t q = rec / 6;
        const int k = (int)(rec - 6 * q);
        if (q < nbs) {
            const int64_t r = q / a.S;
            if (!a.valid[r]) return false;
            float o[3], w[3];
            load3(a.o + 3 * r, o);
            load3(a.w + 3 * r, w);
            const float t = a.t[q];
            p[0] = o[0] + t * w[0];
            p[1] = o[1] + t * w[1];
            p[2] = o[2] + t * w[2];
        } else {
            load3(a.P + 3 * (q - nbs), p);
        }
        p[k >> 1] += (k & 1) ? -a.h : a.h;
        x = make_float3(p[0], p[1], p[2]);
        key = cell_at(a, p[0], p[1], p[2]);
        return true;
    }
    const int64_t q = rec - nfd;
    const int64_t r = q / a.S;
    if (!a.valid[r]) return false;
    float o[3], w[3];
    load3(a.o + 3 * r, o);
    load3(a.w + 3 * r, w);
    const float t = a.t[q];
    x = make_float3(o[0] + t * w[0], o[1] + t * w[1], o[2] + t * w[2]);
    key = a.NC + cell_at(a, x.x, x.y, x.z);
    return true;
}
template <int WHICH>
__device__ __forceinline__ bool make_record(const TrainArgs &a, int64_t rec, float3 &x, int &key) {
    return WHICH == TRAIN_COARSE ? coarse_record(a, rec, x, key) : fine_record(a, rec, x, key);
}

// ------------------------------------------------------------------ counting sort by key
__device__ __forceinline__ unsigned lanes_below() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <int WHICH>
__global__ void __launch_bounds__(256) k_hist(TrainArgs a, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t rec = base + threadIdx.x;
        float3 x;
        int key = -1;
        const bool ok = rec < n && make_record<WHICH>(a, rec, x, key);
        const unsigned act = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            const unsigned peers = __match_any_sync(act, key);
            if ((peers & lanes_below()) == 0) atomicAdd(a.count + key, __popc(peers));
        }
    }
}

// exclusive scans of count (-> off) and of chunks per key (-> chunk_off); clears the scatter cursors
__global__ void __launch_bounds__(1024) k_scan(TrainArgs a) {
    __shared__ int s_a[1024], s_b[1024];
    const int n = a.nkeys, per = (n + blockDim.x - 1) / blockDim.x;
    const int k0 = threadIdx.x * per, k1 = min(k0 + per, n);
    int sa = 0, sb = 0;
    for (int k = k0; k < k1; ++k) {
        const int c = a.count[k];
        sa += c;
        sb += (c + CHUNK - 1) / CHUNK;
    }
    s_a[threadIdx.x] = sa;
    s_b[threadIdx.x] = sb;
    __syncthreads();
    for (int d = 1; d < (int)blockDim.x; d <<= 1) {
        const int va = threadIdx.x >= (unsigned)d ? s_a[threadIdx.x - d] : 0;
        const int vb = threadIdx.x >= (unsigned)d ? s_b[threadIdx.x - d] : 0;
        __syncthreads();
        s_a[threadIdx.x] += va;
        s_b[threadIdx.x] += vb;
        __syncthreads();
    }
    int ra = s_a[threadIdx.x] - sa, rb = s_b[threadIdx.x] - sb;
    for (int k = k0; k < k1; ++k) {
        const int c = a.count[k];
        a.off[k] = ra;
        a.chunk_off[k] = rb;
        a.fill[k] = 0;
        ra += c;
        rb += (c + CHUNK - 1) / CHUNK;
    }
    if (threadIdx.x == blockDim.x - 1) {
        a.off[n] = s_a[threadIdx.x];
        a.chunk_off[n] = s_b[threadIdx.x];
    }
}

template <int WHICH>
__global__ void __launch_bounds__(256) k_scatter(TrainArgs a, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t rec = base + threadIdx.x;
        float3 x;
        int key = -1;
        const bool ok = rec < n && make_record<WHICH>(a, rec, x, key);
        const unsigned act = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            const unsigned peers = __match_any_sync(act, key);
            const int leader = __ffs(peers) - 1;
            int pos = 0;
            if ((int)(threadIdx.x & 31) == leader) pos = atomicAdd(a.fill + key, __popc(peers));
            pos = __shfl_sync(peers, pos, leader) + __popc(peers & lanes_below());
            a.sorted[a.off[key] + pos] = make_float4(x.x, x.y, x.z, __int_as_float((int)rec));
        }
    }
}

// ------------------------------------------------------------------ importance sampling
__global__ void __launch_bounds__(128) k_importance(TrainArgs a) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.B) return;
    float o[3], w[3], tn, tf;
    load3(a.o + 3 * r, o);
    load3(a.w + 3 * r, w);
    float *t = a.t + r * a.S;
    if (!clip_ray(a, o, w, tn, tf)) {
        a.valid[r] = 0;
        for (int i = 0; i < a.S; ++i) t[i] = 0.f;
        return;
    }
    a.valid[r] = 1;
    const int Ns = a.Ns, Ni = a.Ni;
    float tc[MAXS], cdf[MAXS];
    for (int i = 0; i < Ns; ++i) tc[i] = strat_t(tn, tf, i, __ldg(a.u_s + r * Ns + i), Ns);
    // coarse NeuS weights on the Ns - 1 intervals (+1e-5 floor), cumulated
    const float *dc = a.d_coarse + r * Ns;
    float T = 1.f, tot = 0.f, ls = log_sigm(a.s_up * dc[0]);
    cdf[0] = 0.f;
    for (int i = 0; i + 1 < Ns; ++i) {
        const float ls1 = log_sigm(a.s_up * dc[i + 1]);
        const float alpha = fmaxf(1.f - expf(ls1 - ls), 0.f);
        tot += T * alpha + 1e-5f;
        T *= 1.f - alpha;
        cdf[i + 1] = tot;
        ls = ls1;
    }
    const float inv = 1.f / tot;
    for (int i = 1; i < Ns; ++i) cdf[i] *= inv;
    // invert at the (ascending) uniforms and merge with the stratified samples
    int ia = 0, ib = 0, k = 0, j = 0;
    float timp = INFINITY;
    auto next_imp = [&](int b) {
        const float u = __ldg(a.u_i + r * Ni + b);
        while (j + 2 < Ns && cdf[j + 1] <= u) ++j;
        const float den = cdf[j + 1] - cdf[j];
        return tc[j] + (den > 0.f ? (u - cdf[j]) / den : 0.f) * (tc[j + 1] - tc[j]);
    };
    if (Ni > 0) timp = next_imp(0);
    while (ia < Ns || ib < Ni) {
        if (ia < Ns && (ib >= Ni || tc[ia] <= timp)) {
            t[k++] = tc[ia++];
        } else {
            t[k++] = timp;
            ++ib;
            timp = ib < Ni ? next_imp(ib) : INFINITY;
        }
    }
}

// rays given fixed sample positions: only the box test
__global__ void __launch_bounds__(128) k_valid(TrainArgs a) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.B) return;
    float o[3], w[3], tn, tf;
    load3(a.o + 3 * r, o);
    load3(a.w + 3 * r, w);
    a.valid[r] = clip_ray(a, o, w, tn, tf) ? 1 : 0;
}

// ------------------------------------------------------------------ volume rendering and loss
__device__ __forceinline__ void block_add(double v, double *dst) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0 && v != 0.0) atomicAdd(dst, v);
    }
}

__global__ void __launch_bounds__(128) k_composite_fwd(TrainArgs a, float *rgb_out) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double l1 = 0.0;
    if (r < a.B) {
        float C[3] = {0.f, 0.f, 0.f};
        if (a.valid[r]) {
            const int64_t q0 = r * a.S;
            float Tr = 1.f, ls = log_sigm(a.s * a.d_c[q0]);
            for (int i = 0; i + 1 < a.S; ++i) {
                const float ls1 = log_sigm(a.s * a.d_c[q0 + i + 1]);
                const float alpha = fmaxf(1.f - expf(ls1 - ls), 0.f);
                const float wgt = Tr * alpha;
                C[0] = fmaf(wgt, a.rgb_c[3 * (q0 + i)], C[0]);
                C[1] = fmaf(wgt, a.rgb_c[3 * (q0 + i) + 1], C[1]);
                C[2] = fmaf(wgt, a.rgb_c[3 * (q0 + i) + 2], C[2]);
                Tr *= 1.f - alpha;
                ls = ls1;
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            a.C[3 * r + c] = C[c];
            if (rgb_out) rgb_out[3 * r + c] = C[c];
            l1 += fabs((double)C[c] - (double)__ldg(a.target + 3 * r + c));
        }
    }
    block_add(l1, a.acc);
}

__global__ void __launch_bounds__(128) k_eik_fwd(TrainArgs a) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0;
    if (m < a.M) {
        float g[3], n[3];
        const float gn = fd_normal(a, a.B * a.S + m, g, n);
        e = (double)(gn - 1.f) * (double)(gn - 1.f);
    }
    block_add(e, a.acc + 1);
}

__global__ void k_finalize(TrainArgs a) {
    const double lc = a.B > 0 ? a.acc[0] / (double)a.B : 0.0;
    const double le = a.M > 0 ? a.acc[1] / (double)a.M : 0.0;
    a.loss[0] = (float)(lc + (double)a.lambda * le);
    a.loss[1] = (float)lc;
    a.loss[2] = (float)le;
}

// upstream of the sample centres' d and colour from dL/dC = sign(C - I) dloss / B
__global__ void __launch_bounds__(128) k_composite_bwd(TrainArgs a) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.B || !a.valid[r]) return;
    const float dl = a.dloss ? *a.dloss : 1.f;
    float gC[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float e = a.C[3 * r + c] - __ldg(a.target + 3 * r + c);
        gC[c] = (e > 0.f ? 1.f : (e < 0.f ? -1.f : 0.f)) * dl / (float)a.B;
    }
    const int64_t q0 = r * a.S;
    const int S = a.S;
    float Tl[MAXS];
    {
        float Tr = 1.f, ls = log_sigm(a.s * a.d_c[q0]);
        for (int i = 0; i + 1 < S; ++i) {
            const float ls1 = log_sigm(a.s * a.d_c[q0 + i + 1]);
            Tl[i] = Tr;
            Tr *= 1.f - fmaxf(1.f - expf(ls1 - ls), 0.f);
            ls = ls1;
        }
    }
    // back to front: Chat = colour rendered from sample i + 1 on with unit transmittance
    float Ch[3] = {0.f, 0.f, 0.f};
    float dd_next = 0.f;
    a.g_rgb[3 * (q0 + S - 1)] = a.g_rgb[3 * (q0 + S - 1) + 1] = a.g_rgb[3 * (q0 + S - 1) + 2] = 0.f;
    float d1 = a.d_c[q0 + S - 1];
    for (int i = S - 2; i >= 0; --i) {
        const float d0 = a.d_c[q0 + i];
        const float ls0 = log_sigm(a.s * d0), ls1 = log_sigm(a.s * d1);
        const float rho = expf(ls1 - ls0);
        const float alpha = fmaxf(1.f - rho, 0.f);
        const float c0 = a.rgb_c[3 * (q0 + i)], c1 = a.rgb_c[3 * (q0 + i) + 1], c2 = a.rgb_c[3 * (q0 + i) + 2];
        const float dalpha = Tl[i] * (gC[0] * (c0 - Ch[0]) + gC[1] * (c1 - Ch[1]) + gC[2] * (c2 - Ch[2]));
        float dd0 = 0.f;
        if (1.f - rho > 0.f) {
            dd0 = dalpha * a.s * rho * sigm(-a.s * d0);
            dd_next -= dalpha * a.s * rho * sigm(-a.s * d1);
        }
        a.g_dc[q0 + i + 1] = dd_next;
        dd_next = dd0;
        const float wgt = Tl[i] * alpha;
        a.g_rgb[3 * (q0 + i)] = wgt * gC[0];
        a.g_rgb[3 * (q0 + i) + 1] = wgt * gC[1];
        a.g_rgb[3 * (q0 + i) + 2] = wgt * gC[2];
        Ch[0] = alpha * c0 + (1.f - alpha) * Ch[0];
        Ch[1] = alpha * c1 + (1.f - alpha) * Ch[1];
        Ch[2] = alpha * c2 + (1.f - alpha) * Ch[2];
        d1 = d0;
    }
    a.g_dc[q0] = dd_next;
}

// upstream of the eikonal points' difference records
__global__ void __launch_bounds__(128) k_eik_bwd(TrainArgs a) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= a.M) return;
    const int64_t q = a.B * a.S + m;
    float g[3], n[3];
    const float gn = fd_normal(a, q, g, n);
    const float dl = a.dloss ? *a.dloss : 1.f;
    const float coef = gn > 0.f ? dl * a.lambda / (float)a.M * 2.f * (gn - 1.f) / gn / (2.f * a.h) : 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        a.g_fd[6 * q + 2 * k] = coef * g[k];
        a.g_fd[6 * q + 2 * k + 1] = -coef * g[k];
    }
}

}  // namespace

int train_chunk_records() { return CHUNK; }

cudaError_t train_sort(const TrainArgs &a, int which, int64_t n_rec, int sm_count, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(a.count, 0, sizeof(int) * (a.nkeys + 1), s);
    if (e != cudaSuccess) return e;
    const int blocks = grid_for(sm_count, 8, (n_rec + 255) / 256);
    if (which == TRAIN_COARSE) k_hist<TRAIN_COARSE><<<blocks, 256, 0, s>>>(a, n_rec);
    else k_hist<TRAIN_FINE><<<blocks, 256, 0, s>>>(a, n_rec);
    k_scan<<<1, 1024, 0, s>>>(a);
    if (which == TRAIN_COARSE) k_scatter<TRAIN_COARSE><<<blocks, 256, 0, s>>>(a, n_rec);
    else k_scatter<TRAIN_FINE><<<blocks, 256, 0, s>>>(a, n_rec);
    return cudaGetLastError();
}

cudaError_t train_importance(const TrainArgs &a, cudaStream_t s) {
    if (a.B == 0) return cudaSuccess;
    k_importance<<<(unsigned)((a.B + 127) / 128), 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t train_valid(const TrainArgs &a, cudaStream_t s) {
    if (a.B == 0) return cudaSuccess;
    k_valid<<<(unsigned)((a.B + 127) / 128), 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t train_loss_forward(const TrainArgs &a, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(a.acc, 0, 2 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    if (a.B > 0) k_composite_fwd<<<(unsigned)((a.B + 127) / 128), 128, 0, s>>>(a, nullptr);
    if (a.M > 0) k_eik_fwd<<<(unsigned)((a.M + 127) / 128), 128, 0, s>>>(a);
    k_finalize<<<1, 1, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t train_rgb_out(const TrainArgs &a, float *rgb, cudaStream_t s) {
    if (a.B > 0 && rgb) return cudaMemcpyAsync(rgb, a.C, sizeof(float) * 3 * a.B, cudaMemcpyDeviceToDevice, s);
    return cudaSuccess;
}

cudaError_t train_upstream(const TrainArgs &a, cudaStream_t s) {
    if (a.B > 0) k_composite_bwd<<<(unsigned)((a.B + 127) / 128), 128, 0, s>>>(a);
    if (a.M > 0) k_eik_bwd<<<(unsigned)((a.M + 127) / 128), 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace kns
