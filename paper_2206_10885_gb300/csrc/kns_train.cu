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
// How: every SDF evaluation is a record (a point and an id).  Records are counting-sorted by the
// cell that evaluates them, and cut into chunks of at most CHUNK records of one cell.  A block takes
// a chunk, stages the cell's weights in shared memory and gives each thread one record at a time:
// the forward pass runs in registers with weights read as warp-uniform float4 broadcasts.  In the
// backward kernels each thread also writes its record's layer inputs and output deltas as one
// column of a shared-memory tile (128 records), and the block then forms the weight gradient of
// the tile as outer-product sums: thread-owned 4x4 blocks of (output, input) entries accumulate in
// registers over every tile of the chunk and are added to the global gradient once per chunk.
// Bias gradients come out of the same sums through a constant-one input row.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kns_device.cuh"
#include "kns_kernels.h"

namespace kns {
namespace {

constexpr int PE_L = 4;                   // encoding frequencies of x
constexpr int A0ROWS = 28;                // 27 encoded inputs + the constant-one row
constexpr int TILE = 128;                 // records per tile = threads per block
constexpr int RS = TILE + 4;              // shared row stride (floats): 16-byte rows, shifted banks
constexpr int CHUNK = 4096;               // records per work chunk
constexpr int MAXS = 256;                 // samples per ray

// Shared-memory weight layout (rows padded to 4 floats) and the canonical layout, per cell.
template <int H>
struct TL {
    static constexpr int sW0 = 0, sb0 = 32 * 28, sH = sb0 + 32;
    static constexpr int HS = 32 * 32 + 32;  // one hidden layer (W, b)
    static constexpr int sWo = sH + (H - 1) * HS, sbo = sWo + 16 * 32, SDF = sbo + 16;
    static constexpr int sC0 = SDF, sc0 = sC0 + 32 * 36, sC1 = sc0 + 32, sc1 = sC1 + 4 * 32, ALL = sc1 + 4;
    static constexpr int cW0 = 0, cb0 = 32 * 27, cH = cb0 + 32;
    static constexpr int cWo = cH + (H - 1) * HS, cbo = cWo + 16 * 32, PSDF = cbo + 16;
    static constexpr int cC0 = PSDF, cc0 = cC0 + 32 * 33, cC1 = cc0 + 32, cc1 = cC1 + 3 * 32;
    // tile rows: A0 (28), A_l (36 each: 32 + one + 3 zero), D_l (32 each), Dout, then the colour rows
    static constexpr int rA0 = 0;
    __host__ __device__ static constexpr int rA(int l) { return A0ROWS + (l - 1) * 36; }  // l = 1..H
    __host__ __device__ static constexpr int rD(int l) { return A0ROWS + H * 36 + (l - 1) * 32; }
    static constexpr int rDout = A0ROWS + H * 36 + H * 32;
    static constexpr int ROWS_FD = rDout + 4;
    static constexpr int rU = rDout + 16, rHc = rU + 36, rDh = rHc + 36, rDc = rDh + 32;
    static constexpr int ROWS_C = rDc + 4;
};

// canonical index of shared weight slot j (-1: zero pad)
template <int H>
__device__ __forceinline__ int canon_of(int j) {
    using T = TL<H>;
    if (j < T::sb0) {
        const int o = j / 28, i = j - o * 28;
        return i < 27 ? o * 27 + i : -1;
    }
    if (j < T::sH) return T::cb0 + (j - T::sb0);
    if (j < T::SDF) return T::cH + (j - T::sH);  // hidden and output layers: same order, no padding
    j -= T::SDF;
    if (j < 32 * 36) {
        const int o = j / 36, i = j - o * 36;
        return i < 33 ? T::cC0 + o * 33 + i : -1;
    }
    j -= 32 * 36;
    if (j < 32) return T::cc0 + j;
    j -= 32;
    if (j < 128) {
        const int o = j >> 5, i = j & 31;
        return o < 3 ? T::cC1 + o * 32 + i : -1;
    }
    j -= 128;
    return j < 3 ? T::cc1 + j : -1;
}

template <int H>
__device__ __forceinline__ void load_weights(const float *__restrict__ cw, float *sw, int n) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int c = canon_of<H>(j);
        sw[j] = c >= 0 ? __ldg(cw + c) : 0.f;
    }
}

// ------------------------------------------------------------------ activations (accurate forms)
__device__ __forceinline__ float sp(float s, float beta, float inv_beta) {
    return fmaxf(s, 0.f) + log1pf(expf(-beta * fabsf(s))) * inv_beta;
}
// softplus_beta'(s) = sigmoid(beta s) = 1 - exp(-beta softplus_beta(s)), from the activation a
__device__ __forceinline__ float dsp_from_act(float a, float beta) { return -expm1f(-beta * a); }
__device__ __forceinline__ float sigm(float s) { return 1.f / (1.f + expf(-s)); }
// log sigmoid(x), stable for any x
__device__ __forceinline__ float log_sigm(float x) {
    return x < 0.f ? x - log1pf(expf(x)) : -log1pf(expf(-x));
}

// shared-memory float4 load kept in program order, so that unrolled layers do not hoist every
// weight load ahead of its use (which spills)
__device__ __forceinline__ float4 lds4(const float *p) {
    float4 v;
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}
// y = b + W x, W[OUT][RSTR] row-major in shared memory (RSTR % 4 == 0, IN <= RSTR, IN % 4 == 0)
template <int IN, int OUT, int RSTR>
__device__ __forceinline__ void lin(const float *W, const float *b, const float (&x)[IN], float (&y)[OUT]) {
#pragma unroll
    for (int o = 0; o < OUT; ++o) {
        float acc = b[o];
#pragma unroll
        for (int i = 0; i < IN; i += 4) {
            const float4 w4 = lds4(W + o * RSTR + i);
            acc = fmaf(w4.x, x[i], acc);
            acc = fmaf(w4.y, x[i + 1], acc);
            acc = fmaf(w4.z, x[i + 2], acc);
            acc = fmaf(w4.w, x[i + 3], acc);
        }
        y[o] = acc;
    }
}

// SDF forward: out = [d, z]; with STORE, the layer inputs go to column `col` of the tile rows.
template <int H, bool STORE>
__device__ __forceinline__ void sdf_forward(const float *sw, float px, float py, float pz, float beta,
                                            float inv_beta, float (&out)[16], float *rows, int col) {
    using T = TL<H>;
    float a0[28];
    encode3<PE_L, 28>(px, py, pz, a0);
    if (STORE) {
#pragma unroll
        for (int i = 0; i < 27; ++i) rows[(T::rA0 + i) * RS + col] = a0[i];
    }
    float h[32];
    lin<28, 32, 28>(sw + T::sW0, sw + T::sb0, a0, h);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        h[j] = sp(h[j], beta, inv_beta);
        if (STORE) rows[(T::rA(1) + j) * RS + col] = h[j];
    }
#pragma unroll
    for (int l = 1; l < H; ++l) {
        float hn[32];
        lin<32, 32, 32>(sw + T::sH + (l - 1) * T::HS, sw + T::sH + (l - 1) * T::HS + 1024, h, hn);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            h[j] = sp(hn[j], beta, inv_beta);
            if (STORE) rows[(T::rA(l + 1) + j) * RS + col] = h[j];
        }
    }
    lin<32, 16, 32>(sw + T::sWo, sw + T::sbo, h, out);
}

// SDF backward from the output deltas dout[0..NO) (rows written: Dout, D_H .. D_1).
template <int H, int NO>
__device__ __forceinline__ void sdf_backward(const float *sw, const float (&dout)[NO], float beta, float *rows,
                                             int col) {
    using T = TL<H>;
#pragma unroll
    for (int o = 0; o < NO; ++o) rows[(T::rDout + o) * RS + col] = dout[o];
    float dl[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) dl[j] = 0.f;
#pragma unroll
    for (int o = 0; o < NO; ++o) {
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
            const float4 w4 = lds4(sw + T::sWo + o * 32 + j);
            dl[j] = fmaf(w4.x, dout[o], dl[j]);
            dl[j + 1] = fmaf(w4.y, dout[o], dl[j + 1]);
            dl[j + 2] = fmaf(w4.z, dout[o], dl[j + 2]);
            dl[j + 3] = fmaf(w4.w, dout[o], dl[j + 3]);
        }
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        dl[j] *= dsp_from_act(rows[(T::rA(H) + j) * RS + col], beta);
        rows[(T::rD(H) + j) * RS + col] = dl[j];
    }
#pragma unroll
    for (int l = H - 1; l >= 1; --l) {
        const float *Wl = sw + T::sH + (l - 1) * T::HS;  // maps A_l -> pre-activation of layer l + 1
        float dn[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) dn[j] = 0.f;
#pragma unroll
        for (int o = 0; o < 32; ++o) {
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
                const float4 w4 = lds4(Wl + o * 32 + j);
                dn[j] = fmaf(w4.x, dl[o], dn[j]);
                dn[j + 1] = fmaf(w4.y, dl[o], dn[j + 1]);
                dn[j + 2] = fmaf(w4.z, dl[o], dn[j + 2]);
                dn[j + 3] = fmaf(w4.w, dl[o], dn[j + 3]);
            }
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            dl[j] = dn[j] * dsp_from_act(rows[(T::rA(l) + j) * RS + col], beta);
            rows[(T::rD(l) + j) * RS + col] = dl[j];
        }
    }
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
__device__ __forceinline__ void load3(const float *p, float *v) {
    v[0] = __ldg(p);
    v[1] = __ldg(p + 1);
    v[2] = __ldg(p + 2);
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

// chunk c of keys [k0, k1): its key (largest k with chunk_off[k] <= c) and record range
__device__ __forceinline__ int chunk_key(const int *chunk_off, int k0, int k1, int c) {
    int lo = k0, hi = k1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(chunk_off + mid) <= c) lo = mid;
        else hi = mid;
    }
    return lo;
}

// ------------------------------------------------------------------ forward: d at sorted records
// out[rec] = d(x_rec) for the records of keys [k0, k1) (key = cell)
template <int H>
__global__ void __launch_bounds__(TILE, 4) k_eval_d(TrainArgs a, int k0, int k1, float *out) {
    extern __shared__ float4 smem4[];
    float *sw = reinterpret_cast<float *>(smem4);
    const int c0 = a.chunk_off[k0], total = a.chunk_off[k1] - c0;
    for (int ci = blockIdx.x; ci < total; ci += gridDim.x) {
        const int key = chunk_key(a.chunk_off, k0, k1, c0 + ci);
        const int j = c0 + ci - a.chunk_off[key];
        const int beg = a.off[key] + j * CHUNK, end = min(beg + CHUNK, a.off[key + 1]);
        __syncthreads();
        load_weights<H>(a.params + (int64_t)key * a.p_cell, sw, TL<H>::SDF);
        __syncthreads();
        for (int i = beg + (int)threadIdx.x; i < end; i += TILE) {
            const float4 r = a.sorted[i];
            float y[16];
            sdf_forward<H, false>(sw, r.x, r.y, r.z, a.beta, a.inv_beta, y, nullptr, 0);
            out[__float_as_int(r.w)] = y[0];
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

// ------------------------------------------------------------------ sample centres: SDF, normal, colour
// normal from the six difference records of centre q; returns |g| (n = 0 when |g| = 0)
__device__ __forceinline__ float fd_normal(const TrainArgs &a, int64_t q, float (&g)[3], float (&n)[3]) {
    const float inv2h = 1.f / (2.f * a.h);
    const float *d = a.d_fd + 6 * q;
#pragma unroll
    for (int k = 0; k < 3; ++k) g[k] = (d[2 * k] - d[2 * k + 1]) * inv2h;
    const float gn = sqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    const float ig = gn > 0.f ? 1.f / gn : 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) n[k] = g[k] * ig;
    return gn;
}

// colour input u = [z (15), n (3), gamma_2(v) (15), 0 0 0]
__device__ __forceinline__ void colour_input(const float (&y)[16], const float (&n)[3], const float *v,
                                             float (&u)[36]) {
#pragma unroll
    for (int k = 0; k < 15; ++k) u[k] = y[1 + k];
    u[15] = n[0];
    u[16] = n[1];
    u[17] = n[2];
    float e[16];
    encode3<2, 16>(v[0], v[1], v[2], e);
#pragma unroll
    for (int k = 0; k < 15; ++k) u[18 + k] = e[k];
    u[33] = u[34] = u[35] = 0.f;
}

template <int H>
__global__ void __launch_bounds__(TILE, 4) k_centre_fwd(TrainArgs a) {
    using T = TL<H>;
    extern __shared__ float4 smem4[];
    float *sw = reinterpret_cast<float *>(smem4);
    const int k0 = a.NC, k1 = 2 * a.NC;
    const int64_t nfd = 6 * (a.B * a.S + a.M);
    const int c0 = a.chunk_off[k0], total = a.chunk_off[k1] - c0;
    for (int ci = blockIdx.x; ci < total; ci += gridDim.x) {
        const int key = chunk_key(a.chunk_off, k0, k1, c0 + ci);
        const int j = c0 + ci - a.chunk_off[key];
        const int beg = a.off[key] + j * CHUNK, end = min(beg + CHUNK, a.off[key + 1]);
        __syncthreads();
        load_weights<H>(a.params + (int64_t)(key - a.NC) * a.p_cell, sw, T::ALL);
        __syncthreads();
        for (int i = beg + (int)threadIdx.x; i < end; i += TILE) {
            const float4 rr = a.sorted[i];
            const int64_t q = (int64_t)__float_as_int(rr.w) - nfd;
            const int64_t r = q / a.S;
            float y[16], g[3], n[3], v[3], u[36], hid[32], lg[4];
            sdf_forward<H, false>(sw, rr.x, rr.y, rr.z, a.beta, a.inv_beta, y, nullptr, 0);
            fd_normal(a, q, g, n);
            load3(a.w + 3 * r, v);
            colour_input(y, n, v, u);
            lin<36, 32, 36>(sw + T::sC0, sw + T::sc0, u, hid);
#pragma unroll
            for (int k = 0; k < 32; ++k) hid[k] = fmaxf(hid[k], 0.f);
            lin<32, 4, 32>(sw + T::sC1, sw + T::sc1, hid, lg);
            a.d_c[q] = y[0];
            a.rgb_c[3 * q] = sigm(lg[0]);
            a.rgb_c[3 * q + 1] = sigm(lg[1]);
            a.rgb_c[3 * q + 2] = sigm(lg[2]);
        }
    }
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

// ------------------------------------------------------------------ backward: weight gradients
// One (output rows) x (input rows) layer of the tile GEMM: thread blocks of 4 x 4 entries with rows
// ob + OB jo and ib + IB ji.
struct GemmLayer {
    int drow, OB, arow, IB, out_real, in_real, cW, cb;
};

template <int H, bool CENTRE>
struct GemmPlan {
    static constexpr int NL = H + 1 + (CENTRE ? 2 : 0);
    __device__ static GemmLayer layer(int l) {
        using T = TL<H>;
        if (l == 0) return {T::rD(1), 8, T::rA0, 7, 32, 27, T::cW0, T::cb0};
        if (l < H) return {T::rD(l + 1), 8, T::rA(l), 9, 32, 32, T::cH + (l - 1) * T::HS, T::cH + (l - 1) * T::HS + 1024};
        if (l == H) return {T::rDout, CENTRE ? 4 : 1, T::rA(H), 9, CENTRE ? 16 : 1, 32, T::cWo, T::cbo};
        if (l == H + 1) return {T::rDh, 8, T::rU, 9, 32, 33, T::cC0, T::cc0};
        return {T::rDc, 1, T::rHc, 9, 3, 32, T::cC1, T::cc1};
    }
    __host__ __device__ static constexpr int blocks() {
        return 56 + 72 * (H - 1) + (CENTRE ? 36 + 72 + 9 : 9);
    }
    static constexpr int NB = (blocks() + TILE - 1) / TILE;
};

struct Blk {
    int drow, OB, arow, IB, out_real, in_real, cW, cb, ob, ib;
};

template <class Plan>
__device__ __forceinline__ Blk block_of(int b) {
    Blk k{};
    k.drow = -1;
    if (b >= Plan::blocks()) return k;
#pragma unroll 1
    for (int l = 0; l < Plan::NL; ++l) {
        const GemmLayer L = Plan::layer(l);
        const int n = L.OB * L.IB;
        if (b < n) {
            k.drow = L.drow;
            k.OB = L.OB;
            k.arow = L.arow;
            k.IB = L.IB;
            k.out_real = L.out_real;
            k.in_real = L.in_real;
            k.cW = L.cW;
            k.cb = L.cb;
            k.ob = b / L.IB;
            k.ib = b - k.ob * L.IB;
            return k;
        }
        b -= n;
    }
    return k;
}

template <class Plan>
__device__ __forceinline__ void gemm_tile(const float *rows, int b, float (&acc)[16]) {
    const Blk k = block_of<Plan>(b);
    if (k.drow < 0) return;
    const float *D = rows + (k.drow + k.ob) * RS;
    const float *A = rows + (k.arow + k.ib) * RS;
    const int sd = k.OB * RS, sa = k.IB * RS;
#pragma unroll 2
    for (int r = 0; r < TILE; r += 4) {
        float4 dv[4], av[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            dv[q] = *reinterpret_cast<const float4 *>(D + q * sd + r);
            av[q] = *reinterpret_cast<const float4 *>(A + q * sa + r);
        }
#pragma unroll
        for (int jo = 0; jo < 4; ++jo)
#pragma unroll
            for (int ji = 0; ji < 4; ++ji) {
                float s = acc[jo * 4 + ji];
                s = fmaf(dv[jo].x, av[ji].x, s);
                s = fmaf(dv[jo].y, av[ji].y, s);
                s = fmaf(dv[jo].z, av[ji].z, s);
                s = fmaf(dv[jo].w, av[ji].w, s);
                acc[jo * 4 + ji] = s;
            }
    }
}

template <class Plan>
__device__ __forceinline__ void flush_block(float *gcell, int b, float (&acc)[16]) {
    const Blk k = block_of<Plan>(b);
    if (k.drow < 0) return;
#pragma unroll
    for (int jo = 0; jo < 4; ++jo)
#pragma unroll
        for (int ji = 0; ji < 4; ++ji) {
            const int o = k.ob + k.OB * jo, i = k.ib + k.IB * ji;
            const float v = acc[jo * 4 + ji];
            acc[jo * 4 + ji] = 0.f;
            if (v == 0.f || o >= k.out_real || i > k.in_real) continue;
            atomicAdd(gcell + (i < k.in_real ? k.cW + o * k.in_real + i : k.cb + o), v);
        }
}

// CENTRE: sample-centre records (colour MLP + SDF with upstream on d and z; writes the difference
// records' upstream).  Otherwise: difference records (SDF with upstream on d only).
template <int H, bool CENTRE>
__global__ void __launch_bounds__(TILE, 1) k_backward(TrainArgs a) {
    using T = TL<H>;
    using Plan = GemmPlan<H, CENTRE>;
    constexpr int NROWS = CENTRE ? T::ROWS_C : T::ROWS_FD;
    constexpr int NW = CENTRE ? T::ALL : T::SDF;
    extern __shared__ float4 smem4[];
    float *rows = reinterpret_cast<float *>(smem4);
    float *sw = rows + NROWS * RS;
    const int tid = threadIdx.x;
    // zero every row once (stale columns of later partial tiles stay finite), then the one-rows
    for (int i = tid; i < NROWS * RS; i += TILE) rows[i] = 0.f;
    __syncthreads();
    for (int c = tid; c < RS; c += TILE) {
        rows[(T::rA0 + 27) * RS + c] = 1.f;
        for (int l = 1; l <= H; ++l) rows[(T::rA(l) + 32) * RS + c] = 1.f;
        if (CENTRE) {
            rows[(T::rU + 33) * RS + c] = 1.f;
            rows[(T::rHc + 32) * RS + c] = 1.f;
        }
    }
    float acc[Plan::NB][16];
#pragma unroll
    for (int k = 0; k < Plan::NB; ++k)
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[k][e] = 0.f;
    const int k0 = CENTRE ? a.NC : 0, k1 = CENTRE ? 2 * a.NC : a.NC;
    const int64_t nfd = 6 * (a.B * a.S + a.M);
    const int c0 = a.chunk_off[k0], total = a.chunk_off[k1] - c0;
    const float inv2h = 1.f / (2.f * a.h);
    for (int ci = blockIdx.x; ci < total; ci += gridDim.x) {
        const int key = chunk_key(a.chunk_off, k0, k1, c0 + ci);
        const int cell = key - k0;
        const int j = c0 + ci - a.chunk_off[key];
        const int beg = a.off[key] + j * CHUNK, end = min(beg + CHUNK, a.off[key + 1]);
        __syncthreads();
        load_weights<H>(a.params + (int64_t)cell * a.p_cell, sw, NW);
        __syncthreads();
        for (int tb = beg; tb < end; tb += TILE) {
            const int i = tb + tid;
            if (i < end) {
                const float4 rr = a.sorted[i];
                const int64_t rec = (int64_t)__float_as_int(rr.w);
                float y[16];
                sdf_forward<H, true>(sw, rr.x, rr.y, rr.z, a.beta, a.inv_beta, y, rows, tid);
                if (CENTRE) {
                    const int64_t q = rec - nfd, r = q / a.S;
                    float g[3], n[3], v[3], u[36], hid[32], lg[4];
                    const float gn = fd_normal(a, q, g, n);
                    load3(a.w + 3 * r, v);
                    colour_input(y, n, v, u);
#pragma unroll
                    for (int k = 0; k < 33; ++k) rows[(T::rU + k) * RS + tid] = u[k];
                    lin<36, 32, 36>(sw + T::sC0, sw + T::sc0, u, hid);
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        hid[k] = fmaxf(hid[k], 0.f);
                        rows[(T::rHc + k) * RS + tid] = hid[k];
                    }
                    lin<32, 4, 32>(sw + T::sC1, sw + T::sc1, hid, lg);
                    // colour backward: logits, hidden (ReLU), inputs z and n
                    float dc[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float rgb = sigm(lg[c]);
                        dc[c] = a.g_rgb[3 * q + c] * rgb * (1.f - rgb);
                        rows[(T::rDc + c) * RS + tid] = dc[c];
                    }
                    float dh[32];
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        float s = sw[T::sC1 + k] * dc[0];
                        s = fmaf(sw[T::sC1 + 32 + k], dc[1], s);
                        s = fmaf(sw[T::sC1 + 64 + k], dc[2], s);
                        dh[k] = hid[k] > 0.f ? s : 0.f;
                        rows[(T::rDh + k) * RS + tid] = dh[k];
                    }
                    float gu[20];
#pragma unroll
                    for (int k = 0; k < 20; ++k) gu[k] = 0.f;
#pragma unroll
                    for (int o = 0; o < 32; ++o) {
#pragma unroll
                        for (int k = 0; k < 20; k += 4) {
                            const float4 w4 = lds4(sw + T::sC0 + o * 36 + k);
                            gu[k] = fmaf(w4.x, dh[o], gu[k]);
                            gu[k + 1] = fmaf(w4.y, dh[o], gu[k + 1]);
                            gu[k + 2] = fmaf(w4.z, dh[o], gu[k + 2]);
                            gu[k + 3] = fmaf(w4.w, dh[o], gu[k + 3]);
                        }
                    }
                    // normal n = g / |g|: dL/dg = (dL/dn - n (n . dL/dn)) / |g|; g_k = (d+ - d-) / 2h
                    const float nd = n[0] * gu[15] + n[1] * gu[16] + n[2] * gu[17];
                    const float ig = gn > 0.f ? 1.f / gn : 0.f;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const float dg = (gu[15 + k] - n[k] * nd) * ig * inv2h;
                        a.g_fd[6 * q + 2 * k] = dg;
                        a.g_fd[6 * q + 2 * k + 1] = -dg;
                    }
                    float dout[16];
                    dout[0] = a.g_dc[q];
#pragma unroll
                    for (int k = 0; k < 15; ++k) dout[1 + k] = gu[k];
                    sdf_backward<H, 16>(sw, dout, a.beta, rows, tid);
                } else {
                    const float dout[1] = {a.g_fd[rec]};
                    sdf_backward<H, 1>(sw, dout, a.beta, rows, tid);
                }
            } else {
                // no record: zero deltas
                for (int l = 1; l <= H; ++l)
                    for (int k = 0; k < 32; ++k) rows[(T::rD(l) + k) * RS + tid] = 0.f;
                for (int k = 0; k < (CENTRE ? 16 : 1); ++k) rows[(T::rDout + k) * RS + tid] = 0.f;
                if (CENTRE) {
                    for (int k = 0; k < 32; ++k) rows[(T::rDh + k) * RS + tid] = 0.f;
                    for (int k = 0; k < 3; ++k) rows[(T::rDc + k) * RS + tid] = 0.f;
                }
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < Plan::NB; ++k) gemm_tile<Plan>(rows, tid + k * TILE, acc[k]);
            __syncthreads();
        }
        float *gcell = a.grad + (int64_t)cell * a.p_cell;
#pragma unroll
        for (int k = 0; k < Plan::NB; ++k) flush_block<Plan>(gcell, tid + k * TILE, acc[k]);
    }
}

template <int H>
size_t backward_smem(bool centre) {
    using T = TL<H>;
    return ((size_t)(centre ? T::ROWS_C : T::ROWS_FD) * RS + (centre ? T::ALL : T::SDF)) * sizeof(float);
}

int grid_for(int sm_count, int per_sm, int64_t work_upper) {
    int64_t b = (int64_t)sm_count * per_sm;
    if (work_upper < b) b = work_upper;
    return (int)(b > 0 ? b : 1);
}

template <int H>
cudaError_t eval_d_h(const TrainArgs &a, int k0, int k1, float *out, int blocks, cudaStream_t s) {
    const size_t sm = TL<H>::SDF * sizeof(float);
    k_eval_d<H><<<blocks, TILE, sm, s>>>(a, k0, k1, out);
    return cudaGetLastError();
}

template <int H>
cudaError_t centre_fwd_h(const TrainArgs &a, int blocks, cudaStream_t s) {
    const size_t sm = TL<H>::ALL * sizeof(float);
    k_centre_fwd<H><<<blocks, TILE, sm, s>>>(a);
    return cudaGetLastError();
}

template <int H, bool CENTRE>
cudaError_t backward_h(const TrainArgs &a, int blocks, cudaStream_t s) {
    const size_t sm = backward_smem<H>(CENTRE);
    cudaError_t e = cudaFuncSetAttribute(k_backward<H, CENTRE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_backward<H, CENTRE><<<blocks, TILE, sm, s>>>(a);
    return cudaGetLastError();
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

cudaError_t train_coarse_eval(const TrainArgs &a, int sm_count, cudaStream_t s) {
    const int64_t chunks = a.B * a.Ns / CHUNK + a.NC + 1;
    const int blocks = grid_for(sm_count, 4, chunks);
    return a.H == 3 ? eval_d_h<3>(a, 0, a.NC, a.d_coarse, blocks, s) : eval_d_h<2>(a, 0, a.NC, a.d_coarse, blocks, s);
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

cudaError_t train_fd_forward(const TrainArgs &a, int sm_count, cudaStream_t s) {
    const int64_t fd_chunks = 6 * (a.B * a.S + a.M) / CHUNK + a.NC + 1;
    return a.H == 3 ? eval_d_h<3>(a, 0, a.NC, a.d_fd, grid_for(sm_count, 4, fd_chunks), s)
                    : eval_d_h<2>(a, 0, a.NC, a.d_fd, grid_for(sm_count, 4, fd_chunks), s);
}

cudaError_t train_centre_forward(const TrainArgs &a, int sm_count, cudaStream_t s) {
    const int64_t c_chunks = a.B * a.S / CHUNK + a.NC + 1;
    const int blocks = grid_for(sm_count, 4, c_chunks);
    return a.H == 3 ? centre_fwd_h<3>(a, blocks, s) : centre_fwd_h<2>(a, blocks, s);
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

cudaError_t train_centre_backward(const TrainArgs &a, int sm_count, cudaStream_t s) {
    const int64_t c_chunks = a.B * a.S / CHUNK + a.NC + 1;
    return a.H == 3 ? backward_h<3, true>(a, grid_for(sm_count, 1, c_chunks), s)
                    : backward_h<2, true>(a, grid_for(sm_count, 1, c_chunks), s);
}

cudaError_t train_fd_backward(const TrainArgs &a, int sm_count, cudaStream_t s) {
    const int64_t fd_chunks = 6 * (a.B * a.S + a.M) / CHUNK + a.NC + 1;
    return a.H == 3 ? backward_h<3, false>(a, grid_for(sm_count, 1, fd_chunks), s)
                    : backward_h<2, false>(a, grid_for(sm_count, 1, fd_chunks), s);
}

}  // namespace kns
