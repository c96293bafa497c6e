// kns_train_tile.cu -- the grouped MLP kernels of the training step: SDF and colour MLPs of one cell
// evaluated, and differentiated, on tiles of 128 same-cell records as register-blocked block GEMMs.
//
// A block of 256 threads takes a chunk (up to 4096 records of one cell, from the counting sort),
// stages the cell's weights in shared memory (forward layers k-major, backward layers row-major) and
// walks the chunk in tiles of 128 records.  Activations and deltas of a tile live in shared memory
// as rows of 128 records (row stride 132 floats).  Every dense layer, forward (A_l = act(W A_{l-1} +
// b)) and backward (D_l = (W^T D_{l+1}) . act'(A_l)), is a [32 x K] by [K x 128] product in which a
// thread owns 4 outputs x 4 records: per k one warp-uniform float4 of weights and one float4 of
// activations feed 16 FMAs.  The weight gradient of the tile, dW_l = D_l A_{l-1}^T summed over the
// tile's records, is formed by thread-owned 4 x 4 blocks of (output, input) entries that accumulate
// in registers over every tile of the chunk and are added to the global gradient once per chunk;
// bias gradients come out of the same sums through a constant-one input row.
//
// Kernels: d at records (coarse samples and difference points); sample centres forward (d, z,
// colour); sample centres backward (colour and SDF, writes the difference points' upstream);
// difference points backward.  Model: Sec. 3.1 (Eq. 1-3) with the training loss of Sec. 3.2.2.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kns_device.cuh"
#include "kns_kernels.h"
#include "kns_train.cuh"

namespace kns {
namespace {

using train::CHUNK;
using train::chunk_key;
using train::fd_normal;
using train::grid_for;
using train::load3;

constexpr int TPB = 256;     // threads per block
constexpr int TILE = 128;    // records per tile
constexpr int RS = TILE + 4;  // shared row stride (floats)
constexpr int PE_L = 4;

// ------------------------------------------------------------------ shared weight layout
// [forward SDF | forward colour | backward SDF | backward colour], every block 16-byte aligned:
//   forward SDF:  T0[28][32] (T0[k][o] = W0[o][k], row 27 zero), b0[32]; per hidden layer l = 1..H-1
//                 Tl[32][32], bl[32]; To[32][16] (To[k][o] = Wo[o][k]), bo[16]
//   forward colour: C0t[36][32] (k < 33), c0[32], C1t[32][4] (c < 3), c1[4]
//   backward SDF: W_l[32][32] row-major (l = 1..H-1), Wo[16][32]
//   backward colour: Wc0[32][36] row-major (i < 33), Wc1[4][32] (row 3 zero)
template <int H>
struct WL {
    static constexpr int T0 = 0, b0 = 28 * 32, HL = 32 * 32 + 32;
    __host__ __device__ static constexpr int Tl(int l) { return b0 + 32 + (l - 1) * HL; }
    __host__ __device__ static constexpr int bl(int l) { return Tl(l) + 1024; }
    static constexpr int To = b0 + 32 + (H - 1) * HL, bo = To + 512, FS = bo + 16;
    static constexpr int C0t = FS, c0 = C0t + 36 * 32, C1t = c0 + 32, c1 = C1t + 128, FC = c1 + 4;
    __host__ __device__ static constexpr int Wr(int l) { return FC + (l - 1) * 1024; }
    static constexpr int Wo = FC + (H - 1) * 1024, BS = Wo + 512;
    static constexpr int Wc0 = BS, Wc1 = Wc0 + 32 * 36, END = Wc1 + 128;
    // canonical offsets (per cell)
    static constexpr int cW0 = 0, cb0 = 27 * 32, cH = cb0 + 32;
    static constexpr int cWo = cH + (H - 1) * HL, cbo = cWo + 512, cC0 = cbo + 16;
    static constexpr int cc0 = cC0 + 33 * 32, cC1 = cc0 + 32, cc1 = cC1 + 96;
};

// canonical index of shared weight slot j (-1: zero)
template <int H>
__device__ int canon_slot(int j) {
    using L = WL<H>;
    if (j < L::b0) {  // T0[k][o]
        const int k = j >> 5, o = j & 31;
        return k < 27 ? L::cW0 + o * 27 + k : -1;
    }
    if (j < L::To) {
        if (j < L::Tl(1)) return L::cb0 + (j - L::b0);
        const int r = j - L::Tl(1), l = r / L::HL, u = r - l * L::HL;
        if (u < 1024) return L::cH + l * L::HL + (u & 31) * 32 + (u >> 5);  // Tl[k][o] = W[o][k]
        return L::cH + l * L::HL + u;                                        // bias
    }
    if (j < L::bo) {
        const int u = j - L::To, k = u >> 4, o = u & 15;
        return L::cWo + o * 32 + k;
    }
    if (j < L::FS) return L::cbo + (j - L::bo);
    if (j < L::c0) {
        const int u = j - L::C0t, k = u >> 5, o = u & 31;
        return k < 33 ? L::cC0 + o * 33 + k : -1;
    }
    if (j < L::C1t) return L::cc0 + (j - L::c0);
    if (j < L::c1) {
        const int u = j - L::C1t, k = u >> 2, c = u & 3;
        return c < 3 ? L::cC1 + c * 32 + k : -1;
    }
    if (j < L::FC) return j - L::c1 < 3 ? L::cc1 + (j - L::c1) : -1;
    if (j < L::Wo) {
        const int r = j - L::FC, l = r >> 10, u = r & 1023;
        return L::cH + l * L::HL + u;  // row-major as stored
    }
    if (j < L::BS) return L::cWo + (j - L::Wo);
    if (j < L::Wc1) {
        const int u = j - L::Wc0, o = u / 36, i = u - o * 36;
        return i < 33 ? L::cC0 + o * 33 + i : -1;
    }
    const int u = j - L::Wc1, c = u >> 5, k = u & 31;
    return c < 3 ? L::cC1 + c * 32 + k : -1;
}

template <int H>
__device__ __forceinline__ void load_slots(const float *__restrict__ cw, float *sw, int j0, int j1) {
    for (int j = j0 + (int)threadIdx.x; j < j1; j += TPB) {
        const int c = canon_slot<H>(j);
        sw[j] = c >= 0 ? __ldg(cw + c) : 0.f;
    }
}

// ------------------------------------------------------------------ tile rows
// A0 (28: encoding + one), A_l (36: 32 + one + 3 zero), D_l (32), Dout (16: d and z deltas),
// then the colour rows: the d output row, U (36: z, n, gamma(v), one, 2 zero), Hc (36), Dh (32), Dc (4)
template <int H>
struct RL {
    static constexpr int A0 = 0;
    __host__ __device__ static constexpr int A(int l) { return 28 + (l - 1) * 36; }
    __host__ __device__ static constexpr int D(int l) { return 28 + 36 * H + (l - 1) * 32; }
    static constexpr int Dout = 28 + 68 * H;
    // difference records backward in place: D_l over A_l (rows 0..31; the one row stays), then Dout
    static constexpr int DoutF = 28 + 36 * H, FDI_ROWS = DoutF + 4;
    static constexpr int Ud = Dout + 16, U = Ud + 1, Hc = U + 36, Dh = Hc + 36, Dc = Dh + 32;
    static constexpr int C_ROWS = Dc + 4;
    // forward-only kernels: A0, two ping-pong layers, then (centres) the output row, U and Hc
    static constexpr int P = 28, Q = P + 32, F_ROWS = Q + 32;
    static constexpr int FUd = Q + 32, FU = FUd + 1, FHc = FU + 36, FC_ROWS = FHc + 32;
};

// ------------------------------------------------------------------ activations
__device__ __forceinline__ float softplus(float s, float beta, float inv_beta) {
    return fmaxf(s, 0.f) + __logf(1.f + __expf(-beta * fabsf(s))) * inv_beta;
}
// softplus_beta'(s) = sigmoid(beta s) = 1 - exp(-beta a) with a = softplus_beta(s) (series for small a)
__device__ __forceinline__ float dsoftplus_act(float a, float beta) {
    const float x = beta * a;
    return x < 1e-2f ? x * (1.f - x * (0.5f - x * (1.f / 6.f))) : 1.f - __expf(-x);
}
__device__ __forceinline__ float sigm(float s) { return 1.f / (1.f + __expf(-s)); }

// ------------------------------------------------------------------ block GEMMs
// thread blocking: outputs o0 .. o0+3 (o0 = 4 warp), records r0 .. r0+3 (r0 = 4 lane)
__device__ __forceinline__ int o0_32() { return (threadIdx.x >> 5) * 4; }
__device__ __forceinline__ int r0_t() { return (threadIdx.x & 31) * 4; }

// acc[i][j] += sum_k Wk[k WS + o0 + i] X[k RS + r0 + j]
template <int K, int WS>
__device__ __forceinline__ void mm32(const float *Wk, const float *X, float (&acc)[4][4]) {
    const float *w = Wk + o0_32();
    const float *x = X + r0_t();
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
        const float4 wv = *reinterpret_cast<const float4 *>(w + k * WS);
        const float4 xv = *reinterpret_cast<const float4 *>(x + k * RS);
        const float wa[4] = {wv.x, wv.y, wv.z, wv.w}, xa[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(wa[i], xa[j], acc[i][j]);
    }
}

// 16 outputs: o0 = 2 warp, outputs o0, o0+1; acc[i][j] += sum_k Wk[k 16 + o0 + i] X[k RS + r0 + j]
template <int K>
__device__ __forceinline__ void mm16(const float *Wk, const float *X, float (&acc)[2][4]) {
    const float *w = Wk + (threadIdx.x >> 5) * 2;
    const float *x = X + r0_t();
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
        const float2 wv = *reinterpret_cast<const float2 *>(w + k * 16);
        const float4 xv = *reinterpret_cast<const float4 *>(x + k * RS);
        const float xa[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            acc[0][j] = fmaf(wv.x, xa[j], acc[0][j]);
            acc[1][j] = fmaf(wv.y, xa[j], acc[1][j]);
        }
    }
}

__device__ __forceinline__ void init_bias(const float *b, float (&acc)[4][4]) {
    const float4 bv = *reinterpret_cast<const float4 *>(b + o0_32());
    const float ba[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = ba[i];
}
__device__ __forceinline__ void zero(float (&acc)[4][4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
}
__device__ __forceinline__ void store_rows(float *rows, int row0, const float (&v)[4][4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
        *reinterpret_cast<float4 *>(rows + (row0 + o0_32() + i) * RS + r0_t()) =
            make_float4(v[i][0], v[i][1], v[i][2], v[i][3]);
}
__device__ __forceinline__ void load_rows(const float *rows, int row0, float (&v)[4][4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float4 x = *reinterpret_cast<const float4 *>(rows + (row0 + o0_32() + i) * RS + r0_t());
        v[i][0] = x.x;
        v[i][1] = x.y;
        v[i][2] = x.z;
        v[i][3] = x.w;
    }
}

// one SDF hidden layer: rows[dst] = softplus(W rows[src] + b)
template <int K>
__device__ __forceinline__ void hidden_layer(const float *Wk, const float *b, float *rows, int src, int dst,
                                             float beta, float inv_beta) {
    float acc[4][4];
    init_bias(b, acc);
    mm32<K, 32>(Wk, rows + src * RS, acc);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = softplus(acc[i][j], beta, inv_beta);
    store_rows(rows, dst, acc);
}

// encoding of record column col into rows A0 .. A0+26, split between two threads: half 0 writes x
// and frequencies 0, 1; half 1 frequencies 2, 3 (rows 3 + 6k + c: sin, 3 + 6k + 3 + c: cos)
__device__ __forceinline__ void encode_half(float *rows, int a0, int col, int half, float x, float y, float z) {
    const float p[3] = {x, y, z};
    if (half == 0) {
        rows[(a0 + 0) * RS + col] = x;
        rows[(a0 + 1) * RS + col] = y;
        rows[(a0 + 2) * RS + col] = z;
    }
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
        const int k = 2 * half + kk;
        const float f = (float)(1 << k);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float sn, cs;
            sincospif(f * p[c], &sn, &cs);
            rows[(a0 + 3 + 6 * k + c) * RS + col] = sn;
            rows[(a0 + 6 + 6 * k + c) * RS + col] = cs;
        }
    }
}

// ------------------------------------------------------------------ forward: d at records
template <int H>
__global__ void __launch_bounds__(TPB, 3) k_tile_eval_d(TrainArgs a, int k0, int k1, float *out) {
    using L = WL<H>;
    using R = RL<H>;
    extern __shared__ float4 smem4[];
    float *rows = reinterpret_cast<float *>(smem4);
    float *sw = rows + R::F_ROWS * RS;
    __shared__ int s_rec[TILE];
    const int tid = threadIdx.x;
    const int c0 = a.chunk_off[k0], total = a.chunk_off[k1] - c0;
    constexpr int last = (H % 2 == 1) ? R::P : R::Q;  // A0 -> P -> Q -> P ...
    for (int ci = blockIdx.x; ci < total; ci += gridDim.x) {
        const int key = chunk_key(a.chunk_off, k0, k1, c0 + ci);
        const int j = c0 + ci - a.chunk_off[key];
        const int beg = a.off[key] + j * CHUNK, end = min(beg + CHUNK, a.off[key + 1]);
        __syncthreads();
        load_slots<H>(a.params + (int64_t)key * a.p_cell, sw, 0, L::FS);
        for (int tb = beg; tb < end; tb += TILE) {
            {
                const int col = tid & (TILE - 1), i = tb + col;
                float4 r = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
                if (i < end) r = a.sorted[i];
                if (tid < TILE) s_rec[tid] = __float_as_int(r.w);
                encode_half(rows, R::A0, col, tid >> 7, r.x, r.y, r.z);
            }
            __syncthreads();
            hidden_layer<27>(sw + L::T0, sw + L::b0, rows, R::A0, R::P, a.beta, a.inv_beta);
#pragma unroll
            for (int l = 1; l < H; ++l) {
                __syncthreads();
                hidden_layer<32>(sw + L::Tl(l), sw + L::bl(l), rows, (l % 2) ? R::P : R::Q, (l % 2) ? R::Q : R::P,
                                 a.beta, a.inv_beta);
            }
            __syncthreads();
            if (tid < TILE && s_rec[tid] >= 0) {
                float d = sw[L::bo];
#pragma unroll 8
                for (int k = 0; k < 32; ++k) d = fmaf(sw[L::To + k * 16], rows[(last + k) * RS + tid], d);
                out[s_rec[tid]] = d;
            }
        }
    }
}

// ------------------------------------------------------------------ sample centres
// colour input rows U: z (0..14), n (15..17), gamma_2(v) (18..32), one (33), zero (34, 35)
__device__ __forceinline__ void centre_inputs(const TrainArgs &a, float *rows, int u, int col, int64_t q) {
    const int64_t r = q / a.S;
    float g[3], n[3], v[3];
    fd_normal(a, q, g, n);
    load3(a.w + 3 * r, v);
    rows[(u + 15) * RS + col] = n[0];
    rows[(u + 16) * RS + col] = n[1];
    rows[(u + 17) * RS + col] = n[2];
    float e[16];
    encode3<2, 16>(v[0], v[1], v[2], e);
#pragma unroll
    for (int k = 0; k < 15; ++k) rows[(u + 18 + k) * RS + col] = e[k];
}

// SDF output layer (16 rows: d, z) of the tile into rows[dst .. dst+15]
__device__ __forceinline__ void output_layer(const float *To, const float *bo, float *rows, int src, int dst) {
    float acc[2][4];
    const int o0 = (threadIdx.x >> 5) * 2;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        acc[0][j] = bo[o0];
        acc[1][j] = bo[o0 + 1];
    }
    mm16<32>(To, rows + src * RS, acc);
#pragma unroll
    for (int i = 0; i < 2; ++i)
        *reinterpret_cast<float4 *>(rows + (dst + o0 + i) * RS + r0_t()) =
            make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
}

// colour hidden layer: rows[dst] = relu(C0 rows[u] + c0)
template <int H>
__device__ __forceinline__ void colour_hidden(const float *sw, float *rows, int u, int dst) {
    using L = WL<H>;
    float acc[4][4];
    init_bias(sw + L::c0, acc);
    mm32<33, 32>(sw + L::C0t, rows + u * RS, acc);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaxf(acc[i][j], 0.f);
    store_rows(rows, dst, acc);
}

// colour logits of record column col from the hidden rows
template <int H>
__device__ __forceinline__ void colour_logits(const float *sw, const float *rows, int hc, int col, float (&lg)[3]) {
    using L = WL<H>;
    lg[0] = sw[L::c1];
    lg[1] = sw[L::c1 + 1];
    lg[2] = sw[L::c1 + 2];
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
        const float4 w = *reinterpret_cast<const float4 *>(sw + L::C1t + 4 * k);
        const float h = rows[(hc + k) * RS + col];
        lg[0] = fmaf(w.x, h, lg[0]);
        lg[1] = fmaf(w.y, h, lg[1]);
        lg[2] = fmaf(w.z, h, lg[2]);
    }
}

template <int H>
__global__ void __launch_bounds__(TPB, 2) k_tile_centre_fwd(TrainArgs a) {
    using L = WL<H>;
    using R = RL<H>;
    extern __shared__ float4 smem4[];
    float *rows = reinterpret_cast<float *>(smem4);
    float *sw = rows + R::FC_ROWS * RS;
    __shared__ long long s_q[TILE];
    const int tid = threadIdx.x;
    const int k0 = a.NC, k1 = 2 * a.NC;
    const int64_t nfd = 6 * (a.B * a.S + a.M);
    const int c0 = a.chunk_off[k0], total = a.chunk_off[k1] - c0;
    constexpr int last = (H % 2 == 1) ? R::P : R::Q;
    for (int i = tid; i < R::FC_ROWS * RS; i += TPB) rows[i] = 0.f;
    __syncthreads();
    if (tid < TILE) rows[(R::FU + 33) * RS + tid] = 1.f;
    for (int ci = blockIdx.x; ci < total; ci += gridDim.x) {
        const int key = chunk_key(a.chunk_off, k0, k1, c0 + ci);
        const int j = c0 + ci - a.chunk_off[key];
        const int beg = a.off[key] + j * CHUNK, end = min(beg + CHUNK, a.off[key + 1]);
        __syncthreads();
        load_slots<H>(a.params + (int64_t)(key - a.NC) * a.p_cell, sw, 0, L::FC);
        for (int tb = beg; tb < end; tb += TILE) {
            {
                const int col = tid & (TILE - 1), i = tb + col;
                float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
                long long q = -1;
                if (i < end) {
                    r = a.sorted[i];
                    q = (long long)__float_as_int(r.w) - nfd;
                }
                encode_half(rows, R::A0, col, tid >> 7, r.x, r.y, r.z);
                if (tid < TILE) {
                    s_q[tid] = q;
                    if (q >= 0) centre_inputs(a, rows, R::FU, tid, q);
                }
            }
            __syncthreads();
            hidden_layer<27>(sw + L::T0, sw + L::b0, rows, R::A0, R::P, a.beta, a.inv_beta);
#pragma unroll
            for (int l = 1; l < H; ++l) {
                __syncthreads();
                hidden_layer<32>(sw + L::Tl(l), sw + L::bl(l), rows, (l % 2) ? R::P : R::Q, (l % 2) ? R::Q : R::P,
                                 a.beta, a.inv_beta);
            }
            __syncthreads();
            output_layer(sw + L::To, sw + L::bo, rows, last, R::FUd);  // d, then z into U rows 0..14
            __syncthreads();
            colour_hidden<H>(sw, rows, R::FU, R::FHc);
            __syncthreads();
            if (tid < TILE && s_q[tid] >= 0) {
                const long long q = s_q[tid];
                float lg[3];
                colour_logits<H>(sw, rows, R::FHc, tid, lg);
                a.d_c[q] = rows[R::FUd * RS + tid];
                a.rgb_c[3 * q] = sigm(lg[0]);
                a.rgb_c[3 * q + 1] = sigm(lg[1]);
                a.rgb_c[3 * q + 2] = sigm(lg[2]);
            }
        }
    }
}

// ------------------------------------------------------------------ backward
// weight-gradient plan: per layer (delta rows, OB, input rows, IB, real outputs, real inputs, canonical
// W and b offsets); thread block b covers outputs ob + OB jo and inputs ib + IB ji (jo, ji < 4)
struct GemmLayer {
    int drow, OB, arow, IB, out_real, in_real, cW, cb;
};

template <int H, bool CENTRE>
struct GemmPlan {
    static constexpr int NL = H + 1 + (CENTRE ? 2 : 0);
    // the delta rows of layer l's output: difference records keep D_l in place of A_l
    __host__ __device__ static constexpr int drow(int l) { return CENTRE ? RL<H>::D(l) : RL<H>::A(l); }
    __host__ __device__ static constexpr int dout() { return CENTRE ? RL<H>::Dout : RL<H>::DoutF; }
    __device__ static GemmLayer layer(int l) {
        using L = WL<H>;
        using R = RL<H>;
        if (l == 0) return {drow(1), 8, R::A0, 7, 32, 27, L::cW0, L::cb0};
        if (l < H) return {drow(l + 1), 8, R::A(l), 9, 32, 32, L::cH + (l - 1) * L::HL, L::cH + (l - 1) * L::HL + 1024};
        if (l == H) return {dout(), CENTRE ? 4 : 1, R::A(H), 9, CENTRE ? 16 : 1, 32, L::cWo, L::cbo};
        if (l == H + 1) return {R::Dh, 8, R::U, 9, 32, 33, L::cC0, L::cc0};
        return {R::Dc, 1, R::Hc, 9, 3, 32, L::cC1, L::cc1};
    }
    __host__ __device__ static constexpr int blocks() { return 56 + 72 * (H - 1) + (CENTRE ? 36 + 72 + 9 : 9); }
    static constexpr int NB = (blocks() + TPB - 1) / TPB;
};

struct Blk {
    int drow, OB, arow, IB, out_real, in_real, cW, cb, ob, ib, layer;
};

template <class Plan>
__device__ __forceinline__ Blk block_of(int b) {
    Blk k{};
    k.drow = -1;
    if (b >= Plan::blocks()) return k;
#pragma unroll 1
    for (int l = 0; l < Plan::NL; ++l) {
        const GemmLayer G = Plan::layer(l);
        const int n = G.OB * G.IB;
        if (b < n) {
            k.layer = l;
            k.drow = G.drow;
            k.OB = G.OB;
            k.arow = G.arow;
            k.IB = G.IB;
            k.out_real = G.out_real;
            k.in_real = G.in_real;
            k.cW = G.cW;
            k.cb = G.cb;
            if (G.IB == 9) {
                // eight consecutive lanes (one shared-memory phase of a 16-byte load) take input rows
                // ib = 0..7 of one output group, so their rows fall in distinct bank groups; the
                // ib = 8 blocks follow, one per output group
                if (b < 8 * G.OB) {
                    k.ob = b >> 3;
                    k.ib = b & 7;
                } else {
                    k.ob = b - 8 * G.OB;
                    k.ib = 8;
                }
            } else {
                k.ob = b / G.IB;
                k.ib = b - k.ob * G.IB;
            }
            return k;
        }
        b -= n;
    }
    return k;
}

// layer >= 0: only the blocks of that plan layer
template <class Plan>
__device__ __forceinline__ void grad_tile(const float *rows, int b, float (&acc)[16], int layer = -1) {
    const Blk k = block_of<Plan>(b);
    if (k.drow < 0 || (layer >= 0 && k.layer != layer)) return;
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
__device__ __forceinline__ void flush_grad(float *gcell, int b, float (&acc)[16]) {
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

// D_l = (W_l^T D_{l+1}) . softplus'(A_l) for l = H-1 .. 1 (D_H already in its rows)
template <int H>
__device__ __forceinline__ void hidden_backward(const float *sw, float *rows, float beta) {
    using L = WL<H>;
    using R = RL<H>;
#pragma unroll
    for (int l = H - 1; l >= 1; --l) {
        __syncthreads();
        float acc[4][4], act[4][4];
        zero(acc);
        mm32<32, 32>(sw + L::Wr(l), rows + R::D(l + 1) * RS, acc);
        load_rows(rows, R::A(l), act);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] *= dsoftplus_act(act[i][j], beta);
        store_rows(rows, R::D(l), acc);
    }
}

// CENTRE: sample-centre records (colour MLP + SDF with upstream on d and z; writes the difference
// records' upstream).  Otherwise: difference records (SDF with upstream on d only).
template <int H, bool CENTRE>
__global__ void __launch_bounds__(TPB, CENTRE ? 1 : 2) k_tile_backward(TrainArgs a) {
    using L = WL<H>;
    using R = RL<H>;
    using Plan = GemmPlan<H, CENTRE>;
    constexpr int NROWS = CENTRE ? R::C_ROWS : R::FDI_ROWS;
    extern __shared__ float4 smem4[];
    float *rows = reinterpret_cast<float *>(smem4);
    float *sw = rows + NROWS * RS;
    __shared__ long long s_q[TILE];
    const int tid = threadIdx.x;
    for (int i = tid; i < NROWS * RS; i += TPB) rows[i] = 0.f;
    __syncthreads();
    if (tid < TILE) {
        rows[(R::A0 + 27) * RS + tid] = 1.f;
        for (int l = 1; l <= H; ++l) rows[(R::A(l) + 32) * RS + tid] = 1.f;
        if (CENTRE) {
            rows[(R::U + 33) * RS + tid] = 1.f;
            rows[(R::Hc + 32) * RS + tid] = 1.f;
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
        const float *cw = a.params + (int64_t)cell * a.p_cell;
        __syncthreads();
        load_slots<H>(cw, sw, 0, L::FS);
        if (CENTRE) load_slots<H>(cw, sw, L::FS, L::END);
        else load_slots<H>(cw, sw, L::FC, L::BS);
        for (int tb = beg; tb < end; tb += TILE) {
            // records: encoding, and the upstream of d (difference points) or the colour inputs (centres)
            {
                const int col = tid & (TILE - 1), i = tb + col;
                float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
                long long q = -1;
                if (i < end) {
                    r = a.sorted[i];
                    q = (long long)__float_as_int(r.w) - (CENTRE ? nfd : 0);
                }
                encode_half(rows, R::A0, col, tid >> 7, r.x, r.y, r.z);
                if (tid < TILE) {
                    s_q[tid] = q;
                    if (CENTRE) {
                        if (q >= 0) centre_inputs(a, rows, R::U, tid, q);
                    } else {
                        rows[R::DoutF * RS + tid] = q >= 0 ? a.g_fd[q] : 0.f;
                    }
                }
            }
            __syncthreads();
            hidden_layer<27>(sw + L::T0, sw + L::b0, rows, R::A0, R::A(1), a.beta, a.inv_beta);
#pragma unroll
            for (int l = 1; l < H; ++l) {
                __syncthreads();
                hidden_layer<32>(sw + L::Tl(l), sw + L::bl(l), rows, R::A(l), R::A(l + 1), a.beta, a.inv_beta);
            }
            __syncthreads();
            if (CENTRE) {
                output_layer(sw + L::To, sw + L::bo, rows, R::A(H), R::Ud);  // d, then z into U rows 0..14
                __syncthreads();
                colour_hidden<H>(sw, rows, R::U, R::Hc);
                __syncthreads();
                // logits -> colour delta (rows Dc)
                if (tid < TILE) {
                    const long long q = s_q[tid];
                    float lg[3];
                    colour_logits<H>(sw, rows, R::Hc, tid, lg);
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float rgb = sigm(lg[c]);
                        rows[(R::Dc + c) * RS + tid] = q >= 0 ? a.g_rgb[3 * q + c] * rgb * (1.f - rgb) : 0.f;
                    }
                }
                __syncthreads();
                // hidden delta: Dh = (Wc1^T Dc) . [Hc > 0]
                {
                    float dh[4][4], hv[4][4];
                    load_rows(rows, R::Hc, hv);
                    const int o0 = o0_32(), r0 = r0_t();
                    float dc[3][4];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float4 x = *reinterpret_cast<const float4 *>(rows + (R::Dc + c) * RS + r0);
                        dc[c][0] = x.x;
                        dc[c][1] = x.y;
                        dc[c][2] = x.z;
                        dc[c][3] = x.w;
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float w0 = sw[L::Wc1 + o0 + i], w1 = sw[L::Wc1 + 32 + o0 + i],
                                    w2 = sw[L::Wc1 + 64 + o0 + i];
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) {
                            const float s = fmaf(w0, dc[0][jj], fmaf(w1, dc[1][jj], w2 * dc[2][jj]));
                            dh[i][jj] = hv[i][jj] > 0.f ? s : 0.f;
                        }
                    }
                    store_rows(rows, R::Dh, dh);
                }
                __syncthreads();
                // input deltas of z and n: gu[i] = sum_o Wc0[o][i] Dh[o]; two threads per record
                {
                    const int col = tid & (TILE - 1), half = tid >> 7;
                    const long long q = s_q[col];
                    const int i0 = half ? 9 : 0;
                    float gu[9];
#pragma unroll
                    for (int m = 0; m < 9; ++m) gu[m] = 0.f;
#pragma unroll 4
                    for (int o = 0; o < 32; ++o) {
                        const float dh = rows[(R::Dh + o) * RS + col];
#pragma unroll
                        for (int m = 0; m < 9; ++m) gu[m] = fmaf(sw[L::Wc0 + o * 36 + i0 + m], dh, gu[m]);
                    }
                    // z deltas (+ the d upstream) into Dout; the normal's delta to the difference records
#pragma unroll
                    for (int m = 0; m < 9; ++m)
                        if (i0 + m < 15) rows[(R::Dout + 1 + i0 + m) * RS + col] = gu[m];
                    if (half == 0) {
                        rows[R::Dout * RS + col] = q >= 0 ? a.g_dc[q] : 0.f;
                    } else if (q >= 0) {
                        float g[3], n[3];
                        const float gn = fd_normal(a, q, g, n);
                        const float gx = gu[6], gy = gu[7], gz = gu[8];  // inputs 15, 16, 17
                        const float nd = n[0] * gx + n[1] * gy + n[2] * gz;
                        const float ig = gn > 0.f ? inv2h / gn : 0.f;
                        const float dg[3] = {(gx - n[0] * nd) * ig, (gy - n[1] * nd) * ig, (gz - n[2] * nd) * ig};
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            a.g_fd[6 * q + 2 * k] = dg[k];
                            a.g_fd[6 * q + 2 * k + 1] = -dg[k];
                        }
                    }
                }
                __syncthreads();
                // D_H = (Wo^T Dout) . softplus'(A_H)
                {
                    float acc2[4][4], act[4][4];
                    zero(acc2);
                    mm32<16, 32>(sw + L::Wo, rows + R::Dout * RS, acc2);
                    load_rows(rows, R::A(H), act);
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) acc2[i][jj] *= dsoftplus_act(act[i][jj], a.beta);
                    store_rows(rows, R::D(H), acc2);
                }
                hidden_backward<H>(sw, rows, a.beta);
                __syncthreads();
#pragma unroll
                for (int k = 0; k < Plan::NB; ++k) grad_tile<Plan>(rows, tid + k * TPB, acc[k]);
                __syncthreads();
            } else {
                // Difference records, deltas in place of the activations (so two blocks fit per SM): each
                // layer's weight gradient is taken while its input activations are still in their rows.
                // Output layer first (Dout x A_H), then D_H = Wo[0] g . softplus'(A_H) over A_H.
#pragma unroll
                for (int k = 0; k < Plan::NB; ++k) grad_tile<Plan>(rows, tid + k * TPB, acc[k], H);
                __syncthreads();
                {
                    float act[4][4], dd[4][4];
                    load_rows(rows, R::A(H), act);
                    const float4 g4 = *reinterpret_cast<const float4 *>(rows + R::DoutF * RS + r0_t());
                    const float g[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float w = sw[L::Wo + o0_32() + i];
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) dd[i][jj] = w * g[jj] * dsoftplus_act(act[i][jj], a.beta);
                    }
                    store_rows(rows, R::A(H), dd);  // each thread reads and writes only its own block
                }
                // hidden layer l: its weight gradient (D_{l+1} x A_l), then D_l over A_l
#pragma unroll
                for (int l = H - 1; l >= 1; --l) {
                    __syncthreads();
#pragma unroll
                    for (int k = 0; k < Plan::NB; ++k) grad_tile<Plan>(rows, tid + k * TPB, acc[k], l);
                    __syncthreads();
                    float dacc[4][4], act[4][4];
                    zero(dacc);
                    mm32<32, 32>(sw + L::Wr(l), rows + R::A(l + 1) * RS, dacc);
                    load_rows(rows, R::A(l), act);
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) dacc[i][jj] *= dsoftplus_act(act[i][jj], a.beta);
                    store_rows(rows, R::A(l), dacc);
                }
                __syncthreads();
#pragma unroll
                for (int k = 0; k < Plan::NB; ++k) grad_tile<Plan>(rows, tid + k * TPB, acc[k], 0);
                __syncthreads();
            }
        }
        float *gcell = a.grad + (int64_t)cell * a.p_cell;
#pragma unroll
        for (int k = 0; k < Plan::NB; ++k) flush_grad<Plan>(gcell, tid + k * TPB, acc[k]);
    }
}

// ------------------------------------------------------------------ launchers
template <int H>
size_t eval_smem() { return ((size_t)RL<H>::F_ROWS * RS + WL<H>::FS) * sizeof(float); }
template <int H>
size_t centre_fwd_smem() { return ((size_t)RL<H>::FC_ROWS * RS + WL<H>::FC) * sizeof(float); }
template <int H>
size_t backward_smem(bool centre) {
    return ((size_t)(centre ? RL<H>::C_ROWS : RL<H>::FDI_ROWS) * RS + (centre ? WL<H>::END : WL<H>::BS)) *
           sizeof(float);
}

template <class F>
cudaError_t set_smem(F f, size_t bytes) {
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int H>
cudaError_t eval_d_h(const TrainArgs &a, int k0, int k1, float *out, int64_t chunks, int sm_count, cudaStream_t s) {
    const size_t sm = eval_smem<H>();
    cudaError_t e = set_smem(k_tile_eval_d<H>, sm);
    if (e != cudaSuccess) return e;
    k_tile_eval_d<H><<<grid_for(sm_count, 3, chunks), TPB, sm, s>>>(a, k0, k1, out);
    return cudaGetLastError();
}

template <int H>
cudaError_t centre_fwd_h(const TrainArgs &a, int64_t chunks, int sm_count, cudaStream_t s) {
    const size_t sm = centre_fwd_smem<H>();
    cudaError_t e = set_smem(k_tile_centre_fwd<H>, sm);
    if (e != cudaSuccess) return e;
    k_tile_centre_fwd<H><<<grid_for(sm_count, 2, chunks), TPB, sm, s>>>(a);
    return cudaGetLastError();
}

template <int H, bool CENTRE>
cudaError_t backward_h(const TrainArgs &a, int64_t chunks, int sm_count, cudaStream_t s) {
    const size_t sm = backward_smem<H>(CENTRE);
    cudaError_t e = set_smem(k_tile_backward<H, CENTRE>, sm);
    if (e != cudaSuccess) return e;
    // difference records hold their deltas in place of the activations: two blocks fit per SM
    k_tile_backward<H, CENTRE><<<grid_for(sm_count, CENTRE ? 1 : 2, chunks), TPB, sm, s>>>(a);
    return cudaGetLastError();
}

int64_t fd_chunks(const TrainArgs &a) { return 6 * (a.B * a.S + a.M) / CHUNK + a.NC + 1; }
int64_t centre_chunks(const TrainArgs &a) { return a.B * a.S / CHUNK + a.NC + 1; }

}  // namespace

cudaError_t train_coarse_eval(const TrainArgs &a, int sm_count, cudaStream_t s) {
    const int64_t chunks = a.B * a.Ns / CHUNK + a.NC + 1;
    return a.H == 3 ? eval_d_h<3>(a, 0, a.NC, a.d_coarse, chunks, sm_count, s)
                    : eval_d_h<2>(a, 0, a.NC, a.d_coarse, chunks, sm_count, s);
}

cudaError_t train_fd_forward(const TrainArgs &a, int sm_count, cudaStream_t s) {
    return a.H == 3 ? eval_d_h<3>(a, 0, a.NC, a.d_fd, fd_chunks(a), sm_count, s)
                    : eval_d_h<2>(a, 0, a.NC, a.d_fd, fd_chunks(a), sm_count, s);
}

cudaError_t train_centre_forward(const TrainArgs &a, int sm_count, cudaStream_t s) {
    return a.H == 3 ? centre_fwd_h<3>(a, centre_chunks(a), sm_count, s)
                    : centre_fwd_h<2>(a, centre_chunks(a), sm_count, s);
}

cudaError_t train_centre_backward(const TrainArgs &a, int sm_count, cudaStream_t s) {
    return a.H == 3 ? backward_h<3, true>(a, centre_chunks(a), sm_count, s)
                    : backward_h<2, true>(a, centre_chunks(a), sm_count, s);
}

cudaError_t train_fd_backward(const TrainArgs &a, int sm_count, cudaStream_t s) {
    return a.H == 3 ? backward_h<3, false>(a, fd_chunks(a), sm_count, s)
                    : backward_h<2, false>(a, fd_chunks(a), sm_count, s);
}

}  // namespace kns
