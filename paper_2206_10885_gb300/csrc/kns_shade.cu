// kns_shade.cu -- shading of the converged rays on block tiles (Sec. 3.1: full SDF [d, z], the
// analytic input gradient as the normal, the colour MLP of Eq. 3 at the hit).
// kns:instantiate (compiled once per grid configuration)
//
// The hits of a render are counting-sorted by cell and cut into tiles of 4096 / W same-cell hits (128
// for width 32, 64 for width 64).  A block of 256 threads stages the cell's weights in shared memory
// with one TMA bulk copy of the cell's block of the shading layout, which the grid load writes once
// (forward layers k-major, the layers the gradient runs back through row-major), and evaluates the
// tile as block GEMMs on rows of hits (row stride tile + 4 floats): thread (warp w, lane l) owns W/8
// output units x tile/32 hits.  Forward:
// A_l = softplus(W_l A_{l-1} + b_l), the 16 outputs [d, z].  Reverse mode in place: A_H becomes
// D_H = w_d . softplus'(A_H), each A_l becomes D_l = (W_l^T D_{l+1}) . softplus'(A_l), and the
// encoding rows become W_0^T D_1; the chain rule through the encoding (d sin(fx) = f cos(fx) dx,
// d cos(fx) = -f sin(fx) dx) gives grad d, normalised to n.  The colour MLP then runs on
// u = [z, n, gamma(v), x].
#include <algorithm>

#include "kns_wave.cuh"

namespace kns {
namespace {

constexpr int STHREADS = 256;

// shared layout of one cell and of a tile (floats, 16-byte aligned blocks)
template <class C>
struct SL {
    static constexpr int W = C::W, R0 = (C::INP + 31) / 32 * 32;  // encoding rows, padded to 32
    static constexpr int ST = 4096 / W, SRS = ST + 4;              // hits per tile (shade_hit_tile), row stride
    static constexpr int OPT = W / 8, SPT = ST / 32;               // outputs x hits per thread
    // forward, k-major
    static constexpr int T0 = 0, b0 = T0 + C::INP * W, HL = W * W + W;
    __host__ __device__ static constexpr int Tl(int l) { return b0 + W + (l - 1) * HL; }
    __host__ __device__ static constexpr int bl(int l) { return Tl(l) + W * W; }
    static constexpr int To = b0 + W + (C::H - 1) * HL, bo = To + W * 16;
    // reverse, row-major
    static constexpr int W0r = bo + 16;  // [W][R0]
    __host__ __device__ static constexpr int Wlr(int l) { return W0r + W * R0 + (l - 1) * W * W; }
    static constexpr int wd = W0r + W * R0 + (C::H - 1) * W * W;
    // colour, k-major
    static constexpr int C0t = wd + W, c0 = C0t + C::CINP * W, C1t = c0 + W, c1 = C1t + W * 4, END = c1 + 4;
    // tile rows
    static constexpr int A0 = 0;
    __host__ __device__ static constexpr int A(int l) { return R0 + (l - 1) * W; }
    static constexpr int Ud = R0 + C::H * W, U = Ud + 1, Hc = U + C::CINP, ROWS = Hc + W;
};

// per-thread layout index (kns_device.cuh) of shared slot j, or -1 for zero padding
template <class C>
__device__ int src_of(int j) {
    using L = SL<C>;
    constexpr int W = C::W;
    if (j < L::b0) {
        const int k = j / W, o = j % W;
        return C::oW0 + o * C::INP + k;
    }
    if (j < L::b0 + W) return C::ob0 + (j - L::b0);
    if (j < L::To) {
        const int u = j - (L::b0 + W), l = u / L::HL, v = u % L::HL;
        if (v < W * W) return C::oWl(l + 1) + (v % W) * W + v / W;  // Tl[k][o] = W_l[o][k]
        return C::obl(l + 1) + (v - W * W);
    }
    if (j < L::bo) {
        const int u = j - L::To, k = u / 16, o = u % 16;
        return C::oWL + o * W + k;
    }
    if (j < L::W0r) return C::obL + (j - L::bo);
    if (j < L::Wlr(1)) {
        const int u = j - L::W0r, o = u / L::R0, k = u % L::R0;
        return k < C::INP ? C::oW0 + o * C::INP + k : -1;
    }
    if (j < L::wd) {
        const int u = j - L::Wlr(1), l = u / (W * W), v = u % (W * W);
        return C::oWl(l + 1) + v;
    }
    if (j < L::C0t) return C::oWL + (j - L::wd);  // row 0 of the output layer (the d row)
    if (j < L::c0) {
        const int u = j - L::C0t, k = u / W, o = u % W;
        return C::oC0 + o * C::CINP + k;
    }
    if (j < L::C1t) return C::oc0 + (j - L::c0);
    if (j < L::c1) {
        const int u = j - L::C1t, k = u / 4, r = u % 4;
        return r < 3 ? C::oC1 + r * W + k : -1;
    }
    return (j - L::c1) < 3 ? C::oc1 + (j - L::c1) : -1;
}

__device__ __forceinline__ float dsoftplus_from_act(float a, float beta) {
    const float x = beta * a;  // sigmoid(beta s) = 1 - exp(-beta softplus_beta(s)); series for small x
    return x < 1e-2f ? x * (1.f - x * (0.5f - x * (1.f / 6.f))) : 1.f - __expf(-x);
}

template <class L>
__device__ __forceinline__ int o0_of() { return (threadIdx.x >> 5) * L::OPT; }
template <class L>
__device__ __forceinline__ int s0_of() { return (threadIdx.x & 31) * L::SPT; }

template <int N>
__device__ __forceinline__ void load_n(const float *p, float (&v)[N]) {
    if constexpr (N == 4) {
        const float4 x = *reinterpret_cast<const float4 *>(p);
        v[0] = x.x;
        v[1] = x.y;
        v[2] = x.z;
        v[3] = x.w;
    } else if constexpr (N == 2) {
        const float2 x = *reinterpret_cast<const float2 *>(p);
        v[0] = x.x;
        v[1] = x.y;
    } else {
#pragma unroll
        for (int i = 0; i < N; i += 4) {
            const float4 x = *reinterpret_cast<const float4 *>(p + i);
            v[i] = x.x;
            v[i + 1] = x.y;
            v[i + 2] = x.z;
            v[i + 3] = x.w;
        }
    }
}

template <int N>
__device__ __forceinline__ void store_n(float *p, const float (&v)[N]) {
    if constexpr (N == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    }
}

// acc[i][j] += sum_{k < K} Wk[k WS + o0 + i] X[k SRS + s0 + j]
template <class L, int K, int WS>
__device__ __forceinline__ void mm(const float *Wk, const float *X, float (&acc)[L::OPT][L::SPT]) {
    const float *w = Wk + o0_of<L>();
    const float *x = X + s0_of<L>();
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
        float wa[L::OPT], xa[L::SPT];
        load_n<L::OPT>(w + k * WS, wa);
        load_n<L::SPT>(x + k * L::SRS, xa);
#pragma unroll
        for (int i = 0; i < L::OPT; ++i)
#pragma unroll
            for (int j = 0; j < L::SPT; ++j) acc[i][j] = fmaf(wa[i], xa[j], acc[i][j]);
    }
}

template <class L>
__device__ __forceinline__ void bias_n(const float *b, float (&acc)[L::OPT][L::SPT]) {
#pragma unroll
    for (int i = 0; i < L::OPT; ++i)
#pragma unroll
        for (int j = 0; j < L::SPT; ++j) acc[i][j] = b[o0_of<L>() + i];
}

template <class L>
__device__ __forceinline__ void zero_n(float (&acc)[L::OPT][L::SPT]) {
#pragma unroll
    for (int i = 0; i < L::OPT; ++i)
#pragma unroll
        for (int j = 0; j < L::SPT; ++j) acc[i][j] = 0.f;
}

template <class L>
__device__ __forceinline__ void put_n(float *rows, int row0, const float (&v)[L::OPT][L::SPT]) {
#pragma unroll
    for (int i = 0; i < L::OPT; ++i) store_n<L::SPT>(rows + (row0 + o0_of<L>() + i) * L::SRS + s0_of<L>(), v[i]);
}

template <class L>
__device__ __forceinline__ void get_n(const float *rows, int row0, float (&v)[L::OPT][L::SPT]) {
#pragma unroll
    for (int i = 0; i < L::OPT; ++i) load_n<L::SPT>(rows + (row0 + o0_of<L>() + i) * L::SRS + s0_of<L>(), v[i]);
}

// The shading layout of every cell (grid load): slot j of cell c is canonical weight src_of(j), or 0.
template <class C>
__global__ void shade_layout_kernel(const float *__restrict__ w, int cell_stride, int64_t ncell, float *ws,
                                    int ws_stride) {
    const int64_t n = ncell * ws_stride;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i / ws_stride;
        const int j = (int)(i - c * ws_stride);
        const int k = j < SL<C>::END ? src_of<C>(j) : -1;
        ws[i] = k >= 0 ? w[c * cell_stride + k] : 0.f;
    }
}

constexpr uint32_t kShadePolls = 1u << 26;  // bound of the weight copy's wait

template <class C>
__global__ void __launch_bounds__(STHREADS) shade_block_kernel(GridView g, WaveArgs a) {
    using L = SL<C>;
    constexpr int W = C::W, ST = L::ST, SRS = L::SRS, OPT = L::OPT, SPT = L::SPT;
    static_assert(L::END % 4 == 0, "the weight copy must be a multiple of 16 bytes");
    extern __shared__ __align__(16) float sdyn[];
    float *sw = sdyn;
    float *rows = sdyn + L::END;
    __shared__ float s_x[3][ST], s_v[3][ST], s_t[ST];
    __shared__ int s_r[ST];
    __shared__ int s_tile[3];
    __shared__ __align__(8) uint64_t s_bar;
    const int tid = threadIdx.x;
    // padding rows stay zero
    for (int i = tid; i < L::ROWS * SRS; i += STHREADS) rows[i] = 0.f;
    if (tid == 0) mbar_init(&s_bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    const int n_tiles = a.ctrl->n_tiles;
    // a contiguous run of tiles per block, so consecutive tiles mostly share the cell's staged
    // weights; thread 0 holds the next tile's descriptor (loaded a tile ahead)
    const int per = (n_tiles + gridDim.x - 1) / gridDim.x;
    const int t_begin = blockIdx.x * per, t_end = min(n_tiles, t_begin + per);
    int cached = -1;
    int4 nd = make_int4(-1, 0, 0, 0);
    if (tid == 0 && t_begin < t_end) nd = a.tiles[t_begin];
    for (int tile = t_begin; tile < t_end; ++tile) {
        if (tid == 0) {
            s_tile[0] = nd.x;
            s_tile[1] = nd.y;
            s_tile[2] = nd.z;
            if (tile + 1 < t_end) nd = a.tiles[tile + 1];
        }
        __syncthreads();
        const int c = s_tile[0], start = s_tile[1], len = s_tile[2];
        // a new cell: its weights are copied while the tile's rays are read and encoded (the previous
        // tile finished with a barrier, so nobody reads the old weights any more)
        const bool fresh = c != cached;
        if (fresh && tid == 0) bulk_load(sw, g.ws + (int64_t)c * g.ws_stride, L::END * (uint32_t)sizeof(float), &s_bar);
        cached = c;
        if (tid < ST) {
            float x = 0.f, y = 0.f, z = 0.f, wx = 0.f, wy = 0.f, wz = 1.f, t = 0.f;
            int r = -1;
            if (tid < len) {
                r = a.sorted[start + tid];
                t = a.t_ray[r];
                int cam;
                const Ray ray = ray_of(a, r, cam);
                x = fmaf(t, ray.wx, ray.ox);
                y = fmaf(t, ray.wy, ray.oy);
                z = fmaf(t, ray.wz, ray.oz);
                wx = ray.wx;
                wy = ray.wy;
                wz = ray.wz;
            }
            s_x[0][tid] = x;
            s_x[1][tid] = y;
            s_x[2][tid] = z;
            s_v[0][tid] = wx;
            s_v[1][tid] = wy;
            s_v[2][tid] = wz;
            s_t[tid] = t;
            s_r[tid] = r;
        }
        __syncthreads();
        if (tid < 2 * ST) {  // encoding (Eq. 1), two threads per hit: x and frequencies [0, L/2) | [L/2, L)
            const int s = tid % ST, half = tid / ST;
            const float p[3] = {s_x[0][s], s_x[1][s], s_x[2][s]};
            if (half == 0)
                for (int k = 0; k < 3; ++k) rows[(L::A0 + k) * SRS + s] = p[k];
#pragma unroll
            for (int kk = 0; kk < C::L / 2; ++kk) {
                const int k = half * (C::L / 2) + kk;
                const float f = (float)(1 << k);
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    float sn, cs;
                    sincospif(f * p[q], &sn, &cs);
                    rows[(L::A0 + 3 + 6 * k + q) * SRS + s] = sn;
                    rows[(L::A0 + 6 + 6 * k + q) * SRS + s] = cs;
                }
            }
        }
        if (fresh) {
            const bool ok = mbar_wait(&s_bar, phase, kShadePolls);
            phase ^= 1u;
            if (__syncthreads_or(!ok)) {  // the weights never landed: report and leave
                if (tid == 0) atomicCAS(a.status, 0, (int)6 /* KNS_ERR_TIMEOUT */);
                return;
            }
        }
        __syncthreads();
        float acc[OPT][SPT];
        // forward
        bias_n<L>(sw + L::b0, acc);
        mm<L, C::INP, W>(sw + L::T0, rows + L::A0 * SRS, acc);
#pragma unroll
        for (int i = 0; i < OPT; ++i)
#pragma unroll
            for (int j = 0; j < SPT; ++j) acc[i][j] = softplus_f32(acc[i][j], g.beta, g.inv_beta);
        put_n<L>(rows, L::A(1), acc);
#pragma unroll
        for (int l = 1; l < C::H; ++l) {
            __syncthreads();
            bias_n<L>(sw + L::bl(l), acc);
            mm<L, W, W>(sw + L::Tl(l), rows + L::A(l) * SRS, acc);
#pragma unroll
            for (int i = 0; i < OPT; ++i)
#pragma unroll
                for (int j = 0; j < SPT; ++j) acc[i][j] = softplus_f32(acc[i][j], g.beta, g.inv_beta);
            put_n<L>(rows, L::A(l + 1), acc);
        }
        __syncthreads();
        {  // outputs [d, z]: 16 rows from Ud (z lands in U rows 0..14); warp w owns outputs 2w, 2w+1
            const int o0 = (tid >> 5) * 2, s0 = s0_of<L>();
            float out[2][SPT];
#pragma unroll
            for (int j = 0; j < SPT; ++j) {
                out[0][j] = sw[L::bo + o0];
                out[1][j] = sw[L::bo + o0 + 1];
            }
            const float *X = rows + L::A(C::H) * SRS + s0;
#pragma unroll 4
            for (int k = 0; k < W; ++k) {
                const float2 wv = *reinterpret_cast<const float2 *>(sw + L::To + k * 16 + o0);
                float xa[SPT];
                load_n<SPT>(X + k * SRS, xa);
#pragma unroll
                for (int j = 0; j < SPT; ++j) {
                    out[0][j] = fmaf(wv.x, xa[j], out[0][j]);
                    out[1][j] = fmaf(wv.y, xa[j], out[1][j]);
                }
            }
#pragma unroll
            for (int i = 0; i < 2; ++i) store_n<SPT>(rows + (L::Ud + o0 + i) * SRS + s0, out[i]);
        }
        __syncthreads();
        if (a.coarse && tid < ST) {
            // BF16 render: this FP32 evaluation re-evaluates the BF16 trace's last step; a hit it does not
            // confirm (|d| >= eps) goes to the refinement list with its d, and is not shaded here
            const int r = s_r[tid];
            const float d = rows[L::Ud * SRS + tid];
            const bool refine = r >= 0 && !(fabsf(d) < a.eps);
            const int q = warp_append(&a.ctrl->n_refine, refine);
            if (refine) {
                a.pend_r[0][q] = r;
                a.pend_t[0][q] = d;
                s_r[tid] = -1;
            }
            const unsigned long long nv = warp_sum_u64(r >= 0 ? 1u : 0u);
            if ((tid & 31) == 0 && nv) atomicAdd(&a.ctrl->samples_f32, nv);
        }
        __syncthreads();
        // reverse mode, in place: D_H = w_d . softplus'(A_H)
        {
            float act[OPT][SPT];
            get_n<L>(rows, L::A(C::H), act);
#pragma unroll
            for (int i = 0; i < OPT; ++i)
#pragma unroll
                for (int j = 0; j < SPT; ++j)
                    act[i][j] = sw[L::wd + o0_of<L>() + i] * dsoftplus_from_act(act[i][j], g.beta);
            put_n<L>(rows, L::A(C::H), act);
        }
#pragma unroll
        for (int l = C::H - 1; l >= 1; --l) {
            __syncthreads();
            float act[OPT][SPT];
            zero_n<L>(acc);
            mm<L, W, W>(sw + L::Wlr(l), rows + L::A(l + 1) * SRS, acc);
            get_n<L>(rows, L::A(l), act);
#pragma unroll
            for (int i = 0; i < OPT; ++i)
#pragma unroll
                for (int j = 0; j < SPT; ++j) acc[i][j] *= dsoftplus_from_act(act[i][j], g.beta);
            put_n<L>(rows, L::A(l), acc);  // each thread reads and writes only its own block of A_l
        }
        __syncthreads();
        // encoding rows <- W_0^T D_1, in groups of W outputs (the thread's outputs o0 .. o0 + OPT - 1)
#pragma unroll
        for (int grp = 0; grp < (L::R0 + W - 1) / W; ++grp) {
            zero_n<L>(acc);
            mm<L, W, L::R0>(sw + L::W0r + W * grp, rows + L::A(1) * SRS, acc);
            if (W * grp + o0_of<L>() < L::R0) put_n<L>(rows, L::A0 + W * grp, acc);
        }
        __syncthreads();
        // per hit: grad d through the encoding, the normal, the colour inputs and the geometry outputs
        if (tid < ST) {
            const int s = tid;
            const float p[3] = {s_x[0][s], s_x[1][s], s_x[2][s]};
            float gr[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                float gc = rows[(L::A0 + q) * SRS + s];
#pragma unroll
                for (int k = 0; k < C::L; ++k) {
                    const float f = 3.14159265358979323846f * (float)(1 << k);
                    float sn, cs;
                    sincospif((float)(1 << k) * p[q], &sn, &cs);
                    gc = fmaf(rows[(L::A0 + 3 + 6 * k + q) * SRS + s] * f, cs, gc);
                    gc = fmaf(-rows[(L::A0 + 6 + 6 * k + q) * SRS + s] * f, sn, gc);
                }
                gr[q] = gc;
            }
            const float gn = sqrtf(fmaf(gr[0], gr[0], fmaf(gr[1], gr[1], gr[2] * gr[2])));
            const float inv = gn > 0.f ? 1.f / gn : 0.f;
            const float n[3] = {gr[0] * inv, gr[1] * inv, gr[2] * inv};
            rows[(L::U + FEAT) * SRS + s] = n[0];
            rows[(L::U + FEAT + 1) * SRS + s] = n[1];
            rows[(L::U + FEAT + 2) * SRS + s] = n[2];
            float gv[3 + 6 * C::LD];
            encode3<C::LD>(s_v[0][s], s_v[1][s], s_v[2][s], gv);
#pragma unroll
            for (int k = 0; k < 3 + 6 * C::LD; ++k) rows[(L::U + FEAT + 3 + k) * SRS + s] = gv[k];
            rows[(L::U + C::CIN - 3) * SRS + s] = p[0];
            rows[(L::U + C::CIN - 2) * SRS + s] = p[1];
            rows[(L::U + C::CIN - 1) * SRS + s] = p[2];
            const int r = s_r[s];
            if (r >= 0) {
                int cam = a.ray_view[r];
                const ViewDev &V = a.views[cam];
                const int64_t px = r - V.ray_base;
                V.depth[px] = s_t[s];
                if (V.normal) {
                    V.normal[3 * px + 0] = n[0];
                    V.normal[3 * px + 1] = n[1];
                    V.normal[3 * px + 2] = n[2];
                }
                if (V.cell) V.cell[px] = c - V.grid * g.ncl;  // the cell within the view's grid
                if (V.steps) V.steps[px] = a.steps_ray[r];
                if (V.hit) V.hit[px] = 1;
            }
        }
        __syncthreads();
        // colour hidden layer (ReLU)
        bias_n<L>(sw + L::c0, acc);
        mm<L, C::CINP, W>(sw + L::C0t, rows + L::U * SRS, acc);
#pragma unroll
        for (int i = 0; i < OPT; ++i)
#pragma unroll
            for (int j = 0; j < SPT; ++j) acc[i][j] = fmaxf(acc[i][j], 0.f);
        put_n<L>(rows, L::Hc, acc);
        __syncthreads();
        if (tid < ST && s_r[tid] >= 0) {
            const int s = tid;
            float lg[3] = {sw[L::c1], sw[L::c1 + 1], sw[L::c1 + 2]};
#pragma unroll 8
            for (int k = 0; k < W; ++k) {
                const float4 w = *reinterpret_cast<const float4 *>(sw + L::C1t + 4 * k);
                const float h = rows[(L::Hc + k) * SRS + s];
                lg[0] = fmaf(w.x, h, lg[0]);
                lg[1] = fmaf(w.y, h, lg[1]);
                lg[2] = fmaf(w.z, h, lg[2]);
            }
            const int r = s_r[s];
            const ViewDev &V = a.views[a.ray_view[r]];
            const int64_t px = r - V.ray_base;
            V.rgb[3 * px + 0] = sigmoid_f32(lg[0]);
            V.rgb[3 * px + 1] = sigmoid_f32(lg[1]);
            V.rgb[3 * px + 2] = sigmoid_f32(lg[2]);
        }
        __syncthreads();
    }
}

}  // namespace

template <class C>
cudaError_t launch_shade_block_cfg(const GridView &g, const WaveArgs &a, int sm_count, cudaStream_t s) {
    constexpr int smem = (SL<C>::END + SL<C>::ROWS * SL<C>::SRS) * (int)sizeof(float);
    static_assert(smem <= 220 * 1024, "shade tile does not fit in shared memory");
    cudaError_t e = cudaFuncSetAttribute(shade_block_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    shade_block_kernel<C><<<sm_count, STHREADS, smem, s>>>(g, a);
    return cudaGetLastError();
}

template <class C>
int shade_cell_floats_cfg() {
    return (SL<C>::END + 31) / 32 * 32;
}
template <class C>
cudaError_t launch_shade_layout_cfg(const float *w, int cell_stride, int64_t ncell, float *ws, int ws_stride,
                                    cudaStream_t s) {
    const int64_t n = ncell * ws_stride;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 1 << 20);
    shade_layout_kernel<C><<<(unsigned)blocks, 256, 0, s>>>(w, cell_stride, ncell, ws, ws_stride);
    return cudaGetLastError();
}

#ifdef KNS_W
using InstCfg = Cfg<KNS_W, KNS_H, KNS_L, KNS_LD>;
template cudaError_t launch_shade_block_cfg<InstCfg>(const GridView &, const WaveArgs &, int, cudaStream_t);
template int shade_cell_floats_cfg<InstCfg>();
template cudaError_t launch_shade_layout_cfg<InstCfg>(const float *, int, int64_t, float *, int, cudaStream_t);
#endif

}  // namespace kns
