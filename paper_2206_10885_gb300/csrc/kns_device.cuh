// kns_device.cuh -- private device-side definitions of the KiloNeuS CUDA library.
//
// Device weight layout (FP32, one block per cell, cell stride a multiple of 32 floats):
//   SDF layer 0:    W0[W][INP]  b0[W]          INP = 3+6L rounded up to 4 (zero pad)
//   SDF layer l:    Wl[W][W]    bl[W]          l = 1..H-1
//   SDF last:       WL[16][W]   bL[16]         row 0 = d, rows 1..15 = feature z
//   colour layer 0: C0[CW][CIN] c0[CW]         CIN = 15 + 3 + (3+6LD) + 3 (x slot; zero when unused)
//   colour last:    C1[4][CW]   c1[4]          row 3 zero
// Rows are 16-byte aligned so a warp that shares a cell reads weights with uniform float4 loads.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kns {

constexpr int FEAT = 15;
constexpr int SDF_OUT = 1 + FEAT;

__host__ __device__ constexpr int round4(int v) { return (v + 3) & ~3; }
__host__ __device__ constexpr int round32(int v) { return (v + 31) & ~31; }

// Compile-time shape of one supported grid configuration.
template <int W_, int H_, int L_, int LD_>
struct Cfg {
    static constexpr int W = W_;    // SDF hidden width (= colour hidden width)
    static constexpr int H = H_;    // SDF hidden layers
    static constexpr int L = L_;    // encoding frequencies of x
    static constexpr int LD = LD_;  // encoding frequencies of the view direction
    static constexpr int IN = 3 + 6 * L;
    static constexpr int INP = round4(IN);
    static constexpr int CIN = FEAT + 3 + (3 + 6 * LD) + 3;
    static constexpr int CINP = round4(CIN);
    // offsets (floats) inside one cell block
    static constexpr int oW0 = 0;
    static constexpr int ob0 = oW0 + W * INP;
    static constexpr int oH1 = ob0 + W;  // start of hidden layer 1
    static constexpr int HSZ = W * W + W;
    __host__ __device__ static constexpr int oWl(int l) { return oH1 + (l - 1) * HSZ; }
    __host__ __device__ static constexpr int obl(int l) { return oH1 + (l - 1) * HSZ + W * W; }
    static constexpr int oWL = oH1 + (H - 1) * HSZ;
    static constexpr int obL = oWL + SDF_OUT * W;
    static constexpr int oC0 = obL + SDF_OUT;
    static constexpr int oc0 = oC0 + W * CINP;
    static constexpr int oC1 = oc0 + W;
    static constexpr int oc1 = oC1 + 4 * W;
    static constexpr int SIZE = round32(oc1 + 4);
    // k-major copy of the SDF trace weights (used by the wavefront tile GEMM):
    //   T0[INP][W] t0[W]  |  Tl[W][W] tl[W] (l = 1..H-1)  |  dL[W] (row 0 of the last layer) bL0 (+3 pad)
    static constexpr int tW0 = 0;
    static constexpr int tb0 = INP * W;
    static constexpr int tH1 = tb0 + W;
    __host__ __device__ static constexpr int tWl(int l) { return tH1 + (l - 1) * HSZ; }
    __host__ __device__ static constexpr int tbl(int l) { return tH1 + (l - 1) * HSZ + W * W; }
    static constexpr int tdL = tH1 + (H - 1) * HSZ;
    static constexpr int tbL = tdL + W;
    static constexpr int TSIZE = round32(tbL + 4);
};

// Everything a kernel needs to read a resident grid (passed by value).
struct GridView {
    const float *w;       // FP32 device layout
    int cell_stride;      // floats per cell block
    int N;                // cells per axis
    float bmin[3], bmax[3];
    float cscale[3];      // N / (bmax - bmin)
    const uint32_t *occ;  // occupancy bits (x-fastest), NULL = no skipping
    int occ_res;
    int occ_per_cell;     // occ_res / N
    float oscale[3];      // occ_res / (bmax - bmin)
    float ovox[3];        // voxel edge (bmax - bmin) / occ_res
    float beta, inv_beta;
    const uint32_t *occ_coarse;  // bit per block of 8^3 voxels: any voxel occupied (NULL = none)
    int cres;                    // blocks per axis (occ_res / 8)
    int olo[3], ohi[3];          // index box of the occupied voxels (inclusive; olo > ohi: none occupied)
    const float *ws;             // shading layout of every cell (kns_shade.cu), one bulk copy per cell
    int ws_stride;               // floats per cell of it
    // A stack of grids of one shape (kns_load_grid_stack) numbers the cells of grid k from k * ncl and keeps
    // the grids' occupancy masks back to back; sub_grid() gives the view of grid k (a single grid: k = 0).
    int cell_base;     // number of this grid's first cell
    int ncl;           // cells of one grid, N^3
    int occ_words;     // 32-bit words of one grid's occupancy mask
    int coarse_words;  // 32-bit words of one grid's coarse mask
    const int *sub_boxes;  // a stack: each grid's index box of occupied voxels (lo xyz, hi xyz); else NULL
};

// The view of grid k of a stack: its cell numbers and occupancy masks (the weights of every grid of the
// stack are indexed by cell number already).
__device__ __forceinline__ GridView sub_grid(const GridView &g, int k) {
    GridView s = g;
    if (k > 0) {
        s.cell_base = k * g.ncl;
        if (s.occ) s.occ += (size_t)k * g.occ_words;
        if (s.occ_coarse) s.occ_coarse += (size_t)k * g.coarse_words;
    }
    if (g.sub_boxes) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            s.olo[a] = __ldg(g.sub_boxes + 6 * k + a);
            s.ohi[a] = __ldg(g.sub_boxes + 6 * k + 3 + a);
        }
    }
    return s;
}

// ------------------------------------------------------------------ activations
__device__ __forceinline__ float softplus_f32(float s, float beta, float inv_beta) {
    // max(s, 0) + log(1 + exp(-beta |s|)) / beta
    float e = __expf(-beta * fabsf(s));
    return fmaxf(s, 0.f) + __logf(1.f + e) * inv_beta;
}
// derivative of softplus_beta: sigmoid(beta s)
__device__ __forceinline__ float dsoftplus_f32(float s, float beta) {
    return 1.f / (1.f + __expf(-beta * s));
}
__device__ __forceinline__ float sigmoid_f32(float s) { return 1.f / (1.f + __expf(-s)); }

// ------------------------------------------------------------------ Eq. 1 encoding
// out[0..2] = p; out[3+6k+c] = sin(2^k pi p_c); out[3+6k+3+c] = cos(2^k pi p_c); zero pad.
template <int L, int NOUT>
__device__ __forceinline__ void encode3(float px, float py, float pz, float (&out)[NOUT]) {
    out[0] = px;
    out[1] = py;
    out[2] = pz;
#pragma unroll
    for (int k = 0; k < L; ++k) {
        const float f = (float)(1 << k);
        float s, c;
        sincospif(f * px, &s, &c);
        out[3 + 6 * k + 0] = s;
        out[3 + 6 * k + 3] = c;
        sincospif(f * py, &s, &c);
        out[3 + 6 * k + 1] = s;
        out[3 + 6 * k + 4] = c;
        sincospif(f * pz, &s, &c);
        out[3 + 6 * k + 2] = s;
        out[3 + 6 * k + 5] = c;
    }
#pragma unroll
    for (int i = 3 + 6 * L; i < NOUT; ++i) out[i] = 0.f;
}

// y = act(W x + b) with W[OUT][IN] row-major (IN % 4 == 0), weights through the read-only path.
template <int IN, int OUT, bool SOFTPLUS>
__device__ __forceinline__ void dense_f32(const float *__restrict__ Wt, const float *__restrict__ bias,
                                          const float (&x)[IN], float (&y)[OUT], float beta, float inv_beta) {
#pragma unroll
    for (int o = 0; o < OUT; ++o) {
        float acc = __ldg(bias + o);
#pragma unroll
        for (int i = 0; i < IN; i += 4) {
            const float4 w4 = __ldg(reinterpret_cast<const float4 *>(Wt + o * IN + i));
            acc = fmaf(w4.x, x[i + 0], acc);
            acc = fmaf(w4.y, x[i + 1], acc);
            acc = fmaf(w4.z, x[i + 2], acc);
            acc = fmaf(w4.w, x[i + 3], acc);
        }
        y[o] = SOFTPLUS ? softplus_f32(acc, beta, inv_beta) : acc;
    }
}

// Trace form of the SDF MLP (Eq. 2): only the d row of the last layer.
template <class C>
__device__ __forceinline__ float sdf_trace_f32(const float *__restrict__ cw, float px, float py, float pz,
                                               float beta, float inv_beta) {
    float in[C::INP];
    encode3<C::L>(px, py, pz, in);
    float h[C::W], g[C::W];
    dense_f32<C::INP, C::W, true>(cw + C::oW0, cw + C::ob0, in, h, beta, inv_beta);
#pragma unroll
    for (int l = 1; l < C::H; ++l) {
        dense_f32<C::W, C::W, true>(cw + C::oWl(l), cw + C::obl(l), h, g, beta, inv_beta);
#pragma unroll
        for (int i = 0; i < C::W; ++i) h[i] = g[i];
    }
    float d = __ldg(cw + C::obL);
#pragma unroll
    for (int i = 0; i < C::W; i += 4) {
        const float4 w4 = __ldg(reinterpret_cast<const float4 *>(cw + C::oWL + i));
        d = fmaf(w4.x, h[i], d);
        d = fmaf(w4.y, h[i + 1], d);
        d = fmaf(w4.z, h[i + 2], d);
        d = fmaf(w4.w, h[i + 3], d);
    }
    return d;
}

// Full form: d, the feature z, and the analytic input gradient by reverse mode (Sec. 3.1).
template <class C>
__device__ __noinline__ float sdf_full_f32(const float *__restrict__ cw, float px, float py, float pz,
                                           float beta, float inv_beta, float (&z)[FEAT], float (&grad)[3]) {
    float in[C::INP];
    encode3<C::L>(px, py, pz, in);
    float dsp[C::H][C::W];  // softplus'(pre-activation) of every hidden unit
    float h[C::W];
    // layer 0
#pragma unroll
    for (int o = 0; o < C::W; ++o) {
        float acc = __ldg(cw + C::ob0 + o);
#pragma unroll
        for (int i = 0; i < C::INP; i += 4) {
            const float4 w4 = __ldg(reinterpret_cast<const float4 *>(cw + C::oW0 + o * C::INP + i));
            acc = fmaf(w4.x, in[i], fmaf(w4.y, in[i + 1], fmaf(w4.z, in[i + 2], fmaf(w4.w, in[i + 3], acc))));
        }
        h[o] = softplus_f32(acc, beta, inv_beta);
        dsp[0][o] = dsoftplus_f32(acc, beta);
    }
#pragma unroll
    for (int l = 1; l < C::H; ++l) {
        float g[C::W];
#pragma unroll
        for (int o = 0; o < C::W; ++o) {
            float acc = __ldg(cw + C::obl(l) + o);
#pragma unroll
            for (int i = 0; i < C::W; i += 4) {
                const float4 w4 = __ldg(reinterpret_cast<const float4 *>(cw + C::oWl(l) + o * C::W + i));
                acc = fmaf(w4.x, h[i], fmaf(w4.y, h[i + 1], fmaf(w4.z, h[i + 2], fmaf(w4.w, h[i + 3], acc))));
            }
            g[o] = softplus_f32(acc, beta, inv_beta);
            dsp[l][o] = dsoftplus_f32(acc, beta);
        }
#pragma unroll
        for (int i = 0; i < C::W; ++i) h[i] = g[i];
    }
    float out[SDF_OUT];
#pragma unroll
    for (int o = 0; o < SDF_OUT; ++o) {
        float acc = __ldg(cw + C::obL + o);
#pragma unroll
        for (int i = 0; i < C::W; i += 4) {
            const float4 w4 = __ldg(reinterpret_cast<const float4 *>(cw + C::oWL + o * C::W + i));
            acc = fmaf(w4.x, h[i], fmaf(w4.y, h[i + 1], fmaf(w4.z, h[i + 2], fmaf(w4.w, h[i + 3], acc))));
        }
        out[o] = acc;
    }
#pragma unroll
    for (int k = 0; k < FEAT; ++k) z[k] = out[1 + k];
    // reverse mode: delta = dd/dh of the last hidden layer = row 0 of WL
    float delta[C::W];
#pragma unroll
    for (int i = 0; i < C::W; ++i) delta[i] = __ldg(cw + C::oWL + i);
#pragma unroll
    for (int l = C::H - 1; l >= 1; --l) {
        float nd[C::W];
#pragma unroll
        for (int i = 0; i < C::W; ++i) nd[i] = 0.f;
#pragma unroll
        for (int o = 0; o < C::W; ++o) {
            const float dl = delta[o] * dsp[l][o];
#pragma unroll
            for (int i = 0; i < C::W; i += 4) {
                const float4 w4 = __ldg(reinterpret_cast<const float4 *>(cw + C::oWl(l) + o * C::W + i));
                nd[i] = fmaf(w4.x, dl, nd[i]);
                nd[i + 1] = fmaf(w4.y, dl, nd[i + 1]);
                nd[i + 2] = fmaf(w4.z, dl, nd[i + 2]);
                nd[i + 3] = fmaf(w4.w, dl, nd[i + 3]);
            }
        }
#pragma unroll
        for (int i = 0; i < C::W; ++i) delta[i] = nd[i];
    }
    float din[C::INP];
#pragma unroll
    for (int i = 0; i < C::INP; ++i) din[i] = 0.f;
#pragma unroll
    for (int o = 0; o < C::W; ++o) {
        const float dl = delta[o] * dsp[0][o];
#pragma unroll
        for (int i = 0; i < C::INP; i += 4) {
            const float4 w4 = __ldg(reinterpret_cast<const float4 *>(cw + C::oW0 + o * C::INP + i));
            din[i] = fmaf(w4.x, dl, din[i]);
            din[i + 1] = fmaf(w4.y, dl, din[i + 1]);
            din[i + 2] = fmaf(w4.z, dl, din[i + 2]);
            din[i + 3] = fmaf(w4.w, dl, din[i + 3]);
        }
    }
    // through the encoding: d sin(f p)/dp = f cos(f p), d cos(f p)/dp = -f sin(f p)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float gc = din[c];
#pragma unroll
        for (int k = 0; k < C::L; ++k) {
            const float f = 3.14159265358979323846f * (float)(1 << k);
            gc = fmaf(din[3 + 6 * k + c] * f, in[3 + 6 * k + 3 + c], gc);
            gc = fmaf(-din[3 + 6 * k + 3 + c] * f, in[3 + 6 * k + c], gc);
        }
        grad[c] = gc;
    }
    return out[0];
}

// Colour MLP (Eq. 3): u = [z, n, gamma_LD(v), x] -> ReLU(W) -> 3 -> sigmoid.
template <class C>
__device__ __noinline__ void colour_f32(const float *__restrict__ cw, const float (&z)[FEAT], const float (&n)[3],
                                        float vx, float vy, float vz, float px, float py, float pz,
                                        float (&rgb)[3]) {
    float u[C::CINP];
#pragma unroll
    for (int k = 0; k < FEAT; ++k) u[k] = z[k];
    u[FEAT + 0] = n[0];
    u[FEAT + 1] = n[1];
    u[FEAT + 2] = n[2];
    float gv[3 + 6 * C::LD];
    encode3<C::LD>(vx, vy, vz, gv);
#pragma unroll
    for (int k = 0; k < 3 + 6 * C::LD; ++k) u[FEAT + 3 + k] = gv[k];
    u[C::CIN - 3] = px;
    u[C::CIN - 2] = py;
    u[C::CIN - 1] = pz;
#pragma unroll
    for (int i = C::CIN; i < C::CINP; ++i) u[i] = 0.f;
    float h[C::W];
#pragma unroll
    for (int o = 0; o < C::W; ++o) {
        float acc = __ldg(cw + C::oc0 + o);
#pragma unroll
        for (int i = 0; i < C::CINP; i += 4) {
            const float4 w4 = __ldg(reinterpret_cast<const float4 *>(cw + C::oC0 + o * C::CINP + i));
            acc = fmaf(w4.x, u[i], fmaf(w4.y, u[i + 1], fmaf(w4.z, u[i + 2], fmaf(w4.w, u[i + 3], acc))));
        }
        h[o] = fmaxf(acc, 0.f);
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        float acc = __ldg(cw + C::oc1 + r);
#pragma unroll
        for (int i = 0; i < C::W; i += 4) {
            const float4 w4 = __ldg(reinterpret_cast<const float4 *>(cw + C::oC1 + r * C::W + i));
            acc = fmaf(w4.x, h[i], fmaf(w4.y, h[i + 1], fmaf(w4.z, h[i + 2], fmaf(w4.w, h[i + 3], acc))));
        }
        rgb[r] = sigmoid_f32(acc);
    }
}

// ------------------------------------------------------------------ cell map m(x) (Sec. 3.1)
__device__ __forceinline__ int grid_axis(float x, float bmin, float scale, int res) {
    float u = floorf((x - bmin) * scale);
    u = fminf(fmaxf(u, 0.f), (float)(res - 1));
    return (int)u;
}
__device__ __forceinline__ int cell_of(const GridView &g, float x, float y, float z) {
    const int ix = grid_axis(x, g.bmin[0], g.cscale[0], g.N);
    const int iy = grid_axis(y, g.bmin[1], g.cscale[1], g.N);
    const int iz = grid_axis(z, g.bmin[2], g.cscale[2], g.N);
    return g.cell_base + ix + g.N * (iy + g.N * iz);
}

__device__ __forceinline__ bool occ_test(const uint32_t *__restrict__ occ, int res, int ix, int iy, int iz) {
    const unsigned v = (unsigned)ix + (unsigned)res * ((unsigned)iy + (unsigned)res * (unsigned)iz);
    return (__ldg(occ + (v >> 5)) >> (v & 31u)) & 1u;
}

// ------------------------------------------------------------------ rays
struct Ray {
    float ox, oy, oz, wx, wy, wz;
};

// Pixel (i, j) of camera cam (16 floats: c2w 3x4 row-major, fx, fy, cx, cy).
__device__ __forceinline__ Ray make_ray(const float *cam, int i, int j) {
    const float dx = ((float)j + 0.5f - cam[14]) / cam[12];
    const float dy = ((float)i + 0.5f - cam[15]) / cam[13];
    float wx = fmaf(cam[0], dx, fmaf(cam[1], dy, cam[2]));
    float wy = fmaf(cam[4], dx, fmaf(cam[5], dy, cam[6]));
    float wz = fmaf(cam[8], dx, fmaf(cam[9], dy, cam[10]));
    const float inv = 1.f / sqrtf(fmaf(wx, wx, fmaf(wy, wy, wz * wz)));
    Ray r;
    r.wx = wx * inv;
    r.wy = wy * inv;
    r.wz = wz * inv;
    r.ox = cam[3];
    r.oy = cam[7];
    r.oz = cam[11];
    return r;
}

// Slab test against the grid box; on overlap returns true with t0 = max(t_near, 0) and tf = t_far.
__device__ __forceinline__ bool clip_box(const GridView &g, const Ray &r, float &t0, float &tf) {
    float a = -INFINITY, b = INFINITY;
    const float o[3] = {r.ox, r.oy, r.oz}, w[3] = {r.wx, r.wy, r.wz};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (w[k] != 0.f) {
            const float t1 = (g.bmin[k] - o[k]) / w[k], t2 = (g.bmax[k] - o[k]) / w[k];
            a = fmaxf(a, fminf(t1, t2));
            b = fminf(b, fmaxf(t1, t2));
        } else if (o[k] < g.bmin[k] || o[k] > g.bmax[k]) {
            return false;
        }
    }
    if (a > b || b < 0.f) return false;
    t0 = fmaxf(a, 0.f);
    tf = b;
    return true;
}

// Crossing parameter of a voxel face on one axis: (face - o) times 1/w (inv_w, computed once per
// walk), the face coordinate exact; a ray parallel to the axis never crosses.
__device__ __forceinline__ float dda_face_t(float bmin, int v, bool up, float vox, float o, float inv_w) {
    return isinf(inv_w) ? INFINITY : (bmin + (float)(v + (up ? 1 : 0)) * vox - o) * inv_w;
}
__device__ __forceinline__ bool coarse_empty(const GridView &g, int vx, int vy, int vz) {
    if (!g.occ_coarse) return false;
    return !occ_test(g.occ_coarse, g.cres, vx >> 3, vy >> 3, vz >> 3);
}

// Fine voxel index along one axis at parameter t, or -1 when x(t) lies within 1e-3 voxel of a
// voxel face (where rounding could disagree with the face-by-face walk).
__device__ __forceinline__ int unambiguous_index(float o, float w, float t, float bmin, float scale, int res) {
    const float u = (fmaf(t, w, o) - bmin) * scale;
    const float f = floorf(u);
    if (u - f < 1e-3f || f + 1.f - u < 1e-3f) return -1;
    return (int)fminf(fmaxf(f, 0.f), (float)(res - 1));
}

// Outside the index box [olo, ohi] of the occupied voxels every voxel is empty, so the walk from a voxel
// outside it either never finds an occupied voxel -- the ray is outside the box on an axis and moving
// away from it (or parallel to it), or it leaves one of the box's slabs before it has entered all
// three -- or crosses empty voxels up to the box's entry face.  Returns 0: the walk ends without an
// occupied voxel; 1: (vx, vy, vz, T) is the voxel the walk enters the box in and the parameter of that
// crossing (the entry axis' index is the box's first layer; the other two are taken from the position
// at T, as for a coarse block's exit); 2: walk on from where the ray is (inside the box, or an entry
// within 1e-3 voxel of another face, which the voxel walk settles).
__device__ __forceinline__ int occ_box_entry(const GridView &g, const Ray &r, int &vx, int &vy, int &vz, float ix,
                                             float iy, float iz, float &T) {
    const int v[3] = {vx, vy, vz};
    const float w[3] = {r.wx, r.wy, r.wz}, o[3] = {r.ox, r.oy, r.oz}, inv[3] = {ix, iy, iz};
    if (v[0] >= g.olo[0] && v[0] <= g.ohi[0] && v[1] >= g.olo[1] && v[1] <= g.ohi[1] && v[2] >= g.olo[2] &&
        v[2] <= g.ohi[2])
        return 2;
    if (g.olo[0] > g.ohi[0]) return 0;  // no voxel is occupied
    float t_in = -INFINITY, t_out = INFINITY;
    int ax = -1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const bool up = w[k] > 0.f, still = isinf(inv[k]);
        if ((v[k] < g.olo[k] && (!up || still)) || (v[k] > g.ohi[k] && (up || still))) return 0;
        if (still) continue;
        // the crossing into the box's first layer on this axis (when outside it), and out of its last
        if (v[k] < g.olo[k] || v[k] > g.ohi[k]) {
            const float t = up ? dda_face_t(g.bmin[k], g.olo[k] - 1, true, g.ovox[k], o[k], inv[k])
                               : dda_face_t(g.bmin[k], g.ohi[k] + 1, false, g.ovox[k], o[k], inv[k]);
            if (t > t_in) {
                t_in = t;
                ax = k;
            }
        }
        t_out = fminf(t_out, up ? dda_face_t(g.bmin[k], g.ohi[k], true, g.ovox[k], o[k], inv[k])
                                : dda_face_t(g.bmin[k], g.olo[k], false, g.ovox[k], o[k], inv[k]));
    }
    if (t_in > t_out) return 0;  // it leaves a slab of the box before it has entered the others
    int n[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (k == ax) {
            n[k] = w[k] > 0.f ? g.olo[k] : g.ohi[k];
        } else {
            const float bm = g.bmin[k], sc = g.oscale[k];
            n[k] = unambiguous_index(o[k], w[k], t_in, bm, sc, g.occ_res);
            if (n[k] < g.olo[k] || n[k] > g.ohi[k]) return 2;  // ambiguous (or fuzzy): walk
        }
    }
    vx = n[0];
    vy = n[1];
    vz = n[2];
    T = t_in;
    return 1;
}

// Integer 3D-DDA (Amanatides & Woo) from voxel (vx, vy, vz) to the entry of the next occupied voxel.
// Returns true with te and the voxel updated; false when the ray leaves the grid or passes tf.
// The crossing parameter of each axis is (face - o) / w (dda_face_t, by the reciprocal of w); after
// a step only the crossed axis' value changes, so only it is recomputed.  Blocks of 8^3 voxels that
// the coarse mask marks empty are crossed in one step: the exit face is found among the block's
// faces with the same formula and tie rule, and the other two voxel indices at the exit are taken
// from the position there unless it lies within 1e-3 voxel of a face, in which case the block is
// walked voxel by voxel.  Outside the index box of the occupied voxels the walk jumps to the box's
// entry, or ends when the ray cannot reach the box (occ_box_entry).  Either way the voxel and parameter
// reached are those of the voxel walk.
__device__ __forceinline__ bool dda_next(const GridView &g, const Ray &r, int &vx, int &vy, int &vz, float tf,
                                         float &te) {
    const int res = g.occ_res;
    const bool ux = r.wx > 0.f, uy = r.wy > 0.f, uz = r.wz > 0.f;
    const float ix = 1.f / r.wx, iy = 1.f / r.wy, iz = 1.f / r.wz;
    float tx = dda_face_t(g.bmin[0], vx, ux, g.ovox[0], r.ox, ix);
    float ty = dda_face_t(g.bmin[1], vy, uy, g.ovox[1], r.oy, iy);
    float tz = dda_face_t(g.bmin[2], vz, uz, g.ovox[2], r.oz, iz);
    // at most 3*res voxel crossings before the ray leaves the grid
    for (int guard = 0; guard < 3 * res + 3; ++guard) {
        float Tb;
        const int ob = occ_box_entry(g, r, vx, vy, vz, ix, iy, iz, Tb);
        if (ob == 0) return false;
        if (ob == 1) {  // crossed the empty space up to the occupied voxels' box
            if (Tb > tf) return false;
            if (occ_test(g.occ, res, vx, vy, vz)) {
                te = Tb;
                return true;
            }
            tx = dda_face_t(g.bmin[0], vx, ux, g.ovox[0], r.ox, ix);
            ty = dda_face_t(g.bmin[1], vy, uy, g.ovox[1], r.oy, iy);
            tz = dda_face_t(g.bmin[2], vz, uz, g.ovox[2], r.oz, iz);
            continue;
        }
        if (coarse_empty(g, vx, vy, vz)) {
            // the last voxel of this block along each axis in the direction of travel
            const int bx = ux ? (vx | 7) : (vx & ~7), by = uy ? (vy | 7) : (vy & ~7), bz = uz ? (vz | 7) : (vz & ~7);
            const float Tx = dda_face_t(g.bmin[0], bx, ux, g.ovox[0], r.ox, ix);
            const float Ty = dda_face_t(g.bmin[1], by, uy, g.ovox[1], r.oy, iy);
            const float Tz = dda_face_t(g.bmin[2], bz, uz, g.ovox[2], r.oz, iz);
            int nx, ny, nz, va;
            float T;
            if (Tx <= Ty && Tx <= Tz) {
                T = Tx;
                nx = bx + (ux ? 1 : -1);
                ny = unambiguous_index(r.oy, r.wy, T, g.bmin[1], g.oscale[1], res);
                nz = unambiguous_index(r.oz, r.wz, T, g.bmin[2], g.oscale[2], res);
                va = nx;
            } else if (Ty <= Tz) {
                T = Ty;
                ny = by + (uy ? 1 : -1);
                nx = unambiguous_index(r.ox, r.wx, T, g.bmin[0], g.oscale[0], res);
                nz = unambiguous_index(r.oz, r.wz, T, g.bmin[2], g.oscale[2], res);
                va = ny;
            } else {
                T = Tz;
                nz = bz + (uz ? 1 : -1);
                nx = unambiguous_index(r.ox, r.wx, T, g.bmin[0], g.oscale[0], res);
                ny = unambiguous_index(r.oy, r.wy, T, g.bmin[1], g.oscale[1], res);
                va = nz;
            }
            if (nx >= 0 && ny >= 0 && nz >= 0) {
                if (va < 0 || va >= res) return false;  // left the grid inside empty space
                if (T > tf) return false;
                vx = nx;
                vy = ny;
                vz = nz;
                if (occ_test(g.occ, res, vx, vy, vz)) {
                    te = T;
                    return true;
                }
                tx = dda_face_t(g.bmin[0], vx, ux, g.ovox[0], r.ox, ix);
                ty = dda_face_t(g.bmin[1], vy, uy, g.ovox[1], r.oy, iy);
                tz = dda_face_t(g.bmin[2], vz, uz, g.ovox[2], r.oz, iz);
                continue;
            }
            // ambiguous exit: walk this block voxel by voxel
        }
        float tm;
        int va;
        if (tx <= ty && tx <= tz) {  // ties go to the lowest axis
            tm = tx;
            vx += ux ? 1 : -1;
            va = vx;
            tx = dda_face_t(g.bmin[0], vx, ux, g.ovox[0], r.ox, ix);
        } else if (ty <= tz) {
            tm = ty;
            vy += uy ? 1 : -1;
            va = vy;
            ty = dda_face_t(g.bmin[1], vy, uy, g.ovox[1], r.oy, iy);
        } else {
            tm = tz;
            vz += uz ? 1 : -1;
            va = vz;
            tz = dda_face_t(g.bmin[2], vz, uz, g.ovox[2], r.oz, iz);
        }
        if (va < 0 || va >= res) return false;
        if (tm > tf) return false;
        if (occ_test(g.occ, res, vx, vy, vz)) {
            te = tm;
            return true;
        }
    }
    return false;
}

}  // namespace kns
