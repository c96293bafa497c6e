// kns_fp32.cu -- FP32 CUDA-core kernels: sphere-traced render, batch field query, occupancy build.
//
// Render (Sec. 3.4.1): one thread per ray; a warp covers an 8x4 pixel tile so that the rays of a
// warp usually share their cell and read the cell's weights with uniform (broadcast) loads.  Each
// thread loops: cell lookup m(x) (Sec. 3.1), optional empty-space skip (occupancy bit test, then an
// integer DDA to the next occupied voxel), the SDF MLP of Eq. 2 in trace form (d only), the hit
// test |d| < eps and the step t += d.  Hit rays then evaluate the full SDF MLP with its reverse-mode
// input gradient (normal) and the colour MLP of Eq. 3 together, after every lane of the warp has
// finished tracing, so the hit epilogue runs once per warp instead of once per step.
// kns:instantiate (compiled once per grid configuration)
#include "kns_device.cuh"
#include "kns_kernels.h"

namespace kns {

template <class C>
__global__ void __launch_bounds__(128) render_f32_kernel(GridView g, CamBatch cams, RenderArgs a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = blockIdx.x * 16 + (warp & 1) * 8 + (lane & 7);
    const int i = blockIdx.y * 8 + (warp >> 1) * 4 + (lane >> 3);
    const int cam = blockIdx.z;
    if (i >= a.H || j >= a.W) return;
    const int64_t p = (int64_t)(a.cam_base + cam) * a.H * a.W + (int64_t)i * a.W + j;
    const Ray r = make_ray(cams.c[cam], i, j);

    int steps = 0, hit_cell = -1;
    float t = 0.f, tf = 0.f;
    bool hit = false;
    float t_lo = 0.f;
    if (clip_box(g, r, t_lo, tf)) {
        t = t_lo;
        for (int k = 0; k < a.max_steps; ++k) {
            float x = fmaf(t, r.wx, r.ox), y = fmaf(t, r.wy, r.oy), z = fmaf(t, r.wz, r.oz);
            int cell;
            if (g.occ) {
                int v[3] = {grid_axis(x, g.bmin[0], g.oscale[0], g.occ_res),
                            grid_axis(y, g.bmin[1], g.oscale[1], g.occ_res),
                            grid_axis(z, g.bmin[2], g.oscale[2], g.occ_res)};
                if (!occ_test(g.occ, g.occ_res, v[0], v[1], v[2])) {
                    float te;
                    if (!dda_next(g, r, v, tf, te)) break;
                    // evaluate on the entry face; the entered voxel fixes the cell exactly
                    t = te;
                    x = fmaf(t, r.wx, r.ox);
                    y = fmaf(t, r.wy, r.oy);
                    z = fmaf(t, r.wz, r.oz);
                    const int f = g.occ_per_cell;
                    cell = v[0] / f + g.N * (v[1] / f + g.N * (v[2] / f));
                } else {
                    cell = cell_of(g, x, y, z);
                }
            } else {
                cell = cell_of(g, x, y, z);
            }
            const float d = sdf_trace_f32<C>(g.w + (int64_t)cell * g.cell_stride, x, y, z, g.beta, g.inv_beta);
            ++steps;
            if (fabsf(d) < a.eps) {
                hit = true;
                hit_cell = cell;
                break;
            }
            t += d;
            if (t > tf || t < t_lo) break;
        }
    }

    float rgb[3] = {0.f, 0.f, 0.f}, nrm[3] = {0.f, 0.f, 0.f};
    if (hit) {
        const float x = fmaf(t, r.wx, r.ox), y = fmaf(t, r.wy, r.oy), z = fmaf(t, r.wz, r.oz);
        const float *cw = g.w + (int64_t)hit_cell * g.cell_stride;
        float feat[FEAT], grad[3];
        sdf_full_f32<C>(cw, x, y, z, g.beta, g.inv_beta, feat, grad);
        const float gn = sqrtf(fmaf(grad[0], grad[0], fmaf(grad[1], grad[1], grad[2] * grad[2])));
        const float inv = gn > 0.f ? 1.f / gn : 0.f;
        nrm[0] = grad[0] * inv;
        nrm[1] = grad[1] * inv;
        nrm[2] = grad[2] * inv;
        colour_f32<C>(cw, feat, nrm, r.wx, r.wy, r.wz, x, y, z, rgb);
    }
    a.rgb[3 * p + 0] = rgb[0];
    a.rgb[3 * p + 1] = rgb[1];
    a.rgb[3 * p + 2] = rgb[2];
    a.depth[p] = hit ? t : INFINITY;
    if (a.normal) {
        a.normal[3 * p + 0] = nrm[0];
        a.normal[3 * p + 1] = nrm[1];
        a.normal[3 * p + 2] = nrm[2];
    }
    if (a.cell) a.cell[p] = hit_cell;
    if (a.steps) a.steps[p] = steps;
    if (a.hit) a.hit[p] = hit ? 1 : 0;
}

// Batch field query: d, z and grad d of cell m(x) at each point.
template <class C>
__global__ void __launch_bounds__(128) sdf_batch_kernel(GridView g, const float *__restrict__ pts, int64_t n,
                                                        float *sdf, float *feat, float *grad) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float x = pts[3 * q], y = pts[3 * q + 1], z = pts[3 * q + 2];
    const int cell = cell_of(g, x, y, z);
    const float *cw = g.w + (int64_t)cell * g.cell_stride;
    float zf[FEAT], gr[3];
    const float d = sdf_full_f32<C>(cw, x, y, z, g.beta, g.inv_beta, zf, gr);
    sdf[q] = d;
    if (feat)
        for (int k = 0; k < FEAT; ++k) feat[q * FEAT + k] = zf[k];
    if (grad) {
        grad[3 * q] = gr[0];
        grad[3 * q + 1] = gr[1];
        grad[3 * q + 2] = gr[2];
    }
}

// Occupancy: voxel v is occupied iff |d(centre of v)| < thresh; the voxel's cell is exact
// (voxels nest inside cells).  One thread per voxel, x fastest; a warp writes one 32-bit word.
template <class C>
__global__ void __launch_bounds__(128) occupancy_kernel(GridView g, float thresh, uint32_t *words) {
    const int res = g.occ_res;
    const int64_t nvox = (int64_t)res * res * res;
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool occ = false;
    if (v < nvox) {
        const int ix = (int)(v % res), iy = (int)((v / res) % res), iz = (int)(v / ((int64_t)res * res));
        const float x = g.bmin[0] + ((float)ix + 0.5f) * g.ovox[0];
        const float y = g.bmin[1] + ((float)iy + 0.5f) * g.ovox[1];
        const float z = g.bmin[2] + ((float)iz + 0.5f) * g.ovox[2];
        const int f = g.occ_per_cell;
        const int cell = ix / f + g.N * (iy / f + g.N * (iz / f));
        const float d = sdf_trace_f32<C>(g.w + (int64_t)cell * g.cell_stride, x, y, z, g.beta, g.inv_beta);
        occ = fabsf(d) < thresh;
    }
    const unsigned ball = __ballot_sync(0xffffffffu, occ);
    if ((threadIdx.x & 31) == 0 && v < nvox) words[v >> 5] = ball;
}

// ------------------------------------------------------------------ launchers
template <class C>
cudaError_t launch_render_cfg(const GridView &g, const CamBatch &cams, int n_cams, const RenderArgs &a,
                              cudaStream_t s) {
    dim3 grid((a.W + 15) / 16, (a.H + 7) / 8, n_cams);
    render_f32_kernel<C><<<grid, 128, 0, s>>>(g, cams, a);
    return cudaGetLastError();
}
template <class C>
cudaError_t launch_sdf_cfg(const GridView &g, const float *pts, int64_t n, float *sdf, float *feat, float *grad,
                           cudaStream_t s) {
    const int64_t blocks = (n + 127) / 128;
    sdf_batch_kernel<C><<<(unsigned)blocks, 128, 0, s>>>(g, pts, n, sdf, feat, grad);
    return cudaGetLastError();
}
template <class C>
cudaError_t launch_occ_cfg(const GridView &g, float thresh, uint32_t *words, cudaStream_t s) {
    const int64_t nvox = (int64_t)g.occ_res * g.occ_res * g.occ_res;
    occupancy_kernel<C><<<(unsigned)((nvox + 127) / 128), 128, 0, s>>>(g, thresh, words);
    return cudaGetLastError();
}

// One object file per grid configuration: the build compiles this file once per (W, H, L, LD).
#ifdef KNS_W
using InstCfg = Cfg<KNS_W, KNS_H, KNS_L, KNS_LD>;
template cudaError_t launch_render_cfg<InstCfg>(const GridView &, const CamBatch &, int, const RenderArgs &,
                                                cudaStream_t);
template cudaError_t launch_sdf_cfg<InstCfg>(const GridView &, const float *, int64_t, float *, float *, float *,
                                             cudaStream_t);
template cudaError_t launch_occ_cfg<InstCfg>(const GridView &, float, uint32_t *, cudaStream_t);
#endif

}  // namespace kns
