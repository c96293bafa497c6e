// kns_fp32.cu -- FP32 CUDA-core kernels: batch field query (Sec. 3.3's per-cell MLP query) and the
// occupancy-mask build.  One thread per point / voxel; the per-thread MLP evaluators live in
// kns_device.cuh.
// kns:instantiate (compiled once per grid configuration)
#include "kns_wave.cuh"

namespace kns {

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
        const int cell = g.cell_base + ix / f + g.N * (iy / f + g.N * (iz / f));
        const float d = sdf_trace_f32<C>(g.w + (int64_t)cell * g.cell_stride, x, y, z, g.beta, g.inv_beta);
        occ = fabsf(d) < thresh;
    }
    const unsigned ball = __ballot_sync(0xffffffffu, occ);
    if ((threadIdx.x & 31) == 0 && v < nvox) words[v >> 5] = ball;
}

// FP32 refinement of a BF16 render's unconfirmed hits (Sec. 3.4.1's steps, in FP32): the shading's
// evaluation at t was the first FP32 evaluation; up to refine_steps in all, a hit at the first
// |d| < eps or at the last if |d| < eps_coarse there, otherwise a miss; a hit is then shaded here
// (full SDF, analytic normal, colour MLP).  One thread per ray: the list is short (the BF16 trace is
// accurate to ~1e-5, so most hits are confirmed at once).
template <class C>
__global__ void __launch_bounds__(128) refine_kernel(GridView g, WaveArgs a) {
    const int n = a.ctrl->n_refine;
    unsigned n_eval = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int r = a.pend_r[0][i];
        float d = a.pend_t[0][i];
        float t = a.t_ray[r];
        int steps = a.steps_ray[r], cell = a.cell_ray[r];
        int cam;
        const Ray ray = ray_of(a, r, cam);
        const GridView gv = sub_grid(g, a.views[cam].grid);  // the ray's grid (a stack of grids)
        float t0, tf;
        clip_box(gv, ray, t0, tf);
        bool hit = false;
        for (int ev = 1;; ++ev) {
            if (fabsf(d) < a.eps) {
                hit = true;
                break;
            }
            if (ev >= a.refine_steps) {
                hit = fabsf(d) < a.eps_coarse;
                break;
            }
            t += d;
            if (t > tf || t < t0 || steps >= a.max_steps) break;
            cell = advance_ray(gv, ray, t, tf);
            if (cell < 0) break;
            d = sdf_trace_f32<C>(g.w + (int64_t)cell * g.cell_stride, fmaf(t, ray.wx, ray.ox), fmaf(t, ray.wy, ray.oy),
                                 fmaf(t, ray.wz, ray.oz), g.beta, g.inv_beta);
            ++steps;
            ++n_eval;
        }
        if (!hit) {
            write_miss(a, r, steps);
            continue;
        }
        const float px = fmaf(t, ray.wx, ray.ox), py = fmaf(t, ray.wy, ray.oy), pz = fmaf(t, ray.wz, ray.oz);
        const float *cw = g.w + (int64_t)cell * g.cell_stride;
        float z[FEAT], gr[3], rgb[3];
        sdf_full_f32<C>(cw, px, py, pz, g.beta, g.inv_beta, z, gr);
        const float gn = sqrtf(fmaf(gr[0], gr[0], fmaf(gr[1], gr[1], gr[2] * gr[2])));
        const float inv = gn > 0.f ? 1.f / gn : 0.f;
        const float nrm[3] = {gr[0] * inv, gr[1] * inv, gr[2] * inv};
        colour_f32<C>(cw, z, nrm, ray.wx, ray.wy, ray.wz, px, py, pz, rgb);
        const ViewDev &V = a.views[cam];
        const int64_t p = r - V.ray_base;
        V.rgb[3 * p + 0] = rgb[0];
        V.rgb[3 * p + 1] = rgb[1];
        V.rgb[3 * p + 2] = rgb[2];
        V.depth[p] = t;
        if (V.normal) {
            V.normal[3 * p + 0] = nrm[0];
            V.normal[3 * p + 1] = nrm[1];
            V.normal[3 * p + 2] = nrm[2];
        }
        if (V.cell) V.cell[p] = cell - gv.cell_base;  // the cell within the view's grid
        if (V.steps) V.steps[p] = steps;
        if (V.hit) V.hit[p] = 1;
    }
    const unsigned long long ne = warp_sum_u64(n_eval);
    if ((threadIdx.x & 31) == 0 && ne) atomicAdd(&a.ctrl->samples_f32, ne);
}

// ------------------------------------------------------------------ launchers
template <class C>
cudaError_t launch_refine_cfg(const GridView &g, const WaveArgs &a, int sm_count, cudaStream_t s) {
    refine_kernel<C><<<sm_count, 128, 0, s>>>(g, a);
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
template cudaError_t launch_sdf_cfg<InstCfg>(const GridView &, const float *, int64_t, float *, float *, float *,
                                             cudaStream_t);
template cudaError_t launch_occ_cfg<InstCfg>(const GridView &, float, uint32_t *, cudaStream_t);
template cudaError_t launch_refine_cfg<InstCfg>(const GridView &, const WaveArgs &, int, cudaStream_t);
#endif

}  // namespace kns
