// kns_wave.cuh -- wavefront sphere tracing: shared state, ray advance, warp-aggregated queues.
//
// One render is a sequence of waves.  Wave k holds every ray that still needs its k-th SDF
// evaluation.  Per wave:
//   sort:  counting sort of the wave's samples by cell (histogram built while the samples were
//          emitted, one exclusive scan over the N^3 cells, a scatter into cell order);
//   eval:  each warp takes a tile of up to 16 samples of one cell and evaluates the cell's SDF
//          MLP (Eq. 2) for all of them at once (a small GEMM per layer), then updates each ray:
//          hit test |d| < eps, step t += d, interval and budget checks, and the advance to its
//          next sample (cell lookup m(x), occupancy skip) which it emits into wave k+1.
// Hits are shaded after the last wave (normal from the analytic gradient, colour MLP of Eq. 3).
#pragma once

#include "kns_device.cuh"
#include "kns_kernels.h"

namespace kns {

constexpr int TILE = 16;  // samples per warp tile
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Appends the predicated lanes of a warp to a queue; returns this lane's slot (or -1).
// Must be called by all 32 lanes.
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned v) {
    unsigned long long x = v;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    return x;
}
__device__ __forceinline__ int warp_append(int *counter, bool pred) {
    const unsigned m = __ballot_sync(FULL, pred);
    if (!m) return -1;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(counter, __popc(m));
    base = __shfl_sync(FULL, base, leader);
    return pred ? base + __popc(m & lanemask_lt()) : -1;
}

// Adds one to count[cell] for each predicated lane, one atomic per distinct cell in the warp.
__device__ __forceinline__ void warp_count_cells(int *count, bool pred, int cell) {
    const unsigned m = __ballot_sync(FULL, pred);
    if (pred) {
        const unsigned grp = __match_any_sync(m, cell);
        if ((threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(count + cell, __popc(grp));
    }
}

// ---------------------------------------------------------------- TMA bulk copy + mbarrier
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// One 1-D bulk copy global -> shared (TMA engine), completion counted in bytes on the mbarrier.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// Waits for the phase with the given parity to complete; gives up after max_polls polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t max_polls) {
    for (uint32_t i = 0; i < max_polls; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// The ray with id r: its view v, pixel index in the view, and world-space origin and direction (a
// camera pixel, or row r of the explicit ray table).
__device__ __forceinline__ Ray table_ray(const WaveArgs &a, int r) {
    Ray ray;
    ray.ox = __ldg(a.ray_o + 3 * r);
    ray.oy = __ldg(a.ray_o + 3 * r + 1);
    ray.oz = __ldg(a.ray_o + 3 * r + 2);
    ray.wx = __ldg(a.ray_w + 3 * r);
    ray.wy = __ldg(a.ray_w + 3 * r + 1);
    ray.wz = __ldg(a.ray_w + 3 * r + 2);
    return ray;
}

__device__ __forceinline__ Ray ray_of(const WaveArgs &a, int r, int &v) {
    v = a.ray_view[r];
    if (a.ray_o) return table_ray(a, r);
    const ViewDev &V = a.views[v];
    const int pix = r - V.ray_base;
    const int i = pix / V.W, j = pix - i * V.W;
    return make_ray(V.cam, i, j);
}

__device__ __forceinline__ void write_miss(const WaveArgs &a, int r, int steps) {
    const ViewDev &V = a.views[a.ray_view[r]];
    const int64_t p = r - V.ray_base;
    V.rgb[3 * p + 0] = 0.f;
    V.rgb[3 * p + 1] = 0.f;
    V.rgb[3 * p + 2] = 0.f;
    V.depth[p] = INFINITY;
    if (V.normal) {
        V.normal[3 * p + 0] = 0.f;
        V.normal[3 * p + 1] = 0.f;
        V.normal[3 * p + 2] = 0.f;
    }
    if (V.cell) V.cell[p] = -1;
    if (V.steps) V.steps[p] = steps;
    if (V.hit) V.hit[p] = 0;
}

// Cycle test.  A ray's next sample position is a deterministic function of its current position
// (the cell's d, the step, the occupancy skip), so a ray whose next position t_next equals one it
// evaluated before repeats those evaluations for ever: none of them met |d| < eps or left the
// interval, so the ray ends as a miss when its step budget runs out, with steps = max_steps.  hist
// holds the four positions evaluated before t_eval (newest first; NaN where none): a match finds
// cycles of period 2 to 5.  Returns true for a cycle; otherwise shifts t_eval into hist.
__device__ __forceinline__ bool cycle_step(float4 &hist, float t_eval, float t_next) {
    if (t_next == hist.x || t_next == hist.y || t_next == hist.z || t_next == hist.w) return true;
    hist = make_float4(t_eval, hist.x, hist.y, hist.z);
    return false;
}
__device__ __forceinline__ float4 no_history() { return make_float4(NAN, NAN, NAN, NAN); }

// Moves a ray at parameter t to its next sample: the cell at x(t), or, when x(t) lies in an empty
// occupancy voxel, the entry face of the next occupied voxel (t moves there; the voxel fixes the
// cell exactly).  Returns the cell, or -1 when the ray leaves the grid (a miss).
__device__ __forceinline__ int advance_ray(const GridView &g, const Ray &r, float &t, float tf) {
    const float x = fmaf(t, r.wx, r.ox), y = fmaf(t, r.wy, r.oy), z = fmaf(t, r.wz, r.oz);
    if (g.occ) {
        int vx = grid_axis(x, g.bmin[0], g.oscale[0], g.occ_res), vy = grid_axis(y, g.bmin[1], g.oscale[1], g.occ_res),
            vz = grid_axis(z, g.bmin[2], g.oscale[2], g.occ_res);
        if (!occ_test(g.occ, g.occ_res, vx, vy, vz)) {
            float te;
            if (!dda_next(g, r, vx, vy, vz, tf, te)) return -1;
            t = te;
            const int f = g.occ_per_cell;
            return vx / f + g.N * (vy / f + g.N * (vz / f));
        }
    }
    return cell_of(g, x, y, z);
}

// The first part of advance_ray: the cell of x(t) when its occupancy voxel is occupied (or there is no
// mask), or -2 when the voxel is empty and the ray needs the DDA (advance_ray then gives the same
// result as from the start).
__device__ __forceinline__ int advance_fast(const GridView &g, const Ray &r, float t) {
    const float x = fmaf(t, r.wx, r.ox), y = fmaf(t, r.wy, r.oy), z = fmaf(t, r.wz, r.oz);
    if (g.occ) {
        const int vx = grid_axis(x, g.bmin[0], g.oscale[0], g.occ_res),
                  vy = grid_axis(y, g.bmin[1], g.oscale[1], g.occ_res),
                  vz = grid_axis(z, g.bmin[2], g.oscale[2], g.occ_res);
        if (!occ_test(g.occ, g.occ_res, vx, vy, vz)) return -2;
    }
    return cell_of(g, x, y, z);
}

}  // namespace kns
