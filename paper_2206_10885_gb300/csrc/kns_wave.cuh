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

#include <atomic>

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
// The cycle test of the BF16 trace.  Its d carries the split-BF16 rounding noise (~1e-6), so a ray
// oscillating across a cell seam jitters by a few ulps around its 2-cycle instead of repeating a
// position exactly; a return to within 2^-19 |t| (~4e-6 near the object, 1/25 of eps = 1e-4) of one of
// the last four positions ends it as the exact test would.  A ray that has not converged cannot come
// back that close while stepping by |d| >= eps_coarse unless its steps alternate in sign.
__device__ __forceinline__ bool cycle_step_tol(float4 &hist, float t_eval, float t_next) {
    const float tol = fmaxf(fabsf(t_next), 1.f) * 1.9073486e-6f;  // 2^-19
    if (fabsf(t_next - hist.x) <= tol || fabsf(t_next - hist.y) <= tol || fabsf(t_next - hist.z) <= tol ||
        fabsf(t_next - hist.w) <= tol)
        return true;
    hist = make_float4(t_eval, hist.x, hist.y, hist.z);
    return false;
}

// Seam trap of the BF16 trace.  Near a cell face where the two cells' SDFs disagree about the surface
// (each cell is perturbed on its own), a grazing ray can shuttle between the two cells for ever: one
// cell's d pushes it across the face, the other's pushes it back, neither |d| reaches eps, and the
// positions wander quasi-periodically inside a small interval instead of repeating exactly (so the
// cycle tests above never fire).  The plain iteration ends such a ray as a miss when its budget runs
// out.  The tracker watches the ray's latest run of samples: it restarts on an occupancy skip, on a
// third cell, when the run's positions spread beyond `span` along the ray, or at |d| < dmin; a run of
// 16 samples confined to two cells that reversed direction at least twice is a trapped ray.  Measured
// on FP64 trajectories of the 1080p workloads (16^3 and 32^3 grids, span 0.02, dmin 5 eps): 75-83 % of
// the rays that exhaust the budget are caught near step 19 instead of 128, and none of 5000 rays that
// converge or leave after 12+ steps is caught before it does.
// State (int4): x, y = lowest and highest t of the run (float bits), z = first cell, w = second cell
// (19 bits, 0x7FFFF: none) | samples (5 bits) << 19 | reversals (4 bits) << 24 | sign of the last d << 28.
constexpr int TRAP_NONE = 0x7FFFF;
__device__ __forceinline__ int4 trap_empty() { return make_int4(0, 0, -1, TRAP_NONE); }
__device__ __forceinline__ bool trap_step(int4 &s, float t, float d, int c, float span, float dmin) {
    if (!(fabsf(d) >= dmin)) {
        s = trap_empty();
        return false;
    }
    const unsigned w = (unsigned)s.w;
    int n = (int)((w >> 19) & 31u), rev = (int)((w >> 24) & 15u), c2 = (int)(w & 0x7FFFFu);
    const unsigned sg = d > 0.f ? 1u : 0u;
    const float lo = fminf(__int_as_float(s.x), t), hi = fmaxf(__int_as_float(s.y), t);
    const bool restart = n == 0 || (c != s.z && c2 != TRAP_NONE && c != c2) || hi - lo > span;
    if (restart) {
        s = make_int4(__float_as_int(t), __float_as_int(t), c, (int)(TRAP_NONE | (1u << 19) | (sg << 28)));
        return false;
    }
    if (c != s.z && c2 == TRAP_NONE) c2 = c;
    if (sg != ((w >> 28) & 1u)) rev = rev < 15 ? rev + 1 : 15;
    n = n < 31 ? n + 1 : 31;
    s = make_int4(__float_as_int(lo), __float_as_int(hi), s.z,
                  (int)((unsigned)c2 | ((unsigned)n << 19) | ((unsigned)rev << 24) | (sg << 28)));
    return n >= 16 && rev >= 2;
}

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
            return g.cell_base + vx / f + g.N * (vy / f + g.N * (vz / f));
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

// Entry i of the pending list of parity p_in (i < n; every lane of the warp calls it): the ray walks the
// occupancy DDA from its position to its next occupied voxel (or leaves the grid: a miss), takes the
// cycle test on the position reached, and joins the queue, counts and live counter of parity p_out.
__device__ __forceinline__ void advance_pending(const GridView &g, const WaveArgs &a, int p_in, int p_out, int i,
                                                int n) {
    bool emit = false;
    int ncell = -1, r = 0, key = 0;
    if (i < n) {
        r = a.pend_r[p_in][i];
        const bool cycles = a.t_hist != nullptr;
        const float t_eval = a.pend_t[p_in][i];
        int cam;
        const Ray ray = ray_of(a, r, cam);
        const GridView gv = sub_grid(g, a.views[cam].grid);
        float t0, tf;
        clip_box(gv, ray, t0, tf);
        float t = a.t_ray[r];
        ncell = advance_ray(gv, ray, t, tf);
        if (ncell < 0) {
            write_miss(a, r, a.steps_ray[r]);
        } else {
            float4 hist = cycles ? a.t_hist[r] : no_history();
            // BF16 renders: the BF16 trace's cycle test (the rays on these lists are all in it)
            const bool cyc = cycles && (a.coarse ? cycle_step_tol(hist, t_eval, t) : cycle_step(hist, t_eval, t));
            if (cyc) {
                write_miss(a, r, a.max_steps);
                ncell = -1;
            } else {
                emit = true;
                key = ncell;
                a.t_ray[r] = t;
                if (cycles) a.t_hist[r] = hist;
                if (a.trap) a.trap[r] = trap_empty();  // a run of samples ends at an occupancy skip
            }
        }
    }
    const int qp = warp_append(&a.ctrl->n_live[p_out], emit);
    if (emit) {
        a.q[p_out][qp] = r;
        a.qcell[p_out][qp] = key;
    }
    warp_count_cells(a.count[p_out], emit, key);
}

constexpr uint32_t kGridPolls = 1u << 22;  // bound of every grid-barrier wait (polls of ~0.1 us)

// Grid-wide barrier of a cooperative launch (every block resident): the blocks' thread 0 count in on
// a global counter; the last to arrive resets it and advances the generation the others poll.  Bounded:
// false after kGridPolls polls (the caller reports KNS_ERR_TIMEOUT and leaves).  Block-uniform result.
__device__ __forceinline__ bool grid_sync(WaveCtrl *ctrl, unsigned &gen, int *s_flag, uint32_t polls = kGridPolls) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned target = gen + 1;
        __threadfence();
        if (atomicAdd(&ctrl->bar_count, 1u) == gridDim.x - 1) {
            atomicExch(&ctrl->bar_count, 0u);
            __threadfence();
            atomicExch(&ctrl->bar_gen, target);
        } else {
            uint32_t i = 0;
            while (*(volatile unsigned *)&ctrl->bar_gen != target) {
                if (++i > polls) {
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        gen = target;
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Resident blocks per SM of a kernel with `smem` bytes of dynamic shared memory (registers and shared
// memory both count), after allowing it the largest shared-memory carve-out; asked once per kernel.
template <class K>
cudaError_t resident_blocks(K kernel, int threads, int smem, std::atomic<int> &cache, int &out) {
    out = cache.load();
    if (out > 0) return cudaSuccess;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&out, kernel, threads, smem)) != cudaSuccess)
        return e;
    if (out < 1) out = 1;
    cache.store(out);
    return cudaSuccess;
}

}  // namespace kns
