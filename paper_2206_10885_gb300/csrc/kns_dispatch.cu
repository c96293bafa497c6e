// kns_dispatch.cu -- maps a runtime grid shape to the compiled configuration's launchers.
#include "kns_device.cuh"
#include "kns_kernels.h"

namespace kns {

// Calls f(Cfg<...>{}) for the compiled configuration matching sh.  The list must match the
// configurations build.py instantiates.
template <class F>
static cudaError_t dispatch(const Shape &sh, F &&f) {
    if (sh.W == 32 && sh.H == 2 && sh.L == 4 && sh.LD == 2) return f(Cfg<32, 2, 4, 2>{});
    if (sh.W == 32 && sh.H == 3 && sh.L == 4 && sh.LD == 2) return f(Cfg<32, 3, 4, 2>{});
    if (sh.W == 64 && sh.H == 2 && sh.L == 4 && sh.LD == 2) return f(Cfg<64, 2, 4, 2>{});
    if (sh.W == 64 && sh.H == 3 && sh.L == 4 && sh.LD == 2) return f(Cfg<64, 3, 4, 2>{});
    if (sh.W == 32 && sh.H == 2 && sh.L == 6 && sh.LD == 4) return f(Cfg<32, 2, 6, 4>{});
    if (sh.W == 32 && sh.H == 3 && sh.L == 6 && sh.LD == 4) return f(Cfg<32, 3, 6, 4>{});
    if (sh.W == 64 && sh.H == 2 && sh.L == 6 && sh.LD == 4) return f(Cfg<64, 2, 6, 4>{});
    if (sh.W == 64 && sh.H == 3 && sh.L == 6 && sh.LD == 4) return f(Cfg<64, 3, 6, 4>{});
    return cudaErrorInvalidValue;
}

cudaError_t launch_sdf_f32(const Shape &sh, const GridView &g, const float *pts, int64_t n, float *sdf,
                           float *feat, float *grad, cudaStream_t s) {
    return dispatch(sh, [&](auto c) { return launch_sdf_cfg<decltype(c)>(g, pts, n, sdf, feat, grad, s); });
}

cudaError_t launch_occupancy_f32(const Shape &sh, const GridView &g, float thresh, uint32_t *words,
                                 cudaStream_t s) {
    return dispatch(sh, [&](auto c) { return launch_occ_cfg<decltype(c)>(g, thresh, words, s); });
}

cudaError_t launch_wave_gen(const Shape &sh, const GridView &g, const WaveArgs &a, cudaStream_t s) {
    return dispatch(sh, [&](auto c) { return launch_wave_gen_cfg<decltype(c)>(g, a, s); });
}
cudaError_t launch_wave_eval(const Shape &sh, const GridView &g, const WaveArgs &a, int cur, int blocks,
                             int block_tiles, int sm_count, cudaStream_t s) {
    return dispatch(sh, [&](auto c) {
        return launch_wave_eval_cfg<decltype(c)>(g, a, cur, blocks, block_tiles, sm_count, s);
    });
}
cudaError_t launch_shade_block(const Shape &sh, const GridView &g, const WaveArgs &a, int sm_count, cudaStream_t s) {
    return dispatch(sh, [&](auto c) { return launch_shade_block_cfg<decltype(c)>(g, a, sm_count, s); });
}

cudaError_t launch_refine(const Shape &sh, const GridView &g, const WaveArgs &a, int sm_count, cudaStream_t s) {
    return dispatch(sh, [&](auto c) { return launch_refine_cfg<decltype(c)>(g, a, sm_count, s); });
}
cudaError_t launch_wave_tail(const Shape &sh, const GridView &g, const WaveArgs &a, int cur, int sm_count,
                             cudaStream_t s) {
    return dispatch(sh, [&](auto c) { return launch_wave_tail_cfg<decltype(c)>(g, a, cur, sm_count, s); });
}
cudaError_t launch_trace_tc(const Shape &sh, const GridView &g, const WaveArgs &a, int sm_count, cudaStream_t s) {
    return dispatch(sh, [&](auto c) { return launch_trace_tc_cfg<decltype(c)>(g, a, sm_count, s); });
}
cudaError_t launch_wave_eval_tc(const Shape &sh, const GridView &g, const WaveArgs &a, int cur, int sm_count,
                                cudaStream_t s) {
    return dispatch(sh, [&](auto c) { return launch_wave_eval_tc_cfg<decltype(c)>(g, a, cur, sm_count, s); });
}

int trace_cell_floats(const Shape &sh) {
    int size = 0;
    dispatch(sh, [&](auto c) {
        size = decltype(c)::TSIZE;
        return cudaSuccess;
    });
    return size;
}

int shade_cell_floats(const Shape &sh) {
    int size = 0;
    dispatch(sh, [&](auto c) {
        size = shade_cell_floats_cfg<decltype(c)>();
        return cudaSuccess;
    });
    return size;
}
cudaError_t launch_shade_layout(const Shape &sh, const float *w, int cell_stride, int64_t ncell, float *ws,
                                int ws_stride, cudaStream_t s) {
    return dispatch(sh, [&](auto c) {
        return launch_shade_layout_cfg<decltype(c)>(w, cell_stride, ncell, ws, ws_stride, s);
    });
}

bool shape_supported(const Shape &sh) {
    const bool wl = (sh.W == 32 || sh.W == 64) && (sh.H == 2 || sh.H == 3);
    const bool enc = (sh.L == 4 && sh.LD == 2) || (sh.L == 6 && sh.LD == 4);
    return wl && enc;
}

int cell_floats(const Shape &sh) {
    int size = 0;
    dispatch(sh, [&](auto c) {
        size = decltype(c)::SIZE;
        return cudaSuccess;
    });
    return size;
}

}  // namespace kns
