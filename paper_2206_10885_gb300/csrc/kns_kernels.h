// kns_kernels.h -- host-visible launch interface between the C ABI runtime and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kns {

struct GridView;

// Supported grid shape (template dispatch key).
struct Shape {
    int W, H, L, LD;
};

constexpr int MAX_CAMS_PER_LAUNCH = 64;

// Cameras passed by value as kernel parameters (no device scratch needed for them).
struct CamBatch {
    float c[MAX_CAMS_PER_LAUNCH][16];
};

struct RenderArgs {
    int W, H, max_steps;
    float eps;
    int cam_base;  // index of the first camera of this launch in the output frame
    float *rgb, *depth, *normal;
    int32_t *cell, *steps;
    uint8_t *hit;
};

// Per-configuration launchers (explicitly instantiated, one object file per configuration).
template <class C>
cudaError_t launch_render_cfg(const GridView &g, const CamBatch &cams, int n_cams, const RenderArgs &a,
                              cudaStream_t s);
template <class C>
cudaError_t launch_sdf_cfg(const GridView &g, const float *pts, int64_t n, float *sdf, float *feat, float *grad,
                           cudaStream_t s);
template <class C>
cudaError_t launch_occ_cfg(const GridView &g, float thresh, uint32_t *words, cudaStream_t s);

bool shape_supported(const Shape &sh);
int cell_floats(const Shape &sh);

cudaError_t launch_render_f32(const Shape &sh, const GridView &g, const CamBatch &cams, int n_cams,
                              const RenderArgs &a, cudaStream_t s);
cudaError_t launch_sdf_f32(const Shape &sh, const GridView &g, const float *pts, int64_t n, float *sdf,
                           float *feat, float *grad, cudaStream_t s);
cudaError_t launch_occupancy_f32(const Shape &sh, const GridView &g, float thresh, uint32_t *words,
                                 cudaStream_t s);

}  // namespace kns
