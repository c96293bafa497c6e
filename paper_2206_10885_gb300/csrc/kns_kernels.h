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

// Device counters of one wavefront render.
struct WaveCtrl {
    int n_live[2];  // samples queued for the current / next round
    int n_hits;     // rays that converged (queued for shading)
    int n_tiles;    // block tiles of the current round
    int next_tile;     // dynamic tile counter of the current round (FP32 tiles)
    int tail;          // 1: the current round is small enough to finish one thread per ray
    int n_tiles_fine;  // tiles of FP32 samples (keys < NC); BF16 tiles follow them
    int next_tile_bf;  // dynamic tile counter of the BF16 tiles
    unsigned long long samples_f32;   // SDF evaluations in FP32 tiles and the per-thread tail
    unsigned long long samples_bf16;  // SDF evaluations in BF16 tiles
};

// One view of a render: its camera, image size, first ray id and output buffers (device, 128 B).
struct ViewDev {
    float cam[16];  // c2w[12], fx, fy, cx, cy
    float *rgb, *depth, *normal;
    int32_t *cell, *steps;
    uint8_t *hit;
    int W, H, ray_base, pad;
};

// Everything the wavefront kernels read and write (device pointers; passed by value).
struct WaveArgs {
    int n_views, max_W, max_H, max_steps;
    const ViewDev *views;  // n_views entries; rays of view v are ray_base .. ray_base + W*H - 1
    int *ray_view;         // view of each ray
    float eps;
    int NC;               // cells N^3
    int nkeys;            // sort keys: key = cell + NC * coarse (NC for FP32 renders, 2 NC for BF16)
    int coarse;           // 1: BF16 render (rays start in the coarse BF16 phase and refine in FP32)
    float eps_coarse;     // BF16 phase hit threshold
    int refine_steps;     // FP32 evaluations after a BF16 hit before the final decision
    const unsigned char *wb;  // BF16 mma fragment trace weights
    int wb_stride;            // bytes per cell
    int btile;            // samples per block tile (cell-sorted samples are cut into such tiles)
    int inner_steps;      // sphere steps a tile may take in one round while its rays stay in its cells
    int tail_max;         // a round with at most this many rays is finished one thread per ray
    int min_active;       // warp tiles with fewer live rays hand them to the next round
    int static_tiles;     // 1: contiguous runs of tiles per block (weight reuse); 0: dynamic
    int *status;          // context status word (kns_status of a device-side failure, 0 = fine)
    const float *wt;      // k-major trace weights (see kns_device.cuh)
    int wt_stride;        // floats per cell
    // per-ray state
    float *t_ray;
    int *steps_ray, *cell_ray;
    // wave queues (double-buffered), cell-sorted samples, hits
    int *q[2], *qcell[2];
    int *sorted, *hits;
    int *count[2], *fill[2];  // per-cell sample counts and scatter cursors
    int *off, *tile_off;      // NC+1 exclusive scans: samples and tiles per cell
    WaveCtrl *ctrl;
};

// Per-configuration launchers (explicitly instantiated, one object file per configuration).
template <class C>
cudaError_t launch_wave_gen_cfg(const GridView &g, const WaveArgs &a, cudaStream_t s);
template <class C>
cudaError_t launch_wave_eval_cfg(const GridView &g, const WaveArgs &a, int cur, int blocks, cudaStream_t s);
template <class C>
cudaError_t launch_wave_shade_cfg(const GridView &g, const WaveArgs &a, int blocks, cudaStream_t s);
template <class C>
cudaError_t launch_wave_eval_bf16_cfg(const GridView &g, const WaveArgs &a, int cur, int blocks, cudaStream_t s);
template <class C>
cudaError_t launch_sdf_cfg(const GridView &g, const float *pts, int64_t n, float *sdf, float *feat, float *grad,
                           cudaStream_t s);
template <class C>
cudaError_t launch_occ_cfg(const GridView &g, float thresh, uint32_t *words, cudaStream_t s);

bool shape_supported(const Shape &sh);
int cell_floats(const Shape &sh);
int trace_cell_floats(const Shape &sh);
int bf16_cell_bytes(const Shape &sh, int *k0p);

cudaError_t launch_wave_gen(const Shape &sh, const GridView &g, const WaveArgs &a, cudaStream_t s);
cudaError_t launch_wave_eval(const Shape &sh, const GridView &g, const WaveArgs &a, int cur, int blocks,
                             cudaStream_t s);
cudaError_t launch_wave_shade(const Shape &sh, const GridView &g, const WaveArgs &a, int blocks, cudaStream_t s);
cudaError_t launch_wave_eval_bf16(const Shape &sh, const GridView &g, const WaveArgs &a, int cur, int blocks,
                                  cudaStream_t s);
cudaError_t launch_wave_scan(const WaveArgs &a, int cur, cudaStream_t s);
cudaError_t launch_coarse_occupancy(const uint32_t *occ, int res, uint32_t *coarse, cudaStream_t s);
cudaError_t launch_wave_scatter(const WaveArgs &a, int cur, int blocks, cudaStream_t s);

cudaError_t launch_sdf_f32(const Shape &sh, const GridView &g, const float *pts, int64_t n, float *sdf,
                           float *feat, float *grad, cudaStream_t s);
cudaError_t launch_occupancy_f32(const Shape &sh, const GridView &g, float thresh, uint32_t *words,
                                 cudaStream_t s);

}  // namespace kns
