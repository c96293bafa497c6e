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
    int next_tile;     // dynamic tile counter of the current round (FP32 tiles; rays in a tail round)
    int tail;          // 1: the current round is small enough to finish one warp per ray
    int n_tiles_fine;  // tiles of FP32 samples (keys < NC); BF16 tiles follow them
    int next_tile_bf;  // dynamic tile counter of the BF16 tiles
    int n_pend[2];     // rays a round (by parity) left in an empty voxel (its pending list)
    unsigned long long samples_f32;   // SDF evaluations in FP32 (tiles and the tail)
    unsigned long long samples_bf16;  // SDF evaluations in BF16 tiles
    unsigned long long samples_tail;  // the part of samples_f32 evaluated by the one-warp-per-ray tail
    int scan_part[2][256];            // per scan block of a round: its samples and tiles (the sort's scan)
    int n_refine;                     // BF16 renders: hits the shading's FP32 evaluation did not confirm
    // persistent BF16 trace (one cooperative launch runs every round)
    unsigned bar_count, bar_gen;      // grid barrier: arrivals, generation
    int next_adv;                     // the previous round's pending rays handed out to warps
    int rounds;                       // rounds it ran
    int tail_parity;                  // queue parity of the round it left to the one-warp-per-ray tail
    int round_live[512];              // samples queued for each round
    int round_tiles[512];             // tiles of each round (persistent BF16 trace)
    unsigned long long round_end_ns[512];  // global timer at the end of each round
    unsigned long long round_phase_ns[512][4];  // ... and at the end of its sort, scatter and tile phases
    unsigned long long start_ns;      // global timer at its start
};
constexpr int kMaxTraceRounds = 512;

// One view of a render: its camera, image size, first ray id and output buffers (device, 128 B).
struct ViewDev {
    float cam[16];  // c2w[12], fx, fy, cx, cy
    float *rgb, *depth, *normal;
    int32_t *cell, *steps;
    uint8_t *hit;
    int W, H, ray_base, grid;  // grid: which grid of a stack the view renders (0 for a single grid)
};

// Everything the wavefront kernels read and write (device pointers; passed by value).
// Tile descriptors a round can need: every key's partial tile plus full tiles of the smallest size.
inline int64_t max_tiles(int64_t rays, int nkeys) { return rays / 16 + nkeys + 1; }

struct WaveArgs {
    int n_views, max_W, max_H, max_steps;
    const ViewDev *views;  // n_views entries; rays of view v are ray_base .. ray_base + W*H - 1
    const float *ray_o, *ray_w;  // explicit rays (n_table x 3 each) instead of camera pixels, or NULL
    int n_table;
    int *ray_view;         // view of each ray
    float eps;
    int NC;               // cells N^3
    int nkeys;            // sort keys: the cells (NC)
    int coarse;           // 1: BF16 render (tensor-core trace; FP32 re-evaluates its hits at shading)
    float eps_coarse;     // BF16 trace hit threshold
    int refine_steps;     // FP32 evaluations of a BF16 hit (the shading's first) before the final decision
    const unsigned char *wb;  // BF16 hi/lo tensor-core trace weights (kns_tc.cuh)
    int wb_stride;            // bytes per cell
    int btile;            // samples per FP32 tile (cell-sorted samples are cut into such tiles)
    int btile_bf;         // samples per BF16 tile (keys >= NC)
    int inner_steps;      // sphere steps a tile may take in one round while its rays stay in its cells
    int tail_max;         // a round with at most this many rays is finished one warp per ray
    int min_active;       // warp tiles with fewer live rays hand them to the next round
    int inner_steps_bf;   // the same two knobs for the tensor-core tiles of BF16 renders
    int min_active_bf;
    int static_tiles;     // 1: contiguous runs of tiles per block (weight reuse); 0: dynamic
    int *status;          // context status word (kns_status of a device-side failure, 0 = fine)
    const float *wt;      // k-major trace weights (see kns_device.cuh)
    int wt_stride;        // floats per cell
    // per-ray state
    float *t_ray;
    float4 *t_hist;       // the ray's last four evaluated positions, newest first (NULL: no cycle test)
    int4 *trap;           // BF16 renders: the ray's seam-trap tracker (NULL: none; kns_wave.cuh)
    float trap_span;      // its span limit along the ray (scene units)
    int *steps_ray, *cell_ray;
    // wave queues (double-buffered), cell-sorted samples, hits
    int *q[2], *qcell[2];
    int *sorted, *hits;
    int *count[2], *fill[2];  // per-cell sample counts and scatter cursors
    int *off, *tile_off;      // NC+1 exclusive scans: samples and tiles per cell
    int4 *tiles;              // per tile of the round: key, first sorted sample, samples (max_tiles entries)
    int *pend_r[2];           // per round parity: rays waiting for the occupancy DDA (bit 31: BF16 phase) ...
    float *pend_t[2];         // ... and the position each was last evaluated at
    WaveCtrl *ctrl;
};

// Per-configuration launchers (explicitly instantiated, one object file per configuration).
template <class C>
cudaError_t launch_wave_gen_cfg(const GridView &g, const WaveArgs &a, cudaStream_t s);
// The rays round k left in empty voxels (pending list of parity p = k & 1) walk to their next
// occupied voxel and join the queue, counts and live counter of parity p: round k + 2's input.  Runs
// beside round k + 1, after round k + 1's scan has cleared those counters.
cudaError_t launch_wave_advance(const GridView &g, const WaveArgs &a, int p, int sm_count, cudaStream_t s);
template <class C>
cudaError_t launch_wave_eval_cfg(const GridView &g, const WaveArgs &a, int cur, int blocks, int block_tiles,
                                 int sm_count, cudaStream_t s);
// The one-warp-per-ray tail of a round (returns at once unless ctrl->tail is set).
template <class C>
cudaError_t launch_wave_tail_cfg(const GridView &g, const WaveArgs &a, int cur, int sm_count, cudaStream_t s);
template <class C>
cudaError_t launch_shade_block_cfg(const GridView &g, const WaveArgs &a, int sm_count, cudaStream_t s);
template <class C>
int shade_cell_floats_cfg();
template <class C>
cudaError_t launch_shade_layout_cfg(const float *w, int cell_stride, int64_t ncell, float *ws, int ws_stride,
                                    cudaStream_t s);
template <class C>
cudaError_t launch_wave_eval_tc_cfg(const GridView &g, const WaveArgs &a, int cur, int sm_count, cudaStream_t s);
// Every round of a BF16 render after ray generation, in one cooperative launch (one block per SM);
// the rounds run in the kernel, separated by grid barriers.
template <class C>
cudaError_t launch_trace_tc_cfg(const GridView &g, const WaveArgs &a, int sm_count, cudaStream_t s);
// BF16 renders, after the shading: the FP32 steps of the hits on the refinement list (pend_r[0],
// pend_t[0] = the FP32 d at the ray's t), then their shading, one thread per ray.
template <class C>
cudaError_t launch_refine_cfg(const GridView &g, const WaveArgs &a, int sm_count, cudaStream_t s);
template <class C>
cudaError_t launch_sdf_cfg(const GridView &g, const float *pts, int64_t n, float *sdf, float *feat, float *grad,
                           cudaStream_t s);
template <class C>
cudaError_t launch_occ_cfg(const GridView &g, float thresh, uint32_t *words, cudaStream_t s);

bool shape_supported(const Shape &sh);
int cell_floats(const Shape &sh);
int trace_cell_floats(const Shape &sh);
int shade_cell_floats(const Shape &sh);
cudaError_t launch_shade_layout(const Shape &sh, const float *w, int cell_stride, int64_t ncell, float *ws,
                                int ws_stride, cudaStream_t s);


cudaError_t launch_wave_gen(const Shape &sh, const GridView &g, const WaveArgs &a, cudaStream_t s);
cudaError_t launch_wave_eval(const Shape &sh, const GridView &g, const WaveArgs &a, int cur, int blocks,
                             int block_tiles, int sm_count, cudaStream_t s);
cudaError_t launch_wave_eval_tc(const Shape &sh, const GridView &g, const WaveArgs &a, int cur, int sm_count,
                                cudaStream_t s);
cudaError_t launch_trace_tc(const Shape &sh, const GridView &g, const WaveArgs &a, int sm_count, cudaStream_t s);
cudaError_t launch_wave_tail(const Shape &sh, const GridView &g, const WaveArgs &a, int cur, int sm_count,
                             cudaStream_t s);
cudaError_t launch_wave_scan(const WaveArgs &a, int cur, cudaStream_t s);
cudaError_t launch_hit_sort(const WaveArgs &a, int tile, int sm_count, cudaStream_t s);  // tile: shade_hit_tile
cudaError_t launch_shade_block(const Shape &sh, const GridView &g, const WaveArgs &a, int sm_count, cudaStream_t s);
cudaError_t launch_refine(const Shape &sh, const GridView &g, const WaveArgs &a, int sm_count, cudaStream_t s);
inline int shade_hit_tile(int sdf_width) { return 4096 / sdf_width; }  // hits per shading tile
cudaError_t launch_coarse_occupancy(const uint32_t *occ, int res, uint32_t *coarse, cudaStream_t s);
cudaError_t launch_occ_bounds(const uint32_t *occ, int res, int *bounds, cudaStream_t s);
cudaError_t launch_selftest_timeout(WaveCtrl *ctrl, int *status, int which, uint32_t polls, cudaStream_t s);
cudaError_t launch_wave_scatter(const WaveArgs &a, int cur, int blocks, cudaStream_t s);

// Measured FP32 FMA (FLOP/s) and ex2 (operations/s) throughput of the device (kns_peak.cu).
cudaError_t measure_peaks(int sm_count, cudaStream_t s, double *ffma_flops, double *mufu_ops);

cudaError_t launch_sdf_f32(const Shape &sh, const GridView &g, const float *pts, int64_t n, float *sdf,
                           float *feat, float *grad, cudaStream_t s);
cudaError_t launch_occupancy_f32(const Shape &sh, const GridView &g, float thresh, uint32_t *words,
                                 cudaStream_t s);

// ------------------------------------------------------------------ path tracing
struct PtArgs {
    int n_cams, W, H, spp, max_depth;
    int64_t n_paths;            // n_cams * W * H * spp
    const float *cams;          // device, n_cams x 16
    uint64_t seed;
    float offset;               // bounce origin = hit + offset * normal
    float horizon[3], zenith[3];
    float bmax[3];              // box corner (dead paths get a ray that misses the box)
    float *o, *w, *beta, *L;    // per path x 3
    uint8_t *alive;
    const float *t_rgb, *t_depth, *t_normal;  // the current depth's trace results
    const uint8_t *t_hit;
    float *rgb_out;             // per pixel x 3
};
int pt_max_depth();
cudaError_t pt_primary(const PtArgs &a, cudaStream_t s);
cudaError_t pt_bounce(const PtArgs &a, int depth, cudaStream_t s);
cudaError_t pt_resolve(const PtArgs &a, cudaStream_t s);

// ------------------------------------------------------------------ training step
// Everything the training kernels read and write (device pointers unless noted; passed by value).
// Records: coarse samples (B x Ns), central-difference points (6 per fine sample and per eikonal
// point) and fine-sample centres (B x S).  Records are counting-sorted by key: coarse records by
// cell; fine records by cell (difference points) and NC + cell (centres).
struct TrainArgs {
    int N, NC, H;                      // cells per axis, N^3, SDF hidden layers (width 32)
    float bmin[3], bmax[3], cscale[3];
    float beta, inv_beta;
    int p_cell, p_sdf;                 // canonical floats per cell and in its SDF part
    const float *params;               // canonical weights
    float *grad;                       // canonical gradient (accumulated; zeroed by the caller)
    int64_t B;                         // rays
    const float *o, *w, *target;       // B x 3
    int Ns, Ni, S;                     // stratified, importance, total samples per ray
    const float *u_s, *u_i;            // B x Ns, B x Ni
    int64_t M;                         // eikonal points
    const float *P;                    // M x 3
    float s, s_up, lambda, h;
    const float *dloss;                // upstream scalar (NULL = 1)
    // scratch
    float *t;                          // B x S sample positions
    uint8_t *valid;                    // B: the ray meets the box
    float *d_coarse;                   // B x Ns
    float *d_fd, *g_fd;                // (B S + M) x 6: SDF at the difference points and its upstream
    float *d_c, *g_dc;                 // B x S: SDF at the sample centres and its upstream
    float *rgb_c, *g_rgb;              // B x S x 3: colour and its upstream
    float *C;                          // B x 3 rendered colour
    double *acc;                       // [0] sum |C - I|, [1] sum (|grad| - 1)^2
    float *loss;                       // 3: total, colour, eikonal
    int nkeys;
    int *count, *off, *fill, *chunk_off;  // nkeys + 1 each
    float4 *sorted;                    // x, y, z, record id (bit pattern)
    int *status;
};

// record sets of the training sort
enum TrainRecords { TRAIN_COARSE = 0, TRAIN_FINE = 1 };

cudaError_t train_sort(const TrainArgs &a, int which, int64_t n_rec, int sm_count, cudaStream_t s);
cudaError_t train_coarse_eval(const TrainArgs &a, int sm_count, cudaStream_t s);
cudaError_t train_importance(const TrainArgs &a, cudaStream_t s);
cudaError_t train_valid(const TrainArgs &a, cudaStream_t s);
cudaError_t train_fd_forward(const TrainArgs &a, int sm_count, cudaStream_t s);
cudaError_t train_centre_forward(const TrainArgs &a, int sm_count, cudaStream_t s);
cudaError_t train_loss_forward(const TrainArgs &a, cudaStream_t s);
cudaError_t train_rgb_out(const TrainArgs &a, float *rgb, cudaStream_t s);
cudaError_t train_upstream(const TrainArgs &a, cudaStream_t s);
cudaError_t train_centre_backward(const TrainArgs &a, int sm_count, cudaStream_t s);
cudaError_t train_fd_backward(const TrainArgs &a, int sm_count, cudaStream_t s);
int train_chunk_records();

}  // namespace kns
