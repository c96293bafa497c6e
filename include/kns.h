/*
 * kns.h -- C ABI of the KiloNeuS sphere-tracing library (GB300, sm_103a).
 *
 * KiloNeuS (Sec. 3.1) stores a signed distance field and a colour field in a
 * regular N^3 grid of tiny MLPs over a fixed bounding box.  Rendering
 * (Sec. 3.4.1) sphere-traces each camera ray inside the box: at every sample
 * it finds the sample's cell m(x), evaluates that cell's SDF MLP on the
 * positional encoding gamma(x) (Eq. 1, Eq. 2), and stops when |d| < eps; at
 * the hit it takes the normalised analytic input-gradient of the SDF as the
 * normal and evaluates the cell's colour MLP (Eq. 3).
 *
 * Conventions shared by every entry point
 *  - Status: every call returns a kns_status; KNS_OK (0) is success.  A
 *    failing call enqueues nothing.  kns_last_error() gives a message.
 *  - Argument errors are detected on the host before any work is enqueued.
 *  - Asynchrony: compute calls enqueue on the caller's CUDA stream
 *    (`cuda_stream`, a cudaStream_t; NULL = the legacy default stream) and
 *    return without waiting.  A render also runs work on a stream the context
 *    owns, forked from and joined back into the caller's stream with events
 *    inside the call, so the render is complete, like any other work, when
 *    the caller's stream reaches the point after it.  An FP32 render's loop
 *    reads a small pinned counter on the host between rounds; a BF16 render
 *    runs its rounds on the device in one persistent launch.  Device-side failures (a bounded wait that
 *    ran out, a bounds check that tripped) are recorded in a per-context
 *    status word and returned by the next kns_sync() on that context.
 *  - Memory: the caller owns every input and output buffer and passes plain
 *    pointers (device pointers unless stated "host").  The library never
 *    frees caller memory.  Grids own the device copies of their weights.
 *  - Threads: a context may be used from several host threads; calls on one
 *    context are serialised on the host.  Their GPU work shares the context's
 *    scratch, so one context's renders must also be ordered on the GPU: issue
 *    them on one stream, or order their streams with events (two renders of
 *    one context running at once on different streams race).  Use a context
 *    per concurrent stream, as the render server does.
 *
 * Canonical weight layout (host, FP32, every loader takes it)
 *   cells in x-fastest order, cell = ix + N*(iy + N*iz); per cell the SDF MLP
 *   layers, then the colour MLP layers; per layer W[out][in] row-major, then
 *   b[out].  SDF layers: (3+6*pe_pos_L) -> sdf_width (x sdf_hidden, softplus)
 *   -> 1+feat_dim (linear: row 0 is d, rows 1.. are the feature z).  Colour
 *   layers: (feat_dim + 3 + 3+6*pe_dir_L [+3 if col_use_x]) -> col_width
 *   (x col_hidden, ReLU) -> 3 (sigmoid).  Colour input order: z, n, gamma(v),
 *   then x when col_use_x.  gamma_L(p) = [p, then for k = 0..L-1:
 *   sin(2^k pi p_c) for c = x,y,z, then cos(2^k pi p_c) for c = x,y,z].
 *
 * Occupancy mask layout: res^3 bits, bit index ix + res*(iy + res*iz), packed
 *   little-endian into uint64 words (bit b of word k is voxel 64k + b).
 */
#ifndef KNS_H_
#define KNS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum kns_status {
    KNS_OK = 0,
    KNS_ERR_INVALID_ARG = 1,   /* a null required pointer, a size out of range, ... */
    KNS_ERR_OUT_OF_MEMORY = 2, /* a device or host allocation failed */
    KNS_ERR_CUDA = 3,          /* a CUDA runtime call failed (message has the CUDA error) */
    KNS_ERR_FORMAT = 4,        /* a grid file is malformed or truncated */
    KNS_ERR_UNSUPPORTED = 5,   /* a descriptor shape the kernels are not built for */
    KNS_ERR_TIMEOUT = 6,       /* kns_sync ran out of time, or a device wait gave up */
    KNS_ERR_BUSY = 7,          /* the resource is in use */
    KNS_ERR_INTERNAL = 8       /* a device-side consistency check failed */
} kns_status;

/* Arithmetic of the render path. */
enum { KNS_FP32 = 0, /* every MLP evaluation in FP32 on the CUDA cores */
       KNS_BF16 = 1  /* trace MLPs on the tensor cores as split BF16 products (hi + lo parts, FP32
                        accumulation), then the last sphere step(s), the normal and the colour in FP32 */ };

typedef struct kns_ctx kns_ctx;   /* opaque: one device, its scratch, its status word */
typedef struct kns_grid kns_grid; /* opaque: one resident Kilo-grid */

/* Shape of a Kilo-grid (Sec. 3.1).  The paper uses N = 16, pe_pos_L = 6, pe_dir_L = 4,
 * bounding box [-1,1]^3 (Sec. 3.2.1). */
typedef struct kns_grid_desc {
    int32_t N;           /* cells per axis (1..64) */
    int32_t pe_pos_L;    /* encoding frequencies of x (Eq. 1) */
    int32_t pe_dir_L;    /* encoding frequencies of the view direction */
    int32_t sdf_hidden;  /* hidden layers of the SDF MLP */
    int32_t sdf_width;   /* their width */
    int32_t feat_dim;    /* feature z passed to the colour MLP */
    int32_t col_hidden;  /* hidden layers of the colour MLP */
    int32_t col_width;   /* their width */
    int32_t col_use_x;   /* 1: the colour MLP also takes raw x (Eq. 3); 0: it does not */
    int32_t occ_res;     /* occupancy voxels per axis (0 = no empty-space skipping; a multiple of N) */
    float softplus_beta; /* softplus sharpness of the SDF MLP (100 in the synthetic grids) */
    float bbox_min[3];   /* bounding box of the grid */
    float bbox_max[3];
} kns_grid_desc;

/* Pinhole camera: c2w is a row-major 3x4 matrix whose columns are the camera's right, down and
 * forward axes and its position in world space; pixel (i, j) (row i from the top, column j)
 * looks along normalize(c2w[:, :3] * ((j+0.5-cx)/fx, (i+0.5-cy)/fy, 1)). */
typedef struct kns_camera {
    float c2w[12];
    float fx, fy, cx, cy;
} kns_camera;

/* Per-pixel outputs (device pointers), indexed p = cam*H*W + i*W + j.  rgb and depth are
 * required; the rest may be NULL.  Misses: rgb = 0, depth = +inf, normal = 0, cell = -1,
 * hit = 0.  steps counts SDF evaluations of the trace (the hit evaluation included). */
typedef struct kns_frame {
    float *rgb;     /* 3 floats per pixel */
    float *depth;   /* ray parameter t at the hit (unit directions: distance from the camera) */
    float *normal;  /* 3 floats per pixel, unit length on hits */
    int32_t *cell;  /* hit cell m(x) */
    int32_t *steps; /* SDF evaluations */
    uint8_t *hit;   /* 1 on a hit */
} kns_frame;

/* Options of kns_render (NULL = FP32 defaults).  The tuning fields change only the schedule of
 * the work, never a result; 0 selects the built-in default. */
typedef struct kns_render_opts {
    int32_t precision;    /* KNS_FP32 or KNS_BF16 */
    float eps_coarse;     /* KNS_BF16: hit threshold of the BF16 trace (> 0; 0: 0.9 eps); FP32 decides the hit */
    int32_t refine_steps; /* KNS_BF16: FP32 evaluations of a BF16 hit (<= 0: 2): the first re-evaluates the
                             BF16 trace's last step; the ray is a hit at the first |d| < eps, or at the last
                             of them if |d| < eps_coarse there, else a miss */
    /* tuning (0 = default) */
    int32_t inner_steps;   /* evaluations a tile may make per round while its rays stay in its cell (1..1024;
                              default 4 for warp tiles, 2 for block tiles) */
    int32_t min_active;    /* a tile continues only while at least this many of its rays stay in its cell
                              (1..256; a warp tile holds 16; default 8 for warp tiles, 16 for block tiles) */
    int32_t tail_rays;     /* a round with at most this many rays is finished one warp per ray, in FP32 (>= 0;
                              -1: never; default: KNS_FP32 131072 at SDF width 32, 32768 at width 64; KNS_BF16
                              32768 at width 32, 16384 at width 64) */
    int32_t blocks_per_sm; /* evaluation blocks (one warp each) launched per SM (1..64) */
    int32_t static_tiles;  /* 1: each block takes a contiguous run of tiles; 2: tiles handed out dynamically */
    int32_t timing;        /* 1: time each kernel class with CUDA events for kns_get_render_stats (adds host work) */
    int32_t block_tiles;   /* FP32 evaluation (KNS_FP32 renders): 1 = 128-sample tiles per
                              256-thread block (block GEMMs); 3 = 256-sample tiles per 256 threads; 4 = 128-sample
                              tiles per 128 threads; 2 = 16-sample tiles per warp (in-tile stepping, min_active);
                              0 = default (4) */
    int32_t bf16_inner_steps; /* KNS_BF16: evaluations a tensor-core tile may make per round while its rays stay in
                                 its cell (1..1024; default 4 at SDF width 32, 2 at width 64) */
    int32_t bf16_min_active;  /* KNS_BF16: a tensor-core tile continues while at least this many of its rays stay
                                 (1..128; default 16) */
    int32_t bf16_rounds;      /* KNS_BF16: 1 = every round of the trace in one persistent launch (rounds run on the
                                 device, no host synchronisation); 2 = one launch sequence per round driven by
                                 the host; 0 = default (1).  Results are identical when no round is handed
                                 to the tail (tail_rays = -1); with the hand-over they agree within the
                                 BF16 accuracy gates. */
} kns_render_opts;

/* Counters of the last kns_render on a context (kns_get_render_stats). */
typedef struct kns_render_stats {
    int32_t rounds;        /* sort + evaluate rounds that ran */
    int64_t rays;          /* primary rays */
    int64_t hits;          /* rays that converged (shaded) */
    int64_t samples_fp32;  /* SDF evaluations in FP32 (sphere-trace samples, refinement included) */
    int64_t samples_bf16;  /* SDF evaluations in BF16 */
    /* device time (ms) per kernel class, summed over the render's launches; 0 unless opts->timing */
    float ms_generate, ms_sort, ms_eval_fp32, ms_eval_bf16, ms_shade, ms_total;
    int64_t samples_tail;  /* the part of samples_fp32 evaluated one warp per ray (rounds of <= tail_rays rays) */
    int64_t refined;       /* KNS_BF16: hits whose FP32 re-evaluation at shading was not within eps (FP32 steps) */
} kns_render_stats;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  *out receives the handle.
 * Errors: INVALID_ARG (out NULL, bad device), CUDA, OUT_OF_MEMORY. */
kns_status kns_create(int device, kns_ctx **out);

/* Destroy a context after its work has finished (grids must be freed first).  NULL is a no-op. */
void kns_destroy(kns_ctx *ctx);

/* Message of the last failure on this context (or of the last kns_create failure when ctx is NULL).
 * The string stays valid until the next call on the context. */
const char *kns_last_error(const kns_ctx *ctx);

/* Wait up to timeout_ms (< 0: forever) for the work enqueued on `cuda_stream`, then report the
 * context's device status word.  Returns OK, TIMEOUT (work still running), CUDA (an asynchronous
 * CUDA error), or the status a kernel recorded (TIMEOUT, INTERNAL).  Reading clears the word. */
kns_status kns_sync(kns_ctx *ctx, void *cuda_stream, int64_t timeout_ms);

/* ------------------------------------------------------------------ grids */

/* Upload a Kilo-grid (Sec. 3.1).  host_weights: canonical FP32 layout (header comment), exactly
 * n_floats = N^3 * (SDF + colour parameters) floats, host memory, copied.  occ_words: host uint64
 * occupancy words for desc->occ_res (copied), or NULL to build the mask on the device as
 * |d(voxel centre)| < voxel diagonal when occ_res > 0.  The call returns after the upload.  The grid
 * keeps four device copies of the weights, each in the layout one kernel family stages with bulk
 * copies (per-thread FP32, the FP32 tiles' k-major layout, the tensor-core split-BF16 layout, the
 * shading layout: about 235 KB per cell at width 64, 7.7 GB for 32^3 cells), the occupancy mask,
 * its 8^3-block mask and the index box of its occupied voxels.
 * Errors: INVALID_ARG (NULL pointer, n_floats mismatch, N or occ_res out of range),
 * UNSUPPORTED (a width, depth or encoding the kernels are not built for), OUT_OF_MEMORY, CUDA. */
kns_status kns_load_grid(kns_ctx *ctx, const kns_grid_desc *desc, const float *host_weights,
                         size_t n_floats, const uint64_t *occ_words, kns_grid **out);

/* Upload n_grids Kilo-grids of one descriptor as one resident stack, so that one kns_render_views call
 * can render views of different grids (a render server's requests for several scenes, Sec. 3.4.1's
 * renderer applied to each).  host_weights: the n_grids grids' canonical FP32 weights back to back
 * (n_floats = n_grids * N^3 * parameters per cell); occ_words: the n_grids occupancy masks back to back
 * (ceil(occ_res^3 / 64) words each), or NULL to build each from its own grid as kns_load_grid does.
 * Every grid of the stack keeps its own weights, mask, 8^3-block mask and results: a view of grid k
 * renders exactly as a kns_render of grid k loaded alone (bit for bit in FP32).  kns_render_views picks
 * the grid per view (kns_view.grid); kns_render, kns_render_noalloc, kns_trace_rays, kns_path_trace
 * and kns_sdf use grid 0 of a stack.
 * The stack's device memory is n_grids times a single grid's.  Errors: as kns_load_grid, plus
 * INVALID_ARG for n_grids < 1 or more than 262,144 cells in all (the BF16 seam trap's cell field). */
kns_status kns_load_grid_stack(kns_ctx *ctx, const kns_grid_desc *desc, int32_t n_grids, const float *host_weights,
                               size_t n_floats, const uint64_t *occ_words, kns_grid **out);

/* The number of grids a grid object holds (1 unless it came from kns_load_grid_stack).  Errors:
 * INVALID_ARG (NULL pointer). */
kns_status kns_grid_stack_size(const kns_grid *grid, int32_t *n_grids);

/* Load a grid file ("KNS1" header, canonical FP32 weights, optional occupancy words; all
 * little-endian).  Errors: as kns_load_grid, plus FORMAT for a bad magic, version or size. */
kns_status kns_load_grid_file(kns_ctx *ctx, const char *path, kns_grid **out);

/* Free a grid and its device memory (waits for the device first).  NULL is a no-op. */
void kns_free_grid(kns_grid *grid);

/* Copy a grid's descriptor to *out (host). */
kns_status kns_grid_get_desc(const kns_grid *grid, kns_grid_desc *out);

/* Copy the grid's occupancy mask into host_words (n_words uint64 words, host; a stack: its grids'
 * masks back to back, ceil(occ_res^3 / 64) words each).  Synchronous.
 * Errors: INVALID_ARG (no mask, or n_words too small), CUDA. */
kns_status kns_copy_occupancy(kns_ctx *ctx, const kns_grid *grid, uint64_t *host_words, size_t n_words);

/* ---------------------------------------------------------------- compute */

/* Sphere-trace and shade n_cams x H x W primary rays (Sec. 3.4.1), one per pixel centre.
 * cams: n_cams cameras in HOST memory (read before the call returns).  max_steps: SDF
 * evaluations per ray (>= 1).  eps: hit threshold on |d| (> 0).  out: device buffers of
 * n_cams*H*W pixels (kns_frame).  opts: NULL or precision options.  Rays start at the box
 * entry max(t_near, 0) and miss when t leaves [max(t_near, 0), t_far] or the budget is spent.
 * n_cams, W or H equal to 0 is a successful no-op.
 * Errors: INVALID_ARG (NULL grid/cams/out/rgb/depth, negative sizes, n_cams*W*H > 2^40,
 * max_steps < 1, eps <= 0 or not finite, unknown precision), CUDA. */
kns_status kns_render(kns_ctx *ctx, const kns_grid *grid, const kns_camera *cams, int n_cams,
                      int W, int H, int max_steps, float eps, const kns_render_opts *opts,
                      const kns_frame *out, void *cuda_stream);

/* Counters (and, when the render ran with opts->timing = 1, per-kernel-class device times) of the last
 * kns_render on this context.  Waits for that render to finish.  Errors: INVALID_ARG (no render yet), CUDA. */
kns_status kns_get_render_stats(kns_ctx *ctx, kns_render_stats *out);

/* One round of kns_render's wavefront sphere trace (Sec. 3.4.1): every ray still tracing takes its
 * next sample (and, in-tile, possibly a few more). */
typedef struct kns_round_info {
    int32_t live;        /* samples queued for the round */
    float ms_sort;       /* device time of the round's sort (scan and scatter), FP32 and BF16 evaluation and, */
    float ms_eval_fp32;  /* in a persistent BF16 trace, its empty-space walk: per-class CUDA events under     */
    float ms_eval_bf16;  /* opts->timing for host-driven rounds, the device timer for the persistent trace    */
    float ms_advance;
    int32_t tiles;       /* tensor-core tiles of the round (persistent BF16 trace; 0 otherwise) */
} kns_round_info;

/* Per-round trace of the last render call on this context: writes min(*n_rounds, max_rounds) entries
 * (rounds of all batches of the call, in order) and sets *n_rounds to the number of rounds.  Waits for
 * the render to finish.  Errors: INVALID_ARG (NULL n_rounds, out NULL with max_rounds > 0, no render
 * yet), CUDA. */
kns_status kns_get_round_trace(kns_ctx *ctx, kns_round_info *out, int32_t max_rounds, int32_t *n_rounds);

/* Measured throughput ceilings of the device a context runs on (for roofline reporting; not part of the
 * method): FP32 fused multiply-add in FLOP/s (2 per FMA) and the multi-function unit's ex2 in
 * operations/s, each from a micro-kernel with eight independent dependency chains per thread over every
 * SM, best of three timed launches; the SM count and the SM clock (kHz) the driver reports. */
typedef struct kns_peaks {
    double ffma_flops;
    double mufu_ops;
    int32_t sm_count;
    int32_t sm_clock_khz;
} kns_peaks;

/* Runs the micro-kernels on `cuda_stream` and waits for them (about 0.1 s).  Allocates a few KB of
 * device memory for the duration of the call.  Errors: INVALID_ARG (NULL), CUDA. */
kns_status kns_measure_peaks(kns_ctx *ctx, void *cuda_stream, kns_peaks *out);

/* Self-test of the failure path of the bounded device waits (not part of the method): runs, on
 * cuda_stream, a wait that nothing satisfies with a short poll limit -- which = 0: an mbarrier wait of
 * the kind a tensor-core tile makes for its weights and products; 1: the persistent trace's grid
 * barrier, with one of two blocks never arriving -- and waits for it.  The waiting threads give up,
 * record KNS_ERR_TIMEOUT in the context's status word (returned and cleared by the next kns_sync) and
 * return; the context stays usable.  Errors: INVALID_ARG (which not 0 or 1), CUDA. */
kns_status kns_selftest_timeout(kns_ctx *ctx, int32_t which, void *cuda_stream);

/* One view of a multi-view render: camera, image size, its own output buffers (device pointers for
 * W*H pixels, layout as kns_frame) and which grid of a stack it renders (0 for a single grid; its
 * output cell ids are that grid's). */
typedef struct kns_view {
    kns_camera cam;
    int32_t W, H;
    kns_frame out;
    int32_t grid;
    int32_t reserved; /* 0 */
} kns_view;

/* Sphere-trace and shade several views of one grid, or of the grids of a stack, in one launch sequence
 * (Sec. 3.4.1): the views may differ in camera, resolution and grid (requests of a render server).
 * views: host array, read before the call returns; each view writes only its own buffers, and every
 * pixel gets the same result as a kns_render of that view alone (of its grid loaded alone).  Views
 * with W*H = 0 are skipped.  Errors: INVALID_ARG (NULL grid or views, a view with negative size,
 * without rgb/depth or with a grid index outside the stack, more than 2^31-1 rays in total,
 * max_steps < 1, eps <= 0, bad opts), CUDA, OUT_OF_MEMORY. */
kns_status kns_render_views(kns_ctx *ctx, const kns_grid *grid, const kns_view *views, int n_views, int max_steps,
                            float eps, const kns_render_opts *opts, void *cuda_stream);

/* Sphere-trace and shade explicit rays (Sec. 3.4.1 for arbitrary rays, e.g. the bounce rays of a path
 * tracer): origins and unit directions (device, n x 3 FP32); ray k writes element k of every output
 * of `out` (device buffers of n elements; rgb and depth required, the rest nullable) exactly as
 * kns_render writes a pixel.  n = 0 is a successful no-op.  Errors: INVALID_ARG (NULL grid, rays or
 * rgb/depth, n out of [0, 2^31 - 4097], max_steps < 1, eps <= 0, bad opts), CUDA, OUT_OF_MEMORY. */
kns_status kns_trace_rays(kns_ctx *ctx, const kns_grid *grid, const float *origins, const float *dirs, int64_t n,
                          int max_steps, float eps, const kns_frame *out, const kns_render_opts *opts,
                          void *cuda_stream);

/* Lambertian path tracing (Sec. 3.4: the surface is treated as Lambertian; the colour network gives
 * its albedo, the normalised SDF gradient its normal).  Per path: a primary ray through the point
 * (j + u0, i + u1) of pixel (i, j); at each of at most max_depth traces a miss adds beta * E(w) and
 * ends the path, E(w) = (1 - a) horizon + a zenith with a = (w_z + 1) / 2; a hit multiplies beta by
 * the albedo and, below the last depth, continues from hit + offset * normal in a cosine-weighted
 * direction about the normal (a hit at the last depth gathers no light).  Random numbers: SplitMix64
 * outputs k = (path * 16 + depth) * 4 + dim of the generator seeded with `seed`, top 24 bits / 2^24;
 * path = pixel * spp + sample, pixel = (cam * H + i) * W + j. */
typedef struct {
    int32_t spp;          /* paths per pixel (>= 1) */
    int32_t max_depth;    /* traces per path (1..16) */
    uint64_t seed;
    float offset;         /* bounce origin offset along the normal (>= 0) */
    float horizon[3], zenith[3];
} kns_pt_opts;

/* Path-traced image: rgb_out (device, n_cams x H x W x 3, camera-major, row-major) gets the mean of
 * each pixel's spp paths.  cams: host array.  Tracing uses kns_render's sphere tracer with max_steps,
 * eps and opts.  Errors: INVALID_ARG (NULL grid/opts/cams/rgb_out, sizes or pt fields out of range,
 * more than 2^31 - 4097 paths), CUDA, OUT_OF_MEMORY. */
kns_status kns_path_trace(kns_ctx *ctx, const kns_grid *grid, const kns_camera *cams, int n_cams, int W, int H,
                          const kns_pt_opts *pt, int max_steps, float eps, float *rgb_out,
                          const kns_render_opts *opts, void *cuda_stream);

/* Batch field query (the vectorised per-cell MLP query of Sec. 3.3): for n points (device,
 * n x 3 FP32, row-major) evaluate the SDF MLP of cell m(x): sdf (device, n floats), feat (device,
 * n x feat_dim, or NULL), grad (device, n x 3 analytic input gradient, or NULL).
 * n = 0 is a successful no-op.  Errors: INVALID_ARG (NULL pts/sdf with n > 0, n < 0), CUDA. */
kns_status kns_sdf(kns_ctx *ctx, const kns_grid *grid, const float *pts, int64_t n, float *sdf,
                   float *feat, float *grad, void *cuda_stream);

/* ------------------------------------------------------- training step */

/* One batch of the fine-tuning loss of Sec. 3.2.2.  Device pointers, FP32, row-major.  Rays: origins
 * and unit directions (n_rays x 3), target colours (n_rays x 3).  The random draws of the step are
 * inputs: u_strat (n_rays x n_strat, in [0, 1)) jitters the stratified samples, u_imp (n_rays x
 * n_imp, each row ascending in [0, 1)) places the importance samples; eik_points (n_eik x 3) are the
 * eikonal points.  s: sharpness of the NeuS opacity Phi_s = sigmoid(s d) of the rendered samples;
 * s_up: the same for the coarse pass that places the importance samples; lambda: eikonal weight;
 * h: central-difference step of the SDF gradient (Sec. 3.3).  t_fixed (device, n_rays x (n_strat +
 * n_imp), each row ascending, or NULL): sample positions to render instead of placing them (the
 * coarse pass and u_strat, u_imp are then unused). */
typedef struct {
    int64_t n_rays;
    const float *origins, *dirs, *target;
    int32_t n_strat, n_imp; /* n_strat >= 2, n_strat + n_imp <= 256 */
    const float *u_strat, *u_imp;
    int64_t n_eik;
    const float *eik_points;
    float s, s_up, lambda, h;
    const float *t_fixed;
    int32_t timing; /* 1: time the phases with CUDA events (kns_train_get_stats) */
} kns_train_batch;

/* Work counts and, when the forward ran with timing = 1, per-phase device milliseconds of the latest
 * training forward (and its backward, once run).  Records are SDF evaluations: coarse samples,
 * central-difference points (6 per sample and per eikonal point) and sample centres. */
typedef struct {
    int64_t rays, eik_points;
    int32_t samples_per_ray, pad;
    int64_t records_coarse, records_fd, records_centre;
    float ms_coarse, ms_sort, ms_fd_forward, ms_centre_forward, ms_loss;
    float ms_upstream, ms_centre_backward, ms_fd_backward, ms_total;
} kns_train_stats;

/* Training loss (Sec. 3.2.2: L = L_color + lambda L_eikonal) of a Kilo-grid whose canonical FP32 weights
 * `params` (device, N^3 x params-per-cell) the caller owns, e.g. a framework parameter tensor.
 * Per ray (NeuS volume rendering with one importance pass): the box interval [t_n, t_f] gets n_strat
 * samples t_i = t_n + (i + u_i)/n_strat (t_f - t_n); their SDF values give coarse weights T_i alpha_i
 * (Phi_{s_up}); n_imp samples invert the CDF of those weights (+1e-5 per interval); all samples, merged
 * in order, are rendered: alpha_i = max(1 - Phi_s(d_{i+1}) / Phi_s(d_i), 0), T_i = prod_{j<i} (1 -
 * alpha_j), C = sum_i T_i alpha_i c_i (black background), with c_i the colour MLP on the cell's
 * feature, the normal g/|g| and gamma(v), where g is the central difference of d with step h, each
 * difference point evaluated in its own cell (Sec. 3.3).  L_color = mean over rays of |C - I|_1;
 * L_eikonal = mean over points of (|g| - 1)^2.  Sample positions are not differentiated.
 * loss: device, 3 floats written (L, L_color, L_eikonal).  rgb (device n_rays x 3) and t_samples
 * (device n_rays x (n_strat + n_imp); 0 for rays that miss the box) are optional outputs.
 * Supported shapes: sdf_width 32, sdf_hidden 2 or 3, pe_pos_L 4, pe_dir_L 2, col_use_x 0.
 * The pass keeps its state in the context for kns_train_backward and returns a token for it; the
 * next forward on the context replaces that state.  params and the batch arrays must stay valid and
 * unchanged until the backward has run.  Errors: INVALID_ARG (NULL pointers, counts or sizes out of
 * range, s, s_up, h <= 0, lambda < 0), UNSUPPORTED (grid shape), CUDA, OUT_OF_MEMORY. */
kns_status kns_train_forward(kns_ctx *ctx, const kns_grid_desc *desc, const float *params,
                             const kns_train_batch *batch, float *loss, float *rgb, float *t_samples,
                             uint64_t *token, void *cuda_stream);

/* Gradient of dloss * L (dloss: device scalar, NULL = 1) with respect to every weight of the forward
 * pass `token`, written to grad (device, canonical layout, same size as params; overwritten).  The
 * hand-written backward of the forward above: |.| and max(., 0) take derivative 0 at their kinks.
 * Errors: INVALID_ARG (token not the context's latest forward, NULL grad), CUDA. */
kns_status kns_train_backward(kns_ctx *ctx, uint64_t token, const float *dloss, float *grad, void *cuda_stream);

/* Statistics of the latest training forward/backward on the context (waits for its timing events).
 * Errors: INVALID_ARG (no forward yet), CUDA. */
kns_status kns_train_get_stats(kns_ctx *ctx, kns_train_stats *out);

/* kns_train_forward followed by kns_train_backward (grad NULL: forward only). */
kns_status kns_train_step(kns_ctx *ctx, const kns_grid_desc *desc, const float *params,
                          const kns_train_batch *batch, float *loss, float *grad, void *cuda_stream);

/* ------------------------------------------------------- allocation-free render */

/* Limits of kns_render_noalloc's built-in scratch. */
#define KNS_NOALLOC_MAX_RAYS 262144 /* n_cams * W * H per call */
#define KNS_NOALLOC_MAX_CELLS 32768 /* N^3 of the grid */
#define KNS_NOALLOC_MAX_CAMS 64

/* An FP32 render for callers that may not allocate device memory while they run: an application
 * that gives all device memory to its own pool allocator at start-up, or a latency-bound loop that
 * cannot take cudaMalloc's implicit device synchronisation.  The paper has no counterpart; it is a
 * deployment convenience.  It runs kns_render's FP32 wavefront on 16-sample warp tiles and the
 * one-warp-per-ray tail, without the cycle test (a cycling ray runs on until max_steps), and shades
 * like kns_render: the outputs are kns_render's.  Its scratch is a fixed device array built into
 * the library (about 14 MB on every GPU that loads it, kept until the process exits); the call
 * allocates nothing and frees nothing.  The context and the grid must already exist: creating them
 * allocates, and kns_create also loads the array on its device and looks up its address (should that
 * fail there, the first kns_render_noalloc on the device does it).  All calls
 * share the one array and each clears the counters it needs, so calls that overlap on the GPU race:
 * serialise them (one stream, or events).  Arguments, outputs and errors as kns_render, plus
 * INVALID_ARG when n_cams*W*H > KNS_NOALLOC_MAX_RAYS, n_cams > KNS_NOALLOC_MAX_CAMS or
 * N^3 > KNS_NOALLOC_MAX_CELLS. */
kns_status kns_render_noalloc(kns_ctx *ctx, const kns_grid *grid, const kns_camera *cams, int n_cams, int W,
                              int H, int max_steps, float eps, const kns_frame *out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* KNS_H_ */
