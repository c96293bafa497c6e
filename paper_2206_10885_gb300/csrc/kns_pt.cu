// kns_pt.cu -- Lambertian path tracing of the KiloNeuS surface (Sec. 3.4: the path tracer treats the
// surface as Lambertian; the colour network gives its albedo, the normalised SDF gradient its normal).
//
// The runtime traces every path's current ray with the wavefront (kns_trace_rays); these kernels
// make the primary rays, turn each trace result into the next ray, and average the paths of a pixel.
// Random numbers: SplitMix64 (Steele, Lea & Flood 2014), the k-th output of the generator seeded with
// `seed` being mix(seed + (k + 1) * 0x9E3779B97F4A7C15); a uniform is its top 24 bits times 2^-24;
// path p, trace depth t and dimension i use k = (p * 16 + t) * 4 + i.  Cosine-weighted directions
// use the branchless orthonormal basis of Duff et al. (JCGT 2017).
#include <cuda_runtime.h>
#include <stdint.h>

#include "kns_kernels.h"

namespace kns {
namespace {

constexpr int PT_MAXDEPTH = 16;

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float pt_uniform(uint64_t seed, int64_t path, int depth, int dim) {
    const uint64_t k = ((uint64_t)path * PT_MAXDEPTH + (uint64_t)depth) * 4u + (uint64_t)dim;
    return (float)(splitmix64(seed, k) >> 40) * 0x1p-24f;
}

__device__ __forceinline__ void cosine_dir(const float n[3], float u1, float u2, float w[3]) {
    const float sign = n[2] >= 0.f ? 1.f : -1.f;
    const float a = -1.f / (sign + n[2]);
    const float b = n[0] * n[1] * a;
    const float t[3] = {1.f + sign * n[0] * n[0] * a, sign * b, -sign * n[0]};
    const float bb[3] = {b, sign + n[1] * n[1] * a, -n[1]};
    const float r = sqrtf(u2), z = sqrtf(1.f - u2);
    float sp, cp;
    sincospif(2.f * u1, &sp, &cp);
#pragma unroll
    for (int k = 0; k < 3; ++k) w[k] = r * cp * t[k] + r * sp * bb[k] + z * n[k];
}

__device__ __forceinline__ void set_null_ray(const PtArgs &a, int64_t p) {
    // outside the box and moving away from it: the slab test misses at once
    a.o[3 * p] = a.bmax[0] + 1.f;
    a.o[3 * p + 1] = a.bmax[1] + 1.f;
    a.o[3 * p + 2] = a.bmax[2] + 1.f;
    a.w[3 * p] = 1.f;
    a.w[3 * p + 1] = 0.f;
    a.w[3 * p + 2] = 0.f;
}

__global__ void __launch_bounds__(256) k_pt_primary(PtArgs a) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.n_paths) return;
    const int64_t pix = p / a.spp;
    const int64_t hw = (int64_t)a.W * a.H;
    const int c = (int)(pix / hw);
    const int i = (int)((pix / a.W) % a.H), j = (int)(pix % a.W);
    const float *cam = a.cams + 16 * c;
    const float u0 = pt_uniform(a.seed, p, 0, 0), u1 = pt_uniform(a.seed, p, 0, 1);
    const float dx = ((float)j + u0 - cam[14]) / cam[12];
    const float dy = ((float)i + u1 - cam[15]) / cam[13];
    float w[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) w[r] = cam[4 * r] * dx + cam[4 * r + 1] * dy + cam[4 * r + 2];
    const float inv = 1.f / sqrtf(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        a.o[3 * p + r] = cam[4 * r + 3];
        a.w[3 * p + r] = w[r] * inv;
        a.beta[3 * p + r] = 1.f;
        a.L[3 * p + r] = 0.f;
    }
    a.alive[p] = 1;
}

// the trace result of depth `depth` -> light gathered and the next ray
__global__ void __launch_bounds__(256) k_pt_bounce(PtArgs a, int depth) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.n_paths || !a.alive[p]) return;
    float w[3] = {a.w[3 * p], a.w[3 * p + 1], a.w[3 * p + 2]};
    if (!a.t_hit[p]) {
        const float s = 0.5f * (w[2] + 1.f);
#pragma unroll
        for (int k = 0; k < 3; ++k) a.L[3 * p + k] += a.beta[3 * p + k] * ((1.f - s) * a.horizon[k] + s * a.zenith[k]);
        a.alive[p] = 0;
        set_null_ray(a, p);
        return;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) a.beta[3 * p + k] *= a.t_rgb[3 * p + k];
    if (depth + 1 >= a.max_depth) {  // a hit at the last depth gathers no light
        a.alive[p] = 0;
        set_null_ray(a, p);
        return;
    }
    const float t = a.t_depth[p];
    const float n[3] = {a.t_normal[3 * p], a.t_normal[3 * p + 1], a.t_normal[3 * p + 2]};
    float nw[3];
    cosine_dir(n, pt_uniform(a.seed, p, depth, 2), pt_uniform(a.seed, p, depth, 3), nw);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        a.o[3 * p + k] = a.o[3 * p + k] + t * w[k] + a.offset * n[k];
        a.w[3 * p + k] = nw[k];
    }
}

__global__ void __launch_bounds__(256) k_pt_resolve(PtArgs a) {
    const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= a.n_paths / a.spp) return;
    float acc[3] = {0.f, 0.f, 0.f};
    for (int s = 0; s < a.spp; ++s)
#pragma unroll
        for (int k = 0; k < 3; ++k) acc[k] += a.L[3 * (pix * a.spp + s) + k];
#pragma unroll
    for (int k = 0; k < 3; ++k) a.rgb_out[3 * pix + k] = acc[k] / (float)a.spp;
}

unsigned blocks_for(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

int pt_max_depth() { return PT_MAXDEPTH; }

cudaError_t pt_primary(const PtArgs &a, cudaStream_t s) {
    k_pt_primary<<<blocks_for(a.n_paths), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t pt_bounce(const PtArgs &a, int depth, cudaStream_t s) {
    k_pt_bounce<<<blocks_for(a.n_paths), 256, 0, s>>>(a, depth);
    return cudaGetLastError();
}

cudaError_t pt_resolve(const PtArgs &a, cudaStream_t s) {
    k_pt_resolve<<<blocks_for(a.n_paths / a.spp), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace kns
