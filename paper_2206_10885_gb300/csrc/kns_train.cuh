// kns_train.cuh -- device helpers shared by the training-step kernels (kns_train.cu, kns_train_tile.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kns_kernels.h"

namespace kns {
namespace train {

constexpr int CHUNK = 4096;  // records of one cell per work chunk
constexpr int MAXS = 256;    // samples per ray

__device__ __forceinline__ void load3(const float *p, float *v) {
    v[0] = __ldg(p);
    v[1] = __ldg(p + 1);
    v[2] = __ldg(p + 2);
}

// central-difference gradient g of d at sample (or eikonal point) q from its six difference records,
// and n = g / |g|; returns |g| (n = 0 when |g| = 0)
__device__ __forceinline__ float fd_normal(const TrainArgs &a, int64_t q, float (&g)[3], float (&n)[3]) {
    const float inv2h = 1.f / (2.f * a.h);
    const float *d = a.d_fd + 6 * q;
#pragma unroll
    for (int k = 0; k < 3; ++k) g[k] = (d[2 * k] - d[2 * k + 1]) * inv2h;
    const float gn = sqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    const float ig = gn > 0.f ? 1.f / gn : 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) n[k] = g[k] * ig;
    return gn;
}

// chunk c of keys [k0, k1): its key, the largest k with chunk_off[k] <= c
__device__ __forceinline__ int chunk_key(const int *chunk_off, int k0, int k1, int c) {
    int lo = k0, hi = k1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(chunk_off + mid) <= c) lo = mid;
        else hi = mid;
    }
    return lo;
}

inline int grid_for(int sm_count, int per_sm, int64_t work_upper) {
    int64_t b = (int64_t)sm_count * per_sm;
    if (work_upper < b) b = work_upper;
    return (int)(b > 0 ? b : 1);
}

}  // namespace train
}  // namespace kns
