// Helpers shared by the scoring kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "sam_internal.h"

namespace sam {

__device__ __forceinline__ float2 load_field(const float2 *f, size_t i) { return __ldg(f + i); }
__device__ __forceinline__ float2 load_field(const __nv_bfloat162 *f, size_t i) {
    return __bfloat1622float2(__ldg(f + i));
}
__device__ __forceinline__ float2 load_field(const __half2 *f, size_t i) { return __half22float2(__ldg(f + i)); }

// Per-term error bound of the stored unit field (component rounding).
inline float term_eps(int precision) {
    return precision == SAM_FP32 ? 1e-6f : (precision == SAM_FP16 ? 1e-3f : 4e-3f);
}

// Early termination: prune when S_j + (n - j) < n * min_score - margin,
// margin = 1e-3 + n * eps_term; returns the right-hand side.
inline float prune_threshold(int n, float min_score, int precision) {
    return (float)n * min_score - (1e-3f + (float)n * term_eps(precision));
}

}  // namespace sam
