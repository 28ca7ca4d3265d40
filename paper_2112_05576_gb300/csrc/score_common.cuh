// Helpers shared by the scoring kernels.
#pragma once

#include <cmath>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "sam_internal.h"

namespace sam {

__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f32(__half v) { return __half2float(v); }

// (wx, wy) of pixel (x, y) of a field in either layout; E is the component
// type (float, bf16, fp16), pitch the row pitch in pixels.
template <typename E, int LAYOUT>
__device__ __forceinline__ float2 load_field(const E *f, int pitch, int x, int y) {
    if (LAYOUT == SAM_LAYOUT_PAIRS) {
        const size_t q4 = 2 * ((size_t)y * pitch + (x & ~1));
        return make_float2(to_f32(__ldg(f + q4 + (x & 1))), to_f32(__ldg(f + q4 + 2 + (x & 1))));
    }
    const size_t i = 2 * ((size_t)y * pitch + x);
    return make_float2(to_f32(__ldg(f + i)), to_f32(__ldg(f + i + 1)));
}

// The point direction as the scoring arithmetic sees it: 16-bit fields are
// scored with directions rounded to the same type (mixed-precision FMA, exact
// 16-bit products), FP32 fields in FP32.
template <typename E>
__device__ __forceinline__ float dir_round(float v) {
    return v;
}
template <>
__device__ __forceinline__ float dir_round<__half>(float v) {
    return __half2float(__float2half_rn(v));
}
template <>
__device__ __forceinline__ float dir_round<__nv_bfloat16>(float v) {
    return __bfloat162float(__float2bfloat16_rn(v));
}

// Per-term error bound of 16-bit storage against exact arithmetic: each
// component of the unit field and of the direction is rounded by at most
// 2^-12 (FP16) or 2^-9 (BF16), so a term moves by at most 2 sqrt(2) times
// that (6.9e-4, 5.5e-3), plus FP32 rounding.
inline float term_eps(int precision) {
    // angle codes are expanded to FP32 unit vectors (within 2.4e-7 of exact)
    // and scored in FP32 like an FP32 field
    if (precision == SAM_FP32 || precision == SAM_ANGLE16)
        return 1e-6f;
    return precision == SAM_FP16 ? 1e-3f : 6e-3f;
}

// Early termination: prune when S_j + (n - j) < n * min_score - margin,
// margin = 1e-3 + n * eps_term; returns the right-hand side.
inline float prune_threshold(int n, float min_score, int precision) {
    return (float)n * min_score - (1e-3f + (float)n * term_eps(precision));
}

// Edge-presence bound: a point's vote is 0 unless its 3x3 window holds an
// edge pixel, and at most 1 + eps_term otherwise, so a pose whose count E of
// such points satisfies E (1 + eps_term) < thresh is below min_score.  The
// smallest E that can survive, less one for safety (0: never prunes).
inline int edge_count_threshold(float thresh, int precision) {
    if (!(thresh > 0.f))
        return 0;
    const double t = std::ceil((double)thresh / (1.0 + (double)term_eps(precision))) - 1.0;
    return t > 0.0 ? (int)t : 0;
}

}  // namespace sam
