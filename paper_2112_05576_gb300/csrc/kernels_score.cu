// Kernel (c): exhaustive score map of one pyramid level (Sec. II, CPU and
// GPU designs: every pose (x, y, theta) scored by Eq. (1) over the model
// points projected by Eq. (2), each point taking its best vote over the
// neighbouring-search window).
//
// This file holds the generic path: one thread per pose, the angle's
// rotated points read through the read-only cache (every thread of a block
// reads the same point at the same time), neighbouring w_hat samples read
// with coalesced loads (adjacent threads score adjacent x).  It handles
// any translation step and both window sizes, and is the cross-check of the
// tiled kernel in score_tiled.cu.
//
// Early termination (exact-safe): after j of n terms with partial sum S_j,
// every remaining term is at most 1, so the pose's score cannot reach
// min_score when S_j + (n - j) < n * min_score - margin.  The margin covers
// the FP32 rounding of S_j and the storage rounding of w_hat:
// margin = 1e-3 + n * eps_term (eps_term 1e-6 FP32, 1e-3 FP16, 6e-3 BF16).
// Pruned poses are written as -inf.

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "sam_internal.h"
#include "score_common.cuh"

namespace sam {
namespace {

// One thread per pose (x, y) of angle blockIdx.y (Eq. (1) over the Eq. (2)
// projections, neighbouring search NB), image blockIdx.z.
template <typename E, int LAYOUT, int NB>
__global__ void __launch_bounds__(256)
    score_map_generic(const E *__restrict__ field, size_t field_img_px, int pitch, int w, int h,
                      const RotPt *__restrict__ rot, int n, int step_x, int step_y, int gw, int gh, int polarity,
                      float prune_thresh, int early, float *__restrict__ map, size_t map_img) {
    const int img = blockIdx.z, k = blockIdx.y;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= gw * gh)
        return;
    field += 2 * (size_t)img * field_img_px;
    const int gxi = idx % gw, gyi = idx / gw;
    const int ux = gxi * step_x, uy = gyi * step_y;
    const RotPt *P = rot + (size_t)k * n;
    constexpr int R = NB / 2;
    float sum = 0.f, comp = 0.f;   // compensated (Kahan) sum
    bool pruned = false;
    for (int i = 0; i < n; ++i) {
        const RotPt p = P[i];
        const int x0 = ux + p.ox, y0 = uy + p.oy;
        float best = -INFINITY;
#pragma unroll
        for (int b = -R; b <= R; ++b) {
#pragma unroll
            for (int a = -R; a <= R; ++a) {
                const int x = x0 + a, y = y0 + b;
                float v = 0.f;
                if (x >= 0 && y >= 0 && x < w && y < h) {
                    const float2 f = load_field<E, LAYOUT>(field, pitch, x, y);
                    // 16-bit fields: the direction is rounded to the same
                    // type and the product px*wx is exact, matching the tiled
                    // kernel's mixed-precision FMA bit for bit
                    const float px = dir_round<E>(p.px), py = dir_round<E>(p.py);
                    v = fmaf(py, f.y, px * f.x);
                    if (polarity)
                        v = fabsf(v);
                }
                best = fmaxf(best, v);
            }
        }
        const float yk = best - comp;
        const float t = sum + yk;
        comp = (t - sum) - yk;
        sum = t;
        if (early && sum + (float)(n - 1 - i) < prune_thresh) {
            pruned = true;
            break;
        }
    }
    map[(size_t)img * map_img + ((size_t)k * gh + gyi) * gw + gxi] = pruned ? -INFINITY : sum / (float)n;
}

template <typename E, int LAYOUT>
cudaError_t launch_generic_t(const LevelDev &L, const ScoreArgs &a, cudaStream_t st) {
    const int gw = (a.w + a.step_x - 1) / a.step_x, gh = (a.h + a.step_y - 1) / a.step_y;
    const float thresh = prune_threshold(L.n, a.min_score, a.precision);
    dim3 grid((unsigned)((gw * gh + 255) / 256), (unsigned)L.ntheta, (unsigned)a.count);
    const E *f = reinterpret_cast<const E *>(a.field);
    const int pitch = field_pitch(a.w, LAYOUT);
    if (a.nbhd == 3)
        score_map_generic<E, LAYOUT, 3><<<grid, 256, 0, st>>>(f, a.field_img_px, pitch, a.w, a.h, L.rot, L.n,
                                                              a.step_x, a.step_y, gw, gh, a.polarity, thresh,
                                                              a.early, a.map, a.map_img);
    else
        score_map_generic<E, LAYOUT, 1><<<grid, 256, 0, st>>>(f, a.field_img_px, pitch, a.w, a.h, L.rot, L.n,
                                                              a.step_x, a.step_y, gw, gh, a.polarity, thresh,
                                                              a.early, a.map, a.map_img);
    count_launches(1);
    return cudaGetLastError();
}

template <typename E>
cudaError_t launch_generic_e(const LevelDev &L, const ScoreArgs &a, cudaStream_t st) {
    return a.layout == SAM_LAYOUT_PAIRS ? launch_generic_t<E, SAM_LAYOUT_PAIRS>(L, a, st)
                                        : launch_generic_t<E, SAM_LAYOUT_PIXEL>(L, a, st);
}

}  // namespace

cudaError_t launch_score_map_generic(const LevelDev &L, const ScoreArgs &a, cudaStream_t st) {
    switch (a.precision) {
    case SAM_FP32:
        return launch_generic_e<float>(L, a, st);
    case SAM_BF16:
        return launch_generic_e<__nv_bfloat16>(L, a, st);
    default:
        return launch_generic_e<__half>(L, a, st);
    }
}

}  // namespace sam
