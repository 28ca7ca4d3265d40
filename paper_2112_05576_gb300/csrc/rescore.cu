// FP32 rescoring of a score map computed from a 16-bit stored field.
//
// A unit vector stored in FP16 (BF16) moves each component by at most 2^-12
// (2^-9), so each Eq. (1) term moves by at most sqrt(2) times that; the
// 16-bit scorers also round the point direction to the field's type, doubling
// the bound.  The score M -- a mean of per-point maxima of such terms --
// therefore moves by at most delta = 6.9e-4 (FP16) or 5.5e-3 (BF16), plus
// FP32 rounding.  After the
// exhaustive 16-bit
// search, every pose with M16 >= min_score - delta is therefore rescored from
// the FP32 field, and every other pose (including poses the 16-bit kernel
// pruned) is provably below min_score in FP32 and is written -inf.  Candidate
// extraction then sees FP32 scores wherever a pose can reach min_score, so
// the detections equal those of the FP32 path.
//
// Two kernels: a grid-stride scan that applies the -inf rule and appends the
// poses to rescore to a list, and one warp per listed pose (lanes over model
// points, compensated per-lane sums, shuffle tree) that writes the FP32 score.

#include <algorithm>

#include "sam_internal.h"
#include "score_common.cuh"

namespace sam {
namespace {

// The -inf rule and the rescoring list over `count` maps (grid-stride).
__global__ void rescore_select_kernel(float *__restrict__ map, size_t map_img, size_t per_img, float thr,
                                      unsigned *__restrict__ list, unsigned *__restrict__ count, unsigned cap) {
    const int img = blockIdx.y;
    float *m = map + (size_t)img * map_img;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < per_img; i += (size_t)gridDim.x * blockDim.x) {
        const float s = m[i];
        if (s >= thr) {
            const unsigned pos = atomicAdd(count, 1u);
            if (pos < cap) {
                list[2 * (size_t)pos] = (unsigned)img;
                list[2 * (size_t)pos + 1] = (unsigned)i;
            } else {
                m[i] = __int_as_float(0x7fc00000);   // list full: flag the pose NaN
            }
        } else {
            m[i] = -INFINITY;
        }
    }
}

// Eq. (1) in FP32 from the FP32 field for every listed pose, one warp each.
template <int NB>
__global__ void __launch_bounds__(256) rescore_kernel(const float2 *__restrict__ field, size_t field_img_px, int w,
                                                      int h, int gw, int gh, int step_x, int step_y, int x0, int y0,
                                                      int k0, const RotPt *__restrict__ rot, int n, int polarity,
                                                      float *__restrict__ map, size_t map_img,
                                                      const unsigned *__restrict__ list,
                                                      const unsigned *__restrict__ count, unsigned cap) {
    const unsigned total = min(*count, cap);
    const int lane = threadIdx.x & 31;
    const unsigned warps = (gridDim.x * blockDim.x) >> 5;
    constexpr int R = NB / 2;
    for (unsigned e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < total; e += warps) {
        const unsigned img = list[2 * (size_t)e], idx = list[2 * (size_t)e + 1];
        const unsigned plane = (unsigned)gw * (unsigned)gh;
        const int kl = (int)(idx / plane);
        const int rem = (int)(idx - (unsigned)kl * plane);
        const int gyi = rem / gw;
        const int ux = x0 + (rem - gyi * gw) * step_x, uy = y0 + gyi * step_y;
        const int k = k0 + kl;
        const float2 *F = field + (size_t)img * field_img_px;
        const RotPt *P = rot + (size_t)k * n;
        float sum = 0.f, comp = 0.f;
        for (int i = lane; i < n; i += 32) {
            const RotPt p = P[i];
            float best = -INFINITY;
#pragma unroll
            for (int b = -R; b <= R; ++b)
#pragma unroll
                for (int a = -R; a <= R; ++a) {
                    const int x = ux + p.ox + a, y = uy + p.oy + b;
                    float v = 0.f;
                    if (x >= 0 && y >= 0 && x < w && y < h) {
                        const float2 f = __ldg(F + (size_t)y * w + x);
                        v = fmaf(p.px, f.x, p.py * f.y);
                        if (polarity)
                            v = fabsf(v);
                    }
                    best = fmaxf(best, v);
                }
            const float yk = best - comp;
            const float t = sum + yk;
            comp = (t - sum) - yk;
            sum = t;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0)
            map[(size_t)img * map_img + idx] = sum / (float)n;
    }
}

// Job-list forms: blockIdx.y is the job.
__global__ void rescore_select_jobs_kernel(const RescoreJob *__restrict__ jobs, float thr) {
    const RescoreJob J = jobs[blockIdx.y];
    const size_t per = (size_t)J.nth * J.w * J.h;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < per; i += (size_t)gridDim.x * blockDim.x) {
        const float s = J.map[i];
        if (s >= thr) {
            const unsigned pos = atomicAdd(J.count, 1u);
            if (pos < J.cap) {
                J.list[2 * (size_t)pos] = 0u;
                J.list[2 * (size_t)pos + 1] = (unsigned)i;
            } else {
                J.map[i] = __int_as_float(0x7fc00000);
            }
        } else {
            J.map[i] = -INFINITY;
        }
    }
}

template <int NB>
__global__ void __launch_bounds__(256) rescore_jobs_kernel(const RescoreJob *__restrict__ jobs, int polarity) {
    const RescoreJob J = jobs[blockIdx.y];
    const unsigned total = min(*J.count, J.cap);
    const int lane = threadIdx.x & 31;
    const unsigned warps = (gridDim.x * blockDim.x) >> 5;
    constexpr int R = NB / 2;
    const unsigned plane = (unsigned)J.w * (unsigned)J.h;
    for (unsigned e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < total; e += warps) {
        const unsigned idx = J.list[2 * (size_t)e + 1];
        const int k = (int)(idx / plane);
        const int rem = (int)(idx - (unsigned)k * plane);
        const int uy = rem / J.w, ux = rem - uy * J.w;
        const RotPt *P = J.rot + (size_t)k * J.n;
        float sum = 0.f, comp = 0.f;
        for (int i = lane; i < J.n; i += 32) {
            const RotPt p = P[i];
            float best = -INFINITY;
#pragma unroll
            for (int b = -R; b <= R; ++b)
#pragma unroll
                for (int a = -R; a <= R; ++a) {
                    const int x = ux + p.ox + a, y = uy + p.oy + b;
                    float v = 0.f;
                    if (x >= 0 && y >= 0 && x < J.w && y < J.h) {
                        const float2 f = __ldg(J.field + (size_t)y * J.w + x);
                        v = fmaf(p.px, f.x, p.py * f.y);
                        if (polarity)
                            v = fabsf(v);
                    }
                    best = fmaxf(best, v);
                }
            const float yk = best - comp;
            const float t = sum + yk;
            comp = (t - sum) - yk;
            sum = t;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0)
            J.map[idx] = sum / (float)J.n;
    }
}

}  // namespace

float rescore_delta(int precision) {
    // storage error bound of M plus FP32 rounding slack
    return precision == SAM_FP16 ? 8e-4f : (precision == SAM_BF16 ? 6e-3f : 0.f);
}

size_t rescore_scratch_bytes(size_t poses) { return 256 + poses * 8; }

cudaError_t launch_rescore(const LevelDev &L, const float2 *field32, size_t field_img_px, int w, int h, int step_x,
                           int step_y, int count, int nbhd, int polarity, float min_score, int precision, float *map,
                           size_t map_img, void *scratch, size_t poses_cap, cudaStream_t st,
                           const PoseWindow *window) {
    unsigned *cnt = reinterpret_cast<unsigned *>(scratch);
    unsigned *list = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(scratch) + 256);
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(unsigned), st);
    if (e != cudaSuccess)
        return e;
    const PoseWindow pw =
        window ? *window : PoseWindow{0, 0, (w + step_x - 1) / step_x, (h + step_y - 1) / step_y, 0, L.ntheta};
    const int gw = pw.gw, gh = pw.gh;
    const size_t per_img = (size_t)pw.nk * gw * gh;
    const float thr = min_score - rescore_delta(precision);
    const unsigned cap = (unsigned)std::min<size_t>(poses_cap, 0xFFFFFFFFu);
    dim3 g1((unsigned)std::min<size_t>((per_img + 255) / 256, 1024), (unsigned)count);
    rescore_select_kernel<<<g1, 256, 0, st>>>(map, map_img, per_img, thr, list, cnt, cap);
    const unsigned blocks = 152 * 8;
    if (nbhd == 3)
        rescore_kernel<3><<<blocks, 256, 0, st>>>(field32, field_img_px, w, h, gw, gh, step_x, step_y, pw.x0, pw.y0,
                                                  pw.k0, L.rot, L.n, polarity, map, map_img, list, cnt, cap);
    else
        rescore_kernel<1><<<blocks, 256, 0, st>>>(field32, field_img_px, w, h, gw, gh, step_x, step_y, pw.x0, pw.y0,
                                                  pw.k0, L.rot, L.n, polarity, map, map_img, list, cnt, cap);
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace sam

namespace sam {

cudaError_t launch_rescore_jobs(const RescoreJob *jobs, int n_jobs, size_t max_map, int nbhd, int polarity,
                                float min_score, int precision, cudaStream_t st) {
    if (n_jobs <= 0)
        return cudaSuccess;
    const float thr = min_score - rescore_delta(precision);
    dim3 g1((unsigned)std::max<size_t>(1, std::min<size_t>((max_map + 255) / 256, 256)), (unsigned)n_jobs);
    rescore_select_jobs_kernel<<<g1, 256, 0, st>>>(jobs, thr);
    dim3 g2(8, (unsigned)n_jobs);
    if (nbhd == 3)
        rescore_jobs_kernel<3><<<g2, 256, 0, st>>>(jobs, polarity);
    else
        rescore_jobs_kernel<1><<<g2, 256, 0, st>>>(jobs, polarity);
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace sam
