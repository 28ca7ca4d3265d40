// Sub-pixel and sub-angle poses: the quadratic fit of the 3x3x3
// neighbourhood of Eq. (1) scores around an integer level-0 pose.  The
// paper's search is digitised (pixel and angle steps); this refines its
// final poses without a continuous score.  The coarse-to-fine descent can
// stop at the edge of its 27-pose window, so the pose first moves to the
// best of its 27 neighbours until none scores strictly higher (at most
// kMaxMoves moves; among equal best neighbours the first in (dk, dy, dx)
// order), then the neighbourhood of that pose is fitted.
//
// One CTA per pose: the threads split the model points, each thread scores
// the 27 poses (x + dx, y + dy, k + dk) of its points -- for one point and
// one angle the (N + 2) x (N + 2) dot products around the projected point
// (N the neighbourhood size) serve all nine translations -- and a block
// reduction gives the 27 sums.  Thread 0 then fits, in FP64:
//   g_a = (M(+a) - M(-a)) / 2,  H_aa = M(+a) - 2 M(0) + M(-a),
//   H_ab = (M(+a+b) - M(+a-b) - M(-a+b) + M(-a-b)) / 4,
//   delta = -H^-1 g when H is negative definite, else per axis -g_a / H_aa
//   where H_aa < 0 (0 elsewhere); each component clamped to [-1/2, 1/2].

#include <math.h>
#include <stdint.h>

#include "sam_internal.h"

namespace sam {
namespace {

constexpr int kSubThreads = 256;
constexpr int kMaxMoves = 8;

struct SubField {
    const float2 *f;
    int w, h, pitch;
};

struct SubArgs {
    const RotPt *rot;   // level-0 rotated points [nth][n]
    int n, nth;
    int polarity;
    double angle_step;   // degrees per angle index at level 0
    int n_fields;
    SubField fields[SAM_MAX_BILINEAR_FIELDS];
};

template <int NB>
__global__ void __launch_bounds__(kSubThreads) subpixel_kernel(const __grid_constant__ SubArgs a,
                                                               const int32_t *__restrict__ pose_field,
                                                               const int32_t *__restrict__ kyx, int n_poses,
                                                               float *__restrict__ out) {
    __shared__ float red[kSubThreads / 32][27];
    __shared__ int s_pose[4];   // k, y, x, done
    __shared__ double s_sc[27];
    const int b = blockIdx.x;
    if (b >= n_poses)
        return;
    const int fi = pose_field ? pose_field[b] : 0;
    const bool ok = fi >= 0 && fi < a.n_fields && kyx[3 * b] >= 0 && kyx[3 * b] < a.nth;
    if (threadIdx.x == 0) {
        s_pose[0] = kyx[3 * b];
        s_pose[1] = kyx[3 * b + 1];
        s_pose[2] = kyx[3 * b + 2];
        s_pose[3] = 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int move = 0; move <= kMaxMoves; ++move) {
        const int k = s_pose[0], y = s_pose[1], x = s_pose[2];
        float acc[27];
#pragma unroll
        for (int q = 0; q < 27; ++q)
            acc[q] = 0.f;
        if (ok) {
            const SubField F = a.fields[fi];
            constexpr int D = NB + 2;   // dot-product window side
#pragma unroll
            for (int dk = 0; dk < 3; ++dk) {
                const int kk = (k + dk - 1 + a.nth) % a.nth;
                const RotPt *P = a.rot + (size_t)kk * a.n;
                for (int i = threadIdx.x; i < a.n; i += kSubThreads) {
                    const RotPt p = P[i];
                    const int bx = x + p.ox, by = y + p.oy;
                    float d[D][D];
#pragma unroll
                    for (int yy = 0; yy < D; ++yy)
#pragma unroll
                        for (int xx = 0; xx < D; ++xx) {
                            const int X = bx + xx - D / 2, Y = by + yy - D / 2;
                            float v = 0.f;
                            if (X >= 0 && Y >= 0 && X < F.w && Y < F.h) {
                                const float2 w = __ldg(F.f + (size_t)Y * F.pitch + X);
                                v = fmaf(p.px, w.x, p.py * w.y);
                                if (a.polarity)
                                    v = fabsf(v);
                            }
                            d[yy][xx] = v;
                        }
#pragma unroll
                    for (int ty = 0; ty < 3; ++ty)
#pragma unroll
                        for (int tx = 0; tx < 3; ++tx) {
                            float m = -INFINITY;
#pragma unroll
                            for (int u = 0; u < NB; ++u)
#pragma unroll
                                for (int v = 0; v < NB; ++v)
                                    m = fmaxf(m, d[ty + u][tx + v]);
                            acc[dk * 9 + ty * 3 + tx] += m;
                        }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 27; ++q) {
            float v = acc[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0)
                red[warp][q] = v;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int j = 13;
            double best = 0.0;
            for (int q = 0; q < 27; ++q) {
                double v = 0.0;
                for (int w = 0; w < kSubThreads / 32; ++w)
                    v += red[w][q];
                s_sc[q] = v / a.n;
            }
            best = s_sc[13];
            for (int q = 0; q < 27; ++q)
                if (s_sc[q] > best) {
                    best = s_sc[q];
                    j = q;
                }
            if (j == 13 || move == kMaxMoves || !ok) {
                s_pose[3] = 1;
            } else {
                s_pose[0] = (k + j / 9 - 1 + a.nth) % a.nth;
                s_pose[1] = y + (j / 3) % 3 - 1;
                s_pose[2] = x + j % 3 - 1;
            }
        }
        __syncthreads();
        if (s_pose[3])
            break;
    }
    if (threadIdx.x != 0)
        return;
    float *o = out + 4 * (size_t)b;
    if (!ok) {
        o[0] = o[1] = o[2] = o[3] = NAN;
        return;
    }
    const int k = s_pose[0], y = s_pose[1], x = s_pose[2];
    const double *s = s_sc;
    // s[(dk + 1) * 9 + (dy + 1) * 3 + (dx + 1)]
    auto S = [&](int dk, int dy, int dx) { return s[(dk + 1) * 9 + (dy + 1) * 3 + (dx + 1)]; };
    const double c = S(0, 0, 0);
    const double g0 = 0.5 * (S(0, 0, 1) - S(0, 0, -1));
    const double g1 = 0.5 * (S(0, 1, 0) - S(0, -1, 0));
    const double g2 = 0.5 * (S(1, 0, 0) - S(-1, 0, 0));
    const double hxx = S(0, 0, 1) - 2.0 * c + S(0, 0, -1);
    const double hyy = S(0, 1, 0) - 2.0 * c + S(0, -1, 0);
    const double hkk = S(1, 0, 0) - 2.0 * c + S(-1, 0, 0);
    const double hxy = 0.25 * (S(0, 1, 1) - S(0, -1, 1) - S(0, 1, -1) + S(0, -1, -1));
    const double hxk = 0.25 * (S(1, 0, 1) - S(-1, 0, 1) - S(1, 0, -1) + S(-1, 0, -1));
    const double hyk = 0.25 * (S(1, 1, 0) - S(-1, 1, 0) - S(1, -1, 0) + S(-1, -1, 0));
    // A = -H; delta = A^-1 g by cofactors when A is positive definite
    const double a00 = -hxx, a01 = -hxy, a02 = -hxk, a11 = -hyy, a12 = -hyk, a22 = -hkk;
    const double c00 = a11 * a22 - a12 * a12, c01 = a02 * a12 - a01 * a22, c02 = a01 * a12 - a02 * a11;
    const double det = a00 * c00 + a01 * c01 + a02 * c02;
    double dx, dy, dk;
    if (a00 > 0.0 && a00 * a11 - a01 * a01 > 0.0 && det > 0.0) {
        const double c11 = a00 * a22 - a02 * a02, c12 = a01 * a02 - a00 * a12, c22 = a00 * a11 - a01 * a01;
        dx = (c00 * g0 + c01 * g1 + c02 * g2) / det;
        dy = (c01 * g0 + c11 * g1 + c12 * g2) / det;
        dk = (c02 * g0 + c12 * g1 + c22 * g2) / det;
    } else {
        dx = hxx < 0.0 ? -g0 / hxx : 0.0;
        dy = hyy < 0.0 ? -g1 / hyy : 0.0;
        dk = hkk < 0.0 ? -g2 / hkk : 0.0;
    }
    dx = fmin(0.5, fmax(-0.5, dx));
    dy = fmin(0.5, fmax(-0.5, dy));
    dk = fmin(0.5, fmax(-0.5, dk));
    double th = fmod((k + dk) * a.angle_step, 360.0);
    if (th < 0.0)
        th += 360.0;
    o[0] = (float)(x + dx);
    o[1] = (float)(y + dy);
    o[2] = (float)th;
    o[3] = (float)c;
}

}  // namespace
}  // namespace sam

using namespace sam;

extern "C" sam_status sam_subpixel_poses(sam_model *m, const sam_field_ref *fields, int n_fields,
                                         const int32_t *pose_field, const int32_t *kyx, int n_poses,
                                         int neighbourhood, float *out, void *stream) {
    if (!m || !fields || n_fields < 1 || n_fields > SAM_MAX_BILINEAR_FIELDS || n_poses < 0 ||
        (neighbourhood != 1 && neighbourhood != 3) || (n_poses > 0 && (!kyx || !out)) || m->nscales != 1 ||
        m->scale_min != 1.0)   // the fit's neighbourhood is (x, y, angle): rigid models
        return SAM_ERR_ARG;
    for (int i = 0; i < n_fields; ++i) {
        const sam_field_ref &f = fields[i];
        if (!f.field || f.w < 1 || f.h < 1 || f.pitch < f.w || (uintptr_t)f.field % 8)
            return SAM_ERR_ARG;
    }
    sam_status s = upload_model(m);
    if (s != SAM_OK || n_poses == 0)
        return s;
    SubArgs a;
    a.rot = m->dev[0].rot;
    a.n = m->dev[0].n;
    a.nth = m->lv[0].ntheta;
    a.polarity = m->p.polarity ? 1 : 0;
    a.angle_step = m->p.angle_step_deg;
    a.n_fields = n_fields;
    for (int i = 0; i < SAM_MAX_BILINEAR_FIELDS; ++i)
        a.fields[i] = i < n_fields ? SubField{(const float2 *)fields[i].field, fields[i].w, fields[i].h,
                                              fields[i].pitch}
                                   : SubField{nullptr, 0, 0, 0};
    cudaStream_t st = (cudaStream_t)stream;
    if (neighbourhood == 3)
        subpixel_kernel<3><<<n_poses, kSubThreads, 0, st>>>(a, pose_field, kyx, n_poses, out);
    else
        subpixel_kernel<1><<<n_poses, kSubThreads, 0, st>>>(a, pose_field, kyx, n_poses, out);
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? SAM_OK : SAM_ERR_CUDA;
}
