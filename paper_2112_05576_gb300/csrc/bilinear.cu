// Differentiable score on continuous poses, its adjoint, and one-launch
// damped Gauss-Newton refinement of many poses.
//
// M_c(x, y, theta) = (1/n) sum_i d_i . w_bil(p_i), with p_i = R(theta) t_i +
// (x, y) (Eq. (2) without rounding), d_i = R(theta) g_i/|g_i| and w_bil the
// bilinear sample of the unit search field (Eq. (1) at a continuous pose,
// without the neighbourhood maximum).  Inside the pixel cell of p_i, with
// d0 = w10 - w00, d1 = w11 - w01, top = w00 + fx d0, bot = w01 + fx d1:
//   w_bil = top + fy (bot - top),  dw/dx = d0 + fy (d1 - d0),  dw/dy = bot - top.
// With r_i = R(theta) t_i, dR/dtheta = R(theta) turned by 90 degrees gives
// d(d_i)/dtheta = (-d_iy, d_ix) and d(p_i)/dtheta = (-r_iy, r_ix), so
//   dterm/dx = d . dw/dx,  dterm/dy = d . dw/dy,
//   dterm/dtheta = [d_x w_y - d_y w_x + r_x dterm/dy - r_y dterm/dx] pi/180.
//
// One CTA per pose; lanes stride over the model points (the unrotated
// (tx, ty, ux, uy) table, shared by every pose and L2-resident), gather the
// four field pixels around each sample with read-only loads, and accumulate
// in FP32 registers; a shuffle tree and a fixed-order sum over the warps
// reduce.  The pose's sin/cos come from FP64 sincospi once per CTA.  Sample
// coordinates are formed as (integer part of x) + (fraction of x + r_x), so
// the fraction keeps FP32 resolution however large the image is.
//
// The refinement kernel keeps each CTA on its pose for all iterations: one
// evaluation of M_c and its normal equations per iteration, the 3x3 damped
// system solved in FP64 by one thread, the pose carried in FP64.

#include <math.h>
#include <stdint.h>

#include "sam_internal.h"

namespace sam {
namespace {

constexpr int kBilThreads = 128;
constexpr int kBilWarps = kBilThreads / 32;
constexpr float kDegToRad = 0.017453292519943295f;

struct BilField {
    const float2 *f;
    int w, h, pitch;
};

struct BilArgs {
    const float4 *pts;
    int n;
    int polarity;
    int n_fields;
    BilField fields[SAM_MAX_BILINEAR_FIELDS];
};

// Pose split for the per-point arithmetic.
struct PoseF {
    int xi, yi;     // integer parts
    float xf, yf;   // fractions in [0, 1)
    float c, s;     // cos, sin of theta
    bool ok;
};

__device__ __forceinline__ PoseF split_pose(double x, double y, double th) {
    PoseF q;
    q.ok = isfinite(x) && isfinite(y) && isfinite(th) && fabs(x) < 16777216.0 && fabs(y) < 16777216.0;
    if (!q.ok) {
        q.xi = q.yi = 0;
        q.xf = q.yf = q.c = q.s = 0.f;
        return q;
    }
    double fx = floor(x), fy = floor(y);
    q.xi = (int)fx;
    q.yi = (int)fy;
    q.xf = (float)(x - fx);
    q.yf = (float)(y - fy);
    double s, c;
    sincospi(th / 180.0, &s, &c);
    q.c = (float)c;
    q.s = (float)s;
    return q;
}

__device__ __forceinline__ float2 fetch(const BilField &F, int x, int y) {
    if ((unsigned)x < (unsigned)F.w && (unsigned)y < (unsigned)F.h)
        return __ldg(F.f + (size_t)y * F.pitch + x);
    return make_float2(0.f, 0.f);
}

// Accumulator layouts: K = 1 (score), 4 (score, J), 13 (score, J, J J^T, J r).
template <int K>
__device__ __forceinline__ void eval_points(const BilArgs &a, const BilField &F, const PoseF &q, float *acc) {
#pragma unroll
    for (int k = 0; k < K; ++k)
        acc[k] = 0.f;
    for (int i = threadIdx.x; i < a.n; i += kBilThreads) {
        const float4 P = __ldg(a.pts + i);
        const float rx = fmaf(q.c, P.x, -q.s * P.y);
        const float ry = fmaf(q.s, P.x, q.c * P.y);
        const float dx = fmaf(q.c, P.z, -q.s * P.w);
        const float dy = fmaf(q.s, P.z, q.c * P.w);
        const float qx = q.xf + rx, qy = q.yf + ry;
        const float cx = floorf(qx), cy = floorf(qy);
        const float fx = qx - cx, fy = qy - cy;
        const int X = q.xi + (int)cx, Y = q.yi + (int)cy;
        const float2 w00 = fetch(F, X, Y), w10 = fetch(F, X + 1, Y);
        const float2 w01 = fetch(F, X, Y + 1), w11 = fetch(F, X + 1, Y + 1);
        const float d0x = w10.x - w00.x, d0y = w10.y - w00.y;
        const float d1x = w11.x - w01.x, d1y = w11.y - w01.y;
        const float tpx = fmaf(fx, d0x, w00.x), tpy = fmaf(fx, d0y, w00.y);
        const float btx = fmaf(fx, d1x, w01.x), bty = fmaf(fx, d1y, w01.y);
        const float dyx = btx - tpx, dyy = bty - tpy;          // dw/dy
        const float wx = fmaf(fy, dyx, tpx), wy = fmaf(fy, dyy, tpy);
        float term = fmaf(dx, wx, dy * wy);
        if (K == 1) {
            acc[0] += a.polarity ? fabsf(term) : term;
            continue;
        }
        const float dxx = fmaf(fy, d1x - d0x, d0x), dxy = fmaf(fy, d1y - d0y, d0y);   // dw/dx
        float jx = fmaf(dx, dxx, dy * dxy);
        float jy = fmaf(dx, dyx, dy * dyy);
        float jt = (fmaf(dx, wy, -dy * wx) + fmaf(rx, jy, -ry * jx)) * kDegToRad;
        if (a.polarity) {
            const float sg = term > 0.f ? 1.f : (term < 0.f ? -1.f : 0.f);
            term = fabsf(term);
            jx *= sg;
            jy *= sg;
            jt *= sg;
        }
        acc[0] += term;
        acc[1] += jx;
        acc[2] += jy;
        acc[3] += jt;
        if (K == 13) {
            const float r = 1.f - term;
            acc[4] = fmaf(jx, jx, acc[4]);
            acc[5] = fmaf(jx, jy, acc[5]);
            acc[6] = fmaf(jx, jt, acc[6]);
            acc[7] = fmaf(jy, jy, acc[7]);
            acc[8] = fmaf(jy, jt, acc[8]);
            acc[9] = fmaf(jt, jt, acc[9]);
            acc[10] = fmaf(jx, r, acc[10]);
            acc[11] = fmaf(jy, r, acc[11]);
            acc[12] = fmaf(jt, r, acc[12]);
        }
    }
}

// Block sum of K accumulators into tot[K] (all threads must call; tot is
// valid after the function returns).
template <int K>
__device__ __forceinline__ void block_sum(float *acc, float (*red)[K], float *tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0)
            red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < kBilWarps; ++w)
            v += red[w][threadIdx.x];
        tot[threadIdx.x] = v;
    }
    __syncthreads();
}

__device__ __forceinline__ bool pose_field_ok(const BilArgs &a, const int32_t *pose_field, int b, int *fi) {
    const int f = pose_field ? pose_field[b] : 0;
    *fi = f;
    return f >= 0 && f < a.n_fields;
}

// Forward of the continuous-pose score (Eq. (1) without the neighbourhood
// maximum, Eq. (2) without rounding, bilinear samples); K = 1, 4 or 13
// accumulators.
template <int K>
__global__ void __launch_bounds__(kBilThreads) bilinear_kernel(const __grid_constant__ BilArgs a,
                                                               const int32_t *__restrict__ pose_field,
                                                               const float *__restrict__ poses, int B,
                                                               float *__restrict__ score, float *__restrict__ grad,
                                                               float *__restrict__ normal) {
    __shared__ float red[kBilWarps][K];
    __shared__ float tot[K];
    const int b = blockIdx.x;
    if (b >= B)
        return;
    int fi;
    const bool fok = pose_field_ok(a, pose_field, b, &fi);
    const PoseF q = split_pose(poses[3 * b], poses[3 * b + 1], poses[3 * b + 2]);
    if (!fok || !q.ok) {
        if (threadIdx.x == 0) {
            const float nan = __int_as_float(0x7fc00000);
            if (score)
                score[b] = nan;
            if (grad)
                for (int j = 0; j < 3; ++j)
                    grad[3 * b + j] = nan;
            if (normal)
                for (int j = 0; j < 9; ++j)
                    normal[9 * (size_t)b + j] = nan;
        }
        return;
    }
    float acc[K];
    eval_points<K>(a, a.fields[fi], q, acc);
    block_sum<K>(acc, red, tot);
    if (threadIdx.x == 0) {
        const float inv = 1.f / (float)a.n;
        if (score)
            score[b] = tot[0] * inv;
        if (K >= 4 && grad)
            for (int j = 0; j < 3; ++j)
                grad[3 * b + j] = tot[1 + j] * inv;
        if (K == 13 && normal)
            for (int j = 0; j < 9; ++j)
                normal[9 * (size_t)b + j] = tot[4 + j] * inv;
    }
}

// Adjoint: grad_pose = grad_score * dM_c/dpose.
__global__ void __launch_bounds__(kBilThreads) bilinear_adjoint_kernel(const __grid_constant__ BilArgs a,
                                                                       const int32_t *__restrict__ pose_field,
                                                                       const float *__restrict__ poses, int B,
                                                                       const float *__restrict__ grad_score,
                                                                       float *__restrict__ grad_pose) {
    __shared__ float red[kBilWarps][4];
    __shared__ float tot[4];
    const int b = blockIdx.x;
    if (b >= B)
        return;
    int fi;
    const bool fok = pose_field_ok(a, pose_field, b, &fi);
    const PoseF q = split_pose(poses[3 * b], poses[3 * b + 1], poses[3 * b + 2]);
    if (!fok || !q.ok) {
        if (threadIdx.x < 3)
            grad_pose[3 * b + threadIdx.x] = __int_as_float(0x7fc00000);
        return;
    }
    float acc[4];
    eval_points<4>(a, a.fields[fi], q, acc);
    block_sum<4>(acc, red, tot);
    if (threadIdx.x < 3)
        grad_pose[3 * b + threadIdx.x] = grad_score[b] * (tot[1 + threadIdx.x] / (float)a.n);
}

// Symmetric 3x3 solve by cofactors (A packed xx, xy, xt, yy, yt, tt).
__device__ bool solve3(const double *A, const double *r, double *d) {
    const double a00 = A[0], a01 = A[1], a02 = A[2], a11 = A[3], a12 = A[4], a22 = A[5];
    const double c00 = a11 * a22 - a12 * a12;
    const double c01 = a02 * a12 - a01 * a22;
    const double c02 = a01 * a12 - a02 * a11;
    const double det = a00 * c00 + a01 * c01 + a02 * c02;
    if (!(det > 0.0))
        return false;
    const double c11 = a00 * a22 - a02 * a02;
    const double c12 = a01 * a02 - a00 * a12;
    const double c22 = a00 * a11 - a01 * a01;
    d[0] = (c00 * r[0] + c01 * r[1] + c02 * r[2]) / det;
    d[1] = (c01 * r[0] + c11 * r[1] + c12 * r[2]) / det;
    d[2] = (c02 * r[0] + c12 * r[1] + c22 * r[2]) / det;
    return true;
}

// Gauss-Newton refinement of continuous poses (one CTA per pose, damped
// normal equations of the continuous-pose score, FP64 3x3 solve).
__global__ void __launch_bounds__(kBilThreads) refine_gn_kernel(const __grid_constant__ BilArgs a,
                                                                const int32_t *__restrict__ pose_field,
                                                                float *__restrict__ poses, int B, int iterations,
                                                                float *__restrict__ score) {
    __shared__ float red[kBilWarps][13];
    __shared__ float tot[13];
    __shared__ double trial[3];
    __shared__ int skip;
    const int b = blockIdx.x;
    if (b >= B)
        return;
    int fi;
    const bool fok = pose_field_ok(a, pose_field, b, &fi);
    double p[3] = {poses[3 * b], poses[3 * b + 1], poses[3 * b + 2]};
    PoseF q = split_pose(p[0], p[1], p[2]);
    if (!fok || !q.ok) {
        if (threadIdx.x == 0 && score)
            score[b] = __int_as_float(0x7fc00000);
        return;
    }
    const BilField F = a.fields[fi];
    const float inv = 1.f / (float)a.n;
    float acc[13];
    eval_points<13>(a, F, q, acc);
    block_sum<13>(acc, red, tot);
    // state, meaningful in thread 0
    double S = 0.0, A[6], r[3], lambda = 1e-3;
    if (threadIdx.x == 0) {
        S = (double)(tot[0] * inv);
        for (int j = 0; j < 6; ++j)
            A[j] = (double)(tot[4 + j] * inv);
        for (int j = 0; j < 3; ++j)
            r[j] = (double)(tot[10 + j] * inv);
    }
    for (int it = 0; it < iterations; ++it) {
        if (threadIdx.x == 0) {
            double M[6] = {A[0], A[1], A[2], A[3], A[4], A[5]};
            M[0] += lambda * A[0] + 1e-9;
            M[3] += lambda * A[3] + 1e-9;
            M[5] += lambda * A[5] + 1e-9;
            double d[3];
            if (!solve3(M, r, d)) {
                lambda = fmin(4.0 * lambda, 1e7);
                skip = 1;
            } else {
                const double big = fmax(fabs(d[0]), fmax(fabs(d[1]), fabs(d[2])));
                if (big > 1.0) {
                    d[0] /= big;
                    d[1] /= big;
                    d[2] /= big;
                }
                trial[0] = p[0] + d[0];
                trial[1] = p[1] + d[1];
                trial[2] = p[2] + d[2];
                skip = 0;
            }
        }
        __syncthreads();
        if (!skip) {
            q = split_pose(trial[0], trial[1], trial[2]);
            eval_points<13>(a, F, q, acc);
            block_sum<13>(acc, red, tot);
            if (threadIdx.x == 0) {
                const double S2 = (double)(tot[0] * inv);
                if (q.ok && S2 > S) {
                    p[0] = trial[0];
                    p[1] = trial[1];
                    p[2] = trial[2];
                    S = S2;
                    for (int j = 0; j < 6; ++j)
                        A[j] = (double)(tot[4 + j] * inv);
                    for (int j = 0; j < 3; ++j)
                        r[j] = (double)(tot[10 + j] * inv);
                    lambda = fmax(lambda / 3.0, 1e-7);
                } else {
                    lambda = fmin(4.0 * lambda, 1e7);
                }
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        poses[3 * b] = (float)p[0];
        poses[3 * b + 1] = (float)p[1];
        poses[3 * b + 2] = (float)p[2];
        if (score)
            score[b] = (float)S;
    }
}

sam_status make_args(sam_model *m, int level, const sam_field_ref *fields, int n_fields, BilArgs *a) {
    // the continuous pose (x, y, theta) is rigid: scaled models are not served
    if (!m || level < 0 || level >= m->levels || !fields || n_fields < 1 || n_fields > SAM_MAX_BILINEAR_FIELDS ||
        m->nscales != 1 || m->scale_min != 1.0)
        return SAM_ERR_ARG;
    for (int i = 0; i < n_fields; ++i) {
        const sam_field_ref &f = fields[i];
        if (!f.field || f.w < 1 || f.h < 1 || f.pitch < f.w || (uintptr_t)f.field % 8)
            return SAM_ERR_ARG;
    }
    sam_status s = upload_model(m);
    if (s != SAM_OK)
        return s;
    a->pts = m->dev[level].base;
    a->n = m->dev[level].n;
    a->polarity = m->p.polarity ? 1 : 0;
    a->n_fields = n_fields;
    for (int i = 0; i < SAM_MAX_BILINEAR_FIELDS; ++i) {
        if (i < n_fields)
            a->fields[i] = BilField{(const float2 *)fields[i].field, fields[i].w, fields[i].h, fields[i].pitch};
        else
            a->fields[i] = BilField{nullptr, 0, 0, 0};
    }
    return SAM_OK;
}

}  // namespace
}  // namespace sam

using namespace sam;

extern "C" sam_status sam_score_bilinear(sam_model *m, int level, const sam_field_ref *fields, int n_fields,
                                         const int32_t *pose_field, const float *poses, int n_poses, float *score,
                                         float *grad, float *normal, void *stream) {
    if (n_poses < 0 || (n_poses > 0 && (!poses || !score)))
        return SAM_ERR_ARG;
    BilArgs a;
    sam_status s = make_args(m, level, fields, n_fields, &a);
    if (s != SAM_OK || n_poses == 0)
        return s;
    cudaStream_t st = (cudaStream_t)stream;
    if (normal)
        bilinear_kernel<13><<<n_poses, kBilThreads, 0, st>>>(a, pose_field, poses, n_poses, score, grad, normal);
    else if (grad)
        bilinear_kernel<4><<<n_poses, kBilThreads, 0, st>>>(a, pose_field, poses, n_poses, score, grad, nullptr);
    else
        bilinear_kernel<1><<<n_poses, kBilThreads, 0, st>>>(a, pose_field, poses, n_poses, score, nullptr, nullptr);
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? SAM_OK : SAM_ERR_CUDA;
}

extern "C" sam_status sam_score_bilinear_adjoint(sam_model *m, int level, const sam_field_ref *fields, int n_fields,
                                                 const int32_t *pose_field, const float *poses, int n_poses,
                                                 const float *grad_score, float *grad_pose, void *stream) {
    if (n_poses < 0 || (n_poses > 0 && (!poses || !grad_score || !grad_pose)))
        return SAM_ERR_ARG;
    BilArgs a;
    sam_status s = make_args(m, level, fields, n_fields, &a);
    if (s != SAM_OK || n_poses == 0)
        return s;
    bilinear_adjoint_kernel<<<n_poses, kBilThreads, 0, (cudaStream_t)stream>>>(a, pose_field, poses, n_poses,
                                                                                grad_score, grad_pose);
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? SAM_OK : SAM_ERR_CUDA;
}

extern "C" sam_status sam_refine_poses(sam_model *m, int level, const sam_field_ref *fields, int n_fields,
                                       const int32_t *pose_field, float *poses, int n_poses, int iterations,
                                       float *score, void *stream) {
    if (n_poses < 0 || (n_poses > 0 && !poses) || iterations < 0 || iterations > 10000)
        return SAM_ERR_ARG;
    BilArgs a;
    sam_status s = make_args(m, level, fields, n_fields, &a);
    if (s != SAM_OK || n_poses == 0)
        return s;
    refine_gn_kernel<<<n_poses, kBilThreads, 0, (cudaStream_t)stream>>>(a, pose_field, poses, n_poses, iterations,
                                                                         score);
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? SAM_OK : SAM_ERR_CUDA;
}
