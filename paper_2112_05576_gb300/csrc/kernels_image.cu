// Kernels (a) and (b): edge extraction and the image pyramid (Sec. II).
//
// (b) pyramid step: each thread produces 16 output bytes from two 32-byte
//     input row segments, 128-bit loads and stores on the aligned fast path;
//     the 2x2 rounded mean is computed two bytes at a time in 16-bit lanes.
// (a) gradient: one CTA stages an (TY+2) x (TX+2) byte tile of the image in
//     shared memory (128-bit global loads on the aligned path), every thread
//     computes 8 consecutive pixels of one row: integer Sobel gx, gy, the
//     exact edge test gx^2+gy^2 >= 16 low^2 and the unit vector g/|g| (FP32,
//     rsqrt), written as FP32 pairs (8 B/px) or bf16/fp16 pairs (4 B/px).
// Both are HBM-bound: (b) moves 5 B per output pixel, (a) 1 B in + 8 (or 4)
// B out per pixel.

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "image_common.cuh"
#include "sam_internal.h"

namespace sam {
namespace {

// ---------------------------------------------------------------------------
// (b) pyramid step
// ---------------------------------------------------------------------------

// Four input bytes of row 0 (p) and row 1 (q) -> two output bytes in byte
// lanes 0 and 2 of the result: (p0+p1+q0+q1+2)>>2, (p2+p3+q2+q3+2)>>2.
__device__ __forceinline__ uint32_t mean2x2_pair(uint32_t p, uint32_t q) {
    const uint32_t m = 0x00FF00FFu;
    const uint32_t s = (p & m) + ((p >> 8) & m) + (q & m) + ((q >> 8) & m) + 0x00020002u;
    return (s >> 2) & m;
}

// 8 input bytes per row -> 4 output bytes.
__device__ __forceinline__ uint32_t mean2x2_quad(uint32_t p0, uint32_t p1, uint32_t q0, uint32_t q1) {
    const uint32_t lo = mean2x2_pair(p0, q0);   // outputs 0, 1 in bytes 0, 2
    const uint32_t hi = mean2x2_pair(p1, q1);   // outputs 2, 3 in bytes 0, 2
    return __byte_perm(lo, hi, 0x6420);
}

// 16 output pixels of output row y starting at column x0.
__device__ __forceinline__ void pyramid_16(const uint8_t *__restrict__ src, int w, int h, int ss,
                                           uint8_t *__restrict__ dst, int ds, int vec, int y, int x0) {
    const int w2 = w >> 1, h2 = h >> 1;
    if (y >= h2 || x0 >= w2)
        return;
    const uint8_t *r0 = src + (size_t)(2 * y) * ss;
    const uint8_t *r1 = r0 + ss;
    uint8_t *o = dst + (size_t)y * ds;
    if (vec && x0 + 16 <= w2) {
        const uint4 a0 = __ldg(reinterpret_cast<const uint4 *>(r0 + 2 * x0));
        const uint4 a1 = __ldg(reinterpret_cast<const uint4 *>(r0 + 2 * x0 + 16));
        const uint4 b0 = __ldg(reinterpret_cast<const uint4 *>(r1 + 2 * x0));
        const uint4 b1 = __ldg(reinterpret_cast<const uint4 *>(r1 + 2 * x0 + 16));
        uint4 r;
        r.x = mean2x2_quad(a0.x, a0.y, b0.x, b0.y);
        r.y = mean2x2_quad(a0.z, a0.w, b0.z, b0.w);
        r.z = mean2x2_quad(a1.x, a1.y, b1.x, b1.y);
        r.w = mean2x2_quad(a1.z, a1.w, b1.z, b1.w);
        *reinterpret_cast<uint4 *>(o + x0) = r;
    } else {
        const int xe = min(x0 + 16, w2);
        for (int x = x0; x < xe; ++x)
            o[x] = (uint8_t)((r0[2 * x] + r0[2 * x + 1] + r1[2 * x] + r1[2 * x + 1] + 2) >> 2);
    }
}

// Pyramid step (Sec. II image pyramid) of `count` images of equal size,
// image blockIdx.z, output row blockIdx.y, 16 output pixels per thread.
__global__ void pyramid_down_kernel(const uint8_t *__restrict__ src, int w, int h, int ss, size_t src_img,
                                    uint8_t *__restrict__ dst, int ds, size_t dst_img, int vec) {
    const int img = blockIdx.z;
    pyramid_16(src + (size_t)img * src_img, w, h, ss, dst + (size_t)img * dst_img, ds, vec, blockIdx.y,
               (blockIdx.x * blockDim.x + threadIdx.x) * 16);
}

// Every pyramid level below level 0 in one pass (levels 1 .. D, D <= 6):
// one CTA per 128 x 64 block of level 0 (image blockIdx.z) computes its
// 64 x 32 block of level 1 from 16-byte loads of level 0, then each further
// level from the previous one held in shared memory.  A level-l pixel
// depends only on the 2^l x 2^l level-0 pixels under it, so the blocks are
// independent, and each level is the 2x2 rounded mean of the one above it
// exactly as the one-step kernel computes it (floor of odd sizes
// included).  Level l's image starts at dst[l] + image * dst_img[l], row
// pitch dst_pitch[l] (a multiple of 16).
constexpr int kPyrBW = 128, kPyrBH = 64;   // level-0 block
struct PyramidLevels {
    uint8_t *dst[kMaxLevels];
    int pitch[kMaxLevels];
    size_t img[kMaxLevels];
};

__global__ void __launch_bounds__(256) pyramid_levels_kernel(const uint8_t *__restrict__ src, int w, int h, int ss,
                                                             size_t src_img, PyramidLevels out, int D, int vec) {
    __shared__ __align__(16) uint8_t buf[2][(kPyrBW / 2) * (kPyrBH / 2)];
    const int img = blockIdx.z, tid = threadIdx.x;
    src += (size_t)img * src_img;
    // level 1: 64 x 32 outputs, 8 per thread (row tid / 8, columns 8 (tid % 8) ..)
    {
        const int w1 = w >> 1, h1 = h >> 1;
        const int r = tid >> 3, c = (tid & 7) * 8;
        const int y = blockIdx.y * (kPyrBH / 2) + r, x0 = blockIdx.x * (kPyrBW / 2) + c;
        uint32_t lo = 0u, hi = 0u;
        if (y < h1 && x0 < w1) {
            const uint8_t *r0 = src + (size_t)(2 * y) * ss + 2 * x0;
            const uint8_t *r1 = r0 + ss;
            uint8_t *o = out.dst[1] + (size_t)img * out.img[1] + (size_t)y * out.pitch[1] + x0;
            if (vec && x0 + 8 <= w1) {
                const uint4 a = __ldg(reinterpret_cast<const uint4 *>(r0));
                const uint4 b = __ldg(reinterpret_cast<const uint4 *>(r1));
                lo = mean2x2_quad(a.x, a.y, b.x, b.y);
                hi = mean2x2_quad(a.z, a.w, b.z, b.w);
                *reinterpret_cast<uint2 *>(o) = make_uint2(lo, hi);
            } else {
                for (int j = 0; j < 8 && x0 + j < w1; ++j) {
                    const uint32_t v = (r0[2 * j] + r0[2 * j + 1] + r1[2 * j] + r1[2 * j + 1] + 2) >> 2;
                    o[j] = (uint8_t)v;
                    if (j < 4)
                        lo |= v << (8 * j);
                    else
                        hi |= v << (8 * (j - 4));
                }
            }
        }
        *reinterpret_cast<uint2 *>(&buf[0][r * (kPyrBW / 2) + c]) = make_uint2(lo, hi);
    }
    __syncthreads();
    // levels 2 .. D from the previous level's block in shared memory
    int lw = w >> 1, lh = h >> 1;
    for (int l = 2; l <= D; ++l) {
        const int pbw = kPyrBW >> (l - 1);          // previous block width
        const int bw = pbw >> 1, bh = kPyrBH >> l;  // this block
        lw >>= 1;
        lh >>= 1;
        const uint8_t *prev = buf[l & 1];
        uint8_t *cur = buf[(l + 1) & 1];
        for (int i = tid; i < bw * bh; i += 256) {
            const int r = i / bw, c = i - r * bw;
            const int y = blockIdx.y * bh + r, x = blockIdx.x * bw + c;
            const uint8_t *p0 = prev + (2 * r) * pbw + 2 * c;
            const uint8_t v = (uint8_t)((p0[0] + p0[1] + p0[pbw] + p0[pbw + 1] + 2) >> 2);
            cur[i] = v;
            if (y < lh && x < lw)
                out.dst[l][(size_t)img * out.img[l] + (size_t)y * out.pitch[l] + x] = v;
        }
        __syncthreads();
    }
}

// One pyramid step of many images of different sizes: job blockIdx.z,
// rows strided over gridDim.y.
__global__ void pyramid_jobs_kernel(const ImageJob *__restrict__ jobs) {
    const ImageJob j = jobs[blockIdx.z];
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * 16;
    for (int y = blockIdx.y; y < (j.h >> 1); y += gridDim.y)
        pyramid_16(j.src, j.w, j.h, j.src_stride, static_cast<uint8_t *>(j.dst), j.dst_stride, j.vec, y, x0);
}

// ---------------------------------------------------------------------------
// (a) gradient / threshold / normalise
// ---------------------------------------------------------------------------

constexpr int GTX = 128;   // tile width (pixels)
constexpr int GTY = 16;    // tile height
constexpr int GPT = 8;     // pixels per thread (one row segment)
constexpr int GTHREADS = GTX / GPT * GTY;   // 256
constexpr int GSW = GTX + 32;               // smem row pitch: 16-byte halo on each side

template <int PREC>
struct FieldStore;

template <>
struct FieldStore<SAM_FP32> {
    // 8 pixels -> 64 bytes
    static __device__ __forceinline__ void store8(void *field, size_t idx, const float *wx, const float *wy) {
        float4 *p = reinterpret_cast<float4 *>(reinterpret_cast<float2 *>(field) + idx);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            p[j] = make_float4(wx[2 * j], wy[2 * j], wx[2 * j + 1], wy[2 * j + 1]);
    }
    static __device__ __forceinline__ void store1(void *field, size_t idx, float wx, float wy) {
        reinterpret_cast<float2 *>(field)[idx] = make_float2(wx, wy);
    }
    // pixel pair q of a pairs-layout field: {wx0, wx1, wy0, wy1}
    static __device__ __forceinline__ void store_pair(void *field, size_t q, float x0, float x1, float y0, float y1) {
        reinterpret_cast<float4 *>(field)[q] = make_float4(x0, x1, y0, y1);
    }
};

template <>
struct FieldStore<SAM_BF16> {
    static __device__ __forceinline__ uint32_t pack(float a, float b) {
        __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&v);
    }
    static __device__ __forceinline__ void store8(void *field, size_t idx, const float *wx, const float *wy) {
        uint4 *p = reinterpret_cast<uint4 *>(reinterpret_cast<uint32_t *>(field) + idx);
        p[0] = make_uint4(pack(wx[0], wy[0]), pack(wx[1], wy[1]), pack(wx[2], wy[2]), pack(wx[3], wy[3]));
        p[1] = make_uint4(pack(wx[4], wy[4]), pack(wx[5], wy[5]), pack(wx[6], wy[6]), pack(wx[7], wy[7]));
    }
    static __device__ __forceinline__ void store1(void *field, size_t idx, float wx, float wy) {
        reinterpret_cast<uint32_t *>(field)[idx] = pack(wx, wy);
    }
    static __device__ __forceinline__ void store_pair(void *field, size_t q, float x0, float x1, float y0, float y1) {
        reinterpret_cast<uint2 *>(field)[q] = make_uint2(pack(x0, x1), pack(y0, y1));
    }
};

template <>
struct FieldStore<SAM_FP16> {
    static __device__ __forceinline__ uint32_t pack(float a, float b) {
        __half2 v = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&v);
    }
    static __device__ __forceinline__ void store8(void *field, size_t idx, const float *wx, const float *wy) {
        uint4 *p = reinterpret_cast<uint4 *>(reinterpret_cast<uint32_t *>(field) + idx);
        p[0] = make_uint4(pack(wx[0], wy[0]), pack(wx[1], wy[1]), pack(wx[2], wy[2]), pack(wx[3], wy[3]));
        p[1] = make_uint4(pack(wx[4], wy[4]), pack(wx[5], wy[5]), pack(wx[6], wy[6]), pack(wx[7], wy[7]));
    }
    static __device__ __forceinline__ void store1(void *field, size_t idx, float wx, float wy) {
        reinterpret_cast<uint32_t *>(field)[idx] = pack(wx, wy);
    }
    static __device__ __forceinline__ void store_pair(void *field, size_t q, float x0, float x1, float y0, float y1) {
        reinterpret_cast<uint2 *>(field)[q] = make_uint2(pack(x0, x1), pack(y0, y1));
    }
};

// Angle-only storage: the 16-bit code of an integer gradient, 0x8000 | a with
// a = round(atan2(gy, gx) 32768 / (2 pi)) mod 32768 on an edge, else 0.  The
// FP32 atan2 (a few ulp, below 0.01 of a step with the scaling) decides the
// code unless its scaled value lies within 0.02 of a rounding boundary; there
// the FP64 atan2 decides.  No Sobel gradient has its exact angle within
// 1.2e-6 steps of a boundary, so both give the rounding of the exact angle.
__device__ __forceinline__ uint32_t angle_code(int gx, int gy, int thr) {
    const int m2 = gx * gx + gy * gy;
    if (m2 < thr || m2 == 0)
        return 0u;
    const float sf = atan2f((float)gy, (float)gx) * (32768.0f / 6.28318530717958648f) + 0.5f;
    const float fl = floorf(sf);
    const float d = sf - fl;
    int a;
    if (d > 0.02f && d < 0.98f) {
        a = (int)fl;
    } else {
        const double t = atan2((double)gy, (double)gx) * 32768.0 / (2.0 * 3.14159265358979323846);
        a = (int)floor(t + 0.5);
    }
    return 0x8000u | ((uint32_t)a & 0x7FFFu);
}

// One GTX x GTY tile of one image whose field starts fbase pixels into
// `field` (the caller returns early, block-uniformly, for tiles outside).
template <int PREC, int LAYOUT>
__device__ __forceinline__ void gradient_tile(const uint8_t *__restrict__ img, int w, int h, int ss, int low,
                                              void *__restrict__ field, size_t fbase, int16_t *__restrict__ ogx,
                                              int16_t *__restrict__ ogy, int vec, int x0, int y0) {
    __shared__ __align__(16) uint8_t tile[GTY + 2][GSW];
    const int tid = threadIdx.x;

    // Stage rows y0-1 .. y0+GTY, columns x0-16 .. x0+GTX+15 (zero outside).
    // tile[r][c] holds image pixel (x0 - 16 + c, y0 - 1 + r).
    if (vec) {
        constexpr int CH = GSW / 16;   // 16-byte chunks per row
        for (int e = tid; e < (GTY + 2) * CH; e += GTHREADS) {
            const int r = e / CH, c = e - r * CH;
            const int y = y0 - 1 + r, x = x0 - 16 + 16 * c;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (y >= 0 && y < h) {
                const uint8_t *row = img + (size_t)y * ss;
                if (x >= 0 && x + 16 <= w) {
                    v = __ldg(reinterpret_cast<const uint4 *>(row + x));
                } else {
                    uint32_t wd[4] = {0, 0, 0, 0};
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (x + j >= 0 && x + j < w)
                            wd[j >> 2] |= (uint32_t)row[x + j] << (8 * (j & 3));
                    v = make_uint4(wd[0], wd[1], wd[2], wd[3]);
                }
            }
            *reinterpret_cast<uint4 *>(&tile[r][16 * c]) = v;
        }
    } else {
        for (int e = tid; e < (GTY + 2) * GSW; e += GTHREADS) {
            const int r = e / GSW, c = e - r * GSW;
            const int y = y0 - 1 + r, x = x0 - 16 + c;
            tile[r][c] = (y >= 0 && y < h && x >= 0 && x < w) ? img[(size_t)y * ss + x] : 0;
        }
    }
    __syncthreads();

    const int ty = tid / (GTX / GPT);
    const int tx = (tid - ty * (GTX / GPT)) * GPT;
    const int y = y0 + ty;
    const int xb = x0 + tx;
    if constexpr (PREC == SAM_ANGLE16) {
        // 8 codes (16 bytes) per thread; with the padded pitch (a multiple of
        // 8) a thread's group never straddles the row end, and its codes
        // beyond w are 0 (zero gradient)
        const int cp = code_pitch(w, LAYOUT);
        if (y >= h || xb >= cp)
            return;
        const int r = ty + 1, cb = tx + 16;
        int a[GPT + 2], b[GPT + 2], c[GPT + 2];
#pragma unroll
        for (int j = 0; j < GPT + 2; ++j) {
            a[j] = tile[r - 1][cb - 1 + j];
            b[j] = tile[r][cb - 1 + j];
            c[j] = tile[r + 1][cb - 1 + j];
        }
        const int thr = 16 * low * low;
        uint32_t code[GPT];
#pragma unroll
        for (int j = 0; j < GPT; ++j) {
            const int x = xb + j;
            int gx = 0, gy = 0;
            if (x > 0 && x < w - 1 && y > 0 && y < h - 1) {
                gx = (a[j + 2] + 2 * b[j + 2] + c[j + 2]) - (a[j] + 2 * b[j] + c[j]);
                gy = (c[j] + 2 * c[j + 1] + c[j + 2]) - (a[j] + 2 * a[j + 1] + a[j + 2]);
            }
            code[j] = angle_code(gx, gy, thr);
        }
        uint16_t *out = reinterpret_cast<uint16_t *>(field) + fbase + (size_t)y * cp + xb;
        if (vec && xb + GPT <= cp) {
            *reinterpret_cast<uint4 *>(out) = make_uint4(code[0] | (code[1] << 16), code[2] | (code[3] << 16),
                                                         code[4] | (code[5] << 16), code[6] | (code[7] << 16));
        } else {
#pragma unroll
            for (int j = 0; j < GPT; ++j)
                if (xb + j < cp)
                    out[j] = (uint16_t)code[j];
        }
    } else {
    // FP32 pixel-layout fields of whole rows (the large fields of the lower
    // levels) are written through a per-warp staging buffer so that every
    // store instruction covers 512 contiguous bytes: a warp owns two rows of
    // the tile, 1 KB of output each, whose 16-byte slots are written to
    // shared memory in thread order and read back in address order (slot s
    // kept at column (s mod 8) xor (s div 8 mod 8) of its 8-slot row, which
    // keeps both accesses free of bank conflicts)
    if constexpr (PREC == SAM_FP32 && LAYOUT == SAM_LAYOUT_PIXEL) {
        const bool rows_full = vec && !ogx && (w & 7) == 0 && __all_sync(0xffffffffu, y < h && x0 + GTX <= w);
        if (rows_full) {
            __shared__ __align__(16) float4 stage[GTHREADS / 32][128];
            const int lane = tid & 31;
            float4 *S = stage[tid >> 5];
            const int r = ty + 1, cb = tx + 16;
            int a[GPT + 2], b[GPT + 2], c[GPT + 2];
#pragma unroll
            for (int j = 0; j < GPT + 2; ++j) {
                a[j] = tile[r - 1][cb - 1 + j];
                b[j] = tile[r][cb - 1 + j];
                c[j] = tile[r + 1][cb - 1 + j];
            }
            const int thr = 16 * low * low;
#pragma unroll
            for (int q = 0; q < GPT / 2; ++q) {
                float2 u[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int j = 2 * q + e, x = xb + j;
                    int gx = 0, gy = 0;
                    if (x > 0 && x < w - 1 && y > 0 && y < h - 1) {
                        gx = (a[j + 2] + 2 * b[j + 2] + c[j + 2]) - (a[j] + 2 * b[j] + c[j]);
                        gy = (c[j] + 2 * c[j + 1] + c[j + 2]) - (a[j] + 2 * a[j + 1] + a[j + 2]);
                    }
                    u[e] = unit_of_gradient(gx, gy, thr);
                }
                const int sl = 4 * lane + q;
                S[(sl & ~7) | ((sl & 7) ^ ((sl >> 3) & 7))] = make_float4(u[0].x, u[0].y, u[1].x, u[1].y);
            }
            __syncwarp();
            // slots 0..63: the warp's first row, 64..127: its second row
            const int yw = y0 + (ty & ~1);
            float4 *out = reinterpret_cast<float4 *>(reinterpret_cast<float2 *>(field) + fbase + (size_t)yw * w + x0);
            const size_t rowf4 = (size_t)w / 2;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int sl = 32 * i + lane;
                out[(size_t)(sl >> 6) * rowf4 + (sl & 63)] = S[(sl & ~7) | ((sl & 7) ^ ((sl >> 3) & 7))];
            }
            return;
        }
    }
    // Pairs-layout fields (the scored level): the same per-warp staging.  A
    // warp's 32 threads hold 4 pixel pairs each, two tile rows of 64 pairs
    // whose slots 4 lane + q are already in address order; FP32 pairs are one
    // 16-byte slot each, 16-bit pairs two to a slot.  Read back in address
    // order, every store instruction covers 512 (FP32) or 256 (16-bit)
    // contiguous bytes instead of one 16- or 8-byte piece per thread.
    if constexpr (LAYOUT == SAM_LAYOUT_PAIRS) {
        const bool rows_full = vec && __all_sync(0xffffffffu, y < h && x0 + GTX <= w);
        if (rows_full) {
            __shared__ __align__(16) uint4 pstage[GTHREADS / 32][128];
            const int lane = tid & 31;
            uint4 *S = pstage[tid >> 5];
            const int r = ty + 1, cb = tx + 16;
            int a[GPT + 2], b[GPT + 2], c[GPT + 2];
#pragma unroll
            for (int j = 0; j < GPT + 2; ++j) {
                a[j] = tile[r - 1][cb - 1 + j];
                b[j] = tile[r][cb - 1 + j];
                c[j] = tile[r + 1][cb - 1 + j];
            }
            const int thr = 16 * low * low;
            float wx[GPT], wy[GPT];
#pragma unroll
            for (int j = 0; j < GPT; ++j) {
                const int x = xb + j;
                int gx = 0, gy = 0;
                if (x > 0 && x < w - 1 && y > 0 && y < h - 1) {
                    gx = (a[j + 2] + 2 * b[j + 2] + c[j + 2]) - (a[j] + 2 * b[j] + c[j]);
                    gy = (c[j] + 2 * c[j + 1] + c[j + 2]) - (a[j] + 2 * a[j + 1] + a[j + 2]);
                }
                const float2 u = unit_of_gradient(gx, gy, thr);
                wx[j] = u.x;
                wy[j] = u.y;
            }
            const int wp = field_pitch(w, SAM_LAYOUT_PAIRS);
            const int yw = y0 + (ty & ~1);
            const size_t q0 = (fbase + (size_t)yw * wp + x0) >> 1;   // first pair of the warp's first row
            if constexpr (PREC == SAM_FP32) {
#pragma unroll
                for (int q = 0; q < GPT / 2; ++q) {
                    const int sl = 4 * lane + q;
                    const float4 v = make_float4(wx[2 * q], wx[2 * q + 1], wy[2 * q], wy[2 * q + 1]);
                    S[(sl & ~7) | ((sl & 7) ^ ((sl >> 3) & 7))] = *reinterpret_cast<const uint4 *>(&v);
                }
                __syncwarp();
                uint4 *out = reinterpret_cast<uint4 *>(field) + q0;
                const size_t rowq = (size_t)wp / 2;   // 16-byte pairs per field row
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int sl = 32 * i + lane;
                    out[(size_t)(sl >> 6) * rowq + (sl & 63)] = S[(sl & ~7) | ((sl & 7) ^ ((sl >> 3) & 7))];
                }
            } else {
                uint2 pr[GPT / 2];
#pragma unroll
                for (int q = 0; q < GPT / 2; ++q)
                    pr[q] = make_uint2(FieldStore<PREC>::pack(wx[2 * q], wx[2 * q + 1]),
                                       FieldStore<PREC>::pack(wy[2 * q], wy[2 * q + 1]));
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int sl = 2 * lane + hh;
                    S[(sl & ~7) | ((sl & 7) ^ ((sl >> 3) & 7))] =
                        make_uint4(pr[2 * hh].x, pr[2 * hh].y, pr[2 * hh + 1].x, pr[2 * hh + 1].y);
                }
                __syncwarp();
                uint4 *out = reinterpret_cast<uint4 *>(reinterpret_cast<uint2 *>(field) + q0);
                const size_t rowu = (size_t)wp / 4;   // 16-byte slots (two 8-byte pairs) per field row
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int sl = 32 * i + lane;
                    out[(size_t)(sl >> 5) * rowu + (sl & 31)] = S[(sl & ~7) | ((sl & 7) ^ ((sl >> 3) & 7))];
                }
            }
            return;
        }
    }
    if (y >= h || xb >= w)
        return;
    const int r = ty + 1;      // centre row in tile
    const int cb = tx + 16;    // column of pixel xb in tile
    int a[GPT + 2], b[GPT + 2], c[GPT + 2];
#pragma unroll
    for (int j = 0; j < GPT + 2; ++j) {
        a[j] = tile[r - 1][cb - 1 + j];
        b[j] = tile[r][cb - 1 + j];
        c[j] = tile[r + 1][cb - 1 + j];
    }
    const int thr = 16 * low * low;
    float wx[GPT], wy[GPT];
    int gxs[GPT], gys[GPT];
#pragma unroll
    for (int j = 0; j < GPT; ++j) {
        const int x = xb + j;
        int gx = 0, gy = 0;
        if (x > 0 && x < w - 1 && y > 0 && y < h - 1) {
            gx = (a[j + 2] + 2 * b[j + 2] + c[j + 2]) - (a[j] + 2 * b[j] + c[j]);
            gy = (c[j] + 2 * c[j + 1] + c[j + 2]) - (a[j] + 2 * a[j + 1] + a[j + 2]);
        }
        const float2 u = unit_of_gradient(gx, gy, thr);
        wx[j] = u.x;
        wy[j] = u.y;
        gxs[j] = gx;
        gys[j] = gy;
    }
    if (LAYOUT == SAM_LAYOUT_PAIRS) {
        // pixels beyond w were computed as zero, so the padding pixels up to
        // the row pitch (a multiple of 4, at most the thread's 8-pixel group
        // end) are written as zero too
        const int wp = field_pitch(w, SAM_LAYOUT_PAIRS);
        const size_t q0 = (fbase + (size_t)y * wp + xb) >> 1;
        const bool full = (xb + GPT <= wp) && vec;
#pragma unroll
        for (int q = 0; q < GPT / 2; ++q)
            if (full || xb + 2 * q < wp)
                FieldStore<PREC>::store_pair(field, q0 + q, wx[2 * q], wx[2 * q + 1], wy[2 * q], wy[2 * q + 1]);
        return;
    }
    const size_t base = fbase + (size_t)y * w + xb;
    const bool full = (xb + GPT <= w) && vec && ((w & 7) == 0);
    if (full) {
        FieldStore<PREC>::store8(field, base, wx, wy);
        if (ogx) {
            uint4 vx, vy;
            vx.x = (gxs[0] & 0xFFFF) | (gxs[1] << 16);
            vx.y = (gxs[2] & 0xFFFF) | (gxs[3] << 16);
            vx.z = (gxs[4] & 0xFFFF) | (gxs[5] << 16);
            vx.w = (gxs[6] & 0xFFFF) | (gxs[7] << 16);
            vy.x = (gys[0] & 0xFFFF) | (gys[1] << 16);
            vy.y = (gys[2] & 0xFFFF) | (gys[3] << 16);
            vy.z = (gys[4] & 0xFFFF) | (gys[5] << 16);
            vy.w = (gys[6] & 0xFFFF) | (gys[7] << 16);
            *reinterpret_cast<uint4 *>(ogx + base) = vx;
            *reinterpret_cast<uint4 *>(ogy + base) = vy;
        }
    } else {
#pragma unroll
        for (int j = 0; j < GPT; ++j) {
            if (xb + j >= w)
                break;
            FieldStore<PREC>::store1(field, base + j, wx[j], wy[j]);
            if (ogx) {
                ogx[base + j] = (int16_t)gxs[j];
                ogy[base + j] = (int16_t)gys[j];
            }
        }
    }
    }   // PREC != SAM_ANGLE16
}

// `count` images of equal size, image blockIdx.z.
template <int PREC, int LAYOUT>
__global__ void __launch_bounds__(GTHREADS) gradient_kernel(const uint8_t *__restrict__ img, int w, int h, int ss,
                                                            size_t img_bytes, int low, void *__restrict__ field,
                                                            size_t field_img_px, int16_t *__restrict__ ogx,
                                                            int16_t *__restrict__ ogy, int vec) {
    const int im = blockIdx.z;
    gradient_tile<PREC, LAYOUT>(img + (size_t)im * img_bytes, w, h, ss, low, field, (size_t)im * field_img_px, ogx,
                                ogy, vec, blockIdx.x * GTX, blockIdx.y * GTY);
}

// Images of different sizes: job blockIdx.z, tiles strided over the grid.
template <int PREC, int LAYOUT>
__global__ void __launch_bounds__(GTHREADS) gradient_jobs_kernel(const ImageJob *__restrict__ jobs, int low) {
    const ImageJob j = jobs[blockIdx.z];
    for (int y0 = blockIdx.y * GTY; y0 < j.h; y0 += gridDim.y * GTY)
        for (int x0 = blockIdx.x * GTX; x0 < j.w; x0 += gridDim.x * GTX) {
            gradient_tile<PREC, LAYOUT>(j.src, j.w, j.h, j.src_stride, low, j.dst, 0, nullptr, nullptr, j.vec, x0,
                                        y0);
            __syncthreads();   // the tile buffer is reused by the next iteration
        }
}

// Marked tiles of the refinement levels (FP32 pixel layout), each computed
// exactly as gradient_kernel computes it: the persistent CTAs walk the list
// that mark_tiles_kernel built.
__global__ void __launch_bounds__(GTHREADS) gradient_tiles_kernel(const GradTiles g) {
    const unsigned n = min(*g.list_cnt, g.list_cap);
    for (unsigned i = blockIdx.x; i < n; i += gridDim.x) {
        const uint2 t = g.list[i];
        const int l = (int)(t.x >> 24), im = (int)(t.x & 0xFFFFFFu);
        const int ty = (int)(t.y >> 16), tx = (int)(t.y & 0xFFFFu);
        gradient_tile<SAM_FP32, SAM_LAYOUT_PIXEL>(g.img[l] + (size_t)im * g.img_bytes[l], g.w[l], g.h[l], g.pitch[l],
                                                 g.low, g.field[l], (size_t)im * g.field_px[l], nullptr, nullptr,
                                                 g.vec, tx * GTX, ty * GTY);
        __syncthreads();   // the tile buffers are reused by the next tile
    }
}

// The gradient tiles of the refinement levels that the coarse-to-fine
// refinement of candidate blockIdx.y of image blockIdx.x can read: at level
// l the pixels within reach[l] of 2^(top - l) times the candidate's
// position.  Each tile is listed once (the first CTA to set its bit in the
// mask lists it).
__global__ void mark_tiles_kernel(const TileMarks a) {
    const int im = blockIdx.x, c = blockIdx.y;
    if (c >= min(a.count[im], a.K))
        return;
    const int32_t *q = a.kyx + ((size_t)im * a.K + c) * 3;
    const int xT = q[2] * a.step_x, yT = q[1] * a.step_y;
    for (int l = 0; l < a.nlev; ++l) {
        const int sc = 1 << (a.top - l);
        const int x0 = max(0, sc * xT + a.reach[l].x), x1 = min(a.w[l] - 1, sc * xT + a.reach[l].y);
        const int y0 = max(0, sc * yT + a.reach[l].z), y1 = min(a.h[l] - 1, sc * yT + a.reach[l].w);
        if (x0 > x1 || y0 > y1)
            continue;
        const int tx0 = x0 / GTX, tx1 = x1 / GTX, ty0 = y0 / GTY, ty1 = y1 / GTY;
        const int ntx = tx1 - tx0 + 1, nt = ntx * (ty1 - ty0 + 1);
        for (int i = threadIdx.x; i < nt; i += blockDim.x) {
            const int ty = ty0 + i / ntx, tx = tx0 + i % ntx;
            const size_t bit = a.tile_base[l] + ((size_t)im * a.tiles_y[l] + ty) * a.tiles_x[l] + tx;
            const uint32_t mb = 1u << (bit & 31);
            if (!(atomicOr(a.mask + (bit >> 5), mb) & mb)) {
                const unsigned pos = atomicAdd(a.list_cnt, 1u);
                if (pos < a.list_cap)
                    a.list[pos] = make_uint2(((unsigned)l << 24) | (unsigned)im, ((unsigned)ty << 16) | (unsigned)tx);
            }
        }
    }
}

}  // namespace

int gradient_tile_w() { return GTX; }
int gradient_tile_h() { return GTY; }

cudaError_t launch_refine_fields(const TileMarks &marks, const GradTiles &g, size_t clear_bytes, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(marks.mask, 0, clear_bytes, st);
    if (e != cudaSuccess)
        return e;
    mark_tiles_kernel<<<dim3((unsigned)marks.count_images, (unsigned)marks.K), 128, 0, st>>>(marks);
    gradient_tiles_kernel<<<152 * 8, GTHREADS, 0, st>>>(g);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_pyramid_jobs(const ImageJob *jobs, int n_jobs, int max_w, int max_h, cudaStream_t st) {
    if (n_jobs <= 0)
        return cudaSuccess;
    const int threads = 128;
    dim3 grid((unsigned)std::max(1, (max_w / 2 + 16 * threads - 1) / (16 * threads)),
              (unsigned)std::min(std::max(1, max_h / 2), 512), (unsigned)n_jobs);
    pyramid_jobs_kernel<<<grid, threads, 0, st>>>(jobs);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gradient_jobs(const ImageJob *jobs, int n_jobs, int max_w, int max_h, int low, int precision,
                                 int layout, cudaStream_t st) {
    if (n_jobs <= 0)
        return cudaSuccess;
    dim3 grid((unsigned)std::min((max_w + GTX - 1) / GTX, 32), (unsigned)std::min((max_h + GTY - 1) / GTY, 64),
              (unsigned)n_jobs);
    const bool pairs = layout == SAM_LAYOUT_PAIRS;
    switch (precision) {
    case SAM_FP32:
        if (pairs)
            gradient_jobs_kernel<SAM_FP32, SAM_LAYOUT_PAIRS><<<grid, GTHREADS, 0, st>>>(jobs, low);
        else
            gradient_jobs_kernel<SAM_FP32, SAM_LAYOUT_PIXEL><<<grid, GTHREADS, 0, st>>>(jobs, low);
        break;
    case SAM_BF16:
        if (pairs)
            gradient_jobs_kernel<SAM_BF16, SAM_LAYOUT_PAIRS><<<grid, GTHREADS, 0, st>>>(jobs, low);
        else
            gradient_jobs_kernel<SAM_BF16, SAM_LAYOUT_PIXEL><<<grid, GTHREADS, 0, st>>>(jobs, low);
        break;
    default:
        if (pairs)
            gradient_jobs_kernel<SAM_FP16, SAM_LAYOUT_PAIRS><<<grid, GTHREADS, 0, st>>>(jobs, low);
        else
            gradient_jobs_kernel<SAM_FP16, SAM_LAYOUT_PIXEL><<<grid, GTHREADS, 0, st>>>(jobs, low);
        break;
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_pyramid_down(const uint8_t *src, int w, int h, int src_stride, size_t src_img, uint8_t *dst,
                                int dst_stride, size_t dst_img, int count, cudaStream_t st) {
    const int w2 = w / 2, h2 = h / 2;
    if (w2 <= 0 || h2 <= 0 || count <= 0)
        return cudaSuccess;
    const int vec = ((uintptr_t)src % 16 == 0) && (src_stride % 16 == 0) && (count == 1 || src_img % 16 == 0) &&
                    ((uintptr_t)dst % 16 == 0) && (dst_stride % 16 == 0) && (count == 1 || dst_img % 16 == 0);
    const int threads = 128;
    dim3 grid((unsigned)((w2 + 16 * threads - 1) / (16 * threads)), (unsigned)h2, (unsigned)count);
    pyramid_down_kernel<<<grid, threads, 0, st>>>(src, w, h, src_stride, src_img, dst, dst_stride, dst_img, vec);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_pyramid_levels(const uint8_t *src, int w, int h, int src_stride, size_t src_img, int D,
                                  uint8_t *const *dst, const int *dst_stride, const size_t *dst_img, int count,
                                  cudaStream_t st) {
    if (D <= 0 || count <= 0)
        return cudaSuccess;
    if (D > 6 || (w >> 1) <= 0 || (h >> 1) <= 0) {
        // deeper pyramids: one launch per level
        const uint8_t *s = src;
        int sw = w, sh = h, sp = src_stride;
        size_t si = src_img;
        for (int l = 1; l <= D; ++l) {
            const cudaError_t e = launch_pyramid_down(s, sw, sh, sp, si, dst[l], dst_stride[l], dst_img[l], count, st);
            if (e != cudaSuccess)
                return e;
            s = dst[l];
            sw >>= 1;
            sh >>= 1;
            sp = dst_stride[l];
            si = dst_img[l];
        }
        return cudaSuccess;
    }
    PyramidLevels out;
    bool aligned = true;
    for (int l = 0; l < kMaxLevels; ++l) {
        out.dst[l] = l >= 1 && l <= D ? dst[l] : nullptr;
        out.pitch[l] = l >= 1 && l <= D ? dst_stride[l] : 0;
        out.img[l] = l >= 1 && l <= D ? dst_img[l] : 0;
        if (l >= 1 && l <= D)
            aligned = aligned && ((uintptr_t)dst[l] % 16 == 0) && (dst_stride[l] % 16 == 0) &&
                      (count == 1 || dst_img[l] % 16 == 0);
    }
    const int vec = aligned && ((uintptr_t)src % 16 == 0) && (src_stride % 16 == 0) &&
                    (count == 1 || src_img % 16 == 0);
    dim3 grid((unsigned)(((w >> 1) + kPyrBW / 2 - 1) / (kPyrBW / 2)), (unsigned)(((h >> 1) + kPyrBH / 2 - 1) / (kPyrBH / 2)),
              (unsigned)count);
    pyramid_levels_kernel<<<grid, 256, 0, st>>>(src, w, h, src_stride, src_img, out, D, vec);
    count_launches(1);
    return cudaGetLastError();
}

template <int PREC>
void gradient_dispatch(int layout, dim3 grid, cudaStream_t st, const uint8_t *img, int w, int h, int stride,
                       size_t img_bytes, int low, void *field, size_t field_img_px, int16_t *gx, int16_t *gy,
                       int vec) {
    if (layout == SAM_LAYOUT_PAIRS)
        gradient_kernel<PREC, SAM_LAYOUT_PAIRS><<<grid, GTHREADS, 0, st>>>(img, w, h, stride, img_bytes, low, field,
                                                                          field_img_px, gx, gy, vec);
    else
        gradient_kernel<PREC, SAM_LAYOUT_PIXEL><<<grid, GTHREADS, 0, st>>>(img, w, h, stride, img_bytes, low, field,
                                                                          field_img_px, gx, gy, vec);
}

cudaError_t launch_gradient(const uint8_t *img, int w, int h, int stride, size_t img_bytes, int low, int precision,
                            int layout, void *field, size_t field_img_px, int16_t *gx, int16_t *gy, int count,
                            cudaStream_t st) {
    if (w <= 0 || h <= 0 || count <= 0)
        return cudaSuccess;
    if ((layout == SAM_LAYOUT_PAIRS || precision == SAM_ANGLE16) && gx)
        return cudaErrorInvalidValue;
    const size_t esz = precision == SAM_FP32 ? 8 : (precision == SAM_ANGLE16 ? 2 : 4);
    const int vec = ((uintptr_t)img % 16 == 0) && (stride % 16 == 0) && (count == 1 || img_bytes % 16 == 0) &&
                    ((uintptr_t)field % 16 == 0) && (count == 1 || (field_img_px * esz) % 16 == 0) &&
                    (!gx || (((uintptr_t)gx % 16 == 0) && ((uintptr_t)gy % 16 == 0) &&
                             (count == 1 || field_img_px % 8 == 0)));
    dim3 grid((unsigned)((w + GTX - 1) / GTX), (unsigned)((h + GTY - 1) / GTY), (unsigned)count);
    switch (precision) {
    case SAM_FP32:
        gradient_dispatch<SAM_FP32>(layout, grid, st, img, w, h, stride, img_bytes, low, field, field_img_px, gx, gy,
                                    vec);
        break;
    case SAM_ANGLE16:
        // 16-byte code stores need 8-code-aligned rows and images
        gradient_dispatch<SAM_ANGLE16>(layout, grid, st, img, w, h, stride, img_bytes, low, field, field_img_px,
                                       nullptr, nullptr,
                                       vec && code_pitch(w, layout) % 8 == 0 && (count == 1 || field_img_px % 8 == 0));
        break;
    case SAM_BF16:
        gradient_dispatch<SAM_BF16>(layout, grid, st, img, w, h, stride, img_bytes, low, field, field_img_px, gx, gy,
                                    vec);
        break;
    default:
        gradient_dispatch<SAM_FP16>(layout, grid, st, img, w, h, stride, img_bytes, low, field, field_img_px, gx, gy,
                                    vec);
        break;
    }
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace sam
