// Edge extraction arithmetic of kernel (a) (Sec. II edge extraction: 3x3
// Sobel, |g|/4 threshold, unit direction), in one place for every kernel
// that turns an integer gradient into a unit direction.
#pragma once

#include <stdint.h>

namespace sam {

// Unit gradient direction of an integer Sobel gradient, (0, 0) below the
// threshold (thr = 16 T^2) or for a zero gradient.
__device__ __forceinline__ float2 unit_of_gradient(int gx, int gy, int thr) {
    const int m2 = gx * gx + gy * gy;
    float fx = 0.f, fy = 0.f;
    if (m2 >= thr && m2 > 0) {
        const float inv = rsqrtf((float)m2);
        fx = (float)gx * inv;
        fy = (float)gy * inv;
    }
    return make_float2(fx, fy);
}

}  // namespace sam
