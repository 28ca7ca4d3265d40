// Instantiation of the single-level tiled scorers for angle-code fields
// (SAM_ANGLE16: the window is staged as 16-bit codes and expanded to FP32
// unit vectors in shared memory; device code in score_tiled_kernels.cuh).
#include "score_tiled_kernels.cuh"

namespace sam {

cudaError_t launch_tiled_a16(const CUtensorMap &tm, const TiledArgs &a, dim3 grid, size_t smem, int nbhd, bool pol,
                             int warps, int tc, cudaStream_t st) {
    return tiled_dispatch<AngleCode>(tm, a, grid, smem, nbhd, pol, warps, tc, st);
}

}  // namespace sam
