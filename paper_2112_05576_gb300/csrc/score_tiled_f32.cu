// Instantiation of the tiled scorers for FP32-stored fields (device code in
// score_tiled_kernels.cuh; one translation unit per field type so the
// variants compile in parallel).
#include "score_tiled_kernels.cuh"

namespace sam {

cudaError_t launch_tiled_f32(const CUtensorMap &tm, const TiledArgs &a, dim3 grid, size_t smem, int nbhd, bool pol,
                           int warps, int tc, cudaStream_t st) {
    return tiled_dispatch<float>(tm, a, grid, smem, nbhd, pol, warps, tc, st);
}

cudaError_t launch_chunked_f32(const CUtensorMap &tm, const ChunkArgs &a, dim3 grid, size_t smem, int nbhd, bool pol,
                             int warps, cudaStream_t st) {
    return chunked_dispatch<float>(tm, a, grid, smem, nbhd, pol, warps, st);
}

cudaError_t launch_chunk_bound_f32(const void *field, int wp, int H, size_t img_px, bool pol, uint32_t *nplanes,
                                 const ChunkBoundArgs &b, cudaStream_t st) {
    return chunk_bound_dispatch<float>(field, wp, H, img_px, pol, nplanes, b, st);
}

cudaError_t launch_pairs_f32(const PairScore *pairs, int n_pairs, int total, const TileConfig &cfg, int nbhd, bool pol,
                           int early, size_t smem, size_t win_bytes, unsigned *counter, int *err,
                           unsigned long long *exec, cudaStream_t st) {
    return pairs_dispatch<float>(pairs, n_pairs, total, cfg, nbhd, pol, early, smem, win_bytes, counter, err, exec,
                             st);
}

cudaError_t launch_wait_selftest(int *err, unsigned long long limit_ns, unsigned long long *waited_ns, int mode,
                                 unsigned *fake, cudaStream_t st) {
    wait_selftest_kernel<<<1, 32, 0, st>>>(err, limit_ns, waited_ns, mode, fake);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace sam
