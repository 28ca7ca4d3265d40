// Instantiation of the tiled scorers for BF16-stored fields (device code in
// score_tiled_kernels.cuh; one translation unit per field type so the
// variants compile in parallel).
#include "score_tiled_kernels.cuh"

namespace sam {

cudaError_t launch_tiled_bf16(const CUtensorMap &tm, const TiledArgs &a, dim3 grid, size_t smem, int nbhd, bool pol,
                           int warps, int tc, cudaStream_t st) {
    return tiled_dispatch<__nv_bfloat16>(tm, a, grid, smem, nbhd, pol, warps, tc, st);
}

cudaError_t launch_chunked_bf16(const CUtensorMap &tm, const ChunkArgs &a, dim3 grid, size_t smem, int nbhd, bool pol,
                             int warps, cudaStream_t st) {
    return chunked_dispatch<__nv_bfloat16>(tm, a, grid, smem, nbhd, pol, warps, st);
}

cudaError_t launch_chunk_bound_bf16(const void *field, int wp, int H, size_t img_px, bool pol, uint32_t *nplanes,
                                 const ChunkBoundArgs &b, cudaStream_t st) {
    return chunk_bound_dispatch<__nv_bfloat16>(field, wp, H, img_px, pol, nplanes, b, st);
}

cudaError_t launch_pairs_bf16(const PairScore *pairs, int n_pairs, int total, const TileConfig &cfg, int nbhd, bool pol,
                           int early, size_t smem, size_t win_bytes, unsigned *counter, int *err,
                           unsigned long long *exec, cudaStream_t st) {
    return pairs_dispatch<__nv_bfloat16>(pairs, n_pairs, total, cfg, nbhd, pol, early, smem, win_bytes, counter, err, exec,
                             st);
}

}  // namespace sam
