// Tile alignment (Sec. 3.2) for motion tiles of 32 raw px (16-texel tiles on every level):
// the searches and the refinement, instantiated in their own translation unit.
#include "align_search.cuh"

namespace hmfsr {
template cudaError_t align_search_tiles<16>(const Geom &, const hmfsr_align_params &, const AlignLevels &, float *,
                                           int32_t *, cudaStream_t);
template cudaError_t align_quadfit_tiles<16>(const Geom &, const AlignLevels &, float *, int32_t *, cudaStream_t);
}  // namespace hmfsr
