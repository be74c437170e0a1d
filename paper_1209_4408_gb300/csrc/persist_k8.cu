// Persistent dataflow step kernel, 8 generation(s) per pass.
#include "wavefront.cuh"

namespace gol {
GOL_INSTANTIATE_PERSISTENT(8)
}  // namespace gol
