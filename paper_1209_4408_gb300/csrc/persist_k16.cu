// Persistent dataflow step kernel, 16 generation(s) per pass.
#include "wavefront.cuh"

namespace gol {
GOL_INSTANTIATE_PERSISTENT(16)
}  // namespace gol
