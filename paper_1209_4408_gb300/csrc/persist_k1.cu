// Persistent dataflow step kernel, 1 generation(s) per pass.
#include "wavefront.cuh"

namespace gol {
GOL_INSTANTIATE_PERSISTENT(1)
}  // namespace gol
