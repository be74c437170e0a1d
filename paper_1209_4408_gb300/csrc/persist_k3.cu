// Persistent dataflow step kernel, 3 generations per pass.
#include "wavefront.cuh"

namespace gol {
GOL_INSTANTIATE_PERSISTENT(3)
}  // namespace gol
