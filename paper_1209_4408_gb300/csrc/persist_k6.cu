// Persistent dataflow step kernel, 6 generations per pass.
#include "wavefront.cuh"

namespace gol {
GOL_INSTANTIATE_PERSISTENT(6)
}  // namespace gol
