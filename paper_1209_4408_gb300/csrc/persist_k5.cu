// Persistent dataflow step kernel, 5 generations per pass.
#include "wavefront.cuh"

namespace gol {
GOL_INSTANTIATE_PERSISTENT(5)
}  // namespace gol
