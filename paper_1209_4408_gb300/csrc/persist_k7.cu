// Persistent dataflow step kernel, 7 generations per pass.
#include "wavefront.cuh"

namespace gol {
GOL_INSTANTIATE_PERSISTENT(7)
}  // namespace gol
