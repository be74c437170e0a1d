// Persistent dataflow step kernel, 2 generation(s) per pass.
#include "wavefront.cuh"

namespace gol {
GOL_INSTANTIATE_PERSISTENT(2)
}  // namespace gol
