// Persistent dataflow step kernel, 4 generation(s) per pass.
#include "wavefront.cuh"

namespace gol {
GOL_INSTANTIATE_PERSISTENT(4)
}  // namespace gol
