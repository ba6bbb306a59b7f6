// Instantiation of the kernels of the block sizes 6, 10, 12, 14 for T = double.
#include "kernels_ext_impl.cuh"

namespace lgf {

template struct LaunchExt<double>;

}  // namespace lgf
