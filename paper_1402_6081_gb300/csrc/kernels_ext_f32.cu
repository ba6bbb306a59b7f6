// Instantiation of the kernels of the block sizes 6, 10, 12, 14 for T = float.
#include "kernels_ext_impl.cuh"

namespace lgf {

template struct LaunchExt<float>;

bool persist_supported(int S) {
    switch (S) {
        case 8: case 10: case 12: case 16: case 17: case 18: case 20: case 24: case 28: case 32: case 33: case 34:
        case 36: return true;
        default: return persist_large_supported(S);
    }
}

}  // namespace lgf
