// Persistent interaction-list products (FP32) for the transform lengths of
// the block sizes 18..32: level 0 at S0 = 2 n_b (36 is built with the base
// sizes) and the interval levels at S_I = 2 n_b + 2, i.e. every even S of
// [38, 66].  Same kernel as the base sizes (k_mac_persist), instantiated here
// so its compile runs beside the other units.
#include "kernels_impl.cuh"

namespace lgf {

bool persist_large_supported(int S) { return S >= 38 && S <= 66 && S % 2 == 0; }

cudaError_t mac_persist_large(const void* fh, const void* kh, void* uh, const PersistPlan& pp, int S, int early,
                              cudaStream_t st) {
#define LGF_MACP(SS) \
    case SS: return launch_mac_persist_form<SS>(fh, kh, uh, pp, early, st);
    switch (S) {
        LGF_MACP(38) LGF_MACP(40) LGF_MACP(42) LGF_MACP(44) LGF_MACP(46) LGF_MACP(48) LGF_MACP(50) LGF_MACP(52)
        LGF_MACP(54) LGF_MACP(56) LGF_MACP(58) LGF_MACP(60) LGF_MACP(62) LGF_MACP(64) LGF_MACP(66)
        default: return cudaErrorInvalidValue;
    }
#undef LGF_MACP
}

}  // namespace lgf
