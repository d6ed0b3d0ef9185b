// gram_tc.cu -- tensor-core (tcgen05) Gram assembly: placeholder until the kernel lands.
#include "fst_internal.cuh"

namespace fst {
fst_status gram_tc_launch(const fst_model*, const float*, const float*, const float*, int64_t, float*, fst_prec,
                          cudaStream_t) {
    set_error("tensor-core Gram assembly not built yet");
    return FST_EUNSUPPORTED;
}
}  // namespace fst
