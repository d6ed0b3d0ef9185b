// eval_tc.cu -- tensor-core (tcgen05) evaluation: placeholder until the kernel lands.
#include "fst_internal.cuh"

namespace fst {
fst_status eval_tc_launch(fst_model*, const float*, int64_t, float*, fst_prec, cudaStream_t) {
    set_error("tensor-core evaluation not built yet");
    return FST_EUNSUPPORTED;
}
}  // namespace fst
