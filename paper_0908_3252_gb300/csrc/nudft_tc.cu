// nudft_tc.cu -- tensor-core (tcgen05) contractions; placeholder until the
// split-precision kernels land.
#include "internal.cuh"

namespace spirec {

size_t kpart_floats_tc(int, int64_t, int) { return 0; }
int tc_setup_attributes() { return SPIREC_OK; }

int launch_gram_tc(spirec_plan)
{
    set_error("mixed-precision contraction not built");
    return SPIREC_EUNSUPPORTED;
}

int launch_adjoint_tc(spirec_plan, const float2*, float2*)
{
    set_error("mixed-precision contraction not built");
    return SPIREC_EUNSUPPORTED;
}

}  // namespace spirec
