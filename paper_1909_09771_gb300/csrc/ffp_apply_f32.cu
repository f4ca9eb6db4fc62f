// Explicit instantiations of the apply kernels for float factors (one TU per
// storage precision so the build compiles them in parallel).
#include "ffp_apply.cuh"

namespace ffp {
#define FFP_INST(SS) template cudaError_t apply_for_slots<SS, float>(const KernelCtx &, const double *, double *, cudaStream_t, const cudaEvent_t *, const double *); \
    template cudaError_t apply_table_for_slots<SS, float>(const ApplyArgs *, int, int, int, cudaStream_t); \
    template bool two_rhs_supported<SS, float>();
FFP_SLOT_LIST(FFP_INST)
#undef FFP_INST
}  // namespace ffp

#ifdef FFP_STEP_PROFILE
// Profiling builds only (build.py --profile; not part of include/ffp.h): the
// step profile of the last FP32-factor apply, 16 counters (see g_step_prof).
extern "C" int ffp_step_profile(unsigned long long *host16) {
    return ffp::step_profile_read(host16) == cudaSuccess ? 0 : -2;
}
#endif
