// Explicit instantiations of the setup kernels for a subset of the line
// slot counts (split across TUs so the build compiles them in parallel).
#include "ffp_setup.cuh"

namespace ffp {
#define X(SS)                                                                                   \
    template cudaError_t setup_for_slots<SS>(const KernelCtx &, const double *, cudaStream_t); \
    template cudaError_t setup_table_for_slots<SS>(const SetupArgs *, int, int, cudaStream_t);
X(8) X(11)
#undef X
}  // namespace ffp

#ifdef FFP_STEP_PROFILE
// Profiling builds only (build.py --profile; not part of include/ffp.h): the setup
// profile of the last setup with the slot counts of this unit, 16 counters.
extern "C" int ffp_setup_profile(unsigned long long *host16) {
    return ffp::setup_profile_read(host16) == cudaSuccess ? 0 : -2;
}
#endif
