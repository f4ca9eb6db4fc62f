// Explicit instantiations of the setup kernels for a subset of the line
// slot counts (split across TUs so the build compiles them in parallel).
#include "ffp_setup.cuh"

namespace ffp {
#define X(SS)                                                                                   \
    template cudaError_t setup_for_slots<SS>(const KernelCtx &, const double *, cudaStream_t); \
    template cudaError_t setup_table_for_slots<SS>(const SetupArgs *, int, int, cudaStream_t);
X(32)
#undef X
}  // namespace ffp
