// Explicit instantiations of the apply kernels for double factors (one TU per
// storage precision so the build compiles them in parallel).
#include "ffp_apply.cuh"

namespace ffp {
#define FFP_INST(SS) template cudaError_t apply_for_slots<SS, double>(const KernelCtx &, const double *, double *, cudaStream_t, const cudaEvent_t *, const double *); \
    template cudaError_t apply_table_for_slots<SS, double>(const ApplyArgs *, int, int, int, cudaStream_t); \
    template bool two_rhs_supported<SS, double>();
FFP_SLOT_LIST(FFP_INST)
#undef FFP_INST
}  // namespace ffp
