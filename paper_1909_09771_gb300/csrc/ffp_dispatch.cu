// ffp_dispatch.cu -- selects the kernel instantiation for the line length
// (slot count S) and the factor storage precision.
#include <cuda_bf16.h>

#include "ffp_kernels.h"

namespace ffp {

template <int S> cudaError_t setup_for_slots(const KernelCtx &, const double *, cudaStream_t);
template <int S, typename F>
cudaError_t apply_for_slots(const KernelCtx &, const double *, double *, cudaStream_t);

cudaError_t launch_setup(const KernelCtx &c, const double *t, cudaStream_t st) {
    switch (c.slots) {
#define FFP_CASE(SS) case SS: return setup_for_slots<SS>(c, t, st);
        FFP_SLOT_LIST(FFP_CASE)
#undef FFP_CASE
        default: return cudaErrorInvalidValue;
    }
}

template <typename F>
static cudaError_t apply_t(const KernelCtx &c, const double *r, double *z, cudaStream_t st) {
    switch (c.slots) {
#define FFP_CASE(SS) case SS: return apply_for_slots<SS, F>(c, r, z, st);
        FFP_SLOT_LIST(FFP_CASE)
#undef FFP_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_apply(const KernelCtx &c, const double *r, double *z, cudaStream_t st) {
    switch (c.prec) {
        case FFP_FP64: return apply_t<double>(c, r, z, st);
        case FFP_FP32: return apply_t<float>(c, r, z, st);
        case FFP_BF16: return apply_t<__nv_bfloat16>(c, r, z, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ffp
