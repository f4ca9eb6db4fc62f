// ffp_dispatch.cu -- selects the kernel instantiation for the line length
// (slot count S) and the factor storage precision.
#include <cuda_bf16.h>

#include "ffp_kernels.h"

namespace ffp {

template <int S> cudaError_t setup_for_slots(const KernelCtx &, const double *, cudaStream_t);
template <int S> cudaError_t setup_table_for_slots(const SetupArgs *, int, int, cudaStream_t);
template <int S, typename F>
cudaError_t apply_for_slots(const KernelCtx &, const double *, double *, cudaStream_t,
                            const cudaEvent_t *, const double *);
template <int S, typename F>
cudaError_t apply_table_for_slots(const ApplyArgs *, int, int, int, cudaStream_t);
template <int S, typename F>
bool two_rhs_supported();

cudaError_t launch_setup(const KernelCtx &c, const double *t, cudaStream_t st) {
    switch (c.slots) {
#define FFP_CASE(SS) case SS: return setup_for_slots<SS>(c, t, st);
        FFP_SLOT_LIST(FFP_CASE)
#undef FFP_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_setup_table(int slots, const SetupArgs *table, int count, int nx_max,
                               cudaStream_t st) {
    switch (slots) {
#define FFP_CASE(SS) case SS: return setup_table_for_slots<SS>(table, count, nx_max, st);
        FFP_SLOT_LIST(FFP_CASE)
#undef FFP_CASE
        default: return cudaErrorInvalidValue;
    }
}

template <typename F>
static cudaError_t apply_t(const KernelCtx &c, const double *r, double *z, cudaStream_t st,
                           const cudaEvent_t *ev, const double *add) {
    switch (c.slots) {
#define FFP_CASE(SS) case SS: return apply_for_slots<SS, F>(c, r, z, st, ev, add);
        FFP_SLOT_LIST(FFP_CASE)
#undef FFP_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_apply(const KernelCtx &c, const double *r, double *z, cudaStream_t st,
                         const cudaEvent_t *ev, const double *add) {
    switch (c.prec) {
        case FFP_FP64: return apply_t<double>(c, r, z, st, ev, add);
        case FFP_FP32: return apply_t<float>(c, r, z, st, ev, add);
        case FFP_BF16: return apply_t<__nv_bfloat16>(c, r, z, st, ev, add);
        default: return cudaErrorInvalidValue;
    }
}

template <typename F>
static cudaError_t apply_table_t(int slots, const ApplyArgs *t, int n, int nxm, int nr, cudaStream_t st) {
    switch (slots) {
#define FFP_CASE(SS) case SS: return apply_table_for_slots<SS, F>(t, n, nxm, nr, st);
        FFP_SLOT_LIST(FFP_CASE)
#undef FFP_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_apply_table(int prec, int slots, const ApplyArgs *table, int n, int nx_max, int nr,
                               cudaStream_t st) {
    switch (prec) {
        case FFP_FP64: return apply_table_t<double>(slots, table, n, nx_max, nr, st);
        case FFP_FP32: return apply_table_t<float>(slots, table, n, nx_max, nr, st);
        case FFP_BF16: return apply_table_t<__nv_bfloat16>(slots, table, n, nx_max, nr, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename F>
static bool two_rhs_t(int slots) {
    switch (slots) {
#define FFP_CASE(SS) case SS: return two_rhs_supported<SS, F>();
        FFP_SLOT_LIST(FFP_CASE)
#undef FFP_CASE
        default: return false;
    }
}

bool apply_two_rhs_ok(int prec, int slots) {
    switch (prec) {
        case FFP_FP64: return two_rhs_t<double>(slots);
        case FFP_FP32: return two_rhs_t<float>(slots);
        case FFP_BF16: return two_rhs_t<__nv_bfloat16>(slots);
        default: return false;
    }
}

}  // namespace ffp
