// Entry points whose kernels are not built yet: they reject every call.
#include "apm_internal.cuh"

extern "C" {
apm_status_t apm_keldysh_sum(const double *, int, int64_t, int, double *, double *, uint32_t *,
                             apm_stream_t) {
    return APM_ERR_UNSUPPORTED_N;
}
apm_status_t apm_perm_minors(const double *, int, int64_t, double *, void *, size_t, apm_stream_t) {
    return APM_ERR_UNSUPPORTED_N;
}
}
