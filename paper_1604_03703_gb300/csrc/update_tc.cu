// update_tc.cu -- tensor-core (tcgen05) forms of the trailing update.
// Placeholder: the mixed form falls back to the SIMT kernels until the
// tcgen05 kernels are in place.
#include "common.cuh"

namespace sev {

template <typename T>
int tc_update_supported(sev_ctx *, int, int) {
    return 0;
}
template <typename T>
int tc_symm(sev_ctx *, int, int, const T *, int, const T *, T *, void *) {
    return SEV_ERR_UNSUPPORTED;
}
template <typename T>
int tc_syr2k(sev_ctx *, int, int, T *, int, const T *, const T *, void *) {
    return SEV_ERR_UNSUPPORTED;
}
template <typename T>
size_t tc_workspace(int, int) {
    return 0;
}

template int tc_update_supported<float>(sev_ctx *, int, int);
template int tc_update_supported<double>(sev_ctx *, int, int);
template int tc_symm<float>(sev_ctx *, int, int, const float *, int, const float *, float *, void *);
template int tc_symm<double>(sev_ctx *, int, int, const double *, int, const double *, double *, void *);
template int tc_syr2k<float>(sev_ctx *, int, int, float *, int, const float *, const float *, void *);
template int tc_syr2k<double>(sev_ctx *, int, int, double *, int, const double *, const double *, void *);
template size_t tc_workspace<float>(int, int);
template size_t tc_workspace<double>(int, int);

}  // namespace sev
