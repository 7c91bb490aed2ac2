// lstsq.cu — placeholder.
#include "msk_internal.h"
extern "C" {
int msk_householder_qr(double*, int64_t, int64_t, int64_t, void*) { return MSK_ENOTSUP; }
int msk_trsv_upper(const double*, int64_t, int64_t, const double*, double*, void*) { return MSK_ENOTSUP; }
size_t msk_lstsq_workspace(int64_t, int64_t, int64_t, int64_t, int, int, int) { return 0; }
int ms_lstsq(const void*, int, int64_t, int64_t, int64_t, const double*, int64_t, int64_t, uint64_t,
             int, int, double, int32_t, double*, msk_lstsq_info*, void*, size_t, void*) { return MSK_ENOTSUP; }
size_t msk_ne_workspace(int64_t, int64_t) { return 0; }
int ne_lstsq(const double*, int64_t, int64_t, int64_t, const double*, double*, void*, size_t, void*) { return MSK_ENOTSUP; }
}
