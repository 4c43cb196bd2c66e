// Blocked LU (P1)-(P4) and the solve; filled in by the LU driver.
#include "ozlu_handle.h"

extern "C" int ozlu_getrf(ozlu_handle* h, int nc, int p, int n, double* A, long long lda,
                          int* ipiv, int nb, int* info, const ozlu_opts* opts) {
    (void)nc; (void)p; (void)n; (void)A; (void)lda; (void)ipiv; (void)nb; (void)info; (void)opts;
    if (!h) return -1;
    return OZLU_ERR_UNSUPPORTED;
}

extern "C" int ozlu_getrs(ozlu_handle* h, int nc, int p, int n, int nrhs, const double* LU,
                          long long lda, const int* ipiv, double* B, long long ldb,
                          const ozlu_opts* opts) {
    (void)nc; (void)p; (void)n; (void)nrhs; (void)LU; (void)lda; (void)ipiv; (void)B; (void)ldb;
    (void)opts;
    if (!h) return -1;
    return OZLU_ERR_UNSUPPORTED;
}
