// Split-precision tensor-core path (exact BF16 digit planes on tcgen05). Placeholder until the
// kernels land: every entry refuses with NOF_EINVAL so the option cannot silently fall back.
#include "internal.h"

struct FastState {};

int fast_prepare(nof_ctx* c) {
    (void)c;
    nof_set_error("NOF_PREC_SPLIT_BF16 is not available in this build");
    return NOF_EINVAL;
}
int fast_release(nof_ctx* c) {
    c->fast = nullptr;
    return NOF_OK;
}
int fast_jk(nof_ctx* c, const double* C) {
    (void)c; (void)C;
    nof_set_error("NOF_PREC_SPLIT_BF16 is not available in this build");
    return NOF_EINVAL;
}
int fast_grad(nof_ctx* c, const double* C, const double* gamma, bool want_grad) {
    (void)c; (void)C; (void)gamma; (void)want_grad;
    nof_set_error("NOF_PREC_SPLIT_BF16 is not available in this build");
    return NOF_EINVAL;
}
int fast_get_B(nof_ctx* c, double* B) {
    (void)c; (void)B;
    nof_set_error("NOF_PREC_SPLIT_BF16 is not available in this build");
    return NOF_EINVAL;
}
