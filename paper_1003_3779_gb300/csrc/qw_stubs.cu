// qw_stubs.cu -- entry points whose kernels live in later translation units.
#include "qw_handle.h"

extern "C" {

struct qw_batch_placeholder;

qw_status qw_backward(qw_walk *w, const int64_t rect[4], int64_t T, int64_t K, double *loss_out,
                      double *grad_phi, int on_device) {
    (void)rect; (void)T; (void)K; (void)loss_out; (void)grad_phi; (void)on_device;
    if (!w) return QW_EINVAL;
    return qw::set_error(w, QW_EUNSUPPORTED, "qw_backward is not built yet");
}

qw_status qw_batch_create(int, const int64_t *, const int64_t *, const double *, const int64_t *,
                          const double *, qw_precision, void *, qw_batch **out) {
    if (out) *out = nullptr;
    return QW_EUNSUPPORTED;
}
qw_status qw_batch_step(qw_batch *) { return QW_EUNSUPPORTED; }
qw_status qw_batch_probabilities(qw_batch *, float *, int, double *) { return QW_EUNSUPPORTED; }
qw_status qw_batch_get_state(qw_batch *, int, void *, qw_cdtype) { return QW_EUNSUPPORTED; }
qw_status qw_batch_destroy(qw_batch *) { return QW_OK; }
const char *qw_batch_last_error(const qw_batch *) { return "batches are not built yet"; }
}
