// Internal interface between the solver (capi.cu) and the learned
// preconditioner (cnn.cu).
#pragma once
#include <stddef.h>

struct pic_ctx;

namespace pic {

struct CnnState;

void cnn_state_free(CnnState* s);
bool cnn_ready(const pic_ctx* c);
// z = s N(r / s), s = sqrt(*rr / n): the network applied to the periodic
// N^3 field r (FP32), enqueued on the context stream.
int cnn_apply(pic_ctx* c, const float* r, float* z, const double* rr, size_t n);

}  // namespace pic
