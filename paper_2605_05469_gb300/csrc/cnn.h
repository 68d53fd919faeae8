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
// Whether the context's preconditioner runs as the tensor-core composed
// kernel, and whether flexible CG fuses its update into it (the forms below).
bool cnn_tc_ok(const pic_ctx* c);
bool cnn_fused_ok(const pic_ctx* c);
// One flexible-CG step fused around the preconditioner (tensor-core form):
// r_new = r - alpha q, x += alpha p, z = N r_new, plus the update's and the
// direction's reductions and bookkeeping in the context scalars.
int cnn_apply_fused(pic_ctx* c, const float* r, float* r_new, float* z, const float* q, const float* p, float* x);
// z = N r, only if a reliable update replaced r in this iteration.
int cnn_apply_redo(pic_ctx* c, const float* r, float* z);
// The training state: FP32 master weights, Adam moments m and v (three
// blocks of PIC_CNN_WEIGHTS floats in device memory) and the Adam step count.
// cnn_state_set also clears the gradients and rebuilds the packed and
// composed inference kernels. Both enqueue on the context stream.
int cnn_state_get(pic_ctx* c, float* dev3, int* adam_t);
int cnn_state_set(pic_ctx* c, const float* dev3, int adam_t);

}  // namespace pic
