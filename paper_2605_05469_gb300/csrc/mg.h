// Internal interface between the solver (capi.cu) and the multigrid
// preconditioner (mg.cu).
#pragma once

struct pic_ctx;

namespace pic {

struct MgState;

void mg_state_free(MgState* s);
// z = V(r): one V-cycle on the context grid for the scaled system
// (6 I - adj) z = r (FP32 device arrays, N^3), enqueued on the context
// stream; learned = the network's composed kernel smooths the finest level.
// done (device flag, may be null): when set, the launched kernels return at
// once (iterations launched past convergence).
// sample: time the finest level's kernels with the PIC_KER_MG_* event pools
// (profiling on).
int mg_apply(pic_ctx* c, const float* r, float* z, bool learned, const int* done, bool sample = false);

}  // namespace pic
