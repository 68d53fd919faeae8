// Red-black SSOR preconditioner (the paper's PCG configuration, Sec. 4.1).
#pragma once
#include "ctx.h"

namespace pic {

// z = M r on the solver's scaled system (h^2 A) z = r (r, z FP32 device,
// N^3), enqueued on the context stream. done (device flag, may be null): the
// kernels return at once when it is set.
int ssor_apply(pic_ctx* c, const float* r, float* z, const int* done);

}  // namespace pic
