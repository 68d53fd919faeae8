// Particle-in-Fourier field (Sec. 3.4, Appendix A): plans and buffers.
#pragma once
#include "ctx.h"

namespace pic {

struct PifState;
void pif_state_free(PifState* s);

// Field at the particles, Ep = (E_x, E_y, E_z) [3 np] FP64 in the current
// particle order, from type-1 / type-2 NUFFTs with a window width chosen for
// the relative tolerance tol. Enqueued on the context stream.
int pif_field(pic_ctx* c, double tol, double* Ep);

}  // namespace pic
