// FFT pseudo-spectral periodic Poisson solve (Sec. 3.1): plans and buffers.
#pragma once
#include "ctx.h"

namespace pic {

struct FftState;
void fft_state_free(FftState* s);

}  // namespace pic
