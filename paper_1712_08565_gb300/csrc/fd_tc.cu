// Tensor-core (tcgen05) FD mode products: placeholder translation unit, filled
// in with the TF32/BF16 kernels.
#include <cuda_runtime.h>

#include "kernels.h"
