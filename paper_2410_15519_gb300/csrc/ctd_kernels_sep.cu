// The step kernel with the separated nonlinear term (Eq. MxySep), compiled as its own
// translation unit from the same step code: the grid-form kernels hold none of its code.
#define CTD_SEPARATED_TU
#include "ctd_kernels.cu"
