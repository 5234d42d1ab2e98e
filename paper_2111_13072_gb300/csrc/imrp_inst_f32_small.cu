// Per-degree kernels: precision float, degrees 1,2,4,8.
#include "imrp_inst.cuh"
IMRP_UNIT(register_f32_small, float, 1,2,4,8)
