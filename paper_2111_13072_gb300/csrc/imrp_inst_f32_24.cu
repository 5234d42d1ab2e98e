// Per-degree kernels: precision float, degrees 24.
#include "imrp_inst.cuh"
IMRP_UNIT(register_f32_24, float, 24)
