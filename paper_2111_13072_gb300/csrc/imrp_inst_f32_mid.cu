// Per-degree kernels: precision float, degrees 12,16.
#include "imrp_inst.cuh"
IMRP_UNIT(register_f32_mid, float, 12,16)
