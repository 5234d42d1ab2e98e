// Per-degree kernels: precision double, degrees 1,2,4,8.
#include "imrp_inst.cuh"
IMRP_UNIT(register_f64_small, double, 1,2,4,8)
