// Per-degree kernels: precision double, degrees 24.
#include "imrp_inst.cuh"
IMRP_UNIT(register_f64_24, double, 24)
