// Per-degree kernels: precision double, degrees 12,16.
#include "imrp_inst.cuh"
IMRP_UNIT(register_f64_mid, double, 12,16)
