// FP32-bulk instantiation of the step kernels.
#define AT_DNS_SCALAR float
#include "kernels_impl.cuh"
