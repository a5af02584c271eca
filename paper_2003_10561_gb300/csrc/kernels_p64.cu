// FP64 instantiation of the step kernels.
#define AT_DNS_SCALAR double
#include "kernels_impl.cuh"
