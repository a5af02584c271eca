// FP64 instantiation of the step kernels, 6th-order scheme (half width 3).
#define AT_DNS_SCALAR double
#define AT_DNS_HALF_WIDTH 3
#include "kernels_impl.cuh"
