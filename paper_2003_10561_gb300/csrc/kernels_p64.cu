// FP64 instantiation of the step kernels, 4th-order scheme (half width 2).
#define AT_DNS_SCALAR double
#define AT_DNS_HALF_WIDTH 2
#include "kernels_impl.cuh"
