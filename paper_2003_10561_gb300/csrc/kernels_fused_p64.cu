// FP64 instantiation of the fused step kernel.
#define AT_DNS_SCALAR double
#include "fused_impl.cuh"
