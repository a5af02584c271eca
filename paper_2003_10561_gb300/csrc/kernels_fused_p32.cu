// FP32-bulk instantiation of the fused step kernel.
#define AT_DNS_SCALAR float
#include "fused_impl.cuh"
