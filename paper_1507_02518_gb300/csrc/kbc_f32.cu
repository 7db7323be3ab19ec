// kbc_f32.cu -- instantiation of the KBC kernels for FP32 storage (f - W) and FP32 arithmetic.
#include "kbc_kernels.cuh"

template struct kbc::Ops<float>;
