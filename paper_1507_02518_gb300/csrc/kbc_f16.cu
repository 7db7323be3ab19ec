// kbc_f16.cu -- instantiation of the KBC kernels for shifted FP16 storage ((f - W)/W) and FP32 arithmetic.
#include "kbc_kernels.cuh"

template struct kbc::Ops<uint16_t>;
