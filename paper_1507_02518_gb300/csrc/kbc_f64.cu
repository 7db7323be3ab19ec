// kbc_f64.cu -- instantiation of the KBC kernels for FP64 storage and FP64 arithmetic.
#include "kbc_kernels.cuh"

template struct kbc::Ops<double>;
