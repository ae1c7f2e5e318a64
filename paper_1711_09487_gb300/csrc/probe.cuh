// Throughput probes (measurement hooks): TF32 tensor, FP64 and FP32 fused multiply-add.
#pragma once

namespace rfdd {
// TFLOP/s measured on the current device: which = 0 TF32 MMAs from shared memory (the tensor
// pipe's rate), 1 FP64 FMA on the CUDA cores, 2 FP32 FMA on the CUDA cores, 3 plain TF32 GEMM
// through the tensor-core kernel (8192^3, one MMA per product, kernel time only).
double peak_probe(int which);
}  // namespace rfdd
