// Throughput probes (measurement hooks): TF32 tensor, FP64 and FP32 fused multiply-add.
#pragma once

namespace rfdd {
// TFLOP/s measured on the current device: which = 0 plain TF32 tensor GEMM (8192^3, one MMA per
// product, kernel time only), 1 FP64 FMA on the CUDA cores, 2 FP32 FMA on the CUDA cores.
double peak_probe(int which);
}  // namespace rfdd
