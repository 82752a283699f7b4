// probe_kernels.cuh -- a measurement kernel, not a step of the method: the GPU's
// binary64 FMA issue rate, the peak against which the kernels bound by the FP64
// pipe (the binary64 column solve) are reported.
//
// Every thread runs CHAINS independent chains a <- a * x + y of `iters` FMAs
// each (no dependence between chains, so a warp always has an FMA ready); the
// sum of the chains is stored only when it equals a value it never takes, which
// keeps every FMA live without a store per thread.  With x in (0, 1) and y small
// the chains converge to y / (1 - x): no overflow, no subnormals.
#pragma once

#include <cuda_runtime.h>

namespace gtb {

constexpr int kFp64ProbeChains = 8;

__global__ void __launch_bounds__(256) fp64_fma_probe_kernel(int iters, double x, double y, double *sink) {
    double a[kFp64ProbeChains];
#pragma unroll
    for (int c = 0; c < kFp64ProbeChains; ++c) a[c] = 1e-3 * (threadIdx.x + 1) + c;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kFp64ProbeChains; ++c) a[c] = fma(a[c], x, y);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kFp64ProbeChains; ++c) s += a[c];
    if (s == -1.0) sink[0] = s;  // never true: the chains stay positive
}

}  // namespace gtb
