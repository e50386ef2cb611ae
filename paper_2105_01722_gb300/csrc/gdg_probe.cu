// FP64 throughput probe (measurement support; not part of the method).
//
// The constant-coefficient stage kernels are bound by the FP64 pipe, whose
// nominal rate on this GPU comes only from unit counts and the clock.  This
// kernel measures the rate the pipe actually sustains: every thread runs
// kChains independent chains x <- x * a + b of FP64 fused multiply-adds,
// kUnroll per chain per loop trip (no loads or stores inside the loop), on a grid that fills every SM.  The
// caller times the launch with CUDA events on the same stream; the flop
// count (an FMA counts 2) is returned through *flops.

#include "gdg_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 4;   // FMAs per chain per loop trip (loop overhead off the FP64 pipe)
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_fp64_fma_chains(int iters, double a, double b, double *sink) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < kUnroll; ++r)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    // keep every thread's chains live: a store that depends on them (the
    // condition is never met in practice; thread 0 of block 0 always stores)
    if (s == 12345.678 || (threadIdx.x == 0 && blockIdx.x == 0)) sink[0] = s;
}

}  // namespace

extern "C" int gdg_probe_fp64(int iters, double *sink, double *flops, void *stream) {
    if (iters < 1 || !sink || !flops) return GDG_EINVAL;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GDG_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GDG_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_fma_chains, kThreads, 0) != cudaSuccess)
        return GDG_ECUDA;
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    // x -> x a + b with a slightly below 1 and b = 1 - a keeps x near 1 (no
    // overflow, no subnormals) for any number of iterations
    const double a = 0.999999, b = 1.0 - a;
    k_fp64_fma_chains<<<blocks, kThreads, 0, (cudaStream_t)stream>>>(iters, a, b, sink);
    *flops = 2.0 * kChains * kUnroll * (double)iters * (double)kThreads * (double)blocks;
    return cudaGetLastError() == cudaSuccess ? GDG_OK : GDG_ECUDA;
}
