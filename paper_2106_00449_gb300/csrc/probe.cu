// FP32 FMA throughput probe: the denominator of the pair kernels' roofline, measured.
// Each thread runs 8 independent chains of FP32 pairs, x <- x a + b lane by lane, for
// `iters` iterations, with no other instruction in the loop body but the loop counter, and
// writes the sum of its chains (so nothing is eliminated).  MODE 0 issues scalar FMAs
// (fma.rn.f32, 16 per iteration), MODE 1 packed ones (fma.rn.f32x2, 8 per iteration, the
// form the pair kernels use), MODE 2 half and half (4 packed + 8 scalar).  All three compute
// the same values with the same roundings; work per launch: blocks x 256 threads x iters x
// 32 flops.
#include "common.cuh"
#include "pair_common.cuh"

namespace gdc {

template <int MODE>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, float* __restrict__ out) {
    const float s = 1e-3f * (float)(threadIdx.x & 7);
    const float2 a = make_float2(0.999f, 0.998f), b = make_float2(1e-3f, 2e-3f);
    float2 x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = make_float2(s + k, s - k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (MODE == 1 || (MODE == 2 && k < 4)) {
                x[k] = fma2(x[k], a, b);
            } else {
                x[k].x = fmaf(x[k].x, a.x, b.x);
                x[k].y = fmaf(x[k].y, a.y, b.y);
            }
        }
    }
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) acc += x[k].x + x[k].y;
    out[blockIdx.x * 256 + threadIdx.x] = acc;
}

}  // namespace gdc

extern "C" gdc_status gdc_fma_probe(int mode, int n_blocks, int iters, float* out, void* stream) {
    if (mode < 0 || mode > 2 || n_blocks < 1 || iters < 1 || !out) return GDC_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (mode == 1)
        gdc::k_fma_probe<1><<<n_blocks, 256, 0, st>>>(iters, out);
    else if (mode == 2)
        gdc::k_fma_probe<2><<<n_blocks, 256, 0, st>>>(iters, out);
    else
        gdc::k_fma_probe<0><<<n_blocks, 256, 0, st>>>(iters, out);
    return cudaGetLastError() == cudaSuccess ? GDC_OK : GDC_ERR_CUDA;
}
