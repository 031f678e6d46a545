// Throughput of the FP32 pipe on this device, measured: independent FMA
// chains (scalar fmaf, and packed fma.rn.f32x2 on two lanes per
// instruction) in registers only, enough warps per SM to hide the FMA
// latency.  It gives the near-field kernel's FP32 roofline a measured
// companion to the count-based figure (SMs x 128 lanes x clock).  No
// counterpart in the paper.
#include "common.cuh"

#include <algorithm>

namespace hsma {

namespace {

constexpr int kPeakThreads = 128;
constexpr int kPeakCtasPerSm = 16;
constexpr int kPeakChains = 16;  // scalar chains per thread (packed: 8 pairs)

__global__ void __launch_bounds__(kPeakThreads) peak_fma_kernel(float *out, int iters)
{
    float acc[kPeakChains];
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) acc[j] = threadIdx.x * 1e-3f + j;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kPeakChains; ++j) acc[j] = fmaf(acc[j], 0.999f, 1e-3f);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) s += acc[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) peak_fma2_kernel(float *out, int iters)
{
    float2 acc[kPeakChains / 2];
#pragma unroll
    for (int j = 0; j < kPeakChains / 2; ++j) acc[j] = make_float2(threadIdx.x * 1e-3f + j, 0.5f * j);
    const float2 m = make_float2(0.999f, 0.998f), c = make_float2(1e-3f, 2e-3f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kPeakChains / 2; ++j) acc[j] = __ffma2_rn(acc[j], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kPeakChains / 2; ++j) s += acc[j].x + acc[j].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

}  // namespace hsma

using namespace hsma;

extern "C" int hsma_fp32_peak(double *scalar_lane_ops_per_s, double *packed_lane_ops_per_s)
{
    if (!scalar_lane_ops_per_s || !packed_lane_ops_per_s) return HSMA_E_ARG;
    int dev = 0, sms = 0;
    HSMA_CUDA_TRY(cudaGetDevice(&dev));
    HSMA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = sms * kPeakCtasPerSm, iters = 20000;
    float *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = HSMA_OK;
    auto cuda_ok = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == HSMA_OK) rc = HSMA_E_CUDA;
        return rc == HSMA_OK;
    };
    if (cuda_ok(dev_malloc(&out, sizeof(float) * grid * kPeakThreads)) &&
        cuda_ok(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) && cuda_ok(cudaEventCreate(&e0)) &&
        cuda_ok(cudaEventCreate(&e1))) {
        double best[2] = {0.0, 0.0};
        for (int rep = 0; rep < 3 && rc == HSMA_OK; ++rep) {  // rep 0 also warms the clocks
            for (int k = 0; k < 2 && rc == HSMA_OK; ++k) {
                cuda_ok(cudaEventRecord(e0, st));
                if (k == 0)
                    peak_fma_kernel<<<grid, kPeakThreads, 0, st>>>(out, iters);
                else
                    peak_fma2_kernel<<<grid, kPeakThreads, 0, st>>>(out, iters);
                HSMA_LAUNCHED();
                cuda_ok(cudaGetLastError());
                cuda_ok(cudaEventRecord(e1, st));
                cuda_ok(cudaEventSynchronize(e1));
                float ms = 0.f;
                if (cuda_ok(cudaEventElapsedTime(&ms, e0, e1)) && ms > 0.f) {
                    const double ops = (double)kPeakChains * iters * grid * kPeakThreads;  // lane FMAs
                    best[k] = std::max(best[k], ops / (ms * 1e-3));
                }
            }
        }
        *scalar_lane_ops_per_s = best[0];
        *packed_lane_ops_per_s = best[1];
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (out) dev_free(out);
    return rc;
}
