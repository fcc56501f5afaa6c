// peaks.cu -- arithmetic throughput probes for the roofline denominators of the
// hopping kernels (sm_103a): FP64 DFMA, FP32 FFMA, paired FP32 FFMA2 and FP16
// HFMA2.  Each thread runs kChains independent FMA recurrences (so the pipes,
// not the FMA latency, bound the rate) on loop-invariant operands that keep the
// values normal; 8 CTAs of 256 threads per SM keep every scheduler busy.  The
// result is written only under a condition the data never meets, so nothing
// is optimised away.  Built as libdwf_probe.so beside libdwf.so.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <int KIND>
__global__ void __launch_bounds__(kThreads) fma_probe(int iters, float* sink) {
  if constexpr (KIND == 0) {  // FP64 DFMA
    double a[kChains];
    const double b = 0.999999, c = 1e-6;
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    for (int i = 0; i < iters; i++)
#pragma unroll
      for (int k = 0; k < kChains; k++) a[k] = fma(a[k], b, c);
    double s = 0;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += a[k];
    if (s == 12345.0) sink[0] = (float)s;
  } else if constexpr (KIND == 1) {  // FP32 FFMA
    float a[kChains];
    const float b = 0.9999f, c = 1e-4f;
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = 1.f + 1e-3f * (threadIdx.x + k);
    for (int i = 0; i < iters; i++)
#pragma unroll
      for (int k = 0; k < kChains; k++) a[k] = fmaf(a[k], b, c);
    float s = 0;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += a[k];
    if (s == 12345.f) sink[0] = s;
  } else if constexpr (KIND == 2) {  // paired FP32 FFMA2
    float2 a[kChains];
    const float2 b = make_float2(0.9999f, 0.9998f), c = make_float2(1e-4f, 2e-4f);
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = make_float2(1.f + 1e-3f * (threadIdx.x + k), 1.f);
    for (int i = 0; i < iters; i++)
#pragma unroll
      for (int k = 0; k < kChains; k++) a[k] = __ffma2_rn(a[k], b, c);
    float s = 0;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += a[k].x + a[k].y;
    if (s == 12345.f) sink[0] = s;
  } else {  // FP16 HFMA2
    __half2 a[kChains];
    const __half2 b = __floats2half2_rn(0.999f, 0.998f), c = __floats2half2_rn(1e-3f, 2e-3f);
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = __floats2half2_rn(1.f, 0.5f + 1e-3f * k);
    for (int i = 0; i < iters; i++)
#pragma unroll
      for (int k = 0; k < kChains; k++) a[k] = __hfma2(a[k], b, c);
    float s = 0;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += __low2float(a[k]) + __high2float(a[k]);
    if (s == 12345.f) sink[0] = s;
  }
}

template <int KIND>
cudaError_t run_probe(int iters, int blocks, float* sink, double* ms_out) {
  cudaEvent_t e0, e1;
  cudaError_t e;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) return e;
  fma_probe<KIND><<<blocks, kThreads>>>(iters / 10, sink);  // warm-up
  cudaEventRecord(e0);
  fma_probe<KIND><<<blocks, kThreads>>>(iters, sink);
  cudaEventRecord(e1);
  if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_out = ms;
  return cudaGetLastError();
}

}  // namespace

// Throughput of one FMA kind on the current device: 0 FP64 DFMA, 1 FP32 FFMA,
// 2 paired FP32 FFMA2, 3 FP16 HFMA2.  *tflops = flops / time (an FMA counts two
// flops per lane; the paired forms have two lanes), *ms the kernel time.
// Returns 0 on success, else the CUDA error code.
extern "C" int dwf_probe_fma(int kind, int iters, double* tflops, double* ms) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  const int blocks = sms * 8;
  float* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(float)) != cudaSuccess) return 2;
  double t = 0.0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (kind) {
    case 0: e = run_probe<0>(iters, blocks, sink, &t); break;
    case 1: e = run_probe<1>(iters, blocks, sink, &t); break;
    case 2: e = run_probe<2>(iters, blocks, sink, &t); break;
    case 3: e = run_probe<3>(iters, blocks, sink, &t); break;
  }
  cudaFree(sink);
  if (e != cudaSuccess) return (int)e;
  const double lanes = (kind >= 2) ? 2.0 : 1.0;
  const double flops = 2.0 * lanes * kChains * (double)iters * blocks * kThreads;
  *ms = t;
  *tflops = flops / (t * 1e-3) / 1e12;
  return 0;
}
