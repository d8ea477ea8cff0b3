// FMA-pipe probe for the benchmark (built as libfmaprobe.so, not part of the library's ABI): the
// achievable FP32 and FP64 FMA rates of this GPU, measured with independent dependency chains per
// thread (enough in flight to hide the pipe latency) over a grid that fills every SM.  The
// benchmark sets it beside the derived peaks (SMs x lanes x 2 x clock) of the ALU-bound kernels.
#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;

template <typename T>
__global__ void k_fma_chains(T a, T b, T* out) {
  T v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  if (s == (T)-1.2345) out[0] = s;        // never true for the inputs used: keeps the chains alive
}

}  // namespace

// fp64 != 0: FP64 FMA, else FP32.  *tflops: 2 flop per FMA over the fastest of three timed
// launches (after one warm-up).  Returns 0, or a CUDA error code (no device, allocation failure).
extern "C" int fma_probe_tflops(int fp64, double* tflops) {
  if (!tflops) return (int)cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  void* out = nullptr;
  if (err == cudaSuccess) err = cudaMalloc(&out, 16);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return (int)err;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int threads = 256, blocks = sms * 8;
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0);
    if (fp64)
      k_fma_chains<double><<<blocks, threads>>>(0.9999999, 1e-7, (double*)out);
    else
      k_fma_chains<float><<<blocks, threads>>>(0.9999f, 1e-4f, (float*)out);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  err = cudaGetLastError();
  if (err != cudaSuccess) return (int)err;
  const double flop = 2.0 * kChains * (double)kIters * threads * blocks;
  *tflops = flop / (best / 1e3) / 1e12;
  return 0;
}
