// sdpd_peak.cu -- fused multiply-add throughput of the device, measured: the
// denominator of the arithmetic rooflines of the pair passes (float32 in the
// mixed path, float64 in the float64 path and the reverse passes).
#include "sdpd_internal.cuh"

namespace {

constexpr int kChains = 8;  // independent FMA chains per thread (covers the pipe latency)

__device__ double g_fma_sink;  // written only if the chains' sum were -1 (never)

// x <- x * a + b with |a| < 1: every chain converges to b / (1 - a), so no
// value overflows or turns subnormal however long the loop runs
template <class T>
__global__ void __launch_bounds__(256) k_fma(int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (T)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll 16
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
    }
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == (T)-1.0) g_fma_sink = (double)s;  // never true: the chains stay positive
}

template <class T>
int measure(int iters, cudaStream_t st, double* flops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SDPD_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SDPD_ERR_CUDA;
  const unsigned blocks = (unsigned)sms * 8u;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return SDPD_ERR_CUDA;
  k_fma<T><<<blocks, 256, 0, st>>>(iters / 4 + 1, (T)0.999, (T)0.001);  // warm-up
  cudaEventRecord(e0, st);
  k_fma<T><<<blocks, 256, 0, st>>>(iters, (T)0.999, (T)0.001);
  cudaEventRecord(e1, st);
  int e = cudaEventSynchronize(e1) == cudaSuccess ? SDPD_OK : SDPD_ERR_CUDA;
  float ms = 0.0f;
  if (!e && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) e = SDPD_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!e) *flops = 2.0 * kChains * 16.0 * iters * (double)blocks * 256.0 / (ms * 1e-3);
  return e ? e : (cudaGetLastError() == cudaSuccess ? SDPD_OK : SDPD_ERR_CUDA);
}

}  // namespace

extern "C" int sdpd_fma_peak(int precision, void* stream, double* flops) {
  if (!flops || (precision != SDPD_FP64 && precision != SDPD_MIXED)) return SDPD_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  return precision == SDPD_MIXED ? measure<float>(8192, st, flops) : measure<double>(512, st, flops);
}
