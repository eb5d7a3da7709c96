// peaks.cu -- arithmetic peaks of this GPU for the roofline of the transform
// kernels: the FP64 and FP32 fused-multiply-add rates of the CUDA cores
// (the FP64 path's butterflies and products are DFMA/DADD/DMUL work on those
// cores; no tensor-core format takes part).  Every thread runs independent
// FMA chains long enough that the issue rate, not latency, sets the time.
#include <cuda_runtime.h>

#include <string>

#include "../../include/lagmean.h"

namespace lm {
void set_handleless_error(const std::string& msg);
}

namespace {

constexpr int CHAINS = 8;   // independent FMA chains per thread
constexpr int UNROLL = 16;  // FMAs per chain per loop trip

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T* __restrict__ out, int trips, T b, T c) {
  T a[CHAINS];
#pragma unroll
  for (int i = 0; i < CHAINS; ++i) a[i] = (T)(threadIdx.x + i) * (T)1e-3;
  for (int t = 0; t < trips; ++t) {
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
#pragma unroll
      for (int i = 0; i < CHAINS; ++i) a[i] = fma(a[i], b, c);
    }
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < CHAINS; ++i) s += a[i];
  // one store per thread keeps the chains live; the value is never read
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int measure(int trips, double* tflops, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    lm::set_handleless_error(std::string("sw_fma_peak: ") + cudaGetErrorString(e));
    return SW_ECUDA;
  }
  const int blocks = sms * 8, threads = 256;
  T* buf = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float best = 0.f;
  if ((e = cudaMalloc(&buf, (size_t)blocks * threads * sizeof(T))) == cudaSuccess &&
      (e = cudaEventCreate(&e0)) == cudaSuccess && (e = cudaEventCreate(&e1)) == cudaSuccess) {
    // b just below 1 and c small keep the chains finite for any trip count
    const T b = (T)0.999999, c = (T)1e-7;
    k_fma_peak<T><<<blocks, threads, 0, s>>>(buf, trips, b, c);  // warm-up
    for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) {
      cudaEventRecord(e0, s);
      k_fma_peak<T><<<blocks, threads, 0, s>>>(buf, trips, b, c);
      cudaEventRecord(e1, s);
      if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
      float ms = 0.f;
      if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
      if (rep == 0 || ms < best) best = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (buf) cudaFree(buf);
  if (e != cudaSuccess) {
    lm::set_handleless_error(std::string("sw_fma_peak: ") + cudaGetErrorString(e));
    return SW_ECUDA;
  }
  const double flops = 2.0 * (double)blocks * threads * (double)trips * UNROLL * CHAINS;
  *tflops = flops / (best * 1e-3) / 1e12;
  return SW_OK;
}

}  // namespace

extern "C" int sw_fma_peak(int precision, int trips, double* tflops, void* stream) {
  if (!tflops || trips < 1 || trips > (1 << 20) || (precision != SW_PREC_FP64 && precision != SW_PREC_FP32)) {
    lm::set_handleless_error("sw_fma_peak: precision must be SW_PREC_FP64 or SW_PREC_FP32, trips in 1..2^20, "
                             "tflops non-NULL");
    return SW_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  return precision == SW_PREC_FP64 ? measure<double>(trips, tflops, s) : measure<float>(trips, tflops, s);
}
