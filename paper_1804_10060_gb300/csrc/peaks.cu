// FMA throughput of the device's FP64 and FP32 pipes (instrumentation, not
// part of the method).  GB300's FP64 rate decides how this library multiplies
// matrices: a plain FP64 3x3 block SpMV needs 9 FP64 FMAs per 76 bytes, and
// when the FP64 pipe cannot issue them at HBM speed the products move to
// double-float arithmetic on the FP32 pipe (see sparse.cuh).  Every thread
// runs 8 independent FMA chains so that the pipe, not the chain latency, is
// the limit; the chains' sum is stored so the compiler keeps them.
#include "common.cuh"

namespace tam {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_chain_kernel(T a, T b, int iters, T* __restrict__ out) {
  T v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = fma(v[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += v[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
double fma_tflops(cudaStream_t s) {
  const int blocks = sm_count() * 8, threads = 256, iters = 4096;
  DBuf<T> out((size_t)blocks * threads, s);
  cudaEvent_t e0, e1;
  TAM_CUDA(cudaEventCreate(&e0));
  TAM_CUDA(cudaEventCreate(&e1));
  // a = 1 - 2^-20, b = 2^-20: the chains stay bounded (no overflow or denormals)
  const T a = (T)(1.0 - 1.0 / 1048576.0), b = (T)(1.0 / 1048576.0);
  fma_chain_kernel<T><<<blocks, threads, 0, s>>>(a, b, iters, out.p);  // warm-up
  TAM_LAUNCH_CHECK();
  float best = 1e30f;
  for (int rep = 0; rep < 5; ++rep) {
    TAM_CUDA(cudaEventRecord(e0, s));
    fma_chain_kernel<T><<<blocks, threads, 0, s>>>(a, b, iters, out.p);
    TAM_LAUNCH_CHECK();
    TAM_CUDA(cudaEventRecord(e1, s));
    TAM_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    TAM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    best = ms < best ? ms : best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
  return flops / (best * 1e-3) / 1e12;
}

}  // namespace
}  // namespace tam

extern "C" int tam_fma_throughput(double* fp64_tflops_host, double* fp32_tflops_host, void* stream) {
  try {
    tam::set_last_error("");
    TAM_CHECK(fp64_tflops_host || fp32_tflops_host, TAM_ERR_INVALID_ARG, "tam_fma_throughput: NULL arguments");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (fp64_tflops_host) *fp64_tflops_host = tam::fma_tflops<double>(s);
    if (fp32_tflops_host) *fp32_tflops_host = tam::fma_tflops<float>(s);
    return TAM_OK;
  } catch (const tam::Error& e) {
    tam::set_last_error(e.what());
    return e.code;
  }
}
