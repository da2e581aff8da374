// Measurement support: the FP64 FMA issue rate of the device, the roofline of the FP64 run
// kernel (its work is one FP64 FMA per stored entry). The paper has no counterpart.
//
// One CTA per SM, 16 warps, every lane runs four independent FMA chains (so a warp never
// waits on its own previous FMA); the device time of the launch gives the FMA rate, and
// clock64 around each warp's loop gives the SM cycles one warp-wide FMA takes per SM
// sub-partition (four sub-partitions per SM share the warps evenly).
#include <cuda_runtime.h>

#include <cstdio>
#include <string>
#include <vector>

#include "../../include/cbspmv.h"
#include "cb_noalloc.h"

namespace {

constexpr int kWarps = 16;
constexpr int kChains = 4;

__global__ void __launch_bounds__(32 * kWarps, 1)
    fp64_fma_probe_kernel(double* out, long long* cycles, int iters, double a, double b) {
  double c[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) c[k] = 1e-3 * threadIdx.x + k;
  __syncwarp();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) c[k] = fma(c[k], a, b);
  }
  const long long t1 = clock64();
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += c[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
  if ((threadIdx.x & 31) == 0) cycles[blockIdx.x * kWarps + threadIdx.x / 32] = t1 - t0;
}

}  // namespace

extern "C" cbspmv_status_t cbspmv_measure_fp64_fma(int device, void* stream, double* gflops,
                                                   double* cycles_per_warp_fma) {
  if (!gflops || !cycles_per_warp_fma) {
    cb::set_last_error("NULL output");
    return CBSPMV_ERR_INVALID;
  }
  int prev = -1;
  cudaError_t e = cudaGetDevice(&prev);
  if (e == cudaSuccess && prev != device) e = cudaSetDevice(device);
  int sms = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  double* out = nullptr;
  long long* cyc = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const cudaStream_t s = (cudaStream_t)stream;
  const int iters = 8192;
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaMalloc((void**)&out, sizeof(double) * sms * 32 * kWarps);
  if (e == cudaSuccess) e = cudaMalloc((void**)&cyc, sizeof(long long) * sms * kWarps);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    fp64_fma_probe_kernel<<<sms, 32 * kWarps, 0, s>>>(out, cyc, iters / 8, 1.0000001, 1e-9);   // warm-up
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) {
    fp64_fma_probe_kernel<<<sms, 32 * kWarps, 0, s>>>(out, cyc, iters, 1.0000001, 1e-9);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  std::vector<long long> h((size_t)sms * kWarps);
  if (e == cudaSuccess) e = cudaMemcpy(h.data(), cyc, h.size() * sizeof(long long), cudaMemcpyDeviceToHost);
  if (out) cudaFree(out);
  if (cyc) cudaFree(cyc);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  if (e != cudaSuccess) {
    cb::set_last_error(std::string("cbspmv_measure_fp64_fma: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? CBSPMV_ERR_OOM : CBSPMV_ERR_CUDA;
  }
  const double fmas = (double)sms * 32 * kWarps * (double)iters * kChains;
  *gflops = 2.0 * fmas / (ms * 1e-3) / 1e9;
  double mean = 0.0;
  for (long long v : h) mean += (double)v;
  mean /= (double)h.size();
  // each sub-partition runs kWarps / 4 warps; a warp issues iters * kChains FMAs
  *cycles_per_warp_fma = mean / ((double)iters * kChains * (kWarps / 4));
  cb::set_last_error("");
  return CBSPMV_OK;
}
