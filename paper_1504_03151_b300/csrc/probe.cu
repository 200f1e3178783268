// probe.cu - a measurement helper, not part of the tracer: the read
// bandwidth of the L2 cache, which is where the traversal kernels' working
// set (nodes and primitive records of scenes up to a few million
// triangles) lives.  The roofline of those kernels is taken against it.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "rtb_internal.cuh"

namespace rtb {

// Every thread streams float4s through L2 (ld.global.cg: not kept in L1),
// `reps` times over the buffer; four independent loads are in flight per
// thread and iteration.  One sum per block keeps the loads alive.
__global__ void __launch_bounds__(512) k_l2_read(const float4* __restrict__ buf, size_t n4, int reps,
                                                 float* __restrict__ sink) {
  float acc = 0.f;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t first = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int r = 0; r < reps; ++r) {
    size_t i = first;
    for (; i + 3 * stride < n4; i += 4 * stride) {
      float4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride);
      float4 c = __ldcg(buf + i + 2 * stride), d = __ldcg(buf + i + 3 * stride);
      acc += (a.x + b.y) + (c.z + d.w);
    }
    for (; i < n4; i += stride) acc += __ldcg(buf + i).x;
  }
  __shared__ float s[512];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) sink[blockIdx.x] = s[0];
}

}  // namespace rtb

using namespace rtb;

extern "C" rt_status rt_probe_l2_read(size_t bytes, int reps, float* gbs, void* stream) {
  if (!gbs || bytes < 16 * 4096 || bytes > ((size_t)1 << 31) || reps < 1 || reps > 10000)
    return set_error(RT_ERR_INVALID_ARG, "rt_probe_l2_read: bytes in [64 KB, 2 GB], reps in [1, 10000]");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_error(e, "rt_probe_l2_read");
  const int blocks = sms * 4;   // 4 blocks of 512 threads fill an SM's 2048 thread slots
  const size_t n4 = bytes / 16;
  float4* buf = nullptr;
  float* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc(&buf, n4 * 16);
  if (e == cudaSuccess) e = cudaMalloc(&sink, blocks * sizeof(float));
  if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, n4 * 16, st);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.f;
  if (e == cudaSuccess) {
    k_l2_read<<<blocks, 512, 0, st>>>(buf, n4, 1, sink);   // brings the buffer into L2
    cudaEventRecord(e0, st);
    k_l2_read<<<blocks, 512, 0, st>>>(buf, n4, reps, sink);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (buf) cudaFree(buf);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) return cuda_error(e, "rt_probe_l2_read");
  *gbs = (float)((double)n4 * 16.0 * reps / (ms * 1e-3) / 1e9);
  return RT_OK;
}
