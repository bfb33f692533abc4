// GPU check of the bounded shared-memory barrier wait that the persistent
// cell kernel uses in place of a CTA barrier per tile (mbar_wait in
// csrc/dg_kernels.cuh).
//
// Case 1: a barrier initialised for 2 arrivals gets 1, so its phase never
// completes (nothing else arrives).  Every thread's wait must give up after
// the bounded time (about 2 s), report it through bit 1 of a device flag, as
// the cell kernel does, and the kernel must return.  Case 2 (control): a
// barrier initialised for 1 arrival gets it; the wait must succeed at once.
// Afterwards the context must still run kernels (a third launch).
//
// Prints "flag <f1> <f2> <f3> elapsed_ms <t1> <t2>" and exits 0 when
// f1 == 2, f2 == 0, f3 == 7 and 1500 ms <= t1 <= 30000 ms, t2 < 1000 ms.
#include <cstdio>

#include "dg_kernels.cuh"

using namespace dghgks;

__global__ void k_wait(unsigned count, unsigned* flag) {
  __shared__ unsigned long long bar;
  if (threadIdx.x == 0) mbar_init(&bar, count);
  __syncthreads();
  if (threadIdx.x == 0) mbar_arrive(&bar);
  if (!mbar_wait(&bar, 0)) atomicOr(flag, 2u);
}

__global__ void k_after(unsigned* flag) {
  if (threadIdx.x == 0) *flag = 7u;
}

int main() {
  unsigned* d = nullptr;
  if (cudaMalloc(&d, 3 * sizeof(unsigned)) != cudaSuccess) return 2;
  cudaMemset(d, 0, 3 * sizeof(unsigned));
  cudaEvent_t e[4];
  for (auto& x : e) cudaEventCreate(&x);
  cudaEventRecord(e[0]);
  k_wait<<<1, 32>>>(2u, d);
  cudaEventRecord(e[1]);
  cudaEventRecord(e[2]);
  k_wait<<<1, 32>>>(1u, d + 1);
  cudaEventRecord(e[3]);
  k_after<<<1, 32>>>(d + 2);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    std::printf("CUDA error: %s\n", cudaGetErrorString(cudaGetLastError()));
    return 3;
  }
  unsigned h[3];
  cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  float t1 = 0, t2 = 0;
  cudaEventElapsedTime(&t1, e[0], e[1]);
  cudaEventElapsedTime(&t2, e[2], e[3]);
  std::printf("flag %u %u %u elapsed_ms %.1f %.3f\n", h[0], h[1], h[2], t1, t2);
  cudaFree(d);
  const bool ok = h[0] == 2u && h[1] == 0u && h[2] == 7u && t1 >= 1500.f && t1 <= 30000.f && t2 < 1000.f;
  return ok ? 0 : 1;
}
