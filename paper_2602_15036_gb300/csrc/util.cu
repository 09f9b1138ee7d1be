// Small device utilities that belong to no stage of the imaging path.
#include "litho_internal.h"

namespace litho {

namespace {

// One thread spinning on the SM clock for a fixed number of cycles: it always
// ends (no flag or peer is waited on).
__global__ void k_delay(long long cycles) {
  const long long t0 = clock64();
  while (clock64() - t0 < cycles) __nanosleep(1000);
}

}  // namespace

cudaError_t launch_delay(cudaStream_t st, double ms) {
  int dev = 0, khz = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  if (e != cudaSuccess) return e;
  k_delay<<<1, 1, 0, st>>>((long long)(ms * double(khz > 0 ? khz : 2000000)));
  return cudaGetLastError();
}

}  // namespace litho
