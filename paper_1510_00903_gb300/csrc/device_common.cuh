// device_common.cuh -- complex type and multiply-add shared by the sm_103a
// kernels of libbbc.
#pragma once

#include "kernels.cuh"

namespace bbc {

template <typename R>
struct __align__(2 * sizeof(R)) cpx {
  R re, im;
  __host__ __device__ cpx() {}
  __host__ __device__ cpx(R r, R i) : re(r), im(i) {}
  template <typename Q>
  __host__ __device__ explicit cpx(const cpx<Q>& o) : re((R)o.re), im((R)o.im) {}
};
template <typename R>
__device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) { return cpx<R>(a.re + b.re, a.im + b.im); }
template <typename R>
__device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) { return cpx<R>(a.re - b.re, a.im - b.im); }
template <typename R>
__device__ __forceinline__ cpx<R> operator*(cpx<R> a, cpx<R> b) {
  return cpx<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// acc += a * b (four FMAs)
template <typename R>
__device__ __forceinline__ void cmac(cpx<R>& acc, cpx<R> a, cpx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}

// Raise a kernel's dynamic shared-memory limit only when a launch needs more
// than was granted before (per device), so that launches captured into a
// CUDA graph after a first eager run issue no attribute call.
template <typename K>
inline cudaError_t ensure_smem(K kernel, size_t bytes, int* granted /* [64] per device */) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if ((int)bytes <= granted[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) granted[dev] = (int)bytes;
  return e;
}

}  // namespace bbc
