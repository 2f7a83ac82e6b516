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

// ---------------------------------------------------------- double-float
// A real as an unevaluated sum hi + lo of two FP32 values (48-bit
// significand), for FP64-accurate arithmetic on the FP32 pipes.  Built from
// error-free transformations: Knuth's TwoSum (the exact rounding error of a
// sum) and the FMA-based TwoProduct (the exact error of a product, Ogita,
// Rump and Oishi, SIAM J. Sci. Comput. 26 (2005)).  The _rn intrinsics keep
// the compiler from contracting the products and sums these rely on.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Accumulator s + e, normalised only now and then (|e| stays far below |s|
// for the short sums it is used for).
struct df64acc {
  float s, e;
};

// acc += x * y (x, y double-float): TwoProduct of the high parts, the cross
// terms into the error word, TwoSum of the product into the accumulator.
__device__ __forceinline__ void df_mac(df64acc& acc, float xh, float xl, float yh, float yl) {
  const float p = __fmul_rn(xh, yh);
  float e = __fmaf_rn(xh, yh, -p);
  e = __fmaf_rn(xh, yl, e);
  e = __fmaf_rn(xl, yh, e);
  float s, t;
  two_sum(acc.s, p, s, t);
  acc.s = s;
  acc.e = __fadd_rn(acc.e, __fadd_rn(t, e));
}

__device__ __forceinline__ void df_renorm(df64acc& acc) {
  float s, e;
  two_sum(acc.s, acc.e, s, e);
  acc.s = s;
  acc.e = e;
}

// Double-float real with arithmetic operators, for kernels templated on the
// real type (block build, FFT).  The operators keep the pair unnormalised: a
// sum is the TwoSum of the high words with the low words added into its
// error word, a product the TwoProduct of the high words with the cross
// terms added into its error word, and neither renormalises (hi, lo) so that
// |lo| <= ulp(hi) / 2.  The low word then holds the accumulated rounding
// errors of a few operations at most a few ulps of the high word; every
// later TwoSum and TwoProduct on the high words is still exact, so the error
// of a sum or product stays about 2^-44 (|a| + |b|) or 2^-44 |a b|: an
// absolute error at the scale of the operands, which is what the correlator
// tolerance measures.  Consumers read hi + lo (the pair products, the
// conversion to double), never hi alone.
struct dfr {
  float hi, lo;
  __host__ __device__ dfr() {}
  __host__ __device__ constexpr dfr(float h, float l) : hi(h), lo(l) {}
  // split of a double (constant-folded for literals; FP64 instructions otherwise)
  __host__ __device__ constexpr explicit dfr(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ constexpr dfr(int x) : hi((float)x), lo(0.f) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ dfr operator-(dfr a) { return dfr(-a.hi, -a.lo); }
__device__ __forceinline__ dfr operator+(dfr a, dfr b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return dfr(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfr operator-(dfr a, dfr b) { return a + (-b); }
__device__ __forceinline__ dfr operator*(dfr a, dfr b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return dfr(p, e);
}
__device__ __forceinline__ dfr& operator+=(dfr& a, dfr b) { return a = a + b; }
// Multiply-add overloads in this namespace (the double-float one would
// otherwise hide the floating-point ones from unqualified calls).
__device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
// a * b + c: the product's two words folded into the sum (TwoSum of the high
// words), unnormalised like the operators
__device__ __forceinline__ dfr fma(dfr a, dfr b, dfr c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s, t;
  two_sum(c.hi, p, s, t);
  return dfr(s, __fadd_rn(t, __fadd_rn(e, c.lo)));
}

// Asynchronous global -> shared copies (cp.async; the data bypasses the
// registers, so a thread issues all its copies before waiting on any).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N of this thread's committed groups are still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

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
