// fft.cu -- batched in-register 3-D FFT passes (radix 2 and 3) of the block fields and of the q-space correlators (Sec. 3 Eq. LN.pLLp.FFT)
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <utility>

#include "device_common.cuh"

namespace bbc {

// --------------------------------------------------------------- twiddles
constexpr int kTw = 96;  // common multiple of every supported transform length
__constant__ double c_tw64[kTw][2];
__constant__ float c_tw32[kTw][2];
__constant__ float c_twdf[kTw][4];  // double-float (re.hi, re.lo, im.hi, im.lo)

cudaError_t upload_twiddles() {
  double h64[kTw][2];
  float h32[kTw][2];
  for (int k = 0; k < kTw; k++) {
    long double a = 2.0L * 3.14159265358979323846264338327950288L * k / kTw;
    h64[k][0] = (double)cosl(a);
    h64[k][1] = (double)-sinl(a);
    h32[k][0] = (float)cosl(a);
    h32[k][1] = (float)-sinl(a);
  }
  float hdf[kTw][4];
  for (int k = 0; k < kTw; k++) {
    long double a = 2.0L * 3.14159265358979323846264338327950288L * k / kTw;
    const long double c = cosl(a), sn = -sinl(a);
    hdf[k][0] = (float)c;
    hdf[k][1] = (float)(c - (long double)hdf[k][0]);
    hdf[k][2] = (float)sn;
    hdf[k][3] = (float)(sn - (long double)hdf[k][2]);
  }
  cudaError_t e = cudaMemcpyToSymbol(c_tw64, h64, sizeof(h64));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_twdf, hdf, sizeof(hdf));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_tw32, h32, sizeof(h32));
}

template <typename R>
__device__ __forceinline__ cpx<R> twiddle(int k);
template <>
__device__ __forceinline__ cpx<double> twiddle<double>(int k) { return cpx<double>(c_tw64[k][0], c_tw64[k][1]); }
template <>
__device__ __forceinline__ cpx<float> twiddle<float>(int k) { return cpx<float>(c_tw32[k][0], c_tw32[k][1]); }
template <>
__device__ __forceinline__ cpx<dfr> twiddle<dfr>(int k) {
  return cpx<dfr>(dfr(c_twdf[k][0], c_twdf[k][1]), dfr(c_twdf[k][2], c_twdf[k][3]));
}

__host__ __device__ constexpr int bitrev(int k, int n) {
  int r = 0;
  for (int b = 1; b < n; b <<= 1) { r = (r << 1) | (k & 1); k >>= 1; }
  return r;
}

// One radix-2 stage of span M (butterflies v[k+j], v[k+j+M/2], twiddle
// exp(-+2 pi i j/M)); stages recurse at compile time so every index is constant.
// FP32 / FP64 butterflies with a non-trivial twiddle fold the product into
// FMAs, hi = a + w b (four FMAs), and take lo = 2a - hi (two): six
// instructions instead of eight, with the same absolute error bound.
template <typename R, int N, int M, bool INV>
__device__ __forceinline__ void fft_stage(cpx<R> (&v)[N]) {
#pragma unroll
  for (int k = 0; k < N; k += M) {
#pragma unroll
    for (int j = 0; j < M / 2; j++) {
      const int ti = j * (kTw / M);
      const cpx<R> a = v[k + j], b = v[k + j + M / 2];
      if (ti == 0 || ti == kTw / 4) {
        const cpx<R> t = ti == 0 ? b : (INV ? cpx<R>(-b.im, b.re) : cpx<R>(b.im, -b.re));
        v[k + j + M / 2] = a - t;
        v[k + j] = a + t;
      } else {
        cpx<R> w = twiddle<R>(ti);
        if (INV) w.im = -w.im;
        if constexpr (std::is_floating_point<R>::value) {
          const cpx<R> hi(fma(-w.im, b.im, fma(w.re, b.re, a.re)), fma(w.im, b.re, fma(w.re, b.im, a.im)));
          v[k + j] = hi;
          v[k + j + M / 2] = cpx<R>(fma((R)2, a.re, -hi.re), fma((R)2, a.im, -hi.im));
        } else {
          const cpx<R> t = w * b;
          v[k + j + M / 2] = a - t;
          v[k + j] = a + t;
        }
      }
    }
  }
  if constexpr (M < N) fft_stage<R, N, 2 * M, INV>(v);
}

// Radix-2 decimation in time, input bit-reversed, output natural order.
// Forward: exp(-2 pi i jk/N); INV: exp(+2 pi i jk/N), unnormalised.
template <typename R, int N, bool INV>
__device__ __forceinline__ void fft_pow2(cpx<R> (&v)[N]) {
  if constexpr (N > 1) fft_stage<R, N, 2, INV>(v);
}

// N = 3 M (M a power of two): decimation in time into three size-M transforms
// of x[3 n2 + n1], then per k2 the twiddles exp(-+2 pi i n1 k2 / N) and a
// radix-3 butterfly giving X[k2 + M k1] (k1 = 0, 1, 2).  On entry u[n1][.]
// holds x[3 n2 + n1] in bit-reversed n2 order; on exit v holds X (natural).
template <typename R, int M, bool INV>
__device__ __forceinline__ void fft_radix3(cpx<R> (&u)[3][M], cpx<R> (&v)[3 * M]) {
  constexpr int N = 3 * M;
  fft_pow2<R, M, INV>(u[0]);
  fft_pow2<R, M, INV>(u[1]);
  fft_pow2<R, M, INV>(u[2]);
  // omega = exp(-+2 pi i / 3) = -1/2 -+ i sqrt(3)/2
  const R hs = (R)0.86602540378443864676;  // sqrt(3)/2
#pragma unroll
  for (int k2 = 0; k2 < M; k2++) {
    cpx<R> t1 = u[1][k2], t2 = u[2][k2];
    const int i1 = k2 * (kTw / N), i2 = 2 * k2 * (kTw / N);
    if (i1 != 0) {
      cpx<R> w = twiddle<R>(i1 % kTw);
      if (INV) w.im = -w.im;
      t1 = w * t1;
    }
    if (i2 != 0) {
      cpx<R> w = twiddle<R>(i2 % kTw);
      if (INV) w.im = -w.im;
      t2 = w * t2;
    }
    const cpx<R> t0 = u[0][k2];
    const cpx<R> s = t1 + t2, d = t1 - t2;
    // X[k2] = t0 + s; X[k2 + M] = t0 - s/2 -+ i hs d; X[k2 + 2M] = t0 - s/2 +- i hs d
    const cpx<R> m(t0.re - (R)0.5 * s.re, t0.im - (R)0.5 * s.im);
    const cpx<R> r = INV ? cpx<R>(-hs * d.im, hs * d.re) : cpx<R>(hs * d.im, -hs * d.re);  // -+ i hs d
    v[k2] = t0 + s;
    v[k2 + M] = m + r;
    v[k2 + 2 * M] = m - r;
  }
}

// --------------------------------------------------------------- FFT pass
// v[bitrev(k)] = p[k * step] with compile-time indices (keeps v in registers)
template <typename S, typename R, int N, int... Ks>
__device__ __forceinline__ void load_bitrev(cpx<R> (&v)[N], const cpx<S>* p, long long step,
                                            std::integer_sequence<int, Ks...>) {
  ((v[bitrev(Ks, N)] = cpx<R>(p[Ks * step])), ...);
}

// u[n1][bitrev(n2)] = p[(3 n2 + n1) * step], compile-time indices
template <typename S, typename R, int M, int... Ks>
__device__ __forceinline__ void load_radix3(cpx<R> (&u)[3][M], const cpx<S>* p, long long step,
                                            std::integer_sequence<int, Ks...>) {
  ((u[Ks % 3][bitrev(Ks / 3, M)] = cpx<R>(p[Ks * step])), ...);
}

// Length-N transform of one line (N = 2^k, or 3 * 2^k), natural order in and out.
template <typename S, typename R, int N, bool INV>
__device__ __forceinline__ void line_fft(const cpx<S>* p, long long step, cpx<R> (&v)[N]) {
  if constexpr ((N & (N - 1)) == 0) {
    load_bitrev<S, R, N>(v, p, step, std::make_integer_sequence<int, N>{});
    fft_pow2<R, N, INV>(v);
  } else {
    constexpr int M = N / 3;
    cpx<R> u[3][M];
    load_radix3<S, R, M>(u, p, step, std::make_integer_sequence<int, N>{});
    fft_radix3<R, M, INV>(u, v);
  }
}

__device__ __forceinline__ void line_base(int N, int axis, int line, int& base, int& stride) {
  const int a = line % N, b = line / N;
  if (axis == 0) { base = N * (a + N * b); stride = 1; }           // x varies, (y, z) = (a, b)
  else if (axis == 1) { base = a + N * N * b; stride = N; }        // y varies, (x, z) = (a, b)
  else { base = a + N * b; stride = N * N; }                       // z varies, (x, y) = (a, b)
}

// Mode SITE2FIELD (x axis): in[o][site][n_inner] -> out[o][inner][site] (the
// transpose to field-major storage rides on the first pass; lanes run over
// the contiguous inner index).
// Mode FIELD (any axis, in place on in = out): data[n_fields][V]; lanes run
// over the line index, which is contiguous for the y and z passes.
// Mode FIELD2OUT (z axis): in[ch][s][V] -> out[ch][r][16] times scale[ch]
// (the last inverse pass writes the output layout and normalises it).
// Mode SITE (any axis, in place): data[o][site][n_inner], lanes over inner.
// Mode SITE2OUT (z axis): in[site][n_ch*16] -> out[ch][r][16] times scale[ch].
// Mode FIELD_SUM: FIELD, and sum[o][q] = re + im of every value written (the
// sums the three-multiplication complex products of the contraction read).
enum { FFT_SITE2FIELD = 0, FFT_FIELD = 1, FFT_FIELD2OUT = 2, FFT_SITE = 3, FFT_SITE2OUT = 4, FFT_FIELD_SUM = 5 };

// S: storage of the input (and of the output in the in-place modes), R:
// compute type, O: storage of the output of the last inverse pass.
template <typename S, typename R, int N, bool INV, int MODE, typename O = S>
__global__ void __launch_bounds__(256)
k_fft(const cpx<S>* __restrict__ in, cpx<O>* __restrict__ out, long long n_outer, int n_inner, int axis,
      const double* __restrict__ scale, O* __restrict__ sum) {
  const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int lines = N * N;
  const long long V = (long long)N * N * N;
  int line, inner;
  long long o;
  if (MODE == FFT_SITE2FIELD || MODE == FFT_SITE || MODE == FFT_SITE2OUT) {
    if (gid >= n_outer * lines * n_inner) return;
    inner = (int)(gid % n_inner);
    const long long rest = gid / n_inner;
    line = (int)(rest % lines);
    o = rest / lines;
  } else if (MODE == FFT_FIELD || MODE == FFT_FIELD_SUM) {
    if (gid >= n_outer * lines) return;
    line = (int)(gid % lines);
    o = gid / lines;
    inner = 0;
  } else {  // FIELD2OUT: spin fastest so that each site's 16 spins are written together
    if (gid >= n_outer * lines * 16) return;
    inner = (int)(gid % 16);
    const long long rest = gid / 16;
    line = (int)(rest % lines);
    o = rest / lines;  // channel
  }
  int base, stride;
  line_base(N, axis, line, base, stride);
  cpx<R> v[N];
  if (MODE == FFT_SITE2FIELD || MODE == FFT_SITE || MODE == FFT_SITE2OUT) {
    line_fft<S, R, N, INV>(in + (o * V + base) * n_inner + inner, (long long)stride * n_inner, v);
  } else if (MODE == FFT_FIELD || MODE == FFT_FIELD_SUM) {
    line_fft<S, R, N, INV>(in + o * V + base, stride, v);
  } else {
    line_fft<S, R, N, INV>(in + (o * 16 + inner) * V + base, stride, v);
  }
  if (MODE == FFT_SITE2FIELD) {
    cpx<O>* p = out + (o * n_inner + inner) * V + base;
#pragma unroll
    for (int k = 0; k < N; k++) p[k * stride] = cpx<O>(v[k]);
  } else if (MODE == FFT_FIELD) {
    cpx<O>* p = out + o * V + base;
#pragma unroll
    for (int k = 0; k < N; k++) p[k * stride] = cpx<O>(v[k]);
  } else if (MODE == FFT_FIELD_SUM) {
    cpx<O>* p = out + o * V + base;
    O* ps = sum + o * V + base;
#pragma unroll
    for (int k = 0; k < N; k++) {
      const cpx<O> w(v[k]);
      p[k * stride] = w;
      ps[k * stride] = w.re + w.im;
    }
  } else if (MODE == FFT_SITE) {
    cpx<O>* p = out + (o * V + base) * n_inner + inner;
#pragma unroll
    for (int k = 0; k < N; k++) p[(long long)k * stride * n_inner] = cpx<O>(v[k]);
  } else if (MODE == FFT_SITE2OUT) {
    // inner = channel * 16 + spin; out[ch][r][16].  The scale (1/V, the
    // undone propagator rescaling, the mass factor) may lie far outside the
    // compute precision's range: it multiplies in the output precision.
    const O f = (O)scale[inner >> 4];
    cpx<O>* p = out + ((long long)(inner >> 4) * V + base) * 16 + (inner & 15);
#pragma unroll
    for (int k = 0; k < N; k++) p[(long long)k * stride * 16] = cpx<O>((O)v[k].re * f, (O)v[k].im * f);
  } else {
    const O f = (O)scale[o];
#pragma unroll
    for (int k = 0; k < N; k++) {
      cpx<O> w((O)v[k].re * f, (O)v[k].im * f);
      out[(o * V + base + (long long)k * stride) * 16 + inner] = w;
    }
  }
}

// Lines of N = 3 M points in FP64 or double-float (N = 48: a whole line in
// one thread's registers would spill) split over three threads: thread j of a
// line transforms the decimated sequence x[3 n2 + j] (M points, in registers),
// applies the twiddles exp(-+2 pi i j k2 / N) and leaves the result in shared
// memory; after a barrier, thread j combines k2 = j, j + 3, ... with the
// radix-3 butterfly into X[k2], X[k2 + M], X[k2 + 2M] and stores them.  The
// modes, index decomposition and output forms are those of k_fft
// (FIELD-type passes and the site-major first pass).
constexpr int kSplitLines = 64;  // lines per CTA of 3 x 64 threads
template <typename S, typename R, int M, bool INV, int MODE, typename O = S>
__global__ void __launch_bounds__(3 * kSplitLines)
k_fft3split(const cpx<S>* __restrict__ in, cpx<O>* __restrict__ out, long long n_outer, int n_inner, int axis,
            const double* __restrict__ scale, O* __restrict__ sum) {
  constexpr int N = 3 * M;
  // sh[line][j][k2 ^ (line & 7)]: a line's 3 M values are 3 M x 16 bytes
  // apart from the next line's, a multiple of the 128-byte bank period, so the
  // XOR spreads eight lanes' 16-byte accesses over the eight 16-byte slots of
  // a wavefront (without it the 32 lanes of a warp hit the same four banks)
  static_assert(M >= 8 && (M & (M - 1)) == 0, "swizzle within a power-of-two line of 8 or more");
  __shared__ cpx<R> sh[kSplitLines][3][M];
  auto at = [&](int l, int jj, int k2) -> cpx<R>& { return sh[l][jj][k2 ^ (l & 7)]; };
  const int ls = threadIdx.x % kSplitLines, j = threadIdx.x / kSplitLines;
  const long long gid = blockIdx.x * (long long)kSplitLines + ls;
  const int lines = N * N;
  const long long V = (long long)N * N * N;
  int line = 0, inner = 0;
  long long o = 0;
  bool live;
  if (MODE == FFT_SITE2FIELD) {
    live = gid < n_outer * lines * n_inner;
    inner = (int)(gid % n_inner);
    const long long rest = gid / n_inner;
    line = (int)(rest % lines);
    o = rest / lines;
  } else if (MODE == FFT_FIELD || MODE == FFT_FIELD_SUM) {
    live = gid < n_outer * lines;
    line = (int)(gid % lines);
    o = gid / lines;
  } else {  // FIELD2OUT
    live = gid < n_outer * lines * 16;
    inner = (int)(gid % 16);
    const long long rest = gid / 16;
    line = (int)(rest % lines);
    o = rest / lines;
  }
  int base = 0, stride = 0;
  line_base(N, axis, line, base, stride);
  if (live) {
    const cpx<S>* p;
    long long step;
    if (MODE == FFT_SITE2FIELD) { p = in + (o * V + base) * n_inner + inner; step = (long long)stride * n_inner; }
    else if (MODE == FFT_FIELD || MODE == FFT_FIELD_SUM) { p = in + o * V + base; step = stride; }
    else { p = in + (o * 16 + inner) * V + base; step = stride; }
    cpx<R> u[M];
    load_bitrev<S, R, M>(u, p + j * step, 3 * step, std::make_integer_sequence<int, M>{});
    fft_pow2<R, M, INV>(u);
#pragma unroll
    for (int k2 = 0; k2 < M; k2++) {
      const int ti = (j * k2 * (kTw / N)) % kTw;
      if (ti != 0) {
        cpx<R> w = twiddle<R>(ti);
        if (INV) w.im = -w.im;
        u[k2] = w * u[k2];
      }
      at(ls, j, k2) = u[k2];
    }
  }
  __syncthreads();
  const R hs = (R)0.86602540378443864676;  // sqrt(3)/2
  if (MODE == FFT_SITE2FIELD) {
    // The x lines of consecutive inner columns land in different output rows:
    // the radix-3 results go back into the line's own shared-memory slots
    // (column k2 of line ls is read and written by one thread only), and the
    // CTA then stores each line's N points as one contiguous run, consecutive
    // threads on consecutive points.
    if (live) {
      for (int k2 = j; k2 < M; k2 += 3) {
        const cpx<R> t0 = at(ls, 0, k2), t1 = at(ls, 1, k2), t2 = at(ls, 2, k2);
        const cpx<R> sm = t1 + t2, d = t1 - t2;
        const cpx<R> m(t0.re - (R)0.5 * sm.re, t0.im - (R)0.5 * sm.im);
        const cpx<R> r = INV ? cpx<R>(-hs * d.im, hs * d.re) : cpx<R>(hs * d.im, -hs * d.re);
        at(ls, 0, k2) = t0 + sm;  // X[k2 + c M] at (ls, c, k2)
        at(ls, 1, k2) = m + r;
        at(ls, 2, k2) = m - r;
      }
    }
    __syncthreads();
    // thread t stores point k = t mod N of lines t / N, t / N + kStep, ...
    // (the CTA's 3 x 64 threads = kStep whole lines per round); the line's
    // (outer, row, line) decomposition is carried from one of its lines to
    // the next by additions, not recomputed with 64-bit divisions per point
    constexpr int kStep = 3 * kSplitLines / N;
    static_assert(kStep * N == 3 * kSplitLines, "whole lines per round of stores");
    const long long total = n_outer * lines * n_inner;
    const int k = threadIdx.x % N, kj = k / M, kk = k % M;
    int l = threadIdx.x / N;
    long long gl = blockIdx.x * (long long)kSplitLines + l;
    int inn = (int)(gl % n_inner), ln = (int)((gl / n_inner) % lines);
    long long oo = gl / n_inner / lines;
    for (; l < kSplitLines && gl < total; l += kStep) {  // lines past the end come last
      int b = 0, sd = 0;
      line_base(N, axis, ln, b, sd);
      out[(oo * n_inner + inn) * V + b + (long long)k * sd] = cpx<O>(at(l, kj, kk));
      gl += kStep;
      inn += kStep;
      while (inn >= n_inner) {
        inn -= n_inner;
        if (++ln == lines) {
          ln = 0;
          ++oo;
        }
      }
    }
    return;
  }
  if (!live) return;
  for (int k2 = j; k2 < M; k2 += 3) {
    const cpx<R> t0 = at(ls, 0, k2), t1 = at(ls, 1, k2), t2 = at(ls, 2, k2);
    const cpx<R> sm = t1 + t2, d = t1 - t2;
    const cpx<R> m(t0.re - (R)0.5 * sm.re, t0.im - (R)0.5 * sm.im);
    const cpx<R> r = INV ? cpx<R>(-hs * d.im, hs * d.re) : cpx<R>(hs * d.im, -hs * d.re);
    const cpx<R> x[3] = {t0 + sm, m + r, m - r};
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const int k = k2 + c * M;
      if (MODE == FFT_FIELD) {
        out[o * V + base + (long long)k * stride] = cpx<O>(x[c]);
      } else if (MODE == FFT_FIELD_SUM) {
        const cpx<O> w(x[c]);
        out[o * V + base + (long long)k * stride] = w;
        sum[o * V + base + (long long)k * stride] = w.re + w.im;
      } else {  // FIELD2OUT, the scale in the output precision
        const O f = (O)scale[o];
        out[(o * V + base + (long long)k * stride) * 16 + inner] = cpx<O>((O)x[c].re * f, (O)x[c].im * f);
      }
    }
  }
}

// x and y passes of the site-major layout data[o][site][n_inner] fused in one
// kernel: a CTA takes one z plane of one outer index and TI consecutive inner
// columns, stages the N x N x TI plane in shared memory (compute precision),
// runs the x lines there, then the y lines, writing the result in place.
// One HBM round trip for two passes.
template <int N>
__host__ __device__ constexpr int xy_tile() {
  return N <= 16 ? 32 : (N == 24 ? 16 : (N == 32 ? 8 : 4));  // planes of <= 74 KB
}

template <typename S, typename R, int N, bool INV>
__global__ void __launch_bounds__(256) k_fft_xy_site(cpx<S>* __restrict__ data, int n_inner) {
  constexpr int TI = xy_tile<N>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* tile = reinterpret_cast<cpx<R>*>(smem_raw);  // [N * N][TI]
  const int i0 = blockIdx.x * TI, z = blockIdx.y;
  const long long o = blockIdx.z;
  const long long V = (long long)N * N * N;
  cpx<S>* plane = data + (o * V + (long long)z * N * N) * n_inner + i0;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < N * N * TI; idx += 256) {
    const int site = idx / TI, i = idx - site * TI;
    tile[idx] = i0 + i < n_inner ? cpx<R>(plane[(long long)site * n_inner + i]) : cpx<R>((R)0, (R)0);
  }
  __syncthreads();
  for (int li = tid; li < N * TI; li += 256) {  // x lines: (y, i)
    const int y = li / TI, i = li - y * TI;
    cpx<R> v[N];
    line_fft<R, R, N, INV>(tile + (y * N) * TI + i, TI, v);
#pragma unroll
    for (int k = 0; k < N; k++) tile[(y * N + k) * TI + i] = v[k];
  }
  __syncthreads();
  for (int li = tid; li < N * TI; li += 256) {  // y lines: (x, i), straight to global memory
    const int x = li / TI, i = li - x * TI;
    cpx<R> v[N];
    line_fft<R, R, N, INV>(tile + x * TI + i, N * TI, v);
    if (i0 + i < n_inner) {
#pragma unroll
      for (int k = 0; k < N; k++) plane[(long long)(x + N * k) * n_inner + i] = cpx<S>(v[k]);
    }
  }
}

template <typename S, typename R>
static cudaError_t fft_xy_site(void* data, int L, long long n_outer, int n_inner, bool inv, cudaStream_t st) {
#define BBC_XY_CASE(NN)                                                                                          \
  case NN: {                                                                                                     \
    constexpr int TI = xy_tile<NN>();                                                                            \
    const size_t sm = sizeof(cpx<R>) * NN * NN * TI;                                                             \
    dim3 grid((unsigned)((n_inner + TI - 1) / TI), NN, (unsigned)n_outer);                                      \
    static int granted_f[64] = {0}, granted_i[64] = {0};                                                         \
    cudaError_t e = inv ? ensure_smem(k_fft_xy_site<S, R, NN, true>, sm, granted_i)                              \
                        : ensure_smem(k_fft_xy_site<S, R, NN, false>, sm, granted_f);                            \
    if (e != cudaSuccess) return e;                                                                              \
    if (inv) k_fft_xy_site<S, R, NN, true><<<grid, 256, sm, st>>>((cpx<S>*)data, n_inner);                       \
    else k_fft_xy_site<S, R, NN, false><<<grid, 256, sm, st>>>((cpx<S>*)data, n_inner);                          \
    break;                                                                                                       \
  }
  switch (L) {
    BBC_XY_CASE(2)
    BBC_XY_CASE(4)
    BBC_XY_CASE(8)
    BBC_XY_CASE(16)
    BBC_XY_CASE(24)
    BBC_XY_CASE(32)
    BBC_XY_CASE(48)
    default: return cudaErrorInvalidValue;
  }
#undef BBC_XY_CASE
  return cudaGetLastError();
}

// ------------------------------------------------ persistent site-major FFT
// The forward x, y and z passes of the site-major layout data[o][site][n_inner]
// (L <= 32) in one persistent launch over a device work queue.  The inner
// columns are cut into row tiles g of TI columns of one outer index; tile g
// has N plane units (the x and y lines of one z plane, staged in shared
// memory as in k_fft_xy_site) and ZU line units (its z lines, 256 (line,
// column) pairs each).  A CTA takes tickets from a global counter; tickets
// run in steps of N + ZU, step s holding the plane units of tile s and the
// line units of tile s - lag, so a tile's z lines are read back from L2 soon
// after its planes were written (one HBM round trip for the three passes
// instead of two).  A CTA holds the ticket it runs and the next one, whose
// plane it copies into its second buffer (cp.async) meanwhile.  A line unit
// waits until the N plane units of its tile have signalled (q.words =
// [ticket counter, done[n_tiles]], zeroed before the launch).  The wait
// ends: it points at smaller tickets only, all taken by running CTAs, and
// the smallest unfinished ticket is always a running unit whose own
// dependencies are done.  It is bounded all the same: after spin_limit polls
// the CTA sets bit 0 of the sticky word *q.err (cleared only by the host),
// and no CTA takes a ticket while that bit is set.
__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ float2 ldcg_f2(const cpx<float>* p) { return __ldcg(reinterpret_cast<const float2*>(p)); }

template <int N, int... Ks>
__device__ __forceinline__ void load_bitrev_cg(cpx<float> (&v)[N], const cpx<float>* p, long long step,
                                               std::integer_sequence<int, Ks...>) {
  ((v[bitrev(Ks, N)] = [](float2 f) { return cpx<float>(f.x, f.y); }(ldcg_f2(p + Ks * step))), ...);
}
template <int M, int... Ks>
__device__ __forceinline__ void load_radix3_cg(cpx<float> (&u)[3][M], const cpx<float>* p, long long step,
                                               std::integer_sequence<int, Ks...>) {
  ((u[Ks % 3][bitrev(Ks / 3, M)] = [](float2 f) { return cpx<float>(f.x, f.y); }(ldcg_f2(p + Ks * step))), ...);
}
// line_fft with L2-only loads (the line was written by other CTAs of the launch)
template <int N, bool INV>
__device__ __forceinline__ void line_fft_cg(const cpx<float>* p, long long step, cpx<float> (&v)[N]) {
  if constexpr ((N & (N - 1)) == 0) {
    load_bitrev_cg<N>(v, p, step, std::make_integer_sequence<int, N>{});
    fft_pow2<float, N, INV>(v);
  } else {
    constexpr int M = N / 3;
    cpx<float> u[3][M];
    load_radix3_cg<M>(u, p, step, std::make_integer_sequence<int, N>{});
    fft_radix3<float, M, INV>(u, v);
  }
}

// Row-tile width of the queue-driven transform: two plane buffers of
// N * N * QT complex64 values fit three CTAs per SM.
template <int N>
__host__ __device__ constexpr int queue_tile() {
  return N <= 16 ? 16 : (N == 24 ? 8 : 4);
}
template <int N>
__host__ __device__ constexpr int queue_line_units() {
  return (N * N * queue_tile<N>() + 255) / 256;
}

template <int N, bool INV>
__global__ void __launch_bounds__(256)
k_fft_site_queue(cpx<float>* __restrict__ data, int n_inner, int tiles_per_outer, int n_tiles, int lag,
                 FftQueue q, int expect, long long spin_limit) {
  constexpr int TI = queue_tile<N>();
  constexpr int ZU = queue_line_units<N>();
  constexpr int U = N + ZU;
  constexpr int PLANE = N * N * TI;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<float>* bufs = reinterpret_cast<cpx<float>*>(smem_raw);  // [2][N * N][TI]
  __shared__ int s_next, s_ok;
  const long long V = (long long)N * N * N;
  const long long total = (long long)(n_tiles + lag) * U;
  const int tid = threadIdx.x;
  // plane unit of ticket t, or -1
  auto plane_tile = [&](long long t) -> int {
    if (t < 0 || t >= total) return -1;
    const int st = (int)(t / U), j = (int)(t % U);
    return (j < N && st < n_tiles) ? st : -1;
  };
  // asynchronous copy of a plane unit's N x N x TI values into buffer b
  // (columns past n_inner are zeroed with plain stores: the buffer is idle)
  auto fetch_plane = [&](long long t, cpx<float>* buf) {
    const int g = plane_tile(t);
    if (g < 0) return;
    const long long o = g / tiles_per_outer;
    const int i0 = (g % tiles_per_outer) * TI, z = (int)(t % U);
    const cpx<float>* plane = data + (o * V + (long long)z * N * N) * n_inner + i0;
    for (int idx = tid; idx < PLANE; idx += 256) {
      const int site = idx / TI, i = idx - site * TI;
      if (i0 + i < n_inner) cp_async8(buf + idx, plane + (long long)site * n_inner + i);
      else buf[idx] = cpx<float>(0.f, 0.f);
    }
  };
  // Each CTA holds two tickets: the unit it runs and the next one, whose
  // plane is on its way meanwhile.  Waits still point only at smaller
  // tickets, so the smallest unfinished ticket always belongs to a unit that
  // is running and whose own dependencies are complete.
  if (tid == 0) s_next = (*(volatile int*)q.err & 1) ? -1 : atomicAdd(q.words, 1);
  __syncthreads();
  long long cur = s_next;
  int b = 0;
  fetch_plane(cur, bufs);
  cp_async_commit();
  __syncthreads();
  while (cur >= 0 && cur < total) {
    if (tid == 0) s_next = (*(volatile int*)q.err & 1) ? -1 : atomicAdd(q.words, 1);
    __syncthreads();
    const long long nxt = s_next;
    fetch_plane(nxt, bufs + (b ^ 1) * PLANE);
    cp_async_commit();
    const int st = (int)(cur / U), j = (int)(cur % U);
    if (j < N) {  // plane unit: x and y lines of z plane j of tile st
      const int g = st;
      if (g < n_tiles) {
        const long long o = g / tiles_per_outer;
        const int i0 = (g % tiles_per_outer) * TI, z = j;
        cpx<float>* tile = bufs + b * PLANE;
        cpx<float>* plane = data + (o * V + (long long)z * N * N) * n_inner + i0;
        cp_async_wait_group<1>();  // this unit's plane has landed (the next one may still fly)
        __syncthreads();
        for (int li = tid; li < N * TI; li += 256) {  // x lines: (y, i)
          const int y = li / TI, i = li - y * TI;
          cpx<float> v[N];
          line_fft<float, float, N, INV>(tile + (y * N) * TI + i, TI, v);
#pragma unroll
          for (int k = 0; k < N; k++) tile[(y * N + k) * TI + i] = v[k];
        }
        __syncthreads();
        for (int li = tid; li < N * TI; li += 256) {  // y lines: (x, i), to global memory
          const int x = li / TI, i = li - x * TI;
          cpx<float> v[N];
          line_fft<float, float, N, INV>(tile + x * TI + i, N * TI, v);
          if (i0 + i < n_inner) {
#pragma unroll
            for (int k = 0; k < N; k++) plane[(long long)(x + N * k) * n_inner + i] = v[k];
          }
        }
        __syncthreads();  // the plane is written ...
        if (tid == 0) {   // ... and released to the line units of the tile
          __threadfence();
          atomicAdd(q.words + 1 + g, 1);
        }
      }
    } else {  // line unit j - N: z lines of tile st - lag
      const int g = st - lag;
      if (g >= 0) {
        if (tid == 0) {
          int ok = 1;
          long long polls = 0;
          while (ld_acquire_gpu(q.words + 1 + g) < expect) {
            if (++polls > spin_limit) {
              atomicOr(q.err, 1);
              ok = 0;
              break;
            }
            __nanosleep(256);
          }
          s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) break;
        const long long o = g / tiles_per_outer;
        const int i0 = (g % tiles_per_outer) * TI;
        const int pr = (j - N) * 256 + tid;  // (line, column) pair, column fastest
        const int line = pr / TI, i = pr - line * TI;
        if (line < N * N && i0 + i < n_inner) {
          cpx<float>* p = data + (o * V + line) * n_inner + i0 + i;
          cpx<float> v[N];
          line_fft_cg<N, INV>(p, (long long)N * N * n_inner, v);
#pragma unroll
          for (int k = 0; k < N; k++) p[(long long)k * N * N * n_inner] = v[k];
        }
      }
    }
    __syncthreads();  // s_next and the current buffer are reused
    cur = nxt;
    b ^= 1;
  }
  cp_async_wait_all();  // no copy outlives the CTA
}

template <int N>
static cudaError_t fft_site_queue_n(void* data, int n_outer, int n_inner, const FftQueue& q, int expect,
                                    long long spin_limit, cudaStream_t st) {
  constexpr int TI = queue_tile<N>();
  constexpr int U = N + queue_line_units<N>();
  const size_t sm = 2 * sizeof(cpx<float>) * N * N * TI;
  static int granted[64] = {0};
  static int resident[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  e = ensure_smem(k_fft_site_queue<N, false>, sm, granted);
  if (e != cudaSuccess) return e;
  if (resident[dev] == 0) {  // CTAs resident on the device (queried once per device)
    int n = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fft_site_queue<N, false>, 256, sm);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    resident[dev] = std::max(1, n) * std::max(1, sms);
  }
  const int tiles_per_outer = (n_inner + TI - 1) / TI;
  const int n_tiles = n_outer * tiles_per_outer;
  // lag: about 1.5 x the CTAs in flight, in steps, so that a tile's planes
  // are done before its line units are taken
  const int lag = std::max(1, (3 * resident[dev] / 2 + U - 1) / U);
  const long long units = (long long)(n_tiles + lag) * U;
  const int grid = (int)std::min<long long>(resident[dev], units);
  e = cudaMemsetAsync(q.words, 0, sizeof(int) * (1 + (size_t)n_tiles), st);  // ticket counter, done[]
  if (e != cudaSuccess) return e;
  k_fft_site_queue<N, false><<<grid, 256, sm, st>>>((cpx<float>*)data, n_inner, tiles_per_outer, n_tiles, lag, q,
                                                    expect < 0 ? N : expect, spin_limit);
  return cudaGetLastError();
}

int fft_queue_ints(int L, int n_outer, int n_inner) {
  const int ti = L <= 16 ? 16 : (L == 24 ? 8 : 4);  // queue_tile
  return 1 + n_outer * ((n_inner + ti - 1) / ti);
}

bool fft_queue_supported(int L) { return L == 2 || L == 4 || L == 8 || L == 16 || L == 24 || L == 32; }

cudaError_t launch_fft_forward_queue(void* blk, int L, int n_slots, int n_rows, const FftQueue& q, int expect,
                                     long long spin_limit, cudaStream_t st) {
  switch (L) {
    case 2: return fft_site_queue_n<2>(blk, n_slots, n_rows, q, expect, spin_limit, st);
    case 4: return fft_site_queue_n<4>(blk, n_slots, n_rows, q, expect, spin_limit, st);
    case 8: return fft_site_queue_n<8>(blk, n_slots, n_rows, q, expect, spin_limit, st);
    case 16: return fft_site_queue_n<16>(blk, n_slots, n_rows, q, expect, spin_limit, st);
    case 24: return fft_site_queue_n<24>(blk, n_slots, n_rows, q, expect, spin_limit, st);
    case 32: return fft_site_queue_n<32>(blk, n_slots, n_rows, q, expect, spin_limit, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename S, typename R, int MODE, typename O = S>
static cudaError_t fft_dispatch(const void* in, void* out, int L, long long n_outer, int n_inner, int axis, bool inv,
                                const double* scale, cudaStream_t st, O* sum = nullptr) {
  long long per = (MODE == FFT_SITE2FIELD || MODE == FFT_SITE || MODE == FFT_SITE2OUT) ? n_inner
                  : ((MODE == FFT_FIELD || MODE == FFT_FIELD_SUM) ? 1 : 16);
  long long total = n_outer * (long long)L * L * per;
  unsigned blocks = (unsigned)((total + 255) / 256);
  const cpx<S>* i = (const cpx<S>*)in;
  cpx<O>* o = (cpx<O>*)out;
  if constexpr (sizeof(R) == 8 && MODE != FFT_SITE && MODE != FFT_SITE2OUT) {
    // FP64 and double-float 48-point lines: three threads per line
    if (L == 48) {
      const unsigned b3 = (unsigned)((total + kSplitLines - 1) / kSplitLines);
      if (inv) k_fft3split<S, R, 16, true, MODE, O><<<b3, 3 * kSplitLines, 0, st>>>(i, o, n_outer, n_inner, axis, scale, sum);
      else k_fft3split<S, R, 16, false, MODE, O><<<b3, 3 * kSplitLines, 0, st>>>(i, o, n_outer, n_inner, axis, scale, sum);
      return cudaGetLastError();
    }
  }
#define BBC_FFT_CASE(NN)                                                                                      \
  case NN:                                                                                                    \
    if (inv) k_fft<S, R, NN, true, MODE, O><<<blocks, 256, 0, st>>>(i, o, n_outer, n_inner, axis, scale, sum); \
    else k_fft<S, R, NN, false, MODE, O><<<blocks, 256, 0, st>>>(i, o, n_outer, n_inner, axis, scale, sum);     \
    break;
  switch (L) {
    BBC_FFT_CASE(2)
    BBC_FFT_CASE(4)
    BBC_FFT_CASE(8)
    BBC_FFT_CASE(16)
    BBC_FFT_CASE(32)
    BBC_FFT_CASE(24)
    BBC_FFT_CASE(48)
    default: return cudaErrorInvalidValue;
  }
#undef BBC_FFT_CASE
  return cudaGetLastError();
}

cudaError_t launch_fft_forward(const void* blk_site, void* blk_field, int L, int n_slots, int n_rows, bool fp64,
                               cudaStream_t st, double* blk_sum) {
  cudaError_t e;
  if (fp64) {
    e = fft_dispatch<double, double, FFT_SITE2FIELD>(blk_site, blk_field, L, n_slots, n_rows, 0, false, nullptr, st);
    if (e != cudaSuccess) return e;
    e = fft_dispatch<double, double, FFT_FIELD>(blk_field, blk_field, L, (long long)n_slots * n_rows, 1, 1, false,
                                                nullptr, st);
    if (e != cudaSuccess) return e;
    // z pass; with blk_sum it also writes re + im of every Fourier-space value
    e = blk_sum ? fft_dispatch<double, double, FFT_FIELD_SUM>(blk_field, blk_field, L, (long long)n_slots * n_rows, 1,
                                                              2, false, nullptr, st, blk_sum)
                : fft_dispatch<double, double, FFT_FIELD>(blk_field, blk_field, L, (long long)n_slots * n_rows, 1, 2,
                                                          false, nullptr, st);
    if (e != cudaSuccess) return e;
  } else {
    e = fft_dispatch<float, float, FFT_SITE2FIELD>(blk_site, blk_field, L, n_slots, n_rows, 0, false, nullptr, st);
    if (e != cudaSuccess) return e;
    for (int axis = 1; axis < 3; axis++) {
      e = fft_dispatch<float, float, FFT_FIELD>(blk_field, blk_field, L, (long long)n_slots * n_rows, 1, axis, false,
                                                nullptr, st);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

cudaError_t launch_fft_forward_df(const void* blk_site, void* blk_field, int L, int n_slots, int n_rows,
                                  cudaStream_t st) {
  cudaError_t e =
      fft_dispatch<dfr, dfr, FFT_SITE2FIELD>(blk_site, blk_field, L, n_slots, n_rows, 0, false, nullptr, st);
  if (e != cudaSuccess) return e;
  for (int axis = 1; axis < 3; axis++) {
    e = fft_dispatch<dfr, dfr, FFT_FIELD>(blk_field, blk_field, L, (long long)n_slots * n_rows, 1, axis, false,
                                          nullptr, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_fft_forward_site(void* blk, int L, int n_slots, int n_rows, bool fp64, cudaStream_t st) {
  cudaError_t e;
  if (L <= 32) {  // x and y fused (one HBM round trip), then z
    e = fp64 ? fft_xy_site<double, double>(blk, L, n_slots, n_rows, false, st)
             : fft_xy_site<float, float>(blk, L, n_slots, n_rows, false, st);
    if (e != cudaSuccess) return e;
  } else {  // L = 48: the 48-point lines leave too few registers for a fused plane
    for (int axis = 0; axis < 2; axis++) {
      e = fp64 ? fft_dispatch<double, double, FFT_SITE>(blk, blk, L, n_slots, n_rows, axis, false, nullptr, st)
               : fft_dispatch<float, float, FFT_SITE>(blk, blk, L, n_slots, n_rows, axis, false, nullptr, st);
      if (e != cudaSuccess) return e;
    }
  }
  return fp64 ? fft_dispatch<double, double, FFT_SITE>(blk, blk, L, n_slots, n_rows, 2, false, nullptr, st)
              : fft_dispatch<float, float, FFT_SITE>(blk, blk, L, n_slots, n_rows, 2, false, nullptr, st);
}

cudaError_t launch_fft_inverse_site(void* ct, void* out, int L, int n_ch, const double* scale, bool fp64_compute,
                                    cudaStream_t st, bool ct_f32) {
  cudaError_t e;
  if (ct_f32) {  // complex64 q-space correlators, FP32 transform, complex128 output
    if (L <= 32) {
      e = fft_xy_site<float, float>(ct, L, 1, n_ch * 16, true, st);
    } else {
      e = cudaSuccess;
      for (int axis = 0; axis < 2 && e == cudaSuccess; axis++)
        e = fft_dispatch<float, float, FFT_SITE>(ct, ct, L, 1, n_ch * 16, axis, true, nullptr, st);
    }
    if (e != cudaSuccess) return e;
    return fft_dispatch<float, float, FFT_SITE2OUT, double>(ct, out, L, 1, n_ch * 16, 2, true, scale, st);
  }
  if (L <= 32) {
    e = fp64_compute ? fft_xy_site<double, double>(ct, L, 1, n_ch * 16, true, st)
                     : fft_xy_site<double, float>(ct, L, 1, n_ch * 16, true, st);
    if (e != cudaSuccess) return e;
  } else {
    for (int axis = 0; axis < 2; axis++) {
      e = fp64_compute ? fft_dispatch<double, double, FFT_SITE>(ct, ct, L, 1, n_ch * 16, axis, true, nullptr, st)
                       : fft_dispatch<double, float, FFT_SITE>(ct, ct, L, 1, n_ch * 16, axis, true, nullptr, st);
      if (e != cudaSuccess) return e;
    }
  }
  return fp64_compute ? fft_dispatch<double, double, FFT_SITE2OUT>(ct, out, L, 1, n_ch * 16, 2, true, scale, st)
                      : fft_dispatch<double, float, FFT_SITE2OUT>(ct, out, L, 1, n_ch * 16, 2, true, scale, st);
}

cudaError_t launch_fft_inverse_df(void* ct, void* out, int L, int n_ch, const double* scale, cudaStream_t st) {
  cudaError_t e;
  for (int axis = 0; axis < 2; axis++) {
    e = fft_dispatch<dfr, dfr, FFT_FIELD>(ct, ct, L, (long long)n_ch * 16, 1, axis, true, nullptr, st);
    if (e != cudaSuccess) return e;
  }
  return fft_dispatch<dfr, dfr, FFT_FIELD2OUT, double>(ct, out, L, n_ch, 16, 2, true, scale, st);
}

cudaError_t launch_fft_inverse(void* ct, void* out, int L, int n_ch, const double* scale, bool fp64_compute,
                               cudaStream_t st) {
  cudaError_t e;
  for (int axis = 0; axis < 2; axis++) {
    e = fp64_compute ? fft_dispatch<double, double, FFT_FIELD>(ct, ct, L, (long long)n_ch * 16, 1, axis, true, nullptr, st)
                     : fft_dispatch<double, float, FFT_FIELD>(ct, ct, L, (long long)n_ch * 16, 1, axis, true, nullptr, st);
    if (e != cudaSuccess) return e;
  }
  return fp64_compute ? fft_dispatch<double, double, FFT_FIELD2OUT>(ct, out, L, n_ch, 16, 2, true, scale, st)
                      : fft_dispatch<double, float, FFT_FIELD2OUT>(ct, out, L, n_ch, 16, 2, true, scale, st);
}

}  // namespace bbc
