// kernels.cu -- sm_103a kernels of the effective block algorithm
// (Nemura, arXiv:1510.00903).
//
// Per time slice:
//   ingest      exact power-of-two rescaling of each propagator (keeps every
//               six-quark product inside the FP32 range; undone in FP64)
//   block_build per site: two diquarks, up to two sink-tensor families in
//               shared memory, then every aggregated block output as a sparse
//               integer-weighted sum (Sec. 3 blocks, Appendix A aggregation)
//   fft_pass    batched in-register 1-D DFTs along x, y, z (Sec. 3 Eq.
//               LN.pLLp.FFT), batch index contiguous in memory
//   contract    per q: every aligned block-pair product A(q) B(-q) summed
//               over its open colour/spin indices, then the signed FP64 sum
//               over Wick diagrams into each channel and spin
//   normalise   1/V, the rescaling, exp((m_B1 + m_B2) d) (Sec. 2 Eq. 2)
#include "kernels.cuh"

#include <algorithm>
#include <cmath>
#include <utility>

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

// --------------------------------------------------------------- twiddles
constexpr int kTw = 96;  // common multiple of every supported transform length
__constant__ double c_tw64[kTw][2];
__constant__ float c_tw32[kTw][2];

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
  cudaError_t e = cudaMemcpyToSymbol(c_tw64, h64, sizeof(h64));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_tw32, h32, sizeof(h32));
}

template <typename R>
__device__ __forceinline__ cpx<R> twiddle(int k);
template <>
__device__ __forceinline__ cpx<double> twiddle<double>(int k) { return cpx<double>(c_tw64[k][0], c_tw64[k][1]); }
template <>
__device__ __forceinline__ cpx<float> twiddle<float>(int k) { return cpx<float>(c_tw32[k][0], c_tw32[k][1]); }

__host__ __device__ constexpr int bitrev(int k, int n) {
  int r = 0;
  for (int b = 1; b < n; b <<= 1) { r = (r << 1) | (k & 1); k >>= 1; }
  return r;
}

// One radix-2 stage of span M (butterflies v[k+j], v[k+j+M/2], twiddle
// exp(-+2 pi i j/M)); stages recurse at compile time so every index is constant.
template <typename R, int N, int M, bool INV>
__device__ __forceinline__ void fft_stage(cpx<R> (&v)[N]) {
#pragma unroll
  for (int k = 0; k < N; k += M) {
#pragma unroll
    for (int j = 0; j < M / 2; j++) {
      const int ti = j * (kTw / M);
      cpx<R> b = v[k + j + M / 2], t;
      if (ti == 0) {
        t = b;
      } else if (ti == kTw / 4) {
        t = INV ? cpx<R>(-b.im, b.re) : cpx<R>(b.im, -b.re);
      } else {
        cpx<R> w = twiddle<R>(ti);
        if (INV) w.im = -w.im;
        t = w * b;
      }
      v[k + j + M / 2] = v[k + j] - t;
      v[k + j] = v[k + j] + t;
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

// ------------------------------------------------------------------ ingest
__global__ void k_absmax(const void* __restrict__ src, int dtype, long long n_real,
                         unsigned long long* amax) {
  double m = 0.0;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_real; i += stride) {
    double x = dtype == 0 ? ((const double*)src)[i] : (double)((const float*)src)[i];
    m = fmax(m, fabs(x));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(amax, (unsigned long long)__double_as_longlong(m));
}

template <typename R>
__global__ void k_convert(const void* __restrict__ src, int dtype, long long n_real,
                          const unsigned long long* __restrict__ amax, int* kexp, R* __restrict__ dst) {
  double m = __longlong_as_double((long long)*amax);
  int k = (m > 0.0 && m <= 1.7976931348623157e308) ? ilogb(m) + 1 : 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) *kexp = k;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_real; i += stride) {
    double x = dtype == 0 ? ((const double*)src)[i] : (double)((const float*)src)[i];
    dst[i] = (R)ldexp(x, -k);
  }
}

cudaError_t launch_absmax(const void* src, int dtype, long long n_complex, unsigned long long* amax,
                          cudaStream_t st) {
  long long n = 2 * n_complex;
  int blocks = (int)std::min<long long>((n + 255) / 256, 152 * 8);
  k_absmax<<<blocks, 256, 0, st>>>(src, dtype, n, amax);
  return cudaGetLastError();
}

cudaError_t launch_convert(const void* src, int dtype, long long n_complex, const unsigned long long* amax,
                           int* kexp, void* dst, bool fp64, cudaStream_t st) {
  long long n = 2 * n_complex;
  int blocks = (int)std::min<long long>((n + 255) / 256, 152 * 8);
  if (fp64) k_convert<double><<<blocks, 256, 0, st>>>(src, dtype, n, amax, kexp, (double*)dst);
  else k_convert<float><<<blocks, 256, 0, st>>>(src, dtype, n, amax, kexp, (float*)dst);
  return cudaGetLastError();
}

// ------------------------------------------------------------ block build
// C gamma5 (Dirac representation): (0,1)=+1, (1,0)=-1, (2,3)=+1, (3,2)=-1.
__constant__ int c_cg5[4][3] = {{0, 1, 1}, {1, 0, -1}, {2, 3, 1}, {3, 2, -1}};

constexpr int kBuildThreads = 256;

template <typename R>
__global__ void __launch_bounds__(kBuildThreads)
k_block_build(const cpx<R>* __restrict__ prop, int V, const int* __restrict__ row_ptr,
              const uint32_t* __restrict__ entries, const uint32_t* __restrict__ zneed, DevGroups g,
              cpx<R>* __restrict__ blk, int n_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* sS = reinterpret_cast<cpx<R>*>(smem_raw);  // [2][144]  light, strange
  cpx<R>* sD = sS + 288;                              // [2][432]  diquarks (l,l), (l,s)
  cpx<R>* sZ = sD + 864;                              // [g.z_slots] the tensor entries the rows read
  R* sW = reinterpret_cast<R*>(sZ + g.z_slots);       // weights -16..15 (no int->float conversion per term)
  const int site = blockIdx.x, slot = blockIdx.y, tid = threadIdx.x;
  if (tid < 32) sW[tid] = (R)(tid - 16);
  const cpx<R>* P = prop + (size_t)slot * 2 * V * 144;
  for (int i = tid; i < 288; i += kBuildThreads) sS[i] = P[(size_t)(i / 144) * V * 144 + (size_t)site * 144 + i % 144];
  __syncthreads();
  // D_{l f1}[e0][e1][c2] = sum eps(c0,c1,c2) Cg5(a0,a1) S_l[(a0,c0),e0] S_f1[(a1,c1),e1]
  for (int i = tid; i < 864; i += kBuildThreads) {
    const int dq = i / 432, r = i % 432, e0 = r / 36, e1 = (r / 3) % 12, c2 = r % 3;
    const int ca = (c2 + 1) % 3, cb = (c2 + 2) % 3;  // eps(ca,cb,c2) = +1, eps(cb,ca,c2) = -1
    const cpx<R>* S0 = sS;
    const cpx<R>* S1 = sS + 144 * dq;
    cpx<R> acc(0, 0);
#pragma unroll
    for (int gi = 0; gi < 4; gi++) {
      const int a0 = c_cg5[gi][0], a1 = c_cg5[gi][1];
      const R sg = (R)c_cg5[gi][2];
      cpx<R> t(0, 0);
      cmac(t, S0[(3 * a0 + ca) * 12 + e0], S1[(3 * a1 + cb) * 12 + e1]);
      cpx<R> u(0, 0);
      cmac(u, S0[(3 * a0 + cb) * 12 + e0], S1[(3 * a1 + ca) * 12 + e1]);
      acc.re += sg * (t.re - u.re);
      acc.im += sg * (t.im - u.im);
    }
    sD[i] = acc;
  }
  __syncthreads();
  for (int gi = 0; gi < g.n; gi++) {
    // the tensor entries this group reads (and the previous group did not leave)
    const int z1 = g.zneed_first[gi + 1];
    for (int j = g.zneed_first[gi] + tid; j < z1; j += kBuildThreads) {
      const uint32_t zn = zneed[j];
      const int pos = zn & 0x1fff, sl = (zn >> 13) & 1, i = zn >> 14;
      const int fam = sl == 0 ? g.fam0[gi] : g.fam1[gi];
      // F[a][e0][e1][e2] = sum_c2 D[e0][e1][c2] S_f2[(a,c2),e2]
      const int dq = (fam == 2 || fam == 3) ? 1 : 0;  // LSL, LSS read the (l,s) diquark
      const int f2 = (fam == 1 || fam == 3) ? 1 : 0;  // LLS, LSS: strange third quark
      const cpx<R>* D = sD + 432 * dq;
      const cpx<R>* S2 = sS + 144 * f2;
      const int a = i / 1728, r = i % 1728, e01 = r / 12, e2 = r % 12;
      cpx<R> acc(0, 0);
#pragma unroll
      for (int c2 = 0; c2 < 3; c2++) cmac(acc, D[e01 * 3 + c2], S2[(3 * a + c2) * 12 + e2]);
      sZ[pos] = acc;
    }
    __syncthreads();
    const int r0 = g.first[gi], r1 = r0 + g.rows[gi];
    cpx<R>* out = blk + ((size_t)slot * V + site) * n_out;
    for (int r = r0 + tid; r < r1; r += kBuildThreads) {
      cpx<R> acc(0, 0);
      const int k1 = row_ptr[r + 1];
      for (int k = row_ptr[r]; k < k1; k++) {
        const uint32_t e = __ldg(entries + k);
        const R w = sW[((int)(int16_t)(e >> 16)) + 16];
        const cpx<R> z = sZ[e & 0xffffu];
        acc.re = fma(w, z.re, acc.re);
        acc.im = fma(w, z.im, acc.im);
      }
      out[r] = acc;
    }
    __syncthreads();
  }
}

cudaError_t launch_block_build(const void* prop, int V, int n_slots, const int* row_ptr,
                               const uint32_t* entries, const uint32_t* zneed, const DevGroups& g, void* blk,
                               int n_out, bool fp64, cudaStream_t st) {
  dim3 grid(V, n_slots);
  if (fp64) {
    size_t sm = (288 + 864 + g.z_slots) * sizeof(cpx<double>) + 32 * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_block_build<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_block_build<double><<<grid, kBuildThreads, sm, st>>>((const cpx<double>*)prop, V, row_ptr, entries, zneed,
                                                           g, (cpx<double>*)blk, n_out);
  } else {
    size_t sm = (288 + 864 + g.z_slots) * sizeof(cpx<float>) + 32 * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_block_build<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_block_build<float><<<grid, kBuildThreads, sm, st>>>((const cpx<float>*)prop, V, row_ptr, entries, zneed,
                                                          g, (cpx<float>*)blk, n_out);
  }
  return cudaGetLastError();
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
enum { FFT_SITE2FIELD = 0, FFT_FIELD = 1, FFT_FIELD2OUT = 2, FFT_SITE = 3, FFT_SITE2OUT = 4 };

template <typename S, typename R, int N, bool INV, int MODE>
__global__ void __launch_bounds__(256)
k_fft(const cpx<S>* __restrict__ in, cpx<S>* __restrict__ out, long long n_outer, int n_inner, int axis,
      const double* __restrict__ scale) {
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
  } else if (MODE == FFT_FIELD) {
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
  } else if (MODE == FFT_FIELD) {
    line_fft<S, R, N, INV>(in + o * V + base, stride, v);
  } else {
    line_fft<S, R, N, INV>(in + (o * 16 + inner) * V + base, stride, v);
  }
  if (MODE == FFT_SITE2FIELD) {
    cpx<S>* p = out + (o * n_inner + inner) * V + base;
#pragma unroll
    for (int k = 0; k < N; k++) p[k * stride] = cpx<S>(v[k]);
  } else if (MODE == FFT_FIELD) {
    cpx<S>* p = out + o * V + base;
#pragma unroll
    for (int k = 0; k < N; k++) p[k * stride] = cpx<S>(v[k]);
  } else if (MODE == FFT_SITE) {
    cpx<S>* p = out + (o * V + base) * n_inner + inner;
#pragma unroll
    for (int k = 0; k < N; k++) p[(long long)k * stride * n_inner] = cpx<S>(v[k]);
  } else if (MODE == FFT_SITE2OUT) {
    // inner = channel * 16 + spin; out[ch][r][16]
    const R f = (R)scale[inner >> 4];
    cpx<S>* p = out + ((long long)(inner >> 4) * V + base) * 16 + (inner & 15);
#pragma unroll
    for (int k = 0; k < N; k++) p[(long long)k * stride * 16] = cpx<S>(cpx<R>(v[k].re * f, v[k].im * f));
  } else {
    const R f = (R)scale[o];
#pragma unroll
    for (int k = 0; k < N; k++) {
      cpx<S> w(v[k].re * f, v[k].im * f);
      out[(o * V + base + (long long)k * stride) * 16 + inner] = w;
    }
  }
}

template <typename S, typename R, int MODE>
static cudaError_t fft_dispatch(const void* in, void* out, int L, long long n_outer, int n_inner, int axis, bool inv,
                                const double* scale, cudaStream_t st) {
  long long per = (MODE == FFT_SITE2FIELD || MODE == FFT_SITE || MODE == FFT_SITE2OUT) ? n_inner
                  : (MODE == FFT_FIELD ? 1 : 16);
  long long total = n_outer * (long long)L * L * per;
  unsigned blocks = (unsigned)((total + 255) / 256);
  const cpx<S>* i = (const cpx<S>*)in;
  cpx<S>* o = (cpx<S>*)out;
#define BBC_FFT_CASE(NN)                                                                                   \
  case NN:                                                                                                 \
    if (inv) k_fft<S, R, NN, true, MODE><<<blocks, 256, 0, st>>>(i, o, n_outer, n_inner, axis, scale);    \
    else k_fft<S, R, NN, false, MODE><<<blocks, 256, 0, st>>>(i, o, n_outer, n_inner, axis, scale);        \
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
                               cudaStream_t st) {
  cudaError_t e;
  if (fp64) {
    e = fft_dispatch<double, double, FFT_SITE2FIELD>(blk_site, blk_field, L, n_slots, n_rows, 0, false, nullptr, st);
    if (e != cudaSuccess) return e;
    for (int axis = 1; axis < 3; axis++) {
      e = fft_dispatch<double, double, FFT_FIELD>(blk_field, blk_field, L, (long long)n_slots * n_rows, 1, axis, false,
                                                  nullptr, st);
      if (e != cudaSuccess) return e;
    }
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

cudaError_t launch_fft_forward_site(void* blk, int L, int n_slots, int n_rows, bool fp64, cudaStream_t st) {
  for (int axis = 0; axis < 3; axis++) {
    cudaError_t e = fp64 ? fft_dispatch<double, double, FFT_SITE>(blk, blk, L, n_slots, n_rows, axis, false, nullptr, st)
                         : fft_dispatch<float, float, FFT_SITE>(blk, blk, L, n_slots, n_rows, axis, false, nullptr, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_fft_inverse_site(void* ct, void* out, int L, int n_ch, const double* scale, bool fp64_compute,
                                    cudaStream_t st) {
  cudaError_t e;
  for (int axis = 0; axis < 2; axis++) {
    e = fp64_compute ? fft_dispatch<double, double, FFT_SITE>(ct, ct, L, 1, n_ch * 16, axis, true, nullptr, st)
                     : fft_dispatch<double, float, FFT_SITE>(ct, ct, L, 1, n_ch * 16, axis, true, nullptr, st);
    if (e != cudaSuccess) return e;
  }
  return fp64_compute ? fft_dispatch<double, double, FFT_SITE2OUT>(ct, out, L, 1, n_ch * 16, 2, true, scale, st)
                      : fft_dispatch<double, float, FFT_SITE2OUT>(ct, out, L, 1, n_ch * 16, 2, true, scale, st);
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

// --------------------------------------------------------------- contract
// Pair products with one q per lane: a warp runs a fixed list of tasks for 32
// consecutive q (uniform control flow, coalesced loads from the field-major
// block storage), every nA x nB spin product of a task accumulated in
// registers over its open index; P[task*16 + rA*nB + rB][q] is stored for the
// signed sums.
template <typename R, int NA, int NB>
__device__ __forceinline__ void task_products(const cpx<R>* __restrict__ F, long long V, int q, int nq,
                                              const DevTask& t, cpx<R>* __restrict__ P) {
  const int n2 = t.n2, K = t.n1 * n2;
  const int sA1 = t.sA & 0xffff, sA2 = t.sA >> 16, sB1 = t.sB & 0xffff, sB2 = t.sB >> 16;
  cpx<R> acc[NA * NB];
#pragma unroll
  for (int i = 0; i < NA * NB; i++) acc[i] = cpx<R>(0, 0);
  if constexpr (sizeof(R) == 8) {
    // FP64: three real products per complex product (Gauss), sums formed once
    // per loaded value and reused across the register tile
    double s1[NA * NB], s2[NA * NB], s3[NA * NB];
#pragma unroll
    for (int i = 0; i < NA * NB; i++) { s1[i] = 0.0; s2[i] = 0.0; s3[i] = 0.0; }
    int i1 = 0, i2 = 0, oA = 0, oB = 0;
    for (int k = 0; k < K; k++) {
      cpx<R> a[NA], b[NB];
      double as[NA], bs[NB];
#pragma unroll
      for (int r = 0; r < NA; r++) { a[r] = F[(long long)(t.offA[r] + oA) * V + q]; as[r] = a[r].re + a[r].im; }
#pragma unroll
      for (int r = 0; r < NB; r++) { b[r] = F[(long long)(t.offB[r] + oB) * V + nq]; bs[r] = b[r].re + b[r].im; }
#pragma unroll
      for (int ra = 0; ra < NA; ra++)
#pragma unroll
        for (int rb = 0; rb < NB; rb++) {
          const int i = ra * NB + rb;
          s1[i] = fma(a[ra].re, b[rb].re, s1[i]);
          s2[i] = fma(a[ra].im, b[rb].im, s2[i]);
          s3[i] = fma(as[ra], bs[rb], s3[i]);
        }
      if (++i2 == n2) { i2 = 0; ++i1; oA = i1 * sA1; oB = i1 * sB1; }
      else { oA += sA2; oB += sB2; }
    }
#pragma unroll
    for (int i = 0; i < NA * NB; i++) acc[i] = cpx<R>(s1[i] - s2[i], s3[i] - s1[i] - s2[i]);
  } else {
    int i1 = 0, i2 = 0, oA = 0, oB = 0;
    for (int k = 0; k < K; k++) {
      cpx<R> a[NA], b[NB];
#pragma unroll
      for (int r = 0; r < NA; r++) a[r] = F[(long long)(t.offA[r] + oA) * V + q];
#pragma unroll
      for (int r = 0; r < NB; r++) b[r] = F[(long long)(t.offB[r] + oB) * V + nq];
#pragma unroll
      for (int ra = 0; ra < NA; ra++)
#pragma unroll
        for (int rb = 0; rb < NB; rb++) cmac(acc[ra * NB + rb], a[ra], b[rb]);
      if (++i2 == n2) { i2 = 0; ++i1; oA = i1 * sA1; oB = i1 * sB1; }
      else { oA += sA2; oB += sB2; }
    }
  }
#pragma unroll
  for (int i = 0; i < NA * NB; i++) P[(long long)i * V] = acc[i];
}

constexpr int kPairWarps = 4;

template <typename R>
__global__ void __launch_bounds__(32 * kPairWarps)
k_pair_products(const cpx<R>* __restrict__ F, int L, const DevTask* __restrict__ tasks,
                const int* __restrict__ group_ptr, const int* __restrict__ group_task, int n_groups,
                cpx<R>* __restrict__ P) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // task groups of one q tile are adjacent in the grid, so the tile's block
  // rows are shared in L2 while its groups run
  const int g = blockIdx.x * kPairWarps + warp;
  const int V = L * L * L;
  const int q = blockIdx.y * 32 + lane;
  if (g >= n_groups || q >= V) return;
  const int qx = q % L, qy = (q / L) % L, qz = q / (L * L);
  const int nq = (L - qx) % L + L * ((L - qy) % L + L * ((L - qz) % L));
  const int j1 = group_ptr[g + 1];
  for (int j = group_ptr[g]; j < j1; j++) {
    const int ti = group_task[j];
    const DevTask t = tasks[ti];
    cpx<R>* p = P + (long long)ti * 16 * V + q;
    const int nA = t.nAnB & 0xff;
    if (nA == 4) task_products<R, 4, 4>(F, V, q, nq, t, p);
    else if (nA == 2) task_products<R, 2, 8>(F, V, q, nq, t, p);
    else task_products<R, 8, 2>(F, V, q, nq, t, p);
  }
}

// Signed FP64 sums over Wick diagrams: Ct[o][q] = sum_c coef_c P[item_c][q],
// o = channel*16 + spin.
template <typename R>
__global__ void __launch_bounds__(128)
k_wick_sums(const cpx<R>* __restrict__ P, int V, const int* __restrict__ cptr, const int* __restrict__ citem,
            const double* __restrict__ ccoef, cpx<double>* __restrict__ Ct) {
  const int q = blockIdx.x * 128 + threadIdx.x, o = blockIdx.y;
  if (q >= V) return;
  cpx<double> s(0, 0);
  const int c1 = cptr[o + 1];
  for (int c = cptr[o]; c < c1; c++) {
    const double w = ccoef[c];
    const cpx<R> p = P[(long long)citem[c] * V + q];
    s.re = fma(w, (double)p.re, s.re);
    s.im = fma(w, (double)p.im, s.im);
  }
  Ct[(long long)o * V + q] = s;
}

cudaError_t launch_pair_products(const void* blk_field, int L, const DevTask* tasks, const int* group_ptr,
                                 const int* group_task, int n_groups, void* P, bool fp64, cudaStream_t st) {
  const int V = L * L * L;
  dim3 g1((n_groups + kPairWarps - 1) / kPairWarps, (V + 31) / 32);
  if (fp64)
    k_pair_products<double><<<g1, 32 * kPairWarps, 0, st>>>((const cpx<double>*)blk_field, L, tasks, group_ptr,
                                                            group_task, n_groups, (cpx<double>*)P);
  else
    k_pair_products<float><<<g1, 32 * kPairWarps, 0, st>>>((const cpx<float>*)blk_field, L, tasks, group_ptr,
                                                           group_task, n_groups, (cpx<float>*)P);
  return cudaGetLastError();
}

cudaError_t launch_wick_sums(const void* P, int L, const int* cptr, const int* citem, const double* ccoef, int n_ch,
                             void* ct, bool fp64, cudaStream_t st) {
  const int V = L * L * L;
  dim3 g2((V + 127) / 128, n_ch * 16);
  if (fp64) k_wick_sums<double><<<g2, 128, 0, st>>>((const cpx<double>*)P, V, cptr, citem, ccoef, (cpx<double>*)ct);
  else k_wick_sums<float><<<g2, 128, 0, st>>>((const cpx<float>*)P, V, cptr, citem, ccoef, (cpx<double>*)ct);
  return cudaGetLastError();
}

// ------------------------------------------------- fused contraction (FP32)
// One CTA per pair {q, -q}.  The q-row and the -q row of the q-major
// Fourier-space blocks (blk[q][n_out]) are staged in shared memory once,
// interleaved as R[i] = (F_q[i], F_-q[i]), so one 16-byte load serves both
// products A(q) B(-q) (side 0) and A(-q) B(q) (side 1); every block element is
// read from HBM exactly once.  Warps run units (batch of up to 32 tasks of
// one shape and one open-index length, k range): lane l takes task l, so
// control flow is uniform within the warp.  Products accumulate in FP32
// registers and are added into P[side][task*16 + spin pair] in shared memory.
// The products are then converted once to FP64 and the signed FP64 sums over
// Wick diagrams run in the same CTA, writing ct[q][o].
template <int NA, int NB>
__device__ __forceinline__ void unit_products_pair(const float4* __restrict__ R, const DevTask& t, int k0, int k1,
                                                   cpx<float>* P0, cpx<float>* P1, int rot, bool self) {
  const int n2 = t.n2;
  const int sA1 = t.sA & 0xffff, sA2 = t.sA >> 16, sB1 = t.sB & 0xffff, sB2 = t.sB >> 16;
  int i1 = k0 / n2, i2 = k0 - i1 * n2;
  int oA = i1 * sA1 + i2 * sA2, oB = i1 * sB1 + i2 * sB2;
  const int wrapA = sA1 - (n2 - 1) * sA2, wrapB = sB1 - (n2 - 1) * sB2;
  cpx<float> acc0[NA * NB], acc1[NA * NB];
#pragma unroll
  for (int i = 0; i < NA * NB; i++) { acc0[i] = cpx<float>(0.f, 0.f); acc1[i] = cpx<float>(0.f, 0.f); }
  for (int k = k0; k < k1; k++) {
    float4 a[NA], b[NB];
#pragma unroll
    for (int r = 0; r < NA; r++) a[r] = R[t.offA[r] + oA];
#pragma unroll
    for (int r = 0; r < NB; r++) b[r] = R[t.offB[r] + oB];
#pragma unroll
    for (int ra = 0; ra < NA; ra++)
#pragma unroll
      for (int rb = 0; rb < NB; rb++) {
        cmac(acc0[ra * NB + rb], cpx<float>(a[ra].x, a[ra].y), cpx<float>(b[rb].z, b[rb].w));
        cmac(acc1[ra * NB + rb], cpx<float>(a[ra].z, a[ra].w), cpx<float>(b[rb].x, b[rb].y));
      }
    if (++i2 == n2) { i2 = 0; oA += wrapA; oB += wrapB; }
    else { oA += sA2; oB += sB2; }
  }
  // P slot of product i of task ti: ti*16 + ((i + ti) & 15) -- the rotation
  // spreads the 32 lanes' (distinct tasks') slots over the shared-memory banks
#pragma unroll
  for (int i = 0; i < NA * NB; i++) {
    cpx<float>* d0 = P0 + ((i + rot) & 15);
    atomicAdd(&d0->re, acc0[i].re);
    atomicAdd(&d0->im, acc0[i].im);
    if (!self) {
      cpx<float>* d1 = P1 + ((i + rot) & 15);
      atomicAdd(&d1->re, acc1[i].re);
      atomicAdd(&d1->im, acc1[i].im);
    }
  }
}

constexpr int kFusedThreads = 512;

__global__ void __launch_bounds__(kFusedThreads, 1)
k_contract_fused(const cpx<float>* __restrict__ blk, int L, int n_out, const int* __restrict__ qlist,
                 const DevTask* __restrict__ tasks, int n_tasks, const WarpBatch* __restrict__ batches,
                 const int* __restrict__ wptr, const int4* __restrict__ wunits, const int* __restrict__ cptr,
                 const int* __restrict__ citem, const double* __restrict__ ccoef, int n_outputs,
                 cpx<double>* __restrict__ ct) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int np = n_tasks * 16;                                        // products per side
  const size_t region = max((size_t)n_out * 16, (size_t)2 * np * 16);  // rows, later the FP64 products
  float4* R = reinterpret_cast<float4*>(smem_raw);                     // [n_out] (F_q, F_-q)
  cpx<double>* Pd = reinterpret_cast<cpx<double>*>(smem_raw);         // [2][np], after the products
  cpx<float>* P = reinterpret_cast<cpx<float>*>(smem_raw + region);   // [2][np]
  const int q = qlist[blockIdx.x];
  const int qx = q % L, qy = (q / L) % L, qz = q / (L * L);
  const int nq = (L - qx) % L + L * ((L - qy) % L + L * ((L - qz) % L));
  const bool self = nq == q;
  {
    const float2* s0 = reinterpret_cast<const float2*>(blk + (size_t)q * n_out);
    const float2* s1 = reinterpret_cast<const float2*>(blk + (size_t)nq * n_out);
    for (int i = tid; i < n_out; i += kFusedThreads) {
      const float2 x = __ldg(s0 + i), y = self ? x : __ldg(s1 + i);
      R[i] = make_float4(x.x, x.y, y.x, y.y);
    }
    float4* pz = reinterpret_cast<float4*>(P);
    for (int i = tid; i < np; i += kFusedThreads) pz[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  const int u1 = wptr[warp + 1];
  for (int u = wptr[warp]; u < u1; u++) {
    const int4 un = wunits[u];  // batch, -, k0, k1
    const WarpBatch& wb = batches[un.x];
    if (lane >= wb.n) continue;
    const int ti = wb.task[lane];
    const DevTask t = tasks[ti];
    cpx<float>* p0 = P + ti * 16;
    cpx<float>* p1 = P + np + ti * 16;
    if (wb.nA == 4) unit_products_pair<4, 4>(R, t, un.z, un.w, p0, p1, ti, self);
    else if (wb.nA == 2) unit_products_pair<2, 8>(R, t, un.z, un.w, p0, p1, ti, self);
    else unit_products_pair<8, 2>(R, t, un.z, un.w, p0, p1, ti, self);
  }
  __syncthreads();
  // products to FP64 once (undoing the slot rotation), over the rows' space
  const int sides = self ? 1 : 2;
  for (int j = tid; j < sides * np; j += kFusedThreads) {
    const int side = j / np, it = j - side * np, ti = it >> 4;
    const cpx<float> v = P[side * np + (ti << 4) + ((it + ti) & 15)];
    Pd[j] = cpx<double>((double)v.re, (double)v.im);
  }
  __syncthreads();
  for (int j = tid; j < sides * n_outputs; j += kFusedThreads) {
    const int side = j / n_outputs, o = j - side * n_outputs;
    const cpx<double>* Ps = Pd + side * np;
    cpx<double> acc(0, 0);
    const int c1 = cptr[o + 1];
    for (int c = cptr[o]; c < c1; c++) {
      const double w = ccoef[c];
      const cpx<double> v = Ps[citem[c]];
      acc.re = fma(w, v.re, acc.re);
      acc.im = fma(w, v.im, acc.im);
    }
    ct[(size_t)(side ? nq : q) * n_outputs + o] = acc;
  }
}

size_t contract_fused_smem(int n_out, int n_tasks) {
  const size_t np = (size_t)n_tasks * 16;
  return std::max((size_t)n_out * 16, 2 * np * 16) + 2 * np * sizeof(cpx<float>);
}

cudaError_t launch_contract_fused(const void* blk, int L, int n_out, const int* qlist, int n_q, const DevTask* tasks,
                                  int n_tasks, const WarpBatch* batches, const int* wptr, const int4* wunits,
                                  const int* cptr, const int* citem, const double* ccoef, int n_ch, void* ct,
                                  cudaStream_t st) {
  const size_t sm = contract_fused_smem(n_out, n_tasks);
  cudaError_t e = cudaFuncSetAttribute(k_contract_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_contract_fused<<<n_q, kFusedThreads, sm, st>>>((const cpx<float>*)blk, L, n_out, qlist, tasks, n_tasks, batches,
                                                   wptr, wunits, cptr, citem, ccoef, n_ch * 16, (cpx<double>*)ct);
  return cudaGetLastError();
}

// ------------------------------------------------------------ normalisation
// scale[ch] = f[ch] * 2^(nl[ch] k_l + ns[ch] k_s): 1/V, the mass factor and the
// undoing of the power-of-two propagator rescaling of this slice.
__global__ void k_scales(ScaleParams p, const int* __restrict__ kexp, double* __restrict__ scale) {
  const int ch = threadIdx.x;
  if (ch < p.n_ch) scale[ch] = ldexp(p.f[ch], p.nl[ch] * kexp[0] + p.ns[ch] * kexp[1]);
}

cudaError_t launch_scales(const ScaleParams& p, const int* kexp, double* scale, cudaStream_t st) {
  k_scales<<<1, kMaxChannels, 0, st>>>(p, kexp, scale);
  return cudaGetLastError();
}

}  // namespace bbc
