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
              const uint32_t* __restrict__ entries, const uint16_t* __restrict__ zneed, DevGroups g,
              cpx<R>* __restrict__ blk, int n_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* sS = reinterpret_cast<cpx<R>*>(smem_raw);  // [2][144]  light, strange
  cpx<R>* sD = sS + 288;                              // [2][432]  diquarks (l,l), (l,s)
  cpx<R>* sZ = sD + 864;                              // [2][3456] sink-tensor families
  R* sW = reinterpret_cast<R*>(sZ + 2 * 3456);        // weights -16..15 (no int->float conversion per term)
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
      const int zi = zneed[j], sl = zi / 3456, i = zi % 3456;
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
      sZ[zi] = acc;
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
                               const uint32_t* entries, const uint16_t* zneed, const DevGroups& g, void* blk,
                               int n_out, bool fp64, cudaStream_t st) {
  dim3 grid(V, n_slots);
  if (fp64) {
    size_t sm = (288 + 864 + 2 * 3456) * sizeof(cpx<double>) + 32 * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_block_build<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_block_build<double><<<grid, kBuildThreads, sm, st>>>((const cpx<double>*)prop, V, row_ptr, entries, zneed,
                                                           g, (cpx<double>*)blk, n_out);
  } else {
    size_t sm = (288 + 864 + 2 * 3456) * sizeof(cpx<float>) + 32 * sizeof(float);
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

template <typename S, typename R, int N, bool INV>
__global__ void __launch_bounds__(256)
k_fft_pass(cpx<S>* __restrict__ data, long long n_outer, int n_inner, int axis) {
  const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long lines = (long long)N * N;
  if (gid >= n_outer * lines * n_inner) return;
  const int i = (int)(gid % n_inner);
  const long long rest = gid / n_inner;
  const int line = (int)(rest % lines);
  const long long o = rest / lines;
  const int a = line % N, b = line / N;
  int base, stride;
  if (axis == 0) { base = N * (a + N * b); stride = 1; }
  else if (axis == 1) { base = a + N * N * b; stride = N; }
  else { base = a + N * b; stride = N * N; }
  const long long V = (long long)N * N * N;
  cpx<S>* p = data + (o * V + base) * (long long)n_inner + i;
  const long long step = (long long)stride * n_inner;
  cpx<R> v[N];
  load_bitrev<S, R, N>(v, p, step, std::make_integer_sequence<int, N>{});
  fft_pow2<R, N, INV>(v);
#pragma unroll
  for (int k = 0; k < N; k++) p[k * step] = cpx<S>(v[k]);
}

template <typename S, typename R>
static cudaError_t fft_dispatch(void* data, int L, long long n_outer, int n_inner, int axis, bool inv,
                                cudaStream_t st) {
  long long total = n_outer * (long long)L * L * n_inner;
  unsigned blocks = (unsigned)((total + 255) / 256);
  cpx<S>* d = (cpx<S>*)data;
#define BBC_FFT_CASE(NN)                                                              \
  case NN:                                                                            \
    if (inv) k_fft_pass<S, R, NN, true><<<blocks, 256, 0, st>>>(d, n_outer, n_inner, axis); \
    else k_fft_pass<S, R, NN, false><<<blocks, 256, 0, st>>>(d, n_outer, n_inner, axis);    \
    break;
  switch (L) {
    BBC_FFT_CASE(2)
    BBC_FFT_CASE(4)
    BBC_FFT_CASE(8)
    BBC_FFT_CASE(16)
    BBC_FFT_CASE(32)
    default: return cudaErrorInvalidValue;
  }
#undef BBC_FFT_CASE
  return cudaGetLastError();
}

cudaError_t launch_fft_pass(void* data, int L, long long n_outer, int n_inner, int axis, bool inverse,
                            bool fp64_store, bool fp64_compute, cudaStream_t st) {
  if (fp64_store && fp64_compute) return fft_dispatch<double, double>(data, L, n_outer, n_inner, axis, inverse, st);
  if (fp64_store) return fft_dispatch<double, float>(data, L, n_outer, n_inner, axis, inverse, st);
  return fft_dispatch<float, float>(data, L, n_outer, n_inner, axis, inverse, st);
}

// --------------------------------------------------------------- contract
// One schedule unit: the open-index range [k0, k1) of one task, all nA x nB
// spin products accumulated in registers (each loaded block value is reused
// nB or nA times).
template <typename R, int NA, int NB>
__device__ __forceinline__ void run_unit(const cpx<R>* __restrict__ A, const cpx<R>* __restrict__ B,
                                         const DevTask& t, int k0, int k1, cpx<R> (&acc)[16]) {
  const int n2 = t.n2;
  const int sA1 = t.sA & 0xffff, sA2 = t.sA >> 16, sB1 = t.sB & 0xffff, sB2 = t.sB >> 16;
  int i1 = k0 / n2, i2 = k0 - i1 * n2;
  int oA = i1 * sA1 + i2 * sA2, oB = i1 * sB1 + i2 * sB2;
  const int wrapA = sA1 - (n2 - 1) * sA2, wrapB = sB1 - (n2 - 1) * sB2;
  for (int k = k0; k < k1; k++) {
    cpx<R> a[NA], b[NB];
#pragma unroll
    for (int r = 0; r < NA; r++) a[r] = A[t.offA[r] + oA];
#pragma unroll
    for (int r = 0; r < NB; r++) b[r] = B[t.offB[r] + oB];
#pragma unroll
    for (int ra = 0; ra < NA; ra++)
#pragma unroll
      for (int rb = 0; rb < NB; rb++) cmac(acc[ra * NB + rb], a[ra], b[rb]);
    if (++i2 == n2) { i2 = 0; oA += wrapA; oB += wrapB; }
    else { oA += sA2; oB += sB2; }
  }
}

// FP64 variant with three real products per complex product (Gauss):
// s1 += ar br, s2 += ai bi, s3 += (ar + ai)(br + bi); then re = s1 - s2,
// im = s3 - s1 - s2.  The sums ar + ai, br + bi are formed once per loaded
// value and reused across the register tile: 3 instead of 4 FP64 FMAs per
// complex multiply-add on the FP64-bound path.
template <int NA, int NB>
__device__ __forceinline__ void run_unit_gauss(const cpx<double>* __restrict__ A, const cpx<double>* __restrict__ B,
                                               const DevTask& t, int k0, int k1, cpx<double> (&acc)[16]) {
  const int n2 = t.n2;
  const int sA1 = t.sA & 0xffff, sA2 = t.sA >> 16, sB1 = t.sB & 0xffff, sB2 = t.sB >> 16;
  int i1 = k0 / n2, i2 = k0 - i1 * n2;
  int oA = i1 * sA1 + i2 * sA2, oB = i1 * sB1 + i2 * sB2;
  const int wrapA = sA1 - (n2 - 1) * sA2, wrapB = sB1 - (n2 - 1) * sB2;
  double s1[NA * NB], s2[NA * NB], s3[NA * NB];
#pragma unroll
  for (int i = 0; i < NA * NB; i++) { s1[i] = 0.0; s2[i] = 0.0; s3[i] = 0.0; }
  for (int k = k0; k < k1; k++) {
    cpx<double> a[NA], b[NB];
    double as[NA], bs[NB];
#pragma unroll
    for (int r = 0; r < NA; r++) { a[r] = A[t.offA[r] + oA]; as[r] = a[r].re + a[r].im; }
#pragma unroll
    for (int r = 0; r < NB; r++) { b[r] = B[t.offB[r] + oB]; bs[r] = b[r].re + b[r].im; }
#pragma unroll
    for (int ra = 0; ra < NA; ra++)
#pragma unroll
      for (int rb = 0; rb < NB; rb++) {
        const int i = ra * NB + rb;
        s1[i] = fma(a[ra].re, b[rb].re, s1[i]);
        s2[i] = fma(a[ra].im, b[rb].im, s2[i]);
        s3[i] = fma(as[ra], bs[rb], s3[i]);
      }
    if (++i2 == n2) { i2 = 0; oA += wrapA; oB += wrapB; }
    else { oA += sA2; oB += sB2; }
  }
#pragma unroll
  for (int i = 0; i < NA * NB; i++) acc[i] = cpx<double>(s1[i] - s2[i], s3[i] - s1[i] - s2[i]);
}

template <typename R, int NA, int NB>
__device__ __forceinline__ void run_unit_any(const cpx<R>* A, const cpx<R>* B, const DevTask& t, int k0, int k1,
                                             cpx<R> (&acc)[16]) {
  if constexpr (sizeof(R) == 8) run_unit_gauss<NA, NB>(A, B, t, k0, k1, acc);
  else run_unit<R, NA, NB>(A, B, t, k0, k1, acc);
}

template <typename R>
__device__ __forceinline__ void smem_add(cpx<R>* p, cpx<R> v) {
  atomicAdd(&p->re, v.re);
  atomicAdd(&p->im, v.im);
}

// PAIR = false: one CTA per q, block rows read from global memory (FP64).
// PAIR = true: one CTA per pair {q, -q}; both block rows staged in shared
// memory once and used for the products at q (A(q) B(-q)) and at -q (FP32).
template <typename R, bool PAIR, int THREADS>
__global__ void __launch_bounds__(THREADS)
k_contract(const cpx<R>* __restrict__ blk, int L, int n_out, const int* __restrict__ qlist,
           const DevTask* __restrict__ tasks, int n_tasks, const int* __restrict__ sched_ptr,
           const int2* __restrict__ units, const int* __restrict__ cptr, const int* __restrict__ citem,
           const double* __restrict__ ccoef, int n_outputs, cpx<double>* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, V = L * L * L;
  const int q = PAIR ? qlist[blockIdx.x] : blockIdx.x;
  const int qx = q % L, qy = (q / L) % L, qz = q / (L * L);
  const int nq = (L - qx) % L + L * ((L - qy) % L + L * ((L - qz) % L));
  const int sides = (PAIR && nq != q) ? 2 : 1;
  cpx<R>* rows = reinterpret_cast<cpx<R>*>(smem_raw);
  cpx<R>* P = PAIR ? rows + 2 * n_out : rows;
  const cpx<R>* gq = blk + (size_t)q * n_out;
  const cpx<R>* gn = blk + (size_t)nq * n_out;
  if (PAIR) {
    // n_out * sizeof(cpx<R>) is a multiple of 16 bytes (n_out even)
    const int n16 = n_out * (int)sizeof(cpx<R>) / 16;
    const float4* s0 = reinterpret_cast<const float4*>(gq);
    const float4* s1 = reinterpret_cast<const float4*>(gn);
    float4* d = reinterpret_cast<float4*>(rows);
    for (int i = tid; i < n16; i += THREADS) {
      d[i] = __ldg(s0 + i);
      if (sides == 2) d[n16 + i] = __ldg(s1 + i);
    }
  }
  for (int side = 0; side < sides; side++) {
    const cpx<R>* A = PAIR ? rows + side * n_out : gq;
    const cpx<R>* B = PAIR ? rows + (sides == 2 ? 1 - side : 0) * n_out : gn;
    const int qq = side ? nq : q;
    for (int i = tid; i < n_tasks * 16; i += THREADS) P[i] = cpx<R>(0, 0);
    __syncthreads();
    const int u1 = sched_ptr[tid + 1];
    for (int u = sched_ptr[tid]; u < u1; u++) {
      const int2 un = units[u];
      const DevTask t = tasks[un.x];
      const int k0 = un.y & 0xffff, k1 = un.y >> 16;
      cpx<R> acc[16];
#pragma unroll
      for (int i = 0; i < 16; i++) acc[i] = cpx<R>(0, 0);
      const int nA = t.nAnB & 0xff;
      if (nA == 4) run_unit_any<R, 4, 4>(A, B, t, k0, k1, acc);
      else if (nA == 2) run_unit_any<R, 2, 8>(A, B, t, k0, k1, acc);
      else run_unit_any<R, 8, 2>(A, B, t, k0, k1, acc);
      cpx<R>* p = P + un.x * 16;
#pragma unroll
      for (int i = 0; i < 16; i++) smem_add(p + i, acc[i]);
    }
    __syncthreads();
    // signed FP64 sum over Wick diagrams into channels and spins
    for (int o = tid; o < n_outputs; o += THREADS) {
      cpx<double> s(0, 0);
      const int c1 = cptr[o + 1];
      for (int c = cptr[o]; c < c1; c++) {
        const double w = ccoef[c];
        const cpx<R> p = P[citem[c]];
        s.re = fma(w, (double)p.re, s.re);
        s.im = fma(w, (double)p.im, s.im);
      }
      out[((size_t)(o >> 4) * V + qq) * 16 + (o & 15)] = s;
    }
    __syncthreads();
  }
}

int contract_threads(bool fp64) { return fp64 ? 256 : 512; }

size_t contract_smem(bool fp64, int n_out, int n_tasks) {
  return fp64 ? (size_t)n_tasks * 16 * sizeof(cpx<double>)
              : (size_t)(2 * n_out + n_tasks * 16) * sizeof(cpx<float>);
}

cudaError_t launch_contract(const void* blk, int L, int n_out, const int* qlist, int n_q, const DevTask* tasks,
                            int n_tasks, const int* sched_ptr, const int2* units, const int* cptr, const int* citem,
                            const double* ccoef, int n_ch, void* out, bool fp64, cudaStream_t st) {
  const int V = L * L * L;
  const size_t sm = contract_smem(fp64, n_out, n_tasks);
  if (fp64) {
    auto k = k_contract<double, false, 256>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k<<<V, 256, sm, st>>>((const cpx<double>*)blk, L, n_out, qlist, tasks, n_tasks, sched_ptr, units, cptr, citem,
                          ccoef, n_ch * 16, (cpx<double>*)out);
  } else {
    auto k = k_contract<float, true, 512>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k<<<n_q, 512, sm, st>>>((const cpx<float>*)blk, L, n_out, qlist, tasks, n_tasks, sched_ptr, units, cptr, citem,
                            ccoef, n_ch * 16, (cpx<double>*)out);
  }
  return cudaGetLastError();
}

// -------------------------------------------------------------- normalise
__global__ void k_normalise(cpx<double>* __restrict__ out, int V, NormParams p, const int* __restrict__ kexp) {
  const long long n = (long long)p.n_ch * V * 16;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const int kl = kexp[0], ks = kexp[1];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
    const int ch = (int)(i / ((long long)V * 16));
    const double s = ldexp(p.f[ch], p.nl[ch] * kl + p.ns[ch] * ks);
    cpx<double> v = out[i];
    out[i] = cpx<double>(v.re * s, v.im * s);
  }
}

cudaError_t launch_normalise(void* out, int V, const NormParams& p, const int* kexp, cudaStream_t st) {
  long long n = (long long)p.n_ch * V * 16;
  int blocks = (int)std::min<long long>((n + 255) / 256, 152 * 16);
  k_normalise<<<blocks, 256, 0, st>>>((cpx<double>*)out, V, p, kexp);
  return cudaGetLastError();
}

}  // namespace bbc
