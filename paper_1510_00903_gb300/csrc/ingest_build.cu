// ingest_build.cu -- propagator ingest with exact power-of-two rescaling, per-site baryon blocks (Sec. 3 blocks, Appendix A aggregation), per-channel normalisation factors (Sec. 2 Eq. 2)
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <utility>

#include "device_common.cuh"

namespace bbc {

// ------------------------------------------------------------------ ingest
// Largest |x| of the slice (a NaN counts as infinite: a max would drop it),
// as the bits of a non-negative double, which order like the values.  The
// scan runs on the bit patterns in integer arithmetic: |x| is x with the sign
// bit cleared, and every NaN pattern lies above the infinite one (clamped to
// it); complex64 input is widened to double bits once per warp.
__global__ void k_absmax(const void* __restrict__ src, int dtype, long long n_real,
                         unsigned long long* amax) {
  // 16-byte loads: two doubles or four floats per thread and step (n_real is
  // a multiple of 4: 288 reals per site; the source is 16-byte aligned)
  unsigned long long m = 0;
  long long stride = (long long)gridDim.x * blockDim.x;
  if (dtype == 0) {
    const ulonglong2* x = (const ulonglong2*)src;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_real / 2; i += stride) {
      const ulonglong2 v = x[i];
      const unsigned long long a = v.x & 0x7fffffffffffffffull, b = v.y & 0x7fffffffffffffffull;
      m = a > m ? a : m;
      m = b > m ? b : m;
    }
    m = m > 0x7ff0000000000000ull ? 0x7ff0000000000000ull : m;
  } else {
    const uint4* x = (const uint4*)src;
    unsigned mf = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_real / 4; i += stride) {
      const uint4 v = x[i];
      const unsigned a = max(v.x & 0x7fffffffu, v.y & 0x7fffffffu), b = max(v.z & 0x7fffffffu, v.w & 0x7fffffffu);
      mf = max(mf, max(a, b));
    }
    mf = mf > 0x7f800000u ? 0x7f800000u : mf;
    m = (unsigned long long)__double_as_longlong((double)__uint_as_float(mf));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(amax, m);
}

// x * 2^-k with k = ilogb(max |x|) + 1, an exact rescaling into [-1, 1).
// complex64 input into FP32 or double-float storage scales in FP32 (exact
// for every result in the normal range; the double-float low word is 0).
template <typename R>
__global__ void k_convert(const void* __restrict__ src, int dtype, long long n_real,
                          const unsigned long long* __restrict__ amax, int* kexp, R* __restrict__ dst) {
  double m = __longlong_as_double((long long)*amax);
  int k = (m > 0.0 && m <= 1.7976931348623157e308) ? ilogb(m) + 1 : 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) *kexp = k;
  long long stride = (long long)gridDim.x * blockDim.x;
  // 16-byte loads (n_real is a multiple of 4, the source 16-byte aligned)
  if constexpr (!std::is_same<R, double>::value) {
    if (dtype == 1) {
      for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_real / 4; i += stride) {
        const float4 v = ((const float4*)src)[i];
        const float y0 = ldexpf(v.x, -k), y1 = ldexpf(v.y, -k), y2 = ldexpf(v.z, -k), y3 = ldexpf(v.w, -k);
        if constexpr (std::is_same<R, dfr>::value) {
          float4* d = (float4*)(dst + 4 * i);
          d[0] = make_float4(y0, 0.f, y1, 0.f);
          d[1] = make_float4(y2, 0.f, y3, 0.f);
        } else {
          ((float4*)dst)[i] = make_float4(y0, y1, y2, y3);
        }
      }
      return;
    }
  }
  if (dtype == 0) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_real / 2; i += stride) {
      const double2 v = ((const double2*)src)[i];
      dst[2 * i] = (R)ldexp(v.x, -k);
      dst[2 * i + 1] = (R)ldexp(v.y, -k);
    }
  } else {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_real / 2; i += stride) {
      const float2 v = ((const float2*)src)[i];
      dst[2 * i] = (R)ldexp((double)v.x, -k);
      dst[2 * i + 1] = (R)ldexp((double)v.y, -k);
    }
  }
}

cudaError_t launch_absmax(const void* src, int dtype, long long n_complex, unsigned long long* amax,
                          cudaStream_t st) {
  long long n = 2 * n_complex;
  if (n % 4) return cudaErrorInvalidValue;  // whole 16-byte loads
  int blocks = (int)std::min<long long>((n / 2 + 255) / 256, 152 * 8);
  k_absmax<<<blocks, 256, 0, st>>>(src, dtype, n, amax);
  return cudaGetLastError();
}

cudaError_t launch_convert(const void* src, int dtype, long long n_complex, const unsigned long long* amax,
                           int* kexp, void* dst, int kind, cudaStream_t st) {
  long long n = 2 * n_complex;
  if (n % 4) return cudaErrorInvalidValue;  // whole 16-byte loads
  int blocks = (int)std::min<long long>((n / 2 + 255) / 256, 152 * 8);
  if (kind == RK_F64) k_convert<double><<<blocks, 256, 0, st>>>(src, dtype, n, amax, kexp, (double*)dst);
  else if (kind == RK_DF) k_convert<dfr><<<blocks, 256, 0, st>>>(src, dtype, n, amax, kexp, (dfr*)dst);
  else k_convert<float><<<blocks, 256, 0, st>>>(src, dtype, n, amax, kexp, (float*)dst);
  return cudaGetLastError();
}

// ------------------------------------------------------------ block build
// Diquark matrices Gamma1 (Dirac representation, C = gamma4 gamma2), four
// non-zero entries (a0, a1, sign) each: C gamma5 = diag(J, J); the decuplet's
// i C gamma_1 = diag(s3, -s3), C gamma_2 = diag(1, -1), -i C gamma_3 =
// diag(s1, -s1) (Sec. 4 footnote, with the phase that makes them real).
__constant__ int c_gam[4][4][3] = {{{0, 1, 1}, {1, 0, -1}, {2, 3, 1}, {3, 2, -1}},
                                   {{0, 0, 1}, {1, 1, -1}, {2, 2, -1}, {3, 3, 1}},
                                   {{0, 0, 1}, {1, 1, 1}, {2, 2, -1}, {3, 3, -1}},
                                   {{0, 1, 1}, {1, 0, 1}, {2, 3, -1}, {3, 2, -1}}};

// One CTA builds the blocks of SITES consecutive sites with THREADS threads:
// the propagators, diquarks and tensor entries of every site sit in shared
// memory, and each thread runs one block row for all SITES sites, so every
// row's entry list is read once per SITES sites.
template <typename R, int SITES, int THREADS>
__global__ void __launch_bounds__(THREADS)
k_block_build(const cpx<R>* __restrict__ prop, int V, const int2* __restrict__ ell_chunk,
              const uint32_t* __restrict__ ell, const uint32_t* __restrict__ zneed, DevGroups g,
              cpx<R>* __restrict__ blk, int n_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nd = g.n_dq * 432;
  cpx<R>* sS = reinterpret_cast<cpx<R>*>(smem_raw);  // [SITES][2][144]  light, strange
  cpx<R>* sD = sS + SITES * 288;                      // [SITES][n_dq][432]  the diquarks the families read
  cpx<R>* sZ = sD + SITES * nd;                       // [SITES][g.z_slots] the tensor entries the rows read
  R* sW = reinterpret_cast<R*>(sZ + SITES * g.z_slots);  // weights -16..15 (no int->float conversion per term)
  const int site0 = blockIdx.x * SITES, slot = blockIdx.y, tid = threadIdx.x;
  const int zs = g.z_slots;
  if (tid < 32) sW[tid] = (R)(tid - 16);
  const cpx<R>* P = prop + (size_t)slot * 2 * V * 144;
  for (int i = tid; i < SITES * 288; i += THREADS) {
    const int s = i / 288, j = i - s * 288;
    sS[i] = P[(size_t)(j / 144) * V * 144 + (size_t)(site0 + s) * 144 + j % 144];
  }
  __syncthreads();
  // D_{f0 f1}[e0][e1][c2] = sum eps(c0,c1,c2) Gamma1(a0,a1) S_f0[(a0,c0),e0] S_f1[(a1,c1),e1]
  for (int ii = tid; ii < SITES * nd; ii += THREADS) {
    const int s = ii / nd, i = ii - s * nd;
    const int dq = i / 432, r = i % 432, e0 = r / 36, e1 = (r / 3) % 12, c2 = r % 3;
    const int ca = (c2 + 1) % 3, cb = (c2 + 2) % 3;  // eps(ca,cb,c2) = +1, eps(cb,ca,c2) = -1
    const cpx<R>* S0 = sS + s * 288 + 144 * g.dq_f0[dq];
    const cpx<R>* S1 = sS + s * 288 + 144 * g.dq_f1[dq];
    const int gam = g.dq_gam[dq];
    cpx<R> acc(0, 0);
#pragma unroll
    for (int gi = 0; gi < 4; gi++) {
      const int a0 = c_gam[gam][gi][0], a1 = c_gam[gam][gi][1];
      const R sg = (R)c_gam[gam][gi][2];
      cpx<R> t(0, 0);
      cmac(t, S0[(3 * a0 + ca) * 12 + e0], S1[(3 * a1 + cb) * 12 + e1]);
      cpx<R> u(0, 0);
      cmac(u, S0[(3 * a0 + cb) * 12 + e0], S1[(3 * a1 + ca) * 12 + e1]);
      acc.re += sg * (t.re - u.re);
      acc.im += sg * (t.im - u.im);
    }
    sD[ii] = acc;
  }
  __syncthreads();
  for (int gi = 0; gi < g.n; gi++) {
    // the tensor entries this group reads (and the previous group did not leave)
    const int z0 = g.zneed_first[gi], nz = g.zneed_first[gi + 1] - z0;
    for (int jj = tid; jj < nz * SITES; jj += THREADS) {
      const int j = z0 + jj / SITES, s = jj % SITES;
      const uint32_t zn = __ldg(zneed + j);
      const int pos = zn & 0x1fff, sl = (zn >> 13) & 1, i = zn >> 14;
      const int fam = sl == 0 ? g.fam0[gi] : g.fam1[gi];
      // F[a][e0][e1][e2] = sum_c2 D[e0][e1][c2] S_f2[(a,c2),e2]
      const cpx<R>* D = sD + s * nd + 432 * g.fam_dq[fam];
      const cpx<R>* S2 = sS + s * 288 + 144 * g.fam_f2[fam];
      const int a = i / 1728 + g.spin0, r = i % 1728, e01 = r / 12, e2 = r % 12;
      cpx<R> acc(0, 0);
#pragma unroll
      for (int c2 = 0; c2 < 3; c2++) cmac(acc, D[e01 * 3 + c2], S2[(3 * a + c2) * 12 + e2]);
      sZ[s * zs + pos] = acc;
    }
    __syncthreads();
    const int r0 = g.first[gi], r1 = r0 + g.rows[gi];
    cpx<R>* out = blk + ((size_t)slot * V + site0) * n_out;
    for (int r = r0 + tid; r < r1; r += THREADS) {
      // the warp's 32 rows are one chunk: entry k of all of them is 128 contiguous bytes
      const int2 ch = __ldg(ell_chunk + g.chunk_first[gi] + ((r - r0) >> 5));
      const uint32_t* ep = ell + ch.x + ((r - r0) & 31);
      cpx<R> acc[SITES];
#pragma unroll
      for (int s = 0; s < SITES; s++) acc[s] = cpx<R>(0, 0);
      for (int k = 0; k < ch.y; k++) {
        const uint32_t e = __ldg(ep + 32 * k);  // padding: weight 0 at position 0
        // FP64 is bound by its narrow pipe: skip the padding's multiply-adds
        // there; the other types run them (no divergent branch)
        if constexpr (sizeof(R) == 8 && std::is_floating_point<R>::value)
          if ((e >> 16) == 0) continue;
        const R w = sW[((int)(int16_t)(e >> 16)) + 16];
        const int pos = e & 0xffffu;
#pragma unroll
        for (int s = 0; s < SITES; s++) {
          const cpx<R> z = sZ[s * zs + pos];
          acc[s].re = fma(w, z.re, acc[s].re);
          acc[s].im = fma(w, z.im, acc[s].im);
        }
      }
#pragma unroll
      for (int s = 0; s < SITES; s++) out[(size_t)s * n_out + r] = acc[s];
    }
    __syncthreads();
  }
}

// FP32 blocks from dense entry tuples (host tables: dense_build.cpp).  Per
// site: the propagators (16-byte loads) and the diquarks as above; then per
// group one thread forms the twelve e2 entries of a tuple (slot, a, e0 e1),
// F[e2] = sum_c2 D[e0 e1][c2] S_f2[(a, c2)][e2], with the three diquark values
// in registers and the propagator row shared by the warp (consecutive tuples
// mostly share (slot, a): broadcast loads), writing entry (j, e2) to position
// e2 * stride + j (contiguous stores); the rows then sum their terms, weight
// = the top 16 bits of the table entry read as an FP32 value.
template <int SITES, int THREADS>
__global__ void __launch_bounds__(THREADS)
k_block_build_dense(const cpx<float>* __restrict__ prop, int V, const int2* __restrict__ ell_chunk,
                    const uint32_t* __restrict__ ell, const uint32_t* __restrict__ tuples, DevGroups g,
                    cpx<float>* __restrict__ blk, int n_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int kThreads = THREADS;
  const int nd = g.n_dq * 432, zs = g.dense_z_slots;
  cpx<float>* sS = reinterpret_cast<cpx<float>*>(smem_raw);  // [SITES][2][144]  light, strange
  cpx<float>* sD = sS + SITES * 288;                          // [SITES][n_dq][432]
  cpx<float>* sZ = sD + SITES * nd;                           // [SITES][zs]
  const int site0 = blockIdx.x * SITES, slot = blockIdx.y, tid = threadIdx.x;
  {
    const float4* P4 = reinterpret_cast<const float4*>(prop + (size_t)slot * 2 * V * 144);
    for (int i = tid; i < SITES * 144; i += kThreads) {  // 72 16-byte loads per site and flavour
      const int s = i / 144, j = i - 144 * s, f = j / 72, w = j - 72 * f;
      reinterpret_cast<float4*>(sS + s * 288 + f * 144)[w] = __ldg(P4 + ((size_t)f * V + site0 + s) * 72 + w);
    }
  }
  __syncthreads();
  for (int ii = tid; ii < SITES * nd; ii += kThreads) {
    const int s = ii / nd, i = ii - s * nd;
    const int dq = i / 432, r = i % 432, e0 = r / 36, e1 = (r / 3) % 12, c2 = r % 3;
    const int ca = (c2 + 1) % 3, cb = (c2 + 2) % 3;  // eps(ca,cb,c2) = +1, eps(cb,ca,c2) = -1
    const cpx<float>* S0 = sS + s * 288 + 144 * g.dq_f0[dq];
    const cpx<float>* S1 = sS + s * 288 + 144 * g.dq_f1[dq];
    const int gam = g.dq_gam[dq];
    cpx<float> acc(0.f, 0.f);
#pragma unroll
    for (int gi = 0; gi < 4; gi++) {
      const int a0 = c_gam[gam][gi][0], a1 = c_gam[gam][gi][1];
      const float sg = (float)c_gam[gam][gi][2];
      cpx<float> t(0.f, 0.f);
      cmac(t, S0[(3 * a0 + ca) * 12 + e0], S1[(3 * a1 + cb) * 12 + e1]);
      cpx<float> u(0.f, 0.f);
      cmac(u, S0[(3 * a0 + cb) * 12 + e0], S1[(3 * a1 + ca) * 12 + e1]);
      acc.re += sg * (t.re - u.re);
      acc.im += sg * (t.im - u.im);
    }
    sD[ii] = acc;
  }
  __syncthreads();
  for (int gi = 0; gi < g.n; gi++) {
    const int t0 = g.tuple_first[gi], nt = g.tuple_first[gi + 1] - t0, str = g.stride[gi];
    for (int jj = tid; jj < nt * SITES; jj += kThreads) {
      const int s = jj / nt, j = jj - s * nt;
      const uint32_t tu = __ldg(tuples + t0 + j);
      const int sl = tu / 288, a = (tu % 288) / 144, e01 = tu % 144;
      const int fam = sl == 0 ? g.fam0[gi] : g.fam1[gi];
      const cpx<float>* D = sD + s * nd + 432 * g.fam_dq[fam] + 3 * e01;
      const cpx<float>* S2 = sS + s * 288 + 144 * g.fam_f2[fam] + 36 * (a + g.spin0);
      const cpx<float> d0 = D[0], d1 = D[1], d2 = D[2];
      cpx<float>* z = sZ + s * zs + j;
#pragma unroll
      for (int e2 = 0; e2 < 12; e2++) {
        cpx<float> acc(0.f, 0.f);
        cmac(acc, d0, S2[e2]);
        cmac(acc, d1, S2[12 + e2]);
        cmac(acc, d2, S2[24 + e2]);
        z[e2 * str] = acc;
      }
    }
    __syncthreads();
    const int r0 = g.first[gi], r1 = r0 + g.rows[gi];
    cpx<float>* out = blk + ((size_t)slot * V + site0) * n_out;
    for (int r = r0 + tid; r < r1; r += kThreads) {
      cpx<float> acc[SITES];
#pragma unroll
      for (int s = 0; s < SITES; s++) acc[s] = cpx<float>(0.f, 0.f);
      const int2 ch = __ldg(ell_chunk + g.dchunk_first[gi] + ((r - r0) >> 5));
      const uint32_t* ep = ell + ch.x + ((r - r0) & 31);
      for (int k = 0; k < ch.y; k++) {
        const uint32_t e = __ldg(ep + 32 * k);  // padding: weight 0 at position 0
        const float w = __uint_as_float(e & 0xffff0000u);
        const int pos = e & 0xffffu;
#pragma unroll
        for (int s = 0; s < SITES; s++) {
          const cpx<float> zv = sZ[s * zs + pos];
          acc[s].re = fmaf(w, zv.re, acc[s].re);
          acc[s].im = fmaf(w, zv.im, acc[s].im);
        }
      }
#pragma unroll
      for (int s = 0; s < SITES; s++) out[(size_t)s * n_out + r] = acc[s];
    }
    __syncthreads();
  }
}

bool dense_build_supported(int sites, int threads) {
  return (threads == 256 || threads == 512) && (sites == 1 || sites == 2);
}

size_t dense_build_smem(const DevGroups& g, int sites) {
  return (size_t)sites * (288 + 432 * (size_t)g.n_dq + g.dense_z_slots) * sizeof(cpx<float>);
}

template <int SITES, int THREADS>
cudaError_t launch_dense_variant(const void* prop, int V, int n_slots, const int2* ell_chunk, const uint32_t* ell,
                                 const uint32_t* tuples, const DevGroups& g, void* blk, int n_out, cudaStream_t st) {
  const size_t sm = dense_build_smem(g, SITES);
  static int granted[64] = {0};
  cudaError_t e = ensure_smem(k_block_build_dense<SITES, THREADS>, sm, granted);
  if (e != cudaSuccess) return e;
  dim3 grid(V / SITES, n_slots);
  k_block_build_dense<SITES, THREADS><<<grid, THREADS, sm, st>>>((const cpx<float>*)prop, V, ell_chunk, ell,
                                                                 tuples, g, (cpx<float>*)blk, n_out);
  return cudaGetLastError();
}

cudaError_t launch_block_build_dense(const void* prop, int V, int n_slots, const int2* ell_chunk, const uint32_t* ell,
                                     const uint32_t* tuples, const DevGroups& g, void* blk, int n_out, cudaStream_t st,
                                     int sites, int threads) {
  if (!dense_build_supported(sites, threads) || V % sites != 0 || g.n_dq < 1 || g.n_dq > kMaxDiquarks ||
      dense_build_smem(g, sites) > kMaxSmemPerBlock)
    return cudaErrorInvalidValue;
  if (sites == 1 && threads == 256)
    return launch_dense_variant<1, 256>(prop, V, n_slots, ell_chunk, ell, tuples, g, blk, n_out, st);
  if (sites == 1) return launch_dense_variant<1, 512>(prop, V, n_slots, ell_chunk, ell, tuples, g, blk, n_out, st);
  if (threads == 256)
    return launch_dense_variant<2, 256>(prop, V, n_slots, ell_chunk, ell, tuples, g, blk, n_out, st);
  return launch_dense_variant<2, 512>(prop, V, n_slots, ell_chunk, ell, tuples, g, blk, n_out, st);
}

size_t block_build_smem(int z_slots, int sites, bool fp64, int n_dq) {  // fp64: 8-byte reals (FP64 or double-float)
  const size_t cb = fp64 ? sizeof(cpx<double>) : sizeof(cpx<float>);
  return (size_t)sites * (288 + 432 * (size_t)n_dq + z_slots) * cb + 32 * (fp64 ? sizeof(double) : sizeof(float));
}

bool build_variant_supported(int sites, int threads) {
  return (sites == 1 && (threads == 256 || threads == 512)) || (sites == 2 && (threads == 256 || threads == 512)) ||
         (sites == 4 && threads == 512);
}

template <typename R, int SITES, int THREADS>
cudaError_t launch_build_variant(const void* prop, int V, int n_slots, const int2* ell_chunk, const uint32_t* ell,
                                 const uint32_t* zneed, const DevGroups& g, void* blk, int n_out, cudaStream_t st) {
  const size_t sm = block_build_smem(g.z_slots, SITES, sizeof(R) == 8, g.n_dq);  // double or double-float
  static int granted[64] = {0};
  cudaError_t e = ensure_smem(k_block_build<R, SITES, THREADS>, sm, granted);
  if (e != cudaSuccess) return e;
  dim3 grid(V / SITES, n_slots);
  k_block_build<R, SITES, THREADS><<<grid, THREADS, sm, st>>>((const cpx<R>*)prop, V, ell_chunk, ell, zneed, g,
                                                              (cpx<R>*)blk, n_out);
  return cudaGetLastError();
}

cudaError_t launch_block_build(const void* prop, int V, int n_slots, const int2* ell_chunk,
                               const uint32_t* ell, const uint32_t* zneed, const DevGroups& g, void* blk,
                               int n_out, int kind, cudaStream_t st, int sites, int threads) {
  const bool wide = kind != RK_F32;
  if (!build_variant_supported(sites, threads) || V % sites != 0 || g.n_dq < 1 || g.n_dq > kMaxDiquarks ||
      block_build_smem(g.z_slots, sites, wide, g.n_dq) > kMaxSmemPerBlock)
    return cudaErrorInvalidValue;
#define BBC_BUILD(S, T)                                                                                            \
  if (sites == S && threads == T)                                                                                  \
    return kind == RK_F64 ? launch_build_variant<double, S, T>(prop, V, n_slots, ell_chunk, ell, zneed, g, blk, n_out, st) \
         : kind == RK_DF  ? launch_build_variant<dfr, S, T>(prop, V, n_slots, ell_chunk, ell, zneed, g, blk, n_out, st)    \
                          : launch_build_variant<float, S, T>(prop, V, n_slots, ell_chunk, ell, zneed, g, blk, n_out, st);
  BBC_BUILD(1, 256) BBC_BUILD(2, 256) BBC_BUILD(2, 512) BBC_BUILD(4, 512) BBC_BUILD(1, 512)
#undef BBC_BUILD
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------ checks
// *flag |= 1 if any of the n doubles is not finite.
__global__ void k_nonfinite(const double* __restrict__ x, long long n, int* flag) {
  int bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    bad |= !isfinite(x[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

cudaError_t launch_nonfinite(const double* x, long long n, int* flag, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)std::min<long long>((n + 255) / 256, 152 * 8);
  k_nonfinite<<<blocks, 256, 0, st>>>(x, n, flag);
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
