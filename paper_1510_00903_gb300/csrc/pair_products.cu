// pair_products.cu -- FP64 q-space contraction: block-pair products with one q per lane, signed FP64 sums over Wick diagrams (Sec. 3 Eq. LN.pLLp.FFT)
#include <algorithm>
#include <cmath>
#include <utility>

#include "device_common.cuh"

namespace bbc {

// --------------------------------------------------------------- contract
// Pair products with one q per lane: a warp runs a fixed list of tasks for 32
// consecutive q (uniform control flow, coalesced loads from the field-major
// block storage), every nA x nB spin product of a task accumulated in
// registers over its open index; P[task*16 + rA*nB + rB][q] is stored for the
// signed sums.  FP64 with Fs: the sums re + im of every value come from the
// plane the forward FFT wrote (the same FP64 additions, made once per value
// instead of once per use), so each complex multiply-add is three FMAs.
template <typename R, int NA, int NB, bool SUMS>
__device__ __forceinline__ void task_products(const cpx<R>* __restrict__ F, const double* __restrict__ Fs,
                                              long long V, int q, int nq, const DevTask& t, cpx<R>* __restrict__ P) {
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
      if constexpr (SUMS) {
#pragma unroll
        for (int r = 0; r < NA; r++) {
          a[r] = F[(long long)(t.offA[r] + oA) * V + q];
          as[r] = __ldg(Fs + (long long)(t.offA[r] + oA) * V + q);
        }
#pragma unroll
        for (int r = 0; r < NB; r++) {
          b[r] = F[(long long)(t.offB[r] + oB) * V + nq];
          bs[r] = __ldg(Fs + (long long)(t.offB[r] + oB) * V + nq);
        }
      } else {
#pragma unroll
        for (int r = 0; r < NA; r++) { a[r] = F[(long long)(t.offA[r] + oA) * V + q]; as[r] = a[r].re + a[r].im; }
#pragma unroll
        for (int r = 0; r < NB; r++) { b[r] = F[(long long)(t.offB[r] + oB) * V + nq]; bs[r] = b[r].re + b[r].im; }
      }
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

template <typename R, bool SUMS>
__global__ void __launch_bounds__(32 * kPairWarps)
k_pair_products(const cpx<R>* __restrict__ F, const double* __restrict__ Fs, int L, const DevTask* __restrict__ tasks,
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
    if (nA == 4) task_products<R, 4, 4, SUMS>(F, Fs, V, q, nq, t, p);
    else if (nA == 2) task_products<R, 2, 8, SUMS>(F, Fs, V, q, nq, t, p);
    else task_products<R, 8, 2, SUMS>(F, Fs, V, q, nq, t, p);
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
                                 const int* group_task, int n_groups, void* P, bool fp64, cudaStream_t st,
                                 const double* blk_sum) {
  const int V = L * L * L;
  if (n_groups <= 0) return cudaSuccess;  // a plan whose products all vanish has no tasks
  dim3 g1((n_groups + kPairWarps - 1) / kPairWarps, (V + 31) / 32);
  if (fp64 && blk_sum)
    k_pair_products<double, true><<<g1, 32 * kPairWarps, 0, st>>>((const cpx<double>*)blk_field, blk_sum, L, tasks,
                                                                  group_ptr, group_task, n_groups, (cpx<double>*)P);
  else if (fp64)
    k_pair_products<double, false><<<g1, 32 * kPairWarps, 0, st>>>((const cpx<double>*)blk_field, nullptr, L, tasks,
                                                                   group_ptr, group_task, n_groups, (cpx<double>*)P);
  else
    k_pair_products<float, false><<<g1, 32 * kPairWarps, 0, st>>>((const cpx<float>*)blk_field, nullptr, L, tasks,
                                                                  group_ptr, group_task, n_groups, (cpx<float>*)P);
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

}  // namespace bbc
