// pair_products_df.cu -- the q-space block-pair products of the FP64 path in
// double-float arithmetic (pairs of FP32 values) on the FP32 pipes: the same
// lanes-over-q design as pair_products.cu, FP64-accurate to about 2^-44.
#include "device_common.cuh"

namespace bbc {

constexpr int kPairWarpsDf = 4;

// Double-float variant: the Fourier-space blocks as (re.hi, re.lo, im.hi,
// im.lo) FP32 quadruples (from the double-float forward FFT), every complex
// product as four double-float multiply-adds on the FP32 pipes, accumulators
// renormalised every 16 open-index steps, the products stored as
// double-float pairs for the double-float Wick sums.
template <int NA, int NB>
__device__ __forceinline__ void task_products_df(const float4* __restrict__ F, long long V, int q, int nq,
                                                 const DevTask& t, cpx<dfr>* __restrict__ P) {
  const int n2 = t.n2, K = t.n1 * n2;
  const int sA1 = t.sA & 0xffff, sA2 = t.sA >> 16, sB1 = t.sB & 0xffff, sB2 = t.sB >> 16;
  df64acc re[NA * NB], im[NA * NB];
#pragma unroll
  for (int i = 0; i < NA * NB; i++) { re[i] = df64acc{0.f, 0.f}; im[i] = df64acc{0.f, 0.f}; }
  int i1 = 0, i2 = 0, oA = 0, oB = 0;
  for (int k = 0; k < K; k++) {
    float4 a[NA], b[NB];  // (re.hi, re.lo, im.hi, im.lo)
#pragma unroll
    for (int r = 0; r < NA; r++) a[r] = F[(long long)(t.offA[r] + oA) * V + q];
#pragma unroll
    for (int r = 0; r < NB; r++) b[r] = F[(long long)(t.offB[r] + oB) * V + nq];
#pragma unroll
    for (int ra = 0; ra < NA; ra++)
#pragma unroll
      for (int rb = 0; rb < NB; rb++) {
        const int i = ra * NB + rb;
        df_mac(re[i], a[ra].x, a[ra].y, b[rb].x, b[rb].y);    // + Re a Re b
        df_mac(re[i], -a[ra].z, -a[ra].w, b[rb].z, b[rb].w);  // - Im a Im b
        df_mac(im[i], a[ra].x, a[ra].y, b[rb].z, b[rb].w);    // + Re a Im b
        df_mac(im[i], a[ra].z, a[ra].w, b[rb].x, b[rb].y);    // + Im a Re b
      }
    if ((k & 15) == 15) {
#pragma unroll
      for (int i = 0; i < NA * NB; i++) { df_renorm(re[i]); df_renorm(im[i]); }
    }
    if (++i2 == n2) { i2 = 0; ++i1; oA = i1 * sA1; oB = i1 * sB1; }
    else { oA += sA2; oB += sB2; }
  }
#pragma unroll
  for (int i = 0; i < NA * NB; i++) {
    df_renorm(re[i]);
    df_renorm(im[i]);
    P[(long long)i * V] = cpx<dfr>(dfr(re[i].s, re[i].e), dfr(im[i].s, im[i].e));
  }
}

__global__ void __launch_bounds__(32 * kPairWarpsDf, 4)
k_pair_products_df(const float4* __restrict__ F, int L, const DevTask* __restrict__ tasks,
                   const int* __restrict__ group_ptr, const int* __restrict__ group_task, int n_groups,
                   cpx<dfr>* __restrict__ P) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = blockIdx.x * kPairWarpsDf + warp;
  const int V = L * L * L;
  const int q = blockIdx.y * 32 + lane;
  if (g >= n_groups || q >= V) return;
  const int qx = q % L, qy = (q / L) % L, qz = q / (L * L);
  const int nq = (L - qx) % L + L * ((L - qy) % L + L * ((L - qz) % L));
  const int j1 = group_ptr[g + 1];
  for (int j = group_ptr[g]; j < j1; j++) {
    const int ti = group_task[j];
    const DevTask t = tasks[ti];
    cpx<dfr>* p = P + (long long)ti * 16 * V + q;
    const int nA = t.nAnB & 0xff;
    if (nA == 4) task_products_df<4, 4>(F, V, q, nq, t, p);
    else if (nA == 2) task_products_df<2, 8>(F, V, q, nq, t, p);
    else task_products_df<8, 2>(F, V, q, nq, t, p);
  }
}

cudaError_t launch_pair_products_df(const void* blk_field, int L, const DevTask* tasks, const int* group_ptr,
                                    const int* group_task, int n_groups, void* P, cudaStream_t st) {
  const int V = L * L * L;
  if (n_groups <= 0) return cudaSuccess;  // a plan whose products all vanish has no tasks
  dim3 g1((n_groups + kPairWarpsDf - 1) / kPairWarpsDf, (V + 31) / 32);
  k_pair_products_df<<<g1, 32 * kPairWarpsDf, 0, st>>>((const float4*)blk_field, L, tasks, group_ptr, group_task,
                                                       n_groups, (cpx<dfr>*)P);
  return cudaGetLastError();
}

// Signed sums over Wick diagrams in double-float arithmetic: the products and
// the coefficients (split once on the host) as double-float pairs, every
// term one double-float multiply-add per real part; ct stored as
// double-float pairs for the double-float inverse transform.
__global__ void __launch_bounds__(128)
k_wick_sums_df(const cpx<dfr>* __restrict__ P, int V, const int* __restrict__ cptr, const int* __restrict__ citem,
               const float2* __restrict__ ccoef, cpx<dfr>* __restrict__ Ct) {
  const int q = blockIdx.x * 128 + threadIdx.x, o = blockIdx.y;
  if (q >= V) return;
  df64acc re{0.f, 0.f}, im{0.f, 0.f};
  const int c1 = cptr[o + 1];
  for (int c = cptr[o]; c < c1; c++) {
    const float2 w = __ldg(ccoef + c);
    const cpx<dfr> p = P[(long long)citem[c] * V + q];
    df_mac(re, w.x, w.y, p.re.hi, p.re.lo);
    df_mac(im, w.x, w.y, p.im.hi, p.im.lo);
    if (((c - cptr[o]) & 15) == 15) { df_renorm(re); df_renorm(im); }
  }
  df_renorm(re);
  df_renorm(im);
  Ct[(long long)o * V + q] = cpx<dfr>(dfr(re.s, re.e), dfr(im.s, im.e));
}

cudaError_t launch_wick_sums_df(const void* P, int L, const int* cptr, const int* citem, const float2* ccoef_df,
                                int n_ch, void* ct, cudaStream_t st) {
  const int V = L * L * L;
  dim3 g2((V + 127) / 128, n_ch * 16);
  k_wick_sums_df<<<g2, 128, 0, st>>>((const cpx<dfr>*)P, V, cptr, citem, ccoef_df, (cpx<dfr>*)ct);
  return cudaGetLastError();
}

}  // namespace bbc
