// pair_products_df.cu -- the q-space block-pair products of the FP64 path in
// double-float arithmetic (pairs of FP32 values) on the FP32 pipes: the same
// lanes-over-q design as pair_products.cu, FP64-accurate to about 2^-44.
#include "device_common.cuh"

namespace bbc {

constexpr int kPairWarpsDf = 4;

// Double-float variant: the Fourier-space blocks as (re.hi, re.lo, im.hi,
// im.lo) FP32 quadruples (written by the last forward FFT pass), every
// complex product as four double-float multiply-adds on the FP32 pipes,
// accumulators renormalised every 16 open-index steps, the products stored
// as complex128 for the FP64 Wick sums.  Each task's 16 products run as two
// register tiles of 8.
// One register tile of a task: rows ra0 .. ra0+TA-1 of A against rows
// rb0 .. rb0+TB-1 of B (the task's full nA x nB products are split into two
// tiles, so a lane holds half the accumulators and more warps fit on an SM).
template <int TA, int TB>
__device__ __forceinline__ void tile_products_df(const float4* __restrict__ F, long long V, int q, int nq,
                                                 const DevTask& t, int nB, int ra0, int rb0,
                                                 cpx<double>* __restrict__ P) {
  const int n2 = t.n2, K = t.n1 * n2;
  const int sA1 = t.sA & 0xffff, sA2 = t.sA >> 16, sB1 = t.sB & 0xffff, sB2 = t.sB >> 16;
  int offA[TA], offB[TB];
#pragma unroll
  for (int r = 0; r < TA; r++) offA[r] = t.offA[ra0 + r];
#pragma unroll
  for (int r = 0; r < TB; r++) offB[r] = t.offB[rb0 + r];
  df64acc re[TA * TB], im[TA * TB];
#pragma unroll
  for (int i = 0; i < TA * TB; i++) { re[i] = df64acc{0.f, 0.f}; im[i] = df64acc{0.f, 0.f}; }
  int i1 = 0, i2 = 0, oA = 0, oB = 0;
  float4 a[TA], b[TB];  // (re.hi, re.lo, im.hi, im.lo) of step k; loads of step k + 1 are issued before its products
#pragma unroll
  for (int r = 0; r < TA; r++) a[r] = F[(long long)offA[r] * V + q];
#pragma unroll
  for (int r = 0; r < TB; r++) b[r] = F[(long long)offB[r] * V + nq];
  for (int k = 0; k < K; k++) {
    if (++i2 == n2) { i2 = 0; ++i1; oA = i1 * sA1; oB = i1 * sB1; }
    else { oA += sA2; oB += sB2; }
    float4 an[TA], bn[TB];
    const bool more = k + 1 < K;
#pragma unroll
    for (int r = 0; r < TA; r++) an[r] = more ? F[(long long)(offA[r] + oA) * V + q] : a[r];
#pragma unroll
    for (int r = 0; r < TB; r++) bn[r] = more ? F[(long long)(offB[r] + oB) * V + nq] : b[r];
#pragma unroll
    for (int ra = 0; ra < TA; ra++)
#pragma unroll
      for (int rb = 0; rb < TB; rb++) {
        const int i = ra * TB + rb;
        df_mac(re[i], a[ra].x, a[ra].y, b[rb].x, b[rb].y);    // + Re a Re b
        df_mac(re[i], -a[ra].z, -a[ra].w, b[rb].z, b[rb].w);  // - Im a Im b
        df_mac(im[i], a[ra].x, a[ra].y, b[rb].z, b[rb].w);    // + Re a Im b
        df_mac(im[i], a[ra].z, a[ra].w, b[rb].x, b[rb].y);    // + Im a Re b
      }
    if ((k & 15) == 15) {
#pragma unroll
      for (int i = 0; i < TA * TB; i++) { df_renorm(re[i]); df_renorm(im[i]); }
    }
#pragma unroll
    for (int r = 0; r < TA; r++) a[r] = an[r];
#pragma unroll
    for (int r = 0; r < TB; r++) b[r] = bn[r];
  }
#pragma unroll
  for (int ra = 0; ra < TA; ra++)
#pragma unroll
    for (int rb = 0; rb < TB; rb++)
      P[(long long)((ra0 + ra) * nB + rb0 + rb) * V] =
          cpx<double>(df_to_double(re[ra * TB + rb]), df_to_double(im[ra * TB + rb]));
}

__global__ void __launch_bounds__(32 * kPairWarpsDf, 4)
k_pair_products_df(const float4* __restrict__ F, int L, const DevTask* __restrict__ tasks,
                   const int* __restrict__ group_ptr, const int* __restrict__ group_task, int n_groups,
                   cpx<double>* __restrict__ P) {
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
    cpx<double>* p = P + (long long)ti * 16 * V + q;
    const int nA = t.nAnB & 0xff;
    if (nA == 4) {         // 4 x 4 as two 4 x 2 tiles
      tile_products_df<4, 2>(F, V, q, nq, t, 4, 0, 0, p);
      tile_products_df<4, 2>(F, V, q, nq, t, 4, 0, 2, p);
    } else if (nA == 2) {  // 2 x 8 as two 2 x 4 tiles
      tile_products_df<2, 4>(F, V, q, nq, t, 8, 0, 0, p);
      tile_products_df<2, 4>(F, V, q, nq, t, 8, 0, 4, p);
    } else {               // 8 x 2 as two 4 x 2 tiles
      tile_products_df<4, 2>(F, V, q, nq, t, 2, 0, 0, p);
      tile_products_df<4, 2>(F, V, q, nq, t, 2, 4, 0, p);
    }
  }
}

cudaError_t launch_pair_products_df(const void* blk_field, int L, const DevTask* tasks, const int* group_ptr,
                                    const int* group_task, int n_groups, void* P, cudaStream_t st) {
  const int V = L * L * L;
  dim3 g1((n_groups + kPairWarpsDf - 1) / kPairWarpsDf, (V + 31) / 32);
  k_pair_products_df<<<g1, 32 * kPairWarpsDf, 0, st>>>((const float4*)blk_field, L, tasks, group_ptr, group_task,
                                                       n_groups, (cpx<double>*)P);
  return cudaGetLastError();
}

}  // namespace bbc
