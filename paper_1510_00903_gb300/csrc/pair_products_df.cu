// pair_products_df.cu -- the q-space block-pair products of the FP64 path in
// double-float arithmetic (pairs of FP32 values) on the FP32 pipes: the same
// lanes-over-q design as pair_products.cu, FP64-accurate to about 2^-44.
#include "device_common.cuh"

namespace bbc {

constexpr int kPairWarpsDf = 4;
constexpr int kDfStages = 2;      // open-index steps of rows in flight per lane
constexpr int kDfMaxRows = 10;    // nA + nB of the widest task shape (2 x 8, 8 x 2)

// Double-float variant: the Fourier-space blocks as (re.hi, re.lo, im.hi,
// im.lo) FP32 quadruples (from the double-float forward FFT), every complex
// product as four double-float multiply-adds on the FP32 pipes, accumulators
// renormalised every 16 open-index steps, the products stored as
// double-float pairs for the double-float Wick sums.
//
// The rows of an open-index step reach the lane through a ring of kDfStages
// shared-memory stages filled by cp.async: while the lane multiplies step k,
// the rows of step k + 1 are on their way, so the L2 and DRAM latency of the
// row loads overlaps the arithmetic instead of stalling it.  A lane reads
// only the 16-byte slots it copied itself (slot [stage][row][lane]), so the
// ring needs no barrier, and the 32 lanes' slots of one row are contiguous
// (conflict-free 128-bit shared loads).
template <int NA, int NB>
struct DfRows {
  static constexpr int NR = NA + NB;
  const float4* F;
  long long V;
  int q, nq;
  int i1, i2, oA, oB;  // open-index position of the next step to fetch
  // rows of the next step into stage `st` of this lane's ring, then advance
  __device__ __forceinline__ void fetch(const DevTask& t, float4* ring, int st) {
    float4* dst = ring + st * NR * 32;
#pragma unroll
    for (int r = 0; r < NA; r++) cp_async16(dst + r * 32, F + (long long)(t.offA[r] + oA) * V + q);
#pragma unroll
    for (int r = 0; r < NB; r++) cp_async16(dst + (NA + r) * 32, F + (long long)(t.offB[r] + oB) * V + nq);
    if (++i2 == t.n2) {
      i2 = 0;
      ++i1;
      oA = i1 * (t.sA & 0xffff);
      oB = i1 * (t.sB & 0xffff);
    } else {
      oA += t.sA >> 16;
      oB += t.sB >> 16;
    }
  }
};

// SWAPPED: t is a 2 x 8 task with its two sides exchanged (see the kernel):
// product (ra', rb') of the swapped task is product (rb', ra') of the
// original, and the P pointer is at -q.
template <int NA, int NB, bool SWAPPED = false>
__device__ __forceinline__ void task_products_df(const float4* __restrict__ F, long long V, int q, int nq,
                                                 const DevTask& t, cpx<dfr>* __restrict__ P, float4* ring) {
  constexpr int NR = NA + NB;
  const int K = t.n1 * t.n2;
  DfRows<NA, NB> rows{F, V, q, nq, 0, 0, 0, 0};
  df64acc re[NA * NB], im[NA * NB];
#pragma unroll
  for (int i = 0; i < NA * NB; i++) { re[i] = df64acc{0.f, 0.f}; im[i] = df64acc{0.f, 0.f}; }
#pragma unroll
  for (int s = 0; s < kDfStages; s++) {
    if (s < K) rows.fetch(t, ring, s);
    cp_async_commit();
  }
  for (int k = 0; k < K; k++) {
    const int st = k % kDfStages;
    cp_async_wait_group<kDfStages - 1>();  // the rows of step k have landed
    const float4* src = ring + st * NR * 32;
    float4 b[NB];  // (re.hi, re.lo, im.hi, im.lo)
#pragma unroll
    for (int r = 0; r < NB; r++) b[r] = src[(NA + r) * 32];
#pragma unroll
    for (int ra = 0; ra < NA; ra++) {
      const float4 a = src[ra * 32];
#pragma unroll
      for (int rb = 0; rb < NB; rb++) {
        const int i = ra * NB + rb;
        df_mac(re[i], a.x, a.y, b[rb].x, b[rb].y);    // + Re a Re b
        df_mac(re[i], -a.z, -a.w, b[rb].z, b[rb].w);  // - Im a Im b
        df_mac(im[i], a.x, a.y, b[rb].z, b[rb].w);    // + Re a Im b
        df_mac(im[i], a.z, a.w, b[rb].x, b[rb].y);    // + Im a Re b
      }
    }
    if ((k & 15) == 15) {
#pragma unroll
      for (int i = 0; i < NA * NB; i++) { df_renorm(re[i]); df_renorm(im[i]); }
    }
    // the stage just read takes the rows of step k + kDfStages (an empty
    // group past the end keeps the group count in step)
    if (k + kDfStages < K) rows.fetch(t, ring, st);
    cp_async_commit();
  }
#pragma unroll
  for (int i = 0; i < NA * NB; i++) {
    df_renorm(re[i]);
    df_renorm(im[i]);
    const int o = SWAPPED ? (i % NB) * NA + i / NB : i;
    P[(long long)o * V] = cpx<dfr>(dfr(re[i].s, re[i].e), dfr(im[i].s, im[i].e));
  }
}

__global__ void __launch_bounds__(32 * kPairWarpsDf, 4)
k_pair_products_df(const float4* __restrict__ F, int L, const DevTask* __restrict__ tasks,
                   const int* __restrict__ group_ptr, const int* __restrict__ group_task, int n_groups,
                   cpx<dfr>* __restrict__ P) {
  extern __shared__ float4 df_ring[];  // [warp][kDfStages][kDfMaxRows][32]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = blockIdx.x * kPairWarpsDf + warp;
  const int V = L * L * L;
  const int q = blockIdx.y * 32 + lane;
  if (g >= n_groups || q >= V) return;
  float4* ring = df_ring + warp * kDfStages * kDfMaxRows * 32 + lane;
  const int qx = q % L, qy = (q / L) % L, qz = q / (L * L);
  const int nq = (L - qx) % L + L * ((L - qy) % L + L * ((L - qz) % L));
  const int j1 = group_ptr[g + 1];
  for (int j = group_ptr[g]; j < j1; j++) {
    const int ti = group_task[j];
    const DevTask t = tasks[ti];
    const int nA = t.nAnB & 0xff;
    if (nA == 4) {
      task_products_df<4, 4>(F, V, q, nq, t, P + (long long)ti * 16 * V + q, ring);
    } else if (nA == 8) {
      task_products_df<8, 2>(F, V, q, nq, t, P + (long long)ti * 16 * V + q, ring);
    } else {
      // a 2 x 8 task runs on the 8 x 2 code (one unrolled body less): sum_k
      // B(q; k) A(-q; k) is the task's product at -q, transposed, so the lane
      // reads B at q and A at -q and stores at -q
      DevTask s = t;
      for (int r = 0; r < 8; r++) {
        s.offA[r] = t.offB[r];
        s.offB[r] = r < 2 ? t.offA[r] : 0;
      }
      s.nAnB = 8 | (2 << 8);
      s.sA = t.sB;
      s.sB = t.sA;
      task_products_df<8, 2, true>(F, V, q, nq, s, P + (long long)ti * 16 * V + nq, ring);
    }
  }
}

cudaError_t launch_pair_products_df(const void* blk_field, int L, const DevTask* tasks, const int* group_ptr,
                                    const int* group_task, int n_groups, void* P, cudaStream_t st) {
  const int V = L * L * L;
  if (n_groups <= 0) return cudaSuccess;  // a plan whose products all vanish has no tasks
  constexpr size_t sm = sizeof(float4) * kPairWarpsDf * kDfStages * kDfMaxRows * 32;
  static_assert(sm <= 48 * 1024, "the ring fits the default dynamic shared-memory limit");
  dim3 g1((n_groups + kPairWarpsDf - 1) / kPairWarpsDf, (V + 31) / 32);
  k_pair_products_df<<<g1, 32 * kPairWarpsDf, sm, st>>>((const float4*)blk_field, L, tasks, group_ptr, group_task,
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
