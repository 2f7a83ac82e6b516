// tc_contract.cu -- the block-pair products of the trace form on the tensor
// cores (mixed precisions): one complex matrix product per pair {q, -q},
//
//   G(q)[i][j] = sum_{u,v} M_i(q)[u][v] M_j(-q)[v][u]      (G(-q) = G(q)^T),
//
// over the 12 x 12 open-index matrices M of the blocks that such tasks read
// (Sec. 3 Eq. LN.pLLp.FFT: sum over the open colour and spin indices of
// A(q) B(-q); the host split is in tensor_split.cpp).
//
// One CTA per pair {q, -q}.  The q row of every block is staged as X[i][k]
// = M_i(q)[u][v] and the -q row transposed, Y[j][k] = M_j(-q)[v][u] (k =
// 12 u + v), so that G = X Y^T over k = 0..143.  A warp owns one 16-row
// m-tile and up to three 8-column n-tiles of G and runs the complex product
// as four real products (Gr += Xr Yr - Xi Yi, Gi += Xr Yi + Xi Yr) with
// mma.sync m16n8k8 on TF32 operands and FP32 accumulators.  FP32 accuracy
// (kTc3x) comes from splitting every operand into two TF32 words, x = hi +
// lo, and summing hi lo + lo hi + hi hi (the products the TF32 rounding of
// one word would drop); the TF32 trial (kTc1x) rounds every operand once.
// Rows are padded to 148 complex (1184 bytes): the fragment loads of a warp
// (rows g, columns t) then fall in distinct shared-memory banks.
#include "device_common.cuh"

namespace bbc {

namespace {

constexpr int kLd = 148;     // staged row stride in complex (144 + 4)
constexpr int kChunks = 72;  // 16-byte chunks of one block row (144 complex64)

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// x = hi + lo, both TF32 (hi the nearest TF32 value, lo the rounded rest)
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(__fsub_rn(x, __uint_as_float(hi)));
}

// d += a b, m16n8k8, A row-major (16 x 8), B column-major (8 x 8), TF32 in, FP32 accumulate
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t neg(uint32_t x) { return x ^ 0x80000000u; }

}  // namespace

template <int MODE>
__global__ void __launch_bounds__(kTcMaxWarps * 32)
k_contract_tc(const float2* __restrict__ blk, int L, int n_out, const int* __restrict__ base, int nb, int nbp,
              const int* __restrict__ qlist, const int* __restrict__ units, int n_units, float2* __restrict__ G) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* X = reinterpret_cast<float2*>(smem_raw);  // [nbp][kLd]  M_i(q)[u][v] at 12 u + v
  float2* Y = X + (size_t)nbp * kLd;                // [nbp][kLd]  M_j(-q)[v][u] at 12 u + v
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int p = blockIdx.x, q = qlist[p];
  const int qx = q % L, qy = (q / L) % L, qz = q / (L * L);
  const int nq = (L - qx) % L + L * ((L - qy) % L + L * ((L - qz) % L));
  const float4* rq = reinterpret_cast<const float4*>(blk + (size_t)q * n_out);
  const float4* rmq = reinterpret_cast<const float4*>(blk + (size_t)nq * n_out);
  // rows nb .. nbp-1 are padding: zero (they enter G's unread rows and columns only)
  for (int i = nb * kLd + tid; i < nbp * kLd; i += nthr) {
    X[i] = make_float2(0.f, 0.f);
    Y[i] = make_float2(0.f, 0.f);
  }
  // staging: six 16-byte loads in flight per thread before their stores
  constexpr int U = 6;
  const int n_chunks = nb * kChunks;
  for (int c0 = tid; c0 < 2 * n_chunks; c0 += U * nthr) {
    float4 v[U];
#pragma unroll
    for (int s = 0; s < U; s++) {
      const int c = c0 + s * nthr;
      if (c < 2 * n_chunks) {
        const int side = c >= n_chunks, cc = side ? c - n_chunks : c;
        const int b = cc / kChunks, w = cc - b * kChunks;
        v[s] = __ldg((side ? rmq : rq) + (base[b] >> 1) + w);
      }
    }
#pragma unroll
    for (int s = 0; s < U; s++) {
      const int c = c0 + s * nthr;
      if (c < 2 * n_chunks) {
        const int side = c >= n_chunks, cc = side ? c - n_chunks : c;
        const int b = cc / kChunks, w = cc - b * kChunks;
        if (!side) {
          reinterpret_cast<float4*>(X + (size_t)b * kLd)[w] = v[s];
        } else {  // elements e = 2w, 2w + 1 of M_b(-q): (u, v) and (u, v + 1) -> k = 12 v + u
          const int e = 2 * w, u = e / 12, vv = e - 12 * u;
          Y[(size_t)b * kLd + 12 * vv + u] = make_float2(v[s].x, v[s].y);
          Y[(size_t)b * kLd + 12 * (vv + 1) + u] = make_float2(v[s].z, v[s].w);
        }
      }
    }
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  if (warp >= n_units) return;
  const int un = units[warp], mt = un & 0xff, nt0 = (un >> 8) & 0xff, cnt = un >> 16;
  float dr[kTcTilesPerWarp][4], di[kTcTilesPerWarp][4];
#pragma unroll
  for (int n = 0; n < kTcTilesPerWarp; n++)
#pragma unroll
    for (int i = 0; i < 4; i++) dr[n][i] = di[n][i] = 0.f;
  const float2* xa = X + (size_t)(16 * mt + g) * kLd + t;
  const float2* yb = Y + (size_t)(8 * nt0 + g) * kLd + t;
#pragma unroll 2
  for (int k0 = 0; k0 < 144; k0 += 8) {
    // A fragment: (g, t), (g + 8, t), (g, t + 4), (g + 8, t + 4)
    const float2 x[4] = {xa[k0], xa[8 * kLd + k0], xa[k0 + 4], xa[8 * kLd + k0 + 4]};
    uint32_t arh[4], arl[4], aih[4], ail[4], naih[4], nail[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
      if (MODE == kTc3x) {
        split_tf32(x[i].x, arh[i], arl[i]);
        split_tf32(x[i].y, aih[i], ail[i]);
        nail[i] = neg(ail[i]);
      } else {
        arh[i] = tf32_rna(x[i].x);
        aih[i] = tf32_rna(x[i].y);
      }
      naih[i] = neg(aih[i]);
    }
#pragma unroll
    for (int n = 0; n < kTcTilesPerWarp; n++) {
      if (n >= cnt) break;
      // B fragment: (k = t, col g), (k = t + 4, col g)
      const float2 y0 = yb[(size_t)8 * n * kLd + k0], y1 = yb[(size_t)8 * n * kLd + k0 + 4];
      uint32_t brh[2], brl[2], bih[2], bil[2];
      if (MODE == kTc3x) {
        split_tf32(y0.x, brh[0], brl[0]);
        split_tf32(y1.x, brh[1], brl[1]);
        split_tf32(y0.y, bih[0], bil[0]);
        split_tf32(y1.y, bih[1], bil[1]);
        // small terms first
        mma_tf32(dr[n], arl, brh); mma_tf32(dr[n], arh, brl); mma_tf32(dr[n], arh, brh);
        mma_tf32(dr[n], nail, bih); mma_tf32(dr[n], naih, bil); mma_tf32(dr[n], naih, bih);
        mma_tf32(di[n], arl, bih); mma_tf32(di[n], arh, bil); mma_tf32(di[n], arh, bih);
        mma_tf32(di[n], ail, brh); mma_tf32(di[n], aih, brl); mma_tf32(di[n], aih, brh);
      } else {
        brh[0] = tf32_rna(y0.x); brh[1] = tf32_rna(y1.x);
        bih[0] = tf32_rna(y0.y); bih[1] = tf32_rna(y1.y);
        mma_tf32(dr[n], arh, brh); mma_tf32(dr[n], naih, bih);
        mma_tf32(di[n], arh, bih); mma_tf32(di[n], aih, brh);
      }
    }
  }
  // D fragment: (g, 2t), (g, 2t + 1), (g + 8, 2t), (g + 8, 2t + 1); G[p][m][n] complex64
  float4* Gp = reinterpret_cast<float4*>(G + (size_t)p * nbp * nbp);
#pragma unroll
  for (int n = 0; n < kTcTilesPerWarp; n++) {
    if (n >= cnt) break;
    const int col = 8 * (nt0 + n) + 2 * t, m0 = 16 * mt + g;
    Gp[((size_t)m0 * nbp + col) >> 1] = make_float4(dr[n][0], di[n][0], dr[n][1], di[n][1]);
    Gp[((size_t)(m0 + 8) * nbp + col) >> 1] = make_float4(dr[n][2], di[n][2], dr[n][3], di[n][3]);
  }
}

size_t contract_tc_smem(int nbp) { return (size_t)2 * nbp * kLd * sizeof(float2); }

cudaError_t launch_contract_tc(const void* blk, int L, int n_out, const int* base, int nb, int nbp, const int* qlist,
                               int n_q, const int* units, int n_units, void* G, int mode, cudaStream_t st) {
  if (n_q == 0) return cudaSuccess;
  if (nb < 1 || nb > nbp || nbp % 16 || nbp > kMaxTcBlocks || n_units < 1 || n_units > kTcMaxWarps || (n_out & 1))
    return cudaErrorInvalidValue;
  const size_t sm = contract_tc_smem(nbp);
  static int granted[2][64] = {{0}};
  cudaError_t e;
  if (mode == kTc3x) {
    e = ensure_smem(k_contract_tc<kTc3x>, sm, granted[0]);
    if (e != cudaSuccess) return e;
    k_contract_tc<kTc3x><<<n_q, n_units * 32, sm, st>>>((const float2*)blk, L, n_out, base, nb, nbp, qlist, units,
                                                        n_units, (float2*)G);
  } else {
    e = ensure_smem(k_contract_tc<kTc1x>, sm, granted[1]);
    if (e != cudaSuccess) return e;
    k_contract_tc<kTc1x><<<n_q, n_units * 32, sm, st>>>((const float2*)blk, L, n_out, base, nb, nbp, qlist, units,
                                                        n_units, (float2*)G);
  }
  return cudaGetLastError();
}

}  // namespace bbc
