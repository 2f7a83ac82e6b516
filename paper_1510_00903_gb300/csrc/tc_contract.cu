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
// m-tile and up to TILES (2 or 3, tuned) 8-column n-tiles of G and runs the complex product
// as three real products (t1 = Xr Yr, t2 = Xi Yi, t3 = (Xr + Xi)(Yr + Yi);
// Gr = t1 - t2, Gi = t3 - t1 - t2) with mma.sync m16n8k8 on TF32 operands and
// FP32 accumulators.  FP32 accuracy (kTc3x) comes from splitting every
// operand into two TF32 words, x = hi + lo, and summing lo hi + hi lo + hi hi
// (the products the TF32 rounding of one word would drop); the TF32 trial
// (kTc1x) rounds every operand once.  The rows are staged with asynchronous
// copies (cp.async) in two groups by open-index half, so the second half
// lands while the first is multiplied.
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


}  // namespace

template <int MODE, int TILES>
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
  const float2* rq = blk + (size_t)q * n_out;
  const float2* rmq = blk + (size_t)nq * n_out;
  // rows nb .. nbp-1 are padding: zero (they enter G's unread rows and columns only)
  for (int i = nb * kLd + tid; i < nbp * kLd; i += nthr) {
    X[i] = make_float2(0.f, 0.f);
    Y[i] = make_float2(0.f, 0.f);
  }
  // staging with asynchronous copies, in two groups: k < 72 (rows u < 6 of
  // every X block, columns u < 6 of every Y block) first, then k >= 72, so
  // that the second half lands while the first half is multiplied.  X moves
  // in 16-byte chunks, Y element by element to its transposed place.
#pragma unroll
  for (int half = 0; half < 2; half++) {
    const int n_chunks = nb * (kChunks / 2);
#pragma unroll 4
    for (int c = tid; c < n_chunks; c += nthr) {
      const int b = c / (kChunks / 2), w = half * (kChunks / 2) + (c - b * (kChunks / 2));
      cp_async16(X + (size_t)b * kLd + 2 * w, rq + base[b] + 2 * w);
    }
#pragma unroll 4
    for (int c = tid; c < 72 * nb; c += nthr) {
      const int b = c / 72, i = c - 72 * b, v = i / 6, u = half * 6 + (i - 6 * v);  // element (v, u) of M_b(-q)
      cp_async8(Y + (size_t)b * kLd + 12 * u + v, rmq + base[b] + 12 * v + u);
    }
    cp_async_commit();
  }
  cp_async_wait_group<1>();
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  // launched with n_units warps: every warp owns tiles (and reaches both barriers)
  const int un = units[warp], mt = un & 0xff, nt0 = (un >> 8) & 0xff, cnt = un >> 16;
  // three real products per complex one: t1 = Xr Yr, t2 = Xi Yi, t3 = (Xr + Xi)(Yr + Yi);
  // Gr = t1 - t2, Gi = t3 - t1 - t2
  float acc[3][TILES][4];
#pragma unroll
  for (int k = 0; k < 3; k++)
#pragma unroll
    for (int n = 0; n < TILES; n++)
#pragma unroll
      for (int i = 0; i < 4; i++) acc[k][n][i] = 0.f;
  const float2* xa = X + (size_t)(16 * mt + g) * kLd + t;
  const float2* yb = Y + (size_t)(8 * nt0 + g) * kLd + t;
  for (int k0 = 0; k0 < 144; k0 += 8) {
    if (k0 == 72) {  // the second half of the rows
      cp_async_wait_group<0>();
      __syncthreads();
    }
    // A fragment: (g, t), (g + 8, t), (g, t + 4), (g + 8, t + 4)
    const float2 x[4] = {xa[k0], xa[8 * kLd + k0], xa[k0 + 4], xa[8 * kLd + k0 + 4]};
    uint32_t ah[3][4], al[3][4];  // [re, im, re + im][fragment register]
#pragma unroll
    for (int i = 0; i < 4; i++) {
      const float v[3] = {x[i].x, x[i].y, __fadd_rn(x[i].x, x[i].y)};
#pragma unroll
      for (int k = 0; k < 3; k++) {
        if (MODE == kTc3x) split_tf32(v[k], ah[k][i], al[k][i]);
        else ah[k][i] = tf32_rna(v[k]);
      }
    }
    // B fragments of every tile: (k = t, col g), (k = t + 4, col g)
    uint32_t bh[TILES][3][2], bl[TILES][3][2];
#pragma unroll
    for (int n = 0; n < TILES; n++) {
      if (n >= cnt) break;
      const float2 y[2] = {yb[(size_t)8 * n * kLd + k0], yb[(size_t)8 * n * kLd + k0 + 4]};
#pragma unroll
      for (int j = 0; j < 2; j++) {
        const float v[3] = {y[j].x, y[j].y, __fadd_rn(y[j].x, y[j].y)};
#pragma unroll
        for (int k = 0; k < 3; k++) {
          if (MODE == kTc3x) split_tf32(v[k], bh[n][k][j], bl[n][k][j]);
          else bh[n][k][j] = tf32_rna(v[k]);
        }
      }
    }
    // products interleaved over the tiles (independent accumulators back to
    // back); 3xTF32: the two small cross terms before the large one
#pragma unroll
    for (int k = 0; k < 3; k++) {
      if (MODE == kTc3x) {
#pragma unroll
        for (int n = 0; n < TILES; n++)
          if (n < cnt) mma_tf32(acc[k][n], al[k], bh[n][k]);
#pragma unroll
        for (int n = 0; n < TILES; n++)
          if (n < cnt) mma_tf32(acc[k][n], ah[k], bl[n][k]);
      }
#pragma unroll
      for (int n = 0; n < TILES; n++)
        if (n < cnt) mma_tf32(acc[k][n], ah[k], bh[n][k]);
    }
  }
  // D fragment: (g, 2t), (g, 2t + 1), (g + 8, 2t), (g + 8, 2t + 1); G[p][m][n] complex64
  float4* Gp = reinterpret_cast<float4*>(G + (size_t)p * nbp * nbp);
#pragma unroll
  for (int n = 0; n < TILES; n++) {
    if (n >= cnt) break;
    float gr[4], gi[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
      gr[i] = acc[0][n][i] - acc[1][n][i];
      gi[i] = acc[2][n][i] - acc[0][n][i] - acc[1][n][i];
    }
    const int col = 8 * (nt0 + n) + 2 * t, m0 = 16 * mt + g;
    Gp[((size_t)m0 * nbp + col) >> 1] = make_float4(gr[0], gi[0], gr[1], gi[1]);
    Gp[((size_t)(m0 + 8) * nbp + col) >> 1] = make_float4(gr[2], gi[2], gr[3], gi[3]);
  }
}

size_t contract_tc_smem(int nbp) { return (size_t)2 * nbp * kLd * sizeof(float2); }

template <int MODE, int TILES>
static cudaError_t launch_tc_variant(size_t sm, int n_q, int n_units, cudaStream_t st, const void* blk, int L, int n_out,
                                    const int* base, int nb, int nbp, const int* qlist, const int* units, void* G) {
  static int granted[64] = {0};
  cudaError_t e = ensure_smem(k_contract_tc<MODE, TILES>, sm, granted);
  if (e != cudaSuccess) return e;
  k_contract_tc<MODE, TILES><<<n_q, n_units * 32, sm, st>>>((const float2*)blk, L, n_out, base, nb, nbp, qlist, units,
                                                           n_units, (float2*)G);
  return cudaGetLastError();
}

cudaError_t launch_contract_tc(const void* blk, int L, int n_out, const int* base, int nb, int nbp, const int* qlist,
                               int n_q, const int* units, int n_units, void* G, int mode, cudaStream_t st, int tiles) {
  if (n_q == 0) return cudaSuccess;
  if (nb < 1 || nb > nbp || nbp % 16 || nbp > kMaxTcBlocks || n_units < 1 || n_units > kTcMaxWarps || (n_out & 1))
    return cudaErrorInvalidValue;
  const size_t sm = contract_tc_smem(nbp);
  if (mode == kTc3x && tiles == 3)
    return launch_tc_variant<kTc3x, 3>(sm, n_q, n_units, st, blk, L, n_out, base, nb, nbp, qlist, units, G);
  if (mode == kTc3x && tiles == 2)
    return launch_tc_variant<kTc3x, 2>(sm, n_q, n_units, st, blk, L, n_out, base, nb, nbp, qlist, units, G);
  if (mode == kTc1x && tiles == 3)
    return launch_tc_variant<kTc1x, 3>(sm, n_q, n_units, st, blk, L, n_out, base, nb, nbp, qlist, units, G);
  if (mode == kTc1x && tiles == 2)
    return launch_tc_variant<kTc1x, 2>(sm, n_q, n_units, st, blk, L, n_out, base, nb, nbp, qlist, units, G);
  return cudaErrorInvalidValue;
}

}  // namespace bbc
