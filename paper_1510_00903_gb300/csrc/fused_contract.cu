// fused_contract.cu -- FP32 q-space contraction fused with the FP64 Wick sums, one CTA per pair {q, -q} (mixed precision path)
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <utility>

#include <cuda_bf16.h>

#include "device_common.cuh"

namespace bbc {

// ------------------------------------------------- fused contraction (FP32)
// One CTA per pair {q, -q}.  The q-row and the -q row of the q-major
// Fourier-space blocks (blk[q][n_out]) are staged in shared memory once,
// interleaved as R[i] = (F_q[i], F_-q[i]), so one 16-byte load serves both
// products A(q) B(-q) (side 0) and A(-q) B(q) (side 1); every block element is
// read from HBM exactly once.  Warps run units (batch of up to 32 tasks of
// one shape and one open-index length, k range): lane l takes task l, so
// control flow is uniform within the warp.  Products accumulate in FP32
// registers and are added into P[side][task*16 + spin pair] in shared memory.
// The signed FP64 sums over Wick diagrams then run in the same CTA, widening
// each FP32 product as they read it, and write ct[q][o].
// Products of one warp unit (open-index steps k0 .. k1-1) of one task: NA x NB
// complex products for q (A(q) B(-q)) and for -q (A(-q) B(q)) in FP32
// registers.
// FP32 -> FP64 by the IEEE-754 bit layouts (sign, exponent rebiased by
// 1023 - 127 = 896, the 23 mantissa bits at the top of the 52): integer
// instructions only, leaving GB300's narrow FP64 pipe to the Wick sums.
// Exact for normal numbers, infinities and NaNs; FP32 subnormals (|x| below
// 2^-126, far under any product's scale here) become signed zeros.
__device__ __forceinline__ double widen(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned sign = u & 0x80000000u;
  if (e == 0) return __hiloint2double((int)sign, 0);
  const unsigned e64 = e == 0xffu ? 0x7ffu : e + 896u;
  return __hiloint2double((int)(sign | (e64 << 20) | ((u >> 3) & 0xfffffu)), (int)(u << 29));
}

// A staged row: (F_q, F_-q) as complex64 pairs, or as bfloat16 (re, im)
// pairs widened to FP32 (a bfloat16 is the high half of a float).
__device__ __forceinline__ float4 load_row(const float4* R, int i) { return R[i]; }
__device__ __forceinline__ float4 load_row(const uint2* R, int i) {
  const uint2 u = R[i];
  return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u), __uint_as_float(u.y << 16),
                     __uint_as_float(u.y & 0xffff0000u));
}

// STEPS > 1 loads the rows of STEPS consecutive open-index steps before
// multiplying any of them (more shared-memory loads in flight per warp, for
// launch shapes with registers to spare).
template <int NA, int NB, int STEPS, typename Row>
__device__ __forceinline__ void unit_products_pair(const Row* __restrict__ R, const DevTask& t, int k0, int k1,
                                                   cpx<float>* P0, cpx<float>* P1, int rot, bool self) {
  const int n2 = t.n2;
  const int sA1 = t.sA & 0xffff, sA2 = t.sA >> 16, sB1 = t.sB & 0xffff, sB2 = t.sB >> 16;
  int i1 = k0 / n2, i2 = k0 - i1 * n2;
  int oA = i1 * sA1 + i2 * sA2, oB = i1 * sB1 + i2 * sB2;
  const int wrapA = sA1 - (n2 - 1) * sA2, wrapB = sB1 - (n2 - 1) * sB2;
  cpx<float> acc0[NA * NB], acc1[NA * NB];
#pragma unroll
  for (int i = 0; i < NA * NB; i++) { acc0[i] = cpx<float>(0.f, 0.f); acc1[i] = cpx<float>(0.f, 0.f); }
  auto advance = [&]() {
    if (++i2 == n2) { i2 = 0; oA += wrapA; oB += wrapB; }
    else { oA += sA2; oB += sB2; }
  };
  auto multiply = [&](const float4 (&a)[NA], const float4 (&b)[NB]) {
#pragma unroll
    for (int ra = 0; ra < NA; ra++)
#pragma unroll
      for (int rb = 0; rb < NB; rb++) {
        cmac(acc0[ra * NB + rb], cpx<float>(a[ra].x, a[ra].y), cpx<float>(b[rb].z, b[rb].w));
        cmac(acc1[ra * NB + rb], cpx<float>(a[ra].z, a[ra].w), cpx<float>(b[rb].x, b[rb].y));
      }
  };
  int k = k0;
  if (STEPS > 1) {
    for (; k + STEPS <= k1; k += STEPS) {
      float4 a[STEPS][NA], b[STEPS][NB];
#pragma unroll
      for (int s = 0; s < STEPS; s++) {
#pragma unroll
        for (int r = 0; r < NA; r++) a[s][r] = load_row(R, t.offA[r] + oA);
#pragma unroll
        for (int r = 0; r < NB; r++) b[s][r] = load_row(R, t.offB[r] + oB);
        advance();
      }
#pragma unroll
      for (int s = 0; s < STEPS; s++) multiply(a[s], b[s]);
    }
  }
  for (; k < k1; k++) {
    float4 a[NA], b[NB];
#pragma unroll
    for (int r = 0; r < NA; r++) a[r] = load_row(R, t.offA[r] + oA);
#pragma unroll
    for (int r = 0; r < NB; r++) b[r] = load_row(R, t.offB[r] + oB);
    multiply(a, b);
    advance();
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

template <int WARPS, int STEPS, bool BF16>
__global__ void __launch_bounds__(WARPS * 32, 1)
k_contract_fused(const void* __restrict__ blk, int L, int n_out, const int* __restrict__ row_slot, int n_slots,
                 const int* __restrict__ qlist,
                 const DevTask* __restrict__ tasks, int n_tasks, const WarpBatch* __restrict__ batches,
                 const int* __restrict__ wptr, const int4* __restrict__ wunits, const int* __restrict__ cptr,
                 const int* __restrict__ citem, const double* __restrict__ ccoef, int n_outputs,
                 cpx<double>* __restrict__ ct) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int kFusedThreads = WARPS * 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int np = n_tasks * 16;                                        // products per side
  using Row = typename std::conditional<BF16, uint2, float4>::type;
  const size_t region = ((size_t)n_slots * sizeof(Row) + 15) & ~(size_t)15;  // P is zeroed as float4
  Row* R = reinterpret_cast<Row*>(smem_raw);                          // [n_slots] (F_q, F_-q)
  cpx<float>* P = reinterpret_cast<cpx<float>*>(smem_raw + region);   // [2][np]
  const int q = qlist[blockIdx.x];
  const int qx = q % L, qy = (q / L) % L, qz = q / (L * L);
  const int nq = (L - qx) % L + L * ((L - qy) % L + L * ((L - qz) % L));
  const bool self = nq == q;
  {
    if constexpr (BF16) {
      const unsigned* s0 = reinterpret_cast<const unsigned*>(blk) + (size_t)q * n_out;
      const unsigned* s1 = reinterpret_cast<const unsigned*>(blk) + (size_t)nq * n_out;
      for (int i = tid; i < n_out; i += kFusedThreads) {
        const unsigned x = __ldg(s0 + i), y = self ? x : __ldg(s1 + i);
        R[__ldg(row_slot + i)] = make_uint2(x, y);
      }
    } else {
      const float2* s0 = reinterpret_cast<const float2*>(blk) + (size_t)q * n_out;
      const float2* s1 = reinterpret_cast<const float2*>(blk) + (size_t)nq * n_out;
      for (int i = tid; i < n_out; i += kFusedThreads) {
        const float2 x = __ldg(s0 + i), y = self ? x : __ldg(s1 + i);
        R[__ldg(row_slot + i)] = make_float4(x.x, x.y, y.x, y.y);
      }
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
    if (wb.nA == 4) unit_products_pair<4, 4, STEPS>(R, t, un.z, un.w, p0, p1, ti, self);
    else if (wb.nA == 2) unit_products_pair<2, 8, STEPS>(R, t, un.z, un.w, p0, p1, ti, self);
    else unit_products_pair<8, 2, STEPS>(R, t, un.z, un.w, p0, p1, ti, self);
  }
  __syncthreads();
  // signed FP64 sums, each FP32 product widened as it is read (undoing the
  // slot rotation of its spin pair)
  const int sides = self ? 1 : 2;
  for (int j = tid; j < sides * n_outputs; j += kFusedThreads) {
    const int side = j / n_outputs, o = j - side * n_outputs;
    const cpx<float>* Ps = P + side * np;
    cpx<double> acc(0, 0);
    const int c1 = cptr[o + 1];
    for (int c = cptr[o]; c < c1; c++) {
      const double w = ccoef[c];
      const int item = citem[c], ti = item >> 4;
      const cpx<float> v = Ps[(ti << 4) + ((item + ti) & 15)];
      acc.re = fma(w, widen(v.re), acc.re);
      acc.im = fma(w, widen(v.im), acc.im);
    }
    ct[(size_t)(side ? nq : q) * n_outputs + o] = acc;
  }
}

// ------------------------------------- rest of the tensor-core contraction
// acc (s + e) += (ch + cl) x v in double-float arithmetic: the product's
// rounding error is kept exactly by an FMA, the sum's by TwoSum, and the error
// word gathers both (a few terms per output: no renormalisation needed).
__device__ __forceinline__ void df_axpy(float& s, float& e, float ch, float cl, float v) {
  const float p = __fmul_rn(ch, v);
  float err = __fmaf_rn(ch, v, -p);
  err = __fmaf_rn(cl, v, err);
  float sum, t;
  two_sum(s, p, sum, t);
  s = sum;
  e = __fadd_rn(e, __fadd_rn(t, err));
}

// The CUDA-core half of the mixed contraction beside k_contract_tc.  One CTA
// per pair {q, -q}: the rows the remaining tasks read are staged from the
// q-major blocks through the compact row map (row_map[i] = block row |
// shared-memory slot << 16; stored interleaved (F_q, F_-q)) with asynchronous
// copies; their products run as in k_contract_fused; G(q) of the pair is
// staged beside them; the signed sums over Wick diagrams add coef x V, V =
// [P_q | P_-q | G], in double-float arithmetic on the FP32 pipes (the
// products are FP32; the sums keep their cancellations exact to 2^-48 of the
// terms), one thread per output for both q and -q.  A term is (source q |
// source -q << 16, coefficient index) into the pair's coefficient table
// (hi, lo).  The sums are rounded to FP32 and stored as complex64 (the inverse
// transform computes in FP32).
template <int WARPS, int STEPS>
__global__ void __launch_bounds__(WARPS * 32, 2)
k_contract_rest(const float2* __restrict__ blk, int L, int n_out, const uint32_t* __restrict__ row_map, int n_rows,
                int n_slots, const int* __restrict__ qlist, const DevTask* __restrict__ tasks, int n_tasks,
                const WarpBatch* __restrict__ batches, const int* __restrict__ wptr, const int4* __restrict__ wunits,
                const float4* __restrict__ G, int g_elems, const int* __restrict__ cptr, const uint2* __restrict__ terms,
                const float2* __restrict__ coefs, int n_coefs, int n_outputs, float2* __restrict__ ct) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int kThreads = WARPS * 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int np = n_tasks * 16;                                      // products per side
  float4* R = reinterpret_cast<float4*>(smem_raw);                  // [n_slots] (F_q, F_-q)
  cpx<float>* V = reinterpret_cast<cpx<float>*>(smem_raw + (size_t)n_slots * sizeof(float4));  // [2 np | g_elems]
  float2* C = reinterpret_cast<float2*>(V + 2 * np + g_elems);      // [n_coefs] (hi, lo)
  const int p = blockIdx.x, q = qlist[p];
  const int qx = q % L, qy = (q / L) % L, qz = q / (L * L);
  const int nq = (L - qx) % L + L * ((L - qy) % L + L * ((L - qz) % L));
  const bool self = nq == q;
  {
    const float2* s0 = blk + (size_t)q * n_out;
    const float2* s1 = blk + (size_t)nq * n_out;
#pragma unroll 4
    for (int i = tid; i < n_rows; i += kThreads) {
      const uint32_t m = __ldg(row_map + i);
      const int src = (int)(m & 0xffffu), slot = (int)(m >> 16);
      cp_async8(R + slot, s0 + src);
      cp_async8(reinterpret_cast<float2*>(R + slot) + 1, s1 + src);
    }
    const float4* gp = G + (size_t)p * (g_elems >> 1);
    float4* gs = reinterpret_cast<float4*>(V + 2 * np);
#pragma unroll 4
    for (int i = tid; i < (g_elems >> 1); i += kThreads) cp_async16(gs + i, gp + i);
    float4* pz = reinterpret_cast<float4*>(V);
    for (int i = tid; i < np; i += kThreads) pz[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = tid; i < n_coefs; i += kThreads) C[i] = __ldg(coefs + i);
    cp_async_wait_all();
  }
  __syncthreads();
  const int u1 = wptr[warp + 1];
  for (int u = wptr[warp]; u < u1; u++) {
    const int4 un = wunits[u];  // batch, -, k0, k1
    const WarpBatch& wb = batches[un.x];
    if (lane >= wb.n) continue;
    const int ti = wb.task[lane];
    const DevTask t = tasks[ti];
    cpx<float>* p0 = V + ti * 16;
    cpx<float>* p1 = V + np + ti * 16;
    // both sides even for q = -q: a swapped task's products for q are read from its -q side
    if (wb.nA == 4) unit_products_pair<4, 4, STEPS>(R, t, un.z, un.w, p0, p1, ti, false);
    else if (wb.nA == 2) unit_products_pair<2, 8, STEPS>(R, t, un.z, un.w, p0, p1, ti, false);
    else unit_products_pair<8, 2, STEPS>(R, t, un.z, un.w, p0, p1, ti, false);
  }
  __syncthreads();
  for (int o = tid; o < n_outputs; o += kThreads) {
    float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // (re s, re e, im s, im e) for q, then -q
    const int c1 = __ldg(cptr + o + 1);
    for (int c = __ldg(cptr + o); c < c1; c++) {
      const uint2 tm = __ldg(terms + c);
      const float2 cf = C[tm.y];
      const cpx<float> vq = V[tm.x & 0xffffu];
      df_axpy(a[0], a[1], cf.x, cf.y, vq.re);
      df_axpy(a[2], a[3], cf.x, cf.y, vq.im);
      if (!self) {
        const cpx<float> vm = V[tm.x >> 16];
        df_axpy(a[4], a[5], cf.x, cf.y, vm.re);
        df_axpy(a[6], a[7], cf.x, cf.y, vm.im);
      }
    }
    ct[(size_t)q * n_outputs + o] = make_float2(__fadd_rn(a[0], a[1]), __fadd_rn(a[2], a[3]));
    if (!self) ct[(size_t)nq * n_outputs + o] = make_float2(__fadd_rn(a[4], a[5]), __fadd_rn(a[6], a[7]));
  }
}

size_t contract_rest_smem(int n_slots, int n_tasks, int g_elems, int n_coefs) {
  return (size_t)n_slots * sizeof(float4) + (size_t)2 * n_tasks * 16 * sizeof(cpx<float>) +
         (size_t)g_elems * sizeof(cpx<float>) + (size_t)n_coefs * sizeof(float2);
}

bool rest_variant_supported(int warps, int steps) {
  return (warps == 4 && (steps == 1 || steps == 2)) || (warps == 8 && steps == 1);
}

template <int WARPS, int STEPS>
cudaError_t launch_rest_variant(size_t sm, int n_q, cudaStream_t st, const void* blk, int L, int n_out,
                                const uint32_t* row_map, int n_rows, int n_slots, const int* qlist,
                                const DevTask* tasks, int n_tasks, const WarpBatch* batches, const int* wptr,
                                const int4* wunits, const void* G, int g_elems, const int* cptr, const uint2* terms,
                                const float2* coefs, int n_coefs, int n_outputs, float2* ct) {
  static int granted[64] = {0};
  cudaError_t e = ensure_smem(k_contract_rest<WARPS, STEPS>, sm, granted);
  if (e != cudaSuccess) return e;
  k_contract_rest<WARPS, STEPS><<<n_q, WARPS * 32, sm, st>>>((const float2*)blk, L, n_out, row_map, n_rows, n_slots,
                                                             qlist, tasks, n_tasks, batches, wptr, wunits,
                                                             (const float4*)G, g_elems, cptr, terms, coefs, n_coefs,
                                                             n_outputs, ct);
  return cudaGetLastError();
}

cudaError_t launch_contract_rest(const void* blk, int L, int n_out, const uint32_t* row_map, int n_rows, int n_slots,
                                 const int* qlist, int n_q, const DevTask* tasks, int n_tasks,
                                 const WarpBatch* batches, const int* wptr, const int4* wunits, const void* G,
                                 int g_elems, const int* cptr, const uint2* terms, const float2* coefs, int n_coefs,
                                 int n_ch, void* ct, int warps, int steps, cudaStream_t st) {
  if (n_q == 0) return cudaSuccess;
  if ((g_elems & 1) || (g_elems && !G) || n_out > 65536 || n_slots > 65536 || 2 * n_tasks * 16 + g_elems > 65536)
    return cudaErrorInvalidValue;
  const size_t sm = contract_rest_smem(n_slots, n_tasks, g_elems, n_coefs);
  if (sm > kMaxSmemPerBlock) return cudaErrorInvalidValue;
  float2* o = (float2*)ct;
  const int n_outputs = n_ch * 16;
#define BBC_REST(W, S)                                                                                             \
  if (warps == W && steps == S)                                                                                    \
    return launch_rest_variant<W, S>(sm, n_q, st, blk, L, n_out, row_map, n_rows, n_slots, qlist, tasks, n_tasks,   \
                                     batches, wptr, wunits, G, g_elems, cptr, terms, coefs, n_coefs, n_outputs, o);
  BBC_REST(4, 1) BBC_REST(4, 2) BBC_REST(8, 1)
#undef BBC_REST
  return cudaErrorInvalidValue;
}

size_t contract_fused_smem(int n_slots, int n_tasks, bool bf16) {
  const size_t np = (size_t)n_tasks * 16;
  return (((size_t)n_slots * (bf16 ? 8 : 16) + 15) & ~(size_t)15) + 2 * np * sizeof(cpx<float>);
}

__global__ void k_to_bf16(const float2* __restrict__ src, __nv_bfloat162* __restrict__ dst, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = __float22bfloat162_rn(src[i]);
}

cudaError_t launch_to_bf16(const void* src, void* dst, size_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 16);
  k_to_bf16<<<blocks, 256, 0, st>>>((const float2*)src, (__nv_bfloat162*)dst, n);
  return cudaGetLastError();
}

template <int WARPS, int STEPS, bool BF16>
cudaError_t launch_fused_variant(size_t sm, int n_q, cudaStream_t st, const void* blk, int L, int n_out,
                                 const int* row_slot, int n_slots, const int* qlist, const DevTask* tasks, int n_tasks,
                                 const WarpBatch* batches, const int* wptr, const int4* wunits, const int* cptr,
                                 const int* citem, const double* ccoef, int n_outputs, cpx<double>* ct) {
  static int granted[64] = {0};
  cudaError_t e = ensure_smem(k_contract_fused<WARPS, STEPS, BF16>, sm, granted);
  if (e != cudaSuccess) return e;
  k_contract_fused<WARPS, STEPS, BF16><<<n_q, WARPS * 32, sm, st>>>(blk, L, n_out, row_slot, n_slots, qlist, tasks,
                                                                     n_tasks, batches, wptr, wunits, cptr, citem,
                                                                     ccoef, n_outputs, ct);
  return cudaGetLastError();
}

// (warps, steps) shapes: 16 warps leave 128 registers a thread, room for one
// step of rows; 8 and 12 warps can hold two.
bool fused_variant_supported(int warps, int steps) {
  return ((warps == 8 || warps == 12) && (steps == 1 || steps == 2)) || (warps == 16 && steps == 1);
}

cudaError_t launch_contract_fused(const void* blk, int L, int n_out, const int* row_slot, int n_slots, const int* qlist,
                                  int n_q, const DevTask* tasks, int n_tasks, const WarpBatch* batches,
                                  const int* wptr, const int4* wunits, const int* cptr, const int* citem,
                                  const double* ccoef, int n_ch, void* ct, int warps, int steps, bool bf16,
                                  cudaStream_t st) {
  const size_t sm = contract_fused_smem(n_slots, n_tasks, bf16);
  cpx<double>* o = (cpx<double>*)ct;
  const int n_outputs = n_ch * 16;
#define BBC_FUSED(W, S, B)                                                                                        \
  if (warps == W && steps == S && bf16 == B)                                                                      \
    return launch_fused_variant<W, S, B>(sm, n_q, st, blk, L, n_out, row_slot, n_slots, qlist, tasks, n_tasks,     \
                                         batches, wptr, wunits, cptr, citem, ccoef, n_outputs, o);
  BBC_FUSED(8, 1, false) BBC_FUSED(8, 2, false) BBC_FUSED(12, 1, false) BBC_FUSED(12, 2, false)
  BBC_FUSED(16, 1, false)
  BBC_FUSED(8, 1, true) BBC_FUSED(8, 2, true) BBC_FUSED(12, 1, true) BBC_FUSED(12, 2, true) BBC_FUSED(16, 1, true)
#undef BBC_FUSED
  return cudaErrorInvalidValue;
}

}  // namespace bbc
