// tc_umma.cu -- the trace-form block-pair products of the mixed precisions on
// the fifth-generation tensor cores (tcgen05, accumulators in tensor memory):
// per pair {q, -q} the complex matrix
//
//   G(q)[i][j] = sum_{u,v} M_i(q)[u][v] M_j(-q)[v][u]      (G(-q) = G(q)^T)
//
// over the 12 x 12 open-index matrices M of the nb blocks that the
// trace-form tasks read (Sec. 3 Eq. LN.pLLp.FFT: the sum over the open colour
// and spin indices of A(q) B(-q); the host split is in tensor_split.cpp).
//
// One real matrix product per pair carries all four real parts.  With
// X[i][12u + v] = M_i(q)[u][v], Y[j][12u + v] = M_j(-q)[v][u], A = [Xr; Xi]
// (2 nbp rows) and B = [Yr; Yi] (2 nbp rows), D = A B^T holds Xr Yr^T,
// Xr Yi^T, Xi Yr^T and Xi Yi^T as its four nbp x nbp quadrants, and
//
//   Re G = Xr Yr^T - Xi Yi^T,   Im G = Xr Yi^T + Xi Yr^T.
//
// D is one M = 128, N = 2 nbp, K = 144 product of kind::tf32 with FP32
// accumulation in tensor memory (rows 2 nbp .. 127 of A are not staged; the
// rows of D they give are not read).  FP32 accuracy (kTc3x): every operand is
// split into x = hi + lo, hi the nearest TF32 value and lo the FP32 rest, and
// the open indices are run three times, over (lo, hi), (hi, lo) and (hi, hi);
// the TF32 trial (kTc1x) runs (hi, hi) only.
//
// A persistent CTA per SM walks its pairs in units of 48 open indices (four
// consecutive u): its warps load a unit's rows from the q-major blocks,
// split them and store them in the canonical K-major layout without swizzle
// (core matrices of 8 rows x 16 bytes) in one of two shared-memory stages,
// and one thread issues the unit's MMAs and commits them to the stage's
// mbarrier, so that the loads of the next unit overlap the MMAs of this one.
// The rows of the pair after next are prefetched into L2 by bulk prefetches.  Two
// accumulators in tensor memory let the epilogue of a pair (tensor memory to
// registers to G, the Xi rows handed to the Xr rows through shared memory)
// run two units after the pair's last MMA, while the next pair is
// multiplied.  Every mbarrier wait is bounded: past its poll limit the CTA
// records the timeout in the error word, stops issuing, waits (bounded) for
// the MMAs in flight and frees its tensor memory.
#include <cstdint>

#include "device_common.cuh"
#include "kernels.cuh"
#include "umma_schedule.hpp"

namespace bbc {

namespace {

constexpr int kUmK = 48;                      // open indices per unit (four values of u)
constexpr int kUmUnits = umsched::kUnitsPerPair;  // units per pair
static_assert(kUmUnits * kUmK == 144, "the units of a pair cover its open indices");
constexpr int kUmKg = kUmK / 4;               // 16-byte k-groups of one operand row in a unit
constexpr int kUmLbo = 128;                   // bytes between core matrices adjacent in K
constexpr int kUmSbo = kUmKg * 128;           // bytes between 8-row groups
constexpr int kUmBuf = 128 / 8 * kUmSbo;      // one operand buffer of 128 rows (24 KB)
constexpr int kUmStage = 4 * kUmBuf;          // A hi, A lo, B hi, B lo
constexpr int kUmWarps = 8;                   // warps 4..7 also run the epilogue (tensor-memory lanes 32 (w - 4) ..)
constexpr int kUmMaxTasks = 6;                // warp tasks per unit and warp: 6 nbp / 8 <= 48 over 8 warps
constexpr int kUmXld = kMaxTcBlocks + 4;      // row stride (floats) of the epilogue exchange
constexpr int kUmXch = 2 * kMaxTcBlocks * kUmXld * 4;
constexpr int kUmCols = 256;                  // tensor-memory columns: two accumulators of up to 128
constexpr size_t kUmSmem = 2 * (size_t)kUmStage + kUmXch + 64 + 4 * kMaxTcBlocks;
static_assert(kUmSmem <= kMaxSmemPerBlock, "two stages and the exchange fit one CTA");
static_assert(6 * (kMaxTcBlocks / 8) <= kUmMaxTasks * kUmWarps, "every warp task has a warp");
static_assert(2 * kMaxTcBlocks <= 128, "A fits the M = 128 instruction");

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of tcgen05: start address, leading byte
// offset (core matrices adjacent in K), stride byte offset (8-row groups),
// the descriptor version of tcgen05 (bit 46), no swizzle (bits 61..63 = 0).
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(kUmLbo >> 4) << 16) | ((uint64_t)(kUmSbo >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor of kind::tf32: D FP32 (bits 4..5 = 1), A and B TF32
// (bits 7..9, 10..12 = 2), both K-major (bits 15, 16 = 0), N / 8 at bit 17,
// M / 16 at bit 24.
__device__ __forceinline__ uint32_t umma_idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void umma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Completion of the phase of the given parity; false after spin_limit polls.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long spin_limit) {
  for (long long polls = 0; !mbar_test(bar, parity); polls++) {
    if (polls >= spin_limit) return false;
    __nanosleep(64);
  }
  return true;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// The registers of the warp's earlier tcgen05.ld are valid after this wait;
// tied to them, so that no use of them is scheduled above it.
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15])
               :
               : "memory");
}

// byte offset of (row, 16-byte k-group) in an operand buffer
__device__ __forceinline__ int umma_off(int row, int kg) { return (row >> 3) * kUmSbo + kg * kUmLbo + (row & 7) * 16; }

// x = hi + lo: hi the nearest TF32 value (ties away from zero: the 13 low
// mantissa bits rounded into the rest of the magnitude), lo the FP32 rest
__device__ __forceinline__ void split4(float a, float b, float c, float d, uint4& hi, float4& lo) {
  hi = make_uint4((__float_as_uint(a) + 0x1000u) & 0xffffe000u, (__float_as_uint(b) + 0x1000u) & 0xffffe000u,
                  (__float_as_uint(c) + 0x1000u) & 0xffffe000u, (__float_as_uint(d) + 0x1000u) & 0xffffe000u);
  lo = make_float4(a - __uint_as_float(hi.x), b - __uint_as_float(hi.y), c - __uint_as_float(hi.z),
                   d - __uint_as_float(hi.w));
}

// A thread's warp tasks, fixed for the whole launch: task t of warp w is T
// = w + 8 t = (side, 8-row group rg, h) and lane = (row in the group bl, u
// offset ul), block b = 8 rg + bl.  Side X reads M_b(q)[u][4h .. 4h + 3] (32
// bytes), side Y M_b(-q)[4h .. 4h + 3][u] (four 8-byte values 96 bytes
// apart): both the 4 consecutive open indices k = 12 u + 4h .. 12 u + 4h + 3,
// u = 4 c + ul in unit c.  Packed per task: the row offset of the pair's
// first unit (bits 0..15), the stage offset / 16 of the real part (bits
// 16..28), side (bit 29), b < nb (bit 30).
template <int MAXT>
struct UmRows {
  float4 v[MAXT][2];
};

template <int MAXT>
__device__ __forceinline__ void um_tasks(uint32_t (&tk)[MAXT], const int* s_base, int nb, int nrg, int n_tasks,
                                         int warp, int bl, int ul) {
#pragma unroll
  for (int t = 0; t < MAXT; t++) {
    const int T = warp + t * kUmWarps;
    tk[t] = 0;
    if (T < n_tasks) {
      const bool side = T >= 3 * nrg;
      const int rem = side ? T - 3 * nrg : T, rg = rem / 3, h = rem - 3 * rg, b = 8 * rg + bl;
      const int soff = umma_off(b, 3 * ul + h) + (side ? 2 * kUmBuf : 0);
      const int goff = b < nb ? s_base[b] + (side ? 48 * h + ul : 12 * ul + 4 * h) : 0;
      tk[t] = (uint32_t)goff | ((uint32_t)(soff >> 4) << 16) | ((uint32_t)side << 29) | ((uint32_t)(b < nb) << 30);
    }
  }
}

template <int MAXT>
__device__ __forceinline__ void um_load(UmRows<MAXT>& R, const uint32_t (&tk)[MAXT], const float2* rq,
                                        const float2* rmq, int c, int n_tasks, int warp) {
#pragma unroll
  for (int t = 0; t < MAXT; t++) {
    R.v[t][0] = R.v[t][1] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (warp + t * kUmWarps < n_tasks && (tk[t] >> 30)) {
      const int goff = (int)(tk[t] & 0xffffu);
      if (!((tk[t] >> 29) & 1u)) {
        const float4* src = reinterpret_cast<const float4*>(rq + goff + 48 * c);
        R.v[t][0] = __ldg(src);
        R.v[t][1] = __ldg(src + 1);
      } else {
        const float2* src = rmq + goff + 4 * c;
        const float2 y0 = __ldg(src), y1 = __ldg(src + 12), y2 = __ldg(src + 24), y3 = __ldg(src + 36);
        R.v[t][0] = make_float4(y0.x, y0.y, y1.x, y1.y);
        R.v[t][1] = make_float4(y2.x, y2.y, y3.x, y3.y);
      }
    }
  }
}

// the unit's rows, split, into a stage: real parts to rows b, imaginary
// parts to rows nbp + b (nrg 8-row groups further) of A (side X) or B (side Y)
template <int MODE, int MAXT>
__device__ __forceinline__ void um_store(const UmRows<MAXT>& R, const uint32_t (&tk)[MAXT], unsigned char* st,
                                         int nrg, int n_tasks, int warp) {
#pragma unroll
  for (int t = 0; t < MAXT; t++) {
    if (warp + t * kUmWarps < n_tasks) {
      unsigned char* dst = st + (((tk[t] >> 16) & 0x1fffu) << 4);
      const float4 a = R.v[t][0], d = R.v[t][1];
      uint4 hre, him;
      float4 lre, lim;
      split4(a.x, a.z, d.x, d.z, hre, lre);
      split4(a.y, a.w, d.y, d.w, him, lim);
      const int oim = nrg * kUmSbo;
      *reinterpret_cast<uint4*>(dst) = hre;
      *reinterpret_cast<uint4*>(dst + oim) = him;
      if (MODE == kTc3x) {
        *reinterpret_cast<float4*>(dst + kUmBuf) = lre;
        *reinterpret_cast<float4*>(dst + kUmBuf + oim) = lim;
      }
    }
  }
}

__device__ __forceinline__ int neg_site(int q, int L) {
  const int qx = q % L, qy = (q / L) % L, qz = q / (L * L);
  return (L - qx) % L + L * ((L - qy) % L + L * ((L - qz) % L));
}

}  // namespace

// blk: q-major blocks [V][n_out] complex64; base[nb]: first row of each block
// (even); qlist[n_q]: q of each pair; G[n_q][nbp][nbp] complex64 (all
// entries written); err: set to 2 when a wait gave up.  Grid <= n_q.
template <int MODE, int MAXT>
__global__ void __launch_bounds__(kUmWarps * 32, 1)
k_contract_umma(const float2* __restrict__ blk, int L, int n_out, const int* __restrict__ base, int nb, int nbp,
                const int* __restrict__ qlist, int n_q, float2* __restrict__ G, int* __restrict__ err,
                long long spin_limit) {
  extern __shared__ __align__(1024) unsigned char smem[];
  float* xch = reinterpret_cast<float*>(smem + 2 * kUmStage);  // [2][nbp][kUmXld]: Xi Yr^T, Xi Yi^T
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * kUmStage + kUmXch);  // stages 0, 1; accumulators 0, 1
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 4);
  int* s_base = reinterpret_cast<int*>(bars + 8);  // [nb]: first row of each block
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_mine = (n_q - 1 - (int)blockIdx.x) / (int)gridDim.x + 1;
  const int n_units = umsched::n_units(n_mine);
  const uint32_t bar0 = smem_u32(bars);
  if (tid == 0) {
    for (int i = 0; i < 4; i++) mbar_init(bar0 + 8 * i, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int b = tid; b < nb; b += blockDim.x) s_base[b] = base[b];
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kUmCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(tslot);
  const int nrg = nbp >> 3, n_tasks = 6 * nrg, n2 = 2 * nbp;
  const uint32_t idesc = umma_idesc_tf32(128, n2);
  uint32_t tk[MAXT];
  um_tasks<MAXT>(tk, s_base, nb, nrg, n_tasks, warp, lane & 7, lane >> 3);
  int issued = -1;   // last unit whose MMAs thread 0 issued
  bool bad = false;  // this thread saw a wait give up
  bool aborted = false;
  // the loader runs one unit ahead of the stores: rows of the pair being
  // loaded, and the q of the pair after it (read a pair ahead)
  int q_next = qlist[blockIdx.x];
  const float2 *lrq = blk, *lrmq = blk;
  // bulk prefetches of a pair's rows into L2, two pairs ahead of the loads:
  // thread t < nbp the X row of block t at q, thread nbp + t the Y row at -q
  int q_pf = -1;
  auto prefetch_rows = [&](int qp) {
    const int b = tid >= nbp ? tid - nbp : tid;
    const int qs = tid >= nbp ? neg_site(qp, L) : qp;
    if (b < nb)
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(blk + (size_t)qs * n_out + s_base[b]),
                   "r"(144 * 8)
                   : "memory");
  };
  if (tid < n2 && n_mine > 1) prefetch_rows(qlist[blockIdx.x + gridDim.x]);
  auto load_unit = [&](int w, UmRows<MAXT>& R) {
    const int j = umsched::pair_of(w), cw = umsched::chunk_of(w);
    if (cw == 0) {
      lrq = blk + (size_t)q_next * n_out;
      lrmq = blk + (size_t)neg_site(q_next, L) * n_out;
      if (j + 1 < n_mine) q_next = qlist[blockIdx.x + (size_t)(j + 1) * gridDim.x];
    }
    um_load<MAXT>(R, tk, lrq, lrmq, cw, n_tasks, warp);
  };
  // one unit: loads of unit u + 1 issued first, then (warps 4..7) the
  // epilogue of pair (u - 4) / 3, then unit u into stage u & 1 once the MMAs
  // of unit u - 2 have read it, then one barrier and the MMAs of unit u
  auto step = [&](int u, const UmRows<MAXT>& cur, UmRows<MAXT>& nxt) -> bool {
    if (u > umsched::last_step(n_mine)) return false;
    const int i = umsched::pair_of(u), c = umsched::chunk_of(u), s = umsched::stage(u);
    if (u + 1 < n_units) load_unit(u + 1, nxt);
    // the rows of the pair after next into L2 (its q read one unit earlier)
    if (tid < n2 && u < n_units) {
      if (c == 0) q_pf = i + 2 < n_mine ? qlist[blockIdx.x + (size_t)(i + 2) * gridDim.x] : -1;
      if (c == 1 && q_pf >= 0) prefetch_rows(q_pf);
    }
    if (warp >= 4 && umsched::is_epilogue_step(u)) {
      const int e = umsched::epilogue_pair(u);
      bool ok = mbar_wait(bar0 + 8 * (2 + umsched::acc(e)), umsched::acc_parity(e), spin_limit);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) bad = true;
      tc_fence_after();
      const int r0 = 32 * (warp - 4), r = r0 + lane;
      const uint32_t tw = tmem + ((uint32_t)r0 << 16) + (uint32_t)(umsched::acc(e) * 128);
      if (ok && r0 + 32 > nbp && r0 < n2) {  // this warp holds Xi rows: to the exchange
        for (int c0 = 0; c0 < n2; c0 += 16) {
          uint32_t v[16];
          tmem_ld16(tw + c0, v);
          tmem_wait_ld(v);
          if (r >= nbp && r < n2) {
            const int hf = c0 >= nbp;
            float* dst = xch + (size_t)(hf * nbp + r - nbp) * kUmXld + (c0 - hf * nbp);
#pragma unroll
            for (int j = 0; j < 16; j += 4)
              *reinterpret_cast<uint4*>(dst + j) = make_uint4(v[j], v[j + 1], v[j + 2], v[j + 3]);
          }
        }
      }
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (ok && r0 < nbp) {  // this warp holds Xr rows: combine and store row r of G
        const int p = blockIdx.x + e * gridDim.x;
        float2* gr = G + ((size_t)p * nbp + r) * nbp;
        for (int c0 = 0; c0 < nbp; c0 += 16) {
          uint32_t rr[16], ri[16];
          tmem_ld16(tw + c0, rr);        // Xr Yr^T
          tmem_ld16(tw + nbp + c0, ri);  // Xr Yi^T
          tmem_wait_ld(rr);
          tmem_wait_ld(ri);
          if (r < nbp) {
            const float* xir = xch + (size_t)r * kUmXld + c0;          // Xi Yr^T
            const float* xii = xch + (size_t)(nbp + r) * kUmXld + c0;  // Xi Yi^T
#pragma unroll
            for (int j = 0; j < 16; j += 2)
              *reinterpret_cast<float4*>(gr + c0 + j) =
                  make_float4(__uint_as_float(rr[j]) - xii[j], __uint_as_float(ri[j]) + xir[j],
                              __uint_as_float(rr[j + 1]) - xii[j + 1], __uint_as_float(ri[j + 1]) + xir[j + 1]);
          }
        }
      }
      tc_fence_before();
    }
    if (u < n_units) {
      const bool ok = !umsched::stage_waits(u) || mbar_wait(bar0 + 8 * s, umsched::stage_parity(u), spin_limit);
      if (!ok) bad = true;
      if (ok) um_store<MODE, MAXT>(cur, tk, smem + (size_t)s * kUmStage, nrg, n_tasks, warp);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    tc_fence_before();
    const int any_bad = __syncthreads_or(bad ? 1 : 0);
    tc_fence_after();
    if (any_bad) {
      aborted = true;
      return false;
    }
    // D(pair i) += A B^T over the unit's 48 open indices
    if (tid == 0 && u < n_units) {
      const uint32_t sa = smem_u32(smem + (size_t)s * kUmStage);
      const uint32_t d = tmem + (uint32_t)(umsched::acc(i) * 128);
#pragma unroll
      for (int kk = 0; kk < kUmK / 8; kk++) {
        const uint32_t o = 2 * kUmLbo * kk;  // 8 TF32 values = 2 core matrices along K
        const uint64_t ahi = umma_desc(sa + o), alo = umma_desc(sa + kUmBuf + o);
        const uint64_t bhi = umma_desc(sa + 2 * kUmBuf + o), blo = umma_desc(sa + 3 * kUmBuf + o);
        const uint32_t first = (c == 0 && kk == 0) ? 0u : 1u;
        if (MODE == kTc3x) {
          umma_tf32(d, alo, bhi, idesc, first);
          umma_tf32(d, ahi, blo, idesc, 1u);
          umma_tf32(d, ahi, bhi, idesc, 1u);
        } else {
          umma_tf32(d, ahi, bhi, idesc, first);
        }
      }
      umma_commit(bar0 + 8 * s);
      if (c == kUmUnits - 1) umma_commit(bar0 + 8 * (2 + umsched::acc(i)));
      issued = u;
    }
    return true;
  };
  UmRows<MAXT> ra, rb;
  load_unit(0, ra);
  for (int u = 0;; u += 2) {
    if (!step(u, ra, rb)) break;
    if (!step(u + 1, rb, ra)) break;
  }
  // after a wait gave up: the record, and the MMAs in flight finish before
  // the tensor memory is freed
  if (aborted && tid == 0) {
    atomicOr(err, 2);
    if (issued >= 0) mbar_wait(bar0 + 8 * umsched::stage(issued), (uint32_t)((issued >> 1) & 1), spin_limit);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kUmCols) : "memory");
}

size_t contract_umma_smem() { return kUmSmem; }

template <int MODE, int MAXT>
static cudaError_t launch_umma_variant(int grid, cudaStream_t st, const void* blk, int L, int n_out, const int* base,
                                       int nb, int nbp, const int* qlist, int n_q, void* G, int* err,
                                       long long spin_limit) {
  static int granted[64] = {0};
  cudaError_t e = ensure_smem(k_contract_umma<MODE, MAXT>, kUmSmem, granted);
  if (e != cudaSuccess) return e;
  k_contract_umma<MODE, MAXT><<<grid, kUmWarps * 32, kUmSmem, st>>>((const float2*)blk, L, n_out, base, nb, nbp,
                                                                   qlist, n_q, (float2*)G, err, spin_limit);
  return cudaGetLastError();
}

// warp tasks per warp: 6 nbp / 8 tasks over the 8 warps
template <int MODE>
static cudaError_t launch_umma_mode(int grid, cudaStream_t st, const void* blk, int L, int n_out, const int* base,
                                    int nb, int nbp, const int* qlist, int n_q, void* G, int* err, long long spin_limit) {
  const int maxt = (6 * (nbp / 8) + kUmWarps - 1) / kUmWarps;
  if (maxt <= 2)
    return launch_umma_variant<MODE, 2>(grid, st, blk, L, n_out, base, nb, nbp, qlist, n_q, G, err, spin_limit);
  if (maxt <= 3)
    return launch_umma_variant<MODE, 3>(grid, st, blk, L, n_out, base, nb, nbp, qlist, n_q, G, err, spin_limit);
  if (maxt <= 5)
    return launch_umma_variant<MODE, 5>(grid, st, blk, L, n_out, base, nb, nbp, qlist, n_q, G, err, spin_limit);
  return launch_umma_variant<MODE, kUmMaxTasks>(grid, st, blk, L, n_out, base, nb, nbp, qlist, n_q, G, err,
                                                spin_limit);
}

cudaError_t launch_contract_umma(const void* blk, int L, int n_out, const int* base, int nb, int nbp,
                                 const int* qlist, int n_q, void* G, int mode, int* err, long long spin_limit,
                                 cudaStream_t st) {
  if (n_q == 0) return cudaSuccess;
  if (nb < 1 || nb > nbp || nbp % 16 || nbp > kMaxTcBlocks || (n_out & 1) || spin_limit < 1 || !err)
    return cudaErrorInvalidValue;
  static int n_sm[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!n_sm[dev]) {
    e = cudaDeviceGetAttribute(&n_sm[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
  }
  const int grid = n_q < n_sm[dev] ? n_q : n_sm[dev];  // one CTA per SM (shared memory), each with >= 1 pair
  if (mode == kTc3x)
    return launch_umma_mode<kTc3x>(grid, st, blk, L, n_out, base, nb, nbp, qlist, n_q, G, err, spin_limit);
  if (mode == kTc1x)
    return launch_umma_mode<kTc1x>(grid, st, blk, L, n_out, base, nb, nbp, qlist, n_q, G, err, spin_limit);
  return cudaErrorInvalidValue;
}

}  // namespace bbc
