// kernels.cuh -- launchers of the sm_103a kernels of the effective block
// algorithm (arXiv:1510.00903).  Host-callable, plain pointers.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace bbc {

// Device copy of one block-pair task (planner PairTask).
struct DevTask {
  int offA[8], offB[8];
  int nAnB;  // nA | nB << 8
  int n1, n2;
  int sA;    // sA1 | sA2 << 16
  int sB;    // sB1 | sB2 << 16
};

// A warp batch: up to 32 tasks of one shape (nA) and one open-index length.
struct WarpBatch {
  int n, nA;
  int task[32];
};

constexpr int kMaxDiquarks = 11;   // (l,l), (l,s) with C gamma5; (s,s), (l,l), (l,s) with eta_l C gamma_l
constexpr int kMaxFamilies = 22;   // lll, lls, lsl, lss (C gamma5); sss, lll, lls, lsl, lss, ssl (vector, x y z)
constexpr int kMaxBuildGroups = 16;
struct DevGroups {  // block-build groups (rows that read the same tensor families)
  int n;
  int first[kMaxBuildGroups], rows[kMaxBuildGroups], fam0[kMaxBuildGroups], fam1[kMaxBuildGroups];
  int zneed_first[kMaxBuildGroups + 1];  // group gi computes tensor entries zneed[zneed_first[gi] .. zneed_first[gi+1])
  int z_slots;         // shared-memory positions for tensor entries
  int spin0;           // Dirac index of the first external spin component (0 upper, 2 lower)
  int chunk_first[kMaxBuildGroups + 1];  // first 32-row chunk of each group in the lane-interleaved entry table
  int n_dq;            // diquarks computed per site
  int dq_f0[kMaxDiquarks], dq_f1[kMaxDiquarks];  // their quark flavours (0 light, 1 strange)
  int dq_gam[kMaxDiquarks];                      // their Gamma1: 0 = C gamma5, l = eta_l C gamma_l
  int fam_dq[kMaxFamilies];                      // per family: index of its diquark in shared memory
  int fam_f2[kMaxFamilies];                      // per family: third quark strange (1) or light (0)
  // dense-tuple FP32 build (k_block_build_dense): tuples of each group, their
  // entry stride, entry positions per site, 32-row chunks of each group
  int tuple_first[kMaxBuildGroups + 1], stride[kMaxBuildGroups], dense_z_slots, dchunk_first[kMaxBuildGroups + 1];
};

constexpr int kMaxChannels = 160;  // channels of one context (every id fits)
// Real type of the propagators, blocks and forward transforms: FP32, FP64,
// or double-float (two FP32 words, FP64-accurate on the FP32 pipes).
enum RealKind { RK_F32 = 0, RK_F64 = 1, RK_DF = 2 };
constexpr size_t kMaxSmemPerBlock = 227 * 1024;  // opt-in dynamic shared memory per CTA
struct ScaleParams {  // per channel: host factor (1/V, mass normalisation) and quark counts
  int n_ch;
  double f[kMaxChannels];
  int nl[kMaxChannels], ns[kMaxChannels];
};
// scale[ch] = f[ch] * 2^(nl[ch] kexp[0] + ns[ch] kexp[1]) on the device.
cudaError_t launch_scales(const ScaleParams& p, const int* kexp, double* scale, cudaStream_t st);

// Twiddle tables e^{-2 pi i k / 96} (double and float) into __constant__ memory.
cudaError_t upload_twiddles();

// |S| maximum of one propagator slice (V*144 complex, dtype 0 = c128, 1 = c64)
// into *amax (bit pattern of a non-negative double; caller zeroes it first);
// a NaN entry makes it +infinity.
cudaError_t launch_absmax(const void* src, int dtype, long long n_complex,
                          unsigned long long* amax, cudaStream_t st);
// *flag |= 1 when one of the n doubles at x is NaN or infinite.
cudaError_t launch_nonfinite(const double* x, long long n, int* flag, cudaStream_t st);
// dst = src * 2^-k with k = ilogb(max) + 1 (exact), k stored to *kexp.
cudaError_t launch_convert(const void* src, int dtype, long long n_complex,
                           const unsigned long long* amax, int* kexp, void* dst, int kind,
                           cudaStream_t st);
// Baryon blocks of every site: prop [slots][2][V][144], blk [slots][V][n_out];
// `sites` consecutive sites per CTA of `threads` threads: (1, 256), (2, 256),
// (2, 512) or (4, 512) (V a multiple of sites).
bool build_variant_supported(int sites, int threads);
// FP32 blocks from dense entry tuples (dense_build.cpp tables): prop
// [slots][2][V][144] complex64, blk [slots][V][n_out]; `sites` (1 or 2)
// consecutive sites per CTA of `threads` (256 or 512) threads.
bool dense_build_supported(int sites, int threads);
size_t dense_build_smem(const DevGroups& g, int sites);
cudaError_t launch_block_build_dense(const void* prop, int V, int n_slots, const int2* ell_chunk, const uint32_t* ell,
                                     const uint32_t* tuples, const DevGroups& g, void* blk, int n_out, cudaStream_t st,
                                     int sites, int threads);
size_t block_build_smem(int z_slots, int sites, bool fp64, int n_dq);
// ell_chunk[c] = (offset, length) of 32-row chunk c in ell (lane-interleaved rows).
cudaError_t launch_block_build(const void* prop, int V, int n_slots, const int2* ell_chunk,
                               const uint32_t* ell, const uint32_t* zneed, const DevGroups& g,
                               void* blk, int n_out, int kind, cudaStream_t st, int sites, int threads);
// Forward 3-D FFT of every block field: x pass from the site-major build
// output blk_site[slots][V][n_rows] into field-major blk_field[slots][n_rows][V],
// then the y and z passes in place (exp(-i q.x), unnormalised).
// fp64 with blk_sum: the last pass also writes blk_sum[slots][n_rows][V] =
// re + im of every FP64 value (read by the FP64 pair products).
cudaError_t launch_fft_forward(const void* blk_site, void* blk_field, int L, int n_slots, int n_rows, bool fp64,
                               cudaStream_t st, double* blk_sum = nullptr);
// The same transform on double-float blocks in double-float arithmetic; the
// field-major result holds (re.hi, re.lo, im.hi, im.lo) per value.
cudaError_t launch_fft_forward_df(const void* blk_site, void* blk_field, int L, int n_slots, int n_rows,
                                  cudaStream_t st);
// Forward 3-D FFT in place on site-major blocks blk[slots][V][n_rows] (lanes
// over the contiguous row index); output is q-major.
cudaError_t launch_fft_forward_site(void* blk, int L, int n_slots, int n_rows, bool fp64, cudaStream_t st);
// The forward FP32 transform of launch_fft_forward_site (L <= 32) as one
// persistent launch over a device work queue (fft.cu): words = [ticket
// counter, done[tiles]] (fft_queue_ints(L, n_slots, n_rows) ints, zeroed by the
// launch), err a sticky word the kernel sets to 1 when a bounded wait gives
// up (after spin_limit polls); expect < 0 for the plane count the waits need
// (a larger value makes them run out: the timeout self-test).
struct FftQueue {
  int* words;
  int* err;
};
int fft_queue_ints(int L, int n_outer, int n_inner);
bool fft_queue_supported(int L);
constexpr long long kFftSpinLimit = 1LL << 22;  // polls of about 0.3 us: about a second
cudaError_t launch_fft_forward_queue(void* blk, int L, int n_slots, int n_rows, const FftQueue& q, int expect,
                                     long long spin_limit, cudaStream_t st);
// Inverse 3-D FFT of q-major ct[V][n_ch*16] (complex128, x and y in place),
// the z pass writing out[n_ch][V][16] multiplied by scale[ch].
// ct_f32: ct holds complex64 values (then the transform computes in FP32).
cudaError_t launch_fft_inverse_site(void* ct, void* out, int L, int n_ch, const double* scale, bool fp64_compute,
                                    cudaStream_t st, bool ct_f32 = false);
// Fused FP32 contraction of one slice from q-major blocks blk[V][n_out]: one
// CTA per pair {q, -q} (qlist[n_q]), block row i staged at shared-memory slot
// row_slot[i] < n_slots (task offsets are slots), warp units wunits {batch,
// side, k0, k1} (warp w owns wunits[wptr[w] .. wptr[w+1])), FP64 Wick sums
// into ct[V][n_ch*16].
size_t contract_fused_smem(int n_slots, int n_tasks, bool bf16);
// Launch configurations: warps per CTA in {8, 12, 16}.
// bf16: blk holds bfloat16 (re, im) pairs (4 bytes per complex) instead of
// complex64; the products multiply and accumulate in FP32 either way.
// Shapes: warps per CTA 8, 12 or 16; steps = open-index steps whose rows are
// loaded before multiplying (1, or 2 with 8 or 12 warps).
bool fused_variant_supported(int warps, int steps);
cudaError_t launch_contract_fused(const void* blk, int L, int n_out, const int* row_slot, int n_slots, const int* qlist,
                                  int n_q, const DevTask* tasks, int n_tasks, const WarpBatch* batches,
                                  const int* wptr, const int4* wunits, const int* cptr, const int* citem,
                                  const double* ccoef, int n_ch, void* ct, int warps, int steps, bool bf16,
                                  cudaStream_t st);
// Tensor-core products of the trace-form block pairs (tc_contract.cu): per
// pair {q, -q} (qlist[n_q]) the complex matrix G(q)[i][j] = sum_{u,v}
// M_i(q)[u][v] M_j(-q)[v][u] of the nb blocks at rows base[nb] of the q-major
// blocks blk[V][n_out] (complex64), written to G[n_q][nbp][nbp] (complex64);
// warp w computes the tiles units[w] = m-tile | first n-tile << 8 | n-tiles << 16.
// mode kTc3x: operands split into two TF32 words (FP32 accuracy); kTc1x: one
// TF32 rounding per operand (trial precision).
constexpr int kMaxTcBlocks = 64;     // blocks of G (G is at most 64 x 64)
constexpr int kTcTilesPerWarp = 3;   // 16 x 8 complex tiles of G per warp (at most)
constexpr int kTcMaxWarps = 16;
constexpr int kTc3x = 0, kTc1x = 1;
size_t contract_tc_smem(int nbp);
cudaError_t launch_contract_tc(const void* blk, int L, int n_out, const int* base, int nb, int nbp, const int* qlist,
                               int n_q, const int* units, int n_units, void* G, int mode, cudaStream_t st,
                               int tiles = kTcTilesPerWarp);
// The same products on the fifth-generation tensor cores (tc_umma.cu): G of
// every pair, all nbp x nbp entries, from one tcgen05 product per pair with
// FP32 accumulators in tensor memory; a persistent CTA per SM.  Its mbarrier
// waits give up after spin_limit polls (about 0.1 us each), set *err = 2 and
// free the tensor memory.
size_t contract_umma_smem();
cudaError_t launch_contract_umma(const void* blk, int L, int n_out, const int* base, int nb, int nbp,
                                 const int* qlist, int n_q, void* G, int mode, int* err, long long spin_limit,
                                 cudaStream_t st);
// The rest of the mixed contraction (fused_contract.cu): per pair {q, -q}
// the CUDA-core products of the other tasks on compact rows (row_map[i] =
// block row | shared-memory slot << 16, i < n_rows) and the signed
// double-float sums over Wick diagrams of V = [P_q | P_-q | G(q)]: output o
// sums, over terms c in [cptr[o], cptr[o+1]), coefs[terms[c].y] (hi, lo) x
// V[terms[c].x & 0xffff] for q and x V[terms[c].x >> 16] for -q; g_elems =
// nbp^2 (0 without tensor-core products).  ct[V][n_ch*16] complex64.
size_t contract_rest_smem(int n_slots, int n_tasks, int g_elems, int n_coefs);
bool rest_variant_supported(int warps, int steps);
cudaError_t launch_contract_rest(const void* blk, int L, int n_out, const uint32_t* row_map, int n_rows, int n_slots,
                                 const int* qlist, int n_q, const DevTask* tasks, int n_tasks,
                                 const WarpBatch* batches, const int* wptr, const int4* wunits, const void* G,
                                 int g_elems, const int* cptr, const uint2* terms, const float2* coefs, int n_coefs,
                                 int n_ch, void* ct, int warps, int steps, cudaStream_t st);
// dst[i] = (bf16(src[i].re), bf16(src[i].im)), round to nearest even, n complex64 values.
cudaError_t launch_to_bf16(const void* src, void* dst, size_t n, cudaStream_t st);
// Inverse 3-D FFT of ct[n_ch][16][V] (complex128, x and y in place), the z
// pass writing out[n_ch][V][16] (complex128) multiplied by scale[ch].
cudaError_t launch_fft_inverse(void* ct, void* out, int L, int n_ch, const double* scale, bool fp64_compute,
                               cudaStream_t st);
// q-space contraction of one slice from field-major blocks blk_field[n_rows][V]:
// pair products of every task (warp task groups group_ptr/group_task) into
// P[n_tasks*16][V] ...
// fp64: blk_sum (or nullptr) is the re + im plane launch_fft_forward wrote.
cudaError_t launch_pair_products(const void* blk_field, int L, const DevTask* tasks, const int* group_ptr,
                                 const int* group_task, int n_groups, void* P, bool fp64, cudaStream_t st,
                                 const double* blk_sum = nullptr);
// Double-float variant: blk_field and P hold (re.hi, re.lo, im.hi, im.lo)
// FP32 quadruples per complex value.
cudaError_t launch_pair_products_df(const void* blk_field, int L, const DevTask* tasks, const int* group_ptr,
                                    const int* group_task, int n_groups, void* P, cudaStream_t st);
// Wick sums of double-float products with double-float coefficients
// (ccoef_df[c] = (hi, lo) of ccoef[c]) into double-float ct, and the inverse
// transform of such ct in double-float arithmetic whose last pass writes
// complex128 out[n_ch][V][16] times scale[ch].
cudaError_t launch_wick_sums_df(const void* P, int L, const int* cptr, const int* citem, const float2* ccoef_df,
                                int n_ch, void* ct, cudaStream_t st);
cudaError_t launch_fft_inverse_df(void* ct, void* out, int L, int n_ch, const double* scale, cudaStream_t st);
// ... then the signed FP64 sums over Wick diagrams into ct[n_ch*16][V] (complex128).
cudaError_t launch_wick_sums(const void* P, int L, const int* cptr, const int* citem, const double* ccoef, int n_ch,
                             void* ct, bool fp64, cudaStream_t st);

// Orbits of the 24 cubic rotations on the periodic L^3 lattice (host):
// orbit k = orb_site[orb_ptr[k] .. orb_ptr[k+1]), each site exactly once.
void cubic_orbits(int L, std::vector<int>& orb_ptr, std::vector<int>& orb_site);
// Source spin-state projection R and/or (Ra1 not null) its average over the
// 24 cubic rotations of r, of C[n_fields][L^3][16] complex128; orbit tables
// on the device.
cudaError_t launch_project(const void* C, int L, const int* orb_ptr, const int* orb_site, int n_orb, int n_fields,
                           void* R, void* Ra1, cudaStream_t st);

}  // namespace bbc
