// kernels.cuh -- launchers of the sm_103a kernels of the effective block
// algorithm (arXiv:1510.00903).  Host-callable, plain pointers.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace bbc {

// Device copy of one block-pair task (planner PairTask).
struct DevTask {
  int offA[8], offB[8];
  int nAnB;  // nA | nB << 8
  int n2;
  int sA;    // sA1 | sA2 << 16
  int sB;    // sB1 | sB2 << 16
};

struct DevGroups {  // block-build groups (rows that read the same tensor families)
  int n;
  int first[8], rows[8], fam0[8], fam1[8];
  int zneed_first[9];  // group gi computes tensor entries zneed[zneed_first[gi] .. zneed_first[gi+1])
};

constexpr int kMaxChannels = 64;
struct NormParams {  // per channel: host factor (1/V, mass normalisation) and quark counts
  int n_ch;
  double f[kMaxChannels];
  int nl[kMaxChannels], ns[kMaxChannels];
};

// Twiddle tables e^{-2 pi i k / 96} (double and float) into __constant__ memory.
cudaError_t upload_twiddles();

// |S| maximum of one propagator slice (V*144 complex, dtype 0 = c128, 1 = c64)
// into *amax (bit pattern of a non-negative double; caller zeroes it first).
cudaError_t launch_absmax(const void* src, int dtype, long long n_complex,
                          unsigned long long* amax, cudaStream_t st);
// dst = src * 2^-k with k = ilogb(max) + 1 (exact), k stored to *kexp.
cudaError_t launch_convert(const void* src, int dtype, long long n_complex,
                           const unsigned long long* amax, int* kexp, void* dst, bool fp64,
                           cudaStream_t st);
// Baryon blocks of every site: prop [slots][2][V][144], blk [slots][V][n_out].
cudaError_t launch_block_build(const void* prop, int V, int n_slots, const int* row_ptr,
                               const uint32_t* entries, const uint16_t* zneed, const DevGroups& g,
                               void* blk, int n_out, bool fp64, cudaStream_t st);
// In-place 1-D DFTs of length L along `axis` of data[n_outer][V][n_inner];
// storage and compute precision: fp64_store / fp64_compute; inverse = e^{+i}.
cudaError_t launch_fft_pass(void* data, int L, long long n_outer, int n_inner, int axis,
                            bool inverse, bool fp64_store, bool fp64_compute, cudaStream_t st);
// q-space contraction of one slice: blk [V][n_out] -> out [n_ch][V][16] (c128).
// qlist[n_q]: one q of every pair {q, -q} (FP32 path); tasks, per-thread
// schedule (sched_ptr[threads+1], units {task, k0 | k1 << 16}) and the signed
// sums (cptr, citem, ccoef) over task products P[task*16 + rA*nB + rB].
int contract_threads(bool fp64);
size_t contract_smem(bool fp64, int n_out, int n_tasks);
cudaError_t launch_contract(const void* blk, int L, int n_out, const int* qlist, int n_q, const DevTask* tasks,
                            int n_tasks, const int* sched_ptr, const int2* units, const int* cptr,
                            const int* citem, const double* ccoef, int n_ch, void* out, bool fp64,
                            cudaStream_t st);
// out[ch][r][s] *= f[ch] * 2^(nl[ch] k_l + ns[ch] k_s).
cudaError_t launch_normalise(void* out, int V, const NormParams& p, const int* kexp,
                             cudaStream_t st);

}  // namespace bbc
