// ctx_internal.hpp -- definition of the opaque bbc_ctx (internal to libbbc).
#pragma once

#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/bbc.h"
#include "kernels.cuh"
#include "planner.hpp"

struct bbc_ctx {
  bbc_lattice lat{};
  int prec = BBC_FP64;
  cudaStream_t stream = nullptr;
  int V = 0;
  bbc::Plan plan;
  mutable std::string err;  // last failure message (inspection calls on a const context set it too)
  // workspace view
  char* ws = nullptr;
  size_t ws_bytes = 0;
  int slots = 0;
  int2* d_ell_chunk = nullptr;           // (offset, length) of each 32-row chunk of block rows
  uint32_t* d_ell = nullptr;             // lane-interleaved row entries
  uint32_t* d_zneed = nullptr;
  bbc::DevTask* d_tasks = nullptr;
  int* d_group_ptr = nullptr;
  int* d_group_task = nullptr;
  int* d_cptr = nullptr;
  int* d_citem = nullptr;
  double* d_ccoef = nullptr;
  float2* d_ccoef_df = nullptr;          // the coefficients as double-float pairs (BBC_DF64)
  std::vector<int> group_ptr;            // warp task groups of the pair products (FP64)
  std::vector<int> group_task;
  // fused FP32 contraction: warp batches, per-warp units, one q per pair {q, -q}
  std::vector<bbc::Batch> batches;
  std::vector<int> wptr;
  std::vector<bbc::BatchUnit> wunits;
  std::vector<int> qlist;
  bbc::WarpBatch* d_batches = nullptr;
  int* d_wptr = nullptr;
  int4* d_wunits = nullptr;
  int* d_qlist = nullptr;
  // launch configuration (bbc_set_tuning / bbc_autotune)
  // FP32 / bfloat16 products in one fused kernel per pair {q, -q}; plans
  // whose rows and products do not fit one CTA's shared memory take the
  // unfused FP32 route (field-major FFT, pair products, Wick sums)
  bool fused = false;
  // mixed FP32 / TF32 with tensor cores: the trace-form block pairs as one
  // complex matrix product per pair {q, -q} (k_contract_tc), the other tasks
  // and the Wick sums in k_contract_rest; the fused fields above then
  // describe the rest kernel (its tasks, rows and warp units)
  bool tc = false;
  bbc::TcSplit tcs;
  // FP32 block build from dense entry tuples (k_block_build_dense)
  bool dense = false;
  bbc::DenseBuild db;
  uint32_t* d_dtuples = nullptr;
  int2* d_dchunk = nullptr;
  uint32_t* d_dell = nullptr;
  int* d_tc_base = nullptr;              // [nb] first block row of each block of G
  int* d_tc_units = nullptr;             // [warps] tiles of G per warp
  uint32_t* d_row_map = nullptr;         // [rest rows] block row | shared-memory slot << 16
  int* d_tc_cptr = nullptr;              // [n_ch*16 + 1] Wick-term ranges per output
  uint2* d_tc_terms = nullptr;           // [terms] (source q | source -q << 16, coefficient index)
  float2* d_tc_coefs = nullptr;          // [distinct coefficients] (hi, lo)
  char* d_G = nullptr;                   // [pairs][nbp][nbp] complex64
  bbc_tuning tune{1, 256, 16, 18, 1, 48, 0};
  size_t max_units = 0;                  // warp units the workspace holds (largest chunk candidate)
  std::vector<int> row_slot;             // shared-memory slot of every block row (bank layout)
  int n_slots = 0;
  int* d_row_slot = nullptr;
  // orbits of the cubic rotations on the lattice (bbc_project)
  std::vector<int> orb_ptr, orb_site;
  int* d_orb_ptr = nullptr;
  int* d_orb_site = nullptr;
  char* d_stage = nullptr;               // [slots][2][V*144] c128 staging of host input
  char* d_prop = nullptr;                // [slots][2][V*144] compute precision
  unsigned long long* d_amax = nullptr;  // [slots][2]
  int* d_kexp = nullptr;                 // [slots][2]
  char* d_blk = nullptr;                 // [slots][V][n_out] site-major build output
  char* d_blk16 = nullptr;               // [slots][V][n_out] bfloat16 (re, im) pairs, Fourier space
  char* d_blkf = nullptr;                // [slots][n_out][V] field-major, Fourier space
  double* d_blks = nullptr;              // [slots][n_out][V] re + im of d_blkf (BBC_FP64)
  char* d_P = nullptr;                   // [n_tasks*16][V] pair products of one slice
  char* d_ct = nullptr;                  // [n_ch*16][V] complex128 q-space correlators
  double* d_scale = nullptr;             // [kMaxChannels]
  int* d_flag = nullptr;                 // non-finite output flag (bbc_set_checks)
  int* d_qerr = nullptr;                 // sticky: a bounded wait of the queue-driven FFT gave up
  int* d_fftq = nullptr;                 // queue-driven FFT: ticket counter, per-tile counters
  int checks = 0;                        // BBC_CHECK_INPUT | BBC_CHECK_OUTPUT
  std::vector<int> slot_t;               // time slice of each slot (-1: none)
  std::vector<int> slot_loaded;          // bit 0: light, bit 1: strange
  std::vector<int> slot_built;
  bool twiddles = false;
  // stage timing: event pairs per stage, recycled through a pool
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending[BBC_N_STAGES];
  std::vector<cudaEvent_t> pool;
  // tensor-core contraction: a second stream and its fork / join events, so
  // that the CUDA-core half of one chunk of pairs {q, -q} runs beside the
  // tensor-core half of the next (created on first use)
  static constexpr int kTcChunks = 4;
  cudaStream_t side = nullptr;
  cudaEvent_t fork[kTcChunks] = {};
  cudaEvent_t join = nullptr;
  ~bbc_ctx() {
    for (auto& v : pending)
      for (auto& p : v) { cudaEventDestroy(p.first); cudaEventDestroy(p.second); }
    for (auto e : pool) cudaEventDestroy(e);
    for (auto e : fork)
      if (e) cudaEventDestroy(e);
    if (join) cudaEventDestroy(join);
    if (side) cudaStreamDestroy(side);
  }
};


namespace bbc {

// Device copies of plan tasks; with row_slot (fused kernels) the offsets
// become shared-memory slots (a task side's rows lie in one segment, so
// slot(off + k) = slot(off) + k).
inline void to_dev_tasks(const PairTask* src, size_t n, const std::vector<int>* row_slot, DevTask* dst) {
  for (size_t i = 0; i < n; i++) {
    const PairTask& t = src[i];
    DevTask& d = dst[i];
    for (int r = 0; r < 8; r++) {
      d.offA[r] = r < t.nA ? (row_slot ? (*row_slot)[t.offA[r]] : t.offA[r]) : 0;
      d.offB[r] = r < t.nB ? (row_slot ? (*row_slot)[t.offB[r]] : t.offB[r]) : 0;
    }
    d.nAnB = t.nA | (t.nB << 8);
    d.n1 = t.n1;
    d.n2 = t.n2;
    d.sA = t.sA1 | (t.sA2 << 16);
    d.sB = t.sB1 | (t.sB2 << 16);
  }
}

static_assert(N_DIQUARK == kMaxDiquarks && N_FAMILY == kMaxFamilies && kMaxGroups == kMaxBuildGroups,
              "diquark, family and group tables");

// The block-build groups of a plan as the kernel reads them: row ranges,
// families per tensor slot, and the diquarks (flavours, Gamma1) those
// families are made of, in the plan's shared-memory order.
inline DevGroups dev_groups(const Plan& p, const DenseBuild* db = nullptr) {
  DevGroups g{};
  if (db) {  // the dense-tuple FP32 build's tables
    for (size_t i = 0; i < db->tuple_first.size() && i <= (size_t)kMaxBuildGroups; i++)
      g.tuple_first[i] = db->tuple_first[i];
    for (size_t i = 0; i < db->stride.size() && i < (size_t)kMaxBuildGroups; i++) g.stride[i] = db->stride[i];
    for (size_t i = 0; i < db->chunk_first.size() && i <= (size_t)kMaxBuildGroups; i++)
      g.dchunk_first[i] = db->chunk_first[i];
    g.dense_z_slots = db->z_slots;
  }
  g.n = (int)p.groups.size();
  for (int i = 0; i < g.n; i++) {
    g.first[i] = p.groups[i].first_row;
    g.rows[i] = p.groups[i].n_rows;
    g.fam0[i] = p.groups[i].fam[0];
    g.fam1[i] = p.groups[i].fam[1];
  }
  for (int i = 0; i <= g.n; i++) g.zneed_first[i] = p.zneed_first[i];
  g.z_slots = p.z_slots;
  g.spin0 = p.spin_offset;
  for (int i = 0; i <= g.n; i++) g.chunk_first[i] = p.chunk_first[i];
  g.n_dq = (int)p.diquarks.size();
  for (int j = 0; j < g.n_dq; j++) {
    const int d = p.diquarks[j];
    g.dq_f0[j] = kDqFlavour[d][0];
    g.dq_f1[j] = kDqFlavour[d][1];
    g.dq_gam[j] = kDqGamma[d];
  }
  for (int f = 0; f < N_FAMILY; f++) {
    g.fam_dq[f] = 0;  // families no group reads point at diquark 0
    for (int j = 0; j < g.n_dq; j++)
      if (p.diquarks[j] == kFamDiquark[f]) g.fam_dq[f] = j;
    g.fam_f2[f] = kFamThird[f];
  }
  return g;
}

}  // namespace bbc
