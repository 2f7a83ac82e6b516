// planner.hpp -- host-side contraction planner of the effective block algorithm.
//
// Turns a list of baryon-baryon channels into (a) the aggregated baryon
// blocks, each a sparse linear functional of per-site sink tensors, and
// (b) the q-space contraction as block-pair products and signed sums into
// channels (Nemura, arXiv:1510.00903, Sec. 3 diagrams (i)-(vi) and Eq.
// LN.pLLp.FFT; Sec. 4 for all channels; Appendix A for block sharing).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace bbc {

// Sink-tensor families: the diquark pair and the third (delta) quark of a
// baryon term, by numeric flavour (l = u = d, s) and diquark matrix Gamma1
// (C gamma5 for the octet; eta_l C gamma_l, l = x, y, z, for the decuplet of
// the Sec. 4 footnote: Omega (s s s), Delta++ (l l l), Sigma*+ (l l s and
// l s l terms), Xi*0 (s s l and l s s terms)):
//   F[a][e0][e1][e2] = sum eps(c0,c1,c2) Gamma1(a0,a1) S_f0[(a0,c0),e0] S_f1[(a1,c1),e1] S_f2[(a,c2),e2]
enum Family {
  F_LLL = 0, F_LLS = 1, F_LSL = 2, F_LSS = 3,  // C gamma5
  F_SSS_X = 4, F_SSS_Y = 5, F_SSS_Z = 6,       // eta_l C gamma_l, l = x, y, z (each vector family below too)
  F_LLLV_X = 7, F_LLSV_X = 10, F_LSLV_X = 13, F_LSSV_X = 16, F_SSLV_X = 19,
  N_FAMILY = 22
};
// Diquarks D[e0][e1][c2] = sum eps Gamma1(a0,a1) S_f0[(a0,c0),e0] S_f1[(a1,c1),e1]
// the families read: (l, l) and (l, s) with C gamma5; (s, s), (l, l) and
// (l, s) with eta_l C gamma_l.
enum Diquark { DQ_LL5 = 0, DQ_LS5 = 1, DQ_SSX = 2, DQ_LLX = 5, DQ_LSX = 8, N_DIQUARK = 11 };
// Diquark and strange third quark (0 / 1) of each family.
constexpr int kFamDiquark[N_FAMILY] = {DQ_LL5,  DQ_LL5,     DQ_LS5,     DQ_LS5,     DQ_SSX,     DQ_SSX + 1,
                                       DQ_SSX + 2, DQ_LLX,  DQ_LLX + 1, DQ_LLX + 2, DQ_LLX,     DQ_LLX + 1,
                                       DQ_LLX + 2, DQ_LSX,  DQ_LSX + 1, DQ_LSX + 2, DQ_LSX,     DQ_LSX + 1,
                                       DQ_LSX + 2, DQ_SSX,  DQ_SSX + 1, DQ_SSX + 2};
constexpr int kFamThird[N_FAMILY] = {0, 1, 0, 1, 1, 1, 1, 0, 0, 0, 1, 1, 1, 0, 0, 0, 1, 1, 1, 0, 0, 0};
// Exchange symmetry of a family's first two indices (e0, e1): +1 for a
// C gamma5 diquark of two equal flavours (eps and C gamma5 both
// antisymmetric), -1 for a vector diquark of two equal flavours (eta_l C
// gamma_l is symmetric), 0 for two different flavours.
constexpr int kFamSym[N_FAMILY] = {1, 1, 0, 0, -1, -1, -1, -1, -1, -1, -1, -1, -1, 0, 0, 0, 0, 0, 0, -1, -1, -1};
// Flavours (0 light, 1 strange) and Gamma1 (0 = C gamma5, l = eta_l C gamma_l) of each diquark.
constexpr int kDqFlavour[N_DIQUARK][2] = {{0, 0}, {0, 1}, {1, 1}, {1, 1}, {1, 1}, {0, 0},
                                          {0, 0}, {0, 0}, {0, 1}, {0, 1}, {0, 1}};
constexpr int kDqGamma[N_DIQUARK] = {0, 0, 1, 2, 3, 1, 2, 3, 1, 2, 3};
// Block-build groups (rows that read the same families) a plan may have.
constexpr int kMaxGroups = 16;
constexpr int kFamEntries = 2 * 1728;  // sink spin a in {0,1} (upper) x 12^3

struct GroupInfo {
  int first_row, n_rows;  // block-output rows of this group
  int fam[2];             // families held in the two tensor slots (-1 = unused)
};

// One aligned block pair at one q: P[rA][rB] = sum_k A[offA[rA] + k] B[offB[rB] + k]
// over the flattened open index k = (i1, i2) (offsets i1*s1 + i2*s2); rA runs
// over (sink spin a, external spins carried by A), rB likewise for B, and
// nA * nB = 16 spin combinations.
struct PairTask {
  int nA, nB;            // (2,8), (4,4) or (8,2)
  int offA[8], offB[8];  // row offsets in the block row of one site
  int n1, n2, sA1, sA2, sB1, sB2;
};

struct DiagramInfo {
  int ch_pos, term3, term4;  // channel position, source operator terms
  int K;                     // open-index iterations
  int parity;                // parity of the Wick permutation (+1 / -1)
  double coef;               // parity x operator coefficients
};

struct Plan {
  std::vector<int> channels;
  // Dirac index of the first external spin component: 0 for the upper two
  // components (0, 1), 2 for the lower two (2, 3) of every external spinor
  // index (Sec. 5); every external spin below is relative to it.
  int spin_offset = 0;
  // block build: rows (block outputs per site) grouped by the families they read
  int n_out = 0;
  int n_blocks = 0;
  std::vector<GroupInfo> groups;
  std::vector<int> row_ptr;          // n_out + 1
  std::vector<uint32_t> entries;     // low 16 bits: compact position of a tensor entry in shared memory,
                                     // high 16 bits: signed integer weight
  // The same rows as 32-row chunks (chunk j of group g: rows first_row + 32j ..
  // + 31) stored lane-interleaved: entry k of the chunk's lane l at
  // ell[ell_chunk[c].x + 32 k + l], k < ell_chunk[c].y (the chunk's longest
  // row; shorter rows padded with weight-0 entries at position 0), so a warp
  // reading entry k of 32 consecutive rows reads 128 contiguous bytes.
  std::vector<int> chunk_first;      // groups + 1: first chunk of each group
  std::vector<std::pair<int, int>> ell_chunk;  // (offset, length) per chunk
  std::vector<uint32_t> ell;
  std::vector<int> diquarks;         // the Diquark kinds the groups' families need, in shared-memory order
  std::vector<uint32_t> zneed;       // entries each group computes: pos | slot << 13 | (a*1728 + e0*144 + e1*12 + e2) << 14
  std::vector<int> zneed_first;      // groups + 1 offsets into zneed
  int z_slots = 0;                   // shared-memory positions needed (max over groups)
  // contraction: unique aligned pair products and their signed sums into channels
  std::vector<PairTask> tasks;       // products of block pairs; P index = task*16 + rA*nB + rB
  std::vector<int> tcontrib_ptr;     // n_channels*16 + 1, contributions over task products
  std::vector<int> tcontrib_item;
  std::vector<double> tcontrib_coef;
  long long pair_macs = 0;           // complex multiply-adds of all task products per site
  // normalisation data per channel position
  std::vector<int> n_strange;        // strange quarks of the sink pair (light = 6 - n_strange)
  // statistics for the paper's tables
  std::vector<DiagramInfo> diagrams;
};

// Number of supported channel ids (52 printed, 4 omitted, 8 other charge
// states, 81 Omega Omega, 9 p Omega).
int channel_count();
// Names of the four baryons of a channel (B1, B2 | B3, B4).
void channel_names(int id, const char* out[4]);
// Build the plan; returns false and sets *err on a bad channel list.
// spin_offset: 0 (upper components) or 2 (lower components).
bool build_plan(const int* channels, int n, Plan* plan, std::string* err, int spin_offset = 0);

// Warp batches for the fused contraction: tasks grouped by (nA, nB, n1*n2),
// at most 32 per batch (one per lane).
struct Batch {
  int nA;
  std::vector<int> tasks;
};
struct BatchUnit {
  int batch, side, k0, k1;
};
void make_batches(const Plan& plan, std::vector<Batch>* batches);
// Warp units (batch, k0, k1) covering both sides {q, -q}.  chunk > 0: open
// indices longer than `chunk` are split and units go longest first to the
// least loaded of `warps` warps; chunk = 0: the batches' steps laid end to
// end are cut into `warps` contiguous pieces of equal modelled cost.
// Output: warp_ptr[warps + 1], units.
void make_units(const Plan& plan, const std::vector<Batch>& batches, int warps, int chunk, std::vector<int>* warp_ptr,
                std::vector<BatchUnit>* units);

// Shared-memory row layout of the fused contraction.  The block rows one task
// side reads lie in one operand segment (the union of overlapping operand
// spans); a segment's rows move together by shift[s] (so a task's open-index
// strides are unchanged), and only shift mod 8 decides the bank group of a
// 16-byte row (eight groups of four 4-byte banks).  optimise_fused_layout
// chooses the segment shifts and the task order inside every class of
// batches (tasks may trade places between batches of one class) to minimise
// the shared-memory wavefronts of the products' 128-bit loads, on an exact
// model of the banks: a warp's 128-bit load runs as four phases of eight
// lanes; distinct addresses in one bank group serialise, equal ones broadcast.
struct FusedLayout {
  std::vector<int> row_slot;  // n_out: shared-memory slot of each block row
  int n_slots = 0;            // slots including the gaps
  long long wavefronts = 0;   // modelled 128-bit wavefronts of one {q, -q} pair
  long long ideal = 0;        // the same without any bank conflict
};
void optimise_fused_layout(const Plan& plan, std::vector<Batch>* batches, FusedLayout* out);

// FP32 block build with dense entry tuples (dense_build.cpp): per group, the
// tuples (family slot, a, e0 e1) its rows read; one thread forms the twelve
// e2 entries of a tuple at positions e2 * stride + j; the rows re-addressed
// to them as 32-row lane-interleaved chunks, entry = position | (weight as
// bfloat16 bits in the top 16 bits).
struct DenseBuild {
  std::vector<uint32_t> tuples;      // group by group: slot * 288 + a * 144 + e01
  std::vector<int> tuple_first;      // groups + 1
  std::vector<int> stride;           // per group (odd, >= its tuple count)
  int z_slots = 0;                   // entry positions per site (max over groups)
  std::vector<int> chunk_first;      // groups + 1
  std::vector<std::pair<int, int>> ell_chunk;
  std::vector<uint32_t> ell;
};
bool make_dense_build(const Plan& plan, DenseBuild* out, std::string* err);

// Tensor-core split of a plan (tensor_split.cpp).  Tasks whose operands are
// whole 12 x 12 blocks in the trace form tr(M_A(q) M_B(-q)) become entries
// of one complex matrix product per pair {q, -q} over the blocks they read,
//   G(q)[i][j] = sum_{u,v} M_i(q)[u][v] M_j(-q)[v][u],  G(-q) = G(q)^T;
// the other tasks keep the CUDA-core products on a compact copy of the rows
// they read.  (G's limits kMaxTcBlocks, kTcTilesPerWarp, kTcMaxWarps are in
// kernels.cuh.)
struct TcSplit {
  int nb = 0, nbp = 0;               // blocks in G, and nb rounded up to 16 (G is nbp x nbp)
  std::vector<int> base;             // nb: first block row of each block (M[u][v] at base + 12 u + v)
  std::vector<int> units;            // per warp: m-tile | first n-tile << 8 | n-tiles << 16
  long long tc_macs = 0;             // complex multiply-adds per site taken by G (as the plan counts them)
  Plan rest;                         // the other tasks (tasks, pair_macs, n_out = compact rows)
  std::vector<int> row_src;          // rest.n_out: block row behind each compact row
  // signed sums over Wick diagrams into output o = 16 channel_pos + spin:
  // terms [out_ptr[o], out_ptr[o+1]) of coef x V[src_q] for q and coef x
  // V[src_mq] for -q, V = [P_q (16 n_rest) | P_-q (16 n_rest) | G (nbp^2)]
  std::vector<int> out_ptr;
  std::vector<double> coef;
  std::vector<int> src_q, src_mq;
  std::vector<double> coef_values;   // the distinct coefficients (exact copies)
  std::vector<int> coef_index;       // per term: its coefficient in coef_values
  std::vector<char> need;            // [mt_n][nt_n]: 16 x 8 tiles of G with an entry the sums read
  int mt_n = 0, nt_n = 0;
};
// Warp units of G for `tiles` (2 or 3) n-tiles per warp.
void tc_units(const TcSplit& split, int tiles, std::vector<int>* units);
// nb = 0 when no task has the trace form (or G would exceed kMaxTcBlocks):
// then every task is in rest.  Returns false only on an internal inconsistency.
bool split_tensor_tasks(const Plan& plan, TcSplit* out, std::string* err);

// Partition of the tasks into `groups` lists of near-equal cost (longest task
// first to the cheapest list); each list is run by one warp for 32 q at a time.
// by_shape: lists hold tasks of one shape (nA) only and come shape by shape,
// so warps that run side by side run the same code (instruction cache).
void make_task_groups(const Plan& plan, int groups, std::vector<int>* group_ptr, std::vector<int>* group_task,
                      bool by_shape = false);

}  // namespace bbc
