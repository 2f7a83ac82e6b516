// tensor_split.cpp -- host schedule of the tensor-core q-space contraction.
//
// The products of Sec. 3 Eq. LN.pLLp.FFT, sum_k A(q; k) B(-q; k), come in
// the plan as block-pair tasks (planner.cpp).  For most of the work both
// operands are whole aggregated blocks with their open index pairs
// (c, alpha) x (c', alpha') laid out as a 12 x 12 matrix M[u][v] (row
// offset 12 u + v), read by the A side as M_A[i1][i2] and by the B side as
// M_B[i2][i1]: the product is the trace tr(M_A(q) M_B(-q)).  Over all such
// blocks i, j this is one dense matrix product per pair {q, -q},
//
//   G(q)[i][j] = sum_{u,v} M_i(q)[u][v] M_j(-q)[v][u],
//
// and G(-q)[i][j] = tr(M_i(-q) M_j(q)) = tr(M_j(q) M_i(-q)) = G(q)[j][i], so
// one product serves both q and -q.  This file picks those tasks, lays out
// G's tiles for the tensor-core kernel, moves the remaining tasks onto a
// compact copy of the rows they read (CUDA-core products), and rewrites the
// signed sums over Wick diagrams to read either kind of product.
#include <algorithm>
#include <map>
#include <set>
#include <string>

#include "kernels.cuh"
#include "planner.hpp"

namespace bbc {

namespace {

bool trace_form(const PairTask& t) {
  return t.nA == 4 && t.nB == 4 && t.n1 == 12 && t.n2 == 12 && t.sA1 == 12 && t.sA2 == 1 && t.sB1 == 1 &&
         t.sB2 == 12;
}

}  // namespace

void tc_units(const TcSplit& S, int tiles, std::vector<int>* units) {
  // one m-tile and up to `tiles` consecutive n-tiles per warp (unneeded tiles
  // inside a run are computed and not read)
  units->clear();
  for (int mt = 0; mt < S.mt_n; mt++) {
    int nt = 0;
    while (nt < S.nt_n) {
      if (!S.need[(size_t)mt * S.nt_n + nt]) { nt++; continue; }
      int cnt = 1;
      while (nt + cnt < S.nt_n && cnt < tiles && S.need[(size_t)mt * S.nt_n + nt + cnt]) cnt++;
      units->push_back(mt | (nt << 8) | (cnt << 16));
      nt += cnt;
    }
  }
}

bool split_tensor_tasks(const Plan& plan, TcSplit* out, std::string* err) {
  TcSplit S;
  const int n_tasks = (int)plan.tasks.size();
  std::vector<char> tc(n_tasks, 0);
  std::set<int> bases;
  for (int t = 0; t < n_tasks; t++) {
    const PairTask& k = plan.tasks[t];
    if (!trace_form(k)) continue;
    tc[t] = 1;
    for (int r = 0; r < 4; r++) {
      bases.insert(k.offA[r]);
      bases.insert(k.offB[r]);
    }
  }
  S.base.assign(bases.begin(), bases.end());
  S.nb = (int)S.base.size();
  // blocks must be disjoint 144-row ranges inside the block rows
  for (int i = 0; i < S.nb; i++) {
    if (S.base[i] < 0 || S.base[i] + 144 > plan.n_out || (i && S.base[i] < S.base[i - 1] + 144)) {
      *err = "internal: tensor-core blocks overlap";
      return false;
    }
  }
  // the kernel stages blocks with 16-byte loads: rows of an even length, blocks at even rows
  bool aligned = (plan.n_out & 1) == 0;
  for (int b : S.base) aligned &= (b & 1) == 0;
  if (S.nb == 0 || S.nb > kMaxTcBlocks || !aligned) {
    S.nb = 0;  // nothing for the tensor cores (or too many blocks): every task stays on the CUDA cores
    std::fill(tc.begin(), tc.end(), 0);
    S.base.clear();
  }
  std::map<int, int> block_of;
  for (int i = 0; i < S.nb; i++) block_of[S.base[i]] = i;
  S.nbp = (S.nb + 15) / 16 * 16;
  // tiles of G with a needed entry: (i, j) for side q and (j, i) for side -q
  const int mt_n = S.nbp / 16, nt_n = S.nbp / 8;
  std::vector<char> need((size_t)mt_n * nt_n, 0);
  for (int t = 0; t < n_tasks; t++) {
    if (!tc[t]) continue;
    const PairTask& k = plan.tasks[t];
    for (int ra = 0; ra < 4; ra++)
      for (int rb = 0; rb < 4; rb++) {
        const int i = block_of[k.offA[ra]], j = block_of[k.offB[rb]];
        need[(size_t)(i / 16) * nt_n + j / 8] = 1;
        need[(size_t)(j / 16) * nt_n + i / 8] = 1;
      }
  }
  S.need = need;
  S.mt_n = mt_n;
  S.nt_n = nt_n;
  tc_units(S, kTcTilesPerWarp, &S.units);
  if ((int)S.units.size() > kTcMaxWarps) {
    *err = "internal: tensor-core tiles exceed one CTA's warps";
    return false;
  }
  // the other tasks on compact rows: every operand row's run of rows is kept
  // whole (its open-index strides stay valid) and the runs are packed in order
  std::vector<std::pair<int, int>> runs;
  for (int t = 0; t < n_tasks; t++) {
    if (tc[t]) continue;
    const PairTask& k = plan.tasks[t];
    const int extA = (k.n1 - 1) * k.sA1 + (k.n2 - 1) * k.sA2, extB = (k.n1 - 1) * k.sB1 + (k.n2 - 1) * k.sB2;
    if (extA < 0 || extB < 0) {
      *err = "internal: negative open-index stride";
      return false;
    }
    for (int r = 0; r < k.nA; r++) runs.push_back({k.offA[r], k.offA[r] + extA});
    for (int r = 0; r < k.nB; r++) runs.push_back({k.offB[r], k.offB[r] + extB});
  }
  std::sort(runs.begin(), runs.end());
  std::vector<std::pair<int, int>> merged;
  for (const auto& r : runs) {
    if (!merged.empty() && r.first <= merged.back().second)
      merged.back().second = std::max(merged.back().second, r.second);
    else
      merged.push_back(r);
  }
  std::vector<int> compact(plan.n_out, -1);
  for (const auto& m : merged)
    for (int row = m.first; row <= m.second; row++) {
      if (row < 0 || row >= plan.n_out) {
        *err = "internal: task reads outside the block rows";
        return false;
      }
      compact[row] = (int)S.row_src.size();
      S.row_src.push_back(row);
    }
  S.rest.n_out = (int)S.row_src.size();
  // A task of shape 2 x 8 runs as the 8 x 2 task with its operands swapped:
  // sum_k B(q; k) A(-q; k) is the original product at -q, transposed, so the
  // kernel's two sides trade places and the swapped tasks share the lanes of
  // one batch class with the 8 x 2 ones.
  std::vector<int> rest_index(n_tasks, -1);
  std::vector<char> swapped(n_tasks, 0);
  for (int t = 0; t < n_tasks; t++) {
    if (tc[t]) continue;
    PairTask k = plan.tasks[t];
    for (int r = 0; r < k.nA; r++) k.offA[r] = compact[k.offA[r]];
    for (int r = 0; r < k.nB; r++) k.offB[r] = compact[k.offB[r]];
    if (k.nA == 2 && k.nB == 8) {
      PairTask w = k;
      w.nA = k.nB;
      w.nB = k.nA;
      for (int r = 0; r < 8; r++) {
        w.offA[r] = r < k.nB ? k.offB[r] : 0;
        w.offB[r] = r < k.nA ? k.offA[r] : 0;
      }
      w.sA1 = k.sB1;
      w.sA2 = k.sB2;
      w.sB1 = k.sA1;
      w.sB2 = k.sA2;
      k = w;
      swapped[t] = 1;
    }
    rest_index[t] = (int)S.rest.tasks.size();
    S.rest.tasks.push_back(k);
  }
  for (const PairTask& k : S.rest.tasks) S.rest.pair_macs += 16LL * k.n1 * k.n2;
  S.tc_macs = plan.pair_macs - S.rest.pair_macs;
  // signed sums: V = [P_q (np) | P_-q (np) | G (nbp x nbp)]; a rest task's
  // product i sits at 16 t + ((i + t) & 15) (the kernel's bank rotation)
  const int np = 16 * (int)S.rest.tasks.size();
  S.out_ptr.assign(1, 0);
  for (size_t o = 0; o + 1 < plan.tcontrib_ptr.size(); o++) {
    for (int c = plan.tcontrib_ptr[o]; c < plan.tcontrib_ptr[o + 1]; c++) {
      const int item = plan.tcontrib_item[c], t = item >> 4, i = item & 15;
      const PairTask& k = plan.tasks[t];
      int sq, smq;
      if (tc[t]) {
        const int ra = i / k.nB, rb = i % k.nB;
        const int a = block_of[k.offA[ra]], b = block_of[k.offB[rb]];
        sq = 2 * np + a * S.nbp + b;
        smq = 2 * np + b * S.nbp + a;
      } else if (!swapped[t]) {
        const int rt = rest_index[t];
        sq = 16 * rt + ((i + rt) & 15);
        smq = np + sq;
      } else {  // product (rA, rB) of the original is (rB, rA) of the swapped task, sides exchanged
        const int rt = rest_index[t], ra = i / k.nB, rb = i % k.nB, j = rb * k.nA + ra;
        smq = 16 * rt + ((j + rt) & 15);
        sq = np + smq;
      }
      S.coef.push_back(plan.tcontrib_coef[c]);
      S.src_q.push_back(sq);
      S.src_mq.push_back(smq);
    }
    S.out_ptr.push_back((int)S.coef.size());
  }
  std::map<double, int> distinct;
  for (double x : S.coef) {
    auto it = distinct.find(x);
    if (it == distinct.end()) {
      it = distinct.emplace(x, (int)S.coef_values.size()).first;
      S.coef_values.push_back(x);
    }
    S.coef_index.push_back(it->second);
  }
  *out = std::move(S);
  return true;
}

}  // namespace bbc
