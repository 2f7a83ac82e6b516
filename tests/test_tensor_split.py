"""Host check of the tensor-core split of the q-space contraction (CPU).

The planner's C++ and the split (tensor_split.cpp) are compiled with g++ into
a checker that evaluates, for one pair {q, -q} with random complex block rows,
the signed sums over Wick diagrams twice in FP64:

* as the plan states them: every block-pair product sum_k A(q; k) B(-q; k)
  (and A(-q; k) B(q; k) for -q) over its open index, then the signed sums;
* as the kernels run them: G(q)[i][j] = sum_{u,v} M_i(q)[u][v] M_j(-q)[v][u]
  over the split's blocks (the tensor-core product, read at [i][j] for q and
  at [j][i] for -q), the other products on the compact rows (row i = block row
  row_src[i]) at the kernel's rotated slots, and the sums through the
  split's (coef, source q, source -q) table.

The two must agree to rounding (1e-12 of the largest output).  It also checks
that G's warp tiles cover every entry the sums read and stay inside G, that
the CUDA-core kernel's shared-memory row map keeps every task's strides, and
that the work is conserved.  A planted mistake (G read untransposed for -q)
must fail.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1510_00903_gb300", "csrc")


def cuda_include():
    nvcc = shutil.which("nvcc")
    home = os.path.dirname(os.path.dirname(os.path.realpath(nvcc))) if nvcc else "/usr/local/cuda"
    return os.path.join(home, "include")


CHECKER = r"""
#include "kernels.cuh"
#include "planner.hpp"
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <string>
#include <vector>
using namespace bbc;
using C = std::complex<double>;
#define CHECK(c, msg) do { if (!(c)) { std::printf("FAIL %s\n", msg); return 1; } } while (0)

static C prod(const std::vector<C>& A, const std::vector<C>& B, const PairTask& t, int ra, int rb) {
  C s = 0;
  for (int i1 = 0; i1 < t.n1; i1++)
    for (int i2 = 0; i2 < t.n2; i2++)
      s += A[t.offA[ra] + i1 * t.sA1 + i2 * t.sA2] * B[t.offB[rb] + i1 * t.sB1 + i2 * t.sB2];
  return s;
}

static int check(const std::vector<int>& ch, int off, int plant) {
  Plan P;
  std::string err;
  if (!build_plan(ch.data(), (int)ch.size(), &P, &err, off)) { std::printf("FAIL plan %s\n", err.c_str()); return 1; }
  TcSplit S;
  if (!split_tensor_tasks(P, &S, &err)) { std::printf("FAIL split %s\n", err.c_str()); return 1; }
  std::mt19937_64 rng(7);
  std::normal_distribution<double> nd;
  std::vector<C> Fq(P.n_out), Fmq(P.n_out);
  for (auto& x : Fq) x = C(nd(rng), nd(rng));
  for (auto& x : Fmq) x = C(nd(rng), nd(rng));
  // as the plan states them
  const int n_o = (int)P.tcontrib_ptr.size() - 1;
  std::vector<C> ref_q(n_o), ref_mq(n_o);
  double scale = 0;
  for (int o = 0; o < n_o; o++) {
    for (int c = P.tcontrib_ptr[o]; c < P.tcontrib_ptr[o + 1]; c++) {
      const int it = P.tcontrib_item[c], t = it >> 4, i = it & 15;
      const PairTask& k = P.tasks[t];
      ref_q[o] += P.tcontrib_coef[c] * prod(Fq, Fmq, k, i / k.nB, i % k.nB);
      ref_mq[o] += P.tcontrib_coef[c] * prod(Fmq, Fq, k, i / k.nB, i % k.nB);
    }
    scale = std::max(scale, std::max(std::abs(ref_q[o]), std::abs(ref_mq[o])));
  }
  // as the kernels run them
  const int nt = (int)S.rest.tasks.size(), np = 16 * nt, nbp = S.nbp;
  std::vector<C> V(2 * np + nbp * nbp);
  for (int i = 0; i < S.nb; i++)
    for (int j = 0; j < S.nb; j++) {
      C g = 0;
      for (int u = 0; u < 12; u++)
        for (int v = 0; v < 12; v++) g += Fq[S.base[i] + 12 * u + v] * Fmq[S.base[j] + 12 * v + u];
      V[2 * np + i * nbp + j] = g;
    }
  std::vector<C> Rq(S.rest.n_out), Rmq(S.rest.n_out);
  for (int r = 0; r < S.rest.n_out; r++) { Rq[r] = Fq[S.row_src[r]]; Rmq[r] = Fmq[S.row_src[r]]; }
  for (int t = 0; t < nt; t++) {
    const PairTask& k = S.rest.tasks[t];
    for (int i = 0; i < 16; i++) {
      V[16 * t + ((i + t) & 15)] = prod(Rq, Rmq, k, i / k.nB, i % k.nB);
      V[np + 16 * t + ((i + t) & 15)] = prod(Rmq, Rq, k, i / k.nB, i % k.nB);
    }
  }
  CHECK((int)S.out_ptr.size() == n_o + 1, "output table size");
  double worst = 0;
  for (int o = 0; o < n_o; o++) {
    C gq = 0, gmq = 0;
    for (int c = S.out_ptr[o]; c < S.out_ptr[o + 1]; c++) {
      int smq = S.src_mq[c];
      if (plant && smq >= 2 * np) smq = S.src_q[c];  // planted: G not transposed for -q
      CHECK(S.src_q[c] >= 0 && S.src_q[c] < (int)V.size() && smq >= 0 && smq < (int)V.size(), "source index");
      gq += S.coef[c] * V[S.src_q[c]];
      gmq += S.coef[c] * V[smq];
    }
    worst = std::max(worst, std::max(std::abs(gq - ref_q[o]), std::abs(gmq - ref_mq[o])));
  }
  CHECK(worst <= 1e-12 * scale, "signed sums through the split differ from the plan's");
  CHECK(S.coef_index.size() == S.coef.size(), "coefficient index per term");
  for (size_t c = 0; c < S.coef.size(); c++)
    CHECK(S.coef_index[c] >= 0 && S.coef_index[c] < (int)S.coef_values.size() &&
              S.coef_values[S.coef_index[c]] == S.coef[c], "coefficient table");
  // G's warp tiles: inside G, and covering every entry the sums read
  std::vector<char> cov((size_t)nbp * nbp, 0);
  CHECK((int)S.units.size() <= kTcMaxWarps, "warps");
  for (int u : S.units) {
    const int mt = u & 0xff, nt0 = (u >> 8) & 0xff, cnt = u >> 16;
    CHECK(cnt >= 1 && cnt <= kTcTilesPerWarp && 16 * (mt + 1) <= nbp && 8 * (nt0 + cnt) <= nbp, "tile inside G");
    for (int m = 16 * mt; m < 16 * mt + 16; m++)
      for (int n = 8 * nt0; n < 8 * (nt0 + cnt); n++) cov[(size_t)m * nbp + n]++;
  }
  for (size_t c = 0; c < S.coef.size(); c++)
    for (int s : {S.src_q[c], S.src_mq[c]})
      if (s >= 2 * np) CHECK(cov[s - 2 * np] == 1, "G entry computed by exactly one warp");
  // the rest kernel's shared-memory row map keeps every task side's strides
  if (nt > 0) {
    std::vector<Batch> batches;
    make_batches(S.rest, &batches);
    FusedLayout lay;
    optimise_fused_layout(S.rest, &batches, &lay);
    CHECK((int)lay.row_slot.size() == S.rest.n_out, "rest row map size");
    for (int r = 1; r < S.rest.n_out; r++) CHECK(lay.row_slot[r] > lay.row_slot[r - 1], "rest row map increasing");
    for (const PairTask& t : S.rest.tasks)
      for (int side = 0; side < 2; side++) {
        const int n = side ? t.nB : t.nA;
        const int* o = side ? t.offB : t.offA;
        const int s1 = side ? t.sB1 : t.sA1, s2 = side ? t.sB2 : t.sA2;
        for (int r = 0; r < n; r++)
          for (int i1 = 0; i1 < t.n1; i1++)
            for (int i2 = 0; i2 < t.n2; i2++) {
              const int row = o[r] + i1 * s1 + i2 * s2;
              CHECK(row >= 0 && row < S.rest.n_out, "rest row inside the compact rows");
              CHECK(lay.row_slot[row] == lay.row_slot[o[r]] + i1 * s1 + i2 * s2, "rest slot strides");
              CHECK(lay.row_slot[row] < lay.n_slots, "rest slot inside");
            }
      }
    std::printf("rest smem %zu bytes (slots %d) ", (size_t)lay.n_slots * 16 + (size_t)2 * np * 8 + (size_t)nbp * nbp * 8,
                lay.n_slots);
  }
  long long macs = 0;
  for (const PairTask& k : P.tasks) macs += 16LL * k.n1 * k.n2;
  CHECK(S.tc_macs + S.rest.pair_macs == macs, "work conserved");
  std::printf("\nOK nb %d rest tasks %d of %zu, tensor-core share %.3f, max diff %.2e of %.2e\n", S.nb, nt,
              P.tasks.size(), (double)S.tc_macs / macs, worst, scale);
  return 0;
}

int main(int argc, char** argv) {
  // argv: plant, spin offset, then channel ids
  const int plant = std::atoi(argv[1]), off = std::atoi(argv[2]);
  std::vector<int> ch;
  for (int i = 3; i < argc; i++) ch.push_back(std::atoi(argv[i]));
  return check(ch, off, plant);
}
"""


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    d = tmp_path_factory.mktemp("tcsplit")
    src = d / "check.cpp"
    exe = d / "check"
    src.write_text(CHECKER)
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", CSRC, "-I", cuda_include(), "-o", str(exe), str(src),
                           os.path.join(CSRC, "planner.cpp"), os.path.join(CSRC, "tensor_split.cpp")])
    return str(exe)


LISTS = {
    "52": list(range(52)),
    "64 octet ids": list(range(64)),
    "90 decuplet ids": list(range(64, 154)),
    "one channel": [1],
    "p n only": [0],
    "Delta++ ids": list(range(154, 163)) + [397, 405],
    "Sigma*+ and Xi*0 ids": [235, 260, 300, 316, 340, 396],
}


@pytest.mark.parametrize("name", list(LISTS))
@pytest.mark.parametrize("off", [0, 2])
def test_split_reproduces_the_plans_sums(checker, name, off):
    r = subprocess.run([checker, "0", str(off)] + [str(c) for c in LISTS[name]], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "\nOK" in r.stdout, r.stdout + r.stderr
    print(name, r.stdout.strip())


def test_split_puts_most_octet_work_on_the_tensor_cores(checker):
    r = subprocess.run([checker, "0", "0"] + [str(c) for c in range(52)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout
    share = float(r.stdout.split("tensor-core share")[1].split(",")[0])
    assert share > 0.75  # 59 of the 153 tasks, 135,936 of the 174,208 complex MACs per site


def test_planted_untransposed_read_is_caught(checker):
    r = subprocess.run([checker, "1", "0"] + [str(c) for c in range(52)], capture_output=True, text=True, timeout=600)
    assert r.returncode != 0 and "differ" in r.stdout
