"""Host check of the dense-tuple FP32 block build (CPU).

The planner's C++ and dense_build.cpp are compiled with g++ into a checker
that emulates both block-build kernels on the host, in FP64, for one site
with random sink-tensor families F[slot][a][e0 e1][e2]:

* the entry-per-thread kernel: each group computes its zneed entries at their
  positions (entries of an unchanged family stay in place from the previous
  group), then every row sums weight x entry over its lane-interleaved chunk;
* the dense kernel: each group writes all twelve e2 entries of each of its
  tuples (slot, a, e0 e1) at e2 * stride + j, then the rows sum the re-addressed
  terms with the weight read from the top 16 bits as an FP32 value.

Every block row must agree (rounding only), positions must stay inside the
per-site entry storage, and a planted slip (tuple index off by one) must fail.
"""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1510_00903_gb300", "csrc")

CHECKER = r"""
#include "planner.hpp"
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <string>
#include <vector>
using namespace bbc;
using C = std::complex<double>;
#define CHECK(c, msg) do { if (!(c)) { std::printf("FAIL %s\n", msg); return 1; } } while (0)

static int check(const std::vector<int>& ch, int off, int plant) {
  Plan P;
  std::string err;
  if (!build_plan(ch.data(), (int)ch.size(), &P, &err, off)) { std::printf("FAIL plan %s\n", err.c_str()); return 1; }
  DenseBuild D;
  if (!make_dense_build(P, &D, &err)) { std::printf("FAIL dense %s\n", err.c_str()); return 1; }
  std::mt19937_64 rng(3);
  std::normal_distribution<double> nd;
  // F[family][local] for every family a group may hold
  std::vector<std::vector<C>> F(N_FAMILY, std::vector<C>(kFamEntries));
  for (auto& f : F) for (auto& x : f) x = C(nd(rng), nd(rng));
  // entry-per-thread kernel
  std::vector<C> zold(P.z_slots), rows_old(P.n_out), rows_new(P.n_out);
  for (size_t g = 0; g < P.groups.size(); g++) {
    const GroupInfo& gi = P.groups[g];
    for (int z = P.zneed_first[g]; z < P.zneed_first[g + 1]; z++) {
      const uint32_t zn = P.zneed[z];
      const int pos = zn & 0x1fff, sl = (zn >> 13) & 1, local = zn >> 14;
      zold[pos] = F[gi.fam[sl]][local];
    }
    for (int c = 0; c < (gi.n_rows + 31) / 32; c++) {
      const auto& chk = P.ell_chunk[P.chunk_first[g] + c];
      for (int l = 0; l < 32 && 32 * c + l < gi.n_rows; l++) {
        C acc = 0;
        for (int k = 0; k < chk.second; k++) {
          const uint32_t e = P.ell[chk.first + 32 * k + l];
          acc += (double)(int16_t)(e >> 16) * zold[e & 0xffff];
        }
        rows_old[gi.first_row + 32 * c + l] = acc;
      }
    }
  }
  // dense kernel
  CHECK((int)D.tuple_first.size() == (int)P.groups.size() + 1 && (int)D.chunk_first.size() == (int)P.groups.size() + 1,
        "table sizes");
  std::vector<C> znew(D.z_slots);
  for (size_t g = 0; g < P.groups.size(); g++) {
    const GroupInfo& gi = P.groups[g];
    const int t0 = D.tuple_first[g], nt = D.tuple_first[g + 1] - t0, str = D.stride[g];
    CHECK(str >= nt && (str & 1) && 12 * str <= D.z_slots, "stride");
    for (int j = 0; j < nt; j++) {
      const uint32_t tu = D.tuples[t0 + j];
      const int sl = tu / 288, a = (tu % 288) / 144, e01 = tu % 144;
      CHECK(gi.fam[sl] >= 0, "tuple family");
      for (int e2 = 0; e2 < 12; e2++) {
        const int jj = plant ? (j + 1) % nt : j;
        znew[e2 * str + jj] = F[gi.fam[sl]][a * 1728 + e01 * 12 + e2];
      }
    }
    for (int c = 0; c < (gi.n_rows + 31) / 32; c++) {
      const auto& chk = D.ell_chunk[D.chunk_first[g] + c];
      for (int l = 0; l < 32 && 32 * c + l < gi.n_rows; l++) {
        C acc = 0;
        for (int k = 0; k < chk.second; k++) {
          const uint32_t e = D.ell[chk.first + 32 * k + l];
          const uint32_t wb = e & 0xffff0000u;
          float w;
          std::memcpy(&w, &wb, sizeof w);
          CHECK((int)(e & 0xffff) < D.z_slots, "position inside");
          if (w == 0.f) CHECK((e & 0xffff) == 0, "padding at position 0");
          acc += (double)w * znew[e & 0xffff];
        }
        rows_new[gi.first_row + 32 * c + l] = acc;
      }
    }
  }
  double worst = 0, scale = 0;
  for (int r = 0; r < P.n_out; r++) {
    worst = std::max(worst, std::abs(rows_new[r] - rows_old[r]));
    scale = std::max(scale, std::abs(rows_old[r]));
  }
  CHECK(worst <= 1e-12 * scale, "dense rows differ");
  std::printf("OK rows %d groups %zu tuples %zu z_slots %d (entry-per-thread %d), max diff %.1e of %.1e\n",
              P.n_out, P.groups.size(), D.tuples.size(), D.z_slots, P.z_slots, worst, scale);
  return 0;
}

int main(int argc, char** argv) {
  const int plant = std::atoi(argv[1]), off = std::atoi(argv[2]);
  std::vector<int> ch;
  for (int i = 3; i < argc; i++) ch.push_back(std::atoi(argv[i]));
  return check(ch, off, plant);
}
"""


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    d = tmp_path_factory.mktemp("dense")
    src = d / "check.cpp"
    exe = d / "check"
    src.write_text(CHECKER)
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", CSRC, "-o", str(exe), str(src),
                           os.path.join(CSRC, "planner.cpp"), os.path.join(CSRC, "dense_build.cpp")])
    return str(exe)


LISTS = {"52": list(range(52)), "64 octet ids": list(range(64)), "90 decuplet ids": list(range(64, 154)),
         "octet and decuplet": list(range(52)) + list(range(64, 154)), "one channel": [1],
         "Delta++ and p Delta++": list(range(154, 235)) + list(range(397, 406)),
         "Sigma*+ pairs": list(range(235, 316)), "Xi*0 pairs": list(range(316, 397)),
         "every family": [0, 10, 51, 64, 150, 154, 200, 240, 300, 320, 396, 400]}


@pytest.mark.parametrize("name", list(LISTS))
@pytest.mark.parametrize("off", [0, 2])
def test_dense_rows_equal_the_entry_per_thread_rows(checker, name, off):
    r = subprocess.run([checker, "0", str(off)] + [str(c) for c in LISTS[name]], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout + r.stderr
    print(name, r.stdout.strip())


def test_planted_tuple_slip_is_caught(checker):
    r = subprocess.run([checker, "1", "0"] + [str(c) for c in range(52)], capture_output=True, text=True, timeout=600)
    assert r.returncode != 0 and "differ" in r.stdout
