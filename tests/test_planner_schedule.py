"""Host schedules of the contraction kernels (CPU): the planner's C++ is
compiled with g++ into a small checker, which verifies for several channel
lists and every launch-shape candidate that

* the warp task lists of the block-pair products hold every task once;
* the warp batches of the fused contraction hold every task once, with one
  shape and one open-index length per batch, at most 32 tasks;
* the shared-memory row map is increasing and keeps every task side's rows
  at the planner's strides (the kernel addresses slot(off) + i1 s1 + i2 s2);
* the warp units of every (warps, chunk) candidate cover each batch's open
  index exactly once;
* the block build's lane-interleaved 32-row chunks hold exactly each row's
  terms (in the bank-conflict order) and weight-0 padding at position 0.
"""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1510_00903_gb300", "csrc")

CHECKER = r"""
#include "planner.hpp"
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>
using namespace bbc;
#define CHECK(c, msg) do { if (!(c)) { std::printf("FAIL %s\n", msg); return 1; } } while (0)

static int check(const std::vector<int>& ch, int off) {
  Plan P;
  std::string err;
  if (!build_plan(ch.data(), (int)ch.size(), &P, &err, off)) { std::printf("FAIL plan %s\n", err.c_str()); return 1; }
  const int nt = (int)P.tasks.size();
  for (int groups : {48, 96, 192, 384})
    for (int by_shape = 0; by_shape < 2; by_shape++) {
      std::vector<int> gp, gt;
      make_task_groups(P, groups, &gp, &gt, by_shape != 0);
      CHECK(!gp.empty() && gp.front() == 0 && gp.back() == (int)gt.size() && (int)gt.size() == nt, "task lists");
      for (size_t i = 0; i + 1 < gp.size(); i++) CHECK(gp[i] <= gp[i + 1], "task lists monotone");
      std::vector<int> seen(nt, 0);
      for (int t : gt) seen[t]++;
      for (int t = 0; t < nt; t++) CHECK(seen[t] == 1, "task in one list");
    }
  std::vector<Batch> batches;
  make_batches(P, &batches);
  FusedLayout lay;
  optimise_fused_layout(P, &batches, &lay);
  std::vector<int> seen(nt, 0);
  for (const Batch& b : batches) {
    CHECK(!b.tasks.empty() && b.tasks.size() <= 32, "batch size");
    const PairTask& t0 = P.tasks[b.tasks[0]];
    for (int t : b.tasks) {
      seen[t]++;
      const PairTask& t1 = P.tasks[t];
      CHECK(t1.nA == t0.nA && t1.nB == t0.nB && t1.n1 * t1.n2 == t0.n1 * t0.n2 && b.nA == t0.nA, "batch shape");
    }
  }
  for (int t = 0; t < nt; t++) CHECK(seen[t] == 1, "task in one batch");
  CHECK((int)lay.row_slot.size() == P.n_out, "row map size");
  for (int r = 1; r < P.n_out; r++) CHECK(lay.row_slot[r] > lay.row_slot[r - 1], "row map increasing");
  for (int r = 0; r < P.n_out; r++) CHECK(lay.row_slot[r] < lay.n_slots, "row map inside the slots");
  for (const PairTask& t : P.tasks)
    for (int side = 0; side < 2; side++) {
      const int n = side ? t.nB : t.nA;
      const int* o = side ? t.offB : t.offA;
      const int s1 = side ? t.sB1 : t.sA1, s2 = side ? t.sB2 : t.sA2;
      for (int r = 0; r < n; r++)
        for (int i1 = 0; i1 < t.n1; i1++)
          for (int i2 = 0; i2 < t.n2; i2++)
            CHECK(lay.row_slot[o[r] + i1 * s1 + i2 * s2] == lay.row_slot[o[r]] + i1 * s1 + i2 * s2, "slot strides");
    }
  for (int warps : {8, 12, 16})
    for (int chunk : {0, 18, 36, 72, 144}) {
      std::vector<int> wp;
      std::vector<BatchUnit> units;
      make_units(P, batches, warps, chunk, &wp, &units);
      CHECK((int)wp.size() == warps + 1 && wp.front() == 0 && wp.back() == (int)units.size(), "warp pointers");
      for (int w = 0; w < warps; w++) CHECK(wp[w] <= wp[w + 1], "warp pointers monotone");
      std::vector<std::vector<int>> cover(batches.size());
      for (size_t b = 0; b < batches.size(); b++) {
        const PairTask& t = P.tasks[batches[b].tasks[0]];
        cover[b].assign(t.n1 * t.n2, 0);
      }
      for (const BatchUnit& u : units) {
        CHECK(u.batch >= 0 && u.batch < (int)batches.size() && u.k0 < u.k1 && u.k1 <= (int)cover[u.batch].size(),
              "unit range");
        for (int k = u.k0; k < u.k1; k++) cover[u.batch][k]++;
      }
      for (const auto& c : cover)
        for (int x : c) CHECK(x == 1, "open index covered once");
    }
  // block build: lane l of chunk j of group g holds the terms of row
  // first_row + 32 j + l (in some order) and weight-0 padding otherwise
  CHECK((int)P.chunk_first.size() == (int)P.groups.size() + 1, "chunk table");
  for (size_t g = 0; g < P.groups.size(); g++) {
    const GroupInfo& gi = P.groups[g];
    const int n_chunks = (gi.n_rows + 31) / 32;
    CHECK(P.chunk_first[g + 1] - P.chunk_first[g] == n_chunks, "chunks per group");
    for (int j = 0; j < n_chunks; j++) {
      const auto& ch = P.ell_chunk[P.chunk_first[g] + j];
      CHECK(ch.first >= 0 && (size_t)ch.first + 32 * (size_t)ch.second <= P.ell.size(), "chunk range");
      for (int l = 0; l < 32; l++) {
        const int r = gi.first_row + 32 * j + l;
        std::vector<uint32_t> got, want;
        for (int k = 0; k < ch.second; k++) {
          const uint32_t e = P.ell[ch.first + 32 * k + l];
          if ((e >> 16) != 0) got.push_back(e);
          else CHECK((e & 0xffffu) == 0, "padding reads position 0");
        }
        if (32 * j + l < gi.n_rows) want.assign(P.entries.begin() + P.row_ptr[r], P.entries.begin() + P.row_ptr[r + 1]);
        std::sort(got.begin(), got.end());
        std::sort(want.begin(), want.end());
        CHECK(got == want, "row terms in the chunk");
      }
    }
  }
  std::printf("OK %d tasks %zu batches\n", nt, batches.size());
  return 0;
}

int main(int argc, char** argv) {
  // argv: spin offset, then channel ids
  const int off = std::atoi(argv[1]);
  std::vector<int> ch;
  for (int i = 2; i < argc; i++) ch.push_back(std::atoi(argv[i]));
  return check(ch, off);
}
"""


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    d = tmp_path_factory.mktemp("schedule")
    src = d / "check.cpp"
    exe = d / "check"
    src.write_text(CHECKER)
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", CSRC, "-o", str(exe), str(src),
                           os.path.join(CSRC, "planner.cpp")])
    return str(exe)


LISTS = {
    "52": list(range(52)),
    "64 octet ids": list(range(64)),
    "90 decuplet ids": list(range(64, 154)),
    "octet and decuplet": list(range(52)) + list(range(64, 154)),
    "one channel": [1],
    "omitted only (no task)": [52, 53, 54, 55],
}


@pytest.mark.parametrize("name", list(LISTS))
@pytest.mark.parametrize("off", [0, 2])
def test_schedules(checker, name, off):
    r = subprocess.run([checker, str(off)] + [str(c) for c in LISTS[name]], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout + r.stderr
