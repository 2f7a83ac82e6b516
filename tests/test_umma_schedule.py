"""Host check of the step schedule of the persistent tcgen05 contraction (CPU).

The schedule functions the kernel uses (csrc/umma_schedule.hpp) are compiled
with g++ into a checker that replays a CTA's steps for 1 to 200 pairs and
counts, per mbarrier, the commits issued so far:

* every wait on completion k of a barrier starts after that completion's
  commit was issued and before the commit of completion k + 1 (so the polled
  phase parity names exactly that completion: a wait cannot miss it nor
  alias a later phase), hence every wait ends once the MMAs it names finish;
* a stage is stored into only after the MMAs of the previous unit that read
  it have completed, and the MMAs of a unit read the stage in the step it
  was stored (after the CTA barrier);
* an accumulator is overwritten (the first MMA of a pair) only in a later
  step than the epilogue that read the previous pair in it, and every
  epilogue runs after its pair's last MMA and inside the loop;
* the step <-> (pair, chunk, epilogue pair) maps are consistent.

A planted mistake (the stage wait naming the unit's own commit, as u / 2 would)
must fail.
"""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1510_00903_gb300", "csrc")

CHECKER = r"""
#include "umma_schedule.hpp"
#include <cstdio>
#include <cstdlib>
#include <vector>
using namespace bbc::umsched;

static int fails = 0;
#define CHECK(c, ...) do { if (!(c)) { if (fails++ < 10) { std::printf(__VA_ARGS__); std::printf("\n"); } } } while (0)

int main(int argc, char** argv) {
  const int plant = std::atoi(argv[1]);
  for (int n_mine = 1; n_mine <= 200; n_mine++) {
    const int nu = n_units(n_mine), last = last_step(n_mine);
    int stage_commits[2] = {0, 0}, acc_commits[2] = {0, 0};
    std::vector<int> stored_step(nu, -1), stage_reader_done(2, -1);  // last unit whose MMAs read each stage
    std::vector<int> epi_step(n_mine, -1), first_mma_step(n_mine, -1), last_mma_step(n_mine, -1);
    for (int u = 0; u <= last; u++) {
      // 1. epilogue
      if (is_epilogue_step(u)) {
        const int e = epilogue_pair(u);
        CHECK(e >= 0 && e < n_mine && epilogue_step(e) == u, "n %d step %d: epilogue pair %d", n_mine, u, e);
        if (e >= 0 && e < n_mine) {
          const int k = acc_completion(e), a = acc(e);
          CHECK(acc_commits[a] == k + 1, "n %d step %d: epilogue of pair %d waits for completion %d of acc %d with %d commits",
                n_mine, u, e, k, a, acc_commits[a]);
          CHECK(acc_parity(e) == (unsigned)(k & 1), "acc parity");
          CHECK(last_mma_step[e] >= 0 && last_mma_step[e] < u, "n %d: epilogue of pair %d before its last MMA", n_mine, e);
          epi_step[e] = u;
        }
      }
      // 2. the stage wait and the stores of unit u
      if (u < nu) {
        const int s = stage(u);
        CHECK(s == (u & 1), "stage");
        if (stage_waits(u)) {
          const int k = plant ? (u >> 1) : stage_completion(u);
          CHECK(stage_commits[s] == k + 1, "n %d step %d: stage wait for completion %d of stage %d with %d commits",
                n_mine, u, k, s, stage_commits[s]);
          CHECK(plant || stage_parity(u) == (unsigned)(k & 1), "stage parity");
          // every earlier reader of the stage committed completion <= k: done when k is
          CHECK(stage_reader_done[s] == u - 2, "n %d step %d: stage %d last read by unit %d", n_mine, u, s,
                stage_reader_done[s]);
        } else {
          CHECK(stage_commits[s] == 0, "n %d step %d: unwaited stage %d already read", n_mine, u, s);
        }
        stored_step[u] = u;
      }
      // 3. CTA barrier; 4. the MMAs of unit u, then their commits
      if (u < nu) {
        const int i = pair_of(u), c = chunk_of(u);
        CHECK(i * kUnitsPerPair + c == u && c >= 0 && c < kUnitsPerPair, "pair/chunk of %d", u);
        CHECK(stored_step[u] == u, "unit %d read before it was stored", u);
        if (c == 0) {
          first_mma_step[i] = u;
          if (i >= 2) CHECK(epi_step[i - 2] >= 0 && epi_step[i - 2] < u,
                            "n %d: pair %d overwrites acc %d before the epilogue of pair %d", n_mine, i, acc(i), i - 2);
        }
        stage_reader_done[stage(u)] = u;
        stage_commits[stage(u)]++;
        if (c == kUnitsPerPair - 1) {
          acc_commits[acc(i)]++;
          last_mma_step[i] = u;
        }
      }
    }
    for (int e = 0; e < n_mine; e++) CHECK(epi_step[e] >= 0, "n %d: pair %d has no epilogue", n_mine, e);
  }
  if (fails) { std::printf("FAIL %d\n", fails); return 1; }
  std::printf("OK\n");
  return 0;
}
"""


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    d = tmp_path_factory.mktemp("umsched")
    src = d / "check.cpp"
    exe = d / "check"
    src.write_text(CHECKER)
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", CSRC, "-o", str(exe), str(src)])
    return str(exe)


def test_schedule_waits_end_and_buffers_are_not_raced(checker):
    r = subprocess.run([checker, "0"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout + r.stderr


def test_planted_wrong_stage_completion_is_caught(checker):
    r = subprocess.run([checker, "1"], capture_output=True, text=True, timeout=120)
    assert r.returncode != 0 and "stage wait" in r.stdout, r.stdout
