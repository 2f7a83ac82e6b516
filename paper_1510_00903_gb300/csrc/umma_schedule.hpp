// umma_schedule.hpp -- the step schedule of the persistent tcgen05 contraction
// (tc_umma.cu), as host + device functions so that a host program can check
// it (tests/test_umma_schedule.py).
//
// A CTA owns pairs i = 0 .. n_mine - 1; pair i is units u = 3 i + c (c = 0,
// 1, 2: 48 open indices each).  Step u of the CTA's loop (u = 0 .. n_mine * 3
// + 1):
//   1. the epilogue of pair e if u = 3 e + 4: wait for completion e / 2 of
//      the accumulator barrier acc(e), read accumulator acc(e);
//   2. if u < n_units: wait (u >= 2) for completion (u - 2) / 2 of the stage
//      barrier stage(u), then store unit u into stage(u);
//   3. one CTA barrier;
//   4. if u < n_units: the MMAs of unit u read stage(u) and write accumulator
//      acc(u / 3), then commit to the stage barrier stage(u) and, for c = 2,
//      to the accumulator barrier acc(u / 3).
// Every barrier completes once per commit (arrival count 1), and a wait on
// completion k polls for the phase parity k mod 2: it must start after the
// commit of completion k is issued and before the commit of completion k + 2
// (else the parity would name a later phase).
#pragma once

#ifdef __CUDACC__
#define UMS_HD __host__ __device__
#else
#define UMS_HD
#endif

namespace bbc {
namespace umsched {

constexpr int kUnitsPerPair = 3;

UMS_HD constexpr int n_units(int n_mine) { return n_mine * kUnitsPerPair; }
UMS_HD constexpr int last_step(int n_mine) { return n_units(n_mine) + 1; }
UMS_HD constexpr int pair_of(int u) { return u / kUnitsPerPair; }
UMS_HD constexpr int chunk_of(int u) { return u - kUnitsPerPair * pair_of(u); }

// the two shared-memory stages, alternating by unit
UMS_HD constexpr int stage(int u) { return u & 1; }
UMS_HD constexpr bool stage_waits(int u) { return u >= 2; }
UMS_HD constexpr int stage_completion(int u) { return (u - 2) >> 1; }  // the MMAs of unit u - 2
UMS_HD constexpr unsigned stage_parity(int u) { return (unsigned)(stage_completion(u) & 1); }

// the two tensor-memory accumulators, alternating by pair
UMS_HD constexpr int acc(int pair) { return pair & 1; }
UMS_HD constexpr int acc_completion(int pair) { return pair >> 1; }
UMS_HD constexpr unsigned acc_parity(int pair) { return (unsigned)(acc_completion(pair) & 1); }

// the epilogue of pair e runs in step 3 e + 4, two steps after its last MMAs
UMS_HD constexpr int epilogue_step(int e) { return kUnitsPerPair * e + kUnitsPerPair + 1; }
UMS_HD constexpr bool is_epilogue_step(int u) {
  return u >= kUnitsPerPair + 1 && (u - kUnitsPerPair - 1) % kUnitsPerPair == 0;
}
UMS_HD constexpr int epilogue_pair(int u) { return (u - kUnitsPerPair - 1) / kUnitsPerPair; }

}  // namespace umsched
}  // namespace bbc
