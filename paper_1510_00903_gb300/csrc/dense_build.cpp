// dense_build.cpp -- host tables of the FP32 block build with dense entry tuples.
//
// A block row is a sparse integer-weighted sum of sink-tensor entries
// F[a][e0][e1][e2] = sum_c2 D[e0][e1][c2] S_f2[(a, c2), e2] (Sec. 3 blocks,
// Appendix A aggregation; planner.cpp).  The planner stores the entries each
// group of rows reads at compact shared-memory positions, one thread per
// entry.  Here the entries are regrouped by tuple (family slot, a, e0 e1): one
// thread forms all twelve e2 values of a tuple (three diquark values reused
// twelve times, the propagator row shared by a warp whose tuples have the same
// (slot, a)), and writes entry (tuple j, e2) to position e2 * NT + j, so a
// warp's stores are contiguous.  The row terms are re-addressed to these
// positions, their weights stored as bfloat16 bits (small integers are exact)
// so the kernel reads them with one AND, and each 32-row chunk's terms are
// reordered against shared-memory bank conflicts as the planner does.
#include <algorithm>
#include <cstring>
#include <map>
#include <string>

#include "planner.hpp"

namespace bbc {

namespace {

uint32_t bf16_bits(int w) {  // an integer weight as the top 16 bits of an FP32 value (exact for |w| <= 256)
  const float f = (float)w;
  uint32_t u;
  std::memcpy(&u, &f, sizeof u);
  return u & 0xffff0000u;
}

}  // namespace

bool make_dense_build(const Plan& P, DenseBuild* out, std::string* err) {
  DenseBuild D;
  // the (slot, local index) behind every position, group by group, as the
  // planner laid them out (positions of a slot whose family is unchanged
  // carry over from the previous group)
  std::vector<int> pos_slot(8192, -1), pos_local(8192, -1);
  int prev_fam[2] = {-1, -1};
  D.chunk_first.assign(1, 0);
  for (size_t g = 0; g < P.groups.size(); g++) {
    const GroupInfo& gi = P.groups[g];
    for (int sl = 0; sl < 2; sl++)
      if (gi.fam[sl] != prev_fam[sl])
        for (int k = 0; k < 8192; k++)
          if (pos_slot[k] == sl) pos_slot[k] = -1;
    for (int z = P.zneed_first[g]; z < P.zneed_first[g + 1]; z++) {
      const uint32_t zn = P.zneed[z];
      const int pos = (int)(zn & 0x1fff);
      pos_slot[pos] = (int)((zn >> 13) & 1);
      pos_local[pos] = (int)(zn >> 14);
    }
    prev_fam[0] = gi.fam[0];
    prev_fam[1] = gi.fam[1];
    // the tuples (slot, a, e01) this group's rows read, sorted (a warp's
    // tuples then share (slot, a) except at run boundaries)
    std::map<int, int> tuple_of;  // slot * 288 + a * 144 + e01 -> index
    for (int r = gi.first_row; r < gi.first_row + gi.n_rows; r++)
      for (int k = P.row_ptr[r]; k < P.row_ptr[r + 1]; k++) {
        const int pos = (int)(P.entries[k] & 0xffffu);
        if (pos >= 8192 || pos_slot[pos] < 0) {
          *err = "internal: dense build position";
          return false;
        }
        const int local = pos_local[pos], a = local / 1728, e01 = (local % 1728) / 12;
        tuple_of[pos_slot[pos] * 288 + a * 144 + e01] = 0;
      }
    const int nt = (int)tuple_of.size();
    int idx = 0;
    for (auto& kv : tuple_of) {
      kv.second = idx++;
      D.tuples.push_back((uint32_t)kv.first);  // slot * 288 + a * 144 + e01
    }
    D.tuple_first.push_back((int)D.tuples.size() - nt);
    // an odd stride: entries e2 and e2 + 1 of one tuple fall in different banks
    const int ntp = nt | 1;
    D.stride.push_back(ntp);
    D.z_slots = std::max(D.z_slots, 12 * ntp);
    // the group's rows as lane-interleaved 32-row chunks with the new positions
    for (int c0 = 0; c0 < gi.n_rows; c0 += 32) {
      const int r0 = gi.first_row + c0, nr = std::min(32, gi.n_rows - c0);
      std::vector<std::vector<uint32_t>> left(nr);
      int len = 0;
      for (int l = 0; l < nr; l++) {
        for (int k = P.row_ptr[r0 + l]; k < P.row_ptr[r0 + l + 1]; k++) {
          const int pos = (int)(P.entries[k] & 0xffffu), local = pos_local[pos];
          const int key = pos_slot[pos] * 288 + (local / 1728) * 144 + (local % 1728) / 12, e2 = local % 12;
          const int np = e2 * ntp + tuple_of[key];
          const int w = (int)(int16_t)(P.entries[k] >> 16);
          if (w == 0) continue;
          if (w < -256 || w > 256 || np >= 65536) {
            *err = "internal: dense build weight or position";
            return false;
          }
          left[l].push_back((uint32_t)np | bf16_bits(w));
        }
        len = std::max(len, (int)left[l].size());
      }
      const int base = (int)D.ell.size();
      D.ell.resize(D.ell.size() + (size_t)32 * len, 0u);  // padding: weight 0 at position 0
      // per step and half-warp, a term in a bank pair (position mod 16) no
      // other lane of the half-warp uses at that step, where one exists
      for (int k = 0; k < len; k++)
        for (int h = 0; h < 32; h += 16) {
          bool used[16] = {false};
          for (int l = h; l < std::min(nr, h + 16); l++) {
            std::vector<uint32_t>& v = left[l];
            if (v.empty()) continue;
            size_t pick = 0;
            for (size_t j = 0; j < v.size(); j++)
              if (!used[(v[j] & 0xffffu) % 16]) { pick = j; break; }
            used[(v[pick] & 0xffffu) % 16] = true;
            D.ell[base + 32 * k + l] = v[pick];
            v.erase(v.begin() + (long)pick);
          }
        }
      D.ell_chunk.push_back({base, len});
    }
    D.chunk_first.push_back((int)D.ell_chunk.size());
  }
  if (D.z_slots >= 65536 || D.tuples.size() > 65535) {
    *err = "internal: dense build too large";
    return false;
  }
  D.tuple_first.push_back((int)D.tuples.size());
  *out = std::move(D);
  return true;
}

}  // namespace bbc
