// projection.cu -- the projections of Sec. 2 on the correlators C_ch(r):
// source spin states |J M> (the coefficients P^(J,M)_{a'b'} of the source
// operator) and the cubic-group average P = (1/24) sum over the rotations of
// O acting on r (the 3S1 / 3D1 split; the D-wave part is 1 - P).
//
// The average over the 24 rotations of a site is the mean over the site's
// orbit under O (each orbit member is hit 24 / |orbit| times), and it is the
// same for every member.  So the kernel walks orbits: a 4-lane group (one
// lane per sink spin pair ab, holding the four source-spin components of a
// site) reads every member of one orbit once, writes its spin-state
// projection R (two of the four states are copies, the other two
// (v2 -+ v1)/sqrt2), sums the records in FP64, and writes the projected mean
// to every member of Ra1: every site is read once and written once per
// output (the HBM minimum) with four FP64 instructions per value read.
// Both projections are linear and act on different indices, so they commute.
#include <algorithm>
#include <cstring>

#include "device_common.cuh"

namespace bbc {

// Orbits of the 24 proper cube rotations (signed axis permutations with
// determinant +1) on the periodic L^3 lattice: orbit k is
// orb_site[orb_ptr[k] .. orb_ptr[k+1]), every site exactly once; orbits come
// in order of size, so that the orbits a warp walks have equal lengths.
void cubic_orbits(int L, std::vector<int>& orb_ptr, std::vector<int>& orb_site) {
  const int perms[6][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}, {0, 2, 1}, {2, 1, 0}, {1, 0, 2}};
  const int V = L * L * L;
  std::vector<char> seen(V, 0);
  std::vector<std::vector<int>> orbits;
  int img[24];
  for (int r = 0; r < V; r++) {
    if (seen[r]) continue;
    const int c[3] = {r % L, (r / L) % L, r / (L * L)};
    int n = 0;
    for (int p = 0; p < 6; p++) {
      const int parity = p < 3 ? 1 : -1;  // cyclic permutations are even
      for (int s = 0; s < 8; s++) {
        const int neg = (s & 1) + ((s >> 1) & 1) + ((s >> 2) & 1);
        if (parity * ((neg & 1) ? -1 : 1) != 1) continue;
        int g[3];
        for (int i = 0; i < 3; i++) {
          const int v = c[perms[p][i]];
          g[i] = ((s >> i) & 1) ? (L - v) % L : v;
        }
        img[n++] = g[0] + L * (g[1] + L * g[2]);
      }
    }
    std::sort(img, img + n);
    const int m = (int)(std::unique(img, img + n) - img);
    for (int i = 0; i < m; i++) seen[img[i]] = 1;
    orbits.emplace_back(img, img + m);
  }
  std::stable_sort(orbits.begin(), orbits.end(),
                   [](const std::vector<int>& a, const std::vector<int>& b) { return a.size() < b.size(); });
  orb_ptr.assign(1, 0);
  orb_site.clear();
  orb_site.reserve(V);
  for (const auto& o : orbits) {
    orb_site.insert(orb_site.end(), o.begin(), o.end());
    orb_ptr.push_back((int)orb_site.size());
  }
}

namespace {

// The four source spin states of one sink spin pair (index 0 = spin up,
// p = a' + 2b'): |0 0> = (|ud> - |du>)/sqrt2 = h (v2 - v1), |1 1> = v0,
// |1 0> = h (v2 + v1), |1 -1> = v3; written at o[4 jm].
__device__ __forceinline__ void write_states(double2* __restrict__ o, const double2 (&v)[4]) {
  const double h = 0.70710678118654752440;  // 1/sqrt(2)
  o[0] = make_double2(h * (v[2].x - v[1].x), h * (v[2].y - v[1].y));
  o[4] = v[0];
  o[8] = make_double2(h * (v[2].x + v[1].x), h * (v[2].y + v[1].y));
  o[12] = v[3];
}

// C, R, Ra1: [n_fields][V][16] complex128 (component ab + 4p); one 4-lane
// group per (orbit, field), lane ab.
__global__ void __launch_bounds__(256) k_project(const double2* __restrict__ C, int V, const int* __restrict__ orb_ptr,
                                                 const int* __restrict__ orb_site, int n_orb, double2* __restrict__ R,
                                                 double2* __restrict__ Ra1) {
  const int ab = threadIdx.x & 3;
  const int k = blockIdx.x * 64 + (threadIdx.x >> 2);
  if (k >= n_orb) return;  // no warp-wide operation follows
  const size_t fbase = (size_t)blockIdx.y * V * 16 + ab;
  const int m0 = __ldg(orb_ptr + k), m1 = __ldg(orb_ptr + k + 1);
  double2 acc[4];
#pragma unroll
  for (int p = 0; p < 4; p++) acc[p] = make_double2(0.0, 0.0);
  for (int m = m0; m < m1; m++) {
    const size_t base = fbase + (size_t)__ldg(orb_site + m) * 16;
    double2 v[4];
#pragma unroll
    for (int p = 0; p < 4; p++) v[p] = __ldg(C + base + 4 * p);
#pragma unroll
    for (int p = 0; p < 4; p++) { acc[p].x += v[p].x; acc[p].y += v[p].y; }
    if (R) write_states(R + base, v);
  }
  if (!Ra1) return;
  const double inv = 1.0 / (m1 - m0);
#pragma unroll
  for (int p = 0; p < 4; p++) acc[p] = make_double2(acc[p].x * inv, acc[p].y * inv);
  for (int m = m0; m < m1; m++) write_states(Ra1 + fbase + (size_t)__ldg(orb_site + m) * 16, acc);
}

}  // namespace

cudaError_t launch_project(const void* C, int L, const int* orb_ptr, const int* orb_site, int n_orb, int n_fields,
                           void* R, void* Ra1, cudaStream_t st) {
  if (n_fields <= 0 || n_orb <= 0) return cudaSuccess;
  const int V = L * L * L;
  dim3 grid((n_orb + 63) / 64, n_fields);
  k_project<<<grid, 256, 0, st>>>((const double2*)C, V, orb_ptr, orb_site, n_orb, (double2*)R, (double2*)Ra1);
  return cudaGetLastError();
}

}  // namespace bbc
