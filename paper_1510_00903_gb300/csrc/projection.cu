// projection.cu -- the projections of Sec. 2 on the correlators C_ch(r):
// source spin states |J M> (the coefficients P^(J,M)_{a'b'} of the source
// operator) and the cubic-group average P = (1/24) sum over the rotations of
// O acting on r (the 3S1 / 3D1 split; the D-wave part is 1 - P).
//
// The average over the 24 rotations of a site is the mean over the site's
// orbit under O (each orbit member is hit 24 / |orbit| times), and it is the
// same for every member.  So the kernel walks orbits: a 16-lane group (one
// lane per spin component, one 256-byte record per site) reads every member
// of one orbit once, writes its spin-state projection R, sums the records in
// FP64, and writes the projected mean to every member of Ra1.  Every site is
// read once and written once per output: the HBM minimum.  Both projections
// are linear and act on different indices, so they commute.
#include <algorithm>
#include <cstring>

#include "device_common.cuh"

namespace bbc {

// Orbits of the 24 proper cube rotations (signed axis permutations with
// determinant +1) on the periodic L^3 lattice: orbit k is
// orb_site[orb_ptr[k] .. orb_ptr[k+1]), every site exactly once.
void cubic_orbits(int L, std::vector<int>& orb_ptr, std::vector<int>& orb_site) {
  const int perms[6][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}, {0, 2, 1}, {2, 1, 0}, {1, 0, 2}};
  const int V = L * L * L;
  std::vector<char> seen(V, 0);
  orb_ptr.assign(1, 0);
  orb_site.clear();
  orb_site.reserve(V);
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
    for (int i = 0; i < m; i++) {
      seen[img[i]] = 1;
      orb_site.push_back(img[i]);
    }
    orb_ptr.push_back((int)orb_site.size());
  }
}

namespace {

__device__ __forceinline__ cpx<double> shfl(cpx<double> v, int src) {
  return cpx<double>(__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src));
}

// Lane s of a 16-lane group holds component a + 2b + 4p (p = a' + 2b') of one
// site; returns state jm = s >> 2 at sink spins ab = s & 3 as c_x v_x + c_y v_y
// with the lane's two source-spin components and coefficients:
//   jm = 0: (|ud> - |du>)/sqrt2 = h v_{p=2} - h v_{p=1}   jm = 1: |uu> = v_{p=0}
//   jm = 2: (|ud> + |du>)/sqrt2 = h v_{p=2} + h v_{p=1}   jm = 3: |dd> = v_{p=3}
// (one instruction stream for every lane: no divergent FP64 paths).
__device__ __forceinline__ cpx<double> spin_states(cpx<double> v, int grp, int s) {
  const int ab = s & 3, jm = s >> 2;
  const double h = 0.70710678118654752440;  // 1/sqrt(2)
  const int px = jm == 1 ? 0 : (jm == 3 ? 3 : 2), py = jm == 1 ? 0 : (jm == 3 ? 3 : 1);
  const double cx = (jm & 1) ? 1.0 : h, cy = (jm & 1) ? 0.0 : (jm == 0 ? -h : h);
  const cpx<double> vx = shfl(v, grp + ab + 4 * px), vy = shfl(v, grp + ab + 4 * py);
  return cpx<double>(fma(cy, vy.re, cx * vx.re), fma(cy, vy.im, cx * vx.im));
}

// C, R, Ra1: [n_fields][V][16] complex128; one 16-lane group per (orbit, field).
__global__ void __launch_bounds__(256) k_project(const double2* __restrict__ C, int V, const int* __restrict__ orb_ptr,
                                                 const int* __restrict__ orb_site, int n_orb, double2* __restrict__ R,
                                                 double2* __restrict__ Ra1) {
  const int s = threadIdx.x & 15, grp = threadIdx.x & 16;
  const int k = blockIdx.x * 16 + (threadIdx.x >> 4);
  const size_t fbase = (size_t)blockIdx.y * V * 16;
  const bool valid = k < n_orb;
  const int m0 = valid ? orb_ptr[k] : 0, m1 = valid ? orb_ptr[k + 1] : 0;
  const int n = m1 - m0;
  const int n_other = __shfl_xor_sync(0xffffffffu, n, 16);
  const int n_max = n > n_other ? n : n_other;  // both groups of the warp loop together (shuffles)
  // member sites: lane s of the group holds members s and s + 16 (orbits have
  // at most 24), broadcast by shuffles so the record loads do not wait on them
  const int site_a = s < n ? __ldg(&orb_site[m0 + s]) : 0;
  const int site_b = s + 16 < n ? __ldg(&orb_site[m0 + 16 + s]) : 0;
  cpx<double> acc(0.0, 0.0);
  for (int i0 = 0; i0 < n_max; i0 += 8) {
    cpx<double> v[8];
    int site[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {  // eight independent record loads in flight
      const int i = i0 + j;
      site[j] = __shfl_sync(0xffffffffu, i < 16 ? site_a : site_b, grp + (i & 15));
      v[j] = cpx<double>(0.0, 0.0);
      if (i < n) {
        const double2 d = __ldg(&C[fbase + (size_t)site[j] * 16 + s]);
        v[j] = cpx<double>(d.x, d.y);
      }
    }
#pragma unroll
    for (int j = 0; j < 8; j++) {
      acc.re += v[j].re;
      acc.im += v[j].im;
      if (R) {
        const cpx<double> o = spin_states(v[j], grp, s);
        if (i0 + j < n) R[fbase + (size_t)site[j] * 16 + s] = make_double2(o.re, o.im);
      }
    }
  }
  if (!Ra1) return;  // uniform over the grid
  const double inv = n > 0 ? 1.0 / n : 0.0;
  const cpx<double> o = spin_states(cpx<double>(acc.re * inv, acc.im * inv), grp, s);
  for (int i = 0; i < n_max; i++) {
    const int site = __shfl_sync(0xffffffffu, i < 16 ? site_a : site_b, grp + (i & 15));
    if (i < n) Ra1[fbase + (size_t)site * 16 + s] = make_double2(o.re, o.im);
  }
}

}  // namespace

cudaError_t launch_project(const void* C, int L, const int* orb_ptr, const int* orb_site, int n_orb, int n_fields,
                           void* R, void* Ra1, cudaStream_t st) {
  if (n_fields <= 0 || n_orb <= 0) return cudaSuccess;
  const int V = L * L * L;
  dim3 grid((n_orb + 15) / 16, n_fields);
  k_project<<<grid, 256, 0, st>>>((const double2*)C, V, orb_ptr, orb_site, n_orb, (double2*)R, (double2*)Ra1);
  return cudaGetLastError();
}

}  // namespace bbc
