// projection.cu -- the projections of Sec. 2 on the correlators C_ch(r):
// source spin states |J M> (the coefficients P^(J,M)_{a'b'} of the source
// operator) and the cubic-group average P = (1/24) sum over the rotations of
// O acting on r (the 3S1 / 3D1 split; the D-wave part is 1 - P).
//
// One thread per (field, site, spin component); the 16 spin components of a
// site are 16 adjacent lanes (one 256-byte segment per site, coalesced for
// every rotated site).  Both projections are linear and act on different
// indices (source spins, relative coordinate), so they commute: each thread
// sums the 24 rotated copies of its own component in FP64, then 16-lane
// shuffles combine the four source-spin components of each state.
#include "device_common.cuh"

namespace bbc {
namespace {

// The 24 proper rotations of the cube as signed axis permutations:
// component i of the rotated vector is sign_i * r[perm_i].  Entry bits:
// perm0 | perm1 << 2 | perm2 << 4 | (sign0 < 0) << 6 | (sign1 < 0) << 7 | (sign2 < 0) << 8.
__constant__ int c_rot[24];

int host_rotations(int* out) {
  const int perms[6][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}, {0, 2, 1}, {2, 1, 0}, {1, 0, 2}};
  int n = 0;
  for (int p = 0; p < 6; p++) {
    const int parity = p < 3 ? 1 : -1;  // the first three are cyclic (even)
    for (int s = 0; s < 8; s++) {
      const int neg = (s & 1) + ((s >> 1) & 1) + ((s >> 2) & 1);
      const int det = parity * ((neg & 1) ? -1 : 1);
      if (det != 1) continue;
      out[n++] = perms[p][0] | (perms[p][1] << 2) | (perms[p][2] << 4) | ((s & 7) << 6);
    }
  }
  return n;
}

__device__ __forceinline__ int rot_coord(int code, int i, int x, int y, int z, int L) {
  const int pi = (code >> (2 * i)) & 3;
  const int v = pi == 0 ? x : (pi == 1 ? y : z);
  return ((code >> (6 + i)) & 1) ? (v == 0 ? 0 : L - v) : v;
}

__device__ __forceinline__ cpx<double> shfl(cpx<double> v, int src) {
  return cpx<double>(__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src));
}

// C, R, Ra1: [n_fields][V][16] complex128.  R or Ra1 may be null.
__global__ void __launch_bounds__(256) k_project(const cpx<double>* __restrict__ C, int L, int V,
                                                 cpx<double>* __restrict__ R, cpx<double>* __restrict__ Ra1) {
  const int s = threadIdx.x & 15;
  const int site = blockIdx.x * 16 + (threadIdx.x >> 4);
  const size_t fbase = (size_t)blockIdx.y * V * 16;
  const bool valid = site < V;
  cpx<double> c(0.0, 0.0), a(0.0, 0.0);
  if (valid) {
    c = C[fbase + (size_t)site * 16 + s];
    if (Ra1) {
      const int x = site % L, y = (site / L) % L, z = site / (L * L);
#pragma unroll 4
      for (int g = 0; g < 24; g++) {
        const int code = c_rot[g];
        const int gx = rot_coord(code, 0, x, y, z, L), gy = rot_coord(code, 1, x, y, z, L),
                  gz = rot_coord(code, 2, x, y, z, L);
        const double2 v =
            __ldg(reinterpret_cast<const double2*>(C) + fbase + ((size_t)gx + (size_t)L * (gy + (size_t)L * gz)) * 16 + s);
        a.re += v.x;
        a.im += v.y;
      }
      a.re *= 1.0 / 24.0;
      a.im *= 1.0 / 24.0;
    }
  }
  // lane s holds component a + 2b + 4 p (p = a' + 2 b'); the output of lane
  // s is the state jm = s >> 2 at sink spins ab = s & 3.
  const int lane = threadIdx.x & 31, grp = lane & 16, ab = s & 3, jm = s >> 2;
  const double h = 0.70710678118654752440;  // 1/sqrt(2)
  for (int which = 0; which < 2; which++) {
    cpx<double>* out = which == 0 ? R : Ra1;
    if (!out) continue;
    const cpx<double> v = which == 0 ? c : a;
    const cpx<double> v0 = shfl(v, grp + ab), v1 = shfl(v, grp + ab + 4), v2 = shfl(v, grp + ab + 8),
                      v3 = shfl(v, grp + ab + 12);
    cpx<double> o;
    if (jm == 0) o = cpx<double>(h * (v2.re - v1.re), h * (v2.im - v1.im));        // (|ud> - |du>)/sqrt2
    else if (jm == 1) o = v0;                                                       // |uu>
    else if (jm == 2) o = cpx<double>(h * (v2.re + v1.re), h * (v2.im + v1.im));   // (|ud> + |du>)/sqrt2
    else o = v3;                                                                    // |dd>
    if (valid) out[fbase + (size_t)site * 16 + s] = o;
  }
}

int g_rot_uploaded[64] = {0};

}  // namespace

cudaError_t launch_project(const void* C, int L, int n_fields, void* R, void* Ra1, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!g_rot_uploaded[dev]) {
    int rot[48];
    if (host_rotations(rot) != 24) return cudaErrorInvalidValue;
    e = cudaMemcpyToSymbol(c_rot, rot, sizeof(int) * 24);
    if (e != cudaSuccess) return e;
    g_rot_uploaded[dev] = 1;
  }
  if (n_fields <= 0) return cudaSuccess;
  const int V = L * L * L;
  dim3 grid((V + 15) / 16, n_fields);
  k_project<<<grid, 256, 0, st>>>((const cpx<double>*)C, L, V, (cpx<double>*)R, (cpx<double>*)Ra1);
  return cudaGetLastError();
}

}  // namespace bbc
