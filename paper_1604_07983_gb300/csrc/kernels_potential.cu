// kernels_potential.cu -- the stencil that turns NBS correlators into a local
// potential (the downstream step that Sec. 1 of arXiv:1604.07983 motivates:
// the potential follows from the NBS wave function).
//
// For correlator components R(r, t) on an L^3 periodic lattice (any
// normalisation the caller has applied, e.g. division by the single-baryon
// correlators) it forms, with central differences,
//   K(r) = a (R(t+1) - 2 R(t) + R(t-1)) + b (R(t+1) - R(t-1)) / 2
//        + c sum_i (R(r + e_i) + R(r - e_i) - 2 R(r))      (all at t unless marked)
// and optionally the local ratio P(r) = K(r) / R(r, t).  One thread per
// (component, site); the six neighbours are read from the same component's
// cube (L1/L2 reuse), so the kernel moves 3 reads and 1-2 writes of 16 bytes
// per point: HBM-bound.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"

namespace nbs {

namespace {

__global__ void __launch_bounds__(256) k_potential(const double2* __restrict__ Rm, const double2* __restrict__ R0,
                                                   const double2* __restrict__ Rp, int L, long long n, double a,
                                                   double b, double c, double2* __restrict__ K,
                                                   double2* __restrict__ P) {
  const long long V = (long long)L * L * L;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long base = i - i % V;
    const int s = (int)(i % V);
    const int x = s % L, y = (s / L) % L, z = s / (L * L);
    const int xp = x + 1 == L ? 0 : x + 1, xm = x == 0 ? L - 1 : x - 1;
    const int yp = y + 1 == L ? 0 : y + 1, ym = y == 0 ? L - 1 : y - 1;
    const int zp = z + 1 == L ? 0 : z + 1, zm = z == 0 ? L - 1 : z - 1;
    const double2 r = R0[i], rm = Rm[i], rp = Rp[i];
    const int yz = L * (y + L * z);
    const double2 n1 = R0[base + xp + yz], n2 = R0[base + xm + yz];
    const double2 n3 = R0[base + x + L * (yp + L * z)], n4 = R0[base + x + L * (ym + L * z)];
    const double2 n5 = R0[base + x + L * (y + L * zp)], n6 = R0[base + x + L * (y + L * zm)];
    const double lx = n1.x + n2.x + n3.x + n4.x + n5.x + n6.x - 6.0 * r.x;
    const double ly = n1.y + n2.y + n3.y + n4.y + n5.y + n6.y - 6.0 * r.y;
    const double kx = a * (rp.x - 2.0 * r.x + rm.x) + b * 0.5 * (rp.x - rm.x) + c * lx;
    const double ky = a * (rp.y - 2.0 * r.y + rm.y) + b * 0.5 * (rp.y - rm.y) + c * ly;
    K[i] = make_double2(kx, ky);
    if (P) {
      const double inv = 1.0 / (r.x * r.x + r.y * r.y);  // K / R (IEEE: infinite or NaN where R = 0)
      P[i] = make_double2((kx * r.x + ky * r.y) * inv, (ky * r.x - kx * r.y) * inv);
    }
  }
}

}  // namespace

cudaError_t launch_potential(const double2* Rm, const double2* R0, const double2* Rp, int L, long long ncomp, double a,
                             double b, double c, double2* K, double2* P, cudaStream_t st) {
  const long long n = ncomp * L * L * L;
  if (n <= 0) return cudaSuccess;
  const long long blocks = std::min<long long>((n + 255) / 256, 152LL * 16);
  k_potential<<<(unsigned)blocks, 256, 0, st>>>(Rm, R0, Rp, L, n, a, b, c, K, P);
  return cudaGetLastError();
}

}  // namespace nbs
