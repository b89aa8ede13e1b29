// slab.cu -- data movement of the L-parallel path (the paper's second
// parallelisation, Sec. 4 (i) and Sec. 5: the lattice split over ranks, an
// all-to-all per 3-D FFT).
//
// Rank r holds the z-planes [z0[r], z0[r+1]) of the propagators, builds the
// blocks of its sites and transforms them along x and y.  The forward
// exchange sends to rank d the lines whose y belongs to d's y-set; after it
// rank r holds, for every z, the y values of its own set and transforms along
// z.  The y-sets are closed under y -> -y (mod L), so with x and z complete a
// rank holds both q and -q of every momentum it owns, and the contraction of
// Eq. (4.3) needs no further exchange.  The inverse transform runs the other
// way: z on the y-set, the inverse exchange back to z-planes, then y and x.
//
// This file holds the host layout (the z ranges and the mirror-closed y-sets)
// and the four pack/unpack kernels around the two exchanges; the exchanges
// themselves are the caller's (NCCL, or device copies between ranks that
// share a GPU).
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace nbs {

// Layout of nranks ranks on an L^3 lattice: z-planes in contiguous ranges of
// floor(p L / nranks); y-sets built from the units {0}, {L/2} (L even) and
// {y, L - y}, largest first, each to the rank with the fewest y so far (ties:
// the lowest rank), sorted ascending.  false if some rank would get no y or
// no z-plane.
bool slab_layout(int L, int nranks, SlabGeom& g) {
  if (L < 1 || L > 64 || nranks < 1 || nranks > NBS_SLAB_MAX_RANKS) return false;
  g = SlabGeom();
  g.L = L;
  g.P = nranks;
  for (int p = 0; p <= nranks; ++p) g.z0[p] = p * L / nranks;
  std::vector<std::vector<int>> units;
  for (int y = 1; 2 * y < L; ++y) units.push_back({y, L - y});
  units.push_back({0});
  if (L % 2 == 0 && L > 1) units.push_back({L / 2});
  std::vector<std::vector<int>> sets(nranks);
  for (auto& u : units) {
    int best = 0;
    for (int p = 1; p < nranks; ++p)
      if (sets[p].size() < sets[best].size()) best = p;
    sets[best].insert(sets[best].end(), u.begin(), u.end());
  }
  for (int p = 0; p < nranks; ++p) {
    if (sets[p].empty() || g.z0[p + 1] == g.z0[p]) return false;
    std::sort(sets[p].begin(), sets[p].end());
    g.ny[p] = (int)sets[p].size();
    for (int i = 0; i < g.ny[p]; ++i) {
      g.yowner[sets[p][i]] = p;
      g.yloc[sets[p][i]] = i;
    }
  }
  for (int p = 0; p < nranks; ++p)
    for (int z = g.z0[p]; z < g.z0[p + 1]; ++z) g.zowner[z] = p;
  return true;
}

// the y values of rank p's set in local order
std::vector<int> slab_yset(const SlabGeom& g, int p) {
  std::vector<int> ys(g.ny[p]);
  for (int y = 0; y < g.L; ++y)
    if (g.yowner[y] == p) ys[g.yloc[y]] = y;
  return ys;
}

namespace {

// 32 bytes: the four sink spins of one stored-block cell at one site, FP32 complex
struct alignas(16) Cell4 {
  float4 a, b;
};

// forward pack at rank r: element (c, zl, y, x) of the slab [c][zl][y][x] goes to the block of y's
// owner d, [c][zl][yd][x] with yd the local index of y in d's set; off[d] = start of d's block
template <typename E>
__global__ void __launch_bounds__(256) k_pack_by_y(const E* __restrict__ src, E* __restrict__ dst, long long ncomp,
                                                   const __grid_constant__ SlabGeom g, const __grid_constant__ SlabOff o) {
  const int L = g.L, r = o.rank, Lz = g.z0[r + 1] - g.z0[r];
  const long long n = ncomp * Lz * L * L;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(e % L);
    long long t = e / L;
    const int y = (int)(t % L);
    t /= L;
    const int zl = (int)(t % Lz);
    const long long c = t / Lz;
    const int d = g.yowner[y];
    dst[o.off[d] + ((c * Lz + zl) * g.ny[d] + g.yloc[y]) * L + x] = src[e];
  }
}

// forward unpack at rank r: element (c, z, yl, x) of [c][z][yl][x] comes from the block of z's owner s,
// [c][zl][yl][x] with zl = z - z0[s]
template <typename E>
__global__ void __launch_bounds__(256) k_unpack_by_z(const E* __restrict__ src, E* __restrict__ dst, long long ncomp,
                                                     const __grid_constant__ SlabGeom g,
                                                     const __grid_constant__ SlabOff o) {
  const int L = g.L, ny = g.ny[o.rank];
  const long long n = ncomp * L * ny * L;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(e % L);
    long long t = e / L;
    const int yl = (int)(t % ny);
    t /= ny;
    const int z = (int)(t % L);
    const long long c = t / L;
    const int s = g.zowner[z], Lzs = g.z0[s + 1] - g.z0[s];
    dst[e] = src[o.off[s] + ((c * Lzs + (z - g.z0[s])) * ny + yl) * L + x];
  }
}

// inverse pack at rank r: element (c, z, yl, x) of [c][z][yl][x] goes to the block of z's owner d,
// [c][zl][yl][x]
template <typename E>
__global__ void __launch_bounds__(256) k_pack_by_z(const E* __restrict__ src, E* __restrict__ dst, long long ncomp,
                                                   const __grid_constant__ SlabGeom g, const __grid_constant__ SlabOff o) {
  const int L = g.L, ny = g.ny[o.rank];
  const long long n = ncomp * L * ny * L;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(e % L);
    long long t = e / L;
    const int yl = (int)(t % ny);
    t /= ny;
    const int z = (int)(t % L);
    const long long c = t / L;
    const int d = g.zowner[z], Lzd = g.z0[d + 1] - g.z0[d];
    dst[o.off[d] + ((c * Lzd + (z - g.z0[d])) * ny + yl) * L + x] = src[e];
  }
}

// inverse unpack at rank r: element (c, zl, y, x) of the slab [c][zl][y][x] comes from the block of y's
// owner s, [c][zl][ys][x] with ys the local index of y in s's set
template <typename E>
__global__ void __launch_bounds__(256) k_unpack_by_y(const E* __restrict__ src, E* __restrict__ dst, long long ncomp,
                                                     const __grid_constant__ SlabGeom g,
                                                     const __grid_constant__ SlabOff o) {
  const int L = g.L, r = o.rank, Lz = g.z0[r + 1] - g.z0[r];
  const long long n = ncomp * Lz * L * L;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(e % L);
    long long t = e / L;
    const int y = (int)(t % L);
    t /= L;
    const int zl = (int)(t % Lz);
    const long long c = t / Lz;
    const int s = g.yowner[y];
    dst[e] = src[o.off[s] + ((c * Lz + zl) * g.ny[s] + g.yloc[y]) * L + x];
  }
}

unsigned grid_for(long long n) { return (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 32)); }

}  // namespace

cudaError_t launch_slab_move(int kind, const void* src, void* dst, long long ncomp, const SlabGeom& g,
                             const SlabOff& o, cudaStream_t st) {
  const int L = g.L, r = o.rank;
  if (r < 0 || r >= g.P) return cudaErrorInvalidValue;
  const long long nslab = ncomp * (g.z0[r + 1] - g.z0[r]) * L * L, nmom = ncomp * L * g.ny[r] * L;
  switch (kind) {
    case SLAB_PACK_BLOCKS:
      k_pack_by_y<Cell4><<<grid_for(nslab), 256, 0, st>>>((const Cell4*)src, (Cell4*)dst, ncomp, g, o);
      break;
    case SLAB_UNPACK_BLOCKS:
      k_unpack_by_z<Cell4><<<grid_for(nmom), 256, 0, st>>>((const Cell4*)src, (Cell4*)dst, ncomp, g, o);
      break;
    case SLAB_PACK_CORR:
      k_pack_by_z<float2><<<grid_for(nmom), 256, 0, st>>>((const float2*)src, (float2*)dst, ncomp, g, o);
      break;
    case SLAB_UNPACK_CORR:
      k_unpack_by_y<float2><<<grid_for(nslab), 256, 0, st>>>((const float2*)src, (float2*)dst, ncomp, g, o);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace nbs
