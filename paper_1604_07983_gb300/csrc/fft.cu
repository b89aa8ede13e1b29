// fft.cu -- batched in-place 3-D FFT of L^3 cubes (Eq. (2.6) of arXiv:1604.07983).
//
// forward: X(q) = sum_x e^{-2 pi i q.x / L} x(x)       (dir = -1)
// inverse: x(r) = sum_q e^{+2 pi i q.r / L} X(q)       (dir = +1, unnormalised)
//
// Each line of L points is transformed by one thread in registers with a
// mixed-radix (3, 2, 2, ...) decimation-in-time FFT whose index arithmetic is
// resolved at compile time: the input is read in digit-reversed order,
// stage s combines sub-transforms of length n_{s-1} into n_s = n_{s-1} r_s
// with twiddles W_{n_s}^{j u}.  Lines along y and z are read straight from
// HBM (consecutive threads own consecutive lines, so each of the L loads is
// coalesced); lines along x are contiguous and are staged through shared
// memory.  The cube layout is [batch][z][y][x][i], i < IL interleaved values
// (IL = 4 for the stored blocks, 1 for the correlators).
#include "common.cuh"

#include <cmath>

namespace nbs {

namespace {

__host__ __device__ constexpr int fft_nst(int L) {
  int n = 0;
  while (L % 2 == 0) { L /= 2; ++n; }
  while (L % 3 == 0) { L /= 3; ++n; }
  return n;
}
__host__ __device__ constexpr int fft_radix(int L, int s) { return (L % 3 == 0 && s == 0) ? 3 : 2; }
__host__ __device__ constexpr int fft_nprod(int L, int s) {
  int n = 1;
  for (int i = 0; i < s; ++i) n *= fft_radix(L, i);
  return n;
}
// input index held at array position p before the first stage: the last
// stage's radix digit of p is the least significant digit of the input index
__host__ __device__ constexpr int fft_perm(int L, int p) {
  int res = 0, mult = 1;
  for (int s = fft_nst(L); s >= 1; --s) {
    const int np = fft_nprod(L, s - 1);
    res += mult * (p / np);
    p %= np;
    mult *= fft_radix(L, s - 1);
  }
  return res;
}
template <int L, int P> struct PermV { static constexpr int value = fft_perm(L, P); };

// x[p] = src[perm(p) * stride], unrolled with compile-time offsets
template <typename T, int L, int P = 0> struct LoadPerm {
  static __device__ __forceinline__ void run(C<T> (&x)[L], const C<T>* src, long long stride) {
    if constexpr (P < L) {
      x[P] = src[PermV<L, P>::value * stride];
      LoadPerm<T, L, P + 1>::run(x, src, stride);
    }
  }
};

// supported line lengths and their twiddle-table offsets
__host__ __device__ constexpr int size_at(int i) {
  return i == 0 ? 1 : i == 1 ? 2 : i == 2 ? 3 : i == 3 ? 4 : i == 4 ? 6 : i == 5 ? 8 : i == 6 ? 12
       : i == 7 ? 16 : i == 8 ? 24 : i == 9 ? 32 : i == 10 ? 48 : 0;
}
constexpr int kNSizes = 11;
__host__ __device__ constexpr int tw_offset(int L) {
  int off = 0;
  for (int i = 0; i < kNSizes; ++i) {
    if (size_at(i) == L) return off;
    off += size_at(i);
  }
  return -1;
}
constexpr int kTwTotal = 1 + 2 + 3 + 4 + 6 + 8 + 12 + 16 + 24 + 32 + 48;

// tw[k] = exp(-2 pi i k / L), k < L, computed on the host in double precision
__constant__ double2 c_tw64[kTwTotal];
__constant__ float2 c_tw32[kTwTotal];

template <typename T> __device__ __forceinline__ C<T> twiddle(int idx);
template <> __device__ __forceinline__ double2 twiddle<double>(int idx) { return c_tw64[idx]; }
template <> __device__ __forceinline__ float2 twiddle<float>(int idx) { return c_tw32[idx]; }

template <typename T, int DIR>
__device__ __forceinline__ C<T> mul_tw(C<T> v, C<T> w) {
  // forward multiplies by w, inverse by conj(w)
  if (DIR < 0) return cmake<T>(v.x * w.x - v.y * w.y, v.x * w.y + v.y * w.x);
  return cmake<T>(v.x * w.x + v.y * w.y, v.y * w.x - v.x * w.y);
}

template <typename T, int R, int DIR> struct Butterfly;
template <typename T, int DIR> struct Butterfly<T, 2, DIR> {
  static __device__ __forceinline__ void run(C<T>* z) {
    C<T> a = z[0], b = z[1];
    z[0] = cadd<T>(a, b);
    z[1] = csub<T>(a, b);
  }
};
template <typename T, int DIR> struct Butterfly<T, 3, DIR> {
  static __device__ __forceinline__ void run(C<T>* z) {
    // y_t = sum_u W3^{tu} z_u,  W3 = exp(DIR * 2 pi i / 3) = -1/2 + DIR i sqrt(3)/2
    const T h = T(0.86602540378443864676);  // sqrt(3)/2
    C<T> s = cadd<T>(z[1], z[2]), d = csub<T>(z[1], z[2]);
    C<T> m = cmake<T>(z[0].x - T(0.5) * s.x, z[0].y - T(0.5) * s.y);
    // i * DIR * h * d
    C<T> rot = cmake<T>(-T(DIR) * h * d.y, T(DIR) * h * d.x);
    z[0] = cadd<T>(z[0], s);
    z[1] = cadd<T>(m, rot);
    z[2] = csub<T>(m, rot);
  }
};

template <typename T, int L, int DIR, int S>
struct Stage {
  static __device__ __forceinline__ void run(C<T> (&x)[L]) {
    if constexpr (S < fft_nst(L)) {
      constexpr int r = fft_radix(L, S);
      constexpr int np = fft_nprod(L, S);
      constexpr int ns = np * r;
      constexpr int tw0 = tw_offset(L);
#pragma unroll
      for (int b = 0; b < L / ns; ++b) {
#pragma unroll
        for (int j = 0; j < np; ++j) {
          C<T> z[r];
#pragma unroll
          for (int u = 0; u < r; ++u) {
            C<T> v = x[b * ns + j + u * np];
            if (j * u != 0) v = mul_tw<T, DIR>(v, twiddle<T>(tw0 + (j * u) * (L / ns)));
            z[u] = v;
          }
          Butterfly<T, r, DIR>::run(z);
#pragma unroll
          for (int t = 0; t < r; ++t) x[b * ns + j + t * np] = z[t];
        }
      }
      Stage<T, L, DIR, S + 1>::run(x);
    }
  }
};

// lines along y or z: line l -> base = (l / inner) * group + (l % inner), step = stride
template <typename T, int L, int DIR>
__global__ void __launch_bounds__(256) k_fft_strided(C<T>* __restrict__ data, long long nlines, int inner,
                                                     long long group, int stride) {
  long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nlines) return;
  C<T>* base = data + (l / inner) * group + (l % inner);
  C<T> x[L];
  LoadPerm<T, L>::run(x, base, stride);
  Stage<T, L, DIR, 0>::run(x);
#pragma unroll
  for (int p = 0; p < L; ++p) base[(long long)p * stride] = x[p];
}

// lines along x: IL interleaved lines per row of L*IL contiguous elements
// (IL = 4 for blocks stored [cell][site][alpha]); NT lines per block staged
// through shared memory, line t of a block = (row t / IL, offset t % IL).
// FP32 with four interleaved values: rows padded by 4 (16-byte aligned rows, and
// the lines of a warp fall on distinct bank pairs); otherwise by 1
template <typename T, int IL>
constexpr int contig_pad() { return (sizeof(C<T>) == 8 && IL == 4) ? 4 : 1; }

template <typename T, int L, int DIR, int NT, int IL>
__global__ void __launch_bounds__(NT) k_fft_contig(C<T>* __restrict__ data, long long nlines) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* sm = reinterpret_cast<C<T>*>(smem_raw);
  constexpr int RL = L * IL;                        // row length
  constexpr int RP = RL + contig_pad<T, IL>();      // padded row
  const long long l0 = (long long)blockIdx.x * NT;  // NT is a multiple of IL
  const int nl = (int)min((long long)NT, nlines - l0);
  const int nrow = nl / IL;
  C<T>* g = data + (l0 / IL) * RL;
  if constexpr ((RP * sizeof(C<T>)) % 16 == 0 && (RL * sizeof(C<T>)) % 16 == 0) {
    // whole 16-byte pieces on both sides: copy without waiting on each load
    constexpr int V16 = 16 / (int)sizeof(C<T>);
    for (int e = threadIdx.x * V16; e < nrow * RL; e += NT * V16) {
      const unsigned sa = (unsigned)__cvta_generic_to_shared(sm + (e / RL) * RP + (e % RL));
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(g + e) : "memory");
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
  } else {
    for (int e = threadIdx.x; e < nrow * RL; e += NT) sm[(e / RL) * RP + (e % RL)] = g[e];
  }
  __syncthreads();
  if (threadIdx.x < nl) {
    C<T>* row = sm + (threadIdx.x / IL) * RP + (threadIdx.x % IL);
    C<T> x[L];
    LoadPerm<T, L>::run(x, row, IL);
    Stage<T, L, DIR, 0>::run(x);
#pragma unroll
    for (int p = 0; p < L; ++p) row[p * IL] = x[p];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nrow * RL; e += NT) g[e] = sm[(e / RL) * RP + (e % RL)];
}

// lines along y and z in one pass: a block stages the (z, y) planes of XB
// consecutive x (IL interleaved values each) of one cube in shared memory --
// each (z, y) row of XB * IL values is one contiguous run in HBM -- transforms
// every y line, then every z line, in place, and writes the planes back.  One
// read and one write of the data instead of two of each.
template <typename T, int L, int DIR, int IL, int XB, int NT>
__global__ void __launch_bounds__(NT) k_fft_yz(C<T>* __restrict__ data, long long ncubes) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* sm = reinterpret_cast<C<T>*>(smem_raw);  // [z][y][xi][i]
  constexpr int RUN = XB * IL;                    // contiguous values per (z, y) row
  constexpr int NE = L * L * RUN;
  constexpr int NLINE = L * RUN;                  // lines per direction
  const long long cube = blockIdx.x / (L / XB);
  const int x0 = (int)(blockIdx.x % (L / XB)) * XB;
  if (cube >= ncubes) return;
  C<T>* g = data + cube * (long long)L * L * L * IL + (long long)x0 * IL;
  if constexpr ((RUN * sizeof(C<T>)) % 16 == 0 && (L * IL * sizeof(C<T>)) % 16 == 0) {
    // rows of RUN values start on 16-byte boundaries: copy the tile 16 bytes at a
    // time without waiting on each load, so the whole tile is in flight at once
    constexpr int V16 = 16 / (int)sizeof(C<T>);  // values per 16-byte piece
    for (int e = threadIdx.x * V16; e < NE; e += NT * V16) {
      const int zy = e / RUN, r = e % RUN;
      const unsigned sa = (unsigned)__cvta_generic_to_shared(sm + e);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(g + (long long)zy * L * IL + r)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
  } else {
    for (int e = threadIdx.x; e < NE; e += NT) {
      const int zy = e / RUN, r = e % RUN;
      sm[e] = g[(long long)zy * L * IL + r];
    }
  }
  __syncthreads();
  for (int l = threadIdx.x; l < NLINE; l += NT) {  // y lines: (z, run offset)
    C<T>* row = sm + (l / RUN) * L * RUN + (l % RUN);
    C<T> x[L];
    LoadPerm<T, L>::run(x, row, RUN);
    Stage<T, L, DIR, 0>::run(x);
#pragma unroll
    for (int p = 0; p < L; ++p) row[p * RUN] = x[p];
  }
  __syncthreads();
  for (int l = threadIdx.x; l < NLINE; l += NT) {  // z lines: (y, run offset)
    C<T>* row = sm + (l / RUN) * RUN + (l % RUN);
    C<T> x[L];
    LoadPerm<T, L>::run(x, row, L * RUN);
    Stage<T, L, DIR, 0>::run(x);
#pragma unroll
    for (int p = 0; p < L; ++p) row[p * L * RUN] = x[p];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NE; e += NT) {
    const int zy = e / RUN, r = e % RUN;
    g[(long long)zy * L * IL + r] = sm[e];
  }
}

// x values per block of the fused y/z pass: the planes take about 64 KB
template <typename T, int L, int IL>
constexpr int yz_xb() {
  int xb = (int)(65536 / ((long long)L * L * IL * (int)sizeof(C<T>)));
  if (xb < 1) xb = 1;
  while (L % xb) --xb;
  return xb;
}

// batch cubes of L^3 elements, each element a vector of IL interleaved values
// sb: threads per block of the two strided passes (64, 128 or 256; a tuning parameter)
template <typename T, int L, int DIR, int IL>
cudaError_t run3d(C<T>* data, long long nbatch, int sb, cudaStream_t st) {
  const long long nlines = nbatch * IL * L * L;
  if (nlines == 0 || L == 1) return cudaSuccess;
  {
    constexpr int NT = 64;
    size_t sm = (size_t)(NT / IL) * (L * IL + contig_pad<T, IL>()) * sizeof(C<T>);
    auto kern = k_fft_contig<T, L, DIR, NT, IL>;
    if (sm > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    long long blocks = (nlines + NT - 1) / NT;
    kern<<<(unsigned)blocks, NT, sm, st>>>(data, nlines);
  }
  if (sb != 64 && sb != 128 && sb != 256) return cudaErrorInvalidValue;
  if constexpr (L >= 16 && sizeof(T) == 4) {  // FP32: y and z in one pass through shared memory (for FP64
                                              // the planes leave one block per SM and the strided passes win)
    constexpr int XB = yz_xb<T, L, IL>();
    constexpr int NT = 256;
    const size_t sm = (size_t)L * L * XB * IL * sizeof(C<T>);
    auto kern = k_fft_yz<T, L, DIR, IL, XB, NT>;
    if (sm > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    const long long blocks = nbatch * (L / XB);
    if (blocks > 2147483647LL) return cudaErrorInvalidValue;
    kern<<<(unsigned)blocks, NT, sm, st>>>(data, nbatch);
    return cudaGetLastError();
  }
  // y: lines (batch, z, x, i): inner = IL*L, group = IL*L^2, stride IL*L
  {
    long long blocks = (nlines + sb - 1) / sb;
    k_fft_strided<T, L, DIR><<<(unsigned)blocks, sb, 0, st>>>(data, nlines, IL * L, (long long)IL * L * L, IL * L);
  }
  // z: lines (batch, y, x, i): inner = IL*L^2, group = IL*L^3, stride IL*L^2
  {
    long long blocks = (nlines + sb - 1) / sb;
    k_fft_strided<T, L, DIR><<<(unsigned)blocks, sb, 0, st>>>(data, nlines, IL * L * L, (long long)IL * L * L * L,
                                                              IL * L * L);
  }
  return cudaGetLastError();
}

template <typename T, int DIR, int IL>
cudaError_t dispatch(C<T>* data, long long nbatch, int L, int sb, cudaStream_t st) {
  switch (L) {
    case 1: return cudaSuccess;
    case 2: return run3d<T, 2, DIR, IL>(data, nbatch, sb, st);
    case 3: return run3d<T, 3, DIR, IL>(data, nbatch, sb, st);
    case 4: return run3d<T, 4, DIR, IL>(data, nbatch, sb, st);
    case 6: return run3d<T, 6, DIR, IL>(data, nbatch, sb, st);
    case 8: return run3d<T, 8, DIR, IL>(data, nbatch, sb, st);
    case 12: return run3d<T, 12, DIR, IL>(data, nbatch, sb, st);
    case 16: return run3d<T, 16, DIR, IL>(data, nbatch, sb, st);
    case 24: return run3d<T, 24, DIR, IL>(data, nbatch, sb, st);
    case 32: return run3d<T, 32, DIR, IL>(data, nbatch, sb, st);
    case 48: return run3d<T, 48, DIR, IL>(data, nbatch, sb, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int DIR>
cudaError_t lines_L(C<T>* data, long long nlines, int inner, long long group, long long stride, int L, int sb,
                    cudaStream_t st) {
  const long long blocks = (nlines + sb - 1) / sb;
  if (blocks > 2147483647LL || stride > 2147483647LL) return cudaErrorInvalidValue;
  switch (L) {
#define NBS_LINES(n) \
  case n: k_fft_strided<T, n, DIR><<<(unsigned)blocks, sb, 0, st>>>(data, nlines, inner, group, (int)stride); break;
    NBS_LINES(2) NBS_LINES(3) NBS_LINES(4) NBS_LINES(6) NBS_LINES(8) NBS_LINES(12) NBS_LINES(16) NBS_LINES(24)
    NBS_LINES(32) NBS_LINES(48)
#undef NBS_LINES
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T, int L, int DIR, int IL>
cudaError_t rows_L(C<T>* data, long long nrows, cudaStream_t st) {
  constexpr int NT = 64;
  const long long nlines = nrows * IL;
  const size_t sm = (size_t)(NT / IL) * (L * IL + contig_pad<T, IL>()) * sizeof(C<T>);
  auto kern = k_fft_contig<T, L, DIR, NT, IL>;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  const long long blocks = (nlines + NT - 1) / NT;
  if (blocks > 2147483647LL) return cudaErrorInvalidValue;
  kern<<<(unsigned)blocks, NT, sm, st>>>(data, nlines);
  return cudaGetLastError();
}

template <typename T, int DIR, int IL>
cudaError_t rows_dispatch(C<T>* data, long long nrows, int L, cudaStream_t st) {
  switch (L) {
    case 1: return cudaSuccess;
    case 2: return rows_L<T, 2, DIR, IL>(data, nrows, st);
    case 3: return rows_L<T, 3, DIR, IL>(data, nrows, st);
    case 4: return rows_L<T, 4, DIR, IL>(data, nrows, st);
    case 6: return rows_L<T, 6, DIR, IL>(data, nrows, st);
    case 8: return rows_L<T, 8, DIR, IL>(data, nrows, st);
    case 12: return rows_L<T, 12, DIR, IL>(data, nrows, st);
    case 16: return rows_L<T, 16, DIR, IL>(data, nrows, st);
    case 24: return rows_L<T, 24, DIR, IL>(data, nrows, st);
    case 32: return rows_L<T, 32, DIR, IL>(data, nrows, st);
    case 48: return rows_L<T, 48, DIR, IL>(data, nrows, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

template <typename T>
cudaError_t fft_lines(C<T>* data, long long nlines, int inner, long long group, long long stride, int L, int dir,
                      int sb, cudaStream_t st) {
  if (nlines == 0 || L == 1) return cudaSuccess;
  if (sb != 64 && sb != 128 && sb != 256) return cudaErrorInvalidValue;
  return dir < 0 ? lines_L<T, -1>(data, nlines, inner, group, stride, L, sb, st)
                 : lines_L<T, 1>(data, nlines, inner, group, stride, L, sb, st);
}

template <typename T>
cudaError_t fft_rows(C<T>* data, long long nrows, int L, int IL, int dir, cudaStream_t st) {
  if (nrows == 0 || L == 1) return cudaSuccess;
  if (IL == 4) return dir < 0 ? rows_dispatch<T, -1, 4>(data, nrows, L, st) : rows_dispatch<T, 1, 4>(data, nrows, L, st);
  if (IL == 1) return dir < 0 ? rows_dispatch<T, -1, 1>(data, nrows, L, st) : rows_dispatch<T, 1, 1>(data, nrows, L, st);
  return cudaErrorInvalidValue;
}

template cudaError_t fft_lines<float>(float2*, long long, int, long long, long long, int, int, int, cudaStream_t);
template cudaError_t fft_lines<double>(double2*, long long, int, long long, long long, int, int, int, cudaStream_t);
template cudaError_t fft_rows<float>(float2*, long long, int, int, int, cudaStream_t);
template cudaError_t fft_rows<double>(double2*, long long, int, int, int, cudaStream_t);

bool fft_supported(int L) { return tw_offset(L) >= 0; }

cudaError_t fft_init() {
  double2 t64[kTwTotal];
  float2 t32[kTwTotal];
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < kNSizes; ++i) {
    int L = size_at(i), off = tw_offset(L);
    for (int k = 0; k < L; ++k) {
      double a = -2.0 * pi * k / L;
      t64[off + k] = make_double2(std::cos(a), std::sin(a));
      t32[off + k] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
  }
  cudaError_t e = cudaMemcpyToSymbol(c_tw64, t64, sizeof(t64));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_tw32, t32, sizeof(t32));
}

// forward transform of the stored blocks [cell][site][alpha] (4 interleaved cubes per cell)
template <typename T>
cudaError_t fft3d_blocks(C<T>* data, long long ncells, int L, cudaStream_t st, int sb) {
  return dispatch<T, -1, 4>(data, ncells, L, sb, st);
}

// inverse transform of nbatch contiguous cubes
template <typename T>
cudaError_t fft3d_inverse(C<T>* data, long long nbatch, int L, cudaStream_t st, int sb) {
  return dispatch<T, +1, 1>(data, nbatch, L, sb, st);
}

template cudaError_t fft3d_blocks<float>(float2*, long long, int, cudaStream_t, int);
template cudaError_t fft3d_blocks<double>(double2*, long long, int, cudaStream_t, int);
template cudaError_t fft3d_inverse<float>(float2*, long long, int, cudaStream_t, int);
template cudaError_t fft3d_inverse<double>(double2*, long long, int, cudaStream_t, int);

}  // namespace nbs
