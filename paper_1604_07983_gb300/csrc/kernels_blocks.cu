// kernels_blocks.cu -- propagator rescale and baryon blocks (Sec. 4 (i), Eq. (4.1)).
//
// Stage a0: per-timeslice, per-flavour scale 2^e with max|S| * 2^-e in [1/2, 1)
// (power of two, so the FP64 restore of the result is exact), applied while
// the propagators are transposed from [site][i][j] to the site-contiguous
// [flavour][i*12 + j][site] layout every later kernel reads coalesced.
//
// Stage a1: the diquarks
//   Q^{d}_c(x; j1, j2) = sum_{ab} eps_abc sum_{beta gamma} (Cg5)_{beta gamma}
//                        S_f0[x](beta a; j1) S_f1[x](gamma b; j2)
// for the diquark flavour pairs d = (f0, f1) of plan.h (ll, ls with u = d;
// uu, ud, dd, us, ds with three propagators)
// then the stored field blocks
//   FB_T(alpha; y0, y1, y2) = sum_terms coef * sum_c Q^{d}_c(y_a0, y_a1) S_f3[x](alpha c; y_a2),
// i.e. the normal block of Eq. (4.1) N^{f1 f2 f3}_alpha(j1, j2, j3)
//   = sum_c Q^{f1 f2}_c(j1, j2) S_f3(alpha c; j3), summed over the
// monomials and same-flavour assignments of the field (the flavour merge
// that the paper does per field, Sec. 4 (i)-(ii)).
// Output layout: FB[cell][site][alpha]: per cell four interleaved L^3 cubes.
#include "common.cuh"
#include "plan.h"

namespace nbs {

namespace {

template <typename Tin> struct InC;
template <> struct InC<double> { using type = double2; };
template <> struct InC<float> { using type = float2; };

__device__ __forceinline__ double cabs2(double2 z) { return z.x * z.x + z.y * z.y; }
__device__ __forceinline__ double cabs2(float2 z) { return (double)z.x * z.x + (double)z.y * z.y; }

template <typename Tin>
__global__ void __launch_bounds__(256) k_maxabs(const PropPtrs props, long long n,
                                                unsigned long long* __restrict__ maxbits, int* __restrict__ flags) {
  const auto* src = reinterpret_cast<const typename InC<Tin>::type*>(props.p[blockIdx.y]);
  double m = 0.0;
  bool bad = false;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    auto z = src[i];
    double a = cabs2(z);
    bad |= !isfinite(a);
    m = fmax(m, a);
  }
  // warp then block reduction of the maximum
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    // non-negative doubles order like their bit patterns
    atomicMax(maxbits + blockIdx.y, (unsigned long long)__double_as_longlong(sqrt(m)));
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, 1);
}

__device__ __forceinline__ int scale_exponent(unsigned long long bits) {
  double m = __longlong_as_double((long long)bits);
  if (!(m > 0.0) || !isfinite(m)) return 0;
  int e;
  frexp(m, &e);  // m = f * 2^e, f in [1/2, 1)
  return e;
}

// 16 sites per block; out[f][e][site] = in[site][e] * 2^-exp_f
template <typename Tin, typename T>
__global__ void __launch_bounds__(256) k_scale_transpose(const PropPtrs props, int V,
                                                         const unsigned long long* __restrict__ maxbits,
                                                         int* __restrict__ exps, C<T>* __restrict__ out) {
  constexpr int NS = 16;
  __shared__ C<T> tile[144][NS + 1];
  const int f = blockIdx.y;
  const auto* src = reinterpret_cast<const typename InC<Tin>::type*>(props.p[f]);
  const int e = scale_exponent(maxbits[f]);
  if (blockIdx.x == 0 && threadIdx.x == 0) exps[f] = e;
  const int site0 = blockIdx.x * NS;
  const int ns = min(NS, V - site0);
  for (int k = threadIdx.x; k < ns * 144; k += blockDim.x) {
    auto z = src[(long long)site0 * 144 + k];
    tile[k % 144][k / 144] = cmake<T>((T)ldexp((double)z.x, -e), (T)ldexp((double)z.y, -e));
  }
  __syncthreads();
  C<T>* o = out + (long long)f * 144 * V;
  for (int k = threadIdx.x; k < ns * 144; k += blockDim.x) {
    int el = k / ns, st = k % ns;
    o[(long long)el * V + site0 + st] = tile[el][st];
  }
}

// Q[(d*3 + c)*144 + j1*12 + j2][site] for diquark d = (f0, f1)
struct DiquarkPairs { int f0[NBS_MAX_DIQUARKS], f1[NBS_MAX_DIQUARKS]; };

template <typename T>
__global__ void __launch_bounds__(128) k_diquarks(const C<T>* __restrict__ P, int V, const DiquarkPairs dp,
                                                  C<T>* __restrict__ Q) {
  const int site = blockIdx.x * blockDim.x + threadIdx.x;
  if (site >= V) return;
  const int d = blockIdx.y / 12, j1 = blockIdx.y % 12;
  const C<T>* S1 = P + (long long)dp.f0[d] * 144 * V;
  const C<T>* S2 = P + (long long)dp.f1[d] * 144 * V;
  C<T> a[12];  // S1[(beta, a); j1], index 3*beta + a
#pragma unroll
  for (int i = 0; i < 12; ++i) a[i] = S1[(long long)(i * 12 + j1) * V + site];
  for (int j2 = 0; j2 < 12; ++j2) {
    C<T> b[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) b[i] = S2[(long long)(i * 12 + j2) * V + site];
    // D_ab = sum_{beta gamma} Cg5_{beta gamma} a(beta, a) b(gamma, b)
    //      = a0 b1 - a1 b0 + a2 b3 - a3 b2   (spin indices)
    C<T> D[3][3];
#pragma unroll
    for (int ca = 0; ca < 3; ++ca)
#pragma unroll
      for (int cb = 0; cb < 3; ++cb) {
        if (ca == cb) continue;
        C<T> acc = czero<T>();
        cfma<T>(acc, a[0 * 3 + ca], b[1 * 3 + cb]);
        cfma<T>(acc, a[1 * 3 + ca], cmake<T>(-b[0 * 3 + cb].x, -b[0 * 3 + cb].y));
        cfma<T>(acc, a[2 * 3 + ca], b[3 * 3 + cb]);
        cfma<T>(acc, a[3 * 3 + ca], cmake<T>(-b[2 * 3 + cb].x, -b[2 * 3 + cb].y));
        D[ca][cb] = acc;
      }
    // Q_c = sum_ab eps_abc D_ab
    C<T> q0 = csub<T>(D[1][2], D[2][1]);
    C<T> q1 = csub<T>(D[2][0], D[0][2]);
    C<T> q2 = csub<T>(D[0][1], D[1][0]);
    const long long base = (long long)((d * 3) * 144 + j1 * 12 + j2) * V + site;
    Q[base] = q0;
    Q[base + 144LL * V] = q1;
    Q[base + 288LL * V] = q2;
  }
}

// one cell per blockIdx.y, sites along x; cells[g] = y0 + 12 y1 + 144 y2 + (type << 11)
template <typename T, int NF>
__global__ void __launch_bounds__(128) k_field_blocks(const C<T>* __restrict__ P, const C<T>* __restrict__ Q,
                                                      const int* __restrict__ cells, const TypeRecipeSet rs, int V,
                                                      C<T>* __restrict__ FB) {
  const int site = blockIdx.x * blockDim.x + threadIdx.x;
  if (site >= V) return;
  const int g = blockIdx.y;
  const int code = cells[g];
  const int type = code >> 11;
  const int key = code & 2047;
  int y[3] = {key % 12, (key / 12) % 12, key / 144};
  const TypeRecipe& R = rs.t[type];
  C<T> out[4] = {czero<T>(), czero<T>(), czero<T>(), czero<T>()};
  for (int t = 0; t < R.nterms; ++t) {
    const int pat = R.pat[t], arg = R.arg[t];
    const T coef = (T)R.coef[t];
    const int j1 = y[arg & 3], j2 = y[(arg >> 2) & 3], j3 = y[(arg >> 4) & 3];
    const int d = pat / NF;   // pattern = diquark * NF + flavour of the third quark
    const int f3 = pat % NF;
    const C<T>* S3 = P + (long long)f3 * 144 * V;
    C<T> q[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) q[c] = Q[(long long)((d * 3 + c) * 144 + j1 * 12 + j2) * V + site];
#pragma unroll
    for (int al = 0; al < 4; ++al) {
      C<T> n = czero<T>();
#pragma unroll
      for (int c = 0; c < 3; ++c) cfma<T>(n, q[c], S3[(long long)((3 * al + c) * 12 + j3) * V + site]);
      crfma<T>(out[al], coef, n);
    }
  }
  // [cell][site][alpha]: the four spins of a site are one 32-byte (FP32) or 64-byte (FP64) run
  C<T>* o = FB + ((long long)g * V + site) * 4;
#pragma unroll
  for (int al = 0; al < 4; ++al) o[al] = out[al];
}

// Site-tiled form of the two kernels above: a block owns TS consecutive sites,
// stages their scaled propagators ([flavour][144][TS]) in shared memory, forms
// their diquarks there ([diquark][c][144][TS]) and writes every stored cell of
// those sites.  Propagators are read from HBM once and the diquarks never
// leave the SM; the cell loop reads its 15 values per term from shared memory
// instead of L2.
template <typename T, int NF, int TS>
__global__ void __launch_bounds__(256) k_blocks_tiled(const C<T>* __restrict__ P, const int* __restrict__ cells,
                                                      int ncells, const TypeRecipeSet rs, int V, const DiquarkPairs dp,
                                                      C<T>* __restrict__ FB) {
  constexpr int NT = 256;
  constexpr int ND = NF == 2 ? 2 : 5;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* Ps = reinterpret_cast<C<T>*>(smem_raw);  // [NF][144][TS]
  C<T>* Qs = Ps + NF * 144 * TS;                  // [ND][3][144][TS]
  const int site0 = blockIdx.x * TS;
  const int ns = min(TS, V - site0);
  for (int e = threadIdx.x; e < NF * 144 * TS; e += NT) {
    const int row = e / TS, st = e % TS;
    Ps[e] = st < ns ? P[(long long)row * V + site0 + st] : czero<T>();
  }
  __syncthreads();
  for (int it = threadIdx.x; it < ND * 12 * TS; it += NT) {  // (d, j1, site), loop over j2
    const int st = it % TS, j1 = (it / TS) % 12, d = it / (12 * TS);
    const C<T>* S1 = Ps + dp.f0[d] * 144 * TS + st;
    const C<T>* S2 = Ps + dp.f1[d] * 144 * TS + st;
    C<T> a[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) a[i] = S1[(i * 12 + j1) * TS];
    for (int j2 = 0; j2 < 12; ++j2) {
      C<T> b[12];
#pragma unroll
      for (int i = 0; i < 12; ++i) b[i] = S2[(i * 12 + j2) * TS];
      C<T> D[3][3];
#pragma unroll
      for (int ca = 0; ca < 3; ++ca)
#pragma unroll
        for (int cb = 0; cb < 3; ++cb) {
          if (ca == cb) continue;
          C<T> acc = czero<T>();
          cfma<T>(acc, a[0 * 3 + ca], b[1 * 3 + cb]);
          cfma<T>(acc, a[1 * 3 + ca], cmake<T>(-b[0 * 3 + cb].x, -b[0 * 3 + cb].y));
          cfma<T>(acc, a[2 * 3 + ca], b[3 * 3 + cb]);
          cfma<T>(acc, a[3 * 3 + ca], cmake<T>(-b[2 * 3 + cb].x, -b[2 * 3 + cb].y));
          D[ca][cb] = acc;
        }
      C<T>* q = Qs + ((d * 3) * 144 + j1 * 12 + j2) * TS + st;
      q[0] = csub<T>(D[1][2], D[2][1]);
      q[144 * TS] = csub<T>(D[2][0], D[0][2]);
      q[288 * TS] = csub<T>(D[0][1], D[1][0]);
    }
  }
  __syncthreads();
  for (int it = threadIdx.x; it < ncells * TS; it += NT) {
    const int st = it % TS, g = it / TS;
    const int code = cells[g];
    const int key = code & 2047;
    const int y0 = key % 12, y1 = (key / 12) % 12, y2 = key / 144;
    const TypeRecipe& R = rs.t[code >> 11];
    C<T> out[4] = {czero<T>(), czero<T>(), czero<T>(), czero<T>()};
    for (int t = 0; t < R.nterms; ++t) {
      const int pat = R.pat[t], arg = R.arg[t];
      const T coef = (T)R.coef[t];
      // positions a0, a1, a2 of the normal block's arguments among (y0, y1, y2), by selects
      const int a0 = arg & 3, a1 = (arg >> 2) & 3, a2 = (arg >> 4) & 3;
      const int j1 = a0 == 0 ? y0 : (a0 == 1 ? y1 : y2);
      const int j2 = a1 == 0 ? y0 : (a1 == 1 ? y1 : y2);
      const int j3 = a2 == 0 ? y0 : (a2 == 1 ? y1 : y2);
      const int d = pat / NF, f3 = pat % NF;
      const C<T>* S3 = Ps + f3 * 144 * TS + st;
      const C<T>* q = Qs + ((d * 3) * 144 + j1 * 12 + j2) * TS + st;
      const C<T> q0 = q[0], q1 = q[144 * TS], q2 = q[288 * TS];
#pragma unroll
      for (int al = 0; al < 4; ++al) {
        C<T> n = czero<T>();
        cfma<T>(n, q0, S3[((3 * al + 0) * 12 + j3) * TS]);
        cfma<T>(n, q1, S3[((3 * al + 1) * 12 + j3) * TS]);
        cfma<T>(n, q2, S3[((3 * al + 2) * 12 + j3) * TS]);
        crfma<T>(out[al], coef, n);
      }
    }
    if (st < ns) {
      C<T>* o = FB + ((long long)g * V + site0 + st) * 4;
#pragma unroll
      for (int al = 0; al < 4; ++al) o[al] = out[al];
    }
  }
}

template <typename T, int NF>
constexpr int tiled_sites() { return (sizeof(T) == 8 && NF == 3) ? 4 : 8; }

}  // namespace

template <typename T>
size_t blocks_tiled_smem(int nflav) {
  const int ts = nflav == 2 ? tiled_sites<T, 2>() : tiled_sites<T, 3>();
  return (size_t)(nflav + 3 * n_diquarks(nflav)) * 144 * ts * sizeof(C<T>);
}

template <typename T>
cudaError_t launch_blocks_tiled(const C<T>* props, const int* cells, int ncells, const TypeRecipeSet& recipes, int V,
                                int nflav, C<T>* FB, cudaStream_t st) {
  DiquarkPairs dp = {};
  for (int d = 0; d < n_diquarks(nflav); ++d) diquark_flavours(nflav, d, dp.f0[d], dp.f1[d]);
  const size_t sm = blocks_tiled_smem<T>(nflav);
  if (nflav == 2) {
    constexpr int TS = tiled_sites<T, 2>();
    auto kern = k_blocks_tiled<T, 2, TS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    kern<<<(V + TS - 1) / TS, 256, sm, st>>>(props, cells, ncells, recipes, V, dp, FB);
  } else if (nflav == 3) {
    constexpr int TS = tiled_sites<T, 3>();
    auto kern = k_blocks_tiled<T, 3, TS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    kern<<<(V + TS - 1) / TS, 256, sm, st>>>(props, cells, ncells, recipes, V, dp, FB);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_props_maxabs(const PropPtrs& props, int nflav, int in_c64, int V, unsigned long long* maxbits,
                                int* flags, cudaStream_t st) {
  long long n = (long long)V * 144;
  int blocks = (int)min((n + 255) / 256, 1216LL);
  dim3 grid(blocks, nflav);
  if (in_c64)
    k_maxabs<float><<<grid, 256, 0, st>>>(props, n, maxbits, flags);
  else
    k_maxabs<double><<<grid, 256, 0, st>>>(props, n, maxbits, flags);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_props_scale(const PropPtrs& props, int nflav, int in_c64, int V, const unsigned long long* maxbits,
                               int* exps, C<T>* out, cudaStream_t st) {
  dim3 grid((V + 15) / 16, nflav);
  if (in_c64)
    k_scale_transpose<float, T><<<grid, 256, 0, st>>>(props, V, maxbits, exps, out);
  else
    k_scale_transpose<double, T><<<grid, 256, 0, st>>>(props, V, maxbits, exps, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_diquarks(const C<T>* props, int V, int nflav, C<T>* Q, cudaStream_t st) {
  DiquarkPairs dp = {};
  const int nd = n_diquarks(nflav);
  for (int d = 0; d < nd; ++d) diquark_flavours(nflav, d, dp.f0[d], dp.f1[d]);
  dim3 grid((V + 127) / 128, nd * 12);
  k_diquarks<T><<<grid, 128, 0, st>>>(props, V, dp, Q);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_field_blocks(const C<T>* props, const C<T>* Q, const int* cells, int ncells,
                                const TypeRecipeSet& recipes, int V, int nflav, C<T>* FB, cudaStream_t st) {
  if (ncells > 65535) return cudaErrorInvalidValue;
  dim3 grid((V + 127) / 128, ncells);
  if (nflav == 2)
    k_field_blocks<T, 2><<<grid, 128, 0, st>>>(props, Q, cells, recipes, V, FB);
  else if (nflav == 3)
    k_field_blocks<T, 3><<<grid, 128, 0, st>>>(props, Q, cells, recipes, V, FB);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template cudaError_t launch_props_scale<float>(const PropPtrs&, int, int, int, const unsigned long long*, int*,
                                               float2*, cudaStream_t);
template cudaError_t launch_props_scale<double>(const PropPtrs&, int, int, int, const unsigned long long*, int*,
                                                double2*, cudaStream_t);
template cudaError_t launch_blocks_tiled<float>(const float2*, const int*, int, const TypeRecipeSet&, int, int, float2*,
                                                cudaStream_t);
template cudaError_t launch_blocks_tiled<double>(const double2*, const int*, int, const TypeRecipeSet&, int, int,
                                                 double2*, cudaStream_t);
template cudaError_t launch_diquarks<float>(const float2*, int, int, float2*, cudaStream_t);
template cudaError_t launch_diquarks<double>(const double2*, int, int, double2*, cudaStream_t);
template cudaError_t launch_field_blocks<float>(const float2*, const float2*, const int*, int,
                                                const TypeRecipeSet&, int, int, float2*, cudaStream_t);
template cudaError_t launch_field_blocks<double>(const double2*, const double2*, const int*, int,
                                                 const TypeRecipeSet&, int, int, double2*, cudaStream_t);

}  // namespace nbs
