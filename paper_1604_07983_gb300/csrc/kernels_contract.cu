// kernels_contract.cu -- effective blocks and their product in momentum space
// (Sec. 4 (ii)-(iii), Eqs. (4.2)-(4.3) of arXiv:1604.07983), and the restore
// of the correlator after the inverse FFT.
//
// One thread owns one momentum q (and A1 of the four sink spins alpha1); the
// threads of a warp own 32 consecutive q, so every gather of a stored block
// cell reads one contiguous run of 32 x 4 spins (FP32: 1 KB) and every thread
// runs the same table-driven program (the SoA layout the paper uses against
// warp divergence).  For each term of the channel and each shared source index
// xi~ the thread forms
//   e1[alpha1][h1] = sum_i coef1_i * FB~[cell1_i](q)     (B1 block at  q)
//   e2[alpha2][h2] = sum_i coef2_i * FB~[cell2_i](-q)    (B2 block at -q)
// and accumulates F~[alpha1][alpha2][alpha3][alpha4](q) += e1 * e2, the
// held spins (h1, h2) carrying alpha3 / alpha4 as the term's shape says.
#include "common.cuh"
#include "plan.h"

#include <algorithm>

namespace nbs {

namespace {

// N consecutive complex values (the sink spins of one stored cell and site),
// from a 16-byte aligned address, with 16-byte loads through the read-only path
template <typename T, int N> struct AlphaLoad;
template <int N> struct AlphaLoad<float, N> {
  static __device__ __forceinline__ void run(const float2* p, float2 (&x)[N]) {
    if constexpr (N == 1) {
      x[0] = __ldg(p);
    } else {
#pragma unroll
      for (int v = 0; v < N / 2; ++v) {
        const float4 w = __ldg(reinterpret_cast<const float4*>(p) + v);
        x[2 * v] = make_float2(w.x, w.y);
        x[2 * v + 1] = make_float2(w.z, w.w);
      }
    }
  }
};
template <int N> struct AlphaLoad<double, N> {
  static __device__ __forceinline__ void run(const double2* p, double2 (&x)[N]) {
#pragma unroll
    for (int v = 0; v < N; ++v) x[v] = __ldg(p + v);
  }
};

// one term: for each shared index k, the two effective blocks from their
// gather lists (ordered [i][h], i even) and their outer product into acc
template <typename T, int A1, int SHAPE>
__device__ __forceinline__ void run_term(const DevTerm& h, const C<T>* __restrict__ FB, long long cs, long long qoff,
                                         long long qmoff, const Ent<T>* __restrict__ E1,
                                         const Ent<T>* __restrict__ E2, C<T> (&acc)[A1][4][4]) {
  constexpr int NH1 = 1 << ((SHAPE & 1) + ((SHAPE >> 1) & 1));
  constexpr int NH2 = 4 / NH1;
  const int n1 = h.n1, n2 = h.n2;
  const Ent<T>* p1 = E1 + h.off1;
  const Ent<T>* p2 = E2 + h.off2;
  for (int k = 0; k < h.K; ++k) {
    C<T> v1[NH1][A1];
    C<T> v2[NH2][4];
#pragma unroll
    for (int hh = 0; hh < NH1; ++hh)
#pragma unroll
      for (int a = 0; a < A1; ++a) v1[hh][a] = czero<T>();
#pragma unroll
    for (int hh = 0; hh < NH2; ++hh)
#pragma unroll
      for (int b = 0; b < 4; ++b) v2[hh][b] = czero<T>();
    for (int i = 0; i < n1; i += 2, p1 += 2 * NH1) {
      int cell[2 * NH1];
      T coef[2 * NH1];
#pragma unroll
      for (int j = 0; j < 2 * NH1; ++j) { cell[j] = __ldg(&p1[j].cell); coef[j] = __ldg(&p1[j].coef); }
      C<T> x[2 * NH1][A1];
#pragma unroll
      for (int j = 0; j < 2 * NH1; ++j) AlphaLoad<T, A1>::run(FB + cell[j] * cs + qoff, x[j]);
#pragma unroll
      for (int j = 0; j < 2 * NH1; ++j)
#pragma unroll
        for (int a = 0; a < A1; ++a) crfma<T>(v1[j % NH1][a], coef[j], x[j][a]);
    }
    for (int i = 0; i < n2; i += 2, p2 += 2 * NH2) {
      int cell[2 * NH2];
      T coef[2 * NH2];
#pragma unroll
      for (int j = 0; j < 2 * NH2; ++j) { cell[j] = __ldg(&p2[j].cell); coef[j] = __ldg(&p2[j].coef); }
      C<T> x[2 * NH2][4];
#pragma unroll
      for (int j = 0; j < 2 * NH2; ++j) AlphaLoad<T, 4>::run(FB + cell[j] * cs + qmoff, x[j]);
#pragma unroll
      for (int j = 0; j < 2 * NH2; ++j)
#pragma unroll
        for (int b = 0; b < 4; ++b) crfma<T>(v2[j % NH2][b], coef[j], x[j][b]);
    }
#pragma unroll
    for (int a = 0; a < A1; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int h1 = 0; h1 < NH1; ++h1)
#pragma unroll
          for (int h2 = 0; h2 < NH2; ++h2) {
            // spin slot s = alpha3 + 2 alpha4
            int s;
            if (SHAPE == 0) s = h2;                 // both on the B2 block
            else if (SHAPE == 3) s = h1;            // both on the B1 block
            else if (SHAPE == 1) s = h1 + 2 * h2;   // alpha3 on B1, alpha4 on B2
            else s = h2 + 2 * h1;                   // alpha4 on B1, alpha3 on B2
            cfma<T>(acc[a][b][s], v1[h1][a], v2[h2][b]);
          }
  }
}

// grid.x = channel x alpha1-group (fastest, so that every channel of a q-tile
// runs at the same time and the tile's stored blocks are reused from L2),
// grid.y = q-tile of NT consecutive momenta.  Stored blocks: FB[cell][q][alpha].
template <typename T, int A1, int NT>
__global__ void __launch_bounds__(NT) k_contract(const C<T>* __restrict__ FB, int L, const DevTerm* __restrict__ terms,
                                                 const int* __restrict__ ch_tb, const Ent<T>* __restrict__ E1,
                                                 const Ent<T>* __restrict__ E2, C<T>* __restrict__ Ft) {
  const long long V = (long long)L * L * L;
  const int q = blockIdx.y * NT + threadIdx.x;
  if (q >= V) return;
  constexpr int NG = 4 / A1;
  const int ch = blockIdx.x / NG;
  const int a0 = (blockIdx.x % NG) * A1;
  const int qx = q % L, qy = (q / L) % L, qz = q / (L * L);
  const int qm = (L - qx) % L + L * ((L - qy) % L + L * ((L - qz) % L));
  C<T> acc[A1][4][4];
#pragma unroll
  for (int a = 0; a < A1; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int s = 0; s < 4; ++s) acc[a][b][s] = czero<T>();
  const long long cs = 4 * V, qoff = 4LL * q + a0, qmoff = 4LL * qm;
  const int t1 = ch_tb[ch + 1];
  for (int t = ch_tb[ch]; t < t1; ++t) {
    DevTerm h = terms[t];
    switch (h.shape) {
      case 0: run_term<T, A1, 0>(h, FB, cs, qoff, qmoff, E1, E2, acc); break;
      case 1: run_term<T, A1, 1>(h, FB, cs, qoff, qmoff, E1, E2, acc); break;
      case 2: run_term<T, A1, 2>(h, FB, cs, qoff, qmoff, E1, E2, acc); break;
      default: run_term<T, A1, 3>(h, FB, cs, qoff, qmoff, E1, E2, acc); break;
    }
  }
  C<T>* o = Ft + (long long)ch * 64 * V + q;
#pragma unroll
  for (int a = 0; a < A1; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        // acc holds s = alpha3 + 2 alpha4; the output layout is [alpha1][alpha2][alpha3][alpha4]
        const int spin = ((a0 + a) * 4 + b) * 4 + 2 * (s & 1) + (s >> 1);
        o[(long long)spin * V] = acc[a][b][s];
      }
}

// f * 2^ex as a double, by integer operations on the bit pattern (exact): a
// normal FP32 value keeps its sign and mantissa and gets the FP64 exponent
// E - 127 + 1023 + ex; zeros stay zeros; FP32 subnormals, infinities, NaNs
// and results outside the FP64 normal range go through ldexp.
__device__ __forceinline__ double scaled_double(float f, int ex) {
  const unsigned b = __float_as_uint(f);
  const unsigned E = (b >> 23) & 255u;
  const int DE = (int)E + (1023 - 127) + ex;
  if (E - 1u < 254u && DE > 0 && DE < 2047) {
    // high word: sign, 11-bit exponent, top 20 mantissa bits; low word: last 3 mantissa bits
    const unsigned hi = (b & 0x80000000u) | ((unsigned)DE << 20) | ((b & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)(b << 29));
  }
  if ((b & 0x7fffffffu) == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
  return ldexp((double)f, ex);
}

// out[ch * ch_stride + c*V + r] = Ft[ch][c][r] * 2^(sum_f e_f n_f) / V
// FP32 input: 1/V applied in FP32, the power of two added to the exponent
// (no FP64 arithmetic, which is scarce on GB300); two complex values per
// 16-byte load and RS independent loads in flight per thread.  FP64 input:
// FP64 multiply.
template <typename T>
__global__ void __launch_bounds__(256) k_restore(const C<T>* __restrict__ Ft, long long V, const int* __restrict__ ch_fl,
                                                 const int* __restrict__ exps, int nflav, double2* __restrict__ out,
                                                 long long ch_stride, long long norm) {
  const int ch = blockIdx.y;
  int ex = 0;  // sum over the propagators of (their exponent) x (their quarks in the sink pair)
  for (int f = 0; f < nflav; ++f) ex += exps[f] * ch_fl[3 * ch + f];
  const long long n = 64 * V;
  const C<T>* src = Ft + ch * n;
  double2* dst = out + ch * ch_stride;
  const long long stride = (long long)gridDim.x * blockDim.x;
  if constexpr (sizeof(T) == 4) {
    // one complex value per lane and load: each warp store writes 512 contiguous bytes
    constexpr int RS = 4;
    const float inv = 1.0f / (float)norm;
    for (long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += RS * stride) {
      float2 z[RS];
#pragma unroll
      for (int u = 0; u < RS; ++u) {
        const long long i = i0 + u * stride;
        z[u] = i < n ? __ldcs(reinterpret_cast<const float2*>(src) + i) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < RS; ++u) {
        const long long i = i0 + u * stride;
        if (i < n) __stcs(dst + i, make_double2(scaled_double(z[u].x * inv, ex), scaled_double(z[u].y * inv, ex)));
      }
    }
  } else {
    const double scale = ldexp(1.0, ex) / (double)norm;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
      const C<T> z = src[i];
      dst[i] = make_double2((double)z.x * scale, (double)z.y * scale);
    }
  }
}

}  // namespace

template <typename T, int A1, int NT>
cudaError_t launch_contract_cfg(const C<T>* FB, int L, const DevTerm* terms, const int* ch_tb, int nch,
                                const Ent<T>* e1, const Ent<T>* e2, C<T>* Ft, cudaStream_t st) {
  const long long V = (long long)L * L * L;
  dim3 grid((unsigned)(nch * (4 / A1)), (unsigned)((V + NT - 1) / NT));
  k_contract<T, A1, NT><<<grid, NT, 0, st>>>(FB, L, terms, ch_tb, e1, e2, Ft);
  return cudaGetLastError();
}

// cfg: alpha1 values per thread (1, 2, 4) x 10 + threads per block / 32 (1, 2, 4)
template <typename T>
cudaError_t launch_contract(const C<T>* FB, int L, const DevTerm* terms, const int* ch_tb, int nch, const Ent<T>* e1,
                            const Ent<T>* e2, C<T>* Ft, int cfg, cudaStream_t st) {
  if (cfg == 0) cfg = sizeof(T) == 4 ? 42 : 21;
  if (nch * 4 > 2147483647 / 4) return cudaErrorInvalidValue;
  switch (cfg) {
#define NBS_CFG(a, w) \
  case a * 10 + w: return launch_contract_cfg<T, a, 32 * w>(FB, L, terms, ch_tb, nch, e1, e2, Ft, st);
    NBS_CFG(1, 1) NBS_CFG(1, 2) NBS_CFG(1, 4)
    NBS_CFG(2, 1) NBS_CFG(2, 2) NBS_CFG(2, 4)
    NBS_CFG(4, 1) NBS_CFG(4, 2) NBS_CFG(4, 4)
#undef NBS_CFG
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_restore(const C<T>* Ft, int V, int nch, const int* ch_fl, const int* exps, int nflav, double2* out,
                           long long ch_stride, cudaStream_t st, long long norm) {
  long long n = 64LL * V;
  if (sizeof(T) == 4) n /= 4;  // four values per thread per pass
  int bx = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 4096));
  dim3 grid(bx, nch);
  k_restore<T><<<grid, 256, 0, st>>>(Ft, (long long)V, ch_fl, exps, nflav, out, ch_stride, norm ? norm : (long long)V);
  return cudaGetLastError();
}

template cudaError_t launch_contract<float>(const float2*, int, const DevTerm*, const int*, int, const Ent<float>*,
                                            const Ent<float>*, float2*, int, cudaStream_t);
template cudaError_t launch_contract<double>(const double2*, int, const DevTerm*, const int*, int, const Ent<double>*,
                                             const Ent<double>*, double2*, int, cudaStream_t);
template cudaError_t launch_restore<float>(const float2*, int, int, const int*, const int*, int, double2*, long long,
                                           cudaStream_t, long long);
template cudaError_t launch_restore<double>(const double2*, int, int, const int*, const int*, int, double2*, long long,
                                            cudaStream_t, long long);

}  // namespace nbs
