// Four-step pencil FFTs with compile-time lengths L = L1 * L2.
//
// A length-L transform of one pencil is done as
//   step A (thread n2 < L2): v[n1] = x[L2 n1 + n2], DFT_L1 in registers,
//                            times w_L^(n2 k1), stored to shared memory;
//   step B (thread k1 < L1): the L2 values of row k1, DFT_L2 in registers,
//                            X[k1 + L1 k2] = result[k2].
// (X[k1 + L1 k2] = sum_n2 w_L2^(n2 k2) w_L^(n2 k1) sum_n1 x[L2 n1 + n2] w_L1^(n1 k1).)
// Compared with one shared-memory round trip per radix stage, a pencil makes
// two round trips and all index arithmetic inside the register DFTs is
// resolved at compile time.  These kernels serve the padded lengths in
// kFourStepLengths; other lengths use the Stockham kernels of fft.cu.
//
// fft4_strided: the z and y passes (pencil along a strided axis, TX
// consecutive x columns per block, as in fft.cu).
// fft4_x: the fused x pass: forward transform of the nx zero-padded samples
// of RY rows (ky) x TG grids per block, product with the Ghat rows (folded
// into step B of the forward transform), inverse transform, nx samples kept.
#pragma once

#include "fft_policy.h"

namespace aim {

struct StridedArgs4 {
  int n_in, n_out;  // samples read (rest zero) / samples written
  int X, A;         // contiguous extent, other-axis extent
  long long sG_in, sA_in, sP_in;
  long long sG_out, sA_out, sP_out;
};

struct XArgs4 {
  int nx, Ly, Lz, G;
  int RY, TG;      // rows and grids per block
  long long sG;    // grid stride (elements)
  int hx, hy;      // octant extents of Ghat (x, y)
};

template <class S, class O> struct OutConv4 {
  __device__ static O f(const S& s) { return s; }
};
template <> struct OutConv4<float4, double2> {
  __device__ static double2 f(const float4& s) {
    return make_double2((double)s.x + (double)s.y, (double)s.z + (double)s.w);
  }
};

// A block transforms AY consecutive other-axis indices (ia) x TX columns, so
// short pencils still give every thread work.
template <class P, bool INV, int L1, int L2, class O>
__global__ void __launch_bounds__(256) fft4_strided(const typename P::S* __restrict__ in, O* __restrict__ out,
                                                    StridedArgs4 a, const typename P::S* __restrict__ twL, int AY) {
  using S = typename P::S;
  using T = typename P::T;
  constexpr int L = L1 * L2, TX = P::kTX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S* b0 = reinterpret_cast<S*>(smem_raw);  // [AY][L][TX]
  S* b1 = b0 + AY * L * TX;
  const int x0 = blockIdx.x * TX;
  const int ia0 = blockIdx.y * AY;
  const int nay = min(AY, a.A - ia0);
  const long long g = blockIdx.z;
  const S* src = in + g * a.sG_in + (long long)ia0 * a.sA_in + x0;
  if (nay == 1) {
    for (int e = threadIdx.x; e < L * TX; e += blockDim.x) {
      const int p = e / TX, c = e % TX;
      S v = P::st(P::zero());
      if (p < a.n_in && x0 + c < a.X) v = src[p * a.sP_in + c];
      b0[e] = v;
    }
  } else {  // several short pencils per block: one flat loop keeps every thread loading
    for (int e = threadIdx.x; e < nay * L * TX; e += blockDim.x) {
      const int t = e / (L * TX), rem = e - t * (L * TX);
      const int p = rem / TX, c = rem % TX;
      S v = P::st(P::zero());
      if (p < a.n_in && x0 + c < a.X) v = src[t * a.sA_in + p * a.sP_in + c];
      b0[e] = v;
    }
  }
  __syncthreads();
  for (int u = threadIdx.x; u < nay * TX * L2; u += blockDim.x) {
    const int t = u / (TX * L2), rem = u - t * (TX * L2);
    const int c = rem % TX, n2 = rem / TX;
    const S* x = b0 + t * L * TX;
    T v[L1];
    static_for<0, L1>([&](auto n1) { v[n1] = P::ld(x[(L2 * decltype(n1)::value + n2) * TX + c]); });
    RegDFT<P, L1, INV>::run(v);
    if (n2 > 0)
      static_for<1, L1>([&](auto k1) { v[k1] = P::mul(v[k1], P::conj_if(P::ld(twL[n2 * decltype(k1)::value]), INV)); });
    S* y = b1 + t * L * TX;
    static_for<0, L1>([&](auto k1) { y[(decltype(k1)::value * L2 + n2) * TX + c] = P::st(v[k1]); });
  }
  __syncthreads();
  for (int u = threadIdx.x; u < nay * TX * L1; u += blockDim.x) {
    const int t = u / (TX * L1), rem = u - t * (TX * L1);
    const int c = rem % TX, k1 = rem / TX;
    const S* y = b1 + t * L * TX;
    T w[L2];
    static_for<0, L2>([&](auto n2) { w[n2] = P::ld(y[(k1 * L2 + decltype(n2)::value) * TX + c]); });
    RegDFT<P, L2, INV>::run(w);
    O* dst = out + g * a.sG_out + (long long)(ia0 + t) * a.sA_out + x0;
    if (x0 + c < a.X)
      static_for<0, L2>([&](auto k2) {
        const int p = k1 + L1 * decltype(k2)::value;
        if (p < a.n_out) dst[p * a.sP_out + c] = OutConv4<S, O>::f(P::st(w[k2]));
      });
  }
}

template <class P, int L1, int L2>
__global__ void __launch_bounds__(256) fft4_x(typename P::S* __restrict__ buf, XArgs4 a,
                                              const typename P::S* __restrict__ ghat,
                                              const typename P::S* __restrict__ twL) {
  using S = typename P::S;
  using T = typename P::T;
  constexpr int L = L1 * L2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int RY = a.RY, TG = a.TG;
  S* gr = reinterpret_cast<S*>(smem_raw);  // [RY][L]
  S* b0 = gr + RY * L;                      // [RY * TG][L]
  S* b1 = b0 + RY * TG * L;
  const int ky0 = blockIdx.x * RY, kz = blockIdx.y;
  const int nry = min(RY, a.Ly - ky0);
  const int iz = min(kz, a.Lz - kz);
  for (int e = threadIdx.x; e < nry * L; e += blockDim.x) {
    const int r = e / L, p = e % L;
    const int ky = ky0 + r;
    const int iy = min(ky, a.Ly - ky);
    gr[e] = ghat[((long long)iz * a.hy + iy) * a.hx + min(p, L - p)];
  }
  const long long row0 = ((long long)kz * a.Ly + ky0) * a.nx;
  for (int g0 = 0; g0 < a.G; g0 += TG) {
    const int ng = min(TG, a.G - g0);
    const int np = nry * ng;  // pencil pc = r * ng + gl
    __syncthreads();
    for (int e = threadIdx.x; e < np * L; e += blockDim.x) {
      const int pc = e / L, p = e % L;
      const int r = pc / ng, gl = pc - r * ng;
      S v = P::st(P::zero());
      if (p < a.nx) v = buf[(long long)(g0 + gl) * a.sG + row0 + (long long)r * a.nx + p];
      b0[e] = v;
    }
    __syncthreads();
    // forward, step A
    for (int u = threadIdx.x; u < np * L2; u += blockDim.x) {
      const int n2 = u % L2, pc = u / L2;
      const S* x = b0 + pc * L;
      T v[L1];
      static_for<0, L1>([&](auto n1) { v[n1] = P::ld(x[L2 * decltype(n1)::value + n2]); });
      RegDFT<P, L1, false>::run(v);
      if (n2 > 0) static_for<1, L1>([&](auto k1) { v[k1] = P::mul(v[k1], P::ld(twL[n2 * decltype(k1)::value])); });
      S* y = b1 + pc * L;
      static_for<0, L1>([&](auto k1) { y[decltype(k1)::value * L2 + n2] = P::st(v[k1]); });
    }
    __syncthreads();
    // forward, step B, times Ghat -> b0 in natural order
    for (int u = threadIdx.x; u < np * L1; u += blockDim.x) {
      const int k1 = u % L1, pc = u / L1;
      const int r = pc / ng;
      const S* y = b1 + pc * L;
      T w[L2];
      static_for<0, L2>([&](auto n2) { w[n2] = P::ld(y[k1 * L2 + decltype(n2)::value]); });
      RegDFT<P, L2, false>::run(w);
      S* x = b0 + pc * L;
      const S* gg = gr + r * L;
      static_for<0, L2>([&](auto k2) {
        const int p = k1 + L1 * decltype(k2)::value;
        x[p] = P::st(P::mul(w[k2], P::ld(gg[p])));
      });
    }
    __syncthreads();
    // inverse, step A
    for (int u = threadIdx.x; u < np * L2; u += blockDim.x) {
      const int n2 = u % L2, pc = u / L2;
      const S* x = b0 + pc * L;
      T v[L1];
      static_for<0, L1>([&](auto n1) { v[n1] = P::ld(x[L2 * decltype(n1)::value + n2]); });
      RegDFT<P, L1, true>::run(v);
      if (n2 > 0)
        static_for<1, L1>([&](auto k1) { v[k1] = P::mul(v[k1], P::conj_if(P::ld(twL[n2 * decltype(k1)::value]), true)); });
      S* y = b1 + pc * L;
      static_for<0, L1>([&](auto k1) { y[decltype(k1)::value * L2 + n2] = P::st(v[k1]); });
    }
    __syncthreads();
    // inverse, step B -> global (first nx samples)
    for (int u = threadIdx.x; u < np * L1; u += blockDim.x) {
      const int k1 = u % L1, pc = u / L1;
      const int r = pc / ng, gl = pc - r * ng;
      const S* y = b1 + pc * L;
      T w[L2];
      static_for<0, L2>([&](auto n2) { w[n2] = P::ld(y[k1 * L2 + decltype(n2)::value]); });
      RegDFT<P, L2, true>::run(w);
      S* dst = buf + (long long)(g0 + gl) * a.sG + row0 + (long long)r * a.nx;
      static_for<0, L2>([&](auto k2) {
        const int p = k1 + L1 * decltype(k2)::value;
        if (p < a.nx) dst[p] = P::st(w[k2]);
      });
    }
  }
}

// Padded lengths with a four-step kernel, as (L, L1, L2).
#define AIM_FOURSTEP_LENGTHS(X) \
  X(5, 5, 1)                    \
  X(24, 4, 6)                   \
  X(25, 5, 5)                   \
  X(45, 5, 9)                   \
  X(81, 9, 9)                   \
  X(90, 9, 10)                  \
  X(162, 9, 18)                 \
  X(180, 12, 15)                \
  X(324, 18, 18)                \
  X(360, 18, 20)                \
  X(648, 24, 27)

}  // namespace aim
