// Four-step pencil FFTs with compile-time lengths L = L1 * L2.
//
// A length-L transform of one pencil is done as
//   step A (thread n2 < L2): v[n1] = x[L2 n1 + n2], DFT_L1 in registers,
//                            times w_L^(n2 k1), stored to shared memory;
//   step B (thread k1 < L1): the L2 values of row k1, DFT_L2 in registers,
//                            X[k1 + L1 k2] = result[k2].
// (X[k1 + L1 k2] = sum_n2 w_L2^(n2 k2) w_L^(n2 k1) sum_n1 x[L2 n1 + n2] w_L1^(n1 k1).)
// Compared with one shared-memory round trip per radix stage, a pencil makes
// one round trip (two for the fused forward-product-inverse x pass) and all
// index arithmetic inside the register DFTs is resolved at compile time.  These kernels serve the padded lengths in
// kFourStepLengths; other lengths use the Stockham kernels of fft.cu.
//
// Twiddles: twL holds w_L^t for t < L (the Stockham kernels' table), then
// the same factors w_L^(k1 n2) laid out twice for the four-step kernels: as
// [k1][n2] at twL + L (step A: the lanes of a warp take consecutive n2) and
// as [n2][k1] at twL + 2L (the x pass's step B: consecutive k1), so each
// warp-wide twiddle load touches one or two cache lines instead of one line
// per lane.
//
// fft4_strided: the z and y passes (pencil along a strided axis, TX
// consecutive x columns per block, as in fft.cu).
// fft4_x: the fused x pass: forward transform of the nx zero-padded samples
// of RY rows (ky) x TG grids per block, product with the Ghat rows and the
// inverse transform, nx samples kept.
#pragma once

#include "fft_policy.h"

namespace aim {

struct StridedArgs4 {
  int n_in, n_out;  // samples read (rest zero) / samples written
  int X, A;         // contiguous extent, other-axis extent
  long long sG_in, sA_in, sP_in;
  long long sG_out, sA_out, sP_out;
  // optional [A][X] flags of the pencils that matter (z passes of a 3-D grid:
  // the (x, y) columns that hold a stencil node): the others read no input
  // (it is zero) and, in an inverse pass, write no output (nothing reads it)
  const uint8_t* cols = nullptr;
};

struct XArgs4 {
  int nx, Ly, Lz, G;
  int RY, TG;      // rows and grids per block (fft4_x); fft4_x_groups: all G grids of RY rows
  int GT, PPG;     // fft4_x_groups: threads per pencil group (a multiple of 32), pencils per group at a time
  long long sG;    // grid stride (elements)
  int hx, hy;      // octant extents of Ghat (x, y)
};

// Barrier of one pencil group: __syncthreads when the group is the whole
// block, the warp itself when it is one warp, else the named barrier
// 1 + grp over the group's GT threads.  Also orders the group's
// shared-memory accesses.
__device__ __forceinline__ void group_sync(int grp, int GT) {
  if (GT == (int)blockDim.x)
    __syncthreads();
  else if (GT == 32)
    __syncwarp();
  else
    asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(GT) : "memory");
}

template <class S, class O> struct OutConv4 {
  __device__ static O f(const S& s) { return s; }
};

// Columns per block of the strided kernels for length L: the policy's
// preferred width, halved while one pencil set would need more than 48 KB of
// shared memory (so long pencils still leave several blocks per SM).  The
// wide variant starts from twice that width with a 96 KB limit: longer
// contiguous runs per pencil row, fewer blocks per SM.
template <class P, int L, bool WIDE = false> constexpr int strided_tx() {
  int tx = WIDE ? 2 * P::kTX : P::kTX;
  const long long cap = (WIDE ? 96 : 48) * 1024;
  while (tx > 4 && (long long)L * tx * (long long)sizeof(typename P::S) > cap) tx /= 2;
  return tx;
}

// Shared-memory row length: odd, so lanes that walk a strided row hit
// distinct banks.
constexpr int odd_row(int n) { return n + (n % 2 == 0 ? 1 : 0); }

// A block transforms AY consecutive other-axis indices (ia) x TX columns, so
// short pencils still give every thread work.  Step A loads its L1 samples
// straight from global memory into registers (samples >= n_in are zero and
// never read); the only shared-memory round trip is the transpose between
// the two steps.  Step B writes the first n_out outputs.
template <class P, bool INV, int L1, int L2, class O, bool WIDE>
__device__ __forceinline__ void strided_body(const typename P::S* __restrict__ in, O* __restrict__ out,
                                             const StridedArgs4 a, const typename P::S* __restrict__ twL, int AY) {
  using S = typename P::S;
  using T = typename P::T;
  constexpr int L = L1 * L2, TX = strided_tx<P, L, WIDE>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S* b = reinterpret_cast<S*>(smem_raw);  // [AY][L1][L2][TX]
  const int x0 = blockIdx.x * TX;
  const int ia0 = blockIdx.y * AY;
  const int nay = min(AY, a.A - ia0);
  const long long g = blockIdx.z;
  for (int u = threadIdx.x; u < nay * TX * L2; u += blockDim.x) {
    const int t = u / (TX * L2), rem = u - t * (TX * L2);
    const int c = rem % TX, n2 = rem / TX;
    const bool col = x0 + c < a.X && (!a.cols || a.cols[(long long)(ia0 + t) * a.X + x0 + c]);
    const S* src = in + g * a.sG_in + (long long)(ia0 + t) * a.sA_in + x0 + c;
    T v[L1];
    static_for<0, L1>([&](auto n1) {
      const int p = L2 * decltype(n1)::value + n2;
      v[n1] = (col && p < a.n_in) ? P::ld(src[(long long)p * a.sP_in]) : P::zero();
    });
    RegDFT<P, L1, INV>::run(v);
    if (n2 > 0)
      static_for<1, L1>([&](auto k1) { v[k1] = P::mul(v[k1], P::conj_if(P::ld(twL[L + decltype(k1)::value * L2 + n2]), INV)); });
    S* y = b + t * L * TX;
    static_for<0, L1>([&](auto k1) { y[(decltype(k1)::value * L2 + n2) * TX + c] = P::st(v[k1]); });
  }
  __syncthreads();
  for (int u = threadIdx.x; u < nay * TX * L1; u += blockDim.x) {
    const int t = u / (TX * L1), rem = u - t * (TX * L1);
    const int c = rem % TX, k1 = rem / TX;
    const S* y = b + t * L * TX;
    T w[L2];
    static_for<0, L2>([&](auto n2) { w[n2] = P::ld(y[(k1 * L2 + decltype(n2)::value) * TX + c]); });
    RegDFT<P, L2, INV>::run(w);
    O* dst = out + g * a.sG_out + (long long)(ia0 + t) * a.sA_out + x0 + c;
    if (x0 + c < a.X && (!INV || !a.cols || a.cols[(long long)(ia0 + t) * a.X + x0 + c]))
      static_for<0, L2>([&](auto k2) {
        const int p = k1 + L1 * decltype(k2)::value;
        if (p < a.n_out) dst[(long long)p * a.sP_out] = OutConv4<S, O>::f(P::st(w[k2]));
      });
  }
}

template <class P, bool INV, int L1, int L2, class O, bool WIDE = false>
__global__ void __launch_bounds__(256) fft4_strided(const typename P::S* __restrict__ in, O* __restrict__ out,
                                                    StridedArgs4 a, const typename P::S* __restrict__ twL, int AY) {
  strided_body<P, INV, L1, L2, O, WIDE>(in, out, a, twL, AY);
}
// The same with four resident 256-thread blocks per SM required of the
// register allocation: used for the complex64 length-648 pencils, which
// otherwise take about 74 registers (the few values spilled at 64 cost less
// than the lost warps).
template <class P, bool INV, int L1, int L2, class O, bool WIDE = false>
__global__ void __launch_bounds__(256, 4) fft4_strided_occ4(const typename P::S* __restrict__ in, O* __restrict__ out,
                                                            StridedArgs4 a, const typename P::S* __restrict__ twL,
                                                            int AY) {
  strided_body<P, INV, L1, L2, O, WIDE>(in, out, a, twL, AY);
}
template <class P, int L> constexpr bool strided_occ4() { return sizeof(typename P::S) <= 8 && L == 648; }

// The fused x pass.  With k = k1 + L1 k2 and n = n2 + L2 n1,
//   forward  X[k1 + L1 k2] = sum_n2 w_L2^(n2 k2) w_L^(n2 k1) sum_n1 x[L2 n1 + n2] w_L1^(n1 k1),
//   inverse  y[n2 + L2 n1] = sum_k1 w_L1^(-k1 n1) w_L^(-k1 n2) sum_k2 X[k1 + L1 k2] w_L2^(-k2 n2).
// The thread that finishes the forward transform for one k1 holds X[k1 + L1 k2]
// for every k2, which is exactly the input of the inverse's first step, so it
// multiplies by Ghat and starts the inverse in registers:
//   step A (thread n2, from global):   DFT_L1, twiddle, into row k1 column n2 of the tile;
//   step B (thread k1):                row k1: DFT_L2, x Ghat, inverse DFT_L2, twiddle,
//                                      written back over the same row;
//   step C (thread n2, to global):     column n2: inverse DFT_L1, samples < nx written.
// One [L1][odd L2] tile per pencil, two shared-memory round trips.  The block
// handles RY rows (ky) x TG grids at a time with at most one work item per
// thread in each step (the launcher sizes RY * TG * max(L1, L2) <= blockDim)
// and keeps the RY rows of Ghat in shared memory.
// Resident 256-thread blocks per SM the register allocation must allow: four
// for complex64 (three for the longest compiled length, 648, which would
// spill at four; two above it), two for the 16-byte policies (one above 648).
template <class P, int L> constexpr int x_min_blocks() {
  return sizeof(typename P::S) <= 8 ? (L > 648 ? 2 : L == 648 ? 3 : 4) : (L > 648 ? 1 : 2);
}

template <class P, int L1, int L2>
__global__ void __launch_bounds__(256, x_min_blocks<P, L1 * L2>()) fft4_x(typename P::S* __restrict__ buf, XArgs4 a,
                                              const typename P::S* __restrict__ ghat,
                                              const typename P::S* __restrict__ twL) {
  using S = typename P::S;
  using T = typename P::T;
  constexpr int L = L1 * L2;
  constexpr int RA = odd_row(L2);
  constexpr int PA = L1 * RA;  // per-pencil tile
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int RY = a.RY, TG = a.TG;
  S* gr = reinterpret_cast<S*>(smem_raw);  // [RY][L]
  S* tile = gr + RY * L;                    // [RY * TG][L1][RA]
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
  const int u = threadIdx.x;
  for (int g0 = 0; g0 < a.G; g0 += TG) {
    const int ng = min(TG, a.G - g0);
    const int np = nry * ng;  // pencil pc = r * ng + gl
    if (g0 > 0) __syncthreads();  // the previous group's step C has read its tiles
    // step A: forward DFT_L1 of the zero-padded row, straight from global memory
    if (u < np * L2) {
      const int n2 = u % L2, pc = u / L2;
      const int r = pc / ng, gl = pc - r * ng;
      const S* src = buf + (long long)(g0 + gl) * a.sG + row0 + (long long)r * a.nx;
      T v[L1];
      static_for<0, L1>([&](auto n1) {
        const int p = L2 * decltype(n1)::value + n2;
        v[n1] = p < a.nx ? P::ld(src[p]) : P::zero();
      });
      RegDFT<P, L1, false>::run(v);
      if (n2 > 0) static_for<1, L1>([&](auto k1) { v[k1] = P::mul(v[k1], P::ld(twL[L + decltype(k1)::value * L2 + n2])); });
      S* y = tile + pc * PA + n2;
      static_for<0, L1>([&](auto k1) { y[decltype(k1)::value * RA] = P::st(v[k1]); });
    }
    __syncthreads();  // also orders Ghat's staging before the first step B
    // step B: forward DFT_L2, product with Ghat, inverse DFT_L2, over one row
    if (u < np * L1) {
      const int k1 = u % L1, pc = u / L1;
      const int r = pc / ng;
      S* y = tile + pc * PA + k1 * RA;
      T w[L2];
      static_for<0, L2>([&](auto n2) { w[n2] = P::ld(y[decltype(n2)::value]); });
      RegDFT<P, L2, false>::run(w);
      const S* gg = gr + r * L + k1;
      static_for<0, L2>([&](auto k2) { w[k2] = P::mul(w[k2], P::ld(gg[L1 * decltype(k2)::value])); });
      RegDFT<P, L2, true>::run(w);
      if (k1 > 0)
        static_for<1, L2>([&](auto n2) { w[n2] = P::mul(w[n2], P::conj_if(P::ld(twL[2 * L + decltype(n2)::value * L1 + k1]), true)); });
      static_for<0, L2>([&](auto n2) { y[decltype(n2)::value] = P::st(w[n2]); });
    }
    __syncthreads();
    // step C: inverse DFT_L1 over one column, the first nx samples back to global memory
    if (u < np * L2) {
      const int n2 = u % L2, pc = u / L2;
      const int r = pc / ng, gl = pc - r * ng;
      const S* z = tile + pc * PA + n2;
      T v[L1];
      static_for<0, L1>([&](auto k1) { v[k1] = P::ld(z[decltype(k1)::value * RA]); });
      RegDFT<P, L1, true>::run(v);
      S* dst = buf + (long long)(g0 + gl) * a.sG + row0 + (long long)r * a.nx;
      static_for<0, L1>([&](auto n1) {
        const int p = n2 + L2 * decltype(n1)::value;
        if (p < a.nx) dst[p] = P::st(v[n1]);
      });
    }
  }
}

// The fused x pass in pencil groups: the same three steps and tiles as
// fft4_x, but the block's threads form groups of GT (one or more warps).  A
// group takes PPG pencils at a time (PPG * max(L1, L2) <= GT) through the
// three steps with its own tiles, and only the group's own barrier separates
// the steps, so groups in different steps overlap instead of waiting for the
// whole block.  A block owns RY rows (ky) x all G grids.
template <class P, int L1, int L2>
__global__ void __launch_bounds__(256, x_min_blocks<P, L1 * L2>()) fft4_x_groups(typename P::S* __restrict__ buf, XArgs4 a,
                                                     const typename P::S* __restrict__ ghat,
                                                     const typename P::S* __restrict__ twL) {
  using S = typename P::S;
  using T = typename P::T;
  constexpr int L = L1 * L2;
  constexpr int RA = odd_row(L2);
  constexpr int PA = L1 * RA;  // per-pencil tile
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int RY = a.RY, GT = a.GT, PPG = a.PPG;
  const int grp = threadIdx.x / GT, u = threadIdx.x - grp * GT;
  const int ngroups = blockDim.x / GT;
  S* gr = reinterpret_cast<S*>(smem_raw);     // [RY][L]
  S* tile = gr + RY * L + grp * PPG * PA;      // this group's [PPG][L1][RA]
  const int ky0 = blockIdx.x * RY, kz = blockIdx.y;
  const int nry = min(RY, a.Ly - ky0);
  const int iz = min(kz, a.Lz - kz);
  for (int e = threadIdx.x; e < nry * L; e += blockDim.x) {
    const int r = e / L, p = e % L;
    const int ky = ky0 + r;
    const int iy = min(ky, a.Ly - ky);
    gr[e] = ghat[((long long)iz * a.hy + iy) * a.hx + min(p, L - p)];
  }
  // Ghat rows staged: a block-wide group's first barrier (after step A)
  // orders them before step B; smaller groups need a barrier of their own
  if (GT != (int)blockDim.x) __syncthreads();
  const long long row0 = ((long long)kz * a.Ly + ky0) * a.nx;
  const int npen = nry * a.G;  // pencil q: row q / G, grid q % G
  // q0 is the same for every thread of a group, so the group meets its barriers together
  for (int q0 = grp * PPG; q0 < npen; q0 += ngroups * PPG) {
    if (q0 != grp * PPG) group_sync(grp, GT);  // the previous step C has read the tiles
    // step A: forward DFT_L1 of the zero-padded row, straight from global memory
    if (u < PPG * L2) {
      const int n2 = u % L2, lp = u / L2, q = q0 + lp;
      if (q < npen) {
        const int r = q / a.G, gl = q - r * a.G;
        const S* src = buf + (long long)gl * a.sG + row0 + (long long)r * a.nx;
        T v[L1];
        static_for<0, L1>([&](auto n1) {
          const int p = L2 * decltype(n1)::value + n2;
          v[n1] = p < a.nx ? P::ld(src[p]) : P::zero();
        });
        RegDFT<P, L1, false>::run(v);
        if (n2 > 0) static_for<1, L1>([&](auto k1) { v[k1] = P::mul(v[k1], P::ld(twL[L + decltype(k1)::value * L2 + n2])); });
        S* y = tile + lp * PA + n2;
        static_for<0, L1>([&](auto k1) { y[decltype(k1)::value * RA] = P::st(v[k1]); });
      }
    }
    group_sync(grp, GT);
    // step B: forward DFT_L2, product with Ghat, inverse DFT_L2, over one row
    if (u < PPG * L1) {
      const int k1 = u % L1, lp = u / L1, q = q0 + lp;
      if (q < npen) {
        const int r = q / a.G;
        S* y = tile + lp * PA + k1 * RA;
        T w[L2];
        static_for<0, L2>([&](auto n2) { w[n2] = P::ld(y[decltype(n2)::value]); });
        RegDFT<P, L2, false>::run(w);
        const S* gg = gr + r * L + k1;
        static_for<0, L2>([&](auto k2) { w[k2] = P::mul(w[k2], P::ld(gg[L1 * decltype(k2)::value])); });
        RegDFT<P, L2, true>::run(w);
        if (k1 > 0)
          static_for<1, L2>([&](auto n2) { w[n2] = P::mul(w[n2], P::conj_if(P::ld(twL[2 * L + decltype(n2)::value * L1 + k1]), true)); });
        static_for<0, L2>([&](auto n2) { y[decltype(n2)::value] = P::st(w[n2]); });
      }
    }
    group_sync(grp, GT);
    // step C: inverse DFT_L1 over one column, the first nx samples back to global memory
    if (u < PPG * L2) {
      const int n2 = u % L2, lp = u / L2, q = q0 + lp;
      if (q < npen) {
        const int r = q / a.G, gl = q - r * a.G;
        const S* z = tile + lp * PA + n2;
        T v[L1];
        static_for<0, L1>([&](auto k1) { v[k1] = P::ld(z[decltype(k1)::value * RA]); });
        RegDFT<P, L1, true>::run(v);
        S* dst = buf + (long long)gl * a.sG + row0 + (long long)r * a.nx;
        static_for<0, L1>([&](auto n1) {
          const int p = n2 + L2 * decltype(n1)::value;
          if (p < a.nx) dst[p] = P::st(v[n1]);
        });
      }
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
  X(648, 24, 27)                \
  X(1296, 36, 36)

}  // namespace aim
