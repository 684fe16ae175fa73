// Complex arithmetic policies of the FFT kernels and compile-time register
// DFTs.
//
// Policies: P32 complex64 (float2), P64 complex128 (double2), PFF complex
// float-float (float4 = re.hi, re.lo, im.hi, im.lo; about 48 bits on the FP32
// pipes, see ff.h).  Every butterfly is written once over a policy.
//
// RegDFT<P, N, INV>::run(v) transforms N values held in registers (natural
// order in and out) by recursive decimation in time, N = R * M:
//   X[k2 + M q] = sum_j w_N^(j k2) E_j[k2] w_R^(j q),  E_j = DFT_M(x[R i + j]),
// with every index and every twiddle known at compile time.  The twiddle
// constants w_N^e = cos(2 pi e / N) - i sin(2 pi e / N) are evaluated by
// constexpr Taylor series (after an exact octant reduction of e / N), so no
// table is read and the float-float policy gets both halves of each constant
// folded into the instruction stream.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>
#include <utility>

#include "common.h"
#include "ff.h"

namespace aim {

// ------------------------------------------------------------------ compile-time trigonometry
constexpr double kTwoPi = 6.283185307179586476925286766559;

// Taylor series for |x| <= pi/4 (the 16-term truncation error is far below 1e-20).
constexpr double cx_sin_small(double x) {
  double term = x, sum = x;
  for (int n = 1; n < 16; ++n) {
    term *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
    sum += term;
  }
  return sum;
}
constexpr double cx_cos_small(double x) {
  double term = 1.0, sum = 1.0;
  for (int n = 1; n < 16; ++n) {
    term *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
    sum += term;
  }
  return sum;
}
// cos and sin of 2 pi e / N for integers e, N > 0: reduce e / N to the first
// octant exactly in integer arithmetic (8 e mod 8 N), then use the series.
struct CS {
  double c, s;
};
constexpr CS cx_cossin_2pi(long e, long N) {
  e %= N;
  if (e < 0) e += N;
  const long e8 = 8 * e;       // angle in units of (2 pi / 8N) ... octant index = e8 / N
  const long oct = e8 / N;     // 0..7
  const long rem = e8 - oct * N;  // 0 <= rem < N, angle within the octant = (pi/4) rem / N
  double a = (kTwoPi / 8.0) * (double)rem / (double)N;
  // octants: angle = oct * pi/4 + a
  double c0 = cx_cos_small(a), s0 = cx_sin_small(a);
  double b = (kTwoPi / 8.0) - a;  // for odd octants use the complement for accuracy
  double c1 = cx_cos_small(b), s1 = cx_sin_small(b);
  switch (oct) {
    case 0: return CS{c0, s0};
    case 1: return CS{s1, c1};
    case 2: return CS{-s0, c0};
    case 3: return CS{-c1, s1};
    case 4: return CS{-c0, -s0};
    case 5: return CS{-s1, -c1};
    case 6: return CS{s0, -c0};
    default: return CS{c1, -s1};
  }
}

template <int B, int E, class F> AIM_HD __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// ------------------------------------------------------------------ policies
struct P32 {
  using S = float2;  // storage
  using T = float2;  // work
  static constexpr int kTX = 16;
  AIM_HD static T ld(const S& s) { return s; }
  AIM_HD static S st(const T& t) { return t; }
  AIM_HD static T zero() { return make_float2(0.f, 0.f); }
  AIM_HD static T add(T a, T b) { return make_float2(a.x + b.x, a.y + b.y); }
  AIM_HD static T sub(T a, T b) { return make_float2(a.x - b.x, a.y - b.y); }
  AIM_HD static T neg(T a) { return make_float2(-a.x, -a.y); }
  AIM_HD static T mul(T a, T b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
  AIM_HD static T mulr(T a, double, float c, float) { return make_float2(a.x * c, a.y * c); }
  // a * (c + i s) for compile-time constants
  AIM_HD static T mulc(T a, double, float c, float, double, float s, float) {
    return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
  }
  AIM_HD static T half(T a) { return make_float2(0.5f * a.x, 0.5f * a.y); }
  template <bool INV> AIM_HD static T mul_mi(T a) { return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x); }
  // m + sg * mul_mi(c d) with one fused multiply-add per component (sg = +-1)
  template <bool INV, int SG> AIM_HD static T add_mi_scaled(T m, T d, double, float c, float) {
    const float cs = SG * (INV ? -c : c);
    return make_float2(fmaf(cs, d.y, m.x), fmaf(-cs, d.x, m.y));
  }
  AIM_HD static T conj_if(T w, bool c) { return c ? make_float2(w.x, -w.y) : w; }
};

struct P64 {
  using S = double2;
  using T = double2;
  static constexpr int kTX = 8;
  AIM_HD static T ld(const S& s) { return s; }
  AIM_HD static S st(const T& t) { return t; }
  AIM_HD static T zero() { return make_double2(0.0, 0.0); }
  AIM_HD static T add(T a, T b) { return make_double2(a.x + b.x, a.y + b.y); }
  AIM_HD static T sub(T a, T b) { return make_double2(a.x - b.x, a.y - b.y); }
  AIM_HD static T neg(T a) { return make_double2(-a.x, -a.y); }
  AIM_HD static T mul(T a, T b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
  AIM_HD static T mulr(T a, double c, float, float) { return make_double2(a.x * c, a.y * c); }
  AIM_HD static T mulc(T a, double c, float, float, double s, float, float) {
    return make_double2(a.x * c - a.y * s, a.x * s + a.y * c);
  }
  AIM_HD static T half(T a) { return make_double2(0.5 * a.x, 0.5 * a.y); }
  template <bool INV> AIM_HD static T mul_mi(T a) { return INV ? make_double2(-a.y, a.x) : make_double2(a.y, -a.x); }
  template <bool INV, int SG> AIM_HD static T add_mi_scaled(T m, T d, double c, float, float) {
    const double cs = SG * (INV ? -c : c);
    return make_double2(fma(cs, d.y, m.x), fma(-cs, d.x, m.y));
  }
  AIM_HD static T conj_if(T w, bool c) { return c ? make_double2(w.x, -w.y) : w; }
};

struct PFF {
  using S = float4;
  using T = cff;
  static constexpr int kTX = 8;
  __device__ static T ld(const S& s) { return cff{ff{s.x, s.y}, ff{s.z, s.w}}; }
  __device__ static S st(const T& t) { return make_float4(t.re.hi, t.re.lo, t.im.hi, t.im.lo); }
  __device__ static T zero() { return cff{ff{0.f, 0.f}, ff{0.f, 0.f}}; }
  __device__ static T add(T a, T b) { return cff{ff_add_lazy(a.re, b.re), ff_add_lazy(a.im, b.im)}; }
  __device__ static T sub(T a, T b) { return cff{ff_sub_lazy(a.re, b.re), ff_sub_lazy(a.im, b.im)}; }
  __device__ static T neg(T a) { return cff{ff_neg(a.re), ff_neg(a.im)}; }
  __device__ static T mul(T a, T b) {
    return cff{ff_dot2(a.re, b.re, ff_neg(a.im), b.im), ff_dot2(a.re, b.im, a.im, b.re)};
  }
  __device__ static T mulr(T a, double, float ch, float cl) {
    const ff c{ch, cl};
    return cff{ff_mul(a.re, c), ff_mul(a.im, c)};
  }
  __device__ static T mulc(T a, double, float ch, float cl, double, float sh, float sl) {
    const ff c{ch, cl}, s{sh, sl};
    return cff{ff_dot2(a.re, c, ff_neg(a.im), s), ff_dot2(a.re, s, a.im, c)};
  }
  __device__ static T half(T a) { return cff{ff{0.5f * a.re.hi, 0.5f * a.re.lo}, ff{0.5f * a.im.hi, 0.5f * a.im.lo}}; }
  template <bool INV> __device__ static T mul_mi(T a) { return INV ? cff{ff_neg(a.im), a.re} : cff{a.im, ff_neg(a.re)}; }
  template <bool INV, int SG> __device__ static T add_mi_scaled(T m, T d, double c, float ch, float cl) {
    const T t = mul_mi<INV>(mulr(d, c, ch, cl));
    return SG > 0 ? add(m, t) : sub(m, t);
  }
  __device__ static T conj_if(T w, bool c) { return c ? cff{w.re, ff_neg(w.im)} : w; }
};

// Real constants as (double value, float hi, float lo).
#define AIM_RC(c) (c), (float)(c), (float)((c) - (double)(float)(c))

// ------------------------------------------------------------------ small butterflies
template <class P, bool INV> AIM_HD __forceinline__ void dft2(typename P::T* v) {
  const typename P::T a = v[0], b = v[1];
  v[0] = P::add(a, b);
  v[1] = P::sub(a, b);
}
template <class P, bool INV> AIM_HD __forceinline__ void dft3(typename P::T* v) {
  using T = typename P::T;
  const T a = v[0], s = P::add(v[1], v[2]), d = P::sub(v[1], v[2]);
  const T m = P::sub(a, P::half(s));
  // v1, v2 = m +- (-i) sin(2 pi / 3) d (forward; +i inverse), each a fused multiply-add
  v[0] = P::add(a, s);
  v[1] = P::template add_mi_scaled<INV, 1>(m, d, AIM_RC(0.86602540378443864676));
  v[2] = P::template add_mi_scaled<INV, -1>(m, d, AIM_RC(0.86602540378443864676));
}
template <class P, bool INV> AIM_HD __forceinline__ void dft4(typename P::T* v) {
  using T = typename P::T;
  const T s02 = P::add(v[0], v[2]), d02 = P::sub(v[0], v[2]);
  const T s13 = P::add(v[1], v[3]), d13 = P::template mul_mi<INV>(P::sub(v[1], v[3]));
  v[0] = P::add(s02, s13);
  v[2] = P::sub(s02, s13);
  v[1] = P::add(d02, d13);
  v[3] = P::sub(d02, d13);
}
template <class P, bool INV> AIM_HD __forceinline__ void dft5(typename P::T* v) {
  using T = typename P::T;
  const T a0 = v[0];
  const T t1 = P::add(v[1], v[4]), t2 = P::add(v[2], v[3]);
  const T t3 = P::sub(v[1], v[4]), t4 = P::sub(v[2], v[3]);
  // cos(2pi/5), cos(4pi/5), sin(2pi/5), sin(4pi/5)
  const T b1 = P::add(a0, P::add(P::mulr(t1, AIM_RC(0.30901699437494742410)), P::mulr(t2, AIM_RC(-0.80901699437494742410))));
  const T b2 = P::add(a0, P::add(P::mulr(t1, AIM_RC(-0.80901699437494742410)), P::mulr(t2, AIM_RC(0.30901699437494742410))));
  const T u1 = P::add(P::mulr(t3, AIM_RC(0.95105651629515357212)), P::mulr(t4, AIM_RC(0.58778525229247312917)));
  const T u2 = P::sub(P::mulr(t3, AIM_RC(0.58778525229247312917)), P::mulr(t4, AIM_RC(0.95105651629515357212)));
  const T e1 = P::template mul_mi<INV>(u1), e2 = P::template mul_mi<INV>(u2);
  v[0] = P::add(a0, P::add(t1, t2));
  v[1] = P::add(b1, e1);
  v[4] = P::sub(b1, e1);
  v[2] = P::add(b2, e2);
  v[3] = P::sub(b2, e2);
}

// ------------------------------------------------------------------ register DFT
constexpr int first_factor(int n) {
  return (n % 4 == 0) ? 4 : (n % 3 == 0) ? 3 : (n % 5 == 0) ? 5 : (n % 2 == 0) ? 2 : n;
}
constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }
// A radix R in {4, 3, 5, 2} with N = R M and gcd(R, M) = 1 (a prime-factor
// split, which needs no twiddle factors), or 0 when N has none.
constexpr int coprime_factor(int n) {
  const int rs[4] = {4, 3, 5, 2};
  for (int i = 0; i < 4; ++i)
    if (n % rs[i] == 0 && n / rs[i] > 1 && gcd_c(rs[i], n / rs[i]) == 1) return rs[i];
  return 0;
}
// a^-1 mod m for gcd(a, m) = 1
constexpr int inv_mod(int a, int m) {
  for (int x = 1; x < m; ++x)
    if ((a * x) % m == 1) return x;
  return m == 1 ? 0 : -1;
}

// x * w_N^E (forward) or x * conj(w_N^E) (inverse), E compile-time
template <class P, int N, int E, bool INV> AIM_HD __forceinline__ typename P::T twiddle_c(typename P::T x) {
  constexpr int e = E % N;
  if constexpr (e == 0) {
    return x;
  } else if constexpr (2 * e == N) {
    return P::neg(x);
  } else if constexpr (4 * e == N) {
    return P::template mul_mi<INV>(x);  // w^(N/4) = -i
  } else if constexpr (4 * e == 3 * N) {
    return P::template mul_mi<!INV>(x);  // w^(3N/4) = +i
  } else {
    constexpr CS cs = cx_cossin_2pi(e, N);
    constexpr double c = cs.c;
    constexpr double s = INV ? cs.s : -cs.s;  // forward: exp(-i theta)
    return P::mulc(x, c, (float)c, (float)(c - (double)(float)c), s, (float)s, (float)(s - (double)(float)s));
  }
}

template <class P, int N, bool INV> struct RegDFT {
  using T = typename P::T;
  AIM_HD __forceinline__ static void run(T* v) {
    if constexpr (N == 1) {
    } else if constexpr (N == 2) {
      dft2<P, INV>(v);
    } else if constexpr (N == 3) {
      dft3<P, INV>(v);
    } else if constexpr (N == 4) {
      dft4<P, INV>(v);
    } else if constexpr (N == 5) {
      dft5<P, INV>(v);
    } else if constexpr (coprime_factor(N) != 0) {
      // Good-Thomas prime-factor split N = R M, gcd(R, M) = 1: input index
      // n = (M j + R i) mod N, output index k = (M a k1 + R b k2) mod N with
      // a = M^-1 mod R, b = R^-1 mod M; the two DFT stages need no twiddles.
      constexpr int R = coprime_factor(N);
      constexpr int M = N / R;
      constexpr int A = inv_mod(M % R, R), B = inv_mod(R % M, M);
      T sub[R][M];
      static_for<0, R>([&](auto j) {
        static_for<0, M>([&](auto i) { sub[j][i] = v[(M * decltype(j)::value + R * decltype(i)::value) % N]; });
        RegDFT<P, M, INV>::run(sub[j]);
      });
      static_for<0, M>([&](auto k2) {
        T t[R];
        static_for<0, R>([&](auto j) { t[j] = sub[j][k2]; });
        RegDFT<P, R, INV>::run(t);
        static_for<0, R>([&](auto k1) {
          v[(M * A * decltype(k1)::value + R * B * decltype(k2)::value) % N] = t[k1];
        });
      });
    } else {
      constexpr int R = first_factor(N);
      constexpr int M = N / R;
      static_assert(R * M == N && R > 1 && R <= 5, "register DFT length must be 2,3,5-smooth");
      T sub[R][M];
      static_for<0, R>([&](auto j) {
        static_for<0, M>([&](auto i) { sub[j][i] = v[R * i + j]; });
        RegDFT<P, M, INV>::run(sub[j]);
      });
      static_for<0, M>([&](auto k2) {
        T t[R];
        static_for<0, R>([&](auto j) {
          t[j] = twiddle_c<P, N, decltype(j)::value * decltype(k2)::value, INV>(sub[j][k2]);
        });
        RegDFT<P, R, INV>::run(t);
        static_for<0, R>([&](auto q) { v[k2 + M * q] = t[q]; });
      });
    }
  }
};

}  // namespace aim
