// Pruned mixed-radix Stockham FFT convolution on the zero-padded AIM grid.
//
// Paper Section 4.1: the propagation step is a 3-D FFT of the projected grid
// sources on the doubled grid, a pointwise product with the transformed grid
// Green's function, and an inverse 3-D FFT; only the slabs that hold the
// scatterer are transformed forward, and only the outputs that are
// interpolated back are transformed inverse (footnote 2).  Here that pruning
// is done per axis: with n the unpadded and L the padded extent,
//
//   z pass  : [G][nz][ny][nx]  -> [G][Lz][ny][nx]   (reads nz, writes Lz)
//   y pass  : [G][Lz][ny][nx]  -> [G][Lz][Ly][nx]   (reads ny, writes Ly)
//   x pass  : per (ky, kz) row: forward FFT of nx zero-padded inputs,
//             product with Ghat, inverse FFT, keep nx outputs (in place)
//   y^-1    : [G][Lz][Ly][nx]  -> [G][Lz][ny][nx]   (reads Ly, writes ny)
//   z^-1    : [G][Lz][ny][nx]  -> [G][nz][ny][nx]   (reads Lz, writes nz)
//
// Each pencil is staged in shared memory and transformed with the Stockham
// autosort algorithm (ping-pong buffers, natural-order output), radices
// {4, 3, 5, 2}.  Strided passes stage a tile of TX consecutive x columns so
// that every global access is a contiguous run of TX complex values.  Ghat is
// stored as one octant (it is even in each axis) and pre-scaled by 1/(LxLyLz),
// so the inverse transforms are unnormalised.
//
// The butterflies are written once over an arithmetic policy:
//   P32 complex64 (float2), P64 complex128 (double2) and PFF complex
//   float-float (float4 = re.hi, re.lo, im.hi, im.lo; about 48 bits, on the
//   FP32 pipes; see ff.h).  Per-stage index arithmetic uses precomputed
//   multiply-shift division, so no integer division runs in the kernels.
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "common.h"
#include "ff.h"
#include "fft4.cuh"
#include "fft_policy.h"
#include "geom.h"

namespace aim {

// ------------------------------------------------------------------ plans
static Div32 make_div(uint32_t d) {
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;
  const uint64_t m = ((1ull << 32) * ((1ull << l) - d)) / d + 1;
  return Div32{(uint32_t)m, l, d};
}
__device__ __forceinline__ uint32_t qdiv(uint32_t n, const Div32& D) { return (__umulhi(n, D.m) + n) >> D.l; }

FftPlan make_plan(int L) {
  FftPlan p{};
  p.L = L;
  p.nst = 0;
  int x = L;
  const int order[4] = {4, 3, 5, 2};
  for (int oi = 0; oi < 4; ++oi) {
    const int r = order[oi];
    while (x % r == 0 && p.nst < kMaxStages) {
      p.rad[p.nst++] = r;
      x /= r;
    }
  }
  if (x != 1) {
    p.nst = -1;  // not 2,3,5-smooth
    return p;
  }
  int Ns = 1;
  for (int s = 0; s < p.nst; ++s) {
    p.Ns[s] = Ns;
    p.dNs[s] = make_div((uint32_t)Ns);
    p.dnb[s] = make_div((uint32_t)(L / p.rad[s]));
    Ns *= p.rad[s];
  }
  return p;
}

// One Stockham stage over `count` pencils of length L in shared memory.
// COLS: element p of pencil c at buf[p * kTX + c] (column tiles, count = kTX);
// otherwise at buf[c * L + p] (row tiles).
// nvalid: samples p >= nvalid of every pencil are zero (only used by the
// first stage, where Ns = 1: a radix-4 butterfly whose two upper inputs are
// zero costs half the additions).
template <class P, bool INV, int RAD, bool COLS>
__device__ __forceinline__ void stage_r(const typename P::S* __restrict__ src, typename P::S* __restrict__ dst,
                                        const FftPlan& pl, int s, int count, const typename P::S* __restrict__ tw,
                                        int nvalid) {
  using T = typename P::T;
  const int L = pl.L;
  const int nb = L / RAD;
  const int Ns = pl.Ns[s];
  const int tstep = L / (Ns * RAD);
  const Div32 dNs = pl.dNs[s], dnb = pl.dnb[s];
  const int total = nb * count;
  for (int item = threadIdx.x; item < total; item += blockDim.x) {
    int c, j;
    if (COLS) {
      c = item & (P::kTX - 1);  // count == kTX, a power of two
      j = item / P::kTX;
    } else {
      c = (int)qdiv((uint32_t)item, dnb);
      j = item - c * nb;
    }
    const int q = (int)qdiv((uint32_t)j, dNs);
    const int k = j - q * Ns;
    T v[RAD];
    if (RAD == 4 && s == 0 && j + 2 * nb >= nvalid) {
      // first stage (Ns = 1, idxD = 4 j): inputs 2 and 3 are zero
      const T a = P::ld(src[COLS ? j * P::kTX + c : c * L + j]);
      const T b = (j + nb < nvalid) ? P::ld(src[COLS ? (j + nb) * P::kTX + c : c * L + j + nb]) : P::zero();
      const T ib = P::template mul_mi<INV>(b);
      v[0] = P::add(a, b);
      v[1] = P::add(a, ib);
      v[2] = P::sub(a, b);
      v[3] = P::sub(a, ib);
#pragma unroll
      for (int r = 0; r < RAD; ++r) {
        const int p = 4 * j + r;
        dst[COLS ? p * P::kTX + c : c * L + p] = P::st(v[r]);
      }
      continue;
    }
#pragma unroll
    for (int r = 0; r < RAD; ++r) {
      const int p = j + r * nb;
      T a = P::ld(src[COLS ? p * P::kTX + c : c * L + p]);
      if (r > 0 && Ns > 1) a = P::mul(a, P::conj_if(P::ld(tw[r * k * tstep]), INV));  // r k tstep < L
      v[r] = a;
    }
    if (RAD == 2) dft2<P, INV>(v);
    if (RAD == 3) dft3<P, INV>(v);
    if (RAD == 4) dft4<P, INV>(v);
    if (RAD == 5) dft5<P, INV>(v);
    const int idxD = q * Ns * RAD + k;
#pragma unroll
    for (int r = 0; r < RAD; ++r) {
      const int p = idxD + r * Ns;
      dst[COLS ? p * P::kTX + c : c * L + p] = P::st(v[r]);
    }
  }
}

// Full transform in shared memory; returns the buffer that holds the result.
template <class P, bool INV, bool COLS>
__device__ typename P::S* stockham(typename P::S* b0, typename P::S* b1, const FftPlan& pl, int count,
                                   const typename P::S* __restrict__ tw, int nvalid) {
  for (int s = 0; s < pl.nst; ++s) {
    switch (pl.rad[s]) {
      case 2: stage_r<P, INV, 2, COLS>(b0, b1, pl, s, count, tw, nvalid); break;
      case 3: stage_r<P, INV, 3, COLS>(b0, b1, pl, s, count, tw, nvalid); break;
      case 4: stage_r<P, INV, 4, COLS>(b0, b1, pl, s, count, tw, nvalid); break;
      default: stage_r<P, INV, 5, COLS>(b0, b1, pl, s, count, tw, nvalid); break;
    }
    __syncthreads();
    typename P::S* t = b0;
    b0 = b1;
    b1 = t;
  }
  return b0;
}

// ------------------------------------------------------------------ strided pass
using StridedArgs = StridedArgs4;

// Four-step kernels per policy (fft4_p32.cu, fft4_p64.cu, fft4_pff.cu):
// 1 launched, 0 no kernel for this length, < 0 minus an error code.
int fft4_strided_p32(aim_ctx*, const char*, bool, const float2*, float2*, const StridedArgs4&, int, int,
                     const float2*, bool);
int fft4_strided_p64(aim_ctx*, const char*, bool, const double2*, double2*, const StridedArgs4&, int, int,
                     const double2*, bool);
int fft4_strided_pff(aim_ctx*, const char*, bool, const float4*, float4*, const StridedArgs4&, int, int,
                     const float4*, bool);
int fft4_x_p32(aim_ctx*, const char*, float2*, const XArgs4&, int, const float2*, const float2*, int, bool);
int fft4_x_p64(aim_ctx*, const char*, double2*, const XArgs4&, int, const double2*, const double2*, int, bool);
int fft4_x_pff(aim_ctx*, const char*, float4*, const XArgs4&, int, const float4*, const float4*, int, bool);
template <class P> struct Fft4;
template <> struct Fft4<P32> {
  template <class... A> static int strided(A... a) { return fft4_strided_p32(a...); }
  template <class... A> static int x(A... a) { return fft4_x_p32(a...); }
};
template <> struct Fft4<P64> {
  template <class... A> static int strided(A... a) { return fft4_strided_p64(a...); }
  template <class... A> static int x(A... a) { return fft4_x_p64(a...); }
};
template <> struct Fft4<PFF> {
  template <class... A> static int strided(A... a) { return fft4_strided_pff(a...); }
  template <class... A> static int x(A... a) { return fft4_x_pff(a...); }
};

// Output element conversion of a pass (identity for every policy in use).
template <class S, class O> struct OutConv {
  __device__ static O f(const S& s) { return s; }
};

template <class P, bool INV, class O>
__global__ void __launch_bounds__(256) fft_strided(const typename P::S* __restrict__ in, O* __restrict__ out,
                                                   StridedArgs a, const FftPlan* __restrict__ plan,
                                                   const typename P::S* __restrict__ tw) {
  using S = typename P::S;
  constexpr int TX = P::kTX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const FftPlan& pl = *plan;
  S* b0 = reinterpret_cast<S*>(smem_raw);
  const int L = pl.L;
  S* b1 = b0 + L * TX;
  const int x0 = blockIdx.x * TX;
  const int ia = blockIdx.y;
  const long long g = blockIdx.z;
  const S* src = in + g * a.sG_in + ia * a.sA_in + x0;
  for (int e = threadIdx.x; e < L * TX; e += blockDim.x) {
    const int p = e / TX, c = e & (TX - 1);
    S v = P::st(P::zero());
    if (p < a.n_in && x0 + c < a.X) v = src[p * a.sP_in + c];
    b0[e] = v;
  }
  __syncthreads();
  S* res = stockham<P, INV, true>(b0, b1, pl, TX, tw, a.n_in);
  O* dst = out + g * a.sG_out + ia * a.sA_out + x0;
  for (int e = threadIdx.x; e < a.n_out * TX; e += blockDim.x) {
    const int p = e / TX, c = e & (TX - 1);
    if (x0 + c < a.X) dst[p * a.sP_out + c] = OutConv<S, O>::f(res[e]);
  }
}

// ------------------------------------------------------------------ x pass
struct XArgs {
  int nx;          // samples per row kept (read and written)
  int rows_y;      // Ly
  int rows_z;      // Lz
  int G;           // grids
  int TG;          // grids per shared-memory tile
  long long sG;    // grid stride (elements)
  int hx, hy, hz;  // octant extents of Ghat
};

// MODE 0: forward, times Ghat, inverse (keep nx); MODE 1: forward only on full rows.
template <class P, int MODE>
__global__ void __launch_bounds__(256) fft_x(typename P::S* __restrict__ buf, XArgs a, const FftPlan* __restrict__ plan,
                                             const typename P::S* __restrict__ ghat, const typename P::S* __restrict__ tw) {
  using S = typename P::S;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const FftPlan& pl = *plan;
  const int L = pl.L;
  S* gr = reinterpret_cast<S*>(smem_raw);
  S* b0 = gr + L;
  S* b1 = b0 + a.TG * L;
  const int ky = blockIdx.x, kz = blockIdx.y;
  const long long row = ((long long)kz * a.rows_y + ky) * a.nx;
  if (MODE == 0) {
    const int iy = min(ky, a.rows_y - ky), iz = min(kz, a.rows_z - kz);
    const S* grow = ghat + ((long long)iz * a.hy + iy) * a.hx;
    for (int e = threadIdx.x; e < L; e += blockDim.x) gr[e] = grow[min(e, L - e)];
  }
  for (int g0 = 0; g0 < a.G; g0 += a.TG) {
    const int ng = min(a.TG, a.G - g0);
    __syncthreads();
    for (int c = 0; c < ng; ++c)
      for (int p = threadIdx.x; p < L; p += blockDim.x) {
        S v = P::st(P::zero());
        if (p < a.nx) v = buf[(g0 + c) * a.sG + row + p];
        b0[c * L + p] = v;
      }
    __syncthreads();
    S* res = stockham<P, false, false>(b0, b1, pl, ng, tw, a.nx);
    if (MODE == 0) {
      S* oth = (res == b0) ? b1 : b0;
      for (int c = 0; c < ng; ++c)
        for (int p = threadIdx.x; p < L; p += blockDim.x) res[c * L + p] = P::st(P::mul(P::ld(res[c * L + p]), P::ld(gr[p])));
      __syncthreads();
      res = stockham<P, true, false>(res, oth, pl, ng, tw, L);
    }
    for (int c = 0; c < ng; ++c)
      for (int p = threadIdx.x; p < a.nx; p += blockDim.x) buf[(g0 + c) * a.sG + row + p] = res[c * L + p];
  }
}

// ------------------------------------------------------------------ drivers
template <class P, bool INV, class O = typename P::S>
static int launch_strided(aim_ctx* c, const char* name, const typename P::S* in, O* out, const StridedArgs& a, int G,
                          const FftPlan* plan_dev, int L, const typename P::S* tw) {
  constexpr int TX = P::kTX;
  const size_t sm = 2ull * L * TX * sizeof(typename P::S);
  if (sm > 227 * 1024) {
    set_error(std::string(name) + ": padded length too large for shared memory");
    return AIM_EINVAL;
  }
  // once per template instance (thread-safe static initialisation)
  static const cudaError_t attr =
      cudaFuncSetAttribute(fft_strided<P, INV, O>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  AIM_CUDA_TRY(attr);
  dim3 grid((a.X + TX - 1) / TX, a.A, G);
  AIM_LAUNCH(c, name, fft_strided<P, INV, O><<<grid, 256, sm, c->stream>>>(in, out, a, plan_dev, tw));
  return launch_check(c, name);
}

template <class P, int MODE>
static int launch_x(aim_ctx* c, const char* name, typename P::S* buf, XArgs a, const FftPlan* plan_dev, int L,
                    const typename P::S* ghat, const typename P::S* tw) {
  using S = typename P::S;
  // grids per tile: keep shared memory under ~100 KB so two blocks fit an SM
  int TG = (int)((100 * 1024) / (2ull * L * sizeof(S)));
  TG = TG < 1 ? 1 : TG;
  TG = TG > a.G ? a.G : TG;
  TG = TG > 16 ? 16 : TG;
  a.TG = TG;
  const size_t sm = (size_t)(2 * TG + 1) * L * sizeof(S);
  if (sm > 227 * 1024) {
    set_error(std::string(name) + ": padded x length too large for shared memory");
    return AIM_EINVAL;
  }
  static const cudaError_t attr =
      cudaFuncSetAttribute(fft_x<P, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  AIM_CUDA_TRY(attr);
  dim3 grid(a.rows_y, a.rows_z);
  AIM_LAUNCH(c, name, fft_x<P, MODE><<<grid, 256, sm, c->stream>>>(buf, a, plan_dev, ghat, tw));
  return launch_check(c, name);
}

bool fourstep_split(int L, int* L1, int* L2) {
  switch (L) {
#define AIM_CASE(LL, A1, A2) \
  case LL: *L1 = A1; *L2 = A2; return true;
    AIM_FOURSTEP_LENGTHS(AIM_CASE)
#undef AIM_CASE
    default: return false;
  }
}

int fft_policy_of(int precision) { return precision == AIM_C64 ? 0 : precision == AIM_C128_F64 ? 1 : 2; }

int fft_kernel_for(const aim_ctx* c, int pol, int pass) {
  const int k = c->fft_kernel[pol][pass];
  return k != AIM_FFT_AUTO ? k : AIM_FFT_FOURSTEP;
}

template <class P> constexpr int policy_index() {
  return std::is_same<P, P32>::value ? 0 : std::is_same<P, P64>::value ? 1 : 2;
}

// Strided pass with the selected kernel (four-step where the length has one).
template <class P, bool INV, class O = typename P::S>
static int strided_pass(aim_ctx* c, int pass, const char* name, const typename P::S* in, O* out,
                        const StridedArgs& a, int G, const FftPlan* plan_dev, int L, const typename P::S* tw) {
  const int k = fft_kernel_for(c, policy_index<P>(), pass);
  if (k != AIM_FFT_STOCKHAM) {
    const int rc = Fft4<P>::strided(c, name, INV, in, out, a, G, L, tw, k == AIM_FFT_FOURSTEP_WIDE);
    if (rc == 1) return AIM_OK;
    if (rc < 0) return -rc;
  }
  return launch_strided<P, INV, O>(c, name, in, out, a, G, plan_dev, L, tw);
}

template <class P>
static int x_pass(aim_ctx* c, const char* name, typename P::S* buf, XArgs a, const FftPlan* plan_dev, int L,
                  const typename P::S* ghat, const typename P::S* tw) {
  const int k = fft_kernel_for(c, policy_index<P>(), 2);
  if (k != AIM_FFT_STOCKHAM) {
    XArgs4 x4{};
    x4.nx = a.nx; x4.Ly = a.rows_y; x4.Lz = a.rows_z; x4.G = a.G; x4.sG = a.sG; x4.hx = a.hx; x4.hy = a.hy;
    const int rc = Fft4<P>::x(c, name, buf, x4, L, ghat, tw, k == AIM_FFT_FOURSTEP_SMALL ? 128 : 256,
                              k == AIM_FFT_FOURSTEP_WARP);
    if (rc == 1) return AIM_OK;
    if (rc < 0) return -rc;
  }
  return launch_x<P, 0>(c, name, buf, a, plan_dev, L, ghat, tw);
}

template <class P>
static int convolve(aim_ctx* c, typename P::S* g0, typename P::S* g1, typename P::S* g2, const typename P::S* ghat,
                    typename P::S* const* tw, int G, typename P::S* phi) {
  const int nx = c->n[0], ny = c->n[1], nz = c->n[2];
  const int Lx = c->L[0], Ly = c->L[1], Lz = c->L[2];
  const FftPlan* pd = c->plan_dev;
  // A planar grid (Lz = nz = 1) has no z passes: the y passes read and write g0.
  const bool zpass = Lz > 1;
  typename P::S* gz = zpass ? g1 : g0;
  if (zpass) {  // z forward: g0 [G][nz][ny][nx] -> g1 [G][Lz][ny][nx]
    StridedArgs a{};
    a.n_in = nz; a.n_out = Lz; a.X = nx; a.A = ny;
    a.cols = c->colmask;  // empty (x, y) columns read nothing
    a.sG_in = (long long)nz * ny * nx; a.sA_in = nx; a.sP_in = (long long)ny * nx;
    a.sG_out = (long long)Lz * ny * nx; a.sA_out = nx; a.sP_out = (long long)ny * nx;
    AIM_TRY((strided_pass<P, false>(c, 0, "fft_z_fwd", g0, g1, a, G, pd + 2, Lz, tw[2])));
  }
  {  // y forward: gz [G][Lz][ny][nx] -> g2 [G][Lz][Ly][nx]
    StridedArgs a{};
    a.n_in = ny; a.n_out = Ly; a.X = nx; a.A = Lz;
    a.sG_in = (long long)Lz * ny * nx; a.sA_in = (long long)ny * nx; a.sP_in = nx;
    a.sG_out = (long long)Lz * Ly * nx; a.sA_out = (long long)Ly * nx; a.sP_out = nx;
    AIM_TRY((strided_pass<P, false>(c, 1, "fft_y_fwd", gz, g2, a, G, pd + 1, Ly, tw[1])));
  }
  {  // x: forward, times Ghat, inverse, in place on g2
    XArgs a{};
    a.nx = nx; a.rows_y = Ly; a.rows_z = Lz; a.G = G;
    a.sG = (long long)Lz * Ly * nx;
    a.hx = Lx / 2 + 1; a.hy = Ly / 2 + 1; a.hz = Lz / 2 + 1;
    AIM_TRY((x_pass<P>(c, "fft_x_conv", g2, a, pd + 0, Lx, ghat, tw[0])));
  }
  {  // y inverse: g2 -> gz [G][Lz][ny][nx]
    StridedArgs a{};
    a.n_in = Ly; a.n_out = ny; a.X = nx; a.A = Lz;
    a.sG_in = (long long)Lz * Ly * nx; a.sA_in = (long long)Ly * nx; a.sP_in = nx;
    a.sG_out = (long long)Lz * ny * nx; a.sA_out = (long long)ny * nx; a.sP_out = nx;
    AIM_TRY((strided_pass<P, true>(c, 3, "fft_y_inv", g2, gz, a, G, pd + 1, Ly, tw[1])));
  }
  if (zpass) {  // z inverse: g1 -> phi [G][nz][ny][nx] (g0, or g2 when grid0 keeps the projection's zeros)
    StridedArgs a{};
    a.n_in = Lz; a.n_out = nz; a.X = nx; a.A = ny;
    a.cols = c->colmask;  // columns without a stencil node are never interpolated from
    a.sG_in = (long long)Lz * ny * nx; a.sA_in = nx; a.sP_in = (long long)ny * nx;
    a.sG_out = (long long)nz * ny * nx; a.sA_out = nx; a.sP_out = (long long)ny * nx;
    AIM_TRY((strided_pass<P, true>(c, 4, "fft_z_inv", g1, phi, a, G, pd + 2, Lz, tw[2])));
  }
  return AIM_OK;
}

int fft_convolve_c64(aim_ctx* c, int G) {
  PrecData<float>& p = c->p32;
  return convolve<P32>(c, p.grid0, p.grid1, p.grid2, p.ghat, p.tw, G, phi_grid(c, p.grid0, p.grid2));
}
int fft_convolve_c128(aim_ctx* c, int G) {
  PrecData<double>& p = c->p64;
  return convolve<P64>(c, p.grid0, p.grid1, p.grid2, p.ghat, p.tw, G, phi_grid(c, p.grid0, p.grid2));
}
int fft_convolve_ff(aim_ctx* c, int G) {
  FFData& p = c->pff;
  return convolve<PFF>(c, p.grid0, p.grid1, p.grid2, p.ghat, p.tw, G, phi_grid(c, p.grid0, p.grid2));
}

// ------------------------------------------------------------------ Ghat
// Circulant embedding of G_h on the padded grid: per axis, index i maps to
// offset i (i < n), i - L (i > L - n), and the gap in between is zero;
// G_h(D) = exp(-j k h |D|) / (4 pi h |D|), G_h(0) = 0.
__global__ void sample_green(double2* g, int Lx, int Ly, int Lz, int nx, int ny, int nz, double k, double h) {
  long long total = (long long)Lx * Ly * Lz;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e % Lx);
    int j = (int)((e / Lx) % Ly);
    int l = (int)(e / ((long long)Lx * Ly));
    bool vx = (i < nx) || (i > Lx - nx), vy = (j < ny) || (j > Ly - ny), vz = (l < nz) || (l > Lz - nz);
    int ox = (i < nx) ? i : i - Lx, oy = (j < ny) ? j : j - Ly, oz = (l < nz) ? l : l - Lz;
    double2 v = make_double2(0.0, 0.0);
    if (vx && vy && vz && (ox | oy | oz) != 0) {
      double r = h * sqrt((double)ox * ox + (double)oy * oy + (double)oz * oz);
      double s = 1.0 / (4.0 * kPi * r);
      double sn, cs;
      sincos(k * r, &sn, &cs);
      v = make_double2(cs * s, -sn * s);
    }
    g[e] = v;
  }
}

__global__ void extract_octant(const double2* full, double2* oct64, float2* oct32, float4* octff, int Lx, int Ly,
                               int Lz, double scale) {
  int hx = Lx / 2 + 1, hy = Ly / 2 + 1, hz = Lz / 2 + 1;
  long long total = (long long)hx * hy * hz;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e % hx);
    int j = (int)((e / hx) % hy);
    int l = (int)(e / ((long long)hx * hy));
    double2 v = full[((long long)l * Ly + j) * Lx + i];
    v.x *= scale;
    v.y *= scale;
    oct64[e] = v;
    oct32[e] = make_float2((float)v.x, (float)v.y);
    const ff re = ff_from_double(v.x), im = ff_from_double(v.y);
    octff[e] = make_float4(re.hi, re.lo, im.hi, im.lo);
  }
}

int build_ghat(aim_ctx* c) {
  const int Lx = c->L[0], Ly = c->L[1], Lz = c->L[2];
  const long long total = (long long)Lx * Ly * Lz;
  double2 *a = nullptr, *b = nullptr;
  AIM_CUDA_TRY(cudaMallocAsync(&a, total * sizeof(double2), c->stream));
  AIM_CUDA_TRY(cudaMallocAsync(&b, total * sizeof(double2), c->stream));
  AIM_LAUNCH(c, "sample_green",
             sample_green<<<1024, 256, 0, c->stream>>>(a, Lx, Ly, Lz, c->n[0], c->n[1], c->n[2], c->k, c->h));
  AIM_TRY(launch_check(c, "sample_green"));
  // z: full transform a -> b (none for a planar grid, Lz = 1); y: b -> a;
  // x: rows of a in place (FP64)
  StridedArgs s{};
  s.n_in = Lz; s.n_out = Lz; s.X = Lx; s.A = Ly;
  s.sG_in = total; s.sA_in = Lx; s.sP_in = (long long)Ly * Lx;
  s.sG_out = total; s.sA_out = Lx; s.sP_out = (long long)Ly * Lx;
  // full transforms; four-step kernels where the length has one (longer than the Stockham kernel allows)
  const auto pass = [&](const char* name, const double2* in, double2* out, const StridedArgs& sa, int d) -> int {
    const int rc = Fft4<P64>::strided(c, name, false, in, out, sa, 1, c->L[d], c->p64.tw[d], false);
    if (rc == 1) return AIM_OK;
    if (rc < 0) return -rc;
    return launch_strided<P64, false>(c, name, in, out, sa, 1, c->plan_dev + d, c->L[d], c->p64.tw[d]);
  };
  if (Lz > 1)
    AIM_TRY(pass("ghat_z", a, b, s, 2));
  else
    std::swap(a, b);
  s.n_in = Ly; s.n_out = Ly; s.X = Lx; s.A = Lz;
  s.sA_in = (long long)Ly * Lx; s.sP_in = Lx;
  s.sA_out = (long long)Ly * Lx; s.sP_out = Lx;
  AIM_TRY(pass("ghat_y", b, a, s, 1));
  XArgs x{};
  x.nx = Lx; x.rows_y = Ly; x.rows_z = Lz; x.G = 1; x.sG = total;
  x.hx = Lx / 2 + 1; x.hy = Ly / 2 + 1; x.hz = Lz / 2 + 1;
  AIM_TRY((launch_x<P64, 1>(c, "ghat_x", a, x, c->plan_dev + 0, Lx, nullptr, c->p64.tw[0])));
  AIM_LAUNCH(c, "extract_octant",
             extract_octant<<<1024, 256, 0, c->stream>>>(a, c->p64.ghat, c->p32.ghat, c->pff.ghat, Lx, Ly, Lz,
                                                         1.0 / (double)total));
  AIM_TRY(launch_check(c, "extract_octant"));
  AIM_CUDA_TRY(cudaFreeAsync(a, c->stream));
  AIM_CUDA_TRY(cudaFreeAsync(b, c->stream));
  return AIM_OK;
}

}  // namespace aim

namespace aim {
// Complex64 convolution on caller-provided pass buffers (used by the
// product variant that allocates nothing; same kernels and launch shapes).
int fft_convolve_c64_bufs(aim_ctx* c, int G, float2* g0, float2* g1, float2* g2) {
  return convolve<P32>(c, g0, g1, g2, c->p32.ghat, c->p32.tw, G, g0);
}
}  // namespace aim
