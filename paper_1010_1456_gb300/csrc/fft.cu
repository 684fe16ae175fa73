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
#include <cmath>

#include "common.h"
#include "geom.h"

namespace aim {

FftPlan make_plan(int L) {
  FftPlan p{};
  p.L = L;
  p.nst = 0;
  int x = L;
  const int order[4] = {4, 3, 5, 2};
  for (int oi = 0; oi < 4; ++oi) {
    int r = order[oi];
    while (x % r == 0) {
      p.radix[p.nst++] = r;
      x /= r;
    }
  }
  if (x != 1) p.nst = -1;  // not 2,3,5-smooth
  return p;
}

// ------------------------------------------------------------------ butterflies
template <typename C, bool INV> __device__ __forceinline__ C mul_mi(C a) {
  // forward: multiply by -i; inverse: by +i
  C r;
  if (!INV) { r.x = a.y; r.y = -a.x; }
  else { r.x = -a.y; r.y = a.x; }
  return r;
}

template <typename R, bool INV> __device__ __forceinline__ void dft2(cplx<R>* v) {
  cplx<R> a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}
template <typename R, bool INV> __device__ __forceinline__ void dft3(cplx<R>* v) {
  const R h = (R)0.86602540378443864676;  // sin(2 pi / 3)
  cplx<R> a = v[0], s = cadd(v[1], v[2]), d = csub(v[1], v[2]);
  cplx<R> m = a;
  m.x -= (R)0.5 * s.x;
  m.y -= (R)0.5 * s.y;
  cplx<R> t = mul_mi<cplx<R>, INV>(cscale(d, h));
  v[0] = cadd(a, s);
  v[1] = cadd(m, t);
  v[2] = csub(m, t);
}
template <typename R, bool INV> __device__ __forceinline__ void dft4(cplx<R>* v) {
  cplx<R> s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
  cplx<R> s13 = cadd(v[1], v[3]), d13 = mul_mi<cplx<R>, INV>(csub(v[1], v[3]));
  v[0] = cadd(s02, s13);
  v[2] = csub(s02, s13);
  v[1] = cadd(d02, d13);
  v[3] = csub(d02, d13);
}
template <typename R, bool INV> __device__ __forceinline__ void dft5(cplx<R>* v) {
  const R c1 = (R)0.30901699437494742410, c2 = (R)-0.80901699437494742410;  // cos(2pi/5), cos(4pi/5)
  const R s1 = (R)0.95105651629515357212, s2 = (R)0.58778525229247312917;   // sin(2pi/5), sin(4pi/5)
  cplx<R> a0 = v[0];
  cplx<R> t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
  cplx<R> t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
  cplx<R> b1, b2, e1, e2;
  b1.x = a0.x + c1 * t1.x + c2 * t2.x;
  b1.y = a0.y + c1 * t1.y + c2 * t2.y;
  b2.x = a0.x + c2 * t1.x + c1 * t2.x;
  b2.y = a0.y + c2 * t1.y + c1 * t2.y;
  cplx<R> u1, u2;
  u1.x = s1 * t3.x + s2 * t4.x;
  u1.y = s1 * t3.y + s2 * t4.y;
  u2.x = s2 * t3.x - s1 * t4.x;
  u2.y = s2 * t3.y - s1 * t4.y;
  e1 = mul_mi<cplx<R>, INV>(u1);
  e2 = mul_mi<cplx<R>, INV>(u2);
  v[0] = cadd(a0, cadd(t1, t2));
  v[1] = cadd(b1, e1);
  v[4] = csub(b1, e1);
  v[2] = cadd(b2, e2);
  v[3] = csub(b2, e2);
}

// One Stockham stage over `count` independent pencils of length L.
// Element p of pencil c lives at buf[idx(p, c)] with idx = p*pstride + c*cstride.
template <typename R, bool INV, int RAD>
__device__ __forceinline__ void stage_r(const cplx<R>* __restrict__ src, cplx<R>* __restrict__ dst, int L, int Ns,
                                        int count, int pstride, int cstride, const cplx<R>* __restrict__ tw) {
  const int nb = L / RAD;
  const int tstep = L / (Ns * RAD);
  for (int item = threadIdx.x; item < nb * count; item += blockDim.x) {
    int c, j;
    if (cstride == 1) { c = item % count; j = item / count; }  // column tiles: adjacent threads adjacent columns
    else { j = item % nb; c = item / nb; }                     // row tiles: adjacent threads adjacent j
    const int k = j % Ns;
    cplx<R> v[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) {
      cplx<R> a = src[(j + r * nb) * pstride + c * cstride];
      if (r > 0 && Ns > 1) {
        cplx<R> w = tw[r * k * tstep];  // r k tstep < L
        if (INV) w.y = -w.y;
        a = cmul(a, w);
      }
      v[r] = a;
    }
    if (RAD == 2) dft2<R, INV>(v);
    if (RAD == 3) dft3<R, INV>(v);
    if (RAD == 4) dft4<R, INV>(v);
    if (RAD == 5) dft5<R, INV>(v);
    const int idxD = (j / Ns) * Ns * RAD + k;
#pragma unroll
    for (int r = 0; r < RAD; ++r) dst[(idxD + r * Ns) * pstride + c * cstride] = v[r];
  }
}

// Full transform in shared memory; returns the buffer that holds the result.
template <typename R, bool INV>
__device__ cplx<R>* stockham(cplx<R>* b0, cplx<R>* b1, const FftPlan& plan, int count, int pstride, int cstride,
                             const cplx<R>* __restrict__ tw) {
  int Ns = 1;
  const int L = plan.L;
  for (int s = 0; s < plan.nst; ++s) {
    const int rad = plan.radix[s];
    switch (rad) {
      case 2: stage_r<R, INV, 2>(b0, b1, L, Ns, count, pstride, cstride, tw); break;
      case 3: stage_r<R, INV, 3>(b0, b1, L, Ns, count, pstride, cstride, tw); break;
      case 4: stage_r<R, INV, 4>(b0, b1, L, Ns, count, pstride, cstride, tw); break;
      default: stage_r<R, INV, 5>(b0, b1, L, Ns, count, pstride, cstride, tw); break;
    }
    __syncthreads();
    cplx<R>* t = b0;
    b0 = b1;
    b1 = t;
    Ns *= rad;
  }
  return b0;
}

// ------------------------------------------------------------------ strided pass
struct StridedArgs {
  int n_in, n_out;  // samples read (rest zero) / samples written
  int X, A;         // contiguous extent, other-axis extent
  long long sG_in, sA_in, sP_in;
  long long sG_out, sA_out, sP_out;
  FftPlan plan;
};

template <typename R> AIM_HD constexpr int tile_x() { return sizeof(R) == 4 ? 16 : 8; }

template <typename R, bool INV>
__global__ void __launch_bounds__(256) fft_strided(const cplx<R>* __restrict__ in, cplx<R>* __restrict__ out,
                                                   StridedArgs a, const cplx<R>* __restrict__ tw) {
  constexpr int TX = tile_x<R>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* b0 = reinterpret_cast<cplx<R>*>(smem_raw);
  const int L = a.plan.L;
  cplx<R>* b1 = b0 + L * TX;
  const int x0 = blockIdx.x * TX;
  const int ia = blockIdx.y;
  const long long g = blockIdx.z;
  const cplx<R>* src = in + g * a.sG_in + ia * a.sA_in + x0;
  for (int e = threadIdx.x; e < L * TX; e += blockDim.x) {
    int p = e / TX, c = e % TX;
    cplx<R> v = cmake<cplx<R>>(0.0, 0.0);
    if (p < a.n_in && x0 + c < a.X) v = src[p * a.sP_in + c];
    b0[e] = v;
  }
  __syncthreads();
  cplx<R>* res = stockham<R, INV>(b0, b1, a.plan, TX, TX, 1, tw);
  cplx<R>* dst = out + g * a.sG_out + ia * a.sA_out + x0;
  for (int e = threadIdx.x; e < a.n_out * TX; e += blockDim.x) {
    int p = e / TX, c = e % TX;
    if (x0 + c < a.X) dst[p * a.sP_out + c] = res[e];
  }
}

// ------------------------------------------------------------------ x pass
struct XArgs {
  int nx;        // samples per row kept (read and written)
  int rows_y;    // Ly
  int rows_z;    // Lz
  int G;         // grids
  int TG;        // grids per shared-memory tile
  long long sG;  // grid stride (elements)
  int hx, hy, hz;  // octant extents of Ghat
  FftPlan plan;
};

// mode 0: forward, times Ghat, inverse (keep nx); mode 1: forward only on full rows.
template <typename R, int MODE>
__global__ void __launch_bounds__(256) fft_x(cplx<R>* __restrict__ buf, XArgs a, const cplx<R>* __restrict__ ghat,
                                             const cplx<R>* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = a.plan.L;
  cplx<R>* gr = reinterpret_cast<cplx<R>*>(smem_raw);
  cplx<R>* b0 = gr + L;
  cplx<R>* b1 = b0 + a.TG * L;
  const int ky = blockIdx.x, kz = blockIdx.y;
  const long long row = ((long long)kz * a.rows_y + ky) * a.nx;
  if (MODE == 0) {
    const int iy = min(ky, a.rows_y - ky), iz = min(kz, a.rows_z - kz);
    const cplx<R>* grow = ghat + ((long long)iz * a.hy + iy) * a.hx;
    for (int e = threadIdx.x; e < L; e += blockDim.x) gr[e] = grow[min(e, L - e)];
  }
  for (int g0 = 0; g0 < a.G; g0 += a.TG) {
    const int ng = min(a.TG, a.G - g0);
    __syncthreads();
    for (int e = threadIdx.x; e < ng * L; e += blockDim.x) {
      int c = e / L, p = e % L;
      cplx<R> v = cmake<cplx<R>>(0.0, 0.0);
      if (p < a.nx) v = buf[(g0 + c) * a.sG + row + p];
      b0[e] = v;
    }
    __syncthreads();
    cplx<R>* res = stockham<R, false>(b0, b1, a.plan, ng, 1, L, tw);
    if (MODE == 0) {
      cplx<R>* oth = (res == b0) ? b1 : b0;
      for (int e = threadIdx.x; e < ng * L; e += blockDim.x) res[e] = cmul(res[e], gr[e % L]);
      __syncthreads();
      res = stockham<R, true>(res, oth, a.plan, ng, 1, L, tw);
    }
    for (int e = threadIdx.x; e < ng * a.nx; e += blockDim.x) {
      int c = e / a.nx, p = e % a.nx;
      buf[(g0 + c) * a.sG + row + p] = res[c * L + p];
    }
  }
}

// ------------------------------------------------------------------ drivers
template <typename R> static size_t strided_smem(int L) { return 2ull * L * tile_x<R>() * sizeof(cplx<R>); }

template <typename R, bool INV>
static int launch_strided(aim_ctx* c, const char* name, const cplx<R>* in, cplx<R>* out, const StridedArgs& a, int G,
                          const cplx<R>* tw) {
  constexpr int TX = tile_x<R>();
  size_t sm = strided_smem<R>(a.plan.L);
  // once per template instance (thread-safe static initialisation)
  static const cudaError_t attr =
      cudaFuncSetAttribute(fft_strided<R, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  AIM_CUDA_TRY(attr);
  dim3 grid((a.X + TX - 1) / TX, a.A, G);
  AIM_LAUNCH(c, name, fft_strided<R, INV><<<grid, 256, sm, c->stream>>>(in, out, a, tw));
  return launch_check(c, "fft_strided");
}

template <typename R, int MODE>
static int launch_x(aim_ctx* c, const char* name, cplx<R>* buf, XArgs a, const cplx<R>* ghat, const cplx<R>* tw) {
  const int L = a.plan.L;
  // grids per tile: keep shared memory under ~100 KB so two blocks fit an SM
  int TG = (int)((100 * 1024) / (2ull * L * sizeof(cplx<R>)) );
  TG = TG < 1 ? 1 : TG;
  TG = TG > a.G ? a.G : TG;
  TG = TG > 16 ? 16 : TG;
  a.TG = TG;
  size_t sm = (size_t)(2 * TG + 1) * L * sizeof(cplx<R>);
  if (sm > 227 * 1024) {
    set_error("fft_x: padded x length too large for shared memory");
    return AIM_EINVAL;
  }
  static const cudaError_t attr =
      cudaFuncSetAttribute(fft_x<R, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  AIM_CUDA_TRY(attr);
  dim3 grid(a.rows_y, a.rows_z);
  AIM_LAUNCH(c, name, fft_x<R, MODE><<<grid, 256, sm, c->stream>>>(buf, a, ghat, tw));
  return launch_check(c, "fft_x");
}

template <typename R>
int fft_convolve(aim_ctx* c, PrecData<R>& p, int G) {
  const int nx = c->n[0], ny = c->n[1], nz = c->n[2];
  const int Lx = c->L[0], Ly = c->L[1], Lz = c->L[2];
  // z forward: grid0 [G][nz][ny][nx] -> grid1 [G][Lz][ny][nx]
  {
    StridedArgs a{};
    a.n_in = nz; a.n_out = Lz; a.X = nx; a.A = ny;
    a.sG_in = (long long)nz * ny * nx; a.sA_in = nx; a.sP_in = (long long)ny * nx;
    a.sG_out = (long long)Lz * ny * nx; a.sA_out = nx; a.sP_out = (long long)ny * nx;
    a.plan = c->plan[2];
    AIM_TRY((launch_strided<R, false>(c, "fft_z_fwd", p.grid0, p.grid1, a, G, p.tw[2])));
  }
  // y forward: grid1 [G][Lz][ny][nx] -> grid2 [G][Lz][Ly][nx]
  {
    StridedArgs a{};
    a.n_in = ny; a.n_out = Ly; a.X = nx; a.A = Lz;
    a.sG_in = (long long)Lz * ny * nx; a.sA_in = (long long)ny * nx; a.sP_in = nx;
    a.sG_out = (long long)Lz * Ly * nx; a.sA_out = (long long)Ly * nx; a.sP_out = nx;
    a.plan = c->plan[1];
    AIM_TRY((launch_strided<R, false>(c, "fft_y_fwd", p.grid1, p.grid2, a, G, p.tw[1])));
  }
  // x: forward, times Ghat, inverse, in place on grid2
  {
    XArgs a{};
    a.nx = nx; a.rows_y = Ly; a.rows_z = Lz; a.G = G;
    a.sG = (long long)Lz * Ly * nx;
    a.hx = Lx / 2 + 1; a.hy = Ly / 2 + 1; a.hz = Lz / 2 + 1;
    a.plan = c->plan[0];
    AIM_TRY((launch_x<R, 0>(c, "fft_x_conv", p.grid2, a, p.ghat, p.tw[0])));
  }
  // y inverse: grid2 -> grid1 [G][Lz][ny][nx]
  {
    StridedArgs a{};
    a.n_in = Ly; a.n_out = ny; a.X = nx; a.A = Lz;
    a.sG_in = (long long)Lz * Ly * nx; a.sA_in = (long long)Ly * nx; a.sP_in = nx;
    a.sG_out = (long long)Lz * ny * nx; a.sA_out = (long long)ny * nx; a.sP_out = nx;
    a.plan = c->plan[1];
    AIM_TRY((launch_strided<R, true>(c, "fft_y_inv", p.grid2, p.grid1, a, G, p.tw[1])));
  }
  // z inverse: grid1 -> grid0 [G][nz][ny][nx]
  {
    StridedArgs a{};
    a.n_in = Lz; a.n_out = nz; a.X = nx; a.A = ny;
    a.sG_in = (long long)Lz * ny * nx; a.sA_in = nx; a.sP_in = (long long)ny * nx;
    a.sG_out = (long long)nz * ny * nx; a.sA_out = nx; a.sP_out = (long long)ny * nx;
    a.plan = c->plan[2];
    AIM_TRY((launch_strided<R, true>(c, "fft_z_inv", p.grid1, p.grid0, a, G, p.tw[2])));
  }
  return AIM_OK;
}

template int fft_convolve<float>(aim_ctx*, PrecData<float>&, int);
template int fft_convolve<double>(aim_ctx*, PrecData<double>&, int);

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

__global__ void extract_octant(const double2* full, double2* oct64, float2* oct32, int Lx, int Ly, int Lz, double scale) {
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
  }
}

int build_ghat(aim_ctx* c) {
  const int Lx = c->L[0], Ly = c->L[1], Lz = c->L[2];
  const long long total = (long long)Lx * Ly * Lz;
  double2 *a = nullptr, *b = nullptr;
  AIM_CUDA_TRY(cudaMallocAsync(&a, total * sizeof(double2), c->stream));
  AIM_CUDA_TRY(cudaMallocAsync(&b, total * sizeof(double2), c->stream));
  AIM_LAUNCH(c, "sample_green", sample_green<<<1024, 256, 0, c->stream>>>(a, Lx, Ly, Lz, c->n[0], c->n[1], c->n[2], c->k, c->h));
  AIM_TRY(launch_check(c, "sample_green"));
  // z: full transform a -> b ; y: b -> a ; x: rows of a in place
  StridedArgs s{};
  s.n_in = Lz; s.n_out = Lz; s.X = Lx; s.A = Ly;
  s.sG_in = total; s.sA_in = Lx; s.sP_in = (long long)Ly * Lx;
  s.sG_out = total; s.sA_out = Lx; s.sP_out = (long long)Ly * Lx;
  s.plan = c->plan[2];
  AIM_TRY((launch_strided<double, false>(c, "ghat_z", a, b, s, 1, c->p64.tw[2])));
  s.n_in = Ly; s.n_out = Ly; s.X = Lx; s.A = Lz;
  s.sA_in = (long long)Ly * Lx; s.sP_in = Lx;
  s.sA_out = (long long)Ly * Lx; s.sP_out = Lx;
  s.plan = c->plan[1];
  AIM_TRY((launch_strided<double, false>(c, "ghat_y", b, a, s, 1, c->p64.tw[1])));
  XArgs x{};
  x.nx = Lx; x.rows_y = Ly; x.rows_z = Lz; x.G = 1; x.sG = total;
  x.hx = Lx / 2 + 1; x.hy = Ly / 2 + 1; x.hz = Lz / 2 + 1;
  x.plan = c->plan[0];
  AIM_TRY((launch_x<double, 1>(c, "ghat_x", a, x, nullptr, c->p64.tw[0])));
  AIM_LAUNCH(c, "extract_octant", extract_octant<<<1024, 256, 0, c->stream>>>(a, c->p64.ghat, c->p32.ghat, Lx, Ly, Lz, 1.0 / (double)total));
  AIM_TRY(launch_check(c, "extract_octant"));
  AIM_CUDA_TRY(cudaFreeAsync(a, c->stream));
  AIM_CUDA_TRY(cudaFreeAsync(b, c->stream));
  return AIM_OK;
}

}  // namespace aim
