// AIM matrix-vector product: projection, FFT convolution, interpolation and
// near-zone correction (paper Section 4.1 propagation step and footnote 2;
// Section 2.2 near-zone correction with gamma = 3).
//
//   Q_c(u) = sum_m Lambda^c_m(u - a_m) x_m                       (projection)
//   Phi_c  = G_h * Q_c                                             (fft.cu)
//   y_m    = j k eta [ sum_{c=x,y,z} <Lambda^c_m, Phi_c> - k^-2 <Lambda^rho_m, Phi_rho> ]
//            + sum_n Znear_mn x_n                                  (interpolation + near)
//
// The projection is a gather over each grid node's list of (basis, weight)
// entries, built at setup, so it needs no atomics and is deterministic.  The
// interpolation and the near row of a basis function are handled by one
// 8-lane group: the lanes split the stencil nodes and the near entries and
// reduce with warp shuffles.
//
// Modes: M32 (complex64, FP32 accumulation), M64 (complex128 throughout) and
// MFF (complex128 vectors, FP64 weights and accumulation, grids stored as
// float-float for the FFT passes).
#include <algorithm>

#include "common.h"
#include "ff.h"
#include "geom.h"

namespace aim {

int launch_check(aim_ctx* c, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return AIM_ECUDA;
  }
  return AIM_OK;
}

struct M32 {
  using R = float;
  using S = float2;
  __device__ static S put(float2 v) { return v; }
  __device__ static float2 get(const S& s) { return s; }
};
struct M64 {
  using R = double;
  using S = double2;
  __device__ static S put(double2 v) { return v; }
  __device__ static double2 get(const S& s) { return s; }
};
struct MFF {
  using R = double;
  using S = float4;
  __device__ static S put(double2 v) {
    const ff re = ff_from_double(v.x), im = ff_from_double(v.y);
    return make_float4(re.hi, re.lo, im.hi, im.lo);
  }
  __device__ static double2 get(const S& s) {
    return make_double2((double)s.x + (double)s.y, (double)s.z + (double)s.w);
  }
};

// Four projection weights of one entry (x, y, z, charge).
template <typename R> struct W4 {
  R x, y, z, w;
};
__device__ __forceinline__ W4<float> load_w4(const float* p, int e) {
  const float4 v = reinterpret_cast<const float4*>(p)[e];
  return W4<float>{v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ W4<double> load_w4(const double* p, int e) {
  const double2 a = reinterpret_cast<const double2*>(p)[2 * e];
  const double2 b = reinterpret_cast<const double2*>(p)[2 * e + 1];
  return W4<double>{a.x, a.y, b.x, b.y};
}

// 4 lanes per grid node: the lanes take every fourth entry of the node's list
// (adjacent lanes read adjacent entries) and combine with warp shuffles.
template <class MD>
__global__ void __launch_bounds__(256) proj_gather(const cplx<typename MD::R>* __restrict__ x, typename MD::S* __restrict__ Q,
                                                   const int32_t* __restrict__ ptr, const int32_t* __restrict__ mm,
                                                   const typename MD::R* __restrict__ w, int N, long long Nc, int nrhs) {
  using R = typename MD::R;
  using C = cplx<R>;
  const int lane = threadIdx.x & 3;
  const long long stride = ((long long)gridDim.x * blockDim.x) >> 2;
  for (long long u0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 2;; u0 += stride) {
    // the warp leaves together, so every lane takes part in the shuffles below
    const bool live = u0 < Nc;
    if (!__any_sync(0xffffffffu, live)) break;
    const long long u = live ? u0 : Nc - 1;
    const int e0 = ptr[u], e1 = ptr[u + 1];
    for (int b = 0; b < nrhs; ++b) {
      C a0 = cmake<C>(0, 0), a1 = a0, a2 = a0, a3 = a0;
      const C* xb = x + (long long)b * N;
      for (int e = e0 + lane; e < e1; e += 4) {
        const W4<R> ww = load_w4(w, e);
        const C xv = xb[mm[e]];
        a0.x += ww.x * xv.x; a0.y += ww.x * xv.y;
        a1.x += ww.y * xv.x; a1.y += ww.y * xv.y;
        a2.x += ww.z * xv.x; a2.y += ww.z * xv.y;
        a3.x += ww.w * xv.x; a3.y += ww.w * xv.y;
      }
#pragma unroll
      for (int o = 1; o < 4; o <<= 1) {
        a0.x += __shfl_xor_sync(0xffffffffu, a0.x, o, 4); a0.y += __shfl_xor_sync(0xffffffffu, a0.y, o, 4);
        a1.x += __shfl_xor_sync(0xffffffffu, a1.x, o, 4); a1.y += __shfl_xor_sync(0xffffffffu, a1.y, o, 4);
        a2.x += __shfl_xor_sync(0xffffffffu, a2.x, o, 4); a2.y += __shfl_xor_sync(0xffffffffu, a2.y, o, 4);
        a3.x += __shfl_xor_sync(0xffffffffu, a3.x, o, 4); a3.y += __shfl_xor_sync(0xffffffffu, a3.y, o, 4);
      }
      if (live) {
        typename MD::S* Qb = Q + (long long)b * 4 * Nc;
        // lane c writes component c (one conversion per value)
        const C val = lane == 0 ? a0 : lane == 1 ? a1 : lane == 2 ? a2 : a3;
        Qb[(long long)lane * Nc + u] = MD::put(val);
      }
    }
  }
}

// 8 lanes per basis function.
template <class MD, int M>
__global__ void __launch_bounds__(256) interp_near(const typename MD::S* __restrict__ Phi,
                                                   const cplx<typename MD::R>* __restrict__ x,
                                                   cplx<typename MD::R>* __restrict__ y,
                                                   const typename MD::R* __restrict__ lam,
                                                   const int32_t* __restrict__ base, const int32_t* __restrict__ nptr,
                                                   const int32_t* __restrict__ ncol,
                                                   const cplx<typename MD::R>* __restrict__ nval, int N, long long Nc,
                                                   int nx, int ny, int nrhs, typename MD::R fvec, typename MD::R frho) {
  using R = typename MD::R;
  using C = cplx<R>;
  constexpr int P = M + 1;
  constexpr int S = P * P * P;
  const int lane = threadIdx.x & 7;
  const int m = (blockIdx.x * blockDim.x + threadIdx.x) >> 3;
  const bool live = m < N;
  const int mm = live ? m : N - 1;
  const int b0 = base[mm];
  const R* lm = lam + (long long)mm * 4 * S;
  const int r0 = nptr[mm], r1 = nptr[mm + 1];
  for (int b = 0; b < nrhs; ++b) {
    const typename MD::S* Pb = Phi + (long long)b * 4 * Nc;
    C av = cmake<C>(0, 0), ar = av, an = av;
    for (int s = lane; s < S; s += 8) {
      const int i = s % P, j = (s / P) % P, kk = s / (P * P);
      const long long node = b0 + ((long long)kk * ny + j) * nx + i;
      const C px = MD::get(Pb[node]), py = MD::get(Pb[Nc + node]), pz = MD::get(Pb[2 * Nc + node]),
              pr = MD::get(Pb[3 * Nc + node]);
      const R wx = lm[s], wy = lm[S + s], wz = lm[2 * S + s], wr = lm[3 * S + s];
      av.x += wx * px.x + wy * py.x + wz * pz.x;
      av.y += wx * px.y + wy * py.y + wz * pz.y;
      ar.x += wr * pr.x;
      ar.y += wr * pr.y;
    }
    const C* xb = x + (long long)b * N;
    for (int e = r0 + lane; e < r1; e += 8) {
      const C v = nval[e], xv = xb[ncol[e]];
      an.x += v.x * xv.x - v.y * xv.y;
      an.y += v.x * xv.y + v.y * xv.x;
    }
    // grid part: j (fvec av - frho ar)  with fvec = k eta, frho = eta / k
    C t;
    t.x = fvec * av.x - frho * ar.x;
    t.y = fvec * av.y - frho * ar.y;
    C out;
    out.x = an.x - t.y;
    out.y = an.y + t.x;
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
      out.x += __shfl_xor_sync(0xffffffffu, out.x, o, 8);
      out.y += __shfl_xor_sync(0xffffffffu, out.y, o, 8);
    }
    if (live && lane == 0) y[(long long)b * N + m] = out;
  }
}

// MD: storage of the projected grid; MI: storage of Phi read by the interpolation.
template <class MD, class MI>
static int run_product(aim_ctx* c, const cplx<typename MD::R>* x, cplx<typename MD::R>* y, int nrhs,
                       typename MD::S* grid0, const typename MI::S* phi, const typename MD::R* pw,
                       const typename MD::R* lam, const cplx<typename MD::R>* nval, int (*convolve)(aim_ctx*, int)) {
  using R = typename MD::R;
  const long long Nc = (long long)c->n[0] * c->n[1] * c->n[2];
  {
    const int blocks = (int)std::min<long long>((4 * Nc + 255) / 256, 152LL * 16);
    AIM_LAUNCH(c, "proj_gather",
               proj_gather<MD><<<blocks, 256, 0, c->stream>>>(x, grid0, c->pnode_ptr, c->pnode_m, pw, c->N, Nc, nrhs));
    AIM_TRY(launch_check(c, "proj_gather"));
  }
  AIM_TRY(convolve(c, 4 * nrhs));
  {
    const long long threads = (long long)c->N * 8;
    const int blocks = (int)((threads + 255) / 256);
    const R fvec = (R)(c->k * kEta0), frho = (R)(kEta0 / c->k);
#define AIM_INTERP(MM)                                                                                          \
  AIM_LAUNCH(c, "interp_near",                                                                                  \
             (interp_near<MI, MM><<<blocks, 256, 0, c->stream>>>(phi, x, y, lam, c->base, c->near_ptr,          \
                                                                 c->near_col, nval, c->N, Nc, c->n[0], c->n[1], \
                                                                 nrhs, fvec, frho)))
    switch (c->M) {
      case 1: AIM_INTERP(1); break;
      case 2: AIM_INTERP(2); break;
      default: AIM_INTERP(3); break;
    }
#undef AIM_INTERP
    AIM_TRY(launch_check(c, "interp_near"));
  }
  return AIM_OK;
}

int ensure_grids(aim_ctx* c, int precision) {
  const long long B = c->max_rhs;
  const long long nx = c->n[0], ny = c->n[1], nz = c->n[2], Ly = c->L[1], Lz = c->L[2];
  const long long e0 = B * 4 * nz * ny * nx, e1 = B * 4 * Lz * ny * nx, e2 = B * 4 * Lz * Ly * nx;
  if (precision == AIM_C64) {
    PrecData<float>& p = c->p32;
    if (!p.grid0) {
      AIM_CUDA_TRY(cudaMalloc(&p.grid0, sizeof(float2) * e0));
      AIM_CUDA_TRY(cudaMalloc(&p.grid1, sizeof(float2) * e1));
      AIM_CUDA_TRY(cudaMalloc(&p.grid2, sizeof(float2) * e2));
    }
  } else if (precision == AIM_C128_F64) {
    PrecData<double>& p = c->p64;
    if (!p.grid0) {
      AIM_CUDA_TRY(cudaMalloc(&p.grid0, sizeof(double2) * e0));
      AIM_CUDA_TRY(cudaMalloc(&p.grid1, sizeof(double2) * e1));
      AIM_CUDA_TRY(cudaMalloc(&p.grid2, sizeof(double2) * e2));
    }
  } else {
    FFData& p = c->pff;
    if (!p.grid0) {
      AIM_CUDA_TRY(cudaMalloc(&p.grid0, sizeof(float4) * e0));
      AIM_CUDA_TRY(cudaMalloc(&p.grid1, sizeof(float4) * e1));
      AIM_CUDA_TRY(cudaMalloc(&p.grid2, sizeof(float4) * e2));
      AIM_CUDA_TRY(cudaMalloc(&p.phi64, sizeof(double2) * e0));
    }
  }
  return AIM_OK;
}

int matvec(aim_ctx* c, const void* x, void* y, int nrhs, int precision) {
  AIM_TRY(ensure_grids(c, precision));
  if (precision == AIM_C64)
    return run_product<M32, M32>(c, (const float2*)x, (float2*)y, nrhs, c->p32.grid0, c->p32.grid0, c->p32.pnode_w,
                                 c->p32.lam, c->p32.near_val, fft_convolve_c64);
  if (precision == AIM_C128_F64)
    return run_product<M64, M64>(c, (const double2*)x, (double2*)y, nrhs, c->p64.grid0, c->p64.grid0,
                                 c->p64.pnode_w, c->p64.lam, c->p64.near_val, fft_convolve_c128);
  return run_product<MFF, M64>(c, (const double2*)x, (double2*)y, nrhs, c->pff.grid0, c->pff.phi64, c->p64.pnode_w,
                               c->p64.lam, c->p64.near_val, fft_convolve_ff);
}

__global__ void k_c128_to_c64(const double2* __restrict__ in, float2* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = make_float2((float)in[i].x, (float)in[i].y);
}
__global__ void k_c64_to_c128(const float2* __restrict__ in, double2* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = make_double2((double)in[i].x, (double)in[i].y);
}

int convert_c128_to_c64(aim_ctx* c, const double2* in, float2* out, int64_t count) {
  int blocks = (int)std::min<long long>((count + 255) / 256, 152LL * 8);
  AIM_LAUNCH(c, "k_c128_to_c64", k_c128_to_c64<<<blocks, 256, 0, c->stream>>>(in, out, count));
  return launch_check(c, "c128_to_c64");
}
int convert_c64_to_c128(aim_ctx* c, const float2* in, double2* out, int64_t count) {
  int blocks = (int)std::min<long long>((count + 255) / 256, 152LL * 8);
  AIM_LAUNCH(c, "k_c64_to_c128", k_c64_to_c128<<<blocks, 256, 0, c->stream>>>(in, out, count));
  return launch_check(c, "c64_to_c128");
}

}  // namespace aim

namespace aim {
// The complex64 product on caller-provided grids g0 [B][4][nz][ny][nx],
// g1 [B][4][Lz][ny][nx], g2 [B][4][Lz][Ly][nx]: the launches of the
// complex64 path of matvec() without its grid allocation.
int matvec_c64_bufs(aim_ctx* c, const float2* x, float2* y, int nrhs, float2* g0, float2* g1, float2* g2) {
  const long long Nc = (long long)c->n[0] * c->n[1] * c->n[2];
  {
    const int blocks = (int)std::min<long long>((Nc + 255) / 256, 152LL * 16);
    AIM_LAUNCH(c, "proj_gather",
               proj_gather<M32><<<blocks, 256, 0, c->stream>>>(x, g0, c->pnode_ptr, c->pnode_m, c->p32.pnode_w, c->N,
                                                              Nc, nrhs));
    AIM_TRY(launch_check(c, "proj_gather"));
  }
  AIM_TRY(fft_convolve_c64_bufs(c, 4 * nrhs, g0, g1, g2));
  {
    const long long threads = (long long)c->N * 8;
    const int blocks = (int)((threads + 255) / 256);
    const float fvec = (float)(c->k * kEta0), frho = (float)(kEta0 / c->k);
#define AIM_INTERP32(MM)                                                                                      \
  AIM_LAUNCH(c, "interp_near",                                                                                \
             (interp_near<M32, MM><<<blocks, 256, 0, c->stream>>>(g0, x, y, c->p32.lam, c->base, c->near_ptr, \
                                                                  c->near_col, c->p32.near_val, c->N, Nc,     \
                                                                  c->n[0], c->n[1], nrhs, fvec, frho)))
    switch (c->M) {
      case 1: AIM_INTERP32(1); break;
      case 2: AIM_INTERP32(2); break;
      default: AIM_INTERP32(3); break;
    }
#undef AIM_INTERP32
    AIM_TRY(launch_check(c, "interp_near"));
  }
  return AIM_OK;
}
}  // namespace aim
