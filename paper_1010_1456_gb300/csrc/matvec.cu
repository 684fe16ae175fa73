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
// reduce with warp shuffles.  FP32 (complex64) or FP64 (complex128) end to
// end, accumulating in the same precision.
#include "common.h"
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

template <typename R>
__global__ void __launch_bounds__(256) proj_gather(const cplx<R>* __restrict__ x, cplx<R>* __restrict__ Q,
                                                   const int32_t* __restrict__ ptr, const int32_t* __restrict__ mm,
                                                   const R* __restrict__ w, int N, long long Nc, int nrhs) {
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < Nc; u += (long long)gridDim.x * blockDim.x) {
    const int e0 = ptr[u], e1 = ptr[u + 1];
    for (int b = 0; b < nrhs; ++b) {
      cplx<R> a0 = cmake<cplx<R>>(0, 0), a1 = a0, a2 = a0, a3 = a0;
      const cplx<R>* xb = x + (long long)b * N;
      for (int e = e0; e < e1; ++e) {
        const W4<R> ww = load_w4(w, e);
        const cplx<R> xv = xb[mm[e]];
        a0.x += ww.x * xv.x; a0.y += ww.x * xv.y;
        a1.x += ww.y * xv.x; a1.y += ww.y * xv.y;
        a2.x += ww.z * xv.x; a2.y += ww.z * xv.y;
        a3.x += ww.w * xv.x; a3.y += ww.w * xv.y;
      }
      cplx<R>* Qb = Q + (long long)b * 4 * Nc;
      Qb[u] = a0;
      Qb[Nc + u] = a1;
      Qb[2 * Nc + u] = a2;
      Qb[3 * Nc + u] = a3;
    }
  }
}

// 8 lanes per basis function.
template <typename R, int M>
__global__ void __launch_bounds__(256) interp_near(const cplx<R>* __restrict__ Phi, const cplx<R>* __restrict__ x,
                                                   cplx<R>* __restrict__ y, const R* __restrict__ lam,
                                                   const int32_t* __restrict__ base, const int32_t* __restrict__ nptr,
                                                   const int32_t* __restrict__ ncol, const cplx<R>* __restrict__ nval,
                                                   int N, long long Nc, int nx, int ny, int nrhs, R fvec, R frho) {
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
    const cplx<R>* Pb = Phi + (long long)b * 4 * Nc;
    cplx<R> av = cmake<cplx<R>>(0, 0), ar = av, an = av;
    for (int s = lane; s < S; s += 8) {
      const int i = s % P, j = (s / P) % P, kk = s / (P * P);
      const long long node = b0 + ((long long)kk * ny + j) * nx + i;
      const cplx<R> px = Pb[node], py = Pb[Nc + node], pz = Pb[2 * Nc + node], pr = Pb[3 * Nc + node];
      const R wx = lm[s], wy = lm[S + s], wz = lm[2 * S + s], wr = lm[3 * S + s];
      av.x += wx * px.x + wy * py.x + wz * pz.x;
      av.y += wx * px.y + wy * py.y + wz * pz.y;
      ar.x += wr * pr.x;
      ar.y += wr * pr.y;
    }
    const cplx<R>* xb = x + (long long)b * N;
    for (int e = r0 + lane; e < r1; e += 8) {
      const cplx<R> v = nval[e], xv = xb[ncol[e]];
      an.x += v.x * xv.x - v.y * xv.y;
      an.y += v.x * xv.y + v.y * xv.x;
    }
    // grid part: j (fvec av - frho ar)  with fvec = k eta, frho = eta / k
    cplx<R> t;
    t.x = fvec * av.x - frho * ar.x;
    t.y = fvec * av.y - frho * ar.y;
    cplx<R> out;
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

template <typename R> static PrecData<R>& prec(aim_ctx* c);
template <> PrecData<float>& prec<float>(aim_ctx* c) { return c->p32; }
template <> PrecData<double>& prec<double>(aim_ctx* c) { return c->p64; }

template <typename R>
int matvec(aim_ctx* c, const cplx<R>* x, cplx<R>* y, int nrhs) {
  PrecData<R>& p = prec<R>(c);
  const long long Nc = (long long)c->n[0] * c->n[1] * c->n[2];
  {
    int blocks = (int)std::min<long long>((Nc + 255) / 256, 152LL * 16);
    AIM_LAUNCH(c, "proj_gather", proj_gather<R><<<blocks, 256, 0, c->stream>>>(x, p.grid0, c->pnode_ptr, c->pnode_m, p.pnode_w, c->N, Nc, nrhs));
    AIM_TRY(launch_check(c, "proj_gather"));
  }
  AIM_TRY(fft_convolve<R>(c, p, 4 * nrhs));
  {
    long long threads = (long long)c->N * 8;
    int blocks = (int)((threads + 255) / 256);
    const R fvec = (R)(c->k * kEta0), frho = (R)(kEta0 / c->k);
    switch (c->M) {
      case 1:
        AIM_LAUNCH(c, "interp_near", interp_near<R, 1><<<blocks, 256, 0, c->stream>>>(p.grid0, x, y, p.lam, c->base, c->near_ptr, c->near_col,
                                                         p.near_val, c->N, Nc, c->n[0], c->n[1], nrhs, fvec, frho));
        break;
      case 2:
        AIM_LAUNCH(c, "interp_near", interp_near<R, 2><<<blocks, 256, 0, c->stream>>>(p.grid0, x, y, p.lam, c->base, c->near_ptr, c->near_col,
                                                         p.near_val, c->N, Nc, c->n[0], c->n[1], nrhs, fvec, frho));
        break;
      default:
        AIM_LAUNCH(c, "interp_near", interp_near<R, 3><<<blocks, 256, 0, c->stream>>>(p.grid0, x, y, p.lam, c->base, c->near_ptr, c->near_col,
                                                         p.near_val, c->N, Nc, c->n[0], c->n[1], nrhs, fvec, frho));
        break;
    }
    AIM_TRY(launch_check(c, "interp_near"));
  }
  return AIM_OK;
}

template int matvec<float>(aim_ctx*, const float2*, float2*, int);
template int matvec<double>(aim_ctx*, const double2*, double2*, int);

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
