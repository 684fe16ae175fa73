// Batched right-preconditioned restarted GMRES(m) on the device.
//
// Paper Section 2.2: diagonal preconditioner, iteration stopped on the
// relative residual.  All right-hand sides advance in lockstep; each keeps
// its own Arnoldi basis, Hessenberg matrix and Givens rotations.  Dot
// products, norms and rotations are FP64 (two-level block reductions, so the
// results do not depend on launch timing).  Orthogonalisation is classical
// Gram-Schmidt with one re-orthogonalisation (CGS2).  The Arnoldi product is
// complex64 or complex128 (aim_opts.precision); every restart recomputes the
// true residual V - Z~ X with the complex128 product, so the complex64 mode
// is FP64 iterative refinement wrapped around a complex64 inner solve.
#include <algorithm>
#include <cmath>

#include "common.h"

namespace aim {

constexpr int kDotGroup = 8;  // basis vectors per pass of the dot kernel

__device__ __forceinline__ double2 cfma_conj(double2 a, double2 b, double2 acc) {
  // acc + conj(a) * b
  acc.x += a.x * b.x + a.y * b.y;
  acc.y += a.x * b.y - a.y * b.x;
  return acc;
}

template <int NV>
__device__ __forceinline__ void block_reduce_store(double2* v, double2* out, int stride) {
  __shared__ double2 red[32][kDotGroup];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i)
    for (int o = 16; o > 0; o >>= 1) {
      v[i].x += __shfl_xor_sync(0xffffffffu, v[i].x, o);
      v[i].y += __shfl_xor_sync(0xffffffffu, v[i].y, o);
    }
  if (lane == 0)
    for (int i = 0; i < NV; ++i) red[warp][i] = v[i];
  __syncthreads();
  if (threadIdx.x < NV) {
    double2 s = make_double2(0, 0);
    for (int w = 0; w < nw; ++w) {
      s.x += red[w][threadIdx.x].x;
      s.y += red[w][threadIdx.x].y;
    }
    out[threadIdx.x * stride] = s;
  }
  __syncthreads();
}

// partial[b][blk][i] = sum over this block's chunk of conj(V[b][i]) . w[b], i in [0, nvec)
__global__ void k_dots(const double2* __restrict__ V, const double2* __restrict__ w, double2* __restrict__ partial,
                       int N, int nvec, int ldv_vec, int nblk, int ldp) {
  const int b = blockIdx.y, blk = blockIdx.x;
  const double2* Vb = V + (long long)b * ldv_vec * N;
  const double2* wb = w + (long long)b * N;
  const int chunk = (N + nblk - 1) / nblk;
  const int n0 = blk * chunk, n1 = min(N, n0 + chunk);
  double2* pout = partial + ((long long)b * nblk + blk) * ldp;
  for (int i0 = 0; i0 < nvec; i0 += kDotGroup) {
    double2 acc[kDotGroup];
#pragma unroll
    for (int i = 0; i < kDotGroup; ++i) acc[i] = make_double2(0, 0);
    const int ni = min(kDotGroup, nvec - i0);
    for (int n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
      const double2 wv = wb[n];
#pragma unroll
      for (int i = 0; i < kDotGroup; ++i)
        if (i < ni) acc[i] = cfma_conj(Vb[(long long)(i0 + i) * N + n], wv, acc[i]);
    }
    block_reduce_store<kDotGroup>(acc, pout + i0, 1);
  }
}

// hcol[b][i] = sum_blk partial; H[b][i][j] (+)= hcol (accumulate when add != 0)
__global__ void k_dots_reduce(const double2* __restrict__ partial, double2* __restrict__ hcol, double2* __restrict__ H,
                              int nvec, int nblk, int ldp, int m, int j, int add) {
  const int b = blockIdx.x;
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
    double2 s = make_double2(0, 0);
    for (int blk = 0; blk < nblk; ++blk) {
      const double2 p = partial[((long long)b * nblk + blk) * ldp + i];
      s.x += p.x;
      s.y += p.y;
    }
    hcol[(long long)b * (m + 1) + i] = s;
    double2* h = H + ((long long)b * (m + 1) + i) * m + j;
    if (add) {
      h->x += s.x;
      h->y += s.y;
    } else {
      *h = s;
    }
  }
}

// w[b] -= sum_i hcol[b][i] V[b][i]
__global__ void k_update(const double2* __restrict__ V, double2* __restrict__ w, const double2* __restrict__ hcol,
                         int N, int nvec, int ldv_vec, int m) {
  __shared__ double2 hs[256];
  const int b = blockIdx.y;
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) hs[i] = hcol[(long long)b * (m + 1) + i];
  __syncthreads();
  const double2* Vb = V + (long long)b * ldv_vec * N;
  double2* wb = w + (long long)b * N;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
    double2 acc = wb[n];
    for (int i = 0; i < nvec; ++i) {
      const double2 v = Vb[(long long)i * N + n], h = hs[i];
      acc.x -= h.x * v.x - h.y * v.y;
      acc.y -= h.x * v.y + h.y * v.x;
    }
    wb[n] = acc;
  }
}

// partial[b][blk] = sum |x|^2 over the block's chunk
__global__ void k_norm2(const double2* __restrict__ x, double* __restrict__ partial, int N, long long ldx, int nblk) {
  const int b = blockIdx.y, blk = blockIdx.x;
  const double2* xb = x + (long long)b * ldx;
  const int chunk = (N + nblk - 1) / nblk;
  const int n0 = blk * chunk, n1 = min(N, n0 + chunk);
  double s = 0.0;
  for (int n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
    const double2 v = xb[n];
    s += v.x * v.x + v.y * v.y;
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    partial[(long long)b * nblk + blk] = t;
  }
}
// out[b] = sqrt(sum partial)  (one thread per rhs)
__global__ void k_sqrt_sum(const double* __restrict__ partial, double* __restrict__ out, int nblk, int nrhs) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nrhs) return;
  double s = 0.0;
  for (int blk = 0; blk < nblk; ++blk) s += partial[(long long)b * nblk + blk];
  out[b] = sqrt(s);
}

// dst[b] = src[b] * (1 / nrm[b])
__global__ void k_scale(const double2* __restrict__ src, double2* __restrict__ dst, const double* __restrict__ nrm,
                        int N, long long lds, long long ldd) {
  const int b = blockIdx.y;
  const double s = nrm[b] > 0.0 ? 1.0 / nrm[b] : 0.0;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
    double2 v = src[(long long)b * lds + n];
    v.x *= s;
    v.y *= s;
    dst[(long long)b * ldd + n] = v;
  }
}

// z = dinv .* v, in precision R
template <typename R>
__global__ void k_precond(const double2* __restrict__ v, const double2* __restrict__ dinv, cplx<R>* __restrict__ z,
                          int N, long long ldv) {
  const int b = blockIdx.y;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
    const double2 a = v[(long long)b * ldv + n], d = dinv[n];
    z[(long long)b * N + n] = cmake<cplx<R>>(a.x * d.x - a.y * d.y, a.x * d.y + a.y * d.x);
  }
}

// r = V - y (masked: inactive right-hand sides get r = 0)
__global__ void k_residual(const double2* __restrict__ Vrhs, const double2* __restrict__ y, double2* __restrict__ r,
                           int N, const int* __restrict__ active) {
  const int b = blockIdx.y;
  const bool on = active[b] != 0;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
    const long long i = (long long)b * N + n;
    double2 v = Vrhs[i], t = y[i];
    r[i] = on ? make_double2(v.x - t.x, v.y - t.y) : make_double2(0, 0);
  }
}

// Givens step for column j, one thread per rhs.  Rotation
// [[conj(c), conj(s)], [-s, c]], c = a/d, s = b/d maps (a, b) to (d, 0).
__global__ void k_givens(double2* __restrict__ H, double2* __restrict__ cs, double2* __restrict__ sn,
                         double2* __restrict__ g, const double* __restrict__ hnext, const double* __restrict__ bnorm,
                         double* __restrict__ est, int m, int j, int nrhs) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nrhs) return;
  double2* Hb = H + (long long)b * (m + 1) * m;
  double2* cb = cs + (long long)b * m;
  double2* sb = sn + (long long)b * m;
  double2* gb = g + (long long)b * (m + 1);
  Hb[(long long)(j + 1) * m + j] = make_double2(hnext[b], 0.0);
  for (int i = 0; i < j; ++i) {
    const double2 c = cb[i], s = sb[i];
    const double2 hi = Hb[(long long)i * m + j], hn = Hb[(long long)(i + 1) * m + j];
    double2 t, u;
    t.x = (c.x * hi.x + c.y * hi.y) + (s.x * hn.x + s.y * hn.y);
    t.y = (c.x * hi.y - c.y * hi.x) + (s.x * hn.y - s.y * hn.x);
    u.x = -(s.x * hi.x - s.y * hi.y) + (c.x * hn.x - c.y * hn.y);
    u.y = -(s.x * hi.y + s.y * hi.x) + (c.x * hn.y + c.y * hn.x);
    Hb[(long long)i * m + j] = t;
    Hb[(long long)(i + 1) * m + j] = u;
  }
  const double2 a = Hb[(long long)j * m + j], bb = Hb[(long long)(j + 1) * m + j];
  const double d = sqrt(a.x * a.x + a.y * a.y + bb.x * bb.x + bb.y * bb.y);
  double2 c = make_double2(1.0, 0.0), s = make_double2(0.0, 0.0);
  if (d > 0.0) {
    c = make_double2(a.x / d, a.y / d);
    s = make_double2(bb.x / d, bb.y / d);
  }
  cb[j] = c;
  sb[j] = s;
  Hb[(long long)j * m + j] = make_double2(d, 0.0);
  Hb[(long long)(j + 1) * m + j] = make_double2(0.0, 0.0);
  const double2 gj = gb[j];
  gb[j + 1] = make_double2(-(s.x * gj.x - s.y * gj.y), -(s.x * gj.y + s.y * gj.x));
  gb[j] = make_double2(c.x * gj.x + c.y * gj.y, c.x * gj.y - c.y * gj.x);
  const double2 r = gb[j + 1];
  est[b] = bnorm[b] > 0.0 ? sqrt(r.x * r.x + r.y * r.y) / bnorm[b] : 0.0;
}

// g = (beta, 0, ...), one thread per rhs
__global__ void k_ginit(double2* __restrict__ g, const double* __restrict__ beta, int m, int nrhs) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nrhs) return;
  for (int i = 0; i <= m; ++i) g[(long long)b * (m + 1) + i] = make_double2(i == 0 ? beta[b] : 0.0, 0.0);
}

// back substitution H y = g on the leading kk x kk block, one thread per rhs
__global__ void k_backsolve(const double2* __restrict__ H, const double2* __restrict__ g, double2* __restrict__ y,
                            int m, int kk, int nrhs) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nrhs) return;
  const double2* Hb = H + (long long)b * (m + 1) * m;
  const double2* gb = g + (long long)b * (m + 1);
  double2* yb = y + (long long)b * m;
  for (int i = kk - 1; i >= 0; --i) {
    double2 s = gb[i];
    for (int l = i + 1; l < kk; ++l) {
      const double2 h = Hb[(long long)i * m + l], yl = yb[l];
      s.x -= h.x * yl.x - h.y * yl.y;
      s.y -= h.x * yl.y + h.y * yl.x;
    }
    const double2 d = Hb[(long long)i * m + i];
    const double dd = d.x * d.x + d.y * d.y;
    yb[i] = dd > 0.0 ? make_double2((s.x * d.x + s.y * d.y) / dd, (s.y * d.x - s.x * d.y) / dd) : make_double2(0, 0);
  }
}

// X[b] += dinv .* (sum_i y_i V_i)   (active right-hand sides only)
__global__ void k_xupdate(const double2* __restrict__ V, const double2* __restrict__ y, const double2* __restrict__ dinv,
                          double2* __restrict__ X, int N, int kk, int m, int ldv_vec, const int* __restrict__ active) {
  __shared__ double2 ys[256];
  const int b = blockIdx.y;
  if (!active[b]) return;
  for (int i = threadIdx.x; i < kk; i += blockDim.x) ys[i] = y[(long long)b * m + i];
  __syncthreads();
  const double2* Vb = V + (long long)b * ldv_vec * N;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
    double2 s = make_double2(0, 0);
    for (int i = 0; i < kk; ++i) {
      const double2 v = Vb[(long long)i * N + n], t = ys[i];
      s.x += t.x * v.x - t.y * v.y;
      s.y += t.x * v.y + t.y * v.x;
    }
    const double2 d = dinv[n];
    double2& x = X[(long long)b * N + n];
    x.x += s.x * d.x - s.y * d.y;
    x.y += s.x * d.y + s.y * d.x;
  }
}

// ------------------------------------------------------------------ host driver
int alloc_krylov(aim_ctx* c) {
  KrylovWork& k = c->kw;
  if (k.V) return AIM_OK;
  const int B = c->max_rhs, m = c->opts.restart, N = c->N;
  k.m = m;
  // about four blocks per SM over all right-hand sides, at least 256 elements per block
  k.nblk = std::max(1, std::min((4 * 152 + B - 1) / B, (N + 255) / 256));
  const size_t vec = (size_t)N * sizeof(double2);
  AIM_CUDA_TRY(cudaMalloc(&k.V, vec * B * (m + 1)));
  AIM_CUDA_TRY(cudaMalloc(&k.w, vec * B));
  AIM_CUDA_TRY(cudaMalloc(&k.r, vec * B));
  AIM_CUDA_TRY(cudaMalloc(&k.H, sizeof(double2) * B * (m + 1) * m));
  AIM_CUDA_TRY(cudaMalloc(&k.hcol, sizeof(double2) * B * (m + 1)));
  AIM_CUDA_TRY(cudaMalloc(&k.partial, sizeof(double2) * B * k.nblk * (m + 1 + kDotGroup)));
  AIM_CUDA_TRY(cudaMalloc(&k.cs, sizeof(double2) * B * m));
  AIM_CUDA_TRY(cudaMalloc(&k.sn, sizeof(double2) * B * m));
  AIM_CUDA_TRY(cudaMalloc(&k.g, sizeof(double2) * B * (m + 1)));
  AIM_CUDA_TRY(cudaMalloc(&k.y, sizeof(double2) * B * m));
  AIM_CUDA_TRY(cudaMalloc(&k.nrm, sizeof(double) * B * (2 + k.nblk)));
  AIM_CUDA_TRY(cudaMalloc(&k.bnorm, sizeof(double) * B));
  AIM_CUDA_TRY(cudaMalloc(&k.active, sizeof(int) * B));
  AIM_CUDA_TRY(cudaMallocHost(&k.h_est, sizeof(double) * B));
  return AIM_OK;
}

void free_krylov(aim_ctx* c) {
  KrylovWork& k = c->kw;
  cudaFree(k.V); cudaFree(k.w); cudaFree(k.r); cudaFree(k.H); cudaFree(k.hcol); cudaFree(k.partial);
  cudaFree(k.cs); cudaFree(k.sn); cudaFree(k.g); cudaFree(k.y); cudaFree(k.nrm); cudaFree(k.bnorm);
  cudaFree(k.active);
  if (k.h_est) cudaFreeHost(k.h_est);
  k = KrylovWork{};
}

namespace {
struct Solver {
  aim_ctx* c;
  KrylovWork& k;
  int B, N, m;
  cudaStream_t st;
  double* est;       // device [B]
  double* npart;     // device [B][nblk]
  Solver(aim_ctx* cc, int nrhs) : c(cc), k(cc->kw), B(nrhs), N(cc->N), m(cc->kw.m), st(cc->stream) {
    est = k.nrm + B;
    npart = k.nrm + 2 * B;
  }
  dim3 vgrid() const { return dim3((unsigned)std::min(1024, std::max(1, (N + 255) / 256)), B); }
  int chk(const char* w) { return launch_check(c, w); }

  int norms(const double2* x, long long ldx, double* out) {
    AIM_LAUNCH(c, "k_norm2", k_norm2<<<dim3(k.nblk, B), 256, 0, st>>>(x, npart, N, ldx, k.nblk));
    AIM_TRY(chk("k_norm2"));
    AIM_LAUNCH(c, "k_sqrt_sum", k_sqrt_sum<<<(B + 127) / 128, 128, 0, st>>>(npart, out, k.nblk, B));
    return chk("k_sqrt_sum");
  }
  double2* Vcol(int i) { return k.V + (size_t)i * N; }  // basis i of rhs 0; rhs stride (m+1) N
  long long ldV() const { return (long long)(m + 1) * N; }

  // w = Z~ (dinv .* v_j) in the requested precision
  int apply(int j, int precision) {
    if (precision == AIM_C64) {
      AIM_LAUNCH(c, "k_precond", k_precond<float><<<vgrid(), 256, 0, st>>>(Vcol(j), c->dinv64, c->p32.xbuf, N, ldV()));
      AIM_TRY(chk("k_precond"));
      AIM_TRY(matvec(c, c->p32.xbuf, c->p32.ybuf, B, AIM_C64));
      return convert_c64_to_c128(c, c->p32.ybuf, k.w, (int64_t)B * N);
    }
    AIM_LAUNCH(c, "k_precond", k_precond<double><<<vgrid(), 256, 0, st>>>(Vcol(j), c->dinv64, c->p64.xbuf, N, ldV()));
    AIM_TRY(chk("k_precond"));
    return matvec(c, c->p64.xbuf, k.w, B, precision);
  }

  int orthogonalise(int j) {
    const int nvec = j + 1;
    const int ldp = m + 1 + kDotGroup;
    for (int pass = 0; pass < 2; ++pass) {
      AIM_LAUNCH(c, "k_dots", k_dots<<<dim3(k.nblk, B), 256, 0, st>>>(k.V, k.w, k.partial, N, nvec, m + 1, k.nblk, ldp));
      AIM_TRY(chk("k_dots"));
      AIM_LAUNCH(c, "k_dots_reduce", k_dots_reduce<<<B, 64, 0, st>>>(k.partial, k.hcol, k.H, nvec, k.nblk, ldp, m, j, pass));
      AIM_TRY(chk("k_dots_reduce"));
      AIM_LAUNCH(c, "k_update", k_update<<<vgrid(), 256, 0, st>>>(k.V, k.w, k.hcol, N, nvec, m + 1, m));
      AIM_TRY(chk("k_update"));
    }
    AIM_TRY(norms(k.w, N, k.nrm));
    AIM_LAUNCH(c, "k_scale", k_scale<<<vgrid(), 256, 0, st>>>(k.w, Vcol(j + 1), k.nrm, N, N, ldV()));
    return chk("k_scale");
  }
};
}  // namespace

int solve(aim_ctx* c, const double2* V, double2* X, int nrhs, double tol, aim_solve_info* info) {
  AIM_TRY(alloc_krylov(c));
  Solver s(c, nrhs);
  KrylovWork& k = c->kw;
  const int N = c->N, m = k.m;
  const int prec = c->opts.precision;
  const int exact = prec == AIM_C128_F64 ? AIM_C128_F64 : AIM_C128;  // FP64-accurate product for true residuals
  const int check = std::max(1, c->opts.check_every);
  std::vector<int> act(nrhs, 1);
  std::vector<double> bn(nrhs), rel(nrhs, 1.0);
  AIM_CUDA_TRY(cudaMemsetAsync(X, 0, sizeof(double2) * (size_t)nrhs * N, c->stream));
  AIM_TRY(s.norms(V, N, k.bnorm));
  AIM_CUDA_TRY(cudaMemcpyAsync(bn.data(), k.bnorm, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, c->stream));
  AIM_CUDA_TRY(cudaStreamSynchronize(c->stream));
  for (int b = 0; b < nrhs; ++b)
    if (bn[b] == 0.0) {
      act[b] = 0;
      rel[b] = 0.0;
    }
  int iters = 0, restarts = 0;
  bool first = true;
  for (;;) {
    // true residual (FP64 product) and convergence check
    AIM_CUDA_TRY(cudaMemcpyAsync(k.active, act.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, c->stream));
    if (first) {
      AIM_LAUNCH(c, "k_residual", k_residual<<<s.vgrid(), 256, 0, c->stream>>>(V, X, k.r, N, k.active));  // X = 0: r = V
      AIM_TRY(s.chk("k_residual"));
    } else {
      AIM_TRY(matvec(c, X, k.w, nrhs, exact));
      AIM_LAUNCH(c, "k_residual", k_residual<<<s.vgrid(), 256, 0, c->stream>>>(V, k.w, k.r, N, k.active));
      AIM_TRY(s.chk("k_residual"));
    }
    AIM_TRY(s.norms(k.r, N, k.nrm));
    std::vector<double> beta(nrhs);
    AIM_CUDA_TRY(cudaMemcpyAsync(beta.data(), k.nrm, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, c->stream));
    AIM_CUDA_TRY(cudaStreamSynchronize(c->stream));
    bool all = true;
    for (int b = 0; b < nrhs; ++b) {
      if (bn[b] == 0.0) continue;
      if (act[b]) rel[b] = beta[b] / bn[b];
      if (act[b] && rel[b] <= tol) act[b] = 0;
      all = all && !act[b];
    }
    if (all || iters >= c->opts.maxit) break;
    first = false;
    ++restarts;
    AIM_CUDA_TRY(cudaMemcpyAsync(k.active, act.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, c->stream));
    // v0 = r / beta, g = (beta, 0, ...)
    AIM_LAUNCH(c, "k_scale", k_scale<<<s.vgrid(), 256, 0, c->stream>>>(k.r, k.V, k.nrm, N, N, s.ldV()));
    AIM_TRY(s.chk("k_scale"));
    AIM_LAUNCH(c, "k_ginit", k_ginit<<<(nrhs + 127) / 128, 128, 0, c->stream>>>(k.g, k.nrm, m, nrhs));
    AIM_TRY(s.chk("k_ginit"));
    int kk = 0;
    for (int j = 0; j < m && iters < c->opts.maxit; ++j) {
      AIM_TRY(s.apply(j, prec));
      AIM_TRY(s.orthogonalise(j));
      AIM_LAUNCH(c, "k_givens", k_givens<<<(nrhs + 127) / 128, 128, 0, c->stream>>>(k.H, k.cs, k.sn, k.g, k.nrm, k.bnorm, s.est, m, j, nrhs));
      AIM_TRY(s.chk("k_givens"));
      ++iters;
      kk = j + 1;
      if ((j + 1) % check == 0 || j == m - 1) {
        AIM_CUDA_TRY(cudaMemcpyAsync(k.h_est, s.est, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, c->stream));
        AIM_CUDA_TRY(cudaStreamSynchronize(c->stream));
        bool done = true;
        for (int b = 0; b < nrhs; ++b)
          if (act[b] && !(k.h_est[b] <= tol)) done = false;
        if (done) break;
      }
    }
    AIM_LAUNCH(c, "k_backsolve", k_backsolve<<<(nrhs + 127) / 128, 128, 0, c->stream>>>(k.H, k.g, k.y, m, kk, nrhs));
    AIM_TRY(s.chk("k_backsolve"));
    AIM_LAUNCH(c, "k_xupdate", k_xupdate<<<s.vgrid(), 256, 0, c->stream>>>(k.V, k.y, c->dinv64, X, N, kk, m, m + 1, k.active));
    AIM_TRY(s.chk("k_xupdate"));
  }
  bool conv = true;
  for (int b = 0; b < nrhs; ++b) conv = conv && (rel[b] <= tol);
  if (info) {
    info->iterations = iters;
    info->restarts = restarts;
    for (int b = 0; b < nrhs; ++b) {
      if (info->rel_res) info->rel_res[b] = rel[b];
      if (info->converged) info->converged[b] = rel[b] <= tol ? 1 : 0;
    }
  }
  if (!conv) {
    set_error("aim_solve: iteration limit reached before the tolerance");
    return AIM_ENOCONV;
  }
  return AIM_OK;
}

}  // namespace aim
