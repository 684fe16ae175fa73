// Batched right-preconditioned restarted GMRES(m).
//
// Paper Section 2.2: diagonal preconditioner, iteration stopped on the
// relative residual.  All right-hand sides advance in lockstep; each keeps
// its own Arnoldi basis and Hessenberg matrix.  On the device: the product,
// dot products and norms in FP64 (two-level block reductions, so the results
// do not depend on launch timing), classical Gram-Schmidt with a second pass
// where the Daniel-Gragg-Kaufman-Stewart test asks for it.  One Arnoldi step
// is captured once as a CUDA graph and replayed (its kernels take the column
// index from device memory).  On the host, every few steps: the new
// Hessenberg columns, their Givens rotations in FP64, the residual estimate,
// and at the end of a cycle the small triangular solve.  The Arnoldi product
// is complex64 or complex128 (aim_opts.precision); every restart recomputes
// the true residual V - Z~ X with the FP64-accurate product, so the complex64
// mode is FP64 iterative refinement wrapped around a complex64 inner solve.
#include <algorithm>
#include <cmath>
#include <complex>

#include "common.h"

namespace aim {

constexpr int kDotGroup = 8;  // basis vectors per pass of the dot kernel
constexpr int kTfqmrVecs = 9;      // vectors per right-hand side of the TFQMR iteration
constexpr int kTfqmrScalars = 8;   // complex scalars per right-hand side of the TFQMR iteration

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

// Every kernel of the Arnoldi step reads the column index j from device
// memory (jdev), so one captured CUDA graph serves every step of a cycle.

// Pass `pass` of classical Gram-Schmidt for column j, partial dot products:
// partial[b][blk][i] = sum over block blk's chunk of conj(V[b][i]) . w[b],
// i <= j; on the first pass the slot i = j + 1 receives |w|^2 (the norm before
// orthogonalising, for the re-orthogonalisation test).  Grid: (vector groups
// of kDotGroup, nblk, B); blocks past the column's vectors, and the second
// pass of right-hand sides that need no re-orthogonalisation, return at once.
__global__ void __launch_bounds__(256) k_dots(const double2* __restrict__ V, const double2* __restrict__ w,
                                              double2* __restrict__ partial, const int* __restrict__ jdev,
                                              const int* __restrict__ reorth, int N, int ldv_vec, int nblk, int ldp,
                                              int pass) {
  const int b = blockIdx.z, blk = blockIdx.y, i0 = blockIdx.x * kDotGroup;
  const int nvec = *jdev + 1;
  const int nslot = pass == 0 ? nvec + 1 : nvec;
  if (i0 >= nslot || (pass == 1 && !reorth[b])) return;
  const double2* Vb = V + (long long)b * ldv_vec * N;
  const double2* wb = w + (long long)b * N;
  const int chunk = (N + nblk - 1) / nblk;
  const int n0 = blk * chunk, n1 = min(N, n0 + chunk);
  double2 acc[kDotGroup];
#pragma unroll
  for (int i = 0; i < kDotGroup; ++i) acc[i] = make_double2(0, 0);
  const int ni = min(kDotGroup, nslot - i0);
  for (int n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
    const double2 wv = wb[n];
#pragma unroll
    for (int i = 0; i < kDotGroup; ++i)
      if (i < ni) acc[i] = cfma_conj(i0 + i < nvec ? Vb[(long long)(i0 + i) * N + n] : wv, wv, acc[i]);
  }
  block_reduce_store<kDotGroup>(acc, partial + ((long long)b * nblk + blk) * ldp + i0, 1);
}

// w[b] -= sum_{i <= j} h[b][i] V[b][i], where every block first sums the dot
// kernel's partials itself (h[i] = sum over blk of partial[b][blk][i], in a
// fixed order, so every block holds the same values) and block 0 stores the
// Hessenberg column: H[j][b][i] = h (first pass) or += h (second pass).  On
// the first pass slot i = j + 1 holds |w|^2 before orthogonalising, and
// block 0 evaluates the re-orthogonalisation test of Daniel, Gragg, Kaufman
// and Stewart, |w1|^2 = |w0|^2 - |h|^2 < |w0|^2 / 2; the second pass runs
// only where it holds.
__global__ void __launch_bounds__(256) k_update(const double2* __restrict__ V, double2* __restrict__ w,
                                                const double2* __restrict__ partial, double2* __restrict__ H,
                                                int* __restrict__ reorth, const int* __restrict__ jdev, int N,
                                                int ldv_vec, int m, int B, int nblk, int ldp, int pass) {
  __shared__ double2 hs[256];
  const int b = blockIdx.y;
  if (pass == 1 && !reorth[b]) return;
  const int j = *jdev, nvec = j + 1;
  const int nslot = pass == 0 ? nvec + 1 : nvec;
  for (int i = threadIdx.x; i < nslot; i += blockDim.x) {
    double2 t = make_double2(0, 0);
    for (int blk = 0; blk < nblk; ++blk) {
      const double2 p = partial[((long long)b * nblk + blk) * ldp + i];
      t.x += p.x;
      t.y += p.y;
    }
    hs[i] = t;
  }
  __syncthreads();
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
      double2* h = H + ((long long)j * B + b) * (m + 1) + i;
      if (pass == 1) {
        h->x += hs[i].x;
        h->y += hs[i].y;
      } else {
        *h = hs[i];
      }
    }
    if (pass == 0 && threadIdx.x == 0) {
      double h2 = 0.0;
      for (int i = 0; i < nvec; ++i) h2 += hs[i].x * hs[i].x + hs[i].y * hs[i].y;
      const double w0 = hs[nvec].x;
      reorth[b] = (w0 - h2) < 0.5 * w0 ? 1 : 0;
    }
  }
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

// End of the step: |w| from the norm kernel's partial sums (every block
// reduces them in the same order), V[b][j + 1] = w[b] / |w|; block 0 stores
// |w| as the subdiagonal H[j][b][j + 1].
__global__ void __launch_bounds__(256) k_normalize(const double2* __restrict__ w, double2* __restrict__ V,
                                                   const double* __restrict__ npart, double2* __restrict__ H,
                                                   const int* __restrict__ jdev, int N, long long ldv, int nblk,
                                                   int m, int B) {
  __shared__ double red[8];
  __shared__ double nrm_s;
  const int b = blockIdx.y;
  const int j = *jdev;
  double t = 0.0;
  for (int blk = threadIdx.x; blk < nblk; blk += blockDim.x) t += npart[(long long)b * nblk + blk];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) u += red[i];
    nrm_s = sqrt(u);
    if (blockIdx.x == 0) H[((long long)j * B + b) * (m + 1) + j + 1] = make_double2(nrm_s, 0.0);
  }
  __syncthreads();
  const double s = nrm_s > 0.0 ? 1.0 / nrm_s : 0.0;
  double2* dst = V + (long long)b * ldv + (long long)(j + 1) * N;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
    double2 v = w[(long long)b * N + n];
    v.x *= s;
    v.y *= s;
    dst[n] = v;
  }
}

__global__ void k_next_j(int* jdev) { *jdev += 1; }
__global__ void k_set_j(int* jdev, int j) { *jdev = j; }

// z = dinv .* V_j, in precision R (dinv: row b at b * ldd; ldd = 0 shares one diagonal)
template <typename R>
__global__ void k_precond(const double2* __restrict__ V, const double2* __restrict__ dinv, cplx<R>* __restrict__ z,
                          const int* __restrict__ jdev, int N, long long ldv, long long ldd) {
  const int b = blockIdx.y;
  const double2* v = V + (long long)b * ldv + (long long)(*jdev) * N;
  const double2* db = dinv + (long long)b * ldd;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
    const double2 a = v[n], d = db[n];
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

// X[b] += dinv .* (sum_i y_i V_i)   (active right-hand sides only)
__global__ void k_xupdate(const double2* __restrict__ V, const double2* __restrict__ y, const double2* __restrict__ dinv,
                          double2* __restrict__ X, int N, int kk, int m, int ldv_vec, const int* __restrict__ active,
                          long long ldd) {
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
    const double2 d = dinv[(long long)b * ldd + n];
    double2& x = X[(long long)b * N + n];
    x.x += s.x * d.x - s.y * d.y;
    x.y += s.x * d.y + s.y * d.x;
  }
}

// ------------------------------------------------------------------ host driver
int alloc_krylov(aim_ctx* c) {
  KrylovWork& k = c->kw;
  const int B = c->max_rhs, m = c->opts.restart, N = c->N;
  // vectors per right-hand side: the GMRES basis, or the TFQMR vectors
  const int slots = c->opts.krylov == AIM_TFQMR ? kTfqmrVecs : m + 1;
  if (k.V && k.slots < slots) {  // a method that needs more vectors than the storage holds
    drop_step_graph(c);          // its captured step reads the old storage
    cudaFree(k.V);
    k.V = nullptr;
    AIM_CUDA_TRY(cudaMalloc(&k.V, (size_t)N * sizeof(double2) * B * slots));
    k.slots = slots;
  }
  if (k.V) return AIM_OK;
  k.m = m;
  // norm kernel: about four blocks per SM over all right-hand sides, at least 256 elements per block
  k.nblk = std::max(1, std::min((4 * 152 + B - 1) / B, (N + 255) / 256));
  // dot kernel: at least 1024 elements per block, about two blocks per SM per vector group
  k.nblk_dot = std::max(1, std::min((2 * 152 + B - 1) / B, (N + 1023) / 1024));
  const int nb = std::max(k.nblk, k.nblk_dot);
  const size_t vec = (size_t)N * sizeof(double2);
  AIM_CUDA_TRY(cudaMalloc(&k.V, vec * B * slots));
  k.slots = slots;
  AIM_CUDA_TRY(cudaMalloc(&k.w, vec * B));
  AIM_CUDA_TRY(cudaMalloc(&k.r, vec * B));
  AIM_CUDA_TRY(cudaMalloc(&k.H, sizeof(double2) * B * (m + 1) * m));
  AIM_CUDA_TRY(cudaMalloc(&k.partial, sizeof(double2) * B * nb * (m + 1 + kDotGroup)));
  AIM_CUDA_TRY(cudaMalloc(&k.y, sizeof(double2) * B * std::max(m, kTfqmrScalars)));
  AIM_CUDA_TRY(cudaMalloc(&k.nrm, sizeof(double) * B * (2 + nb)));
  AIM_CUDA_TRY(cudaMalloc(&k.bnorm, sizeof(double) * B));
  AIM_CUDA_TRY(cudaMalloc(&k.active, sizeof(int) * B));
  AIM_CUDA_TRY(cudaMalloc(&k.reorth, sizeof(int) * B));
  AIM_CUDA_TRY(cudaMalloc(&k.jdev, sizeof(int)));
  AIM_CUDA_TRY(cudaMallocHost(&k.h_H, sizeof(double2) * (size_t)B * (m + 1) * m));
  AIM_CUDA_TRY(cudaStreamCreateWithFlags(&k.cap_stream, cudaStreamNonBlocking));
  return AIM_OK;
}

void drop_step_graph(aim_ctx* c) {
  if (c->kw.step_exec) cudaGraphExecDestroy(c->kw.step_exec);
  c->kw.step_exec = nullptr;
}

void free_krylov(aim_ctx* c) {
  KrylovWork& k = c->kw;
  if (k.step_exec) cudaGraphExecDestroy(k.step_exec);
  if (k.cap_stream) cudaStreamDestroy(k.cap_stream);
  cudaFree(k.V); cudaFree(k.w); cudaFree(k.r); cudaFree(k.H); cudaFree(k.partial);
  cudaFree(k.y); cudaFree(k.nrm); cudaFree(k.bnorm);
  cudaFree(k.active); cudaFree(k.reorth); cudaFree(k.jdev);
  if (k.h_H) cudaFreeHost(k.h_H);
  k = KrylovWork{};
}

namespace {
struct Solver {
  aim_ctx* c;
  KrylovWork& k;
  int B, N, m;
  cudaStream_t st;
  double* npart;     // device [B][nblk]
  Solver(aim_ctx* cc, int nrhs) : c(cc), k(cc->kw), B(nrhs), N(cc->N), m(cc->kw.m), st(cc->stream) {
    npart = k.nrm + 2 * B;
  }
  dim3 vgrid() const { return dim3((unsigned)std::min(1024, std::max(1, (N + 255) / 256)), B); }
  int chk(const char* w) { return launch_check(c, w); }
  long long ldV() const { return (long long)(m + 1) * N; }

  int norm_partials(const double2* x, long long ldx) {
    AIM_LAUNCH(c, "k_norm2", k_norm2<<<dim3(k.nblk, B), 256, 0, st>>>(x, npart, N, ldx, k.nblk));
    return chk("k_norm2");
  }
  int norms(const double2* x, long long ldx, double* out) {
    AIM_TRY(norm_partials(x, ldx));
    AIM_LAUNCH(c, "k_sqrt_sum", k_sqrt_sum<<<(B + 127) / 128, 128, 0, st>>>(npart, out, k.nblk, B));
    return chk("k_sqrt_sum");
  }

  // One Arnoldi step for the column j held in device memory (k.jdev):
  // w = Z~ (dinv .* v_j) in `precision`, CGS with selective second pass into
  // the Hessenberg column H[j], v_{j+1} = w / |w|, j += 1.
  int step(int precision) {
    if (precision == AIM_C64) {
      AIM_LAUNCH(c, "k_precond", k_precond<float><<<vgrid(), 256, 0, st>>>(k.V, c->dinv64, c->p32.xbuf, k.jdev, N, ldV(),
                                                                           c->dinv_ld));
      AIM_TRY(chk("k_precond"));
      AIM_TRY(matvec(c, c->p32.xbuf, c->p32.ybuf, B, AIM_C64));
      AIM_TRY(convert_c64_to_c128(c, c->p32.ybuf, k.w, (int64_t)B * N));
    } else {
      AIM_LAUNCH(c, "k_precond", k_precond<double><<<vgrid(), 256, 0, st>>>(k.V, c->dinv64, c->p64.xbuf, k.jdev, N, ldV(),
                                                                            c->dinv_ld));
      AIM_TRY(chk("k_precond"));
      AIM_TRY(matvec(c, c->p64.xbuf, k.w, B, precision));
    }
    const int ldp = m + 1 + kDotGroup;
    const dim3 dgrid((m + 2 + kDotGroup - 1) / kDotGroup, k.nblk_dot, B);
    for (int pass = 0; pass < 2; ++pass) {
      AIM_LAUNCH(c, "k_dots", k_dots<<<dgrid, 256, 0, st>>>(k.V, k.w, k.partial, k.jdev, k.reorth, N, m + 1,
                                                            k.nblk_dot, ldp, pass));
      AIM_TRY(chk("k_dots"));
      AIM_LAUNCH(c, "k_update", k_update<<<vgrid(), 256, 0, st>>>(k.V, k.w, k.partial, k.H, k.reorth, k.jdev, N,
                                                                  m + 1, m, B, k.nblk_dot, ldp, pass));
      AIM_TRY(chk("k_update"));
    }
    AIM_TRY(norm_partials(k.w, N));
    AIM_LAUNCH(c, "k_normalize", k_normalize<<<vgrid(), 256, 0, st>>>(k.w, k.V, npart, k.H, k.jdev, N, ldV(), k.nblk,
                                                                     m, B));
    AIM_TRY(chk("k_normalize"));
    AIM_LAUNCH(c, "k_next_j", k_next_j<<<1, 1, 0, st>>>(k.jdev));
    return chk("k_next_j");
  }

  // The step as a CUDA graph (captured on first use for this precision and
  // batch size), or launched directly while the profiler is on.
  int run_step(int precision, bool allow_graph) {
#ifdef AIM_CHECK
    allow_graph = false;  // the check build reads its index checks (a synchronisation) after every product
#endif
    if (!allow_graph || c->prof.on) return step(precision);
    if (!k.step_exec || k.step_prec != precision || k.step_nrhs != B) {
      if (k.step_exec) {
        cudaGraphExecDestroy(k.step_exec);
        k.step_exec = nullptr;
      }
      const int64_t l0 = c->launches;
      const cudaStream_t st0 = st;
      AIM_CUDA_TRY(cudaStreamBeginCapture(k.cap_stream, cudaStreamCaptureModeThreadLocal));
      c->stream = st = k.cap_stream;  // every launch of the step goes to the capturing stream
      const int rc = step(precision);
      c->stream = st = st0;
      cudaGraph_t graph = nullptr;
      const cudaError_t e = cudaStreamEndCapture(k.cap_stream, &graph);
      k.step_launches = c->launches - l0;
      c->launches = l0;
      if (rc != AIM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      if (e != cudaSuccess) {
        set_error(std::string("aim_solve: stream capture of the Arnoldi step: ") + cudaGetErrorString(e));
        return AIM_ECUDA;
      }
      const cudaError_t ei = cudaGraphInstantiate(&k.step_exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ei != cudaSuccess) {
        k.step_exec = nullptr;
        set_error(std::string("aim_solve: graph instantiation: ") + cudaGetErrorString(ei));
        return AIM_ECUDA;
      }
      k.step_prec = precision;
      k.step_nrhs = B;
    }
    c->launches += k.step_launches;
    AIM_CUDA_TRY(cudaGraphLaunch(k.step_exec, st));
    return AIM_OK;
  }
};
}  // namespace

// Givens QR of one right-hand side's Hessenberg matrix, on the host in FP64
// (the rotations are a sequential chain of a few flops each: on the device it
// would keep one warp on GB300's narrow FP64 pipe for every step).  Rotation
// [[conj(c), conj(s)], [-s, c]], c = a/d, s = b/d, maps (a, b) to (d, 0).
struct HostLsq {
  using cd = std::complex<double>;
  int m;
  std::vector<cd> R, cs, sn, g;  // R column-major [m][m+1]
  explicit HostLsq(int mm) : m(mm), R((size_t)mm * (mm + 1)), cs(mm), sn(mm), g(mm + 1) {}
  void start(double beta) {
    std::fill(g.begin(), g.end(), cd(0.0, 0.0));
    g[0] = cd(beta, 0.0);
  }
  // column j (rows 0..j+1 of the raw Hessenberg matrix); returns |g[j+1]|
  double add_column(int j, const double2* col) {
    cd* r = &R[(size_t)j * (m + 1)];
    for (int i = 0; i <= j + 1; ++i) r[i] = cd(col[i].x, col[i].y);
    for (int i = 0; i < j; ++i) {
      const cd t = std::conj(cs[i]) * r[i] + std::conj(sn[i]) * r[i + 1];
      const cd u = -sn[i] * r[i] + cs[i] * r[i + 1];
      r[i] = t;
      r[i + 1] = u;
    }
    const double d = std::sqrt(std::norm(r[j]) + std::norm(r[j + 1]));
    cd cc(1.0, 0.0), ss(0.0, 0.0);
    if (d > 0.0) {
      cc = r[j] / d;
      ss = r[j + 1] / d;
    }
    cs[j] = cc;
    sn[j] = ss;
    r[j] = cd(d, 0.0);
    r[j + 1] = cd(0.0, 0.0);
    g[j + 1] = -ss * g[j];
    g[j] = std::conj(cc) * g[j];
    return std::abs(g[j + 1]);
  }
  // back substitution R y = g on the leading kk x kk block
  void solve(int kk, double2* y) const {
    std::vector<cd> yy(kk);
    for (int i = kk - 1; i >= 0; --i) {
      cd sum = g[i];
      for (int l = i + 1; l < kk; ++l) sum -= R[(size_t)l * (m + 1) + i] * yy[l];
      const cd dii = R[(size_t)i * (m + 1) + i];
      yy[i] = std::norm(dii) > 0.0 ? sum / dii : cd(0.0, 0.0);
    }
    for (int i = 0; i < kk; ++i) y[i] = make_double2(yy[i].real(), yy[i].imag());
  }
};

static int solve_gmres(aim_ctx* c, const double2* V, double2* X, int nrhs, double tol, aim_solve_info* info) {
  AIM_TRY(alloc_krylov(c));
  Solver s(c, nrhs);
  KrylovWork& k = c->kw;
  const int N = c->N, m = k.m;
  const int prec = c->opts.precision;
  const int exact = prec == AIM_C128_F64 ? AIM_C128_F64 : AIM_C128;  // FP64-accurate product for true residuals
  const int check = std::max(1, c->opts.check_every);
  AIM_TRY(prepare_product(c, prec));
  AIM_TRY(prepare_product(c, exact));
  std::vector<int> act(nrhs, 1);
  std::vector<double> bn(nrhs), rel(nrhs, 1.0);
  std::vector<HostLsq> lsq(nrhs, HostLsq(m));
  std::vector<double2> ybuf((size_t)nrhs * m);
  const size_t colsz = (size_t)nrhs * (m + 1);  // one Hessenberg column of every right-hand side
  AIM_CUDA_TRY(cudaMemsetAsync(X, 0, sizeof(double2) * (size_t)nrhs * N, c->stream));
  AIM_TRY(s.norms(V, N, k.bnorm));
  AIM_CUDA_TRY(cudaMemcpyAsync(bn.data(), k.bnorm, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, c->stream));
  AIM_CUDA_TRY(cudaStreamSynchronize(c->stream));
  for (int b = 0; b < nrhs; ++b) {
    if (!std::isfinite(bn[b])) {  // the norm pass sees every NaN and infinity of V
      set_error("aim_solve: right-hand side " + std::to_string(b) + " holds NaN or an infinity");
      return AIM_EINVAL;
    }
    if (bn[b] == 0.0) {
      act[b] = 0;
      rel[b] = 0.0;
    }
  }
  int iters = 0, restarts = 0;
  bool first = true, stepped = false;
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
    // v0 = r / beta, g = (beta, 0, ...), j = 0
    AIM_LAUNCH(c, "k_scale", k_scale<<<s.vgrid(), 256, 0, c->stream>>>(k.r, k.V, k.nrm, N, N, s.ldV()));
    AIM_TRY(s.chk("k_scale"));
    AIM_LAUNCH(c, "k_set_j", k_set_j<<<1, 1, 0, c->stream>>>(k.jdev, 0));
    AIM_TRY(s.chk("k_set_j"));
    for (int b = 0; b < nrhs; ++b) lsq[b].start(beta[b]);
    int kk = 0, done_cols = 0;
    // Hessenberg columns done_cols .. kk-1 to the host, Givens rotations; true when every active RHS is converged
    auto absorb = [&](bool* converged) -> int {
      const int ncol = kk - done_cols;
      if (ncol > 0) {
        AIM_CUDA_TRY(cudaMemcpyAsync(k.h_H, k.H + (size_t)done_cols * colsz, sizeof(double2) * colsz * ncol,
                                     cudaMemcpyDeviceToHost, c->stream));
        AIM_CUDA_TRY(cudaStreamSynchronize(c->stream));
      }
      bool done = true;
      for (int q = 0; q < ncol; ++q)
        for (int b = 0; b < nrhs; ++b) {
          const double r = lsq[b].add_column(done_cols + q, k.h_H + ((size_t)q * nrhs + b) * (m + 1));
          if (q == ncol - 1 && act[b] && !(bn[b] > 0.0 && r / bn[b] <= tol)) done = false;
        }
      done_cols = kk;
      *converged = done;
      return AIM_OK;
    };
    for (int j = 0; j < m && iters < c->opts.maxit; ++j) {
      // the very first step runs uncaptured (first launches set kernel attributes)
      AIM_TRY(s.run_step(prec, stepped));
      stepped = true;
      ++iters;
      kk = j + 1;
      if ((j + 1) % check == 0 || j == m - 1) {
        bool done = false;
        AIM_TRY(absorb(&done));
        if (done) break;
      }
    }
    bool unused = false;
    AIM_TRY(absorb(&unused));
    for (int b = 0; b < nrhs; ++b) lsq[b].solve(kk, &ybuf[(size_t)b * m]);
    AIM_CUDA_TRY(cudaMemcpyAsync(k.y, ybuf.data(), sizeof(double2) * (size_t)nrhs * m, cudaMemcpyHostToDevice,
                                 c->stream));
    AIM_LAUNCH(c, "k_xupdate", k_xupdate<<<s.vgrid(), 256, 0, c->stream>>>(k.V, k.y, c->dinv64, X, N, kk, m, m + 1, k.active,
                                                                        c->dinv_ld));
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


// ------------------------------------------------------------------ TFQMR
// Transpose-free QMR (Freund 1993; the form of Saad, Iterative Methods for
// Sparse Linear Systems, 2nd ed., Algorithm 7.8), an alternative to GMRES
// that needs no basis: nine vectors per right-hand side whatever the number
// of steps.  It runs on the right-preconditioned correction equation
// A M^-1 u = r, M = diag(Z~), batched over right-hand sides in lockstep: the
// vectors live in the basis storage (slot q of right-hand side b at
// V + (b kTfqmrVecs + q) N), the scalars of every right-hand side on the
// device (k.y, kTfqmrScalars complex values each), so the host only reads
// the residual bounds every check_every step pairs.  One step pair (two
// products) is captured as a CUDA graph and replayed.  A cycle ends when the
// quasi-residual bound tau sqrt(m + 1) of every active right-hand side is
// below its target; then x += M^-1 u, the true residual V - Z~ X is taken
// with the FP64-accurate product (iterative refinement, as for GMRES), and a
// new cycle starts from it until ||V - Z~ X|| / ||V|| <= tol.
namespace {
enum { TQ_UE, TQ_UO, TQ_AUE, TQ_AUO, TQ_V, TQ_W, TQ_D, TQ_R0, TQ_E };       // vector slots
enum { SQ_ALPHA, SQ_RHO, SQ_BETA, SQ_ETA, SQ_TT, SQ_COEF, SQ_ON, SQ_SPARE };  // scalar slots
// SQ_TT = (theta, tau); SQ_COEF = theta^2 eta / alpha of the next d update; SQ_ON.x = 1 for an active RHS

struct TqVecs {
  double2* base;
  int N;
  __device__ double2* at(int b, int q) const { return base + ((long long)b * kTfqmrVecs + q) * N; }
};

__device__ __forceinline__ double2 cmul2(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cdiv2(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return d > 0.0 ? make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d) : make_double2(0.0, 0.0);
}

// Block sums of |w|^2 (npart[b][blk]) and, when dpart is set, of conj(r0) . w
// (dpart[b][blk]); each block covers a chunk of N.
__device__ __forceinline__ void tq_reduce(double nw, double2 dw, double* npart, double2* dpart, int b, int blk,
                                          int nblk) {
  __shared__ double rn[32];
  __shared__ double2 rd[32];
  for (int o = 16; o > 0; o >>= 1) {
    nw += __shfl_xor_sync(0xffffffffu, nw, o);
    dw.x += __shfl_xor_sync(0xffffffffu, dw.x, o);
    dw.y += __shfl_xor_sync(0xffffffffu, dw.y, o);
  }
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    rn[warp] = nw;
    rd[warp] = dw;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    double2 u = make_double2(0.0, 0.0);
    for (int i = 0; i < nwarps; ++i) {
      t += rn[i];
      u.x += rd[i].x;
      u.y += rd[i].y;
    }
    if (npart) npart[(long long)b * nblk + blk] = t;
    if (dpart) dpart[(long long)b * nblk + blk] = u;
  }
}

// Cycle start: w = ue = r0 = r, d = e = 0; |r|^2 partials.  (Then Aue = A M^-1 ue.)
__global__ void __launch_bounds__(256) k_tq_init(const double2* __restrict__ r, TqVecs T, int N, double* npart,
                                                 int nblk) {
  const int b = blockIdx.y, blk = blockIdx.x;
  const int chunk = (N + nblk - 1) / nblk, n0 = blk * chunk, n1 = min(N, n0 + chunk);
  double nw = 0.0;
  for (int n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
    const double2 v = r[(long long)b * N + n];
    T.at(b, TQ_W)[n] = v;
    T.at(b, TQ_UE)[n] = v;
    T.at(b, TQ_R0)[n] = v;
    T.at(b, TQ_D)[n] = make_double2(0.0, 0.0);
    T.at(b, TQ_E)[n] = make_double2(0.0, 0.0);
    nw += v.x * v.x + v.y * v.y;
  }
  tq_reduce(nw, make_double2(0.0, 0.0), npart, nullptr, b, blk, nblk);
}

// After the first product: Aue = v = y; conj(r0) . v partials.
__global__ void __launch_bounds__(256) k_tq_init2(const double2* __restrict__ y, TqVecs T, int N, double2* dpart,
                                                  int nblk) {
  const int b = blockIdx.y, blk = blockIdx.x;
  const int chunk = (N + nblk - 1) / nblk, n0 = blk * chunk, n1 = min(N, n0 + chunk);
  double2 dv = make_double2(0.0, 0.0);
  for (int n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
    const double2 a = y[(long long)b * N + n], r0 = T.at(b, TQ_R0)[n];
    T.at(b, TQ_AUE)[n] = a;
    T.at(b, TQ_V)[n] = a;
    dv.x += r0.x * a.x + r0.y * a.y;
    dv.y += r0.x * a.y - r0.y * a.x;
  }
  tq_reduce(0.0, dv, nullptr, dpart, b, blk, nblk);
}

// Scalars at a cycle start: tau = |r|, theta = eta = 0, rho = |r|^2 (r0 = r),
// alpha = rho / (r0, v); the right-hand side takes part when `active`.
__global__ void k_tq_start(const double* __restrict__ npart, const double2* __restrict__ dpart, double2* sc,
                           const int* __restrict__ active, int nblk, int B) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double t = 0.0;
  double2 dv = make_double2(0.0, 0.0);
  for (int i = 0; i < nblk; ++i) {
    t += npart[(long long)b * nblk + i];
    dv.x += dpart[(long long)b * nblk + i].x;
    dv.y += dpart[(long long)b * nblk + i].y;
  }
  double2* q = sc + (long long)b * kTfqmrScalars;
  const bool on = active[b] != 0 && t > 0.0;
  q[SQ_RHO] = make_double2(t, 0.0);
  q[SQ_ALPHA] = on ? cdiv2(make_double2(t, 0.0), dv) : make_double2(0.0, 0.0);
  q[SQ_BETA] = make_double2(0.0, 0.0);
  q[SQ_ETA] = make_double2(0.0, 0.0);
  q[SQ_TT] = make_double2(0.0, sqrt(t));
  q[SQ_COEF] = make_double2(0.0, 0.0);
  q[SQ_ON] = make_double2(on ? 1.0 : 0.0, 0.0);
}

// Even step m: uo = ue - alpha v; w -= alpha Aue; d = ue + coef d; |w|^2 partials.
__global__ void __launch_bounds__(256) k_tq_even(TqVecs T, const double2* __restrict__ sc, int N, double* npart,
                                                 int nblk) {
  const int b = blockIdx.y, blk = blockIdx.x;
  const double2* q = sc + (long long)b * kTfqmrScalars;
  const double2 al = q[SQ_ALPHA], cf = q[SQ_COEF];
  const int chunk = (N + nblk - 1) / nblk, n0 = blk * chunk, n1 = min(N, n0 + chunk);
  double nw = 0.0;
  for (int n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
    const double2 ue = T.at(b, TQ_UE)[n], v = T.at(b, TQ_V)[n], au = T.at(b, TQ_AUE)[n];
    const double2 av = cmul2(al, v), aa = cmul2(al, au), cd = cmul2(cf, T.at(b, TQ_D)[n]);
    T.at(b, TQ_UO)[n] = make_double2(ue.x - av.x, ue.y - av.y);
    double2 w = T.at(b, TQ_W)[n];
    w.x -= aa.x;
    w.y -= aa.y;
    T.at(b, TQ_W)[n] = w;
    T.at(b, TQ_D)[n] = make_double2(ue.x + cd.x, ue.y + cd.y);
    nw += w.x * w.x + w.y * w.y;
  }
  tq_reduce(nw, make_double2(0.0, 0.0), npart, nullptr, b, blk, nblk);
}

// theta' = |w| / tau, c = (1 + theta'^2)^-1/2, tau' = tau theta' c, eta = c^2 alpha,
// and the coefficient theta'^2 eta / alpha of the next d update.  With
// `rho_step` (an odd step) also rho' = (r0, w), beta = rho' / rho, rho = rho'.
__global__ void k_tq_qmr(const double* __restrict__ npart, const double2* __restrict__ dpart, double2* sc, int nblk,
                         int B, int rho_step) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double2* q = sc + (long long)b * kTfqmrScalars;
  const bool on = q[SQ_ON].x != 0.0;
  double t = 0.0;
  double2 dw = make_double2(0.0, 0.0);
  for (int i = 0; i < nblk; ++i) {
    t += npart[(long long)b * nblk + i];
    if (rho_step) {
      dw.x += dpart[(long long)b * nblk + i].x;
      dw.y += dpart[(long long)b * nblk + i].y;
    }
  }
  const double tau = q[SQ_TT].y;
  const double th = tau > 0.0 ? sqrt(t) / tau : 0.0;
  const double cc = 1.0 / sqrt(1.0 + th * th);
  const double2 al = q[SQ_ALPHA];
  const double2 eta = on ? make_double2(cc * cc * al.x, cc * cc * al.y) : make_double2(0.0, 0.0);
  q[SQ_TT] = make_double2(th, tau * th * cc);
  q[SQ_ETA] = eta;
  q[SQ_COEF] = on ? cdiv2(make_double2(th * th * eta.x, th * th * eta.y), al) : make_double2(0.0, 0.0);
  if (rho_step) {
    const double2 rho = q[SQ_RHO];
    q[SQ_BETA] = on ? cdiv2(dw, rho) : make_double2(0.0, 0.0);
    q[SQ_RHO] = dw;
  }
}

// Odd step, first half: e += eta d (the even step's x update); Auo = y;
// w -= alpha Auo; d = uo + coef d; |w|^2 and conj(r0) . w partials.
__global__ void __launch_bounds__(256) k_tq_odd1(const double2* __restrict__ y, TqVecs T, const double2* __restrict__ sc,
                                                 int N, double* npart, double2* dpart, int nblk) {
  const int b = blockIdx.y, blk = blockIdx.x;
  const double2* q = sc + (long long)b * kTfqmrScalars;
  const double2 al = q[SQ_ALPHA], et = q[SQ_ETA], cf = q[SQ_COEF];
  const int chunk = (N + nblk - 1) / nblk, n0 = blk * chunk, n1 = min(N, n0 + chunk);
  double nw = 0.0;
  double2 dw = make_double2(0.0, 0.0);
  for (int n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
    const double2 d = T.at(b, TQ_D)[n], a = y[(long long)b * N + n], uo = T.at(b, TQ_UO)[n];
    const double2 ed = cmul2(et, d), aa = cmul2(al, a), cd = cmul2(cf, d);
    double2 e = T.at(b, TQ_E)[n];
    e.x += ed.x;
    e.y += ed.y;
    T.at(b, TQ_E)[n] = e;
    T.at(b, TQ_AUO)[n] = a;
    double2 w = T.at(b, TQ_W)[n];
    w.x -= aa.x;
    w.y -= aa.y;
    T.at(b, TQ_W)[n] = w;
    T.at(b, TQ_D)[n] = make_double2(uo.x + cd.x, uo.y + cd.y);
    const double2 r0 = T.at(b, TQ_R0)[n];
    nw += w.x * w.x + w.y * w.y;
    dw.x += r0.x * w.x + r0.y * w.y;
    dw.y += r0.x * w.y - r0.y * w.x;
  }
  tq_reduce(nw, dw, npart, dpart, b, blk, nblk);
}

// Odd step, second half: e += eta d; ue = w + beta uo.
__global__ void __launch_bounds__(256) k_tq_odd2(TqVecs T, const double2* __restrict__ sc, int N) {
  const int b = blockIdx.y;
  const double2* q = sc + (long long)b * kTfqmrScalars;
  const double2 et = q[SQ_ETA], be = q[SQ_BETA];
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
    const double2 ed = cmul2(et, T.at(b, TQ_D)[n]), bu = cmul2(be, T.at(b, TQ_UO)[n]);
    double2 e = T.at(b, TQ_E)[n];
    e.x += ed.x;
    e.y += ed.y;
    T.at(b, TQ_E)[n] = e;
    const double2 w = T.at(b, TQ_W)[n];
    T.at(b, TQ_UE)[n] = make_double2(w.x + bu.x, w.y + bu.y);
  }
}

// Odd step, last: Aue = y; v = Aue + beta (Auo + beta v); conj(r0) . v partials.
__global__ void __launch_bounds__(256) k_tq_odd3(const double2* __restrict__ y, TqVecs T, const double2* __restrict__ sc,
                                                 int N, double2* dpart, int nblk) {
  const int b = blockIdx.y, blk = blockIdx.x;
  const double2 be = sc[(long long)b * kTfqmrScalars + SQ_BETA];
  const int chunk = (N + nblk - 1) / nblk, n0 = blk * chunk, n1 = min(N, n0 + chunk);
  double2 dv = make_double2(0.0, 0.0);
  for (int n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
    const double2 a = y[(long long)b * N + n], ao = T.at(b, TQ_AUO)[n];
    T.at(b, TQ_AUE)[n] = a;
    const double2 bv = cmul2(be, T.at(b, TQ_V)[n]);
    const double2 inner = cmul2(be, make_double2(ao.x + bv.x, ao.y + bv.y));
    const double2 v = make_double2(a.x + inner.x, a.y + inner.y);
    T.at(b, TQ_V)[n] = v;
    const double2 r0 = T.at(b, TQ_R0)[n];
    dv.x += r0.x * v.x + r0.y * v.y;
    dv.y += r0.x * v.y - r0.y * v.x;
  }
  tq_reduce(0.0, dv, nullptr, dpart, b, blk, nblk);
}

// alpha = rho / (r0, v) for the next even step, and that step's d coefficient.
__global__ void k_tq_alpha(const double2* __restrict__ dpart, double2* sc, int nblk, int B) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double2* q = sc + (long long)b * kTfqmrScalars;
  double2 dv = make_double2(0.0, 0.0);
  for (int i = 0; i < nblk; ++i) {
    dv.x += dpart[(long long)b * nblk + i].x;
    dv.y += dpart[(long long)b * nblk + i].y;
  }
  const double2 al = q[SQ_ON].x != 0.0 ? cdiv2(q[SQ_RHO], dv) : make_double2(0.0, 0.0);
  q[SQ_ALPHA] = al;
  // the even step's d update divides by its own alpha: theta^2 eta / alpha
  const double th = q[SQ_TT].x;
  const double2 eta = q[SQ_ETA];
  q[SQ_COEF] = cdiv2(make_double2(th * th * eta.x, th * th * eta.y), al);
}

// End of the even step that closes a cycle early (the bound was met after an
// even step): e += eta d.  And the cycle's correction X += M^-1 e.
__global__ void __launch_bounds__(256) k_tq_finish(TqVecs T, const double2* __restrict__ sc, int N, int even_tail,
                                                   const double2* __restrict__ dinv, long long ldd, double2* X,
                                                   const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  const double2 et = sc[(long long)b * kTfqmrScalars + SQ_ETA];
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
    double2 e = T.at(b, TQ_E)[n];
    if (even_tail) {
      const double2 ed = cmul2(et, T.at(b, TQ_D)[n]);
      e.x += ed.x;
      e.y += ed.y;
    }
    const double2 x = cmul2(dinv[(long long)b * ldd + n], e);
    double2& X_ = X[(long long)b * N + n];
    X_.x += x.x;
    X_.y += x.y;
  }
}

struct Tfqmr {
  aim_ctx* c;
  KrylovWork& k;
  int B, N, nblk;
  TqVecs T;
  double* npart;
  double2* dpart;
  Tfqmr(aim_ctx* cc, int nrhs) : c(cc), k(cc->kw), B(nrhs), N(cc->N) {
    nblk = k.nblk;
    T = TqVecs{k.V, N};
    npart = k.nrm + 2 * B;
    dpart = k.partial;
  }
  dim3 vgrid() const { return dim3((unsigned)nblk, B); }
  int chk(const char* w) { return launch_check(c, w); }

  // y (k.w) = A M^-1 (slot q) in `precision`
  int product(int q, int precision) {
    const cudaStream_t st = c->stream;
    const long long ldv = (long long)kTfqmrVecs * N;
    AIM_LAUNCH(c, "k_set_j", k_set_j<<<1, 1, 0, st>>>(k.jdev, q));
    AIM_TRY(chk("k_set_j"));
    const dim3 g((unsigned)std::min(1024, std::max(1, (N + 255) / 256)), B);
    if (precision == AIM_C64) {
      AIM_LAUNCH(c, "k_precond", k_precond<float><<<g, 256, 0, st>>>(k.V, c->dinv64, c->p32.xbuf, k.jdev, N, ldv,
                                                                     c->dinv_ld));
      AIM_TRY(chk("k_precond"));
      AIM_TRY(matvec(c, c->p32.xbuf, c->p32.ybuf, B, AIM_C64));
      return convert_c64_to_c128(c, c->p32.ybuf, k.w, (int64_t)B * N);
    }
    AIM_LAUNCH(c, "k_precond", k_precond<double><<<g, 256, 0, st>>>(k.V, c->dinv64, c->p64.xbuf, k.jdev, N, ldv,
                                                                    c->dinv_ld));
    AIM_TRY(chk("k_precond"));
    return matvec(c, c->p64.xbuf, k.w, B, precision);
  }

  // One even and one odd step (two products).
  int pair(int precision) {
    const cudaStream_t st = c->stream;
    const unsigned sb = (unsigned)((B + 127) / 128);
    AIM_LAUNCH(c, "k_tq_even", k_tq_even<<<vgrid(), 256, 0, st>>>(T, k.y, N, npart, nblk));
    AIM_TRY(chk("k_tq_even"));
    AIM_LAUNCH(c, "k_tq_qmr", k_tq_qmr<<<sb, 128, 0, st>>>(npart, dpart, k.y, nblk, B, 0));
    AIM_TRY(chk("k_tq_qmr"));
    AIM_TRY(product(TQ_UO, precision));
    AIM_LAUNCH(c, "k_tq_odd1", k_tq_odd1<<<vgrid(), 256, 0, st>>>(k.w, T, k.y, N, npart, dpart, nblk));
    AIM_TRY(chk("k_tq_odd1"));
    AIM_LAUNCH(c, "k_tq_qmr", k_tq_qmr<<<sb, 128, 0, st>>>(npart, dpart, k.y, nblk, B, 1));
    AIM_TRY(chk("k_tq_qmr"));
    AIM_LAUNCH(c, "k_tq_odd2", k_tq_odd2<<<vgrid(), 256, 0, st>>>(T, k.y, N));
    AIM_TRY(chk("k_tq_odd2"));
    AIM_TRY(product(TQ_UE, precision));
    AIM_LAUNCH(c, "k_tq_odd3", k_tq_odd3<<<vgrid(), 256, 0, st>>>(k.w, T, k.y, N, dpart, nblk));
    AIM_TRY(chk("k_tq_odd3"));
    AIM_LAUNCH(c, "k_tq_alpha", k_tq_alpha<<<sb, 128, 0, st>>>(dpart, k.y, nblk, B));
    return chk("k_tq_alpha");
  }

  // The step pair as a CUDA graph (kept with the GMRES step graph's slot,
  // keyed by precision + 16), or launched directly while the profiler is on.
  int run_pair(int precision, bool allow_graph) {
#ifdef AIM_CHECK
    allow_graph = false;  // the check build synchronises after every product
#endif
    if (!allow_graph || c->prof.on) return pair(precision);
    const int key = precision + 16;
    if (!k.step_exec || k.step_prec != key || k.step_nrhs != B) {
      if (k.step_exec) {
        cudaGraphExecDestroy(k.step_exec);
        k.step_exec = nullptr;
      }
      const int64_t l0 = c->launches;
      const cudaStream_t st0 = c->stream;
      AIM_CUDA_TRY(cudaStreamBeginCapture(k.cap_stream, cudaStreamCaptureModeThreadLocal));
      c->stream = k.cap_stream;
      const int rc = pair(precision);
      c->stream = st0;
      cudaGraph_t graph = nullptr;
      const cudaError_t e = cudaStreamEndCapture(k.cap_stream, &graph);
      k.step_launches = c->launches - l0;
      c->launches = l0;
      if (rc != AIM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      if (e != cudaSuccess) {
        set_error(std::string("aim_solve: stream capture of the TFQMR step: ") + cudaGetErrorString(e));
        return AIM_ECUDA;
      }
      const cudaError_t ei = cudaGraphInstantiate(&k.step_exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ei != cudaSuccess) {
        k.step_exec = nullptr;
        set_error(std::string("aim_solve: graph instantiation: ") + cudaGetErrorString(ei));
        return AIM_ECUDA;
      }
      k.step_prec = key;
      k.step_nrhs = B;
    }
    c->launches += k.step_launches;
    AIM_CUDA_TRY(cudaGraphLaunch(k.step_exec, c->stream));
    return AIM_OK;
  }
};
}  // namespace

static int solve_tfqmr(aim_ctx* c, const double2* V, double2* X, int nrhs, double tol, aim_solve_info* info) {
  AIM_TRY(alloc_krylov(c));
  Solver s(c, nrhs);
  Tfqmr q(c, nrhs);
  KrylovWork& k = c->kw;
  const int N = c->N;
  const int prec = c->opts.precision;
  const int exact = prec == AIM_C128_F64 ? AIM_C128_F64 : AIM_C128;
  const int check = std::max(1, c->opts.check_every);
  // a cycle's target relative to its starting residual: what the inner products can reach
  const double inner = prec == AIM_C64 ? 1e-5 : 1e-12;
  AIM_TRY(prepare_product(c, prec));
  AIM_TRY(prepare_product(c, exact));
  std::vector<int> act(nrhs, 1);
  std::vector<double> bn(nrhs), rel(nrhs, 1.0), target(nrhs);
  std::vector<double2> sc((size_t)nrhs * kTfqmrScalars);
  AIM_CUDA_TRY(cudaMemsetAsync(X, 0, sizeof(double2) * (size_t)nrhs * N, c->stream));
  AIM_TRY(s.norms(V, N, k.bnorm));
  AIM_CUDA_TRY(cudaMemcpyAsync(bn.data(), k.bnorm, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, c->stream));
  AIM_CUDA_TRY(cudaStreamSynchronize(c->stream));
  for (int b = 0; b < nrhs; ++b) {
    if (!std::isfinite(bn[b])) {
      set_error("aim_solve: right-hand side " + std::to_string(b) + " holds NaN or an infinity");
      return AIM_EINVAL;
    }
    if (bn[b] == 0.0) {
      act[b] = 0;
      rel[b] = 0.0;
    }
  }
  int iters = 0, cycles = 0;
  bool first = true, stepped = false;
  for (;;) {
    // true residual (FP64-accurate product) and convergence check
    AIM_CUDA_TRY(cudaMemcpyAsync(k.active, act.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, c->stream));
    if (first) {
      AIM_LAUNCH(c, "k_residual", k_residual<<<s.vgrid(), 256, 0, c->stream>>>(V, X, k.r, N, k.active));
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
      target[b] = std::max(0.5 * tol * bn[b], inner * beta[b]);
    }
    if (all || iters >= c->opts.maxit) break;
    first = false;
    ++cycles;
    AIM_CUDA_TRY(cudaMemcpyAsync(k.active, act.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, c->stream));
    // cycle start on the correction equation A M^-1 u = r
    AIM_LAUNCH(c, "k_tq_init", k_tq_init<<<q.vgrid(), 256, 0, c->stream>>>(k.r, q.T, N, q.npart, q.nblk));
    AIM_TRY(q.chk("k_tq_init"));
    AIM_TRY(q.product(TQ_UE, prec));
    AIM_LAUNCH(c, "k_tq_init2", k_tq_init2<<<q.vgrid(), 256, 0, c->stream>>>(k.w, q.T, N, q.dpart, q.nblk));
    AIM_TRY(q.chk("k_tq_init2"));
    AIM_LAUNCH(c, "k_tq_start", k_tq_start<<<(nrhs + 127) / 128, 128, 0, c->stream>>>(q.npart, q.dpart, k.y, k.active,
                                                                                        q.nblk, nrhs));
    AIM_TRY(q.chk("k_tq_start"));
    int m = 0;  // steps of the cycle (two per pair)
    for (int p = 0; iters < c->opts.maxit; ++p) {
      AIM_TRY(q.run_pair(prec, stepped));
      stepped = true;
      m += 2;
      iters += 2;
      if ((p + 1) % check == 0) {
        AIM_CUDA_TRY(cudaMemcpyAsync(sc.data(), k.y, sizeof(double2) * sc.size(), cudaMemcpyDeviceToHost, c->stream));
        AIM_CUDA_TRY(cudaStreamSynchronize(c->stream));
        bool done = true;
        for (int b = 0; b < nrhs; ++b) {
          const double2* qb = &sc[(size_t)b * kTfqmrScalars];
          if (qb[SQ_ON].x == 0.0) continue;
          // ||r_m|| <= tau_m sqrt(m + 1) (Freund); a non-finite tau ends the cycle too
          const double bound = qb[SQ_TT].y * std::sqrt((double)m + 1.0);
          if (std::isfinite(bound) && bound > target[b]) done = false;
        }
        if (done) break;
      }
    }
    // the cycle ends after an odd step: e is complete, X += M^-1 e
    AIM_LAUNCH(c, "k_tq_finish", k_tq_finish<<<s.vgrid(), 256, 0, c->stream>>>(q.T, k.y, N, 0, c->dinv64, c->dinv_ld, X,
                                                                                 k.active));
    AIM_TRY(q.chk("k_tq_finish"));
  }
  bool conv = true;
  for (int b = 0; b < nrhs; ++b) conv = conv && (rel[b] <= tol);
  if (info) {
    info->iterations = iters;
    info->restarts = cycles;
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

int solve(aim_ctx* c, const double2* V, double2* X, int nrhs, double tol, aim_solve_info* info) {
  if (c->opts.krylov == AIM_TFQMR) return solve_tfqmr(c, V, X, nrhs, tol, info);
  return solve_gmres(c, V, X, nrhs, tol, info);
}

}  // namespace aim
