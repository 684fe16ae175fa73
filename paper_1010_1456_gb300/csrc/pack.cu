// Multi-instance batching: several contexts of small scatterers go through
// one launch per product stage (aim_pack_* in aim.h).
//
// Each instance is one scatterer of its own: the product of an instance is
// the paper's (Section 4.1: projection, FFT convolution, interpolation;
// Section 2.2: near-zone correction), with its own weights, lists and CFIE
// weight.  What the instances share is the launches: their grids are laid
// over one box (per axis the largest unpadded extent n_p and the largest
// padded length L_p of the instances), right-hand side b owns the pack's grids
// 4b .. 4b + 3, and the z, y and x passes of fft.cu run over all of them as
// one batch.  The pack's spectrum is the circulant embedding of G_h over n_p
// on L_p.  Every instance's nodes fill the corner [0, n_i) of the box and
// L_p >= 2 n_p - 1 per axis (both maxima come from instances whose own
// padded length satisfies it), so the circular convolution on the box,
// observed on [0, n_i), sums exactly the offsets |d| < n_i, where this
// embedding and the instance's own agree: the packed product equals each
// instance's product up to rounding.
//
// The projection kernel walks (instance, 8-node group of the box) tasks and
// reads an instance's node-ordered lists at the node's local index (nodes
// outside the instance's box get zeros); the interpolation kernel walks the
// instances' basis functions (8 lanes each, as interp_near) with stencil
// bases remapped to the box at creation.  The packed vectors have rows of
// length ld = max N_i; the interpolation kernel also writes the padding of
// every row as zero.
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "common.h"
#include "geom.h"

namespace aim {

// Device descriptor of one instance.
struct PackInst {
  int N, nrhs, b0;               // basis functions; its rows b0 .. b0 + nrhs - 1
  int nx, ny, nz;                // its grid box (a corner of the pack's box)
  const int32_t* pptr;           // [nx ny nz + 1] projection entries per local node
  const int32_t* pm;             // [nent] basis function of each entry
  const float* pw;               // [nent][4] weights (x, y, z, charge)
  const float* lam;              // [N][4][S]
  const float* lamM;             // [N][3][S] MFIE weights, or null (EFIE)
  const int32_t* base;           // [N] first stencil node, flat index in the pack's box
  const int32_t* nptr;           // [N + 1] near rows
  const int32_t* ncol;           // [nnz]
  const float2* nval;            // [nnz]
  float fvec, frho, fmf;         // alpha k eta, alpha eta / k, (1 - alpha) eta
};

}  // namespace aim

struct aim_pack {
  aim_ctx* pc = nullptr;                 // internal context: box, grids, spectrum, Krylov state
  std::vector<aim_ctx*> inst;
  std::vector<int> nrhs, b0;
  int K = 0, B = 0, ld = 0;
  long long rows = 0;                    // sum of N_i
  aim::PackInst* d_inst = nullptr;       // [K]
  int32_t* d_row0 = nullptr;             // [K + 1] first interpolation row of each instance
  int32_t* d_rhsN = nullptr;             // [B] N of the instance that owns each row
  int32_t* d_base = nullptr;             // [rows] remapped stencil bases
  double2* stage_x = nullptr;            // per-instance staging of the FP64-accurate products
  double2* stage_y = nullptr;
};

namespace aim {

constexpr int kPackMaxStencil = 216;

// Projection, one warp per task (instance i, 8 consecutive nodes of the box),
// 4 lanes per node taking every fourth entry, right-hand sides in chunks of
// 4; nodes outside the instance's box (or without entries) are written as
// zeros, so every grid of the pack is rewritten by every product.
__global__ void __launch_bounds__(256) proj_pack(const float2* __restrict__ x, float2* __restrict__ Q,
                                                 const PackInst* __restrict__ inst, int K, int ldx, int nxp, int nyp,
                                                 long long Ncp, long long ntask) {
  const int lane = threadIdx.x & 3, slot = (threadIdx.x & 31) >> 2;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < (long long)K * ntask; t += nwarps) {
    const int i = (int)(t / ntask);  // the same for the whole warp
    const PackInst& d = inst[i];
    const long long u = 8 * (t - (long long)i * ntask) + slot;
    int e0 = 0, e1 = 0;
    if (u < Ncp) {
      const int ux = (int)(u % nxp);
      const long long r = u / nxp;
      const int uy = (int)(r % nyp), uz = (int)(r / nyp);
      if (ux < d.nx && uy < d.ny && uz < d.nz) {
        const long long loc = ((long long)uz * d.ny + uy) * d.nx + ux;
        e0 = d.pptr[loc];
        e1 = d.pptr[loc + 1];
#ifdef AIM_CHECK
        if (!indices_ok(d.pm, e0, e1, d.N, 4)) e1 = e0;
#endif
      }
    }
    for (int bc = 0; bc < d.nrhs; bc += 4) {
      float2 a[4][4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < 4; ++c) a[q][c] = make_float2(0.f, 0.f);
      for (int e = e0 + lane; e < e1; e += 4) {
        const float4 w = reinterpret_cast<const float4*>(d.pw)[e];
        const float2* xc = x + (long long)(d.b0 + bc) * ldx + d.pm[e];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float2 xv = bc + q < d.nrhs ? xc[(long long)q * ldx] : make_float2(0.f, 0.f);
          a[q][0].x += w.x * xv.x; a[q][0].y += w.x * xv.y;
          a[q][1].x += w.y * xv.x; a[q][1].y += w.y * xv.y;
          a[q][2].x += w.z * xv.x; a[q][2].y += w.z * xv.y;
          a[q][3].x += w.w * xv.x; a[q][3].y += w.w * xv.y;
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int o = 1; o < 4; o <<= 1)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            a[q][c].x += __shfl_xor_sync(0xffffffffu, a[q][c].x, o, 4);
            a[q][c].y += __shfl_xor_sync(0xffffffffu, a[q][c].y, o, 4);
          }
        if (u < Ncp && bc + q < d.nrhs) {
          const float2 v = lane == 0 ? a[q][0] : lane == 1 ? a[q][1] : lane == 2 ? a[q][2] : a[q][3];
          Q[((long long)(d.b0 + bc + q) * 4 + lane) * Ncp + u] = v;
        }
      }
    }
  }
}

// Interpolation + near correction, 8 lanes per basis function of any
// instance (the 8 lanes of a group share one instance, the groups of a warp
// may not, so the reductions use the group's own lane mask), then the
// padding of every packed row written as zero.
__global__ void __launch_bounds__(256) interp_pack(const float2* __restrict__ Phi, const float2* __restrict__ x,
                                                   float2* __restrict__ y, const PackInst* __restrict__ inst,
                                                   const int32_t* __restrict__ row0, int K, long long rows, int ldx,
                                                   int nxp, int nyp, long long Ncp, int S, int P,
                                                   const int32_t* __restrict__ rhsN, int B) {
  __shared__ int s_off[kPackMaxStencil];
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    const int ii = s % P, j = (s / P) % P, kk = s / (P * P);
    s_off[s] = (kk * nyp + j) * nxp + ii;
  }
  __syncthreads();
  const int lane = threadIdx.x & 7;
  const unsigned gmask = 0xffu << (threadIdx.x & 24);
  const long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
  if (r < rows) {
    int lo = 0, hi = K - 1;  // instance i with row0[i] <= r < row0[i + 1]
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (row0[mid] <= r) lo = mid; else hi = mid - 1;
    }
    const PackInst& d = inst[lo];
    const int m = (int)(r - row0[lo]);
    const int bs = d.base[m];
    const float* lm = d.lam + (long long)m * 4 * S;
    const float* wm = d.lamM ? d.lamM + (long long)m * 3 * S : nullptr;
    const int r0 = d.nptr[m];
    int r1 = d.nptr[m + 1];
#ifdef AIM_CHECK
    const int Sc = stencil_ok(bs, nxp, nyp, Ncp, P, S, 5) ? S : 0;
    if (!indices_ok(d.ncol, r0, r1, d.N, 6)) r1 = r0;
#else
    const int Sc = S;
#endif
    for (int b = 0; b < d.nrhs; ++b) {
      const long long g = d.b0 + b;
      const float2* Pb = Phi + g * 4 * Ncp;
      float2 av = make_float2(0.f, 0.f), ar = av, an = av, am = av;
      for (int s = lane; s < Sc; s += 8) {
        const long long node = bs + (long long)s_off[s];
        const float2 px = Pb[node], py = Pb[Ncp + node], pz = Pb[2 * Ncp + node], pr = Pb[3 * Ncp + node];
        const float wx = lm[s], wy = lm[S + s], wz = lm[2 * S + s], wr = lm[3 * S + s];
        av.x += wx * px.x + wy * py.x + wz * pz.x;
        av.y += wx * px.y + wy * py.y + wz * pz.y;
        ar.x += wr * pr.x;
        ar.y += wr * pr.y;
        if (wm) {
          const float mx = wm[s], my = wm[S + s], mz = wm[2 * S + s];
          am.x += mx * px.x + my * py.x + mz * pz.x;
          am.y += mx * px.y + my * py.y + mz * pz.y;
        }
      }
      const float2* xb = x + g * ldx;
      for (int e = r0 + lane; e < r1; e += 8) {
        const float2 v = d.nval[e], xv = xb[d.ncol[e]];
        an.x += v.x * xv.x - v.y * xv.y;
        an.y += v.x * xv.y + v.y * xv.x;
      }
      // j (fvec av - frho ar) - fmf am + near
      float2 out;
      out.x = an.x - (d.fvec * av.y - d.frho * ar.y) - d.fmf * am.x;
      out.y = an.y + (d.fvec * av.x - d.frho * ar.x) - d.fmf * am.y;
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) {
        out.x += __shfl_xor_sync(gmask, out.x, o, 8);
        out.y += __shfl_xor_sync(gmask, out.y, o, 8);
      }
      if (lane == 0) y[g * ldx + m] = out;
    }
  }
  const long long nth = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)B * ldx; e += nth) {
    const int b = (int)(e / ldx), n = (int)(e - (long long)b * ldx);
    if (n >= rhsN[b]) y[e] = make_float2(0.f, 0.f);
  }
}

// Stencil base of each basis function from the instance's box (nx, ny) to the pack's (nxp, nyp).
__global__ void k_remap_base(const int32_t* __restrict__ in, int32_t* __restrict__ out, int N, int nx, int ny,
                             int nxp, int nyp) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < N; m += gridDim.x * blockDim.x) {
    const int b = in[m];
    const int x = b % nx, t = b / nx;
    const int y = t % ny, z = t / ny;
    out[m] = (z * nyp + y) * nxp + x;
  }
}

static int pack_c64(aim_pack* P, const float2* x, float2* y) {
  aim_ctx* c = P->pc;
  const long long Ncp = (long long)c->n[0] * c->n[1] * c->n[2];
  {
    const long long ntask = (Ncp + 7) / 8;
    const int blocks = (int)std::min<long long>((P->K * ntask + 7) / 8, 152LL * 16);
    AIM_LAUNCH(c, "proj_pack", (proj_pack<<<blocks, 256, 0, c->stream>>>(x, c->p32.grid0, P->d_inst, P->K, P->ld,
                                                                         c->n[0], c->n[1], Ncp, ntask)));
    AIM_TRY(launch_check(c, "proj_pack"));
  }
  AIM_TRY(fft_convolve_c64(c, 4 * P->B));
  {
    const long long threads = P->rows * 8;
    const int blocks = (int)std::max<long long>(1, (threads + 255) / 256);
    AIM_LAUNCH(c, "interp_pack",
               (interp_pack<<<blocks, 256, 0, c->stream>>>(phi_grid(c, c->p32.grid0, c->p32.grid2), x, y, P->d_inst,
                                                           P->d_row0, P->K, P->rows, P->ld, c->n[0], c->n[1], Ncp,
                                                           c->S, c->M + 1, P->d_rhsN, P->B)));
    AIM_TRY(launch_check(c, "interp_pack"));
  }
  return AIM_OK;
}

// FP64-accurate (or native FP64) product of every instance in turn, through
// contiguous staging rows, on the pack's stream.
static int pack_exact(aim_pack* P, const double2* x, double2* y, int precision) {
  aim_ctx* c = P->pc;
  const size_t ld = (size_t)P->ld * sizeof(double2);
  AIM_CUDA_TRY(cudaMemsetAsync(y, 0, ld * P->B, c->stream));
  for (int i = 0; i < P->K; ++i) {
    aim_ctx* ci = P->inst[i];
    const size_t row = (size_t)ci->N * sizeof(double2);
    AIM_CUDA_TRY(cudaMemcpy2DAsync(P->stage_x, row, x + (size_t)P->b0[i] * P->ld, ld, row, P->nrhs[i],
                                   cudaMemcpyDeviceToDevice, c->stream));
    const cudaStream_t own = ci->stream;
    ci->stream = c->stream;
    const int rc = matvec(ci, P->stage_x, P->stage_y, P->nrhs[i], precision);
    ci->stream = own;
    AIM_TRY(rc);
    AIM_CUDA_TRY(cudaMemcpy2DAsync(y + (size_t)P->b0[i] * P->ld, ld, P->stage_y, row, row, P->nrhs[i],
                                   cudaMemcpyDeviceToDevice, c->stream));
  }
  return AIM_OK;
}

int pack_matvec(aim_ctx* c, const void* x, void* y, int nrhs, int precision) {
  aim_pack* P = c->pack;
  if (nrhs != P->B) {
    set_error("pack product: every packed row takes part (nrhs must equal the pack's total)");
    return AIM_EINVAL;
  }
  if (precision != AIM_C64) return pack_exact(P, (const double2*)x, (double2*)y, precision);
  AIM_TRY(pack_c64(P, (const float2*)x, (float2*)y));
#ifdef AIM_CHECK
  AIM_TRY(read_index_checks(c, "packed product"));
#endif
  return AIM_OK;
}

int pack_prepare(aim_ctx* c, int precision) {
  aim_pack* P = c->pack;
  if (precision == AIM_C64) return ensure_grids(c, AIM_C64);
  for (aim_ctx* ci : P->inst) {
    const cudaStream_t own = ci->stream;
    ci->stream = c->stream;
    const int rc = prepare_product(ci, precision);
    ci->stream = own;
    AIM_TRY(rc);
  }
  return AIM_OK;
}

static void free_pack(aim_pack* P) {
  if (!P) return;
  cudaDeviceSynchronize();
  cudaFree(P->d_inst);
  cudaFree(P->d_row0);
  cudaFree(P->d_rhsN);
  cudaFree(P->d_base);
  cudaFree(P->stage_x);
  cudaFree(P->stage_y);
  if (P->pc) {
    P->pc->pack = nullptr;
    free_context(P->pc);
  }
  delete P;
}

static int build_pack(aim_pack* P) {
  aim_ctx* c0 = P->inst[0];
  aim_ctx* c = P->pc;
  const cudaStream_t st = c->stream;
  // the box and the padded lengths
  for (int d = 0; d < 3; ++d) {
    c->n[d] = 0;
    c->L[d] = 0;
    for (aim_ctx* ci : P->inst) {
      c->n[d] = std::max(c->n[d], ci->n[d]);
      c->L[d] = std::max(c->L[d], ci->L[d]);
    }
    c->plan[d] = make_plan(c->L[d]);
  }
  c->k = c0->k;
  c->h = c0->h;
  c->M = c0->M;
  c->S = c0->S;
  c->planar = c0->planar;
  c->alpha = 1.0;
  c->sparse_proj = 0;  // the projection rewrites every node of every grid; Phi lands in grid0
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < AIM_FFT_PASSES; ++q) c->fft_kernel[p][q] = c0->fft_kernel[p][q];
  AIM_TRY(fft_tables(c));
  AIM_TRY(build_ghat(c));
  // remapped bases, row offsets, owners of the rows
  AIM_CUDA_TRY(cudaMalloc(&P->d_base, sizeof(int32_t) * std::max<long long>(1, P->rows)));
  std::vector<int32_t> row0(P->K + 1, 0), rhsN(P->B, 0);
  std::vector<PackInst> h(P->K);
  for (int i = 0; i < P->K; ++i) {
    aim_ctx* ci = P->inst[i];
    row0[i + 1] = row0[i] + ci->N;
    for (int b = 0; b < P->nrhs[i]; ++b) rhsN[P->b0[i] + b] = ci->N;
    AIM_LAUNCH(c, "k_remap_base", (k_remap_base<<<std::min(1024, (ci->N + 255) / 256), 256, 0, st>>>(
                                      ci->base, P->d_base + row0[i], ci->N, ci->n[0], ci->n[1], c->n[0], c->n[1])));
    AIM_TRY(launch_check(c, "k_remap_base"));
    PackInst& d = h[i];
    d.N = ci->N;
    d.nrhs = P->nrhs[i];
    d.b0 = P->b0[i];
    d.nx = ci->n[0];
    d.ny = ci->n[1];
    d.nz = ci->n[2];
    d.pptr = ci->pnode_ptr;
    d.pm = ci->pnode_m;
    d.pw = ci->p32.pnode_w;
    d.lam = ci->p32.lam;
    d.lamM = ci->p32.lamM;
    d.base = P->d_base + row0[i];
    d.nptr = ci->near_ptr;
    d.ncol = ci->near_col;
    d.nval = ci->p32.near_val;
    d.fvec = (float)(ci->alpha * ci->k * kEta0);
    d.frho = (float)(ci->alpha * kEta0 / ci->k);
    d.fmf = (float)((1.0 - ci->alpha) * kEta0);
  }
  AIM_CUDA_TRY(cudaMalloc(&P->d_inst, sizeof(PackInst) * P->K));
  AIM_CUDA_TRY(cudaMalloc(&P->d_row0, sizeof(int32_t) * (P->K + 1)));
  AIM_CUDA_TRY(cudaMalloc(&P->d_rhsN, sizeof(int32_t) * P->B));
  AIM_CUDA_TRY(cudaMemcpyAsync(P->d_inst, h.data(), sizeof(PackInst) * P->K, cudaMemcpyHostToDevice, st));
  AIM_CUDA_TRY(cudaMemcpyAsync(P->d_row0, row0.data(), sizeof(int32_t) * (P->K + 1), cudaMemcpyHostToDevice, st));
  AIM_CUDA_TRY(cudaMemcpyAsync(P->d_rhsN, rhsN.data(), sizeof(int32_t) * P->B, cudaMemcpyHostToDevice, st));
  // one inverse diagonal per packed row (zero on the padding)
  const size_t ldb = (size_t)P->ld * sizeof(double2);
  AIM_CUDA_TRY(cudaMalloc(&c->dinv64, ldb * P->B));
  AIM_CUDA_TRY(cudaMemsetAsync(c->dinv64, 0, ldb * P->B, st));
  for (int i = 0; i < P->K; ++i)
    for (int b = 0; b < P->nrhs[i]; ++b)
      AIM_CUDA_TRY(cudaMemcpyAsync(c->dinv64 + (size_t)(P->b0[i] + b) * P->ld, P->inst[i]->dinv64,
                                   sizeof(double2) * P->inst[i]->N, cudaMemcpyDeviceToDevice, st));
  c->dinv_ld = P->ld;
  // staging of the per-instance FP64-accurate products, the solver's vectors, the grids
  size_t stage = 1;
  for (int i = 0; i < P->K; ++i) stage = std::max(stage, (size_t)P->nrhs[i] * P->inst[i]->N);
  AIM_CUDA_TRY(cudaMalloc(&P->stage_x, sizeof(double2) * stage));
  AIM_CUDA_TRY(cudaMalloc(&P->stage_y, sizeof(double2) * stage));
  AIM_CUDA_TRY(cudaMalloc(&c->p32.xbuf, sizeof(float2) * P->B * (size_t)P->ld));
  AIM_CUDA_TRY(cudaMalloc(&c->p32.ybuf, sizeof(float2) * P->B * (size_t)P->ld));
  AIM_TRY(ensure_grids(c, AIM_C64));
  AIM_CUDA_TRY(cudaStreamSynchronize(st));
  return AIM_OK;
}

}  // namespace aim

using namespace aim;

int aim_pack_create(aim_ctx* const* ctxs, int K, const int32_t* nrhs, aim_pack** out) {
  if (!ctxs || !nrhs || !out || K < 1 || K > 256) {
    set_error("aim_pack_create: need 1 <= K <= 256 and non-null ctxs, nrhs, out");
    return AIM_EINVAL;
  }
  *out = nullptr;
  long long B = 0;
  int ld = 0;
  for (int i = 0; i < K; ++i) {
    const aim_ctx* ci = ctxs[i];
    if (!ci || ci->pack) {
      set_error("aim_pack_create: context " + std::to_string(i) + " is null or a pack's own");
      return AIM_EINVAL;
    }
    if (nrhs[i] < 1 || nrhs[i] > ci->max_rhs) {
      set_error("aim_pack_create: nrhs[" + std::to_string(i) + "] must be in 1 .. max_rhs of its context");
      return AIM_EINVAL;
    }
    const aim_ctx* c0 = ctxs[0];
    if (ci->device != c0->device || ci->k != c0->k || ci->h != c0->h || ci->M != c0->M || ci->S != c0->S ||
        ci->planar != c0->planar) {
      set_error("aim_pack_create: context " + std::to_string(i) +
                " differs from the first in device, k, h, M or stencil layout");
      return AIM_EINVAL;
    }
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ci) {
        set_error("aim_pack_create: a context appears twice (give it more right-hand sides instead)");
        return AIM_EINVAL;
      }
    B += nrhs[i];
    ld = std::max(ld, ci->N);
  }
  if (B > 256) {
    set_error("aim_pack_create: at most 256 right-hand sides in total");
    return AIM_EINVAL;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != ctxs[0]->device) {
    set_error("aim_pack_create: the contexts' device must be current");
    return AIM_EINVAL;
  }
  aim_pack* P = new (std::nothrow) aim_pack();
  if (!P) return AIM_ENOMEM;
  P->pc = new (std::nothrow) aim_ctx();
  if (!P->pc) {
    delete P;
    return AIM_ENOMEM;
  }
  P->K = K;
  P->B = (int)B;
  P->ld = ld;
  P->inst.assign(ctxs, ctxs + K);
  P->nrhs.assign(nrhs, nrhs + K);
  P->b0.resize(K);
  for (int i = 0, b = 0; i < K; b += nrhs[i], ++i) {
    P->b0[i] = b;
    P->rows += ctxs[i]->N;
  }
  aim_ctx* c = P->pc;
  c->pack = P;
  c->opts = ctxs[0]->opts;
  c->opts.precision = AIM_C64;
  c->opts.max_rhs = P->B;
  c->opts.mem_budget = 0;
  c->max_rhs = P->B;
  c->N = ld;
  c->stream = ctxs[0]->stream;
  c->device = dev;
  int rc = AIM_OK;
  try {
    rc = build_pack(P);
  } catch (const std::bad_alloc&) {
    set_error("aim_pack_create: host allocation failed");
    rc = AIM_ENOMEM;
  }
  if (rc != AIM_OK) {
    if (rc == AIM_ECUDA && cudaGetLastError() == cudaErrorMemoryAllocation) rc = AIM_ENOMEM;
    free_pack(P);
    return rc;
  }
  *out = P;
  return AIM_OK;
}

int aim_pack_dims(const aim_pack* pack, int64_t* ld, int32_t* nrhs_total, int32_t* b0) {
  if (!pack) {
    set_error("null pack");
    return AIM_EINVAL;
  }
  if (ld) *ld = pack->ld;
  if (nrhs_total) *nrhs_total = pack->B;
  if (b0)
    for (int i = 0; i < pack->K; ++i) b0[i] = pack->b0[i];
  return AIM_OK;
}

int aim_pack_matvec(aim_pack* pack, const void* x_dev, void* y_dev, int precision) {
  if (!pack || !x_dev || !y_dev || x_dev == y_dev) {
    set_error("aim_pack_matvec: need a pack and distinct non-null x, y");
    return AIM_EINVAL;
  }
  if (precision != AIM_C64 && precision != AIM_C128 && precision != AIM_C128_F64) {
    set_error("aim_pack_matvec: precision must be AIM_C64, AIM_C128 or AIM_C128_F64");
    return AIM_EINVAL;
  }
  AIM_TRY(pack_prepare(pack->pc, precision));
  return pack_matvec(pack->pc, x_dev, y_dev, pack->B, precision);
}

int aim_pack_solve(aim_pack* pack, const void* V_dev, void* X_dev, double tol, aim_solve_info* info) {
  if (!pack || !V_dev || !X_dev || V_dev == X_dev || !(tol > 0.0)) {
    set_error("aim_pack_solve: need a pack, tol > 0 and distinct non-null V, X");
    return AIM_EINVAL;
  }
  return solve(pack->pc, (const double2*)V_dev, (double2*)X_dev, pack->B, tol, info);
}

int aim_pack_set_stream(aim_pack* pack, void* stream) {
  if (!pack) {
    set_error("null pack");
    return AIM_EINVAL;
  }
  pack->pc->stream = (cudaStream_t)stream;
  return AIM_OK;
}

void aim_pack_destroy(aim_pack* pack) { free_pack(pack); }
