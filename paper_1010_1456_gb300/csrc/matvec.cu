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
// Modes: M32 (complex64, FP32 accumulation) and M64 (complex128 throughout);
// the float-float product (complex128 vectors, float-float grids, weights and
// accumulation) has its own kernels below.
#include <algorithm>

#include <type_traits>

#include <climits>

#include "common.h"
#include "ff.h"
#include "geom.h"
#include "setup_dev.h"

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

// Warp tasks of the projection: task t is the 8 consecutive nodes of group
// g = groups[t] (or g = t when every group is a task), lane slot s of the
// warp's 8 takes node 8 g + s.  bounds() loads a node's entry range, empty for
// a node past the grid or a task past the end.
struct ProjTasks {
  const int32_t* groups;
  long long ntask, Nc;
  int slot;
  __device__ long long node(long long t) const { return 8LL * (groups ? (long long)groups[t] : t) + slot; }
  __device__ void bounds(const int32_t* __restrict__ ptr, long long t, int* e0, int* e1) const {
    *e0 = *e1 = 0;
    if (t < ntask) {
      const long long u = node(t);
      if (u < Nc) {
        *e0 = ptr[u];
        *e1 = ptr[u + 1];
      }
    }
  }
};

// One warp per task of 8 nodes, 4 lanes per node: the lanes take every
// fourth entry of the node's list (adjacent lanes read adjacent entries) and
// combine with warp shuffles.  Without a group list every group is a task
// and a warp whose 8 nodes have no entries only writes their zeros; with
// one, the unlisted groups are never written (they hold zeros from the
// start).  The next task's list bounds are loaded while the current one is
// summed, and the right-hand sides go in chunks of BC: an entry's weights
// and column are loaded once per chunk and its BC gathers of x are
// independent loads.
template <class MD, int BC>
__global__ void __launch_bounds__(256) proj_gather(const cplx<typename MD::R>* __restrict__ x, typename MD::S* __restrict__ Q,
                                                   const int32_t* __restrict__ ptr, const int32_t* __restrict__ mm,
                                                   const typename MD::R* __restrict__ w, int N, long long Nc, int nrhs,
                                                   const int32_t* __restrict__ groups, long long ntask) {
  using R = typename MD::R;
  using C = cplx<R>;
  const int lane = threadIdx.x & 3;
  const ProjTasks tasks{groups, ntask, Nc, (int)((threadIdx.x & 31) >> 2)};
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int pe0, pe1;
  tasks.bounds(ptr, t, &pe0, &pe1);
  // t is the same for the whole warp, so every lane takes part in the shuffles below
  for (; t < ntask; t += nwarps) {
    const long long u0 = tasks.node(t);
    const bool live = u0 < Nc;
    const long long u = live ? u0 : Nc - 1;
    const int e0 = pe0;
    int e1 = pe1;
#ifdef AIM_CHECK
    if (!indices_ok(mm, e0, e1, N, 1)) e1 = e0;
#endif
    tasks.bounds(ptr, t + nwarps, &pe0, &pe1);
    if (__all_sync(0xffffffffu, e0 == e1)) {  // the warp's 8 nodes are empty: zeros, no reduction
      if (live)
        for (int b = 0; b < nrhs; ++b) Q[(long long)b * 4 * Nc + (long long)lane * Nc + u] = MD::put(cmake<C>(0, 0));
      continue;
    }
    for (int b0 = 0; b0 < nrhs; b0 += BC) {
      C a[BC][4];
#pragma unroll
      for (int q = 0; q < BC; ++q)
#pragma unroll
        for (int c = 0; c < 4; ++c) a[q][c] = cmake<C>(0, 0);
      for (int e = e0 + lane; e < e1; e += 4) {
        const W4<R> ww = load_w4(w, e);
        const C* xc = x + mm[e];
        C xv[BC];
#pragma unroll
        for (int q = 0; q < BC; ++q) xv[q] = b0 + q < nrhs ? xc[(long long)(b0 + q) * N] : cmake<C>(0, 0);
#pragma unroll
        for (int q = 0; q < BC; ++q) {
          a[q][0].x += ww.x * xv[q].x; a[q][0].y += ww.x * xv[q].y;
          a[q][1].x += ww.y * xv[q].x; a[q][1].y += ww.y * xv[q].y;
          a[q][2].x += ww.z * xv[q].x; a[q][2].y += ww.z * xv[q].y;
          a[q][3].x += ww.w * xv[q].x; a[q][3].y += ww.w * xv[q].y;
        }
      }
#pragma unroll
      for (int q = 0; q < BC; ++q) {
#pragma unroll
        for (int o = 1; o < 4; o <<= 1)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            a[q][c].x += __shfl_xor_sync(0xffffffffu, a[q][c].x, o, 4);
            a[q][c].y += __shfl_xor_sync(0xffffffffu, a[q][c].y, o, 4);
          }
        if (live && b0 + q < nrhs) {
          // lane c writes component c (one conversion per value)
          const C val = lane == 0 ? a[q][0] : lane == 1 ? a[q][1] : lane == 2 ? a[q][2] : a[q][3];
          Q[(long long)(b0 + q) * 4 * Nc + (long long)lane * Nc + u] = MD::put(val);
        }
      }
    }
  }
}

// Grid-index offset of each stencil node s = (kk P + j) P + i from the
// stencil's first node, staged once per block (S <= 216 for M <= 5).
__device__ __forceinline__ void stencil_offsets_smem(int* s_off, int S, int P, int nx, int ny) {
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    const int i = s % P, j = (s / P) % P, kk = s / (P * P);
    s_off[s] = (kk * ny + j) * nx + i;
  }
  __syncthreads();
}
constexpr int kMaxStencil = 216;

// 8 lanes per basis function.
template <class MD, bool MF>
__global__ void __launch_bounds__(256) interp_near(const typename MD::S* __restrict__ Phi,
                                                   const cplx<typename MD::R>* __restrict__ x,
                                                   cplx<typename MD::R>* __restrict__ y,
                                                   const typename MD::R* __restrict__ lam,
                                                   const int32_t* __restrict__ base, const int32_t* __restrict__ nptr,
                                                   const int32_t* __restrict__ ncol,
                                                   const cplx<typename MD::R>* __restrict__ nval, int N, long long Nc,
                                                   int nx, int ny, int nrhs, typename MD::R fvec, typename MD::R frho,
                                                   int S, int P, const typename MD::R* __restrict__ lamM,
                                                   typename MD::R fmf) {
  using R = typename MD::R;
  using C = cplx<R>;
  __shared__ int s_off[kMaxStencil];
  stencil_offsets_smem(s_off, S, P, nx, ny);
  const int lane = threadIdx.x & 7;
  const int m = (blockIdx.x * blockDim.x + threadIdx.x) >> 3;
  const bool live = m < N;
  const int mm = live ? m : N - 1;
  const int b0 = base[mm];
  const R* lm = lam + (long long)mm * 4 * S;
  const R* wm = MF ? lamM + (long long)mm * 3 * S : nullptr;
  const int r0 = nptr[mm];
  int r1 = nptr[mm + 1];
#ifdef AIM_CHECK
  const int Sc = stencil_ok(b0, nx, ny, Nc, P, S, 2) ? S : 0;
  if (!indices_ok(ncol, r0, r1, N, 3)) r1 = r0;
#else
  const int Sc = S;
#endif
  for (int b = 0; b < nrhs; ++b) {
    const typename MD::S* Pb = Phi + (long long)b * 4 * Nc;
    C av = cmake<C>(0, 0), ar = av, an = av, am = av;
    for (int s = lane; s < Sc; s += 8) {
      const long long node = b0 + (long long)s_off[s];
      const C px = MD::get(Pb[node]), py = MD::get(Pb[Nc + node]), pz = MD::get(Pb[2 * Nc + node]),
              pr = MD::get(Pb[3 * Nc + node]);
      const R wx = lm[s], wy = lm[S + s], wz = lm[2 * S + s], wr = lm[3 * S + s];
      av.x += wx * px.x + wy * py.x + wz * pz.x;
      av.y += wx * px.y + wy * py.y + wz * pz.y;
      ar.x += wr * pr.x;
      ar.y += wr * pr.y;
      if constexpr (MF) {
        const R mx = wm[s], my = wm[S + s], mz = wm[2 * S + s];
        am.x += mx * px.x + my * py.x + mz * pz.x;
        am.y += mx * px.y + my * py.y + mz * pz.y;
      }
    }
    const C* xb = x + (long long)b * N;
    for (int e = r0 + lane; e < r1; e += 8) {
      const C v = nval[e], xv = xb[ncol[e]];
      an.x += v.x * xv.x - v.y * xv.y;
      an.y += v.x * xv.y + v.y * xv.x;
    }
    // grid part: j (fvec av - frho ar) - fmf am  with fvec = alpha k eta,
    // frho = alpha eta / k, fmf = (1 - alpha) eta (am: the MFIE weights' sum)
    C t;
    t.x = fvec * av.x - frho * ar.x;
    t.y = fvec * av.y - frho * ar.y;
    C out;
    out.x = an.x - t.y;
    out.y = an.y + t.x;
    if constexpr (MF) {
      out.x -= fmf * am.x;
      out.y -= fmf * am.y;
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
      out.x += __shfl_xor_sync(0xffffffffu, out.x, o, 8);
      out.y += __shfl_xor_sync(0xffffffffu, out.y, o, 8);
    }
    if (live && lane == 0) y[(long long)b * N + m] = out;
  }
}

// out[c][r] = in[r][c] for an R x Cn row-major matrix (32 x 32 tiles through
// shared memory, so both the reads and the writes are coalesced).
template <class E>
__global__ void __launch_bounds__(256) k_transpose(const E* __restrict__ in, E* __restrict__ out, int R, long long Cn) {
  __shared__ E t[32][33];
  const long long c0 = blockIdx.x * 32LL;
  const int r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int r = r0 + i;
    const long long cc = c0 + threadIdx.x;
    if (r < R && cc < Cn) t[i][threadIdx.x] = in[(long long)r * Cn + cc];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const long long cc = c0 + i;
    const int r = r0 + threadIdx.x;
    if (r < R && cc < Cn) out[cc * R + r] = t[threadIdx.x][i];
  }
}

template <class E>
static int transpose(aim_ctx* c, const char* name, const E* in, E* out, int R, long long Cn) {
  dim3 grid((unsigned)((Cn + 31) / 32), (unsigned)((R + 31) / 32));
  AIM_LAUNCH(c, name, (k_transpose<E><<<grid, dim3(32, 8), 0, c->stream>>>(in, out, R, Cn)));
  return launch_check(c, name);
}

// RL consecutive complex values as one load (16 bytes for two complex64).
template <class C, int RL> struct Run {
  C v[RL];
};
template <class C, int RL> __device__ __forceinline__ Run<C, RL> load_run(const C* p) {
  Run<C, RL> r;
  if constexpr (RL == 2 && sizeof(C) == 8) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    r.v[0] = cmake<C>(q.x, q.y);
    r.v[1] = cmake<C>(q.z, q.w);
  } else {
#pragma unroll
    for (int i = 0; i < RL; ++i) r.v[i] = p[i];
  }
  return r;
}

// ---- row groups of the many-RHS near product ----
// Group g holds rows m0 = kNearGroup g .. m0 + kNearGroup - 1 (the last one
// fewer).  Its near columns are the sorted union of the rows' (sorted)
// columns; for each union column the group stores kNearGroup entries, the
// rows' own values or zero.  One thread per group walks the rows' lists
// together (a merge); FILL = false counts the union, FILL = true writes it.
template <bool FILL, class C>
__global__ void k_near_groups(const int32_t* __restrict__ nptr, const int32_t* __restrict__ ncol,
                              const C* __restrict__ nval, int N, long long ngroups, int32_t* __restrict__ cnt_or_ptr,
                              int32_t* __restrict__ gcol, C* __restrict__ gval) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= ngroups) return;
  const int m0 = (int)(g * kNearGroup);
  int p[kNearGroup], e[kNearGroup];
#pragma unroll
  for (int r = 0; r < kNearGroup; ++r) {
    const bool row = m0 + r < N;
    p[r] = row ? nptr[m0 + r] : 0;
    e[r] = row ? nptr[m0 + r + 1] : 0;
  }
  long long u = FILL ? cnt_or_ptr[g] : 0;
  for (;;) {
    int col = INT_MAX;
#pragma unroll
    for (int r = 0; r < kNearGroup; ++r)
      if (p[r] < e[r]) col = min(col, ncol[p[r]]);
    if (col == INT_MAX) break;
    if constexpr (FILL) gcol[u] = col;
#pragma unroll
    for (int r = 0; r < kNearGroup; ++r) {
      const bool has = p[r] < e[r] && ncol[p[r]] == col;
      if constexpr (FILL) gval[u * kNearGroup + r] = has ? nval[p[r]] : cmake<C>(0, 0);
      if (has) ++p[r];
    }
    ++u;
  }
  if constexpr (!FILL) cnt_or_ptr[g] = (int32_t)u;
}

// The group's kNearGroup entries of union column u (one 32-byte row for complex64).
template <class C> struct GroupVals {
  C v[kNearGroup];
};
__device__ __forceinline__ GroupVals<float2> load_group(const float2* p) {
  const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
  return GroupVals<float2>{{make_float2(a.x, a.y), make_float2(a.z, a.w), make_float2(b.x, b.y), make_float2(b.z, b.w)}};
}
__device__ __forceinline__ GroupVals<double2> load_group(const double2* p) {
  return GroupVals<double2>{{p[0], p[1], p[2], p[3]}};
}
static_assert(kNearGroup == 4, "load_group reads four entries");

// Interpolation + near correction for many right-hand sides over groups of
// kNearGroup consecutive basis functions: one warp per group, lanes over
// right-hand sides (RL consecutive ones per lane) on RHS-minor Phi and x.
// The grid part runs row by row (each stencil node's four grid values are
// contiguous runs of right-hand sides; weights warp-uniform); the near part walks
// the group's union of columns, so each x run is gathered once per group
// rather than once per row that holds the column (neighbouring basis
// functions share most of their near zone), at the price of multiplying the
// zeros of the rows that lack a column.  The block's 32 rows of y are staged
// in shared memory and written back in the [B][N] layout.
template <class MI, int RL, bool MF>
__global__ void __launch_bounds__(256) interp_near_grp(const cplx<typename MI::R>* __restrict__ PhiT,
                                                       const cplx<typename MI::R>* __restrict__ xT,
                                                       cplx<typename MI::R>* __restrict__ y,
                                                       const typename MI::R* __restrict__ lam,
                                                       const int32_t* __restrict__ base,
                                                       const int32_t* __restrict__ gptr,
                                                       const int32_t* __restrict__ gcol,
                                                       const cplx<typename MI::R>* __restrict__ gval, int N,
                                                       long long Nc, int nx, int ny, int B, typename MI::R fvec,
                                                       typename MI::R frho, int S, int P,
                                                       const typename MI::R* __restrict__ lamM, typename MI::R fmf) {
  using R = typename MI::R;
  using C = cplx<R>;
  constexpr int G = kNearGroup;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* ys = reinterpret_cast<C*>(smem_raw);  // [8 G][B + 1] (a padded row: the write-back reads down a column)
  const int YS = B + 1;
  __shared__ int s_off[kMaxStencil];
  stencil_offsets_smem(s_off, S, P, nx, ny);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long g = blockIdx.x * 8LL + warp;
  const int m0 = (int)(g * G);
  if (m0 < N) {
    const int nr = min(G, N - m0);
    const int u0 = gptr[g];
    int u1 = gptr[g + 1];
#ifdef AIM_CHECK
    if (!indices_ok(gcol, u0, u1, N, 3)) u1 = u0;
#endif
    const long long cs = Nc * B;  // component stride of PhiT
    for (int bc = 0; bc < B; bc += 32 * RL) {
      const int b = bc + RL * lane;  // B is a multiple of RL
      if (b >= B) continue;
      C acc[G][RL];
#pragma unroll
      for (int r = 0; r < G; ++r)
#pragma unroll
        for (int q = 0; q < RL; ++q) acc[r][q] = cmake<C>(0, 0);
      // grid part, row by row: j (fvec av - frho ar) - fmf am
#pragma unroll
      for (int r = 0; r < G; ++r) {
        if (r >= nr) break;
        const int m = m0 + r;
        const int b0 = base[m];
#ifdef AIM_CHECK
        const int Sc = stencil_ok(b0, nx, ny, Nc, P, S, 2) ? S : 0;
#else
        const int Sc = S;
#endif
        const R* lm = lam + (long long)m * 4 * S;
        const R* wm = MF ? lamM + (long long)m * 3 * S : nullptr;
        C av[RL], ar[RL], am[RL];
#pragma unroll
        for (int q = 0; q < RL; ++q) av[q] = ar[q] = am[q] = cmake<C>(0, 0);
#pragma unroll 3
        for (int s = 0; s < Sc; ++s) {
          const C* ph = PhiT + (b0 + (long long)s_off[s]) * B + b;
          const Run<C, RL> px = load_run<C, RL>(ph), py = load_run<C, RL>(ph + cs), pz = load_run<C, RL>(ph + 2 * cs),
                           pr = load_run<C, RL>(ph + 3 * cs);
          const R wx = lm[s], wy = lm[S + s], wz = lm[2 * S + s], wr = lm[3 * S + s];
#pragma unroll
          for (int q = 0; q < RL; ++q) {
            av[q].x += wx * px.v[q].x + wy * py.v[q].x + wz * pz.v[q].x;
            av[q].y += wx * px.v[q].y + wy * py.v[q].y + wz * pz.v[q].y;
            ar[q].x += wr * pr.v[q].x;
            ar[q].y += wr * pr.v[q].y;
          }
          if constexpr (MF) {
            const R mx = wm[s], my = wm[S + s], mz = wm[2 * S + s];
#pragma unroll
            for (int q = 0; q < RL; ++q) {
              am[q].x += mx * px.v[q].x + my * py.v[q].x + mz * pz.v[q].x;
              am[q].y += mx * px.v[q].y + my * py.v[q].y + mz * pz.v[q].y;
            }
          }
        }
#pragma unroll
        for (int q = 0; q < RL; ++q) {
          const R tx = fvec * av[q].x - frho * ar[q].x, ty = fvec * av[q].y - frho * ar[q].y;
          acc[r][q].x = -ty;
          acc[r][q].y = tx;
          if constexpr (MF) {
            acc[r][q].x -= fmf * am[q].x;
            acc[r][q].y -= fmf * am[q].y;
          }
        }
      }
      // near part over the group's union of columns, EB columns in flight
      constexpr int EB = 4;
      int u = u0;
      for (; u + EB <= u1; u += EB) {
        int col[EB];
#pragma unroll
        for (int i = 0; i < EB; ++i) col[i] = gcol[u + i];
        Run<C, RL> xv[EB];
#pragma unroll
        for (int i = 0; i < EB; ++i) xv[i] = load_run<C, RL>(xT + (long long)col[i] * B + b);
#pragma unroll
        for (int i = 0; i < EB; ++i) {
          const GroupVals<C> gv = load_group(gval + (long long)(u + i) * G);
#pragma unroll
          for (int r = 0; r < G; ++r) {
            const C v = gv.v[r];
#pragma unroll
            for (int q = 0; q < RL; ++q) {
              acc[r][q].x += v.x * xv[i].v[q].x - v.y * xv[i].v[q].y;
              acc[r][q].y += v.x * xv[i].v[q].y + v.y * xv[i].v[q].x;
            }
          }
        }
      }
      for (; u < u1; ++u) {
        const Run<C, RL> xv = load_run<C, RL>(xT + (long long)gcol[u] * B + b);
        const GroupVals<C> gv = load_group(gval + (long long)u * G);
#pragma unroll
        for (int r = 0; r < G; ++r) {
          const C v = gv.v[r];
#pragma unroll
          for (int q = 0; q < RL; ++q) {
            acc[r][q].x += v.x * xv.v[q].x - v.y * xv.v[q].y;
            acc[r][q].y += v.x * xv.v[q].y + v.y * xv.v[q].x;
          }
        }
      }
#pragma unroll
      for (int r = 0; r < G; ++r)
#pragma unroll
        for (int q = 0; q < RL; ++q) ys[(warp * G + r) * YS + b + q] = acc[r][q];
    }
  }
  __syncthreads();
  const long long mb = blockIdx.x * 8LL * G;
  const int rows = (int)min(8LL * G, (long long)N - mb);
  for (int t = threadIdx.x; t < 8 * G * B; t += blockDim.x) {
    const int i = t % (8 * G), bb = t / (8 * G);
    if (i < rows) y[(long long)bb * N + mb + i] = ys[i * YS + bb];
  }
}

// Projection for many right-hand sides: one warp per grid node, lanes over
// right-hand sides (RL consecutive ones per lane) on the RHS-minor x, so each
// entry's x values are one contiguous run; the entry's four weights are
// warp-uniform.  A block's 32 nodes are staged in shared memory (node-major,
// rows padded by one element against bank conflicts) and written back in the
// [B][4][Nc] layout, 32 consecutive nodes per (RHS, component) row.  One
// launch covers B right-hand sides of an x with ldx of them per row.
template <class MD, int RL>
__global__ void __launch_bounds__(256) proj_gather_rhs(const cplx<typename MD::R>* __restrict__ xT,
                                                       typename MD::S* __restrict__ Q, const int32_t* __restrict__ ptr,
                                                       const int32_t* __restrict__ mm,
                                                       const typename MD::R* __restrict__ w, long long Nc, int B,
                                                       int ldx, int N) {
  using R = typename MD::R;
  using C = cplx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* qs = reinterpret_cast<C*>(smem_raw);  // [32][4 B + 1]
  const int NS = 4 * B + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long u0 = blockIdx.x * 32LL;
  for (int i = warp; i < 32; i += 8) {
    const long long u = u0 + i;
    if (u >= Nc) break;
    const int e0 = ptr[u];
    int e1 = ptr[u + 1];
#ifdef AIM_CHECK
    if (!indices_ok(mm, e0, e1, N, 1)) e1 = e0;
#endif
    for (int bc = 0; bc < B; bc += 32 * RL) {
      const int b = bc + RL * lane;  // B is a multiple of RL
      if (b >= B) continue;
      C a[4][RL];
#pragma unroll
      for (int cc = 0; cc < 4; ++cc)
#pragma unroll
        for (int q = 0; q < RL; ++q) a[cc][q] = cmake<C>(0, 0);
      // entries in batches of EB: the batch's columns, then its EB gathers of x, in flight together
      constexpr int EB = 4;
      const auto add = [&](const W4<R>& ww, const Run<C, RL>& xv) {
#pragma unroll
        for (int q = 0; q < RL; ++q) {
          a[0][q].x += ww.x * xv.v[q].x; a[0][q].y += ww.x * xv.v[q].y;
          a[1][q].x += ww.y * xv.v[q].x; a[1][q].y += ww.y * xv.v[q].y;
          a[2][q].x += ww.z * xv.v[q].x; a[2][q].y += ww.z * xv.v[q].y;
          a[3][q].x += ww.w * xv.v[q].x; a[3][q].y += ww.w * xv.v[q].y;
        }
      };
      int e = e0;
      for (; e + EB <= e1; e += EB) {
        int col[EB];
#pragma unroll
        for (int i = 0; i < EB; ++i) col[i] = mm[e + i];
        Run<C, RL> xv[EB];
#pragma unroll
        for (int i = 0; i < EB; ++i) xv[i] = load_run<C, RL>(xT + (long long)col[i] * ldx + b);
#pragma unroll
        for (int i = 0; i < EB; ++i) add(load_w4(w, e + i), xv[i]);
      }
      for (; e < e1; ++e) add(load_w4(w, e), load_run<C, RL>(xT + (long long)mm[e] * ldx + b));
#pragma unroll
      for (int cc = 0; cc < 4; ++cc)
#pragma unroll
        for (int q = 0; q < RL; ++q) qs[i * NS + cc * B + b + q] = a[cc][q];
    }
  }
  __syncthreads();
  const int nodes = (int)min(32LL, Nc - u0);
  for (int t = threadIdx.x; t < 32 * 4 * B; t += blockDim.x) {
    const int i = t & 31, row = t >> 5;  // row = b * 4 + component
    const int b = row >> 2, cc = row & 3;
    if (i < nodes) Q[((long long)b * 4 + cc) * Nc + u0 + i] = MD::put(qs[i * NS + cc * B + b]);
  }
}


// ---- float-float projection and interpolation (AIM_C128) ----
// The FP64-accurate product keeps its grids in float-float form for the FFT
// passes; these kernels do the projection, interpolation and near SpMV in the
// same arithmetic on the FP32 pipes (GB300 retires about 64 FP32 FMAs for
// every FP64 FMA), with weights and near entries rounded once to float-float
// at the first product.  Only the input and the output vectors are FP64.

__device__ __forceinline__ ff ffv(float hi, float lo) { return ff{hi, lo}; }

__global__ void k_real_to_ff(const double* __restrict__ in, float2* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const ff v = ff_from_double(in[i]);
    out[i] = make_float2(v.hi, v.lo);
  }
}
__global__ void k_cplx_to_ff(const double2* __restrict__ in, float4* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const ff re = ff_from_double(in[i].x), im = ff_from_double(in[i].y);
    out[i] = make_float4(re.hi, re.lo, im.hi, im.lo);
  }
}
// [nent][4] FP64 weights -> [nent][2] float4: high parts, then low parts.
__global__ void k_w4_to_ff(const double* __restrict__ in, float4* __restrict__ out, long long nent) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nent;
       e += (long long)gridDim.x * blockDim.x) {
    const ff a = ff_from_double(in[4 * e]), b = ff_from_double(in[4 * e + 1]), c = ff_from_double(in[4 * e + 2]),
             d = ff_from_double(in[4 * e + 3]);
    out[2 * e] = make_float4(a.hi, b.hi, c.hi, d.hi);
    out[2 * e + 1] = make_float4(a.lo, b.lo, c.lo, d.lo);
  }
}

// Projection with float-float arithmetic: the tasks, layout and order of
// proj_gather (4 lanes per node, empty warps write zeros, next bounds
// prefetched, right-hand sides in chunks of BC).
template <int BC>
__global__ void __launch_bounds__(256) proj_gather_ff(const float4* __restrict__ x, float4* __restrict__ Q,
                                                      const int32_t* __restrict__ ptr, const int32_t* __restrict__ mm,
                                                      const float4* __restrict__ w, int N, long long Nc, int nrhs,
                                                      const int32_t* __restrict__ groups, long long ntask) {
  const int lane = threadIdx.x & 3;
  const ProjTasks tasks{groups, ntask, Nc, (int)((threadIdx.x & 31) >> 2)};
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int pe0, pe1;
  tasks.bounds(ptr, t, &pe0, &pe1);
  for (; t < ntask; t += nwarps) {
    const long long u0 = tasks.node(t);
    const bool live = u0 < Nc;
    const long long u = live ? u0 : Nc - 1;
    const int e0 = pe0;
    int e1 = pe1;
#ifdef AIM_CHECK
    if (!indices_ok(mm, e0, e1, N, 1)) e1 = e0;
#endif
    tasks.bounds(ptr, t + nwarps, &pe0, &pe1);
    if (__all_sync(0xffffffffu, e0 == e1)) {  // the warp's 8 nodes are empty: zeros, no reduction
      if (live)
        for (int b = 0; b < nrhs; ++b) Q[(long long)b * 4 * Nc + (long long)lane * Nc + u] = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    for (int b0 = 0; b0 < nrhs; b0 += BC) {
      ff a[BC][4][2];
#pragma unroll
      for (int q = 0; q < BC; ++q)
#pragma unroll
        for (int c = 0; c < 4; ++c) a[q][c][0] = a[q][c][1] = ffv(0.f, 0.f);
      for (int e = e0 + lane; e < e1; e += 4) {
        const float4 wh = w[2 * e], wl = w[2 * e + 1];
        const float4* xc = x + mm[e];
        float4 xv[BC];
#pragma unroll
        for (int q = 0; q < BC; ++q) xv[q] = b0 + q < nrhs ? xc[(long long)(b0 + q) * N] : make_float4(0.f, 0.f, 0.f, 0.f);
        const ff wc[4] = {ffv(wh.x, wl.x), ffv(wh.y, wl.y), ffv(wh.z, wl.z), ffv(wh.w, wl.w)};
#pragma unroll
        for (int q = 0; q < BC; ++q) {
          const ff xr = ffv(xv[q].x, xv[q].y), xi = ffv(xv[q].z, xv[q].w);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            a[q][c][0] = ff_mad(wc[c], xr, a[q][c][0]);
            a[q][c][1] = ff_mad(wc[c], xi, a[q][c][1]);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < BC; ++q) {
#pragma unroll
        for (int o = 1; o < 4; o <<= 1)
#pragma unroll
          for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int r = 0; r < 2; ++r) {
              const ff t = ffv(__shfl_xor_sync(0xffffffffu, a[q][c][r].hi, o, 4),
                               __shfl_xor_sync(0xffffffffu, a[q][c][r].lo, o, 4));
              a[q][c][r] = ff_add(a[q][c][r], t);
            }
        if (live && b0 + q < nrhs) {
          // lane c writes component c
          ff re = a[q][0][0], im = a[q][0][1];
#pragma unroll
          for (int c = 1; c < 4; ++c)
            if (lane == c) {
              re = a[q][c][0];
              im = a[q][c][1];
            }
          Q[(long long)(b0 + q) * 4 * Nc + (long long)lane * Nc + u] = make_float4(re.hi, re.lo, im.hi, im.lo);
        }
      }
    }
  }
}

// Interpolation + near correction: 8 lanes per basis function, as interp_near.
template <bool MF>
__global__ void __launch_bounds__(256) interp_near_ff(const float4* __restrict__ Phi, const float4* __restrict__ x,
                                                      double2* __restrict__ y, const float2* __restrict__ lam,
                                                      const int32_t* __restrict__ base, const int32_t* __restrict__ nptr,
                                                      const int32_t* __restrict__ ncol,
                                                      const float4* __restrict__ nval, int N, long long Nc, int nx,
                                                      int ny, int nrhs, float2 fvec, float2 frho, int S, int P,
                                                      const float2* __restrict__ lamM, float2 fmf) {
  __shared__ int s_off[kMaxStencil];
  stencil_offsets_smem(s_off, S, P, nx, ny);
  const int lane = threadIdx.x & 7;
  const int m = (blockIdx.x * blockDim.x + threadIdx.x) >> 3;
  const bool live = m < N;
  const int mm = live ? m : N - 1;
  const int b0 = base[mm];
  const float2* lm = lam + (long long)mm * 4 * S;
  const float2* wm = MF ? lamM + (long long)mm * 3 * S : nullptr;
  const int r0 = nptr[mm];
  int r1 = nptr[mm + 1];
#ifdef AIM_CHECK
  const int Sc = stencil_ok(b0, nx, ny, Nc, P, S, 2) ? S : 0;
  if (!indices_ok(ncol, r0, r1, N, 3)) r1 = r0;
#else
  const int Sc = S;
#endif
  const ff kv = ffv(fvec.x, fvec.y), kr = ffv(frho.x, frho.y), km = ffv(fmf.x, fmf.y);
  for (int b = 0; b < nrhs; ++b) {
    const float4* Pb = Phi + (long long)b * 4 * Nc;
    ff avr = ffv(0.f, 0.f), avi = avr, arr = avr, ari = avr, anr = avr, ani = avr, amr = avr, ami = avr;
    for (int s = lane; s < Sc; s += 8) {
      const long long node = b0 + (long long)s_off[s];
      const float4 px = Pb[node], py = Pb[Nc + node], pz = Pb[2 * Nc + node], pr = Pb[3 * Nc + node];
      const float2 wx = lm[s], wy = lm[S + s], wz = lm[2 * S + s], wr = lm[3 * S + s];
      avr = ff_mad(ffv(wx.x, wx.y), ffv(px.x, px.y), avr);
      avi = ff_mad(ffv(wx.x, wx.y), ffv(px.z, px.w), avi);
      avr = ff_mad(ffv(wy.x, wy.y), ffv(py.x, py.y), avr);
      avi = ff_mad(ffv(wy.x, wy.y), ffv(py.z, py.w), avi);
      avr = ff_mad(ffv(wz.x, wz.y), ffv(pz.x, pz.y), avr);
      avi = ff_mad(ffv(wz.x, wz.y), ffv(pz.z, pz.w), avi);
      arr = ff_mad(ffv(wr.x, wr.y), ffv(pr.x, pr.y), arr);
      ari = ff_mad(ffv(wr.x, wr.y), ffv(pr.z, pr.w), ari);
      if constexpr (MF) {
        const float2 mx = wm[s], my = wm[S + s], mz = wm[2 * S + s];
        amr = ff_mad(ffv(mx.x, mx.y), ffv(px.x, px.y), amr);
        ami = ff_mad(ffv(mx.x, mx.y), ffv(px.z, px.w), ami);
        amr = ff_mad(ffv(my.x, my.y), ffv(py.x, py.y), amr);
        ami = ff_mad(ffv(my.x, my.y), ffv(py.z, py.w), ami);
        amr = ff_mad(ffv(mz.x, mz.y), ffv(pz.x, pz.y), amr);
        ami = ff_mad(ffv(mz.x, mz.y), ffv(pz.z, pz.w), ami);
      }
    }
    const float4* xb = x + (long long)b * N;
    for (int e = r0 + lane; e < r1; e += 8) {
      const float4 v = nval[e], xv = xb[ncol[e]];
      const ff vr = ffv(v.x, v.y), vi = ffv(v.z, v.w), xr = ffv(xv.x, xv.y), xi = ffv(xv.z, xv.w);
      anr = ff_mad(vr, xr, anr);
      anr = ff_mad(ff_neg(vi), xi, anr);
      ani = ff_mad(vr, xi, ani);
      ani = ff_mad(vi, xr, ani);
    }
    // grid part j (fvec av - frho ar): out = an + j t
    const ff tr = ff_sub(ff_mul(kv, avr), ff_mul(kr, arr));
    const ff ti = ff_sub(ff_mul(kv, avi), ff_mul(kr, ari));
    ff outr = ff_sub(anr, ti), outi = ff_add(ani, tr);
    if constexpr (MF) {
      outr = ff_sub(outr, ff_mul(km, amr));
      outi = ff_sub(outi, ff_mul(km, ami));
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
      outr = ff_add(outr, ffv(__shfl_xor_sync(0xffffffffu, outr.hi, o, 8), __shfl_xor_sync(0xffffffffu, outr.lo, o, 8)));
      outi = ff_add(outi, ffv(__shfl_xor_sync(0xffffffffu, outi.hi, o, 8), __shfl_xor_sync(0xffffffffu, outi.lo, o, 8)));
    }
    if (live && lane == 0) y[(long long)b * N + m] = make_double2(ff_to_double(outr), ff_to_double(outi));
  }
}

// Warp tasks of the projection: the listed groups, or every 8-node group.
static long long proj_tasks(const aim_ctx* c, long long Nc) { return c->sparse_proj ? c->ngroups : (Nc + 7) / 8; }

static int ensure_ff_arrays(aim_ctx* c) {
  FFData& p = c->pff;
  if (p.pnode_w) return AIM_OK;
  const long long nent = c->nent, nl = (long long)c->N * 4 * c->S;
  AIM_CUDA_TRY(cudaMalloc(&p.pnode_w, sizeof(float4) * 2 * nent));
  AIM_CUDA_TRY(cudaMalloc(&p.lam, sizeof(float2) * nl));
  AIM_CUDA_TRY(cudaMalloc(&p.near_val, sizeof(float4) * std::max<long long>(1, c->nnz)));
  AIM_CUDA_TRY(cudaMalloc(&p.xff, sizeof(float4) * c->max_rhs * c->N));
  const int blocks = 152 * 8;
  AIM_LAUNCH(c, "weights_to_ff", (k_w4_to_ff<<<blocks, 256, 0, c->stream>>>(c->p64.pnode_w, p.pnode_w, nent)));
  AIM_TRY(launch_check(c, "weights_to_ff"));
  AIM_LAUNCH(c, "weights_to_ff", (k_real_to_ff<<<blocks, 256, 0, c->stream>>>(c->p64.lam, p.lam, nl)));
  AIM_TRY(launch_check(c, "weights_to_ff"));
  if (c->p64.lamM) {
    const long long nm = (long long)c->N * 3 * c->S;
    AIM_CUDA_TRY(cudaMalloc(&p.lamM, sizeof(float2) * nm));
    AIM_LAUNCH(c, "weights_to_ff", (k_real_to_ff<<<blocks, 256, 0, c->stream>>>(c->p64.lamM, p.lamM, nm)));
    AIM_TRY(launch_check(c, "weights_to_ff"));
  }
  if (c->nnz > 0) {
    AIM_LAUNCH(c, "weights_to_ff", (k_cplx_to_ff<<<blocks, 256, 0, c->stream>>>(c->p64.near_val, p.near_val, c->nnz)));
    AIM_TRY(launch_check(c, "weights_to_ff"));
  }
  return AIM_OK;
}

static int run_product_ff(aim_ctx* c, const double2* x, double2* y, int nrhs) {
  AIM_TRY(ensure_ff_arrays(c));
  FFData& p = c->pff;
  const long long Nc = (long long)c->n[0] * c->n[1] * c->n[2];
  const long long nx_ = (long long)nrhs * c->N;
  {
    const int blocks = (int)std::min<long long>((nx_ + 255) / 256, 152LL * 8);
    AIM_LAUNCH(c, "x_to_ff", (k_cplx_to_ff<<<blocks, 256, 0, c->stream>>>(x, p.xff, nx_)));
    AIM_TRY(launch_check(c, "x_to_ff"));
  }
  {
    const long long ntask = proj_tasks(c, Nc);
    const int blocks = (int)std::min<long long>((ntask + 7) / 8, 152LL * 16);
    const int32_t* groups = c->sparse_proj ? c->pgroups : nullptr;
    const auto go = [&](auto bc) {
      AIM_LAUNCH(c, "proj_gather",
                 (proj_gather_ff<decltype(bc)::value><<<blocks, 256, 0, c->stream>>>(p.xff, p.grid0, c->pnode_ptr,
                                                                                      c->pnode_m, p.pnode_w, c->N, Nc,
                                                                                      nrhs, groups, ntask)));
    };
    if (nrhs == 1) go(std::integral_constant<int, 1>{});
    else if (nrhs == 2) go(std::integral_constant<int, 2>{});
    else go(std::integral_constant<int, 4>{});
    AIM_TRY(launch_check(c, "proj_gather"));
  }
  AIM_TRY(fft_convolve_ff(c, 4 * nrhs));
  {
    const long long threads = (long long)c->N * 8;
    const int blocks = (int)((threads + 255) / 256);
    const double fv = c->alpha * c->k * kEta0, fr = c->alpha * kEta0 / c->k, fm = (1.0 - c->alpha) * kEta0;
    const float fvh = (float)fv, frh = (float)fr, fmh = (float)fm;
    const float2 fvec = make_float2(fvh, (float)(fv - (double)fvh)), frho = make_float2(frh, (float)(fr - (double)frh));
    const float2 fmf = make_float2(fmh, (float)(fm - (double)fmh));
    const auto go = [&](auto mf) {
      AIM_LAUNCH(c, "interp_near",
             (interp_near_ff<decltype(mf)::value><<<blocks, 256, 0, c->stream>>>(phi_grid(c, p.grid0, p.grid2), p.xff, y, p.lam, c->base, c->near_ptr,
                                                                c->near_col, p.near_val, c->N, Nc, c->n[0], c->n[1],
                                                                nrhs, fvec, frho, c->S, c->M + 1, p.lamM, fmf)));
    };
    if (p.lamM) go(std::true_type{}); else go(std::false_type{});

    AIM_TRY(launch_check(c, "interp_near"));
  }
  return AIM_OK;
}

template <typename R> PrecData<R>& prec_data(aim_ctx* c);
template <> PrecData<float>& prec_data<float>(aim_ctx* c) { return c->p32; }
template <> PrecData<double>& prec_data<double>(aim_ctx* c) { return c->p64; }

// The row groups of the many-RHS near product: the union columns once, the
// entries of a precision on its first use.
template <typename R>
static int ensure_near_groups(aim_ctx* c, PrecData<R>& pd) {
  const long long ng = ((long long)c->N + kNearGroup - 1) / kNearGroup;
  const unsigned blocks = (unsigned)((ng + 255) / 256);
  if (!c->ngrp_ptr) {
    AIM_CUDA_TRY(cudaMalloc(&c->ngrp_ptr, sizeof(int32_t) * (ng + 1)));
    AIM_LAUNCH(c, "near_groups", (k_near_groups<false, cplx<R>><<<blocks, 256, 0, c->stream>>>(
                                     c->near_ptr, c->near_col, nullptr, c->N, ng, c->ngrp_ptr, nullptr, nullptr)));
    AIM_TRY(launch_check(c, "near_groups"));
    long long total = 0;
    AIM_TRY(scan_exclusive(c, c->ngrp_ptr, ng, &total));
    const int32_t t32 = (int32_t)total;
    AIM_CUDA_TRY(cudaMemcpyAsync(c->ngrp_ptr + ng, &t32, sizeof(t32), cudaMemcpyHostToDevice, c->stream));
    AIM_CUDA_TRY(cudaMalloc(&c->ngrp_col, sizeof(int32_t) * std::max(1LL, total)));
    AIM_CUDA_TRY(cudaStreamSynchronize(c->stream));  // t32 is read by the copy
    c->ngrp_nnz = total;
  }
  if (!pd.ngrp_val) {
    AIM_CUDA_TRY(cudaMalloc(&pd.ngrp_val, sizeof(cplx<R>) * std::max(1LL, c->ngrp_nnz) * kNearGroup));
    AIM_LAUNCH(c, "near_groups", (k_near_groups<true, cplx<R>><<<blocks, 256, 0, c->stream>>>(
                                     c->near_ptr, c->near_col, pd.near_val, c->N, ng, c->ngrp_ptr, c->ngrp_col,
                                     pd.ngrp_val)));
    AIM_TRY(launch_check(c, "near_groups"));
  }
  return AIM_OK;
}

// MD: storage of the projected grid; MI: storage of Phi read by the interpolation.
template <class MD, class MI>
static int run_product(aim_ctx* c, const cplx<typename MD::R>* x, cplx<typename MD::R>* y, int nrhs,
                       typename MD::S* grid0, const typename MI::S* phi, const typename MD::R* pw,
                       const typename MD::R* lam, const cplx<typename MD::R>* nval, int (*convolve)(aim_ctx*, int)) {
  using R = typename MD::R;
  const long long Nc = (long long)c->n[0] * c->n[1] * c->n[2];
  const bool many = nrhs >= kRhsLanesMin;
  // two right-hand sides per lane once a warp has 64 to cover
  const bool two = nrhs >= 64 && nrhs % 2 == 0;
  PrecData<R>& pd = prec_data<R>(c);
  if (many) {
    if (!pd.phiT) {
      AIM_CUDA_TRY(cudaMalloc(&pd.phiT, sizeof(cplx<R>) * c->max_rhs * 4 * Nc));
      AIM_CUDA_TRY(cudaMalloc(&pd.xT, sizeof(cplx<R>) * c->max_rhs * c->N));
    }
    AIM_TRY(transpose(c, "transpose_x", x, pd.xT, nrhs, (long long)c->N));
    // right-hand sides per launch: up to 64, shared memory 32 (4 B + 1) elements
    const int chunk = std::min(nrhs, 64);
    const size_t sm = sizeof(cplx<R>) * 32 * (4 * chunk + 1);
    const int blocks = (int)((Nc + 31) / 32);
    static const cudaError_t attr1 = cudaFuncSetAttribute(proj_gather_rhs<MD, 1>,
                                                          cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    static const cudaError_t attr2 = cudaFuncSetAttribute(proj_gather_rhs<MD, 2>,
                                                          cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    AIM_CUDA_TRY(attr1);
    AIM_CUDA_TRY(attr2);
    for (int b0 = 0; b0 < nrhs; b0 += chunk) {
      const int nb = std::min(chunk, nrhs - b0);
      const cplx<R>* xs = pd.xT + b0;
      typename MD::S* qd = grid0 + (long long)b0 * 4 * Nc;
      if (nb == 64 && nrhs % 2 == 0)  // two per lane: 16-byte loads need an even row stride
        AIM_LAUNCH(c, "proj_gather", (proj_gather_rhs<MD, 2><<<blocks, 256, sm, c->stream>>>(xs, qd, c->pnode_ptr,
                                                                                            c->pnode_m, pw, Nc, nb,
                                                                                            nrhs, c->N)));
      else
        AIM_LAUNCH(c, "proj_gather", (proj_gather_rhs<MD, 1><<<blocks, 256, sm, c->stream>>>(xs, qd, c->pnode_ptr,
                                                                                            c->pnode_m, pw, Nc, nb,
                                                                                            nrhs, c->N)));
      AIM_TRY(launch_check(c, "proj_gather"));
    }
  } else {
    const long long ntask = proj_tasks(c, Nc);
    const int blocks = (int)std::min<long long>((ntask + 7) / 8, 152LL * 16);
    const int32_t* groups = c->sparse_proj ? c->pgroups : nullptr;
    const auto go = [&](auto bc) {
      AIM_LAUNCH(c, "proj_gather", (proj_gather<MD, decltype(bc)::value><<<blocks, 256, 0, c->stream>>>(
                                       x, grid0, c->pnode_ptr, c->pnode_m, pw, c->N, Nc, nrhs, groups, ntask)));
    };
    if (nrhs == 1) go(std::integral_constant<int, 1>{});
    else if (nrhs == 2) go(std::integral_constant<int, 2>{});
    else go(std::integral_constant<int, 4>{});
    AIM_TRY(launch_check(c, "proj_gather"));
  }
  AIM_TRY(convolve(c, 4 * nrhs));
  if (many) {
    AIM_TRY(transpose(c, "transpose_phi", reinterpret_cast<const cplx<R>*>(phi), pd.phiT, nrhs, 4 * Nc));
    AIM_TRY(ensure_near_groups(c, pd));
    const int blocks = (int)((c->N + 8 * kNearGroup - 1) / (8 * kNearGroup));
    const size_t sm = sizeof(cplx<R>) * 8 * kNearGroup * (nrhs + 1);
    const R fvec = (R)(c->alpha * c->k * kEta0), frho = (R)(c->alpha * kEta0 / c->k),
            fmf = (R)((1.0 - c->alpha) * kEta0);
    const auto go = [&](auto mf, auto rl) {
      constexpr bool MF = decltype(mf)::value;
      constexpr int RL = decltype(rl)::value;
      // staged rows: at most 32 x 256 complex128 (128 KB), beside the stencil offsets
      static const cudaError_t attr = cudaFuncSetAttribute(interp_near_grp<MI, RL, MF>,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      AIM_CUDA_TRY(attr);
      AIM_LAUNCH(c, "interp_near",
                 (interp_near_grp<MI, RL, MF><<<blocks, 256, sm, c->stream>>>(
                     pd.phiT, pd.xT, y, lam, c->base, c->ngrp_ptr, c->ngrp_col, pd.ngrp_val, c->N, Nc, c->n[0],
                     c->n[1], nrhs, fvec, frho, c->S, c->M + 1, pd.lamM, fmf)));
      return AIM_OK;
    };
    using T2 = std::integral_constant<int, 2>;
    using T1 = std::integral_constant<int, 1>;
    if (pd.lamM)
      AIM_TRY(two ? go(std::true_type{}, T2{}) : go(std::true_type{}, T1{}));
    else
      AIM_TRY(two ? go(std::false_type{}, T2{}) : go(std::false_type{}, T1{}));
    return launch_check(c, "interp_near");
  }
  {
    const long long threads = (long long)c->N * 8;
    const int blocks = (int)((threads + 255) / 256);
    const R fvec = (R)(c->alpha * c->k * kEta0), frho = (R)(c->alpha * kEta0 / c->k),
            fmf = (R)((1.0 - c->alpha) * kEta0);
    const auto go = [&](auto mf) {
    AIM_LAUNCH(c, "interp_near",
             (interp_near<MI, decltype(mf)::value><<<blocks, 256, 0, c->stream>>>(phi, x, y, lam, c->base, c->near_ptr,
                                                                 c->near_col, nval, c->N, Nc, c->n[0], c->n[1],
                                                                 nrhs, fvec, frho, c->S, c->M + 1, pd.lamM, fmf)));
    };
    if (pd.lamM) go(std::true_type{}); else go(std::false_type{});

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
      AIM_TRY(budget_grids(c, precision));
      AIM_CUDA_TRY(cudaMalloc(&p.grid0, sizeof(float2) * e0));
      AIM_CUDA_TRY(cudaMalloc(&p.grid1, sizeof(float2) * e1));
      AIM_CUDA_TRY(cudaMalloc(&p.grid2, sizeof(float2) * e2));
      if (c->sparse_proj) AIM_CUDA_TRY(cudaMemsetAsync(p.grid0, 0, sizeof(float2) * e0, c->stream));
    }
  } else if (precision == AIM_C128_F64) {
    PrecData<double>& p = c->p64;
    if (!p.grid0) {
      AIM_TRY(budget_grids(c, precision));
      AIM_CUDA_TRY(cudaMalloc(&p.grid0, sizeof(double2) * e0));
      AIM_CUDA_TRY(cudaMalloc(&p.grid1, sizeof(double2) * e1));
      AIM_CUDA_TRY(cudaMalloc(&p.grid2, sizeof(double2) * e2));
      if (c->sparse_proj) AIM_CUDA_TRY(cudaMemsetAsync(p.grid0, 0, sizeof(double2) * e0, c->stream));
    }
  } else {
    FFData& p = c->pff;
    if (!p.grid0) {
      AIM_TRY(budget_grids(c, precision));
      AIM_CUDA_TRY(cudaMalloc(&p.grid0, sizeof(float4) * e0));
      AIM_CUDA_TRY(cudaMalloc(&p.grid1, sizeof(float4) * e1));
      AIM_CUDA_TRY(cudaMalloc(&p.grid2, sizeof(float4) * e2));
      if (c->sparse_proj) AIM_CUDA_TRY(cudaMemsetAsync(p.grid0, 0, sizeof(float4) * e0, c->stream));
    }
  }
  return AIM_OK;
}

int prepare_product(aim_ctx* c, int precision) {
  if (c->pack) return pack_prepare(c, precision);
  AIM_TRY(ensure_grids(c, precision));
  if (precision == AIM_C128) return ensure_ff_arrays(c);
  if (c->max_rhs >= kRhsLanesMin) {
    const long long Nc = (long long)c->n[0] * c->n[1] * c->n[2];
    if (precision == AIM_C64 && !c->p32.phiT) {
      AIM_CUDA_TRY(cudaMalloc(&c->p32.phiT, sizeof(float2) * c->max_rhs * 4 * Nc));
      AIM_CUDA_TRY(cudaMalloc(&c->p32.xT, sizeof(float2) * c->max_rhs * c->N));
    }
    if (precision == AIM_C128_F64 && !c->p64.phiT) {
      AIM_CUDA_TRY(cudaMalloc(&c->p64.phiT, sizeof(double2) * c->max_rhs * 4 * Nc));
      AIM_CUDA_TRY(cudaMalloc(&c->p64.xT, sizeof(double2) * c->max_rhs * c->N));
    }
    if (precision == AIM_C64) AIM_TRY(ensure_near_groups(c, c->p32));
    if (precision == AIM_C128_F64) AIM_TRY(ensure_near_groups(c, c->p64));
  }
  return AIM_OK;
}

int matvec(aim_ctx* c, const void* x, void* y, int nrhs, int precision) {
  if (c->pack) return pack_matvec(c, x, y, nrhs, precision);
  AIM_TRY(ensure_grids(c, precision));
  int rc;
  if (precision == AIM_C64)
    rc = run_product<M32, M32>(c, (const float2*)x, (float2*)y, nrhs, c->p32.grid0,
                               phi_grid(c, c->p32.grid0, c->p32.grid2), c->p32.pnode_w,
                               c->p32.lam, c->p32.near_val, fft_convolve_c64);
  else if (precision == AIM_C128_F64)
    rc = run_product<M64, M64>(c, (const double2*)x, (double2*)y, nrhs, c->p64.grid0,
                               phi_grid(c, c->p64.grid0, c->p64.grid2),
                               c->p64.pnode_w, c->p64.lam, c->p64.near_val, fft_convolve_c128);
  else
    rc = run_product_ff(c, (const double2*)x, (double2*)y, nrhs);
#ifdef AIM_CHECK
  if (rc == AIM_OK) rc = read_index_checks(c, "product");
#endif
  return rc;
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
    // every group is a task here: the caller's g0 holds no zeros of ours
    const long long ntask = (Nc + 7) / 8;
    const int blocks = (int)std::min<long long>((ntask + 7) / 8, 152LL * 16);
    const auto go = [&](auto bc) {
      AIM_LAUNCH(c, "proj_gather", (proj_gather<M32, decltype(bc)::value><<<blocks, 256, 0, c->stream>>>(
                                       x, g0, c->pnode_ptr, c->pnode_m, c->p32.pnode_w, c->N, Nc, nrhs, nullptr,
                                       ntask)));
    };
    if (nrhs == 1) go(std::integral_constant<int, 1>{});
    else if (nrhs == 2) go(std::integral_constant<int, 2>{});
    else go(std::integral_constant<int, 4>{});
    AIM_TRY(launch_check(c, "proj_gather"));
  }
  AIM_TRY(fft_convolve_c64_bufs(c, 4 * nrhs, g0, g1, g2));
  {
    const long long threads = (long long)c->N * 8;
    const int blocks = (int)((threads + 255) / 256);
    const float fvec = (float)(c->alpha * c->k * kEta0), frho = (float)(c->alpha * kEta0 / c->k),
                fmf = (float)((1.0 - c->alpha) * kEta0);
    const auto go = [&](auto mf) {
    AIM_LAUNCH(c, "interp_near",
             (interp_near<M32, decltype(mf)::value><<<blocks, 256, 0, c->stream>>>(g0, x, y, c->p32.lam, c->base, c->near_ptr,
                                                                  c->near_col, c->p32.near_val, c->N, Nc,
                                                                  c->n[0], c->n[1], nrhs, fvec, frho, c->S, c->M + 1, c->p32.lamM, fmf)));
    };
    if (c->p32.lamM) go(std::true_type{}); else go(std::false_type{});

    AIM_TRY(launch_check(c, "interp_near"));
  }
#ifdef AIM_CHECK
  AIM_TRY(read_index_checks(c, "product (no allocation)"));
#endif
  return AIM_OK;
}
}  // namespace aim
