// Device kernels of the context setup (paper Section 2.2 "matrix fill" for
// AIM; Section 2.4: the fill is O(N)).  setup.cu keeps the mesh topology,
// the anchors and the grid extents on the host and runs everything that
// scales with the basis count here:
//   * moment-matching weights in their tensor-product Lagrange form (one warp
//     per basis function, lanes over stencil nodes), with CFIE also the
//     differentiated-interpolation (MFIE) weights;
//   * the near list |c_m - c_n| <= r by cell binning (d2 = (dx dx + dy dy) +
//     dz dz in FP64 without contraction, the same test as the oracle), rows
//     sorted by column;
//   * the triangle-pair lists of the near fill (per test triangle the sorted,
//     unique source triangles of its near basis pairs; singular pairs, which
//     share a vertex, listed first), the entry-to-row map, the largest anchor
//     offset of a near pair and G_h on the offsets the near fill reads;
//   * plane-collapse detection, the node-ordered projection lists (entries of
//     a node ordered by basis index) and the 8-node groups that hold entries;
//   * the FP32 copies and the inverse diagonal.
// Exclusive prefix sums over int32 counts use a two-level block scan.
#include <algorithm>
#include <climits>
#include <vector>

#include "common.h"
#include "geom.h"
#include "setup_dev.h"

namespace aim {

// ------------------------------------------------------------------ scan
constexpr int kScanItems = 1024;  // per block: 256 threads x 4

__global__ void k_scan_block(int32_t* __restrict__ a, int32_t* __restrict__ bsum, long long n) {
  __shared__ int32_t warp_tot[8];
  const long long base = (long long)blockIdx.x * kScanItems + 4 * threadIdx.x;
  int32_t v[4], t = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[i] = base + i < n ? a[base + i] : 0;
    t += v[i];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t inc = t;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  int32_t woff = 0;
  for (int i = 0; i < w; ++i) woff += warp_tot[i];
  int32_t run = woff + inc - t;  // exclusive offset of this thread
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (base + i < n) a[base + i] = run;
    run += v[i];
  }
  if (threadIdx.x == 255) bsum[blockIdx.x] = woff + inc;
}

__global__ void k_scan_add(int32_t* __restrict__ a, const int32_t* __restrict__ boff, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] += boff[i / kScanItems];
}

// In place: a[0..n) -> exclusive prefix sums; *total (host) receives the sum.
// The counts must sum below 2^31.
int scan_exclusive(aim_ctx* c, int32_t* a, long long n, long long* total) {
  if (n <= 0) {
    *total = 0;
    return AIM_OK;
  }
  const long long nb = (n + kScanItems - 1) / kScanItems;
  int32_t* bsum = nullptr;
  AIM_CUDA_TRY(cudaMallocAsync(&bsum, sizeof(int32_t) * (nb + 1), c->stream));
  k_scan_block<<<(unsigned)nb, 256, 0, c->stream>>>(a, bsum, n);
  int rc = launch_check(c, "setup_scan");
  long long btot = 0;
  if (rc == AIM_OK && nb > 1) {
    rc = scan_exclusive(c, bsum, nb, &btot);
    if (rc == AIM_OK) {
      k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(a, bsum, n);
      rc = launch_check(c, "setup_scan");
    }
  } else if (rc == AIM_OK) {
    int32_t t = 0;
    AIM_CUDA_TRY(cudaMemcpyAsync(&t, bsum, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    AIM_CUDA_TRY(cudaStreamSynchronize(c->stream));
    btot = t;
  }
  cudaFreeAsync(bsum, c->stream);
  *total = btot;
  return rc;
}

// ------------------------------------------------------------------ weights
__constant__ double c_wrule[3][kMaxRule * kMaxRule];

__device__ __forceinline__ V3 ldv3(const double* v, int i) { return v3(v[3 * i], v[3 * i + 1], v[3 * i + 2]); }

// One warp per basis function m.  The quadrature points of its two triangles
// are taken 32 at a time: lane p evaluates point p's weight, the basis
// function's components g = (f_x, f_y, f_z, div f) and the 1-D Lagrange
// values (with CFIE their derivatives and the triangle normal) into shared
// memory; then lane s accumulates stencil node s over those points.
constexpr int kWMaxP = 6;                       // M + 1 <= 6
constexpr int kWPt = 1 + 4 + 3 * kWMaxP;        // per point: weight, g[4], lx, ly, lz
constexpr int kWPtM = 3 + 3 * kWMaxP;           // CFIE extra: normal, dlx, dly, dlz
__global__ void __launch_bounds__(128) k_weights(DevGeom g, const int32_t* __restrict__ anchor, int N, int M, double h,
                                                 int nq, double* __restrict__ lam, double* __restrict__ lamM,
                                                 const double* __restrict__ nrm) {
  __shared__ double pt[4][32][kWPt + kWPtM];
  const int m = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (m >= N) return;
  const int P = M + 1, S = P * P * P;
  const double ax = anchor[3 * m], ay = anchor[3 * m + 1], az = anchor[3 * m + 2];
  const double hinv = 1.0 / h;
  double acc[7][4], accM[7][3];  // lane s = lane + 32 u, u < 7 (S <= 216)
#pragma unroll
  for (int u = 0; u < 7; ++u)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[u][c] = 0.0;
#pragma unroll
  for (int u = 0; u < 7; ++u)
#pragma unroll
    for (int c = 0; c < 3; ++c) accM[u][c] = 0.0;
  const int npt = 2 * nq;
  for (int p0 = 0; p0 < npt; p0 += 32) {
    const int p = p0 + lane;
    if (p < npt) {
      const int half = p >= nq, q = p - half * nq;
      const int t = half ? g.tm[m] : g.tp[m];
      const V3 fv = ldv3(g.vert, half ? g.fm[m] : g.fp[m]);
      const double sg = half ? -1.0 : 1.0, A = g.area[t];
      const V3 r0 = ldv3(g.vert, g.tri[3 * t]), r1 = ldv3(g.vert, g.tri[3 * t + 1]), r2 = ldv3(g.vert, g.tri[3 * t + 2]);
      const double cf = sg * g.len[m] / (2.0 * A), dv = sg * g.len[m] / A;
      const V3 r = tri_point(r0, r1, r2, c_wrule[0][q], c_wrule[1][q]);
      double* o = pt[w][lane];
      o[0] = A * c_wrule[2][q];
      o[1] = cf * (r.x - fv.x);
      o[2] = cf * (r.y - fv.y);
      o[3] = cf * (r.z - fv.z);
      o[4] = dv;
      const double xi = (r.x - h * ax) / h, up = (r.y - h * ay) / h, ze = (r.z - h * az) / h;
      for (int i = 0; i < P; ++i) {
        o[5 + i] = lagrange(M, i, xi);
        o[5 + kWMaxP + i] = lagrange(M, i, up);
        o[5 + 2 * kWMaxP + i] = lagrange(M, i, ze);
      }
      if (lamM) {
        const V3 n = ldv3(nrm, t);
        o[kWPt] = n.x;
        o[kWPt + 1] = n.y;
        o[kWPt + 2] = n.z;
        for (int i = 0; i < P; ++i) {
          o[kWPt + 3 + i] = lagrange_d(M, i, xi) * hinv;
          o[kWPt + 3 + kWMaxP + i] = lagrange_d(M, i, up) * hinv;
          o[kWPt + 3 + 2 * kWMaxP + i] = lagrange_d(M, i, ze) * hinv;
        }
      }
    }
    __syncwarp();
    const int np = min(32, npt - p0);
#pragma unroll
    for (int u = 0; u < 7; ++u) {
      const int s = lane + 32 * u;
      if (s >= S) continue;
      const int i = s % P, j = (s / P) % P, kk = s / (P * P);
      for (int e = 0; e < np; ++e) {
        const double* o = pt[w][e];
        const double lx = o[5 + i], ly = o[5 + kWMaxP + j], lz = o[5 + 2 * kWMaxP + kk];
        const double b = o[0] * lx * ly * lz;
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[u][c] += b * o[1 + c];
        if (lamM) {
          // W^c = int f . (n x (grad L_u x e_c)) = int (f . grad L_u) n_c - f_c (n . grad L_u)
          const double dx = o[kWPt + 3 + i], dy = o[kWPt + 3 + kWMaxP + j], dz = o[kWPt + 3 + 2 * kWMaxP + kk];
          const double gx = dx * ly * lz, gy = lx * dy * lz, gz = lx * ly * dz;
          const double fgr = o[1] * gx + o[2] * gy + o[3] * gz;
          const double ng = o[kWPt] * gx + o[kWPt + 1] * gy + o[kWPt + 2] * gz;
#pragma unroll
          for (int c = 0; c < 3; ++c) accM[u][c] += o[0] * (fgr * o[kWPt + c] - o[1 + c] * ng);
        }
      }
    }
    __syncwarp();
  }
#pragma unroll
  for (int u = 0; u < 7; ++u) {
    const int s = lane + 32 * u;
    if (s >= S) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) lam[((size_t)m * 4 + c) * S + s] = acc[u][c];
    if (lamM)
#pragma unroll
      for (int c = 0; c < 3; ++c) lamM[((size_t)m * 3 + c) * S + s] = accM[u][c];
  }
}

int weights_device(aim_ctx* c, const DevGeom& g, const int32_t* anchor, const TriRule& rw, double* lam, double* lamM,
                   const double* nrm) {
  double hr[3][kMaxRule * kMaxRule];
  for (int q = 0; q < rw.q; ++q) {
    hr[0][q] = rw.xi1[q];
    hr[1][q] = rw.xi2[q];
    hr[2][q] = rw.w[q];
  }
  AIM_CUDA_TRY(cudaMemcpyToSymbolAsync(c_wrule, hr, sizeof(hr), 0, cudaMemcpyHostToDevice, c->stream));
  const long long threads = 32LL * c->N;
  AIM_LAUNCH(c, "setup_weights", (k_weights<<<(unsigned)((threads + 127) / 128), 128, 0, c->stream>>>(
                                     g, anchor, c->N, c->M, c->h, rw.q, lam, lamM, nrm)));
  return launch_check(c, "setup_weights");
}

// ------------------------------------------------------------------ near list
struct CellGrid {
  double lo[3];
  double cs;
  int nc[3];
};

__device__ __forceinline__ void cell_of(const CellGrid& cg, const V3& p, int* ci) {
  const double v[3] = {p.x, p.y, p.z};
#pragma unroll
  for (int d = 0; d < 3; ++d) ci[d] = min(cg.nc[d] - 1, max(0, (int)((v[d] - cg.lo[d]) / cg.cs)));
}

__global__ void k_cell_count(const double* __restrict__ cen, int N, CellGrid cg, int32_t* __restrict__ cid,
                             int32_t* __restrict__ ccount) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= N) return;
  int ci[3];
  cell_of(cg, ldv3(cen, m), ci);
  const int id = (ci[2] * cg.nc[1] + ci[1]) * cg.nc[0] + ci[0];
  cid[m] = id;
  atomicAdd(&ccount[id], 1);
}

__global__ void k_cell_fill(const int32_t* __restrict__ cid, int N, const int32_t* __restrict__ cstart,
                            int32_t* __restrict__ cfill, int32_t* __restrict__ items) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= N) return;
  const int id = cid[m];
  items[cstart[id] + atomicAdd(&cfill[id], 1)] = m;
}

// FILL = false: cnt[m] = row length; FILL = true: the row's columns (unsorted) at col[ptr[m]..]
template <bool FILL>
__global__ void k_near_rows(const double* __restrict__ cen, int N, CellGrid cg, double r, double r2,
                            const int32_t* __restrict__ cstart, const int32_t* __restrict__ items,
                            int32_t* __restrict__ cnt_or_ptr, int32_t* __restrict__ col) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= N) return;
  const V3 cm = ldv3(cen, m);
  int ci[3];
  cell_of(cg, cm, ci);
  const int span = (r <= cg.cs) ? 1 : (int)ceil(r / cg.cs);
  int c = 0;
  const int32_t out0 = FILL ? cnt_or_ptr[m] : 0;
  for (int z = max(0, ci[2] - span); z <= min(cg.nc[2] - 1, ci[2] + span); ++z)
    for (int y = max(0, ci[1] - span); y <= min(cg.nc[1] - 1, ci[1] + span); ++y)
      for (int x = max(0, ci[0] - span); x <= min(cg.nc[0] - 1, ci[0] + span); ++x) {
        const int cc = (z * cg.nc[1] + y) * cg.nc[0] + x;
        for (int32_t e = cstart[cc]; e < cstart[cc + 1]; ++e) {
          const int n = items[e];
          const V3 cn = ldv3(cen, n);
          const double dx = cm.x - cn.x, dy = cm.y - cn.y, dz = cm.z - cn.z;
          const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
          if (d2 <= r2) {
            if (FILL) col[out0 + c] = n;
            ++c;
          }
        }
      }
  if (!FILL) cnt_or_ptr[m] = c;
}

// Sort each segment [ptr[i], ptr[i+1]) of key (and its payload, when given)
// ascending: one warp per segment, bitonic sort in shared memory over the
// next power of two >= its length (CAP per warp); longer segments are
// insertion-sorted by one thread.
template <int CAP>
__global__ void __launch_bounds__(128) k_sort_segments(const int32_t* __restrict__ ptr, long long nseg,
                                                       int32_t* __restrict__ key) {
  __shared__ int32_t buf[4][CAP];
  const long long seg = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (seg >= nseg) return;
  const int32_t b0 = ptr[seg], len = ptr[seg + 1] - b0;
  if (len <= 1) return;
  if (len > CAP) {
    if (lane == 0)
      for (int i = 1; i < len; ++i) {
        const int32_t v = key[b0 + i];
        int j = i - 1;
        while (j >= 0 && key[b0 + j] > v) {
          key[b0 + j + 1] = key[b0 + j];
          --j;
        }
        key[b0 + j + 1] = v;
      }
    return;
  }
  int n2 = 1;
  while (n2 < len) n2 <<= 1;
  for (int i = lane; i < n2; i += 32) buf[w][i] = i < len ? key[b0 + i] : INT_MAX;
  __syncwarp();
  for (int k = 2; k <= n2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < n2; i += 32) {
        const int l = i ^ j;
        if (l > i) {
          const int32_t a = buf[w][i], b = buf[w][l];
          const bool up = (i & k) == 0;
          if ((a > b) == up) {
            buf[w][i] = b;
            buf[w][l] = a;
          }
        }
      }
      __syncwarp();
    }
  for (int i = lane; i < len; i += 32) key[b0 + i] = buf[w][i];
}

int sort_segments(aim_ctx* c, const int32_t* ptr, long long nseg, int32_t* key) {
  if (nseg <= 0) return AIM_OK;
  AIM_LAUNCH(c, "setup_sort", (k_sort_segments<512><<<(unsigned)((nseg + 3) / 4), 128, 0, c->stream>>>(ptr, nseg, key)));
  return launch_check(c, "setup_sort");
}

int near_list_device(aim_ctx* c, const double* cen, const double* hcen, double r, int32_t** ptr_out,
                     int32_t** col_out, long long* nnz_out) {
  const int N = c->N;
  CellGrid cg{};
  double hi[3] = {-1e300, -1e300, -1e300};
  for (int d = 0; d < 3; ++d) cg.lo[d] = 1e300;
  for (int m = 0; m < N; ++m)
    for (int d = 0; d < 3; ++d) {
      cg.lo[d] = std::min(cg.lo[d], hcen[3 * (size_t)m + d]);
      hi[d] = std::max(hi[d], hcen[3 * (size_t)m + d]);
    }
  cg.cs = r;
  for (int d = 0; d < 3; ++d) cg.cs = std::max(cg.cs, (hi[d] - cg.lo[d]) / 256.0);
  if (!(cg.cs > 0.0)) cg.cs = 1.0;
  for (int d = 0; d < 3; ++d) cg.nc[d] = (int)((hi[d] - cg.lo[d]) / cg.cs) + 1;
  const long long ncell = (long long)cg.nc[0] * cg.nc[1] * cg.nc[2];
  int32_t *cid = nullptr, *cstart = nullptr, *cfill = nullptr, *items = nullptr, *ptr = nullptr, *col = nullptr;
  AIM_CUDA_TRY(cudaMallocAsync(&cid, sizeof(int32_t) * N, c->stream));
  AIM_CUDA_TRY(cudaMallocAsync(&cstart, sizeof(int32_t) * (ncell + 1), c->stream));
  AIM_CUDA_TRY(cudaMallocAsync(&cfill, sizeof(int32_t) * ncell, c->stream));
  AIM_CUDA_TRY(cudaMallocAsync(&items, sizeof(int32_t) * N, c->stream));
  AIM_CUDA_TRY(cudaMalloc(&ptr, sizeof(int32_t) * (N + 1)));
  AIM_CUDA_TRY(cudaMemsetAsync(cstart, 0, sizeof(int32_t) * (ncell + 1), c->stream));
  AIM_CUDA_TRY(cudaMemsetAsync(cfill, 0, sizeof(int32_t) * ncell, c->stream));
  const unsigned nb = (unsigned)((N + 255) / 256);
  AIM_LAUNCH(c, "setup_near_list", (k_cell_count<<<nb, 256, 0, c->stream>>>(cen, N, cg, cid, cstart)));
  AIM_TRY(launch_check(c, "setup_near_list"));
  long long tot = 0;
  AIM_TRY(scan_exclusive(c, cstart, ncell + 1, &tot));
  AIM_LAUNCH(c, "setup_near_list", (k_cell_fill<<<nb, 256, 0, c->stream>>>(cid, N, cstart, cfill, items)));
  AIM_TRY(launch_check(c, "setup_near_list"));
  const double r2 = r * r;
  AIM_LAUNCH(c, "setup_near_list",
             (k_near_rows<false><<<nb, 256, 0, c->stream>>>(cen, N, cg, r, r2, cstart, items, ptr, nullptr)));
  AIM_TRY(launch_check(c, "setup_near_list"));
  long long nnz = 0;
  AIM_CUDA_TRY(cudaMemsetAsync(ptr + N, 0, sizeof(int32_t), c->stream));
  AIM_TRY(scan_exclusive(c, ptr, (long long)N + 1, &nnz));
  if (nnz >= (1LL << 31) - 1) {
    set_error("aim_setup: near list too long");
    return AIM_EINVAL;
  }
  AIM_CUDA_TRY(cudaMalloc(&col, sizeof(int32_t) * std::max<long long>(1, nnz)));
  AIM_LAUNCH(c, "setup_near_list",
             (k_near_rows<true><<<nb, 256, 0, c->stream>>>(cen, N, cg, r, r2, cstart, items, ptr, col)));
  AIM_TRY(launch_check(c, "setup_near_list"));
  AIM_TRY(sort_segments(c, ptr, N, col));
  cudaFreeAsync(cid, c->stream);
  cudaFreeAsync(cstart, c->stream);
  cudaFreeAsync(cfill, c->stream);
  cudaFreeAsync(items, c->stream);
  *ptr_out = ptr;
  *col_out = col;
  *nnz_out = nnz;
  return AIM_OK;
}

// ------------------------------------------------------------------ triangle pairs
// Candidates of test triangle P: the two triangles of every near column of
// the basis functions whose free vertex is a slot of P.
__device__ __forceinline__ int tri_candidates(const int32_t* __restrict__ tri_rwg, const int32_t* __restrict__ nptr,
                                              int P) {
  int c = 0;
  for (int a = 0; a < 3; ++a) {
    const int m = tri_rwg[3 * P + a];
    if (m >= 0) c += 2 * (nptr[m + 1] - nptr[m]);
  }
  return c;
}

__global__ void k_tri_cand(const int32_t* __restrict__ tri_rwg, const int32_t* __restrict__ nptr, int nt,
                           int32_t* __restrict__ cand) {
  const int P = blockIdx.x * blockDim.x + threadIdx.x;
  if (P < nt) cand[P] = tri_candidates(tri_rwg, nptr, P);
}

// One warp per test triangle: gather the candidates into shared memory, sort
// (bitonic), and count (FILL = false) or write (FILL = true) the unique ones.
template <bool FILL>
__global__ void __launch_bounds__(128) k_tri_pairs(DevGeom g, const int32_t* __restrict__ tri_rwg,
                                                   const int32_t* __restrict__ nptr, const int32_t* __restrict__ ncol,
                                                   int nt, int cap, int32_t* __restrict__ tcount_or_ptr,
                                                   int32_t* __restrict__ pQ, int32_t* __restrict__ pP) {
  extern __shared__ int32_t sbuf[];
  const int P = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (P >= nt) return;
  int32_t* buf = sbuf + w * cap;
  int len = 0;
  for (int a = 0; a < 3; ++a) {
    const int m = tri_rwg[3 * P + a];
    if (m < 0) continue;
    const int e0 = nptr[m], e1 = nptr[m + 1];
    for (int e = e0 + lane; e < e1; e += 32) {
      const int n = ncol[e];
      buf[len + 2 * (e - e0)] = g.tp[n];
      buf[len + 2 * (e - e0) + 1] = g.tm[n];
    }
    len += 2 * (e1 - e0);
  }
  int n2 = 1;
  while (n2 < len) n2 <<= 1;
  for (int i = len + lane; i < n2; i += 32) buf[i] = INT_MAX;
  __syncwarp();
  for (int k = 2; k <= n2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < n2; i += 32) {
        const int l = i ^ j;
        if (l > i) {
          const int32_t x = buf[i], y = buf[l];
          const bool up = (i & k) == 0;
          if ((x > y) == up) {
            buf[i] = y;
            buf[l] = x;
          }
        }
      }
      __syncwarp();
    }
  // unique: element i is kept when it differs from i - 1
  int base = FILL ? tcount_or_ptr[P] : 0;
  for (int i0 = 0; i0 < len; i0 += 32) {
    const int i = i0 + lane;
    const bool keep = i < len && (i == 0 || buf[i] != buf[i - 1]);
    const unsigned ball = __ballot_sync(0xffffffffu, keep);
    if (FILL && keep) {
      const int pos = base + __popc(ball & ((1u << lane) - 1));
      pQ[pos] = buf[i];
      pP[pos] = P;
    }
    base += __popc(ball);
  }
  if (!FILL && lane == 0) tcount_or_ptr[P] = base;
}

// flag[i] = 1 when the pair shares a vertex (singular rule), else 0
__global__ void k_pair_flags(const int32_t* __restrict__ tri, const int32_t* __restrict__ pP,
                             const int32_t* __restrict__ pQ, long long npairs, int32_t* __restrict__ flag) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npairs) return;
  const int P = pP[i], Q = pQ[i];
  bool s = false;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) s |= tri[3 * P + a] == tri[3 * Q + b];
  flag[i] = s ? 1 : 0;
}

// ids: singular pairs in index order, then the regular ones in index order
// (spos = exclusive scan of the flags, nsing = their sum).
__global__ void k_pair_ids(const int32_t* __restrict__ flag, const int32_t* __restrict__ spos, long long npairs,
                           long long nsing, int32_t* __restrict__ ids) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npairs) return;
  const long long pos = flag[i] ? spos[i] : nsing + (i - spos[i]);
  ids[pos] = (int32_t)i;
}

__global__ void k_erow(const int32_t* __restrict__ nptr, int N, int32_t* __restrict__ erow) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= N) return;
  for (int32_t e = nptr[m]; e < nptr[m + 1]; ++e) erow[e] = m;
}

// largest |a_m - a_n| per axis over the near pairs
__global__ void k_anchor_span(const int32_t* __restrict__ erow, const int32_t* __restrict__ ecol,
                              const int32_t* __restrict__ anchor, long long nnz, int* __restrict__ dmax) {
  int d = 0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (long long)gridDim.x * blockDim.x) {
    const int m = erow[e], n = ecol[e];
#pragma unroll
    for (int k = 0; k < 3; ++k) d = max(d, abs(anchor[3 * m + k] - anchor[3 * n + k]));
  }
  for (int o = 16; o > 0; o >>= 1) d = max(d, __shfl_xor_sync(0xffffffffu, d, o));
  if ((threadIdx.x & 31) == 0) atomicMax(dmax, d);
}

// G_h on the integer offsets [-TE, TE]^3, G_h(0) = 0
__global__ void k_gtab(double2* __restrict__ gtab, int TE, double h, double k) {
  const int TW = 2 * TE + 1;
  const long long total = (long long)TW * TW * TW;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int ox = (int)(i % TW) - TE, oy = (int)((i / TW) % TW) - TE, oz = (int)(i / ((long long)TW * TW)) - TE;
    double re = 0.0, im = 0.0;
    if ((ox | oy | oz) != 0) {
      const double r = h * sqrt((double)ox * ox + (double)oy * oy + (double)oz * oz);
      const double sc = 1.0 / (4.0 * kPi * r);
      double s, cs;
      sincos(k * r, &s, &cs);
      re = cs * sc;
      im = -s * sc;
    }
    gtab[i] = make_double2(re, im);
  }
}

int pair_lists_device(aim_ctx* c, const DevGeom& g, const int32_t* tri_rwg, const int32_t* nptr,
                      const int32_t* ncol, long long nnz, PairLists* out) {
  const int nt = c->nt;
  int32_t *cand = nullptr, *tptr = nullptr;
  AIM_CUDA_TRY(cudaMallocAsync(&cand, sizeof(int32_t) * nt, c->stream));
  AIM_CUDA_TRY(cudaMalloc(&tptr, sizeof(int32_t) * (nt + 1)));
  AIM_LAUNCH(c, "setup_pairs", (k_tri_cand<<<(nt + 255) / 256, 256, 0, c->stream>>>(tri_rwg, nptr, nt, cand)));
  AIM_TRY(launch_check(c, "setup_pairs"));
  // shared-memory buffer per warp: the next power of two >= the most candidates
  int maxc = 0;
  {
    std::vector<int32_t> h(nt);
    AIM_CUDA_TRY(cudaMemcpyAsync(h.data(), cand, sizeof(int32_t) * nt, cudaMemcpyDeviceToHost, c->stream));
    AIM_CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (int v : h) maxc = std::max(maxc, v);
  }
  int cap = 32;
  while (cap < maxc) cap <<= 1;
  if (cap > 16384) {
    set_error("aim_setup: a triangle has " + std::to_string(maxc) +
              " candidate near source triangles (more than 16384): near radius too large for this mesh");
    return AIM_EINVAL;
  }
  const int wpb = std::max(1, std::min(4, (48 * 1024) / (cap * 4)));
  const size_t sm = (size_t)wpb * cap * 4;
  static const cudaError_t a0 =
      cudaFuncSetAttribute(k_tri_pairs<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  static const cudaError_t a1 =
      cudaFuncSetAttribute(k_tri_pairs<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  AIM_CUDA_TRY(a0);
  AIM_CUDA_TRY(a1);
  const unsigned nb = (unsigned)((nt + wpb - 1) / wpb);
  AIM_LAUNCH(c, "setup_pairs", (k_tri_pairs<false><<<nb, 32 * wpb, sm, c->stream>>>(g, tri_rwg, nptr, ncol, nt, cap,
                                                                                     tptr, nullptr, nullptr)));
  AIM_TRY(launch_check(c, "setup_pairs"));
  long long npairs = 0;
  AIM_CUDA_TRY(cudaMemsetAsync(tptr + nt, 0, sizeof(int32_t), c->stream));
  AIM_TRY(scan_exclusive(c, tptr, (long long)nt + 1, &npairs));
  if (npairs >= (1LL << 31) - 1) {
    set_error("aim_setup: too many near triangle pairs");
    return AIM_EINVAL;
  }
  int32_t *pQ = nullptr, *pP = nullptr, *ids = nullptr, *flag = nullptr, *spos = nullptr;
  AIM_CUDA_TRY(cudaMalloc(&pQ, sizeof(int32_t) * std::max<long long>(1, npairs)));
  AIM_CUDA_TRY(cudaMalloc(&pP, sizeof(int32_t) * std::max<long long>(1, npairs)));
  AIM_CUDA_TRY(cudaMalloc(&ids, sizeof(int32_t) * std::max<long long>(1, npairs)));
  AIM_LAUNCH(c, "setup_pairs", (k_tri_pairs<true><<<nb, 32 * wpb, sm, c->stream>>>(g, tri_rwg, nptr, ncol, nt, cap,
                                                                                    tptr, pQ, pP)));
  AIM_TRY(launch_check(c, "setup_pairs"));
  AIM_CUDA_TRY(cudaMallocAsync(&flag, sizeof(int32_t) * std::max<long long>(1, npairs), c->stream));
  AIM_CUDA_TRY(cudaMallocAsync(&spos, sizeof(int32_t) * (npairs + 1), c->stream));
  const unsigned pb = (unsigned)((npairs + 255) / 256);
  long long nsing = 0;
  if (npairs > 0) {
    AIM_LAUNCH(c, "setup_pairs", (k_pair_flags<<<pb, 256, 0, c->stream>>>(g.tri, pP, pQ, npairs, flag)));
    AIM_TRY(launch_check(c, "setup_pairs"));
    AIM_CUDA_TRY(cudaMemcpyAsync(spos, flag, sizeof(int32_t) * npairs, cudaMemcpyDeviceToDevice, c->stream));
    AIM_TRY(scan_exclusive(c, spos, npairs, &nsing));
    AIM_LAUNCH(c, "setup_pairs", (k_pair_ids<<<pb, 256, 0, c->stream>>>(flag, spos, npairs, nsing, ids)));
    AIM_TRY(launch_check(c, "setup_pairs"));
  }
  cudaFreeAsync(cand, c->stream);
  cudaFreeAsync(flag, c->stream);
  cudaFreeAsync(spos, c->stream);
  out->tptr = tptr;
  out->pQ = pQ;
  out->pP = pP;
  out->ids = ids;
  out->npairs = npairs;
  out->nsing = nsing;
  (void)nnz;
  return AIM_OK;
}

int erow_and_span_device(aim_ctx* c, const int32_t* nptr, const int32_t* ncol, long long nnz,
                         const int32_t* anchor, int32_t** erow_out, int* dmax_out) {
  int32_t* erow = nullptr;
  int* dm = nullptr;
  AIM_CUDA_TRY(cudaMalloc(&erow, sizeof(int32_t) * std::max<long long>(1, nnz)));
  AIM_CUDA_TRY(cudaMallocAsync(&dm, sizeof(int), c->stream));
  AIM_CUDA_TRY(cudaMemsetAsync(dm, 0, sizeof(int), c->stream));
  AIM_LAUNCH(c, "setup_pairs", (k_erow<<<(c->N + 255) / 256, 256, 0, c->stream>>>(nptr, c->N, erow)));
  AIM_TRY(launch_check(c, "setup_pairs"));
  if (nnz > 0) {
    AIM_LAUNCH(c, "setup_pairs", (k_anchor_span<<<152 * 8, 256, 0, c->stream>>>(erow, ncol, anchor, nnz, dm)));
    AIM_TRY(launch_check(c, "setup_pairs"));
  }
  int h = 0;
  AIM_CUDA_TRY(cudaMemcpyAsync(&h, dm, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  AIM_CUDA_TRY(cudaStreamSynchronize(c->stream));
  cudaFreeAsync(dm, c->stream);
  *erow_out = erow;
  *dmax_out = h;
  return AIM_OK;
}

int gtab_device(aim_ctx* c, int TE, double2** out) {
  const long long TW = 2 * TE + 1;
  AIM_CUDA_TRY(cudaMalloc(out, sizeof(double2) * TW * TW * TW));
  AIM_LAUNCH(c, "setup_gtab", (k_gtab<<<152 * 4, 256, 0, c->stream>>>(*out, TE, c->h, c->k)));
  return launch_check(c, "setup_gtab");
}

// ------------------------------------------------------------------ plane collapse
// used[kk] = 1 when some weight on stencil plane kk is nonzero
__global__ void k_planes_used(const double* __restrict__ lam, long long nmc, int S, int P, int* __restrict__ used) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nmc * S; i += (long long)gridDim.x * blockDim.x)
    if (lam[i] != 0.0) used[(int)(i % S) / (P * P)] = 1;
}

__global__ void k_keep_plane(const double* __restrict__ lam, long long nmc, int S, int S2, int kk0,
                             double* __restrict__ lam2) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nmc * S2; i += (long long)gridDim.x * blockDim.x) {
    const long long mc = i / S2;
    const int t = (int)(i - mc * S2);
    lam2[i] = lam[mc * S + (long long)kk0 * S2 + t];
  }
}

int planes_used_device(aim_ctx* c, const double* lam, int S, int P, std::vector<int>& used) {
  int* d = nullptr;
  AIM_CUDA_TRY(cudaMallocAsync(&d, sizeof(int) * P, c->stream));
  AIM_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(int) * P, c->stream));
  AIM_LAUNCH(c, "setup_planar", (k_planes_used<<<152 * 8, 256, 0, c->stream>>>(lam, 4LL * c->N, S, P, d)));
  AIM_TRY(launch_check(c, "setup_planar"));
  used.assign(P, 0);
  AIM_CUDA_TRY(cudaMemcpyAsync(used.data(), d, sizeof(int) * P, cudaMemcpyDeviceToHost, c->stream));
  AIM_CUDA_TRY(cudaStreamSynchronize(c->stream));
  cudaFreeAsync(d, c->stream);
  return AIM_OK;
}

int keep_plane_device(aim_ctx* c, const double* lam, int S, int S2, int kk0, double** lam2) {
  AIM_CUDA_TRY(cudaMalloc(lam2, sizeof(double) * 4 * (size_t)c->N * S2));
  AIM_LAUNCH(c, "setup_planar", (k_keep_plane<<<152 * 8, 256, 0, c->stream>>>(lam, 4LL * c->N, S, S2, kk0, *lam2)));
  return launch_check(c, "setup_planar");
}

// ------------------------------------------------------------------ projection lists
__global__ void k_base(const int32_t* __restrict__ anchor, int N, int lo0, int lo1, int lo2, int kk0, int nx, int ny,
                       int32_t* __restrict__ base) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= N) return;
  const int ix = anchor[3 * m] - lo0, iy = anchor[3 * m + 1] - lo1, iz = anchor[3 * m + 2] + kk0 - lo2;
  base[m] = (int32_t)(((long long)iz * ny + iy) * nx + ix);
}

__device__ __forceinline__ bool weight_nonzero(const double* lam, int m, int s, int S) {
  const double* l = lam + (size_t)m * 4 * S;
  return l[s] != 0.0 || l[S + s] != 0.0 || l[2 * S + s] != 0.0 || l[3 * S + s] != 0.0;
}
__device__ __forceinline__ long long node_of(const int32_t* base, int m, int s, int P, int S, int nx, int ny) {
  const int i = s % P, j = (s / P) % P, kk = s / (P * P);
  (void)S;
  return (long long)base[m] + ((long long)kk * ny + j) * nx + i;
}

// FILL = false: count entries per node; FILL = true: write them (unordered within a node)
template <bool FILL>
__global__ void k_proj(const double* __restrict__ lam, const int32_t* __restrict__ base, int N, int S, int P, int nx,
                       int ny, int32_t* __restrict__ pcount_or_ptr, int32_t* __restrict__ pfill,
                       int32_t* __restrict__ pm, double* __restrict__ pw) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)N * S) return;
  const int m = (int)(i / S), s = (int)(i - (long long)m * S);
  if (!weight_nonzero(lam, m, s, S)) return;
  const long long u = node_of(base, m, s, P, S, nx, ny);
  if (!FILL) {
    atomicAdd(&pcount_or_ptr[u], 1);
    return;
  }
  const int32_t e = pcount_or_ptr[u] + atomicAdd(&pfill[u], 1);
  pm[e] = m;
  const double* l = lam + (size_t)m * 4 * S;
#pragma unroll
  for (int c = 0; c < 4; ++c) pw[4 * (size_t)e + c] = l[c * S + s];
}

// order each node's entries by basis index (insertion sort, one thread per node)
__global__ void k_proj_sort(const int32_t* __restrict__ ptr, long long Nc, int32_t* __restrict__ pm,
                            double* __restrict__ pw) {
  const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= Nc) return;
  const int32_t b0 = ptr[u], b1 = ptr[u + 1];
  for (int32_t i = b0 + 1; i < b1; ++i) {
    const int32_t key = pm[i];
    const double w0 = pw[4 * (size_t)i], w1 = pw[4 * (size_t)i + 1], w2 = pw[4 * (size_t)i + 2], w3 = pw[4 * (size_t)i + 3];
    int32_t j = i - 1;
    while (j >= b0 && pm[j] > key) {
      pm[j + 1] = pm[j];
      for (int c = 0; c < 4; ++c) pw[4 * (size_t)(j + 1) + c] = pw[4 * (size_t)j + c];
      --j;
    }
    pm[j + 1] = key;
    pw[4 * (size_t)(j + 1)] = w0;
    pw[4 * (size_t)(j + 1) + 1] = w1;
    pw[4 * (size_t)(j + 1) + 2] = w2;
    pw[4 * (size_t)(j + 1) + 3] = w3;
  }
}

// flag[g] = 1 when the 8-node group g holds projection entries
__global__ void k_group_flags(const int32_t* __restrict__ ptr, long long Nc, long long ng, int32_t* __restrict__ flag) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ng) return;
  const long long e = min(Nc, 8 * g + 8);
  flag[g] = ptr[e] > ptr[8 * g] ? 1 : 0;
}
__global__ void k_group_list(const int32_t* __restrict__ flag, const int32_t* __restrict__ pos, long long ng,
                             int32_t* __restrict__ groups) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < ng && flag[g]) groups[pos[g]] = (int32_t)g;
}

int projection_device(aim_ctx* c, const double* lam, int S, int P, long long Nc, ProjLists* out) {
  const int N = c->N, nx = c->n[0], ny = c->n[1];
  int32_t *base = nullptr, *ptr = nullptr, *fill = nullptr, *pm = nullptr;
  double* pw = nullptr;
  AIM_CUDA_TRY(cudaMalloc(&base, sizeof(int32_t) * N));
  AIM_LAUNCH(c, "setup_projection", (k_base<<<(N + 255) / 256, 256, 0, c->stream>>>(
                                        out->anchor, N, c->lo[0], c->lo[1], c->lo[2], c->kk0, nx, ny, base)));
  AIM_TRY(launch_check(c, "setup_projection"));
  AIM_CUDA_TRY(cudaMalloc(&ptr, sizeof(int32_t) * (Nc + 1)));
  AIM_CUDA_TRY(cudaMallocAsync(&fill, sizeof(int32_t) * Nc, c->stream));
  AIM_CUDA_TRY(cudaMemsetAsync(ptr, 0, sizeof(int32_t) * (Nc + 1), c->stream));
  AIM_CUDA_TRY(cudaMemsetAsync(fill, 0, sizeof(int32_t) * Nc, c->stream));
  const long long items = (long long)N * S;
  const unsigned nb = (unsigned)((items + 255) / 256);
  AIM_LAUNCH(c, "setup_projection", (k_proj<false><<<nb, 256, 0, c->stream>>>(lam, base, N, S, P, nx, ny, ptr, nullptr,
                                                                             nullptr, nullptr)));
  AIM_TRY(launch_check(c, "setup_projection"));
  long long nent = 0;
  AIM_TRY(scan_exclusive(c, ptr, Nc + 1, &nent));
  AIM_CUDA_TRY(cudaMalloc(&pm, sizeof(int32_t) * std::max<long long>(1, nent)));
  AIM_CUDA_TRY(cudaMalloc(&pw, sizeof(double) * 4 * std::max<long long>(1, nent)));
  AIM_LAUNCH(c, "setup_projection", (k_proj<true><<<nb, 256, 0, c->stream>>>(lam, base, N, S, P, nx, ny, ptr, fill, pm,
                                                                            pw)));
  AIM_TRY(launch_check(c, "setup_projection"));
  AIM_LAUNCH(c, "setup_projection", (k_proj_sort<<<(unsigned)((Nc + 255) / 256), 256, 0, c->stream>>>(ptr, Nc, pm, pw)));
  AIM_TRY(launch_check(c, "setup_projection"));
  cudaFreeAsync(fill, c->stream);
  out->base = base;
  out->ptr = ptr;
  out->pm = pm;
  out->pw = pw;
  out->nent = nent;
  out->groups = nullptr;
  out->ngroups = 0;
  if (out->want_groups) {
    const long long ng = (Nc + 7) / 8;
    int32_t *flag = nullptr, *pos = nullptr;
    AIM_CUDA_TRY(cudaMallocAsync(&flag, sizeof(int32_t) * ng, c->stream));
    AIM_CUDA_TRY(cudaMallocAsync(&pos, sizeof(int32_t) * (ng + 1), c->stream));
    const unsigned gb = (unsigned)((ng + 255) / 256);
    AIM_LAUNCH(c, "setup_projection", (k_group_flags<<<gb, 256, 0, c->stream>>>(ptr, Nc, ng, flag)));
    AIM_TRY(launch_check(c, "setup_projection"));
    AIM_CUDA_TRY(cudaMemcpyAsync(pos, flag, sizeof(int32_t) * ng, cudaMemcpyDeviceToDevice, c->stream));
    long long ngrp = 0;
    AIM_TRY(scan_exclusive(c, pos, ng, &ngrp));
    if (ngrp > 0) {
      AIM_CUDA_TRY(cudaMalloc(&out->groups, sizeof(int32_t) * ngrp));
      AIM_LAUNCH(c, "setup_projection", (k_group_list<<<gb, 256, 0, c->stream>>>(flag, pos, ng, out->groups)));
      AIM_TRY(launch_check(c, "setup_projection"));
    }
    out->ngroups = ngrp;
    cudaFreeAsync(flag, c->stream);
    cudaFreeAsync(pos, c->stream);
  }
  return AIM_OK;
}

// ------------------------------------------------------------------ conversions
__global__ void k_to_f32(const double* __restrict__ in, float* __restrict__ out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}
__global__ void k_inverse(const double2* __restrict__ d, double2* __restrict__ inv, int N) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= N) return;
  const double a = d[m].x, b = d[m].y, q = a * a + b * b;
  inv[m] = make_double2(a / q, -b / q);
}

int to_f32_device(aim_ctx* c, const double* in, long long n, float** out) {
  AIM_CUDA_TRY(cudaMalloc(out, sizeof(float) * std::max<long long>(1, n)));
  if (n == 0) return AIM_OK;
  AIM_LAUNCH(c, "setup_convert", (k_to_f32<<<152 * 8, 256, 0, c->stream>>>(in, *out, n)));
  return launch_check(c, "setup_convert");
}

int inverse_diag_device(aim_ctx* c, const double2* d, double2** out) {
  AIM_CUDA_TRY(cudaMalloc(out, sizeof(double2) * c->N));
  AIM_LAUNCH(c, "setup_convert", (k_inverse<<<(c->N + 255) / 256, 256, 0, c->stream>>>(d, *out, c->N)));
  return launch_check(c, "setup_convert");
}


// ---- column flags of the z passes
__global__ void k_colmask(const int32_t* __restrict__ ptr, long long Nc, long long plane, uint8_t* __restrict__ mask) {
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < Nc; u += (long long)gridDim.x * blockDim.x)
    if (ptr[u + 1] > ptr[u]) mask[u % plane] = 1;  // every writer stores the same value
}

int column_mask_device(aim_ctx* c, const int32_t* pnode_ptr, long long Nc, uint8_t** out) {
  const long long plane = (long long)c->n[0] * c->n[1];
  AIM_CUDA_TRY(cudaMalloc(out, plane));
  AIM_CUDA_TRY(cudaMemsetAsync(*out, 0, plane, c->stream));
  AIM_LAUNCH(c, "setup_colmask", (k_colmask<<<(unsigned)std::min<long long>((Nc + 255) / 256, 152LL * 32), 256, 0,
                                              c->stream>>>(pnode_ptr, Nc, plane, *out)));
  return launch_check(c, "setup_colmask");
}

}  // namespace aim
