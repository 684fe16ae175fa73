// Near-zone fill on the device (paper Section 2.2: near-zone correction with
// gamma = 3; Section 2.4: the near-field matrix is filled in O(N) time).
//
//   1. EFIE triangle-pair blocks T[a][b] for every (test triangle, source
//      triangle) pair that some near RWG pair touches (geom.h pair_block:
//      collapsed Gauss-Legendre rules, singular extraction for pairs that
//      share a vertex), one thread per pair;
//   2. each near entry's two test halves, Z_mn = j k eta l_m l_n
//      sum s_m s_n T[a(m)][b(n)], one thread per (entry, half);
//   3. symmetrisation (Z_mn + Z_nm) / 2 and the subtraction of the pair's
//      grid approximation j k eta [sum_xyz L_m G_h L_n - k^-2 L^rho_m G_h L^rho_n],
//      one warp per entry (lanes over the test stencil nodes).
// With CFIE (alpha < 1, Section 2.2 for closed bodies) the same kernels also
// produce the MFIE blocks 1/2 <f_m, f_n> - <f_m, n x int grad G x f_n>
// (unsymmetrised) and subtract their grid form -sum_c W^c_m . G Lambda^c_n;
// the entry is alpha EFIE + (1 - alpha) eta MFIE.
// Every value is FP64.  The pair lists, weights and near list come from the
// device setup (setup_dev.cu); the results stay on the device.
#include <algorithm>

#include "common.h"
#include "geom.h"
#include "setup_dev.h"

namespace aim {

// The three rules (test, test near a singularity, source) as raw bytes:
// TriRule has a default member initializer, which __constant__ storage does
// not allow.
__constant__ double c_rules[3 * (sizeof(TriRule) / sizeof(double) + 1)];
constexpr size_t kRuleStride = (sizeof(TriRule) / sizeof(double) + 1) * sizeof(double);
__device__ __forceinline__ const TriRule& rule(int i) {
  return *reinterpret_cast<const TriRule*>(reinterpret_cast<const char*>(c_rules) + i * kRuleStride);
}

struct FillGeom {
  const double* vert;     // [nv][3]
  const int32_t* tri;     // [nt][3]
  const double* area;     // [nt]
  const int32_t* tp;      // [N] "+" triangle
  const int32_t* tm;      // [N] "-" triangle
  const int32_t* sp;      // [N] slot of the free vertex in the "+" triangle
  const int32_t* sm;      // [N] slot in the "-" triangle
  const double* len;      // [N] edge length
};

__device__ __forceinline__ V3 vtx(const FillGeom& g, int t, int s) {
  const double* p = g.vert + 3 * (size_t)g.tri[3 * (size_t)t + s];
  return v3(p[0], p[1], p[2]);
}

// MFIE triangle-pair block T[a][b] = C[a][b] / 2 - B[a][b] with
//   B[a][b] = 1/(4 A_P A_Q) int_P int_Q (r - P_a) . (n_P x (grad G(r - r') x (r' - Q_b))) dS' dS,
//   grad G(D) = -(1 + j k R) exp(-j k R) / (4 pi R^3) D,   D = r - r',
//   C[a][b] = 1/(4 A_P^2) int_P (r - P_a) . (r - P_b) dS   (equal triangles only);
// so that <f_m, f_n>/2 - <f_m, n x int grad G x f_n> += s_m s_n l_m l_n T[a][b].
// Coplanar triangles (a triangle with itself included) have B = 0: every
// vector of the integrand lies in their plane.
__device__ void mfie_block(const V3 Pv[3], const V3 Qv[3], double AP, double AQ, bool same, double k,
                           const TriRule& test, const TriRule& src, Cd T[3][3]) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) T[a][b] = cd(0, 0);
  if (same) {
    const TriRule& g3 = rule(0);  // 3 x 3 points: exact for the degree-2 Gram integrand
    for (int i = 0; i < g3.q; ++i) {
      const V3 r = tri_point(Pv[0], Pv[1], Pv[2], g3.xi1[i], g3.xi2[i]);
      const double W = AP * g3.w[i] * 0.5 / (4.0 * AP * AP);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) T[a][b].re += W * dot(r - Pv[a], r - Pv[b]);
    }
    return;
  }
  const V3 nP0 = cross(Pv[1] - Pv[0], Pv[2] - Pv[0]), nQ0 = cross(Qv[1] - Qv[0], Qv[2] - Qv[0]);
  const V3 nP = (1.0 / norm(nP0)) * nP0, nQ = (1.0 / norm(nQ0)) * nQ0;
  const V3 nx = cross(nP, nQ);
  if (fmax(fabs(nx.x), fmax(fabs(nx.y), fabs(nx.z))) == 0.0 && fabs(dot(Qv[0] - Pv[0], nP)) == 0.0) return;
  (void)nQ;
  // With positions taken from O = Q_0 (r' = r - O, r'_q = r_q - O), x = ra.r',
  // v = n.r', z = ra.Q'_b, p = n.Q'_b, the integrand (ra.D)(n.rb) - (ra.rb)(n.D)
  // summed over the source points with weights gw is
  //   A1 (x - z) + A0 (z v - x p) + (ra.C)(p - v),
  // A0 = sum gw, A1 = sum gw n.r'_q, C = sum gw r'_q: five complex sums per
  // source point instead of nine (a, b) integrands.
  const V3 O = Qv[0];
  const V3 Qp[3] = {Qv[0] - O, Qv[1] - O, Qv[2] - O};
  double pq[3];
  for (int b = 0; b < 3; ++b) pq[b] = dot(nP, Qp[b]);
  Cd acc[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) acc[a][b] = cd(0, 0);
  for (int i = 0; i < test.q; ++i) {
    const V3 r = tri_point(Pv[0], Pv[1], Pv[2], test.xi1[i], test.xi2[i]);
    const V3 rp = r - O;
    const double W = AP * test.w[i];
    Cd A0 = cd(0, 0), A1 = cd(0, 0), C[3] = {cd(0, 0), cd(0, 0), cd(0, 0)};
    for (int q = 0; q < src.q; ++q) {
      const V3 rq = tri_point(Qv[0], Qv[1], Qv[2], src.xi1[q], src.xi2[q]);
      const V3 rqp = rq - O;
      const V3 D = r - rq;
      const double R = norm(D);
      const double kr = k * R, s = W * AQ * src.w[q] / (4.0 * kPi * R * R * R);
      double sr, cr;
      sincos(kr, &sr, &cr);
      // -(1 + j kR)(cos kR - j sin kR) = -(cos + kR sin) + j (sin - kR cos)
      const Cd gw = cd(-(cr + kr * sr) * s, (sr - kr * cr) * s);
      A0 = A0 + gw;
      A1 = A1 + dot(nP, rqp) * gw;
      C[0] = C[0] + rqp.x * gw;
      C[1] = C[1] + rqp.y * gw;
      C[2] = C[2] + rqp.z * gw;
    }
    const double v = dot(nP, rp);
    for (int a = 0; a < 3; ++a) {
      const V3 ra = r - Pv[a];
      const double x = dot(ra, rp);
      const Cd raC = ra.x * C[0] + ra.y * C[1] + ra.z * C[2];
      for (int b = 0; b < 3; ++b) {
        const double z = dot(ra, Qp[b]);
        acc[a][b] = acc[a][b] + (x - z) * A1 + (z * v - x * pq[b]) * A0 + (pq[b] - v) * raC;
      }
    }
  }
  const double f = -1.0 / (4.0 * AP * AQ);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) T[a][b] = f * acc[a][b];
}

// Triangle-pair blocks: pair i = (pP[i], pQ[i]); out[i][a][b] (EFIE) and,
// when outM is set, outM[i][a][b] (MFIE).
template <bool SING>
__global__ void __launch_bounds__(128) k_pair_blocks(FillGeom g, const int32_t* __restrict__ ids,
                                                     const int32_t* __restrict__ pP, const int32_t* __restrict__ pQ,
                                                     int n, double k, Cd* __restrict__ out, Cd* __restrict__ outM) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int i = ids[t];
  const int P = pP[i], Q = pQ[i];
  const V3 Pv[3] = {vtx(g, P, 0), vtx(g, P, 1), vtx(g, P, 2)};
  const V3 Qv[3] = {vtx(g, Q, 0), vtx(g, Q, 1), vtx(g, Q, 2)};
  Cd T[3][3];
  pair_block(Pv, Qv, g.area[P], g.area[Q], SING, k, rule(SING ? 1 : 0), rule(2), T);
  Cd* o = out + (size_t)i * 9;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) o[a * 3 + b] = T[a][b];
  if (outM) {
    mfie_block(Pv, Qv, g.area[P], g.area[Q], P == Q, k, rule(SING ? 1 : 0), rule(2), T);
    Cd* oM = outM + (size_t)i * 9;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) oM[a * 3 + b] = T[a][b];
  }
}

// Index of triangle Q in the sorted pair list of test triangle P.
__device__ __forceinline__ int64_t pair_of(const int32_t* tptr, const int32_t* pQ, int P, int Q) {
  int64_t lo = tptr[P], hi = tptr[P + 1];
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (pQ[mid] < Q) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// zhalf[half][e] = j k eta l_m l_n sum over n's two triangles of s_m s_n T[a][b]
// and, with blkM, zMhalf[half][e] = l_m l_n sum s_m s_n TM[a][b] (the MFIE entry's halves).
__global__ void k_near_halves(FillGeom g, const int32_t* __restrict__ erow, const int32_t* __restrict__ ecol,
                              const int32_t* __restrict__ tptr, const int32_t* __restrict__ pQ,
                              const Cd* __restrict__ blk, int64_t nnz, double jke, double2* __restrict__ zhalf,
                              const Cd* __restrict__ blkM, double2* __restrict__ zMhalf) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < 2 * nnz; t += (int64_t)gridDim.x * blockDim.x) {
    const int half = (int)(t / nnz);
    const int64_t e = t - half * nnz;
    const int m = erow[e], n = ecol[e];
    const int P = half ? g.tm[m] : g.tp[m];
    const int a = half ? g.sm[m] : g.sp[m];
    const double sm_ = half ? -1.0 : 1.0;
    double re = 0.0, im = 0.0, mre = 0.0, mim = 0.0;
    for (int th = 0; th < 2; ++th) {
      const int Qt = th ? g.tm[n] : g.tp[n];
      const int b = th ? g.sm[n] : g.sp[n];
      const double sn_ = th ? -1.0 : 1.0;
      const size_t ib = (size_t)pair_of(tptr, pQ, P, Qt) * 9 + a * 3 + b;
      const Cd v = blk[ib];
      re += sm_ * sn_ * v.re;
      im += sm_ * sn_ * v.im;
      if (blkM) {
        const Cd w = blkM[ib];
        mre += sm_ * sn_ * w.re;
        mim += sm_ * sn_ * w.im;
      }
    }
    const double ll = g.len[m] * g.len[n], f = jke * ll;
    zhalf[half * nnz + e] = make_double2(-f * im, f * re);
    if (blkM) zMhalf[half * nnz + e] = make_double2(ll * mre, ll * mim);
  }
}

// Symmetrised entry minus the grid approximation; one warp per entry, lane s
// over the test stencil nodes.  gtab: G_h on offsets [-TE, TE]^3.
// CFIE (lamM set): alpha (symmetrised EFIE entry - its grid form) + (1 - alpha) eta
// (MFIE entry - its grid form -sum_c W^c_m . G Lambda^c_n).
__global__ void __launch_bounds__(256) k_near_values(const int32_t* __restrict__ erow, const int32_t* __restrict__ ecol,
                                                     const int32_t* __restrict__ nptr, const double2* __restrict__ zhalf,
                                                     const double* __restrict__ lam, const int32_t* __restrict__ anchor,
                                                     const double2* __restrict__ gtab, int TE, int P, int64_t nnz,
                                                     double k, double jke, double2* __restrict__ val,
                                                     double2* __restrict__ diag, const double2* __restrict__ zMhalf,
                                                     const double* __restrict__ lamM, double alpha) {
  const int lane = threadIdx.x & 31;
  const int S = P * P * P, TW = 2 * TE + 1;
  for (int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; e < nnz;
       e += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int m = erow[e], n = ecol[e];
    // transposed entry (n, m) in row n
    int64_t lo = nptr[n], hi = nptr[n + 1];
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (ecol[mid] < m) lo = mid + 1;
      else hi = mid;
    }
    const int64_t et = lo;
    // EFIE: the grid part is symmetric (G_h depends on |offset|), so the
    // entry of the pair with m <= n computes it once for both; with CFIE the
    // MFIE part is not, and every entry computes its own
    if (!lamM && m > n) continue;
    const double2 a0 = zhalf[e], a1 = zhalf[nnz + e], b0 = zhalf[et], b1 = zhalf[nnz + et];
    const double zr = 0.5 * ((a0.x + a1.x) + (b0.x + b1.x));
    const double zi = 0.5 * ((a0.y + a1.y) + (b0.y + b1.y));
    const int dx = anchor[3 * (size_t)m] - anchor[3 * (size_t)n];
    const int dy = anchor[3 * (size_t)m + 1] - anchor[3 * (size_t)n + 1];
    const int dz = anchor[3 * (size_t)m + 2] - anchor[3 * (size_t)n + 2];
    const double* lm = lam + (size_t)m * 4 * S;
    const double* ln = lam + (size_t)n * 4 * S;
    double sr = 0.0, si = 0.0;  // sum over c of +-(lm^T G ln), vector minus k^-2 charge
    double mr = 0.0, mi = 0.0;  // CFIE: sum over c = x, y, z of W^c_m . G Lambda^c_n
    const double* wm = lamM ? lamM + (size_t)m * 3 * S : nullptr;
    for (int s = lane; s < S; s += 32) {
      const int si_ = s % P, sj = (s / P) % P, sk = s / (P * P);
      double ar[4] = {0, 0, 0, 0}, ai[4] = {0, 0, 0, 0};
      for (int t = 0; t < S; ++t) {
        const int ti = t % P, tj = (t / P) % P, tk = t / (P * P);
        const double2 gv = gtab[((size_t)(dz + sk - tk + TE) * TW + (dy + sj - tj + TE)) * TW + (dx + si_ - ti + TE)];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const double l = ln[c * S + t];
          ar[c] += gv.x * l;
          ai[c] += gv.y * l;
        }
      }
      const double kinv2 = 1.0 / (k * k);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const double f = (c < 3 ? 1.0 : -kinv2) * lm[c * S + s];
        sr += f * ar[c];
        si += f * ai[c];
      }
      if (wm) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          mr += wm[c * S + s] * ar[c];
          mi += wm[c * S + s] * ai[c];
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      si += __shfl_xor_sync(0xffffffffu, si, o);
      mr += __shfl_xor_sync(0xffffffffu, mr, o);
      mi += __shfl_xor_sync(0xffffffffu, mi, o);
    }
    if (lane == 0) {
      // j k eta (sr + j si) = k eta (-si + j sr)
      double2 v = make_double2(zr + jke * si, zi - jke * sr);
      double2 d = make_double2(zr, zi);
      if (wm) {
        const double2 zm0 = zMhalf[e], zm1 = zMhalf[nnz + e];
        const double zmr = zm0.x + zm1.x, zmi = zm0.y + zm1.y;
        const double be = (1.0 - alpha) * kEta0;
        v = make_double2(alpha * v.x + be * (zmr + mr), alpha * v.y + be * (zmi + mi));
        d = make_double2(alpha * d.x + be * zmr, alpha * d.y + be * zmi);
      }
      val[e] = v;
      if (!wm && m != n) val[et] = v;  // the transposed entry: same symmetrised MoM value and grid part
      if (m == n) diag[m] = d;
    }
  }
}

// Device part of the near fill on device inputs (see setup_dev.h).
int near_fill_dev(aim_ctx* c, const NearFillDev& A, double2* val, double2* diag) {
  const long long nnz = A.nnz, npairs = A.pairs->npairs;
  const size_t N = (size_t)c->N;
  Cd *blk = nullptr, *blkM = nullptr;
  double2 *zhalf = nullptr, *zMhalf = nullptr;
  int rc = AIM_OK;
  do {
    if ((rc = [&]() -> int {
           AIM_CUDA_TRY(cudaMallocAsync(&blk, sizeof(Cd) * 9 * std::max<long long>(1, npairs), c->stream));
           AIM_CUDA_TRY(cudaMallocAsync(&zhalf, sizeof(double2) * 2 * std::max<long long>(1, nnz), c->stream));
           if (A.lamM) {
             AIM_CUDA_TRY(cudaMallocAsync(&blkM, sizeof(Cd) * 9 * std::max<long long>(1, npairs), c->stream));
             AIM_CUDA_TRY(cudaMallocAsync(&zMhalf, sizeof(double2) * 2 * std::max<long long>(1, nnz), c->stream));
           }
           const TriRule* rs[3] = {A.rule_test, A.rule_test_sing, A.rule_src};
           for (int i = 0; i < 3; ++i)
             AIM_CUDA_TRY(cudaMemcpyToSymbolAsync(c_rules, rs[i], sizeof(TriRule), i * kRuleStride,
                                                  cudaMemcpyHostToDevice, c->stream));
           AIM_CUDA_TRY(cudaMemsetAsync(diag, 0, sizeof(double2) * N, c->stream));
           return AIM_OK;
         }()))
      break;
    FillGeom g{};
    g.vert = A.g.vert; g.tri = A.g.tri; g.area = A.g.area; g.tp = A.g.tp; g.tm = A.g.tm; g.sp = A.g.sp;
    g.sm = A.g.sm; g.len = A.g.len;
    const PairLists& pl = *A.pairs;
    // ids: the nsing singular pairs first, then the regular ones
    const long long nreg = npairs - pl.nsing;
    if (pl.nsing > 0) {
      AIM_LAUNCH(c, "near_pair_blocks", (k_pair_blocks<true><<<(unsigned)((pl.nsing + 127) / 128), 128, 0, c->stream>>>(
                                            g, pl.ids, pl.pP, pl.pQ, (int)pl.nsing, c->k, blk, blkM)));
      if ((rc = launch_check(c, "near_pair_blocks"))) break;
    }
    if (nreg > 0) {
      AIM_LAUNCH(c, "near_pair_blocks", (k_pair_blocks<false><<<(unsigned)((nreg + 127) / 128), 128, 0, c->stream>>>(
                                            g, pl.ids + pl.nsing, pl.pP, pl.pQ, (int)nreg, c->k, blk, blkM)));
      if ((rc = launch_check(c, "near_pair_blocks"))) break;
    }
    const double jke = c->k * kEta0;
    AIM_LAUNCH(c, "near_halves", (k_near_halves<<<152 * 16, 256, 0, c->stream>>>(g, A.erow, A.ecol, pl.tptr, pl.pQ, blk,
                                                                                   nnz, jke, zhalf, blkM, zMhalf)));
    if ((rc = launch_check(c, "near_halves"))) break;
    AIM_LAUNCH(c, "near_values", (k_near_values<<<152 * 16, 256, 0, c->stream>>>(A.erow, A.ecol, A.nptr, zhalf, A.lam,
                                                                                   A.anchor, A.gtab, A.TE, A.P, nnz,
                                                                                   c->k, jke, val, diag, zMhalf,
                                                                                   A.lamM, A.alpha)));
    if ((rc = launch_check(c, "near_values"))) break;
  } while (false);
  cudaFreeAsync(blk, c->stream);
  cudaFreeAsync(zhalf, c->stream);
  if (blkM) cudaFreeAsync(blkM, c->stream);
  if (zMhalf) cudaFreeAsync(zMhalf, c->stream);
  return rc;
}

}  // namespace aim
