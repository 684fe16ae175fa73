// Plane-wave right-hand sides and bistatic RCS.
//
// Excitation (paper Section 2.1): E_inc = pol exp(-j k khat . r) and
// V_m = int f_m . E_inc dS (collapsed Gauss-Legendre 4x4 rule per triangle).
// Far field (paper eq. 1 ingredients): N(rhat) = sum_m x_m int f_m
// exp(+j k rhat . r) dS (3x3 rule), sigma = k^2 eta^2 / (4 pi) |e . N|^2.
// The far field is evaluated as a sum over triangle quadrature points that
// carry the point current J_p = sum over the basis functions on the
// triangle of x_m f_m(r_p) A w_p (FP64, then rounded to FP32).  Every
// (direction, point) pair needs one phase factor exp(j k rhat . r_p): the
// phase is formed in float-float arithmetic (k rhat and r_p as pairs of
// floats, about 48 bits), reduced modulo 2 pi with a three-part constant,
// and its cosine and sine are taken in FP32 at the reduced high part with a
// first-order correction by the low part; the products with J_p are FP32,
// summed in FP32 over runs of 64 points and in FP64 beyond.  Per pair the
// phase factor is good to about 1 FP32 ulp and the product to a few, all on
// the FP32 pipes: a 16 lambda sphere's 5.4 M points times 326 k directions
// take seconds instead of the minutes of FP64 phases.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.h"
#include "ff.h"
#include "geom.h"

namespace aim {

constexpr int kRhsRule = 4, kFarRule = 3;
__constant__ double c_rhs_rule[3][kMaxRule * kMaxRule];
__constant__ double c_far_rule[3][kMaxRule * kMaxRule];

static int upload_rules() {
  static const int rc = [] {
    TriRule a = make_tri_rule(kRhsRule), b = make_tri_rule(kFarRule);
    double ha[3][kMaxRule * kMaxRule], hb[3][kMaxRule * kMaxRule];
    for (int q = 0; q < a.q; ++q) {
      ha[0][q] = a.xi1[q];
      ha[1][q] = a.xi2[q];
      ha[2][q] = a.w[q];
    }
    for (int q = 0; q < b.q; ++q) {
      hb[0][q] = b.xi1[q];
      hb[1][q] = b.xi2[q];
      hb[2][q] = b.w[q];
    }
    if (cudaMemcpyToSymbol(c_rhs_rule, ha, sizeof(ha)) != cudaSuccess) return 1;
    if (cudaMemcpyToSymbol(c_far_rule, hb, sizeof(hb)) != cudaSuccess) return 1;
    return 0;
  }();
  if (rc) {
    set_error("failed to upload quadrature rules");
    return AIM_ECUDA;
  }
  return AIM_OK;
}

__device__ __forceinline__ V3 ldv(const double* v, int i) { return v3(v[3 * i], v[3 * i + 1], v[3 * i + 2]); }

__global__ void k_rhs(const double* __restrict__ verts, const int32_t* __restrict__ tris,
                      const int32_t* __restrict__ rtri, const int32_t* __restrict__ rfree,
                      const double* __restrict__ len, const double* __restrict__ area, const double* __restrict__ khat,
                      const double* __restrict__ pol, double2* __restrict__ V, int N, double k,
                      const double* __restrict__ nrm, double alpha) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (m >= N) return;
  const V3 kh = v3(khat[3 * b], khat[3 * b + 1], khat[3 * b + 2]);
  const V3 pe = v3(pol[3 * b], pol[3 * b + 1], pol[3 * b + 2]);
  double re = 0.0, im = 0.0;
  const int nq = kRhsRule * kRhsRule;
  for (int half = 0; half < 2; ++half) {
    const int t = rtri[2 * m + half];
    const V3 fv = ldv(verts, rfree[2 * m + half]);
    const V3 r0 = ldv(verts, tris[3 * t]), r1 = ldv(verts, tris[3 * t + 1]), r2 = ldv(verts, tris[3 * t + 2]);
    const double A = area[t];
    const double cf = (half ? -1.0 : 1.0) * len[m] / (2.0 * A);
    // CFIE: alpha E_inc + (1 - alpha) eta n x H_inc, both tangential-tested;
    // eta H_inc = khat x pol times the same phase, n constant on the triangle.
    V3 pt = pe;
    if (nrm) pt = alpha * pe + (1.0 - alpha) * cross(ldv(nrm, t), cross(kh, pe));
    for (int q = 0; q < nq; ++q) {
      const V3 r = tri_point(r0, r1, r2, c_rhs_rule[0][q], c_rhs_rule[1][q]);
      const double fp = cf * dot(r - fv, pt) * A * c_rhs_rule[2][q];
      double s, c;
      sincos(k * dot(kh, r), &s, &c);
      re += fp * c;
      im -= fp * s;
    }
  }
  V[(long long)b * N + m] = make_double2(re, im);
}

// point currents: J[b][p][3] for p = t * 9 + q, positions rp[p][3]
__global__ void k_point_currents(const double* __restrict__ verts, const int32_t* __restrict__ tris,
                                 const int32_t* __restrict__ rtri, const int32_t* __restrict__ rfree,
                                 const double* __restrict__ len, const double* __restrict__ area,
                                 const double2* __restrict__ X, double2* __restrict__ J, double* __restrict__ rp,
                                 int N, int nt, int nrhs) {
  // one thread per (basis, half, point); contributions added with atomics
  const int nq = kFarRule * kFarRule;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= (long long)N * 2 * nq) return;
  const int q = (int)(tid % nq);
  const int half = (int)((tid / nq) % 2);
  const int m = (int)(tid / (2 * nq));
  const int t = rtri[2 * m + half];
  const V3 fv = ldv(verts, rfree[2 * m + half]);
  const V3 r0 = ldv(verts, tris[3 * t]), r1 = ldv(verts, tris[3 * t + 1]), r2 = ldv(verts, tris[3 * t + 2]);
  const double A = area[t];
  const V3 r = tri_point(r0, r1, r2, c_far_rule[0][q], c_far_rule[1][q]);
  const double cf = (half ? -1.0 : 1.0) * len[m] / (2.0 * A) * A * c_far_rule[2][q];
  const V3 f = cf * (r - fv);
  const long long p = (long long)t * nq + q;
  // every basis function on the triangle writes the same position
  rp[3 * p] = r.x;
  rp[3 * p + 1] = r.y;
  rp[3 * p + 2] = r.z;
  for (int b = 0; b < nrhs; ++b) {
    const double2 x = X[(long long)b * N + m];
    double2* Jp = J + ((long long)b * nt * nq + p) * 3;
    atomicAdd(&Jp[0].x, f.x * x.x);
    atomicAdd(&Jp[0].y, f.x * x.y);
    atomicAdd(&Jp[1].x, f.y * x.x);
    atomicAdd(&Jp[1].y, f.y * x.y);
    atomicAdd(&Jp[2].x, f.z * x.x);
    atomicAdd(&Jp[2].y, f.z * x.y);
  }
}

// Positions as float-float triples and currents in FP32 for the far-field
// kernel: rff [p][6] = (x.hi, x.lo, y.hi, y.lo, z.hi, z.lo), J32 [b][p][3].
__global__ void k_pack_points(const double* __restrict__ rp, const double2* __restrict__ J, float* __restrict__ rff,
                              float2* __restrict__ J32, long long npts, int nrhs) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npts;
       p += (long long)gridDim.x * blockDim.x) {
    for (int d = 0; d < 3; ++d) {
      const ff v = ff_from_double(rp[3 * p + d]);
      rff[6 * p + 2 * d] = v.hi;
      rff[6 * p + 2 * d + 1] = v.lo;
    }
    for (int b = 0; b < nrhs; ++b)
      for (int d = 0; d < 3; ++d) {
        const double2 j = J[((long long)b * npts + p) * 3 + d];
        J32[((long long)b * npts + p) * 3 + d] = make_float2((float)j.x, (float)j.y);
      }
  }
}

// 2 pi = kC1 + kC2 + kC3 with 12-bit kC1 and kC2: n * kC1 and n * kC2 are
// exact for integers |n| < 2^12 (phases below 2.5e4 rad).
constexpr float kC1 = 6.283203125f, kC2 = -1.7814338207244873e-05f, kC3 = -3.482206523131026e-09f;
constexpr float kInv2Pi = 0.15915493667125702f;
constexpr int kFarDirs = 4;      // directions per thread
constexpr int kFarChunk = 256;   // points staged per shared-memory chunk
constexpr int kFarRun = 64;      // points summed in FP32 before an FP64 add

// cos and sin of the phase k rhat . r for one direction (kr, float-float
// triple) and one point (r, float-float triple).
__device__ __forceinline__ void far_phase(const ff kr[3], const float* r, float& c, float& s) {
  ff p = ff_mul(kr[0], ff{r[0], r[1]});
  p = ff_mad(kr[1], ff{r[2], r[3]}, p);
  p = ff_mad(kr[2], ff{r[4], r[5]}, p);
  const float n = rintf(p.hi * kInv2Pi);
  const float a = __fmaf_rn(-n, kC1, p.hi);  // exact (Sterbenz; n kC1 has <= 24 bits)
  const ff b = ff_two_sum(a, -n * kC2);       // n kC2 exact
  const float lo = __fmaf_rn(-n, kC3, __fadd_rn(b.lo, p.lo));
  float sn, cs;
  sincosf(b.hi, &sn, &cs);
  s = __fmaf_rn(lo, cs, sn);
  c = __fmaf_rn(-lo, sn, cs);
}

// N[d][3] += sum over points [p_begin, p_end) of J_p exp(j k rhat_d . r_p),
// one right-hand side.  Block: 256 threads x kFarDirs directions
// (d = blockIdx.x * 1024 + i * 256 + threadIdx.x); blockIdx.y picks the
// point range.  N (FP64 complex [ndir][3]) must be zeroed; partial sums of
// the point ranges are added atomically.
__global__ void __launch_bounds__(256) k_farfield(const float* __restrict__ rff, const float2* __restrict__ J32,
                                                  const double* __restrict__ theta, const double* __restrict__ phi,
                                                  double2* __restrict__ Nacc, long long npts, int ndir,
                                                  long long pts_per_block, double k) {
  __shared__ float sr[kFarChunk][6];
  __shared__ float2 sj[kFarChunk][3];
  ff kr[kFarDirs][3];
  double2 acc[kFarDirs][3];
  float2 part[kFarDirs][3];
#pragma unroll
  for (int i = 0; i < kFarDirs; ++i) {
    const int d = min(blockIdx.x * (256 * kFarDirs) + i * 256 + threadIdx.x, ndir - 1);
    const double st = sin(theta[d]), ct = cos(theta[d]), sp = sin(phi[d]), cp = cos(phi[d]);
    kr[i][0] = ff_from_double(k * st * cp);
    kr[i][1] = ff_from_double(k * st * sp);
    kr[i][2] = ff_from_double(k * ct);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      acc[i][c] = make_double2(0.0, 0.0);
      part[i][c] = make_float2(0.f, 0.f);
    }
  }
  const long long p_begin = blockIdx.y * pts_per_block;
  const long long p_end = min(npts, p_begin + pts_per_block);
  for (long long p0 = p_begin; p0 < p_end; p0 += kFarChunk) {
    const int cnt = (int)(p_end - p0 < kFarChunk ? p_end - p0 : kFarChunk);
    __syncthreads();  // the previous chunk has been read
    if (threadIdx.x < cnt) {
      const long long p = p0 + threadIdx.x;
#pragma unroll
      for (int e = 0; e < 6; ++e) sr[threadIdx.x][e] = rff[6 * p + e];
#pragma unroll
      for (int c = 0; c < 3; ++c) sj[threadIdx.x][c] = J32[3 * p + c];
    }
    __syncthreads();
    for (int q = 0; q < cnt; ++q) {
      const float2 jx = sj[q][0], jy = sj[q][1], jz = sj[q][2];
#pragma unroll
      for (int i = 0; i < kFarDirs; ++i) {
        float c, s;
        far_phase(kr[i], sr[q], c, s);
        part[i][0].x = __fmaf_rn(jx.x, c, __fmaf_rn(-jx.y, s, part[i][0].x));
        part[i][0].y = __fmaf_rn(jx.x, s, __fmaf_rn(jx.y, c, part[i][0].y));
        part[i][1].x = __fmaf_rn(jy.x, c, __fmaf_rn(-jy.y, s, part[i][1].x));
        part[i][1].y = __fmaf_rn(jy.x, s, __fmaf_rn(jy.y, c, part[i][1].y));
        part[i][2].x = __fmaf_rn(jz.x, c, __fmaf_rn(-jz.y, s, part[i][2].x));
        part[i][2].y = __fmaf_rn(jz.x, s, __fmaf_rn(jz.y, c, part[i][2].y));
      }
      if ((q & (kFarRun - 1)) == kFarRun - 1 || q == cnt - 1) {
#pragma unroll
        for (int i = 0; i < kFarDirs; ++i)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            acc[i][c].x += (double)part[i][c].x;
            acc[i][c].y += (double)part[i][c].y;
            part[i][c] = make_float2(0.f, 0.f);
          }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < kFarDirs; ++i) {
    const int d = blockIdx.x * (256 * kFarDirs) + i * 256 + threadIdx.x;
    if (d >= ndir) continue;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      atomicAdd(&Nacc[3 * (long long)d + c].x, acc[i][c].x);
      atomicAdd(&Nacc[3 * (long long)d + c].y, acc[i][c].y);
    }
  }
}

// (N_theta, N_phi) [ndir] from the Cartesian far field N [ndir][3]
__global__ void k_far_project(const double2* __restrict__ Nacc, const double* __restrict__ theta,
                              const double* __restrict__ phi, double2* __restrict__ out, int ndir) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= ndir) return;
  const double st = sin(theta[d]), ct = cos(theta[d]), sp = sin(phi[d]), cp = cos(phi[d]);
  const double2 nx = Nacc[3 * (long long)d], ny = Nacc[3 * (long long)d + 1], nz = Nacc[3 * (long long)d + 2];
  out[2 * (long long)d] = make_double2(ct * cp * nx.x + ct * sp * ny.x - st * nz.x, ct * cp * nx.y + ct * sp * ny.y - st * nz.y);
  out[2 * (long long)d + 1] = make_double2(-sp * nx.x + cp * ny.x, -sp * nx.y + cp * ny.y);
}

int rhs_planewave(aim_ctx* c, int nrhs, const double* khat, const double* pol, double2* V) {
  AIM_TRY(upload_rules());
  double* dk = nullptr;
  AIM_CUDA_TRY(cudaMallocAsync(&dk, sizeof(double) * 6 * nrhs, c->stream));
  AIM_CUDA_TRY(cudaMemcpyAsync(dk, khat, sizeof(double) * 3 * nrhs, cudaMemcpyHostToDevice, c->stream));
  AIM_CUDA_TRY(cudaMemcpyAsync(dk + 3 * nrhs, pol, sizeof(double) * 3 * nrhs, cudaMemcpyHostToDevice, c->stream));
  dim3 grid((c->N + 127) / 128, nrhs);
  AIM_LAUNCH(c, "k_rhs", k_rhs<<<grid, 128, 0, c->stream>>>(c->d_verts, c->d_tris, c->rwg_tri, c->rwg_free, c->rwg_len, c->tri_area, dk,
                                     dk + 3 * nrhs, V, c->N, c->k, c->alpha < 1.0 ? c->tri_nrm : nullptr,
                                     c->alpha));
  AIM_TRY(launch_check(c, "k_rhs"));
  AIM_CUDA_TRY(cudaFreeAsync(dk, c->stream));
  AIM_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return AIM_OK;
}

int rcs(aim_ctx* c, const double2* X, int nrhs, int ndir, const double* theta, const double* phi, double* sig_tt,
        double* sig_pp) {
  AIM_TRY(upload_rules());
  const int nq = kFarRule * kFarRule;
  const long long npts = (long long)c->nt * nq;
  double2* J = nullptr;
  double *rp = nullptr, *dang = nullptr;
  double2 *Nacc = nullptr, *out = nullptr;
  float* rff = nullptr;
  float2* J32 = nullptr;
  AIM_CUDA_TRY(cudaMallocAsync(&J, sizeof(double2) * 3 * npts * nrhs, c->stream));
  AIM_CUDA_TRY(cudaMallocAsync(&rp, sizeof(double) * 3 * npts, c->stream));
  AIM_CUDA_TRY(cudaMallocAsync(&rff, sizeof(float) * 6 * npts, c->stream));
  AIM_CUDA_TRY(cudaMallocAsync(&J32, sizeof(float2) * 3 * npts * nrhs, c->stream));
  AIM_CUDA_TRY(cudaMallocAsync(&dang, sizeof(double) * 2 * ndir, c->stream));
  AIM_CUDA_TRY(cudaMallocAsync(&Nacc, sizeof(double2) * 3 * (size_t)ndir * nrhs, c->stream));
  AIM_CUDA_TRY(cudaMallocAsync(&out, sizeof(double2) * 2 * (size_t)ndir * nrhs, c->stream));
  AIM_CUDA_TRY(cudaMemsetAsync(J, 0, sizeof(double2) * 3 * npts * nrhs, c->stream));
  AIM_CUDA_TRY(cudaMemsetAsync(rp, 0, sizeof(double) * 3 * npts, c->stream));
  AIM_CUDA_TRY(cudaMemsetAsync(Nacc, 0, sizeof(double2) * 3 * (size_t)ndir * nrhs, c->stream));
  AIM_CUDA_TRY(cudaMemcpyAsync(dang, theta, sizeof(double) * ndir, cudaMemcpyHostToDevice, c->stream));
  AIM_CUDA_TRY(cudaMemcpyAsync(dang + ndir, phi, sizeof(double) * ndir, cudaMemcpyHostToDevice, c->stream));
  const long long nthr = (long long)c->N * 2 * nq;
  AIM_LAUNCH(c, "k_point_currents", k_point_currents<<<(unsigned)((nthr + 255) / 256), 256, 0, c->stream>>>(
      c->d_verts, c->d_tris, c->rwg_tri, c->rwg_free, c->rwg_len, c->tri_area, X, J, rp, c->N, c->nt, nrhs));
  AIM_TRY(launch_check(c, "k_point_currents"));
  AIM_LAUNCH(c, "k_pack_points", k_pack_points<<<(unsigned)std::min<long long>((npts + 255) / 256, 152LL * 16), 256, 0,
                                                  c->stream>>>(rp, J, rff, J32, npts, nrhs));
  AIM_TRY(launch_check(c, "k_pack_points"));
  // direction tiles x point ranges: at least about four blocks per SM in total
  const int per_block = 256 * kFarDirs;
  const int bx = (ndir + per_block - 1) / per_block;
  long long by = std::max<long long>(1, (4LL * 152 + bx - 1) / bx);
  by = std::min<long long>(by, std::max<long long>(1, npts / (4 * kFarChunk)));
  long long ppb = (npts + by - 1) / by;
  ppb = (ppb + kFarChunk - 1) / kFarChunk * kFarChunk;
  by = (npts + ppb - 1) / ppb;
  for (int b = 0; b < nrhs; ++b) {
    AIM_LAUNCH(c, "k_farfield", (k_farfield<<<dim3(bx, (unsigned)by), 256, 0, c->stream>>>(
                                    rff, J32 + (size_t)b * npts * 3, dang, dang + ndir, Nacc + (size_t)b * ndir * 3,
                                    npts, ndir, ppb, c->k)));
    AIM_TRY(launch_check(c, "k_farfield"));
    AIM_LAUNCH(c, "k_far_project", (k_far_project<<<(ndir + 255) / 256, 256, 0, c->stream>>>(
                                       Nacc + (size_t)b * ndir * 3, dang, dang + ndir, out + (size_t)b * ndir * 2, ndir)));
    AIM_TRY(launch_check(c, "k_far_project"));
  }
  std::vector<double2> h((size_t)2 * ndir * nrhs);
  AIM_CUDA_TRY(cudaMemcpyAsync(h.data(), out, sizeof(double2) * h.size(), cudaMemcpyDeviceToHost, c->stream));
  AIM_CUDA_TRY(cudaFreeAsync(J, c->stream));
  AIM_CUDA_TRY(cudaFreeAsync(rp, c->stream));
  AIM_CUDA_TRY(cudaFreeAsync(rff, c->stream));
  AIM_CUDA_TRY(cudaFreeAsync(J32, c->stream));
  AIM_CUDA_TRY(cudaFreeAsync(dang, c->stream));
  AIM_CUDA_TRY(cudaFreeAsync(Nacc, c->stream));
  AIM_CUDA_TRY(cudaFreeAsync(out, c->stream));
  AIM_CUDA_TRY(cudaStreamSynchronize(c->stream));
  const double fac = c->k * c->k * kEta0 * kEta0 / (4.0 * kPi);
  for (int b = 0; b < nrhs; ++b)
    for (int d = 0; d < ndir; ++d) {
      const double2 nt_ = h[((size_t)b * ndir + d) * 2], np_ = h[((size_t)b * ndir + d) * 2 + 1];
      sig_tt[(size_t)b * ndir + d] = fac * (nt_.x * nt_.x + nt_.y * nt_.y);
      if (sig_pp) sig_pp[(size_t)b * ndir + d] = fac * (np_.x * np_.x + np_.y * np_.y);
    }
  return AIM_OK;
}

}  // namespace aim
