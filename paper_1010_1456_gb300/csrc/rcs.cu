// Plane-wave right-hand sides and bistatic RCS.
//
// Excitation (paper Section 2.1): E_inc = pol exp(-j k khat . r) and
// V_m = int f_m . E_inc dS (collapsed Gauss-Legendre 4x4 rule per triangle).
// Far field (paper eq. 1 ingredients): N(rhat) = sum_m x_m int f_m
// exp(+j k rhat . r) dS (3x3 rule), sigma = k^2 eta^2 / (4 pi) |e . N|^2.
// The far field is evaluated as a sum over triangle quadrature points that
// carry the point current J_p = sum over the basis functions on the
// triangle of x_m f_m(r_p) A w_p; the phase k rhat . r_p is formed and reduced
// modulo 2 pi in FP64, its sine and cosine taken in FP32, and the sums are
// accumulated in FP64.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.h"
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

// one block per direction: N_theta and N_phi for every rhs
__global__ void __launch_bounds__(256) k_farfield(const double2* __restrict__ J, const double* __restrict__ rp,
                                                  const double* __restrict__ theta, const double* __restrict__ phi,
                                                  double2* __restrict__ out, long long npts, int nrhs, double k) {
  const int d = blockIdx.x;
  const double st = sin(theta[d]), ct = cos(theta[d]), sp = sin(phi[d]), cp = cos(phi[d]);
  const V3 rh = v3(st * cp, st * sp, ct), th = v3(ct * cp, ct * sp, -st), ph = v3(-sp, cp, 0.0);
  const double twopi = 2.0 * kPi;
  __shared__ double2 red[8][2];
  for (int b = 0; b < nrhs; ++b) {
    double2 at = make_double2(0, 0), ap = make_double2(0, 0);
    const double2* Jb = J + (long long)b * npts * 3;
    for (long long p = threadIdx.x; p < npts; p += blockDim.x) {
      const double phs = k * (rh.x * rp[3 * p] + rh.y * rp[3 * p + 1] + rh.z * rp[3 * p + 2]);
      const double red_ph = phs - twopi * rint(phs / twopi);
      float sf, cf;
      sincosf((float)red_ph, &sf, &cf);
      const double c = cf, s = sf;
      const double2 jx = Jb[3 * p], jy = Jb[3 * p + 1], jz = Jb[3 * p + 2];
      const double2 jt = make_double2(th.x * jx.x + th.y * jy.x + th.z * jz.x, th.x * jx.y + th.y * jy.y + th.z * jz.y);
      const double2 jp = make_double2(ph.x * jx.x + ph.y * jy.x, ph.x * jx.y + ph.y * jy.y);
      // (jt) * (c + j s)
      at.x += jt.x * c - jt.y * s;
      at.y += jt.x * s + jt.y * c;
      ap.x += jp.x * c - jp.y * s;
      ap.y += jp.x * s + jp.y * c;
    }
    for (int o = 16; o > 0; o >>= 1) {
      at.x += __shfl_xor_sync(0xffffffffu, at.x, o);
      at.y += __shfl_xor_sync(0xffffffffu, at.y, o);
      ap.x += __shfl_xor_sync(0xffffffffu, ap.x, o);
      ap.y += __shfl_xor_sync(0xffffffffu, ap.y, o);
    }
    if ((threadIdx.x & 31) == 0) {
      red[threadIdx.x >> 5][0] = at;
      red[threadIdx.x >> 5][1] = ap;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double2 a = make_double2(0, 0), c2 = make_double2(0, 0);
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        a.x += red[w][0].x;
        a.y += red[w][0].y;
        c2.x += red[w][1].x;
        c2.y += red[w][1].y;
      }
      out[((long long)b * gridDim.x + d) * 2] = a;
      out[((long long)b * gridDim.x + d) * 2 + 1] = c2;
    }
    __syncthreads();
  }
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
  double2* out = nullptr;
  AIM_CUDA_TRY(cudaMallocAsync(&J, sizeof(double2) * 3 * npts * nrhs, c->stream));
  AIM_CUDA_TRY(cudaMallocAsync(&rp, sizeof(double) * 3 * npts, c->stream));
  AIM_CUDA_TRY(cudaMallocAsync(&dang, sizeof(double) * 2 * ndir, c->stream));
  AIM_CUDA_TRY(cudaMallocAsync(&out, sizeof(double2) * 2 * (size_t)ndir * nrhs, c->stream));
  AIM_CUDA_TRY(cudaMemsetAsync(J, 0, sizeof(double2) * 3 * npts * nrhs, c->stream));
  AIM_CUDA_TRY(cudaMemsetAsync(rp, 0, sizeof(double) * 3 * npts, c->stream));
  AIM_CUDA_TRY(cudaMemcpyAsync(dang, theta, sizeof(double) * ndir, cudaMemcpyHostToDevice, c->stream));
  AIM_CUDA_TRY(cudaMemcpyAsync(dang + ndir, phi, sizeof(double) * ndir, cudaMemcpyHostToDevice, c->stream));
  const long long nthr = (long long)c->N * 2 * nq;
  AIM_LAUNCH(c, "k_point_currents", k_point_currents<<<(unsigned)((nthr + 255) / 256), 256, 0, c->stream>>>(
      c->d_verts, c->d_tris, c->rwg_tri, c->rwg_free, c->rwg_len, c->tri_area, X, J, rp, c->N, c->nt, nrhs));
  AIM_TRY(launch_check(c, "k_point_currents"));
  AIM_LAUNCH(c, "k_farfield", k_farfield<<<ndir, 256, 0, c->stream>>>(J, rp, dang, dang + ndir, out, npts, nrhs, c->k));
  AIM_TRY(launch_check(c, "k_farfield"));
  std::vector<double2> h((size_t)2 * ndir * nrhs);
  AIM_CUDA_TRY(cudaMemcpyAsync(h.data(), out, sizeof(double2) * h.size(), cudaMemcpyDeviceToHost, c->stream));
  AIM_CUDA_TRY(cudaFreeAsync(J, c->stream));
  AIM_CUDA_TRY(cudaFreeAsync(rp, c->stream));
  AIM_CUDA_TRY(cudaFreeAsync(dang, c->stream));
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
