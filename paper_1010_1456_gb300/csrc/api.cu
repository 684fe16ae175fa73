// C ABI entry points (include/aim.h): argument checks, context lifetime,
// buffer management, dispatch to the setup, product, solver and RCS code.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "common.h"

namespace aim {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

// staging vectors of a precision (grids are allocated on first use)
template <typename R> static int ensure_buffers(aim_ctx* c, PrecData<R>& p) {
  if (p.xbuf) return AIM_OK;
  const size_t e = sizeof(cplx<R>);
  AIM_CUDA_TRY(cudaMalloc(&p.xbuf, e * c->max_rhs * c->N));
  AIM_CUDA_TRY(cudaMalloc(&p.ybuf, e * c->max_rhs * c->N));
  return AIM_OK;
}

template <typename R> static void free_prec(PrecData<R>& p) {
  cudaFree(p.lam); cudaFree(p.lamM); cudaFree(p.pnode_w); cudaFree(p.ghat); cudaFree(p.near_val);
  for (int d = 0; d < 3; ++d) cudaFree(p.tw[d]);
  cudaFree(p.grid0); cudaFree(p.grid1); cudaFree(p.grid2); cudaFree(p.xbuf); cudaFree(p.ybuf);
  cudaFree(p.phiT); cudaFree(p.xT); cudaFree(p.ngrp_val);
  p = PrecData<R>{};
}

void free_context(aim_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  free_prec(c->p64);
  free_prec(c->p32);
  cudaFree(c->pff.ghat);
  for (int d = 0; d < 3; ++d) cudaFree(c->pff.tw[d]);
  cudaFree(c->pff.grid0); cudaFree(c->pff.grid1); cudaFree(c->pff.grid2);
  cudaFree(c->pff.pnode_w); cudaFree(c->pff.lam); cudaFree(c->pff.lamM); cudaFree(c->pff.near_val);
  cudaFree(c->pff.xff);
  cudaFree(c->plan_dev);
  free_krylov(c);
  profile_free(c);
  cudaFree(c->ngrp_ptr); cudaFree(c->ngrp_col); cudaFree(c->colmask);
  cudaFree(c->base); cudaFree(c->near_ptr); cudaFree(c->near_col); cudaFree(c->pnode_ptr); cudaFree(c->pnode_m);
  cudaFree(c->diag); cudaFree(c->dinv64); cudaFree(c->d_verts); cudaFree(c->d_tris); cudaFree(c->rwg_tri);
  cudaFree(c->rwg_free); cudaFree(c->rwg_len); cudaFree(c->tri_area); cudaFree(c->tri_nrm); cudaFree(c->pgroups);
  delete c;
}

static int check_ctx(const aim_ctx* c) {
  if (!c) {
    set_error("null context");
    return AIM_EINVAL;
  }
  return AIM_OK;
}

static int check_device() {
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    cudaGetLastError();
    set_error(std::string("no CUDA device: ") + cudaGetErrorString(e));
    return AIM_ENODEV;
  }
  return AIM_OK;
}

static bool mesh_finite(const aim_mesh* mesh) {
  for (long long i = 0; i < 3LL * mesh->nv; ++i)
    if (!std::isfinite(mesh->verts[i])) return false;
  return true;
}

// Device bytes of a context for this mesh once it has solved in `precision`
// (see aim_footprint in aim.h).
int footprint_estimate(const aim_mesh* mesh, double h, int M, double near_radius, int max_rhs, double alpha,
                       int precision, size_t* bytes) {
  (void)near_radius;
  if (mesh->nv < 1 || mesh->nt < 1 || !mesh->verts || !mesh->tris) {
    set_error("aim_footprint: empty mesh");
    return AIM_EINVAL;
  }
  if (!mesh_finite(mesh)) {
    set_error("aim_footprint: a vertex coordinate is NaN or infinite");
    return AIM_EINVAL;
  }
  // grid box from the vertices' bounding box, basis count from the edge count
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int i = 0; i < mesh->nv; ++i)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], mesh->verts[3 * i + d]);
      hi[d] = std::max(hi[d], mesh->verts[3 * i + d]);
    }
  long long n[3], L[3];
  for (int d = 0; d < 3; ++d) {
    n[d] = (long long)std::floor(hi[d] / h) - (long long)std::floor(lo[d] / h) + M + 1;
    long long m = 2 * n[d] - 1, x;
    for (L[d] = m;; ++L[d]) {
      x = L[d];
      for (int p : {2, 3, 5})
        while (x % p == 0) x /= p;
      if (x == 1) break;
    }
  }
  const long long N = (long long)(1.5 * mesh->nt);  // interior edges of a closed surface
  const long long S = (long long)(M + 1) * (M + 1) * (M + 1);
  const long long nnz = N * 100LL;  // generous near-row length
  const long long nc = n[0] * n[1] * n[2];
  const double cells = (double)max_rhs * 4 * (nc + L[2] * n[1] * n[0] + L[2] * L[1] * n[0]);
  double b = 0;
  b += (double)N * 4 * S * (8 + 4) * 2;                               // weights f64/f32 + node lists
  b += (double)nnz * (16 + 8 + 4);                                     // near values + columns
  b += (double)(L[0] / 2 + 1) * (L[1] / 2 + 1) * (L[2] / 2 + 1) * 24; // spectra
  b += (double)L[0] * L[1] * L[2] * 32;                                // setup transform scratch
  // pass grids of the precisions a solve in `precision` allocates
  b += cells * (precision == AIM_C64 ? 8 + 16 : 16);
  b += (double)max_rhs * N * (16 * 53 + 48);                           // Krylov basis (m = 50) and vectors
  if (precision != AIM_C128_F64)
    b += (double)N * 4 * S * 8 * 2 + (double)nnz * 16;                 // float-float weights and near values
  if (max_rhs >= kRhsLanesMin) {
    b += (double)max_rhs * (4.0 * nc + N) * 16;  // RHS-minor copies of Phi and x
    // near row groups: union columns (about 0.4 nnz) with kNearGroup entries each, in the solver precision
    b += (double)N / kNearGroup * 4 + 0.4 * nnz * (4 + kNearGroup * (precision == AIM_C64 ? 8 : 16));
  }
  b += (double)mesh->nt * 60 * (144 + 12) + (double)nnz * 56;          // near-fill scratch at setup (peak)
  if (alpha < 1.0)  // MFIE weights in three precisions, MFIE pair blocks and halves at setup
    b += (double)N * 3 * S * (8 + 4 + 8) + (double)mesh->nt * 60 * 144 + (double)nnz * 32;
  *bytes = (size_t)b;
  return AIM_OK;
}

// Grid bytes a product in `precision` allocates on first use, and whether
// the setup's estimate (solver precision opts.precision) already counts them.
size_t grid_bytes(const aim_ctx* c, int precision) {
  const double cells = (double)c->max_rhs * 4 *
                       ((double)c->n[0] * c->n[1] * c->n[2] + (double)c->L[2] * c->n[1] * c->n[0] +
                        (double)c->L[2] * c->L[1] * c->n[0]);
  return (size_t)(cells * (precision == AIM_C64 ? 8 : 16));
}

int budget_grids(aim_ctx* c, int precision) {
  if (c->opts.mem_budget == 0) return AIM_OK;
  const int sp = c->opts.precision;
  const bool planned = precision == sp || (sp == AIM_C64 && precision == AIM_C128);
  if (planned) return AIM_OK;
  const size_t need = grid_bytes(c, precision);
  if (c->planned_bytes + need > c->opts.mem_budget) {
    set_error("product grids of " + std::to_string(need) + " bytes would take the planned total above mem_budget (" +
              std::to_string(c->opts.mem_budget) + " bytes)");
    return AIM_ENOMEM;
  }
  c->planned_bytes += need;
  return AIM_OK;
}

}  // namespace aim

using namespace aim;

extern "C" {

const char* aim_last_error(void) { return g_last_error.c_str(); }

const char* aim_strerror(int code) {
  switch (code) {
    case AIM_OK: return "ok";
    case AIM_EINVAL: return "invalid argument";
    case AIM_ENOMEM: return "out of memory";
    case AIM_ECUDA: return "CUDA error";
    case AIM_ENOCONV: return "solver did not converge";
    case AIM_ETIMEOUT: return "device wait timed out";
    case AIM_ENODEV: return "no CUDA device";
    default: return "unknown error";
  }
}

void aim_default_opts(aim_opts* o) {
  if (!o) return;
  o->precision = AIM_C128;
  o->restart = 50;
  o->maxit = 3000;
  o->check_every = 5;
  o->max_rhs = 1;
  o->verbose = 0;
  o->stream = nullptr;
  o->planar = 1;
  o->cfie_alpha = 1.0;
  o->mem_budget = 0;
  o->krylov = AIM_GMRES;
}

int aim_setup(const aim_mesh* mesh, double k, double h, int M, double near_radius, const aim_opts* opts,
              aim_ctx** out) {
  if (!out) {
    set_error("aim_setup: out is NULL");
    return AIM_EINVAL;
  }
  *out = nullptr;
  if (!(k > 0.0) || !(h > 0.0) || M < 1 || M > 5 || !(near_radius >= 0.0)) {
    set_error("aim_setup: need k > 0, h > 0, 1 <= M <= 5, near_radius >= 0");
    return AIM_EINVAL;
  }
  aim_opts o;
  aim_default_opts(&o);
  if (opts) o = *opts;
  if (o.precision != AIM_C64 && o.precision != AIM_C128 && o.precision != AIM_C128_F64) {
    set_error("aim_setup: precision must be AIM_C64, AIM_C128 or AIM_C128_F64");
    return AIM_EINVAL;
  }
  if (!(o.cfie_alpha > 0.0 && o.cfie_alpha <= 1.0)) {
    set_error("aim_setup: cfie_alpha must be in (0, 1]");
    return AIM_EINVAL;
  }
  if (o.krylov != AIM_GMRES && o.krylov != AIM_TFQMR) {
    set_error("aim_setup: krylov must be AIM_GMRES or AIM_TFQMR");
    return AIM_EINVAL;
  }
  if (o.restart < 1 || o.restart > 200 || o.max_rhs < 1 || o.max_rhs > 256 || o.maxit < 1 || o.check_every < 1) {
    set_error("aim_setup: restart in 1..200, max_rhs in 1..256, maxit >= 1, check_every >= 1");
    return AIM_EINVAL;
  }
  if (!mesh || mesh->nv < 1 || mesh->nt < 1 || !mesh->verts || !mesh->tris) {
    set_error("aim_setup: empty mesh");
    return AIM_EINVAL;
  }
  if (!mesh_finite(mesh)) {
    set_error("aim_setup: a vertex coordinate is NaN or infinite");
    return AIM_EINVAL;
  }
  size_t planned = 0;
  if (o.mem_budget > 0) {
    AIM_TRY(footprint_estimate(mesh, h, M, near_radius, o.max_rhs, o.cfie_alpha, o.precision, &planned));
    if (planned > o.mem_budget) {
      set_error("aim_setup: footprint estimate " + std::to_string(planned) + " bytes exceeds mem_budget " +
                std::to_string(o.mem_budget));
      return AIM_ENOMEM;
    }
  }
  AIM_TRY(check_device());
  aim_ctx* c = new (std::nothrow) aim_ctx();
  if (!c) return AIM_ENOMEM;
  c->k = k;
  c->h = h;
  c->M = M;
  c->radius = near_radius;
  c->opts = o;
  c->max_rhs = o.max_rhs;
  c->stream = (cudaStream_t)o.stream;
  c->planned_bytes = planned;
  cudaGetDevice(&c->device);
  int rc = AIM_OK;
  try {
    rc = build_context(c, mesh);
  } catch (const std::bad_alloc&) {
    set_error("aim_setup: host allocation failed");
    rc = AIM_ENOMEM;
  }
  if (rc == AIM_OK) rc = ensure_buffers(c, c->p64);
  if (rc == AIM_OK) rc = ensure_buffers(c, c->p32);
  if (rc == AIM_OK) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      set_error(std::string("aim_setup: ") + cudaGetErrorString(e));
      rc = AIM_ECUDA;
    }
  }
  if (rc != AIM_OK) {
    if (rc == AIM_ECUDA && cudaGetLastError() == cudaErrorMemoryAllocation) rc = AIM_ENOMEM;
    free_context(c);
    return rc;
  }
  *out = c;
  return AIM_OK;
}

void aim_destroy(aim_ctx* ctx) { free_context(ctx); }

int aim_set_stream(aim_ctx* ctx, void* stream) {
  AIM_TRY(check_ctx(ctx));
  ctx->stream = (cudaStream_t)stream;
  return AIM_OK;
}

int aim_set_precision(aim_ctx* ctx, int precision) {
  AIM_TRY(check_ctx(ctx));
  if (precision != AIM_C64 && precision != AIM_C128 && precision != AIM_C128_F64) {
    set_error("aim_set_precision: precision must be AIM_C64, AIM_C128 or AIM_C128_F64");
    return AIM_EINVAL;
  }
  ctx->opts.precision = precision;
  return AIM_OK;
}

int aim_set_krylov(aim_ctx* ctx, int krylov) {
  AIM_TRY(check_ctx(ctx));
  if (krylov != AIM_GMRES && krylov != AIM_TFQMR) {
    set_error("aim_set_krylov: krylov must be AIM_GMRES or AIM_TFQMR");
    return AIM_EINVAL;
  }
  ctx->opts.krylov = krylov;
  return AIM_OK;
}

int aim_num_unknowns(const aim_ctx* ctx, int64_t* N) {
  AIM_TRY(check_ctx(ctx));
  if (!N) return AIM_EINVAL;
  *N = ctx->N;
  return AIM_OK;
}

int aim_grid_info(const aim_ctx* ctx, int32_t n[3], int32_t L[3], int64_t* nnz) {
  AIM_TRY(check_ctx(ctx));
  for (int d = 0; d < 3; ++d) {
    if (n) n[d] = ctx->n[d];
    if (L) L[d] = ctx->L[d];
  }
  if (nnz) *nnz = ctx->nnz;
  return AIM_OK;
}

int aim_rhs_planewave(aim_ctx* ctx, int nrhs, const double* khat, const double* pol, void* V_dev) {
  AIM_TRY(check_ctx(ctx));
  if (nrhs < 1 || !khat || !pol || !V_dev) {
    set_error("aim_rhs_planewave: bad arguments");
    return AIM_EINVAL;
  }
  for (int i = 0; i < 3 * nrhs; ++i)
    if (!std::isfinite(khat[i]) || !std::isfinite(pol[i])) {
      set_error("aim_rhs_planewave: khat or pol holds NaN or an infinity");
      return AIM_EINVAL;
    }
  return rhs_planewave(ctx, nrhs, khat, pol, (double2*)V_dev);
}

int aim_matvec(aim_ctx* ctx, const void* x_dev, void* y_dev, int nrhs, int precision) {
  AIM_TRY(check_ctx(ctx));
  if (nrhs < 1 || nrhs > ctx->max_rhs || !x_dev || !y_dev || x_dev == y_dev) {
    set_error("aim_matvec: need 1 <= nrhs <= max_rhs and distinct non-null x, y");
    return AIM_EINVAL;
  }
  if (precision != AIM_C64 && precision != AIM_C128 && precision != AIM_C128_F64) {
    set_error("aim_matvec: precision must be AIM_C64, AIM_C128 or AIM_C128_F64");
    return AIM_EINVAL;
  }
  return matvec(ctx, x_dev, y_dev, nrhs, precision);
}

int aim_matvec_host(aim_ctx* ctx, const void* x_host, void* y_host, int nrhs, int precision) {
  AIM_TRY(check_ctx(ctx));
  if (nrhs < 1 || nrhs > ctx->max_rhs || !x_host || !y_host) {
    set_error("aim_matvec_host: bad arguments");
    return AIM_EINVAL;
  }
  if (precision != AIM_C64 && precision != AIM_C128 && precision != AIM_C128_F64) {
    set_error("aim_matvec_host: precision must be AIM_C64, AIM_C128 or AIM_C128_F64");
    return AIM_EINVAL;
  }
  const bool wide = precision != AIM_C64;
  const size_t bytes = (size_t)nrhs * ctx->N * (wide ? 16 : 8);
  void* xd = wide ? (void*)ctx->p64.xbuf : (void*)ctx->p32.xbuf;
  void* yd = wide ? (void*)ctx->p64.ybuf : (void*)ctx->p32.ybuf;
  AIM_CUDA_TRY(cudaMemcpyAsync(xd, x_host, bytes, cudaMemcpyHostToDevice, ctx->stream));
  AIM_TRY(aim_matvec(ctx, xd, yd, nrhs, precision));
  AIM_CUDA_TRY(cudaMemcpyAsync(y_host, yd, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  AIM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return AIM_OK;
}

int aim_solve(aim_ctx* ctx, const void* V_dev, void* X_dev, int nrhs, double tol, aim_solve_info* info) {
  AIM_TRY(check_ctx(ctx));
  if (nrhs < 1 || nrhs > ctx->max_rhs || !V_dev || !X_dev || V_dev == X_dev || !(tol > 0.0)) {
    set_error("aim_solve: need 1 <= nrhs <= max_rhs, tol > 0, distinct non-null V, X");
    return AIM_EINVAL;
  }
  return solve(ctx, (const double2*)V_dev, (double2*)X_dev, nrhs, tol, info);
}

int aim_rcs(aim_ctx* ctx, const void* X_dev, int nrhs, int ndir, const double* theta, const double* phi,
            double* sig_tt, double* sig_pp) {
  AIM_TRY(check_ctx(ctx));
  if (nrhs < 1 || ndir < 1 || !X_dev || !theta || !phi || !sig_tt) {
    set_error("aim_rcs: bad arguments");
    return AIM_EINVAL;
  }
  for (int d = 0; d < ndir; ++d)
    if (!std::isfinite(theta[d]) || !std::isfinite(phi[d])) {
      set_error("aim_rcs: a direction angle is NaN or infinite");
      return AIM_EINVAL;
    }
  return rcs(ctx, (const double2*)X_dev, nrhs, ndir, theta, phi, sig_tt, sig_pp);
}

int aim_rcs_grid(int n_theta, int n_phi, double* theta, double* phi, double* weight) {
  if (n_theta < 1 || n_phi < 1 || n_theta > 100000 || !theta || !phi || !weight) {
    set_error("aim_rcs_grid: need 1 <= n_theta <= 100000, n_phi >= 1 and non-null outputs");
    return AIM_EINVAL;
  }
  return rcs_grid(n_theta, n_phi, theta, phi, weight);
}

int aim_err_thth(int nrhs, int ndir, const double* sigma, const double* ref, const double* weight, double* err) {
  if (nrhs < 1 || ndir < 1 || !sigma || !ref || !weight || !err) {
    set_error("aim_err_thth: bad arguments");
    return AIM_EINVAL;
  }
  return err_thth(nrhs, ndir, sigma, ref, weight, err);
}

int aim_mie_sigma_thth(double radius, double k, int ndir, const double* theta, const double* phi, double* sigma) {
  if (!(radius > 0.0) || !(k > 0.0) || !(k * radius <= 1e4) || ndir < 1 || !theta || !phi || !sigma) {
    set_error("aim_mie_sigma_thth: need radius > 0, k > 0, k radius <= 1e4, ndir >= 1, non-null arrays");
    return AIM_EINVAL;
  }
  return mie_sigma_thth(radius, k, ndir, theta, phi, sigma);
}

int aim_footprint(const aim_mesh* mesh, double h, int M, double near_radius, int max_rhs, double cfie_alpha,
                  int precision, size_t* bytes) {
  if (!mesh || !bytes || !(h > 0.0) || M < 1 || M > 5 || max_rhs < 1 || !(cfie_alpha > 0.0 && cfie_alpha <= 1.0) ||
      (precision != AIM_C64 && precision != AIM_C128 && precision != AIM_C128_F64)) {
    set_error("aim_footprint: bad arguments");
    return AIM_EINVAL;
  }
  return footprint_estimate(mesh, h, M, near_radius, max_rhs, cfie_alpha, precision, bytes);
}

int aim_export(aim_ctx* c, int what, void* dst, size_t bytes) {
  AIM_TRY(check_ctx(c));
  if (what != AIM_EXPORT_ANCHORS && what != AIM_EXPORT_GHAT) AIM_TRY(fetch_host_arrays(c));
  const void* src = nullptr;
  size_t need = 0;
  std::vector<double> full;
  switch (what) {
    case AIM_EXPORT_ANCHORS: src = c->h_anchor.data(); need = c->h_anchor.size() * 4; break;
    case AIM_EXPORT_WEIGHTS:
      if (c->planar) {  // the full stencil: the kept plane's weights, zeros elsewhere
        const int P = c->M + 1, S3 = P * P * P, S2 = P * P;
        full.assign((size_t)c->N * 4 * S3, 0.0);
        for (size_t mc = 0; mc < (size_t)c->N * 4; ++mc)
          for (int t = 0; t < S2; ++t) full[mc * S3 + (size_t)c->kk0 * S2 + t] = c->h_lam[mc * S2 + t];
        src = full.data();
        need = full.size() * 8;
      } else {
        src = c->h_lam.data();
        need = c->h_lam.size() * 8;
      }
      break;
    case AIM_EXPORT_NEAR_PTR: src = c->h_near_ptr.data(); need = c->h_near_ptr.size() * 4; break;
    case AIM_EXPORT_NEAR_COL: src = c->h_near_col.data(); need = c->h_near_col.size() * 4; break;
    case AIM_EXPORT_NEAR_VAL: src = c->h_near_val.data(); need = c->h_near_val.size() * 8; break;
    case AIM_EXPORT_DIAG: src = c->h_diag.data(); need = c->h_diag.size() * 8; break;
    case AIM_EXPORT_GHAT: src = c->h_ghat.data(); need = c->h_ghat.size() * 8; break;
    case AIM_EXPORT_PROJ_PTR: src = c->h_pnode_ptr.data(); need = c->h_pnode_ptr.size() * 4; break;
    case AIM_EXPORT_MFIE_WEIGHTS:
      if (c->h_lamM.empty()) {
        set_error("aim_export: MFIE weights exist only for a CFIE context (cfie_alpha < 1)");
        return AIM_EINVAL;
      }
      src = c->h_lamM.data();
      need = c->h_lamM.size() * 8;
      break;
    default: set_error("aim_export: unknown array"); return AIM_EINVAL;
  }
  if (!dst || bytes != need) {
    set_error("aim_export: size mismatch, need " + std::to_string(need) + " bytes");
    return AIM_EINVAL;
  }
  std::memcpy(dst, src, need);
  return AIM_OK;
}

int aim_launch_count(const aim_ctx* ctx, int64_t* count) {
  AIM_TRY(check_ctx(ctx));
  if (!count) return AIM_EINVAL;
  *count = ctx->launches;
  return AIM_OK;
}

int aim_probe_fma_peak(int which, double* tflops) {
  if (!tflops || (which != 32 && which != 64)) {
    set_error("aim_probe_fma_peak: which must be 32 or 64");
    return AIM_EINVAL;
  }
  AIM_TRY(check_device());
  return probe_fma(which, tflops);
}

}  // extern "C"
