// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/aim.h"

#define AIM_HD __host__ __device__

namespace aim {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);

struct Status {
  int code = AIM_OK;
};

#define AIM_CUDA_TRY(expr)                                                              \
  do {                                                                                  \
    cudaError_t _e = (expr);                                                            \
    if (_e != cudaSuccess) {                                                            \
      ::aim::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));             \
      return AIM_ECUDA;                                                                 \
    }                                                                                   \
  } while (0)

#define AIM_TRY(expr)              \
  do {                             \
    int _c = (expr);               \
    if (_c != AIM_OK) return _c;   \
  } while (0)

// ---------------------------------------------------------------- debug index checks
// Built with -DAIM_CHECK (build.py check=True, libaim_check.so), the product
// kernels test the indices they gather through before using them: every
// projection entry's basis function and every near column must lie in
// [0, N), and every stencil (its first node plus M along each axis) inside the
// grid.  A failed test skips the entries or the stencil in question and
// records the first failure (site, index) in the translation unit's own copy
// of the variables below; the host reads them after every product
// (read_index_checks), so a check build synchronises per product, and its
// solver launches the Arnoldi step without a CUDA graph.  Sites: 1 projection
// entry, 2 stencil, 3 near column (4, 5, 6: the same in the packed kernels).
#ifdef AIM_CHECK
static __device__ unsigned int g_check_fails;
static __device__ long long g_check_first[2];
__device__ __forceinline__ void index_fail(int site, long long idx) {
  if (atomicAdd(&g_check_fails, 1u) == 0) {
    g_check_first[0] = site;
    g_check_first[1] = idx;
  }
}
// every idx[e], e0 <= e < e1, in [0, n)
__device__ __forceinline__ bool indices_ok(const int32_t* idx, long long e0, long long e1, long long n, int site) {
  for (long long e = e0; e < e1; ++e)
    if (idx[e] < 0 || idx[e] >= n) {
      index_fail(site, idx[e]);
      return false;
    }
  return true;
}
// the stencil of (M+1) nodes per axis (one plane when S = (M+1)^2) from flat
// node `base` lies inside an nx x ny x (Nc / (nx ny)) grid
__device__ __forceinline__ bool stencil_ok(long long base, int nx, int ny, long long Nc, int P, int S, int site) {
  const long long plane = (long long)nx * ny;
  const bool ok = base >= 0 && base % nx + P - 1 < nx && (base / nx) % ny + P - 1 < ny &&
                  (base / plane + (S == P * P * P ? P - 1 : 0)) * plane < Nc;
  if (!ok) index_fail(site, base);
  return ok;
}
#endif

// ---------------------------------------------------------------- complex
template <typename R> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };
template <typename R> using cplx = typename cplx_t<R>::type;

template <typename C> AIM_HD inline C cmake(double re, double im) {
  C c;
  c.x = (decltype(c.x))re;
  c.y = (decltype(c.y))im;
  return c;
}
template <typename C> AIM_HD inline C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> AIM_HD inline C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> AIM_HD inline C cmul(C a, C b) {
  C c;
  c.x = a.x * b.x - a.y * b.y;
  c.y = a.x * b.y + a.y * b.x;
  return c;
}
template <typename C, typename R> AIM_HD inline C cscale(C a, R s) { a.x *= s; a.y *= s; return a; }
template <typename C> AIM_HD inline C cconj(C a) { a.y = -a.y; return a; }

// ---------------------------------------------------------------- plans
// Exact floor(n / d) for 0 <= n < 2^31 as (umulhi(n, m) + n) >> l.
struct Div32 {
  uint32_t m, l, d;
};
constexpr int kMaxStages = 16;
struct FftPlan {
  int L;                  // transform length
  int nst;                // number of stages (-1: L is not 2,3,5-smooth)
  int rad[kMaxStages];    // radix per stage, applied in order
  int Ns[kMaxStages];     // product of the radices of the earlier stages
  Div32 dNs[kMaxStages];  // division by Ns
  Div32 dnb[kMaxStages];  // division by L / rad
};
FftPlan make_plan(int L);  // radices from {4, 3, 5, 2}

// ---------------------------------------------------------------- per-precision device data
template <typename R> struct PrecData {
  R* lam = nullptr;               // [N][4][S] moment weights
  R* lamM = nullptr;              // [N][3][S] MFIE weights (CFIE only)
  R* pnode_w = nullptr;           // [nent][4] projection weights, node-ordered
  cplx<R>* ghat = nullptr;        // octant [Lz/2+1][Ly/2+1][Lx/2+1], scaled by 1/(LxLyLz)
  cplx<R>* near_val = nullptr;    // [nnz]
  cplx<R>* tw[3] = {nullptr, nullptr, nullptr};  // forward twiddles exp(-2 pi i t / L_d), t < L_d, then the
                                                 // four-step factors as [L1][L2] and [L2][L1] (3 L_d entries)
  cplx<R>* grid0 = nullptr;       // [B][4][nz][ny][nx]  Q, then Phi
  cplx<R>* grid1 = nullptr;       // [B][4][Lz][ny][nx]
  cplx<R>* grid2 = nullptr;       // [B][4][Lz][Ly][nx]
  cplx<R>* xbuf = nullptr;        // [B][N] staging for host/solver conversions
  cplx<R>* ybuf = nullptr;        // [B][N]
  cplx<R>* phiT = nullptr;        // [4][nz][ny][nx][B] Phi, RHS-minor (many-RHS interpolation)
  cplx<R>* xT = nullptr;          // [N][B] x, RHS-minor
  cplx<R>* ngrp_val = nullptr;    // [ngrp_nnz][kNearGroup] near entries per union column of a row group
};

// Float-float copies of the AIM_C128 path: spectrum, twiddles and grids of
// the FFT passes, and (rounded once from the FP64 setup arrays) the weights
// and near entries of the projection and interpolation.  A float-float real
// is (hi, lo) with value hi + lo; a complex one is float4 (re.hi, re.lo,
// im.hi, im.lo).
struct FFData {
  float4* ghat = nullptr;
  float4* tw[3] = {nullptr, nullptr, nullptr};
  float4* grid0 = nullptr;
  float4* grid1 = nullptr;
  float4* grid2 = nullptr;
  float4* pnode_w = nullptr;   // [nent][2]: (x, y, z, charge) high parts, then low parts
  float2* lam = nullptr;       // [N][4][S]
  float2* lamM = nullptr;      // [N][3][S] (CFIE only)
  float4* near_val = nullptr;  // [nnz]
  float4* xff = nullptr;       // [B][N] the product's input
};

// Per-kernel timing with CUDA events on the context stream (aim_profile).
struct ProfEvent {
  const char* name;
  cudaEvent_t a, b;
};
struct Profiler {
  bool on = false;
  std::vector<ProfEvent> pending;
  std::vector<cudaEvent_t> pool;
  std::vector<std::string> names;
  std::vector<double> ms;
  std::vector<int64_t> count;
};

struct KrylovWork {
  double2* V = nullptr;      // [B][m+1][N] Arnoldi basis (TFQMR: [B][9][N], its vectors)
  int slots = 0;             // vectors per right-hand side V holds
  double2* w = nullptr;      // [B][N]
  double2* r = nullptr;      // [B][N]
  double2* H = nullptr;      // [m][B][m+1] Hessenberg columns (column j of every RHS is contiguous)
  double2* partial = nullptr;// [B][nblk][m+1+kDotGroup] partial dots
  double2* y = nullptr;      // [B][m] least-squares solution of the cycle
  double* nrm = nullptr;     // [B] norms, [B] spare, then [B][nblk] norm partials
  double* bnorm = nullptr;   // [B]
  double2* h_H = nullptr;    // pinned host copy of H columns
  int* active = nullptr;     // [B]
  int* reorth = nullptr;     // [B] second Gram-Schmidt pass needed for the current column
  int* jdev = nullptr;       // current Arnoldi column (read by the step's kernels)
  int m = 0;
  int nblk = 0;              // blocks per right-hand side of the norm kernel
  int nblk_dot = 0;          // blocks per right-hand side and vector group of the dot kernel
  // CUDA graph of one Arnoldi step (per precision and batch size), captured
  // on a private stream (the legacy default stream cannot be captured)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t step_exec = nullptr;
  int step_prec = 0, step_nrhs = 0;
  int64_t step_launches = 0;
};

}  // namespace aim

struct aim_ctx {
  // problem
  int N = 0, M = 2, S = 27;  // S: stencil nodes per basis function ((M+1)^3, or (M+1)^2 on a planar grid)
  int planar = 0;            // grid reduced to the one z plane that holds every nonzero weight
  // Projection over node groups: the projection writes only the listed
  // 8-node groups (those with entries) into grid0, which was zeroed once, and
  // the inverse z pass leaves Phi in grid2 so grid0 keeps its zeros (grids
  // with z passes only)
  int sparse_proj = 0;
  int32_t* pgroups = nullptr;  // [ngroups] indices g of the groups [8g, 8g + 8) with entries
  // Grids with z passes: [ny][nx] flags of the (x, y) columns that hold a
  // stencil node.  The forward z pass reads no other column (its input is
  // zero there) and the inverse z pass writes no other (nothing interpolates
  // from it).
  uint8_t* colmask = nullptr;
  int64_t ngroups = 0;
  double alpha = 1.0;        // CFIE weight of the EFIE (1: EFIE)
  int kk0 = 0;               // that plane's offset in the stencil
  double k = 0, h = 0, radius = 0;
  int lo[3] = {0, 0, 0};
  int n[3] = {0, 0, 0};  // grid nodes x, y, z
  int L[3] = {0, 0, 0};  // padded
  int64_t nnz = 0;
  int64_t nent = 0;      // projection entries
  aim_opts opts;
  cudaStream_t stream = nullptr;
  int device = 0;
  size_t planned_bytes = 0;  // aim_footprint estimate at setup plus grids added beyond it (mem_budget)
  bool host_synced = false;  // the h_* copies below hold the device setup arrays (fetch_host_arrays)
  int64_t launches = 0;
  // FFT kernel per arithmetic policy (complex64, native FP64, float-float) and
  // pass (z fwd, y fwd, x, y inv, z inv): AIM_FFT_AUTO, AIM_FFT_STOCKHAM,
  // AIM_FFT_FOURSTEP, AIM_FFT_FOURSTEP_SMALL, AIM_FFT_FOURSTEP_WARP or AIM_FFT_FOURSTEP_WIDE (set by aim_fft_config and
  // aim_autotune).
  int32_t fft_kernel[3][AIM_FFT_PASSES] = {};
  aim::FftPlan plan[3];
  aim::FftPlan* plan_dev = nullptr;  // device copy of plan[3]

  // host copies: anchors always, the rest filled by fetch_host_arrays on aim_export
  std::vector<int32_t> h_anchor;  // [N][3] absolute
  std::vector<double> h_lam;      // [N][4][S]
  std::vector<double> h_lamM;     // [N][3][S] CFIE: differentiated-interpolation (MFIE) weights
  std::vector<int32_t> h_near_ptr, h_near_col;
  std::vector<double> h_near_val; // [nnz][2]
  std::vector<double> h_diag;     // [N][2]
  std::vector<double> h_ghat;     // octant [..][2]
  std::vector<int32_t> h_pnode_ptr;  // [Nc+1]

  // device, precision independent
  int32_t* base = nullptr;        // [N] flat index of the stencil's first node
  int32_t* near_ptr = nullptr;    // [N+1]
  int32_t* near_col = nullptr;    // [nnz]
  int32_t* pnode_ptr = nullptr;   // [Nc+1]
  int32_t* pnode_m = nullptr;     // [nent]
  // many-RHS near product: rows in groups of kNearGroup consecutive basis
  // functions, each group's near columns merged (sorted union), built on the
  // first product with lanes over right-hand sides
  int32_t* ngrp_ptr = nullptr;    // [ngroups + 1]
  int32_t* ngrp_col = nullptr;    // [ngrp_nnz]
  long long ngrp_nnz = 0;
  double2* diag = nullptr;        // [N] diag(Z~) FP64
  double2* dinv64 = nullptr;      // [N] 1/diag
  // RWG geometry on device (for RHS and far field)
  double* d_verts = nullptr;      // [nv][3]
  double* tri_nrm = nullptr;      // [nt][3] unit normals (CFIE right-hand side)
  int32_t* d_tris = nullptr;      // [nt][3]
  int32_t* rwg_tri = nullptr;     // [N][2] (T+, T-)
  int32_t* rwg_free = nullptr;    // [N][2] free vertex of T+, T-
  double* rwg_len = nullptr;      // [N]
  double* tri_area = nullptr;     // [nt]
  int nv = 0, nt = 0;

  aim::PrecData<double> p64;
  aim::PrecData<float> p32;
  aim::FFData pff;
  aim::KrylovWork kw;
  aim::Profiler prof;
  int max_rhs = 1;
  // Multi-instance packs (pack.cu): the pack's internal context has `pack`
  // set, so its products run the packed kernels, and holds one diagonal per
  // right-hand side (dinv_ld = N, the packed row length; 0: one diagonal for
  // every right-hand side).
  aim_pack* pack = nullptr;
  long long dinv_ld = 0;
};

namespace aim {
// Brackets one kernel launch with profiling events when profiling is on and
// counts the launch.
struct LaunchScope {
  aim_ctx* c;
  bool on;
  cudaEvent_t b = nullptr;
  const char* name;
  LaunchScope(aim_ctx* ctx, const char* nm);
  ~LaunchScope();
};
#define AIM_LAUNCH(ctx, name, ...)        \
  do {                                    \
    ::aim::LaunchScope _ls((ctx), (name)); \
    __VA_ARGS__;                          \
  } while (0)
int profile_collect(aim_ctx* c);
void profile_free(aim_ctx* c);
// setup.cu
int build_context(aim_ctx* c, const aim_mesh* mesh);
// matvec.cu: y = Z~ x; precision AIM_C64 (float2 vectors) or AIM_C128 /
// AIM_C128_F64 (double2 vectors).  Allocates the grids of a precision on its
// first use.
int matvec(aim_ctx* c, const void* x, void* y, int nrhs, int precision);
int ensure_grids(aim_ctx* c, int precision);
int launch_check(aim_ctx* c, const char* what);
int convert_c128_to_c64(aim_ctx* c, const double2* in, float2* out, int64_t count);
int convert_c64_to_c128(aim_ctx* c, const float2* in, double2* out, int64_t count);
// fft.cu
// grid0 (Q) -> grid0 (Phi) of each precision, G = 4 * nrhs grids
// Phi's grid: grid2 for a context that projects over node groups, else grid0.
template <class T> inline T* phi_grid(const aim_ctx* c, T* g0, T* g2) { return c->sparse_proj ? g2 : g0; }
// The four-step split L = L1 * L2 of a padded length that has four-step
// kernels (false for the Stockham-only lengths).
bool fourstep_split(int L, int* L1, int* L2);
int fft_convolve_c64(aim_ctx* c, int G);
int fft_convolve_c128(aim_ctx* c, int G);
int fft_convolve_ff(aim_ctx* c, int G);
// complex64 product and convolution on caller-provided grids (noalloc.cu)
int fft_convolve_c64_bufs(aim_ctx* c, int G, float2* g0, float2* g1, float2* g2);
// FFT kernel tables: policy index of a precision (0 complex64, 1 native FP64,
// 2 float-float) and the kernel a pass runs (AIM_FFT_AUTO resolved).
int fft_policy_of(int precision);
int fft_kernel_for(const aim_ctx* c, int pol, int pass);
int matvec_c64_bufs(aim_ctx* c, const float2* x, float2* y, int nrhs, float2* g0, float2* g1, float2* g2);
int build_ghat(aim_ctx* c);
// krylov.cu
int solve(aim_ctx* c, const double2* V, double2* X, int nrhs, double tol, aim_solve_info* info);

// setup.cu: copies of the device setup arrays (weights, near list and
// values, diagonal, projection pointers) into the context's host vectors,
// once, for aim_export.
int fetch_host_arrays(aim_ctx* c);
int alloc_krylov(aim_ctx* c);
// api.cu: footprint estimate (aim_footprint), and the mem_budget check of the
// grids of a product precision the setup's estimate did not count.
int footprint_estimate(const aim_mesh* mesh, double h, int M, double near_radius, int max_rhs, double alpha,
                       int precision, size_t* bytes);
size_t grid_bytes(const aim_ctx* c, int precision);
int budget_grids(aim_ctx* c, int precision);
// Allocates everything a product of this precision allocates lazily, so a
// product can be captured into a CUDA graph.
int prepare_product(aim_ctx* c, int precision);
// Right-hand sides from which the products run with lanes over them.
constexpr int kRhsLanesMin = 16;
// Rows per group of the many-RHS near product.
constexpr int kNearGroup = 4;
// Forgets the solver's captured Arnoldi step (after the kernel choice changed).
void drop_step_graph(aim_ctx* c);
void free_krylov(aim_ctx* c);
// setup.cu: FFT plans (c->plan set), twiddle tables and spectrum storage.
int fft_tables(aim_ctx* c);
// api.cu: frees a context and everything it owns.
void free_context(aim_ctx* c);
// pack.cu: products and preparation of a pack's internal context.
int pack_matvec(aim_ctx* c, const void* x, void* y, int nrhs, int precision);
int pack_prepare(aim_ctx* c, int precision);
#ifdef AIM_CHECK
// The index checks of this translation unit's kernels since the last read:
// AIM_EINVAL with the first failure (site, index) in aim_last_error, then the
// count is cleared.  Synchronises the stream.
[[maybe_unused]] static int read_index_checks(aim_ctx* c, const char* where) {
  unsigned int n = 0;
  long long first[2] = {0, 0};
  AIM_CUDA_TRY(cudaMemcpyFromSymbolAsync(&n, g_check_fails, sizeof(n), 0, cudaMemcpyDeviceToHost, c->stream));
  AIM_CUDA_TRY(cudaMemcpyFromSymbolAsync(first, g_check_first, sizeof(first), 0, cudaMemcpyDeviceToHost, c->stream));
  AIM_CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (n == 0) return AIM_OK;
  const unsigned int zero = 0;
  AIM_CUDA_TRY(cudaMemcpyToSymbolAsync(g_check_fails, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, c->stream));
  AIM_CUDA_TRY(cudaStreamSynchronize(c->stream));
  set_error(std::string(where) + ": index check failed " + std::to_string(n) + " time(s); first at site " +
            std::to_string(first[0]) + ", index " + std::to_string(first[1]));
  return AIM_EINVAL;
}
#endif
// rcs.cu
int rhs_planewave(aim_ctx* c, int nrhs, const double* khat, const double* pol, double2* V);
int rcs(aim_ctx* c, const double2* X, int nrhs, int ndir, const double* theta, const double* phi,
        double* sig_tt, double* sig_pp);
// rcs_ref.cu (host only)
int rcs_grid(int n_theta, int n_phi, double* theta, double* phi, double* weight);
int err_thth(int nrhs, int ndir, const double* sig, const double* ref, const double* w, double* err);
int mie_sigma_thth(double radius, double k, int ndir, const double* theta, const double* phi, double* sigma);
// probe.cu
int probe_fma(int which, double* tflops);
}  // namespace aim
