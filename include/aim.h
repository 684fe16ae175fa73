/*
 * aim.h - C ABI of the GB300 AIM library: AIM-accelerated EFIE method of
 * moments for time-harmonic scattering from PEC surfaces (Wei & Yilmaz,
 * "A Hybrid Parallelization of AIM for Multi-Core Clusters", Sections 2.2
 * and 4.1; eq. 1 for the RCS error).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Units: lengths in wavelengths is customary (k = 2 pi) but any consistent
 * unit works; k is the wavenumber in the same unit.  Time convention
 * exp(+j w t), Green's function exp(-j k R) / (4 pi R), free-space impedance
 * 376.730313668 ohm.
 *
 * Complex vectors are interleaved (re, im) and RHS-major: element (b, m) of a
 * batch of nrhs vectors of length N sits at offset b*N + m.  AIM_C128 vectors
 * are pairs of doubles (16 bytes per element), AIM_C64 vectors pairs of
 * floats (8 bytes).  Pointers named *_dev are CUDA device pointers; all other
 * pointers are host pointers.  Device work is enqueued on the context's
 * stream (aim_opts.stream, changeable with aim_set_stream); a call returns
 * once its work is enqueued unless its comment says it synchronises.
 *
 * The unknowns are the RWG functions of the mesh's interior edges, ordered by
 * (low vertex index, high vertex index); the RWG's "+" triangle is the lower-
 * indexed of its two triangles.
 *
 * Errors: every int-returning call returns AIM_OK (0) or one of the AIM_E*
 * codes below and never aborts the process; aim_strerror() gives a message
 * and aim_last_error() the detail of the calling thread's last failure.
 * Ownership: the context owns all of its device and host memory; caller
 * buffers are only read or written during the call (or its enqueued work).
 */
#ifndef AIM_H
#define AIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  AIM_OK = 0,
  AIM_EINVAL = 1,   /* bad argument, bad mesh, unsupported size */
  AIM_ENOMEM = 2,   /* device or host allocation failed */
  AIM_ECUDA = 3,    /* a CUDA runtime call or kernel launch failed */
  AIM_ENOCONV = 4,  /* solver hit its iteration limit; X holds the last iterate */
  AIM_ETIMEOUT = 5, /* a bounded device wait gave up */
  AIM_ENODEV = 6    /* no CUDA device visible */
};

/*
 * Precisions of the product.  All three keep the setup arrays in FP64 and
 * round them once where a lower precision is used.
 *   AIM_C64      complex64 vectors; FP32 weights, spectrum, near entries,
 *                grids and accumulation (the mixed-precision inner product).
 *   AIM_C128     complex128 vectors (FP64 in and out); every step in between
 *                -- projection, FFT passes, spectral product, interpolation
 *                and near SpMV, with their weights, spectrum, near entries,
 *                grids and accumulations -- in float-float arithmetic (pairs
 *                of FP32 numbers, about 48 significant bits) on the FP32
 *                pipes: FP64-accurate (1e-12 against an FP64 reference), not
 *                native FP64.
 *   AIM_C128_F64 complex128 vectors; every step in native FP64 (the plain
 *                FP64 path; on GB300 its FFT is bound by the FP64 pipe).
 */
enum { AIM_C64 = 1, AIM_C128 = 2, AIM_C128_F64 = 3 };

typedef struct aim_ctx aim_ctx; /* opaque, library-owned */
typedef struct aim_pack aim_pack; /* opaque, library-owned: several contexts batched (aim_pack_create) */

/* Triangle mesh, copied by aim_setup (caller keeps ownership). */
typedef struct {
  int32_t nv;           /* number of vertices */
  int32_t nt;           /* number of triangles */
  const double* verts;  /* [nv][3] host, vertex coordinates */
  const int32_t* tris;  /* [nt][3] host, vertex indices, any orientation */
} aim_mesh;

/* Options; aim_default_opts() fills the defaults shown. */
typedef struct {
  int precision;   /* solver inner-product precision: AIM_C128 (default), AIM_C128_F64 or AIM_C64 */
  int restart;     /* GMRES restart length m (default 50, 1..200) */
  int maxit;       /* total inner iteration cap per solve (default 3000) */
  int check_every; /* host reads the residual estimate every k iterations (default 5) */
  int max_rhs;     /* largest nrhs the context is sized for (default 1, <= 256) */
  int verbose;     /* 0: silent (default); 1: aim_setup prints the wall time of its phases to stderr */
  void* stream;    /* cudaStream_t; NULL = the legacy default stream */
  int planar;      /* 1 (default): when every basis function's weights vanish off one z plane of
                      the grid (a planar scatterer at constant z on a node plane), keep only that
                      plane: the grid becomes nx x ny x 1 and the convolution two-dimensional
                      (same product up to rounding; aim_grid_info reports the reduced grid).
                      0: always three-dimensional. */
  double cfie_alpha; /* 1 (default): EFIE.  0 < alpha < 1: combined-field equation (paper Section
                      2.2, alpha = 0.6 for closed bodies) alpha EFIE + (1 - alpha) eta MFIE, for a
                      closed surface with outward-oriented triangles (vertex order (r0, r1, r2)
                      with (r1 - r0) x (r2 - r0) pointing out); aim_setup returns AIM_EINVAL for an
                      open mesh.  Products, right-hand sides and solves then use the CFIE. */
  size_t mem_budget; /* 0 (default): no limit.  Otherwise the most device memory, in bytes, the
                      context may plan to hold: aim_setup returns AIM_ENOMEM, before it allocates
                      anything, when aim_footprint's estimate for this mesh, max_rhs, cfie_alpha
                      and precision exceeds it; a later product in a precision whose grids that
                      estimate does not include (see aim_footprint) returns AIM_ENOMEM when its
                      grids would take the planned total above the budget. */
  int krylov;        /* AIM_GMRES (default): restarted GMRES(restart); AIM_TFQMR: transpose-free QMR
                      (nine vectors per right-hand side, no basis; restart is not used).  See aim_solve. */
} aim_opts;

/* Krylov methods of aim_solve (aim_opts.krylov, aim_set_krylov). */
enum { AIM_GMRES = 0, AIM_TFQMR = 1 };

/* Per-solve report. rel_res and iters are caller arrays of length nrhs. */
typedef struct {
  int32_t iterations;    /* inner steps taken, all right-hand sides in lockstep (GMRES: Arnoldi
                            steps; TFQMR: products) */
  int32_t restarts;      /* cycles (each ends with an FP64-accurate true residual) */
  double* rel_res;       /* [nrhs] out: final true relative residual ||b - Z x|| / ||b|| */
  int32_t* converged;    /* [nrhs] out: 1 if rel_res <= tol */
} aim_solve_info;

void aim_default_opts(aim_opts* opts);

/*
 * Build a context for one scatterer (paper Section 2.2: AIM fill), in FP64.
 * On the host: RWG functions (mesh topology), stencil anchors
 * a = floor(c/h - (M-1)/2) and the grid box.  On the device: moment-matching
 * weights on (M+1)^3 grid nodes (with CFIE also the MFIE's differentiated-
 * interpolation weights), near list |c_m - c_n| <= near_radius, projection
 * lists, near entries (symmetrised MoM entry minus its grid approximation;
 * with CFIE plus the MFIE entry minus its grid form) and the grid Green's
 * function spectrum on the zero-padded grid (padded length per axis =
 * smallest 2,3,5-smooth integer >= 2n-1), all kept resident.
 *   k > 0, h > 0, M in {1, ..., 5} (M = 2: 27 nodes; the paper's production
 *   setting is M = 3, its reference solutions go to M = 5), near_radius >= 0.
 *   Synchronises.
 * Returns AIM_EINVAL for a non-manifold or degenerate mesh, a mesh without
 * interior edges, vertex coordinates that are NaN or infinite, or a grid
 * whose padded size exceeds 2^31 points; AIM_ENOMEM when opts.mem_budget is
 * set and the footprint estimate exceeds it.
 */
int aim_setup(const aim_mesh* mesh, double k, double h, int M, double near_radius,
              const aim_opts* opts, aim_ctx** out);

void aim_destroy(aim_ctx* ctx); /* frees everything; NULL is a no-op; synchronises */

int aim_set_stream(aim_ctx* ctx, void* stream);

/* Change the solver's inner-product precision (AIM_C64, AIM_C128 or AIM_C128_F64)
 * after setup; AIM_EINVAL for anything else. */
int aim_set_precision(aim_ctx* ctx, int precision);

/* Change the solver's Krylov method (AIM_GMRES or AIM_TFQMR) after setup;
 * AIM_EINVAL for anything else. */
int aim_set_krylov(aim_ctx* ctx, int krylov);

/* N (number of unknowns). */
int aim_num_unknowns(const aim_ctx* ctx, int64_t* N);

/* Grid extents n[3] and padded extents L[3] (x, y, z), near-list nnz. */
int aim_grid_info(const aim_ctx* ctx, int32_t n[3], int32_t L[3], int64_t* nnz_near);

/*
 * Plane-wave right-hand sides V_m = int f_m . pol exp(-j k khat . r) dS
 * (paper Section 2.1 excitation), collapsed Gauss-Legendre 4x4 rule per
 * triangle; with CFIE, alpha V_m + (1 - alpha) int f_m . (n x (khat x pol))
 * exp(-j k khat . r) dS.  khat, pol: host [nrhs][3].  V_dev: device c128 [nrhs][N].
 * AIM_EINVAL if khat or pol holds NaN or an infinity.
 */
int aim_rhs_planewave(aim_ctx* ctx, int nrhs, const double* khat, const double* pol, void* V_dev);

/*
 * y = Z~ x: one AIM product for nrhs vectors (paper Section 4.1: projection,
 * pruned FFT convolution on the doubled grid, interpolation, near
 * correction).  precision AIM_C128 or AIM_C128_F64: x_dev, y_dev c128
 * [nrhs][N]; AIM_C64: x_dev, y_dev c64 [nrhs][N] (see the precision enum).
 * 1 <= nrhs <= opts.max_rhs.  x and y must not overlap.  Enqueued on the
 * context stream; does not synchronise, except that the first product in a
 * precision allocates that precision's grids (cudaMalloc).
 */
int aim_matvec(aim_ctx* ctx, const void* x_dev, void* y_dev, int nrhs, int precision);

/*
 * Same product with HOST buffers (x_host, y_host as in aim_matvec): copies x
 * to the device, runs the product and copies y back; synchronises.
 */
int aim_matvec_host(aim_ctx* ctx, const void* x_host, void* y_host, int nrhs, int precision);

/*
 * Solve Z~ X = V for nrhs right-hand sides (paper Section 2.2: diagonal
 * preconditioner, stop on the relative residual; the paper does not name its
 * Krylov method).  opts.krylov = AIM_GMRES: right-preconditioned restarted
 * GMRES(m), M^-1 = diag(Z~)^-1.  AIM_TFQMR: transpose-free QMR (Freund) on
 * the same preconditioned system, two products per step pair, its scalars on
 * the device and the step pair replayed from a CUDA graph; each cycle runs
 * until the quasi-residual bound falls below its target, then the true
 * residual is recomputed as for GMRES (info->restarts counts those cycles,
 * info->iterations the products).  GMRES:  On the device: the products,
 * classical Gram-Schmidt with FP64 dot products and a second pass where the
 * Daniel-Gragg-Kaufman-Stewart test asks for it, one Arnoldi step replayed
 * from a CUDA graph.  On the host, every opts.check_every steps: Givens
 * rotations of the new Hessenberg columns in FP64 and the residual estimate.
 * The Arnoldi products use opts.precision; every restart computes
 * the true residual with an FP64-accurate product (AIM_C128, or AIM_C128_F64
 * when that is opts.precision), so AIM_C64 is FP64 iterative refinement
 * around a complex64 inner solve.  Stops when every right-hand
 * side has ||V - Z~ X|| / ||V|| <= tol (true residual) or after opts.maxit
 * steps (AIM_ENOCONV).  V_dev, X_dev: device c128 [nrhs][N]; X is
 * overwritten (initial guess 0).  info may be NULL.  Synchronises.  A
 * right-hand side holding NaN or an infinity is rejected with AIM_EINVAL
 * before any iteration (its norm, computed first, is not finite).
 */
int aim_solve(aim_ctx* ctx, const void* V_dev, void* X_dev, int nrhs, double tol, aim_solve_info* info);

/*
 * Bistatic RCS of solved currents (paper eq. 1 ingredients):
 * sigma_tt = k^2 eta^2 / (4 pi) |theta . N|^2, sigma_pp likewise with phi,
 * N(rhat) = sum_m x_m int f_m exp(+j k rhat . r) dS (collapsed 3x3 rule).
 * theta, phi: host [ndir]; sig_tt, sig_pp: host [nrhs][ndir] (sig_pp may be
 * NULL).  X_dev: device c128 [nrhs][N].  Synchronises.
 */
int aim_rcs(aim_ctx* ctx, const void* X_dev, int nrhs, int ndir, const double* theta,
            const double* phi, double* sig_tt, double* sig_pp);

/*
 * Direction quadrature of the error measure of eq. (1) (the paper does not
 * state its quadrature): Gauss-Legendre nodes in cos(theta) (n_theta of
 * them, theta descending from pi) times n_phi uniform midpoint nodes in phi;
 * weight = Gauss weight * 2 pi / n_phi (the weights sum to 4 pi).  theta,
 * phi, weight: host [n_theta * n_phi], theta-major.  Host only; needs no GPU.
 */
int aim_rcs_grid(int n_theta, int n_phi, double* theta, double* phi, double* weight);

/*
 * Eq. (1): err[b] = sqrt( sum_d w_d (sigma[b][d] - ref[b][d])^2 / sum_d w_d ref[b][d]^2 ),
 * the relative RMS difference of two bistatic RCS patterns over the sphere of
 * directions.  sigma, ref: host [nrhs][ndir]; weight [ndir]; err [nrhs].
 * AIM_EINVAL if a reference pattern is zero.  Host only.
 */
int aim_err_thth(int nrhs, int ndir, const double* sigma, const double* ref, const double* weight, double* err);

/*
 * Reference RCS of a PEC sphere (paper Section 2.2: the sphere results of
 * Table 2 are measured against the analytic Mie series): bistatic sigma_thth
 * in m^2 (units of the length unit squared) of a sphere of radius `radius`
 * centred at the origin, lit by an x-polarised plane wave of unit amplitude
 * travelling along -z, at the directions (theta[d], phi[d]); wavenumber k in
 * the inverse length unit.  Series cut at n = ceil(ka + 4 (ka)^(1/3) + 10).
 * sigma: host [ndir].  Host only.
 */
int aim_mie_sigma_thth(double radius, double k, int ndir, const double* theta, const double* phi, double* sigma);

/* Bytes of device memory a context for this mesh would hold (estimate, +-10 %)
 * once it has solved with the solver precision `precision` (as aim_opts):
 * AIM_C64 counts the complex64 grids and the float-float grids of the
 * FP64-accurate refinement, AIM_C128 the float-float grids, AIM_C128_F64 the
 * native FP64 grids; cfie_alpha as in aim_opts (1: EFIE; < 1 adds the MFIE
 * arrays).  Not included: the fixed 64 MiB array of aim_matvec_c64_noalloc.
 * Host only.  AIM_EINVAL for a bad argument or a mesh with non-finite vertex
 * coordinates. */
int aim_footprint(const aim_mesh* mesh, double h, int M, double near_radius, int max_rhs, double cfie_alpha,
                  int precision, size_t* bytes);

/*
 * Copy internal setup arrays to host memory for inspection and testing.
 * what: AIM_EXPORT_ANCHORS int32 [N][3] (absolute node index),
 *       AIM_EXPORT_WEIGHTS f64 [N][4][(M+1)^3] (full stencil, also for a planar grid),
 *       AIM_EXPORT_NEAR_PTR int32 [N+1], AIM_EXPORT_NEAR_COL int32 [nnz],
 *       AIM_EXPORT_NEAR_VAL c128 [nnz], AIM_EXPORT_DIAG c128 [N],
 *       AIM_EXPORT_GHAT c128 octant [Lz/2+1][Ly/2+1][Lx/2+1] (scaled by 1/(Lx Ly Lz)),
 *       AIM_EXPORT_PROJ_PTR int32 [nx*ny*nz + 1] (per grid node, offsets into
 *       the node-ordered projection entries; the last value is their count),
 *       AIM_EXPORT_MFIE_WEIGHTS f64 [N][3][(M+1)^3] (CFIE contexts only: the
 *       differentiated-interpolation weights W^c_m(u) = int f_m . (n x (grad L_u x e_c)),
 *       c = x, y, z; AIM_EINVAL for an EFIE context).
 * bytes must equal the array size exactly.  Synchronises.
 */
enum {
  AIM_EXPORT_ANCHORS = 1,
  AIM_EXPORT_WEIGHTS = 2,
  AIM_EXPORT_NEAR_PTR = 3,
  AIM_EXPORT_NEAR_COL = 4,
  AIM_EXPORT_NEAR_VAL = 5,
  AIM_EXPORT_DIAG = 6,
  AIM_EXPORT_GHAT = 7,
  AIM_EXPORT_PROJ_PTR = 8,
  AIM_EXPORT_MFIE_WEIGHTS = 9
};
int aim_export(aim_ctx* ctx, int what, void* host_dst, size_t bytes);

/*
 * Kernel launches the library has issued from this context so far (all
 * entry points).  Lets a caller count launches inside a timed region.
 */
int aim_launch_count(const aim_ctx* ctx, int64_t* count);

/*
 * Per-kernel device timing of this context.  mode 1: from now on every kernel
 * launch is bracketed by two CUDA events on the context stream; mode 0: stop;
 * mode 2: clear the totals.  aim_profile_read synchronises the stream, then
 * reports for up to max_kernels kernel names (48-byte NUL-terminated slots in
 * names) the number of profiled launches and their total device time in ms;
 * *count receives the number of distinct names.
 */
int aim_profile(aim_ctx* ctx, int mode);
int aim_profile_read(aim_ctx* ctx, int max_kernels, char* names, int64_t* launches, double* ms, int* count);

/*
 * Measure the device's FP64 (which = 64) or FP32 (which = 32) FMA throughput
 * in TFLOP/s with a register-resident FMA loop on the current device.
 * Synchronises.
 */
int aim_probe_fma_peak(int which, double* tflops);

/*
 * FFT kernel selection.  The paper (Section 4.1) runs the convolution's
 * FFTs through a library and does not fix the transform; the choice here
 * changes the product only by rounding.  For each precision, each of the
 * five passes of the convolution (z forward, y forward, the fused x pass --
 * forward transform, spectral product, inverse -- y inverse, z inverse, in
 * that order) runs one of:
 *   AIM_FFT_AUTO            the built-in rule (default): four-step;
 *   AIM_FFT_STOCKHAM        mixed-radix Stockham kernel (any 2,3,5-smooth length);
 *   AIM_FFT_FOURSTEP        four-step register kernel (compiled lengths; any
 *                           other length falls back to the Stockham kernel);
 *   AIM_FFT_FOURSTEP_SMALL  four-step with blocks of at most 128 threads
 *                           (the x pass; elsewhere as AIM_FFT_FOURSTEP);
 *   AIM_FFT_FOURSTEP_WARP   four-step x pass whose pencils go through the
 *                           three steps in groups of 1-8 warps, each group
 *                           with its own barrier (the x pass; elsewhere as
 *                           AIM_FFT_FOURSTEP);
 *   AIM_FFT_FOURSTEP_WIDE   four-step strided pass with twice the columns per
 *                           block (the z and y passes; on the x pass as
 *                           AIM_FFT_FOURSTEP).
 * aim_fft_config sets (set != NULL, [5]) and/or reads (get != NULL, [5]) the
 * choices of one precision; get receives them with AUTO resolved by the rule.
 */
enum {
  AIM_FFT_AUTO = 0,
  AIM_FFT_STOCKHAM = 1,
  AIM_FFT_FOURSTEP = 2,
  AIM_FFT_FOURSTEP_SMALL = 3,
  AIM_FFT_FOURSTEP_WARP = 4,
  AIM_FFT_FOURSTEP_WIDE = 5
};
#define AIM_FFT_KERNELS 6 /* AIM_FFT_AUTO .. AIM_FFT_FOURSTEP_WIDE */
#define AIM_FFT_PASSES 5
int aim_fft_config(aim_ctx* ctx, int precision, const int32_t* set, int32_t* get);

/*
 * Autotune the FFT kernels of one precision for products of nrhs vectors
 * (1 <= nrhs <= opts.max_rhs, reps >= 1): pass by pass, each candidate
 * kernel runs one warm-up product and `reps` products timed with CUDA events
 * on the context stream, and the fastest stays selected.  Allocates (and
 * frees) one input and one output batch, and the precision's grids like the
 * first aim_matvec.  kernel_out [5] (may be NULL) receives the choices (a
 * planar grid has no z passes: those two keep their setting, untimed);
 * ms_out [5][AIM_FFT_KERNELS] (may be NULL) the mean time in ms of each pass under each
 * AIM_FFT_* value (-1 where not tried).  The profiler's totals and on/off
 * state are left as they were.  Synchronises.
 */
int aim_autotune(aim_ctx* ctx, int precision, int nrhs, int reps, int32_t* kernel_out, double* ms_out);

/*
 * Complex64 AIM product (same result as aim_matvec with AIM_C64) that
 * allocates no device memory.  The paper has no counterpart: this serves
 * callers that cannot let the library call cudaMalloc, because their device
 * memory belongs to another allocator or pool, or because an allocation
 * (which can synchronise the device) is not allowed in their loop.
 *   x_dev, y_dev: device c64 [nrhs][N], 1 <= nrhs <= opts.max_rhs, distinct.
 * The pass grids live in one fixed 64 MiB device array compiled into the
 * library (held by every GPU that loads the library until the process
 * exits); a product needs 8 * 4 * nrhs * (nx*ny*nz + Lz*ny*nx + Lz*Ly*nx)
 * bytes (each part rounded up to 256), and larger requests return
 * AIM_EINVAL with the size in aim_last_error().  The context's device must
 * be current (AIM_EINVAL otherwise).  Every call looks up the array's device
 * address (cudaGetSymbolAddress) in the current context; with lazy module
 * loading the driver maps the array at the first lookup in a context (the
 * set-up of that device), so the device's free memory drops by 64 MiB on the
 * first call and stays there until exit.  Make that first call before any
 * stream capture.  All calls share the array: calls whose work overlaps on
 * the GPU race and must be ordered by the caller.  The 64 MiB are not part of
 * aim_footprint's estimate.  The context itself is built by aim_setup.
 */
int aim_matvec_c64_noalloc(aim_ctx* ctx, const void* x_dev, void* y_dev, int nrhs);

/*
 * Multi-instance batching: several contexts (small scatterers, each with its
 * own mesh, weights, near list, CFIE weight and right-hand sides) go through
 * one launch per product stage.  The paper has no counterpart (it solves one
 * scatterer at a time); this serves a stream of many small requests, whose
 * products are launch-bound one by one.
 *
 * The pack lays every instance's grids over one box: per axis the largest
 * unpadded extent n_p and the largest padded length L_p among the instances.
 * Both come from an instance, so L_p >= 2 n_p - 1, and the pack's Green's
 * function spectrum (the circulant embedding over n_p on L_p, built at
 * creation) reproduces every instance's convolution exactly: an instance's
 * nodes fill the corner [0, n_i) of the box, so its products only involve
 * offsets |d| < n_i, where the two embeddings agree.  Products therefore equal
 * each instance's own to rounding.  Right-hand side b of the packed vectors
 * belongs to one instance; its four grids are the pack's grids 4b .. 4b+3,
 * and the z, y and x passes run over all of them at once.  Projection and
 * interpolation read each instance's own lists through a table of
 * descriptors.
 *
 * Packed vectors are RHS-major with row length ld = max N_i (aim_pack_dims):
 * element (b, m) at b*ld + m; instance i owns rows b0_i .. b0_i + nrhs_i - 1
 * (b0_0 = 0, in the order of ctxs), and entries m >= N_i of its rows are
 * padding, which products write as zero and solves keep at zero (right-hand
 * sides must be zero there).
 *
 * aim_pack_create: ctxs[K] (1 <= K <= 256, distinct), nrhs[K] (1 <= nrhs_i
 *   <= max_rhs of ctxs[i], sum <= 256).  The contexts must share the device,
 *   k, h, M and the stencil layout (all planar, or none), and must outlive
 *   the pack; while the pack is in use they must not run work of their own.
 *   The pack takes stream, restart, maxit, check_every and krylov from
 *   ctxs[0]'s options; its solver runs complex64 products with FP64-accurate
 *   true residuals (AIM_C64 refinement).  Allocates the pack's grids
 *   (complex64, 4 B grids over the pack's box, three pass buffers), spectrum,
 *   staging vectors and, at its first solve, solver storage; none of it is
 *   part of any context's aim_footprint estimate.  Synchronises.  AIM_EINVAL
 *   for mismatched contexts or bad counts.
 * aim_pack_dims: ld, total right-hand sides, and the first row b0 of each
 *   instance (b0 may be NULL, else [K]).
 * aim_pack_matvec: y = Z~ x for every packed row.  AIM_C64: x_dev, y_dev c64
 *   [B][ld], one launch per stage for all instances.  AIM_C128 or
 *   AIM_C128_F64: c128 [B][ld], each instance's FP64-accurate product in turn
 *   (the solver's true residuals).  x and y must not overlap.
 * aim_pack_solve: every instance's system at once, each right-hand side with
 *   its own Arnoldi process and diagonal preconditioner (as aim_solve); V_dev,
 *   X_dev c128 [B][ld]; info->rel_res and converged have B entries.
 *   Synchronises.
 * aim_pack_set_stream: the stream of the pack's work.
 * aim_pack_destroy: frees the pack (not the contexts); NULL is a no-op.
 */
int aim_pack_create(aim_ctx* const* ctxs, int K, const int32_t* nrhs, aim_pack** out);
int aim_pack_dims(const aim_pack* pack, int64_t* ld, int32_t* nrhs_total, int32_t* b0);
int aim_pack_matvec(aim_pack* pack, const void* x_dev, void* y_dev, int precision);
int aim_pack_solve(aim_pack* pack, const void* V_dev, void* X_dev, double tol, aim_solve_info* info);
int aim_pack_set_stream(aim_pack* pack, void* stream);
void aim_pack_destroy(aim_pack* pack);

const char* aim_strerror(int code);
const char* aim_last_error(void); /* thread-local detail of the last failure */

#ifdef __cplusplus
}
#endif
#endif /* AIM_H */
