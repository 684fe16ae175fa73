// FFT kernel selection per pass (aim_fft_config) and its autotuner
// (aim_autotune).  Every candidate computes the same transform; they differ
// in how a pencil is split between registers and shared memory, so the
// fastest depends on the padded lengths, the number of grids and the
// arithmetic policy, and is measured rather than predicted.
#include <cstdint>

#include "common.h"

namespace aim {

static const char* const kPassName[AIM_FFT_PASSES] = {"fft_z_fwd", "fft_y_fwd", "fft_x_conv", "fft_y_inv",
                                                      "fft_z_inv"};

static bool valid_precision(int p) { return p == AIM_C64 || p == AIM_C128 || p == AIM_C128_F64; }

// Deterministic test input: uniform values in [-1, 1) from an integer hash
// of the element index (timing only; the values do not matter).
template <class C>
__global__ void k_fill_hash(C* x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)i * 2654435761u;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    const float re = (float)(h & 0xffff) / 32768.f - 1.f;
    const float im = (float)(h >> 16) / 32768.f - 1.f;
    x[i].x = re;
    x[i].y = im;
  }
}

// Mean device time (ms) of one pass over `reps` products, profiler on.
static int time_pass(aim_ctx* c, int pass, const void* x, void* y, int nrhs, int precision, int reps, double* ms) {
  AIM_TRY(matvec(c, x, y, nrhs, precision));  // warm-up: first launch of the kernel, its attributes
  AIM_TRY(profile_collect(c));
  c->prof.names.clear();
  c->prof.ms.clear();
  c->prof.count.clear();
  for (int r = 0; r < reps; ++r) AIM_TRY(matvec(c, x, y, nrhs, precision));
  AIM_TRY(profile_collect(c));
  *ms = -1.0;
  for (size_t i = 0; i < c->prof.names.size(); ++i)
    if (c->prof.names[i] == kPassName[pass] && c->prof.count[i] > 0) *ms = c->prof.ms[i] / (double)c->prof.count[i];
  if (*ms < 0) {
    set_error(std::string("aim_autotune: no timed launch of ") + kPassName[pass]);
    return AIM_ECUDA;
  }
  return AIM_OK;
}

static int autotune(aim_ctx* c, int precision, int nrhs, int reps, int32_t* kernel_out, double* ms_out) {
  const int pol = fft_policy_of(precision);
  const size_t elem = precision == AIM_C64 ? sizeof(float2) : sizeof(double2);
  const long long n = (long long)nrhs * c->N;
  void* x = nullptr;
  void* y = nullptr;
  if (cudaMalloc(&x, n * elem) != cudaSuccess || cudaMalloc(&y, n * elem) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(x);
    set_error("aim_autotune: cannot allocate the scratch batch");
    return AIM_ENOMEM;
  }
  int rc = AIM_OK;
  {
    const int blocks = (int)std::min<long long>((n + 255) / 256, 4 * 152);
    if (precision == AIM_C64)
      AIM_LAUNCH(c, "autotune_fill", (k_fill_hash<<<blocks, 256, 0, c->stream>>>(static_cast<float2*>(x), n)));
    else
      AIM_LAUNCH(c, "autotune_fill", (k_fill_hash<<<blocks, 256, 0, c->stream>>>(static_cast<double2*>(x), n)));
    rc = launch_check(c, "autotune_fill");
  }
  if (ms_out)
    for (int i = 0; i < AIM_FFT_PASSES * AIM_FFT_KERNELS; ++i) ms_out[i] = -1.0;
  for (int pass = 0; pass < AIM_FFT_PASSES && rc == AIM_OK; ++pass) {
    if ((pass == 0 || pass == 4) && c->L[2] == 1) continue;  // a planar grid has no z passes
    int best = AIM_FFT_AUTO;
    double best_ms = 0.0;
    for (int k = AIM_FFT_STOCKHAM; k < AIM_FFT_KERNELS && rc == AIM_OK; ++k) {
      // the x pass has the block-size and warp-group variants, the strided passes the wide one
      const bool x_only = k == AIM_FFT_FOURSTEP_SMALL || k == AIM_FFT_FOURSTEP_WARP;
      if (pass == 2 ? k == AIM_FFT_FOURSTEP_WIDE : x_only) continue;
      c->fft_kernel[pol][pass] = k;
      double ms = 0.0;
      rc = time_pass(c, pass, x, y, nrhs, precision, reps, &ms);
      if (rc == AIM_EINVAL) {  // this kernel does not serve the length (shared memory): not a candidate
        rc = AIM_OK;
        continue;
      }
      if (rc != AIM_OK) break;
      if (ms_out) ms_out[pass * AIM_FFT_KERNELS + k] = ms;
      if (best == AIM_FFT_AUTO || ms < best_ms) {
        best = k;
        best_ms = ms;
      }
    }
    c->fft_kernel[pol][pass] = best;
  }
  if (rc == AIM_OK && kernel_out)
    for (int pass = 0; pass < AIM_FFT_PASSES; ++pass) kernel_out[pass] = fft_kernel_for(c, pol, pass);
  cudaStreamSynchronize(c->stream);
  cudaFree(x);
  cudaFree(y);
  return rc;
}

}  // namespace aim

using namespace aim;

extern "C" int aim_fft_config(aim_ctx* ctx, int precision, const int32_t* set, int32_t* get) {
  if (!ctx || !valid_precision(precision)) {
    set_error("aim_fft_config: need a context and AIM_C64, AIM_C128 or AIM_C128_F64");
    return AIM_EINVAL;
  }
  const int pol = fft_policy_of(precision);
  if (set) {
    for (int i = 0; i < AIM_FFT_PASSES; ++i)
      if (set[i] < AIM_FFT_AUTO || set[i] >= AIM_FFT_KERNELS) {
        set_error("aim_fft_config: kernel choices are AIM_FFT_AUTO .. AIM_FFT_FOURSTEP_WIDE");
        return AIM_EINVAL;
      }
    for (int i = 0; i < AIM_FFT_PASSES; ++i) ctx->fft_kernel[pol][i] = set[i];
    drop_step_graph(ctx);
  }
  if (get)
    for (int i = 0; i < AIM_FFT_PASSES; ++i) get[i] = fft_kernel_for(ctx, pol, i);
  return AIM_OK;
}

extern "C" int aim_autotune(aim_ctx* ctx, int precision, int nrhs, int reps, int32_t* kernel_out, double* ms_out) {
  if (!ctx || !valid_precision(precision) || nrhs < 1 || nrhs > ctx->max_rhs || reps < 1) {
    set_error("aim_autotune: need a context, a precision, 1 <= nrhs <= max_rhs and reps >= 1");
    return AIM_EINVAL;
  }
  // Keep the caller's profiler state: flush what is pending into its totals,
  // tune with a private set of totals, then put the caller's back.
  AIM_TRY(profile_collect(ctx));
  const bool was_on = ctx->prof.on;
  std::vector<std::string> names = std::move(ctx->prof.names);
  std::vector<double> ms = std::move(ctx->prof.ms);
  std::vector<int64_t> count = std::move(ctx->prof.count);
  ctx->prof.names.clear();
  ctx->prof.ms.clear();
  ctx->prof.count.clear();
  ctx->prof.on = true;
  int32_t saved[AIM_FFT_PASSES];
  const int pol = fft_policy_of(precision);
  for (int i = 0; i < AIM_FFT_PASSES; ++i) saved[i] = ctx->fft_kernel[pol][i];
  const int rc = autotune(ctx, precision, nrhs, reps, kernel_out, ms_out);
  drop_step_graph(ctx);
  if (rc != AIM_OK)
    for (int i = 0; i < AIM_FFT_PASSES; ++i) ctx->fft_kernel[pol][i] = saved[i];
  profile_collect(ctx);
  ctx->prof.on = was_on;
  ctx->prof.names = std::move(names);
  ctx->prof.ms = std::move(ms);
  ctx->prof.count = std::move(count);
  return rc;
}
