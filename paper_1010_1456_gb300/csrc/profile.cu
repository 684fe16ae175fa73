// Per-kernel device timing (aim_profile / aim_profile_read): each launch of
// a profiled context is bracketed by two CUDA events recorded on the
// context's stream; totals are accumulated per kernel name when read.
#include <cstring>

#include "common.h"

namespace aim {

static cudaEvent_t take_event(aim_ctx* c) {
  if (!c->prof.pool.empty()) {
    cudaEvent_t e = c->prof.pool.back();
    c->prof.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

LaunchScope::LaunchScope(aim_ctx* ctx, const char* nm) : c(ctx), on(ctx->prof.on), name(nm) {
  c->launches++;
  if (on) {
    b = take_event(c);
    cudaEventRecord(b, c->stream);
  }
}

LaunchScope::~LaunchScope() {
  if (!on) return;
  cudaEvent_t e = take_event(c);
  cudaEventRecord(e, c->stream);
  c->prof.pending.push_back(ProfEvent{name, b, e});
}

int profile_collect(aim_ctx* c) {
  Profiler& p = c->prof;
  if (p.pending.empty()) return AIM_OK;
  AIM_CUDA_TRY(cudaStreamSynchronize(c->stream));
  for (const ProfEvent& ev : p.pending) {
    float ms = 0.f;
    AIM_CUDA_TRY(cudaEventElapsedTime(&ms, ev.a, ev.b));
    size_t i = 0;
    while (i < p.names.size() && p.names[i] != ev.name) ++i;
    if (i == p.names.size()) {
      p.names.push_back(ev.name);
      p.ms.push_back(0.0);
      p.count.push_back(0);
    }
    p.ms[i] += ms;
    p.count[i] += 1;
    p.pool.push_back(ev.a);
    p.pool.push_back(ev.b);
  }
  p.pending.clear();
  return AIM_OK;
}

void profile_free(aim_ctx* c) {
  for (const ProfEvent& ev : c->prof.pending) {
    cudaEventDestroy(ev.a);
    cudaEventDestroy(ev.b);
  }
  for (cudaEvent_t e : c->prof.pool) cudaEventDestroy(e);
  c->prof = Profiler{};
}

}  // namespace aim

using namespace aim;

extern "C" int aim_profile(aim_ctx* ctx, int mode) {
  if (!ctx || mode < 0 || mode > 2) {
    set_error("aim_profile: need a context and mode 0, 1 or 2");
    return AIM_EINVAL;
  }
  if (mode == 2) {
    AIM_TRY(profile_collect(ctx));
    ctx->prof.names.clear();
    ctx->prof.ms.clear();
    ctx->prof.count.clear();
    return AIM_OK;
  }
  ctx->prof.on = mode == 1;
  return AIM_OK;
}

extern "C" int aim_profile_read(aim_ctx* ctx, int max_kernels, char* names, int64_t* launches, double* ms,
                                int* count) {
  if (!ctx || !count || max_kernels < 0 || (max_kernels > 0 && (!names || !launches || !ms))) {
    set_error("aim_profile_read: bad arguments");
    return AIM_EINVAL;
  }
  AIM_TRY(profile_collect(ctx));
  const int n = (int)ctx->prof.names.size();
  *count = n;
  for (int i = 0; i < n && i < max_kernels; ++i) {
    std::strncpy(names + 48 * i, ctx->prof.names[i].c_str(), 47);
    names[48 * i + 47] = 0;
    launches[i] = ctx->prof.count[i];
    ms[i] = ctx->prof.ms[i];
  }
  return AIM_OK;
}
