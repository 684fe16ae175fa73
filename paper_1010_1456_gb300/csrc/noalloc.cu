// Complex64 AIM product that allocates no device memory.
//
// Some callers cannot let a library call cudaMalloc: their device memory is
// owned by another allocator (a framework's caching allocator or a fixed
// memory pool that must account for every byte), or they run a latency-bound
// loop in which an allocation, which can synchronise the device, would stall
// the other streams.  aim_matvec allocates its pass grids on the first
// product of a precision; this variant instead runs the same kernels on
// grids carved from one fixed, file-scope device array.
//
// The array (kNoallocScratchBytes = 64 MiB) is part of the library's device
// image: every GPU that loads the library holds it until the process exits.
// The host-side name of the array is only a stand-in and must never be passed
// to a kernel; its device address is looked up with cudaGetSymbolAddress in
// every call, with the context's device current.  The address belongs to
// the CUDA context it was looked up in, so it is never cached: a caller that
// makes another context current, or a call after cudaDeviceReset, gets the
// address of the array in the context that is current now.  With lazy module
// loading the driver maps the array during the first lookup in a context
// (the set-up of that device); later lookups are host-side and allocate
// nothing.  All calls share the array and it keeps the last call's
// contents; every kernel of the product writes every grid element it later
// reads, so nothing has to start at zero.  Calls whose work overlaps on the
// GPU (different streams, or different contexts at the same time) race on
// the array; callers must order them.
#include <string>

#include "common.h"

namespace aim {

constexpr size_t kNoallocScratchBytes = 64ull << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Device address of the scratch array in the current context, which must be
// the context of device `dev`.
static int noalloc_scratch(int dev, void** out) {
  int cur = -1;
  AIM_CUDA_TRY(cudaGetDevice(&cur));
  if (cur != dev) {
    set_error("aim_matvec_c64_noalloc: the context was built on device " + std::to_string(dev) +
              " but device " + std::to_string(cur) + " is current; make the context's device current first");
    return AIM_EINVAL;
  }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    set_error(std::string("aim_matvec_c64_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
    return AIM_ECUDA;
  }
  *out = p;
  return AIM_OK;
}

static size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace aim

using namespace aim;

extern "C" int aim_matvec_c64_noalloc(aim_ctx* ctx, const void* x_dev, void* y_dev, int nrhs) {
  if (!ctx) {
    set_error("aim_matvec_c64_noalloc: null context");
    return AIM_EINVAL;
  }
  if (nrhs < 1 || nrhs > ctx->max_rhs || !x_dev || !y_dev || x_dev == y_dev) {
    set_error("aim_matvec_c64_noalloc: need 1 <= nrhs <= max_rhs and distinct non-null x, y");
    return AIM_EINVAL;
  }
  const size_t nx = ctx->n[0], ny = ctx->n[1], nz = ctx->n[2], Ly = ctx->L[1], Lz = ctx->L[2];
  const size_t G = 4 * (size_t)nrhs;
  const size_t b0 = round256(sizeof(float2) * G * nz * ny * nx);
  const size_t b1 = round256(sizeof(float2) * G * Lz * ny * nx);
  const size_t b2 = round256(sizeof(float2) * G * Lz * Ly * nx);
  if (b0 + b1 + b2 > kNoallocScratchBytes) {
    set_error("aim_matvec_c64_noalloc: the pass grids need " + std::to_string(b0 + b1 + b2) +
              " bytes, more than the fixed scratch of " + std::to_string(kNoallocScratchBytes) +
              " bytes; use aim_matvec");
    return AIM_EINVAL;
  }
  void* base = nullptr;
  AIM_TRY(noalloc_scratch(ctx->device, &base));
  unsigned char* s = static_cast<unsigned char*>(base);
  float2* g0 = reinterpret_cast<float2*>(s);
  float2* g1 = reinterpret_cast<float2*>(s + b0);
  float2* g2 = reinterpret_cast<float2*>(s + b0 + b1);
  return matvec_c64_bufs(ctx, static_cast<const float2*>(x_dev), static_cast<float2*>(y_dev), nrhs, g0, g1, g2);
}
