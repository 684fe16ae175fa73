// Launchers of the four-step FFT kernels for one arithmetic policy; each
// fft4_<policy>.cu includes this with AIM_FFT4_POLICY and AIM_FFT4_NAME set,
// so the three policies compile in parallel.
#include <algorithm>

#include "fft4.cuh"

namespace aim {

namespace {
constexpr int kNotHandled = -1;
using Pol = AIM_FFT4_POLICY;
using S = Pol::S;

template <bool INV, int L1, int L2, class O>
int launch_strided4(aim_ctx* c, const char* name, const S* in, O* out, const StridedArgs4& a, int G, const S* tw) {
  constexpr int L = L1 * L2, TX = Pol::kTX;
  // other-axis indices per block: about 256 work units per step, <= 100 KB of shared memory
  int AY = std::max(1, 256 / (TX * std::min(L1, L2)));
  AY = std::min<int>(AY, (int)std::max<long long>(1, (100 * 1024) / (2ll * L * TX * (long long)sizeof(S))));
  AY = std::min(AY, a.A);
  const size_t sm = 2ull * AY * L * TX * sizeof(S);
  static const cudaError_t attr =
      cudaFuncSetAttribute(fft4_strided<Pol, INV, L1, L2, O>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  AIM_CUDA_TRY(attr);
  dim3 grid((a.X + TX - 1) / TX, (a.A + AY - 1) / AY, G);
  AIM_LAUNCH(c, name, (fft4_strided<Pol, INV, L1, L2, O><<<grid, 256, sm, c->stream>>>(in, out, a, tw, AY)));
  return launch_check(c, name);
}

template <int L1, int L2>
int launch_x4(aim_ctx* c, const char* name, S* buf, XArgs4 a, const S* ghat, const S* tw) {
  constexpr int L = L1 * L2;
  // pencils per block: about 256 work units per step, shared memory <= 100 KB
  const long long budget = (100 * 1024) / sizeof(S);
  const int want = std::max(1, 256 / std::min(L1, L2));
  const int npmax = (int)std::max<long long>(1, std::min<long long>(want, (budget - L) / (2 * L)));
  int TG = std::min(a.G, npmax);
  int RY = std::max(1, npmax / TG);
  RY = std::min(RY, a.Ly);
  while (RY > 1 && (long long)(RY * L + 2 * RY * TG * L) > budget) --RY;
  a.RY = RY;
  a.TG = TG;
  const size_t sm = (size_t)(RY * L + 2 * RY * TG * L) * sizeof(S);
  if (sm > 227 * 1024) return kNotHandled;  // leave it to the Stockham kernel
  static const cudaError_t attr =
      cudaFuncSetAttribute(fft4_x<Pol, L1, L2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  AIM_CUDA_TRY(attr);
  dim3 grid((a.Ly + RY - 1) / RY, a.Lz);
  AIM_LAUNCH(c, name, (fft4_x<Pol, L1, L2><<<grid, 256, sm, c->stream>>>(buf, a, ghat, tw)));
  return launch_check(c, name);
}
}  // namespace

// 1: launched; 0: no four-step kernel for this length; < 0: -error code.
int AIM_FFT4_NAME(strided)(aim_ctx* c, const char* name, bool inv, const S* in, S* out, double2* out64,
                           const StridedArgs4& a, int G, int L, const S* tw) {
  int rc = AIM_OK;
  switch (L) {
#define AIM_CASE(LL, A1, A2)                                                                         \
  case LL:                                                                                           \
    if (out64) {                                                                                     \
      if constexpr (std::is_same<S, float4>::value)                                                  \
        rc = launch_strided4<true, A1, A2, double2>(c, name, in, out64, a, G, tw);                   \
      else                                                                                           \
        return 0;                                                                                    \
    } else if (inv) {                                                                                \
      rc = launch_strided4<true, A1, A2, S>(c, name, in, out, a, G, tw);                             \
    } else {                                                                                         \
      rc = launch_strided4<false, A1, A2, S>(c, name, in, out, a, G, tw);                            \
    }                                                                                                \
    return rc == AIM_OK ? 1 : -rc;
    AIM_FOURSTEP_LENGTHS(AIM_CASE)
#undef AIM_CASE
    default: return 0;
  }
}

int AIM_FFT4_NAME(x)(aim_ctx* c, const char* name, S* buf, const XArgs4& a, int L, const S* ghat, const S* tw) {
  int rc = kNotHandled;
  switch (L) {
#define AIM_CASE(LL, A1, A2) \
  case LL: rc = launch_x4<A1, A2>(c, name, buf, a, ghat, tw); break;
    AIM_FOURSTEP_LENGTHS(AIM_CASE)
#undef AIM_CASE
    default: break;
  }
  return rc == kNotHandled ? 0 : rc == AIM_OK ? 1 : -rc;
}

}  // namespace aim
