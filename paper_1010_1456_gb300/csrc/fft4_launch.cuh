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

template <bool INV, int L1, int L2, class O, bool WIDE>
int launch_strided4(aim_ctx* c, const char* name, const S* in, O* out, const StridedArgs4& a, int G, const S* tw) {
  constexpr int L = L1 * L2, TX = strided_tx<Pol, L, WIDE>();
  constexpr long long pencil_set = (long long)L * TX * sizeof(S);
  // other-axis indices per block: about 256 work units in the heavier step,
  // one buffer of at most 48 KB (96 KB for the wide variant)
  int AY = std::max(1, 256 / (TX * std::min(L1, L2)));
  AY = std::min<int>(AY, (int)std::max<long long>(1, ((WIDE ? 96 : 48) * 1024) / pencil_set));
  AY = std::min(AY, a.A);
  const int items = AY * TX * std::max(L1, L2);
  const int threads = std::min(256, (items + 31) / 32 * 32);
  const size_t sm = (size_t)AY * pencil_set;
  auto kern = fft4_strided<Pol, INV, L1, L2, O, WIDE>;
  if constexpr (strided_occ4<Pol, L>()) kern = fft4_strided_occ4<Pol, INV, L1, L2, O, WIDE>;
  static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  AIM_CUDA_TRY(attr);
  dim3 grid((a.X + TX - 1) / TX, (a.A + AY - 1) / AY, G);
  AIM_LAUNCH(c, name, (kern<<<grid, threads, sm, c->stream>>>(in, out, a, tw, AY)));
  return launch_check(c, name);
}

// Pencil groups of fft4_x_groups for pencil steps of at most LM threads
// within `threads` threads: the smallest group (1, 2, 4 or 8 warps) whose
// pencils keep at least 90 % of its lanes busy in the wider step, else the
// busiest.
inline void x_groups(int LM, int threads, int* GT, int* PPG) {
  int best_gt = 0, best_ppg = 0;
  double best = -1.0;
  for (int w = 1; 32 * w <= threads; w *= 2) {
    const int gt = 32 * w, ppg = gt / LM;
    if (ppg < 1) continue;
    const double util = (double)(ppg * LM) / gt;
    if (util >= 0.9) {
      best_gt = gt;
      best_ppg = ppg;
      break;
    }
    if (util > best) {
      best = util;
      best_gt = gt;
      best_ppg = ppg;
    }
  }
  *GT = best_gt;
  *PPG = best_ppg;
}

template <int L1, int L2>
int launch_x4_groups(aim_ctx* c, const char* name, S* buf, XArgs4 a, const S* ghat, const S* tw, int threads) {
  constexpr int L = L1 * L2;
  constexpr long long per_pencil = (long long)L1 * odd_row(L2);
  constexpr int LM = std::max(L1, L2);
  int GT = 0, PPG = 0;
  x_groups(LM, threads, &GT, &PPG);
  if (GT == 0) return kNotHandled;  // a pencil wider than the block: the Stockham kernel
  // groups per block: the block's threads, fewer while the tiles and the
  // Ghat rows would not fit in 200 KB; rows per block: as many whole rows
  // (each G pencils) as the groups take at a time, at least one
  const long long cap = (200 * 1024) / sizeof(S);
  int ng = threads / GT;
  int RY = 1;
  for (;;) {
    RY = std::max(1, std::min(ng * PPG / a.G, a.Ly));
    PPG = std::min(PPG, (RY * a.G + ng - 1) / ng);  // no tile beyond the block's pencils
    if (ng == 1 || RY * L + (long long)ng * PPG * per_pencil <= cap) break;
    --ng;
  }
  while (PPG > 1 && RY * L + (long long)ng * PPG * per_pencil > cap) --PPG;
  const size_t sm = (size_t)(RY * L + (long long)ng * PPG * per_pencil) * sizeof(S);
  if (sm > 227 * 1024) return kNotHandled;  // leave it to the Stockham kernel
  a.RY = RY;
  a.GT = GT;
  a.PPG = PPG;
  static const cudaError_t attr =
      cudaFuncSetAttribute(fft4_x_groups<Pol, L1, L2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  AIM_CUDA_TRY(attr);
  dim3 grid((a.Ly + RY - 1) / RY, a.Lz);
  AIM_LAUNCH(c, name, (fft4_x_groups<Pol, L1, L2><<<grid, ng * GT, sm, c->stream>>>(buf, a, ghat, tw)));
  return launch_check(c, name);
}

template <int L1, int L2>
int launch_x4(aim_ctx* c, const char* name, S* buf, XArgs4 a, const S* ghat, const S* tw, int threads, bool warp) {
  if (warp) return launch_x4_groups<L1, L2>(c, name, buf, a, ghat, tw, threads);
  constexpr int L = L1 * L2;
  constexpr long long per_pencil = (long long)L1 * odd_row(L2);
  constexpr int LM = std::max(L1, L2);
  // pencils per block: one work item per thread in each step, shared memory
  // within what one block may hold
  const long long cap = (200 * 1024) / sizeof(S);
  int np = std::max(1, threads / LM);
  while (np > 1 && L + np * per_pencil > cap) --np;
  const int TG = std::min(a.G, np);
  const int RY = std::max(1, std::min(np / TG, a.Ly));
  a.RY = RY;
  a.TG = TG;
  const size_t sm = (size_t)(RY * L + RY * TG * per_pencil) * sizeof(S);
  if (sm > 227 * 1024 || RY * TG * LM > 256) return kNotHandled;  // leave it to the Stockham kernel
  const int nthreads = (RY * TG * LM + 31) / 32 * 32;
  static const cudaError_t attr =
      cudaFuncSetAttribute(fft4_x<Pol, L1, L2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  AIM_CUDA_TRY(attr);
  dim3 grid((a.Ly + RY - 1) / RY, a.Lz);
  AIM_LAUNCH(c, name, (fft4_x<Pol, L1, L2><<<grid, nthreads, sm, c->stream>>>(buf, a, ghat, tw)));
  return launch_check(c, name);
}
}  // namespace

// 1: launched; 0: no four-step kernel for this length; < 0: -error code.
int AIM_FFT4_NAME(strided)(aim_ctx* c, const char* name, bool inv, const S* in, S* out, const StridedArgs4& a, int G,
                           int L, const S* tw, bool wide) {
  int rc = AIM_OK;
  switch (L) {
#define AIM_CASE(LL, A1, A2)                                                                      \
  case LL:                                                                                        \
    rc = wide ? (inv ? launch_strided4<true, A1, A2, S, true>(c, name, in, out, a, G, tw)         \
                     : launch_strided4<false, A1, A2, S, true>(c, name, in, out, a, G, tw))       \
              : (inv ? launch_strided4<true, A1, A2, S, false>(c, name, in, out, a, G, tw)        \
                     : launch_strided4<false, A1, A2, S, false>(c, name, in, out, a, G, tw));     \
    return rc == AIM_OK ? 1 : -rc;
    AIM_FOURSTEP_LENGTHS(AIM_CASE)
#undef AIM_CASE
    default: return 0;
  }
}

int AIM_FFT4_NAME(x)(aim_ctx* c, const char* name, S* buf, const XArgs4& a, int L, const S* ghat, const S* tw,
                     int threads, bool warp) {
  int rc = kNotHandled;
  switch (L) {
#define AIM_CASE(LL, A1, A2) \
  case LL: rc = launch_x4<A1, A2>(c, name, buf, a, ghat, tw, threads, warp); break;
    AIM_FOURSTEP_LENGTHS(AIM_CASE)
#undef AIM_CASE
    default: break;
  }
  return rc == kNotHandled ? 0 : rc == AIM_OK ? 1 : -rc;
}

}  // namespace aim
