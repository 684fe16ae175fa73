// Context setup (paper Section 2.2 "matrix fill" for AIM, Section 2.4: O(N)).
//
// Host FP64: the mesh topology (RWG functions of the interior edges, sorted
// by (low, high) vertex; "+" triangle = lower index), triangle normals, the
// stencil anchors a = floor(c/h - (M-1)/2) per axis and the grid extents
// (padded L = smallest 2,3,5-smooth integer >= 2n-1).  Device (setup_dev.cu,
// nearfill.cu), everything that scales with the number of unknowns:
//   1. moment-matching weights in their tensor-product Lagrange form,
//      Lambda^c_m(i,j,k) = int g^c_m l_i(xi) l_j(upsilon) l_k(zeta) dS, with
//      g = f_x, f_y, f_z, div f and a collapsed Gauss-Legendre rule exact for
//      the integrand degree 3M+1 (this solves the moment-matching system:
//      the Lagrange basis reproduces every monomial of per-axis degree <= M);
//   2. near list |c_m - c_n| <= r (cell binning; d2 = (dx dx + dy dy) + dz dz
//      <= r r in FP64, self pairs included), CSR with sorted columns;
//   3. near entries: symmetrised EFIE Galerkin entry minus the entry's grid
//      approximation, from triangle-pair blocks;
//   4. plane collapse and the node-ordered projection lists (the transpose
//      of the weights); FP32 copies.
// Then the twiddles and the Green's function spectrum (fft.cu).  The host
// copies of the setup arrays are made only when aim_export asks for them.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "common.h"
#include "geom.h"
#include "setup_dev.h"

namespace aim {

static int smooth_length(int m) {
  for (int L = std::max(m, 1);; ++L) {
    int x = L;
    for (int p : {2, 3, 5})
      while (x % p == 0) x /= p;
    if (x == 1) return L;
  }
}

// ------------------------------------------------------------------ topology
struct Topo {
  int N = 0, nv = 0, nt = 0;
  std::vector<V3> vert;
  std::vector<int32_t> tri;  // [nt][3]
  std::vector<double> area;  // [nt]
  std::vector<int32_t> e0, e1, tp, tm, fp, fm, sp, sm;
  std::vector<double> len;
  std::vector<V3> cen;
  std::vector<int32_t> tri_rwg;  // [nt][3]: RWG whose free vertex is slot s of the triangle, or -1
};

static int build_topology(const aim_mesh* mesh, Topo& T) {
  if (!mesh || mesh->nv <= 0 || mesh->nt <= 0 || !mesh->verts || !mesh->tris) {
    set_error("aim_setup: empty mesh");
    return AIM_EINVAL;
  }
  T.nv = mesh->nv;
  T.nt = mesh->nt;
  T.vert.resize(T.nv);
  for (int i = 0; i < T.nv; ++i) T.vert[i] = v3(mesh->verts[3 * i], mesh->verts[3 * i + 1], mesh->verts[3 * i + 2]);
  T.tri.assign(mesh->tris, mesh->tris + 3 * (size_t)T.nt);
  T.area.resize(T.nt);
  for (int t = 0; t < T.nt; ++t) {
    int a = T.tri[3 * t], b = T.tri[3 * t + 1], c = T.tri[3 * t + 2];
    if (a < 0 || b < 0 || c < 0 || a >= T.nv || b >= T.nv || c >= T.nv || a == b || b == c || a == c) {
      set_error("aim_setup: triangle " + std::to_string(t) + " has a bad vertex index");
      return AIM_EINVAL;
    }
    V3 cr = cross(T.vert[b] - T.vert[a], T.vert[c] - T.vert[a]);
    T.area[t] = 0.5 * norm(cr);
    if (!(T.area[t] > 0.0)) {
      set_error("aim_setup: triangle " + std::to_string(t) + " is degenerate");
      return AIM_EINVAL;
    }
  }
  struct E {
    int32_t a, b, t, slot;
  };
  std::vector<E> ed;
  ed.reserve(3 * (size_t)T.nt);
  for (int t = 0; t < T.nt; ++t)
    for (int k = 0; k < 3; ++k) {
      int u = T.tri[3 * t + k], v = T.tri[3 * t + (k + 1) % 3];
      ed.push_back(E{std::min(u, v), std::max(u, v), t, (k + 2) % 3});
    }
  std::sort(ed.begin(), ed.end(), [](const E& x, const E& y) {
    if (x.a != y.a) return x.a < y.a;
    if (x.b != y.b) return x.b < y.b;
    return x.t < y.t;
  });
  T.tri_rwg.assign(3 * (size_t)T.nt, -1);
  for (size_t i = 0; i < ed.size();) {
    size_t j = i;
    while (j < ed.size() && ed[j].a == ed[i].a && ed[j].b == ed[i].b) ++j;
    if (j - i > 2) {
      set_error("aim_setup: non-manifold edge (" + std::to_string(ed[i].a) + "," + std::to_string(ed[i].b) + ")");
      return AIM_EINVAL;
    }
    if (j - i == 2) {
      const E& p = ed[i];
      const E& q = ed[i + 1];
      int m = (int)T.e0.size();
      T.e0.push_back(p.a);
      T.e1.push_back(p.b);
      T.tp.push_back(p.t);
      T.tm.push_back(q.t);
      T.sp.push_back(p.slot);
      T.sm.push_back(q.slot);
      T.fp.push_back(T.tri[3 * p.t + p.slot]);
      T.fm.push_back(T.tri[3 * q.t + q.slot]);
      T.tri_rwg[3 * p.t + p.slot] = m;
      T.tri_rwg[3 * q.t + q.slot] = m;
    }
    i = j;
  }
  T.N = (int)T.e0.size();
  if (T.N == 0) {
    set_error("aim_setup: mesh has no interior edges");
    return AIM_EINVAL;
  }
  T.len.resize(T.N);
  T.cen.resize(T.N);
  for (int m = 0; m < T.N; ++m) {
    V3 a = T.vert[T.e0[m]], b = T.vert[T.e1[m]];
    T.len[m] = norm(b - a);
    T.cen[m] = v3((a.x + b.x) * 0.5, (a.y + b.y) * 0.5, (a.z + b.z) * 0.5);
  }
  return AIM_OK;
}

// ------------------------------------------------------------------ setup
static int upload(void** dst, const void* src, size_t bytes) {
  if (bytes == 0) bytes = 16;
  AIM_CUDA_TRY(cudaMalloc(dst, bytes));
  if (src) AIM_CUDA_TRY(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
  return AIM_OK;
}
template <typename T> static int up(T** dst, const std::vector<T>& v) {
  return upload(reinterpret_cast<void**>(dst), v.data(), v.size() * sizeof(T));
}

// Device temporaries of the setup, freed when it returns.
struct DevTemp {
  std::vector<void*> p;
  ~DevTemp() {
    for (void* q : p) cudaFree(q);
  }
  void own(void* q) {
    if (q) p.push_back(q);
  }
  template <typename T> int up(T** dst, const std::vector<T>& v) {
    AIM_TRY(upload(reinterpret_cast<void**>(dst), v.data(), v.size() * sizeof(T)));
    p.push_back(*dst);
    return AIM_OK;
  }
};

int fetch_host_arrays(aim_ctx* c) {
  if (c->host_synced) return AIM_OK;
  const size_t N = (size_t)c->N, nnz = (size_t)c->nnz;
  const long long Nc = (long long)c->n[0] * c->n[1] * c->n[2];
  c->h_lam.resize(N * 4 * c->S);
  c->h_near_ptr.resize(N + 1);
  c->h_near_col.resize(nnz);
  c->h_near_val.resize(2 * nnz);
  c->h_diag.resize(2 * N);
  c->h_pnode_ptr.resize(Nc + 1);
  AIM_CUDA_TRY(cudaMemcpy(c->h_lam.data(), c->p64.lam, c->h_lam.size() * sizeof(double), cudaMemcpyDeviceToHost));
  if (c->p64.lamM) {
    const int P = c->M + 1;
    c->h_lamM.resize(N * 3 * P * P * P);
    AIM_CUDA_TRY(cudaMemcpy(c->h_lamM.data(), c->p64.lamM, c->h_lamM.size() * sizeof(double), cudaMemcpyDeviceToHost));
  }
  AIM_CUDA_TRY(cudaMemcpy(c->h_near_ptr.data(), c->near_ptr, (N + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (nnz) {
    AIM_CUDA_TRY(cudaMemcpy(c->h_near_col.data(), c->near_col, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost));
    AIM_CUDA_TRY(cudaMemcpy(c->h_near_val.data(), c->p64.near_val, nnz * sizeof(double2), cudaMemcpyDeviceToHost));
  }
  AIM_CUDA_TRY(cudaMemcpy(c->h_diag.data(), c->diag, N * sizeof(double2), cudaMemcpyDeviceToHost));
  AIM_CUDA_TRY(cudaMemcpy(c->h_pnode_ptr.data(), c->pnode_ptr, (Nc + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
  c->host_synced = true;
  return AIM_OK;
}

// Wall time of the setup phases, printed to stderr when opts.verbose is set.
struct PhaseClock {
  bool on;
  std::chrono::steady_clock::time_point t0;
  explicit PhaseClock(bool v) : on(v), t0(std::chrono::steady_clock::now()) {}
  void mark(const char* what) {
    if (!on) return;
    const auto t = std::chrono::steady_clock::now();
    std::fprintf(stderr, "aim_setup: %-28s %8.3f s\n", what, std::chrono::duration<double>(t - t0).count());
    t0 = t;
  }
};

// FFT plans (c->plan must hold make_plan of each padded length), the
// twiddle tables of the three arithmetic policies and the storage of the
// Green's function spectrum octants (filled by build_ghat).
int fft_tables(aim_ctx* c) {
  AIM_TRY(upload((void**)&c->plan_dev, c->plan, sizeof(c->plan)));
  for (int d = 0; d < 3; ++d) {
    if (c->plan[d].nst < 0) {
      set_error("aim_setup: padded length is not 2,3,5-smooth");
      return AIM_EINVAL;
    }
    // w^t for t < L, then (four-step lengths) w^(k1 n2) as [k1][n2] and as [n2][k1]
    const int L = c->L[d];
    int L1 = 0, L2 = 0;
    const bool four = fourstep_split(L, &L1, &L2);
    std::vector<double> t64(6 * (size_t)L, 0.0);
    std::vector<float> t32(6 * (size_t)L, 0.f), tff(12 * (size_t)L, 0.f);
    const auto put = [&](size_t slot, long long t) {
      const double ang = (2.0 * kPi * (double)(t % L)) / L;
      t64[2 * slot] = std::cos(ang);
      t64[2 * slot + 1] = -std::sin(ang);
      for (int q = 0; q < 2; ++q) {
        const float hi = (float)t64[2 * slot + q];
        t32[2 * slot + q] = hi;
        tff[4 * slot + 2 * q] = hi;
        tff[4 * slot + 2 * q + 1] = (float)(t64[2 * slot + q] - (double)hi);
      }
    };
    for (int t = 0; t < L; ++t) put(t, t);
    if (four)
      for (int k1 = 0; k1 < L1; ++k1)
        for (int n2 = 0; n2 < L2; ++n2) {
          put((size_t)L + (size_t)k1 * L2 + n2, (long long)k1 * n2);
          put(2 * (size_t)L + (size_t)n2 * L1 + k1, (long long)k1 * n2);
        }
    AIM_TRY(upload((void**)&c->p64.tw[d], t64.data(), t64.size() * sizeof(double)));
    AIM_TRY(upload((void**)&c->p32.tw[d], t32.data(), t32.size() * sizeof(float)));
    AIM_TRY(upload((void**)&c->pff.tw[d], tff.data(), tff.size() * sizeof(float)));
  }
  const size_t oct = (size_t)(c->L[0] / 2 + 1) * (c->L[1] / 2 + 1) * (c->L[2] / 2 + 1);
  AIM_TRY(upload((void**)&c->p64.ghat, nullptr, oct * sizeof(double2)));
  AIM_TRY(upload((void**)&c->p32.ghat, nullptr, oct * sizeof(float2)));
  AIM_TRY(upload((void**)&c->pff.ghat, nullptr, oct * sizeof(float4)));
  return AIM_OK;
}

int build_context(aim_ctx* c, const aim_mesh* mesh) {
  PhaseClock clk(c->opts.verbose != 0);
  Topo T;
  AIM_TRY(build_topology(mesh, T));
  clk.mark("topology");
  const int N = T.N, M = c->M, P = M + 1, S = P * P * P;
  c->N = N;
  c->S = S;
  c->nv = T.nv;
  c->nt = T.nt;
  const double h = c->h, k = c->k;
  c->alpha = c->opts.cfie_alpha;
  const bool cfie = c->alpha < 1.0;
  if (cfie)
    for (int t = 0; t < 3 * T.nt; ++t)
      if (T.tri_rwg[t] < 0) {
        set_error("aim_setup: CFIE (cfie_alpha < 1) needs a closed surface; the mesh has boundary edges");
        return AIM_EINVAL;
      }
  // unit normals (r1 - r0) x (r2 - r0) / |.| (outward for an outward-oriented closed mesh)
  std::vector<V3> nrm(T.nt);
  for (int t = 0; t < T.nt; ++t) {
    const V3 r0 = T.vert[T.tri[3 * t]], r1 = T.vert[T.tri[3 * t + 1]], r2 = T.vert[T.tri[3 * t + 2]];
    const V3 cr = cross(r1 - r0, r2 - r0);
    nrm[t] = (1.0 / norm(cr)) * cr;
  }

  // ---- anchors and grid
  c->h_anchor.resize(3 * (size_t)N);
  int amin[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, amax[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
  for (int m = 0; m < N; ++m) {
    const double cc[3] = {T.cen[m].x, T.cen[m].y, T.cen[m].z};
    for (int d = 0; d < 3; ++d) {
      double t = cc[d] / h;
      double a = std::floor(t - 0.5 * (M - 1));
      if (!(std::fabs(a) < 1e9)) {
        set_error("aim_setup: grid index out of range (check h and the mesh)");
        return AIM_EINVAL;
      }
      int ai = (int)a;
      c->h_anchor[3 * (size_t)m + d] = ai;
      amin[d] = std::min(amin[d], ai);
      amax[d] = std::max(amax[d], ai);
    }
  }
  long long Nc = 1, Lprod = 1;
  for (int d = 0; d < 3; ++d) {
    c->lo[d] = amin[d];
    c->n[d] = amax[d] + M - amin[d] + 1;
    c->L[d] = smooth_length(2 * c->n[d] - 1);
    c->plan[d] = make_plan(c->L[d]);
    Nc *= c->n[d];
    Lprod *= c->L[d];
  }
  // strided (y, z) passes: a four-step length up to 1296, any other 2,3,5-smooth length up to 900 (the
  // Stockham kernel's shared-memory limit)
  int l1 = 0, l2 = 0;
  const auto strided_ok = [&](int L) { return L <= 900 || (L <= 1296 && fourstep_split(L, &l1, &l2)); };
  if (Nc >= (1LL << 31) || Lprod >= (1LL << 31) || !strided_ok(c->L[1]) || !strided_ok(c->L[2]) || c->L[0] > 4096) {
    set_error("aim_setup: grid too large (padded " + std::to_string(c->L[0]) + "x" + std::to_string(c->L[1]) + "x" +
              std::to_string(c->L[2]) + "; y and z must be <= 900, or 1296)");
    return AIM_EINVAL;
  }

  clk.mark("anchors and grid");
  // ---- geometry on the device
  DevTemp tmp;
  int32_t *d_tp = nullptr, *d_tm = nullptr, *d_sp = nullptr, *d_sm = nullptr, *d_fp = nullptr, *d_fm = nullptr;
  int32_t *d_anchor = nullptr, *d_tri_rwg = nullptr;
  double *d_cen = nullptr, *d_nrm = nullptr;
  std::vector<double> hcen(3 * (size_t)N);
  for (int m = 0; m < N; ++m) {
    hcen[3 * (size_t)m] = T.cen[m].x;
    hcen[3 * (size_t)m + 1] = T.cen[m].y;
    hcen[3 * (size_t)m + 2] = T.cen[m].z;
  }
  {
    std::vector<double> vv(3 * (size_t)T.nv);
    for (int i = 0; i < T.nv; ++i) {
      vv[3 * i] = T.vert[i].x;
      vv[3 * i + 1] = T.vert[i].y;
      vv[3 * i + 2] = T.vert[i].z;
    }
    std::vector<int32_t> rt2(2 * (size_t)N), rf2(2 * (size_t)N);
    for (int m = 0; m < N; ++m) {
      rt2[2 * m] = T.tp[m];
      rt2[2 * m + 1] = T.tm[m];
      rf2[2 * m] = T.fp[m];
      rf2[2 * m + 1] = T.fm[m];
    }
    AIM_TRY(up(&c->d_verts, vv));
    AIM_TRY(up(&c->d_tris, T.tri));
    AIM_TRY(up(&c->rwg_tri, rt2));
    AIM_TRY(up(&c->rwg_free, rf2));
    AIM_TRY(up(&c->rwg_len, T.len));
    AIM_TRY(up(&c->tri_area, T.area));
    AIM_TRY(tmp.up(&d_tp, T.tp));
    AIM_TRY(tmp.up(&d_tm, T.tm));
    AIM_TRY(tmp.up(&d_sp, T.sp));
    AIM_TRY(tmp.up(&d_sm, T.sm));
    AIM_TRY(tmp.up(&d_fp, T.fp));
    AIM_TRY(tmp.up(&d_fm, T.fm));
    AIM_TRY(tmp.up(&d_cen, hcen));
    AIM_TRY(tmp.up(&d_anchor, c->h_anchor));
    AIM_TRY(tmp.up(&d_tri_rwg, T.tri_rwg));
    std::vector<double> nv(3 * (size_t)T.nt);
    for (int t = 0; t < T.nt; ++t) {
      nv[3 * t] = nrm[t].x;
      nv[3 * t + 1] = nrm[t].y;
      nv[3 * t + 2] = nrm[t].z;
    }
    if (cfie) {
      AIM_TRY(up(&c->tri_nrm, nv));
      d_nrm = c->tri_nrm;
    }
  }
  DevGeom g;
  g.vert = c->d_verts; g.tri = c->d_tris; g.area = c->tri_area; g.len = c->rwg_len;
  g.tp = d_tp; g.tm = d_tm; g.sp = d_sp; g.sm = d_sm; g.fp = d_fp; g.fm = d_fm;
  clk.mark("uploads");

  // ---- moment weights (Lagrange form), full stencil
  const TriRule rw = make_tri_rule((3 * M + 4) / 2);
  double *lam = nullptr, *lamM = nullptr;
  AIM_CUDA_TRY(cudaMalloc(&lam, sizeof(double) * (size_t)N * 4 * S));
  c->p64.lam = lam;  // owned by the context from here on
  if (cfie) {
    AIM_CUDA_TRY(cudaMalloc(&lamM, sizeof(double) * (size_t)N * 3 * S));
    c->p64.lamM = lamM;
  }
  AIM_TRY(weights_device(c, g, d_anchor, rw, lam, lamM, d_nrm));
  AIM_CUDA_TRY(cudaStreamSynchronize(c->stream));
  clk.mark("moment weights");

  // ---- near list
  long long nnz = 0;
  AIM_TRY(near_list_device(c, d_cen, hcen.data(), c->radius, &c->near_ptr, &c->near_col, &nnz));
  c->nnz = nnz;
  AIM_CUDA_TRY(cudaStreamSynchronize(c->stream));
  clk.mark("near list");

  // ---- near entries: triangle pairs touched by a near RWG pair, G_h table, fill
  PairLists pl;
  AIM_TRY(pair_lists_device(c, g, d_tri_rwg, c->near_ptr, c->near_col, nnz, &pl));
  tmp.own(pl.tptr); tmp.own(pl.pQ); tmp.own(pl.pP); tmp.own(pl.ids);
  int32_t* erow = nullptr;
  int dmax = 0;
  AIM_TRY(erow_and_span_device(c, c->near_ptr, c->near_col, nnz, d_anchor, &erow, &dmax));
  tmp.own(erow);
  clk.mark("near triangle pairs");
  const int TE = dmax + M, TW = 2 * TE + 1;
  if ((int64_t)TW * TW * TW > (1LL << 26)) {
    set_error("aim_setup: near radius too large for the grid Green's function table");
    return AIM_EINVAL;
  }
  double2* gtab = nullptr;
  AIM_TRY(gtab_device(c, TE, &gtab));
  tmp.own(gtab);
  {
    const TriRule rt = make_tri_rule(3), rts = make_tri_rule(5), rs = make_tri_rule(4);
    AIM_CUDA_TRY(cudaMalloc(&c->p64.near_val, sizeof(double2) * std::max<long long>(1, nnz)));
    AIM_CUDA_TRY(cudaMalloc(&c->diag, sizeof(double2) * N));
    NearFillDev A;
    A.g = g; A.P = P; A.S = S; A.TE = TE; A.nnz = nnz;
    A.erow = erow; A.ecol = c->near_col; A.nptr = c->near_ptr; A.anchor = d_anchor;
    A.lam = lam; A.lamM = lamM; A.gtab = gtab; A.pairs = &pl;
    A.rule_test = &rt; A.rule_test_sing = &rts; A.rule_src = &rs;
    A.alpha = c->alpha;
    AIM_TRY(near_fill_dev(c, A, c->p64.near_val, c->diag));
    AIM_CUDA_TRY(cudaStreamSynchronize(c->stream));
  }
  clk.mark("near entries (device)");

  // ---- plane collapse: every weight off one z plane of the grid is zero
  // (a planar scatterer at constant z on a node plane).  Q and Phi vanish off
  // that plane, so the grid keeps only it and the convolution becomes 2-D with
  // G_h(dx, dy, 0); the near entries above used the full stencil and are
  // unchanged.
  int S_run = S;
  if (c->opts.planar && !cfie) {
    bool same = true;
    for (int m = 1; m < N && same; ++m) same = c->h_anchor[3 * (size_t)m + 2] == c->h_anchor[2];
    std::vector<int> used;
    if (same) AIM_TRY(planes_used_device(c, lam, S, P, used));
    int nused = 0, kk0 = 0;
    if (same)
      for (int kk = 0; kk < P; ++kk)
        if (used[kk]) {
          ++nused;
          kk0 = kk;
        }
    if (same && nused == 1) {
      const int S2 = P * P;
      double* lam2 = nullptr;
      AIM_TRY(keep_plane_device(c, lam, S, S2, kk0, &lam2));
      AIM_CUDA_TRY(cudaStreamSynchronize(c->stream));
      cudaFree(lam);
      c->p64.lam = lam = lam2;
      c->planar = 1;
      c->kk0 = kk0;
      c->S = S_run = S2;
      c->lo[2] = c->h_anchor[2] + kk0;
      c->n[2] = 1;
      c->L[2] = 1;
      c->plan[2] = make_plan(1);
      Nc = (long long)c->n[0] * c->n[1];
    }
  }

  // ---- projection lists (node-ordered transpose of the weights).  With z
  // passes the projection writes only the 8-node groups that hold entries
  // (most of the box around a closed surface holds none); the rest of grid0
  // is zeroed once when the grids are allocated.
  c->sparse_proj = c->L[2] > 1;
  {
    ProjLists pj;
    pj.anchor = d_anchor;
    pj.want_groups = c->sparse_proj != 0;
    AIM_TRY(projection_device(c, lam, S_run, P, Nc, &pj));
    c->base = pj.base;
    c->pnode_ptr = pj.ptr;
    c->pnode_m = pj.pm;
    c->p64.pnode_w = pj.pw;
    c->nent = pj.nent;
    c->pgroups = pj.groups;
    c->ngroups = pj.ngroups;
  }
  if (c->L[2] > 1) AIM_TRY(column_mask_device(c, c->pnode_ptr, Nc, &c->colmask));
  clk.mark("projection lists");

  // ---- FP32 copies and the inverse diagonal
  AIM_TRY(to_f32_device(c, lam, (long long)N * 4 * S_run, &c->p32.lam));
  if (cfie) AIM_TRY(to_f32_device(c, lamM, (long long)N * 3 * S, &c->p32.lamM));
  AIM_TRY(to_f32_device(c, reinterpret_cast<const double*>(c->p64.near_val), 2 * nnz,
                        reinterpret_cast<float**>(&c->p32.near_val)));
  AIM_TRY(to_f32_device(c, c->p64.pnode_w, 4 * c->nent, &c->p32.pnode_w));
  AIM_TRY(inverse_diag_device(c, c->diag, &c->dinv64));
  AIM_CUDA_TRY(cudaStreamSynchronize(c->stream));
  clk.mark("conversions");
  // FFT plans, twiddles and Ghat
  AIM_TRY(fft_tables(c));
  clk.mark("twiddles");
  AIM_TRY(build_ghat(c));
  const size_t oct = (size_t)(c->L[0] / 2 + 1) * (c->L[1] / 2 + 1) * (c->L[2] / 2 + 1);
  c->h_ghat.resize(2 * oct);
  AIM_CUDA_TRY(cudaMemcpyAsync(c->h_ghat.data(), c->p64.ghat, oct * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
  AIM_CUDA_TRY(cudaStreamSynchronize(c->stream));
  clk.mark("Green's function spectrum");
  return AIM_OK;
}

}  // namespace aim
