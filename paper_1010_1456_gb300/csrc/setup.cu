// Context setup (paper Section 2.2 "matrix fill" for AIM, Section 2.4: O(N)).
//
// Host FP64, multi-threaded:
//   1. RWG functions of the interior edges (sorted by (low, high) vertex;
//      "+" triangle = lower index);
//   2. stencil anchors a = floor(c/h - (M-1)/2) per axis, grid box, padded
//      extents (smallest 2,3,5-smooth L >= 2n-1);
//   3. moment-matching weights in their tensor-product Lagrange form,
//      Lambda^c_m(i,j,k) = int g^c_m l_i(xi) l_j(upsilon) l_k(zeta) dS, with
//      g = f_x, f_y, f_z, div f and a collapsed Gauss-Legendre rule exact for
//      the integrand degree 3M+1 (this solves the moment-matching system:
//      the Lagrange basis reproduces every monomial of per-axis degree <= M);
//   4. near list |c_m - c_n| <= r (cell hashing; d2 = (dx dx + dy dy) + dz dz
//      <= r r in FP64, self pairs included), CSR with sorted columns;
//   5. near entries: symmetrised EFIE Galerkin entry minus the entry's grid
//      approximation, computed per test triangle from triangle-pair blocks;
//   6. node-ordered projection lists (the transpose of the weights).
// Device: uploads, twiddles and the Green's function spectrum (fft.cu).
#include <algorithm>
#include <chrono>
#include <atomic>
#include <cmath>
#include <cstring>
#include <thread>

#include "common.h"
#include "geom.h"

namespace aim {

// ------------------------------------------------------------------ threads
template <typename F> static void parallel_for(int64_t n, F f, int64_t grain = 64) {
  unsigned nt = std::max(1u, std::thread::hardware_concurrency());
  if (n <= grain || nt == 1) {
    for (int64_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<int64_t> next(0);
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nt; ++t)
    th.emplace_back([&]() {
      for (;;) {
        int64_t s = next.fetch_add(grain);
        if (s >= n) break;
        int64_t e = std::min(n, s + grain);
        for (int64_t i = s; i < e; ++i) f(i);
      }
    });
  for (auto& t : th) t.join();
}

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

// near list by cell hashing; rows sorted by column
static void near_list(const Topo& T, double r, std::vector<int32_t>& ptr, std::vector<int32_t>& col) {
  const int N = T.N;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int m = 0; m < N; ++m) {
    const double c[3] = {T.cen[m].x, T.cen[m].y, T.cen[m].z};
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], c[d]);
      hi[d] = std::max(hi[d], c[d]);
    }
  }
  double cs = r;
  for (int d = 0; d < 3; ++d) cs = std::max(cs, (hi[d] - lo[d]) / 256.0);
  if (!(cs > 0.0)) cs = 1.0;
  int nc[3];
  for (int d = 0; d < 3; ++d) nc[d] = (int)((hi[d] - lo[d]) / cs) + 1;
  auto cell_of = [&](const V3& c, int* ci) {
    const double v[3] = {c.x, c.y, c.z};
    for (int d = 0; d < 3; ++d) ci[d] = std::min(nc[d] - 1, std::max(0, (int)((v[d] - lo[d]) / cs)));
  };
  const int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
  std::vector<int32_t> cstart(ncell + 1, 0), items(N);
  std::vector<int64_t> cid(N);
  for (int m = 0; m < N; ++m) {
    int ci[3];
    cell_of(T.cen[m], ci);
    cid[m] = ((int64_t)ci[2] * nc[1] + ci[1]) * nc[0] + ci[0];
    cstart[cid[m] + 1]++;
  }
  for (int64_t i = 0; i < ncell; ++i) cstart[i + 1] += cstart[i];
  {
    std::vector<int32_t> fill(cstart.begin(), cstart.end() - 1);
    for (int m = 0; m < N; ++m) items[fill[cid[m]]++] = m;
  }
  const double r2 = r * r;
  auto visit = [&](int m, auto&& emit) {
    int ci[3];
    cell_of(T.cen[m], ci);
    const int span = (r <= cs) ? 1 : (int)std::ceil(r / cs);
    for (int z = std::max(0, ci[2] - span); z <= std::min(nc[2] - 1, ci[2] + span); ++z)
      for (int y = std::max(0, ci[1] - span); y <= std::min(nc[1] - 1, ci[1] + span); ++y)
        for (int x = std::max(0, ci[0] - span); x <= std::min(nc[0] - 1, ci[0] + span); ++x) {
          int64_t cc = ((int64_t)z * nc[1] + y) * nc[0] + x;
          for (int32_t e = cstart[cc]; e < cstart[cc + 1]; ++e) {
            int n = items[e];
            double dx = T.cen[m].x - T.cen[n].x, dy = T.cen[m].y - T.cen[n].y, dz = T.cen[m].z - T.cen[n].z;
            double d2 = (dx * dx + dy * dy) + dz * dz;
            if (d2 <= r2) emit(n);
          }
        }
  };
  std::vector<int32_t> cnt(N, 0);
  parallel_for(N, [&](int64_t m) {
    int c = 0;
    visit((int)m, [&](int) { ++c; });
    cnt[m] = c;
  });
  ptr.assign(N + 1, 0);
  for (int m = 0; m < N; ++m) ptr[m + 1] = ptr[m] + cnt[m];
  col.resize(ptr[N]);
  parallel_for(N, [&](int64_t m) {
    int32_t* out = &col[ptr[m]];
    int c = 0;
    visit((int)m, [&](int n) { out[c++] = n; });
    std::sort(out, out + c);
  });
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
  if (Nc >= (1LL << 31) || Lprod >= (1LL << 31) || c->L[1] > 900 || c->L[2] > 900 || c->L[0] > 4096) {
    set_error("aim_setup: grid too large (padded " + std::to_string(c->L[0]) + "x" + std::to_string(c->L[1]) + "x" +
              std::to_string(c->L[2]) + "; y and z must be <= 900)");
    return AIM_EINVAL;
  }

  // ---- moment weights (Lagrange form)
  const int nw = (3 * M + 4) / 2;
  const TriRule rw = make_tri_rule(nw);
  c->h_lam.assign((size_t)N * 4 * S, 0.0);
  if (cfie) c->h_lamM.assign((size_t)N * 3 * S, 0.0);
  parallel_for(N, [&](int64_t mi) {
    const int m = (int)mi;
    double* lm = &c->h_lam[(size_t)m * 4 * S];
    double* wm = cfie ? &c->h_lamM[(size_t)m * 3 * S] : nullptr;
    const double ax = c->h_anchor[3 * (size_t)m], ay = c->h_anchor[3 * (size_t)m + 1], az = c->h_anchor[3 * (size_t)m + 2];
    for (int half = 0; half < 2; ++half) {
      const int t = half ? T.tm[m] : T.tp[m];
      const V3 fv = T.vert[half ? T.fm[m] : T.fp[m]];
      const double sg = half ? -1.0 : 1.0, A = T.area[t];
      const V3 r0 = T.vert[T.tri[3 * t]], r1 = T.vert[T.tri[3 * t + 1]], r2 = T.vert[T.tri[3 * t + 2]];
      const double cf = sg * T.len[m] / (2.0 * A), dv = sg * T.len[m] / A;
      for (int q = 0; q < rw.q; ++q) {
        V3 r = tri_point(r0, r1, r2, rw.xi1[q], rw.xi2[q]);
        const double wq = A * rw.w[q];
        const double g[4] = {cf * (r.x - fv.x), cf * (r.y - fv.y), cf * (r.z - fv.z), dv};
        const double xi = (r.x - h * ax) / h, up = (r.y - h * ay) / h, ze = (r.z - h * az) / h;
        double lx[6], ly[6], lz[6];
        for (int i = 0; i < P; ++i) {
          lx[i] = lagrange(M, i, xi);
          ly[i] = lagrange(M, i, up);
          lz[i] = lagrange(M, i, ze);
        }
        for (int kk = 0; kk < P; ++kk)
          for (int j = 0; j < P; ++j)
            for (int i = 0; i < P; ++i) {
              const int s = (kk * P + j) * P + i;
              const double b = wq * lx[i] * ly[j] * lz[kk];
              for (int cc = 0; cc < 4; ++cc) lm[cc * S + s] += b * g[cc];
            }
        if (cfie) {
          // W^c = int f . (n x (grad L_u x e_c)) = int (f . grad L_u) n_c - f_c (n . grad L_u)
          const V3 n = nrm[t];
          double dx[6], dy[6], dz[6];
          for (int i = 0; i < P; ++i) {
            dx[i] = lagrange_d(M, i, xi) / h;
            dy[i] = lagrange_d(M, i, up) / h;
            dz[i] = lagrange_d(M, i, ze) / h;
          }
          const double nn[3] = {n.x, n.y, n.z};
          for (int kk = 0; kk < P; ++kk)
            for (int j = 0; j < P; ++j)
              for (int i = 0; i < P; ++i) {
                const int s = (kk * P + j) * P + i;
                const double gx = dx[i] * ly[j] * lz[kk], gy = lx[i] * dy[j] * lz[kk], gz = lx[i] * ly[j] * dz[kk];
                const double fg = g[0] * gx + g[1] * gy + g[2] * gz, ng = n.x * gx + n.y * gy + n.z * gz;
                for (int cc = 0; cc < 3; ++cc) wm[cc * S + s] += wq * (fg * nn[cc] - g[cc] * ng);
              }
        }
      }
    }
  });

  clk.mark("moment weights");
  // ---- near list
  near_list(T, c->radius, c->h_near_ptr, c->h_near_col);
  clk.mark("near list");
  const int64_t nnz = c->h_near_ptr[N];
  c->nnz = nnz;

  // ---- near entries on the device: triangle pairs touched by a near RWG pair
  const TriRule rt = make_tri_rule(3), rts = make_tri_rule(5), rs = make_tri_rule(4);
  std::vector<int32_t> tptr(T.nt + 1, 0), pQ;
  {
    std::vector<std::vector<int32_t>> qs(T.nt);
    parallel_for(T.nt, [&](int64_t Pi) {
      const int Pt = (int)Pi;
      std::vector<int32_t>& Qs = qs[Pt];
      for (int a = 0; a < 3; ++a) {
        const int m = T.tri_rwg[3 * (size_t)Pt + a];
        if (m < 0) continue;
        for (int32_t e = c->h_near_ptr[m]; e < c->h_near_ptr[m + 1]; ++e) {
          const int n = c->h_near_col[e];
          Qs.push_back(T.tp[n]);
          Qs.push_back(T.tm[n]);
        }
      }
      std::sort(Qs.begin(), Qs.end());
      Qs.erase(std::unique(Qs.begin(), Qs.end()), Qs.end());
    }, 16);
    for (int t = 0; t < T.nt; ++t) tptr[t + 1] = tptr[t] + (int32_t)qs[t].size();
    pQ.resize(tptr[T.nt]);
    for (int t = 0; t < T.nt; ++t) std::copy(qs[t].begin(), qs[t].end(), pQ.begin() + tptr[t]);
  }
  const int64_t npairs = (int64_t)pQ.size();
  if (npairs >= (1LL << 31)) {
    set_error("aim_setup: too many near triangle pairs");
    return AIM_EINVAL;
  }
  std::vector<int32_t> pP(npairs), ids(npairs);
  int64_t nsing = 0;
  {
    std::vector<char> sing(npairs, 0);
    parallel_for(T.nt, [&](int64_t Pi) {
      const int Pt = (int)Pi;
      for (int32_t i = tptr[Pt]; i < tptr[Pt + 1]; ++i) {
        pP[i] = Pt;
        const int Qt = pQ[i];
        bool sg = false;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) sg |= (T.tri[3 * (size_t)Pt + a] == T.tri[3 * (size_t)Qt + b]);
        sing[i] = sg ? 1 : 0;
      }
    }, 64);
    for (int64_t i = 0; i < npairs; ++i)
      if (sing[i]) ids[nsing++] = (int32_t)i;
    int64_t r = nsing;
    for (int64_t i = 0; i < npairs; ++i)
      if (!sing[i]) ids[r++] = (int32_t)i;
  }
  std::vector<int32_t> erow(nnz);
  for (int m = 0; m < N; ++m)
    for (int32_t e = c->h_near_ptr[m]; e < c->h_near_ptr[m + 1]; ++e) erow[e] = m;
  clk.mark("near triangle pairs");

  // G_h on the anchor offsets of near pairs plus the stencil extent
  int dmax = 0;
  for (int m = 0; m < N; ++m)
    for (int32_t e = c->h_near_ptr[m]; e < c->h_near_ptr[m + 1]; ++e) {
      int n = c->h_near_col[e];
      for (int d = 0; d < 3; ++d)
        dmax = std::max(dmax, std::abs(c->h_anchor[3 * (size_t)m + d] - c->h_anchor[3 * (size_t)n + d]));
    }
  const int TE = dmax + M, TW = 2 * TE + 1;
  if ((int64_t)TW * TW * TW > (1LL << 26)) {
    set_error("aim_setup: near radius too large for the grid Green's function table");
    return AIM_EINVAL;
  }
  std::vector<double2> gtab((size_t)TW * TW * TW);
  parallel_for((int64_t)TW * TW * TW, [&](int64_t i) {
    const int ox = (int)(i % TW) - TE, oy = (int)((i / TW) % TW) - TE, oz = (int)(i / ((int64_t)TW * TW)) - TE;
    double re = 0.0, im = 0.0;
    if ((ox | oy | oz) != 0) {  // G_h(0) = 0
      const double r = h * std::sqrt((double)ox * ox + (double)oy * oy + (double)oz * oz);
      const double sc = 1.0 / (4.0 * kPi * r);
      re = std::cos(k * r) * sc;
      im = -std::sin(k * r) * sc;
    }
    gtab[i] = make_double2(re, im);
  });
  {
    std::vector<double> vv(3 * (size_t)T.nv);
    for (int i = 0; i < T.nv; ++i) {
      vv[3 * i] = T.vert[i].x;
      vv[3 * i + 1] = T.vert[i].y;
      vv[3 * i + 2] = T.vert[i].z;
    }
    NearFillArgs A;
    A.N = N; A.nv = T.nv; A.nt = T.nt; A.P = P; A.S = S; A.TE = TE;
    A.nnz = nnz; A.npairs = npairs; A.nsing = nsing; A.ntab = (int64_t)gtab.size();
    A.vert = vv.data(); A.tri = T.tri.data(); A.area = T.area.data();
    A.tp = T.tp.data(); A.tm = T.tm.data(); A.sp = T.sp.data(); A.sm = T.sm.data(); A.len = T.len.data();
    A.tptr = tptr.data(); A.pP = pP.data(); A.pQ = pQ.data(); A.ids = ids.data();
    A.erow = erow.data(); A.ecol = c->h_near_col.data(); A.nptr = c->h_near_ptr.data(); A.anchor = c->h_anchor.data();
    A.lam = c->h_lam.data(); A.gtab = gtab.data();
    A.rule_test = &rt; A.rule_test_sing = &rts; A.rule_src = &rs;
    A.alpha = c->alpha;
    A.lamM = cfie ? c->h_lamM.data() : nullptr;
    c->h_near_val.assign(2 * (size_t)nnz, 0.0);
    c->h_diag.assign(2 * (size_t)N, 0.0);
    AIM_TRY(near_fill_device(c, A, c->h_near_val.data(), c->h_diag.data()));
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
    std::vector<char> used(P, 0);
    if (same)
      for (size_t mc = 0; mc < (size_t)N * 4; ++mc)
        for (int s = 0; s < S; ++s)
          if (c->h_lam[mc * S + s] != 0.0) used[s / (P * P)] = 1;
    int nused = 0, kk0 = 0;
    for (int kk = 0; kk < P; ++kk)
      if (used[kk]) {
        ++nused;
        kk0 = kk;
      }
    if (same && nused == 1) {
      const int S2 = P * P;
      std::vector<double> lam2((size_t)N * 4 * S2);
      for (size_t mc = 0; mc < (size_t)N * 4; ++mc)
        for (int t = 0; t < S2; ++t) lam2[mc * S2 + t] = c->h_lam[mc * S + (size_t)kk0 * S2 + t];
      c->h_lam.swap(lam2);
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

  // ---- projection lists (node-ordered transpose of the weights)
  const int nx = c->n[0], ny = c->n[1];
  std::vector<int32_t> base(N);
  for (int m = 0; m < N; ++m) {
    const int ix = c->h_anchor[3 * (size_t)m] - c->lo[0], iy = c->h_anchor[3 * (size_t)m + 1] - c->lo[1],
              iz = c->h_anchor[3 * (size_t)m + 2] + c->kk0 - c->lo[2];
    base[m] = (int32_t)(((int64_t)iz * ny + iy) * nx + ix);
  }
  std::vector<int32_t> pptr(Nc + 1, 0);
  auto nonzero = [&](int m, int s) {
    const double* lm = &c->h_lam[(size_t)m * 4 * S_run];
    return lm[s] != 0.0 || lm[S_run + s] != 0.0 || lm[2 * S_run + s] != 0.0 || lm[3 * S_run + s] != 0.0;
  };
  auto node_of = [&](int m, int s) {
    const int i = s % P, j = (s / P) % P, kk = s / (P * P);
    return (int64_t)base[m] + ((int64_t)kk * ny + j) * nx + i;
  };
  for (int m = 0; m < N; ++m)
    for (int s = 0; s < S_run; ++s)
      if (nonzero(m, s)) pptr[node_of(m, s) + 1]++;
  for (long long u = 0; u < Nc; ++u) pptr[u + 1] += pptr[u];
  const int64_t nent = pptr[Nc];
  c->nent = nent;
  std::vector<int32_t> pm(nent);
  std::vector<double> pw64(4 * (size_t)nent);
  std::vector<float> pw32(4 * (size_t)nent);
  {
    std::vector<int32_t> fill(pptr.begin(), pptr.end() - 1);
    for (int m = 0; m < N; ++m)
      for (int s = 0; s < S_run; ++s)
        if (nonzero(m, s)) {
          const int64_t e = fill[node_of(m, s)]++;
          pm[e] = m;
          for (int cc = 0; cc < 4; ++cc) {
            pw64[4 * e + cc] = c->h_lam[(size_t)m * 4 * S_run + cc * S_run + s];
            pw32[4 * e + cc] = (float)pw64[4 * e + cc];
          }
        }
  }

  clk.mark("projection lists");
  // ---- uploads
  std::vector<float> lam32(c->h_lam.size());
  for (size_t i = 0; i < lam32.size(); ++i) lam32[i] = (float)c->h_lam[i];
  std::vector<float> nv32(c->h_near_val.size());
  for (size_t i = 0; i < nv32.size(); ++i) nv32[i] = (float)c->h_near_val[i];
  std::vector<double> dinv(2 * (size_t)N);
  for (int m = 0; m < N; ++m) {
    const double a = c->h_diag[2 * (size_t)m], b = c->h_diag[2 * (size_t)m + 1];
    const double d = a * a + b * b;
    dinv[2 * (size_t)m] = a / d;
    dinv[2 * (size_t)m + 1] = -b / d;
  }
  AIM_TRY(up(&c->base, base));
  AIM_TRY(up(&c->near_ptr, c->h_near_ptr));
  AIM_TRY(up(&c->near_col, c->h_near_col));
  AIM_TRY(up(&c->pnode_ptr, pptr));
  c->h_pnode_ptr = pptr;
  // With z passes the projection writes only the 8-node groups that hold
  // entries (most of the box around a closed surface holds none); the rest
  // of grid0 is zeroed once when the grids are allocated.
  c->sparse_proj = c->L[2] > 1;
  if (c->sparse_proj) {
    std::vector<int32_t> grp;
    for (long long g = 0; 8 * g < Nc; ++g)
      if (pptr[std::min(Nc, 8 * g + 8)] > pptr[8 * g]) grp.push_back((int32_t)g);
    c->ngroups = (int64_t)grp.size();
    if (!grp.empty()) AIM_TRY(up(&c->pgroups, grp));
  }
  AIM_TRY(up(&c->pnode_m, pm));
  AIM_TRY(upload((void**)&c->p64.pnode_w, pw64.data(), pw64.size() * sizeof(double)));
  AIM_TRY(upload((void**)&c->p32.pnode_w, pw32.data(), pw32.size() * sizeof(float)));
  AIM_TRY(upload((void**)&c->p64.lam, c->h_lam.data(), c->h_lam.size() * sizeof(double)));
  if (cfie) {
    std::vector<float> lamM32(c->h_lamM.size());
    for (size_t i = 0; i < lamM32.size(); ++i) lamM32[i] = (float)c->h_lamM[i];
    AIM_TRY(upload((void**)&c->p64.lamM, c->h_lamM.data(), c->h_lamM.size() * sizeof(double)));
    AIM_TRY(upload((void**)&c->p32.lamM, lamM32.data(), lamM32.size() * sizeof(float)));
    std::vector<double> nv(3 * (size_t)T.nt);
    for (int t = 0; t < T.nt; ++t) {
      nv[3 * t] = nrm[t].x;
      nv[3 * t + 1] = nrm[t].y;
      nv[3 * t + 2] = nrm[t].z;
    }
    AIM_TRY(up(&c->tri_nrm, nv));
  }
  AIM_TRY(upload((void**)&c->p32.lam, lam32.data(), lam32.size() * sizeof(float)));
  AIM_TRY(upload((void**)&c->p64.near_val, c->h_near_val.data(), c->h_near_val.size() * sizeof(double)));
  AIM_TRY(upload((void**)&c->p32.near_val, nv32.data(), nv32.size() * sizeof(float)));
  AIM_TRY(upload((void**)&c->diag, c->h_diag.data(), c->h_diag.size() * sizeof(double)));
  AIM_TRY(upload((void**)&c->dinv64, dinv.data(), dinv.size() * sizeof(double)));
  // geometry for right-hand sides and far fields
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
  }
  // FFT plans, twiddles and Ghat
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
  clk.mark("uploads");
  AIM_TRY(build_ghat(c));
  c->h_ghat.resize(2 * oct);
  AIM_CUDA_TRY(cudaMemcpyAsync(c->h_ghat.data(), c->p64.ghat, oct * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
  AIM_CUDA_TRY(cudaStreamSynchronize(c->stream));
  clk.mark("Green's function spectrum");
  return AIM_OK;
}

}  // namespace aim
