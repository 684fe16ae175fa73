// Device setup steps (setup_dev.cu) and the device near fill (nearfill.cu):
// plain device pointers, owned by the caller unless stated.
#pragma once

#include <vector>

#include "common.h"

namespace aim {

struct TriRule;

// Mesh and basis geometry on the device.
struct DevGeom {
  const double* vert = nullptr;   // [nv][3]
  const int32_t* tri = nullptr;   // [nt][3]
  const double* area = nullptr;   // [nt]
  const int32_t* tp = nullptr;    // [N] "+" triangle
  const int32_t* tm = nullptr;    // [N] "-" triangle
  const int32_t* sp = nullptr;    // [N] slot of the free vertex in the "+" triangle
  const int32_t* sm = nullptr;    // [N] slot in the "-" triangle
  const int32_t* fp = nullptr;    // [N] free vertex of the "+" triangle
  const int32_t* fm = nullptr;    // [N] free vertex of the "-" triangle
  const double* len = nullptr;    // [N] edge length
};

// In place exclusive prefix sum of n int32 counts; *total receives their sum.
int scan_exclusive(aim_ctx* c, int32_t* a, long long n, long long* total);
// Sort each segment [ptr[i], ptr[i+1]) of key ascending.
int sort_segments(aim_ctx* c, const int32_t* ptr, long long nseg, int32_t* key);

// Moment weights lam [N][4][S] and, when lamM is set, the MFIE weights
// [N][3][S] (nrm: unit triangle normals [nt][3]); S = (M+1)^3, rule rw.
int weights_device(aim_ctx* c, const DevGeom& g, const int32_t* anchor, const TriRule& rw, double* lam, double* lamM,
                   const double* nrm);

// Near list |c_m - c_n| <= r: CSR (cudaMalloc'ed ptr [N+1], col [nnz]) with
// sorted rows.  cen: device [N][3]; hcen: the same on the host.
int near_list_device(aim_ctx* c, const double* cen, const double* hcen, double r, int32_t** ptr, int32_t** col,
                     long long* nnz);

// Triangle-pair lists of the near fill (cudaMalloc'ed).
struct PairLists {
  int32_t* tptr = nullptr;  // [nt+1] per test triangle, offsets into pQ
  int32_t* pQ = nullptr;    // [npairs] source triangles, sorted within a test triangle
  int32_t* pP = nullptr;    // [npairs] test triangle of each pair
  int32_t* ids = nullptr;   // [npairs] pair indices, the nsing singular ones first
  long long npairs = 0, nsing = 0;
};
int pair_lists_device(aim_ctx* c, const DevGeom& g, const int32_t* tri_rwg, const int32_t* nptr, const int32_t* ncol,
                      long long nnz, PairLists* out);
// erow [nnz] (row of each entry, cudaMalloc'ed) and the largest anchor offset of a near pair.
int erow_and_span_device(aim_ctx* c, const int32_t* nptr, const int32_t* ncol, long long nnz, const int32_t* anchor,
                         int32_t** erow, int* dmax);
// G_h on offsets [-TE, TE]^3 (cudaMalloc'ed).
int gtab_device(aim_ctx* c, int TE, double2** out);

// Stencil planes with a nonzero weight, and the weights of plane kk0 alone.
int planes_used_device(aim_ctx* c, const double* lam, int S, int P, std::vector<int>& used);
int keep_plane_device(aim_ctx* c, const double* lam, int S, int S2, int kk0, double** lam2);

// Node-ordered projection lists (cudaMalloc'ed): base [N] (flat index of the
// stencil's first node), ptr [Nc+1], pm [nent], pw [nent][4] (FP64), and the
// 8-node groups with entries when want_groups is set.
struct ProjLists {
  const int32_t* anchor = nullptr;  // in: [N][3]
  bool want_groups = false;         // in
  int32_t *base = nullptr, *ptr = nullptr, *pm = nullptr, *groups = nullptr;
  double* pw = nullptr;
  long long nent = 0, ngroups = 0;
};
int projection_device(aim_ctx* c, const double* lam, int S, int P, long long Nc, ProjLists* out);
// [n_y][n_x] flags of the grid columns (x, y) that hold a node with projection entries.
int column_mask_device(aim_ctx* c, const int32_t* pnode_ptr, long long Nc, uint8_t** out);

int to_f32_device(aim_ctx* c, const double* in, long long n, float** out);
int inverse_diag_device(aim_ctx* c, const double2* d, double2** out);

// Near fill (nearfill.cu) on device inputs: writes the near values val [nnz]
// and the MoM diagonal diag [N] (device c128).
struct NearFillDev {
  DevGeom g;
  int P = 3, S = 27, TE = 0;
  long long nnz = 0;
  const int32_t *erow = nullptr, *ecol = nullptr, *nptr = nullptr, *anchor = nullptr;
  const double* lam = nullptr;   // [N][4][S] full stencil
  const double* lamM = nullptr;  // [N][3][S] (CFIE only)
  const double2* gtab = nullptr;
  const PairLists* pairs = nullptr;
  const TriRule *rule_test = nullptr, *rule_test_sing = nullptr, *rule_src = nullptr;
  double alpha = 1.0;
};
int near_fill_dev(aim_ctx* c, const NearFillDev& a, double2* val, double2* diag);

}  // namespace aim
