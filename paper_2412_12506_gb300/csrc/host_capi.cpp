// Host-setup inspection API (include/ldgmg_host.h): the setup of ldgmg_setup
// without the device upload, so the host logic can be checked on any machine.
#include "ldgmg_host.h"

#include <algorithm>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "host.h"
#include "kernels.h"

using namespace ldgmg;

// shared with capi.cu (thread-local last error)
void ldgmg_set_error(const std::string& msg);

struct ldgmg_host_hier {
  std::vector<HostLevel> lv;
  int smoother = 1;
};

static ldgmg_status herr(ldgmg_status s, const std::string& m) {
  ldgmg_set_error(m);
  return s;
}

extern "C" {

}  // extern "C"

template <class Assemble>
static ldgmg_status host_build(const ldgmg_mesh* mesh, const ldgmg_setup_opts* o, ldgmg_host_hier** out,
                               Assemble assemble) {
  if (!mesh || !o || !out) return herr(LDGMG_EINVAL, "null argument");
  *out = nullptr;
  if (!mesh->periodic) return herr(LDGMG_EUNSUPPORTED, "only periodic meshes are supported");
  auto* h = new ldgmg_host_hier();
  h->smoother = o->smoother;
  h->lv.emplace_back();
  std::string err = assemble(h->lv[0]);
  if (!err.empty()) {
    delete h;
    return herr(LDGMG_EINVAL, err);
  }
  {
    std::vector<HostLevel> coarse;
    err = build_coarse_levels(h->lv[0], coarse);
    if (!err.empty()) {
      delete h;
      return herr(LDGMG_EINVAL, err);
    }
    for (auto& c : coarse) h->lv.push_back(std::move(c));
  }
  SetupParams sp;
  sp.smoother = o->smoother;
  sp.sai_level = o->sai_level;
  sp.balance = o->balance;
  sp.zeta = o->zeta;
  const int nth = int(std::max(1u, std::thread::hardware_concurrency()));
  for (size_t l = 0; l + 1 < h->lv.size(); ++l) {
    err = setup_smoother(h->lv[l], sp, nth);
    if (!err.empty()) {
      delete h;
      return herr(err.find("rank") != std::string::npos ? LDGMG_EUNSUPPORTED : LDGMG_EINVAL, err);
    }
  }
  *out = h;
  return LDGMG_OK;
}

extern "C" {

ldgmg_status ldgmg_host_build(const ldgmg_mesh* mesh, int p, const double* mu, double tau0,
                              const ldgmg_setup_opts* o, ldgmg_host_hier** out) {
  return host_build(mesh, o, out, [&](HostLevel& L) { return assemble_fine(L, mesh->dim, mesh->n, p, mu, tau0); });
}

ldgmg_status ldgmg_host_build_stokes(const ldgmg_mesh* mesh, int p, const double* mu, int gamma, double tau0,
                                     double taup, const ldgmg_setup_opts* o, ldgmg_host_hier** out) {
  return host_build(mesh, o, out, [&](HostLevel& L) {
    return assemble_stokes_fine(L, mesh->dim, mesh->n, p, mu, gamma, tau0, taup);
  });
}

ldgmg_status ldgmg_host_level_info(const ldgmg_host_hier* h, int l, int* nlevels, int* n, int64_t* N,
                                   int* b, int64_t* nnzb_A, int64_t* nnzb_S, int64_t* distinct_A) {
  if (!h) return herr(LDGMG_EINVAL, "null handle");
  if (nlevels) *nlevels = int(h->lv.size());
  if (l < 0 || l >= int(h->lv.size())) return herr(LDGMG_EINVAL, "level out of range");
  const HostLevel& L = h->lv[l];
  const bool bottom = l + 1 == int(h->lv.size());
  if (n) *n = L.n;
  if (N) *N = L.N;
  if (b) *b = L.b;
  if (nnzb_A) *nnzb_A = L.A.nnzb();
  if (nnzb_S) *nnzb_S = bottom ? 0 : (h->smoother == LDGMG_SAI ? L.B.nnzb() : L.N);
  if (distinct_A) *distinct_A = L.A.pool.size();
  return LDGMG_OK;
}

ldgmg_status ldgmg_host_export(const ldgmg_host_hier* h, int l, int which, int64_t* row_ptr, int32_t* col,
                               double* vals) {
  if (!h) return herr(LDGMG_EINVAL, "null handle");
  if (l < 0 || l >= int(h->lv.size())) return herr(LDGMG_EINVAL, "level out of range");
  const HostLevel& L = h->lv[l];
  const bool bottom = l + 1 == int(h->lv.size());
  const int b = L.b;
  const size_t bb = size_t(b) * b;
  if (which == LDGMG_MAT_D) {
    if (bottom || h->smoother == LDGMG_SAI) return herr(LDGMG_EINVAL, "no Jacobi blocks on this level");
    for (int64_t i = 0; i < L.N; ++i) {
      if (row_ptr) row_ptr[i] = i;
      if (col) col[i] = int32_t(i);
      if (vals) std::memcpy(vals + i * bb, L.dinv_pool.get(L.dinv[i]), bb * sizeof(double));
    }
    if (row_ptr) row_ptr[L.N] = L.N;
    return LDGMG_OK;
  }
  const PBSR* M = nullptr;
  if (which == LDGMG_MAT_A) M = &L.A;
  else if ((which == LDGMG_MAT_B || which == LDGMG_MAT_BT) && !bottom && h->smoother == LDGMG_SAI)
    M = which == LDGMG_MAT_B ? &L.B : &L.BT;
  if (!M) return herr(LDGMG_EINVAL, "matrix not present on this level");
  if (row_ptr) std::copy(M->row_ptr.begin(), M->row_ptr.end(), row_ptr);
  if (col) std::copy(M->col.begin(), M->col.end(), col);
  if (vals)
    for (int64_t z = 0; z < M->nnzb(); ++z) std::memcpy(vals + z * bb, M->pool.get(M->id[z]), bb * sizeof(double));
  return LDGMG_OK;
}

ldgmg_status ldgmg_host_tc_plan(int n, const int64_t* row_ptr, const int32_t* col, int rcap, int prec, int ctas,
                                int strip, int* info, int64_t* nloads, int32_t* rec, int32_t* seg,
                                int32_t* ld_elem) {
  if (n < 1 || !row_ptr || !col || !info || !nloads) return herr(LDGMG_EINVAL, "null argument or bad size");
  if (prec != LDGMG_FP32 && prec != LDGMG_BF16) return herr(LDGMG_EINVAL, "prec must be FP32 or BF16");
  TcSchedHost H;
  const std::string why = tc_sched_plan(2, n, int64_t(n) * n, row_ptr, col, rcap, prec, ctas, strip, &H);
  if (!why.empty()) return herr(LDGMG_EUNSUPPORTED, why);
  info[0] = H.G;
  info[1] = H.S;
  info[2] = H.L;
  info[3] = H.kmax;
  *nloads = H.nloads;
  if (rec) std::memcpy(rec, H.rec.data(), H.rec.size());
  if (seg) std::copy(H.seg.begin(), H.seg.end(), seg);
  if (ld_elem) std::copy(H.ld_elem.begin(), H.ld_elem.begin() + H.nloads, ld_elem);
  return LDGMG_OK;
}

ldgmg_status ldgmg_host_colours(const ldgmg_host_hier* h, int l, int* colour, int* ncolours) {
  if (!h) return herr(LDGMG_EINVAL, "null handle");
  if (l < 0 || l + 1 >= int(h->lv.size())) return herr(LDGMG_EINVAL, "level out of range or bottom level");
  const HostLevel& L = h->lv[l];
  if (h->smoother != LDGMG_GS || L.colour_ptr.empty()) return herr(LDGMG_EINVAL, "not a Gauss-Seidel hierarchy");
  const int nc = int(L.colour_ptr.size()) - 1;
  if (ncolours) *ncolours = nc;
  if (colour)
    for (int c = 0; c < nc; ++c)
      for (int64_t k = L.colour_ptr[c]; k < L.colour_ptr[c + 1]; ++k) colour[L.colour_rows[k]] = c;
  return LDGMG_OK;
}

void ldgmg_host_free(ldgmg_host_hier* h) { delete h; }

}  // extern "C"
