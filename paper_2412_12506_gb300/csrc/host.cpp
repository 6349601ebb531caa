// Host-side setup of the LDG multigrid hierarchy.  See host.h for the pooled
// storage scheme.  Paper references: Sec. 2.1 (LDG operator), Sec. 2.2
// (hierarchy, injection, operator coarsening), Sec. 2.3.1 (block Jacobi,
// Eq. Jsmooth), Sec. 2.3.3 (balanced block SAI).
#include "host.h"

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <thread>

namespace ldgmg {

// --------------------------------------------------------------------------
// small utilities
// --------------------------------------------------------------------------

static uint64_t mix64(uint64_t h, uint64_t v) {
  h ^= v + 0x9e3779b97f4a7c15ULL + (h << 6) + (h >> 2);
  h *= 0xff51afd7ed558ccdULL;
  return h ^ (h >> 33);
}

struct VecHash {
  size_t operator()(const std::vector<uint64_t>& v) const {
    uint64_t h = 0x12345678abcdefULL ^ v.size();
    for (uint64_t x : v) h = mix64(h, x);
    return size_t(h);
  }
};
using Memo = std::unordered_map<std::vector<uint64_t>, uint32_t, VecHash>;

static uint64_t dbits(double x) {
  uint64_t u;
  std::memcpy(&u, &x, 8);
  return u;
}

uint32_t Pool::intern(const double* blk) {
  const size_t bb = size_t(b) * b;
  uint64_t h = 0xcbf29ce484222325ULL;
  for (size_t i = 0; i < bb; ++i) h = mix64(h, dbits(blk[i]));
  auto& cands = index[h];
  for (uint32_t id : cands)
    if (std::memcmp(get(id), blk, bb * sizeof(double)) == 0) return id;
  uint32_t id = size();
  data.insert(data.end(), blk, blk + bb);
  cands.push_back(id);
  return id;
}

uint32_t PBSR::find(int64_t r, int32_t c) const {
  auto b0 = col.begin() + row_ptr[r], b1 = col.begin() + row_ptr[r + 1];
  auto it = std::lower_bound(b0, b1, c);
  if (it == b1 || *it != c) return UINT32_MAX;
  return id[size_t(it - col.begin())];
}

// C = A * B (row-major b x b)
static void mm(const double* A, const double* B, double* C, int b) {
  for (int i = 0; i < b; ++i) {
    double* ci = C + size_t(i) * b;
    for (int j = 0; j < b; ++j) ci[j] = 0.0;
    for (int k = 0; k < b; ++k) {
      const double a = A[size_t(i) * b + k];
      if (a == 0.0) continue;
      const double* bk = B + size_t(k) * b;
      for (int j = 0; j < b; ++j) ci[j] += a * bk[j];
    }
  }
}

// C += A^T * B
static void mtm_acc(const double* A, const double* B, double* C, int b) {
  for (int k = 0; k < b; ++k) {
    const double* ak = A + size_t(k) * b;
    const double* bk = B + size_t(k) * b;
    for (int i = 0; i < b; ++i) {
      const double a = ak[i];
      if (a == 0.0) continue;
      double* ci = C + size_t(i) * b;
      for (int j = 0; j < b; ++j) ci[j] += a * bk[j];
    }
  }
}

static int ipow(int a, int e) {
  int r = 1;
  while (e--) r *= a;
  return r;
}

// --------------------------------------------------------------------------
// 1D basis: orthonormal Legendre phi_k = sqrt((2k+1)/2) P_k on [-1, 1]
// --------------------------------------------------------------------------

// Legendre P_0..P_m at x by the three-term recurrence.
static void legendre_all(int m, double x, double* P) {
  P[0] = 1.0;
  if (m >= 1) P[1] = x;
  for (int k = 1; k < m; ++k) P[k + 1] = ((2.0 * k + 1.0) * x * P[k] - k * P[k - 1]) / (k + 1.0);
}

// Gauss-Legendre rule with q points: Newton's method on P_q from the
// asymptotic initial guesses cos(pi (i + 3/4) / (q + 1/2)).
static void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w) {
  x.resize(q);
  w.resize(q);
  std::vector<double> P(q + 1);
  for (int i = 0; i < q; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (q + 0.5));
    for (int it = 0; it < 100; ++it) {
      legendre_all(q, z, P.data());
      double dp = q * (z * P[q] - P[q - 1]) / (z * z - 1.0);
      double dz = P[q] / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    legendre_all(q, z, P.data());
    double dp = q * (z * P[q] - P[q - 1]) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

static void phi_all(int p, double x, double* out) {
  std::vector<double> P(p + 1);
  legendre_all(p, x, P.data());
  for (int k = 0; k <= p; ++k) out[k] = std::sqrt((2.0 * k + 1.0) / 2.0) * P[k];
}

Basis1D make_basis(int p) {
  Basis1D B;
  B.p = p;
  const int q = B.q = p + 1;
  B.K.assign(q * q, 0.0);
  // int phi_i phi_j' = sqrt((2i+1)(2j+1)) for j > i with j - i odd (derivative
  // of P_j expands in P_k, k < j, k = j-1, j-3, ..., with weight 2k+1).
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j)
      if (j > i && ((j - i) & 1)) B.K[i * q + j] = std::sqrt((2.0 * i + 1.0) * (2.0 * j + 1.0));
  B.lo.resize(q);
  B.hi.resize(q);
  for (int k = 0; k < q; ++k) {
    B.hi[k] = std::sqrt((2.0 * k + 1.0) / 2.0);
    B.lo[k] = (k & 1) ? -B.hi[k] : B.hi[k];
  }
  // child injection by Gauss quadrature (integrand of degree 2p)
  std::vector<double> xg, wg;
  gauss_legendre(p + 2, xg, wg);
  std::vector<double> fa(q), fc(q);
  for (int s = 0; s < 2; ++s) {
    B.P[s].assign(q * q, 0.0);
    for (size_t g = 0; g < xg.size(); ++g) {
      phi_all(p, xg[g], fa.data());
      phi_all(p, (xg[g] + 2.0 * s - 1.0) / 2.0, fc.data());
      for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) B.P[s][i * q + j] += wg[g] * fa[i] * fc[j];
    }
  }
  return B;
}

// 1D matrix M1 (q x q) along axis a, identity along the others (mode index
// kx + q ky + q^2 kz).
static std::vector<double> axis_op(const std::vector<double>& M1, int a, int d, int q) {
  const int b = ipow(q, d);
  std::vector<double> out(size_t(b) * b, 0.0);
  int kr[3], kc[3];
  for (int r = 0; r < b; ++r) {
    for (int t = 0, v = r; t < d; ++t, v /= q) kr[t] = v % q;
    for (int c = 0; c < b; ++c) {
      for (int t = 0, v = c; t < d; ++t, v /= q) kc[t] = v % q;
      bool same = true;
      for (int t = 0; t < d; ++t)
        if (t != a && kr[t] != kc[t]) same = false;
      if (same) out[size_t(r) * b + c] = M1[kr[a] * q + kc[a]];
    }
  }
  return out;
}

static std::vector<double> outer(const std::vector<double>& u, const std::vector<double>& v) {
  const int q = int(u.size());
  std::vector<double> o(q * q);
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j) o[i * q + j] = u[i] * v[j];
  return o;
}

// Injection block of child offset s (bit a of sidx = s_a): kron of P[s_a].
static std::vector<double> child_block(const Basis1D& B, int sidx, int d) {
  const int q = B.q, b = ipow(q, d);
  std::vector<double> out(size_t(b) * b);
  int kr[3], kc[3];
  for (int r = 0; r < b; ++r) {
    for (int t = 0, v = r; t < d; ++t, v /= q) kr[t] = v % q;
    for (int c = 0; c < b; ++c) {
      for (int t = 0, v = c; t < d; ++t, v /= q) kc[t] = v % q;
      double prod = 1.0;
      for (int t = 0; t < d; ++t) prod *= B.P[(sidx >> t) & 1][kr[t] * q + kc[t]];
      out[size_t(r) * b + c] = prod;
    }
  }
  return out;
}

// --------------------------------------------------------------------------
// mesh helpers (uniform periodic)
// --------------------------------------------------------------------------

struct Grid {
  int d, n;
  int64_t N;
  void coords(int64_t e, int* c) const {
    for (int t = 0; t < d; ++t) {
      c[t] = int(e % n);
      e /= n;
    }
  }
  int64_t index(const int* c) const {
    int64_t e = 0;
    for (int t = d - 1; t >= 0; --t) e = e * n + ((c[t] % n) + n) % n;
    return e;
  }
  int64_t shift(int64_t e, int a, int delta) const {
    int c[3];
    coords(e, c);
    c[a] += delta;
    return index(c);
  }
};

// Build a PBSR from per-row (col, id) lists; entries of a row must have distinct cols.
static void finish_rows(PBSR& M, std::vector<std::vector<std::pair<int32_t, uint32_t>>>& rows) {
  M.nrows = int64_t(rows.size());
  M.row_ptr.assign(rows.size() + 1, 0);
  M.col.clear();
  M.id.clear();
  for (size_t r = 0; r < rows.size(); ++r) {
    auto& v = rows[r];
    std::sort(v.begin(), v.end());
    for (auto& e : v) {
      M.col.push_back(e.first);
      M.id.push_back(e.second);
    }
    M.row_ptr[r + 1] = int64_t(M.col.size());
  }
}

// --------------------------------------------------------------------------
// Products of the scalar pieces (Sec. 2.1): block (i, j) of
//   sum over (l, r) in `pairs` of G_l^T M_mu G_r   (+ E when add_E)
// The scalar operator is A = sum_a G_a^T M_mu G_a + E (pairs (a, a)); the
// stress-form coupling of Sec. 3.1 uses single pairs (g, f).  Terms of a
// block are summed in a fixed order (column, pair, ...), E last.
// --------------------------------------------------------------------------

static void build_products(const HostLevel& L, const std::vector<std::pair<int, int>>& pairs, bool add_E,
                           PBSR& out) {
  const int b = L.bs;
  const int64_t N = L.N;
  const size_t bb = size_t(b) * b;
  // transposed structure of each G_a: for column i, the (row k, id) entries
  std::vector<std::vector<std::pair<int32_t, uint32_t>>> Gt[3];
  for (int a = 0; a < L.dim; ++a) {
    Gt[a].assign(N, {});
    const PBSR& G = L.G[a];
    for (int64_t k = 0; k < N; ++k)
      for (int64_t z = G.row_ptr[k]; z < G.row_ptr[k + 1]; ++z) Gt[a][G.col[z]].push_back({int32_t(k), G.id[z]});
  }
  out = PBSR();
  out.pool.b = b;
  Memo memo;
  std::vector<std::vector<std::pair<int32_t, uint32_t>>> rows(N);
  std::vector<std::pair<int32_t, std::array<uint32_t, 4>>> terms;
  std::vector<double> acc(bb), tmp(bb);
  for (int64_t i = 0; i < N; ++i) {
    terms.clear();
    for (size_t pi = 0; pi < pairs.size(); ++pi) {
      const PBSR& Gl = L.G[pairs[pi].first];
      const PBSR& Gr = L.G[pairs[pi].second];
      (void)Gl;
      for (auto& ki : Gt[pairs[pi].first][i]) {
        const int32_t k = ki.first;
        const uint32_t m = L.mmu[k];
        for (int64_t z = Gr.row_ptr[k]; z < Gr.row_ptr[k + 1]; ++z)
          terms.push_back({Gr.col[z], {uint32_t(pi), ki.second, m, Gr.id[z]}});
      }
    }
    if (add_E)
      for (int64_t z = L.E.row_ptr[i]; z < L.E.row_ptr[i + 1]; ++z)
        terms.push_back({L.E.col[z], {0xFFFFu, L.E.id[z], 0u, 0u}});
    std::sort(terms.begin(), terms.end());
    size_t s = 0;
    while (s < terms.size()) {
      size_t e = s;
      std::vector<uint64_t> key;
      while (e < terms.size() && terms[e].first == terms[s].first) {
        const auto& t = terms[e].second;
        const uint32_t tag = t[0] == 0xFFFFu ? 0xFFFFu
                                             : uint32_t(pairs[t[0]].first * 4 + pairs[t[0]].second);
        key.push_back((uint64_t(tag) << 32) | t[1]);
        key.push_back((uint64_t(t[2]) << 32) | t[3]);
        ++e;
      }
      auto it = memo.find(key);
      uint32_t id;
      if (it != memo.end()) {
        id = it->second;
      } else {
        std::fill(acc.begin(), acc.end(), 0.0);
        for (size_t u = s; u < e; ++u) {
          const auto& t = terms[u].second;
          if (t[0] == 0xFFFFu) {
            const double* Eb = L.E.pool.get(t[1]);
            for (size_t x = 0; x < bb; ++x) acc[x] += Eb[x];
          } else {
            const PBSR& Gl = L.G[pairs[t[0]].first];
            const PBSR& Gr = L.G[pairs[t[0]].second];
            mm(L.mmu_pool.get(t[2]), Gr.pool.get(t[3]), tmp.data(), b);
            mtm_acc(Gl.pool.get(t[1]), tmp.data(), acc.data(), b);
          }
        }
        id = out.pool.intern(acc.data());
        memo.emplace(std::move(key), id);
      }
      rows[i].push_back({terms[s].first, id});
      s = e;
    }
  }
  finish_rows(out, rows);
}

static void build_A(HostLevel& L) {
  std::vector<std::pair<int, int>> pairs;
  for (int a = 0; a < L.dim; ++a) pairs.push_back({a, a});
  build_products(L, pairs, true, L.A);
}

// --------------------------------------------------------------------------
// Stokes saddle-point operator (Sec. 3.1, Eq. components), field order
// (u_1, .., u_d, p) inside each block of size (d + 1) bs:
//   (u_f, u_g): delta_fg (sum_a G_a^T M_mu G_a + E) + gamma G_g^T M_mu G_f
//   (u_f, p):   -G_f^T M        (p, u_g): -M G_g        (p, p): -E_p
// M = (h/2)^d I is the unweighted mass of the orthonormal modal basis.
// --------------------------------------------------------------------------

static void build_A_stokes(HostLevel& L) {
  const int d = L.dim, bs = L.bs, nf = d + 1, b = nf * bs;
  const int64_t N = L.N;
  const double m = std::pow(L.h / 2.0, d);
  PBSR lap;
  {
    std::vector<std::pair<int, int>> pairs;
    for (int a = 0; a < d; ++a) pairs.push_back({a, a});
    build_products(L, pairs, true, lap);
  }
  PBSR X[3][3];  // X[f][g] = G_g^T M_mu G_f (test field f, trial field g)
  if (L.gamma)
    for (int f = 0; f < d; ++f)
      for (int g = 0; g < d; ++g) build_products(L, {{g, f}}, false, X[f][g]);
  // transposed pattern of each G_f: rows j with G_f(j, i) stored, per column i
  std::vector<std::vector<int32_t>> Gtc[3];
  for (int a = 0; a < d; ++a) {
    Gtc[a].assign(N, {});
    for (int64_t k = 0; k < N; ++k)
      for (int64_t z = L.G[a].row_ptr[k]; z < L.G[a].row_ptr[k + 1]; ++z) Gtc[a][L.G[a].col[z]].push_back(int32_t(k));
  }
  L.A = PBSR();
  L.A.pool.b = b;
  Memo memo;
  std::vector<std::vector<std::pair<int32_t, uint32_t>>> rows(N);
  std::vector<double> blk(size_t(b) * b);
  std::vector<int32_t> cols;
  for (int64_t i = 0; i < N; ++i) {
    cols.clear();
    auto add_row = [&](const PBSR& M) {
      for (int64_t z = M.row_ptr[i]; z < M.row_ptr[i + 1]; ++z) cols.push_back(M.col[z]);
    };
    add_row(lap);
    add_row(L.Ep);
    for (int a = 0; a < d; ++a) {
      add_row(L.G[a]);
      for (int32_t j : Gtc[a][i]) cols.push_back(j);
      if (L.gamma)
        for (int g = 0; g < d; ++g) add_row(X[a][g]);
    }
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
    for (int32_t j : cols) {
      std::vector<uint64_t> key;
      key.push_back(lap.find(i, j));
      key.push_back(L.Ep.find(i, j));
      for (int a = 0; a < d; ++a) {
        key.push_back(L.G[a].find(j, int32_t(i)));   // G_a(j, i), for -G_a^T M
        key.push_back(L.G[a].find(i, j));            // G_a(i, j), for -M G_a
        if (L.gamma)
          for (int g = 0; g < d; ++g) key.push_back(X[a][g].find(i, j));
      }
      auto it = memo.find(key);
      if (it == memo.end()) {
        std::fill(blk.begin(), blk.end(), 0.0);
        auto put = [&](int f, int g, const double* src, double s, bool transpose) {
          for (int r = 0; r < bs; ++r)
            for (int c = 0; c < bs; ++c)
              blk[size_t(f * bs + r) * b + g * bs + c] += s * (transpose ? src[size_t(c) * bs + r] : src[size_t(r) * bs + c]);
        };
        size_t u = 0;
        const uint32_t lid = uint32_t(key[u++]), eid = uint32_t(key[u++]);
        if (lid != UINT32_MAX)
          for (int f = 0; f < d; ++f) put(f, f, lap.pool.get(lid), 1.0, false);
        if (eid != UINT32_MAX) put(d, d, L.Ep.pool.get(eid), -1.0, false);
        for (int a = 0; a < d; ++a) {
          const uint32_t gt = uint32_t(key[u++]), gi = uint32_t(key[u++]);
          if (gt != UINT32_MAX) put(a, d, L.G[a].pool.get(gt), -m, true);
          if (gi != UINT32_MAX) put(d, a, L.G[a].pool.get(gi), -m, false);
          if (L.gamma)
            for (int g = 0; g < d; ++g) {
              const uint32_t xid = uint32_t(key[u++]);
              if (xid != UINT32_MAX) put(a, g, X[a][g].pool.get(xid), 1.0, false);
            }
        }
        it = memo.emplace(key, L.A.pool.intern(blk.data())).first;
      }
      rows[i].push_back({j, it->second});
    }
  }
  finish_rows(L.A, rows);
}

// Interior-penalty operator sum_faces c_f int_f [u][v] on the periodic grid
// (Sec. 2.1); coef(x, e) is the face coefficient between element e and its
// neighbour x, including the face Jacobian.
template <class Coef>
static void build_penalty(PBSR& out, const Grid& g, const Basis1D& B, int dim, int b, Coef coef) {
  const int q = B.q;
  const size_t bb = size_t(b) * b;
  {
    std::vector<std::vector<double>> lolo(dim), lohi(dim), hihi(dim), hilo(dim);
    for (int a = 0; a < dim; ++a) {
      lolo[a] = axis_op(outer(B.lo, B.lo), a, dim, q);
      lohi[a] = axis_op(outer(B.lo, B.hi), a, dim, q);
      hihi[a] = axis_op(outer(B.hi, B.hi), a, dim, q);
      hilo[a] = axis_op(outer(B.hi, B.lo), a, dim, q);
    }
    out = PBSR();
    out.pool.b = b;
    std::vector<std::vector<std::pair<int32_t, uint32_t>>> rows(g.N);
    Memo memo;  // key: per axis (flags, c_lo, c_up) -> encoded in a list of (col-role, id)
    std::unordered_map<std::vector<uint64_t>, std::vector<std::pair<int, uint32_t>>, VecHash> rmemo;
    for (int64_t e = 0; e < g.N; ++e) {
      int64_t nb[3][2];
      std::vector<uint64_t> key;
      double clo[3], cup[3];
      for (int a = 0; a < dim; ++a) {
        nb[a][0] = g.shift(e, a, -1);
        nb[a][1] = g.shift(e, a, +1);
        clo[a] = coef(nb[a][0], e);
        cup[a] = coef(nb[a][1], e);
        key.push_back(uint64_t(nb[a][0] == e) | (uint64_t(nb[a][1] == e) << 1) |
                      (uint64_t(nb[a][0] == nb[a][1]) << 2));
        key.push_back(dbits(clo[a]));
        key.push_back(dbits(cup[a]));
      }
      auto it = rmemo.find(key);
      if (it == rmemo.end()) {
        // distinct neighbour roles: 0 self, 1 + 2a lower of axis a, 2 + 2a upper
        std::map<int, std::vector<double>> blk;
        auto add = [&](int role, const std::vector<double>& M, double c) {
          auto& v = blk[role];
          if (v.empty()) v.assign(bb, 0.0);
          for (size_t x = 0; x < bb; ++x) v[x] += c * M[x];
        };
        for (int a = 0; a < dim; ++a) {
          const int rl = (nb[a][0] == e) ? 0 : 1 + 2 * a;
          const int ru = (nb[a][1] == e) ? 0 : ((nb[a][1] == nb[a][0]) ? rl : 2 + 2 * a);
          add(0, lolo[a], clo[a]);   // face (Lo, e): e is the upper element
          add(rl, lohi[a], -clo[a]);
          add(0, hihi[a], cup[a]);   // face (e, Up): e is the lower element
          add(ru, hilo[a], -cup[a]);
        }
        std::vector<std::pair<int, uint32_t>> lst;
        for (auto& kv : blk) lst.push_back({kv.first, out.pool.intern(kv.second.data())});
        it = rmemo.emplace(key, lst).first;
      }
      for (auto& r : it->second) {
        int64_t c = e;
        if (r.first > 0) {
          const int a = (r.first - 1) / 2;
          c = nb[a][(r.first - 1) % 2];
        }
        rows[e].push_back({int32_t(c), r.second});
      }
    }
    finish_rows(out, rows);
  }
}

// --------------------------------------------------------------------------
// Fine-level assembly (Sec. 2.1)
// --------------------------------------------------------------------------

std::string assemble_fine(HostLevel& L, int dim, int n, int p, const double* mu_in, double tau0) {
  if (dim != 2 && dim != 3) return "dim must be 2 or 3";
  if (n < 1) return "n must be >= 1";
  if (p < 1 || p > 5) return "p must be in 1..5";
  if (!(tau0 > 0.0) || !std::isfinite(tau0)) return "tau0 must be positive and finite";
  const Basis1D B = make_basis(p);
  const int q = B.q, b = ipow(q, dim);
  Grid g{dim, n, 1};
  for (int t = 0; t < dim; ++t) g.N *= n;
  L.dim = dim;
  L.n = n;
  L.p = p;
  L.b = b;
  L.bs = b;
  L.nf = 1;
  L.gamma = 0;
  L.N = g.N;
  L.h = 1.0 / n;
  const double h = L.h;
  std::vector<double> mu(g.N, 1.0);
  if (mu_in)
    for (int64_t e = 0; e < g.N; ++e) {
      if (!(mu_in[e] > 0.0) || !std::isfinite(mu_in[e])) return "mu must be positive and finite";
      mu[e] = mu_in[e];
    }
  const size_t bb = size_t(b) * b;
  const double sG = 2.0 / h;                     // M_E^{-1} times the face/volume Jacobians
  const double wface = std::pow(h / 2.0, dim - 1);

  // --- discrete gradient G_a: strong lifting form with one-sided fluxes ---
  for (int a = 0; a < dim; ++a) {
    const auto vol = axis_op(B.K, a, dim, q);
    const auto lolo = axis_op(outer(B.lo, B.lo), a, dim, q);
    const auto lohi = axis_op(outer(B.lo, B.hi), a, dim, q);
    const auto hihi = axis_op(outer(B.hi, B.hi), a, dim, q);
    const auto hilo = axis_op(outer(B.hi, B.lo), a, dim, q);
    PBSR& G = L.G[a];
    G = PBSR();
    G.pool.b = b;
    std::vector<std::vector<std::pair<int32_t, uint32_t>>> rows(g.N);
    // local configuration -> (role, id) list; roles: 0 self, 1 lower, 2 upper
    std::map<int, std::vector<std::pair<int, uint32_t>>> cfg_memo;
    for (int64_t e = 0; e < g.N; ++e) {
      const int64_t Lo = g.shift(e, a, -1), Up = g.shift(e, a, +1);
      // face (Lo, e): u_hat from Lo when mu_Lo >= mu_e, lifting then acts on e
      const bool low_lift = mu[Lo] >= mu[e];
      // face (e, Up): u_hat from Up when mu_Up > mu_e
      const bool up_lift = mu[Up] > mu[e];
      const int key = int(low_lift) | (int(up_lift) << 1) | (int(Lo == e) << 2) |
                      (int(Up == e) << 3) | (int(Lo == Up) << 4);
      auto it = cfg_memo.find(key);
      if (it == cfg_memo.end()) {
        std::vector<double> blk[3];
        for (auto& v : blk) v.assign(bb, 0.0);
        const int role_lo = (Lo == e) ? 0 : 1;
        const int role_up = (Up == e) ? 0 : ((Up == Lo) ? 1 : 2);
        for (size_t x = 0; x < bb; ++x) blk[0][x] += sG * vol[x];
        if (low_lift)  // -phi(-1) (phi(+1)^T u_Lo - phi(-1)^T u_e)
          for (size_t x = 0; x < bb; ++x) {
            blk[0][x] += sG * lolo[x];
            blk[role_lo][x] -= sG * lohi[x];
          }
        if (up_lift)  // +phi(+1) (phi(-1)^T u_Up - phi(+1)^T u_e)
          for (size_t x = 0; x < bb; ++x) {
            blk[0][x] -= sG * hihi[x];
            blk[role_up][x] += sG * hilo[x];
          }
        std::vector<std::pair<int, uint32_t>> lst;
        lst.push_back({0, G.pool.intern(blk[0].data())});
        if (low_lift && role_lo != 0) lst.push_back({role_lo, 0});
        if (up_lift && role_up != 0 && !(role_up == 1 && low_lift)) lst.push_back({role_up, 0});
        for (auto& r : lst)
          if (r.first != 0) r.second = G.pool.intern(blk[r.first].data());
        it = cfg_memo.emplace(key, lst).first;
      }
      for (auto& r : it->second) {
        const int64_t c = r.first == 0 ? e : (r.first == 1 ? Lo : Up);
        rows[e].push_back({int32_t(c), r.second});
      }
    }
    finish_rows(G, rows);
  }

  // --- mu-weighted mass: mu_e (h/2)^d I ---
  L.mmu_pool = Pool();
  L.mmu_pool.b = b;
  L.mmu.resize(g.N);
  {
    const double mE = std::pow(h / 2.0, dim);
    std::unordered_map<uint64_t, uint32_t> mm_memo;
    std::vector<double> blk(bb);
    for (int64_t e = 0; e < g.N; ++e) {
      auto it = mm_memo.find(dbits(mu[e]));
      if (it == mm_memo.end()) {
        std::fill(blk.begin(), blk.end(), 0.0);
        for (int r = 0; r < b; ++r) blk[size_t(r) * b + r] = mu[e] * mE;
        it = mm_memo.emplace(dbits(mu[e]), L.mmu_pool.intern(blk.data())).first;
      }
      L.mmu[e] = it->second;
    }
  }

  // --- penalty E = sum_faces tau_f int_f [u][v], tau_f = tau0 min(mu) / h ---
  build_penalty(L.E, g, B, dim, b,
                [&](int64_t x, int64_t e) { return tau0 * std::min(mu[x], mu[e]) / h * wface; });
  build_A(L);
  return "";
}

double stokes_zeta(int gamma, int dim, int p) {
  static const double z2[2][5] = {{0.0382, 0.131, 0.0990, 0.153, 0.142}, {0.118, 0.131, 0.0814, 0.123, 0.0745}};
  static const double z3[2][3] = {{0.0462, 0.107, 0.113}, {0.0384, 0.0928, 0.0930}};
  const int g = gamma ? 1 : 0;
  if (dim == 2 && p >= 1 && p <= 5) return z2[g][p - 1];
  if (dim == 3 && p >= 1 && p <= 3) return z3[g][p - 1];
  return 0.1;
}

std::string assemble_stokes_fine(HostLevel& L, int dim, int n, int p, const double* mu_in, int gamma,
                                 double tau0, double taup) {
  if (gamma != 0 && gamma != 1) return "gamma must be 0 (standard form) or 1 (stress form)";
  if (!(taup >= 0.0) || !std::isfinite(taup)) return "taup must be non-negative and finite";
  std::string err = assemble_fine(L, dim, n, p, mu_in, tau0);
  if (!err.empty()) return err;
  const Basis1D B = make_basis(p);
  Grid g{dim, n, L.N};
  const double h = L.h, wface = std::pow(h / 2.0, dim - 1);
  std::vector<double> mu(L.N, 1.0);
  if (mu_in)
    for (int64_t e = 0; e < L.N; ++e) mu[e] = mu_in[e];
  // E_p = sum_faces tau_p int_f [p][q], tau_p = taup h / min(mu) (scaling E_p ~ h^d / mu, Sec. 3.3)
  build_penalty(L.Ep, g, B, dim, L.bs,
                [&](int64_t x, int64_t e) { return taup * h / std::min(mu[x], mu[e]) * wface; });
  L.gamma = gamma;
  L.nf = dim + 1;
  L.b = L.nf * L.bs;
  build_A_stokes(L);
  return "";
}

// --------------------------------------------------------------------------
// Operator coarsening (Sec. 2.2):
//   G_c = M_c^{-1} I^T M_f G_f I = 2^{-d} sum_{c,c'} P_c^T G_f[c,c'] P_c'
//   M_mu,c = I^T M_mu,f I,   E_c = (1/2) I^T E_f I,   A_c = sum G_c^T M_mu,c G_c + E_c
// --------------------------------------------------------------------------

static void coarsen_pbsr(const PBSR& F, PBSR& C, const Grid& gf, const Grid& gc,
                         const std::vector<std::vector<double>>& Pc, double factor, int b) {
  const int d = gf.d, nch = 1 << d;
  const size_t bb = size_t(b) * b;
  C = PBSR();
  C.pool.b = b;
  Memo memo;
  std::vector<std::vector<std::pair<int32_t, uint32_t>>> rows(gc.N);
  std::vector<std::pair<int32_t, std::array<uint32_t, 3>>> terms;
  std::vector<double> acc(bb), tmp(bb), tmp2(bb);
  int cc[3], cf[3];
  for (int64_t Ce = 0; Ce < gc.N; ++Ce) {
    gc.coords(Ce, cc);
    terms.clear();
    for (int s = 0; s < nch; ++s) {
      for (int t = 0; t < d; ++t) cf[t] = 2 * cc[t] + ((s >> t) & 1);
      const int64_t f = gf.index(cf);
      for (int64_t z = F.row_ptr[f]; z < F.row_ptr[f + 1]; ++z) {
        int c2[3];
        gf.coords(F.col[z], c2);
        int sp = 0, pc[3];
        for (int t = 0; t < d; ++t) {
          sp |= (c2[t] & 1) << t;
          pc[t] = c2[t] >> 1;
        }
        terms.push_back({int32_t(gc.index(pc)), {uint32_t(s), uint32_t(sp), F.id[z]}});
      }
    }
    std::sort(terms.begin(), terms.end());
    size_t s0 = 0;
    while (s0 < terms.size()) {
      size_t e = s0;
      std::vector<uint64_t> key;
      while (e < terms.size() && terms[e].first == terms[s0].first) {
        const auto& t = terms[e].second;
        key.push_back((uint64_t(t[0]) << 40) | (uint64_t(t[1]) << 32) | t[2]);
        ++e;
      }
      auto it = memo.find(key);
      uint32_t id;
      if (it != memo.end()) {
        id = it->second;
      } else {
        std::fill(acc.begin(), acc.end(), 0.0);
        for (size_t u = s0; u < e; ++u) {
          const auto& t = terms[u].second;
          mm(F.pool.get(t[2]), Pc[t[1]].data(), tmp.data(), b);  // G P_c'
          mtm_acc(Pc[t[0]].data(), tmp.data(), acc.data(), b);   // P_c^T (G P_c')
        }
        for (auto& v : acc) v *= factor;
        id = C.pool.intern(acc.data());
        memo.emplace(std::move(key), id);
      }
      rows[Ce].push_back({terms[s0].first, id});
      s0 = e;
    }
  }
  finish_rows(C, rows);
}

std::string coarsen(const HostLevel& F, HostLevel& C) {
  if (F.n % 2 != 0 || F.n < 2) return "cannot coarsen odd n";
  const int d = F.dim, b = F.bs, nch = 1 << d;
  const Basis1D B = make_basis(F.p);
  std::vector<std::vector<double>> Pc(nch);
  for (int s = 0; s < nch; ++s) Pc[s] = child_block(B, s, d);
  Grid gf{d, F.n, F.N}, gc{d, F.n / 2, F.N >> d};
  C.dim = d;
  C.n = F.n / 2;
  C.p = F.p;
  C.b = F.b;
  C.bs = b;
  C.nf = F.nf;
  C.gamma = F.gamma;
  C.N = gc.N;
  C.h = 2.0 * F.h;
  for (int a = 0; a < d; ++a) coarsen_pbsr(F.G[a], C.G[a], gf, gc, Pc, std::ldexp(1.0, -d), b);
  coarsen_pbsr(F.E, C.E, gf, gc, Pc, 0.5, b);
  if (F.nf > 1) coarsen_pbsr(F.Ep, C.Ep, gf, gc, Pc, 2.0, b);
  // M_mu,c[C] = sum_c P_c^T M_mu,f[c] P_c
  C.mmu_pool = Pool();
  C.mmu_pool.b = b;
  C.mmu.resize(gc.N);
  Memo memo;
  const size_t bb = size_t(b) * b;
  std::vector<double> acc(bb), tmp(bb);
  int cc[3], cf[3];
  for (int64_t Ce = 0; Ce < gc.N; ++Ce) {
    gc.coords(Ce, cc);
    std::vector<uint64_t> key;
    for (int s = 0; s < nch; ++s) {
      for (int t = 0; t < d; ++t) cf[t] = 2 * cc[t] + ((s >> t) & 1);
      key.push_back(F.mmu[gf.index(cf)]);
    }
    auto it = memo.find(key);
    if (it == memo.end()) {
      std::fill(acc.begin(), acc.end(), 0.0);
      for (int s = 0; s < nch; ++s) {
        mm(F.mmu_pool.get(uint32_t(key[s])), Pc[s].data(), tmp.data(), b);
        mtm_acc(Pc[s].data(), tmp.data(), acc.data(), b);
      }
      it = memo.emplace(key, C.mmu_pool.intern(acc.data())).first;
    }
    C.mmu[Ce] = it->second;
  }
  if (C.nf > 1) build_A_stokes(C);
  else build_A(C);
  return "";
}

std::string build_coarse_levels(const HostLevel& fine, std::vector<HostLevel>& out) {
  const HostLevel* F = &fine;
  while (F->n % 2 == 0 && F->n > 1) {
    HostLevel c;
    std::string err = coarsen(*F, c);
    if (!err.empty()) return err;
    out.push_back(std::move(c));
    F = &out.back();            // taken after push_back: no dangling reference
  }
  return "";
}

// --------------------------------------------------------------------------
// Dense symmetric eigen-decomposition by the cyclic Jacobi method
// (Golub & Van Loan, Matrix Computations, Sec. 8.5): used for the b x b
// diagonal blocks of block Jacobi.
// --------------------------------------------------------------------------

static void sym_eig_jacobi(std::vector<double> A, int n, std::vector<double>& lam,
                           std::vector<double>& V) {
  V.assign(size_t(n) * n, 0.0);
  for (int i = 0; i < n; ++i) V[size_t(i) * n + i] = 1.0;
  double fro = 0.0;
  for (double x : A) fro += x * x;
  fro = std::sqrt(fro);
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += A[size_t(i) * n + j] * A[size_t(i) * n + j];
    if (std::sqrt(off) <= 1e-17 * fro) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[size_t(p) * n + q];
        if (std::fabs(apq) <= 1e-300) continue;
        const double app = A[size_t(p) * n + p], aqq = A[size_t(q) * n + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = A[size_t(k) * n + p], akq = A[size_t(k) * n + q];
          A[size_t(k) * n + p] = c * akp - s * akq;
          A[size_t(k) * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = A[size_t(p) * n + k], aqk = A[size_t(q) * n + k];
          A[size_t(p) * n + k] = c * apk - s * aqk;
          A[size_t(q) * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[size_t(k) * n + p], vkq = V[size_t(k) * n + q];
          V[size_t(k) * n + p] = c * vkp - s * vkq;
          V[size_t(k) * n + q] = s * vkp + c * vkq;
        }
      }
  }
  lam.resize(n);
  for (int i = 0; i < n; ++i) lam[i] = A[size_t(i) * n + i];
}

static std::vector<double> sym_pinv(const double* S, int n, double cutoff) {
  std::vector<double> A(S, S + size_t(n) * n), lam, V;
  // symmetrise against rounding in the assembled block
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      const double m = 0.5 * (A[size_t(i) * n + j] + A[size_t(j) * n + i]);
      A[size_t(i) * n + j] = A[size_t(j) * n + i] = m;
    }
  sym_eig_jacobi(A, n, lam, V);
  double lmax = 0.0;
  for (double l : lam) lmax = std::max(lmax, std::fabs(l));
  std::vector<double> out(size_t(n) * n, 0.0);
  for (int k = 0; k < n; ++k) {
    if (std::fabs(lam[k]) <= cutoff * lmax) continue;
    const double inv = 1.0 / lam[k];
    for (int i = 0; i < n; ++i) {
      const double vi = V[size_t(i) * n + k] * inv;
      for (int j = 0; j < n; ++j) out[size_t(i) * n + j] += vi * V[size_t(j) * n + k];
    }
  }
  return out;
}

// --------------------------------------------------------------------------
// Dense least squares by Householder QR (the paper uses a LAPACK QR least
// squares solver, Sec. 2.3.3).  M: m x nc column-major, R: m x nr
// column-major, overwritten.  X: nc x nr column-major.  Returns false when M
// is numerically rank deficient (|R_jj| <= 1e-12 max |R_jj|).
// --------------------------------------------------------------------------

static bool householder_ls(std::vector<double>& M, int m, int nc, std::vector<double>& Rhs, int nr,
                           std::vector<double>& X) {
  std::vector<double> diag(nc), v(m);
  for (int j = 0; j < nc; ++j) {
    double* colj = M.data() + size_t(j) * m;
    double nrm2 = 0.0;
    for (int i = j; i < m; ++i) nrm2 += colj[i] * colj[i];
    const double nrm = std::sqrt(nrm2);
    if (nrm == 0.0) {
      diag[j] = 0.0;
      continue;
    }
    const double alpha = colj[j] > 0 ? -nrm : nrm;
    for (int i = j; i < m; ++i) v[i] = colj[i];
    v[j] -= alpha;
    double vv = 0.0;
    for (int i = j; i < m; ++i) vv += v[i] * v[i];
    diag[j] = alpha;
    colj[j] = alpha;
    for (int i = j + 1; i < m; ++i) colj[i] = 0.0;
    if (vv == 0.0) continue;
    const double beta = 2.0 / vv;
    for (int c = j + 1; c < nc; ++c) {
      double* cc = M.data() + size_t(c) * m;
      double s = 0.0;
      for (int i = j; i < m; ++i) s += v[i] * cc[i];
      s *= beta;
      for (int i = j; i < m; ++i) cc[i] -= s * v[i];
    }
    for (int c = 0; c < nr; ++c) {
      double* cc = Rhs.data() + size_t(c) * m;
      double s = 0.0;
      for (int i = j; i < m; ++i) s += v[i] * cc[i];
      s *= beta;
      for (int i = j; i < m; ++i) cc[i] -= s * v[i];
    }
  }
  double dmax = 0.0;
  for (double x : diag) dmax = std::max(dmax, std::fabs(x));
  for (double x : diag)
    if (!(std::fabs(x) > 1e-12 * dmax)) return false;
  X.assign(size_t(nc) * nr, 0.0);
  for (int c = 0; c < nr; ++c) {
    const double* rc = Rhs.data() + size_t(c) * m;
    double* xc = X.data() + size_t(c) * nc;
    for (int j = nc - 1; j >= 0; --j) {
      double s = rc[j];
      for (int l = j + 1; l < nc; ++l) s -= M[size_t(l) * m + j] * xc[l];
      xc[j] = s / M[size_t(j) * m + j];
    }
  }
  return true;
}

// Minimum-norm least squares for a rank-deficient M (tiny periodic levels
// where S(i) covers the whole mesh and the kernel of A lies in its span):
// X = V Sigma^+ U^T Rhs from a one-sided Jacobi SVD of M (Hestenes: plane
// rotations of column pairs until all pairs are orthogonal to 1e-15), singular
// values at or below 1e-12 of the largest treated as zero.
static void minnorm_ls(const std::vector<double>& M0, int m, int nc, const std::vector<double>& Rhs, int nr,
                       std::vector<double>& X) {
  std::vector<double> W = M0;                       // m x nc column-major, becomes U Sigma
  std::vector<double> V(size_t(nc) * nc, 0.0);      // nc x nc column-major
  for (int i = 0; i < nc; ++i) V[size_t(i) * nc + i] = 1.0;
  auto col = [&](std::vector<double>& A, int rows, int j) { return A.data() + size_t(j) * rows; };
  for (int sweep = 0; sweep < 60; ++sweep) {
    bool rotated = false;
    for (int i = 0; i < nc - 1; ++i)
      for (int j = i + 1; j < nc; ++j) {
        double* wi = col(W, m, i);
        double* wj = col(W, m, j);
        double a = 0.0, bq = 0.0, g = 0.0;
        for (int k = 0; k < m; ++k) {
          a += wi[k] * wi[k];
          bq += wj[k] * wj[k];
          g += wi[k] * wj[k];
        }
        if (!(std::fabs(g) > 1e-15 * std::sqrt(a * bq))) continue;
        rotated = true;
        const double zeta = (bq - a) / (2.0 * g);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
        for (int k = 0; k < m; ++k) {
          const double x = wi[k], y = wj[k];
          wi[k] = c * x - sn * y;
          wj[k] = sn * x + c * y;
        }
        double* vi = col(V, nc, i);
        double* vj = col(V, nc, j);
        for (int k = 0; k < nc; ++k) {
          const double x = vi[k], y = vj[k];
          vi[k] = c * x - sn * y;
          vj[k] = sn * x + c * y;
        }
      }
    if (!rotated) break;
  }
  std::vector<double> sig(nc);
  double smax = 0.0;
  for (int j = 0; j < nc; ++j) {
    double s2 = 0.0;
    const double* wj = col(W, m, j);
    for (int k = 0; k < m; ++k) s2 += wj[k] * wj[k];
    sig[j] = std::sqrt(s2);
    smax = std::max(smax, sig[j]);
  }
  X.assign(size_t(nc) * nr, 0.0);  // column-major nc x nr
  for (int j = 0; j < nc; ++j) {
    if (!(sig[j] > 1e-12 * smax)) continue;
    const double* wj = col(W, m, j);          // sigma_j u_j
    const double* vj = col(V, nc, j);
    for (int c = 0; c < nr; ++c) {
      const double* rc = Rhs.data() + size_t(c) * m;
      double proj = 0.0;
      for (int k = 0; k < m; ++k) proj += wj[k] * rc[k];
      proj /= sig[j] * sig[j];                // (u_j . r) / sigma_j
      for (int i = 0; i < nc; ++i) X[size_t(c) * nc + i] += proj * vj[i];
    }
  }
}

template <class F>
static void parallel_for(int64_t n, int nthreads, F&& f) {
  nthreads = std::max(1, std::min<int>(nthreads, int(std::max<int64_t>(n, 1))));
  if (nthreads == 1) {
    for (int64_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<int64_t> next{0};
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&] {
      for (;;) {
        const int64_t i = next.fetch_add(1);
        if (i >= n) break;
        f(i);
      }
    });
  for (auto& t : th) t.join();
}

// --------------------------------------------------------------------------
// Smoothers (Sec. 2.3)
// --------------------------------------------------------------------------

std::vector<int> greedy_colouring(const PBSR& A) {
  const int64_t N = A.nrows;
  std::vector<std::vector<int32_t>> nb(N);
  for (int64_t i = 0; i < N; ++i)
    for (int64_t z = A.row_ptr[i]; z < A.row_ptr[i + 1]; ++z) {
      const int32_t j = A.col[z];
      if (j == i) continue;
      nb[i].push_back(j);
      nb[j].push_back(int32_t(i));
    }
  std::vector<int> colour(N, -1);
  std::vector<char> used;
  for (int64_t i = 0; i < N; ++i) {
    used.assign(nb[i].size() + 2, 0);
    for (int32_t j : nb[i])
      if (colour[j] >= 0 && colour[j] < int(used.size())) used[colour[j]] = 1;
    int c = 0;
    while (used[c]) ++c;
    colour[i] = c;
  }
  return colour;
}

std::string setup_smoother(HostLevel& L, const SetupParams& sp, int nthreads) {
  const int b = L.b;
  const size_t bb = size_t(b) * b;
  const int64_t N = L.N;
  const PBSR& A = L.A;
  if (sp.smoother == 2) {
    // multi-coloured Gauss-Seidel: the Jacobi blocks plus the colour classes
    SetupParams jp = sp;
    jp.smoother = 0;
    std::string err = setup_smoother(L, jp, nthreads);
    if (!err.empty()) return err;
    const std::vector<int> colour = greedy_colouring(A);
    int nc = 0;
    for (int c : colour) nc = std::max(nc, c + 1);
    L.colour_ptr.assign(nc + 1, 0);
    for (int c : colour) L.colour_ptr[c + 1]++;
    for (int c = 0; c < nc; ++c) L.colour_ptr[c + 1] += L.colour_ptr[c];
    L.colour_rows.assign(N, 0);
    std::vector<int64_t> fill(L.colour_ptr.begin(), L.colour_ptr.end() - 1);
    for (int64_t i = 0; i < N; ++i) L.colour_rows[fill[colour[i]]++] = int32_t(i);
    return "";
  }
  if (sp.smoother == 0) {
    // block Jacobi: pseudo-inverse of A_ii from a symmetric eigendecomposition (Eq. Jsmooth)
    L.dinv_pool = Pool();
    L.dinv_pool.b = b;
    L.dinv.resize(N);
    std::unordered_map<uint32_t, uint32_t> memo;
    for (int64_t i = 0; i < N; ++i) {
      const uint32_t did = A.find(i, int32_t(i));
      auto it = memo.find(did);
      if (it == memo.end()) {
        auto P = sym_pinv(A.pool.get(did), b, 1e-12);
        it = memo.emplace(did, L.dinv_pool.intern(P.data())).first;
      }
      L.dinv[i] = it->second;
    }
    return "";
  }
  if (sp.smoother != 1) return "unknown smoother";
  if (sp.sai_level < 0 || sp.sai_level > 2) return "sai_level must be 0, 1 or 2";
  // balancing, one value per dof (N x b): alpha = ||A_ii||_F^{-1/2} on every dof
  // of element i (Sec. 2.3.3); for Stokes alpha_u = ||A_ii^uu||_F^{-1/2} on the
  // velocity dofs and alpha_p = zeta ||A_ii^uu||_F^{1/2} ||D_ii||_F^{-1} on the
  // pressure dofs, D_ii the divergence sub-block (Sec. 3.3).
  std::vector<double> alpha(size_t(N) * b, 1.0);
  std::vector<uint32_t> diag_id(N);
  const double zeta = sp.zeta > 0.0 ? sp.zeta : stokes_zeta(L.gamma, L.dim, L.p);
  for (int64_t i = 0; i < N; ++i) {
    diag_id[i] = A.find(i, int32_t(i));
    if (!sp.balance) continue;
    const double* D = A.pool.get(diag_id[i]);
    double* al = alpha.data() + size_t(i) * b;
    if (L.nf == 1) {
      double f = 0.0;
      for (size_t x = 0; x < bb; ++x) f += D[x] * D[x];
      const double a = 1.0 / std::sqrt(std::sqrt(f));
      for (int r = 0; r < b; ++r) al[r] = a;
    } else {
      const int nu = L.dim * L.bs;
      double fuu = 0.0, fpu = 0.0;
      for (int r = 0; r < b; ++r)
        for (int c = 0; c < nu; ++c) {
          const double v = D[size_t(r) * b + c];
          if (r < nu) fuu += v * v;
          else fpu += v * v;
        }
      const double nuu = std::sqrt(fuu), npu = std::sqrt(fpu);
      if (!(nuu > 0.0) || !(npu > 0.0)) return "Stokes balancing: zero viscous or divergence diagonal block";
      const double au = 1.0 / std::sqrt(nuu), ap = zeta * std::sqrt(nuu) / npu;
      for (int r = 0; r < b; ++r) al[r] = r < nu ? au : ap;
    }
  }
  Grid g{L.dim, L.n, N};
  auto rel_key = [&](int64_t i, int64_t k) {
    int ci[3], ck[3];
    g.coords(i, ci);
    g.coords(k, ck);
    int64_t key = 0;
    for (int t = L.dim - 1; t >= 0; --t) key = key * L.n + (((ck[t] - ci[t]) % L.n) + L.n) % L.n;
    return key;
  };
  // S(i): ell hops in the (symmetric) block graph of A; R(i): rows of A[:, S(i)]
  struct Col {
    std::vector<int32_t> S, R;
    uint32_t key_id;
  };
  std::vector<Col> cols(N);
  Memo key_memo;
  std::vector<std::vector<uint64_t>> keys;
  std::vector<int64_t> rep;  // representative column per key
  std::vector<char> mark(N, 0);
  for (int64_t i = 0; i < N; ++i) {
    std::vector<int32_t> S{int32_t(i)};
    mark[i] = 1;
    size_t frontier = 0;
    for (int hop = 0; hop < sp.sai_level; ++hop) {
      const size_t end = S.size();
      for (size_t u = frontier; u < end; ++u)
        for (int64_t z = A.row_ptr[S[u]]; z < A.row_ptr[S[u] + 1]; ++z)
          if (!mark[A.col[z]]) {
            mark[A.col[z]] = 1;
            S.push_back(A.col[z]);
          }
      frontier = end;
    }
    for (int32_t k : S) mark[k] = 0;
    std::vector<int32_t> R;
    for (int32_t k : S)
      for (int64_t z = A.row_ptr[k]; z < A.row_ptr[k + 1]; ++z)
        if (!mark[A.col[z]]) {
          mark[A.col[z]] = 1;
          R.push_back(A.col[z]);
        }
    for (int32_t r : R) mark[r] = 0;
    auto by_offset = [&](int32_t x, int32_t y) { return rel_key(i, x) < rel_key(i, y); };
    std::sort(S.begin(), S.end(), by_offset);
    std::sort(R.begin(), R.end(), by_offset);
    std::vector<uint64_t> key;
    key.push_back((uint64_t(S.size()) << 32) | R.size());
    for (int32_t r : R) key.push_back(diag_id[r]);
    for (int32_t r : R)
      for (int32_t k : S) key.push_back(A.find(r, k));
    auto it = key_memo.find(key);
    if (it == key_memo.end()) {
      it = key_memo.emplace(key, uint32_t(keys.size())).first;
      keys.push_back(key);
      rep.push_back(i);
    }
    cols[i].S = std::move(S);
    cols[i].R = std::move(R);
    cols[i].key_id = it->second;
  }
  // one balanced least-squares problem per distinct key, in chunks (bounded
  // host memory): W = [Atilde[R, S] | E[R, i]] built on the host threads,
  // solved by sp.ls (the device) or by Householder QR on the host threads;
  // rank-deficient ones take the minimum-norm solution on the host
  const int64_t nkeys = int64_t(keys.size());
  std::vector<std::vector<double>> sol(nkeys);
  auto build_W = [&](int64_t kid, LsProblem& P) {
    const int64_t i = rep[kid];
    const auto& S = cols[i].S;
    const auto& R = cols[i].R;
    const int m = int(R.size()) * b, nc = int(S.size()) * b;
    P.m = m;
    P.nc = nc;
    P.nr = b;
    P.W.assign(size_t(m) * (nc + b), 0.0);
    for (size_t ri = 0; ri < R.size(); ++ri)
      for (size_t kj = 0; kj < S.size(); ++kj) {
        const uint32_t id = A.find(R[ri], S[kj]);
        if (id == UINT32_MAX) continue;
        const double* blk = A.pool.get(id);
        const double* ar = alpha.data() + size_t(R[ri]) * b;
        const double* ac = alpha.data() + size_t(S[kj]) * b;
        for (int c = 0; c < b; ++c) {
          double* dst = P.W.data() + size_t(kj * b + c) * m + ri * b;
          for (int r = 0; r < b; ++r) dst[r] = (ar[r] * ac[c]) * blk[size_t(r) * b + c];
        }
      }
    size_t pos = 0;
    while (R[pos] != i) ++pos;
    for (int c = 0; c < b; ++c) P.W[size_t(nc + c) * m + pos * b + c] = 1.0;
  };
  const size_t per = size_t(cols[rep[0]].R.size()) * b * (cols[rep[0]].S.size() * b + b) * sizeof(double);
  const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(nkeys, int64_t((size_t(1) << 30) / std::max<size_t>(per, 1))));
  std::vector<LsProblem> batch;
  for (int64_t k0 = 0; k0 < nkeys; k0 += chunk) {
    const int64_t k1 = std::min(nkeys, k0 + chunk);
    batch.assign(size_t(k1 - k0), LsProblem());
    parallel_for(k1 - k0, nthreads, [&](int64_t t) { build_W(k0 + t, batch[size_t(t)]); });
    if (sp.ls) {
      const std::string err = sp.ls(batch);
      if (!err.empty()) return err;
    } else {
      parallel_for(k1 - k0, nthreads, [&](int64_t t) {
        LsProblem& P = batch[size_t(t)];
        std::vector<double> M(P.W.begin(), P.W.begin() + size_t(P.m) * P.nc);
        std::vector<double> Rhs(P.W.begin() + size_t(P.m) * P.nc, P.W.end());
        P.ok = householder_ls(M, P.m, P.nc, Rhs, P.nr, P.X);
      });
    }
    parallel_for(k1 - k0, nthreads, [&](int64_t t) {
      LsProblem& P = batch[size_t(t)];
      if (!P.ok) {
        const std::vector<double> M0(P.W.begin(), P.W.begin() + size_t(P.m) * P.nc);
        const std::vector<double> R0(P.W.begin() + size_t(P.m) * P.nc, P.W.end());
        minnorm_ls(M0, P.m, P.nc, R0, P.nr, P.X);
      }
      sol[size_t(k0 + t)] = std::move(P.X);   // nc x b column-major: Btilde[S, i]
    });
  }
  // B_ki = alpha_k Btilde_ki alpha_i, pooled per (key, position)
  L.B = PBSR();
  L.B.pool.b = b;
  L.BT = PBSR();
  L.BT.pool.b = b;
  std::unordered_map<uint64_t, std::pair<uint32_t, uint32_t>> bmemo;  // (key,t) -> (B id, BT id)
  std::vector<std::vector<std::pair<int32_t, uint32_t>>> brows(N), btrows(N);
  std::vector<double> blk(bb), blkT(bb);
  for (int64_t i = 0; i < N; ++i) {
    const auto& S = cols[i].S;
    const int nc = int(S.size()) * b;
    for (size_t t = 0; t < S.size(); ++t) {
      const uint64_t mk = (uint64_t(cols[i].key_id) << 20) | t;
      auto it = bmemo.find(mk);
      if (it == bmemo.end()) {
        const auto& X = sol[cols[i].key_id];
        const double* ar = alpha.data() + size_t(S[t]) * b;
        const double* ac = alpha.data() + size_t(i) * b;
        for (int r = 0; r < b; ++r)
          for (int c = 0; c < b; ++c) {
            const double v = (ar[r] * ac[c]) * X[size_t(c) * nc + t * b + r];
            blk[size_t(r) * b + c] = v;
            blkT[size_t(c) * b + r] = v;
          }
        it = bmemo.emplace(mk, std::make_pair(L.B.pool.intern(blk.data()), L.BT.pool.intern(blkT.data())))
                 .first;
      }
      brows[S[t]].push_back({int32_t(i), it->second.first});
      btrows[i].push_back({S[t], it->second.second});
    }
  }
  finish_rows(L.B, brows);
  finish_rows(L.BT, btrows);
  return "";
}

void dense_A(const HostLevel& L, std::vector<double>& out) {
  const int b = L.b;
  const int64_t n = L.N * b;
  out.assign(size_t(n) * n, 0.0);
  for (int64_t i = 0; i < L.N; ++i)
    for (int64_t z = L.A.row_ptr[i]; z < L.A.row_ptr[i + 1]; ++z) {
      const double* blk = L.A.pool.get(L.A.id[z]);
      const int64_t j = L.A.col[z];
      for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c) out[size_t(i * b + r) * n + j * b + c] = blk[size_t(r) * b + c];
    }
}

}  // namespace ldgmg
