// Host-side setup of the LDG multigrid hierarchy (assembly, operator
// coarsening, smoother construction).  Pure C++17; no CUDA.
//
// Every block-sparse operator is stored "pooled": a block-CSR pattern whose
// nonzero blocks are ids into a pool of distinct dense blocks.  Pools
// deduplicate by exact bytes, and every derived block is computed once per
// distinct combination of input block ids (memoised).  On a uniform periodic
// mesh each level therefore holds only a handful of distinct blocks and setup
// cost is independent of N; near an interface the number of distinct blocks
// grows with the interface length.  This generalises the SAI column cache of
// the paper (a hash table plus a one-to-one stencil mapping, Sec. 4 item (i))
// to every setup product.  Results are identical to computing every block
// separately, because a block is reused only when its inputs are bitwise equal.
#pragma once

#include <cstdint>
#include <functional>
#include <string>
#include <unordered_map>
#include <vector>

namespace ldgmg {

struct Basis1D {
  int p = 0, q = 0;                // degree, q = p + 1 modes
  std::vector<double> K;           // q*q, K[i*q+j] = int phi_i phi_j'
  std::vector<double> lo, hi;      // phi_k(-1), phi_k(+1)
  std::vector<double> P[2];        // q*q, P[s][i*q+j] = int phi_i(xi) phi_j((xi+2s-1)/2)
};
Basis1D make_basis(int p);

struct Pool {
  int b = 0;
  std::vector<double> data;        // block id -> b*b values, row-major (r, c)
  std::unordered_map<uint64_t, std::vector<uint32_t>> index;
  uint32_t intern(const double* blk);
  const double* get(uint32_t id) const { return data.data() + size_t(id) * b * b; }
  uint32_t size() const { return b ? uint32_t(data.size() / (size_t(b) * b)) : 0; }
};

struct PBSR {
  int64_t nrows = 0;
  std::vector<int64_t> row_ptr;    // nrows + 1
  std::vector<int32_t> col;        // sorted within each row
  std::vector<uint32_t> id;        // pool id per stored block
  Pool pool;
  int64_t nnzb() const { return int64_t(col.size()); }
  // pool id of block (r, c), or UINT32_MAX if structurally absent
  uint32_t find(int64_t r, int32_t c) const;
};

struct HostLevel {
  int dim = 0, n = 0, p = 0;
  int b = 0;                       // block size of the system A (nf * bs)
  int bs = 0;                      // block size of one scalar field, (p+1)^dim
  int nf = 1;                      // fields per element: 1 (scalar) or dim + 1 (Stokes)
  int gamma = 0;                   // Stokes form: 0 standard, 1 stress
  int64_t N = 0;
  double h = 0.0;
  // scalar pieces, block size bs
  PBSR G[3];                       // discrete gradient per axis
  std::vector<uint32_t> mmu;       // mu-weighted mass, one block per element
  Pool mmu_pool;
  PBSR E;                          // penalty
  PBSR Ep;                         // Stokes pressure penalty (nf > 1 only)
  // the system: sum_a G_a^T M_mu G_a + E (scalar), or the Stokes saddle-point
  // operator with field order (u_1, .., u_dim, p) inside each block (Sec. 3.1)
  PBSR A;
  // smoother
  PBSR B, BT;                      // SAI (BT holds the transposed blocks of B, row-wise)
  std::vector<uint32_t> dinv;      // Jacobi / Gauss-Seidel: pseudo-inverse of A_ii per element
  Pool dinv_pool;
  // multi-coloured Gauss-Seidel: elements of colour c are
  // colour_rows[colour_ptr[c] .. colour_ptr[c+1]), increasing
  std::vector<int32_t> colour_rows;
  std::vector<int64_t> colour_ptr;
};

// One balanced SAI least-squares problem (Sec. 2.3.3): W = [M | Rhs], m rows,
// nc + nr columns, column-major; the solution X (nc x nr, column-major)
// minimises ||M X - Rhs||_F.  ok = false: M is numerically rank deficient
// (|R_jj| <= 1e-12 max |R_jj| in its QR factor); the caller then takes the
// minimum-norm solution.
struct LsProblem {
  int m = 0, nc = 0, nr = 0;
  std::vector<double> W;
  std::vector<double> X;
  bool ok = false;
};
// Solves a batch of problems (fills X and ok); returns "" or an error message.
typedef std::function<std::string(std::vector<LsProblem>&)> LsSolver;

struct SetupParams {
  int smoother = 1;                // 0 Jacobi, 1 SAI, 2 multi-coloured Gauss-Seidel
  int sai_level = 1;
  int balance = 1;
  double zeta = 0.0;               // Stokes balancing (Sec. 3.3); <= 0: Table tab:zeta
  LsSolver ls;                     // SAI least squares; empty: Householder QR on the host threads
};

// Table tab:zeta: tuned Stokes balancing value for (gamma, dim, p); 0.1 where
// the table has no entry.
double stokes_zeta(int gamma, int dim, int p);

// Fine-level assembly (Sec. 2.1).  mu: N values or nullptr for mu == 1.
// Returns an empty string on success, else an error message.
std::string assemble_fine(HostLevel& L, int dim, int n, int p, const double* mu, double tau0);

// Fine-level Stokes assembly (Sec. 3.1, Eq. components): the scalar pieces as
// in assemble_fine, the pressure penalty E_p (tau_p = taup h / min(mu) per
// face), and the saddle-point system with blocks of size (dim + 1) bs.
std::string assemble_stokes_fine(HostLevel& L, int dim, int n, int p, const double* mu, int gamma,
                                 double tau0, double taup);

// Operator coarsening of `fine` onto n/2 (Sec. 2.2; per field for Stokes,
// with E_p,c = 2 I^T E_p I because tau_p scales with h).
std::string coarsen(const HostLevel& fine, HostLevel& coarse);

// Coarse levels of `fine` (n/2, n/4, ... while n is even and > 1), appended
// to `out` (which must not alias `fine`).
std::string build_coarse_levels(const HostLevel& fine, std::vector<HostLevel>& out);

// Greedy colouring of the (symmetrised) block pattern of A in element order
// (Sec. 2.3.2): colour of each element; red-black on the 5 / 7-point stencil.
std::vector<int> greedy_colouring(const PBSR& A);

// Smoother setup on one level (Jacobi blocks, Gauss-Seidel blocks and
// colours, or balanced SAI, Sec. 2.3).
std::string setup_smoother(HostLevel& L, const SetupParams& sp, int nthreads);

// Dense copy of A (row-major, (N*b)^2) for the bottom solver.
void dense_A(const HostLevel& L, std::vector<double>& out);

}  // namespace ldgmg
