// Smoothed-aggregation AMG setup on the host (timed apart from the solve).
//
// Single-field objects P^l_i, R^l_i, A^l_ii and smoother data per field and
// level (Sec. 3.3, Sec. 4.3), blockwise Galerkin coarse blocks for the
// monolithic hierarchy (Sec. 4.3), the SIMPLE approximation A~_11 and the
// explicit S~ (Sec. 4.2), and dense LU factors of the coarsest operators.
// Aggregation and the tentative prolongator follow the steps fixed for this
// library (the paper cites smoothed aggregation without detail):
//   strength |A_IJ|_F > theta sqrt(|A_II|_F |A_JJ|_F), symmetrised;
//   roots = lexicographically-first distance-2 maximal independent set in
//   decreasing SplitMix64 priority (ties: lower index); neighbours of a root
//   join it; remaining nodes join the neighbouring aggregate whose root has
//   the highest priority; nodes without strong neighbours stay unaggregated;
//   per-aggregate Gram-Schmidt QR (two passes, columns with remaining norm
//   <= 1e-10 of the original dropped) of the near-nullspace, rotations about
//   the aggregate centroid; lambda_max(D^-1 A) by 10 power iterations from a
//   SplitMix64 start vector; P = (I - 4/(3 lambda) D^-1 A) P_tent; R = P^T.
#pragma once
#include <cstdint>
#include <map>
#include <utility>
#include <vector>

#include "host_sparse.h"

namespace mfs {

struct FieldInfo {
  int64_t nnodes = 0;
  int b = 1, dim = 3;
  int ns = 0;  // 0 constants, 1 rigid-body modes, 2 the caller's vectors (user_B)
  int ns_dim = 0;              // ns == 2: vectors per dof
  std::vector<double> user_B;  // ns == 2: nnodes * b * ns_dim, dof-major
  std::vector<uint8_t> dirichlet;  // empty or nnodes * b flags of eliminated Dirichlet dofs
  double theta = 0.0;
  std::vector<double> coords;
  bool pg = false;  // Petrov-Galerkin transfers (non-symmetric block)
  // nodes whose every dof is a flagged Dirichlet dof (empty: none flagged)
  std::vector<uint8_t> fixed_nodes() const {
    std::vector<uint8_t> m;
    if (dirichlet.empty()) return m;
    m.assign(nnodes, 1);
    for (int64_t I = 0; I < nnodes; ++I)
      for (int c = 0; c < b; ++c)
        if (!dirichlet[I * b + c]) m[I] = 0;
    return m;
  }
};

struct HLevelField {
  HBsr A;                      // diagonal block A^l_ii
  std::vector<double> dinv;    // inverse point diagonal
  double lam = 0.0;            // lambda_max(D^-1 A) estimate (levels < coarsest)
  std::vector<int32_t> agg;    // node -> aggregate (-1 unaggregated)
  int64_t nagg = 0;
  HBsr P, R;                   // to level l+1
  std::vector<double> B;       // near-nullspace on coarse levels (n x b)
  std::vector<int32_t> color;  // Gauss-Seidel node colours (smoothed levels, MFS_GS only)
};

struct HDenseLU {
  int n = 0;
  std::vector<double> lu;      // column-major n x n, unit-lower L below the diagonal
  std::vector<int32_t> perm;   // y = b[perm]
};

using BlockMap = std::map<std::pair<int, int>, HBsr>;

struct HGroup {
  int nf = 0;
  std::vector<FieldInfo> info;
  std::vector<std::vector<HLevelField>> lv;  // [level][field]
  std::vector<BlockMap> off;                 // [level] off-diagonal blocks (monolithic AMG only)
  std::vector<HDenseLU> coarse_field;        // per-field LU of the coarsest A_ii
  HDenseLU coarse_coupled;                   // LU of the assembled coarsest coupled matrix
  int nlevels() const { return (int)lv.size(); }
};

void build_group(HGroup &g, const std::vector<HBsr> &diag, const std::vector<FieldInfo> &info,
                 int max_levels, int64_t coarse_max, uint64_t seed, bool want_off,
                 const BlockMap *fine_off, int verbose = 0);
HDenseLU dense_lu(int n, std::vector<double> a_rowmajor);
// lambda_max(D^-1 A) estimate (10 power iterations) and the inverse point
// diagonal, as used by the setup for every smoothed level
double amg_power_lambda(const HBsr &A, const std::vector<double> &dinv, uint64_t seed);
std::vector<double> amg_dinv(const HBsr &A);
// Greedy node colouring for multicolour Gauss-Seidel: node i (increasing
// order) takes the smallest colour not held by a lower-numbered node it
// couples with; i != j couple when some entry of block (i, j) or (j, i)
// exceeds 1e-12 times the largest entry of that block row (so rounding-level
// Galerkin entries do not count).
std::vector<int32_t> node_colors(const HBsr &A);
// Petrov-Galerkin transfers after Sala & Tuminaro (2008), for non-symmetric
// blocks (the paper's fluid field, Sec. 7.2): with Q = D^-1 A Pt, per coarse
// scalar dof j omega_j = <A q_j, q_j> / <A q_j, D^-1 A q_j> (the minimiser of
// ||A (p_j - w q_j)||_{D^-1}; 0 unless positive); row i of P takes the
// minimum of omega_j over its columns with |Q_ij| > 1e-12 max|Q| (0 if none),
// which keeps P Bc = B when A B = 0; P = Pt - diag(omega) Q.  R is the
// transpose of the same construction on A^T (same D).
void pg_transfers(const HBsr &A, const std::vector<double> &dinv, const HBsr &Pt, HBsr &P, HBsr &R);
std::vector<double> bsr_to_dense(const HBsr &A);

}  // namespace mfs
