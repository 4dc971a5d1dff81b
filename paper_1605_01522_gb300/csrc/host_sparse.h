// Host-side block-CSR containers and the sparse kernels of the AMG setup
// (Galerkin products R A P of Sec. 3.3 / blockwise R_i A_ij P_j of Sec. 4.3,
// prolongator smoothing, the explicit SIMPLE Schur complement of Sec. 4.2).
#pragma once
#include <cstdint>
#include <vector>
#include <string>
#include <stdexcept>

namespace mfs {

struct SetupError : std::runtime_error {
  int code;
  SetupError(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};

// Node-level block-CSR: block k is v[k*br*bc ...] row-major, columns sorted.
struct HBsr {
  int br = 0, bc = 0;
  int64_t nbr = 0, nbc = 0;
  std::vector<int64_t> rp;  // nbr + 1
  std::vector<int32_t> ci;
  std::vector<double> v;
  int64_t nnzb() const { return (int64_t)ci.size(); }
  bool empty() const { return nbr == 0 && nbc == 0; }
  int64_t nrows() const { return nbr * br; }
  int64_t ncols() const { return nbc * bc; }
  const double *blk(int64_t k) const { return v.data() + k * br * bc; }
  double *blk(int64_t k) { return v.data() + k * br * bc; }
};

HBsr bsr_spgemm(const HBsr &A, const HBsr &B);                 // A * B
HBsr bsr_transpose(const HBsr &A);                              // A^T (blocks transposed)
HBsr bsr_axpby(double a, const HBsr &A, double b, const HBsr &B);  // a A + b B, union pattern
void bsr_scale_rows(HBsr &A, const std::vector<double> &d);     // row r *= d[r] (point rows)
void bsr_matvec(const HBsr &A, const double *x, double *y);     // y = A x (point vectors)
std::vector<double> bsr_point_diagonal(const HBsr &A);
std::vector<double> bsr_abs_row_sums(const HBsr &A);            // sum_j |a_rj| per point row

// SplitMix64 (Steele, Lea & Flood 2014), output i of the stream seeded with s.
inline uint64_t splitmix64_at(uint64_t s, uint64_t i) {
  uint64_t z = s + (i + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
inline double uniform01_at(uint64_t s, uint64_t i) {
  return (double)(splitmix64_at(s, i) >> 11) * 0x1.0p-53;
}

}  // namespace mfs
