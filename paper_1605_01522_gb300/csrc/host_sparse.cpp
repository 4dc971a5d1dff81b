// Host block-CSR kernels used by the AMG setup.  Row-parallel (OpenMP) with a
// fixed accumulation order per row, so results do not depend on the thread
// count.
#include "host_sparse.h"

#include <algorithm>
#include <cmath>
#include <numeric>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace mfs {

static void concat_rows(HBsr &C, std::vector<std::vector<int32_t>> &cols,
                        std::vector<std::vector<double>> &vals) {
  const int64_t bs = (int64_t)C.br * C.bc;
  C.rp.assign(C.nbr + 1, 0);
  for (int64_t i = 0; i < C.nbr; ++i) C.rp[i + 1] = C.rp[i] + (int64_t)cols[i].size();
  C.ci.resize(C.rp[C.nbr]);
  C.v.resize(C.rp[C.nbr] * bs);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < C.nbr; ++i) {
    std::copy(cols[i].begin(), cols[i].end(), C.ci.begin() + C.rp[i]);
    std::copy(vals[i].begin(), vals[i].end(), C.v.begin() + C.rp[i] * bs);
    std::vector<int32_t>().swap(cols[i]);
    std::vector<double>().swap(vals[i]);
  }
}

HBsr bsr_spgemm(const HBsr &A, const HBsr &B) {
  if (A.bc != B.br || A.nbc != B.nbr) throw SetupError(-1, "spgemm: shape mismatch");
  HBsr C;
  C.br = A.br;
  C.bc = B.bc;
  C.nbr = A.nbr;
  C.nbc = B.nbc;
  const int ar = A.br, ac = A.bc, bc = B.bc;
  const int cbs = ar * bc;
  std::vector<std::vector<int32_t>> cols(C.nbr);
  std::vector<std::vector<double>> vals(C.nbr);
#pragma omp parallel
  {
    std::vector<int32_t> mark(B.nbc, -1);
    std::vector<int32_t> touched;
    std::vector<double> acc;
    std::vector<int32_t> ord;
#pragma omp for schedule(dynamic, 512)
    for (int64_t I = 0; I < A.nbr; ++I) {
      touched.clear();
      acc.clear();
      for (int64_t a = A.rp[I]; a < A.rp[I + 1]; ++a) {
        const int32_t K = A.ci[a];
        const double *Ab = A.blk(a);
        for (int64_t q = B.rp[K]; q < B.rp[K + 1]; ++q) {
          const int32_t J = B.ci[q];
          if (mark[J] < 0) {
            mark[J] = (int32_t)touched.size();
            touched.push_back(J);
            acc.resize(acc.size() + cbs, 0.0);
          }
          double *Cb = acc.data() + (int64_t)mark[J] * cbs;
          const double *Bb = B.blk(q);
          for (int r = 0; r < ar; ++r)
            for (int k = 0; k < ac; ++k) {
              const double arv = Ab[r * ac + k];
              for (int c = 0; c < bc; ++c) Cb[r * bc + c] += arv * Bb[k * bc + c];
            }
        }
      }
      ord.resize(touched.size());
      std::iota(ord.begin(), ord.end(), 0);
      std::sort(ord.begin(), ord.end(), [&](int x, int y) { return touched[x] < touched[y]; });
      cols[I].resize(touched.size());
      vals[I].resize(touched.size() * cbs);
      for (size_t t = 0; t < ord.size(); ++t) {
        cols[I][t] = touched[ord[t]];
        std::copy(acc.begin() + (int64_t)ord[t] * cbs, acc.begin() + (int64_t)(ord[t] + 1) * cbs,
                  vals[I].begin() + (int64_t)t * cbs);
      }
      for (int32_t J : touched) mark[J] = -1;
    }
  }
  concat_rows(C, cols, vals);
  return C;
}

HBsr bsr_transpose(const HBsr &A) {
  HBsr T;
  T.br = A.bc;
  T.bc = A.br;
  T.nbr = A.nbc;
  T.nbc = A.nbr;
  const int64_t bs = (int64_t)A.br * A.bc;
  T.rp.assign(T.nbr + 1, 0);
  for (int32_t c : A.ci) T.rp[c + 1]++;
  for (int64_t i = 0; i < T.nbr; ++i) T.rp[i + 1] += T.rp[i];
  T.ci.resize(A.ci.size());
  T.v.resize(A.v.size());
  std::vector<int64_t> pos(T.rp.begin(), T.rp.end() - 1);
  for (int64_t I = 0; I < A.nbr; ++I)
    for (int64_t a = A.rp[I]; a < A.rp[I + 1]; ++a) {
      const int64_t p = pos[A.ci[a]]++;
      T.ci[p] = (int32_t)I;
      const double *s = A.blk(a);
      double *d = T.v.data() + p * bs;
      for (int r = 0; r < A.br; ++r)
        for (int c = 0; c < A.bc; ++c) d[c * A.br + r] = s[r * A.bc + c];
    }
  return T;
}

HBsr bsr_axpby(double a, const HBsr &A, double b, const HBsr &B) {
  if (A.br != B.br || A.bc != B.bc || A.nbr != B.nbr || A.nbc != B.nbc)
    throw SetupError(-1, "axpby: shape mismatch");
  HBsr C;
  C.br = A.br;
  C.bc = A.bc;
  C.nbr = A.nbr;
  C.nbc = A.nbc;
  const int64_t bs = (int64_t)A.br * A.bc;
  std::vector<std::vector<int32_t>> cols(C.nbr);
  std::vector<std::vector<double>> vals(C.nbr);
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t I = 0; I < A.nbr; ++I) {
    int64_t p = A.rp[I], q = B.rp[I];
    const int64_t pe = A.rp[I + 1], qe = B.rp[I + 1];
    auto &cc = cols[I];
    auto &vv = vals[I];
    while (p < pe || q < qe) {
      int32_t ca = p < pe ? A.ci[p] : INT32_MAX;
      int32_t cb = q < qe ? B.ci[q] : INT32_MAX;
      const int32_t c = std::min(ca, cb);
      cc.push_back(c);
      const size_t o = vv.size();
      vv.resize(o + bs, 0.0);
      if (ca == c) {
        for (int64_t e = 0; e < bs; ++e) vv[o + e] += a * A.v[p * bs + e];
        ++p;
      }
      if (cb == c) {
        for (int64_t e = 0; e < bs; ++e) vv[o + e] += b * B.v[q * bs + e];
        ++q;
      }
    }
  }
  concat_rows(C, cols, vals);
  return C;
}

void bsr_scale_rows(HBsr &A, const std::vector<double> &d) {
#pragma omp parallel for schedule(static)
  for (int64_t I = 0; I < A.nbr; ++I)
    for (int64_t a = A.rp[I]; a < A.rp[I + 1]; ++a) {
      double *blk = A.blk(a);
      for (int r = 0; r < A.br; ++r)
        for (int c = 0; c < A.bc; ++c) blk[r * A.bc + c] *= d[I * A.br + r];
    }
}

void bsr_matvec(const HBsr &A, const double *x, double *y) {
#pragma omp parallel for schedule(static)
  for (int64_t I = 0; I < A.nbr; ++I) {
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t a = A.rp[I]; a < A.rp[I + 1]; ++a) {
      const double *blk = A.blk(a);
      const double *xv = x + (int64_t)A.ci[a] * A.bc;
      for (int r = 0; r < A.br; ++r)
        for (int c = 0; c < A.bc; ++c) acc[r] += blk[r * A.bc + c] * xv[c];
    }
    for (int r = 0; r < A.br; ++r) y[I * A.br + r] = acc[r];
  }
}

std::vector<double> bsr_point_diagonal(const HBsr &A) {
  std::vector<double> d(A.nbr * A.br, 0.0);
  for (int64_t I = 0; I < A.nbr; ++I)
    for (int64_t a = A.rp[I]; a < A.rp[I + 1]; ++a)
      if (A.ci[a] == I)
        for (int r = 0; r < A.br; ++r) d[I * A.br + r] = A.blk(a)[r * A.bc + r];
  return d;
}

std::vector<double> bsr_abs_row_sums(const HBsr &A) {
  std::vector<double> s(A.nbr * A.br, 0.0);
#pragma omp parallel for schedule(static)
  for (int64_t I = 0; I < A.nbr; ++I)
    for (int64_t a = A.rp[I]; a < A.rp[I + 1]; ++a)
      for (int r = 0; r < A.br; ++r)
        for (int c = 0; c < A.bc; ++c) s[I * A.br + r] += std::fabs(A.blk(a)[r * A.bc + c]);
  return s;
}

}  // namespace mfs
