// Smoothed-aggregation setup on the host; see amg_setup.h for the steps.
#include "amg_setup.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <numeric>

namespace mfs {

namespace {

struct Graph {
  int64_t n = 0;
  std::vector<int64_t> rp;
  std::vector<int32_t> ci;
};

// Strong-connection node graph (symmetrised, no self loops); nodes flagged
// in `fixed` (if not empty) keep no edge.
Graph strength_graph(const HBsr &A, double theta, const std::vector<uint8_t> &fixed) {
  const int64_t n = A.nbr;
  const int64_t bs = (int64_t)A.br * A.bc;
  std::vector<double> dnorm(n, 0.0);
  std::vector<double> fro(A.ci.size());
#pragma omp parallel for schedule(static)
  for (int64_t I = 0; I < n; ++I)
    for (int64_t a = A.rp[I]; a < A.rp[I + 1]; ++a) {
      double s = 0.0;
      for (int64_t e = 0; e < bs; ++e) s += A.v[a * bs + e] * A.v[a * bs + e];
      fro[a] = std::sqrt(s);
      if (A.ci[a] == I) dnorm[I] = fro[a];
    }
  std::vector<std::vector<int32_t>> adj(n);
  for (int64_t I = 0; I < n; ++I)
    for (int64_t a = A.rp[I]; a < A.rp[I + 1]; ++a) {
      const int32_t J = A.ci[a];
      if (J == I) continue;
      if (!fixed.empty() && (fixed[I] || fixed[J])) continue;
      if (fro[a] > theta * std::sqrt(dnorm[I] * dnorm[J])) {
        adj[I].push_back(J);
        adj[J].push_back((int32_t)I);
      }
    }
  Graph G;
  G.n = n;
  G.rp.assign(n + 1, 0);
  for (int64_t I = 0; I < n; ++I) {
    std::sort(adj[I].begin(), adj[I].end());
    adj[I].erase(std::unique(adj[I].begin(), adj[I].end()), adj[I].end());
    G.rp[I + 1] = G.rp[I] + (int64_t)adj[I].size();
  }
  G.ci.resize(G.rp[n]);
  for (int64_t I = 0; I < n; ++I) std::copy(adj[I].begin(), adj[I].end(), G.ci.begin() + G.rp[I]);
  return G;
}

void aggregate(const Graph &G, uint64_t seed, std::vector<int32_t> &agg, int64_t &nagg) {
  const int64_t n = G.n;
  std::vector<uint64_t> prio(n);
  for (int64_t i = 0; i < n; ++i) prio[i] = splitmix64_at(seed, (uint64_t)i);
  std::vector<int64_t> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    return prio[a] != prio[b] ? prio[a] > prio[b] : a < b;
  });
  std::vector<char> marked(n, 0);
  std::vector<int64_t> roots;
  for (int64_t I : order) {
    if (G.rp[I + 1] == G.rp[I] || marked[I]) continue;
    roots.push_back(I);
    marked[I] = 1;
    for (int64_t p = G.rp[I]; p < G.rp[I + 1]; ++p) {
      const int32_t K = G.ci[p];
      marked[K] = 1;
      for (int64_t q = G.rp[K]; q < G.rp[K + 1]; ++q) marked[G.ci[q]] = 1;
    }
  }
  std::sort(roots.begin(), roots.end());
  nagg = (int64_t)roots.size();
  agg.assign(n, -1);
  for (int64_t a = 0; a < nagg; ++a) agg[roots[a]] = (int32_t)a;
  for (int64_t a = 0; a < nagg; ++a) {
    const int64_t R = roots[a];
    for (int64_t p = G.rp[R]; p < G.rp[R + 1]; ++p) agg[G.ci[p]] = (int32_t)a;
  }
  std::vector<int32_t> agg2(agg);
  for (int64_t I = 0; I < n; ++I) {
    if (agg2[I] >= 0 || G.rp[I + 1] == G.rp[I]) continue;
    int32_t best = -1;
    for (int64_t p = G.rp[I]; p < G.rp[I + 1]; ++p) {
      const int32_t a = agg2[G.ci[p]];
      if (a < 0) continue;
      if (best < 0) {
        best = a;
        continue;
      }
      const int64_t ra = roots[a], rb = roots[best];
      if (prio[ra] > prio[rb] || (prio[ra] == prio[rb] && ra < rb)) best = a;
    }
    if (best < 0) throw SetupError(-7, "aggregation: node not within distance 2 of a root");
    agg[I] = best;
  }
}

double norm2(const std::vector<double> &v) {
  double s = 0.0;
  for (double x : v) s += x * x;
  return std::sqrt(s);
}

// Column-wise Gram-Schmidt, two passes, rank-dropping; Q m x k row-major.
void gs_qr(int m, int k, const std::vector<double> &B, std::vector<double> &Q, std::vector<double> &R) {
  Q.assign((size_t)m * k, 0.0);
  R.assign((size_t)k * k, 0.0);
  std::vector<double> v(m), h(k);
  for (int c = 0; c < k; ++c) {
    for (int r = 0; r < m; ++r) v[r] = B[(size_t)r * k + c];
    const double n0 = norm2(v);
    for (int pass = 0; pass < 2; ++pass) {
      for (int q = 0; q < c; ++q) {
        double s = 0.0;
        for (int r = 0; r < m; ++r) s += Q[(size_t)r * k + q] * v[r];
        h[q] = s;
      }
      for (int r = 0; r < m; ++r) {
        double s = 0.0;
        for (int q = 0; q < c; ++q) s += Q[(size_t)r * k + q] * h[q];
        v[r] -= s;
      }
      for (int q = 0; q < c; ++q) R[(size_t)q * k + c] += h[q];
    }
    const double nv = norm2(v);
    if (nv > 1e-10 * n0 && nv > 0.0) {
      for (int r = 0; r < m; ++r) Q[(size_t)r * k + c] = v[r] / nv;
      R[(size_t)c * k + c] = nv;
    }
  }
}

int nullspace_dim(const FieldInfo &f) {
  if (f.ns == 0) return f.b;
  if (f.ns == 2) return f.ns_dim;
  return f.dim == 2 ? 3 : 6;
}

// Tentative prolongator (b x k blocks) and coarse nullspace (nagg*k x k).
void tentative(const std::vector<int32_t> &agg, int64_t nagg, int b, int k, bool fine,
               const FieldInfo &f, const std::vector<double> &B, HBsr &P, std::vector<double> &Bc) {
  const int64_t n = (int64_t)agg.size();
  std::vector<int64_t> start(nagg + 1, 0);
  for (int32_t a : agg)
    if (a >= 0) start[a + 1]++;
  for (int64_t a = 0; a < nagg; ++a) start[a + 1] += start[a];
  std::vector<int64_t> members(start[nagg]);
  {
    std::vector<int64_t> pos(start.begin(), start.end() - 1);
    for (int64_t I = 0; I < n; ++I)
      if (agg[I] >= 0) members[pos[agg[I]]++] = I;  // ascending node index
  }
  P = HBsr();
  P.br = b;
  P.bc = k;
  P.nbr = n;
  P.nbc = nagg;
  P.rp.assign(n + 1, 0);
  for (int64_t I = 0; I < n; ++I) P.rp[I + 1] = P.rp[I] + (agg[I] >= 0 ? 1 : 0);
  P.ci.resize(P.rp[n]);
  P.v.assign(P.rp[n] * b * k, 0.0);
  Bc.assign((size_t)nagg * k * k, 0.0);
  bool fail = false;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t a = 0; a < nagg; ++a) {
    const int64_t m0 = start[a], cnt = start[a + 1] - start[a];
    const int m = (int)(cnt * b);
    std::vector<double> Ba((size_t)m * k, 0.0), Q, R;
    if (fine && f.ns == 0) {
      for (int64_t t = 0; t < cnt; ++t)
        for (int c = 0; c < b; ++c) Ba[(size_t)(t * b + c) * k + c] = 1.0;
    } else if (fine && f.ns == 2) {
      for (int64_t t = 0; t < cnt; ++t)
        for (int c = 0; c < b; ++c)
          for (int q = 0; q < k; ++q)
            Ba[(size_t)(t * b + c) * k + q] = f.user_B[(size_t)(members[m0 + t] * b + c) * k + q];
    } else if (fine) {
      const int d = f.dim;
      double cen[3] = {0, 0, 0};
      for (int64_t t = 0; t < cnt; ++t)
        for (int e = 0; e < d; ++e) cen[e] += f.coords[members[m0 + t] * d + e];
      for (int e = 0; e < d; ++e) cen[e] /= (double)cnt;
      for (int64_t t = 0; t < cnt; ++t) {
        const double *xc = &f.coords[members[m0 + t] * d];
        const double x = xc[0] - cen[0], y = xc[1] - cen[1], z = d == 3 ? xc[2] - cen[2] : 0.0;
        double *r0 = &Ba[(size_t)(t * b) * k];
        if (d == 2) {  // rows: ux, uy; cols: tx, ty, rot
          r0[0] = 1.0;
          r0[2] = -y;
          r0[k + 1] = 1.0;
          r0[k + 2] = x;
        } else {  // rows: ux, uy, uz; cols: tx, ty, tz, rx, ry, rz
          double *r1 = r0 + k, *r2 = r0 + 2 * k;
          r0[0] = 1.0;
          r1[1] = 1.0;
          r2[2] = 1.0;
          r1[3] = -z;
          r2[3] = y;
          r0[4] = z;
          r2[4] = -x;
          r0[5] = -y;
          r1[5] = x;
        }
      }
    } else {
      for (int64_t t = 0; t < cnt; ++t)
        for (int c = 0; c < b; ++c)
          for (int q = 0; q < k; ++q)
            Ba[(size_t)(t * b + c) * k + q] = B[(size_t)(members[m0 + t] * b + c) * k + q];
    }
    if (fine && !f.dirichlet.empty())  // no nullspace component at a Dirichlet dof
      for (int64_t t = 0; t < cnt; ++t)
        for (int c = 0; c < b; ++c)
          if (f.dirichlet[(size_t)members[m0 + t] * b + c])
            for (int q = 0; q < k; ++q) Ba[(size_t)(t * b + c) * k + q] = 0.0;
    gs_qr(m, k, Ba, Q, R);
    for (int64_t t = 0; t < cnt; ++t) {
      const int64_t I = members[m0 + t];
      const int64_t p = P.rp[I];
      P.ci[p] = (int32_t)a;
      double *blk = P.v.data() + p * b * k;
      for (int c = 0; c < b; ++c)
        for (int q = 0; q < k; ++q) blk[c * k + q] = Q[(size_t)(t * b + c) * k + q];
    }
    for (int r = 0; r < k; ++r)
      for (int q = 0; q < k; ++q) Bc[(size_t)(a * k + r) * k + q] = R[(size_t)r * k + q];
  }
  if (fail) throw SetupError(-7, "tentative prolongator failed");
}

double power_lambda(const HBsr &A, const std::vector<double> &dinv, uint64_t seed) {
  const int64_t n = A.nrows();
  std::vector<double> v(n), w(n);
  for (int64_t i = 0; i < n; ++i) v[i] = uniform01_at(seed, (uint64_t)i);
  double nv = norm2(v);
  for (auto &x : v) x /= nv;
  double lam = 0.0;
  for (int it = 0; it < 10; ++it) {
    bsr_matvec(A, v.data(), w.data());
    for (int64_t i = 0; i < n; ++i) w[i] *= dinv[i];
    lam = norm2(w);
    for (int64_t i = 0; i < n; ++i) v[i] = w[i] / lam;
  }
  return lam;
}

void fill_dinv(HLevelField &fl) {
  fl.dinv = bsr_point_diagonal(fl.A);
  for (double &d : fl.dinv) {
    if (d == 0.0) throw SetupError(-4, "zero diagonal entry in a diagonal block");
    d = 1.0 / d;
  }
}

}  // namespace

double amg_power_lambda(const HBsr &A, const std::vector<double> &dinv, uint64_t seed) {
  return power_lambda(A, dinv, seed);
}

std::vector<double> amg_dinv(const HBsr &A) {
  HLevelField f;
  f.A = A;
  fill_dinv(f);
  return f.dinv;
}

// Row damping parameters of the Petrov-Galerkin smoothing of Pt by A (see
// pg_transfers); returns Q = D^-1 A Pt scaled by them (row i times omega_i).
static HBsr pg_damped(const HBsr &A, const std::vector<double> &dinv, const HBsr &Pt) {
  HBsr Q = bsr_spgemm(A, Pt);
  bsr_scale_rows(Q, dinv);
  const HBsr AQ = bsr_spgemm(A, Q);
  const int br = Q.br, bc = Q.bc;
  const int64_t nc = Q.ncols();
  std::vector<double> num(nc, 0.0), den(nc, 0.0);
  double qmax = 0.0;
  for (double v : Q.v) qmax = std::max(qmax, std::fabs(v));
  // column sums in row order: <A q_j, q_j> over Q's blocks, <A q_j, D^-1 A q_j> over AQ's
  for (int64_t I = 0; I < AQ.nbr; ++I) {
    int64_t q = Q.rp[I];
    for (int64_t a = AQ.rp[I]; a < AQ.rp[I + 1]; ++a) {
      const int64_t J = AQ.ci[a];
      const double *w = AQ.blk(a);
      while (q < Q.rp[I + 1] && Q.ci[q] < J) ++q;
      const bool inq = q < Q.rp[I + 1] && Q.ci[q] == J;
      for (int r = 0; r < br; ++r)
        for (int c = 0; c < bc; ++c) {
          const double x = w[r * bc + c];
          den[J * bc + c] += x * x * dinv[I * br + r];
          if (inq) num[J * bc + c] += x * Q.blk(q)[r * bc + c];
        }
    }
  }
  std::vector<double> wcol(nc, 0.0);
  for (int64_t j = 0; j < nc; ++j)
    if (den[j] > 0.0 && num[j] > 0.0) wcol[j] = num[j] / den[j];
  const double thr = 1e-12 * qmax;
  std::vector<double> wrow(Q.nrows(), 0.0);
  for (int64_t I = 0; I < Q.nbr; ++I)
    for (int r = 0; r < br; ++r) {
      double m = 0.0;
      bool any = false;
      for (int64_t a = Q.rp[I]; a < Q.rp[I + 1]; ++a)
        for (int c = 0; c < bc; ++c)
          if (std::fabs(Q.blk(a)[r * bc + c]) > thr) {
            const double wc = wcol[(int64_t)Q.ci[a] * bc + c];
            m = any ? std::min(m, wc) : wc;
            any = true;
          }
      wrow[I * br + r] = any ? m : 0.0;
    }
  bsr_scale_rows(Q, wrow);
  return Q;
}

void pg_transfers(const HBsr &A, const std::vector<double> &dinv, const HBsr &Pt, HBsr &P, HBsr &R) {
  P = bsr_axpby(1.0, Pt, -1.0, pg_damped(A, dinv, Pt));
  const HBsr At = bsr_transpose(A);
  R = bsr_transpose(bsr_axpby(1.0, Pt, -1.0, pg_damped(At, dinv, Pt)));
}

std::vector<int32_t> node_colors(const HBsr &A) {
  const int64_t n = A.nbr;
  const int bs = A.br * A.bc;
  std::vector<double> rowmax(n, 0.0);
  for (int64_t I = 0; I < n; ++I)
    for (int64_t a = A.rp[I]; a < A.rp[I + 1]; ++a)
      for (int e = 0; e < bs; ++e) rowmax[I] = std::max(rowmax[I], std::fabs(A.v[a * bs + e]));
  // coupling edges, both directions
  std::vector<std::vector<int64_t>> nbr(n);
  for (int64_t I = 0; I < n; ++I)
    for (int64_t a = A.rp[I]; a < A.rp[I + 1]; ++a) {
      const int64_t J = A.ci[a];
      if (J == I) continue;
      double m = 0.0;
      for (int e = 0; e < bs; ++e) m = std::max(m, std::fabs(A.v[a * bs + e]));
      if (m > 1e-12 * rowmax[I]) {
        nbr[I].push_back(J);
        nbr[J].push_back(I);
      }
    }
  std::vector<int32_t> color(n, -1);
  std::vector<int64_t> mark;  // mark[c] == i: colour c is taken for node i
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j : nbr[i])
      if (j < i) {
        const int32_t c = color[j];
        if ((int64_t)mark.size() <= c) mark.resize(c + 1, -1);
        mark[c] = i;
      }
    int32_t c = 0;
    while (c < (int32_t)mark.size() && mark[c] == i) ++c;
    color[i] = c;
  }
  return color;
}

std::vector<double> bsr_to_dense(const HBsr &A) {
  const int64_t nr = A.nrows(), nc = A.ncols();
  std::vector<double> D((size_t)(nr * nc), 0.0);
  for (int64_t I = 0; I < A.nbr; ++I)
    for (int64_t a = A.rp[I]; a < A.rp[I + 1]; ++a)
      for (int r = 0; r < A.br; ++r)
        for (int c = 0; c < A.bc; ++c)
          D[(size_t)((I * A.br + r) * nc + (int64_t)A.ci[a] * A.bc + c)] += A.blk(a)[r * A.bc + c];
  return D;
}

HDenseLU dense_lu(int n, std::vector<double> a) {
  HDenseLU out;
  out.n = n;
  out.perm.resize(n);
  std::iota(out.perm.begin(), out.perm.end(), 0);
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::fabs(a[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(a[(size_t)i * n + k]) > best) {
        best = std::fabs(a[(size_t)i * n + k]);
        p = i;
      }
    if (!(best > 0.0) || !std::isfinite(best)) throw SetupError(-4, "singular coarsest matrix");
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(a[(size_t)k * n + j], a[(size_t)p * n + j]);
      std::swap(out.perm[k], out.perm[p]);
    }
    const double piv = a[(size_t)k * n + k];
    for (int i = k + 1; i < n; ++i) {
      const double l = a[(size_t)i * n + k] / piv;
      a[(size_t)i * n + k] = l;
      if (l != 0.0)
        for (int j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= l * a[(size_t)k * n + j];
    }
  }
  out.lu.resize((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) out.lu[(size_t)j * n + i] = a[(size_t)i * n + j];
  return out;
}

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

void build_group(HGroup &g, const std::vector<HBsr> &diag, const std::vector<FieldInfo> &info,
                 int max_levels, int64_t coarse_max, uint64_t seed, bool want_off,
                 const BlockMap *fine_off, int verbose) {
  double tm[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // power, strength, aggregate, tentative, AP, RAP, off, LU
  g.nf = (int)diag.size();
  g.info = info;
  g.lv.assign(1, std::vector<HLevelField>(g.nf));
  for (int i = 0; i < g.nf; ++i) {
    g.lv[0][i].A = diag[i];
    fill_dinv(g.lv[0][i]);
  }
  g.off.assign(1, BlockMap());
  if (want_off && fine_off) g.off[0] = *fine_off;
  auto total = [&](int l) {
    int64_t s = 0;
    for (auto &fl : g.lv[l]) s += fl.A.nrows();
    return s;
  };
  while ((int)g.lv.size() < max_levels && total((int)g.lv.size() - 1) > coarse_max) {
    const int l = (int)g.lv.size() - 1;
    const bool fine = l == 0;
    std::vector<HLevelField> nxt(g.nf);
    for (int i = 0; i < g.nf; ++i) {
      HLevelField &fl = g.lv[l][i];
      const FieldInfo &f = info[i];
      double t = now_s();
      fl.lam = power_lambda(fl.A, fl.dinv, seed);
      tm[0] += now_s() - t;
      t = now_s();
      Graph G = strength_graph(fl.A, f.theta, fine ? f.fixed_nodes() : std::vector<uint8_t>());
      tm[1] += now_s() - t;
      t = now_s();
      aggregate(G, seed, fl.agg, fl.nagg);
      tm[2] += now_s() - t;
      if (fl.nagg == 0) throw SetupError(-7, "aggregation produced no aggregate");
      const int k = fine ? nullspace_dim(f) : fl.A.br;
      HBsr Pt;
      std::vector<double> Bc;
      t = now_s();
      tentative(fl.agg, fl.nagg, fl.A.br, k, fine, f, fl.B, Pt, Bc);
      tm[3] += now_s() - t;
      t = now_s();
      if (f.pg) {
        pg_transfers(fl.A, fl.dinv, Pt, fl.P, fl.R);
      } else {
        HBsr DAP = bsr_spgemm(fl.A, Pt);
        bsr_scale_rows(DAP, fl.dinv);
        const double omega = 4.0 / (3.0 * fl.lam);
        fl.P = bsr_axpby(1.0, Pt, -omega, DAP);
        fl.R = bsr_transpose(fl.P);
      }
      tm[4] += now_s() - t;
      t = now_s();
      nxt[i].A = bsr_spgemm(fl.R, bsr_spgemm(fl.A, fl.P));
      tm[5] += now_s() - t;
      nxt[i].B = std::move(Bc);
      fill_dinv(nxt[i]);
    }
    if (want_off) {
      const double t = now_s();
      BlockMap noff;
      for (auto &kv : g.off[l]) {
        const int i = kv.first.first, j = kv.first.second;
        noff[kv.first] = bsr_spgemm(g.lv[l][i].R, bsr_spgemm(kv.second, g.lv[l][j].P));
      }
      g.off.push_back(std::move(noff));
      tm[6] += now_s() - t;
    }
    g.lv.push_back(std::move(nxt));
  }
  // coarsest-level direct solvers
  const double tlu = now_s();
  const int L = (int)g.lv.size() - 1;
  g.coarse_field.resize(g.nf);
  for (int i = 0; i < g.nf; ++i) {
    const HBsr &A = g.lv[L][i].A;
    g.coarse_field[i] = dense_lu((int)A.nrows(), bsr_to_dense(A));
  }
  if (want_off) {
    std::vector<int64_t> off(g.nf + 1, 0);
    for (int i = 0; i < g.nf; ++i) off[i + 1] = off[i] + g.lv[L][i].A.nrows();
    const int64_t n = off[g.nf];
    std::vector<double> D((size_t)(n * n), 0.0);
    auto put = [&](const HBsr &A, int i, int j) {
      std::vector<double> d = bsr_to_dense(A);
      const int64_t nr = A.nrows(), nc = A.ncols();
      for (int64_t r = 0; r < nr; ++r)
        for (int64_t c = 0; c < nc; ++c) D[(size_t)((off[i] + r) * n + off[j] + c)] += d[r * nc + c];
    };
    for (int i = 0; i < g.nf; ++i) put(g.lv[L][i].A, i, i);
    for (auto &kv : g.off[L]) put(kv.second, kv.first.first, kv.first.second);
    g.coarse_coupled = dense_lu((int)n, std::move(D));
  }
  tm[7] += now_s() - tlu;
  if (verbose)
    std::fprintf(stderr,
                 "mfs setup group (%d fields, %d levels): power %.3f strength %.3f aggregate %.3f tentative %.3f "
                 "smooth+transpose %.3f RAP %.3f offdiag %.3f LU %.3f s\n",
                 g.nf, (int)g.lv.size(), tm[0], tm[1], tm[2], tm[3], tm[4], tm[5], tm[6], tm[7]);
}

}  // namespace mfs
