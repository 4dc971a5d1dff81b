// Smoothed-aggregation setup on the GPU.  Same steps and definitions as the
// host setup (amg_setup.h); every accumulation runs in a fixed order, so the
// result does not depend on scheduling.
//
//  * strength graph: Frobenius norms of node blocks, symmetrised by a
//    transpose + sorted union;
//  * aggregation: the lexicographically-first distance-2 maximal independent
//    set, found in parallel rounds (a node joins when it is the best
//    undecided node within distance two; nodes within distance two of a
//    root drop out), which equals the greedy rule in decreasing priority;
//    then the two joining phases;
//  * tentative prolongator: one warp per aggregate, two-pass Gram-Schmidt;
//  * lambda_max: 10 power iterations; smoothing, transpose and Galerkin
//    products with a warp-per-row block SpGEMM (hash set for the pattern,
//    then a sequential sweep over the row's products for the values).
#include "setup_gpu.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <string>
#include <utility>

namespace mfs {

namespace {

#define GS_CUDA(call)                                                                            \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      throw SetupError(e_ == cudaErrorMemoryAllocation ? -3 : -2,                                \
                       std::string("GPU setup: ") + #call + ": " + cudaGetErrorString(e_));      \
  } while (0)

constexpr int kT = 256;

// Every GPU-setup launch, copy and allocation goes to this thread's private
// non-blocking stream (stream-ordered allocation), so a setup never touches
// the legacy stream or synchronises the device while other threads replay
// or capture solve graphs.
thread_local cudaStream_t tls_stream = nullptr;
inline cudaStream_t gstream() { return tls_stream; }

struct StreamScope {
  cudaStream_t prev;
  cudaStream_t s = nullptr;
  StreamScope() : prev(tls_stream) {
    GS_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    tls_stream = s;
  }
  ~StreamScope() {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    tls_stream = prev;
  }
};

inline void sync() { GS_CUDA(cudaStreamSynchronize(gstream())); }

inline unsigned nblocks(int64_t n, int t = kT) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

template <typename T> struct DVec {
  T *p = nullptr;
  int64_t n = 0;
  DVec() = default;
  explicit DVec(int64_t m, bool zero = false) { resize(m, zero); }
  DVec(const DVec &) = delete;
  DVec &operator=(const DVec &) = delete;
  DVec(DVec &&o) noexcept : p(o.p), n(o.n) { o.p = nullptr, o.n = 0; }
  DVec &operator=(DVec &&o) noexcept {
    std::swap(p, o.p);
    std::swap(n, o.n);
    return *this;
  }
  ~DVec() {
    if (p) cudaFreeAsync(p, gstream());
  }
  void resize(int64_t m, bool zero = false) {
    if (p) cudaFreeAsync(p, gstream());
    p = nullptr;
    n = m;
    if (m > 0) {
      GS_CUDA(cudaMallocAsync((void **)&p, (size_t)m * sizeof(T), gstream()));
      if (zero) GS_CUDA(cudaMemsetAsync(p, 0, (size_t)m * sizeof(T), gstream()));
    }
  }
  void upload(const T *h, int64_t m) {
    resize(m);
    if (m) GS_CUDA(cudaMemcpyAsync(p, h, (size_t)m * sizeof(T), cudaMemcpyHostToDevice, gstream()));
    sync();
  }
  std::vector<T> download() const {
    std::vector<T> h(n);
    if (n) GS_CUDA(cudaMemcpyAsync(h.data(), p, (size_t)n * sizeof(T), cudaMemcpyDeviceToHost, gstream()));
    sync();
    return h;
  }
};

// Device block-CSR (int32 offsets).
struct DB {
  int br = 0, bc = 0;
  int64_t nbr = 0, nbc = 0, nnzb = 0;
  DVec<int32_t> rp, ci;
  DVec<double> v;
  void shape(int r, int c, int64_t nr, int64_t nc) {
    br = r, bc = c, nbr = nr, nbc = nc;
    rp.resize(nr + 1, true);
  }
};

// raw view passed to kernels
struct BV {
  int br, bc;
  int64_t nbr, nbc;
  const int32_t *rp, *ci;
  const double *v;
};
BV view(const DB &A) { return BV{A.br, A.bc, A.nbr, A.nbc, A.rp.p, A.ci.p, A.v.p}; }

DB upload(const HBsr &H) {
  DB A;
  if (H.nnzb() > INT32_MAX) throw SetupError(-1, "GPU setup: matrix too large for 32-bit offsets");
  A.br = H.br, A.bc = H.bc, A.nbr = H.nbr, A.nbc = H.nbc, A.nnzb = H.nnzb();
  std::vector<int32_t> rp(H.rp.begin(), H.rp.end());
  A.rp.upload(rp.data(), (int64_t)rp.size());
  A.ci.upload(H.ci.data(), (int64_t)H.ci.size());
  A.v.upload(H.v.data(), (int64_t)H.v.size());
  return A;
}

HBsr download(const DB &A) {
  HBsr H;
  H.br = A.br, H.bc = A.bc, H.nbr = A.nbr, H.nbc = A.nbc;
  std::vector<int32_t> rp = A.rp.download();
  H.rp.assign(rp.begin(), rp.end());
  if (H.rp.empty()) H.rp.assign(A.nbr + 1, 0);
  H.ci = A.ci.download();
  H.v = A.v.download();
  return H;
}

// ---------------------------------------------------------------- scan ---
__global__ void k_scan_add(int64_t *__restrict__ out, int64_t n, const int64_t *__restrict__ offs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += offs[blockIdx.x];
}

__global__ void k_to_i32(const int64_t *__restrict__ in, int32_t *__restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (int32_t)in[i];
}

// exclusive prefix of the int64 array `in` (length n) into out (length n)
void scan64(const int64_t *in, int64_t n, int64_t *out);

__global__ void k_widen(const int32_t *__restrict__ in, int64_t *__restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[i];
}

__global__ void k_scan_block64(const int64_t *__restrict__ in, int64_t n, int64_t *__restrict__ out,
                               int64_t *__restrict__ sums) {
  __shared__ int64_t ws[32];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t v = i < n ? in[i] : 0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int64_t s = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    ws[lane] = s;
  }
  __syncthreads();
  const int64_t incl = x + (w > 0 ? ws[w - 1] : 0);
  if (i < n) out[i] = incl - v;
  if (threadIdx.x == blockDim.x - 1) sums[blockIdx.x] = incl;
}

void scan64(const int64_t *in, int64_t n, int64_t *out) {
  if (n <= 0) return;
  const int t = 1024;
  const int64_t nb = (n + t - 1) / t;
  DVec<int64_t> sums(nb), offs(nb);
  k_scan_block64<<<(unsigned)nb, t, 0, gstream()>>>(in, n, out, sums.p);
  if (nb > 1) {
    scan64(sums.p, nb, offs.p);
    k_scan_add<<<(unsigned)nb, t, 0, gstream()>>>(out, n, offs.p);
  }
  GS_CUDA(cudaGetLastError());
}

// counts (int32, n entries) -> row pointer (int32, n + 1 entries); returns the total
int64_t counts_to_rowptr(const int32_t *cnt, int64_t n, int32_t *rp) {
  DVec<int64_t> w(n + 1, true), o(n + 1);
  if (n) k_widen<<<nblocks(n), kT, 0, gstream()>>>(cnt, w.p, n);
  scan64(w.p, n + 1, o.p);
  int64_t total = 0;
  GS_CUDA(cudaMemcpyAsync(&total, o.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, gstream()));
  sync();
  if (total > INT32_MAX) throw SetupError(-1, "GPU setup: product too large for 32-bit offsets");
  k_to_i32<<<nblocks(n + 1), kT, 0, gstream()>>>(o.p, rp, n + 1);
  GS_CUDA(cudaGetLastError());
  return total;
}

// ----------------------------------------------------------- reductions ---
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void k_sumsq_partial(const double *__restrict__ x, int64_t n, double *__restrict__ part) {
  __shared__ double ws[32];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += x[i] * x[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
  }
}

__global__ void k_final_sqrt(const double *__restrict__ part, int np, double *__restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < np; ++i) s += part[i];
    *out = sqrt(s);
  }
}

// --------------------------------------------------------------- basics ---
__device__ __forceinline__ uint64_t sm64(uint64_t s, uint64_t i) {
  uint64_t z = s + (i + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__global__ void k_uniform(double *__restrict__ v, int64_t n, uint64_t seed) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = (double)(sm64(seed, (uint64_t)i) >> 11) * 0x1.0p-53;
}

__global__ void k_scale_by(double *__restrict__ v, int64_t n, const double *__restrict__ s) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = v[i] / *s;
}

__global__ void k_div_into(const double *__restrict__ w, double *__restrict__ v, int64_t n, const double *__restrict__ s) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = w[i] / *s;
}

// y = dinv .* (A x), one thread per block row
__global__ void k_dinv_spmv(BV A, const double *__restrict__ x, const double *__restrict__ dinv, double *__restrict__ y) {
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= A.nbr) return;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  const int bs = A.br * A.bc;
  for (int a = A.rp[I]; a < A.rp[I + 1]; ++a) {
    const double *blk = A.v + (int64_t)a * bs;
    const double *xv = x + (int64_t)A.ci[a] * A.bc;
    for (int r = 0; r < A.br; ++r)
      for (int c = 0; c < A.bc; ++c) acc[r] += blk[r * A.bc + c] * xv[c];
  }
  for (int r = 0; r < A.br; ++r) y[I * A.br + r] = dinv[I * A.br + r] * acc[r];
}

__global__ void k_diag_inv(BV A, double *__restrict__ dinv, int *__restrict__ bad) {
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= A.nbr) return;
  const int bs = A.br * A.bc;
  double d[6] = {0, 0, 0, 0, 0, 0};
  for (int a = A.rp[I]; a < A.rp[I + 1]; ++a)
    if (A.ci[a] == I)
      for (int r = 0; r < A.br; ++r) d[r] = A.v[(int64_t)a * bs + r * A.bc + r];
  for (int r = 0; r < A.br; ++r) {
    if (d[r] == 0.0) atomicOr(bad, 1);
    dinv[I * A.br + r] = d[r] == 0.0 ? 0.0 : 1.0 / d[r];
  }
}

__global__ void k_scale_rows(double *__restrict__ v, const int32_t *__restrict__ rp, int64_t nbr, int br, int bc,
                             const double *__restrict__ d) {
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nbr) return;
  for (int a = rp[I]; a < rp[I + 1]; ++a)
    for (int r = 0; r < br; ++r)
      for (int c = 0; c < bc; ++c) v[((int64_t)a * br + r) * bc + c] *= d[I * br + r];
}

double power_lambda_gpu(const DB &A, const double *dinv, uint64_t seed) {
  const int64_t n = A.nbr * A.br;
  DVec<double> v(n), w(n), part(256), nrm(1);
  k_uniform<<<nblocks(n), kT, 0, gstream()>>>(v.p, n, seed);
  k_sumsq_partial<<<256, kT, 0, gstream()>>>(v.p, n, part.p);
  k_final_sqrt<<<1, 32, 0, gstream()>>>(part.p, 256, nrm.p);
  k_scale_by<<<nblocks(n), kT, 0, gstream()>>>(v.p, n, nrm.p);
  for (int it = 0; it < 10; ++it) {
    k_dinv_spmv<<<nblocks(A.nbr), kT, 0, gstream()>>>(view(A), v.p, dinv, w.p);
    k_sumsq_partial<<<256, kT, 0, gstream()>>>(w.p, n, part.p);
    k_final_sqrt<<<1, 32, 0, gstream()>>>(part.p, 256, nrm.p);
    k_div_into<<<nblocks(n), kT, 0, gstream()>>>(w.p, v.p, n, nrm.p);
  }
  GS_CUDA(cudaGetLastError());
  double lam = 0.0;
  GS_CUDA(cudaMemcpyAsync(&lam, nrm.p, sizeof(double), cudaMemcpyDeviceToHost, gstream()));
  sync();
  return lam;
}

// ---------------------------------------------------------- warp sort ---
// Sort keys[0..m) (and vals, if given) ascending in place; m <= cap, cap a
// power of two; one warp, shared-memory arrays of length cap.
__device__ void warp_bitonic(int *keys, int *vals, int m, int cap) {
  const int lane = threadIdx.x & 31;
  int P = 1;
  while (P < m) P <<= 1;
  for (int i = m + lane; i < P; i += 32) {
    keys[i] = INT32_MAX;
    if (vals) vals[i] = -1;
  }
  __syncwarp();
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < P; i += 32) {
        const int l = i ^ j;
        if (l > i) {
          const bool up = (i & k) == 0;
          const int a = keys[i], b = keys[l];
          if ((a > b) == up) {
            keys[i] = b;
            keys[l] = a;
            if (vals) {
              const int t = vals[i];
              vals[i] = vals[l];
              vals[l] = t;
            }
          }
        }
      }
      __syncwarp();
    }
}

// --------------------------------------------------------------- SpGEMM ---
constexpr int kHash = 2048;  // hash slots per warp
constexpr int kCap = 1024;   // distinct columns per output row handled on the GPU
constexpr int kWarpsSp = 4;

__device__ __forceinline__ int hash_insert(int *h, int key, int *ovf) {
  int slot = (int)(((unsigned)key * 2654435761u) & (kHash - 1));
  for (int probe = 0; probe < kHash; ++probe) {
    const int prev = atomicCAS(&h[slot], -1, key);
    if (prev == -1) return 1;
    if (prev == key) return 0;
    slot = (slot + 1) & (kHash - 1);
  }
  atomicOr(ovf, 1);
  return 0;
}

__global__ void k_spgemm_count(BV A, BV B, int32_t *__restrict__ cnt, int *__restrict__ ovf) {
  __shared__ int hs[kWarpsSp * kHash];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t I = (int64_t)blockIdx.x * kWarpsSp + warp;
  if (I >= A.nbr) return;
  int *h = hs + warp * kHash;
  for (int i = lane; i < kHash; i += 32) h[i] = -1;
  __syncwarp();
  int c = 0;
  for (int a = A.rp[I]; a < A.rp[I + 1]; ++a) {
    const int K = A.ci[a];
    for (int q = B.rp[K] + lane; q < B.rp[K + 1]; q += 32) c += hash_insert(h, B.ci[q], ovf);
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) {
    cnt[I] = c;
    if (c > kCap) atomicOr(ovf, 1);
  }
}

__global__ void k_spgemm_fill(BV A, BV B, const int32_t *__restrict__ crp, int32_t *__restrict__ cci,
                              double *__restrict__ cv, int *__restrict__ ovf) {
  __shared__ int hs[kWarpsSp * kHash];
  __shared__ int cs[kWarpsSp * kCap];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t I = (int64_t)blockIdx.x * kWarpsSp + warp;
  if (I >= A.nbr) return;
  int *h = hs + warp * kHash;
  int *cols = cs + warp * kCap;
  for (int i = lane; i < kHash; i += 32) h[i] = -1;
  __syncwarp();
  for (int a = A.rp[I]; a < A.rp[I + 1]; ++a) {
    const int K = A.ci[a];
    for (int q = B.rp[K] + lane; q < B.rp[K + 1]; q += 32) hash_insert(h, B.ci[q], ovf);
  }
  __syncwarp();
  // compact the set into cols (order of slots), then sort
  int m = 0;
  for (int base = 0; base < kHash; base += 32) {
    const int key = h[base + lane];
    const unsigned bal = __ballot_sync(0xffffffffu, key >= 0);
    const int pos = m + __popc(bal & ((1u << lane) - 1));
    if (key >= 0 && pos < kCap) cols[pos] = key;
    m += __popc(bal);
  }
  __syncwarp();
  if (m > kCap) return;  // flagged by the count pass; the caller falls back
  warp_bitonic(cols, nullptr, m, kCap);
  const int64_t r0 = crp[I];
  for (int p = lane; p < m; p += 32) cci[r0 + p] = cols[p];
  const int ob = A.br * B.bc;
  for (int64_t e = lane; e < (int64_t)m * ob; e += 32) cv[r0 * ob + e] = 0.0;
  __syncwarp();
  // values: every product in (a, q) order; lane e owns output entry e of a block
  for (int a = A.rp[I]; a < A.rp[I + 1]; ++a) {
    const int K = A.ci[a];
    const double *ab = A.v + (int64_t)a * A.br * A.bc;
    for (int q = B.rp[K]; q < B.rp[K + 1]; ++q) {
      const int j = B.ci[q];
      int lo = 0, hi = m - 1;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cols[mid] < j) lo = mid + 1;
        else hi = mid;
      }
      const double *bb = B.v + (int64_t)q * B.br * B.bc;
      double *cb = cv + (r0 + lo) * ob;
      for (int e = lane; e < ob; e += 32) {
        const int r = e / B.bc, c = e % B.bc;
        double s = 0.0;
        for (int t = 0; t < A.bc; ++t) s += ab[r * A.bc + t] * bb[t * B.bc + c];
        cb[e] += s;
      }
    }
  }
}

DB spgemm(const DB &A, const DB &B) {
  if (A.bc != B.br || A.nbc != B.nbr) throw SetupError(-1, "GPU setup: spgemm shape mismatch");
  DB C;
  C.shape(A.br, B.bc, A.nbr, B.nbc);
  if (A.nbr == 0) return C;
  DVec<int32_t> cnt(A.nbr, true);
  DVec<int> ovf(1, true);
  const unsigned g = (unsigned)((A.nbr + kWarpsSp - 1) / kWarpsSp);
  k_spgemm_count<<<g, 32 * kWarpsSp, 0, gstream()>>>(view(A), view(B), cnt.p, ovf.p);
  GS_CUDA(cudaGetLastError());
  int o = 0;
  GS_CUDA(cudaMemcpyAsync(&o, ovf.p, sizeof(int), cudaMemcpyDeviceToHost, gstream()));
  sync();
  if (o) {  // a row with more than kCap distinct columns: do this product on the host
    C = upload(bsr_spgemm(download(A), download(B)));
    return C;
  }
  C.nnzb = counts_to_rowptr(cnt.p, A.nbr, C.rp.p);
  C.ci.resize(C.nnzb);
  C.v.resize(C.nnzb * C.br * C.bc);
  k_spgemm_fill<<<g, 32 * kWarpsSp, 0, gstream()>>>(view(A), view(B), C.rp.p, C.ci.p, C.v.p, ovf.p);
  GS_CUDA(cudaGetLastError());
  return C;
}

// ------------------------------------------------------------ transpose ---
__global__ void k_col_count(const int32_t *__restrict__ ci, int64_t nnz, int32_t *__restrict__ cnt) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a < nnz) atomicAdd(&cnt[ci[a]], 1);
}

__global__ void k_t_scatter(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int64_t nbr,
                            const int32_t *__restrict__ trp, int32_t *__restrict__ fill, int32_t *__restrict__ trow,
                            int32_t *__restrict__ tsrc) {
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nbr) return;
  for (int a = rp[I]; a < rp[I + 1]; ++a) {
    const int j = ci[a];
    const int p = trp[j] + atomicAdd(&fill[j], 1);
    trow[p] = (int32_t)I;
    tsrc[p] = a;
  }
}

constexpr int kTCap = 2048;
constexpr int kWarpsT = 2;

// sort each transposed row by source row (warp per row); rows longer than kTCap flag
__global__ void k_t_sort(const int32_t *__restrict__ trp, int64_t n, int32_t *__restrict__ trow,
                         int32_t *__restrict__ tsrc, int *__restrict__ ovf) {
  __shared__ int ks[kWarpsT * kTCap], vs[kWarpsT * kTCap];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t j = (int64_t)blockIdx.x * kWarpsT + warp;
  if (j >= n) return;
  const int lo = trp[j], m = trp[j + 1] - lo;
  if (m > kTCap) {
    if (lane == 0) atomicOr(ovf, 1);
    return;
  }
  int *k = ks + warp * kTCap, *v = vs + warp * kTCap;
  for (int i = lane; i < m; i += 32) {
    k[i] = trow[lo + i];
    v[i] = tsrc[lo + i];
  }
  __syncwarp();
  warp_bitonic(k, v, m, kTCap);
  for (int i = lane; i < m; i += 32) {
    trow[lo + i] = k[i];
    tsrc[lo + i] = v[i];
  }
}

__global__ void k_t_values(const double *__restrict__ v, const int32_t *__restrict__ tsrc, int64_t nnz, int br, int bc,
                           double *__restrict__ tv) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nnz) return;
  const double *s = v + (int64_t)tsrc[p] * br * bc;
  double *d = tv + p * br * bc;
  for (int r = 0; r < br; ++r)
    for (int c = 0; c < bc; ++c) d[c * br + r] = s[r * bc + c];
}

DB transpose(const DB &A, bool values = true) {
  DB T;
  T.shape(A.bc, A.br, A.nbc, A.nbr);
  T.nnzb = A.nnzb;
  if (A.nbc == 0) return T;
  DVec<int32_t> cnt(A.nbc, true), fill(A.nbc, true);
  if (A.nnzb) k_col_count<<<nblocks(A.nnzb), kT, 0, gstream()>>>(A.ci.p, A.nnzb, cnt.p);
  counts_to_rowptr(cnt.p, A.nbc, T.rp.p);
  T.ci.resize(A.nnzb);
  DVec<int32_t> src(A.nnzb);
  k_t_scatter<<<nblocks(A.nbr), kT, 0, gstream()>>>(A.rp.p, A.ci.p, A.nbr, T.rp.p, fill.p, T.ci.p, src.p);
  DVec<int> ovf(1, true);
  k_t_sort<<<(unsigned)((A.nbc + kWarpsT - 1) / kWarpsT), 32 * kWarpsT, 0, gstream()>>>(T.rp.p, A.nbc, T.ci.p, src.p, ovf.p);
  GS_CUDA(cudaGetLastError());
  int o = 0;
  GS_CUDA(cudaMemcpyAsync(&o, ovf.p, sizeof(int), cudaMemcpyDeviceToHost, gstream()));
  sync();
  if (o) {  // a transposed row longer than the warp sort handles: host transpose
    HBsr H = download(A);
    if (!values) H.v.assign((size_t)H.nnzb() * H.br * H.bc, 0.0);
    return upload(bsr_transpose(H));
  }
  if (values) {
    T.v.resize(A.nnzb * A.br * A.bc);
    if (A.nnzb) k_t_values<<<nblocks(A.nnzb), kT, 0, gstream()>>>(A.v.p, src.p, A.nnzb, A.br, A.bc, T.v.p);
  }
  GS_CUDA(cudaGetLastError());
  return T;
}

// ------------------------------------------------ union / axpby (merge) ---
__global__ void k_merge_count(const int32_t *__restrict__ arp, const int32_t *__restrict__ aci,
                              const int32_t *__restrict__ brp, const int32_t *__restrict__ bci, int64_t n,
                              int32_t *__restrict__ cnt) {
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  int p = arp[I], q = brp[I], c = 0;
  const int pe = arp[I + 1], qe = brp[I + 1];
  while (p < pe || q < qe) {
    const int ca = p < pe ? aci[p] : INT32_MAX, cb = q < qe ? bci[q] : INT32_MAX;
    const int m = min(ca, cb);
    if (ca == m) ++p;
    if (cb == m) ++q;
    ++c;
  }
  cnt[I] = c;
}

// C = a*A + b*B over the union pattern (values optional)
__global__ void k_merge_fill(const int32_t *__restrict__ arp, const int32_t *__restrict__ aci,
                             const double *__restrict__ av, const int32_t *__restrict__ brp,
                             const int32_t *__restrict__ bci, const double *__restrict__ bv, int64_t n, int bs,
                             double sa, double sb, const int32_t *__restrict__ crp, int32_t *__restrict__ cci,
                             double *__restrict__ cv) {
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  int p = arp[I], q = brp[I], o = crp[I];
  const int pe = arp[I + 1], qe = brp[I + 1];
  while (p < pe || q < qe) {
    const int ca = p < pe ? aci[p] : INT32_MAX, cb = q < qe ? bci[q] : INT32_MAX;
    const int m = min(ca, cb);
    cci[o] = m;
    if (cv) {
      for (int e = 0; e < bs; ++e) {
        double v = 0.0;
        if (ca == m) v += sa * av[(int64_t)p * bs + e];
        if (cb == m) v += sb * bv[(int64_t)q * bs + e];
        cv[(int64_t)o * bs + e] = v;
      }
    }
    if (ca == m) ++p;
    if (cb == m) ++q;
    ++o;
  }
}

DB merge(double sa, const DB &A, double sb, const DB &B, bool values) {
  DB C;
  C.shape(A.br, A.bc, A.nbr, A.nbc);
  if (A.nbr == 0) return C;
  DVec<int32_t> cnt(A.nbr);
  k_merge_count<<<nblocks(A.nbr), kT, 0, gstream()>>>(A.rp.p, A.ci.p, B.rp.p, B.ci.p, A.nbr, cnt.p);
  C.nnzb = counts_to_rowptr(cnt.p, A.nbr, C.rp.p);
  C.ci.resize(C.nnzb);
  if (values) C.v.resize(C.nnzb * A.br * A.bc);
  k_merge_fill<<<nblocks(A.nbr), kT, 0, gstream()>>>(A.rp.p, A.ci.p, values ? A.v.p : nullptr, B.rp.p, B.ci.p,
                                       values ? B.v.p : nullptr, A.nbr, A.br * A.bc, sa, sb, C.rp.p, C.ci.p,
                                       values ? C.v.p : nullptr);
  GS_CUDA(cudaGetLastError());
  return C;
}

// ------------------------------------------------------ strength graph ---
__global__ void k_block_fro(BV A, double *__restrict__ fro, double *__restrict__ dn) {
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= A.nbr) return;
  const int bs = A.br * A.bc;
  for (int a = A.rp[I]; a < A.rp[I + 1]; ++a) {
    double s = 0.0;
    for (int e = 0; e < bs; ++e) s += A.v[(int64_t)a * bs + e] * A.v[(int64_t)a * bs + e];
    fro[a] = sqrt(s);
    if (A.ci[a] == I) dn[I] = fro[a];
  }
}

// fixed (or null): nodes that keep no edge (every dof a Dirichlet dof)
__global__ void k_strong(BV A, const double *__restrict__ fro, const double *__restrict__ dn, double theta,
                         const uint8_t *__restrict__ fixed, const int32_t *__restrict__ srp,
                         int32_t *__restrict__ cnt, int32_t *__restrict__ sci) {
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= A.nbr) return;
  int c = 0;
  for (int a = A.rp[I]; a < A.rp[I + 1]; ++a) {
    const int J = A.ci[a];
    if (J == I) continue;
    if (fixed && (fixed[I] || fixed[J])) continue;
    if (fro[a] > theta * sqrt(dn[I] * dn[J])) {
      if (sci) sci[srp[I] + c] = J;
      ++c;
    }
  }
  if (!sci) cnt[I] = c;
}

// node graph of strong connections, symmetrised (pattern only)
DB strength(const DB &A, double theta, const uint8_t *fixed) {
  DVec<double> fro(std::max<int64_t>(1, A.nnzb)), dn(A.nbr, true);
  k_block_fro<<<nblocks(A.nbr), kT, 0, gstream()>>>(view(A), fro.p, dn.p);
  DB S;
  S.shape(1, 1, A.nbr, A.nbr);
  DVec<int32_t> cnt(A.nbr);
  k_strong<<<nblocks(A.nbr), kT, 0, gstream()>>>(view(A), fro.p, dn.p, theta, fixed, nullptr, cnt.p, nullptr);
  S.nnzb = counts_to_rowptr(cnt.p, A.nbr, S.rp.p);
  S.ci.resize(S.nnzb);
  k_strong<<<nblocks(A.nbr), kT, 0, gstream()>>>(view(A), fro.p, dn.p, theta, fixed, S.rp.p, cnt.p, S.ci.p);
  GS_CUDA(cudaGetLastError());
  DB ST = transpose(S, false);
  return merge(1.0, S, 1.0, ST, false);
}

// ---------------------------------------------------------- aggregation ---
enum : int8_t { UND = 0, ROOT = 1, OUT = 2, ISO = 3 };

__device__ __forceinline__ bool better(uint64_t seed, int a, int b) {  // a ranks before b
  if (b < 0) return a >= 0;
  if (a < 0) return false;
  const uint64_t pa = sm64(seed, (uint64_t)a), pb = sm64(seed, (uint64_t)b);
  return pa != pb ? pa > pb : a < b;
}

__global__ void k_agg_init(const int32_t *__restrict__ rp, int64_t n, int8_t *__restrict__ st) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) st[i] = rp[i + 1] == rp[i] ? ISO : UND;
}

// r1[u] = a root in {u} + N(u)
__global__ void k_root_near(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int64_t n,
                            const int8_t *__restrict__ st, int8_t *__restrict__ r1) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n) return;
  int8_t f = st[u] == ROOT;
  for (int p = rp[u]; p < rp[u + 1] && !f; ++p) f = st[ci[p]] == ROOT;
  r1[u] = f;
}

__global__ void k_mark_out(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int64_t n,
                           int8_t *__restrict__ st, const int8_t *__restrict__ r1) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n || st[v] != UND) return;
  bool f = r1[v];
  for (int p = rp[v]; p < rp[v + 1] && !f; ++p) f = r1[ci[p]];
  if (f) st[v] = OUT;
}

// b1[u] = best undecided node in {u} + N(u) (or -1)
__global__ void k_best_near(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int64_t n,
                            const int8_t *__restrict__ st, int32_t *__restrict__ b1, uint64_t seed) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n) return;
  int b = st[u] == UND ? (int)u : -1;
  for (int p = rp[u]; p < rp[u + 1]; ++p) {
    const int w = ci[p];
    if (st[w] == UND && better(seed, w, b)) b = w;
  }
  b1[u] = b;
}

__global__ void k_pick(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int64_t n,
                       int8_t *__restrict__ st, const int32_t *__restrict__ b1, uint64_t seed,
                       int *__restrict__ left) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n || st[v] != UND) return;
  int b = b1[v];
  for (int p = rp[v]; p < rp[v + 1]; ++p) {
    const int w = b1[ci[p]];
    if (better(seed, w, b)) b = w;
  }
  if (b == (int)v) st[v] = ROOT;
  else atomicAdd(left, 1);
}

__global__ void k_root_flags(const int8_t *__restrict__ st, int64_t n, int32_t *__restrict__ f) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) f[i] = st[i] == ROOT;
}

__global__ void k_phase12(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int64_t n,
                          const int8_t *__restrict__ st, const int32_t *__restrict__ rid,
                          int32_t *__restrict__ agg, int32_t *__restrict__ roots) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  int a = -1;
  if (st[v] == ROOT) {
    a = rid[v];
    roots[a] = (int32_t)v;
  } else if (st[v] != ISO) {
    for (int p = rp[v]; p < rp[v + 1]; ++p)
      if (st[ci[p]] == ROOT) {
        a = rid[ci[p]];
        break;
      }
  }
  agg[v] = a;
}

__global__ void k_phase3(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int64_t n,
                         const int8_t *__restrict__ st, const int32_t *__restrict__ agg2,
                         const int32_t *__restrict__ roots, int32_t *__restrict__ agg, uint64_t seed,
                         int *__restrict__ bad) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n || agg2[v] >= 0 || st[v] == ISO) return;
  int best = -1;
  for (int p = rp[v]; p < rp[v + 1]; ++p) {
    const int a = agg2[ci[p]];
    if (a < 0) continue;
    if (best < 0 || better(seed, roots[a], roots[best])) best = a;
  }
  if (best < 0) atomicOr(bad, 1);
  agg[v] = best;
}

// aggregation of the node graph G (pattern); returns the aggregate count
int64_t aggregate_gpu(const DB &G, uint64_t seed, DVec<int32_t> &agg) {
  const int64_t n = G.nbr;
  DVec<int8_t> st(n), r1(n);
  DVec<int32_t> b1(n), flags(n), rid(n + 1);
  DVec<int> left(1);
  k_agg_init<<<nblocks(n), kT, 0, gstream()>>>(G.rp.p, n, st.p);
  for (int round = 0; round < 10000; ++round) {
    k_root_near<<<nblocks(n), kT, 0, gstream()>>>(G.rp.p, G.ci.p, n, st.p, r1.p);
    k_mark_out<<<nblocks(n), kT, 0, gstream()>>>(G.rp.p, G.ci.p, n, st.p, r1.p);
    k_best_near<<<nblocks(n), kT, 0, gstream()>>>(G.rp.p, G.ci.p, n, st.p, b1.p, seed);
    GS_CUDA(cudaMemsetAsync(left.p, 0, sizeof(int), gstream()));
    k_pick<<<nblocks(n), kT, 0, gstream()>>>(G.rp.p, G.ci.p, n, st.p, b1.p, seed, left.p);
    int l = 0;
    GS_CUDA(cudaMemcpyAsync(&l, left.p, sizeof(int), cudaMemcpyDeviceToHost, gstream()));
  sync();
    if (l == 0) break;
    if (round == 9999) throw SetupError(-7, "GPU setup: aggregation did not settle");
  }
  k_root_flags<<<nblocks(n), kT, 0, gstream()>>>(st.p, n, flags.p);
  const int64_t nagg = counts_to_rowptr(flags.p, n, rid.p);
  agg.resize(n);
  DVec<int32_t> agg2(n), roots(std::max<int64_t>(1, nagg));
  k_phase12<<<nblocks(n), kT, 0, gstream()>>>(G.rp.p, G.ci.p, n, st.p, rid.p, agg2.p, roots.p);
  GS_CUDA(cudaMemcpyAsync(agg.p, agg2.p, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, gstream()));
  DVec<int> bad(1, true);
  k_phase3<<<nblocks(n), kT, 0, gstream()>>>(G.rp.p, G.ci.p, n, st.p, agg2.p, roots.p, agg.p, seed, bad.p);
  GS_CUDA(cudaGetLastError());
  int b = 0;
  GS_CUDA(cudaMemcpyAsync(&b, bad.p, sizeof(int), cudaMemcpyDeviceToHost, gstream()));
  sync();
  if (b) throw SetupError(-7, "GPU setup: node not within distance 2 of a root");
  return nagg;
}

// ---------------------------------------------------- tentative P (QR) ---
__global__ void k_agg_count(const int32_t *__restrict__ agg, int64_t n, int32_t *__restrict__ cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && agg[i] >= 0) atomicAdd(&cnt[agg[i]], 1);
}

__global__ void k_agg_scatter(const int32_t *__restrict__ agg, int64_t n, const int32_t *__restrict__ start,
                              int32_t *__restrict__ fill, int32_t *__restrict__ members) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && agg[i] >= 0) members[start[agg[i]] + atomicAdd(&fill[agg[i]], 1)] = (int32_t)i;
}

constexpr int kMCap = 1024;  // nodes per aggregate sorted on the GPU

__global__ void k_agg_sort(const int32_t *__restrict__ start, int64_t nagg, int32_t *__restrict__ members,
                           int *__restrict__ ovf) {
  __shared__ int ks[kWarpsT * kMCap];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t a = (int64_t)blockIdx.x * kWarpsT + warp;
  if (a >= nagg) return;
  const int lo = start[a], m = start[a + 1] - lo;
  if (m > kMCap) {
    if (lane == 0) atomicOr(ovf, 1);
    return;
  }
  int *k = ks + warp * kMCap;
  for (int i = lane; i < m; i += 32) k[i] = members[lo + i];
  __syncwarp();
  warp_bitonic(k, nullptr, m, kMCap);
  for (int i = lane; i < m; i += 32) members[lo + i] = k[i];
}

// pt_rp: row pointer of P_tent (1 block per aggregated node)
__global__ void k_agg_flag(const int32_t *__restrict__ agg, int64_t n, int32_t *__restrict__ f) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) f[i] = agg[i] >= 0;
}

// One warp per aggregate: near-nullspace rows into Q (in the P_tent value
// slots of the members), two-pass Gram-Schmidt, R into Bc.
// kind: 0 constants, 1 rigid-body modes from coords (fine), 2 rows of Bprev
// (coarse levels, or the caller's vectors on the fine level); rows of dofs
// flagged in dmask (fine level, or null) are zero.
__global__ void k_tentative(const int32_t *__restrict__ start, const int32_t *__restrict__ members, int64_t nagg,
                            int b, int k, int kind, int dim, const double *__restrict__ coords,
                            const double *__restrict__ Bprev, const uint8_t *__restrict__ dmask,
                            const int32_t *__restrict__ ptrp, int32_t *__restrict__ ptci, double *__restrict__ ptv,
                            double *__restrict__ Bc) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t a = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (a >= nagg) return;
  const int lo = start[a], cnt = start[a + 1] - lo;
  const int m = cnt * b;
  // Q[r][q] lives at the P_tent slot of member r / b, entry (r % b, q)
  auto Q = [&](int r, int q) -> double & {
    return ptv[((int64_t)ptrp[members[lo + r / b]] * b + (r % b)) * k + q];
  };
  double cen[3] = {0, 0, 0};
  if (kind == 1) {
    for (int d = 0; d < dim; ++d) {
      double s = 0.0;
      for (int t = lane; t < cnt; t += 32) s += coords[(int64_t)members[lo + t] * dim + d];
      cen[d] = warp_sum(s) / (double)cnt;
    }
  }
  for (int t = lane; t < cnt; t += 32) {
    const int I = members[lo + t];
    ptci[ptrp[I]] = (int32_t)a;
    for (int c = 0; c < b; ++c)
      for (int q = 0; q < k; ++q) {
        double val = 0.0;
        if (kind == 0) {
          val = c == q ? 1.0 : 0.0;
        } else if (kind == 1) {
          const double x = coords[(int64_t)I * dim] - cen[0], y = coords[(int64_t)I * dim + 1] - cen[1];
          const double z = dim == 3 ? coords[(int64_t)I * dim + 2] - cen[2] : 0.0;
          if (q < dim) val = c == q ? 1.0 : 0.0;
          else if (dim == 2) val = c == 0 ? -y : x;  // rotation (-y, x)
          else if (q == 3) val = c == 1 ? -z : (c == 2 ? y : 0.0);
          else if (q == 4) val = c == 0 ? z : (c == 2 ? -x : 0.0);
          else val = c == 0 ? -y : (c == 1 ? x : 0.0);
        } else {
          val = Bprev[((int64_t)I * b + c) * k + q];
        }
        if (dmask && dmask[(int64_t)I * b + c]) val = 0.0;
        ptv[((int64_t)ptrp[I] * b + c) * k + q] = val;
      }
  }
  __syncwarp();
  double R[6][6];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) R[i][j] = 0.0;
  for (int c = 0; c < k; ++c) {
    double s = 0.0;
    for (int r = lane; r < m; r += 32) s += Q(r, c) * Q(r, c);
    const double n0 = sqrt(warp_sum(s));
    for (int pass = 0; pass < 2; ++pass) {
      double h[6] = {0, 0, 0, 0, 0, 0};
      for (int q = 0; q < c; ++q) {
        double t = 0.0;
        for (int r = lane; r < m; r += 32) t += Q(r, q) * Q(r, c);
        h[q] = warp_sum(t);
      }
      __syncwarp();
      for (int r = lane; r < m; r += 32) {
        double t = 0.0;
        for (int q = 0; q < c; ++q) t += Q(r, q) * h[q];
        Q(r, c) -= t;
      }
      __syncwarp();
      for (int q = 0; q < c; ++q) R[q][c] += h[q];
    }
    double t = 0.0;
    for (int r = lane; r < m; r += 32) t += Q(r, c) * Q(r, c);
    const double nv = sqrt(warp_sum(t));
    const bool keep = nv > 1e-10 * n0 && nv > 0.0;
    for (int r = lane; r < m; r += 32) Q(r, c) = keep ? Q(r, c) / nv : 0.0;
    __syncwarp();
    if (keep) R[c][c] = nv;
  }
  if (lane == 0)
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) Bc[((int64_t)a * k + i) * k + j] = R[i][j];
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct GLevel {
  DB A, P, R;
  DVec<double> dinv, B;
  DVec<int32_t> agg;
  int64_t nagg = 0;
  double lam = 0.0;
};

void fill_dinv(const DB &A, DVec<double> &dinv) {
  dinv.resize(A.nbr * A.br);
  DVec<int> bad(1, true);
  k_diag_inv<<<nblocks(A.nbr), kT, 0, gstream()>>>(view(A), dinv.p, bad.p);
  GS_CUDA(cudaGetLastError());
  int b = 0;
  GS_CUDA(cudaMemcpyAsync(&b, bad.p, sizeof(int), cudaMemcpyDeviceToHost, gstream()));
  sync();
  if (b) throw SetupError(-4, "zero diagonal entry in a diagonal block");
}

}  // namespace

HBsr gpu_spgemm(const HBsr &A, const HBsr &B) {
  StreamScope scope;
  HBsr C;
  {
    DB a = upload(A), b = upload(B);
    C = download(spgemm(a, b));
  }
  return C;
}

// DB of the shape of H from a device copy (D2D on the setup stream)
static DB from_device(const HBsr &H, const DevBlock &d) {
  DB A;
  A.br = H.br, A.bc = H.bc, A.nbr = H.nbr, A.nbc = H.nbc, A.nnzb = H.nnzb();
  A.rp.resize(A.nbr + 1);
  A.ci.resize(A.nnzb);
  A.v.resize(A.nnzb * A.br * A.bc);
  GS_CUDA(cudaMemcpyAsync(A.rp.p, d.rp, (size_t)(A.nbr + 1) * sizeof(int32_t), cudaMemcpyDeviceToDevice, gstream()));
  if (A.nnzb) {
    GS_CUDA(cudaMemcpyAsync(A.ci.p, d.ci, (size_t)A.nnzb * sizeof(int32_t), cudaMemcpyDeviceToDevice, gstream()));
    GS_CUDA(cudaMemcpyAsync(A.v.p, d.v, (size_t)A.v.n * sizeof(double), cudaMemcpyDeviceToDevice, gstream()));
  }
  return A;
}

void build_group_gpu(HGroup &g, const std::vector<HBsr> &diag, const std::vector<FieldInfo> &info,
                     int max_levels, int64_t coarse_max, uint64_t seed, bool want_off,
                     const BlockMap *fine_off, int verbose, const std::vector<DevBlock> *dev_diag,
                     const std::map<std::pair<int, int>, DevBlock> *dev_off, std::vector<HBsr> *steal) {
  StreamScope scope;  // outlives every device array below
  double tm[7] = {0, 0, 0, 0, 0, 0, 0};  // power, strength, aggregate, tentative, smooth+transpose, RAP, offdiag
  g.nf = (int)diag.size();
  g.info = info;
  std::vector<std::vector<GLevel>> lv(1);
  lv[0].resize(g.nf);
  for (int i = 0; i < g.nf; ++i) {
    lv[0][i].A = dev_diag ? from_device(diag[i], (*dev_diag)[i]) : upload(diag[i]);
    fill_dinv(lv[0][i].A, lv[0][i].dinv);
  }
  std::vector<std::map<std::pair<int, int>, DB>> off(1);
  if (want_off && fine_off)
    for (auto &kv : *fine_off)
      off[0][kv.first] = dev_off ? from_device(kv.second, dev_off->at(kv.first)) : upload(kv.second);
  auto total = [&](int l) {
    int64_t s = 0;
    for (auto &f : lv[l]) s += f.A.nbr * f.A.br;
    return s;
  };
  while ((int)lv.size() < max_levels && total((int)lv.size() - 1) > coarse_max) {
    const int l = (int)lv.size() - 1;
    const bool fine = l == 0;
    std::vector<GLevel> nxt(g.nf);
    for (int i = 0; i < g.nf; ++i) {
      GLevel &fl = lv[l][i];
      const FieldInfo &f = info[i];
      double t = now_s();
      fl.lam = power_lambda_gpu(fl.A, fl.dinv.p, seed);
      sync();
      tm[0] += now_s() - t;
      t = now_s();
      DVec<uint8_t> fixed, dmask;
      if (fine && !f.dirichlet.empty()) {
        const std::vector<uint8_t> fx = f.fixed_nodes();
        fixed.upload(fx.data(), (int64_t)fx.size());
        dmask.upload(f.dirichlet.data(), (int64_t)f.dirichlet.size());
      }
      DB G = strength(fl.A, f.theta, fixed.p);
      sync();
      tm[1] += now_s() - t;
      t = now_s();
      fl.nagg = aggregate_gpu(G, seed, fl.agg);
      tm[2] += now_s() - t;
      if (fl.nagg == 0) throw SetupError(-7, "aggregation produced no aggregate");
      t = now_s();
      const int b = fl.A.br;
      const int k = fine ? (f.ns == 0 ? f.b : (f.ns == 2 ? f.ns_dim : (f.dim == 2 ? 3 : 6))) : b;
      const int64_t n = fl.A.nbr;
      DVec<int32_t> cnt(fl.nagg, true), start(fl.nagg + 1), fillc(fl.nagg, true), members(n), flg(n);
      k_agg_count<<<nblocks(n), kT, 0, gstream()>>>(fl.agg.p, n, cnt.p);
      const int64_t nmem = counts_to_rowptr(cnt.p, fl.nagg, start.p);
      members.resize(std::max<int64_t>(1, nmem));
      k_agg_scatter<<<nblocks(n), kT, 0, gstream()>>>(fl.agg.p, n, start.p, fillc.p, members.p);
      DVec<int> ovf(1, true);
      k_agg_sort<<<(unsigned)((fl.nagg + kWarpsT - 1) / kWarpsT), 32 * kWarpsT, 0, gstream()>>>(start.p, fl.nagg, members.p, ovf.p);
      int o = 0;
      GS_CUDA(cudaMemcpyAsync(&o, ovf.p, sizeof(int), cudaMemcpyDeviceToHost, gstream()));
  sync();
      if (o) throw SetupError(-7, "GPU setup: aggregate larger than 1024 nodes");
      DB Pt;
      Pt.shape(b, k, n, fl.nagg);
      k_agg_flag<<<nblocks(n), kT, 0, gstream()>>>(fl.agg.p, n, flg.p);
      Pt.nnzb = counts_to_rowptr(flg.p, n, Pt.rp.p);
      Pt.ci.resize(Pt.nnzb);
      Pt.v.resize(Pt.nnzb * b * k);
      DVec<double> coords, userB;
      if (fine && f.ns == 1) coords.upload(f.coords.data(), (int64_t)f.coords.size());
      if (fine && f.ns == 2) userB.upload(f.user_B.data(), (int64_t)f.user_B.size());
      nxt[i].B.resize(fl.nagg * k * k);
      const int kind = fine ? (f.ns == 0 ? 0 : (f.ns == 1 ? 1 : 2)) : 2;
      k_tentative<<<(unsigned)((fl.nagg + 3) / 4), 128, 0, gstream()>>>(start.p, members.p, fl.nagg, b, k, kind, f.dim, coords.p,
                                                          fine && f.ns == 2 ? userB.p : fl.B.p, dmask.p, Pt.rp.p,
                                                          Pt.ci.p, Pt.v.p, nxt[i].B.p);
      GS_CUDA(cudaGetLastError());
      sync();
      tm[3] += now_s() - t;
      t = now_s();
      if (f.pg) {
        // Petrov-Galerkin damping parameters (column dot products, row
        // minima) on the host, as in the host setup; P and R come back up
        HBsr hP, hR;
        pg_transfers(l == 0 ? diag[i] : download(fl.A), fl.dinv.download(), download(Pt), hP, hR);
        fl.P = upload(hP);
        fl.R = upload(hR);
      } else {
        DB DAP = spgemm(fl.A, Pt);
        k_scale_rows<<<nblocks(DAP.nbr), kT, 0, gstream()>>>(DAP.v.p, DAP.rp.p, DAP.nbr, DAP.br, DAP.bc, fl.dinv.p);
        const double omega = 4.0 / (3.0 * fl.lam);
        fl.P = merge(1.0, Pt, -omega, DAP, true);
        fl.R = transpose(fl.P, true);
      }
      sync();
      tm[4] += now_s() - t;
      t = now_s();
      {
        DB AP = spgemm(fl.A, fl.P);
        nxt[i].A = spgemm(fl.R, AP);
      }
      fill_dinv(nxt[i].A, nxt[i].dinv);
      sync();
      tm[5] += now_s() - t;
    }
    if (want_off) {
      const double t = now_s();
      std::map<std::pair<int, int>, DB> noff;
      for (auto &kv : off[l]) {
        const int i = kv.first.first, j = kv.first.second;
        DB AP = spgemm(kv.second, lv[l][j].P);
        noff[kv.first] = spgemm(lv[l][i].R, AP);
      }
      off.push_back(std::move(noff));
      sync();
      tm[6] += now_s() - t;
    }
    lv.push_back(std::move(nxt));
  }
  // download into the host structures
  const double td = now_s();
  g.lv.assign(lv.size(), std::vector<HLevelField>(g.nf));
  for (size_t l = 0; l < lv.size(); ++l)
    for (int i = 0; i < g.nf; ++i) {
      GLevel &d = lv[l][i];
      HLevelField &h = g.lv[l][i];
      if (l > 0) h.A = download(d.A);
      else if (steal) h.A = std::move((*steal)[i]);
      else h.A = diag[i];
      h.dinv = d.dinv.download();
      h.lam = d.lam;
      if (l + 1 < lv.size()) {
        h.agg = d.agg.download();
        h.nagg = d.nagg;
        h.P = download(d.P);
        h.R = download(d.R);
      }
    }
  g.off.assign(1, BlockMap());
  if (want_off && fine_off) g.off[0] = *fine_off;
  for (size_t l = 1; l < off.size(); ++l) {
    BlockMap m;
    for (auto &kv : off[l]) m[kv.first] = download(kv.second);
    g.off.push_back(std::move(m));
  }
  const double tdl = now_s() - td;
  // coarsest-level direct solvers (host LU, as in build_group)
  const int L = (int)g.lv.size() - 1;
  g.coarse_field.resize(g.nf);
  for (int i = 0; i < g.nf; ++i) {
    const HBsr &A = g.lv[L][i].A;
    g.coarse_field[i] = dense_lu((int)A.nrows(), bsr_to_dense(A));
  }
  if (want_off) {
    std::vector<int64_t> of(g.nf + 1, 0);
    for (int i = 0; i < g.nf; ++i) of[i + 1] = of[i] + g.lv[L][i].A.nrows();
    const int64_t nn = of[g.nf];
    std::vector<double> D((size_t)(nn * nn), 0.0);
    auto put = [&](const HBsr &A, int i, int j) {
      std::vector<double> dd = bsr_to_dense(A);
      const int64_t nr = A.nrows(), nc = A.ncols();
      for (int64_t r = 0; r < nr; ++r)
        for (int64_t c = 0; c < nc; ++c) D[(size_t)((of[i] + r) * nn + of[j] + c)] += dd[r * nc + c];
    };
    for (int i = 0; i < g.nf; ++i) put(g.lv[L][i].A, i, i);
    for (auto &kv : g.off[L]) put(kv.second, kv.first.first, kv.first.second);
    g.coarse_coupled = dense_lu((int)nn, std::move(D));
  }
  if (verbose)
    std::fprintf(stderr,
                 "mfs GPU setup group (%d fields, %d levels): power %.3f strength %.3f aggregate %.3f tentative %.3f "
                 "smooth+transpose %.3f RAP %.3f offdiag %.3f download %.3f s\n",
                 g.nf, (int)g.lv.size(), tm[0], tm[1], tm[2], tm[3], tm[4], tm[5], tm[6], tdl);
}

}  // namespace mfs
