// libmfs: device hierarchy, block preconditioners, FGMRES and the C ABI.
//
//  * BGS(AMG)  (Sec. 4.1): k_max sweeps of block Gauss-Seidel from x = 0, one
//    single-field V-cycle (Algorithm 1) per diagonal block;
//  * SIMPLE    (Sec. 4.2): predictor / Schur / update steps on a 2 x 2 merging
//    of the fields, SIMPLEC or diagonal A~_11, explicit S~;
//  * AMG(BGS)  (Sec. 4.3): coupled V-cycle with block-diagonal transfers,
//    blockwise Galerkin coarse blocks, BGS level smoothing and a dense LU of
//    the assembled coarsest coupled matrix;
//  * FGMRES(m) (Sec. 3.1-3.2, right preconditioning) with CGS2 Arnoldi and
//    the Sec. 7.1 stopping rule.
// Every step of a solve runs as a kernel of kernels.cu; the host only
// sequences launches and runs the (m+1) x m Givens least-squares update.
#include <algorithm>
#include <atomic>
#include <thread>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <memory>
#include <stdexcept>
#include <string>
#include <type_traits>
#include <vector>

#include "amg_setup.h"
#include "setup_gpu.h"
#include "kernels.cuh"
#include "mfs.h"

namespace mfs {

struct CudaError : std::runtime_error {
  int code;
  CudaError(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};

static thread_local std::string g_last_error;
void set_last_error(const char *msg) { g_last_error = msg; }

#define MFS_CUDA(call)                                                                      \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      throw CudaError(e_ == cudaErrorMemoryAllocation ? MFS_ERR_OOM : MFS_ERR_CUDA,         \
                      std::string(#call) + ": " + cudaGetErrorString(e_));                  \
  } while (0)

// Device memory of the library comes from the device's stream-ordered pool
// (cudaMallocAsync / cudaFreeAsync on the legacy stream): unlike cudaFree, a
// free does not wait for the whole device, so handles can come and go while
// other handles' work runs (setups and solves of a server).  Memory is freed
// only when no stream still uses it (the owner has synchronised its
// streams).  Freed memory above the pool's release threshold goes back to
// the system.
void pool_setup_once() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = 4ull << 30;  // keep up to 4 GB of freed memory for reuse
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  done[dev] = true;
}

struct Arena {
  std::vector<std::pair<void *, int64_t>> ptrs;
  int64_t bytes = 0;
  template <typename T> T *alloc(int64_t count) {
    if (count <= 0) return nullptr;
    pool_setup_once();
    void *p = nullptr;
    MFS_CUDA(cudaMallocAsync(&p, (size_t)count * sizeof(T), 0));
    // the allocation is ordered on the legacy stream; once that stream has
    // passed it, any stream may use the memory
    MFS_CUDA(cudaStreamSynchronize(0));
    ptrs.push_back({p, count * (int64_t)sizeof(T)});
    // the plain-BSR kernels read blocks with 16-byte loads from the start of
    // a value array (pool allocations are 256-byte aligned)
    if (reinterpret_cast<uintptr_t>(p) & 15) throw CudaError(MFS_ERR_CUDA, "device allocation not 16-byte aligned");
    bytes += count * (int64_t)sizeof(T);
    return (T *)p;
  }
  // synchronous copy on the legacy stream (after the allocation there): a
  // copy from pageable memory may still be in flight when this returns, so
  // work on other (non-blocking) streams that reads the result must first
  // synchronise with stream 0
  template <typename T> T *upload(const std::vector<T> &h) {
    T *p = alloc<T>((int64_t)h.size());
    if (p) MFS_CUDA(cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return p;
  }
  template <typename T> T *zeros(int64_t count) {
    T *p = alloc<T>(count);
    if (p) MFS_CUDA(cudaMemsetAsync(p, 0, (size_t)count * sizeof(T), 0));
    return p;
  }
  // callers free only memory no stream is still using (the owner's streams
  // have been synchronised)
  void release(const void *p) {
    if (!p) return;
    for (size_t k = 0; k < ptrs.size(); ++k)
      if (ptrs[k].first == p) {
        cudaFreeAsync(ptrs[k].first, 0);
        bytes -= ptrs[k].second;
        ptrs.erase(ptrs.begin() + (long)k);
        return;
      }
  }
  ~Arena() {
    for (auto &q : ptrs) cudaFreeAsync(q.first, 0);
  }
};

// Pinned host blocks, kept by power-of-two size for reuse (cudaFreeHost
// would wait for the whole device): a handle's or a fused plan's few small
// pinned buffers come and go with it.
struct PinnedCache {
  std::mutex mu;
  std::map<size_t, std::vector<void *>> free;
  static size_t round_up(size_t b) {
    size_t c = 256;
    while (c < b) c <<= 1;
    return c;
  }
  void *get(size_t bytes) {
    const size_t c = round_up(bytes);
    {
      std::lock_guard<std::mutex> lock(mu);
      auto &v = free[c];
      if (!v.empty()) {
        void *p = v.back();
        v.pop_back();
        return p;
      }
    }
    void *p = nullptr;
    MFS_CUDA(cudaMallocHost(&p, c));
    return p;
  }
  void put(void *p, size_t bytes) {
    if (!p) return;
    std::lock_guard<std::mutex> lock(mu);
    free[round_up(bytes)].push_back(p);
  }
};
// never destroyed (the CUDA runtime may be gone at process exit)
static PinnedCache &g_pinned = *new PinnedCache();

// Layout autotuning: matrices with at least kTuneMinRows block rows are built
// in both layouts (SELL-32, one thread per block row, with 2, 4 or 8 block
// slots in flight; plain BSR, one warp per block row), each timed with CUDA
// events, and the fastest is kept.  Smaller
// matrices are latency bound and take the warp layout.  Decisions are cached
// per (block shape, rows, blocks, precision) for the life of the process.
constexpr int64_t kTuneMinRows = 2048;

static dev::Sell upload_layout(Arena &ar, const HBsr &A, bool want64, bool want32, int kind) {
  dev::Sell S;
  S.br = A.br;
  S.bc = A.bc;
  S.nbr = A.nbr;
  S.nbc = A.nbc;
  S.nnzb = A.nnzb();
  if (A.nbr == 0) return S;
  const int bs = A.br * A.bc;
  if (kind == 1) {
    // plain BSR, one warp per block row
    if (A.nnzb() > INT32_MAX) throw SetupError(MFS_ERR_INVALID, "matrix too large for 32-bit block offsets");
    S.kind = 1;
    std::vector<int32_t> rp(A.rp.begin(), A.rp.end());
    S.sp = ar.upload(rp);
    S.col = ar.upload(A.ci);
    if (want64) S.v64 = ar.upload(A.v);
    if (want32) {
      std::vector<float> v32(A.v.begin(), A.v.end());
      S.v32 = ar.upload(v32);
    }
    return S;
  }
  S.nslices = (A.nbr + 31) / 32;
  std::vector<int32_t> sp(S.nslices + 1, 0), rl(A.nbr);
  for (int64_t s = 0; s < S.nslices; ++s) {
    int w = 0;
    for (int64_t I = s * 32; I < std::min<int64_t>(A.nbr, s * 32 + 32); ++I) {
      rl[I] = (int32_t)(A.rp[I + 1] - A.rp[I]);
      w = std::max(w, rl[I]);
    }
    if ((int64_t)sp[s] + w > INT32_MAX / 32) throw SetupError(MFS_ERR_INVALID, "matrix too large for 32-bit slot offsets");
    sp[s + 1] = sp[s] + w;
  }
  S.nslots = sp[S.nslices];
  std::vector<int32_t> col((size_t)S.nslots * 32, 0);
  std::vector<double> v64;
  std::vector<float> v32;
  if (want64) v64.assign((size_t)S.nslots * bs * 32, 0.0);
  if (want32) v32.assign((size_t)S.nslots * bs * 32, 0.0f);
#pragma omp parallel for schedule(static)
  for (int64_t I = 0; I < A.nbr; ++I) {
    const int64_t s = I >> 5, lane = I & 31;
    for (int64_t t = 0; t < A.rp[I + 1] - A.rp[I]; ++t) {
      const int64_t a = A.rp[I] + t, slot = sp[s] + t;
      col[slot * 32 + lane] = A.ci[a];
      for (int e = 0; e < bs; ++e) {
        const size_t o = (size_t)(slot * bs + e) * 32 + lane;
        if (want64) v64[o] = A.v[a * bs + e];
        if (want32) v32[o] = (float)A.v[a * bs + e];
      }
    }
  }
  S.sp = ar.upload(sp);
  S.rl = ar.upload(rl);
  S.col = ar.upload(col);
  if (want64) S.v64 = ar.upload(v64);
  if (want32) S.v32 = ar.upload(v32);
  return S;
}

// An input block in device memory as plain BSR (int32 row pointer and block
// columns, float64 blocks), uploaded once per setup; the fine layouts are
// built from it on the device.
struct RawDev {
  int32_t *rp = nullptr, *ci = nullptr;
  double *v = nullptr;
  int br = 0, bc = 0;
  int64_t nbr = 0, nbc = 0, nnzb = 0;
};

static RawDev upload_raw(Arena &tmp, const HBsr &A, cudaStream_t st) {
  RawDev R;
  R.br = A.br;
  R.bc = A.bc;
  R.nbr = A.nbr;
  R.nbc = A.nbc;
  R.nnzb = A.nnzb();
  if (A.nnzb() > INT32_MAX) throw SetupError(MFS_ERR_INVALID, "matrix too large for 32-bit block offsets");
  std::vector<int32_t> rp(A.rp.begin(), A.rp.end());
  R.rp = tmp.alloc<int32_t>((int64_t)rp.size());
  R.ci = tmp.alloc<int32_t>(R.nnzb);
  R.v = tmp.alloc<double>(R.nnzb * R.br * R.bc);
  MFS_CUDA(cudaMemcpyAsync(R.rp, rp.data(), rp.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  if (R.nnzb) {
    MFS_CUDA(cudaMemcpyAsync(R.ci, A.ci.data(), A.ci.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    MFS_CUDA(cudaMemcpyAsync(R.v, A.v.data(), A.v.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  }
  MFS_CUDA(cudaStreamSynchronize(st));  // rp is a temporary host vector
  return R;
}

// upload_layout for a device-resident block (or nsrc blocks of one pattern
// merged column-wise, kind 0 only), converted by kernels on stream st.
static dev::Sell upload_layout_dev(Arena &ar, const RawDev *const *src, int nsrc, bool want64, bool want32, int kind,
                                   cudaStream_t st) {
  const RawDev &A = *src[0];
  dev::Sell S;
  int bcs[3] = {0, 0, 0};
  S.bc = 0;
  for (int j = 0; j < nsrc; ++j) {
    bcs[j] = src[j]->bc;
    S.bc += src[j]->bc;
  }
  S.br = A.br;
  S.nbr = A.nbr;
  S.nbc = A.nbc;
  S.nnzb = A.nnzb;
  if (A.nbr == 0) return S;
  const int64_t bs = (int64_t)S.br * S.bc;
  if (kind == 1) {
    if (nsrc != 1) throw SetupError(MFS_ERR_INVALID, "merged rows need the SELL layout");
    S.kind = 1;
    int32_t *rp = ar.alloc<int32_t>(A.nbr + 1), *col = ar.alloc<int32_t>(A.nnzb);
    MFS_CUDA(cudaMemcpyAsync(rp, A.rp, (A.nbr + 1) * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    if (A.nnzb) MFS_CUDA(cudaMemcpyAsync(col, A.ci, A.nnzb * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    S.sp = rp;
    S.col = col;
    if (want64) {
      double *v = ar.alloc<double>(A.nnzb * bs);
      if (A.nnzb) MFS_CUDA(cudaMemcpyAsync(v, A.v, A.nnzb * bs * sizeof(double), cudaMemcpyDeviceToDevice, st));
      S.v64 = v;
    }
    if (want32) {
      float *v = ar.alloc<float>(A.nnzb * bs);
      dev::convert<double, float>(A.v, v, A.nnzb * bs, st);
      S.v32 = v;
    }
    MFS_CUDA(cudaStreamSynchronize(st));
    return S;
  }
  S.nslices = (A.nbr + 31) / 32;
  int32_t *rl = ar.alloc<int32_t>(A.nbr);
  int32_t *w = nullptr;
  MFS_CUDA(cudaMallocAsync((void **)&w, (size_t)S.nslices * sizeof(int32_t), st));
  dev::sell_widths(A.rp, A.nbr, rl, w, st);
  std::vector<int32_t> hw(S.nslices), sp(S.nslices + 1, 0);
  MFS_CUDA(cudaMemcpyAsync(hw.data(), w, S.nslices * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MFS_CUDA(cudaFreeAsync(w, st));
  MFS_CUDA(cudaStreamSynchronize(st));
  for (int64_t k = 0; k < S.nslices; ++k) {
    if ((int64_t)sp[k] + hw[k] > INT32_MAX / 32) throw SetupError(MFS_ERR_INVALID, "matrix too large for 32-bit slot offsets");
    sp[k + 1] = sp[k] + hw[k];
  }
  S.nslots = sp[S.nslices];
  // on st, like the kernels below: a synchronous cudaMemcpy from pageable
  // memory may return before the data reach the device, and its legacy stream
  // does not order the non-blocking stream st
  int32_t *dsp = ar.alloc<int32_t>((int64_t)sp.size());
  MFS_CUDA(cudaMemcpyAsync(dsp, sp.data(), sp.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  int32_t *col = ar.alloc<int32_t>(S.nslots * 32);
  double *v64 = want64 ? ar.alloc<double>(S.nslots * bs * 32) : nullptr;
  float *v32 = want32 ? ar.alloc<float>(S.nslots * bs * 32) : nullptr;
  if (col) MFS_CUDA(cudaMemsetAsync(col, 0, S.nslots * 32 * sizeof(int32_t), st));
  if (v64) MFS_CUDA(cudaMemsetAsync(v64, 0, S.nslots * bs * 32 * sizeof(double), st));
  if (v32) MFS_CUDA(cudaMemsetAsync(v32, 0, S.nslots * bs * 32 * sizeof(float), st));
  dev::sell_fill(A.rp, A.ci, nsrc, src[0]->v, nsrc > 1 ? src[1]->v : nullptr, nsrc > 2 ? src[2]->v : nullptr, bcs,
                 A.br, A.nbr, dsp, col, v64, v32, st);
  MFS_CUDA(cudaGetLastError());
  MFS_CUDA(cudaStreamSynchronize(st));
  S.sp = dsp;
  S.rl = rl;
  S.col = col;
  S.v64 = v64;
  S.v32 = v32;
  return S;
}

template <typename T> static float time_spmv(const dev::Sell &S, cudaStream_t st) {
  T *x = nullptr, *y = nullptr;
  MFS_CUDA(cudaMallocAsync((void **)&x, (size_t)std::max<int64_t>(1, S.ncols()) * sizeof(T), st));
  MFS_CUDA(cudaMallocAsync((void **)&y, (size_t)std::max<int64_t>(1, S.nrows()) * sizeof(T), st));
  MFS_CUDA(cudaMemsetAsync(x, 0, (size_t)S.ncols() * sizeof(T), st));
  cudaEvent_t e0, e1;
  MFS_CUDA(cudaEventCreate(&e0));
  MFS_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    MFS_CUDA(cudaEventRecord(e0, st));
    dev::spmv<T>(S, x, y, T(1), T(0), nullptr, st);
    MFS_CUDA(cudaEventRecord(e1, st));
    MFS_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    MFS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0) best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(x, st);
  cudaFreeAsync(y, st);
  MFS_CUDA(cudaStreamSynchronize(st));
  return best;
}

static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int64_t, int64_t, int>, int> g_tune;
// mfs_params.layout_tune of the setup running on this thread
static thread_local int g_layout_tune = 0;

// Layout candidates of the autotuner: 0 SELL-32 with 2 slots in flight,
// 1 with 4, 2 plain BSR with one warp per row, 3 SELL-32 with 8 slots in
// flight (only for blocks of at most 3 entries, whose rows are short on bytes).
static int tune_pick(const dev::Sell &a, const dev::Sell &b, bool want32, cudaStream_t st) {
  dev::Sell a4 = a, a8 = a;
  a4.unroll = 4;
  a8.unroll = 8;
  const bool small = a.br * a.bc <= 3;
  float t[4];
  t[0] = want32 ? time_spmv<float>(a, st) : time_spmv<double>(a, st);
  t[1] = want32 ? time_spmv<float>(a4, st) : time_spmv<double>(a4, st);
  // throughput tuning leaves the one-warp-per-row layout out for short rows
  // (fewer blocks than lanes: idle lanes; SELL-32 moves more rows per
  // microsecond when the GPU is full) but keeps it for long rows such as a
  // restriction's, which one thread per row would walk serially
  const bool short_rows = a.nnzb < 32 * a.nbr;
  t[2] = g_layout_tune == 1 && short_rows ? 1e30f : (want32 ? time_spmv<float>(b, st) : time_spmv<double>(b, st));
  t[3] = !small ? 1e30f : (want32 ? time_spmv<float>(a8, st) : time_spmv<double>(a8, st));
  int best = 0;
  for (int c = 1; c < 4; ++c)
    if (t[c] < t[best]) best = c;
  return best;
}

static void tune_apply(dev::Sell &S, int best) {
  if (best == 1) S.unroll = 4;
  if (best == 3) S.unroll = 8;
}

// keep the chosen candidate, release the other layout
static dev::Sell tune_keep(Arena &ar, dev::Sell &a, dev::Sell &b, int best) {
  dev::Sell &loser = best == 2 ? a : b;
  ar.release(loser.sp);
  ar.release(loser.rl);
  ar.release(loser.col);
  ar.release(loser.v64);
  ar.release(loser.v32);
  dev::Sell S = best == 2 ? b : a;
  tune_apply(S, best);
  return S;
}

static dev::Sell upload_sell(Arena &ar, const HBsr &A, bool want64, bool want32) {
  if (A.nbr < kTuneMinRows) return upload_layout(ar, A, want64, want32, 1);
  const auto key = std::make_tuple(A.br, A.bc, (int64_t)A.nbr, (int64_t)A.nnzb(), (want32 ? 1 : 0) + 2 * g_layout_tune);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      dev::Sell S = upload_layout(ar, A, want64, want32, it->second == 2 ? 1 : 0);
      tune_apply(S, it->second);
      return S;
    }
  }
  dev::Sell a = upload_layout(ar, A, want64, want32, 0);
  dev::Sell b = upload_layout(ar, A, want64, want32, 1);
  cudaStream_t st;
  MFS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  MFS_CUDA(cudaStreamSynchronize(0));  // uploads and memsets of the legacy stream
  int best = 0;
  try {
    best = tune_pick(a, b, want32, st);
  } catch (...) {
    cudaStreamDestroy(st);
    throw;
  }
  cudaStreamDestroy(st);
  {
    // a setup that tuned the same shape concurrently and finished first
    // decides, so that every handle of the process runs the same variant
    std::lock_guard<std::mutex> lock(g_tune_mu);
    best = g_tune.emplace(key, best).first->second;
  }
  return tune_keep(ar, a, b, best);
}

// upload_sell for a device-resident input block: the same tuning and cache,
// the candidate layouts built on the device.
static dev::Sell upload_sell_dev(Arena &ar, const RawDev &A, bool want64, bool want32, cudaStream_t st) {
  const RawDev *src[1] = {&A};
  if (A.nbr < kTuneMinRows) return upload_layout_dev(ar, src, 1, want64, want32, 1, st);
  const auto key = std::make_tuple(A.br, A.bc, (int64_t)A.nbr, (int64_t)A.nnzb, (want32 ? 1 : 0) + 2 * g_layout_tune);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      dev::Sell S = upload_layout_dev(ar, src, 1, want64, want32, it->second == 2 ? 1 : 0, st);
      tune_apply(S, it->second);
      return S;
    }
  }
  dev::Sell a = upload_layout_dev(ar, src, 1, want64, want32, 0, st);
  dev::Sell b = upload_layout_dev(ar, src, 1, want64, want32, 1, st);
  MFS_CUDA(cudaStreamSynchronize(0));
  int best = tune_pick(a, b, want32, st);
  {
    // a setup that tuned the same shape concurrently and finished first
    // decides, so that every handle of the process runs the same variant
    std::lock_guard<std::mutex> lock(g_tune_mu);
    best = g_tune.emplace(key, best).first->second;
  }
  return tune_keep(ar, a, b, best);
}

// Explicit inverse (row-major) of a factored coarsest matrix: column j solves
// L U x = P e_j with the stored factors; the coarse solve then becomes one
// parallel matrix-vector product instead of two dependent triangular sweeps.
static std::vector<double> lu_inverse(const HDenseLU &lu) {
  const int n = lu.n;
  std::vector<double> inv((size_t)n * n);
#pragma omp parallel for schedule(static)
  for (int j = 0; j < n; ++j) {
    std::vector<double> y(n);
    for (int i = 0; i < n; ++i) y[i] = lu.perm[i] == j ? 1.0 : 0.0;
    for (int k = 0; k < n; ++k)  // unit-lower L, column-major
      for (int i = k + 1; i < n; ++i) y[i] -= lu.lu[(size_t)k * n + i] * y[k];
    for (int k = n - 1; k >= 0; --k) {
      y[k] /= lu.lu[(size_t)k * n + k];
      for (int i = 0; i < k; ++i) y[i] -= lu.lu[(size_t)k * n + i] * y[k];
    }
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + j] = y[i];
  }
  return inv;
}

// coarsest levels up to this size are solved through their explicit inverse
constexpr int kCoarseInverseMax = 4096;

static dev::DenseLU upload_lu(Arena &ar, const HDenseLU &lu) {
  dev::DenseLU d;
  d.n = lu.n;
  if (lu.n > 16384) throw SetupError(MFS_ERR_INVALID, "coarsest level too large for the dense LU (raise max_levels or lower coarse_max)");
  d.lu = ar.upload(lu.lu);
  d.perm = ar.upload(lu.perm);
  if (lu.n > 0 && lu.n <= kCoarseInverseMax) d.inv = ar.upload(lu_inverse(lu));
  return d;
}

template <typename T> static T *upload_as(Arena &ar, const std::vector<double> &h) {
  std::vector<T> t(h.begin(), h.end());
  return ar.upload(t);
}

template <typename T> struct FL {
  int64_t n = 0;
  dev::Sell A, P, R;
  T *dinv = nullptr;
  std::vector<T> c1, c2;  // smoother step coefficients
  T *bv = nullptr, *xv = nullptr, *t = nullptr, *d = nullptr, *r = nullptr, *c = nullptr, *e = nullptr;
  // multicolour Gauss-Seidel (smoother MFS_GS): the block rows in colour
  // order and the br x br diagonal block of every node
  dev::GsLevel gs;
  T *dblk = nullptr;
};

template <typename T> struct DGroup {
  int nf = 0, L = 0;
  bool mono = false;
  std::vector<std::vector<FL<T>>> lv;
  std::vector<std::map<std::pair<int, int>, dev::Sell>> off;
  std::vector<dev::DenseLU> cf;
  dev::DenseLU cc;
  T *cb = nullptr, *cx = nullptr;
  const dev::Sell *block(int l, int i, int j) const {
    if (i == j) return &lv[l][i].A;
    auto it = off[l].find({i, j});
    return it == off[l].end() ? nullptr : &it->second;
  }
};

static void smoother_coeffs(const mfs_params &p, double lam, std::vector<double> &c1, std::vector<double> &c2) {
  c1.clear();
  c2.clear();
  if (p.smoother == MFS_JACOBI) {
    for (int k = 0; k < p.jacobi_sweeps; ++k) {
      c1.push_back(0.0);
      c2.push_back(p.jacobi_omega);
    }
    return;
  }
  const double hi = p.cheb_boost * lam, lo = lam / p.cheb_ratio;
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  c1.push_back(0.0);
  c2.push_back(1.0 / theta);
  for (int k = 1; k < p.cheb_degree; ++k) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    c1.push_back(rn * rho);
    c2.push_back(2.0 * rn / delta);
    rho = rn;
  }
}

// Gauss-Seidel data of one smoothed level field: its block rows reordered by
// colour (increasing node order inside a colour) as plain BSR, the node of
// each, the colour offsets, and every node's diagonal block.  Lanes per row
// follow the average row length; levels whose vector fits in 48 KB run all
// colours in one single-CTA launch with x in shared memory.
constexpr int64_t kGsSmallBytes = 48 * 1024;
template <typename T>
static void upload_gs(Arena &ar, FL<T> &f, const HBsr &A, const std::vector<int32_t> &color) {
  const bool f32 = std::is_same<T, float>::value;
  const int bs = A.br * A.bc;
  std::vector<double> dg((size_t)A.nbr * bs, 0.0);
  for (int64_t I = 0; I < A.nbr; ++I)
    for (int64_t a = A.rp[I]; a < A.rp[I + 1]; ++a)
      if (A.ci[a] == I) std::copy(A.v.begin() + a * bs, A.v.begin() + (a + 1) * bs, dg.begin() + I * bs);
  f.dblk = upload_as<T>(ar, dg);
  int nc = 0;
  for (int32_t c : color) nc = std::max(nc, c + 1);
  std::vector<std::vector<int32_t>> rows(nc);
  for (int64_t I = 0; I < A.nbr; ++I) rows[color[I]].push_back((int32_t)I);
  HBsr S;
  S.br = A.br;
  S.bc = A.bc;
  S.nbr = A.nbr;
  S.nbc = A.nbc;
  S.rp.assign(1, 0);
  std::vector<int32_t> order, coff(1, 0);
  dev::GsLevel &g = f.gs;
  g.hoff.assign(1, 0);
  g.cnnzb.clear();
  for (int c = 0; c < nc; ++c) {
    const int64_t nz0 = (int64_t)S.ci.size();
    for (int32_t I : rows[c]) {
      for (int64_t a = A.rp[I]; a < A.rp[I + 1]; ++a) {
        S.ci.push_back(A.ci[a]);
        S.v.insert(S.v.end(), A.v.begin() + a * bs, A.v.begin() + (a + 1) * bs);
      }
      S.rp.push_back((int64_t)S.ci.size());
      order.push_back(I);
    }
    g.hoff.push_back((int64_t)order.size());
    coff.push_back((int32_t)order.size());
    g.cnnzb.push_back((int64_t)S.ci.size() - nz0);
  }
  g.M = upload_layout(ar, S, !f32, f32, 1);
  g.rowidx = ar.upload(order);
  g.coff = ar.upload(coff);
  const double avg = A.nbr ? (double)A.nnzb() / (double)A.nbr : 0.0;
  g.G = avg <= 12 ? 4 : avg <= 40 ? 8 : avg <= 100 ? 16 : 32;
  g.small = A.nrows() * (int64_t)sizeof(T) <= kGsSmallBytes;
}

// Device copy of a host group's matrices and smoother data (read-only after
// setup, shared by clones).  level0 gives the Sell objects of the level-0
// diagonal / off-diagonal blocks (shared with the fine operator).
template <typename T>
static void upload_group(Arena &ar, DGroup<T> &g, const HGroup &h, const mfs_params &p,
                         const std::vector<dev::Sell> &level0_diag,
                         const std::map<std::pair<int, int>, dev::Sell> &level0_off, bool mono) {
  const bool f32 = std::is_same<T, float>::value;
  g.nf = h.nf;
  g.L = h.nlevels();
  g.mono = mono;
  g.lv.assign(g.L, std::vector<FL<T>>(g.nf));
  g.off.assign(g.L, {});
  g.off[0] = level0_off;
  for (int l = 0; l < g.L; ++l) {
    for (int i = 0; i < g.nf; ++i) {
      const HLevelField &hf = h.lv[l][i];
      FL<T> &f = g.lv[l][i];
      f.n = hf.A.nrows();
      f.A = l == 0 ? level0_diag[i] : upload_sell(ar, hf.A, !f32, f32);
      if (l + 1 < g.L) {
        f.P = upload_sell(ar, hf.P, !f32, f32);
        f.R = upload_sell(ar, hf.R, !f32, f32);
        std::vector<double> c1, c2;
        smoother_coeffs(p, hf.lam, c1, c2);
        f.c1.assign(c1.begin(), c1.end());
        f.c2.assign(c2.begin(), c2.end());
        f.dinv = upload_as<T>(ar, hf.dinv);
      }
      if (!hf.color.empty()) upload_gs(ar, f, hf.A, hf.color);
    }
    if (l > 0 && mono)
      for (auto &kv : h.off[l]) g.off[l][kv.first] = upload_sell(ar, kv.second, !f32, f32);
  }
  g.cf.resize(g.nf);
  for (int i = 0; i < g.nf && i < (int)h.coarse_field.size(); ++i) g.cf[i] = upload_lu(ar, h.coarse_field[i]);
  if (mono) g.cc = upload_lu(ar, h.coarse_coupled);
}

// Work vectors of a group (per handle; a clone gets its own).
template <typename T> static void alloc_group_work(Arena &ar, DGroup<T> &g) {
  for (int l = 0; l < g.L; ++l)
    for (int i = 0; i < g.nf; ++i) {
      FL<T> &f = g.lv[l][i];
      f.t = f.d = f.r = f.bv = f.xv = nullptr;
      if (l + 1 < g.L) {
        f.t = ar.zeros<T>(f.n);
        f.d = ar.zeros<T>(f.n);
        f.r = ar.zeros<T>(f.n);
      }
      f.c = ar.zeros<T>(f.n);
      f.e = ar.zeros<T>(f.n);
    }
  // level vectors of coarse levels; the coarsest ones contiguous for the coupled LU
  int64_t ctot = 0;
  for (int i = 0; i < g.nf; ++i) ctot += g.lv[g.L - 1][i].n;
  g.cb = g.cx = nullptr;
  if (g.L > 1 || g.mono) {
    g.cb = ar.zeros<T>(ctot);
    g.cx = ar.zeros<T>(ctot);
  }
  int64_t o = 0;
  for (int i = 0; i < g.nf; ++i) {
    for (int l = 1; l < g.L - 1; ++l) {
      g.lv[l][i].bv = ar.zeros<T>(g.lv[l][i].n);
      g.lv[l][i].xv = ar.zeros<T>(g.lv[l][i].n);
    }
    if (g.L > 1 || g.mono) {
      g.lv[g.L - 1][i].bv = g.cb + o;
      g.lv[g.L - 1][i].xv = g.cx + o;
    }
    o += g.lv[g.L - 1][i].n;
  }
}

template <typename T> struct Precond {
  int kind = 0, nf = 0, order = 0, sweeps = 1;
  int smoother = MFS_CHEBYSHEV, gs_sweeps = 1;
  bool use_tail = false;  // one-CTA V-cycle tails where they apply (mfs_params.vcycle_tail)
  T gs_omega = T(0.79);
  std::vector<int64_t> fsize, foff;
  DGroup<T> g0, g1;
  std::vector<int> G1, G2;
  std::map<std::pair<int, int>, dev::Sell> cross;
  std::vector<T *> dtinv, sr2, st;
  std::vector<FL<T>> ms;                // AMG(SIMPLE): level Schur complements S~^l
  std::vector<std::vector<T *>> ms_dtinv;  // AMG(SIMPLE): [level][predictor field] 1 / A~_11
  cudaStream_t s = nullptr;

  // (re)allocate every work vector in `ar` (setup, and each clone)
  void alloc_work(Arena &ar) {
    if (g0.L) alloc_group_work(ar, g0);
    if (g1.L) alloc_group_work(ar, g1);
    st.clear();
    sr2.clear();
    if (kind == MFS_SIMPLE) {
      for (int j : G1) st.push_back(ar.zeros<T>(fsize[j]));
      for (int k : G2) sr2.push_back(ar.zeros<T>(fsize[k]));
    }
    for (auto &f : ms) {
      f.t = ar.zeros<T>(f.n);
      f.d = ar.zeros<T>(f.n);
      f.c = ar.zeros<T>(f.n);
      f.e = ar.zeros<T>(f.n);
    }
  }

  // single-field smoother S^l_i; zero: x enters as 0; post: the application
  // after the coarse correction (Gauss-Seidel then sweeps backward)
  void smooth(FL<T> &f, const T *rhs, T *x, bool zero, bool post = false) {
    if (smoother == MFS_GS) {
      if (zero) dev::fill<T>(x, f.n, T(0), s);
      dev::gs_sweeps<T>(f.gs, f.dblk, rhs, x, gs_omega, gs_sweeps, post, s);
      return;
    }
    const int ns = (int)f.c1.size();
    T *cur = x, *oth = f.t;
    int k0 = 0;
    if (zero) {
      T *tgt = ((ns - 1) % 2 == 0) ? x : f.t;
      dev::smooth_first<T>(f.n, f.dinv, rhs, tgt, f.d, f.c2[0], s);
      cur = tgt;
      oth = tgt == x ? f.t : x;
      k0 = 1;
    }
    for (int k = k0; k < ns; ++k) {
      dev::smooth_step<T>(f.A, f.dinv, rhs, cur, oth, f.d, f.c1[k], f.c2[k], s);
      std::swap(cur, oth);
    }
    if (cur != x) dev::convert<T, T>(cur, x, f.n, s);
  }

  // the level above the coarsest, small enough that one CTA runs the rest of
  // the V-cycle (dev::vcycle_tail) with the same arithmetic
  bool tail_ok(const DGroup<T> &g, int i, int l) const {
    if (!use_tail || smoother == MFS_GS || l != g.L - 2) return false;
    const FL<T> &f = g.lv[l][i];
    const dev::DenseLU &lu = g.cf[i];
    const dev::Sell &A = f.A, &R = f.R, &P = f.P;
    if (!lu.inv || lu.n == 0 || A.kind != 1 || R.kind != 1 || P.kind != 1) return false;
    if (dev::cta_rows(A) || dev::cta_rows(R) || dev::cta_rows(P)) return false;
    if (!dev::tail_supported(A.br, R.br) || R.bc != A.br || P.br != A.br || P.bc != R.br) return false;
    if (f.c1.size() > 8 || lu.n != R.nrows()) return false;
    return dev::tail_smem_bytes(A.nrows(), lu.n, sizeof(T)) <= 48 * 1024;
  }

  // Algorithm 1 for field i of group g from level l, zero initial guess
  void vcycle(DGroup<T> &g, int i, int l, const T *rhs, T *x) {
    FL<T> &f = g.lv[l][i];
    if (l == g.L - 1) {
      dev::lu_solve<T>(g.cf[i], rhs, x, s);
      return;
    }
    if (tail_ok(g, i, l)) {
      dev::vcycle_tail<T>(f.A, f.dinv, f.R, f.P, g.cf[i], (int)f.c1.size(), f.c1.data(), f.c2.data(), rhs, x, s);
      return;
    }
    FL<T> &c = g.lv[l + 1][i];
    smooth(f, rhs, x, true);
    dev::spmv<T>(f.A, x, f.r, T(-1), T(1), rhs, s);
    dev::spmv<T>(f.R, f.r, c.bv, T(1), T(0), nullptr, s);
    vcycle(g, i, l + 1, c.bv, c.xv);
    dev::spmv<T>(f.P, c.xv, x, T(1), T(1), x, s);
    smooth(f, rhs, x, false, true);
  }

  static std::vector<std::vector<int>> orders(int order, int nf) {
    std::vector<int> fwd(nf), bwd(nf);
    for (int i = 0; i < nf; ++i) {
      fwd[i] = i;
      bwd[i] = nf - 1 - i;
    }
    if (order == MFS_FWD) return {fwd};
    if (order == MFS_BWD) return {bwd};
    return {fwd, bwd};
  }

  // block solve of BGS: one V-cycle, or for the single-level BGS(GS) the
  // Gauss-Seidel sweeps from zero on the fine block
  void leaf(DGroup<T> &g, int i, const T *rhs, T *x) {
    if (kind == MFS_BGS_GS) smooth(g.lv[0][i], rhs, x, true, false);
    else vcycle(g, i, 0, rhs, x);
  }

  // block Gauss-Seidel on level 0 of group g with V-cycle block solves
  void bgs(DGroup<T> &g, const std::vector<const T *> &b, const std::vector<T *> &x) {
    std::vector<char> nz(g.nf, 0);
    for (int sw = 0; sw < sweeps; ++sw)
      for (auto &seq : orders(order, g.nf))
        for (int i : seq) {
          FL<T> &f = g.lv[0][i];
          const T *rhs = b[i];
          for (int j = 0; j < g.nf; ++j) {
            if (!nz[j]) continue;
            const dev::Sell *M = g.block(0, i, j);
            if (!M) continue;
            dev::spmv<T>(*M, x[j], f.c, T(-1), T(1), rhs, s);
            rhs = f.c;
          }
          if (!nz[i]) {
            leaf(g, i, rhs, x[i]);
            nz[i] = 1;
          } else {
            leaf(g, i, rhs, f.e);
            dev::axpy<T>(x[i], f.e, T(1), f.n, s);
          }
        }
  }

  void mono_smooth(DGroup<T> &g, int l, const std::vector<const T *> &b, const std::vector<T *> &x, bool zero,
                   bool post) {
    std::vector<char> nz(g.nf, zero ? 0 : 1);
    for (int sw = 0; sw < sweeps; ++sw)
      for (auto &seq : orders(order, g.nf))
        for (int i : seq) {
          FL<T> &f = g.lv[l][i];
          const T *rhs = b[i];
          for (int j = 0; j < g.nf; ++j) {
            if (j == i || !nz[j]) continue;
            const dev::Sell *M = g.block(l, i, j);
            if (!M) continue;
            dev::spmv<T>(*M, x[j], f.c, T(-1), T(1), rhs, s);
            rhs = f.c;
          }
          smooth(f, rhs, x[i], !nz[i], post);
          nz[i] = 1;
        }
  }

  void mono_cycle(DGroup<T> &g, int l, const std::vector<const T *> &b, const std::vector<T *> &x) {
    if (l == g.L - 1) {
      for (int i = 0; i < g.nf; ++i)
        if (b[i] != g.lv[l][i].bv)
          dev::convert<T, T>(b[i], g.lv[l][i].bv, g.lv[l][i].n, s);
      dev::lu_solve<T>(g.cc, g.cb, g.cx, s);
      for (int i = 0; i < g.nf; ++i)
        if (x[i] != g.lv[l][i].xv)
          dev::convert<T, T>(g.lv[l][i].xv, x[i], g.lv[l][i].n, s);
      return;
    }
    level_smooth(g, l, b, x, true);
    std::vector<const T *> bc(g.nf);
    std::vector<T *> xc(g.nf);
    for (int i = 0; i < g.nf; ++i) {
      FL<T> &f = g.lv[l][i];
      dev::spmv<T>(f.A, x[i], f.r, T(-1), T(1), b[i], s);
      for (int j = 0; j < g.nf; ++j) {
        if (j == i) continue;
        const dev::Sell *M = g.block(l, i, j);
        if (M) dev::spmv<T>(*M, x[j], f.r, T(-1), T(1), f.r, s);
      }
      dev::spmv<T>(f.R, f.r, g.lv[l + 1][i].bv, T(1), T(0), nullptr, s);
      bc[i] = g.lv[l + 1][i].bv;
      xc[i] = g.lv[l + 1][i].xv;
    }
    mono_cycle(g, l + 1, bc, xc);
    for (int i = 0; i < g.nf; ++i) dev::spmv<T>(g.lv[l][i].P, xc[i], x[i], T(1), T(1), x[i], s);
    level_smooth(g, l, b, x, false);
  }

  // pre-smoothing enters with x = 0, post-smoothing after the coarse correction
  void level_smooth(DGroup<T> &g, int l, const std::vector<const T *> &b, const std::vector<T *> &x, bool zero) {
    if (kind == MFS_AMG_SIMPLE) simple_smooth(g, l, b, x, zero, !zero);
    else mono_smooth(g, l, b, x, zero, !zero);
  }

  // AMG(SIMPLE) level smoother: r = b - A x; one BGS sweep of the field
  // smoothers over the predictor fields (into e); one smoother application on
  // S~^l (into its e); e_1 -= A~11^-1 A_12 e_2; x += e.
  void simple_smooth(DGroup<T> &g, int l, const std::vector<const T *> &b, const std::vector<T *> &x, bool zero,
                     bool post) {
    const int k = G2[0];
    FL<T> &sk = ms[l];
    for (int sw = 0; sw < sweeps; ++sw) {
      std::vector<const T *> r(g.nf);
      for (int i = 0; i < g.nf; ++i) {
        if (zero) {
          r[i] = b[i];
          continue;
        }
        FL<T> &f = g.lv[l][i];
        dev::spmv<T>(f.A, x[i], f.r, T(-1), T(1), b[i], s);
        for (int j = 0; j < g.nf; ++j) {
          if (j == i) continue;
          const dev::Sell *M = g.block(l, i, j);
          if (M) dev::spmv<T>(*M, x[j], f.r, T(-1), T(1), f.r, s);
        }
        r[i] = f.r;
      }
      std::vector<char> done(g.nf, 0);
      const int n1 = (int)G1.size();
      for (auto &seq : orders(order, n1))
        for (int jj : seq) {
          const int i = G1[jj];
          FL<T> &f = g.lv[l][i];
          const T *rhs = r[i];
          for (int q : G1) {
            if (q == i || !done[q]) continue;
            const dev::Sell *M = g.block(l, i, q);
            if (!M) continue;
            dev::spmv<T>(*M, g.lv[l][q].e, f.c, T(-1), T(1), rhs, s);
            rhs = f.c;
          }
          if (!done[i]) {
            smooth(f, rhs, f.e, true, post);
            done[i] = 1;
          } else {  // second visit of a symmetric sweep: correction form
            smooth(f, rhs, f.e, false, post);
          }
        }
      const T *rhs2 = r[k];
      for (int j : G1) {
        const dev::Sell *M = g.block(l, k, j);
        if (!M) continue;
        dev::spmv<T>(*M, g.lv[l][j].e, sk.c, T(-1), T(1), rhs2, s);
        rhs2 = sk.c;
      }
      smooth(sk, rhs2, sk.e, true, post);
      for (int jj = 0; jj < n1; ++jj) {
        const int j = G1[jj];
        const dev::Sell *M = g.block(l, j, k);
        if (!M) continue;
        FL<T> &f = g.lv[l][j];
        dev::spmv<T>(*M, sk.e, f.c, T(1), T(0), nullptr, s);
        dev::axpy_diag<T>(f.e, ms_dtinv[l][jj], f.c, f.n, s);
      }
      for (int j : G1) {
        FL<T> &f = g.lv[l][j];
        if (zero) dev::convert<T, T>(f.e, x[j], f.n, s);
        else dev::axpy<T>(x[j], f.e, T(1), f.n, s);
      }
      if (zero) dev::convert<T, T>(sk.e, x[k], sk.n, s);
      else dev::axpy<T>(x[k], sk.e, T(1), sk.n, s);
      zero = false;
    }
  }

  void apply(const T *in, T *out) {
    std::vector<const T *> b(nf);
    std::vector<T *> x(nf);
    for (int i = 0; i < nf; ++i) {
      b[i] = in + foff[i];
      x[i] = out + foff[i];
    }
    if (kind == MFS_BGS_AMG || kind == MFS_BGS_GS) {
      bgs(g0, b, x);
    } else if (kind == MFS_AMG_BGS || kind == MFS_AMG_SIMPLE) {
      mono_cycle(g0, 0, b, x);
    } else {
      std::vector<const T *> b1, b2;
      std::vector<T *> x1, x2;
      for (int j : G1) {
        b1.push_back(b[j]);
        x1.push_back(x[j]);
      }
      for (int k : G2) x2.push_back(x[k]);
      // predictor: one V-cycle, one BGS(AMG) sweep or one AMG(BGS) V-cycle
      if (g0.mono) mono_cycle(g0, 0, b1, x1);
      else if (G1.size() == 1) vcycle(g0, 0, 0, b1[0], x1[0]);
      else bgs(g0, b1, x1);
      // Schur right-hand side b_2 - A_21 dx_1
      for (size_t kk = 0; kk < G2.size(); ++kk) {
        const T *rhs = b[G2[kk]];
        for (size_t jj = 0; jj < G1.size(); ++jj) {
          auto it = cross.find({G2[kk], G1[jj]});
          if (it == cross.end()) continue;
          dev::spmv<T>(it->second, x1[jj], sr2[kk], T(-1), T(1), rhs, s);
          rhs = sr2[kk];
        }
        b2.push_back(rhs);
      }
      if (G2.size() == 1) vcycle(g1, 0, 0, b2[0], x2[0]);
      else bgs(g1, b2, x2);
      // update x_1 = dx_1 - A~11^-1 A_12 dx_2
      for (size_t jj = 0; jj < G1.size(); ++jj) {
        bool any = false;
        for (size_t kk = 0; kk < G2.size(); ++kk) {
          auto it = cross.find({G1[jj], G2[kk]});
          if (it == cross.end()) continue;
          dev::spmv<T>(it->second, x2[kk], st[jj], T(1), any ? T(1) : T(0), any ? st[jj] : nullptr, s);
          any = true;
        }
        if (any) dev::axpy_diag<T>(x1[jj], dtinv[jj], st[jj], fsize[G1[jj]], s);
      }
    }
  }
};

// Per-launch CUDA-event accounting (enabled by params.profile).  Direct
// launches take events from a pool that is read back at each collect();
// launches recorded while a graph is being captured become external event
// record nodes of that graph, owned by the graph's record list and read back
// after every replay.
struct ProfRec {
  cudaEvent_t e0, e1;
  int cls, sig;
  int64_t rows;
  double bytes, flops;
};

struct KStat {
  double launches = 0, ms = 0, bytes = 0, flops = 0;
};

struct EventProf : dev::LaunchHook {
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> *cap_events = nullptr;  // non-null while capturing
  std::vector<ProfRec> *cap_recs = nullptr;
  std::vector<const std::vector<ProfRec> *> pending;  // graph records replayed since the last collect
  cudaEvent_t open = nullptr;
  KStat cls[dev::K_NCLASS];
  std::map<std::pair<int, int64_t>, KStat> detail;  // (cls*100000 + sig, rows)

  cudaEvent_t take() {
    if (cap_events) {
      cudaEvent_t e;
      MFS_CUDA(cudaEventCreate(&e));
      cap_events->push_back(e);
      return e;
    }
    if (used == pool.size()) {
      cudaEvent_t e;
      MFS_CUDA(cudaEventCreate(&e));
      pool.push_back(e);
    }
    return pool[used++];
  }
  void record(cudaEvent_t e, cudaStream_t s) {
    if (cap_events) MFS_CUDA(cudaEventRecordWithFlags(e, s, cudaEventRecordExternal));
    else MFS_CUDA(cudaEventRecord(e, s));
  }
  int filter_key = 0;        // 0: record every launch; else only cls*100000 + sig ...
  int64_t filter_rows = 0;   // ... with this many rows (0: any)
  bool before(cudaStream_t s, int c, int sig, int64_t rows) override {
    if (filter_key && (c * 100000 + sig != filter_key || (filter_rows && rows != filter_rows))) return false;
    open = take();
    record(open, s);
    return true;
  }
  void after(cudaStream_t s, int c, double b, int sig, int64_t rows, double f) override {
    cudaEvent_t e1 = take();
    record(e1, s);
    ProfRec r{open, e1, c, sig, rows, b, f};
    (cap_recs ? cap_recs : &recs)->push_back(r);
  }
  void add(const ProfRec &r) {
    float t = 0.f;
    MFS_CUDA(cudaEventElapsedTime(&t, r.e0, r.e1));
    KStat &a = cls[r.cls];
    a.launches += 1;
    a.ms += t;
    a.bytes += r.bytes;
    a.flops += r.flops;
    KStat &d = detail[{r.cls * 100000 + r.sig, r.rows}];
    d.launches += 1;
    d.ms += t;
    d.bytes += r.bytes;
    d.flops += r.flops;
  }
  // caller has synchronised the stream
  void collect() {
    for (auto &r : recs) add(r);
    recs.clear();
    used = 0;
    for (auto *g : pending)
      for (auto &r : *g) add(r);
    pending.clear();
  }
  void reset() {
    for (auto &c : cls) c = KStat();
    detail.clear();
  }
  ~EventProf() override {
    for (auto e : pool) cudaEventDestroy(e);
  }
};

// One captured GMRES iteration body (fixed pointers for a given Krylov index).
struct IterGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaEvent_t> events;
  std::vector<ProfRec> recs;
  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    for (auto e : events) cudaEventDestroy(e);
    exec = nullptr;
    events.clear();
    recs.clear();
  }
};

// Host copy of the hierarchy (for the export calls), shared by clones.
struct HostSide {
  HGroup hg0, hg1;
  std::vector<std::vector<double>> dtilde;
  std::vector<std::vector<std::vector<double>>> mono_dtilde;  // AMG(SIMPLE): [level][predictor field]
  BlockMap schur_off;
  std::vector<HBsr> schur_diag;
  std::vector<int> G1, G2;
};

}  // namespace mfs

using namespace mfs;

constexpr int kHostSlots = 520;  // doubles in hdev / hpin
constexpr int kDotSlot = 512;

struct mfs_handle {
  mfs_params prm{};
  const std::map<std::pair<int, int>, RawDev> *raw = nullptr;  // input blocks on the device (setup only)
  int nf = 0;
  std::vector<int64_t> fsize, foff;
  int64_t n = 0;
  cudaStream_t s = nullptr;
  Arena ar;
  std::map<std::pair<int, int>, dev::Sell> A64;
  std::vector<dev::RowMerged> rows64;  // per row field, when its blocks share one pattern
  std::unique_ptr<Precond<double>> p64;
  std::unique_ptr<Precond<float>> p32;
  std::shared_ptr<HostSide> host = std::make_shared<HostSide>();
  std::shared_ptr<Arena> mat = std::make_shared<Arena>();  // matrices, shared by clones
  int device = 0;
  bool host_only = false;
  // solve workspace
  int m = 0, nblk = 1;
  double *V = nullptr, *Z = nullptr, *xd = nullptr, *bd = nullptr, *rd = nullptr, *partial = nullptr;
  double *hdev = nullptr, *ydev = nullptr;
  float *in32 = nullptr, *out32 = nullptr;
  // hdev / hpin: the Arnoldi sums of iterations of even and odd Krylov index
  // at 0 and 256 (136 each), a dot product at kDotSlot
  double *hpin = nullptr;
  cudaEvent_t iter_ev[2] = {nullptr, nullptr};  // completion of the last iteration of each parity
  double setup_ms = 0.0;
  std::unique_ptr<EventProf> prof;
  bool own_stream = false;
  cudaEvent_t entry = nullptr;
  bool use_graphs = true;
  std::vector<IterGraph> graphs;  // per Krylov index j
  ~mfs_handle() {
    for (auto &g : graphs) g.release();
    if (hpin) g_pinned.put(hpin, kHostSlots * sizeof(double));
    for (auto e : iter_ev)
      if (e) cudaEventDestroy(e);
    if (entry) cudaEventDestroy(entry);
    if (own_stream && s) cudaStreamDestroy(s);
  }
};

namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void matvec(mfs_handle *h, const double *x, double *y) {
  if (!h->rows64.empty()) {
    for (int i = 0; i < h->nf; ++i) dev::spmv_rows(h->rows64[i], x, y + h->foff[i], h->s);
    return;
  }
  for (int i = 0; i < h->nf; ++i) {
    bool first = true;
    for (int j = 0; j < h->nf; ++j) {
      auto it = h->A64.find({i, j});
      if (it == h->A64.end()) continue;
      dev::spmv<double>(it->second, x + h->foff[j], y + h->foff[i], 1.0, first ? 0.0 : 1.0,
                        first ? nullptr : y + h->foff[i], h->s);
      first = false;
    }
    if (first) dev::fill<double>(y + h->foff[i], h->fsize[i], 0.0, h->s);
  }
}

void precond_apply(mfs_handle *h, const double *v, double *z, bool staged = false) {
  if (h->p64) {
    h->p64->apply(v, z);
  } else {
    if (!staged) dev::convert<double, float>(v, h->in32, h->n, h->s);  // staged: in32 holds v already
    h->p32->apply(h->in32, h->out32);
    dev::convert<float, double>(h->out32, z, h->n, h->s);
  }
}

// ||x||^2 of n doubles, deterministic, result in host memory
double dot_host(mfs_handle *h, const double *x, const double *y) {
  dev::mdot(x, 0, 1, y, h->n, h->partial, h->nblk, h->s);
  dev::reduce_partials(h->partial, 1, h->nblk, h->hdev + kDotSlot, h->s);
  MFS_CUDA(cudaMemcpyAsync(h->hpin + kDotSlot, h->hdev + kDotSlot, sizeof(double), cudaMemcpyDeviceToHost, h->s));
  dev::pdl_break();
  MFS_CUDA(cudaStreamSynchronize(h->s));
  return h->hpin[kDotSlot];
}

// Capture body() once per Krylov index j into a CUDA graph and replay it:
// one launch per GMRES iteration instead of one per kernel.
template <typename F> void run_graph(mfs_handle *h, int j, F &&body, bool prof) {
  IterGraph &g = h->graphs[j];
  if (!g.exec) {
    if (prof) {
      h->prof->cap_events = &g.events;
      h->prof->cap_recs = &g.recs;
    }
    cudaGraph_t graph = nullptr;
    MFS_CUDA(cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal));
    dev::pdl_break();  // the graph's first kernel has no kernel before it
    try {
      body();
    } catch (...) {
      cudaStreamEndCapture(h->s, &graph);
      if (graph) cudaGraphDestroy(graph);
      if (prof) h->prof->cap_events = nullptr, h->prof->cap_recs = nullptr;
      g.release();
      throw;
    }
    if (prof) h->prof->cap_events = nullptr, h->prof->cap_recs = nullptr;
    MFS_CUDA(cudaStreamEndCapture(h->s, &graph));
    const cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    MFS_CUDA(e);
  }
  MFS_CUDA(cudaGraphLaunch(g.exec, h->s));
  dev::pdl_break();
  if (prof) h->prof->pending.push_back(&g.recs);
}

// Host side of FGMRES(m): the Hessenberg columns, their Givens rotations,
// the least-squares right-hand side g and the back substitution (shared by
// the single-system loop and the fused batch, so both do the same
// arithmetic in the same order).
struct KrylovLS {
  int m = 0;
  std::vector<double> H, cs, sn, g, y;
  double r0 = 0.0, est = 1.0, hn = 0.0;
  int iters = 0, jend = 0;
  bool happy = false;
  explicit KrylovLS(int m_ = 0) : m(m_), H((size_t)(m_ + 1) * m_), cs(m_), sn(m_), g(m_ + 1), y(m_) {}
  void start_cycle(double beta) {
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    jend = 0;
  }
  // column j from the Arnoldi sums hp (h1 at [0, j], |w|^2 before the
  // projections at [j + 1], h2 at [64, 64 + j], |w|^2 after at [128]);
  // false when a sum is not finite
  bool column(const double *hp, int j) {
    const double nw0 = std::sqrt(hp[j + 1]);
    hn = std::sqrt(hp[128]);
    if (!std::isfinite(hn) || !std::isfinite(nw0)) return false;
    double *Hj = H.data() + (size_t)j * (m + 1);  // column j
    for (int k = 0; k <= j; ++k) Hj[k] = hp[k] + hp[64 + k];
    Hj[j + 1] = hn;
    for (int k = 0; k < j; ++k) {
      const double a = Hj[k], c = Hj[k + 1];
      Hj[k] = cs[k] * a + sn[k] * c;
      Hj[k + 1] = -sn[k] * a + cs[k] * c;
    }
    if (Hj[j + 1] == 0.0) {
      cs[j] = 1.0;
      sn[j] = 0.0;
    } else {
      const double rr = std::hypot(Hj[j], Hj[j + 1]);
      cs[j] = Hj[j] / rr;
      sn[j] = Hj[j + 1] / rr;
    }
    Hj[j] = cs[j] * Hj[j] + sn[j] * Hj[j + 1];
    Hj[j + 1] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    ++iters;
    jend = j + 1;
    est = std::fabs(g[j + 1]) / r0;
    happy = hn <= 1e-14 * nw0;
    return true;
  }
  void back_substitute() {
    for (int k = jend - 1; k >= 0; --k) {
      double sum = g[k];
      for (int q = k + 1; q < jend; ++q) sum -= H[(size_t)q * (m + 1) + k] * y[q];
      y[k] = sum / H[(size_t)k * (m + 1) + k];
    }
  }
};

// one CGS2 Arnoldi step on w = A z_j against V_0..V_j: the sums of the host
// update land in hd (see KrylovLS::column)
void arnoldi(mfs_handle *h, int j, double *w, double *hd, cudaStream_t s) {
  const int64_t n = h->n;
  // CGS2: h1 = V^T w (and |w|^2), w -= V h1, h2 = V^T w, w -= V h2 (and |w|^2)
  dev::mdot(h->V, n, j + 2, w, n, h->partial, h->nblk, s);
  dev::reduce_partials(h->partial, j + 2, h->nblk, hd, s);
  dev::cgs_fused(h->V, n, j + 1, hd, w, n, h->partial, h->nblk, s);
  dev::reduce_partials(h->partial, j + 1, h->nblk, hd + 64, s);
  dev::cgs_update(h->V, n, j + 1, hd + 64, w, n, h->partial, h->nblk, s);
  dev::reduce_partials(h->partial, 1, h->nblk, hd + 128, s);
}

// Solves and other solve-phase calls (apply, matvec) running in this process.
// A solve queues iterations ahead only while it runs alone: with other solves
// on the GPU its host turnaround is covered by their work, and queued-ahead
// iterations measured slower for 16 concurrent solves.
static std::atomic<int> g_solves_running{0};

// One solve-phase call: counted in g_solves_running, and its launches made
// programmatic dependent launches as mfs_params.pdl says.  The automatic
// choice: every launch of a small system, the launches of at most 160 CTAs
// (coarse levels, reductions) of a larger one - its big launches measured
// slower that way - and only while the call runs alone (16 concurrent solves
// of small systems measured 2 % slower with them).
struct SolvePhase {
  explicit SolvePhase(const mfs_handle *h) {
    const bool alone = ++g_solves_running == 1;
    const int p = h->prm.pdl;
    dev::set_pdl(p == 1 ? ~0u : p > 1 ? (unsigned)p : (p == -1 && alone) ? (h->n <= 65536 ? ~0u : 160u) : 0u);
  }
  ~SolvePhase() {
    dev::set_pdl(0);
    --g_solves_running;
  }
};

int fgmres(mfs_handle *h, const double *b, double *x, double tol, mfs_info *info, bool prof) {
  SolvePhase phase(h);
  const int64_t n = h->n;
  const int m = h->m;
  cudaStream_t s = h->s;
  double *r = h->rd;
  // r = b - A x
  matvec(h, x, r);
  dev::axpy<double>(r, b, -1.0, n, s);
  dev::scale(r, -1.0, r, n, s);
  const double r0 = std::sqrt(dot_host(h, r, r));
  int restarts = 0;
  double relres = 0.0;
  if (r0 == 0.0) {
    info->iters = 0;
    info->converged = 1;
    info->true_relres = 0.0;
    info->est_relres = 0.0;
    return MFS_OK;
  }
  if (!std::isfinite(r0)) return MFS_ERR_BREAKDOWN;
  KrylovLS ls(m);
  ls.r0 = r0;
  double *hdb[2] = {h->hdev, h->hdev + 256};
  double *hpb[2] = {h->hpin, h->hpin + 256};
  // Iteration j of a cycle: for j > 0 v_j = w / |w| (w = V_j as the previous
  // iteration left it, its norm read on the device), z_j = P^-1 v_j,
  // w = A z_j and the CGS2 passes, whose sums land in buffer j % 2 (device
  // and pinned host), then event j % 2.  Nothing in it waits for the host's
  // Givens step of iteration j - 1, so iteration j + 1 is queued before the
  // host reads column j unless the residual estimate says iteration j may end
  // the cycle (and this solve runs alone in the process); the GPU then runs
  // the iterations back to back.  An iteration
  // queued past the end of a cycle writes only V_{j+2}, Z_{j+1} and its own
  // buffers, none of which the cycle end reads.
  auto enqueue = [&](int j) {
    double *vj = h->V + (int64_t)j * n;
    double *zj = h->Z + (int64_t)j * n;
    double *w = h->V + (int64_t)(j + 1) * n;
    auto body = [&]() {
      if (j > 0) {
        const double *nrm2 = hdb[(j - 1) & 1] + 128;
        if (h->p32) dev::scale_convert_dev<float>(vj, nrm2, h->in32, n, s);
        else dev::scale_convert_dev<double>(vj, nrm2, nullptr, n, s);
      }
      precond_apply(h, vj, zj, j > 0);
      matvec(h, zj, w);
      arnoldi(h, j, w, hdb[j & 1], s);
      MFS_CUDA(cudaMemcpyAsync(hpb[j & 1], hdb[j & 1], 136 * sizeof(double), cudaMemcpyDeviceToHost, s));
      dev::pdl_break();
    };
    if (h->use_graphs) run_graph(h, j, body, prof);
    else body();
    MFS_CUDA(cudaEventRecord(h->iter_ev[j & 1], s));
    dev::pdl_break();
  };
  auto fail_drained = [&](int code) {  // no queued iteration may outlive the call
    cudaStreamSynchronize(s);
    return code;
  };
  while (true) {
    const double beta = restarts == 0 ? r0 : std::sqrt(dot_host(h, r, r));
    if (prof) h->prof->collect();  // the stream is idle here
    dev::scale(r, 1.0 / beta, h->V, n, s);
    ls.start_cycle(beta);
    double e_last = beta / r0, rho = 1.0;  // last estimate and its last ratio
    int queued = 0;
    enqueue(queued++);
    for (int j = 0; j < m; ++j) {
      // queue iteration j + 1 ahead unless iteration j may end the cycle
      // (predicted estimate: the last one times the last ratio cubed)
      if (queued == j + 1 && j + 1 < m && ls.iters + 2 <= h->prm.max_iters && e_last * rho * rho * rho > tol &&
          g_solves_running.load() == 1)
        enqueue(queued++);
      MFS_CUDA(cudaEventSynchronize(h->iter_ev[j & 1]));
      if (!ls.column(hpb[j & 1], j)) return fail_drained(MFS_ERR_BREAKDOWN);
      if (ls.est <= tol || ls.happy || ls.iters >= h->prm.max_iters) break;
      rho = std::min(1.0, ls.est / e_last);
      e_last = ls.est;
      if (queued == j + 1 && j + 1 < m) enqueue(queued++);
    }
    ls.back_substitute();
    MFS_CUDA(cudaMemcpyAsync(h->ydev, ls.y.data(), ls.jend * sizeof(double), cudaMemcpyHostToDevice, s));
    dev::pdl_break();
    dev::gemv_add(h->Z, n, ls.jend, h->ydev, x, n, s);
    matvec(h, x, r);
    dev::axpy<double>(r, b, -1.0, n, s);
    dev::scale(r, -1.0, r, n, s);
    relres = std::sqrt(dot_host(h, r, r)) / r0;
    if (!std::isfinite(relres)) return MFS_ERR_BREAKDOWN;
    if (relres <= tol || ls.iters >= h->prm.max_iters) break;
    ++restarts;
  }
  if (prof) h->prof->collect();
  info->iters = ls.iters;
  info->restarts = restarts;
  info->true_relres = relres;
  info->est_relres = ls.est;
  info->converged = relres <= tol ? 1 : 0;
  return info->converged ? MFS_OK : MFS_ERR_NOT_CONVERGED;
}

// ---------------------------------------------------------------------------
// Fused batch: the FGMRES iterations of a group of independent systems
// advance in lockstep, each step of an iteration being ONE launch over all of
// them.  Every system's launch sequence (its preconditioner application,
// recorded once from the same code that issues a solo solve, plus the Krylov
// steps, re-recorded every iteration with that iteration's vectors) is merged
// with the others' into multi-system launches: kernel K runs the blocks of
// every system's launch of K in one grid, each CTA reading its system's
// argument block from a table (the k_multi form of K).  The merged launches
// form one CUDA graph per group, replayed once per iteration; a per-system
// flag stops the CTAs of systems that have finished.  Each system's kernels,
// arguments and order are the ones of its solo solve, so its result is the
// solo result bit for bit.  Restarts and the end of a cycle (x update, true
// residual) run as ordinary launches for the systems concerned.  A batch is
// split into groups of similar systems, each driven by its own host thread
// (mfs_solve_batch).
// ---------------------------------------------------------------------------

// Merge per-system launch sequences: repeatedly take the kernel (and block
// size) shared by most systems' next launches - ties to the systems with
// more launches left - and issue it for all of them at once; each system's
// launches keep their order.  groups[g] = (system, index) of merged launch g.
static void merge_sequences(const std::vector<const std::vector<dev::RecOp> *> &seqs,
                            std::vector<std::vector<std::pair<int, int>>> &groups) {
  const size_t ns = seqs.size();
  std::vector<size_t> p(ns, 0);
  while (true) {
    std::map<std::pair<const void *, unsigned>, std::pair<int, size_t>> cnt;
    for (size_t k = 0; k < ns; ++k) {
      if (p[k] >= seqs[k]->size()) continue;
      const dev::RecOp &op = (*seqs[k])[p[k]];
      auto &c = cnt[{op.fn, op.threads}];
      c.first += 1;
      c.second = std::max(c.second, seqs[k]->size() - p[k]);
    }
    if (cnt.empty()) break;
    auto best = cnt.begin();
    for (auto it = cnt.begin(); it != cnt.end(); ++it)
      if (it->second.first > best->second.first ||
          (it->second.first == best->second.first && it->second.second > best->second.second))
        best = it;
    std::vector<std::pair<int, int>> grp;
    for (size_t k = 0; k < ns; ++k) {
      if (p[k] >= seqs[k]->size()) continue;
      const dev::RecOp &op = (*seqs[k])[p[k]];
      if (op.fn == best->first.first && op.threads == best->first.second) {
        grp.push_back({(int)k, (int)p[k]});
        ++p[k];
      }
    }
    groups.push_back(std::move(grp));
  }
}

struct FusedBatch {
  std::vector<mfs_handle *> hs;
  int nsys = 0;
  cudaStream_t s = nullptr;
  Arena ar;
  struct Launch {
    dev::RecOp proto;       // kernel and block size
    unsigned grid = 0;      // CTAs over all entries
    size_t smem = 0;        // largest entry's dynamic shared memory
    size_t tab = 0, map = 0, asz = 0;
    int nent = 0;
    std::vector<int> sys;  // the system of each entry
  };
  std::vector<Launch> launches;  // in issue order: heads, preconditioners, tails
  // per system: (launch, entry) of each of its head / tail launches
  std::vector<std::vector<std::pair<int, int>>> head_at, tail_at;
  unsigned char *htab = nullptr;  // pinned host copy of every argument table
  size_t tab_bytes = 0, patch_bytes = 0;
  unsigned char *dtab = nullptr;
  dev::MsBlock *dmap = nullptr;
  int *dactive = nullptr, *hactive = nullptr;
  double *hb = nullptr, *hbpin = nullptr, *ypin = nullptr;  // Arnoldi sums (136 per system), y (64 per system)
  std::vector<double *> vin, zout;  // float64 systems: fixed preconditioner input / output
  cudaGraphExec_t exec = nullptr;
  size_t nhead = 0, npre = 0, ntail = 0;  // merged launches per segment
  int64_t ctas = 0;                       // CTAs of one replay
  double build_ms = 0.0;
  bool own_stream = true;
  // plans over the systems still running, once at most half of this plan's
  // are (keyed by their positions in this plan; kept for later calls)
  std::map<std::vector<int>, std::unique_ptr<FusedBatch>> subs;
  FusedBatch() = default;
  FusedBatch(const FusedBatch &) = delete;
  ~FusedBatch() {
    subs.clear();
    if (s) cudaStreamSynchronize(s);
    if (exec) cudaGraphExecDestroy(exec);
    g_pinned.put(htab, std::max<size_t>(tab_bytes, 16));
    g_pinned.put(hactive, (size_t)nsys * sizeof(int));
    g_pinned.put(hbpin, (size_t)136 * nsys * sizeof(double));
    g_pinned.put(ypin, (size_t)64 * nsys * sizeof(double));
    if (s && own_stream) cudaStreamDestroy(s);
  }
  double *sums(int k) { return hb + (int64_t)k * 136; }

  // launches of system k before its preconditioner: v_j = a v_j and the
  // preconditioner's copy of it
  void record_head(int k, int j, double a, dev::Recorder &rec) {
    mfs_handle *h = hs[k];
    double *vj = h->V + (int64_t)j * h->n;
    dev::set_recorder(&rec);
    if (h->p32) dev::scale_convert<float>(vj, a, h->in32, h->n, s);
    else dev::scale_convert<double>(vj, a, vin[k], h->n, s);
    dev::set_recorder(nullptr);
  }
  void record_precond(int k, dev::Recorder &rec) {
    mfs_handle *h = hs[k];
    dev::set_recorder(&rec);
    if (h->p32) h->p32->apply(h->in32, h->out32);
    else h->p64->apply(vin[k], zout[k]);
    dev::set_recorder(nullptr);
  }
  // after it: z_j, w = A z_j, CGS2 against V_0..V_j
  void record_tail(int k, int j, dev::Recorder &rec) {
    mfs_handle *h = hs[k];
    double *zj = h->Z + (int64_t)j * h->n;
    double *w = h->V + (int64_t)(j + 1) * h->n;
    dev::set_recorder(&rec);
    if (h->p32) dev::convert<float, double>(h->out32, zj, h->n, s);
    else dev::convert<double, double>(zout[k], zj, h->n, s);
    matvec(h, zj, w);
    arnoldi(h, j, w, sums(k), s);
    dev::set_recorder(nullptr);
  }

  // merge one segment; its launches go to `launches`, its tables at the
  // current end of the table layout
  void add_segment(std::vector<dev::Recorder> &recs, std::vector<std::vector<std::pair<int, int>>> *at,
                   std::vector<unsigned char> &tabs, std::vector<dev::MsBlock> &maps) {
    std::vector<const std::vector<dev::RecOp> *> seqs;
    for (auto &r : recs) seqs.push_back(&r.ops);
    std::vector<std::vector<std::pair<int, int>>> groups;
    merge_sequences(seqs, groups);
    if (at) {
      at->assign(nsys, {});
      for (int k = 0; k < nsys; ++k) (*at)[k].resize(recs[k].ops.size());
    }
    for (auto &grp : groups) {
      Launch L;
      const dev::RecOp &p0 = recs[grp[0].first].ops[grp[0].second];
      L.proto = p0;
      L.proto.args.clear();
      L.asz = p0.args.size();
      L.nent = (int)grp.size();
      L.tab = (tabs.size() + 15) / 16 * 16;
      tabs.resize(L.tab + L.asz * grp.size());
      L.map = maps.size();
      for (size_t e = 0; e < grp.size(); ++e) {
        const dev::RecOp &op = recs[grp[e].first].ops[grp[e].second];
        if (op.args.size() != L.asz) throw CudaError(MFS_ERR_INVALID, "fused batch: argument blocks differ");
        std::memcpy(tabs.data() + L.tab + e * L.asz, op.args.data(), L.asz);
        for (unsigned b = 0; b < op.grid; ++b) maps.push_back({(int)e, (int)b, (int)op.grid, grp[e].first});
        L.grid += op.grid;
        L.smem = std::max(L.smem, op.smem);
        if (at) (*at)[grp[e].first][grp[e].second] = {(int)launches.size(), (int)e};
        L.sys.push_back(grp[e].first);
      }
      launches.push_back(std::move(L));
    }
  }

  // stream: the stream to run on (a sub-plan takes its parent's), or null
  // for a new library stream
  void build(mfs_handle *const *hv, int n, cudaStream_t stream = nullptr) {
    hs.assign(hv, hv + n);
    nsys = n;
    MFS_CUDA(cudaSetDevice(hs[0]->device));
    if (stream) {
      s = stream;
      own_stream = false;
    } else {
      MFS_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    }
    vin.assign(nsys, nullptr);
    zout.assign(nsys, nullptr);
    for (int k = 0; k < nsys; ++k)
      if (!hs[k]->p32) {
        vin[k] = ar.zeros<double>(hs[k]->n);
        zout[k] = ar.zeros<double>(hs[k]->n);
      }
    hb = ar.zeros<double>((int64_t)136 * nsys);
    dactive = ar.zeros<int>(nsys);
    hbpin = (double *)g_pinned.get((size_t)136 * nsys * sizeof(double));
    ypin = (double *)g_pinned.get((size_t)64 * nsys * sizeof(double));
    hactive = (int *)g_pinned.get((size_t)nsys * sizeof(int));
    std::vector<dev::Recorder> heads(nsys), pre(nsys), tails(nsys);
    for (int k = 0; k < nsys; ++k) {
      record_head(k, 0, 1.0, heads[k]);
      record_precond(k, pre[k]);
      record_tail(k, 0, tails[k]);
    }
    // tables of the per-iteration launches first (one upload per iteration)
    std::vector<unsigned char> tabs;
    std::vector<dev::MsBlock> maps;
    add_segment(heads, &head_at, tabs, maps);
    const size_t nhead = launches.size();
    add_segment(tails, &tail_at, tabs, maps);
    patch_bytes = tabs.size();
    const size_t ntail_end = launches.size();
    add_segment(pre, nullptr, tabs, maps);
    tab_bytes = tabs.size();
    // issue order: heads, preconditioners, tails
    std::vector<Launch> order;
    for (size_t i = 0; i < nhead; ++i) order.push_back(launches[i]);
    for (size_t i = ntail_end; i < launches.size(); ++i) order.push_back(launches[i]);
    std::vector<int> remap(launches.size());
    for (size_t i = nhead; i < ntail_end; ++i) order.push_back(launches[i]);
    for (size_t i = 0; i < nhead; ++i) remap[i] = (int)i;
    const size_t npre = launches.size() - ntail_end;
    for (size_t i = ntail_end; i < launches.size(); ++i) remap[i] = (int)(nhead + (i - ntail_end));
    for (size_t i = nhead; i < ntail_end; ++i) remap[i] = (int)(nhead + npre + (i - nhead));
    for (auto &v : head_at)
      for (auto &pr : v) pr.first = remap[pr.first];
    for (auto &v : tail_at)
      for (auto &pr : v) pr.first = remap[pr.first];
    launches.swap(order);
    this->nhead = nhead;
    this->npre = npre;
    ntail = ntail_end - nhead;
    for (const Launch &L : launches) ctas += L.grid;
    htab = (unsigned char *)g_pinned.get(std::max<size_t>(tab_bytes, 16));
    std::memcpy(htab, tabs.data(), tab_bytes);
    dtab = ar.alloc<unsigned char>((int64_t)std::max<size_t>(tab_bytes, 16));
    dmap = ar.alloc<dev::MsBlock>((int64_t)std::max<size_t>(maps.size(), 1));
    MFS_CUDA(cudaMemcpyAsync(dtab, htab, tab_bytes, cudaMemcpyHostToDevice, s));
    MFS_CUDA(cudaMemcpyAsync(dmap, maps.data(), maps.size() * sizeof(dev::MsBlock), cudaMemcpyHostToDevice, s));
    MFS_CUDA(cudaStreamSynchronize(s));
    MFS_CUDA(cudaStreamSynchronize(0));
    // one graph: every merged launch, then the Arnoldi sums to the host.  A
    // launch depends on the previous launches of the systems it serves, so
    // launches over disjoint sets of systems (where the systems' sequences
    // differ) may run at the same time; each system's own launches keep
    // their order.
    cudaGraph_t graph = nullptr;
    MFS_CUDA(cudaGraphCreate(&graph, 0));
    struct GraphGuard {
      cudaGraph_t &g;
      ~GraphGuard() {
        if (g) cudaGraphDestroy(g);
      }
    } guard{graph};
    std::vector<cudaGraphNode_t> last(nsys, nullptr);
    std::vector<cudaGraphNode_t> deps;
    for (const Launch &L : launches) {
      deps.clear();
      for (int k : L.sys)
        if (last[k] && std::find(deps.begin(), deps.end(), last[k]) == deps.end()) deps.push_back(last[k]);
      const void *tab = dtab + L.tab;
      const dev::MsBlock *map = dmap + L.map;
      const int *act = dactive;
      void *kargs[3] = {(void *)&tab, (void *)&map, (void *)&act};
      cudaKernelNodeParams kp{};
      kp.func = const_cast<void *>(L.proto.fn);
      kp.gridDim = dim3(L.grid);
      kp.blockDim = dim3(L.proto.threads);
      kp.sharedMemBytes = (unsigned)L.smem;
      kp.kernelParams = kargs;
      cudaGraphNode_t node = nullptr;
      MFS_CUDA(cudaGraphAddKernelNode(&node, graph, deps.data(), deps.size(), &kp));
      for (int k : L.sys) last[k] = node;
    }
    deps.clear();
    for (cudaGraphNode_t n : last)
      if (n && std::find(deps.begin(), deps.end(), n) == deps.end()) deps.push_back(n);
    cudaGraphNode_t copy = nullptr;
    MFS_CUDA(cudaGraphAddMemcpyNode1D(&copy, graph, deps.data(), deps.size(), hbpin, hb,
                                      (size_t)136 * nsys * sizeof(double), cudaMemcpyDeviceToHost));
    MFS_CUDA(cudaGraphInstantiate(&exec, graph, 0));
  }

  // the plan over this plan's systems at positions `live` (built on first use)
  FusedBatch *sub(const std::vector<int> &live) {
    auto it = subs.find(live);
    if (it != subs.end()) return it->second.get();
    if (subs.size() >= 16) subs.clear();
    std::vector<mfs_handle *> hv;
    for (int p : live) hv.push_back(hs[p]);
    std::unique_ptr<FusedBatch> b(new FusedBatch());
    b->build(hv.data(), (int)hv.size(), s);
    return subs.emplace(live, std::move(b)).first->second.get();
  }

  // write system k's freshly recorded launches into its slots of the tables
  void patch(const dev::Recorder &rec, const std::vector<std::pair<int, int>> &at) {
    if (rec.ops.size() != at.size()) throw CudaError(MFS_ERR_INVALID, "fused batch: launch sequence changed");
    for (size_t q = 0; q < rec.ops.size(); ++q) {
      const Launch &L = launches[at[q].first];
      if (rec.ops[q].args.size() != L.asz || rec.ops[q].fn != L.proto.fn)
        throw CudaError(MFS_ERR_INVALID, "fused batch: launch changed between iterations");
      std::memcpy(htab + L.tab + (size_t)at[q].second * L.asz, rec.ops[q].args.data(), L.asz);
    }
  }
};

// Systems in `ngroups` groups of about equal dof totals, each of systems of
// similar size (sorted by size, cut into consecutive runs; positions in hs).
static std::vector<std::vector<int>> size_groups(mfs_handle *const *hs, int nsys, int ngroups) {
  ngroups = std::max(1, std::min(ngroups, nsys));
  std::vector<int> order(nsys);
  for (int k = 0; k < nsys; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return hs[a]->n > hs[b]->n; });
  double total = 0.0;
  for (int k = 0; k < nsys; ++k) total += (double)hs[k]->n;
  std::vector<std::vector<int>> g(1);
  double acc = 0.0;
  for (int k : order) {
    if (!g.back().empty() && acc >= total * (double)g.size() / ngroups && (int)g.size() < ngroups) g.emplace_back();
    g.back().push_back(k);
    acc += (double)hs[k]->n;
  }
  for (auto &m : g) std::sort(m.begin(), m.end());
  return g;
}

// Process-wide cache of fused batches by their handle list (a batch holds
// the handles' device addresses; mfs_free drops every batch of a handle).
// (never destroyed itself: at process exit the CUDA runtime may already be
// gone, so the batches' streams and pinned buffers are left to the OS)
static std::mutex g_fused_mu;
static std::vector<std::unique_ptr<FusedBatch>> &g_fused = *new std::vector<std::unique_ptr<FusedBatch>>();

static void drop_fused(const mfs_handle *h) {
  std::lock_guard<std::mutex> lock(g_fused_mu);
  for (size_t i = 0; i < g_fused.size();)
    if (std::find(g_fused[i]->hs.begin(), g_fused[i]->hs.end(), h) != g_fused[i]->hs.end())
      g_fused.erase(g_fused.begin() + (long)i);
    else
      ++i;
}

static FusedBatch *fused_for(mfs_handle *const *hv, int n) {
  std::lock_guard<std::mutex> lock(g_fused_mu);
  for (auto &b : g_fused)
    if (b->nsys == n && std::equal(b->hs.begin(), b->hs.end(), hv))
      return b.get();
  std::unique_ptr<FusedBatch> b(new FusedBatch());
  const double t0 = now_ms();
  b->build(hv, n);
  b->build_ms = now_ms() - t0;
  if (hv[0]->prm.verbose)
    fprintf(stderr,
            "mfs fused batch: %d systems, %zu + %zu + %zu merged launches per iteration (heads, preconditioners, "
            "Krylov steps), %lld CTAs per replay, %.1f KB patched per iteration, built in %.1f ms\n",
            n, b->nhead, b->npre, b->ntail, (long long)b->ctas, b->patch_bytes / 1024.0, b->build_ms);
  if (g_fused.size() >= 64) g_fused.erase(g_fused.begin());
  g_fused.push_back(std::move(b));
  return g_fused.back().get();
}

// FGMRES of every system of the batch, lockstep (see FusedBatch).
static void fused_solve(FusedBatch &B, const double *const *rhs, double *const *x, double tol,
                        std::vector<mfs_info> &info, std::vector<int> &status) {
  const int ns = B.nsys;
  cudaStream_t s = B.s;
  std::vector<mfs_handle *> &hs = B.hs;
  // every launch of the handles' own code goes to the batch stream meanwhile
  std::vector<cudaStream_t> saved(ns);
  for (int k = 0; k < ns; ++k) {
    saved[k] = hs[k]->s;
    hs[k]->s = s;
    if (hs[k]->p32) hs[k]->p32->s = s;
    if (hs[k]->p64) hs[k]->p64->s = s;
  }
  struct Restore {
    std::vector<mfs_handle *> &hs;
    std::vector<cudaStream_t> &saved;
    ~Restore() {
      for (size_t k = 0; k < hs.size(); ++k) {
        hs[k]->s = saved[k];
        if (hs[k]->p32) hs[k]->p32->s = saved[k];
        if (hs[k]->p64) hs[k]->p64->s = saved[k];
      }
    }
  } restore{hs, saved};
  // the caller's vectors come from the legacy default stream
  cudaEvent_t entry = nullptr;
  MFS_CUDA(cudaEventCreateWithFlags(&entry, cudaEventDisableTiming));
  MFS_CUDA(cudaEventRecord(entry, 0));
  MFS_CUDA(cudaStreamWaitEvent(s, entry, 0));
  cudaEventDestroy(entry);
  for (int k = 0; k < ns; ++k) MFS_CUDA(cudaStreamSynchronize(saved[k]));
  std::vector<const double *> b(ns);
  std::vector<double *> xx(ns);
  std::vector<char> hostx(ns, 0);
  for (int k = 0; k < ns; ++k) {
    mfs_handle *h = hs[k];
    b[k] = rhs[k];
    xx[k] = x[k];
    if (!is_device_ptr(rhs[k])) {
      MFS_CUDA(cudaMemcpyAsync(h->bd, rhs[k], h->n * sizeof(double), cudaMemcpyHostToDevice, s));
      b[k] = h->bd;
    }
    if (!is_device_ptr(x[k])) {
      MFS_CUDA(cudaMemcpyAsync(h->xd, x[k], h->n * sizeof(double), cudaMemcpyHostToDevice, s));
      xx[k] = h->xd;
      hostx[k] = 1;
    }
  }
  // residual norms of the systems in `which` (r = b - A x, then |r|^2 into
  // sums(k)[132]); one synchronisation for all
  auto residuals = [&](const std::vector<int> &which, std::vector<double> &rn) {
    for (int k : which) {
      mfs_handle *h = hs[k];
      matvec(h, xx[k], h->rd);
      dev::axpy<double>(h->rd, b[k], -1.0, h->n, s);
      dev::scale(h->rd, -1.0, h->rd, h->n, s);
      dev::mdot(h->rd, 0, 1, h->rd, h->n, h->partial, h->nblk, s);
      dev::reduce_partials(h->partial, 1, h->nblk, B.sums(k) + 132, s);
    }
    MFS_CUDA(cudaMemcpyAsync(B.hbpin, B.hb, (size_t)136 * ns * sizeof(double), cudaMemcpyDeviceToHost, s));
    MFS_CUDA(cudaStreamSynchronize(s));
    for (int k : which) rn[k] = std::sqrt(B.hbpin[(int64_t)k * 136 + 132]);
  };
  std::vector<KrylovLS> ls;
  for (int k = 0; k < ns; ++k) ls.emplace_back(hs[k]->m);
  std::vector<int> j(ns, 0), restarts(ns, 0);
  std::vector<double> a(ns, 1.0), rn(ns, 0.0), relres(ns, 0.0);
  std::vector<char> active(ns, 0);
  std::vector<int> all(ns);
  for (int k = 0; k < ns; ++k) all[k] = k;
  residuals(all, rn);
  auto start_cycle = [&](int k, double beta) {
    mfs_handle *h = hs[k];
    dev::scale(h->rd, 1.0 / beta, h->V, h->n, s);
    ls[k].start_cycle(beta);
    j[k] = 0;
    a[k] = 1.0;
  };
  auto finish = [&](int k, int rc) {
    active[k] = 0;
    status[k] = rc;
    info[k].iters = ls[k].iters;
    info[k].restarts = restarts[k];
    info[k].true_relres = relres[k];
    info[k].est_relres = ls[k].est;
    info[k].converged = rc == MFS_OK ? 1 : 0;
  };
  for (int k = 0; k < ns; ++k) {
    ls[k].r0 = rn[k];
    if (rn[k] == 0.0) {
      info[k].converged = 1;
      status[k] = MFS_OK;
    } else if (!std::isfinite(rn[k])) {
      status[k] = MFS_ERR_BREAKDOWN;
    } else {
      active[k] = 1;
      start_cycle(k, rn[k]);
    }
  }
  dev::Recorder rec;
  // current plan and the global system at each of its positions
  FusedBatch *P = &B;
  std::vector<int> gidx(ns);
  for (int k = 0; k < ns; ++k) gidx[k] = k;
  int switches = 0;
  const bool verbose = hs[0]->prm.verbose != 0;
  cudaEvent_t ga = nullptr, gb = nullptr;
  if (verbose) {
    MFS_CUDA(cudaEventCreate(&ga));
    MFS_CUDA(cudaEventCreate(&gb));
  }
  double t_host = 0.0, t_graph = 0.0, t_cycle = 0.0, t_all = now_ms();
  int replays = 0;
  std::vector<int> live_per_replay;
  while (std::find(active.begin(), active.end(), 1) != active.end()) {
    const double th = now_ms();
    // once at most half of the current plan's systems run, move to the plan
    // over the running ones (fewer CTAs that would only check their flag)
    {
      std::vector<int> live;
      for (int p = 0; p < P->nsys; ++p)
        if (active[gidx[p]]) live.push_back(p);
      if (P->nsys >= 16 && 2 * (int)live.size() <= P->nsys) {
        std::vector<int> g2;
        for (int p : live) g2.push_back(gidx[p]);
        P = P->sub(live);
        gidx.swap(g2);
        ++switches;
      }
    }
    for (int p = 0; p < P->nsys; ++p) {
      const int k = gidx[p];
      P->hactive[p] = active[k];
      if (!active[k]) continue;
      rec.ops.clear();
      P->record_head(p, j[k], a[k], rec);
      P->patch(rec, P->head_at[p]);
      rec.ops.clear();
      P->record_tail(p, j[k], rec);
      P->patch(rec, P->tail_at[p]);
    }
    MFS_CUDA(cudaMemcpyAsync(P->dtab, P->htab, P->patch_bytes, cudaMemcpyHostToDevice, s));
    MFS_CUDA(cudaMemcpyAsync(P->dactive, P->hactive, P->nsys * sizeof(int), cudaMemcpyHostToDevice, s));
    t_host += now_ms() - th;
    if (verbose) MFS_CUDA(cudaEventRecord(ga, s));
    MFS_CUDA(cudaGraphLaunch(P->exec, s));
    if (verbose) MFS_CUDA(cudaEventRecord(gb, s));
    MFS_CUDA(cudaStreamSynchronize(s));
    ++replays;
    if (verbose) {
      float ms = 0.f;
      MFS_CUDA(cudaEventElapsedTime(&ms, ga, gb));
      t_graph += ms;
      live_per_replay.push_back((int)std::count(active.begin(), active.end(), 1));
    }
    const double tc = now_ms();
    std::vector<int> ending;
    for (int p = 0; p < P->nsys; ++p) {
      const int k = gidx[p];
      if (!active[k]) continue;
      if (!ls[k].column(P->hbpin + (int64_t)p * 136, j[k])) {
        finish(k, MFS_ERR_BREAKDOWN);
        continue;
      }
      if (ls[k].est <= tol || ls[k].happy || ls[k].iters >= hs[k]->prm.max_iters || j[k] + 1 == hs[k]->m) {
        ending.push_back(k);
      } else {
        a[k] = 1.0 / ls[k].hn;
        ++j[k];
      }
    }
    if (ending.empty()) {
      t_cycle += now_ms() - tc;
      continue;
    }
    // end of a cycle: x += Z y, true residual; stop or restart
    for (int k : ending) {
      mfs_handle *h = hs[k];
      ls[k].back_substitute();
      double *yp = B.ypin + (int64_t)k * 64;
      std::copy(ls[k].y.begin(), ls[k].y.begin() + ls[k].jend, yp);
      MFS_CUDA(cudaMemcpyAsync(h->ydev, yp, ls[k].jend * sizeof(double), cudaMemcpyHostToDevice, s));
      dev::gemv_add(h->Z, h->n, ls[k].jend, h->ydev, xx[k], h->n, s);
    }
    residuals(ending, rn);
    for (int k : ending) {
      relres[k] = rn[k] / ls[k].r0;
      if (!std::isfinite(relres[k])) {
        finish(k, MFS_ERR_BREAKDOWN);
      } else if (relres[k] <= tol || ls[k].iters >= hs[k]->prm.max_iters) {
        finish(k, relres[k] <= tol ? MFS_OK : MFS_ERR_NOT_CONVERGED);
      } else {
        ++restarts[k];
        start_cycle(k, rn[k]);
      }
    }
    t_cycle += now_ms() - tc;
  }
  if (verbose) {
    cudaEventDestroy(ga);
    cudaEventDestroy(gb);
    std::string live;
    for (size_t q = 0; q < live_per_replay.size(); q += 5) live += " " + std::to_string(live_per_replay[q]);
    fprintf(stderr,
            "mfs fused solve: %d replays (%d plan switches), %.2f ms total: graphs %.2f ms (GPU), host "
            "recording/patching %.2f ms, Givens + cycle ends %.2f ms; live systems every 5th replay:%s\n",
            replays, switches, now_ms() - t_all, t_graph, t_host, t_cycle, live.c_str());
  }
  for (int k = 0; k < ns; ++k)
    if (hostx[k]) MFS_CUDA(cudaMemcpyAsync(x[k], xx[k], hs[k]->n * sizeof(double), cudaMemcpyDeviceToHost, s));
  MFS_CUDA(cudaStreamSynchronize(s));
  MFS_CUDA(cudaGetLastError());
}

HBsr to_hbsr(const mfs_block &b) {
  HBsr A;
  A.br = b.br;
  A.bc = b.bc;
  A.nbr = b.nbrows;
  A.nbc = b.nbcols;
  A.rp.assign(b.rowptr, b.rowptr + b.nbrows + 1);
  A.ci.assign(b.colind, b.colind + b.nnzb);
  A.v.assign(b.vals, b.vals + b.nnzb * b.br * b.bc);
  if (A.rp[0] != 0 || A.rp[A.nbr] != b.nnzb) throw SetupError(MFS_ERR_INVALID, "block rowptr inconsistent with nnzb");
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int64_t I = 0; I < A.nbr; ++I) {
    if (A.rp[I + 1] < A.rp[I]) {
      bad |= 1;
      continue;
    }
    for (int64_t a = A.rp[I]; a < A.rp[I + 1]; ++a) {
      if (A.ci[a] < 0 || A.ci[a] >= A.nbc) bad |= 2;
      else if (a > A.rp[I] && A.ci[a] <= A.ci[a - 1]) bad |= 4;
    }
  }
  if (bad & 1) throw SetupError(MFS_ERR_INVALID, "block rowptr not monotone");
  if (bad & 2) throw SetupError(MFS_ERR_INVALID, "block column index out of range");
  if (bad & 4) throw SetupError(MFS_ERR_INVALID, "block columns not sorted/unique");
  return A;
}

// Threads per block row of the merged float64 matvec (1, 2 or 4): timed
// once per (row block shape, rows, blocks) and process, like the layouts.
static std::map<std::tuple<int, int, int, int, int64_t, int64_t>, int> g_tune_rows;

static int tune_rows(const dev::RowMerged &R, int64_t n, cudaStream_t st) {
  const dev::Sell &A = R.M;
  const auto key = std::make_tuple(A.br, R.b[0], R.b[1], R.nb > 2 ? R.b[2] : 0, (int64_t)A.nbr, (int64_t)A.nnzb);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_rows.find(key);
    if (it != g_tune_rows.end()) return it->second;
  }
  double *x = nullptr, *y = nullptr;
  MFS_CUDA(cudaMallocAsync((void **)&x, (size_t)std::max<int64_t>(1, n) * sizeof(double), st));
  MFS_CUDA(cudaMallocAsync((void **)&y, (size_t)std::max<int64_t>(1, A.nrows()) * sizeof(double), st));
  MFS_CUDA(cudaMemsetAsync(x, 0, (size_t)n * sizeof(double), st));
  cudaEvent_t e0, e1;
  MFS_CUDA(cudaEventCreate(&e0));
  MFS_CUDA(cudaEventCreate(&e1));
  int best = 1;
  float tbest = 1e30f;
  for (int split : {1, 2, 4}) {
    dev::RowMerged T = R;
    T.split = split;
    for (int rep = 0; rep < 4; ++rep) {
      MFS_CUDA(cudaEventRecord(e0, st));
      dev::spmv_rows(T, x, y, st);
      MFS_CUDA(cudaEventRecord(e1, st));
      MFS_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      MFS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (rep > 0 && ms < tbest) {
        tbest = ms;
        best = split;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(x, st);
  cudaFreeAsync(y, st);
  MFS_CUDA(cudaStreamSynchronize(st));
  std::lock_guard<std::mutex> lock(g_tune_mu);
  return g_tune_rows.emplace(key, best).first->second;
}

// Fine operator rows: when every block A_ij of a block row i exists and all
// share one sparsity pattern (fields on the same nodes), store the row's
// blocks side by side so one kernel reads each column index once and writes
// y_i once; built on the device from the row field's uploaded input blocks.
// Empty result = per-block SpMVs.
std::vector<dev::RowMerged> merge_rows_dev(Arena &ar, const std::map<std::pair<int, int>, HBsr> &hb,
                                           const std::map<std::pair<int, int>, RawDev> &raw, int nf,
                                           const std::vector<int64_t> &foff, int split, cudaStream_t st) {
  std::vector<dev::RowMerged> out;
  if (nf < 2 || nf > 3) return out;
  for (int i = 0; i < nf; ++i) {
    int b[3] = {0, 0, 0};
    const RawDev *src[3] = {nullptr, nullptr, nullptr};
    const HBsr *h0 = nullptr;
    for (int j = 0; j < nf; ++j) {
      auto it = hb.find({i, j});
      if (it == hb.end()) return {};
      if (!h0) h0 = &it->second;
      if (it->second.rp != h0->rp || it->second.ci != h0->ci) return {};
      b[j] = it->second.bc;
      src[j] = &raw.at({i, j});
    }
    if (!dev::rows_supported(h0->br, b, nf)) return {};
    dev::RowMerged R;
    R.M = upload_layout_dev(ar, src, nf, true, false, 0, st);
    R.nb = nf;
    int64_t n = 0;
    for (int j = 0; j < nf; ++j) {
      R.b[j] = b[j];
      R.off[j] = foff[j];
      n = std::max(n, foff[j] + src[j]->nbc * src[j]->bc);
    }
    R.split = split > 0 ? split : tune_rows(R, n, st);
    out.push_back(R);
  }
  return out;
}

// Multicolour Gauss-Seidel colours of every smoothed level field (levels
// below the coarsest; every level of the single-level BGS(GS) and of
// AMG(SIMPLE)'s level Schur complements).
void color_levels(mfs_handle *h) {
  const mfs_params &p = h->prm;
  if (p.smoother != MFS_GS) return;
  auto run = [](HGroup &g, bool all) {
    for (int l = 0; l < g.nlevels(); ++l)
      if (all || l + 1 < g.nlevels())
        for (auto &f : g.lv[l]) f.color = node_colors(f.A);
  };
  run(h->host->hg0, p.precond == MFS_BGS_GS);
  run(h->host->hg1, p.precond == MFS_AMG_SIMPLE);
}

// Host half of the setup: hierarchies, SIMPLE diagonal and explicit S~.
void build_host(mfs_handle *h, const std::map<std::pair<int, int>, HBsr> &blocks,
                const std::vector<FieldInfo> &info) {
  const mfs_params &p = h->prm;
  const bool gpu = p.setup_device == 1 && !p.setup_only;
  // gf: the input fields of the group's members (empty: blocks not among the inputs)
  // steal: d itself, when the caller no longer needs it (moved into level 0)
  auto group = [&](HGroup &g, const std::vector<HBsr> &d, const std::vector<FieldInfo> &fi, bool off,
                   const BlockMap *fo, const std::vector<int> &gf, std::vector<HBsr> *steal = nullptr) {
    if (!gpu) {
      build_group(g, d, fi, p.max_levels, p.coarse_max, p.seed, off, fo, p.verbose);
      return;
    }
    std::vector<DevBlock> dd;
    std::map<std::pair<int, int>, DevBlock> dof;
    const bool have = h->raw && !gf.empty();
    if (have) {
      auto view = [&](int i, int j) {
        const RawDev &r = h->raw->at({gf[i], gf[j]});
        return DevBlock{r.rp, r.ci, r.v};
      };
      for (int k = 0; k < (int)gf.size(); ++k) dd.push_back(view(k, k));
      if (fo)
        for (auto &kv : *fo) dof[kv.first] = view(kv.first.first, kv.first.second);
    }
    build_group_gpu(g, d, fi, p.max_levels, p.coarse_max, p.seed, off, fo, p.verbose, have ? &dd : nullptr,
                    have && fo ? &dof : nullptr, steal);
  };
  auto split_groups = [&]() {
    h->host->G1.clear();
    h->host->G2.clear();
    bool any = false;
    for (int i = 0; i < h->nf; ++i) any |= p.simple_group[i] != 0;
    for (int i = 0; i < h->nf; ++i) {
      const bool schur = any ? p.simple_group[i] != 0 : i == h->nf - 1;
      (schur ? h->host->G2 : h->host->G1).push_back(i);
    }
    if (h->host->G1.empty() || h->host->G2.empty())
      throw SetupError(MFS_ERR_INVALID, "SIMPLE needs a non-empty predictor and Schur group");
  };
  if (p.precond == MFS_BGS_GS) {
    // single level: the fine diagonal blocks and their smoother data only
    HGroup &g = h->host->hg0;
    g.nf = h->nf;
    g.info = info;
    g.lv.assign(1, std::vector<HLevelField>(h->nf));
    g.off.assign(1, BlockMap());
    for (int i = 0; i < h->nf; ++i) {
      g.lv[0][i].A = blocks.at({i, i});
      g.lv[0][i].dinv = amg_dinv(g.lv[0][i].A);
    }
    return;
  }
  if (p.precond == MFS_BGS_AMG || p.precond == MFS_AMG_BGS || p.precond == MFS_AMG_SIMPLE) {
    std::vector<HBsr> diag;
    BlockMap off;
    for (auto &kv : blocks)
      if (kv.first.first == kv.first.second) diag.push_back(kv.second);
      else off[kv.first] = kv.second;
    std::vector<int> all(h->nf);
    for (int i = 0; i < h->nf; ++i) all[i] = i;
    group(h->host->hg0, diag, info, p.precond != MFS_BGS_AMG, &off, all, &diag);
    if (p.precond != MFS_AMG_SIMPLE) return;
    // AMG(SIMPLE): per smoothed level, A~_11 of the merged predictor rows and
    // the explicit level Schur complement S~^l with its smoother data
    split_groups();
    if (h->host->G2.size() != 1) throw SetupError(MFS_ERR_INVALID, "AMG(SIMPLE) takes one Schur field");
    const int k = h->host->G2[0];
    const HGroup &g = h->host->hg0;
    HGroup &hs = h->host->hg1;
    hs.nf = 1;
    hs.lv.assign(std::max(0, g.nlevels() - 1), std::vector<HLevelField>(1));
    h->host->mono_dtilde.assign(hs.lv.size(), {});
    for (int l = 0; l + 1 < g.nlevels(); ++l) {
      auto blk = [&](int i, int j) -> const HBsr * {
        if (i == j) return &g.lv[l][i].A;
        auto it = g.off[l].find({i, j});
        return it == g.off[l].end() ? nullptr : &it->second;
      };
      std::vector<std::vector<double>> dts;
      for (int j : h->host->G1) {
        std::vector<double> d(g.lv[l][j].A.nrows(), 0.0);
        if (p.simple_approx == MFS_DIAG) {
          d = bsr_point_diagonal(g.lv[l][j].A);
        } else {
          for (int q : h->host->G1) {
            const HBsr *M = blk(j, q);
            if (!M) continue;
            std::vector<double> sr = bsr_abs_row_sums(*M);
            for (size_t r = 0; r < d.size(); ++r) d[r] += sr[r];
          }
        }
        for (double v : d)
          if (v == 0.0) throw SetupError(MFS_ERR_SINGULAR, "zero entry in a level's SIMPLE diagonal approximation");
        dts.push_back(d);
      }
      HBsr S = g.lv[l][k].A;
      for (size_t jj = 0; jj < h->host->G1.size(); ++jj) {
        const int j = h->host->G1[jj];
        const HBsr *a = blk(k, j), *c = blk(j, k);
        if (!a || !c) continue;
        HBsr Cs = *c;
        std::vector<double> inv(dts[jj].size());
        for (size_t r = 0; r < inv.size(); ++r) inv[r] = 1.0 / dts[jj][r];
        bsr_scale_rows(Cs, inv);
        HBsr Tm = gpu ? gpu_spgemm(*a, Cs) : bsr_spgemm(*a, Cs);
        S = bsr_axpby(1.0, S, -1.0, Tm);
      }
      HLevelField &f = hs.lv[l][0];
      f.A = std::move(S);
      f.dinv = amg_dinv(f.A);
      f.lam = amg_power_lambda(f.A, f.dinv, p.seed);
      h->host->mono_dtilde[l] = std::move(dts);
    }
    return;
  }
  split_groups();
  std::map<int, int> l2;
  for (size_t a = 0; a < h->host->G2.size(); ++a) l2[h->host->G2[a]] = (int)a;
  std::vector<HBsr> diag1;
  std::vector<FieldInfo> info1;
  std::map<int, int> l1;
  for (int j : h->host->G1) {
    l1[j] = (int)diag1.size();
    diag1.push_back(blocks.at({j, j}));
    info1.push_back(info[j]);
  }
  // SIMPLE(AMG(BGS)): the predictor group gets a monolithic hierarchy with
  // blockwise Galerkin coupling blocks
  const bool mono_pred = p.simple_pred == MFS_PRED_AMG_BGS;
  BlockMap off1;
  if (mono_pred)
    for (auto &kv : blocks) {
      const int i = kv.first.first, j = kv.first.second;
      if (i != j && l1.count(i) && l1.count(j)) off1[{l1[i], l1[j]}] = kv.second;
    }
  group(h->host->hg0, diag1, info1, mono_pred, mono_pred ? &off1 : nullptr, h->host->G1, &diag1);
  // A~_11: SIMPLEC sums of absolute entries over the merged predictor rows, or the diagonal
  h->host->dtilde.clear();
  for (int j : h->host->G1) {
    std::vector<double> d(h->fsize[j], 0.0);
    if (p.simple_approx == MFS_DIAG) {
      d = bsr_point_diagonal(blocks.at({j, j}));
    } else {
      for (int l : h->host->G1) {
        auto it = blocks.find({j, l});
        if (it == blocks.end()) continue;
        std::vector<double> sr = bsr_abs_row_sums(it->second);
        for (int64_t r = 0; r < (int64_t)d.size(); ++r) d[r] += sr[r];
      }
    }
    for (double v : d)
      if (v == 0.0) throw SetupError(MFS_ERR_SINGULAR, "zero entry in the SIMPLE diagonal approximation");
    h->host->dtilde.push_back(d);
  }
  // S~_kl = A_kl - sum_j A_kj diag(1/d~_j) A_jl
  std::vector<FieldInfo> sinfo;
  h->host->schur_off.clear();
  h->host->schur_diag.clear();
  for (int k : h->host->G2)
    for (int l : h->host->G2) {
      HBsr M;
      bool have = false;
      auto it = blocks.find({k, l});
      if (it != blocks.end()) {
        M = it->second;
        have = true;
      }
      for (size_t jj = 0; jj < h->host->G1.size(); ++jj) {
        const int j = h->host->G1[jj];
        auto a = blocks.find({k, j});
        auto c = blocks.find({j, l});
        if (a == blocks.end() || c == blocks.end()) continue;
        HBsr Cs = c->second;
        std::vector<double> inv(h->host->dtilde[jj].size());
        for (size_t r = 0; r < inv.size(); ++r) inv[r] = 1.0 / h->host->dtilde[jj][r];
        bsr_scale_rows(Cs, inv);
        HBsr Tm = gpu ? gpu_spgemm(a->second, Cs) : bsr_spgemm(a->second, Cs);
        if (have) {
          M = bsr_axpby(1.0, M, -1.0, Tm);
        } else {
          M = bsr_axpby(0.0, Tm, -1.0, Tm);
          have = true;
        }
      }
      if (!have) continue;
      if (k == l) {
        h->host->schur_diag.push_back(M);
        FieldInfo fi = info[k];
        fi.ns = 0;
        fi.user_B.clear();
        fi.dirichlet.clear();
        sinfo.push_back(fi);
      } else {
        h->host->schur_off[{l2[k], l2[l]}] = M;
      }
    }
  if (h->host->schur_diag.size() != h->host->G2.size()) throw SetupError(MFS_ERR_INVALID, "missing Schur diagonal block");
  group(h->host->hg1, h->host->schur_diag, sinfo, false, nullptr, {});
}

// Device half of the setup: upload the host hierarchy in precision T
// (matrices into the shared arena `mat`), then the work vectors into h->ar.
template <typename T>
void upload_precond(mfs_handle *h, Arena &mat, Precond<T> &P, const std::map<std::pair<int, int>, HBsr> &blocks,
                    bool f32) {
  const mfs_params &p = h->prm;
  const HostSide &hs = *h->host;
  P.kind = p.precond;
  P.nf = h->nf;
  P.order = p.bgs_order;
  P.sweeps = p.bgs_sweeps;
  P.fsize = h->fsize;
  P.foff = h->foff;
  P.s = h->s;
  auto fine_sell = [&](int i, int j) { return h->A64.at({i, j}); };
  P.smoother = p.smoother;
  P.use_tail = p.vcycle_tail != 0;
  P.gs_sweeps = p.gs_sweeps;
  P.gs_omega = (T)p.gs_omega;
  if (p.precond == MFS_BGS_AMG || p.precond == MFS_AMG_BGS || p.precond == MFS_AMG_SIMPLE ||
      p.precond == MFS_BGS_GS) {
    std::vector<dev::Sell> d0;
    std::map<std::pair<int, int>, dev::Sell> o0;
    for (int i = 0; i < h->nf; ++i) d0.push_back(fine_sell(i, i));
    for (auto &kv : blocks)
      if (kv.first.first != kv.first.second) o0[kv.first] = fine_sell(kv.first.first, kv.first.second);
    upload_group(mat, P.g0, hs.hg0, p, d0, o0, p.precond == MFS_AMG_BGS || p.precond == MFS_AMG_SIMPLE);
    if (p.precond == MFS_AMG_SIMPLE) {
      P.G1 = hs.G1;
      P.G2 = hs.G2;
      P.ms.assign(hs.hg1.lv.size(), FL<T>());
      P.ms_dtinv.assign(hs.hg1.lv.size(), {});
      for (size_t l = 0; l < hs.hg1.lv.size(); ++l) {
        const HLevelField &hf = hs.hg1.lv[l][0];
        FL<T> &f = P.ms[l];
        f.n = hf.A.nrows();
        f.A = upload_sell(mat, hf.A, !f32, f32);
        std::vector<double> c1, c2;
        smoother_coeffs(p, hf.lam, c1, c2);
        f.c1.assign(c1.begin(), c1.end());
        f.c2.assign(c2.begin(), c2.end());
        f.dinv = upload_as<T>(mat, hf.dinv);
        if (!hf.color.empty()) upload_gs(mat, f, hf.A, hf.color);
        for (auto &d : hs.mono_dtilde[l]) {
          std::vector<double> inv(d.size());
          for (size_t r = 0; r < inv.size(); ++r) inv[r] = 1.0 / d[r];
          P.ms_dtinv[l].push_back(upload_as<T>(mat, inv));
        }
      }
    }
  } else {
    P.G1 = hs.G1;
    P.G2 = hs.G2;
    std::map<int, int> l1, l2;
    for (size_t a = 0; a < hs.G1.size(); ++a) l1[hs.G1[a]] = (int)a;
    for (size_t a = 0; a < hs.G2.size(); ++a) l2[hs.G2[a]] = (int)a;
    std::vector<dev::Sell> d0;
    std::map<std::pair<int, int>, dev::Sell> o0;
    for (int j : hs.G1) d0.push_back(fine_sell(j, j));
    for (auto &kv : blocks) {
      const int i = kv.first.first, j = kv.first.second;
      if (i != j && l1.count(i) && l1.count(j)) o0[{l1[i], l1[j]}] = fine_sell(i, j);
      if ((l1.count(i) && l2.count(j)) || (l2.count(i) && l1.count(j))) P.cross[kv.first] = fine_sell(i, j);
    }
    upload_group(mat, P.g0, hs.hg0, p, d0, o0, p.simple_pred == MFS_PRED_AMG_BGS);
    std::vector<dev::Sell> sd0;
    std::map<std::pair<int, int>, dev::Sell> so0;
    for (auto &M : hs.schur_diag) sd0.push_back(upload_sell(mat, M, !f32, f32));
    for (auto &kv : hs.schur_off) so0[kv.first] = upload_sell(mat, kv.second, !f32, f32);
    upload_group(mat, P.g1, hs.hg1, p, sd0, so0, false);
    for (size_t jj = 0; jj < hs.G1.size(); ++jj) {
      std::vector<double> inv(hs.dtilde[jj].size());
      for (size_t r = 0; r < inv.size(); ++r) inv[r] = 1.0 / hs.dtilde[jj][r];
      P.dtinv.push_back(upload_as<T>(mat, inv));
    }
  }
  P.alloc_work(h->ar);
}

// GMRES workspace of a handle.
void alloc_solver_work(mfs_handle *h) {
  h->m = h->prm.restart;
  h->graphs.assign(h->m, IterGraph());
  h->nblk = dev::mdot_blocks(h->n);
  h->V = h->ar.zeros<double>((int64_t)(h->m + 1) * h->n);
  h->Z = h->ar.zeros<double>((int64_t)h->m * h->n);
  h->rd = h->ar.zeros<double>(h->n);
  h->xd = h->ar.zeros<double>(h->n);
  h->bd = h->ar.zeros<double>(h->n);
  h->partial = h->ar.zeros<double>((int64_t)64 * h->nblk);
  h->hdev = h->ar.zeros<double>(kHostSlots);
  h->ydev = h->ar.zeros<double>(64);
  if (h->prm.precision == MFS_FP32P) {
    h->in32 = h->ar.zeros<float>(h->n);
    h->out32 = h->ar.zeros<float>(h->n);
  }
  h->hpin = (double *)g_pinned.get(kHostSlots * sizeof(double));
  for (auto &e : h->iter_ev)
    if (!e) MFS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
}

int fail(int code, const std::string &msg) {
  g_last_error = msg;
  return code;
}

}  // namespace

extern "C" {

void mfs_default_params(mfs_params *p) {
  std::memset(p, 0, sizeof(*p));
  p->precond = MFS_BGS_AMG;
  p->bgs_order = MFS_BWD;
  p->bgs_sweeps = 1;
  for (int i = 0; i < MFS_MAX_FIELDS; ++i) p->simple_group[i] = 0;
  p->simple_approx = MFS_ABSROWSUM;
  p->max_levels = 4;
  p->coarse_max = 1000;
  p->smoother = MFS_CHEBYSHEV;
  p->cheb_degree = 2;
  p->cheb_ratio = 30.0;
  p->cheb_boost = 1.1;
  p->jacobi_omega = 2.0 / 3.0;
  p->jacobi_sweeps = 1;
  p->gs_sweeps = 1;
  p->gs_omega = 0.79;
  p->restart = 50;
  p->max_iters = 1000;
  p->precision = MFS_FP64;
  p->seed = 7;
  p->cuda_stream = nullptr;
  p->verbose = 0;
  p->setup_device = 1;
  p->vcycle_tail = 0;
  p->pdl = -1;
}

int mfs_setup(const mfs_block *blocks, int nblocks, const mfs_field *fields, int nfields,
              const mfs_params *params, mfs_handle **out) {
  if (!out) return fail(MFS_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!blocks || !fields || !params || nfields < 1 || nfields > MFS_MAX_FIELDS || nblocks < nfields)
    return fail(MFS_ERR_INVALID, "bad block/field arguments");
  const mfs_params &p = *params;
  if (p.precond < 0 || p.precond > 4 || p.bgs_order < 0 || p.bgs_order > 2 || p.bgs_sweeps < 1 ||
      p.max_levels < 1 || p.coarse_max < 0 || p.restart < 1 || p.restart > 60 || p.max_iters < 1 ||
      (p.smoother == MFS_CHEBYSHEV && (p.cheb_degree < 1 || !(p.cheb_ratio > 1.0) || !(p.cheb_boost > 0.0))) ||
      (p.smoother == MFS_JACOBI && p.jacobi_sweeps < 1) ||
      (p.smoother != MFS_CHEBYSHEV && p.smoother != MFS_JACOBI && p.smoother != MFS_GS) ||
      (p.smoother == MFS_GS && (p.gs_sweeps < 1 || !(p.gs_omega > 0.0) || !(p.gs_omega < 2.0))) ||
      (p.precond == MFS_BGS_GS && p.smoother != MFS_GS) ||
      (p.precision != MFS_FP64 && p.precision != MFS_FP32P) || p.setup_device < 0 || p.setup_device > 1 ||
      (p.simple_pred != MFS_PRED_BGS_AMG && p.simple_pred != MFS_PRED_AMG_BGS) ||
      (p.rows_split != 0 && p.rows_split != 1 && p.rows_split != 2 && p.rows_split != 4) ||
      (p.layout_tune != 0 && p.layout_tune != 1) || (p.vcycle_tail != 0 && p.vcycle_tail != 1) || p.pdl < -1)
    return fail(MFS_ERR_INVALID, "bad parameters");
  const bool host_only = p.setup_only != 0;
  int ndev = 0;
  if (!host_only && (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)) {
    cudaGetLastError();
    return fail(MFS_ERR_CUDA, "no CUDA device");
  }
  const double t0 = now_ms();
  std::unique_ptr<mfs_handle> h(new mfs_handle());
  struct TuneMode {  // the layout tuning mode of this setup, for this thread
    explicit TuneMode(int m) { g_layout_tune = m; }
    ~TuneMode() { g_layout_tune = 0; }
  } tune_mode(p.layout_tune);
  try {
    h->prm = p;
    h->nf = nfields;
    h->s = (cudaStream_t)p.cuda_stream;
    h->use_graphs = p.no_graphs == 0;
    std::vector<FieldInfo> info(nfields);
    h->foff.assign(nfields + 1, 0);
    for (int i = 0; i < nfields; ++i) {
      const mfs_field &f = fields[i];
      if (f.nnodes < 1 || f.dofs_per_node < 1 || f.dofs_per_node > 6 || f.strength_theta < 0)
        throw SetupError(MFS_ERR_INVALID, "bad field");
      info[i].nnodes = f.nnodes;
      info[i].b = f.dofs_per_node;
      info[i].dim = f.dim;
      info[i].ns = f.nullspace;
      info[i].theta = f.strength_theta;
      if (f.petrov_galerkin != 0 && f.petrov_galerkin != 1) throw SetupError(MFS_ERR_INVALID, "bad field");
      info[i].pg = f.petrov_galerkin == 1;
      if (f.nullspace == MFS_NS_RBM) {
        if (!f.coords || f.dim != f.dofs_per_node || (f.dim != 2 && f.dim != 3))
          throw SetupError(MFS_ERR_INVALID, "rigid-body modes need coords and dofs_per_node == dim in {2,3}");
        info[i].coords.assign(f.coords, f.coords + f.nnodes * f.dim);
      } else if (f.nullspace == MFS_NS_USER) {
        auto shape_ok = [](int v) { return v == 1 || v == 2 || v == 3 || v == 6; };
        if (!f.ns_user || !shape_ok(f.ns_dim) || !shape_ok(f.dofs_per_node))
          throw SetupError(MFS_ERR_INVALID, "MFS_NS_USER needs ns_user and ns_dim, dofs_per_node in {1, 2, 3, 6}");
        info[i].ns_dim = f.ns_dim;
        info[i].user_B.assign(f.ns_user, f.ns_user + f.nnodes * f.dofs_per_node * f.ns_dim);
        for (double v : info[i].user_B)
          if (!std::isfinite(v)) throw SetupError(MFS_ERR_INVALID, "non-finite value in ns_user");
      } else if (f.nullspace != MFS_NS_CONST) {
        throw SetupError(MFS_ERR_INVALID, "bad nullspace kind");
      }
      if (f.dirichlet) {
        info[i].dirichlet.resize(f.nnodes * f.dofs_per_node);
        for (size_t d = 0; d < info[i].dirichlet.size(); ++d) info[i].dirichlet[d] = f.dirichlet[d] ? 1 : 0;
      }
      h->fsize.push_back(f.nnodes * f.dofs_per_node);
      h->foff[i + 1] = h->foff[i] + h->fsize[i];
    }
    h->n = h->foff[nfields];
    std::map<std::pair<int, int>, HBsr> hb;
    for (int k = 0; k < nblocks; ++k) {
      const mfs_block &b = blocks[k];
      if (b.i < 0 || b.j < 0 || b.i >= nfields || b.j >= nfields || hb.count({b.i, b.j}))
        throw SetupError(MFS_ERR_INVALID, "bad or repeated block index");
      if (b.br != fields[b.i].dofs_per_node || b.bc != fields[b.j].dofs_per_node ||
          b.nbrows != fields[b.i].nnodes || b.nbcols != fields[b.j].nnodes || !b.rowptr || (b.nnzb && (!b.colind || !b.vals)))
        throw SetupError(MFS_ERR_INVALID, "block shape does not match the field map");
      hb[{b.i, b.j}] = to_hbsr(b);
    }
    for (int i = 0; i < nfields; ++i)
      if (!hb.count({i, i})) throw SetupError(MFS_ERR_INVALID, "missing diagonal block");
    // a flagged Dirichlet dof's row is the identity across its block row
    for (int i = 0; i < nfields; ++i) {
      const std::vector<uint8_t> &dm = info[i].dirichlet;
      if (dm.empty()) continue;
      for (auto &kv : hb) {
        if (kv.first.first != i) continue;
        const HBsr &B = kv.second;
        const bool diag = kv.first.second == i;
        for (int64_t I = 0; I < B.nbr; ++I)
          for (int64_t a = B.rp[I]; a < B.rp[I + 1]; ++a)
            for (int c = 0; c < B.br; ++c) {
              if (!dm[I * B.br + c]) continue;
              for (int q = 0; q < B.bc; ++q) {
                const double want = diag && B.ci[a] == I && q == c ? 1.0 : 0.0;
                if (B.v[(a * B.br + c) * B.bc + q] != want)
                  throw SetupError(MFS_ERR_INVALID, "a flagged Dirichlet dof's row is not an identity row");
              }
            }
      }
    }
    // one upload of the input blocks, shared by the GPU setup and the fine layouts
    std::unique_ptr<Arena> raw_arena;
    std::map<std::pair<int, int>, RawDev> rd;
    struct StreamGuard {
      cudaStream_t s = nullptr;
      ~StreamGuard() {
        if (s) {
          cudaStreamSynchronize(s);
          cudaStreamDestroy(s);
        }
      }
    } rst;
    struct RawReset {
      mfs_handle *h;
      ~RawReset() { h->raw = nullptr; }
    } raw_reset{h.get()};
    if (!host_only) {
      dev::init();
      raw_arena.reset(new Arena());
      MFS_CUDA(cudaStreamCreateWithFlags(&rst.s, cudaStreamNonBlocking));
      for (auto &kv : hb) rd[kv.first] = upload_raw(*raw_arena, kv.second, rst.s);
      h->raw = &rd;
    }
    const double t_in = now_ms();
    build_host(h.get(), hb, info);
    color_levels(h.get());
    const double t_host = now_ms();
    h->host_only = host_only;
    if (host_only) {
      h->setup_ms = now_ms() - t0;
      *out = h.release();
      return MFS_OK;
    }
    if (!h->s) {
      // the legacy default stream cannot be captured: use a stream of our own,
      // non-blocking so that legacy-stream work of other threads (another
      // handle's setup) never joins a graph capture running on it
      MFS_CUDA(cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking));
      h->own_stream = true;
    }
    const bool f32 = p.precision == MFS_FP32P;
    MFS_CUDA(cudaGetDevice(&h->device));
    Arena &mat = *h->mat;
    const double t_dev = now_ms();
    // fine layouts built on the device from the uploaded input blocks
    for (auto &kv : hb) h->A64[kv.first] = upload_sell_dev(mat, rd.at(kv.first), true, f32, rst.s);
    h->rows64 = merge_rows_dev(mat, hb, rd, h->nf, h->foff, p.rows_split, rst.s);
    MFS_CUDA(cudaStreamSynchronize(rst.s));
    h->raw = nullptr;
    raw_arena.reset();
    const double t_fine = now_ms();
    if (f32) {
      h->p32.reset(new Precond<float>());
      upload_precond<float>(h.get(), mat, *h->p32, hb, true);
    } else {
      h->p64.reset(new Precond<double>());
      upload_precond<double>(h.get(), mat, *h->p64, hb, false);
    }
    const double t_pre = now_ms();
    alloc_solver_work(h.get());
    if (p.profile) h->prof.reset(new EventProf());
    MFS_CUDA(cudaStreamSynchronize(0));  // uploads and memsets ran on the legacy stream
    if (p.verbose)
      fprintf(stderr,
              "mfs_setup: input %.1f ms, hierarchy %.1f ms, init %.1f ms, fine layouts %.1f ms, "
              "preconditioner upload %.1f ms, workspace %.1f ms (%lld arrays)\n",
              t_in - t0, t_host - t_in, t_dev - t_host, t_fine - t_dev, t_pre - t_fine, now_ms() - t_pre,
              (long long)(h->mat->ptrs.size() + h->ar.ptrs.size()));
  } catch (const SetupError &e) {
    return fail(e.code, e.what());
  } catch (const CudaError &e) {
    return fail(e.code, e.what());
  } catch (const std::bad_alloc &) {
    return fail(MFS_ERR_OOM, "host allocation failed");
  } catch (const std::exception &e) {
    return fail(MFS_ERR_INVALID, e.what());
  }
  h->setup_ms = now_ms() - t0;
  *out = h.release();
  return MFS_OK;
}

int64_t mfs_ndofs(const mfs_handle *h) { return h ? h->n : 0; }

int64_t mfs_device_bytes(const mfs_handle *h, int shared) {
  if (!h) return 0;
  return shared ? h->mat->bytes : h->ar.bytes;
}

int mfs_num_levels(const mfs_handle *h, int group) {
  if (!h) return 0;
  if (group == 0) return h->host->hg0.nlevels();
  if (group == 1) return h->host->hg1.nlevels();
  return 0;
}

static int solve_impl(mfs_handle *h, const double *rhs, double *x, double tol, mfs_info *info, bool hook) {
  if (!h || !rhs || !x || !(tol > 0.0)) return fail(MFS_ERR_INVALID, "bad solve arguments");
  if (h->host_only) return fail(MFS_ERR_INVALID, "handle was built with setup_only");
  mfs_info local{};
  if (!info) info = &local;
  std::memset(info, 0, sizeof(*info));
  const double t0 = now_ms();
  int rc = MFS_OK;
  try {
    if (h->own_stream) {
      // the caller's vectors come from the legacy default stream: start after it
      if (!h->entry) MFS_CUDA(cudaEventCreateWithFlags(&h->entry, cudaEventDisableTiming));
      MFS_CUDA(cudaEventRecord(h->entry, 0));
      MFS_CUDA(cudaStreamWaitEvent(h->s, h->entry, 0));
    }
    const bool drhs = is_device_ptr(rhs), dx = is_device_ptr(x);
    const double *b = rhs;
    double *xx = x;
    if (!drhs) {
      MFS_CUDA(cudaMemcpyAsync(h->bd, rhs, h->n * sizeof(double), cudaMemcpyHostToDevice, h->s));
      b = h->bd;
    }
    if (!dx) {
      MFS_CUDA(cudaMemcpyAsync(h->xd, x, h->n * sizeof(double), cudaMemcpyHostToDevice, h->s));
      xx = h->xd;
    }
    const bool prof = hook && h->prof;
    if (prof) dev::set_launch_hook(h->prof.get());
    try {
      rc = fgmres(h, b, xx, tol, info, prof);
    } catch (...) {
      if (prof) dev::set_launch_hook(nullptr);
      throw;
    }
    if (prof) {
      dev::set_launch_hook(nullptr);
      h->prof->collect();
    }
    if (!dx) MFS_CUDA(cudaMemcpyAsync(x, h->xd, h->n * sizeof(double), cudaMemcpyDeviceToHost, h->s));
    MFS_CUDA(cudaStreamSynchronize(h->s));
    MFS_CUDA(cudaGetLastError());
  } catch (const CudaError &e) {
    return fail(e.code, e.what());
  }
  info->solve_ms = now_ms() - t0;
  info->setup_ms = h->setup_ms;
  info->levels[0] = h->host->hg0.nlevels();
  info->levels[1] = h->host->hg1.nlevels();
  if (rc == MFS_ERR_NOT_CONVERGED) g_last_error = "GMRES reached max_iters";
  return rc;
}

int mfs_solve(mfs_handle *h, const double *rhs, double *x, double tol, mfs_info *info) {
  return solve_impl(h, rhs, x, tol, info, true);
}

int mfs_clone(const mfs_handle *src, void *stream, mfs_handle **out) {
  if (!src || !out) return fail(MFS_ERR_INVALID, "bad clone arguments");
  *out = nullptr;
  if (src->host_only) return fail(MFS_ERR_INVALID, "handle was built with setup_only");
  std::unique_ptr<mfs_handle> h(new mfs_handle());
  try {
    MFS_CUDA(cudaSetDevice(src->device));
    h->prm = src->prm;
    h->prm.profile = 0;
    h->prm.cuda_stream = stream;
    h->nf = src->nf;
    h->fsize = src->fsize;
    h->foff = src->foff;
    h->n = src->n;
    h->device = src->device;
    h->host = src->host;
    h->mat = src->mat;
    h->A64 = src->A64;
    h->rows64 = src->rows64;
    h->setup_ms = src->setup_ms;
    h->use_graphs = src->use_graphs;
    h->s = (cudaStream_t)stream;
    if (!h->s) {
      MFS_CUDA(cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking));
      h->own_stream = true;
    }
    if (src->p32) {
      h->p32.reset(new Precond<float>(*src->p32));
      h->p32->s = h->s;
      h->p32->alloc_work(h->ar);
    } else {
      h->p64.reset(new Precond<double>(*src->p64));
      h->p64->s = h->s;
      h->p64->alloc_work(h->ar);
    }
    alloc_solver_work(h.get());
    MFS_CUDA(cudaStreamSynchronize(0));  // uploads and memsets ran on the legacy stream
  } catch (const CudaError &e) {
    return fail(e.code, e.what());
  } catch (const std::bad_alloc &) {
    return fail(MFS_ERR_OOM, "host allocation failed");
  }
  *out = h.release();
  return MFS_OK;
}

int mfs_solve_batch(mfs_handle *const *hs, int nsys, const double *const *rhs, double *const *x, double tol,
                    mfs_info *infos, int *status, int nthreads) {
  if (!hs || nsys < 0 || !rhs || !x || !(tol > 0.0)) return fail(MFS_ERR_INVALID, "bad batch arguments");
  for (int k = 0; k < nsys; ++k) {
    if (!hs[k] || !rhs[k] || !x[k]) return fail(MFS_ERR_INVALID, "NULL handle or vector in batch");
    for (int q = 0; q < k; ++q)
      if (hs[q] == hs[k]) return fail(MFS_ERR_INVALID, "a handle appears twice in one batch");
  }
  if (nsys == 0) return MFS_OK;
  for (int k = 0; k < nsys; ++k) {
    if (hs[k]->host_only) return fail(MFS_ERR_INVALID, "a handle of the batch was built with setup_only");
    if (hs[k]->device != hs[0]->device) return fail(MFS_ERR_INVALID, "fused batch: handles on different devices");
  }
  if (nthreads <= 0) {
    // fused: -nthreads groups, or (0) one group per 32 systems, at most 8;
    // each group (systems of similar size) is one fused plan driven by its
    // own host thread on its own stream, so the groups progress
    // independently (one group's float64 Arnoldi passes overlap another's
    // bandwidth-bound V-cycles, and host work overlaps GPU work)
    const int ngroups = nthreads < 0 ? -nthreads : std::max(1, std::min(8, (nsys + 31) / 32));
    const std::vector<std::vector<int>> groups = size_groups(hs, nsys, ngroups);
    std::vector<mfs_info> inf(nsys);
    std::vector<int> st(nsys, MFS_OK);
    std::vector<int> gcode(groups.size(), MFS_OK);
    std::vector<std::string> gmsg(groups.size());
    const double t0 = now_ms();
    auto run = [&](size_t g) {
      try {
        MFS_CUDA(cudaSetDevice(hs[0]->device));
        const std::vector<int> &m = groups[g];
        std::vector<mfs_handle *> hv;
        std::vector<const double *> rv;
        std::vector<double *> xv;
        for (int k : m) {
          hv.push_back(hs[k]);
          rv.push_back(rhs[k]);
          xv.push_back(x[k]);
        }
        std::vector<mfs_info> ginf(m.size());
        std::vector<int> gst(m.size(), MFS_OK);
        FusedBatch *B = fused_for(hv.data(), (int)hv.size());
        fused_solve(*B, rv.data(), xv.data(), tol, ginf, gst);
        for (size_t q = 0; q < m.size(); ++q) {
          inf[m[q]] = ginf[q];
          st[m[q]] = gst[q];
        }
      } catch (const CudaError &e) {
        gcode[g] = e.code;
        gmsg[g] = e.what();
      } catch (const std::bad_alloc &) {
        gcode[g] = MFS_ERR_OOM;
        gmsg[g] = "host allocation failed";
      }
    };
    std::vector<std::thread> pool;
    for (size_t g = 1; g < groups.size(); ++g) pool.emplace_back(run, g);
    run(0);
    for (auto &t : pool) t.join();
    for (size_t g = 0; g < groups.size(); ++g)
      if (gcode[g] != MFS_OK) return fail(gcode[g], gmsg[g]);
    const double ms = now_ms() - t0;
    int rc = MFS_OK;
    for (int k = 0; k < nsys; ++k) {
      inf[k].solve_ms = ms;
      inf[k].setup_ms = hs[k]->setup_ms;
      inf[k].levels[0] = hs[k]->host->hg0.nlevels();
      inf[k].levels[1] = hs[k]->host->hg1.nlevels();
      if (infos) infos[k] = inf[k];
      if (status) status[k] = st[k];
      if (st[k] != MFS_OK && rc == MFS_OK) {
        rc = st[k];
        g_last_error = "system " + std::to_string(k) + ": " + mfs_strerror(st[k]);
      }
    }
    return rc;
  }
  int nt = nthreads;
  if (nt > nsys) nt = nsys;
  std::atomic<int> next(0);
  std::vector<int> st(nsys, MFS_OK);
  std::vector<mfs_info> inf(nsys);
  std::vector<std::string> err(nsys);
  auto worker = [&]() {
    int dev_set = -1;
    for (int k = next++; k < nsys; k = next++) {
      if (hs[k]->device != dev_set) {
        cudaSetDevice(hs[k]->device);
        dev_set = hs[k]->device;
      }
      st[k] = solve_impl(hs[k], rhs[k], x[k], tol, &inf[k], false);
      if (st[k] != MFS_OK) err[k] = g_last_error;
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
  worker();
  for (auto &t : pool) t.join();
  int rc = MFS_OK;
  for (int k = 0; k < nsys; ++k) {
    if (infos) infos[k] = inf[k];
    if (status) status[k] = st[k];
    if (st[k] != MFS_OK && rc == MFS_OK) {
      rc = st[k];
      g_last_error = "system " + std::to_string(k) + ": " + err[k];
    }
  }
  return rc;
}

static int with_io(mfs_handle *h, const double *in, double *out, void (*fn)(mfs_handle *, const double *, double *)) {
  if (h->host_only) return fail(MFS_ERR_INVALID, "handle was built with setup_only");
  try {
    if (h->own_stream) {
      if (!h->entry) MFS_CUDA(cudaEventCreateWithFlags(&h->entry, cudaEventDisableTiming));
      MFS_CUDA(cudaEventRecord(h->entry, 0));
      MFS_CUDA(cudaStreamWaitEvent(h->s, h->entry, 0));
    }
    const bool din = is_device_ptr(in), dout = is_device_ptr(out);
    const double *a = in;
    double *b = out;
    if (!din) {
      MFS_CUDA(cudaMemcpyAsync(h->bd, in, h->n * sizeof(double), cudaMemcpyHostToDevice, h->s));
      a = h->bd;
    }
    if (!dout) b = h->xd;
    {
      SolvePhase phase(h);
      fn(h, a, b);
    }
    if (!dout) MFS_CUDA(cudaMemcpyAsync(out, h->xd, h->n * sizeof(double), cudaMemcpyDeviceToHost, h->s));
    MFS_CUDA(cudaStreamSynchronize(h->s));
    MFS_CUDA(cudaGetLastError());
  } catch (const CudaError &e) {
    return fail(e.code, e.what());
  }
  return MFS_OK;
}

int mfs_dot(mfs_handle *h, const double *x, const double *y, double *out) {
  if (!h || !x || !y || !out) return fail(MFS_ERR_INVALID, "bad dot arguments");
  if (h->host_only) return fail(MFS_ERR_INVALID, "handle was built with setup_only");
  if (!is_device_ptr(x) || !is_device_ptr(y)) return fail(MFS_ERR_INVALID, "mfs_dot needs device vectors");
  try {
    if (h->own_stream) {
      if (!h->entry) MFS_CUDA(cudaEventCreateWithFlags(&h->entry, cudaEventDisableTiming));
      MFS_CUDA(cudaEventRecord(h->entry, 0));
      MFS_CUDA(cudaStreamWaitEvent(h->s, h->entry, 0));
    }
    *out = dot_host(h, x, y);
    MFS_CUDA(cudaGetLastError());
  } catch (const CudaError &e) {
    return fail(e.code, e.what());
  }
  return MFS_OK;
}

int mfs_fp64_rate(double *tflops, void *stream) {
  if (!tflops) return fail(MFS_ERR_INVALID, "mfs_fp64_rate: NULL output");
  const double r = dev::fp64_rate((cudaStream_t)stream);
  if (!(r > 0.0)) {
    cudaGetLastError();
    return fail(MFS_ERR_CUDA, "mfs_fp64_rate: CUDA error");
  }
  *tflops = r;
  return MFS_OK;
}

int mfs_apply(mfs_handle *h, const double *v, double *z) {
  if (!h || !v || !z || v == z) return fail(MFS_ERR_INVALID, "bad apply arguments");
  return with_io(h, v, z, [](mfs_handle *hh, const double *vv, double *zz) { precond_apply(hh, vv, zz); });
}

int mfs_matvec(mfs_handle *h, const double *x, double *y) {
  if (!h || !x || !y || x == y) return fail(MFS_ERR_INVALID, "bad matvec arguments");
  return with_io(h, x, y, matvec);
}

static const HBsr *export_matrix(const mfs_handle *h, int what, int group, int level, int i, int j) {
  const HGroup &g = group == 0 ? h->host->hg0 : h->host->hg1;
  if (group < 0 || group > 1 || level < 0 || level >= g.nlevels() || i < 0 || i >= g.nf) return nullptr;
  if (what == 0) {
    if (j < 0 || j >= g.nf) return nullptr;
    if (i == j) return &g.lv[level][i].A;
    if (level < (int)g.off.size()) {
      auto it = g.off[level].find({i, j});
      if (it != g.off[level].end()) return &it->second;
    }
    if (group == 1 && level == 0) {
      auto it = h->host->schur_off.find({i, j});
      if (it != h->host->schur_off.end()) return &it->second;
    }
    return nullptr;
  }
  if (level >= g.nlevels() - 1) return nullptr;
  if (what == 1) return &g.lv[level][i].P;
  if (what == 2) return &g.lv[level][i].R;
  return nullptr;
}

int mfs_export_csr(const mfs_handle *h, int what, int group, int level, int i, int j, int64_t *nrows,
                   int64_t *ncols, int64_t *nnz, int32_t *rowptr, int32_t *colind, double *vals) {
  if (!h || !nrows || !ncols || !nnz) return fail(MFS_ERR_INVALID, "bad export arguments");
  const HBsr *A = export_matrix(h, what, group, level, i, j);
  if (!A) return fail(MFS_ERR_INVALID, "no such matrix");
  const int64_t nr = A->nrows();
  *nrows = nr;
  *ncols = A->ncols();
  *nnz = A->nnzb() * A->br * A->bc;
  if (!rowptr || !colind || !vals) return MFS_OK;
  const int bs = A->br * A->bc;
  int64_t k = 0;
  rowptr[0] = 0;
  for (int64_t I = 0; I < A->nbr; ++I)
    for (int r = 0; r < A->br; ++r) {
      for (int64_t a = A->rp[I]; a < A->rp[I + 1]; ++a)
        for (int c = 0; c < A->bc; ++c) {
          colind[k] = (int32_t)(A->ci[a] * A->bc + c);
          vals[k] = A->v[a * bs + r * A->bc + c];
          ++k;
        }
      rowptr[I * A->br + r + 1] = (int32_t)k;
    }
  return MFS_OK;
}

int mfs_export_array(const mfs_handle *h, int what, int group, int level, int i, void *buf, int64_t cap,
                     int64_t *count) {
  if (!h || !count) return fail(MFS_ERR_INVALID, "bad export arguments");
  const HGroup &g = group == 0 ? h->host->hg0 : h->host->hg1;
  if (group < 0 || group > 1 || level < 0 || level >= g.nlevels() || i < 0 || i >= g.nf)
    return fail(MFS_ERR_INVALID, "no such level/field");
  const HLevelField &f = g.lv[level][i];
  if (what == 0) {
    *count = (int64_t)f.agg.size();
    if (buf && cap >= *count) std::memcpy(buf, f.agg.data(), f.agg.size() * sizeof(int32_t));
  } else if (what == 1) {
    *count = 1;
    if (buf && cap >= 1) *(double *)buf = f.lam;
  } else if (what == 2) {
    const std::vector<std::vector<double>> *src = nullptr;
    if (group == 0 && h->prm.precond == MFS_SIMPLE && level == 0) src = &h->host->dtilde;
    if (group == 0 && h->prm.precond == MFS_AMG_SIMPLE && level < (int)h->host->mono_dtilde.size())
      src = &h->host->mono_dtilde[level];
    if (!src || i >= (int)src->size()) return fail(MFS_ERR_INVALID, "no SIMPLE diagonal");
    *count = (int64_t)(*src)[i].size();
    if (buf && cap >= *count) std::memcpy(buf, (*src)[i].data(), (*src)[i].size() * sizeof(double));
  } else if (what == 3) {
    if (f.color.empty()) return fail(MFS_ERR_INVALID, "no Gauss-Seidel colours on this level");
    *count = (int64_t)f.color.size();
    if (buf && cap >= *count) std::memcpy(buf, f.color.data(), f.color.size() * sizeof(int32_t));
  } else {
    return fail(MFS_ERR_INVALID, "bad export kind");
  }
  return MFS_OK;
}

int mfs_kernel_stats(mfs_handle *h, double *out, int cap, int reset) {
  if (!h || !out) return fail(MFS_ERR_INVALID, "bad stats arguments");
  if (!h->prof) return fail(MFS_ERR_INVALID, "handle was built without profile");
  int k = 0;
  for (int c = 0; c < dev::K_NCLASS && 3 * c + 2 < cap; ++c, ++k) {
    out[3 * c] = h->prof->cls[c].launches;
    out[3 * c + 1] = h->prof->cls[c].ms;
    out[3 * c + 2] = h->prof->cls[c].bytes;
  }
  if (reset) h->prof->reset();
  return k;
}

int mfs_profile_filter(mfs_handle *h, int key, int64_t rows) {
  if (!h) return fail(MFS_ERR_INVALID, "bad handle");
  if (!h->prof) return fail(MFS_ERR_INVALID, "handle was built without profile");
  h->prof->filter_key = key;
  h->prof->filter_rows = rows;
  for (auto &g : h->graphs) g.release();  // recapture with the new set of event nodes
  return MFS_OK;
}

int mfs_kernel_detail(mfs_handle *h, double *out, int cap) {
  if (!h || !out) return fail(MFS_ERR_INVALID, "bad stats arguments");
  if (!h->prof) return fail(MFS_ERR_INVALID, "handle was built without profile");
  std::vector<std::pair<std::pair<int, int64_t>, KStat>> rows(h->prof->detail.begin(), h->prof->detail.end());
  std::sort(rows.begin(), rows.end(), [](const auto &a, const auto &b) { return a.second.ms > b.second.ms; });
  int k = 0;
  for (auto &r : rows) {
    if (6 * k + 5 >= cap) break;
    out[6 * k] = r.first.first;
    out[6 * k + 1] = (double)r.first.second;
    out[6 * k + 2] = r.second.launches;
    out[6 * k + 3] = r.second.ms;
    out[6 * k + 4] = r.second.bytes;
    out[6 * k + 5] = r.second.flops;
    ++k;
  }
  return k;
}

void mfs_free(mfs_handle *h) {
  if (!h) return;
  drop_fused(h);
  if (!h->host_only) {
    if (h->s) cudaStreamSynchronize(h->s);
    else cudaDeviceSynchronize();
  }
  delete h;
}

const char *mfs_strerror(int code) {
  switch (code) {
    case MFS_OK: return "ok";
    case MFS_ERR_INVALID: return "invalid argument";
    case MFS_ERR_CUDA: return "CUDA error";
    case MFS_ERR_OOM: return "out of device memory";
    case MFS_ERR_SINGULAR: return "singular matrix in setup";
    case MFS_ERR_NOT_CONVERGED: return "GMRES did not converge within max_iters";
    case MFS_ERR_BREAKDOWN: return "non-finite value in GMRES";
    case MFS_ERR_SETUP: return "aggregation failed";
    default: return "unknown error";
  }
}

const char *mfs_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
