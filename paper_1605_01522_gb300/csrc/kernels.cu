// Solve-phase CUDA kernels for sm_103a: blocked SELL-32 and plain-BSR SpMV,
// the fused residual + polynomial smoothing step, multicolour Gauss-Seidel,
// the coarse solves and the CGS2 Arnoldi reductions.  The float32 sparse work
// is bound by HBM bandwidth (small coarse levels by latency), the float64
// matvec and CGS2 passes by GB300's FP64 rate; loads of a warp are contiguous
// per slot and every reduction has a fixed order.
#include "kernels.cuh"

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <type_traits>

namespace mfs {
namespace dev {

namespace {

constexpr int kThreads = 256;
// CTAs of the one-thread-per-row SELL-32 kernels: two slices, so that a grid
// of a few thousand CTAs spreads evenly over the SMs (with 256-thread CTAs
// the busiest SM held 8 where the average was 7.1)
constexpr int kSellThreads = 64;
// plain-BSR matrices with at most kCtaRowsMax rows averaging at least
// kCtaRowBlocks blocks per row take one CTA per row instead of one warp
constexpr int64_t kCtaRowsMax = 4096;
constexpr int64_t kCtaRowBlocks = 128;
constexpr int kGsCtaThreads = 1024;  // threads of the one-CTA Gauss-Seidel kernel for small levels
LaunchHook *g_hook = nullptr;
// > 0 while this thread's launches must bypass the process-wide hook
thread_local int g_hook_off = 0;

// While set, this thread's launches are appended here instead of issued.
thread_local Recorder *g_rec = nullptr;
// While set, this thread's solve-phase launches are programmatic dependent
// launches where they directly follow another of its kernel launches on the
// same stream (g_pdl_prev): a kernel after a copy, an event or a graph launch
// is launched normally.
thread_local unsigned g_pdl = 0;  // largest grid (CTAs) launched this way; 0: none
thread_local cudaStream_t g_pdl_prev = nullptr;
// accounting of the launch being issued (HookScope fills it for the recorder)
thread_local RecOp g_acct;

struct HookScope {
  cudaStream_t s;
  int cls;
  double bytes;
  int sig;
  int64_t rows;
  double flops;
  bool on = false;
  HookScope(cudaStream_t s_, int c, double b, int sg, int64_t r, double f)
      : s(s_), cls(c), bytes(b), sig(sg), rows(r), flops(f) {
    if (g_rec) {
      g_acct.cls = c;
      g_acct.sig = sg;
      g_acct.rows = r;
      g_acct.bytes = b;
      g_acct.flops = f;
      return;
    }
    if (g_hook && !g_hook_off) on = g_hook->before(s, cls, sig, rows);
    if (on) g_pdl_prev = nullptr;  // an event precedes the launch
  }
  ~HookScope() {
    if (on) {
      g_hook->after(s, cls, bytes, sig, rows, flops);
      g_pdl_prev = nullptr;
    }
  }
};

// Every solve-phase kernel is a traits struct K: K::Args (its arguments),
// K::run(args, block, blocks) (its body for one block of a grid of `blocks`)
// and K::kMaxThreads.  k_solo runs it over a normal grid; k_multi runs many
// independent launches of K (one per system of a batch) as ONE grid: CTA c
// runs block map[c].bid of the launch whose arguments are tab[map[c].t],
// unless that launch's system map[c].g is inactive.
// Launched as a programmatic dependent launch (set_pdl), a kernel may be
// scheduled while its predecessor in the stream still runs: it first waits
// until that predecessor has completed and its writes are visible, then lets
// its own successor start launching.  Launched normally, both are no-ops.
template <class K>
__global__ void __launch_bounds__(K::kMaxThreads) k_solo(const __grid_constant__ typename K::Args a) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  K::run(a, (int)blockIdx.x, (int)gridDim.x);
}

// CTAs per SM the multi-system form of K must fit (K::kMinBlocks, default 1):
// its arguments come from a table instead of the constant bank, which costs
// registers; the one-thread-per-row SELL kernels are held to the 32 registers
// of their single-system form so that as many CTAs stay resident
template <class K, class = void> struct MinBlocks {
  static constexpr int value = 1;
};
template <class K> struct MinBlocks<K, std::void_t<decltype(K::kMinBlocks)>> {
  static constexpr int value = K::kMinBlocks;
};

template <class K>
__global__ void __launch_bounds__(K::kMaxThreads, MinBlocks<K>::value)
k_multi(const typename K::Args *__restrict__ tab, const MsBlock *__restrict__ map, const int *__restrict__ active) {
  const MsBlock m = map[blockIdx.x];
  if (active != nullptr && active[m.g] == 0) return;
  K::run(tab[m.t], m.bid, m.nb);
}

// issue one launch of K, or record it (with the accounting of the enclosing
// HookScope) when this thread has a recorder
template <class K>
void go(unsigned grid, unsigned threads, size_t smem, cudaStream_t s, const typename K::Args &a) {
  if (g_rec) {
    RecOp op = g_acct;
    op.fn = (const void *)&k_multi<K>;
    op.grid = grid;
    op.threads = threads;
    op.smem = smem;
    op.args.assign((const unsigned char *)&a, (const unsigned char *)&a + sizeof(a));
    g_rec->ops.push_back(std::move(op));
    g_acct = RecOp();
    return;
  }
  const bool pdl = grid <= g_pdl && g_pdl_prev == s;
  g_pdl_prev = g_pdl ? s : nullptr;
  if (pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_solo<K>, a);
    return;
  }
  k_solo<K><<<grid, threads, smem, s>>>(a);
}

template <typename T> int sparse_sig(const Sell &A) {
  // 3 / 9: SELL-32 with 4 / 8 slots in flight
  const int layout = A.kind == 0 && A.unroll == 4 ? 3 : (A.kind == 0 && A.unroll == 8 ? 9 : A.kind);
  return layout * 1000 + A.br * 100 + A.bc * 10 + (sizeof(T) == 8 ? 1 : 0);
}

// algorithmic bytes of one pass over a block matrix: values + block-column
// indices + row lengths, each read once
template <typename T> double matrix_bytes(const Sell &A) {
  return (double)A.nnzb * (A.br * A.bc * sizeof(T) + sizeof(int32_t)) + (double)A.nbr * sizeof(int32_t);
}

// The N entries of one plain-BSR block (row-major, consecutive) in the widest
// loads its size allows: 16-byte loads when N * sizeof(T) is a multiple of
// 16, 8-byte ones when a multiple of 8, else one load per entry.  Block k
// starts k * N * sizeof(T) bytes into a value array that starts on a 16-byte
// boundary (every value array is its own allocation; the setup checks it), so
// every vector is aligned.  Fewer, wider loads keep the load queue of one-warp-per-row
// kernels from filling (6x6 float blocks: 9 loads instead of 36).
template <int N, typename T>
__device__ __forceinline__ void ldg_block(const T *__restrict__ p, T (&o)[N]) {
  constexpr int B = N * (int)sizeof(T);
  if constexpr (sizeof(T) == 8 && B % 16 == 0) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      const double2 v = __ldg(q + i);
      o[2 * i] = v.x;
      o[2 * i + 1] = v.y;
    }
  } else if constexpr (sizeof(T) == 4 && B % 16 == 0) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int i = 0; i < N / 4; ++i) {
      const float4 v = __ldg(q + i);
      o[4 * i] = v.x;
      o[4 * i + 1] = v.y;
      o[4 * i + 2] = v.z;
      o[4 * i + 3] = v.w;
    }
  } else if constexpr (sizeof(T) == 4 && B % 8 == 0) {
    const float2 *q = reinterpret_cast<const float2 *>(p);
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      const float2 v = __ldg(q + i);
      o[2 * i] = v.x;
      o[2 * i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) o[i] = __ldg(p + i);
  }
}

inline unsigned grid_for(int64_t n, int threads = kThreads) {
  return (unsigned)((n + threads - 1) / threads);
}

template <int BR, int BC, typename T, int U>
__device__ __forceinline__ void sell_row(const int32_t *__restrict__ sp, const int32_t *__restrict__ rl,
                                         const int32_t *__restrict__ col, const T *__restrict__ val,
                                         const T *__restrict__ x, int64_t row, T (&acc)[BR]) {
  const int lane = (int)(row & 31);
  const int64_t slice = row >> 5;
  const int64_t base = sp[slice];
  const int len = rl[row];
  const int32_t *cp = col + base * 32 + lane;
  const T *vp = val + base * (BR * BC * 32) + lane;
#pragma unroll
  for (int r = 0; r < BR; ++r) acc[r] = T(0);
  // U slots in flight per thread (chosen per matrix by the layout autotuner)
#pragma unroll U
  for (int t = 0; t < len; ++t) {
    const int64_t c = __ldg(cp + (int64_t)t * 32);
    T xv[BC];
#pragma unroll
    for (int q = 0; q < BC; ++q) xv[q] = __ldg(x + c * BC + q);
    const T *v = vp + (int64_t)t * (BR * BC * 32);
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int q = 0; q < BC; ++q) acc[r] += __ldg(v + (r * BC + q) * 32) * xv[q];
  }
}

// One warp per block row of a plain BSR matrix: lanes stride over the row's
// blocks, then a fixed xor-butterfly sums the lanes (all lanes get the sums).
template <int BR, int BC, typename T>
__device__ __forceinline__ void bsr_warp_row(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                             const T *__restrict__ val, const T *__restrict__ x, int64_t row,
                                             int lane, T (&acc)[BR]) {
  const int lo = rp[row], hi = rp[row + 1];
#pragma unroll
  for (int r = 0; r < BR; ++r) acc[r] = T(0);
  for (int k = lo + lane; k < hi; k += 32) {
    const int64_t c = __ldg(col + k);
    T xv[BC];
#pragma unroll
    for (int q = 0; q < BC; ++q) xv[q] = __ldg(x + c * BC + q);
    T blk[BR * BC];
    ldg_block<BR * BC, T>(val + (int64_t)k * (BR * BC), blk);
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int q = 0; q < BC; ++q) acc[r] += blk[r * BC + q] * xv[q];
  }
#pragma unroll
  for (int r = 0; r < BR; ++r)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
}

// dx of one node from its row sums acc (see gs_sweeps), written into x
template <int BR, typename T>
__device__ __forceinline__ void gs_update(const T (&acc)[BR], int64_t node, const T *__restrict__ dblk,
                                          const T *__restrict__ b, T *x, T omega, bool backward) {
  const T *D = dblk + node * (BR * BR);
  T dx[BR];
  if (!backward) {
#pragma unroll
    for (int r = 0; r < BR; ++r) {
      T res = b[node * BR + r] - acc[r];
#pragma unroll
      for (int c = 0; c < r; ++c) res -= D[r * BR + c] * dx[c];
      dx[r] = omega * res / D[r * BR + r];
    }
  } else {
#pragma unroll
    for (int r = BR - 1; r >= 0; --r) {
      T res = b[node * BR + r] - acc[r];
#pragma unroll
      for (int c = r + 1; c < BR; ++c) res -= D[r * BR + c] * dx[c];
      dx[r] = omega * res / D[r * BR + r];
    }
  }
#pragma unroll
  for (int r = 0; r < BR; ++r) x[node * BR + r] += dx[r];
}

template <int BR, typename T>
__device__ __forceinline__ T pick(const T (&acc)[BR], int r) {
  T a = acc[0];
#pragma unroll
  for (int q = 1; q < BR; ++q)
    if (q == r) a = acc[q];
  return a;
}

template <int BR, int BC, typename T>
__device__ __forceinline__ void d_spmv_warp(int64_t nbr, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
            const T *__restrict__ val, const T *__restrict__ x, T *y, T alpha, T beta, const T *z, int bid_, int nb_) {
  const int64_t row = ((int64_t)bid_ * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= nbr) return;
  T acc[BR];
  bsr_warp_row<BR, BC, T>(rp, col, val, x, row, lane, acc);
  if (lane < BR) {
    const int64_t i = row * BR + lane;
    const T a = pick<BR, T>(acc, lane);
    y[i] = z != nullptr ? alpha * a + beta * z[i] : alpha * a;
  }
}
template <int BR, int BC, typename T>
struct KSpmvWarp {
  static constexpr int kMaxThreads = kThreads;
  struct Args {
    int64_t nbr;
    const int32_t *rp;
    const int32_t *col;
    const T *val;
    const T *x;
    T *y;
    T alpha;
    T beta;
    const T *z;
  };
  static __device__ __forceinline__ void run(const Args &a, int bid, int nb) {
    d_spmv_warp<BR, BC, T>(a.nbr, a.rp, a.col, a.val, a.x, a.y, a.alpha, a.beta, a.z, bid, nb);
  }
};

// One CTA per block row, for few and long rows (restrictions to small coarse
// levels): threads stride over the row's blocks, then a fixed butterfly per
// warp and a fixed-order sum over the warps.
template <int BR, int BC, typename T>
__device__ __forceinline__ void d_spmv_cta(int64_t nbr, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
           const T *__restrict__ val, const T *__restrict__ x, T *y, T alpha, T beta, const T *z, int bid_, int nb_) {
  __shared__ T part[kThreads / 32][BR];
  const int64_t row = bid_;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T acc[BR];
#pragma unroll
  for (int r = 0; r < BR; ++r) acc[r] = T(0);
  for (int k = rp[row] + threadIdx.x; k < rp[row + 1]; k += blockDim.x) {
    const int64_t c = __ldg(col + k);
    T xv[BC];
#pragma unroll
    for (int q = 0; q < BC; ++q) xv[q] = __ldg(x + c * BC + q);
    T blk[BR * BC];
    ldg_block<BR * BC, T>(val + (int64_t)k * (BR * BC), blk);
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int q = 0; q < BC; ++q) acc[r] += blk[r * BC + q] * xv[q];
  }
#pragma unroll
  for (int r = 0; r < BR; ++r) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
    if (lane == 0) part[warp][r] = acc[r];
  }
  __syncthreads();
  if (threadIdx.x < BR) {
    T a = T(0);
    for (int w = 0; w < kThreads / 32; ++w) a += part[w][threadIdx.x];
    const int64_t i = row * BR + threadIdx.x;
    y[i] = z != nullptr ? alpha * a + beta * z[i] : alpha * a;
  }
}
template <int BR, int BC, typename T>
struct KSpmvCta {
  static constexpr int kMaxThreads = kThreads;
  struct Args {
    int64_t nbr;
    const int32_t *rp;
    const int32_t *col;
    const T *val;
    const T *x;
    T *y;
    T alpha;
    T beta;
    const T *z;
  };
  static __device__ __forceinline__ void run(const Args &a, int bid, int nb) {
    d_spmv_cta<BR, BC, T>(a.nbr, a.rp, a.col, a.val, a.x, a.y, a.alpha, a.beta, a.z, bid, nb);
  }
};

template <int BR, typename T>
__device__ __forceinline__ void d_smooth_warp(int64_t nbr, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
              const T *__restrict__ val, const T *__restrict__ dinv, const T *__restrict__ b,
              const T *__restrict__ x, T *__restrict__ xout, T *__restrict__ d, T c1, T c2, int bid_, int nb_) {
  const int64_t row = ((int64_t)bid_ * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= nbr) return;
  T acc[BR];
  bsr_warp_row<BR, BR, T>(rp, col, val, x, row, lane, acc);
  if (lane < BR) {
    const int64_t i = row * BR + lane;
    const T res = b[i] - pick<BR, T>(acc, lane);
    const T dd = c1 * d[i] + c2 * dinv[i] * res;
    d[i] = dd;
    xout[i] = x[i] + dd;
  }
}
template <int BR, typename T>
struct KSmoothWarp {
  static constexpr int kMaxThreads = kThreads;
  struct Args {
    int64_t nbr;
    const int32_t *rp;
    const int32_t *col;
    const T *val;
    const T *dinv;
    const T *b;
    const T *x;
    T *xout;
    T *d;
    T c1;
    T c2;
  };
  static __device__ __forceinline__ void run(const Args &a, int bid, int nb) {
    d_smooth_warp<BR, T>(a.nbr, a.rp, a.col, a.val, a.dinv, a.b, a.x, a.xout, a.d, a.c1, a.c2, bid, nb);
  }
};

template <int BR, int BC, typename T, int U>
__device__ __forceinline__ void d_spmv(int64_t nbr, const int32_t *__restrict__ sp, const int32_t *__restrict__ rl,
       const int32_t *__restrict__ col, const T *__restrict__ val, const T *__restrict__ x, T *y,
       T alpha, T beta, const T *z, int bid_, int nb_) {
  const int64_t row = (int64_t)bid_ * blockDim.x + threadIdx.x;
  if (row >= nbr) return;
  T acc[BR];
  sell_row<BR, BC, T, U>(sp, rl, col, val, x, row, acc);
  T *yp = y + row * BR;
  if (z != nullptr) {
    const T *zp = z + row * BR;
    T zv[BR];
#pragma unroll
    for (int r = 0; r < BR; ++r) zv[r] = zp[r];
#pragma unroll
    for (int r = 0; r < BR; ++r) yp[r] = alpha * acc[r] + beta * zv[r];
  } else {
#pragma unroll
    for (int r = 0; r < BR; ++r) yp[r] = alpha * acc[r];
  }
}
template <int BR, int BC, typename T, int U>
struct KSpmvSell {
  static constexpr int kMaxThreads = kThreads;
  static constexpr int kMinBlocks = BR * BC <= 9 ? 8 : 1;  // multi-system form: <= 32 registers
  struct Args {
    int64_t nbr;
    const int32_t *sp;
    const int32_t *rl;
    const int32_t *col;
    const T *val;
    const T *x;
    T *y;
    T alpha;
    T beta;
    const T *z;
  };
  static __device__ __forceinline__ void run(const Args &a, int bid, int nb) {
    d_spmv<BR, BC, T, U>(a.nbr, a.sp, a.rl, a.col, a.val, a.x, a.y, a.alpha, a.beta, a.z, bid, nb);
  }
};

// Merged coupled rows in float64, H threads per block row.  H = 1: one
// thread per row, 64-thread CTAs (two slices).  H > 1: a CTA of 32 H threads
// takes one slice of 32 rows, its warp h the slots h, h + H, ...; the H
// partial sums of a row are added in the fixed order h = 0, 1, ... through
// shared memory.  More threads per row keep more FP64 FMAs in flight (the
// FP64 pipe bounds this kernel on GB300).
template <int BR, int B0, int B1, int B2, int H>
__device__ __forceinline__ void d_spmv_rows(int64_t nbr, const int32_t *__restrict__ sp, const int32_t *__restrict__ rl,
            const int32_t *__restrict__ col, const double *__restrict__ val, const double *__restrict__ x0,
            const double *__restrict__ x1, const double *__restrict__ x2, double *__restrict__ y, int bid_, int nb_) {
  constexpr int BCT = B0 + B1 + B2;
  const int lane = threadIdx.x & 31, h = H == 1 ? 0 : threadIdx.x >> 5;
  const int64_t row = H == 1 ? (int64_t)bid_ * 64 + threadIdx.x : (int64_t)bid_ * 32 + lane;
  const bool active = row < nbr;
  double acc[BR];
#pragma unroll
  for (int r = 0; r < BR; ++r) acc[r] = 0.0;
  if (active) {
    const int64_t base = sp[row >> 5];
    const int len = rl[row];
    const int32_t *cp = col + base * 32 + lane;
    const double *vp = val + base * (BR * BCT * 32) + lane;
#pragma unroll 2
    for (int t = h; t < len; t += H) {
      const int64_t c = __ldg(cp + (int64_t)t * 32);
      double xv[BCT];
#pragma unroll
      for (int q = 0; q < B0; ++q) xv[q] = __ldg(x0 + c * B0 + q);
#pragma unroll
      for (int q = 0; q < B1; ++q) xv[B0 + q] = __ldg(x1 + c * B1 + q);
#pragma unroll
      for (int q = 0; q < B2; ++q) xv[B0 + B1 + q] = __ldg(x2 + c * B2 + q);
      const double *v = vp + (int64_t)t * (BR * BCT * 32);
#pragma unroll
      for (int r = 0; r < BR; ++r)
#pragma unroll
        for (int q = 0; q < BCT; ++q) acc[r] += __ldg(v + (r * BCT + q) * 32) * xv[q];
    }
  }
  if constexpr (H == 1) {
    if (active)
#pragma unroll
      for (int r = 0; r < BR; ++r) y[row * BR + r] = acc[r];
  } else {
    __shared__ double part[H - 1][BR][32];
    if (h > 0)
#pragma unroll
      for (int r = 0; r < BR; ++r) part[h - 1][r][lane] = acc[r];
    __syncthreads();
    if (h == 0 && active)
#pragma unroll
      for (int r = 0; r < BR; ++r) {
        double a = acc[r];
#pragma unroll
        for (int q = 0; q < H - 1; ++q) a += part[q][r][lane];
        y[row * BR + r] = a;
      }
  }
}
template <int BR, int B0, int B1, int B2, int H>
struct KSpmvRows {
  static constexpr int kMaxThreads = (H == 1 ? 64 : 32 * H);
  struct Args {
    int64_t nbr;
    const int32_t *sp;
    const int32_t *rl;
    const int32_t *col;
    const double *val;
    const double *x0;
    const double *x1;
    const double *x2;
    double *y;
  };
  static __device__ __forceinline__ void run(const Args &a, int bid, int nb) {
    d_spmv_rows<BR, B0, B1, B2, H>(a.nbr, a.sp, a.rl, a.col, a.val, a.x0, a.x1, a.x2, a.y, bid, nb);
  }
};

template <int BR, typename T, int U>
__device__ __forceinline__ void d_smooth(int64_t nbr, const int32_t *__restrict__ sp, const int32_t *__restrict__ rl,
         const int32_t *__restrict__ col, const T *__restrict__ val, const T *__restrict__ dinv,
         const T *__restrict__ b, const T *__restrict__ x, T *__restrict__ xout, T *__restrict__ d,
         T c1, T c2, int bid_, int nb_) {
  const int64_t row = (int64_t)bid_ * blockDim.x + threadIdx.x;
  if (row >= nbr) return;
  T acc[BR];
  sell_row<BR, BR, T, U>(sp, rl, col, val, x, row, acc);
#pragma unroll
  for (int r = 0; r < BR; ++r) {
    const int64_t i = row * BR + r;
    const T res = b[i] - acc[r];
    const T dd = c1 * d[i] + c2 * dinv[i] * res;
    d[i] = dd;
    xout[i] = x[i] + dd;
  }
}
template <int BR, typename T, int U>
struct KSmoothSell {
  static constexpr int kMaxThreads = kThreads;
  static constexpr int kMinBlocks = BR <= 3 ? 8 : 1;  // multi-system form: <= 32 registers
  struct Args {
    int64_t nbr;
    const int32_t *sp;
    const int32_t *rl;
    const int32_t *col;
    const T *val;
    const T *dinv;
    const T *b;
    const T *x;
    T *xout;
    T *d;
    T c1;
    T c2;
  };
  static __device__ __forceinline__ void run(const Args &a, int bid, int nb) {
    d_smooth<BR, T, U>(a.nbr, a.sp, a.rl, a.col, a.val, a.dinv, a.b, a.x, a.xout, a.d, a.c1, a.c2, bid, nb);
  }
};

// G lanes per row of a plain BSR matrix: the lanes of a group stride over the
// row's blocks, then a fixed xor-butterfly inside the group sums them.  x goes
// through the read-only path: in a one-colour launch only rows of that colour
// write x, and they never read each other's entries (earlier colours wrote in
// earlier launches).
template <int BR, int G, typename T>
__device__ __forceinline__ void gs_group_row(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                             const T *__restrict__ val, const T *x, int64_t row, bool active,
                                             int gl, T (&acc)[BR]) {
#pragma unroll
  for (int r = 0; r < BR; ++r) acc[r] = T(0);
  const int lo = active ? rp[row] : 0, hi = active ? rp[row + 1] : 0;
  for (int k = lo + gl; k < hi; k += G) {
    const int64_t c = __ldg(col + k);
    T xv[BR];
#pragma unroll
    for (int q = 0; q < BR; ++q) xv[q] = __ldg(x + c * BR + q);
    T blk[BR * BR];
    ldg_block<BR * BR, T>(val + (int64_t)k * (BR * BR), blk);
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int q = 0; q < BR; ++q) acc[r] += blk[r * BR + q] * xv[q];
  }
#pragma unroll
  for (int r = 0; r < BR; ++r)
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
}

// One colour: reordered rows [r0, r1), G lanes per row.
template <int BR, typename T, int G>
__device__ __forceinline__ void d_gs_color(int64_t r0, int64_t r1, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
           const T *__restrict__ val, const int32_t *__restrict__ rowidx, const T *__restrict__ dblk,
           const T *__restrict__ b, T *x, T omega, int backward, int bid_, int nb_) {
  const int64_t t = (int64_t)bid_ * blockDim.x + threadIdx.x;
  const int64_t row = r0 + t / G;
  const int gl = (int)(t % G);
  const bool active = row < r1;
  T acc[BR];
  gs_group_row<BR, G, T>(rp, col, val, x, row, active, gl, acc);
  if (active && gl == 0) gs_update<BR, T>(acc, rowidx[row], dblk, b, x, omega, backward != 0);
}
template <int BR, typename T, int G>
struct KGsColor {
  static constexpr int kMaxThreads = kThreads;
  struct Args {
    int64_t r0;
    int64_t r1;
    const int32_t *rp;
    const int32_t *col;
    const T *val;
    const int32_t *rowidx;
    const T *dblk;
    const T *b;
    T *x;
    T omega;
    int backward;
  };
  static __device__ __forceinline__ void run(const Args &a, int bid, int nb) {
    d_gs_color<BR, T, G>(a.r0, a.r1, a.rp, a.col, a.val, a.rowidx, a.dblk, a.b, a.x, a.omega, a.backward, bid, nb);
  }
};

// All colours and sweeps of a small level in one CTA: x lives in shared
// memory for the whole launch (loaded first, written back last), so the
// colour-to-colour dependency goes through shared memory and __syncthreads;
// groups of G lanes stride over the rows of a colour.  Every thread reaches
// every barrier (uniform loops, no early exit).
template <int BR, typename T, int G>
__device__ __forceinline__ void d_gs_small(int nc, int64_t n, const int32_t *__restrict__ coff, const int32_t *__restrict__ rp,
           const int32_t *__restrict__ col, const T *__restrict__ val, const int32_t *__restrict__ rowidx,
           const T *__restrict__ dblk, const T *__restrict__ b, T *__restrict__ x, T omega, int sweeps,
           int backward, int bid_, int nb_) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *xs = reinterpret_cast<T *>(smem_raw);
  const int tid = threadIdx.x;
  for (int64_t k = tid; k < n * BR; k += blockDim.x) xs[k] = x[k];
  __syncthreads();
  const int ngroups = blockDim.x / G;
  const int gid = tid / G, gl = tid % G;
  for (int sw = 0; sw < sweeps; ++sw)
    for (int q = 0; q < nc; ++q) {
      const int c = backward ? nc - 1 - q : q;
      const int lo = coff[c], hi = coff[c + 1];
      for (int base = lo; base < hi; base += ngroups) {
        const int row = base + gid;
        const bool active = row < hi;
        T acc[BR];
#pragma unroll
        for (int r = 0; r < BR; ++r) acc[r] = T(0);
        const int k0 = active ? rp[row] : 0, k1 = active ? rp[row + 1] : 0;
        for (int k = k0 + gl; k < k1; k += G) {
          const int64_t cc = __ldg(col + k);
          const T *v = val + (int64_t)k * (BR * BR);
#pragma unroll
          for (int r = 0; r < BR; ++r)
#pragma unroll
            for (int qq = 0; qq < BR; ++qq) acc[r] += __ldg(v + r * BR + qq) * xs[cc * BR + qq];
        }
#pragma unroll
        for (int r = 0; r < BR; ++r)
#pragma unroll
          for (int o = G / 2; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
        if (active && gl == 0) gs_update<BR, T>(acc, rowidx[row], dblk, b, xs, omega, backward != 0);
      }
      __syncthreads();
    }
  for (int64_t k = tid; k < n * BR; k += blockDim.x) x[k] = xs[k];
}
template <int BR, typename T, int G>
struct KGsSmall {
  static constexpr int kMaxThreads = kGsCtaThreads;
  struct Args {
    int nc;
    int64_t n;
    const int32_t *coff;
    const int32_t *rp;
    const int32_t *col;
    const T *val;
    const int32_t *rowidx;
    const T *dblk;
    const T *b;
    T *x;
    T omega;
    int sweeps;
    int backward;
  };
  static __device__ __forceinline__ void run(const Args &a, int bid, int nb) {
    d_gs_small<BR, T, G>(a.nc, a.n, a.coff, a.rp, a.col, a.val, a.rowidx, a.dblk, a.b, a.x, a.omega, a.sweeps, a.backward, bid, nb);
  }
};

// x = inv b for the explicit inverse of a coarsest matrix (row-major, float64):
// b staged in shared memory as float64, one warp per row, fixed butterfly sum.
template <typename T>
__device__ __forceinline__ void d_inv_apply(int n, const double *__restrict__ inv, const T *__restrict__ b, T *__restrict__ x, int bid_, int nb_) {
  extern __shared__ double bs[];
  for (int j = threadIdx.x; j < n; j += blockDim.x) bs[j] = (double)b[j];
  __syncthreads();
  const int row = bid_ * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const double *a = inv + (int64_t)row * n;
  double acc = 0.0;
  for (int j = lane; j < n; j += 32) acc += __ldg(a + j) * bs[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) x[row] = (T)acc;
}
template <typename T>
struct KInvApply {
  static constexpr int kMaxThreads = kThreads;
  struct Args {
    int n;
    const double *inv;
    const T *b;
    T *x;
  };
  static __device__ __forceinline__ void run(const Args &a, int bid, int nb) {
    d_inv_apply<T>(a.n, a.inv, a.b, a.x, bid, nb);
  }
};

template <typename T>
__device__ __forceinline__ void d_smooth_first(int64_t n, const T *__restrict__ dinv, const T *__restrict__ b,
                               T *__restrict__ x, T *__restrict__ d, T c2, int bid_, int nb_) {
  for (int64_t i = (int64_t)bid_ * blockDim.x + threadIdx.x; i < n; i += (int64_t)nb_ * blockDim.x) {
    const T dd = c2 * dinv[i] * b[i];
    d[i] = dd;
    x[i] = dd;
  }
}
template <typename T>
struct KSmoothFirst {
  static constexpr int kMaxThreads = kThreads;
  struct Args {
    int64_t n;
    const T *dinv;
    const T *b;
    T *x;
    T *d;
    T c2;
  };
  static __device__ __forceinline__ void run(const Args &a, int bid, int nb) {
    d_smooth_first<T>(a.n, a.dinv, a.b, a.x, a.d, a.c2, bid, nb);
  }
};

// Dense LU solve in one CTA, blocked by 32: one warp solves each 32 x 32
// diagonal block with shuffles, then all warps update the rows below (above)
// with that block's 32 new unknowns.  y lives in shared memory, and so do the
// factors when they fit (staged == 1), which keeps the warp's sequential
// steps off global-memory latency.
template <typename T>
__device__ __forceinline__ void d_lu_solve(int n, const double *__restrict__ lu_g, const int32_t *__restrict__ perm,
           const T *__restrict__ b, T *__restrict__ x, int staged, int bid_, int nb_) {
  extern __shared__ double sm[];
  double *y = sm;
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31;
  const double *lu = lu_g;
  if (staged) {
    double *ls = sm + n;
    for (int64_t i = tid; i < (int64_t)n * n; i += nt) ls[i] = lu_g[i];
    lu = ls;
  }
  for (int i = tid; i < n; i += nt) y[i] = (double)b[perm[i]];
  __syncthreads();
  // forward: L y = Pb, unit lower triangle
  for (int k0 = 0; k0 < n; k0 += 32) {
    const int nb = min(32, n - k0);
    if (warp == 0) {
      // this lane's row of the 32 x 32 diagonal block, loaded up front
      double Lr[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) Lr[c] = (c < nb && lane < nb) ? lu[(int64_t)(k0 + c) * n + k0 + lane] : 0.0;
      double yv = lane < nb ? y[k0 + lane] : 0.0;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        if (c < nb) {
          const double yc = __shfl_sync(0xffffffffu, yv, c);
          if (lane > c && lane < nb) yv -= Lr[c] * yc;
        }
      }
      if (lane < nb) y[k0 + lane] = yv;
    }
    __syncthreads();
    for (int i = k0 + nb + tid; i < n; i += nt) {
      double s = 0.0;
#pragma unroll
      for (int c = 0; c < 32; ++c)  // all 32 loads in flight at once
        if (c < nb) s += lu[(int64_t)(k0 + c) * n + i] * y[k0 + c];
      y[i] -= s;
    }
    __syncthreads();
  }
  // backward: U x = y
  const int last = ((n - 1) / 32) * 32;
  for (int k0 = last; k0 >= 0; k0 -= 32) {
    const int nb = min(32, n - k0);
    if (warp == 0) {
      double Ur[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) Ur[c] = (c < nb && lane < nb) ? lu[(int64_t)(k0 + c) * n + k0 + lane] : 1.0;
      double yv = lane < nb ? y[k0 + lane] : 0.0;
#pragma unroll
      for (int c = 31; c >= 0; --c) {
        if (c < nb) {
          if (lane == c) yv /= Ur[c];
          const double yc = __shfl_sync(0xffffffffu, yv, c);
          if (lane < c) yv -= Ur[c] * yc;
        }
      }
      if (lane < nb) y[k0 + lane] = yv;
    }
    __syncthreads();
    for (int i = tid; i < k0; i += nt) {
      double s = 0.0;
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c < nb) s += lu[(int64_t)(k0 + c) * n + i] * y[k0 + c];
      y[i] -= s;
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += nt) x[i] = (T)y[i];
}
template <typename T>
struct KLuSolve {
  static constexpr int kMaxThreads = 512;
  struct Args {
    int n;
    const double *lu_g;
    const int32_t *perm;
    const T *b;
    T *x;
    int staged;
  };
  static __device__ __forceinline__ void run(const Args &a, int bid, int nb) {
    d_lu_solve<T>(a.n, a.lu_g, a.perm, a.b, a.x, a.staged, bid, nb);
  }
};

template <typename T>
__device__ __forceinline__ void d_fill(T *x, int64_t n, T v, int bid_, int nb_) {
  for (int64_t i = (int64_t)bid_ * blockDim.x + threadIdx.x; i < n; i += (int64_t)nb_ * blockDim.x)
    x[i] = v;
}
template <typename T>
struct KFill {
  static constexpr int kMaxThreads = kThreads;
  struct Args {
    T *x;
    int64_t n;
    T v;
  };
  static __device__ __forceinline__ void run(const Args &a, int bid, int nb) {
    d_fill<T>(a.x, a.n, a.v, bid, nb);
  }
};

template <typename T>
__device__ __forceinline__ void d_axpy_diag(T *__restrict__ x, const T *__restrict__ dinv, const T *__restrict__ t, int64_t n, int bid_, int nb_) {
  for (int64_t i = (int64_t)bid_ * blockDim.x + threadIdx.x; i < n; i += (int64_t)nb_ * blockDim.x)
    x[i] -= dinv[i] * t[i];
}
template <typename T>
struct KAxpyDiag {
  static constexpr int kMaxThreads = kThreads;
  struct Args {
    T *x;
    const T *dinv;
    const T *t;
    int64_t n;
  };
  static __device__ __forceinline__ void run(const Args &a, int bid, int nb) {
    d_axpy_diag<T>(a.x, a.dinv, a.t, a.n, bid, nb);
  }
};

template <typename T>
__device__ __forceinline__ void d_axpy(T *__restrict__ y, const T *__restrict__ x, T a, int64_t n, int bid_, int nb_) {
  for (int64_t i = (int64_t)bid_ * blockDim.x + threadIdx.x; i < n; i += (int64_t)nb_ * blockDim.x)
    y[i] += a * x[i];
}
template <typename T>
struct KAxpy {
  static constexpr int kMaxThreads = kThreads;
  struct Args {
    T *y;
    const T *x;
    T a;
    int64_t n;
  };
  static __device__ __forceinline__ void run(const Args &a, int bid, int nb) {
    d_axpy<T>(a.y, a.x, a.a, a.n, bid, nb);
  }
};

template <typename TI, typename TO>
__device__ __forceinline__ void d_convert(const TI *__restrict__ in, TO *__restrict__ out, int64_t n, int bid_, int nb_) {
  for (int64_t i = (int64_t)bid_ * blockDim.x + threadIdx.x; i < n; i += (int64_t)nb_ * blockDim.x)
    out[i] = (TO)in[i];
}
template <typename TI, typename TO>
struct KConvert {
  static constexpr int kMaxThreads = kThreads;
  struct Args {
    const TI *in;
    TO *out;
    int64_t n;
  };
  static __device__ __forceinline__ void run(const Args &a, int bid, int nb) {
    d_convert<TI, TO>(a.in, a.out, a.n, bid, nb);
  }
};

__global__ void k_sell_widths(const int32_t *__restrict__ rp, int64_t nbr, int32_t *__restrict__ rl,
                              int32_t *__restrict__ w) {
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int len = I < nbr ? rp[I + 1] - rp[I] : 0;
  if (I < nbr) rl[I] = len;
  int m = len;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0 && (I >> 5) * 32 < nbr) w[I >> 5] = m;
}

// one thread per block row: slot t of row I goes to slice I/32, lane I%32
__global__ void k_sell_fill(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int nsrc,
                            const double *__restrict__ v0, const double *__restrict__ v1,
                            const double *__restrict__ v2, int b0, int b1, int b2, int br, int64_t nbr,
                            const int32_t *__restrict__ sp, int32_t *__restrict__ col, double *__restrict__ v64,
                            float *__restrict__ v32) {
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nbr) return;
  const int64_t lane = I & 31, base = sp[I >> 5];
  const int bct = b0 + b1 + b2, bs = br * bct;
  for (int64_t a = rp[I]; a < rp[I + 1]; ++a) {
    const int64_t slot = base + (a - rp[I]);
    col[slot * 32 + lane] = ci[a];
    for (int r = 0; r < br; ++r) {
      int o = 0;
      for (int j = 0; j < nsrc; ++j) {
        const double *v = j == 0 ? v0 : (j == 1 ? v1 : v2);
        const int bj = j == 0 ? b0 : (j == 1 ? b1 : b2);
        for (int q = 0; q < bj; ++q) {
          const double x = v[(a * br + r) * bj + q];
          const int64_t e = (slot * bs + r * bct + o + q) * 32 + lane;
          if (v64) v64[e] = x;
          if (v32) v32[e] = (float)x;
        }
        o += bj;
      }
    }
  }
}

__device__ __forceinline__ void d_scale(const double *x, double a, double *y, int64_t n, int bid_, int nb_) {
  for (int64_t i = (int64_t)bid_ * blockDim.x + threadIdx.x; i < n; i += (int64_t)nb_ * blockDim.x)
    y[i] = a * x[i];
}
struct KScale {
  static constexpr int kMaxThreads = kThreads;
  struct Args {
    const double *x;
    double a;
    double *y;
    int64_t n;
  };
  static __device__ __forceinline__ void run(const Args &a, int bid, int nb) {
    d_scale(a.x, a.a, a.y, a.n, bid, nb);
  }
};

// v = a v (in place) and out = v converted to TO: the normalisation of a new
// Krylov vector fused with the copy the preconditioner reads
template <typename TO>
__device__ __forceinline__ void d_scale_convert(double *__restrict__ v, double a, TO *__restrict__ out, int64_t n,
                                                int bid_, int nb_) {
  for (int64_t i = (int64_t)bid_ * blockDim.x + threadIdx.x; i < n; i += (int64_t)nb_ * blockDim.x) {
    const double t = a * v[i];
    v[i] = t;
    out[i] = (TO)t;
  }
}
template <typename TO>
struct KScaleConvert {
  static constexpr int kMaxThreads = kThreads;
  struct Args {
    double *v;
    double a;
    TO *out;
    int64_t n;
  };
  static __device__ __forceinline__ void run(const Args &a, int bid, int nb) {
    d_scale_convert<TO>(a.v, a.a, a.out, a.n, bid, nb);
  }
};

// the same with a = 1 / sqrt(nrm2[0]) read from device memory (the norm of
// the previous Arnoldi vector, so that a captured iteration graph normalises
// its input itself); out may be null (in-place scaling only)
template <typename TO>
__device__ __forceinline__ void d_scale_convert_dev(double *__restrict__ v, const double *__restrict__ nrm2,
                                                    TO *__restrict__ out, int64_t n, int bid_, int nb_) {
  const double a = 1.0 / sqrt(nrm2[0]);
  for (int64_t i = (int64_t)bid_ * blockDim.x + threadIdx.x; i < n; i += (int64_t)nb_ * blockDim.x) {
    const double t = a * v[i];
    v[i] = t;
    if (out) out[i] = (TO)t;
  }
}
template <typename TO>
struct KScaleConvertDev {
  static constexpr int kMaxThreads = kThreads;
  struct Args {
    double *v;
    const double *nrm2;
    TO *out;
    int64_t n;
  };
  static __device__ __forceinline__ void run(const Args &a, int bid, int nb) {
    d_scale_convert_dev<TO>(a.v, a.nrm2, a.out, a.n, bid, nb);
  }
};

__device__ __forceinline__ double block_sum(double v, double *sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

constexpr int kTile = kThreads;  // rows of w staged per step
constexpr int kMaxQ = 64;        // rows of V handled per launch (8 per warp)

// partial[q*nblk + b] = sum over chunk b of V_q[i] * ws[i] for the staged tile;
// warp p owns rows q = p, p+8, ... and reads them coalesced.
__device__ __forceinline__ void tile_dots(const double *__restrict__ V, int64_t ldv, int k, int64_t t0, int cnt,
                                          const double *ws, double (&acc)[kMaxQ / 8]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int m = 0; m < kMaxQ / 8; ++m) {
    const int q = warp + 8 * m;
    if (q < k) {
      const double *vq = V + (int64_t)q * ldv + t0;
      double s = acc[m];  // one FMA chain per row across the tiles (no extra add per tile)
      for (int t = lane; t < cnt; t += 32) s = fma(vq[t], ws[t], s);
      acc[m] = s;
    }
  }
}

__device__ __forceinline__ void store_dots(int k, int nblk, double (&acc)[kMaxQ / 8], double *__restrict__ partial,
                                           int bid) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int m = 0; m < kMaxQ / 8; ++m) {
    const int q = warp + 8 * m;
    if (q < k) {
      double v = acc[m];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) partial[(int64_t)q * nblk + bid] = v;
    }
  }
}

// h_q = V_q . w for q < k (w may be one of the rows of V)
__device__ __forceinline__ void d_mdot(const double *__restrict__ V, int64_t ldv, int k, const double *__restrict__ w, int64_t n,
       double *__restrict__ partial, int nblk, int bid_, int nb_) {
  __shared__ double ws[kTile];
  const int64_t chunk = (n + nblk - 1) / nblk;
  const int64_t lo = (int64_t)bid_ * chunk;
  const int64_t hi = min(n, lo + chunk);
  double acc[kMaxQ / 8];
#pragma unroll
  for (int m = 0; m < kMaxQ / 8; ++m) acc[m] = 0.0;
  for (int64_t t0 = lo; t0 < hi; t0 += kTile) {
    const int cnt = (int)min((int64_t)kTile, hi - t0);
    ws[threadIdx.x] = threadIdx.x < cnt ? w[t0 + threadIdx.x] : 0.0;
    __syncthreads();
    tile_dots(V, ldv, k, t0, cnt, ws, acc);
    __syncthreads();
  }
  store_dots(k, nblk, acc, partial, bid_);
}
struct KMdot {
  static constexpr int kMaxThreads = kThreads;
  struct Args {
    const double *V;
    int64_t ldv;
    int k;
    const double *w;
    int64_t n;
    double *partial;
    int nblk;
  };
  static __device__ __forceinline__ void run(const Args &a, int bid, int nb) {
    d_mdot(a.V, a.ldv, a.k, a.w, a.n, a.partial, a.nblk, bid, nb);
  }
};

// w <- w - sum_q V_q h_q, then partial dots V_q . w_new (CGS2 second pass)
__device__ __forceinline__ void d_cgs_fused(const double *__restrict__ V, int64_t ldv, int k, const double *__restrict__ h, double *__restrict__ w,
            int64_t n, double *__restrict__ partial, int nblk, int bid_, int nb_) {
  __shared__ double ws[kTile];
  __shared__ double hs[kMaxQ];
  for (int q = threadIdx.x; q < k; q += blockDim.x) hs[q] = h[q];
  __syncthreads();
  const int64_t chunk = (n + nblk - 1) / nblk;
  const int64_t lo = (int64_t)bid_ * chunk;
  const int64_t hi = min(n, lo + chunk);
  double acc[kMaxQ / 8];
#pragma unroll
  for (int m = 0; m < kMaxQ / 8; ++m) acc[m] = 0.0;
  for (int64_t t0 = lo; t0 < hi; t0 += kTile) {
    const int cnt = (int)min((int64_t)kTile, hi - t0);
    double wn = 0.0;
    if (threadIdx.x < cnt) {
      const int64_t i = t0 + threadIdx.x;
      double s = 0.0;  // (a chain started from w_i would wait for its load)
      for (int q = 0; q < k; ++q) s += V[(int64_t)q * ldv + i] * hs[q];
      wn = w[i] - s;
      w[i] = wn;
    }
    ws[threadIdx.x] = wn;
    __syncthreads();
    tile_dots(V, ldv, k, t0, cnt, ws, acc);
    __syncthreads();
  }
  store_dots(k, nblk, acc, partial, bid_);
}
struct KCgsFused {
  static constexpr int kMaxThreads = kThreads;
  struct Args {
    const double *V;
    int64_t ldv;
    int k;
    const double *h;
    double *w;
    int64_t n;
    double *partial;
    int nblk;
  };
  static __device__ __forceinline__ void run(const Args &a, int bid, int nb) {
    d_cgs_fused(a.V, a.ldv, a.k, a.h, a.w, a.n, a.partial, a.nblk, bid, nb);
  }
};

__device__ __forceinline__ void d_reduce_partials(const double *__restrict__ partial, int k, int nblk, double *__restrict__ out, int bid_, int nb_) {
  __shared__ double sh[32];
  if (bid_ >= k) return;
  const double *p = partial + (int64_t)bid_ * nblk;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += p[i];
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) out[bid_] = s;
}
struct KReducePartials {
  static constexpr int kMaxThreads = kThreads;
  struct Args {
    const double *partial;
    int k;
    int nblk;
    double *out;
  };
  static __device__ __forceinline__ void run(const Args &a, int bid, int nb) {
    d_reduce_partials(a.partial, a.k, a.nblk, a.out, bid, nb);
  }
};

__device__ __forceinline__ void d_cgs_update(const double *__restrict__ V, int64_t ldv, int k, const double *__restrict__ h,
             double *__restrict__ w, int64_t n, double *__restrict__ partial, int nblk, int bid_, int nb_) {
  __shared__ double hs[64];
  __shared__ double sh[32];
  for (int q = threadIdx.x; q < k; q += blockDim.x) hs[q] = h[q];
  __syncthreads();
  const int64_t chunk = (n + nblk - 1) / nblk;
  const int64_t lo = (int64_t)bid_ * chunk;
  const int64_t hi = min(n, lo + chunk);
  double nrm = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    double s = 0.0;  // (a chain started from w_i would wait for its load)
    for (int q = 0; q < k; ++q) s += V[(int64_t)q * ldv + i] * hs[q];
    const double wn = w[i] - s;
    w[i] = wn;
    nrm += wn * wn;
  }
  if (partial != nullptr) {
    const double t = block_sum(nrm, sh);
    if (threadIdx.x == 0) partial[bid_] = t;
  }
}
struct KCgsUpdate {
  static constexpr int kMaxThreads = kThreads;
  struct Args {
    const double *V;
    int64_t ldv;
    int k;
    const double *h;
    double *w;
    int64_t n;
    double *partial;
    int nblk;
  };
  static __device__ __forceinline__ void run(const Args &a, int bid, int nb) {
    d_cgs_update(a.V, a.ldv, a.k, a.h, a.w, a.n, a.partial, a.nblk, bid, nb);
  }
};

__device__ __forceinline__ void d_gemv_add(const double *__restrict__ Z, int64_t ldz, int k, const double *__restrict__ y,
                           double *__restrict__ x, int64_t n, int bid_, int nb_) {
  __shared__ double ys[64];
  for (int q = threadIdx.x; q < k; q += blockDim.x) ys[q] = y[q];
  __syncthreads();
  for (int64_t i = (int64_t)bid_ * blockDim.x + threadIdx.x; i < n; i += (int64_t)nb_ * blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < k; ++q) s += Z[(int64_t)q * ldz + i] * ys[q];
    x[i] += s;
  }
}
struct KGemvAdd {
  static constexpr int kMaxThreads = kThreads;
  struct Args {
    const double *Z;
    int64_t ldz;
    int k;
    const double *y;
    double *x;
    int64_t n;
  };
  static __device__ __forceinline__ void run(const Args &a, int bid, int nb) {
    d_gemv_add(a.Z, a.ldz, a.k, a.y, a.x, a.n, bid, nb);
  }
};

// The tail of a single-field V-cycle (Algorithm 1 on the level above the
// coarsest and the coarse solve) in ONE CTA, for levels small enough that
// their vectors live in shared memory: Chebyshev / Jacobi pre-smoothing from
// zero, residual, restriction, the coarsest solve through the explicit
// inverse, prolongation and post-smoothing, separated by __syncthreads
// instead of kernel boundaries.  Every step reduces a row exactly as the
// separate launches do (one warp per block row, lanes striding over the
// row's blocks, the same xor butterfly; the inverse applied in float64), so
// the result is the one of the step-by-step V-cycle bit for bit.
constexpr int kTailThreads = 1024;
constexpr int kTailMaxSteps = 8;

template <typename T> struct TailArgs {
  int64_t n, nbr, nc, ncbr;  // level dofs / block rows; coarse dofs / block rows
  const int32_t *arp, *acol;
  const T *aval, *dinv;
  const int32_t *rrp, *rcol;
  const T *rval;  // R: ncbr block rows of BC x BR blocks
  const int32_t *prp, *pcol;
  const T *pval;  // P: nbr block rows of BR x BC blocks
  const double *inv;  // nc x nc row-major inverse of the coarsest matrix
  const T *b;
  T *x;
  int ns;  // smoothing steps per application
  T c1[kTailMaxSteps], c2[kTailMaxSteps];
};

// row sums of a plain-BSR block row against x in shared memory (the
// arithmetic of bsr_warp_row)
template <int BR, int BC, typename T>
__device__ __forceinline__ void tail_row(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                         const T *__restrict__ val, const T *x, int64_t row, int lane,
                                         T (&acc)[BR]) {
  const int lo = rp[row], hi = rp[row + 1];
#pragma unroll
  for (int r = 0; r < BR; ++r) acc[r] = T(0);
  for (int k = lo + lane; k < hi; k += 32) {
    const int64_t c = __ldg(col + k);
    T xv[BC];
#pragma unroll
    for (int q = 0; q < BC; ++q) xv[q] = x[c * BC + q];
    T blk[BR * BC];
    ldg_block<BR * BC, T>(val + (int64_t)k * (BR * BC), blk);
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int q = 0; q < BC; ++q) acc[r] += blk[r * BC + q] * xv[q];
  }
#pragma unroll
  for (int r = 0; r < BR; ++r)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
}

// one smoothing step in shared memory: xo = x + d, d = c1 d + c2 dinv (b - A x)
template <int BR, typename T>
__device__ __forceinline__ void tail_smooth(const TailArgs<T> &a, const T *b, const T *x, T *xo, T *d, T c1, T c2) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t row = warp; row < a.nbr; row += kTailThreads / 32) {
    T acc[BR];
    tail_row<BR, BR, T>(a.arp, a.acol, a.aval, x, row, lane, acc);
    if (lane < BR) {
      const int64_t i = row * BR + lane;
      const T res = b[i] - pick<BR, T>(acc, lane);
      const T dd = c1 * d[i] + c2 * a.dinv[i] * res;
      d[i] = dd;
      xo[i] = x[i] + dd;
    }
  }
  __syncthreads();
}

template <int BR, int BC, typename T>
__device__ __forceinline__ void d_vcycle_tail(const TailArgs<T> &a) {
  extern __shared__ __align__(16) unsigned char tail_smem[];
  double *bc = reinterpret_cast<double *>(tail_smem);  // coarse right-hand side (float64 copy)
  T *xc = reinterpret_cast<T *>(bc + a.nc);
  T *bcT = xc + a.nc;
  T *b = bcT + a.nc;
  T *x0 = b + a.n;
  T *x1 = x0 + a.n;
  T *d = x1 + a.n;
  T *r = d + a.n;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int64_t i = tid; i < a.n; i += kTailThreads) b[i] = a.b[i];
  __syncthreads();
  // pre-smoothing from zero: the first step d = x = c2 dinv b, then steps
  for (int64_t i = tid; i < a.n; i += kTailThreads) {
    const T dd = a.c2[0] * a.dinv[i] * b[i];
    d[i] = dd;
    x0[i] = dd;
  }
  __syncthreads();
  T *cur = x0, *oth = x1;
  for (int k = 1; k < a.ns; ++k) {
    tail_smooth<BR, T>(a, b, cur, oth, d, a.c1[k], a.c2[k]);
    T *t = cur;
    cur = oth;
    oth = t;
  }
  // residual r = b - A x  (as y = -1 * A x + 1 * b)
  for (int64_t row = warp; row < a.nbr; row += kTailThreads / 32) {
    T acc[BR];
    tail_row<BR, BR, T>(a.arp, a.acol, a.aval, cur, row, lane, acc);
    if (lane < BR) {
      const int64_t i = row * BR + lane;
      r[i] = T(-1) * pick<BR, T>(acc, lane) + T(1) * b[i];
    }
  }
  __syncthreads();
  // restriction bc = R r
  for (int64_t row = warp; row < a.ncbr; row += kTailThreads / 32) {
    T acc[BC];
    tail_row<BC, BR, T>(a.rrp, a.rcol, a.rval, r, row, lane, acc);
    if (lane < BC) bcT[row * BC + lane] = T(1) * pick<BC, T>(acc, lane);
  }
  __syncthreads();
  // coarsest solve through the explicit inverse, in float64
  for (int64_t j = tid; j < a.nc; j += kTailThreads) bc[j] = (double)bcT[j];
  __syncthreads();
  for (int64_t row = warp; row < a.nc; row += kTailThreads / 32) {
    const double *ar = a.inv + row * a.nc;
    double acc = 0.0;
    for (int64_t j = lane; j < a.nc; j += 32) acc += __ldg(ar + j) * bc[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) xc[row] = (T)acc;
  }
  __syncthreads();
  // prolongation x += P xc  (as y = 1 * P xc + 1 * x)
  for (int64_t row = warp; row < a.nbr; row += kTailThreads / 32) {
    T acc[BR];
    tail_row<BR, BC, T>(a.prp, a.pcol, a.pval, xc, row, lane, acc);
    if (lane < BR) {
      const int64_t i = row * BR + lane;
      cur[i] = T(1) * pick<BR, T>(acc, lane) + T(1) * cur[i];
    }
  }
  __syncthreads();
  // post-smoothing from the corrected x
  for (int k = 0; k < a.ns; ++k) {
    tail_smooth<BR, T>(a, b, cur, oth, d, a.c1[k], a.c2[k]);
    T *t = cur;
    cur = oth;
    oth = t;
  }
  for (int64_t i = tid; i < a.n; i += kTailThreads) a.x[i] = cur[i];
}
template <int BR, int BC, typename T>
struct KVcycleTail {
  static constexpr int kMaxThreads = kTailThreads;
  using Args = TailArgs<T>;
  static __device__ __forceinline__ void run(const Args &a, int, int) { d_vcycle_tail<BR, BC, T>(a); }
};

inline unsigned ew_grid(int64_t n) {
  int64_t g = (n + kThreads - 1) / kThreads;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g > 0 ? g : 1);
}

// FP64 FMA throughput probe: C independent chains a = a * m + c per thread;
// the sum is stored only when it equals a value it cannot take (m, c are
// runtime values), so no chain can be dropped by the compiler.
__device__ double g_fp64_sink;
template <int C>
__global__ void __launch_bounds__(1024) k_fp64_rate(int iters, double m, double c) {
  double a[C];
#pragma unroll
  for (int k = 0; k < C; ++k) a[k] = 1e-3 * threadIdx.x + k;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int k = 0; k < C; ++k) a[k] = fma(a[k], m, c);
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < C; ++k) s += a[k];
  if (s == -12345.678) g_fp64_sink = s;
}

}  // namespace

// best rate over a few launch shapes (chains per thread, CTA size, CTAs per
// SM): the highest FMA throughput the part delivers, not one shape's
double fp64_rate(cudaStream_t s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return -1.0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1.0;
  struct Shape {
    int chains, threads, per_sm;
  };
  const Shape shapes[] = {{8, 256, 8}, {16, 256, 8}, {16, 512, 4}, {32, 256, 4}, {8, 1024, 2}};
  double best = 0.0;
  bool ok = true;
  for (const Shape &sh : shapes) {
    const int ctas = sms * sh.per_sm, iters = 65536 / sh.chains;
    for (int r = 0; r < 4 && ok; ++r) {
      ok = cudaEventRecord(e0, s) == cudaSuccess;
      if (sh.chains == 8) k_fp64_rate<8><<<ctas, sh.threads, 0, s>>>(iters, 0.999999, 1e-7);
      else if (sh.chains == 16) k_fp64_rate<16><<<ctas, sh.threads, 0, s>>>(iters, 0.999999, 1e-7);
      else k_fp64_rate<32><<<ctas, sh.threads, 0, s>>>(iters, 0.999999, 1e-7);
      ok = ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
      float ms = 0.f;
      ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
      const double flops = 2.0 * sh.chains * (double)iters * sh.threads * ctas;
      if (ok && r > 0 && ms > 0.f) best = std::max(best, flops / (ms * 1e-3) / 1e12);  // r = 0 warms up
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok || cudaGetLastError() != cudaSuccess) return -1.0;
  return best;
}

#define MFS_BLOCK_DISPATCH(BRV, BCV, CALL)                                      \
  switch (BRV * 16 + BCV) {                                                     \
    case 1 * 16 + 1: { constexpr int BR_ = 1, BC_ = 1; CALL; } break;           \
    case 1 * 16 + 2: { constexpr int BR_ = 1, BC_ = 2; CALL; } break;           \
    case 1 * 16 + 3: { constexpr int BR_ = 1, BC_ = 3; CALL; } break;           \
    case 1 * 16 + 6: { constexpr int BR_ = 1, BC_ = 6; CALL; } break;           \
    case 2 * 16 + 1: { constexpr int BR_ = 2, BC_ = 1; CALL; } break;           \
    case 2 * 16 + 2: { constexpr int BR_ = 2, BC_ = 2; CALL; } break;           \
    case 2 * 16 + 3: { constexpr int BR_ = 2, BC_ = 3; CALL; } break;           \
    case 2 * 16 + 6: { constexpr int BR_ = 2, BC_ = 6; CALL; } break;           \
    case 3 * 16 + 1: { constexpr int BR_ = 3, BC_ = 1; CALL; } break;           \
    case 3 * 16 + 2: { constexpr int BR_ = 3, BC_ = 2; CALL; } break;           \
    case 3 * 16 + 3: { constexpr int BR_ = 3, BC_ = 3; CALL; } break;           \
    case 3 * 16 + 6: { constexpr int BR_ = 3, BC_ = 6; CALL; } break;           \
    case 6 * 16 + 1: { constexpr int BR_ = 6, BC_ = 1; CALL; } break;           \
    case 6 * 16 + 2: { constexpr int BR_ = 6, BC_ = 2; CALL; } break;           \
    case 6 * 16 + 3: { constexpr int BR_ = 6, BC_ = 3; CALL; } break;           \
    case 6 * 16 + 6: { constexpr int BR_ = 6, BC_ = 6; CALL; } break;           \
    default: fprintf(stderr, "mfs: unsupported block shape %dx%d\n", BRV, BCV); \
  }

void set_launch_hook(LaunchHook *h) { g_hook = h; }
void set_recorder(Recorder *r) { g_rec = r; }
void set_pdl(unsigned max_grid) {
  g_pdl = max_grid;
  g_pdl_prev = nullptr;
}
void pdl_break() { g_pdl_prev = nullptr; }

HookBypass::HookBypass() { ++g_hook_off; }
HookBypass::~HookBypass() { --g_hook_off; }

void init() {
  // once per device and process (concurrent setups must not race on it)
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return;
  cudaFuncSetAttribute(k_solo<KLuSolve<float>>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_solo<KLuSolve<double>>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_multi<KLuSolve<float>>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_multi<KLuSolve<double>>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  done[dev] = true;
}

template <typename T>
void spmv(const Sell &A, const T *x, T *y, T alpha, T beta, const T *z, cudaStream_t s) {
  if (A.nbr == 0) return;
  const T *v = vals<T>(A);
  const bool cta = A.kind == 1 && A.nbr <= kCtaRowsMax && A.nnzb >= kCtaRowBlocks * A.nbr;
  HookScope hs(s, K_SPMV, matrix_bytes<T>(A) + (double)sizeof(T) * (A.ncols() + A.nrows() * (z ? 2 : 1)),
               cta ? 7000 + sparse_sig<T>(A) % 1000 : sparse_sig<T>(A), A.nbr,
               2.0 * A.nnzb * A.br * A.bc + (z ? 3.0 : 1.0) * A.nrows());
  if (A.kind == 1) {
    if (cta) {
      MFS_BLOCK_DISPATCH(A.br, A.bc,
                         (go<KSpmvCta<BR_, BC_, T>>((unsigned)A.nbr, kThreads, 0, s, {
                             A.nbr, A.sp, A.col, v, x, y, alpha, beta, z})));
    } else {
      MFS_BLOCK_DISPATCH(A.br, A.bc,
                         (go<KSpmvWarp<BR_, BC_, T>>(grid_for(A.nbr * 32), kThreads, 0, s, {
                             A.nbr, A.sp, A.col, v, x, y, alpha, beta, z})));
    }
    return;
  }
  if (A.unroll == 4) {
    MFS_BLOCK_DISPATCH(A.br, A.bc,
                       (go<KSpmvSell<BR_, BC_, T, 4>>(grid_for(A.nbr, kSellThreads), kSellThreads, 0, s, {
                           A.nbr, A.sp, A.rl, A.col, v, x, y, alpha, beta, z})));
  } else if (A.unroll == 8) {
    MFS_BLOCK_DISPATCH(A.br, A.bc,
                       (go<KSpmvSell<BR_, BC_, T, 8>>(grid_for(A.nbr, kSellThreads), kSellThreads, 0, s, {
                           A.nbr, A.sp, A.rl, A.col, v, x, y, alpha, beta, z})));
  } else {
    MFS_BLOCK_DISPATCH(A.br, A.bc,
                       (go<KSpmvSell<BR_, BC_, T, 2>>(grid_for(A.nbr, kSellThreads), kSellThreads, 0, s, {
                           A.nbr, A.sp, A.rl, A.col, v, x, y, alpha, beta, z})));
  }
}

#define MFS_SQUARE_DISPATCH(BRV, CALL)                                  \
  switch (BRV) {                                                        \
    case 1: { constexpr int BR_ = 1; CALL; } break;                     \
    case 2: { constexpr int BR_ = 2; CALL; } break;                     \
    case 3: { constexpr int BR_ = 3; CALL; } break;                     \
    case 6: { constexpr int BR_ = 6; CALL; } break;                     \
    default: fprintf(stderr, "mfs: unsupported block size %d\n", BRV); \
  }

#define MFS_ROWS_DISPATCH(BR, B, CALL)                                          \
  switch (BR * 1000 + B[0] * 100 + B[1] * 10 + B[2]) {                          \
    case 3311: { constexpr int R_ = 3, X0 = 3, X1 = 1, X2 = 1; CALL; } break;   \
    case 1311: { constexpr int R_ = 1, X0 = 3, X1 = 1, X2 = 1; CALL; } break;   \
    case 3310: { constexpr int R_ = 3, X0 = 3, X1 = 1, X2 = 0; CALL; } break;   \
    case 1310: { constexpr int R_ = 1, X0 = 3, X1 = 1, X2 = 0; CALL; } break;   \
    case 2210: { constexpr int R_ = 2, X0 = 2, X1 = 1, X2 = 0; CALL; } break;   \
    case 1210: { constexpr int R_ = 1, X0 = 2, X1 = 1, X2 = 0; CALL; } break;   \
    default: break;                                                             \
  }

bool rows_supported(int br, const int *b, int nb) {
  const int code = br * 1000 + b[0] * 100 + b[1] * 10 + (nb > 2 ? b[2] : 0);
  switch (code) {
    case 3311: case 1311: case 3310: case 1310: case 2210: case 1210: return nb >= 2 && nb <= 3;
    default: return false;
  }
}

void spmv_rows(const RowMerged &R, const double *x, double *y, cudaStream_t s) {
  const Sell &A = R.M;
  if (A.nbr == 0) return;
  HookScope hs(s, K_SPMV,
               (double)A.nnzb * (A.br * A.bc * 8.0 + 4.0) + 4.0 * A.nbr + 8.0 * (A.nbc * A.bc + A.nrows()),
               2000 + A.br * 100 + A.bc * 10 + 1, A.nbr, 2.0 * A.nnzb * A.br * A.bc);
  const double *x0 = x + R.off[0], *x1 = x + R.off[1], *x2 = R.nb > 2 ? x + R.off[2] : x;
  const int b3[3] = {R.b[0], R.b[1], R.nb > 2 ? R.b[2] : 0};
  const unsigned grid = (unsigned)A.nslices;  // H > 1: one slice per CTA
  if (R.split == 4) {
    MFS_ROWS_DISPATCH(A.br, b3, (go<KSpmvRows<R_, X0, X1, X2, 4>>(grid, 128, 0, s, {
                                    A.nbr, A.sp, A.rl, A.col, A.v64, x0, x1, x2, y})));
  } else if (R.split == 2) {
    MFS_ROWS_DISPATCH(A.br, b3, (go<KSpmvRows<R_, X0, X1, X2, 2>>(grid, 64, 0, s, {
                                    A.nbr, A.sp, A.rl, A.col, A.v64, x0, x1, x2, y})));
  } else {
    MFS_ROWS_DISPATCH(A.br, b3, (go<KSpmvRows<R_, X0, X1, X2, 1>>(grid_for(A.nbr, 64), 64, 0, s, {
                                    A.nbr, A.sp, A.rl, A.col, A.v64, x0, x1, x2, y})));
  }
}

template <typename T>
void smooth_step(const Sell &A, const T *dinv, const T *b, const T *x, T *xout, T *d, T c1, T c2,
                 cudaStream_t s) {
  if (A.nbr == 0) return;
  const T *v = vals<T>(A);
  HookScope hs(s, K_SMOOTH, matrix_bytes<T>(A) + (double)sizeof(T) * (A.ncols() + 5.0 * A.nrows()),
               sparse_sig<T>(A), A.nbr, 2.0 * A.nnzb * A.br * A.bc + 6.0 * A.nrows());
  if (A.kind == 1) {
    MFS_SQUARE_DISPATCH(A.br, (go<KSmoothWarp<BR_, T>>(grid_for(A.nbr * 32), kThreads, 0, s, {
                                  A.nbr, A.sp, A.col, v, dinv, b, x, xout, d, c1, c2})));
    return;
  }
  if (A.unroll == 4) {
    MFS_SQUARE_DISPATCH(A.br, (go<KSmoothSell<BR_, T, 4>>(grid_for(A.nbr, kSellThreads), kSellThreads, 0, s, {
                                  A.nbr, A.sp, A.rl, A.col, v, dinv, b, x, xout, d, c1, c2})));
  } else if (A.unroll == 8) {
    MFS_SQUARE_DISPATCH(A.br, (go<KSmoothSell<BR_, T, 8>>(grid_for(A.nbr, kSellThreads), kSellThreads, 0, s, {
                                  A.nbr, A.sp, A.rl, A.col, v, dinv, b, x, xout, d, c1, c2})));
  } else {
    MFS_SQUARE_DISPATCH(A.br, (go<KSmoothSell<BR_, T, 2>>(grid_for(A.nbr, kSellThreads), kSellThreads, 0, s, {
                                  A.nbr, A.sp, A.rl, A.col, v, dinv, b, x, xout, d, c1, c2})));
  }
}

template <typename T>
void smooth_first(int64_t n, const T *dinv, const T *b, T *x, T *d, T c2, cudaStream_t s) {
  if (n == 0) return;
  HookScope hs(s, K_VECTOR, 4.0 * n * sizeof(T), 1, n, 2.0 * n);
  go<KSmoothFirst<T>>(ew_grid(n), kThreads, 0, s, {n, dinv, b, x, d, c2});
}

#define MFS_GS_G_DISPATCH(GV, CALL)                              \
  switch (GV) {                                                  \
    case 4: { constexpr int G_ = 4; CALL; } break;               \
    case 8: { constexpr int G_ = 8; CALL; } break;               \
    case 16: { constexpr int G_ = 16; CALL; } break;             \
    default: { constexpr int G_ = 32; CALL; } break;             \
  }

template <typename T>
void gs_sweeps(const GsLevel &g, const T *dblk, const T *b, T *x, T omega, int sweeps, bool backward,
               cudaStream_t s) {
  const Sell &A = g.M;
  if (A.nbr == 0) return;
  const T *v = vals<T>(A);
  const int bw = backward ? 1 : 0;
  const int sig = (A.kind == 1 ? 5 : 4) * 1000 + sparse_sig<T>(A) % 1000;
  if (!g.small) {
    const int nc = g.ncolors();
    for (int sw = 0; sw < sweeps; ++sw)
      for (int q = 0; q < nc; ++q) {
        const int c = backward ? nc - 1 - q : q;
        const int64_t r0 = g.hoff[c], r1 = g.hoff[c + 1], nr = r1 - r0;
        // this colour's blocks + gathered x + diagonal blocks + b and x of its rows
        HookScope hs(s, K_SMOOTH,
                     (double)g.cnnzb[c] * (A.br * A.bc * sizeof(T) + sizeof(int32_t)) +
                         (double)sizeof(T) * (g.cnnzb[c] * A.bc + (A.br + 2.0) * A.br * nr) + 8.0 * nr,
                     sig, nr, 2.0 * g.cnnzb[c] * A.br * A.bc + 2.0 * A.br * A.br * nr);
        MFS_GS_G_DISPATCH(g.G, MFS_SQUARE_DISPATCH(A.br, (go<KGsColor<BR_, T, G_>>(grid_for(nr * G_), kThreads, 0, s, {
                                                             r0, r1, A.sp, A.col, v, g.rowidx, dblk, b, x, omega, bw}))));
      }
    return;
  }
  HookScope hs(s, K_SMOOTH,
               sweeps * (matrix_bytes<T>(A) + (double)sizeof(T) * ((A.br + 2.0) * A.nrows())) +
                   2.0 * sizeof(T) * A.nrows(),
               sig, A.nbr, sweeps * (2.0 * A.nnzb * A.br * A.bc + 2.0 * A.br * A.nrows()));
  const int nc = g.ncolors();
  const size_t shm = (size_t)A.nrows() * sizeof(T);
  MFS_GS_G_DISPATCH(g.G, MFS_SQUARE_DISPATCH(A.br, (go<KGsSmall<BR_, T, G_>>(1, kGsCtaThreads, shm, s, {
                                                       nc, A.nbr, g.coff, A.sp, A.col, v, g.rowidx, dblk, b, x,
                                                       omega, sweeps, bw}))));
}

template <typename T>
void lu_solve(const DenseLU &lu, const T *b, T *x, cudaStream_t s) {
  if (lu.n == 0) return;
  if (lu.inv) {
    HookScope hs(s, K_COARSE, 8.0 * lu.n * (double)lu.n + 2.0 * sizeof(T) * lu.n, 2, lu.n, 2.0 * lu.n * (double)lu.n);
    constexpr int kRowsPerCta = kThreads / 32;
    go<KInvApply<T>>((unsigned)((lu.n + kRowsPerCta - 1) / kRowsPerCta), kThreads, (size_t)lu.n * sizeof(double), s, {
        lu.n, lu.inv, b, x});
    return;
  }
  HookScope hs(s, K_COARSE, 8.0 * lu.n * (double)lu.n + (4.0 + 2 * sizeof(T)) * lu.n, 1, lu.n,
               2.0 * lu.n * (double)lu.n);
  // stage the factors in shared memory when y and LU fit in 200 KB
  const int staged = (size_t)lu.n * (lu.n + 1) * sizeof(double) <= 200 * 1024 ? 1 : 0;
  const size_t smem = (size_t)lu.n * (staged ? lu.n + 1 : 1) * sizeof(double);
  const int threads = lu.n <= 64 ? 256 : 512;
  go<KLuSolve<T>>(1, threads, smem, s, {lu.n, lu.lu, lu.perm, b, x, staged});
}

size_t tail_smem_bytes(int64_t n, int64_t nc, size_t tsize) {
  return (size_t)nc * (sizeof(double) + 2 * tsize) + (size_t)n * 5 * tsize;
}

bool tail_supported(int br, int bc) { return br == bc && (br == 1 || br == 2 || br == 3 || br == 6); }

bool cta_rows(const Sell &A) { return A.kind == 1 && A.nbr <= kCtaRowsMax && A.nnzb >= kCtaRowBlocks * A.nbr; }

template <typename T>
void vcycle_tail(const Sell &A, const T *dinv, const Sell &R, const Sell &P, const DenseLU &lu, int ns,
                 const T *c1, const T *c2, const T *b, T *x, cudaStream_t s) {
  TailArgs<T> a{};
  a.n = A.nrows();
  a.nbr = A.nbr;
  a.nc = lu.n;
  a.ncbr = R.nbr;
  a.arp = A.sp;
  a.acol = A.col;
  a.aval = vals<T>(A);
  a.dinv = dinv;
  a.rrp = R.sp;
  a.rcol = R.col;
  a.rval = vals<T>(R);
  a.prp = P.sp;
  a.pcol = P.col;
  a.pval = vals<T>(P);
  a.inv = lu.inv;
  a.b = b;
  a.x = x;
  a.ns = ns;
  for (int k = 0; k < ns && k < kTailMaxSteps; ++k) {
    a.c1[k] = c1[k];
    a.c2[k] = c2[k];
  }
  const size_t smem = tail_smem_bytes(a.n, a.nc, sizeof(T));
  const double bytes = ns * 2.0 * matrix_bytes<T>(A) + matrix_bytes<T>(A) + matrix_bytes<T>(R) + matrix_bytes<T>(P) +
                       8.0 * lu.n * (double)lu.n + 2.0 * sizeof(T) * A.nrows();
  HookScope hs(s, K_COARSE, bytes, 3, A.nbr, 0.0);
  switch (A.br) {
    case 1: go<KVcycleTail<1, 1, T>>(1, kTailThreads, smem, s, a); break;
    case 2: go<KVcycleTail<2, 2, T>>(1, kTailThreads, smem, s, a); break;
    case 3: go<KVcycleTail<3, 3, T>>(1, kTailThreads, smem, s, a); break;
    case 6: go<KVcycleTail<6, 6, T>>(1, kTailThreads, smem, s, a); break;
    default: break;
  }
}
template void vcycle_tail<float>(const Sell &, const float *, const Sell &, const Sell &, const DenseLU &, int,
                                 const float *, const float *, const float *, float *, cudaStream_t);
template void vcycle_tail<double>(const Sell &, const double *, const Sell &, const Sell &, const DenseLU &, int,
                                  const double *, const double *, const double *, double *, cudaStream_t);

template <typename T>
void fill(T *x, int64_t n, T v, cudaStream_t s) {
  HookScope hs(s, K_VECTOR, (double)n * sizeof(T), 2, n, 0.0);
  if (n) go<KFill<T>>(ew_grid(n), kThreads, 0, s, {x, n, v});
}
template <typename T>
void axpy_diag(T *x, const T *dinv, const T *t, int64_t n, cudaStream_t s) {
  HookScope hs(s, K_VECTOR, 4.0 * n * sizeof(T), 3, n, 2.0 * n);
  if (n) go<KAxpyDiag<T>>(ew_grid(n), kThreads, 0, s, {x, dinv, t, n});
}
template <typename T>
void axpy(T *y, const T *x, T a, int64_t n, cudaStream_t s) {
  HookScope hs(s, K_VECTOR, 3.0 * n * sizeof(T), 4, n, 2.0 * n);
  if (n) go<KAxpy<T>>(ew_grid(n), kThreads, 0, s, {y, x, a, n});
}
void sell_widths(const int32_t *rp, int64_t nbr, int32_t *rl, int32_t *w, cudaStream_t s) {
  if (nbr) k_sell_widths<<<grid_for(nbr), kThreads, 0, s>>>(rp, nbr, rl, w);
}

void sell_fill(const int32_t *rp, const int32_t *ci, int nsrc, const double *v0, const double *v1,
               const double *v2, const int *bcs, int br, int64_t nbr, const int32_t *sp, int32_t *col,
               double *v64, float *v32, cudaStream_t s) {
  if (nbr)
    k_sell_fill<<<grid_for(nbr), kThreads, 0, s>>>(rp, ci, nsrc, v0, v1, v2, bcs[0], nsrc > 1 ? bcs[1] : 0,
                                                   nsrc > 2 ? bcs[2] : 0, br, nbr, sp, col, v64, v32);
}

template <typename TI, typename TO>
void convert(const TI *in, TO *out, int64_t n, cudaStream_t s) {
  HookScope hs(s, K_VECTOR, (double)n * (sizeof(TI) + sizeof(TO)), 5, n, 0.0);
  if (n) go<KConvert<TI, TO>>(ew_grid(n), kThreads, 0, s, {in, out, n});
}
template <typename TO>
void scale_convert(double *v, double a, TO *out, int64_t n, cudaStream_t s) {
  HookScope hs(s, K_VECTOR, (16.0 + sizeof(TO)) * n, 7, n, (double)n);
  if (n) go<KScaleConvert<TO>>(ew_grid(n), kThreads, 0, s, {v, a, out, n});
}
template void scale_convert<float>(double *, double, float *, int64_t, cudaStream_t);
template void scale_convert<double>(double *, double, double *, int64_t, cudaStream_t);
template <typename TO>
void scale_convert_dev(double *v, const double *nrm2, TO *out, int64_t n, cudaStream_t s) {
  HookScope hs(s, K_VECTOR, (16.0 + (out ? sizeof(TO) : 0)) * n, 8, n, (double)n);
  if (n) go<KScaleConvertDev<TO>>(ew_grid(n), kThreads, 0, s, {v, nrm2, out, n});
}
template void scale_convert_dev<float>(double *, const double *, float *, int64_t, cudaStream_t);
template void scale_convert_dev<double>(double *, const double *, double *, int64_t, cudaStream_t);

void scale(const double *x, double a, double *y, int64_t n, cudaStream_t s) {
  HookScope hs(s, K_VECTOR, 16.0 * n, 6, n, (double)n);
  if (n) go<KScale>(ew_grid(n), kThreads, 0, s, {x, a, y, n});
}

// CTAs of the CGS2 passes over a length-n basis: one per 2048 entries, up
// to four per SM; small systems (below 32 k entries) take up to 16, one
// staged tile of w (kTile entries) each at least, so that their passes do
// not loop over tiles in one or two CTAs.  (More CTAs for mid-size systems
// would help a system solved alone but slow down batches, whose merged
// launches fill the GPU already; the count is per system, so a batch and a
// solo solve reduce in the same order.)
int mdot_blocks(int64_t n) {
  int64_t b = n / 2048;
  b = std::max(b, std::min<int64_t>((n + kTile - 1) / kTile, 16));
  if (b < 1) b = 1;
  if (b > 152 * 4) b = 152 * 4;
  return (int)b;
}

void mdot(const double *V, int64_t ldv, int k, const double *w, int64_t n, double *partial, int nblk,
          cudaStream_t s) {
  HookScope hs(s, K_ARNOLDI, 8.0 * n * (k + 1), 1, n, 2.0 * n * k);
  go<KMdot>(nblk, kThreads, 0, s, {V, ldv, k, w, n, partial, nblk});
}

void reduce_partials(const double *partial, int k, int nblk, double *out, cudaStream_t s) {
  HookScope hs(s, K_ARNOLDI, 8.0 * (double)k * nblk, 2, k, (double)k * nblk);
  // recorded launches take a grid that does not depend on k (blocks >= k return)
  go<KReducePartials>(g_rec ? (unsigned)kMaxQ : (unsigned)k, kThreads, 0, s, {partial, k, nblk, out});
}

void cgs_fused(const double *V, int64_t ldv, int k, const double *h, double *w, int64_t n, double *partial,
               int nblk, cudaStream_t s) {
  HookScope hs(s, K_ARNOLDI, 8.0 * n * (k + 2), 3, n, 4.0 * n * k);
  go<KCgsFused>(nblk, kThreads, 0, s, {V, ldv, k, h, w, n, partial, nblk});
}

void cgs_update(const double *V, int64_t ldv, int k, const double *h, double *w, int64_t n,
                double *partial, int nblk, cudaStream_t s) {
  HookScope hs(s, K_ARNOLDI, 8.0 * n * (k + 2), 4, n, 2.0 * n * k + 2.0 * n);
  go<KCgsUpdate>(nblk, kThreads, 0, s, {V, ldv, k, h, w, n, partial, nblk});
}

void gemv_add(const double *Z, int64_t ldz, int k, const double *y, double *x, int64_t n, cudaStream_t s) {
  HookScope hs(s, K_ARNOLDI, 8.0 * n * (k + 2), 5, n, 2.0 * n * k);
  go<KGemvAdd>(ew_grid(n), kThreads, 0, s, {Z, ldz, k, y, x, n});
}

#define MFS_INST(T)                                                                                   \
  template void spmv<T>(const Sell &, const T *, T *, T, T, const T *, cudaStream_t);                 \
  template void smooth_step<T>(const Sell &, const T *, const T *, const T *, T *, T *, T, T,         \
                               cudaStream_t);                                                         \
  template void smooth_first<T>(int64_t, const T *, const T *, T *, T *, T, cudaStream_t);            \
  template void gs_sweeps<T>(const GsLevel &, const T *, const T *, T *, T, int, bool, cudaStream_t);   \
  template void lu_solve<T>(const DenseLU &, const T *, T *, cudaStream_t);                           \
  template void fill<T>(T *, int64_t, T, cudaStream_t);                                               \
  template void axpy_diag<T>(T *, const T *, const T *, int64_t, cudaStream_t);                       \
  template void axpy<T>(T *, const T *, T, int64_t, cudaStream_t);
MFS_INST(double)
MFS_INST(float)
template void convert<double, float>(const double *, float *, int64_t, cudaStream_t);
template void convert<float, double>(const float *, double *, int64_t, cudaStream_t);
template void convert<double, double>(const double *, double *, int64_t, cudaStream_t);
template void convert<float, float>(const float *, float *, int64_t, cudaStream_t);

}  // namespace dev
}  // namespace mfs
