// Device data layouts and kernel launchers of the solve phase.
//
// Block matrices are stored in a blocked SELL-32 layout: block rows are cut
// into slices of 32 consecutive rows, one thread per block row; slot t of a
// slice holds the t-th nonzero block of each of its 32 rows, with the 32
// lanes' copies of block entry e next to each other, so every load of a warp
// is one contiguous 128/256-byte segment.  Rows shorter than the slice width
// are padded but the padding is never read (per-row lengths).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include <vector>

namespace mfs {
namespace dev {

struct Sell {
  int kind = 0;                // 0: SELL-32, one thread per block row;
                               // 1: plain BSR, one warp per block row (long rows /
                               //    few rows: restriction, coarse levels); then sp is
                               //    the row pointer, col the block columns and the
                               //    values are contiguous per block (br*bc, row-major)
  int unroll = 2;              // SELL-32: slots of a row in flight per thread (2 or 4)
  int br = 0, bc = 0;
  int64_t nbr = 0, nbc = 0;
  int64_t nslices = 0, nslots = 0;
  int64_t nnzb = 0;            // true nonzero blocks (algorithmic size)
  const int32_t *sp = nullptr; // nslices + 1 slot offsets
  const int32_t *rl = nullptr; // nbr row lengths
  const int32_t *col = nullptr;// nslots * 32 block-column indices
  const double *v64 = nullptr; // nslots * br*bc * 32
  const float *v32 = nullptr;
  bool valid() const { return nbr > 0 || nbc > 0; }
  int64_t nrows() const { return nbr * br; }
  int64_t ncols() const { return nbc * bc; }
};

// Optional per-launch accounting (CUDA events around every launch, with the
// launch's algorithmic byte count); installed by the solver when profiling.
enum KernelClass { K_SPMV = 0, K_SMOOTH = 1, K_VECTOR = 2, K_COARSE = 3, K_ARNOLDI = 4, K_NCLASS = 5 };
// sig identifies the kernel variant: for SpMV / smoothing
// layout*1000 + br*100 + bc*10 + (float64 ? 1 : 0) with layout 0 SELL-32,
// 1 warp BSR, 2 merged rows, 3 SELL-32 with 4 slots in flight, 4 / 5 / 6 the
// Gauss-Seidel colour kernels on SELL-32 / warp BSR / SELL-32 x4, 7 one CTA per
// BSR row; otherwise a small id.
// rows = block rows (sparse kernels) or vector length.
struct LaunchHook {
  // returns false when this launch is not to be recorded (after() is then skipped)
  virtual bool before(cudaStream_t s, int cls, int sig, int64_t rows) = 0;
  virtual void after(cudaStream_t s, int cls, double bytes, int sig, int64_t rows, double flops) = 0;
  virtual ~LaunchHook() {}
};
void set_launch_hook(LaunchHook *h);
// While one of these lives, launches made by the constructing thread skip
// the hook (calls that serve no handle must not feed a handle's profile).
struct HookBypass {
  HookBypass();
  ~HookBypass();
  HookBypass(const HookBypass &) = delete;
  HookBypass &operator=(const HookBypass &) = delete;
};
// one-time device settings (call before any stream capture)
void init();

// Launch recording, for running many independent systems' launches as one
// grid per step.  While a thread has a recorder, every launcher below appends
// its launch (the multi-system form of its kernel, grid, block, dynamic
// shared memory, argument block and accounting) instead of issuing it.
struct RecOp {
  const void *fn = nullptr;  // multi-system kernel
  unsigned grid = 0, threads = 0;
  size_t smem = 0;
  std::vector<unsigned char> args;  // the kernel's argument block for this launch
  int cls = 0, sig = 0;
  int64_t rows = 0;
  double bytes = 0.0, flops = 0.0;
};
struct Recorder {
  std::vector<RecOp> ops;
};
void set_recorder(Recorder *r);
// this thread's solve-phase launches of at most max_grid CTAs overlap the end
// of their predecessor in the stream (programmatic dependent launch); 0: none
void set_pdl(unsigned max_grid);
// the caller queued something other than a kernel on a stream: the next
// launch waits for it the ordinary way
void pdl_break();
// CTA c of a multi-system launch of op.fn runs block bid (of nb) of table
// entry t, which belongs to system g; the kernel takes (tab, map, active):
// the device array of argument blocks (op.args layout, consecutive), the
// CTA map and the per-system flags (0: skip) or null
struct MsBlock {
  int t, bid, nb, g;
};

template <typename T> inline const T *vals(const Sell &A);
template <> inline const double *vals<double>(const Sell &A) { return A.v64; }
template <> inline const float *vals<float>(const Sell &A) { return A.v32; }

struct DenseLU {
  int n = 0;
  const double *lu = nullptr;   // column-major, unit-lower L and U
  const int32_t *perm = nullptr;
  const double *inv = nullptr;  // row-major inverse built from the factors (small n), or null
};

// y = alpha * A x + beta * z   (z may alias y or be null when beta == 0)
template <typename T>
void spmv(const Sell &A, const T *x, T *y, T alpha, T beta, const T *z, cudaStream_t s);

// All blocks of one block row of fields that share one sparsity pattern,
// merged: each slot holds [A_i0 | A_i1 | A_i2] (br x (b0+b1+b2), row-major,
// SELL-32 layout of M); y = A_i0 x_0 + A_i1 x_1 + A_i2 x_2 (float64).
struct RowMerged {
  Sell M;          // br x bct blocks, bct = b[0] + b[1] + b[2]
  int nb = 0;      // number of merged column fields (2 or 3)
  int b[3] = {0, 0, 0};
  int64_t off[3] = {0, 0, 0};  // offset of each column field in the coupled vector
  int split = 1;   // threads per block row (1, 2 or 4), timed at setup
};
bool rows_supported(int br, const int *b, int nb);
void spmv_rows(const RowMerged &R, const double *x, double *y, cudaStream_t s);

// One smoothing step on A with point-diagonal inverse dinv:
//   r = b - A x;  d = c1 * d + c2 * dinv * r;  xout = x + d
template <typename T>
void smooth_step(const Sell &A, const T *dinv, const T *b, const T *x, T *xout, T *d, T c1, T c2,
                 cudaStream_t s);
// First step from x = 0:  d = c2 * dinv * b;  x = d
template <typename T>
void smooth_first(int64_t n, const T *dinv, const T *b, T *x, T *d, T c2, cudaStream_t s);

// Multicolour damped Gauss-Seidel (SOR(omega) in the order colour, node,
// dof) on one level field.  M holds the field's block rows reordered by
// colour as plain BSR (kind 1, all blocks of each row); rowidx[k] is the node
// of reordered row k; colour c owns rows [hoff[c], hoff[c+1]) (coff is the
// device copy); dblk (caller's precision) the br x br diagonal block of every
// node, node order, row-major.  For each row's node i, with the sums
// s = (A x)_i taken from the x before its colour,
//   forward:  for r = 0..br-1:  dx_r = omega (b_r - s_r - sum_{c<r} D_rc dx_c) / D_rr
//   backward: for r = br-1..0:  the same with c > r;   x_i += dx;
// a forward sweep visits colours 0..nc-1, a backward one nc-1..0.  Rows of a
// colour do not couple, so they update in parallel; G lanes share a row.
// Large levels launch one kernel per colour; small ones (x fits in 48 KB of
// shared memory) run all colours and sweeps in one single-CTA launch.
struct GsLevel {
  Sell M;
  const int32_t *rowidx = nullptr;
  const int32_t *coff = nullptr;
  std::vector<int64_t> hoff;   // nc + 1 colour row offsets
  std::vector<int64_t> cnnzb;  // blocks per colour (algorithmic bytes)
  int G = 32;                  // lanes per row: 4, 8, 16 or 32
  bool small = false;          // one single-CTA launch for all colours (x in shared memory)
  int ncolors() const { return (int)hoff.size() - 1; }
};
template <typename T>
void gs_sweeps(const GsLevel &g, const T *dblk, const T *b, T *x, T omega, int sweeps, bool backward,
               cudaStream_t s);

// Tail of a single-field V-cycle in one CTA (Algorithm 1 from the level
// above the coarsest down through the coarse solve and back): A (level l,
// plain BSR, br x br blocks), its inverse point diagonal, R (to the coarsest,
// br x br blocks), P, the coarsest inverse (lu.inv, required), ns smoothing
// steps with coefficients c1, c2 (host arrays, ns <= 8), x = V-cycle(b) from
// zero.  Same arithmetic as the step-by-step launches.  Shared memory:
// tail_smem_bytes, which the caller keeps within 48 KB.
bool tail_supported(int br, int bc);
// true when spmv runs this plain-BSR matrix with one CTA per row (few, long rows)
bool cta_rows(const Sell &A);
size_t tail_smem_bytes(int64_t n, int64_t nc, size_t tsize);
template <typename T>
void vcycle_tail(const Sell &A, const T *dinv, const Sell &R, const Sell &P, const DenseLU &lu, int ns,
                 const T *c1, const T *c2, const T *b, T *x, cudaStream_t s);

// x = LU^-1 b  (dense; b, x of type T, arithmetic in float64): with lu.inv one
// warp per row of the explicit inverse, else one CTA of triangular sweeps
template <typename T>
void lu_solve(const DenseLU &lu, const T *b, T *x, cudaStream_t s);

// Layout building on the device (setup): from a plain BSR matrix already in
// device memory (int32 row pointer and block columns, float64 row-major
// blocks), row lengths rl and per-slice widths w (max row length of each slice
// of 32 rows) ...
void sell_widths(const int32_t *rp, int64_t nbr, int32_t *rl, int32_t *w, cudaStream_t s);
// ... then, with slice offsets sp (slots), the SELL-32 arrays (zeroed before):
// col, and v64 and/or v32 (either may be null).  With nsrc > 1 the sources
// share rp / ci and are merged column-wise per block ([A_0 | A_1 | A_2],
// bcs[j] columns each).
void sell_fill(const int32_t *rp, const int32_t *ci, int nsrc, const double *v0, const double *v1,
               const double *v2, const int *bcs, int br, int64_t nbr, const int32_t *sp, int32_t *col,
               double *v64, float *v32, cudaStream_t s);

// Measured FP64 FMA rate of this device in TFLOP/s (independent FMA chains
// on every SM, best over a few launch shapes, CUDA events on s); < 0 on error.
double fp64_rate(cudaStream_t s);

// elementwise helpers
template <typename T> void fill(T *x, int64_t n, T v, cudaStream_t s);
template <typename T> void axpy_diag(T *x, const T *dinv, const T *t, int64_t n, cudaStream_t s);  // x -= dinv*t
template <typename T> void axpy(T *y, const T *x, T a, int64_t n, cudaStream_t s);                 // y += a x
template <typename TI, typename TO> void convert(const TI *in, TO *out, int64_t n, cudaStream_t s);  // also a copy (TI = TO)
void scale(const double *x, double a, double *y, int64_t n, cudaStream_t s);                      // y = a x
// v = a v and out = (TO) v in one pass
template <typename TO> void scale_convert(double *v, double a, TO *out, int64_t n, cudaStream_t s);
// the same with a = 1 / sqrt(nrm2[0]) taken from device memory; out may be null
template <typename TO>
void scale_convert_dev(double *v, const double *nrm2, TO *out, int64_t n, cudaStream_t s);

// Arnoldi (float64).  V holds k row vectors of length n, row q at V + q*ldv.
int mdot_blocks(int64_t n);
void mdot(const double *V, int64_t ldv, int k, const double *w, int64_t n, double *partial,
          int nblk, cudaStream_t s);                                   // partial[q*nblk+b]
void reduce_partials(const double *partial, int k, int nblk, double *out, cudaStream_t s);
// w -= sum_q V_q h_q and partial dots V_q . w_new in one pass (k <= 64)
void cgs_fused(const double *V, int64_t ldv, int k, const double *h, double *w, int64_t n, double *partial,
               int nblk, cudaStream_t s);
// w -= sum_q V_q h_q; if partial != null also partial[b] = sum w_new^2 over block b
void cgs_update(const double *V, int64_t ldv, int k, const double *h, double *w, int64_t n,
                double *partial, int nblk, cudaStream_t s);
// x += sum_q Z_q y_q
void gemv_add(const double *Z, int64_t ldz, int k, const double *y, double *x, int64_t n,
              cudaStream_t s);

}  // namespace dev
}  // namespace mfs
