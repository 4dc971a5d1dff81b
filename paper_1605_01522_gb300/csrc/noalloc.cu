// Allocation-free dot product: the two-stage reduction of mfs_dot with its
// partial sums in a file-scope device array instead of handle scratch.
//
// For callers that must not call cudaMalloc at run time: host frameworks
// whose caching allocator has already reserved the device memory (a driver
// allocation would fail or fragment it), latency-critical loops that cannot
// take cudaMalloc's implicit device-wide synchronisation, and plug-ins that
// are only allowed to allocate during their initialisation.  The array below
// is part of the library image, so it exists on every device that loads the
// library and stays there until the process exits.
#include <cstdint>
#include <mutex>

#include "kernels.cuh"
#include "mfs.h"

namespace mfs {
void set_last_error(const char *msg);  // thread-local detail behind mfs_last_error
}

namespace {

// MFS_DOT_NOALLOC_PARTIALS partial sums (one per reduction block; the
// chunking of dev::mdot_blocks never asks for more than 608) plus the result.
constexpr int kPartials = MFS_DOT_NOALLOC_PARTIALS;
static __device__ __align__(256) double g_dot_scratch[kPartials + 32];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_dot_scratch on the current device, resolved once per
// device (the host-side symbol is only a stand-in and must not reach a kernel).
int scratch_for_current_device(double **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return MFS_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_dot_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return MFS_ERR_CUDA;
    }
    g_scratch_addr[dev] = (double *)p;
  }
  *out = g_scratch_addr[dev];
  return MFS_OK;
}

// device (or managed) memory of device `dev`
bool on_device(const void *p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" int mfs_dot_noalloc(const double *x, const double *y, int64_t n, double *out, void *stream) {
  if (!x || !y || !out || n < 0) {
    mfs::set_last_error("mfs_dot_noalloc: NULL pointer or negative length");
    return MFS_ERR_INVALID;
  }
  if (n > MFS_DOT_NOALLOC_MAX_N) {
    mfs::set_last_error("mfs_dot_noalloc: n exceeds MFS_DOT_NOALLOC_MAX_N (2^32)");
    return MFS_ERR_INVALID;
  }
  if (n == 0) {
    *out = 0.0;
    return MFS_OK;
  }
  // first CUDA call: nothing else may run on a stream under capture
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    mfs::set_last_error("mfs_dot_noalloc: the stream is being captured (the call synchronises it)");
    return MFS_ERR_INVALID;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    mfs::set_last_error("mfs_dot_noalloc: no current CUDA device");
    return MFS_ERR_CUDA;
  }
  // the scratch address is the current device's, so the vectors must live there too
  if (!on_device(x, dev) || !on_device(y, dev)) {
    mfs::set_last_error("mfs_dot_noalloc: x and y must be device pointers on the current device");
    return MFS_ERR_INVALID;
  }
  double *scratch = nullptr;
  const int rc = scratch_for_current_device(&scratch);
  if (rc != MFS_OK) {
    mfs::set_last_error("mfs_dot_noalloc: cannot resolve the scratch array on this device");
    return rc;
  }
  const int nblk = mfs::dev::mdot_blocks(n);
  if (nblk > kPartials) {
    mfs::set_last_error("mfs_dot_noalloc: more reduction blocks than MFS_DOT_NOALLOC_PARTIALS");
    return MFS_ERR_INVALID;
  }
  // every partial that the second stage reads is written by the first stage,
  // so the contents left by the previous call need no clearing; the launches
  // bypass the profiling hook of any handle that another thread is solving with
  mfs::dev::HookBypass bypass;
  mfs::dev::mdot(x, 0, 1, y, n, scratch, nblk, s);
  mfs::dev::reduce_partials(scratch, 1, nblk, scratch + kPartials, s);
  double result = 0.0;
  if (cudaMemcpyAsync(&result, scratch + kPartials, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    mfs::set_last_error("mfs_dot_noalloc: CUDA error");
    return MFS_ERR_CUDA;
  }
  *out = result;
  return MFS_OK;
}
