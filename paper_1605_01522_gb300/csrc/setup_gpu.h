// Smoothed-aggregation setup on the GPU (same steps and results as the host
// setup of amg_setup.h; the results are downloaded into the same host
// structures so the export calls and the solve-phase upload are unchanged).
#pragma once
#include <cstdint>
#include <vector>

#include "amg_setup.h"

namespace mfs {

// Device copy of a block whose shape is given by its host HBsr: int32 row
// pointer and block columns, float64 row-major blocks.
struct DevBlock {
  const int32_t *rp = nullptr, *ci = nullptr;
  const double *v = nullptr;
};

// Build the single-field hierarchies of a group on the current device
// (level structure, aggregation, prolongators, Galerkin blocks, lambda,
// coarse LU factors) into g, like build_group.  dev_diag / dev_off, when
// given, hold device copies of diag / *fine_off (same order and keys), which
// are then copied on the device instead of uploaded again.  With steal (the
// same matrices as diag), level 0 of g takes them by move instead of a copy.
void build_group_gpu(HGroup &g, const std::vector<HBsr> &diag, const std::vector<FieldInfo> &info,
                     int max_levels, int64_t coarse_max, uint64_t seed, bool want_off,
                     const BlockMap *fine_off, int verbose, const std::vector<DevBlock> *dev_diag = nullptr,
                     const std::map<std::pair<int, int>, DevBlock> *dev_off = nullptr,
                     std::vector<HBsr> *steal = nullptr);

// C = A * B on the GPU (deterministic accumulation order), host in / out.
HBsr gpu_spgemm(const HBsr &A, const HBsr &B);

}  // namespace mfs
