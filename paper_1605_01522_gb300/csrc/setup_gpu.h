// Smoothed-aggregation setup on the GPU (same steps and results as the host
// setup of amg_setup.h; the results are downloaded into the same host
// structures so the export calls and the solve-phase upload are unchanged).
#pragma once
#include <cstdint>
#include <vector>

#include "amg_setup.h"

namespace mfs {

// Build the single-field hierarchies of a group on the current device
// (level structure, aggregation, prolongators, Galerkin blocks, lambda,
// coarse LU factors) into g, like build_group.
void build_group_gpu(HGroup &g, const std::vector<HBsr> &diag, const std::vector<FieldInfo> &info,
                     int max_levels, int64_t coarse_max, uint64_t seed, bool want_off,
                     const BlockMap *fine_off, int verbose);

// C = A * B on the GPU (deterministic accumulation order), host in / out.
HBsr gpu_spgemm(const HBsr &A, const HBsr &B);

}  // namespace mfs
