// Internal: the plan's front end built on the device (plan_gpu.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "plan.h"

#include <stdexcept>
#include <string>

namespace defmm {

// A failure of the device front end: a device allocation (out_of_memory) or
// another CUDA call.
struct DeviceFailure : std::runtime_error {
    bool out_of_memory;
    DeviceFailure(const std::string& what, bool oom) : std::runtime_error(what), out_of_memory(oom) {}
};

// Fills hp.tt (and hp.ts_own when Y is given), the M2L pairs with their best
// directions, the P2P pairs and the directional marks of Alg. 2 (each cell's
// distinct directions, sorted) from host coordinates, on the device, equal to
// the host construction entry for entry.  Needs hp.corner, hp.side and hp.lv.
// *device_ms receives the elapsed time on `stream`.  Throws DeviceFailure on
// a CUDA failure, std::runtime_error on a plan beyond its limits.
void device_front(const double* X, int64_t nx, const double* Y, int64_t ny, int ncrit, HostPlan& hp,
                  cudaStream_t stream, double* device_ms);

}  // namespace defmm
