// Error handling and small helpers shared by the CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#include <stdexcept>
#include <string>

#include "ph.h"

namespace ph {

struct Error : std::runtime_error {
    ph_status status;
    Error(ph_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

inline void cuda_check(cudaError_t e, const char* what, const char* file, int line) {
    if (e != cudaSuccess) {
        ph_status s = (e == cudaErrorMemoryAllocation) ? PH_ERR_OOM : PH_ERR_CUDA;
        throw Error(s, std::string(what) + ": " + cudaGetErrorString(e) + " (" + file + ":" +
                           std::to_string(line) + ")");
    }
}

#define PH_CUDA(call) ::ph::cuda_check((call), #call, __FILE__, __LINE__)
#define PH_LAUNCH(what) ::ph::cuda_check(cudaGetLastError(), what, __FILE__, __LINE__)

inline long long ceil_div(long long a, long long b) { return (a + b - 1) / b; }

}  // namespace ph
