// Host-side helpers of the C ABI: argument checks, launch error capture and
// device properties cached per device.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gbar.h"

namespace gbar {

void set_cuda_error(cudaError_t e);

// Returns AR_OK when the last launch on this thread succeeded, else records
// the CUDA error and returns AR_ERR_CUDA.
int check_launch();

struct DeviceInfo {
  int device = -1;
  int sm_count = 0;
  int max_smem_optin = 0;  // bytes of dynamic shared memory a CTA may opt in to
};
// Properties of the current device (queried once per device).
const DeviceInfo& device_info();

inline bool aligned(const void* p, uintptr_t a) {
  return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0;
}
inline size_t dtype_size(int dtype) { return dtype == AR_F64 ? 8 : 4; }
inline bool valid_dtype(int d) { return d == AR_F32 || d == AR_F64; }
inline bool valid_cmp(int c) { return c == AR_CMP_F32 || c == AR_CMP_F64; }

}  // namespace gbar
