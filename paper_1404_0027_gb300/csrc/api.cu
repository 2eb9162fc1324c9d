// Library-wide entry points: version, CUDA error capture, device properties.
#include <mutex>

#include "host.hpp"

namespace gbar {

static thread_local int g_last_cuda_error = 0;

void set_cuda_error(cudaError_t e) { g_last_cuda_error = (int)e; }

int check_launch() {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return AR_ERR_CUDA;
  }
  return AR_OK;
}

const DeviceInfo& device_info() {
  static DeviceInfo infos[64];
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  std::lock_guard<std::mutex> lock(mu);
  DeviceInfo& d = infos[dev];
  if (d.device != dev) {
    cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&d.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    d.device = dev;
  }
  return d;
}

}  // namespace gbar

extern "C" int ar_version(void) { return 100; }
extern "C" int ar_last_cuda_error(void) { return gbar::g_last_cuda_error; }
