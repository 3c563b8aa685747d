// CIC deposit that allocates nothing: the 64-bit fixed-point accumulator lives in a
// file-scope device array instead of memory obtained from cudaMalloc/cudaMallocAsync.
//
// Callers that cannot allocate device memory use this entry point, for example code that
// runs while a framework's caching allocator holds the device memory (a direct driver
// allocation can then fail even though the framework has free blocks), code that must keep
// a fixed device-memory footprint after start-up, or latency-critical loops that cannot
// afford the implicit synchronisation of cudaFree.
#include <mutex>

#include "pm.cuh"

namespace dh {

// 2,097,152 cells (128^3) x 8 bytes = 16 MiB per device, held from module load until exit.
static __device__ __align__(256) unsigned long long g_deposit_scratch[SIM_DEPOSIT_STATIC_MAX_CELLS];

// Device address of g_deposit_scratch, looked up once per device with that device current.
// In host code the symbol name is only a host-side stand-in, never a device address.
static sim_status scratch_address(unsigned long long** out) {
  static std::mutex mu;
  static unsigned long long* addr[64] = {nullptr};
  int dev = 0;
  DH_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("sim_deposit_cic_static: device index %d out of range", dev);
    return SIM_EINVAL;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    DH_CUDA_TRY(cudaGetSymbolAddress(&p, g_deposit_scratch));
    addr[dev] = static_cast<unsigned long long*>(p);
  }
  *out = addr[dev];
  return SIM_OK;
}

}  // namespace dh

using namespace dh;

extern "C" sim_status sim_deposit_cic_static(const float* s, const float* values, int32_t n,
                                             double box, float* grid, void* stream) {
  if (!s || !grid || n < 1 || !(box > 0)) {
    set_error("sim_deposit_cic_static: invalid arguments");
    return SIM_EINVAL;
  }
  const long long N3 = (long long)n * n * n;
  if (N3 > SIM_DEPOSIT_STATIC_MAX_CELLS) {
    set_error("sim_deposit_cic_static: n^3 = %lld cells exceeds the static scratch of %d cells "
              "(n <= 128); use sim_deposit_cic", N3, SIM_DEPOSIT_STATIC_MAX_CELLS);
    return SIM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long* acc = nullptr;
  DH_TRY(scratch_address(&acc));
  // the array keeps the previous call's contents: clear the part this call accumulates into
  DH_CUDA_TRY(cudaMemsetAsync(acc, 0, N3 * sizeof(unsigned long long), st));
  DH_TRY(launch_deposit(s, values, n, (float)(n / box), acc, 1, st));
  return launch_fix_to_float(acc, sarg(1.0f), grid, (int)N3, 0.0f, grid, n, 1, st);
}
