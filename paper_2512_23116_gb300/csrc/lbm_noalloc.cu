// Structure functions of a caller-owned device velocity field, computed
// without allocating any device memory.
//
// Who needs this: code that shares the GPU with a framework that owns the
// device memory through its own pool allocator (PyTorch's caching allocator,
// for instance) and must not grow the device footprint behind that pool's
// back, and latency-sensitive pipelines that cannot afford the implicit
// device-wide synchronisation cudaMalloc / cudaFree may cause.  They hand in
// an input velocity field and an output buffer they already own; the per-block
// partial sums that the reduction needs live in one fixed-size array of
// device memory declared below, which every GPU that loads this library keeps
// until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/lbm.h"
#include "lbm_kernels.h"

#define LBM_API extern "C" __attribute__((visibility("default")))

namespace lbm {
void set_global_error(const char* msg);
}

namespace {

constexpr int kBlocks = 512;            // blocks of each separation's reduction
constexpr int kMaxSeparations = LBM_MAX_R;
constexpr int kMaxDevices = 64;

// Partial sums of (d)^p, p = 1..6, per separation and block: 24 x 512 x 6
// doubles = 576 KiB.
static __device__ __align__(256) double g_sf_scratch[kMaxSeparations * kBlocks * 6];

std::mutex g_mutex;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of g_sf_scratch on the current device (looked up once per
// device, with that device current).
cudaError_t scratch_address(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sf_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// sp[k][p] = (sum over blocks of part[k][block][p]) * inv_count.
__global__ void k_sf_finish(const double* __restrict__ part, int nr, int blocks, double inv_count,
                            double* __restrict__ sp) {
  for (int idx = threadIdx.x; idx < nr * 6; idx += blockDim.x) {
    const int k = idx / 6, p = idx - k * 6;
    double s = 0.0;
    for (int b = 0; b < blocks; ++b) s += part[((int64_t)k * blocks + b) * 6 + p];
    sp[idx] = s * inv_count;
  }
}

int reject(int code, const char* msg) {
  lbm::set_global_error(msg);
  return code;
}

// True when [p, p + bytes) starts and ends in device (or managed) memory of
// device `dev`: both ends are looked up with cudaPointerGetAttributes, which
// allocates nothing.  A host pointer, a pointer of another device or an
// unknown address is rejected before any launch (a kernel given one would
// fault).  A lookup failure this call caused is not left pending on the
// thread; an error the caller left pending is not touched.
bool device_range(const void* p, size_t bytes, int dev) {
  const bool pending = cudaPeekAtLastError() != cudaSuccess;
  const char* ends[2] = {static_cast<const char*>(p), static_cast<const char*>(p) + bytes - 1};
  for (const char* q : ends) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, q) != cudaSuccess) {
      if (!pending) (void)cudaGetLastError();
      return false;
    }
    if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev ||
        !at.devicePointer)
      return false;
  }
  return true;
}

}  // namespace

LBM_API int lbm_structure_functions_noalloc(const float* u, int32_t nx, int32_t ny, int32_t nz,
                                            const int32_t* r, int32_t nr, double* sp,
                                            void* stream) {
  if (!u || !r || !sp) return reject(LBM_ERR_INVALID_ARG, "null pointer argument");
  if (nx < 1 || ny < 1 || nz < 1) return reject(LBM_ERR_INVALID_ARG, "lattice extents must be >= 1");
  if (nr < 1 || nr > kMaxSeparations)
    return reject(LBM_ERR_INVALID_ARG,
                  "nr must be between 1 and 24: the fixed scratch holds 24 separations");
  for (int k = 0; k < nr; ++k)
    if (r[k] < 1) return reject(LBM_ERR_INVALID_ARG, "separations must be >= 1");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return reject(LBM_ERR_CUDA, cudaGetErrorString(e));
  const size_t ncell = (size_t)nx * (size_t)ny * (size_t)nz;
  if (!device_range(u, 3 * ncell * sizeof(float), dev))
    return reject(LBM_ERR_INVALID_ARG, "u must be device memory of the current device (3 nx ny nz floats)");
  if (!device_range(sp, (size_t)nr * 6 * sizeof(double), dev))
    return reject(LBM_ERR_INVALID_ARG, "sp must be device memory of the current device (nr x 6 doubles)");
  double* scratch = nullptr;
  e = scratch_address(&scratch);
  if (e != cudaSuccess) return reject(LBM_ERR_CUDA, cudaGetErrorString(e));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int k = 0; k < nr; ++k) {
    e = lbm::launch_struct(u, nx, ny, nz, r[k], scratch + (size_t)k * kBlocks * 6, kBlocks, st);
    if (e != cudaSuccess) return reject(LBM_ERR_CUDA, cudaGetErrorString(e));
  }
  const double inv_count = 1.0 / (3.0 * (double)ncell);
  e = lbm::launch_kernel(k_sf_finish, 1, 160, 0, st, (const double*)scratch, nr, kBlocks, inv_count, sp);
  if (e != cudaSuccess) return reject(LBM_ERR_CUDA, cudaGetErrorString(e));
  return LBM_OK;
}
