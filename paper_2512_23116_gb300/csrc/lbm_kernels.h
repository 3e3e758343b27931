// Host-side launchers of the device kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <utility>

#include "lbm_internal.h"

namespace lbm {

// Launch `kernel` and return the status of this launch alone.  A <<<...>>>
// launch reports only through cudaGetLastError(), which also returns (and
// clears) any error the caller's own earlier work left pending on the thread;
// cudaLaunchKernelEx returns the launch's status and leaves that state alone.
template <typename... P, typename... A>
inline cudaError_t launch_kernel(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                 A&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = nullptr;
  cfg.numAttrs = 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

struct LaunchArgs {
  const InstDesc* insts;   // device table
  int ninst;
  int64_t tile_lo, tile_hi;
  int precision;           // 0 fp32, 1 fp16, 2 bf16
  bool odd;                // AA parity of the step (time t odd)
  int mode;                // MODE_STEP | MODE_STEP_STATS | MODE_DIAG
  StatsArgs sa;
  DiagOut dout;
  int grid, threads;
  // TMA kernel configuration
  int stages;
  int slot_bytes;          // shared-memory slot per population segment: kSlot3, kSlot2, kSlot2h, or the runtime
                           // stride rows x nxp: 0, or kSlotGrouped for the row-interleaved array
  int smem_bytes;          // dynamic shared memory of the TMA kernel
  int tile_bytes_max;      // bytes of one stage (19 segments)
  uint32_t* err;           // device error word
  long long wait_ns;       // bound of every device-side wait (nanoseconds)
  int withhold_first_load; // test hook: block 0 never loads its first tile
  int hist_smem;           // TMA statistics pass: byte offset of the theta histogram in
                           // dynamic shared memory (0: global counts)
  int hist_lo, hist_win;   // bins [hist_lo, hist_lo + hist_win) of it counted in shared memory
                           // (hist_smem > 0), the rest in the global counts
};

cudaError_t launch_step_direct(const LaunchArgs& la, cudaStream_t st);
int direct_max_blocks_per_sm(int precision, int threads);

// Compile-time shared-memory slots of the TMA kernel's population segments:
// 19 slots per stage, three stages of kSlot3 or two of kSlot2 bytes fill the
// 220 KB dynamic shared-memory budget (with the Fz table of x-lines up to 1440
// values).  A tile of R x-lines of nxp values fits a slot when R nxp (value
// size) <= slot.
constexpr int kSlot3 = 3840;
constexpr int kSlot2 = 5760;
// Two stages of 19 slots of kSlot2h bytes (109 KB) leave room for a second
// co-resident block on the SM.
constexpr int kSlot2h = 2880;
// Runtime-stride tiles of the row-interleaved array: segments at the grouped
// positions of their slots (odd steps then copy whole slot groups).
constexpr int kSlotGrouped = -1;

cudaError_t launch_step_tma(const LaunchArgs& la, cudaStream_t st);
// Dynamic shared memory a block may request (227 KB on sm_100 / sm_103).
constexpr int kMaxDynSmem = 232448;
// Dynamic shared memory of the TMA kernel: barriers, `stages` tile buffers and
// the Fz(x) table of the widest instance.
int tma_smem_bytes(int stages, int tile_bytes, int max_nx);
// Resident blocks per SM of the step variants (diag = false) or of the
// read-only statistics pass (diag = true).
int tma_max_blocks_per_sm(int precision, int slot_bytes, int threads, int smem_bytes, bool diag = false);
cudaError_t tma_prepare(int precision, int smem_bytes);
// Largest dynamic shared memory a launch of the read-only statistics pass can
// take (0 when the query fails).
int tma_diag_smem_limit(int precision);

// Initial condition: f' = equilibrium of (drho, u), written at AA parity `odd`,
// for the canonical cells [c0, c0 + n) (linear index (z ny + y) nx + x).
// mode: 0 rest, 1 TGV3D, 2 TGV2D, 3 velocity from device FP64 `u` with
// components at u[k], u[ustride + k], u[2 ustride + k] for cell c0 + k.
cudaError_t launch_init(const InstDesc& d, int precision, bool odd, int mode, double amp,
                        const double* u, int64_t ustride, int64_t c0, int64_t n,
                        cudaStream_t st);
// The same from an FP32 velocity (mode 3): identical populations for the FP32
// rounding of an FP64 field.
cudaError_t launch_init(const InstDesc& d, int precision, bool odd, const float* u, int64_t ustride,
                        int64_t c0, int64_t n, cudaStream_t st);
// Canonical population a of cells [c0, c0 + n) -> FP64 out[0..n) (+ w_a when !shifted).
cudaError_t launch_get_pop(const InstDesc& d, int precision, bool odd, int a, double* out,
                           int shifted, int64_t c0, int64_t n, cudaStream_t st);
cudaError_t launch_set_pop(const InstDesc& d, int precision, bool odd, int a, const double* in,
                           int shifted, int64_t c0, int64_t n, cudaStream_t st);
// Re-lay out the pair (a, opp a) from parity `from_odd` to the other parity
// using a scratch buffer of 2 * nz * ny * nxp storage elements.
cudaError_t launch_relayout_pair(const InstDesc& d, int precision, bool from_odd, int a,
                                 void* scratch, cudaStream_t st);
// Reduce block partials: results[i][kNP] for instances i in [0, ninst); when
// ring != null also append to ring[(seq[0] % cap)][ninst][kNP] and bump seq[0]
// (seq points at two words: the record count and a block counter kept at 0
// between launches).
cudaError_t launch_finish(const double* partials, int ninst, int grid, double* results,
                          double* ring, unsigned long long* seq, int cap, uint32_t* err,
                          cudaStream_t st);
// Shell sums of |u_hat|^2 / ncell^2 from an R2C spectrum [nz][ny][nx/2+1]:
// partials [blocks][kmax + 1] (accumulated onto), then summed by launch_spec_finish.
cudaError_t launch_spec_bin(const void* coeffs, int nx, int ny, int nz, int kmax,
                            double* partials, int blocks, cudaStream_t st);
cudaError_t launch_spec_finish(const double* partials, int blocks, int kmax, double* E,
                               cudaStream_t st);
// Structure functions: per block b, partials[b * block_stride + p - 1] = sum over
// its cells and the three axes of (u_a(x + r e_a) - u_a(x))^p, p = 1..6, for the
// velocity u [3][nz][ny][nx] FP32.
cudaError_t launch_struct(const float* u, int nx, int ny, int nz, int r, double* partials,
                          int blocks, cudaStream_t st, int64_t block_stride = 6);
// The separations of one launch (kernel parameter).
constexpr int kMaxStructSeps = 24;
struct StructSeps {
  int r[kMaxStructSeps];
};
// Structure functions of nr <= 24 separations r[0..nr) in one launch, FP32
// powers folded into FP64: partials [blocks][nr][6] of the per-block sums over
// cells and the three axes of d^p, p = 1..6.
cudaError_t launch_struct_multi(const float* u, int nx, int ny, int nz, const int* r, int nr, double* partials,
                                int blocks, cudaStream_t st);
cudaError_t launch_sum_cols(const double* partials, int rows, int cols, double* out,
                            cudaStream_t st);

// Seeded random solenoidal velocity (lbm_random_field.cu): the FP32 field
// u[3][nz][ny][nx] (device memory, 3 nx ny nz floats) of the recipe described
// there.  Allocates and frees its own FP64 / complex work buffers and a cuFFT
// plan; synchronises the stream.  Returns null on success, else the failed
// step (*cuda_err: the CUDA error, cudaErrorUnknown for a cuFFT failure).
const char* random_velocity_f32(int nx, int ny, int nz, uint64_t seed, double urms, double k0, float* u,
                                cudaStream_t st, cudaError_t* cuda_err);
// Largest |k| of the random field's modes: max(1, min(n_min / 2 - 1, floor(6 k0))).
int random_field_cutoff(int nx, int ny, int nz, double k0);

// Checked build (-DLBM_BOUNDS_CHECK): each kernel file's bounds word, read and
// cleared (0 in the normal build).
uint32_t bounds_word_tma();
uint32_t bounds_word_direct();
uint32_t bounds_word_aux();
uint32_t bounds_word_random();

}  // namespace lbm
