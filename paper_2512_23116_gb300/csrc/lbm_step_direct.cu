// Direct-load stream + collide kernel (AA pattern, one population array).
//
// Even step: cell x reads f_a from its own slot a and writes f*_a to its own
// slot opp(a).  Odd step: cell x reads f_a from slot opp(a) of x - c_a and
// writes f*_a to slot a of x + c_a.  Each cell reads exactly the locations it
// writes, so all cells of a step are independent (Eq. mrt_les_guo, with
// periodic streaming of Sec. 3.1).  One thread per cell, plain coalesced
// loads and stores; the grid walks tiles of `rows` x-lines.
#include <cuda_runtime.h>

#include "lbm_device.cuh"
#include "lbm_kernels.h"
#include "lbm_reduce.cuh"

namespace lbm {

constexpr int kSmemHistBins = 12000;  // (bins + 1) * 4 bytes below 48 KB

template <typename T, bool ODD, int MODE>
__global__ void __launch_bounds__(256, 2)
k_step_direct(const InstDesc* __restrict__ insts, int ninst, int64_t tile_lo, int64_t tile_hi,
              StatsArgs sa, DiagOut dout) {
  using S = Storage<T>;
  extern __shared__ uint32_t shist[];
  // theta histogram in shared memory when it fits the default 48 KB, else
  // straight into the global counts
  const bool use_hist = (MODE == MODE_DIAG) && dout.hist != nullptr && dout.hist_bins < kSmemHistBins;
  if (use_hist) {
    for (int i = threadIdx.x; i <= dout.hist_bins; i += blockDim.x) shist[i] = 0u;
    __syncthreads();
  }
  Acc acc;
  acc.reset();
  HistRun run;
  uint32_t* const hist_sm = use_hist ? shist : nullptr;
  const int hist_win = use_hist ? dout.hist_bins + 1 : 0;
  uint32_t* const hist_gl = use_hist ? nullptr : dout.hist;
  int cur = -1, hint = 0;
  for (int64_t t = tile_lo + blockIdx.x; t < tile_hi; t += gridDim.x) {
    const int ii = find_instance(insts, ninst, t, cur < 0 ? hint : cur);
    hint = ii;
    if (MODE != MODE_STEP && ii != cur) {
      if (cur >= 0)
        block_flush(acc, sa.partials + ((int64_t)cur * sa.grid + blockIdx.x) * kNP, blockDim.x, 0);
      acc.reset();
      cur = ii;
    }
    const InstDesc& d = insts[ii];
    const int nx = d.nx, ny = d.ny, nz = d.nz;
    const int64_t ps = d.slot_stride, pls = d.plane_stride, rs = d.row_stride;
    const bool grouped = d.slot_grouped != 0;
    // position of cell (x, y, z) within a population slot; offset of slot a
    auto at = [pls, rs](int x, int y, int z) { return z * pls + y * rs + x; };
    auto slot = [ps, grouped](int a) { return (grouped ? gpos(a) : a) * ps; };
    const int64_t local = t - d.tile_begin;
    const int z = (int)(local / d.tiles_per_plane);
    const int y0 = (int)(local - (int64_t)z * d.tiles_per_plane) * d.rows;
    const int rows = min(d.rows, ny - y0);
    const int ncell = rows * nx;
    T* __restrict__ fb = static_cast<T*>(d.f);
    const int zm = wrap_dec(z, nz), zp = wrap_inc(z, nz);
    const float Fy = (in_bounds(z >= 0 && z < nz) ? d.fy_of_z[z] : 0.f) + d.fconst[1];
    const float nu0 = d.nu0, s_nu0 = d.s_nu0, C = d.C;
    const int dr = blockDim.x / nx, dx = blockDim.x - dr * nx;  // a pass of blockDim.x cells
    int r = threadIdx.x / nx, x = threadIdx.x - r * nx;
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
      const int y = y0 + r;
      const int ym = wrap_dec(y, ny), yp = wrap_inc(y, ny);
      const int xm = wrap_dec(x, nx), xp = wrap_inc(x, nx);
      float f[19];
      if (!ODD) {
        const int64_t o = at(x, y, z);
#pragma unroll
        for (int a = 0; a < 19; ++a) {
          const int64_t i = slot(a) + o;
          f[a] = in_bounds(i >= 0 && i < d.f_elems) ? S::load(fb + i) : 0.f;
        }
      } else {
#pragma unroll
        for (int a = 0; a < 19; ++a) {
          const int xs = cx(a) > 0 ? xm : (cx(a) < 0 ? xp : x);
          const int ys = cy(a) > 0 ? ym : (cy(a) < 0 ? yp : y);
          const int zs = cz(a) > 0 ? zm : (cz(a) < 0 ? zp : z);
          const int64_t i = slot(opp(a)) + at(xs, ys, zs);
          f[a] = in_bounds(i >= 0 && i < d.f_elems) ? S::load(fb + i) : 0.f;
        }
      }
      const float Fx = (in_bounds(y >= 0 && y < ny) ? d.fx_of_y[y] : 0.f) + d.fconst[0];
      const float Fz = (in_bounds(x >= 0 && x < nx) ? d.fz_of_x[x] : 0.f) + d.fconst[2];
      CellDiag g;
      mrt_collide(f, Fx, Fy, Fz, nu0, s_nu0, C, g, d.strain_mode);
      if (MODE != MODE_DIAG) {
        if (!ODD) {
          const int64_t o = at(x, y, z);
#pragma unroll
          for (int a = 0; a < 19; ++a) {
            const int64_t i = slot(opp(a)) + o;
            if (in_bounds(i >= 0 && i < d.f_elems)) fb[i] = S::pack(f[a]);
          }
        } else {
#pragma unroll
          for (int a = 0; a < 19; ++a) {
            const int xd = cx(a) > 0 ? xp : (cx(a) < 0 ? xm : x);
            const int yd = cy(a) > 0 ? yp : (cy(a) < 0 ? ym : y);
            const int zd = cz(a) > 0 ? zp : (cz(a) < 0 ? zm : z);
            const int64_t i = slot(a) + at(xd, yd, zd);
            if (in_bounds(i >= 0 && i < d.f_elems)) fb[i] = S::pack(f[a]);
          }
        }
      }
      if (MODE != MODE_STEP) acc.add(g, Fx, Fy, Fz, C);
      if (MODE == MODE_DIAG) diag_write(dout, g, x, y, z, nx, ny, nz, hist_sm, 0, hist_win, hist_gl, run);
      x += dx;
      r += dr;
      if (x >= nx) {
        x -= nx;
        r += 1;
      }
    }
    if (MODE != MODE_STEP) acc.fold_if_full();
  }
  if (MODE != MODE_STEP) {
    if (cur >= 0)
      block_flush(acc, sa.partials + ((int64_t)cur * sa.grid + blockIdx.x) * kNP, blockDim.x, 0);
  }
  if (MODE == MODE_DIAG && dout.hist) run.flush(hist_sm, 0, hist_win, hist_gl);
  if (use_hist) {
    __syncthreads();
    for (int i = threadIdx.x; i <= dout.hist_bins; i += blockDim.x)
      if (shist[i]) atomicAdd(&dout.hist[i], shist[i]);
  }
}

template <typename T, bool ODD, int MODE>
static cudaError_t launch_direct_t(const LaunchArgs& la, cudaStream_t st) {
  const size_t smem = (MODE == MODE_DIAG && la.dout.hist && la.dout.hist_bins < kSmemHistBins)
                          ? (size_t)(la.dout.hist_bins + 1) * 4
                          : 0;
  return launch_kernel(k_step_direct<T, ODD, MODE>, la.grid, la.threads, smem, st, la.insts, la.ninst,
                       la.tile_lo, la.tile_hi, la.sa, la.dout);
}

template <typename T>
static cudaError_t dispatch_direct(const LaunchArgs& la, cudaStream_t st) {
  if (la.odd) {
    if (la.mode == MODE_STEP) return launch_direct_t<T, true, MODE_STEP>(la, st);
    if (la.mode == MODE_STEP_STATS) return launch_direct_t<T, true, MODE_STEP_STATS>(la, st);
    return launch_direct_t<T, true, MODE_DIAG>(la, st);
  }
  if (la.mode == MODE_STEP) return launch_direct_t<T, false, MODE_STEP>(la, st);
  if (la.mode == MODE_STEP_STATS) return launch_direct_t<T, false, MODE_STEP_STATS>(la, st);
  return launch_direct_t<T, false, MODE_DIAG>(la, st);
}

cudaError_t launch_step_direct(const LaunchArgs& la, cudaStream_t st) {
  switch (la.precision) {
    case 0: return dispatch_direct<float>(la, st);
    case 1: return dispatch_direct<__half>(la, st);
    case 2: return dispatch_direct<__nv_bfloat16>(la, st);
    default: return cudaErrorInvalidValue;
  }
}

int direct_max_blocks_per_sm(int precision, int threads) {
  int n = 0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (precision) {
    case 0: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_direct<float, true, MODE_STEP>, threads, 0); break;
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_direct<__half, true, MODE_STEP>, threads, 0); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_direct<__nv_bfloat16, true, MODE_STEP>, threads, 0); break;
  }
  return e == cudaSuccess ? n : 0;
}

uint32_t bounds_word_direct() { return take_bounds_word(); }

}  // namespace lbm
