// TMA bulk-copy stream + collide kernel (AA pattern, one population array).
//
// A tile is `rows` consecutive x-lines of one z-plane.  In the AA pattern the
// locations a tile reads are exactly the locations it writes, and they form
// 19 contiguous segments of rows x nxp values (one per population slot):
//   even step: slot a of the tile's own rows;
//   odd step:  slot opp(a) of rows y - cy_a of plane z - cz_a (a periodic wrap
//              in y splits a segment in two; the x wrap is resolved in shared
//              memory because whole lines are loaded).
// Each persistent block runs one producer warp and `threads/32 - 1` consumer
// warps.  The producer streams the segments of the block's next tiles into a
// ring of `stages` shared-memory buffers with cp.async.bulk (the TMA engine;
// 16-byte aligned rows, nxp padded for that) and mbarrier transaction counts;
// consumers read the 19 populations of a cell from shared memory, collide in
// FP32 registers (lbm_device.cuh), and store the 19 results with coalesced
// global stores.  A buffer is released to the producer as soon as its
// consumers have read it.  Every mbarrier wait is bounded by the global timer:
// on expiry the block records ERR_TIMEOUT, stops issuing, waits (bounded) for
// its copies in flight and returns.
#include <cuda_runtime.h>

#include "lbm_device.cuh"
#include "lbm_kernels.h"
#include "lbm_reduce.cuh"

namespace lbm {

namespace {

constexpr int kBarBytes = 128;          // mbarriers at the start of dynamic smem
constexpr long long kWaitNs = 2000000000ll;  // 2 s per wait

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: true when the phase with the given parity has completed.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (global_ns() - t0 > (unsigned long long)kWaitNs) return false;
  }
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

struct TileGeom {
  int ii, z, y0, rows;
};

__device__ __forceinline__ TileGeom tile_geom(const InstDesc* __restrict__ insts, int ninst, int64_t t) {
  TileGeom g;
  g.ii = find_instance(insts, ninst, t);
  const InstDesc& d = insts[g.ii];
  const int64_t local = t - d.tile_begin;
  g.z = (int)(local / d.tiles_per_plane);
  g.y0 = (int)(local - (int64_t)g.z * d.tiles_per_plane) * d.rows;
  g.rows = min(d.rows, d.ny - g.y0);
  return g;
}

// Producer: issue the 19 (or up to 38, when a y wrap splits a segment) bulk
// copies of one tile into stage buffer `buf`, completing on mbarrier `bar`.
template <typename T, bool ODD>
__device__ __forceinline__ void issue_tile(const InstDesc& d, const TileGeom& g, uint32_t buf,
                                           uint32_t bar) {
  const uint32_t row_bytes = (uint32_t)d.nxp * (uint32_t)sizeof(T);
  const uint32_t seg_bytes = row_bytes * (uint32_t)g.rows;
  mbar_expect_tx(bar, 19u * seg_bytes);
  const char* base = static_cast<const char*>(d.f);
  const int64_t plane_bytes = (int64_t)d.ny * row_bytes;
  const int64_t slot_bytes = d.pop_stride * (int64_t)sizeof(T);
#pragma unroll 1
  for (int j = 0; j < 19; ++j) {
    const uint32_t dst = buf + (uint32_t)j * seg_bytes;
    if (!ODD) {
      const char* src = base + j * slot_bytes + g.z * plane_bytes + (int64_t)g.y0 * row_bytes;
      bulk_load(dst, src, seg_bytes, bar);
    } else {
      const int slot = opp(j);
      int zs = g.z - cz(j);
      zs = zs < 0 ? zs + d.nz : (zs >= d.nz ? zs - d.nz : zs);
      int ys = g.y0 - cy(j);
      ys = ys < 0 ? ys + d.ny : (ys >= d.ny ? ys - d.ny : ys);
      const char* plane = base + slot * slot_bytes + zs * plane_bytes;
      if (ys + g.rows <= d.ny) {
        bulk_load(dst, plane + (int64_t)ys * row_bytes, seg_bytes, bar);
      } else {
        const int first = d.ny - ys;
        bulk_load(dst, plane + (int64_t)ys * row_bytes, (uint32_t)first * row_bytes, bar);
        bulk_load(dst + (uint32_t)first * row_bytes, plane, (uint32_t)(g.rows - first) * row_bytes, bar);
      }
    }
  }
}

template <typename T, bool ODD, int MODE>
__global__ void __launch_bounds__(512, 1)
k_step_tma(const InstDesc* __restrict__ insts, int ninst, int64_t tile_lo, int64_t tile_hi,
           StatsArgs sa, int stages, int tile_bytes, uint32_t* __restrict__ err) {
  using S = Storage<T>;
  extern __shared__ __align__(128) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nconsumer_warps = (blockDim.x >> 5) - 1;
  const int nct = nconsumer_warps * 32;
  const uint32_t bar_full = smem_addr(smem);
  const uint32_t bar_empty = bar_full + 8u * stages;
  const uint32_t buf0 = smem_addr(smem + kBarBytes);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 8 * 2 * stages);

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(bar_full + 8u * s, 1u);
      mbar_init(bar_empty + 8u * s, (uint32_t)nconsumer_warps);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  if (warp == nconsumer_warps) {
    // ---------------- producer warp ----------------
    if (lane != 0) return;
    uint32_t outstanding = 0;  // bit s: stage s has a load not yet seen consumed
    int last_use[8];           // last issued use of each stage
    for (int s = 0; s < 8; ++s) last_use[s] = -1;
    int k = 0;
    for (int64_t t = tile_lo + blockIdx.x; t < tile_hi; t += gridDim.x, ++k) {
      const int s = k % stages;
      const int use = k / stages;
      if (use > 0) {
        if (!mbar_wait(bar_empty + 8u * s, (uint32_t)((use - 1) & 1))) {
          atomicOr(err, ERR_TIMEOUT);
          *abort_flag = 1;
          break;
        }
        outstanding &= ~(1u << s);  // its consumers saw the data: that load completed
      }
      if (*abort_flag) break;
      const TileGeom g = tile_geom(insts, ninst, t);
      issue_tile<T, ODD>(insts[g.ii], g, buf0 + (uint32_t)s * tile_bytes, bar_full + 8u * s);
      outstanding |= 1u << s;
      last_use[s] = use;
    }
    if (*abort_flag) {
      // drain: wait (bounded) for every copy still in flight into this block
      for (int s = 0; s < stages; ++s)
        if ((outstanding & (1u << s)) && last_use[s] >= 0)
          (void)mbar_wait(bar_full + 8u * s, (uint32_t)(last_use[s] & 1));
    }
    return;
  }

  // ---------------- consumer warps ----------------
  const int ctid = threadIdx.x;
  Acc acc;
  acc.reset();
  int cur = -1;
  bool ok = true;
  int k = 0;
  for (int64_t t = tile_lo + blockIdx.x; t < tile_hi; t += gridDim.x, ++k) {
    const TileGeom g = tile_geom(insts, ninst, t);
    if (MODE == MODE_STEP_STATS && g.ii != cur) {
      if (cur >= 0)
        block_flush(acc, sa.partials + ((int64_t)cur * sa.grid + blockIdx.x) * kNP, nct, 1);
      acc.reset();
      cur = g.ii;
    }
    const int s = k % stages;
    const int use = k / stages;
    if (ok) {
      if (*abort_flag) {
        ok = false;
      } else if (!mbar_wait(bar_full + 8u * s, (uint32_t)(use & 1))) {
        atomicOr(err, ERR_TIMEOUT);
        *abort_flag = 1;
        ok = false;
      }
    }
    if (!ok) {
      if (MODE == MODE_STEP_STATS) continue;  // keep the named-barrier schedule of the flushes
      break;
    }
    const InstDesc& d = insts[g.ii];
    const int nx = d.nx, ny = d.ny, nz = d.nz, nxp = d.nxp;
    const int64_t ps = d.pop_stride;
    T* __restrict__ fb = static_cast<T*>(d.f);
    const T* sbuf = reinterpret_cast<const T*>(smem + kBarBytes + (size_t)s * tile_bytes);
    const int seg = g.rows * nxp;
    const int ncell = g.rows * nx;
    const int z = g.z;
    const int zm = wrap_dec(z, nz), zp = wrap_inc(z, nz);
    const float Fy = d.fy_of_z[z] + d.fconst[1];
    const float nu0 = d.nu0, s_nu0 = d.s_nu0, C = d.C;
    for (int c = ctid; c < ncell; c += nct) {
      const int r = c / nx;
      const int x = c - r * nx;
      const int y = g.y0 + r;
      const int xm = wrap_dec(x, nx), xp = wrap_inc(x, nx);
      float f[19];
#pragma unroll
      for (int a = 0; a < 19; ++a) {
        const int xs = ODD ? (cx(a) > 0 ? xm : (cx(a) < 0 ? xp : x)) : x;
        f[a] = S::cvt(sbuf[a * seg + r * nxp + xs]);
      }
      const float Fx = d.fx_of_y[y] + d.fconst[0];
      const float Fz = d.fz_of_x[x] + d.fconst[2];
      CellDiag cd;
      mrt_collide(f, Fx, Fy, Fz, nu0, s_nu0, C, cd);
      if (!ODD) {
        const int64_t o = cell_off(x, y, z, ny, nxp);
#pragma unroll
        for (int a = 0; a < 19; ++a) fb[opp(a) * ps + o] = S::pack(f[a]);
      } else {
        const int ym = wrap_dec(y, ny), yp = wrap_inc(y, ny);
#pragma unroll
        for (int a = 0; a < 19; ++a) {
          const int xd = cx(a) > 0 ? xp : (cx(a) < 0 ? xm : x);
          const int yd = cy(a) > 0 ? yp : (cy(a) < 0 ? ym : y);
          const int zd = cz(a) > 0 ? zp : (cz(a) < 0 ? zm : z);
          fb[a * ps + cell_off(xd, yd, zd, ny, nxp)] = S::pack(f[a]);
        }
      }
      if (MODE == MODE_STEP_STATS) acc.add(cd, Fx, Fy, Fz, C);
    }
    // release the stage to the producer once this warp has read it
    __syncwarp();
    if (lane == 0) mbar_arrive(bar_empty + 8u * s);
  }
  if (MODE == MODE_STEP_STATS && cur >= 0)
    block_flush(acc, sa.partials + ((int64_t)cur * sa.grid + blockIdx.x) * kNP, nct, 1);
}

template <typename T, bool ODD, int MODE>
cudaError_t launch_tma_t(const LaunchArgs& la, cudaStream_t st) {
  (void)cudaGetLastError();  // errors of earlier calls were reported by their return codes
  k_step_tma<T, ODD, MODE><<<la.grid, la.threads, la.smem_bytes, st>>>(
      la.insts, la.ninst, la.tile_lo, la.tile_hi, la.sa, la.stages, la.tile_bytes_max, la.err);
  return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch_tma(const LaunchArgs& la, cudaStream_t st) {
  if (la.mode == MODE_DIAG) return cudaErrorInvalidValue;
  if (la.odd)
    return la.mode == MODE_STEP ? launch_tma_t<T, true, MODE_STEP>(la, st)
                                : launch_tma_t<T, true, MODE_STEP_STATS>(la, st);
  return la.mode == MODE_STEP ? launch_tma_t<T, false, MODE_STEP>(la, st)
                              : launch_tma_t<T, false, MODE_STEP_STATS>(la, st);
}

template <typename T>
cudaError_t set_smem(int smem) {
  const void* fns[] = {(const void*)k_step_tma<T, false, MODE_STEP>, (const void*)k_step_tma<T, true, MODE_STEP>,
                       (const void*)k_step_tma<T, false, MODE_STEP_STATS>,
                       (const void*)k_step_tma<T, true, MODE_STEP_STATS>};
  for (const void* f : fns) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_step_tma(const LaunchArgs& la, cudaStream_t st) {
  if (la.threads < 64 || la.threads > 512 || (la.threads & 31) || la.stages < 1 || la.stages > 6 ||
      (la.tile_bytes_max & 15))
    return cudaErrorInvalidValue;
  switch (la.precision) {
    case 0: return dispatch_tma<float>(la, st);
    case 1: return dispatch_tma<__half>(la, st);
    case 2: return dispatch_tma<__nv_bfloat16>(la, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t tma_prepare(int precision, int smem_bytes) {
  // The dynamic shared-memory limit is a property of the kernel function,
  // shared by every handle of the process: only ever raise it.
  static int granted[3] = {0, 0, 0};
  if (precision < 0 || precision > 2) return cudaErrorInvalidValue;
  if (smem_bytes <= granted[precision]) return cudaSuccess;
  cudaError_t e = cudaErrorInvalidValue;
  switch (precision) {
    case 0: e = set_smem<float>(smem_bytes); break;
    case 1: e = set_smem<__half>(smem_bytes); break;
    case 2: e = set_smem<__nv_bfloat16>(smem_bytes); break;
  }
  if (e == cudaSuccess) granted[precision] = smem_bytes;
  return e;
}

int tma_max_blocks_per_sm(int precision, int threads, int smem_bytes) {
  int n = 0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (precision) {
    case 0: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_tma<float, true, MODE_STEP_STATS>, threads, smem_bytes); break;
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_tma<__half, true, MODE_STEP_STATS>, threads, smem_bytes); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_tma<__nv_bfloat16, true, MODE_STEP_STATS>, threads, smem_bytes); break;
  }
  return e == cudaSuccess ? n : 0;
}

}  // namespace lbm
