// TMA bulk-copy stream + collide kernel (AA pattern, one population array).
//
// A tile is `rows` consecutive x-lines of one z-plane.  In the AA pattern the
// locations a tile reads are exactly the locations it writes, and they form
// 19 contiguous segments of rows x nxp values (one per population slot):
//   even step: slot a of the tile's own rows;
//   odd step:  slot opp(a) of rows y - cy_a of plane z - cz_a (a periodic wrap
//              in y splits a segment in two; the x wrap is resolved in shared
//              memory because whole lines are loaded).
// Segment a of the shared-memory tile holds what cell x reads as f_a at
// position x - [odd] cx_a; the cell writes f*_a into segment opp(a) at position
// x + [odd] cx_a.  Over the 19 populations the positions a cell writes are the
// positions it read, so every thread updates its cells in place with no
// hazard against other threads, and the tile goes back to global memory as
// the same 19 segments.
//
// Each persistent block runs one producer warp and `threads/32 - 1` consumer
// warps.  Producer lane j (j < 19) owns segment j: it streams that segment of
// the block's next tiles into a ring of `stages` shared-memory buffers with
// cp.async.bulk (the TMA engine; x-lines start on 16-byte boundaries, nxp is
// padded for that) completing on mbarrier transaction counts, and writes each
// finished tile back with cp.async.bulk shared->global (its own bulk group, so
// it reloads its segment as soon as its own store has read it).  Consumers read the 19
// populations of a cell from shared memory, collide in FP32 registers
// (lbm_device.cuh) and write the 19 results back in place; global memory is
// touched by the TMA engine only.  Every mbarrier wait is bounded by the
// global timer: on expiry the block records ERR_TIMEOUT, stops issuing, waits
// (bounded) for its loads in flight and for its stores, and returns.
#include <cuda_runtime.h>

#include "lbm_device.cuh"
#include "lbm_kernels.h"
#include "lbm_reduce.cuh"

namespace lbm {

namespace {

constexpr int kBarBytes = 128;  // mbarriers + abort flag

// Per population j: the slot read by the odd step (opp j) and the row shift
// (cy_j, cz_j), for the producer lanes (one lane per segment).
__constant__ int8_t c_seg_opp[19] = {1, 0, 3, 2, 5, 4, 7, 6, 9, 8, 11, 10, 13, 12, 15, 14, 17, 16, 18};
__constant__ int8_t c_seg_cy[19] = {0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 1, -1, 1, -1, 0, 0, 0, 0, 0};
__constant__ int8_t c_seg_cz[19] = {0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1, 0};

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

// Bounded wait: true when the phase with the given parity has completed,
// false once wait_ns nanoseconds of the global timer have passed.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long wait_ns) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (global_ns() - t0 > (unsigned long long)wait_ns) return false;
  }
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void bulk_store(void* dst, uint32_t src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// All committed bulk stores of this thread have finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// All committed bulk stores of this thread are complete (writes performed).
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

struct TileGeom {
  int ii, z, y0, rows;
};

__device__ __forceinline__ TileGeom tile_geom(const InstDesc* __restrict__ insts, int ninst, int64_t t,
                                              int hint) {
  TileGeom g;
  g.ii = find_instance(insts, ninst, t, hint);
  const InstDesc& d = insts[g.ii];
  const int64_t local = t - d.tile_begin;
  g.z = (int)(local / d.tiles_per_plane);
  g.y0 = (int)(local - (int64_t)g.z * d.tiles_per_plane) * d.rows;
  g.rows = min(d.rows, d.ny - g.y0);
  return g;
}

// The global rows of segment j of a tile: `first` rows from row ys, then the
// remaining rows from row 0 of the same plane (periodic wrap in y).
struct SegRows {
  const char* plane;  // start of the plane (slot, z) in global memory
  int ys, first;
};

template <typename T, bool ODD>
__device__ __forceinline__ SegRows seg_rows(const InstDesc& d, const TileGeom& g, int j) {
  const int64_t row_bytes = (int64_t)d.nxp * (int64_t)sizeof(T);
  const int64_t slot_bytes = d.pop_stride * (int64_t)sizeof(T);
  const char* base = static_cast<const char*>(d.f);
  SegRows s;
  if (!ODD) {
    s.plane = base + j * slot_bytes + (int64_t)g.z * d.ny * row_bytes;
    s.ys = g.y0;
    s.first = g.rows;
  } else {
    int zs = g.z - c_seg_cz[j];
    zs = zs < 0 ? zs + d.nz : (zs >= d.nz ? zs - d.nz : zs);
    int ys = g.y0 - c_seg_cy[j];
    ys = ys < 0 ? ys + d.ny : (ys >= d.ny ? ys - d.ny : ys);
    s.plane = base + c_seg_opp[j] * slot_bytes + (int64_t)zs * d.ny * row_bytes;
    s.ys = ys;
    s.first = min(g.rows, d.ny - ys);
  }
  return s;
}

// Producer lane j < 19: the bulk load(s) of segment j of a tile.  Without
// padding a segment is one contiguous run (two when a y wrap splits it); with
// padded x-lines every line is copied on its own, live cells only.  Lane 0
// must have posted the tile's expected bytes.
template <typename T, bool ODD>
__device__ __forceinline__ void load_segment(const InstDesc& d, const TileGeom& g, int j, uint32_t buf,
                                             uint32_t bar) {
  const uint32_t row_bytes = (uint32_t)d.nxp * (uint32_t)sizeof(T);
  const uint32_t seg_bytes = row_bytes * (uint32_t)g.rows;
  const SegRows sr = seg_rows<T, ODD>(d, g, j);
  const uint32_t dst = buf + (uint32_t)j * seg_bytes;
  if ((uint32_t)d.row_copy_bytes == row_bytes) {
    bulk_load(dst, sr.plane + (int64_t)sr.ys * row_bytes, (uint32_t)sr.first * row_bytes, bar);
    if (sr.first < g.rows)
      bulk_load(dst + (uint32_t)sr.first * row_bytes, sr.plane, (uint32_t)(g.rows - sr.first) * row_bytes, bar);
  } else {
    for (int r = 0; r < g.rows; ++r) {
      const int y = r < sr.first ? sr.ys + r : r - sr.first;
      bulk_load(dst + (uint32_t)r * row_bytes, sr.plane + (int64_t)y * row_bytes, (uint32_t)d.row_copy_bytes, bar);
    }
  }
}

// Producer lane j < 19: write segment j of a finished tile back to where it was
// loaded from, as this lane's bulk async-group.
template <typename T, bool ODD>
__device__ __forceinline__ void store_segment(const InstDesc& d, const TileGeom& g, int j, uint32_t buf) {
  const uint32_t row_bytes = (uint32_t)d.nxp * (uint32_t)sizeof(T);
  const uint32_t seg_bytes = row_bytes * (uint32_t)g.rows;
  const SegRows sr = seg_rows<T, ODD>(d, g, j);
  const uint32_t src = buf + (uint32_t)j * seg_bytes;
  if ((uint32_t)d.row_copy_bytes == row_bytes) {
    bulk_store(const_cast<char*>(sr.plane) + (int64_t)sr.ys * row_bytes, src, (uint32_t)sr.first * row_bytes);
    if (sr.first < g.rows)
      bulk_store(const_cast<char*>(sr.plane), src + (uint32_t)sr.first * row_bytes,
                 (uint32_t)(g.rows - sr.first) * row_bytes);
  } else {
    for (int r = 0; r < g.rows; ++r) {
      const int y = r < sr.first ? sr.ys + r : r - sr.first;
      bulk_store(const_cast<char*>(sr.plane) + (int64_t)y * row_bytes, src + (uint32_t)r * row_bytes,
                 (uint32_t)d.row_copy_bytes);
    }
  }
  bulk_commit();
}

// Bytes that the bulk loads of one tile deliver.
__device__ __forceinline__ uint32_t tile_bytes_of(const InstDesc& d, const TileGeom& g, int esize) {
  const uint32_t row_bytes = (uint32_t)d.nxp * (uint32_t)esize;
  const uint32_t per_row = (uint32_t)d.row_copy_bytes == row_bytes ? row_bytes : (uint32_t)d.row_copy_bytes;
  return 19u * per_row * (uint32_t)g.rows;
}

template <typename T, bool ODD, int MODE>
__global__ void __launch_bounds__(512, 1)
k_step_tma(const InstDesc* __restrict__ insts, int ninst, int64_t tile_lo, int64_t tile_hi,
           StatsArgs sa, int stages, int tile_bytes, uint32_t* __restrict__ err, long long wait_ns,
           int withhold_first_load) {
  using S = Storage<T>;
  extern __shared__ __align__(128) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nconsumer_warps = (blockDim.x >> 5) - 1;
  const int nct = nconsumer_warps * 32;
  const uint32_t bar_full = smem_addr(smem);                // stages x 8 B
  const uint32_t bar_done = bar_full + 8u * stages;          // stages x 8 B
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 16 * stages);
  const uint32_t buf0 = smem_addr(smem + kBarBytes);
  float* fz_table = reinterpret_cast<float*>(smem + kBarBytes + (size_t)stages * tile_bytes);

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(bar_full + 8u * s, 1u);
      mbar_init(bar_done + 8u * s, (uint32_t)nconsumer_warps);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_async_smem();
  }
  __syncthreads();

  if (warp == nconsumer_warps) {
    // ---------------- producer warp: lane j < 19 issues segment j's bulk copies ----------------
    const int64_t first = tile_lo + blockIdx.x;
    const int64_t stride = gridDim.x;
    const int ntiles = first < tile_hi ? (int)((tile_hi - 1 - first) / stride) + 1 : 0;
    const bool seg_lane = lane < 19;
    // test hook: block 0 leaves the barrier of its first tile without an
    // arrival, so that its consumers' bounded wait runs out
    const bool withheld = withhold_first_load && blockIdx.x == 0;
    int loaded = 0;  // tiles whose loads were issued
    int hint_load = 0, hint_store = 0;
    for (; loaded < ntiles && loaded < stages; ++loaded) {
      if (withheld && loaded == 0) continue;
      const TileGeom g = tile_geom(insts, ninst, first + loaded * stride, hint_load);
      hint_load = g.ii;
      const InstDesc& d = insts[g.ii];
      const uint32_t bar = bar_full + 8u * loaded;
      if (lane == 0) mbar_expect_tx(bar, tile_bytes_of(d, g, (int)sizeof(T)));
      __syncwarp();
      if (seg_lane) load_segment<T, ODD>(d, g, lane, buf0 + (uint32_t)loaded * tile_bytes, bar);
    }
    int stored = 0;
    bool aborted = false;
    for (; stored < ntiles; ++stored) {
      const int s = stored % stages;
      int done_ok = 1;
      if (lane == 0) done_ok = mbar_wait(bar_done + 8u * s, (uint32_t)((stored / stages) & 1), wait_ns) ? 1 : 0;
      done_ok = __shfl_sync(0xffffffffu, done_ok, 0);
      if (!done_ok) {
        if (lane == 0) {
          atomicOr(err, ERR_TIMEOUT);
          *abort_flag = 1;
        }
        aborted = true;
        break;
      }
      const TileGeom g = tile_geom(insts, ninst, first + stored * stride, hint_store);
      hint_store = g.ii;
      const uint32_t buf = buf0 + (uint32_t)s * tile_bytes;
      if (seg_lane) store_segment<T, ODD>(insts[g.ii], g, lane, buf);
      if (loaded < ntiles) {
        const TileGeom gn = tile_geom(insts, ninst, first + loaded * stride, hint_load);
        hint_load = gn.ii;
        const InstDesc& dn = insts[gn.ii];
        const uint32_t bar = bar_full + 8u * s;
        if (lane == 0) mbar_expect_tx(bar, tile_bytes_of(dn, gn, (int)sizeof(T)));
        __syncwarp();
        if (seg_lane) {
          // this lane's segment region is free once its own store has read it
          bulk_wait_read_all();
          load_segment<T, ODD>(dn, gn, lane, buf, bar);
        }
        ++loaded;
      }
    }
    if (aborted && lane == 0) {
      // loads issued but never consumed: wait (bounded) for them to land
      for (int k = stored; k < loaded; ++k) {
        if (withheld && k == 0) continue;
        (void)mbar_wait(bar_full + 8u * (k % stages), (uint32_t)((k / stages) & 1), wait_ns);
      }
    }
    bulk_wait_all();
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
    const TileGeom g = tile_geom(insts, ninst, t, cur < 0 ? 0 : cur);
    const InstDesc& d = insts[g.ii];
    if (g.ii != cur) {
      // new instance: flush its predecessor's statistics, reload Fz(x)
      if (MODE == MODE_STEP_STATS && cur >= 0)
        block_flush(acc, sa.partials + ((int64_t)cur * sa.grid + blockIdx.x) * kNP, nct, 1);
      acc.reset();
      named_sync(2, nct);
      for (int x = ctid; x < d.nx; x += nct) fz_table[x] = d.fz_of_x[x] + d.fconst[2];
      named_sync(2, nct);
      cur = g.ii;
    }
    const int s = k % stages;
    if (ok) {
      if (*abort_flag) {
        ok = false;
      } else if (!mbar_wait(bar_full + 8u * s, (uint32_t)((k / stages) & 1), wait_ns)) {
        atomicOr(err, ERR_TIMEOUT);
        *abort_flag = 1;
        ok = false;
      }
    }
    if (!ok) continue;  // keep the named-barrier schedule of the other consumers
    const int nx = d.nx, nxp = d.nxp;
    T* sbuf = reinterpret_cast<T*>(smem + kBarBytes + (size_t)s * tile_bytes);
    const int seg = g.rows * nxp;
    const int ncell = g.rows * nx;
    const float Fy = d.fy_of_z[g.z] + d.fconst[1];
    const float nu0 = d.nu0, s_nu0 = d.s_nu0, C = d.C;
    const int dr = nct / nx, dx = nct - dr * nx;
    int r = ctid / nx, x = ctid - r * nx;
    for (int c = ctid; c < ncell; c += nct) {
      const int xm = wrap_dec(x, nx), xp = wrap_inc(x, nx);
      T* row = sbuf + r * nxp;
      float f[19];
#pragma unroll
      for (int a = 0; a < 19; ++a) {
        const int xs = ODD ? (cx(a) > 0 ? xm : (cx(a) < 0 ? xp : x)) : x;
        f[a] = S::cvt(row[a * seg + xs]);
      }
      const float Fx = d.fx_of_y[g.y0 + r] + d.fconst[0];
      const float Fz = fz_table[x];
      CellDiag cd;
      mrt_collide(f, Fx, Fy, Fz, nu0, s_nu0, C, cd, d.strain_mode);
#pragma unroll
      for (int a = 0; a < 19; ++a) {
        const int xd = ODD ? (cx(a) > 0 ? xp : (cx(a) < 0 ? xm : x)) : x;
        row[opp(a) * seg + xd] = S::pack(f[a]);
      }
      if (MODE == MODE_STEP_STATS) acc.add(cd, Fx, Fy, Fz, C);
      x += dx;
      r += dr;
      if (x >= nx) {
        x -= nx;
        r += 1;
      }
    }
    if (MODE == MODE_STEP_STATS) acc.fold();
    // hand the tile back: make this warp's shared-memory writes visible to the
    // TMA engine, then one arrival per warp
    fence_async_smem();
    __syncwarp();
    if (lane == 0) mbar_arrive(bar_done + 8u * s);
  }
  if (MODE == MODE_STEP_STATS && cur >= 0)
    block_flush(acc, sa.partials + ((int64_t)cur * sa.grid + blockIdx.x) * kNP, nct, 1);
}

template <typename T, bool ODD, int MODE>
cudaError_t launch_tma_t(const LaunchArgs& la, cudaStream_t st) {
  (void)cudaGetLastError();  // errors of earlier calls were reported by their return codes
  k_step_tma<T, ODD, MODE><<<la.grid, la.threads, la.smem_bytes, st>>>(
      la.insts, la.ninst, la.tile_lo, la.tile_hi, la.sa, la.stages, la.tile_bytes_max, la.err,
      la.wait_ns, la.withhold_first_load);
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

int tma_smem_bytes(int stages, int tile_bytes, int max_nx) {
  return kBarBytes + stages * tile_bytes + (max_nx * 4 + 15) / 16 * 16;
}

cudaError_t launch_step_tma(const LaunchArgs& la, cudaStream_t st) {
  if (la.threads < 64 || la.threads > 512 || (la.threads & 31) || la.stages < 1 || la.stages > 6 ||
      (la.tile_bytes_max & 15) || la.wait_ns <= 0)
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
