// TMA bulk-copy stream + collide kernel (AA pattern, one population array).
//
// A tile is `rows` consecutive x-lines of one z-plane.  In the AA pattern the
// locations a tile reads are exactly the locations it writes, and they form
// 19 segments of rows x-lines (one per population slot; contiguous in the
// population-major layout, x-line by x-line in the row-interleaved one):
//   even step: slot a of the tile's own rows;
//   odd step:  slot opp(a) of rows y - cy_a of plane z - cz_a (a periodic wrap
//              in y splits a segment in two; the x wrap is resolved in shared
//              memory because whole lines are loaded).
// In shared memory segment a of a stage starts at a x SLOT bytes, SLOT a
// compile-time slot size (3840 B with three stages, 5760 B with two: 19 slots
// per stage, the stages fill the 220 KB budget), so each of a cell's 19
// shared-memory accesses is one base register plus an immediate offset.  Tiles
// whose rows do not fit a slot use the runtime stride rows x nxp (SLOT = 0).
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
// it reloads its segment as soon as its own store has read it; in the odd steps
// of one-x-line runtime-stride tiles of the row-interleaved array lane g < 9
// moves a whole slot group instead, see grouped_copies).  Consumers read
// the 19 populations of a cell from shared memory, collide in FP32 registers
// (lbm_device.cuh) and write the 19 results back in place; the populations in
// global memory are moved by the TMA engine only.  Producer and consumers walk
// the block's tiles with the same incremental tile walker.  Every mbarrier
// wait is bounded by the global timer: on expiry the block records
// ERR_TIMEOUT, stops issuing, waits (bounded) for its loads in flight and for
// its stores, and returns.
//
// MODE_DIAG is the read-only statistics pass over the current state: the same
// loads and collision arithmetic, no stores (a stage is reloaded as soon as
// its consumers are done), the FP64 block partials of the step with
// statistics, and the per-cell outputs (velocity, theta slices, theta
// histogram: a window of bins that fits the room the launch reserves behind
// the stages in shared memory, the rest in global counts).
#include <cuda_runtime.h>

#include <algorithm>
#include <utility>

#include "lbm_device.cuh"
#include "lbm_kernels.h"
#include "lbm_reduce.cuh"

namespace lbm {

namespace {

constexpr int kBarBytes = 128;  // mbarriers + abort flag
// Bound of the drain after an abort, in units of the launch's wait_ns.
constexpr int kDrainRounds = 4;

// Per population j: the slot read by the odd step (opp j) and the row shift
// (cy_j, cz_j), for the producer lanes (one lane per segment).
__constant__ int8_t c_seg_opp[19] = {1, 0, 3, 2, 5, 4, 7, 6, 9, 8, 11, 10, 13, 12, 15, 14, 17, 16, 18};
__constant__ int8_t c_seg_cy[19] = {0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 1, -1, 1, -1, 0, 0, 0, 0, 0};
__constant__ int8_t c_seg_cz[19] = {0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1, 0};
// gpos(a) (lbm_device.cuh) for the producer lanes
__constant__ int8_t c_gpos[19] = {0, 1, 15, 4, 11, 8, 16, 5, 6, 17, 18, 3, 14, 7, 12, 9, 10, 13, 2};
// The 9 slot groups of a cell row in position order: first position, length
// and the slots' own (cy, cz) -- an odd-step tile at row (y, z) reads group g
// whole from cell row (y + cy_g, z + cz_g).
__constant__ int8_t c_grp_start[9] = {0, 3, 4, 7, 8, 11, 14, 15, 18};
__constant__ int8_t c_grp_len[9] = {3, 1, 3, 1, 3, 3, 1, 3, 1};
__constant__ int8_t c_grp_cy[9] = {0, -1, -1, -1, 0, 0, 1, 1, 1};
__constant__ int8_t c_grp_cz[9] = {0, -1, 0, 1, -1, 1, -1, 0, 1};

// Shared-memory position of segment j of a tile (what its cells read as f_j).
// SLOT = kSlotGrouped (runtime stride, row-interleaved array): the grouped
// position of the slot it is copied from, so that a slot group of a cell row
// lands in one piece; otherwise position j.
template <int SLOT>
__host__ __device__ constexpr int spos(int j, bool odd) {
  return SLOT == kSlotGrouped ? gpos(odd ? opp(j) : j) : j;
}
// Bytes between segment positions of a stage: the compile-time slot, or the
// runtime stride of `rows` x-lines.
template <int SLOT>
__host__ __device__ constexpr bool slotted() { return SLOT > 0; }

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

// One test of the phase; a thread whose phase has not completed is suspended
// in hardware (no issue slots) until it completes or kSuspendNs pass.
constexpr uint32_t kSuspendNs = 100000;

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  if (kSuspendNs == 0) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(kSuspendNs)
        : "memory");
  }
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

// Walks a block's tiles t0, t0 + stride, ... (tiles are numbered instance by
// instance, plane by plane, tile row by tile row), keeping the instance and
// the (plane, tile row) coordinates up to date incrementally: divisions happen
// only when the walk enters another instance.
struct TileWalker {
  int64_t t;       // current global tile
  int64_t end;     // one past the last tile of instance ii
  int ii;          // instance of tile t
  int tpp;         // tiles per plane of instance ii
  int rows, ny;    // tile rows and y extent of instance ii
  int z, ty;       // plane and tile row of tile t
  int sz, sy;      // stride = sz planes + sy tile rows
};

__device__ __forceinline__ void walker_enter(TileWalker& w, const InstDesc* __restrict__ insts, int ninst,
                                             int64_t stride) {
  w.ii = find_instance(insts, ninst, w.t, w.ii);
  const InstDesc& d = insts[w.ii];
  w.end = d.tile_end;
  w.tpp = d.tiles_per_plane;
  w.rows = d.rows;
  w.ny = d.ny;
  const int64_t local = w.t - d.tile_begin;
  w.z = (int)(local / w.tpp);
  w.ty = (int)(local - (int64_t)w.z * w.tpp);
  w.sz = (int)(stride / w.tpp);
  w.sy = (int)(stride - (int64_t)w.sz * w.tpp);
}

__device__ __forceinline__ TileWalker walker_start(const InstDesc* __restrict__ insts, int ninst, int64_t t0,
                                                   int64_t stride) {
  TileWalker w;
  w.t = t0;
  w.ii = 0;
  walker_enter(w, insts, ninst, stride);
  return w;
}

// Step to the next tile of the block; true when it lies in another instance.
__device__ __forceinline__ bool walker_next(TileWalker& w, const InstDesc* __restrict__ insts, int ninst,
                                            int64_t stride, int64_t tile_hi) {
  w.t += stride;
  if (w.t >= w.end) {
    if (w.t < tile_hi) walker_enter(w, insts, ninst, stride);
    return true;
  }
  w.z += w.sz;
  w.ty += w.sy;
  if (w.ty >= w.tpp) {
    w.ty -= w.tpp;
    w.z += 1;
  }
  return false;
}

__device__ __forceinline__ TileGeom walker_geom(const TileWalker& w) {
  const int y0 = w.ty * w.rows;
  return TileGeom{w.ii, w.z, y0, min(w.rows, w.ny - y0)};
}

// The global rows of segment j of a tile: `first` rows from row ys, then the
// remaining rows from row 0 of the same plane (periodic wrap in y).
struct SegRows {
  const char* plane;  // row 0 of the slot's plane z in global memory
  int64_t step;       // bytes from one y row of the slot to the next
  int ys, first;
};

// The per-instance fields the producer's copies need, kept in registers (the
// producer is on the critical path of every stage turnaround: no descriptor
// loads per tile).
struct SegInst {
  const void* f;
  int64_t slot_stride, plane_stride, row_stride;
  int32_t nxp, ny, nz, rows, row_copy_bytes, slot_grouped;
  int64_t f_elems;  // checked build: storage elements of the array
};

__device__ __forceinline__ SegInst seg_inst(const InstDesc& d) {
  return SegInst{d.f, d.slot_stride, d.plane_stride, d.row_stride, d.nxp, d.ny, d.nz, d.rows,
                 d.row_copy_bytes, d.slot_grouped, d.f_elems};
}

// Checked build: a bulk copy of `bytes` between global address g and shared
// address s stays inside the instance's array and inside the stage [buf,
// buf + stage_bytes).  Always true in the normal build.
template <typename T>
__device__ __forceinline__ bool copy_ok(const SegInst& d, const void* g, uint32_t s, uint32_t bytes, uint32_t buf,
                                        uint32_t stage_bytes) {
  if constexpr (!kBoundsCheck) return true;
  return in_bounds(range_in(g, bytes, d.f, d.f_elems * (int64_t)sizeof(T)) && s >= buf &&
                   (uint64_t)s + bytes <= (uint64_t)buf + stage_bytes);
}

template <typename T, bool ODD>
__device__ __forceinline__ SegRows seg_rows(const SegInst& d, const TileGeom& g, int j) {
  const int64_t es = (int64_t)sizeof(T);
  const char* base = static_cast<const char*>(d.f);
  SegRows s;
  s.step = d.row_stride * es;
  const int slot = ODD ? c_seg_opp[j] : j;
  const int64_t spos_g = d.slot_grouped ? c_gpos[slot] : slot;  // its position in global memory
  if (!ODD) {
    s.plane = base + (spos_g * d.slot_stride + g.z * d.plane_stride) * es;
    s.ys = g.y0;
    s.first = g.rows;
  } else {
    int zs = g.z - c_seg_cz[j];
    zs = zs < 0 ? zs + d.nz : (zs >= d.nz ? zs - d.nz : zs);
    int ys = g.y0 - c_seg_cy[j];
    ys = ys < 0 ? ys + d.ny : (ys >= d.ny ? ys - d.ny : ys);
    s.plane = base + (spos_g * d.slot_stride + zs * d.plane_stride) * es;
    s.ys = ys;
    s.first = min(g.rows, d.ny - ys);
  }
  return s;
}

// Producer lane j < 19: the bulk load(s) of segment j of a tile.  In the
// population-major layout without padding a segment is one contiguous run (two
// when a y wrap splits it); otherwise (padded x-lines, or the row-interleaved
// layout, where the rows of a slot are 19 x-lines apart) every x-line is copied
// on its own, live cells only.  Lane 0 must have posted the tile's expected
// bytes.
template <typename T, bool ODD, int SLOT>
__device__ __forceinline__ void load_segment(const SegInst& d, const TileGeom& g, int j, uint32_t buf,
                                             uint32_t bar, uint32_t stage_bytes) {
  const uint32_t row_bytes = (uint32_t)d.nxp * (uint32_t)sizeof(T);
  const uint32_t seg_bytes = slotted<SLOT>() ? (uint32_t)SLOT : row_bytes * (uint32_t)d.rows;
  const SegRows sr = seg_rows<T, ODD>(d, g, j);
  const uint32_t pos = SLOT == kSlotGrouped ? (uint32_t)c_gpos[ODD ? c_seg_opp[j] : j] : (uint32_t)j;  // spos
  const uint32_t dst = buf + pos * seg_bytes;
  if ((uint32_t)d.row_copy_bytes == row_bytes && sr.step == (int64_t)row_bytes) {
    const char* src = sr.plane + (int64_t)sr.ys * row_bytes;
    if (copy_ok<T>(d, src, dst, (uint32_t)sr.first * row_bytes, buf, stage_bytes))
      bulk_load(dst, src, (uint32_t)sr.first * row_bytes, bar);
    if (sr.first < g.rows && copy_ok<T>(d, sr.plane, dst + (uint32_t)sr.first * row_bytes,
                                        (uint32_t)(g.rows - sr.first) * row_bytes, buf, stage_bytes))
      bulk_load(dst + (uint32_t)sr.first * row_bytes, sr.plane, (uint32_t)(g.rows - sr.first) * row_bytes, bar);
  } else {
    for (int r = 0; r < g.rows; ++r) {
      const int y = r < sr.first ? sr.ys + r : r - sr.first;
      const char* src = sr.plane + (int64_t)y * sr.step;
      if (copy_ok<T>(d, src, dst + (uint32_t)r * row_bytes, (uint32_t)d.row_copy_bytes, buf, stage_bytes))
        bulk_load(dst + (uint32_t)r * row_bytes, src, (uint32_t)d.row_copy_bytes, bar);
    }
  }
}

// Producer lane j < 19: write segment j of a finished tile back to where it was
// loaded from, as this lane's bulk async-group.
template <typename T, bool ODD, int SLOT>
__device__ __forceinline__ void store_segment(const SegInst& d, const TileGeom& g, int j, uint32_t buf,
                                              uint32_t stage_bytes) {
  const uint32_t row_bytes = (uint32_t)d.nxp * (uint32_t)sizeof(T);
  const uint32_t seg_bytes = slotted<SLOT>() ? (uint32_t)SLOT : row_bytes * (uint32_t)d.rows;
  const SegRows sr = seg_rows<T, ODD>(d, g, j);
  const uint32_t pos = SLOT == kSlotGrouped ? (uint32_t)c_gpos[ODD ? c_seg_opp[j] : j] : (uint32_t)j;  // spos
  const uint32_t src = buf + pos * seg_bytes;
  if ((uint32_t)d.row_copy_bytes == row_bytes && sr.step == (int64_t)row_bytes) {
    char* dst = const_cast<char*>(sr.plane) + (int64_t)sr.ys * row_bytes;
    if (copy_ok<T>(d, dst, src, (uint32_t)sr.first * row_bytes, buf, stage_bytes))
      bulk_store(dst, src, (uint32_t)sr.first * row_bytes);
    if (sr.first < g.rows && copy_ok<T>(d, sr.plane, src + (uint32_t)sr.first * row_bytes,
                                        (uint32_t)(g.rows - sr.first) * row_bytes, buf, stage_bytes))
      bulk_store(const_cast<char*>(sr.plane), src + (uint32_t)sr.first * row_bytes,
                 (uint32_t)(g.rows - sr.first) * row_bytes);
  } else {
    for (int r = 0; r < g.rows; ++r) {
      const int y = r < sr.first ? sr.ys + r : r - sr.first;
      char* dst = const_cast<char*>(sr.plane) + (int64_t)y * sr.step;
      if (copy_ok<T>(d, dst, src + (uint32_t)r * row_bytes, (uint32_t)d.row_copy_bytes, buf, stage_bytes))
        bulk_store(dst, src + (uint32_t)r * row_bytes, (uint32_t)d.row_copy_bytes);
    }
  }
  bulk_commit();
}

// Odd steps of the row-interleaved layout with one-x-line tiles in the runtime
// stride (shared-memory positions one x-line apart, like the global ones):
// the tile's 19 segments are the 9 slot groups of its 9 neighbouring cell
// rows, each adjacent in global and in shared memory, so producer lane g < 9
// moves group g in one piece.
template <typename T, bool ODD, int SLOT>
__device__ __forceinline__ bool grouped_copies(const SegInst& d) {
  return ODD && SLOT == kSlotGrouped && d.slot_grouped && d.rows == 1 &&
         (uint32_t)d.row_copy_bytes == (uint32_t)d.nxp * (uint32_t)sizeof(T);
}

template <typename T>
__device__ __forceinline__ const char* group_src(const SegInst& d, const TileGeom& g, int k) {
  int zs = g.z + c_grp_cz[k];
  zs = zs < 0 ? zs + d.nz : (zs >= d.nz ? zs - d.nz : zs);
  int ys = g.y0 + c_grp_cy[k];
  ys = ys < 0 ? ys + d.ny : (ys >= d.ny ? ys - d.ny : ys);
  return static_cast<const char*>(d.f) +
         (c_grp_start[k] * d.slot_stride + zs * d.plane_stride + ys * d.row_stride) * (int64_t)sizeof(T);
}

template <typename T>
__device__ __forceinline__ void load_group(const SegInst& d, const TileGeom& g, int k, uint32_t buf, uint32_t bar,
                                           uint32_t stage_bytes) {
  const uint32_t row_bytes = (uint32_t)d.nxp * (uint32_t)sizeof(T);
  const char* src = group_src<T>(d, g, k);
  const uint32_t dst = buf + (uint32_t)c_grp_start[k] * row_bytes, bytes = (uint32_t)c_grp_len[k] * row_bytes;
  if (copy_ok<T>(d, src, dst, bytes, buf, stage_bytes)) bulk_load(dst, src, bytes, bar);
}

template <typename T>
__device__ __forceinline__ void store_group(const SegInst& d, const TileGeom& g, int k, uint32_t buf,
                                            uint32_t stage_bytes) {
  const uint32_t row_bytes = (uint32_t)d.nxp * (uint32_t)sizeof(T);
  char* dst = const_cast<char*>(group_src<T>(d, g, k));
  const uint32_t src = buf + (uint32_t)c_grp_start[k] * row_bytes, bytes = (uint32_t)c_grp_len[k] * row_bytes;
  if (copy_ok<T>(d, dst, src, bytes, buf, stage_bytes)) bulk_store(dst, src, bytes);
  bulk_commit();
}

// Producer lane `lane`: its share of the loads / stores of a tile (a slot
// group or a segment, or nothing).
template <typename T, bool ODD, int SLOT>
__device__ __forceinline__ void tile_load(const SegInst& d, const TileGeom& g, int lane, uint32_t buf,
                                          uint32_t bar, uint32_t stage_bytes) {
  if (grouped_copies<T, ODD, SLOT>(d)) {
    if (lane < 9) load_group<T>(d, g, lane, buf, bar, stage_bytes);
  } else if (lane < 19) {
    load_segment<T, ODD, SLOT>(d, g, lane, buf, bar, stage_bytes);
  }
}

template <typename T, bool ODD, int SLOT>
__device__ __forceinline__ void tile_store(const SegInst& d, const TileGeom& g, int lane, uint32_t buf,
                                           uint32_t stage_bytes) {
  if (grouped_copies<T, ODD, SLOT>(d)) {
    if (lane < 9) store_group<T>(d, g, lane, buf, stage_bytes);
  } else if (lane < 19) {
    store_segment<T, ODD, SLOT>(d, g, lane, buf, stage_bytes);
  }
}

// Bytes that the bulk loads of one tile deliver.
__device__ __forceinline__ uint32_t tile_bytes_of(const SegInst& d, const TileGeom& g, int esize) {
  const uint32_t row_bytes = (uint32_t)d.nxp * (uint32_t)esize;
  const uint32_t per_row = (uint32_t)d.row_copy_bytes == row_bytes ? row_bytes : (uint32_t)d.row_copy_bytes;
  return 19u * per_row * (uint32_t)g.rows;
}

// Shared-memory accesses of the compile-time slot variants with the slot
// offset in the instruction: one address register per distinct x position of
// a cell (x, and x -+ 1 in odd steps), the population's slot offset as an
// immediate (the compiler did not fold these offsets on its own: ~40 integer
// instructions per cell went to addressing).  Volatile asm keeps them in
// program order with the barrier waits and fences around them.
template <typename T> struct SmemIO;
template <> struct SmemIO<float> {
  template <int OFF> static __device__ __forceinline__ float ld(uint32_t a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(a), "n"(OFF));
    return v;
  }
  template <int OFF> static __device__ __forceinline__ void st(uint32_t a, float v) {
    asm volatile("st.shared.f32 [%0+%1], %2;" ::"r"(a), "n"(OFF), "f"(v) : "memory");
  }
};
template <> struct SmemIO<__half> {
  template <int OFF> static __device__ __forceinline__ float ld(uint32_t a) {
    unsigned short h;
    asm volatile("ld.shared.b16 %0, [%1+%2];" : "=h"(h) : "r"(a), "n"(OFF));
    return __half2float(__ushort_as_half(h));
  }
  template <int OFF> static __device__ __forceinline__ void st(uint32_t a, float v) {
    asm volatile("st.shared.b16 [%0+%1], %2;" ::"r"(a), "n"(OFF), "h"(__half_as_ushort(__float2half_rn(v)))
                 : "memory");
  }
};
template <> struct SmemIO<__nv_bfloat16> {
  template <int OFF> static __device__ __forceinline__ float ld(uint32_t a) {
    unsigned short h;
    asm volatile("ld.shared.b16 %0, [%1+%2];" : "=h"(h) : "r"(a), "n"(OFF));
    return __bfloat162float(__ushort_as_bfloat16(h));
  }
  template <int OFF> static __device__ __forceinline__ void st(uint32_t a, float v) {
    asm volatile("st.shared.b16 [%0+%1], %2;" ::"r"(a), "n"(OFF),
                 "h"(__bfloat16_as_ushort(__float2bfloat16_rn(v)))
                 : "memory");
  }
};

// f_A of a cell: segment spos(A) at x - [odd] cx_A (address bm for x - 1, bp
// for x + 1, b0 for x).
template <typename T, bool ODD, int SLOT, int A>
__device__ __forceinline__ float ld_pop(uint32_t b0, uint32_t bm, uint32_t bp) {
  constexpr int kOff = spos<SLOT>(A, ODD) * SLOT;
  const uint32_t b = ODD ? (cx(A) > 0 ? bm : (cx(A) < 0 ? bp : b0)) : b0;
  return SmemIO<T>::template ld<kOff>(b);
}
template <typename T, bool ODD, int SLOT, int... A>
__device__ __forceinline__ void ld_pops(float (&f)[19], uint32_t b0, uint32_t bm, uint32_t bp,
                                        std::integer_sequence<int, A...>) {
  ((f[A] = ld_pop<T, ODD, SLOT, A>(b0, bm, bp)), ...);
}
// f*_A of a cell into segment spos(opp A) at x + [odd] cx_A.
template <typename T, bool ODD, int SLOT, int A>
__device__ __forceinline__ void st_pop(const float (&f)[19], uint32_t b0, uint32_t bm, uint32_t bp) {
  constexpr int kOff = spos<SLOT>(opp(A), ODD) * SLOT;
  const uint32_t b = ODD ? (cx(A) > 0 ? bp : (cx(A) < 0 ? bm : b0)) : b0;
  SmemIO<T>::template st<kOff>(b, f[A]);
}
template <typename T, bool ODD, int SLOT, int... A>
__device__ __forceinline__ void st_pops(const float (&f)[19], uint32_t b0, uint32_t bm, uint32_t bp,
                                        std::integer_sequence<int, A...>) {
  (st_pop<T, ODD, SLOT, A>(f, b0, bm, bp), ...);
}

// Per-instance constants of a consumer thread's cell loop.
struct CellLoop {
  int nx, nxp;
  int stage_elems;       // checked build: values of one stage
  int ny;                // checked build: rows of the Fx table
  int seg;               // population stride in shared memory (values)
  int dr, dx;            // a pass of nct cells advances dr rows and dx cells
  int r0, x0;            // the thread's first cell of a tile
  float fx_const;        // uniform part of Fx
  float nu0, s_nu0, C;
};

// Per-cell outputs of the read-only statistics pass (MODE_DIAG) for a tile:
// the outputs, the tile's first row and plane, the extents, the histogram
// (bins [hist_lo, hist_lo + hist_win) in shared memory, the rest in global
// counts).
struct DiagTile {
  DiagOut o;
  int y0, z, ny, nz;
  uint32_t* hist_sm;
  int hist_lo, hist_win;
  uint32_t* hist_gl;
};

// Consumer thread of nct: collide cells r0 nx + x0, + nct, ... of a tile of
// ncell cells in place in shared memory (the AA read and write positions
// coincide, see the file comment).  fx: Fx(y) from the tile's first row; SMODE:
// the strain evaluation (lbm_params.strain_mode).  MODE_DIAG leaves the tile
// unchanged and writes the per-cell outputs instead.
template <typename T, bool ODD, int MODE, int SMODE, int SLOT>
__device__ __forceinline__ void collide_tile(const CellLoop& cl, int ncell, const float* __restrict__ fx,
                                             const float Fy, T* __restrict__ sbuf,
                                             const float* __restrict__ fz_table, int nct, Acc& acc,
                                             const DiagTile& dt, HistRun& run) {
  using S = Storage<T>;
  // compile-time slots: immediate offsets (SmemIO); otherwise indexed accesses
  constexpr bool kImm = slotted<SLOT>() && !kBoundsCheck;
  using Pops = std::make_integer_sequence<int, 19>;
  const int nx = cl.nx, seg = cl.seg;
  const uint32_t sbase = smem_addr(sbuf);
  int r = cl.r0, x = cl.x0;
  for (int c = r * nx + x; c < ncell; c += nct) {
    const int xm = wrap_dec(x, nx), xp = wrap_inc(x, nx);
    T* row = sbuf + r * cl.nxp;
    const uint32_t b0 = sbase + (uint32_t)(r * cl.nxp + x) * (uint32_t)sizeof(T);
    const uint32_t bm = b0 + (uint32_t)((xm - x) * (int)sizeof(T));
    const uint32_t bp = b0 + (uint32_t)((xp - x) * (int)sizeof(T));
    float f[19];
    if constexpr (kImm) {
      ld_pops<T, ODD, SLOT>(f, b0, bm, bp, Pops{});
    } else {
#pragma unroll
      for (int a = 0; a < 19; ++a) {
        const int xs = ODD ? (cx(a) > 0 ? xm : (cx(a) < 0 ? xp : x)) : x;
        if constexpr (kBoundsCheck) {
          const int e = r * cl.nxp + spos<SLOT>(a, ODD) * seg + xs;
          f[a] = in_bounds(e >= 0 && e < cl.stage_elems) ? S::cvt(sbuf[e]) : 0.f;
        } else {
          f[a] = S::cvt(row[spos<SLOT>(a, ODD) * seg + xs]);
        }
      }
    }
    float Fx, Fz;
    if constexpr (kBoundsCheck) {
      Fx = (in_bounds(dt.y0 + r >= 0 && dt.y0 + r < cl.ny) ? __ldg(fx + r) : 0.f) + cl.fx_const;
      Fz = in_bounds(x >= 0 && x < nx) ? fz_table[x] : 0.f;
    } else {
      Fx = __ldg(fx + r) + cl.fx_const;
      Fz = fz_table[x];
    }
    CellDiag cd;
    mrt_collide(f, Fx, Fy, Fz, cl.nu0, cl.s_nu0, cl.C, cd, SMODE);
    if (MODE != MODE_DIAG) {
      if constexpr (kImm) {
        st_pops<T, ODD, SLOT>(f, b0, bm, bp, Pops{});
      } else {
#pragma unroll
        for (int a = 0; a < 19; ++a) {
          const int xd = ODD ? (cx(a) > 0 ? xp : (cx(a) < 0 ? xm : x)) : x;
          if constexpr (kBoundsCheck) {
            const int e = r * cl.nxp + spos<SLOT>(opp(a), ODD) * seg + xd;
            if (in_bounds(e >= 0 && e < cl.stage_elems)) sbuf[e] = S::pack(f[a]);
          } else {
            row[spos<SLOT>(opp(a), ODD) * seg + xd] = S::pack(f[a]);
          }
        }
      }
    }
    if (MODE != MODE_STEP) acc.add(cd, Fx, Fy, Fz, cl.C);
    if (MODE == MODE_DIAG) diag_write(dt.o, cd, x, dt.y0 + r, dt.z, nx, dt.ny, dt.nz, dt.hist_sm, dt.hist_lo, dt.hist_win, dt.hist_gl, run);
    x += cl.dx;
    r += cl.dr;
    if (x >= nx) {
      x -= nx;
      r += 1;
    }
  }
}

template <typename T, bool ODD, int MODE, int SLOT>
__global__ void __launch_bounds__(512, 1)
k_step_tma(const InstDesc* __restrict__ insts, int ninst, int64_t tile_lo, int64_t tile_hi,
           StatsArgs sa, int stages, int tile_bytes, uint32_t* __restrict__ err, long long wait_ns,
           int withhold_first_load, DiagOut dout, int hist_smem, int hist_lo, int hist_win) {
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
    // ---------------- producer warp: lane j < 19 issues segment j's bulk copies (lane g < 9
    // slot group g's in the odd steps of grouped runtime-stride tiles) ----------------
    const int64_t first = tile_lo + blockIdx.x;
    const int64_t stride = gridDim.x;
    const int ntiles = first < tile_hi ? (int)((tile_hi - 1 - first) / stride) + 1 : 0;
    // test hook: block 0 leaves the barrier of its first tile without an
    // arrival, so that its consumers' bounded wait runs out
    const bool withheld = withhold_first_load && blockIdx.x == 0;
    int loaded = 0;  // tiles whose loads were issued
    if (ntiles == 0) return;
    TileWalker wl = walker_start(insts, ninst, first, stride);  // next tile to load
    TileWalker ws = wl;                                         // next tile to store
    SegInst sil = seg_inst(insts[wl.ii]), sis = sil;            // their instances' fields
    int sil_ii = wl.ii, sis_ii = wl.ii;
    for (; loaded < ntiles && loaded < stages; ++loaded) {
      if (!(withheld && loaded == 0)) {
        const TileGeom g = walker_geom(wl);
        if (g.ii != sil_ii) {
          sil = seg_inst(insts[g.ii]);
          sil_ii = g.ii;
        }
        const SegInst& d = sil;
        const uint32_t bar = bar_full + 8u * loaded;
        if (lane == 0) mbar_expect_tx(bar, tile_bytes_of(d, g, (int)sizeof(T)));
        __syncwarp();
        tile_load<T, ODD, SLOT>(d, g, lane, buf0 + (uint32_t)loaded * tile_bytes, bar, (uint32_t)tile_bytes);
      }
      walker_next(wl, insts, ninst, stride, tile_hi);
    }
    int stored = 0;
    bool aborted = false;
    int s = 0;           // stage of tile `stored`
    uint32_t phase = 0;  // parity of its barriers' current phase
    for (; stored < ntiles; ++stored) {
      int done_ok = 1;
      if (lane == 0) done_ok = mbar_wait(bar_done + 8u * s, phase, wait_ns) ? 1 : 0;
      done_ok = __shfl_sync(0xffffffffu, done_ok, 0);
      if (!done_ok) {
        if (lane == 0) {
          atomicOr(err, ERR_TIMEOUT);
          *abort_flag = 1;
        }
        aborted = true;
        break;
      }
      const TileGeom g = walker_geom(ws);
      const uint32_t buf = buf0 + (uint32_t)s * tile_bytes;
      if (g.ii != sis_ii) {
        sis = seg_inst(insts[g.ii]);
        sis_ii = g.ii;
      }
      if (MODE != MODE_DIAG) tile_store<T, ODD, SLOT>(sis, g, lane, buf, (uint32_t)tile_bytes);
      walker_next(ws, insts, ninst, stride, tile_hi);
      if (loaded < ntiles) {
        const TileGeom gn = walker_geom(wl);
        walker_next(wl, insts, ninst, stride, tile_hi);
        if (gn.ii != sil_ii) {
          sil = seg_inst(insts[gn.ii]);
          sil_ii = gn.ii;
        }
        const SegInst& dn = sil;
        const uint32_t bar = bar_full + 8u * s;
        if (lane == 0) mbar_expect_tx(bar, tile_bytes_of(dn, gn, (int)sizeof(T)));
        __syncwarp();
        // a lane's region is free once its own store has read it; when the
        // next tile belongs to another instance the regions of the lanes may
        // differ (tile rows, slot groups), so then every lane's store must
        // have read the stage first
        bulk_wait_read_all();
        if (gn.ii != g.ii) __syncwarp();
        tile_load<T, ODD, SLOT>(dn, gn, lane, buf, bar, (uint32_t)tile_bytes);
        ++loaded;
      }
      if (++s == stages) {
        s = 0;
        phase ^= 1u;
      }
    }
    if (aborted && lane == 0) {
      // loads issued but never consumed target this block's shared memory and
      // must land before it leaves: wait for each in rounds of wait_ns, at most
      // kDrainRounds of them; one still missing after that sets ERR_DRAIN
      for (int k = stored; k < loaded; ++k) {
        if (withheld && k == 0) continue;
        bool landed = false;
        for (int round = 0; round < kDrainRounds && !landed; ++round)
          landed = mbar_wait(bar_full + 8u * (k % stages), (uint32_t)((k / stages) & 1), wait_ns);
        if (!landed) atomicOr(err, ERR_DRAIN);
      }
    }
    bulk_wait_all();
    return;
  }

  // ---------------- consumer warps ----------------
  const int ctid = threadIdx.x;
  const int64_t first = tile_lo + blockIdx.x;
  const int64_t stride = gridDim.x;
  if (first >= tile_hi) return;
  // MODE_DIAG: theta histogram bins [hist_lo, hist_lo + hist_win) in shared
  // memory when the launch reserved room at byte hist_smem, the others
  // straight into the global counts
  uint32_t* hist_sm = nullptr;
  uint32_t* hist_gl = nullptr;
  int lo = 0, win = 0;
  if (MODE == MODE_DIAG && dout.hist) {
    if (hist_smem > 0) {
      hist_sm = reinterpret_cast<uint32_t*>(smem + hist_smem);
      lo = min(max(hist_lo, 0), dout.hist_bins);
      win = min(hist_win, dout.hist_bins + 1 - lo);
      for (int i = ctid; i < win; i += nct) hist_sm[i] = 0u;
    }
    if (lo > 0 || win <= dout.hist_bins) hist_gl = dout.hist;
  }
  Acc acc;
  acc.reset();
  HistRun run;
  int cur = -1;
  bool ok = true;
  CellLoop cl{};
  int smode = 0;
  const float* fy_of_z = nullptr;
  float fy_const = 0.f;
  int s = 0;
  uint32_t phase = 0;
  for (TileWalker w = walker_start(insts, ninst, first, stride); w.t < tile_hi;
       walker_next(w, insts, ninst, stride, tile_hi)) {
    if (w.ii != cur) {
      // new instance: flush its predecessor's statistics, reload Fz(x) and the
      // per-instance constants
      if (MODE != MODE_STEP && cur >= 0)
        block_flush(acc, sa.partials + ((int64_t)cur * sa.grid + blockIdx.x) * kNP, nct, 1);
      acc.reset();
      const InstDesc& d = insts[w.ii];
      named_sync(2, nct);
      for (int x = ctid; x < d.nx; x += nct) fz_table[x] = d.fz_of_x[x] + d.fconst[2];
      named_sync(2, nct);
      cur = w.ii;
      cl.nx = d.nx;
      cl.nxp = d.nxp;
      cl.ny = d.ny;
      cl.stage_elems = tile_bytes / (int)sizeof(T);
      cl.seg = slotted<SLOT>() ? SLOT / (int)sizeof(T) : d.rows * d.nxp;
      cl.dr = nct / d.nx;
      cl.dx = nct - cl.dr * d.nx;
      cl.r0 = ctid / d.nx;
      cl.x0 = ctid - cl.r0 * d.nx;
      cl.fx_const = d.fconst[0];
      cl.nu0 = d.nu0;
      cl.s_nu0 = d.s_nu0;
      cl.C = d.C;
      smode = d.strain_mode;
      fy_of_z = d.fy_of_z;
      fy_const = d.fconst[1];
    }
    const int st = s;
    const uint32_t ph = phase;
    if (++s == stages) {
      s = 0;
      phase ^= 1u;
    }
    if (ok) {
      if (*abort_flag) {
        ok = false;
      } else if (!mbar_wait(bar_full + 8u * st, ph, wait_ns)) {
        atomicOr(err, ERR_TIMEOUT);
        *abort_flag = 1;
        ok = false;
      }
    }
    if (!ok) continue;  // keep the named-barrier schedule of the other consumers
    const TileGeom g = walker_geom(w);
    const float* fx = insts[w.ii].fx_of_y + g.y0;
    const float Fy = __ldg(fy_of_z + g.z) + fy_const;
    const int ncell = g.rows * cl.nx;
    T* sbuf = reinterpret_cast<T*>(smem + kBarBytes + (size_t)st * tile_bytes);
    const DiagTile dt{dout, g.y0, g.z, insts[w.ii].ny, insts[w.ii].nz, hist_sm, lo, win, hist_gl};
    if (smode == 1)
      collide_tile<T, ODD, MODE, 1, SLOT>(cl, ncell, fx, Fy, sbuf, fz_table, nct, acc, dt, run);
    else
      collide_tile<T, ODD, MODE, 0, SLOT>(cl, ncell, fx, Fy, sbuf, fz_table, nct, acc, dt, run);
    if (MODE != MODE_STEP) acc.fold_if_full();
    // hand the tile back: make this warp's shared-memory writes visible to the
    // TMA engine, then one arrival per warp
    fence_async_smem();
    __syncwarp();
    if (lane == 0) mbar_arrive(bar_done + 8u * st);
  }
  if (MODE != MODE_STEP && cur >= 0)
    block_flush(acc, sa.partials + ((int64_t)cur * sa.grid + blockIdx.x) * kNP, nct, 1);
  if (MODE == MODE_DIAG && dout.hist) run.flush(hist_sm, lo, win, hist_gl);
  if (MODE == MODE_DIAG && dout.hist && hist_sm) {
    named_sync(2, nct);
    for (int i = ctid; i < win; i += nct)
      if (hist_sm[i]) atomicAdd(&dout.hist[lo + i], hist_sm[i]);
  }
}

template <typename T, bool ODD, int MODE, int SLOT>
cudaError_t launch_tma_t(const LaunchArgs& la, cudaStream_t st) {
  return launch_kernel(k_step_tma<T, ODD, MODE, SLOT>, la.grid, la.threads, la.smem_bytes, st, la.insts,
                       la.ninst, la.tile_lo, la.tile_hi, la.sa, la.stages, la.tile_bytes_max, la.err,
                       la.wait_ns, la.withhold_first_load, la.dout, la.hist_smem, la.hist_lo, la.hist_win);
}

template <typename T, int SLOT>
cudaError_t dispatch_tma_s(const LaunchArgs& la, cudaStream_t st) {
  if (la.odd) {
    if (la.mode == MODE_STEP) return launch_tma_t<T, true, MODE_STEP, SLOT>(la, st);
    if (la.mode == MODE_STEP_STATS) return launch_tma_t<T, true, MODE_STEP_STATS, SLOT>(la, st);
    return launch_tma_t<T, true, MODE_DIAG, SLOT>(la, st);
  }
  if (la.mode == MODE_STEP) return launch_tma_t<T, false, MODE_STEP, SLOT>(la, st);
  if (la.mode == MODE_STEP_STATS) return launch_tma_t<T, false, MODE_STEP_STATS, SLOT>(la, st);
  return launch_tma_t<T, false, MODE_DIAG, SLOT>(la, st);
}

template <typename T>
cudaError_t dispatch_tma(const LaunchArgs& la, cudaStream_t st) {
  switch (la.slot_bytes) {
    case 0: return dispatch_tma_s<T, 0>(la, st);
    case kSlotGrouped: return dispatch_tma_s<T, kSlotGrouped>(la, st);
    case kSlot3: return dispatch_tma_s<T, kSlot3>(la, st);
    case kSlot2: return dispatch_tma_s<T, kSlot2>(la, st);
    case kSlot2h: return dispatch_tma_s<T, kSlot2h>(la, st);
  }
  return cudaErrorInvalidValue;
}

template <typename T, int SLOT>
cudaError_t set_smem_s(int smem) {
  const void* fns[] = {(const void*)k_step_tma<T, false, MODE_STEP, SLOT>,
                       (const void*)k_step_tma<T, true, MODE_STEP, SLOT>,
                       (const void*)k_step_tma<T, false, MODE_STEP_STATS, SLOT>,
                       (const void*)k_step_tma<T, true, MODE_STEP_STATS, SLOT>,
                       (const void*)k_step_tma<T, false, MODE_DIAG, SLOT>,
                       (const void*)k_step_tma<T, true, MODE_DIAG, SLOT>};
  for (const void* f : fns) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t set_smem(int smem) {
  cudaError_t e = set_smem_s<T, 0>(smem);
  if (e == cudaSuccess) e = set_smem_s<T, kSlotGrouped>(smem);
  if (e == cudaSuccess) e = set_smem_s<T, kSlot3>(smem);
  if (e == cudaSuccess) e = set_smem_s<T, kSlot2>(smem);
  if (e == cudaSuccess) e = set_smem_s<T, kSlot2h>(smem);
  return e;
}

template <typename T, int MODE>
cudaError_t occupancy(int* n, int slot_bytes, int threads, int smem_bytes) {
  switch (slot_bytes) {
    case 0:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_step_tma<T, true, MODE, 0>, threads, smem_bytes);
    case kSlotGrouped:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_step_tma<T, true, MODE, kSlotGrouped>, threads,
                                                           smem_bytes);
    case kSlot3:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_step_tma<T, true, MODE, kSlot3>, threads,
                                                           smem_bytes);
    case kSlot2h:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_step_tma<T, true, MODE, kSlot2h>, threads,
                                                           smem_bytes);
    case kSlot2:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_step_tma<T, true, MODE, kSlot2>, threads,
                                                           smem_bytes);
  }
  return cudaErrorInvalidValue;
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

int tma_diag_smem_limit(int precision) {
  // the per-block opt-in maximum less the pass's static shared memory (the
  // block reduction's scratch)
  cudaFuncAttributes a{};
  cudaError_t e = cudaErrorInvalidValue;
  switch (precision) {
    case 0: e = cudaFuncGetAttributes(&a, k_step_tma<float, false, MODE_DIAG, 0>); break;
    case 1: e = cudaFuncGetAttributes(&a, k_step_tma<__half, false, MODE_DIAG, 0>); break;
    case 2: e = cudaFuncGetAttributes(&a, k_step_tma<__nv_bfloat16, false, MODE_DIAG, 0>); break;
  }
  int dev = 0, optin = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return 0;
  return std::min(kMaxDynSmem, optin - (int)a.sharedSizeBytes);
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

int tma_max_blocks_per_sm(int precision, int slot_bytes, int threads, int smem_bytes, bool diag) {
  int n = 0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (precision) {
    case 0:
      e = diag ? occupancy<float, MODE_DIAG>(&n, slot_bytes, threads, smem_bytes)
               : occupancy<float, MODE_STEP_STATS>(&n, slot_bytes, threads, smem_bytes);
      break;
    case 1:
      e = diag ? occupancy<__half, MODE_DIAG>(&n, slot_bytes, threads, smem_bytes)
               : occupancy<__half, MODE_STEP_STATS>(&n, slot_bytes, threads, smem_bytes);
      break;
    case 2:
      e = diag ? occupancy<__nv_bfloat16, MODE_DIAG>(&n, slot_bytes, threads, smem_bytes)
               : occupancy<__nv_bfloat16, MODE_STEP_STATS>(&n, slot_bytes, threads, smem_bytes);
      break;
  }
  return e == cudaSuccess ? n : 0;
}

uint32_t bounds_word_tma() { return take_bounds_word(); }

}  // namespace lbm
