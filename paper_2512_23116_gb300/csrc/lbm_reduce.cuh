// Fused FP64 statistics of the step kernels: per-thread accumulation of the
// per-cell quantities, warp-shuffle + shared-memory block reduction into one
// partial per block and instance (deterministic order), and the per-cell
// outputs of the read-only diagnostic pass.
#pragma once

#include <cfloat>
#include <cstdint>

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

// Cells a thread sums in FP32 before it adds the sums to its FP64 totals:
// FP64 arithmetic is slow on this part (a fold per tile of one x-line cost ~9
// FP64 operations per cell, a quarter of the statistics pass at 800^3), and
// an FP32 sum of 32 terms is exact to ~32 x 2^-24 of its magnitude.
constexpr uint32_t kFoldCells = 32;

// Per-thread accumulation: the cells a thread updates are summed in FP32 (`t`)
// and added to the FP64 totals (`s`) by fold(), at the end of a tile once at
// least kFoldCells cells have been summed (fold_if_full); the block and grid
// reductions are FP64.
struct Acc {
  double s[kNSum];
  float t[kNSum];
  float thmin, thmax;
  uint32_t bad, cells, tn;

  __device__ __forceinline__ void reset() {
#pragma unroll
    for (int k = 0; k < kNSum; ++k) {
      s[k] = 0.0;
      t[k] = 0.f;
    }
    thmin = FLT_MAX;
    thmax = -FLT_MAX;
    bad = 0;
    cells = 0;
    tn = 0;
  }

  // Energy E_k = <u.u>/2, injection <F.u>, dissipation 2 nu <S_ij S_ij> with
  // S_ij S_ij = |S|^2/2 (Eqs. energy_balance, strain_norm), theta = tau_e - 1/2.
  // Every rounding is spelled out (fused multiply-adds as __fmaf_rn): left to
  // the compiler, the contraction of these sums into FMAs differed between the
  // kernel variants, and equal per-cell values must give equal statistics in
  // every tile layout and kernel configuration.
  __device__ __forceinline__ void add(const CellDiag& g, float Fx, float Fy, float Fz, float C) {
    const float rho = __fadd_rn(1.f, g.drho);
    const float ux = g.ux, uy = g.uy, uz = g.uz;
    const float sn = g.snorm, th = g.theta;
    const float ss = __fmul_rn(sn, sn);
    t[P_DRHO] = __fadd_rn(t[P_DRHO], g.drho);
    t[P_MX] = __fmaf_rn(rho, ux, t[P_MX]);
    t[P_MY] = __fmaf_rn(rho, uy, t[P_MY]);
    t[P_MZ] = __fmaf_rn(rho, uz, t[P_MZ]);
    t[P_UU] = __fadd_rn(t[P_UU], __fmaf_rn(ux, ux, __fmaf_rn(uy, uy, __fmul_rn(uz, uz))));
    t[P_FU] = __fadd_rn(t[P_FU], __fmaf_rn(Fx, ux, __fmaf_rn(Fy, uy, __fmul_rn(Fz, uz))));
    t[P_SS] = __fadd_rn(t[P_SS], ss);
    t[P_NUTSS] = __fmaf_rn(__fmul_rn(C, sn), ss, t[P_NUTSS]);
    t[P_TH] = __fadd_rn(t[P_TH], th);
    t[P_TH2] = __fmaf_rn(th, th, t[P_TH2]);
    t[P_XX] = __fmaf_rn(ux, ux, t[P_XX]);
    t[P_YY] = __fmaf_rn(uy, uy, t[P_YY]);
    t[P_ZZ] = __fmaf_rn(uz, uz, t[P_ZZ]);
    t[P_XY] = __fmaf_rn(ux, uy, t[P_XY]);
    t[P_XZ] = __fmaf_rn(ux, uz, t[P_XZ]);
    t[P_YZ] = __fmaf_rn(uy, uz, t[P_YZ]);
    thmin = fminf(thmin, g.theta);
    thmax = fmaxf(thmax, g.theta);
    const float chk = g.drho + g.ux + g.uy + g.uz + g.snorm;
    bad += isfinite(chk) ? 0u : 1u;
    cells += 1u;
    tn += 1u;
  }

  // Move the FP32 sums into the FP64 totals.
  __device__ __forceinline__ void fold() {
#pragma unroll
    for (int k = 0; k < kNSum; ++k) {
      s[k] += (double)t[k];
      t[k] = 0.f;
    }
    tn = 0;
  }

  __device__ __forceinline__ void fold_if_full() {
    if (tn >= kFoldCells) fold();
  }
};

// A thread's run of cells in one theta-histogram bin: the count goes to the
// histogram (one atomic add) when the bin changes and at the end.  Theta
// concentrates in a few bins, so per-cell increments, even warp-aggregated
// ones, would serialise on the same words.  Bins [lo, lo + win) are counted in
// shared memory `sm` (at bin - lo); the others (when `gl` is not null) in the
// global counts `gl`, summed first over the warp's lanes that flush the same
// bin: contended atomics in L2 cost far more than the match; in shared memory
// they do not.
struct HistRun {
  int bin = -1;
  uint32_t n = 0;

  // Called by every active lane; lanes with `go` add their run.  gl is null
  // (for the whole block) when the window holds every bin.
  __device__ __forceinline__ void flush_if(uint32_t* sm, int lo, int win, uint32_t* gl, bool go) {
    go = go && n > 0;
    const bool local = go && (unsigned)(bin - lo) < (unsigned)win;
    if (local) atomicAdd(&sm[bin - lo], n);
    if (gl) {
      const bool far = go && !local;
      const unsigned fl = __ballot_sync(__activemask(), far);
      if (far) {
        const unsigned grp = __match_any_sync(fl, bin);
        const unsigned tot = __reduce_add_sync(grp, n);
        if ((int)(threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&gl[bin], tot);
      }
    }
    if (go) n = 0;
  }

  __device__ __forceinline__ void flush(uint32_t* sm, int lo, int win, uint32_t* gl) {
    flush_if(sm, lo, win, gl, true);
  }
};

// Reduce the accumulators of the `nthreads` threads that call this (a whole
// block, or the consumer warps of a specialised block synchronised with named
// barrier `bar_id`) and write kNP doubles to dst.  Fixed order: lane tree,
// then warps in index order.  Inlined into its kernel: an out-of-line call
// takes the accumulator's address, which keeps its sums in local memory for
// the whole cell loop.
__device__ __forceinline__ void named_sync(int bar_id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(nthreads) : "memory");
}

static __device__ __forceinline__ void block_flush(Acc& acc, double* __restrict__ dst, int nthreads,
                                         int bar_id) {
  __shared__ double red[32][kNP];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  acc.fold();
  double v[kNP];
#pragma unroll
  for (int k = 0; k < kNSum; ++k) v[k] = acc.s[k];
  v[P_THMIN] = acc.thmin;
  v[P_THMAX] = acc.thmax;
  v[P_BAD] = acc.bad;
  v[P_CELLS] = acc.cells;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int k = 0; k < kNP; ++k) {
      const double o = __shfl_down_sync(0xffffffffu, v[k], off);
      if (k == P_THMIN) v[k] = fmin(v[k], o);
      else if (k == P_THMAX) v[k] = fmax(v[k], o);
      else v[k] += o;
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < kNP; ++k) red[warp][k] = v[k];
  }
  named_sync(bar_id, nthreads);
  if (threadIdx.x < kNP) {
    const int k = threadIdx.x;
    const int nw = nthreads >> 5;
    double r = red[0][k];
    for (int w = 1; w < nw; ++w) {
      const double o = red[w][k];
      if (k == P_THMIN) r = fmin(r, o);
      else if (k == P_THMAX) r = fmax(r, o);
      else r += o;
    }
    dst[k] = r;
  }
  named_sync(bar_id, nthreads);
}

// Per-cell outputs of the read-only diagnostic pass; when o.hist is set the
// thread's histogram runs go to the shared-memory counts hist_sm (bins
// [hist_lo, hist_lo + hist_win)) and to the global counts hist_gl (the rest;
// null when none).
__device__ __forceinline__ void diag_write(const DiagOut& o, const CellDiag& g, int x, int y, int z,
                                           int nx, int ny, int nz, uint32_t* hist_sm, int hist_lo,
                                           int hist_win, uint32_t* hist_gl, HistRun& run) {
  const int64_t n = (int64_t)nx * ny * nz;
  const int64_t i = ((int64_t)z * ny + y) * nx + x;
  if (!in_bounds(x >= 0 && x < nx && y >= 0 && y < ny && z >= 0 && z < nz)) return;
  if (o.u) {
    o.u[i] = g.ux;
    o.u[n + i] = g.uy;
    o.u[2 * n + i] = g.uz;
  }
  if (o.aux) {
    o.aux[i] = g.drho;
    o.aux[n + i] = g.snorm;
    o.aux[2 * n + i] = g.theta;
  }
  if (o.plane) {
    if (o.plane_axis == 0 && x == o.plane_index) o.plane[(int64_t)z * ny + y] = g.theta;
    if (o.plane_axis == 1 && y == o.plane_index) o.plane[(int64_t)z * nx + x] = g.theta;
    if (o.plane_axis == 2 && z == o.plane_index) o.plane[(int64_t)y * nx + x] = g.theta;
  }
  if (o.hist) {
    int b = o.hist_bins;
    const float q = g.theta * o.hist_scale;
    if (q >= 0.f && q < (float)o.hist_bins) b = min((int)q, o.hist_bins - 1);
    const bool change = b != run.bin;
    run.flush_if(hist_sm, hist_lo, hist_win, hist_gl, change);
    if (change) run.bin = b;
    run.n += 1u;
  }
}

}  // namespace lbm
