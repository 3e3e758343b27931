// Auxiliary kernels: initial equilibrium, canonical population access in the
// AA layout, parity re-layout, the FP64 reduction finisher, the shell binning
// of the energy spectrum and the structure-function reductions.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>

#include "lbm_device.cuh"
#include "lbm_kernels.h"

namespace lbm {

namespace {

constexpr int kAuxThreads = 256;

__device__ __forceinline__ void cell_xyz(int64_t c, int nx, int ny, int& x, int& y, int& z) {
  if (c < (int64_t)0x7fffffff) {  // 32-bit division for lattices below 2^31 cells
    const uint32_t cu = (uint32_t)c, row = cu / (uint32_t)nx;
    x = (int)(cu - row * (uint32_t)nx);
    z = (int)(row / (uint32_t)ny);
    y = (int)(row - (uint32_t)z * (uint32_t)ny);
    return;
  }
  const int64_t row = c / nx;
  x = (int)(c - row * nx);
  z = (int)(row / ny);
  y = (int)(row - (int64_t)z * ny);
}

// Where canonical population a of cell (x, y, z) lives at the given parity:
// even time: slot a of x; odd time: slot opp(a) of x - c_a.
__device__ __forceinline__ int64_t canon_index(const InstDesc& d, int a, bool odd, int x, int y,
                                               int z) {
  if (!odd) return pop_off(d, a, x, y, z);
  int xs = x - cx(a), ys = y - cy(a), zs = z - cz(a);
  xs = xs < 0 ? xs + d.nx : (xs >= d.nx ? xs - d.nx : xs);
  ys = ys < 0 ? ys + d.ny : (ys >= d.ny ? ys - d.ny : ys);
  zs = zs < 0 ? zs + d.nz : (zs >= d.nz ? zs - d.nz : zs);
  return pop_off(d, opp(a), xs, ys, zs);
}

// U: type of the given velocity (mode 3), FP64 or FP32; the equilibrium is
// computed from its FP32 rounding either way.
template <typename T, typename U>
__global__ void k_init(InstDesc d, bool odd, int mode, double amp, const U* __restrict__ u,
                       int64_t ustride, int64_t c0, int64_t n) {
  T* fb = static_cast<T*>(d.f);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(c0 + k, d.nx, d.ny, x, y, z);
    double ux = 0.0, uy = 0.0, uz = 0.0, drho = 0.0;
    if (mode == 1 || mode == 2) {
      double sX, cX, sY, cY, sZ, cZ;
      sincospi(2.0 * x / d.nx, &sX, &cX);
      sincospi(2.0 * y / d.ny, &sY, &cY);
      sincospi(2.0 * z / d.nz, &sZ, &cZ);
      if (mode == 1) {
        ux = amp * sX * cY * cZ;
        uy = -amp * cX * sY * cZ;
      } else {
        ux = amp * sX * cY;
        uy = -amp * cX * sY;
        // pressure of the 2-D vortex: p = (A^2/4)(cos 2X + cos 2Y), drho = 3 p
        drho = 0.75 * amp * amp * ((cX * cX - sX * sX) + (cY * cY - sY * sY));
      }
    } else if (mode == 3) {
      ux = u[k];
      uy = u[ustride + k];
      uz = u[2 * ustride + k];
    }
    float f[19];
    equilibrium((float)drho, (float)ux, (float)uy, (float)uz, f);
#pragma unroll
    for (int a = 0; a < 19; ++a) {
      const int64_t i = canon_index(d, a, odd, x, y, z);
      if (in_bounds(i >= 0 && i < d.f_elems)) fb[i] = Storage<T>::pack(f[a]);
    }
  }
}

template <typename T>
__global__ void k_get_pop(InstDesc d, bool odd, int a, double* __restrict__ out, int shifted,
                          int64_t c0, int64_t n) {
  const T* fb = static_cast<const T*>(d.f);
  const double w = shifted ? 0.0 : weight(a);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(c0 + k, d.nx, d.ny, x, y, z);
    const int64_t i = canon_index(d, a, odd, x, y, z);
    out[k] = (in_bounds(i >= 0 && i < d.f_elems) ? (double)Storage<T>::cvt(fb[i]) : 0.0) + w;
  }
}

template <typename T>
__global__ void k_set_pop(InstDesc d, bool odd, int a, const double* __restrict__ in, int shifted,
                          int64_t c0, int64_t n) {
  T* fb = static_cast<T*>(d.f);
  const double w = shifted ? 0.0 : weight(a);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(c0 + k, d.nx, d.ny, x, y, z);
    const int64_t i = canon_index(d, a, odd, x, y, z);
    if (in_bounds(i >= 0 && i < d.f_elems)) fb[i] = Storage<T>::pack((float)(in[k] - w));
  }
}

// sa, sb: dense [nz][ny][nxp] copies of slots a and opp(a) taken at the old parity.
template <typename T>
__global__ void k_relayout(InstDesc d, bool from_odd, int a, const T* __restrict__ sa,
                           const T* __restrict__ sb) {
  T* fb = static_cast<T*>(d.f);
  const int b = opp(a);
  const int64_t n = (int64_t)d.nx * d.ny * d.nz;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(k, d.nx, d.ny, x, y, z);
    const int64_t o = cell_off(x, y, z, d.ny, d.nxp);
    // canonical values at this cell, from the old layout
    double fa, fbv;
    if (!from_odd) {
      fa = Storage<T>::cvt(sa[o]);
      fbv = Storage<T>::cvt(sb[o]);
    } else {
      // f_a(x) = slot b of x - c_a ; f_b(x) = slot a of x + c_a
      int xs = x - cx(a), ys = y - cy(a), zs = z - cz(a);
      xs = (xs + d.nx) % d.nx;
      ys = (ys + d.ny) % d.ny;
      zs = (zs + d.nz) % d.nz;
      int xq = x + cx(a), yq = y + cy(a), zq = z + cz(a);
      xq = (xq + d.nx) % d.nx;
      yq = (yq + d.ny) % d.ny;
      zq = (zq + d.nz) % d.nz;
      fa = Storage<T>::cvt(sb[cell_off(xs, ys, zs, d.ny, d.nxp)]);
      fbv = Storage<T>::cvt(sa[cell_off(xq, yq, zq, d.ny, d.nxp)]);
    }
    const bool to_odd = !from_odd;
    const int64_t ia = canon_index(d, a, to_odd, x, y, z), ib = canon_index(d, b, to_odd, x, y, z);
    if (in_bounds(ia >= 0 && ia < d.f_elems)) fb[ia] = Storage<T>::pack((float)fa);
    if (in_bounds(ib >= 0 && ib < d.f_elems)) fb[ib] = Storage<T>::pack((float)fbv);
  }
}

// One warp per output value: lane l folds blocks l, l + 32, ... in that order,
// then a fixed shuffle tree combines the lanes, so a result depends only on
// the partials and the grid size, never on scheduling.  seq[0] counts the
// records in the ring; seq[1] counts the blocks of a launch that are done, and
// the last of them advances seq[0] (every block has read it by then).
__global__ void k_finish(const double* __restrict__ partials, int ninst, int grid,
                         double* __restrict__ results, double* ring, unsigned long long* seq,
                         int cap, uint32_t* err) {
  const unsigned long long slot = ring ? (__ldcg(seq) % (unsigned long long)cap) : 0ull;
  const int lane = threadIdx.x & 31;
  const int warps = (int)((gridDim.x * blockDim.x) >> 5);
  for (int idx = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); idx < ninst * kNP; idx += warps) {
    const int i = idx / kNP, k = idx - i * kNP;
    const bool lo = k == P_THMIN, hi = k == P_THMAX;
    double r = lo ? DBL_MAX : (hi ? -DBL_MAX : 0.0);
    for (int b = lane; b < grid; b += 32) {
      const double* p = partials + ((int64_t)i * grid + b) * kNP;
      if (p[P_CELLS] == 0.0) continue;  // block saw no cell of instance i
      const double v = p[k];
      r = lo ? fmin(r, v) : (hi ? fmax(r, v) : r + v);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double o = __shfl_down_sync(0xffffffffu, r, off);
      r = lo ? fmin(r, o) : (hi ? fmax(r, o) : r + o);
    }
    if (lane == 0) {
      results[idx] = r;
      if (k == P_BAD && r > 0.0) atomicOr(err, ERR_NONFINITE);
      if (ring) ring[slot * (unsigned long long)(ninst * kNP) + idx] = r;
    }
  }
  if (!ring) return;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(seq + 1, 1ull) == (unsigned long long)gridDim.x - 1ull) {
      seq[0] += 1ull;
      seq[1] = 0ull;
    }
  }
}

// Exact integer shell: s with s^2 - s + 1 <= K <= s^2 + s (s - 1/2 <= sqrt K < s + 1/2).
__device__ __forceinline__ int shell_of(long long K) {
  long long r = (long long)sqrt((double)K);
  while (r * r > K) --r;
  while ((r + 1) * (r + 1) <= K) ++r;
  return (int)(K > r * r + r ? r + 1 : r);
}

// shell_of for K < 2^24, where K is exact in FP32 and the FP32 square root is
// within one of the integer root: no FP64 arithmetic (slow on this part).
__device__ __forceinline__ int shell_of_small(int K) {
  int r = (int)sqrtf((float)K);
  while (r * r > K) --r;
  while ((r + 1) * (r + 1) <= K) ++r;
  return K > r * r + r ? r + 1 : r;
}

// A warp takes one (ky, kz) line of the half-spectrum at a time, lanes over kx
// (no division per mode).  The shell does not decrease with kx, so the lanes
// of one group of 32 modes that fall in one shell form a run: their FP32
// energies are summed within the run (a segmented shuffle sum) and the run's
// first lane adds the sum, scaled, to the block's FP64 shell total in shared
// memory.
__global__ void k_spec_bin(const float2* __restrict__ c, int nx, int ny, int nz, int kmax,
                           double* __restrict__ partials) {
  extern __shared__ double sh[];
  for (int s = threadIdx.x; s <= kmax; s += blockDim.x) sh[s] = 0.0;
  __syncthreads();
  const int nxh = nx / 2 + 1;
  const double ncell = (double)nx * ny * nz;
  const double scale = 0.5 / (ncell * ncell);
  const int lane = threadIdx.x & 31;
  const int64_t lines = (int64_t)ny * nz;
  const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t l = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); l < lines; l += wstride) {
    const int kz = (int)(l / ny), ky = (int)(l - (int64_t)kz * ny);
    const long long sy = ky <= ny / 2 ? ky : ky - ny;
    const long long sz = kz <= nz / 2 ? kz : kz - nz;
    const long long Kp = sy * sy + sz * sz;
    const float2* row = c + l * nxh;
    for (int x0 = 0; x0 < nxh; x0 += 32) {
      const int kx = x0 + lane;
      int s = kmax + 1;  // no contribution
      float e = 0.f;
      if (kx < nxh) {
        const long long K = (long long)kx * kx + Kp;
        const int sk = K < (1ll << 24) ? shell_of_small((int)K) : shell_of(K);
        if (sk <= kmax) {
          // the R2C half-spectrum holds each kx > 0 mode once for the pair
          // (k, -k), except kx = 0 and the Nyquist plane kx = nx/2 (even nx)
          const float2 v = row[kx];
          s = sk;
          e = ((kx == 0 || 2 * kx == nx) ? 1.f : 2.f) * (v.x * v.x + v.y * v.y);
        }
      }
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const float eo = __shfl_down_sync(0xffffffffu, e, off);
        const int so = __shfl_down_sync(0xffffffffu, s, off);
        if (lane + off < 32 && so == s) e += eo;
      }
      const int sp = __shfl_up_sync(0xffffffffu, s, 1);
      if (s <= kmax && (lane == 0 || sp != s)) atomicAdd(&sh[s], scale * (double)e);
    }
  }
  __syncthreads();
  for (int s = threadIdx.x; s <= kmax; s += blockDim.x)
    partials[(int64_t)blockIdx.x * (kmax + 1) + s] += sh[s];
}

// Column sums of a [rows][cols] table, one warp per column in the fixed order
// of k_finish (lane l adds rows l, l + 32, ...; then a shuffle tree).
__global__ void k_sum_cols(const double* __restrict__ p, int rows, int cols, double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int warps = (int)((gridDim.x * blockDim.x) >> 5);
  for (int c = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); c < cols; c += warps) {
    double r = 0.0;
    for (int b = lane; b < rows; b += 32) r += p[(int64_t)b * cols + c];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) r += __shfl_down_sync(0xffffffffu, r, off);
    if (lane == 0) out[c] = r;
  }
}

__global__ void k_struct(const float* __restrict__ u, int nx, int ny, int nz, int r,
                         double* __restrict__ partials, int64_t block_stride) {
  const int64_t n = (int64_t)nx * ny * nz;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  const int rx = r % nx, ry = r % ny, rz = r % nz;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(i, nx, ny, x, y, z);
    const int xr = x + rx >= nx ? x + rx - nx : x + rx;
    const int yr = y + ry >= ny ? y + ry - ny : y + ry;
    const int zr = z + rz >= nz ? z + rz - nz : z + rz;
    if (!in_bounds(xr >= 0 && xr < nx && yr >= 0 && yr < ny && zr >= 0 && zr < nz)) continue;
    const double d3[3] = {
        (double)u[((int64_t)z * ny + y) * nx + xr] - (double)u[i],
        (double)u[n + ((int64_t)z * ny + yr) * nx + x] - (double)u[n + i],
        (double)u[2 * n + ((int64_t)zr * ny + y) * nx + x] - (double)u[2 * n + i]};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double p = d3[a];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        acc[k] += p;
        p *= d3[a];
      }
    }
  }
  __shared__ double red[32][6];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    double v = acc[k];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][threadIdx.x];
    partials[(int64_t)blockIdx.x * block_stride + threadIdx.x] = v;
  }
}

// Structure functions of up to 24 separations in one launch: blockIdx.y takes
// a chunk of kStructChunk separations, a warp one x-line at a time (lanes over
// x: no division per cell), so a cell's own velocity is read once per chunk
// rather than once per separation.  Per block b and separation k,
// partials[(b * nr + k) * 6 + p - 1] = sum over its cells and the three axes
// of d^p, d = u_a(x + r_k e_a) - u_a(x), p = 1..6.  The powers and the running
// sums are FP32 (FP64 arithmetic is slow on this part: with FP64 powers the
// 256^3 structure functions took 17 ms), folded into FP64 totals every
// kFoldStruct cells; the block reduction is FP64.
constexpr int kFoldStruct = 32;
constexpr int kStructChunk = 3;

__global__ void __launch_bounds__(kAuxThreads, 2)
k_struct_multi(const float* __restrict__ u, int nx, int ny, int nz, StructSeps seps, int nr,
               double* __restrict__ partials) {
  const int k0 = blockIdx.y * kStructChunk;
  const int kn = min(kStructChunk, nr - k0);
  const int64_t n = (int64_t)nx * ny * nz;
  // a chunk shorter than kStructChunk is padded with r = 0, whose increments
  // are exactly zero: the cell loop has no branch per separation, so the
  // loads of all separations are in flight together
  int rx[kStructChunk], ry[kStructChunk], rz[kStructChunk];
#pragma unroll
  for (int j = 0; j < kStructChunk; ++j) {
    const int r = j < kn ? seps.r[k0 + j] : 0;
    rx[j] = r % nx;
    ry[j] = r % ny;
    rz[j] = r % nz;
  }
  // FP64 totals of each thread in shared memory, leaving the registers to the
  // loads in flight
  __shared__ double tot[kStructChunk * 6][kAuxThreads];
  float t[kStructChunk][6];
#pragma unroll
  for (int j = 0; j < kStructChunk; ++j)
#pragma unroll
    for (int p = 0; p < 6; ++p) {
      tot[j * 6 + p][threadIdx.x] = 0.0;
      t[j][p] = 0.f;
    }
  int cnt = 0;
  const int lane = threadIdx.x & 31;
  const int64_t lines = (int64_t)ny * nz;
  const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t l = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); l < lines; l += wstride) {
    const int z = (int)(l / ny), y = (int)(l - (int64_t)z * ny);
    const int64_t base = l * nx;
    // two cells per lane and pass (x and x + 32; the second one weighted 0
    // past the end of the line), so that twice the loads are in flight
    for (int x0 = lane; x0 < nx; x0 += 64) {
      const int x1 = x0 + 32 < nx ? x0 + 32 : x0;
      const float w1 = x0 + 32 < nx ? 1.f : 0.f;
      const int xs[2] = {x0, x1};
      float own[2][3];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        own[h][0] = u[base + xs[h]];
        own[h][1] = u[n + base + xs[h]];
        own[h][2] = u[2 * n + base + xs[h]];
      }
#pragma unroll
      for (int j = 0; j < kStructChunk; ++j) {
        const int yr = y + ry[j] >= ny ? y + ry[j] - ny : y + ry[j];
        const int zr = z + rz[j] >= nz ? z + rz[j] - nz : z + rz[j];
        float d[2][3];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int x = xs[h];
          const int xr = x + rx[j] >= nx ? x + rx[j] - nx : x + rx[j];
          const bool ok = in_bounds(xr >= 0 && xr < nx && yr >= 0 && yr < ny && zr >= 0 && zr < nz);
          const float m = ok ? (h ? w1 : 1.f) : 0.f;
          d[h][0] = m * (u[base + (ok ? xr : x)] - own[h][0]);
          d[h][1] = m * (u[n + ((int64_t)z * ny + (ok ? yr : y)) * nx + x] - own[h][1]);
          d[h][2] = m * (u[2 * n + ((int64_t)(ok ? zr : z) * ny + y) * nx + x] - own[h][2]);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            float q = d[h][a];
#pragma unroll
            for (int p = 0; p < 6; ++p) {
              t[j][p] += q;
              q *= d[h][a];
            }
          }
      }
      cnt += 2;
      if (cnt >= kFoldStruct) {
#pragma unroll
        for (int j = 0; j < kStructChunk; ++j)
#pragma unroll
          for (int p = 0; p < 6; ++p) {
            tot[j * 6 + p][threadIdx.x] += (double)t[j][p];
            t[j][p] = 0.f;
          }
        cnt = 0;
      }
    }
  }
  __shared__ double red[kAuxThreads / 32][6];
  const int warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < kStructChunk; ++j) {
    if (j >= kn) break;
#pragma unroll
    for (int p = 0; p < 6; ++p) {
      double v = tot[j * 6 + p][threadIdx.x] + (double)t[j][p];
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if (lane == 0) red[warp][p] = v;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
      double v = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][threadIdx.x];
      partials[((int64_t)blockIdx.x * nr + k0 + j) * 6 + threadIdx.x] = v;
    }
    __syncthreads();
  }
}

int grid_for(int64_t n) {
  int64_t b = (n + kAuxThreads - 1) / kAuxThreads;
  if (b < 1) b = 1;
  if (b > 4096) b = 4096;
  return (int)b;
}

template <typename T, typename U>
cudaError_t init_t(const InstDesc& d, bool odd, int mode, double amp, const U* u,
                   int64_t ustride, int64_t c0, int64_t n, cudaStream_t st) {
  return launch_kernel(k_init<T, U>, grid_for(n), kAuxThreads, 0, st, d, odd, mode, amp, u, ustride, c0, n);
}

template <typename U>
cudaError_t launch_init_u(const InstDesc& d, int precision, bool odd, int mode, double amp,
                          const U* u, int64_t ustride, int64_t c0, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  switch (precision) {
    case 0: return init_t<float, U>(d, odd, mode, amp, u, ustride, c0, n, st);
    case 1: return init_t<__half, U>(d, odd, mode, amp, u, ustride, c0, n, st);
    case 2: return init_t<__nv_bfloat16, U>(d, odd, mode, amp, u, ustride, c0, n, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_init(const InstDesc& d, int precision, bool odd, int mode, double amp,
                        const double* u, int64_t ustride, int64_t c0, int64_t n, cudaStream_t st) {
  return launch_init_u<double>(d, precision, odd, mode, amp, u, ustride, c0, n, st);
}

cudaError_t launch_init(const InstDesc& d, int precision, bool odd, const float* u, int64_t ustride,
                        int64_t c0, int64_t n, cudaStream_t st) {
  return launch_init_u<float>(d, precision, odd, 3, 0.0, u, ustride, c0, n, st);
}

cudaError_t launch_get_pop(const InstDesc& d, int precision, bool odd, int a, double* out,
                           int shifted, int64_t c0, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int g = grid_for(n);
  switch (precision) {
    case 0: return launch_kernel(k_get_pop<float>, g, kAuxThreads, 0, st, d, odd, a, out, shifted, c0, n);
    case 1: return launch_kernel(k_get_pop<__half>, g, kAuxThreads, 0, st, d, odd, a, out, shifted, c0, n);
    case 2: return launch_kernel(k_get_pop<__nv_bfloat16>, g, kAuxThreads, 0, st, d, odd, a, out, shifted, c0, n);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_set_pop(const InstDesc& d, int precision, bool odd, int a, const double* in,
                           int shifted, int64_t c0, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int g = grid_for(n);
  switch (precision) {
    case 0: return launch_kernel(k_set_pop<float>, g, kAuxThreads, 0, st, d, odd, a, in, shifted, c0, n);
    case 1: return launch_kernel(k_set_pop<__half>, g, kAuxThreads, 0, st, d, odd, a, in, shifted, c0, n);
    case 2: return launch_kernel(k_set_pop<__nv_bfloat16>, g, kAuxThreads, 0, st, d, odd, a, in, shifted, c0, n);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_relayout_pair(const InstDesc& d, int precision, bool from_odd, int a,
                                 void* scratch, cudaStream_t st) {
  const size_t es = precision == 0 ? 4 : 2;
  const size_t row = (size_t)d.nxp * es;
  const size_t rows = (size_t)d.nz * d.ny;
  const size_t plane = row * rows;
  char* s = static_cast<char*>(scratch);
  const char* base = static_cast<const char*>(d.f);
  const size_t pa = d.slot_grouped ? gpos(a) : a, pb = d.slot_grouped ? gpos(opp(a)) : opp(a);
  // slots a and opp(a), x-line by x-line (row_stride apart in either layout), into dense planes
  cudaError_t e = cudaMemcpy2DAsync(s, row, base + pa * d.slot_stride * es, (size_t)d.row_stride * es,
                                    row, rows, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  e = cudaMemcpy2DAsync(s + plane, row, base + pb * d.slot_stride * es, (size_t)d.row_stride * es,
                        row, rows, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  const int g = grid_for((int64_t)d.nx * d.ny * d.nz);
  switch (precision) {
    case 0:
      return launch_kernel(k_relayout<float>, g, kAuxThreads, 0, st, d, from_odd, a, (const float*)s,
                           (const float*)(s + plane));
    case 1:
      return launch_kernel(k_relayout<__half>, g, kAuxThreads, 0, st, d, from_odd, a, (const __half*)s,
                           (const __half*)(s + plane));
    case 2:
      return launch_kernel(k_relayout<__nv_bfloat16>, g, kAuxThreads, 0, st, d, from_odd, a,
                           (const __nv_bfloat16*)s, (const __nv_bfloat16*)(s + plane));
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_finish(const double* partials, int ninst, int grid, double* results,
                          double* ring, unsigned long long* seq, int cap, uint32_t* err,
                          cudaStream_t st) {
  const int warps_per_block = 256 / 32;
  const int blocks = std::max(1, std::min(1024, (ninst * kNP + warps_per_block - 1) / warps_per_block));
  return launch_kernel(k_finish, blocks, 256, 0, st, partials, ninst, grid, results, ring, seq, cap, err);
}

cudaError_t launch_spec_bin(const void* coeffs, int nx, int ny, int nz, int kmax,
                            double* partials, int blocks, cudaStream_t st) {
  return launch_kernel(k_spec_bin, blocks, kAuxThreads, (size_t)(kmax + 1) * sizeof(double), st,
                       static_cast<const float2*>(coeffs), nx, ny, nz, kmax, partials);
}

cudaError_t launch_spec_finish(const double* partials, int blocks, int kmax, double* E,
                               cudaStream_t st) {
  return launch_sum_cols(partials, blocks, kmax + 1, E, st);
}

cudaError_t launch_sum_cols(const double* partials, int rows, int cols, double* out,
                            cudaStream_t st) {
  const int blocks = std::max(1, std::min(1024, (cols + 7) / 8));  // 8 warps per block, a warp per column
  return launch_kernel(k_sum_cols, blocks, 256, 0, st, partials, rows, cols, out);
}

cudaError_t launch_struct_multi(const float* u, int nx, int ny, int nz, const int* r, int nr, double* partials,
                                int blocks, cudaStream_t st) {
  if (nr < 1 || nr > kMaxStructSeps) return cudaErrorInvalidValue;
  StructSeps seps{};
  for (int k = 0; k < nr; ++k) seps.r[k] = r[k];
  const int chunks = (nr + kStructChunk - 1) / kStructChunk;
  return launch_kernel(k_struct_multi, dim3(blocks, chunks), kAuxThreads, 0, st, u, nx, ny, nz, seps, nr,
                       partials);
}

cudaError_t launch_struct(const float* u, int nx, int ny, int nz, int r, double* partials,
                          int blocks, cudaStream_t st, int64_t block_stride) {
  return launch_kernel(k_struct, blocks, kAuxThreads, 0, st, u, nx, ny, nz, r, partials, block_stride);
}

uint32_t bounds_word_aux() { return take_bounds_word(); }

}  // namespace lbm
