// Seeded random solenoidal velocity field on the device: the synthetic
// stand-in for the paper's forced-turbulence states (the paper's own fields
// are not available; its runs start from a Taylor-Green field, Sec. 3.1).
//
// Recipe (the same one the host-side input generator of the test suite
// follows, so that both sides draw the same field from a seed):
//  1. modes: every integer wavevector k with 0 < |k|^2 <= kc^2,
//     kc = max(1, min(n_min / 2 - 1, floor(6 k0))), in the half space
//     kz > 0, or kz = 0 and ky > 0, or kz = ky = 0 and kx > 0; -k carries the
//     complex conjugate (a real field);
//  2. draws: per mode and component two standard normals (real, imaginary
//     part), each by the Box-Muller transform of two uniforms, each uniform
//     from SplitMix64 (Steele, Lea & Flood 2014) applied twice to a counter
//     that encodes (seed, k, component, draw);
//  3. projection onto the plane normal to k (solenoidal);
//  4. each integer shell s = round(|k|) scaled to the energy
//     1/2 sum |u_hat|^2 = s^4 exp(-2 (s/k0)^2);
//  5. a global factor giving u_rms = sqrt(<u.u>/3) = urms (Parseval);
//  6. u(x) = sum_k u_hat(k) exp(2 pi i k.x / n): a cuFFT complex-to-real
//     transform in FP64 per component, rounded to FP32.
// The shell sums are deterministic (one block per shell, fixed reduction
// order), so a seed always gives the same field bit for bit.
#include <cuda_runtime.h>
#include <cufft.h>

#include <cmath>
#include <vector>

#include "lbm_check.cuh"
#include "lbm_kernels.h"

namespace lbm {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Uniform in (0, 1]: the top 53 bits of SplitMix64 of the counter of
// (seed, k, component d, draw q), plus one, times 2^-53.
__device__ __forceinline__ double uniform(uint64_t seed, int kx, int ky, int kz, int d, int q) {
  uint64_t c = (seed & 0xFFFFFFFFull) * 0x100000001B3ull;
  c += (uint64_t)(kx + 512) << 40;
  c += (uint64_t)(ky + 512) << 28;
  c += (uint64_t)(kz + 512) << 16;
  c += (uint64_t)(d * 4 + q);
  const uint64_t r = splitmix64(splitmix64(c));
  return ((double)(r >> 11) + 1.0) * (1.0 / 9007199254740992.0);
}

// Standard normal number `part` (0: real, 1: imaginary) of component d.
__device__ __forceinline__ double normal(uint64_t seed, int kx, int ky, int kz, int d, int part) {
  const double u1 = uniform(seed, kx, ky, kz, d, 2 * part);
  const double u2 = uniform(seed, kx, ky, kz, d, 2 * part + 1);
  return sqrt(-2.0 * log(u1)) * cos(2.0 * 3.14159265358979323846 * u2);
}

struct Mode {
  int kx, ky, kz, shell;
  bool valid;
};

// Candidate i of the cube [-kc, kc]^3: the wavevector, whether it is a mode of
// the half space inside the cutoff, and its shell round(|k|).
__device__ __forceinline__ Mode candidate(int64_t i, int kc) {
  const int K = 2 * kc + 1;
  Mode m;
  m.kx = (int)(i % K) - kc;
  m.ky = (int)((i / K) % K) - kc;
  m.kz = (int)(i / ((int64_t)K * K)) - kc;
  const int k2 = m.kx * m.kx + m.ky * m.ky + m.kz * m.kz;
  const bool half = m.kz > 0 || (m.kz == 0 && m.ky > 0) || (m.kz == 0 && m.ky == 0 && m.kx > 0);
  m.valid = half && k2 > 0 && k2 <= kc * kc;
  m.shell = (int)floor(sqrt((double)k2) + 0.5);
  return m;
}

// The projected (solenoidal) coefficient of a mode, three components.
__device__ __forceinline__ void coefficient(uint64_t seed, const Mode& m, double (&re)[3], double (&im)[3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    re[d] = normal(seed, m.kx, m.ky, m.kz, d, 0);
    im[d] = normal(seed, m.kx, m.ky, m.kz, d, 1);
  }
  const double k[3] = {(double)m.kx, (double)m.ky, (double)m.kz};
  const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
  const double kr = (k[0] * re[0] + k[1] * re[1] + k[2] * re[2]) / k2;
  const double ki = (k[0] * im[0] + k[1] * im[1] + k[2] * im[2]) / k2;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    re[d] -= k[d] * kr;
    im[d] -= k[d] * ki;
  }
}

// Block s: the energy sum_modes in shell s of sum_d |a_d|^2 (unscaled),
// summed in a fixed order.
__global__ void k_shell_energy(uint64_t seed, int kc, double* __restrict__ shell_e) {
  const int s = blockIdx.x;
  const int K = 2 * kc + 1;
  const int64_t ncand = (int64_t)K * K * K;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < ncand; i += blockDim.x) {
    const Mode m = candidate(i, kc);
    if (!m.valid || m.shell != s) continue;
    double re[3], im[3];
    coefficient(seed, m, re, im);
    acc += re[0] * re[0] + im[0] * im[0] + re[1] * re[1] + im[1] * im[1] + re[2] * re[2] + im[2] * im[2];
  }
  __shared__ double red[kThreads];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) shell_e[s] = red[0];
}

// Component d of every mode, times the factor of its shell, into the
// half-spectrum [nz][ny][nx/2 + 1] of a complex-to-real transform: a mode with
// kx > 0 at (kx, ky, kz), one with kx < 0 as its conjugate at -k, one with
// kx = 0 at both k and -k (the transform's input must be Hermitian there).
__global__ void k_fill_half_spectrum(uint64_t seed, int kc, int d, const double* __restrict__ factor, int nx,
                                     int ny, int nz, double2* __restrict__ U) {
  const int K = 2 * kc + 1;
  const int64_t ncand = (int64_t)K * K * K;
  const int nh = nx / 2 + 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ncand;
       i += (int64_t)gridDim.x * blockDim.x) {
    const Mode m = candidate(i, kc);
    if (!m.valid) continue;
    double re[3], im[3];
    coefficient(seed, m, re, im);
    const double g = factor[m.shell];
    const double ar = g * re[d], ai = g * im[d];
    auto slot = [&](int kx, int ky, int kz) {
      const int y = ky < 0 ? ky + ny : ky, z = kz < 0 ? kz + nz : kz;
      return ((int64_t)z * ny + y) * nh + kx;
    };
    const int64_t nU = (int64_t)nz * ny * nh;
    auto put = [&](int64_t at, double re_, double im_) {
      if (in_bounds(at >= 0 && at < nU)) U[at] = make_double2(re_, im_);
    };
    if (m.kx > 0) {
      put(slot(m.kx, m.ky, m.kz), ar, ai);
    } else if (m.kx < 0) {
      put(slot(-m.kx, -m.ky, -m.kz), ar, -ai);
    } else {
      put(slot(0, m.ky, m.kz), ar, ai);
      put(slot(0, -m.ky, -m.kz), ar, -ai);
    }
  }
}

__global__ void k_round_f32(const double* __restrict__ in, int64_t n, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

int grid_of(int64_t n) {
  const int64_t b = (n + kThreads - 1) / kThreads;
  return (int)(b < 1 ? 1 : (b > 8192 ? 8192 : b));
}

}  // namespace

int random_field_cutoff(int nx, int ny, int nz, double k0) {
  int nmin = nx < ny ? nx : ny;
  nmin = nmin < nz ? nmin : nz;
  int kc = nmin / 2 - 1;
  const double k6 = 6.0 * k0;
  if (k6 < (double)kc) kc = (int)k6;
  return kc < 1 ? 1 : kc;
}

const char* random_velocity_f32(int nx, int ny, int nz, uint64_t seed, double urms, double k0, float* u,
                                cudaStream_t st, cudaError_t* cuda_err) {
  *cuda_err = cudaSuccess;
  const int kc = random_field_cutoff(nx, ny, nz, k0);
  const int nshell = kc + 1;
  const int64_t ncell = (int64_t)nx * ny * nz;
  const int64_t nhalf = (int64_t)nz * ny * (nx / 2 + 1);
  double* shell = nullptr;   // [nshell] energies, then [nshell] factors
  double2* U = nullptr;      // half spectrum of one component
  double* real = nullptr;    // one component in FP64
  cufftHandle plan = 0;
  bool have_plan = false;
  const char* what = nullptr;
  cudaError_t e = cudaSuccess;
  std::vector<double> E(nshell), factor(nshell, 0.0);
  double total = 0.0;
#define RF_CK(call)              \
  do {                           \
    e = (call);                  \
    if (e != cudaSuccess) {      \
      what = #call;              \
      goto done;                 \
    }                            \
  } while (0)
  RF_CK(cudaMalloc(&shell, sizeof(double) * 2 * nshell));
  RF_CK(cudaMalloc(&U, sizeof(double2) * nhalf));
  RF_CK(cudaMalloc(&real, sizeof(double) * ncell));
  RF_CK(launch_kernel(k_shell_energy, nshell, kThreads, 0, st, seed, kc, shell));
  RF_CK(cudaMemcpyAsync(E.data(), shell, sizeof(double) * nshell, cudaMemcpyDeviceToHost, st));
  RF_CK(cudaStreamSynchronize(st));
  // step 4: shell s scaled to s^4 exp(-2 (s/k0)^2); step 5: global u_rms
  for (int s = 1; s < nshell; ++s) {
    const double target = std::pow((double)s, 4) * std::exp(-2.0 * ((double)s / k0) * ((double)s / k0));
    factor[s] = std::sqrt(target / (E[s] > 1e-300 ? E[s] : 1e-300));
    total += factor[s] * factor[s] * E[s];
  }
  total *= 2.0;  // the pair (k, -k): <u.u> = 2 sum over the half space of |a|^2
  if (!(total > 0.0)) {
    what = "the random field has no energy";
    goto done;
  }
  for (int s = 1; s < nshell; ++s) factor[s] *= urms / std::sqrt(total / 3.0);
  RF_CK(cudaMemcpyAsync(shell + nshell, factor.data(), sizeof(double) * nshell, cudaMemcpyHostToDevice, st));
  if (cufftPlan3d(&plan, nz, ny, nx, CUFFT_Z2D) != CUFFT_SUCCESS) {
    what = "cufftPlan3d (Z2D)";
    goto done;
  }
  have_plan = true;
  if (cufftSetStream(plan, st) != CUFFT_SUCCESS) {
    what = "cufftSetStream";
    goto done;
  }
  for (int d = 0; d < 3; ++d) {
    RF_CK(cudaMemsetAsync(U, 0, sizeof(double2) * nhalf, st));
    const int64_t ncand = (int64_t)(2 * kc + 1) * (2 * kc + 1) * (2 * kc + 1);
    RF_CK(launch_kernel(k_fill_half_spectrum, grid_of(ncand), kThreads, 0, st, seed, kc, d,
                        (const double*)(shell + nshell), nx, ny, nz, U));
    if (cufftExecZ2D(plan, reinterpret_cast<cufftDoubleComplex*>(U), real) != CUFFT_SUCCESS) {
      what = "cufftExecZ2D";
      goto done;
    }
    RF_CK(launch_kernel(k_round_f32, grid_of(ncell), kThreads, 0, st, (const double*)real, ncell,
                        u + (int64_t)d * ncell));
  }
  RF_CK(cudaStreamSynchronize(st));
#undef RF_CK
done:
  if (what && e == cudaSuccess) e = cudaErrorUnknown;
  *cuda_err = what ? e : cudaSuccess;
  if (have_plan) cufftDestroy(plan);
  if (what) cudaStreamSynchronize(st);  // nothing may still use the buffers freed below
  cudaFree(real);
  cudaFree(U);
  cudaFree(shell);
  return what;
}

uint32_t bounds_word_random() { return take_bounds_word(); }

}  // namespace lbm
