// Diagnostics reductions (Sec. 4.2-4.3): mass of both phases, max |u| and the
// bulk pressures that give the Laplace pressure, accumulated in float64.
//
// Two passes with a fixed grid so that the result does not depend on the
// order in which CTAs finish: pass 1 writes one record of partial sums per
// CTA (warp-shuffle tree inside the CTA) to a scratch array, pass 2 reduces
// the records in one CTA in a fixed order.
#include "lbm_internal.cuh"

#include <math.h>

namespace lbm {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 1024;
constexpr int kRec = 8;   // doubles per partial record

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Reduce kRec values across the CTA; slot 2 is a maximum, the others sums.
__device__ void block_reduce(double (&v)[kRec], double (*sh)[kRec]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kRec; ++q) v[q] = (q == 2) ? warp_max(v[q]) : warp_sum(v[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < kRec; ++q) sh[warp][q] = v[q];
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < kRec; ++q) {
      double x = lane < nw ? sh[lane][q] : (q == 2 ? 0.0 : 0.0);
      v[q] = (q == 2) ? warp_max(x) : warp_sum(x);
    }
  }
}

__global__ void __launch_bounds__(kThreads) obs_pass1(const float* __restrict__ phi0,
                                                      const float* __restrict__ phi1,
                                                      const float* __restrict__ u, int d,
                                                      const float* __restrict__ p, long long n,
                                                      double* __restrict__ partials) {
  __shared__ double sh[kThreads / 32][kRec];
  double v[kRec] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float a0 = phi0[i], a1 = phi1[i];
    float u2 = 0.f;
    for (int q = 0; q < d; ++q) {
      const float uq = u[(long long)q * n + i];
      u2 += uq * uq;
    }
    const float pv = p[i];
    v[0] += a1;
    v[1] += a0;
    v[2] = fmax(v[2], (double)sqrtf(u2));
    if (a1 >= 0.99f) {
      v[3] += pv;
      v[4] += 1.0;
    }
    if (1.f - a0 - a1 >= 0.99f) {
      v[5] += pv;
      v[6] += 1.0;
    }
    if (!isfinite(a1) || !isfinite(u2) || !isfinite(pv)) v[7] += 1.0;
  }
  block_reduce(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < kRec; ++q) partials[(long long)blockIdx.x * kRec + q] = v[q];
  }
}

__global__ void __launch_bounds__(kThreads) obs_pass2(const double* __restrict__ partials, int nblocks,
                                                      double* __restrict__ out) {
  __shared__ double sh[kThreads / 32][kRec];
  double v[kRec] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
#pragma unroll
    for (int q = 0; q < kRec; ++q) {
      const double x = partials[(long long)b * kRec + q];
      v[q] = (q == 2) ? fmax(v[q], x) : v[q] + x;
    }
  }
  block_reduce(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < kRec; ++q) out[q] = v[q];
  }
}

// Phase fluxes for the relative permeability (Sec. 4.6, Eq. eq-Kp): over the
// pore space phi0 <= 1/2, slot 0 = sum phi1 u_a, 1 = sum phi2 u_a, 3 = sum u_a,
// 4 = pore nodes, 5 = sum phi1, 6 = sum phi2, 7 = non-finite values (slot 2,
// the maximum slot of block_reduce, stays 0).
__global__ void __launch_bounds__(kThreads) flux_pass1(const float* __restrict__ phi0,
                                                       const float* __restrict__ phi1,
                                                       const float* __restrict__ ua, long long n,
                                                       double* __restrict__ partials) {
  __shared__ double sh[kThreads / 32][kRec];
  double v[kRec] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float a0 = phi0[i], a1 = phi1[i], u = ua[i];
    if (!isfinite(a1) || !isfinite(u)) {
      v[7] += 1.0;
      continue;
    }
    if (a0 > 0.5f) continue;
    const double a2 = 1.0 - (double)a0 - (double)a1;
    v[0] += (double)a1 * u;
    v[1] += a2 * u;
    v[3] += u;
    v[4] += 1.0;
    v[5] += a1;
    v[6] += a2;
  }
  block_reduce(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < kRec; ++q) partials[(long long)blockIdx.x * kRec + q] = v[q];
  }
}

}  // namespace

cudaError_t launch_phase_flux(const float* phi0, const float* phi1, const float* ua, long long n, double* partials,
                              double* out, cudaStream_t s) {
  const int nb = obs_partials_blocks(n);
  flux_pass1<<<nb, kThreads, 0, s>>>(phi0, phi1, ua, n, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  obs_pass2<<<1, kThreads, 0, s>>>(partials, nb, out);
  return cudaGetLastError();
}

int obs_partials_blocks(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  if (b > kMaxBlocks) b = kMaxBlocks;
  if (b < 1) b = 1;
  return (int)b;
}

long long obs_partials_len(long long n) { return (long long)obs_partials_blocks(n) * kRec; }

cudaError_t launch_observables(const float* phi0, const float* phi1, const float* u, int d, const float* p,
                               long long n, double* partials, double* out, cudaStream_t s) {
  const int nb = obs_partials_blocks(n);
  obs_pass1<<<nb, kThreads, 0, s>>>(phi0, phi1, u, d, p, n, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  obs_pass2<<<1, kThreads, 0, s>>>(partials, nb, out);
  return cudaGetLastError();
}

}  // namespace lbm
