// Diagnostics reduction that allocates no device memory.
//
// Who needs this: code that may not call cudaMalloc at the moment it wants
// the diagnostics -- a solver embedded in a host application whose device
// memory is owned by that application's pool, a time-critical loop where
// cudaMalloc would synchronise the device, or a caller that has already
// spent its memory budget.  Such a caller passes its own field and output
// buffers; the per-CTA partial sums live in a fixed array compiled into the
// library instead of in memory allocated by the call.
//
// The array below is resident on every GPU that loads the library until the
// process exits.  All calls share it and it keeps whatever the last call left
// there; the first pass overwrites every record the second pass reads, so
// nothing has to be cleared between calls.  Two calls whose kernels overlap
// on the GPU (different streams, or graphs replayed concurrently) race on
// the array and may return wrong sums.
#include <cuda_runtime.h>

#include <math.h>
#include <stdio.h>

#include <mutex>

#include "../../include/lbm.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 4;                    // nodes per thread in pass 1
constexpr int kRec = 8;                          // doubles per partial record
constexpr long long kMaxRecords = 16384;         // 1 MiB of float64 records
constexpr long long kNodesPerRecord = (long long)kThreads * kPerThread;
constexpr long long kMaxNodes = kMaxRecords * kNodesPerRecord;   // 16,777,216
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_partials[kMaxRecords * kRec];

std::mutex g_setup_mutex;
double* g_partials_addr[kMaxDevices] = {};

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

// slot 2 is a maximum, the others sums; result in thread 0
__device__ void reduce_block(double (&v)[kRec]) {
  __shared__ double sh[kThreads / 32][kRec];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kRec; ++q) v[q] = (q == 2) ? warp_max(v[q]) : warp_sum(v[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < kRec; ++q) sh[warp][q] = v[q];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < kRec; ++q) {
      const double x = lane < kThreads / 32 ? sh[lane][q] : 0.0;
      v[q] = (q == 2) ? warp_max(x) : warp_sum(x);
    }
  }
}

// pass 1: CTA k reduces nodes [k * 1024, (k + 1) * 1024) into record k
__global__ void __launch_bounds__(kThreads) tile_sums(const float* __restrict__ phi0, const float* __restrict__ phi1,
                                                      const float* __restrict__ u, int d,
                                                      const float* __restrict__ p, long long n,
                                                      double* __restrict__ partials) {
  double v[kRec] = {0, 0, 0, 0, 0, 0, 0, 0};
  const long long base = (long long)blockIdx.x * kNodesPerRecord;
#pragma unroll
  for (int j = 0; j < kPerThread; ++j) {
    const long long i = base + (long long)j * kThreads + threadIdx.x;
    if (i < n) {
      const float a0 = phi0[i], a1 = phi1[i], pv = p[i];
      float u2 = 0.f;
      for (int q = 0; q < d; ++q) {
        const float uq = u[(long long)q * n + i];
        u2 += uq * uq;
      }
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
  }
  reduce_block(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < kRec; ++q) partials[(long long)blockIdx.x * kRec + q] = v[q];
  }
}

// pass 2: one CTA folds the records in a fixed order
__global__ void __launch_bounds__(kThreads) fold_records(const double* __restrict__ partials, int nrec,
                                                         double* __restrict__ out) {
  double v[kRec] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int r = threadIdx.x; r < nrec; r += kThreads) {
#pragma unroll
    for (int q = 0; q < kRec; ++q) {
      const double x = partials[(long long)r * kRec + q];
      v[q] = (q == 2) ? fmax(v[q], x) : v[q] + x;
    }
  }
  reduce_block(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < kRec; ++q) out[q] = v[q];
  }
}

// Device address of the record array on the current device (looked up once per device).
int partials_on_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_ECUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partials_addr[dev]) {
    void* addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_partials) != cudaSuccess || !addr) return LBM_ECUDA;
    g_partials_addr[dev] = static_cast<double*>(addr);
  }
  *out = g_partials_addr[dev];
  return LBM_OK;
}

}  // namespace

extern "C" int lbm_observables_noalloc(const float* phi0, const float* phi1, const float* u, int d, const float* p,
                                       long long n, double* out, void* stream) {
  if (n < 1 || n > kMaxNodes) return LBM_EINVAL;   // beyond the fixed record array
  if (!phi0 || !phi1 || !u || !p || !out || d < 1 || d > 3) return LBM_EINVAL;
  // an error left by earlier work on this device is reported, not cleared, so the caller can still read it
  if (cudaPeekAtLastError() != cudaSuccess) return LBM_ECUDA;
  double* partials = nullptr;
  if (int s = partials_on_current_device(&partials)) return s;
  const int nrec = (int)((n + kNodesPerRecord - 1) / kNodesPerRecord);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  tile_sums<<<nrec, kThreads, 0, st>>>(phi0, phi1, u, d, p, n, partials);
  if (cudaPeekAtLastError() != cudaSuccess) return LBM_ECUDA;
  fold_records<<<1, kThreads, 0, st>>>(partials, nrec, out);
  if (cudaPeekAtLastError() != cudaSuccess) return LBM_ECUDA;
  return LBM_OK;
}
