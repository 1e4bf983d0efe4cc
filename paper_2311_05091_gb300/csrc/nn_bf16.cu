// Kernels of the learned warm start: a small convolutional encoder-decoder
// that maps (solid indicator, initial phase field, cos theta) to a phase field
// close to equilibrium, followed by plain lattice Boltzmann relaxation.  The
// network is not part of the paper; it is a throughput device for the
// method (the paper's steps still decide the final state).
//
// Tensors are NHWC float32 in memory (pixel p = (n h + y) w + x, channel
// innermost).  3x3 convolutions run on the tensor cores with BF16 operands
// and FP32 accumulation: the forward (and data-gradient) convolution with
// tcgen05.mma and a TMEM accumulator, the weight gradient likewise with
// both operands MN-major; activations are rounded to BF16 as they enter a convolution,
// weights are kept as a BF16 copy of FP32 master weights.  Weight layout: wt[tap][cout][cin], tap = 3 ky + kx, so a
// pair of input channels is one 32-bit word.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "../../include/lbm_nn.h"

namespace {

constexpr int kThreads = 128;
constexpr int kProjectPasses = 3;   // mass-correction passes of lbm_nn_project

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// ---------------------------------------------------------------------------
// forward: y[p][co] = act(b[co] + sum_{tap, ci} x[p + shift(tap)][ci] wt[tap][co][ci])
//
// Implicit GEMM on the 5th-generation tensor cores: D (128 output pixels x N
// output channels, FP32 in TMEM) += A_tap (128 x 16 input channels, BF16) *
// B_tap^T (N x 16) for the nine taps and every chunk of 16 input channels.
// The 128 pixels of a CTA are R image rows of W = 128 / R columns (W = 128,
// 64, 32 or 16, the smallest that covers the image width, so narrow levels
// keep the M = 128 tile full).  Per chunk the CTA stages in shared memory, as
// BF16 in the canonical K-major layout without swizzle (core matrices of 8
// rows x 16 bytes; rows 16 bytes apart, 8-row groups 128 bytes apart, the
// two 8-channel halves of the chunk LBO bytes apart):
//   A: for each column offset kx, rows y0 - 1 .. y0 + R of the input at
//      columns x0 + kx - 1 .. x0 + kx - 2 + W (zero outside the image), so
//      that tap (ky, kx) is the 128-row window starting at row ky of copy kx;
//   B: the weights of all nine taps, [tap][half][co].
// One thread issues the nine tcgen05.mma of the chunk and commits them to the
// stage's mbarrier; with two stages the next chunk is staged while the tensor
// cores work; a stage is refilled only after the bounded wait for the
// products that read it.  The epilogue reads the accumulator with tcgen05.ld
// (warp w owns TMEM lanes 32 w .. 32 w + 31 = pixels), adds the bias, applies
// the ReLU and stores FP32.  grid (segments, cout / N), 128 threads.
// ---------------------------------------------------------------------------
__device__ unsigned int g_nn_fault = 0;    // set when a bounded wait on the tensor cores gave up

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, K-major, start / LBO / SBO in bytes
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t umma_idesc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// bounded wait for the completion of phase `parity` of an mbarrier; false when it gave up
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < (1 << 24) && !done; ++it)
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity));
  return done != 0;
}

constexpr int kTcM = 128;
constexpr int kTcThreads = 256;   // 8 warps stage the tiles; warps w and w + 4 share TMEM lane quarter w % 4
constexpr int kFwdBatch = 3;      // staging items whose loads a thread has in flight at once

// (A, B) tiles in S stages: with two, one chunk is staged while the tensor cores multiply the previous one.
// Two stages pay only where the tiles are small enough to keep several CTAs per SM (measured on GB300: wide
// images with N <= 64 gain 5-12 %, the 128-channel tiles lose up to 35 % when their occupancy halves).
// A holds at most 24 KB: WIDE 2 x 3 x 130 x 16 bytes; otherwise 6 (R + 2) W 16 <= 24576 bytes (R = 2).
template <int N, bool WIDE>
struct FwdTcSmem {
  static constexpr int S = (WIDE && N <= 64) ? 2 : 1;
  static constexpr int kA = WIDE ? 13312 : 24576;
  static constexpr int kB = 9 * 2 * N * 16;
  static constexpr int kStage = kA + kB;
  static constexpr int bytes() { return S * kStage + 64; }
};

// WIDE (one image row of 128 columns per CTA): a single copy of the three input rows with one halo column each
// side, [half][row][column] x 16 bytes; the window of tap (ky, kx) starts at row ky, column kx, i.e. 16 kx bytes
// further, and its 128 rows stay 16 bytes apart.  Otherwise (R > 1 rows per CTA) the rows of the window cross
// image rows, so the input is staged once per column offset kx as described above.
template <int N, bool WIDE>
__global__ void __launch_bounds__(kTcThreads) conv3x3_fwd_tc(const float* __restrict__ x,
                                                           const __nv_bfloat16* __restrict__ wt,
                                                           const float* __restrict__ bias, float* __restrict__ y,
                                                           int n, int h, int w, int cin, int cout, int relu,
                                                           int R) {
  extern __shared__ __align__(1024) unsigned char smem[];
  using SM = FwdTcSmem<N, WIDE>;
  constexpr int S = SM::S;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + S * SM::kStage);   // one mbarrier per stage
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int W = kTcM / R;
  const int segx = (w + W - 1) / W, segy = (h + R - 1) / R;
  const int sx = blockIdx.x % segx, sy = (blockIdx.x / segx) % segy, img = blockIdx.x / (segx * segy);
  const int x0 = sx * W, y0 = sy * R;
  const int co0 = blockIdx.y * N;
  const uint32_t bar0 = smem_addr(bar);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "r"(N < 32 ? 32 : N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int k = 0; k < S; ++k) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar0 + 8 * k), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(tslot);

  const int rows = R + 2;
  const int pitch = WIDE ? W + 2 : W;                    // staged columns per row
  const uint32_t lbo_a = (uint32_t)(rows * pitch * 16), lbo_b = (uint32_t)(N * 16);
  const int nchunks = cin / 16;
  bool ok = true;
  for (int c = 0; c < nchunks; ++c) {
    const int ci0 = c * 16, st = c % S;
    unsigned char* sA = smem + st * SM::kStage;
    unsigned char* sB = sA + SM::kA;
    // the products of chunk c - S read this stage: wait for them (phase (c - S) / S of this stage's barrier)
    if (c >= S) ok = ok && mbar_wait(bar0 + 8 * st, ((c - S) / S) & 1);
    // B: the BF16 weights of the nine taps, copied asynchronously (16 bytes, no register round trip)
    for (int e = tid; e < 18 * N; e += kTcThreads) {
      const int co = e % N, kc = (e / N) & 1, tap = e / (2 * N);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(sB + ((tap * 2 + kc) * N + co) * 16)),
                   "l"(wt + ((long long)tap * cout + co0 + co) * cin + ci0 + 8 * kc)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    // A: WIDE, one copy of rows y0 - 1 .. y0 + 1 at columns x0 - 1 .. x0 + 128; else one copy per kx.  The global
    // loads of kFwdBatch items per thread are issued before their conversions and shared stores (a store may not
    // be moved above a later load through pointers that could alias)
    const int nA = (WIDE ? 2 : 6) * rows * pitch;
    for (int e0 = 0; e0 < nA; e0 += kFwdBatch * kTcThreads) {
      float4 pv[kFwdBatch], qv[kFwdBatch];
      int off[kFwdBatch];   // destination byte offset from sA, -1: none
#pragma unroll
      for (int k = 0; k < kFwdBatch; ++k) {
        const int e = e0 + k * kTcThreads + tid;
        off[k] = -1;
        pv[k] = qv[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e < nA) {
          const int px = e % pitch, r = (e / pitch) % rows, kc = (e / (pitch * rows)) & 1;
          const int kx = WIDE ? 0 : e / (pitch * rows * 2);
          const int yy = y0 + r - 1, xc = x0 + px + kx - 1;
          off[k] = (((kx * 2 + kc) * rows + r) * pitch + px) * 16;
          if (yy >= 0 && yy < h && xc >= 0 && xc < w) {
            const float* src = x + (((long long)img * h + yy) * w + xc) * cin + ci0 + 8 * kc;
            pv[k] = __ldg(reinterpret_cast<const float4*>(src));
            qv[k] = __ldg(reinterpret_cast<const float4*>(src + 4));
          }
        }
      }
#pragma unroll
      for (int k = 0; k < kFwdBatch; ++k)
        if (off[k] >= 0)
          *reinterpret_cast<uint4*>(sA + off[k]) =
              make_uint4(pack_bf16(pv[k].x, pv[k].y), pack_bf16(pv[k].z, pv[k].w), pack_bf16(qv[k].x, qv[k].y),
                         pack_bf16(qv[k].z, qv[k].w));
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;");       // generic-proxy stores visible to the tensor cores
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0 && ok) {
      constexpr uint32_t idesc = umma_idesc(kTcM, N);
#pragma unroll 1
      for (int tap = 0; tap < 9; ++tap) {
        const int ky = tap / 3, kx = tap % 3;
        const uint64_t ad = WIDE ? umma_desc(smem_addr(sA + (ky * pitch + kx) * 16), lbo_a, 128)
                                 : umma_desc(smem_addr(sA + ((kx * 2) * rows + ky) * W * 16), lbo_a, 128);
        const uint64_t bd = umma_desc(smem_addr(sB + tap * 2 * N * 16), lbo_b, 128);
        const uint32_t acc = (c > 0 || tap > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar0 + 8 * st));
    }
  }
  // the last commit completes after every product issued before it
  ok = ok && mbar_wait(bar0 + 8 * ((nchunks - 1) % S), ((nchunks - 1) / S) & 1);
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    const int q = warp & 3;                                // TMEM lane quarter of this warp
    const int m = q * 32 + lane;
    const int yo = y0 + m / W, xo = x0 + m % W;
    const bool valid = yo < h && xo < w;
    float* dst = y + (((long long)img * h + yo) * w + xo) * cout + co0;
    constexpr int HALF = N / 2;                            // warps 0-3 take columns 0 .. N/2, warps 4-7 the rest
#pragma unroll 1
    for (int c0 = (warp >> 2) * HALF; c0 < (warp >> 2) * HALF + HALF; c0 += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (valid) {
#pragma unroll
        for (int j = 0; j < 16; j += 4) {
          float4 o;
          o.x = __uint_as_float(r[j]) + (bias ? bias[co0 + c0 + j] : 0.f);
          o.y = __uint_as_float(r[j + 1]) + (bias ? bias[co0 + c0 + j + 1] : 0.f);
          o.z = __uint_as_float(r[j + 2]) + (bias ? bias[co0 + c0 + j + 2] : 0.f);
          o.w = __uint_as_float(r[j + 3]) + (bias ? bias[co0 + c0 + j + 3] : 0.f);
          if (relu) {
            o.x = fmaxf(o.x, 0.f);
            o.y = fmaxf(o.y, 0.f);
            o.z = fmaxf(o.z, 0.f);
            o.w = fmaxf(o.w, 0.f);
          }
          *reinterpret_cast<float4*>(dst + c0 + j) = o;
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(&g_nn_fault, 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(N < 32 ? 32 : N));
}

// ---------------------------------------------------------------------------
// weight gradient on the 5th-generation tensor cores, per chunk z of W-pixel row segments (W = 64, or 32 on
// images narrower than 64):
//   part[z][tap][co][ci] = sum_{p in chunk z} dy[p][co] x[p + shift(tap)][ci]
// A CTA owns 128 output channels x 32 input channels of the three taps (ky, 0..2) of one kernel row ky:
// D_kx (128 x 32, FP32 in TMEM columns 32 kx ..) += A (128 co x 16 pixels) * B_kx^T (32 ci x 16 pixels),
// sixteen pixels of the chunk at a time.  The reduction runs over pixels, and both tensors keep their channels
// innermost, so both operands are staged as BF16 in the canonical MN-major layout without swizzle: core
// matrices of 8 pixels x 16 bytes (8 channels), the pixels of a segment 16 bytes apart (consecutive core
// matrices along K 128 bytes apart), the 8-channel groups SBO bytes apart:
//   A: dy of the segment's W pixels, [co group][pixel];
//   B: x of image row y + ky - 1 at columns x0 - 1 .. x0 + W, [ci group][column]; tap kx is the window that
//      starts kx columns (16 kx bytes) further.
// Channels beyond cout or cin and pixels outside the image are zero.  Two stages as in the forward kernel:
// a stage is refilled only after the bounded wait for the products that read it.
// grid (cout tiles of 128, 3 x cin tiles of 32, chunks), 256 threads.
// ---------------------------------------------------------------------------
constexpr int kWtM = 128, kWtN = 32, kWtThreads = 256, kWtBatch = 4;

template <int W>
struct WgTcSmem {
  static constexpr int kA = (kWtM / 8) * W * 16;
  static constexpr int kB = (kWtN / 8) * (W + 2) * 16;
  static constexpr int kStage = kA + kB;
  static constexpr int bytes() { return 2 * kStage + 64; }
};

// instruction descriptor of kind::f16 with both operands MN-major (transpose bits 15 and 16)
__host__ __device__ constexpr uint32_t umma_idesc_mn(int m, int n) { return umma_idesc(m, n) | (1u << 15) | (1u << 16); }

template <int W>
__global__ void __launch_bounds__(kWtThreads) conv3x3_wgrad_tc(const float* __restrict__ x,
                                                             const float* __restrict__ dy,
                                                             float* __restrict__ part, int n, int h, int w,
                                                             int cin, int cout, long long segs_per_chunk) {
  extern __shared__ __align__(1024) unsigned char smem[];
  using SM = WgTcSmem<W>;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * SM::kStage);   // one mbarrier per stage
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int co0 = blockIdx.x * kWtM;
  const int ky = blockIdx.y % 3, ci0 = (blockIdx.y / 3) * kWtN;
  const int spr = (w + W - 1) / W;                           // segments per image row
  const long long nseg = (long long)n * h * spr;
  const long long s0 = (long long)blockIdx.z * segs_per_chunk;
  const long long s1 = min(nseg, s0 + segs_per_chunk);
  const int cga = min(kWtM, cout - co0) / 8, cgb = min(kWtN, cin - ci0) / 8;   // channel groups present
  const uint32_t bar0 = smem_addr(bar);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "r"(128));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int k = 0; k < 2; ++k) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar0 + 8 * k), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  // the channel groups that are not present stay zero in both stages
  for (int st = 0; st < 2; ++st) {
    unsigned char* sA = smem + st * SM::kStage;
    for (int e = tid; e < (kWtM / 8 - cga) * W; e += kWtThreads)
      *reinterpret_cast<uint4*>(sA + (cga * W + e) * 16) = make_uint4(0u, 0u, 0u, 0u);
    for (int e = tid; e < (kWtN / 8 - cgb) * (W + 2); e += kWtThreads)
      *reinterpret_cast<uint4*>(sA + SM::kA + (cgb * (W + 2) + e) * 16) = make_uint4(0u, 0u, 0u, 0u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(tslot);

  bool ok = true;
  long long it = 0;
  for (long long sg = s0; sg < s1; ++sg, ++it) {
    const int st = (int)(it & 1);
    unsigned char* sA = smem + st * SM::kStage;
    unsigned char* sB = sA + SM::kA;
    // the products of segment it - 2 read this stage: wait for them (phase (it - 2) / 2 of its barrier)
    if (it >= 2) ok = ok && mbar_wait(bar0 + 8 * st, (uint32_t)(((it - 2) >> 1) & 1));
    const int img = (int)(sg / ((long long)h * spr));
    const int y = (int)((sg / spr) % h);
    const int x0 = (int)(sg % spr) * W;
    // A: dy of pixels x0 .. x0 + W - 1 of row y, then B: x of row y + ky - 1 at columns x0 - 1 .. x0 + W, in
    // batches of kWtBatch items per thread whose global loads are all issued before the first conversion and
    // shared store (a store may not be moved above a later load through pointers that could alias)
    const int yy = y + ky - 1;
    const bool row_in = yy >= 0 && yy < h;
    const int nA = cga * W, nAB = nA + cgb * (W + 2);
    for (int e0 = 0; e0 < nAB; e0 += kWtBatch * kWtThreads) {
      float4 pv[kWtBatch], qv[kWtBatch];
      int off[kWtBatch];   // destination byte offset from sA, -1: none
#pragma unroll
      for (int k = 0; k < kWtBatch; ++k) {
        const int e = e0 + k * kWtThreads + tid;
        const float* src = nullptr;
        off[k] = -1;
        if (e < nA) {
          const int px = e % W, cg = e / W;
          const int xc = x0 + px;
          if (xc < w) src = dy + (((long long)img * h + y) * w + xc) * cout + co0 + 8 * cg;
          off[k] = (cg * W + px) * 16;
        } else if (e < nAB) {
          const int j = (e - nA) % (W + 2), cg = (e - nA) / (W + 2);
          const int xc = x0 + j - 1;
          if (row_in && xc >= 0 && xc < w) src = x + (((long long)img * h + yy) * w + xc) * cin + ci0 + 8 * cg;
          off[k] = SM::kA + (cg * (W + 2) + j) * 16;
        }
        pv[k] = qv[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (src) {
          pv[k] = __ldg(reinterpret_cast<const float4*>(src));
          qv[k] = __ldg(reinterpret_cast<const float4*>(src + 4));
        }
      }
#pragma unroll
      for (int k = 0; k < kWtBatch; ++k)
        if (off[k] >= 0)
          *reinterpret_cast<uint4*>(sA + off[k]) =
              make_uint4(pack_bf16(pv[k].x, pv[k].y), pack_bf16(pv[k].z, pv[k].w), pack_bf16(qv[k].x, qv[k].y),
                         pack_bf16(qv[k].z, qv[k].w));
    }
    asm volatile("fence.proxy.async.shared::cta;");       // generic-proxy stores visible to the tensor cores
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0 && ok) {
      constexpr uint32_t idesc = umma_idesc_mn(kWtM, kWtN);
#pragma unroll 1
      for (int kx = 0; kx < 3; ++kx) {
#pragma unroll
        for (int ks = 0; ks < W / 16; ++ks) {
          // MN-major, no swizzle: LBO = stride of core matrices along K, SBO = along M / N
          const uint64_t ad = umma_desc(smem_addr(sA + ks * 256), 128, W * 16);
          const uint64_t bd = umma_desc(smem_addr(sB + (kx + 16 * ks) * 16), 128, (W + 2) * 16);
          const uint32_t acc = (it > 0 || ks > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + 32u * kx),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar0 + 8 * st));
    }
  }
  // the last commit completes after every product issued before it
  if (it > 0) ok = ok && mbar_wait(bar0 + 8 * (int)((it - 1) & 1), (uint32_t)(((it - 1) >> 1) & 1));
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    // warps w and w + 4 read TMEM lanes 32 (w % 4) .. + 31 (= output channels); of the six 16-column blocks
    // (kx = block / 2) warps 0-3 take the first three, warps 4-7 the others
    const int q = warp & 3;
    const int co = co0 + q * 32 + lane;
#pragma unroll 1
    for (int blk = 3 * (warp >> 2); blk < 3 * (warp >> 2) + 3; ++blk) {
      const int kx = blk >> 1, c0 = (blk & 1) * 16;
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(32 * kx + c0)));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (co < cout && c0 < cgb * 8) {
        float* dst = part + (((long long)blockIdx.z * 9 + 3 * ky + kx) * cout + co) * cin + ci0 + c0;
#pragma unroll
        for (int j = 0; j < 16; j += 4) {
          const float4 o = it > 0 ? make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                                __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]))
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
          *reinterpret_cast<float4*>(dst + j) = o;
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(&g_nn_fault, 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
}

// ---------------------------------------------------------------------------
// weight gradient for at most 64 output channels: the three kernel rows folded into the 128 rows of M, 32
// output channels per CTA.
// With q = p + shift(tap), part[z][tap][co][ci] = sum_q dy[q - shift(tap)][co] x[q][ci]: for a segment of W
// pixels q of row y, B is x of those pixels (32 input channels, unshifted) and A row (ky, co), 32 ky + co, is dy
// of image row y - ky + 1, so one product per column offset kx covers the three kernel rows:
// D_kx (128 x 32, rows 96 .. 127 zero, TMEM columns 32 kx ..) += A_kx (128 x 16 pixels) * B^T (32 x 16 pixels).
// Both operands are BF16 in the canonical MN-major layout without swizzle, as in conv3x3_wgrad_tc:
//   A: [ky][co group][column] for columns x0 - 1 .. x0 + W of dy rows y + 1, y, y - 1; the window of kx starts
//      2 - kx columns (16 (2 - kx) bytes) in;
//   B: [ci group][pixel] for pixels x0 .. x0 + W - 1 of x row y.
// grid (cout tiles of 32, cin tiles of 32, chunks), 256 threads, two stages.
// ---------------------------------------------------------------------------
template <int W>
struct WgRowsSmem {
  static constexpr int kA = (kWtM / 8) * (W + 2) * 16;
  static constexpr int kB = (kWtN / 8) * W * 16;
  static constexpr int kStage = kA + kB;
  static constexpr int bytes() { return 2 * kStage + 64; }
};

template <int W>
__global__ void __launch_bounds__(kWtThreads) conv3x3_wgrad_tc_rows(const float* __restrict__ x,
                                                                  const float* __restrict__ dy,
                                                                  float* __restrict__ part, int n, int h, int w,
                                                                  int cin, int cout, long long segs_per_chunk) {
  extern __shared__ __align__(1024) unsigned char smem[];
  using SM = WgRowsSmem<W>;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * SM::kStage);   // one mbarrier per stage
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int co0 = blockIdx.x * 32, ci0 = blockIdx.y * kWtN;
  const int spr = (w + W - 1) / W;                           // segments per image row
  const long long nseg = (long long)n * h * spr;
  const long long s0 = (long long)blockIdx.z * segs_per_chunk;
  const long long s1 = min(nseg, s0 + segs_per_chunk);
  const int cga = min(32, cout - co0) / 8, cgb = min(kWtN, cin - ci0) / 8;   // channel groups present
  const uint32_t bar0 = smem_addr(bar);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "r"(128));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int k = 0; k < 2; ++k) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar0 + 8 * k), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  // both stages start zero: the channel groups that are not present, and rows 96 .. 127 of A, stay so
  for (int e = tid; e < 2 * SM::kStage / 16; e += kWtThreads)
    *reinterpret_cast<uint4*>(smem + 16 * e) = make_uint4(0u, 0u, 0u, 0u);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(tslot);

  bool ok = true;
  long long it = 0;
  for (long long sg = s0; sg < s1; ++sg, ++it) {
    const int st = (int)(it & 1);
    unsigned char* sA = smem + st * SM::kStage;
    // the products of segment it - 2 read this stage: wait for them (phase (it - 2) / 2 of its barrier)
    if (it >= 2) ok = ok && mbar_wait(bar0 + 8 * st, (uint32_t)(((it - 2) >> 1) & 1));
    const int img = (int)(sg / ((long long)h * spr));
    const int y = (int)((sg / spr) % h);
    const int x0 = (int)(sg % spr) * W;
    // A: dy rows y + 1, y, y - 1 (ky = 0, 1, 2) at columns x0 - 1 .. x0 + W; then B: x row y at x0 .. x0 + W - 1.
    // The global loads of kWtBatch items per thread are issued before their conversions and shared stores.
    const int nA = 3 * cga * (W + 2), nAB = nA + cgb * W;
    for (int e0 = 0; e0 < nAB; e0 += kWtBatch * kWtThreads) {
      float4 pv[kWtBatch], qv[kWtBatch];
      int off[kWtBatch];   // destination byte offset from sA, -1: none
#pragma unroll
      for (int k = 0; k < kWtBatch; ++k) {
        const int e = e0 + k * kWtThreads + tid;
        const float* src = nullptr;
        off[k] = -1;
        if (e < nA) {
          const int j = e % (W + 2), cg = (e / (W + 2)) % cga, ky = e / ((W + 2) * cga);
          const int yy = y - ky + 1, xc = x0 + j - 1;
          if (yy >= 0 && yy < h && xc >= 0 && xc < w)
            src = dy + (((long long)img * h + yy) * w + xc) * cout + co0 + 8 * cg;
          off[k] = ((ky * 4 + cg) * (W + 2) + j) * 16;
        } else if (e < nAB) {
          const int j = (e - nA) % W, cg = (e - nA) / W;
          const int xc = x0 + j;
          if (xc < w) src = x + (((long long)img * h + y) * w + xc) * cin + ci0 + 8 * cg;
          off[k] = SM::kA + (cg * W + j) * 16;
        }
        pv[k] = qv[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (src) {
          pv[k] = __ldg(reinterpret_cast<const float4*>(src));
          qv[k] = __ldg(reinterpret_cast<const float4*>(src + 4));
        }
      }
#pragma unroll
      for (int k = 0; k < kWtBatch; ++k)
        if (off[k] >= 0)
          *reinterpret_cast<uint4*>(sA + off[k]) =
              make_uint4(pack_bf16(pv[k].x, pv[k].y), pack_bf16(pv[k].z, pv[k].w), pack_bf16(qv[k].x, qv[k].y),
                         pack_bf16(qv[k].z, qv[k].w));
    }
    asm volatile("fence.proxy.async.shared::cta;");       // generic-proxy stores visible to the tensor cores
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0 && ok) {
      constexpr uint32_t idesc = umma_idesc_mn(kWtM, kWtN);
#pragma unroll 1
      for (int kx = 0; kx < 3; ++kx) {
#pragma unroll
        for (int ks = 0; ks < W / 16; ++ks) {
          const uint64_t ad = umma_desc(smem_addr(sA + (2 - kx + 16 * ks) * 16), 128, (W + 2) * 16);
          const uint64_t bd = umma_desc(smem_addr(sA + SM::kA + ks * 256), 128, W * 16);
          const uint32_t acc = (it > 0 || ks > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + 32u * kx),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar0 + 8 * st));
    }
  }
  // the last commit completes after every product issued before it
  if (it > 0) ok = ok && mbar_wait(bar0 + 8 * (int)((it - 1) & 1), (uint32_t)(((it - 1) >> 1) & 1));
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    // warps w and w + 4 read TMEM lanes 32 (w % 4) .. + 31 = (ky = w % 4, co); lanes 96 .. 127 are the zero rows.
    // Of the six 16-column blocks (kx = block / 2) warps 0-3 take the first three, warps 4-7 the others.
    const int ky = warp & 3, co = co0 + lane;
#pragma unroll 1
    for (int blk = 3 * (warp >> 2); blk < 3 * (warp >> 2) + 3; ++blk) {
      const int kx = blk >> 1, c0 = (blk & 1) * 16;
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(tmem + ((uint32_t)(ky * 32) << 16) + (uint32_t)(32 * kx + c0)));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (ky < 3 && co < cout && c0 < cgb * 8) {
        float* dst = part + (((long long)blockIdx.z * 9 + 3 * ky + kx) * cout + co) * cin + ci0 + c0;
#pragma unroll
        for (int j = 0; j < 16; j += 4) {
          const float4 o = it > 0 ? make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                                __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]))
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
          *reinterpret_cast<float4*>(dst + j) = o;
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(&g_nn_fault, 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
}

// out[i] = sum_z part[z][i]: 8 lanes per output take the chunks z = lane, lane + 8, ... in order, then the 8 lane
// sums are added in a fixed tree (deterministic).  Block = 32 outputs x 8 lanes.
__global__ void __launch_bounds__(256) sum_parts(const float* __restrict__ part, float* __restrict__ out, long long n,
                                                 int chunks) {
  __shared__ float red[8][32];
  const int o = threadIdx.x & 31, lane = threadIdx.x >> 5;
  const long long i = (long long)blockIdx.x * 32 + o;
  float s = 0.f;
  if (i < n) {
#pragma unroll 4
    for (int z = lane; z < chunks; z += 8) s += part[(long long)z * n + i];
  }
  red[lane][o] = s;
  __syncthreads();
  if (lane == 0 && i < n)
    out[i] = ((red[0][o] + red[1][o]) + (red[2][o] + red[3][o])) + ((red[4][o] + red[5][o]) + (red[6][o] + red[7][o]));
}

// bias gradient partials: part[z][c] = sum_{p in chunk z} dy[p][c]; block = 32 channels x 8 pixel lanes,
// lanes combined in a fixed order (deterministic).  grid (ceil(c / 32), chunks)
__global__ void __launch_bounds__(256) colsum_part(const float* __restrict__ dy, float* __restrict__ part, long long P,
                                                   int c, long long chunk) {
  __shared__ float red[8][32];
  const int ch = blockIdx.x * 32 + (threadIdx.x & 31), r = threadIdx.x >> 5;
  const long long pb = (long long)blockIdx.y * chunk, pe = min(P, pb + chunk);
  float s = 0.f;
  if (ch < c) {
#pragma unroll 8
    for (long long p = pb + r; p < pe; p += 8) s += dy[p * c + ch];
  }
  red[r][threadIdx.x & 31] = s;
  __syncthreads();
  if (r == 0 && ch < c) {
    float v = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) v += red[k][threadIdx.x & 31];
    part[(long long)blockIdx.y * c + ch] = v;
  }
}

// wt'[tap][ci][co] = wt[8 - tap][co][ci]: the kernel of the data gradient
__global__ void flip_transpose(const __nv_bfloat16* __restrict__ wt, __nv_bfloat16* __restrict__ wf, int cin,
                               int cout) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = 9LL * cin * cout;
  if (i >= total) return;
  const int co = (int)(i % cout), ci = (int)((i / cout) % cin), tap = (int)(i / ((long long)cout * cin));
  wf[i] = wt[((long long)(8 - tap) * cout + co) * cin + ci];
}

// dx = dy where y > 0, else 0 (dx may be dy)
__global__ void relu_bwd(const float* dy, const float* __restrict__ y, float* dx, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dx[i] = y[i] > 0.f ? dy[i] : 0.f;
}

// 2x2 average pooling and its adjoint
__global__ void pool2_fwd(const float* __restrict__ x, float* __restrict__ y, int n, int h, int w, int c) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int h2 = h / 2, w2 = w / 2;
  if (i >= (long long)n * h2 * w2 * c) return;
  const int ch = (int)(i % c);
  const long long q = i / c;
  const int xx = (int)(q % w2), yy = (int)((q / w2) % h2), nn = (int)(q / ((long long)w2 * h2));
  const long long b = (((long long)nn * h + 2 * yy) * w + 2 * xx) * c + ch;
  y[i] = 0.25f * ((x[b] + x[b + c]) + (x[b + (long long)w * c] + x[b + (long long)w * c + c]));
}
__global__ void pool2_bwd(const float* __restrict__ dy, float* __restrict__ dx, int n, int h, int w, int c) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)n * h * w * c) return;
  const int ch = (int)(i % c);
  const long long q = i / c;
  const int xx = (int)(q % w), yy = (int)((q / w) % h), nn = (int)(q / ((long long)w * h));
  dx[i] = 0.25f * dy[(((long long)nn * (h / 2) + yy / 2) * (w / 2) + xx / 2) * c + ch];
}

// nearest 2x upsampling and its adjoint (h, w: the coarse size)
__global__ void up2_fwd(const float* __restrict__ x, float* __restrict__ y, int n, int h, int w, int c) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)n * 4 * h * w * c) return;
  const int ch = (int)(i % c);
  const long long q = i / c;
  const int xx = (int)(q % (2 * w)), yy = (int)((q / (2 * w)) % (2 * h)), nn = (int)(q / (4LL * w * h));
  y[i] = x[(((long long)nn * h + yy / 2) * w + xx / 2) * c + ch];
}
__global__ void up2_bwd(const float* __restrict__ dy, float* __restrict__ dx, int n, int h, int w, int c) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)n * h * w * c) return;
  const int ch = (int)(i % c);
  const long long q = i / c;
  const int xx = (int)(q % w), yy = (int)((q / w) % h), nn = (int)(q / ((long long)w * h));
  const long long b = (((long long)nn * 2 * h + 2 * yy) * 2 * w + 2 * xx) * c + ch;
  const long long row = 2LL * w * c;
  dx[i] = (dy[b] + dy[b + c]) + (dy[b + row] + dy[b + row + c]);
}

// The same four maps on float4 groups of channels with 32-bit index arithmetic (c4 = c / 4 groups; the callers
// use them when c % 4 == 0 and the element count fits 32 bits)
__global__ void pool2_fwd4(const float4* __restrict__ x, float4* __restrict__ y, int n, int h, int w, int c4) {
  const unsigned h2 = h / 2, w2 = w / 2;
  const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (unsigned)n * h2 * w2 * c4) return;
  const unsigned ch = i % c4, q = i / c4;
  const unsigned xx = q % w2, r = q / w2, yy = r % h2, nn = r / h2;
  const unsigned b = ((nn * h + 2 * yy) * w + 2 * xx) * c4 + ch, row = (unsigned)w * c4;
  const float4 a = x[b], bb = x[b + c4], cc = x[b + row], d = x[b + row + c4];
  y[i] = make_float4(0.25f * ((a.x + bb.x) + (cc.x + d.x)), 0.25f * ((a.y + bb.y) + (cc.y + d.y)),
                     0.25f * ((a.z + bb.z) + (cc.z + d.z)), 0.25f * ((a.w + bb.w) + (cc.w + d.w)));
}
__global__ void pool2_bwd4(const float4* __restrict__ dy, float4* __restrict__ dx, int n, int h, int w, int c4) {
  const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (unsigned)n * h * w * c4) return;
  const unsigned ch = i % c4, q = i / c4;
  const unsigned xx = q % w, r = q / w, yy = r % h, nn = r / h;
  const float4 v = dy[((nn * (h / 2) + yy / 2) * (w / 2) + xx / 2) * c4 + ch];
  dx[i] = make_float4(0.25f * v.x, 0.25f * v.y, 0.25f * v.z, 0.25f * v.w);
}
__global__ void up2_fwd4(const float4* __restrict__ x, float4* __restrict__ y, int n, int h, int w, int c4) {
  const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (unsigned)n * 4 * h * w * c4) return;
  const unsigned ch = i % c4, q = i / c4;
  const unsigned xx = q % (2 * w), r = q / (2 * w), yy = r % (2 * h), nn = r / (2 * h);
  y[i] = x[((nn * h + yy / 2) * w + xx / 2) * c4 + ch];
}
__global__ void up2_bwd4(const float4* __restrict__ dy, float4* __restrict__ dx, int n, int h, int w, int c4) {
  const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (unsigned)n * h * w * c4) return;
  const unsigned ch = i % c4, q = i / c4;
  const unsigned xx = q % w, r = q / w, yy = r % h, nn = r / h;
  const unsigned b = ((nn * 2 * h + 2 * yy) * 2 * w + 2 * xx) * c4 + ch, row = 2u * w * c4;
  const float4 a = dy[b], bb = dy[b + c4], cc = dy[b + row], d = dy[b + row + c4];
  dx[i] = make_float4((a.x + bb.x) + (cc.x + d.x), (a.y + bb.y) + (cc.y + d.y), (a.z + bb.z) + (cc.z + d.z),
                      (a.w + bb.w) + (cc.w + d.w));
}

// float4 forms of relu_bwd and add (n % 4 == 0, 16-byte aligned pointers)
__global__ void relu_bwd4(const float4* dy, const float4* __restrict__ y, float4* dx, long long n4) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n4) return;
  const float4 g = dy[i], v = y[i];
  dx[i] = make_float4(v.x > 0.f ? g.x : 0.f, v.y > 0.f ? g.y : 0.f, v.z > 0.f ? g.z : 0.f, v.w > 0.f ? g.w : 0.f);
}
__global__ void add4(float4* z, const float4* x, const float4* y, float a, long long n4) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n4) return;
  const float4 u = x[i], v = y[i];
  z[i] = make_float4(u.x + a * v.x, u.y + a * v.y, u.z + a * v.z, u.w + a * v.w);
}

// z = x + a y (z may be x or y)
__global__ void add(float* z, const float* x, const float* y, float a, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = x[i] + a * y[i];
}

// input tensor [p][16]: phi0, phi1, cos theta of the image, zeros
__global__ void pack_input(const float* __restrict__ phi0, const float* __restrict__ phi1,
                           const float* __restrict__ costh, float* __restrict__ x, int n, long long hw) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n * hw) return;
  float* o = x + p * 16;
  o[0] = phi0[p];
  o[1] = phi1[p];
  o[2] = costh[p / hw];
#pragma unroll
  for (int c = 3; c < 16; ++c) o[c] = 0.f;
}

// prediction = base + out[p][0]; loss partials (FP64) and d loss / d out = 2 (pred - target) / P in channel 0
__global__ void mse_residual(const float* __restrict__ out, int cpad, const float* __restrict__ base,
                             const float* __restrict__ target, float* __restrict__ dout, double* __restrict__ part,
                             long long P) {
  __shared__ double s[kThreads];
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double e2 = 0.0;
  if (p < P) {
    const float d = (base[p] + out[p * cpad]) - target[p];
    e2 = (double)d * d;
    dout[p * cpad] = 2.f * d / (float)P;
    for (int c = 1; c < cpad; ++c) dout[p * cpad + c] = 0.f;
  }
  s[threadIdx.x] = e2;
  __syncthreads();
  for (int k = kThreads / 2; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// out = sum of n partials: one CTA, strided per-thread sums, then a fixed-order tree (deterministic)
__global__ void __launch_bounds__(256) sum_double(const double* __restrict__ part, int n, double* __restrict__ out) {
  __shared__ double s[256];
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) v += part[i];
  s[threadIdx.x] = v;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

// Adam with bias correction; writes the BF16 copy of the updated weights
__global__ void adam_step(float* __restrict__ wm, float* __restrict__ m, float* __restrict__ v,
                          const float* __restrict__ grad, __nv_bfloat16* __restrict__ wb, long long n, float lr,
                          float b1, float b2, float eps, float c1, float c2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = grad[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = wm[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  wm[i] = wi;
  if (wb) wb[i] = __float2bfloat16_rn(wi);
}

__global__ void to_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

// warm-start projection.  hi = max(1 - phi0, 0); the bump b(q) = q (hi - q) / hi (0 where hi = 0) vanishes at
// both bounds, and for |lambda| <= 1 the map q -> q + lambda b(q) is monotone on [0, hi] with fixed points 0 and
// hi, so a correction step never leaves the bounds.
__device__ __forceinline__ float proj_bump(float q, float hi) { return hi > 0.f ? q * (hi - q) / hi : 0.f; }

// field = clamp(phi1 + out[p][0], 0, hi)
__global__ void project_init(const float* __restrict__ out, int cpad, const float* __restrict__ phi0,
                             const float* __restrict__ phi1, float* __restrict__ field, long long n) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const float hi = fmaxf(1.f - phi0[p], 0.f);
  field[p] = fminf(fmaxf(phi1[p] + out[p * cpad], 0.f), hi);
}

// per image and part: sums of phi1 (target mass), of the field and of its bump
__global__ void project_sums(const float* __restrict__ field, const float* __restrict__ phi0,
                             const float* __restrict__ phi1, double* __restrict__ sums, long long hw) {
  __shared__ double s[3][kThreads];
  const int img = blockIdx.y;
  double a = 0.0, b = 0.0, c = 0.0;
  for (long long k = (long long)blockIdx.x * kThreads + threadIdx.x; k < hw; k += (long long)gridDim.x * kThreads) {
    const long long p = img * hw + k;
    const float q = field[p];
    a += phi1[p];
    b += q;
    c += proj_bump(q, fmaxf(1.f - phi0[p], 0.f));
  }
  s[0][threadIdx.x] = a;
  s[1][threadIdx.x] = b;
  s[2][threadIdx.x] = c;
  __syncthreads();
  for (int k = kThreads / 2; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k)
      for (int j = 0; j < 3; ++j) s[j][threadIdx.x] += s[j][threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int j = 0; j < 3; ++j) sums[((long long)img * gridDim.x + blockIdx.x) * 3 + j] = s[j][0];
}

// field += lambda b(field), lambda = clamp((sum phi1 - sum field) / sum b, -1, 1) per image
__global__ void project_apply(const float* __restrict__ phi0, const double* __restrict__ sums, int parts,
                              float* __restrict__ field, long long hw) {
  const int img = blockIdx.y;
  double a = 0.0, b = 0.0, c = 0.0;
  for (int k = 0; k < parts; ++k) {
    a += sums[((long long)img * parts + k) * 3];
    b += sums[((long long)img * parts + k) * 3 + 1];
    c += sums[((long long)img * parts + k) * 3 + 2];
  }
  const float lam = c > 0.0 ? (float)fmin(1.0, fmax(-1.0, (a - b) / c)) : 0.f;
  for (long long k = (long long)blockIdx.x * kThreads + threadIdx.x; k < hw; k += (long long)gridDim.x * kThreads) {
    const long long p = img * hw + k;
    const float q = field[p];
    field[p] = q + lam * proj_bump(q, fmaxf(1.f - phi0[p], 0.f));
  }
}

unsigned blocks(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

int status(cudaError_t e) { return e == cudaSuccess ? 0 : -3; }

}  // namespace

extern "C" {

int lbm_nn_conv3x3(const float* x, const void* wt_bf16, const float* bias, float* y, int n, int h, int w, int cin,
                   int cout, int relu, void* stream) {
  if (!x || !wt_bf16 || !y || n < 1 || h < 1 || w < 1 || cin < 16 || cin % 16 || cout < 32 || cout % 32) return -1;
  // the opt-in above 48 KB of shared memory is a per-device attribute: set it once for each device used
  static unsigned long long attr_set = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -3;
  if (!(attr_set & (1ull << dev))) {
    bool good = true;
    auto opt_in = [&](const void* fn, int bytes) {
      good = good && cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess;
    };
    opt_in((const void*)conv3x3_fwd_tc<128, true>, FwdTcSmem<128, true>::bytes());
    opt_in((const void*)conv3x3_fwd_tc<64, true>, FwdTcSmem<64, true>::bytes());
    opt_in((const void*)conv3x3_fwd_tc<32, true>, FwdTcSmem<32, true>::bytes());
    opt_in((const void*)conv3x3_fwd_tc<128, false>, FwdTcSmem<128, false>::bytes());
    opt_in((const void*)conv3x3_fwd_tc<64, false>, FwdTcSmem<64, false>::bytes());
    opt_in((const void*)conv3x3_fwd_tc<32, false>, FwdTcSmem<32, false>::bytes());
    if (!good) return -3;
    attr_set |= 1ull << dev;
  }
  // R image rows of 128 / R columns per CTA: the narrowest tile that covers the width
  const int R = w > 64 ? 1 : (w > 32 ? 2 : (w > 16 ? 4 : 8));
  const int W = kTcM / R;
  const long long segs = (long long)n * ((h + R - 1) / R) * ((w + W - 1) / W);
  if (segs > 0x7fffffffLL) return -1;
  const auto* wb = static_cast<const __nv_bfloat16*>(wt_bf16);
  cudaStream_t s = (cudaStream_t)stream;
  const int N = cout % 128 == 0 ? 128 : (cout % 64 == 0 ? 64 : 32);
  const dim3 grid((unsigned)segs, cout / N);
  const bool wide = R == 1;
#define LBM_NN_FWD(NN, WD)                                                                                        \
  conv3x3_fwd_tc<NN, WD><<<grid, kTcThreads, FwdTcSmem<NN, WD>::bytes(), s>>>(x, wb, bias, y, n, h, w, cin, cout, relu, \
                                                                              R)
  if (N == 128) {
    if (wide) LBM_NN_FWD(128, true); else LBM_NN_FWD(128, false);
  } else if (N == 64) {
    if (wide) LBM_NN_FWD(64, true); else LBM_NN_FWD(64, false);
  } else {
    if (wide) LBM_NN_FWD(32, true); else LBM_NN_FWD(32, false);
  }
#undef LBM_NN_FWD
  return status(cudaGetLastError());
}

int lbm_nn_check(void) {
  unsigned int f = 0;
  if (cudaMemcpyFromSymbol(&f, g_nn_fault, sizeof f) != cudaSuccess) return -3;
  if (f) {
    const unsigned int zero = 0;
    cudaMemcpyToSymbol(g_nn_fault, &zero, sizeof zero);
    return -5;
  }
  return 0;
}

}  // extern "C"

namespace {

constexpr long long kBiasChunk = 4096;

// row segments per CTA of the weight gradient: at most four CTAs per SM (the TMEM of 4 x 128 columns) over the
// (co, ky, ci) tiles, so that every CTA is resident in one wave
struct WgradPlan {
  int W;
  long long segs, per_chunk, chunks, bias_chunks, tiles;
};

WgradPlan wgrad_plan(int n, int h, int w, int cin, int cout) {
  WgradPlan p;
  p.W = w >= 64 ? 64 : 32;
  p.segs = (long long)n * h * ((w + p.W - 1) / p.W);
  // at most 64 output channels: the kernel rows folded into M (a CTA per 32 x 32 channel tile); else a CTA per
  // kernel row and 128 x 32 tile
  p.tiles = cout <= 64 ? (long long)((cout + 31) / 32) * ((cin + kWtN - 1) / kWtN)
                       : (long long)((cout + kWtM - 1) / kWtM) * 3 * ((cin + kWtN - 1) / kWtN);
  const long long want = std::max(1LL, (4LL * 152) / p.tiles);
  p.per_chunk = std::max(1LL, (p.segs + want - 1) / want);
  p.chunks = (p.segs + p.per_chunk - 1) / p.per_chunk;
  p.bias_chunks = ((long long)n * h * w + kBiasChunk - 1) / kBiasChunk;
  return p;
}

}  // namespace

extern "C" {

long long lbm_nn_wgrad_workspace(int n, int h, int w, int cin, int cout) {
  if (n < 1 || h < 1 || w < 1 || cin < 1 || cout < 1) return 0;
  const WgradPlan p = wgrad_plan(n, h, w, cin, cout);
  return p.chunks * 9LL * cin * cout + p.bias_chunks * cout;
}

int lbm_nn_conv3x3_wgrad(const float* x, const float* dy, float* dw, float* db, float* work, long long work_len,
                         int n, int h, int w, int cin, int cout, void* stream) {
  if (!x || !dy || !dw || !work || n < 1 || h < 1 || w < 1 || cin < 16 || cin % 16 || cout < 16 || cout % 16)
    return -1;
  if (work_len < lbm_nn_wgrad_workspace(n, h, w, cin, cout)) return -1;
  cudaStream_t s = (cudaStream_t)stream;
  const WgradPlan p = wgrad_plan(n, h, w, cin, cout);
  const long long nw = 9LL * cin * cout;
  if (p.chunks > 65535) return -1;
  static unsigned long long attr_set = 0;   // shared-memory opt-in, per device
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -3;
  if (!(attr_set & (1ull << dev))) {
    if (cudaFuncSetAttribute((const void*)conv3x3_wgrad_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             WgTcSmem<64>::bytes()) != cudaSuccess ||
        cudaFuncSetAttribute((const void*)conv3x3_wgrad_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             WgTcSmem<32>::bytes()) != cudaSuccess ||
        cudaFuncSetAttribute((const void*)conv3x3_wgrad_tc_rows<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             WgRowsSmem<64>::bytes()) != cudaSuccess ||
        cudaFuncSetAttribute((const void*)conv3x3_wgrad_tc_rows<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             WgRowsSmem<32>::bytes()) != cudaSuccess)
      return -3;
    attr_set |= 1ull << dev;
  }
  if (cout <= 64) {
    const dim3 grid((cout + 31) / 32, (cin + kWtN - 1) / kWtN, (unsigned)p.chunks);
    if (p.W == 64)
      conv3x3_wgrad_tc_rows<64><<<grid, kWtThreads, WgRowsSmem<64>::bytes(), s>>>(x, dy, work, n, h, w, cin, cout,
                                                                                  p.per_chunk);
    else
      conv3x3_wgrad_tc_rows<32><<<grid, kWtThreads, WgRowsSmem<32>::bytes(), s>>>(x, dy, work, n, h, w, cin, cout,
                                                                                  p.per_chunk);
  } else {
    const dim3 grid((cout + kWtM - 1) / kWtM, 3 * ((cin + kWtN - 1) / kWtN), (unsigned)p.chunks);
    if (p.W == 64)
      conv3x3_wgrad_tc<64><<<grid, kWtThreads, WgTcSmem<64>::bytes(), s>>>(x, dy, work, n, h, w, cin, cout,
                                                                           p.per_chunk);
    else
      conv3x3_wgrad_tc<32><<<grid, kWtThreads, WgTcSmem<32>::bytes(), s>>>(x, dy, work, n, h, w, cin, cout,
                                                                           p.per_chunk);
  }
  sum_parts<<<(unsigned)((nw + 31) / 32), 256, 0, s>>>(work, dw, nw, (int)p.chunks);
  if (db) {
    float* bpart = work + p.chunks * nw;
    const long long P = (long long)n * h * w;
    colsum_part<<<dim3((cout + 31) / 32, (unsigned)p.bias_chunks), 256, 0, s>>>(dy, bpart, P, cout, kBiasChunk);
    sum_parts<<<(unsigned)((cout + 31) / 32), 256, 0, s>>>(bpart, db, cout, (int)p.bias_chunks);
  }
  return status(cudaGetLastError());
}

int lbm_nn_flip_transpose(const void* wt_bf16, void* wf_bf16, int cin, int cout, void* stream) {
  if (!wt_bf16 || !wf_bf16 || cin < 1 || cout < 1) return -1;
  flip_transpose<<<blocks(9LL * cin * cout), 256, 0, (cudaStream_t)stream>>>(
      static_cast<const __nv_bfloat16*>(wt_bf16), static_cast<__nv_bfloat16*>(wf_bf16), cin, cout);
  return status(cudaGetLastError());
}

int lbm_nn_relu_bwd(const float* dy, const float* y, float* dx, long long n, void* stream) {
  if (!dy || !y || !dx || n < 0) return -1;
  if (n % 4 == 0 && ((uintptr_t)dy | (uintptr_t)y | (uintptr_t)dx) % 16 == 0) {
    if (n)
      relu_bwd4<<<blocks(n / 4), 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<const float4*>(dy),
                                                                  reinterpret_cast<const float4*>(y),
                                                                  reinterpret_cast<float4*>(dx), n / 4);
  } else if (n) {
    relu_bwd<<<blocks(n), 256, 0, (cudaStream_t)stream>>>(dy, y, dx, n);
  }
  return status(cudaGetLastError());
}

int lbm_nn_pool2(const float* x, float* y, int n, int h, int w, int c, int backward, void* stream) {
  if (!x || !y || n < 1 || h < 2 || w < 2 || h % 2 || w % 2 || c < 1) return -1;
  cudaStream_t s = (cudaStream_t)stream;
  const long long total = (long long)n * h * w * c;
  if (c % 4 == 0 && total < (1LL << 31) && ((uintptr_t)x | (uintptr_t)y) % 16 == 0) {
    const int c4 = c / 4;
    if (!backward)
      pool2_fwd4<<<blocks(total / 16), 256, 0, s>>>(reinterpret_cast<const float4*>(x), reinterpret_cast<float4*>(y),
                                                     n, h, w, c4);
    else
      pool2_bwd4<<<blocks(total / 4), 256, 0, s>>>(reinterpret_cast<const float4*>(x), reinterpret_cast<float4*>(y),
                                                    n, h, w, c4);
  } else if (!backward) {
    pool2_fwd<<<blocks(total / 4), 256, 0, s>>>(x, y, n, h, w, c);
  } else {
    pool2_bwd<<<blocks(total), 256, 0, s>>>(x, y, n, h, w, c);
  }
  return status(cudaGetLastError());
}

int lbm_nn_up2(const float* x, float* y, int n, int h, int w, int c, int backward, void* stream) {
  if (!x || !y || n < 1 || h < 1 || w < 1 || c < 1) return -1;
  cudaStream_t s = (cudaStream_t)stream;
  const long long fine = 4LL * n * h * w * c;
  if (c % 4 == 0 && fine < (1LL << 31) && ((uintptr_t)x | (uintptr_t)y) % 16 == 0) {
    const int c4 = c / 4;
    if (!backward)
      up2_fwd4<<<blocks(fine / 4), 256, 0, s>>>(reinterpret_cast<const float4*>(x), reinterpret_cast<float4*>(y), n,
                                                 h, w, c4);
    else
      up2_bwd4<<<blocks(fine / 16), 256, 0, s>>>(reinterpret_cast<const float4*>(x), reinterpret_cast<float4*>(y), n,
                                                  h, w, c4);
  } else if (!backward) {
    up2_fwd<<<blocks(fine), 256, 0, s>>>(x, y, n, h, w, c);
  } else {
    up2_bwd<<<blocks(fine / 4), 256, 0, s>>>(x, y, n, h, w, c);
  }
  return status(cudaGetLastError());
}

int lbm_nn_add(float* z, const float* x, const float* y, float a, long long n, void* stream) {
  if (!z || !x || !y || n < 0) return -1;
  if (n % 4 == 0 && ((uintptr_t)z | (uintptr_t)x | (uintptr_t)y) % 16 == 0) {
    if (n)
      add4<<<blocks(n / 4), 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<float4*>(z),
                                                             reinterpret_cast<const float4*>(x),
                                                             reinterpret_cast<const float4*>(y), a, n / 4);
  } else if (n) {
    add<<<blocks(n), 256, 0, (cudaStream_t)stream>>>(z, x, y, a, n);
  }
  return status(cudaGetLastError());
}

int lbm_nn_pack_input(const float* phi0, const float* phi1, const float* costh, float* x, int n, int h, int w,
                      void* stream) {
  if (!phi0 || !phi1 || !costh || !x || n < 1 || h < 1 || w < 1) return -1;
  const long long hw = (long long)h * w;
  pack_input<<<blocks(n * hw), 256, 0, (cudaStream_t)stream>>>(phi0, phi1, costh, x, n, hw);
  return status(cudaGetLastError());
}

int lbm_nn_mse_residual(const float* out, int cpad, const float* base, const float* target, float* dout,
                        double* work, long long work_len, double* loss, long long P, void* stream) {
  if (!out || !base || !target || !dout || !work || !loss || P < 1 || cpad < 1) return -1;
  const int nb = (int)((P + kThreads - 1) / kThreads);
  if (work_len < nb) return -1;
  cudaStream_t s = (cudaStream_t)stream;
  mse_residual<<<nb, kThreads, 0, s>>>(out, cpad, base, target, dout, work, P);
  sum_double<<<1, 256, 0, s>>>(work, nb, loss);
  return status(cudaGetLastError());
}

int lbm_nn_adam(float* w, float* m, float* v, const float* grad, void* w_bf16, long long n, float lr, float b1,
                float b2, float eps, int t, void* stream) {
  if (!w || !m || !v || !grad || n < 0 || t < 1) return -1;
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  if (n)
    adam_step<<<blocks(n), 256, 0, (cudaStream_t)stream>>>(w, m, v, grad, static_cast<__nv_bfloat16*>(w_bf16), n, lr,
                                                           b1, b2, eps, c1, c2);
  return status(cudaGetLastError());
}

int lbm_nn_to_bf16(const float* a, void* b, long long n, void* stream) {
  if (!a || !b || n < 0) return -1;
  if (n) to_bf16<<<blocks(n), 256, 0, (cudaStream_t)stream>>>(a, static_cast<__nv_bfloat16*>(b), n);
  return status(cudaGetLastError());
}

int lbm_nn_project(const float* out, int cpad, const float* phi0, const float* phi1, float* field, double* work,
                   long long work_len, int n, int h, int w, void* stream) {
  if (!out || cpad < 1 || !phi0 || !phi1 || !field || !work || n < 1 || h < 1 || w < 1) return -1;
  const int parts = 64;
  if (work_len < 3LL * parts * n) return -1;
  const long long hw = (long long)h * w;
  cudaStream_t s = (cudaStream_t)stream;
  project_init<<<blocks(n * hw), 256, 0, s>>>(out, cpad, phi0, phi1, field, n * hw);
  for (int pass = 0; pass < kProjectPasses; ++pass) {
    project_sums<<<dim3(parts, n), kThreads, 0, s>>>(field, phi0, phi1, work, hw);
    project_apply<<<dim3(parts, n), kThreads, 0, s>>>(phi0, work, parts, field, hw);
  }
  return status(cudaGetLastError());
}

}  // extern "C"
