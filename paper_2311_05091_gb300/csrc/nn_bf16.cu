// Kernels of the learned warm start: a small convolutional encoder-decoder
// that maps (solid indicator, initial phase field, cos theta) to a phase field
// close to equilibrium, followed by plain lattice Boltzmann relaxation.  The
// network is not part of the paper; it is a throughput device for the
// method (the paper's steps stay the judge of the final state).
//
// Tensors are NHWC float32 in memory (pixel p = (n h + y) w + x, channel
// innermost).  3x3 convolutions run on the tensor cores with BF16 operands
// and FP32 accumulation (mma.sync m16n8k16): activations are rounded to BF16
// as they enter a convolution, weights are kept as a BF16 copy of FP32
// master weights.  Weight layout: wt[tap][cout][cin], tap = 3 ky + kx, so a
// pair of input channels is one 32-bit word.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lbm_nn.h"

namespace {

constexpr int kThreads = 128;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// neighbour of pixel p (image n, row y, column x) at tap (ky, kx), or -1 outside the image (zero padding)
__device__ __forceinline__ long long tap_pixel(long long p, int n, int y, int x, int h, int w, int ky, int kx) {
  const int yy = y + ky - 1, xx = x + kx - 1;
  if (p < 0 || yy < 0 || yy >= h || xx < 0 || xx >= w) return -1;
  return ((long long)n * h + yy) * w + xx;
}

// two consecutive channels of pixel q as one BF16 pair (zero outside)
__device__ __forceinline__ uint32_t load_pair(const float* __restrict__ x, long long q, int cin, int c) {
  if (q < 0) return 0u;
  const float2 v = *reinterpret_cast<const float2*>(x + q * cin + c);
  return pack_bf16(v.x, v.y);
}

// ---------------------------------------------------------------------------
// forward: y[p][co] = act(b[co] + sum_{tap, ci} x[p + shift(tap)][ci] wt[tap][co][ci])
// CTA: 4 warps x 16 pixels, 32 output channels; grid (ceil(P / 64), cout / 32)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) conv3x3_fwd(const float* __restrict__ x,
                                                        const __nv_bfloat16* __restrict__ wt,
                                                        const float* __restrict__ bias, float* __restrict__ y,
                                                        int n, int h, int w, int cin, int cout, int relu) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const long long P = (long long)n * h * w;
  const long long p0 = (long long)blockIdx.x * 64 + warp * 16;
  const int co0 = blockIdx.y * 32;
  long long pr[2];
  int pn[2], py[2], px[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const long long p = p0 + g + 8 * r;
    pr[r] = p < P ? p : -1;
    const long long q = p < P ? p : 0;
    px[r] = (int)(q % w);
    py[r] = (int)((q / w) % h);
    pn[r] = (int)(q / ((long long)w * h));
  }
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  const uint32_t* __restrict__ wt32 = reinterpret_cast<const uint32_t*>(wt);
  for (int tap = 0; tap < 9; ++tap) {
    const int ky = tap / 3, kx = tap % 3;
    const long long q0 = tap_pixel(pr[0], pn[0], py[0], px[0], h, w, ky, kx);
    const long long q1 = tap_pixel(pr[1], pn[1], py[1], px[1], h, w, ky, kx);
    for (int ci0 = 0; ci0 < cin; ci0 += 16) {
      uint32_t a[4];
      a[0] = load_pair(x, q0, cin, ci0 + 2 * t);
      a[1] = load_pair(x, q1, cin, ci0 + 2 * t);
      a[2] = load_pair(x, q0, cin, ci0 + 2 * t + 8);
      a[3] = load_pair(x, q1, cin, ci0 + 2 * t + 8);
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const long long wrow = ((long long)tap * cout + co0 + nt * 8 + g) * cin + ci0 + 2 * t;
        mma_bf16(acc[nt], a, wt32[wrow >> 1], wt32[(wrow + 8) >> 1]);
      }
    }
  }
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    const int co = co0 + nt * 8 + 2 * t;
    const float b0 = bias ? bias[co] : 0.f, b1 = bias ? bias[co + 1] : 0.f;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      if (pr[r] < 0) continue;
      float v0 = acc[nt][2 * r] + b0, v1 = acc[nt][2 * r + 1] + b1;
      if (relu) {
        v0 = fmaxf(v0, 0.f);
        v1 = fmaxf(v1, 0.f);
      }
      *reinterpret_cast<float2*>(y + pr[r] * cout + co) = make_float2(v0, v1);
    }
  }
}

// ---------------------------------------------------------------------------
// weight gradient, per pixel chunk z:
//   part[z][tap][co][ci] = sum_{p in chunk z} dy[p][co] x[p + shift(tap)][ci]
// CTA: 4 warps over 16 output channels x up to 32 input channels; each warp
// takes every fourth group of 16 pixels of the chunk; the four partial tiles
// are summed in shared memory.  grid (9 cout / 16, ceil(cin / 32), chunks)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) conv3x3_wgrad_part(const float* __restrict__ x,
                                                               const float* __restrict__ dy,
                                                               float* __restrict__ part, int n, int h, int w,
                                                               int cin, int cout, long long chunk) {
  __shared__ float red[4][16][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const long long P = (long long)n * h * w;
  const int ntile_co = cout / 16;
  const int tap = blockIdx.x / ntile_co, co0 = (blockIdx.x % ntile_co) * 16;
  const int ky = tap / 3, kx = tap % 3;
  const int ci0 = blockIdx.y * 32;
  const int nnt = min(4, (cin - ci0) / 8);
  const long long pb = (long long)blockIdx.z * chunk, pe = min(P, pb + chunk);
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  auto dyv = [&](long long p, int co) { return p < pe ? dy[p * cout + co] : 0.f; };
  auto xv = [&](long long p, int ci) {
    if (p >= pe) return 0.f;
    const int px = (int)(p % w), py = (int)((p / w) % h), pn = (int)(p / ((long long)w * h));
    const long long q = tap_pixel(p, pn, py, px, h, w, ky, kx);
    return q < 0 ? 0.f : x[q * cin + ci];
  };
  for (long long pk = pb + 16 * warp; pk < pe; pk += 64) {
    uint32_t a[4];
    const long long k0 = pk + 2 * t, k8 = pk + 2 * t + 8;
    a[0] = pack_bf16(dyv(k0, co0 + g), dyv(k0 + 1, co0 + g));
    a[1] = pack_bf16(dyv(k0, co0 + g + 8), dyv(k0 + 1, co0 + g + 8));
    a[2] = pack_bf16(dyv(k8, co0 + g), dyv(k8 + 1, co0 + g));
    a[3] = pack_bf16(dyv(k8, co0 + g + 8), dyv(k8 + 1, co0 + g + 8));
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      if (nt >= nnt) break;
      const int ci = ci0 + nt * 8 + g;
      const uint32_t b0 = pack_bf16(xv(k0, ci), xv(k0 + 1, ci));
      const uint32_t b1 = pack_bf16(xv(k8, ci), xv(k8 + 1, ci));
      mma_bf16(acc[nt], a, b0, b1);
    }
  }
  // acc[nt] covers rows co0 + g (+8), columns ci0 + nt 8 + 2 t (+1)
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    red[warp][g][nt * 8 + 2 * t] = acc[nt][0];
    red[warp][g][nt * 8 + 2 * t + 1] = acc[nt][1];
    red[warp][g + 8][nt * 8 + 2 * t] = acc[nt][2];
    red[warp][g + 8][nt * 8 + 2 * t + 1] = acc[nt][3];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 16 * 32; e += kThreads) {
    const int r = e / 32, c = e % 32;
    if (c >= nnt * 8) continue;
    const float v = (red[0][r][c] + red[1][r][c]) + (red[2][r][c] + red[3][r][c]);
    part[(((long long)blockIdx.z * 9 + tap) * cout + co0 + r) * cin + ci0 + c] = v;
  }
}

// out[i] = sum_z part[z][i] in chunk order (deterministic)
__global__ void sum_parts(const float* __restrict__ part, float* __restrict__ out, long long n, int chunks) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.f;
  for (int z = 0; z < chunks; ++z) s += part[(long long)z * n + i];
  out[i] = s;
}

// bias gradient partials: part[z][c] = sum_{p in chunk z} dy[p][c]
__global__ void colsum_part(const float* __restrict__ dy, float* __restrict__ part, long long P, int c,
                            long long chunk) {
  const int ch = blockIdx.x * blockDim.x + threadIdx.x;
  if (ch >= c) return;
  const long long pb = (long long)blockIdx.y * chunk, pe = min(P, pb + chunk);
  float s = 0.f;
  for (long long p = pb; p < pe; ++p) s += dy[p * c + ch];
  part[(long long)blockIdx.y * c + ch] = s;
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

__global__ void sum_double(const double* __restrict__ part, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    *out = s;
  }
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

// warm-start projection, pass 1: per image, sums of phi1 (target mass), of the clamped prediction
// q = clamp(phi1 + out[p][0]) and of its interface weight 4 q (1 - q)
__global__ void project_sums(const float* __restrict__ out, int cpad, const float* __restrict__ phi0,
                             const float* __restrict__ phi1, double* __restrict__ sums, long long hw) {
  __shared__ double s[3][kThreads];
  const int img = blockIdx.y;
  double a = 0.0, b = 0.0, c = 0.0;
  for (long long k = (long long)blockIdx.x * kThreads + threadIdx.x; k < hw; k += (long long)gridDim.x * kThreads) {
    const long long p = img * hw + k;
    const float hi = 1.f - phi0[p];
    const float q = fminf(fmaxf(phi1[p] + out[p * cpad], 0.f), fmaxf(hi, 0.f));
    a += phi1[p];
    b += q;
    c += 4.0 * q * (1.0 - q);
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

// pass 2: field = q + lambda 4 q (1 - q) with lambda fixing the image's phi1 mass
__global__ void project_apply(const float* __restrict__ out, int cpad, const float* __restrict__ phi0,
                              const float* __restrict__ phi1, const double* __restrict__ sums, int parts,
                              float* __restrict__ field, long long hw) {
  const int img = blockIdx.y;
  double a = 0.0, b = 0.0, c = 0.0;
  for (int k = 0; k < parts; ++k) {
    a += sums[((long long)img * parts + k) * 3];
    b += sums[((long long)img * parts + k) * 3 + 1];
    c += sums[((long long)img * parts + k) * 3 + 2];
  }
  const float lam = c > 0.0 ? (float)((a - b) / c) : 0.f;
  for (long long k = (long long)blockIdx.x * kThreads + threadIdx.x; k < hw; k += (long long)gridDim.x * kThreads) {
    const long long p = img * hw + k;
    const float hi = fmaxf(1.f - phi0[p], 0.f);
    const float q = fminf(fmaxf(phi1[p] + out[p * cpad], 0.f), hi);
    field[p] = q + lam * 4.f * q * (1.f - q);
  }
}

unsigned blocks(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

int status(cudaError_t e) { return e == cudaSuccess ? 0 : -3; }

}  // namespace

extern "C" {

int lbm_nn_conv3x3(const float* x, const void* wt_bf16, const float* bias, float* y, int n, int h, int w, int cin,
                   int cout, int relu, void* stream) {
  if (!x || !wt_bf16 || !y || n < 1 || h < 1 || w < 1 || cin < 16 || cin % 16 || cout < 32 || cout % 32) return -1;
  const long long P = (long long)n * h * w;
  dim3 grid((unsigned)((P + 63) / 64), cout / 32);
  conv3x3_fwd<<<grid, kThreads, 0, (cudaStream_t)stream>>>(x, static_cast<const __nv_bfloat16*>(wt_bf16), bias, y,
                                                           n, h, w, cin, cout, relu);
  return status(cudaGetLastError());
}

long long lbm_nn_wgrad_workspace(int n, int h, int w, int cin, int cout) {
  const long long P = (long long)n * h * w;
  const long long chunk = 4096;
  const long long chunks = (P + chunk - 1) / chunk;
  return chunks * (9LL * cin * cout + cout);
}

int lbm_nn_conv3x3_wgrad(const float* x, const float* dy, float* dw, float* db, float* work, long long work_len,
                         int n, int h, int w, int cin, int cout, void* stream) {
  if (!x || !dy || !dw || !work || n < 1 || h < 1 || w < 1 || cin < 16 || cin % 16 || cout < 16 || cout % 16)
    return -1;
  if (work_len < lbm_nn_wgrad_workspace(n, h, w, cin, cout)) return -1;
  cudaStream_t s = (cudaStream_t)stream;
  const long long P = (long long)n * h * w;
  const long long chunk = 4096;
  const int chunks = (int)((P + chunk - 1) / chunk);
  dim3 grid(9 * (cout / 16), (cin + 31) / 32, chunks);
  conv3x3_wgrad_part<<<grid, kThreads, 0, s>>>(x, dy, work, n, h, w, cin, cout, chunk);
  const long long nw = 9LL * cin * cout;
  sum_parts<<<blocks(nw), 256, 0, s>>>(work, dw, nw, chunks);
  if (db) {
    float* bpart = work + (long long)chunks * nw;
    colsum_part<<<dim3((cout + 127) / 128, chunks), 128, 0, s>>>(dy, bpart, P, cout, chunk);
    sum_parts<<<blocks(cout), 256, 0, s>>>(bpart, db, cout, chunks);
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
  if (n) relu_bwd<<<blocks(n), 256, 0, (cudaStream_t)stream>>>(dy, y, dx, n);
  return status(cudaGetLastError());
}

int lbm_nn_pool2(const float* x, float* y, int n, int h, int w, int c, int backward, void* stream) {
  if (!x || !y || n < 1 || h < 2 || w < 2 || h % 2 || w % 2 || c < 1) return -1;
  cudaStream_t s = (cudaStream_t)stream;
  if (!backward) pool2_fwd<<<blocks((long long)n * h * w * c / 4), 256, 0, s>>>(x, y, n, h, w, c);
  else pool2_bwd<<<blocks((long long)n * h * w * c), 256, 0, s>>>(x, y, n, h, w, c);
  return status(cudaGetLastError());
}

int lbm_nn_up2(const float* x, float* y, int n, int h, int w, int c, int backward, void* stream) {
  if (!x || !y || n < 1 || h < 1 || w < 1 || c < 1) return -1;
  cudaStream_t s = (cudaStream_t)stream;
  if (!backward) up2_fwd<<<blocks(4LL * n * h * w * c), 256, 0, s>>>(x, y, n, h, w, c);
  else up2_bwd<<<blocks((long long)n * h * w * c), 256, 0, s>>>(x, y, n, h, w, c);
  return status(cudaGetLastError());
}

int lbm_nn_add(float* z, const float* x, const float* y, float a, long long n, void* stream) {
  if (!z || !x || !y || n < 0) return -1;
  if (n) add<<<blocks(n), 256, 0, (cudaStream_t)stream>>>(z, x, y, a, n);
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
  sum_double<<<1, 32, 0, s>>>(work, nb, loss);
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
  project_sums<<<dim3(parts, n), kThreads, 0, s>>>(out, cpad, phi0, phi1, work, hw);
  project_apply<<<dim3(parts, n), kThreads, 0, s>>>(out, cpad, phi0, phi1, work, parts, field, hw);
  return status(cudaGetLastError());
}

}  // extern "C"
