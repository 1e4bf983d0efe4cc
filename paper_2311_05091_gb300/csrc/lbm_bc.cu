// Velocity inlet and pressure outlet by non-equilibrium extrapolation.
//
// The paper imposes velocity or pressure at inlets and outlets with the
// non-equilibrium extrapolation scheme of Guo, Zheng and Shi (Sec. 4 intro).
// Here the first x column (x = 0) can be a velocity inlet and the last
// (x = nx - 1) a pressure outlet.  After a step has streamed, every
// population of a boundary node x_b is replaced by the population of its
// neighbour x_f = x_b +- 1 plus the difference of the equilibria at the
// boundary state and at the neighbour's state:
//
//   f_i(x_b) = f_i(x_f) + f_i^eq(phi_b, u_b) - f_i^eq(phi_f, u_f)
//   g_i(x_b) = g_i(x_f) + g_i^eq(p_b, rho_b, u_b) - g_i^eq(p_f, rho_f, u_f)
//
// so the boundary node carries the neighbour's non-equilibrium part.  The
// neighbour's state comes from its own streamed populations: phi_f = sum f_i,
// rho_f from the three densities, u_f = sum c_i g_i / rho_f, and the local
// part of the pressure formula p_f = cs2/(1 - w0) (sum_{i != 0} g_i -
// w0 rho_f |u_f|^2 / (1 - cs2)) (the terms with u.grad rho and the time
// derivative need stencils or history and are left out).  The chemical
// potential and the flux S enter both equilibria alike and cancel.
// Inlet: u_b from the caller's profile, phi_b given (or phi_f), p_b = p_f.
// Outlet: u_b = u_f, phi_b = phi_f, p_b given.
#include <cuda_fp16.h>

#include <type_traits>

#include "lbm_internal.cuh"

namespace lbm {
namespace {

// Lattice velocities in the order of include/lbm.h.
// D2Q9: 0 rest, 1 +x, 2 +y, 3 -x, 4 -y, 5 (+x,+y), 6 (-x,+y), 7 (-x,-y), 8 (+x,-y).
// D3Q19: 0, 1 +x, 2 -x, 3 +y, 4 -y, 5 +z, 6 -z, 7 (+x,+y), 8 (-x,-y), 9 (+x,-y), 10 (-x,+y),
//        11 (+x,+z), 12 (-x,-z), 13 (+x,-z), 14 (-x,+z), 15 (+y,+z), 16 (-y,-z), 17 (+y,-z), 18 (-y,+z).
// D3Q15: 0, 1-6 axes as D3Q19, 7-14 corners (1,1,1) (-1,1,1) (1,-1,1) (-1,-1,1) (1,1,-1) (-1,1,-1)
//        (1,-1,-1) (-1,-1,-1).
__constant__ signed char kC9[9][3] = {{0, 0, 0}, {1, 0, 0},  {0, 1, 0},  {-1, 0, 0}, {0, -1, 0},
                                      {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
__constant__ signed char kC19[19][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                                        {0, 0, 1},  {0, 0, -1}, {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                                        {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                        {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
__constant__ signed char kC15[15][3] = {{0, 0, 0}, {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                                        {0, 0, 1}, {0, 0, -1}, {1, 1, 1},  {-1, 1, 1}, {1, -1, 1},
                                        {-1, -1, 1}, {1, 1, -1}, {-1, 1, -1}, {1, -1, -1}, {-1, -1, -1}};

template <int Q>
__device__ __forceinline__ int cvel(int i, int a) {
  return Q == 9 ? kC9[i][a] : (Q == 19 ? kC19[i][a] : kC15[i][a]);
}

template <class GT>
__device__ __forceinline__ float gload(const GT* p, const InstanceConsts& k) {
  if constexpr (std::is_same<GT, __half>::value) return __half2float(*p) * k.gsci;
  else return *p;
}
template <class GT>
__device__ __forceinline__ void gstore(GT* p, float v, const InstanceConsts& k) {
  if constexpr (std::is_same<GT, __half>::value) *p = __float2half_rn(v * k.gsc);
  else *p = v;
}

// One thread per boundary node: blockIdx.y = side (0 inlet, 1 outlet), blockIdx.z = instance.
template <int Q, class GT>
__global__ void inout_kernel(float* __restrict__ f, GT* __restrict__ g, const float* __restrict__ phi0,
                             const InstanceConsts* __restrict__ consts, const float* __restrict__ u_in, int mode,
                             float phi_in, float p_out, int nx, int ny, int nz, long long nodes) {
  constexpr int D = Q == 9 ? 2 : 3;
  const long long cols = (long long)ny * nz;
  const long long col = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int side = blockIdx.y, b = blockIdx.z;
  if (col >= cols || !(mode & (1 << side))) return;
  const InstanceConsts k = consts[b];
  const int xb = side == 0 ? 0 : nx - 1, xf = side == 0 ? 1 : nx - 2;
  const long long nb = col * nx + xb, nf = col * nx + xf;
  float* fb = f + (long long)b * Q * nodes;
  GT* gb = g + (long long)b * Q * nodes;
  const float* p0 = phi0 + (long long)b * nodes;
  float ff[Q], gf[Q];
  float phi_f = 0.f, j[3] = {0.f, 0.f, 0.f}, sum_nz = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    ff[i] = fb[(long long)i * nodes + nf];
    gf[i] = gload(gb + (long long)i * nodes + nf, k);
    phi_f += ff[i];
    if (i) sum_nz += gf[i];
#pragma unroll
    for (int a = 0; a < D; ++a) j[a] += (float)cvel<Q>(i, a) * gf[i];
  }
  auto rho_of = [&](float s0, float s1) { return k.rho0 * s0 + k.rho1 * s1 + k.rho2 * (1.f - s0 - s1); };
  const float rho_f = rho_of(p0[nf], phi_f);
  float uf[3] = {0.f, 0.f, 0.f}, u2 = 0.f;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    uf[a] = j[a] / rho_f;
    u2 += uf[a] * uf[a];
  }
  const float p_f = k.pf * (sum_nz - k.wq * rho_f * u2);
  float phi_b, p_b, ub[3] = {0.f, 0.f, 0.f};
  if (side == 0) {
    phi_b = phi_in >= 0.f ? phi_in : phi_f;
    p_b = p_f;
#pragma unroll
    for (int a = 0; a < D; ++a) ub[a] = u_in[(long long)a * cols + col];
  } else {
    phi_b = phi_f;
    p_b = p_out;
#pragma unroll
    for (int a = 0; a < D; ++a) ub[a] = uf[a];
  }
  const float rho_b = rho_of(p0[nb], phi_b);
  const float cs2 = k.cs2, cs4 = k.cs4;
  const float dp = p_b - p_f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    int nzc = 0;
    float cu_phi = 0.f, cu_rho = 0.f, diag = 0.f, off = 0.f;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const float c = (float)cvel<Q>(i, a);
      nzc += c != 0.f;
      cu_phi += c * (phi_b * ub[a] - phi_f * uf[a]);
      cu_rho += c * (rho_b * ub[a] - rho_f * uf[a]);
      diag += (c * c - cs2) * (rho_b * ub[a] * ub[a] - rho_f * uf[a] * uf[a]);
#pragma unroll
      for (int e = a + 1; e < D; ++e)
        off += c * (float)cvel<Q>(i, e) * (rho_b * ub[a] * ub[e] - rho_f * uf[a] * uf[e]);
    }
    const float w = i == 0 ? k.w0 : (nzc == 1 ? k.wa : k.we);
    const float dfeq = i == 0 ? phi_b - phi_f : w * cu_phi / cs2;
    const float lam = i == 0 ? (k.w0 - 1.f) * dp / cs2 : w * dp / cs2;
    const float dgeq = lam + w * (cu_rho / cs2 + diag / (cs2 - cs4) + off / cs4);
    fb[(long long)i * nodes + nb] = ff[i] + dfeq;
    gstore(gb + (long long)i * nodes + nb, gf[i] + dgeq, k);
  }
}

template <int Q>
cudaError_t launch_q(float* f, void* g, int g_half, const float* phi0, const InstanceConsts* consts,
                     const float* u_in, int mode, float phi_in, float p_out, int nx, int ny, int nz, long long nodes,
                     int nbatch, cudaStream_t s) {
  const long long cols = (long long)ny * nz;
  dim3 grid((unsigned)((cols + 127) / 128), 2, nbatch);
  if (g_half)
    inout_kernel<Q, __half><<<grid, 128, 0, s>>>(f, static_cast<__half*>(g), phi0, consts, u_in, mode, phi_in,
                                                 p_out, nx, ny, nz, nodes);
  else
    inout_kernel<Q, float><<<grid, 128, 0, s>>>(f, static_cast<float*>(g), phi0, consts, u_in, mode, phi_in, p_out,
                                                nx, ny, nz, nodes);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_inout(float* f, void* g, int g_half, const float* phi0, const InstanceConsts* consts,
                         const float* u_in, int mode, float phi_in, float p_out, int q, int nx, int ny, int nz,
                         long long nodes, int nbatch, cudaStream_t s) {
  if (q == 9) return launch_q<9>(f, g, g_half, phi0, consts, u_in, mode, phi_in, p_out, nx, ny, nz, nodes, nbatch, s);
  if (q == 19)
    return launch_q<19>(f, g, g_half, phi0, consts, u_in, mode, phi_in, p_out, nx, ny, nz, nodes, nbatch, s);
  return launch_q<15>(f, g, g_half, phi0, consts, u_in, mode, phi_in, p_out, nx, ny, nz, nodes, nbatch, s);
}

}  // namespace lbm
