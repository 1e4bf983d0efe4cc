// D3Q19 kernels of the coupled CH + NS step (Zhan, Chai, Shi, arXiv 2311.05091).
//
// Two launches per time step:
//
//   d3q19_moments  phi1 = sum_i f_i and the first moment j = sum_i c_i f_i of
//                  the push-streamed CH populations (Sec. 3).  phi1 goes to
//                  plane 0 of this step's history, j to a 3-plane scratch.
//   d3q19_step     the fused rest of the step.  A CTA owns a TX x TY column
//                  tile and sweeps a strip of z planes with shared-memory
//                  rings: phi0 / phi1 with two halo columns (four planes),
//                  mubar_1 and the antisymmetric products S_a u_b - u_a S_b of
//                  the previous step with one halo column (three planes).
//                  Per node it evaluates the stencils, forces, velocity and
//                  pressure, both Hermite-moment collisions in closed form and
//                  the push-streaming store with half-way bounce-back.
//
// Why the split: the CH populations enter the collision only through phi1,
// j and, for the free rates of the Hermite basis, the higher moments.  With
// every free CH rate equal to 1 (the default), f* = f^eq + R/2 - (s1 - 1) P1 v
// needs phi1 and j alone, so the fused kernel never reads f and the moment
// pass moves the f read off the stencil path.  With other free rates the
// fused kernel reads f once more.
//
// Collision in closed form.  Lambda = T^-1 K T with T the w-orthogonal
// Hermite basis (Sec. 4 intro, Appendix A) acts on each group of equal rate
// through the w-orthogonal projector P_g onto that group's span, which does
// not depend on the basis chosen inside the group:
//     Lambda v = s4 v + sum_{g != 4} (s_g - s4) P_g v.
// The fourth-order group therefore never has to be built.  The third-order
// span is spanned, per axis a with the other two axes (b, c) in cyclic
// order, by the w-orthogonal pair A_a = c_a (c_b^2 + c_c^2) - 2 cs2 c_a and
// B_a = c_a (c_b^2 - c_c^2), of w-norms 2 cs2^2 (1 - 2 cs2) and 2 cs2^2.
//
// HBM traffic per node and step (algorithmic): f and g read and written
// (304 B), phi0 read (4 B), history phi1 / u / S read and written (56 B):
// 364 B.  The split adds the j scratch (12 B written, 12 B read) and the
// second read of phi1 (4 B).
//
// The NS rest population is stored minus the constant rho_0 of lambda_0.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>
#include <string.h>

#include <algorithm>
#include <type_traits>

#include "lbm_internal.cuh"

namespace lbm {
namespace {

constexpr int NS = 19;                       // points of the isotropic stencil (D3Q19 velocities)
constexpr int NH = 7;                        // history planes: phi1, u (3), S (3)
constexpr int TX = 32, TY = 8, NT = TX * TY; // owned column tile, one thread per column
constexpr int HX2 = TX + 4, HY2 = TY + 4, N2 = HX2 * HY2;   // tile with two halo columns
constexpr int HX1 = TX + 2, HY1 = TY + 2, N1 = HX1 * HY1;   // tile with one halo column
constexpr int RP = 4;                        // phi ring planes: z-1 .. z+2
constexpr int RM = 3;                        // mubar / product ring planes: z-1 .. z+1
constexpr float kOneMinusPhi0Floor = 5.9604644775390625e-8f;  // 2^-24

// Stencil points (the D3Q19 velocities of include/lbm.h): 0 centre, 1-6 axes, 7-18 edges.
__host__ __device__ constexpr int SX(int i) {
  return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int SY(int i) {
  return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int SZ(int i) {
  return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
__host__ __device__ constexpr int SA(int i, int a) { return a == 0 ? SX(i) : (a == 1 ? SY(i) : SZ(i)); }

// Lattice velocities of the two 3D lattices (include/lbm.h).  D3Q19: as the
// stencil points.  D3Q15 (the order of the printed M0, Appendix A): 0 rest,
// 1-6 axes (+x, -x, +y, -y, +z, -z), 7-14 corners (1,1,1) (-1,1,1) (1,-1,1)
// (-1,-1,1) (1,1,-1) (-1,1,-1) (1,-1,-1) (-1,-1,-1).
template <int QL>
__host__ __device__ constexpr int LX(int i) {
  return QL == 19 ? SX(i) : (i == 1 || (i >= 7 && (i & 1))) ? 1 : ((i == 2 || (i >= 7 && !(i & 1))) ? -1 : 0);
}
template <int QL>
__host__ __device__ constexpr int LY(int i) {
  return QL == 19 ? SY(i)
                  : (i == 3 || i == 7 || i == 8 || i == 11 || i == 12)
                        ? 1
                        : ((i == 4 || i == 9 || i == 10 || i == 13 || i == 14) ? -1 : 0);
}
template <int QL>
__host__ __device__ constexpr int LZ(int i) {
  return QL == 19 ? SZ(i) : (i == 5 || (i >= 7 && i <= 10)) ? 1 : ((i == 6 || i >= 11) ? -1 : 0);
}
// opposite direction
template <int QL>
__host__ __device__ constexpr int LOPP(int i) {
  return i == 0 ? 0 : (i < 7 || QL == 19) ? ((i & 1) ? i + 1 : i - 1) : 21 - i;
}

// Index i, a few nodes outside [0, n) at most, folded back: periodic wrap, or
// the mirror ghost across the half-way wall (bounded loops, no division).
__device__ __forceinline__ int wrap_or_mirror(int i, int n, int per) {
  if (per) {
    while (i < 0) i += n;
    while (i >= n) i -= n;
    return i;
  }
  if (i < 0) return -1 - i;
  if (i >= n) return 2 * n - 1 - i;
  return i;
}

// slot of logical plane r in a ring of n slots (r >= -8 n)
__device__ __forceinline__ int ring(int r, int n) { return (r + 8 * n) % n; }

// value of a ring-stored field at x + c_d: planes pm (z-1), p0 (z), pp (z+1), row stride sw
__device__ __forceinline__ float nb(const float* pm, const float* p0, const float* pp, int i, int sw, int d) {
  const float* pl = SZ(d) > 0 ? pp : (SZ(d) < 0 ? pm : p0);
  return pl[i + SY(d) * sw + SX(d)];
}

// Isotropic central derivative along axis A with the D3Q19 weights of d0 = 1/3
// (1/18 axis, 1/36 edge): d_A v = sum_i w_i c_iA v(x + c_i) / (1/3).
template <int A>
__device__ __forceinline__ float dgrad(const float* pm, const float* p0, const float* pp, int i, int sw) {
  float axis = 0.f, edge = 0.f;
#pragma unroll
  for (int d = 1; d < NS; ++d) {
    const int c = SA(d, A);
    if (c == 0) continue;
    const float v = nb(pm, p0, pp, i, sw, d);
    if (d < 7) axis += c > 0 ? v : -v;
    else edge += c > 0 ? v : -v;
  }
  return axis * (1.f / 6.f) + edge * (1.f / 12.f);
}

// Isotropic Laplacian: sum_i 2 w_i (v(x + c_i) - v(x)) / (1/3).
__device__ __forceinline__ float lap3(const float* pm, const float* p0, const float* pp, int i, int sw) {
  const float c = p0[i];
  float axis = 0.f, edge = 0.f;
#pragma unroll
  for (int d = 1; d < NS; ++d) {
    const float v = nb(pm, p0, pp, i, sw, d) - c;
    if (d < 7) axis += v;
    else edge += v;
  }
  return __fmaf_rn(axis, 1.f / 3.f, __fmul_rn(edge, 1.f / 6.f));   // as lap_v, rounding for rounding
}

// The same two operators on the 19 values v[d] = v(x + c_d), gathered once.
__device__ __forceinline__ void gather19(const float* pm, const float* p0, const float* pp, int i, int sw,
                                         float (&v)[NS]) {
#pragma unroll
  for (int d = 0; d < NS; ++d) v[d] = nb(pm, p0, pp, i, sw, d);
}

template <int A>
__device__ __forceinline__ float dgrad_v(const float (&v)[NS]) {
  float axis = 0.f, edge = 0.f;
#pragma unroll
  for (int d = 1; d < NS; ++d) {
    const int c = SA(d, A);
    if (c == 0) continue;
    if (d < 7) axis += c > 0 ? v[d] : -v[d];
    else edge += c > 0 ? v[d] : -v[d];
  }
  return axis * (1.f / 6.f) + edge * (1.f / 12.f);
}

__device__ __forceinline__ float lap_v(const float (&v)[NS]) {
  float axis = 0.f, edge = 0.f;
#pragma unroll
  for (int d = 1; d < NS; ++d) {
    const float w = v[d] - v[0];
    if (d < 7) axis += w;
    else edge += w;
  }
  return __fmaf_rn(axis, 1.f / 3.f, __fmul_rn(edge, 1.f / 6.f));   // as lap3, rounding for rounding
}

// mu_p = gamma_p psi_p, psi_p = (12/D) phi_p (1 - phi_p)(1 - 2 phi_p) - (3D/4) lap phi_p (Sec. 2.1).
__device__ __forceinline__ void chem_pot(const InstanceConsts& k, float ph0, float ph1, float lap0,
                                         float lap1, float& mu0, float& mu1, float& mu2) {
  // every product and sum is spelled out (no contraction left to the compiler), so the pipelined kernel's
  // mubar_1 pass and the node update round these values identically wherever they are inlined
  const float ph2 = __fsub_rn(__fsub_rn(1.f, ph0), ph1);
  const float lap2 = __fsub_rn(-lap0, lap1);
  auto psi = [&](float ph, float lap) {
    const float bulk = __fmul_rn(__fmul_rn(__fmul_rn(k.c12_W, ph), __fsub_rn(1.f, ph)), __fmaf_rn(-2.f, ph, 1.f));
    return __fmaf_rn(-k.c34_W, lap, bulk);
  };
  mu0 = __fmul_rn(k.gam0, psi(ph0, lap0));
  mu1 = __fmul_rn(k.gam1, psi(ph1, lap1));
  mu2 = __fmul_rn(k.gam2, psi(ph2, lap2));
}

// mubar_1 = gamma_T/3 [ (mu1 - mu0)/gamma_0 + (mu1 - mu2)/gamma_2 ] (Eq. CHmodel).
__device__ __forceinline__ float mubar1_of(const InstanceConsts& k, float mu0, float mu1, float mu2) {
  return k.gT3 * ((mu1 - mu0) * k.inv_gam0 + (mu1 - mu2) * k.inv_gam2);
}

__device__ __forceinline__ float weight(const InstanceConsts& k, int i) {
  return i == 0 ? k.w0 : (i < 7 ? k.wa : k.we);
}

// NS population storage: float32, or FP16 holding g * gsc (gsc a power of two)
__device__ __forceinline__ float g_load(float v, const InstanceConsts&) { return v; }
__device__ __forceinline__ float g_load(__half v, const InstanceConsts& k) { return __half2float(v) * k.gsci; }
__device__ __forceinline__ void g_store(float* p, float v, const InstanceConsts&) { *p = v; }
__device__ __forceinline__ void g_store(__half* p, float v, const InstanceConsts& k) {
  *p = __float2half_rn(v * k.gsc);
}

// ---------------------------------------------------------------------------
// initial state: f = f^eq(phi1, mubar_1, u = 0), g = g^eq(p = 0, u = 0) - rho_0 e_0 = 0,
// history = (phi1, 0, ..., 0).  phi1 arrives staged in plane 0 of a spare history buffer.
// ---------------------------------------------------------------------------
template <int QL, typename GT>
__global__ void d3q19_init(const float* __restrict__ phi0_all, const float* __restrict__ phi1_all,
                           float* __restrict__ f_all, GT* __restrict__ g_all, float* __restrict__ hist_all,
                           const InstanceConsts* __restrict__ consts, int nx, int ny, int nz, int per_x,
                           int per_y, int per_z, int nbatch) {
  const long long nodes = (long long)nx * ny * nz;
  const long long total = nodes * nbatch;
  for (long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x; gi < total;
       gi += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(gi / nodes);
    const long long node = gi - (long long)b * nodes;
    const int x = (int)(node % nx), y = (int)((node / nx) % ny), z = (int)(node / ((long long)nx * ny));
    const InstanceConsts& k = consts[b];
    const float* phi0 = phi0_all + (long long)b * nodes;
    const float* phi1 = phi1_all + (long long)b * NH * nodes;
    auto at = [&](const float* a, int d) {
      const int xx = wrap_or_mirror(x + SX(d), nx, per_x);
      const int yy = wrap_or_mirror(y + SY(d), ny, per_y);
      const int zz = wrap_or_mirror(z + SZ(d), nz, per_z);
      return a[((long long)zz * ny + yy) * nx + xx];
    };
    const float c0 = phi0[node], c1 = phi1[node];
    float a0 = 0.f, e0 = 0.f, a1 = 0.f, e1 = 0.f;
#pragma unroll
    for (int d = 1; d < NS; ++d) {
      const float v0 = at(phi0, d) - c0, v1 = at(phi1, d) - c1;
      if (d < 7) {
        a0 += v0;
        a1 += v1;
      } else {
        e0 += v0;
        e1 += v1;
      }
    }
    const float lap0 = a0 * (1.f / 3.f) + e0 * (1.f / 6.f);
    const float lap1 = a1 * (1.f / 3.f) + e1 * (1.f / 6.f);
    float mu0, mu1, mu2;
    chem_pot(k, c0, c1, lap0, lap1, mu0, mu1, mu2);
    const float emb = k.eta * mubar1_of(k, mu0, mu1, mu2);
    float* f = f_all + (long long)b * QL * nodes;
    GT* g = g_all + (long long)b * QL * nodes;
    float* h = hist_all + (long long)b * NH * nodes;
    f[node] = c1 + (k.w0 - 1.f) * emb;
#pragma unroll
    for (int i = 1; i < QL; ++i) f[(long long)i * nodes + node] = (i < 7 ? k.wa : k.we) * emb;
#pragma unroll
    for (int i = 0; i < QL; ++i) g[(long long)i * nodes + node] = GT(0.f);
    h[node] = c1;
#pragma unroll
    for (int q = 1; q < NH; ++q) h[(long long)q * nodes + node] = 0.f;
  }
}

// ---------------------------------------------------------------------------
// moment pass: phi1 = sum_i f_i -> history plane 0, j = sum_i c_i f_i -> scratch
// ---------------------------------------------------------------------------
template <int QL>
__device__ __forceinline__ void moments_q(const float (&v)[QL], float& s, float& jx, float& jy, float& jz) {
  s = v[0];
  jx = 0.f;
  jy = 0.f;
  jz = 0.f;
#pragma unroll
  for (int i = 1; i < QL; ++i) {
    s += v[i];
    if (LX<QL>(i)) jx += LX<QL>(i) > 0 ? v[i] : -v[i];
    if (LY<QL>(i)) jy += LY<QL>(i) > 0 ? v[i] : -v[i];
    if (LZ<QL>(i)) jz += LZ<QL>(i) > 0 ? v[i] : -v[i];
  }
}

template <int QL>
__global__ void __launch_bounds__(256) d3q_moments(const float* __restrict__ f_all, float* __restrict__ hist_all,
                                                     float* __restrict__ mom_all, int nodes, int vec4) {
  const int b = blockIdx.y;
  const float* f = f_all + (long long)b * QL * nodes;
  float* h = hist_all + (long long)b * NH * nodes;
  float* m = mom_all + (long long)b * 3 * nodes;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (vec4) {
    const int n4 = nodes >> 2;
    if (t >= n4) return;
    float4 v[QL];
#pragma unroll
    for (int i = 0; i < QL; ++i) v[i] = __ldcs(reinterpret_cast<const float4*>(f + (long long)i * nodes) + t);
    float4 s, jx, jy, jz;
    {
      float a[QL];
#pragma unroll
      for (int i = 0; i < QL; ++i) a[i] = v[i].x;
      moments_q<QL>(a, s.x, jx.x, jy.x, jz.x);
#pragma unroll
      for (int i = 0; i < QL; ++i) a[i] = v[i].y;
      moments_q<QL>(a, s.y, jx.y, jy.y, jz.y);
#pragma unroll
      for (int i = 0; i < QL; ++i) a[i] = v[i].z;
      moments_q<QL>(a, s.z, jx.z, jy.z, jz.z);
#pragma unroll
      for (int i = 0; i < QL; ++i) a[i] = v[i].w;
      moments_q<QL>(a, s.w, jx.w, jy.w, jz.w);
    }
    reinterpret_cast<float4*>(h)[t] = s;
    reinterpret_cast<float4*>(m)[t] = jx;
    reinterpret_cast<float4*>(m + nodes)[t] = jy;
    reinterpret_cast<float4*>(m + 2 * (long long)nodes)[t] = jz;
  } else {
    if (t >= nodes) return;
    float a[QL];
#pragma unroll
    for (int i = 0; i < QL; ++i) a[i] = __ldcs(f + (long long)i * nodes + t);
    float s, jx, jy, jz;
    moments_q<QL>(a, s, jx, jy, jz);
    h[t] = s;
    m[t] = jx;
    m[nodes + t] = jy;
    m[2 * (long long)nodes + t] = jz;
  }
}

// Moments of the moving NS populations, summed over pairs of opposite velocities (s = g_i + g_opp,
// d = g_i - g_opp, i the member listed first): the sum, the first moments m, the off-diagonal second
// moments p_ab and the third-order sums e_a = sum c_a (c_b^2 + c_c^2) g and b_a = sum c_a (c_b^2 - c_c^2) g
// (D3Q19, cyclic a, b, c); D3Q15: e_a = sum over corners c_a g, bx = sum cx cy cz g, by = bz = 0.
template <int QL, typename GA>
__device__ __forceinline__ void ns_moments(const GA& g, float& sum_nz, float& mx, float& my, float& mz,
                                           float& pxy, float& pxz, float& pyz, float& ex, float& ey,
                                           float& ez, float& bxm, float& bym, float& bzm) {
  auto S = [&](int i) { return g(i) + g(LOPP<QL>(i)); };
  auto D = [&](int i) { return g(i) - g(LOPP<QL>(i)); };
  const float sa = S(1) + S(3) + S(5);
  if constexpr (QL == 19) {
    // first members: 7 (1,1,0), 9 (1,-1,0), 11 (1,0,1), 13 (1,0,-1), 15 (0,1,1), 17 (0,1,-1)
    const float d7 = D(7), d9 = D(9), d11 = D(11), d13 = D(13), d15 = D(15), d17 = D(17);
    const float s7 = S(7), s9 = S(9), s11 = S(11), s13 = S(13), s15 = S(15), s17 = S(17);
    sum_nz = sa + ((s7 + s9) + (s11 + s13) + (s15 + s17));
    pxy = s7 - s9;
    pxz = s11 - s13;
    pyz = s15 - s17;
    const float xa = d7 + d9, xb = d11 + d13;   // x-edges in the xy and xz planes
    const float ya = d15 + d17, yb = d7 - d9;   // y-edges in the yz and xy planes
    const float za = d11 - d13, zb = d15 - d17; // z-edges in the xz and yz planes
    ex = xa + xb;
    bxm = xa - xb;
    ey = ya + yb;
    bym = ya - yb;
    ez = za + zb;
    bzm = za - zb;
  } else {
    // first members of the corner pairs: 7 (1,1,1), 8 (-1,1,1), 9 (1,-1,1), 10 (-1,-1,1)
    const float d7 = D(7), d8 = D(8), d9 = D(9), d10 = D(10);
    const float s7 = S(7), s8 = S(8), s9 = S(9), s10 = S(10);
    const float sp = s7 + s10, sq = s8 + s9, sr = s7 - s10, st = s8 - s9;
    sum_nz = sa + (sp + sq);
    pxy = sp - sq;
    pxz = sr - st;
    pyz = sr + st;
    const float dp = d7 + d10, dq = d8 + d9, dr = d7 - d10, dt = d8 - d9;
    ex = dr - dt;
    ey = dr + dt;
    ez = dp + dq;
    bxm = dp - dq;
    bym = bzm = 0.f;
  }
  mx = D(1) + ex;
  my = D(3) + ey;
  mz = D(5) + ez;
}

// ---------------------------------------------------------------------------
// per-node update shared by both fused kernels
// ---------------------------------------------------------------------------
// Inputs of one node that do not come from a stencil: its NS populations, the
// first moment j of its CH populations and its previous-step history.
template <int QL>
struct OwnIn {
  float g[QL];
  float jx, jy, jz;
  float php, upx, upy, upz, spx, spy, spz;
  float d02, d12;   // mu0 - mu2 and mu1 - mu2 of the node, when the caller computed them already (MU_IN)
};

// Ring planes (z-1, z, z+1) around the node: phi0 / phi1 on the two-halo tile
// (index i2, row stride sw2), mubar_1 and the products on the one-halo tile
// (index i1, row stride sw1).
struct Rings {
  const float* p0[3];
  const float* p1[3];
  int i2, sw2;
  const float* mu[3];
  const float* ac[3][3];   // [product][plane]
  int i1, sw1;
};

struct Outs {
  const float* f_in;   // instance base, read by the general CH path
  float* f_out;
  void* g_out;            // float, or FP16 scaled by gsc
  float* h_out;
  float* p_out;
  unsigned int* flag;
  int nx, ny, nz, per_x, per_y, per_z, nodes, plane;
};

// MU_IN: the chemical-potential differences of the node come in `in` (the pipelined kernel keeps them from its
// mubar_1 pass over the same planes, bitwise the values computed here otherwise).  SZ: rho1 == rho2, so the mass
// flux S = (rho1 - rho2) M grad(mubar_1) / gamma_1 is zero and with it the correction force F_c = div(S u - u S) / 2;
// its stencils are skipped (the same values up to the sign of zeros).  PER: the lattice is periodic on all
// three axes (the bounce-back selection of the pushes is compiled out).
template <int QL, bool OBS, typename GT, bool MU_IN = false, bool SZ = false, bool PER = false, typename GA,
          typename GB>
__device__ __forceinline__ void node_update(const InstanceConsts& k, const Rings& R, const OwnIn<QL>& in,
                                            const GA& g, const GB& g_late, const Outs& o, int x, int y, int z) {
  const int nx = o.nx, ny = o.ny, nz = o.nz, nodes = o.nodes, plane = o.plane;
  const int node = z * plane + y * nx + x;
  const float cs2 = k.cs2, cs4 = k.cs4;
  const int i2 = R.i2, s2 = R.sw2, i1 = R.i1, s1 = R.sw1;

  // NS moments first: the populations then wait in their owned slot (or registers) until the collision
  float sum_nz, mx, my, mz, pxy, pxz, pyz, ex, ey, ez, bxm, bym, bzm;
  ns_moments<QL>(g, sum_nz, mx, my, mz, pxy, pxz, pyz, ex, ey, ez, bxm, bym, bzm);

  // stencils of phi0, phi1 and mubar_1, products; each neighbourhood is read once
  float ph0, ph1, g0x, g0y, g0z, g1x, g1y, g1z, lap0, lap1;
  {
    float v[NS];
    gather19(R.p0[0], R.p0[1], R.p0[2], i2, s2, v);
    ph0 = v[0];
    g0x = dgrad_v<0>(v);
    g0y = dgrad_v<1>(v);
    g0z = dgrad_v<2>(v);
    if (!MU_IN) lap0 = lap_v(v);
    gather19(R.p1[0], R.p1[1], R.p1[2], i2, s2, v);
    ph1 = v[0];
    g1x = dgrad_v<0>(v);
    g1y = dgrad_v<1>(v);
    g1z = dgrad_v<2>(v);
    if (!MU_IN) lap1 = lap_v(v);
  }
  const float ph2 = 1.f - ph0 - ph1;
  float d02, d12;
  if (MU_IN) {
    d02 = in.d02;
    d12 = in.d12;
  } else {
    float mu0, mu1, mu2;
    chem_pot(k, ph0, ph1, lap0, lap1, mu0, mu1, mu2);
    d02 = mu0 - mu2;
    d12 = mu1 - mu2;
  }
  float mub, gmx, gmy, gmz, dAxy_x, dAxy_y, dAxz_x, dAxz_z, dAyz_y, dAyz_z;
  {
    float v[NS];
    gather19(R.mu[0], R.mu[1], R.mu[2], i1, s1, v);
    mub = v[0];
    gmx = dgrad_v<0>(v);
    gmy = dgrad_v<1>(v);
    gmz = dgrad_v<2>(v);
    // correction force F_c,b = 1/2 sum_a d_a (S_a u_b - u_a S_b), products A_xy, A_xz, A_yz
    if (SZ) {
      dAxy_x = dAxy_y = dAxz_x = dAxz_z = dAyz_y = dAyz_z = 0.f;
    } else {
      gather19(R.ac[0][0], R.ac[0][1], R.ac[0][2], i1, s1, v);
      dAxy_x = dgrad_v<0>(v);
      dAxy_y = dgrad_v<1>(v);
      gather19(R.ac[1][0], R.ac[1][1], R.ac[1][2], i1, s1, v);
      dAxz_x = dgrad_v<0>(v);
      dAxz_z = dgrad_v<2>(v);
      gather19(R.ac[2][0], R.ac[2][1], R.ac[2][2], i1, s1, v);
      dAyz_y = dgrad_v<1>(v);
      dAyz_z = dgrad_v<2>(v);
    }
  }
  const float Fcx = -0.5f * (dAxy_y + dAxz_z);
  const float Fcy = 0.5f * (dAxy_x - dAyz_z);
  const float Fcz = 0.5f * (dAxz_x + dAyz_y);

  const float php = in.php, upx = in.upx, upy = in.upy, upz = in.upz;
  const float spx = in.spx, spy = in.spy, spz = in.spz;

  // degenerate mobility, flux S (frozen phi0), mixture properties
  const float fdeg = ph1 * (1.f - ph1) * (1.f - ph0);
  const float mob = k.M_cst + k.M_deg * fdeg;
  const float sfac = (k.rho1 - k.rho2) * mob * k.inv_gam1;
  const float Sx = sfac * gmx, Sy = sfac * gmy, Sz = sfac * gmz;
  const float rho = k.rho0 * ph0 + k.rho1 * ph1 + k.rho2 * ph2;
  const float grx = (k.rho0 - k.rho2) * g0x + (k.rho1 - k.rho2) * g1x;
  const float gry = (k.rho0 - k.rho2) * g0y + (k.rho1 - k.rho2) * g1y;
  const float grz = (k.rho0 - k.rho2) * g0z + (k.rho1 - k.rho2) * g1z;
  const float muv = k.mu0 * ph0 + k.mu1 * ph1 + k.mu2 * ph2;

  // F = F_s + F_b + F_c with F_s = (mu0 - mu2) grad phi0 + (mu1 - mu2) grad phi1
  const float one_m0 = 1.f - ph0;
  const float Fx = d02 * g0x + d12 * g1x + one_m0 * k.bx + Fcx;
  const float Fy = d02 * g0y + d12 * g1y + one_m0 * k.by + Fcy;
  const float Fz = d02 * g0z + d12 * g1z + one_m0 * k.bz + Fcz;

  // velocity with the solid penalisation force (u_w = 0)
  const float inv_rho = __frcp_rn(rho);
  const float usx = (mx + 0.5f * Fx) * inv_rho;
  const float usy = (my + 0.5f * Fy) * inv_rho;
  const float usz = (mz + 0.5f * Fz) * inv_rho;
  const float damp = 1.f - 0.5f * ph0;
  const float ux = usx * damp, uy = usy * damp, uz = usz * damp;
  const float Ftx = Fx - ph0 * rho * usx, Fty = Fy - ph0 * rho * usy, Ftz = Fz - ph0 * rho * usz;

  // local viscous rates (s0 = s4 = s2a)
  const float om = fmaxf(one_m0, kOneMinusPhi0Floor);
  // 1/s2a = 1/2 + mu / (rho (1 - phi0) a2a), likewise s2b; IEEE-rounded reciprocals
  const float nu_e = muv * __frcp_rn(rho * om);
  const float inv_s2a = 0.5f + nu_e * k.ia2a;
  const float s2a = __frcp_rn(inv_s2a);
  const float s2b = __frcp_rn(0.5f + nu_e * k.ia2b);

  // pressure (Sec. 3)
  const float udg = ux * grx + uy * gry + uz * grz;
  const float q = (rho * ux - Sx) * ux + (rho * uy - Sy) * uy + (rho * uz - Sz) * uz;
  const float rhop = k.rho0 * ph0 + k.rho1 * php + k.rho2 * (1.f - ph0 - php);
  const float qp = (rhop * upx - spx) * upx + (rhop * upy - spy) * upy + (rhop * upz - spz) * upz;
  const float H = k.Kp * ((k.h0 - k.h2) * inv_s2a + k.h3);
  const float p = k.pf * (sum_nz + (0.5f + H) * udg - k.wq * q + 0.5f * k.Kp * (q - qp));

  // push destinations without branches: per axis and sign, the offset of the
  // neighbour (periodic wrap folded in) and whether a wall reflects instead
  // (PER: every axis periodic, no push meets a wall)
  const bool wxp = !PER && x + 1 >= nx && !o.per_x, wxm = !PER && x == 0 && !o.per_x;
  const bool wyp = !PER && y + 1 >= ny && !o.per_y, wym = !PER && y == 0 && !o.per_y;
  const bool wzp = !PER && z + 1 >= nz && !o.per_z, wzm = !PER && z == 0 && !o.per_z;
  const int oxp = x + 1 < nx ? 1 : 1 - nx, oxm = x > 0 ? -1 : nx - 1;
  const int oyp = y + 1 < ny ? nx : nx - plane, oym = y > 0 ? -nx : plane - nx;
  const int ozp = z + 1 < nz ? plane : plane - nodes, ozm = z > 0 ? -plane : nodes - plane;
  auto store = [&](auto* __restrict__ out, int i, float v) {
    const int cx = LX<QL>(i), cy = LY<QL>(i), cz = LZ<QL>(i);
    int off = 0;
    bool bb = false;
    if (cx) { off += cx > 0 ? oxp : oxm; bb = bb || (cx > 0 ? wxp : wxm); }
    if (cy) { off += cy > 0 ? oyp : oym; bb = bb || (cy > 0 ? wyp : wym); }
    if (cz) { off += cz > 0 ? ozp : ozm; bb = bb || (cz > 0 ? wzp : wzm); }
    g_store(out + (bb ? LOPP<QL>(i) * nodes + node : i * nodes + node + off), v, k);
  };

  // ---- NS collision: g* = (1 - s2a) g + w_i X_i (see the file header) ----
  {
    const float om2a = 1.f - 0.5f * s2a;
    // equilibrium second moments e_ab and the force moment M^2F_ab (Sec. 3)
    const float exx = rho * ux * ux - Sx * ux, eyy = rho * uy * uy - Sy * uy, ezz = rho * uz * uz - Sz * uz;
    const float exy = rho * ux * uy - 0.5f * (Sx * uy + ux * Sy);
    const float exz = rho * ux * uz - 0.5f * (Sx * uz + ux * Sz);
    const float eyz = rho * uy * uz - 0.5f * (Sy * uz + uy * Sz);
    const float dSxx = Sx * ux - spx * upx, dSyy = Sy * uy - spy * upy, dSzz = Sz * uz - spz * upz;
    const float dSxy = 0.5f * (Sx * uy + ux * Sy) - 0.5f * (spx * upy + upx * spy);
    const float dSxz = 0.5f * (Sx * uz + ux * Sz) - 0.5f * (spx * upz + upx * spz);
    const float dSyz = 0.5f * (Sy * uz + uy * Sz) - 0.5f * (spy * upz + upy * spz);
    const float iso = (1.f - 3.f * cs2) * udg;
    const float Mxx = 2.f * ux * Fx - dSxx + 2.f * cs2 * ux * grx + iso;
    const float Myy = 2.f * uy * Fy - dSyy + 2.f * cs2 * uy * gry + iso;
    const float Mzz = 2.f * uz * Fz - dSzz + 2.f * cs2 * uz * grz + iso;
    const float Mxy = ux * Fy + Fx * uy - dSxy + cs2 * (ux * gry + grx * uy);
    const float Mxz = ux * Fz + Fx * uz - dSxz + cs2 * (ux * grz + grx * uz);
    const float Myz = uy * Fz + Fy * uz - dSyz + cs2 * (uy * grz + gry * uz);
    const float i2n = __frcp_rn(cs2 - cs4), ic2 = __frcp_rn(cs2), ic4 = __frcp_rn(cs4);
    const float Dx = (s2a * exx + om2a * Mxx) * i2n;
    const float Dy = (s2a * eyy + om2a * Myy) * i2n;
    const float Dz = (s2a * ezz + om2a * Mzz) * i2n;
    const float base = s2a * p * ic2 + om2a * udg - cs2 * (Dx + Dy + Dz);
    const float d1 = k.s1n - s2a;
    const float Vx = (s2a * rho * ux + om2a * Ftx - d1 * (mx - rho * ux + 0.5f * Ftx)) * ic2;
    const float Vy = (s2a * rho * uy + om2a * Fty - d1 * (my - rho * uy + 0.5f * Fty)) * ic2;
    const float Vz = (s2a * rho * uz + om2a * Ftz - d1 * (mz - rho * uz + 0.5f * Ftz)) * ic2;
    const float db = s2b - s2a;
    const float Oxy = (s2a * exy + om2a * Mxy - db * (pxy - exy + 0.5f * Mxy)) * ic4;
    const float Oxz = (s2a * exz + om2a * Mxz - db * (pxz - exz + 0.5f * Mxz)) * ic4;
    const float Oyz = (s2a * eyz + om2a * Myz - db * (pyz - eyz + 0.5f * Myz)) * ic4;
    // third-order group: T_a = (s3 - s2a) m_A,a / |A|^2, U_a = (s3 - s2a) m_B,a / |B|^2.  D3Q15: A_a =
    // corner c_a - cs2 c_a with |A|^2 = cs2^2 (1 - cs2), one B = cx cy cz with |B|^2 = cs2^2 (in Ux)
    const float d3 = k.s3n - s2a;
    const float iB = __frcp_rn(QL == 19 ? 2.f * cs4 : cs4);
    const float iA = __frcp_rn(QL == 19 ? 2.f * cs4 * (1.f - 2.f * cs2) : cs4 * (1.f - cs2));
    const float k3 = QL == 19 ? 1.f - 2.f * cs2 : 1.f - cs2;
    const float cA = QL == 19 ? 2.f * cs2 : cs2;
    const float Tx = d3 * (ex - cA * mx) * iA, Ty = d3 * (ey - cA * my) * iA, Tz = d3 * (ez - cA * mz) * iA;
    const float Ux = d3 * bxm * iB, Uy = d3 * bym * iB, Uz = d3 * bzm * iB;
    const float Px = k3 * Tx + Ux, Qx = k3 * Tx - Ux;   // edge factors per axis: B_a = +c_a or -c_a
    const float Py = k3 * Ty + Uy, Qy = k3 * Ty - Uy;
    const float Pz = k3 * Tz + Uz, Qz = k3 * Tz - Uz;
    const float om1 = 1.f - s2a;
    GT* const g_out = static_cast<GT*>(o.g_out);
    store(g_out, 0, om1 * g_late(0) + k.w0 * base - s2a * p * ic2);
    // X_i = E + O and X_opp(i) = E - O: the part E even in c (base, D, O terms) and the part O odd in c
    // (V and the third-order terms) are formed once per pair of opposite velocities
    auto put2 = [&](int i, float E, float O) {
      store(g_out, i, om1 * g_late(i) + weight(k, i) * (E + O));
      store(g_out, LOPP<QL>(i), om1 * g_late(LOPP<QL>(i)) + weight(k, i) * (E - O));
    };
    // axis: A_a(c) = -2 cs2 c_a (D3Q19), -cs2 c_a (D3Q15); B = 0
    put2(1, base + Dx, Vx + cA * Tx);
    put2(3, base + Dy, Vy + cA * Ty);
    put2(5, base + Dz, Vz + cA * Tz);
    if constexpr (QL == 19) {
      // edge: -c_a [(1 - 2 cs2) T_a + B_a U_a / c_a] over its two axes, B_a U_a / c_a = +U_a on the edges of
      // the axis that follows a cyclically (P_a), -U_a on the other (Q_a)
      const float Bxy = base + Dx + Dy, Bxz = base + Dx + Dz, Byz = base + Dy + Dz;
      {
        const float u = Vx - Px, v = Vy - Qy;   // edges (1, +-1, 0)
        put2(7, Bxy + Oxy, u + v);
        put2(9, Bxy - Oxy, u - v);
      }
      {
        const float u = Vx - Qx, v = Vz - Pz;   // edges (1, 0, +-1)
        put2(11, Bxz + Oxz, u + v);
        put2(13, Bxz - Oxz, u - v);
      }
      {
        const float u = Vy - Py, v = Vz - Qz;   // edges (0, 1, +-1)
        put2(15, Byz + Oyz, u + v);
        put2(17, Byz - Oyz, u - v);
      }
    } else {
      // corner: -(1 - cs2) c.T - cx cy cz U
      const float B = base + Dx + Dy + Dz;
      const float u = Vx - k3 * Tx, v = Vy - k3 * Ty, w = Vz - k3 * Tz;
      put2(7, B + Oxy + Oxz + Oyz, u + v + w - Ux);     // (1, 1, 1)
      put2(8, B - Oxy - Oxz + Oyz, v + w - u + Ux);     // (-1, 1, 1)
      put2(9, B - Oxy + Oxz - Oyz, u - v + w + Ux);     // (1, -1, 1)
      put2(10, B + Oxy - Oxz - Oyz, w - u - v - Ux);    // (-1, -1, 1)
    }
  }

  // ---- CH collision ----
  {
    const float emb = k.eta * mub;
    const float corr = k.corr_scale * (1.f - fdeg);
    // first moment of R: d_t(phi1 u) + cs2 corr eta grad mubar
    const float Rx = (ph1 * ux - php * upx) + cs2 * corr * k.eta * gmx;
    const float Ry = (ph1 * uy - php * upy) + cs2 * corr * k.eta * gmy;
    const float Rz = (ph1 * uz - php * upz) + cs2 * corr * k.eta * gmz;
    const float ic2 = __frcp_rn(cs2);
    if (k.ch_fast != 0.f) {
      // f* = f^eq + R/2 - (s1 - 1) P1 v: only j = sum c f enters
      const float jx = in.jx, jy = in.jy, jz = in.jz;
      const float ax = (ph1 * ux + (1.f - k.s1c) * (jx - ph1 * ux) + (1.f - 0.5f * k.s1c) * Rx) * ic2;
      const float ay = (ph1 * uy + (1.f - k.s1c) * (jy - ph1 * uy) + (1.f - 0.5f * k.s1c) * Ry) * ic2;
      const float az = (ph1 * uz + (1.f - k.s1c) * (jz - ph1 * uz) + (1.f - 0.5f * k.s1c) * Rz) * ic2;
      float rest = ph1;
#pragma unroll
      for (int i = 1; i < QL; ++i) {
        const int cx = LX<QL>(i), cy = LY<QL>(i), cz = LZ<QL>(i);
        float s = emb;
        if (cx) s += cx > 0 ? ax : -ax;
        if (cy) s += cy > 0 ? ay : -ay;
        if (cz) s += cz > 0 ? az : -az;
        const float v = weight(k, i) * s;
        rest -= v;
        store(o.f_out, i, v);
      }
      store(o.f_out, 0, rest);   // the rest population closes the zeroth moment
    } else {
      float f[QL];
#pragma unroll
      for (int i = 0; i < QL; ++i) f[i] = o.f_in[i * nodes + node];
      float jx = 0.f, jy = 0.f, jz = 0.f, qxx = 0.f, qyy = 0.f, qzz = 0.f, qxy = 0.f, qxz = 0.f, qyz = 0.f;
      float ex = 0.f, ey = 0.f, ez = 0.f, bxm = 0.f, bym = 0.f, bzm = 0.f;
#pragma unroll
      for (int i = 1; i < QL; ++i) {
        const int cx = LX<QL>(i), cy = LY<QL>(i), cz = LZ<QL>(i);
        const float v = f[i];
        if (cx) { jx += cx > 0 ? v : -v; qxx += v; }
        if (cy) { jy += cy > 0 ? v : -v; qyy += v; }
        if (cz) { jz += cz > 0 ? v : -v; qzz += v; }
        if (cx && cy) qxy += cx * cy > 0 ? v : -v;
        if (cx && cz) qxz += cx * cz > 0 ? v : -v;
        if (cy && cz) qyz += cy * cz > 0 ? v : -v;
        if (cx && (cy || cz)) { ex += cx > 0 ? v : -v; if constexpr (QL == 19) bxm += ((cy ? 1 : -1) * cx > 0) ? v : -v; }
        if (cy && (cz || cx)) { ey += cy > 0 ? v : -v; if constexpr (QL == 19) bym += ((cz ? 1 : -1) * cy > 0) ? v : -v; }
        if (cz && (cx || cy)) { ez += cz > 0 ? v : -v; if constexpr (QL == 19) bzm += ((cx ? 1 : -1) * cz > 0) ? v : -v; }
        if constexpr (QL == 15)
          if (cx && cy && cz) bxm += cx * cy * cz > 0 ? v : -v;
      }
      const float s4 = k.s4c, om4 = 1.f - s4, oh4 = 1.f - 0.5f * s4;
      const float d1 = (k.s1c - s4) * ic2;
      const float m1x = jx - ph1 * ux + 0.5f * Rx, m1y = jy - ph1 * uy + 0.5f * Ry, m1z = jz - ph1 * uz + 0.5f * Rz;
      const float d2a = (k.s2ac - s4) * __frcp_rn(cs2 - cs4);
      const float m2x = qxx - cs2 * emb, m2y = qyy - cs2 * emb, m2z = qzz - cs2 * emb;
      const float d2b = (k.s2bc - s4) * __frcp_rn(cs4);
      const float d3 = k.s3c - s4;
      const float iB = __frcp_rn(QL == 19 ? 2.f * cs4 : cs4);
      const float iA = __frcp_rn(QL == 19 ? 2.f * cs4 * (1.f - 2.f * cs2) : cs4 * (1.f - cs2));
      const float k3 = QL == 19 ? 1.f - 2.f * cs2 : 1.f - cs2;
      const float cA = QL == 19 ? 2.f * cs2 : cs2;
      const float Tx = d3 * (ex - cA * jx) * iA, Ty = d3 * (ey - cA * jy) * iA, Tz = d3 * (ez - cA * jz) * iA;
      const float Ux = d3 * bxm * iB, Uy = d3 * bym * iB, Uz = d3 * bzm * iB;
      const float Px = k3 * Tx + Ux, Qx = k3 * Tx - Ux;
      const float Py = k3 * Ty + Uy, Qy = k3 * Ty - Uy;
      const float Pz = k3 * Tz + Uz, Qz = k3 * Tz - Uz;
      const float p2 = -cs2 * d2a * (m2x + m2y + m2z);   // c-independent part of the P2a term
      // rest population: f^eq_0 = phi1 + (w0 - 1) eta mubar, R_0 = 0
      store(o.f_out, 0, om4 * f[0] + s4 * (ph1 + (k.w0 - 1.f) * emb) - k.w0 * p2);
      const float ux1 = ph1 * ux * ic2, uy1 = ph1 * uy * ic2, uz1 = ph1 * uz * ic2;
      const float rx = Rx * ic2, ry = Ry * ic2, rz = Rz * ic2;
#pragma unroll
      for (int i = 1; i < QL; ++i) {
        const int cx = LX<QL>(i), cy = LY<QL>(i), cz = LZ<QL>(i);
        // f^eq_i / w_i = eta mubar + c.phi u / cs2;  R_i / w_i = c.R / cs2
        float feq = emb, Rc = 0.f, L = p2;
        if (cx) { feq += cx > 0 ? ux1 : -ux1; Rc += cx > 0 ? rx : -rx; L += (cx > 0 ? m1x : -m1x) * d1 + d2a * m2x; }
        if (cy) { feq += cy > 0 ? uy1 : -uy1; Rc += cy > 0 ? ry : -ry; L += (cy > 0 ? m1y : -m1y) * d1 + d2a * m2y; }
        if (cz) { feq += cz > 0 ? uz1 : -uz1; Rc += cz > 0 ? rz : -rz; L += (cz > 0 ? m1z : -m1z) * d1 + d2a * m2z; }
        if (cx && cy) L += (cx * cy > 0 ? qxy : -qxy) * d2b;
        if (cx && cz) L += (cx * cz > 0 ? qxz : -qxz) * d2b;
        if (cy && cz) L += (cy * cz > 0 ? qyz : -qyz) * d2b;
        if (i < 7) {
          const float T = cx ? Tx : (cy ? Ty : Tz);
          const int c = cx + cy + cz;
          L -= c > 0 ? cA * T : -cA * T;
        } else if constexpr (QL == 19) {
          if (cx) { const float e = cy ? Px : Qx; L += cx > 0 ? e : -e; }
          if (cy) { const float e = cz ? Py : Qy; L += cy > 0 ? e : -e; }
          if (cz) { const float e = cx ? Pz : Qz; L += cz > 0 ? e : -e; }
        } else {
          const float ct = (cx > 0 ? Tx : -Tx) + (cy > 0 ? Ty : -Ty) + (cz > 0 ? Tz : -Tz);
          L += k3 * ct + (cx * cy * cz > 0 ? Ux : -Ux);
        }
        const float w = weight(k, i);
        store(o.f_out, i, om4 * f[i] + w * (s4 * feq + oh4 * Rc - L));
      }
    }
  }

  // history of this step (phi1 was written by the moment pass)
  o.h_out[nodes + node] = ux;
  o.h_out[2 * nodes + node] = uy;
  o.h_out[3 * nodes + node] = uz;
  o.h_out[4 * nodes + node] = Sx;
  o.h_out[5 * nodes + node] = Sy;
  o.h_out[6 * nodes + node] = Sz;
  if (OBS) {
    o.p_out[node] = p;
    const float u2 = ux * ux + uy * uy + uz * uz;
    if (!(u2 <= 0.25f) || !(fabsf(ph1) < 1e30f)) atomicOr(o.flag, 1u);
  }
}

// ---------------------------------------------------------------------------
// fused step, generic form (any nx): synchronous loads into the rings
// ---------------------------------------------------------------------------
struct StepSmem3 {
  float phi1[RP][N2];
  float phi0[RP][N2];
  float mub[RM][N1];
  float acor[RM][3][N1];   // S_x u_y - u_x S_y, S_x u_z - u_x S_z, S_y u_z - u_y S_z (previous step)
  InstanceConsts k;
};

template <int QL, bool OBS, typename GT>
__global__ void __launch_bounds__(NT, 2) d3q19_step(const StepArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  StepSmem3& S = *reinterpret_cast<StepSmem3*>(smem_raw);

  const int t = threadIdx.x;
  const int tx = t % TX, ty = t / TX;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int per_x = a.per_x, per_y = a.per_y, per_z = a.per_z;
  const int ntx = (nx + TX - 1) / TX;
  const int x0 = (blockIdx.x % ntx) * TX;
  const int zs = (blockIdx.x / ntx) * a.strip;
  const int ze = min(zs + a.strip, nz);
  const int y0 = blockIdx.y * TY;
  const int b = blockIdx.z;
  const int nodes = (int)a.nodes;   // < 2^31 / 19 (checked at creation)
  const int plane = nx * ny;
  static_assert(sizeof(InstanceConsts) / 4 <= NT, "constants copied one word per thread");
  if (t < (int)(sizeof(InstanceConsts) / 4))
    reinterpret_cast<float*>(&S.k)[t] = reinterpret_cast<const float*>(a.consts + b)[t];

  const GT* __restrict__ g_in = static_cast<const GT*>(a.g_in) + (long long)b * QL * nodes;
  const float* __restrict__ p0_in = a.phi0 + (long long)b * nodes;
  const float* __restrict__ h_in = a.hist_in + (long long)b * NH * nodes;
  const float* __restrict__ phi1_now = a.hist_out + (long long)b * NH * nodes;   // moment pass of this step
  const float* __restrict__ j_in = a.mom + (long long)b * 3 * nodes;
  Outs o;
  o.f_in = a.f_in + (long long)b * QL * nodes;
  o.f_out = a.f_out + (long long)b * QL * nodes;
  o.g_out = static_cast<GT*>(a.g_out) + (long long)b * QL * nodes;
  o.h_out = a.hist_out + (long long)b * NH * nodes;
  o.p_out = a.p_out + (long long)b * nodes;
  o.flag = a.flag;
  o.nx = nx; o.ny = ny; o.nz = nz; o.per_x = per_x; o.per_y = per_y; o.per_z = per_z;
  o.nodes = nodes; o.plane = plane;

  // phi0 / phi1 of logical plane zl on the two-halo tile into ring slot sl
  auto load_phi = [&](int zl, int sl) {
    const int zo = wrap_or_mirror(zl, nz, per_z) * plane;
    for (int p = t; p < N2; p += NT) {
      const int px = p % HX2, py = p / HX2;
      const int xl = x0 - 2 + px, yl = y0 - 2 + py;
      if (xl > nx + 1 || yl > ny + 1) continue;   // beyond what the last real column needs
      const int off = zo + wrap_or_mirror(yl, ny, per_y) * nx + wrap_or_mirror(xl, nx, per_x);
      S.phi1[sl][p] = phi1_now[off];
      S.phi0[sl][p] = p0_in[off];
    }
  };
  // antisymmetric products of the previous step's S and u on the one-halo tile
  auto load_hist = [&](int zl, int sl) {
    const int zo = wrap_or_mirror(zl, nz, per_z) * plane;
    for (int p = t; p < N1; p += NT) {
      const int px = p % HX1, py = p / HX1;
      const int xl = x0 - 1 + px, yl = y0 - 1 + py;
      if (xl > nx || yl > ny) continue;
      const int off = zo + wrap_or_mirror(yl, ny, per_y) * nx + wrap_or_mirror(xl, nx, per_x);
      const float ux = h_in[nodes + off], uy = h_in[2 * nodes + off], uz = h_in[3 * nodes + off];
      const float sx = h_in[4 * nodes + off], sy = h_in[5 * nodes + off], sz = h_in[6 * nodes + off];
      S.acor[sl][0][p] = sx * uy - ux * sy;
      S.acor[sl][1][p] = sx * uz - ux * sz;
      S.acor[sl][2][p] = sy * uz - uy * sz;
    }
  };
  const InstanceConsts& k = S.k;
  // mubar_1 of logical plane zl on the one-halo tile; phi ring slots of zl-1, zl, zl+1
  auto calc_mub = [&](int rm, int r0, int rp, int sl) {
    for (int p = t; p < N1; p += NT) {
      const int px = p % HX1, py = p / HX1;
      if (x0 - 1 + px > nx || y0 - 1 + py > ny) continue;
      const int i = (py + 1) * HX2 + (px + 1);
      const float lap0 = lap3(S.phi0[rm], S.phi0[r0], S.phi0[rp], i, HX2);
      const float lap1 = lap3(S.phi1[rm], S.phi1[r0], S.phi1[rp], i, HX2);
      float mu0, mu1, mu2;
      chem_pot(k, S.phi0[r0][i], S.phi1[r0][i], lap0, lap1, mu0, mu1, mu2);
      S.mub[sl][p] = mubar1_of(k, mu0, mu1, mu2);
    }
  };

  // prologue: phi planes zs-2 .. zs+1, products zs-1, zs, mubar zs-1, zs
  __syncthreads();   // constants visible
  for (int q = -2; q <= 1; ++q) load_phi(zs + q, ring(zs + q, RP));
  load_hist(zs - 1, ring(zs - 1, RM));
  load_hist(zs, ring(zs, RM));
  __syncthreads();
  calc_mub(ring(zs - 2, RP), ring(zs - 1, RP), ring(zs, RP), ring(zs - 1, RM));
  calc_mub(ring(zs - 1, RP), ring(zs, RP), ring(zs + 1, RP), ring(zs, RM));

  const int x = x0 + tx, y = y0 + ty;
  const bool own = x < nx && y < ny;
  for (int z = zs; z < ze; ++z) {
    __syncthreads();   // the rings of plane z-1 are no longer read
    load_phi(z + 2, ring(z + 2, RP));
    load_hist(z + 1, ring(z + 1, RM));
    __syncthreads();
    calc_mub(ring(z, RP), ring(z + 1, RP), ring(z + 2, RP), ring(z + 1, RM));
    __syncthreads();
    if (!own) continue;

    const int node = z * plane + y * nx + x;
    OwnIn<QL> in;
#pragma unroll
    for (int i = 0; i < QL; ++i) {
      if constexpr (std::is_same<GT, float>::value) in.g[i] = __ldcs(g_in + i * nodes + node);
      else in.g[i] = g_load(g_in[i * nodes + node], k);
    }
    in.jx = j_in[node];
    in.jy = j_in[nodes + node];
    in.jz = j_in[2 * nodes + node];
    in.php = h_in[node];
    in.upx = h_in[nodes + node];
    in.upy = h_in[2 * nodes + node];
    in.upz = h_in[3 * nodes + node];
    in.spx = h_in[4 * nodes + node];
    in.spy = h_in[5 * nodes + node];
    in.spz = h_in[6 * nodes + node];
    Rings R;
    const int rp[3] = {ring(z - 1, RP), ring(z, RP), ring(z + 1, RP)};
    const int rm[3] = {ring(z - 1, RM), ring(z, RM), ring(z + 1, RM)};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      R.p0[q] = S.phi0[rp[q]];
      R.p1[q] = S.phi1[rp[q]];
      R.mu[q] = S.mub[rm[q]];
#pragma unroll
      for (int c = 0; c < 3; ++c) R.ac[c][q] = S.acor[rm[q]][c];
    }
    R.i2 = (ty + 2) * HX2 + (tx + 2);
    R.sw2 = HX2;
    R.i1 = (ty + 1) * HX1 + (tx + 1);
    R.sw1 = HX1;
    auto ga = [&](int i) { return in.g[i]; };
    node_update<QL, OBS, GT>(k, R, in, ga, ga, o, x, y, z);
  }
}

// ---------------------------------------------------------------------------
// fused step, pipelined form (nx % 4 == 0).  The owned columns of plane z+1
// (g, j, history: 29 planes of 32 x 8 floats) arrive by three TMA tile loads
// while plane z is computed; the halo tiles of phi0 / phi1 (plane z+3) and of
// the history u, S (plane z+2) arrive by 16-byte asynchronous copies issued
// one plane ahead, with the wrap / mirror of each 4-column chunk fixed per
// CTA.  Every wait on the TMA barrier is bounded.
// ---------------------------------------------------------------------------
constexpr int PW = 40;                       // halo tile row: columns x0-4 .. x0+35 (16-byte aligned chunks)
// The pipelined kernel's tile height: 32 x kPipeTY owned columns, one thread each.  16 rows would cut the halo
// overhead per owned column (two-halo tile 1.41x instead of 1.69x the owned columns, one-halo tile 1.21x instead of
// 1.33x), but at one CTA of 16 warps per SM instead of two of 8 the barriers of the plane sweep stall the whole SM:
// measured 9 % slower on the 256^3 porous step, so 8.
constexpr int kPipeTY = 8;
constexpr int RP5 = 5;                       // phi ring: z-1 .. z+2 in use, z+3 in flight

struct TmaMaps {
  CUtensorMap g, j, h;   // g: (nx, ny, nz, QL nb), j: (.., 3 nb), h: (.., 7 nb); boxes 32 x kPipeTY x 1 x {QL, 3, 7}
};

template <int QL, typename GT, int TYP>
struct alignas(128) PipeSmem3 {
  static constexpr int NTP = TX * TYP, PR2 = TYP + 4, PR1 = TYP + 2, N1P = HX1 * (TYP + 2);
  GT gown[2][QL][NTP];              // TMA destinations: g of the owned columns (planes z, z+1),
  float own[3 + NH][NTP];           // then j 0-2 and history 3-9
  float phi1[RP5][PR2 * PW];        // two-halo tile rows y0-2 .. y0+TYP+1
  float phi0[RP5][PR2 * PW];
  float hus[2][6][PR1 * PW];        // history u, S (planes 1-6) on the one-halo tile
  float mub[RM][N1P];
  float acor[RM][3][N1P];
  float dmu[2][2][NTP];             // mu0 - mu2, mu1 - mu2 of the owned points of planes z, z+1
  InstanceConsts k;
  unsigned long long bar;
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// a shared-memory load kept where it is written (volatile asm: never merged with an earlier load)
__device__ __forceinline__ float lds_again(const float* p) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];\n" : "=f"(v) : "r"(smem_u32(p)));
  return v;
}
__device__ __forceinline__ __half lds_again(const __half* p) {
  unsigned short v;
  asm volatile("ld.shared.b16 %0, [%1];\n" : "=h"(v) : "r"(smem_u32(p)));
  return __ushort_as_half(v);
}

__device__ __forceinline__ void cp16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ void bar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_expect(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// bounded wait for phase `parity`; returns false after `polls` unsuccessful polls
__device__ __forceinline__ bool bar_wait(unsigned long long* bar, unsigned parity, int polls) {
  for (int it = 0; it < polls; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void tma_load4(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                          unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

template <int QL, bool OBS, typename GT, bool SZ = false, bool PER = false, int TYP = kPipeTY>
__global__ void __launch_bounds__(TX * TYP, TYP <= 8 ? 2 : 1)
    d3q19_step_pipe(const StepArgs a, const __grid_constant__ TmaMaps maps) {
  using Smem = PipeSmem3<QL, GT, TYP>;
  constexpr int NTP = Smem::NTP, PR2 = Smem::PR2, PR1 = Smem::PR1, N1P = Smem::N1P;
  static_assert(2 * PR2 * 10 <= NTP && 6 * PR1 * 10 <= 3 * NTP, "one phi chunk, at most three history chunks a thread");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Smem& S = *reinterpret_cast<Smem*>(smem_raw);
  constexpr unsigned kOwnBytes = QL * NTP * sizeof(GT) + (3 + NH) * NTP * 4;   // one plane's owned tiles

  const int t = threadIdx.x;
  const int tx = t % TX, ty = t / TX;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int per_x = a.per_x, per_y = a.per_y, per_z = a.per_z;
  const int ntx = (nx + TX - 1) / TX;
  const int x0 = (blockIdx.x % ntx) * TX;
  const int zs = (blockIdx.x / ntx) * a.strip;
  const int ze = min(zs + a.strip, nz);
  const int y0 = blockIdx.y * TYP;
  const int b = blockIdx.z;
  const int nodes = (int)a.nodes;
  const int plane = nx * ny;
  if (t < (int)(sizeof(InstanceConsts) / 4))
    reinterpret_cast<float*>(&S.k)[t] = reinterpret_cast<const float*>(a.consts + b)[t];

  const float* __restrict__ p0_in = a.phi0 + (long long)b * nodes;
  const float* __restrict__ h_in = a.hist_in + (long long)b * NH * nodes;
  const float* __restrict__ phi1_now = a.hist_out + (long long)b * NH * nodes;   // moment pass of this step
  Outs o;
  o.f_in = a.f_in + (long long)b * QL * nodes;
  o.f_out = a.f_out + (long long)b * QL * nodes;
  o.g_out = static_cast<GT*>(a.g_out) + (long long)b * QL * nodes;
  o.h_out = a.hist_out + (long long)b * NH * nodes;
  o.p_out = a.p_out + (long long)b * nodes;
  o.flag = a.flag;
  o.nx = nx; o.ny = ny; o.nz = nz; o.per_x = per_x; o.per_y = per_y; o.per_z = per_z;
  o.nodes = nodes; o.plane = plane;

  // Chunk copies of this thread, fixed for the whole sweep.  A chunk is four
  // columns xs .. xs+3 of one row: inside the lattice or wrapped it is one
  // 16-byte copy from column `off`; mirrored it is four 4-byte copies from
  // off, off-1, off-2, off-3; mode -1 skips it.
  //   phi chunk  t        (t < 2 PR2 10): array t / (PR2 10) (phi1, phi0), row, chunk of the two-halo tile
  //   hist chunk t + NTP m (< 6 PR1 10): array id / (PR1 10) (u_x .. S_z), row, chunk of the one-halo tile
  auto chunk = [&](int ylog, int xs, int ymax, int xmax, int& off, int& mode) {
    mode = -1;
    off = 0;
    if (ylog > ymax || xs > xmax) return;
    const int yr = wrap_or_mirror(ylog, ny, per_y) * nx;
    if (xs >= 0 && xs < nx) {
      mode = 0;
      off = yr + xs;
    } else if (per_x) {
      mode = 0;
      off = yr + (xs < 0 ? xs + nx : xs - nx);
    } else {
      mode = 1;
      off = yr + (xs < 0 ? -1 - xs : 2 * nx - 1 - xs);
    }
  };
  int pc_off, pc_mode, pc_dst;
  const float* pc_src;
  {
    const int arr = t / (PR2 * 10), rem = t % (PR2 * 10), r = rem / 10, kk = rem % 10;
    chunk(y0 - 2 + r, x0 - 4 + 4 * kk, ny + 1, nx + 1, pc_off, pc_mode);
    if (t >= 2 * PR2 * 10) pc_mode = -1;
    pc_dst = r * PW + 4 * kk;
    pc_src = arr == 0 ? phi1_now : p0_in;
  }
  int hc_off[3], hc_mode[3], hc_dst[3], hc_arr[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const int id = t + NTP * m;
    const int arr = id / (PR1 * 10), rem = id % (PR1 * 10), r = rem / 10, kk = rem % 10;
    chunk(y0 - 1 + r, x0 - 4 + 4 * kk, ny, nx, hc_off[m], hc_mode[m]);
    if (id >= 6 * PR1 * 10) hc_mode[m] = -1;
    hc_dst[m] = r * PW + 4 * kk;
    hc_arr[m] = arr;
  }
  auto copy_chunk = [&](float* dst, const float* src, int mode) {
    if (mode == 0) {
      cp16(dst, src);
    } else if (mode == 1) {
      cp4(dst, src);
      cp4(dst + 1, src - 1);
      cp4(dst + 2, src - 2);
      cp4(dst + 3, src - 3);
    }
  };
  auto issue_phi = [&](int zl) {
    if (pc_mode < 0) return;
    const int zo = wrap_or_mirror(zl, nz, per_z) * plane;
    float* base = (t / (PR2 * 10) == 0 ? S.phi1 : S.phi0)[ring(zl, RP5)];
    copy_chunk(base + pc_dst, pc_src + zo + pc_off, pc_mode);
  };
  auto issue_hist = [&](int zl) {
    const int zo = wrap_or_mirror(zl, nz, per_z) * plane;
    const int sl = zl & 1;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      if (hc_mode[m] < 0) continue;
      copy_chunk(&S.hus[sl][hc_arr[m]][hc_dst[m]], h_in + (hc_arr[m] + 1) * nodes + zo + hc_off[m], hc_mode[m]);
    }
  };
  // The owned tiles of plane z complete one phase of the barrier: g into its slot of the two-plane ring
  // (armed with the bytes of all three tiles), then j and the history into their single slot.
  auto issue_own_g = [&](int z) {   // one thread
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    bar_expect(&S.bar, kOwnBytes);
    tma_load4(S.gown[z & 1][0], &maps.g, x0, y0, z, b * QL, &S.bar);
  };
  auto issue_own_jh = [&](int z) {   // one thread, after issue_own_g(z)
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    tma_load4(S.own[0], &maps.j, x0, y0, z, b * 3, &S.bar);
    tma_load4(S.own[3], &maps.h, x0, y0, z, b * NH, &S.bar);
  };

  const InstanceConsts& k = S.k;
  auto mub_at = [&](int zl, int p) {   // phi ring planes zl-1 .. zl+1 -> mubar ring slot of zl, point p
    const int px = p % HX1, py = p / HX1;
    if (x0 - 1 + px > nx || y0 - 1 + py > ny) return;
    const float* q0[3] = {S.phi0[ring(zl - 1, RP5)], S.phi0[ring(zl, RP5)], S.phi0[ring(zl + 1, RP5)]};
    const float* q1[3] = {S.phi1[ring(zl - 1, RP5)], S.phi1[ring(zl, RP5)], S.phi1[ring(zl + 1, RP5)]};
    const int i = (py + 1) * PW + (px + 3);
    float mu0, mu1, mu2;
    chem_pot(k, q0[1][i], q1[1][i], lap3(q0[0], q0[1], q0[2], i, PW), lap3(q1[0], q1[1], q1[2], i, PW), mu0, mu1,
             mu2);
    S.mub[ring(zl, RM)][p] = mubar1_of(k, mu0, mu1, mu2);
    // owned point: keep the differences the node update of plane zl uses
    if (px >= 1 && px <= TX && py >= 1 && py <= TYP) {
      const int ow = (py - 1) * TX + (px - 1);
      S.dmu[zl & 1][0][ow] = mu0 - mu2;
      S.dmu[zl & 1][1][ow] = mu1 - mu2;
    }
  };
  auto prod_at = [&](int zl, int p) {  // history slot of zl -> product ring slot of zl, point p
    const int px = p % HX1, py = p / HX1;
    if (x0 - 1 + px > nx || y0 - 1 + py > ny) return;
    const int sl = zl & 1;
    const int rm = ring(zl, RM);
    const int i = py * PW + (px + 3);
    const float ux = S.hus[sl][0][i], uy = S.hus[sl][1][i], uz = S.hus[sl][2][i];
    const float sx = S.hus[sl][3][i], sy = S.hus[sl][4][i], sz = S.hus[sl][5][i];
    S.acor[rm][0][p] = sx * uy - ux * sy;
    S.acor[rm][1][p] = sx * uz - ux * sz;
    S.acor[rm][2][p] = sy * uz - uy * sz;
  };
  auto calc_mub = [&](int zl) {
    for (int p = t; p < N1P; p += NTP) mub_at(zl, p);
  };
  auto calc_prod = [&](int zl) {
    for (int p = t; p < N1P; p += NTP) prod_at(zl, p);
  };
  // Both on the one-halo tile (N1P points: 340 on 256 threads for 8 rows, 612 on 512 for 16), balanced by whole
  // warps: every thread takes the mubar_1 point t; the first XW threads the remaining mubar_1 points, the others
  // all the products (about a seventh of a mubar_1 point's work each), so no warp runs two of both while the others
  // wait at the barrier.
  constexpr int XW = ((N1P - NTP + 31) / 32) * 32;
  static_assert(N1P > NTP && N1P <= 3 * (NTP - XW), "halo work split of the tile");
  auto calc_halo = [&](int zl) {
    mub_at(zl, t);
    if (t < XW) {
      if (t + NTP < N1P) mub_at(zl, t + NTP);
    } else if (!SZ) {
      for (int p = t - XW; p < N1P; p += NTP - XW) prod_at(zl, p);
    }
  };

  // prologue
  if (t == 0) {
    bar_init(&S.bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();   // constants and barrier visible
  if (t == 0) {
    issue_own_g(zs);
    issue_own_jh(zs);
  }
  for (int q = -2; q <= 1; ++q) issue_phi(zs + q);
  issue_hist(zs - 1);
  issue_hist(zs);
  cp_commit();
  cp_wait_all();
  __syncthreads();
  calc_mub(zs - 1);
  calc_mub(zs);
  if (!SZ) {
    calc_prod(zs - 1);
    calc_prod(zs);
  }
  __syncthreads();   // history slot of zs-1 is free again
  issue_phi(zs + 2);
  issue_hist(zs + 1);
  cp_commit();

  const int x = x0 + tx, y = y0 + ty;
  const bool own = x < nx && y < ny;
  bool ok = true;
  unsigned pending = 0;
  for (int z = zs; z < ze; ++z) {
    cp_wait_all();                                      // phi z+2, history z+1
    const unsigned parity = (unsigned)(z - zs) & 1u;
    // every thread records the phase it waits on: after a block-wide give-up, the drain below waits on that
    // load (immediately satisfied for threads that saw it land) and not on the next, never-issued phase
    pending = parity;
    if (!bar_wait(&S.bar, parity, a.wait_polls)) ok = false;   // owned planes of z
    if (!__syncthreads_and(ok)) {
      if (t == 0) atomicOr(o.flag, 2u);
      ok = false;
      break;
    }
    // the g slot of z+1 held z-1, whose node updates are done
    if (t == 0 && z + 1 < ze) issue_own_g(z + 1);
    if (z + 3 <= ze + 1) issue_phi(z + 3);
    if (z + 2 <= ze) issue_hist(z + 2);
    cp_commit();
    calc_halo(z + 1);
    __syncthreads();

    // owned j and history of plane z into registers, then their slot takes plane z+1; g stays in its slot and
    // is read where the node update uses it
    OwnIn<QL> in;
    in.jx = S.own[0][t];
    in.jy = S.own[1][t];
    in.jz = S.own[2][t];
    in.php = S.own[3][t];
    in.upx = S.own[4][t];
    in.upy = S.own[5][t];
    in.upz = S.own[6][t];
    in.spx = S.own[7][t];
    in.spy = S.own[8][t];
    in.spz = S.own[9][t];
    in.d02 = S.dmu[z & 1][0][t];
    in.d12 = S.dmu[z & 1][1][t];
    __syncthreads();
    if (t == 0 && z + 1 < ze) issue_own_jh(z + 1);
    if (!own) continue;

    Rings R;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      R.p0[q] = S.phi0[ring(z - 1 + q, RP5)];
      R.p1[q] = S.phi1[ring(z - 1 + q, RP5)];
      R.mu[q] = S.mub[ring(z - 1 + q, RM)];
#pragma unroll
      for (int c = 0; c < 3; ++c) R.ac[c][q] = S.acor[ring(z - 1 + q, RM)][c];
    }
    R.i2 = (ty + 2) * PW + (tx + 4);
    R.sw2 = PW;
    R.i1 = (ty + 1) * HX1 + (tx + 1);
    R.sw1 = HX1;
    const GT* gs = &S.gown[z & 1][0][t];
    auto ga = [&](int i) { return g_load(gs[i * NTP], k); };
    // the collision reads the populations again, by loads the compiler does not merge with the first ones,
    // so they need no registers over the stencil and force evaluation
    auto gl = [&](int i) { return g_load(lds_again(gs + i * NTP), k); };
    node_update<QL, OBS, GT, true, SZ, PER>(k, R, in, ga, gl, o, x, y, z);
  }
  // leave no copy in flight: asynchronous copies, and a TMA load issued for a plane not processed
  cp_wait_all();
  // one more bounded wait, at the default limit, for the TMA load that was late
  if (!ok) (void)bar_wait(&S.bar, pending, kWaitPollsDefault);
}

}  // namespace

cudaError_t launch_d3q19_init(const float* phi0, const float* phi1, float* f, void* g, int g_half, float* hist,
                              const InstanceConsts* consts, int nx, int ny, int nz, int per_x, int per_y,
                              int per_z, int nbatch, int q, cudaStream_t s) {
  const long long total = (long long)nx * ny * nz * nbatch;
  const unsigned blocks = (unsigned)std::min<long long>((total + 255) / 256, 1LL << 20);
  auto run = [&](auto qtag, auto* gp) {
    constexpr int QL = decltype(qtag)::value;
    d3q19_init<QL><<<blocks, 256, 0, s>>>(phi0, phi1, f, gp, hist, consts, nx, ny, nz, per_x, per_y, per_z, nbatch);
  };
  if (q == 15) {
    if (g_half) run(std::integral_constant<int, 15>(), static_cast<__half*>(g));
    else run(std::integral_constant<int, 15>(), static_cast<float*>(g));
  } else {
    if (g_half) run(std::integral_constant<int, 19>(), static_cast<__half*>(g));
    else run(std::integral_constant<int, 19>(), static_cast<float*>(g));
  }
  return cudaGetLastError();
}

cudaError_t launch_d3q19_moments(const StepArgs& a, int nbatch, cudaStream_t s) {
  const int nodes = (int)a.nodes;
  const int vec4 = (nodes & 3) == 0;
  const int per_thread = vec4 ? 4 : 1;
  const int mblocks = (nodes / per_thread + 255) / 256;
  const float* f = static_cast<const float*>(a.f_in);
  if (a.q == 15) d3q_moments<15><<<dim3(mblocks, nbatch), 256, 0, s>>>(f, a.hist_out, a.mom, nodes, vec4);
  else d3q_moments<19><<<dim3(mblocks, nbatch), 256, 0, s>>>(f, a.hist_out, a.mom, nodes, vec4);
  return cudaGetLastError();
}

size_t d3q19_maps_bytes() { return sizeof(TmaMaps); }

int build_d3q19_maps(const void* g, int g_half, const float* mom, const float* hist, int nx, int ny, int nz,
                     int nbatch, int q, void* out) {
  if (nx % (g_half ? 8 : 4) != 0) return 1;   // TMA strides must be multiples of 16 bytes
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr) != cudaSuccess ||
        qr != cudaDriverEntryPointSuccess || !fn)
      return -1;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  TmaMaps m;
  auto one = [&](CUtensorMap* map, const void* base, int planes, bool half) {
    const cuuint64_t es = half ? 2 : 4;
    const cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)planes * nbatch};
    const cuuint64_t strides[3] = {(cuuint64_t)nx * es, (cuuint64_t)nx * ny * es, (cuuint64_t)nx * ny * nz * es};
    const cuuint32_t box[4] = {TX, kPipeTY, 1, (cuuint32_t)planes};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return encode(map, half ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                  const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  if (!one(&m.g, g, q, g_half != 0) || !one(&m.j, mom, 3, false) || !one(&m.h, hist, NH, false)) return -1;
  memcpy(out, &m, sizeof m);
  return 0;
}

template <int QL, typename GT>
cudaError_t launch_step_q(const StepArgs& a, int nbatch, bool observe, cudaStream_t s, const void* maps) {
  cudaError_t e = cudaSuccess;
  const int ntx = (a.nx + TX - 1) / TX;
  const int nstrips = (a.nz + a.strip - 1) / a.strip;
  dim3 grid(ntx * nstrips, (a.ny + TY - 1) / TY, nbatch);
  if (maps) {
    TmaMaps m;
    memcpy(&m, maps, sizeof m);
    const size_t smem = sizeof(PipeSmem3<QL, GT, kPipeTY>);
    constexpr int NTP = TX * kPipeTY;
    grid.y = (a.ny + kPipeTY - 1) / kPipeTY;
    static std::atomic<unsigned long long> configured{0};
    e = smem_opt_in(configured, smem, d3q19_step_pipe<QL, true, GT>, d3q19_step_pipe<QL, false, GT>,
                    d3q19_step_pipe<QL, true, GT, true>, d3q19_step_pipe<QL, false, GT, true>,
                    d3q19_step_pipe<QL, false, GT, false, true>, d3q19_step_pipe<QL, false, GT, true, true>);
    if (e != cudaSuccess) return e;
    // the periodic form for the non-observing steps of fully periodic lattices (observing steps are rare)
    const bool per = a.per_x && a.per_y && a.per_z && !observe;
    if (a.s_zero) {   // equal fluid densities: no mass flux, no correction force
      if (observe) d3q19_step_pipe<QL, true, GT, true><<<grid, NTP, smem, s>>>(a, m);
      else if (per) d3q19_step_pipe<QL, false, GT, true, true><<<grid, NTP, smem, s>>>(a, m);
      else d3q19_step_pipe<QL, false, GT, true><<<grid, NTP, smem, s>>>(a, m);
    } else {
      if (observe) d3q19_step_pipe<QL, true, GT><<<grid, NTP, smem, s>>>(a, m);
      else if (per) d3q19_step_pipe<QL, false, GT, false, true><<<grid, NTP, smem, s>>>(a, m);
      else d3q19_step_pipe<QL, false, GT><<<grid, NTP, smem, s>>>(a, m);
    }
    return cudaGetLastError();
  }
  const size_t smem = sizeof(StepSmem3);
  static std::atomic<unsigned long long> configured{0};   // devices where both variants were raised
  e = smem_opt_in(configured, smem, d3q19_step<QL, true, GT>, d3q19_step<QL, false, GT>);
  if (e != cudaSuccess) return e;
  if (observe) d3q19_step<QL, true, GT><<<grid, NT, smem, s>>>(a);
  else d3q19_step<QL, false, GT><<<grid, NT, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_d3q19_step(const StepArgs& a, int nbatch, bool observe, cudaStream_t s, const void* maps) {
  if (a.q == 15)
    return a.g_half ? launch_step_q<15, __half>(a, nbatch, observe, s, maps)
                    : launch_step_q<15, float>(a, nbatch, observe, s, maps);
  return a.g_half ? launch_step_q<19, __half>(a, nbatch, observe, s, maps)
                  : launch_step_q<19, float>(a, nbatch, observe, s, maps);
}

}  // namespace lbm
