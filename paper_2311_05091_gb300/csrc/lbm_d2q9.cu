// D2Q9 kernels of the coupled CH + NS step (Zhan, Chai, Shi, arXiv 2311.05091).
//
// One fused kernel per time step.  Each CTA owns a strip of BX columns and
// `strip` rows and sweeps it from bottom to top with shared-memory rings:
//
//   stage 1, row y+2: phi1 = sum_i f_i (push-streamed populations at rest in
//            HBM) for the CTA's columns plus two halo columns each side, and
//            phi0; the owned populations are kept for the collision.
//   stage 2, row y+1: mubar_1 from the isotropic stencil of phi0 / phi1
//            (Sec. 2.1, Eq. CHmodel) on BX + 2 columns; history (u, S) of the
//            previous step for the correction-force stencil.
//   stage 3, row y:   gradients, forces, velocity, pressure, both Hermite
//            collisions in closed form (Sec. 3, Sec. 4 intro, Appendix A) and
//            the push-streaming store with half-way bounce-back.
//
// HBM traffic per node and step: f and g read and written (144 B), phi0 read
// (4 B), history phi1/u/S read and written (40 B): 188 B.  Halo rows and
// columns are re-read from L2.
//
// Layouts: see include/lbm.h.  The NS rest population is stored minus the
// constant rho_0 of lambda_0, so every stored g is O(p/cs2) and float32 keeps
// its relative precision; the dynamics do not depend on that constant.
#include <cuda_fp16.h>

#include <type_traits>

#include "lbm_internal.cuh"

namespace lbm {
namespace {

constexpr int BX = 128;   // columns (threads) per CTA
constexpr int RP = 4;     // ring depth of phi0 / phi1 rows (y-1 .. y+2 live in one iteration)
constexpr int RM = 3;     // ring depth of mubar / history rows
constexpr float kOneMinusPhi0Floor = 5.9604644775390625e-8f;  // 2^-24

__device__ __forceinline__ int wrap_or_mirror(int i, int n, int per) {
  if (per) {
    i %= n;
    return i < 0 ? i + n : i;
  }
  if (i < 0) return -1 - i;          // mirror ghost across the half-way wall
  if (i >= n) return 2 * n - 1 - i;
  return i;
}

// Row index inside the lattice for a row that lies at most one period outside
// it (every row the sweep touches: ys - 4 .. ye + D + 2 with a strip no
// longer than the lattice), without an integer division; other rows take the
// general form.
__device__ __forceinline__ int wrap_or_mirror_row(int i, int n, int per) {
  if (i >= 0 && i < n) return i;
  if (per && i >= -n && i < 2 * n) return i < 0 ? i + n : i - n;
  return wrap_or_mirror(i, n, per);
}

// Ring slot of row r >= -64 n (the sweep starts at most four rows below 0):
// one unsigned modulo by the compile-time ring depth.
__device__ __forceinline__ int ring(int r, int n) { return (int)((unsigned)(r + 64 * n) % (unsigned)n); }

// 3x3 neighbourhood: centre, axis (e, n, w, s) and diagonal (ne, nw, sw, se).
struct P9 {
  float c, e, n, w, s, ne, nw, sw, se;
};

// Isotropic central gradient with the D2Q9 weights of d0 = 1/3:
// grad v = sum_i w_i c_i v(x + c_i) / (1/3), w = 1/9 (axis), 1/36 (diagonal).
__device__ __forceinline__ void iso_grad(const P9& v, float& gx, float& gy) {
  gx = (v.e - v.w) * (1.f / 3.f) + ((v.ne + v.se) - (v.nw + v.sw)) * (1.f / 12.f);
  gy = (v.n - v.s) * (1.f / 3.f) + ((v.ne + v.nw) - (v.se + v.sw)) * (1.f / 12.f);
}

// Isotropic Laplacian: sum_i 2 w_i (v(x + c_i) - v(x)) / (1/3).
__device__ __forceinline__ float iso_lap(const P9& v) {
  const float a = (v.e - v.c) + (v.w - v.c) + (v.n - v.c) + (v.s - v.c);
  const float d = (v.ne - v.c) + (v.nw - v.c) + (v.sw - v.c) + (v.se - v.c);
  return a * (2.f / 3.f) + d * (1.f / 6.f);
}

// mu_p = gamma_p psi_p, psi_p = (12/D) phi_p (1 - phi_p)(1 - 2 phi_p) - (3D/4) lap phi_p.
__device__ __forceinline__ void chem_pot(const InstanceConsts& k, float ph0, float ph1, float lap0,
                                         float lap1, float& mu0, float& mu1, float& mu2) {
  const float ph2 = 1.f - ph0 - ph1;
  const float lap2 = -lap0 - lap1;
  const float psi0 = k.c12_W * ph0 * (1.f - ph0) * (1.f - 2.f * ph0) - k.c34_W * lap0;
  const float psi1 = k.c12_W * ph1 * (1.f - ph1) * (1.f - 2.f * ph1) - k.c34_W * lap1;
  const float psi2 = k.c12_W * ph2 * (1.f - ph2) * (1.f - 2.f * ph2) - k.c34_W * lap2;
  mu0 = k.gam0 * psi0;
  mu1 = k.gam1 * psi1;
  mu2 = k.gam2 * psi2;
}

// mubar_1 = gamma_T/3 [ (mu1 - mu0)/gamma_0 + (mu1 - mu2)/gamma_2 ].
__device__ __forceinline__ float mubar1_of(const InstanceConsts& k, float mu0, float mu1, float mu2) {
  return k.gT3 * ((mu1 - mu0) * k.inv_gam0 + (mu1 - mu2) * k.inv_gam2);
}

// Natural moments (rows of M0, Appendix A) of nine populations.
struct Nat {
  float m0, mx, my, mxx, myy, mxy, mxyy, mxxy, mxxyy;
};

__device__ __forceinline__ Nat natural(const float* v) {
  Nat m;
  const float d5678 = v[5] + v[6] + v[7] + v[8];
  m.m0 = ((v[0] + v[1]) + (v[2] + v[3])) + (v[4] + d5678);
  m.mx = (v[1] - v[3]) + (v[5] - v[6]) - (v[7] - v[8]);
  m.my = (v[2] - v[4]) + (v[5] + v[6]) - (v[7] + v[8]);
  m.mxx = (v[1] + v[3]) + d5678;
  m.myy = (v[2] + v[4]) + d5678;
  m.mxy = (v[5] - v[6]) + (v[7] - v[8]);
  m.mxyy = (v[5] - v[6]) - (v[7] - v[8]);
  m.mxxy = (v[5] + v[6]) - (v[7] + v[8]);
  m.mxxyy = d5678;
  return m;
}

// Populations from natural moments (M0^-1 in closed form).
__device__ __forceinline__ void from_natural(const Nat& m, float* v) {
  v[0] = m.m0 - m.mxx - m.myy + m.mxxyy;
  v[1] = 0.5f * (m.mx + m.mxx - m.mxyy - m.mxxyy);
  v[2] = 0.5f * (m.my + m.myy - m.mxxy - m.mxxyy);
  v[3] = 0.5f * (-m.mx + m.mxx + m.mxyy - m.mxxyy);
  v[4] = 0.5f * (-m.my + m.myy + m.mxxy - m.mxxyy);
  v[5] = 0.25f * (m.mxy + m.mxyy + m.mxxy + m.mxxyy);
  v[6] = 0.25f * (-m.mxy - m.mxyy + m.mxxy + m.mxxyy);
  v[7] = 0.25f * (m.mxy - m.mxyy - m.mxxy + m.mxxyy);
  v[8] = 0.25f * (-m.mxy + m.mxyy - m.mxxy + m.mxxyy);
}

// Hermite moments H = N M0 v with the printed N (Appendix A) and back.
struct Her {
  float h0, hx, hy, hxx, hyy, hxy, hxyy, hxxy, h4;
};

__device__ __forceinline__ Her hermite(const Nat& m, float cs2, float cs4) {
  Her h;
  h.h0 = m.m0;
  h.hx = m.mx;
  h.hy = m.my;
  h.hxx = m.mxx - cs2 * m.m0;
  h.hyy = m.myy - cs2 * m.m0;
  h.hxy = m.mxy;
  h.hxyy = m.mxyy - cs2 * m.mx;
  h.hxxy = m.mxxy - cs2 * m.my;
  h.h4 = m.mxxyy - cs2 * (m.mxx + m.myy) + cs4 * m.m0;
  return h;
}

__device__ __forceinline__ Nat natural_of(const Her& h, float cs2, float cs4) {
  Nat m;
  m.m0 = h.h0;
  m.mx = h.hx;
  m.my = h.hy;
  m.mxx = h.hxx + cs2 * h.h0;
  m.myy = h.hyy + cs2 * h.h0;
  m.mxy = h.hxy;
  m.mxyy = h.hxyy + cs2 * h.hx;
  m.mxxy = h.hxxy + cs2 * h.hy;
  m.mxxyy = h.h4 + cs2 * (h.hxx + h.hyy) + cs4 * h.h0;
  return m;
}




// ---------------------------------------------------------------------------
// initial state: f = f^eq(phi1, mubar_1, u = 0), g = g^eq(p = 0, u = 0) - rho_0 e_0 = 0,
// history = (phi1, 0, 0, 0, 0)
// ---------------------------------------------------------------------------
template <typename GT>
__global__ void d2q9_init(const float* __restrict__ phi0_all, const float* __restrict__ phi1_all,
                          float* __restrict__ f_all, GT* __restrict__ g_all, float* __restrict__ hist_all,
                          const InstanceConsts* __restrict__ consts, int nx, int ny, int per_x, int per_y) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  const int b = blockIdx.z;
  if (x >= nx) return;
  const InstanceConsts& k = consts[b];
  const long long plane = (long long)nx * ny;
  const float* phi0 = phi0_all + (long long)b * plane;
  const float* phi1 = phi1_all + (long long)b * 5 * plane;   // staged in a history plane
  auto at = [&](const float* a, int dx, int dy) {
    const int xx = wrap_or_mirror(x + dx, nx, per_x), yy = wrap_or_mirror(y + dy, ny, per_y);
    return a[(long long)yy * nx + xx];
  };
  P9 v0{at(phi0, 0, 0), at(phi0, 1, 0), at(phi0, 0, 1), at(phi0, -1, 0), at(phi0, 0, -1),
        at(phi0, 1, 1), at(phi0, -1, 1), at(phi0, -1, -1), at(phi0, 1, -1)};
  P9 v1{at(phi1, 0, 0), at(phi1, 1, 0), at(phi1, 0, 1), at(phi1, -1, 0), at(phi1, 0, -1),
        at(phi1, 1, 1), at(phi1, -1, 1), at(phi1, -1, -1), at(phi1, 1, -1)};
  float mu0, mu1, mu2;
  chem_pot(k, v0.c, v1.c, iso_lap(v0), iso_lap(v1), mu0, mu1, mu2);
  const float emb = k.eta * mubar1_of(k, mu0, mu1, mu2);
  const long long node = (long long)y * nx + x;
  float* f = f_all + (long long)b * 9 * plane;
  GT* g = g_all + (long long)b * 9 * plane;
  float* h = hist_all + (long long)b * 5 * plane;
  f[node] = v1.c + (k.w0 - 1.f) * emb;
#pragma unroll
  for (int i = 1; i < 9; ++i) f[(long long)i * plane + node] = (i < 5 ? k.wa : k.we) * emb;
#pragma unroll
  for (int i = 0; i < 9; ++i) g[(long long)i * plane + node] = GT(0.f);
  h[node] = v1.c;
#pragma unroll
  for (int q = 1; q < 5; ++q) h[(long long)q * plane + node] = 0.f;
}

// ---------------------------------------------------------------------------
// fused step, software-pipelined: the CTA streams row y+2+D of every array it
// reads into a shared-memory slot with asynchronous copies while rows y+2 ..
// y are processed, so D rows of loads stay in flight across the compute.
// Own columns travel in 16-byte copies when the row length allows it; halo
// columns (two each side for f and phi0, one for the history) in 4-byte
// copies with periodic wrap or mirror ghosts.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__device__ __forceinline__ int inc_mod(int v, int n) { return v + 1 == n ? 0 : v + 1; }

constexpr int PAD = 4;          // own columns start 16 bytes into each slot row
constexpr int W = BX + 2 * PAD; // slot row width

// Rows staged by asynchronous copies, one ring per group of arrays, each as
// deep as that group's rows live: f and phi0 only feed stage 1 (phi1 = sum f
// of row y+2, first moment j of the owned columns), the history feeds stage 2
// (row y+1) and stage 3 (row y), g only stage 3.
struct ARow {
  float rows[10][W];   // f 0-8, phi0 9; two halo columns each side
};
struct HRow {
  float rows[5][W];    // history phi1, ux, uy, Sx, Sy; one halo column each side
};
// g rows start 16 bytes in, like the float rows, whatever the element size
template <typename GT>
__host__ __device__ constexpr int gpad() { return 16 / (int)sizeof(GT); }
template <typename GT>
struct GRow {
  GT rows[9][BX + 2 * gpad<GT>()];   // g, owned columns (float, or FP16 scaled by gsc)
};

// NS population element conversions: float storage is exact; FP16 storage
// keeps g * gsc, gsc a power of two, rounded to nearest.
__device__ __forceinline__ float g_load(float v, const InstanceConsts&) { return v; }
__device__ __forceinline__ float g_load(__half v, const InstanceConsts& k) { return __half2float(v) * k.gsci; }
__device__ __forceinline__ void g_store(float* p, float v, const InstanceConsts&) { *p = v; }
__device__ __forceinline__ void g_store(__half* p, float v, const InstanceConsts& k) {
  *p = __float2half_rn(v * k.gsc);
}

template <int D, typename GT>
struct StepSmem {
  ARow a[D + 1];
  HRow h[D + 2];
  GRow<GT> g[D + 1];
  float phi1[RP][BX + 4];
  float phi0[RP][BX + 4];
  float mub[RM][BX + 2];
  float acorr[RM][BX + 2];   // S_x u_y - u_x S_y of the previous step
  InstanceConsts k;
};

template <int D, typename GT>
constexpr size_t step_smem_bytes() { return sizeof(StepSmem<D, GT>); }

// One CTA's work: columns x0 .. x0+127 and rows ys .. ys+strip-1 of instance b.
// PER: both axes periodic (known at compile time), so no push can meet a wall
template <bool OBS, int D, typename GT, bool PER>
__device__ __forceinline__ void step_tile(const StepArgs& a, StepSmem<D, GT>& S, const int x0, const int ys,
                                          const int b) {
  constexpr bool kHalf = std::is_same<GT, __half>::value;

  const int t = threadIdx.x;
  const int nx = a.nx, ny = a.ny, per_x = a.per_x, per_y = a.per_y;
  const int ye = min(ys + a.strip, ny);
  const long long plane = a.nodes;
  static_assert(sizeof(InstanceConsts) / 4 <= BX, "constants copied one word per thread");
  if (t < (int)(sizeof(InstanceConsts) / 4))
    reinterpret_cast<float*>(&S.k)[t] = reinterpret_cast<const float*>(a.consts + b)[t];

  // base pointers of the 24 source planes: f 0-8, phi0 9, history 10-14, g 15-23
  const float* __restrict__ f_in = a.f_in + (long long)b * 9 * plane;
  const GT* __restrict__ g_in = static_cast<const GT*>(a.g_in) + (long long)b * 9 * plane;
  const float* __restrict__ p0_in = a.phi0 + (long long)b * plane;
  const float* __restrict__ h_in = a.hist_in + (long long)b * 5 * plane;
  float* __restrict__ f_out = a.f_out + (long long)b * 9 * plane;
  GT* __restrict__ g_out = static_cast<GT*>(a.g_out) + (long long)b * 9 * plane;
  float* __restrict__ h_out = a.hist_out + (long long)b * 5 * plane;
  // the 15 float source planes: f 0-8, phi0 9, history 10-14 (g, 15-23, separately)
  auto src_plane = [&](int arr) -> const float* {
    return arr < 9 ? f_in + arr * plane : (arr == 9 ? p0_in : h_in + (arr - 10) * plane);
  };
  // destination row of float array arr in the slots of rows ra (f, phi0), rh (history)
  auto dst_row = [&](int arr, int ra, int rh) -> float* {
    return arr < 10 ? S.a[ring(ra, D + 1)].rows[arr] : S.h[ring(rh, D + 2)].rows[arr - 10];
  };

  // 16-byte copies need 16-byte aligned rows: nx % 4 == 0 and instance bases on 16 bytes (an instance of a
  // multi-size context follows the others' nodes, whose count need not be a multiple of four)
  const bool vec16 = (nx & 3) == 0 &&
                     ((reinterpret_cast<uintptr_t>(f_in) | reinterpret_cast<uintptr_t>(g_in) |
                       reinterpret_cast<uintptr_t>(p0_in) | reinterpret_cast<uintptr_t>(h_in)) & 15) == 0;
  const int x = x0 + t;

  // halo copy assignment: 40 copies of f / phi0 (two columns each side), 10 of the
  // history (one column each side).  The right halo starts at xr, the first
  // column after the CTA's last real column, so a ragged last CTA stages the
  // wrapped / mirrored columns nx, nx+1 right after its real ones.
  const int xr = min(x0 + BX, nx);
  // the 50 halo copies are spread over the four warps (copy k on thread 32 (k % 4) + k / 4)
  const int hk = (t & 31) * 4 + (t >> 5);
  int h_arr = -1, h_col = 0, h_xl = 0;
  if (hk < 40) {
    const int side = hk / 10, arr = hk % 10;
    h_arr = arr;
    h_col = side < 2 ? PAD - 2 + side : PAD + (xr - x0) + (side - 2);
    h_xl = side < 2 ? x0 - 2 + side : xr + (side - 2);
  } else if (hk < 50) {
    const int side = (hk - 40) / 5, arr = 10 + (hk - 40) % 5;
    h_arr = arr;
    h_col = side == 0 ? PAD - 1 : PAD + (xr - x0);
    h_xl = side == 0 ? x0 - 1 : xr;
  }
  const bool h_active = h_arr >= 0 && h_xl <= nx + (h_arr < 10 ? 1 : 0);
  const int h_px = wrap_or_mirror(h_xl, nx, per_x);
  const float* __restrict__ h_src = h_arr >= 0 ? src_plane(h_arr) : f_in;

  // The copies issued for iteration target q: f / phi0 of row q+2, history of
  // row q+1, g of row q -- each only where a later stage reads it.
  auto issue = [&](int q) {
    const int ra = q + 2, rh = q + 1, rg = q;
    const bool need_a = ra >= ys - 2 && ra <= ye + 1;
    const bool need_h = rh >= ys - 1 && rh <= ye;
    const bool need_g = rg >= ys && rg < ye;
    const int ba = wrap_or_mirror_row(ra, ny, per_y) * nx;
    const int bh = wrap_or_mirror_row(rh, ny, per_y) * nx;
    const int bg = wrap_or_mirror_row(rg, ny, per_y) * nx;
    auto need = [&](int arr) { return arr < 10 ? need_a : need_h; };
    auto rowb = [&](int arr) { return arr < 10 ? ba : bh; };
    GT* const grow = S.g[ring(rg, D + 1)].rows[0];
    constexpr int GP = gpad<GT>(), GW = BX + 2 * GP;
    if (vec16) {
      // float chunk m of this thread: array (t >> 5) + 4 m, columns x0 + 4 (t & 31) .. + 3
      const int j = t & 31;
      const int xc = x0 + 4 * j;
      if (xc < nx) {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int arr = (t >> 5) + 4 * m;
          if (arr < 15 && need(arr)) cp_async16(dst_row(arr, ra, rh) + PAD + 4 * j, src_plane(arr) + rowb(arr) + xc);
        }
      }
      if (need_g) {
        if (!kHalf) {
#pragma unroll
          for (int m = 3; m < 6; ++m) {
            const int arr = (t >> 5) + 4 * m;
            if (arr >= 15 && xc < nx)
              cp_async16(reinterpret_cast<float*>(grow + (arr - 15) * GW + GP + 4 * j),
                         reinterpret_cast<const float*>(g_in + (arr - 15) * plane + bg + xc));
          }
        } else {
          // FP16 rows: 16 chunks of eight columns per array, 144 chunks on 128 threads
#pragma unroll
          for (int m = 0; m < 2; ++m) {
            const int id = t + BX * m;
            const int arr = id >> 4, xh = x0 + 8 * (id & 15);
            if (id < 144 && xh < nx)
              cp_async16(reinterpret_cast<float*>(grow + arr * GW + GP + 8 * (id & 15)),
                         reinterpret_cast<const float*>(g_in + arr * plane + bg + xh));
          }
        }
      }
    } else if (x < nx) {
#pragma unroll
      for (int arr = 0; arr < 15; ++arr)
        if (need(arr)) cp_async4(dst_row(arr, ra, rh) + PAD + t, src_plane(arr) + rowb(arr) + x);
      if (need_g && !kHalf) {
#pragma unroll
        for (int i = 0; i < 9; ++i)
          cp_async4(reinterpret_cast<float*>(grow + i * GW + GP + t),
                    reinterpret_cast<const float*>(g_in + i * plane + bg + x));
      }
    }
    if (h_active && need(h_arr)) cp_async4(dst_row(h_arr, ra, rh) + h_col, h_src + rowb(h_arr) + h_px);
    cp_commit();   // empty groups keep the group count uniform
  };

  const InstanceConsts& k = S.k;

  // stage 1: phi1 = sum f and phi0 of row r into phi ring row sp (ring column c = owned column c - 2); the
  // first moment j of this thread's own column stays in registers until stage 3 of row r
  auto stage1 = [&](int r, int sp, float& jx, float& jy) {
    const ARow& slot = S.a[ring(r, D + 1)];
    auto one = [&](int c, bool own) {
      const int xl = x0 - 2 + c;
      if (xl > nx + 1) return;
      const int col = c + PAD - 2;
      float v[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) v[i] = slot.rows[i][col];
      float sum = v[0];
#pragma unroll
      for (int i = 1; i < 9; ++i) sum += v[i];
      S.phi1[sp][c] = sum;
      S.phi0[sp][c] = slot.rows[9][col];
      if (own) {
        jx = (v[1] - v[3]) + (v[5] - v[6]) - (v[7] - v[8]);
        jy = (v[2] - v[4]) + (v[5] + v[6]) - (v[7] + v[8]);
      }
    };
    one(t + 2, true);
    // the four halo columns 0, 1, BX+2, BX+3, one per warp
    if ((t & 31) == 0) one((t >> 5) < 2 ? (t >> 5) : BX + (t >> 5), false);
  };

  // stage 2: mubar_1 and the correction-force product of row r (phi ring rows
  // cm, cp, cq = r-1, r, r+1) into mubar ring row sm; returns mu0 - mu2 and
  // mu1 - mu2 of this thread's own column
  auto stage2 = [&](int r, int cm, int cp, int cq, int sm, float& d02, float& d12) {
    const HRow& slot = S.h[ring(r, D + 2)];
    const float* A1m = S.phi1[cm];
    const float* A1p = S.phi1[cp];
    const float* A1q = S.phi1[cq];
    const float* A0m = S.phi0[cm];
    const float* A0p = S.phi0[cp];
    const float* A0q = S.phi0[cq];
    auto one = [&](int s, bool own) {
      const int xl = x0 - 1 + s;
      if (xl > nx) return;
      const int c = s + 1;
      const P9 v1{A1p[c], A1p[c + 1], A1q[c], A1p[c - 1], A1m[c], A1q[c + 1], A1q[c - 1], A1m[c - 1], A1m[c + 1]};
      const P9 v0{A0p[c], A0p[c + 1], A0q[c], A0p[c - 1], A0m[c], A0q[c + 1], A0q[c - 1], A0m[c - 1], A0m[c + 1]};
      float mu0, mu1, mu2;
      chem_pot(k, v0.c, v1.c, iso_lap(v0), iso_lap(v1), mu0, mu1, mu2);
      S.mub[sm][s] = mubar1_of(k, mu0, mu1, mu2);
      const int col = s + PAD - 1;
      S.acorr[sm][s] = slot.rows[3][col] * slot.rows[2][col] - slot.rows[1][col] * slot.rows[4][col];
      if (own) {
        d02 = mu0 - mu2;
        d12 = mu1 - mu2;
      }
    };
    one(t + 1, true);                 // this thread's own column
    if (t == 64) one(0, false);       // halo columns, on warps 2 and 3
    if (t == 96) one(BX + 1, false);
  };

  // The sweep starts four iterations early: iterations ys-4 .. ys-1 only run
  // the stages whose rows exist (stage 1 from row ys-2, stage 2 from row ys-1).
  const int yb = ys - 4;
  for (int q = yb; q < yb + D; ++q) issue(q);
  __syncthreads();   // constants visible
  // rotating ring indices of rows y-1, y, y+1, y+2 (phi rings) and y-1, y, y+1 (mubar rings)
  int pm = ring(yb - 1, RP), p0 = ring(yb, RP), pp = ring(yb + 1, RP), pq = ring(yb + 2, RP);
  int mm = ring(yb - 1, RM), m0 = ring(yb, RM), mp = ring(yb + 1, RM);
  float d02 = 0.f, d12 = 0.f;       // mu differences of this thread's column, row y
  float jx0 = 0.f, jy0 = 0.f, jx1 = 0.f, jy1 = 0.f;   // j of this thread's column, rows y and y+1
  for (int y = yb; y < ye; ++y) {
    cp_wait<D - 1>();          // rows of target y have landed
    __syncthreads();           // ... for every thread, and the slots refilled next are no longer read
    issue(y + D);
    float jx2 = 0.f, jy2 = 0.f;
    stage1(y + 2, pq, jx2, jy2);
    __syncthreads();
    float n02 = 0.f, n12 = 0.f;
    if (y + 1 >= ys - 1) stage2(y + 1, p0, pp, pq, mp, n02, n12);
    __syncthreads();

    // ---------------- stage 3: collide and stream row y ----------------
    if (y >= ys && x < nx) {
      const GRow<GT>& gs = S.g[ring(y, D + 1)];
      const HRow& hs = S.h[ring(y, D + 2)];
      const int c = t + 2, s = t + 1, col = t + PAD;
      const int node = y * nx + x;         // instance-relative, < 2^31 (checked at creation)
      const int pl = (int)plane;
      const float cs2 = k.cs2, cs4 = k.cs4;
      float g[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) g[i] = g_load(gs.rows[i][t + gpad<GT>()], k);
      const float php = hs.rows[0][col], uxp = hs.rows[1][col], uyp = hs.rows[2][col];
      const float Sxp = hs.rows[3][col], Syp = hs.rows[4][col];

      const float* B1m = S.phi1[pm] + c;
      const float* B10 = S.phi1[p0] + c;
      const float* B1p = S.phi1[pp] + c;
      const float* B0m = S.phi0[pm] + c;
      const float* B00 = S.phi0[p0] + c;
      const float* B0p = S.phi0[pp] + c;
      const float* Mm = S.mub[mm] + s;
      const float* M0 = S.mub[m0] + s;
      const float* Mp = S.mub[mp] + s;
      const float* Am = S.acorr[mm] + s;
      const float* A0 = S.acorr[m0] + s;
      const float* Ap = S.acorr[mp] + s;
      const P9 v1{B10[0], B10[1], B1p[0], B10[-1], B1m[0], B1p[1], B1p[-1], B1m[-1], B1m[1]};
      const P9 v0{B00[0], B00[1], B0p[0], B00[-1], B0m[0], B0p[1], B0p[-1], B0m[-1], B0m[1]};
      const P9 vm{M0[0], M0[1], Mp[0], M0[-1], Mm[0], Mp[1], Mp[-1], Mm[-1], Mm[1]};
      const P9 va{0.f, A0[1], Ap[0], A0[-1], Am[0], Ap[1], Ap[-1], Am[-1], Am[1]};

      const float ph1 = v1.c, ph0 = v0.c, ph2 = 1.f - ph0 - ph1;
      float g1x, g1y, g0x, g0y, gmx, gmy, dAx, dAy;
      iso_grad(v1, g1x, g1y);
      iso_grad(v0, g0x, g0y);
      iso_grad(vm, gmx, gmy);
      iso_grad(va, dAx, dAy);
      const float mub = vm.c;

      // degenerate mobility, mass flux S (frozen phi0), mixture properties
      const float fdeg = ph1 * (1.f - ph1) * (1.f - ph0);
      const float mob = k.M_cst + k.M_deg * fdeg;
      const float sfac = (k.rho1 - k.rho2) * mob * k.inv_gam1;
      const float Sx = sfac * gmx, Sy = sfac * gmy;
      const float rho = k.rho0 * ph0 + k.rho1 * ph1 + k.rho2 * ph2;
      const float grx = (k.rho0 - k.rho2) * g0x + (k.rho1 - k.rho2) * g1x;
      const float gry = (k.rho0 - k.rho2) * g0y + (k.rho1 - k.rho2) * g1y;
      const float muv = k.mu0 * ph0 + k.mu1 * ph1 + k.mu2 * ph2;

      // F = F_s + F_b + F_c, F_s = (mu0 - mu2) grad phi0 + (mu1 - mu2) grad phi1
      const float one_m0 = 1.f - ph0;
      const float Fx = d02 * g0x + d12 * g1x + one_m0 * k.bx - 0.5f * dAy;
      const float Fy = d02 * g0y + d12 * g1y + one_m0 * k.by + 0.5f * dAx;

      // NS moments, velocity with the solid penalisation force
      const Nat ng = natural(g);
      const float inv_rho = __frcp_rn(rho);
      const float usx = (ng.mx + 0.5f * Fx) * inv_rho;
      const float usy = (ng.my + 0.5f * Fy) * inv_rho;
      const float damp = 1.f - 0.5f * ph0;
      const float ux = usx * damp, uy = usy * damp;
      const float Ftx = Fx - ph0 * rho * usx, Fty = Fy - ph0 * rho * usy;

      // local viscous rates (s0 = s4 = s2a)
      const float om = fmaxf(one_m0, kOneMinusPhi0Floor);
      // 1/s2a = 1/2 + mu / (rho (1 - phi0) a2a), likewise s2b; IEEE-rounded reciprocals
      const float nu_e = muv * __frcp_rn(rho * om);
      const float inv_s2a = 0.5f + nu_e * k.ia2a;
      const float s2a = __frcp_rn(inv_s2a);
      const float s2b = __frcp_rn(0.5f + nu_e * k.ia2b);

      // pressure
      const float udg = ux * grx + uy * gry;
      const float q = (rho * ux - Sx) * ux + (rho * uy - Sy) * uy;
      const float rhop = k.rho0 * ph0 + k.rho1 * php + k.rho2 * (1.f - ph0 - php);
      const float qp = (rhop * uxp - Sxp) * uxp + (rhop * uyp - Syp) * uyp;
      const float H = k.Kp * ((k.h0 - k.h2) * inv_s2a + k.h3);
      const float sum_nz = ng.m0 - g[0];
      const float p = k.pf * (sum_nz + (0.5f + H) * udg - k.wq * q + 0.5f * k.Kp * (q - qp));

      // destinations of the nine pushes without branches: per axis and sign the
      // neighbour's offset (periodic wrap folded in) and whether a wall reflects
      const bool wxp = !PER && x + 1 >= nx && !per_x, wxm = !PER && x == 0 && !per_x;
      const bool wyp = !PER && y + 1 >= ny && !per_y, wym = !PER && y == 0 && !per_y;
      const int oxp = x + 1 < nx ? 1 : 1 - nx, oxm = x > 0 ? -1 : nx - 1;
      const int oyp = y + 1 < ny ? nx : nx - pl, oym = y > 0 ? -nx : pl - nx;
      auto store = [&](auto* __restrict__ out, int i, int io, int cx, int cy, float v) {
        int off = 0;
        bool bb = false;
        if (cx) { off += cx > 0 ? oxp : oxm; bb = bb || (cx > 0 ? wxp : wxm); }
        if (cy) { off += cy > 0 ? oyp : oym; bb = bb || (cy > 0 ? wyp : wym); }
        g_store(out + (bb ? io * pl + node : i * pl + node + off), v, k);
      };

      // ---- NS collision in Hermite space ----
      {
        const Her h = hermite(ng, cs2, cs4);
        const float exx = p + rho * ux * ux - Sx * ux;
        const float eyy = p + rho * uy * uy - Sy * uy;
        const float exy = rho * ux * uy - 0.5f * (Sx * uy + ux * Sy);
        const float e4 = -cs2 * p;
        const float dSxx = Sx * ux - Sxp * uxp;
        const float dSyy = Sy * uy - Syp * uyp;
        const float dSxy = 0.5f * (Sx * uy + ux * Sy) - 0.5f * (Sxp * uyp + uxp * Syp);
        const float iso = (1.f - 3.f * cs2) * udg;
        const float Mxx = 2.f * ux * Fx - dSxx + 2.f * cs2 * ux * grx + iso;
        const float Myy = 2.f * uy * Fy - dSyy + 2.f * cs2 * uy * gry + iso;
        const float Mxy = ux * Fy + Fx * uy - dSxy + cs2 * (ux * gry + grx * uy);
        Her o;
        o.h0 = h.h0 - s2a * h.h0 + (1.f - 0.5f * s2a) * udg;
        o.hx = h.hx - k.s1n * (h.hx - rho * ux) + (1.f - 0.5f * k.s1n) * Ftx;
        o.hy = h.hy - k.s1n * (h.hy - rho * uy) + (1.f - 0.5f * k.s1n) * Fty;
        o.hxx = h.hxx - s2a * (h.hxx - exx) + (1.f - 0.5f * s2a) * Mxx;
        o.hyy = h.hyy - s2a * (h.hyy - eyy) + (1.f - 0.5f * s2a) * Myy;
        o.hxy = h.hxy - s2b * (h.hxy - exy) + (1.f - 0.5f * s2b) * Mxy;
        o.hxyy = h.hxyy * (1.f - k.s3n);
        o.hxxy = h.hxxy * (1.f - k.s3n);
        o.h4 = h.h4 - s2a * (h.h4 - e4);
        float go[9];
        from_natural(natural_of(o, cs2, cs4), go);
        store(g_out, 0, 0, 0, 0, go[0]);
        store(g_out, 1, 3, 1, 0, go[1]);
        store(g_out, 2, 4, 0, 1, go[2]);
        store(g_out, 3, 1, -1, 0, go[3]);
        store(g_out, 4, 2, 0, -1, go[4]);
        store(g_out, 5, 7, 1, 1, go[5]);
        store(g_out, 6, 8, -1, 1, go[6]);
        store(g_out, 7, 5, -1, -1, go[7]);
        store(g_out, 8, 6, 1, -1, go[8]);
      }

      // ---- CH collision ----
      {
        const float jx = jx0, jy = jy0;
        const float emb = k.eta * mub;
        const float corr = k.corr_scale * (1.f - fdeg);
        // R first moment: d_t(phi1 u) + cs2 * corr * eta grad mubar
        const float Rx = (ph1 * ux - php * uxp) + cs2 * corr * k.eta * gmx;
        const float Ry = (ph1 * uy - php * uyp) + cs2 * corr * k.eta * gmy;
        float fo[9];
        if (k.ch_fast != 0.f) {
          // every moment but the first relaxes at rate 1, so f* = f^eq + w_i c_i . dj / cs2 with
          // the post-collision first moment o = phi u + (1 - s1)(j - phi u) + (1 - s1/2) R
          const float ox = ph1 * ux + (1.f - k.s1c) * (jx - ph1 * ux) + (1.f - 0.5f * k.s1c) * Rx;
          const float oy = ph1 * uy + (1.f - k.s1c) * (jy - ph1 * uy) + (1.f - 0.5f * k.s1c) * Ry;
          const float ic = __frcp_rn(cs2);
          const float ax = ox * ic, ay = oy * ic;
          fo[1] = k.wa * (emb + ax);
          fo[3] = k.wa * (emb - ax);
          fo[2] = k.wa * (emb + ay);
          fo[4] = k.wa * (emb - ay);
          fo[5] = k.we * (emb + ax + ay);
          fo[6] = k.we * (emb - ax + ay);
          fo[7] = k.we * (emb - ax - ay);
          fo[8] = k.we * (emb + ax - ay);
          // rest population closes the zeroth moment exactly
          fo[0] = ph1 - (((fo[1] + fo[3]) + (fo[2] + fo[4])) + ((fo[5] + fo[7]) + (fo[6] + fo[8])));
        } else {
          // every moment enters: the populations of this node again (L2-resident)
          float fv[9];
#pragma unroll
          for (int i = 0; i < 9; ++i) fv[i] = f_in[i * pl + node];
          Nat nf = natural(fv);
          nf.m0 = ph1;   // zeroth moment is the phase field itself
          const Her h = hermite(nf, cs2, cs4);
          const float exx = cs2 * (emb - ph1);
          Her o;
          o.h0 = ph1;
          o.hx = h.hx - k.s1c * (h.hx - ph1 * ux) + (1.f - 0.5f * k.s1c) * Rx;
          o.hy = h.hy - k.s1c * (h.hy - ph1 * uy) + (1.f - 0.5f * k.s1c) * Ry;
          o.hxx = h.hxx - k.s2ac * (h.hxx - exx);
          o.hyy = h.hyy - k.s2ac * (h.hyy - exx);
          o.hxy = h.hxy * (1.f - k.s2bc);
          o.hxyy = h.hxyy * (1.f - k.s3c);
          o.hxxy = h.hxxy * (1.f - k.s3c);
          o.h4 = h.h4 - k.s4c * (h.h4 - cs4 * (ph1 - emb));
          from_natural(natural_of(o, cs2, cs4), fo);
        }
        store(f_out, 0, 0, 0, 0, fo[0]);
        store(f_out, 1, 3, 1, 0, fo[1]);
        store(f_out, 2, 4, 0, 1, fo[2]);
        store(f_out, 3, 1, -1, 0, fo[3]);
        store(f_out, 4, 2, 0, -1, fo[4]);
        store(f_out, 5, 7, 1, 1, fo[5]);
        store(f_out, 6, 8, -1, 1, fo[6]);
        store(f_out, 7, 5, -1, -1, fo[7]);
        store(f_out, 8, 6, 1, -1, fo[8]);
      }

      // history of this step
      h_out[node] = ph1;
      h_out[pl + node] = ux;
      h_out[2 * pl + node] = uy;
      h_out[3 * pl + node] = Sx;
      h_out[4 * pl + node] = Sy;
      if (OBS) {
        a.p_out[(long long)b * plane + node] = p;
        const float u2 = ux * ux + uy * uy;
        if (!(u2 <= 0.25f) || !(fabsf(ph1) < 1e30f)) atomicOr(a.flag, 1u);
      }
    }
    d02 = n02;
    d12 = n12;
    jx0 = jx1; jy0 = jy1; jx1 = jx2; jy1 = jy2;
    // rotate the rings to row y+1
    pm = p0; p0 = pp; pp = pq; pq = inc_mod(pq, RP);
    mm = m0; m0 = mp; mp = inc_mod(mp, RM);
  }
  cp_wait<0>();
}

// one tile per CTA: grid (column tiles, row strips, instances)
template <bool OBS, int D, typename GT, bool PER>
__global__ void __launch_bounds__(BX, 5) d2q9_step(const StepArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  StepSmem<D, GT>& S = *reinterpret_cast<StepSmem<D, GT>*>(smem_raw);
  step_tile<OBS, D, GT, PER>(a, S, blockIdx.x * BX, blockIdx.y * a.strip, blockIdx.z);
}

// Persistent form for instances of different sizes: every CTA claims the next
// work item from a device counter (queue[0]) until the list is done, so CTAs
// that drew smaller items take more of them; item = (instance, x0, ys), with
// per-instance launch arguments (base pointers of that instance, its sizes and
// strip).  Which CTA runs an item does not change its result.  The CTA that
// finishes last (queue[1] counts finished CTAs) zeroes both counters for the
// next launch on the stream.
template <bool OBS, int D, typename GT, bool PER>
__global__ void __launch_bounds__(BX, 5) d2q9_step_items(const StepArgs* __restrict__ args,
                                                      const int4* __restrict__ items, int nitems,
                                                      unsigned int* __restrict__ queue) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  StepSmem<D, GT>& S = *reinterpret_cast<StepSmem<D, GT>*>(smem_raw);
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(&queue[0], 1u);
    __syncthreads();
    const int it = s_item;
    __syncthreads();   // every thread has read the claim before the next one overwrites it
    if (it >= nitems) break;
    const int4 w = items[it];
    const StepArgs a = args[w.x];
    step_tile<OBS, D, GT, PER>(a, S, w.y, w.z, 0);
    __syncthreads();   // shared memory is reused by the next item
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&queue[1], 1u) == gridDim.x - 1) {   // every other CTA has made its last claim
      queue[0] = 0u;
      queue[1] = 0u;
    }
  }
}

}  // namespace

cudaError_t launch_d2q9_init(const float* phi0, const float* phi1, float* f, void* g, int g_half, float* hist,
                             const InstanceConsts* consts, int nx, int ny, int per_x, int per_y,
                             int nbatch, cudaStream_t s) {
  dim3 block(128), grid((nx + 127) / 128, ny, nbatch);
  if (g_half)
    d2q9_init<__half><<<grid, block, 0, s>>>(phi0, phi1, f, static_cast<__half*>(g), hist, consts, nx, ny, per_x,
                                             per_y);
  else
    d2q9_init<float><<<grid, block, 0, s>>>(phi0, phi1, f, static_cast<float*>(g), hist, consts, nx, ny, per_x,
                                            per_y);
  return cudaGetLastError();
}

template <int D, typename GT, bool PER>
cudaError_t launch_per(const StepArgs& a, int nbatch, bool observe, cudaStream_t s) {
  const size_t smem = step_smem_bytes<D, GT>();
  static std::atomic<unsigned long long> configured{0};   // devices where both variants were raised
  if (cudaError_t e = smem_opt_in(configured, smem, d2q9_step<true, D, GT, PER>, d2q9_step<false, D, GT, PER>))
    return e;
  dim3 block(BX), grid((a.nx + BX - 1) / BX, (a.ny + a.strip - 1) / a.strip, nbatch);
  if (observe) d2q9_step<true, D, GT, PER><<<grid, block, smem, s>>>(a);
  else d2q9_step<false, D, GT, PER><<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

template <int D, typename GT>
cudaError_t launch_depth(const StepArgs& a, int nbatch, bool observe, cudaStream_t s) {
  return (a.per_x && a.per_y) ? launch_per<D, GT, true>(a, nbatch, observe, s)
                              : launch_per<D, GT, false>(a, nbatch, observe, s);
}

template <typename GT>
cudaError_t launch_typed(const StepArgs& a, int nbatch, bool observe, cudaStream_t s) {
  switch (a.depth) {
    case 1: return launch_depth<1, GT>(a, nbatch, observe, s);
    case 3: return launch_depth<3, GT>(a, nbatch, observe, s);
    default: return launch_depth<2, GT>(a, nbatch, observe, s);
  }
}

cudaError_t launch_d2q9_step(const StepArgs& a, int nbatch, bool observe, cudaStream_t s) {
  return a.g_half ? launch_typed<__half>(a, nbatch, observe, s) : launch_typed<float>(a, nbatch, observe, s);
}

template <int D, typename GT, bool PER>
cudaError_t items_per(const StepArgs* args, const int4* items, int nitems, int grid, bool observe,
                      unsigned int* queue, cudaStream_t s) {
  const size_t smem = step_smem_bytes<D, GT>();
  static std::atomic<unsigned long long> configured{0};
  if (cudaError_t e =
          smem_opt_in(configured, smem, d2q9_step_items<true, D, GT, PER>, d2q9_step_items<false, D, GT, PER>))
    return e;
  if (grid <= 0) {
    // persistent grid: every SM filled to its occupancy, no more CTAs than items
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, d2q9_step_items<false, D, GT, PER>, BX, smem);
    grid = sms * (per_sm > 0 ? per_sm : 1);
  }
  if (grid > nitems) grid = nitems;
  if (grid < 1) return cudaSuccess;
  if (observe) d2q9_step_items<true, D, GT, PER><<<grid, BX, smem, s>>>(args, items, nitems, queue);
  else d2q9_step_items<false, D, GT, PER><<<grid, BX, smem, s>>>(args, items, nitems, queue);
  return cudaGetLastError();
}

template <int D, typename GT>
cudaError_t items_depth(const StepArgs* args, const int4* items, int nitems, int grid, bool observe, bool periodic,
                        unsigned int* queue, cudaStream_t s) {
  return periodic ? items_per<D, GT, true>(args, items, nitems, grid, observe, queue, s)
                  : items_per<D, GT, false>(args, items, nitems, grid, observe, queue, s);
}

template <typename GT>
cudaError_t items_typed(const StepArgs* args, const int4* items, int nitems, int depth, int grid, bool observe,
                        bool periodic, unsigned int* queue, cudaStream_t s) {
  switch (depth) {
    case 1: return items_depth<1, GT>(args, items, nitems, grid, observe, periodic, queue, s);
    case 3: return items_depth<3, GT>(args, items, nitems, grid, observe, periodic, queue, s);
    default: return items_depth<2, GT>(args, items, nitems, grid, observe, periodic, queue, s);
  }
}

cudaError_t launch_d2q9_items(const StepArgs* args, const int4* items, int nitems, int depth, int g_half, int grid,
                              bool observe, bool periodic, unsigned int* queue, cudaStream_t s) {
  return g_half ? items_typed<__half>(args, items, nitems, depth, grid, observe, periodic, queue, s)
                : items_typed<float>(args, items, nitems, depth, grid, observe, periodic, queue, s);
}

}  // namespace lbm
