// Internal declarations shared by the library's translation units.
//
// Per-instance constants are derived on the host in double precision (model
// parameters of Sec. 2.2 and Sec. 3 of the paper) and stored on the device as
// float32 in one `InstanceConsts` record per batch instance.  Kernels read the
// record of their instance once (uniform address, broadcast) into registers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <initializer_list>

namespace lbm {

// Kernels with more than 48 KB of dynamic shared memory need an opt-in on
// every device they run on.  `mask` records the device ordinals (bit d) on
// which `kernels` were already raised to `bytes`; ordinals from 64 up are
// configured on every call.
template <typename... K>
cudaError_t smem_opt_in(std::atomic<unsigned long long>& mask, size_t bytes, K... kernels) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
  if (bit && (mask.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  for (const void* k : {reinterpret_cast<const void*>(kernels)...}) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
  }
  mask.fetch_or(bit, std::memory_order_acq_rel);
  return cudaSuccess;
}

struct InstanceConsts {
  // lattice (cs2 = d0, weights of the scale-factor lattice)
  float cs2, cs4, w0, wa, we;      // D2Q9: wa = axis weight, we = diagonal weight
                                   // D3Q19: wa = axis weight, we = edge weight
  // free energy (Sec. 2.1): 12/D and 3D/4
  float c12_W, c34_W;
  // spreading coefficients gamma_p, gamma_T/3, their inverses
  float gam0, gam1, gam2, gT3, inv_gam0, inv_gam1, inv_gam2;
  // CH: eta_1, mobility, rates (s1 from Sec. 3 relation, free rates)
  float eta, M_cst, M_deg, corr_scale;   // corr_scale = M_deg / (M_cst + M_deg)
  float s1c, s0c, s2ac, s2bc, s3c, s4c;
  // NS: free rates s1, s3 (s0 and s4 follow the local s2a)
  float s1n, s3n;
  // densities and dynamic viscosities of solid, fluid 1, fluid 2
  float rho0, rho1, rho2, mu0, mu1, mu2;
  // body force density
  float bx, by, bz;
  // viscosity relation mu / (rho (1 - phi0)) = (1/s2a - 1/2) a2a = (1/s2b - 1/2) a2b with
  // a2a = (c^2 - cs2)/2, a2b = cs2: their inverses
  float ia2a, ia2b;
  // pressure formula (Sec. 3): p = pf * [sum_{i!=0} g_i + (1/2 + H) u.grad rho
  //   - wq * (rho u - S).u + K/2 * d_t((rho u - S).u)],
  // H = K * (h0 * inv_s0 - h2 * inv_s2a + h3), pf = cs2/(1-w0), wq = w0/(1-cs2)
  float pf, wq, Kp, h0, h2, h3;
  float ch_fast;   // 1 when every free CH rate is 1: closed form f* = f^eq + first-moment part
  // FP16 storage of the NS populations: stored value = g * gsc (a power of two), g = stored * gsci
  float gsc, gsci;
};

// Launch arguments of the fused step kernel (both lattices).
struct StepArgs {
  const float* f_in;
  float* f_out;
  const void* g_in;       // NS populations: float, or __half scaled by gsc when g_half
  void* g_out;
  const float* phi0;
  const float* hist_in;   // [b][k][nodes]: phi1, u (d), S (d) at the previous step
  float* hist_out;
  float* p_out;           // written only by the observing variant
  float* mom;             // D3Q19: [b][3][nodes] first moment of f, written by the moment pass
  const InstanceConsts* consts;
  unsigned int* flag;     // divergence flag (observing variant)
  int nx, ny, nz;
  int per_x, per_y, per_z;
  int strip;              // rows (2D) or planes (3D) per CTA
  int depth;              // rows of asynchronous copies kept in flight (1..3)
  long long nodes;        // nodes per instance
  int g_half;             // NS populations stored as FP16
  int q;                  // lattice directions (9, 15 or 19)
  int wait_polls;         // polls of a bounded tile-load wait before it gives up (3D pipelined kernel)
  int s_zero;             // rho1 == rho2 in every instance: the mass flux S and the correction force vanish
};

// Default poll limit of a bounded device wait (mbarrier try_wait polls).
constexpr int kWaitPollsDefault = 1 << 22;

// Kernel launchers (return cudaGetLastError of the launch).
cudaError_t launch_d2q9_init(const float* phi0, const float* phi1, float* f, void* g, int g_half,
                             float* hist, const InstanceConsts* consts, int nx, int ny,
                             int per_x, int per_y, int nbatch, cudaStream_t s);
cudaError_t launch_d2q9_step(const StepArgs& a, int nbatch, bool observe, cudaStream_t s);
// Work-list form for instances of different sizes: args[inst] holds the
// instance's own base pointers, sizes and strip (device memory), items[k] =
// (inst, x0, ys, 0).  grid <= 0 picks a persistent grid of SMs x occupancy.
// periodic: every instance is periodic on both axes (no pushes meet walls).
// queue: two zeroed device counters (item claims, finished CTAs), zero again
// when the launch ends.
cudaError_t launch_d2q9_items(const StepArgs* args, const int4* items, int nitems, int depth, int g_half, int grid,
                              bool observe, bool periodic, unsigned int* queue, cudaStream_t s);

// Velocity inlet (mode bit 0, x = 0) and pressure outlet (bit 1, x = nx - 1)
// by non-equilibrium extrapolation, applied to the streamed populations of
// every instance; u_in: [d][nz][ny] inlet velocity, phi_in < 0 extrapolates phi1.
cudaError_t launch_inout(float* f, void* g, int g_half, const float* phi0, const InstanceConsts* consts,
                         const float* u_in, int mode, float phi_in, float p_out, int q, int nx, int ny, int nz,
                         long long nodes, int nbatch, cudaStream_t s);

// 3D lattices (D3Q19, D3Q15 by q) share these launchers.
cudaError_t launch_d3q19_init(const float* phi0, const float* phi1, float* f, void* g, int g_half,
                              float* hist, const InstanceConsts* consts, int nx, int ny, int nz,
                              int per_x, int per_y, int per_z, int nbatch, int q, cudaStream_t s);
// D3Q19 steps are two launches: the moment pass, then the fused kernel.
cudaError_t launch_d3q19_moments(const StepArgs& a, int nbatch, cudaStream_t s);
// maps: tensor maps of the buffers the step reads (from build_d3q19_maps), or
// nullptr for the generic kernel (any nx)
cudaError_t launch_d3q19_step(const StepArgs& a, int nbatch, bool observe, cudaStream_t s, const void* maps);
// Tensor maps of one set of input buffers (g, j scratch, history) for the
// pipelined 3D kernel: 0 on success, 1 if nx % 4 (FP16 g: 8) != 0 (not supported),
// -1 on a driver error.  out receives d3q19_maps_bytes() bytes and must be
// 64-byte aligned.
size_t d3q19_maps_bytes();
int build_d3q19_maps(const void* g, int g_half, const float* mom, const float* hist, int nx, int ny, int nz,
                     int nbatch, int q, void* out);

// Observables: deterministic two-pass reduction of one instance.
//   phi0, phi1, u (d planes), p: device fields of one instance, n nodes.
//   partials: scratch of obs_partials_len(n) doubles.  out: 8 doubles
//   [sum phi1, sum phi0, max|u|, sum p_in, n_in, sum p_out, n_out, nonfinite].
int obs_partials_blocks(long long n);
long long obs_partials_len(long long n);
// Pore-space phase fluxes of one instance along one axis (ua: that velocity component), 8 doubles to out.
cudaError_t launch_phase_flux(const float* phi0, const float* phi1, const float* ua, long long n, double* partials,
                              double* out, cudaStream_t s);
cudaError_t launch_observables(const float* phi0, const float* phi1, const float* u, int d,
                               const float* p, long long n, double* partials, double* out,
                               cudaStream_t s);

}  // namespace lbm
