// Host implementation of the C ABI declared in include/lbm.h.
//
// Parameter derivation follows the paper (arXiv 2311.05091) in float64 on
// the host; the device receives one float32 InstanceConsts record per batch
// instance.  All device work goes to the context's stream; graphs of
// kGraphSteps steps are captured once per starting buffer and replayed.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <math.h>

#include <cmath>
#include <unordered_map>

#include <nvtx3/nvToolsExt.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.cuh"

using lbm::InstanceConsts;
using lbm::StepArgs;

namespace {

constexpr int kGraphSteps = 16;     // even: a replay returns to the same buffer
constexpr uint32_t kStateMagic = 0x314d424cu;   // "LBM1"

thread_local char g_last_error[256] = "";

struct StateHeader {
  uint32_t magic;
  int32_t lattice, nx, ny, nz, nbatch, q, d;
  int64_t step;
  int64_t nodes;
  int32_t pad[4];
};

}  // namespace

struct lbm_ctx {
  int lattice = 0;
  int nx = 0, ny = 0, nz = 1, nbatch = 1, q = 9, d = 2;
  int per[3] = {0, 0, 0};
  long long nodes = 0;        // per instance
  int strip = 32;
  int depth = 1;
  int wait_polls = lbm::kWaitPollsDefault;   // lbm_set_wait_limit
  int device = 0;             // CUDA device the context was created on
  std::vector<InstanceConsts> hconsts;
  InstanceConsts* dconsts = nullptr;
  float* f[2] = {nullptr, nullptr};
  void* g[2] = {nullptr, nullptr};   // NS populations: float, or FP16 scaled by gsc (g_half)
  int g_half = 0;
  size_t g_elem = sizeof(float);
  float* hist[2] = {nullptr, nullptr};
  float* phi0 = nullptr;
  float* p = nullptr;
  float* mom = nullptr;        // D3Q19 moment-pass scratch
  // caller's device-memory callbacks (lbm_create_alloc); NULL: cudaMalloc / cudaFree
  lbm_alloc_fn alloc_fn = nullptr;
  lbm_free_fn free_fn = nullptr;
  void* alloc_user = nullptr;
  std::unordered_map<void*, size_t> alloc_bytes;
  // inlet / outlet columns (lbm_set_inout)
  int inout_mode = 0;
  float inout_phi_in = -1.f, inout_p_out = 0.f;
  float* inout_u = nullptr;    // [d][nz][ny]
  // instances of different sizes (lbm_create_multi): per-instance shape, node
  // offset into every buffer, strip; launch arguments and work items on the device
  bool multi = false;
  std::vector<int> inx, iny, istrip;
  std::vector<long long> ioff;
  long long total = 0;                 // nodes of all instances
  StepArgs* dargs[2] = {nullptr, nullptr};
  int4* ditems = nullptr;
  unsigned int* dqueue = nullptr;   // work-item claims and finished CTAs of the batched kernel (zero between launches)
  int nitems = 0, items_cap = 0;
  // D3Q19 tensor maps of the step's input buffers, one set per starting buffer
  alignas(64) unsigned char d3maps[2][512];
  bool d3maps_ok = false;
  unsigned int* dflag = nullptr;
  double* dpart = nullptr;
  double* dobs = nullptr;
  int cur = 0;
  long long step = 0;
  bool solid_set = false, phase_set = false, failed = false;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  bool profiling = false;
  std::vector<cudaEvent_t> ev;     // pairs: [2k] before, [2k+1] after launch k
  size_t ev_used = 0;
  char err[256] = "";
};

namespace {

// NVTX range for the duration of a scope (host side; a no-op unless a profiler is attached)
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

int set_err(lbm_ctx* c, int code, const char* fmt, const char* a = "", const char* b = "") {
  char* dst = c ? c->err : g_last_error;
  snprintf(dst, 256, fmt, a, b);
  if (c) snprintf(g_last_error, 256, "%s", c->err);
  return code;
}

int cuda_fail(lbm_ctx* c, cudaError_t e, const char* what) {
  if (c) c->failed = true;
  return set_err(c, LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Device memory of a context: the caller's callbacks when it gave some, else the runtime.  Memory returned to a
// caller's pool may be reused at once on other streams, so the context's stream is drained first.
cudaError_t dev_alloc(lbm_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (!c->alloc_fn) return cudaMalloc(p, bytes);
  *p = c->alloc_fn(bytes, c->stream, c->alloc_user);
  if (!*p) return cudaErrorMemoryAllocation;
  c->alloc_bytes[*p] = bytes;
  return cudaSuccess;
}

template <class T>
cudaError_t dalloc(lbm_ctx* c, T** p, size_t bytes) {
  void* v = nullptr;
  const cudaError_t e = dev_alloc(c, &v, bytes);
  *p = static_cast<T*>(v);
  return e;
}

void dev_free(lbm_ctx* c, void* p) {
  if (!p) return;
  if (!c->free_fn) {
    cudaFree(p);
    return;
  }
  if (c->stream) cudaStreamSynchronize(c->stream);
  auto it = c->alloc_bytes.find(p);
  const size_t bytes = it == c->alloc_bytes.end() ? 0 : it->second;
  if (it != c->alloc_bytes.end()) c->alloc_bytes.erase(it);
  c->free_fn(p, bytes, c->stream, c->alloc_user);
}

#define LBM_CK(c, call)                                       \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail((c), e_, #call);  \
  } while (0)

bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

// Model constants of one instance (Sec. 2.2 Eq. kk and gamma_p; Sec. 3
// relations for s1, the viscosity relation and the pressure constants).
int derive(const lbm_params& p, int lattice, InstanceConsts& k, char* why, lbm_derived* dv = nullptr) {
  const bool is3d = lattice != LBM_D2Q9;
  const double d0 = p.d0;
  if (!finite_pos(p.W)) return snprintf(why, 128, "W must be > 0"), LBM_EINVAL;
  if (!(p.M_deg >= 0.0) || !(p.M_cst >= 0.0) || !finite_pos(p.M_deg + p.M_cst))
    return snprintf(why, 128, "mobility must be >= 0 with M_cst + M_deg > 0"), LBM_EINVAL;
  if (!(p.theta_deg > 0.0 && p.theta_deg < 180.0))
    return snprintf(why, 128, "theta_deg must lie in (0, 180)"), LBM_EINVAL;
  if (!(p.kappa > -1.0) || !isfinite(p.kappa)) return snprintf(why, 128, "kappa must be > -1"), LBM_EINVAL;
  if (!finite_pos(p.sigma)) return snprintf(why, 128, "sigma must be > 0"), LBM_EINVAL;
  for (int i = 0; i < 3; ++i)
    if (!finite_pos(p.rho[i]) || !finite_pos(p.mu[i]))
      return snprintf(why, 128, "densities and viscosities must be > 0"), LBM_EINVAL;
  const double d0max = is3d ? 0.5 : 1.0;
  if (!(d0 > 0.0 && d0 < d0max)) return snprintf(why, 128, "d0 out of range for the lattice"), LBM_EINVAL;
  if (!finite_pos(p.eta_hat)) return snprintf(why, 128, "eta_hat must be > 0"), LBM_EINVAL;
  if (!(p.s_free_ch > 0.0 && p.s_free_ch < 2.0) || !(p.s_free_ns > 0.0 && p.s_free_ns < 2.0))
    return snprintf(why, 128, "free relaxation rates must lie in (0, 2)"), LBM_EINVAL;
  for (int i = 0; i < 3; ++i)
    if (!isfinite(p.body_force[i])) return snprintf(why, 128, "body force must be finite"), LBM_EINVAL;

  const double th = p.theta_deg * M_PI / 180.0;
  const double sgn = p.theta_deg > 90.0 ? 1.0 : (p.theta_deg < 90.0 ? -1.0 : 0.0);
  const double s = sin(M_PI / 4.0 * cos(th));
  const double kk = 9.0 / (1.0 + p.kappa) * (1.0 + 2.0 * sgn * s * s);
  const double s12 = p.sigma, s01 = kk * s12, s02 = s01 + s12 * cos(th);
  const double g0 = s01 + s02 - s12, g1 = s01 + s12 - s02, g2 = s02 + s12 - s01;
  if (!(g0 > 0.0 && g1 > 0.0 && g2 > 0.0))
    return snprintf(why, 128, "spreading coefficients must be positive (check kappa, theta)"), LBM_EINVAL;
  const double gT = 3.0 / (1.0 / g0 + 1.0 / g1 + 1.0 / g2);
  // The kernels compute in float32 with cs2 = float(d0).  Every lattice
  // constant below is derived from that rounded value, so identities such as
  // w0 = (1 - cs2)^2 and cs2 / (1 - w0) = 1 / (2 - cs2) hold to one rounding
  // instead of mixing two different scale factors.
  const double df = (double)(float)d0;
  const double cs2 = df;
  const double eta = p.eta_hat / g1;
  const double s1c = 1.0 / (0.5 + (p.M_cst + p.M_deg) / (g1 * eta * cs2));
  double w0, wa, we;
  if (lattice == LBM_D3Q19) {
    w0 = 1.0 - 3.0 * df + 3.0 * df * df;
    wa = (df - 2.0 * df * df) / 2.0;
    we = df * df / 4.0;
  } else if (lattice == LBM_D3Q15) {   // Appendix A: corner weight d0^2 / 8
    w0 = 1.0 - 3.0 * df + 2.0 * df * df;
    wa = (df - df * df) / 2.0;
    we = df * df / 8.0;
  } else {
    w0 = (1.0 - df) * (1.0 - df);
    wa = (df - df * df) / 2.0;
    we = df * df / 4.0;
  }
  memset(&k, 0, sizeof(k));
  k.cs2 = (float)cs2;
  k.cs4 = (float)(cs2 * cs2);
  k.w0 = (float)w0;
  k.wa = (float)wa;
  k.we = (float)we;
  k.c12_W = (float)(12.0 / p.W);
  k.c34_W = (float)(0.75 * p.W);
  k.gam0 = (float)g0;
  k.gam1 = (float)g1;
  k.gam2 = (float)g2;
  k.gT3 = (float)(gT / 3.0);
  k.inv_gam0 = (float)(1.0 / g0);
  k.inv_gam1 = (float)(1.0 / g1);
  k.inv_gam2 = (float)(1.0 / g2);
  k.eta = (float)eta;
  k.M_cst = (float)p.M_cst;
  k.M_deg = (float)p.M_deg;
  k.corr_scale = (float)(p.M_deg / (p.M_cst + p.M_deg));
  k.s1c = (float)s1c;
  k.s0c = k.s2ac = k.s2bc = k.s3c = k.s4c = (float)p.s_free_ch;
  k.ch_fast = p.s_free_ch == 1.0 ? 1.0f : 0.0f;
  // FP16 storage scale of the NS populations: 2^12 maps |g| in [1.5e-8, 16] onto normal FP16 numbers
  k.gsc = 4096.0f;
  k.gsci = 1.0f / 4096.0f;
  k.s1n = k.s3n = (float)p.s_free_ns;
  k.rho0 = (float)p.rho[0];
  k.rho1 = (float)p.rho[1];
  k.rho2 = (float)p.rho[2];
  k.mu0 = (float)p.mu[0];
  k.mu1 = (float)p.mu[1];
  k.mu2 = (float)p.mu[2];
  k.bx = (float)p.body_force[0];
  k.by = (float)p.body_force[1];
  k.bz = (float)p.body_force[2];
  k.ia2a = (float)(2.0 / (1.0 - df));
  k.ia2b = (float)(1.0 / df);
  // pressure: pf = cs2 / (1 - w0), wq = w0 / (c^2 - cs2)
  k.pf = (float)(cs2 / (1.0 - w0));
  k.wq = (float)(w0 / (1.0 - cs2));
  if (is3d) {
    k.Kp = (float)(1.0 - 2.0 * df);
    k.h0 = (float)(1.0 - df);
    k.h2 = (float)(3.0 - 7.0 * df);
    k.h3 = (float)(1.0 - 3.0 * df);
  } else {
    k.Kp = (float)(1.0 - df);
    k.h0 = (float)(1.0 - df);
    k.h2 = (float)(2.0 - 4.0 * df);
    k.h3 = (float)((1.0 - 3.0 * df) / 2.0);
  }
  if (dv) {   // the same values before rounding, for lbm_derive
    memset(dv, 0, sizeof(*dv));
    dv->k = kk;
    dv->gamma[0] = g0;
    dv->gamma[1] = g1;
    dv->gamma[2] = g2;
    dv->gamma_T = gT;
    dv->eta = eta;
    dv->s1_ch = s1c;
    dv->cs2 = cs2;
    dv->w[0] = w0;
    dv->w[1] = wa;
    dv->w[2] = we;
    dv->visc[0] = (1.0 - df) / 2.0;
    dv->visc[1] = df;
    dv->p_f = cs2 / (1.0 - w0);
    dv->p_w = w0 / (1.0 - cs2);
    dv->p_K = is3d ? 1.0 - 2.0 * df : 1.0 - df;
    dv->p_h[0] = 1.0 - df;
    dv->p_h[1] = is3d ? 3.0 - 7.0 * df : 2.0 - 4.0 * df;
    dv->p_h[2] = is3d ? 1.0 - 3.0 * df : (1.0 - 3.0 * df) / 2.0;
  }
  return LBM_OK;
}

int default_strip(const lbm_ctx* c) {
  // 16 rows per CTA measured best for the D2Q9 kernel on GB300 (sweep over
  // 16..64 rows on the 1024^2 x 5 workload: shorter strips balance the
  // 152 SMs better than the two-row prologue of each strip costs)
  // 32 planes per CTA for the D3Q19 sweep: 2048 CTAs on 256^3
  const bool is2d = c->lattice == LBM_D2Q9;
  const long long rows = is2d ? c->ny : c->nz;
  long long strip = is2d ? 16 : 32;
  // A lattice that gives fewer CTAs than two waves at that strip leaves SMs
  // idle: take the shorter strip with the least modelled time, waves x (rows
  // per CTA + the sweep's prologue rows), with 5 (2D) or 2 (3D) resident
  // CTAs per SM.  The autotuner (lbm_tune) measures instead of modelling.
  int sms = 0;
  if (!c->multi && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) == cudaSuccess && sms > 0) {
    const long long tiles = is2d ? (c->nx + 127) / 128 : (long long)((c->nx + 31) / 32) * ((c->ny + 7) / 8);
    const long long slots = (long long)sms * (is2d ? 5 : 2);
    const long long prologue = is2d ? 4 : 3;
    auto ctas = [&](long long s) { return tiles * ((rows + s - 1) / s) * c->nbatch; };
    if (ctas(strip) < 2 * slots) {
      long long best = strip, best_cost = -1;
      for (long long s : {4LL, 8LL, 12LL, 16LL, 20LL, 24LL, 32LL}) {
        if (s > strip) break;
        const long long cost = ((ctas(s) + slots - 1) / slots) * (std::min(s, rows) + prologue);
        if (best_cost < 0 || cost < best_cost) best = s, best_cost = cost;
      }
      strip = best;
    }
  }
  if (strip > rows) strip = rows;
  return (int)std::max(1LL, strip);
}

StepArgs step_args(lbm_ctx* c, int from) {
  StepArgs a;
  a.f_in = c->f[from];
  a.f_out = c->f[1 - from];
  a.g_in = c->g[from];
  a.g_out = c->g[1 - from];
  a.phi0 = c->phi0;
  a.hist_in = c->hist[from];
  a.hist_out = c->hist[1 - from];
  a.p_out = c->p;
  a.mom = c->mom;
  a.consts = c->dconsts;
  a.flag = c->dflag;
  a.nx = c->nx;
  a.ny = c->ny;
  a.nz = c->nz;
  a.per_x = c->per[0];
  a.per_y = c->per[1];
  a.per_z = c->per[2];
  a.strip = c->strip;
  a.depth = c->depth;
  a.wait_polls = c->wait_polls;
  a.s_zero = 1;
  for (const auto& k : c->hconsts) a.s_zero &= k.rho1 == k.rho2 ? 1 : 0;
  a.nodes = c->nodes;
  a.g_half = c->g_half;
  a.q = c->q;
  return a;
}

long long inst_nodes(const lbm_ctx* c, int b) { return (long long)c->inx[b] * c->iny[b] * c->nz; }

void drop_graphs(lbm_ctx* c) {
  for (int i = 0; i < 2; ++i)
    if (c->graph[i]) {
      cudaGraphExecDestroy(c->graph[i]);
      c->graph[i] = nullptr;
    }
}

// Per-instance launch arguments (both starting buffers) and the work list of a
// multi-size context: items (instance, x0, ys) for every 128-column tile and
// strip of every instance, largest tiles first.
cudaError_t upload_multi(lbm_ctx* c) {
  const int nb = c->nbatch;
  std::vector<StepArgs> v(nb);
  for (int from = 0; from < 2; ++from) {
    for (int b = 0; b < nb; ++b) {
      StepArgs a = step_args(c, from);
      const long long o = c->ioff[b];
      a.f_in = c->f[from] + (size_t)c->q * o;
      a.f_out = c->f[1 - from] + (size_t)c->q * o;
      a.g_in = static_cast<const char*>(c->g[from]) + (size_t)c->q * o * c->g_elem;
      a.g_out = static_cast<char*>(c->g[1 - from]) + (size_t)c->q * o * c->g_elem;
      a.phi0 = c->phi0 + o;
      a.hist_in = c->hist[from] + (size_t)(1 + 2 * c->d) * o;
      a.hist_out = c->hist[1 - from] + (size_t)(1 + 2 * c->d) * o;
      a.p_out = c->p + o;
      a.consts = c->dconsts + b;
      a.nx = c->inx[b];
      a.ny = c->iny[b];
      a.nz = 1;
      a.strip = c->istrip[b];
      a.nodes = inst_nodes(c, b);
      v[b] = a;
    }
    cudaError_t e = cudaMemcpy(c->dargs[from], v.data(), sizeof(StepArgs) * nb, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
  }
  std::vector<int4> items;
  for (int b = 0; b < nb; ++b)
    for (int x0 = 0; x0 < c->inx[b]; x0 += 128)
      for (int ys = 0; ys < c->iny[b]; ys += c->istrip[b]) items.push_back(make_int4(b, x0, ys, 0));
  auto work = [&](const int4& w) {
    return (long long)std::min(128, c->inx[w.x] - w.y) * std::min(c->istrip[w.x], c->iny[w.x] - w.z);
  };
  std::stable_sort(items.begin(), items.end(), [&](const int4& a, const int4& b) { return work(a) > work(b); });
  if ((int)items.size() > c->items_cap) {
    dev_free(c, c->ditems);
    c->ditems = nullptr;
    c->items_cap = 0;
    cudaError_t e = dalloc(c, &c->ditems, sizeof(int4) * items.size());
    if (e != cudaSuccess) return e;
    c->items_cap = (int)items.size();
  }
  c->nitems = (int)items.size();
  drop_graphs(c);
  return cudaMemcpy(c->ditems, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice);
}

// One time step.  D3Q19 runs its moment pass first; `mid`, when given, is
// recorded between the moment pass and the fused kernel (D2Q9: before it).
cudaError_t launch_step(lbm_ctx* c, int from, bool observe, cudaStream_t s, cudaEvent_t mid = nullptr) {
  if (c->multi) {
    if (mid) cudaEventRecord(mid, s);
    return lbm::launch_d2q9_items(c->dargs[from], c->ditems, c->nitems, c->depth, c->g_half, 0, observe,
                                  c->per[0] && c->per[1], c->dqueue, s);
  }
  const StepArgs a = step_args(c, from);
  cudaError_t e = cudaSuccess;
  if (c->lattice == LBM_D2Q9) {
    if (mid) cudaEventRecord(mid, s);
    Range r("d2q9_step (fused stencils, collisions, streaming)");
    e = lbm::launch_d2q9_step(a, c->nbatch, observe, s);
  } else {
    Range r("3D step: moment pass + fused kernel");
    e = lbm::launch_d3q19_moments(a, c->nbatch, s);
    if (e != cudaSuccess) return e;
    if (mid) {
      e = cudaEventRecord(mid, s);
      if (e != cudaSuccess) return e;
    }
    // depth 1 selects the generic kernel; otherwise the pipelined one where its tensor maps exist
    const void* maps = (c->d3maps_ok && c->depth != 1) ? c->d3maps[from] : nullptr;
    e = lbm::launch_d3q19_step(a, c->nbatch, observe, s, maps);
  }
  if (e != cudaSuccess || !c->inout_mode) return e;
  return lbm::launch_inout(c->f[1 - from], c->g[1 - from], c->g_half, c->phi0, c->dconsts, c->inout_u,
                           c->inout_mode, c->inout_phi_in, c->inout_p_out, c->q, c->nx, c->ny, c->nz, c->nodes,
                           c->nbatch, s);
}

int ensure_graph(lbm_ctx* c, int from) {
  if (c->graph[from]) return LBM_OK;
  cudaStream_t cs = nullptr;
  LBM_CK(c, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t gr = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  int b = from;
  for (int i = 0; i < kGraphSteps && e == cudaSuccess; ++i) {
    e = launch_step(c, b, false, cs);
    b = 1 - b;
  }
  cudaError_t e2 = cudaStreamEndCapture(cs, &gr);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph[from], gr, 0);
  if (gr) cudaGraphDestroy(gr);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) return cuda_fail(c, e, "capture of the step graph");
  return LBM_OK;
}

// Captures the step graphs of both starting buffers ahead of use, so that the
// first lbm_step after a launch-shape change replays a graph instead of
// capturing one (capture and instantiation are host work of a few hundred
// microseconds during which the stream would otherwise sit idle).
int prepare_graphs(lbm_ctx* c) {
  if (c->stream == nullptr || c->profiling) return LBM_OK;
  for (int from = 0; from < 2; ++from)
    if (int s = ensure_graph(c, from)) return s;
  return LBM_OK;
}

int check_ready(lbm_ctx* c, bool need_state) {
  if (!c) return set_err(nullptr, LBM_EINVAL, "null context");
  if (c->failed) return LBM_ESTATE;   // c->err keeps the first failure
  if (need_state && !c->phase_set) return set_err(c, LBM_ESTATE, "state not initialised (call lbm_set_phase)");
  return LBM_OK;
}

int check_flag(lbm_ctx* c) {
  unsigned int flag = 0;
  LBM_CK(c, cudaMemcpyAsync(&flag, c->dflag, sizeof(flag), cudaMemcpyDeviceToHost, c->stream));
  LBM_CK(c, cudaStreamSynchronize(c->stream));
  if (flag) {
    LBM_CK(c, cudaMemsetAsync(c->dflag, 0, sizeof(unsigned int), c->stream));
    if (flag & 2u)
      return set_err(c, LBM_ETIMEOUT, "a bounded wait for an asynchronous tile load gave up; the step is incomplete");
    return set_err(c, LBM_EDIVERGED, "divergence: NaN or |u| > 0.5 at the last observed step");
  }
  return LBM_OK;
}

// Makes the context's device current for one entry point and gives the
// calling thread its own device back on return, so contexts on different
// devices can be driven from one thread.
struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(const lbm_ctx* c) {
    int cur = -1;
    if (c && cudaGetDevice(&cur) == cudaSuccess && cur != c->device && cudaSetDevice(c->device) == cudaSuccess)
      prev = cur;
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
  DeviceScope(const DeviceScope&) = delete;
  DeviceScope& operator=(const DeviceScope&) = delete;
};

void free_all(lbm_ctx* c) {
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  c->ev.clear();
  for (int i = 0; i < 2; ++i) {
    if (c->graph[i]) cudaGraphExecDestroy(c->graph[i]);
    dev_free(c, c->f[i]);
    dev_free(c, c->g[i]);
    dev_free(c, c->hist[i]);
  }
  dev_free(c, c->dargs[0]);
  dev_free(c, c->dargs[1]);
  dev_free(c, c->ditems);
  dev_free(c, c->dqueue);
  dev_free(c, c->phi0);
  dev_free(c, c->p);
  dev_free(c, c->mom);
  dev_free(c, c->inout_u);
  dev_free(c, c->dflag);
  dev_free(c, c->dpart);
  dev_free(c, c->dobs);
  dev_free(c, c->dconsts);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

// --- host-side geometry of the droplet diagnostics ---------------------------

double crossing_from_top(const std::vector<float>& v, double level) {
  for (int k = (int)v.size() - 2; k >= 0; --k)
    if (v[k] >= level && level > v[k + 1]) return k + (v[k] - level) / ((double)v[k] - v[k + 1]);
  return NAN;
}

double crossing_from_bottom(const std::vector<float>& v, double level) {
  for (int k = 0; k + 1 < (int)v.size(); ++k)
    if (v[k] >= level && level > v[k + 1]) return k + (v[k] - level) / ((double)v[k] - v[k + 1]);
  return NAN;
}

template <class F>
double bisect(F fn, double lo, double hi, double target) {
  double flo = fn(lo) - target;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    const double fm = fn(mid) - target;
    if ((fm > 0) == (flo > 0)) {
      lo = mid;
      flo = fm;
    } else {
      hi = mid;
    }
  }
  return 0.5 * (lo + hi);
}

// H / R0 of a 2D cap of contact angle t holding the area of a half disk R0.
double flat_ratio(double t) { return (1.0 - cos(t)) * sqrt((M_PI / 2.0) / (t - sin(t) * cos(t))); }

// Area of a circle (radius r, centre at distance k from the disk centre) outside the disk Rs.
double area_outside(double r, double Rs, double k) {
  const double a = (k * k - r * r + Rs * Rs) / (2.0 * k);
  const double h2 = std::max(Rs * Rs - a * a, 0.0);
  const double c1 = std::min(1.0, std::max(-1.0, (k * k + r * r - Rs * Rs) / (2.0 * k * r)));
  const double c2 = std::min(1.0, std::max(-1.0, (k * k - r * r + Rs * Rs) / (2.0 * k * Rs)));
  return M_PI * r * r - r * r * acos(c1) - Rs * Rs * acos(c2) + k * sqrt(h2);
}

double disk_hmax(double t, double Rs, double S0) {
  auto area = [&](double r) { return area_outside(r, Rs, sqrt(r * r + Rs * Rs - 2.0 * r * Rs * cos(t))); };
  const double r = bisect(area, 1e-6, 10.0 * (Rs + sqrt(S0)), S0);
  return r + sqrt(r * r + Rs * Rs - 2.0 * r * Rs * cos(t));
}

// launch one step, bracketed by an event pair when profiling
int timed_step(lbm_ctx* c, bool observe) {
  if (c->profiling) {
    while (c->ev.size() < 3 * (c->ev_used + 1)) {
      cudaEvent_t e;
      LBM_CK(c, cudaEventCreate(&e));
      c->ev.push_back(e);
    }
    LBM_CK(c, cudaEventRecord(c->ev[3 * c->ev_used], c->stream));
  }
  cudaError_t e = launch_step(c, c->cur, observe, c->stream, c->profiling ? c->ev[3 * c->ev_used + 1] : nullptr);
  if (e != cudaSuccess) return cuda_fail(c, e, "step kernel");
  if (c->profiling) {
    LBM_CK(c, cudaEventRecord(c->ev[3 * c->ev_used + 2], c->stream));
    ++c->ev_used;
  }
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_derive(lbm_lattice lattice, const lbm_params* p, lbm_derived* out) {
  if (!p || !out) return set_err(nullptr, LBM_EINVAL, "params and out must not be NULL");
  if (lattice != LBM_D2Q9 && lattice != LBM_D3Q19 && lattice != LBM_D3Q15)
    return set_err(nullptr, LBM_EINVAL, "unknown lattice");
  char why[128] = "";
  InstanceConsts k;
  if (derive(*p, lattice, k, why, out) != LBM_OK) return set_err(nullptr, LBM_EINVAL, "%s", why);
  return LBM_OK;
}

int lbm_default_params(lbm_params* p) {
  if (!p) return LBM_EINVAL;
  memset(p, 0, sizeof(*p));
  p->W = 4.0;
  p->M_deg = 0.1;
  p->M_cst = 0.0;
  p->theta_deg = 90.0;
  p->kappa = 0.0;
  p->sigma = 0.01;
  for (int i = 0; i < 3; ++i) {
    p->rho[i] = 1.0;
    p->mu[i] = 0.01;
  }
  p->d0 = 0.5;
  p->eta_hat = 0.1;
  p->s_free_ch = 1.0;
  p->s_free_ns = 1.0;
  return LBM_OK;
}

static int create_impl(lbm_lattice lattice, int nbatch, const int* nxs, const int* nys, int nz, int periodic_mask,
                       const lbm_params* params, int flags, bool multi, lbm_ctx** out, void* stream = nullptr,
                       lbm_alloc_fn alloc_fn = nullptr, lbm_free_fn free_fn = nullptr, void* alloc_user = nullptr) {
  if (!out) return set_err(nullptr, LBM_EINVAL, "out is NULL");
  *out = nullptr;
  if ((alloc_fn == nullptr) != (free_fn == nullptr))
    return set_err(nullptr, LBM_EINVAL, "give both device-memory callbacks or neither");
  if (flags & ~LBM_STORE_G_F16) return set_err(nullptr, LBM_EINVAL, "unknown flag");
  if (lattice != LBM_D2Q9 && lattice != LBM_D3Q19 && lattice != LBM_D3Q15)
    return set_err(nullptr, LBM_EINVAL, "unknown lattice");
  if (!params || nbatch < 1 || !nxs || !nys) return set_err(nullptr, LBM_EINVAL, "need nbatch >= 1 parameter sets");
  if (nbatch > 65535) return set_err(nullptr, LBM_EINVAL, "at most 65535 instances");
  const int g_half = (flags & LBM_STORE_G_F16) ? 1 : 0;
  const bool is3d = lattice != LBM_D2Q9;
  const int q = lattice == LBM_D3Q19 ? 19 : (lattice == LBM_D3Q15 ? 15 : 9);
  if (multi && is3d) return set_err(nullptr, LBM_EUNSUPPORTED, "instances of different sizes are built for D2Q9 only");
  if (!is3d && nz != 1) return set_err(nullptr, LBM_EINVAL, "D2Q9 needs nz = 1");
  const int per[3] = {(periodic_mask & LBM_PERIODIC_X) ? 1 : 0, (periodic_mask & LBM_PERIODIC_Y) ? 1 : 0,
                      (periodic_mask & LBM_PERIODIC_Z) ? 1 : 0};
  long long total = 0, max_nodes = 0;
  for (int b = 0; b < nbatch; ++b) {
    const int nx = nxs[b], ny = nys[b];
    if (nx < 1 || ny < 1 || nz < 1) return set_err(nullptr, LBM_EINVAL, "sizes must be positive");
    if (g_half && nx % 8 != 0) return set_err(nullptr, LBM_EINVAL, "FP16 population storage needs nx % 8 == 0");
    const int dims[3] = {nx, ny, nz};
    for (int a = 0; a < (is3d ? 3 : 2); ++a)
      if (!per[a] && dims[a] < 2) return set_err(nullptr, LBM_EINVAL, "a wall axis needs at least 2 nodes");
    const long long nodes = (long long)nx * ny * nz;
    // kernels index the planes of one instance with 32-bit offsets
    if (nodes * q >= (1LL << 31))
      return set_err(nullptr, LBM_EINVAL, "lattice too large for one instance");
    total += nodes;
    max_nodes = std::max(max_nodes, nodes);
    if (total > (1LL << 40)) return set_err(nullptr, LBM_EINVAL, "lattice too large");
  }
  const int nx = nxs[0], ny = nys[0];

  lbm_ctx* c = new (std::nothrow) lbm_ctx();
  if (!c) return set_err(nullptr, LBM_ENOMEM, "host allocation failed");
  c->lattice = lattice;
  c->multi = multi;
  c->nx = multi ? 0 : nx;
  c->ny = multi ? 0 : ny;
  c->nz = nz;
  c->nbatch = nbatch;
  c->q = q;
  c->d = is3d ? 3 : 2;
  for (int a = 0; a < 3; ++a) c->per[a] = per[a];
  c->nodes = multi ? 0 : (long long)nx * ny * nz;
  c->total = total;
  c->inx.assign(nxs, nxs + nbatch);
  c->iny.assign(nys, nys + nbatch);
  c->ioff.resize(nbatch);
  long long o = 0;
  for (int b = 0; b < nbatch; ++b) {
    c->ioff[b] = o;
    o += (long long)c->inx[b] * c->iny[b] * nz;
  }
  c->hconsts.resize(nbatch);
  for (int b = 0; b < nbatch; ++b) {
    char why[128] = "";
    if (derive(params[b], lattice, c->hconsts[b], why) != LBM_OK) {
      char msg[200];
      snprintf(msg, sizeof msg, "instance %d: %s", b, why);
      set_err(nullptr, LBM_EINVAL, "%s", msg);
      delete c;
      return LBM_EINVAL;
    }
  }
  if (cudaError_t e = cudaGetDevice(&c->device)) {   // the first device call: parameters are valid
    delete c;
    return cuda_fail(nullptr, e, "cudaGetDevice");
  }
  c->strip = default_strip(c);
  c->depth = is3d ? 2 : 1;
  c->g_half = g_half;
  c->g_elem = g_half ? sizeof(__half) : sizeof(float);
  c->istrip.resize(nbatch);
  for (int b = 0; b < nbatch; ++b) c->istrip[b] = std::max(1, std::min(16, c->iny[b]));
  const size_t pop = sizeof(float) * (size_t)c->q * total;
  const size_t his = sizeof(float) * (size_t)(1 + 2 * c->d) * total;
  const size_t fld = sizeof(float) * (size_t)total;
  c->alloc_fn = alloc_fn;
  c->free_fn = free_fn;
  c->alloc_user = alloc_user;
  cudaError_t e = cudaSuccess;
  if (stream) {
    c->stream = static_cast<cudaStream_t>(stream);
  } else {
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) c->own_stream = true;
  }
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = dalloc(c, &c->f[i], pop);
    if (e == cudaSuccess) e = dalloc(c, &c->g[i], pop / sizeof(float) * c->g_elem);
    if (e == cudaSuccess) e = dalloc(c, &c->hist[i], his);
  }
  if (e == cudaSuccess) e = dalloc(c, &c->phi0, fld);
  if (e == cudaSuccess) e = dalloc(c, &c->p, fld);
  if (e == cudaSuccess && is3d) e = dalloc(c, &c->mom, 3 * fld);
  if (e == cudaSuccess) e = dalloc(c, &c->dflag, sizeof(unsigned int));
  if (e == cudaSuccess) e = dalloc(c, &c->dpart, sizeof(double) * lbm::obs_partials_len(max_nodes));
  if (e == cudaSuccess) e = dalloc(c, &c->dobs, sizeof(double) * 8);
  if (e == cudaSuccess) e = dalloc(c, &c->dconsts, sizeof(InstanceConsts) * nbatch);
  if (e == cudaSuccess)
    e = cudaMemcpy(c->dconsts, c->hconsts.data(), sizeof(InstanceConsts) * nbatch, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(c->dflag, 0, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(c->p, 0, fld);
  if (e == cudaSuccess && multi) {
    e = dalloc(c, &c->dargs[0], sizeof(StepArgs) * nbatch);
    if (e == cudaSuccess) e = dalloc(c, &c->dargs[1], sizeof(StepArgs) * nbatch);
    if (e == cudaSuccess) e = dalloc(c, &c->dqueue, 2 * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(c->dqueue, 0, 2 * sizeof(unsigned int));
    if (e == cudaSuccess) e = upload_multi(c);
  }
  if (e == cudaSuccess && is3d && lbm::d3q19_maps_bytes() <= sizeof(c->d3maps[0])) {
    int r = 0;
    for (int i = 0; i < 2 && r == 0; ++i)
      r = lbm::build_d3q19_maps(c->g[i], g_half, c->mom, c->hist[i], nx, ny, nz, nbatch, q, c->d3maps[i]);
    if (r < 0) e = cudaErrorInvalidValue;   // the CUDA driver refused a tensor map
    c->d3maps_ok = r == 0;
  }
  if (e != cudaSuccess) {
    const int code = (e == cudaErrorMemoryAllocation) ? LBM_ENOMEM : LBM_ECUDA;
    set_err(nullptr, code, "device set-up failed: %s", cudaGetErrorString(e));
    free_all(c);
    delete c;
    return code;
  }
  *out = c;
  return LBM_OK;
}

int lbm_create_ex(lbm_lattice lattice, int nx, int ny, int nz, int periodic_mask, int nbatch,
                  const lbm_params* params, int flags, lbm_ctx** out) {
  if (nbatch < 1 || nbatch > 65535) {
    if (out) *out = nullptr;
    return set_err(nullptr, LBM_EINVAL, "need 1 <= nbatch <= 65535");
  }
  std::vector<int> nxs(nbatch, nx), nys(nbatch, ny);
  return create_impl(lattice, nbatch, nxs.data(), nys.data(), nz, periodic_mask, params, flags, false, out);
}

int lbm_create_alloc(lbm_lattice lattice, int nx, int ny, int nz, int periodic_mask, int nbatch,
                     const lbm_params* params, int flags, void* stream, lbm_alloc_fn alloc_fn, lbm_free_fn free_fn,
                     void* user, lbm_ctx** out) {
  if (nbatch < 1 || nbatch > 65535) {
    if (out) *out = nullptr;
    return set_err(nullptr, LBM_EINVAL, "need 1 <= nbatch <= 65535");
  }
  std::vector<int> nxs(nbatch, nx), nys(nbatch, ny);
  return create_impl(lattice, nbatch, nxs.data(), nys.data(), nz, periodic_mask, params, flags, false, out, stream,
                     alloc_fn, free_fn, user);
}

int lbm_create_multi(lbm_lattice lattice, int ninst, const int* nx, const int* ny, int periodic_mask,
                     const lbm_params* params, int flags, lbm_ctx** out) {
  if (ninst < 1 || ninst > 65535) {
    if (out) *out = nullptr;
    return set_err(nullptr, LBM_EINVAL, "need 1 <= ninst <= 65535");
  }
  return create_impl(lattice, ninst, nx, ny, 1, periodic_mask, params, flags, true, out);
}

int lbm_get_instance_shape(const lbm_ctx* c, int instance, int* nx, int* ny, int64_t* offset) {
  if (!c || instance < 0 || instance >= c->nbatch) return LBM_EINVAL;
  if (nx) *nx = c->inx[instance];
  if (ny) *ny = c->iny[instance];
  if (offset) *offset = c->ioff[instance];
  return LBM_OK;
}

int lbm_create_batch(lbm_lattice lattice, int nx, int ny, int nz, int periodic_mask, int nbatch,
                     const lbm_params* params, lbm_ctx** out) {
  return lbm_create_ex(lattice, nx, ny, nz, periodic_mask, nbatch, params, 0, out);
}

int lbm_create(lbm_lattice lattice, int nx, int ny, int nz, int periodic_mask, const lbm_params* p,
               lbm_ctx** out) {
  return lbm_create_batch(lattice, nx, ny, nz, periodic_mask, 1, p, out);
}

void lbm_destroy(lbm_ctx* c) {
  DeviceScope ds(c);
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
}

int lbm_set_stream(lbm_ctx* c, void* stream) {
  DeviceScope ds(c);
  if (!c) return set_err(nullptr, LBM_EINVAL, "null context");
  if (c->failed) return check_ready(c, false);
  LBM_CK(c, cudaStreamSynchronize(c->stream));
  if (c->own_stream) {
    cudaStreamDestroy(c->stream);
    c->own_stream = false;
  }
  c->stream = (cudaStream_t)stream;
  return LBM_OK;
}

int lbm_set_launch(lbm_ctx* c, int strip, int depth) {
  DeviceScope ds(c);
  if (int s = check_ready(c, false)) return s;
  if (strip < 1) return set_err(c, LBM_EINVAL, "strip must be >= 1");
  if (depth < 0 || depth > 3) return set_err(c, LBM_EINVAL, "depth must lie in 0..3 (0 keeps the current)");
  LBM_CK(c, cudaStreamSynchronize(c->stream));
  c->strip = strip;
  if (depth > 0) c->depth = depth;
  drop_graphs(c);
  if (c->multi) {
    for (int b = 0; b < c->nbatch; ++b) c->istrip[b] = std::min(strip, c->iny[b]);
    LBM_CK(c, upload_multi(c));
  }
  return c->phase_set ? prepare_graphs(c) : LBM_OK;
}

int lbm_set_wait_limit(lbm_ctx* c, int polls) {
  DeviceScope ds(c);
  if (int s = check_ready(c, false)) return s;
  LBM_CK(c, cudaStreamSynchronize(c->stream));
  c->wait_polls = polls < 0 ? lbm::kWaitPollsDefault : polls;
  drop_graphs(c);
  if (c->multi) LBM_CK(c, upload_multi(c));
  return LBM_OK;
}

// Autotuner: strip per size class by coordinate descent on the measured time
// of `trial` steps (after one untimed step), two passes over the classes.
// The evolving state is saved before and restored after, bitwise.
int lbm_tune(lbm_ctx* c, int trial, int* strips_out) {
  DeviceScope ds(c);
  Range range("lbm_tune");
  if (int s = check_ready(c, true)) return s;
  if (trial < 1) return set_err(c, LBM_EINVAL, "trial must be >= 1");
  LBM_CK(c, cudaStreamSynchronize(c->stream));
  const size_t pop = sizeof(float) * (size_t)c->q * c->total;
  const size_t gpop = pop / sizeof(float) * c->g_elem;
  const size_t his = sizeof(float) * (size_t)(1 + 2 * c->d) * c->total;
  void *sf = nullptr, *sg = nullptr, *sh = nullptr;
  cudaError_t e = dev_alloc(c, &sf, pop);
  if (e == cudaSuccess) e = dev_alloc(c, &sg, gpop);
  if (e == cudaSuccess) e = dev_alloc(c, &sh, his);
  const int cur0 = c->cur;
  if (e == cudaSuccess) e = cudaMemcpyAsync(sf, c->f[cur0], pop, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sg, c->g[cur0], gpop, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sh, c->hist[cur0], his, cudaMemcpyDeviceToDevice, c->stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // size classes: instances of equal (nx, ny)
  std::vector<std::vector<int>> classes;
  for (int b = 0; b < c->nbatch; ++b) {
    bool placed = false;
    for (auto& cl : classes)
      if (c->inx[cl[0]] == c->inx[b] && c->iny[cl[0]] == c->iny[b]) {
        cl.push_back(b);
        placed = true;
        break;
      }
    if (!placed) classes.push_back({b});
  }
  auto apply = [&](int cl, int strip) -> cudaError_t {
    if (c->multi) {
      for (int b : classes[cl]) c->istrip[b] = std::min(strip, c->iny[b]);
      return upload_multi(c);
    }
    c->strip = strip;
    drop_graphs(c);
    return cudaSuccess;
  };
  auto measure = [&](float& ms) -> cudaError_t {
    cudaError_t r = launch_step(c, c->cur, false, c->stream);
    c->cur = 1 - c->cur;
    if (r == cudaSuccess) r = cudaEventRecord(e0, c->stream);
    for (int i = 0; i < trial && r == cudaSuccess; ++i) {
      r = launch_step(c, c->cur, false, c->stream);
      c->cur = 1 - c->cur;
    }
    if (r == cudaSuccess) r = cudaEventRecord(e1, c->stream);
    if (r == cudaSuccess) r = cudaEventSynchronize(e1);
    if (r == cudaSuccess) r = cudaEventElapsedTime(&ms, e0, e1);
    return r;
  };
  // powers of two plus the steps between 12 and 24 rows: on GB300 the best D2Q9 strip of a 1024^2 x 5 batch is 18
  // (its CTA count is three full waves of 152 SMs x 5 CTAs), 1.8 % faster than 16
  static const int cand[] = {4, 8, 12, 16, 18, 20, 24, 32, 48, 64};
  constexpr int ncand = (int)(sizeof(cand) / sizeof(cand[0]));
  for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
    for (int cl = 0; cl < (int)classes.size() && e == cudaSuccess; ++cl) {
      const int rows = c->multi ? c->iny[classes[cl][0]] : (c->lattice == LBM_D2Q9 ? c->ny : c->nz);
      int best = c->multi ? c->istrip[classes[cl][0]] : c->strip;
      float best_ms = 1e30f;
      for (int sidx = 0; sidx < ncand && e == cudaSuccess; ++sidx) {
        const int strip = cand[sidx];
        if (strip > rows && sidx > 0 && cand[sidx - 1] >= rows) break;   // larger strips change nothing
        float ms = 0.f;
        e = apply(cl, strip);
        if (e == cudaSuccess) e = measure(ms);
        if (e == cudaSuccess && ms < best_ms) {
          best_ms = ms;
          best = strip;
        }
      }
      if (e == cudaSuccess) e = apply(cl, best);
      if (!c->multi) break;   // one strip for the whole context
    }
  }
  // restore the state the tuner found
  c->cur = cur0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->f[cur0], sf, pop, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->g[cur0], sg, gpop, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->hist[cur0], sh, his, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  dev_free(c, sf);
  dev_free(c, sg);
  dev_free(c, sh);
  if (e != cudaSuccess) return cuda_fail(c, e, "autotuner");
  if (strips_out)
    for (int b = 0; b < c->nbatch; ++b) strips_out[b] = c->multi ? c->istrip[b] : c->strip;
  return prepare_graphs(c);
}

static int set_solid_impl(lbm_ctx* c, const float* src, cudaMemcpyKind kind) {
  DeviceScope ds(c);
  if (int s = check_ready(c, false)) return s;
  if (!src) return set_err(c, LBM_EINVAL, "phi0 is NULL");
  LBM_CK(c, cudaMemcpyAsync(c->phi0, src, sizeof(float) * c->total, kind, c->stream));
  if (kind == cudaMemcpyHostToDevice) LBM_CK(c, cudaStreamSynchronize(c->stream));
  c->solid_set = true;
  return LBM_OK;
}

int lbm_set_solid(lbm_ctx* c, const float* phi0_host) { return set_solid_impl(c, phi0_host, cudaMemcpyHostToDevice); }
int lbm_set_solid_device(lbm_ctx* c, const float* phi0_dev) {
  DeviceScope ds(c);
  return set_solid_impl(c, phi0_dev, cudaMemcpyDeviceToDevice);
}

static int set_phase_impl(lbm_ctx* c, const float* src, cudaMemcpyKind kind) {
  DeviceScope ds(c);
  if (int s = check_ready(c, false)) return s;
  if (!src) return set_err(c, LBM_EINVAL, "phi1 is NULL");
  if (!c->solid_set) return set_err(c, LBM_ESTATE, "call lbm_set_solid before lbm_set_phase");
  const int nh = 1 + 2 * c->d;
  // stage phi1 in plane 0 of the spare history buffer, then initialise the current one
  float* stage = c->hist[1 - c->cur];
  cudaError_t e = cudaSuccess;
  if (c->multi) {
    for (int b = 0; b < c->nbatch && e == cudaSuccess; ++b) {
      const long long o = c->ioff[b];
      e = cudaMemcpyAsync(stage + nh * o, src + o, sizeof(float) * inst_nodes(c, b), kind, c->stream);
      if (e == cudaSuccess)
        e = lbm::launch_d2q9_init(c->phi0 + o, stage + nh * o, c->f[c->cur] + c->q * o,
                                  static_cast<char*>(c->g[c->cur]) + c->q * o * c->g_elem, c->g_half,
                                  c->hist[c->cur] + nh * o, c->dconsts + b, c->inx[b], c->iny[b], c->per[0],
                                  c->per[1], 1, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
    LBM_CK(c, cudaMemsetAsync(c->p, 0, sizeof(float) * c->total, c->stream));
    if (kind == cudaMemcpyHostToDevice) LBM_CK(c, cudaStreamSynchronize(c->stream));
    c->phase_set = true;
    c->step = 0;
    return LBM_OK;
  }
  const size_t row = sizeof(float) * c->nodes;
  LBM_CK(c, cudaMemcpy2DAsync(stage, row * nh, src, row, row, c->nbatch, kind, c->stream));
  if (c->lattice == LBM_D2Q9)
    e = lbm::launch_d2q9_init(c->phi0, stage, c->f[c->cur], c->g[c->cur], c->g_half, c->hist[c->cur], c->dconsts,
                              c->nx,
                              c->ny, c->per[0], c->per[1], c->nbatch, c->stream);
  else
    e = lbm::launch_d3q19_init(c->phi0, stage, c->f[c->cur], c->g[c->cur], c->g_half, c->hist[c->cur],
                               c->dconsts, c->nx,
                               c->ny, c->nz, c->per[0], c->per[1], c->per[2], c->nbatch, c->q, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
  LBM_CK(c, cudaMemsetAsync(c->p, 0, sizeof(float) * c->total, c->stream));
  if (kind == cudaMemcpyHostToDevice) LBM_CK(c, cudaStreamSynchronize(c->stream));
  c->phase_set = true;
  c->step = 0;
  return LBM_OK;
}

int lbm_set_phase(lbm_ctx* c, const float* phi1_host) { return set_phase_impl(c, phi1_host, cudaMemcpyHostToDevice); }
int lbm_set_phase_device(lbm_ctx* c, const float* phi1_dev) {
  DeviceScope ds(c);
  return set_phase_impl(c, phi1_dev, cudaMemcpyDeviceToDevice);
}

int lbm_set_profiling(lbm_ctx* c, int enable) {
  DeviceScope ds(c);
  if (int s = check_ready(c, false)) return s;
  c->profiling = enable != 0;
  c->ev_used = 0;
  return LBM_OK;
}

int lbm_kernel_time_split(lbm_ctx* c, double* part_ms, int64_t* steps) {
  DeviceScope ds(c);
  if (int s = check_ready(c, false)) return s;
  LBM_CK(c, cudaStreamSynchronize(c->stream));
  double t0 = 0.0, t1 = 0.0;
  for (size_t k = 0; k < c->ev_used; ++k) {
    float a = 0.f, b = 0.f;
    LBM_CK(c, cudaEventElapsedTime(&a, c->ev[3 * k], c->ev[3 * k + 1]));
    LBM_CK(c, cudaEventElapsedTime(&b, c->ev[3 * k + 1], c->ev[3 * k + 2]));
    t0 += a;
    t1 += b;
  }
  if (part_ms) {
    part_ms[0] = t0;
    part_ms[1] = t1;
  }
  if (steps) *steps = (int64_t)c->ev_used;
  c->ev_used = 0;
  return LBM_OK;
}

int lbm_kernel_time(lbm_ctx* c, double* total_ms, int64_t* launches) {
  DeviceScope ds(c);
  double part[2] = {0.0, 0.0};
  int64_t steps = 0;
  if (int s = lbm_kernel_time_split(c, part, &steps)) return s;
  if (total_ms) *total_ms = part[0] + part[1];
  if (launches) *launches = steps;
  return LBM_OK;
}

int lbm_set_inout(lbm_ctx* c, int mode, const float* u_in, double phi_in, double p_out) {
  DeviceScope ds(c);
  if (!c) return set_err(nullptr, LBM_EINVAL, "null context");
  if (c->failed) return LBM_ESTATE;
  if (mode < 0 || mode > 3) return set_err(c, LBM_EINVAL, "mode must be 0..3");
  if (c->multi) return set_err(c, LBM_EUNSUPPORTED, "inlet / outlet columns need a single-size context");
  if (mode && c->per[0]) return set_err(c, LBM_EINVAL, "inlet / outlet columns need a non-periodic x axis");
  if (mode && c->nx < 4) return set_err(c, LBM_EINVAL, "inlet / outlet columns need nx >= 4");
  if ((mode & 1) && !u_in) return set_err(c, LBM_EINVAL, "a velocity inlet needs its profile");
  if (!std::isfinite(phi_in) || phi_in > 1.0 || !std::isfinite(p_out))
    return set_err(c, LBM_EINVAL, "phi_in must be <= 1 (negative: extrapolated) and p_out finite");
  const size_t cols = (size_t)c->ny * c->nz;
  if (mode & 1) {
    for (size_t i = 0; i < cols * c->d; ++i)
      if (!std::isfinite(u_in[i]) || std::fabs(u_in[i]) > 0.5f)
        return set_err(c, LBM_EINVAL, "inlet velocity must be finite and below 0.5 in magnitude");
    if (!c->inout_u) LBM_CK(c, dalloc(c, &c->inout_u, sizeof(float) * cols * c->d));
    LBM_CK(c, cudaMemcpyAsync(c->inout_u, u_in, sizeof(float) * cols * c->d, cudaMemcpyHostToDevice, c->stream));
    LBM_CK(c, cudaStreamSynchronize(c->stream));
  }
  c->inout_mode = mode;
  c->inout_phi_in = phi_in < 0 ? -1.f : (float)phi_in;
  c->inout_p_out = (float)p_out;
  drop_graphs(c);                  // recaptured with (or without) the boundary launch
  return LBM_OK;
}

int lbm_step(lbm_ctx* c, int n) {
  DeviceScope ds(c);
  Range range("lbm_step");
  if (int s = check_ready(c, true)) return s;
  if (n < 0) return set_err(c, LBM_EINVAL, "n must be >= 0");
  const bool graphs = c->stream != nullptr && !c->profiling;
  while (n > 0) {
    if (n > kGraphSteps && graphs) {
      if (int s = ensure_graph(c, c->cur)) return s;
      LBM_CK(c, cudaGraphLaunch(c->graph[c->cur], c->stream));
      n -= kGraphSteps;
      c->step += kGraphSteps;
      continue;
    }
    const bool observe = (n == 1);
    if (int s = timed_step(c, observe)) return s;
    c->cur = 1 - c->cur;
    c->step += 1;
    --n;
  }
  return LBM_OK;
}

int lbm_sync(lbm_ctx* c) {
  DeviceScope ds(c);
  if (int s = check_ready(c, false)) return s;
  LBM_CK(c, cudaStreamSynchronize(c->stream));
  return check_flag(c);
}

int lbm_get_fields(lbm_ctx* c, float* phi1, float* u, float* p) {
  DeviceScope ds(c);
  Range range("lbm_get_fields");
  if (int s = check_ready(c, true)) return s;
  const int nh = 1 + 2 * c->d;
  const float* h = c->hist[c->cur];
  if (c->multi) {
    for (int b = 0; b < c->nbatch; ++b) {
      const long long o = c->ioff[b], n = inst_nodes(c, b);
      if (phi1)
        LBM_CK(c, cudaMemcpyAsync(phi1 + o, h + nh * o, sizeof(float) * n, cudaMemcpyDeviceToHost, c->stream));
      if (u)
        LBM_CK(c, cudaMemcpyAsync(u + c->d * o, h + nh * o + n, sizeof(float) * c->d * n, cudaMemcpyDeviceToHost,
                                  c->stream));
    }
    if (p) LBM_CK(c, cudaMemcpyAsync(p, c->p, sizeof(float) * c->total, cudaMemcpyDeviceToHost, c->stream));
    LBM_CK(c, cudaStreamSynchronize(c->stream));
    return check_flag(c);
  }
  const size_t row = sizeof(float) * c->nodes;
  if (phi1) LBM_CK(c, cudaMemcpy2DAsync(phi1, row, h, row * nh, row, c->nbatch, cudaMemcpyDeviceToHost, c->stream));
  if (u)
    LBM_CK(c, cudaMemcpy2DAsync(u, row * c->d, h + c->nodes, row * nh, row * c->d, c->nbatch,
                                cudaMemcpyDeviceToHost, c->stream));
  if (p) LBM_CK(c, cudaMemcpyAsync(p, c->p, row * c->nbatch, cudaMemcpyDeviceToHost, c->stream));
  LBM_CK(c, cudaStreamSynchronize(c->stream));
  return check_flag(c);
}

int lbm_get_populations(lbm_ctx* c, float* f, float* g) {
  DeviceScope ds(c);
  if (int s = check_ready(c, true)) return s;
  const size_t n = (size_t)c->q * c->total;
  if (f) LBM_CK(c, cudaMemcpyAsync(f, c->f[c->cur], sizeof(float) * n, cudaMemcpyDeviceToHost, c->stream));
  std::vector<__half> h;
  if (g && c->g_half) {
    h.resize(n);
    LBM_CK(c, cudaMemcpyAsync(h.data(), c->g[c->cur], sizeof(__half) * n, cudaMemcpyDeviceToHost, c->stream));
  } else if (g) {
    LBM_CK(c, cudaMemcpyAsync(g, c->g[c->cur], sizeof(float) * n, cudaMemcpyDeviceToHost, c->stream));
  }
  LBM_CK(c, cudaStreamSynchronize(c->stream));
  if (g && c->g_half) {
    // unscale per instance (every instance uses the same power-of-two scale)
    const float inv = c->hconsts[0].gsci;
    for (size_t i = 0; i < n; ++i) g[i] = __half2float(h[i]) * inv;
  }
  return LBM_OK;
}

static size_t state_bytes(const lbm_ctx* c) {
  const size_t n = (size_t)c->q * c->total;
  const size_t his = sizeof(float) * (size_t)(1 + 2 * c->d) * c->total;
  return sizeof(StateHeader) + sizeof(float) * n + c->g_elem * n + his;
}

int lbm_get_state(lbm_ctx* c, void* buf, size_t* bytes) {
  DeviceScope ds(c);
  if (int s = check_ready(c, true)) return s;
  if (!bytes) return set_err(c, LBM_EINVAL, "bytes is NULL");
  const size_t need = state_bytes(c);
  if (!buf) {
    *bytes = need;
    return LBM_OK;
  }
  if (*bytes < need) return set_err(c, LBM_EINVAL, "state buffer too small");
  StateHeader hd;
  memset(&hd, 0, sizeof hd);
  hd.magic = kStateMagic;
  hd.lattice = c->lattice;
  hd.nx = c->nx;
  hd.ny = c->ny;
  hd.nz = c->nz;
  hd.nbatch = c->nbatch;
  hd.q = c->q;
  hd.d = c->d;
  hd.step = c->step;
  hd.nodes = c->total;
  hd.pad[0] = c->g_half;   // storage of g: 0 float32, 1 FP16 scaled
  char* o = static_cast<char*>(buf);
  memcpy(o, &hd, sizeof hd);
  o += sizeof hd;
  const size_t pop = sizeof(float) * (size_t)c->q * c->total;
  const size_t gpop = pop / sizeof(float) * c->g_elem;
  const size_t his = sizeof(float) * (size_t)(1 + 2 * c->d) * c->total;
  LBM_CK(c, cudaMemcpyAsync(o, c->f[c->cur], pop, cudaMemcpyDeviceToHost, c->stream));
  LBM_CK(c, cudaMemcpyAsync(o + pop, c->g[c->cur], gpop, cudaMemcpyDeviceToHost, c->stream));
  LBM_CK(c, cudaMemcpyAsync(o + pop + gpop, c->hist[c->cur], his, cudaMemcpyDeviceToHost, c->stream));
  LBM_CK(c, cudaStreamSynchronize(c->stream));
  *bytes = need;
  return LBM_OK;
}

int lbm_set_state(lbm_ctx* c, const void* buf, size_t bytes) {
  DeviceScope ds(c);
  if (int s = check_ready(c, false)) return s;
  if (!buf || bytes < sizeof(StateHeader)) return set_err(c, LBM_EINVAL, "state image too small");
  StateHeader hd;
  memcpy(&hd, buf, sizeof hd);
  if (hd.magic != kStateMagic || hd.lattice != c->lattice || hd.nx != c->nx || hd.ny != c->ny ||
      hd.nz != c->nz || hd.nbatch != c->nbatch || hd.q != c->q || hd.d != c->d || hd.pad[0] != c->g_half ||
      hd.nodes != c->total ||
      bytes != state_bytes(c))
    return set_err(c, LBM_EINVAL, "state image does not match this context");
  if (!c->solid_set) return set_err(c, LBM_ESTATE, "call lbm_set_solid before lbm_set_state");
  const char* o = static_cast<const char*>(buf) + sizeof hd;
  const size_t pop = sizeof(float) * (size_t)c->q * c->total;
  const size_t gpop = pop / sizeof(float) * c->g_elem;
  const size_t his = sizeof(float) * (size_t)(1 + 2 * c->d) * c->total;
  LBM_CK(c, cudaMemcpyAsync(c->f[c->cur], o, pop, cudaMemcpyHostToDevice, c->stream));
  LBM_CK(c, cudaMemcpyAsync(c->g[c->cur], o + pop, gpop, cudaMemcpyHostToDevice, c->stream));
  LBM_CK(c, cudaMemcpyAsync(c->hist[c->cur], o + pop + gpop, his, cudaMemcpyHostToDevice, c->stream));
  LBM_CK(c, cudaStreamSynchronize(c->stream));
  c->step = hd.step;
  c->phase_set = true;
  return LBM_OK;
}

int lbm_observables(lbm_ctx* c, int instance, lbm_obs* out) {
  DeviceScope ds(c);
  Range range("lbm_observables");
  if (int s = check_ready(c, true)) return s;
  if (!out || instance < 0 || instance >= c->nbatch) return set_err(c, LBM_EINVAL, "bad instance or output");
  const int nh = 1 + 2 * c->d;
  const long long o = c->ioff[instance], n = inst_nodes(c, instance);
  const float* h = c->hist[c->cur] + (size_t)nh * o;
  cudaError_t e = lbm::launch_observables(c->phi0 + o, h, h + n, c->d, c->p + o, n, c->dpart, c->dobs,
                                          c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "observables kernel");
  double r[8];
  LBM_CK(c, cudaMemcpyAsync(r, c->dobs, sizeof r, cudaMemcpyDeviceToHost, c->stream));
  LBM_CK(c, cudaStreamSynchronize(c->stream));
  out->mass1 = r[0];
  out->mass0 = r[1];
  out->umax = r[2];
  out->n_in = (int64_t)r[4];
  out->n_out = (int64_t)r[6];
  out->p_in = r[4] > 0 ? r[3] / r[4] : NAN;
  out->p_out = r[6] > 0 ? r[5] / r[6] : NAN;
  out->dp = out->p_in - out->p_out;
  out->step = c->step;
  if (r[7] > 0) return set_err(c, LBM_EDIVERGED, "non-finite values in the fields");
  return check_flag(c);
}

int lbm_phase_flux(lbm_ctx* c, int instance, int axis, lbm_flux* out) {
  DeviceScope ds(c);
  Range range("lbm_phase_flux");
  if (int s = check_ready(c, true)) return s;
  if (!out || instance < 0 || instance >= c->nbatch || axis < 0 || axis >= c->d)
    return set_err(c, LBM_EINVAL, "bad instance, axis or output");
  const int nh = 1 + 2 * c->d;
  const long long o = c->ioff[instance], n = inst_nodes(c, instance);
  const float* h = c->hist[c->cur] + (size_t)nh * o;
  cudaError_t e = lbm::launch_phase_flux(c->phi0 + o, h, h + (size_t)(1 + axis) * n, n, c->dpart, c->dobs, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "phase flux kernel");
  double r[8];
  LBM_CK(c, cudaMemcpyAsync(r, c->dobs, sizeof r, cudaMemcpyDeviceToHost, c->stream));
  LBM_CK(c, cudaStreamSynchronize(c->stream));
  out->q1 = r[0];
  out->q2 = r[1];
  out->q = r[3];
  out->n_pore = (int64_t)r[4];
  const double fl = r[5] + r[6];
  out->s1 = fl != 0.0 ? r[5] / fl : NAN;
  out->s2 = fl != 0.0 ? r[6] / fl : NAN;
  if (r[7] > 0) return set_err(c, LBM_EDIVERGED, "non-finite values in the fields");
  return check_flag(c);
}

int lbm_contact_angle(lbm_ctx* c, int instance, int mode, int column, double y_c, double disk_radius,
                      double* theta_deg, double* height) {
  DeviceScope ds(c);
  if (int s = check_ready(c, true)) return s;
  if (c->lattice != LBM_D2Q9) return set_err(c, LBM_EUNSUPPORTED, "contact angle is measured on 2D lattices");
  if (instance < 0 || instance >= c->nbatch || column < 0 || column >= c->inx[instance] || (mode != 0 && mode != 1))
    return set_err(c, LBM_EINVAL, "bad instance, column or mode");
  if (mode == 1 && !(disk_radius > 0)) return set_err(c, LBM_EINVAL, "disk radius must be > 0");
  lbm_obs ob;
  if (int s = lbm_observables(c, instance, &ob)) return s;
  const int nh = 1 + 2 * c->d;
  const int inx = c->inx[instance], iny = c->iny[instance];
  std::vector<float> col1(iny), col0(iny);
  const float* h = c->hist[c->cur] + (size_t)nh * c->ioff[instance] + column;
  const float* s0 = c->phi0 + c->ioff[instance] + column;
  LBM_CK(c, cudaMemcpy2DAsync(col1.data(), sizeof(float), h, sizeof(float) * inx, sizeof(float), iny,
                              cudaMemcpyDeviceToHost, c->stream));
  LBM_CK(c, cudaMemcpy2DAsync(col0.data(), sizeof(float), s0, sizeof(float) * inx, sizeof(float), iny,
                              cudaMemcpyDeviceToHost, c->stream));
  LBM_CK(c, cudaStreamSynchronize(c->stream));
  const double ytop = crossing_from_top(col1, 0.5);
  double H, th;
  if (mode == 0) {
    const double ywall = crossing_from_bottom(col0, 0.5);
    H = ytop - ywall;
    const double R0 = sqrt(2.0 * ob.mass1 / M_PI);
    th = bisect(flat_ratio, 1e-6, M_PI - 1e-6, H / R0);
  } else {
    H = ytop - y_c;
    const double S0 = ob.mass1;
    th = bisect([&](double t) { return disk_hmax(t, disk_radius, S0); }, 1e-3, M_PI - 1e-3, H);
  }
  if (theta_deg) *theta_deg = th * 180.0 / M_PI;
  if (height) *height = H;
  if (!isfinite(H)) return set_err(c, LBM_EINVAL, "no phi1 = 1/2 crossing on that column");
  return LBM_OK;
}

int lbm_get_shape(const lbm_ctx* c, int* nx, int* ny, int* nz, int* nbatch, int* q) {
  if (!c) return LBM_EINVAL;
  if (nx) *nx = c->nx;
  if (ny) *ny = c->ny;
  if (nz) *nz = c->nz;
  if (nbatch) *nbatch = c->nbatch;
  if (q) *q = c->q;
  return LBM_OK;
}

const char* lbm_strerror(int s) {
  switch (s) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "out of memory";
    case LBM_ECUDA: return "CUDA error";
    case LBM_EDIVERGED: return "simulation diverged";
    case LBM_ETIMEOUT: return "device wait timed out";
    case LBM_ESTATE: return "invalid context state";
    case LBM_EUNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err : g_last_error; }

}  // extern "C"
