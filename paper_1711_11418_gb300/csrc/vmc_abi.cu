// C ABI of the library (include/vmc.h): context, validation, memory, and the
// orchestration of the kernels in vmc_walker.cu and vmc_sr.cu.
#include "../../include/vmc.h"
#include "vmc_common.cuh"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

namespace {

struct SysHost {
  int Ns = 0, Ne = 0, N = 0, ldm = 0, Np = 0, n_g = 0, n_v = 0, n_f = 0, ldO = 0;
  int W = 0, max_samples = 0;
  int rows = 0;              // stored sample rows (W * n_samples or set_samples rows)
  int n_samples = 0;         // samples per walker of the stored rows
  bool dirty = true;         // inverses must be rebuilt before sampling
  double p_exchange = 0.0;
  SysDev dev{};              // host copy of the device descriptor
  SrWork sr{};
  bool sr_alloc = false;
  bool S_alloc = false;
  void *tc_hi = nullptr, *tc_lo = nullptr;   // split-BF16 operands (mixed form)
  int *tc_status = nullptr;
  int2 *tc_tiles = nullptr;                   // tile order of the S GEMM
  int s_kernel = VMC_S_KERNEL_NONE;           // kernel of the last dense S~ build
  std::vector<signed char> lsite;             // local_site mask (empty = none)
};

}  // namespace

struct vmc_ctx {
  int n_sys = 0;
  int precision = 0;
  uint64_t seed = 0;
  cudaStream_t st = nullptr;
  std::vector<SysHost> sys;
  std::vector<void *> allocs;
  SysDev *d_sys = nullptr;
  int2 *d_work = nullptr;
  int n_work = 0;
  int *d_work_ctr = nullptr;
  size_t smem_sample = 0, smem_init = 0;
  int grid_sample = 0;
  long long n_launch = 0;
  double *d_scalar = nullptr;
  int recompute_every = 0;
  int delay_k = 0;            // as set by the caller (0/1 = immediate)
  int spec_b = 1;             // proposals formed together by the sweep
  bool rebuild_pending = false;  // the last sweep launch's periodic rebuild is still to run
  unsigned char *pin = nullptr;   // pinned staging for vmc_sr_step_all's results (per system)
  // vmc_sr_step_all: systems run on a small pool of streams forked from st
  static constexpr int NPOOL = 8;
  cudaStream_t pool[NPOOL] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[NPOOL] = {};
  size_t smem_cap = 0;        // dynamic shared-memory limit set on the sweep kernels
  size_t smem_proj = 0;       // projected sweep kernel (vmc_set_projection)
  int grid_proj = 0;
  void *corr_buf = nullptr;   // vmc_measure_corr scratch (grown on demand)
  size_t corr_bytes = 0;
  void *lz_buf = nullptr;     // vmc_lanczos_moments scratch (grown on demand)
  size_t lz_bytes = 0;
  // timing (CUDA events on st): 0 sweep, 1 init, 2 SR step, 3 S GEMM
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[4];
  double ms[4] = {0, 0, 0, 0};
  long long cnt[4] = {0, 0, 0, 0};
};

namespace {

void ctx_free(vmc_ctx *c) {
  if (!c) return;
  for (SysHost &s : c->sys) {
    vmc_sr_release(s.sr);
    vmc_sr_ir_release(s.sr);
  }
  if (c->pin) cudaFreeHost(c->pin);
  c->pin = nullptr;
  for (int k = 0; k < vmc_ctx::NPOOL; ++k) {
    if (c->pool[k]) cudaStreamDestroy(c->pool[k]);
    if (c->join_ev[k]) cudaEventDestroy(c->join_ev[k]);
    c->pool[k] = nullptr;
    c->join_ev[k] = nullptr;
  }
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  c->fork_ev = nullptr;
  if (c->corr_buf) cudaFree(c->corr_buf);
  c->corr_buf = nullptr;
  c->corr_bytes = 0;
  if (c->lz_buf) cudaFree(c->lz_buf);
  c->lz_buf = nullptr;
  c->lz_bytes = 0;
  for (void *p : c->allocs) cudaFree(p);
  c->allocs.clear();
}

template <typename P>
int dalloc(vmc_ctx *c, P **out, size_t bytes) {
  void *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return VMC_ENOMEM;
  }
  c->allocs.push_back(p);
  *out = (P *)p;
  return VMC_OK;
}

template <typename P>
int dupload(vmc_ctx *c, P **out, const P *src, size_t count) {
  int e = dalloc(c, out, sizeof(P) * count);
  if (e) return e;
  if (count && src) {
    if (cudaMemcpyAsync(*out, src, sizeof(P) * count, cudaMemcpyHostToDevice, c->st) != cudaSuccess)
      return VMC_ECUDA;
  } else if (count) {
    if (cudaMemsetAsync(*out, 0, sizeof(P) * count, c->st) != cudaSuccess) return VMC_ECUDA;
  }
  return VMC_OK;
}

#define CK(x)                       \
  do {                              \
    int _e = (x);                   \
    if (_e != VMC_OK) return _e;    \
  } while (0)
#define CKC(x)                                   \
  do {                                           \
    if ((x) != cudaSuccess) return VMC_ECUDA;    \
  } while (0)

// splitmix64: seeded initial placements (not part of the Markov chain).
uint64_t splitmix(uint64_t &s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Seeded placement of N up and N down electrons (label order).  Under
// local_spin every site holds at most one electron; with a local_site mask
// each marked site gets exactly one electron (a shuffled half up, within
// what the itinerant sites can take) and the rest go to unmarked sites.
void random_placement(int Ns, int Ne, bool local_spin, const signed char *lsite, uint64_t &state,
                      int32_t *ele) {
  const int N = Ne / 2;
  std::vector<int> perm(Ns);
  auto shuffle = [&]() {
    for (int i = 0; i < Ns; ++i) perm[i] = i;
    for (int i = Ns - 1; i > 0; --i) {
      const int j = (int)(splitmix(state) % (uint64_t)(i + 1));
      std::swap(perm[i], perm[j]);
    }
  };
  shuffle();
  if (local_spin) {
    for (int k = 0; k < Ne; ++k) ele[k] = perm[k];
    return;
  }
  if (lsite) {
    std::vector<int> loc, itin;
    for (int q = 0; q < Ns; ++q) (lsite[perm[q]] ? loc : itin).push_back(perm[q]);
    const int nl = (int)loc.size(), ni = (int)itin.size();
    // up electrons on marked sites: k with k <= N, nl - k <= N, N - k <= ni,
    // N - (nl - k) <= ni; the one nearest nl / 2 (validated at create)
    int k = nl / 2;
    const int lo = std::max(std::max(0, nl - N), std::max(N - ni, 0));
    const int hi = std::min(std::min(nl, N), ni + nl - N);
    k = std::min(std::max(k, lo), hi);
    int u = 0, d = N;
    for (int q = 0; q < nl; ++q) ele[q < k ? u++ : d++] = loc[q];
    for (int q = 0; u < N; ++q) ele[u++] = itin[q];
    shuffle();
    std::vector<int> it2;
    for (int q = 0; q < Ns; ++q)
      if (!lsite[perm[q]]) it2.push_back(perm[q]);
    for (int q = 0; d < Ne; ++q) ele[d++] = it2[q];
    return;
  }
  for (int k = 0; k < N; ++k) ele[k] = perm[k];
  shuffle();
  for (int k = 0; k < N; ++k) ele[N + k] = perm[k];
}

int validate_configs(const SysHost &s, bool local_spin, const int32_t *ele, int W) {
  std::vector<int> occ(2 * s.Ns);
  for (int w = 0; w < W; ++w) {
    std::fill(occ.begin(), occ.end(), 0);
    for (int k = 0; k < s.Ne; ++k) {
      const int site = ele[(size_t)w * s.Ne + k];
      if (site < 0 || site >= s.Ns) return VMC_EINVAL;
      const int sp = k >= s.N;
      if (occ[sp * s.Ns + site]) return VMC_EINVAL;
      occ[sp * s.Ns + site] = 1;
    }
    if (local_spin)
      for (int i = 0; i < s.Ns; ++i)
        if (occ[i] && occ[s.Ns + i]) return VMC_EINVAL;
    if (!s.lsite.empty())
      for (int i = 0; i < s.Ns; ++i)
        if (s.lsite[i] && occ[i] + occ[s.Ns + i] != 1) return VMC_EINVAL;
  }
  return VMC_OK;
}

int validate_system(const vmc_model *m, int32_t Ne, const vmc_layout *l, const double *params) {
  if (!m || !l || !params) return VMC_EINVAL;
  const int Ns = m->Ns;
  if (Ns < 2 || Ns > 4096) return VMC_EINVAL;
  if (Ne < 2 || Ne % 2 || Ne / 2 > VMC_MAX_N || Ne / 2 > Ns) return VMC_EINVAL;
  if (m->local_spin && Ne != Ns) return VMC_EINVAL;
  if (m->local_site) {
    // each marked site takes one electron: some split k (up) + nl - k (down)
    // of the marked sites must leave N - k up and N - nl + k down electrons
    // for the ni unmarked sites
    int nl = 0;
    for (int i = 0; i < Ns; ++i) {
      if (m->local_site[i] != 0 && m->local_site[i] != 1) return VMC_EINVAL;
      nl += m->local_site[i];
    }
    const int N = Ne / 2, ni = Ns - nl;
    const int lo = std::max(std::max(0, nl - N), N - ni), hi = std::min(std::min(nl, N), ni + nl - N);
    if (lo > hi || m->local_spin) return VMC_EINVAL;
  }
  if (m->n_hop < 0 || m->n_V < 0 || m->n_J < 0) return VMC_EINVAL;
  if (m->n_hop && (!m->hop_i || !m->hop_j || !m->hop_t)) return VMC_EINVAL;
  if (m->n_V && (!m->V_i || !m->V_j || !m->V_val)) return VMC_EINVAL;
  if (m->n_J && (!m->J_i || !m->J_j || !m->J_val)) return VMC_EINVAL;
  for (int k = 0; k < m->n_hop; ++k)
    if (m->hop_i[k] < 0 || m->hop_i[k] >= Ns || m->hop_j[k] < 0 || m->hop_j[k] >= Ns ||
        m->hop_i[k] == m->hop_j[k])
      return VMC_EINVAL;
  for (int k = 0; k < m->n_V; ++k)
    if (m->V_i[k] < 0 || m->V_i[k] >= Ns || m->V_j[k] < 0 || m->V_j[k] >= Ns) return VMC_EINVAL;
  for (int k = 0; k < m->n_J; ++k)
    if (m->J_i[k] < 0 || m->J_i[k] >= Ns || m->J_j[k] < 0 || m->J_j[k] >= Ns ||
        m->J_i[k] == m->J_j[k])
      return VMC_EINVAL;
  if (l->n_g < 0 || l->n_v < 0 || l->n_f < 1) return VMC_EINVAL;
  if (l->n_hidden < 0 || l->n_hidden > 4096) return VMC_EINVAL;
  if (!l->f_idx || !l->f_sign) return VMC_EINVAL;
  if (l->n_g && !l->g_idx) return VMC_EINVAL;
  if (l->n_v && !l->v_idx) return VMC_EINVAL;
  if (l->n_g)
    for (int i = 0; i < Ns; ++i)
      if (l->g_idx[i] < -1 || l->g_idx[i] >= l->n_g) return VMC_EINVAL;
  const size_t n2 = (size_t)Ns * Ns;
  if (l->n_v)
    for (size_t q = 0; q < n2; ++q) {
      const int i = (int)(q / Ns), j = (int)(q % Ns);
      if (l->v_idx[q] < -1 || l->v_idx[q] >= l->n_v) return VMC_EINVAL;
      if (l->v_idx[q] != l->v_idx[(size_t)j * Ns + i]) return VMC_EINVAL;
    }
  for (size_t q = 0; q < n2; ++q) {
    if (l->f_idx[q] < -1 || l->f_idx[q] >= l->n_f) return VMC_EINVAL;
    if (l->f_sign[q] != 1 && l->f_sign[q] != -1 && l->f_idx[q] >= 0) return VMC_EINVAL;
  }
  const long long nm = l->n_hidden ? (long long)l->n_hidden * 2 * Ns + 2LL * l->n_hidden + 1 : 0;
  const long long Np = (long long)l->n_g + l->n_v + l->n_f + nm;
  if (Np > (1LL << 30)) return VMC_EINVAL;
  for (long long k = 0; k < Np; ++k)
    if (!isfinite(params[k])) return VMC_EINVAL;
  return VMC_OK;
}

// Event pair around a region of kernels on the context stream.
struct TimedRegion {
  vmc_ctx *c;
  int k;
  cudaEvent_t a = nullptr, b = nullptr;
  TimedRegion(vmc_ctx *c_, int k_) : c(c_), k(k_) {
    if (c->timing && cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess)
      cudaEventRecord(a, c->st);
  }
  ~TimedRegion() {
    if (a && b) {
      cudaEventRecord(b, c->st);
      c->ev[k].push_back({a, b});
    }
  }
};

void collect_times(vmc_ctx *c) {
  for (int k = 0; k < 4; ++k) {
    for (auto &p : c->ev[k]) {
      float t = 0.f;
      if (cudaEventSynchronize(p.second) == cudaSuccess &&
          cudaEventElapsedTime(&t, p.first, p.second) == cudaSuccess) {
        c->ms[k] += t;
        c->cnt[k] += 1;
      }
      cudaEventDestroy(p.first);
      cudaEventDestroy(p.second);
    }
    c->ev[k].clear();
  }
}

int upload_sysdesc(vmc_ctx *c) {
  std::vector<SysDev> h(c->n_sys);
  for (int s = 0; s < c->n_sys; ++s) h[s] = c->sys[s].dev;
  CKC(cudaMemcpyAsync(c->d_sys, h.data(), sizeof(SysDev) * c->n_sys, cudaMemcpyHostToDevice, c->st));
  return VMC_OK;
}

// Delay depth k: shared-memory size and grid of the sweep kernel follow it.
int set_delay_impl(vmc_ctx *c, int k) {
  if (k < 0 || k > VMC_DELAY_MAX) return VMC_EINVAL;
  const int kd = k <= 1 ? 0 : k;
  size_t smem = 0;
  for (auto &s : c->sys)
    smem = std::max(smem, vmc_walker_smem(c->precision == VMC_FP64 ? 0 : 1, s.N, s.Ns, s.Np,
                                          s.dev.n_hidden, kd, nullptr,
                                          c->precision == VMC_MIXED));
  if (smem > c->smem_cap) return VMC_EINVAL;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int occ = vmc_sample_occupancy(c->precision, smem);
  if (occ < 1) return VMC_EINVAL;
  // Delayed updates keep FP32 words only: entering them, the mixed form's low
  // words are zeroed so that hi + lo stays the inverse when immediate
  // (double-float) updates resume.
  if (c->precision == VMC_MIXED && c->delay_k <= 1 && k > 1)
    for (auto &s : c->sys)
      if (s.dev.minv_lo) {
        const size_t mb = ((size_t)s.N * s.ldm * 4 + 127) / 128 * 128;
        CKC(cudaMemsetAsync(s.dev.minv_lo, 0, (size_t)s.W * mb, c->st));
      }
  for (auto &s : c->sys) s.dev.delay_k = kd;
  c->smem_sample = smem;
  c->grid_sample = std::min(c->n_work, nsm * occ);
  c->delay_k = k;
  return VMC_OK;
}

// Rebuild the walkers' inverses from scratch (FP64) where needed; returns
// VMC_ESINGULAR if any walker's M is singular.
bool projected(const vmc_ctx *c);

// Periodic FP64 from-scratch inverses (fast updates accumulate rounding):
// every walker with at least recompute_every accepted moves since its last
// inverse is rebuilt.
int periodic_rebuild(vmc_ctx *c) {
  TimedRegion tr(c, 1);
  if (projected(c))
    CKC(vmc_launch_proj_build(c->d_sys, c->d_work, c->n_work, c->sys[0].dev.n_ops, c->precision,
                              1, c->recompute_every, c->smem_init, c->st, &c->n_launch));
  else
    CKC(vmc_launch_init(c->d_sys, c->d_work, c->n_work, c->d_work_ctr + 1, c->precision, 1,
                        c->recompute_every, c->smem_init, c->st, &c->n_launch));
  c->rebuild_pending = false;
  return VMC_OK;
}

// Every inverse current before it is read: the full rebuild after a parameter
// or configuration change, else the periodic rebuild the last vmc_sample left
// pending (a full rebuild makes that one moot).
int ensure_init(vmc_ctx *c, bool redraw_illcond = false) {
  bool any = false;
  for (auto &s : c->sys) any |= s.dirty;
  if (!any) {
    if (c->rebuild_pending) {
      CK(upload_sysdesc(c));
      CK(periodic_rebuild(c));
    }
    return VMC_OK;
  }
  c->rebuild_pending = false;
  CK(upload_sysdesc(c));
  {
    TimedRegion tr(c, 1);
    if (c->n_sys == 1 && c->sys[0].dev.n_ops > 0)
      CKC(vmc_launch_proj_build(c->d_sys, c->d_work, c->n_work, c->sys[0].dev.n_ops, c->precision,
                                0, 0, c->smem_init, c->st, &c->n_launch));
    else
      CKC(vmc_launch_init(c->d_sys, c->d_work, c->n_work, c->d_work_ctr + 1, c->precision, 0, 0,
                          c->smem_init, c->st,
                          &c->n_launch));
  }
  int bad = 0;
  for (auto &s : c->sys) {
    std::vector<int> st(s.W);
    CKC(cudaMemcpyAsync(st.data(), s.dev.status, sizeof(int) * s.W, cudaMemcpyDeviceToHost, c->st));
    CKC(cudaStreamSynchronize(c->st));
    for (int w = 0; w < s.W; ++w) bad |= st[w];
    s.dirty = false;
  }
  if ((bad & VMC_ST_SINGULAR) || (redraw_illcond && (bad & VMC_ST_ILLCOND))) {
    for (auto &s : c->sys) s.dirty = true;
    return VMC_ESINGULAR;
  }
  return VMC_OK;
}

int sr_alloc(vmc_ctx *c, SysHost &s, bool need_S, bool need_ir = false) {
  const int rows_cap = s.W * s.max_samples;
  if (!s.sr_alloc) {
    SrWork &w = s.sr;
    const int Np = s.Np;
    CK(dalloc(c, &w.obar, sizeof(double) * Np));
    CK(dalloc(c, &w.ebar, sizeof(double) * 8));
    CK(dalloc(c, &w.g, sizeof(double) * Np));
    CK(dalloc(c, &w.diagS, sizeof(double) * Np));
    CK(dalloc(c, &w.x, sizeof(double) * Np));
    CK(dalloc(c, &w.r, sizeof(double) * 2 * Np));
    CK(dalloc(c, &w.p, sizeof(double) * Np));
    CK(dalloc(c, &w.w, sizeof(double) * Np));
    CK(dalloc(c, &w.t, sizeof(double) * rows_cap));
    CK(dalloc(c, &w.scal, sizeof(double) * 8));
    CK(dalloc(c, &w.info, sizeof(int) * 4));
    CK(dalloc(c, &w.dblk, sizeof(double) * 32 * 32));
    CK(dalloc(c, &w.vf, sizeof(float) * Np));
    CK(dalloc(c, &w.tf, sizeof(float) * rows_cap));
    CK(dalloc(c, &w.dpart, sizeof(double) * 512));
    const size_t nparts = (size_t)vmc_colreduce_parts(rows_cap, Np);
    CK(dalloc(c, &w.part, sizeof(double) * nparts * Np));
    s.sr_alloc = true;
  }
  if (need_S && !s.S_alloc) {
    CK(dalloc(c, &s.sr.S, sizeof(double) * (size_t)s.Np * s.Np));
    if (c->precision == VMC_MIXED) {
      int ldK, Np_pad;
      vmc_tc_dims(rows_cap, s.Np, &ldK, &Np_pad);
      CK(dalloc(c, &s.tc_hi, 2 * (size_t)Np_pad * ldK));
      CK(dalloc(c, &s.tc_lo, 2 * (size_t)Np_pad * ldK));
      CK(dalloc(c, &s.tc_status, sizeof(int) * 4));
      const int ntile = vmc_tc_tile_list(s.Np, nullptr);
      std::vector<int2> tl(ntile);
      vmc_tc_tile_list(s.Np, tl.data());
      CK(dupload(c, &s.tc_tiles, tl.data(), tl.size()));
    }
    s.S_alloc = true;
  }
  s.sr.Np = s.Np;
  s.sr.rows = s.rows;
  s.sr.ldO = s.ldO;
  s.sr.precision = c->precision;
  s.sr.O = s.dev.O;
  s.sr.E = s.dev.E;
  if (need_ir && !s.sr.S32) {
    SrWork &w = s.sr;
    CK(dalloc(c, &w.S32, sizeof(float) * (size_t)s.Np * s.Np));
    CK(dalloc(c, &w.gjP, sizeof(float) * 32 * 32));
    CK(dalloc(c, &w.gjC, sizeof(float) * (size_t)(s.Np + 64) * 32));
    CK(dalloc(c, &w.rs32, sizeof(float) * s.Np));
    CK(dalloc(c, &w.dsc, sizeof(double) * s.Np));
    CK(dalloc(c, &w.irflag, sizeof(int) * 4));
  }
  return VMC_OK;
}

// Dense S~: FP64 SIMT GEMM (plain form) or split-BF16 tensor-core GEMM (mixed).
// Enqueue the S~ build (no host synchronisation; the tensor-core path's
// status stays on the device).
int build_S_launch(vmc_ctx *c, SysHost &s, double shift_rel, double shift_abs, cudaStream_t st) {
  if (c->precision == VMC_MIXED) {
    const cudaError_t e = vmc_sr_build_S_tc(s.sr, s.tc_hi, s.tc_lo, s.tc_status, shift_rel,
                                            shift_abs, s.tc_tiles, st, &c->n_launch, &s.s_kernel);
    s.sr.stall = 0;   // the test hook is armed for one build
    CKC(e);
  } else {
    CKC(vmc_sr_build_S(s.sr, shift_rel, shift_abs, st, &c->n_launch));
    s.s_kernel = VMC_S_KERNEL_FP64;
  }
  return VMC_OK;
}

int build_S(vmc_ctx *c, SysHost &s, double shift_rel, double shift_abs) {
  TimedRegion tr(c, 3);
  if (c->precision == VMC_MIXED) {
    const cudaError_t e = vmc_sr_build_S_tc(s.sr, s.tc_hi, s.tc_lo, s.tc_status, shift_rel,
                                            shift_abs, s.tc_tiles, c->st, &c->n_launch,
                                            &s.s_kernel);
    s.sr.stall = 0;   // the test hook is armed for one build
    CKC(e);
    int bad = 0;
    CKC(cudaMemcpyAsync(&bad, s.tc_status, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CKC(cudaStreamSynchronize(c->st));
    if (bad) return VMC_ETIMEOUT;
    return VMC_OK;
  }
  CKC(vmc_sr_build_S(s.sr, shift_rel, shift_abs, c->st, &c->n_launch));
  s.s_kernel = VMC_S_KERNEL_FP64;
  return VMC_OK;
}

// From-scratch inverses of every walker; walkers whose M (or, for a projected
// context, whose projected amplitude) is singular or ill-conditioned get a
// new seeded placement, at most 20 times.
int init_with_redraw(vmc_ctx *c, uint64_t state) {
  for (int attempt = 0;; ++attempt) {
    const int rc = ensure_init(c, true);
    if (rc == VMC_OK) return VMC_OK;
    if (rc != VMC_ESINGULAR || attempt >= 20) return rc;
    for (SysHost &s : c->sys) {
      std::vector<int> st(s.W);
      std::vector<int32_t> ele((size_t)s.W * s.Ne);
      if (cudaMemcpy(st.data(), s.dev.status, sizeof(int) * s.W, cudaMemcpyDeviceToHost) ||
          cudaMemcpy(ele.data(), s.dev.ele, sizeof(int32_t) * ele.size(), cudaMemcpyDeviceToHost))
        return VMC_ECUDA;
      for (int w = 0; w < s.W; ++w)
        if (st[w] & (VMC_ST_SINGULAR | VMC_ST_ILLCOND))
          random_placement(s.Ns, s.Ne, s.dev.local_spin != 0,
                           s.lsite.empty() ? nullptr : s.lsite.data(), state,
                           ele.data() + (size_t)w * s.Ne);
      std::vector<int> zero(s.W, 0);
      if (cudaMemcpy(s.dev.ele, ele.data(), sizeof(int32_t) * ele.size(), cudaMemcpyHostToDevice) ||
          cudaMemcpy(s.dev.status, zero.data(), sizeof(int) * s.W, cudaMemcpyHostToDevice))
        return VMC_ECUDA;
    }
  }
}

int create_impl(vmc_ctx **out, int n_sys, const vmc_model *models, const int32_t *Ne,
                const vmc_layout *layouts, const double *const *params, const double *pex,
                const vmc_opts *o) {
  if (!out || n_sys < 1 || !models || !Ne || !layouts || !params || !o) return VMC_EINVAL;
  *out = nullptr;
  if (o->n_walkers < 1 || o->max_samples < 1) return VMC_EINVAL;
  if (o->precision != VMC_FP64 && o->precision != VMC_MIXED) return VMC_EINVAL;
  if (o->rebuild != VMC_REBUILD_FP64 && o->rebuild != VMC_REBUILD_DOUBLE_FLOAT) return VMC_EINVAL;
  for (int s = 0; s < n_sys; ++s) {
    CK(validate_system(&models[s], Ne[s], &layouts[s], params[s]));
    if (pex && (!(pex[s] >= 0.0) || pex[s] > 1.0)) return VMC_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return VMC_ECUDA;
  }
  vmc_ctx *c = new (std::nothrow) vmc_ctx();
  if (!c) return VMC_ENOMEM;
  c->n_sys = n_sys;
  c->precision = o->precision;
  c->seed = o->seed;
  c->st = (cudaStream_t)o->stream;
  c->sys.resize(n_sys);
  const int esize = o->precision == VMC_FP64 ? 8 : 4;
  int rc = VMC_OK;
  size_t smem64 = 0, smem32 = 0;
  int maxN = 1;
  auto fail = [&](int e) {
    ctx_free(c);
    delete c;
    return e;
  };
  for (int si = 0; si < n_sys; ++si) {
    const vmc_model &m = models[si];
    const vmc_layout &l = layouts[si];
    SysHost &s = c->sys[si];
    s.Ns = m.Ns;
    s.Ne = Ne[si];
    s.N = s.Ne / 2;
    s.ldm = (s.N % 2) ? s.N : s.N + 1;
    s.n_g = l.n_g;
    s.n_v = l.n_v;
    s.n_f = l.n_f;
    const int H = l.n_hidden;
    s.Np = l.n_g + l.n_v + l.n_f + (H ? H * 2 * m.Ns + 2 * H + 1 : 0);
    s.ldO = (s.Np + 3) / 4 * 4;
    s.W = o->n_walkers;
    s.max_samples = o->max_samples;
    s.p_exchange = m.local_spin ? 1.0 : (pex ? pex[si] : 0.0);
    maxN = std::max(maxN, s.N);
    SysDev &d = s.dev;
    d.Ns = s.Ns;
    d.Ne = s.Ne;
    d.N = s.N;
    d.ldm = s.ldm;
    d.n_hop = m.n_hop;
    d.n_V = m.n_V;
    d.n_J = m.n_J;
    d.local_spin = m.local_spin ? 1 : 0;
    d.stall_walker = -1;
    d.spec_b = 1;
    d.lsite = nullptr;
    if (m.local_site) {
      s.lsite.assign((const signed char *)m.local_site, (const signed char *)m.local_site + m.Ns);
      if ((rc = dupload(c, (signed char **)&d.lsite, s.lsite.data(), (size_t)m.Ns))) return fail(rc);
    }
    {
      const double t = s.p_exchange * 4294967296.0;
      d.pex = t >= 4294967296.0 ? 4294967296ull : (unsigned long long)t;
    }
    d.Np = s.Np;
    d.n_g = s.n_g;
    d.n_v = s.n_v;
    d.n_f = s.n_f;
    d.ldO = s.ldO;
    d.W = s.W;
    d.sys_index = si;
    d.n_samples = s.max_samples;
    const size_t Ns = s.Ns, n2 = Ns * Ns;
    std::vector<double> Uz(Ns, 0.0);
    const int *hi = nullptr, *hj = nullptr;
    const double *ht = nullptr;
    if ((rc = dupload(c, (int **)&hi, m.hop_i, m.n_hop))) return fail(rc);
    if ((rc = dupload(c, (int **)&hj, m.hop_j, m.n_hop))) return fail(rc);
    if ((rc = dupload(c, (double **)&ht, m.hop_t, m.n_hop))) return fail(rc);
    d.hop_i = hi;
    d.hop_j = hj;
    {
      // hopping terms grouped by target site (CSR) for the measurement kernel
      std::vector<int> ptr(Ns + 1, 0), term(m.n_hop);
      for (int k = 0; k < m.n_hop; ++k) ptr[m.hop_i[k] + 1]++;
      for (size_t i = 0; i < Ns; ++i) ptr[i + 1] += ptr[i];
      std::vector<int> fill(ptr.begin(), ptr.end() - 1);
      for (int k = 0; k < m.n_hop; ++k) term[fill[m.hop_i[k]]++] = k;
      if ((rc = dupload(c, (int **)&d.tgt_ptr, ptr.data(), Ns + 1))) return fail(rc);
      if ((rc = dupload(c, (int **)&d.tgt_term, term.data(), m.n_hop))) return fail(rc);
      std::vector<int> tj(m.n_hop);
      std::vector<double> tt(m.n_hop);
      for (int q = 0; q < m.n_hop; ++q) {
        tj[q] = m.hop_j[term[q]];
        tt[q] = m.hop_t[term[q]];
      }
      if ((rc = dupload(c, (int **)&d.tgt_j, tj.data(), m.n_hop))) return fail(rc);
      if ((rc = dupload(c, (double **)&d.tgt_t, tt.data(), m.n_hop))) return fail(rc);
      if ((rc = dalloc(c, &d.tgt_v64, sizeof(double) * (m.n_hop ? m.n_hop : 1)))) return fail(rc);
      if ((rc = dalloc(c, &d.tgt_v32, sizeof(float) * (m.n_hop ? m.n_hop : 1)))) return fail(rc);
    }
    d.hop_t = ht;
    if ((rc = dupload(c, (double **)&d.U, m.U ? m.U : Uz.data(), Ns))) return fail(rc);
    if ((rc = dupload(c, (int **)&d.V_i, m.V_i, m.n_V))) return fail(rc);
    if ((rc = dupload(c, (int **)&d.V_j, m.V_j, m.n_V))) return fail(rc);
    if ((rc = dupload(c, (double **)&d.V_val, m.V_val, m.n_V))) return fail(rc);
    if ((rc = dupload(c, (int **)&d.J_i, m.J_i, m.n_J))) return fail(rc);
    if ((rc = dupload(c, (int **)&d.J_j, m.J_j, m.n_J))) return fail(rc);
    if ((rc = dupload(c, (double **)&d.J_val, m.J_val, m.n_J))) return fail(rc);
    {
      // the exchange terms by site (each term under both of its sites), for
      // the measurement's grouping by the site that receives the up electron
      std::vector<int> jp(Ns + 1, 0);
      std::vector<int2> ja(m.n_J ? 2 * (size_t)m.n_J : 1);
      for (int k = 0; k < m.n_J; ++k) {
        jp[m.J_i[k] + 1]++;
        jp[m.J_j[k] + 1]++;
      }
      for (size_t i = 0; i < Ns; ++i) jp[i + 1] += jp[i];
      std::vector<int> cur(jp.begin(), jp.end() - 1);
      for (int k = 0; k < m.n_J; ++k) {
        ja[cur[m.J_i[k]]++] = make_int2(k, m.J_j[k]);
        ja[cur[m.J_j[k]]++] = make_int2(k, m.J_i[k]);
      }
      if ((rc = dupload(c, (int **)&d.jptr, jp.data(), Ns + 1))) return fail(rc);
      if ((rc = dupload(c, (int2 **)&d.jadj, ja.data(), ja.size()))) return fail(rc);
    }
    std::vector<int> gneg(Ns, -1), vneg;
    if ((rc = dupload(c, (int **)&d.g_idx, l.n_g ? l.g_idx : gneg.data(), Ns))) return fail(rc);
    if (!l.n_v) vneg.assign(n2, -1);
    if ((rc = dupload(c, (int **)&d.v_idx, l.n_v ? l.v_idx : vneg.data(), n2))) return fail(rc);
    if ((rc = dupload(c, (int **)&d.f_idx, l.f_idx, n2))) return fail(rc);
    if ((rc = dupload(c, (signed char **)&d.f_sign, (const signed char *)l.f_sign, n2))) return fail(rc);
    {
      // measurement tables: packed pair-orbital class + sign, Jastrow pairs by class
      std::vector<int> fc(n2);
      for (size_t q = 0; q < n2; ++q) fc[q] = l.f_idx[q] >= 0 ? 2 * l.f_idx[q] + (l.f_sign[q] < 0) : -1;
      if ((rc = dupload(c, (int **)&d.fcode, fc.data(), n2))) return fail(rc);
      std::vector<int> vp(l.n_v + 1, 0);
      std::vector<unsigned> pr;
      if (l.n_v) {
        for (size_t i = 0; i < Ns; ++i)
          for (size_t j = i + 1; j < Ns; ++j)
            if (l.v_idx[i * Ns + j] >= 0) vp[l.v_idx[i * Ns + j] + 1]++;
        for (int k = 0; k < l.n_v; ++k) vp[k + 1] += vp[k];
        pr.resize(vp[l.n_v]);
        std::vector<int> fill(vp.begin(), vp.end() - 1);
        for (size_t i = 0; i < Ns; ++i)
          for (size_t j = i + 1; j < Ns; ++j) {
            const int k = l.v_idx[i * Ns + j];
            if (k >= 0) pr[fill[k]++] = (unsigned)i | ((unsigned)j << 16);
          }
      }
      if ((rc = dupload(c, (int **)&d.vptr, vp.data(), vp.size()))) return fail(rc);
      if ((rc = dupload(c, (unsigned **)&d.vpair, pr.empty() ? nullptr : pr.data(), pr.size())))
        return fail(rc);
    }
    if ((rc = dupload(c, (double **)&d.params, params[si], s.Np))) return fail(rc);
    if ((rc = dalloc(c, &d.f64, sizeof(double) * n2))) return fail(rc);
    if ((rc = dalloc(c, &d.fT64, sizeof(double) * n2))) return fail(rc);
    if ((rc = dalloc(c, &d.f32, sizeof(float) * n2))) return fail(rc);
    if ((rc = dalloc(c, &d.fT32, sizeof(float) * n2))) return fail(rc);
    if ((rc = dalloc(c, &d.vmat, sizeof(double) * n2))) return fail(rc);
    if ((rc = dalloc(c, &d.gsite, sizeof(double) * Ns))) return fail(rc);
    if ((rc = dalloc(c, &d.vmat32, sizeof(float) * n2))) return fail(rc);
    if ((rc = dalloc(c, &d.gsite32, sizeof(float) * Ns))) return fail(rc);
    d.n_hidden = H;
    d.mlp_base = l.n_g + l.n_v + l.n_f;
    if (H) {
      if ((rc = dalloc(c, &d.W1T64, sizeof(double) * (size_t)H * 2 * Ns))) return fail(rc);
      if ((rc = dalloc(c, &d.W1T16, 2 * (size_t)H * 2 * Ns))) return fail(rc);
      if ((rc = dalloc(c, &d.hmlp, (size_t)esize * H * o->n_walkers))) return fail(rc);
    }
    const size_t W = s.W;
    const size_t mb = ((size_t)s.N * s.ldm * esize + 127) / 128 * 128;
    if ((rc = dalloc(c, &d.ele, sizeof(int) * W * s.Ne))) return fail(rc);
    if ((rc = dalloc(c, &d.occ, sizeof(int) * W * 2 * Ns))) return fail(rc);
    if ((rc = dalloc(c, &d.minv, mb * W))) return fail(rc);
    d.minv_lo = nullptr;
    if (o->precision == VMC_MIXED && (rc = dalloc(c, &d.minv_lo, mb * W))) return fail(rc);
    d.rebuild_df = (o->precision == VMC_MIXED && o->rebuild == VMC_REBUILD_DOUBLE_FLOAT) ? 1 : 0;
    if ((rc = dalloc(c, &d.jf, (size_t)esize * W * Ns))) return fail(rc);
    if ((rc = dupload(c, &d.ctr, (const unsigned long long *)nullptr, W))) return fail(rc);
    if ((rc = dupload(c, &d.logdet, (const double *)nullptr, W))) return fail(rc);
    if ((rc = dupload(c, &d.detsign, (const int *)nullptr, W))) return fail(rc);
    if ((rc = dupload(c, &d.n_prop, (const long long *)nullptr, W))) return fail(rc);
    if ((rc = dupload(c, &d.n_acc, (const long long *)nullptr, W))) return fail(rc);
    if ((rc = dupload(c, &d.cnt, (const long long *)nullptr, 8 * W))) return fail(rc);
    if ((rc = dupload(c, &d.n_rec, (const long long *)nullptr, W))) return fail(rc);
    if ((rc = dupload(c, &d.acc_since, (const int *)nullptr, W))) return fail(rc);
    if ((rc = dupload(c, &d.status, (const int *)nullptr, W))) return fail(rc);
    if ((rc = dupload(c, &d.drift, (const double *)nullptr, W))) return fail(rc);
    const size_t rows_cap = W * s.max_samples;
    if ((rc = dupload(c, &d.E, (const double *)nullptr, rows_cap))) return fail(rc);
    if ((rc = dalloc(c, &d.O, (size_t)esize * rows_cap * s.ldO))) return fail(rc);
    int acc_len = 0;
    smem64 = std::max(smem64, vmc_walker_smem(0, s.N, s.Ns, s.Np, H, 0, &acc_len, 0));
    smem32 = std::max(smem32, vmc_walker_smem(1, s.N, s.Ns, s.Np, H, 0, &acc_len, 1));
    d.acc_len = acc_len;
    c->smem_init = std::max(c->smem_init, vmc_init_smem(s.N, s.Ns));
    if (vmc_launch_expand(&d, c->st, &c->n_launch) != cudaSuccess) return fail(VMC_ECUDA);
    // seeded random placement
    std::vector<int32_t> ele(W * s.Ne);
    uint64_t state = o->seed ^ (0xA0761D6478BD642Full * (uint64_t)(si + 1));
    for (size_t w = 0; w < W; ++w)
      random_placement(s.Ns, s.Ne, m.local_spin != 0, s.lsite.empty() ? nullptr : s.lsite.data(),
                       state, ele.data() + w * s.Ne);
    if (cudaMemcpyAsync(d.ele, ele.data(), sizeof(int32_t) * ele.size(), cudaMemcpyHostToDevice,
                        c->st) != cudaSuccess)
      return fail(VMC_ECUDA);
  }
  c->smem_sample = (c->precision == VMC_FP64) ? smem64 : smem32;
  {
    // The sweep kernels may use up to the device's opt-in limit (less the
    // static part): delayed updates enlarge the walker's shared state.
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    c->smem_cap = optin > 4096 ? (size_t)optin - 4096 : 0;
    if (c->smem_sample > c->smem_cap || c->smem_init > (size_t)optin) return fail(VMC_EINVAL);
    if (vmc_walker_set_smem_limits(c->smem_cap, c->smem_cap, c->smem_init) != cudaSuccess) {
      cudaGetLastError();
      return fail(VMC_EINVAL);  // does not fit in shared memory
    }
  }
  // work list: (system, walker), larger N first
  std::vector<int2> work;
  std::vector<int> order(n_sys);
  for (int s = 0; s < n_sys; ++s) order[s] = s;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return c->sys[a].N > c->sys[b].N; });
  for (int s : order)
    for (int w = 0; w < c->sys[s].W; ++w) work.push_back(make_int2(s, w));
  c->n_work = (int)work.size();
  if ((rc = dupload(c, &c->d_work, work.data(), work.size()))) return fail(rc);
  if ((rc = dalloc(c, &c->d_work_ctr, sizeof(int) * 4))) return fail(rc);
  if ((rc = dalloc(c, &c->d_sys, sizeof(SysDev) * n_sys))) return fail(rc);
  if ((rc = dalloc(c, &c->d_scalar, sizeof(double) * 8))) return fail(rc);
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int occ = std::max(1, vmc_sample_occupancy(c->precision, c->smem_sample));
  c->grid_sample = std::min(c->n_work, nsm * occ);
  if ((rc = set_delay_impl(c, o->delay_k))) return fail(rc);
  c->recompute_every = o->recompute_every > 0 ? o->recompute_every
                       : (o->recompute_every == 0 && o->precision == VMC_MIXED) ? 64 : 0;
  // Initial inverses; re-draw placements whose M is singular (bounded).
  if ((rc = init_with_redraw(c, o->seed ^ 0x5851F42D4C957F2Dull))) return fail(rc);
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return fail(VMC_ECUDA);
  *out = c;
  return VMC_OK;
}

bool sys_ok(vmc_ctx *c, int s) { return c && s >= 0 && s < c->n_sys; }

bool projected(const vmc_ctx *c) { return c->n_sys == 1 && c->sys[0].dev.n_ops > 0; }



}  // namespace

extern "C" {

const char *vmc_strerror(int code) {
  switch (code) {
    case VMC_OK: return "ok";
    case VMC_EINVAL: return "invalid argument";
    case VMC_ENOMEM: return "out of memory";
    case VMC_ECUDA: return "CUDA error";
    case VMC_ESINGULAR: return "singular matrix (Pf(X) = 0 or S not positive definite)";
    case VMC_ENUMERIC: return "numerical fault (NaN/Inf or breakdown)";
    case VMC_ETIMEOUT: return "bounded device wait expired";
    case VMC_ESTATE: return "call not valid in the current state";
    default: return "unknown error";
  }
}

int vmc_create(vmc_ctx **out, const vmc_model *model, int32_t Ne, const vmc_layout *layout,
               const double *params, double p_exchange, const vmc_opts *opts) {
  const double *pp[1] = {params};
  return create_impl(out, 1, model, &Ne, layout, pp, &p_exchange, opts);
}

int vmc_create_batch(vmc_ctx **out, int32_t n_systems, const vmc_model *models, const int32_t *Ne,
                     const vmc_layout *layouts, const double *const *params,
                     const double *p_exchange, const vmc_opts *opts) {
  return create_impl(out, n_systems, models, Ne, layouts, params, p_exchange, opts);
}

void vmc_destroy(vmc_ctx *ctx) {
  if (!ctx) return;
  if (ctx->st) cudaStreamSynchronize(ctx->st);
  else cudaDeviceSynchronize();
  collect_times(ctx);
  ctx_free(ctx);
  delete ctx;
}

int vmc_set_configs(vmc_ctx *c, int32_t system, const int32_t *ele, const uint64_t *counters) {
  if (!sys_ok(c, system) || !ele) return VMC_EINVAL;
  SysHost &s = c->sys[system];
  CK(validate_configs(s, s.dev.local_spin != 0, ele, s.W));
  CKC(cudaMemcpyAsync(s.dev.ele, ele, sizeof(int32_t) * (size_t)s.W * s.Ne, cudaMemcpyHostToDevice, c->st));
  if (counters)
    CKC(cudaMemcpyAsync(s.dev.ctr, counters, sizeof(uint64_t) * s.W, cudaMemcpyHostToDevice, c->st));
  CKC(cudaMemsetAsync(s.dev.status, 0, sizeof(int) * s.W, c->st));
  CKC(cudaStreamSynchronize(c->st));
  s.dirty = true;
  return VMC_OK;
}

int vmc_get_configs(vmc_ctx *c, int32_t system, int32_t *ele, uint64_t *counters) {
  if (!sys_ok(c, system)) return VMC_EINVAL;
  SysHost &s = c->sys[system];
  if (ele)
    CKC(cudaMemcpyAsync(ele, s.dev.ele, sizeof(int32_t) * (size_t)s.W * s.Ne, cudaMemcpyDeviceToHost, c->st));
  if (counters)
    CKC(cudaMemcpyAsync(counters, s.dev.ctr, sizeof(uint64_t) * s.W, cudaMemcpyDeviceToHost, c->st));
  CKC(cudaStreamSynchronize(c->st));
  return VMC_OK;
}

int vmc_sample(vmc_ctx *c, int32_t n_warmup, int32_t n_samples, int32_t sweeps_between) {
  if (!c || n_warmup < 0 || n_samples < 0 || sweeps_between < 0) return VMC_EINVAL;
  for (auto &s : c->sys)
    if (n_samples > s.max_samples) return VMC_EINVAL;
  CK(ensure_init(c));
  for (auto &s : c->sys) {
    s.dev.n_samples = n_samples > 0 ? n_samples : s.max_samples;
    if (n_samples > 0) {
      s.n_samples = n_samples;
      s.rows = s.W * n_samples;
    }
  }
  CK(upload_sysdesc(c));
  // the sweep test hook is armed for this call's launches only
  for (auto &s : c->sys) s.dev.stall_walker = -1;
  const bool proj = projected(c);
  auto sweep = [&](int n_first, int ns, int sb, int base) -> int {
    TimedRegion tr(c, 0);
    if (proj)
      CKC(vmc_launch_proj_sample(c->d_sys, c->d_work, c->n_work, c->d_work_ctr, c->precision,
                                 c->seed, n_first, ns, sb, base, c->grid_proj, c->smem_proj, c->st,
                                 &c->n_launch));
    else
      CKC(vmc_launch_sample(c->d_sys, c->d_work, c->n_work, c->d_work_ctr, c->precision, c->seed,
                            n_first, ns, sb, base, c->grid_sample, c->smem_sample, c->st,
                            &c->n_launch));
    return VMC_OK;
  };
  if (c->recompute_every <= 0) {
    CK(sweep(n_warmup, n_samples, sweeps_between, 0));
  } else {
    // The periodic rebuild follows every sweep launch but the call's last:
    // that one is left pending and runs when an inverse is next needed (the
    // next call's sweeps, or a check hook), unless a parameter change first
    // makes every inverse a full rebuild, as an SR step does.
    const int launches = n_warmup + n_samples;
    int done = 0;
    for (int k = 0; k < n_warmup; ++k) {
      CK(sweep(1, 0, 0, 0));
      if (++done < launches) CK(periodic_rebuild(c));
    }
    for (int k = 0; k < n_samples; ++k) {
      CK(sweep(0, 1, sweeps_between, k));
      if (++done < launches) CK(periodic_rebuild(c));
    }
    if (launches > 0) c->rebuild_pending = true;
  }
  int bad = 0;
  for (auto &s : c->sys) {
    std::vector<int> st(s.W);
    CKC(cudaMemcpyAsync(st.data(), s.dev.status, sizeof(int) * s.W, cudaMemcpyDeviceToHost, c->st));
    CKC(cudaStreamSynchronize(c->st));
    for (int w = 0; w < s.W; ++w) bad |= st[w];
  }
  if (bad & VMC_ST_TIMEOUT) return VMC_ETIMEOUT;
  if (bad & VMC_ST_SINGULAR) return VMC_ESINGULAR;
  if (bad & VMC_ST_NUMERIC) return VMC_ENUMERIC;
  return VMC_OK;
}

int vmc_measure(vmc_ctx *c, int32_t system, vmc_stats *out) {
  if (!sys_ok(c, system) || !out) return VMC_EINVAL;
  SysHost &s = c->sys[system];
  memset(out, 0, sizeof(*out));
  std::vector<long long> np(s.W), na(s.W);
  std::vector<int> st(s.W);
  std::vector<double> dr(s.W);
  CKC(cudaMemcpyAsync(np.data(), s.dev.n_prop, sizeof(long long) * s.W, cudaMemcpyDeviceToHost, c->st));
  CKC(cudaMemcpyAsync(na.data(), s.dev.n_acc, sizeof(long long) * s.W, cudaMemcpyDeviceToHost, c->st));
  CKC(cudaMemcpyAsync(st.data(), s.dev.status, sizeof(int) * s.W, cudaMemcpyDeviceToHost, c->st));
  CKC(cudaMemcpyAsync(dr.data(), s.dev.drift, sizeof(double) * s.W, cudaMemcpyDeviceToHost, c->st));
  std::vector<long long> cn(8 * (size_t)s.W), nr(s.W);
  CKC(cudaMemcpyAsync(cn.data(), s.dev.cnt, sizeof(long long) * cn.size(), cudaMemcpyDeviceToHost, c->st));
  CKC(cudaMemcpyAsync(nr.data(), s.dev.n_rec, sizeof(long long) * s.W, cudaMemcpyDeviceToHost, c->st));
  std::vector<double> E(s.rows);
  if (s.rows)
    CKC(cudaMemcpyAsync(E.data(), s.dev.E, sizeof(double) * s.rows, cudaMemcpyDeviceToHost, c->st));
  CKC(cudaStreamSynchronize(c->st));
  for (int w = 0; w < s.W; ++w) {
    out->n_proposals += np[w];
    out->n_accepted += na[w];
    out->n_flagged += (st[w] & (VMC_ST_SINGULAR | VMC_ST_NUMERIC | VMC_ST_TIMEOUT)) != 0;
    out->max_drift = std::max(out->max_drift, dr[w]);
    out->n_hop_tested += cn[8 * w + 0];
    out->n_exchange_tested += cn[8 * w + 1];
    out->n_hop_accepted += cn[8 * w + 2];
    out->n_exchange_accepted += cn[8 * w + 3];
    out->n_measured_hops += cn[8 * w + 4];
    out->n_measured_exchanges += cn[8 * w + 5];
    out->n_measurements += cn[8 * w + 6];
    out->n_recomputes += nr[w];
  }
  out->acceptance = out->n_proposals ? (double)out->n_accepted / out->n_proposals : 0.0;
  out->n_samples = s.rows;
  if (s.rows) {
    double sum = 0.0;
    for (double e : E) sum += e;
    const double mean = sum / s.rows;
    double var = 0.0;
    for (double e : E) var += (e - mean) * (e - mean);
    out->energy = mean;
    out->variance = s.rows > 1 ? var / (s.rows - 1) : 0.0;
    const int per = s.n_samples > 0 ? s.n_samples : 1;
    const int nw = s.rows / per;
    if (nw > 1) {
      double m1 = 0.0, m2 = 0.0;
      for (int w = 0; w < nw; ++w) {
        double a = 0.0;
        for (int k = 0; k < per; ++k) a += E[(size_t)w * per + k];
        a /= per;
        m1 += a;
        m2 += a * a;
      }
      m1 /= nw;
      const double vw = (m2 / nw - m1 * m1) * nw / (nw - 1);
      out->stderr_walkers = sqrt(std::max(vw, 0.0) / nw);
    }
  }
  return VMC_OK;
}

int vmc_get_samples(vmc_ctx *c, int32_t system, double *E, double *O) {
  if (!sys_ok(c, system)) return VMC_EINVAL;
  SysHost &s = c->sys[system];
  if (!s.rows) return VMC_ESTATE;
  if (E) CKC(cudaMemcpyAsync(E, s.dev.E, sizeof(double) * s.rows, cudaMemcpyDeviceToHost, c->st));
  if (O) {
    if (c->precision == VMC_FP64) {
      CKC(cudaMemcpy2DAsync(O, sizeof(double) * s.Np, s.dev.O, sizeof(double) * s.ldO,
                            sizeof(double) * s.Np, s.rows, cudaMemcpyDeviceToHost, c->st));
    } else {
      std::vector<float> tmp((size_t)s.rows * s.ldO);
      CKC(cudaMemcpyAsync(tmp.data(), s.dev.O, sizeof(float) * tmp.size(), cudaMemcpyDeviceToHost, c->st));
      CKC(cudaStreamSynchronize(c->st));
      for (size_t r = 0; r < (size_t)s.rows; ++r)
        for (int k = 0; k < s.Np; ++k) O[r * s.Np + k] = tmp[r * s.ldO + k];
    }
  }
  CKC(cudaStreamSynchronize(c->st));
  return VMC_OK;
}

int vmc_set_samples(vmc_ctx *c, int32_t system, int32_t rows, const double *E, const double *O) {
  if (!sys_ok(c, system) || !E || !O) return VMC_EINVAL;
  SysHost &s = c->sys[system];
  if (rows < 1 || rows > s.W * s.max_samples) return VMC_EINVAL;
  CKC(cudaMemcpyAsync(s.dev.E, E, sizeof(double) * rows, cudaMemcpyHostToDevice, c->st));
  if (c->precision == VMC_FP64) {
    CKC(cudaMemcpy2DAsync(s.dev.O, sizeof(double) * s.ldO, O, sizeof(double) * s.Np,
                          sizeof(double) * s.Np, rows, cudaMemcpyHostToDevice, c->st));
  } else {
    std::vector<float> tmp((size_t)rows * s.ldO, 0.0f);
    for (size_t r = 0; r < (size_t)rows; ++r)
      for (int k = 0; k < s.Np; ++k) tmp[r * s.ldO + k] = (float)O[r * s.Np + k];
    CKC(cudaMemcpyAsync(s.dev.O, tmp.data(), sizeof(float) * tmp.size(), cudaMemcpyHostToDevice, c->st));
    CKC(cudaStreamSynchronize(c->st));
  }
  CKC(cudaStreamSynchronize(c->st));
  s.rows = rows;
  s.n_samples = 1;
  return VMC_OK;
}

int vmc_get_sr_matrices(vmc_ctx *c, int32_t system, double shift_rel, double shift_abs, double *S,
                        double *g) {
  if (!sys_ok(c, system)) return VMC_EINVAL;
  SysHost &s = c->sys[system];
  if (!s.rows) return VMC_ESTATE;
  CK(sr_alloc(c, s, S != nullptr));
  CKC(vmc_sr_means(s.sr, c->st, &c->n_launch));
  CKC(vmc_sr_build_g(s.sr, c->st, &c->n_launch));
  if (S) {
    CK(build_S(c, s, shift_rel, shift_abs));
    CKC(cudaMemcpyAsync(S, s.sr.S, sizeof(double) * (size_t)s.Np * s.Np, cudaMemcpyDeviceToHost, c->st));
  }
  if (g) CKC(cudaMemcpyAsync(g, s.sr.g, sizeof(double) * s.Np, cudaMemcpyDeviceToHost, c->st));
  CKC(cudaStreamSynchronize(c->st));
  return VMC_OK;
}

int vmc_sr_step(vmc_ctx *c, int32_t system, const vmc_sr_opts *o, vmc_sr_report *rep) {
  if (!sys_ok(c, system) || !o) return VMC_EINVAL;
  if (!(o->dtau > 0.0) || o->shift_rel < 0.0 || o->shift_abs < 0.0) return VMC_EINVAL;
  if (o->solver != VMC_SOLVE_CHOLESKY && o->solver != VMC_SOLVE_CG &&
      o->solver != VMC_SOLVE_CG_DENSE && o->solver != VMC_SOLVE_MIXED_IR)
    return VMC_EINVAL;
  SysHost &s = c->sys[system];
  if (!s.rows) return VMC_ESTATE;
  const bool chol = o->solver == VMC_SOLVE_CHOLESKY;
  const bool dense = o->solver == VMC_SOLVE_CG_DENSE;
  const bool ir = o->solver == VMC_SOLVE_MIXED_IR;
  CK(sr_alloc(c, s, chol || dense || ir, ir));
  SrWork &w = s.sr;
  s.s_kernel = VMC_S_KERNEL_NONE;
  TimedRegion tr(c, 2);
  CKC(vmc_sr_means(w, c->st, &c->n_launch));
  CKC(vmc_sr_build_g(w, c->st, &c->n_launch));
  int iters = 0, fallback = 0;
  double rel_res = 0.0;
  if (ir) {
    CK(build_S(c, s, o->shift_rel, o->shift_abs));
    const double eps = o->cg_eps > 0.0 ? o->cg_eps : 1e-12;
    const int kmax = o->cg_kmax > 0 ? std::min(o->cg_kmax, 16) : 8;
    const int rc = vmc_sr_ir_solve(w, kmax, eps, &iters, &rel_res, c->st, &c->n_launch);
    if (rc < 0) return rc;
    if (rc == 1) {
      fallback = 1;
      const int rc2 = vmc_sr_cholesky_solve(w, c->st, &c->n_launch);
      if (rc2) return rc2;
    }
  } else if (chol) {
    CK(build_S(c, s, o->shift_rel, o->shift_abs));
    const int rc = vmc_sr_cholesky_solve(w, c->st, &c->n_launch);
    if (rc) return rc;
  } else {
    const double eps = o->cg_eps > 0.0 ? o->cg_eps : 1e-10;
    const int kmax = o->cg_kmax > 0 ? o->cg_kmax : 1000;
    if (dense) CK(build_S(c, s, o->shift_rel, o->shift_abs));
    else CKC(vmc_sr_diag(w, c->st, &c->n_launch));
    const int rc = vmc_sr_cg_solve(w, o->shift_rel, o->shift_abs, eps, kmax, &iters, c->st,
                                   &c->n_launch, dense ? 1 : 0);
    if (rc) return rc;
  }
  double gg = 0.0, xx = 0.0, eb = 0.0;
  CKC(vmc_dot_host(w.g, w.g, s.Np, &gg, c->d_scalar, c->st, &c->n_launch));
  CKC(vmc_dot_host(w.x, w.x, s.Np, &xx, c->d_scalar, c->st, &c->n_launch));
  CKC(cudaMemcpyAsync(&eb, w.ebar, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CKC(cudaStreamSynchronize(c->st));
  if (!isfinite(xx)) return VMC_ENUMERIC;
  CKC(vmc_sr_update_params((double *)s.dev.params, w.x, o->dtau, s.Np, c->st, &c->n_launch));
  CKC(vmc_launch_expand(&s.dev, c->st, &c->n_launch));
  CKC(cudaStreamSynchronize(c->st));
  s.dirty = true;
  if (rep) {
    rep->energy = eb;
    rep->norm_g = sqrt(gg);
    rep->norm_dalpha = o->dtau * sqrt(xx);
    rep->cg_iters = iters;
    rep->n_params = s.Np;
    rep->rel_residual = rel_res;
    rep->fallback = fallback;
    rep->s_kernel = s.s_kernel;
  }
  return VMC_OK;
}

// Results of one system's SR step copied to pinned host memory, read after
// the single synchronisation of vmc_sr_step_all.
struct SrStage {
  int irflag[4];
  int info[4];
  int tcstat[4];
  double irsc[3];
  double ebar, gg, xx;
};

int vmc_sr_step_all(vmc_ctx *c, const vmc_sr_opts *o, vmc_sr_report *reps) {
  if (!c || !o) return VMC_EINVAL;
  if (!(o->dtau > 0.0) || o->shift_rel < 0.0 || o->shift_abs < 0.0) return VMC_EINVAL;
  if (o->solver == VMC_SOLVE_CG || o->solver == VMC_SOLVE_CG_DENSE) {
    // the CG loop reads its convergence flag on the host: system by system
    for (int si = 0; si < c->n_sys; ++si) CK(vmc_sr_step(c, si, o, reps ? reps + si : nullptr));
    return VMC_OK;
  }
  if (o->solver != VMC_SOLVE_CHOLESKY && o->solver != VMC_SOLVE_MIXED_IR) return VMC_EINVAL;
  for (auto &s : c->sys)
    if (!s.rows) return VMC_ESTATE;
  const bool ir = o->solver == VMC_SOLVE_MIXED_IR;
  if (!c->pin) {
    if (cudaHostAlloc((void **)&c->pin, sizeof(SrStage) * (size_t)c->n_sys, cudaHostAllocDefault) !=
        cudaSuccess) {
      cudaGetLastError();
      c->pin = nullptr;
      return VMC_ENOMEM;
    }
  }
  SrStage *stg = (SrStage *)c->pin;
  if (!c->fork_ev) {
    bool okp = cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; okp && k < vmc_ctx::NPOOL; ++k)
      okp = cudaStreamCreateWithFlags(&c->pool[k], cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&c->join_ev[k], cudaEventDisableTiming) == cudaSuccess;
    if (!okp) {
      cudaGetLastError();
      return VMC_ECUDA;
    }
  }
  for (auto &s : c->sys) CK(sr_alloc(c, s, true, ir));
  const double eps = o->cg_eps > 0.0 ? o->cg_eps : 1e-12;
  const int kmax = o->cg_kmax > 0 ? std::min(o->cg_kmax, 16) : 8;
  const int np = std::min(c->n_sys, (int)vmc_ctx::NPOOL);
  // fork: the pool streams wait for everything queued on st so far; join:
  // st waits for the pool.  System si runs on pool[si % np].
  auto fork = [&]() -> int {
    CKC(cudaEventRecord(c->fork_ev, c->st));
    for (int k = 0; k < np; ++k) CKC(cudaStreamWaitEvent(c->pool[k], c->fork_ev, 0));
    return VMC_OK;
  };
  auto join = [&]() -> int {
    for (int k = 0; k < np; ++k) {
      CKC(cudaEventRecord(c->join_ev[k], c->pool[k]));
      CKC(cudaStreamWaitEvent(c->st, c->join_ev[k], 0));
    }
    return VMC_OK;
  };
  TimedRegion tr(c, 2);
  // (1) every system's means, force, S~ and solve, enqueued without a wait.
  // An error stops the enqueueing; the pool is joined back in every case.
  auto enqueue = [&](int si) -> int {
    SysHost &s = c->sys[si];
    SrWork &w = s.sr;
    cudaStream_t st = c->pool[si % np];
    CKC(vmc_sr_means(w, st, &c->n_launch));
    CKC(vmc_sr_build_g(w, st, &c->n_launch));
    CK(build_S_launch(c, s, o->shift_rel, o->shift_abs, st));
    if (c->precision == VMC_MIXED)
      CKC(cudaMemcpyAsync(stg[si].tcstat, s.tc_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    else
      stg[si].tcstat[0] = 0;
    if (ir) {
      if (vmc_sr_ir_launch(w, kmax, eps, st, &c->n_launch)) return VMC_ECUDA;
      if (vmc_sr_ir_fetch(w, stg[si].irflag, stg[si].irsc, st)) return VMC_ECUDA;
    } else {
      if (vmc_sr_cholesky_launch(w, st, &c->n_launch)) return VMC_ECUDA;
      CKC(cudaMemcpyAsync(stg[si].info, w.info, sizeof(int), cudaMemcpyDeviceToHost, st));
    }
    return VMC_OK;
  };
  CK(fork());
  int rq = VMC_OK;
  for (int si = 0; si < c->n_sys && rq == VMC_OK; ++si) rq = enqueue(si);
  CK(join());
  CKC(cudaStreamSynchronize(c->st));
  if (rq != VMC_OK) return rq;
  // (2) systems whose refinement did not converge: FP64 Cholesky (rare)
  int rc = VMC_OK;
  std::vector<int> iters(c->n_sys, 0), fallback(c->n_sys, 0), ok(c->n_sys, 1);
  std::vector<double> relres(c->n_sys, 0.0);
  for (int si = 0; si < c->n_sys; ++si) {
    SysHost &s = c->sys[si];
    if (stg[si].tcstat[0]) {
      ok[si] = 0;
      if (rc == VMC_OK) rc = VMC_ETIMEOUT;
      continue;
    }
    if (ir) {
      if (vmc_sr_ir_eval(stg[si].irflag, stg[si].irsc, &iters[si], &relres[si]) == 1) {
        fallback[si] = 1;
        const int r2 = vmc_sr_cholesky_solve(s.sr, c->st, &c->n_launch);
        if (r2) {
          ok[si] = 0;
          if (rc == VMC_OK) rc = r2;
        }
      }
    } else if (stg[si].info[0]) {
      ok[si] = 0;
      if (rc == VMC_OK) rc = VMC_ESINGULAR;
    }
  }
  // (3) norms for the reports, then the updates of the systems that solved
  auto norms = [&](int si) -> int {
    SrWork &w = c->sys[si].sr;
    cudaStream_t st = c->pool[si % np];
    CKC(vmc_dot_dev(w.g, w.g, w.Np, w.scal + 5, w.dpart, st, &c->n_launch));
    CKC(vmc_dot_dev(w.x, w.x, w.Np, w.scal + 6, w.dpart, st, &c->n_launch));
    CKC(cudaMemcpyAsync(&stg[si].gg, w.scal + 5, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CKC(cudaMemcpyAsync(&stg[si].ebar, w.ebar, sizeof(double), cudaMemcpyDeviceToHost, st));
    return VMC_OK;
  };
  CK(fork());
  for (int si = 0; si < c->n_sys && rq == VMC_OK; ++si)
    if (ok[si]) rq = norms(si);
  CK(join());
  CKC(cudaStreamSynchronize(c->st));
  if (rq != VMC_OK) return rq;
  auto update = [&](int si) -> int {
    SysHost &s = c->sys[si];
    cudaStream_t st = c->pool[si % np];
    CKC(vmc_sr_update_params((double *)s.dev.params, s.sr.x, o->dtau, s.Np, st, &c->n_launch));
    CKC(vmc_launch_expand(&s.dev, st, &c->n_launch));
    return VMC_OK;
  };
  CK(fork());
  for (int si = 0; si < c->n_sys && rq == VMC_OK; ++si) {
    SysHost &s = c->sys[si];
    if (!ok[si]) continue;
    if (!isfinite(stg[si].xx)) {
      if (rc == VMC_OK) rc = VMC_ENUMERIC;
      continue;
    }
    if ((rq = update(si)) != VMC_OK) break;
    s.dirty = true;
    if (reps) {
      vmc_sr_report &r = reps[si];
      r.energy = stg[si].ebar;
      r.norm_g = sqrt(stg[si].gg);
      r.norm_dalpha = o->dtau * sqrt(stg[si].xx);
      r.cg_iters = iters[si];
      r.n_params = s.Np;
      r.rel_residual = relres[si];
      r.fallback = fallback[si];
      r.s_kernel = s.s_kernel;
    }
  }
  CK(join());
  CKC(cudaStreamSynchronize(c->st));
  return rq != VMC_OK ? rq : rc;
}

int vmc_get_params(vmc_ctx *c, int32_t system, double *params) {
  if (!sys_ok(c, system) || !params) return VMC_EINVAL;
  SysHost &s = c->sys[system];
  CKC(cudaMemcpyAsync(params, s.dev.params, sizeof(double) * s.Np, cudaMemcpyDeviceToHost, c->st));
  CKC(cudaStreamSynchronize(c->st));
  return VMC_OK;
}

int vmc_set_params(vmc_ctx *c, int32_t system, const double *params) {
  if (!sys_ok(c, system) || !params) return VMC_EINVAL;
  SysHost &s = c->sys[system];
  for (int k = 0; k < s.Np; ++k)
    if (!isfinite(params[k])) return VMC_EINVAL;
  CKC(cudaMemcpyAsync((double *)s.dev.params, params, sizeof(double) * s.Np, cudaMemcpyHostToDevice, c->st));
  CKC(vmc_launch_expand(&s.dev, c->st, &c->n_launch));
  CKC(cudaStreamSynchronize(c->st));
  s.dirty = true;
  return VMC_OK;
}

int vmc_num_params(vmc_ctx *c, int32_t system) {
  if (!sys_ok(c, system)) return VMC_EINVAL;
  return c->sys[system].Np;
}

int vmc_eval_ratios(vmc_ctx *c, int32_t system, int32_t walker, int32_t n_moves,
                    const int32_t *moves, double *ratios) {
  if (!sys_ok(c, system) || n_moves < 1 || !moves || !ratios) return VMC_EINVAL;
  SysHost &s = c->sys[system];
  if (walker < 0 || walker >= s.W) return VMC_EINVAL;
  CK(ensure_init(c));
  CK(upload_sysdesc(c));
  int *dm = nullptr;
  double *dout = nullptr;
  if (cudaMalloc(&dm, sizeof(int) * 3 * n_moves) != cudaSuccess) return VMC_ENOMEM;
  if (cudaMalloc(&dout, sizeof(double) * n_moves) != cudaSuccess) {
    cudaFree(dm);
    return VMC_ENOMEM;
  }
  int rc = VMC_OK;
  if (cudaMemcpyAsync(dm, moves, sizeof(int) * 3 * n_moves, cudaMemcpyHostToDevice, c->st) ||
      (projected(c) ? vmc_launch_proj_eval(c->d_sys, system, walker, c->precision, n_moves, dm,
                                           dout, c->smem_proj, c->st, &c->n_launch)
                    : vmc_launch_eval_ratios(c->d_sys, system, walker, c->precision, n_moves, dm,
                                             dout, c->smem_sample, c->st, &c->n_launch)) ||
      cudaMemcpyAsync(ratios, dout, sizeof(double) * n_moves, cudaMemcpyDeviceToHost, c->st) ||
      cudaStreamSynchronize(c->st))
    rc = VMC_ECUDA;
  cudaFree(dm);
  cudaFree(dout);
  return rc;
}

int vmc_get_inverse(vmc_ctx *c, int32_t system, int32_t walker, double *minv, double *logabsdet,
                    int32_t *sign) {
  if (!sys_ok(c, system) || projected(c)) return VMC_EINVAL;
  SysHost &s = c->sys[system];
  if (walker < 0 || walker >= s.W) return VMC_EINVAL;
  CK(ensure_init(c));
  const int esize = c->precision == VMC_FP64 ? 8 : 4;
  const size_t mb = ((size_t)s.N * s.ldm * esize + 127) / 128 * 128;
  std::vector<unsigned char> buf(mb), blo(s.dev.minv_lo ? mb : 0);
  CKC(cudaMemcpyAsync(buf.data(), (unsigned char *)s.dev.minv + mb * walker, mb, cudaMemcpyDeviceToHost, c->st));
  if (s.dev.minv_lo)
    CKC(cudaMemcpyAsync(blo.data(), (unsigned char *)s.dev.minv_lo + mb * walker, mb,
                        cudaMemcpyDeviceToHost, c->st));
  double ld = 0.0;
  int sg = 0;
  CKC(cudaMemcpyAsync(&ld, s.dev.logdet + walker, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CKC(cudaMemcpyAsync(&sg, s.dev.detsign + walker, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CKC(cudaStreamSynchronize(c->st));
  if (minv)
    for (int r = 0; r < s.N; ++r)
      for (int k = 0; k < s.N; ++k)
        minv[(size_t)r * s.N + k] =
            esize == 8 ? ((double *)buf.data())[(size_t)r * s.ldm + k]
                       : (double)((float *)buf.data())[(size_t)r * s.ldm + k] +
                             (blo.empty() ? 0.0 : (double)((float *)blo.data())[(size_t)r * s.ldm + k]);
  if (logabsdet) *logabsdet = ld;
  if (sign) *sign = sg;
  return VMC_OK;
}

int vmc_measure_corr(vmc_ctx *c, int32_t system, double *corr, double *ms) {
  if (!sys_ok(c, system) || !corr) return VMC_EINVAL;
  SysHost &s = c->sys[system];
  if (s.dev.n_hidden || projected(c)) return VMC_EINVAL;
  CK(ensure_init(c));
  CK(upload_sysdesc(c));
  const int prec = c->precision == VMC_FP64 ? 0 : 1;
  // the pair-correlation kernel reads the FP32 words only
  const size_t smem_corr = vmc_walker_smem(prec, s.N, s.Ns, s.Np, s.dev.n_hidden, 0, nullptr, 0);
  const int grid = vmc_corr_grid(prec, smem_corr, s.W, s.Ns);
  const size_t ns2 = (size_t)s.Ns * s.Ns;
  const size_t part_b = 3 * ns2 * sizeof(double);
  const size_t cnt_b = (4 * ns2 * sizeof(int) + 255) / 256 * 256;
  const size_t out_b = 6 * ns2 * sizeof(double);
  const size_t need = part_b + cnt_b + out_b;
  if (c->corr_bytes < need) {
    if (c->corr_buf) cudaFree(c->corr_buf);
    c->corr_buf = nullptr;
    c->corr_bytes = 0;
    if (cudaMalloc(&c->corr_buf, need) != cudaSuccess) {
      cudaGetLastError();
      c->corr_buf = nullptr;
      return VMC_ENOMEM;
    }
    c->corr_bytes = need;
  }
  double *part = (double *)c->corr_buf;
  int *cnt = (int *)((unsigned char *)c->corr_buf + part_b);
  double *out = (double *)((unsigned char *)c->corr_buf + part_b + cnt_b);
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  if (ms)
    for (auto &e : ev)
      if (cudaEventCreate(&e) != cudaSuccess) {
        for (auto &f : ev)
          if (f) cudaEventDestroy(f);
        return VMC_ECUDA;
      }
  int rc = VMC_OK;
  if ((ms && cudaEventRecord(ev[0], c->st)) || cudaMemsetAsync(part, 0, part_b, c->st) ||
      vmc_launch_corr_occ(c->d_sys, system, s.Ns, cnt, c->st, &c->n_launch) ||
      (ms && cudaEventRecord(ev[1], c->st)) ||
      vmc_launch_corr(c->d_sys, system, prec, grid, part, smem_corr, c->st, &c->n_launch) ||
      (ms && cudaEventRecord(ev[2], c->st)) ||
      vmc_launch_corr_reduce(part, 1, cnt, s.Ns, s.W, s.dev.lsite, out, c->st, &c->n_launch) ||
      (ms && cudaEventRecord(ev[3], c->st)) ||
      cudaMemcpyAsync(corr, out, out_b, cudaMemcpyDeviceToHost, c->st) ||
      cudaStreamSynchronize(c->st))
    rc = VMC_ECUDA;
  if (ms && rc == VMC_OK) {
    float t1 = 0.f, t2 = 0.f;
    cudaEventElapsedTime(&t1, ev[1], ev[2]);
    cudaEventElapsedTime(&t2, ev[0], ev[3]);
    ms[0] = t1;
    ms[1] = t2;
  }
  for (auto &e : ev)
    if (e) cudaEventDestroy(e);
  return rc;
}

int64_t vmc_kernel_launches(vmc_ctx *c) { return c ? c->n_launch : -1; }

int vmc_sweep_launch(vmc_ctx *c, int32_t *grid, int32_t *ctas_per_sm, int64_t *smem_bytes) {
  if (!c) return VMC_EINVAL;
  const bool pj = projected(c);
  if (grid) *grid = pj ? c->grid_proj : c->grid_sample;
  if (ctas_per_sm)
    *ctas_per_sm = pj ? vmc_proj_occupancy(c->precision, c->smem_proj)
                      : vmc_sample_occupancy(c->precision, c->smem_sample);
  if (smem_bytes) *smem_bytes = (int64_t)(pj ? c->smem_proj : c->smem_sample);
  return VMC_OK;
}

int vmc_test_stall(vmc_ctx *c, int32_t target, int32_t system, int32_t walker) {
  if (!sys_ok(c, system)) return VMC_EINVAL;
  SysHost &s = c->sys[system];
  switch (target) {
    case VMC_STALL_NONE:
      s.dev.stall_walker = -1;
      s.sr.stall = 0;
      return VMC_OK;
    case VMC_STALL_SAMPLE:
      if (walker < 0 || walker >= s.W) return VMC_EINVAL;
      s.dev.stall_walker = walker;
      return VMC_OK;
    case VMC_STALL_S_BUILD:
      if (c->precision != VMC_MIXED) return VMC_EINVAL;
      s.sr.stall = 1;
      return VMC_OK;
    default:
      return VMC_EINVAL;
  }
}

int vmc_lanczos_moments(vmc_ctx *c, int32_t system, double *F1, double *F2, double *moments) {
  if (!sys_ok(c, system) || !moments) return VMC_EINVAL;
  SysHost &s = c->sys[system];
  if (s.dev.n_hidden || s.dev.n_J || projected(c)) return VMC_EINVAL;
  CK(ensure_init(c));
  CK(upload_sysdesc(c));
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int prec = c->precision == VMC_FP64 ? 0 : 1;
  const int grid = std::min(s.W, std::max(1, vmc_lanczos_occupancy(prec, s.Ns)) * nsm);
  const size_t slot = (vmc_lanczos_slot_bytes(prec, s.Ns, s.N) + 255) / 256 * 256;
  const size_t need = slot * grid + sizeof(double) * (2 * (size_t)s.W + 8);
  if (c->lz_bytes < need) {
    if (c->lz_buf) cudaFree(c->lz_buf);
    c->lz_buf = nullptr;
    c->lz_bytes = 0;
    if (cudaMalloc(&c->lz_buf, need) != cudaSuccess) {
      cudaGetLastError();
      return VMC_ENOMEM;
    }
    c->lz_bytes = need;
  }
  double *f1 = (double *)((unsigned char *)c->lz_buf + slot * grid);
  double *f2 = f1 + s.W;
  double *mom = f2 + s.W;
  CKC(vmc_launch_lanczos(c->d_sys, system, prec, s.Ns, grid, c->lz_buf, f1, f2, s.W, mom, c->st,
                         &c->n_launch));
  if (F1) CKC(cudaMemcpyAsync(F1, f1, sizeof(double) * s.W, cudaMemcpyDeviceToHost, c->st));
  if (F2) CKC(cudaMemcpyAsync(F2, f2, sizeof(double) * s.W, cudaMemcpyDeviceToHost, c->st));
  CKC(cudaMemcpyAsync(moments, mom, sizeof(double) * 4, cudaMemcpyDeviceToHost, c->st));
  CKC(cudaStreamSynchronize(c->st));
  return VMC_OK;
}

int vmc_lanczos_alpha(const double *h, double *alpha, double *E1) {
  if (!h || !alpha) return VMC_EINVAL;
  // E_1(t) = (a + b t + c t^2) / (1 + d t + e t^2); dE_1/dt = 0 is
  // (b - a d) + 2 (c - a e) t + (c d - b e) t^2 = 0; the root with the lower E_1
  const double a = h[0], b = h[2] + h[1], cc = h[3], d = 2.0 * h[0], e = h[1];
  auto energy = [&](double t) { return (a + b * t + cc * t * t) / (1.0 + d * t + e * t * t); };
  const double q2 = cc * d - b * e, q1 = 2.0 * (cc - a * e), q0 = b - a * d;
  double best;
  if (fabs(q2) < 1e-300) {
    if (q1 == 0.0) return VMC_ENUMERIC;
    best = -q0 / q1;
  } else {
    const double disc = q1 * q1 - 4.0 * q2 * q0;
    if (!(disc >= 0.0)) return VMC_ENUMERIC;
    const double sq = sqrt(disc);
    const double t1 = (-q1 + sq) / (2.0 * q2), t2 = (-q1 - sq) / (2.0 * q2);
    best = energy(t1) <= energy(t2) ? t1 : t2;
  }
  *alpha = best;
  if (E1) *E1 = energy(best);
  return VMC_OK;
}

int vmc_set_delay(vmc_ctx *c, int32_t k) {
  if (!c || (projected(c) && k > 1)) return VMC_EINVAL;
  return set_delay_impl(c, k);
}

int vmc_set_projection(vmc_ctx *c, int32_t n_ops, const int32_t *perm, const int8_t *sign,
                       const double *weight) {
  if (!c || c->n_sys != 1 || n_ops < 0 || n_ops > VMC_PROJ_MAX_OPS) return VMC_EINVAL;
  SysHost &s = c->sys[0];
  if (n_ops == 0) {
    s.dev.n_ops = 0;
    s.dirty = true;
    return upload_sysdesc(c);
  }
  if (!perm || !sign || !weight || s.dev.n_hidden || c->delay_k > 1) return VMC_EINVAL;
  const int Ns = s.Ns;
  // T_g c^dag_r T_g^-1 = sign[r] c^dag_perm[r]: keep g^-1 and the sign of
  // T_g^-1 on each site, sign[g^-1(q)]
  std::vector<int> inv((size_t)n_ops * Ns);
  std::vector<signed char> isg((size_t)n_ops * Ns);
  for (int g = 0; g < n_ops; ++g) {
    if (!isfinite(weight[g])) return VMC_EINVAL;
    std::vector<char> seen(Ns, 0);
    for (int r = 0; r < Ns; ++r) {
      const int q = perm[(size_t)g * Ns + r];
      const int sg = sign[(size_t)g * Ns + r];
      if (q < 0 || q >= Ns || seen[q] || (sg != 1 && sg != -1)) return VMC_EINVAL;
      seen[q] = 1;
      inv[(size_t)g * Ns + q] = r;
      isg[(size_t)g * Ns + q] = (signed char)sg;
    }
    // the operation must map the local-spin sites onto local-spin sites
    if (!s.lsite.empty())
      for (int r = 0; r < Ns; ++r)
        if (s.lsite[r] != s.lsite[perm[(size_t)g * Ns + r]]) return VMC_EINVAL;
  }
  const int esize = c->precision == VMC_FP64 ? 8 : 4;
  const size_t W = s.W, N = s.N;
  const size_t smem = vmc_proj_smem(c->precision == VMC_FP64 ? 0 : 1, s.N, s.Ns, n_ops);
  int optin = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem > (size_t)optin) return VMC_EINVAL;
  CKC(cudaStreamSynchronize(c->st));
  SysDev &d = s.dev;
  int rc;
  if ((rc = dupload(c, (int **)&d.pinv, inv.data(), inv.size()))) return rc;
  if ((rc = dupload(c, (signed char **)&d.psgn, isg.data(), isg.size()))) return rc;
  if ((rc = dupload(c, (double **)&d.pw, weight, (size_t)n_ops))) return rc;
  if ((rc = dalloc(c, &d.pminv, (size_t)esize * W * n_ops * N * N))) return rc;
  if ((rc = dalloc(c, &d.ppi, sizeof(double) * W * n_ops))) return rc;
  if ((rc = dalloc(c, &d.plog, sizeof(double) * W * n_ops))) return rc;
  if ((rc = dalloc(c, &d.psign, sizeof(int) * W * n_ops))) return rc;
  CKC(vmc_proj_set_smem(smem, c->smem_init));
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int occ = std::max(1, vmc_proj_occupancy(c->precision, smem));
  c->smem_proj = smem;
  c->grid_proj = std::min(c->n_work, nsm * occ);
  d.n_ops = n_ops;
  s.dirty = true;
  CK(upload_sysdesc(c));
  CK(init_with_redraw(c, c->seed ^ 0x2545F4914F6CDD1Dull));
  CKC(cudaStreamSynchronize(c->st));
  return VMC_OK;
}

int32_t vmc_get_delay(vmc_ctx *c) { return c ? c->delay_k : -1; }

int vmc_tune_delay(vmc_ctx *c, int32_t sweeps, const int32_t *cand, int32_t n_cand,
                   int32_t *chosen, double *ms) {
  static const int32_t def[] = {1, 4, 8, 16, 32};
  if (!c || sweeps < 1 || (cand && n_cand < 1) || !chosen || projected(c)) return VMC_EINVAL;
  if (!cand) {
    cand = def;
    n_cand = 5;
  }
  for (int q = 0; q < n_cand; ++q)
    if (cand[q] < 0 || cand[q] > VMC_DELAY_MAX) return VMC_EINVAL;
  CK(ensure_init(c));
  const int prev = c->delay_k;
  // In-sweep recomputes come in bursts and would swamp the timing: they are
  // off while tuning (the accepted-move counts keep running, so walkers that
  // fall due are rebuilt by the next vmc_sample).
  const int rec = c->recompute_every;
  c->recompute_every = 0;
  cudaEvent_t e0, e1;
  CKC(cudaEventCreate(&e0));
  CKC(cudaEventCreate(&e1));
  int best = -1;
  double best_ms = 0.0;
  int rc = VMC_OK;
  for (int q = 0; q < n_cand && rc == VMC_OK; ++q) {
    if (ms) ms[q] = -1.0;
    if (set_delay_impl(c, cand[q]) != VMC_OK) continue;
    cudaEventRecord(e0, c->st);
    rc = vmc_sample(c, 0, 1, sweeps);
    cudaEventRecord(e1, c->st);
    if (rc != VMC_OK) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      rc = VMC_ECUDA;
      break;
    }
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    const double per = (double)t / sweeps;
    if (ms) ms[q] = per;
    if (best < 0 || per < best_ms) {
      best = cand[q];
      best_ms = per;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->recompute_every = rec;
  if (rc != VMC_OK || best < 0) {
    set_delay_impl(c, prev);
    return rc != VMC_OK ? rc : VMC_EINVAL;
  }
  *chosen = best;
  return set_delay_impl(c, best);
}

int vmc_set_proposal_batch(vmc_ctx *c, int32_t b) {
  if (!c || b < 1 || b > VMC_SPEC_MAX) return VMC_EINVAL;
  for (auto &s : c->sys) s.dev.spec_b = b;
  c->spec_b = b;
  return VMC_OK;
}

int32_t vmc_get_proposal_batch(vmc_ctx *c) { return c ? c->spec_b : -1; }

int vmc_tune_proposal_batch(vmc_ctx *c, int32_t sweeps, const int32_t *cand, int32_t n_cand,
                            int32_t *chosen, double *ms) {
  static const int32_t def[] = {1, 2, 4, 8};
  if (!c || sweeps < 1 || (cand && n_cand < 1) || !chosen || projected(c)) return VMC_EINVAL;
  if (!cand) {
    cand = def;
    n_cand = 4;
  }
  for (int q = 0; q < n_cand; ++q)
    if (cand[q] < 1 || cand[q] > VMC_SPEC_MAX) return VMC_EINVAL;
  CK(ensure_init(c));
  const int prev = c->spec_b;
  // as in vmc_tune_delay: no periodic rebuilds while timing
  const int rec = c->recompute_every;
  c->recompute_every = 0;
  cudaEvent_t e0, e1;
  CKC(cudaEventCreate(&e0));
  CKC(cudaEventCreate(&e1));
  int best = -1;
  double best_ms = 0.0;
  int rc = VMC_OK;
  for (int q = 0; q < n_cand && rc == VMC_OK; ++q) {
    if (ms) ms[q] = -1.0;
    vmc_set_proposal_batch(c, cand[q]);
    cudaEventRecord(e0, c->st);
    rc = vmc_sample(c, sweeps, 0, 0);
    cudaEventRecord(e1, c->st);
    if (rc != VMC_OK) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      rc = VMC_ECUDA;
      break;
    }
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    const double per = (double)t / sweeps;
    if (ms) ms[q] = per;
    if (best < 0 || per < best_ms) {
      best = cand[q];
      best_ms = per;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->recompute_every = rec;
  if (rc != VMC_OK || best < 0) {
    vmc_set_proposal_batch(c, prev);
    return rc != VMC_OK ? rc : VMC_EINVAL;
  }
  *chosen = best;
  return vmc_set_proposal_batch(c, best);
}

int vmc_enable_timing(vmc_ctx *c, int32_t on) {
  if (!c) return VMC_EINVAL;
  collect_times(c);
  c->timing = on != 0;
  return VMC_OK;
}

int vmc_kernel_times(vmc_ctx *c, double *ms, int64_t *count) {
  if (!c || !ms || !count) return VMC_EINVAL;
  collect_times(c);
  for (int k = 0; k < 4; ++k) {
    ms[k] = c->ms[k];
    count[k] = c->cnt[k];
    c->ms[k] = 0.0;
    c->cnt[k] = 0;
  }
  return VMC_OK;
}

}  // extern "C"
