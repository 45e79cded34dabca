// Shared declarations of the CUDA path (device structures, Philox, launch
// wrappers).  Used only by the library's own translation units.
#pragma once

#include <cuda_runtime.h>
#include "../../include/vmc.h"
#include <stdint.h>

#define VMC_NT 128          // threads per walker CTA (one per row of M^-1)
#define VMC_MAX_N 128       // N = Ne/2 limit of the walker kernels
#define VMC_ACC_MAX 2048    // O-row accumulator kept in shared memory up to this Np

// Per-walker status bits.
#define VMC_ST_SINGULAR 1
#define VMC_ST_NUMERIC 2
#define VMC_ST_ILLCOND 4     // min/max |pivot| of the last from-scratch inverse below 1e-12
#define VMC_ST_TIMEOUT 8     // a bounded wait on a bulk copy expired

// One system of a (possibly batched) context, as the kernels see it.  All
// pointers are device pointers.
struct SysDev {
  int Ns, Ne, N, ldm;          // ldm: row stride of M^-1 (odd, >= N)
  int n_hop, n_V, n_J, local_spin;
  const signed char *lsite;    // [Ns] 1 = site with exactly one electron (Kondo local spin), or NULL
  unsigned long long pex;      // exchange iff r0 < pex (pex <= 2^32)
  int Np, n_g, n_v, n_f, ldO;
  int W;                       // walkers
  int sys_index;               // system index (Philox counter word 3)
  int n_samples;               // sample rows per walker in the buffers
  int acc_len;                 // O-row accumulator length in shared memory (0 = global)
  const int *hop_i, *hop_j;
  const double *hop_t;
  const int *tgt_ptr;          // [Ns+1] hopping terms grouped by target site i (CSR)
  const int *tgt_term;         // [n_hop] term indices
  const int *tgt_j;            // [n_hop] source site of each grouped term
  const double *tgt_t;         // [n_hop] its t
  double *tgt_v64;             // [n_hop] v(j, i) of each grouped term (refreshed with v)
  float *tgt_v32;
  const double *U;
  const int *V_i, *V_j;
  const double *V_val;
  const int *J_i, *J_j;
  const int *jptr;              // [Ns + 1] exchange terms by site (CSR)
  const int2 *jadj;            // [2 n_J] {term, other site} of each site's terms
  const double *J_val;
  const int *g_idx, *v_idx, *f_idx;
  const signed char *f_sign;
  const int *fcode;            // [Ns*Ns] 2 f_idx + (f_sign < 0), or -1 (no parameter)
  const int *vptr;             // [n_v + 1] Jastrow class -> its site pairs (CSR)
  const unsigned *vpair;       // i | j << 16, i < j, grouped by class
  const double *params;
  double *f64, *fT64;          // expanded f_ij and its transpose [Ns*Ns]
  float *f32, *fT32;
  double *vmat;                // v_ij [Ns*Ns]
  double *gsite;               // g_i [Ns]
  float *vmat32, *gsite32;     // FP32 copies (mixed form)
  // walker state
  int *ele;                    // [W*Ne]
  int *occ;                    // [W*2*Ns]: occ[s*Ns + i] = label or -1
  void *minv;                  // [W*N*ldm] (double or float)
  float *minv_lo;              // mixed form: low words of the double-float M^-1, same layout
  int rebuild_df;              // mixed form: from-scratch inverses in double-float (opt-in)
  void *jf;                    // [W*Ns] Jastrow field sum_{j != i} v_ij (n_j - 1) (double or float)
  unsigned long long *ctr;     // [W] Philox proposal counters
  double *logdet;              // [W]
  int *detsign;                // [W]
  double *E;                   // [W*n_samples]
  void *O;                     // [W*n_samples*ldO] (double or float)
  long long *n_prop, *n_acc;   // [W]
  long long *cnt;              // [W*8]: valid hops, valid exchanges, accepted hops, accepted
                               // exchanges, measured hop ratios, measured exchange ratios, samples
  long long *n_rec;            // [W] periodic from-scratch inverses
  int *acc_since;              // [W] accepted moves since the last FP64 inverse
  int *status;                 // [W]
  double *drift;               // [W]
  int recompute_every;         // accepted moves between FP64 from-scratch inverses (0 = never)
  int delay_k;                 // pending delayed updates before a flush (<= 1: immediate)
  int stall_walker;            // test hook: this walker's copy is not issued (-1: none)
  int spec_b;                  // proposals formed together by the sweep (<= 1: one at a time)
  // quantum-number projection (Sec. 3.2.2): n_ops operations g (0 = none)
  int n_ops;
  const int *pinv;             // [n_ops*Ns] g^-1(site)
  const signed char *psgn;     // [n_ops*Ns] sign of T_g^-1 on that site
  const double *pw;            // [n_ops] weights w_g
  void *pminv;                 // [W*n_ops*N*N] M_g^-1 (double or float), row-major, ld N
  double *ppi;                 // [W*n_ops] shares pi_g of the projected amplitude
  double *plog;                // [W*n_ops] log|A_g| of the last from-scratch build
  int *psign;                  // [W*n_ops] sign of A_g (0: M_g singular)
  // MLP correlation factor exp(w2 . tanh(W1 n + b1) + b2) (H = 0: absent);
  // params hold [W1 (H x 2Ns) | b1 | w2 | b2] after the pair orbitals.
  int n_hidden;
  int mlp_base;
  double *W1T64;               // [2Ns][H] FP64 (column c of W1 contiguous)
  void *W1T16;                 // [2Ns][H] BF16 copy (mixed form)
  void *hmlp;                  // [W][H] pre-activations h = W1 n + b1 (double or float)
};

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its published
// definition: ten rounds of two 32x32->64 multiplies with a Weyl key schedule.
__device__ __forceinline__ uint4 vmc_philox(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ int vmc_mulhi(uint32_t r, int n) {
  return (int)(((unsigned long long)r * (unsigned long long)n) >> 32);
}

// ---- launch wrappers (defined in vmc_walker.cu / vmc_sr.cu) ----
// All return cudaError_t from the launch; they count launches in *n_launch.
cudaError_t vmc_launch_expand(const SysDev *h_sys, cudaStream_t st, long long *n_launch);
cudaError_t vmc_launch_init(const SysDev *d_sys, const int2 *d_work, int n_work, int *d_ctr,
                            int precision, int only_due, int due_threshold, size_t smem,
                            cudaStream_t st, long long *nl);
cudaError_t vmc_launch_sample(const SysDev *d_sys, const int2 *d_work, int n_work,
                              int *d_work_ctr, int precision, uint64_t seed,
                              int n_first, int n_samples, int sweeps_between,
                              int sample_base, int grid, size_t smem,
                              cudaStream_t st, long long *n_launch);
cudaError_t vmc_launch_eval_ratios(const SysDev *d_sys, int sys, int walker,
                                   int precision, int n_moves, const int *d_moves,
                                   double *d_out, size_t smem, cudaStream_t st,
                                   long long *n_launch);
// Pair correlations (measurement mode): CTA count of k_corr (occupancy x SMs,
// at most W), the ratio kernel (adds into FP64 planes [3][Ns][Ns]), the
// occupation-count kernel (int [4][Ns][Ns]) and the reduction into
// double [6][Ns][Ns].
int vmc_corr_grid(int precision, size_t smem, int W, int Ns);
cudaError_t vmc_launch_corr(const SysDev *d_sys, int sys, int precision, int grid,
                            double *part, size_t smem, cudaStream_t st, long long *n_launch);
cudaError_t vmc_launch_corr_occ(const SysDev *d_sys, int sys, int Ns, int *cnt,
                                cudaStream_t st, long long *n_launch);
cudaError_t vmc_launch_corr_reduce(const double *part, int n_part, const int *cnt, int Ns,
                                   int W, const signed char *lsite, double *out, cudaStream_t st,
                                   long long *n_launch);
// with_lo: the mixed form's sweep keeps the low words of its double-float
// M^-1 in shared memory as well (the pair-correlation kernel does not).
size_t vmc_walker_smem(int precision, int N, int Ns, int Np, int H, int kd, int *acc_len,
                       int with_lo);
size_t vmc_init_smem(int N, int Ns);
int vmc_sample_occupancy(int precision, size_t smem);
// the mixed form's 168-register sweep variant (vmc_sweep3.cu)
int vmc_sample_occupancy_v3(size_t smem);
cudaError_t vmc_sample_set_smem_v3(size_t s32);
cudaError_t vmc_launch_sample_v3(const SysDev *d_sys, const int2 *d_work, int n_work,
                                 int *d_work_ctr, uint2 key, int n_first, int n_samples,
                                 int sweeps_between, int sample_base, int grid, size_t smem,
                                 cudaStream_t st, long long *nl);
cudaError_t vmc_walker_set_smem_limits(size_t smem_sample64, size_t smem_sample32,
                                       size_t smem_init);

// Projected wave function (vmc_proj.cu)
size_t vmc_proj_smem(int precision, int N, int Ns, int n_ops);
int vmc_proj_occupancy(int precision, size_t smem);
cudaError_t vmc_proj_set_smem(size_t s_sample, size_t s_build);
cudaError_t vmc_launch_proj_build(const SysDev *d_sys, const int2 *d_work, int n_work, int n_ops,
                                  int precision, int only_due, int due_threshold, size_t smem,
                                  cudaStream_t st, long long *n_launch);
cudaError_t vmc_launch_proj_sample(const SysDev *d_sys, const int2 *d_work, int n_work,
                                   int *d_work_ctr, int precision, uint64_t seed, int n_first,
                                   int n_samples, int sweeps_between, int sample_base, int grid,
                                   size_t smem, cudaStream_t st, long long *n_launch);
cudaError_t vmc_launch_proj_eval(const SysDev *d_sys, int sys, int walker, int precision,
                                 int n_moves, const int *d_moves, double *d_out, size_t smem,
                                 cudaStream_t st, long long *n_launch);

// First-step power-Lanczos local values and moments (vmc_lanczos.cu): table
// slot bytes per CTA, and the launch (k_lanczos over the walkers, then the
// four walker means into moments[4]).
int vmc_lanczos_occupancy(int precision, int Ns);
size_t vmc_lanczos_slot_bytes(int precision, int Ns, int N);
cudaError_t vmc_launch_lanczos(const SysDev *d_sys, int sys, int precision, int Ns, int grid,
                               void *slots, double *F1, double *F2, int W, double *moments,
                               cudaStream_t st, long long *n_launch);

// SR (vmc_sr.cu)
struct SrWork {
  int Np, rows, ldO;
  int precision;               // layout of O: 0 double, 1 float
  const void *O;
  const double *E;
  double *obar;                // [Np]
  double *ebar;                // [1] (+ scratch)
  double *S;                   // [Np*Np]
  double *g;                   // [Np]
  double *diagS;               // [Np]
  double *x, *r, *p, *w, *t;   // CG vectors (t: [rows])
  double *scal;                // device scalars
  int *info;                   // device status
  double *dblk;                // [32*32] factored diagonal block in flight (Cholesky)
  double *part;                // column-reduction partials [vmc_colreduce_parts(rows, Np) * Np]
  float *vf, *tf;              // FP32 copies of the SR-CG vectors (mixed form) [Np], [rows]
  double *dpart;               // dot-product partials [512]
  void *chol_graph;            // cudaGraphExec_t of the Cholesky factor + solve (lazily built)
  // mixed-precision iterative refinement (vmc_sr_mixed.cu)
  float *S32;                  // [Np*Np] scaled S~, inverted in place
  float *gjP, *gjC;            // [32*32] pivot-block inverse, [Np*32] column block
  float *rs32;                 // [Np] scaled residual
  double *dsc;                 // [Np] S~_kk^-1/2
  int *irflag;                 // [4] converged, unusable, steps
  void *ir_graph;
  int ir_iter;
  double ir_eps;
  int stall;                   // test hook: CTA 0 of the next tensor-core S build waits on a
                               // barrier nothing arrives on (then no copy or MMA is issued)
};
int vmc_colreduce_parts(int rows, int Np);
cudaError_t vmc_sr_means(const SrWork &w, cudaStream_t st, long long *nl);
cudaError_t vmc_sr_build_S(const SrWork &w, double shift_rel, double shift_abs,
                           cudaStream_t st, long long *nl);
cudaError_t vmc_sr_build_g(const SrWork &w, cudaStream_t st, long long *nl);
cudaError_t vmc_sr_diag(const SrWork &w, cudaStream_t st, long long *nl);
int vmc_sr_cholesky_solve(SrWork &w, cudaStream_t st, long long *nl);
void vmc_sr_release(SrWork &w);
int vmc_sr_ir_solve(SrWork &w, int max_iter, double eps, int *iters, double *rel_res,
                    cudaStream_t st, long long *nl);
int vmc_sr_ir_launch(SrWork &w, int max_iter, double eps, cudaStream_t st, long long *nl);
int vmc_sr_ir_fetch(const SrWork &w, int *flags4, double *scal3, cudaStream_t st);
int vmc_sr_ir_eval(const int *fl, const double *sc, int *iters, double *rel_res);
int vmc_sr_cholesky_launch(SrWork &w, cudaStream_t st, long long *nl);
cudaError_t vmc_dot_dev(const double *a, const double *b, int n, double *out_dev, double *dpart,
                        cudaStream_t st, long long *nl);
void vmc_sr_ir_release(SrWork &w);
int vmc_sr_cg_solve(const SrWork &w, double shift_rel, double shift_abs, double eps,
                    int kmax, int *iters, cudaStream_t st, long long *nl, int dense);
void vmc_tc_dims(int rows, int Np, int *ldK, int *Np_pad);
int vmc_tc_tile_list(int Np, int2 *out);
// which (may be NULL) receives the kernel that built S: VMC_S_KERNEL_TMA or
// VMC_S_KERNEL_TILES (include/vmc.h).
cudaError_t vmc_sr_build_S_tc(const SrWork &w, void *hi, void *lo, int *status, double shift_rel,
                              double shift_abs, const int2 *tiles, cudaStream_t st, long long *nl,
                              int *which);
cudaError_t vmc_sr_update_params(double *params, const double *x, double dtau, int Np,
                                 cudaStream_t st, long long *nl);
cudaError_t vmc_dot_host(const double *a, const double *b, int n, double *out_host,
                         double *d_scratch, cudaStream_t st, long long *nl);
