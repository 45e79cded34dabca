/*
 * vmc.h - C ABI of the GB300 many-variable VMC hot path.
 *
 * The library samples a Gutzwiller-Jastrow projected anti-parallel Pfaffian
 * wave function  psi(x) = P_G P_J <x|phi_AP-Pf>  (mVMC paper, Sec. 3.2:
 * Eqs. Pf, AP-Pf and the correlation factors of Sec. 3.2.3) with many
 * Metropolis walkers (Sec. 3.1.1-3.1.2), measures the local energy and the
 * log-derivatives O_k (Eq. MC, Sec. 3.3.1), and performs stochastic
 * reconfiguration steps (Eq. SR_equation_system, Sec. 3.3.2, Algorithm 1).
 * One GPU; every numerical step runs in the library's own CUDA kernels.
 *
 * Conventions
 *  - Sites i = 0..Ns-1; electrons: Ne = 2N with S^z = 0; ele[n] (n < N) is
 *    the site of up electron n, ele[N+m] the site of down electron m.
 *    Labels are kept through every move.
 *  - Hamiltonian (Sec. 2.3, Eq. GHam and the Hubbard / Spin models):
 *      H = sum_k -t_k c^dag_{i_k s} c_{j_k s}  (each directed term, both spins)
 *        + sum_i U_i n_i,up n_i,dn + sum_k V_k n_{i_k} n_{j_k}
 *        + sum_k J_k S_{i_k} . S_{j_k}.
 *  - Parameters: one real vector [g (n_g) | v (n_v) | f (n_f) | mlp]:
 *      g_i  = p[g_idx[i]]                (0 where g_idx = -1)
 *      v_ij = p[n_g + v_idx[i*Ns+j]]     (v_idx symmetric, -1 = absent)
 *      f_ij = f_sign[i*Ns+j] * p[n_g + n_v + f_idx[i*Ns+j]]
 *    (sublattice classes and anti-periodic signs, Sec. 3.2.1 and App. A).
 *    With n_hidden = H > 0 the wave function carries a learned correlation
 *    factor exp(w2 . tanh(W1 n + b1) + b2) (not in the paper) on the
 *    spin-resolved occupations n_c, c = i + Ns*spin; its H*2Ns + 2H + 1
 *    parameters follow f as [W1 (H x 2Ns, row-major) | b1 (H) | w2 (H) | b2].
 *    The plain form evaluates it in FP64, the mixed form with BF16 W1 and
 *    FP32 arithmetic.
 *  - Ownership: every pointer argument is a HOST pointer owned by the caller
 *    and only read (or written, for outputs) during the call; the library
 *    copies what it keeps.  Device memory is allocated by the library in
 *    vmc_create and released by vmc_destroy.
 *  - Every call returns VMC_OK (0) or a negative error code; on error the
 *    context is left as it was before the call, except after VMC_ECUDA
 *    (the CUDA context may be unusable) and VMC_ENUMERIC / VMC_ESINGULAR
 *    from vmc_sample (the affected walkers are flagged, see vmc_measure).
 *  - Calls on one context are not thread-safe; all work is ordered on the
 *    stream given in vmc_opts.
 */
#ifndef VMC_H
#define VMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  VMC_OK = 0,
  VMC_EINVAL = -1,     /* bad argument or size */
  VMC_ENOMEM = -2,     /* device or host allocation failed */
  VMC_ECUDA = -3,      /* a CUDA call failed */
  VMC_ESINGULAR = -4,  /* an initial configuration has Pf(X) = 0 */
  VMC_ENUMERIC = -5,   /* NaN/Inf or a vanishing ratio denominator */
  VMC_ETIMEOUT = -6,   /* a bounded device wait expired */
  VMC_ESTATE = -7      /* call not valid in the current state */
};

enum { VMC_FP64 = 0, VMC_MIXED = 1 };
/* SR solvers: dense S~ + Cholesky; CG (Algorithm 1) with the SR-CG product
 * from the sample matrix (S never formed); CG with the dense S~ built by the
 * GEMM (tensor cores in the mixed form); dense S~ solved by iterative
 * refinement in FP64 (residuals and solution) with an FP32 inverse of the
 * Jacobi-scaled S~ as the correction operator, falling back to the FP64
 * Cholesky when the residual target is not met (not in the paper: the
 * O(Np^3) part in FP32, the result to FP64 residual). */
enum { VMC_SOLVE_CHOLESKY = 0, VMC_SOLVE_CG = 1, VMC_SOLVE_CG_DENSE = 2,
       VMC_SOLVE_MIXED_IR = 3 };

typedef struct vmc_ctx vmc_ctx;

/* Lattice and Hamiltonian of one system (host arrays, copied). */
typedef struct {
  int32_t Ns;
  int32_t n_hop;                 /* directed hopping terms -t c^dag_i c_j */
  const int32_t *hop_i, *hop_j;
  const double *hop_t;
  const double *U;               /* [Ns] on-site U_i (may be NULL = 0) */
  int32_t n_V;                   /* off-site V n_i n_j terms */
  const int32_t *V_i, *V_j;
  const double *V_val;
  int32_t n_J;                   /* Heisenberg bonds J S_i.S_j, each once */
  const int32_t *J_i, *J_j;
  const double *J_val;
  int32_t local_spin;            /* 1: no doublons (g -> -inf), exchange moves only */
  const int8_t *local_site;      /* [Ns] or NULL.  1 marks a site that holds exactly one
                                    electron: a local spin of the Kondo lattice (Sec. 2.3
                                    Kondo model, Sec. 4.2), with double occupancy excluded
                                    and no empty state.  Hops never enter or leave a marked
                                    site; only exchanges change its spin.  0 elsewhere. */
} vmc_model;

/* Variational-parameter layout of one system (host arrays, copied). */
typedef struct {
  int32_t n_g, n_v, n_f;
  const int32_t *g_idx;          /* [Ns] */
  const int32_t *v_idx;          /* [Ns*Ns], symmetric, diagonal -1 */
  const int32_t *f_idx;          /* [Ns*Ns] */
  const int8_t *f_sign;          /* [Ns*Ns], +1 / -1 */
  int32_t n_hidden;              /* MLP hidden units H (0 = no MLP factor, <= 4096) */
} vmc_layout;

typedef struct {
  int32_t n_walkers;             /* walkers per system (>= 1) */
  uint64_t seed;                 /* Philox4x32-10 key */
  int32_t precision;             /* VMC_FP64 or VMC_MIXED */
  int32_t delay_k;               /* delayed-update depth k of the sweep (0 or 1 =
                                    immediate updates, 2..VMC_DELAY_MAX); see
                                    vmc_set_delay */
  int32_t recompute_every;       /* FP64 from-scratch inverse between sweep launches
                                    once a walker has this many accepted moves since
                                    the last one (the one after a vmc_sample call's
                                    last launch runs when an inverse is next read,
                                    and is dropped when a parameter change rebuilds
                                    every walker first); 0 = default (mixed: 64,
                                    FP64: never), -1 = never */
  int32_t max_samples;           /* sample rows kept per walker (>= 1) */
  void *stream;                  /* cudaStream_t; NULL = default stream */
  int32_t rebuild;               /* from-scratch inverses of the mixed form:
                                    VMC_REBUILD_FP64 (0, default: FP64 Gauss-Jordan)
                                    or VMC_REBUILD_DOUBLE_FLOAT (Gauss-Jordan on
                                    hi + lo FP32 words, about 2^-46 rounding, the
                                    precision of the sweep's updates; faster on a
                                    part whose FP64 rate is 1/64 of FP32).  The
                                    FP64 form always rebuilds in FP64. */
} vmc_opts;
enum { VMC_REBUILD_FP64 = 0, VMC_REBUILD_DOUBLE_FLOAT = 1 };

typedef struct {
  double energy;                 /* mean local energy over the stored samples */
  double variance;               /* sample variance of E_loc */
  double stderr_walkers;         /* standard error from per-walker means */
  double acceptance;             /* accepted / proposals, cumulative */
  int64_t n_proposals, n_accepted;
  int32_t n_samples;             /* stored rows (walkers x samples) */
  int32_t n_flagged;             /* walkers with a numerical fault, or skipped by the last
                                    vmc_sample because a bounded wait expired */
  double max_drift;              /* max |Minv_updated - Minv_fresh| / max |Minv_fresh|
                                    seen at the in-sweep FP64 recomputes */
  int64_t n_hop_tested;          /* valid hop proposals whose ratio was computed */
  int64_t n_exchange_tested;     /* valid exchange proposals whose ratio was computed */
  int64_t n_hop_accepted;
  int64_t n_exchange_accepted;
  int64_t n_recomputes;          /* in-sweep FP64 from-scratch inverses */
  int64_t n_measured_hops;       /* hop ratios evaluated for E_loc */
  int64_t n_measured_exchanges;  /* exchange ratios evaluated for E_loc */
  int64_t n_measurements;        /* E_loc / O_k rows measured */
} vmc_stats;

typedef struct {
  double dtau;                   /* Delta tau of Eq. SR_equation_system */
  double shift_rel;              /* S~_kk = S_kk (1 + shift_rel) + shift_abs */
  double shift_abs;
  int32_t solver;                /* VMC_SOLVE_* */
  double cg_eps;                 /* Algorithm 1 / refinement: stop when |r| < eps |b| */
  int32_t cg_kmax;               /* Algorithm 1: iteration limit; refinement:
                                    min(cg_kmax, 16) steps */
} vmc_sr_opts;

typedef struct {
  double energy;                 /* <H> of the samples used */
  double norm_g;                 /* |g|_2 */
  double norm_dalpha;            /* |Delta alpha|_2 */
  int32_t cg_iters;              /* iterations used (CG or refinement), 0 for Cholesky */
  int32_t n_params;
  double rel_residual;           /* refinement: |g - S~ x| / |g| reached (else 0) */
  int32_t fallback;              /* refinement: 1 if the FP64 Cholesky solved instead */
  int32_t s_kernel;              /* kernel that built the dense S~: VMC_S_KERNEL_* */
} vmc_sr_report;

/* vmc_sr_report.s_kernel: no dense S~ (SR-CG product); FP64 SIMT product
 * (plain form); persistent TMA-fed tcgen05 kernel (mixed form); one CTA per
 * tile tcgen05 kernel with cp.async staging (mixed form, used when the
 * driver's tensor-map encoder is unavailable or VMC_TC_KERNEL=tiles is set). */
enum { VMC_S_KERNEL_NONE = 0, VMC_S_KERNEL_FP64 = 1, VMC_S_KERNEL_TMA = 2,
       VMC_S_KERNEL_TILES = 3 };

/* Create a context for one system (the problem statement of Sec. 2.3: the
 * Hamiltonian, and the variational wave function of Sec. 3.2).
 * The sector is S^z = 0 (Ne/2 up and Ne/2 down electrons, the anti-parallel
 * pair product of Eq. AP-Pf); there is no argument for another S^z.
 * params: initial parameter vector [n_g + n_v + n_f (+ MLP block)].  p_exchange: the
 * probability that a proposal is an exchange (Sec. 3.1.2); forced to 1 when
 * local_spin.  Walker configurations start from a seeded random placement;
 * vmc_set_configs replaces them.
 * Errors: VMC_EINVAL (sizes, Ne odd, Ne/2 > 128, Ns > 4096, index out of
 * range, local_site entries other than 0/1, or marked sites that Ne/2 up and
 * Ne/2 down electrons cannot fill one each), VMC_ENOMEM, VMC_ECUDA. */
int vmc_create(vmc_ctx **out, const vmc_model *model, int32_t Ne,
               const vmc_layout *layout, const double *params,
               double p_exchange, const vmc_opts *opts);

/* Batched form: n_systems independent systems (uneven sizes allowed) sampled
 * by one persistent launch.  Arrays are indexed by system. */
int vmc_create_batch(vmc_ctx **out, int32_t n_systems, const vmc_model *models,
                     const int32_t *Ne, const vmc_layout *layouts,
                     const double *const *params, const double *p_exchange,
                     const vmc_opts *opts);

void vmc_destroy(vmc_ctx *ctx);
const char *vmc_strerror(int code);

/* Replace the walkers' configurations of one system: ele [n_walkers*Ne]
 * (label order, see above), counters [n_walkers] Philox proposal counters
 * (NULL = keep).  Inverses are rebuilt from scratch (FP64) on the next
 * vmc_sample.  Errors: VMC_EINVAL (out-of-range or doubly occupied spin
 * orbital; doublon under local_spin; a local_site not holding exactly one
 * electron). */
int vmc_set_configs(vmc_ctx *ctx, int32_t system, const int32_t *ele,
                    const uint64_t *counters);
int vmc_get_configs(vmc_ctx *ctx, int32_t system, int32_t *ele,
                    uint64_t *counters);

/* Markov chains (Sec. 3.1.1-3.1.2): every walker makes n_warmup sweeps,
 * then n_samples times (sweeps_between sweeps, then a measurement of E_loc
 * and the O_k row).  One sweep = Ne proposals.  Replaces the stored
 * samples (n_samples <= max_samples).  Errors: VMC_EINVAL, VMC_ESINGULAR
 * (a walker's X is singular), VMC_ENUMERIC, VMC_ECUDA. */
int vmc_sample(vmc_ctx *ctx, int32_t n_warmup, int32_t n_samples,
               int32_t sweeps_between);

/* Statistics of the stored samples of one system (Eq. MC) and counters. */
int vmc_measure(vmc_ctx *ctx, int32_t system, vmc_stats *out);

/* Equal-time pair correlations of the walkers' CURRENT configurations (the
 * physical-quantity mode of Sec. 2.2.3, NVMCCalMode = 1): for every kind and
 * site pair (i, j), the mean over the system's walkers of the local
 * estimator of Eq. MC, A_loc(x) = <psi|A|x> / <psi|x> (A acting on the ket),
 *   kind 0  c^dag_{i up} c_{j up}         kind 3  S^z_i S^z_j
 *   kind 1  c^dag_{i dn} c_{j dn}         kind 4  S^+_i S^-_j
 *   kind 2  n_i n_j                       kind 5  S_i . S_j
 * with n_i = n_i,up + n_i,dn, S^z_i = (n_i,up - n_i,dn)/2,
 * S^+_i = c^dag_{i up} c_{i dn}.  Averaging the results of calls between
 * vmc_sample calls gives the Monte Carlo estimate of <A>; the structure
 * factors of Sec. 2.4.2 (n_sigma(k), N(k), S^z(k), S(k)) and the doublon
 * density and nearest-neighbour spin correlation of Sec. 4.1.1 follow from
 * these matrices.  With local_site marks (Kondo local spins), a hop into or
 * out of a marked site leaves the constrained space, where psi = 0, so those
 * entries of kinds 0 and 1 are 0.  Hops and spin swaps are evaluated from the walker's
 * M^-1 in the context's precision (FP64, or FP32 in the mixed form), the
 * diagonal kinds are exact; the walker means are FP64 (summed by atomic
 * adds, so their last bit may differ between calls).
 * corr: host [6 * Ns * Ns], layout [kind][i][j] row-major.  ms: NULL or
 * host [2]: the device milliseconds of the ratio kernel and of the whole
 * measurement (CUDA events on the context's stream).  Rebuilds walker
 * inverses first if parameters or configurations changed.  Device scratch
 * (88 Ns^2 bytes) is kept by the context.  Errors: VMC_EINVAL (bad system, NULL corr, or a context
 * with the MLP factor, which this measurement does not evaluate),
 * VMC_ESINGULAR, VMC_ENOMEM, VMC_ECUDA. */
int vmc_measure_corr(vmc_ctx *ctx, int32_t system, double *corr, double *ms);

/* Copy the stored samples of one system to host buffers: E [rows],
 * O [rows * Np] row-major, row = walker * n_samples + sample.  Either
 * pointer may be NULL. */
int vmc_get_samples(vmc_ctx *ctx, int32_t system, double *E, double *O);

/* Replace the stored samples of one system with caller data (rows x Np,
 * row-major); rows <= n_walkers * max_samples.  vmc_sr_step then uses them. */
int vmc_set_samples(vmc_ctx *ctx, int32_t system, int32_t rows,
                    const double *E, const double *O);

/* One SR step on the stored samples of one system (Sec. 3.3.1-3.3.2):
 * S_km = <O_k O_m> - <O_k><O_m>, g_m = <E O_m> - <E><O_m>,
 * S~ = S with diagonal shift, solve S~ x = g by Cholesky (S~ = L L^T), by
 * CG (Algorithm 1) with the SR-CG product or the dense S~, or by mixed-precision
 * iterative refinement, alpha += -dtau x.  Walker
 * inverses are rebuilt on the next vmc_sample.  Errors: VMC_EINVAL,
 * VMC_ESTATE (no samples), VMC_ESINGULAR (S~ not positive definite),
 * VMC_ENUMERIC (CG breakdown), VMC_ECUDA. */
int vmc_sr_step(vmc_ctx *ctx, int32_t system, const vmc_sr_opts *opts,
                vmc_sr_report *report);

/* One SR step for every system of the context with the same options
 * (Sec. 3.3.1-3.3.2, as vmc_sr_step), for batches of independent systems:
 * the work of all systems is enqueued before the host waits, so a batch of
 * small systems costs two synchronisations instead of several per system.
 * reports: NULL or n_sys entries (index = system).  With VMC_SOLVE_CHOLESKY
 * and VMC_SOLVE_MIXED_IR the systems are solved together; with the CG
 * solvers (their loop reads a convergence flag on the host) the call is
 * vmc_sr_step for each system in turn.  Every system with samples is stepped
 * even if another fails; the return value is the first error (VMC_ESTATE if
 * a system has no samples, before any work).  Results equal vmc_sr_step's. */
int vmc_sr_step_all(vmc_ctx *ctx, const vmc_sr_opts *opts, vmc_sr_report *reports);

/* S~ (Np x Np, row-major, FP64) and g (Np) of the stored samples, as built
 * by vmc_sr_step's dense path (for checks).  Either pointer may be NULL. */
int vmc_get_sr_matrices(vmc_ctx *ctx, int32_t system, double shift_rel,
                        double shift_abs, double *S, double *g);

int vmc_get_params(vmc_ctx *ctx, int32_t system, double *params);
int vmc_set_params(vmc_ctx *ctx, int32_t system, const double *params);
int vmc_num_params(vmc_ctx *ctx, int32_t system);

/* Pfaffian-ratio check hook (Sec. 3.1.2 fast update): for walker w of a
 * system, psi(x')/psi(x) of n_moves candidate moves of its current
 * configuration, each moves[3k..3k+2] = {kind, a, b}: kind 0 = hop of
 * electron a to site b; kind 1 = exchange of up electron a with down
 * electron b.  Invalid moves give 0 (a hop onto an occupied spin orbital,
 * onto any electron under local_spin, or into or out of a local_site; an
 * exchange unless both sites are singly occupied).  Uses the same device
 * routines as the
 * sampler, on the walker's current inverse.  ratios: host [n_moves]. */
int vmc_eval_ratios(vmc_ctx *ctx, int32_t system, int32_t walker,
                    int32_t n_moves, const int32_t *moves, double *ratios);

/* Walker inverse check hook: M^-1 (N x N, row-major, FP64 copy; in the mixed
 * form the double-float value hi + lo the sweep keeps) of walker w,
 * M_nm = f(r_n,up, r_m,dn); log|det M| and its sign from the last
 * from-scratch factorisation. */
int vmc_get_inverse(vmc_ctx *ctx, int32_t system, int32_t walker,
                    double *minv, double *logabsdet, int32_t *sign);

/* Quantum-number projection of the pair product (Sec. 3.2.2, Eqs. momP and
 * pointP; boundary signs of App. A): after this call the context samples
 *   psi(x) = P(x) sum_g w_g <T_g^-1 x | phi_Pf>,
 * with the correlation factors P applied after the projector, where
 * T_g c^dag_{r,s} T_g^-1 = sign[g*Ns + r] c^dag_{perm[g*Ns + r], s}: operation g
 * maps site r to perm[g*Ns + r] with the fermion sign an anti-periodic
 * boundary gives (a permutation of the sites for every g, signs +1 / -1).
 * weight: w_g, real (momentum projection L_K with K components 0 or pi:
 * w_R = cos(K.R) / N_g; point groups: real characters / N_g; products of both
 * as the composed operations).  vmc_sample, vmc_measure, vmc_sr_step and
 * vmc_eval_ratios then use the projected state: every walker keeps one M_g^-1
 * per operation (N_g N^2 entries in device memory, allocated here) and the
 * share of each operation in its projected amplitude; the E_loc and O_k rows
 * are those of the projected state (the pair-orbital O_k are the
 * amplitude-weighted means over the operations).  Inverses are rebuilt (FP64)
 * before the next sample; walkers whose projected amplitude vanishes get new
 * seeded placements.  n_ops = 0 removes the projection.
 * Restrictions: a single-system context, no MLP factor, immediate updates
 * (delay depth 0 or 1); vmc_measure_corr, vmc_get_inverse and
 * vmc_tune_delay return VMC_EINVAL while a projection is set, and so does a
 * local_site mask that some operation does not map onto itself.
 * Errors: VMC_EINVAL (as above, n_ops > VMC_PROJ_MAX_OPS, a perm that is not
 * a permutation, a bad sign or weight), VMC_ENOMEM, VMC_ESINGULAR, VMC_ECUDA. */
#define VMC_PROJ_MAX_OPS 1024
int vmc_set_projection(vmc_ctx *ctx, int32_t n_ops, const int32_t *perm, const int8_t *sign,
                       const double *weight);

/* First-step power-Lanczos (Sec. 3.4): for every walker's CURRENT
 * configuration x of one system, the local values
 *   F1(x) = F(x, H) = <x|H|psi>/<x|psi>  (the local energy) and
 *   F2(x) = F(x, H^2) = sum_x' <x|H|x'> (H psi)(x') / psi(x),
 * every amplitude ratio taken from x (psi(x'')/psi(x), two moves away at
 * most; nothing divides by psi(x')), and their walker means
 *   moments = [h1, h2(11), h2(20), h3(12)] = [<F1>, <F1^2>, <F2>, <F1 F2>].
 * Averaging the moments of calls between vmc_sample calls gives the Monte
 * Carlo estimates of Sec. 3.4; vmc_lanczos_alpha then gives alpha_1.
 * F1, F2: NULL or host [n_walkers]; moments: host [4].  The Pfaffian ratios
 * come from Green-function tables of each configuration: FP64, or in the
 * mixed form FP32 tables from the hi words of its inverse and FP32 ratio and
 * correlation-factor arithmetic per term; the sums over first terms and over
 * walkers in FP64.  Device scratch
 * (about 8 (2 Ns N + Ns^2) bytes per resident CTA) is kept by the context.
 * Errors: VMC_EINVAL (bad system, NULL moments, a context with the MLP
 * factor, Heisenberg J terms, or a projection: not provided), VMC_ENOMEM,
 * VMC_ESINGULAR, VMC_ECUDA. */
int vmc_lanczos_moments(vmc_ctx *ctx, int32_t system, double *F1, double *F2, double *moments);

/* alpha_1 of Sec. 3.4 from the moments [h1, h2(11), h2(20), h3(12)]:
 * E_1(alpha) = (h1 + alpha (h2(20) + h2(11)) + alpha^2 h3(12))
 *            / (1 + 2 alpha h1 + alpha^2 h2(11)),
 * alpha_1 the root of dE_1/dalpha = 0 (a quadratic) with the lower E_1; E1
 * (may be NULL) receives E_1(alpha_1).  Host arithmetic only.  Errors:
 * VMC_EINVAL (NULL pointers), VMC_ENUMERIC (no real stationary point). */
int vmc_lanczos_alpha(const double *moments, double *alpha, double *E1);

/* Number of kernels this context has launched since creation. */
int64_t vmc_kernel_launches(vmc_ctx *ctx);

/* Launch configuration of the sweep/measurement kernel (no counterpart in the
 * paper): the persistent grid (CTAs, one walker at a time each), the CTAs that
 * fit on one SM at the kernel's shared-memory size (cudaOccupancy), and that
 * size in bytes (dynamic part: the walker's M^-1 block, plus its low words in
 * the mixed form); of the projected sweep kernel once vmc_set_projection has
 * armed operations.  Any output pointer may be NULL.
 * Errors: VMC_EINVAL (NULL ctx). */
int vmc_sweep_launch(vmc_ctx *ctx, int32_t *grid, int32_t *ctas_per_sm, int64_t *smem_bytes);

/* Failure-detection test hook (no counterpart in the paper; off unless
 * called).  Arms, for one call, a device wait that cannot complete: the
 * kernel polls, a bounded number of times (2^14), an mbarrier on which no copy
 * or MMA was issued, gives up with nothing in flight, and the call reports
 * VMC_ETIMEOUT exactly as for a real expired wait.
 *   VMC_STALL_SAMPLE: the next vmc_sample: the CTA that takes `walker` of
 *     `system` issues no copy of that walker's inverse and waits instead; the
 *     walker is skipped (its chain, counters and sample rows stay as they
 *     were) and that CTA stops; every other walker is sampled as usual.  The
 *     next vmc_sample samples it again.
 *   VMC_STALL_S_BUILD: the next dense S~ build of `system` by the persistent
 *     tensor-core kernel (mixed form; vmc_sr_step with a dense solver or
 *     vmc_get_sr_matrices): its first CTA waits before allocating tensor
 *     memory or issuing any copy or MMA; the SR step fails before the
 *     parameters change.
 *   VMC_STALL_NONE: disarm.
 * Errors: VMC_EINVAL (bad system or walker; VMC_STALL_S_BUILD on a FP64
 * context). */
enum { VMC_STALL_NONE = 0, VMC_STALL_SAMPLE = 1, VMC_STALL_S_BUILD = 2 };
int vmc_test_stall(vmc_ctx *ctx, int32_t target, int32_t system, int32_t walker);

/* Kernel timing with CUDA events on the context's stream (no counterpart in
 * the paper; used to report achieved throughput).  vmc_enable_timing(ctx, 1)
 * starts recording; vmc_kernel_times writes the accumulated milliseconds and
 * launch counts since the last reset into ms[4] and count[4], indexed by
 * 0 = sweep/measure kernel, 1 = from-scratch inverse kernel, 2 = SR step
 * (all its kernels), 3 = dense S build (within 2, or by vmc_get_sr_matrices),
 * and resets them.  Synchronises the stream. */
int vmc_enable_timing(vmc_ctx *ctx, int32_t on);
int vmc_kernel_times(vmc_ctx *ctx, double *ms, int64_t *count);

/* Delayed inverse updates (the fast updates of Sec. 3.1.2 applied in
 * batches).  With depth k >= 2 the sweep keeps up to k accepted hops as
 * rank-1 pairs (u_i, v_i), so the current inverse is
 * M^-1 = G0 - sum_i u_i v_i^T with G0 the stored one; proposal ratios are
 * corrected by the sum (O(N k) per ratio instead of reading an updated G),
 * and the pairs are folded into G0 by one rank-k product when k are pending,
 * before an accepted exchange, before each measurement and at the end of a
 * walker's turn.  Mathematically identical to immediate updates; rounding
 * differs.  k = 0 or 1: immediate rank-1 / rank-2 updates.
 * vmc_set_delay returns VMC_EINVAL for k outside [0, VMC_DELAY_MAX] or when
 * the walker state with k pending pairs no longer fits in shared memory. */
#define VMC_DELAY_MAX 32
int vmc_set_delay(vmc_ctx *ctx, int32_t k);
int32_t vmc_get_delay(vmc_ctx *ctx);

/* Autotuner for the delay depth (no counterpart in the paper).  For each
 * candidate depth cand[0..n_cand) (NULL: 1, 4, 8, 16, 32) runs
 * vmc_sample(ctx, 0, 1, sweeps) -- `sweeps` Metropolis sweeps per walker and
 * one measurement, the shape of a sampling step; the sweeps advance the
 * chains and the measurement replaces the stored samples -- timed with CUDA
 * events on the context's stream, then keeps the fastest depth.  In-sweep
 * FP64 recomputes are held off while timing; walkers that fall due meanwhile
 * are rebuilt by the next vmc_sample.  *chosen receives it; ms (optional,
 * n_cand entries) the milliseconds per sweep (measurement included) of each
 * candidate (negative where the depth does not fit). */
int vmc_tune_delay(vmc_ctx *ctx, int32_t sweeps, const int32_t *cand, int32_t n_cand,
                   int32_t *chosen, double *ms);

/* Proposals formed together by the sweep (no counterpart in the paper; a
 * schedule of Sec. 3.1.2's proposals, not a change of the method).  With
 * depth b >= 2 each walker takes the next b proposals of its stream, checks
 * them and forms their ratios at once against the current configuration and
 * inverse (the exchanges' rows R^T M^-1 in one pass over M^-1), then takes
 * the Metropolis decisions in the stream's order; the batch ends at the
 * first accepted proposal, whose move is made, and the proposals after it
 * are formed again against the updated state.  The chain (configurations,
 * counters, samples) is the one b = 1 gives, up to the ratios' summation
 * order.  Applies while the MLP factor and delayed updates are off (the
 * sweep makes proposals one at a time otherwise) and not to a projected
 * context's sweep (vmc_tune_proposal_batch returns VMC_EINVAL there).
 * Default 1.  What pays
 * depends on the workload: where most proposals are tested exchanges (spin
 * models) the shared pass over M^-1 wins; where the FP64 pipe or the
 * inverse updates bound the sweep, the proposals formed past an accepted one
 * are wasted work -- hence the tuner below. 
 * vmc_set_proposal_batch returns VMC_EINVAL for b outside [1, VMC_SPEC_MAX].
 * vmc_tune_proposal_batch times vmc_sample(ctx, sweeps, 0, 0) (sweeps only)
 * for each candidate depth (NULL: 1, 2, 4, 8) with CUDA events on the
 * context's stream, keeps the fastest in *chosen and, optionally, the
 * milliseconds per sweep of each candidate in ms; periodic recomputes are
 * held off while timing, as in vmc_tune_delay. */
#define VMC_SPEC_MAX 8
int vmc_set_proposal_batch(vmc_ctx *ctx, int32_t b);
int32_t vmc_get_proposal_batch(vmc_ctx *ctx);
int vmc_tune_proposal_batch(vmc_ctx *ctx, int32_t sweeps, const int32_t *cand,
                            int32_t n_cand, int32_t *chosen, double *ms);

/* Allocation-free SR means and force.  No counterpart in the paper: it is an
 * access path for callers that cannot let this library allocate device memory
 * (for example because another allocator already owns the GPU's memory, or
 * because cudaMalloc/cudaFree may synchronise the device inside a
 * latency-sensitive loop).  It computes, from caller-owned DEVICE arrays,
 *   ebar[0] = <E>,  obar[k] = <O_k>,  g[k] = <(O_k - obar_k)(E - ebar)>
 * over `rows` samples -- the quantities vmc_sr_step and vmc_get_sr_matrices
 * form from a context's stored FP32 samples, with the same chunked FP64 sums.
 *   O: rows x ldO FP32, row-major (ldO >= Np); E: rows FP64;
 *   obar, g: Np FP64 outputs; ebar: 1 FP64 output; stream: cudaStream_t or
 *   NULL for the default stream.  The work is queued on `stream`; the call
 *   returns without synchronising.
 * It calls no cudaMalloc, cudaFree or other allocating routine.  Its only
 * scratch (partial column sums over 2048-row chunks) is a fixed array of
 * VMC_FORCE_STATIC_MAX_DOUBLES doubles (8 MiB) inside the library, present
 * on every GPU that loads the library until the process exits.
 * Requirements and limits:
 *  - ceil(rows / 2048) * Np <= VMC_FORCE_STATIC_MAX_DOUBLES, else VMC_EINVAL
 *    (nothing is launched); VMC_EINVAL also for NULL pointers, rows < 1,
 *    Np < 1 or ldO < Np.
 *  - The first call on a device looks up the array's device address (with
 *    that device current, under a lock, so host threads may race to it);
 *    make that first call before any stream capture.  The address is kept
 *    for the life of the process: do not call it on a device after
 *    cudaDeviceReset() of that device.
 *  - Every call uses the same array.  Each call writes every scratch entry it
 *    reads, so no state carries over, but calls that overlap on the GPU (on
 *    different streams or host threads) race on it and must be serialised by
 *    the caller.
 * Errors: VMC_EINVAL as above; VMC_ECUDA if one of its launches fails, or,
 * before anything is launched, if a launch error from the caller's earlier
 * work is already pending (that error is left pending, not cleared). */
#define VMC_FORCE_STATIC_MAX_DOUBLES (1 << 20)
int vmc_sr_force_static(const float *O, int32_t ldO, int32_t rows, int32_t Np,
                        const double *E, double *obar, double *g, double *ebar,
                        void *stream);

#ifdef __cplusplus
}
#endif

#endif /* VMC_H */
