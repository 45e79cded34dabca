// Walker kernels: parameter expansion, from-scratch inverse (FP64 Gauss-Jordan),
// the Metropolis sweep with fast Pfaffian-ratio updates, the per-sample
// measurement of E_loc and the O_k row, and the pair correlations of the
// measurement mode.
//
// Wave function (mVMC paper, Sec. 3.2): psi(x) = P_G P_J <x|phi_AP-Pf>.  For
// S^z = 0 and the anti-parallel form (Eq. AP-Pf) the Ne x Ne skew matrix X of
// Sec. 3.2.1 is block off-diagonal, X = [[0, M], [-M^T, 0]] with
// M_nm = f(r_n,up, r_m,dn), so Pf X = (-1)^{N(N-1)/2} det M and
// X^-1 = [[0, -M^-T], [M^-1, 0]].  Each walker keeps M^-1 (N x N).
//
// Fast updates (Sec. 3.1.2, "Sherman-Morrison-type update"): a hop of up
// electron n replaces row n of M, a hop of down electron m replaces column m;
// an exchange replaces both (rank-2).  Ratios are det M'/det M from the
// matrix-determinant lemma; the inverse follows by Sherman-Morrison
// (rank 1) or Woodbury (rank 2).
#include "vmc_common.cuh"
#include "vmc_gj.cuh"
#include "vmc_dev.cuh"

#include <cuda_bf16.h>
#include <type_traits>
#include <math.h>

namespace {

__host__ __device__ __forceinline__ size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Global-memory stride of one walker's M^-1 (bytes, 128-aligned).
__host__ __device__ __forceinline__ size_t minv_bytes(int N, int ldm, int esize) {
  return align_up((size_t)N * ldm * esize, 128);
}

// ---- TMA bulk copies (cp.async.bulk) with an mbarrier, bounded waits ----
constexpr uint32_t WAIT_LIMIT = 1u << 22;   // try_wait attempts before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase with the given parity; false after `limit` attempts.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          uint32_t limit = WAIT_LIMIT) {
  for (uint32_t it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// Attempts of the test hook's wait (vmc_test_stall): a short bounded wait on
// a barrier no copy was issued for.
constexpr uint32_t STALL_LIMIT = 1u << 14;
// Two copies of `bytes` each completing on one mbarrier phase (one arrival
// expecting both transactions).
__device__ __forceinline__ void bulk_load_pair(void *dst0, const void *src0, void *dst1,
                                               const void *src1, uint32_t bytes, uint64_t *bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(2 * bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst0)),
      "l"(src0), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst1)),
      "l"(src1), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void bulk_store(void *dst, const void *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_u32(src)), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Shared-memory carve-up of one walker.
template <typename T>
struct WSmem {
  T *minv;      // N x ldm
  T *vec;       // 8 x VMC_MAX_N: block vectors vA..vD, or 2 per warp
  T *acc;       // O-row accumulator (acc_len); shares its space with ut/vt
  T *ut;        // delayed updates: u_i = ut[i*N ..], i < pending (measurement flushes first)
  T *vt;        //                  v_i = vt[i*N ..]
  T *red;       // 2 buffers x 8
  T *bc;        // 2 broadcast scalars (double-buffered like red)
  T *jf;        // Ns
  double *dred; // 2 buffers x 8 (double reductions)
  int *ele;     // Ne
  short *occ;   // 2 Ns: electron index at (site, spin), -1 if empty (16 bits: N <= 128)
  int *ilist;   // Ns
  int *misc;    // 8
  uint4 *rnd;   // RB Philox draws (one batch)
  T *hm;        // MLP pre-activations h (H)
  T *th;        // tanh(h) (H)
  float *mlo;   // mixed form: low words of the double-float M^-1 (N x ldm), else null
};

// Philox draws made per batch (one per thread of the first warp).
constexpr int RB = 32;

template <typename T>
__host__ __device__ size_t walker_layout(int N, int Ns, int acc_len, int H, int kd, bool lo,
                                         unsigned char *base, WSmem<T> *sm) {
  const int ldm = (N % 2) ? N : N + 1;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 16); return o; };
  const size_t o_minv = take(minv_bytes(N, ldm, sizeof(T)));
  const size_t o_vec = take(sizeof(T) * 8 * VMC_MAX_N);
  const size_t dly = (kd > 1) ? sizeof(T) * 2 * (size_t)kd * N : 0;
  // the O-row accumulator; also the delayed pairs, or a proposal batch's
  // per-warp partial sums (NWARP x 32 values), none of which live together
  size_t acc_b = sizeof(T) * (size_t)acc_len > dly ? sizeof(T) * (size_t)acc_len : dly;
  if (acc_b < sizeof(T) * NWARP * 32) acc_b = sizeof(T) * NWARP * 32;
  const size_t o_acc = take(acc_b);
  const size_t o_red = take(sizeof(T) * 32);
  const size_t o_bc = take(sizeof(T) * 2);
  const size_t o_jf = take(sizeof(T) * Ns);
  const size_t o_dred = take(sizeof(double) * 32);
  const size_t o_ele = take(sizeof(int) * 2 * N);
  const size_t o_occ = take(sizeof(short) * 2 * Ns);
  const size_t o_il = take(sizeof(int) * Ns);
  const size_t o_misc = take(sizeof(int) * 8);
  const size_t o_rnd = take(sizeof(uint4) * RB);
  const size_t o_hm = take(sizeof(T) * (size_t)H);
  const size_t o_th = take(sizeof(T) * (size_t)H);
  const size_t o_mlo = lo ? take(minv_bytes(N, ldm, sizeof(float))) : 0;
  if (sm) {
    sm->minv = (T *)(base + o_minv);
    sm->vec = (T *)(base + o_vec);
    sm->acc = (T *)(base + o_acc);
    sm->ut = (T *)(base + o_acc);
    sm->vt = sm->ut + (size_t)(kd > 1 ? kd : 0) * N;
    sm->red = (T *)(base + o_red);
    sm->bc = (T *)(base + o_bc);
    sm->jf = (T *)(base + o_jf);
    sm->dred = (double *)(base + o_dred);
    sm->ele = (int *)(base + o_ele);
    sm->occ = (short *)(base + o_occ);
    sm->ilist = (int *)(base + o_il);
    sm->misc = (int *)(base + o_misc);
    sm->rnd = (uint4 *)(base + o_rnd);
    sm->hm = (T *)(base + o_hm);
    sm->th = (T *)(base + o_th);
    sm->mlo = lo ? (float *)(base + o_mlo) : nullptr;
  }
  return off;
}

// Block sum with a double-buffered partial array: every thread returns the
// same value (same partials, same order).  One __syncthreads.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T *red, int &buf) {
  v = warp_sum(v);
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) red[buf * 16 + warp] = v;
  __syncthreads();
  const T *r = red + buf * 16;
  T s = r[0];
#pragma unroll
  for (int k = 1; k < NWARP; ++k) s += r[k];
  buf ^= 1;
  return s;
}

template <typename T>
__device__ __forceinline__ void block_sum2(T a, T b, T *red, int &buf, T &A, T &B) {
  a = warp_sum(a);
  b = warp_sum(b);
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[buf * 16 + warp] = a;
    red[buf * 16 + 4 + warp] = b;
  }
  __syncthreads();
  const T *r = red + buf * 16;
  A = r[0];
  B = r[4];
#pragma unroll
  for (int k = 1; k < NWARP; ++k) {
    A += r[k];
    B += r[4 + k];
  }
  buf ^= 1;
}

template <typename T>
__device__ __forceinline__ void block_sum3(T a, T b, T c, T *red, int &buf, T &A, T &B, T &C) {
  a = warp_sum(a);
  b = warp_sum(b);
  c = warp_sum(c);
  const int warp = threadIdx.x >> 5;
  T *r = red + buf * 16;
  if ((threadIdx.x & 31) == 0) {
    r[warp] = a;
    r[4 + warp] = b;
    r[8 + warp] = c;
  }
  __syncthreads();
  A = r[0];
  B = r[4];
  C = r[8];
#pragma unroll
  for (int k = 1; k < NWARP; ++k) {
    A += r[k];
    B += r[4 + k];
    C += r[8 + k];
  }
  buf ^= 1;
}

// ---- MLP correlation factor -------------------------------------------------
// Column c = site + Ns * spin of W1 (H entries, contiguous): FP64 in the plain
// form, BF16 (FP32 arithmetic) in the mixed form.
template <typename T> __device__ __forceinline__ T w1c(const SysDev &S, int c, int k);
template <> __device__ __forceinline__ double w1c<double>(const SysDev &S, int c, int k) {
  return S.W1T64[(size_t)c * S.n_hidden + k];
}
template <> __device__ __forceinline__ float w1c<float>(const SysDev &S, int c, int k) {
  return __bfloat162float(((const __nv_bfloat16 *)S.W1T16)[(size_t)c * S.n_hidden + k]);
}
template <typename T> __device__ __forceinline__ T tanh_t(T x);
template <> __device__ __forceinline__ double tanh_t<double>(double x) { return tanh(x); }
template <> __device__ __forceinline__ float tanh_t<float>(float x) { return tanhf(x); }
template <typename T> __device__ __forceinline__ T exp_t(T x);
template <> __device__ __forceinline__ double exp_t<double>(double x) { return exp(x); }
template <> __device__ __forceinline__ float exp_t<float>(float x) { return expf(x); }

// Change of h for a move: + column cp0 (+ cp1) - column cm0 (- cm1); cp1/cm1 < 0: unused.
template <typename T>
__device__ __forceinline__ T mlp_dh(const SysDev &S, int k, int cp0, int cm0, int cp1, int cm1) {
  T d = w1c<T>(S, cp0, k) - w1c<T>(S, cm0, k);
  if (cp1 >= 0) d += w1c<T>(S, cp1, k) - w1c<T>(S, cm1, k);
  return d;
}

// This thread's share (k = tid, tid + NT, ...) of
// log P_MLP(x')/P_MLP(x) = sum_k w2_k (tanh(h_k + dh_k) - tanh(h_k)).
template <typename T>
__device__ __forceinline__ T mlp_log_ratio_part(const SysDev &S, const WSmem<T> &sm, int cp0,
                                                int cm0, int cp1, int cm1, int k0, int kstep) {
  const int H = S.n_hidden;
  const double *w2 = S.params + S.mlp_base + (size_t)H * 2 * S.Ns + H;
  T part = (T)0;
  for (int k = k0; k < H; k += kstep)
    part += (T)w2[k] * (tanh_t<T>(sm.hm[k] + mlp_dh<T>(S, k, cp0, cm0, cp1, cm1)) - sm.th[k]);
  return part;
}

template <typename T>
__device__ __forceinline__ void mlp_apply(const SysDev &S, const WSmem<T> &sm, int cp0, int cm0,
                                          int cp1, int cm1) {
  for (int k = threadIdx.x; k < S.n_hidden; k += NT) {
    const T h = sm.hm[k] + mlp_dh<T>(S, k, cp0, cm0, cp1, cm1);
    sm.hm[k] = h;
    sm.th[k] = tanh_t<T>(h);
  }
}

// The shared-memory row loops are staged through registers CH elements at a
// time, so a chunk's loads are all issued before its stores (the compiler
// cannot reorder loads of one array past stores to another shared array).
constexpr int CH = 16;

// Four consecutive entries of a 16-byte-aligned shared vector (the x / y
// operands below are always slots of the walker's vector area) by 128-bit
// loads: one load instruction per four entries for FP32, two for FP64.
__device__ __forceinline__ void ld4(const float *p, float &a, float &b, float &c, float &d) {
  const float4 v = *reinterpret_cast<const float4 *>(p);
  a = v.x;
  b = v.y;
  c = v.z;
  d = v.w;
}
__device__ __forceinline__ void ld4(const double *p, double &a, double &b, double &c, double &d) {
  const double2 u = *reinterpret_cast<const double2 *>(p);
  const double2 v = *reinterpret_cast<const double2 *>(p + 2);
  a = u.x;
  b = u.y;
  c = v.x;
  d = v.y;
}

// row[k] -= c x[k]  (x 16-byte aligned)
template <typename T>
__device__ __forceinline__ void row_axpy(T *row, const T *x, T c, int N) {
  int k = 0;
  for (; k + CH <= N; k += CH) {
    T a[CH], b[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) a[u] = row[k + u];
#pragma unroll
    for (int u = 0; u < CH; u += 4) ld4(x + k + u, b[u], b[u + 1], b[u + 2], b[u + 3]);
#pragma unroll
    for (int u = 0; u < CH; ++u) row[k + u] = a[u] - c * b[u];
  }
  for (; k < N; ++k) row[k] -= c * x[k];
}

// row[k] -= c1 x[k] + c2 y[k]  (x, y 16-byte aligned)
template <typename T>
__device__ __forceinline__ void row_axpy2(T *row, const T *x, const T *y, T c1, T c2, int N) {
  int k = 0;
  for (; k + CH <= N; k += CH) {
    T a[CH], b[CH], d[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) a[u] = row[k + u];
#pragma unroll
    for (int u = 0; u < CH; u += 4) {
      ld4(x + k + u, b[u], b[u + 1], b[u + 2], b[u + 3]);
      ld4(y + k + u, d[u], d[u + 1], d[u + 2], d[u + 3]);
    }
#pragma unroll
    for (int u = 0; u < CH; ++u) row[k + u] = a[u] - (c1 * b[u] + c2 * d[u]);
  }
  for (; k < N; ++k) row[k] -= c1 * x[k] + c2 * y[k];
}

// sum_k row[k] x[k] with four accumulators (x 16-byte aligned)
template <typename T>
__device__ __forceinline__ T row_dot(const T *row, const T *x, int N) {
  T a0 = (T)0, a1 = (T)0, a2 = (T)0, a3 = (T)0;
  int k = 0;
  for (; k + 4 <= N; k += 4) {
    T x0, x1, x2, x3;
    ld4(x + k, x0, x1, x2, x3);
    a0 += row[k] * x0;
    a1 += row[k + 1] * x1;
    a2 += row[k + 2] * x2;
    a3 += row[k + 3] * x3;
  }
  for (; k < N; ++k) a0 += row[k] * x[k];
  return (a0 + a1) + (a2 + a3);
}

// sum_l x[l] M[l][col] (column of the shared matrix) with four accumulators
// (x 16-byte aligned)
template <typename T>
__device__ __forceinline__ T col_dot(const T *M, int ldm, int col, const T *x, int N) {
  T a0 = (T)0, a1 = (T)0, a2 = (T)0, a3 = (T)0;
  int l = 0;
  for (; l + 4 <= N; l += 4) {
    T x0, x1, x2, x3;
    ld4(x + l, x0, x1, x2, x3);
    a0 += x0 * M[l * ldm + col];
    a1 += x1 * M[(l + 1) * ldm + col];
    a2 += x2 * M[(l + 2) * ldm + col];
    a3 += x3 * M[(l + 3) * ldm + col];
  }
  for (; l < N; ++l) a0 += x[l] * M[l * ldm + col];
  return (a0 + a1) + (a2 + a3);
}

// ---------------------------------------------------------------------------
// Pfaffian ratios (block-wide; every thread returns the same value)
// ---------------------------------------------------------------------------
// Hop of electron e to empty site t: det M'/det M = sum_l R_l (M^-1)_{l n}
// (up electron n = e, new row R_l = f(t, r_l,dn)) or
// sum_k (M^-1)_{m k} C_k (down electron m = e - N, new column C_k = f(r_k,up, t)).
// fval receives this thread's entry of the new row/column.
// With the MLP factor, mlp receives log P_MLP(x')/P_MLP(x) (same barrier).
// With np pending delayed updates the current inverse is G = G0 - sum_i u_i v_i^T
// (G0 = sm.minv): the column / row entry used here is corrected by the sum, and
// kept in vec slot 4 for the update on acceptance.
template <typename T>
__device__ __forceinline__ T hop_pf_ratio(const SysDev &S, const WSmem<T> &sm, int e, int t,
                                          T &fval, int &buf, T &mlp, int np) {
  const int N = S.N, Ns = S.Ns, tid = threadIdx.x;
  T prod = (T)0;
  fval = (T)0;
  if (tid < N) {
    T gent;
    if (e < N) {
      fval = ftab<T>(S)[(size_t)t * Ns + sm.ele[N + tid]];
      gent = sm.minv[tid * S.ldm + e];
      for (int i = 0; i < np; ++i) gent -= sm.ut[i * N + tid] * sm.vt[i * N + e];
    } else {
      const int m = e - N;
      fval = fTtab<T>(S)[(size_t)t * Ns + sm.ele[tid]];
      gent = sm.minv[m * S.ldm + tid];
      for (int i = 0; i < np; ++i) gent -= sm.ut[i * N + m] * sm.vt[i * N + tid];
    }
    prod = gent * fval;
    if (S.delay_k > 1) sm.vec[4 * VMC_MAX_N + tid] = gent;
  }
  if (!S.n_hidden) {
    mlp = (T)0;
    return block_sum(prod, sm.red, buf);
  }
  const int sp = (e >= N) ? Ns : 0;
  const T part = mlp_log_ratio_part(S, sm, t + sp, sm.ele[e] + sp, -1, -1, tid, NT);
  T A;
  block_sum2(prod, part, sm.red, buf, A, mlp);
  return A;
}

// Exchange of up electron n (site i) with down electron m (site j):
// M' = M + e_n a^T + b e_m^T with a = R - M[n,:] (new row R_l = f(j, r_l,dn),
// R_m = f(j, i)) and b = C - M[:,m] with b_n = 0 (new column
// C_k = f(r'_k,up, i), r'_n = j).  det M'/det M = det(I_2 + V^T M^-1 U),
// U = [e_n, b], V = [a, e_m]:
//   K11 = (R^T M^-1)_n, K12 = sum_{k != n} (R^T M^-1)_k b_k,
//   K21 = (M^-1)_{mn},  K22 = sum_k (M^-1)_{mk} C'_k (C'_n = M_nm).
// On return vB holds w = R^T M^-1, vC holds C, K[0..3] the 2x2 matrix.
// z_i = x_i . y for the np pending vectors x_i = X[i*N ..] (warp per i),
// written to out[i]; the caller synchronises before reading out.
template <typename T>
__device__ __forceinline__ void pending_dots(const T *X, const T *y, int N, int np, T *out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = warp; i < np; i += NWARP) {
    T s = (T)0;
    for (int l = lane; l < N; l += 32) s += X[i * N + l] * y[l];
    s = warp_sum(s);
    if (lane == 0) out[i] = s;
  }
}

template <typename T>
__device__ T exchange_pf_ratio(const SysDev &S, const WSmem<T> &sm, int n, int m, int i, int j,
                               int &buf, T *K, T &mlp, int np) {
  const int N = S.N, Ns = S.Ns, ldm = S.ldm, tid = threadIdx.x;
  const T *F = ftab<T>(S);
  const T *FT = fTtab<T>(S);
  T *vA = sm.vec, *vB = sm.vec + VMC_MAX_N, *vC = sm.vec + 2 * VMC_MAX_N;
  T *vz = sm.vec + 5 * VMC_MAX_N;
  if (tid < N) vA[tid] = (tid == m) ? F[(size_t)j * Ns + i] : F[(size_t)j * Ns + sm.ele[N + tid]];
  __syncthreads();
  T w = (T)0;
  if (tid < N) w = col_dot(sm.minv, ldm, tid, vA, N);
  if (np > 0) {
    // R^T G = R^T G0 - sum_i (R . u_i) v_i^T
    pending_dots(sm.ut, vA, N, np, vz);
    __syncthreads();
    if (tid < N)
      for (int q = 0; q < np; ++q) w -= vz[q] * sm.vt[q * N + tid];
  }
  T a22 = (T)0, a12 = (T)0;
  if (tid < N) {
    vB[tid] = w;
    const int site = (tid == n) ? j : sm.ele[tid];
    const T c = FT[(size_t)i * Ns + site];
    const T mkm = FT[(size_t)j * Ns + sm.ele[tid]];
    vC[tid] = c;
    T mrow = sm.minv[m * ldm + tid];
    for (int q = 0; q < np; ++q) mrow -= sm.ut[q * N + m] * sm.vt[q * N + tid];
    if (tid == n) {
      a22 = mrow * mkm;
    } else {
      a22 = mrow * c;
      a12 = w * (c - mkm);
    }
  }
  T A22, A12;
  if (S.n_hidden) {
    // up electron i -> j, down electron j -> i: +(i,dn) -(i,up) +(j,up) -(j,dn)
    const T part = mlp_log_ratio_part(S, sm, i + Ns, i, j, j + Ns, tid, NT);
    block_sum3(a22, a12, part, sm.red, buf, A22, A12, mlp);
  } else {
    block_sum2(a22, a12, sm.red, buf, A22, A12);
    mlp = (T)0;
  }
  const T A11 = vB[n];
  T A21 = sm.minv[m * ldm + n];
  for (int q = 0; q < np; ++q) A21 -= sm.ut[q * N + m] * sm.vt[q * N + n];
  K[0] = A11;
  K[1] = A12;
  K[2] = A21;
  K[3] = A22;
  return A11 * A22 - A12 * A21;
}

// ---------------------------------------------------------------------------
// Inverse updates on acceptance
// ---------------------------------------------------------------------------

// Row n replaced by the row in vA (up-electron hop): with w = R^T M^-1,
// M'^-1 = M^-1 - M^-1[:,n] (w - e_n)^T / w_n.
template <typename T>
__device__ void row_update(const SysDev &S, const WSmem<T> &sm, int n, const T *R = nullptr) {
  const int N = S.N, ldm = S.ldm, tid = threadIdx.x;
  const T *vA = R ? R : sm.vec;
  T *vB = sm.vec + VMC_MAX_N;
  if (tid < N) vB[tid] = col_dot(sm.minv, ldm, tid, vA, N);
  __syncthreads();
  const T inv = (T)1 / vB[n];
  if (tid < N) {
    T *row = sm.minv + tid * ldm;
    const T c = row[n] * inv;
    row_axpy(row, vB, c, N);
    row[n] = c;
  }
  __syncthreads();
}

// Column m replaced by the column in vA (down-electron hop): with v = M^-1 C,
// M'^-1 = M^-1 - (v - e_m) M^-1[m,:] / v_m.
template <typename T>
__device__ void col_update(const SysDev &S, const WSmem<T> &sm, int m, const T *Cn = nullptr) {
  const int N = S.N, ldm = S.ldm, tid = threadIdx.x;
  const T *vA = Cn ? Cn : sm.vec;
  T *vB = sm.vec + VMC_MAX_N, *vC = sm.vec + 2 * VMC_MAX_N;
  if (tid < N) {
    vB[tid] = row_dot(sm.minv + tid * ldm, vA, N);
    vC[tid] = sm.minv[m * ldm + tid];
  }
  __syncthreads();
  const T inv = (T)1 / vB[m];
  if (tid < N) {
    T *row = sm.minv + tid * ldm;
    if (tid == m) {
      for (int k = 0; k < N; ++k) row[k] = vC[k] * inv;
    } else {
      row_axpy(row, vC, vB[tid] * inv, N);
    }
  }
  __syncthreads();
}

// Rank-2 (Woodbury) update after an accepted exchange; vB = w, vC = C and K
// from exchange_pf_ratio.  M'^-1 = M^-1 - [p q] K^-1 [w - e_n; z] with
// p = M^-1[:,n], q = M^-1 b, z = M^-1[m,:].
template <typename T>
__device__ void exchange_update(const SysDev &S, const WSmem<T> &sm, int n, int m, int j,
                                const T *K, T det, const T *wv = nullptr, const T *cv = nullptr) {
  const int N = S.N, Ns = S.Ns, ldm = S.ldm, tid = threadIdx.x;
  const T *FT = fTtab<T>(S);
  T *vA = sm.vec, *vD = sm.vec + 3 * VMC_MAX_N;
  const T *vB = wv ? wv : sm.vec + VMC_MAX_N, *vC = cv ? cv : sm.vec + 2 * VMC_MAX_N;
  if (tid < N) {
    vA[tid] = (tid == n) ? (T)0 : vC[tid] - FT[(size_t)j * Ns + sm.ele[tid]];
    vD[tid] = sm.minv[m * ldm + tid];
  }
  __syncthreads();
  if (tid < N) {
    T *row = sm.minv + tid * ldm;
    const T q = row_dot(row, vA, N);
    const T p = row[n];
    const T inv = (T)1 / det;
    const T c1 = (p * K[3] - q * K[2]) * inv;
    const T c2 = (q * K[0] - p * K[1]) * inv;
    row_axpy2(row, vB, vD, c1, c2, N);
    row[n] += c1;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Double-float inverse of the mixed form
// ---------------------------------------------------------------------------
// The mixed form keeps M^-1 as hi + lo, two FP32 words per entry: hi is the
// FP32 inverse every ratio and the measurement read; lo holds what lies
// below hi's last bit.  Accepted moves update both with error-free FP32
// transformations (Knuth's TwoSum, the FMA's exact product), so the update
// rounds at about 2^-46 instead of 2^-24 and FP32 ratios keep the accuracy
// of a freshly rebuilt inverse, where FP32 updates alone let the error grow
// with every small ratio.  New rows and columns come from the FP64 tables.
__device__ __forceinline__ void fast2sum(float a, float b, float &s, float &e) {
  s = a + b;
  e = b - (s - a);
}
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float v = s - a;
  e = (a - (s - v)) + (b - v);
}
// x += a b (all double-float)
__device__ __forceinline__ void df_fma(float &xh, float &xl, float ah, float al, float bh, float bl) {
  const float p = ah * bh;
  float pe = fmaf(ah, bh, -p);
  pe = fmaf(ah, bl, pe);
  pe = fmaf(al, bh, pe);
  float sh, se;
  two_sum(xh, p, sh, se);
  se += xl + pe;
  fast2sum(sh, se, xh, xl);
}
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float &h, float &l) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  fast2sum(p, e, h, l);
}
// 1 / (ah + al): the FP32 reciprocal refined by one Newton step in double-float
__device__ __forceinline__ void df_recip(float ah, float al, float &h, float &l) {
  const float q = 1.0f / ah;
  const float p = ah * q;
  float pe = fmaf(ah, q, -p);
  pe = fmaf(al, q, pe);
  const float r = (1.0f - p) - pe;
  fast2sum(q, q * r, h, l);
}
// Compensated dot product in FP32 words (Ogita-Rump-Oishi Dot2): s sums the
// products' heads with TwoSum, c collects every rounding error and the
// products' tails; four independent accumulators, normalised once at the end.
struct Dot2 {
  float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
  __device__ __forceinline__ void add(int q, float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    float pe = fmaf(ah, bh, -p);
    pe = fmaf(ah, bl, pe);
    pe = fmaf(al, bh, pe);
    float t, e;
    two_sum(s[q], p, t, e);
    s[q] = t;
    c[q] += e + pe;
  }
  __device__ __forceinline__ void result(float &h, float &l) const {
    float t0, e0, t1, e1, t, e;
    two_sum(s[0], s[1], t0, e0);
    two_sum(s[2], s[3], t1, e1);
    two_sum(t0, t1, t, e);
    const float cc = ((c[0] + c[1]) + (c[2] + c[3])) + (e0 + e1 + e);
    fast2sum(t, cc, h, l);
  }
};

// sum_l x[l] M[l][col] (x double-float in 16-byte-aligned slots xh / xl)
__device__ __forceinline__ void df_col_dot(const float *Mh, const float *Ml, int ldm, int col,
                                           const float *xh, const float *xl, int N, float &h,
                                           float &l) {
  Dot2 d;
  int k = 0;
  for (; k + 4 <= N; k += 4) {
    float a0, a1, a2, a3, b0, b1, b2, b3;
    ld4(xh + k, a0, a1, a2, a3);
    ld4(xl + k, b0, b1, b2, b3);
    d.add(0, a0, b0, Mh[k * ldm + col], Ml[k * ldm + col]);
    d.add(1, a1, b1, Mh[(k + 1) * ldm + col], Ml[(k + 1) * ldm + col]);
    d.add(2, a2, b2, Mh[(k + 2) * ldm + col], Ml[(k + 2) * ldm + col]);
    d.add(3, a3, b3, Mh[(k + 3) * ldm + col], Ml[(k + 3) * ldm + col]);
  }
  for (; k < N; ++k) d.add(0, xh[k], xl[k], Mh[k * ldm + col], Ml[k * ldm + col]);
  d.result(h, l);
}

// sum_k row[k] x[k] (the thread's row in rh / rl; x as above)
__device__ __forceinline__ void df_row_dot(const float *rh, const float *rl, const float *xh,
                                           const float *xl, int N, float &h, float &l) {
  Dot2 d;
  int k = 0;
  for (; k + 4 <= N; k += 4) {
    float a0, a1, a2, a3, b0, b1, b2, b3;
    ld4(xh + k, a0, a1, a2, a3);
    ld4(xl + k, b0, b1, b2, b3);
    d.add(0, rh[k], rl[k], a0, b0);
    d.add(1, rh[k + 1], rl[k + 1], a1, b1);
    d.add(2, rh[k + 2], rl[k + 2], a2, b2);
    d.add(3, rh[k + 3], rl[k + 3], a3, b3);
  }
  for (; k < N; ++k) d.add(0, rh[k], rl[k], xh[k], xl[k]);
  d.result(h, l);
}

__device__ __forceinline__ void df_split(double x, float &h, float &l) {
  h = (float)x;
  l = (float)(x - (double)h);
}
__device__ __forceinline__ double df_val(float h, float l) { return (double)h + (double)l; }

// row[k] -= c x[k] for the thread's row (hi in rh, lo in rl), x double-float
// vectors in 16-byte-aligned slots
__device__ __forceinline__ void df_row_axpy(float *rh, float *rl, const float *xh, const float *xl,
                                            float ch, float cl, int N) {
  const float nh = -ch, nl = -cl;
  int k = 0;
  for (; k + CH <= N; k += CH) {
    float ah[CH], al[CH], bh[CH], bl[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      ah[u] = rh[k + u];
      al[u] = rl[k + u];
    }
#pragma unroll
    for (int u = 0; u < CH; u += 4) {
      ld4(xh + k + u, bh[u], bh[u + 1], bh[u + 2], bh[u + 3]);
      ld4(xl + k + u, bl[u], bl[u + 1], bl[u + 2], bl[u + 3]);
    }
#pragma unroll
    for (int u = 0; u < CH; ++u) df_fma(ah[u], al[u], nh, nl, bh[u], bl[u]);
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      rh[k + u] = ah[u];
      rl[k + u] = al[u];
    }
  }
  for (; k < N; ++k) {
    float h = rh[k], l = rl[k];
    df_fma(h, l, nh, nl, xh[k], xl[k]);
    rh[k] = h;
    rl[k] = l;
  }
}

// From-scratch inverse in double-float, the mixed form's opt-in alternative
// to the FP64 elimination (VMC_REBUILD_DOUBLE_FLOAT): Gauss-Jordan with
// partial pivoting, in place, on hi + lo words, every multiply-subtract an
// error-free FP32 sequence (df_fma).  The pivot is the largest |hi| of the
// column (ties: lowest row).  GB300's FP64 pipe runs at 1/64 of the FP32
// rate and a double-float multiply-add costs about fifteen FP32 operations,
// so the elimination is faster than in FP64 at about 2^-46 rounding, the
// precision the sweep's updates keep.  The scalars of the determinant stay
// FP64.
struct GJdf {
  double val[NWARP];
  double amax[NWARP];
  double pminw[NWARP];
  int idx[NWARP];
  int piv, bad, sign;
  float ih, il;                 // 1 / pivot
  double logdet, pmin, pmax;    // log|det M|, smallest / largest |pivot|
  float ph[VMC_MAX_N], pl[VMC_MAX_N];   // pivot of every step
  alignas(16) float ch[VMC_MAX_N];      // pivot column of the step (row k zeroed)
  alignas(16) float cl[VMC_MAX_N];
  alignas(16) float rh[VMC_MAX_N];      // scaled pivot row of the step (column k zeroed)
  alignas(16) float rl[VMC_MAX_N];
};

__device__ void gj_invert_df(float *Ah, float *Al, int lda, int N, int *perm, GJdf &g) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    g.sign = 1;
    g.bad = 0;
  }
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    // (1) copy column k; pivot among rows >= k
    float v = -1.f;
    int vi = N;
    for (int i = tid; i < N; i += NT) {
      const float h = Ah[i * lda + k];
      g.ch[i] = h;
      g.cl[i] = Al[i * lda + k];
      if (i >= k && fabsf(h) > v) {
        v = fabsf(h);
        vi = i;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int oi = __shfl_xor_sync(0xffffffffu, vi, o);
      if (ov > v || (ov == v && oi < vi)) {
        v = ov;
        vi = oi;
      }
    }
    if (lane == 0) {
      g.val[warp] = v;
      g.idx[warp] = vi;
    }
    __syncthreads();
    // (2) one thread: pivot row, its entry swapped out of the column copy, 1/pivot
    if (tid == 0) {
      double bv = g.val[0];
      int bi = g.idx[0];
      for (int q = 1; q < NWARP; ++q)
        if (g.val[q] > bv || (g.val[q] == bv && g.idx[q] < bi)) {
          bv = g.val[q];
          bi = g.idx[q];
        }
      if (!(bv > 0.0) || bi >= N) {
        g.bad = 1;
        bi = k;
      }
      g.piv = bi;
      perm[k] = bi;
      const float ph = g.ch[bi], pl = g.cl[bi];
      g.ch[bi] = g.ch[k];
      g.cl[bi] = g.cl[k];
      g.ch[k] = 0.f;   // row k is scaled, not eliminated
      g.cl[k] = 0.f;
      df_recip(ph, pl, g.ih, g.il);
      g.ph[k] = ph;    // log|det| is summed after the elimination
      g.pl[k] = pl;
      if ((ph < 0.f) != (bi != k)) g.sign = -g.sign;   // hi carries the sign
    }
    __syncthreads();
    if (g.bad) return;
    const int p = g.piv;
    const float ih = g.ih, il = g.il;
    // (3a) the new column k; rows k and p swapped, row k scaled and kept
    for (int i = tid; i < N; i += NT) {
      float h = ih, l = il;
      if (i != k) df_mul(-g.ch[i], -g.cl[i], ih, il, h, l);
      Ah[i * lda + k] = h;
      Al[i * lda + k] = l;
    }
    for (int c = tid; c < N; c += NT) {
      if (c == k) {
        g.rh[c] = 0.f;   // column k is final
        g.rl[c] = 0.f;
        continue;
      }
      const float h = Ah[p * lda + c], l = Al[p * lda + c];
      if (p != k) {
        Ah[p * lda + c] = Ah[k * lda + c];
        Al[p * lda + c] = Al[k * lda + c];
      }
      float sh, sl;
      df_mul(h, l, ih, il, sh, sl);
      Ah[k * lda + c] = sh;
      Al[k * lda + c] = sl;
      g.rh[c] = sh;
      g.rl[c] = sl;
    }
    __syncthreads();
    // (3b) A_ic -= colk_i rowk_c: thread c < N takes column c (c != k: rowk_k
    // = 0 leaves column k) over all rows, eight at a time with the pivot
    // column read by 16-byte broadcast loads; colk_k = 0 leaves the value of
    // row k unchanged.
    if (tid < N && tid != k) {
      const float rh = g.rh[tid], rl = g.rl[tid];
      float *qh = Ah + tid, *ql = Al + tid;
      int i = 0;
      for (; i + 8 <= N; i += 8) {
        float c[8], e[8], h[8], l[8];
        ld4(g.ch + i, c[0], c[1], c[2], c[3]);
        ld4(g.ch + i + 4, c[4], c[5], c[6], c[7]);
        ld4(g.cl + i, e[0], e[1], e[2], e[3]);
        ld4(g.cl + i + 4, e[4], e[5], e[6], e[7]);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          h[r] = qh[(i + r) * lda];
          l[r] = ql[(i + r) * lda];
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) df_fma(h[r], l[r], -c[r], -e[r], rh, rl);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          qh[(i + r) * lda] = h[r];
          ql[(i + r) * lda] = l[r];
        }
      }
      for (; i < N; ++i) {
        float h = qh[i * lda], l = ql[i * lda];
        df_fma(h, l, -g.ch[i], -g.cl[i], rh, rl);
        qh[i * lda] = h;
        ql[i * lda] = l;
      }
    }
    __syncthreads();
  }
  // log|det M| and the pivot range
  {
    double ls = 0.0, mn = 1e300, mx = 0.0;
    for (int i = tid; i < N; i += NT) {
      const double a = fabs((double)g.ph[i] + (double)g.pl[i]);
      ls += log(a);
      mn = fmin(mn, a);
      mx = fmax(mx, a);
    }
    for (int o = 16; o > 0; o >>= 1) {
      ls += __shfl_xor_sync(0xffffffffu, ls, o);
      mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) {
      g.val[warp] = ls;
      g.pminw[warp] = mn;
      g.amax[warp] = mx;
    }
    __syncthreads();
    if (tid == 0) {
      double a = 0.0, b = 1e300, c = 0.0;
      for (int q = 0; q < NWARP; ++q) {
        a += g.val[q];
        b = fmin(b, g.pminw[q]);
        c = fmax(c, g.amax[q]);
      }
      g.logdet = a;
      g.pmin = b;
      g.pmax = c;
    }
  }
  // undo the row interchanges as column interchanges of the inverse
  for (int k = N - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p == k) continue;   // uniform: perm is shared
    for (int r = tid; r < N; r += NT) {
      const float h = Ah[r * lda + k], l = Al[r * lda + k];
      Ah[r * lda + k] = Ah[r * lda + p];
      Al[r * lda + k] = Al[r * lda + p];
      Ah[r * lda + p] = h;
      Al[r * lda + p] = l;
    }
    __syncthreads();
  }
  __syncthreads();
}

// Row n replaced (up electron n to site t): w = R^T M^-1 with the new row
// R_l = f(t, r_l,dn), M'^-1 = M^-1 - M^-1[:,n] (w - e_n)^T / w_n (Sherman-Morrison).
__device__ void row_update_df(const SysDev &S, const WSmem<float> &sm, int n, int t) {
  const int N = S.N, Ns = S.Ns, ldm = S.ldm, tid = threadIdx.x;
  float *Rh = sm.vec, *Rl = sm.vec + VMC_MAX_N, *Wh = sm.vec + 2 * VMC_MAX_N,
        *Wl = sm.vec + 3 * VMC_MAX_N;
  if (tid < N) df_split(S.f64[(size_t)t * Ns + sm.ele[N + tid]], Rh[tid], Rl[tid]);
  __syncthreads();
  if (tid < N) df_col_dot(sm.minv, sm.mlo, ldm, tid, Rh, Rl, N, Wh[tid], Wl[tid]);
  __syncthreads();
  float ih, il;
  df_recip(Wh[n], Wl[n], ih, il);
  if (tid < N) {
    float *rh = sm.minv + tid * ldm, *rl = sm.mlo + tid * ldm;
    float ch, cl;
    df_mul(rh[n], rl[n], ih, il, ch, cl);
    df_row_axpy(rh, rl, Wh, Wl, ch, cl, N);
    rh[n] = ch;
    rl[n] = cl;
  }
  __syncthreads();
}

// Column m replaced (down electron m to site t): v = M^-1 C with the new
// column C_k = f(r_k,up, t), M'^-1 = M^-1 - (v - e_m) M^-1[m,:] / v_m.
__device__ void col_update_df(const SysDev &S, const WSmem<float> &sm, int m, int t) {
  const int N = S.N, Ns = S.Ns, ldm = S.ldm, tid = threadIdx.x;
  float *Ch = sm.vec, *Cl = sm.vec + VMC_MAX_N, *Vh = sm.vec + 2 * VMC_MAX_N,
        *Vl = sm.vec + 3 * VMC_MAX_N, *Zh = sm.vec + 4 * VMC_MAX_N, *Zl = sm.vec + 5 * VMC_MAX_N;
  if (tid < N) {
    df_split(S.fT64[(size_t)t * Ns + sm.ele[tid]], Ch[tid], Cl[tid]);
    Zh[tid] = sm.minv[m * ldm + tid];
    Zl[tid] = sm.mlo[m * ldm + tid];
  }
  __syncthreads();
  if (tid < N)
    df_row_dot(sm.minv + tid * ldm, sm.mlo + tid * ldm, Ch, Cl, N, Vh[tid], Vl[tid]);
  __syncthreads();
  float ih, il;
  df_recip(Vh[m], Vl[m], ih, il);
  if (tid < N) {
    float *rh = sm.minv + tid * ldm, *rl = sm.mlo + tid * ldm;
    if (tid == m) {
      for (int k = 0; k < N; ++k) df_mul(Zh[k], Zl[k], ih, il, rh[k], rl[k]);
    } else {
      float ch, cl;
      df_mul(Vh[tid], Vl[tid], ih, il, ch, cl);
      df_row_axpy(rh, rl, Zh, Zl, ch, cl, N);
    }
  }
  __syncthreads();
}

// Exchange of up electron n (site i) with down electron m (site j), rank 2
// (Woodbury): with the new row R (R_l = f(j, r_l,dn), R_m = f(j, i)), w = R^T M^-1,
// b_k = C_k - M_km (C_k = f(r'_k,up, i), r'_n = j; b_n = 0), z = M^-1[m,:],
// K = [[w_n, sum_k w_k b_k], [M^-1_mn, sum_k M^-1_mk C'_k]] (C'_n = M_nm),
// M'^-1 = M^-1 - [p q] K^-1 [w - e_n; z] with p = M^-1[:,n], q = M^-1 b.
// The 2 x 2 and per-row scalars are FP64; the N^2 parts double-float.
__device__ void exchange_update_df(const SysDev &S, const WSmem<float> &sm, int n, int m, int i,
                                   int j, int &buf) {
  const int N = S.N, Ns = S.Ns, ldm = S.ldm, tid = threadIdx.x;
  float *Rh = sm.vec, *Rl = sm.vec + VMC_MAX_N, *Wh = sm.vec + 2 * VMC_MAX_N,
        *Wl = sm.vec + 3 * VMC_MAX_N, *Bh = sm.vec + 4 * VMC_MAX_N, *Bl = sm.vec + 5 * VMC_MAX_N,
        *Zh = sm.vec + 6 * VMC_MAX_N, *Zl = sm.vec + 7 * VMC_MAX_N;
  double cp = 0.0;
  if (tid < N) {
    df_split(tid == m ? S.f64[(size_t)j * Ns + i] : S.f64[(size_t)j * Ns + sm.ele[N + tid]],
             Rh[tid], Rl[tid]);
    const int site = (tid == n) ? j : sm.ele[tid];
    const double ck = S.fT64[(size_t)i * Ns + site];
    const double mk = S.fT64[(size_t)j * Ns + sm.ele[tid]];
    df_split(tid == n ? 0.0 : ck - mk, Bh[tid], Bl[tid]);
    cp = (tid == n) ? mk : ck;
    Zh[tid] = sm.minv[m * ldm + tid];
    Zl[tid] = sm.mlo[m * ldm + tid];
  }
  __syncthreads();
  double t12 = 0.0, t22 = 0.0;
  if (tid < N) {
    float wh, wl;
    df_col_dot(sm.minv, sm.mlo, ldm, tid, Rh, Rl, N, wh, wl);
    Wh[tid] = wh;
    Wl[tid] = wl;
    if (tid != n) t12 = df_val(wh, wl) * df_val(Bh[tid], Bl[tid]);
    t22 = df_val(Zh[tid], Zl[tid]) * cp;
  }
  double K12, K22;
  block_sum2(t12, t22, sm.dred, buf, K12, K22);
  const double K11 = df_val(Wh[n], Wl[n]), K21 = df_val(Zh[n], Zl[n]);
  const double inv = 1.0 / (K11 * K22 - K12 * K21);
  if (tid < N) {
    float *rh = sm.minv + tid * ldm, *rl = sm.mlo + tid * ldm;
    float qh, ql;
    df_row_dot(rh, rl, Bh, Bl, N, qh, ql);
    const double p = df_val(rh[n], rl[n]), q = df_val(qh, ql);
    float c1h, c1l, c2h, c2l;
    df_split((p * K22 - q * K21) * inv, c1h, c1l);
    df_split((q * K11 - p * K12) * inv, c2h, c2l);
    df_row_axpy(rh, rl, Wh, Wl, c1h, c1l, N);
    df_row_axpy(rh, rl, Zh, Zl, c2h, c2l, N);
    float h = rh[n], l = rl[n];
    df_fma(h, l, c1h, c1l, 1.0f, 0.0f);
    rh[n] = h;
    rl[n] = l;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Delayed updates: up to kd accepted hops are kept as rank-1 pairs, so that
// G = G0 - sum_{i<np} u_i v_i^T; ratios read G through the correction above
// and the pairs are folded into G0 by one rank-np product (flush).
// ---------------------------------------------------------------------------

// G0 <- G0 - U V^T: thread l owns row l, CH columns at a time in registers;
// the v_i entries are broadcast reads.
template <typename T>
__device__ void delayed_flush(const SysDev &S, const WSmem<T> &sm, int &np) {
  if (np == 0) return;
  const int N = S.N, ldm = S.ldm, tid = threadIdx.x;
  if (tid < N) {
    T *row = sm.minv + tid * ldm;
    int c = 0;
    for (; c + CH <= N; c += CH) {
      T a[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) a[u] = row[c + u];
      for (int i = 0; i < np; ++i) {
        const T ul = sm.ut[i * N + tid];
        const T *v = sm.vt + i * N + c;
#pragma unroll
        for (int u = 0; u < CH; ++u) a[u] -= ul * v[u];
      }
#pragma unroll
      for (int u = 0; u < CH; ++u) row[c + u] = a[u];
    }
    for (; c < N; ++c) {
      T a = row[c];
      for (int i = 0; i < np; ++i) a -= sm.ut[i * N + tid] * sm.vt[i * N + c];
      row[c] = a;
    }
  }
  np = 0;
  __syncthreads();
}

// Accepted hop of electron e (new row / column of M in vA), delayed form.
// Up electron n = e (row n of M replaced by R): w = R^T G, u = G[:,n] / w_n,
// v = w - e_n.  Down electron m = e - N (column m replaced by C): y = G C,
// u = (y - e_m) / y_m, v = G[m,:].  Both are the rank-1 updates of
// row_update / col_update; G[:,n] or G[m,:] was kept by hop_pf_ratio.
template <typename T>
__device__ void delayed_hop_update(const SysDev &S, const WSmem<T> &sm, int e, int &np) {
  const int N = S.N, ldm = S.ldm, tid = threadIdx.x;
  T *vA = sm.vec, *vB = sm.vec + VMC_MAX_N, *vE = sm.vec + 4 * VMC_MAX_N,
    *vz = sm.vec + 5 * VMC_MAX_N;
  const bool up = e < N;
  T d = (T)0;
  if (tid < N) d = up ? col_dot(sm.minv, ldm, tid, vA, N) : row_dot(sm.minv + tid * ldm, vA, N);
  if (np > 0) {
    pending_dots(up ? sm.ut : sm.vt, vA, N, np, vz);
    __syncthreads();
    if (tid < N) {
      const T *y = up ? sm.vt : sm.ut;
      for (int i = 0; i < np; ++i) d -= vz[i] * y[i * N + tid];
    }
  }
  if (tid < N) vB[tid] = d;
  __syncthreads();
  const int k = up ? e : e - N;
  const T inv = (T)1 / vB[k];
  if (tid < N) {
    const T dk = (tid == k) ? (T)1 : (T)0;
    if (up) {
      sm.ut[np * N + tid] = vE[tid] * inv;
      sm.vt[np * N + tid] = d - dk;
    } else {
      sm.ut[np * N + tid] = (d - dk) * inv;
      sm.vt[np * N + tid] = vE[tid];
    }
  }
  ++np;
  __syncthreads();
  if (np >= S.delay_k) delayed_flush(S, sm, np);
}

// ---------------------------------------------------------------------------
// One Metropolis proposal (Sec. 3.1.2).  Every thread runs it; decisions are
// uniform across the block.
// ---------------------------------------------------------------------------
template <typename T>
__device__ void propose(const SysDev &S, const WSmem<T> &sm, uint2 key, uint32_t walker,
                        unsigned long long &ctr, int &rpos, MoveCounts &mc, int &acc_since,
                        int &buf, int &np) {
  const int N = S.N, Ns = S.Ns, Ne = S.Ne, tid = threadIdx.x;
  if (rpos == RB) {
    // Next RB draws of this walker's stream, one per thread of the first warp.
    __syncthreads();
    if (tid < RB) {
      const unsigned long long c = ctr + tid;
      sm.rnd[tid] = vmc_philox(make_uint4((uint32_t)c, (uint32_t)(c >> 32), walker,
                                          (uint32_t)S.sys_index), key);
    }
    __syncthreads();
    rpos = 0;
  }
  const uint4 r = sm.rnd[rpos++];
  ctr++;
  const T u = (T)(r.w >> 8) * (T)(1.0 / 16777216.0);
  if ((unsigned long long)r.x < S.pex) {
    const int n = vmc_mulhi(r.y, N);
    const int m = N + vmc_mulhi(r.z, N);
    const int i = sm.ele[n], j = sm.ele[m];
    if (i == j || sm.occ[Ns + i] >= 0 || sm.occ[j] >= 0) return;
    mc.ex_t++;
    T K[4], mlp;
    const T rpf = exchange_pf_ratio(S, sm, n, m - N, i, j, buf, K, mlp, np);
    const T ratio = S.n_hidden ? rpf * exp_t<T>(mlp) : rpf;
    if (u < ratio * ratio) {
      delayed_flush(S, sm, np);
      if constexpr (std::is_same<T, float>::value) {
        if (sm.mlo && S.delay_k <= 1) exchange_update_df(S, sm, n, m - N, i, j, buf);
        else exchange_update(S, sm, n, m - N, j, K, rpf);
      } else {
        exchange_update(S, sm, n, m - N, j, K, rpf);
      }
      if (S.n_hidden) mlp_apply(S, sm, i + Ns, i, j, j + Ns);
      if (tid == 0) {
        sm.ele[n] = j;
        sm.ele[m] = i;
        sm.occ[i] = -1;
        sm.occ[j] = n;
        sm.occ[Ns + j] = -1;
        sm.occ[Ns + i] = m;
      }
      __syncthreads();
      mc.ex_a++;
      acc_since = (fabs((double)rpf) < SMALL_RATIO) ? RECOMPUTE_NOW : acc_since + 1;
    }
    return;
  }
  const int e = vmc_mulhi(r.y, Ne);
  const int t = vmc_mulhi(r.z, Ns);
  const int s = (e >= N) ? 1 : 0;
  if (sm.occ[s * Ns + t] >= 0) return;
  if (S.local_spin && sm.occ[(1 - s) * Ns + t] >= 0) return;
  const int rs = sm.ele[e];
  // Kondo local spins hold one electron each: no hop enters or leaves them
  if (S.lsite && (S.lsite[t] | S.lsite[rs])) return;
  mc.hop_t++;
  // P(x')/P(x): one thread evaluates it; the barrier inside hop_pf_ratio publishes it.
  const int slot = buf;
  if (tid == 0)
    sm.bc[slot] = corr_factor<T>(corr_hop_v(sm.occ, sm.jf, gtab<T>(S), Ns, s, rs, t,
                                            vtab<T>(S)[(size_t)rs * Ns + t]));
  // rows t and r of v for the Jastrow-field update, fetched while the ratio is formed
  T vt[2], vr[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int x = tid + u * NT;
    vt[u] = (x < Ns) ? vtab<T>(S)[(size_t)t * Ns + x] : (T)0;
    vr[u] = (x < Ns) ? vtab<T>(S)[(size_t)rs * Ns + x] : (T)0;
  }
  T fval, mlp;
  const T rpf = hop_pf_ratio(S, sm, e, t, fval, buf, mlp, np);
  const T ratio = S.n_hidden ? rpf * sm.bc[slot] * exp_t<T>(mlp) : rpf * sm.bc[slot];
  if (!(u < ratio * ratio)) return;
  if (tid < N) sm.vec[tid] = fval;
  __syncthreads();
  bool done = false;
  if constexpr (std::is_same<T, float>::value) {
    if (sm.mlo && S.delay_k <= 1) {
      if (s == 0) row_update_df(S, sm, e, t);
      else col_update_df(S, sm, e - N, t);
      done = true;
    }
  }
  if (done) {
  } else if (S.delay_k > 1) {
    delayed_hop_update(S, sm, e, np);
  } else if (s == 0) {
    row_update(S, sm, e);
  } else {
    col_update(S, sm, e - N);
  }
  if (S.n_hidden) mlp_apply(S, sm, t + s * Ns, rs + s * Ns, -1, -1);
  // Jastrow field: h_x += v_{x t} - v_{x r}.
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int x = tid + u * NT;
    if (x < Ns) sm.jf[x] += vt[u] - vr[u];
  }
  for (int x = tid + 2 * NT; x < Ns; x += NT)
    sm.jf[x] += vtab<T>(S)[(size_t)t * Ns + x] - vtab<T>(S)[(size_t)rs * Ns + x];
  if (tid == 0) {
    sm.ele[e] = t;
    sm.occ[s * Ns + rs] = -1;
    sm.occ[s * Ns + t] = e;
  }
  __syncthreads();
  mc.hop_a++;
  acc_since = (fabs((double)rpf) < SMALL_RATIO) ? RECOMPUTE_NOW : acc_since + 1;
}

// ---------------------------------------------------------------------------
// Proposals formed in batches (Sec. 3.1.2 proposals, one Markov chain)
// ---------------------------------------------------------------------------
// The next B proposals of the walker's stream are checked and their ratios
// formed together, against the current configuration and inverse; the
// Metropolis decisions are then taken in the stream's order, and the batch
// ends at the first accepted proposal, whose move is made as propose() makes
// it.  The proposals after it are formed again, against the updated state, by
// the next batch.  The chain is therefore the one propose() gives proposal by
// proposal (only the ratios' summation order differs); what changes is the
// cost: the exchanges of a batch share one pass over M^-1, the batch's table
// gathers are in flight together, and a batch has two block barriers where a
// proposal had two or three.  Used when the MLP factor and delayed updates
// are off.
constexpr int SPEC_MAX = 8;

// Per-warp partial sums of a batch: NWARP x 32 values (inside the O-row
// accumulator area, which only the measurement uses).
template <typename T>
__host__ __device__ constexpr size_t spec_scratch_bytes() {
  return sizeof(T) * NWARP * 32;
}

// One step of a transposed butterfly over 2H values per lane: lanes with bit
// H set keep the upper half, the others the lower half, and each adds its
// partner's copy of the half it keeps.
template <int H, typename T>
__device__ __forceinline__ void tb_step(T *p, int lane) {
  const bool up = lane & H;
#pragma unroll
  for (int k = 0; k < H; ++k) {
    const T send = up ? p[k] : p[k + H];
    const T keep = up ? p[k + H] : p[k];
    p[k] = keep + __shfl_xor_sync(0xffffffffu, send, H);
  }
}

// Warp sums of 32 per-lane values (31 shuffles): lane l returns the total of
// value l.
template <typename T>
__device__ __forceinline__ T reduce32_transposed(T *p, int lane) {
  tb_step<16>(p, lane);
  tb_step<8>(p, lane);
  tb_step<4>(p, lane);
  tb_step<2>(p, lane);
  tb_step<1>(p, lane);
  return p[0];
}

// w_q = sum_l R_q[l] M[l][col] for the Q rows R_q in vector slots 0..Q-1:
// one pass over the column, two accumulators per row.
template <int Q, typename T>
__device__ __forceinline__ void spec_gemv(const T *M, int ldm, int col, const T *vec, int N,
                                          T *w) {
  T a[Q], b[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    a[q] = (T)0;
    b[q] = (T)0;
  }
  int l = 0;
  for (; l + 4 <= N; l += 4) {
    const T m0 = M[l * ldm + col], m1 = M[(l + 1) * ldm + col];
    const T m2 = M[(l + 2) * ldm + col], m3 = M[(l + 3) * ldm + col];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      T x0, x1, x2, x3;
      ld4(vec + q * VMC_MAX_N + l, x0, x1, x2, x3);
      a[q] += x0 * m0;
      b[q] += x1 * m1;
      a[q] += x2 * m2;
      b[q] += x3 * m3;
    }
  }
  for (; l < N; ++l) {
    const T m0 = M[l * ldm + col];
#pragma unroll
    for (int q = 0; q < Q; ++q) a[q] += vec[q * VMC_MAX_N + l] * m0;
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) w[q] = a[q] + b[q];
}

template <typename T>
__device__ __forceinline__ void spec_gemv_n(int Q, const T *M, int ldm, int col, const T *vec,
                                            int N, T *w) {
  switch (Q) {
    case 1: spec_gemv<1>(M, ldm, col, vec, N, w); break;
    case 2: spec_gemv<2>(M, ldm, col, vec, N, w); break;
    case 3: spec_gemv<3>(M, ldm, col, vec, N, w); break;
    case 4: spec_gemv<4>(M, ldm, col, vec, N, w); break;
    case 5: spec_gemv<5>(M, ldm, col, vec, N, w); break;
    case 6: spec_gemv<6>(M, ldm, col, vec, N, w); break;
    case 7: spec_gemv<7>(M, ldm, col, vec, N, w); break;
    default: spec_gemv<8>(M, ldm, col, vec, N, w); break;
  }
}

// a[q] for a thread-varying q < SPEC_MAX without local-memory indexing
template <typename T>
__device__ __forceinline__ T sel_spec(const T *a, int q) {
  T r = a[0];
#pragma unroll
  for (int k = 1; k < SPEC_MAX; ++k) r = (q == k) ? a[k] : r;
  return r;
}

// One batch of at most bmax proposals; returns how many it consumed.  Every
// thread runs it; decisions are uniform across the block.  Each warp decodes
// and checks the batch's proposals itself (lane b takes proposal b), so the
// descriptors travel by shuffles; the per-thread products go through one
// transposed reduction per warp and one barrier.
template <typename T>
__device__ int propose_batch(const SysDev &S, const WSmem<T> &sm, uint2 key, uint32_t walker,
                             unsigned long long &ctr, int &rpos, MoveCounts &mc, int &acc_since,
                             int &buf, int bmax) {
  const int N = S.N, Ns = S.Ns, Ne = S.Ne, ldm = S.ldm, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const unsigned full = 0xffffffffu;
  const T *F = ftab<T>(S);
  const T *FT = fTtab<T>(S);
  int B = S.spec_b < SPEC_MAX ? S.spec_b : SPEC_MAX;
  if (B > bmax) B = bmax;
  if (rpos + B > RB) {
    // draws ctr .. ctr + RB - 1 (the stream is indexed by the counter, so a
    // refill at any position gives the draws proposal by proposal would use)
    if (tid < RB) {
      const unsigned long long c = ctr + tid;
      sm.rnd[tid] = vmc_philox(make_uint4((uint32_t)c, (uint32_t)(c >> 32), walker,
                                          (uint32_t)S.sys_index), key);
    }
    __syncthreads();
    rpos = 0;
  }
  // --- decode and check (lane b: proposal b), as propose() does
  int kind = 0, x0 = 0, x1 = 0, x2 = 0, x3 = 0;   // 1 up hop, 2 down hop, 3 exchange
  T u = (T)1, cf = (T)0;
  if (lane < B) {
    const uint4 r = sm.rnd[rpos + lane];
    u = (T)(r.w >> 8) * (T)(1.0 / 16777216.0);
    if ((unsigned long long)r.x < S.pex) {
      const int n = vmc_mulhi(r.y, N), m = vmc_mulhi(r.z, N);
      const int i = sm.ele[n], j = sm.ele[N + m];
      if (!(i == j || sm.occ[Ns + i] >= 0 || sm.occ[j] >= 0)) {
        kind = 3;
        x0 = n;
        x1 = m;
        x2 = i;
        x3 = j;
      }
    } else {
      const int e = vmc_mulhi(r.y, Ne), t = vmc_mulhi(r.z, Ns);
      const int s = (e >= N) ? 1 : 0;
      bool ok = sm.occ[s * Ns + t] < 0;
      if (ok && S.local_spin && sm.occ[(1 - s) * Ns + t] >= 0) ok = false;
      const int rs = sm.ele[e];
      if (ok && S.lsite && (S.lsite[t] | S.lsite[rs])) ok = false;
      if (ok) {
        kind = 1 + s;
        x0 = s ? e - N : e;
        x1 = t;
        x2 = rs;
        cf = corr_factor<T>(corr_hop_v(sm.occ, sm.jf, gtab<T>(S), Ns, s, rs, t,
                                       vtab<T>(S)[(size_t)rs * Ns + t]));
      }
    }
  }
  const unsigned exm = __ballot_sync(full, kind == 3);
  const unsigned hpm = __ballot_sync(full, kind == 1 || kind == 2);
  const int nex = __popc(exm);
  // --- per-thread products: hop ratios' terms; the exchanges' new rows R_q
  // (vector slot q, in the order of the batch) and their row-m and b terms
  // values: [b] hop term or K22 term, [8 + b] K12 term, [16 + b] K11 (w_n)
  T val[32], bk[SPEC_MAX];
  // per slot: exchange row slot q, or -1; and whether this thread is its row n
  int xq[SPEC_MAX];
  unsigned isn = 0;
  const int tr = (tid < N) ? tid : 0;
  const int eup = sm.ele[tr], edn = sm.ele[N + tr];
  // All table gathers of the batch are issued before any is used (branch-free
  // address selection; a slot that fails the checks reads entry 0), so the
  // batch pays one L2 round trip, not one per proposal.
  T g1[SPEC_MAX], g2[SPEC_MAX], g3[SPEC_MAX], s1[SPEC_MAX];
  int kd[SPEC_MAX], z0[SPEC_MAX];
#pragma unroll
  for (int b = 0; b < SPEC_MAX; ++b) {
    const int bb = b < B ? b : 0;
    const int k = __shfl_sync(full, kind, bb);
    const int y0 = __shfl_sync(full, x0, bb), y1 = __shfl_sync(full, x1, bb);
    const int y2 = __shfl_sync(full, x2, bb), y3 = __shfl_sync(full, x3, bb);
    kd[b] = (b < B) ? k : 0;
    z0[b] = y0;
    // up hop (e = y0 to t = y1): f(t, r_tid,dn) and (M^-1)_{tid e}
    // down hop (m = y0 to t = y1): f(r_tid,up, t) and (M^-1)_{m tid}
    // exchange (n = y0 at i = y2, m = y1 at j = y3): R_tid, C_tid, f(r_tid,up, j), (M^-1)_{m tid}
    const T *t1 = (k == 2) ? FT : F;
    const size_t r1 = (k == 3) ? (size_t)y3 : (size_t)y1;
    const int c1 = (k == 2) ? eup : (k == 3 && tid == y1) ? y2 : edn;
    const int site = (tid == y0) ? y3 : eup;
    const bool ex = (k == 3);
    const int mi = (k == 1) ? tr * ldm + y0 : y1 * ldm + tr;
    g1[b] = t1[(k != 0) ? r1 * Ns + c1 : 0];
    g2[b] = FT[ex ? (size_t)y2 * Ns + site : 0];
    g3[b] = FT[ex ? (size_t)y3 * Ns + eup : 0];
    s1[b] = sm.minv[(k == 2) ? y0 * ldm + tr : ((k != 0) ? mi : 0)];
  }
#pragma unroll
  for (int b = 0; b < 32; ++b) val[b] = (T)0;
#pragma unroll
  for (int b = 0; b < SPEC_MAX; ++b) {
    bk[b] = (T)0;
    xq[b] = -1;
    const int k = kd[b];
    if (k == 3) xq[b] = __popc(exm & ((1u << b) - 1));
    if (tid < N) {
      if (k == 1 || k == 2) {
        val[b] = g1[b] * s1[b];
      } else if (k == 3) {
        if (tid == z0[b]) isn |= 1u << b;
        sm.vec[xq[b] * VMC_MAX_N + tid] = g1[b];
        val[b] = (tid == z0[b]) ? s1[b] * g3[b] : s1[b] * g2[b];
        bk[b] = (tid == z0[b]) ? (T)0 : g2[b] - g3[b];
      }
    }
  }
  __syncthreads();
  // --- one pass over M^-1 for all exchanges: w_q = R_q^T M^-1 (column tid)
  T wq[SPEC_MAX];
#pragma unroll
  for (int q = 0; q < SPEC_MAX; ++q) wq[q] = (T)0;
  if (nex > 0 && tid < N) spec_gemv_n(nex, sm.minv, ldm, tid, sm.vec, N, wq);
#pragma unroll
  for (int b = 0; b < SPEC_MAX; ++b) {
    if (xq[b] >= 0) {
      const T w = sel_spec(wq, xq[b]);
      val[SPEC_MAX + b] = w * bk[b];
      val[2 * SPEC_MAX + b] = ((isn >> b) & 1u) ? w : (T)0;
    }
  }
  const T tot = reduce32_transposed(val, lane);
  T *part = sm.acc;
  if (lane < 3 * SPEC_MAX) part[warp * 32 + lane] = tot;
  __syncthreads();
  // --- decisions in the stream's order (every warp takes the same ones)
  bool acc = false;
  T rpf = (T)0;
  if (lane < B && kind != 0) {
    T s0 = part[lane], s1 = part[SPEC_MAX + lane], s2 = part[2 * SPEC_MAX + lane];
#pragma unroll
    for (int k = 1; k < NWARP; ++k) {
      s0 += part[k * 32 + lane];
      s1 += part[k * 32 + SPEC_MAX + lane];
      s2 += part[k * 32 + 2 * SPEC_MAX + lane];
    }
    T ratio;
    if (kind == 3) {
      // det [[K11, K12], [K21, K22]] with K21 = (M^-1)_{mn}
      rpf = s2 * s0 - s1 * sm.minv[x1 * ldm + x0];
      ratio = rpf;
    } else {
      rpf = s0;
      ratio = rpf * cf;
    }
    acc = u < ratio * ratio;
  }
  const unsigned am = __ballot_sync(full, acc);
  const int ka = am ? __ffs(am) - 1 : -1;
  const int used = (ka >= 0) ? ka + 1 : B;
  const unsigned usedm = (used >= 32) ? full : ((1u << used) - 1u);
  mc.hop_t += __popc(hpm & usedm);
  mc.ex_t += __popc(exm & usedm);
  ctr += (unsigned long long)used;
  rpos += used;
  if (ka < 0) return used;
  // --- the accepted proposal ka: its move, as propose() makes it
  const int k = __shfl_sync(full, kind, ka);
  const int y0 = __shfl_sync(full, x0, ka), y1 = __shfl_sync(full, x1, ka);
  const int y2 = __shfl_sync(full, x2, ka), y3 = __shfl_sync(full, x3, ka);
  const T rk = __shfl_sync(full, rpf, ka);
  if (k == 3) {
    const int n = y0, m = y1, i = y2, j = y3;
    bool done = false;
    if constexpr (std::is_same<T, float>::value) {
      if (sm.mlo) {
        exchange_update_df(S, sm, n, m, i, j, buf);
        done = true;
      }
    }
    if (!done) {
      // the rank-2 update wants w = R^T M^-1, C and K as exchange_pf_ratio leaves them
      T K[4], mlp;
      const T r2 = exchange_pf_ratio(S, sm, n, m, i, j, buf, K, mlp, 0);
      exchange_update(S, sm, n, m, j, K, r2);
    }
    if (tid == 0) {
      sm.ele[n] = j;
      sm.ele[N + m] = i;
      sm.occ[i] = -1;
      sm.occ[j] = n;
      sm.occ[Ns + j] = -1;
      sm.occ[Ns + i] = N + m;
    }
    __syncthreads();
    mc.ex_a++;
  } else {
    const int s = k - 1, e = s ? y0 + N : y0, t = y1, rs = y2;
    bool done = false;
    if constexpr (std::is_same<T, float>::value) {
      if (sm.mlo) {
        if (s == 0) row_update_df(S, sm, e, t);
        else col_update_df(S, sm, e - N, t);
        done = true;
      }
    }
    if (!done) {
      if (tid < N) sm.vec[tid] = s ? FT[(size_t)t * Ns + eup] : F[(size_t)t * Ns + edn];
      __syncthreads();
      if (s == 0) row_update(S, sm, e);
      else col_update(S, sm, e - N);
    }
    // Jastrow field: h_x += v_{x t} - v_{x r}.
    for (int x = tid; x < Ns; x += NT)
      sm.jf[x] += vtab<T>(S)[(size_t)t * Ns + x] - vtab<T>(S)[(size_t)rs * Ns + x];
    if (tid == 0) {
      sm.ele[e] = t;
      sm.occ[s * Ns + rs] = -1;
      sm.occ[s * Ns + t] = e;
    }
    __syncthreads();
    mc.hop_a++;
  }
  acc_since = (fabs((double)rk) < SMALL_RATIO) ? RECOMPUTE_NOW : acc_since + 1;
  return used;
}

// Sum of eight per-lane values over the warp by a transposed butterfly
// (nine shuffles instead of eight separate reductions): on return lane l
// holds the total of value k = 4 bit4(l) + 2 bit3(l) + bit2(l).
template <typename T>
__device__ __forceinline__ T reduce8_transposed(const T *p, int lane) {
  T q[4], r[2];
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const T send = b4 ? p[k] : p[k + 4];
    const T keep = b4 ? p[k + 4] : p[k];
    q[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const T send = b3 ? q[k] : q[k + 2];
    const T keep = b3 ? q[k + 2] : q[k];
    r[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  T s = (b2 ? r[1] : r[0]) + __shfl_xor_sync(0xffffffffu, b2 ? r[0] : r[1], 4);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  return s;
}

// ---------------------------------------------------------------------------
// Measurement: E_loc (Eq. MC with A = H) and the O_k row (Sec. 3.3.1)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void acc_add(T *p, T v) { atomicAdd(p, v); }

// a[r] for a warp-varying r < 4 without local-memory indexing
template <typename V>
__device__ __forceinline__ V sel4(const V *a, int r) {
  return r == 0 ? a[0] : r == 1 ? a[1] : r == 2 ? a[2] : a[3];
}

template <typename T>
__device__ void measure(const SysDev &S, const WSmem<T> &sm, int w, int row, int &buf,
                        MoveCounts &mc) {
  const int N = S.N, Ns = S.Ns, ldm = S.ldm, tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const T *F = ftab<T>(S);
  const T *FT = fTtab<T>(S);
  // --- diagonal terms (per-thread partial sums in T, one FP64 block sum)
  T ed = (T)0;
  for (int i = tid; i < Ns; i += NT) {
    const int up = sm.occ[i] >= 0, dn = sm.occ[Ns + i] >= 0;
    if (up && dn) ed += (T)S.U[i];
  }
  for (int k = tid; k < S.n_V; k += NT) {
    const int a = S.V_i[k], b = S.V_j[k];
    const int na = (sm.occ[a] >= 0) + (sm.occ[Ns + a] >= 0);
    const int nb = (sm.occ[b] >= 0) + (sm.occ[Ns + b] >= 0);
    ed += (T)S.V_val[k] * (T)(na * nb);
  }
  for (int k = tid; k < S.n_J; k += NT) {
    const int a = S.J_i[k], b = S.J_j[k];
    const int sa = (sm.occ[a] >= 0) - (sm.occ[Ns + a] >= 0);
    const int sb = (sm.occ[b] >= 0) - (sm.occ[Ns + b] >= 0);
    ed += (T)S.J_val[k] * (T)(0.25f * (float)(sa * sb));
  }
  // --- hopping, one warp per target site i: the warp gathers the rows
  // f(i, r_m,dn) and f(r_n,up, i) once (lane-strided) and, one term per lane,
  // the source sites j, t_ij and v_ji.  The Green-function ratios of up to
  // four neighbouring sites (both spins: eight dot products with a column or
  // row of M^-1) are formed together, reduced by one transposed butterfly
  // (lane 4k ends with the sum for term k), and their correlation-factor
  // ratios are evaluated by those eight lanes in parallel.
  T eo = (T)0;
  const T *TV = tvtab<T>(S);
  // Gathers for site i are issued one site ahead (software pipelining).
  T gu[4], gd[4], nu[4], nd[4];
  int jl = 0, njl = 0;
  T tl = (T)0, vl = (T)0, ntl = (T)0, nvl = (T)0;
  // term ranges of the target sites, staged in shared memory (ilist is free
  // until the O_v part): kb(i) = tp[i], ke(i) = tp[i + 1] or n_hop
  int *tp = sm.ilist;
  for (int i = tid; i < Ns; i += NT) tp[i] = S.tgt_ptr[i];
  __syncthreads();
  auto t_end = [&](int i) { return i + 1 < Ns ? tp[i + 1] : S.n_hop; };
  auto fetch = [&](int i, T *u4, T *d4, int &jj, T &tt, T &vv) {
    const bool uf = sm.occ[i] < 0, df = sm.occ[Ns + i] < 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int q = lane + 32 * u;
      u4[u] = (uf && q < N) ? F[(size_t)i * Ns + sm.ele[N + q]] : (T)0;
      d4[u] = (df && q < N) ? FT[(size_t)i * Ns + sm.ele[q]] : (T)0;
    }
    const int kb = tp[i], ke = t_end(i);
    jj = 0;
    tt = vv = (T)0;
    if (kb + lane < ke) {
      jj = S.tgt_j[kb + lane];
      tt = (T)S.tgt_t[kb + lane];
      vv = TV[kb + lane];
    }
  };
  const int tix = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
  if (warp < Ns) fetch(warp, gu, gd, jl, tl, vl);
  for (int i = warp; i < Ns; i += NWARP) {
    const int inext = i + NWARP;
    if (inext < Ns) fetch(inext, nu, nd, njl, ntl, nvl);
    const int kb = tp[i], ke = t_end(i);
    const bool up_free = sm.occ[i] < 0, dn_free = sm.occ[Ns + i] < 0;
    if (kb < ke && (up_free || dn_free)) {
      for (int q0 = kb; q0 < ke; q0 += 32) {
        int jc = jl;
        T tc = tl, vc = vl;
        if (q0 > kb) {   // more than 32 terms: load this chunk directly
          jc = 0;
          tc = vc = (T)0;
          if (q0 + lane < ke) {
            jc = S.tgt_j[q0 + lane];
            tc = (T)S.tgt_t[q0 + lane];
            vc = TV[q0 + lane];
          }
        }
        const int nq = min(32, ke - q0);
        for (int g0 = 0; g0 < nq; g0 += 4) {
          // terms 2r (up electron on j_r -> i) and 2r+1 (down electron), r < 4
          int jr[4], eur[4], edr[4];
          T tr[4], vr[4];
          bool any = false;
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const bool ex = g0 + r < nq;
            jr[r] = __shfl_sync(0xffffffffu, jc, (g0 + r) & 31);
            tr[r] = __shfl_sync(0xffffffffu, tc, (g0 + r) & 31);
            vr[r] = __shfl_sync(0xffffffffu, vc, (g0 + r) & 31);
            eur[r] = (ex && up_free) ? sm.occ[jr[r]] : -1;
            edr[r] = (ex && dn_free) ? sm.occ[Ns + jr[r]] : -1;
            any |= eur[r] >= 0 || edr[r] >= 0;
          }
          if (!any) continue;
          // Branch-free: absent terms read column / row 0 and are masked, so
          // all 32 shared loads can be in flight together (gu, gd are 0 for
          // q >= N; q is clamped to a valid row).
          T p[8];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int cu = max(eur[r], 0), rd = max(edr[r] - N, 0);
            T su = (T)0, sd = (T)0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int q = min(lane + 32 * u, N - 1);
              su += gu[u] * sm.minv[q * ldm + cu];
              sd += gd[u] * sm.minv[rd * ldm + q];
            }
            p[2 * r] = eur[r] >= 0 ? su : (T)0;
            p[2 * r + 1] = edr[r] >= 0 ? sd : (T)0;
          }
          const T sum = reduce8_transposed(p, lane);
          // this lane's term: r = tix >> 1, spin = tix & 1
          const int r = tix >> 1, sp = tix & 1;
          const int j = sel4(jr, r);
          const int el = sp ? sel4(edr, r) : sel4(eur, r);
          T lm = (T)0;
          if (S.n_hidden) {
            T mq[8];
#pragma unroll
            for (int rr = 0; rr < 4; ++rr) {
              mq[2 * rr] = eur[rr] >= 0 ? mlp_log_ratio_part(S, sm, i, jr[rr], -1, -1, lane, 32) : (T)0;
              mq[2 * rr + 1] =
                  edr[rr] >= 0 ? mlp_log_ratio_part(S, sm, i + Ns, jr[rr] + Ns, -1, -1, lane, 32) : (T)0;
            }
            lm = reduce8_transposed(mq, lane);
          }
          if ((lane & 3) == 0 && el >= 0) {
            const T c = corr_factor<T>(corr_hop_v(sm.occ, sm.jf, gtab<T>(S), Ns, sp, j, i, sel4(vr, r)));
            eo += -sel4(tr, r) * sum * c * (S.n_hidden ? exp_t<T>(lm) : (T)1);
            mc.meas_hop++;
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      gu[u] = nu[u];
      gd[u] = nd[u];
    }
    jl = njl;
    tl = ntl;
    vl = nvl;
  }
  // --- Heisenberg exchange: J/2 (S+_a S-_b + S-_a S+_b) = -J/2 x (labelled swap ratio).
  // The terms are taken by the site b that receives the up electron (b holds
  // exactly a down electron m, a exactly an up electron n).  The new row of
  // every such term differs from f(b, r_dn) only in entry m, so
  // w = R^T M^-1 = g_b + (f(b, a) - f(b, b)) M^-1[m,:] with g_b = f(b, r_dn)^T M^-1
  // formed once per site by one warp (lanes over columns), and each term is
  // the 2 x 2 determinant of exchange_pf_ratio in O(N).
  T *R = sm.vec + (2 * warp) * VMC_MAX_N;
  __syncthreads();   // vec area switches from proposal use to per-warp use
  if (S.n_J > 0) {
    const unsigned full = 0xffffffffu;
    for (int b = warp; b < Ns; b += NWARP) {
      const int md = sm.occ[Ns + b];
      if (md < 0 || sm.occ[b] >= 0) continue;
      const int q0 = S.jptr[b], q1 = S.jptr[b + 1];
      bool any = false;
      for (int q = q0 + lane; q < q1; q += 32) {
        const int a = S.jadj[q].y;
        any |= (sm.occ[a] >= 0 && sm.occ[Ns + a] < 0);
      }
      if (!__any_sync(full, any)) continue;
      const int m = md - N;
      for (int l = lane; l < N; l += 32) R[l] = F[(size_t)b * Ns + sm.ele[N + l]];
      __syncwarp();
      // lane holds columns k = lane + 32 u: g_b[k], (M^-1)_{mk}, r_k,up, f(r_k,up, b)
      T g[4], mr[4], mk[4];
      int ek[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = lane + 32 * u;
        g[u] = (T)0;
        mr[u] = (k < N) ? sm.minv[m * ldm + k] : (T)0;
        ek[u] = (k < N) ? sm.ele[k] : 0;
        mk[u] = (k < N) ? FT[(size_t)b * Ns + ek[u]] : (T)0;
      }
      int l = 0;
      for (; l + 4 <= N; l += 4) {
        T r0, r1, r2, r3;
        ld4(R + l, r0, r1, r2, r3);
        const T *m0 = sm.minv + l * ldm;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int k = lane + 32 * u;
          if (k < N)
            g[u] += r0 * m0[k] + r1 * m0[ldm + k] + r2 * m0[2 * ldm + k] + r3 * m0[3 * ldm + k];
        }
      }
      for (; l < N; ++l) {
        const T rl = R[l];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int k = lane + 32 * u;
          if (k < N) g[u] += rl * sm.minv[l * ldm + k];
        }
      }
      __syncwarp();   // R is written again for the warp's next site
      const T fbb = F[(size_t)b * Ns + b];
      for (int q = q0; q < q1; ++q) {
        const int2 tq = S.jadj[q];
        const int a = tq.y;
        const int n = sm.occ[a];
        if (n < 0 || sm.occ[Ns + a] >= 0) continue;
        const T delta = F[(size_t)b * Ns + a] - fbb;
        T a22 = (T)0, a12 = (T)0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int k = lane + 32 * u;
          if (k < N) {
            const T c = FT[(size_t)a * Ns + ((k == n) ? b : ek[u])];
            if (k == n) {
              a22 += mr[u] * mk[u];
            } else {
              a22 += mr[u] * c;
              a12 += (g[u] + delta * mr[u]) * (c - mk[u]);
            }
          }
        }
        a22 = warp_sum(a22);
        a12 = warp_sum(a12);
        const T gn = __shfl_sync(full, sel4(g, n >> 5), n & 31);
        const T A21 = sm.minv[m * ldm + n];
        const T r = (gn + delta * A21) * a22 - a12 * A21;
        const T lm =
            S.n_hidden ? warp_sum(mlp_log_ratio_part(S, sm, a + Ns, a, b, b + Ns, lane, 32)) : (T)0;
        if (lane == 0) {
          eo += (T)(-0.5 * S.J_val[tq.x]) * r * (S.n_hidden ? exp_t<T>(lm) : (T)1);
          mc.meas_ex++;
        }
      }
    }
  }
  const double etot = block_sum((double)ed + (double)eo, sm.dred, buf);
  if (tid == 0) S.E[(size_t)w * S.n_samples + row] = etot;

  // --- O_k row
  T *Orow = (T *)S.O + ((size_t)w * S.n_samples + row) * S.ldO;
  const bool sh = S.acc_len > 0;
  T *acc = sh ? sm.acc : Orow;
  const int len = sh ? S.acc_len : S.ldO;
  const int mlp_lo = S.n_hidden ? S.mlp_base : S.Np;   // the MLP part is written, not accumulated
  for (int k = tid; k < len; k += NT)
    if (sh || k < mlp_lo || k >= S.Np) acc[k] = (T)0;
  if (tid == 0) sm.misc[0] = 0;
  __syncthreads();
  if (S.n_g > 0) {
    for (int i = tid; i < Ns; i += NT)
      if (sm.occ[i] >= 0 && sm.occ[Ns + i] >= 0 && S.g_idx[i] >= 0) acc_add(acc + S.g_idx[i], (T)1);
  }
  if (S.n_v > 0 && !S.local_spin) {
    // O_v(class) = sum over the class's pairs i < j of m_i m_j, m = n - 1:
    // one warp per class over its pair list, integer sums, no atomics.
    // (Under the local-spin constraint every m_i = 0 and O_v = 0.)
    int *mval = sm.ilist;
    for (int i = tid; i < Ns; i += NT) mval[i] = (sm.occ[i] >= 0) + (sm.occ[Ns + i] >= 0) - 1;
    __syncthreads();
    for (int c = warp; c < S.n_v; c += NWARP) {
      int acc_i = 0;
      const int pe = S.vptr[c + 1];
#pragma unroll 4
      for (int q = S.vptr[c] + lane; q < pe; q += 32) {
        const unsigned pr = S.vpair[q];
        acc_i += mval[pr & 0xFFFFu] * mval[pr >> 16];
      }
      acc_i = warp_sum(acc_i);
      if (lane == 0) acc[S.n_g + c] = (T)acc_i;
    }
  }
  // Pair orbital: d ln Pf / d f_ab = (M^-1)_{mn} for a = r_n,up, b = r_m,dn
  // (= -(X^-1)_{n, N+m}, Eq. DiffPf / Appendix C), times the class sign.
  // One warp per up electron n (site a), lanes over the down electrons m;
  // two rows in flight; the class and sign come from one packed table.
  const int base = S.n_g + S.n_v;
  for (int n0 = warp; n0 < N; n0 += 2 * NWARP) {
    int code[2][4];
    T val[2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int n = n0 + h * NWARP;
      const int *frow = S.fcode + (size_t)(n < N ? sm.ele[n] : 0) * Ns;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int m = lane + 32 * u;
        const bool ok = n < N && m < N;
        code[h][u] = ok ? frow[sm.ele[N + m]] : -1;
        val[h][u] = ok ? sm.minv[m * ldm + n] : (T)0;
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int cd = code[h][u];
        if (cd >= 0) acc_add(acc + base + (cd >> 1), (cd & 1) ? -val[h][u] : val[h][u]);
      }
  }
  if (S.n_hidden) {
    // MLP factor: dW1_kc = w2_k (1 - t_k^2) n_c, db1_k = w2_k (1 - t_k^2),
    // dw2_k = t_k, db2 = 1, with t = tanh(h); n_c = occ[c] >= 0 (c = i + Ns s).
    const int H = S.n_hidden, C = 2 * Ns;
    const double *w2 = S.params + S.mlp_base + (size_t)H * C + H;
    T *Om = acc + S.mlp_base;
    for (size_t q = tid; q < (size_t)H * C; q += NT) {
      const int k = (int)(q / C), c = (int)(q - (size_t)k * C);
      const T tk = sm.th[k];
      Om[q] = (sm.occ[c] >= 0) ? (T)w2[k] * ((T)1 - tk * tk) : (T)0;
    }
    for (int k = tid; k < H; k += NT) {
      const T tk = sm.th[k];
      Om[(size_t)H * C + k] = (T)w2[k] * ((T)1 - tk * tk);
      Om[(size_t)H * C + H + k] = tk;
    }
    if (tid == 0) Om[(size_t)H * C + 2 * H] = (T)1;
  }
  __syncthreads();
  if (sh)
    for (int k = tid; k < S.ldO; k += NT) Orow[k] = (k < S.acc_len) ? acc[k] : (T)0;
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------
// MINB: the CTAs per SM the register budget is sized for.  Walkers of large
// systems fit two CTAs per SM in shared memory and get up to 255 registers
// (MINB = 2); small systems fit three or more and get the 168-register budget
// that keeps three resident (MINB = 3).  The host picks by shared-memory
// occupancy (sample_variant3).
template <typename T, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_sample(const SysDev *systems, const int2 *work, int n_work,
                                               int *work_ctr, uint2 key, int n_first, int n_samples,
                                               int sweeps_between, int sample_base) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ SysDev S;
  __shared__ int s_item;
  __shared__ __align__(8) uint64_t bar;
  uint32_t phase = 0;
  if (threadIdx.x == 0) mbar_init(&bar);
  __syncthreads();
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(work_ctr, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= n_work) break;
    const int2 wk = work[item];
    load_sys(&S, systems + wk.x);
    const int w = wk.y;
    const int N = S.N, Ns = S.Ns, Ne = S.Ne, ldm = S.ldm, tid = threadIdx.x;
    WSmem<T> sm;
    walker_layout<T>(N, Ns, S.acc_len, S.n_hidden, S.delay_k, S.minv_lo != nullptr, smem_raw, &sm);
    // --- load the walker: M^-1 block by a TMA bulk copy, configuration and
    // Jastrow field by plain loads while the copy is in flight
    const uint32_t nbytes = (uint32_t)minv_bytes(N, ldm, sizeof(T));
    // test hook (vmc_test_stall): for this walker no copy is issued, so the
    // bounded wait below runs out with nothing in flight
    const bool stall = (w == S.stall_walker);
    {
      if (tid == 0 && !stall) {
        if (sm.mlo)
          bulk_load_pair(sm.minv, (const unsigned char *)S.minv + (size_t)w * nbytes, sm.mlo,
                         (const unsigned char *)S.minv_lo + (size_t)w * nbytes, nbytes, &bar);
        else
          bulk_load(sm.minv, (const unsigned char *)S.minv + (size_t)w * nbytes, nbytes, &bar);
      }
      for (int k = tid; k < Ne; k += NT) sm.ele[k] = S.ele[(size_t)w * Ne + k];
      for (int k = tid; k < 2 * Ns; k += NT) sm.occ[k] = S.occ[(size_t)w * 2 * Ns + k];
      for (int k = tid; k < Ns; k += NT) sm.jf[k] = ((const T *)S.jf)[(size_t)w * Ns + k];
      for (int k = tid; k < S.n_hidden; k += NT) {
        const T h = ((const T *)S.hmlp)[(size_t)w * S.n_hidden + k];
        sm.hm[k] = h;
        sm.th[k] = tanh_t<T>(h);
      }
    }
    const bool loaded = mbar_wait(&bar, phase, stall ? STALL_LIMIT : WAIT_LIMIT);
    if (!stall) phase ^= 1;
    if (__syncthreads_or(!loaded)) {
      // the copy did not complete within the limit: flag, wait once more for
      // it (bounded; nothing to wait for after the test hook's wait), skip the
      // walker (its chain does not advance) and stop this CTA
      if (tid == 0) {
        S.status[w] |= VMC_ST_TIMEOUT;
        if (!stall) mbar_wait(&bar, phase ^ 1);
      }
      break;
    }
    if (tid == 0) S.status[w] &= ~VMC_ST_TIMEOUT;   // loaded: an earlier timeout is over
    unsigned long long ctr = S.ctr[w];
    int rpos = RB;
    MoveCounts mc;
    int acc_since = S.acc_since[w];
    int buf = 0;
    const uint32_t key_w = (uint32_t)w;
    __syncthreads();
    int np = 0;   // pending delayed updates
    const long long props_first = (long long)n_first * Ne;
    // proposals in batches where the MLP factor and delayed updates are off
    const bool batched = S.spec_b > 1 && S.n_hidden == 0 && S.delay_k <= 1;
    for (long long p = 0; p < props_first;) {
      if (batched) {
        p += propose_batch(S, sm, key, key_w, ctr, rpos, mc, acc_since, buf,
                           (int)(props_first - p < SPEC_MAX ? props_first - p : SPEC_MAX));
      } else {
        propose(S, sm, key, key_w, ctr, rpos, mc, acc_since, buf, np);
        ++p;
      }
    }
    for (int s = 0; s < n_samples; ++s) {
      const long long props = (long long)sweeps_between * Ne;
      for (long long p = 0; p < props;) {
        if (batched) {
          p += propose_batch(S, sm, key, key_w, ctr, rpos, mc, acc_since, buf,
                             (int)(props - p < SPEC_MAX ? props - p : SPEC_MAX));
        } else {
          propose(S, sm, key, key_w, ctr, rpos, mc, acc_since, buf, np);
          ++p;
        }
      }
      __syncthreads();
      delayed_flush(S, sm, np);
      measure(S, sm, w, sample_base + s, buf, mc);
      mc.samples++;
    }
    __syncthreads();
    delayed_flush(S, sm, np);
    if (mc.meas_hop) atomicAdd((unsigned long long *)&S.cnt[8 * w + 4], (unsigned long long)mc.meas_hop);
    if (mc.meas_ex) atomicAdd((unsigned long long *)&S.cnt[8 * w + 5], (unsigned long long)mc.meas_ex);
    __syncthreads();
    // --- store the walker back (M^-1 by a TMA bulk copy)
    fence_proxy_async();
    __syncthreads();
    {
      if (tid == 0) {
        bulk_store((unsigned char *)S.minv + (size_t)w * nbytes, sm.minv, nbytes);
        if (sm.mlo) bulk_store((unsigned char *)S.minv_lo + (size_t)w * nbytes, sm.mlo, nbytes);
      }
      for (int k = tid; k < Ne; k += NT) S.ele[(size_t)w * Ne + k] = sm.ele[k];
      for (int k = tid; k < S.n_hidden; k += NT) ((T *)S.hmlp)[(size_t)w * S.n_hidden + k] = sm.hm[k];
      for (int k = tid; k < 2 * Ns; k += NT) S.occ[(size_t)w * 2 * Ns + k] = sm.occ[k];
      for (int k = tid; k < Ns; k += NT) ((T *)S.jf)[(size_t)w * Ns + k] = sm.jf[k];
      if (tid == 0) {
        const long long total = props_first + (long long)n_samples * sweeps_between * Ne;
        S.ctr[w] = ctr;
        S.n_prop[w] += total;
        S.n_acc[w] += mc.hop_a + mc.ex_a;
        bulk_wait_read();   // shared memory is reused by the next walker
        S.cnt[8 * w + 0] += mc.hop_t;
        S.cnt[8 * w + 1] += mc.ex_t;
        S.cnt[8 * w + 2] += mc.hop_a;
        S.cnt[8 * w + 3] += mc.ex_a;
        S.cnt[8 * w + 6] += mc.samples;
        S.acc_since[w] = acc_since;
      }
    }
    __syncthreads();
  }
}

#ifndef VMC_SWEEP_V3_ONLY
// Expand the parameter vector into dense tables (f, f^T in FP64 and FP32, v, g).
__global__ void k_expand(SysDev S) {
  const int Ns = S.Ns;
  const size_t n2 = (size_t)Ns * Ns;
  const int base = S.n_g + S.n_v;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n2;
       q += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(q / Ns), j = (int)(q - (size_t)i * Ns);
    const int c = S.f_idx[q];
    const double f = (c >= 0) ? S.f_sign[q] * S.params[base + c] : 0.0;
    S.f64[q] = f;
    S.fT64[(size_t)j * Ns + i] = f;
    S.f32[q] = (float)f;
    S.fT32[(size_t)j * Ns + i] = (float)f;
    const int vc = S.v_idx[q];
    const double vv = (vc >= 0 && i != j) ? S.params[S.n_g + vc] : 0.0;
    S.vmat[q] = vv;
    S.vmat32[q] = (float)vv;
    if (q < (size_t)Ns) {
      const int gc = S.g_idx[q];
      const double gv = (gc >= 0) ? S.params[gc] : 0.0;
      S.gsite[q] = gv;
      S.gsite32[q] = (float)gv;
    }
  }
}

// v(j, i) of every hopping term grouped by target site (after k_expand).
__global__ void k_expand_terms(SysDev S) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < S.n_hop; q += gridDim.x * blockDim.x) {
    // target site i of grouped term q: the CSR row that contains q
    int lo = 0, hi = S.Ns;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (S.tgt_ptr[mid] <= q) lo = mid;
      else hi = mid;
    }
    const double v = S.vmat[(size_t)S.tgt_j[q] * S.Ns + lo];
    S.tgt_v64[q] = v;
    S.tgt_v32[q] = (float)v;
  }
}

// MLP weights: W1 (H x 2Ns, row-major in params) -> column-major copies.
__global__ void k_expand_mlp(SysDev S) {
  const int H = S.n_hidden, C = 2 * S.Ns;
  const size_t tot = (size_t)H * C;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < tot;
       q += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(q / C), c = (int)(q - (size_t)k * C);
    const double v = S.params[S.mlp_base + q];
    S.W1T64[(size_t)c * H + k] = v;
    ((__nv_bfloat16 *)S.W1T16)[(size_t)c * H + k] = __double2bfloat16(v);
  }
}

// From-scratch inverse of M (Gauss-Jordan with partial pivoting, in place in
// shared memory: FP64, or double-float by the mixed form's opt-in), log|det M| and its
// sign, Jastrow field and occupation table.  With only_due, only walkers
// whose accepted-move count since the last inverse reached due_threshold are
// rebuilt, and the drift max|M^-1_updated - M^-1_fresh| / max|M^-1_fresh| is
// recorded.  Work items are taken from the counter *ctr (zeroed by the
// launcher) one at a time, so the CTAs share the due walkers evenly whatever
// their positions in the list.
template <typename T>
__global__ void __launch_bounds__(NT) k_init(const SysDev *systems, const int2 *work, int n_work,
                                             int *ctr, int only_due, int due_threshold) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ SysDev S;
  __shared__ int s_item;
  __shared__ double red_d[NWARP], red_a[NWARP];
  // FP64 elimination; the mixed form's opt-in double-float one
  // (VMC_REBUILD_DOUBLE_FLOAT) shares the scratch
  constexpr bool F32 = std::is_same<T, float>::value;
  __shared__ union {
    vmc_gj::GJShared d;
    GJdf f;
  } gs;
  auto next_item = [&]() -> int {
    __syncthreads();   // every thread has read the previous item
    if (threadIdx.x == 0) s_item = atomicAdd(ctr, 1);
    __syncthreads();
    return s_item;
  };
  for (int item = next_item(); item < n_work; item = next_item()) {
    const int2 wk = work[item];
    const int w = wk.y;
    if (only_due && systems[wk.x].acc_since[w] < due_threshold) continue;
    load_sys(&S, systems + wk.x);
    const int N = S.N, Ns = S.Ns, Ne = S.Ne, ldm = S.ldm, tid = threadIdx.x;
    const bool use_df = F32 && S.rebuild_df;
    // N x ldm matrix: FP64 words, or (double-float) hi words then lo words
    double *A = (double *)smem_raw;
    float *Ah = (float *)smem_raw, *Al = Ah + (size_t)N * ldm;
    int *ele = (int *)(A + (size_t)N * ldm);        // Ne
    int *perm = ele + Ne;                            // N
    for (int k = tid; k < Ne; k += NT) ele[k] = S.ele[(size_t)w * Ne + k];
    __syncthreads();
    for (int q = tid; q < N * N; q += NT) {
      const int n = q / N, m = q - n * N;
      const double f = S.f64[(size_t)ele[n] * Ns + ele[N + m]];
      if (use_df)
        df_split(f, Ah[n * ldm + m], Al[n * ldm + m]);
      else
        A[n * ldm + m] = f;
    }
    __syncthreads();
    if (use_df)
      gj_invert_df(Ah, Al, ldm, N, perm, gs.f);
    else
      vmc_gj::gj_invert(A, ldm, N, perm, gs.d);
    const int g_bad = use_df ? gs.f.bad : gs.d.bad;
    const int g_sign = use_df ? gs.f.sign : gs.d.sign;
    const double g_logdet = use_df ? gs.f.logdet : gs.d.logdet;
    const double g_pmin = use_df ? gs.f.pmin : gs.d.pmin;
    const double g_pmax = use_df ? gs.f.pmax : gs.d.pmax;
    // the fresh inverse's entry q (FP64 value)
    auto fresh_at = [&](int q) -> double {
      return use_df ? (double)Ah[q] + (double)Al[q] : A[q];
    };
    const size_t nb = minv_bytes(N, ldm, sizeof(T));
    T *dst = (T *)((unsigned char *)S.minv + (size_t)w * nb);
    // mixed form: low words of the double-float inverse (zero while delayed
    // updates, which keep FP32 words only, are on)
    float *dlo = (F32 && S.minv_lo) ? (float *)((unsigned char *)S.minv_lo + (size_t)w * nb)
                                    : nullptr;
    if (!g_bad) {
      if (only_due) {
        double dmax = 0.0, amax = 0.0;
        for (int q = tid; q < N * N; q += NT) {
          const int r = q / N, c = q - r * N;
          const double fresh = fresh_at(r * ldm + c);
          const double cur = (double)dst[r * ldm + c] + (dlo ? (double)dlo[r * ldm + c] : 0.0);
          dmax = fmax(dmax, fabs(cur - fresh));
          amax = fmax(amax, fabs(fresh));
        }
        for (int o = 16; o > 0; o >>= 1) {
          dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
          amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        }
        if ((tid & 31) == 0) {
          red_d[tid >> 5] = dmax;
          red_a[tid >> 5] = amax;
        }
        __syncthreads();
        if (tid == 0) {
          double d = 0.0, a = 0.0;
          for (int q = 0; q < NWARP; ++q) {
            d = fmax(d, red_d[q]);
            a = fmax(a, red_a[q]);
          }
          S.drift[w] = fmax(S.drift[w], (a > 0.0) ? d / a : d);
        }
        __syncthreads();
      }
      const bool keep_lo = dlo && S.delay_k <= 1;
      for (int q = tid; q < N * ldm; q += NT) {
        if (use_df) {
          dst[q] = Ah[q];
          if (dlo) dlo[q] = keep_lo ? Al[q] : 0.f;
        } else {
          const T h = (T)A[q];
          dst[q] = h;
          if (dlo) dlo[q] = keep_lo ? (float)(A[q] - (double)h) : 0.f;
        }
      }
    }
    if (!only_due) {
      for (int k = tid; k < 2 * Ns; k += NT) S.occ[(size_t)w * 2 * Ns + k] = -1;
      __syncthreads();
      for (int k = tid; k < Ne; k += NT) {
        const int s = (k >= N) ? 1 : 0;
        S.occ[(size_t)w * 2 * Ns + s * Ns + ele[k]] = k;
      }
      __syncthreads();
    }
    {
      // Jastrow field h_i = sum_{j != i} v_ij (n_j - 1), rebuilt in FP64 on
      // every from-scratch inverse: only sites with n_j != 1 contribute; v is
      // symmetric, so row j is read (coalesced).
      int *nsite = perm + N;        // [Ns] n_j
      int *jlist = nsite + Ns;      // [Ns] sites with n_j != 1
      int *jcount = jlist + Ns;     // [1]
      if (tid == 0) *jcount = 0;
      for (int k = tid; k < Ns; k += NT) nsite[k] = 0;
      __syncthreads();
      for (int k = tid; k < Ne; k += NT) atomicAdd(&nsite[ele[k]], 1);
      __syncthreads();
      for (int j = tid; j < Ns; j += NT)
        if (nsite[j] != 1) jlist[atomicAdd(jcount, 1)] = j;
      __syncthreads();
      const int nl = *jcount;
      for (int i = tid; i < Ns; i += NT) {
        double h = 0.0;
        for (int q = 0; q < nl; ++q) {
          const int j = jlist[q];
          h += S.vmat[(size_t)j * Ns + i] * (double)(nsite[j] - 1);
        }
        ((T *)S.jf)[(size_t)w * Ns + i] = (T)h;
      }
      __syncthreads();
    }
    // MLP pre-activations from scratch: h_k = b1_k + sum over electrons of W1[k][c_e]
    for (int k = tid; k < S.n_hidden; k += NT) {
      const int H = S.n_hidden;
      double h = S.params[S.mlp_base + (size_t)H * 2 * Ns + k];
      for (int e = 0; e < Ne; ++e) h += S.W1T64[(size_t)(ele[e] + (e >= N ? Ns : 0)) * H + k];
      ((T *)S.hmlp)[(size_t)w * H + k] = (T)h;
    }
    if (tid == 0) {
      S.acc_since[w] = 0;
      if (only_due) S.n_rec[w] += 1;
      if (g_bad) {
        S.status[w] |= VMC_ST_SINGULAR;
      } else {
        S.status[w] &= ~(VMC_ST_SINGULAR | VMC_ST_ILLCOND);
        if (g_pmin < 1e-12 * g_pmax) S.status[w] |= VMC_ST_ILLCOND;
        S.logdet[w] = g_logdet;
        S.detsign[w] = g_sign;
        if (!isfinite(g_logdet)) S.status[w] |= VMC_ST_NUMERIC;
      }
    }
    __syncthreads();
  }
}

// Ratio check hook: evaluate candidate moves on one walker's current state.
template <typename T>
__global__ void __launch_bounds__(NT) k_eval_ratios(const SysDev *systems, int sys, int w,
                                                    int n_moves, const int *moves, double *out) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ SysDev S;
  load_sys(&S, systems + sys);
  const int N = S.N, Ns = S.Ns, Ne = S.Ne, ldm = S.ldm, tid = threadIdx.x;
  WSmem<T> sm;
  walker_layout<T>(N, Ns, S.acc_len, S.n_hidden, 0, false, smem_raw, &sm);
  const size_t nb = minv_bytes(N, ldm, sizeof(T));
  const T *src = (const T *)((const unsigned char *)S.minv + (size_t)w * nb);
  for (int k = tid; k < N * ldm; k += NT) sm.minv[k] = src[k];
  for (int k = tid; k < Ne; k += NT) sm.ele[k] = S.ele[(size_t)w * Ne + k];
  for (int k = tid; k < 2 * Ns; k += NT) sm.occ[k] = S.occ[(size_t)w * 2 * Ns + k];
  for (int k = tid; k < Ns; k += NT) sm.jf[k] = ((const T *)S.jf)[(size_t)w * Ns + k];
  for (int k = tid; k < S.n_hidden; k += NT) {
    const T h = ((const T *)S.hmlp)[(size_t)w * S.n_hidden + k];
    sm.hm[k] = h;
    sm.th[k] = tanh_t<T>(h);
  }
  __syncthreads();
  int buf = 0;
  for (int q = 0; q < n_moves; ++q) {
    const int kind = moves[3 * q], a = moves[3 * q + 1], b = moves[3 * q + 2];
    double res = 0.0;
    if (kind == 0) {
      if (a >= 0 && a < Ne && b >= 0 && b < Ns) {
        const int s = (a >= N) ? 1 : 0;
        if (sm.occ[s * Ns + b] < 0 && !(S.local_spin && sm.occ[(1 - s) * Ns + b] >= 0) &&
            !(S.lsite && (S.lsite[b] | S.lsite[sm.ele[a]]))) {
          T fval, mlp;
          const T rpf = hop_pf_ratio(S, sm, a, b, fval, buf, mlp, 0);
          res = (double)rpf * (double)corr_factor<T>(corr_hop<T>(S, sm.occ, sm.jf, s, sm.ele[a], b)) *
                (S.n_hidden ? (double)exp_t<T>(mlp) : 1.0);
        }
      }
    } else if (a >= 0 && a < N && b >= N && b < Ne) {
      const int i = sm.ele[a], j = sm.ele[b];
      if (i != j && sm.occ[Ns + i] < 0 && sm.occ[j] < 0) {
        T K[4], mlp;
        res = (double)exchange_pf_ratio(S, sm, a, b - N, i, j, buf, K, mlp, 0) *
              (S.n_hidden ? (double)exp_t<T>(mlp) : 1.0);
      }
    }
    if (tid == 0) out[q] = res;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Pair correlations of the current configurations (measurement mode,
// Sec. 2.2.3; local estimators of Eq. MC, A acting on the ket |x>).
//
// Off-diagonal kinds, per walker, from Green-function ratios of its M^-1 = B:
//   G_up[b, k] = sum_l f(b, r_l,dn) B_lk      (up electron k hops to b)
//   G_dn[a, m] = sum_k f(r_k,up, a) B_mk      (down electron m hops to a)
//   T[b, a]    = sum_k G_up[b, k] f(r_k,up, a)
// and, for the spin swap of up electron n on a with down electron m on b
// (both sites singly occupied; det of M with row n and column m replaced),
//   det M'/det M = G_up[b, n] G_dn[a, m] - B_mn (T[b, a] - f(b, a)).
// One pass over the sites b: G_up[b, :] (N^2); the down-occupied sites are
// collected in groups of CORR_G, and for a group G_dn[:, m] and T[b, :] of
// all its sites are formed together (2 N Ns each), so every gathered
// f(r_k,up, a) serves 2 CORR_G products: Ns N^2 + 2 N_dn N Ns per
// configuration for all Ns^2 pairs.
//   kind 0 (c^dag_{b up} c_{j up}): up electron on j hops to b,
//          G_up[b, k] x P_G P_J ratio;
//   kind 1 (c^dag_{a dn} c_{b dn}): down electron on b hops to a,
//          G_dn[a, m] x P_G P_J ratio;
//   kind 4 (S^+_b S^-_a): the swap above, with the fermion sign -1 of
//          S^+S^- in the labelled basis (P_G, P_J unchanged).
// Each CTA takes walkers blockIdx.x, blockIdx.x + gridDim.x, ... in turn and
// adds their values to one FP64 plane triple part[3][Ns][Ns] (diagonal
// entries stay 0) by atomic adds without return, so the 24 Ns^2 bytes stay
// in L2 and no thread waits on them; the order of the additions, and so the
// last bit of a sum, varies between runs.
// ---------------------------------------------------------------------------
// Down-occupied sites whose second product is formed together (their G_up
// rows wait in vector slots 1..CORR_G of shared memory).
constexpr int CORR_G = 4;

template <typename T>
__global__ void __launch_bounds__(NT) k_corr(const SysDev *systems, int sys, double *part) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ SysDev S;
  load_sys(&S, systems + sys);
  const int N = S.N, Ns = S.Ns, Ne = S.Ne, ldm = S.ldm, tid = threadIdx.x;
  WSmem<T> sm;
  walker_layout<T>(N, Ns, S.acc_len, S.n_hidden, 0, false, smem_raw, &sm);
  T *fb = sm.vec;                    // slot 0: f(b, r_l,dn), l < N
  const T *F = ftab<T>(S);
  const size_t ns2 = (size_t)Ns * Ns;
  double *P0 = part;
  double *P1 = P0 + ns2;
  double *P4 = P1 + ns2;
  const size_t nb = minv_bytes(N, ldm, sizeof(T));
  for (int w = blockIdx.x; w < S.W; w += gridDim.x) {
    const T *src = (const T *)((const unsigned char *)S.minv + (size_t)w * nb);
    for (int k = tid; k < N * ldm; k += NT) sm.minv[k] = src[k];
    for (int k = tid; k < Ne; k += NT) sm.ele[k] = S.ele[(size_t)w * Ne + k];
    for (int k = tid; k < 2 * Ns; k += NT) sm.occ[k] = S.occ[(size_t)w * 2 * Ns + k];
    for (int k = tid; k < Ns; k += NT) sm.jf[k] = ((const T *)S.jf)[(size_t)w * Ns + k];
    __syncthreads();
    // pending group: sites gb[q] with down electron gm[q], G_up row in slot 1 + q
    int ng = 0;
    int gb[CORR_G], gm[CORR_G];
#pragma unroll
    for (int q = 0; q < CORR_G; ++q) gb[q] = gm[q] = 0;
    // G_up[b, :] = f(b, r_dn)^T M^-1 for four sites b at a time: the rows
    // f(b, r_l,dn) in vector slots 0, 5, 6, 7, thread k the column k, one
    // shared load of M^-1 per four multiply-adds; the rows of down-occupied
    // sites go to the group's slots 1..CORR_G.
    T *fbs[4] = {fb, sm.vec + 5 * VMC_MAX_N, sm.vec + 6 * VMC_MAX_N, sm.vec + 7 * VMC_MAX_N};
    for (int b0 = 0; b0 < Ns; b0 += 4) {
      const int nbk = (Ns - b0 < 4) ? Ns - b0 : 4;
      if (tid < N) {
        const int el = sm.ele[N + tid];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          fbs[u][tid] = (u < nbk) ? F[(size_t)(b0 + u) * Ns + el] : (T)0;
      }
      __syncthreads();
      T g4[4] = {(T)0, (T)0, (T)0, (T)0};
      if (tid < N) {
        int l = 0;
        for (; l + 4 <= N; l += 4) {
          const T m0 = sm.minv[l * ldm + tid], m1 = sm.minv[(l + 1) * ldm + tid];
          const T m2 = sm.minv[(l + 2) * ldm + tid], m3 = sm.minv[(l + 3) * ldm + tid];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            T x0, x1, x2, x3;
            ld4(fbs[u] + l, x0, x1, x2, x3);
            g4[u] += x0 * m0;
            g4[u] += x1 * m1;
            g4[u] += x2 * m2;
            g4[u] += x3 * m3;
          }
        }
        for (; l < N; ++l) {
          const T m0 = sm.minv[l * ldm + tid];
#pragma unroll
          for (int u = 0; u < 4; ++u) g4[u] += fbs[u][l] * m0;
        }
      }
      __syncthreads();   // the block's rows are read; slots 0, 5..7 free
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (u >= nbk) break;
        const int b = b0 + u;
        const bool b_up = sm.occ[b] >= 0, b_dn = sm.occ[Ns + b] >= 0;
        // kind 0 at (b, r_k,up)
        if (tid < N && !b_up && !(S.local_spin && b_dn)) {
          const int j = sm.ele[tid];
          const T c = corr_factor<T>(corr_hop<T>(S, sm.occ, sm.jf, 0, j, b));
          atomicAdd(&P0[(size_t)b * Ns + j], (double)(g4[u] * c));
        }
        if (b_dn) {
          if (tid < N) sm.vec[(size_t)(1 + ng) * VMC_MAX_N + tid] = g4[u];
  #pragma unroll
          for (int q = 0; q < CORR_G; ++q)
            if (q == ng) {
              gb[q] = b;
              gm[q] = sm.occ[Ns + b] - N;
            }
          ++ng;
        }
        if (ng == CORR_G || (b == Ns - 1 && ng > 0)) {
          __syncthreads();   // the group's G_up rows are in place
          // G_dn[a, m] and T[b, a] of the group's sites, two sites a per
          // thread: each f(r_k,up, a) feeds 2 x CORR_G pairs of products.
          const T *Bq[CORR_G], *Gq[CORR_G];
  #pragma unroll
          for (int q = 0; q < CORR_G; ++q) {
            Bq[q] = sm.minv + (size_t)gm[q] * ldm;       // unused slots: a valid row
            Gq[q] = sm.vec + (size_t)(1 + q) * VMC_MAX_N;
          }
          for (int a0 = tid; a0 < Ns; a0 += 2 * NT) {
            const int a1 = a0 + NT < Ns ? a0 + NT : a0;
            T d0[CORR_G], t0[CORR_G], d1[CORR_G], t1[CORR_G];
  #pragma unroll
            for (int q = 0; q < CORR_G; ++q) d0[q] = t0[q] = d1[q] = t1[q] = (T)0;
            for (int k = 0; k < N; ++k) {
              const T *Fk = F + (size_t)sm.ele[k] * Ns;
              const T f0 = Fk[a0], f1 = Fk[a1];
  #pragma unroll
              for (int q = 0; q < CORR_G; ++q) {
                const T bk = Bq[q][k], gk = Gq[q][k];
                d0[q] += bk * f0;
                t0[q] += gk * f0;
                d1[q] += bk * f1;
                t1[q] += gk * f1;
              }
            }
  #pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int a = h ? a1 : a0;
              if (h && a1 == a0) break;
              const bool a_up = sm.occ[a] >= 0, a_dn = sm.occ[Ns + a] >= 0;
  #pragma unroll
              for (int q = 0; q < CORR_G; ++q) {
                if (q >= ng) break;
                const int bq = gb[q];
                if (a == bq) continue;
                const T accD = h ? d1[q] : d0[q], accT = h ? t1[q] : t0[q];
                // kind 1 at (a, bq): down electron gm[q] hops bq -> a
                if (!a_dn && !(S.local_spin && a_up)) {
                  const T c = corr_factor<T>(corr_hop<T>(S, sm.occ, sm.jf, 1, bq, a));
                  atomicAdd(&P1[(size_t)a * Ns + bq], (double)(accD * c));
                }
                // kind 4 at (bq, a): spin swap with up electron n on a
                if (a_up && !a_dn && sm.occ[bq] < 0) {
                  const int n = sm.occ[a];
                  const T r = Gq[q][n] * accD - Bq[q][n] * (accT - F[(size_t)bq * Ns + a]);
                  atomicAdd(&P4[(size_t)bq * Ns + a], -(double)r);
                }
              }
            }
          }
          ng = 0;
          __syncthreads();   // the group's slots are written again
        }
      }
    }
    __syncthreads();
  }
}

// Occupation products summed over the walkers of one system, exactly in
// integers: cnt[c][i][j] = sum_w x_i y_j with (x, y) = (n_up, n_up),
// (n_up, n_dn), (n_dn, n_up), (n_dn, n_dn) for c = 0..3.  These give every
// diagonal estimator (n_i n_j, S^z_i S^z_j and the i = j terms of kinds 0, 1,
// 4, 5).  One thread per (i, j) of a 16 x 16 tile.
__global__ void k_corr_occ(const SysDev *systems, int sys, int *cnt) {
  const SysDev &S = systems[sys];
  const int Ns = S.Ns;
  const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
  if (i >= Ns || j >= Ns) return;
  int uu = 0, ud = 0, du = 0, dd = 0;
  for (int w = 0; w < S.W; ++w) {
    const int *o = S.occ + (size_t)w * 2 * Ns;
    const int ui = o[i] >= 0, di = o[Ns + i] >= 0, uj = o[j] >= 0, dj = o[Ns + j] >= 0;
    uu += ui & uj;
    ud += ui & dj;
    du += di & uj;
    dd += di & dj;
  }
  const size_t ns2 = (size_t)Ns * Ns, q = (size_t)i * Ns + j;
  cnt[q] = uu;
  cnt[ns2 + q] = ud;
  cnt[2 * ns2 + q] = du;
  cnt[3 * ns2 + q] = dd;
}

// out[kind][i][j] = walker mean of the local estimators (kinds 0..5 of the
// header): the ratio planes (n_part sets, summed in order) and the integer
// counts, scaled.  With a local_site mask (Kondo local spins: exactly one
// electron each) a hop c^dag_i c_j with i != j into or out of a marked site
// leaves the constrained space, where psi = 0: those entries of kinds 0 and 1
// are 0.  Spin swaps keep every site's occupation and are kept.
__global__ void k_corr_reduce(const double *part, int n_part, const int *cnt, int Ns, int W,
                              const signed char *lsite, double *out) {
  const size_t ns2 = (size_t)Ns * Ns;
  const double inv = 1.0 / (double)W;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < ns2;
       q += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(q / Ns), j = (int)(q % Ns);
    const size_t qt = (size_t)j * Ns + i;
    double g0 = 0.0, g1 = 0.0, s4 = 0.0, s4t = 0.0;
    for (int b = 0; b < n_part; ++b) {
      const double *P = part + (size_t)b * 3 * ns2;
      g0 += P[q];
      g1 += P[ns2 + q];
      s4 += P[2 * ns2 + q];
      s4t += P[2 * ns2 + qt];
    }
    const double uu = cnt[q], ud = cnt[ns2 + q], du = cnt[2 * ns2 + q], dd = cnt[3 * ns2 + q];
    const double szsz = 0.25 * (uu - ud - du + dd);
    double d0 = 0.0, d1 = 0.0, d4 = 0.0, d5 = 0.0;
    if (i == j) {   // n_up, n_dn, n_up (1 - n_dn), (n_up + n_dn - 2 n_up n_dn) / 2
      d0 = uu;
      d1 = dd;
      d4 = uu - ud;
      d5 = 0.5 * (uu - ud + dd - du);
    }
    if (lsite && i != j && (lsite[i] | lsite[j])) g0 = g1 = 0.0;
    out[q] = (g0 + d0) * inv;
    out[ns2 + q] = (g1 + d1) * inv;
    out[2 * ns2 + q] = (uu + ud + du + dd) * inv;
    out[3 * ns2 + q] = szsz * inv;
    out[4 * ns2 + q] = (s4 + d4) * inv;
    out[5 * ns2 + q] = (szsz + 0.5 * (s4 + s4t) + d5) * inv;
  }
}

#endif  // VMC_SWEEP_V3_ONLY
}  // namespace

#ifndef VMC_SWEEP_V3_ONLY

// ---------------------------------------------------------------------------
// Host-side launch wrappers
// ---------------------------------------------------------------------------
size_t vmc_walker_smem(int precision, int N, int Ns, int Np, int H, int kd, int *acc_len,
                       int with_lo) {
  const int al = (Np <= VMC_ACC_MAX) ? Np : 0;
  if (acc_len) *acc_len = al;
  return precision == 0 ? walker_layout<double>(N, Ns, al, H, kd, false, nullptr, nullptr)
                        : walker_layout<float>(N, Ns, al, H, kd, with_lo != 0, nullptr, nullptr);
}

size_t vmc_init_smem(int N, int Ns) {
  const int ldm = (N % 2) ? N : N + 1;
  return (size_t)N * ldm * sizeof(double) + sizeof(int) * (3 * N + 2 * Ns + 1) + 64;
}

// The mixed form's sweep variant for a shared-memory size: the 168-register
// one (vmc_sweep3.cu) where it keeps three or more CTAs per SM resident,
// else the other.
static bool sample_variant3(size_t smem, int *nb3) {
  const int nb = vmc_sample_occupancy_v3(smem);
  if (nb3) *nb3 = nb;
  return nb >= 3;
}

int vmc_sample_occupancy(int precision, size_t smem) {
  int nb = 0;
  if (precision == 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sample<double, 3>, NT, smem);
  } else if (!sample_variant3(smem, &nb)) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sample<float, 2>, NT, smem);
  }
  return nb;
}

cudaError_t vmc_walker_set_smem_limits(size_t s64, size_t s32, size_t sinit) {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_sample<double, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s64))) return e;
  if ((e = cudaFuncSetAttribute(k_eval_ratios<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s64))) return e;
  if ((e = cudaFuncSetAttribute(k_sample<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s32))) return e;
  if ((e = vmc_sample_set_smem_v3(s32))) return e;
  if ((e = cudaFuncSetAttribute(k_eval_ratios<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s32))) return e;
  if ((e = cudaFuncSetAttribute(k_corr<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s64))) return e;
  if ((e = cudaFuncSetAttribute(k_corr<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s32))) return e;
  if ((e = cudaFuncSetAttribute(k_init<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sinit))) return e;
  if ((e = cudaFuncSetAttribute(k_init<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sinit))) return e;
  return cudaSuccess;
}

cudaError_t vmc_launch_expand(const SysDev *h_sys, cudaStream_t st, long long *nl) {
  const size_t n2 = (size_t)h_sys->Ns * h_sys->Ns;
  const int grid = (int)((n2 + 255) / 256 < 4096 ? (n2 + 255) / 256 : 4096);
  k_expand<<<grid, 256, 0, st>>>(*h_sys);
  ++*nl;
  if (h_sys->n_hop) {
    k_expand_terms<<<(h_sys->n_hop + 255) / 256, 256, 0, st>>>(*h_sys);
    ++*nl;
  }
  if (h_sys->n_hidden) {
    k_expand_mlp<<<1024, 256, 0, st>>>(*h_sys);
    ++*nl;
  }
  return cudaGetLastError();
}

cudaError_t vmc_launch_init(const SysDev *d_sys, const int2 *d_work, int n_work, int *d_ctr,
                            int precision, int only_due, int due_threshold, size_t smem,
                            cudaStream_t st, long long *nl) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int per = 1;
  if (precision == 0)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_init<double>, NT, smem);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_init<float>, NT, smem);
  if (per < 1) per = 1;
  int grid = nsm * per;
  if (grid > n_work) grid = n_work;
  if (grid < 1) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(d_ctr, 0, sizeof(int), st);
  if (e) return e;
  if (precision == 0)
    k_init<double><<<grid, NT, smem, st>>>(d_sys, d_work, n_work, d_ctr, only_due, due_threshold);
  else
    k_init<float><<<grid, NT, smem, st>>>(d_sys, d_work, n_work, d_ctr, only_due, due_threshold);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t vmc_launch_sample(const SysDev *d_sys, const int2 *d_work, int n_work, int *d_work_ctr,
                              int precision, uint64_t seed, int n_first, int n_samples,
                              int sweeps_between, int sample_base, int grid, size_t smem,
                              cudaStream_t st, long long *nl) {
  cudaError_t e = cudaMemsetAsync(d_work_ctr, 0, sizeof(int), st);
  if (e) return e;
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  if (grid > n_work) grid = n_work;
  if (grid < 1) return cudaSuccess;
  if (precision == 0)
    k_sample<double, 3><<<grid, NT, smem, st>>>(d_sys, d_work, n_work, d_work_ctr, key, n_first,
                                                n_samples, sweeps_between, sample_base);
  else if (sample_variant3(smem, nullptr))
    return vmc_launch_sample_v3(d_sys, d_work, n_work, d_work_ctr, key, n_first, n_samples,
                                sweeps_between, sample_base, grid, smem, st, nl);
  else
    k_sample<float, 2><<<grid, NT, smem, st>>>(d_sys, d_work, n_work, d_work_ctr, key, n_first,
                                               n_samples, sweeps_between, sample_base);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t vmc_launch_eval_ratios(const SysDev *d_sys, int sys, int walker, int precision,
                                   int n_moves, const int *d_moves, double *d_out, size_t smem,
                                   cudaStream_t st, long long *nl) {
  if (precision == 0)
    k_eval_ratios<double><<<1, NT, smem, st>>>(d_sys, sys, walker, n_moves, d_moves, d_out);
  else
    k_eval_ratios<float><<<1, NT, smem, st>>>(d_sys, sys, walker, n_moves, d_moves, d_out);
  ++*nl;
  return cudaGetLastError();
}

int vmc_corr_grid(int precision, size_t smem, int W, int Ns) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (precision == 0)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_corr<double>, NT, smem);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_corr<float>, NT, smem);
  if (per < 1) per = 1;
  long long grid = (long long)nsm * per;
  if (grid > W) grid = W;
  if (grid < 1) grid = 1;
  return (int)grid;
}

cudaError_t vmc_launch_corr(const SysDev *d_sys, int sys, int precision, int grid, double *part,
                            size_t smem, cudaStream_t st, long long *nl) {
  if (precision == 0)
    k_corr<double><<<grid, NT, smem, st>>>(d_sys, sys, part);
  else
    k_corr<float><<<grid, NT, smem, st>>>(d_sys, sys, part);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t vmc_launch_corr_occ(const SysDev *d_sys, int sys, int Ns, int *cnt, cudaStream_t st,
                                long long *nl) {
  const dim3 blk(16, 16), grd((Ns + 15) / 16, (Ns + 15) / 16);
  k_corr_occ<<<grd, blk, 0, st>>>(d_sys, sys, cnt);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t vmc_launch_corr_reduce(const double *part, int n_part, const int *cnt, int Ns, int W,
                                   const signed char *lsite, double *out, cudaStream_t st,
                                   long long *nl) {
  const size_t ns2 = (size_t)Ns * Ns;
  const size_t blocks = (ns2 + 255) / 256;
  const int grid = (int)(blocks < 4096 ? blocks : 4096);
  k_corr_reduce<<<grid, 256, 0, st>>>(part, n_part, cnt, Ns, W, lsite, out);
  ++*nl;
  return cudaGetLastError();
}

#else  // VMC_SWEEP_V3_ONLY: the mixed form's sweep kernel with the 168-register budget

int vmc_sample_occupancy_v3(size_t smem) {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sample<float, 3>, NT, smem);
  return nb;
}

cudaError_t vmc_sample_set_smem_v3(size_t s32) {
  return cudaFuncSetAttribute(k_sample<float, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)s32);
}

cudaError_t vmc_launch_sample_v3(const SysDev *d_sys, const int2 *d_work, int n_work,
                                 int *d_work_ctr, uint2 key, int n_first, int n_samples,
                                 int sweeps_between, int sample_base, int grid, size_t smem,
                                 cudaStream_t st, long long *nl) {
  k_sample<float, 3><<<grid, NT, smem, st>>>(d_sys, d_work, n_work, d_work_ctr, key, n_first,
                                             n_samples, sweeps_between, sample_base);
  ++*nl;
  return cudaGetLastError();
}
#endif  // VMC_SWEEP_V3_ONLY
