// Quantum-number projection of the pair product on the GPU (mVMC paper,
// Sec. 3.2.2, Eqs. momP and pointP; boundary signs of App. A):
//
//   psi(x) = P(x) sum_g w_g <T_g^-1 x | phi_Pf>,   T_g c^dag_{r s} T_g^-1 = s_g(r) c^dag_{g(r) s}.
//
// In the walker's labelled basis (ele[n] up electrons, ele[N + m] down ones)
// T_g^-1 |x> = sigma_g(x) |x_g>: x_g puts every electron on g^-1 of its site
// under the same label, and sigma_g(x) is the product over the electrons of
// the operation's sign there.  So <T_g^-1 x|phi> is proportional to
//
//   A_g(x) = sigma_g(x) det M_g(x),   M_g[n][m] = f(g^-1(r_n,up), g^-1(r_m,dn)).
//
// Each walker keeps, per operation g, M_g^-1 (N x N, row-major, in HBM) and
// the share pi_g = w_g A_g / sum_h w_h A_h of its projected amplitude.  A move
// of x is the same labelled move in every x_g, so
//
//   psi(x')/psi(x) = P(x')/P(x) sum_g pi_g tau_g rho_g,
//
// rho_g the fast-update ratio det M_g'/det M_g of the mapped move (Sec. 3.1.2)
// and tau_g the change of sigma_g.  On acceptance every M_g^-1 takes its
// Sherman-Morrison (hop) or Woodbury (exchange) update and
// pi_g <- pi_g tau_g rho_g / ratio.  The pair-orbital O_k (Eq. DiffPf) are the
// pi-weighted means of the mapped configurations' d ln det M_g / df; the
// correlation factors multiply the projected pair product, so theirs are
// those of x.
//
// One CTA of 128 threads per walker; its warps take the operations in turn
// (one warp per operation, lanes over the electrons), so no barrier separates
// the operations of one warp.  FP64 (plain form) or FP32 inverses and ratios
// with FP64 from-scratch inverses and FP64 shares pi_g (mixed form).
#include "vmc_common.cuh"
#include "vmc_dev.cuh"
#include "vmc_gj.cuh"

#include <math.h>

namespace {

// Per-warp scratch vectors of the projected kernels (R, w, p, q, z, b).
constexpr int PVEC = 6;

template <typename T>
struct PSmem {
  int *ele;      // Ne
  int *occ;      // 2 Ns
  int *mval;     // Ns: n_i - 1 (Jastrow O_k)
  T *jf;         // Ns Jastrow field
  T *g;          // Ns Gutzwiller g_i
  double *pi;    // n_ops shares of the projected amplitude
  T *rho;        // n_ops tau_g rho_g of the current move
  T *vec;        // NWARP x PVEC x VMC_MAX_N
  double *red;   // 2 x 16
  uint4 *rnd;    // NT Philox draws
  T *bc;         // broadcast scalars
  int *map;      // NWARP x 2 x VMC_MAX_N: electron sites mapped by the warp's operation
};

__host__ __device__ inline size_t pal(size_t x) { return (x + 15) / 16 * 16; }

template <typename T>
__host__ __device__ size_t proj_layout(int N, int Ns, int n_ops, unsigned char *base, PSmem<T> *sm) {
  (void)N;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = pal(off + bytes); return o; };
  const size_t o_ele = take(sizeof(int) * 2 * VMC_MAX_N);
  const size_t o_occ = take(sizeof(int) * 2 * Ns);
  const size_t o_mval = take(sizeof(int) * Ns);
  const size_t o_jf = take(sizeof(T) * Ns);
  const size_t o_g = take(sizeof(T) * Ns);
  const size_t o_pi = take(sizeof(double) * n_ops);
  const size_t o_rho = take(sizeof(T) * n_ops);
  const size_t o_vec = take(sizeof(T) * NWARP * PVEC * VMC_MAX_N);
  const size_t o_red = take(sizeof(double) * 32);
  const size_t o_rnd = take(sizeof(uint4) * NT);
  const size_t o_bc = take(sizeof(T) * 4);
  const size_t o_map = take(sizeof(int) * NWARP * 2 * VMC_MAX_N);
  if (sm) {
    sm->ele = (int *)(base + o_ele);
    sm->occ = (int *)(base + o_occ);
    sm->mval = (int *)(base + o_mval);
    sm->jf = (T *)(base + o_jf);
    sm->g = (T *)(base + o_g);
    sm->pi = (double *)(base + o_pi);
    sm->rho = (T *)(base + o_rho);
    sm->vec = (T *)(base + o_vec);
    sm->red = (double *)(base + o_red);
    sm->rnd = (uint4 *)(base + o_rnd);
    sm->bc = (T *)(base + o_bc);
    sm->map = (int *)(base + o_map);
  }
  return off;
}

// M_g^-1 of walker w (row-major, leading dimension N).
template <typename T>
__device__ __forceinline__ T *proj_minv(const SysDev &S, int w, int g) {
  return (T *)S.pminv + ((size_t)w * S.n_ops + g) * (size_t)S.N * S.N;
}

// Sum over the block (every thread gets the same value, same order).
__device__ __forceinline__ double block_sum_d(double v, double *red, int &buf) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[buf * 16 + (threadIdx.x >> 5)] = v;
  __syncthreads();
  const double *r = red + buf * 16;
  double s = r[0];
#pragma unroll
  for (int k = 1; k < NWARP; ++k) s += r[k];
  buf ^= 1;
  return s;
}

// ---------------------------------------------------------------------------
// Streaming one M_g^-1 (N x N row-major in HBM, N <= 128) by one warp: lanes
// over the columns k = lane + 32 j (j < 4), PR rows loaded before they are
// used, so PR x 4 loads per lane are in flight.
// ---------------------------------------------------------------------------
constexpr int PR = 8;

template <typename T>
__device__ __forceinline__ void rows_load(const T *M, int N, int l0, T (&v)[PR][4]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int r = 0; r < PR; ++r)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int l = l0 + r, k = lane + 32 * j;
      v[r][j] = (l < N && k < N) ? M[(size_t)l * N + k] : (T)0;
    }
}

template <typename T>
__device__ __forceinline__ void rows_store(T *M, int N, int l0, const T (&v)[PR][4]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int r = 0; r < PR; ++r)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int l = l0 + r, k = lane + 32 * j;
      if (l < N && k < N) M[(size_t)l * N + k] = v[r][j];
    }
}

// w_k = sum_l x_l M[l][k] (l ascending, one accumulator per k)
template <typename T>
__device__ void warp_colsum(const T *M, int N, const T *x, T *w) {
  const int lane = threadIdx.x & 31;
  T acc[4] = {(T)0, (T)0, (T)0, (T)0};
  for (int l0 = 0; l0 < N; l0 += PR) {
    T v[PR][4];
    rows_load(M, N, l0, v);
#pragma unroll
    for (int r = 0; r < PR; ++r) {
      const T xl = (l0 + r < N) ? x[l0 + r] : (T)0;
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[j] += xl * v[r][j];
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (lane + 32 * j < N) w[lane + 32 * j] = acc[j];
}

// y_l = sum_k M[l][k] x_k for every row l: per block of PR rows the lanes'
// partial sums are reduced and scattered over the warp (lane groups by bits
// 4..2 keep one row each), then summed over the remaining lane bits.
template <typename T>
__device__ void warp_rowdot(const T *M, int N, const T *x, T *y) {
  const int lane = threadIdx.x & 31;
  T xk[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) xk[j] = (lane + 32 * j < N) ? x[lane + 32 * j] : (T)0;
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  const int row = (b4 ? 4 : 0) + (b3 ? 2 : 0) + (b2 ? 1 : 0);
  for (int l0 = 0; l0 < N; l0 += PR) {
    T v[PR][4];
    rows_load(M, N, l0, v);
    T s[PR];
#pragma unroll
    for (int r = 0; r < PR; ++r) s[r] = v[r][0] * xk[0] + v[r][1] * xk[1] + v[r][2] * xk[2] + v[r][3] * xk[3];
    T a[4], c[2];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const T send = b4 ? s[u] : s[u + 4];
      a[u] = (b4 ? s[u + 4] : s[u]) + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const T send = b3 ? a[u] : a[u + 2];
      c[u] = (b3 ? a[u + 2] : a[u]) + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    const T send = b2 ? c[0] : c[1];
    T d = (b2 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, send, 4);
    d += __shfl_xor_sync(0xffffffffu, d, 2);
    d += __shfl_xor_sync(0xffffffffu, d, 1);
    if ((lane & 3) == 0 && l0 + row < N) y[l0 + row] = d;
  }
}

// ---------------------------------------------------------------------------
// Ratios of one mapped move, by one warp (lanes over the electrons)
// ---------------------------------------------------------------------------
// Hop of electron e to site t, mapped by g: det M_g'/det M_g.  Up electron n:
// sum_m f(t', r'_m,dn) M_g^-1[m][n]; down electron m: sum_n M_g^-1[m][n] f(r'_n,up, t').
template <typename T>
__device__ T proj_hop_ratio(const SysDev &S, const int *ele, const T *Mg, int g, int e, int t) {
  const int N = S.N, Ns = S.Ns, lane = threadIdx.x & 31;
  const int *inv = S.pinv + (size_t)g * Ns;
  const int tg = inv[t];
  T s = (T)0;
  if (e < N) {
    const T *F = ftab<T>(S);
    for (int m = lane; m < N; m += 32) s += F[(size_t)tg * Ns + inv[ele[N + m]]] * Mg[(size_t)m * N + e];
  } else {
    const int m = e - N;
    const T *FT = fTtab<T>(S);
    for (int n = lane; n < N; n += 32) s += Mg[(size_t)m * N + n] * FT[(size_t)tg * Ns + inv[ele[n]]];
  }
  return warp_sum(s);
}

// Exchange of up electron n (site i) with down electron m (site j), mapped
// by g: the 2 x 2 determinant-lemma form of the unprojected sweep on M_g.
// On return R holds the new row of M_g (R_l = f(j', r'_l,dn), R_m = f(j', i')),
// w = R^T M_g^-1, b_k = C_k - M_km (b_n = 0) with C_k = f(r''_k,up, i') the new
// column (r''_n = j), and K the 2 x 2 matrix [K11 K12; K21 K22].
template <typename T>
__device__ T proj_exchange_ratio(const SysDev &S, const int *ele, const T *Mg, int g, int n, int m,
                                 int i, int j, T *R, T *w, T *b, T *K) {
  const int N = S.N, Ns = S.Ns, lane = threadIdx.x & 31;
  const int *inv = S.pinv + (size_t)g * Ns;
  const int ig = inv[i], jg = inv[j];
  const T *F = ftab<T>(S);
  const T *FT = fTtab<T>(S);
  for (int l = lane; l < N; l += 32)
    R[l] = (l == m) ? F[(size_t)jg * Ns + ig] : F[(size_t)jg * Ns + inv[ele[N + l]]];
  __syncwarp();
  warp_colsum(Mg, N, R, w);
  __syncwarp();
  T a12 = (T)0, a22 = (T)0;
  for (int k = lane; k < N; k += 32) {
    const T wk = w[k];
    const int site = (k == n) ? j : ele[k];
    const T c = FT[(size_t)ig * Ns + inv[site]];
    const T mkm = FT[(size_t)jg * Ns + inv[ele[k]]];
    const T mrow = Mg[(size_t)m * N + k];
    if (k == n) {
      a22 += mrow * mkm;
      b[k] = (T)0;
    } else {
      a22 += mrow * c;
      a12 += wk * (c - mkm);
      b[k] = c - mkm;
    }
  }
  a22 = warp_sum(a22);
  a12 = warp_sum(a12);
  __syncwarp();
  K[0] = w[n];
  K[1] = a12;
  K[2] = Mg[(size_t)m * N + n];
  K[3] = a22;
  return K[0] * K[3] - K[1] * K[2];
}

// ---------------------------------------------------------------------------
// Inverse updates of one M_g^-1 in HBM, by one warp
// ---------------------------------------------------------------------------
// Row n replaced by R (up-electron hop): w = R^T M^-1,
// M'^-1 = M^-1 - M^-1[:,n] (w - e_n)^T / w_n.
template <typename T>
__device__ void proj_row_update(T *Mg, int N, int n, const T *R, T *w, T *p) {
  const int lane = threadIdx.x & 31;
  warp_colsum(Mg, N, R, w);
  for (int l = lane; l < N; l += 32) p[l] = Mg[(size_t)l * N + n];
  __syncwarp();
  const T inv = (T)1 / w[n];
  T wk[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) wk[j] = (lane + 32 * j < N) ? w[lane + 32 * j] : (T)0;
  for (int l0 = 0; l0 < N; l0 += PR) {
    T v[PR][4];
    rows_load(Mg, N, l0, v);
#pragma unroll
    for (int r = 0; r < PR; ++r) {
      const T c = (l0 + r < N) ? p[l0 + r] * inv : (T)0;
#pragma unroll
      for (int j = 0; j < 4; ++j) v[r][j] = (lane + 32 * j == n) ? c : v[r][j] - c * wk[j];
    }
    rows_store(Mg, N, l0, v);
  }
  __syncwarp();
}

// Column m replaced by C (down-electron hop): v = M^-1 C,
// M'^-1 = M^-1 - (v - e_m) M^-1[m,:] / v_m.
template <typename T>
__device__ void proj_col_update(T *Mg, int N, int m, const T *C, T *v, T *z) {
  const int lane = threadIdx.x & 31;
  warp_rowdot(Mg, N, C, v);
  for (int k = lane; k < N; k += 32) z[k] = Mg[(size_t)m * N + k];
  __syncwarp();
  const T inv = (T)1 / v[m];
  T zk[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) zk[j] = (lane + 32 * j < N) ? z[lane + 32 * j] : (T)0;
  for (int l0 = 0; l0 < N; l0 += PR) {
    T a[PR][4];
    rows_load(Mg, N, l0, a);
#pragma unroll
    for (int r = 0; r < PR; ++r) {
      const int l = l0 + r;
      const T c = (l < N) ? v[l] * inv : (T)0;
#pragma unroll
      for (int j = 0; j < 4; ++j) a[r][j] = (l == m) ? zk[j] * inv : a[r][j] - c * zk[j];
    }
    rows_store(Mg, N, l0, a);
  }
  __syncwarp();
}

// Rank-2 (Woodbury) update after an accepted exchange, with w, b and K of
// proj_exchange_ratio: p = M^-1[:,n], q = M^-1 b, z = M^-1[m,:],
// M'^-1 = M^-1 - [p q] K^-1 [w - e_n; z].
template <typename T>
__device__ void proj_exchange_update(T *Mg, int N, int n, int m, const T *w, const T *b,
                                     const T *K, T det, T *p, T *q, T *z) {
  const int lane = threadIdx.x & 31;
  warp_rowdot(Mg, N, b, q);
  for (int l = lane; l < N; l += 32) p[l] = Mg[(size_t)l * N + n];
  for (int k = lane; k < N; k += 32) z[k] = Mg[(size_t)m * N + k];
  __syncwarp();
  const T inv = (T)1 / det;
  T wk[4], zk[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int k = lane + 32 * j;
    wk[j] = (k < N) ? w[k] : (T)0;
    zk[j] = (k < N) ? z[k] : (T)0;
  }
  for (int l0 = 0; l0 < N; l0 += PR) {
    T a[PR][4];
    rows_load(Mg, N, l0, a);
#pragma unroll
    for (int r = 0; r < PR; ++r) {
      const int l = l0 + r;
      const T pl = (l < N) ? p[l] : (T)0, ql = (l < N) ? q[l] : (T)0;
      const T c1 = (pl * K[3] - ql * K[2]) * inv;
      const T c2 = (ql * K[0] - pl * K[1]) * inv;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        T x = a[r][j] - (c1 * wk[j] + c2 * zk[j]);
        if (lane + 32 * j == n) x += c1;
        a[r][j] = x;
      }
    }
    rows_store(Mg, N, l0, a);
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// From-scratch inverses: one CTA per (walker, operation)
// ---------------------------------------------------------------------------
// M_g gathered in FP64, Gauss-Jordan in shared memory; M_g^-1 written in the
// context's precision; log|A_g| and the sign of A_g = sigma_g det M_g kept
// for the shares (k_proj_shares).  With only_due, walkers whose accepted-move
// count has not reached due_threshold are skipped.
template <typename T>
__global__ void __launch_bounds__(NT) k_proj_build(const SysDev *systems, const int2 *work,
                                                   int n_work, int Ng, int only_due,
                                                   int due_threshold) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ SysDev S;
  __shared__ vmc_gj::GJShared gs;
  __shared__ int sgm;
  const int tid = threadIdx.x;
  for (long long item = blockIdx.x; item < (long long)n_work * Ng; item += gridDim.x) {
    __syncthreads();
    const int2 wk = work[item / Ng];
    const int g = (int)(item % Ng);
    load_sys(&S, systems + wk.x);
    const int w = wk.y;
    if (only_due && S.acc_since[w] < due_threshold) continue;
    const int N = S.N, Ns = S.Ns, Ne = S.Ne;
    const int ldm = (N % 2) ? N : N + 1;
    double *A = (double *)smem_raw;
    int *ele = (int *)(A + (size_t)N * ldm);
    int *perm = ele + Ne;
    const int *inv = S.pinv + (size_t)g * Ns;
    const signed char *sg = S.psgn + (size_t)g * Ns;
    for (int k = tid; k < Ne; k += NT) ele[k] = S.ele[(size_t)w * Ne + k];
    if (tid == 0) sgm = 1;
    __syncthreads();
    if (tid < 32) {
      // sigma_g(x): the product of the operation's signs over the electrons
      int neg = 0;
      for (int k = tid; k < Ne; k += 32) neg += sg[ele[k]] < 0;
      neg = warp_sum(neg);
      if (tid == 0) sgm = (neg & 1) ? -1 : 1;
    }
    for (int q = tid; q < N * N; q += NT) {
      const int n = q / N, m = q - n * N;
      A[n * ldm + m] = S.f64[(size_t)inv[ele[n]] * Ns + inv[ele[N + m]]];
    }
    __syncthreads();
    vmc_gj::gj_invert(A, ldm, N, perm, gs);
    T *dst = proj_minv<T>(S, w, g);
    for (int q = tid; q < N * N; q += NT) {
      const int n = q / N, m = q - n * N;
      dst[q] = (T)A[n * ldm + m];
    }
    if (tid == 0) {
      const size_t k = (size_t)w * Ng + g;
      S.plog[k] = gs.bad ? -INFINITY : gs.logdet;
      S.psign[k] = gs.bad ? 0 : gs.sign * sgm;
    }
  }
}

// Per walker: the shares pi_g of the projected amplitude from the operations'
// log|A_g| and signs (relative to the largest |A_g|), the occupation table
// and the Jastrow field.  A walker with a singular M_g (weight != 0) or a
// vanishing projected amplitude is flagged singular.
template <typename T>
__global__ void __launch_bounds__(NT) k_proj_shares(const SysDev *systems, const int2 *work,
                                                    int n_work, int only_due, int due_threshold) {
  __shared__ SysDev S;
  __shared__ double red[2 * 16];
  __shared__ int nsite[4096], jlist[4096];
  __shared__ int jcount, bad;
  const int tid = threadIdx.x;
  for (int item = blockIdx.x; item < n_work; item += gridDim.x) {
    __syncthreads();
    const int2 wk = work[item];
    load_sys(&S, systems + wk.x);
    const int w = wk.y;
    if (only_due && S.acc_since[w] < due_threshold) continue;
    const int Ng = S.n_ops, N = S.N, Ns = S.Ns, Ne = S.Ne;
    const double *lg = S.plog + (size_t)w * Ng;
    const int *sgn = S.psign + (size_t)w * Ng;
    if (tid == 0) bad = 0;
    __syncthreads();
    double L = -INFINITY;
    for (int g = tid; g < Ng; g += NT) {
      if (sgn[g] == 0 && S.pw[g] != 0.0) bad = 1;
      L = fmax(L, lg[g]);
    }
    for (int o = 16; o > 0; o >>= 1) L = fmax(L, __shfl_xor_sync(0xffffffffu, L, o));
    if ((tid & 31) == 0) red[tid >> 5] = L;
    __syncthreads();
    L = red[0];
    for (int k = 1; k < NWARP; ++k) L = fmax(L, red[k]);
    __syncthreads();
    double z = 0.0;
    for (int g = tid; g < Ng; g += NT)
      if (sgn[g] != 0) z += S.pw[g] * sgn[g] * exp(lg[g] - L);
    z = warp_sum(z);
    if ((tid & 31) == 0) red[16 + (tid >> 5)] = z;
    __syncthreads();
    double Z = red[16];
    for (int k = 1; k < NWARP; ++k) Z += red[16 + k];
    for (int g = tid; g < Ng; g += NT)
      S.ppi[(size_t)w * Ng + g] = (sgn[g] != 0) ? S.pw[g] * sgn[g] * exp(lg[g] - L) / Z : 0.0;
    if (!only_due) {
      for (int k = tid; k < 2 * Ns; k += NT) S.occ[(size_t)w * 2 * Ns + k] = -1;
      __syncthreads();
      for (int k = tid; k < Ne; k += NT)
        S.occ[(size_t)w * 2 * Ns + (k >= N ? Ns : 0) + S.ele[(size_t)w * Ne + k]] = k;
    }
    // Jastrow field h_i = sum_{j != i} v_ij (n_j - 1), in FP64
    if (tid == 0) jcount = 0;
    for (int k = tid; k < Ns; k += NT) nsite[k] = 0;
    __syncthreads();
    for (int k = tid; k < Ne; k += NT) atomicAdd(&nsite[S.ele[(size_t)w * Ne + k]], 1);
    __syncthreads();
    for (int j = tid; j < Ns; j += NT)
      if (nsite[j] != 1) jlist[atomicAdd(&jcount, 1)] = j;
    __syncthreads();
    for (int i = tid; i < Ns; i += NT) {
      double h = 0.0;
      for (int q = 0; q < jcount; ++q) h += S.vmat[(size_t)jlist[q] * Ns + i] * (double)(nsite[jlist[q]] - 1);
      ((T *)S.jf)[(size_t)w * Ns + i] = (T)h;
    }
    if (tid == 0) {
      S.acc_since[w] = 0;
      if (only_due) S.n_rec[w] += 1;
      S.status[w] &= ~(VMC_ST_SINGULAR | VMC_ST_NUMERIC | VMC_ST_ILLCOND);
      if (bad || !(Z != 0.0) || !isfinite(Z)) S.status[w] |= VMC_ST_SINGULAR;
      S.logdet[w] = L + log(fabs(Z));
      S.detsign[w] = Z < 0.0 ? -1 : 1;
    }
  }
}

// ---------------------------------------------------------------------------
// Metropolis sweep of the projected state and its measurement
// ---------------------------------------------------------------------------
template <typename T>
__device__ void proj_propose(const SysDev &S, const PSmem<T> &sm, int w, uint2 key,
                             unsigned long long &ctr, int &rpos, MoveCounts &mc, int &acc_since,
                             int &buf) {
  const int N = S.N, Ns = S.Ns, Ne = S.Ne, Ng = S.n_ops, tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  if (rpos == NT) {
    __syncthreads();
    const unsigned long long c = ctr + tid;
    sm.rnd[tid] = vmc_philox(make_uint4((uint32_t)c, (uint32_t)(c >> 32), (uint32_t)w,
                                        (uint32_t)S.sys_index), key);
    __syncthreads();
    rpos = 0;
  }
  const uint4 r = sm.rnd[rpos++];
  ctr++;
  const T u = (T)(r.w >> 8) * (T)(1.0 / 16777216.0);
  T *R = sm.vec + (size_t)warp * PVEC * VMC_MAX_N;
  T *W = R + VMC_MAX_N, *P = R + 2 * VMC_MAX_N, *Q = R + 3 * VMC_MAX_N, *Z = R + 4 * VMC_MAX_N,
    *B = R + 5 * VMC_MAX_N;
  if ((unsigned long long)r.x < S.pex) {
    const int n = vmc_mulhi(r.y, N);
    const int m = vmc_mulhi(r.z, N);
    const int i = sm.ele[n], j = sm.ele[N + m];
    if (i == j || sm.occ[Ns + i] >= 0 || sm.occ[j] >= 0) return;
    mc.ex_t++;
    double part = 0.0;
    for (int g = warp; g < Ng; g += NWARP) {
      T K[4];
      const T rho = proj_exchange_ratio(S, sm.ele, proj_minv<T>(S, w, g), g, n, m, i, j, R, W, B, K);
      if (lane == 0) sm.rho[g] = rho;
      part += sm.pi[g] * (double)rho;
    }
    const double ratio = block_sum_d(lane == 0 ? part : 0.0, sm.red, buf);
    if (!(u < (T)(ratio * ratio))) return;
    for (int g = warp; g < Ng; g += NWARP) {
      T K[4];
      T *Mg = proj_minv<T>(S, w, g);
      const T det = proj_exchange_ratio(S, sm.ele, Mg, g, n, m, i, j, R, W, B, K);
      proj_exchange_update(Mg, N, n, m, W, B, K, det, P, Q, Z);
      if (lane == 0) sm.pi[g] = sm.pi[g] * (double)sm.rho[g] / ratio;
    }
    __syncthreads();
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
    acc_since = (fabs(ratio) < SMALL_RATIO) ? RECOMPUTE_NOW : acc_since + 1;
    return;
  }
  const int e = vmc_mulhi(r.y, Ne);
  const int t = vmc_mulhi(r.z, Ns);
  const int s = (e >= N) ? 1 : 0;
  if (sm.occ[s * Ns + t] >= 0) return;
  if (S.local_spin && sm.occ[(1 - s) * Ns + t] >= 0) return;
  const int rs = sm.ele[e];
  if (S.lsite && (S.lsite[t] | S.lsite[rs])) return;
  mc.hop_t++;
  if (tid == 0)
    sm.bc[0] = corr_factor<T>(corr_hop_v(sm.occ, sm.jf, sm.g, Ns, s, rs, t,
                                         vtab<T>(S)[(size_t)rs * Ns + t]));
  double part = 0.0;
  for (int g = warp; g < Ng; g += NWARP) {
    const T rho = proj_hop_ratio(S, sm.ele, proj_minv<T>(S, w, g), g, e, t);
    const signed char *sg = S.psgn + (size_t)g * Ns;
    const T tr = (sg[t] * sg[rs] < 0) ? -rho : rho;
    if (lane == 0) sm.rho[g] = tr;
    part += sm.pi[g] * (double)tr;
  }
  const double rpf = block_sum_d(lane == 0 ? part : 0.0, sm.red, buf);
  const double ratio = rpf * (double)sm.bc[0];
  if (!(u < (T)(ratio * ratio))) return;
  for (int g = warp; g < Ng; g += NWARP) {
    T *Mg = proj_minv<T>(S, w, g);
    const int *inv = S.pinv + (size_t)g * Ns;
    const int tg = inv[t];
    if (s == 0) {
      const T *F = ftab<T>(S);
      for (int l = lane; l < N; l += 32) R[l] = F[(size_t)tg * Ns + inv[sm.ele[N + l]]];
      __syncwarp();
      proj_row_update(Mg, N, e, R, W, P);
    } else {
      const T *FT = fTtab<T>(S);
      for (int k = lane; k < N; k += 32) R[k] = FT[(size_t)tg * Ns + inv[sm.ele[k]]];
      __syncwarp();
      proj_col_update(Mg, N, e - N, R, W, Z);
    }
    if (lane == 0) sm.pi[g] = sm.pi[g] * (double)sm.rho[g] / rpf;
  }
  __syncthreads();
  for (int x = tid; x < Ns; x += NT)
    sm.jf[x] += vtab<T>(S)[(size_t)t * Ns + x] - vtab<T>(S)[(size_t)rs * Ns + x];
  if (tid == 0) {
    sm.ele[e] = t;
    sm.occ[s * Ns + rs] = -1;
    sm.occ[s * Ns + t] = e;
  }
  __syncthreads();
  mc.hop_a++;
  acc_since = (fabs(rpf) < SMALL_RATIO) ? RECOMPUTE_NOW : acc_since + 1;
}

// E_loc (Eq. MC with A = H) and the O_k row of the projected state.
template <typename T>
__device__ void proj_measure(const SysDev &S, const PSmem<T> &sm, int w, int row, int &buf,
                             MoveCounts &mc) {
  const int N = S.N, Ns = S.Ns, Ng = S.n_ops, tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  T *R = sm.vec + (size_t)warp * PVEC * VMC_MAX_N;
  T *W = R + VMC_MAX_N, *B = R + 5 * VMC_MAX_N;
  // diagonal terms
  double ed = 0.0;
  for (int i = tid; i < Ns; i += NT)
    if (sm.occ[i] >= 0 && sm.occ[Ns + i] >= 0) ed += S.U[i];
  for (int k = tid; k < S.n_V; k += NT) {
    const int a = S.V_i[k], b = S.V_j[k];
    const int na = (sm.occ[a] >= 0) + (sm.occ[Ns + a] >= 0);
    const int nb = (sm.occ[b] >= 0) + (sm.occ[Ns + b] >= 0);
    ed += S.V_val[k] * (double)(na * nb);
  }
  for (int k = tid; k < S.n_J; k += NT) {
    const int a = S.J_i[k], b = S.J_j[k];
    const int sa = (sm.occ[a] >= 0) - (sm.occ[Ns + a] >= 0);
    const int sb = (sm.occ[b] >= 0) - (sm.occ[Ns + b] >= 0);
    ed += S.J_val[k] * 0.25 * (double)(sa * sb);
  }
  // hopping: term k moves the spin-s electron on j = hop_j[k] to i = hop_i[k].
  // The (term, spin) pairs with a move are listed in order (q = 2k + s), then
  // taken in chunks that fit the per-warp vector area: for every operation g
  // in turn all warps of the CTA form their terms' ratios from the same M_g^-1
  // (warp per term, lanes over the electrons), so M_g^-1 is read from DRAM
  // once per chunk and then from L2, and each term's sum over g runs in g
  // order in FP64 (its slot is owned by one warp).
  double eo = 0.0;
  {
    const size_t vbytes = sizeof(T) * NWARP * PVEC * VMC_MAX_N;
    const int cap = (int)(vbytes / (sizeof(double) + sizeof(int2)));
    double *tacc = reinterpret_cast<double *>(sm.vec);
    int2 *tdesc = reinterpret_cast<int2 *>(tacc + cap);
    int *wcnt = reinterpret_cast<int *>(sm.red);   // per-warp counts of a listing round
    const int nq = 2 * S.n_hop;
    int q0 = 0;
    while (q0 < nq) {
      // ordered listing of the next pairs with a move, at most cap of them
      int nt = 0;
      __syncthreads();
      while (q0 < nq) {
        const int q = q0 + tid;
        int e = -1;
        if (q < nq) {
          const int k = q >> 1, sp = q & 1;
          const int i = S.hop_i[k], j = S.hop_j[k];
          e = sm.occ[sp * Ns + j];
          if (e >= 0 && sm.occ[sp * Ns + i] >= 0) e = -1;
          if (e >= 0 && S.local_spin && sm.occ[(1 - sp) * Ns + i] >= 0) e = -1;
          if (e >= 0 && S.lsite && (S.lsite[i] | S.lsite[j])) e = -1;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, e >= 0);
        if (lane == 0) wcnt[warp] = __popc(bal);
        __syncthreads();
        int before = 0, total = 0;
#pragma unroll
        for (int k = 0; k < NWARP; ++k) {
          before += (k < warp) ? wcnt[k] : 0;
          total += wcnt[k];
        }
        if (nt + total > cap) break;   // uniform: the round goes to the next chunk
        if (e >= 0) tdesc[nt + before + __popc(bal & ((1u << lane) - 1))] = make_int2(q, e);
        nt += total;
        q0 += NT;
        __syncthreads();   // wcnt is written again by the next round
      }
      for (int t = tid; t < nt; t += NT) tacc[t] = 0.0;
      __syncthreads();
      int *mup = sm.map + warp * 2 * VMC_MAX_N, *mdn = mup + VMC_MAX_N;
      const T *F = ftab<T>(S);
      const T *FT = fTtab<T>(S);
      for (int g = 0; g < Ng; ++g) {
        const T *Mg = proj_minv<T>(S, w, g);
        const int *inv = S.pinv + (size_t)g * Ns;
        const signed char *sg = S.psgn + (size_t)g * Ns;
        const double pg = sm.pi[g];
        // the electrons' sites mapped by g (g^-1 of each), once per operation
        __syncwarp();
        for (int l = lane; l < N; l += 32) {
          mup[l] = inv[sm.ele[l]];
          mdn[l] = inv[sm.ele[N + l]];
        }
        __syncwarp();
        // two terms per iteration, their loads in flight together: an up
        // electron e reads column e of M_g^-1 and f(g^-1 i, mapped down
        // sites); a down electron m row m and f(mapped up sites, g^-1 i)
        for (int t = warp; t < nt; t += 2 * NWARP) {
          const int t2 = t + NWARP;
          const bool two = t2 < nt;
          const int2 d1 = tdesc[t], d2 = tdesc[two ? t2 : t];
          const int i1 = S.hop_i[d1.x >> 1], i2 = S.hop_i[d2.x >> 1];
          const bool up1 = d1.y < N, up2 = d2.y < N;
          const T *tab1 = (up1 ? F : FT) + (size_t)inv[i1] * Ns;
          const T *tab2 = (up2 ? F : FT) + (size_t)inv[i2] * Ns;
          const int *mp1 = up1 ? mdn : mup, *mp2 = up2 ? mdn : mup;
          const int st1 = up1 ? N : 1, st2 = up2 ? N : 1;
          const T *m1 = Mg + (up1 ? d1.y : (d1.y - N) * N);
          const T *m2 = Mg + (up2 ? d2.y : (d2.y - N) * N);
          T s1 = (T)0, s2 = (T)0;
          for (int l = lane; l < N; l += 32) {
            const T a1 = tab1[mp1[l]], b1 = m1[(size_t)l * st1];
            const T a2 = tab2[mp2[l]], b2 = m2[(size_t)l * st2];
            s1 += a1 * b1;
            s2 += a2 * b2;
          }
          s1 = warp_sum(s1);
          s2 = warp_sum(s2);
          if (lane == 0) {
            const int j1 = S.hop_j[d1.x >> 1];
            tacc[t] += pg * (double)((sg[i1] * sg[j1] < 0) ? -s1 : s1);
            if (two) {
              const int j2 = S.hop_j[d2.x >> 1];
              tacc[t2] += pg * (double)((sg[i2] * sg[j2] < 0) ? -s2 : s2);
            }
          }
        }
      }
      __syncthreads();
      for (int t = tid; t < nt; t += NT) {
        const int2 d = tdesc[t];
        const int k = d.x >> 1, sp = d.x & 1;
        const int i = S.hop_i[k], j = S.hop_j[k];
        const T c = corr_factor<T>(corr_hop_v(sm.occ, sm.jf, sm.g, Ns, sp, j, i,
                                              vtab<T>(S)[(size_t)j * Ns + i]));
        eo += -S.hop_t[k] * tacc[t] * (double)c;
      }
      if (tid == 0) mc.meas_hop += nt;
    }
    __syncthreads();   // the vector area is the exchange terms' scratch next
  }
  // Heisenberg exchange: J/2 (S+_a S-_b + S-_a S+_b) = -J/2 x (labelled swap ratio)
  for (int k = warp; k < S.n_J; k += NWARP) {
    int a = S.J_i[k], b = S.J_j[k];
    int nu = sm.occ[a], md = sm.occ[Ns + b];
    bool ok = nu >= 0 && md >= 0 && sm.occ[Ns + a] < 0 && sm.occ[b] < 0;
    if (!ok) {
      const int a2 = b, b2 = a;
      nu = sm.occ[a2];
      md = sm.occ[Ns + b2];
      ok = nu >= 0 && md >= 0 && sm.occ[Ns + a2] < 0 && sm.occ[b2] < 0;
      a = a2;
      b = b2;
    }
    if (!ok || a == b) continue;
    double acc = 0.0;
    for (int g = 0; g < Ng; ++g) {
      T K[4];
      acc += sm.pi[g] * (double)proj_exchange_ratio(S, sm.ele, proj_minv<T>(S, w, g), g, nu,
                                                    md - N, a, b, R, W, B, K);
    }
    if (lane == 0) {
      eo += -0.5 * S.J_val[k] * acc;
      mc.meas_ex++;
    }
  }
  const double etot = block_sum_d(ed + eo, sm.red, buf);
  if (tid == 0) S.E[(size_t)w * S.n_samples + row] = etot;
  // O_k row: accumulated in the vector area (free again here) when it fits,
  // else in the global row; then written to the global row.
  T *Og = (T *)S.O + ((size_t)w * S.n_samples + row) * S.ldO;
  const bool shared_o = (size_t)S.ldO * sizeof(T) <= sizeof(T) * NWARP * PVEC * VMC_MAX_N;
  T *O = shared_o ? sm.vec : Og;
  __syncthreads();   // the exchange terms' scratch is done with
  for (int k = tid; k < S.ldO; k += NT) O[k] = (T)0;
  for (int i = tid; i < Ns; i += NT) sm.mval[i] = (sm.occ[i] >= 0) + (sm.occ[Ns + i] >= 0) - 1;
  __syncthreads();
  if (S.n_g > 0)
    for (int i = tid; i < Ns; i += NT)
      if (sm.occ[i] >= 0 && sm.occ[Ns + i] >= 0 && S.g_idx[i] >= 0) atomicAdd(O + S.g_idx[i], (T)1);
  if (S.n_v > 0 && !S.local_spin) {
    for (int c = warp; c < S.n_v; c += NWARP) {
      int a = 0;
      for (int q = S.vptr[c] + lane; q < S.vptr[c + 1]; q += 32) {
        const unsigned pr = S.vpair[q];
        a += sm.mval[pr & 0xFFFFu] * sm.mval[pr >> 16];
      }
      a = warp_sum(a);
      if (lane == 0) O[S.n_g + c] = (T)a;
    }
  }
  // pair orbital: sum_g pi_g sum_{n,m} M_g^-1[m][n] d M_g[n][m] / d f_k
  const int base = S.n_g + S.n_v;
  for (int g = warp; g < Ng; g += NWARP) {
    const T *Mg = proj_minv<T>(S, w, g);
    const int *inv = S.pinv + (size_t)g * Ns;
    const T pg = (T)sm.pi[g];
    // rows m of M_g^-1 in turn (coalesced), lanes over the up electrons n
    int rn[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int n = lane + 32 * u;
      rn[u] = (n < N) ? inv[sm.ele[n]] * Ns : 0;
    }
    for (int m = 0; m < N; ++m) {
      const int cm = inv[sm.ele[N + m]];
      const T *mrow = Mg + (size_t)m * N;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int n = lane + 32 * u;
        if (n < N) {
          const int cd = S.fcode[(size_t)rn[u] + cm];
          if (cd >= 0) {
            const T v = pg * mrow[n];
            atomicAdd(O + base + (cd >> 1), (cd & 1) ? -v : v);
          }
        }
      }
    }
  }
  __syncthreads();
  if (shared_o) {
    for (int k = tid; k < S.ldO; k += NT) Og[k] = O[k];
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(NT) k_proj_sample(const SysDev *systems, const int2 *work,
                                                    int n_work, int *work_ctr, uint2 key,
                                                    int n_first, int n_samples, int sweeps_between,
                                                    int sample_base) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ SysDev S;
  __shared__ int s_item;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(work_ctr, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= n_work) break;
    const int2 wk = work[item];
    load_sys(&S, systems + wk.x);
    const int w = wk.y;
    const int N = S.N, Ns = S.Ns, Ne = S.Ne, Ng = S.n_ops;
    PSmem<T> sm;
    proj_layout<T>(N, Ns, Ng, smem_raw, &sm);
    for (int k = tid; k < Ne; k += NT) sm.ele[k] = S.ele[(size_t)w * Ne + k];
    for (int k = tid; k < 2 * Ns; k += NT) sm.occ[k] = S.occ[(size_t)w * 2 * Ns + k];
    for (int k = tid; k < Ns; k += NT) sm.jf[k] = ((const T *)S.jf)[(size_t)w * Ns + k];
    for (int k = tid; k < Ns; k += NT) sm.g[k] = gtab<T>(S)[k];
    for (int k = tid; k < Ng; k += NT) sm.pi[k] = S.ppi[(size_t)w * Ng + k];
    __syncthreads();
    unsigned long long ctr = S.ctr[w];
    int rpos = NT, buf = 0;
    MoveCounts mc;
    int acc_since = S.acc_since[w];
    const long long props_first = (long long)n_first * Ne;
    for (long long p = 0; p < props_first; ++p) proj_propose(S, sm, w, key, ctr, rpos, mc, acc_since, buf);
    for (int s = 0; s < n_samples; ++s) {
      const long long props = (long long)sweeps_between * Ne;
      for (long long p = 0; p < props; ++p) proj_propose(S, sm, w, key, ctr, rpos, mc, acc_since, buf);
      __syncthreads();
      proj_measure(S, sm, w, sample_base + s, buf, mc);
      mc.samples++;
    }
    __syncthreads();
    for (int k = tid; k < Ne; k += NT) S.ele[(size_t)w * Ne + k] = sm.ele[k];
    for (int k = tid; k < 2 * Ns; k += NT) S.occ[(size_t)w * 2 * Ns + k] = sm.occ[k];
    for (int k = tid; k < Ns; k += NT) ((T *)S.jf)[(size_t)w * Ns + k] = sm.jf[k];
    for (int k = tid; k < Ng; k += NT) S.ppi[(size_t)w * Ng + k] = sm.pi[k];
    if (tid == 0) {
      const long long total = props_first + (long long)n_samples * sweeps_between * Ne;
      S.ctr[w] = ctr;
      S.n_prop[w] += total;
      S.n_acc[w] += mc.hop_a + mc.ex_a;
      S.cnt[8 * w + 0] += mc.hop_t;
      S.cnt[8 * w + 1] += mc.ex_t;
      S.cnt[8 * w + 2] += mc.hop_a;
      S.cnt[8 * w + 3] += mc.ex_a;
      S.cnt[8 * w + 6] += mc.samples;
      S.acc_since[w] = acc_since;
      S.status[w] &= ~VMC_ST_TIMEOUT;
    }
    // measured-ratio counts are per lane 0 of each warp: every thread adds its own
    if (mc.meas_hop) atomicAdd((unsigned long long *)&S.cnt[8 * w + 4], (unsigned long long)mc.meas_hop);
    if (mc.meas_ex) atomicAdd((unsigned long long *)&S.cnt[8 * w + 5], (unsigned long long)mc.meas_ex);
    __syncthreads();
  }
}

// Ratio check hook: psi(x')/psi(x) of candidate moves of one walker.
template <typename T>
__global__ void __launch_bounds__(NT) k_proj_eval(const SysDev *systems, int sys, int w,
                                                  int n_moves, const int *moves, double *out) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ SysDev S;
  load_sys(&S, systems + sys);
  const int N = S.N, Ns = S.Ns, Ne = S.Ne, Ng = S.n_ops, tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  PSmem<T> sm;
  proj_layout<T>(N, Ns, Ng, smem_raw, &sm);
  for (int k = tid; k < Ne; k += NT) sm.ele[k] = S.ele[(size_t)w * Ne + k];
  for (int k = tid; k < 2 * Ns; k += NT) sm.occ[k] = S.occ[(size_t)w * 2 * Ns + k];
  for (int k = tid; k < Ns; k += NT) sm.jf[k] = ((const T *)S.jf)[(size_t)w * Ns + k];
  for (int k = tid; k < Ns; k += NT) sm.g[k] = gtab<T>(S)[k];
  for (int k = tid; k < Ng; k += NT) sm.pi[k] = S.ppi[(size_t)w * Ng + k];
  __syncthreads();
  T *R = sm.vec + (size_t)warp * PVEC * VMC_MAX_N;
  T *W = R + VMC_MAX_N, *B = R + 5 * VMC_MAX_N;
  int buf = 0;
  for (int q = 0; q < n_moves; ++q) {
    const int kind = moves[3 * q], a = moves[3 * q + 1], b = moves[3 * q + 2];
    double res = 0.0;
    if (kind == 0) {
      if (a >= 0 && a < Ne && b >= 0 && b < Ns) {
        const int s = (a >= N) ? 1 : 0;
        const int rs = sm.ele[a];
        if (sm.occ[s * Ns + b] < 0 && !(S.local_spin && sm.occ[(1 - s) * Ns + b] >= 0) &&
            !(S.lsite && (S.lsite[b] | S.lsite[rs]))) {
          double part = 0.0;
          for (int g = warp; g < Ng; g += NWARP) {
            const T rho = proj_hop_ratio(S, sm.ele, proj_minv<T>(S, w, g), g, a, b);
            const signed char *sg = S.psgn + (size_t)g * Ns;
            part += sm.pi[g] * (double)((sg[b] * sg[rs] < 0) ? -rho : rho);
          }
          const double rpf = block_sum_d(lane == 0 ? part : 0.0, sm.red, buf);
          res = rpf * (double)corr_factor<T>(corr_hop_v(sm.occ, sm.jf, sm.g, Ns, s, rs, b,
                                                         vtab<T>(S)[(size_t)rs * Ns + b]));
        }
      }
    } else if (a >= 0 && a < N && b >= N && b < Ne) {
      const int i = sm.ele[a], j = sm.ele[b];
      if (i != j && sm.occ[Ns + i] < 0 && sm.occ[j] < 0) {
        double part = 0.0;
        for (int g = warp; g < Ng; g += NWARP) {
          T K[4];
          part += sm.pi[g] * (double)proj_exchange_ratio(S, sm.ele, proj_minv<T>(S, w, g), g, a,
                                                         b - N, i, j, R, W, B, K);
        }
        res = block_sum_d(lane == 0 ? part : 0.0, sm.red, buf);
      }
    }
    if (tid == 0) out[q] = res;
    __syncthreads();
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host-side launch wrappers
// ---------------------------------------------------------------------------
size_t vmc_proj_smem(int precision, int N, int Ns, int n_ops) {
  return precision == 0 ? proj_layout<double>(N, Ns, n_ops, nullptr, nullptr)
                        : proj_layout<float>(N, Ns, n_ops, nullptr, nullptr);
}

int vmc_proj_occupancy(int precision, size_t smem) {
  int nb = 0;
  if (precision == 0)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_proj_sample<double>, NT, smem);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_proj_sample<float>, NT, smem);
  return nb;
}

cudaError_t vmc_proj_set_smem(size_t s_sample, size_t s_build) {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_proj_sample<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_sample))) return e;
  if ((e = cudaFuncSetAttribute(k_proj_sample<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_sample))) return e;
  if ((e = cudaFuncSetAttribute(k_proj_eval<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_sample))) return e;
  if ((e = cudaFuncSetAttribute(k_proj_eval<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_sample))) return e;
  if ((e = cudaFuncSetAttribute(k_proj_build<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_build))) return e;
  if ((e = cudaFuncSetAttribute(k_proj_build<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_build))) return e;
  return cudaSuccess;
}

cudaError_t vmc_launch_proj_build(const SysDev *d_sys, const int2 *d_work, int n_work, int n_ops,
                                  int precision, int only_due, int due_threshold, size_t smem,
                                  cudaStream_t st, long long *nl) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long items = (long long)n_work * n_ops;
  const int g1 = (int)(items < 8LL * nsm ? items : 8LL * nsm);
  const int g2 = n_work < 8 * nsm ? n_work : 8 * nsm;
  if (g1 < 1) return cudaSuccess;
  if (precision == 0) {
    k_proj_build<double><<<g1, NT, smem, st>>>(d_sys, d_work, n_work, n_ops, only_due, due_threshold);
    k_proj_shares<double><<<g2, NT, 0, st>>>(d_sys, d_work, n_work, only_due, due_threshold);
  } else {
    k_proj_build<float><<<g1, NT, smem, st>>>(d_sys, d_work, n_work, n_ops, only_due, due_threshold);
    k_proj_shares<float><<<g2, NT, 0, st>>>(d_sys, d_work, n_work, only_due, due_threshold);
  }
  *nl += 2;
  return cudaGetLastError();
}

cudaError_t vmc_launch_proj_sample(const SysDev *d_sys, const int2 *d_work, int n_work,
                                   int *d_work_ctr, int precision, uint64_t seed, int n_first,
                                   int n_samples, int sweeps_between, int sample_base, int grid,
                                   size_t smem, cudaStream_t st, long long *nl) {
  cudaError_t e = cudaMemsetAsync(d_work_ctr, 0, sizeof(int), st);
  if (e) return e;
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  if (grid > n_work) grid = n_work;
  if (grid < 1) return cudaSuccess;
  if (precision == 0)
    k_proj_sample<double><<<grid, NT, smem, st>>>(d_sys, d_work, n_work, d_work_ctr, key, n_first,
                                                  n_samples, sweeps_between, sample_base);
  else
    k_proj_sample<float><<<grid, NT, smem, st>>>(d_sys, d_work, n_work, d_work_ctr, key, n_first,
                                                 n_samples, sweeps_between, sample_base);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t vmc_launch_proj_eval(const SysDev *d_sys, int sys, int walker, int precision,
                                 int n_moves, const int *d_moves, double *d_out, size_t smem,
                                 cudaStream_t st, long long *nl) {
  if (precision == 0)
    k_proj_eval<double><<<1, NT, smem, st>>>(d_sys, sys, walker, n_moves, d_moves, d_out);
  else
    k_proj_eval<float><<<1, NT, smem, st>>>(d_sys, sys, walker, n_moves, d_moves, d_out);
  ++*nl;
  return cudaGetLastError();
}
