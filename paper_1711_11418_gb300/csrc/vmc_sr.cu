// Stochastic reconfiguration kernels (mVMC paper, Sec. 3.3.1-3.3.2):
//   o_k = <O_k>, E = <E_loc>,
//   S_km = <O_k O_m> - <O_k><O_m>  =  (1/N_MC) sum_mu (O_k,mu - o_k)(O_m,mu - o_m),
//   g_m  = <E O_m> - <E><O_m>      =  (1/N_MC) sum_mu (O_m,mu - o_m)(E_mu - E),
//   S~_kk = S_kk (1 + shift_rel) + shift_abs,
//   S~ x = g by Cholesky (S~ = L L^T) or by CG (Algorithm 1) with the SR-CG
//   product y = (1/N_MC) O^T (O v) - o (o . v) + shift terms,
//   alpha += -dtau x  (Eq. SR_equation_system).
// Sample rows are the rows of O (row-major, leading dimension ldO), in FP64
// (plain form) or FP32 (mixed form); every reduction accumulates in FP64.
#include "vmc_common.cuh"

#include <math.h>
#include <vector>

namespace {

constexpr int RB = 256;        // threads of the column-reduction kernels
constexpr int ROWCHUNK = 2048; // rows per partial of a column reduction

template <typename TO>
__device__ __forceinline__ double ld(const TO *p) { return (double)*p; }

// Partial column reductions: part[c][k] = sum over rows of chunk c of
//   mode 0: O_rk                      (mean)
//   mode 1: (O_rk - o_k) (E_r - ebar)  (force g)
//   mode 2: (O_rk - o_k)^2             (diagonal of S)
//   mode 3: O_rk t_r                   (CG: O^T t)
template <typename TO>
__global__ void k_colreduce(const TO *O, int ldO, int rows, int Np, const double *obar,
                            const double *wvec, double wshift, int mode, double *part,
                            const int *done) {
  const int k = blockIdx.x * RB + threadIdx.x;
  const int c = blockIdx.y;
  if (k >= Np || (done && *done)) return;
  const int r0 = c * ROWCHUNK;
  const int r1 = min(rows, r0 + ROWCHUNK);
  const double ok = (mode == 1 || mode == 2) ? obar[k] : 0.0;
  double s = 0.0;
  for (int r = r0; r < r1; ++r) {
    const double o = ld(O + (size_t)r * ldO + k);
    switch (mode) {
      case 0: s += o; break;
      case 1: s += (o - ok) * (wvec[r] - wshift); break;
      case 2: s += (o - ok) * (o - ok); break;
      default: s += o * wvec[r]; break;
    }
  }
  part[(size_t)c * Np + k] = s;
}

__global__ void k_sum_parts(const double *part, int nparts, int Np, double scale, double *out,
                            const int *done) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Np || (done && *done)) return;
  double s = 0.0;
  for (int c = 0; c < nparts; ++c) s += part[(size_t)c * Np + k];
  out[k] = s * scale;
}

__global__ void k_mean_vec(const double *v, int n, double *out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0] / n;
}

// S = (1/rows) (O - o)^T (O - o): 64x64 output tiles of the upper triangle,
// split over row chunks (atomic accumulation into S, which starts at zero).
constexpr int ST = 64, SKK = 16;
template <typename TO>
__global__ void __launch_bounds__(256) k_syrk(const TO *O, int ldO, int rows, int Np,
                                              const double *obar, double scale, int rows_per_split,
                                              double *S) {
  // map blockIdx.x to an upper-triangular tile pair (bi <= bj)
  int t = blockIdx.x, bi = 0;
  const int nt = (Np + ST - 1) / ST;
  while (t >= nt - bi) {
    t -= nt - bi;
    ++bi;
  }
  const int bj = bi + t;
  const int r0 = blockIdx.y * rows_per_split;
  const int r1 = min(rows, r0 + rows_per_split);
  __shared__ double As[SKK][ST + 1];
  __shared__ double Bs[SKK][ST + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4] = {};
  for (int rb = r0; rb < r1; rb += SKK) {
    for (int q = threadIdx.x; q < SKK * ST; q += 256) {
      const int rr = q / ST, cc = q % ST;
      const int r = rb + rr;
      const int ka = bi * ST + cc, kb = bj * ST + cc;
      As[rr][cc] = (r < r1 && ka < Np) ? ld(O + (size_t)r * ldO + ka) - obar[ka] : 0.0;
      Bs[rr][cc] = (r < r1 && kb < Np) ? ld(O + (size_t)r * ldO + kb) - obar[kb] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < SKK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[kk][ty + 16 * u];
        b[u] = Bs[kk][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = bi * ST + ty + 16 * u, j = bj * ST + tx + 16 * v;
      if (i < Np && j < Np && i <= j) {
        atomicAdd(S + (size_t)i * Np + j, acc[u][v] * scale);
      }
    }
}

// FP32 variant for the mixed form: FP32 products and FP32 accumulation over
// at most 1024 rows per split, FP64 accumulation across splits.
__global__ void __launch_bounds__(256) k_syrk32(const float *O, int ldO, int rows, int Np,
                                                const double *obar, double scale,
                                                int rows_per_split, double *S) {
  int t = blockIdx.x, bi = 0;
  const int nt = (Np + ST - 1) / ST;
  while (t >= nt - bi) {
    t -= nt - bi;
    ++bi;
  }
  const int bj = bi + t;
  const int r0 = blockIdx.y * rows_per_split;
  const int r1 = min(rows, r0 + rows_per_split);
  __shared__ float As[SKK][ST + 1];
  __shared__ float Bs[SKK][ST + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float acc[4][4] = {};
  for (int rb = r0; rb < r1; rb += SKK) {
    for (int q = threadIdx.x; q < SKK * ST; q += 256) {
      const int rr = q / ST, cc = q % ST;
      const int r = rb + rr;
      const int ka = bi * ST + cc, kb = bj * ST + cc;
      As[rr][cc] = (r < r1 && ka < Np) ? (float)((double)O[(size_t)r * ldO + ka] - obar[ka]) : 0.f;
      Bs[rr][cc] = (r < r1 && kb < Np) ? (float)((double)O[(size_t)r * ldO + kb] - obar[kb]) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < SKK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[kk][ty + 16 * u];
        b[u] = Bs[kk][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = bi * ST + ty + 16 * u, j = bj * ST + tx + 16 * v;
      if (i < Np && j < Np && i <= j) atomicAdd(S + (size_t)i * Np + j, (double)acc[u][v] * scale);
    }
}

// Mirror the upper triangle and apply the diagonal shift.
__global__ void k_mirror_shift(double *S, int Np, double shift_rel, double shift_abs) {
  const size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (q >= (size_t)Np * Np) return;
  const int i = (int)(q / Np), j = (int)(q % Np);
  if (i > j) S[q] = S[(size_t)j * Np + i];
  else if (i == j) S[q] = S[q] * (1.0 + shift_rel) + shift_abs;
}

// Blocked right-looking Cholesky (lower triangle in place), panels of CB
// columns: factor the diagonal block (one CTA), solve the panel below it
// (L_ij = A_ij L_jj^-T), update the trailing lower triangle (A -= L L^T).
constexpr int CB = 32;

__global__ void k_potrf_diag(double *A, int n, int j0, int nb, int *info) {
  __shared__ double D[CB][CB + 1];
  for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) {
    const int r = q / nb, c = q % nb;
    D[r][c] = A[(size_t)(j0 + r) * n + j0 + c];
  }
  __syncthreads();
  for (int k = 0; k < nb; ++k) {
    if (threadIdx.x == 0) {
      const double a = D[k][k];
      if (!(a > 0.0) || !isfinite(a)) {
        if (*info == 0) *info = j0 + k + 1;
        D[k][k] = 1.0;
      } else {
        D[k][k] = sqrt(a);
      }
    }
    __syncthreads();
    const double inv = 1.0 / D[k][k];
    for (int r = k + 1 + threadIdx.x; r < nb; r += blockDim.x) D[r][k] *= inv;
    __syncthreads();
    for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) {
      const int r = q / nb, c = q % nb;
      if (c > k && r >= c) D[r][c] -= D[r][k] * D[c][k];
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) {
    const int r = q / nb, c = q % nb;
    if (r >= c) A[(size_t)(j0 + r) * n + j0 + c] = D[r][c];
  }
}

__global__ void k_trsm_panel(double *A, int n, int j0, int nb) {
  __shared__ double L[CB][CB + 1];
  for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) {
    const int r = q / nb, c = q % nb;
    L[r][c] = (r >= c) ? A[(size_t)(j0 + r) * n + j0 + c] : 0.0;
  }
  __syncthreads();
  const int i = j0 + nb + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x[CB];
  double *row = A + (size_t)i * n + j0;
#pragma unroll
  for (int k = 0; k < CB; ++k) x[k] = (k < nb) ? row[k] : 0.0;
#pragma unroll
  for (int k = 0; k < CB; ++k) {
    if (k < nb) {
      double v = x[k];
#pragma unroll
      for (int l = 0; l < CB; ++l)
        if (l < k) v -= x[l] * L[k][l];
      x[k] = v / L[k][k];
    }
  }
#pragma unroll
  for (int k = 0; k < CB; ++k)
    if (k < nb) row[k] = x[k];
}

// trailing A[i][k] -= sum_l L[i][j0+l] L[k][j0+l], j1 <= k <= i < n (j1 = j0 + nb)
__global__ void __launch_bounds__(256) k_syrk_trailing(double *A, int n, int j0, int nb) {
  const int j1 = j0 + nb;
  const int m = n - j1;
  const int nt = (m + 63) / 64;
  int t = blockIdx.x, bi = 0;
  while (t >= bi + 1) {
    t -= bi + 1;
    ++bi;
  }
  const int bj = t;   // bj <= bi: lower tiles
  __shared__ double Pi[CB][65];
  __shared__ double Pk[CB][65];
  for (int q = threadIdx.x; q < CB * 64; q += 256) {
    const int l = q / 64, r = q % 64;
    const int ii = j1 + bi * 64 + r, kk = j1 + bj * 64 + r;
    Pi[l][r] = (l < nb && ii < n) ? A[(size_t)ii * n + j0 + l] : 0.0;
    Pk[l][r] = (l < nb && kk < n) ? A[(size_t)kk * n + j0 + l] : 0.0;
  }
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4] = {};
  for (int l = 0; l < nb; ++l) {
    double a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a[u] = Pi[l][ty + 16 * u];
      b[u] = Pk[l][tx + 16 * u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
  }
  (void)nt;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = j1 + bi * 64 + ty + 16 * u, k = j1 + bj * 64 + tx + 16 * v;
      if (i < n && k < n && k <= i) A[(size_t)i * n + k] -= acc[u][v];
    }
}


// Both triangular solves in one CTA of 1024 threads (x holds b on entry):
// per panel of CB rows, warp 0 solves the diagonal block (lane-parallel dot
// products), then all warps update the rest of the vector -- forward: one
// warp per row over the panel's columns; backward: one thread per entry over
// the panel's rows (both coalesced).
__global__ void __launch_bounds__(1024) k_chol_solve_blocked(const double *L, int n, double *x) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int p0 = 0; p0 < n; p0 += CB) {
    const int nb = min(CB, n - p0);
    if (warp == 0) {
      for (int k = 0; k < nb; ++k) {
        double s = (lane < k) ? L[(size_t)(p0 + k) * n + p0 + lane] * x[p0 + lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) x[p0 + k] = (x[p0 + k] - s) / L[(size_t)(p0 + k) * n + p0 + k];
        __syncwarp();
      }
    }
    __syncthreads();
    for (int i = p0 + nb + warp; i < n; i += nw) {
      double s = (lane < nb) ? L[(size_t)i * n + p0 + lane] * x[p0 + lane] : 0.0;
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) x[i] -= s;
    }
    __syncthreads();
  }
  for (int p0 = ((n - 1) / CB) * CB; p0 >= 0; p0 -= CB) {
    const int nb = min(CB, n - p0);
    if (warp == 0) {
      for (int k = nb - 1; k >= 0; --k) {
        double s = (lane > k && lane < nb) ? L[(size_t)(p0 + lane) * n + p0 + k] * x[p0 + lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) x[p0 + k] = (x[p0 + k] - s) / L[(size_t)(p0 + k) * n + p0 + k];
        __syncwarp();
      }
    }
    __syncthreads();
    for (int i = tid; i < p0; i += blockDim.x) {
      double s = 0.0;
      for (int l = 0; l < nb; ++l) s += L[(size_t)(p0 + l) * n + i] * x[p0 + l];
      x[i] -= s;
    }
    __syncthreads();
  }
}



// t = O v (one warp per row)
template <typename TO>
__global__ void k_gemv_rows(const TO *O, int ldO, int rows, int Np, const double *v, double *t,
                            const int *done) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= rows || *done) return;
  const TO *o = O + (size_t)warp * ldO;
  double s = 0.0;
  for (int k = lane; k < Np; k += 32) s += ld(o + k) * v[k];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) t[warp] = s;
}

__global__ void k_dot(const double *a, const double *b, int n, double *out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += a[i] * b[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

// CG (Algorithm 1) on the device.  cg[0..1]: rho ping-pong, cg[2]: p.w,
// cg[3]: o.v, cg[4]: threshold eps^2 |b|^2; flags[0]: done, flags[1]:
// iterations, flags[2]: breakdown.
__global__ void k_cg_finish(const double *u, const double *obar, const double *odv,
                            const double *diagS, const double *v, double shift_rel,
                            double shift_abs, int n, double *w, const int *done) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n || *done) return;
  w[k] = u[k] - obar[k] * odv[0] + (shift_rel * diagS[k] + shift_abs) * v[k];
}

__global__ void k_dot_dev(const double *a, const double *b, int n, double *out, const int *done) {
  __shared__ double red[256];
  if (done && *done) return;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += a[i] * b[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

// x += alpha p, r -= alpha w with alpha = rho / (p.w)
__global__ void k_cg_update_xr(double *x, double *r, const double *p, const double *w,
                               const double *rho, const double *pw, int n, int *flags) {
  if (flags[0]) return;
  const double alpha = rho[0] / pw[0];
  if (!isfinite(alpha) || pw[0] == 0.0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      flags[2] = 1;
      flags[0] = 1;
    }
    return;
  }
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  x[k] += alpha * p[k];
  r[k] -= alpha * w[k];
}

// rho' = r.r; done if rho' < threshold (one block)
__global__ void k_cg_check(const double *r, int n, double *rho_new, const double *thr, int *flags) {
  __shared__ double red[256];
  if (flags[0]) return;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += r[i] * r[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    rho_new[0] = red[0];
    flags[1] += 1;
    if (!(red[0] >= thr[0])) flags[0] = 1;   // converged (or NaN: flagged below)
    if (!isfinite(red[0])) flags[2] = 1;
  }
}

// p = r + (rho'/rho) p
__global__ void k_cg_update_p(double *p, const double *r, const double *rho_new,
                              const double *rho, int n, const int *flags) {
  if (flags[0]) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  p[k] = r[k] + (rho_new[0] / rho[0]) * p[k];
}

__global__ void k_cg_init(double *cg, int *flags, double eps) {
  // cg[0] holds |b|^2 = rho_0 on entry
  cg[4] = eps * eps * cg[0];
  flags[0] = (cg[0] == 0.0) ? 1 : 0;
  flags[1] = 0;
  flags[2] = 0;
}

__global__ void k_update_params(double *p, const double *x, double dtau, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) p[k] += -dtau * x[k];
}

template <typename TO>
cudaError_t colreduce(const SrWork &w, const TO *O, int mode, const double *wvec, double wshift,
                      double scale, double *out, cudaStream_t st, long long *nl,
                      const int *done = nullptr) {
  const int nparts = (w.rows + ROWCHUNK - 1) / ROWCHUNK;
  dim3 grid((w.Np + RB - 1) / RB, nparts);
  k_colreduce<TO><<<grid, RB, 0, st>>>(O, w.ldO, w.rows, w.Np, w.obar, wvec, wshift, mode, w.part,
                                       done);
  k_sum_parts<<<(w.Np + 255) / 256, 256, 0, st>>>(w.part, nparts, w.Np, scale, out, done);
  *nl += 2;
  return cudaGetLastError();
}

cudaError_t colreduce_any(const SrWork &w, int mode, const double *wvec, double wshift,
                          double scale, double *out, cudaStream_t st, long long *nl,
                          const int *done = nullptr) {
  if (w.precision == 0)
    return colreduce<double>(w, (const double *)w.O, mode, wvec, wshift, scale, out, st, nl, done);
  return colreduce<float>(w, (const float *)w.O, mode, wvec, wshift, scale, out, st, nl, done);
}

}  // namespace

cudaError_t vmc_sr_means(const SrWork &w, cudaStream_t st, long long *nl) {
  k_mean_vec<<<1, 256, 0, st>>>(w.E, w.rows, w.ebar);
  ++*nl;
  return colreduce_any(w, 0, nullptr, 0.0, 1.0 / w.rows, w.obar, st, nl);
}

cudaError_t vmc_sr_build_g(const SrWork &w, cudaStream_t st, long long *nl) {
  // wshift must be a host value: read ebar back (small, once per SR step)
  double ebar = 0.0;
  cudaError_t e = cudaMemcpyAsync(&ebar, w.ebar, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e) return e;
  if ((e = cudaStreamSynchronize(st))) return e;
  return colreduce_any(w, 1, w.E, ebar, 1.0 / w.rows, w.g, st, nl);
}

cudaError_t vmc_sr_diag(const SrWork &w, cudaStream_t st, long long *nl) {
  return colreduce_any(w, 2, nullptr, 0.0, 1.0 / w.rows, w.diagS, st, nl);
}

cudaError_t vmc_sr_build_S(const SrWork &w, double shift_rel, double shift_abs, cudaStream_t st,
                           long long *nl) {
  cudaError_t e = cudaMemsetAsync(w.S, 0, sizeof(double) * (size_t)w.Np * w.Np, st);
  if (e) return e;
  const int nt = (w.Np + ST - 1) / ST;
  const int ntiles = nt * (nt + 1) / 2;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int splits = (4 * nsm + ntiles - 1) / ntiles;
  const int max_splits = (w.rows + 255) / 256;
  if (splits > max_splits) splits = max_splits;
  if (w.precision != 0 && splits < (w.rows + 1023) / 1024) splits = (w.rows + 1023) / 1024;
  if (splits < 1) splits = 1;
  int rps = (w.rows + splits - 1) / splits;
  rps = (rps + SKK - 1) / SKK * SKK;
  splits = (w.rows + rps - 1) / rps;
  dim3 grid(ntiles, splits);
  if (w.precision == 0)
    k_syrk<double><<<grid, 256, 0, st>>>((const double *)w.O, w.ldO, w.rows, w.Np, w.obar,
                                         1.0 / w.rows, rps, w.S);
  else
    k_syrk32<<<grid, 256, 0, st>>>((const float *)w.O, w.ldO, w.rows, w.Np, w.obar,
                                   1.0 / w.rows, rps, w.S);
  const size_t n2 = (size_t)w.Np * w.Np;
  k_mirror_shift<<<(unsigned)((n2 + 255) / 256), 256, 0, st>>>(w.S, w.Np, shift_rel, shift_abs);
  *nl += 2;
  return cudaGetLastError();
}

int vmc_sr_cholesky_solve(const SrWork &w, cudaStream_t st, long long *nl) {
  const int n = w.Np;
  cudaMemsetAsync(w.info, 0, sizeof(int), st);
  for (int j0 = 0; j0 < n; j0 += CB) {
    const int nb = n - j0 < CB ? n - j0 : CB;
    k_potrf_diag<<<1, 256, 0, st>>>(w.S, n, j0, nb, w.info);
    ++*nl;
    const int rem = n - j0 - nb;
    if (rem > 0) {
      k_trsm_panel<<<(rem + 127) / 128, 128, 0, st>>>(w.S, n, j0, nb);
      const int nt = (rem + 63) / 64;
      k_syrk_trailing<<<nt * (nt + 1) / 2, 256, 0, st>>>(w.S, n, j0, nb);
      *nl += 2;
    }
  }
  cudaMemcpyAsync(w.x, w.g, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
  k_chol_solve_blocked<<<1, 1024, 0, st>>>(w.S, n, w.x);
  *nl += 1;
  if (cudaGetLastError() != cudaSuccess) return -3;
  int info = 0;
  if (cudaMemcpyAsync(&info, w.info, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return -3;
  if (cudaStreamSynchronize(st) != cudaSuccess) return -3;
  return info ? -4 : 0;
}

// One SR-CG product out = S~ v (Sec. 3.3.2): t = O v, u = O^T t / rows,
// out = u - o (o . v) + shift terms.  2 (rows + 1) Np products for the S part.
static cudaError_t srcg_matvec(const SrWork &w, const double *v, double *out, double shift_rel,
                               double shift_abs, const int *done, cudaStream_t st, long long *nl) {
  const int threads = 256;
  const int blocks = (int)(((size_t)w.rows * 32 + threads - 1) / threads);
  if (w.precision == 0)
    k_gemv_rows<double><<<blocks, threads, 0, st>>>((const double *)w.O, w.ldO, w.rows, w.Np, v, w.t, done);
  else
    k_gemv_rows<float><<<blocks, threads, 0, st>>>((const float *)w.O, w.ldO, w.rows, w.Np, v, w.t, done);
  ++*nl;
  cudaError_t e = colreduce_any(w, 3, w.t, 0.0, 1.0 / w.rows, w.r + w.Np, st, nl, done);
  if (e) return e;
  k_dot_dev<<<1, 256, 0, st>>>(w.obar, v, w.Np, w.scal + 3, done);
  k_cg_finish<<<(w.Np + 255) / 256, 256, 0, st>>>(w.r + w.Np, w.obar, w.scal + 3, w.diagS, v,
                                                   shift_rel, shift_abs, w.Np, out, done);
  *nl += 2;
  return cudaGetLastError();
}

// Dense product out = S~ v with S~ (shift included) stored row-major (one warp per row).
__global__ void k_gemv_dense(const double *S, int n, const double *v, double *out, const int *done) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (row >= n || *done) return;
  const double *r = S + (size_t)row * n;
  double s = 0.0;
  for (int k = lane; k < n; k += 32) s += r[k] * v[k];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[row] = s;
}

// Algorithm 1 with x0 = 0, run on the device in batches of iterations; the
// host reads the convergence flag once per batch.  w.r holds 2 Np doubles.
// dense = 0: SR-CG product from O (S never formed); dense = 1: product with
// the dense S~ in w.S.
int vmc_sr_cg_solve(const SrWork &w, double shift_rel, double shift_abs, double eps, int kmax,
                    int *iters, cudaStream_t st, long long *nl, int dense) {
  const int n = w.Np, g = (n + 255) / 256;
  int *flags = w.info;
  double *cg = w.scal;
  cudaMemsetAsync(w.x, 0, sizeof(double) * n, st);
  cudaMemcpyAsync(w.r, w.g, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(w.p, w.g, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
  k_dot_dev<<<1, 256, 0, st>>>(w.r, w.r, n, cg + 0, nullptr);
  k_cg_init<<<1, 1, 0, st>>>(cg, flags, eps);
  *nl += 2;
  const int batch = 16;
  int h[3] = {0, 0, 0};
  for (int k = 1; k <= kmax; ++k) {
    double *rho = cg + ((k - 1) & 1), *rho_new = cg + (k & 1);
    if (dense) {
      k_gemv_dense<<<(int)(((size_t)n * 32 + 255) / 256), 256, 0, st>>>(w.S, n, w.p, w.w, flags);
      ++*nl;
    } else if (srcg_matvec(w, w.p, w.w, shift_rel, shift_abs, flags, st, nl) != cudaSuccess) {
      return -3;
    }
    k_dot_dev<<<1, 256, 0, st>>>(w.p, w.w, n, cg + 2, flags);
    k_cg_update_xr<<<g, 256, 0, st>>>(w.x, w.r, w.p, w.w, rho, cg + 2, n, flags);
    k_cg_check<<<1, 256, 0, st>>>(w.r, n, rho_new, cg + 4, flags);
    k_cg_update_p<<<g, 256, 0, st>>>(w.p, w.r, rho_new, rho, n, flags);
    *nl += 4;
    if (k % batch == 0 || k == kmax) {
      if (cudaMemcpyAsync(h, flags, sizeof(int) * 3, cudaMemcpyDeviceToHost, st) != cudaSuccess) return -3;
      if (cudaStreamSynchronize(st) != cudaSuccess) return -3;
      if (h[0]) break;
    }
  }
  if (cudaMemcpyAsync(h, flags, sizeof(int) * 3, cudaMemcpyDeviceToHost, st) != cudaSuccess) return -3;
  if (cudaStreamSynchronize(st) != cudaSuccess) return -3;
  *iters = h[1];
  if (h[2]) return -5;
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

cudaError_t vmc_sr_update_params(double *params, const double *x, double dtau, int Np,
                                 cudaStream_t st, long long *nl) {
  k_update_params<<<(Np + 255) / 256, 256, 0, st>>>(params, x, dtau, Np);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t vmc_dot_host(const double *a, const double *b, int n, double *out_host,
                         double *d_scratch, cudaStream_t st, long long *nl) {
  k_dot<<<1, 256, 0, st>>>(a, b, n, d_scratch);
  ++*nl;
  cudaError_t e = cudaMemcpyAsync(out_host, d_scratch, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e) return e;
  return cudaStreamSynchronize(st);
}
