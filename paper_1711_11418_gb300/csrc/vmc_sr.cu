// Stochastic reconfiguration kernels (mVMC paper, Sec. 2.3.1-2.3.2):
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
                            const double *wvec, double wshift, int mode, double *part) {
  const int k = blockIdx.x * RB + threadIdx.x;
  const int c = blockIdx.y;
  if (k >= Np) return;
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

__global__ void k_sum_parts(const double *part, int nparts, int Np, double scale, double *out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Np) return;
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

// Mirror the upper triangle and apply the diagonal shift.
__global__ void k_mirror_shift(double *S, int Np, double shift_rel, double shift_abs) {
  const size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (q >= (size_t)Np * Np) return;
  const int i = (int)(q / Np), j = (int)(q % Np);
  if (i > j) S[q] = S[(size_t)j * Np + i];
  else if (i == j) S[q] = S[q] * (1.0 + shift_rel) + shift_abs;
}

// Right-looking Cholesky, one column per pair of launches (lower triangle in place).
__global__ void k_chol_col(double *A, int n, int j, int *info) {
  __shared__ double d;
  if (threadIdx.x == 0) {
    const double a = A[(size_t)j * n + j];
    if (!(a > 0.0) || !isfinite(a)) {
      if (*info == 0) *info = j + 1;
      d = 1.0;
    } else {
      d = sqrt(a);
    }
    A[(size_t)j * n + j] = d;
  }
  __syncthreads();
  const double inv = 1.0 / d;
  for (int i = j + 1 + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    A[(size_t)i * n + j] *= inv;
}

__global__ void k_chol_update(double *A, int n, int j) {
  // trailing A[i][k] -= L[i][j] L[k][j] for j < k <= i
  const int m = n - j - 1;
  const size_t tot = (size_t)m * m;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < tot;
       q += (size_t)gridDim.x * blockDim.x) {
    const int i = j + 1 + (int)(q / m), k = j + 1 + (int)(q % m);
    if (k <= i) A[(size_t)i * n + k] -= A[(size_t)i * n + j] * A[(size_t)k * n + j];
  }
}

// Forward (L y = b) then backward (L^T x = y) substitution, one block.
__global__ void k_chol_solve(const double *L, int n, const double *b, double *x) {
  extern __shared__ double y[];
  for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = b[i];
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const double yj = y[j] / L[(size_t)j * n + j];
    __syncthreads();
    if (threadIdx.x == 0) y[j] = yj;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) y[i] -= L[(size_t)i * n + j] * yj;
    __syncthreads();
  }
  for (int j = n - 1; j >= 0; --j) {
    const double xj = y[j] / L[(size_t)j * n + j];
    __syncthreads();
    if (threadIdx.x == 0) y[j] = xj;
    for (int i = threadIdx.x; i < j; i += blockDim.x) y[i] -= L[(size_t)j * n + i] * xj;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = y[i];
}

// t = O v (one warp per row)
template <typename TO>
__global__ void k_gemv_rows(const TO *O, int ldO, int rows, int Np, const double *v, double *t) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= rows) return;
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

// w = u - o (o . v) + (shift_rel diagS + shift_abs) v, where u = O^T t / rows
// and odv = o . v is a device scalar.
__global__ void k_cg_finish(const double *u, const double *obar, const double *odv,
                            const double *diagS, const double *v, double shift_rel,
                            double shift_abs, int n, double *w) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  w[k] = u[k] - obar[k] * odv[0] + (shift_rel * diagS[k] + shift_abs) * v[k];
}

__global__ void k_axpy(double *y, const double *x, const double *num, const double *den,
                       double sign, int n) {
  // y += sign * (num/den) * x
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  y[k] += sign * (num[0] / den[0]) * x[k];
}

__global__ void k_xpay(double *p, const double *r, const double *num, const double *den, int n) {
  // p = r + (num/den) p
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  p[k] = r[k] + (num[0] / den[0]) * p[k];
}

__global__ void k_update_params(double *p, const double *x, double dtau, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) p[k] += -dtau * x[k];
}

template <typename TO>
cudaError_t colreduce(const SrWork &w, const TO *O, int mode, const double *wvec, double wshift,
                      double scale, double *out, cudaStream_t st, long long *nl) {
  const int nparts = (w.rows + ROWCHUNK - 1) / ROWCHUNK;
  dim3 grid((w.Np + RB - 1) / RB, nparts);
  k_colreduce<TO><<<grid, RB, 0, st>>>(O, w.ldO, w.rows, w.Np, w.obar, wvec, wshift, mode, w.part);
  k_sum_parts<<<(w.Np + 255) / 256, 256, 0, st>>>(w.part, nparts, w.Np, scale, out);
  *nl += 2;
  return cudaGetLastError();
}

cudaError_t colreduce_any(const SrWork &w, int mode, const double *wvec, double wshift,
                          double scale, double *out, cudaStream_t st, long long *nl) {
  if (w.precision == 0)
    return colreduce<double>(w, (const double *)w.O, mode, wvec, wshift, scale, out, st, nl);
  return colreduce<float>(w, (const float *)w.O, mode, wvec, wshift, scale, out, st, nl);
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
  if (splits < 1) splits = 1;
  int rps = (w.rows + splits - 1) / splits;
  rps = (rps + SKK - 1) / SKK * SKK;
  splits = (w.rows + rps - 1) / rps;
  dim3 grid(ntiles, splits);
  if (w.precision == 0)
    k_syrk<double><<<grid, 256, 0, st>>>((const double *)w.O, w.ldO, w.rows, w.Np, w.obar,
                                         1.0 / w.rows, rps, w.S);
  else
    k_syrk<float><<<grid, 256, 0, st>>>((const float *)w.O, w.ldO, w.rows, w.Np, w.obar,
                                        1.0 / w.rows, rps, w.S);
  const size_t n2 = (size_t)w.Np * w.Np;
  k_mirror_shift<<<(unsigned)((n2 + 255) / 256), 256, 0, st>>>(w.S, w.Np, shift_rel, shift_abs);
  *nl += 2;
  return cudaGetLastError();
}

int vmc_sr_cholesky_solve(const SrWork &w, cudaStream_t st, long long *nl) {
  const int n = w.Np;
  cudaMemsetAsync(w.info, 0, sizeof(int), st);
  for (int j = 0; j < n; ++j) {
    const int rem = n - j - 1;
    k_chol_col<<<rem > 256 ? (rem + 255) / 256 : 1, 256, 0, st>>>(w.S, n, j, w.info);
    if (rem > 0) {
      const size_t tot = (size_t)rem * rem;
      const int g = (int)((tot + 255) / 256 < 8192 ? (tot + 255) / 256 : 8192);
      k_chol_update<<<g, 256, 0, st>>>(w.S, n, j);
      *nl += 1;
    }
    *nl += 1;
  }
  k_chol_solve<<<1, 256, sizeof(double) * n, st>>>(w.S, n, w.g, w.x);
  *nl += 1;
  if (cudaGetLastError() != cudaSuccess) return -3;
  int info = 0;
  if (cudaMemcpyAsync(&info, w.info, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return -3;
  if (cudaStreamSynchronize(st) != cudaSuccess) return -3;
  return info ? -4 : 0;
}

// One SR-CG product w = S~ v (Sec. 2.3.2): t = O v, u = O^T t / rows,
// w = u - o (o . v) + shift terms.
static cudaError_t srcg_matvec(const SrWork &w, const double *v, double *out, double shift_rel,
                               double shift_abs, cudaStream_t st, long long *nl) {
  const int threads = 256;
  const int blocks = (int)(((size_t)w.rows * 32 + threads - 1) / threads);
  if (w.precision == 0)
    k_gemv_rows<double><<<blocks, threads, 0, st>>>((const double *)w.O, w.ldO, w.rows, w.Np, v, w.t);
  else
    k_gemv_rows<float><<<blocks, threads, 0, st>>>((const float *)w.O, w.ldO, w.rows, w.Np, v, w.t);
  ++*nl;
  cudaError_t e = colreduce_any(w, 3, w.t, 0.0, 1.0 / w.rows, w.r + w.Np, st, nl);
  if (e) return e;
  k_dot<<<1, 256, 0, st>>>(w.obar, v, w.Np, w.scal + 4);
  k_cg_finish<<<(w.Np + 255) / 256, 256, 0, st>>>(w.r + w.Np, w.obar, w.scal + 4, w.diagS, v,
                                                   shift_rel, shift_abs, w.Np, out);
  *nl += 2;
  return cudaGetLastError();
}

// Algorithm 1 with x0 = 0.  Device scalars: scal[0] = rho, scal[1] = p.w,
// scal[2] = rho', scal[3] = |b|^2.  w.r holds 2*Np doubles (r and scratch).
int vmc_sr_cg_solve(const SrWork &w, double shift_rel, double shift_abs, double eps, int kmax,
                    int *iters, cudaStream_t st, long long *nl) {
  const int n = w.Np, g = (n + 255) / 256;
  cudaMemsetAsync(w.x, 0, sizeof(double) * n, st);
  cudaMemcpyAsync(w.r, w.g, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(w.p, w.g, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
  k_dot<<<1, 256, 0, st>>>(w.r, w.r, n, w.scal + 0);
  *nl += 1;
  double h[2];
  if (cudaMemcpyAsync(h, w.scal, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess) return -3;
  if (cudaStreamSynchronize(st) != cudaSuccess) return -3;
  const double thr = eps * eps * h[0];
  *iters = 0;
  if (h[0] == 0.0) return 0;
  for (int k = 1; k <= kmax; ++k) {
    if (srcg_matvec(w, w.p, w.w, shift_rel, shift_abs, st, nl) != cudaSuccess) return -3;
    k_dot<<<1, 256, 0, st>>>(w.p, w.w, n, w.scal + 1);
    k_axpy<<<g, 256, 0, st>>>(w.x, w.p, w.scal + 0, w.scal + 1, 1.0, n);
    k_axpy<<<g, 256, 0, st>>>(w.r, w.w, w.scal + 0, w.scal + 1, -1.0, n);
    k_dot<<<1, 256, 0, st>>>(w.r, w.r, n, w.scal + 2);
    *nl += 4;
    double rho[3];
    if (cudaMemcpyAsync(rho, w.scal, sizeof(double) * 3, cudaMemcpyDeviceToHost, st) != cudaSuccess) return -3;
    if (cudaStreamSynchronize(st) != cudaSuccess) return -3;
    *iters = k;
    if (!(rho[1] != 0.0) || !isfinite(rho[2])) return -5;
    if (rho[2] < thr) break;
    k_xpay<<<g, 256, 0, st>>>(w.p, w.r, w.scal + 2, w.scal + 0, n);
    cudaMemcpyAsync(w.scal, w.scal + 2, sizeof(double), cudaMemcpyDeviceToDevice, st);
    *nl += 1;
  }
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
