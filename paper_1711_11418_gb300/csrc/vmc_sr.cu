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
constexpr int RMIN = 64;       // fewest rows per partial of a column reduction

}  // namespace

// Row chunks of a column reduction: enough CTAs to cover the SMs several
// times over, at least RMIN rows each.  Monotone in rows, so the partial
// buffer sized for the largest row count serves every smaller one.
int vmc_colreduce_parts(int rows, int Np) {
  const int ctiles = (Np + RB - 1) / RB;
  int target = (8 * 152 + ctiles - 1) / ctiles;
  const int most = (rows + RMIN - 1) / RMIN;
  if (target > most) target = most;
  return target < 1 ? 1 : target;
}

namespace {

template <typename TO>
__device__ __forceinline__ double ld(const TO *p) { return (double)*p; }

// Partial column reductions: part[c][k] = sum over the rows of chunk c of
//   mode 0: O_rk                      (mean)
//   mode 1: (O_rk - o_k) (E_r - ebar)  (force g)
//   mode 2: (O_rk - o_k)^2             (diagonal of S)
//   mode 3: O_rk t_r                   (CG: O^T t)
// One thread per column, rows unrolled by 4 for independent loads.
template <typename TO>
__global__ void __launch_bounds__(RB) k_colreduce(const TO *O, int ldO, int rows, int Np,
                                                  const double *obar, const double *wvec,
                                                  double wshift_h, const double *wshift_d,
                                                  int mode, int chunk, double *part,
                                                  const int *done) {
  const int k = blockIdx.x * RB + threadIdx.x;
  const int c = blockIdx.y;
  if (k >= Np || (done && *done)) return;
  const int r0 = c * chunk;
  const int r1 = min(rows, r0 + chunk);
  const double ok = (mode == 1 || mode == 2) ? obar[k] : 0.0;
  const double wshift = wshift_d ? *wshift_d : wshift_h;
  const TO *col = O + k;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int r = r0;
  for (; r + 4 <= r1; r += 4) {
    const double o0 = ld(col + (size_t)r * ldO), o1 = ld(col + (size_t)(r + 1) * ldO);
    const double o2 = ld(col + (size_t)(r + 2) * ldO), o3 = ld(col + (size_t)(r + 3) * ldO);
    switch (mode) {
      case 0: s0 += o0; s1 += o1; s2 += o2; s3 += o3; break;
      case 1:
        s0 += (o0 - ok) * (wvec[r] - wshift);
        s1 += (o1 - ok) * (wvec[r + 1] - wshift);
        s2 += (o2 - ok) * (wvec[r + 2] - wshift);
        s3 += (o3 - ok) * (wvec[r + 3] - wshift);
        break;
      case 2:
        s0 += (o0 - ok) * (o0 - ok); s1 += (o1 - ok) * (o1 - ok);
        s2 += (o2 - ok) * (o2 - ok); s3 += (o3 - ok) * (o3 - ok);
        break;
      default:
        s0 += o0 * wvec[r]; s1 += o1 * wvec[r + 1]; s2 += o2 * wvec[r + 2]; s3 += o3 * wvec[r + 3];
        break;
    }
  }
  for (; r < r1; ++r) {
    const double o = ld(col + (size_t)r * ldO);
    switch (mode) {
      case 0: s0 += o; break;
      case 1: s0 += (o - ok) * (wvec[r] - wshift); break;
      case 2: s0 += (o - ok) * (o - ok); break;
      default: s0 += o * wvec[r]; break;
    }
  }
  part[(size_t)c * Np + k] = (s0 + s1) + (s2 + s3);
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
// columns.  Per panel: k_chol_panel factors the diagonal block and solves the
// panel below it (L_ij = A_ij L_jj^-T); k_syrk_trailing updates the trailing
// lower triangle (A -= L L^T) in 32x32 tiles.  FP64 throughput per SM is low
// on this part, so small tiles keep every SM busy on the late panels.
constexpr int CB = 32;

// Cholesky of the nb x nb diagonal block D (lower part, shared memory) by one
// warp: right-looking, column k scaled by 1/L_kk, then the packed triangle
// {(r, c): k < c <= r < nb} updated with one entry per lane (the triangle is
// walked by a linear index, so no lane idles on masked entries).  invd[k]
// receives 1/L_kk; returns the first non-positive pivot (1-based) or 0.
__device__ int warp_potrf(double (*D)[CB + 1], double *invd, int nb) {
  const int lane = threadIdx.x & 31;
  int bad = 0;
  for (int k = 0; k < nb; ++k) {
    if (lane == 0) {
      double a = D[k][k];
      if (!(a > 0.0) || !isfinite(a)) {
        if (!bad) bad = k + 1;
        a = 1.0;
      }
      const double d = sqrt(a);
      D[k][k] = d;
      invd[k] = 1.0 / d;
    }
    __syncwarp();
    const double iv = invd[k];
    if (lane > k && lane < nb) D[lane][k] *= iv;
    __syncwarp();
    const int m = nb - k - 1;
    const int T = m * (m + 1) / 2;
    for (int q = lane; q < T; q += 32) {
      int i = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
      while (i * (i + 1) / 2 > q) --i;
      while ((i + 1) * (i + 2) / 2 <= q) ++i;
      const int r = k + 1 + i, c = k + 1 + (q - i * (i + 1) / 2);
      D[r][c] -= D[r][k] * D[c][k];
    }
    __syncwarp();
  }
  return __shfl_sync(0xffffffffu, bad, 0);
}

// Panel step: every CTA (one warp) factors the diagonal block in shared
// memory and solves CB rows of the panel below it, X_i = A_i L_jj^-T, by
// forward substitution with one row per lane (X_ic = (A_ic - sum_{l<c} X_il
// L_cl) / L_cc).  CTA 0 records the first non-positive pivot in *info
// (1-based) and stores the factored block: straight into A when it is the
// only CTA, else into dblk, from where the trailing update copies it (another
// CTA may still be reading the block).
__global__ void __launch_bounds__(32) k_chol_panel(double *A, int n, int j0, int nb, int *info,
                                                   double *dblk) {
  __shared__ double D[CB][CB + 1];
  __shared__ double invd[CB];
  const int lane = threadIdx.x;
  for (int r = 0; r < CB; ++r)
    D[r][lane] = (r < nb && lane <= r) ? A[(size_t)(j0 + r) * n + j0 + lane] : (r == lane ? 1.0 : 0.0);
  __syncwarp();
  const int bad = warp_potrf(D, invd, nb);
  if (blockIdx.x == 0) {
    const bool direct = gridDim.x == 1;
    for (int r = 0; r < nb; ++r) {
      if (lane > r) continue;
      if (direct) A[(size_t)(j0 + r) * n + j0 + lane] = D[r][lane];
      else dblk[r * nb + lane] = D[r][lane];
    }
    if (lane == 0 && bad && *info == 0) *info = j0 + bad;
  }
  const int i = j0 + nb + blockIdx.x * CB + lane;
  if (i >= n) return;
  double *row = A + (size_t)i * n + j0;
  double x[CB];
#pragma unroll
  for (int c = 0; c < CB; ++c) x[c] = (c < nb) ? row[c] : 0.0;
#pragma unroll
  for (int c = 0; c < CB; ++c) {
    if (c < nb) {
      double v = x[c];
#pragma unroll
      for (int l = 0; l < c; ++l) v -= x[l] * D[c][l];
      x[c] = v * invd[c];
    }
  }
#pragma unroll
  for (int c = 0; c < CB; ++c)
    if (c < nb) row[c] = x[c];
}

// Trailing update A[i][k] -= sum_l L[i][j0+l] L[k][j0+l] for j1 <= k <= i < n
// (j1 = j0 + nb): one 32x32 lower tile per CTA, tile (bi, bj) with bj <= bi
// decoded from the linear block index.  With copy_diag, CTA 0 also stores
// the factored diagonal block from dblk (no CTA here reads that block).
__global__ void __launch_bounds__(256) k_syrk_trailing(double *A, int n, int j0, int nb,
                                                       int copy_diag, const double *dblk) {
  const int j1 = j0 + nb;
  if (copy_diag && blockIdx.x == 0)
    for (int q = threadIdx.x; q < nb * nb; q += 256) {
      const int r = q / nb, c = q % nb;
      if (c <= r) A[(size_t)(j0 + r) * n + j0 + c] = dblk[q];
    }
  int t = blockIdx.x, bi = 0;
  while (t >= bi + 1) {
    t -= bi + 1;
    ++bi;
  }
  const int bj = t;
  __shared__ double Pi[CB][33];
  __shared__ double Pk[CB][33];
  for (int q = threadIdx.x; q < CB * 32; q += 256) {
    const int r = q / CB, l = q % CB;
    const int ii = j1 + bi * 32 + r, kk = j1 + bj * 32 + r;
    Pi[l][r] = (l < nb && ii < n) ? A[(size_t)ii * n + j0 + l] : 0.0;
    Pk[l][r] = (l < nb && kk < n) ? A[(size_t)kk * n + j0 + l] : 0.0;
  }
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double a00 = 0, a01 = 0, a10 = 0, a11 = 0;
#pragma unroll 8
  for (int l = 0; l < CB; ++l) {
    const double x0 = Pi[l][ty], x1 = Pi[l][ty + 16];
    const double y0 = Pk[l][tx], y1 = Pk[l][tx + 16];
    a00 += x0 * y0; a01 += x0 * y1; a10 += x1 * y0; a11 += x1 * y1;
  }
  const double acc[2][2] = {{a00, a01}, {a10, a11}};
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int i = j1 + bi * 32 + ty + 16 * u, k = j1 + bj * 32 + tx + 16 * v;
      if (i < n && k < n && k <= i) A[(size_t)i * n + k] -= acc[u][v];
    }
}

// Triangular solves L y = b and L^T x = y, one launch per panel of CB
// unknowns and direction.  Every CTA stages the panel's diagonal block and
// solves it redundantly with one unknown per lane (column sweep: lane k
// finishes its unknown and broadcasts it, the others subtract), then applies
// the panel to its share of the remaining entries.  The right-hand side is
// read from one vector and the finished panel written to another, so no CTA
// reads a value another CTA of the same launch writes.
//   forward:  rows i >= p0 + nb: y_i -= sum_l L_{i,p0+l} z_{p0+l}   (warp per row);
//             CTA 0 writes z[p0 .. p0+nb).
//   backward: rows i < p0:       y_i -= sum_l L_{p0+l,i} x_{p0+l}   (thread per row);
//             CTA 0 writes x[p0 .. p0+nb).
constexpr int SV_ROWS = 64;    // forward rows per CTA (8 warps x 8 rows)
constexpr int SV_COLS = 256;   // backward rows per CTA (one per thread)

__device__ __forceinline__ double panel_solve_lane(const double (*Dg)[CB + 1], double v, int nb,
                                                   bool transpose) {
  const int lane = threadIdx.x & 31;
  if (!transpose) {
    for (int k = 0; k < nb; ++k) {
      if (lane == k) v /= Dg[k][k];
      const double xk = __shfl_sync(0xffffffffu, v, k);
      if (lane > k) v -= Dg[lane][k] * xk;
    }
  } else {
    for (int k = nb - 1; k >= 0; --k) {
      if (lane == k) v /= Dg[k][k];
      const double xk = __shfl_sync(0xffffffffu, v, k);
      if (lane < k) v -= Dg[k][lane] * xk;
    }
  }
  return v;
}

__global__ void __launch_bounds__(256) k_trsv_panel(const double *L, int n, int p0, int fwd,
                                                    double *y, double *out) {
  __shared__ double Dg[CB][CB + 1];
  __shared__ double xp[CB];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = min(CB, n - p0);
  for (int q = tid; q < CB * CB; q += 256) {
    const int r = q / CB, c = q % CB;
    Dg[r][c] = (r < nb && c <= r) ? L[(size_t)(p0 + r) * n + p0 + c] : (r == c ? 1.0 : 0.0);
  }
  __syncthreads();
  if (warp == 0) {
    double v = lane < nb ? y[p0 + lane] : 0.0;
    v = panel_solve_lane(Dg, v, nb, !fwd);
    xp[lane] = lane < nb ? v : 0.0;
    if (blockIdx.x == 0 && lane < nb) out[p0 + lane] = v;
  }
  __syncthreads();
  if (fwd) {
    const int r0 = p0 + nb + blockIdx.x * SV_ROWS;
    for (int i = r0 + warp; i < min(n, r0 + SV_ROWS); i += 8) {
      double s = (lane < nb) ? L[(size_t)i * n + p0 + lane] * xp[lane] : 0.0;
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) y[i] -= s;
    }
  } else {
    const int i = blockIdx.x * SV_COLS + tid;
    if (i < p0) {
      double s0 = 0.0, s1 = 0.0;
      int l = 0;
      for (; l + 2 <= nb; l += 2) {
        s0 += L[(size_t)(p0 + l) * n + i] * xp[l];
        s1 += L[(size_t)(p0 + l + 1) * n + i] * xp[l + 1];
      }
      if (l < nb) s0 += L[(size_t)(p0 + l) * n + i] * xp[l];
      y[i] -= s0 + s1;
    }
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
                      const int *done = nullptr, const double *wshift_d = nullptr) {
  const int nparts = vmc_colreduce_parts(w.rows, w.Np);
  const int chunk = (w.rows + nparts - 1) / nparts;
  dim3 grid((w.Np + RB - 1) / RB, nparts);
  k_colreduce<TO><<<grid, RB, 0, st>>>(O, w.ldO, w.rows, w.Np, w.obar, wvec, wshift, wshift_d, mode,
                                       chunk, w.part, done);
  k_sum_parts<<<(w.Np + 255) / 256, 256, 0, st>>>(w.part, nparts, w.Np, scale, out, done);
  *nl += 2;
  return cudaGetLastError();
}

cudaError_t colreduce_any(const SrWork &w, int mode, const double *wvec, double wshift,
                          double scale, double *out, cudaStream_t st, long long *nl,
                          const int *done = nullptr, const double *wshift_d = nullptr) {
  if (w.precision == 0)
    return colreduce<double>(w, (const double *)w.O, mode, wvec, wshift, scale, out, st, nl, done,
                             wshift_d);
  return colreduce<float>(w, (const float *)w.O, mode, wvec, wshift, scale, out, st, nl, done,
                          wshift_d);
}

}  // namespace

cudaError_t vmc_sr_means(const SrWork &w, cudaStream_t st, long long *nl) {
  k_mean_vec<<<1, 256, 0, st>>>(w.E, w.rows, w.ebar);
  ++*nl;
  return colreduce_any(w, 0, nullptr, 0.0, 1.0 / w.rows, w.obar, st, nl);
}

cudaError_t vmc_sr_build_g(const SrWork &w, cudaStream_t st, long long *nl) {
  // E - ebar with ebar read by the kernel from device memory (no host round trip)
  return colreduce_any(w, 1, w.E, 0.0, 1.0 / w.rows, w.g, st, nl, nullptr, w.ebar);
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

// The launch sequence of the factorisation and both solves: 2 launches per
// panel plus the solve.  Pointers are fixed for the life of the work area, so
// the sequence is captured once into a CUDA graph and replayed.
static void chol_sequence(const SrWork &w, cudaStream_t st) {
  const int n = w.Np;
  cudaMemsetAsync(w.info, 0, sizeof(int), st);
  for (int j0 = 0; j0 < n; j0 += CB) {
    const int nb = n - j0 < CB ? n - j0 : CB;
    const int rem = n - j0 - nb;
    const int pg = rem > 0 ? (rem + CB - 1) / CB : 1;
    k_chol_panel<<<pg, 32, 0, st>>>(w.S, n, j0, nb, w.info, w.dblk);
    if (rem > 0) {
      const int nt = (rem + 31) / 32;
      k_syrk_trailing<<<nt * (nt + 1) / 2, 256, 0, st>>>(w.S, n, j0, nb, pg > 1, w.dblk);
    }
  }
  // forward: y (= w.p, starts as g) -> z (= w.w); backward: z -> x.
  cudaMemcpyAsync(w.p, w.g, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
  for (int p0 = 0; p0 < n; p0 += CB) {
    const int rem = n - p0 - (n - p0 < CB ? n - p0 : CB);
    const int grid = rem > 0 ? (rem + SV_ROWS - 1) / SV_ROWS : 1;
    k_trsv_panel<<<grid, 256, 0, st>>>(w.S, n, p0, 1, w.p, w.w);
  }
  for (int p0 = ((n - 1) / CB) * CB; p0 >= 0; p0 -= CB) {
    const int grid = p0 > 0 ? (p0 + SV_COLS - 1) / SV_COLS : 1;
    k_trsv_panel<<<grid, 256, 0, st>>>(w.S, n, p0, 0, w.w, w.x);
  }
}

static long long chol_launches(int n) {
  long long c = 0;
  for (int j0 = 0; j0 < n; j0 += CB) c += (n - j0 > CB) ? 4 : 3;
  return c;
}

int vmc_sr_cholesky_launch(SrWork &w, cudaStream_t st, long long *nl) {
  if (!w.chol_graph) {
    // Capture on a private stream (the caller's may be the legacy stream,
    // which cannot be captured).
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return -3;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      chol_sequence(w, cs);
      ok = cudaStreamEndCapture(cs, &g) == cudaSuccess && g;
    }
    if (ok) ok = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (!ok) {
      cudaGetLastError();
      return -3;
    }
    w.chol_graph = (void *)ge;
  }
  if (cudaGraphLaunch((cudaGraphExec_t)w.chol_graph, st) != cudaSuccess) return -3;
  *nl += chol_launches(w.Np);
  return 0;
}

// Factor and solve; returns 0, -4 (S~ not positive definite) or -3.
int vmc_sr_cholesky_solve(SrWork &w, cudaStream_t st, long long *nl) {
  if (vmc_sr_cholesky_launch(w, st, nl)) return -3;
  int info = 0;
  if (cudaMemcpyAsync(&info, w.info, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return -3;
  if (cudaStreamSynchronize(st) != cudaSuccess) return -3;
  return info ? -4 : 0;
}

void vmc_sr_release(SrWork &w) {
  if (w.chol_graph) cudaGraphExecDestroy((cudaGraphExec_t)w.chol_graph);
  w.chol_graph = nullptr;
}

// Mixed form (FP32 O): the two passes of the SR-CG product with FP32
// products summed in FP32 over 16 terms and the partial sums in FP64, so the
// FP64 pipe (1/64 of the FP32 rate on this part) does one add per 16
// products; relative error of each product sum about 1e-6 at most.  The
// operand vectors enter as FP32 copies.
constexpr int CH32 = 16;

__global__ void k_to_float(const double *v, int n, float *vf, const int *done) {
  if (done && *done) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) vf[k] = (float)v[k];
}

// t = O v, one warp per row; t in FP64 and as an FP32 copy
__global__ void k_gemv_rows_f32(const float *O, int ldO, int rows, int Np, const float *vf,
                                double *t, float *tf, const int *done) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= rows || *done) return;
  const float *o = O + (size_t)warp * ldO;
  double s = 0.0;
  for (int k0 = lane; k0 < Np; k0 += 32 * CH32) {
    float a = 0.0f;
#pragma unroll
    for (int u = 0; u < CH32; ++u) {
      const int k = k0 + 32 * u;
      if (k < Np) a = fmaf(o[k], vf[k], a);
    }
    s += (double)a;
  }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) {
    t[warp] = s;
    tf[warp] = (float)s;
  }
}

// part[c][k] = sum over the rows of chunk c of O_rk t_r (thread per column)
__global__ void __launch_bounds__(RB) k_colreduce_t32(const float *O, int ldO, int rows, int Np,
                                                      const float *tf, int chunk, double *part,
                                                      const int *done) {
  const int k = blockIdx.x * RB + threadIdx.x;
  const int c = blockIdx.y;
  if (k >= Np || (done && *done)) return;
  const int r1 = min(rows, c * chunk + chunk);
  const float *col = O + k;
  double s = 0.0;
  for (int r = c * chunk; r < r1; r += CH32) {
    float a = 0.0f;
#pragma unroll
    for (int u = 0; u < CH32; ++u)
      if (r + u < r1) a = fmaf(col[(size_t)(r + u) * ldO], tf[r + u], a);
    s += (double)a;
  }
  part[(size_t)c * Np + k] = s;
}

// Dot products over many CTAs, summed in a fixed order (deterministic):
// dpart[b] = partial of CTA b; out = sum of the partials.
constexpr int DOT_MAXB = 512;

__global__ void k_dotp(const double *a, const double *b, int n, double *dpart, const int *done) {
  __shared__ double red[256];
  if (done && *done) return;
  double s = 0.0;
  for (int i = blockIdx.x * 256 + threadIdx.x; i < n; i += gridDim.x * 256) s += a[i] * b[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) dpart[blockIdx.x] = red[0];
}

__global__ void k_dotf(const double *dpart, int nb, double *out, const int *done) {
  __shared__ double red[256];
  if (done && *done) return;
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += 256) s += dpart[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

static int dot_blocks(int n) {
  const int nb = (n + 4095) / 4096;
  return nb < 1 ? 1 : (nb > DOT_MAXB ? DOT_MAXB : nb);
}

static void dot2(const double *a, const double *b, int n, double *out, double *dpart,
                 const int *done, cudaStream_t st, long long *nl) {
  const int nb = dot_blocks(n);
  k_dotp<<<nb, 256, 0, st>>>(a, b, n, dpart, done);
  k_dotf<<<1, 256, 0, st>>>(dpart, nb, out, done);
  *nl += 2;
}

// convergence test on rho' = r.r (computed by dot2): done if rho' < threshold
__global__ void k_cg_check2(const double *rho_new, const double *thr, int *flags) {
  if (flags[0]) return;
  const double v = rho_new[0];
  flags[1] += 1;
  if (!(v >= thr[0])) flags[0] = 1;   // converged (or NaN: flagged below)
  if (!isfinite(v)) flags[2] = 1;
}

// One SR-CG product out = S~ v (Sec. 3.3.2): t = O v, u = O^T t / rows,
// out = u - o (o . v) + shift terms.  2 (rows + 1) Np products for the S part.
static cudaError_t srcg_matvec(const SrWork &w, const double *v, double *out, double shift_rel,
                               double shift_abs, const int *done, cudaStream_t st, long long *nl) {
  const int threads = 256;
  const int blocks = (int)(((size_t)w.rows * 32 + threads - 1) / threads);
  if (w.precision == 0) {
    k_gemv_rows<double><<<blocks, threads, 0, st>>>((const double *)w.O, w.ldO, w.rows, w.Np, v, w.t, done);
    ++*nl;
    cudaError_t e = colreduce_any(w, 3, w.t, 0.0, 1.0 / w.rows, w.r + w.Np, st, nl, done);
    if (e) return e;
  } else {
    k_to_float<<<(w.Np + 255) / 256, 256, 0, st>>>(v, w.Np, w.vf, done);
    k_gemv_rows_f32<<<blocks, threads, 0, st>>>((const float *)w.O, w.ldO, w.rows, w.Np, w.vf,
                                                w.t, w.tf, done);
    const int nparts = vmc_colreduce_parts(w.rows, w.Np);
    const int chunk = (w.rows + nparts - 1) / nparts;
    dim3 grid((w.Np + RB - 1) / RB, nparts);
    k_colreduce_t32<<<grid, RB, 0, st>>>((const float *)w.O, w.ldO, w.rows, w.Np, w.tf, chunk,
                                         w.part, done);
    k_sum_parts<<<(w.Np + 255) / 256, 256, 0, st>>>(w.part, nparts, w.Np, 1.0 / w.rows,
                                                    w.r + w.Np, done);
    *nl += 4;
  }
  dot2(w.obar, v, w.Np, w.scal + 3, w.dpart, done, st, nl);
  k_cg_finish<<<(w.Np + 255) / 256, 256, 0, st>>>(w.r + w.Np, w.obar, w.scal + 3, w.diagS, v,
                                                   shift_rel, shift_abs, w.Np, out, done);
  *nl += 1;
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
  dot2(w.r, w.r, n, cg + 0, w.dpart, nullptr, st, nl);
  k_cg_init<<<1, 1, 0, st>>>(cg, flags, eps);
  *nl += 1;
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
    dot2(w.p, w.w, n, cg + 2, w.dpart, flags, st, nl);
    k_cg_update_xr<<<g, 256, 0, st>>>(w.x, w.r, w.p, w.w, rho, cg + 2, n, flags);
    dot2(w.r, w.r, n, rho_new, w.dpart, flags, st, nl);
    k_cg_check2<<<1, 1, 0, st>>>(rho_new, cg + 4, flags);
    k_cg_update_p<<<g, 256, 0, st>>>(w.p, w.r, rho_new, rho, n, flags);
    *nl += 3;
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

cudaError_t vmc_dot_dev(const double *a, const double *b, int n, double *out_dev, double *dpart,
                        cudaStream_t st, long long *nl) {
  dot2(a, b, n, out_dev, dpart, nullptr, st, nl);
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
