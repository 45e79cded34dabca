// SR solve S~ x = g (Sec. 3.3.2) by mixed-precision iterative refinement:
// the Jacobi-scaled matrix A = D S~ D (D = diag(S~_kk)^-1/2, unit diagonal)
// is inverted once in FP32 by blocked Gauss-Jordan elimination, and that
// inverse corrects an FP64 solution against FP64 residuals:
//   x_0 = 0,  r_i = g - S~ x_i  (FP64),  x_{i+1} = x_i + D A32^-1 D r_i,
// until |r| <= eps |g| (Wilkinson / Moler iterative refinement).  The
// result carries the FP64 residual of the direct solve; the O(Np^3) work is
// FP32 (this part's FP64 rate is 1/64 of its FP32 rate).  The caller falls
// back to the FP64 Cholesky when the refinement does not converge.
#include "vmc_common.cuh"

#include <math.h>

namespace {

constexpr int GB = 32;    // Gauss-Jordan block
constexpr int GT = 64;    // update tile (GT x GT outputs per CTA)

// d_k = S~_kk^-1/2 (S~_kk > 0 for a shifted overlap matrix; a non-positive
// entry marks the matrix as unusable: flag[1] = 1)
__global__ void k_ir_diag(const double *S, int n, double *dsc, int *flag) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double a = S[(size_t)k * n + k];
  if (!(a > 0.0) || !isfinite(a)) {
    flag[1] = 1;
    dsc[k] = 1.0;
  } else {
    dsc[k] = 1.0 / sqrt(a);
  }
}

__global__ void k_ir_scale(const double *S, int n, const double *dsc, float *A) {
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (size_t)n * n) return;
  const int i = (int)(q / n), j = (int)(q % n);
  A[q] = (float)(dsc[i] * S[q] * dsc[j]);
}

// In-place inverse of the nb x nb block D (padded with the identity to GB)
// by Gauss-Jordan elimination without pivoting (the scaled matrix is
// symmetric positive definite), 256 threads.
__device__ void block_invert(float (*D)[GB + 1], float *rowk, float *colk) {
  const int tid = threadIdx.x;
  for (int k = 0; k < GB; ++k) {
    if (tid < GB) {
      rowk[tid] = D[k][tid];
      colk[tid] = D[tid][k];
    }
    __syncthreads();
    const float ip = 1.0f / rowk[k];
    for (int q = tid; q < GB * GB; q += 256) {
      const int r = q / GB, c = q % GB;
      if (r == k && c == k) D[r][c] = ip;
      else if (r == k) D[r][c] = rowk[c] * ip;
      else if (c == k) D[r][c] = -colk[r] * ip;
      else D[r][c] -= colk[r] * rowk[c] * ip;
    }
    __syncthreads();
  }
}

// Gauss-Jordan step on pivot block K = [k0, k0 + nb): every CTA inverts A_KK
// into shared memory (CTA 0 stores it in P); CTA b then forms the new row
// block A_Kj <- P A_Kj for its columns j in [GT b, GT b + GT) \ K and copies
// the old column block C_i = A_iK for its rows i in the same range.
__global__ void __launch_bounds__(256) k_gj_row(float *A, int n, int k0, int nb, float *P, float *C) {
  __shared__ float D[GB][GB + 1];
  __shared__ float R[GB][GT + 1];
  __shared__ float rowk[GB], colk[GB];
  const int tid = threadIdx.x;
  for (int q = tid; q < GB * GB; q += 256) {
    const int r = q / GB, c = q % GB;
    D[r][c] = (r < nb && c < nb) ? A[(size_t)(k0 + r) * n + k0 + c] : (r == c ? 1.0f : 0.0f);
  }
  __syncthreads();
  block_invert(D, rowk, colk);
  if (blockIdx.x == 0)
    for (int q = tid; q < GB * GB; q += 256) P[q] = D[q / GB][q % GB];
  const int j0 = blockIdx.x * GT;
  for (int q = tid; q < GB * GT; q += 256) {
    const int l = q / GT, c = q % GT, j = j0 + c;
    R[l][c] = (l < nb && j < n) ? A[(size_t)(k0 + l) * n + j] : 0.0f;
  }
  __syncthreads();
  for (int q = tid; q < GB * GT; q += 256) {
    const int l = q / GT, c = q % GT, j = j0 + c;
    if (l >= nb || j >= n || (j >= k0 && j < k0 + nb)) continue;
    float s = 0.0f;
#pragma unroll 8
    for (int m = 0; m < GB; ++m) s += D[l][m] * R[m][c];
    A[(size_t)(k0 + l) * n + j] = s;
  }
  for (int q = tid; q < GT * GB; q += 256) {
    const int r = q / GB, l = q % GB, i = j0 + r;
    if (i >= n) continue;
    C[(size_t)i * GB + l] = (l < nb && !(i >= k0 && i < k0 + nb)) ? A[(size_t)i * n + k0 + l] : 0.0f;
  }
}

// Rest of the step, one GT x GT tile per CTA:
//   i, j not in K:  A_ij <- A_ij - sum_l C_il A_Kj,l   (row block already new)
//   i not in K, j in K:  A_iK <- -C_i P
//   i, j in K:  A_KK <- P
__global__ void __launch_bounds__(256) k_gj_update(float *A, int n, int k0, int nb, const float *P,
                                                   const float *C) {
  __shared__ float Cs[GT][GB + 1];
  __shared__ float Bs[GB][GT + 1];
  const int nt = (n + GT - 1) / GT;
  const int ti = blockIdx.x / nt, tj = blockIdx.x % nt;
  const int i0 = ti * GT, j0 = tj * GT, tid = threadIdx.x;
  auto inK = [&](int x) { return x >= k0 && x < k0 + nb; };
  for (int q = tid; q < GT * GB; q += 256) {
    const int r = q / GB, l = q % GB, i = i0 + r;
    Cs[r][l] = (i < n) ? C[(size_t)i * GB + l] : 0.0f;
  }
  for (int q = tid; q < GB * GT; q += 256) {
    const int l = q / GT, c = q % GT, j = j0 + c;
    float b = 0.0f;
    if (j < n && l < nb) b = inK(j) ? P[l * GB + (j - k0)] : A[(size_t)(k0 + l) * n + j];
    Bs[l][c] = b;
  }
  __syncthreads();
  const int tx = tid % 16, ty = tid / 16;
  float acc[4][4] = {};
#pragma unroll 8
  for (int l = 0; l < GB; ++l) {
    float a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a[u] = Cs[ty + 16 * u][l];
      b[u] = Bs[l][tx + 16 * u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
      if (i >= n || j >= n) continue;
      float *a = A + (size_t)i * n + j;
      if (inK(i)) {
        if (inK(j)) *a = P[(i - k0) * GB + (j - k0)];
      } else if (inK(j)) {
        *a = -acc[u][v];
      } else {
        *a -= acc[u][v];
      }
    }
}

// x = 0, r = g, rs = D g (FP32), scal[1] = |g|^2, flag[0] = 0, iters = 0
__global__ void k_ir_init(const double *g, int n, const double *dsc, double *x, double *r,
                          float *rs, double *scal, int *flag) {
  __shared__ double red[256];
  double s = 0.0;
  for (int k = threadIdx.x; k < n; k += 256) {
    const double v = g[k];
    x[k] = 0.0;
    r[k] = v;
    rs[k] = (float)(dsc[k] * v);
    s += v * v;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    scal[0] = 0.0;
    scal[1] = red[0];
    scal[2] = red[0];
    flag[0] = 0;
    flag[2] = 0;
  }
}

// x += D A32^-1 rs (one warp per row, FP32 products, FP64 update)
__global__ void k_ir_correct(const float *Ainv, int n, const double *dsc, const float *rs,
                             double *x, const int *flag) {
  if (flag[0] | flag[1]) return;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (row >= n) return;
  const float *a = Ainv + (size_t)row * n;
  float s0 = 0.0f, s1 = 0.0f;
  int j = lane;
  for (; j + 32 < n; j += 64) {
    s0 += a[j] * rs[j];
    s1 += a[j + 32] * rs[j + 32];
  }
  if (j < n) s0 += a[j] * rs[j];
  float s = s0 + s1;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) x[row] += dsc[row] * (double)s;
}

// r = g - S~ x (FP64, one warp per row); rs = D r in FP32; scal[0] += |r|^2
__global__ void k_ir_residual(const double *S, int n, const double *g, const double *x,
                              const double *dsc, double *r, float *rs, double *scal,
                              const int *flag) {
  if (flag[0] | flag[1]) return;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (row >= n) return;
  const double *a = S + (size_t)row * n;
  double s0 = 0.0, s1 = 0.0;
  int j = lane;
  for (; j + 32 < n; j += 64) {
    s0 += a[j] * x[j];
    s1 += a[j + 32] * x[j + 32];
  }
  if (j < n) s0 += a[j] * x[j];
  double s = s0 + s1;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    const double v = g[row] - s;
    r[row] = v;
    rs[row] = (float)(dsc[row] * v);
    atomicAdd(scal, v * v);
  }
}

// convergence: |r|^2 <= eps^2 |g|^2 -> flag[0] = 1; scal[2] keeps the last |r|^2
__global__ void k_ir_check(double *scal, int *flag, double eps2) {
  if (flag[0] | flag[1]) return;
  const double rr = scal[0];
  scal[0] = 0.0;
  scal[2] = rr;
  flag[2] += 1;
  if (!(rr <= eps2 * scal[1])) return;
  flag[0] = 1;
}

void ir_sequence(const SrWork &w, int max_iter, double eps, cudaStream_t st) {
  const int n = w.Np;
  cudaMemsetAsync(w.irflag, 0, sizeof(int) * 4, st);
  k_ir_diag<<<(n + 255) / 256, 256, 0, st>>>(w.S, n, w.dsc, w.irflag);
  const size_t n2 = (size_t)n * n;
  k_ir_scale<<<(unsigned)((n2 + 255) / 256), 256, 0, st>>>(w.S, n, w.dsc, w.S32);
  const int nt = (n + GT - 1) / GT;
  for (int k0 = 0; k0 < n; k0 += GB) {
    const int nb = n - k0 < GB ? n - k0 : GB;
    k_gj_row<<<nt, 256, 0, st>>>(w.S32, n, k0, nb, w.gjP, w.gjC);
    k_gj_update<<<nt * nt, 256, 0, st>>>(w.S32, n, k0, nb, w.gjP, w.gjC);
  }
  k_ir_init<<<1, 256, 0, st>>>(w.g, n, w.dsc, w.x, w.r, w.rs32, w.scal, w.irflag);
  const int wb = (int)(((size_t)n * 32 + 255) / 256);
  for (int it = 0; it < max_iter; ++it) {
    k_ir_correct<<<wb, 256, 0, st>>>(w.S32, n, w.dsc, w.rs32, w.x, w.irflag);
    k_ir_residual<<<wb, 256, 0, st>>>(w.S, n, w.g, w.x, w.dsc, w.r, w.rs32, w.scal, w.irflag);
    k_ir_check<<<1, 1, 0, st>>>(w.scal, w.irflag, eps * eps);
  }
}

}  // namespace

long long vmc_sr_ir_launches(int n, int max_iter) {
  return 3 + 2LL * ((n + GB - 1) / GB) + 3LL * max_iter;
}

// Launch the refinement (the captured graph, made on first use).  Returns 0
// or -3 on a CUDA error.
int vmc_sr_ir_launch(SrWork &w, int max_iter, double eps, cudaStream_t st, long long *nl) {
  if (!w.ir_graph || w.ir_iter != max_iter || w.ir_eps != eps) {
    if (w.ir_graph) cudaGraphExecDestroy((cudaGraphExec_t)w.ir_graph);
    w.ir_graph = nullptr;
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return -3;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      ir_sequence(w, max_iter, eps, cs);
      ok = cudaStreamEndCapture(cs, &g) == cudaSuccess && g;
    }
    if (ok) ok = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (!ok) {
      cudaGetLastError();
      return -3;
    }
    w.ir_graph = (void *)ge;
    w.ir_iter = max_iter;
    w.ir_eps = eps;
  }
  if (cudaGraphLaunch((cudaGraphExec_t)w.ir_graph, st) != cudaSuccess) return -3;
  *nl += vmc_sr_ir_launches(w.Np, max_iter);
  return 0;
}

// Enqueue the copies of the refinement's flags (4 ints) and scalars (3
// doubles) to host memory; evaluate them after the stream has synchronised.
int vmc_sr_ir_fetch(const SrWork &w, int *flags4, double *scal3, cudaStream_t st) {
  if (cudaMemcpyAsync(flags4, w.irflag, sizeof(int) * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return -3;
  if (cudaMemcpyAsync(scal3, w.scal, sizeof(double) * 3, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return -3;
  return 0;
}

// 0: converged (*iters refinement steps, *rel_res = |r| / |g|); 1: not
// converged or S~ unusable (the caller solves by FP64 Cholesky).
int vmc_sr_ir_eval(const int *fl, const double *sc, int *iters, double *rel_res) {
  *iters = fl[2];
  *rel_res = sc[1] > 0.0 ? sqrt(sc[2] / sc[1]) : 0.0;
  return (fl[0] && !fl[1]) ? 0 : 1;
}

// Returns 0 (converged; *iters = refinement steps), 1 (not converged or S~
// unusable: the caller solves by FP64 Cholesky), or -3 on a CUDA error.
int vmc_sr_ir_solve(SrWork &w, int max_iter, double eps, int *iters, double *rel_res,
                    cudaStream_t st, long long *nl) {
  if (vmc_sr_ir_launch(w, max_iter, eps, st, nl)) return -3;
  int fl[4] = {0, 0, 0, 0};
  double sc[3] = {0, 0, 0};
  if (vmc_sr_ir_fetch(w, fl, sc, st)) return -3;
  if (cudaStreamSynchronize(st) != cudaSuccess) return -3;
  return vmc_sr_ir_eval(fl, sc, iters, rel_res);
}

void vmc_sr_ir_release(SrWork &w) {
  if (w.ir_graph) cudaGraphExecDestroy((cudaGraphExec_t)w.ir_graph);
  w.ir_graph = nullptr;
}
