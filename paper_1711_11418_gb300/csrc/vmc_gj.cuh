// From-scratch inverse of one walker's M: FP64 Gauss-Jordan elimination with
// partial pivoting in shared memory (mVMC paper, Sec. 3.2.1: the Pfaffian of
// the anti-parallel pair product is det M up to a sign, Pf^2 = det X), with
// log|det M| and its sign.  Shared by the translation units of the walker
// kernels (the plain walker and the projected one).
#pragma once

#include "vmc_common.cuh"

namespace vmc_gj {

constexpr int NT = VMC_NT;
constexpr int NWARP = NT / 32;

// In place on an N x N row-major matrix (row stride lda) in shared or global
// memory; column-parallel elimination (coalesced, bank-conflict free).
struct GJShared {
  double val[NWARP];
  double amax[NWARP];
  int idx[NWARP];
  int piv;
  int bad;
  int sign;
  double logdet;
  double pmin, pmax;   // smallest / largest |pivot|
  double ipiv;
  double colk[VMC_MAX_N];   // pivot column of the current step (row k zeroed)
  double rowk[VMC_MAX_N];   // scaled pivot row of the current step (column k zeroed)
  double apiv[VMC_MAX_N];   // |pivot| of every step
  double pminw[NWARP];
};

__device__ __forceinline__ void gj_invert(double *A, int lda, int N, int *perm, GJShared &g) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    g.logdet = 0.0;
    g.sign = 1;
    g.bad = 0;
    g.pmin = 1e300;
    g.pmax = 0.0;
  }
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    // (1) copy column k and find the pivot among rows >= k
    double v = -1.0;
    int vi = N;
    for (int i = tid; i < N; i += NT) {
      const double a = A[(size_t)i * lda + k];
      g.colk[i] = a;
      if (i >= k && fabs(a) > v) {
        v = fabs(a);
        vi = i;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int oi = __shfl_xor_sync(0xffffffffu, vi, o);
      if (ov > v || (ov == v && oi < vi)) {
        v = ov;
        vi = oi;
      }
    }
    if ((tid & 31) == 0) {
      g.val[tid >> 5] = v;
      g.idx[tid >> 5] = vi;
    }
    __syncthreads();
    // (2) one thread: pivot row p, swap it into the pivot column copy, 1/pivot
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
      const double piv = g.colk[bi];
      g.colk[bi] = g.colk[k];
      g.colk[k] = 0.0;   // row k is scaled, not eliminated
      g.ipiv = 1.0 / piv;
      g.apiv[k] = fabs(piv);   // log|det| is summed after the elimination
      if ((piv < 0.0) != (bi != k)) g.sign = -g.sign;
    }
    __syncthreads();
    if (g.bad) return;
    const int p = g.piv;
    const double ipiv = g.ipiv;
    // (3a) the new column k, one row per thread (from the copy); for every
    // column c != k: swap rows k and p, scale row k, keep it in rowk.
    for (int i = tid; i < N; i += NT) A[(size_t)i * lda + k] = (i == k) ? ipiv : -g.colk[i] * ipiv;
    for (int c = tid; c < N; c += NT) {
      if (c == k) {
        g.rowk[c] = 0.0;   // column k is final: the update below leaves it
        continue;
      }
      double rkc = A[(size_t)p * lda + c];
      if (p != k) A[(size_t)p * lda + c] = A[(size_t)k * lda + c];
      rkc *= ipiv;
      A[(size_t)k * lda + c] = rkc;
      g.rowk[c] = rkc;
    }
    __syncthreads();
    // (3b) A_ic -= colk_i rowk_c over all N x N entries, spread flat over the
    // threads (whole warps for any N; colk_k = 0 leaves row k), four entries
    // in flight per thread.
    {
      const int qn = NT / N, rn = NT - (NT / N) * N;
      auto adv = [&](int &ii, int &cc) {
        ii += qn;
        cc += rn;
        if (cc >= N) {
          cc -= N;
          ++ii;
        }
      };
      int i = tid / N, c = tid - (tid / N) * N;
      while (i < N) {
        int i1 = i, c1 = c;
        adv(i1, c1);
        int i2 = i1, c2 = c1;
        adv(i2, c2);
        int i3 = i2, c3 = c2;
        adv(i3, c3);
        const bool b1 = i1 < N, b2 = i2 < N, b3 = i3 < N;
        double *q0 = A + (size_t)i * lda + c;
        double *q1 = A + (size_t)(b1 ? i1 : i) * lda + (b1 ? c1 : c);
        double *q2 = A + (size_t)(b2 ? i2 : i) * lda + (b2 ? c2 : c);
        double *q3 = A + (size_t)(b3 ? i3 : i) * lda + (b3 ? c3 : c);
        double a0 = *q0, a1 = *q1, a2 = *q2, a3 = *q3;
        a0 -= g.colk[i] * g.rowk[c];
        if (b1) a1 -= g.colk[i1] * g.rowk[c1];
        if (b2) a2 -= g.colk[i2] * g.rowk[c2];
        if (b3) a3 -= g.colk[i3] * g.rowk[c3];
        *q0 = a0;
        if (b1) *q1 = a1;
        if (b2) *q2 = a2;
        if (b3) *q3 = a3;
        i = i3;
        c = c3;
        adv(i, c);
      }
    }
    __syncthreads();
  }
  // log|det M| and the pivot range, off the elimination's serial path
  {
    double ls = 0.0, mn = 1e300, mx = 0.0;
    for (int i = tid; i < N; i += NT) {
      const double a = g.apiv[i];
      ls += log(a);
      mn = fmin(mn, a);
      mx = fmax(mx, a);
    }
    for (int o = 16; o > 0; o >>= 1) {
      ls += __shfl_xor_sync(0xffffffffu, ls, o);
      mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((tid & 31) == 0) {
      g.val[tid >> 5] = ls;
      g.pminw[tid >> 5] = mn;
      g.amax[tid >> 5] = mx;
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
  for (int k = N - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p == k) continue;   // uniform: perm is shared
    for (int r = tid; r < N; r += NT) {
      const double t0 = A[(size_t)r * lda + k];
      A[(size_t)r * lda + k] = A[(size_t)r * lda + p];
      A[(size_t)r * lda + p] = t0;
    }
    __syncthreads();
  }
  __syncthreads();
}

}  // namespace vmc_gj
