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
// memory.  Two barriers per elimination step:
//   (P, B) two warps take the pivot of column k from the per-warp
//       candidates (largest |a|, ties: lowest row) and form 1/pivot; one
//       forms the multipliers m_i = a_ik / pivot (pivot row swapped in,
//       m_k = 0, kept negated so the update is one FMA), the other the raw
//       pivot row, swapping rows k and p and scaling row k;
//   (E) a_ic -= m_i r_c over all entries, spread flat over the threads in
//       whole warps; before it, each thread forms the updated value of its
//       row of column k+1 once more (one FMA, from a copy of the column taken
//       in (B)) for the next step's pivot candidates, reduced per warp by
//       integer compares of |a|'s bit patterns, so the next pivot search
//       needs no barrier of its own.
// Entries of the rank-1 update in flight per thread.
constexpr int GJ_ILP = 4;

struct GJShared {
  double val[NWARP];
  double amax[NWARP];
  unsigned long long ckey[2][NWARP];   // per-warp pivot candidates (|a| bits) ...
  int cidx[2][NWARP];                  // ... and their rows, double-buffered by step
  int bad;
  int sign;
  double logdet;
  double pmin, pmax;   // smallest / largest |pivot|
  double ipiv;         // 1 / pivot of the current step
  double colk[VMC_MAX_N];   // negated multipliers -m_i of the current step (m_k = 0)
  double rowk[VMC_MAX_N];   // raw pivot row of the current step
  double coln[VMC_MAX_N];   // column k+1 before the current step's update
  double apiv[VMC_MAX_N];   // |pivot| of every step
  double pminw[NWARP];
};

// |a| as an ordered integer key; NaN below every number (never a pivot)
__device__ __forceinline__ unsigned long long pivot_key(double a) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(a) & 0x7FFFFFFFFFFFFFFFull;
  return b > 0x7FF0000000000000ull ? 0ull : b + 1ull;
}

// warp-wide largest key (ties: lowest row); lane 0 records it in slot buf
__device__ __forceinline__ void pivot_candidates(unsigned long long key, int row, GJShared &g,
                                                 int buf) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, o);
    const int orow = __shfl_xor_sync(0xffffffffu, row, o);
    if (ok > key || (ok == key && orow < row)) {
      key = ok;
      row = orow;
    }
  }
  if ((threadIdx.x & 31) == 0) {
    g.ckey[buf][threadIdx.x >> 5] = key;
    g.cidx[buf][threadIdx.x >> 5] = row;
  }
}

__device__ __forceinline__ void gj_invert(double *A, int lda, int N, int *perm, GJShared &g) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    g.logdet = 0.0;
    g.sign = 1;
    g.bad = 0;
    g.pmin = 1e300;
    g.pmax = 0.0;
  }
  // candidates of column 0
  {
    unsigned long long key = 0ull;
    int row = N;
    for (int i = tid; i < N; i += NT) {
      const unsigned long long kk = pivot_key(A[(size_t)i * lda]);
      if (kk > key) {
        key = kk;
        row = i;
      }
    }
    pivot_candidates(key, row, g, 0);
  }
  __syncthreads();
  const int qn = NT / N, rn = NT - (NT / N) * N;
  auto adv = [&](int &ii, int &cc) {
    ii += qn;
    cc += rn;
    if (cc >= N) {
      cc -= N;
      ++ii;
    }
  };
  for (int k = 0; k < N; ++k) {
    const int buf = k & 1;
    // (P) + (B) by warps 0 and 1 while the others wait: both take the pivot
    // from the per-warp candidates and form 1/pivot; warp 0 the negated
    // multipliers (pivot row swapped in) and the inverse's column k, warp 1
    // the raw pivot row, the swap of rows k and p with row k scaled, and the
    // copy of column k+1 (the two touch disjoint columns).
    if (tid < 64) {
      unsigned long long bk = g.ckey[buf][0];
      int p = g.cidx[buf][0];
      for (int q = 1; q < NWARP; ++q) {
        const unsigned long long kq = g.ckey[buf][q];
        const int iq = g.cidx[buf][q];
        if (kq > bk || (kq == bk && iq < p)) {
          bk = kq;
          p = iq;
        }
      }
      const int lane = tid & 31;
      if (bk <= 1ull || p >= N) {   // zero (key 1) or no finite entry: singular
        if (tid == 0) g.bad = 1;
      } else if (tid < 32) {
        const double piv = A[(size_t)p * lda + k];
        const double ipiv = __drcp_rn(piv);
        if (tid == 0) {
          perm[k] = p;
          g.ipiv = ipiv;
          g.apiv[k] = fabs(piv);   // log|det| is summed after the elimination
          if ((piv < 0.0) != (p != k)) g.sign = -g.sign;
        }
        const double nipiv = -ipiv;   // negated multipliers: the update is one FMA
        for (int i = lane; i < N; i += 32) {
          const double a = (i == k) ? 0.0 : A[(size_t)(i == p ? k : i) * lda + k];
          g.colk[i] = a * nipiv;
        }
        __syncwarp();
        // the inverse's column k: -m_i, and 1/pivot at row k (rowk_k = 0
        // leaves it through the update)
        for (int i = lane; i < N; i += 32) A[(size_t)i * lda + k] = (i == k) ? ipiv : g.colk[i];
      } else {
        const double ipiv = __drcp_rn(A[(size_t)p * lda + k]);
        for (int c = lane; c < N; c += 32) {
          if (c == k) {
            g.rowk[c] = 0.0;
            continue;
          }
          const double r = A[(size_t)p * lda + c];
          g.rowk[c] = r;
          if (p != k) A[(size_t)p * lda + c] = A[(size_t)k * lda + c];
          A[(size_t)k * lda + c] = r * ipiv;
        }
        __syncwarp();
        // column k+1 as the update below finds it (rows swapped)
        if (k + 1 < N)
          for (int i = lane; i < N; i += 32) g.coln[i] = A[(size_t)i * lda + k + 1];
      }
    }
    __syncthreads();
    if (g.bad) return;   // uniform
    const int k1 = k + 1;
    // (E0) pivot candidates of column k+1 among rows >= k+1, from the values
    // the update below stores there (the same FMA), so the next pivot needs
    // no barrier of its own
    if (k1 < N) {
      unsigned long long key = 0ull;
      int row = N;
      for (int i = tid; i < N; i += NT) {
        const double v = fma(g.colk[i], g.rowk[k1], g.coln[i]);
        const unsigned long long kk = pivot_key(v);
        const bool t = (i >= k1) & (kk > key);
        key = t ? kk : key;
        row = t ? i : row;
      }
      pivot_candidates(key, row, g, buf ^ 1);
    }
    // (E) a_ic += (-m_i) r_c over all entries, spread flat over the threads
    // in whole warps, GJ_ILP entries in flight per thread (m_k = 0 leaves
    // row k, r_k = 0 leaves column k)
    {
      int i = tid / N, c = tid - (tid / N) * N;
      while (i < N) {
        int ii[GJ_ILP], cc[GJ_ILP];
        ii[0] = i;
        cc[0] = c;
#pragma unroll
        for (int u = 1; u < GJ_ILP; ++u) {
          ii[u] = ii[u - 1];
          cc[u] = cc[u - 1];
          adv(ii[u], cc[u]);
        }
        double *q[GJ_ILP];
        double a[GJ_ILP];
#pragma unroll
        for (int u = 0; u < GJ_ILP; ++u) {
          const bool ok = ii[u] < N;
          q[u] = A + (size_t)(ok ? ii[u] : i) * lda + (ok ? cc[u] : c);
          a[u] = *q[u];
        }
#pragma unroll
        for (int u = 0; u < GJ_ILP; ++u) {
          const int iu = ii[u] < N ? ii[u] : i, cu = ii[u] < N ? cc[u] : c;
          a[u] = fma(g.colk[iu], g.rowk[cu], a[u]);
        }
#pragma unroll
        for (int u = 0; u < GJ_ILP; ++u)
          if (u == 0 || ii[u] < N) *q[u] = a[u];
        i = ii[GJ_ILP - 1];
        c = cc[GJ_ILP - 1];
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
