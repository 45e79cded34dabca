// Device helpers shared by the walker kernels (the plain walker and the
// projected one): launch shape, parameter-table access, the correlation-
// factor ratio of a hop (mVMC paper, Sec. 3.2.3), warp sums, the copy of a
// system descriptor into shared memory, and per-walker move counters.
#pragma once

#include "vmc_common.cuh"

#include <math.h>

namespace {

constexpr int NT = VMC_NT;
constexpr int NWARP = NT / 32;

template <typename T> __device__ __forceinline__ const T *ftab(const SysDev &s);
template <> __device__ __forceinline__ const double *ftab<double>(const SysDev &s) { return s.f64; }
template <> __device__ __forceinline__ const float *ftab<float>(const SysDev &s) { return s.f32; }
template <typename T> __device__ __forceinline__ const T *fTtab(const SysDev &s);
template <> __device__ __forceinline__ const double *fTtab<double>(const SysDev &s) { return s.fT64; }
template <> __device__ __forceinline__ const float *fTtab<float>(const SysDev &s) { return s.fT32; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);   // lane 0's value: identical in every lane
}

// log of the correlation-factor ratio P(x')/P(x) for a hop of a spin-s
// electron from site r to site t (Sec. 3.2.3): Gutzwiller g_t n_t,-s - g_r n_r,-s
// and Jastrow h_t - h_r - v_rt with h_i = sum_{j != i} v_ij (n_j - 1).
template <typename T> __device__ __forceinline__ const T *vtab(const SysDev &s);
template <> __device__ __forceinline__ const double *vtab<double>(const SysDev &s) { return s.vmat; }
template <> __device__ __forceinline__ const float *vtab<float>(const SysDev &s) { return s.vmat32; }
template <typename T> __device__ __forceinline__ const T *gtab(const SysDev &s);
template <> __device__ __forceinline__ const double *gtab<double>(const SysDev &s) { return s.gsite; }
template <> __device__ __forceinline__ const float *gtab<float>(const SysDev &s) { return s.gsite32; }

// In the sweep's arithmetic type (FP32 in the mixed form: GB300's FP64 pipe
// is too slow for per-proposal work).
template <typename T, typename OI>
__device__ __forceinline__ T corr_hop(const SysDev &S, const OI *occ, const T *jf, int s, int r,
                                      int t) {
  const int Ns = S.Ns;
  const int o = (1 - s) * Ns;
  const T *g = gtab<T>(S);
  T d = jf[t] - jf[r] - vtab<T>(S)[(size_t)r * Ns + t];
  d += (occ[o + t] >= 0 ? g[t] : (T)0) - (occ[o + r] >= 0 ? g[r] : (T)0);
  return d;
}

template <typename T> __device__ __forceinline__ const T *tvtab(const SysDev &s);
template <> __device__ __forceinline__ const double *tvtab<double>(const SysDev &s) { return s.tgt_v64; }
template <> __device__ __forceinline__ const float *tvtab<float>(const SysDev &s) { return s.tgt_v32; }

// Same, with g from shared memory and v_rt given.
template <typename T, typename OI>
__device__ __forceinline__ T corr_hop_v(const OI *occ, const T *jf, const T *g, int Ns, int s,
                                        int r, int t, T vrt) {
  const int o = (1 - s) * Ns;
  T d = jf[t] - jf[r] - vrt;
  d += (occ[o + t] >= 0 ? g[t] : (T)0) - (occ[o + r] >= 0 ? g[r] : (T)0);
  return d;
}

template <typename T> __device__ __forceinline__ T corr_factor(T dlog);
template <> __device__ __forceinline__ double corr_factor<double>(double dlog) { return exp(dlog); }
template <> __device__ __forceinline__ float corr_factor<float>(float dlog) { return expf(dlog); }

// An accepted move with |det M'/det M| below SMALL_RATIO amplifies the
// rounding already in the updated inverse by more than 1/SMALL_RATIO: the
// walker is then marked due for the next from-scratch rebuild whatever its
// count of accepted moves (the count is set to RECOMPUTE_NOW, above any
// recompute interval).
constexpr double SMALL_RATIO = 1e-3;
constexpr int RECOMPUTE_NOW = 1 << 30;

struct MoveCounts {
  long long hop_t = 0, ex_t = 0, hop_a = 0, ex_a = 0;
  long long meas_hop = 0, meas_ex = 0, samples = 0;
};

__device__ void load_sys(SysDev *dst, const SysDev *src) {
  const int nw = sizeof(SysDev) / sizeof(int);
  const int *s = (const int *)src;
  int *d = (int *)dst;
  for (int k = threadIdx.x; k < nw; k += blockDim.x) d[k] = s[k];
  __syncthreads();
}

}  // namespace
