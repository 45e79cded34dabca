// First-step power-Lanczos on the GPU (mVMC paper, Sec. 3.4): the local
// values F(x, H) = <x|H|psi>/<x|psi> (= E_loc) and F(x, H^2) of every walker's
// current configuration, and their walker means, the moments h1, h2(11),
// h2(20), h3(12) from which E_1(alpha) and alpha_1 follow.
//
// With D the diagonal part of H and h_t the matrix element of an off-diagonal
// term t (a hop: -t_ij, labels kept, so no fermion sign):
//
//   F(x, H)   = D(x) + sum_{t1} h_{t1} R(t1),
//   F(x, H^2) = D(x) F(x, H) + sum_{t1} h_{t1} [ D(x') R(t1) + sum_{t2} h_{t2} R(t1, t2) ],
//
// x' = t1 x, x'' = t2 x', R(t1) = psi(x')/psi(x), R(t1, t2) = psi(x'')/psi(x):
// every ratio is taken from x, so nothing divides by psi(x') (which may
// vanish).  The Pfaffian parts of the ratios come from three tables of the
// configuration, with B = M^-1:
//
//   Gu[b][k] = sum_l f(b, r_l,dn) B[l][k]   (up electron k to site b),
//   Gd[a][m] = sum_k f(r_k,up, a) B[m][k]   (down electron m to site a),
//   T[b][a]  = sum_k Gu[b][k] f(r_k,up, a),
//
// by the determinant lemma: two up electrons k1 -> b1, k2 -> b2 give
// Gu[b1][k1] Gu[b2][k2] - Gu[b1][k2] Gu[b2][k1] (two down electrons alike with
// Gd), and up k -> b with down m -> a give Gu[b][k] Gd[a][m] - B[m][k] (T[b][a] - f(b, a)).
// The correlation factors of x'' are those of two successive hops, the second
// on the occupations and Jastrow field of x'.
//
// One CTA of 128 threads per walker, the tables in a per-CTA slot of global
// memory; warps take the first terms t1, lanes the second terms t2.
#include "vmc_common.cuh"
#include "vmc_dev.cuh"

#include <math.h>

namespace {

// Per-CTA table slot: Gu (Ns x N), Gd (Ns x N), T (Ns x Ns), in elements.
__host__ __device__ inline size_t lz_slot_elems(int Ns, int N) {
  return 2 * (size_t)Ns * N + (size_t)Ns * Ns;
}

template <typename T>
__device__ __forceinline__ const T *minv_of(const SysDev &S, int w) {
  const size_t nb = ((size_t)S.N * S.ldm * sizeof(T) + 127) / 128 * 128;
  return (const T *)((const unsigned char *)S.minv + (size_t)w * nb);
}

// log P(y')/P(y) of a hop of a spin-s electron from site r to site t on a
// configuration y given by its occupations (occ, with the hop's own electron
// at r) and Jastrow field jf (Sec. 3.2.3), in the ratios' type (FP64, or FP32
// in the mixed form: GB300's FP64 pipe is 1/64 of the FP32 rate).
template <typename T>
__device__ __forceinline__ T corr_log(const SysDev &S, const int *occ, const T *jf, int s, int r,
                                      int t) {
  const int Ns = S.Ns, o = (1 - s) * Ns;
  const T *g = gtab<T>(S);
  T d = jf[t] - jf[r] - vtab<T>(S)[(size_t)r * Ns + t];
  d += (occ[o + t] >= 0 ? g[t] : (T)0) - (occ[o + r] >= 0 ? g[r] : (T)0);
  return d;
}

// Diagonal part of H (U n_up n_dn + V n n) of x moved by one hop of a spin-s
// electron r -> t (r = t = -1: x itself), by one warp.
__device__ double diag_energy(const SysDev &S, const int *occ, int s, int r, int t) {
  const int Ns = S.Ns, lane = threadIdx.x & 31;
  auto nsp = [&](int i, int sp) -> int {
    int v = occ[sp * Ns + i] >= 0;
    if (sp == s) v += (i == t) - (i == r);
    return v;
  };
  double d = 0.0;
  for (int i = lane; i < Ns; i += 32)
    if (nsp(i, 0) && nsp(i, 1)) d += S.U[i];
  for (int k = lane; k < S.n_V; k += 32) {
    const int a = S.V_i[k], b = S.V_j[k];
    d += S.V_val[k] * (double)((nsp(a, 0) + nsp(a, 1)) * (nsp(b, 0) + nsp(b, 1)));
  }
  return warp_sum(d);
}

template <typename T>
__global__ void __launch_bounds__(NT) k_lanczos(const SysDev *systems, int sys, T *slots,
                                                double *F1, double *F2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ SysDev S;
  __shared__ int ele[2 * VMC_MAX_N];
  __shared__ double red[2 * 16];
  load_sys(&S, systems + sys);
  const int N = S.N, Ns = S.Ns, Ne = S.Ne, tid = threadIdx.x;
  T *jf = (T *)smem_raw;                       // Ns (space for Ns doubles)
  int *occ = (int *)((double *)smem_raw + Ns); // 2 Ns
  const int warp = tid >> 5, lane = tid & 31;
  const T *F = ftab<T>(S);
  const T *V = vtab<T>(S);
  const T *G = gtab<T>(S);
  T *Gu = slots + (size_t)blockIdx.x * lz_slot_elems(Ns, N);
  T *Gd = Gu + (size_t)Ns * N;
  T *Tt = Gd + (size_t)Ns * N;
  const int nterm = 2 * S.n_hop;
  for (int w = blockIdx.x; w < S.W; w += gridDim.x) {
    __syncthreads();
    for (int k = tid; k < Ne; k += NT) ele[k] = S.ele[(size_t)w * Ne + k];
    for (int k = tid; k < 2 * Ns; k += NT) occ[k] = S.occ[(size_t)w * 2 * Ns + k];
    for (int k = tid; k < Ns; k += NT) jf[k] = ((const T *)S.jf)[(size_t)w * Ns + k];
    __syncthreads();
    const T *B = minv_of<T>(S, w);
    const int ldm = S.ldm;
    for (size_t q = tid; q < (size_t)Ns * N; q += NT) {
      const int b = (int)(q / N), k = (int)(q % N);
      T gu = (T)0, gd = (T)0;
      for (int l = 0; l < N; ++l) {
        gu += F[(size_t)b * Ns + ele[N + l]] * B[(size_t)l * ldm + k];
        gd += F[(size_t)ele[l] * Ns + b] * B[(size_t)k * ldm + l];
      }
      Gu[q] = gu;
      Gd[q] = gd;
    }
    __syncthreads();
    for (size_t q = tid; q < (size_t)Ns * Ns; q += NT) {
      const int b = (int)(q / Ns), a = (int)(q % Ns);
      T s = (T)0;
      for (int k = 0; k < N; ++k) s += Gu[(size_t)b * N + k] * F[(size_t)ele[k] * Ns + a];
      Tt[q] = s;
    }
    __syncthreads();
    // one-hop Pfaffian ratio from x: electron e (spin by label) to site t
    auto r1 = [&](int e, int t) -> T {
      return e < N ? Gu[(size_t)t * N + e] : Gd[(size_t)t * N + (e - N)];
    };
    // two-hop Pfaffian ratio from x: electrons e1 -> t1 and e2 -> t2 (e1 != e2)
    auto r2 = [&](int e1, int t1, int e2, int t2) -> T {
      if (e1 < N && e2 < N)
        return Gu[(size_t)t1 * N + e1] * Gu[(size_t)t2 * N + e2] -
               Gu[(size_t)t1 * N + e2] * Gu[(size_t)t2 * N + e1];
      if (e1 >= N && e2 >= N)
        return Gd[(size_t)t1 * N + (e1 - N)] * Gd[(size_t)t2 * N + (e2 - N)] -
               Gd[(size_t)t1 * N + (e2 - N)] * Gd[(size_t)t2 * N + (e1 - N)];
      const int ku = e1 < N ? e1 : e2, bu = e1 < N ? t1 : t2;
      const int md = (e1 < N ? e2 : e1) - N, ad = e1 < N ? t2 : t1;
      return Gu[(size_t)bu * N + ku] * Gd[(size_t)ad * N + md] -
             B[(size_t)md * ldm + ku] * (Tt[(size_t)bu * Ns + ad] - F[(size_t)bu * Ns + ad]);
    };
    // a hop term q = 2k + s: the spin-s electron on j = hop_j[k] to i = hop_i[k]
    auto valid_on = [&](const int *oc, int s, int i, int j) -> bool {
      if (oc[s * Ns + j] < 0 || oc[s * Ns + i] >= 0) return false;
      if (S.local_spin && oc[(1 - s) * Ns + i] >= 0) return false;
      if (S.lsite && (S.lsite[i] | S.lsite[j])) return false;
      return true;
    };
    const double d0 = diag_energy(S, occ, 0, -1, -1);
    double f1 = 0.0, f2 = 0.0;
    for (int q1 = warp; q1 < nterm; q1 += NWARP) {
      const int k1 = q1 >> 1, s1 = q1 & 1;
      const int i1 = S.hop_i[k1], j1 = S.hop_j[k1];
      if (!valid_on(occ, s1, i1, j1)) continue;
      const int e1 = occ[s1 * Ns + j1];
      const T c1 = corr_log<T>(S, occ, jf, s1, j1, i1);
      const double R1 = (double)(r1(e1, i1) * corr_factor<T>(c1));
      const double h1 = -S.hop_t[k1];
      const double dx = diag_energy(S, occ, s1, j1, i1);
      // second terms on x' = (e1: j1 -> i1) x
      T acc = (T)0;
      for (int q2 = lane; q2 < nterm; q2 += 32) {
        const int k2 = q2 >> 1, s2 = q2 & 1;
        const int i2 = S.hop_i[k2], j2 = S.hop_j[k2];
        // occupations of x' at the sites t2 touches
        auto occp = [&](int sp, int i) -> int {
          if (sp == s1) {
            if (i == j1) return -1;
            if (i == i1) return e1;
          }
          return occ[sp * Ns + i];
        };
        if (occp(s2, j2) < 0 || occp(s2, i2) >= 0) continue;
        if (S.local_spin && occp(1 - s2, i2) >= 0) continue;
        if (S.lsite && (S.lsite[i2] | S.lsite[j2])) continue;
        const int e2 = occp(s2, j2);
        T R;
        if (e2 == e1) {
          // e1 moves again: x'' is x with e1 on i2 (x itself if i2 = j1)
          R = (i2 == j1) ? (T)1 : r1(e1, i2) * corr_factor<T>(corr_log<T>(S, occ, jf, s1, j1, i2));
        } else {
          // second hop on x': Jastrow field and occupations of x'
          const T jfi = jf[i2] + V[(size_t)i2 * Ns + i1] - V[(size_t)i2 * Ns + j1];
          const T jfj = jf[j2] + V[(size_t)j2 * Ns + i1] - V[(size_t)j2 * Ns + j1];
          T c2 = jfi - jfj - V[(size_t)j2 * Ns + i2];
          c2 += (occp(1 - s2, i2) >= 0 ? G[i2] : (T)0) - (occp(1 - s2, j2) >= 0 ? G[j2] : (T)0);
          R = r2(e1, i1, e2, i2) * corr_factor<T>(c1 + c2);
        }
        acc += (T)(-S.hop_t[k2]) * R;
      }
      const double accd = warp_sum((double)acc);
      if (lane == 0) {
        f1 += h1 * R1;
        f2 += h1 * (dx * R1 + accd);
      }
    }
    // block sums (lane 0 of each warp holds its part)
    f1 = warp_sum(f1);
    f2 = warp_sum(f2);
    if (lane == 0) {
      red[warp] = f1;
      red[16 + warp] = f2;
    }
    __syncthreads();
    if (tid == 0) {
      double a = 0.0, b = 0.0;
      for (int k = 0; k < NWARP; ++k) {
        a += red[k];
        b += red[16 + k];
      }
      const double e = d0 + a;
      F1[w] = e;
      F2[w] = d0 * e + b;
    }
  }
}

// h1 = <F1>, h2(11) = <F1^2>, h2(20) = <F2>, h3(12) = <F1 F2> over the walkers.
__global__ void k_lanczos_moments(const double *F1, const double *F2, int W, double *h) {
  __shared__ double red[4][NT];
  double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
  for (int w = threadIdx.x; w < W; w += NT) {
    a += F1[w];
    b += F1[w] * F1[w];
    c += F2[w];
    d += F1[w] * F2[w];
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  red[2][threadIdx.x] = c;
  red[3][threadIdx.x] = d;
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int k = 0; k < NT; ++k) s += red[threadIdx.x][k];
    h[threadIdx.x] = s / W;
  }
}

}  // namespace

size_t vmc_lanczos_slot_bytes(int precision, int Ns, int N) {
  return lz_slot_elems(Ns, N) * (precision == 0 ? sizeof(double) : sizeof(float));
}

size_t vmc_lanczos_smem(int Ns) { return (size_t)Ns * (sizeof(double) + 2 * sizeof(int)); }

// CTAs of k_lanczos per SM (registers and shared memory): the kernel waits on
// L2 reads of its tables, so the grid fills every slot.
int vmc_lanczos_occupancy(int precision, int Ns) {
  int nb = 0;
  const size_t smem = vmc_lanczos_smem(Ns);
  if (precision == 0) {
    cudaFuncSetAttribute(k_lanczos<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_lanczos<double>, NT, smem);
  } else {
    cudaFuncSetAttribute(k_lanczos<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_lanczos<float>, NT, smem);
  }
  return nb;
}

cudaError_t vmc_launch_lanczos(const SysDev *d_sys, int sys, int precision, int Ns, int grid,
                               void *slots, double *F1, double *F2, int W, double *moments,
                               cudaStream_t st, long long *nl) {
  const size_t smem = vmc_lanczos_smem(Ns);
  cudaError_t e;
  if (precision == 0) {
    if ((e = cudaFuncSetAttribute(k_lanczos<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)))
      return e;
    k_lanczos<double><<<grid, NT, smem, st>>>(d_sys, sys, (double *)slots, F1, F2);
  } else {
    if ((e = cudaFuncSetAttribute(k_lanczos<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)))
      return e;
    k_lanczos<float><<<grid, NT, smem, st>>>(d_sys, sys, (float *)slots, F1, F2);
  }
  k_lanczos_moments<<<1, NT, 0, st>>>(F1, F2, W, moments);
  *nl += 2;
  return cudaGetLastError();
}
