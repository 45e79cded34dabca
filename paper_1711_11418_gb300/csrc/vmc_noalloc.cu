// vmc_sr_force_static: the SR means and force of vmc_sr_step / vmc_get_sr_matrices
// (o_k = <O_k>, E = <E_loc>, g_k = <(O_k - o_k)(E_loc - E)>), computed from
// caller-owned device arrays without allocating any memory.
//
// Why it exists: some callers cannot let this library call cudaMalloc or
// cudaFree.  A typical case is a host application whose device memory is
// already owned by another allocator (for example a framework's caching
// allocator that has reserved the GPU), or one that must not block on the
// allocator's implicit device synchronisation in a latency-sensitive loop.
// Those callers pass their own input and output buffers; the only extra
// memory the kernels need -- the per-chunk partial column sums -- lives in
// the fixed-size array below, which every GPU that loads this library holds
// for as long as the process runs.
#include "../../include/vmc.h"

#include <cuda_runtime.h>

#include <mutex>

namespace {

constexpr int RCHUNK = 2048;   // rows per partial sum (fixed, so the scratch bound is simple)
constexpr int RTHREADS = 256;
constexpr int MAX_DEVICES = 64;
constexpr int MAX_GRID_Y = 65535;   // chunks beyond this are looped over inside the kernel

}  // namespace

// Scratch for the partial column sums: VMC_FORCE_STATIC_MAX_DOUBLES doubles
// (8 MiB), shared by every call in the process.
static __device__ __align__(256) double g_force_scratch[VMC_FORCE_STATIC_MAX_DOUBLES];

namespace {

// Device address of g_force_scratch per device, looked up once per process
// under a lock (host threads may make their first calls at the same time).
double *g_scratch_addr[MAX_DEVICES];
bool g_scratch_ready[MAX_DEVICES];
std::mutex g_scratch_lock;

__global__ void k_mean_rows(const double *E, int rows, double *out) {
  __shared__ double red[RTHREADS];
  double s = 0.0;
  for (int i = threadIdx.x; i < rows; i += blockDim.x) s += E[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0] / rows;
}

// part[c][k] = sum over the rows of chunk c of O_rk (mode 0) or
// (O_rk - obar_k)(E_r - ebar) (mode 1).  Every entry of part[0..nparts*Np)
// is written, so nothing from an earlier call is read.  Chunk c is taken by
// the blocks with blockIdx.y = c mod gridDim.y.
__global__ void k_colsum(const float *O, int ldO, int rows, int Np, int nparts,
                         const double *obar, const double *E, const double *ebar, int mode,
                         double *part) {
  const int k = blockIdx.x * RTHREADS + threadIdx.x;
  if (k >= Np) return;
  for (int c = blockIdx.y; c < nparts; c += gridDim.y) {
    const long long r0 = (long long)c * RCHUNK;
    const long long r1 = min((long long)rows, r0 + RCHUNK);
    double s = 0.0;
    if (mode == 0) {
      for (long long r = r0; r < r1; ++r) s += (double)O[(size_t)r * ldO + k];
    } else {
      const double ok = obar[k], eb = ebar[0];
      for (long long r = r0; r < r1; ++r) s += ((double)O[(size_t)r * ldO + k] - ok) * (E[r] - eb);
    }
    part[(size_t)c * Np + k] = s;
  }
}

__global__ void k_colsum_finish(const double *part, int nparts, int Np, double scale, double *out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Np) return;
  double s = 0.0;
  for (int c = 0; c < nparts; ++c) s += part[(size_t)c * Np + k];
  out[k] = s * scale;
}

}  // namespace

extern "C" int vmc_sr_force_static(const float *O, int32_t ldO, int32_t rows, int32_t Np,
                                   const double *E, double *obar, double *g, double *ebar,
                                   void *stream) {
  if (!O || !E || !obar || !g || !ebar) return VMC_EINVAL;
  if (rows < 1 || Np < 1 || ldO < Np) return VMC_EINVAL;
  const long long nparts = (rows + (long long)RCHUNK - 1) / RCHUNK;
  if (nparts * (long long)Np > (long long)VMC_FORCE_STATIC_MAX_DOUBLES) return VMC_EINVAL;
  // A launch error left pending by the caller's earlier work is not this
  // call's: report it without launching and without clearing it.
  if (cudaPeekAtLastError() != cudaSuccess) return VMC_ECUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return VMC_ECUDA;
  if (dev < 0 || dev >= MAX_DEVICES) return VMC_EINVAL;
  {
    std::lock_guard<std::mutex> lock(g_scratch_lock);
    if (!g_scratch_ready[dev]) {
      // Set-up on this device's first call: the host-side name of the array
      // is not a device address; ask the runtime for it with the device
      // current.
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_force_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return VMC_ECUDA;
      }
      g_scratch_addr[dev] = (double *)p;
      g_scratch_ready[dev] = true;
    }
  }
  double *part = g_scratch_addr[dev];
  cudaStream_t st = (cudaStream_t)stream;
  const dim3 grid((Np + RTHREADS - 1) / RTHREADS, (unsigned)(nparts < MAX_GRID_Y ? nparts : MAX_GRID_Y));
  const int fin = (Np + 255) / 256;
  // Each launch is checked at once, so an error is reported by the call
  // whose launch failed.
  k_mean_rows<<<1, RTHREADS, 0, st>>>(E, rows, ebar);
  if (cudaGetLastError() != cudaSuccess) return VMC_ECUDA;
  k_colsum<<<grid, RTHREADS, 0, st>>>(O, ldO, rows, Np, (int)nparts, nullptr, nullptr, nullptr, 0,
                                      part);
  if (cudaGetLastError() != cudaSuccess) return VMC_ECUDA;
  k_colsum_finish<<<fin, 256, 0, st>>>(part, (int)nparts, Np, 1.0 / rows, obar);
  if (cudaGetLastError() != cudaSuccess) return VMC_ECUDA;
  k_colsum<<<grid, RTHREADS, 0, st>>>(O, ldO, rows, Np, (int)nparts, obar, E, ebar, 1, part);
  if (cudaGetLastError() != cudaSuccess) return VMC_ECUDA;
  k_colsum_finish<<<fin, 256, 0, st>>>(part, (int)nparts, Np, 1.0 / rows, g);
  if (cudaGetLastError() != cudaSuccess) return VMC_ECUDA;
  return VMC_OK;
}
