// Macroscopic fields of the stored state (moments of Sec. II: rho, rho u, 2 rho E, and T) and the
// FP64 global sums M = sum_v A_v rho_v, E = sum_v A_v rho_v E_v (mass check of Sec. III.E).
// Deterministic two-pass reduction: fixed-order block partials, then one block over the partials.
#include "kernels.h"

namespace sllbm {

constexpr int kMomThreads = 256;

int moments_blocks(long long nv) { return (int)((nv + kMomThreads - 1) / kMomThreads); }

template <int Store>
__global__ void __launch_bounds__(kMomThreads) moments_kernel(const __grid_constant__ MomentArgs a) {
  __shared__ double sm[2][kMomThreads];
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double m = 0.0, en = 0.0;
  if (v < a.nv) {
    const int ix = (int)(v % a.nx), iy = (int)(v / a.nx);
    const size_t o = (size_t)iy * a.pitch + (size_t)ix * a.xs;
    const int npop = a.cp.npop;
    double rho = 0.0, jx = 0.0, jy = 0.0, e2 = 0.0;
    const int nq1 = a.cs.nq1;
    for (int i = 0; i < nq1 * nq1; ++i) {
      const double cx = a.cs.xi[i / nq1], cy = a.cs.xi[i % nq1];
      double fv, gv = 0.0;
      if (Store == kStoreF64) {
        const double* s = static_cast<const double*>(a.src);
        fv = s[(size_t)i * a.plane_stride + o];
        if (npop == 2) gv = s[(size_t)i * a.plane_stride + a.ps + o];
      } else if (Store == kStoreF32) {
        const float* s = static_cast<const float*>(a.src);
        fv = s[(size_t)i * a.plane_stride + o];
        if (npop == 2) gv = s[(size_t)i * a.plane_stride + a.ps + o];
      } else {
        const __nv_bfloat16* s = static_cast<const __nv_bfloat16*>(a.src);
        fv = __bfloat162float(s[(size_t)i * a.plane_stride + o]);
        if (npop == 2) gv = __bfloat162float(s[(size_t)i * a.plane_stride + a.ps + o]);
      }
      rho += fv;
      jx += fv * cx;
      jy += fv * cy;
      e2 += fv * (cx * cx + cy * cy) + gv;
    }
    if (Store != kStoreF64) {  // deviations: add the lattice-weight parts
      rho += 1.0;
      e2 += 2.0 * a.cp.cv;    // sum w |xi|^2 + K sum w = D + K = 2 C_v
    }
    const double ux = jx / rho, uy = jy / rho;
    const double theta = (e2 - rho * (ux * ux + uy * uy)) / (2.0 * a.cp.cv * rho);
    if (a.rho) a.rho[v] = (float)rho;
    if (a.u) a.u[v] = (float)ux;
    if (a.v) a.v[v] = (float)uy;
    if (a.T) a.T[v] = (float)theta;   // T0 = 1
    if (!(rho > 0.0 && theta > 0.0 && isfinite(rho) && isfinite(theta))) atomicOr(a.flag, 1);
    if (a.A) {
      m = a.A[v] * rho;
      en = a.A[v] * 0.5 * e2;
    }
  }
  if (!a.partials) return;
  sm[0][threadIdx.x] = m;
  sm[1][threadIdx.x] = en;
  __syncthreads();
  for (int s = kMomThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sm[0][threadIdx.x] += sm[0][threadIdx.x + s];
      sm[1][threadIdx.x] += sm[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    a.partials[blockIdx.x] = sm[0][0];
    a.partials[gridDim.x + blockIdx.x] = sm[1][0];
  }
}

__global__ void __launch_bounds__(kMomThreads) reduce_partials_kernel(const double* partials, int n,
                                                                      double* sums) {
  __shared__ double sm[2][kMomThreads];
  double m = 0.0, en = 0.0;
  for (int k = threadIdx.x; k < n; k += kMomThreads) {
    m += partials[k];
    en += partials[n + k];
  }
  sm[0][threadIdx.x] = m;
  sm[1][threadIdx.x] = en;
  __syncthreads();
  for (int s = kMomThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sm[0][threadIdx.x] += sm[0][threadIdx.x + s];
      sm[1][threadIdx.x] += sm[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sums[0] = sm[0][0];
    sums[1] = sm[1][0];
  }
}

cudaError_t launch_moments(const MomentArgs& a, cudaStream_t s) {
  const int blocks = moments_blocks(a.nv);
  switch (a.store) {
    case kStoreF32: moments_kernel<kStoreF32><<<blocks, kMomThreads, 0, s>>>(a); break;
    case kStoreBF16: moments_kernel<kStoreBF16><<<blocks, kMomThreads, 0, s>>>(a); break;
    case kStoreF64: moments_kernel<kStoreF64><<<blocks, kMomThreads, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !a.partials) return e;
  reduce_partials_kernel<<<1, kMomThreads, 0, s>>>(a.partials, blocks, a.sums);
  return cudaGetLastError();
}

}  // namespace sllbm

// ------------------------------------------------------------------------------------------
// Allocation-free variant of the moments / mass-energy reduction (sllbm_moments_noalloc).
//
// The reduction needs per-block FP64 partials and an instability flag.  Here they live in a
// file-scope device array instead of memory the caller or a context allocates.  Every GPU that
// loads the library holds this array until the process exits.  In host code the symbol is only
// a stand-in, so its device address is looked up with cudaGetSymbolAddress on every call, with
// the caller's device current: a host-side query that enqueues nothing, so no address is cached
// that a rebuilt context could invalidate and concurrent first calls share no host state.
// ------------------------------------------------------------------------------------------
#include <math.h>

#include "../../include/sllbm.h"

namespace sllbm {

constexpr int kNoAllocMaxBlocks = 65536;   // => at most 65536 * 256 = 16,777,216 vertices
constexpr long long kNoAllocMaxVertices = (long long)kNoAllocMaxBlocks * kMomThreads;
// layout: [0, 2 * kNoAllocMaxBlocks) doubles of partials, then one int flag (in a double slot)
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocMaxBlocks + 2];

static cudaError_t noalloc_scratch(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

}  // namespace sllbm

extern "C" sllbm_status sllbm_moments_noalloc(const float* state_dev, int nx, int ny, double cv,
                                              const double* A_dev, float* rho_dev, float* u_dev,
                                              float* v_dev, float* T_dev, double* mass_energy_dev,
                                              void* cuda_stream) {
  using namespace sllbm;
  if (!state_dev || nx < 1 || ny < 1 || !(cv >= 1.0)) return SLLBM_ERR_ARG;
  if (A_dev && !mass_energy_dev) return SLLBM_ERR_ARG;   // the sums need somewhere to go
  const long long nv = (long long)nx * ny;
  if (nv > kNoAllocMaxVertices) return SLLBM_ERR_UNSUPPORTED;   // checked before any int cast
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  double* scratch = nullptr;
  if (noalloc_scratch(&scratch) != cudaSuccess) return SLLBM_ERR_CUDA;
  int* flag = reinterpret_cast<int*>(scratch + 2 * kNoAllocMaxBlocks);
  if (cudaMemsetAsync(flag, 0, sizeof(int), s) != cudaSuccess) return SLLBM_ERR_CUDA;  // starts at zero
  MomentArgs a{};
  a.src = state_dev;
  a.nx = nx;
  a.ny = ny;
  a.pitch = nx;
  a.nv = nv;
  a.plane_stride = (size_t)nv;
  a.xs = 1;                       // dense planar input: g planes follow the 25 f planes
  a.ps = (ptrdiff_t)kQ * nv;
  const double s10 = sqrt(10.0), sm = sqrt(5.0 - s10), lg = sqrt(5.0 + s10);
  const double xi[5] = {0.0, sm, lg, -sm, -lg};
  for (int k = 0; k < 5; ++k) a.cs.xi[k] = xi[k];
  a.cs.nq1 = kQ1;                 // the D2Q25 set
  a.cp.cv = cv;
  a.cp.npop = (cv == 1.0) ? 1 : 2;
  a.store = kStoreF32;
  a.A = A_dev;
  a.rho = rho_dev;
  a.u = u_dev;
  a.v = v_dev;
  a.T = T_dev;
  a.partials = A_dev ? scratch : nullptr;   // the block partials are all overwritten: no clearing
  a.sums = A_dev ? mass_energy_dev : nullptr;
  a.flag = flag;
  if (launch_moments(a, s) != cudaSuccess) return SLLBM_ERR_CUDA;
  int host_flag = 0;
  if (cudaMemcpyAsync(&host_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return SLLBM_ERR_CUDA;
  return (host_flag & 1) ? SLLBM_ERR_UNSTABLE : SLLBM_OK;
}
