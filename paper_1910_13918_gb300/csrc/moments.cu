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
    const size_t o = (size_t)iy * a.pitch + ix;
    const int npop = a.cp.npop;
    double rho = 0.0, jx = 0.0, jy = 0.0, e2 = 0.0;
    for (int i = 0; i < kQ; ++i) {
      const double cx = a.cs.xi[i / 5], cy = a.cs.xi[i % 5];
      double fv, gv = 0.0;
      if (Store == kStoreF64) {
        const double* s = static_cast<const double*>(a.src);
        fv = s[(size_t)i * a.plane_stride + o];
        if (npop == 2) gv = s[(size_t)(kQ + i) * a.plane_stride + o];
      } else if (Store == kStoreF32) {
        const float* s = static_cast<const float*>(a.src);
        fv = s[(size_t)i * a.plane_stride + o];
        if (npop == 2) gv = s[(size_t)(kQ + i) * a.plane_stride + o];
      } else {
        const __nv_bfloat16* s = static_cast<const __nv_bfloat16*>(a.src);
        fv = __bfloat162float(s[(size_t)i * a.plane_stride + o]);
        if (npop == 2) gv = __bfloat162float(s[(size_t)(kQ + i) * a.plane_stride + o]);
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
