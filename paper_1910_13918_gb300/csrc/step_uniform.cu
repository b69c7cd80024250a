// Fused SLLBM step for uniform grids, FP32 arithmetic (FP32 or BF16 storage).
//
// Pull streaming (Eq. sl_streaming) + moments + fourth-order equilibrium + BGK (Eq. streaming_fg,
// Pr = 1) in one kernel.  On a uniform grid the departure x_v - dt xi_i separates per axis, so the
// (p+1)^2 interpolation of a velocity plane factorises: first along y (weights depend on the row
// and the y component b only), then along x (weights depend on the column and a only).
//
// CTA = TY warps; tile = 32 columns x TY rows of vertices, one vertex per thread.  For each of the
// 50 population planes the CTA stages the plane's source tile (tile + stencil halo, periodic wrap
// or clamp) in shared memory, warp w computes the y-interpolated row w for every staged column,
// then every thread x-interpolates its vertex.  The next plane's tile is loaded into registers
// while the current one is interpolated.  After the last plane each thread holds the 50
// pre-collision deviations of its vertex, collides, and writes 50 coalesced rows.
#include "kernels.h"

namespace sllbm {

constexpr int kUniformTY = 8;
constexpr int kUniformNSTG = 4;

__device__ __forceinline__ int fold_index(int j, int n, int periodic) {
  if (periodic) {
    j %= n;
    return j < 0 ? j + n : j;
  }
  return j < 0 ? 0 : (j >= n ? n - 1 : j);
}

template <int P, typename Store, int TY, int NSTG>
__global__ void __launch_bounds__(32 * TY, 2) step_uniform_kernel(const __grid_constant__ StepArgs a) {
  extern __shared__ float smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int R = TY + a.offy_max - a.offy_min;
  const int C = 32 + a.offx_max - a.offx_min;
  float* S = smem;                       // [R][C] staged source plane
  float* T = S + R * C;                  // [TY][C] y-interpolated rows
  float* YW = T + TY * C;                // [5][TY][P+1] y weights of the tile rows
  int* YO = reinterpret_cast<int*>(YW + 5 * TY * (P + 1));  // [5][TY] first staged stencil row
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * TY;
  const int x = x0 + lane, y = y0 + warp;
  const int xc = x < a.nx ? x : a.nx - 1;
  const int nthreads = 32 * TY;

  for (int e = threadIdx.x; e < 5 * TY; e += nthreads) {
    const int b = e / TY, r = e % TY;
    const int yy = (y0 + r) < a.ny ? (y0 + r) : a.ny - 1;
    YO[e] = a.offy[b * a.ny + yy] + r - a.offy_min;
#pragma unroll
    for (int k = 0; k <= P; ++k) YW[e * (P + 1) + k] = a.wy[(b * a.ny + yy) * (P + 1) + k];
  }
  int goff[NSTG];
#pragma unroll
  for (int k = 0; k < NSTG; ++k) {
    const int e = threadIdx.x + k * nthreads;
    if (e < R * C) {
      const int row = e / C, col = e - row * C;
      const int gy = fold_index(y0 + a.offy_min + row, a.ny, a.periodic_y);
      const int gx = fold_index(x0 + a.offx_min + col, a.nx, a.periodic_x);
      goff[k] = gy * a.pitch + gx;
    } else {
      goff[k] = -1;
    }
  }
  const Store* src = static_cast<const Store*>(a.src);
  const int npop = a.cp.npop;
  float pre[NSTG];
#pragma unroll
  for (int k = 0; k < NSTG; ++k) pre[k] = goff[k] >= 0 ? ld_store(src + goff[k]) : 0.f;

  float vals[2 * kQ];
#pragma unroll
  for (int ia = 0; ia < kQ1; ++ia) {
    const int ox = a.offx[ia * a.nx + xc] + lane - a.offx_min;
    float wxr[P + 1];
#pragma unroll
    for (int k = 0; k <= P; ++k) wxr[k] = __ldg(a.wx + (ia * a.nx + xc) * (P + 1) + k);
#pragma unroll
    for (int ib = 0; ib < kQ1; ++ib) {
#pragma unroll
      for (int pop = 0; pop < 2; ++pop) {
        const int plane = pop * kQ + 5 * ia + ib;
        if (pop < npop) {
          // stage this plane (its tile is in pre[]), then start loading the next one
#pragma unroll
          for (int k = 0; k < NSTG; ++k)
            if (goff[k] >= 0) S[threadIdx.x + k * nthreads] = pre[k];
          int next;
          if (pop == 0 && npop == 2)
            next = kQ + 5 * ia + ib;
          else
            next = (5 * ia + ib + 1 < kQ) ? 5 * ia + ib + 1 : -1;
          if (next >= 0) {
            const Store* pl = src + (size_t)next * a.plane_stride;
#pragma unroll
            for (int k = 0; k < NSTG; ++k) pre[k] = goff[k] >= 0 ? ld_store(pl + goff[k]) : 0.f;
          }
          __syncthreads();
          {  // y pass: row `warp` of the tile, every staged column
            const int eidx = ib * TY + warp;
            const int oy = YO[eidx];
            float wyr[P + 1];
#pragma unroll
            for (int k = 0; k <= P; ++k) wyr[k] = YW[eidx * (P + 1) + k];
            for (int c = lane; c < C; c += 32) {
              float acc = 0.f;
#pragma unroll
              for (int k = 0; k <= P; ++k) acc += wyr[k] * S[(oy + k) * C + c];
              T[warp * C + c] = acc;
            }
          }
          __syncthreads();
          float acc = 0.f;
#pragma unroll
          for (int k = 0; k <= P; ++k) acc += wxr[k] * T[warp * C + ox + k];
          vals[plane] = acc;
        } else {
          vals[plane] = 0.f;
        }
      }
    }
  }
  const bool ok = collide_deviation_f32(vals, a.cs, a.cp);
  if (x < a.nx && y < a.ny) {
    if (!ok) atomicOr(a.flag, 1);
    Store* dst = static_cast<Store*>(a.dst);
    const size_t o = (size_t)y * a.pitch + x;
#pragma unroll
    for (int i = 0; i < kQ; ++i) st_store(dst + (size_t)i * a.plane_stride + o, vals[i]);
    if (npop == 2) {
#pragma unroll
      for (int i = 0; i < kQ; ++i) st_store(dst + (size_t)(kQ + i) * a.plane_stride + o, vals[kQ + i]);
    }
  }
}

static size_t uniform_smem_bytes(const StepArgs& a) {
  const int TY = kUniformTY;
  const int R = TY + a.offy_max - a.offy_min;
  const int C = 32 + a.offx_max - a.offx_min;
  return sizeof(float) * ((size_t)R * C + (size_t)TY * C + 5 * TY * (a.P + 1)) + sizeof(int) * 5 * TY;
}

bool uniform_kernel_fits(const StepArgs& a) {
  const int TY = kUniformTY;
  const int R = TY + a.offy_max - a.offy_min;
  const int C = 32 + a.offx_max - a.offx_min;
  return R * C <= kUniformNSTG * 32 * TY && uniform_smem_bytes(a) <= 48 * 1024;
}

template <int P, typename Store>
static cudaError_t launch_p(const StepArgs& a, cudaStream_t s) {
  const int TY = kUniformTY;
  dim3 grid((a.nx + 31) / 32, (a.ny + TY - 1) / TY);
  step_uniform_kernel<P, Store, TY, kUniformNSTG><<<grid, 32 * TY, uniform_smem_bytes(a), s>>>(a);
  return cudaGetLastError();
}

template <typename Store>
static cudaError_t launch_store(const StepArgs& a, cudaStream_t s) {
  switch (a.P) {
    case 1: return launch_p<1, Store>(a, s);
    case 2: return launch_p<2, Store>(a, s);
    case 3: return launch_p<3, Store>(a, s);
    case 4: return launch_p<4, Store>(a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_step_uniform(const StepArgs& a, int store, cudaStream_t s) {
  if (!uniform_kernel_fits(a)) return cudaErrorNotSupported;
  if (store == kStoreBF16) return launch_store<__nv_bfloat16>(a, s);
  return launch_store<float>(a, s);
}

}  // namespace sllbm
