// Generic fused SLLBM step, FP32 arithmetic: one thread per vertex gathers the (p+1)^2 stencil of
// every velocity plane straight from global memory (L1/L2 cached), then collides.  The state is
// the interleaved FP32/BF16 layout: each load brings the (f, g) pair of one (velocity, vertex),
// and both populations are interpolated together in packed FP32x2 arithmetic.
//
// Used for transformed grids (per-(velocity, vertex) departure descriptors, Sec. III.E) and for
// uniform grids whose departure offsets exceed the staging halo of the fused uniform kernel.
// Pull streaming of Eq. sl_streaming with the BGK collision of Eq. streaming_fg (Pr = 1).
#include "kernels.h"

namespace sllbm {

template <int P, typename Store, bool Mapped, bool PR>
__global__ void __launch_bounds__(128) step_gather_kernel(const __grid_constant__ StepArgs a) {
  long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (a.vlist) {
    if (v >= a.nlist) return;
    v = a.vlist[v];
  } else if (v >= a.nv) {
    return;
  }
  const int ix = (int)(v % a.nx), iy = (int)(v / a.nx);
  const Store* src = static_cast<const Store*>(a.src);
  Store* dst = static_cast<Store*>(a.dst);
  float2 fg[kQ];   // (f, g) deviations after streaming
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const int ia = i / 5, ib = i % 5;
    int sx, sy;
    float wx[P + 1], wy[P + 1];
    if (Mapped) {
      const long long d = (long long)i * a.nv + v;
      sx = a.dcx[d] * P;
      sy = a.dcy[d] * P;
      lagrange_basis<P, float>(a.nodesf, a.dr[d], wx);
      lagrange_basis<P, float>(a.nodesf, a.ds[d], wy);
    } else {
      sx = ix + a.offx[ia * a.nx + ix];
      sy = iy + a.offy[ib * a.ny + iy];
#pragma unroll
      for (int k = 0; k <= P; ++k) {
        wx[k] = a.wx[(ia * a.nx + ix) * (P + 1) + k];
        wy[k] = a.wy[(ib * a.ny + iy) * (P + 1) + k];
      }
    }
    int col[P + 1];
    long long row[P + 1];
#pragma unroll
    for (int k = 0; k <= P; ++k) {
      col[k] = 2 * wrap_index(sx + k, a.nx, a.periodic_x);
      row[k] = (long long)wrap_index(sy + k, a.ny, a.periodic_y) * a.pitch;
    }
    const Store* pl = src + (size_t)i * a.plane_stride;
    // difference form (see the uniform kernel): constants are reproduced exactly in FP32
    float2 rows[P + 1];
#pragma unroll
    for (int kb = 0; kb <= P; ++kb) {
      const float2 base = ld_pair(pl + row[kb] + col[0]);
      float2 accx = base;
#pragma unroll
      for (int ka = 1; ka <= P; ++ka)
        accx = fma2(bcast2(wx[ka]), sub2(ld_pair(pl + row[kb] + col[ka]), base), accx);
      rows[kb] = accx;
    }
    float2 acc = rows[0];
#pragma unroll
    for (int kb = 1; kb <= P; ++kb) acc = fma2(bcast2(wy[kb]), sub2(rows[kb], rows[0]), acc);
    fg[i] = acc;
  }
  const bool two = a.cp.npop == 2;
  VertexMoments vm;
  const bool ok = collide_deviation_f32<PR>(fg, a.cs, a.cp, vm);
  if (!ok) atomicOr(a.flag, 1);
  if (a.mom) store_moments(a.mom, a.nv, (long long)iy * a.nx + ix, vm);
  if (!two) {   // one population: the g slots stay zero
#pragma unroll
    for (int i = 0; i < kQ; ++i) fg[i].y = 0.f;
  }
  store_images(a.ghost, ix, iy, [&](int xx, int yy) {
    Store* o = dst + (ptrdiff_t)yy * a.pitch + 2 * (ptrdiff_t)xx;
#pragma unroll
    for (int i = 0; i < kQ; ++i, o += a.plane_stride) st_pair(o, fg[i]);
  });
}

template <int P, typename Store, bool PR>
static cudaError_t launch_p(const StepArgs& a, cudaStream_t s) {
  const int threads = 128;
  const long long n = a.vlist ? a.nlist : a.nv;
  if (n == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n + threads - 1) / threads);
  if (a.mapped)
    step_gather_kernel<P, Store, true, PR><<<blocks, threads, 0, s>>>(a);
  else
    step_gather_kernel<P, Store, false, PR><<<blocks, threads, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename Store>
static cudaError_t launch_store(const StepArgs& a, cudaStream_t s) {
  switch (a.P) {
    case 1: return a.cp.pr_on ? launch_p<1, Store, true>(a, s) : launch_p<1, Store, false>(a, s);
    case 2: return a.cp.pr_on ? launch_p<2, Store, true>(a, s) : launch_p<2, Store, false>(a, s);
    case 3: return a.cp.pr_on ? launch_p<3, Store, true>(a, s) : launch_p<3, Store, false>(a, s);
    case 4: return a.cp.pr_on ? launch_p<4, Store, true>(a, s) : launch_p<4, Store, false>(a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_step_gather(const StepArgs& a, int store, cudaStream_t s) {
  if (store == kStoreBF16) return launch_store<__nv_bfloat16>(a, s);
  return launch_store<float>(a, s);
}

}  // namespace sllbm
