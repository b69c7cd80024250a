// SLLBM step on the D2Q9 velocity set, the standard set the paper compares D2Q25 with in the
// isothermal Taylor-Green study (Sec. III.A): the same pull streaming (Eq. sl_streaming), and
// BGK (Eq. streaming_fg) towards the same fourth-order equilibrium (Sec. II.A) evaluated at
// theta = 1 on the D1Q3 tensor-product nodes 0, +sqrt3, -sqrt3 (weights 2/3, 1/6, 1/6).  On those
// nodes He_3 vanishes and He_4 equals -3 He_2, so the expansion aliases onto lower orders: mass
// and momentum are exact, the third moment misses its u^3 term (the defect in Galilean
// invariance that the comparison shows).
//
// One population (the isothermal configuration) in planar storage, velocity i = 3a + b:
// FP32 / BF16 deviations f_i - w_i with FP32 arithmetic, or FP64 full populations.  One thread
// per vertex gathers the (p+1)^2 stencil of each of the 9 planes through L1/L2 -- with 9 values
// a vertex the tile reuse of shared-memory staging buys little -- then collides in registers.
// Uniform grids read the per-axis tables, transformed grids the per-(velocity, vertex) cells and
// local coordinates.
#include <type_traits>

#include "kernels.h"

namespace sllbm {

namespace {

constexpr int kN1 = 3;          // D1Q3
constexpr int kN = kN1 * kN1;   // D2Q9

template <typename Store>
__device__ __forceinline__ double ld_val(const Store* p) {
  if constexpr (std::is_same<Store, double>::value)
    return __ldg(p);
  else
    return (double)ld_store(p);
}

// Stencil of velocity i at vertex (ix, iy): first node column and row, and the 1D weights.
template <int P, bool Mapped, typename T>
__device__ __forceinline__ void stencil(const StepArgs& a, int i, long long v, int ix, int iy, int* sx,
                                        int* sy, T (&wx)[P + 1], T (&wy)[P + 1]) {
  const int ia = i / kN1, ib = i % kN1;
  if (Mapped) {
    const long long d = (long long)i * a.nv + v;
    *sx = a.dcx[d] * P;
    *sy = a.dcy[d] * P;
    if constexpr (std::is_same<T, double>::value) {
      lagrange_basis<P, double>(a.nodes, a.dr64[d], wx);
      lagrange_basis<P, double>(a.nodes, a.ds64[d], wy);
    } else {
      lagrange_basis<P, float>(a.nodesf, a.dr[d], wx);
      lagrange_basis<P, float>(a.nodesf, a.ds[d], wy);
    }
  } else {
    *sx = ix + a.offx[ia * a.nx + ix];
    *sy = iy + a.offy[ib * a.ny + iy];
#pragma unroll
    for (int k = 0; k <= P; ++k) {
      if constexpr (std::is_same<T, double>::value) {
        wx[k] = a.wx64[(ia * a.nx + ix) * (P + 1) + k];
        wy[k] = a.wy64[(ib * a.ny + iy) * (P + 1) + k];
      } else {
        wx[k] = a.wx[(ia * a.nx + ix) * (P + 1) + k];
        wy[k] = a.wy[(ib * a.ny + iy) * (P + 1) + k];
      }
    }
  }
}

// Equilibrium at theta = 1 (q = 0, so A_k(u) = u^k): f_ab^eq = w_a w_b rho (1 + em1(a, b)) with
// em1(a, b) = sum_{(k,l) != (0,0), k+l <= 4} u_x^k he[k][a] u_y^l he[l][b].
template <typename T>
struct Eq9 {
  T X[4][kN1];   // u_x^k he[k][a], k = 1..4
  T S[5][kN1];   // sum_{l=1..m} u_y^l he[l][b]
};

template <typename T>
__device__ __forceinline__ void eq9_factors(const T (&he)[kQ1][kQ1], T ux, T uy, Eq9<T>& e) {
  const T ax[5] = {T(1), ux, ux * ux, ux * ux * ux, ux * ux * ux * ux};
  const T ay[5] = {T(1), uy, uy * uy, uy * uy * uy, uy * uy * uy * uy};
#pragma unroll
  for (int a = 0; a < kN1; ++a)
#pragma unroll
    for (int k = 1; k <= 4; ++k) e.X[k - 1][a] = ax[k] * he[k][a];
#pragma unroll
  for (int b = 0; b < kN1; ++b) {
    e.S[0][b] = T(0);
#pragma unroll
    for (int m = 1; m <= 4; ++m) e.S[m][b] = e.S[m - 1][b] + ay[m] * he[m][b];
  }
}

template <typename T>
__device__ __forceinline__ T eq9_em1(const Eq9<T>& e, int a, int b) {
  T s = e.S[4][b];
#pragma unroll
  for (int k = 1; k <= 4; ++k) s += e.X[k - 1][a] * (T(1) + e.S[4 - k][b]);
  return s;
}

template <int P, typename Store, bool Mapped>
__global__ void __launch_bounds__(128) step_q9_kernel(const __grid_constant__ StepArgs a) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= a.nv) return;
  const int ix = (int)(v % a.nx), iy = (int)(v / a.nx);
  const Store* src = static_cast<const Store*>(a.src);
  Store* dst = static_cast<Store*>(a.dst);
  const size_t o = (size_t)iy * a.pitch + ix;
  constexpr bool F64 = std::is_same<Store, double>::value;

  if constexpr (F64) {
    // full populations: sum_{a,b} psi_a psi_b f(node(a, b)), moments, BGK
    double f[kN];
#pragma unroll
    for (int i = 0; i < kN; ++i) {
      int sx, sy;
      double wx[P + 1], wy[P + 1];
      stencil<P, Mapped, double>(a, i, v, ix, iy, &sx, &sy, wx, wy);
      const Store* pl = src + (size_t)i * a.plane_stride;
      double acc = 0.0;
#pragma unroll
      for (int kb = 0; kb <= P; ++kb) {
        const size_t r = (size_t)wrap_index(sy + kb, a.ny, a.periodic_y) * a.pitch;
        double ax = 0.0;
#pragma unroll
        for (int ka = 0; ka <= P; ++ka) ax += wx[ka] * ld_val(pl + r + wrap_index(sx + ka, a.nx, a.periodic_x));
        acc += wy[kb] * ax;
      }
      f[i] = acc;
    }
    double rho = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
    for (int i = 0; i < kN; ++i) {
      rho += f[i];
      jx += f[i] * a.cs.xi[i / kN1];
      jy += f[i] * a.cs.xi[i % kN1];
    }
    const double ux = jx / rho, uy = jy / rho;
    Eq9<double> e;
    eq9_factors<double>(a.cs.he, ux, uy, e);
    const double om = a.cp.omega;
#pragma unroll
    for (int i = 0; i < kN; ++i) {
      const int ia = i / kN1, ib = i % kN1;
      const double feq = a.cs.w[ia] * a.cs.w[ib] * rho * (1.0 + eq9_em1<double>(e, ia, ib));
      dst[(size_t)i * a.plane_stride + o] = f[i] - om * (f[i] - feq);
    }
    if (!(rho > 0.0 && isfinite(rho))) atomicOr(a.flag, 1);
  } else {
    // deviations fbar = f - w, FP32; interpolation in difference form (constants exact)
    float fb[kN];
#pragma unroll
    for (int i = 0; i < kN; ++i) {
      int sx, sy;
      float wx[P + 1], wy[P + 1];
      stencil<P, Mapped, float>(a, i, v, ix, iy, &sx, &sy, wx, wy);
      const Store* pl = src + (size_t)i * a.plane_stride;
      int col[P + 1];
#pragma unroll
      for (int k = 0; k <= P; ++k) col[k] = wrap_index(sx + k, a.nx, a.periodic_x);
      float rows[P + 1];
#pragma unroll
      for (int kb = 0; kb <= P; ++kb) {
        const Store* r = pl + (size_t)wrap_index(sy + kb, a.ny, a.periodic_y) * a.pitch;
        const float base = ld_store(r + col[0]);
        float acc = base;
#pragma unroll
        for (int ka = 1; ka <= P; ++ka) acc = fmaf(wx[ka], ld_store(r + col[ka]) - base, acc);
        rows[kb] = acc;
      }
      float acc = rows[0];
#pragma unroll
      for (int kb = 1; kb <= P; ++kb) acc = fmaf(wy[kb], rows[kb] - rows[0], acc);
      fb[i] = acc;
    }
    float drho = 0.f, jx = 0.f, jy = 0.f;
#pragma unroll
    for (int i = 0; i < kN; ++i) {   // sum w = 1 and sum w xi = 0: the moments of fbar
      drho += fb[i];
      jx += fb[i] * a.cs.xif[i / kN1];
      jy += fb[i] * a.cs.xif[i % kN1];
    }
    const float rho = 1.f + drho;
    const float ux = jx / rho, uy = jy / rho;
    Eq9<float> e;
    eq9_factors<float>(a.cs.hef, ux, uy, e);
    const float om = a.cp.omegaf;
    // relax, and sum the residual moments of (f^eq - f) to restore mass and momentum to the
    // rounding of those sums (as in the D2Q25 kernels)
    float r0 = 0.f, r1 = 0.f, r2 = 0.f;
#pragma unroll
    for (int i = 0; i < kN; ++i) {
      const int ia = i / kN1, ib = i % kN1;
      const float w = a.cs.wf[ia] * a.cs.wf[ib];
      const float d = w * (drho + rho * eq9_em1<float>(e, ia, ib)) - fb[i];
      r0 += d;
      r1 += d * a.cs.xif[ia];
      r2 += d * a.cs.xif[ib];
      fb[i] = fmaf(om, d, fb[i]);
    }
    // remove om (r0 + r1 xi_x + r2 xi_y) w_i: sum w = 1, sum w xi xi = I on D2Q9
#pragma unroll
    for (int i = 0; i < kN; ++i) {
      const int ia = i / kN1, ib = i % kN1;
      const float w = a.cs.wf[ia] * a.cs.wf[ib];
      const float val = fb[i] - om * w * (r0 + r1 * a.cs.xif[ia] + r2 * a.cs.xif[ib]);
      st_store(dst + (size_t)i * a.plane_stride + o, val);
    }
    if (!(rho > 0.f && isfinite(rho) && isfinite(ux) && isfinite(uy))) atomicOr(a.flag, 1);
  }
}

template <int P, typename Store>
cudaError_t launch_ps(const StepArgs& a, cudaStream_t s) {
  const int threads = 128;
  const unsigned blocks = (unsigned)((a.nv + threads - 1) / threads);
  if (a.mapped)
    step_q9_kernel<P, Store, true><<<blocks, threads, 0, s>>>(a);
  else
    step_q9_kernel<P, Store, false><<<blocks, threads, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename Store>
cudaError_t launch_store(const StepArgs& a, cudaStream_t s) {
  switch (a.P) {
    case 1: return launch_ps<1, Store>(a, s);
    case 2: return launch_ps<2, Store>(a, s);
    case 3: return launch_ps<3, Store>(a, s);
    case 4: return launch_ps<4, Store>(a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_step_q9(const StepArgs& a, int store, cudaStream_t s) {
  if (a.cs.nq1 != kN1 || a.cp.npop != 1 || a.xs != 1 || a.nv == 0) return cudaErrorInvalidValue;
  switch (store) {
    case kStoreF32: return launch_store<float>(a, s);
    case kStoreBF16: return launch_store<__nv_bfloat16>(a, s);
    case kStoreF64: return launch_store<double>(a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace sllbm
