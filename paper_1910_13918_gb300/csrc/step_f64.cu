// Plain FP64 SLLBM step on full populations: the accuracy and speed baseline of the FP32 paths.
// One thread per vertex; (p+1)^2 gathers per velocity plane from global memory with FP64 weights,
// moments (Sec. II), the fourth-order equilibrium (Sec. II.A) and BGK (Eq. streaming_fg, Pr = 1).
#include "kernels.h"

namespace sllbm {

template <int P, bool Mapped, bool PR>
__global__ void __launch_bounds__(128) step_plain_f64_kernel(const __grid_constant__ StepArgs a) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= a.nv) return;
  const int ix = (int)(v % a.nx), iy = (int)(v / a.nx);
  const double* src = static_cast<const double*>(a.src);
  double* dst = static_cast<double*>(a.dst);
  const int npop = a.cp.npop;
  double f[kQ], g[kQ];
#pragma unroll 1
  for (int i = 0; i < kQ; ++i) {
    const int ia = i / 5, ib = i % 5;
    int sx, sy;
    double wx[P + 1], wy[P + 1];
    if (Mapped) {
      const long long d = (long long)i * a.nv + v;
      sx = a.dcx[d] * P;
      sy = a.dcy[d] * P;
      lagrange_basis<P, double>(a.nodes, a.dr64[d], wx);
      lagrange_basis<P, double>(a.nodes, a.ds64[d], wy);
    } else {
      sx = ix + a.offx[ia * a.nx + ix];
      sy = iy + a.offy[ib * a.ny + iy];
#pragma unroll
      for (int k = 0; k <= P; ++k) {
        wx[k] = a.wx64[(ia * a.nx + ix) * (P + 1) + k];
        wy[k] = a.wy64[(ib * a.ny + iy) * (P + 1) + k];
      }
    }
    double accf = 0.0, accg = 0.0;
    const double* pf = src + (size_t)i * a.plane_stride;
    const double* pg = pf + a.ps;
#pragma unroll
    for (int kb = 0; kb <= P; ++kb) {
      const size_t r = (size_t)wrap_index(sy + kb, a.ny, a.periodic_y) * a.pitch;
      double axf = 0.0, axg = 0.0;
#pragma unroll
      for (int ka = 0; ka <= P; ++ka) {
        const size_t o = r + (size_t)wrap_index(sx + ka, a.nx, a.periodic_x) * a.xs;
        axf += wx[ka] * __ldg(pf + o);
        if (npop == 2) axg += wx[ka] * __ldg(pg + o);
      }
      accf += wy[kb] * axf;
      accg += wy[kb] * axg;
    }
    f[i] = accf;
    g[i] = accg;
  }
  // moments
  double rho = 0.0, jx = 0.0, jy = 0.0, e2 = 0.0;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const double cx = a.cs.xi[i / 5], cy = a.cs.xi[i % 5];
    rho += f[i];
    jx += f[i] * cx;
    jy += f[i] * cy;
    e2 += f[i] * (cx * cx + cy * cy) + (npop == 2 ? g[i] : 0.0);
  }
  const double ux = jx / rho, uy = jy / rho;
  const double theta_k = (e2 - rho * (ux * ux + uy * uy)) / (2.0 * a.cp.cv * rho);
  const double theta = a.cp.iso ? 1.0 : theta_k;
  if (a.mom) {
    const long long v = (long long)iy * a.nx + ix;
    a.mom[v] = (float)rho;
    a.mom[a.nv + v] = (float)ux;
    a.mom[2 * a.nv + v] = (float)uy;
    a.mom[3 * a.nv + v] = (float)theta_k;
  }
  const double q = theta - 1.0;
  EqFactors<double> e;
  eq_factors<double>(a.cs.he, ux, uy, q, e);
  const double om = a.cp.omega;
  const size_t o = (size_t)iy * a.pitch + (size_t)ix * a.xs;
  // Pr != 1 (Sec. II.C): non-equilibrium centred third moments of f and g (xxx, xxy, xyy, yyy)
  double qf[4] = {0.0, 0.0, 0.0, 0.0}, qg[4] = {0.0, 0.0, 0.0, 0.0};
  if (PR) {
#pragma unroll 1
    for (int i = 0; i < kQ; ++i) {
      const int ia = i / 5, ib = i % 5;
      const double feq = a.cs.w[ia] * a.cs.w[ib] * rho * (1.0 + eq_em1<double>(e, ia, ib));
      const double df = f[i] - feq, dg = npop == 2 ? g[i] - a.cp.K * theta * feq : 0.0;
      const double cx = a.cs.xi[ia] - ux, cy = a.cs.xi[ib] - uy;
      const double m[4] = {cx * cx * cx, cx * cx * cy, cx * cy * cy, cy * cy * cy};
      for (int k = 0; k < 4; ++k) {
        qf[k] += df * m[k];
        qg[k] += dg * m[k];
      }
    }
  }
#pragma unroll
  for (int ia = 0; ia < kQ1; ++ia)
#pragma unroll
    for (int ib = 0; ib < kQ1; ++ib) {
      const int i = 5 * ia + ib;
      const double feq = a.cs.w[ia] * a.cs.w[ib] * rho * (1.0 + eq_em1<double>(e, ia, ib));
      // quasi-equilibrium: w_a w_b (Q_xxx h3(a) + Q_xxy h2(a) h1(b) + Q_xyy h1(a) h2(b) + Q_yyy h3(b))
      double sf = 0.0, sg = 0.0;
      if (PR) {
        const double wab = a.cs.w[ia] * a.cs.w[ib];
        const double h[4] = {a.cs.he[3][ia], a.cs.he[2][ia] * a.cs.he[1][ib],
                             a.cs.he[1][ia] * a.cs.he[2][ib], a.cs.he[3][ib]};
        for (int k = 0; k < 4; ++k) {
          sf += qf[k] * h[k];
          sg += qg[k] * h[k];
        }
        sf *= a.cp.cpr * wab;
        sg *= a.cp.cpr * wab;
      }
      dst[(size_t)i * a.plane_stride + o] = f[i] - om * (f[i] - feq) + sf;
      if (npop == 2) {
        const double geq = a.cp.K * theta * feq;
        dst[(size_t)i * a.plane_stride + a.ps + o] = g[i] - om * (g[i] - geq) + sg;
      }
    }
  if (!(rho > 0.0 && theta > 0.0 && isfinite(rho) && isfinite(theta))) atomicOr(a.flag, 1);
}

template <int P>
static cudaError_t launch_p(const StepArgs& a, cudaStream_t s) {
  const int threads = 128;
  const unsigned blocks = (unsigned)((a.nv + threads - 1) / threads);
  if (a.mapped)
    a.cp.pr_on ? step_plain_f64_kernel<P, true, true><<<blocks, threads, 0, s>>>(a)
               : step_plain_f64_kernel<P, true, false><<<blocks, threads, 0, s>>>(a);
  else
    a.cp.pr_on ? step_plain_f64_kernel<P, false, true><<<blocks, threads, 0, s>>>(a)
               : step_plain_f64_kernel<P, false, false><<<blocks, threads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_step_plain_f64(const StepArgs& a, cudaStream_t s) {
  switch (a.P) {
    case 1: return launch_p<1>(a, s);
    case 2: return launch_p<2>(a, s);
    case 3: return launch_p<3>(a, s);
    case 4: return launch_p<4>(a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace sllbm
