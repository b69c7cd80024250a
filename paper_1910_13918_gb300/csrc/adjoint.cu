// Adjoint of one SLLBM step (not part of the paper).  The step is s' = C(S s) with S the
// interpolation of Eq. sl_streaming applied per velocity plane and C the pointwise BGK collision
// of Eq. streaming_fg.  Its adjoint is lambda = S^T J_C^T lambda':
//   * J_C^T at one vertex: J_C = (1 - w) I + w (d eq / d m)(d m / d s), with m the conserved
//     moments (rho, j_x, j_y, 2 rho E), linear in (f, g).  So J_C^T lambda = (1 - w) lambda +
//     w M^T z with z = (dp/dm)^T (d eq/dp)^T lambda, p = (rho, u_x, u_y, theta): four reductions
//     over the 50 populations and a rank-4 update.
//   * S^T as a pull: every target vertex sums over the (vertex, weight) pairs of a precomputed
//     transposed stencil (per axis on uniform grids, per velocity on transformed grids).  No
//     atomics; the summation order is fixed, so results are deterministic.
#include "kernels.h"

namespace sllbm {

// E_ab of the factorised equilibrium and its derivatives with respect to u_x, u_y and q.
template <typename T>
struct EqDerivs {
  T X[5][kQ1], Xu[5][kQ1], Xq[5][kQ1];   // per k, a
  T C[5][kQ1], Cu[5][kQ1], Cq[5][kQ1];   // cumulative over l <= m, per b
};

template <typename T>
__device__ __forceinline__ void eq_derivs(const T (&he)[kQ1][kQ1], T ux, T uy, T q, EqDerivs<T>& d) {
  T A[2][5], Au[2][5], Aq[2][5];
  const T u2[2] = {ux, uy};
#pragma unroll
  for (int ax = 0; ax < 2; ++ax) {
    const T u = u2[ax];
    A[ax][0] = T(1);
    A[ax][1] = u;
    A[ax][2] = u * u + q;
    A[ax][3] = u * u * u + T(3) * u * q;
    A[ax][4] = u * u * u * u + T(6) * u * u * q + T(3) * q * q;
    Au[ax][0] = T(0);
    Au[ax][1] = T(1);
    Au[ax][2] = T(2) * u;
    Au[ax][3] = T(3) * u * u + T(3) * q;
    Au[ax][4] = T(4) * u * u * u + T(12) * u * q;
    Aq[ax][0] = T(0);
    Aq[ax][1] = T(0);
    Aq[ax][2] = T(1);
    Aq[ax][3] = T(3) * u;
    Aq[ax][4] = T(6) * u * u + T(6) * q;
  }
#pragma unroll
  for (int k = 0; k < 5; ++k)
#pragma unroll
    for (int a = 0; a < kQ1; ++a) {
      d.X[k][a] = A[0][k] * he[k][a];
      d.Xu[k][a] = Au[0][k] * he[k][a];
      d.Xq[k][a] = Aq[0][k] * he[k][a];
    }
#pragma unroll
  for (int b = 0; b < kQ1; ++b) {
    T c = T(0), cu = T(0), cq = T(0);
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      c += A[1][m] * he[m][b];
      cu += Au[1][m] * he[m][b];
      cq += Aq[1][m] * he[m][b];
      d.C[m][b] = c;
      d.Cu[m][b] = cu;
      d.Cq[m][b] = cq;
    }
  }
}

// E, dE/du_x, dE/du_y, dE/dq at velocity (a, b).
template <typename T>
__device__ __forceinline__ void eq_point(const EqDerivs<T>& d, int a, int b, T* E, T* Eux, T* Euy,
                                         T* Eq) {
  T e = T(0), eux = T(0), euy = T(0), eq = T(0);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    e += d.X[k][a] * d.C[4 - k][b];
    eux += d.Xu[k][a] * d.C[4 - k][b];
    euy += d.X[k][a] * d.Cu[4 - k][b];
    eq += d.Xq[k][a] * d.C[4 - k][b] + d.X[k][a] * d.Cq[4 - k][b];
  }
  *E = e;
  *Eux = eux;
  *Euy = euy;
  *Eq = eq;
}

__global__ void __launch_bounds__(128) adjoint_collide_kernel(const __grid_constant__ AdjointArgs a) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= a.nv) return;
  const float rho = a.moments[v], ux = a.moments[a.nv + v], uy = a.moments[2 * a.nv + v],
              theta = a.moments[3 * a.nv + v];
  const float q = theta - 1.f, K = a.cp.Kf, cv = a.cp.cvf, om = a.cp.omegaf;
  const bool has_g = a.cp.npop == 2;
  EqDerivs<float> d;
  eq_derivs<float>(a.cs.hef, ux, uy, q, d);
  float yr = 0.f, yux = 0.f, yuy = 0.f, yth = 0.f;
#pragma unroll
  for (int ia = 0; ia < kQ1; ++ia)
#pragma unroll
    for (int ib = 0; ib < kQ1; ++ib) {
      const int i = 5 * ia + ib;
      const float lf = a.lam_in[(size_t)i * a.nv + v];
      const float lg = has_g ? a.lam_in[(size_t)(kQ + i) * a.nv + v] : 0.f;
      float E, Eux, Euy, Eq;
      eq_point<float>(d, ia, ib, &E, &Eux, &Euy, &Eq);
      const float w = a.cs.wf[ia] * a.cs.wf[ib];
      const float L = lf + K * theta * lg;  // d(f^eq, g^eq)/dp contracted with lambda, f^eq part
      yr += L * w * E;
      yux += L * w * rho * Eux;
      yuy += L * w * rho * Euy;
      yth += L * w * rho * Eq + K * lg * w * rho * E;
    }
  // z = (dp/dm)^T y with m = (rho, j_x, j_y, e2), e2 = sum f|xi|^2 + sum g
  const float inv = 1.f / rho;
  const float u2 = ux * ux + uy * uy;
  const float z0 = yr - (yux * ux + yuy * uy) * inv + yth * (-theta + u2 / (2.f * cv)) * inv;
  const float z1 = yux * inv - yth * ux / cv * inv;
  const float z2 = yuy * inv - yth * uy / cv * inv;
  const float z3 = yth / (2.f * cv) * inv;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const float cx = a.cs.xif[i / 5], cy = a.cs.xif[i % 5];
    const float lf = a.lam_in[(size_t)i * a.nv + v];
    a.mu[(size_t)i * a.nv + v] = (1.f - om) * lf + om * (z0 + z1 * cx + z2 * cy + z3 * (cx * cx + cy * cy));
    const float lg = a.lam_in[(size_t)(kQ + i) * a.nv + v];
    a.mu[(size_t)(kQ + i) * a.nv + v] = has_g ? (1.f - om) * lg + om * z3 : 0.f;
  }
}

__global__ void __launch_bounds__(128) adjoint_stream_kernel(const __grid_constant__ AdjointArgs a) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)kQ * a.nv) return;
  const int i = (int)(t / a.nv);
  const long long u = t % a.nv;
  const int ia = i / 5, ib = i % 5;
  float accf = 0.f, accg = 0.f;
  const float* mf = a.mu + (size_t)i * a.nv;
  const float* mg = a.mu + (size_t)(kQ + i) * a.nv;
  if (a.mapped) {
    const long long* ptr = a.tm_ptr + (size_t)i * (a.nv + 1);
    for (long long e = ptr[u]; e < ptr[u + 1]; ++e) {
      const int src = a.tm_col[e];
      accf += a.tm_w[e] * mf[src];
      accg += a.tm_w[e] * mg[src];
    }
  } else {
    const int x = (int)(u % a.nx), y = (int)(u / a.nx);
    const int* px = a.tx_ptr + ia * (a.nx + 1);
    const int* py = a.ty_ptr + ib * (a.ny + 1);
    for (int ey = py[y]; ey < py[y + 1]; ++ey) {
      const float wy = a.ty_w[ey];
      const size_t row = (size_t)a.ty_col[ey] * a.nx;
      float sf = 0.f, sg = 0.f;
      for (int ex = px[x]; ex < px[x + 1]; ++ex) {
        sf += a.tx_w[ex] * mf[row + a.tx_col[ex]];
        sg += a.tx_w[ex] * mg[row + a.tx_col[ex]];
      }
      accf += wy * sf;
      accg += wy * sg;
    }
  }
  a.lam_out[(size_t)i * a.nv + u] = accf;
  a.lam_out[(size_t)(kQ + i) * a.nv + u] = (a.cp.npop == 2) ? accg : 0.f;
}

cudaError_t launch_adjoint_step(const AdjointArgs& a, cudaStream_t s) {
  const int threads = 128;
  adjoint_collide_kernel<<<(unsigned)((a.nv + threads - 1) / threads), threads, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long n = (long long)kQ * a.nv;
  adjoint_stream_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(a);
  return cudaGetLastError();
}

// d/du of <lambda, (f^eq, g^eq)(rho, u, v, theta)> per vertex, in FP64.
__global__ void __launch_bounds__(128) init_vjp_kernel(const __grid_constant__ InitVjpArgs a) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= a.nv) return;
  const double rho = a.rho[v], ux = a.u[v], uy = a.v[v], theta = a.T[v];
  const double K = a.cp.K;
  EqDerivs<double> d;
  eq_derivs<double>(a.cs.he, ux, uy, theta - 1.0, d);
  double du = 0.0, dv = 0.0;
  for (int ia = 0; ia < kQ1; ++ia)
    for (int ib = 0; ib < kQ1; ++ib) {
      const int i = 5 * ia + ib;
      double E, Eux, Euy, Eq;
      eq_point<double>(d, ia, ib, &E, &Eux, &Euy, &Eq);
      const double w = a.cs.w[ia] * a.cs.w[ib];
      const double L = (double)a.lam[(size_t)i * a.nv + v] +
                       (a.cp.npop == 2 ? K * theta * (double)a.lam[(size_t)(kQ + i) * a.nv + v] : 0.0);
      du += L * w * rho * Eux;
      dv += L * w * rho * Euy;
    }
  a.du[v] = (float)du;
  a.dv[v] = (float)dv;
}

cudaError_t launch_init_vjp(const InitVjpArgs& a, cudaStream_t s) {
  const int threads = 128;
  init_vjp_kernel<<<(unsigned)((a.nv + threads - 1) / threads), threads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace sllbm
