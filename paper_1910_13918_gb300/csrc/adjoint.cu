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

__global__ void __launch_bounds__(128, 4) adjoint_collide_kernel(const __grid_constant__ AdjointArgs a) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= a.nv) return;
  const float rho = a.moments[v], ux = a.moments[a.nv + v], uy = a.moments[2 * a.nv + v],
              theta = a.moments[3 * a.nv + v];
  const float q = theta - 1.f, K = a.cp.Kf, cv = a.cp.cvf, om = a.cp.omegaf;
  const bool has_g = a.cp.npop == 2;
  EqDerivs<float> d;
  eq_derivs<float>(a.cs.hef, ux, uy, q, d);
  // the vertex's 50 adjoint values, read once and kept in registers for both passes below
  float lfv[kQ], lgv[kQ];
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    lfv[i] = __ldg(a.lam_in + (size_t)i * a.nv + v);
    lgv[i] = has_g ? __ldg(a.lam_in + (size_t)(kQ + i) * a.nv + v) : 0.f;
  }
  float yr = 0.f, yux = 0.f, yuy = 0.f, yth = 0.f;
#pragma unroll
  for (int ia = 0; ia < kQ1; ++ia)
#pragma unroll
    for (int ib = 0; ib < kQ1; ++ib) {
      const int i = 5 * ia + ib;
      const float lf = lfv[i];
      const float lg = lgv[i];
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
    const float lf = lfv[i];
    const float lg = lgv[i];
    a.mu[(size_t)i * a.nv + v] =
        make_float2((1.f - om) * lf + om * (z0 + z1 * cx + z2 * cy + z3 * (cx * cx + cy * cy)),
                    has_g ? (1.f - om) * lg + om * z3 : 0.f);
  }
}

// S^T on a uniform grid, separable like S: first along x (thread = plane, row, target column:
// the entries of the column's transposed x stencil), then along y into lambda (thread = plane,
// target row, column).  Each pass reads its entries from one row / one column of the plane.
// Grid of the streaming kernels: x = blockIdx.x * 256 + threadIdx.x, plane i = blockIdx.z, rows
// y = blockIdx.y, + gridDim.y, ... (no integer division per thread).
template <int KW>
__global__ void __launch_bounds__(256) adjoint_stream_x_kernel(const __grid_constant__ AdjointArgs a) {
  const int x = blockIdx.x * 256 + threadIdx.x, i = blockIdx.z, ia = i / 5;
  if (x >= a.nx) return;
  // the column's transposed x stencil, once for all the rows this thread does
  const size_t e0 = ((size_t)ia * a.nx + x) * a.kw;
  const int deg = __ldg(a.tx_deg + (size_t)ia * a.nx + x);
  int col[KW];
  float w[KW];
#pragma unroll
  for (int k = 0; k < KW; ++k) {
    col[k] = k < deg ? __ldg(a.tx_col + e0 + k) : x;
    w[k] = k < deg ? __ldg(a.tx_w + e0 + k) : 0.f;
  }
  for (int y = blockIdx.y; y < a.ny; y += gridDim.y) {
    const size_t row = (size_t)i * a.nv + (size_t)y * a.nx;
    const float2* mrow = a.mu + row;
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < KW; ++k)
      if (k < deg) acc = fma2(bcast2(w[k]), __ldg(mrow + col[k]), acc);
    a.tmp[row + x] = acc;
  }
}

template <int KW>
__global__ void __launch_bounds__(256) adjoint_stream_y_kernel(const __grid_constant__ AdjointArgs a) {
  const int x = blockIdx.x * 256 + threadIdx.x, i = blockIdx.z, ib = i % 5;
  if (x >= a.nx) return;
  const float2* colp = a.tmp + (size_t)i * a.nv + x;
  for (int y = blockIdx.y; y < a.ny; y += gridDim.y) {
    // the row's transposed y stencil: KW entries in 16-byte rows (the same for the whole block)
    const size_t e0 = ((size_t)ib * a.ny + y) * KW;
    const int deg = __ldg(a.ty_deg + (size_t)ib * a.ny + y);
    int row[KW];
    float w[KW];
#pragma unroll
    for (int k = 0; k < KW; k += 4) {
      const int4 c4 = __ldg(reinterpret_cast<const int4*>(a.ty_col + e0 + k));
      const float4 w4 = __ldg(reinterpret_cast<const float4*>(a.ty_w + e0 + k));
      row[k] = c4.x; row[k + 1] = c4.y; row[k + 2] = c4.z; row[k + 3] = c4.w;
      w[k] = w4.x; w[k + 1] = w4.y; w[k + 2] = w4.z; w[k + 3] = w4.w;
    }
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < KW; ++k)
      if (k < deg) acc = fma2(bcast2(w[k]), __ldg(colp + (size_t)row[k] * a.nx), acc);
    const size_t u = (size_t)y * a.nx + x;
    a.lam_out[(size_t)i * a.nv + u] = acc.x;
    a.lam_out[(size_t)(kQ + i) * a.nv + u] = (a.cp.npop == 2) ? acc.y : 0.f;
  }
}

// S^T on a uniform grid in one pass: a block takes a 32 x 32 tile of target vertices of one
// velocity plane, loads the source region the transposed stencils reach (the tile and a halo of
// H vertices on every side, wrapped on periodic axes) into shared memory, applies the x stencils
// to every row of the region, then the y stencils to the tile.  Small blocks (one plane, few
// registers) keep eight of them resident per SM, which hides the region loads.  The entries of each stencil are
// the same as in the two-pass form and summed in the same order.
constexpr int kAT = 32;   // target tile edge of the fused S^T

// Index of region row/column j on an axis of n vertices: wrapped on periodic axes (the region
// may reach several periods round on very small grids), clamped otherwise (clamped cells are
// loaded but never read: transposed stencils of non-periodic axes stay inside the axis).
__device__ __forceinline__ int wrap_or_clamp(int j, int n, int periodic) {
  if (periodic) {
    if (j < 0) j += n;
    if (j >= n) j -= n;
    if (j < 0 || j >= n) j = ((j % n) + n) % n;   // grids smaller than the region
    return j;
  }
  return j < 0 ? 0 : (j >= n ? n - 1 : j);
}

template <int KW, int H>
__global__ void __launch_bounds__(256) adjoint_stream_fused_kernel(const __grid_constant__ AdjointArgs a) {
  constexpr int RX = kAT + 2 * H, RY = kAT + 2 * H;
  __shared__ float2 Sm[RY][RX];    // source region: rows y0-H.., columns x0-H..
  __shared__ float2 Tm[RY][kAT];   // after the x stencils
  __shared__ int Yo[kAT][KW];      // y stencils of the tile's rows: source row - target row
  __shared__ float Yw[kAT][KW];
  __shared__ int Yd[kAT];
  const int i = blockIdx.z, ia = i / 5, ib = i % 5;
  const int x0 = blockIdx.x * kAT, y0 = blockIdx.y * kAT;
  const float2* m = a.mu + (size_t)i * a.nv;
  for (int e = threadIdx.x; e < RX * RY; e += 256) {
    const int r = e / RX, cc = e - r * RX;
    const int gy = wrap_or_clamp(y0 - H + r, a.ny, a.periodic_y);
    const int gx = wrap_or_clamp(x0 - H + cc, a.nx, a.periodic_x);
    Sm[r][cc] = __ldg(m + (size_t)gy * a.nx + gx);
  }
  for (int e = threadIdx.x; e < kAT * KW; e += 256) {
    const int rr = e / KW, k = e - rr * KW, w = y0 + rr;
    if (w < a.ny) {
      const size_t q = ((size_t)ib * a.ny + w) * KW + k;
      Yo[rr][k] = __ldg(a.ty_rel + q);
      Yw[rr][k] = __ldg(a.ty_w + q);
      if (k == 0) Yd[rr] = __ldg(a.ty_deg + (size_t)ib * a.ny + w);
    }
  }
  // the target column's transposed x stencil, as positions in a region row
  const int c = threadIdx.x & 31, u = x0 + c;
  int xo[KW];
  float xw[KW];
  const int xdeg = u < a.nx ? __ldg(a.tx_deg + (size_t)ia * a.nx + u) : 0;
#pragma unroll
  for (int k = 0; k < KW; ++k) {
    const bool on = k < xdeg;
    const size_t q = ((size_t)ia * a.nx + (on ? u : 0)) * KW + k;
    xo[k] = H + c + (on ? __ldg(a.tx_rel + q) : 0);
    xw[k] = on ? __ldg(a.tx_w + q) : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.x >> 5; r < RY; r += 8) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < KW; ++k)
      if (k < xdeg) acc = fma2(bcast2(xw[k]), Sm[r][xo[k]], acc);
    Tm[r][c] = acc;
  }
  __syncthreads();
  if (u >= a.nx) return;
  for (int rr = threadIdx.x >> 5; rr < kAT; rr += 8) {
    const int w = y0 + rr;
    if (w >= a.ny) break;
    const int deg = Yd[rr];
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < KW; ++k)
      if (k < deg) acc = fma2(bcast2(Yw[rr][k]), Tm[H + rr + Yo[rr][k]][c], acc);
    const size_t t = (size_t)w * a.nx + u;
    a.lam_out[(size_t)i * a.nv + t] = acc.x;
    a.lam_out[(size_t)(kQ + i) * a.nv + t] = (a.cp.npop == 2) ? acc.y : 0.f;
  }
}

template <int KW>
static void launch_fused_kw(const AdjointArgs& a, cudaStream_t s) {
  const dim3 grid((unsigned)((a.nx + kAT - 1) / kAT), (unsigned)((a.ny + kAT - 1) / kAT), kQ);
  if (a.halo <= 4)
    adjoint_stream_fused_kernel<KW, 4><<<grid, 256, 0, s>>>(a);
  else
    adjoint_stream_fused_kernel<KW, 8><<<grid, 256, 0, s>>>(a);
}

// S^T on a mapped grid: CSR over the target vertex, per velocity.
__global__ void __launch_bounds__(256) adjoint_stream_mapped_kernel(const __grid_constant__ AdjointArgs a) {
  const int x = blockIdx.x * 256 + threadIdx.x, i = blockIdx.z;
  if (x >= a.nx) return;
  const float2* m = a.mu + (size_t)i * a.nv;
  const long long* ptr = a.tm_ptr + (size_t)i * (a.nv + 1);
  for (int y = blockIdx.y; y < a.ny; y += gridDim.y) {
    const long long u = (long long)y * a.nx + x;
    float2 acc = make_float2(0.f, 0.f);
    for (long long e = ptr[u]; e < ptr[u + 1]; ++e) acc = fma2(bcast2(a.tm_w[e]), __ldg(m + a.tm_col[e]), acc);
    a.lam_out[(size_t)i * a.nv + u] = acc.x;
    a.lam_out[(size_t)(kQ + i) * a.nv + u] = (a.cp.npop == 2) ? acc.y : 0.f;
  }
}

cudaError_t launch_adjoint_step(const AdjointArgs& a, cudaStream_t s) {
  adjoint_collide_kernel<<<(unsigned)((a.nv + 127) / 128), 128, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((a.nx + 255) / 256), (unsigned)(a.ny < 65535 ? a.ny : 65535), kQ);
  if (a.mapped) {
    adjoint_stream_mapped_kernel<<<grid, 256, 0, s>>>(a);
  } else if (a.halo <= 8 && (a.ny + kAT - 1) / kAT <= 65535) {
    switch (a.kw) {   // one pass: x and y stencils through shared memory
      case 4: launch_fused_kw<4>(a, s); break;
      case 8: launch_fused_kw<8>(a, s); break;
      case 12: launch_fused_kw<12>(a, s); break;
      case 16: launch_fused_kw<16>(a, s); break;
      default: return cudaErrorInvalidValue;
    }
  } else {
    const dim3 gx(grid.x, (unsigned)((a.ny + 15) / 16 < 65535 ? (a.ny + 15) / 16 : 65535), kQ);
    switch (a.kw) {   // x: 16 rows per thread, the column's stencil loaded once
      case 4: adjoint_stream_x_kernel<4><<<gx, 256, 0, s>>>(a); adjoint_stream_y_kernel<4><<<grid, 256, 0, s>>>(a); break;
      case 8: adjoint_stream_x_kernel<8><<<gx, 256, 0, s>>>(a); adjoint_stream_y_kernel<8><<<grid, 256, 0, s>>>(a); break;
      case 12: adjoint_stream_x_kernel<12><<<gx, 256, 0, s>>>(a); adjoint_stream_y_kernel<12><<<grid, 256, 0, s>>>(a); break;
      case 16: adjoint_stream_x_kernel<16><<<gx, 256, 0, s>>>(a); adjoint_stream_y_kernel<16><<<grid, 256, 0, s>>>(a); break;
      default: return cudaErrorInvalidValue;
    }
  }
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
