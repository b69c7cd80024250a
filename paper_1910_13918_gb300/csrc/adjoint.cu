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

// J_C^T through the Hermite moments of lambda.  With f^eq_ab = rho w_a w_b E_ab and the
// factorised E_ab = sum_{k+l<=4} A_k(u_x) he[k][a] A_l(u_y) he[l][b], every sum over the 25
// velocities of w_a w_b lambda_ab times E_ab or one of its derivatives in u_x, u_y, q is a
// combination of the 15 moments M[k][l] = sum_ab (w_a he[k][a]) (w_b he[l][b]) lambda_ab,
// k + l <= 4, with coefficients from A and its derivatives.  So the four reductions take 2 x 15
// moments (of the f and g adjoints) and a few dozen products, not 25 evaluations of E and three
// derivatives.  Result z = (dp/dm)^T y of the moment covector, scaled by omega.
constexpr int kTri = 15;   // pairs (k, l) with k + l <= 4
__device__ __forceinline__ constexpr int tri(int k, int l) { return k * 5 - k * (k - 1) / 2 + l; }

__device__ __forceinline__ void axis_A(float u, float q, float (&A)[5], float (&Au)[5], float (&Aq)[5]) {
  A[0] = 1.f;
  A[1] = u;
  A[2] = u * u + q;
  A[3] = u * u * u + 3.f * u * q;
  A[4] = u * u * u * u + 6.f * u * u * q + 3.f * q * q;
  Au[0] = 0.f;
  Au[1] = 1.f;
  Au[2] = 2.f * u;
  Au[3] = 3.f * u * u + 3.f * q;
  Au[4] = 4.f * u * u * u + 12.f * u * q;
  Aq[0] = 0.f;
  Aq[1] = 0.f;
  Aq[2] = 1.f;
  Aq[3] = 3.f * u;
  Aq[4] = 6.f * u * u + 6.f * q;
}

// omega z of vertex v (z of Eq. J_C^T: lambda_out = (1 - omega) lambda + omega M^T z).
__device__ __forceinline__ float4 adjoint_z(const AdjointArgs& a, long long v) {
  const float rho = a.moments[v], ux = a.moments[a.nv + v], uy = a.moments[2 * a.nv + v],
              theta = a.moments[3 * a.nv + v];
  const float q = theta - 1.f, K = a.cp.Kf, cv = a.cp.cvf, om = a.cp.omegaf;
  const bool has_g = a.cp.npop == 2;
  float Mf[kTri], Mg[kTri];
#pragma unroll
  for (int t = 0; t < kTri; ++t) Mf[t] = Mg[t] = 0.f;
#pragma unroll
  for (int ia = 0; ia < kQ1; ++ia) {
    float lf[kQ1], lg[kQ1];
#pragma unroll
    for (int ib = 0; ib < kQ1; ++ib) {
      lf[ib] = __ldg(a.lam_in + (size_t)(5 * ia + ib) * a.nv + v);
      lg[ib] = has_g ? __ldg(a.lam_in + (size_t)(kQ + 5 * ia + ib) * a.nv + v) : 0.f;
    }
#pragma unroll
    for (int l = 0; l < 5; ++l) {
      float rf = 0.f, rg = 0.f;
#pragma unroll
      for (int ib = 0; ib < kQ1; ++ib) {
        rf = fmaf(a.cs.whf[l][ib], lf[ib], rf);
        rg = fmaf(a.cs.whf[l][ib], lg[ib], rg);
      }
#pragma unroll
      for (int k = 0; k + l <= 4; ++k) {
        Mf[tri(k, l)] = fmaf(a.cs.whf[k][ia], rf, Mf[tri(k, l)]);
        Mg[tri(k, l)] = fmaf(a.cs.whf[k][ia], rg, Mg[tri(k, l)]);
      }
    }
  }
  float Ax[5], Aux[5], Aqx[5], Ay[5], Auy[5], Aqy[5];
  axis_A(ux, q, Ax, Aux, Aqx);
  axis_A(uy, q, Ay, Auy, Aqy);
  // y = sum_ab w_a w_b L_ab (E, rho dE/du_x, rho dE/du_y, rho dE/dq) + K rho sum w_a w_b lambda^g E,
  // with L = lambda^f + K theta lambda^g, contracted along l first
  float yE = 0.f, yux = 0.f, yuy = 0.f, yq = 0.f, yg = 0.f;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    float sy = 0.f, suy = 0.f, sqy = 0.f, sg = 0.f;
#pragma unroll
    for (int l = 0; k + l <= 4; ++l) {
      const float mL = fmaf(K * theta, Mg[tri(k, l)], Mf[tri(k, l)]);
      sy = fmaf(Ay[l], mL, sy);
      suy = fmaf(Auy[l], mL, suy);
      sqy = fmaf(Aqy[l], mL, sqy);
      sg = fmaf(Ay[l], Mg[tri(k, l)], sg);
    }
    yE = fmaf(Ax[k], sy, yE);
    yux = fmaf(Aux[k], sy, yux);
    yuy = fmaf(Ax[k], suy, yuy);
    yq = fmaf(Aqx[k], sy, fmaf(Ax[k], sqy, yq));
    yg = fmaf(Ax[k], sg, yg);
  }
  const float yr = yE;
  yux *= rho;
  yuy *= rho;
  const float yth = rho * (yq + K * yg);
  // z = (dp/dm)^T y with m = (rho, j_x, j_y, e2), e2 = sum f|xi|^2 + sum g
  const float inv = 1.f / rho;
  const float u2 = ux * ux + uy * uy;
  const float z0 = yr - (yux * ux + yuy * uy) * inv + yth * (-theta + u2 / (2.f * cv)) * inv;
  const float z1 = yux * inv - yth * ux / cv * inv;
  const float z2 = yuy * inv - yth * uy / cv * inv;
  const float z3 = yth / (2.f * cv) * inv;
  return make_float4(om * z0, om * z1, om * z2, om * z3);
}

// (f, g) of J_C^T lambda at velocity (cx, cy) from lambda and omega z.
__device__ __forceinline__ float2 adjoint_mu(float lf, float lg, float4 z, float om1, float cx,
                                             float cy, float c2, bool has_g) {
  return make_float2(fmaf(om1, lf, fmaf(c2, z.w, fmaf(cy, z.z, fmaf(cx, z.y, z.x)))),
                     has_g ? fmaf(om1, lg, z.w) : 0.f);
}

// J_C^T of every vertex: omega z into a.z (the one-pass S^T forms the (f, g) pairs itself), or,
// with kWriteMu, the 25 (f, g) pairs into a.mu for the two-pass and mapped S^T.
template <bool kWriteMu>
__global__ void __launch_bounds__(128, 8) adjoint_collide_kernel(const __grid_constant__ AdjointArgs a) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= a.nv) return;
  const float4 z = adjoint_z(a, v);
  if (!kWriteMu) {
    a.z[v] = z;
    return;
  }
  const bool has_g = a.cp.npop == 2;
  const float om1 = 1.f - a.cp.omegaf;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const float cx = a.cs.xif[i / 5], cy = a.cs.xif[i % 5];
    const float lf = __ldg(a.lam_in + (size_t)i * a.nv + v);
    const float lg = has_g ? __ldg(a.lam_in + (size_t)(kQ + i) * a.nv + v) : 0.f;
    a.mu[(size_t)i * a.nv + v] = adjoint_mu(lf, lg, z, om1, cx, cy, cx * cx + cy * cy, has_g);
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

// S^T on a uniform grid in one pass, with J_C^T folded into its loads: a block takes a 32 x 32
// tile of target vertices of one velocity plane and forms the (f, g) pairs of J_C^T lambda on the
// source region the transposed stencils reach (the tile and a halo of H vertices on every side,
// wrapped on periodic axes) from lambda and omega z as it loads them into shared memory; then it
// applies the x stencils to every row of the region and the y stencils to the tile.  Each warp
// loads its region rows with all loads in flight at once (lane = column).  The velocity plane is
// the fastest grid index, so the 25 blocks of one tile run close together and read z from L2.
// The entries of each stencil are those of the two-pass form, summed in the same order.
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
__global__ void __launch_bounds__(256, 3) adjoint_stream_fused_kernel(const __grid_constant__ AdjointArgs a) {
  constexpr int RX = kAT + 2 * H, RY = kAT + 2 * H, NR = RY / 8;
  static_assert(RY % 8 == 0 && 2 * H <= 32, "region rows per warp, second column segment");
  __shared__ float2 Sm[RY][RX];    // J_C^T lambda on the source region: rows y0-H.., columns x0-H..
  __shared__ float2 Tm[RY][kAT];   // after the x stencils
  __shared__ int Yo[kAT][KW];      // y stencils of the tile's rows: source row - target row
  __shared__ float Yw[kAT][KW];
  __shared__ int Yd[kAT];
  const int i = blockIdx.x, ia = i / 5, ib = i % 5;
  const int x0 = blockIdx.y * kAT, y0 = blockIdx.z * kAT;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool has_g = a.cp.npop == 2;
  const float* lfp = a.lam_in + (size_t)i * a.nv;
  const float* lgp = a.lam_in + (size_t)(has_g ? kQ + i : i) * a.nv;
  // this lane's region columns: H + lane - H.. and, for the first 2H lanes, the last 2H columns
  const bool two = lane < 2 * H;
  const int gxa = wrap_or_clamp(x0 - H + lane, a.nx, a.periodic_x);
  const int gxb = wrap_or_clamp(x0 - H + kAT + (two ? lane : 0), a.nx, a.periodic_x);
  float fa[NR], ga[NR], fb[NR], gb[NR];
  float4 za[NR], zb[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    const size_t row = (size_t)wrap_or_clamp(y0 - H + warp + 8 * j, a.ny, a.periodic_y) * a.nx;
    fa[j] = __ldg(lfp + row + gxa);
    ga[j] = __ldg(lgp + row + gxa);
    za[j] = __ldg(a.z + row + gxa);
    if (two) {
      fb[j] = __ldg(lfp + row + gxb);
      gb[j] = __ldg(lgp + row + gxb);
      zb[j] = __ldg(a.z + row + gxb);
    }
  }
  const float om1 = 1.f - a.cp.omegaf, cx = a.cs.xif[ia], cy = a.cs.xif[ib], c2 = cx * cx + cy * cy;
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    Sm[warp + 8 * j][lane] = adjoint_mu(fa[j], ga[j], za[j], om1, cx, cy, c2, has_g);
    if (two) Sm[warp + 8 * j][kAT + lane] = adjoint_mu(fb[j], gb[j], zb[j], om1, cx, cy, c2, has_g);
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
  const int u = x0 + lane;
  int xo[KW];
  float xw[KW];
  const int xdeg = u < a.nx ? __ldg(a.tx_deg + (size_t)ia * a.nx + u) : 0;
#pragma unroll
  for (int k = 0; k < KW; ++k) {
    const bool on = k < xdeg;
    const size_t q = ((size_t)ia * a.nx + (on ? u : 0)) * KW + k;
    xo[k] = H + lane + (on ? __ldg(a.tx_rel + q) : 0);
    xw[k] = on ? __ldg(a.tx_w + q) : 0.f;
  }
  __syncthreads();
  for (int r = warp; r < RY; r += 8) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < KW; ++k)
      if (k < xdeg) acc = fma2(bcast2(xw[k]), Sm[r][xo[k]], acc);
    Tm[r][lane] = acc;
  }
  __syncthreads();
  if (u >= a.nx) return;
  for (int rr = warp; rr < kAT; rr += 8) {
    const int w = y0 + rr;
    if (w >= a.ny) break;
    const int deg = Yd[rr];
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < KW; ++k)
      if (k < deg) acc = fma2(bcast2(Yw[rr][k]), Tm[H + rr + Yo[rr][k]][lane], acc);
    const size_t t = (size_t)w * a.nx + u;
    a.lam_out[(size_t)i * a.nv + t] = acc.x;
    a.lam_out[(size_t)(kQ + i) * a.nv + t] = has_g ? acc.y : 0.f;
  }
}

template <int KW>
static void launch_fused_kw(const AdjointArgs& a, cudaStream_t s) {
  const dim3 grid(kQ, (unsigned)((a.nx + kAT - 1) / kAT), (unsigned)((a.ny + kAT - 1) / kAT));
  if (a.halo <= 4)
    adjoint_stream_fused_kernel<KW, 4><<<grid, 256, 0, s>>>(a);
  else
    adjoint_stream_fused_kernel<KW, 8><<<grid, 256, 0, s>>>(a);
}

bool adjoint_fused_usable(int nx, int ny, int halo) {
  return halo <= 8 && (nx + kAT - 1) / kAT <= 65535 && (ny + kAT - 1) / kAT <= 65535;
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
  const unsigned cblocks = (unsigned)((a.nv + 127) / 128);
  const bool fused = !a.mapped && a.z;   // the host gives z exactly when the one-pass S^T fits
  if (fused)
    adjoint_collide_kernel<false><<<cblocks, 128, 0, s>>>(a);
  else
    adjoint_collide_kernel<true><<<cblocks, 128, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((a.nx + 255) / 256), (unsigned)(a.ny < 65535 ? a.ny : 65535), kQ);
  if (a.mapped) {
    adjoint_stream_mapped_kernel<<<grid, 256, 0, s>>>(a);
  } else if (fused) {
    if (!adjoint_fused_usable(a.nx, a.ny, a.halo)) return cudaErrorInvalidValue;
    switch (a.kw) {   // one pass: J_C^T pairs, x and y stencils through shared memory
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
