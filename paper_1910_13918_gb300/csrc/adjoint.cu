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
#include <atomic>

#include "tma.cuh"

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

// J_C^T of every vertex: the 25 (f, g) pairs into mu, [25][mu_rows][mu_pitch] with mu_g ghost
// columns and rows before the interior origin.  With ghost cells (the one-pass S^T), a vertex
// within mu_g of a periodic edge also writes its periodic images there, so that the S^T regions
// never wrap; the ghosts of non-periodic axes stay zero (never read).
__global__ void __launch_bounds__(128, 7) adjoint_collide_kernel(const __grid_constant__ AdjointArgs a) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= a.nv) return;
  const float4 z = adjoint_z(a, v);
  const bool has_g = a.cp.npop == 2;
  const float om1 = 1.f - a.cp.omegaf;
  const int y = (int)(v / a.nx), x = (int)(v - (long long)y * a.nx), G = a.mu_g;
  // the image column / row (the vertex's own when it has none); grids with ghosts have nx, ny >= 2G
  int xi = x, yi = y;
  if (G > 0 && a.periodic_x) xi = x < G ? x + a.nx : (x >= a.nx - G ? x - a.nx : x);
  if (G > 0 && a.periodic_y) yi = y < G ? y + a.ny : (y >= a.ny - G ? y - a.ny : y);
  const size_t plane = (size_t)a.mu_rows * a.mu_pitch;
  float2* m = a.mu + (size_t)(G + y) * a.mu_pitch + (G + x);   // this vertex in plane 0
  const int dx = xi - x, dy = (yi - y) * a.mu_pitch;           // to its images
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const float cx = a.cs.xif[i / 5], cy = a.cs.xif[i % 5];
    const float lf = __ldg(a.lam_in + (size_t)i * a.nv + v);
    const float lg = has_g ? __ldg(a.lam_in + (size_t)(kQ + i) * a.nv + v) : 0.f;
    const float2 mu = adjoint_mu(lf, lg, z, om1, cx, cy, cx * cx + cy * cy, has_g);
    float2* mi = m + (size_t)i * plane;
    *mi = mu;
    if (dx) mi[dx] = mu;
    if (dy) {
      mi[dy] = mu;
      if (dx) mi[dy + dx] = mu;
    }
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

// S^T on a uniform grid in one pass, persistent CTAs with Tensor Memory Accelerator staging.
// A work item is a tile of 32 x TY target vertices of one velocity plane.  Its source region (the
// tile and a halo of H vertices on every side) arrives as one tensor copy of the ghost-padded
// pairs, and the dense y stencils of its rows as one bulk copy, both on the stage's mbarrier,
// issued NS - 1 items ahead into a ring of NS stages so that the copies overlap the stencil work
// of earlier items.  Items are ordered plane by plane, so the CTAs at work share the halos of
// neighbouring tiles in L2.  The transposed stencils are taken dense by offset d in [-H, H] (zero
// weights where a stencil has no entry), so that each thread slides a register window over the
// region: in the x pass a half-warp takes a region row, a lane two neighbouring target columns
// (2H + 2 pairs read as H + 1 16-byte loads); in the y pass a warp takes TY / 8 neighbouring
// target rows, a lane one column.  TY makes both passes split evenly over the 8 warps.
constexpr int kATX = 32;        // target tile width
constexpr int kAdjNT = 256;     // threads of a CTA
constexpr int kAdjStages = 2;   // stages of the copy ring

template <int H, int NS>
struct AdjTmaShape {
  static constexpr int TY = H == 4 ? 40 : 32;   // target rows: (TY + 2H) / 2 row pairs = 3 per warp
  static constexpr int RX = kATX + 2 * H, RY = TY + 2 * H, RE = RX * RY;
  static constexpr int D = 2 * H + 1, DW = (D + 3) / 4 * 4;   // offsets; dense row width
  static constexpr int RPW = RY / 2 / (kAdjNT / 32), YPW = TY / (kAdjNT / 32);
  // a stage: the region's pairs [RY][RX], then the dense y stencils of the tile's rows [TY][DW]
  static constexpr size_t kStage = sizeof(float2) * RE + sizeof(float) * ((TY * DW + 31) / 32 * 32);
  static constexpr size_t kBytes = 128 + NS * kStage + sizeof(float2) * RY * kATX + sizeof(uint64_t) * NS;
  static_assert(RY % (2 * (kAdjNT / 32)) == 0 && TY % (kAdjNT / 32) == 0, "even split over the warps");
  static_assert((sizeof(float2) * RE) % 128 == 0 && kStage % 128 == 0, "128-byte aligned copies");
};

// (plane, tile column, tile row) of a CTA's items, stepped by the grid size without divisions.
struct AdjCursor {
  int i, tx, ty;
  __device__ __forceinline__ void init(int item, int ntiles, int tiles_x) {
    i = item / ntiles;
    const int t = item - i * ntiles;
    ty = t / tiles_x;
    tx = t - ty * tiles_x;
  }
  __device__ __forceinline__ void next(int sx, int sy, int tiles_x, int tiles_y) {
    tx += sx;
    ty += sy;
    if (tx >= tiles_x) {
      tx -= tiles_x;
      ++ty;
    }
    while (ty >= tiles_y) {
      ty -= tiles_y;
      ++i;
    }
  }
};

// The copies of one item into a stage, completing on bar.
template <int H, int NS>
__device__ __forceinline__ void adj_issue(const AdjointArgs& a, const CUtensorMap& mmap, unsigned char* stage,
                                          uint64_t* bar, const AdjCursor& c) {
  using SH = AdjTmaShape<H, NS>;
  const int x0 = c.tx * kATX, y0 = c.ty * SH::TY, ib = c.i % 5;
  const int rows = a.ny - y0 < SH::TY ? a.ny - y0 : SH::TY;
  const unsigned wy_bytes = (unsigned)(rows * SH::DW * sizeof(float));   // a multiple of 16
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  mbar_expect_tx(bar, (unsigned)(SH::RE * sizeof(float2)) + wy_bytes);
  // x in floats: 2 (mu_g + x0 - H), a multiple of 4 (16 bytes) as mu_g, x0 and H are even
  tma_load_3d(stage, &mmap, 2 * (a.mu_g + x0 - H), a.mu_g + y0 - H, c.i, bar);
  bulk_load(stage + SH::RE * sizeof(float2), a.ty_dense + ((size_t)ib * a.ny + y0) * SH::DW, wy_bytes, bar);
}

template <int H, int NS>
__global__ void __launch_bounds__(kAdjNT, 4) adjoint_stream_tma_kernel(const __grid_constant__ AdjointArgs a,
                                                                       const __grid_constant__ CUtensorMap mmap) {
  using SH = AdjTmaShape<H, NS>;
  constexpr int RX = SH::RX, RY = SH::RY, RE = SH::RE, D = SH::D, DW = SH::DW, TY = SH::TY;
  extern __shared__ unsigned char adj_smem[];
  unsigned char* base = adj_smem + ((128 - (smem_u32(adj_smem) & 127)) & 127);
  float2* Tm = reinterpret_cast<float2*>(base + NS * SH::kStage);   // [RY][kATX], after the x stencils
  uint64_t* BAR = reinterpret_cast<uint64_t*>(Tm + RY * kATX);      // [NS]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int half = lane >> 4, cp2 = 2 * (lane & 15);                // x pass: row of the pair, column pair
  const int tiles_x = (a.nx + kATX - 1) / kATX, tiles_y = (a.ny + TY - 1) / TY, ntiles = tiles_x * tiles_y;
  const int my = (kQ * ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int sx = (int)gridDim.x % tiles_x, sy = (int)gridDim.x / tiles_x;
  const bool has_g = a.cp.npop == 2;
  if (tid == 0) {
    for (int k = 0; k < NS; ++k) mbar_init(&BAR[k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  AdjCursor cur, nxt;   // the item in work; (thread 0) the next item to copy
  cur.init((int)blockIdx.x, ntiles, tiles_x);
  nxt = cur;
  if (tid == 0)
    for (int k = 0; k < NS - 1 && k < my; ++k) {
      adj_issue<H, NS>(a, mmap, base + k * SH::kStage, &BAR[k], nxt);
      nxt.next(sx, sy, tiles_x, tiles_y);
    }
#pragma unroll 1
  for (int k = 0; k < my; ++k) {
    if (k > 0) cur.next(sx, sy, tiles_x, tiles_y);
    const int st = k % NS, i = cur.i, ia = i / 5;
    const int x0 = cur.tx * kATX, y0 = cur.ty * TY;
    // dense x stencils of this lane's two target columns (past the grid's last column, that
    // column's: the outputs of those columns are not stored)
    float wx0[D], wx1[D];
    {
      const int u0 = x0 + cp2;
      const float* w0 = a.tx_dense + ((size_t)ia * a.nx + (u0 < a.nx ? u0 : a.nx - 1)) * DW;
      const float* w1 = a.tx_dense + ((size_t)ia * a.nx + (u0 + 1 < a.nx ? u0 + 1 : a.nx - 1)) * DW;
#pragma unroll
      for (int q = 0; q < DW; q += 4) {
        const float4 v0 = __ldg(reinterpret_cast<const float4*>(w0 + q));
        const float4 v1 = __ldg(reinterpret_cast<const float4*>(w1 + q));
        const float e0[4] = {v0.x, v0.y, v0.z, v0.w}, e1[4] = {v1.x, v1.y, v1.z, v1.w};
#pragma unroll
        for (int m = 0; m < 4; ++m)
          if (q + m < D) {
            wx0[q + m] = e0[m];
            wx1[q + m] = e1[m];
          }
      }
    }
    const bool late = !mbar_wait(&BAR[st], (unsigned)((k / NS) & 1), a.flag);
    if (__syncthreads_or(late)) {
      // a copy did not land in time: every thread stops, after waiting (bounded) for the copies
      // still in flight into this CTA's stages
      for (int t2 = k; t2 < k + NS - 1 && t2 < my; ++t2)
        if (!mbar_wait(&BAR[t2 % NS], (unsigned)((t2 / NS) & 1), a.flag)) break;
      return;
    }
    // every thread is past item k - 1: its stage takes item k + NS - 1
    if (tid == 0 && k + NS - 1 < my) {
      const int sn = (k + NS - 1) % NS;
      adj_issue<H, NS>(a, mmap, base + sn * SH::kStage, &BAR[sn], nxt);
      nxt.next(sx, sy, tiles_x, tiles_y);
    }
    const float2* Sm = reinterpret_cast<const float2*>(base + st * SH::kStage);
    const float* Wy = reinterpret_cast<const float*>(Sm + RE);
    // x pass: target columns cp2, cp2 + 1 of region row r read region columns cp2 .. cp2 + 2H + 1
#pragma unroll
    for (int j = 0; j < SH::RPW; ++j) {
      const int r = 2 * (warp + j * (kAdjNT / 32)) + half;
      const float4* src = reinterpret_cast<const float4*>(Sm + r * RX + cp2);
      float2 win[2 * H + 2];
#pragma unroll
      for (int m = 0; m <= H; ++m) {
        const float4 q = src[m];
        win[2 * m] = make_float2(q.x, q.y);
        win[2 * m + 1] = make_float2(q.z, q.w);
      }
      float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
      for (int d = 0; d < D; ++d) {
        a0 = fma2(bcast2(wx0[d]), win[d], a0);
        a1 = fma2(bcast2(wx1[d]), win[d + 1], a1);
      }
      *reinterpret_cast<float4*>(Tm + r * kATX + cp2) = make_float4(a0.x, a0.y, a1.x, a1.y);
    }
    __syncthreads();
    // y pass: target rows rr0 .. rr0 + YPW - 1 of column lane read Tm rows rr0 .. rr0 + YPW + 2H - 1
    const int rr0 = SH::YPW * warp, u = x0 + lane;
    float2 win[SH::YPW + 2 * H];
#pragma unroll
    for (int m = 0; m < SH::YPW + 2 * H; ++m) win[m] = Tm[(rr0 + m) * kATX + lane];
#pragma unroll
    for (int q = 0; q < SH::YPW; ++q) {
      const int rr = rr0 + q, w = y0 + rr;
      if (w < a.ny && u < a.nx) {
        float wy[DW];
#pragma unroll
        for (int m = 0; m < DW; m += 4) {
          const float4 v = reinterpret_cast<const float4*>(Wy + rr * DW)[m / 4];
          wy[m] = v.x;
          wy[m + 1] = v.y;
          wy[m + 2] = v.z;
          wy[m + 3] = v.w;
        }
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int d = 0; d < D; ++d) acc = fma2(bcast2(wy[d]), win[q + d], acc);
        const size_t o = (size_t)w * a.nx + u;
        a.lam_out[(size_t)i * a.nv + o] = acc.x;
        a.lam_out[(size_t)(kQ + i) * a.nv + o] = has_g ? acc.y : 0.f;
      }
    }
  }
}

// Per device: SM count (cached) for the persistent grids.
static int adj_sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  int n = (dev >= 0 && dev < 64) ? cache[dev].load(std::memory_order_relaxed) : 0;
  if (n > 0) return n;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 0;
  if (dev >= 0 && dev < 64) cache[dev].store(n, std::memory_order_relaxed);
  return n;
}

template <int H>
static cudaError_t launch_tma(const AdjointArgs& a, cudaStream_t s) {
  using SH = AdjTmaShape<H, kAdjStages>;
  auto kern = adjoint_stream_tma_kernel<H, kAdjStages>;
  if (a.dhalo != H || a.dw != SH::DW) return cudaErrorInvalidValue;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  // 3D map of the pairs as floats: (2 x column, row, velocity plane), ghost cells included
  CUtensorMap mmap;
  const cuuint64_t dims[3] = {(cuuint64_t)2 * a.mu_pitch, (cuuint64_t)a.mu_rows, (cuuint64_t)kQ};
  const cuuint64_t strides[2] = {(cuuint64_t)a.mu_pitch * sizeof(float2),
                                 (cuuint64_t)a.mu_rows * a.mu_pitch * sizeof(float2)};
  const cuuint32_t box[3] = {(cuuint32_t)(2 * SH::RX), (cuuint32_t)SH::RY, 1u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  if (enc(&mmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, a.mu, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
      CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  // the shared-memory opt-in is per device: set it on every launch (a cheap host call)
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SH::kBytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kAdjNT, SH::kBytes)) != cudaSuccess) return e;
  const int n_sm = adj_sm_count();
  if (per_sm < 1 || n_sm < 1) return cudaErrorInvalidConfiguration;
  const long long items = (long long)kQ * ((a.nx + kATX - 1) / kATX) * ((a.ny + SH::TY - 1) / SH::TY);
  const long long grid = items < (long long)n_sm * per_sm ? items : (long long)n_sm * per_sm;
  kern<<<(unsigned)grid, kAdjNT, SH::kBytes, s>>>(a, mmap);
  return cudaGetLastError();
}

bool adjoint_tma_usable(int nx, int ny, int periodic_x, int periodic_y, int halo) {
  const long long items = (long long)kQ * ((nx + kATX - 1) / kATX) * ((ny + 31) / 32);
  return halo <= kAdjGhost && items < (1LL << 31) && (!periodic_x || nx >= 2 * kAdjGhost) &&
         (!periodic_y || ny >= 2 * kAdjGhost) && encode_fn() != nullptr;
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
  } else if (a.mu_g > 0) {   // ghost-padded pairs: the one-pass S^T (chosen by the host set-up)
    if (a.mu_g != kAdjGhost || a.halo > kAdjGhost) return cudaErrorInvalidValue;
    return a.dhalo == 4 ? launch_tma<4>(a, s) : launch_tma<8>(a, s);
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
