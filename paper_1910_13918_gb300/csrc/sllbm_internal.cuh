// Internal definitions shared by the kernels and the host library of the SLLBM (arXiv:1910.13918).
//
// Conventions: a population plane is [ny][pitch] (x fastest); the state is [npop][25][ny][pitch];
// velocity i = 5a + b with a (b) the D1Q5 index of the x (y) component (Table I order).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sllbm {

constexpr int kQ1 = 5;   // D1Q5
constexpr int kQ = 25;   // D2Q25

// Velocity set (Sec. II.B, Table I) and the 1D Hermite table he[k][a] = He_k(xi_a) / k!.
// nq1 = 5 (D1Q5, the method's set) or 3 (D1Q3: the D2Q9 set of the comparison in Sec. III.A,
// nodes 0, +sqrt3, -sqrt3 in the first three entries; the arrays keep the D1Q5 size).
// The fourth-order equilibrium of Sec. II.A factorises over the two axes:
//   f_ab^eq = w_a w_b rho sum_{k+l<=4} A_k(u_x) he[k][a] * A_l(u_y) he[l][b]
// with A_0 = 1, A_1 = u, A_2 = u^2 + q, A_3 = u^3 + 3uq, A_4 = u^4 + 6u^2 q + 3q^2, q = theta - 1
// (the 1D Hermite moments of a Maxwellian; the tensor coefficients a_eq^(n) of Eq. moments are
// their products).
struct Consts {
  double xi[kQ1], w[kQ1];
  double he[kQ1][kQ1];
  float xif[kQ1], wf[kQ1], hef[kQ1][kQ1];
  float whf[kQ1][kQ1];   // w_a he[k][a], FP32
  int nq1;   // 1D nodes of the set: 5 (D2Q25) or 3 (D2Q9); velocity i = nq1 a + b
  float inv_xi1f, xi1sqf;   // 1 / xi_1 and xi_1^2 (xi_1 the first nonzero node), FP32
};

// One axis of the grid as the kernels see it (Sec. II.E): n_cells cells of order p on [lo, hi].
struct AxisK {
  int n_cells, p, nv, periodic;
  double lo, hi, hc, len;
  double nodes[5];
};

// Grid transformation (identity or the sine map of sllbm.h).
struct MapK {
  int kind;
  double a;
};

// BGK parameters (Eq. streaming_fg with Pr = 1).
struct CollideK {
  double omega, cv, K;    // 1/tau, C_v, K = 2 C_v - D
  float omegaf, cvf, Kf, inv2cvf;   // inv2cvf = 1 / (2 C_v)
  int npop;
  int iso;                // isothermal: equilibrium at theta = 1, energy not conserved
  int pr_on;              // Prandtl number != 1: quasi-equilibrium term of Eq. streaming_fg
  double cpr;             // 1/tau - 1/tau_Pr, tau_Pr = (tau - 1/2)/Pr + 1/2
  float cprf;
};

// ------------------------------------------------------------------------------------------
// storage helpers
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float ld_store(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld_store(const __nv_bfloat16* p) {
  return __bfloat162float(__ldg(p));
}
__device__ __forceinline__ void st_store(float* p, float v) { *p = v; }
__device__ __forceinline__ void st_store(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

// (f, g) pairs of the interleaved FP32/BF16 state: the two populations of one (velocity, vertex)
// are adjacent and travel together through the interpolation, in packed FP32x2 arithmetic.
__device__ __forceinline__ float2 ld_pair(const float* p) {
  return __ldg(reinterpret_cast<const float2*>(p));
}
__device__ __forceinline__ float2 ld_pair(const __nv_bfloat16* p) {
  return __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(p)));
}
__device__ __forceinline__ void st_pair(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }
__device__ __forceinline__ void st_pair(__nv_bfloat16* p, float2 v) {
  *reinterpret_cast<__nv_bfloat162*>(p) = __float22bfloat162_rn(v);
}
__device__ __forceinline__ float2 bcast2(float a) { return make_float2(a, a); }
// a - b, rounded once (the product b * -1 is exact)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Ghost cells of the state layout.  A plane is stored as rows [-gy, ny + gyb) x columns
// [-gx, nx + gxr) around the interior origin; on periodic axes the ghost cells hold the periodic
// images of interior vertices so that rectangular tile copies never wrap.  Kernels address
// planes from the interior origin with the row pitch, so vertex (x, y) is at y * pitch + x.
struct GhostK {
  int on;              // 1: writers also store the periodic images that fall in the ghost cells
  int px, py;          // periodic axes
  int nx, ny;
  int xlo, xhi;        // image columns kept: [xlo, xhi) = [-gx, nx + gxr)
  int ylo, yhi;        // image rows kept:    [ylo, yhi) = [-gy, ny + gyb)
};

// Store v at vertex (x, y) of a plane (interior origin `pl`) and at its periodic images in the
// ghost cells.
template <typename Fn>
__device__ __forceinline__ void store_images(const GhostK& gk, int x, int y, Fn&& st) {
  st(x, y);
  if (!gk.on) return;
  const bool xi = gk.px && (x < gk.xhi - gk.nx || x >= gk.xlo + gk.nx);
  const bool yi = gk.py && (y < gk.yhi - gk.ny || y >= gk.ylo + gk.ny);
  if (!xi && !yi) return;
  for (int yy = gk.py ? y - ((y - gk.ylo) / gk.ny) * gk.ny : y; yy < (gk.py ? gk.yhi : y + 1);
       yy += (gk.py ? gk.ny : 1))
    for (int xx = gk.px ? x - ((x - gk.xlo) / gk.nx) * gk.nx : x; xx < (gk.px ? gk.xhi : x + 1);
         xx += (gk.px ? gk.nx : 1))
      if (xx != x || yy != y) st(xx, yy);
}

__host__ __device__ __forceinline__ int wrap_index(int j, int n, int periodic) {
  if (!periodic) return j;
  j %= n;
  return j < 0 ? j + n : j;
}

// ------------------------------------------------------------------------------------------
// geometry helpers (FP64)
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ double fold_axis(double x, const AxisK& ax) {
  if (ax.periodic) {
    double s = fmod(x - ax.lo, ax.len);
    if (s < 0.0) s += ax.len;
    return ax.lo + s;
  }
  return fmin(fmax(x, ax.lo), ax.hi);
}

// Cell and local coordinate of a folded coordinate.  A point within rounding (1e-12 of a cell) of a
// cell face is put at r = 0 of the cell on its right, so that vertices whose departure lands on a
// face get the same stencil whatever the rounding of their coordinates (the interpolant is
// continuous there, so the value is the same either way).
__device__ __forceinline__ void locate_axis(double x, const AxisK& ax, int* cell, double* r) {
  double s = (x - ax.lo) / ax.hc;
  int c = (int)floor(s);
  c = c < 0 ? 0 : (c > ax.n_cells - 1 ? ax.n_cells - 1 : c);
  double rr = s - (double)c;
  if (rr > 1.0 - 1e-12) {
    if (c < ax.n_cells - 1) {
      c += 1;
      rr = 0.0;
    } else if (ax.periodic) {
      c = 0;
      rr = 0.0;
    }
  } else if (rr < 1e-12) {
    rr = 0.0;
  }
  *cell = c;
  *r = rr;
}

__device__ __forceinline__ double vertex_ref_coord(int j, const AxisK& ax) {
  if (!ax.periodic && j == ax.nv - 1) return ax.hi;
  int c = j / ax.p, k = j % ax.p;
  return ax.lo + ax.hc * ((double)c + ax.nodes[k]);
}

// Lagrange basis psi_a(r) on the support points of the reference interval (Eq. sl_streaming).
template <int P, typename T>
__device__ __forceinline__ void lagrange_basis(const T* nodes, T r, T* psi) {
#pragma unroll
  for (int a = 0; a <= P; ++a) {
    T acc = T(1);
#pragma unroll
    for (int b = 0; b <= P; ++b)
      if (b != a) acc *= (r - nodes[b]) / (nodes[a] - nodes[b]);
    psi[a] = acc;
  }
}

__device__ __forceinline__ void sine_map(double a, double xi, double eta, double* x, double* y) {
  const double pi = 3.141592653589793238462643383279502884;
  *x = xi + a * sin(2.0 * pi * xi) * sin(pi * eta);
  *y = eta + a * sin(pi * xi) * sin(2.0 * pi * eta);
}

__device__ __forceinline__ void sine_map_jac(double a, double xi, double eta, double* j11,
                                             double* j12, double* j21, double* j22) {
  const double pi = 3.141592653589793238462643383279502884;
  *j11 = 1.0 + 2.0 * pi * a * cos(2.0 * pi * xi) * sin(pi * eta);
  *j12 = pi * a * sin(2.0 * pi * xi) * cos(pi * eta);
  *j21 = pi * a * cos(pi * xi) * sin(2.0 * pi * eta);
  *j22 = 1.0 + 2.0 * pi * a * sin(pi * xi) * cos(2.0 * pi * eta);
}

// ------------------------------------------------------------------------------------------
// equilibrium (closed, factorised form of Sec. II.A) -- templated on the arithmetic type
// ------------------------------------------------------------------------------------------
template <typename T>
struct EqFactors {
  T X[4][kQ1];   // X[k-1][a] = A_k(u_x) he[k][a], k = 1..4
  T S[5][kQ1];   // S[m][b]   = sum_{l=1..m} A_l(u_y) he[l][b]
};

template <typename T>
__device__ __forceinline__ void eq_factors(const T (&he)[kQ1][kQ1], T ux, T uy, T q,
                                           EqFactors<T>& e) {
  T ax[5], ay[5];
  ax[1] = ux;
  ax[2] = ux * ux + q;
  ax[3] = ux * (ux * ux + T(3) * q);
  ax[4] = ux * ux * (ux * ux + T(6) * q) + T(3) * q * q;
  ay[1] = uy;
  ay[2] = uy * uy + q;
  ay[3] = uy * (uy * uy + T(3) * q);
  ay[4] = uy * uy * (uy * uy + T(6) * q) + T(3) * q * q;
#pragma unroll
  for (int a = 0; a < kQ1; ++a) {
#pragma unroll
    for (int k = 1; k <= 4; ++k) e.X[k - 1][a] = ax[k] * he[k][a];
  }
#pragma unroll
  for (int b = 0; b < kQ1; ++b) {
    e.S[0][b] = T(0);
#pragma unroll
    for (int m = 1; m <= 4; ++m) e.S[m][b] = e.S[m - 1][b] + ay[m] * he[m][b];
  }
}

// E_ab - 1 where f_ab^eq = w_ab rho E_ab; computed without cancellation against 1.
template <typename T>
__device__ __forceinline__ T eq_em1(const EqFactors<T>& e, int a, int b) {
  T s = e.S[4][b];
#pragma unroll
  for (int k = 1; k <= 4; ++k) s += e.X[k - 1][a] * (T(1) + e.S[4 - k][b]);
  return s;
}

// Moments (rho, u, v, theta) of the pre-collision values of one vertex: what its collision was
// evaluated at (theta from the moments also in the isothermal configuration, whose equilibrium
// takes theta = 1).
struct VertexMoments {
  float rho, ux, uy, theta;
};

__device__ __forceinline__ void store_moments(float* mom, long long nv, long long v, const VertexMoments& vm) {
  mom[v] = vm.rho;
  mom[nv + v] = vm.ux;
  mom[2 * nv + v] = vm.uy;
  mom[3 * nv + v] = vm.theta;
}

// Collision of one vertex in deviation form, FP32.  fg[i] = (f_i - w_i, g_i - K w_i) before
// collision (g unused with a single population); on return fg holds the post-collision
// deviations and vm the moments of the pre-collision values.  Returns false if the density or
// temperature is non-positive or non-finite.
//
// With X_k(a) = A_k(u_x) he[k][a] and S_m(b) = sum_{l=1..m} A_l(u_y) he[l][b] the equilibrium
// deviation is f_ab^eq - w_ab = w_a w_b (drho + rho S_4(b)) + sum_k (rho w_a X_k(a)) (w_b (1 +
// S_{4-k}(b))): after a per-vertex set-up of 45 factors, five FMAs per velocity.
template <bool PR = false>
__device__ __forceinline__ bool collide_deviation_f32(float2 (&fg)[kQ], const Consts& cs,
                                                      const CollideK& cp, VertexMoments& vm) {
  // moments (Sec. II): rho = 1 + sum fbar, j = sum fbar xi, A2 = sum fbar |xi|^2, G = sum gbar.
  // Row and column sums of the (f, g) pairs in packed FP32x2: rs[a] = (sum_b f_ab, sum_b g_ab).
  float2 rs[kQ1], cl[kQ1];
#pragma unroll
  for (int a = 0; a < kQ1; ++a) {
    rs[a] = fg[5 * a];
#pragma unroll
    for (int b = 1; b < kQ1; ++b) rs[a] = __fadd2_rn(rs[a], fg[5 * a + b]);
  }
#pragma unroll
  for (int b = 0; b < kQ1; ++b) {
    cl[b] = fg[b];
#pragma unroll
    for (int a = 1; a < kQ1; ++a) cl[b] = __fadd2_rn(cl[b], fg[5 * a + b]);
  }
  float drho = 0.f, jx = 0.f, jy = 0.f, a2 = 0.f;
#pragma unroll
  for (int a = 0; a < kQ1; ++a) {
    drho += rs[a].x;
    jx += cs.xif[a] * rs[a].x;
    jy += cs.xif[a] * cl[a].x;
    a2 += cs.xif[a] * cs.xif[a] * (rs[a].x + cl[a].x);
  }
  float G = 0.f;
  if (cp.npop == 2) {
#pragma unroll
    for (int a = 0; a < kQ1; ++a) G += rs[a].y;
  }
  const float rho = 1.f + drho;
  const float inv_rho = __frcp_rn(rho);
  const float ux = jx * inv_rho, uy = jy * inv_rho;
  // Pr != 1 (Sec. II.C): the non-equilibrium centred third moments of f and g, as (f, g) pairs
  // xxx, xxy, xyy, yyy.  The equilibrium's centred third moment is zero, so they are those of the
  // pre-collision populations: of the stored deviations plus the lattice-weight part,
  // sum_i w_i (xi - u)^3 = -(u_a d_bc + u_b d_ac + u_c d_ab) - u_a u_b u_c (times K for g).
  float2 Qn[4];
  if constexpr (PR) {
    float cx[kQ1], cy[kQ1];
#pragma unroll
    for (int a = 0; a < kQ1; ++a) {
      cx[a] = cs.xif[a] - ux;
      cy[a] = cs.xif[a] - uy;
    }
    float2 qxxx = make_float2(0.f, 0.f), qxxy = qxxx, qxyy = qxxx, qyyy = qxxx;
#pragma unroll
    for (int a = 0; a < kQ1; ++a) {
      float2 s1 = make_float2(0.f, 0.f), s2 = s1;   // sum_b cy fg_ab, sum_b cy^2 fg_ab
#pragma unroll
      for (int b = 0; b < kQ1; ++b) {
        s1 = fma2(bcast2(cy[b]), fg[5 * a + b], s1);
        s2 = fma2(bcast2(cy[b] * cy[b]), fg[5 * a + b], s2);
      }
      const float cx2 = cx[a] * cx[a];
      qxxx = fma2(bcast2(cx2 * cx[a]), rs[a], qxxx);
      qxxy = fma2(bcast2(cx2), s1, qxxy);
      qxyy = fma2(bcast2(cx[a]), s2, qxyy);
      qyyy = fma2(bcast2(cy[a] * cy[a] * cy[a]), cl[a], qyyy);
    }
    const float wxxx = -3.f * ux - ux * ux * ux, wxxy = -uy - ux * ux * uy;
    const float wxyy = -ux - ux * uy * uy, wyyy = -3.f * uy - uy * uy * uy;
    Qn[0] = make_float2(qxxx.x + wxxx, qxxx.y + cp.Kf * wxxx);
    Qn[1] = make_float2(qxxy.x + wxxy, qxxy.y + cp.Kf * wxxy);
    Qn[2] = make_float2(qxyy.x + wxyy, qxyy.y + cp.Kf * wxyy);
    Qn[3] = make_float2(qyyy.x + wyyy, qyyy.y + cp.Kf * wyyy);
  }
  (void)Qn;
  // theta - 1 = (A2 + G - rho |u|^2 - 2 C_v drho) / (2 C_v rho)
  const float qk = (a2 + G - rho * (ux * ux + uy * uy) - 2.f * cp.cvf * drho) * inv_rho * cp.inv2cvf;
  const float q = cp.iso ? 0.f : qk;
  vm.rho = rho;
  vm.ux = ux;
  vm.uy = uy;
  vm.theta = 1.f + qk;
  float ax[5], ay[5];
  ax[1] = ux;
  ax[2] = ux * ux + q;
  ax[3] = ux * (ux * ux + 3.f * q);
  ax[4] = ux * ux * (ux * ux + 6.f * q) + 3.f * q * q;
  ay[1] = uy;
  ay[2] = uy * uy + q;
  ay[3] = uy * (uy * uy + 3.f * q);
  ay[4] = uy * uy * (uy * uy + 6.f * q) + 3.f * q * q;
  // The 1D nodes are 0, +s, +l, -s, -l: component a + 2 (a = 1, 2) mirrors a, so with
  // He_k(-xi) = (-1)^k He_k(xi) its X_k(a + 2) is (-1)^k X_k(a), and X_k(0) = 0 for odd k.  Only
  // a = 0, 1, 2 are formed; each mirrored pair takes even part +- odd part.
  float Xw[4][3], Sw[4][kQ1], Bb[kQ1];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float rw = rho * cs.wf[a];
#pragma unroll
    for (int k = 1; k <= 4; ++k) Xw[k - 1][a] = rw * (ax[k] * cs.hef[k][a]);
  }
#pragma unroll
  for (int b = 0; b < kQ1; ++b) {
    float acc = 0.f;   // S_m(b)
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      Sw[m][b] = cs.wf[b] * (1.f + acc);
      acc += ay[m + 1] * cs.hef[m + 1][b];
    }
    Bb[b] = cs.wf[b] * (drho + rho * acc);
  }
  const float om = cp.omegaf;
  const float Kq1 = cp.Kf * (1.f + q), Kq = cp.Kf * q;
  // Post-collision values f + omega (f^eq - f), and the moments of (f^eq - f) itself.  In exact
  // arithmetic the equilibrium has the moments of the pre-collision state; in FP32 its
  // fourth-order polynomial carries rounding of the size of its largest terms, which would leak
  // into the conserved moments every step.  The residuals are summed from the differences
  // f^eq - f (small, and mostly exact in FP32), not as differences of two sums of full-size
  // values: at omega near 2 the state is almost 2-periodic in time, the roundings of such sums
  // repeat every other step, and their mismatch would add up to a steady drift of the moments.
  float2 drow[kQ1];   // sum_b (f^eq - f, g^eq - g) of row a
  float dcol[kQ1], KqW[kQ1];
#pragma unroll
  for (int a = 0; a < kQ1; ++a) {
    drow[a] = make_float2(0.f, 0.f);
    dcol[a] = 0.f;
    KqW[a] = Kq * cs.wf[a];
  }
  // The g lanes are computed whatever the population count (with one population they hold
  // zeros and are never stored); f and g relax together in packed FP32x2 arithmetic.
  const float2 om2 = bcast2(om);
  // g^eq - K w = K ((1 + q)(f^eq - w) + q w)   (g^eq = K theta f^eq, Sec. II.D); t = K q w_a w_b
  auto relax = [&](int a, int b, float ef, float t) {
    const float egi = Kq1 * ef + t;
    const float2 d = sub2(make_float2(ef, egi), fg[5 * a + b]);
    drow[a] = __fadd2_rn(drow[a], d);
    dcol[b] += d.x;
    fg[5 * a + b] = fma2(om2, d, fg[5 * a + b]);
  };
#pragma unroll
  for (int b = 0; b < kQ1; ++b) {
    // f^eq - w for (a, b): w_a B(b) + sum_k X_k(a) S_{4-k}(b), even k and odd k apart
    float ev[3], od[3], t[3];
#pragma unroll
    for (int a = 1; a <= 2; ++a) {
      ev[a] = cs.wf[a] * Bb[b] + Xw[1][a] * Sw[2][b] + Xw[3][a] * Sw[0][b];
      od[a] = Xw[0][a] * Sw[3][b] + Xw[2][a] * Sw[1][b];
      t[a] = cs.wf[a] * KqW[b];
    }
    relax(0, b, cs.wf[0] * Bb[b] + Xw[1][0] * Sw[2][b] + Xw[3][0] * Sw[0][b], cs.wf[0] * KqW[b]);
    relax(1, b, ev[1] + od[1], t[1]);
    relax(2, b, ev[2] + od[2], t[2]);
    relax(3, b, ev[1] - od[1], t[1]);
    relax(4, b, ev[2] - od[2], t[2]);
  }
  // Residual moments of (equilibrium - pre-collision state): mass, x and y momentum of f, and
  // the energy of f and g.
  float r0 = 0.f, r1 = 0.f, r2 = 0.f, r3 = 0.f, rg = 0.f;
#pragma unroll
  for (int a = 0; a < kQ1; ++a) {
    r0 += drow[a].x;
    r1 += cs.xif[a] * drow[a].x;
    r2 += cs.xif[a] * dcol[a];
    r3 += cs.xif[a] * cs.xif[a] * (drow[a].x + dcol[a]);
    rg += drow[a].y;
  }
  if (cp.npop == 2) r3 += rg;
  // Remove the residuals at the fewest velocities that span the conserved moments: mass and
  // momentum on f at the rest velocity and at the two velocities with one small component,
  // xi = (s, 0) (i = 5) and (0, s) (i = 1); the energy left after that on g at the rest velocity
  // (g carries energy only).  This changes nothing in exact arithmetic and restores conservation
  // to the rounding of the sums.
  {
    const float inv_s = cs.inv_xi1f, s2 = cs.xi1sqf;
    const float d1 = r1 * inv_s, d2 = r2 * inv_s;
    const float d0 = r0 - d1 - d2;
    const float de = r3 - s2 * (d1 + d2);   // energy residual left after the mass/momentum fix
    fg[0].x -= om * d0;
    fg[5].x -= om * d1;
    fg[1].x -= om * d2;
    if (cp.npop == 2) {
      fg[0].y -= om * de;
    } else if (!cp.iso) {
      // one population: along (xi = (+-s, 0): +e, rest: -2e), which carries no mass or
      // momentum and the energy 2 s^2 e
      const float e = om * 0.5f * de * inv_s * inv_s;
      fg[5].x -= e;
      fg[15].x -= e;
      fg[0].x += 2.f * e;
    }
  }
  if constexpr (PR) {
    // + (1/tau - 1/tau_Pr) f^qe with f^qe_ab = w_a w_b (Q_xxx h3(a) + Q_xxy h2(a) h1(b) +
    // Q_xyy h1(a) h2(b) + Q_yyy h3(b)), h_n = He_n / n!: the contraction w_i Q : H^(3)(xi_i) / 3!
    // of Sec. II.C written out over the tensor-product velocities (it carries no mass, momentum
    // or energy); the same with g's moments for g
    float wh1[kQ1], wh2[kQ1], wh3[kQ1];
#pragma unroll
    for (int b = 0; b < kQ1; ++b) {
      wh1[b] = cs.wf[b] * cs.hef[1][b];
      wh2[b] = cs.wf[b] * cs.hef[2][b];
      wh3[b] = cs.wf[b] * cs.hef[3][b];
    }
#pragma unroll
    for (int a = 0; a < kQ1; ++a) {
      const float ca = cp.cprf * cs.wf[a];
      const float2 B0 = __fmul2_rn(bcast2(ca * cs.hef[3][a]), Qn[0]);
      const float2 B1 = __fmul2_rn(bcast2(ca * cs.hef[2][a]), Qn[1]);
      const float2 B2 = __fmul2_rn(bcast2(ca * cs.hef[1][a]), Qn[2]);
      const float2 B3 = __fmul2_rn(bcast2(ca), Qn[3]);
#pragma unroll
      for (int b = 0; b < kQ1; ++b) {
        float2 t = fma2(bcast2(cs.wf[b]), B0, fg[5 * a + b]);
        t = fma2(bcast2(wh1[b]), B1, t);
        t = fma2(bcast2(wh2[b]), B2, t);
        fg[5 * a + b] = fma2(bcast2(wh3[b]), B3, t);
      }
    }
  }
  return (rho > 0.f) && (q > -1.f) && isfinite(rho) && isfinite(q);
}

}  // namespace sllbm
