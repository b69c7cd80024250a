// 3D extension of the SLLBM step (the paper's stated next step): D3Q125, the tensor product of
// D1Q5 three times (Sec. II.B), on a uniform grid of hexahedral Lagrange cells (Sec. II.E per
// axis), the fourth-order equilibrium of Sec. II.A with index tuples over {x, y, z}, g^eq =
// (2 C_v - 3) theta f^eq (Sec. II.D) and BGK (Eq. streaming_fg, Pr = 1).  A plain FP64 step on
// full populations, one thread per vertex: the first pass interpolates every velocity of f and g
// at its departure point (tensor product of the three 1D Lagrange bases, per-axis tables as in
// 2D) into the destination and sums the moments, the second relaxes each value in place.  The
// equilibrium is the factorised form: the tensor coefficients a_eq^(n) of an isotropic Maxwellian
// are products of per-axis Hermite moments A_k(u) (A_0 = 1, A_1 = u, A_2 = u^2 + q, A_3 = u^3 +
// 3uq, A_4 = u^4 + 6u^2 q + 3q^2, q = theta - 1), so
//   f_abc^eq = w_a w_b w_c rho sum_{k+l+m <= 4} A_k(u_x) he_k(a) A_l(u_y) he_l(b) A_m(u_z) he_m(c).
// This file has its own context and entry points (sllbm3d_* in include/sllbm.h); it shares the
// axis-table kernel and the device helpers with the 2D library.
#include <math.h>

#include <new>
#include <string>
#include <vector>

#include "../../include/sllbm.h"
#include "kernels.h"

using namespace sllbm;

namespace {

constexpr int kQ3 = kQ1 * kQ1 * kQ1;   // D3Q125

struct Step3Args {
  const double* src;
  double* dst;
  int nx, ny, nz;
  long long nv;
  int px, py, pz;                        // periodic axes
  const int *offx, *offy, *offz;         // [5][n]: stencil start - vertex index
  const double *wx, *wy, *wz;            // [5][n][p+1]
  Consts cs;
  double omega, K, cv;
  int npop, iso;
  int* flag;                             // bit 0: unstable
};

struct Field3Args {
  const double *rho, *u, *v, *w, *T;     // init inputs
  double *orho, *ou, *ov, *ow, *oT;      // moment outputs
  double* state;                         // FP64: full populations [npop][125][nv]
  float2* state32;                       // FP32: (f - w, g - K w) pairs [125][nv] (else null)
  long long nv;
  Consts cs;
  double K, cv;
  int npop;
  int* flag;
};

// FP32 step: deviations from the lattice weights, f and g of a (velocity, vertex) side by side.
struct Step3F32Args {
  const float2* src;
  float2* dst;
  int nx, ny, nz;
  long long nv;
  int px, py, pz;
  const int *offx, *offy, *offz;         // [5][n]
  const float *wx, *wy, *wz;             // [5][n][p+1]
  Consts cs;
  float omega, K, cv, inv2cv;
  int npop, iso;
  int* flag;
};

// Per-axis Hermite moments A_k(u), k = 0..4, of the Maxwellian with q = theta - 1.
__device__ __forceinline__ void hermite_moments(double u, double q, double (&A)[5]) {
  A[0] = 1.0;
  A[1] = u;
  A[2] = u * u + q;
  A[3] = u * (u * u + 3.0 * q);
  A[4] = u * u * (u * u + 6.0 * q) + 3.0 * q * q;
}

// f^eq of velocity (a, b, c), given the per-axis factors X[k] = A_k(u_x) he_k(a) etc.
__device__ __forceinline__ double eq3(const Consts& cs, double rho, const double (&Ax)[5],
                                      const double (&Ay)[5], const double (&Az)[5], int a, int b, int c) {
  double s = 0.0;
#pragma unroll
  for (int k = 0; k <= 4; ++k) {
    const double xk = Ax[k] * cs.he[k][a];
#pragma unroll
    for (int l = 0; l <= 4 - k; ++l) {
      const double yl = Ay[l] * cs.he[l][b];
      double zs = 0.0;
#pragma unroll
      for (int m = 0; m <= 4 - k - l; ++m) zs += Az[m] * cs.he[m][c];
      s += xk * yl * zs;
    }
  }
  return cs.w[a] * cs.w[b] * cs.w[c] * rho * s;
}

template <int P>
__global__ void __launch_bounds__(128) step3d_f64_kernel(const __grid_constant__ Step3Args a) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= a.nv) return;
  const int ix = (int)(v % a.nx);
  const long long t = v / a.nx;
  const int iy = (int)(t % a.ny), iz = (int)(t / a.ny);
  const size_t plane = (size_t)a.nv;
  const bool two = a.npop == 2;
  double rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0, e2 = 0.0;
#pragma unroll 1
  for (int i = 0; i < kQ3; ++i) {
    const int ia = i / 25, ib = (i / 5) % 5, ic = i % 5;
    const int sx = ix + a.offx[ia * a.nx + ix], sy = iy + a.offy[ib * a.ny + iy],
              sz = iz + a.offz[ic * a.nz + iz];
    const double* wx = a.wx + (size_t)(ia * a.nx + ix) * (P + 1);
    const double* wy = a.wy + (size_t)(ib * a.ny + iy) * (P + 1);
    const double* wz = a.wz + (size_t)(ic * a.nz + iz) * (P + 1);
    const double* pf = a.src + (size_t)i * plane;
    const double* pg = two ? a.src + (size_t)(kQ3 + i) * plane : pf;
    double accf = 0.0, accg = 0.0;
#pragma unroll
    for (int kc = 0; kc <= P; ++kc) {
      const size_t zoff = (size_t)wrap_index(sz + kc, a.nz, a.pz) * a.ny;
      double yf = 0.0, yg = 0.0;
#pragma unroll
      for (int kb = 0; kb <= P; ++kb) {
        const size_t row = (zoff + (size_t)wrap_index(sy + kb, a.ny, a.py)) * a.nx;
        double xf = 0.0, xg = 0.0;
#pragma unroll
        for (int ka = 0; ka <= P; ++ka) {
          const size_t o = row + (size_t)wrap_index(sx + ka, a.nx, a.px);
          xf += wx[ka] * __ldg(pf + o);
          if (two) xg += wx[ka] * __ldg(pg + o);
        }
        yf += wy[kb] * xf;
        yg += wy[kb] * xg;
      }
      accf += wz[kc] * yf;
      accg += wz[kc] * yg;
    }
    a.dst[(size_t)i * plane + v] = accf;
    if (two) a.dst[(size_t)(kQ3 + i) * plane + v] = accg;
    const double cx = a.cs.xi[ia], cy = a.cs.xi[ib], cz = a.cs.xi[ic];
    rho += accf;
    jx += accf * cx;
    jy += accf * cy;
    jz += accf * cz;
    e2 += accf * (cx * cx + cy * cy + cz * cz) + accg;
  }
  const double ux = jx / rho, uy = jy / rho, uz = jz / rho;
  const double theta = a.iso ? 1.0 : (e2 - rho * (ux * ux + uy * uy + uz * uz)) / (2.0 * a.cv * rho);
  const double q = theta - 1.0;
  double Ax[5], Ay[5], Az[5];
  hermite_moments(ux, q, Ax);
  hermite_moments(uy, q, Ay);
  hermite_moments(uz, q, Az);
#pragma unroll 1
  for (int i = 0; i < kQ3; ++i) {
    const double feq = eq3(a.cs, rho, Ax, Ay, Az, i / 25, (i / 5) % 5, i % 5);
    double* df = a.dst + (size_t)i * plane + v;
    *df -= a.omega * (*df - feq);
    if (two) {
      double* dg = a.dst + (size_t)(kQ3 + i) * plane + v;
      *dg -= a.omega * (*dg - a.K * theta * feq);
    }
  }
  if (!(rho > 0.0 && theta > 0.0 && isfinite(rho) && isfinite(theta))) atomicOr(a.flag, 1);
}

// Index j of an axis of n vertices, wrapped once on periodic axes: stencil nodes lie within one
// period of the vertex (the departure displacement is far below the domain length).
__device__ __forceinline__ int wrap1(int j, int n, int periodic) {
  if (!periodic) return j;
  return j < 0 ? j + n : (j >= n ? j - n : j);
}

// Weight w_abc of velocity i = 25a + 5b + c (FP32).
__device__ __forceinline__ float w3f(const Consts& cs, int i) {
  return cs.wf[i / 25] * cs.wf[(i / 5) % 5] * cs.wf[i % 5];
}

// Fused FP32 step, one thread per vertex, one launch.  First sweep: every velocity's (f, g) pair
// is interpolated at its departure point (tensor product of the three 1D Lagrange bases, each in
// the difference form v_0 + sum_{k>=1} w_k (v_k - v_0), which keeps constant fields exact) and
// written to the destination, and its moments are summed.  Second sweep: the thread reads its
// own 125 pairs back (from L1/L2: no second pass over HBM), relaxes them toward the factorised
// equilibrium and sums the residual moments of (f^eq - f); the residuals (the FP32 rounding of
// the equilibrium) are then removed at the rest velocity and at (s, 0, 0), (0, s, 0), (0, 0, s)
// for mass and momentum, and on g at the rest velocity for the energy.
template <int P>
__global__ void __launch_bounds__(128) step3d_f32_kernel(const __grid_constant__ Step3F32Args a) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= a.nv) return;
  const int ix = (int)(v % a.nx);
  const long long t = v / a.nx;
  const int iy = (int)(t % a.ny), iz = (int)(t / a.ny);
  const size_t plane = (size_t)a.nv;
  float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f, a2 = 0.f, G = 0.f;
#pragma unroll 1
  for (int i = 0; i < kQ3; ++i) {
    const int ia = i / 25, ib = (i / 5) % 5, ic = i % 5;
    const int sx = ix + a.offx[ia * a.nx + ix], sy = iy + a.offy[ib * a.ny + iy],
              sz = iz + a.offz[ic * a.nz + iz];
    const float* wx = a.wx + (size_t)(ia * a.nx + ix) * (P + 1);
    const float* wy = a.wy + (size_t)(ib * a.ny + iy) * (P + 1);
    const float* wz = a.wz + (size_t)(ic * a.nz + iz) * (P + 1);
    const float2* pl = a.src + (size_t)i * plane;
    int cx[P + 1], cy[P + 1], cz[P + 1];
#pragma unroll
    for (int k = 0; k <= P; ++k) {
      cx[k] = wrap1(sx + k, a.nx, a.px);
      cy[k] = wrap1(sy + k, a.ny, a.py);
      cz[k] = wrap1(sz + k, a.nz, a.pz);
    }
    float2 zs[P + 1];
#pragma unroll
    for (int kc = 0; kc <= P; ++kc) {
      const size_t zoff = (size_t)cz[kc] * a.ny;
      float2 ys[P + 1];
#pragma unroll
      for (int kb = 0; kb <= P; ++kb) {
        const float2* row = pl + (zoff + (size_t)cy[kb]) * a.nx;
        const float2 b0 = __ldg(row + cx[0]);
        float2 acc = b0;
#pragma unroll
        for (int ka = 1; ka <= P; ++ka) acc = fma2(bcast2(__ldg(wx + ka)), sub2(__ldg(row + cx[ka]), b0), acc);
        ys[kb] = acc;
      }
      float2 acc = ys[0];
#pragma unroll
      for (int kb = 1; kb <= P; ++kb) acc = fma2(bcast2(__ldg(wy + kb)), sub2(ys[kb], ys[0]), acc);
      zs[kc] = acc;
    }
    float2 acc = zs[0];
#pragma unroll
    for (int kc = 1; kc <= P; ++kc) acc = fma2(bcast2(__ldg(wz + kc)), sub2(zs[kc], zs[0]), acc);
    a.dst[(size_t)i * plane + v] = acc;
    const float ex = a.cs.xif[ia], ey = a.cs.xif[ib], ez = a.cs.xif[ic];
    drho += acc.x;
    jx += ex * acc.x;
    jy += ey * acc.x;
    jz += ez * acc.x;
    a2 += (ex * ex + ey * ey + ez * ez) * acc.x;
    G += acc.y;
  }
  if (a.npop != 2) G = 0.f;
  const float rho = 1.f + drho, inv_rho = __frcp_rn(rho);
  const float ux = jx * inv_rho, uy = jy * inv_rho, uz = jz * inv_rho;
  // theta - 1 = (A2 + G - rho |u|^2 - 2 C_v drho) / (2 C_v rho)   (sum w |xi|^2 + K = 2 C_v)
  const float qk = (a2 + G - rho * (ux * ux + uy * uy + uz * uz) - 2.f * a.cv * drho) * inv_rho * a.inv2cv;
  const float q = a.iso ? 0.f : qk;
  // per-axis factors X_k(a) = A_k(u_x) he_k(a), Y_l(b) likewise, Zc_n(c) = sum_{m <= n} A_m(u_z)
  // he_m(c): 1 + S_abc = sum_{k + l + m <= 4} X_k(a) Y_l(b) Z_m(c), and f^eq - w = w (drho + rho S)
  float Ax[5], Ay[5], Az[5];
  {
    const float u3[3] = {ux, uy, uz};
    float* A3[3] = {Ax, Ay, Az};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float u = u3[d];
      A3[d][0] = 1.f;
      A3[d][1] = u;
      A3[d][2] = u * u + q;
      A3[d][3] = u * (u * u + 3.f * q);
      A3[d][4] = u * u * (u * u + 6.f * q) + 3.f * q * q;
    }
  }
  float Zc[5][5];   // [n][c], compile-time indices only
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    float acc = 0.f;
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      acc += Az[m] * a.cs.hef[m][c];
      Zc[m][c] = acc;
    }
  }
  const float om = a.omega, Kq1 = a.K * (1.f + q), Kq = a.K * q;
  const float2 om2 = bcast2(om);
  float r0 = 0.f, r1 = 0.f, r2 = 0.f, r3 = 0.f, re = 0.f;
#pragma unroll 1
  for (int ia = 0; ia < kQ1; ++ia) {
    float Xa[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) Xa[k] = Ax[k] * a.cs.hef[k][ia];
    const float ex = a.cs.xif[ia], wa = a.cs.wf[ia];
#pragma unroll 1
    for (int ib = 0; ib < kQ1; ++ib) {
      float Yb[5];
#pragma unroll
      for (int l = 0; l < 5; ++l) Yb[l] = Ay[l] * a.cs.hef[l][ib];
      const float ey = a.cs.xif[ib], wab = wa * a.cs.wf[ib];
#pragma unroll
      for (int ic = 0; ic < kQ1; ++ic) {
        const int i = 25 * ia + 5 * ib + ic;
        float s1 = 0.f;
#pragma unroll
        for (int k = 0; k <= 4; ++k) {
          float sl = 0.f;
#pragma unroll
          for (int l = 0; l <= 4 - k; ++l) sl += Yb[l] * Zc[4 - k - l][ic];
          s1 += Xa[k] * sl;
        }
        const float w = wab * a.cs.wf[ic];
        const float ef = w * (drho + rho * (s1 - 1.f));
        const float eg = Kq1 * ef + Kq * w;   // g^eq - K w = K ((1 + q)(f^eq - w) + q w)
        float2* o = a.dst + (size_t)i * plane + v;
        const float2 fg = *o;
        const float2 d = sub2(make_float2(ef, a.npop == 2 ? eg : 0.f), fg);
        const float ez = a.cs.xif[ic];
        r0 += d.x;
        r1 += ex * d.x;
        r2 += ey * d.x;
        r3 += ez * d.x;
        re += (ex * ex + ey * ey + ez * ez) * d.x + d.y;
        *o = fma2(om2, d, fg);
      }
    }
  }
  {   // remove the residuals (see above): i = 25 a + 5 b + c; s = xi of index 1
    const float inv_s = a.cs.inv_xi1f, s2 = a.cs.xi1sqf;
    const float d1 = r1 * inv_s, d2 = r2 * inv_s, d3 = r3 * inv_s;
    const float d0 = r0 - d1 - d2 - d3;
    const float de = re - s2 * (d1 + d2 + d3);
    float2* o = a.dst + v;
    o[0].x -= om * d0;
    o[25 * plane].x -= om * d1;
    o[5 * plane].x -= om * d2;
    o[1 * plane].x -= om * d3;
    if (a.npop == 2) {
      o[0].y -= om * de;
    } else if (!a.iso) {   // one population: energy along (+-s, 0, 0) and -2 at rest
      const float e = om * 0.5f * de * inv_s * inv_s;
      o[25 * plane].x -= e;
      o[75 * plane].x -= e;
      o[0].x += 2.f * e;
    }
  }
  if (!((rho > 0.f) && (qk > -1.f) && isfinite(rho) && isfinite(qk))) atomicOr(a.flag, 1);
}

// FP32 pairs <-> dense FP64 full populations [npop][125][nv].
__global__ void convert3d_kernel(float2* pairs, double* dense, long long nv, int npop, double K,
                                 Consts cs, int to_dense) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)kQ3 * nv) return;
  const int i = (int)(e / nv);
  const double w = cs.w[i / 25] * cs.w[(i / 5) % 5] * cs.w[i % 5];
  if (to_dense) {
    const float2 p = pairs[e];
    dense[e] = (double)p.x + w;
    if (npop == 2) dense[(size_t)kQ3 * nv + e] = (double)p.y + K * w;
  } else {
    const float f = (float)(dense[e] - w);
    const float g = npop == 2 ? (float)(dense[(size_t)kQ3 * nv + e] - K * w) : 0.f;
    pairs[e] = make_float2(f, g);
  }
}

__global__ void init3d_kernel(const __grid_constant__ Field3Args a) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= a.nv) return;
  const double rho = a.rho[v], theta = a.T[v], q = theta - 1.0;
  double Ax[5], Ay[5], Az[5];
  hermite_moments(a.u[v], q, Ax);
  hermite_moments(a.v[v], q, Ay);
  hermite_moments(a.w[v], q, Az);
  const size_t plane = (size_t)a.nv;
  for (int i = 0; i < kQ3; ++i) {
    const double feq = eq3(a.cs, rho, Ax, Ay, Az, i / 25, (i / 5) % 5, i % 5);
    if (a.state32) {
      const double w = a.cs.w[i / 25] * a.cs.w[(i / 5) % 5] * a.cs.w[i % 5];
      a.state32[(size_t)i * plane + v] =
          make_float2((float)(feq - w), a.npop == 2 ? (float)(a.K * theta * feq - a.K * w) : 0.f);
    } else {
      a.state[(size_t)i * plane + v] = feq;
      if (a.npop == 2) a.state[(size_t)(kQ3 + i) * plane + v] = a.K * theta * feq;
    }
  }
}

__global__ void moments3d_kernel(const __grid_constant__ Field3Args a) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= a.nv) return;
  const size_t plane = (size_t)a.nv;
  double rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0, e2 = 0.0;
  for (int i = 0; i < kQ3; ++i) {
    double f, g;
    if (a.state32) {
      const float2 p = a.state32[(size_t)i * plane + v];
      const double w = a.cs.w[i / 25] * a.cs.w[(i / 5) % 5] * a.cs.w[i % 5];
      f = (double)p.x + w;
      g = a.npop == 2 ? (double)p.y + a.K * w : 0.0;
    } else {
      f = a.state[(size_t)i * plane + v];
      g = a.npop == 2 ? a.state[(size_t)(kQ3 + i) * plane + v] : 0.0;
    }
    const double cx = a.cs.xi[i / 25], cy = a.cs.xi[(i / 5) % 5], cz = a.cs.xi[i % 5];
    rho += f;
    jx += f * cx;
    jy += f * cy;
    jz += f * cz;
    e2 += f * (cx * cx + cy * cy + cz * cz) + g;
  }
  const double ux = jx / rho, uy = jy / rho, uz = jz / rho;
  const double theta = (e2 - rho * (ux * ux + uy * uy + uz * uz)) / (2.0 * a.cv * rho);
  if (a.orho) a.orho[v] = rho;
  if (a.ou) a.ou[v] = ux;
  if (a.ov) a.ov[v] = uy;
  if (a.ow) a.ow[v] = uz;
  if (a.oT) a.oT[v] = theta;
  if (!(rho > 0.0 && theta > 0.0 && isfinite(rho) && isfinite(theta))) atomicOr(a.flag, 1);
}

__global__ void coords3d_kernel(AxisK ax, AxisK ay, AxisK az, double* x, double* y, double* z) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nv = (long long)ax.nv * ay.nv * az.nv;
  if (v >= nv) return;
  const int ix = (int)(v % ax.nv);
  const long long t = v / ax.nv;
  x[v] = vertex_ref_coord(ix, ax);
  y[v] = vertex_ref_coord((int)(t % ay.nv), ay);
  z[v] = vertex_ref_coord((int)(t / ay.nv), az);
}

// D1Q5 in Table I order and he[k][a] = He_k(xi_a) / k! (recurrence He_{k+1} = x He_k - k He_{k-1}).
void d1q5_consts(Consts& cs) {
  cs = Consts{};
  const double s10 = sqrt(10.0), sm = sqrt(5.0 - s10), lg = sqrt(5.0 + s10);
  const double xi[5] = {0.0, sm, lg, -sm, -lg};
  const double w[5] = {8.0 / 15.0, (7.0 + 2.0 * s10) / 60.0, (7.0 - 2.0 * s10) / 60.0,
                       (7.0 + 2.0 * s10) / 60.0, (7.0 - 2.0 * s10) / 60.0};
  cs.nq1 = kQ1;
  for (int a = 0; a < kQ1; ++a) {
    cs.xi[a] = xi[a];
    cs.w[a] = w[a];
    double hm1 = 0.0, h = 1.0, fact = 1.0;
    for (int k = 0; k < kQ1; ++k) {
      if (k > 0) fact *= k;
      cs.he[k][a] = h / fact;
      const double hn = xi[a] * h - k * hm1;
      hm1 = h;
      h = hn;
    }
    cs.xif[a] = (float)xi[a];
    cs.wf[a] = (float)w[a];
    for (int k = 0; k < kQ1; ++k) {
      cs.hef[k][a] = (float)cs.he[k][a];
      cs.whf[k][a] = (float)(cs.w[a] * cs.he[k][a]);
    }
  }
  cs.inv_xi1f = (float)(1.0 / xi[1]);
  cs.xi1sqf = (float)(xi[1] * xi[1]);
}

void axis3(AxisK& ax, int n_cells, int p, double lo, double hi, int periodic, int nodes) {
  ax = AxisK{};
  ax.n_cells = n_cells;
  ax.p = p;
  ax.periodic = periodic;
  ax.nv = periodic ? n_cells * p : n_cells * p + 1;
  ax.lo = lo;
  ax.hi = hi;
  ax.len = hi - lo;
  ax.hc = (hi - lo) / n_cells;
  const double pi = 3.141592653589793238462643383279502884;
  for (int k = 0; k <= p; ++k)   // Gauss-Lobatto-Chebyshev points (Sec. II.E) or equidistant
    ax.nodes[k] = nodes == SLLBM_NODES_GLC ? 0.5 * (1.0 - cos(k * pi / p)) : (double)k / p;
}

}  // namespace

struct sllbm3d_ctx {
  sllbm_grid3_desc g;
  sllbm_params p;
  cudaStream_t stream = nullptr;
  AxisK ax{}, ay{}, az{};
  Consts cs{};
  int npop = 2;
  bool f32 = false;                      // FP32 deviation pairs (else FP64 full populations)
  long long nv = 0;
  double* state[2] = {nullptr, nullptr}; // FP32: reinterpreted as float2 [125][nv]
  int cur = 0;
  bool precomputed = false, initialized = false;
  int* off[3] = {nullptr, nullptr, nullptr};
  float* w32[3] = {nullptr, nullptr, nullptr};
  double* w64[3] = {nullptr, nullptr, nullptr};
  int* flag = nullptr;
  std::vector<void*> allocations;
  std::string err;
};

namespace {

sllbm_status fail3(sllbm3d_ctx* c, sllbm_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

sllbm_status cuda3(sllbm3d_ctx* c, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return SLLBM_OK;
  return fail3(c, SLLBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

template <typename T>
sllbm_status alloc3(sllbm3d_ctx* c, T** ptr, size_t count) {
  void* p = nullptr;
  const cudaError_t e = cudaMalloc(&p, (count ? count : 1) * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail3(c, SLLBM_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  }
  c->allocations.push_back(p);
  *ptr = static_cast<T*>(p);
  return SLLBM_OK;
}

unsigned blocks_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// storage of one state buffer in 8-byte units: FP64 populations or FP32 (f, g) pairs
size_t state_doubles(const sllbm3d_ctx* c) { return (size_t)(c->f32 ? 1 : c->npop) * kQ3 * c->nv; }
// doubles of the dense FP64 layout exchanged by get_state / set_state
size_t dense_doubles(const sllbm3d_ctx* c) { return (size_t)c->npop * kQ3 * c->nv; }
float2* pairs(const sllbm3d_ctx* c, int k) { return reinterpret_cast<float2*>(c->state[k]); }

}  // namespace

extern "C" {

sllbm_status sllbm3d_create(const sllbm_grid3_desc* g, const sllbm_params* p, void* stream, sllbm3d_ctx** out) {
  if (!g || !p || !out) return SLLBM_ERR_ARG;
  *out = nullptr;
  if (g->order < 1 || g->order > 4) return SLLBM_ERR_UNSUPPORTED;
  if (p->velset != SLLBM_VEL_D3Q125 || (p->prec != SLLBM_PREC_F64_PLAIN && p->prec != SLLBM_PREC_F32))
    return SLLBM_ERR_UNSUPPORTED;
  if (p->pr != 0.0 && p->pr != 1.0) return SLLBM_ERR_UNSUPPORTED;
  if (g->nx_cells < 1 || g->ny_cells < 1 || g->nz_cells < 1 || !(g->x1 > g->x0) || !(g->y1 > g->y0) ||
      !(g->z1 > g->z0))
    return SLLBM_ERR_ARG;
  for (int bc : {g->bc_x, g->bc_y, g->bc_z})
    if (bc != SLLBM_BC_PERIODIC && bc != SLLBM_BC_ZERO_GRADIENT) return SLLBM_ERR_ARG;
  if (g->nodes != SLLBM_NODES_GLC && g->nodes != SLLBM_NODES_EQUIDISTANT) return SLLBM_ERR_ARG;
  if (!(p->dt > 0.0) || !(p->tau > 0.5) || !(p->cv >= 1.5) || p->T0 != 1.0) return SLLBM_ERR_ARG;
  if (p->isothermal != 0 && (p->isothermal != 1 || p->cv != 1.5)) return SLLBM_ERR_ARG;
  const long long nvx = (long long)g->nx_cells * g->order + 1, nvy = (long long)g->ny_cells * g->order + 1,
                  nvz = (long long)g->nz_cells * g->order + 1;
  if (nvx > (1 << 16) || nvy > (1 << 16) || nvz > (1 << 16) || nvx * nvy * nvz > (1LL << 27))
    return SLLBM_ERR_UNSUPPORTED;   // 125 x 2 doubles a vertex: keep the state within the device
  sllbm3d_ctx* c = new (std::nothrow) sllbm3d_ctx();
  if (!c) return SLLBM_ERR_OOM;
  c->g = *g;
  c->p = *p;
  c->stream = static_cast<cudaStream_t>(stream);
  d1q5_consts(c->cs);
  axis3(c->ax, g->nx_cells, g->order, g->x0, g->x1, g->bc_x == SLLBM_BC_PERIODIC, g->nodes);
  axis3(c->ay, g->ny_cells, g->order, g->y0, g->y1, g->bc_y == SLLBM_BC_PERIODIC, g->nodes);
  axis3(c->az, g->nz_cells, g->order, g->z0, g->z1, g->bc_z == SLLBM_BC_PERIODIC, g->nodes);
  c->nv = (long long)c->ax.nv * c->ay.nv * c->az.nv;
  c->npop = p->cv == 1.5 ? 1 : 2;
  c->f32 = p->prec == SLLBM_PREC_F32;
  sllbm_status s = SLLBM_OK;
  for (int k = 0; k < 2 && s == SLLBM_OK; ++k) s = alloc3(c, &c->state[k], state_doubles(c));
  if (s == SLLBM_OK) s = alloc3(c, &c->flag, 1);
  if (s == SLLBM_OK) s = cuda3(c, cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream), "cudaMemsetAsync");
  if (s != SLLBM_OK) {
    sllbm3d_destroy(c);
    return s;
  }
  *out = c;
  return SLLBM_OK;
}

sllbm_status sllbm3d_destroy(sllbm3d_ctx* c) {
  if (!c) return SLLBM_ERR_ARG;
  if (c->stream || !c->allocations.empty()) cudaStreamSynchronize(c->stream);
  for (void* p : c->allocations) cudaFree(p);
  delete c;
  return SLLBM_OK;
}

sllbm_status sllbm3d_grid_info(const sllbm3d_ctx* c, int* nx, int* ny, int* nz, int* npop) {
  if (!c) return SLLBM_ERR_ARG;
  if (nx) *nx = c->ax.nv;
  if (ny) *ny = c->ay.nv;
  if (nz) *nz = c->az.nv;
  if (npop) *npop = c->npop;
  return SLLBM_OK;
}

sllbm_status sllbm3d_vertex_coords(sllbm3d_ctx* c, double* x, double* y, double* z) {
  if (!c || !x || !y || !z) return fail3(c, SLLBM_ERR_ARG, "null pointer");
  coords3d_kernel<<<blocks_for(c->nv, 128), 128, 0, c->stream>>>(c->ax, c->ay, c->az, x, y, z);
  return cuda3(c, cudaGetLastError(), "coords3d_kernel");
}

sllbm_status sllbm3d_precompute_departures(sllbm3d_ctx* c) {
  if (!c) return SLLBM_ERR_ARG;
  const AxisK* axes[3] = {&c->ax, &c->ay, &c->az};
  for (int k = 0; k < 3; ++k) {
    const size_t n = (size_t)kQ1 * axes[k]->nv;
    if (!c->off[k]) {
      sllbm_status s = alloc3(c, &c->off[k], n);
      if (s == SLLBM_OK) s = alloc3(c, &c->w32[k], n * (c->g.order + 1));
      if (s == SLLBM_OK) s = alloc3(c, &c->w64[k], n * (c->g.order + 1));
      if (s != SLLBM_OK) return s;
    }
    const sllbm_status s = cuda3(c, launch_axis_tables(*axes[k], c->cs, c->p.dt, c->off[k], c->w32[k], c->w64[k],
                                                       c->stream), "launch_axis_tables");
    if (s != SLLBM_OK) return s;
  }
  c->precomputed = true;
  return SLLBM_OK;
}

sllbm_status sllbm3d_init_equilibrium(sllbm3d_ctx* c, const double* rho, const double* u, const double* v,
                                      const double* w, const double* T) {
  if (!c || !rho || !u || !v || !w || !T) return fail3(c, SLLBM_ERR_ARG, "null pointer");
  if (!c->precomputed) return fail3(c, SLLBM_ERR_STATE, "precompute_departures first");
  Field3Args a{};
  a.rho = rho;
  a.u = u;
  a.v = v;
  a.w = w;
  a.T = T;
  a.state = c->state[c->cur];
  a.state32 = c->f32 ? pairs(c, c->cur) : nullptr;
  a.nv = c->nv;
  a.cs = c->cs;
  a.K = 2.0 * c->p.cv - 3.0;
  a.cv = c->p.cv;
  a.npop = c->npop;
  init3d_kernel<<<blocks_for(c->nv, 128), 128, 0, c->stream>>>(a);
  const sllbm_status s = cuda3(c, cudaGetLastError(), "init3d_kernel");
  if (s == SLLBM_OK) c->initialized = true;
  return s;
}

sllbm_status sllbm3d_step(sllbm3d_ctx* c, int nsteps) {
  if (!c || nsteps < 0) return fail3(c, SLLBM_ERR_ARG, "bad arguments");
  if (!c->precomputed || !c->initialized) return fail3(c, SLLBM_ERR_STATE, "precompute and init first");
  Step3Args a{};
  a.nx = c->ax.nv;
  a.ny = c->ay.nv;
  a.nz = c->az.nv;
  a.nv = c->nv;
  a.px = c->ax.periodic;
  a.py = c->ay.periodic;
  a.pz = c->az.periodic;
  a.offx = c->off[0];
  a.offy = c->off[1];
  a.offz = c->off[2];
  a.wx = c->w64[0];
  a.wy = c->w64[1];
  a.wz = c->w64[2];
  a.cs = c->cs;
  a.omega = 1.0 / c->p.tau;
  a.K = 2.0 * c->p.cv - 3.0;
  a.cv = c->p.cv;
  a.npop = c->npop;
  a.iso = c->p.isothermal;
  a.flag = c->flag;
  const unsigned blocks = blocks_for(c->nv, 128);
  if (c->f32) {
    Step3F32Args b{};
    b.nx = a.nx;
    b.ny = a.ny;
    b.nz = a.nz;
    b.nv = a.nv;
    b.px = a.px;
    b.py = a.py;
    b.pz = a.pz;
    b.offx = a.offx;
    b.offy = a.offy;
    b.offz = a.offz;
    b.wx = c->w32[0];
    b.wy = c->w32[1];
    b.wz = c->w32[2];
    b.cs = c->cs;
    b.omega = (float)a.omega;
    b.K = (float)a.K;
    b.cv = (float)a.cv;
    b.inv2cv = (float)(0.5 / a.cv);
    b.npop = a.npop;
    b.iso = a.iso;
    b.flag = a.flag;
    for (int k = 0; k < nsteps; ++k) {
      b.src = pairs(c, c->cur);
      b.dst = pairs(c, c->cur ^ 1);
      switch (c->g.order) {
        case 1: step3d_f32_kernel<1><<<blocks, 128, 0, c->stream>>>(b); break;
        case 2: step3d_f32_kernel<2><<<blocks, 128, 0, c->stream>>>(b); break;
        case 3: step3d_f32_kernel<3><<<blocks, 128, 0, c->stream>>>(b); break;
        default: step3d_f32_kernel<4><<<blocks, 128, 0, c->stream>>>(b); break;
      }
      const sllbm_status s = cuda3(c, cudaGetLastError(), "step3d_f32_kernel");
      if (s != SLLBM_OK) return s;
      c->cur ^= 1;
    }
    return SLLBM_OK;
  }
  for (int k = 0; k < nsteps; ++k) {
    a.src = c->state[c->cur];
    a.dst = c->state[c->cur ^ 1];
    switch (c->g.order) {
      case 1: step3d_f64_kernel<1><<<blocks, 128, 0, c->stream>>>(a); break;
      case 2: step3d_f64_kernel<2><<<blocks, 128, 0, c->stream>>>(a); break;
      case 3: step3d_f64_kernel<3><<<blocks, 128, 0, c->stream>>>(a); break;
      default: step3d_f64_kernel<4><<<blocks, 128, 0, c->stream>>>(a); break;
    }
    const sllbm_status s = cuda3(c, cudaGetLastError(), "step3d_f64_kernel");
    if (s != SLLBM_OK) return s;
    c->cur ^= 1;
  }
  return SLLBM_OK;
}

sllbm_status sllbm3d_moments(sllbm3d_ctx* c, double* rho, double* u, double* v, double* w, double* T) {
  if (!c) return SLLBM_ERR_ARG;
  if (!c->initialized) return fail3(c, SLLBM_ERR_STATE, "init first");
  Field3Args a{};
  a.orho = rho;
  a.ou = u;
  a.ov = v;
  a.ow = w;
  a.oT = T;
  a.state = c->state[c->cur];
  a.state32 = c->f32 ? pairs(c, c->cur) : nullptr;
  a.nv = c->nv;
  a.cs = c->cs;
  a.K = 2.0 * c->p.cv - 3.0;
  a.cv = c->p.cv;
  a.npop = c->npop;
  a.flag = c->flag;
  moments3d_kernel<<<blocks_for(c->nv, 128), 128, 0, c->stream>>>(a);
  sllbm_status s = cuda3(c, cudaGetLastError(), "moments3d_kernel");
  if (s != SLLBM_OK) return s;
  int flag = 0;
  s = cuda3(c, cudaMemcpyAsync(&flag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "cudaMemcpyAsync");
  if (s == SLLBM_OK) s = cuda3(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  if (s != SLLBM_OK) return s;
  return (flag & 1) ? fail3(c, SLLBM_ERR_UNSTABLE, "non-positive or non-finite density or temperature") : SLLBM_OK;
}

sllbm_status sllbm3d_get_state(sllbm3d_ctx* c, double* dst) {
  if (!c || !dst) return fail3(c, SLLBM_ERR_ARG, "null pointer");
  if (c->f32) {
    convert3d_kernel<<<blocks_for((long long)kQ3 * c->nv, 256), 256, 0, c->stream>>>(
        pairs(c, c->cur), dst, c->nv, c->npop, 2.0 * c->p.cv - 3.0, c->cs, 1);
    return cuda3(c, cudaGetLastError(), "convert3d_kernel");
  }
  return cuda3(c, cudaMemcpyAsync(dst, c->state[c->cur], state_doubles(c) * sizeof(double), cudaMemcpyDeviceToDevice,
                                  c->stream), "cudaMemcpyAsync");
}

sllbm_status sllbm3d_set_state(sllbm3d_ctx* c, const double* src) {
  if (!c || !src) return fail3(c, SLLBM_ERR_ARG, "null pointer");
  if (c->f32) {
    convert3d_kernel<<<blocks_for((long long)kQ3 * c->nv, 256), 256, 0, c->stream>>>(
        pairs(c, c->cur), const_cast<double*>(src), c->nv, c->npop, 2.0 * c->p.cv - 3.0, c->cs, 0);
    const sllbm_status s = cuda3(c, cudaGetLastError(), "convert3d_kernel");
    if (s == SLLBM_OK) c->initialized = true;
    return s;
  }
  const sllbm_status s = cuda3(c, cudaMemcpyAsync(c->state[c->cur], src, state_doubles(c) * sizeof(double),
                                                  cudaMemcpyDeviceToDevice, c->stream), "cudaMemcpyAsync");
  if (s == SLLBM_OK) c->initialized = true;
  return s;
}

const char* sllbm3d_last_error(const sllbm3d_ctx* c) { return c ? c->err.c_str() : "null context"; }

}  // extern "C"
