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
#include "tma.cuh"

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

// Layout of an FP32 pair state: plane i, vertex (x, y, z) at
// i * plane + origin + (z * rows + y) * pitch + x, with g ghost cells before the interior on
// every axis (g = 0: the dense [125][nz][ny][nx]; the sum-factorised step keeps g = 2 and the
// periodic images in the ghost cells, so that its staged regions never wrap).
struct Pad3 {
  int g, pitch, rows;
  size_t plane, origin;
  __host__ __device__ size_t at(int i, int x, int y, int z) const {
    return (size_t)i * plane + origin + ((size_t)z * rows + y) * pitch + x;
  }
};

struct Field3Args {
  const double *rho, *u, *v, *w, *T;     // init inputs
  double *orho, *ou, *ov, *ow, *oT;      // moment outputs
  double* state;                         // FP64: full populations [npop][125][nv]
  float2* state32;                       // FP32: (f - w, g - K w) pairs in layout lay (else null)
  Pad3 lay;
  int nx, ny;
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

// ---- sum-factorised FP32 step (orders 1 and 2; an even number of x vertices, so that the
// pair rows are whole 16-byte units for the tensor copies) ----
//
// Three launches a step.  stream3d_kernel: a CTA takes a tile of 32 x 8 x 4 vertices (two CTAs
// an SM) and walks the
// 125 velocity planes; per plane one TMA tensor copy brings the source region (the tile and the
// stencil halo: x0 - 2 .. x0 + 33, and p on both sides in y and z), one plane ahead in two
// stages.  The state keeps 2 ghost cells on every axis, holding the periodic images on periodic
// axes (zero, and never read by an interior vertex, on zero-gradient ones), so a region never
// wraps.  The interpolation is sum-factorised: z pass over the region's (y, x) columns, y pass
// over the tile's z and the region's x, x pass into the destination, each in a centred tail-sum
// form
//   sum_d W_d v_{c+d} = v_c + sum_{j=1..p} T+_j (v_{c+j} - v_{c+j-1}) - sum_{j=1..p} T-_j (v_{c-j+1} - v_{c-j}),
//   T+_j = sum_{d >= j} W_d, T-_j = sum_{d <= -j} W_d  (d the offset from the vertex, W_d its weight),
// equal to the Lagrange sum because the weights sum to one and exact for constant fields in FP32.
// The tile's tail sums of all five components are loaded once.  The thread of a vertex in the x
// pass sums its moments over the 125 planes.  collide3d_kernel then relaxes every vertex's 125
// pairs in place and writes the periodic images of the vertices next to periodic faces.
constexpr int kT3X = 32, kT3Y = 8, kT3Z = 4, kT3NT = 256;
constexpr int kT3XO = 2;   // the region starts at x0 - 2: 16-byte aligned for both orders
constexpr int kT3G = 2;    // ghost cells of the state on every axis (>= the halo of p <= 2)

template <int P>
struct T3Shape {
  static constexpr int RX = kT3X + 2 * kT3XO, RY = kT3Y + 2 * P, RZ = kT3Z + 2 * P;
  static constexpr int RE = RX * RY * RZ;   // region pairs
  static constexpr int NW = 2 * P;          // tail sums per (component, node): T+_1..p, -T-_1..p
  static constexpr int ZT = RY * RX;        // z-pass columns
  static constexpr int YT = kT3Z * RX;      // y-pass columns
  static constexpr int NWT = kQ1 * (kT3Z + kT3Y + kT3X) * NW;   // the tile's tail sums
  static constexpr size_t kStage = sizeof(float2) * RE;
  static constexpr size_t kBytes = 128 + 2 * kStage +
                                   sizeof(float2) * (size_t)(kT3Z * RY * RX + kT3Z * kT3Y * RX) +
                                   sizeof(float) * NWT + sizeof(uint64_t) * 2;
  static_assert(kStage % 128 == 0, "stages stay 128-byte aligned");
  static constexpr int XR = kT3Y * kT3Z / (kT3NT / 32);   // x-pass rows per warp
  static_assert(YT <= kT3NT && XR * (kT3NT / 32) == kT3Y * kT3Z, "one y column a thread, whole x rows a warp");
  static_assert(P <= kT3G && kT3XO <= kT3G, "the halo stays within the ghost cells");
};

struct Stream3Args {
  const float2* src;     // pairs in layout lay (deviations)
  float2* dst;
  Pad3 lay;
  float* sums;           // [6][nv]: sum f, sum f xi_x, sum f xi_y, sum f xi_z, sum f |xi|^2, sum g
  int nx, ny, nz;
  long long nv;
  const float* tx;       // [5][nx][2p] tail sums per (component, node)
  const float* ty;
  const float* tz;
  Consts cs;
  int* flag;             // bit 2: a staging copy timed out
};

// centred tail-sum interpolation at window position c (see above); w = T+_1..p, -T-_1..p
template <int P, int N>
__device__ __forceinline__ float2 tail_interp(const float2 (&v)[N], const float2 (&d)[N - 1], int c, const float* w) {
  float2 acc = v[c];
#pragma unroll
  for (int j = 1; j <= P; ++j) {
    acc = fma2(bcast2(w[j - 1]), d[c + j - 1], acc);
    acc = fma2(bcast2(w[P + j - 1]), d[c - j], acc);
  }
  return acc;
}

template <int P>
__global__ void __launch_bounds__(kT3NT, 2) stream3d_kernel(const __grid_constant__ Stream3Args a,
                                                            const __grid_constant__ CUtensorMap smap) {
  using SH = T3Shape<P>;
  constexpr int RX = SH::RX, RY = SH::RY, RZ = SH::RZ, RE = SH::RE, NW = SH::NW;
  extern __shared__ unsigned char s3_smem[];
  unsigned char* base = s3_smem + ((128 - (smem_u32(s3_smem) & 127)) & 127);
  float2* S = reinterpret_cast<float2*>(base);                         // [2][RZ][RY][RX]
  float2* Zb = S + 2 * RE;                                             // [TZ][RY][RX]
  float2* Yb = Zb + kT3Z * RY * RX;                                    // [TZ][TY][RX]
  float* Wz = reinterpret_cast<float*>(Yb + kT3Z * kT3Y * RX);         // [5][TZ][NW]
  float* Wy = Wz + kQ1 * kT3Z * NW;                                    // [5][TY][NW]
  float* Wx = Wy + kQ1 * kT3Y * NW;                                    // [5][TX][NW]
  uint64_t* BAR = reinterpret_cast<uint64_t*>(Wx + kQ1 * kT3X * NW);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tiles_x = (a.nx + kT3X - 1) / kT3X, tiles_y = (a.ny + kT3Y - 1) / kT3Y;
  const int byz = (int)blockIdx.x / tiles_x;
  const int x0 = ((int)blockIdx.x - byz * tiles_x) * kT3X, y0 = (byz % tiles_y) * kT3Y,
            z0 = (byz / tiles_y) * kT3Z;
  // the tile's tail sums of all components (nodes past the grid clamped: those outputs are not
  // stored)
  for (int e = tid; e < SH::NWT; e += kT3NT) {
    const int q = e % NW, r = e / NW;
    float t;
    if (r < kQ1 * kT3Z) {
      const int c = r / kT3Z, n = min(z0 + r - c * kT3Z, a.nz - 1);
      t = __ldg(a.tz + ((size_t)c * a.nz + n) * NW + q);
    } else if (r < kQ1 * (kT3Z + kT3Y)) {
      const int r2 = r - kQ1 * kT3Z, c = r2 / kT3Y, n = min(y0 + r2 - c * kT3Y, a.ny - 1);
      t = __ldg(a.ty + ((size_t)c * a.ny + n) * NW + q);
    } else {
      const int r2 = r - kQ1 * (kT3Z + kT3Y), c = r2 / kT3X, n = min(x0 + r2 - c * kT3X, a.nx - 1);
      t = __ldg(a.tx + ((size_t)c * a.nx + n) * NW + q);
    }
    Wz[e] = t;   // Wz, Wy and Wx are consecutive
  }
  if (tid == 0) {
    mbar_init(&BAR[0], 1);
    mbar_init(&BAR[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  // region origin in the ghost-padded layout: x0 - 2 + g (x in floats: 2 (x0 - 2 + g), a multiple
  // of 4, i.e. 16 bytes), y0 - p + g, z0 - p + g
  const int cx = 2 * (x0 - kT3XO + a.lay.g), cy = y0 - P + a.lay.g, cz = z0 - P + a.lay.g;
  auto issue = [&](int i, int st) {   // thread 0: plane i into stage st
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_expect_tx(&BAR[st], (unsigned)SH::kStage);
    tma_load_4d(S + (size_t)st * RE, &smap, cx, cy, cz, i, &BAR[st]);
  };
  if (tid == 0) issue(0, 0);
  // x pass: warp w takes the tile rows XR w .. XR w + XR - 1 (row r: z = r / TY, y = r % TY),
  // lane = x
  constexpr int XR = SH::XR;
  const int vx = x0 + lane;
  float m[XR][6];
#pragma unroll
  for (int j = 0; j < XR; ++j)
#pragma unroll
    for (int q = 0; q < 6; ++q) m[j][q] = 0.f;
  float wx[NW];
#pragma unroll 1
  for (int i = 0; i < kQ3; ++i) {
    const int st = i & 1, ia = i / 25, ib = (i / 5) % 5, ic = i % 5;
    const bool late = !mbar_wait(&BAR[st], (unsigned)((i >> 1) & 1), a.flag);
    if (__syncthreads_or(late)) {   // the copy of plane i did not land in time: stop, after it
      mbar_wait(&BAR[st], (unsigned)((i >> 1) & 1), a.flag);
      return;
    }
    if (tid == 0 && i + 1 < kQ3) issue(i + 1, st ^ 1);   // every thread is past plane i - 1
    if (ic == 0 && ib == 0) {   // a new x component: this lane's x tail sums
#pragma unroll
      for (int q = 0; q < NW; ++q) wx[q] = Wx[(ia * kT3X + lane) * NW + q];
    }
    const float2* Sst = S + (size_t)st * RE;
    // z pass: column (ry, rx) of the region, the tile's z rows
    {
      // the plane's z tail sums in registers; a thread's (up to) ZR columns with all loads in flight
      constexpr int ZR = (SH::ZT + kT3NT - 1) / kT3NT;
      float wz[kT3Z * NW];
#pragma unroll
      for (int q = 0; q < kT3Z * NW; ++q) wz[q] = Wz[ic * kT3Z * NW + q];
      float2 v[ZR][RZ];
#pragma unroll
      for (int c = 0; c < ZR; ++c) {
        const int t = tid + c * kT3NT;
        if (t < SH::ZT) {
#pragma unroll
          for (int r = 0; r < RZ; ++r) v[c][r] = Sst[r * RY * RX + t];
        }
      }
#pragma unroll
      for (int c = 0; c < ZR; ++c) {
        const int t = tid + c * kT3NT;
        if (t < SH::ZT) {
          float2 d[RZ - 1];
#pragma unroll
          for (int r = 0; r + 1 < RZ; ++r) d[r] = sub2(v[c][r + 1], v[c][r]);
#pragma unroll
          for (int tz = 0; tz < kT3Z; ++tz) Zb[tz * RY * RX + t] = tail_interp<P>(v[c], d, tz + P, wz + tz * NW);
        }
      }
    }
    __syncthreads();
    // y pass: column (tz, rx), the tile's y rows
    if (tid < SH::YT) {
      const int tz = tid / RX, rx = tid - tz * RX;
      const float* wy = Wy + ib * kT3Y * NW;
      float2 v[RY], d[RY - 1];
#pragma unroll
      for (int r = 0; r < RY; ++r) v[r] = Zb[(tz * RY + r) * RX + rx];
#pragma unroll
      for (int r = 0; r + 1 < RY; ++r) d[r] = sub2(v[r + 1], v[r]);
#pragma unroll
      for (int ty = 0; ty < kT3Y; ++ty) Yb[(tz * kT3Y + ty) * RX + rx] = tail_interp<P>(v, d, ty + P, wy + ty * NW);
    }
    __syncthreads();
    // x pass: the vertex (x0 + lane, row) into the destination; its moments
    const float ex = a.cs.xif[ia], ey = a.cs.xif[ib], ez = a.cs.xif[ic];
    const float e2 = ex * ex + ey * ey + ez * ez;
#pragma unroll
    for (int j = 0; j < XR; ++j) {
      const int r = XR * warp + j, tz = r / kT3Y, ty = r - tz * kT3Y;
      const float2* row = Yb + (tz * kT3Y + ty) * RX + kT3XO + lane;
      float2 v[2 * P + 1], d[2 * P];
#pragma unroll
      for (int k = 0; k <= 2 * P; ++k) v[k] = row[k - P];
#pragma unroll
      for (int k = 0; k < 2 * P; ++k) d[k] = sub2(v[k + 1], v[k]);
      const float2 acc = tail_interp<P>(v, d, P, wx);
      const int vy = y0 + ty, vz = z0 + tz;
      if (vx < a.nx && vy < a.ny && vz < a.nz) {
        a.dst[a.lay.at(i, vx, vy, vz)] = acc;
        m[j][0] += acc.x;
        m[j][1] += ex * acc.x;
        m[j][2] += ey * acc.x;
        m[j][3] += ez * acc.x;
        m[j][4] += e2 * acc.x;
        m[j][5] += acc.y;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < XR; ++j) {
    const int r = XR * warp + j, tz = r / kT3Y, ty = r - tz * kT3Y;
    const int vy = y0 + ty, vz = z0 + tz;
    if (vx < a.nx && vy < a.ny && vz < a.nz) {
      const size_t v = ((size_t)vz * a.ny + vy) * a.nx + vx;
#pragma unroll
      for (int q = 0; q < 6; ++q) a.sums[(size_t)q * a.nv + v] = m[j][q];
    }
  }
}

// Second sweep of the sum-factorised step: one thread per vertex relaxes its 125 pairs in place
// (read back from the destination, a row of 5 ahead), from the moment sums of the stream
// kernel, with the residual correction of step3d_f32_kernel.  ghost_refresh3d_kernel then copies
// the periodic images into the ghost cells.
struct Collide3Args {
  float2* dst;
  Pad3 lay;
  const float* sums;
  int nx, ny, nz, px, py, pz;
  long long nv;
  Consts cs;
  float omega, K, cv, inv2cv;
  int npop, iso;
  int* flag;
};

__global__ void __launch_bounds__(128, 6) collide3d_kernel(const __grid_constant__ Collide3Args a) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= a.nv) return;
  const int x = (int)(v % a.nx), y = (int)((v / a.nx) % a.ny), z = (int)(v / ((long long)a.nx * a.ny));
  const size_t plane = a.lay.plane;
  float2* own = a.dst + a.lay.at(0, x, y, z);
  const size_t sp = (size_t)a.nv;
  const float drho = a.sums[v], jx = a.sums[sp + v], jy = a.sums[2 * sp + v], jz = a.sums[3 * sp + v],
              a2 = a.sums[4 * sp + v];
  const float G = a.npop == 2 ? a.sums[5 * sp + v] : 0.f;
  const float rho = 1.f + drho, inv_rho = __frcp_rn(rho);
  const float ux = jx * inv_rho, uy = jy * inv_rho, uz = jz * inv_rho;
  const float qk = (a2 + G - rho * (ux * ux + uy * uy + uz * uz) - 2.f * a.cv * drho) * inv_rho * a.inv2cv;
  const float q = a.iso ? 0.f : qk;
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
  float Zc[5][5];   // [n][c]: sum_{m <= n} A_m(u_z) he_m(c)
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
  // rows (a, b) of 5 pairs (c = 0..4), the next row's loads in flight while one row relaxes
  float2 cur[kQ1];
#pragma unroll
  for (int ic = 0; ic < kQ1; ++ic) cur[ic] = own[(size_t)ic * plane];
#pragma unroll 1
  for (int row = 0; row < kQ1 * kQ1; ++row) {
    const int ia = row / kQ1, ib = row - kQ1 * ia;
    float2 nxt[kQ1];
    if (row + 1 < kQ1 * kQ1) {
#pragma unroll
      for (int ic = 0; ic < kQ1; ++ic) nxt[ic] = own[(size_t)(kQ1 * (row + 1) + ic) * plane];
    }
    float Xa[5], Yb[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      Xa[k] = Ax[k] * a.cs.hef[k][ia];
      Yb[k] = Ay[k] * a.cs.hef[k][ib];
    }
    const float ex = a.cs.xif[ia], ey = a.cs.xif[ib], wab = a.cs.wf[ia] * a.cs.wf[ib];
    float2* o5 = own + (size_t)(kQ1 * row) * plane;
#pragma unroll
    for (int ic = 0; ic < kQ1; ++ic) {
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
      const float eg = Kq1 * ef + Kq * w;
      const float2 d = sub2(make_float2(ef, a.npop == 2 ? eg : 0.f), cur[ic]);
      const float ez = a.cs.xif[ic];
      r0 += d.x;
      r1 += ex * d.x;
      r2 += ey * d.x;
      r3 += ez * d.x;
      re += (ex * ex + ey * ey + ez * ez) * d.x + d.y;
      o5[(size_t)ic * plane] = fma2(om2, d, cur[ic]);
    }
    if (row + 1 < kQ1 * kQ1) {
#pragma unroll
      for (int ic = 0; ic < kQ1; ++ic) cur[ic] = nxt[ic];
    }
  }
  {
    const float inv_s = a.cs.inv_xi1f, s2 = a.cs.xi1sqf;
    const float d1 = r1 * inv_s, d2 = r2 * inv_s, d3 = r3 * inv_s;
    const float d0 = r0 - d1 - d2 - d3;
    const float de = re - s2 * (d1 + d2 + d3);
    own[0].x -= om * d0;
    own[25 * plane].x -= om * d1;
    own[5 * plane].x -= om * d2;
    own[1 * plane].x -= om * d3;
    if (a.npop == 2) {
      own[0].y -= om * de;
    } else if (!a.iso) {
      const float e = om * 0.5f * de * inv_s * inv_s;
      own[25 * plane].x -= e;
      own[75 * plane].x -= e;
      own[0].x += 2.f * e;
    }
  }
  if (!((rho > 0.f) && (qk > -1.f) && isfinite(rho) && isfinite(qk))) atomicOr(a.flag, 1);
}

// The periodic images of the ghost cells of a padded pair state, one thread per (plane, ghost
// cell).  The ghost cells of a plane are enumerated as three disjoint sets: the 2g slices before
// and after the interior slices (whole rows), then in the interior slices the 2g ghost rows,
// then in the interior rows the 2g ghost columns.  A cell past a zero-gradient face is skipped.
__global__ void __launch_bounds__(256) ghost_refresh3d_kernel(float2* pairs, Pad3 lay, int nx, int ny, int nz,
                                                              int px, int py, int pz, long long per_plane) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)kQ3 * per_plane) return;
  const int i = (int)(e / per_plane);
  long long r = e - (long long)i * per_plane;
  const int g = lay.g, W = lay.pitch, R = lay.rows;
  const long long nzs = 2LL * g * R * W, nys = (long long)nz * 2 * g * W;
  int X, Y, Z;   // interior coordinates of the ghost cell (outside [0, n) on some axis)
  if (r < nzs) {
    const int zz = (int)(r / ((long long)R * W));
    r -= (long long)zz * R * W;
    Z = zz < g ? zz - g : nz + zz - g;
    Y = (int)(r / W) - g;
    X = (int)(r % W) - g;
  } else if ((r -= nzs) < nys) {
    Z = (int)(r / (2LL * g * W));
    r -= (long long)Z * 2 * g * W;
    const int yy = (int)(r / W);
    Y = yy < g ? yy - g : ny + yy - g;
    X = (int)(r % W) - g;
  } else {
    r -= nys;
    Z = (int)(r / ((long long)ny * 2 * g));
    r -= (long long)Z * ny * 2 * g;
    Y = (int)(r / (2 * g));
    const int xx = (int)(r % (2 * g));
    X = xx < g ? xx - g : nx + xx - g;
  }
  const bool ox = X < 0 || X >= nx, oy = Y < 0 || Y >= ny, oz = Z < 0 || Z >= nz;
  if ((ox && !px) || (oy && !py) || (oz && !pz)) return;
  const int x = ox ? (X < 0 ? X + nx : X - nx) : X, y = oy ? (Y < 0 ? Y + ny : Y - ny) : Y,
            z = oz ? (Z < 0 ? Z + nz : Z - nz) : Z;
  pairs[lay.at(i, X, Y, Z)] = pairs[lay.at(i, x, y, z)];
}

// Tail sums T+_j, -T-_j (j = 1..p) of every (component, node) of one axis, from the FP64 tables:
// the stencil of node n starts at n + off and has weights w_0..w_p, offsets d = off + k.
template <int P>
__global__ void tail_table_kernel(const int* off, const double* w, int n, float* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kQ1 * n) return;
  double W[2 * P + 1];
#pragma unroll
  for (int d = 0; d <= 2 * P; ++d) W[d] = 0.0;
  const int o = off[e];
#pragma unroll
  for (int k = 0; k <= P; ++k) W[o + k + P] += w[(size_t)e * (P + 1) + k];   // o + k in [-P, P]
#pragma unroll
  for (int j = 1; j <= P; ++j) {
    double tp = 0.0, tm = 0.0;
    for (int d = j; d <= P; ++d) tp += W[d + P];
    for (int d = -P; d <= -j; ++d) tm += W[d + P];
    out[(size_t)e * 2 * P + j - 1] = (float)tp;
    out[(size_t)e * 2 * P + P + j - 1] = (float)(-tm);
  }
}

// FP32 pairs (layout lay) <-> dense FP64 full populations [npop][125][nv].
__global__ void convert3d_kernel(float2* pairs, Pad3 lay, double* dense, int nx, int ny, long long nv, int npop,
                                 double K, Consts cs, int to_dense) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)kQ3 * nv) return;
  const int i = (int)(e / nv);
  const long long v = e - (long long)i * nv;
  const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((long long)nx * ny));
  const size_t o = lay.at(i, x, y, z);
  const double w = cs.w[i / 25] * cs.w[(i / 5) % 5] * cs.w[i % 5];
  if (to_dense) {
    const float2 p = pairs[o];
    dense[e] = (double)p.x + w;
    if (npop == 2) dense[(size_t)kQ3 * nv + e] = (double)p.y + K * w;
  } else {
    const float f = (float)(dense[e] - w);
    const float g = npop == 2 ? (float)(dense[(size_t)kQ3 * nv + e] - K * w) : 0.f;
    pairs[o] = make_float2(f, g);
  }
}

// Periodic images of a ghost-padded pair state: every ghost cell whose position lies past
// periodic faces only takes the value of the interior vertex it images (ghosts past a
// zero-gradient face stay as they are: zero, never read by an interior vertex).
__global__ void ghost3d_kernel(float2* pairs, Pad3 lay, int nx, int ny, int nz, int px, int py, int pz) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int slices = nz + 2 * lay.g;
  const long long per_plane = (long long)lay.pitch * lay.rows * slices;
  if (e >= (long long)kQ3 * per_plane) return;
  const int i = (int)(e / per_plane);
  const long long r = e - (long long)i * per_plane;
  const int X = (int)(r % lay.pitch) - lay.g, Y = (int)((r / lay.pitch) % lay.rows) - lay.g,
            Z = (int)(r / ((long long)lay.pitch * lay.rows)) - lay.g;
  const bool ox = X < 0 || X >= nx, oy = Y < 0 || Y >= ny, oz = Z < 0 || Z >= nz;
  if (!(ox || oy || oz) || X >= nx + lay.g) return;   // interior, or row padding past the ghosts
  if ((ox && !px) || (oy && !py) || (oz && !pz)) return;
  const int x = ox ? (X < 0 ? X + nx : X - nx) : X, y = oy ? (Y < 0 ? Y + ny : Y - ny) : Y,
            z = oz ? (Z < 0 ? Z + nz : Z - nz) : Z;
  pairs[(size_t)i * lay.plane + r] = pairs[lay.at(i, x, y, z)];
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
  const int x = (int)(v % a.nx), y = (int)((v / a.nx) % a.ny), z = (int)(v / ((long long)a.nx * a.ny));
  for (int i = 0; i < kQ3; ++i) {
    const double feq = eq3(a.cs, rho, Ax, Ay, Az, i / 25, (i / 5) % 5, i % 5);
    if (a.state32) {
      const double w = a.cs.w[i / 25] * a.cs.w[(i / 5) % 5] * a.cs.w[i % 5];
      a.state32[a.lay.at(i, x, y, z)] =
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
  const int x = (int)(v % a.nx), y = (int)((v / a.nx) % a.ny), z = (int)(v / ((long long)a.nx * a.ny));
  double rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0, e2 = 0.0;
  for (int i = 0; i < kQ3; ++i) {
    double f, g;
    if (a.state32) {
      const float2 p = a.state32[a.lay.at(i, x, y, z)];
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
  // sum-factorised FP32 step (orders 1, 2 with an even x count): tail sums per axis, moment sums
  bool tiled = false;
  Pad3 lay{};                            // layout of the FP32 pair state
  float* tail[3] = {nullptr, nullptr, nullptr};
  float* sums = nullptr;
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
size_t state_doubles(const sllbm3d_ctx* c) {
  return c->f32 ? (size_t)kQ3 * c->lay.plane : (size_t)c->npop * kQ3 * c->nv;
}
float2* pairs(const sllbm3d_ctx* c, int k) { return reinterpret_cast<float2*>(c->state[k]); }

// The sum-factorised FP32 step: stream3d_kernel (a CTA per tile) then collide3d_kernel.
template <int P>
cudaError_t launch_stream3d(const Stream3Args& a, cudaStream_t s) {
  using SH = T3Shape<P>;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  // 4D map of the ghost-padded source pairs as floats: (2 x column, row, slice, velocity plane)
  CUtensorMap smap;
  const cuuint64_t dims[4] = {(cuuint64_t)2 * a.lay.pitch, (cuuint64_t)a.lay.rows,
                              (cuuint64_t)(a.lay.plane / ((size_t)a.lay.pitch * a.lay.rows)), (cuuint64_t)kQ3};
  const cuuint64_t strides[3] = {(cuuint64_t)a.lay.pitch * sizeof(float2),
                                 (cuuint64_t)a.lay.pitch * a.lay.rows * sizeof(float2),
                                 (cuuint64_t)a.lay.plane * sizeof(float2)};
  const cuuint32_t box[4] = {(cuuint32_t)(2 * SH::RX), (cuuint32_t)SH::RY, (cuuint32_t)SH::RZ, 1u};
  const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
  if (enc(&smap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float2*>(a.src), dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(stream3d_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SH::kBytes);
  if (e != cudaSuccess) return e;
  const long long tiles = (long long)((a.nx + kT3X - 1) / kT3X) * ((a.ny + kT3Y - 1) / kT3Y) * ((a.nz + kT3Z - 1) / kT3Z);
  stream3d_kernel<P><<<(unsigned)tiles, kT3NT, SH::kBytes, s>>>(a, smap);
  return cudaGetLastError();
}

// The periodic images of the current state's ghost cells (after init and set_state).
cudaError_t fill_ghosts3d(sllbm3d_ctx* c) {
  if (!c->tiled) return cudaSuccess;
  const long long n = (long long)kQ3 * (long long)c->lay.plane;
  ghost3d_kernel<<<blocks_for(n, 256), 256, 0, c->stream>>>(pairs(c, c->cur), c->lay, c->ax.nv, c->ay.nv, c->az.nv,
                                                           c->ax.periodic, c->ay.periodic, c->az.periodic);
  return cudaGetLastError();
}

cudaError_t launch_tiled3d(sllbm3d_ctx* c, const float2* src, float2* dst) {
  Stream3Args a{};
  a.src = src;
  a.dst = dst;
  a.sums = c->sums;
  a.nx = c->ax.nv;
  a.ny = c->ay.nv;
  a.nz = c->az.nv;
  a.nv = c->nv;
  a.lay = c->lay;
  a.tx = c->tail[0];
  a.ty = c->tail[1];
  a.tz = c->tail[2];
  a.cs = c->cs;
  a.flag = c->flag;
  cudaError_t e = c->g.order == 1 ? launch_stream3d<1>(a, c->stream) : launch_stream3d<2>(a, c->stream);
  if (e != cudaSuccess) return e;
  Collide3Args b{};
  b.dst = dst;
  b.lay = c->lay;
  b.sums = c->sums;
  b.nx = c->ax.nv;
  b.ny = c->ay.nv;
  b.nz = c->az.nv;
  b.px = c->ax.periodic;
  b.py = c->ay.periodic;
  b.pz = c->az.periodic;
  b.nv = c->nv;
  b.cs = c->cs;
  b.omega = (float)(1.0 / c->p.tau);
  b.K = (float)(2.0 * c->p.cv - 3.0);
  b.cv = (float)c->p.cv;
  b.inv2cv = (float)(0.5 / c->p.cv);
  b.npop = c->npop;
  b.iso = c->p.isothermal;
  b.flag = c->flag;
  collide3d_kernel<<<blocks_for(c->nv, 128), 128, 0, c->stream>>>(b);
  cudaError_t e2 = cudaGetLastError();
  if (e2 != cudaSuccess) return e2;
  const long long per_plane = (long long)c->lay.plane - c->nv;   // ghost cells of a plane
  ghost_refresh3d_kernel<<<blocks_for((long long)kQ3 * per_plane, 256), 256, 0, c->stream>>>(
      dst, c->lay, b.nx, b.ny, b.nz, b.px, b.py, b.pz, per_plane);
  return cudaGetLastError();
}

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
  // the sum-factorised FP32 step: orders 1, 2, an even x count (16-byte pair rows), and axes at
  // least as long as its staged region (36 x 12 x 8 vertices); its state keeps ghost cells
  c->tiled = c->f32 && g->order <= 2 && c->ax.nv % 2 == 0 && c->ax.nv >= T3Shape<2>::RX &&
             c->ay.nv >= T3Shape<2>::RY && c->az.nv >= T3Shape<2>::RZ && encode_fn() != nullptr;
  {
    Pad3& L = c->lay;
    L.g = c->tiled ? kT3G : 0;
    L.pitch = c->ax.nv + 2 * L.g;
    L.rows = c->ay.nv + 2 * L.g;
    L.plane = (size_t)L.pitch * L.rows * (c->az.nv + 2 * L.g);
    L.origin = ((size_t)L.g * L.rows + L.g) * L.pitch + L.g;
  }
  sllbm_status s = SLLBM_OK;
  for (int k = 0; k < 2 && s == SLLBM_OK; ++k) s = alloc3(c, &c->state[k], state_doubles(c));
  for (int k = 0; k < 2 && s == SLLBM_OK && c->tiled; ++k)   // ghosts of zero-gradient faces stay 0
    s = cuda3(c, cudaMemsetAsync(c->state[k], 0, state_doubles(c) * sizeof(double), c->stream), "cudaMemsetAsync");
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
  if (c->tiled) {
    const int P = c->g.order;
    for (int k = 0; k < 3; ++k) {
      const int n = axes[k]->nv;
      if (!c->tail[k]) {
        const sllbm_status s = alloc3(c, &c->tail[k], (size_t)kQ1 * n * 2 * P);
        if (s != SLLBM_OK) return s;
      }
      if (P == 1)
        tail_table_kernel<1><<<blocks_for((long long)kQ1 * n, 128), 128, 0, c->stream>>>(c->off[k], c->w64[k], n, c->tail[k]);
      else
        tail_table_kernel<2><<<blocks_for((long long)kQ1 * n, 128), 128, 0, c->stream>>>(c->off[k], c->w64[k], n, c->tail[k]);
      const sllbm_status s = cuda3(c, cudaGetLastError(), "tail_table_kernel");
      if (s != SLLBM_OK) return s;
    }
    if (!c->sums) {
      const sllbm_status s = alloc3(c, &c->sums, (size_t)6 * c->nv);
      if (s != SLLBM_OK) return s;
    }
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
  a.lay = c->lay;
  a.nx = c->ax.nv;
  a.ny = c->ay.nv;
  a.nv = c->nv;
  a.cs = c->cs;
  a.K = 2.0 * c->p.cv - 3.0;
  a.cv = c->p.cv;
  a.npop = c->npop;
  init3d_kernel<<<blocks_for(c->nv, 128), 128, 0, c->stream>>>(a);
  sllbm_status s = cuda3(c, cudaGetLastError(), "init3d_kernel");
  if (s == SLLBM_OK) s = cuda3(c, fill_ghosts3d(c), "ghost3d_kernel");
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
      if (c->tiled) {
        const sllbm_status s = cuda3(c, launch_tiled3d(c, pairs(c, c->cur), pairs(c, c->cur ^ 1)), "stream3d/collide3d");
        if (s != SLLBM_OK) return s;
        c->cur ^= 1;
        continue;
      }
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

const char* sllbm3d_step_kernel_name(const sllbm3d_ctx* c) {
  if (!c) return "";
  return !c->f32 ? "plain_f64" : (c->tiled ? "stream3d" : "gather_f32");
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
  a.lay = c->lay;
  a.nx = c->ax.nv;
  a.ny = c->ay.nv;
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
  if (flag & 4) return fail3(c, SLLBM_ERR_CUDA, "a staging copy of the 3D stream kernel timed out");
  return (flag & 1) ? fail3(c, SLLBM_ERR_UNSTABLE, "non-positive or non-finite density or temperature") : SLLBM_OK;
}

sllbm_status sllbm3d_get_state(sllbm3d_ctx* c, double* dst) {
  if (!c || !dst) return fail3(c, SLLBM_ERR_ARG, "null pointer");
  if (c->f32) {
    convert3d_kernel<<<blocks_for((long long)kQ3 * c->nv, 256), 256, 0, c->stream>>>(
        pairs(c, c->cur), c->lay, dst, c->ax.nv, c->ay.nv, c->nv, c->npop, 2.0 * c->p.cv - 3.0, c->cs, 1);
    return cuda3(c, cudaGetLastError(), "convert3d_kernel");
  }
  return cuda3(c, cudaMemcpyAsync(dst, c->state[c->cur], state_doubles(c) * sizeof(double), cudaMemcpyDeviceToDevice,
                                  c->stream), "cudaMemcpyAsync");
}

sllbm_status sllbm3d_set_state(sllbm3d_ctx* c, const double* src) {
  if (!c || !src) return fail3(c, SLLBM_ERR_ARG, "null pointer");
  if (c->f32) {
    convert3d_kernel<<<blocks_for((long long)kQ3 * c->nv, 256), 256, 0, c->stream>>>(
        pairs(c, c->cur), c->lay, const_cast<double*>(src), c->ax.nv, c->ay.nv, c->nv, c->npop,
        2.0 * c->p.cv - 3.0, c->cs, 0);
    sllbm_status s = cuda3(c, cudaGetLastError(), "convert3d_kernel");
    if (s == SLLBM_OK) s = cuda3(c, fill_ghosts3d(c), "ghost3d_kernel");
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
