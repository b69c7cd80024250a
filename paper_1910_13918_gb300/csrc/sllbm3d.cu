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
  double* state;
  long long nv;
  Consts cs;
  double K, cv;
  int npop;
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
    a.state[(size_t)i * plane + v] = feq;
    if (a.npop == 2) a.state[(size_t)(kQ3 + i) * plane + v] = a.K * theta * feq;
  }
}

__global__ void moments3d_kernel(const __grid_constant__ Field3Args a) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= a.nv) return;
  const size_t plane = (size_t)a.nv;
  double rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0, e2 = 0.0;
  for (int i = 0; i < kQ3; ++i) {
    const double f = a.state[(size_t)i * plane + v];
    const double g = a.npop == 2 ? a.state[(size_t)(kQ3 + i) * plane + v] : 0.0;
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
    for (int k = 0; k < kQ1; ++k) cs.hef[k][a] = (float)cs.he[k][a];
  }
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
  long long nv = 0;
  double* state[2] = {nullptr, nullptr};
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

size_t state_doubles(const sllbm3d_ctx* c) { return (size_t)c->npop * kQ3 * c->nv; }

}  // namespace

extern "C" {

sllbm_status sllbm3d_create(const sllbm_grid3_desc* g, const sllbm_params* p, void* stream, sllbm3d_ctx** out) {
  if (!g || !p || !out) return SLLBM_ERR_ARG;
  *out = nullptr;
  if (g->order < 1 || g->order > 4) return SLLBM_ERR_UNSUPPORTED;
  if (p->velset != SLLBM_VEL_D3Q125 || p->prec != SLLBM_PREC_F64_PLAIN) return SLLBM_ERR_UNSUPPORTED;
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
  a.nv = c->nv;
  a.cs = c->cs;
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
  return cuda3(c, cudaMemcpyAsync(dst, c->state[c->cur], state_doubles(c) * sizeof(double), cudaMemcpyDeviceToDevice,
                                  c->stream), "cudaMemcpyAsync");
}

sllbm_status sllbm3d_set_state(sllbm3d_ctx* c, const double* src) {
  if (!c || !src) return fail3(c, SLLBM_ERR_ARG, "null pointer");
  const sllbm_status s = cuda3(c, cudaMemcpyAsync(c->state[c->cur], src, state_doubles(c) * sizeof(double),
                                                  cudaMemcpyDeviceToDevice, c->stream), "cudaMemcpyAsync");
  if (s == SLLBM_OK) c->initialized = true;
  return s;
}

const char* sllbm3d_last_error(const sllbm3d_ctx* c) { return c ? c->err.c_str() : "null context"; }

}  // extern "C"
