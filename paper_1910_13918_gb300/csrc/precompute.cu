// FP64 precompute kernels of the SLLBM: departure points and Lagrange weights (Eq. streaming_fg,
// Eq. sl_streaming), vertex coordinates and quadrature weights (Sec. II.E), and the equilibrium
// initial state (Sec. II.A, II.D).
#include "kernels.h"

namespace sllbm {

// ------------------------------------------------------------------------------------------
// Uniform grids: the departure of vertex j along one axis for velocity component c is
// x_j - dt xi_c; it depends on (c, j) only, so each axis gets a table [nq1][nv] of the stencil
// start offset (start - j) and p+1 Lagrange weights.
// ------------------------------------------------------------------------------------------
template <int P>
__global__ void axis_table_kernel(AxisK ax, Consts cs, double dt, int* off, float* w32, double* w64) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cs.nq1 * ax.nv) return;
  const int c = t / ax.nv, j = t % ax.nv;
  const double x = vertex_ref_coord(j, ax);
  const double xd = fold_axis(x - dt * cs.xi[c], ax);
  int cell;
  double r;
  locate_axis(xd, ax, &cell, &r);
  double psi[P + 1];
  lagrange_basis<P, double>(ax.nodes, r, psi);
  int o = cell * P - j;
  if (ax.periodic) {  // shortest unwrapped offset
    if (o > ax.nv / 2) o -= ax.nv;
    if (o < -ax.nv / 2) o += ax.nv;
  }
  off[t] = o;
#pragma unroll
  for (int k = 0; k <= P; ++k) {
    w64[(size_t)t * (P + 1) + k] = psi[k];
    w32[(size_t)t * (P + 1) + k] = (float)psi[k];
  }
}

cudaError_t launch_axis_tables(const AxisK& ax, const Consts& cs, double dt, int* off, float* w32,
                               double* w64, cudaStream_t s) {
  const int n = cs.nq1 * ax.nv, threads = 128, blocks = (n + threads - 1) / threads;
  switch (ax.p) {
    case 1: axis_table_kernel<1><<<blocks, threads, 0, s>>>(ax, cs, dt, off, w32, w64); break;
    case 2: axis_table_kernel<2><<<blocks, threads, 0, s>>>(ax, cs, dt, off, w32, w64); break;
    case 3: axis_table_kernel<3><<<blocks, threads, 0, s>>>(ax, cs, dt, off, w32, w64); break;
    case 4: axis_table_kernel<4><<<blocks, threads, 0, s>>>(ax, cs, dt, off, w32, w64); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Per-(velocity, vertex) descriptors: physical departure point, folded into the domain, mapped
// back to reference coordinates (Newton on the analytic map, started at the physical point),
// then located in a cell.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void vertex_physical(const GeomArgs& g, int ix, int iy, double* x,
                                                double* y) {
  const double xi = vertex_ref_coord(ix, g.ax), eta = vertex_ref_coord(iy, g.ay);
  if (g.map.kind == 1) {
    sine_map(g.map.a, xi, eta, x, y);
  } else {
    *x = xi;
    *y = eta;
  }
}

__global__ void descriptor_kernel(const __grid_constant__ GeomArgs g, int* dcx, int* dcy, float* dr,
                                  float* ds, double* dr64, double* ds64) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int nq1 = g.cs.nq1;
  if (t >= (long long)nq1 * nq1 * g.nv) return;
  const int i = (int)(t / g.nv);
  const long long v = t % g.nv;
  const int ix = (int)(v % g.nx), iy = (int)(v / g.nx);
  double x, y;
  vertex_physical(g, ix, iy, &x, &y);
  const double xd = fold_axis(x - g.dt * g.cs.xi[i / nq1], g.ax);
  const double yd = fold_axis(y - g.dt * g.cs.xi[i % nq1], g.ay);
  double ex = xd, ey = yd;
  if (g.map.kind == 1) {
    bool conv = false;
    for (int it = 0; it < 100; ++it) {
      double fx, fy, j11, j12, j21, j22;
      sine_map(g.map.a, ex, ey, &fx, &fy);
      const double rx = fx - xd, ry = fy - yd;
      if (fabs(rx) < 1e-13 && fabs(ry) < 1e-13) {
        conv = true;
        break;
      }
      sine_map_jac(g.map.a, ex, ey, &j11, &j12, &j21, &j22);
      const double det = j11 * j22 - j12 * j21;
      ex -= (j22 * rx - j12 * ry) / det;
      ey -= (-j21 * rx + j11 * ry) / det;
    }
    if (!conv) atomicOr(g.flag, 2);
    ex = fold_axis(ex, g.ax);
    ey = fold_axis(ey, g.ay);
  }
  int cx, cy;
  double r, s;
  locate_axis(ex, g.ax, &cx, &r);
  locate_axis(ey, g.ay, &cy, &s);
  dcx[t] = cx;
  dcy[t] = cy;
  dr[t] = (float)r;
  ds[t] = (float)s;
  dr64[t] = r;
  ds64[t] = s;
}

cudaError_t launch_descriptors(const GeomArgs& g, int* dcx, int* dcy, float* dr, float* ds,
                               double* dr64, double* ds64, cudaStream_t s) {
  const long long n = (long long)g.cs.nq1 * g.cs.nq1 * g.nv;
  const int threads = 128;
  descriptor_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(g, dcx, dcy, dr, ds,
                                                                                dr64, ds64);
  return cudaGetLastError();
}

__global__ void vertex_coords_kernel(const __grid_constant__ GeomArgs g, double* x, double* y) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= g.nv) return;
  vertex_physical(g, (int)(v % g.nx), (int)(v / g.nx), x + v, y + v);
}

cudaError_t launch_vertex_coords(const GeomArgs& g, double* x, double* y, cudaStream_t s) {
  const int threads = 128;
  vertex_coords_kernel<<<(unsigned)((g.nv + threads - 1) / threads), threads, 0, s>>>(g, x, y);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Vertex quadrature weights A_v = sum over the cells containing v of the integral of its shape
// function times |det J|, by Gauss-Legendre quadrature (nodes/weights on [0,1] from the host).
// One thread per vertex: deterministic, no atomics.
// ------------------------------------------------------------------------------------------
struct GL {
  double x[8], w[8];
};

template <int P>
__global__ void vertex_weights_kernel(const __grid_constant__ GeomArgs g, GL gl, int ngl, double* A) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= g.nv) return;
  const int ix = (int)(v % g.nx), iy = (int)(v / g.nx);
  // cells touching the vertex along each axis, with the local node index of the vertex
  int cxs[2], axs[2], ncx = 0, cys[2], ays[2], ncy = 0;
  for (int side = 0; side < 2; ++side) {
    // x
    int c = (ix / P) - side, k = ix - c * P;
    if (side == 1 && ix % P != 0) c = -100;
    if (g.ax.periodic) {
      if (c == -1) { c = g.ax.n_cells - 1; k = P; }
    }
    if (c >= 0 && c < g.ax.n_cells && k >= 0 && k <= P) { cxs[ncx] = c; axs[ncx] = k; ++ncx; }
    // y
    c = (iy / P) - side;
    k = iy - c * P;
    if (side == 1 && iy % P != 0) c = -100;
    if (g.ay.periodic) {
      if (c == -1) { c = g.ay.n_cells - 1; k = P; }
    }
    if (c >= 0 && c < g.ay.n_cells && k >= 0 && k <= P) { cys[ncy] = c; ays[ncy] = k; ++ncy; }
  }
  if (g.map.kind != 1) {  // |det J| = 1: the integral factorises into two 1D integrals
    double sx = 0.0, sy = 0.0;
    for (int q = 0; q < ngl; ++q) {
      double px[P + 1], py[P + 1];
      lagrange_basis<P, double>(g.ax.nodes, gl.x[q], px);
      lagrange_basis<P, double>(g.ay.nodes, gl.x[q], py);
      for (int e = 0; e < ncx; ++e) sx += gl.w[q] * g.ax.hc * px[axs[e]];
      for (int e = 0; e < ncy; ++e) sy += gl.w[q] * g.ay.hc * py[ays[e]];
    }
    A[v] = sx * sy;
    return;
  }
  double acc = 0.0;
  for (int ey = 0; ey < ncy; ++ey)
    for (int ex = 0; ex < ncx; ++ex)
      for (int qy = 0; qy < ngl; ++qy)
        for (int qx = 0; qx < ngl; ++qx) {
          double px[P + 1], py[P + 1];
          lagrange_basis<P, double>(g.ax.nodes, gl.x[qx], px);
          lagrange_basis<P, double>(g.ay.nodes, gl.x[qy], py);
          double det = 1.0;
          if (g.map.kind == 1) {
            const double xi = g.ax.lo + g.ax.hc * (cxs[ex] + gl.x[qx]);
            const double eta = g.ay.lo + g.ay.hc * (cys[ey] + gl.x[qy]);
            double j11, j12, j21, j22;
            sine_map_jac(g.map.a, xi, eta, &j11, &j12, &j21, &j22);
            det = fabs(j11 * j22 - j12 * j21);
          }
          acc += gl.w[qx] * gl.w[qy] * det * g.ax.hc * g.ay.hc * px[axs[ex]] * py[ays[ey]];
        }
  A[v] = acc;
}

cudaError_t launch_vertex_weights(const GeomArgs& g, const double* gl_x, const double* gl_w, int ngl,
                                  double* A, cudaStream_t s) {
  GL gl;
  for (int k = 0; k < ngl && k < 8; ++k) {
    gl.x[k] = gl_x[k];
    gl.w[k] = gl_w[k];
  }
  const int threads = 128;
  const unsigned blocks = (unsigned)((g.nv + threads - 1) / threads);
  switch (g.ax.p) {
    case 1: vertex_weights_kernel<1><<<blocks, threads, 0, s>>>(g, gl, ngl, A); break;
    case 2: vertex_weights_kernel<2><<<blocks, threads, 0, s>>>(g, gl, ngl, A); break;
    case 3: vertex_weights_kernel<3><<<blocks, threads, 0, s>>>(g, gl, ngl, A); break;
    case 4: vertex_weights_kernel<4><<<blocks, threads, 0, s>>>(g, gl, ngl, A); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Initial state: f^eq(rho, u, theta), g^eq = K theta f^eq, stored as deviations (FP32/BF16) or
// full populations (FP64).
// ------------------------------------------------------------------------------------------
template <int Store>
__global__ void init_eq_kernel(const __grid_constant__ InitArgs a) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= a.nv) return;
  const int ix = (int)(v % a.nx), iy = (int)(v / a.nx);
  const double rho = a.rho[v], ux = a.u[v], uy = a.v[v], theta = a.T[v];
  const double q = theta - 1.0;
  EqFactors<double> e;
  eq_factors<double>(a.cs.he, ux, uy, q, e);
  const size_t o = (size_t)iy * a.pitch + (size_t)ix * a.xs;
  const int nq1 = a.cs.nq1;
  for (int ia = 0; ia < nq1; ++ia)
    for (int ib = 0; ib < nq1; ++ib) {
      const int i = nq1 * ia + ib;
      const double w = a.cs.w[ia] * a.cs.w[ib];
      const double em1 = eq_em1<double>(e, ia, ib);
      const double devf = (rho - 1.0) + rho * em1;          // f^eq / w - 1
      const double devg = devf + q * (1.0 + devf);          // g^eq / (K w) - 1
      const size_t of = (size_t)i * a.plane_stride + o, og = of + a.ps;
      if (Store == kStoreF64) {
        double* d = static_cast<double*>(a.dst);
        d[of] = w * (1.0 + devf);
        if (a.cp.npop == 2) d[og] = a.cp.K * w * (1.0 + devg);
      } else if (Store == kStoreF32) {
        float* d = static_cast<float*>(a.dst);
        d[of] = (float)(w * devf);
        if (a.cp.npop == 2) d[og] = (float)(a.cp.K * w * devg);
      } else {
        __nv_bfloat16* d = static_cast<__nv_bfloat16*>(a.dst);
        d[of] = __float2bfloat16_rn((float)(w * devf));
        if (a.cp.npop == 2) d[og] = __float2bfloat16_rn((float)(a.cp.K * w * devg));
      }
    }
}

cudaError_t launch_init_equilibrium(const InitArgs& a, cudaStream_t s) {
  const int threads = 128;
  const unsigned blocks = (unsigned)((a.nv + threads - 1) / threads);
  switch (a.store) {
    case kStoreF32: init_eq_kernel<kStoreF32><<<blocks, threads, 0, s>>>(a); break;
    case kStoreBF16: init_eq_kernel<kStoreBF16><<<blocks, threads, 0, s>>>(a); break;
    case kStoreF64: init_eq_kernel<kStoreF64><<<blocks, threads, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Ghost cells: rows [ylo, 0) and [ny, yhi) over all kept columns, and columns [xlo, 0), [nx, xhi)
// of the interior rows, copied from their periodic (or clamped) source vertex.
// ------------------------------------------------------------------------------------------
template <typename E>
__global__ void ghost_fill_kernel(E* origin, size_t plane_stride, int pitch, int planes, GhostK g) {
  const long long W = g.xhi - g.xlo, topb = -g.ylo + (g.yhi - g.ny), side = -g.xlo + (g.xhi - g.nx);
  const long long per_plane = topb * W + (long long)g.ny * side;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per_plane * planes) return;
  const int plane = (int)(t / per_plane);
  long long e = t - (long long)plane * per_plane;
  int xx, yy;
  if (e < topb * W) {
    const int r = (int)(e / W), c = (int)(e - (long long)r * W);
    yy = r < -g.ylo ? g.ylo + r : g.ny + (r + g.ylo);
    xx = g.xlo + c;
  } else {
    e -= topb * W;
    const int r = (int)(e / side), c = (int)(e - (long long)r * side);
    yy = r;
    xx = c < -g.xlo ? g.xlo + c : g.nx + (c + g.xlo);
  }
  int sx = xx, sy = yy;
  if (g.px) {
    sx %= g.nx;
    if (sx < 0) sx += g.nx;
  } else {
    sx = sx < 0 ? 0 : (sx >= g.nx ? g.nx - 1 : sx);
  }
  if (g.py) {
    sy %= g.ny;
    if (sy < 0) sy += g.ny;
  } else {
    sy = sy < 0 ? 0 : (sy >= g.ny ? g.ny - 1 : sy);
  }
  E* pl = origin + (ptrdiff_t)plane * plane_stride;
  pl[(ptrdiff_t)yy * pitch + xx] = pl[(ptrdiff_t)sy * pitch + sx];
}

cudaError_t launch_ghost_fill(void* origin, int elem, size_t plane_stride, int pitch, int planes,
                              const GhostK& g, cudaStream_t s) {
  const long long W = g.xhi - g.xlo, topb = -g.ylo + (g.yhi - g.ny), side = -g.xlo + (g.xhi - g.nx);
  const long long n = (topb * W + (long long)g.ny * side) * planes;
  if (n == 0) return cudaSuccess;
  const int threads = 256;
  const unsigned blocks = (unsigned)((n + threads - 1) / threads);
  switch (elem) {
    case 2: ghost_fill_kernel<uint16_t><<<blocks, threads, 0, s>>>(static_cast<uint16_t*>(origin), plane_stride, pitch, planes, g); break;
    case 4: ghost_fill_kernel<uint32_t><<<blocks, threads, 0, s>>>(static_cast<uint32_t*>(origin), plane_stride, pitch, planes, g); break;
    case 8: ghost_fill_kernel<uint64_t><<<blocks, threads, 0, s>>>(static_cast<uint64_t*>(origin), plane_stride, pitch, planes, g); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Dense [npop][nq][ny][nx] <-> internal layout (ghost cells, row pitch, interleaved pairs).
// ------------------------------------------------------------------------------------------
template <typename E>
__global__ void state_convert_kernel(const E* src, E* dst, int to_internal, int plane0, int nplanes,
                                     int nq, int nx, int ny, int pitch, size_t plane_stride, int xs,
                                     ptrdiff_t ps) {
  const long long nv = (long long)nx * ny;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t0 >= (long long)nplanes * nv) return;
  const long long t = t0 + (long long)plane0 * nv;   // index in the dense layout
  const long long pl = t / nv, v = t - pl * nv;
  const int pop = (int)(pl / nq), i = (int)(pl - (long long)pop * nq);
  const int x = (int)(v % nx), y = (int)(v / nx);
  const ptrdiff_t o = (ptrdiff_t)i * plane_stride + pop * ps + (ptrdiff_t)y * pitch + (ptrdiff_t)x * xs;
  if (to_internal)
    dst[o] = src[t];
  else
    dst[t] = src[o];
}

// Dense [npop][nq][ny][nx] <-> interleaved (f, g) pairs (xs = 2, ps = 1) for the velocity planes
// i0 .. i0 + gridDim.z - 1: one thread per (plane, vertex), f and g together, so that a pair moves
// as one 8-byte (FP32) or 4-byte (BF16) access (g = 0 with one population).
template <typename E, typename E2>
__global__ void pair_convert_kernel(const E* src, E* dst, int to_internal, int i0, int npop, int nq, int nx,
                                    int ny, int pitch, size_t plane_stride) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, i = i0 + blockIdx.z;
  if (x >= nx) return;
  const size_t nv = (size_t)nx * ny;
  const size_t d = ((size_t)i * ny + y) * nx + x;                            // f in the dense layout
  const size_t o = (size_t)i * plane_stride + (size_t)y * pitch + 2 * (size_t)x;   // the pair
  if (to_internal) {
    E2 p;
    p.x = src[d];
    p.y = npop == 2 ? src[(size_t)nq * nv + d] : E(0);
    *reinterpret_cast<E2*>(dst + o) = p;
  } else {
    const E2 p = *reinterpret_cast<const E2*>(src + o);
    dst[d] = p.x;
    if (npop == 2) dst[(size_t)nq * nv + d] = p.y;
  }
}

cudaError_t launch_pair_convert(const void* src, void* dst, bool to_internal, int elem, int i0, int ni, int npop,
                                int nq, int nx, int ny, int pitch, size_t plane_stride, cudaStream_t s) {
  if (ni == 0) return cudaSuccess;
  if (ny > 65535 || ni > 65535) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)((nx + 255) / 256), (unsigned)ny, (unsigned)ni);
  const int ti = to_internal ? 1 : 0;
  if (elem == 4)
    pair_convert_kernel<uint32_t, uint2><<<grid, 256, 0, s>>>(static_cast<const uint32_t*>(src),
        static_cast<uint32_t*>(dst), ti, i0, npop, nq, nx, ny, pitch, plane_stride);
  else if (elem == 2)
    pair_convert_kernel<uint16_t, ushort2><<<grid, 256, 0, s>>>(static_cast<const uint16_t*>(src),
        static_cast<uint16_t*>(dst), ti, i0, npop, nq, nx, ny, pitch, plane_stride);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_state_convert(const void* src, void* dst, bool to_internal, int elem, int plane0,
                                 int nplanes, int nq, int nx, int ny, int pitch, size_t plane_stride,
                                 int xs, ptrdiff_t ps, cudaStream_t s) {
  const long long n = (long long)nplanes * nx * ny;
  if (n == 0) return cudaSuccess;
  const int threads = 256;
  const unsigned blocks = (unsigned)((n + threads - 1) / threads);
  const int ti = to_internal ? 1 : 0;
  switch (elem) {
    case 2:
      state_convert_kernel<uint16_t><<<blocks, threads, 0, s>>>(static_cast<const uint16_t*>(src),
          static_cast<uint16_t*>(dst), ti, plane0, nplanes, nq, nx, ny, pitch, plane_stride, xs, ps);
      break;
    case 4:
      state_convert_kernel<uint32_t><<<blocks, threads, 0, s>>>(static_cast<const uint32_t*>(src),
          static_cast<uint32_t*>(dst), ti, plane0, nplanes, nq, nx, ny, pitch, plane_stride, xs, ps);
      break;
    case 8:
      state_convert_kernel<uint64_t><<<blocks, threads, 0, s>>>(static_cast<const uint64_t*>(src),
          static_cast<uint64_t*>(dst), ti, plane0, nplanes, nq, nx, ny, pitch, plane_stride, xs, ps);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace sllbm
